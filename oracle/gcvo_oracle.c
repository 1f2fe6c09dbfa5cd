/*
 * gcvo_oracle.c -- FP64 CPU oracle for the G-CVO objective and derivatives.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, brute-force
 * restatement of the paper's method that the CUDA path is checked against.
 * It shares no code, header or constant with the CUDA library; only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark load it.
 *
 * Everything is double precision and every pair (i, j) of the N_X * N_Z
 * pairs is visited (no spatial structure).  Loops over source points are
 * split across OpenMP threads; each source point's contribution is stored
 * separately and the final sums are taken in index order, so results do not
 * depend on the thread count.
 *
 * Notation follows Sec. 2-3 of the paper: target X = {x_i}, source Z = {z_j},
 * pose T = (R, t) with T x = R x + t, p_j = T^{-1} z_j = R^T (z_j - t),
 * r_ij = x_i - p_j.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------- */
/* Small dense helpers (row-major 3x3).                                    */
/* ---------------------------------------------------------------------- */

static void sym6_to_mat(const double *s, double A[9]) {
    /* s = (xx, xy, xz, yy, yz, zz) */
    A[0] = s[0]; A[1] = s[1]; A[2] = s[2];
    A[3] = s[1]; A[4] = s[3]; A[5] = s[4];
    A[6] = s[2]; A[7] = s[4]; A[8] = s[5];
}

/* Inverse of a 3x3 matrix by Gauss-Jordan elimination with partial
 * pivoting (an LU-type factorisation, deliberately not the adjugate).
 * Returns 0 on success, -1 if a pivot is exactly zero. */
static int inv3_lu(const double A_in[9], double Ainv[9]) {
    double a[3][6];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) a[r][c] = A_in[3 * r + c];
        for (int c = 0; c < 3; ++c) a[r][3 + c] = (r == c) ? 1.0 : 0.0;
    }
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int c = 0; c < 6; ++c) { double t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t; }
        double d = a[col][col];
        for (int c = 0; c < 6; ++c) a[col][c] /= d;
        for (int r = 0; r < 3; ++r) {
            if (r == col) continue;
            double m = a[r][col];
            for (int c = 0; c < 6; ++c) a[r][c] -= m * a[col][c];
        }
    }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Ainv[3 * r + c] = a[r][3 + c];
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Per-point covariance, Eq. (7b): Sigma(x; X) = 1/(n-1) sum_{y in N_n(x)}  */
/* (y - x)(y - x)^T, with N_n(x) the n nearest points of the cloud around   */
/* x.  Reading taken: the query point is its own nearest neighbour, so the  */
/* n points are x itself plus its n-1 nearest others; ties in distance are  */
/* broken by the smaller index.  Brute force, O(N^2).                       */
/* ---------------------------------------------------------------------- */

int orc_knn_cov(const double *xyz, int64_t n, int knn, double *cov_out, int64_t *nbr_out,
                double *kth_d2_out) {
    if (knn < 2 || knn > 64 || n < knn) return -1;
    int fail = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double best_d[65];
        int64_t best_i[65];
        int cnt = 0;
        const double *x = xyz + 3 * i;
        for (int64_t k = 0; k < n; ++k) {
            const double *y = xyz + 3 * k;
            double dx = y[0] - x[0], dy = y[1] - x[1], dz = y[2] - x[2];
            double d2 = dx * dx + dy * dy + dz * dz;
            /* keep the knn+1 best (the extra one reports the gap to the next) */
            int pos = cnt;
            while (pos > 0 && (best_d[pos - 1] > d2 || (best_d[pos - 1] == d2 && best_i[pos - 1] > k))) --pos;
            if (pos >= knn + 1) continue;
            int last = cnt < knn + 1 ? cnt : knn;
            for (int q = last; q > pos; --q) { best_d[q] = best_d[q - 1]; best_i[q] = best_i[q - 1]; }
            best_d[pos] = d2;
            best_i[pos] = k;
            if (cnt < knn + 1) ++cnt;
        }
        double S[6] = {0, 0, 0, 0, 0, 0};
        for (int q = 0; q < knn; ++q) {
            const double *y = xyz + 3 * best_i[q];
            double d[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
            S[0] += d[0] * d[0]; S[1] += d[0] * d[1]; S[2] += d[0] * d[2];
            S[3] += d[1] * d[1]; S[4] += d[1] * d[2]; S[5] += d[2] * d[2];
        }
        for (int q = 0; q < 6; ++q) cov_out[6 * i + q] = S[q] / (double)(knn - 1);
        if (nbr_out)
            for (int q = 0; q < knn; ++q) nbr_out[(int64_t)knn * i + q] = best_i[q];
        if (kth_d2_out) {
            kth_d2_out[2 * i] = best_d[knn - 1];
            kth_d2_out[2 * i + 1] = cnt > knn ? best_d[knn] : INFINITY;
        }
    }
    return fail;
}

/* ---------------------------------------------------------------------- */
/* Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations.            */
/* evecs columns are the eigenvectors (row-major, evecs[3*r + c]).          */
/* ---------------------------------------------------------------------- */

void orc_sym3_eig(const double s[6], double evals[3], double evecs[9]) {
    double a[3][3];
    double A[9];
    sym6_to_mat(s, A);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) a[r][c] = A[3 * r + c];
    double v[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        double scale = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2] + 2 * off;
        if (off <= 1e-36 * scale || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                /* rotation that annihilates a[p][q] (Golub & Van Loan, Alg. 8.4.2) */
                double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < 3; ++k) {
                    double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - sn * akq;
                    a[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - sn * aqk;
                    a[q][k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    double vkp = v[k][p], vkq = v[k][q];
                    v[k][p] = c * vkp - sn * vkq;
                    v[k][q] = sn * vkp + c * vkq;
                }
            }
    }
    for (int k = 0; k < 3; ++k) evals[k] = a[k][k];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) evecs[3 * r + c] = v[r][c];
}

/* Remark after Eq. (7): bound the eigenvalues of each per-point covariance.
 * Reading taken: clamp every eigenvalue into [eig_max / eig_ratio, eig_max]
 * and rebuild Sigma = V diag(lambda') V^T.  eig_max <= 0 disables. */
void orc_eig_clamp(double *cov, int64_t n, double eig_max, double eig_ratio) {
    if (eig_max <= 0) return;
    double lo = eig_max / eig_ratio;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double lam[3], V[9];
        orc_sym3_eig(cov + 6 * i, lam, V);
        for (int k = 0; k < 3; ++k) lam[k] = lam[k] < lo ? lo : (lam[k] > eig_max ? eig_max : lam[k]);
        double S[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double s = 0;
                for (int k = 0; k < 3; ++k) s += V[3 * r + k] * lam[k] * V[3 * c + k];
                S[3 * r + c] = s;
            }
        double *o = cov + 6 * i;
        o[0] = S[0]; o[1] = 0.5 * (S[1] + S[3]); o[2] = 0.5 * (S[2] + S[6]);
        o[3] = S[4]; o[4] = 0.5 * (S[5] + S[7]); o[5] = S[8];
    }
}

/* ---------------------------------------------------------------------- */
/* The objective, gradient and Gauss-Newton matrix at a pose.              */
/* ---------------------------------------------------------------------- */

typedef struct {
    int kernel_mode;   /* 0: anisotropic kernel, Eq. (7); 1: isotropic (Sigma_ij = ell^2 I) */
    double sigma2;     /* kernel amplitude sigma^2 of Eq. (7a) */
    double cutoff;     /* keep a pair only if d^2 <= cutoff^2; <= 0 keeps every pair */
    double iso_ell;    /* isotropic length scale ell */
    int feat_dim;      /* l: c_ij = <l_i, l_j> over l channels */
    double rho;        /* count pairs with |r| <= rho (reported only) */
} orc_params;

typedef struct {
    double f;          /* Eq. (5) */
    double g[6];       /* (g_omega, g_v), Lemma 1 / Eq. (8) */
    double M[36];      /* sum_ij f_ij J_j^T Sigma_ij^{-1} J_j, Eq. (11) */
    double gabs[6];    /* sum_ij |g^(ij)| per component (scale for tolerances) */
    double n_pairs_kept;   /* pairs passing the cutoff */
    double n_pairs_rho;    /* pairs with |r_ij| <= rho */
    double n_near_cut;     /* pairs with |d^2 - cutoff^2| < 1e-4 * cutoff^2 */
    /* The terms those near-cutoff pairs have at their own d^2, kept or not:
     * the cutoff test d^2 <= c^2 of Eq. (7) decides them, and a computation
     * in lower precision may decide them the other way; f_near and
     * g_near[a] (sum of |g^(ij)_a|) bound the difference that makes. */
    double f_near;
    double g_near[6];
} orc_eval_out;

/* Per-source-point contribution (summed over all targets i). */
typedef struct {
    double f, g[6], M[36], gabs[6], kept, nrho, near, fnear, gnear[6];
} orc_partial;

static void pair_terms(const double *x, const double *covx, const double *lx, const double *p,
                       const double *Sz_rot /* R^T Sigma_z R, 3x3 */, const double *lz,
                       const orc_params *P, orc_partial *acc) {
    double r[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
    double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    if (P->rho > 0 && rr <= P->rho * P->rho) acc->nrho += 1;
    double Sig[9];
    if (P->kernel_mode == 1) {
        for (int q = 0; q < 9; ++q) Sig[q] = 0;
        Sig[0] = Sig[4] = Sig[8] = P->iso_ell * P->iso_ell;
    } else {
        /* Eq. (7c): Sigma_ij = Sigma(x_i; X) + R^T Sigma(z_j; Z) R */
        double Sx[9];
        sym6_to_mat(covx, Sx);
        for (int q = 0; q < 9; ++q) Sig[q] = Sx[q] + Sz_rot[q];
    }
    double Ainv[9];
    if (inv3_lu(Sig, Ainv) != 0) return;
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = Ainv[3 * a + 0] * r[0] + Ainv[3 * a + 1] * r[1] + Ainv[3 * a + 2] * r[2];
    double d2 = r[0] * u[0] + r[1] * u[1] + r[2] * u[2];
    const double c2 = P->cutoff * P->cutoff;
    const int near = P->cutoff > 0 && fabs(d2 - c2) < 1e-4 * c2;
    const int cut = P->cutoff > 0 && d2 > c2;
    if (cut && !near) return;
    /* Eq. (5), (7a): f_ij = c_ij k(x_i, p_j), c_ij = <l_i^X, l_j^Z> */
    double cij = 0;
    for (int q = 0; q < P->feat_dim; ++q) cij += lx[q] * lz[q];
    double fij = cij * P->sigma2 * exp(-0.5 * d2);
    /* Lemma 1: g_v = -sum f_ij Sigma^-1 r, g_omega = -sum f_ij p^ Sigma^-1 r */
    double pxu[3] = {p[1] * u[2] - p[2] * u[1], p[2] * u[0] - p[0] * u[2], p[0] * u[1] - p[1] * u[0]};
    if (near) {
        acc->near += 1;
        acc->fnear += fabs(fij);
        for (int a = 0; a < 3; ++a) {
            acc->gnear[a] += fabs(fij * pxu[a]);
            acc->gnear[3 + a] += fabs(fij * u[a]);
        }
    }
    if (cut) return;
    acc->kept += 1;
    acc->f += fij;
    for (int a = 0; a < 3; ++a) {
        acc->g[a] -= fij * pxu[a];
        acc->g[3 + a] -= fij * u[a];
        acc->gabs[a] += fabs(fij * pxu[a]);
        acc->gabs[3 + a] += fabs(fij * u[a]);
    }
    /* Eq. (10): J_j = [ -p_j^ , I ] (3 x 6); M += f_ij J^T Sigma^-1 J */
    double J[18];
    double ph[9] = {0, -p[2], p[1], p[2], 0, -p[0], -p[1], p[0], 0};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            J[6 * a + b] = -ph[3 * a + b];
            J[6 * a + 3 + b] = (a == b) ? 1.0 : 0.0;
        }
    double AJ[18];
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 6; ++c) {
            double s = 0;
            for (int b = 0; b < 3; ++b) s += Ainv[3 * a + b] * J[6 * b + c];
            AJ[6 * a + c] = s;
        }
    for (int a = 0; a < 6; ++a)
        for (int c = 0; c < 6; ++c) {
            double s = 0;
            for (int b = 0; b < 3; ++b) s += J[6 * b + a] * AJ[6 * b + c];
            acc->M[6 * a + c] += fij * s;
        }
}

/* T: 4x4 row-major.  tgt/src: n x 3, cov: n x 6 (xx,xy,xz,yy,yz,zz), feat:
 * n x feat_dim.  per_src (optional): n_src partials of (f, g[6]) for
 * sampled-output checks. */
int orc_eval(const double *tgt, const double *tgt_cov, const double *tgt_feat, int64_t n_tgt,
             const double *src, const double *src_cov, const double *src_feat, int64_t n_src,
             const double *T, const orc_params *P, orc_eval_out *out, double *per_src) {
    double R[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
    double t[3] = {T[3], T[7], T[11]};
    orc_partial *part = (orc_partial *)calloc((size_t)(n_src > 0 ? n_src : 1), sizeof(orc_partial));
    if (!part) return -2;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t j = 0; j < n_src; ++j) {
        const double *z = src + 3 * j;
        /* Alg. 1: transform Z with T^{-1}: p_j = R^T (z_j - t) */
        double dz[3] = {z[0] - t[0], z[1] - t[1], z[2] - t[2]};
        double p[3];
        for (int a = 0; a < 3; ++a) p[a] = R[0 + a] * dz[0] + R[3 + a] * dz[1] + R[6 + a] * dz[2];
        double Szr[9];
        if (P->kernel_mode == 0) {
            double Sz[9], SR[9];
            sym6_to_mat(src_cov + 6 * j, Sz);
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) {
                    double s = 0;
                    for (int b = 0; b < 3; ++b) s += Sz[3 * a + b] * R[3 * b + c];
                    SR[3 * a + c] = s;
                }
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) {
                    double s = 0;
                    for (int b = 0; b < 3; ++b) s += R[3 * b + a] * SR[3 * b + c];
                    Szr[3 * a + c] = s;
                }
        }
        orc_partial acc;
        memset(&acc, 0, sizeof(acc));
        for (int64_t i = 0; i < n_tgt; ++i)
            pair_terms(tgt + 3 * i, tgt_cov ? tgt_cov + 6 * i : NULL, tgt_feat + (int64_t)P->feat_dim * i, p,
                       Szr, src_feat + (int64_t)P->feat_dim * j, P, &acc);
        part[j] = acc;
    }
    memset(out, 0, sizeof(*out));
    for (int64_t j = 0; j < n_src; ++j) {
        out->f += part[j].f;
        for (int a = 0; a < 6; ++a) { out->g[a] += part[j].g[a]; out->gabs[a] += part[j].gabs[a]; }
        for (int a = 0; a < 36; ++a) out->M[a] += part[j].M[a];
        out->n_pairs_kept += part[j].kept;
        out->n_pairs_rho += part[j].nrho;
        out->n_near_cut += part[j].near;
        out->f_near += part[j].fnear;
        for (int a = 0; a < 6; ++a) out->g_near[a] += part[j].gnear[a];
        if (per_src) {
            per_src[7 * j] = part[j].f;
            for (int a = 0; a < 6; ++a) per_src[7 * j + 1 + a] = part[j].g[a];
        }
    }
    free(part);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* G-CVO-1 line search (Eq. 9, Appendix B).  Along G(t) = f(T exp(t xi^))  */
/* with Sigma_ij frozen, each pair's exponent -1/2 r(t)^T A r(t) is a power */
/* series in t.  With a_1 = omega^ p + v and a_k = omega^ a_{k-1} (the      */
/* homogeneous powers (xi^)^k p), exp(-t xi^) p = p - t a_1 + t^2/2 a_2 -   */
/* t^3/6 a_3 + t^4/24 a_4 - ..., so r(t) = r + t a_1 - t^2/2 a_2 + t^3/6 a_3 */
/* - t^4/24 a_4.  Expanding the quadratic form to t^4 gives the exponent    */
/* coefficients (beta, gamma, delta, eps); the g^k of Appendix B are the    */
/* Taylor coefficients of exp(beta t + gamma t^2 + delta t^3 + eps t^4).    */
/* Reading taken: Appendix B's printed gamma, delta and eps match the       */
/* expansion of r + sum_k t^k a_k instead (no factorials or signs); the    */
/* exact expansion above is used, the printed one is mode literal = 1.      */
/* out[0..4] = sum_ij f_ij g^k_ij, k = 0..4.                                */
/* ---------------------------------------------------------------------- */

int orc_linesearch_coeffs(const double *tgt, const double *tgt_cov, const double *tgt_feat, int64_t n_tgt,
                          const double *src, const double *src_cov, const double *src_feat, int64_t n_src,
                          const double *T, const double *xi, const orc_params *P, int literal,
                          double out[5]) {
    double R[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
    double t[3] = {T[3], T[7], T[11]};
    double *part = (double *)calloc((size_t)(n_src > 0 ? n_src : 1) * 5, sizeof(double));
    if (!part) return -2;
    const double *w = xi, *v = xi + 3;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t j = 0; j < n_src; ++j) {
        const double *z = src + 3 * j;
        double dz[3] = {z[0] - t[0], z[1] - t[1], z[2] - t[2]};
        double p[3];
        for (int a = 0; a < 3; ++a) p[a] = R[0 + a] * dz[0] + R[3 + a] * dz[1] + R[6 + a] * dz[2];
        double Szr[9] = {0};
        if (P->kernel_mode == 0) {
            double Sz[9], SR[9];
            sym6_to_mat(src_cov + 6 * j, Sz);
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) {
                    double s = 0;
                    for (int b = 0; b < 3; ++b) s += Sz[3 * a + b] * R[3 * b + c];
                    SR[3 * a + c] = s;
                }
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) {
                    double s = 0;
                    for (int b = 0; b < 3; ++b) s += R[3 * b + a] * SR[3 * b + c];
                    Szr[3 * a + c] = s;
                }
        }
        double ak[5][3];
        /* a_1 = omega x p + v, a_k = omega x a_{k-1} */
        ak[1][0] = w[1] * p[2] - w[2] * p[1] + v[0];
        ak[1][1] = w[2] * p[0] - w[0] * p[2] + v[1];
        ak[1][2] = w[0] * p[1] - w[1] * p[0] + v[2];
        for (int k = 2; k <= 4; ++k) {
            ak[k][0] = w[1] * ak[k - 1][2] - w[2] * ak[k - 1][1];
            ak[k][1] = w[2] * ak[k - 1][0] - w[0] * ak[k - 1][2];
            ak[k][2] = w[0] * ak[k - 1][1] - w[1] * ak[k - 1][0];
        }
        double acc[5] = {0, 0, 0, 0, 0};
        for (int64_t i = 0; i < n_tgt; ++i) {
            const double *x = tgt + 3 * i;
            double r[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
            double Sig[9];
            if (P->kernel_mode == 1) {
                for (int q = 0; q < 9; ++q) Sig[q] = 0;
                Sig[0] = Sig[4] = Sig[8] = P->iso_ell * P->iso_ell;
            } else {
                double Sx[9];
                sym6_to_mat(tgt_cov + 6 * i, Sx);
                for (int q = 0; q < 9; ++q) Sig[q] = Sx[q] + Szr[q];
            }
            double A[9];
            if (inv3_lu(Sig, A) != 0) continue;
            double Ar[3];
            for (int a = 0; a < 3; ++a) Ar[a] = A[3 * a] * r[0] + A[3 * a + 1] * r[1] + A[3 * a + 2] * r[2];
            double d2 = r[0] * Ar[0] + r[1] * Ar[1] + r[2] * Ar[2];
            if (P->cutoff > 0 && d2 > P->cutoff * P->cutoff) continue;
            double cij = 0;
            for (int q = 0; q < P->feat_dim; ++q) cij += tgt_feat[(int64_t)P->feat_dim * i + q] * src_feat[(int64_t)P->feat_dim * j + q];
            double fij = cij * P->sigma2 * exp(-0.5 * d2);
            /* bilinear forms <a_k, A a_m> and <a_k, A r> */
            double Aa[5][3];
            for (int k = 1; k <= 4; ++k)
                for (int a = 0; a < 3; ++a)
                    Aa[k][a] = A[3 * a] * ak[k][0] + A[3 * a + 1] * ak[k][1] + A[3 * a + 2] * ak[k][2];
#define DOT(u, q) ((u)[0] * (q)[0] + (u)[1] * (q)[1] + (u)[2] * (q)[2])
            double kr[5], a11 = DOT(ak[1], Aa[1]), a12 = DOT(ak[1], Aa[2]), a13 = DOT(ak[1], Aa[3]),
                          a22 = DOT(ak[2], Aa[2]);
            for (int k = 1; k <= 4; ++k) kr[k] = DOT(ak[k], Ar);
#undef DOT
            double be, ga, de, ep;
            if (!literal) {
                be = -kr[1];
                ga = 0.5 * kr[2] - 0.5 * a11;
                de = -kr[3] / 6.0 + 0.5 * a12;
                ep = kr[4] / 24.0 - a13 / 6.0 - a22 / 8.0;
            } else {
                be = -kr[1];
                ga = -0.5 * a11 - kr[2];
                de = -a12 - kr[3];
                ep = -0.5 * (a22 + 2.0 * a13 + 2.0 * kr[4]);
            }
            double g1 = be, g2 = ga + 0.5 * be * be, g3 = de + be * ga + be * be * be / 6.0,
                   g4 = ep + be * de + 0.5 * be * be * ga + 0.5 * ga * ga + be * be * be * be / 24.0;
            acc[0] += fij;
            acc[1] += fij * g1;
            acc[2] += fij * g2;
            acc[3] += fij * g3;
            acc[4] += fij * g4;
        }
        for (int k = 0; k < 5; ++k) part[5 * j + k] = acc[k];
    }
    for (int k = 0; k < 5; ++k) out[k] = 0;
    for (int64_t j = 0; j < n_src; ++j)
        for (int k = 0; k < 5; ++k) out[k] += part[5 * j + k];
    free(part);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* G-CVO-E (Sec. 3.4): the directional derivative D(g)[xi] of Lemma 1's    */
/* gradient under the right perturbation T exp(xi^), all four terms of the  */
/* product rule kept.  For xi = e_k (k = 0..5, omega first) and each pair:  */
/*   dp = -(omega x p + v),  dr = -dp,                                      */
/*   dSigma' = Sigma' omega^ - omega^ Sigma',  dA = -A dSigma' A,           */
/*   dw = -w (y . dr + r . dA r / 2),  y = A r,  A = Sigma_ij^-1,           */
/*   column k of D -= dw J^T y + w (dp x y, 0) + w J^T dA r + w J^T A dr,   */
/* with J^T a = (p x a, a).  The last term alone is -M.  Pairs beyond the   */
/* cutoff contribute nothing.  D_out: 6x6 row-major, D_out[6 r + k] is      */
/* component r of D(g)[e_k].  Same inputs as orc_eval.                      */
/* ---------------------------------------------------------------------- */

static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static void mat3_mul(const double A[9], const double B[9], double C[9]) {
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int b = 0; b < 3; ++b) s += A[3 * a + b] * B[3 * b + c];
            C[3 * a + c] = s;
        }
}

static void mat3_vec(const double A[9], const double x[3], double y[3]) {
    for (int a = 0; a < 3; ++a) y[a] = A[3 * a] * x[0] + A[3 * a + 1] * x[1] + A[3 * a + 2] * x[2];
}

int orc_grad_derivative(const double *tgt, const double *tgt_cov, const double *tgt_feat, int64_t n_tgt,
                        const double *src, const double *src_cov, const double *src_feat, int64_t n_src,
                        const double *T, const orc_params *P, double *D_out) {
    double R[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
    double t[3] = {T[3], T[7], T[11]};
    double *part = (double *)calloc((size_t)(n_src > 0 ? n_src : 1) * 36, sizeof(double));
    if (!part) return -2;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t j = 0; j < n_src; ++j) {
        const double *z = src + 3 * j;
        double dz[3] = {z[0] - t[0], z[1] - t[1], z[2] - t[2]};
        double p[3];
        for (int a = 0; a < 3; ++a) p[a] = R[0 + a] * dz[0] + R[3 + a] * dz[1] + R[6 + a] * dz[2];
        /* Sigma'_j = R^T Sigma(z_j; Z) R (zero for the isotropic kernel) */
        double Szr[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (P->kernel_mode == 0) {
            double Sz[9], SR[9], Rt[9];
            sym6_to_mat(src_cov + 6 * j, Sz);
            mat3_mul(Sz, R, SR);
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) Rt[3 * a + c] = R[3 * c + a];
            mat3_mul(Rt, SR, Szr);
        }
        double *Dj = part + 36 * j;
        const double *lz = src_feat + (int64_t)P->feat_dim * j;
        for (int64_t i = 0; i < n_tgt; ++i) {
            const double *x = tgt + 3 * i;
            double r[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
            double Sig[9];
            if (P->kernel_mode == 1) {
                for (int q = 0; q < 9; ++q) Sig[q] = 0;
                Sig[0] = Sig[4] = Sig[8] = P->iso_ell * P->iso_ell;
            } else {
                double Sx[9];
                sym6_to_mat(tgt_cov + 6 * i, Sx);
                for (int q = 0; q < 9; ++q) Sig[q] = Sx[q] + Szr[q];
            }
            double A[9];
            if (inv3_lu(Sig, A) != 0) continue;
            double y[3];
            mat3_vec(A, r, y);
            double d2 = r[0] * y[0] + r[1] * y[1] + r[2] * y[2];
            if (P->cutoff > 0 && d2 > P->cutoff * P->cutoff) continue;
            double cij = 0;
            const double *lx = tgt_feat + (int64_t)P->feat_dim * i;
            for (int q = 0; q < P->feat_dim; ++q) cij += lx[q] * lz[q];
            double w = cij * P->sigma2 * exp(-0.5 * d2);
            double pxy[3];
            cross3(p, y, pxy);
            for (int k = 0; k < 6; ++k) {
                double om[3] = {0, 0, 0}, v[3] = {0, 0, 0};
                if (k < 3) om[k] = 1.0; else v[k - 3] = 1.0;
                double oxp[3], dp[3], dr[3];
                cross3(om, p, oxp);
                for (int a = 0; a < 3; ++a) {
                    dp[a] = -(oxp[a] + v[a]);
                    dr[a] = -dp[a];
                }
                /* dSigma' = Sigma' W - W Sigma', W = omega^ */
                double W[9] = {0, -om[2], om[1], om[2], 0, -om[0], -om[1], om[0], 0};
                double SW[9], WS[9], dS[9], AdS[9], dA[9];
                mat3_mul(Szr, W, SW);
                mat3_mul(W, Szr, WS);
                for (int q = 0; q < 9; ++q) dS[q] = SW[q] - WS[q];
                mat3_mul(A, dS, AdS);
                mat3_mul(AdS, A, dA);
                for (int q = 0; q < 9; ++q) dA[q] = -dA[q];
                double dAr[3], Adr[3];
                mat3_vec(dA, r, dAr);
                mat3_vec(A, dr, Adr);
                double ydr = y[0] * dr[0] + y[1] * dr[1] + y[2] * dr[2];
                double rdAr = r[0] * dAr[0] + r[1] * dAr[1] + r[2] * dAr[2];
                double dw = -w * (ydr + 0.5 * rdAr);
                double dpxy[3], pxdAr[3], pxAdr[3];
                cross3(dp, y, dpxy);
                cross3(p, dAr, pxdAr);
                cross3(p, Adr, pxAdr);
                for (int a = 0; a < 3; ++a) {
                    /* rotation rows: (p x .) parts; translation rows: the vectors */
                    Dj[6 * a + k] -= dw * pxy[a] + w * dpxy[a] + w * pxdAr[a] + w * pxAdr[a];
                    Dj[6 * (3 + a) + k] -= dw * y[a] + w * dAr[a] + w * Adr[a];
                }
            }
        }
    }
    for (int q = 0; q < 36; ++q) D_out[q] = 0;
    for (int64_t j = 0; j < n_src; ++j)
        for (int q = 0; q < 36; ++q) D_out[q] += part[36 * j + q];
    free(part);
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
