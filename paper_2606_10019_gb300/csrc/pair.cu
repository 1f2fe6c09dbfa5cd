// The FP64 side of the per-iteration hot path of Algorithm 1, the transform
// of the source points, and the source packing done once per call:
//   k_fin_reduce -- FP64 sums of the item partials over chunks of FIN_CHUNK
//                  work items of one problem (all SMs, whatever the batch);
//   k_fin_step  -- one warp per problem: the sum of its chunk rows, change
//                  of frame, connection term (Eq. 12), the 6x6 solve of
//                  Eq. (13) (or the G-CVO-E Newton step with the exact
//                  Hessian) and the update T <- T exp(xi); the split pose
//                  constants the transform reads.
//   k_transform -- every source point of an active problem moved into the
//                  target grid's frame at the current pose (Algorithm 1,
//                  T^-1 z): p = R^T (z - t) - o in double-float arithmetic,
//                  stored as a float head and tail, and Sigma' = R^T Sigma R.
// Source packing sorts each source cloud by a Morton code of its own voxels
// and writes one float4 record triple per point in that order.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "pair.cuh"
#include "ptx.cuh"

namespace gcvo {
namespace {

// ---------------------------------------------------------------------------
// FP64 finalize: the device-side math of the per-problem step (k_fin_step).
// ---------------------------------------------------------------------------

__device__ void hat3d(const double w[3], double W[9]) {
    W[0] = 0;     W[1] = -w[2]; W[2] = w[1];
    W[3] = w[2];  W[4] = 0;     W[5] = -w[0];
    W[6] = -w[1]; W[7] = w[0];  W[8] = 0;
}

// exp of a twist (omega, v): Rodrigues rotation and V-matrix translation,
// with series coefficients for small angles.
__device__ void exp_twist(const double xi[6], double Rout[9], double tout[3]) {
    double th2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
    double th = sqrt(th2);
    double A, B, C;
    if (th < 1e-4) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        double s, c;
        sincos(th, &s, &c);
        A = s / th;
        B = (1.0 - c) / th2;
        C = (th - s) / (th2 * th);
    }
    double W[9], W2[9];
    hat3d(xi, W);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) W2[3 * r + c] = W[3 * r] * W[c] + W[3 * r + 1] * W[3 + c] + W[3 * r + 2] * W[6 + c];
    for (int k = 0; k < 9; ++k) {
        double I = (k % 4 == 0) ? 1.0 : 0.0;
        Rout[k] = I + A * W[k] + B * W2[k];
    }
    for (int r = 0; r < 3; ++r) {
        double s = 0;
        for (int c = 0; c < 3; ++c) {
            double I = r == c ? 1.0 : 0.0;
            s += (I + B * W[3 * r + c] + C * W2[3 * r + c]) * xi[3 + c];
        }
        tout[r] = s;
    }
}

// Solve A x = b (6x6, row-major) by LU with partial pivoting.  Returns 0,
// or 1 when a pivot is exactly zero.
__device__ int solve_lu6(const double Ain[36], const double b[6], double x[6]) {
    double A[42];
    for (int r = 0; r < 6; ++r) {
        for (int c = 0; c < 6; ++c) A[7 * r + c] = Ain[6 * r + c];
        A[7 * r + 6] = b[r];
    }
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (fabs(A[7 * r + c]) > fabs(A[7 * piv + c])) piv = r;
        if (A[7 * piv + c] == 0.0) return 1;
        if (piv != c)
            for (int k = 0; k < 7; ++k) {
                double tmp = A[7 * c + k];
                A[7 * c + k] = A[7 * piv + k];
                A[7 * piv + k] = tmp;
            }
        for (int r = c + 1; r < 6; ++r) {
            double f = A[7 * r + c] / A[7 * c + c];
            for (int k = c; k < 7; ++k) A[7 * r + k] -= f * A[7 * c + k];
        }
    }
    for (int r = 5; r >= 0; --r) {
        double sm = A[7 * r + 6];
        for (int k = r + 1; k < 6; ++k) sm -= A[7 * r + k] * x[k];
        x[r] = sm / A[7 * r + r];
    }
    return 0;
}

// Gamma of Eq. (12) as a 6x6 row-major matrix: [[-1/2 g_w^, 0], [-g_v^, 0]].
__device__ void gamma6(const double g[6], double Gam[36]) {
#pragma unroll
    for (int k = 0; k < 36; ++k) Gam[k] = 0.0;
    Gam[1] = 0.5 * g[2];   Gam[2] = -0.5 * g[1];
    Gam[6] = -0.5 * g[2];  Gam[8] = 0.5 * g[0];
    Gam[12] = 0.5 * g[1];  Gam[13] = -0.5 * g[0];
    Gam[19] = g[5];  Gam[20] = -g[4];
    Gam[24] = -g[5]; Gam[26] = g[3];
    Gam[30] = g[4];  Gam[31] = -g[3];
}

// Solve (M - Gamma) xi = g (Eq. 13).  M is symmetric positive definite for a
// problem with overlap; Gamma (Eq. 12) has non-zero entries only in its first
// three columns, Gamma = Gc E^T with Gc = [-1/2 g_omega^; -g_v^] (6x3) and
// E = [I3; 0].  With the Cholesky factor of M, y = M^-1 g and Z = M^-1 Gc,
// the Sherman-Morrison-Woodbury identity gives
//   xi = y + Z (I3 - E^T Z)^-1 E^T y.
// Falls back to partial-pivot LU of M - Gamma when M is not positive
// definite.  Returns 0, or 1 when both fail.
__device__ int solve_gn(const double M[36], const double g[6], double xi[6]) {
    double Gc[18];
#pragma unroll
    for (int r = 0; r < 18; ++r) Gc[r] = 0.0;
    // Gc = [-1/2 g_omega^ ; -g_v^]
    Gc[1] = 0.5 * g[2];  Gc[2] = -0.5 * g[1];
    Gc[3] = -0.5 * g[2]; Gc[5] = 0.5 * g[0];
    Gc[6] = 0.5 * g[1];  Gc[7] = -0.5 * g[0];
    Gc[10] = g[5];  Gc[11] = -g[4];
    Gc[12] = -g[5]; Gc[14] = g[3];
    Gc[15] = g[4];  Gc[16] = -g[3];
    // Cholesky M = L L^T (inverse diagonal kept)
    double L[36], id[6];
    bool spd = true;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            double sm = M[6 * i + j];
#pragma unroll
            for (int k = 0; k < j; ++k) sm -= L[6 * i + k] * L[6 * j + k];
            if (i == j) {
                spd = spd && (sm > 0.0);
                double r = sqrt(fmax(sm, 1e-300));
                L[6 * i + i] = r;
                id[i] = 1.0 / r;
            } else {
                L[6 * i + j] = sm * id[j];
            }
        }
    }
    if (spd) {
        // X = M^-1 [g, Gc] (6 x 4)
        double X[24];
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            X[4 * r] = g[r];
#pragma unroll
            for (int c = 0; c < 3; ++c) X[4 * r + 1 + c] = Gc[3 * r + c];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                double sm = X[4 * i + c];
#pragma unroll
                for (int k = 0; k < i; ++k) sm -= L[6 * i + k] * X[4 * k + c];
                X[4 * i + c] = sm * id[i];
            }
#pragma unroll
            for (int i = 5; i >= 0; --i) {
                double sm = X[4 * i + c];
#pragma unroll
                for (int k = i + 1; k < 6; ++k) sm -= L[6 * k + i] * X[4 * k + c];
                X[4 * i + c] = sm * id[i];
            }
        }
        // K = I3 - E^T Z, w = K^-1 E^T y (Cramer), xi = y + Z w
        double K[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) K[3 * r + c] = (r == c ? 1.0 : 0.0) - X[4 * r + 1 + c];
        double c00 = K[4] * K[8] - K[5] * K[7], c01 = K[5] * K[6] - K[3] * K[8], c02 = K[3] * K[7] - K[4] * K[6];
        double detK = K[0] * c00 + K[1] * c01 + K[2] * c02;
        double kn = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) kn = fmax(kn, fabs(K[k]));
        if (fabs(detK) > 1e-12 * kn * kn * kn) {
            double idet = 1.0 / detK;
            double y0 = X[0], y1 = X[4], y2 = X[8];
            // inverse of K by its adjugate
            double w0 = (c00 * y0 + (K[2] * K[7] - K[1] * K[8]) * y1 + (K[1] * K[5] - K[2] * K[4]) * y2) * idet;
            double w1 = (c01 * y0 + (K[0] * K[8] - K[2] * K[6]) * y1 + (K[2] * K[3] - K[0] * K[5]) * y2) * idet;
            double w2 = (c02 * y0 + (K[1] * K[6] - K[0] * K[7]) * y1 + (K[0] * K[4] - K[1] * K[3]) * y2) * idet;
#pragma unroll
            for (int r = 0; r < 6; ++r) xi[r] = X[4 * r] + X[4 * r + 1] * w0 + X[4 * r + 2] * w1 + X[4 * r + 3] * w2;
            return 0;
        }
    }
    // LU with partial pivoting of M - Gamma (Gamma = Gc in the first 3 columns)
    double A[36];
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) A[6 * r + c] = M[6 * r + c] - (c < 3 ? Gc[3 * r + c] : 0.0);
    return solve_lu6(A, g, xi);
}

// G-CVO-E: D(g) in the caller's frame from the grid-frame sums of the exact
// pass.  Per source point, with y = Sigma_ij^-1 r summed over its targets,
// S_y = sum w y, S_B = sum w (y u^T + K) and P = p^ (tile.cu, pair_exact),
// the pass leaves C = sum_points (-S_y^ P + P S_B) in tot[28..36] and
// sum_points S_B in tot[37..45], row-major.  Qm is B^T (Q - M)_o B, already
// moved by the code that moves M; the rest is N_o = [[C, S_y^], [S_B, 0]]
// with S_y summed over all points = -g_v, and D = Qm - B^T N_o B for
// B = [[I, 0], [-o^, I]].
__device__ void exact_derivative(const double *tot, const double Qm[36], const double o[3], double D[36]) {
    double N[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) N[k] = 0.0;
    const double s0 = -tot[4], s1 = -tot[5], s2 = -tot[6];   // S_y
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            N[6 * r + c] = tot[28 + 3 * r + c];
            N[6 * (r + 3) + c] = tot[37 + 3 * r + c];
        }
    N[4] = -s2;  N[5] = s1;
    N[9] = s2;   N[11] = -s0;
    N[15] = -s1; N[16] = s0;
    double O[9];
    hat3d(o, O);
    // X = N B: columns 0..2 get -N[:, 3:6] o^
    double X[36];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            double v = N[6 * r + c];
            if (c < 3)
#pragma unroll
                for (int k = 0; k < 3; ++k) v -= N[6 * r + 3 + k] * O[3 * k + c];
            X[6 * r + c] = v;
        }
    // B^T X: rows 0..2 get +o^ X[3:6, :]  (B^T = [[I, o^], [0, I]])
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            double v = X[6 * r + c];
            if (r < 3)
#pragma unroll
                for (int k = 0; k < 3; ++k) v += O[3 * r + k] * X[6 * (3 + k) + c];
            D[6 * r + c] = Qm[6 * r + c] - v;
        }
}

// Smallest positive real root of the cubic d3 t^3 + d2 t^2 + d1 t + d0
// (G'(t) of Eq. 9), or -1 if none.  Closed forms (trigonometric / Cardano)
// for the cubic, then two Newton polishing steps per root.
__device__ double smallest_pos_root(double d3, double d2, double d1, double d0) {
    double roots[3];
    int nr = 0;
    double sc = fmax(fmax(fabs(d3), fabs(d2)), fmax(fabs(d1), fabs(d0)));
    if (sc == 0.0) return -1.0;
    if (fabs(d3) <= 1e-14 * sc) {
        if (fabs(d2) <= 1e-14 * sc) {
            if (d1 != 0.0) roots[nr++] = -d0 / d1;
        } else {
            double disc = d1 * d1 - 4.0 * d2 * d0;
            if (disc >= 0.0) {
                double sq = sqrt(disc);
                double qq = -0.5 * (d1 + copysign(sq, d1));
                if (qq != 0.0) roots[nr++] = d0 / qq;
                roots[nr++] = qq / d2;
            }
        }
    } else {
        double a = d2 / d3, b = d1 / d3, c = d0 / d3;
        double Q = (a * a - 3.0 * b) / 9.0;
        double Rr = (2.0 * a * a * a - 9.0 * a * b + 27.0 * c) / 54.0;
        double Q3 = Q * Q * Q;
        if (Rr * Rr < Q3) {
            double th = acos(fmin(fmax(Rr / sqrt(Q3), -1.0), 1.0));
            double m = -2.0 * sqrt(Q);
            roots[nr++] = m * cos(th / 3.0) - a / 3.0;
            roots[nr++] = m * cos((th + 2.0 * M_PI) / 3.0) - a / 3.0;
            roots[nr++] = m * cos((th - 2.0 * M_PI) / 3.0) - a / 3.0;
        } else {
            double A = -copysign(cbrt(fabs(Rr) + sqrt(Rr * Rr - Q3)), Rr);
            double B = A != 0.0 ? Q / A : 0.0;
            roots[nr++] = (A + B) - a / 3.0;
        }
    }
    double best = -1.0;
    for (int k = 0; k < nr; ++k) {
        double t = roots[k];
        for (int it = 0; it < 2; ++it) {
            double p = ((d3 * t + d2) * t + d1) * t + d0;
            double dp = (3.0 * d3 * t + 2.0 * d2) * t + d1;
            if (dp != 0.0) t -= p / dp;
        }
        if (t > 0.0 && (best < 0.0 || t < best)) best = t;
    }
    return best;
}

__device__ inline void set_inactive(ProbDev *P, int st, int *n_active) {
    P->status = st;
    atomicSub(n_active, 1);
}

__device__ inline void apply_step(ProbDev *P, const double xi[6], gcvo_iter_log *lg, const FinalizeArgs &a,
                                  int it) {
    double l1 = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) l1 += fabs(xi[k]);
    double dR[9], dt[3];
    exp_twist(xi, dR, dt);
    double Rn[9], tn[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Rn[3 * r + c] = P->T[3 * r] * dR[c] + P->T[3 * r + 1] * dR[3 + c] + P->T[3 * r + 2] * dR[6 + c];
        tn[r] = P->T[3 * r] * dt[0] + P->T[3 * r + 1] * dt[1] + P->T[3 * r + 2] * dt[2] + P->T[9 + r];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) P->T[k] = Rn[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) P->T[9 + k] = tn[k];
    if (lg) {
#pragma unroll
        for (int k = 0; k < 6; ++k) lg->xi[k] = xi[k];
        lg->xi_l1 = l1;
    }
    P->iter = it + 1;
    if (!(l1 == l1)) set_inactive(P, -(int)GCVO_ERR_NONFINITE, a.n_active);
    else if (l1 < a.eps_tol) set_inactive(P, 1, a.n_active);
    else if (it + 1 >= a.k_max) set_inactive(P, 2, a.n_active);
}

// The per-problem FP64 step (one thread): returns 1 when the pose changed
// and the problem stays active, so the transform constants must be refreshed.
__device__ int finalize_thread0(const FinalizeArgs &a, int prob, ProbDev *P, const double *tot,
                                const long long *ctot) {
    const GridDev *G = a.grids + prob;
    const double o0 = G->origin[0], o1 = G->origin[1], o2 = G->origin[2];
    const int it = P->iter;
    gcvo_iter_log *lg = a.logs ? a.logs + (size_t)prob * a.k_max + it : nullptr;

    if (a.mode == FIN_LINESEARCH) {
        // G(t) ~ sum_k c_k t^k along xi = g (Eq. 9).  c_1 = dG/dt(0) = <g, g>
        // exactly; it is taken from the FP64 gradient rather than the FP32
        // pair sums, which cancel towards zero near the optimum.
        double c1 = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) c1 += P->dir[k] * P->dir[k];
        double c2 = tot[2], c3 = tot[3], c4 = tot[4];
        double ts = smallest_pos_root(4.0 * c4, 3.0 * c3, 2.0 * c2, c1);
        double mu = ts > a.mu0 ? ts : a.mu0;
        double xi[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) xi[k] = mu * P->dir[k];
        apply_step(P, xi, lg, a, it);
        return P->status == 0;
    }

    // f, g, M in the grid-origin frame (p relative to o), moved to the
    // caller's frame: with p = p_o + o, J = J_o B for B = [[I, 0], [-o^, I]],
    // so g = B^T g_o and M = B^T M_o B.  In 3x3 blocks (A, Bm, C of M_o and
    // O = o^, X = Bm O): M_ww = A - X - X^T - O C O, M_wv = Bm + O C, M_vv = C,
    // g_w = g_ow + o x g_ov, g_v = g_ov.
    double f = tot[0];
    double A[9], Bm[9], C[9];
    {
        int q = 7;
        double U[36];
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int c = r; c < 6; ++c) {
                U[6 * r + c] = tot[q];
                U[6 * c + r] = tot[q];
                ++q;
            }
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                A[3 * r + c] = U[6 * r + c];
                Bm[3 * r + c] = U[6 * r + 3 + c];
                C[3 * r + c] = U[6 * (r + 3) + 3 + c];
            }
    }
    double X[9], CO[9], OCO[9], OC[9];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        X[3 * r + 0] = Bm[3 * r + 1] * o2 - Bm[3 * r + 2] * o1;
        X[3 * r + 1] = -Bm[3 * r + 0] * o2 + Bm[3 * r + 2] * o0;
        X[3 * r + 2] = Bm[3 * r + 0] * o1 - Bm[3 * r + 1] * o0;
        CO[3 * r + 0] = C[3 * r + 1] * o2 - C[3 * r + 2] * o1;
        CO[3 * r + 1] = -C[3 * r + 0] * o2 + C[3 * r + 2] * o0;
        CO[3 * r + 2] = C[3 * r + 0] * o1 - C[3 * r + 1] * o0;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        OCO[c] = -o2 * CO[3 + c] + o1 * CO[6 + c];
        OCO[3 + c] = o2 * CO[c] - o0 * CO[6 + c];
        OCO[6 + c] = -o1 * CO[c] + o0 * CO[3 + c];
        OC[c] = -o2 * C[3 + c] + o1 * C[6 + c];
        OC[3 + c] = o2 * C[c] - o0 * C[6 + c];
        OC[6 + c] = -o1 * C[c] + o0 * C[3 + c];
    }
    double M[36];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            M[6 * r + c] = A[3 * r + c] - X[3 * r + c] - X[3 * c + r] - OCO[3 * r + c];
            double wv = Bm[3 * r + c] + OC[3 * r + c];
            M[6 * r + 3 + c] = wv;
            M[6 * (c + 3) + r] = wv;
            M[6 * (r + 3) + 3 + c] = C[3 * r + c];
        }
    double g[6];
    {
        double gw0 = tot[1], gw1 = tot[2], gw2 = tot[3], gv0 = tot[4], gv1 = tot[5], gv2 = tot[6];
        g[0] = gw0 + (o1 * gv2 - o2 * gv1);
        g[1] = gw1 + (o2 * gv0 - o0 * gv2);
        g[2] = gw2 + (o0 * gv1 - o1 * gv0);
        g[3] = gv0;
        g[4] = gv1;
        g[5] = gv2;
    }
    bool finite = isfinite(f);
#pragma unroll
    for (int k = 0; k < 6; ++k) finite = finite && isfinite(g[k]);
#pragma unroll
    for (int k = 0; k < 36; ++k) finite = finite && isfinite(M[k]);
    // G-CVO-E: M above holds B^T (Q - M)_o B; D(g) replaces -M
    const bool exact = a.mode == FIN_EXACT || a.mode == FIN_EXACT_EVAL;
    double D[36];
    if (exact) {
        const double o[3] = {o0, o1, o2};
        exact_derivative(tot, M, o, D);
#pragma unroll
        for (int k = 0; k < 36; ++k) finite = finite && isfinite(D[k]);
    }

    if (lg) {
        lg->f = f;
#pragma unroll
        for (int k = 0; k < 6; ++k) lg->g[k] = g[k];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int c = 0; c < 3; ++c) lg->T[4 * r + c] = P->T[3 * r + c];
            lg->T[4 * r + 3] = P->T[9 + r];
        }
        lg->T[12] = lg->T[13] = lg->T[14] = 0.0;
        lg->T[15] = 1.0;
        lg->n_pairs = ctot[0];
        lg->n_kept = ctot[1];
    }

    if (a.mode == FIN_EVAL || a.mode == FIN_EXACT_EVAL) {
        // H_GN = -M + Gamma (Eq. 12); G-CVO-E: H_E = D(g) + Gamma, M <- D(g)
        EvalOut *e = a.evalout + prob;
        e->f = f;
#pragma unroll
        for (int k = 0; k < 6; ++k) e->g[k] = g[k];
        double Gam[36];
        gamma6(g, Gam);
#pragma unroll
        for (int k = 0; k < 36; ++k) {
            e->M[k] = exact ? D[k] : M[k];
            e->H[k] = (exact ? D[k] : -M[k]) + Gam[k];
        }
        e->n_pairs = ctot[0];
        e->n_kept = ctot[1];
        e->n_cand = ctot[2];
        return 0;
    }
    if (!finite) {
        set_inactive(P, -(int)GCVO_ERR_NONFINITE, a.n_active);
        return 0;
    }
    if (ctot[1] == 0 || !(f > 0.0)) {
        set_inactive(P, -(int)GCVO_ERR_NO_OVERLAP, a.n_active);
        return 0;
    }
    if (a.mode == FIN_GRAD) {
        // G-CVO-1: the line search runs along xi = g (Eq. 9); in the
        // grid-origin frame that direction has v' = omega x o + v.
#pragma unroll
        for (int k = 0; k < 6; ++k) P->dir[k] = g[k];
        P->dir32[0] = (float)g[0];
        P->dir32[1] = (float)g[1];
        P->dir32[2] = (float)g[2];
        P->dir32[3] = (float)(g[1] * o2 - g[2] * o1 + g[3]);
        P->dir32[4] = (float)(g[2] * o0 - g[0] * o2 + g[4]);
        P->dir32[5] = (float)(g[0] * o1 - g[1] * o0 + g[5]);
        return 0;
    }
    double xi[6];
    if (exact) {
        // G-CVO-E: Newton step xi = -H_E^-1 g, H_E = D(g) + Gamma (Eq. 12)
        double Gam[36], nH[36];
        gamma6(g, Gam);
#pragma unroll
        for (int k = 0; k < 36; ++k) nH[k] = -(D[k] + Gam[k]);
        if (solve_lu6(nH, g, xi) != 0) {
            set_inactive(P, -(int)GCVO_ERR_SINGULAR, a.n_active);
            return 0;
        }
        apply_step(P, xi, lg, a, it);
        return P->status == 0;
    }
    // G-CVO-2 step, Eq. (13)
    if (solve_gn(M, g, xi) != 0) {
        set_inactive(P, -(int)GCVO_ERR_SINGULAR, a.n_active);
        return 0;
    }
    apply_step(P, xi, lg, a, it);
    return P->status == 0;
}

// The split constants of the transform at the pose P->T: R as float head
// and tail, and c = R^T t + o (o the grid origin) likewise.
__device__ void refresh_pose(const FinalizeArgs &a, int prob, ProbDev *P) {
    const GridDev *G = a.grids + prob;
    double c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        c[k] = P->T[k] * P->T[9] + P->T[3 + k] * P->T[10] + P->T[6 + k] * P->T[11] + G->origin[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float h = (float)P->T[k];
        P->Rh[k] = h;
        P->Rl[k] = (float)(P->T[k] - (double)h);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float h = (float)c[k];
        P->ch[k] = h;
        P->cl[k] = (float)(c[k] - (double)h);
    }
}

constexpr int FIN_RED_THREADS = 256;   // 8 warps: item g goes to warp g % 8
// problems per block of k_fin_step: one, so that problems spread over the
// SMs and their serial FP64 steps do not share one SM's FP64 units
constexpr int FIN_STEP_WARPS = 1;

// The chunk rows: per chunk, per slot, a compensated FP32 sum of the (hi, lo)
// partials over each warp's items (8 loads in flight per warp), the warps
// added in FP64 in a fixed order; the pair counts likewise.  A persistent
// grid walks the chunks; the problem of chunk c is the last one with c0 <= c.
__global__ void __launch_bounds__(FIN_RED_THREADS) k_fin_reduce(FinalizeArgs a) {
    __shared__ double red[FIN_RED_THREADS / 32][64];
    __shared__ long long cred[FIN_RED_THREADS / 32][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // the G-CVO-E pass leaves slots 32..45 in a second partial row per item
    // (its slots 46..63 are never written, and their sums never read)
    const int rows = (a.mode == FIN_EXACT || a.mode == FIN_EXACT_EVAL) ? 2 : 1;
    const int nch = *a.n_chunks;
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        int lo = 0, hi = a.n_problems - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.probs[mid].c0 <= c) lo = mid;
            else hi = mid - 1;
        }
        const ProbDev *P = a.probs + lo;
        if (P->status != 0) continue;   // the same for the whole block
        const int i0 = P->w0 + (c - P->c0) * FIN_CHUNK, i1 = min(P->w1, i0 + FIN_CHUNK);
        for (int row = 0; row < rows; ++row) {
            const float *src = row == 0 ? a.part : a.part2;
            float H = 0.f, Lo = 0.f;
            long long cacc = 0;
#pragma unroll 8
            for (int g = i0 + w; g < i1; g += FIN_RED_THREADS / 32) {
                const float *p = src + (size_t)g * 64;
                const float h = p[lane], l = p[32 + lane];
                const float sm = H + h;
                const float bp = sm - H;
                const float err = (H - (sm - bp)) + (h - bp);
                H = sm;
                Lo += l + err;
                if (row == 0 && lane < 3) cacc += a.counts[(size_t)g * 4 + lane];
            }
            red[w][32 * row + lane] = (double)H + (double)Lo;
            if (row == 0 && lane < 4) cred[w][lane] = cacc;
        }
        __syncthreads();
        if (threadIdx.x < 32 * rows) {
            double sm = 0.0;
#pragma unroll
            for (int q = 0; q < FIN_RED_THREADS / 32; ++q) sm += red[q][threadIdx.x];
            a.chunk[(size_t)c * 64 + threadIdx.x] = sm;
        }
        if (threadIdx.x < 4) {
            long long cs = 0;
#pragma unroll
            for (int q = 0; q < FIN_RED_THREADS / 32; ++q) cs += cred[q][threadIdx.x];
            a.chunk_cnt[(size_t)c * 4 + threadIdx.x] = cs;
        }
        __syncthreads();
    }
}

// One warp per problem: the sums over its chunk rows in chunk order (FP64),
// then the per-problem FP64 step on lane 0.
__global__ void __launch_bounds__(FIN_STEP_WARPS * 32) k_fin_step(FinalizeArgs a) {
    __shared__ double tot[FIN_STEP_WARPS][64];
    __shared__ long long ctot[FIN_STEP_WARPS][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int prob = blockIdx.x * FIN_STEP_WARPS + w;
    if (prob >= a.n_problems) return;
    ProbDev *P = a.probs + prob;
    if (P->status != 0) return;
    if (a.mode == FIN_POSE) {
        if (lane == 0) refresh_pose(a, prob, P);
        return;
    }
    const int rows = (a.mode == FIN_EXACT || a.mode == FIN_EXACT_EVAL) ? 2 : 1;
    const int c0 = P->c0, c1 = P->c1;
    for (int row = 0; row < rows; ++row) {
        double sm = 0.0;
        for (int c = c0; c < c1; ++c) sm += a.chunk[(size_t)c * 64 + 32 * row + lane];
        tot[w][32 * row + lane] = sm;
    }
    if (lane < 4) {
        long long cs = 0;
        for (int c = c0; c < c1; ++c) cs += a.chunk_cnt[(size_t)c * 4 + lane];
        ctot[w][lane] = cs;
    }
    __syncwarp();
    if (lane == 0 && finalize_thread0(a, prob, P, tot[w], ctot[w])) refresh_pose(a, prob, P);
}

// ---------------------------------------------------------------------------
// Source grouping.
// ---------------------------------------------------------------------------
__device__ inline unsigned spread3(unsigned v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ inline int enc_f(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}

__global__ void k_src_keys(SrcArgs a) {
    const int p = blockIdx.y;
    const SrcDesc d = a.desc[p];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const int64_t gi = d.offset + i;
    float c[3], r[3];
    for (int k = 0; k < 3; ++k) {
        c[k] = d.xyz[k * d.n + i];
        r[k] = d.xyz[k * d.n];
    }
    unsigned m = 0;
    for (int k = 0; k < 3; ++k) {
        int q = (int)floorf((c[k] - r[k]) * d.inv_hf) + 512;
        q = min(max(q, 0), 1023);
        m |= spread3((unsigned)q) << k;
    }
    a.keys[gi] = ((unsigned long long)p << 30) | m;
    a.vals[gi] = (int)gi;
    a.prob_of[gi] = p;
    a.local[gi] = (int)i;
    bool bad = false;
    for (int k = 0; k < 3; ++k) bad |= !isfinite(c[k]);
    if (!a.iso && d.cov) {
        float s[6];
        for (int k = 0; k < 6; ++k) {
            s[k] = d.cov[k * d.n + i];
            bad |= !isfinite(s[k]);
        }
        float l = sym3_max_eig(s[0], s[1], s[2], s[3], s[4], s[5]);
        atomicMax(a.lam_enc + p, enc_f(l));
        atomicMin(a.lam_min_enc + p, enc_f(sym3_min_eig(s[0], s[1], s[2], s[3], s[4], s[5])));
    }
    if (bad) atomicOr(a.status_word, DEV_ERR_NONFINITE);
}

// One packed record triple per sorted source point, and its problem.
__global__ void k_src_pack(SrcArgs a, const unsigned long long *keys, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int src = a.vals[i];
    const SrcDesc d = a.desc[a.prob_of[src]];
    const int64_t li = a.local[src];
    const float x = d.xyz[li], y = d.xyz[d.n + li], z = d.xyz[2 * d.n + li];
    const float f0 = d.feat ? d.feat[li] : 1.f;
    const float f1 = (d.feat && a.feat_dim > 1) ? d.feat[d.n + li] : 0.f;
    const float f2 = (d.feat && a.feat_dim > 2) ? d.feat[2 * d.n + li] : 0.f;
    float s6[6] = {0, 0, 0, 0, 0, 0};
    if (!a.iso && d.cov)
        for (int k = 0; k < 6; ++k) s6[k] = d.cov[k * d.n + li];
    a.spos[i] = make_float4(x, y, z, f0);
    a.sca[i] = make_float4(s6[0], s6[1], s6[2], s6[3]);
    a.scb[i] = make_float4(s6[4], s6[5], f1, f2);
    if (a.sfx) {
        float fx[4] = {0.f, 0.f, 0.f, 0.f};
        for (int q = 3; q < a.feat_dim && q < 7; ++q) fx[q - 3] = d.feat[q * d.n + li];
        a.sfx[i] = make_float4(fx[0], fx[1], fx[2], fx[3]);
    }
    a.pprob[i] = (int)(keys[i] >> 30);
}

// ---------------------------------------------------------------------------
// The transform of Algorithm 1 (T^-1 z) for every point of an active
// problem.  p = R^T z - c is formed in double-float arithmetic from the
// float head / tail splits of R and c: each head product R_h z is split
// exactly into a float and its rounding error with one FMA (the
// error-free product of Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005), the products are added with Knuth's
// TwoSum and the rounding errors, the tail products and c's tail are
// summed in a float alongside (their Sum2 / Dot2 scheme), and a final
// FastTwoSum gives p = p_hi + p_lo with an error near 2^-48 |R| |z|.
// Sigma' = R^T Sigma R is formed in float from the head of R.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__global__ void k_transform(TransformArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const ProbDev *P = a.probs + (a.pprob ? a.pprob[i] : 0);
        if (P->status != 0) continue;   // converged or failed: left as it was
        const float4 z = a.spos[i];
        const float4 zb = a.scb[i];
        const float zz[3] = {z.x, z.y, z.z};
        float hi[3], lo[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float s = 0.f, err = 0.f;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float rh = P->Rh[3 * j + k];
                const float pr = __fmul_rn(rh, zz[j]);
                const float pe = __fmaf_rn(rh, zz[j], -pr);
                float e;
                two_sum(s, pr, s, e);
                err = __fadd_rn(err, __fadd_rn(__fadd_rn(e, pe), __fmul_rn(P->Rl[3 * j + k], zz[j])));
            }
            float e;
            two_sum(s, -P->ch[k], s, e);
            err = __fadd_rn(err, __fsub_rn(e, P->cl[k]));
            hi[k] = __fadd_rn(s, err);
            lo[k] = __fsub_rn(err, __fsub_rn(hi[k], s));
        }
        const float sg = P->sigma2;
        a.tpos[i] = make_float4(hi[0], hi[1], hi[2], sg * z.w);
        if (a.tlo) a.tlo[i] = make_float4(lo[0], lo[1], lo[2], 0.f);
        float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (!a.iso) {
            const float4 za = a.sca[i];
            const float sm[9] = {za.x, za.y, za.z, za.y, za.w, zb.x, za.z, zb.x, zb.y};
            float Rf[9], T1[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) Rf[k] = P->Rh[k];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    T1[3 * r + c] = sm[3 * r] * Rf[c] + sm[3 * r + 1] * Rf[3 + c] + sm[3 * r + 2] * Rf[6 + c];
            q[0] = Rf[0] * T1[0] + Rf[3] * T1[3] + Rf[6] * T1[6];
            q[1] = Rf[0] * T1[1] + Rf[3] * T1[4] + Rf[6] * T1[7];
            q[2] = Rf[0] * T1[2] + Rf[3] * T1[5] + Rf[6] * T1[8];
            q[3] = Rf[1] * T1[1] + Rf[4] * T1[4] + Rf[7] * T1[7];
            q[4] = Rf[1] * T1[2] + Rf[4] * T1[5] + Rf[7] * T1[8];
            q[5] = Rf[2] * T1[2] + Rf[5] * T1[5] + Rf[8] * T1[8];
        }
        a.tca[i] = make_float4(q[0], q[1], q[2], q[3]);
        a.tcb[i] = make_float4(q[4], q[5], sg * zb.z, sg * zb.w);
        if (a.tfx) {
            const float4 f = a.sfx[i];
            a.tfx[i] = make_float4(sg * f.x, sg * f.y, sg * f.z, sg * f.w);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t s) {
    if (a.mode != FIN_POSE) {
        k_fin_reduce<<<(unsigned)(a.reduce_blocks > 0 ? a.reduce_blocks : 1024), FIN_RED_THREADS, 0, s>>>(a);
        count_launches(1);
    }
    k_fin_step<<<(unsigned)((a.n_problems + FIN_STEP_WARPS - 1) / FIN_STEP_WARPS), FIN_STEP_WARPS * 32, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_src_keys(const SrcArgs &a, int n_problems, int64_t max_n, cudaStream_t s) {
    dim3 grid((unsigned)((max_n + 255) / 256), (unsigned)n_problems);
    k_src_keys<<<grid, 256, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_src_pack(const SrcArgs &a, const unsigned long long *keys, int64_t n, cudaStream_t s) {
    k_src_pack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, keys, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_transform(const TransformArgs &a, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((a.n + 255) / 256, 1 << 20);
    k_transform<<<(unsigned)blocks, 256, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gcvo
