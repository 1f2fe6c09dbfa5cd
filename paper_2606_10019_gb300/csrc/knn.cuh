// Device helpers of the kNN covariance kernels (Eq. 7b and the eigenvalue
// bound that follows it), shared by grid.cu (pass 1) and knn_far.cu (pass 2).
#pragma once

#include "common.cuh"

namespace gcvo {
namespace knn {

constexpr int KNN_MAX = GCVO_MAX_KNN;

// Symmetric 3x3 eigen-decomposition in double precision by cyclic Jacobi
// sweeps; returns eigenvalues in w and eigenvectors as the columns of V.
__device__ inline void jacobi3(double a[3][3], double w[3], double V[3][3]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) V[r][c] = r == c ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 32; ++sweep) {
        double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
        double dia = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]);
        if (off <= 1e-300 || off < 1e-17 * dia) break;
        const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
        for (int k = 0; k < 3; ++k) {
            int p = P[k], q = Q[k];
            double apq = a[p][q];
            if (apq == 0.0) continue;
            double tau = (a[q][q] - a[p][p]) / (2.0 * apq);
            double t = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
            double c = rsqrt(1.0 + t * t), s = t * c;
            // A <- G^T A G with G the rotation in the (p, q) plane
            for (int m = 0; m < 3; ++m) {
                double amp = a[m][p], amq = a[m][q];
                a[m][p] = c * amp - s * amq;
                a[m][q] = s * amp + c * amq;
            }
            for (int m = 0; m < 3; ++m) {
                double apm = a[p][m], aqm = a[q][m];
                a[p][m] = c * apm - s * aqm;
                a[q][m] = s * apm + c * aqm;
            }
            a[p][q] = a[q][p] = 0.0;
            for (int m = 0; m < 3; ++m) {
                double vmp = V[m][p], vmq = V[m][q];
                V[m][p] = c * vmp - s * vmq;
                V[m][q] = s * vmp + c * vmq;
            }
        }
    }
    for (int k = 0; k < 3; ++k) w[k] = a[k][k];
}

// One cloud of a batched covariance call (device copy).
struct KnnCloud {
    const float *xyz;     // 3 x n SoA
    float *cov;           // 6 x n SoA output
    int64_t n, off;       // points; index of the first one in the gathered array
    double eig_max, eig_ratio;
    double cell0;         // search voxel from the kernel range; 0: from the box
    int knn;
    int pad;
};

// Cloud of a gathered or sorted point: its index is carried in w.
__device__ __forceinline__ int cloud_of(float4 p) { return __float_as_int(p.w); }

// The nearest points found so far, in DESCENDING order of (squared
// distance, original index): slot 0 holds the knn-th nearest, the pruning
// bound, and slots knn .. KNN_MAX-1 are unused.  Every access is to a slot
// fixed at compile time (the loops over slots are unrolled, with knn as a
// predicate), so the list stays in registers.
struct KnnList {
    float d[KNN_MAX];
    int i[KNN_MAX];   // original index (tie-break)
    int k[KNN_MAX];   // sorted index in the grid searched
};

__device__ __forceinline__ void knn_list_init(KnnList &L) {
#pragma unroll
    for (int m = 0; m < KNN_MAX; ++m) {
        L.d[m] = INFINITY;
        L.i[m] = 0x7fffffff;
        L.k[m] = -1;
    }
}

// Insert a candidate that precedes slot 0: slot 0 drops out, the entries
// still farther than the candidate move up one slot, and the candidate takes
// the slot after them.
__device__ __forceinline__ void knn_list_insert(KnnList &L, int knn, float cd, int ci, int ck) {
    bool placing = true;
#pragma unroll
    for (int m = 0; m < KNN_MAX; ++m) {
        if (m < knn && placing) {
            float nd = -INFINITY;
            int ni = -1, nk = -1;
            if (m + 1 < KNN_MAX && m + 1 < knn) {
                nd = L.d[m + 1 < KNN_MAX ? m + 1 : m];
                ni = L.i[m + 1 < KNN_MAX ? m + 1 : m];
                nk = L.k[m + 1 < KNN_MAX ? m + 1 : m];
            }
            if (nd > cd || (nd == cd && ni > ci)) {
                L.d[m] = nd;
                L.i[m] = ni;
                L.k[m] = nk;
            } else {
                L.d[m] = cd;
                L.i[m] = ci;
                L.k[m] = ck;
                placing = false;
            }
        }
    }
}

// The knn nearest points of q in grid g, searching shells R = 1..R_max of
// voxels around q's voxel.  After shell R every point closer than R * h has
// been seen, so the search is complete (returns true) once the knn-th
// distance is within R * h.
__device__ __forceinline__ bool knn_search(const GridDev &g, float4 q, int knn, int R_max, KnnList &L) {
    int cq[3];
    float qc[3] = {q.x, q.y, q.z};
    for (int a = 0; a < 3; ++a) {
        int c = (int)floorf((qc[a] - g.corner[a]) * g.inv_h);
        cq[a] = min(max(c, 0), g.dims[a] - 1);
    }
    knn_list_init(L);
    #pragma unroll 1
    for (int R = 1; R <= R_max; ++R) {
        #pragma unroll 1
        for (int dx = -R; dx <= R; ++dx) {
            int cx = cq[0] + dx;
            if (cx < 0 || cx >= g.dims[0]) continue;
            #pragma unroll 1
            for (int dy = -R; dy <= R; ++dy) {
                int cy = cq[1] + dy;
                if (cy < 0 || cy >= g.dims[1]) continue;
                // shell R: voxels with max(|dx|, |dy|, |dz|) == R; shell 1 is
                // the whole 3 x 3 x 3 block, centre included
                bool xy_edge = (dx == -R || dx == R || dy == -R || dy == R);
                int step = (R == 1 || xy_edge) ? 1 : 2 * R;
                #pragma unroll 1
                for (int dz = -R; dz <= R; dz += step) {
                    int cz = cq[2] + dz;
                    if (cz < 0 || cz >= g.dims[2]) continue;
                    unsigned long long key = g.key_base + ((unsigned long long)cx * g.dims[1] + cy) * g.dims[2] + cz;
                    int c = grid_lookup(g, key);
                    if (c < 0) continue;
                    int s0 = g.cell_start[c], s1 = g.cell_start[c + 1];
                    for (int k = s0; k < s1; ++k) {
                        float4 y = g.pos[k];
                        float ex = y.x - q.x, ey = y.y - q.y, ez = y.z - q.z;
                        float d2 = ex * ex + ey * ey + ez * ez;
                        if (d2 > L.d[0]) continue;
                        int oi = g.orig[k];
                        if (d2 == L.d[0] && oi >= L.i[0]) continue;
                        knn_list_insert(L, knn, d2, oi, k);
                    }
                }
            }
        }
        float reach = (float)R * g.h;
        if (L.i[0] != 0x7fffffff && L.d[0] <= reach * reach * 0.999f) return true;
    }
    return false;
}

// Eq. (7b) over the list, then the eigenvalue bound; writes column o of cov_out.
// DESC: the list is a KnnList from knn_search (descending); otherwise it is
// ascending (the merged list of the warp search).  The sum runs in ascending
// order either way.
template <bool DESC>
__device__ __forceinline__ void knn_write_cov(const GridDev &g, float4 q, const KnnList &L, int knn, double eig_max,
                              double eig_ratio, int64_t n, int o, float *cov_out) {
    // Sigma = 1/(n-1) sum (y - x)(y - x)^T, centred at the query point
    float S[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int mm = 0; mm < KNN_MAX; ++mm) {
        const int m = DESC ? KNN_MAX - 1 - mm : mm;
        if (m < knn) {
            float4 y = g.pos[L.k[m]];
            float d0 = y.x - q.x, d1 = y.y - q.y, d2 = y.z - q.z;
            S[0] += d0 * d0;
            S[1] += d0 * d1;
            S[2] += d0 * d2;
            S[3] += d1 * d1;
            S[4] += d1 * d2;
            S[5] += d2 * d2;
        }
    }
    float inv = 1.0f / (float)(knn - 1);
    for (int k = 0; k < 6; ++k) S[k] *= inv;
    if (eig_max > 0.0) {
        double a[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
        double w[3], V[3][3];
        jacobi3(a, w, V);
        double lo = eig_max / eig_ratio;
        for (int k = 0; k < 3; ++k) w[k] = fmin(fmax(w[k], lo), eig_max);
        double B[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                B[r][c] = V[r][0] * w[0] * V[c][0] + V[r][1] * w[1] * V[c][1] + V[r][2] * w[2] * V[c][2];
        S[0] = (float)B[0][0];
        S[1] = (float)(0.5 * (B[0][1] + B[1][0]));
        S[2] = (float)(0.5 * (B[0][2] + B[2][0]));
        S[3] = (float)B[1][1];
        S[4] = (float)(0.5 * (B[1][2] + B[2][1]));
        S[5] = (float)B[2][2];
    }
    for (int k = 0; k < 6; ++k) cov_out[k * n + o] = S[k];
}


}  // namespace knn
}  // namespace gcvo
