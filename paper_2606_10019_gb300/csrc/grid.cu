// Target voxel hash (gcvo_build_grid) and per-point kNN covariances
// (gcvo_estimate_covariances, Eq. 7b and the eigenvalue bound that follows it).
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace gcvo {
namespace {

__device__ inline int dec_int(int k) { return k >= 0 ? k : k ^ 0x7fffffff; }

__global__ void k_voxel_keys(const float *xyz, int64_t n, GridDev g, bool absolute, unsigned long long *keys,
                             int *vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3];
    for (int a = 0; a < 3; ++a) {
        float v = xyz[a * n + i];
        float cv = absolute ? v : (float)((double)v - g.origin[a]);
        int q = (int)floorf((cv - g.corner[a]) * g.inv_h);
        c[a] = min(max(q, 0), g.dims[a] - 1);
    }
    keys[i] = ((unsigned long long)c[0] * g.dims[1] + c[1]) * g.dims[2] + c[2];
    vals[i] = (int)i;
}

__global__ void k_heads(const unsigned long long *keys, int64_t n, int *head) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_cells(const unsigned long long *keys, const int *incl, int64_t n, int dz, int *cell_start,
                        unsigned long long *hkeys, int *hval, unsigned long long hmask, int2 *col_range,
                        int *cell_z) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long k = keys[i];
    const unsigned long long col = k / (unsigned long long)dz;
    if (i == 0 || k != keys[i - 1]) {
        int c = incl[i] - 1;
        cell_start[c] = (int)i;
        cell_z[c] = (int)(k - col * (unsigned long long)dz);
        unsigned long long s = hash_key(k) & hmask;
        for (;;) {
            unsigned long long prev = atomicCAS(hkeys + s, EMPTY_KEY, k);
            if (prev == EMPTY_KEY || prev == k) {
                hval[s] = c;
                break;
            }
            s = (s + 1) & hmask;
        }
        // voxels of one (cx, cy) column are consecutive: record where each
        // column starts and where the previous one ends
        if (i == 0) {
            col_range[col].x = c;
        } else {
            const unsigned long long pcol = keys[i - 1] / (unsigned long long)dz;
            if (pcol != col) {
                col_range[col].x = c;
                col_range[pcol].y = c;
            }
        }
    }
    if (i == n - 1) {
        cell_start[incl[i]] = (int)n;
        col_range[col].y = incl[i];
    }
}

__global__ void k_fill_u64(unsigned long long *p, int64_t n, unsigned long long v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_reorder(const float *xyz, const float *cov, const float *feat, int feat_dim, int64_t n,
                          const int *vals, GridDev g, bool absolute, float4 *pos, float4 *ca, float4 *cb,
                          int *orig) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = vals[i];
    float p[3];
    for (int a = 0; a < 3; ++a) {
        float v = xyz[a * n + j];
        p[a] = absolute ? v : (float)((double)v - g.origin[a]);
    }
    float l[3] = {0.f, 0.f, 0.f};
    for (int q = 0; q < feat_dim && feat; ++q) l[q] = feat[q * n + j];
    float c[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (cov)
        for (int q = 0; q < 6; ++q) c[q] = cov[q * n + j];
    pos[i] = make_float4(p[0], p[1], p[2], l[0]);
    ca[i] = make_float4(c[0], c[1], c[2], c[3]);
    cb[i] = make_float4(c[4], c[5], l[1], l[2]);
    orig[i] = j;
}

unsigned long long next_pow2(unsigned long long v) {
    unsigned long long p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

gcvo_status build_grid_store(gcvo_ctx *ctx, const float *xyz, const float *cov, const float *feat, int64_t n,
                             const gcvo_kernel_params &kp, bool absolute, double cell, GridStore &out) {
    cudaStream_t s = ctx->stream;
    if (n <= 0 || n > (int64_t)1 << 30) return GCVO_ERR_INVALID_ARG;
    GCVO_TRY(ctx->small.ensure(4096, s));
    float *bb = ctx->small.as<float>();
    GCVO_TRY(bbox_lammax(xyz, kp.kernel_mode == 0 ? cov : nullptr, n, bb, s));
    int hb[8];
    GCVO_CUDA(cudaMemcpyAsync(hb, bb, sizeof(hb), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    auto dec = [](int k) {
        int i = k >= 0 ? k : k ^ 0x7fffffff;
        float f;
        memcpy(&f, &i, 4);
        return f;
    };
    float mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
        mn[a] = dec(hb[a]);
        mx[a] = dec(hb[3 + a]);
    }
    float lam = dec(hb[6]);
    if (hb[7] & 1) return GCVO_ERR_NONFINITE;
    if ((hb[7] & 2) && kp.kernel_mode == 0 && cov) return GCVO_ERR_INVALID_ARG;

    double h = cell;
    if (h <= 0) {
        // half the kernel range: finer voxels hug the range ball more tightly
        if (kp.kernel_mode == 1)
            h = 0.5 * kp.cutoff * kp.iso_ell;
        else
            h = 0.5 * kp.cutoff * std::sqrt(2.0 * (double)lam);
    }
    if (!(h > 0) || !std::isfinite(h)) return GCVO_ERR_INVALID_ARG;

    GridDev g{};
    g.h = (float)h;
    g.inv_h = (float)(1.0 / h);
    g.feat_dim = kp.feat_dim;
    g.kernel_mode = kp.kernel_mode;
    g.lam_max = lam;
    double prod = 1.0;
    for (int a = 0; a < 3; ++a) {
        g.origin[a] = absolute ? 0.0 : 0.5 * ((double)mn[a] + (double)mx[a]);
        g.corner[a] = absolute ? mn[a] : (float)((double)mn[a] - g.origin[a]);
        double ext = ((double)mx[a] - (double)mn[a]) / h;
        if (ext > 1.0e9) return GCVO_ERR_CAPACITY;
        g.dims[a] = (int)std::floor(ext) + 2;
        prod *= g.dims[a];
    }
    if (prod > 4.0e18) return GCVO_ERR_CAPACITY;
    const double n_columns = (double)g.dims[0] * (double)g.dims[1];
    if (n_columns > (double)(1 << 27)) return GCVO_ERR_CAPACITY;
    int bits = 1;
    while ((double)(1ull << bits) < prod && bits < 62) ++bits;

    // voxel keys, sorted
    GCVO_TRY(ctx->sort_keys.ensure(n * sizeof(unsigned long long), s));
    GCVO_TRY(ctx->sort_vals.ensure(n * sizeof(int) * 2 + 1024, s));
    GCVO_TRY(ctx->sort_tmp.ensure(radix_sort_scratch_bytes(n), s));
    GCVO_TRY(ctx->scan_tmp.ensure(scan_scratch_bytes(n) + 1024, s));
    auto *keys = ctx->sort_keys.as<unsigned long long>();
    int *vals = ctx->sort_vals.as<int>();
    int *incl = vals + ((n + 63) / 64) * 64;
    unsigned blocks = (unsigned)((n + 255) / 256);
    k_voxel_keys<<<blocks, 256, 0, s>>>(xyz, n, g, absolute, keys, vals);
    count_launches(1);
    GCVO_CUDA(cudaGetLastError());
    GCVO_TRY(radix_sort_pairs(keys, vals, n, bits, ctx->sort_tmp.ptr, ctx->sort_tmp.bytes, s));

    // voxel ranges and hash of occupied voxels
    k_heads<<<blocks, 256, 0, s>>>(keys, n, incl);
    count_launches(1);
    GCVO_TRY(scan_inclusive_sum(incl, n, ctx->scan_tmp.ptr, s));
    int n_cells = 0;
    GCVO_CUDA(cudaMemcpyAsync(&n_cells, incl + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    unsigned long long H = next_pow2((unsigned long long)std::max<int64_t>(64, 2 * (int64_t)n_cells));
    GCVO_TRY(out.pos.ensure(n * sizeof(float4), s));
    GCVO_TRY(out.ca.ensure(n * sizeof(float4), s));
    GCVO_TRY(out.cb.ensure(n * sizeof(float4), s));
    GCVO_TRY(out.orig.ensure(n * sizeof(int), s));
    GCVO_TRY(out.cell_start.ensure((n_cells + 1) * sizeof(int), s));
    GCVO_TRY(out.hkeys.ensure(H * sizeof(unsigned long long), s));
    GCVO_TRY(out.hval.ensure(H * sizeof(int), s));
    GCVO_TRY(out.col_range.ensure((size_t)n_columns * sizeof(int2), s));
    GCVO_TRY(out.cell_z.ensure((size_t)(n_cells + 1) * sizeof(int), s));
    GCVO_CUDA(cudaMemsetAsync(out.col_range.ptr, 0, (size_t)n_columns * sizeof(int2), s));
    k_fill_u64<<<(unsigned)((H + 255) / 256), 256, 0, s>>>(out.hkeys.as<unsigned long long>(), (int64_t)H,
                                                          EMPTY_KEY);
    k_cells<<<blocks, 256, 0, s>>>(keys, incl, n, g.dims[2], out.cell_start.as<int>(),
                                   out.hkeys.as<unsigned long long>(), out.hval.as<int>(), H - 1,
                                   out.col_range.as<int2>(), out.cell_z.as<int>());
    k_reorder<<<blocks, 256, 0, s>>>(xyz, kp.kernel_mode == 0 ? cov : nullptr, feat, kp.feat_dim, n, vals, g,
                                     absolute, out.pos.as<float4>(), out.ca.as<float4>(), out.cb.as<float4>(),
                                     out.orig.as<int>());
    count_launches(3);
    GCVO_CUDA(cudaGetLastError());

    g.pos = out.pos.as<float4>();
    g.ca = out.ca.as<float4>();
    g.cb = out.cb.as<float4>();
    g.orig = out.orig.as<int>();
    g.cell_start = out.cell_start.as<int>();
    g.hkeys = out.hkeys.as<unsigned long long>();
    g.hval = out.hval.as<int>();
    g.col_range = out.col_range.as<int2>();
    g.cell_z = out.cell_z.as<int>();
    g.hmask = H - 1;
    g.n = (int)n;
    g.n_cells = n_cells;
    out.d = g;
    return GCVO_OK;
}

// ---------------------------------------------------------------------------
// kNN covariances.  One thread per point searches growing shells of voxels
// around its own voxel; after shell R every point closer than R * h has been
// seen, so the search stops once the knn-th distance is within R * h.  The
// neighbour list is ordered by (squared distance, original index).
// ---------------------------------------------------------------------------
namespace {

constexpr int KNN_MAX = GCVO_MAX_KNN;

// Symmetric 3x3 eigen-decomposition in double precision by cyclic Jacobi
// sweeps; returns eigenvalues in w and eigenvectors as the columns of V.
__device__ void jacobi3(double a[3][3], double w[3], double V[3][3]) {
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

struct KnnList {
    float d[KNN_MAX];
    int i[KNN_MAX];   // original index (tie-break)
    int k[KNN_MAX];   // sorted index in the grid searched
};

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
#pragma unroll
    for (int m = 0; m < KNN_MAX; ++m) {
        L.d[m] = INFINITY;
        L.i[m] = 0x7fffffff;
        L.k[m] = -1;
    }
    float wd = INFINITY;   // knn-th distance so far
    int wi = 0x7fffffff;   // its original index (INT_MAX while the list is short)
    for (int R = 1; R <= R_max; ++R) {
        for (int dx = -R; dx <= R; ++dx) {
            int cx = cq[0] + dx;
            if (cx < 0 || cx >= g.dims[0]) continue;
            for (int dy = -R; dy <= R; ++dy) {
                int cy = cq[1] + dy;
                if (cy < 0 || cy >= g.dims[1]) continue;
                // shell R: voxels with max(|dx|, |dy|, |dz|) == R; shell 1 is
                // the whole 3 x 3 x 3 block, centre included
                bool xy_edge = (dx == -R || dx == R || dy == -R || dy == R);
                int step = (R == 1 || xy_edge) ? 1 : 2 * R;
                for (int dz = -R; dz <= R; dz += step) {
                    int cz = cq[2] + dz;
                    if (cz < 0 || cz >= g.dims[2]) continue;
                    unsigned long long key = ((unsigned long long)cx * g.dims[1] + cy) * g.dims[2] + cz;
                    int c = grid_lookup(g, key);
                    if (c < 0) continue;
                    int s0 = g.cell_start[c], s1 = g.cell_start[c + 1];
                    for (int k = s0; k < s1; ++k) {
                        float4 y = g.pos[k];
                        float ex = y.x - q.x, ey = y.y - q.y, ez = y.z - q.z;
                        float d2 = ex * ex + ey * ey + ez * ez;
                        if (d2 > wd) continue;
                        int oi = g.orig[k];
                        if (d2 == wd && oi >= wi) continue;
                        float cd = d2;
                        int ci = oi, ck = k;
#pragma unroll
                        for (int m = 0; m < KNN_MAX; ++m) {
                            if (m < knn) {
                                bool less = cd < L.d[m] || (cd == L.d[m] && ci < L.i[m]);
                                if (less) {
                                    float td = L.d[m];
                                    int ti = L.i[m], tk = L.k[m];
                                    L.d[m] = cd;
                                    L.i[m] = ci;
                                    L.k[m] = ck;
                                    cd = td;
                                    ci = ti;
                                    ck = tk;
                                }
                            }
                        }
#pragma unroll
                        for (int m = 0; m < KNN_MAX; ++m)
                            if (m == knn - 1) {
                                wd = L.d[m];
                                wi = L.i[m];
                            }
                    }
                }
            }
        }
        float reach = (float)R * g.h;
        if (wi != 0x7fffffff && wd <= reach * reach * 0.999f) return true;
    }
    return false;
}

// Eq. (7b) over the list, then the eigenvalue bound; writes column o of cov_out.
__device__ __forceinline__ void knn_write_cov(const GridDev &g, float4 q, const KnnList &L, int knn, double eig_max,
                              double eig_ratio, int64_t n, int o, float *cov_out) {
    // Sigma = 1/(n-1) sum (y - x)(y - x)^T, centred at the query point
    float S[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int m = 0; m < KNN_MAX; ++m) {
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

// Pass 1 on the fine grid (shells 1 and 2); points whose neighbours lie
// farther away are queued for pass 2.
__global__ void k_knn_cov(GridDev g, int knn, double eig_max, double eig_ratio, int64_t n, float *cov_out,
                          int *retry, int *n_retry) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 q = g.pos[i];
    KnnList L;
    if (knn_search(g, q, knn, 2, L))
        knn_write_cov(g, q, L, knn, eig_max, eig_ratio, n, g.orig[i], cov_out);
    else
        retry[atomicAdd(n_retry, 1)] = (int)i;
}

// Pass 2: one warp per queued point, searching the coarse grid shell by
// shell without a limit.  The lanes split each shell's voxels and keep
// private sorted lists; after every shell the warp merges them (repeated
// warp-wide minimum over each lane's next entry) into the knn nearest so
// far, and stops once the knn-th distance is within the shells' reach.
__global__ void k_knn_cov_far(GridDev fine, GridDev coarse, int knn, double eig_max, double eig_ratio, int64_t n,
                              float *cov_out, const int *retry, const int *n_retry, unsigned *status) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int m = *n_retry;
    const int maxR = max(coarse.dims[0], max(coarse.dims[1], coarse.dims[2]));
    for (int t = blockIdx.x * wpb + (threadIdx.x >> 5); t < m; t += gridDim.x * wpb) {
        const int i = retry[t];
        const float4 q = fine.pos[i];
        int cq[3];
        {
            float qc[3] = {q.x, q.y, q.z};
            for (int a = 0; a < 3; ++a) {
                int c = (int)floorf((qc[a] - coarse.corner[a]) * coarse.inv_h);
                cq[a] = min(max(c, 0), coarse.dims[a] - 1);
            }
        }
        KnnList L;   // this lane's private list
#pragma unroll
        for (int k = 0; k < KNN_MAX; ++k) {
            L.d[k] = INFINITY;
            L.i[k] = 0x7fffffff;
            L.k[k] = -1;
        }
        float wd = INFINITY;
        int wi = 0x7fffffff;
        KnnList M;   // merged result (identical in every lane)
        bool done = false;
        for (int R = 1; R <= maxR && !done; ++R) {
            const int side = 2 * R + 1;
            const int cube = side * side * side;
            for (int v = lane; v < cube; v += 32) {
                int dx = v / (side * side) - R, dy = (v / side) % side - R, dz = v % side - R;
                if (R > 1 && max(abs(dx), max(abs(dy), abs(dz))) != R) continue;   // shell only
                int cx = cq[0] + dx, cy = cq[1] + dy, cz = cq[2] + dz;
                if (cx < 0 || cy < 0 || cz < 0 || cx >= coarse.dims[0] || cy >= coarse.dims[1] ||
                    cz >= coarse.dims[2])
                    continue;
                unsigned long long key = ((unsigned long long)cx * coarse.dims[1] + cy) * coarse.dims[2] + cz;
                int c = grid_lookup(coarse, key);
                if (c < 0) continue;
                for (int k = coarse.cell_start[c], k1 = coarse.cell_start[c + 1]; k < k1; ++k) {
                    float4 y = coarse.pos[k];
                    float ex = y.x - q.x, ey = y.y - q.y, ez = y.z - q.z;
                    float d2 = ex * ex + ey * ey + ez * ez;
                    if (d2 > wd) continue;
                    int oi = coarse.orig[k];
                    if (d2 == wd && oi >= wi) continue;
                    float cd = d2;
                    int ci = oi, ck = k;
#pragma unroll
                    for (int mm = 0; mm < KNN_MAX; ++mm) {
                        if (mm < knn) {
                            bool less = cd < L.d[mm] || (cd == L.d[mm] && ci < L.i[mm]);
                            if (less) {
                                float td = L.d[mm];
                                int ti = L.i[mm], tk = L.k[mm];
                                L.d[mm] = cd;
                                L.i[mm] = ci;
                                L.k[mm] = ck;
                                cd = td;
                                ci = ti;
                                ck = tk;
                            }
                        }
                    }
#pragma unroll
                    for (int mm = 0; mm < KNN_MAX; ++mm)
                        if (mm == knn - 1) {
                            wd = L.d[mm];
                            wi = L.i[mm];
                        }
                }
            }
            // merge: knn rounds of a warp-wide minimum over (d, index)
            int head = 0;
            for (int r = 0; r < knn; ++r) {
                float hd = INFINITY;
                int hi = 0x7fffffff, hk = -1;
#pragma unroll
                for (int mm = 0; mm < KNN_MAX; ++mm)
                    if (mm == head) {
                        hd = L.d[mm];
                        hi = L.i[mm];
                        hk = L.k[mm];
                    }
                float bd = hd;
                int bi = hi;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    float od = __shfl_xor_sync(FULL, bd, o);
                    int oi = __shfl_xor_sync(FULL, bi, o);
                    if (od < bd || (od == bd && oi < bi)) {
                        bd = od;
                        bi = oi;
                    }
                }
                const bool mine = (hd == bd && hi == bi && hk >= 0);
                const unsigned who = __ballot_sync(FULL, mine);
                const int src = who ? __ffs(who) - 1 : 0;
                const int bk = __shfl_sync(FULL, hk, src);
                if (lane == src && who) ++head;
#pragma unroll
                for (int mm = 0; mm < KNN_MAX; ++mm)
                    if (mm == r) {
                        M.d[mm] = who ? bd : INFINITY;
                        M.i[mm] = who ? bi : 0x7fffffff;
                        M.k[mm] = who ? bk : -1;
                    }
            }
            // every lane prunes with the merged knn-th distance from now on
            float md = INFINITY;
            int mi = 0x7fffffff, mk = -1;
#pragma unroll
            for (int mm = 0; mm < KNN_MAX; ++mm)
                if (mm == knn - 1) {
                    md = M.d[mm];
                    mi = M.i[mm];
                    mk = M.k[mm];
                }
            if (mk >= 0 && (md < wd || (md == wd && mi < wi))) {
                wd = md;
                wi = mi;
            }
            const float reach = (float)R * coarse.h;
            done = mk >= 0 && md <= reach * reach * 0.999f;
        }
        bool full = true;
#pragma unroll
        for (int mm = 0; mm < KNN_MAX; ++mm)
            if (mm < knn && M.k[mm] < 0) full = false;
        if (!full) {
            if (lane == 0) atomicOr(status, DEV_ERR_CAPACITY);
            continue;
        }
        if (lane == 0) knn_write_cov(coarse, q, M, knn, eig_max, eig_ratio, n, fine.orig[i], cov_out);
    }
}

}  // namespace

gcvo_status knn_covariances(gcvo_ctx *ctx, const float *xyz, int64_t n, const gcvo_kernel_params &kp,
                            float *cov_out) {
    cudaStream_t s = ctx->stream;
    // search voxel: the kernel range when an eigenvalue bound is given,
    // otherwise a size from the bounding box (the shell search adapts).
    gcvo_kernel_params q = kp;
    q.kernel_mode = 1;
    q.feat_dim = 0;
    double cell = 0.0;
    if (kp.eig_max > 0) {
        cell = kp.cutoff * std::sqrt(2.0 * kp.eig_max) * 0.5;
    } else {
        GCVO_TRY(ctx->small.ensure(4096, s));
        float *bb = ctx->small.as<float>();
        GCVO_TRY(bbox_lammax(xyz, nullptr, n, bb, s));
        int hb[8];
        GCVO_CUDA(cudaMemcpyAsync(hb, bb, sizeof(hb), cudaMemcpyDeviceToHost, s));
        GCVO_CUDA(cudaStreamSynchronize(s));
        auto dec = [](int k) {
            int i = k >= 0 ? k : k ^ 0x7fffffff;
            float f;
            memcpy(&f, &i, 4);
            return f;
        };
        double vol = 1.0;
        int nz = 0;
        double ext[3];
        for (int a = 0; a < 3; ++a) {
            ext[a] = (double)dec(hb[3 + a]) - (double)dec(hb[a]);
            if (ext[a] > 0) {
                vol *= ext[a];
                ++nz;
            }
        }
        if (hb[7] & 1) return GCVO_ERR_NONFINITE;
        cell = nz > 0 ? std::pow(vol / (double)n, 1.0 / nz) * 2.0 : 1.0;
        if (!(cell > 0)) cell = 1.0;
    }
    GridStore &fine = ctx->knn_grid;
    GridStore &coarse = ctx->knn_grid2;
    GCVO_TRY(build_grid_store(ctx, xyz, nullptr, nullptr, n, q, true, cell, fine));
    GCVO_TRY(build_grid_store(ctx, xyz, nullptr, nullptr, n, q, true, cell * 8.0, coarse));
    GCVO_TRY(ctx->status_word.ensure(256, s));
    GCVO_TRY(ctx->knn_retry.ensure(n * sizeof(int) + 256, s));
    unsigned *stw = ctx->status_word.as<unsigned>();
    int *n_retry = reinterpret_cast<int *>(stw + 1);
    GCVO_CUDA(cudaMemsetAsync(stw, 0, 2 * sizeof(unsigned), s));
    k_knn_cov<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(fine.d, kp.knn, kp.eig_max, kp.eig_ratio, n, cov_out,
                                                          ctx->knn_retry.as<int>(), n_retry);
    k_knn_cov_far<<<std::max(1, ctx->sm_count) * 4, 128, 0, s>>>(fine.d, coarse.d, kp.knn, kp.eig_max,
                                                                kp.eig_ratio, n, cov_out, ctx->knn_retry.as<int>(),
                                                                n_retry, stw);
    count_launches(2);
    GCVO_CUDA(cudaGetLastError());
    unsigned hs = 0;
    GCVO_CUDA(cudaMemcpyAsync(&hs, stw, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    if (hs & DEV_ERR_CAPACITY) return GCVO_ERR_INVALID_ARG;
    return GCVO_OK;
}

}  // namespace gcvo
