// Target voxel hash (gcvo_build_grid) and per-point kNN covariances
// (gcvo_estimate_covariances, Eq. 7b and the eigenvalue bound that follows it).
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "knn.cuh"

namespace gcvo {
namespace {

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

__global__ void k_cells(const unsigned long long *keys, const int *incl, int64_t n, int *cell_start,
                        unsigned long long *hkeys, int *hval, unsigned long long hmask) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long k = keys[i];
    if (i == 0 || k != keys[i - 1]) {
        int c = incl[i] - 1;
        cell_start[c] = (int)i;
        unsigned long long s = hash_key(k) & hmask;
        for (;;) {
            unsigned long long prev = atomicCAS(hkeys + s, EMPTY_KEY, k);
            if (prev == EMPTY_KEY || prev == k) {
                hval[s] = c;
                break;
            }
            s = (s + 1) & hmask;
        }
    }
    if (i == n - 1) cell_start[incl[i]] = (int)n;
}

// Points per voxel, stored one slot up: after an inclusive scan, entry v is
// the number of points in voxels before v (the first sorted point of v).
__global__ void k_vox_count(const unsigned long long *keys, int64_t n, int *vox) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    atomicAdd(vox + keys[i] + 1, 1);
}

__global__ void k_fill_u64(unsigned long long *p, int64_t n, unsigned long long v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_reorder(const float *xyz, const float *cov, const float *feat, int feat_dim, int64_t n,
                          const int *vals, GridDev g, bool absolute, float4 *pos, float4 *ca, float4 *cb,
                          float4 *plo, float4 *fx, int *orig) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = vals[i];
    float p[3], t[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < 3; ++a) {
        float v = xyz[a * n + j];
        const double d = (double)v - g.origin[a];
        p[a] = absolute ? v : (float)d;
        if (!absolute) t[a] = (float)(d - (double)p[a]);
    }
    if (plo) plo[i] = make_float4(t[0], t[1], t[2], 0.f);
    float l[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int q = 0; q < feat_dim && q < 7 && feat; ++q) l[q] = feat[q * n + j];
    if (fx) fx[i] = make_float4(l[3], l[4], l[5], l[6]);
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
    if (h <= 0 && kp.cutoff == 0) {
        // dense mode: no kernel range; a few large voxels hold the cloud
        double ext = 0.0;
        for (int a = 0; a < 3; ++a) ext = std::max(ext, (double)mx[a] - (double)mn[a]);
        h = std::max(ext / 4.0, 1e-3);
    } else if (h <= 0) {
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
    // a target grid keeps a dense per-voxel table: coarsen voxels beyond
    // 2^26 of them
    while (!absolute && prod > (double)(1 << 26)) {
        h *= 1.26;
        g.h = (float)h;
        g.inv_h = (float)(1.0 / h);
        prod = 1.0;
        for (int a = 0; a < 3; ++a) {
            g.dims[a] = (int)std::floor(((double)mx[a] - (double)mn[a]) / h) + 2;
            prod *= g.dims[a];
        }
    }
    if (prod > 4.0e18) return GCVO_ERR_CAPACITY;
    int bits = 1;
    while ((double)(1ull << bits) < prod && bits < 62) ++bits;

    // voxel keys, sorted
    GCVO_TRY(ctx->sort_keys.ensure(n * sizeof(unsigned long long), s));
    GCVO_TRY(ctx->sort_vals.ensure(n * sizeof(int) * 2 + 1024, s));
    GCVO_TRY(ctx->sort_tmp.ensure(radix_sort_scratch_bytes(n), s));
    const int64_t n_vox = absolute ? 0 : (int64_t)prod;
    GCVO_TRY(ctx->scan_tmp.ensure(scan_scratch_bytes(std::max<int64_t>(n, n_vox + 1)) + 1024, s));
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
    if (!absolute) GCVO_TRY(out.plo.ensure(n * sizeof(float4), s));
    const bool with_fx = !absolute && kp.feat_dim > 3;
    if (with_fx) GCVO_TRY(out.fx.ensure(n * sizeof(float4), s));
    GCVO_TRY(out.orig.ensure(n * sizeof(int), s));
    GCVO_TRY(out.cell_start.ensure((n_cells + 1) * sizeof(int), s));
    GCVO_TRY(out.hkeys.ensure(H * sizeof(unsigned long long), s));
    GCVO_TRY(out.hval.ensure(H * sizeof(int), s));
    k_fill_u64<<<(unsigned)((H + 255) / 256), 256, 0, s>>>(out.hkeys.as<unsigned long long>(), (int64_t)H,
                                                          EMPTY_KEY);
    k_cells<<<blocks, 256, 0, s>>>(keys, incl, n, out.cell_start.as<int>(), out.hkeys.as<unsigned long long>(),
                                   out.hval.as<int>(), H - 1);
    k_reorder<<<blocks, 256, 0, s>>>(xyz, kp.kernel_mode == 0 ? cov : nullptr, feat, kp.feat_dim, n, vals, g,
                                     absolute, out.pos.as<float4>(), out.ca.as<float4>(), out.cb.as<float4>(),
                                     absolute ? nullptr : out.plo.as<float4>(), with_fx ? out.fx.as<float4>() : nullptr,
                                     out.orig.as<int>());
    count_launches(3);
    GCVO_CUDA(cudaGetLastError());
    if (!absolute) {
        GCVO_TRY(out.vox_first.ensure((size_t)(n_vox + 1) * sizeof(int), s));
        GCVO_CUDA(cudaMemsetAsync(out.vox_first.ptr, 0, (size_t)(n_vox + 1) * sizeof(int), s));
        k_vox_count<<<blocks, 256, 0, s>>>(keys, n, out.vox_first.as<int>());
        count_launches(1);
        GCVO_CUDA(cudaGetLastError());
        GCVO_TRY(scan_inclusive_sum(out.vox_first.as<int>(), n_vox + 1, ctx->scan_tmp.ptr, s));
    }

    g.pos = out.pos.as<float4>();
    g.ca = out.ca.as<float4>();
    g.cb = out.cb.as<float4>();
    g.plo = absolute ? nullptr : out.plo.as<float4>();
    g.fx = with_fx ? out.fx.as<float4>() : nullptr;
    g.orig = out.orig.as<int>();
    g.cell_start = out.cell_start.as<int>();
    g.hkeys = out.hkeys.as<unsigned long long>();
    g.hval = out.hval.as<int>();
    g.vox_first = absolute ? nullptr : out.vox_first.as<int>();
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

using namespace knn;

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


}  // namespace

void launch_knn_far(const GridDev &fine, const GridDev &coarse, int knn, double eig_max, double eig_ratio, int64_t n,
                    float *cov_out, const int *retry, const int *n_retry, unsigned *status, int blocks,
                    cudaStream_t s);

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
        cell = (kp.cutoff > 0 ? kp.cutoff : 3.0) * std::sqrt(2.0 * kp.eig_max) * 0.5;
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
    // A voxel from the kernel range can hold hundreds of points of a dense
    // cloud, and every query would sort all of them.  The search is exact
    // at any voxel size, so shrink it towards about knn / 2 points per
    // occupied voxel (points on surfaces: the count scales with the square
    // of the edge), at most 16-fold.
    const double occ = (double)n / std::max(1, fine.d.n_cells);
    if (occ > 2.0 * kp.knn) {
        cell *= std::max(1.0 / 16.0, std::sqrt(0.5 * kp.knn / occ));
        GCVO_TRY(build_grid_store(ctx, xyz, nullptr, nullptr, n, q, true, cell, fine));
    }
    GCVO_TRY(build_grid_store(ctx, xyz, nullptr, nullptr, n, q, true, cell * 8.0, coarse));
    GCVO_TRY(ctx->status_word.ensure(256, s));
    GCVO_TRY(ctx->knn_retry.ensure(n * sizeof(int) + 256, s));
    unsigned *stw = ctx->status_word.as<unsigned>();
    int *n_retry = reinterpret_cast<int *>(stw + 1);
    GCVO_CUDA(cudaMemsetAsync(stw, 0, 2 * sizeof(unsigned), s));
    k_knn_cov<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(fine.d, kp.knn, kp.eig_max, kp.eig_ratio, n, cov_out,
                                                          ctx->knn_retry.as<int>(), n_retry);
    launch_knn_far(fine.d, coarse.d, kp.knn, kp.eig_max, kp.eig_ratio, n, cov_out, ctx->knn_retry.as<int>(), n_retry,
                   stw, std::max(1, ctx->sm_count) * 4, s);
    count_launches(2);
    GCVO_CUDA(cudaGetLastError());
    unsigned hs = 0;
    GCVO_CUDA(cudaMemcpyAsync(&hs, stw, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    if (hs & DEV_ERR_CAPACITY) return GCVO_ERR_INVALID_ARG;
    return GCVO_OK;
}

}  // namespace gcvo
