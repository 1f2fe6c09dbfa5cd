// Target voxel grids (gcvo_build_grid and its batched forms): for every
// target cloud X (Eq. 5's x_i with Sigma(x_i; X) and features l_i^X) the
// points sorted by voxel (cz fastest) in a grid-owned packed layout relative
// to the box centre o, with FP32 heads and tails of x - o, and a dense
// per-voxel prefix table over the box that gives the pair kernel the run of
// points of any column of voxels with two loads.
//
// A batch of clouds shares one set of launches: one pass folds every cloud
// into its box and covariance eigenvalue bounds (one read-back for the
// whole batch), every point gets a voxel key offset by the voxel counts of
// the clouds before its own, one sort orders the batch, the reorder writes
// each point into its own grid's arrays and counts its voxel, and one
// segmented scan turns every grid's counts into its prefix table.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace gcvo {
namespace {

constexpr int TG_CHUNK = 4096;          // points per block of the box pass and the key pass
constexpr int TG_BOX = 10;              // ints per cloud: min xyz, max xyz, lam_max, flags, lam_min, pad
constexpr int TG_SCAN_THREADS = 1024;
constexpr int TG_SCAN_ITEMS = 8;
constexpr int TG_TILE = TG_SCAN_THREADS * TG_SCAN_ITEMS;   // voxel-table entries per scan tile

struct TgCloud {
    const float *xyz, *cov, *feat;   // 3 x n, 6 x n (or null), feat_dim x n, device
    int64_t n, off;                  // points; first index in the batch
    int feat_dim;
    int pad;
};

// Where cloud c's grid goes, and its voxel geometry.
struct TgOut {
    float4 *pos, *ca, *cb, *plo, *fx;   // fx null unless more than 3 feature channels
    int *orig, *vox_first;
    unsigned long long key_base;        // offset of its voxel keys in the batch
    double origin[3];
    float corner[3];
    float inv_h;
    int dims[3];
    int pad;
};

__device__ __forceinline__ int tg_enc(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}

__global__ void k_tg_init(int *box, int n_clouds, int *n_cells) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_clouds * TG_BOX) {
        const int k = i % TG_BOX;
        box[i] = k < 3 ? tg_enc(INFINITY) : k < 6 ? tg_enc(-INFINITY) : k == 6 ? tg_enc(0.f)
                 : k == 8 ? tg_enc(INFINITY) : 0;
    }
    if (i < n_clouds) n_cells[i] = 0;
}

// One block per chunk of one cloud: its box, the largest and smallest
// covariance eigenvalues, and flags (1: non-finite input, 2: a covariance
// with a non-positive diagonal entry).
__global__ void k_tg_box(const TgCloud *cl, const int2 *chunks, int with_cov, int *box) {
    const int2 ch = chunks[blockIdx.x];
    const TgCloud c = cl[ch.x];
    const int64_t i0 = (int64_t)ch.y * TG_CHUNK, i1 = min(c.n, i0 + TG_CHUNK);
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    float lmax = 0.f, lmin = INFINITY;
    int bad = 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float v = c.xyz[a * c.n + i];
            if (!isfinite(v)) bad |= 1;
            mn[a] = fminf(mn[a], v);
            mx[a] = fmaxf(mx[a], v);
        }
        for (int q = 0; q < c.feat_dim; ++q)
            if (!isfinite(c.feat[q * c.n + i])) bad |= 1;
        if (with_cov) {
            float s[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                s[q] = c.cov[q * c.n + i];
                if (!isfinite(s[q])) bad |= 1;
            }
            if (s[0] <= 0.f || s[3] <= 0.f || s[5] <= 0.f) bad |= 2;
            lmax = fmaxf(lmax, sym3_max_eig(s[0], s[1], s[2], s[3], s[4], s[5]));
            lmin = fminf(lmin, sym3_min_eig(s[0], s[1], s[2], s[3], s[4], s[5]));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
        lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        lmin = fminf(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        int *b = box + (int64_t)ch.x * TG_BOX;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (mn[a] <= mx[a]) {
                atomicMin(b + a, tg_enc(mn[a]));
                atomicMax(b + 3 + a, tg_enc(mx[a]));
            }
        }
        atomicMax(b + 6, tg_enc(lmax));
        atomicMin(b + 8, tg_enc(lmin));
        if (bad) atomicOr(b + 7, bad);
    }
}

// The voxel of a point of cloud c, in its grid's frame (x - o rounded to
// float, as the grid stores it), clamped to the box.
__device__ __forceinline__ unsigned long long tg_voxel(const TgOut &g, float x, float y, float z) {
    const float v[3] = {x, y, z};
    int q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float cv = (float)((double)v[a] - g.origin[a]);
        const int k = (int)floorf((cv - g.corner[a]) * g.inv_h);
        q[a] = min(max(k, 0), g.dims[a] - 1);
    }
    return ((unsigned long long)q[0] * g.dims[1] + q[1]) * g.dims[2] + q[2];
}

__global__ void k_tg_keys(const TgCloud *cl, const TgOut *go, const int2 *chunks, unsigned long long *keys,
                          int *vals) {
    const int2 ch = chunks[blockIdx.x];
    const TgCloud c = cl[ch.x];
    const TgOut &g = go[ch.x];
    const int64_t i0 = (int64_t)ch.y * TG_CHUNK, i1 = min(c.n, i0 + TG_CHUNK);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        keys[c.off + i] = g.key_base + tg_voxel(g, c.xyz[i], c.xyz[c.n + i], c.xyz[2 * c.n + i]);
        vals[c.off + i] = (int)(c.off + i);
    }
}

// Sorted point i: into its grid's arrays at i - off (the clouds occupy
// consecutive ranges of the sort, in batch order), its voxel counted one
// slot up in the grid's prefix table, and the first point of every voxel
// counted as an occupied voxel.
__global__ void k_tg_reorder(const TgCloud *cl, const TgOut *go, int n_clouds, const unsigned long long *keys,
                             const int *vals, int64_t N, int *n_cells) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int j = vals[i];
    int lo = 0, hi = n_clouds - 1;   // the cloud of j: the last with off <= j
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cl[mid].off <= j) lo = mid;
        else hi = mid - 1;
    }
    const TgCloud c = cl[lo];
    const TgOut &g = go[lo];
    const int64_t l = j - c.off, o = i - c.off;
    float p[3], t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double d = (double)c.xyz[a * c.n + l] - g.origin[a];
        p[a] = (float)d;
        t[a] = (float)(d - (double)p[a]);
    }
    float f[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int q = 0; q < c.feat_dim && q < 7; ++q) f[q] = c.feat[q * c.n + l];
    float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (c.cov)
#pragma unroll
        for (int q = 0; q < 6; ++q) s[q] = c.cov[q * c.n + l];
    g.pos[o] = make_float4(p[0], p[1], p[2], f[0]);
    g.ca[o] = make_float4(s[0], s[1], s[2], s[3]);
    g.cb[o] = make_float4(s[4], s[5], f[1], f[2]);
    g.plo[o] = make_float4(t[0], t[1], t[2], 0.f);
    if (g.fx) g.fx[o] = make_float4(f[3], f[4], f[5], f[6]);
    g.orig[o] = (int)l;
    const unsigned long long k = keys[i];
    atomicAdd(g.vox_first + (k - g.key_base) + 1, 1);
    if (o == 0 || keys[i - 1] != k) atomicAdd(n_cells + lo, 1);
}

// tiles[t] = (cloud, first entry of the tile in that cloud's prefix table);
// table lengths are n_vox + 1.
__global__ void k_tg_zero(const TgOut *go, const int2 *tiles, const int64_t *len) {
    const int2 tl = tiles[blockIdx.x];
    int *v = go[tl.x].vox_first;
    const int64_t e1 = min(len[tl.x], (int64_t)tl.y + TG_TILE);
    for (int64_t e = tl.y + threadIdx.x; e < e1; e += blockDim.x) v[e] = 0;
}

__device__ __forceinline__ int tg_block_incl(int v, int *warp_tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    return wid > 0 ? v + warp_tot[wid - 1] : v;
}

// Sum of each tile.
__global__ void __launch_bounds__(TG_SCAN_THREADS)
    k_tg_tile_sum(const TgOut *go, const int2 *tiles, const int64_t *len, int *tsum) {
    __shared__ int red[TG_SCAN_THREADS / 32];
    const int2 tl = tiles[blockIdx.x];
    const int *v = go[tl.x].vox_first;
    const int64_t e1 = min(len[tl.x], (int64_t)tl.y + TG_TILE);
    int acc = 0;
    for (int64_t e = tl.y + threadIdx.x; e < e1; e += blockDim.x) acc += v[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < TG_SCAN_THREADS / 32; ++w) s += red[w];
        tsum[blockIdx.x] = s;
    }
}

// One thread per cloud: exclusive offsets of its tiles (in place).
__global__ void k_tg_tile_off(const int64_t *tile0, int n_clouds, int *tsum) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_clouds) return;
    int acc = 0;
    for (int64_t t = tile0[c]; t < tile0[c + 1]; ++t) {
        const int v = tsum[t];
        tsum[t] = acc;
        acc += v;
    }
}

// Inclusive scan of each tile plus its offset, in place.
__global__ void __launch_bounds__(TG_SCAN_THREADS)
    k_tg_tile_scan(const TgOut *go, const int2 *tiles, const int64_t *len, const int *toff) {
    __shared__ int warp_tot[32];
    const int2 tl = tiles[blockIdx.x];
    int *v = go[tl.x].vox_first;
    const int64_t n = len[tl.x];
    const int64_t base = (int64_t)tl.y + (int64_t)threadIdx.x * TG_SCAN_ITEMS;
    int x[TG_SCAN_ITEMS];
    int acc = 0;
#pragma unroll
    for (int k = 0; k < TG_SCAN_ITEMS; ++k) {
        x[k] = base + k < n ? v[base + k] : 0;
        acc += x[k];
        x[k] = acc;
    }
    const int incl = tg_block_incl(acc, warp_tot);
    const int pre = incl - acc + toff[blockIdx.x];
#pragma unroll
    for (int k = 0; k < TG_SCAN_ITEMS; ++k)
        if (base + k < n) v[base + k] = pre + x[k];
}

}  // namespace

size_t tgrid_meta_bytes(int n_clouds, int64_t n_points) {
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t C = (size_t)std::max(n_clouds, 1);
    const size_t chunks = (size_t)(n_points / TG_CHUNK) + C;
    return al(C * sizeof(TgCloud)) + al(C * sizeof(TgOut)) + al(C * TG_BOX * sizeof(int)) + al(C * sizeof(int)) +
           2 * al((C + 1) * sizeof(int64_t)) + al(chunks * sizeof(int2));
}

size_t tgrid_tile_bytes(int64_t n_tiles) {
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al((size_t)std::max<int64_t>(n_tiles, 1) * sizeof(int2)) + al((size_t)std::max<int64_t>(n_tiles, 1) * sizeof(int));
}

int64_t tgrid_max_tiles(int n_clouds) {
    // a grid keeps at most 2^26 voxels (plus the end entry)
    return (int64_t)std::max(n_clouds, 1) * ((((int64_t)1 << 26) + 1 + TG_TILE - 1) / TG_TILE);
}

gcvo_status build_target_grids(gcvo_ctx *ctx, int n_clouds, const TgJob *jobs) {
    cudaStream_t s = ctx->stream;
    const int C = n_clouds;
    if (C < 1) return GCVO_ERR_INVALID_ARG;
    const int mode = jobs[0].kp->kernel_mode, fd = jobs[0].kp->feat_dim;
    std::vector<TgCloud> cl(C);
    std::vector<int2> chunks;
    int64_t N = 0;
    for (int c = 0; c < C; ++c) {
        const TgJob &j = jobs[c];
        if (j.kp->kernel_mode != mode || j.kp->feat_dim != fd) return GCVO_ERR_INVALID_ARG;
        if (j.n < 1 || j.n > ((int64_t)1 << 28)) return GCVO_ERR_INVALID_ARG;
        cl[c] = TgCloud{j.xyz, mode == 0 ? j.cov : nullptr, j.feat, j.n, N, fd, 0};
        for (int64_t q = 0; q * TG_CHUNK < j.n; ++q) chunks.push_back(make_int2(c, (int)q));
        N += j.n;
    }
    if (N >= ((int64_t)1 << 30)) return GCVO_ERR_CAPACITY;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };

    // ---- boxes and eigenvalue bounds (one read-back for the batch)
    GCVO_TRY(ctx->grid_meta.ensure(tgrid_meta_bytes(C, N), s));
    char *m = static_cast<char *>(ctx->grid_meta.ptr);
    auto *d_cl = reinterpret_cast<TgCloud *>(m);
    m += al(C * sizeof(TgCloud));
    auto *d_go = reinterpret_cast<TgOut *>(m);
    m += al(C * sizeof(TgOut));
    int *d_box = reinterpret_cast<int *>(m);
    m += al((size_t)C * TG_BOX * sizeof(int));
    int *d_ncell = reinterpret_cast<int *>(m);
    m += al(C * sizeof(int));
    auto *d_len = reinterpret_cast<int64_t *>(m);
    m += al((C + 1) * sizeof(int64_t));
    auto *d_tile0 = reinterpret_cast<int64_t *>(m);
    m += al((C + 1) * sizeof(int64_t));
    auto *d_chunks = reinterpret_cast<int2 *>(m);
    GCVO_CUDA(cudaMemcpyAsync(d_cl, cl.data(), C * sizeof(TgCloud), cudaMemcpyHostToDevice, s));
    GCVO_CUDA(cudaMemcpyAsync(d_chunks, chunks.data(), chunks.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    k_tg_init<<<(unsigned)((C * TG_BOX + 255) / 256), 256, 0, s>>>(d_box, C, d_ncell);
    k_tg_box<<<(unsigned)chunks.size(), 256, 0, s>>>(d_cl, d_chunks, mode == 0 ? 1 : 0, d_box);
    count_launches(2);
    GCVO_CUDA(cudaGetLastError());
    std::vector<int> hb((size_t)C * TG_BOX);
    GCVO_CUDA(cudaMemcpyAsync(hb.data(), d_box, hb.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    auto dec = [](int k) {
        const int i = k >= 0 ? k : k ^ 0x7fffffff;
        float f;
        memcpy(&f, &i, 4);
        return f;
    };

    // ---- per grid: voxel edge, box, storage
    std::vector<TgOut> go(C);
    std::vector<GridDev> gd(C);
    std::vector<int64_t> len(C + 1, 0), tile0(C + 1, 0);
    std::vector<int2> tiles;
    unsigned long long key_base = 0;
    for (int c = 0; c < C; ++c) {
        const TgJob &j = jobs[c];
        const gcvo_kernel_params &kp = *j.kp;
        const int *b = &hb[(size_t)c * TG_BOX];
        if (b[7] & 1) return GCVO_ERR_NONFINITE;
        if ((b[7] & 2) && mode == 0) return GCVO_ERR_INVALID_ARG;
        float mn[3], mx[3];
        for (int a = 0; a < 3; ++a) {
            mn[a] = dec(b[a]);
            mx[a] = dec(b[3 + a]);
        }
        const float lam = dec(b[6]);
        double h = kp.cell_size;
        if (h <= 0 && kp.cutoff == 0) {
            // dense mode: no kernel range; a few large voxels hold the cloud
            double ext = 0.0;
            for (int a = 0; a < 3; ++a) ext = std::max(ext, (double)mx[a] - (double)mn[a]);
            h = std::max(ext / 4.0, 1e-3);
        } else if (h <= 0) {
            // half the kernel range: finer voxels hug the range ball more tightly
            h = mode == 1 ? 0.5 * kp.cutoff * kp.iso_ell : 0.5 * kp.cutoff * std::sqrt(2.0 * (double)lam);
        }
        if (!(h > 0) || !std::isfinite(h)) return GCVO_ERR_INVALID_ARG;
        GridDev g{};
        TgOut o{};
        double prod = 1.0;
        for (int a = 0; a < 3; ++a) {
            g.origin[a] = 0.5 * ((double)mn[a] + (double)mx[a]);
            g.corner[a] = (float)((double)mn[a] - g.origin[a]);
            const double ext = ((double)mx[a] - (double)mn[a]) / h;
            if (ext > 1.0e9) return GCVO_ERR_CAPACITY;
            g.dims[a] = (int)std::floor(ext) + 2;
            prod *= g.dims[a];
        }
        // the dense per-voxel table: coarsen voxels beyond 2^26 of them
        while (prod > (double)(1 << 26)) {
            h *= 1.26;
            prod = 1.0;
            for (int a = 0; a < 3; ++a) {
                g.dims[a] = (int)std::floor(((double)mx[a] - (double)mn[a]) / h) + 2;
                prod *= g.dims[a];
            }
        }
        g.h = (float)h;
        g.inv_h = (float)(1.0 / h);
        g.feat_dim = fd;
        g.kernel_mode = mode;
        g.lam_max = lam;
        g.lam_min = mode == 0 ? std::max(0.0f, dec(b[8])) : 0.0f;
        const int64_t n = j.n, n_vox = (int64_t)prod;
        GridStore &st = j.grid->store;
        GCVO_TRY(st.pos.ensure(n * sizeof(float4), s));
        GCVO_TRY(st.ca.ensure(n * sizeof(float4), s));
        GCVO_TRY(st.cb.ensure(n * sizeof(float4), s));
        GCVO_TRY(st.plo.ensure(n * sizeof(float4), s));
        if (fd > 3) GCVO_TRY(st.fx.ensure(n * sizeof(float4), s));
        GCVO_TRY(st.orig.ensure(n * sizeof(int), s));
        GCVO_TRY(st.vox_first.ensure((size_t)(n_vox + 1) * sizeof(int), s));
        g.pos = o.pos = st.pos.as<float4>();
        g.ca = o.ca = st.ca.as<float4>();
        g.cb = o.cb = st.cb.as<float4>();
        g.plo = o.plo = st.plo.as<float4>();
        g.fx = o.fx = fd > 3 ? st.fx.as<float4>() : nullptr;
        g.orig = o.orig = st.orig.as<int>();
        g.vox_first = o.vox_first = st.vox_first.as<int>();
        g.n = (int)n;
        for (int a = 0; a < 3; ++a) {
            o.origin[a] = g.origin[a];
            o.corner[a] = g.corner[a];
            o.dims[a] = g.dims[a];
        }
        o.inv_h = g.inv_h;
        o.key_base = key_base;
        key_base += (unsigned long long)n_vox;
        len[c] = n_vox + 1;
        tile0[c] = (int64_t)tiles.size();
        for (int64_t e = 0; e < n_vox + 1; e += TG_TILE) tiles.push_back(make_int2(c, (int)e));
        go[c] = o;
        gd[c] = g;
    }
    tile0[C] = (int64_t)tiles.size();
    const int64_t T = (int64_t)tiles.size();
    GCVO_TRY(ctx->grid_tiles.ensure(tgrid_tile_bytes(T), s));
    auto *d_tiles = ctx->grid_tiles.as<int2>();
    int *d_tsum = reinterpret_cast<int *>(ctx->grid_tiles.as<char>() + al((size_t)T * sizeof(int2)));
    int bits = 1;
    while (bits < 62 && (1ull << bits) < key_base) ++bits;

    // ---- keys, sort, reorder, voxel tables
    GCVO_TRY(ctx->sort_keys.ensure(N * sizeof(unsigned long long), s));
    GCVO_TRY(ctx->sort_vals.ensure(N * sizeof(int) * 2 + 1024, s));
    GCVO_TRY(ctx->sort_tmp.ensure(radix_sort_scratch_bytes(N), s));
    auto *keys = ctx->sort_keys.as<unsigned long long>();
    int *vals = ctx->sort_vals.as<int>();
    GCVO_CUDA(cudaMemcpyAsync(d_go, go.data(), C * sizeof(TgOut), cudaMemcpyHostToDevice, s));
    GCVO_CUDA(cudaMemcpyAsync(d_len, len.data(), (C + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    GCVO_CUDA(cudaMemcpyAsync(d_tile0, tile0.data(), (C + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    GCVO_CUDA(cudaMemcpyAsync(d_tiles, tiles.data(), T * sizeof(int2), cudaMemcpyHostToDevice, s));
    k_tg_zero<<<(unsigned)T, 256, 0, s>>>(d_go, d_tiles, d_len);
    k_tg_keys<<<(unsigned)chunks.size(), 256, 0, s>>>(d_cl, d_go, d_chunks, keys, vals);
    count_launches(2);
    GCVO_CUDA(cudaGetLastError());
    GCVO_TRY(radix_sort_pairs(keys, vals, N, bits, ctx->sort_tmp.ptr, ctx->sort_tmp.bytes, s));
    k_tg_reorder<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(d_cl, d_go, C, keys, vals, N, d_ncell);
    k_tg_tile_sum<<<(unsigned)T, TG_SCAN_THREADS, 0, s>>>(d_go, d_tiles, d_len, d_tsum);
    k_tg_tile_off<<<(unsigned)((C + 127) / 128), 128, 0, s>>>(d_tile0, C, d_tsum);
    k_tg_tile_scan<<<(unsigned)T, TG_SCAN_THREADS, 0, s>>>(d_go, d_tiles, d_len, d_tsum);
    count_launches(4);
    GCVO_CUDA(cudaGetLastError());
    std::vector<int> ncell(C);
    GCVO_CUDA(cudaMemcpyAsync(ncell.data(), d_ncell, C * sizeof(int), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < C; ++c) {
        gd[c].n_cells = ncell[c];
        jobs[c].grid->store.d = gd[c];
        jobs[c].grid->kp = *jobs[c].kp;
    }
    return GCVO_OK;
}

}  // namespace gcvo
