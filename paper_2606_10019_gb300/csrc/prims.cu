// Device primitives used by the grid builder and the source grouping:
// a stable LSD radix sort of (key, value) pairs, inclusive scans, and a
// bounding-box / largest-eigenvalue reduction.
#include <atomic>
#include <cstdio>
#include <cstring>

#include "common.cuh"

namespace gcvo {

static thread_local char g_last_err[256];
static std::atomic<long long> g_launches{0};
static std::atomic<long long> g_allocs{0};

void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
long long device_allocs_so_far() { return g_allocs.load(std::memory_order_relaxed); }

const char *last_cuda_error() { return g_last_err; }

void set_last_cuda_error(cudaError_t e, const char *what, int line) {
    snprintf(g_last_err, sizeof(g_last_err), "%s (%d) at line %d: %s", cudaGetErrorString(e), (int)e, line, what);
}

gcvo_status DevBuf::ensure(size_t need, cudaStream_t s) {
    if (need <= bytes && ptr) return GCVO_OK;
    if (fixed) return GCVO_ERR_WORKSPACE;   // a workspace slice never grows
    if (ptr) {
        GCVO_CUDA(cudaStreamSynchronize(s));
        GCVO_CUDA(cudaFree(ptr));
        ptr = nullptr;
        bytes = 0;
    }
    size_t b = need < 256 ? 256 : need;
    b = (b + 255) & ~size_t(255);
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    if (cudaMalloc(&ptr, b) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
        return GCVO_ERR_WORKSPACE;
    }
    bytes = b;
    return GCVO_OK;
}

void DevBuf::release() {
    if (ptr && !fixed) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
    fixed = false;
}

// ---------------------------------------------------------------------------
// Inclusive scans (sum / max) of int arrays: tiles of 4096 items are reduced,
// the tile totals are scanned by one block, then each tile is scanned with
// its offset.  n <= 4096 * 4096.
// ---------------------------------------------------------------------------
namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

struct OpSum {
    __device__ static int id() { return 0; }
    __device__ static int op(int a, int b) { return a + b; }
};
struct OpMax {
    __device__ static int id() { return INT_MIN; }
    __device__ static int op(int a, int b) { return a > b ? a : b; }
};

// Inclusive block scan of one value per thread; returns the block total too.
template <class Op>
__device__ int block_scan_incl(int v, int *total) {
    __shared__ int warp_tot[32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v = Op::op(u, v);
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    if (wid == 0) {
        int w = lane < nw ? warp_tot[lane] : Op::id();
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w = Op::op(u, w);
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    if (wid > 0) v = Op::op(warp_tot[wid - 1], v);
    *total = warp_tot[nw - 1];
    __syncthreads();
    return v;
}

template <class Op>
__global__ void scan_tile_reduce(const int *data, int64_t n, int *tile_tot) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v = Op::id();
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) v = Op::op(v, data[base + k]);
    int tot;
    block_scan_incl<Op>(v, &tot);
    if (threadIdx.x == 0) tile_tot[blockIdx.x] = tot;
}

// Scans `data` (n items) in place with an optional per-tile offset array
// (exclusive offsets derived from the inclusive scan of tile totals).
template <class Op>
__global__ void scan_tiles(int *data, int64_t n, const int *tile_incl) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int acc = Op::id();
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < n ? data[base + k] : Op::id();
        acc = Op::op(acc, v[k]);
        v[k] = acc;
    }
    int tot;
    int incl = block_scan_incl<Op>(acc, &tot);
    // exclusive prefix of this thread within the tile
    int excl = __shfl_up_sync(0xffffffffu, incl, 1);
    __shared__ int warp_last[32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 31) warp_last[wid] = incl;
    __syncthreads();
    if (lane == 0) excl = wid > 0 ? warp_last[wid - 1] : Op::id();
    int off = (tile_incl && blockIdx.x > 0) ? tile_incl[blockIdx.x - 1] : Op::id();
    int pre = Op::op(off, excl);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) data[base + k] = Op::op(pre, v[k]);
}

template <class Op>
gcvo_status scan_impl(int *data, int64_t n, void *scratch, cudaStream_t s) {
    if (n <= 0) return GCVO_OK;
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles > SCAN_TILE) return GCVO_ERR_CAPACITY;
    if (tiles == 1) {
        scan_tiles<Op><<<1, SCAN_THREADS, 0, s>>>(data, n, nullptr);
        count_launches(1);
        GCVO_CUDA(cudaGetLastError());
        return GCVO_OK;
    }
    int *tot = static_cast<int *>(scratch);
    scan_tile_reduce<Op><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(data, n, tot);
    scan_tiles<Op><<<1, SCAN_THREADS, 0, s>>>(tot, tiles, nullptr);
    scan_tiles<Op><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(data, n, tot);
    count_launches(3);
    GCVO_CUDA(cudaGetLastError());
    return GCVO_OK;
}

}  // namespace

size_t scan_scratch_bytes(int64_t n) { return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE + 1) * sizeof(int); }

gcvo_status scan_inclusive_sum(int *data, int64_t n, void *scratch, cudaStream_t s) {
    return scan_impl<OpSum>(data, n, scratch, s);
}
gcvo_status scan_inclusive_max(int *data, int64_t n, void *scratch, cudaStream_t s) {
    return scan_impl<OpMax>(data, n, scratch, s);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8 bits per pass.  Each warp owns a tile of
// RS_ITEMS * 32 consecutive items; per pass: digit histogram per tile
// (digit-major layout), one inclusive scan over all (digit, tile) counts,
// then a scatter in which each warp walks its tile in order, ranking equal
// digits with __match_any_sync so that the order of equal keys is kept.
// ---------------------------------------------------------------------------
namespace {

constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = 32 * RS_ITEMS;
constexpr int RS_WARPS = 8;

__global__ void rs_hist(const unsigned long long *keys, int64_t n, int shift, int n_tiles, int *hist) {
    __shared__ int cnt[RS_WARPS][256];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = lane; d < 256; d += 32) cnt[w][d] = 0;
    __syncwarp();
    int tile = blockIdx.x * RS_WARPS + w;
    if (tile < n_tiles) {
        int64_t base = (int64_t)tile * RS_TILE;
        for (int it = 0; it < RS_ITEMS; ++it) {
            int64_t i = base + it * 32 + lane;
            if (i < n) atomicAdd(&cnt[w][(int)((keys[i] >> shift) & 255ull)], 1);
        }
        __syncwarp();
        for (int d = lane; d < 256; d += 32) hist[(int64_t)d * n_tiles + tile] = cnt[w][d];
    }
}

__global__ void rs_scatter(const unsigned long long *keys_in, const int *vals_in, unsigned long long *keys_out,
                           int *vals_out, int64_t n, int shift, int n_tiles, const int *hist, const int *incl) {
    __shared__ int run[RS_WARPS][256];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int tile = blockIdx.x * RS_WARPS + w;
    if (tile >= n_tiles) return;
    for (int d = lane; d < 256; d += 32) {
        int64_t q = (int64_t)d * n_tiles + tile;
        run[w][d] = incl[q] - hist[q];
    }
    __syncwarp();
    int64_t base = (int64_t)tile * RS_TILE;
    unsigned lt = (1u << lane) - 1u;
    for (int it = 0; it < RS_ITEMS; ++it) {
        int64_t i = base + it * 32 + lane;
        bool valid = i < n;
        unsigned long long k = valid ? keys_in[i] : 0ull;
        int d = valid ? (int)((k >> shift) & 255ull) : 256 + lane;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        int rank = __popc(peers & lt);
        int b = 0;
        if (valid && lane == leader) {
            b = run[w][d];
            run[w][d] = b + __popc(peers);
        }
        b = __shfl_sync(0xffffffffu, b, leader);
        if (valid) {
            keys_out[b + rank] = k;
            vals_out[b + rank] = vals_in[i];
        }
        __syncwarp();
    }
}

}  // namespace

size_t radix_sort_scratch_bytes(int64_t n) {
    int64_t tiles = (n + RS_TILE - 1) / RS_TILE;
    size_t h = (size_t)tiles * 256 * sizeof(int);
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al(n * sizeof(unsigned long long)) + al(n * sizeof(int)) + 2 * al(h) + al(scan_scratch_bytes(tiles * 256));
}

gcvo_status radix_sort_pairs(unsigned long long *keys, int *vals, int64_t n, int bits, void *scratch,
                             size_t scratch_bytes, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return GCVO_OK;
    if (scratch_bytes < radix_sort_scratch_bytes(n)) return GCVO_ERR_WORKSPACE;
    int n_tiles = (int)((n + RS_TILE - 1) / RS_TILE);
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    char *p = static_cast<char *>(scratch);
    auto *k2 = reinterpret_cast<unsigned long long *>(p);
    p += al(n * sizeof(unsigned long long));
    int *v2 = reinterpret_cast<int *>(p);
    p += al(n * sizeof(int));
    int *hist = reinterpret_cast<int *>(p);
    p += al((size_t)n_tiles * 256 * sizeof(int));
    int *incl = reinterpret_cast<int *>(p);
    p += al((size_t)n_tiles * 256 * sizeof(int));
    void *sc = p;
    unsigned long long *ka = keys, *kb = k2;
    int *va = vals, *vb = v2;
    int passes = (bits + 7) / 8;
    unsigned grid = (unsigned)((n_tiles + RS_WARPS - 1) / RS_WARPS);
    for (int ps = 0; ps < passes; ++ps) {
        int shift = 8 * ps;
        rs_hist<<<grid, RS_WARPS * 32, 0, s>>>(ka, n, shift, n_tiles, hist);
        GCVO_CUDA(cudaMemcpyAsync(incl, hist, (size_t)n_tiles * 256 * sizeof(int), cudaMemcpyDeviceToDevice, s));
        GCVO_TRY(scan_inclusive_sum(incl, (int64_t)n_tiles * 256, sc, s));
        rs_scatter<<<grid, RS_WARPS * 32, 0, s>>>(ka, va, kb, vb, n, shift, n_tiles, hist, incl);
        count_launches(2);
        GCVO_CUDA(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        GCVO_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
        GCVO_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    }
    return GCVO_OK;
}

}  // namespace gcvo
