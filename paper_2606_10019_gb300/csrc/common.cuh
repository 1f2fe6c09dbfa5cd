// Internal declarations shared by the translation units of libgcvo.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstddef>
#include <utility>
#include <vector>

#include "gcvo.h"

namespace gcvo {

// ---------------------------------------------------------------------------
// Error handling: every CUDA call is checked; the first failure is turned into
// a gcvo_status that the C ABI returns.
// ---------------------------------------------------------------------------
#define GCVO_CUDA(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) {                          \
            gcvo::set_last_cuda_error(e_, #call, __LINE__); \
            return GCVO_ERR_CUDA;                         \
        }                                                 \
    } while (0)

#define GCVO_TRY(expr)                                    \
    do {                                                  \
        gcvo_status s_ = (expr);                          \
        if (s_ != GCVO_OK) return s_;                     \
    } while (0)

void set_last_cuda_error(cudaError_t e, const char *what, int line);
const char *last_cuda_error();

// Process-wide count of kernels launched by the library, and of the device
// allocations (cudaMalloc) it made (profiling).
void count_launches(long long n);
long long launches_so_far();
long long device_allocs_so_far();

// Device status word bits (set by kernels with atomicOr, read by the host).
enum : unsigned {
    DEV_ERR_TIMEOUT = 1u,
    DEV_ERR_CAPACITY = 2u,
    DEV_ERR_NONFINITE = 4u,
};

// ---------------------------------------------------------------------------
// A device buffer that only grows (released by the owner's destroy call), or,
// when `fixed`, a slice of a caller-owned workspace that never grows: a need
// beyond it is GCVO_ERR_WORKSPACE and release() forgets it without freeing.
// ---------------------------------------------------------------------------
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    bool fixed = false;
    gcvo_status ensure(size_t need, cudaStream_t s);
    void release();
    template <class T> T *as() const { return static_cast<T *>(ptr); }
};

// ---------------------------------------------------------------------------
// What the kernels see of a target grid (plain data, passed by value or read
// from device memory).
//
// Points are sorted by voxel key.  pos[i] = (x - o, y - o, z - o, l0) for the
// target grid (coordinates relative to the grid origin o, float32), and the
// absolute coordinates for the internal kNN grid; ca[i] = (S00, S01, S02, S11),
// cb[i] = (S12, S22, l1, l2).  Target grids also keep the rounding tails of
// the coordinates, plo[i] = (x - o) - pos[i].xyz (float), so that x - o =
// pos + plo to about 2^-48 relative.  Voxel (cx, cy, cz) holds the points whose
// coordinates c satisfy floor((c - corner) * inv_h) = (cx, cy, cz); its key is
// (cx * ny + cy) * nz + cz, so the voxels of one (cx, cy) column with
// consecutive cz are consecutive in the sorted order.
// ---------------------------------------------------------------------------
struct GridDev {
    const float4 *pos;
    const float4 *ca;
    const float4 *cb;
    const float4 *plo;        // target grids: coordinate tails (x, y, z, 0)
    const float4 *fx;         // feature channels 3..6 (when feat_dim > 3)
    const int *orig;          // original index of each sorted point
    const int *cell_start;    // n_cells + 1 offsets into the sorted points
    const unsigned long long *hkeys;  // open-addressing table of voxel keys
    const int *hval;          // voxel index of each table slot
    const int *vox_first;     // target grids: first sorted point of every voxel, dense (+1 entry)
    unsigned long long hmask; // table size - 1 (power of two)
    unsigned long long key_base;   // batched kNN grids: offset of this cloud's voxel keys (0 otherwise)
    double origin[3];         // o (target grid) or 0 (kNN grid), double
    float corner[3];          // lowest voxel corner, in the coordinates of pos
    float h, inv_h;
    int dims[3];
    int n, n_cells;
    float lam_max;            // largest eigenvalue over the stored covariances
    float lam_min;            // smallest (target grids with covariances; else 0)
    int feat_dim;
    int kernel_mode;
};

static constexpr unsigned long long EMPTY_KEY = ~0ull;

__host__ __device__ inline unsigned long long hash_key(unsigned long long k) {
    // splitmix64 finaliser
    k ^= k >> 30;
    k *= 0xbf58476d1ce4e5b9ull;
    k ^= k >> 27;
    k *= 0x94d049bb133111ebull;
    k ^= k >> 31;
    return k;
}

// Voxel index of `key`, or -1 when the voxel holds no point.
__device__ inline int grid_lookup(const GridDev &g, unsigned long long key) {
    unsigned long long s = hash_key(key) & g.hmask;
    for (int probe = 0; probe <= (int)g.hmask; ++probe) {
        unsigned long long k = __ldg(g.hkeys + s);
        if (k == key) return __ldg(g.hval + s);
        if (k == EMPTY_KEY) return -1;
        s = (s + 1) & g.hmask;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// Primitives (prims.cu).
// ---------------------------------------------------------------------------

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of key.
// Scratch: radix_sort_scratch_bytes(n) bytes.
size_t radix_sort_scratch_bytes(int64_t n);
gcvo_status radix_sort_pairs(unsigned long long *keys, int *vals, int64_t n, int bits, void *scratch,
                             size_t scratch_bytes, cudaStream_t s);

// In-place inclusive scans of int arrays (sum or max).
size_t scan_scratch_bytes(int64_t n);
gcvo_status scan_inclusive_sum(int *data, int64_t n, void *scratch, cudaStream_t s);
gcvo_status scan_inclusive_max(int *data, int64_t n, void *scratch, cudaStream_t s);

// Largest eigenvalue of a symmetric 3x3 (closed form, float).
__host__ __device__ inline float sym3_max_eig(float a00, float a01, float a02, float a11, float a12, float a22) {
    float p1 = a01 * a01 + a02 * a02 + a12 * a12;
    float q = (a00 + a11 + a22) * (1.0f / 3.0f);
    float b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    float p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0f * p1;
    if (p2 <= 0.0f) return q;
    float p = sqrtf(p2 * (1.0f / 6.0f));
    float ip = 1.0f / p;
    b00 *= ip; b11 *= ip; b22 *= ip;
    float c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
    float detb = b00 * (b11 * b22 - c12 * c12) - c01 * (c01 * b22 - c12 * c02) + c02 * (c01 * c12 - b11 * c02);
    float r = fminf(fmaxf(0.5f * detb, -1.0f), 1.0f);
    float phi = acosf(r) * (1.0f / 3.0f);
    return q + 2.0f * p * cosf(phi);
}

// Smallest eigenvalue of a symmetric 3x3 (the same closed form, third root).
__host__ __device__ inline float sym3_min_eig(float a00, float a01, float a02, float a11, float a12, float a22) {
    float p1 = a01 * a01 + a02 * a02 + a12 * a12;
    float q = (a00 + a11 + a22) * (1.0f / 3.0f);
    float b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    float p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0f * p1;
    if (p2 <= 0.0f) return q;
    float p = sqrtf(p2 * (1.0f / 6.0f));
    float ip = 1.0f / p;
    b00 *= ip; b11 *= ip; b22 *= ip;
    float c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
    float detb = b00 * (b11 * b22 - c12 * c12) - c01 * (c01 * b22 - c12 * c02) + c02 * (c01 * c12 - b11 * c02);
    float r = fminf(fmaxf(0.5f * detb, -1.0f), 1.0f);
    float phi = acosf(r) * (1.0f / 3.0f);
    return q + 2.0f * p * cosf(phi + 2.0943951023931953f);   // the third root, phi + 2 pi / 3
}

// ---------------------------------------------------------------------------
// Grids (grid.cu).
// ---------------------------------------------------------------------------
struct GridStore {
    GridDev d{};
    DevBuf pos, ca, cb, plo, fx, orig, cell_start, hkeys, hval, vox_first;
};

// Target grids of a batch of clouds in one set of launches (tgrid.cu):
// cloud k (device SoA xyz, cov (null in kernel mode 1), feat; n points)
// into grid k with its kernel parameters kp (the same kernel mode and
// feature count for all).  The voxel edge is kp->cell_size, or half the
// kernel range when that is <= 0.
struct TgJob {
    const float *xyz, *cov, *feat;
    int64_t n;
    const gcvo_kernel_params *kp;
    gcvo_grid *grid;
};
gcvo_status build_target_grids(gcvo_ctx *ctx, int n_clouds, const TgJob *jobs);
size_t tgrid_meta_bytes(int n_clouds, int64_t n_points);
size_t tgrid_tile_bytes(int64_t n_tiles);
int64_t tgrid_max_tiles(int n_clouds);

// kNN covariances of a batch of clouds in one set of launches: cloud k has
// n[k] points at xyz[k] (3 x n SoA, device) and its own parameters kp[k];
// Sigma goes to cov[k] (6 x n SoA, device).
struct KnnJob {
    const float *xyz;
    float *cov;
    int64_t n;
    const gcvo_kernel_params *kp;
};
gcvo_status knn_covariances(gcvo_ctx *ctx, int n_clouds, const KnnJob *jobs);
size_t knn_meta_bytes(int64_t n_points, int n_clouds);

}  // namespace gcvo

// ---------------------------------------------------------------------------
// The opaque handles of the C ABI.
// ---------------------------------------------------------------------------
struct gcvo_grid {
    gcvo::GridStore store;
    gcvo_kernel_params kp;
    int device;   // the grid outlives nothing but its own memory: no context pointer
};

struct gcvo_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    // scratch
    gcvo::DevBuf sort_keys, sort_vals, sort_tmp, scan_tmp, small;
    gcvo::DevBuf stage_xyz, stage_cov, stage_feat;   // host-input staging
    gcvo::DevBuf src_pos, src_ca, src_cb, pprob;     // packed sources (sorted) and their problems
    gcvo::DevBuf src_fx;                             // their feature channels 3..6 (feat_dim > 3)
    gcvo::DevBuf t_pos, t_ca, t_cb, t_lo, t_fx;      // the same at the current pose (k_transform)
    gcvo::DevBuf partial, probs, grids, logs, evalout, status_word, items, item_prob, pack_tmp;
    gcvo::DevBuf partial2;                           // second partial row of the G-CVO-E pass
    gcvo::GridStore knn_grid, knn_grid2;             // reused by gcvo_estimate_covariances
    gcvo::DevBuf knn_meta;                           // its per-cloud descriptors and grids
    gcvo::DevBuf grid_meta, grid_tiles;              // target-grid builds: per-cloud data, scan tiles
    // gcvo_register_clouds: staged host clouds, covariances and target grids
    gcvo::DevBuf clouds_stage, clouds_cov;
    std::vector<gcvo_grid *> clouds_grids;
    gcvo::DevBuf knn_retry;
    void *host_pinned = nullptr;
    size_t host_pinned_bytes = 0;
    int sm_count = 0;
    // profiling: CUDA events around pair-kernel launches
    int profiling = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_kind;   // per event pair: 0 pair pass, 1 finalize, 2 transform
    size_t ev_used = 0;
    long long launch_base = 0;
    long long alloc_base = 0;
    long long pair_launches = 0;
    double pair_ms = 0.0;
    long long fin_launches = 0;
    double fin_ms = 0.0, transform_ms = 0.0;
    double clouds_cov_ms = 0.0, clouds_grid_ms = 0.0;   // gcvo_register_clouds phases
    cudaStream_t cap_stream = nullptr;   // private stream for graph capture
    // caller-owned workspace (gcvo_set_workspace): null when the library
    // allocates its own scratch
    void *ws_ptr = nullptr;
    size_t ws_bytes = 0;
    // pair-kernel schedule (points per sub-tile): forced (0 = autotune), the
    // autotuner's choices per problem shape, and the last one used
    int forced_sub = 0;
    std::vector<std::pair<long long, int>> tuned;
    int last_sub = 0;
};
