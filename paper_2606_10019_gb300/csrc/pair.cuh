// Interfaces between the C ABI (capi.cu) and the pair / finalize kernels.
#pragma once

#include "common.cuh"

namespace gcvo {

// Pair-kernel tiling: warps per block, points staged per warp and chunk,
// spatial groups per warp item, per-lane owner sums and owner data (float4s).
constexpr int PAIR_WARPS = 4;
constexpr int PAIR_CAP = 96;                       // <= 256 (uint8 queue entries)
constexpr int PAIR_MAX_SUB = 16;
constexpr int PAIR_OWN_S = 12;                     // 10 sums, padded
constexpr int PAIR_SLOTS = 28;
__host__ __device__ constexpr int pair_warp_smem(int mode) {
    return PAIR_CAP * 80 + 16 + PAIR_MAX_SUB * 8 + 64 * 4 + 32 * PAIR_OWN_S * 4 + 32 * 16 * (mode == 0 ? 3 : 6);
}

enum PairMode { PAIR_EVAL = 0, PAIR_LINESEARCH = 1 };
enum FinMode { FIN_EVAL = 0, FIN_GN = 1, FIN_GRAD = 2, FIN_LINESEARCH = 3, FIN_ANCHORS = 4 };

// Per-problem state kept on the device across iterations.
struct ProbDev {
    double T[12];      // current pose: R row-major (9), then t (3)
    double dir[6];     // G-CVO-1 search direction (caller frame)
    float R32[9];      // R rounded to float (pair kernel)
    float dir32[6];    // the search direction with v' = omega x o + v (grid-origin frame)
    int status;        // 0 active, 1 converged, 2 k_max reached, < 0: -gcvo_status
    int iter;
    int g0, g1;        // range of source groups
    int w0, w1;        // range of packed work items
    float rho2;        // Euclidean pre-test radius squared
    float c2;          // cutoff squared
    float sigma2;
    float iso_inv;     // 1 / iso_ell^2
};

struct EvalOut {
    double f, g[6], M[36], H[36];
    long long n_pairs, n_kept, n_cand;
};

struct PairArgs {
    const float4 *spos, *sca, *scb;
    const float4 *anchor;      // per group: R^T (z_g - t) - o, z_g its first point
    const int *gstart;
    const int4 *items;          // first group, groups, first point, points
    const int *item_prob;
    const int *n_items;
    const ProbDev *probs;
    const GridDev *grids;
    float *part;               // n_groups x 64 (hi[32], lo[32])
    long long *counts;         // n_groups x 4
    int *work;                 // dynamic group counter (zeroed before launch)
    unsigned *status_word;
    int ls_literal;
};

struct FinalizeArgs {
    ProbDev *probs;
    const float4 *spos;
    const int *gstart;
    float4 *anchor;
    const GridDev *grids;
    const float *part;
    const long long *counts;
    EvalOut *evalout;
    gcvo_iter_log *logs;
    int *n_active;
    int n_problems;
    int mode;
    int k_max;
    double eps_tol, mu0;
};

struct SrcDesc {
    const float *xyz, *cov, *feat;
    int64_t n, offset;
    float inv_hf;      // 1 / fine Morton voxel edge
};

struct SrcArgs {
    const SrcDesc *desc;
    unsigned long long *keys;
    int *vals, *prob_of, *local;
    int *lam_enc;
    unsigned *status_word;
    float4 *spos, *sca, *scb;
    int feat_dim;
    int iso;
};

size_t pair_smem_bytes(int mode);
int pair_blocks_per_sm(int mode, bool iso, int fd);
cudaError_t launch_pair(const PairArgs &a, int mode, bool iso, int fd, int grid, cudaStream_t s);
cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t s);
cudaError_t launch_src_keys(const SrcArgs &a, int n_problems, int64_t max_n, cudaStream_t s);
cudaError_t launch_src_segments(const unsigned long long *keys, int64_t n, int *seg, cudaStream_t s);
cudaError_t launch_src_group_heads(const int *seg, int64_t n, int *gh, cudaStream_t s);
cudaError_t launch_src_groups(const SrcArgs &a, const unsigned long long *keys, const int *gid, int64_t n,
                              int *gstart, int *gcount, int *gprob, int *pg0, int *pg1, cudaStream_t s);
// Greedy packing of consecutive groups of one problem into warp items of at
// most 32 points and PAIR_MAX_SUB groups.  pass 0 counts items per problem
// into cnt; pass 1 writes them at offsets incl - cnt (incl = inclusive scan).
cudaError_t launch_pack(int pass, int np, const int *gstart, const int *gcount, const int *pg0, const int *pg1,
                        int *cnt, const int *incl, int4 *items, int *item_prob, int *pw0, int *pw1,
                        cudaStream_t s);

}  // namespace gcvo
