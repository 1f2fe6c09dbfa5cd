// Interfaces between the C ABI (capi.cu) and the pair / finalize kernels.
#pragma once

#include "common.cuh"

namespace gcvo {

// Pair-kernel tiling (tile.cu): blocks of PAIR_WARPS independent warps; a
// warp takes one work item, a sub-tile of at most SUB = 4, 8, 16 or 32 source
// points (the schedule: 8, 4, 2 or 1 lanes per point), and stages target
// points PAIR_WCAP at a time in its own shared memory.
constexpr int PAIR_WARPS = 4;
constexpr int PAIR_WCAP = 160;
constexpr int PAIR_GRAB = 2;    // work items a warp takes per atomic (larger grabs of heavy items left long tails)
constexpr int PAIR_SLOTS = 28;         // f, g (6), M (21) per sub-tile
constexpr int PAIR_SLOTS_EXACT = 46;   // f, g, Q - M (21), C (9), S_B (9): G-CVO-E

enum PairMode { PAIR_EVAL = 0, PAIR_LINESEARCH = 1, PAIR_EXACT = 2 };
// FIN_EXACT: the G-CVO-E Newton step with H_E = D(g) + Gamma;
// FIN_EXACT_EVAL: f, g, D(g) and H_E into EvalOut (M holds D(g));
// FIN_POSE: only the split pose constants of ProbDev (Rh, Rl, ch, cl) for
// the initial pose.
enum FinMode {
    FIN_EVAL = 0,
    FIN_GN = 1,
    FIN_GRAD = 2,
    FIN_LINESEARCH = 3,
    FIN_POSE = 4,
    FIN_EXACT = 5,
    FIN_EXACT_EVAL = 6
};

// Per-problem state kept on the device across iterations.
struct ProbDev {
    double T[12];      // current pose: R row-major (9), then t (3)
    double dir[6];     // G-CVO-1 search direction (caller frame)
    // p = R^T (z - t) - o = R^T z - c with c = R^T t + o, every FP64 value
    // split into a float head and a float tail (head + tail = the FP64
    // value to about 2^-48 relative) for the double-float transform
    float Rh[9], Rl[9];
    float ch[3], cl[3];
    float dir32[6];    // the search direction with v' = omega x o + v (grid-origin frame)
    int status;        // 0 active, 1 converged, 2 k_max reached, < 0: -gcvo_status
    int iter;
    int w0, w1;        // range of packed work items
    int c0, c1;        // range of finalize chunks (FIN_CHUNK work items each)
    int lo;            // 1: the pair passes form r from double-float positions
    float rho2;        // Euclidean pre-test radius squared
    float c2;          // cutoff squared
    float sigma2;
    float iso_inv;     // 1 / iso_ell^2
};

struct EvalOut {
    double f, g[6], M[36], H[36];
    long long n_pairs, n_kept, n_cand;
};

// Source points in the target grid's frame at the current pose, written by
// k_transform once per iteration (sorted order, one record per point):
//   tpos = (p_hi, sigma^2 l0), tca = (S'xx, S'xy, S'xz, S'yy),
//   tcb = (S'yz, S'zz, sigma^2 l1, sigma^2 l2), tlo = (p_lo, 0),
//   tfx = sigma^2 (l3, l4, l5, l6) when there are more than 3 feature channels,
// with p = R^T (z - t) - o = p_hi + p_lo (double-float) and S' = R^T S R.
struct PairArgs {
    const float4 *tpos, *tca, *tcb, *tlo, *tfx;
    const int *items;          // per item (sub-tile): first point << 6 | points
    const int *item_prob;
    const int *n_items;
    const ProbDev *probs;
    const GridDev *grids;
    float *part;               // n_items x 64 (hi[32], lo[32])
    float *part2;              // PAIR_EXACT: slots 32.. in a second n_items x 64
    long long *counts;         // n_items x 4
    int *work;                 // dynamic item counter (zeroed before launch)
    unsigned *status_word;
    int ls_literal;
};

// The finalize runs in two launches: k_fin_reduce sums the work items of
// every chunk (FIN_CHUNK consecutive items of one problem) into one FP64 row,
// then k_fin_step, one warp per problem, adds its chunks' rows in order and
// takes the FP64 step.  The chunk rows depend only on the problem's own
// items, so a problem's result does not depend on the rest of the batch.
constexpr int FIN_CHUNK = 256;

// Bytes of the chunk rows for at most n_items work items over np problems.
inline size_t fin_chunk_bytes(int64_t n_items, int np) {
    const size_t chunks = (size_t)(n_items / FIN_CHUNK) + (size_t)np + 1;
    return chunks * (64 * sizeof(double) + 4 * sizeof(long long));
}

struct FinalizeArgs {
    ProbDev *probs;
    const GridDev *grids;
    const float *part;
    const float *part2;        // FIN_EXACT*: slots 32..
    const long long *counts;
    double *chunk;             // per chunk: 64 FP64 slot sums
    long long *chunk_cnt;      // per chunk: 4 count sums
    const int *n_chunks;       // chunks of all problems (written when items are packed)
    int reduce_blocks;         // grid of k_fin_reduce (a few blocks per SM)
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
    int *lam_enc;              // per problem: largest source covariance eigenvalue (ordered int)
    int *lam_min_enc;          // per problem: smallest
    unsigned *status_word;
    float4 *spos, *sca, *scb;
    float4 *sfx;               // feature channels 3..6 (null when feat_dim <= 3)
    int *pprob;                // problem of each sorted point
    int feat_dim;
    int iso;
};

// The per-iteration transform of every source point of the active problems
// into the target grid's frame (k_transform).
struct TransformArgs {
    const float4 *spos, *sca, *scb;   // packed source records, sorted (caller frame)
    const float4 *sfx;                // feature channels 3..6 (may be null)
    const int *pprob;                 // problem of each point (null: all problem 0)
    const ProbDev *probs;
    float4 *tpos, *tca, *tcb, *tlo;   // outputs (tlo may be null)
    float4 *tfx;                      // sigma^2 sfx (null when sfx is)
    int64_t n;
    int iso;
};

size_t pair_smem_bytes(int mode);
// sub: points per sub-tile (4, 8, 16, 32).
int pair_sub_for(int mode, int sub);
int pair_blocks_per_sm(int mode, bool iso, int fd, int sub);
cudaError_t launch_pair(const PairArgs &a, int mode, bool iso, int fd, int sub, int grid, cudaStream_t s);
cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t s);
cudaError_t launch_src_keys(const SrcArgs &a, int n_problems, int64_t max_n, cudaStream_t s);
cudaError_t launch_src_pack(const SrcArgs &a, const unsigned long long *keys, int64_t n, cudaStream_t s);
cudaError_t launch_transform(const TransformArgs &a, cudaStream_t s);
// Work items (sub-tiles of at most `sub` points inside one Morton voxel of
// level `level`: edge rho / 4 * 2^level) over the n sorted source points (keys as sorted; problem p's
// points start at point_off[p]): items[it] = first point << 6 | points,
// item_prob the problem, probs[p].w0 / w1 each problem's item range and
// *d_nitems the count (device side, no synchronisation).
// tmp: 3 x round_up(n, 64) ints.
gcvo_status pack_items(int np, const unsigned long long *keys, int64_t n, int sub, int level,
                       const int64_t *point_off, const int *n_pts, int *tmp, int *items, int *item_prob,
                       int *d_nitems, ProbDev *probs, int *n_chunks, void *scan_tmp, cudaStream_t s);

}  // namespace gcvo
