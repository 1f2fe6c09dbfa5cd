/*
 * gcvo.h -- C ABI of the GB300 (sm_103a) G-CVO registration library.
 *
 * G-CVO registers a source ("new") point cloud Z to a target cloud X by
 * maximising the RKHS inner product of Eq. (4)-(5) of the paper,
 *
 *     f(T) = sum_ij <l_i^X, l_j^Z> k(x_i, T^{-1} z_j),
 *     k(x, z) = sigma^2 exp(-1/2 r^T Sigma_ij^{-1} r),  r = x - T^{-1} z,
 *     Sigma_ij = Sigma(x_i; X) + R^T Sigma(z_j; Z) R            (Eq. 7),
 *
 * with the Riemannian gradient of Lemma 1 (Eq. 8), the Gauss-Newton matrix
 * and Levi-Civita correction of Eq. (10)-(12), and the second-order update
 * T <- T exp(-H_GN^{-1} g) of Eq. (13) inside Algorithm 1.
 *
 * Conventions shared by every call:
 *  - A pose T is a 4x4 row-major double matrix [R t; 0 1] acting as
 *    T x = R x + t (Sec. 2.1).  The optimum satisfies T^{-1} z_j ~ x_i.
 *  - Tangent vectors are twists xi = (omega, v), rotation first (Sec. 2.1),
 *    left-trivialised; the gradient g = (g_omega, g_v).
 *  - Point arrays are structure-of-arrays float32: xyz is 3 x n
 *    (x[0..n), y[0..n), z[0..n)), a covariance array is 6 x n holding
 *    (xx, xy, xz, yy, yz, zz), a feature array is feat_dim x n.
 *  - Point arrays may live in device memory or in host memory; host arrays
 *    are copied to the device by the call.  They are only read, and must stay
 *    valid until the call returns.
 *  - All work runs on the stream given to gcvo_create, in stream order.
 *    Calls that return host results (eval, register) synchronise that stream
 *    before returning.  A context is used by one host thread at a time.
 *  - Every call returns a gcvo_status.  On any status other than GCVO_OK the
 *    outputs are left untouched, except where a call documents otherwise.
 *    Device-side failures (a bounded wait that ran out, a capacity limit, a
 *    non-finite reduction) are reported through a status word that the call
 *    reads back; no kernel traps.
 *  - Device memory for contexts and grids is allocated by the library with
 *    cudaMalloc and released by the matching destroy call.
 */
#ifndef GCVO_H
#define GCVO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GCVO_OK = 0,
    GCVO_ERR_INVALID_ARG = 1,   /* null pointer, bad size or parameter */
    GCVO_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    GCVO_ERR_WORKSPACE = 3,     /* device memory could not be allocated */
    GCVO_ERR_SINGULAR = 4,      /* the 6x6 system of a step (M - Gamma of Eq. 13, or
                                   H_E of G-CVO-E) could not be factorised */
    GCVO_ERR_NO_OVERLAP = 5,    /* no pair passed the kernel cutoff (f = 0) */
    GCVO_ERR_NOT_CONVERGED = 6, /* k_max iterations ran without ||xi||_1 < eps_tol */
    GCVO_ERR_NONFINITE = 7,     /* an input or a reduced value is NaN or Inf */
    GCVO_ERR_TIMEOUT = 8,       /* a bounded device-side wait ran out */
    GCVO_ERR_CAPACITY = 9       /* a size limit of this build was exceeded */
} gcvo_status;

typedef struct gcvo_ctx gcvo_ctx;   /* device, stream, scratch buffers */
typedef struct gcvo_proposal gcvo_proposal; /* learned initial-pose network */
typedef struct gcvo_grid gcvo_grid; /* voxel-hashed copy of a target cloud */

/* Kernel parameters (Eq. 7 and the Remark that follows it). */
typedef struct {
    int kernel_mode;    /* 0: anisotropic kernel of Eq. (7) (default);
                           1: isotropic CVO kernel, Sigma_ij = iso_ell^2 I (Remark 3) */
    double sigma2;      /* kernel amplitude sigma^2 of Eq. (7a); default 1 */
    double cutoff;      /* a pair contributes only if r^T Sigma_ij^{-1} r <= cutoff^2
                           (default 3); 0 disables the cutoff: every target /
                           source pair is evaluated, the paper's dense objective
                           (Sec. 5.4, O(N_X N_Z) per evaluation) */
    double iso_ell;     /* isotropic length scale (kernel_mode 1) */
    int knn;            /* n of Eq. (7b): neighbours per covariance, self included;
                           2..16 (default 10) */
    double eig_max;     /* eigenvalue bound of the Remark after Eq. (7): every
                           eigenvalue of a per-point covariance is clamped to */
    double eig_ratio;   /* [eig_max / eig_ratio, eig_max]; eig_max <= 0 disables */
    int feat_dim;       /* l: channels of the pose-invariant features, 1..7
                           (an intensity, RGB, or a label distribution over up
                           to 7 classes as in SemanticCVO); c_ij = <l_i, l_j>
                           (Eq. 5) */
    double cell_size;   /* target voxel edge; <= 0 picks the kernel range */
} gcvo_kernel_params;

/* Solver parameters (Algorithm 1 inputs mu_0, k_max, eps_tol). */
typedef struct {
    int order;          /* 2: G-CVO-2, Gauss-Newton step of Eq. (13);
                           1: G-CVO-1, gradient step with the line search of Eq. (9);
                           3: G-CVO-E, Newton step xi = -H_E^{-1} g with the exact
                              Riemannian Hessian H_E = D(g) + Gamma (Sec. 3.4, Eq. 12);
                              the step is not damped, so it heads for a maximum only
                              where H_E is negative definite (near one) */
    int k_max;          /* iteration limit, 1..GCVO_MAX_KMAX */
    double eps_tol;     /* stop when ||xi^(k)||_1 < eps_tol */
    double mu0;         /* G-CVO-1 minimum step of Eq. (9) */
} gcvo_solver_params;

/* One row of the iteration log: values at the pose T^(k) the iteration
 * started from, and the step it took. */
typedef struct {
    double f;           /* objective, Eq. (5) */
    double g[6];        /* Riemannian gradient (g_omega, g_v), Eq. (8) */
    double xi[6];       /* step xi^(k) */
    double xi_l1;       /* ||xi^(k)||_1 */
    double T[16];       /* T^(k), row-major */
    int64_t n_pairs;    /* pairs with |r_ij| <= rho, counted by the kernel */
    int64_t n_kept;     /* pairs with d^2 <= cutoff^2 */
} gcvo_iter_log;

/* Counters returned by gcvo_eval. */
typedef struct {
    int64_t n_pairs;      /* pairs with |r_ij| <= rho (pair-evals) */
    int64_t n_kept;       /* pairs with d^2 <= cutoff^2 */
    int64_t n_candidates; /* candidate pairs: each source point times the targets
                             within rho of its sub-tile's box */
    double rho;           /* Euclidean radius that bounds the cutoff ellipsoids */
} gcvo_eval_stats;

/* Description of one problem for gcvo_register_batched. */
typedef struct {
    const gcvo_grid *target;
    const float *src_xyz;   /* 3 x n_src */
    const float *src_cov;   /* 6 x n_src (ignored in kernel_mode 1) */
    const float *src_feat;  /* feat_dim x n_src */
    int64_t n_src;
    double T0[16];          /* initial pose T^(0) */
} gcvo_problem;

/* Library-wide limits of this build. */
#define GCVO_MAX_FEAT 7
#define GCVO_MAX_KNN 16
#define GCVO_MAX_KMAX 100000
#define GCVO_MAX_PROBLEMS 4096

/* Human-readable name of a status code (static storage). */
const char *gcvo_status_string(gcvo_status s);

/* Text of the last CUDA runtime failure seen by this host thread (the call,
 * its error string and code); empty when none.  Valid until the next call. */
const char *gcvo_last_error_detail(void);

/* Default kernel / solver parameters (cutoff 3, sigma2 1, knn 10, G-CVO-2,
 * k_max 200, eps_tol 1e-6, mu0 1e-10; the paper gives no mu0, and a
 * minimum step must stay below 2 / lambda_max(M) or G-CVO-1 leaves its fixed
 * point). */
void gcvo_default_kernel_params(gcvo_kernel_params *p);
void gcvo_default_solver_params(gcvo_solver_params *p);

/* Create a context bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL selects the legacy default stream).  The context
 * owns its scratch memory.  *ctx is set on success. */
gcvo_status gcvo_create(gcvo_ctx **ctx, int device, void *cuda_stream);

/* Release the context and its device memory (synchronises its stream). */
gcvo_status gcvo_destroy(gcvo_ctx *ctx);

/* Caller-owned scratch.  By default a context allocates its scratch with
 * cudaMalloc as calls need it and keeps it until gcvo_destroy.  A caller
 * that owns the device memory (a framework's allocator, a fixed budget)
 * can instead hand the context one workspace: gcvo_workspace_size gives
 * the bytes needed for calls of at most max_points points (the source
 * points of an evaluation or a registration, all problems together, or
 * the cloud of a covariance or grid call), max_problems problems and
 * max_log_rows iteration-log rows (n_problems x k_max of a logged
 * registration; 0 when no log is requested); ctx may be NULL.
 * gcvo_set_workspace gives the context dev_ptr (device memory on the
 * context's device, 256-byte aligned, at least that many bytes, owned by
 * the caller and kept alive until the workspace is replaced, removed or the
 * context destroyed) for the same limits; from then on gcvo_eval,
 * gcvo_eval_exact, gcvo_register, gcvo_register_batched,
 * gcvo_estimate_covariances, gcvo_estimate_covariances_batched (all its
 * clouds together count as its points, and it takes at most
 * 2 x max_problems clouds) and gcvo_build_grid / gcvo_rebuild_grid make no
 * device allocation for their scratch (a grid still owns its own storage),
 * and a call beyond the limits returns GCVO_ERR_WORKSPACE.
 * gcvo_build_grids_batched and gcvo_register_clouds use the same scratch
 * for all their clouds together: with a workspace set they fit when their
 * clouds hold at most max_points points together (at most 2 x max_problems
 * clouds) and only one of their grids reaches the 2^26-voxel limit, and
 * return GCVO_ERR_WORKSPACE otherwise.  dev_ptr = NULL returns the context to library-owned
 * scratch.  gcvo_set_workspace synchronises the stream and may allocate
 * the context's small pinned host buffer.  The paper has no counterpart:
 * this is the memory ownership of the boundary. */
gcvo_status gcvo_workspace_size(const gcvo_ctx *ctx, int64_t max_points, int max_problems, int64_t max_log_rows,
                                size_t *bytes);
gcvo_status gcvo_set_workspace(gcvo_ctx *ctx, void *dev_ptr, size_t bytes, int64_t max_points, int max_problems,
                               int64_t max_log_rows);

/* Eq. (7b) plus the eigenvalue bound of the Remark after Eq. (7): for each
 * point, Sigma = 1/(n-1) sum_{y in N_n(x)} (y - x)(y - x)^T over its n = knn
 * nearest points (the point itself included, ties broken by lower index),
 * then each eigenvalue is clamped to [eig_max/eig_ratio, eig_max].
 * xyz: 3 x n input; cov_out: 6 x n output, device memory, caller-owned.
 * Requires n >= knn.  Synchronises the stream (the search reads back how
 * many points need the coarse second pass, and its status). */
gcvo_status gcvo_estimate_covariances(gcvo_ctx *ctx, const float *xyz, int64_t n,
                                      const gcvo_kernel_params *params, float *cov_out);

/* Build the voxel grid of a target cloud X (Eq. 5's x_i with Sigma(x_i; X)
 * and features l_i^X): points are keyed by voxel, sorted, copied into a
 * grid-owned packed layout relative to the box centre (FP32 heads and
 * tails of x - o), and indexed by a dense per-voxel prefix table over the
 * box (the pair kernel's index; voxels are coarsened while the box holds
 * more than 2^26 of them).  cov may be NULL in kernel_mode 1.  The grid
 * keeps the kernel parameters it was built with.  A non-finite coordinate,
 * covariance or feature returns GCVO_ERR_NONFINITE, a covariance with a
 * non-positive diagonal entry GCVO_ERR_INVALID_ARG.  Synchronises the
 * stream. */
gcvo_status gcvo_build_grid(gcvo_ctx *ctx, const float *xyz, const float *cov, const float *feat,
                            int64_t n, const gcvo_kernel_params *params, gcvo_grid **grid_out);

/* Rebuild an existing grid from a new cloud, reusing its device memory
 * when it is large enough (frame-to-frame tracking re-targets every frame).
 * Same inputs and semantics as gcvo_build_grid; on failure the grid is left
 * in an unusable state and may only be destroyed or rebuilt.  The grid must
 * belong to the context's device.  Synchronises the stream. */
gcvo_status gcvo_rebuild_grid(gcvo_ctx *ctx, gcvo_grid *grid, const float *xyz, const float *cov, const float *feat,
                              int64_t n, const gcvo_kernel_params *params);

/* Release a grid.  May be called after the context that built it was
 * destroyed; waits for work still using the grid's memory. */
gcvo_status gcvo_grid_destroy(gcvo_grid *grid);

/* gcvo_estimate_covariances for n_clouds clouds in one call: cloud k has
 * n[k] points at xyz[k] (3 x n[k]) and its covariances go to cov_out[k]
 * (6 x n[k]); all device memory.  All clouds share one set of launches on
 * the context's stream: their points are gathered into one array, every
 * cloud gets its own voxel box and size, and one sort and one hash table
 * (voxel keys offset per cloud) serve the batch, so the cost no longer
 * grows with the number of clouds beyond their points.  The results equal
 * those of one call per cloud, bit for bit (the neighbour lists do not
 * depend on the voxel grid).  Synchronises the stream; a failure (a
 * non-finite coordinate in any cloud) fails the whole call. */
gcvo_status gcvo_estimate_covariances_batched(gcvo_ctx *ctx, int n_clouds, const float *const *xyz,
                                              const int64_t *n, const gcvo_kernel_params *params,
                                              float *const *cov_out);

/* gcvo_build_grid / gcvo_rebuild_grid for n_clouds target clouds in one
 * call: grids[k] == NULL builds a new grid into grids[k], otherwise
 * grids[k] is rebuilt in place.  Inputs as for gcvo_build_grid, per cloud,
 * device memory only (cov may be NULL in kernel_mode 1).  All clouds share
 * one set of launches on the context's stream (one box pass with one
 * read-back, one sort of all points, one segmented scan of the voxel
 * tables), and every grid equals the one gcvo_build_grid makes of its
 * cloud.  On failure no new grid is returned (grids[k] is NULL again where
 * it was NULL) and the grids given for a rebuild may only be destroyed or
 * rebuilt.  Synchronises the stream. */
gcvo_status gcvo_build_grids_batched(gcvo_ctx *ctx, int n_clouds, const float *const *xyz,
                                     const float *const *cov, const float *const *feat, const int64_t *n,
                                     const gcvo_kernel_params *params, gcvo_grid **grids);

/* Number of points and occupied voxels of a grid. */
gcvo_status gcvo_grid_info(const gcvo_grid *grid, int64_t *n_points, int64_t *n_cells, double *cell_size);

/* One evaluation at pose T (row-major 4x4, host): the objective f of Eq. (5),
 * the gradient g of Eq. (8) and H = H_GN = -M + Gamma of Eq. (11)-(12)
 * (row-major 6x6, host), summed over every pair with d^2 <= cutoff^2.
 * M_out (host 6x6, may be NULL) receives M = sum f_ij J_j^T Sigma_ij^{-1} J_j
 * of Eq. (11); stats may be NULL.  Synchronises the stream. */
gcvo_status gcvo_eval(gcvo_ctx *ctx, const gcvo_grid *target, const float *src_xyz, const float *src_cov,
                      const float *src_feat, int64_t n_src, const double T[16], double *f, double g[6],
                      double H[36], double *M_out, gcvo_eval_stats *stats);

/* The G-CVO-E evaluation at pose T (row-major 4x4, host): f and g as in
 * gcvo_eval, and H_E = D(g) + Gamma (row-major 6x6, host), where D(g) is
 * the exact directional derivative of the gradient field of Lemma 1 under
 * the right perturbation T exp(xi^) -- all four terms of the derivative of
 * g = -sum f_ij J_j^T Sigma_ij^{-1} r_ij: the change of the kernel weight,
 * of the lever arm p_j, of Sigma_ij^{-1} as R turns Sigma_j, and of r_ij
 * (the last alone is the -M of Gauss-Newton) -- and Gamma is the
 * connection term of Eq. (12).  D_out (host 6x6, may be NULL) receives
 * D(g), which is not symmetric away from a critical point; stats may be
 * NULL.  One pair pass, with twice the partial storage and about three
 * times the arithmetic per pair of gcvo_eval.  Synchronises the stream. */
gcvo_status gcvo_eval_exact(gcvo_ctx *ctx, const gcvo_grid *target, const float *src_xyz, const float *src_cov,
                            const float *src_feat, int64_t n_src, const double T[16], double *f, double g[6],
                            double H_E[36], double *D_out, gcvo_eval_stats *stats);

/* Algorithm 1 from T0: at most k_max iterations of transform, pair
 * evaluation, reduction and update (G-CVO-2 solves (M - Gamma) xi = g, Eq.
 * (13); G-CVO-1 takes xi = mu g with mu from Eq. (9); G-CVO-E solves
 * -(D(g) + Gamma) xi = g, see gcvo_eval_exact), stopping when
 * ||xi||_1 < eps_tol.  T_out receives the final pose (row-major, host);
 * log (host, capacity k_max rows, may be NULL) the per-iteration values;
 * n_iter the number of iterations run.  Returns GCVO_ERR_NOT_CONVERGED (with
 * all outputs written) when k_max ran out.  Synchronises the stream. */
gcvo_status gcvo_register(gcvo_ctx *ctx, const gcvo_grid *target, const float *src_xyz, const float *src_cov,
                          const float *src_feat, int64_t n_src, const double T0[16],
                          const gcvo_solver_params *params, double T_out[16], gcvo_iter_log *log, int *n_iter);

/* Algorithm 1 for n_problems independent problems in one set of launches:
 * every iteration evaluates all still-active problems in one pair-kernel
 * launch and updates them in one reduction and one solver launch; a
 * problem that converged
 * or failed is masked out.  T_out: n_problems x 16 (host); logs: n_problems
 * x k_max rows (host, may be NULL); n_iter and status: n_problems (host).
 * The call returns GCVO_OK when every problem ran (per-problem outcomes
 * are in status[]).  All problems must use grids built with the same
 * kernel_mode and feat_dim.  Synchronises the stream. */
gcvo_status gcvo_register_batched(gcvo_ctx *ctx, int n_problems, const gcvo_problem *problems,
                                  const gcvo_solver_params *params, double *T_out, gcvo_iter_log *logs,
                                  int *n_iter, int *status);

/* One registration problem given as raw clouds, for gcvo_register_clouds. */
typedef struct {
    const float *tgt_xyz;   /* 3 x n_tgt: the target cloud X */
    const float *tgt_feat;  /* feat_dim x n_tgt */
    int64_t n_tgt;
    const float *src_xyz;   /* 3 x n_src: the source cloud Z */
    const float *src_feat;  /* feat_dim x n_src */
    int64_t n_src;
    double T0[16];          /* initial pose T^(0) */
    const gcvo_kernel_params *params; /* this pair's kernel parameters, or NULL
                                         for the call's; kernel_mode and
                                         feat_dim must equal the call's */
} gcvo_cloud_pair;

/* The whole hot path from raw clouds: the per-point covariances of Eq.
 * (7b) with the eigenvalue bound for every target and source cloud, the
 * voxel grid of every target, and Algorithm 1 for all pairs in one batched
 * registration (as gcvo_register_batched).  Clouds may be host or device
 * arrays; host arrays are copied in, one copy per array, on the context's
 * stream.  The covariances and grids live in buffers the context keeps
 * and reuses on the next call.  Outputs as gcvo_register_batched: T_out
 * n_pairs x 16 (host), logs n_pairs x k_max rows (host, may be NULL),
 * n_iter and status n_pairs (host, may be NULL).  The covariances of all
 * clouds take one batched set of launches and the grids of all targets
 * another (as gcvo_estimate_covariances_batched and
 * gcvo_build_grids_batched), on the context's stream.  Synchronises the
 * stream. */
gcvo_status gcvo_register_clouds(gcvo_ctx *ctx, int n_pairs, const gcvo_cloud_pair *pairs,
                                 const gcvo_kernel_params *params, const gcvo_solver_params *solver, double *T_out,
                                 gcvo_iter_log *logs, int *n_iter, int *status);

/* The evaluation of gcvo_eval (f, g and H = -M + Gamma at pose T) for
 * callers that must not allocate device memory: an application whose memory
 * pool owns every device byte (a stray cudaMalloc would fail or fragment
 * it), a real-time loop that must not meet an allocation failure or the
 * device-wide synchronisation of cudaMalloc / cudaFree, or a plug-in without
 * a context to keep buffers in.  (The paper has no counterpart; this is a
 * deployment variant of one evaluation.)
 *
 * It needs no gcvo_ctx and allocates nothing: its scratch is one static
 * device array of 6.3 MiB in the library, reserved on every device that
 * loads the library until the process exits.  The caller passes device
 * pointers on the grid's device for every input (host pointers and
 * pointers to another device are rejected with GCVO_ERR_INVALID_ARG, as are
 * grids with more than 3 feature channels), the
 * target grid (built earlier with gcvo_build_grid), the stream, and host
 * outputs.  Source points are processed in the caller's order, 8 per work
 * item.
 *  - n_src above 65536 returns GCVO_ERR_CAPACITY.
 *  - The first call on a device looks up the array's device address (a
 *    one-time set-up).
 *  - Every call reuses the same array and overwrites the previous call's
 *    contents; two calls whose GPU work overlaps (on different streams or
 *    from different host threads without ordering) race and both results
 *    are undefined.
 * Synchronises cuda_stream before returning. */
gcvo_status gcvo_eval_static(const gcvo_grid *target, const float *src_xyz, const float *src_cov,
                             const float *src_feat, int64_t n_src, const double T[16], void *cuda_stream,
                             double *f, double g[6], double H[36]);

/* ------------------------------------------------------------------------
 * Learned initial-pose proposal (no counterpart in the paper: it is the
 * learned-proposal extension of Algorithm 1's initial pose T^(0)).
 *
 * A point-set network maps a (source, target) pair to a twist: per point
 * p = ((xyz - c) / s, l) with c and s the target's centroid and RMS radius,
 * a shared MLP 4 -> 64 -> 128 -> 256 (ReLU after the first two layers),
 * max-pooled over each cloud; the two 256-d features are concatenated and an
 * MLP 512 -> 256 -> 128 -> 6 (ReLU after the first two) gives the twist
 * (omega, v / s) of S T S^-1, S the shift by -c.  Weights are BF16 copies of
 * FP32 master weights; every product accumulates in FP32.
 *
 * Batches: B pairs of n points each.  src_xyz / tgt_xyz: device, B x 3 x n
 * (per pair a 3 x n SoA block); src_feat / tgt_feat: device, the first
 * feature channel of pair b at feat[b * stride .. + n).  The flat parameter
 * vector holds W1 (64x4), b1, W2 (128x64), b2, W3 (256x128), b3, H1
 * (256x512), c1, H2 (128x256), c2, H3 (6x128), c3, row-major.
 * ------------------------------------------------------------------------ */

/* Number of parameters of the proposal network. */
int64_t gcvo_proposal_n_params(void);

/* Create a network with all parameters zero (set them before use). */
gcvo_status gcvo_proposal_create(gcvo_ctx *ctx, gcvo_proposal **out);
gcvo_status gcvo_proposal_destroy(gcvo_proposal *prop);

/* Copy the FP32 master parameters in (host or device pointer, n_params
 * floats) and reset the Adam state (a fresh start from given weights); or
 * copy them out.  Checkpoints that resume training use the state calls
 * below.  Both synchronise the stream. */
gcvo_status gcvo_proposal_set_params(gcvo_ctx *ctx, gcvo_proposal *prop, const float *params);
gcvo_status gcvo_proposal_get_params(gcvo_ctx *ctx, const gcvo_proposal *prop, float *params_out);

/* The full training state, for checkpoints that resume training exactly:
 * state (host or device, 3 x n_params floats) holds the FP32 master
 * parameters, then Adam's first and second moment estimates, in the flat
 * parameter order; step is the number of Adam steps taken (it sets Adam's
 * bias corrections).  set_state also refreshes the BF16 weights.  The
 * round trip set_state(get_state()) is exact, and further training steps
 * then give the parameters of uninterrupted training to float rounding
 * (the backward sums gradients across blocks with float atomics, so two
 * runs of the same steps may differ in the last bits).  Both synchronise
 * the stream. */
gcvo_status gcvo_proposal_get_state(gcvo_ctx *ctx, const gcvo_proposal *prop, float *state_out, int64_t *step_out);
gcvo_status gcvo_proposal_set_state(gcvo_ctx *ctx, gcvo_proposal *prop, const float *state, int64_t step);

/* Forward pass for B pairs.  twist_out (host, B x 6, may be NULL): the
 * normalised twists; T0_out (host, B x 16, may be NULL): the proposed
 * initial poses S^-1 exp(omega, v) S in the caller's frame.  Synchronises. */
gcvo_status gcvo_proposal_infer(gcvo_ctx *ctx, gcvo_proposal *prop, int n_pairs, int n_points,
                                const float *src_xyz, const float *src_feat, int src_feat_stride,
                                const float *tgt_xyz, const float *tgt_feat, int tgt_feat_stride,
                                float *twist_out, double *T0_out);

/* One training step on B labelled pairs (T_label: host, B x 16 poses with
 * T^-1 z ~ x): forward, mean squared error of the normalised twist,
 * backward, and an Adam step with learning rate lr (lr = 0 leaves the
 * parameters unchanged).  loss_out (host, may be NULL) receives the loss,
 * grad_out (host, n_params, may be NULL) the gradient.  Synchronises. */
gcvo_status gcvo_proposal_train_step(gcvo_ctx *ctx, gcvo_proposal *prop, int n_pairs, int n_points,
                                     const float *src_xyz, const float *src_feat, int src_feat_stride,
                                     const float *tgt_xyz, const float *tgt_feat, int tgt_feat_stride,
                                     const double *T_label, float lr, float *loss_out, float *grad_out);

/* Profiling counters (no counterpart in the paper; used to measure the
 * pair kernel against its roofline). */
typedef struct {
    int64_t n_launches;      /* kernels launched by the library in this process
                                since gcvo_profile_enable */
    int64_t n_pair_launches; /* pair-kernel launches timed: evaluation passes
                                and G-CVO-E passes (not G-CVO-1 line searches) */
    double pair_kernel_ms;   /* their summed device time, from CUDA events
                                recorded on the context's stream around each launch */
    int64_t n_device_allocs; /* device allocations (cudaMalloc) the library made in
                                this process since gcvo_profile_enable */
    int64_t n_finalize_launches; /* FP64 finalize launches of the register loops */
    double finalize_ms;      /* their summed device time (CUDA events, as above) */
    double transform_ms;     /* summed device time of the per-iteration source
                                transform launches (CUDA events, as above) */
    double clouds_covariance_ms; /* gcvo_register_clouds: time from the call's
                                start to the end of its covariances, and */
    double clouds_grid_ms;   /* from there to the end of its grids (CUDA events
                                on the context's stream) */
} gcvo_profile;

/* Schedule of the pair passes (the autotuner; not in the paper): the source
 * points are cut into sub-tiles of at most `sub` = 4, 8, 16 or 32 points
 * (8, 4, 2 or 1 threads per point) that never cross a Morton voxel of edge
 * rho / 2 (level 1), rho (level 2) or 2 rho (level 3); a schedule is
 * sub | level << 8, and a bare sub means level 2.  set = 0 lets the autotuner pick per problem shape
 * (the default: on the first call for a shape it times one pass with each
 * candidate and keeps the fastest for the context); any other valid value
 * forces that schedule; set = -1 changes nothing.  *last_used (may be NULL)
 * receives the points per sub-tile of the last evaluation pass (0 before
 * any).  Results do not depend on the schedule beyond FP32 summation order. */
gcvo_status gcvo_pair_schedule(gcvo_ctx *ctx, int set, int *last_used);

/* Turn profiling on (enable != 0) or off and reset the counters.
 * Synchronises the stream. */
gcvo_status gcvo_profile_enable(gcvo_ctx *ctx, int enable);

/* Read the counters accumulated since gcvo_profile_enable (synchronises the
 * stream). */
gcvo_status gcvo_profile_read(gcvo_ctx *ctx, gcvo_profile *out);

#ifdef __cplusplus
}
#endif
#endif /* GCVO_H */
