// The pair kernel: one evaluation of f (Eq. 5), g (Lemma 1, Eq. 8) and the
// Gauss-Newton matrix M (Eq. 11) -- or, for G-CVO-1, the line-search
// polynomial of Eq. (9) / Appendix B -- over every (target, source) pair of
// every active problem within the Euclidean radius rho.
//
// The source points of a problem are sorted by Morton code and cut into
// sub-tiles: runs of at most SUB points inside one Morton voxel of edge rho
// (or rho / 2 or 2 rho, the finer and coarser cuts the autotuner may pick).
// Every warp works alone
// on one sub-tile at a time (a work item); it takes up to PAIR_GRAB items per
// atomic on the global counter (two: a larger grab of heavy items leaves a
// few warps working long after the rest), and no warp waits for another.
//  1. Every point is read in the target grid's frame at the current pose
//     (Algorithm 1: p_j = R^T (z_j - t) - o and Sigma'_j = R^T Sigma_j R),
//     as k_transform (pair.cu) wrote it for this iteration.
//  2. The voxel columns (cx, cy) that meet the sub-tile's bounding box grown
//     by rho are listed, one per lane.  Points are sorted by voxel with cz
//     fastest, so the voxels of one column over the needed cz range hold one
//     run of points, read from the grid's dense per-voxel prefix table with
//     two loads.  The runs are staged into the warp's shared memory
//     PAIR_WCAP points at a time by cp.async.bulk copies completing on the
//     warp's mbarrier.
//  3. SUB = 4, 8, 16 or 32 (8, 4, 2 or 1 lanes per point) is the schedule the
//     autotuner picks.  The warp holds its sub-tile's points one per lane of
//     each group of SUB lanes, keeps the staged targets that lie within rho
//     of the sub-tile's box (one test per target) and walks them 32 / SUB at
//     a time: lane (q, i) pairs target q of the step with point i.  A target
//     is read by SUB lanes at once (a broadcast), a point stays in
//     registers, and no lane waits on another's branch.
//     With a finite cutoff, lambda_max(Sigma_ij) <= |Sigma_i|_F +
//     |Sigma'_j|_F bounds every pair that can pass d^2 <= c^2 to
//     |r|^2 <= c^2 (|Sigma_i|_F + |Sigma'_j|_F).  A sub-tile whose own
//     covariances are well below the problem's largest also lists the
//     targets within that bound of its box (with its points' largest norm).
//     When the second list is at most four fifths of the first, the warp
//     counts the pairs within rho over the first list (the pair-eval unit,
//     a distance test per pair) and evaluates only the second; otherwise
//     it evaluates the first list and counts as it goes.
//  4. Per pair (Eq. 7): Sigma_ij = Sigma_i + Sigma'_j, its adjugate and
//     determinant, d^2 = r^T Sigma_ij^-1 r, w = c_ij sigma^2 exp(-d^2 / 2)
//     for d^2 <= c^2 and |r| <= rho, else 0; the lane sums
//       S_f = sum w,  S_u = sum w Sigma^-1 r,  S_A = sum w Sigma^-1.
//  5. Per point, after the lanes that share it are added: f += S_f,
//     g = -(p x S_u, S_u), M += J^T S_A J with J = [-p^, I]; the warp adds
//     its points' 28 values with compensated (TwoSum) FP32 sums and writes
//     one (hi, lo) partial per sub-tile for the FP64 finalize.
// With no cutoff (dense mode) rho and the cutoff are infinite and every
// staged target meets every point: the same code visits all pairs.
// Features (c_ij = <l_i, l_j>, Eq. 5): channels 0..2 ride in pos.w, cb.z and
// cb.w; channels 3..6 (FD = 7: label distributions over up to 7 classes,
// SemanticCVO) in one more float4 stream staged beside the others.
// The G-CVO-E pass (PAIR_EXACT) visits the same pairs and adds the sums of
// the exact directional derivative of g (pair_exact); its 46 values per
// sub-tile go to two partial rows.
// r from double-float positions: r = (x_hi - p_hi) + (x_lo - p_lo), with
// the target grid's tails staged beside the points.  Positions are relative
// to the target box centre, and a LiDAR frame reaches 50-100 m from it,
// where FP32 rounds a position by 3-6 um.  With the flattest clamped
// covariances (sigma about 3 cm) that moves each pair's d^2 by about 1e-3
// and the gradient sums by about 1e-5 of their scale, which is the
// tolerance itself.  The host marks the problems whose bound
// 4 c R 2^-24 / sigma_min on that shift exceeds 3e-4 (P->lo); only their
// work items take the tails in the evaluation and line-search passes, and
// the others form r = x_hi - p_hi.  The G-CVO-E pass always takes them: the
// exact derivative is more sensitive still, since its weight-change and
// Gauss-Newton terms each reach several times its norm and cancel.  Every
// stage has room for the tails, so one layout serves all passes.
#include <cstddef>
#include <type_traits>

#include "common.cuh"
#include "pair.cuh"
#include "ptx.cuh"

namespace gcvo {
namespace {

static_assert(PAIR_WCAP <= 65535, "target list entries are 16-bit");
static_assert(PAIR_SLOTS * 33 * 4 <= PAIR_WCAP * 32, "epilogue transpose fits in a warp's staged pos, ca");
static_assert(PAIR_WARPS * (PAIR_WCAP * 80 + PAIR_WCAP * 4 + 64) <= 227 * 1024, "the largest block stage fits");
static_assert(PAIR_SLOTS_EXACT * 33 * 4 <= PAIR_WCAP * 48, "exact epilogue transpose fits in pos, ca, cb");

// Per warp: staged target points (with their coordinate tails when LO and
// their feature channels 3..6 when FX), the list of those near the
// sub-tile, and the mbarrier the bulk copies complete on.
template <bool LO, bool FX>
struct __align__(16) WarpStage {
    float4 pos[PAIR_WCAP];
    float4 ca[PAIR_WCAP];
    float4 cb[PAIR_WCAP];
    float4 lo[LO ? PAIR_WCAP : 1];
    float4 fx[FX ? PAIR_WCAP : 1];   // feature channels 3..6
    unsigned short list[PAIR_WCAP];    // staged targets within rho of the sub-tile box
    unsigned short listB[PAIR_WCAP];   // those of them within the per-pair bound
    uint64_t bar;
};

// The stage of one warp in a pass of mode MODE with FD feature channels:
// the kernel's layout and the launch's dynamic shared memory both come from
// this one type.  Every pass stages the target tails (r in double-float).
template <int MODE, int FD>
using StageT = WarpStage<true, (FD > 3)>;
using Stage3 = WarpStage<true, false>;
using Stage7 = WarpStage<true, true>;
static_assert(offsetof(Stage3, listB) == offsetof(Stage3, list) + PAIR_WCAP * sizeof(unsigned short) &&
                  offsetof(Stage7, listB) == offsetof(Stage7, list) + PAIR_WCAP * sizeof(unsigned short),
              "listB follows list: the evaluation indexes both from list");

// One anisotropic pair (Eq. 7), r = x_i - p_j, into the lane sums t[10].
template <int FD>
__device__ __forceinline__ void pair_aniso(const float r0, const float r1, const float r2, const float4 x,
                                           const float4 ca, const float4 cbv, const float4 xf, const float4 lf,
                                           float l0, float l1, float l2,
                                           const float q[6], float rho2, float c2, bool act, float *t, int &n_pairs,
                                           int &n_kept) {
    const float rr = r0 * r0 + r1 * r1 + r2 * r2;
    const bool in = act && rr <= rho2;
    float cij = x.w * l0;
    if (FD > 1) cij += cbv.z * l1 + cbv.w * l2;
    if (FD > 3) cij += xf.x * lf.x + xf.y * lf.y + xf.z * lf.z + xf.w * lf.w;
    const float s00 = ca.x + q[0], s01 = ca.y + q[1], s02 = ca.z + q[2];
    const float s11 = ca.w + q[3], s12 = cbv.x + q[4], s22 = cbv.y + q[5];
    const float c00 = s11 * s22 - s12 * s12;
    const float c01 = s02 * s12 - s01 * s22;
    const float c02 = s01 * s12 - s02 * s11;
    const float c11 = s00 * s22 - s02 * s02;
    const float c12 = s01 * s02 - s00 * s12;
    const float c22 = s00 * s11 - s01 * s01;
    const float det = s00 * c00 + s01 * c01 + s02 * c02;
    const float y0 = c00 * r0 + c01 * r1 + c02 * r2;
    const float y1 = c01 * r0 + c11 * r1 + c12 * r2;
    const float y2 = c02 * r0 + c12 * r1 + c22 * r2;
    const float qf = r0 * y0 + r1 * y1 + r2 * y2;
    const float rdet = rcp_approx(det);
    const float d2 = qf * rdet;
    const bool keep = in && d2 <= c2;
    const float wk = keep ? cij * ex2_approx(d2 * NEG_HALF_LOG2E) : 0.f;
    const float wd = wk * rdet;
    n_pairs += in;
    n_kept += keep;
    t[0] += wk;
    t[1] += wd * y0;
    t[2] += wd * y1;
    t[3] += wd * y2;
    t[4] += wd * c00;
    t[5] += wd * c01;
    t[6] += wd * c02;
    t[7] += wd * c11;
    t[8] += wd * c12;
    t[9] += wd * c22;
}

// One anisotropic pair of the G-CVO-E pass into t[25]: the sums of
// pair_aniso (t[0..9]) and, with y = Sigma_ij^-1 r, s = Sigma'_j y,
// u = y x s and K = Sigma_ij^-1 (Sigma'_j y^ - s^),
//   S_yy = sum w y y^T (t[10..15], upper triangle),
//   S_B  = sum w (y u^T + K) (t[16..24], row-major).
// Along xi = (omega, v) the pair moves by dr = J xi, and the rotation of
// Sigma'_j changes Sigma_ij^-1 r by K omega and r^T Sigma_ij^-1 r by
// -2 u . omega (Sec. 3.4, the four terms of the derivative of Eq. 8).
template <int FD>
__device__ __forceinline__ void pair_exact(const float r0, const float r1, const float r2, const float4 x,
                                           const float4 ca, const float4 cbv, const float4 xf, const float4 lf,
                                           float l0, float l1, float l2,
                                           const float q[6], float rho2, float c2, bool act, float *t, int &n_pairs,
                                           int &n_kept) {
    const float rr = r0 * r0 + r1 * r1 + r2 * r2;
    const bool in = act && rr <= rho2;
    float cij = x.w * l0;
    if (FD > 1) cij += cbv.z * l1 + cbv.w * l2;
    if (FD > 3) cij += xf.x * lf.x + xf.y * lf.y + xf.z * lf.z + xf.w * lf.w;
    const float s00 = ca.x + q[0], s01 = ca.y + q[1], s02 = ca.z + q[2];
    const float s11 = ca.w + q[3], s12 = cbv.x + q[4], s22 = cbv.y + q[5];
    const float c00 = s11 * s22 - s12 * s12;
    const float c01 = s02 * s12 - s01 * s22;
    const float c02 = s01 * s12 - s02 * s11;
    const float c11 = s00 * s22 - s02 * s02;
    const float c12 = s01 * s02 - s00 * s12;
    const float c22 = s00 * s11 - s01 * s01;
    const float det = s00 * c00 + s01 * c01 + s02 * c02;
    const float y0 = c00 * r0 + c01 * r1 + c02 * r2;
    const float y1 = c01 * r0 + c11 * r1 + c12 * r2;
    const float y2 = c02 * r0 + c12 * r1 + c22 * r2;
    const float qf = r0 * y0 + r1 * y1 + r2 * y2;
    const float rdet = rcp_approx(det);
    const float d2 = qf * rdet;
    const bool keep = in && d2 <= c2;
    const float wk = keep ? cij * ex2_approx(d2 * NEG_HALF_LOG2E) : 0.f;
    const float wd = wk * rdet;
    n_pairs += in;
    n_kept += keep;
    t[0] += wk;
    t[1] += wd * y0;
    t[2] += wd * y1;
    t[3] += wd * y2;
    t[4] += wd * c00;
    t[5] += wd * c01;
    t[6] += wd * c02;
    t[7] += wd * c11;
    t[8] += wd * c12;
    t[9] += wd * c22;
    const float ya = y0 * rdet, yb = y1 * rdet, yc = y2 * rdet;
    const float sa = q[0] * ya + q[1] * yb + q[2] * yc;
    const float sb = q[1] * ya + q[3] * yb + q[4] * yc;
    const float sc = q[2] * ya + q[4] * yb + q[5] * yc;
    const float u[3] = {yb * sc - yc * sb, yc * sa - ya * sc, ya * sb - yb * sa};
    const float wy[3] = {wk * ya, wk * yb, wk * yc};
    t[10] += wy[0] * ya;
    t[11] += wy[0] * yb;
    t[12] += wy[0] * yc;
    t[13] += wy[1] * yb;
    t[14] += wy[1] * yc;
    t[15] += wy[2] * yc;
    // Gm = Sigma'_j y^ - s^, then K det = adj(Sigma_ij) Gm
    const float Sp[9] = {q[0], q[1], q[2], q[1], q[3], q[4], q[2], q[4], q[5]};
    float Gm[9];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        Gm[3 * r + 0] = Sp[3 * r + 1] * yc - Sp[3 * r + 2] * yb;
        Gm[3 * r + 1] = Sp[3 * r + 2] * ya - Sp[3 * r + 0] * yc;
        Gm[3 * r + 2] = Sp[3 * r + 0] * yb - Sp[3 * r + 1] * ya;
    }
    Gm[1] += sc;
    Gm[2] -= sb;
    Gm[3] -= sc;
    Gm[5] += sa;
    Gm[6] += sb;
    Gm[7] -= sa;
    const float adj[9] = {c00, c01, c02, c01, c11, c12, c02, c12, c22};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            t[16 + 3 * r + c] += wy[r] * u[c] +
                                 wd * (adj[3 * r] * Gm[c] + adj[3 * r + 1] * Gm[3 + c] + adj[3 * r + 2] * Gm[6 + c]);
}

// J^T S J for J = [-p^, I] and a symmetric 3x3 S (xx, xy, xz, yy, yz, zz):
// the 21 values of its upper triangle, row-major (Eq. 11 per point).
__device__ __forceinline__ void jt_s_j(float A00, float A01, float A02, float A11, float A12, float A22, float px,
                                       float py, float pz, float *v) {
    // [[P^T S P, P S], [-S P, S]], P = p^
    const float B01 = -A00 * pz + A02 * px, B02 = A00 * py - A01 * px;
    const float B10 = A11 * pz - A12 * py, B11 = -A01 * pz + A12 * px, B12 = A01 * py - A11 * px;
    const float B20 = A12 * pz - A22 * py, B21 = -A02 * pz + A22 * px, B22 = A02 * py - A12 * px;
    v[0] = pz * B10 - py * B20;
    v[1] = pz * B11 - py * B21;
    v[2] = pz * B12 - py * B22;
    v[3] = -pz * A01 + py * A02;
    v[4] = -pz * A11 + py * A12;
    v[5] = -pz * A12 + py * A22;
    v[6] = -pz * B01 + px * B21;
    v[7] = -pz * B02 + px * B22;
    v[8] = pz * A00 - px * A02;
    v[9] = pz * A01 - px * A12;
    v[10] = pz * A02 - px * A22;
    v[11] = py * B02 - px * B12;
    v[12] = -py * A00 + px * A01;
    v[13] = -py * A01 + px * A11;
    v[14] = -py * A02 + px * A12;
    v[15] = A00;
    v[16] = A01;
    v[17] = A02;
    v[18] = A11;
    v[19] = A12;
    v[20] = A22;
}

// Line-search sums of one pair (Appendix B): with beta, gamma, delta, eps the
// coefficients of the exponent's expansion along t xi, the kernel value
// w e^(beta t + gamma t^2 + ...) contributes w * (1, beta, gamma + beta^2/2,
// ...) to (S_f, L1, L2, L3, L4).
__device__ __forceinline__ void ls_terms(float wgt, float kr1, float kr2, float kr3, float kr4, float a11, float a12,
                                         float a13, float a22, int literal, float *t) {
    float be, ga, de, ep;
    if (!literal) {
        be = -kr1;
        ga = 0.5f * (kr2 - a11);
        de = -kr3 * (1.f / 6.f) + 0.5f * a12;
        ep = kr4 * (1.f / 24.f) - a13 * (1.f / 6.f) - a22 * 0.125f;
    } else {
        be = -kr1;
        ga = -0.5f * a11 - kr2;
        de = -a12 - kr3;
        ep = -0.5f * (a22 + 2.f * a13 + 2.f * kr4);
    }
    t[0] += wgt;
    t[1] += wgt * be;
    t[2] += wgt * (ga + 0.5f * be * be);
    t[3] += wgt * (de + be * ga + be * be * be * (1.f / 6.f));
    t[4] += wgt * (ep + be * de + 0.5f * be * be * ga + 0.5f * ga * ga + be * be * be * be * (1.f / 24.f));
}

template <int MODE, bool ISO, int FD, int SUB>
__global__ void __launch_bounds__(PAIR_WARPS * 32, MODE == PAIR_EVAL ? 5 : 4) k_tile(PairArgs a) {
    static_assert(SUB == 4 || SUB == 8 || SUB == 16 || SUB == 32, "sub-tile of 4, 8, 16 or 32 points");
    static_assert(FD == 1 || FD == 3 || FD == 7, "1, up to 3 or up to 7 feature channels");
    constexpr int TQ = 32 / SUB;    // targets per warp step
    constexpr int NT = MODE == PAIR_EVAL ? 10 : MODE == PAIR_EXACT ? 25 : 5;
    constexpr int NSLOT = MODE == PAIR_EVAL ? PAIR_SLOTS : MODE == PAIR_EXACT ? PAIR_SLOTS_EXACT : 5;
    // r from double-float positions in every pass (see the header comment)
    constexpr bool LO = true;
    constexpr bool FX = FD > 3;
    using Stage = StageT<MODE, FD>;
    static_assert(std::is_same<Stage, WarpStage<LO, FX>>::value, "the stage type matches LO and FX");
    extern __shared__ __align__(16) unsigned char smem_raw[];   // PAIR_WARPS stages
    Stage *stage = reinterpret_cast<Stage *>(smem_raw);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qi = lane / SUB, si = lane % SUB;
    const unsigned FULL = 0xffffffffu;
    const unsigned lt_mask = (1u << lane) - 1u;
    Stage &S = stage[w];
    if (lane == 0) mbar_init(&S.bar, 1);
    __syncwarp();
    unsigned parity = 0;
    const int n_items = *a.n_items;
    // items per grab: up to PAIR_GRAB, fewer when there are few items per
    // warp, so that small problems still spread over the whole GPU
    const int grab = max(1, min(PAIR_GRAB, n_items / (int)(gridDim.x * PAIR_WARPS * 4)));
    int gbase = 0;          // first item of the current grab
    unsigned pending = 0;   // lanes of the grab whose item is still to do
    int my_word = 0, my_prob = 0;
    for (;;) {
        if (!pending) {
            // grab `grab` items; lane l looks at item gbase + l
            if (lane == 0) gbase = atomicAdd(a.work, grab);
            gbase = __shfl_sync(FULL, gbase, 0);
            if (gbase >= n_items) break;
            bool live = false, last = false;
            if (lane < grab && gbase + lane < n_items) {
                my_prob = a.item_prob[gbase + lane];
                my_word = a.items[gbase + lane];
                live = a.probs[my_prob].status == 0;   // finished problems are skipped
                last = lane == grab - 1 || gbase + lane == n_items - 1;
            }
            // the grab ends in a finished problem: move the counter past the
            // rest of that problem's items in one step
            if (last && !live) atomicMax(a.work, a.probs[my_prob].w1);
            pending = __ballot_sync(FULL, live);
            if (!pending) continue;
        }
        const int src_lane = __ffs(pending) - 1;
        pending &= pending - 1;
        const int it = gbase + src_lane;
        const int prob = __shfl_sync(FULL, my_prob, src_lane);
        const unsigned word = (unsigned)__shfl_sync(FULL, my_word, src_lane);
        const ProbDev *P = a.probs + prob;
        const GridDev *G = a.grids + prob;
        // double-float r for this problem (the same for the whole warp)
        const bool dfr = MODE == PAIR_EXACT || P->lo != 0;
        // the sub-tile: first point << 6 | points
        const int j0 = (int)(word >> 6), cnt = (int)(word & 63u);
        const bool sval = si < cnt;

        // ---- 1. the lane's source point in the grid frame (k_transform)
        const int jj = j0 + (sval ? si : 0);
        const float4 P4 = a.tpos[jj];
        const float px = P4.x, py = P4.y, pz = P4.z;
        const float l0 = P4.w;   // sigma^2 l0
        float l1 = 0.f, l2 = 0.f;
        float qv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // Sigma'_j
        if (FD > 1 || !ISO) {
            const float4 B4 = a.tcb[jj];
            qv[4] = B4.x;
            qv[5] = B4.y;
            l1 = B4.z;
            l2 = B4.w;
        }
        if (!ISO) {
            const float4 A4 = a.tca[jj];
            qv[0] = A4.x;
            qv[1] = A4.y;
            qv[2] = A4.z;
            qv[3] = A4.w;
        }
        float4 lf = make_float4(0.f, 0.f, 0.f, 0.f);   // sigma^2 l3..l6
        if (FX) lf = a.tfx[jj];
        float plx = 0.f, ply = 0.f, plz = 0.f;   // tail of p
        if (dfr) {
            const float4 L4 = a.tlo[jj];
            plx = L4.x;
            ply = L4.y;
            plz = L4.z;
        }
        const float rho2 = P->rho2, c2 = P->c2, iso_inv = P->iso_inv;
        // Two target lists per sub-tile (anisotropic kernel with a cutoff):
        // every pair within rho is counted (the pair-eval unit), but a pair
        // can only pass d^2 <= c^2 if |r|^2 <= c^2 lambda_max(Sigma_ij) <=
        // c^2 (|Sigma'_i|_F + |Sigma_j|_F), so only the targets within that
        // bound of the sub-tile's box are evaluated.
        const bool bounded = !ISO && c2 < INFINITY;
        float lam_i = 0.f;   // |Sigma'_i|_F, an upper bound of its largest eigenvalue
        if (bounded && sval)
            lam_i = sqrtf(qv[0] * qv[0] + qv[3] * qv[3] + qv[5] * qv[5] +
                          2.f * (qv[1] * qv[1] + qv[2] * qv[2] + qv[4] * qv[4]));

        // G-CVO-1 second pass: a_k = (xi^)^k p, xi the search direction
        float b1[3], b2[3], b3[3], b4[3];
        if (MODE == PAIR_LINESEARCH) {
            const float om0 = P->dir32[0], om1 = P->dir32[1], om2 = P->dir32[2];
            b1[0] = om1 * pz - om2 * py + P->dir32[3];
            b1[1] = om2 * px - om0 * pz + P->dir32[4];
            b1[2] = om0 * py - om1 * px + P->dir32[5];
#define CROSS_W(dst, src)                 \
    dst[0] = om1 * src[2] - om2 * src[1]; \
    dst[1] = om2 * src[0] - om0 * src[2]; \
    dst[2] = om0 * src[1] - om1 * src[0];
            CROSS_W(b2, b1)
            CROSS_W(b3, b2)
            CROSS_W(b4, b3)
#undef CROSS_W
        }

        // ---- bounding box of the sub-tile
        float bmin[3], bmax[3];
        {
            const float pp[3] = {px, py, pz};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                bmin[k] = ord_dec(__reduce_min_sync(FULL, ord_enc(sval ? pp[k] : INFINITY)));
                bmax[k] = ord_dec(__reduce_max_sync(FULL, ord_enc(sval ? pp[k] : -INFINITY)));
            }
        }
        const float lam_sub = bounded ? ord_dec(__reduce_max_sync(FULL, ord_enc(lam_i))) : 0.f;
        const float rho = sqrtf(rho2);
        const float h = G->h, ih = G->inv_h;
        // culling radius: rho plus a margin for the float voxel assignment
        const float rc = rho * 1.0001f + 1e-5f * h;
        const float rc2 = rc * rc;
        // the second list only where it can be much shorter: a sub-tile whose
        // own covariances are about as large as the largest (sparse LiDAR)
        // meets targets whose bound is about rho as well
        const bool two_lists = bounded && 2.f * c2 * lam_sub < 0.64f * rc2;
        int lo[3], hi[3];
        bool empty = !(bmin[0] <= bmax[0]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float fl = floorf((bmin[k] - rc - G->corner[k]) * ih);
            float fh = floorf((bmax[k] + rc - G->corner[k]) * ih);
            fl = fminf(fmaxf(fl, 0.0f), (float)G->dims[k]);
            fh = fmaxf(fminf(fh, (float)(G->dims[k] - 1)), -1.0f);
            if (!(fl <= fh)) empty = true;
            lo[k] = empty ? 0 : (int)fl;
            hi[k] = empty ? -1 : (int)fh;
        }
        const int ncy = empty ? 0 : hi[1] - lo[1] + 1;
        const int n_cols = empty ? 0 : (hi[0] - lo[0] + 1) * ncy;

        float t[NT];
#pragma unroll
        for (int k = 0; k < NT; ++k) t[k] = 0.f;
        int n_pairs = 0, n_kept = 0, n_cand = 0;
        int npe = 0;   // pairs within rho counted by the evaluation loop
        const int dy = G->dims[1], dzs = G->dims[2];

        for (int cb0 = 0; cb0 < n_cols; cb0 += 32) {
            // ---- 2. one column per lane: its run of target points.  A
            // column is kept when its xy rectangle lies within rho of the
            // box; its cz range shrinks with that distance.
            const int c = cb0 + lane;
            int rs = 0, rl = 0;
            if (c < n_cols) {
                const int cx = lo[0] + c / ncy, cy = lo[1] + c % ncy;
                const float x0 = G->corner[0] + (float)cx * h, y0 = G->corner[1] + (float)cy * h;
                const float ddx = fmaxf(0.0f, fmaxf(x0 - bmax[0], bmin[0] - (x0 + h)));
                const float ddy = fmaxf(0.0f, fmaxf(y0 - bmax[1], bmin[1] - (y0 + h)));
                const float d2xy = ddx * ddx + ddy * ddy;
                if (d2xy <= rc2) {
                    const float ez = sqrtf(rc2 - d2xy);
                    const int czl = max(lo[2], (int)floorf(fmaxf((bmin[2] - ez - G->corner[2]) * ih, -1.0f)));
                    const int czh = min(hi[2], (int)floorf(fminf((bmax[2] + ez - G->corner[2]) * ih, (float)dzs)));
                    if (czl <= czh) {
                        const size_t base = ((size_t)cx * dy + cy) * dzs;
                        rs = __ldg(G->vox_first + base + czl);
                        rl = __ldg(G->vox_first + base + czh + 1) - rs;
                    }
                }
            }
            // exclusive warp offsets of the runs
            int incl = rl;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(FULL, incl, 31);
            const int off = incl - rl;

            for (int base = 0; base < total; base += PAIR_WCAP) {
                const int m = min(PAIR_WCAP, total - base);
                // ---- stage the chunk [base, base + m) (bulk copies)
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive_expect_tx(&S.bar, (unsigned)m * (48u + (dfr ? 16u : 0u) + (FX ? 16u : 0u)));
                __syncwarp();
                {
                    const int s0 = max(off, base), s1 = min(off + rl, base + m);
                    if (s1 > s0) {
                        const int src = rs + (s0 - off), dst = s0 - base;
                        const unsigned bytes = (unsigned)(s1 - s0) * 16u;
                        bulk_g2s(S.pos + dst, G->pos + src, bytes, &S.bar);
                        bulk_g2s(S.ca + dst, G->ca + src, bytes, &S.bar);
                        bulk_g2s(S.cb + dst, G->cb + src, bytes, &S.bar);
                        if (dfr) bulk_g2s(S.lo + dst, G->plo + src, bytes, &S.bar);
                        if (FX) bulk_g2s(S.fx + dst, G->fx + src, bytes, &S.bar);
                    }
                }
                {
                    // bounded wait; the exit decision is warp-uniform
                    int spin = 0;
                    bool all_done;
                    for (;;) {
                        all_done = __all_sync(FULL, mbar_try_wait(&S.bar, parity));
                        if (all_done || ++spin > (1 << 22)) break;
                    }
                    if (!all_done) {
                        if (lane == 0) atomicOr(a.status_word, DEV_ERR_TIMEOUT);
                        return;
                    }
                    parity ^= 1u;
                }

                // ---- 3. the staged targets within rho of the sub-tile box
                // (list), and those of them within the per-pair bound
                // c^2 (lam_sub + |Sigma_j|_F) of it (listB; a small margin
                // covers the rounding of the box test)
                int L = 0, LB = 0;
                for (int t0 = 0; t0 < m; t0 += 32) {
                    const int tt = t0 + lane;
                    bool hit = false, near = false;
                    if (tt < m) {
                        const float4 x = S.pos[tt];
                        const float dx = fmaxf(0.f, fmaxf(bmin[0] - x.x, x.x - bmax[0]));
                        const float dyy = fmaxf(0.f, fmaxf(bmin[1] - x.y, x.y - bmax[1]));
                        const float dz = fmaxf(0.f, fmaxf(bmin[2] - x.z, x.z - bmax[2]));
                        const float db2 = dx * dx + dyy * dyy + dz * dz;
                        hit = db2 <= rc2;
                        if (two_lists && hit) {
                            const float4 ca = S.ca[tt], cbv = S.cb[tt];
                            const float lam_j = sqrtf(ca.x * ca.x + ca.w * ca.w + cbv.y * cbv.y +
                                                      2.f * (ca.y * ca.y + ca.z * ca.z + cbv.x * cbv.x));
                            near = db2 <= c2 * (lam_sub + lam_j) * 1.001f + 1e-12f;
                        }
                    }
                    const unsigned bal = __ballot_sync(FULL, hit);
                    if (hit) S.list[L + __popc(bal & lt_mask)] = (unsigned short)tt;
                    L += __popc(bal);
                    if (two_lists) {
                        const unsigned balB = __ballot_sync(FULL, near);
                        if (near) S.listB[LB + __popc(balB & lt_mask)] = (unsigned short)tt;
                        LB += __popc(balB);
                    }
                }
                __syncwarp();
                if (qi == 0 && sval) n_cand += L;
                // the counting pass pays off when it removes a fifth or more
                // of the evaluations; otherwise the evaluation counts
                const bool split = two_lists && LB * 5 < L * 4;
                // the evaluated list: listB follows list in the stage
                const int eoff = split ? PAIR_WCAP : 0;
                const int EL = split ? LB : L;
                if (split) {
                    // every pair within rho of the sub-tile, counted with the
                    // same r as the evaluation forms
                    for (int j = 0; j < L; j += TQ) {
                        const int idx = j + qi;
                        const int k = S.list[min(idx, L - 1)];
                        const float4 x = S.pos[k];
                        float r0 = x.x - px, r1 = x.y - py, r2 = x.z - pz;
                        if (dfr) {
                            const float4 xl = S.lo[k];
                            r0 += xl.x - plx;
                            r1 += xl.y - ply;
                            r2 += xl.z - plz;
                        }
                        n_pairs += (sval && idx < L && r0 * r0 + r1 * r1 + r2 * r2 <= rho2) ? 1 : 0;
                    }
                }

                // ---- 4. TQ targets per step, one per group of lanes
                for (int j = 0; j < EL; j += TQ) {
                    const int idx = j + qi;
                    const bool act = sval && idx < EL;
                    const int k = S.list[eoff + min(idx, EL - 1)];
                    const float4 x = S.pos[k];
                    float r0 = x.x - px, r1 = x.y - py, r2 = x.z - pz;
                    if (dfr) {
                        // r = (x_hi - p_hi) + (x_lo - p_lo)
                        const float4 xl = S.lo[k];
                        r0 += xl.x - plx;
                        r1 += xl.y - ply;
                        r2 += xl.z - plz;
                    }
                    const float4 xf = FX ? S.fx[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                    if (MODE == PAIR_EVAL && !ISO) {
                        pair_aniso<FD>(r0, r1, r2, x, S.ca[k], S.cb[k], xf, lf, l0, l1, l2, qv, rho2, c2, act, t,
                                       npe, n_kept);
                        continue;
                    }
                    if constexpr (MODE == PAIR_EXACT && !ISO) {
                        pair_exact<FD>(r0, r1, r2, x, S.ca[k], S.cb[k], xf, lf, l0, l1, l2, qv, rho2, c2, act, t,
                                       npe, n_kept);
                        continue;
                    }
                    const float rr = r0 * r0 + r1 * r1 + r2 * r2;
                    const bool in = act && rr <= rho2;
                    float cij = x.w * l0;
                    if (FD > 1) {
                        const float4 cbv = S.cb[k];
                        cij += cbv.z * l1 + cbv.w * l2;
                    }
                    if (FX) cij += xf.x * lf.x + xf.y * lf.y + xf.z * lf.z + xf.w * lf.w;
                    if (ISO) {
                        const float d2 = rr * iso_inv;
                        const bool keep = in && d2 <= c2;
                        const float wgt = keep ? cij * ex2_approx(d2 * NEG_HALF_LOG2E) : 0.f;
                        npe += in;
                        n_kept += keep;
                        if constexpr (MODE == PAIR_EVAL || MODE == PAIR_EXACT) {
                            t[0] += wgt;
                            t[1] += wgt * r0;
                            t[2] += wgt * r1;
                            t[3] += wgt * r2;
                            if constexpr (MODE == PAIR_EXACT) {
                                // Sigma'_j = 0: y = r / ell^2, u = 0, K = 0
                                t[10] += wgt * r0 * r0;
                                t[11] += wgt * r0 * r1;
                                t[12] += wgt * r0 * r2;
                                t[13] += wgt * r1 * r1;
                                t[14] += wgt * r1 * r2;
                                t[15] += wgt * r2 * r2;
                            }
                        } else {
                            // A = I / ell^2
                            const float kr1 = (b1[0] * r0 + b1[1] * r1 + b1[2] * r2) * iso_inv;
                            const float kr2 = (b2[0] * r0 + b2[1] * r1 + b2[2] * r2) * iso_inv;
                            const float kr3 = (b3[0] * r0 + b3[1] * r1 + b3[2] * r2) * iso_inv;
                            const float kr4 = (b4[0] * r0 + b4[1] * r1 + b4[2] * r2) * iso_inv;
                            const float a11 = (b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2]) * iso_inv;
                            const float a12 = (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2]) * iso_inv;
                            const float a13 = (b1[0] * b3[0] + b1[1] * b3[1] + b1[2] * b3[2]) * iso_inv;
                            const float a22 = (b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]) * iso_inv;
                            ls_terms(wgt, kr1, kr2, kr3, kr4, a11, a12, a13, a22, a.ls_literal, t);
                        }
                    } else {
                        // anisotropic line search (MODE == PAIR_LINESEARCH)
                        const float4 ca = S.ca[k];
                        const float4 cbv = S.cb[k];
                        const float s00 = ca.x + qv[0], s01 = ca.y + qv[1], s02 = ca.z + qv[2];
                        const float s11 = ca.w + qv[3], s12 = cbv.x + qv[4], s22 = cbv.y + qv[5];
                        const float c00 = s11 * s22 - s12 * s12;
                        const float c01 = s02 * s12 - s01 * s22;
                        const float c02 = s01 * s12 - s02 * s11;
                        const float c11 = s00 * s22 - s02 * s02;
                        const float c12 = s01 * s02 - s00 * s12;
                        const float c22 = s00 * s11 - s01 * s01;
                        const float det = s00 * c00 + s01 * c01 + s02 * c02;
                        const float y0 = c00 * r0 + c01 * r1 + c02 * r2;
                        const float y1 = c01 * r0 + c11 * r1 + c12 * r2;
                        const float y2 = c02 * r0 + c12 * r1 + c22 * r2;
                        const float qf = r0 * y0 + r1 * y1 + r2 * y2;
                        const float rdet = rcp_approx(det);
                        const float d2 = qf * rdet;
                        const bool keep = in && d2 <= c2;
                        const float wgt = keep ? cij * ex2_approx(d2 * NEG_HALF_LOG2E) : 0.f;
                        npe += in;
                        n_kept += keep;
                        // bilinear forms of A = adj / det with r and a_k
                        const float kr1 = (b1[0] * y0 + b1[1] * y1 + b1[2] * y2) * rdet;
                        const float kr2 = (b2[0] * y0 + b2[1] * y1 + b2[2] * y2) * rdet;
                        const float kr3 = (b3[0] * y0 + b3[1] * y1 + b3[2] * y2) * rdet;
                        const float kr4 = (b4[0] * y0 + b4[1] * y1 + b4[2] * y2) * rdet;
                        const float w0 = c00 * b1[0] + c01 * b1[1] + c02 * b1[2];
                        const float w1 = c01 * b1[0] + c11 * b1[1] + c12 * b1[2];
                        const float w2 = c02 * b1[0] + c12 * b1[1] + c22 * b1[2];
                        const float a11 = (b1[0] * w0 + b1[1] * w1 + b1[2] * w2) * rdet;
                        const float a12 = (b2[0] * w0 + b2[1] * w1 + b2[2] * w2) * rdet;
                        const float a13 = (b3[0] * w0 + b3[1] * w1 + b3[2] * w2) * rdet;
                        const float v0 = c00 * b2[0] + c01 * b2[1] + c02 * b2[2];
                        const float v1 = c01 * b2[0] + c11 * b2[1] + c12 * b2[2];
                        const float v2 = c02 * b2[0] + c12 * b2[1] + c22 * b2[2];
                        const float a22 = (b2[0] * v0 + b2[1] * v1 + b2[2] * v2) * rdet;
                        ls_terms(wgt, kr1, kr2, kr3, kr4, a11, a12, a13, a22, a.ls_literal, t);
                    }
                }
                if (!split) n_pairs += npe;
                npe = 0;
                __syncwarp();   // the list and staged points are reused by the next chunk
            }
        }

        // ---- 5. per point: add the TQ lanes that share it
#pragma unroll
        for (int k = 0; k < NT; ++k)
#pragma unroll
            for (int o = SUB; o < 32; o <<= 1) t[k] += __shfl_xor_sync(FULL, t[k], o);
        float v[NSLOT];
#pragma unroll
        for (int k = 0; k < NSLOT; ++k) v[k] = 0.f;
        if (qi == 0 && sval) {
            if constexpr (MODE == PAIR_EVAL) {
                float Sf = t[0], Su0 = t[1], Su1 = t[2], Su2 = t[3];
                float A00 = t[4], A01 = t[5], A02 = t[6], A11 = t[7], A12 = t[8], A22 = t[9];
                if (ISO) {
                    Su0 *= iso_inv;
                    Su1 *= iso_inv;
                    Su2 *= iso_inv;
                    A00 = A11 = A22 = Sf * iso_inv;
                    A01 = A02 = A12 = 0.f;
                }
                v[0] = Sf;
                // g_omega = -p x S_u, g_v = -S_u (Lemma 1)
                v[1] = -(py * Su2 - pz * Su1);
                v[2] = -(pz * Su0 - px * Su2);
                v[3] = -(px * Su1 - py * Su0);
                v[4] = -Su0;
                v[5] = -Su1;
                v[6] = -Su2;
                // M = J^T S_A J (Eq. 11 with J = [-p^, I])
                jt_s_j(A00, A01, A02, A11, A12, A22, px, py, pz, v + 7);
            } else if constexpr (MODE == PAIR_EXACT) {
                float Su0 = t[1], Su1 = t[2], Su2 = t[3];
                float E[6], SB[9];
                if (ISO) {
                    Su0 *= iso_inv;
                    Su1 *= iso_inv;
                    Su2 *= iso_inv;
                    const float i2 = iso_inv * iso_inv, a = t[0] * iso_inv;
                    E[0] = t[10] * i2 - a;
                    E[1] = t[11] * i2;
                    E[2] = t[12] * i2;
                    E[3] = t[13] * i2 - a;
                    E[4] = t[14] * i2;
                    E[5] = t[15] * i2 - a;
#pragma unroll
                    for (int k = 0; k < 9; ++k) SB[k] = 0.f;
                } else {
#pragma unroll
                    for (int k = 0; k < 6; ++k) E[k] = t[10 + k] - t[4 + k];
#pragma unroll
                    for (int k = 0; k < 9; ++k) SB[k] = t[16 + k];
                }
                v[0] = t[0];
                v[1] = -(py * Su2 - pz * Su1);
                v[2] = -(pz * Su0 - px * Su2);
                v[3] = -(px * Su1 - py * Su0);
                v[4] = -Su0;
                v[5] = -Su1;
                v[6] = -Su2;
                // Q - M = J^T (S_yy - S_A) J
                jt_s_j(E[0], E[1], E[2], E[3], E[4], E[5], px, py, pz, v + 7);
                // C = -S_y^ p^ + p^ S_B, with S_y^ p^ = p S_y^T - (S_y . p) I
                const float pp[3] = {px, py, pz}, sy[3] = {Su0, Su1, Su2};
                const float dp = px * Su0 + py * Su1 + pz * Su2;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    v[28 + c] = -pz * SB[3 + c] + py * SB[6 + c];
                    v[31 + c] = pz * SB[c] - px * SB[6 + c];
                    v[34 + c] = -py * SB[c] + px * SB[3 + c];
                }
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) v[28 + 3 * r + c] += (r == c ? dp : 0.f) - pp[r] * sy[c];
#pragma unroll
                for (int k = 0; k < 9; ++k) v[37 + k] = SB[k];
            } else {
#pragma unroll
                for (int k = 0; k < 5; ++k) v[k] = t[k];
            }
        }
        // compensated sums over the sub-tile's points: transpose through the
        // warp's staging area (free now), lane k adds slot k
        float *tr = reinterpret_cast<float *>(S.pos);
        __syncwarp();
        if (qi == 0)
#pragma unroll
            for (int k = 0; k < NSLOT; ++k) tr[k * (SUB + 1) + si] = v[k];
        __syncwarp();
        // slots 0..31 to the partial row of a.part, 32.. to that of a.part2
#pragma unroll
        for (int hh = 0; hh < (NSLOT + 31) / 32; ++hh) {
            const int k = hh * 32 + lane;
            if (k < NSLOT) {
                float hs = 0.f, ls = 0.f;
#pragma unroll
                for (int i2 = 0; i2 < SUB; ++i2) {
                    const float x = tr[k * (SUB + 1) + i2];
                    const float sm = hs + x;
                    const float bp = sm - hs;
                    ls += (hs - (sm - bp)) + (x - bp);
                    hs = sm;
                }
                float *out = (hh == 0 ? a.part : a.part2) + (size_t)it * 64;
                out[lane] = hs;
                out[32 + lane] = ls;
            }
        }
        const int tp = __reduce_add_sync(FULL, n_pairs);
        const int tk = __reduce_add_sync(FULL, n_kept);
        const int tc = __reduce_add_sync(FULL, n_cand);
        if (lane == 0) {
            long long *cnts = a.counts + (size_t)it * 4;
            cnts[0] = tp;
            cnts[1] = tk;
            cnts[2] = tc;
        }
        __syncwarp();
    }
}

// Work-item packing over the sorted source points (keys: problem << 30 |
// Morton code of the fine voxels of edge rho / 4): one item per sub-tile.
// Start of each point's run of equal keys >> shift (input of a max-scan).
__global__ void k_seg_heads(const unsigned long long *keys, int64_t n, int shift, int *seg) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool head = i == 0 || (keys[i] >> shift) != (keys[i - 1] >> shift);
    seg[i] = head ? (int)i : 0;
}

// Sub-tile heads: every sub-th point of a run of one voxel.
__global__ void k_sub_heads(const int *seg2, int64_t n, int sub, int *sid) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    sid[i] = ((int)i - seg2[i]) % sub == 0 ? 1 : 0;
}

// Each sub-tile head writes its item word: first point << 6 | points.
__global__ void k_sub_count(const int *sid, int64_t n, int *cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    atomicAdd(cnt + sid[i] - 1, 1);
}

__global__ void k_fill_items(const unsigned long long *keys, const int *sid, const int *cnt, int64_t n, int *items,
                             int *item_prob) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (!(i == 0 || sid[i] != sid[i - 1])) return;
    const int it = sid[i] - 1;
    items[it] = (int)(((unsigned)i << 6) | (unsigned)cnt[it]);
    item_prob[it] = (int)(keys[i] >> 30);
}

// Item range of each problem: its points are [off, off + n).
__global__ void k_item_ranges(int np, const int64_t *point_off, const int *n_pts, const int *sid, ProbDev *probs) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int64_t f = point_off[p];
    probs[p].w0 = sid[f] - 1;
    probs[p].w1 = sid[f + n_pts[p] - 1];
}

// One block: each problem's finalize chunks (FIN_CHUNK of its work items
// each) get consecutive indices [c0, c1); *n_chunks receives the total.
constexpr int CHUNK_THREADS = 1024;
__global__ void __launch_bounds__(CHUNK_THREADS) k_chunk_ranges(int np, ProbDev *probs, int *n_chunks) {
    __shared__ int sc[CHUNK_THREADS];
    const int per = (np + CHUNK_THREADS - 1) / CHUNK_THREADS;
    const int p0 = threadIdx.x * per, p1 = min(np, p0 + per);
    int acc = 0;
    for (int p = p0; p < p1; ++p) acc += (probs[p].w1 - probs[p].w0 + FIN_CHUNK - 1) / FIN_CHUNK;
    sc[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 1; o < CHUNK_THREADS; o <<= 1) {
        const int v = threadIdx.x >= o ? sc[threadIdx.x - o] : 0;
        __syncthreads();
        sc[threadIdx.x] += v;
        __syncthreads();
    }
    int c = sc[threadIdx.x] - acc;
    for (int p = p0; p < p1; ++p) {
        probs[p].c0 = c;
        c += (probs[p].w1 - probs[p].w0 + FIN_CHUNK - 1) / FIN_CHUNK;
        probs[p].c1 = c;
    }
    if (threadIdx.x == CHUNK_THREADS - 1) *n_chunks = sc[threadIdx.x];
}

}  // namespace

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
// Dynamic shared memory of one block (its warps' stages), with the opt-in
// above the 48 KB default made once per kernel instance.
template <int MODE, int FD>
constexpr size_t tile_smem_bytes() {
    return PAIR_WARPS * sizeof(StageT<MODE, FD>);
}

template <int MODE, bool ISO, int FD, int SUB>
static cudaError_t tile_smem_optin() {
    static const cudaError_t once = cudaFuncSetAttribute(
        k_tile<MODE, ISO, FD, SUB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem_bytes<MODE, FD>());
    return once;
}

template <int MODE, bool ISO, int FD, int SUB>
static cudaError_t launch_tile_t(const PairArgs &a, int grid, cudaStream_t s) {
    const cudaError_t e = tile_smem_optin<MODE, ISO, FD, SUB>();
    if (e != cudaSuccess) return e;
    k_tile<MODE, ISO, FD, SUB><<<grid, PAIR_WARPS * 32, tile_smem_bytes<MODE, FD>(), s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int MODE, bool ISO, int FD, int SUB>
static int occupancy_t() {
    int nb = 0;
    if (tile_smem_optin<MODE, ISO, FD, SUB>() != cudaSuccess) return 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tile<MODE, ISO, FD, SUB>, PAIR_WARPS * 32,
                                                  tile_smem_bytes<MODE, FD>());
    return nb;
}

// All three passes in all four schedules (the line-search pass of G-CVO-1
// and the G-CVO-E pass run over the same items as the evaluation pass).
#define PAIR_VARIANTS_U(X, M, U) \
    X(M, false, 1, U) X(M, false, 3, U) X(M, false, 7, U) X(M, true, 1, U) X(M, true, 3, U) X(M, true, 7, U)
#define PAIR_VARIANTS_M(X, M) \
    PAIR_VARIANTS_U(X, M, 4) PAIR_VARIANTS_U(X, M, 8) PAIR_VARIANTS_U(X, M, 16) PAIR_VARIANTS_U(X, M, 32)
#define PAIR_VARIANTS(X) \
    PAIR_VARIANTS_M(X, PAIR_EVAL) PAIR_VARIANTS_M(X, PAIR_LINESEARCH) PAIR_VARIANTS_M(X, PAIR_EXACT)

int pair_sub_for(int, int sub) { return sub == 4 || sub == 16 || sub == 32 ? sub : 8; }

// The kernel instance of a feature count: 1, up to 3, or up to 7 channels.
static int fd_class(int fd) { return fd <= 1 ? 1 : fd <= 3 ? 3 : 7; }

int pair_blocks_per_sm(int mode, bool iso, int fd, int sub) {
    sub = pair_sub_for(mode, sub);
#define OCC(M, I, F, U) \
    if (mode == M && iso == I && fd_class(fd) == F && sub == U) return occupancy_t<M, I, F, U>();
    PAIR_VARIANTS(OCC)
#undef OCC
    return 1;
}

cudaError_t launch_pair(const PairArgs &a, int mode, bool iso, int fd, int sub, int grid, cudaStream_t s) {
    sub = pair_sub_for(mode, sub);
#define L(M, I, F, U) \
    if (mode == M && iso == I && fd_class(fd) == F && sub == U) return launch_tile_t<M, I, F, U>(a, grid, s);
    PAIR_VARIANTS(L)
#undef L
    return cudaErrorInvalidValue;
}

gcvo_status pack_items(int np, const unsigned long long *keys, int64_t n, int sub, int level,
                       const int64_t *point_off, const int *n_pts, int *tmp, int *items, int *item_prob,
                       int *d_nitems, ProbDev *probs, int *n_chunks, void *scan_tmp, cudaStream_t s) {
    if (n >= (1LL << 26) || (sub != 4 && sub != 8 && sub != 16 && sub != 32) || level < 0 || level > 3)
        return GCVO_ERR_CAPACITY;
    const size_t stride = ((size_t)n + 63) / 64 * 64;
    int *seg2 = tmp, *sid = tmp + stride, *cnt = tmp + 2 * stride;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    k_seg_heads<<<blocks, 256, 0, s>>>(keys, n, 3 * level, seg2);
    count_launches(1);
    GCVO_CUDA(cudaGetLastError());
    GCVO_TRY(scan_inclusive_max(seg2, n, scan_tmp, s));
    k_sub_heads<<<blocks, 256, 0, s>>>(seg2, n, sub, sid);
    count_launches(1);
    GCVO_CUDA(cudaGetLastError());
    GCVO_TRY(scan_inclusive_sum(sid, n, scan_tmp, s));
    GCVO_CUDA(cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(int), s));
    k_sub_count<<<blocks, 256, 0, s>>>(sid, n, cnt);
    k_fill_items<<<blocks, 256, 0, s>>>(keys, sid, cnt, n, items, item_prob);
    k_item_ranges<<<(np + 127) / 128, 128, 0, s>>>(np, point_off, n_pts, sid, probs);
    k_chunk_ranges<<<1, CHUNK_THREADS, 0, s>>>(np, probs, n_chunks);
    count_launches(4);
    GCVO_CUDA(cudaGetLastError());
    GCVO_CUDA(cudaMemcpyAsync(d_nitems, sid + n - 1, sizeof(int), cudaMemcpyDeviceToDevice, s));
    return GCVO_OK;
}

}  // namespace gcvo
