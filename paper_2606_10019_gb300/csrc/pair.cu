// The per-iteration hot path of Algorithm 1:
//   k_pair     -- transform the source (Alg. 1, "Transform Z with T^-1"),
//                 scan the target voxels around each group of 32 source
//                 points, and accumulate f (Eq. 5), g (Eq. 8) and the
//                 Gauss-Newton matrix M (Eq. 11) -- or, for G-CVO-1, the
//                 line-search polynomial of Eq. (9) -- per group;
//   k_finalize -- FP64 sum of the group partials per problem, change of
//                 frame, connection term (Eq. 12), the 6x6 solve of Eq. (13)
//                 and the update T <- T exp(xi).
// Source grouping (once per call) sorts each source cloud by a Morton code
// of its own voxels and cuts it into groups of at most 32 points that never
// straddle a coarse voxel.
#include <cstring>

#include "common.cuh"
#include "pair.cuh"

namespace gcvo {
namespace {

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier and bulk (TMA) global->shared copies.
// ---------------------------------------------------------------------------
__device__ inline uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ inline void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ inline void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ inline void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ inline float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ inline float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Compensated (TwoSum) warp reduction: returns (hi, lo) in lane 0.
__device__ inline void warp_sum2(float v, float &hi, float &lo) {
    hi = v;
    lo = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float oh = __shfl_down_sync(0xffffffffu, hi, o);
        float ol = __shfl_down_sync(0xffffffffu, lo, o);
        float s = hi + oh;
        float bp = s - hi;
        float err = (hi - (s - bp)) + (oh - bp);
        hi = s;
        lo = lo + ol + err;
    }
}

constexpr float NEG_HALF_LOG2E = -0.72134752044448170368f;  // -1/2 * log2(e)
static_assert(PAIR_CAP * 48 >= 28 * 33 * 4, "epilogue transpose must fit in the staging area");
static_assert(PAIR_CAP <= 256, "queue entries are uint8");
static_assert(PAIR_CAP * 48 >= (32 * 10 * 2 + 64) * 4, "phase-2 slots must fit in the staging area");

struct WarpSmem {
    float4 *pos, *ca, *cb;
    uint8_t *queue;
    uint64_t *bar;
    int2 *seg;      // per packed group: its candidate segment in the staged list
    int *own_off;   // per lane (owner): offset of its queued pairs in the warp list
    int *own_nq;    // per lane: number of queued pairs
    float *own_S;   // per lane: its point's sums (PAIR_OWN_S floats, smem atomics)
    float4 *own_data;  // per lane: p, Sigma', features (and a_k for the line search)
};

__device__ inline WarpSmem warp_smem(unsigned char *base, int w, int mode) {
    WarpSmem s;
    unsigned char *p = base + (size_t)w * pair_warp_smem(mode);
    s.pos = reinterpret_cast<float4 *>(p);
    s.ca = reinterpret_cast<float4 *>(p + PAIR_CAP * 16);
    s.cb = reinterpret_cast<float4 *>(p + PAIR_CAP * 32);
    s.queue = p + PAIR_CAP * 48;
    unsigned char *q = p + PAIR_CAP * 80;
    s.bar = reinterpret_cast<uint64_t *>(q);
    s.seg = reinterpret_cast<int2 *>(q + 16);
    s.own_off = reinterpret_cast<int *>(q + 16 + PAIR_MAX_SUB * 8);
    s.own_nq = s.own_off + 32;
    s.own_S = reinterpret_cast<float *>(s.own_nq + 32);
    s.own_data = reinterpret_cast<float4 *>(s.own_S + 32 * PAIR_OWN_S);
    return s;
}

// ---------------------------------------------------------------------------
// The pair kernel.
//
// One warp owns one group of <= 32 source points (one per lane).  Per
// group: transform the points by T^{-1} (double), take the bounding box of
// the transformed group, and list the target voxel columns (cx, cy) that
// meet the box grown by rho; the occupied voxels of one column over the
// needed cz range are contiguous in the target's sorted order, so each
// column is one run.  Runs are staged into shared memory in chunks of
// PAIR_CAP points by cp.async.bulk copies completing on an mbarrier.  Each
// lane tests every staged point against its own source point (|r| <= rho,
// broadcast loads) and queues the hits; then the lanes evaluate their
// queues (Eq. 7 with the 3x3 adjugate, FP32) and accumulate
//   S_f = sum w_ij,  S_u = sum w_ij Sigma_ij^-1 r_ij,  S_A = sum w_ij Sigma_ij^-1
// with w_ij = c_ij k(x_i, p_j).  Per source point the contribution to
// (f, g, M) follows from p_j, S_f, S_u, S_A (Eq. 8, 11); the warp reduces the
// 28 values with compensated sums and writes one partial per group.
// ---------------------------------------------------------------------------
__device__ inline int ord_enc(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ inline float ord_dec(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

// One anisotropic pair of Eq. (7): Sigma_ij = Sigma_i + Sigma'_j, the adjugate
// and determinant of the 3x3, d^2 = r^T Sigma^-1 r, w = c_ij sigma^2
// exp(-d^2 / 2) (zero beyond the cutoff), and the sums S_f += w,
// S_u += w Sigma^-1 r, S_A += w Sigma^-1 (od*: the source point's p, Sigma',
// features; x, ca, cb: the staged target point).
template <int FD>
__device__ __forceinline__ void pair_aniso(const float4 x, const float4 ca, const float4 cbv, const float4 od0,
                                           const float4 od1, const float4 od2, const float c2, float *t,
                                           int &n_kept) {
    const float r0 = x.x - od0.x, r1 = x.y - od0.y, r2 = x.z - od0.z;
    float cij = x.w * od0.w;
    if (FD > 1) cij += cbv.z * od2.z + cbv.w * od2.w;
    const float s00 = ca.x + od1.x, s01 = ca.y + od1.y, s02 = ca.z + od1.z;
    const float s11 = ca.w + od1.w, s12 = cbv.x + od2.x, s22 = cbv.y + od2.y;
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
    const bool keep = d2 <= c2;
    const float wgt = keep ? cij * ex2_approx(d2 * NEG_HALF_LOG2E) : 0.f;
    n_kept += keep;
    const float wd = wgt * rdet;
    t[0] += wgt;
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

template <int MODE, bool ISO, int FD>
__global__ void __launch_bounds__(PAIR_WARPS * 32, 5) k_pair(PairArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    constexpr int OWN_STRIDE = MODE == PAIR_EVAL ? 3 : 6;   // float4 per lane in own_data
    static_assert(32 * 16 * OWN_STRIDE == (pair_warp_smem(MODE) - (PAIR_CAP * 80 + 16 + PAIR_MAX_SUB * 8 + 64 * 4 +
                                                                 32 * PAIR_OWN_S * 4)),
                  "own_data region size");
    WarpSmem S = warp_smem(smem, w, MODE);
    if (lane == 0) mbar_init(S.bar, 1);
    __syncwarp();
    unsigned parity = 0;
    const int n_items = *a.n_items;

    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(a.work, 1);
        it = __shfl_sync(FULL, it, 0);
        if (it >= n_items) break;
        const int4 item = a.items[it];   // first group, groups, first point, points
        const int prob = a.item_prob[it];
        const ProbDev *P = a.probs + prob;
        if (P->status != 0) {
            // skip the rest of this finished problem's work items in one step
            if (lane == 0) atomicMax(a.work, P->w1);
            continue;
        }
        const GridDev *G = a.grids + prob;
        const int fg = item.x, ng = item.y, j0 = item.z, cnt = item.w;
        const bool act = lane < cnt;
        // the item packs ng spatial groups (consecutive point ranges); lane
        // s < ng holds the first point of group s, every lane finds its group
        const int gs = lane < ng ? a.gstart[fg + lane] - j0 : 0;
        int sub = 0;
        for (int s2 = 1; s2 < ng; ++s2) sub += (__shfl_sync(FULL, gs, s2) <= lane) ? 1 : 0;
        const int first_of_sub = __shfl_sync(FULL, gs, sub);

        // ---- transform (Alg. 1, Z by T^-1) around the first point z_g of
        // the lane's group: p_j - o = R^T (z_j - z_g) + [R^T (z_g - t) - o],
        // the bracket (the anchor) computed in FP64 by the finalize.
        float Rf[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Rf[k] = P->R32[k];
        const float4 anc = a.anchor[fg + sub];
        const int jj = act ? j0 + lane : j0;
        const float4 zg = a.spos[j0 + first_of_sub];
        float4 z = a.spos[jj];
        float4 zb = a.scb[jj];
        const float e0 = z.x - zg.x, e1 = z.y - zg.y, e2 = z.z - zg.z;
        const float px = anc.x + (Rf[0] * e0 + Rf[3] * e1 + Rf[6] * e2);
        const float py = anc.y + (Rf[1] * e0 + Rf[4] * e1 + Rf[7] * e2);
        const float pz = anc.z + (Rf[2] * e0 + Rf[5] * e1 + Rf[8] * e2);
        // Sigma'_j = R^T Sigma_j R
        float q00 = 0.f, q01 = 0.f, q02 = 0.f, q11 = 0.f, q12 = 0.f, q22 = 0.f;
        if (!ISO) {
            float4 za = a.sca[jj];
            float sm[9] = {za.x, za.y, za.z, za.y, za.w, zb.x, za.z, zb.x, zb.y};
            float T1[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    T1[3 * r + c] = sm[3 * r] * Rf[c] + sm[3 * r + 1] * Rf[3 + c] + sm[3 * r + 2] * Rf[6 + c];
            q00 = Rf[0] * T1[0] + Rf[3] * T1[3] + Rf[6] * T1[6];
            q01 = Rf[0] * T1[1] + Rf[3] * T1[4] + Rf[6] * T1[7];
            q02 = Rf[0] * T1[2] + Rf[3] * T1[5] + Rf[6] * T1[8];
            q11 = Rf[1] * T1[1] + Rf[4] * T1[4] + Rf[7] * T1[7];
            q12 = Rf[1] * T1[2] + Rf[4] * T1[5] + Rf[7] * T1[8];
            q22 = Rf[2] * T1[2] + Rf[5] * T1[5] + Rf[8] * T1[8];
        }
        const float sg = P->sigma2;
        const float l0 = sg * z.w;
        const float l1 = FD > 1 ? sg * zb.z : 0.f;
        const float l2 = FD > 1 ? sg * zb.w : 0.f;
        const float rho2 = P->rho2, c2 = P->c2, iso_inv = P->iso_inv;

        // line-search direction powers a_k (G-CVO-1 second pass)
        float a1[3], a2[3], a3[3], a4[3];
        if (MODE == PAIR_LINESEARCH) {
            float om0 = P->dir32[0], om1 = P->dir32[1], om2 = P->dir32[2];
            a1[0] = om1 * pz - om2 * py + P->dir32[3];
            a1[1] = om2 * px - om0 * pz + P->dir32[4];
            a1[2] = om0 * py - om1 * px + P->dir32[5];
#define CROSS_W(dst, src)                            \
    dst[0] = om1 * src[2] - om2 * src[1];            \
    dst[1] = om2 * src[0] - om0 * src[2];            \
    dst[2] = om0 * src[1] - om1 * src[0];
            CROSS_W(a2, a1)
            CROSS_W(a3, a2)
            CROSS_W(a4, a3)
#undef CROSS_W
        }

        // ---- owner tables: this lane's point data for the balanced phase 2,
        // and its sums (zeroed)
        S.own_data[lane * OWN_STRIDE + 0] = make_float4(px, py, pz, l0);
        S.own_data[lane * OWN_STRIDE + 1] = make_float4(q00, q01, q02, q11);
        S.own_data[lane * OWN_STRIDE + 2] = make_float4(q12, q22, l1, l2);
        if (MODE == PAIR_LINESEARCH) {
            S.own_data[lane * OWN_STRIDE + 3] = make_float4(a1[0], a1[1], a1[2], a2[0]);
            S.own_data[lane * OWN_STRIDE + 4] = make_float4(a2[1], a2[2], a3[0], a3[1]);
            S.own_data[lane * OWN_STRIDE + 5] = make_float4(a3[2], a4[0], a4[1], a4[2]);
        }
#pragma unroll
        for (int k = 0; k < PAIR_OWN_S; ++k) S.own_S[lane * PAIR_OWN_S + k] = 0.f;

        // ---- bounding box of the lane's transformed group
        const unsigned smask = __match_any_sync(FULL, sub);
        float bmin[3], bmax[3];
        {
            const float pp[3] = {px, py, pz};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                bmin[k] = ord_dec(__reduce_min_sync(smask, ord_enc(act ? pp[k] : INFINITY)));
                bmax[k] = ord_dec(__reduce_max_sync(smask, ord_enc(act ? pp[k] : -INFINITY)));
            }
        }
        const float rho = sqrtf(rho2);
        const float h = G->h, ih = G->inv_h;
        // culling radius: rho plus a margin for the float voxel assignment
        const float rc = rho * 1.0001f + 1e-5f * h;
        const float rc2 = rc * rc;
        // voxel ranges of the lane's group (an empty range has hi < lo)
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
        const int my_cols = empty ? 0 : (hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1);
        // lane s < ng: column count of group s and its exclusive offset
        int cols_s = __shfl_sync(FULL, my_cols, gs);
        if (lane >= ng) cols_s = 0;
        int cinc = cols_s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(FULL, cinc, o);
            if (lane >= o) cinc += u;
        }
        const int coff_s = cinc - cols_s;
        const int total_cols = __shfl_sync(FULL, cinc, 31);

        // ---- accumulators
        float Sf = 0.f, Su0 = 0.f, Su1 = 0.f, Su2 = 0.f;
        float A00 = 0.f, A01 = 0.f, A02 = 0.f, A11 = 0.f, A12 = 0.f, A22 = 0.f;
        float L1 = 0.f, L2 = 0.f, L3 = 0.f, L4 = 0.f;  // line-search sums (f in Sf)
        int n_pairs = 0, n_kept = 0, n_cand = 0;

        const int dy = G->dims[1], dzs = G->dims[2];
        for (int cb0 = 0; cb0 < total_cols; cb0 += 32) {
            // ---- one (group, column) per lane.  A column (cx, cy) is kept
            // when its xy rectangle lies within rho of the group box, and its
            // cz range shrinks with that distance; the occupied voxels of the
            // range are contiguous in the sorted target: one run per column.
            const int c = cb0 + lane;
            const bool cvalid = c < total_cols;
            int cs = 0;
            for (int s2 = 1; s2 < ng; ++s2) cs += (__shfl_sync(FULL, coff_s, s2) <= c) ? 1 : 0;
            const int src_lane = __shfl_sync(FULL, gs, cs);          // a lane of group cs
            const int cloc = c - __shfl_sync(FULL, coff_s, cs);
            float cbmin[3], cbmax[3];
            int clo[3], chi[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                cbmin[k] = __shfl_sync(FULL, bmin[k], src_lane);
                cbmax[k] = __shfl_sync(FULL, bmax[k], src_lane);
                clo[k] = __shfl_sync(FULL, lo[k], src_lane);
                chi[k] = __shfl_sync(FULL, hi[k], src_lane);
            }
            int rs = 0, rl = 0;
            if (cvalid) {
                const int ncy = chi[1] - clo[1] + 1;
                const int cx = clo[0] + cloc / ncy, cy = clo[1] + cloc % ncy;
                const float x0 = G->corner[0] + (float)cx * h, y0 = G->corner[1] + (float)cy * h;
                const float ddx = fmaxf(0.0f, fmaxf(x0 - cbmax[0], cbmin[0] - (x0 + h)));
                const float ddy = fmaxf(0.0f, fmaxf(y0 - cbmax[1], cbmin[1] - (y0 + h)));
                const float d2xy = ddx * ddx + ddy * ddy;
                if (d2xy <= rc2) {
                    const float ez = sqrtf(rc2 - d2xy);
                    const int czl = max(clo[2], (int)floorf(fmaxf((cbmin[2] - ez - G->corner[2]) * ih, -1.0f)));
                    const int czh = min(chi[2], (int)floorf(fminf((cbmax[2] + ez - G->corner[2]) * ih, (float)dzs)));
                    // the column's occupied voxels, sorted by cz: keep [czl, czh]
                    const int2 cr = G->col_range[cx * dy + cy];
                    int first = -1, last = -1;
                    for (int cc = cr.x; cc < cr.y; ++cc) {
                        int zc = __ldg(G->cell_z + cc);
                        if (zc >= czl) {
                            if (zc <= czh) first = cc;
                            break;
                        }
                    }
                    if (first >= 0) {
                        last = first;
                        for (int cc = first + 1; cc < cr.y; ++cc) {
                            if (__ldg(G->cell_z + cc) > czh) break;
                            last = cc;
                        }
                        rs = __ldg(G->cell_start + first);
                        rl = __ldg(G->cell_start + last + 1) - rs;
                    }
                }
            }
            // exclusive offsets of the runs; the runs of one group are
            // contiguous, so each group owns one segment [seg_lo, seg_hi)
            int incl = rl;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += u;
            }
            const int total = __shfl_sync(FULL, incl, 31);
            const int off = incl - rl;
            {
                const unsigned pm = __match_any_sync(FULL, cvalid ? cs : -1);
                const int slo = __reduce_min_sync(pm, off);
                const int shi = __reduce_max_sync(pm, incl);
                if (lane < ng) S.seg[lane] = make_int2(0, 0);
                __syncwarp();
                if (cvalid && lane == __ffs(pm) - 1) S.seg[cs] = make_int2(slo, shi);
                __syncwarp();
            }
            const int2 myseg = S.seg[sub];

            for (int base = 0; base < total; base += PAIR_CAP) {
                const int m = min(PAIR_CAP, total - base);
                // ---- stage the chunk [base, base + m) of the runs (TMA bulk copies)
                fence_proxy_async_smem();
                if (lane == 0) mbar_arrive_expect_tx(S.bar, (unsigned)m * 48u);
                __syncwarp();
                {
                    int s0 = max(off, base), s1 = min(off + rl, base + m);
                    if (s1 > s0) {
                        int src = rs + (s0 - off), dst = s0 - base;
                        unsigned bytes = (unsigned)(s1 - s0) * 16u;
                        bulk_g2s(S.pos + dst, G->pos + src, bytes, S.bar);
                        bulk_g2s(S.ca + dst, G->ca + src, bytes, S.bar);
                        bulk_g2s(S.cb + dst, G->cb + src, bytes, S.bar);
                    }
                }
                {
                    // bounded wait; the exit decision is warp-uniform
                    int spin = 0;
                    bool all_done = false;
                    for (;;) {
                        bool done = mbar_try_wait(S.bar, parity);
                        all_done = __all_sync(FULL, done);
                        if (all_done || ++spin > (1 << 22)) break;
                    }
                    if (!all_done) {
                        if (lane == 0) atomicOr(a.status_word, DEV_ERR_TIMEOUT);
                        return;
                    }
                    parity ^= 1u;
                }

                // ---- phase 1: |r| <= rho test against the lane's own
                // group segment of the chunk (a broadcast load per group)
                const int k0 = max(myseg.x, base), k1 = min(myseg.y, base + m);
                const int len = act ? max(0, k1 - k0) : 0;
                const int tmax1 = __reduce_max_sync(FULL, len);
                n_cand += len;
                int nq = 0;
                const int kb0 = k0 - base;
                for (int t = 0; t < tmax1; t += 4) {
                    float dd[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int tt = t + u;
                        const int kk = len > 0 ? kb0 + min(tt, len - 1) : 0;
                        const float4 x = S.pos[kk];
                        const float rx = x.x - px, ry = x.y - py, rz = x.z - pz;
                        dd[u] = tt < len ? rx * rx + ry * ry + rz * rz : INFINITY;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (dd[u] <= rho2) {
                            S.queue[nq * 32 + lane] = (uint8_t)(kb0 + t + u);
                            ++nq;
                        }
                    }
                }
                n_pairs += nq;

                // ---- phase 2: the warp's queued pairs in owner-major order,
                // split evenly over the lanes.  A lane accumulates locally
                // while the owner stays the same and adds its sums into the
                // owner's shared-memory slot when the owner changes.
                int qinc = nq;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int u = __shfl_up_sync(FULL, qinc, o);
                    if (lane >= o) qinc += u;
                }
                const int Q = __shfl_sync(FULL, qinc, 31);
                S.own_off[lane] = qinc - nq;
                S.own_nq[lane] = nq;
                __syncwarp();
                {
                    const int share = (Q + 31) >> 5;
                    int e = lane * share;
                    const int e_end = min(e + share, Q);
                    // owner of entry e: the last lane with a non-empty queue
                    // starting at or before e
                    int ow = 0;
                    for (int l2 = 0; l2 < 32; ++l2)
                        if (S.own_nq[l2] > 0 && S.own_off[l2] <= e) ow = l2;
                    int q = e - S.own_off[ow];
                    int ow_end = S.own_off[ow] + S.own_nq[ow];
                    float4 od0 = S.own_data[ow * OWN_STRIDE + 0];
                    float4 od1 = S.own_data[ow * OWN_STRIDE + 1];
                    float4 od2 = S.own_data[ow * OWN_STRIDE + 2];
                    float4 od3, od4, od5;
                    if (MODE == PAIR_LINESEARCH) {
                        od3 = S.own_data[ow * OWN_STRIDE + 3];
                        od4 = S.own_data[ow * OWN_STRIDE + 4];
                        od5 = S.own_data[ow * OWN_STRIDE + 5];
                    }
                    // this lane's range splits into owner segments: the first
                    // is kept in fS until the range ends, segments wholly inside
                    // the range belong to this lane alone and go straight to the
                    // owner's sums, the last stays in t
                    float t[10], fS[10];
#pragma unroll
                    for (int k = 0; k < 10; ++k) t[k] = fS[k] = 0.f;
                    int seg = 0, f_owner = -1;
                    while (e < e_end) {
                        if (e >= ow_end) {
                            if (MODE == PAIR_EVAL) {
                                if (seg == 0) {
                                    f_owner = ow;
#pragma unroll
                                    for (int k = 0; k < 10; ++k) fS[k] = t[k];
                                } else {
                                    float *dst = S.own_S + ow * PAIR_OWN_S;
#pragma unroll
                                    for (int k = 0; k < 10; ++k) dst[k] += t[k];
                                }
#pragma unroll
                                for (int k = 0; k < 10; ++k) t[k] = 0.f;
                            }
                            ++seg;
                            do {
                                ++ow;
                            } while (S.own_nq[ow] == 0);
                            q = 0;
                            ow_end = S.own_off[ow] + S.own_nq[ow];
                            od0 = S.own_data[ow * OWN_STRIDE + 0];
                            od1 = S.own_data[ow * OWN_STRIDE + 1];
                            od2 = S.own_data[ow * OWN_STRIDE + 2];
                            if (MODE == PAIR_LINESEARCH) {
                                od3 = S.own_data[ow * OWN_STRIDE + 3];
                                od4 = S.own_data[ow * OWN_STRIDE + 4];
                                od5 = S.own_data[ow * OWN_STRIDE + 5];
                            }
                        }
                        const int seg_end = min(e_end, ow_end);
                        if (MODE == PAIR_EVAL && !ISO) {
                            for (; e < seg_end; ++e, ++q) {
                                const int k0 = S.queue[q * 32 + ow];
                                pair_aniso<FD>(S.pos[k0], S.ca[k0], S.cb[k0], od0, od1, od2, c2, t, n_kept);
                            }
                            continue;
                        }
                        for (; e < seg_end; ++e, ++q) {
                            const int k = S.queue[q * 32 + ow];
                            const float4 x = S.pos[k];
                            const float r0 = x.x - od0.x, r1 = x.y - od0.y, r2 = x.z - od0.z;
                            float cij = x.w * od0.w;
                            if (FD > 1) {
                                const float4 b = S.cb[k];
                                cij += b.z * od2.z + b.w * od2.w;
                            }
                            if (ISO) {
                                const float d2 = (r0 * r0 + r1 * r1 + r2 * r2) * iso_inv;
                                const bool keep = d2 <= c2;
                                const float wgt = keep ? cij * ex2_approx(d2 * NEG_HALF_LOG2E) : 0.f;
                                n_kept += keep;
                                if (MODE == PAIR_EVAL) {
                                    t[0] += wgt;
                                    t[1] += wgt * r0;
                                    t[2] += wgt * r1;
                                    t[3] += wgt * r2;
                                } else {
                                    const float b1[3] = {od3.x, od3.y, od3.z}, b2[3] = {od3.w, od4.x, od4.y},
                                                b3[3] = {od4.z, od4.w, od5.x}, b4[3] = {od5.y, od5.z, od5.w};
                                    // A = I / ell^2
                                    const float kr1 = (b1[0] * r0 + b1[1] * r1 + b1[2] * r2) * iso_inv;
                                    const float kr2 = (b2[0] * r0 + b2[1] * r1 + b2[2] * r2) * iso_inv;
                                    const float kr3 = (b3[0] * r0 + b3[1] * r1 + b3[2] * r2) * iso_inv;
                                    const float kr4 = (b4[0] * r0 + b4[1] * r1 + b4[2] * r2) * iso_inv;
                                    const float a11 = (b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2]) * iso_inv;
                                    const float a12 = (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2]) * iso_inv;
                                    const float a13 = (b1[0] * b3[0] + b1[1] * b3[1] + b1[2] * b3[2]) * iso_inv;
                                    const float a22 = (b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]) * iso_inv;
                                    float be, ga, de, ep;
                                    if (!a.ls_literal) {
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
                                    Sf += wgt;
                                    L1 += wgt * be;
                                    L2 += wgt * (ga + 0.5f * be * be);
                                    L3 += wgt * (de + be * ga + be * be * be * (1.f / 6.f));
                                    L4 += wgt * (ep + be * de + 0.5f * be * be * ga + 0.5f * ga * ga +
                                                 be * be * be * be * (1.f / 24.f));
                                }
                            } else {
                                const float4 ca = S.ca[k];
                                const float4 cbv = S.cb[k];
                                const float s00 = ca.x + od1.x, s01 = ca.y + od1.y, s02 = ca.z + od1.z;
                                const float s11 = ca.w + od1.w, s12 = cbv.x + od2.x, s22 = cbv.y + od2.y;
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
                                const bool keep = d2 <= c2;
                                const float wgt = keep ? cij * ex2_approx(d2 * NEG_HALF_LOG2E) : 0.f;
                                n_kept += keep;
                                const float b1[3] = {od3.x, od3.y, od3.z}, b2[3] = {od3.w, od4.x, od4.y},
                                            b3[3] = {od4.z, od4.w, od5.x}, b4[3] = {od5.y, od5.z, od5.w};
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
                                float be, ga, de, ep;
                                if (!a.ls_literal) {
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
                                Sf += wgt;
                                L1 += wgt * be;
                                L2 += wgt * (ga + 0.5f * be * be);
                                L3 += wgt * (de + be * ga + be * be * be * (1.f / 6.f));
                                L4 += wgt * (ep + be * de + 0.5f * be * be * ga + 0.5f * ga * ga +
                                             be * be * be * be * (1.f / 24.f));
                            }
                        }
                    }
                    if (MODE == PAIR_EVAL) {
                        // first / last segment sums to per-lane slots in the
                        // staging area (free once every lane is done with it),
                        // then each owner adds the slots of the lanes that
                        // covered its entries, in lane order
                        __syncwarp();
                        float *fslot = reinterpret_cast<float *>(S.pos);
                        float *lslot = fslot + 32 * 10;
                        int *fown = reinterpret_cast<int *>(lslot + 32 * 10);
                        int *lown = fown + 32;
                        const bool had = lane * share < Q;
                        if (had && seg == 0) {
#pragma unroll
                            for (int k = 0; k < 10; ++k) fslot[lane * 10 + k] = t[k];
                            fown[lane] = ow;
                            lown[lane] = -1;
                        } else if (had) {
#pragma unroll
                            for (int k = 0; k < 10; ++k) {
                                fslot[lane * 10 + k] = fS[k];
                                lslot[lane * 10 + k] = t[k];
                            }
                            fown[lane] = f_owner;
                            lown[lane] = ow;
                        } else {
                            fown[lane] = -1;
                            lown[lane] = -1;
                        }
                        __syncwarp();
                        if (nq > 0) {
                            const int off_me = S.own_off[lane];
                            const int la = off_me / share, lb = (off_me + nq - 1) / share;
                            float acc[10];
#pragma unroll
                            for (int k = 0; k < 10; ++k) acc[k] = 0.f;
                            for (int l2 = la; l2 <= lb; ++l2) {
                                if (fown[l2] == lane)
#pragma unroll
                                    for (int k = 0; k < 10; ++k) acc[k] += fslot[l2 * 10 + k];
                                if (lown[l2] == lane)
#pragma unroll
                                    for (int k = 0; k < 10; ++k) acc[k] += lslot[l2 * 10 + k];
                            }
                            float *dst = S.own_S + lane * PAIR_OWN_S;
#pragma unroll
                            for (int k = 0; k < 10; ++k) dst[k] += acc[k];
                        }
                    }
                }
                __syncwarp();
            }
        }

        // ---- per-source-point epilogue and warp reduction
        float v[PAIR_SLOTS];
#pragma unroll
        for (int k = 0; k < PAIR_SLOTS; ++k) v[k] = 0.f;
        if (MODE == PAIR_EVAL) {
            // this lane's point sums, assembled by the balanced phase 2
            Sf = S.own_S[lane * PAIR_OWN_S + 0];
            Su0 = S.own_S[lane * PAIR_OWN_S + 1];
            Su1 = S.own_S[lane * PAIR_OWN_S + 2];
            Su2 = S.own_S[lane * PAIR_OWN_S + 3];
            A00 = S.own_S[lane * PAIR_OWN_S + 4];
            A01 = S.own_S[lane * PAIR_OWN_S + 5];
            A02 = S.own_S[lane * PAIR_OWN_S + 6];
            A11 = S.own_S[lane * PAIR_OWN_S + 7];
            A12 = S.own_S[lane * PAIR_OWN_S + 8];
            A22 = S.own_S[lane * PAIR_OWN_S + 9];
        }
        if (MODE == PAIR_EVAL ? act : true) {
            if (MODE == PAIR_EVAL) {
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
                // M = [[P^T S_A P, P S_A], [-S_A P, S_A]], P = p^ (Eq. 11 with J = [-p^, I])
                float B00 = A01 * pz - A02 * py, B01 = -A00 * pz + A02 * px, B02 = A00 * py - A01 * px;
                float B10 = A11 * pz - A12 * py, B11 = -A01 * pz + A12 * px, B12 = A01 * py - A11 * px;
                float B20 = A12 * pz - A22 * py, B21 = -A02 * pz + A22 * px, B22 = A02 * py - A12 * px;
                float W00 = pz * B10 - py * B20, W01 = pz * B11 - py * B21, W02 = pz * B12 - py * B22;
                float W11 = -pz * B01 + px * B21, W12 = -pz * B02 + px * B22;
                float W22 = py * B02 - px * B12;
                float X00 = -pz * A01 + py * A02, X01 = -pz * A11 + py * A12, X02 = -pz * A12 + py * A22;
                float X10 = pz * A00 - px * A02, X11 = pz * A01 - px * A12, X12 = pz * A02 - px * A22;
                float X20 = -py * A00 + px * A01, X21 = -py * A01 + px * A11, X22 = -py * A02 + px * A12;
                // upper triangle of M, row-major
                v[7] = W00; v[8] = W01; v[9] = W02; v[10] = X00; v[11] = X01; v[12] = X02;
                v[13] = W11; v[14] = W12; v[15] = X10; v[16] = X11; v[17] = X12;
                v[18] = W22; v[19] = X20; v[20] = X21; v[21] = X22;
                v[22] = A00; v[23] = A01; v[24] = A02;
                v[25] = A11; v[26] = A12;
                v[27] = A22;
            } else {
                v[0] = Sf;
                v[1] = L1;
                v[2] = L2;
                v[3] = L3;
                v[4] = L4;
            }
        }
        const int nslot = MODE == PAIR_EVAL ? 28 : 5;
        // compensated reduction over the lanes: transpose through shared
        // memory (the staging area is free now), then lane k sums slot k
        float *red = reinterpret_cast<float *>(S.pos);
#pragma unroll
        for (int k = 0; k < PAIR_SLOTS; ++k)
            if (k < nslot) red[k * 33 + lane] = v[k];
        __syncwarp();
        float *out = a.part + (size_t)it * 64;
        if (lane < nslot) {
            float hi = 0.f, lo = 0.f;
#pragma unroll 8
            for (int i = 0; i < 32; ++i) {
                float x = red[lane * 33 + i];
                float sm = hi + x;
                float bp = sm - hi;
                lo += (hi - (sm - bp)) + (x - bp);
                hi = sm;
            }
            out[lane] = hi;
            out[32 + lane] = lo;
        }
        int tp = __reduce_add_sync(0xffffffffu, n_pairs);
        int tk = __reduce_add_sync(0xffffffffu, n_kept);
        int tc = __reduce_add_sync(0xffffffffu, n_cand);
        if (lane == 0) {
            long long *cnts = a.counts + (size_t)it * 4;
            cnts[0] = tp;
            cnts[1] = tk;
            cnts[2] = tc;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// FP64 finalize, one block per problem.
// ---------------------------------------------------------------------------

__device__ void hat3d(const double w[3], double W[9]) {
    W[0] = 0;     W[1] = -w[2]; W[2] = w[1];
    W[3] = w[2];  W[4] = 0;     W[5] = -w[0];
    W[6] = -w[1]; W[7] = w[0];  W[8] = 0;
}

// exp of a twist (omega, v): Rodrigues rotation and V-matrix translation,
// with series coefficients for small angles.
__device__ void exp_twist(const double xi[6], double Rout[9], double tout[3]) {
    double th2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
    double th = sqrt(th2);
    double A, B, C;
    if (th < 1e-4) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        double s, c;
        sincos(th, &s, &c);
        A = s / th;
        B = (1.0 - c) / th2;
        C = (th - s) / (th2 * th);
    }
    double W[9], W2[9];
    hat3d(xi, W);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) W2[3 * r + c] = W[3 * r] * W[c] + W[3 * r + 1] * W[3 + c] + W[3 * r + 2] * W[6 + c];
    for (int k = 0; k < 9; ++k) {
        double I = (k % 4 == 0) ? 1.0 : 0.0;
        Rout[k] = I + A * W[k] + B * W2[k];
    }
    for (int r = 0; r < 3; ++r) {
        double s = 0;
        for (int c = 0; c < 3; ++c) {
            double I = r == c ? 1.0 : 0.0;
            s += (I + B * W[3 * r + c] + C * W2[3 * r + c]) * xi[3 + c];
        }
        tout[r] = s;
    }
}

// Solve (M - Gamma) xi = g (Eq. 13).  M is symmetric positive definite for a
// problem with overlap; Gamma (Eq. 12) has non-zero entries only in its first
// three columns, Gamma = Gc E^T with Gc = [-1/2 g_omega^; -g_v^] (6x3) and
// E = [I3; 0].  With the Cholesky factor of M, y = M^-1 g and Z = M^-1 Gc,
// the Sherman-Morrison-Woodbury identity gives
//   xi = y + Z (I3 - E^T Z)^-1 E^T y.
// Falls back to partial-pivot LU of M - Gamma when M is not positive
// definite.  Returns 0, or 1 when both fail.
__device__ int solve_gn(const double M[36], const double g[6], double xi[6]) {
    double Gc[18];
#pragma unroll
    for (int r = 0; r < 18; ++r) Gc[r] = 0.0;
    // Gc = [-1/2 g_omega^ ; -g_v^]
    Gc[1] = 0.5 * g[2];  Gc[2] = -0.5 * g[1];
    Gc[3] = -0.5 * g[2]; Gc[5] = 0.5 * g[0];
    Gc[6] = 0.5 * g[1];  Gc[7] = -0.5 * g[0];
    Gc[10] = g[5];  Gc[11] = -g[4];
    Gc[12] = -g[5]; Gc[14] = g[3];
    Gc[15] = g[4];  Gc[16] = -g[3];
    // Cholesky M = L L^T (inverse diagonal kept)
    double L[36], id[6];
    bool spd = true;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            double sm = M[6 * i + j];
#pragma unroll
            for (int k = 0; k < j; ++k) sm -= L[6 * i + k] * L[6 * j + k];
            if (i == j) {
                spd = spd && (sm > 0.0);
                double r = sqrt(fmax(sm, 1e-300));
                L[6 * i + i] = r;
                id[i] = 1.0 / r;
            } else {
                L[6 * i + j] = sm * id[j];
            }
        }
    }
    if (spd) {
        // X = M^-1 [g, Gc] (6 x 4)
        double X[24];
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            X[4 * r] = g[r];
#pragma unroll
            for (int c = 0; c < 3; ++c) X[4 * r + 1 + c] = Gc[3 * r + c];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                double sm = X[4 * i + c];
#pragma unroll
                for (int k = 0; k < i; ++k) sm -= L[6 * i + k] * X[4 * k + c];
                X[4 * i + c] = sm * id[i];
            }
#pragma unroll
            for (int i = 5; i >= 0; --i) {
                double sm = X[4 * i + c];
#pragma unroll
                for (int k = i + 1; k < 6; ++k) sm -= L[6 * k + i] * X[4 * k + c];
                X[4 * i + c] = sm * id[i];
            }
        }
        // K = I3 - E^T Z, w = K^-1 E^T y (Cramer), xi = y + Z w
        double K[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) K[3 * r + c] = (r == c ? 1.0 : 0.0) - X[4 * r + 1 + c];
        double c00 = K[4] * K[8] - K[5] * K[7], c01 = K[5] * K[6] - K[3] * K[8], c02 = K[3] * K[7] - K[4] * K[6];
        double detK = K[0] * c00 + K[1] * c01 + K[2] * c02;
        double kn = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) kn = fmax(kn, fabs(K[k]));
        if (fabs(detK) > 1e-12 * kn * kn * kn) {
            double idet = 1.0 / detK;
            double y0 = X[0], y1 = X[4], y2 = X[8];
            // inverse of K by its adjugate
            double w0 = (c00 * y0 + (K[2] * K[7] - K[1] * K[8]) * y1 + (K[1] * K[5] - K[2] * K[4]) * y2) * idet;
            double w1 = (c01 * y0 + (K[0] * K[8] - K[2] * K[6]) * y1 + (K[2] * K[3] - K[0] * K[5]) * y2) * idet;
            double w2 = (c02 * y0 + (K[1] * K[6] - K[0] * K[7]) * y1 + (K[0] * K[4] - K[1] * K[3]) * y2) * idet;
#pragma unroll
            for (int r = 0; r < 6; ++r) xi[r] = X[4 * r] + X[4 * r + 1] * w0 + X[4 * r + 2] * w1 + X[4 * r + 3] * w2;
            return 0;
        }
    }
    // LU with partial pivoting of A = M - Gamma (Gamma = Gc in the first 3 columns)
    double A[42];
    for (int r = 0; r < 6; ++r) {
        for (int c = 0; c < 6; ++c) A[7 * r + c] = M[6 * r + c] - (c < 3 ? Gc[3 * r + c] : 0.0);
        A[7 * r + 6] = g[r];
    }
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (fabs(A[7 * r + c]) > fabs(A[7 * piv + c])) piv = r;
        if (A[7 * piv + c] == 0.0) return 1;
        if (piv != c)
            for (int k = 0; k < 7; ++k) {
                double tmp = A[7 * c + k];
                A[7 * c + k] = A[7 * piv + k];
                A[7 * piv + k] = tmp;
            }
        for (int r = c + 1; r < 6; ++r) {
            double f = A[7 * r + c] / A[7 * c + c];
            for (int k = c; k < 7; ++k) A[7 * r + k] -= f * A[7 * c + k];
        }
    }
    for (int r = 5; r >= 0; --r) {
        double sm = A[7 * r + 6];
        for (int k = r + 1; k < 6; ++k) sm -= A[7 * r + k] * xi[k];
        xi[r] = sm / A[7 * r + r];
    }
    return 0;
}

// Smallest positive real root of the cubic d3 t^3 + d2 t^2 + d1 t + d0
// (G'(t) of Eq. 9), or -1 if none.  Closed forms (trigonometric / Cardano)
// for the cubic, then two Newton polishing steps per root.
__device__ double smallest_pos_root(double d3, double d2, double d1, double d0) {
    double roots[3];
    int nr = 0;
    double sc = fmax(fmax(fabs(d3), fabs(d2)), fmax(fabs(d1), fabs(d0)));
    if (sc == 0.0) return -1.0;
    if (fabs(d3) <= 1e-14 * sc) {
        if (fabs(d2) <= 1e-14 * sc) {
            if (d1 != 0.0) roots[nr++] = -d0 / d1;
        } else {
            double disc = d1 * d1 - 4.0 * d2 * d0;
            if (disc >= 0.0) {
                double sq = sqrt(disc);
                double qq = -0.5 * (d1 + copysign(sq, d1));
                if (qq != 0.0) roots[nr++] = d0 / qq;
                roots[nr++] = qq / d2;
            }
        }
    } else {
        double a = d2 / d3, b = d1 / d3, c = d0 / d3;
        double Q = (a * a - 3.0 * b) / 9.0;
        double Rr = (2.0 * a * a * a - 9.0 * a * b + 27.0 * c) / 54.0;
        double Q3 = Q * Q * Q;
        if (Rr * Rr < Q3) {
            double th = acos(fmin(fmax(Rr / sqrt(Q3), -1.0), 1.0));
            double m = -2.0 * sqrt(Q);
            roots[nr++] = m * cos(th / 3.0) - a / 3.0;
            roots[nr++] = m * cos((th + 2.0 * M_PI) / 3.0) - a / 3.0;
            roots[nr++] = m * cos((th - 2.0 * M_PI) / 3.0) - a / 3.0;
        } else {
            double A = -copysign(cbrt(fabs(Rr) + sqrt(Rr * Rr - Q3)), Rr);
            double B = A != 0.0 ? Q / A : 0.0;
            roots[nr++] = (A + B) - a / 3.0;
        }
    }
    double best = -1.0;
    for (int k = 0; k < nr; ++k) {
        double t = roots[k];
        for (int it = 0; it < 2; ++it) {
            double p = ((d3 * t + d2) * t + d1) * t + d0;
            double dp = (3.0 * d3 * t + 2.0 * d2) * t + d1;
            if (dp != 0.0) t -= p / dp;
        }
        if (t > 0.0 && (best < 0.0 || t < best)) best = t;
    }
    return best;
}

__device__ inline void set_inactive(ProbDev *P, int st, int *n_active) {
    P->status = st;
    atomicSub(n_active, 1);
}

__device__ inline void apply_step(ProbDev *P, const double xi[6], gcvo_iter_log *lg, const FinalizeArgs &a,
                                  int it) {
    double l1 = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) l1 += fabs(xi[k]);
    double dR[9], dt[3];
    exp_twist(xi, dR, dt);
    double Rn[9], tn[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Rn[3 * r + c] = P->T[3 * r] * dR[c] + P->T[3 * r + 1] * dR[3 + c] + P->T[3 * r + 2] * dR[6 + c];
        tn[r] = P->T[3 * r] * dt[0] + P->T[3 * r + 1] * dt[1] + P->T[3 * r + 2] * dt[2] + P->T[9 + r];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) P->T[k] = Rn[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) P->T[9 + k] = tn[k];
    if (lg) {
#pragma unroll
        for (int k = 0; k < 6; ++k) lg->xi[k] = xi[k];
        lg->xi_l1 = l1;
    }
    P->iter = it + 1;
    if (!(l1 == l1)) set_inactive(P, -(int)GCVO_ERR_NONFINITE, a.n_active);
    else if (l1 < a.eps_tol) set_inactive(P, 1, a.n_active);
    else if (it + 1 >= a.k_max) set_inactive(P, 2, a.n_active);
}

// The per-problem FP64 step (one thread): returns 1 when the pose changed
// and the problem stays active, so the group anchors must be refreshed.
__device__ int finalize_thread0(const FinalizeArgs &a, int prob, ProbDev *P, const double *tot,
                                const long long *ctot) {
    const GridDev *G = a.grids + prob;
    const double o0 = G->origin[0], o1 = G->origin[1], o2 = G->origin[2];
    const int it = P->iter;
    gcvo_iter_log *lg = a.logs ? a.logs + (size_t)prob * a.k_max + it : nullptr;

    if (a.mode == FIN_LINESEARCH) {
        // G(t) ~ sum_k c_k t^k along xi = g (Eq. 9).  c_1 = dG/dt(0) = <g, g>
        // exactly; it is taken from the FP64 gradient rather than the FP32
        // pair sums, which cancel towards zero near the optimum.
        double c1 = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) c1 += P->dir[k] * P->dir[k];
        double c2 = tot[2], c3 = tot[3], c4 = tot[4];
        double ts = smallest_pos_root(4.0 * c4, 3.0 * c3, 2.0 * c2, c1);
        double mu = ts > a.mu0 ? ts : a.mu0;
        double xi[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) xi[k] = mu * P->dir[k];
        apply_step(P, xi, lg, a, it);
        return P->status == 0;
    }

    // f, g, M in the grid-origin frame (p relative to o), moved to the
    // caller's frame: with p = p_o + o, J = J_o B for B = [[I, 0], [-o^, I]],
    // so g = B^T g_o and M = B^T M_o B.  In 3x3 blocks (A, Bm, C of M_o and
    // O = o^, X = Bm O): M_ww = A - X - X^T - O C O, M_wv = Bm + O C, M_vv = C,
    // g_w = g_ow + o x g_ov, g_v = g_ov.
    double f = tot[0];
    double A[9], Bm[9], C[9];
    {
        int q = 7;
        double U[36];
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int c = r; c < 6; ++c) {
                U[6 * r + c] = tot[q];
                U[6 * c + r] = tot[q];
                ++q;
            }
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                A[3 * r + c] = U[6 * r + c];
                Bm[3 * r + c] = U[6 * r + 3 + c];
                C[3 * r + c] = U[6 * (r + 3) + 3 + c];
            }
    }
    double X[9], CO[9], OCO[9], OC[9];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        X[3 * r + 0] = Bm[3 * r + 1] * o2 - Bm[3 * r + 2] * o1;
        X[3 * r + 1] = -Bm[3 * r + 0] * o2 + Bm[3 * r + 2] * o0;
        X[3 * r + 2] = Bm[3 * r + 0] * o1 - Bm[3 * r + 1] * o0;
        CO[3 * r + 0] = C[3 * r + 1] * o2 - C[3 * r + 2] * o1;
        CO[3 * r + 1] = -C[3 * r + 0] * o2 + C[3 * r + 2] * o0;
        CO[3 * r + 2] = C[3 * r + 0] * o1 - C[3 * r + 1] * o0;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        OCO[c] = -o2 * CO[3 + c] + o1 * CO[6 + c];
        OCO[3 + c] = o2 * CO[c] - o0 * CO[6 + c];
        OCO[6 + c] = -o1 * CO[c] + o0 * CO[3 + c];
        OC[c] = -o2 * C[3 + c] + o1 * C[6 + c];
        OC[3 + c] = o2 * C[c] - o0 * C[6 + c];
        OC[6 + c] = -o1 * C[c] + o0 * C[3 + c];
    }
    double M[36];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            M[6 * r + c] = A[3 * r + c] - X[3 * r + c] - X[3 * c + r] - OCO[3 * r + c];
            double wv = Bm[3 * r + c] + OC[3 * r + c];
            M[6 * r + 3 + c] = wv;
            M[6 * (c + 3) + r] = wv;
            M[6 * (r + 3) + 3 + c] = C[3 * r + c];
        }
    double g[6];
    {
        double gw0 = tot[1], gw1 = tot[2], gw2 = tot[3], gv0 = tot[4], gv1 = tot[5], gv2 = tot[6];
        g[0] = gw0 + (o1 * gv2 - o2 * gv1);
        g[1] = gw1 + (o2 * gv0 - o0 * gv2);
        g[2] = gw2 + (o0 * gv1 - o1 * gv0);
        g[3] = gv0;
        g[4] = gv1;
        g[5] = gv2;
    }
    bool finite = isfinite(f);
#pragma unroll
    for (int k = 0; k < 6; ++k) finite = finite && isfinite(g[k]);
#pragma unroll
    for (int k = 0; k < 36; ++k) finite = finite && isfinite(M[k]);

    if (lg) {
        lg->f = f;
#pragma unroll
        for (int k = 0; k < 6; ++k) lg->g[k] = g[k];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int c = 0; c < 3; ++c) lg->T[4 * r + c] = P->T[3 * r + c];
            lg->T[4 * r + 3] = P->T[9 + r];
        }
        lg->T[12] = lg->T[13] = lg->T[14] = 0.0;
        lg->T[15] = 1.0;
        lg->n_pairs = ctot[0];
        lg->n_kept = ctot[1];
    }

    if (a.mode == FIN_EVAL) {
        // H_GN = -M + Gamma, Gamma = [[-1/2 g_w^, 0], [-g_v^, 0]] (Eq. 12)
        EvalOut *e = a.evalout + prob;
        e->f = f;
#pragma unroll
        for (int k = 0; k < 6; ++k) e->g[k] = g[k];
        double Gam[36];
#pragma unroll
        for (int k = 0; k < 36; ++k) Gam[k] = 0.0;
        Gam[1] = 0.5 * g[2];   Gam[2] = -0.5 * g[1];
        Gam[6] = -0.5 * g[2];  Gam[8] = 0.5 * g[0];
        Gam[12] = 0.5 * g[1];  Gam[13] = -0.5 * g[0];
        Gam[19] = g[5];  Gam[20] = -g[4];
        Gam[24] = -g[5]; Gam[26] = g[3];
        Gam[30] = g[4];  Gam[31] = -g[3];
#pragma unroll
        for (int k = 0; k < 36; ++k) {
            e->M[k] = M[k];
            e->H[k] = -M[k] + Gam[k];
        }
        e->n_pairs = ctot[0];
        e->n_kept = ctot[1];
        e->n_cand = ctot[2];
        return 0;
    }
    if (!finite) {
        set_inactive(P, -(int)GCVO_ERR_NONFINITE, a.n_active);
        return 0;
    }
    if (ctot[1] == 0 || !(f > 0.0)) {
        set_inactive(P, -(int)GCVO_ERR_NO_OVERLAP, a.n_active);
        return 0;
    }
    if (a.mode == FIN_GRAD) {
        // G-CVO-1: the line search runs along xi = g (Eq. 9); in the
        // grid-origin frame that direction has v' = omega x o + v.
#pragma unroll
        for (int k = 0; k < 6; ++k) P->dir[k] = g[k];
        P->dir32[0] = (float)g[0];
        P->dir32[1] = (float)g[1];
        P->dir32[2] = (float)g[2];
        P->dir32[3] = (float)(g[1] * o2 - g[2] * o1 + g[3]);
        P->dir32[4] = (float)(g[2] * o0 - g[0] * o2 + g[4]);
        P->dir32[5] = (float)(g[0] * o1 - g[1] * o0 + g[5]);
        return 0;
    }
    // G-CVO-2 step, Eq. (13)
    double xi[6];
    if (solve_gn(M, g, xi) != 0) {
        set_inactive(P, -(int)GCVO_ERR_SINGULAR, a.n_active);
        return 0;
    }
    apply_step(P, xi, lg, a, it);
    return P->status == 0;
}

// Per-group anchors R^T (z_g - t) - o in FP64 (stored as float), and R as
// float, for the pair kernel's transform at the current pose.
__device__ void refresh_anchors(const FinalizeArgs &a, int prob, ProbDev *P) {
    const GridDev *G = a.grids + prob;
    double R[9], t[3], o[3];
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = P->T[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        t[k] = P->T[9 + k];
        o[k] = G->origin[k];
    }
    for (int g = P->g0 + threadIdx.x; g < P->g1; g += blockDim.x) {
        float4 z = a.spos[a.gstart[g]];
        double d0 = (double)z.x - t[0], d1 = (double)z.y - t[1], d2 = (double)z.z - t[2];
        a.anchor[g] = make_float4((float)(R[0] * d0 + R[3] * d1 + R[6] * d2 - o[0]),
                                  (float)(R[1] * d0 + R[4] * d1 + R[7] * d2 - o[1]),
                                  (float)(R[2] * d0 + R[5] * d1 + R[8] * d2 - o[2]), 0.f);
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 9; ++k) P->R32[k] = (float)R[k];
}

__global__ void __launch_bounds__(256) k_finalize(FinalizeArgs a) {
    const int prob = blockIdx.x;
    if (prob >= a.n_problems) return;
    ProbDev *P = a.probs + prob;
    if (P->status != 0) return;
    if (a.mode == FIN_ANCHORS) {
        refresh_anchors(a, prob, P);
        return;
    }
    __shared__ double red[256];
    __shared__ long long cred[256];
    __shared__ double tot[32];
    __shared__ long long ctot[4];
    const int g0 = P->w0, g1 = P->w1;   // packed work items of this problem
    const int slot = threadIdx.x & 31, part = threadIdx.x >> 5;
    // compensated FP32 sum of the (hi, lo) group partials, one FP64 combine
    float H = 0.f, Lo = 0.f;
    long long cacc = 0;
    for (int g = g0 + part; g < g1; g += 8) {
        const float *p = a.part + (size_t)g * 64;
        float h = p[slot], l = p[32 + slot];
        float sm = H + h;
        float bp = sm - H;
        float err = (H - (sm - bp)) + (h - bp);
        H = sm;
        Lo += l + err;
        if (slot < 3) cacc += a.counts[(size_t)g * 4 + slot];
    }
    red[threadIdx.x] = (double)H + (double)Lo;
    cred[threadIdx.x] = cacc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double sm = 0.0;
        long long cs = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            sm += red[q * 32 + threadIdx.x];
            cs += cred[q * 32 + threadIdx.x];
        }
        tot[threadIdx.x] = sm;
        if (threadIdx.x < 4) ctot[threadIdx.x] = cs;
    }
    __syncthreads();
    __shared__ int s_upd;
    if (threadIdx.x == 0) s_upd = finalize_thread0(a, prob, P, tot, ctot);
    __syncthreads();
    if (s_upd) refresh_anchors(a, prob, P);
}

// ---------------------------------------------------------------------------
// Source grouping.
// ---------------------------------------------------------------------------
__device__ inline unsigned spread3(unsigned v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ inline int enc_f(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}

__global__ void k_src_keys(SrcArgs a) {
    const int p = blockIdx.y;
    const SrcDesc d = a.desc[p];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const int64_t gi = d.offset + i;
    float c[3], r[3];
    for (int k = 0; k < 3; ++k) {
        c[k] = d.xyz[k * d.n + i];
        r[k] = d.xyz[k * d.n];
    }
    unsigned m = 0;
    for (int k = 0; k < 3; ++k) {
        int q = (int)floorf((c[k] - r[k]) * d.inv_hf) + 512;
        q = min(max(q, 0), 1023);
        m |= spread3((unsigned)q) << k;
    }
    a.keys[gi] = ((unsigned long long)p << 30) | m;
    a.vals[gi] = (int)gi;
    a.prob_of[gi] = p;
    a.local[gi] = (int)i;
    bool bad = false;
    for (int k = 0; k < 3; ++k) bad |= !isfinite(c[k]);
    if (!a.iso && d.cov) {
        float s[6];
        for (int k = 0; k < 6; ++k) {
            s[k] = d.cov[k * d.n + i];
            bad |= !isfinite(s[k]);
        }
        float l = sym3_max_eig(s[0], s[1], s[2], s[3], s[4], s[5]);
        atomicMax(a.lam_enc + p, enc_f(l));
    }
    if (bad) atomicOr(a.status_word, DEV_ERR_NONFINITE);
}

__global__ void k_src_segments(const unsigned long long *keys, int64_t n, int *seg) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool head = i == 0 || (keys[i] >> 9) != (keys[i - 1] >> 9);
    seg[i] = head ? (int)i : 0;
}

__global__ void k_src_group_heads(const int *seg_start, int64_t n, int *gh) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    gh[i] = ((i - seg_start[i]) % 32 == 0) ? 1 : 0;
}

__global__ void k_src_groups(SrcArgs a, const unsigned long long *keys, const int *gid_incl, int64_t n,
                             int *gstart, int *gcount, int *gprob, int *pg0, int *pg1) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int g = gid_incl[i] - 1;
    int p = (int)(keys[i] >> 30);
    bool head = i == 0 || gid_incl[i] != gid_incl[i - 1];
    if (head) {
        gstart[g] = (int)i;
        gprob[g] = p;
        atomicMin(pg0 + p, g);
        atomicMax(pg1 + p, g + 1);
    }
    atomicAdd(gcount + g, 1);
    // packed source record in group order
    int src = a.vals[i];
    const SrcDesc d = a.desc[a.prob_of[src]];
    int li = a.local[src];
    float x = d.xyz[li], y = d.xyz[d.n + li], z = d.xyz[2 * d.n + li];
    float f0 = d.feat ? d.feat[li] : 1.f;
    float f1 = (d.feat && a.feat_dim > 1) ? d.feat[d.n + li] : 0.f;
    float f2 = (d.feat && a.feat_dim > 2) ? d.feat[2 * d.n + li] : 0.f;
    float s[6] = {0, 0, 0, 0, 0, 0};
    if (!a.iso && d.cov)
        for (int k = 0; k < 6; ++k) s[k] = d.cov[k * d.n + li];
    a.spos[i] = make_float4(x, y, z, f0);
    a.sca[i] = make_float4(s[0], s[1], s[2], s[3]);
    a.scb[i] = make_float4(s[4], s[5], f1, f2);
}

__global__ void k_pack(int pass, int np, const int *gstart, const int *gcount, const int *pg0, const int *pg1,
                       int *cnt, const int *incl, int4 *items, int *item_prob, int *pw0, int *pw1) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    int g0 = pg0[p], g1 = pg1[p];
    int out = pass ? incl[p] - cnt[p] : 0;
    if (pass) pw0[p] = out;
    int n = 0, first = g0, pts = 0, ng = 0;
    for (int g = g0; g < g1; ++g) {
        int c = gcount[g];
        if (ng > 0 && (pts + c > 32 || ng == PAIR_MAX_SUB)) {
            if (pass) {
                items[out + n] = make_int4(first, ng, gstart[first], pts);
                item_prob[out + n] = p;
            }
            ++n;
            first = g;
            pts = 0;
            ng = 0;
        }
        pts += c;
        ++ng;
    }
    if (ng > 0) {
        if (pass) {
            items[out + n] = make_int4(first, ng, gstart[first], pts);
            item_prob[out + n] = p;
        }
        ++n;
    }
    if (pass) pw1[p] = out + n;
    else cnt[p] = n;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
size_t pair_smem_bytes(int mode) { return (size_t)PAIR_WARPS * pair_warp_smem(mode); }

template <int MODE, bool ISO, int FD>
static cudaError_t launch_pair_t(const PairArgs &a, int grid, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_pair<MODE, ISO, FD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)pair_smem_bytes(MODE));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_pair<MODE, ISO, FD><<<grid, PAIR_WARPS * 32, pair_smem_bytes(MODE), s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int MODE, bool ISO, int FD>
static int occupancy_t() {
    int nb = 0;
    cudaFuncSetAttribute(k_pair<MODE, ISO, FD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pair_smem_bytes(MODE));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pair<MODE, ISO, FD>, PAIR_WARPS * 32, pair_smem_bytes(MODE));
    return nb;
}

int pair_blocks_per_sm(int mode, bool iso, int fd) {
#define OCC(M, I, F) if (mode == M && iso == I && (fd > 1) == (F > 1)) return occupancy_t<M, I, F>();
    OCC(PAIR_EVAL, false, 1) OCC(PAIR_EVAL, false, 3) OCC(PAIR_EVAL, true, 1) OCC(PAIR_EVAL, true, 3)
    OCC(PAIR_LINESEARCH, false, 1) OCC(PAIR_LINESEARCH, false, 3) OCC(PAIR_LINESEARCH, true, 1)
    OCC(PAIR_LINESEARCH, true, 3)
#undef OCC
    return 1;
}

cudaError_t launch_pair(const PairArgs &a, int mode, bool iso, int fd, int grid, cudaStream_t s) {
#define L(M, I, F) if (mode == M && iso == I && (fd > 1) == (F > 1)) return launch_pair_t<M, I, F>(a, grid, s);
    L(PAIR_EVAL, false, 1) L(PAIR_EVAL, false, 3) L(PAIR_EVAL, true, 1) L(PAIR_EVAL, true, 3)
    L(PAIR_LINESEARCH, false, 1) L(PAIR_LINESEARCH, false, 3) L(PAIR_LINESEARCH, true, 1)
    L(PAIR_LINESEARCH, true, 3)
#undef L
    return cudaErrorInvalidValue;
}

cudaError_t launch_pack(int pass, int np, const int *gstart, const int *gcount, const int *pg0, const int *pg1,
                        int *cnt, const int *incl, int4 *items, int *item_prob, int *pw0, int *pw1,
                        cudaStream_t s) {
    k_pack<<<(np + 127) / 128, 128, 0, s>>>(pass, np, gstart, gcount, pg0, pg1, cnt, incl, items, item_prob, pw0,
                                            pw1);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t s) {
    k_finalize<<<a.n_problems, 256, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_src_keys(const SrcArgs &a, int n_problems, int64_t max_n, cudaStream_t s) {
    dim3 grid((unsigned)((max_n + 255) / 256), (unsigned)n_problems);
    k_src_keys<<<grid, 256, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_src_segments(const unsigned long long *keys, int64_t n, int *seg, cudaStream_t s) {
    k_src_segments<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, n, seg);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_src_group_heads(const int *seg, int64_t n, int *gh, cudaStream_t s) {
    k_src_group_heads<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(seg, n, gh);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_src_groups(const SrcArgs &a, const unsigned long long *keys, const int *gid, int64_t n,
                              int *gstart, int *gcount, int *gprob, int *pg0, int *pg1, cudaStream_t s) {
    k_src_groups<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, keys, gid, n, gstart, gcount, gprob, pg0, pg1);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gcvo
