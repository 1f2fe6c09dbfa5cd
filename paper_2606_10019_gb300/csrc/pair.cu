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

struct WarpSmem {
    float4 *pos, *ca, *cb;
    uint8_t *queue;
    uint64_t *bar;
};

__device__ inline WarpSmem warp_smem(unsigned char *base, int w) {
    WarpSmem s;
    unsigned char *p = base + (size_t)w * PAIR_WARP_SMEM;
    s.pos = reinterpret_cast<float4 *>(p);
    s.ca = reinterpret_cast<float4 *>(p + PAIR_CAP * 16);
    s.cb = reinterpret_cast<float4 *>(p + PAIR_CAP * 32);
    s.queue = p + PAIR_CAP * 48;
    s.bar = reinterpret_cast<uint64_t *>(p + PAIR_CAP * 48 + PAIR_CAP * 32);
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
template <int MODE, bool ISO, int FD>
__global__ void __launch_bounds__(PAIR_WARPS * 32) k_pair(PairArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem S = warp_smem(smem, w);
    if (lane == 0) mbar_init(S.bar, 1);
    __syncwarp();
    unsigned parity = 0;
    const int n_groups = *a.n_groups;

    for (;;) {
        int g = 0;
        if (lane == 0) g = atomicAdd(a.work, 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= n_groups) break;
        const int prob = a.gprob[g];
        const ProbDev *P = a.probs + prob;
        if (P->status != 0) {
            // skip the rest of this finished problem's groups in one step
            if (lane == 0) atomicMax(a.work, P->g1);
            continue;
        }
        const GridDev *G = a.grids + prob;
        const int j0 = a.gstart[g], cnt = a.gcount[g];
        const bool act = lane < cnt;

        // ---- transform: p_j = R^T (z_j - t) - o (double), Sigma'_j = R^T Sigma_j R
        double R[9], t[3];
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = P->T[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) t[k] = P->T[9 + k];
        const int jj = act ? j0 + lane : j0;
        float4 z = a.spos[jj];
        float4 zb = a.scb[jj];
        double dz0 = (double)z.x - t[0], dz1 = (double)z.y - t[1], dz2 = (double)z.z - t[2];
        float px = (float)(R[0] * dz0 + R[3] * dz1 + R[6] * dz2 - G->origin[0]);
        float py = (float)(R[1] * dz0 + R[4] * dz1 + R[7] * dz2 - G->origin[1]);
        float pz = (float)(R[2] * dz0 + R[5] * dz1 + R[8] * dz2 - G->origin[2]);
        float q00 = 0.f, q01 = 0.f, q02 = 0.f, q11 = 0.f, q12 = 0.f, q22 = 0.f;
        if (!ISO) {
            float4 za = a.sca[jj];
            float Rf[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) Rf[k] = (float)R[k];
            // T1 = Sigma_z R, Sigma' = R^T T1
            float s[9] = {za.x, za.y, za.z, za.y, za.w, zb.x, za.z, zb.x, zb.y};
            float T1[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) T1[3 * r + c] = s[3 * r] * Rf[c] + s[3 * r + 1] * Rf[3 + c] + s[3 * r + 2] * Rf[6 + c];
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
            float om0 = (float)P->dir_o[0], om1 = (float)P->dir_o[1], om2 = (float)P->dir_o[2];
            a1[0] = om1 * pz - om2 * py + (float)P->dir_o[3];
            a1[1] = om2 * px - om0 * pz + (float)P->dir_o[4];
            a1[2] = om0 * py - om1 * px + (float)P->dir_o[5];
#define CROSS_W(dst, src)                            \
    dst[0] = om1 * src[2] - om2 * src[1];            \
    dst[1] = om2 * src[0] - om0 * src[2];            \
    dst[2] = om0 * src[1] - om1 * src[0];
            CROSS_W(a2, a1)
            CROSS_W(a3, a2)
            CROSS_W(a4, a3)
#undef CROSS_W
        }

        // ---- bounding box of the transformed group
        float bmin[3] = {act ? px : INFINITY, act ? py : INFINITY, act ? pz : INFINITY};
        float bmax[3] = {act ? px : -INFINITY, act ? py : -INFINITY, act ? pz : -INFINITY};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                bmin[k] = fminf(bmin[k], __shfl_xor_sync(0xffffffffu, bmin[k], o));
                bmax[k] = fmaxf(bmax[k], __shfl_xor_sync(0xffffffffu, bmax[k], o));
            }
        const float rho = sqrtf(rho2);
        int lo[3], hi[3];
        bool empty = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float fl = floorf((bmin[k] - rho - G->corner[k]) * G->inv_h);
            float fh = floorf((bmax[k] + rho - G->corner[k]) * G->inv_h);
            fl = fminf(fmaxf(fl, 0.0f), (float)G->dims[k]);
            fh = fmaxf(fminf(fh, (float)(G->dims[k] - 1)), -1.0f);
            if (!(fl <= fh)) {
                empty = true;
                fl = 0.0f;
                fh = 0.0f;
            }
            lo[k] = (int)fl;
            hi[k] = (int)fh;
        }

        // ---- accumulators
        float Sf = 0.f, Su0 = 0.f, Su1 = 0.f, Su2 = 0.f;
        float A00 = 0.f, A01 = 0.f, A02 = 0.f, A11 = 0.f, A12 = 0.f, A22 = 0.f;
        float L1 = 0.f, L2 = 0.f, L3 = 0.f, L4 = 0.f;  // line-search sums (f in Sf)
        int n_pairs = 0, n_kept = 0;
        long long n_cand = 0;

        const int ncy = empty ? 0 : hi[1] - lo[1] + 1;
        const int n_cols = empty ? 0 : (hi[0] - lo[0] + 1) * ncy;
        const int dy = G->dims[1], dzs = G->dims[2];
        for (int cb0 = 0; cb0 < n_cols; cb0 += 32) {
            // one column per lane: the run of occupied voxels cz in [lo2, hi2]
            int rs = 0, rl = 0;
            int col = cb0 + lane;
            if (col < n_cols) {
                int cx = lo[0] + col / ncy, cy = lo[1] + col % ncy;
                unsigned long long kb = ((unsigned long long)cx * dy + cy) * dzs;
                int first = -1, last = -1;
                for (int cz = lo[2]; cz <= hi[2]; ++cz) {
                    int c = grid_lookup(*G, kb + cz);
                    if (c >= 0) {
                        first = c;
                        break;
                    }
                }
                if (first >= 0) {
                    for (int cz = hi[2]; cz >= lo[2]; --cz) {
                        int c = grid_lookup(*G, kb + cz);
                        if (c >= 0) {
                            last = c;
                            break;
                        }
                    }
                    rs = __ldg(G->cell_start + first);
                    rl = __ldg(G->cell_start + last + 1) - rs;
                }
            }
            // exclusive offsets of the runs
            int incl = rl;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            const int off = incl - rl;
            n_cand += act ? total : 0;

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
                        all_done = __all_sync(0xffffffffu, done);
                        if (all_done || ++spin > (1 << 22)) break;
                    }
                    if (!all_done) {
                        if (lane == 0) atomicOr(a.status_word, DEV_ERR_TIMEOUT);
                        return;
                    }
                    parity ^= 1u;
                }

                // ---- phase 1: |r| <= rho test against every staged point
                int nq = 0;
                for (int k = 0; k < m; ++k) {
                    float4 x = S.pos[k];
                    float rx = x.x - px, ry = x.y - py, rz = x.z - pz;
                    float d2 = rx * rx + ry * ry + rz * rz;
                    if (act && d2 <= rho2) {
                        S.queue[nq * 32 + lane] = (uint8_t)k;
                        ++nq;
                    }
                }
                n_pairs += nq;
                const int tmax = __reduce_max_sync(0xffffffffu, nq);

                // ---- phase 2: full evaluation of the queued pairs
                for (int qi = 0; qi < tmax; ++qi) {
                    if (qi < nq) {
                        int k = S.queue[qi * 32 + lane];
                        float4 x = S.pos[k];
                        float r0 = x.x - px, r1 = x.y - py, r2 = x.z - pz;
                        float cij = x.w * l0;
                        if (FD > 1) {
                            float4 b = S.cb[k];
                            cij += b.z * l1 + b.w * l2;
                        }
                        if (ISO) {
                            float d2 = (r0 * r0 + r1 * r1 + r2 * r2) * iso_inv;
                            bool keep = d2 <= c2;
                            float wgt = keep ? cij * ex2_approx(d2 * NEG_HALF_LOG2E) : 0.f;
                            n_kept += keep;
                            Sf += wgt;
                            Su0 += wgt * r0;
                            Su1 += wgt * r1;
                            Su2 += wgt * r2;
                            if (MODE == PAIR_LINESEARCH) {
                                // A = I / ell^2
                                float kr1 = (a1[0] * r0 + a1[1] * r1 + a1[2] * r2) * iso_inv;
                                float kr2 = (a2[0] * r0 + a2[1] * r1 + a2[2] * r2) * iso_inv;
                                float kr3 = (a3[0] * r0 + a3[1] * r1 + a3[2] * r2) * iso_inv;
                                float kr4 = (a4[0] * r0 + a4[1] * r1 + a4[2] * r2) * iso_inv;
                                float a11 = (a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2]) * iso_inv;
                                float a12 = (a1[0] * a2[0] + a1[1] * a2[1] + a1[2] * a2[2]) * iso_inv;
                                float a13 = (a1[0] * a3[0] + a1[1] * a3[1] + a1[2] * a3[2]) * iso_inv;
                                float a22 = (a2[0] * a2[0] + a2[1] * a2[1] + a2[2] * a2[2]) * iso_inv;
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
                                L1 += wgt * be;
                                L2 += wgt * (ga + 0.5f * be * be);
                                L3 += wgt * (de + be * ga + be * be * be * (1.f / 6.f));
                                L4 += wgt * (ep + be * de + 0.5f * be * be * ga + 0.5f * ga * ga +
                                             be * be * be * be * (1.f / 24.f));
                            }
                        } else {
                            float4 ca = S.ca[k];
                            float4 cbv = S.cb[k];
                            // Sigma_ij = Sigma_i + R^T Sigma_j R (Eq. 7c)
                            float s00 = ca.x + q00, s01 = ca.y + q01, s02 = ca.z + q02;
                            float s11 = ca.w + q11, s12 = cbv.x + q12, s22 = cbv.y + q22;
                            // adjugate and determinant
                            float c00 = s11 * s22 - s12 * s12;
                            float c01 = s02 * s12 - s01 * s22;
                            float c02 = s01 * s12 - s02 * s11;
                            float c11 = s00 * s22 - s02 * s02;
                            float c12 = s01 * s02 - s00 * s12;
                            float c22 = s00 * s11 - s01 * s01;
                            float det = s00 * c00 + s01 * c01 + s02 * c02;
                            float y0 = c00 * r0 + c01 * r1 + c02 * r2;
                            float y1 = c01 * r0 + c11 * r1 + c12 * r2;
                            float y2 = c02 * r0 + c12 * r1 + c22 * r2;
                            float qf = r0 * y0 + r1 * y1 + r2 * y2;
                            float rdet = rcp_approx(det);
                            float d2 = qf * rdet;
                            bool keep = d2 <= c2;
                            float wgt = keep ? cij * ex2_approx(d2 * NEG_HALF_LOG2E) : 0.f;
                            n_kept += keep;
                            Sf += wgt;
                            if (MODE == PAIR_EVAL) {
                                float wd = wgt * rdet;
                                Su0 += wd * y0;
                                Su1 += wd * y1;
                                Su2 += wd * y2;
                                A00 += wd * c00;
                                A01 += wd * c01;
                                A02 += wd * c02;
                                A11 += wd * c11;
                                A12 += wd * c12;
                                A22 += wd * c22;
                            } else {
                                // bilinear forms of A = adj / det with r and a_k
                                float kr1 = (a1[0] * y0 + a1[1] * y1 + a1[2] * y2) * rdet;
                                float kr2 = (a2[0] * y0 + a2[1] * y1 + a2[2] * y2) * rdet;
                                float kr3 = (a3[0] * y0 + a3[1] * y1 + a3[2] * y2) * rdet;
                                float kr4 = (a4[0] * y0 + a4[1] * y1 + a4[2] * y2) * rdet;
                                float w0 = c00 * a1[0] + c01 * a1[1] + c02 * a1[2];
                                float w1 = c01 * a1[0] + c11 * a1[1] + c12 * a1[2];
                                float w2 = c02 * a1[0] + c12 * a1[1] + c22 * a1[2];
                                float a11 = (a1[0] * w0 + a1[1] * w1 + a1[2] * w2) * rdet;
                                float a12 = (a2[0] * w0 + a2[1] * w1 + a2[2] * w2) * rdet;
                                float a13 = (a3[0] * w0 + a3[1] * w1 + a3[2] * w2) * rdet;
                                float v0 = c00 * a2[0] + c01 * a2[1] + c02 * a2[2];
                                float v1 = c01 * a2[0] + c11 * a2[1] + c12 * a2[2];
                                float v2 = c02 * a2[0] + c12 * a2[1] + c22 * a2[2];
                                float a22 = (a2[0] * v0 + a2[1] * v1 + a2[2] * v2) * rdet;
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
                                L1 += wgt * be;
                                L2 += wgt * (ga + 0.5f * be * be);
                                L3 += wgt * (de + be * ga + be * be * be * (1.f / 6.f));
                                L4 += wgt * (ep + be * de + 0.5f * be * be * ga + 0.5f * ga * ga +
                                             be * be * be * be * (1.f / 24.f));
                            }
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
        if (act) {
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
        float *out = a.part + (size_t)g * 64;
#pragma unroll
        for (int k = 0; k < PAIR_SLOTS; ++k) {
            if (k >= nslot) break;
            float hi, lo;
            warp_sum2(v[k], hi, lo);
            if (lane == 0) {
                out[k] = hi;
                out[32 + k] = lo;
            }
        }
        int tp = __reduce_add_sync(0xffffffffu, n_pairs);
        int tk = __reduce_add_sync(0xffffffffu, n_kept);
        long long tc = n_cand;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tc += __shfl_down_sync(0xffffffffu, tc, o);
        if (lane == 0) {
            long long *cnts = a.counts + (size_t)g * 4;
            cnts[0] = tp;
            cnts[1] = tk;
            cnts[2] = tc;
        }
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

__global__ void __launch_bounds__(256) k_finalize(FinalizeArgs a) {
    const int prob = blockIdx.x;
    if (prob >= a.n_problems) return;
    ProbDev *P = a.probs + prob;
    if (P->status != 0) return;
    __shared__ double red[256];
    __shared__ long long cred[256];
    __shared__ double tot[32];
    __shared__ long long ctot[4];
    const int g0 = P->g0, g1 = P->g1;
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
    if (threadIdx.x != 0) return;

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
        return;
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
        return;
    }
    if (!finite) {
        set_inactive(P, -(int)GCVO_ERR_NONFINITE, a.n_active);
        return;
    }
    if (ctot[1] == 0 || !(f > 0.0)) {
        set_inactive(P, -(int)GCVO_ERR_NO_OVERLAP, a.n_active);
        return;
    }
    if (a.mode == FIN_GRAD) {
        // G-CVO-1: the line search runs along xi = g (Eq. 9); in the
        // grid-origin frame that direction has v' = omega x o + v.
#pragma unroll
        for (int k = 0; k < 6; ++k) P->dir[k] = g[k];
        P->dir_o[0] = g[0];
        P->dir_o[1] = g[1];
        P->dir_o[2] = g[2];
        P->dir_o[3] = g[1] * o2 - g[2] * o1 + g[3];
        P->dir_o[4] = g[2] * o0 - g[0] * o2 + g[4];
        P->dir_o[5] = g[0] * o1 - g[1] * o0 + g[5];
        return;
    }
    // G-CVO-2 step, Eq. (13)
    double xi[6];
    if (solve_gn(M, g, xi) != 0) {
        set_inactive(P, -(int)GCVO_ERR_SINGULAR, a.n_active);
        return;
    }
    apply_step(P, xi, lg, a, it);
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

}  // namespace

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
size_t pair_smem_bytes() { return (size_t)PAIR_WARPS * PAIR_WARP_SMEM; }

template <int MODE, bool ISO, int FD>
static cudaError_t launch_pair_t(const PairArgs &a, int grid, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_pair<MODE, ISO, FD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)pair_smem_bytes());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_pair<MODE, ISO, FD><<<grid, PAIR_WARPS * 32, pair_smem_bytes(), s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int MODE, bool ISO, int FD>
static int occupancy_t() {
    int nb = 0;
    cudaFuncSetAttribute(k_pair<MODE, ISO, FD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pair_smem_bytes());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pair<MODE, ISO, FD>, PAIR_WARPS * 32, pair_smem_bytes());
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
