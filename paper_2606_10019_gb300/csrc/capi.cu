// The extern "C" entry points declared in include/gcvo.h.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "pair.cuh"

using namespace gcvo;

namespace {

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool valid_kernel_params(const gcvo_kernel_params *p) {
    if (!p) return false;
    if (p->kernel_mode != 0 && p->kernel_mode != 1) return false;
    if (!(p->cutoff >= 0) || !std::isfinite(p->cutoff)) return false;   // 0: dense, no cutoff
    if (!(p->sigma2 > 0) || !std::isfinite(p->sigma2)) return false;
    if (p->kernel_mode == 1 && !(p->iso_ell > 0)) return false;
    if (p->feat_dim < 1 || p->feat_dim > GCVO_MAX_FEAT) return false;
    return true;
}

// Copy `count` floats to the device when `p` is host memory.  `off` is the
// running float offset inside `buf` (grown by the caller beforehand).
gcvo_status stage(gcvo_ctx *ctx, const float *p, size_t count, DevBuf &buf, size_t &off, const float **out) {
    if (!p) {
        *out = nullptr;
        return GCVO_OK;
    }
    if (is_device_ptr(p)) {
        *out = p;
        return GCVO_OK;
    }
    float *d = buf.as<float>() + off;
    GCVO_CUDA(cudaMemcpyAsync(d, p, count * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    off += (count + 63) & ~size_t(63);
    *out = d;
    return GCVO_OK;
}

size_t staged_floats(const float *p, size_t count) {
    if (!p || is_device_ptr(p)) return 0;
    return (count + 63) & ~size_t(63);
}

gcvo_status host_pinned(gcvo_ctx *ctx, size_t bytes, void **out) {
    if (ctx->host_pinned_bytes < bytes) {
        if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
        ctx->host_pinned = nullptr;
        ctx->host_pinned_bytes = 0;
        if (cudaMallocHost(&ctx->host_pinned, bytes) != cudaSuccess) {
            cudaGetLastError();
            return GCVO_ERR_WORKSPACE;
        }
        ctx->host_pinned_bytes = bytes;
    }
    *out = ctx->host_pinned;
    return GCVO_OK;
}

int ceil_log2(int64_t v) {
    int b = 0;
    while (((int64_t)1 << b) < v) ++b;
    return b;
}

// Everything the pair / finalize kernels need for a set of problems.
struct Prepared {
    int n_problems = 0;
    int n_items = 0;            // upper bound of the work items
    int *d_nitems = nullptr;    // their count (device)
    const int64_t *d_poff = nullptr;
    const int *d_npts = nullptr;
    int64_t n_points = 0;
    int feat_dim = 1;
    bool iso = false;
    std::vector<ProbDev> probs;
};

// Whether the pair passes of a problem must form r = x - p from
// double-float positions.  Positions are relative to the target box centre,
// so FP32 rounds both x and p by up to 2^-24 R, R the box half-diagonal
// plus rho; with |Sigma_ij^-1 r| <= c / sigma_min (sigma_min^2 the smallest
// eigenvalue of Sigma_ij, at least the sum of the two clouds' smallest), each
// d^2 moves by up to 4 c R 2^-24 / sigma_min.  Above 3e-4 (a LiDAR frame,
// R about 100 m with sigma_min about 4 cm, reaches 1.7e-3) the sums of a few
// thousand pairs drift towards the 1e-5 relative tolerance of f and g, and
// the tails are worth their 7 instructions per pair; a small scene (2 m,
// sigma_min 1.4 cm: 1e-4) is accurate in FP32.  Dense mode (no cutoff) and
// degenerate covariances always take the tails.
bool pair_needs_lo(const GridDev &g, const gcvo_kernel_params &kp, double rho2, float lmin_src) {
    if (kp.cutoff <= 0 || !std::isfinite(rho2)) return true;
    double half = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double e = 0.5 * (double)g.dims[a] * (double)g.h;
        half += e * e;
    }
    const double R = std::sqrt(half) + std::sqrt(rho2);
    const double s2 = kp.kernel_mode == 1 ? kp.iso_ell * kp.iso_ell
                                          : (double)g.lam_min + (double)std::max(0.0f, lmin_src);
    if (!(s2 > 0.0)) return true;
    return 4.0 * kp.cutoff * R * std::ldexp(1.0, -24) / std::sqrt(s2) > 3e-4;
}

gcvo_status prepare(gcvo_ctx *ctx, int np, const gcvo_problem *pr, Prepared &P) {
    cudaStream_t s = ctx->stream;
    if (np < 1 || np > GCVO_MAX_PROBLEMS || !pr) return GCVO_ERR_INVALID_ARG;
    const gcvo_kernel_params &kp0 = pr[0].target ? pr[0].target->kp : gcvo_kernel_params{};
    for (int p = 0; p < np; ++p) {
        const gcvo_problem &q = pr[p];
        if (!q.target || !q.src_xyz || q.n_src < 1 || q.n_src > (1 << 28)) return GCVO_ERR_INVALID_ARG;
        if (q.target->kp.kernel_mode != kp0.kernel_mode || q.target->kp.feat_dim != kp0.feat_dim)
            return GCVO_ERR_INVALID_ARG;
        if (q.target->kp.kernel_mode == 0 && !q.src_cov) return GCVO_ERR_INVALID_ARG;
        for (int k = 0; k < 16; ++k)
            if (!std::isfinite(q.T0[k])) return GCVO_ERR_NONFINITE;
    }
    P.n_problems = np;
    P.iso = kp0.kernel_mode == 1;
    P.feat_dim = kp0.feat_dim;
    // stage host inputs
    size_t need = 0;
    int64_t N = 0;
    for (int p = 0; p < np; ++p) {
        const gcvo_problem &q = pr[p];
        need += staged_floats(q.src_xyz, 3 * (size_t)q.n_src);
        if (!P.iso) need += staged_floats(q.src_cov, 6 * (size_t)q.n_src);
        need += staged_floats(q.src_feat, (size_t)P.feat_dim * q.n_src);
        N += q.n_src;
    }
    if (N > (int64_t)1 << 30) return GCVO_ERR_CAPACITY;
    P.n_points = N;
    if (need) GCVO_TRY(ctx->stage_xyz.ensure(need * sizeof(float), s));
    std::vector<SrcDesc> desc(np);
    size_t off = 0;
    int64_t max_n = 0;
    for (int p = 0; p < np; ++p) {
        const gcvo_problem &q = pr[p];
        SrcDesc &d = desc[p];
        GCVO_TRY(stage(ctx, q.src_xyz, 3 * (size_t)q.n_src, ctx->stage_xyz, off, &d.xyz));
        d.cov = nullptr;
        if (!P.iso) GCVO_TRY(stage(ctx, q.src_cov, 6 * (size_t)q.n_src, ctx->stage_xyz, off, &d.cov));
        GCVO_TRY(stage(ctx, q.src_feat, (size_t)P.feat_dim * q.n_src, ctx->stage_xyz, off, &d.feat));
        d.n = q.n_src;
        d.offset = 0;
        // fine Morton voxel: h/2, so the coarse voxel (8 fine) is 4 h = twice the
        // kernel range when h = rho/2
        d.inv_hf = 2.0f / q.target->store.d.h;
        max_n = std::max<int64_t>(max_n, q.n_src);
    }
    int64_t acc = 0;
    for (int p = 0; p < np; ++p) {
        desc[p].offset = acc;
        acc += desc[p].n;
    }

    // device buffers
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t small_need = al(np * sizeof(SrcDesc)) + al(np * sizeof(int)) * 7 + al(np * sizeof(int64_t)) +
                        al(sizeof(int)) * 4 + 256;
    GCVO_TRY(ctx->small.ensure(small_need + 4096, s));
    char *sp = ctx->small.as<char>();
    SrcDesc *d_desc = reinterpret_cast<SrcDesc *>(sp);
    sp += al(np * sizeof(SrcDesc));
    int *d_lam = reinterpret_cast<int *>(sp);
    sp += al(np * sizeof(int));
    int *d_lmin = reinterpret_cast<int *>(sp);
    sp += al(np * sizeof(int));
    int *d_nitems = reinterpret_cast<int *>(sp);
    sp += 256;
    int *d_pcnt = reinterpret_cast<int *>(sp);
    sp += al(np * sizeof(int));
    int64_t *d_poff = reinterpret_cast<int64_t *>(sp);
    P.d_nitems = d_nitems;

    GCVO_TRY(ctx->sort_keys.ensure(N * sizeof(unsigned long long), s));
    GCVO_TRY(ctx->sort_vals.ensure(al(N * sizeof(int)) * 3, s));
    GCVO_TRY(ctx->sort_tmp.ensure(radix_sort_scratch_bytes(N), s));
    GCVO_TRY(ctx->scan_tmp.ensure(scan_scratch_bytes(N) + 1024, s));
    GCVO_TRY(ctx->src_pos.ensure(N * sizeof(float4), s));
    GCVO_TRY(ctx->src_ca.ensure(N * sizeof(float4), s));
    GCVO_TRY(ctx->src_cb.ensure(N * sizeof(float4), s));
    GCVO_TRY(ctx->pprob.ensure(N * sizeof(int), s));
    if (P.feat_dim > 3) {
        GCVO_TRY(ctx->src_fx.ensure(N * sizeof(float4), s));
        GCVO_TRY(ctx->t_fx.ensure(N * sizeof(float4), s));
    }
    GCVO_TRY(ctx->t_pos.ensure(N * sizeof(float4), s));
    GCVO_TRY(ctx->t_ca.ensure(N * sizeof(float4), s));
    GCVO_TRY(ctx->t_cb.ensure(N * sizeof(float4), s));
    GCVO_TRY(ctx->items.ensure(N * sizeof(int4), s));
    GCVO_TRY(ctx->item_prob.ensure(N * sizeof(int), s));
    if (N >= (1LL << 26)) return GCVO_ERR_CAPACITY;   // point index of a sub-tile word
    GCVO_TRY(ctx->status_word.ensure(256, s));
    char *vp = ctx->sort_vals.as<char>();
    int *vals = reinterpret_cast<int *>(vp);
    int *prob_of = reinterpret_cast<int *>(vp + al(N * sizeof(int)));
    int *local = reinterpret_cast<int *>(vp + 2 * al(N * sizeof(int)));

    GCVO_CUDA(cudaMemcpyAsync(d_desc, desc.data(), np * sizeof(SrcDesc), cudaMemcpyHostToDevice, s));
    GCVO_CUDA(cudaMemsetAsync(d_lam, 0, np * sizeof(int), s));
    GCVO_CUDA(cudaMemsetAsync(d_lmin, 0x7f, np * sizeof(int), s));   // a huge positive float
    GCVO_CUDA(cudaMemsetAsync(ctx->status_word.ptr, 0, 256, s));

    SrcArgs sa{};
    sa.desc = d_desc;
    sa.keys = ctx->sort_keys.as<unsigned long long>();
    sa.vals = vals;
    sa.prob_of = prob_of;
    sa.local = local;
    sa.lam_enc = d_lam;
    sa.lam_min_enc = d_lmin;
    sa.status_word = ctx->status_word.as<unsigned>();
    sa.spos = ctx->src_pos.as<float4>();
    sa.sca = ctx->src_ca.as<float4>();
    sa.scb = ctx->src_cb.as<float4>();
    sa.pprob = ctx->pprob.as<int>();
    sa.sfx = P.feat_dim > 3 ? ctx->src_fx.as<float4>() : nullptr;
    sa.feat_dim = P.feat_dim;
    sa.iso = P.iso;
    GCVO_CUDA(launch_src_keys(sa, np, max_n, s));
    GCVO_TRY(radix_sort_pairs(sa.keys, vals, N, 30 + std::max(1, ceil_log2(np)), ctx->sort_tmp.ptr,
                              ctx->sort_tmp.bytes, s));
    GCVO_CUDA(launch_src_pack(sa, sa.keys, N, s));
    // per-problem point offsets and sizes for the work-item packing, which
    // depends on the pair schedule and is done by choose_schedule
    std::vector<int> hn(np);
    std::vector<int64_t> hoff(np);
    for (int p = 0; p < np; ++p) {
        hn[p] = (int)desc[p].n;
        hoff[p] = desc[p].offset;
    }
    P.n_items = (int)N;   // upper bound: every item holds a point
    P.d_poff = d_poff;
    P.d_npts = d_pcnt;
    GCVO_CUDA(cudaMemcpyAsync(d_pcnt, hn.data(), np * sizeof(int), cudaMemcpyHostToDevice, s));
    GCVO_CUDA(cudaMemcpyAsync(d_poff, hoff.data(), np * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    GCVO_TRY(ctx->pack_tmp.ensure(5 * (((size_t)N + 63) / 64 * 64) * sizeof(int), s));

    // read back the status word and the source eigenvalue bounds
    void *hp;
    GCVO_TRY(host_pinned(ctx, (size_t)(2 * np + 8) * sizeof(int), &hp));
    int *h = static_cast<int *>(hp);
    GCVO_CUDA(cudaMemcpyAsync(h + 1, ctx->status_word.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaMemcpyAsync(h + 8, d_lam, np * sizeof(int), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaMemcpyAsync(h + 8 + np, d_lmin, np * sizeof(int), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    if (h[1] & DEV_ERR_NONFINITE) return GCVO_ERR_NONFINITE;
    P.probs.assign(np, ProbDev{});
    for (int p = 0; p < np; ++p) {
        ProbDev &d = P.probs[p];
        const gcvo_problem &q = pr[p];
        const gcvo_grid *G = q.target;
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) d.T[3 * r + c] = q.T0[4 * r + c];
            d.T[9 + r] = q.T0[4 * r + 3];
        }
        d.status = 0;
        d.iter = 0;
        d.w0 = 0;   // set with the work items
        d.w1 = 0;
        auto dec = [](int e) {
            const int i = e >= 0 ? e : e ^ 0x7fffffff;
            float f;
            memcpy(&f, &i, 4);
            return f;
        };
        const float lam_src = dec(h[8 + p]);
        const float lmin_src = dec(h[8 + np + p]);
        const gcvo_kernel_params &kp = G->kp;
        double c2 = kp.cutoff * kp.cutoff;
        double rho2;
        if (kp.cutoff == 0)   // dense: every pair, no cutoff
            rho2 = c2 = INFINITY;
        else if (kp.kernel_mode == 1)
            rho2 = c2 * kp.iso_ell * kp.iso_ell * (1.0 + 1e-5);
        else
            rho2 = c2 * ((double)G->store.d.lam_max + (double)lam_src) * (1.0 + 2e-4) + 1e-12;
        d.rho2 = (float)rho2;
        d.c2 = (float)c2;
        d.lo = pair_needs_lo(G->store.d, kp, rho2, lmin_src) ? 1 : 0;
        d.sigma2 = (float)kp.sigma2;
        d.iso_inv = kp.kernel_mode == 1 ? (float)(1.0 / (kp.iso_ell * kp.iso_ell)) : 0.f;
    }
    // per-iteration buffers
    GCVO_TRY(ctx->partial.ensure((size_t)std::max(P.n_items, 1) * (64 * sizeof(float) + 4 * sizeof(long long)) +
                                     fin_chunk_bytes(P.n_items, P.n_problems) + 4096,
                                 s));
    GCVO_TRY(ctx->probs.ensure(np * sizeof(ProbDev), s));
    GCVO_TRY(ctx->grids.ensure(np * sizeof(GridDev), s));
    GCVO_TRY(ctx->evalout.ensure(np * sizeof(EvalOut) + 256, s));
    std::vector<GridDev> gd(np);
    for (int p = 0; p < np; ++p) gd[p] = pr[p].target->store.d;
    GCVO_CUDA(cudaMemcpyAsync(ctx->probs.ptr, P.probs.data(), np * sizeof(ProbDev), cudaMemcpyHostToDevice, s));
    GCVO_CUDA(cudaMemcpyAsync(ctx->grids.ptr, gd.data(), np * sizeof(GridDev), cudaMemcpyHostToDevice, s));
    // host staging buffers must stay valid until the copies ran
    GCVO_CUDA(cudaStreamSynchronize(s));
    return GCVO_OK;
}

struct IterBufs {
    PairArgs pa;
    FinalizeArgs fa;
    TransformArgs ta;
    int *work;
    int grid;   // persistent blocks of the evaluation pass
    int sub;    // its schedule: points per sub-tile
};

// Blocks of a persistent pair launch: one item per block at a time, as many
// blocks as fit on the GPU.
int pair_grid(const gcvo_ctx *ctx, const Prepared &P, int mode, int sub) {
    int per_sm = std::max(1, pair_blocks_per_sm(mode, P.iso, P.feat_dim, sub));
    return std::max(1, std::min(P.n_items, per_sm * ctx->sm_count));
}

// A schedule of the pair passes: sub (points per sub-tile: 4, 8, 16 or 32,
// i.e. 8, 4, 2 or 1 lanes per point) | level << 8 (the Morton voxel level
// that sub-tiles never cross: 1 = edge rho / 2, 2 = edge rho, 3 = edge 2 rho;
// a finer cut gives smaller sub-tile boxes and so fewer targets per box that
// lie out of range of the box's points, at the price of more, emptier
// sub-tiles in sparse parts).  The work items
// are packed for it.
gcvo_status pack(gcvo_ctx *ctx, const Prepared &P, int sched) {
    return pack_items(P.n_problems, ctx->sort_keys.as<unsigned long long>(), P.n_points, sched & 0xff, sched >> 8,
                      P.d_poff, P.d_npts, ctx->pack_tmp.as<int>(), ctx->items.as<int>(), ctx->item_prob.as<int>(),
                      P.d_nitems, ctx->probs.as<ProbDev>(),
                      reinterpret_cast<int *>(ctx->status_word.as<char>() + 64) + 2,   // chunk count
                      ctx->scan_tmp.ptr, ctx->stream);
}

// The autotuner: the schedule for this shape of problem set -- a forced
// one, the cached choice for the same shape, or the fastest of one timed
// evaluation pass with each candidate (the second of two, CUDA events).  The
// shape is the kernel mode, the feature count and the log2 buckets of the
// problem count and of the mean source size.
gcvo_status choose_schedule(gcvo_ctx *ctx, const Prepared &P, IterBufs &b) {
    int sched = ctx->forced_sub ? (ctx->forced_sub < 256 ? ctx->forced_sub | 2 << 8 : ctx->forced_sub) : 0;
    int packed = 0;
    if (!sched) {
        int lb_n = 0, lb_p = 0;
        while ((2LL << lb_n) <= P.n_points / std::max(1, P.n_problems)) ++lb_n;
        while ((2 << lb_p) <= P.n_problems) ++lb_p;
        const long long key = ((long long)P.iso << 40) | ((long long)P.feat_dim << 32) | ((long long)lb_p << 8) | lb_n;
        for (auto &kv : ctx->tuned)
            if (kv.first == key) sched = kv.second;
        if (!sched) {
            constexpr int NC = 9;
            const int cands[NC] = {4 | 2 << 8,  8 | 2 << 8,  16 | 2 << 8, 32 | 2 << 8, 8 | 3 << 8,
                                   16 | 3 << 8, 32 | 3 << 8, 4 | 1 << 8,  8 | 1 << 8};
            cudaEvent_t ev[2 * NC];
            for (auto &e : ev) GCVO_CUDA(cudaEventCreate(&e));
            float best = 0.f;
            gcvo_status st = GCVO_OK;
            for (int c = 0; c < NC && st == GCVO_OK; ++c) {
                const int sub_c = cands[c] & 0xff;
                st = pack(ctx, P, cands[c]);
                packed = cands[c];
                const int g = pair_grid(ctx, P, PAIR_EVAL, sub_c);
                for (int rep = 0; rep < 2 && st == GCVO_OK; ++rep) {
                    cudaError_t e = cudaMemsetAsync(b.work, 0, sizeof(int), ctx->stream);
                    if (e == cudaSuccess && rep == 1) e = cudaEventRecord(ev[2 * c], ctx->stream);
                    if (e == cudaSuccess) e = launch_pair(b.pa, PAIR_EVAL, P.iso, P.feat_dim, sub_c, g, ctx->stream);
                    if (e == cudaSuccess && rep == 1) e = cudaEventRecord(ev[2 * c + 1], ctx->stream);
                    if (e != cudaSuccess) {
                        set_last_cuda_error(e, "schedule timing pass", __LINE__);
                        st = GCVO_ERR_CUDA;
                    }
                }
            }
            if (st == GCVO_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = GCVO_ERR_CUDA;
            for (int c = 0; c < NC && st == GCVO_OK; ++c) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, ev[2 * c], ev[2 * c + 1]) != cudaSuccess) st = GCVO_ERR_CUDA;
                if (c == 0 || ms < best) {
                    best = ms;
                    sched = cands[c];
                }
            }
            for (auto &e : ev) cudaEventDestroy(e);
            if (st != GCVO_OK) return st;
            ctx->tuned.emplace_back(key, sched);
        }
    }
    if (packed != sched) GCVO_TRY(pack(ctx, P, sched));
    const int sub = sched & 0xff;
    b.sub = sub;
    b.grid = pair_grid(ctx, P, PAIR_EVAL, sub);
    ctx->last_sub = sub;
    return GCVO_OK;
}

// The buffers of the per-iteration launches, the split pose constants and
// the transformed source at the initial pose, and the pair schedule.  exact:
// the G-CVO-E pass will run (second partial row).
gcvo_status iter_bufs(gcvo_ctx *ctx, const Prepared &P, IterBufs &b, gcvo_iter_log *dlogs, int k_max,
                      bool exact) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    char *part = ctx->partial.as<char>();
    size_t ng = (size_t)std::max(P.n_items, 1);
    float *pf = reinterpret_cast<float *>(part);
    long long *pc = reinterpret_cast<long long *>(part + al(ng * 64 * sizeof(float)));
    const size_t n_chunk_rows = (size_t)(P.n_items / FIN_CHUNK) + (size_t)P.n_problems + 1;
    double *chunk = reinterpret_cast<double *>(part + al(ng * 64 * sizeof(float)) + al(ng * 4 * sizeof(long long)));
    long long *chunk_cnt = reinterpret_cast<long long *>(reinterpret_cast<char *>(chunk) +
                                                         al(n_chunk_rows * 64 * sizeof(double)));
    int *work = reinterpret_cast<int *>(ctx->status_word.as<char>() + 64);
    int *n_active = work + 1;
    if (exact) GCVO_TRY(ctx->partial2.ensure(ng * 64 * sizeof(float), ctx->stream));
    // the tails of p: every pair pass forms r in double-float
    GCVO_TRY(ctx->t_lo.ensure((size_t)std::max<int64_t>(P.n_points, 1) * sizeof(float4), ctx->stream));
    TransformArgs &t = b.ta;
    t.spos = ctx->src_pos.as<float4>();
    t.sca = ctx->src_ca.as<float4>();
    t.scb = ctx->src_cb.as<float4>();
    t.pprob = ctx->pprob.as<int>();
    t.probs = ctx->probs.as<ProbDev>();
    t.tpos = ctx->t_pos.as<float4>();
    t.tca = ctx->t_ca.as<float4>();
    t.tcb = ctx->t_cb.as<float4>();
    t.tlo = ctx->t_lo.as<float4>();
    t.sfx = P.feat_dim > 3 ? ctx->src_fx.as<float4>() : nullptr;
    t.tfx = P.feat_dim > 3 ? ctx->t_fx.as<float4>() : nullptr;
    t.n = P.n_points;
    t.iso = P.iso;
    PairArgs &a = b.pa;
    a.tpos = t.tpos;
    a.tca = t.tca;
    a.tcb = t.tcb;
    a.tlo = t.tlo;
    a.tfx = t.tfx;
    a.items = ctx->items.as<int>();
    a.item_prob = ctx->item_prob.as<int>();
    a.n_items = P.d_nitems;
    a.probs = ctx->probs.as<ProbDev>();
    a.grids = ctx->grids.as<GridDev>();
    a.part = pf;
    a.part2 = exact ? ctx->partial2.as<float>() : nullptr;
    a.counts = pc;
    a.work = work;
    a.status_word = ctx->status_word.as<unsigned>();
    a.ls_literal = 0;
    FinalizeArgs &f = b.fa;
    f.probs = ctx->probs.as<ProbDev>();
    f.grids = ctx->grids.as<GridDev>();
    f.part = pf;
    f.part2 = a.part2;
    f.counts = pc;
    f.chunk = chunk;
    f.chunk_cnt = chunk_cnt;
    f.n_chunks = work + 2;   // written by pack_items
    f.reduce_blocks = std::max(1, ctx->sm_count) * 8;
    f.evalout = ctx->evalout.as<EvalOut>();
    f.logs = dlogs;
    f.n_active = n_active;
    f.n_problems = P.n_problems;
    f.k_max = k_max;
    f.eps_tol = 0;
    f.mu0 = 0;
    b.work = work;
    // transform constants and the transformed source at the initial pose
    f.mode = FIN_POSE;
    GCVO_CUDA(launch_finalize(f, ctx->stream));
    GCVO_CUDA(launch_transform(t, ctx->stream));
    return choose_schedule(ctx, P, b);
}

gcvo_status check_status_word(gcvo_ctx *ctx) {
    unsigned w = 0;
    GCVO_CUDA(cudaMemcpyAsync(&w, ctx->status_word.ptr, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    GCVO_CUDA(cudaStreamSynchronize(ctx->stream));
    if (w & DEV_ERR_TIMEOUT) return GCVO_ERR_TIMEOUT;
    if (w & DEV_ERR_CAPACITY) return GCVO_ERR_CAPACITY;
    if (w & DEV_ERR_NONFINITE) return GCVO_ERR_NONFINITE;
    return GCVO_OK;
}

// With profiling on, a timed launch is bracketed by two events from the
// pool (kind: 0 pair pass, 1 finalize, 2 transform); inside a stream capture
// they become event-record nodes of the graph.  Returns the index of the
// pair, or -1 when profiling is off.
gcvo_status prof_begin(gcvo_ctx *ctx, cudaStream_t s, bool capturing, int kind, long long *slot) {
    *slot = -1;
    if (!ctx->profiling) return GCVO_OK;
    while (ctx->ev_pool.size() < ctx->ev_used + 2) {
        cudaEvent_t e;
        GCVO_CUDA(cudaEventCreate(&e));
        ctx->ev_pool.push_back(e);
    }
    if (ctx->ev_kind.size() < ctx->ev_pool.size() / 2) ctx->ev_kind.resize(ctx->ev_pool.size() / 2);
    ctx->ev_kind[ctx->ev_used / 2] = kind;
    *slot = (long long)ctx->ev_used;
    ctx->ev_used += 2;
    GCVO_CUDA(cudaEventRecordWithFlags(ctx->ev_pool[*slot], s,
                                       capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
    return GCVO_OK;
}

gcvo_status prof_end(gcvo_ctx *ctx, cudaStream_t s, bool capturing, long long slot) {
    if (slot < 0) return GCVO_OK;
    GCVO_CUDA(cudaEventRecordWithFlags(ctx->ev_pool[slot + 1], s,
                                       capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
    return GCVO_OK;
}

// One pair pass on stream s (the work counter is reset first); evaluation
// and G-CVO-E passes are timed when profiling.
gcvo_status launch_pair_pass(gcvo_ctx *ctx, const Prepared &P, IterBufs &b, int mode, cudaStream_t s,
                             bool capturing = false) {
    GCVO_CUDA(cudaMemsetAsync(b.work, 0, sizeof(int), s));
    long long slot = -1;
    if (mode == PAIR_EVAL || mode == PAIR_EXACT) GCVO_TRY(prof_begin(ctx, s, capturing, 0, &slot));
    const int grid = mode == PAIR_EVAL ? b.grid : pair_grid(ctx, P, mode, b.sub);
    GCVO_CUDA(launch_pair(b.pa, mode, P.iso, P.feat_dim, b.sub, grid, s));
    return prof_end(ctx, s, capturing, slot);
}

gcvo_status finalize_timed(gcvo_ctx *ctx, const FinalizeArgs &fa, cudaStream_t s, bool capturing) {
    long long slot;
    GCVO_TRY(prof_begin(ctx, s, capturing, 1, &slot));
    GCVO_CUDA(launch_finalize(fa, s));
    return prof_end(ctx, s, capturing, slot);
}

gcvo_status transform_timed(gcvo_ctx *ctx, const TransformArgs &ta, cudaStream_t s, bool capturing) {
    long long slot;
    GCVO_TRY(prof_begin(ctx, s, capturing, 2, &slot));
    GCVO_CUDA(launch_transform(ta, s));
    return prof_end(ctx, s, capturing, slot);
}

// Add the device time of the recorded launches (stream must be
// synchronised) and release the events for reuse.
gcvo_status collect_profile(gcvo_ctx *ctx, bool keep = false) {
    for (size_t k = 0; k + 1 < ctx->ev_used; k += 2) {
        float ms = 0.f;
        GCVO_CUDA(cudaEventElapsedTime(&ms, ctx->ev_pool[k], ctx->ev_pool[k + 1]));
        switch (ctx->ev_kind[k / 2]) {
            case 0:
                ctx->pair_ms += ms;
                ctx->pair_launches += 1;
                break;
            case 1:
                ctx->fin_ms += ms;
                ctx->fin_launches += 1;
                break;
            default:
                ctx->transform_ms += ms;
        }
    }
    if (!keep) ctx->ev_used = 0;
    return GCVO_OK;
}

// One iteration of Algorithm 1 on stream s: G-CVO-2 is a pair pass and the
// Gauss-Newton finalize; G-CVO-1 a gradient pass, its finalize (direction),
// the line-search pass and the step; G-CVO-E the exact pass and the Newton
// step with H_E = D(g) + Gamma.
gcvo_status enqueue_iteration(gcvo_ctx *ctx, const Prepared &P, IterBufs &b, int order, cudaStream_t s,
                              bool capturing) {
    if (order == 2) {
        GCVO_TRY(launch_pair_pass(ctx, P, b, PAIR_EVAL, s, capturing));
        b.fa.mode = FIN_GN;
        GCVO_TRY(finalize_timed(ctx, b.fa, s, capturing));
    } else if (order == 3) {
        GCVO_TRY(launch_pair_pass(ctx, P, b, PAIR_EXACT, s, capturing));
        b.fa.mode = FIN_EXACT;
        GCVO_TRY(finalize_timed(ctx, b.fa, s, capturing));
    } else {
        GCVO_TRY(launch_pair_pass(ctx, P, b, PAIR_EVAL, s, capturing));
        b.fa.mode = FIN_GRAD;
        GCVO_TRY(finalize_timed(ctx, b.fa, s, capturing));
        GCVO_TRY(launch_pair_pass(ctx, P, b, PAIR_LINESEARCH, s, capturing));
        b.fa.mode = FIN_LINESEARCH;
        GCVO_TRY(finalize_timed(ctx, b.fa, s, capturing));
    }
    // the source at the new poses (problems that stopped keep theirs)
    return transform_timed(ctx, b.ta, s, capturing);
}

// The U-iteration graph of a register call: captured on a private stream,
// instantiated, and destroyed with this object.
struct ChunkGraph {
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;   // kernel launches per replay
    ~ChunkGraph() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

gcvo_status capture_chunk(gcvo_ctx *ctx, const Prepared &P, IterBufs &b, int order, int U, ChunkGraph &cg) {
    if (!ctx->cap_stream) GCVO_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    const long long l0 = launches_so_far();
    GCVO_CUDA(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    gcvo_status st = GCVO_OK;
    for (int u = 0; u < U && st == GCVO_OK; ++u) st = enqueue_iteration(ctx, P, b, order, ctx->cap_stream, true);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
    // captured launches ran nothing: they are counted per replay instead
    cg.kernels = launches_so_far() - l0;
    count_launches(-cg.kernels);
    if (st != GCVO_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (st != GCVO_OK) return st;
        set_last_cuda_error(e, "cudaStreamEndCapture", __LINE__);
        return GCVO_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&cg.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cg.exec = nullptr;
        set_last_cuda_error(e, "cudaGraphInstantiate", __LINE__);
        return GCVO_ERR_CUDA;
    }
    return GCVO_OK;
}

gcvo_status run_register(gcvo_ctx *ctx, int np, const gcvo_problem *pr, const gcvo_solver_params *sp,
                         double *T_out, gcvo_iter_log *logs, int *n_iter, int *status) {
    if (!sp || !T_out || sp->order < 1 || sp->order > 3 || sp->k_max < 1 || sp->k_max > GCVO_MAX_KMAX ||
        !(sp->eps_tol >= 0) || (sp->order == 1 && !(sp->mu0 > 0)))
        return GCVO_ERR_INVALID_ARG;
    cudaStream_t s = ctx->stream;
    Prepared P;
    GCVO_TRY(prepare(ctx, np, pr, P));
    // device log rows only when the caller asked for the log
    gcvo_iter_log *dlogs = nullptr;
    if (logs) {
        GCVO_TRY(ctx->logs.ensure((size_t)np * sp->k_max * sizeof(gcvo_iter_log), s));
        dlogs = ctx->logs.as<gcvo_iter_log>();
        GCVO_CUDA(cudaMemsetAsync(dlogs, 0, (size_t)np * sp->k_max * sizeof(gcvo_iter_log), s));
    }
    IterBufs b{};
    GCVO_TRY(iter_bufs(ctx, P, b, dlogs, sp->k_max, sp->order == 3));
    b.fa.eps_tol = sp->eps_tol;
    b.fa.mu0 = sp->mu0;
    int *n_active = b.fa.n_active;
    GCVO_CUDA(cudaMemcpyAsync(n_active, &np, sizeof(int), cudaMemcpyHostToDevice, s));
    void *hp;
    GCVO_TRY(host_pinned(ctx, 64, &hp));
    int *h_active = static_cast<int *>(hp);
    // U iterations per host check, replayed from one CUDA graph.  Iterations
    // past a problem's convergence or k_max leave it untouched (the finalize
    // skips inactive problems, the pair kernel their items).
    const int U = std::min(8, sp->k_max);
    ChunkGraph cg;
    GCVO_TRY(capture_chunk(ctx, P, b, sp->order, U, cg));
    int it = 0;
    while (it < sp->k_max) {
        GCVO_CUDA(cudaGraphLaunch(cg.exec, s));
        count_launches(cg.kernels);
        it += U;
        GCVO_CUDA(cudaMemcpyAsync(h_active, n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
        GCVO_CUDA(cudaStreamSynchronize(s));
        GCVO_TRY(collect_profile(ctx, true));
        if (*h_active <= 0) break;
    }
    ctx->ev_used = 0;
    GCVO_TRY(check_status_word(ctx));
    std::vector<ProbDev> out(np);
    GCVO_CUDA(cudaMemcpyAsync(out.data(), ctx->probs.ptr, np * sizeof(ProbDev), cudaMemcpyDeviceToHost, s));
    if (logs)
        GCVO_CUDA(cudaMemcpyAsync(logs, dlogs, (size_t)np * sp->k_max * sizeof(gcvo_iter_log),
                                  cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    for (int p = 0; p < np; ++p) {
        const ProbDev &d = out[p];
        double *T = T_out + 16 * p;
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) T[4 * r + c] = d.T[3 * r + c];
            T[4 * r + 3] = d.T[9 + r];
        }
        T[12] = T[13] = T[14] = 0.0;
        T[15] = 1.0;
        if (n_iter) n_iter[p] = d.iter;
        int st;
        if (d.status == 1) st = GCVO_OK;
        else if (d.status == 2 || d.status == 0) st = GCVO_ERR_NOT_CONVERGED;
        else st = -d.status;
        if (status) status[p] = st;
    }
    return GCVO_OK;
}


// ---------------------------------------------------------------------------
// Caller-owned workspace: every scratch buffer of the single-stream calls
// (evaluation, registration, covariances, grid builds) as a fixed slice of
// one caller allocation, sized for calls of at most N points (source points
// of a registration or evaluation, or the cloud of a covariance or grid
// call), np problems and `rows` iteration-log rows.  The slices follow the
// buffers' own size formulas; a call that needs more fails with
// GCVO_ERR_WORKSPACE instead of allocating.
// ---------------------------------------------------------------------------
std::vector<DevBuf *> ws_bufs(gcvo_ctx *c) {
    std::vector<DevBuf *> v = {&c->stage_xyz, &c->stage_cov, &c->small,    &c->sort_keys, &c->sort_vals,
                               &c->sort_tmp,  &c->scan_tmp,  &c->src_pos,  &c->src_ca,    &c->src_cb,
                               &c->pprob,     &c->t_pos,     &c->t_ca,     &c->t_cb,      &c->t_lo,
                               &c->src_fx,    &c->t_fx,
                               &c->items,     &c->item_prob, &c->pack_tmp, &c->partial,   &c->partial2,
                               &c->probs,     &c->grids,     &c->evalout,  &c->logs,      &c->status_word,
                               &c->knn_retry,  &c->knn_meta,  &c->knn_grid.ca, &c->grid_meta, &c->grid_tiles};
    for (GridStore *g : {&c->knn_grid, &c->knn_grid2})
        for (DevBuf *b : {&g->pos, &g->orig, &g->cell_start, &g->hkeys, &g->hval}) v.push_back(b);
    return v;
}

std::vector<size_t> ws_sizes(int64_t N, int64_t np, int64_t rows) {
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t n = (size_t)std::max<int64_t>(N, 1);
    const size_t n64 = (n + 63) / 64 * 64;
    size_t H = 64;
    while (H < 2 * n) H <<= 1;
    const size_t small = al(np * sizeof(SrcDesc)) + al(np * sizeof(int)) * 7 + al(np * sizeof(int64_t)) +
                         al(sizeof(int)) * 4 + 256 + 4096;
    std::vector<size_t> v = {
        (12 * n + 192 * (size_t)np + 192) * sizeof(float),            // stage_xyz: host xyz, cov, feat
        6 * n * sizeof(float),                                          // stage_cov: host covariance output
        std::max<size_t>(small, 4096),                                  // small
        n * sizeof(unsigned long long),                                 // sort_keys
        std::max(al(n * sizeof(int)) * 3, n * sizeof(int) * 2 + 1024),  // sort_vals
        radix_sort_scratch_bytes((int64_t)n),                           // sort_tmp
        scan_scratch_bytes(std::max<int64_t>((int64_t)n, ((int64_t)1 << 26) + 1)) + 1024,   // scan_tmp
        n * sizeof(float4), n * sizeof(float4), n * sizeof(float4),     // src_pos, src_ca, src_cb
        n * sizeof(int),                                                // pprob
        n * sizeof(float4), n * sizeof(float4), n * sizeof(float4), n * sizeof(float4),   // t_pos, t_ca, t_cb, t_lo
        n * sizeof(float4), n * sizeof(float4),                         // src_fx, t_fx
        n * sizeof(int4), n * sizeof(int),                              // items, item_prob
        5 * n64 * sizeof(int),                                          // pack_tmp
        n * (64 * sizeof(float) + 4 * sizeof(long long)) + fin_chunk_bytes((int64_t)n, (int)np) + 4096,   // partial
        n * 64 * sizeof(float),                                         // partial2
        np * sizeof(ProbDev), np * sizeof(GridDev), np * sizeof(EvalOut) + 256,
        (size_t)std::max<int64_t>(rows, 1) * sizeof(gcvo_iter_log),     // logs
        256,                                                            // status_word
        2 * n * sizeof(int) + 256,                                      // knn_retry: two point lists
        knn_meta_bytes((int64_t)n, (int)std::min<int64_t>(2 * np, (int64_t)n)),   // knn_meta
        n * sizeof(float4),                                             // knn_grid.ca: gathered points
        tgrid_meta_bytes((int)std::min<int64_t>(2 * np, (int64_t)n), (int64_t)n),   // grid_meta
        tgrid_tile_bytes(tgrid_max_tiles(1) + 2 * np)};                 // grid_tiles: one grid of 2^26 voxels
    for (int g = 0; g < 2; ++g)
        for (size_t b : {n * sizeof(float4), n * sizeof(int), (n + 1) * sizeof(int), H * sizeof(unsigned long long),
                         H * sizeof(int)})
            v.push_back(b);
    return v;
}

size_t ws_total(const std::vector<size_t> &sz) {
    size_t t = 0;
    for (size_t b : sz) t += (std::max<size_t>(b, 256) + 255) & ~size_t(255);
    return t;
}

}  // namespace

extern "C" {

const char *gcvo_status_string(gcvo_status s) {
    switch (s) {
        case GCVO_OK: return "ok";
        case GCVO_ERR_INVALID_ARG: return "invalid argument";
        case GCVO_ERR_CUDA: return "CUDA runtime error";
        case GCVO_ERR_WORKSPACE: return "device memory allocation failed";
        case GCVO_ERR_SINGULAR: return "singular Gauss-Newton system";
        case GCVO_ERR_NO_OVERLAP: return "no pair within the kernel cutoff";
        case GCVO_ERR_NOT_CONVERGED: return "k_max reached before convergence";
        case GCVO_ERR_NONFINITE: return "non-finite input or result";
        case GCVO_ERR_TIMEOUT: return "device-side wait timed out";
        case GCVO_ERR_CAPACITY: return "size limit exceeded";
    }
    return "unknown status";
}

const char *gcvo_last_error_detail(void) { return last_cuda_error(); }

void gcvo_default_kernel_params(gcvo_kernel_params *p) {
    if (!p) return;
    p->kernel_mode = 0;
    p->sigma2 = 1.0;
    p->cutoff = 3.0;
    p->iso_ell = 0.1;
    p->knn = 10;
    p->eig_max = 0.0;
    p->eig_ratio = 100.0;
    p->feat_dim = 1;
    p->cell_size = 0.0;
}

void gcvo_default_solver_params(gcvo_solver_params *p) {
    if (!p) return;
    p->order = 2;
    p->k_max = 200;
    p->eps_tol = 1e-6;
    p->mu0 = 1e-10;
}

gcvo_status gcvo_create(gcvo_ctx **ctx, int device, void *cuda_stream) {
    if (!ctx) return GCVO_ERR_INVALID_ARG;
    int nd = 0;
    if (cudaGetDeviceCount(&nd) != cudaSuccess || device < 0 || device >= nd) {
        cudaGetLastError();
        return GCVO_ERR_INVALID_ARG;
    }
    GCVO_CUDA(cudaSetDevice(device));
    gcvo_ctx *c = new (std::nothrow) gcvo_ctx();
    if (!c) return GCVO_ERR_WORKSPACE;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete c;
        return GCVO_ERR_CUDA;
    }
    *ctx = c;
    return GCVO_OK;
}

gcvo_status gcvo_destroy(gcvo_ctx *ctx) {
    if (!ctx) return GCVO_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    DevBuf *bufs[] = {&ctx->sort_keys, &ctx->sort_vals, &ctx->sort_tmp, &ctx->scan_tmp, &ctx->small,
                      &ctx->stage_xyz, &ctx->stage_cov, &ctx->stage_feat, &ctx->src_pos, &ctx->src_ca,
                      &ctx->src_cb, &ctx->pprob, &ctx->t_pos, &ctx->t_ca, &ctx->t_cb, &ctx->t_lo,
                      &ctx->src_fx, &ctx->t_fx,
                      &ctx->partial, &ctx->probs, &ctx->grids, &ctx->logs, &ctx->evalout, &ctx->status_word,
                      &ctx->items, &ctx->item_prob, &ctx->pack_tmp, &ctx->partial2};
    for (DevBuf *b : bufs) b->release();
    for (GridStore *kg : {&ctx->knn_grid, &ctx->knn_grid2}) {
        DevBuf *kb[] = {&kg->pos, &kg->ca, &kg->cb, &kg->plo, &kg->orig, &kg->cell_start, &kg->hkeys, &kg->hval,
                        &kg->vox_first};
        for (DevBuf *b : kb) b->release();
    }
    ctx->knn_retry.release();
    ctx->knn_meta.release();
    ctx->grid_meta.release();
    ctx->grid_tiles.release();
    ctx->clouds_stage.release();
    ctx->clouds_cov.release();
    for (gcvo_grid *g : ctx->clouds_grids)
        if (g) gcvo_grid_destroy(g);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    delete ctx;
    return GCVO_OK;
}

gcvo_status gcvo_profile_enable(gcvo_ctx *ctx, int enable) {
    if (!ctx) return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    GCVO_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->profiling = enable ? 1 : 0;
    ctx->ev_used = 0;
    ctx->pair_launches = 0;
    ctx->pair_ms = 0.0;
    ctx->fin_launches = 0;
    ctx->fin_ms = 0.0;
    ctx->transform_ms = 0.0;
    ctx->clouds_cov_ms = 0.0;
    ctx->clouds_grid_ms = 0.0;
    ctx->launch_base = launches_so_far();
    ctx->alloc_base = device_allocs_so_far();
    return GCVO_OK;
}

gcvo_status gcvo_pair_schedule(gcvo_ctx *ctx, int set, int *last_used) {
    const int sub = set & 0xff, level = set >> 8;
    const bool ok_sub = sub == 4 || sub == 8 || sub == 16 || sub == 32, ok_level = level == 0 || (level >= 1 && level <= 3);
    if (!ctx || (set != -1 && set != 0 && !(ok_sub && ok_level))) return GCVO_ERR_INVALID_ARG;
    if (set >= 0) ctx->forced_sub = set;
    if (last_used) *last_used = ctx->last_sub;
    return GCVO_OK;
}

gcvo_status gcvo_profile_read(gcvo_ctx *ctx, gcvo_profile *out) {
    if (!ctx || !out) return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    GCVO_CUDA(cudaStreamSynchronize(ctx->stream));
    GCVO_TRY(collect_profile(ctx));
    out->n_launches = launches_so_far() - ctx->launch_base;
    out->n_pair_launches = ctx->pair_launches;
    out->pair_kernel_ms = ctx->pair_ms;
    out->n_device_allocs = device_allocs_so_far() - ctx->alloc_base;
    out->n_finalize_launches = ctx->fin_launches;
    out->finalize_ms = ctx->fin_ms;
    out->transform_ms = ctx->transform_ms;
    out->clouds_covariance_ms = ctx->clouds_cov_ms;
    out->clouds_grid_ms = ctx->clouds_grid_ms;
    return GCVO_OK;
}

gcvo_status gcvo_estimate_covariances(gcvo_ctx *ctx, const float *xyz, int64_t n, const gcvo_kernel_params *params,
                                      float *cov_out) {
    if (!ctx || !xyz || !cov_out || !params) return GCVO_ERR_INVALID_ARG;
    if (params->knn < 2 || params->knn > GCVO_MAX_KNN || n < params->knn || n > (1 << 28))
        return GCVO_ERR_INVALID_ARG;
    if (params->eig_max > 0 && !(params->eig_ratio >= 1.0)) return GCVO_ERR_INVALID_ARG;
    if (!(params->cutoff >= 0)) return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    size_t need = staged_floats(xyz, 3 * (size_t)n);
    bool host_out = !is_device_ptr(cov_out);
    if (need) GCVO_TRY(ctx->stage_xyz.ensure(need * sizeof(float), ctx->stream));
    size_t off = 0;
    const float *dx;
    GCVO_TRY(stage(ctx, xyz, 3 * (size_t)n, ctx->stage_xyz, off, &dx));
    float *dcov = cov_out;
    if (host_out) {
        GCVO_TRY(ctx->stage_cov.ensure(6 * (size_t)n * sizeof(float), ctx->stream));
        dcov = ctx->stage_cov.as<float>();
    }
    const KnnJob job{dx, dcov, n, params};
    GCVO_TRY(knn_covariances(ctx, 1, &job));
    if (host_out) {
        GCVO_CUDA(cudaMemcpyAsync(cov_out, dcov, 6 * (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        GCVO_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return GCVO_OK;
}

static gcvo_status build_into(gcvo_ctx *ctx, const float *xyz, const float *cov, const float *feat, int64_t n,
                              const gcvo_kernel_params *params, gcvo_grid *g) {
    if (!ctx || !xyz || !feat || !valid_kernel_params(params)) return GCVO_ERR_INVALID_ARG;
    if (params->kernel_mode == 0 && !cov) return GCVO_ERR_INVALID_ARG;
    if (n < 1 || n > (1 << 28)) return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    size_t need = staged_floats(xyz, 3 * (size_t)n) + staged_floats(feat, (size_t)params->feat_dim * n) +
                  (params->kernel_mode == 0 ? staged_floats(cov, 6 * (size_t)n) : 0);
    if (need) GCVO_TRY(ctx->stage_xyz.ensure(need * sizeof(float), s));
    size_t off = 0;
    const float *dx, *dc = nullptr, *df;
    GCVO_TRY(stage(ctx, xyz, 3 * (size_t)n, ctx->stage_xyz, off, &dx));
    if (params->kernel_mode == 0) GCVO_TRY(stage(ctx, cov, 6 * (size_t)n, ctx->stage_xyz, off, &dc));
    GCVO_TRY(stage(ctx, feat, (size_t)params->feat_dim * n, ctx->stage_xyz, off, &df));
    g->device = ctx->device;
    const TgJob job{dx, dc, df, n, params, g};
    return build_target_grids(ctx, 1, &job);
}

gcvo_status gcvo_build_grid(gcvo_ctx *ctx, const float *xyz, const float *cov, const float *feat, int64_t n,
                            const gcvo_kernel_params *params, gcvo_grid **grid_out) {
    if (!grid_out) return GCVO_ERR_INVALID_ARG;
    gcvo_grid *g = new (std::nothrow) gcvo_grid();
    if (!g) return GCVO_ERR_WORKSPACE;
    g->device = ctx ? ctx->device : 0;
    gcvo_status st = build_into(ctx, xyz, cov, feat, n, params, g);
    if (st != GCVO_OK) {
        gcvo_grid_destroy(g);
        return st;
    }
    *grid_out = g;
    return GCVO_OK;
}

gcvo_status gcvo_rebuild_grid(gcvo_ctx *ctx, gcvo_grid *grid, const float *xyz, const float *cov, const float *feat,
                              int64_t n, const gcvo_kernel_params *params) {
    if (!grid) return GCVO_ERR_INVALID_ARG;
    if (ctx && grid->device != ctx->device) return GCVO_ERR_INVALID_ARG;
    return build_into(ctx, xyz, cov, feat, n, params, grid);
}

gcvo_status gcvo_grid_destroy(gcvo_grid *grid) {
    if (!grid) return GCVO_ERR_INVALID_ARG;
    // cudaFree waits for outstanding work on the device, so no stream of a
    // (possibly destroyed) context is needed here
    cudaSetDevice(grid->device);
    GridStore &s = grid->store;
    s.pos.release();
    s.ca.release();
    s.cb.release();
    s.plo.release();
    s.fx.release();
    s.orig.release();
    s.cell_start.release();
    s.hkeys.release();
    s.hval.release();
    s.vox_first.release();
    delete grid;
    return GCVO_OK;
}

gcvo_status gcvo_grid_info(const gcvo_grid *grid, int64_t *n_points, int64_t *n_cells, double *cell_size) {
    if (!grid) return GCVO_ERR_INVALID_ARG;
    if (n_points) *n_points = grid->store.d.n;
    if (n_cells) *n_cells = grid->store.d.n_cells;
    if (cell_size) *cell_size = grid->store.d.h;
    return GCVO_OK;
}

// One evaluation of a single problem at pose T: the pair pass `mode`
// (PAIR_EVAL or PAIR_EXACT) and the finalize `fin` fill one EvalOut, which
// is copied to the host outputs (H and M_out as the finalize wrote them).
static gcvo_status eval_once(gcvo_ctx *ctx, const gcvo_grid *target, const float *src_xyz, const float *src_cov,
                             const float *src_feat, int64_t n_src, const double T[16], int mode, int fin,
                             double *f, double g[6], double H[36], double *M_out, gcvo_eval_stats *stats) {
    GCVO_CUDA(cudaSetDevice(ctx->device));
    gcvo_problem pr{};
    pr.target = target;
    pr.src_xyz = src_xyz;
    pr.src_cov = src_cov;
    pr.src_feat = src_feat;
    pr.n_src = n_src;
    memcpy(pr.T0, T, 16 * sizeof(double));
    Prepared P;
    GCVO_TRY(prepare(ctx, 1, &pr, P));
    IterBufs b{};
    GCVO_TRY(iter_bufs(ctx, P, b, nullptr, 1, mode == PAIR_EXACT));
    int one = 1;
    GCVO_CUDA(cudaMemcpyAsync(b.fa.n_active, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    GCVO_TRY(launch_pair_pass(ctx, P, b, mode, ctx->stream));
    b.fa.mode = fin;
    GCVO_CUDA(launch_finalize(b.fa, ctx->stream));
    EvalOut e{};
    GCVO_CUDA(cudaMemcpyAsync(&e, ctx->evalout.ptr, sizeof(EvalOut), cudaMemcpyDeviceToHost, ctx->stream));
    GCVO_TRY(check_status_word(ctx));
    GCVO_TRY(collect_profile(ctx));
    *f = e.f;
    memcpy(g, e.g, 6 * sizeof(double));
    memcpy(H, e.H, 36 * sizeof(double));
    if (M_out) memcpy(M_out, e.M, 36 * sizeof(double));
    if (stats) {
        stats->n_pairs = e.n_pairs;
        stats->n_kept = e.n_kept;
        stats->n_candidates = e.n_cand;
        stats->rho = std::sqrt((double)P.probs[0].rho2);
    }
    bool finite = std::isfinite(e.f);
    for (int k = 0; k < 6; ++k) finite = finite && std::isfinite(e.g[k]);
    if (mode == PAIR_EXACT)
        for (int k = 0; k < 36; ++k) finite = finite && std::isfinite(e.H[k]);
    return finite ? GCVO_OK : GCVO_ERR_NONFINITE;
}

gcvo_status gcvo_eval(gcvo_ctx *ctx, const gcvo_grid *target, const float *src_xyz, const float *src_cov,
                      const float *src_feat, int64_t n_src, const double T[16], double *f, double g[6],
                      double H[36], double *M_out, gcvo_eval_stats *stats) {
    if (!ctx || !target || !src_xyz || !src_feat || !T || !f || !g || !H) return GCVO_ERR_INVALID_ARG;
    return eval_once(ctx, target, src_xyz, src_cov, src_feat, n_src, T, PAIR_EVAL, FIN_EVAL, f, g, H, M_out,
                     stats);
}

gcvo_status gcvo_eval_exact(gcvo_ctx *ctx, const gcvo_grid *target, const float *src_xyz, const float *src_cov,
                            const float *src_feat, int64_t n_src, const double T[16], double *f, double g[6],
                            double H_E[36], double *D_out, gcvo_eval_stats *stats) {
    if (!ctx || !target || !src_xyz || !src_feat || !T || !f || !g || !H_E) return GCVO_ERR_INVALID_ARG;
    return eval_once(ctx, target, src_xyz, src_cov, src_feat, n_src, T, PAIR_EXACT, FIN_EXACT_EVAL, f, g, H_E,
                     D_out, stats);
}

gcvo_status gcvo_register(gcvo_ctx *ctx, const gcvo_grid *target, const float *src_xyz, const float *src_cov,
                          const float *src_feat, int64_t n_src, const double T0[16],
                          const gcvo_solver_params *params, double T_out[16], gcvo_iter_log *log, int *n_iter) {
    if (!ctx || !target || !src_xyz || !src_feat || !T0 || !T_out) return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    gcvo_problem pr{};
    pr.target = target;
    pr.src_xyz = src_xyz;
    pr.src_cov = src_cov;
    pr.src_feat = src_feat;
    pr.n_src = n_src;
    memcpy(pr.T0, T0, 16 * sizeof(double));
    int st = 0, ni = 0;
    double Tt[16];
    GCVO_TRY(run_register(ctx, 1, &pr, params, Tt, log, &ni, &st));
    memcpy(T_out, Tt, sizeof(Tt));
    if (n_iter) *n_iter = ni;
    return (gcvo_status)st;
}

gcvo_status gcvo_register_batched(gcvo_ctx *ctx, int n_problems, const gcvo_problem *problems,
                                  const gcvo_solver_params *params, double *T_out, gcvo_iter_log *logs,
                                  int *n_iter, int *status) {
    if (!ctx || !problems || !T_out || n_problems < 1) return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    return run_register(ctx, n_problems, problems, params, T_out, logs, n_iter, status);
}

gcvo_status gcvo_estimate_covariances_batched(gcvo_ctx *ctx, int n_clouds, const float *const *xyz,
                                              const int64_t *n, const gcvo_kernel_params *params,
                                              float *const *cov_out) {
    if (!ctx || n_clouds < 1 || !xyz || !n || !params || !cov_out) return GCVO_ERR_INVALID_ARG;
    for (int k = 0; k < n_clouds; ++k)
        if (!xyz[k] || !cov_out[k] || !is_device_ptr(xyz[k]) || !is_device_ptr(cov_out[k]))
            return GCVO_ERR_INVALID_ARG;
    if (params->knn < 2 || params->knn > GCVO_MAX_KNN) return GCVO_ERR_INVALID_ARG;
    if (params->eig_max > 0 && !(params->eig_ratio >= 1.0)) return GCVO_ERR_INVALID_ARG;
    if (!(params->cutoff >= 0)) return GCVO_ERR_INVALID_ARG;
    std::vector<KnnJob> jobs(n_clouds);
    for (int k = 0; k < n_clouds; ++k) {
        if (n[k] < params->knn || n[k] > (1 << 28)) return GCVO_ERR_INVALID_ARG;
        jobs[k] = KnnJob{xyz[k], cov_out[k], n[k], params};
    }
    GCVO_CUDA(cudaSetDevice(ctx->device));
    return knn_covariances(ctx, n_clouds, jobs.data());
}

gcvo_status gcvo_build_grids_batched(gcvo_ctx *ctx, int n_clouds, const float *const *xyz,
                                     const float *const *cov, const float *const *feat, const int64_t *n,
                                     const gcvo_kernel_params *params, gcvo_grid **grids) {
    if (!ctx || n_clouds < 1 || !xyz || !feat || !n || !params || !grids) return GCVO_ERR_INVALID_ARG;
    if (params->kernel_mode == 0 && !cov) return GCVO_ERR_INVALID_ARG;
    for (int k = 0; k < n_clouds; ++k) {
        if (!xyz[k] || !feat[k] || !is_device_ptr(xyz[k]) || !is_device_ptr(feat[k])) return GCVO_ERR_INVALID_ARG;
        if (params->kernel_mode == 0 && (!cov[k] || !is_device_ptr(cov[k]))) return GCVO_ERR_INVALID_ARG;
        if (grids[k] && grids[k]->device != ctx->device) return GCVO_ERR_INVALID_ARG;
    }
    if (!valid_kernel_params(params)) return GCVO_ERR_INVALID_ARG;
    for (int k = 0; k < n_clouds; ++k)
        if (n[k] < 1 || n[k] > (1 << 28)) return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    // new grids for the empty slots; on failure they are released again
    std::vector<TgJob> jobs(n_clouds);
    std::vector<char> created(n_clouds, 0);
    gcvo_status st = GCVO_OK;
    for (int k = 0; k < n_clouds && st == GCVO_OK; ++k) {
        if (!grids[k]) {
            grids[k] = new (std::nothrow) gcvo_grid();
            if (!grids[k]) {
                st = GCVO_ERR_WORKSPACE;
                break;
            }
            grids[k]->device = ctx->device;
            created[k] = 1;
        }
        jobs[k] = TgJob{xyz[k], params->kernel_mode == 0 ? cov[k] : nullptr, feat[k], n[k], params, grids[k]};
    }
    if (st == GCVO_OK) st = build_target_grids(ctx, n_clouds, jobs.data());
    if (st != GCVO_OK)
        for (int k = 0; k < n_clouds; ++k)
            if (created[k]) {
                gcvo_grid_destroy(grids[k]);
                grids[k] = nullptr;
            }
    return st;
}

gcvo_status gcvo_register_clouds(gcvo_ctx *ctx, int n_pairs, const gcvo_cloud_pair *pairs,
                                 const gcvo_kernel_params *params, const gcvo_solver_params *solver, double *T_out,
                                 gcvo_iter_log *logs, int *n_iter, int *status) {
    if (!ctx || n_pairs < 1 || n_pairs > GCVO_MAX_PROBLEMS || !pairs || !params || !solver || !T_out)
        return GCVO_ERR_INVALID_ARG;
    std::vector<const gcvo_kernel_params *> kp(n_pairs);
    for (int k = 0; k < n_pairs; ++k) {
        const gcvo_cloud_pair &q = pairs[k];
        kp[k] = q.params ? q.params : params;
        if (!valid_kernel_params(kp[k]) || kp[k]->kernel_mode != params->kernel_mode ||
            kp[k]->feat_dim != params->feat_dim)
            return GCVO_ERR_INVALID_ARG;
        if (!q.tgt_xyz || !q.tgt_feat || !q.src_xyz || !q.src_feat) return GCVO_ERR_INVALID_ARG;
        if (q.n_tgt < kp[k]->knn || q.n_src < kp[k]->knn || q.n_tgt > (1 << 28) || q.n_src > (1 << 28))
            return GCVO_ERR_INVALID_ARG;
        if (kp[k]->knn < 2 || kp[k]->knn > GCVO_MAX_KNN) return GCVO_ERR_INVALID_ARG;
    }
    GCVO_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const int fd = params->feat_dim;
    // cloud c = 2k (target of pair k) or 2k + 1 (its source)
    const int nc = 2 * n_pairs;
    std::vector<const float *> hx(nc), hf(nc), dx(nc), df(nc);
    std::vector<int64_t> n(nc);
    std::vector<size_t> cov_off(nc);
    size_t stage_floats = 0, cov_floats = 0;
    for (int c = 0; c < nc; ++c) {
        const gcvo_cloud_pair &q = pairs[c / 2];
        hx[c] = c % 2 ? q.src_xyz : q.tgt_xyz;
        hf[c] = c % 2 ? q.src_feat : q.tgt_feat;
        n[c] = c % 2 ? q.n_src : q.n_tgt;
        stage_floats += staged_floats(hx[c], 3 * (size_t)n[c]) + staged_floats(hf[c], (size_t)fd * n[c]);
        cov_off[c] = cov_floats;
        cov_floats += (6 * (size_t)n[c] + 63) & ~size_t(63);
    }
    // host clouds are copied in, one copy per array, in stream order
    if (stage_floats) GCVO_TRY(ctx->clouds_stage.ensure(stage_floats * sizeof(float), s));
    GCVO_TRY(ctx->clouds_cov.ensure(cov_floats * sizeof(float), s));
    size_t off = 0;
    for (int c = 0; c < nc; ++c) {
        GCVO_TRY(stage(ctx, hx[c], 3 * (size_t)n[c], ctx->clouds_stage, off, &dx[c]));
        GCVO_TRY(stage(ctx, hf[c], (size_t)fd * n[c], ctx->clouds_stage, off, &df[c]));
    }
    float *cov = ctx->clouds_cov.as<float>();
    // phase events (profiling): start, covariances done, grids done
    cudaEvent_t ph[3] = {nullptr, nullptr, nullptr};
    if (ctx->profiling)
        for (auto &e : ph) {
            GCVO_CUDA(cudaEventCreate(&e));
        }
    if (ph[0]) GCVO_CUDA(cudaEventRecord(ph[0], s));
    // Eq. (7b) and the eigenvalue bound for every cloud, in one batch
    {
        std::vector<KnnJob> jobs(nc);
        for (int c = 0; c < nc; ++c) {
            const gcvo_kernel_params *p = kp[c / 2];
            if (p->eig_max > 0 && !(p->eig_ratio >= 1.0)) return GCVO_ERR_INVALID_ARG;
            jobs[c] = KnnJob{dx[c], cov + cov_off[c], n[c], p};
        }
        GCVO_TRY(knn_covariances(ctx, nc, jobs.data()));
    }
    if (ph[1]) GCVO_CUDA(cudaEventRecord(ph[1], s));
    // the target grids, kept by the context and rebuilt in place next call,
    // all in one batch
    if ((int)ctx->clouds_grids.size() < n_pairs) ctx->clouds_grids.resize(n_pairs, nullptr);
    {
        std::vector<TgJob> jobs(n_pairs);
        for (int k = 0; k < n_pairs; ++k) {
            gcvo_grid *&g = ctx->clouds_grids[k];
            if (!g) {
                g = new (std::nothrow) gcvo_grid();
                if (!g) return GCVO_ERR_WORKSPACE;
                g->device = ctx->device;
            }
            jobs[k] = TgJob{dx[2 * k], kp[k]->kernel_mode == 0 ? cov + cov_off[2 * k] : nullptr, df[2 * k],
                            n[2 * k], kp[k], g};
        }
        GCVO_TRY(build_target_grids(ctx, n_pairs, jobs.data()));
    }
    if (ph[2]) {
        GCVO_CUDA(cudaEventRecord(ph[2], s));
        GCVO_CUDA(cudaEventSynchronize(ph[2]));
        float a = 0.f, b = 0.f;
        GCVO_CUDA(cudaEventElapsedTime(&a, ph[0], ph[1]));
        GCVO_CUDA(cudaEventElapsedTime(&b, ph[1], ph[2]));
        ctx->clouds_cov_ms += a;
        ctx->clouds_grid_ms += b;
        for (auto &e : ph) cudaEventDestroy(e);
    }
    std::vector<gcvo_problem> pr(n_pairs);
    for (int k = 0; k < n_pairs; ++k) {
        pr[k].target = ctx->clouds_grids[k];
        pr[k].src_xyz = dx[2 * k + 1];
        pr[k].src_cov = cov + cov_off[2 * k + 1];
        pr[k].src_feat = df[2 * k + 1];
        pr[k].n_src = n[2 * k + 1];
        memcpy(pr[k].T0, pairs[k].T0, sizeof(pr[k].T0));
    }
    return run_register(ctx, n_pairs, pr.data(), solver, T_out, logs, n_iter, status);
}

gcvo_status gcvo_workspace_size(const gcvo_ctx *ctx, int64_t max_points, int max_problems, int64_t max_log_rows,
                                size_t *bytes) {
    (void)ctx;
    if (!bytes || max_points < 1 || max_points > (1 << 26) || max_problems < 1 ||
        max_problems > GCVO_MAX_PROBLEMS || max_log_rows < 0 || max_log_rows > ((int64_t)1 << 32))
        return GCVO_ERR_INVALID_ARG;
    *bytes = ws_total(ws_sizes(max_points, max_problems, max_log_rows));
    return GCVO_OK;
}

gcvo_status gcvo_set_workspace(gcvo_ctx *ctx, void *dev_ptr, size_t bytes, int64_t max_points, int max_problems,
                               int64_t max_log_rows) {
    if (!ctx) return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    GCVO_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<DevBuf *> bufs = ws_bufs(ctx);
    if (!dev_ptr) {
        // back to library-owned scratch, allocated on demand
        for (DevBuf *b : bufs)
            if (b->fixed) b->release();
        ctx->ws_ptr = nullptr;
        ctx->ws_bytes = 0;
        return GCVO_OK;
    }
    size_t need = 0;
    GCVO_TRY(gcvo_workspace_size(ctx, max_points, max_problems, max_log_rows, &need));
    if (bytes < need || (reinterpret_cast<uintptr_t>(dev_ptr) & 255u)) return GCVO_ERR_INVALID_ARG;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, dev_ptr) != cudaSuccess) {
        cudaGetLastError();
        return GCVO_ERR_INVALID_ARG;
    }
    if (at.type != cudaMemoryTypeDevice || at.device != ctx->device) return GCVO_ERR_INVALID_ARG;
    // the host read-back buffer, sized once for the problem limit
    void *hp;
    GCVO_TRY(host_pinned(ctx, (size_t)(2 * max_problems + 64) * sizeof(int), &hp));
    const std::vector<size_t> sz = ws_sizes(max_points, max_problems, max_log_rows);
    char *p = static_cast<char *>(dev_ptr);
    for (size_t k = 0; k < bufs.size(); ++k) {
        bufs[k]->release();
        const size_t b = (std::max<size_t>(sz[k], 256) + 255) & ~size_t(255);
        bufs[k]->ptr = p;
        bufs[k]->bytes = b;
        bufs[k]->fixed = true;
        p += b;
    }
    ctx->ws_ptr = dev_ptr;
    ctx->ws_bytes = bytes;
    return GCVO_OK;
}

}  // extern "C"
