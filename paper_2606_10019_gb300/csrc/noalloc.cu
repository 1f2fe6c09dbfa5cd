// gcvo_eval_static: the evaluation of gcvo_eval for callers that cannot
// allocate device memory, with every scratch buffer carved out of one
// file-scope device array instead of context-owned memory.
//
// Who needs it: code that must not call cudaMalloc -- an application whose
// memory pool owns every device byte (a stray allocation fails or fragments
// the pool), a real-time loop that must not risk an allocation failure or
// the device-wide synchronisation cudaMalloc / cudaFree can cause, or a
// plug-in that has no context object to keep buffers in.
//
// The array is reserved once per device when the library is loaded and kept
// until the process exits.  Host code never uses the symbol itself as a
// pointer (on the host it is only a stand-in for the device address): the
// first call on a device looks the real address up with cudaGetSymbolAddress
// and remembers it.
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "pair.cuh"

namespace gcvo {
namespace {

constexpr int64_t NA_MAX_SRC = 65536;                  // source points per call
constexpr int NA_SUB = 8;                              // points per work item (one warp)
constexpr int NA_ITEM = NA_SUB;
constexpr int NA_MAX_ITEMS = (int)(NA_MAX_SRC / NA_ITEM);

// Byte offsets of the pieces of the scratch array (each 256-aligned).
constexpr size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
// The source records are transformed in place (one evaluation, one pose).
constexpr size_t NA_SPOS = 0;
constexpr size_t NA_SCA = NA_SPOS + al256(NA_MAX_SRC * 16);
constexpr size_t NA_SCB = NA_SCA + al256(NA_MAX_SRC * 16);
constexpr size_t NA_TLO = NA_SCB + al256(NA_MAX_SRC * 16);      // tails of the transformed positions
constexpr size_t NA_ITEMS = NA_TLO + al256(NA_MAX_SRC * 16);
constexpr size_t NA_IPROB = NA_ITEMS + al256(NA_MAX_ITEMS * 4);
constexpr size_t NA_PART = NA_IPROB + al256(NA_MAX_ITEMS * 4);
constexpr size_t NA_COUNTS = NA_PART + al256((size_t)NA_MAX_ITEMS * 64 * 4);
constexpr size_t NA_CHUNK_ROWS = NA_MAX_ITEMS / FIN_CHUNK + 2;
constexpr size_t NA_CHUNK = NA_COUNTS + al256((size_t)NA_MAX_ITEMS * 4 * 8);
constexpr size_t NA_CHUNKCNT = NA_CHUNK + al256(NA_CHUNK_ROWS * 64 * 8);
constexpr size_t NA_PROB = NA_CHUNKCNT + al256(NA_CHUNK_ROWS * 4 * 8);
constexpr size_t NA_GRID = NA_PROB + al256(sizeof(ProbDev));
constexpr size_t NA_EVAL = NA_GRID + al256(sizeof(GridDev));
constexpr size_t NA_WORDS = NA_EVAL + al256(sizeof(EvalOut));   // work, n_items, lam, status, n_active, n_chunks
constexpr size_t NA_BYTES = NA_WORDS + 256;
// 4 MiB of source records and position tails, 2 MiB of partials, 256 KiB of
// counters, 64 KiB of work items and 18 KiB of finalize chunk sums: the
// 6.3 MiB the header documents
static_assert(NA_BYTES >= size_t(6300) * 1048576 / 1000 && NA_BYTES <= size_t(6350) * 1048576 / 1000,
              "the documented size of the static scratch (6.3 MiB)");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Pack the caller's SoA source (in its own order) into the float4 records of
// the pair kernel and the largest covariance eigenvalue.  A work item holds
// NA_ITEM consecutive points of the caller's order.
__global__ void k_na_pack(const float *xyz, const float *cov, const float *feat, int feat_dim, int n, int iso,
                          unsigned char *base) {
    float4 *spos = reinterpret_cast<float4 *>(base + NA_SPOS);
    float4 *sca = reinterpret_cast<float4 *>(base + NA_SCA);
    float4 *scb = reinterpret_cast<float4 *>(base + NA_SCB);
    int *items = reinterpret_cast<int *>(base + NA_ITEMS);
    int *iprob = reinterpret_cast<int *>(base + NA_IPROB);
    int *words = reinterpret_cast<int *>(base + NA_WORDS);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s[6] = {0, 0, 0, 0, 0, 0};
    bool bad = false;
    if (!iso)
        for (int k = 0; k < 6; ++k) {
            s[k] = cov[(size_t)k * n + i];
            bad |= !isfinite(s[k]);
        }
    const float x = xyz[i], y = xyz[n + i], z = xyz[2 * (size_t)n + i];
    bad |= !isfinite(x) || !isfinite(y) || !isfinite(z);
    const float f0 = feat[i];
    const float f1 = feat_dim > 1 ? feat[n + i] : 0.f;
    const float f2 = feat_dim > 2 ? feat[2 * (size_t)n + i] : 0.f;
    spos[i] = make_float4(x, y, z, f0);
    sca[i] = make_float4(s[0], s[1], s[2], s[3]);
    scb[i] = make_float4(s[4], s[5], f1, f2);
    if (!iso) {
        float l = sym3_max_eig(s[0], s[1], s[2], s[3], s[4], s[5]);
        int e = __float_as_int(l);
        atomicMax(words + 2, e >= 0 ? e : e ^ 0x7fffffff);
    }
    if (bad) atomicOr(reinterpret_cast<unsigned *>(words + 3), DEV_ERR_NONFINITE);
    if (i % NA_ITEM == 0) {
        // a work item of NA_ITEM consecutive points: first << 6 | points
        items[i / NA_ITEM] = (int)(((unsigned)i << 6) | (unsigned)min(NA_ITEM, n - i));
        iprob[i / NA_ITEM] = 0;
    }
}

struct NaSetup {
    double T[16];
    double cutoff, sigma2, iso_ell;
    int kernel_mode;
    int n_src, n_items;
};

// The per-problem state of the single problem (what prepare() fills in for
// gcvo_eval): pose, ranges and the Euclidean pre-test radius.
__global__ void k_na_setup(NaSetup a, unsigned char *base) {
    ProbDev *P = reinterpret_cast<ProbDev *>(base + NA_PROB);
    const GridDev *G = reinterpret_cast<const GridDev *>(base + NA_GRID);
    int *words = reinterpret_cast<int *>(base + NA_WORDS);
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) P->T[3 * r + c] = a.T[4 * r + c];
        P->T[9 + r] = a.T[4 * r + 3];
    }
    P->status = 0;
    P->iter = 0;
    P->w0 = 0;
    P->w1 = a.n_items;
    P->c0 = 0;
    P->c1 = (a.n_items + FIN_CHUNK - 1) / FIN_CHUNK;
    P->lo = 1;   // r from double-float positions (no eigenvalue bounds here)
    const int le = words[2];
    const float lam_src = __int_as_float(le >= 0 ? le : le ^ 0x7fffffff);
    double c2 = a.cutoff * a.cutoff;
    double rho2 = a.kernel_mode == 1 ? c2 * a.iso_ell * a.iso_ell * (1.0 + 1e-5)
                                     : c2 * ((double)G->lam_max + (double)lam_src) * (1.0 + 2e-4) + 1e-12;
    if (a.cutoff == 0) rho2 = c2 = INFINITY;   // dense: every pair
    P->rho2 = (float)rho2;
    P->c2 = (float)c2;
    P->sigma2 = (float)a.sigma2;
    P->iso_inv = a.kernel_mode == 1 ? (float)(1.0 / (a.iso_ell * a.iso_ell)) : 0.f;
    words[1] = a.n_items;
    words[4] = 1;
    words[5] = P->c1;
}

std::mutex g_na_mutex;
unsigned char *g_na_addr[64];   // device address of the scratch array, per device

}  // namespace
}  // namespace gcvo

using namespace gcvo;

extern "C" gcvo_status gcvo_eval_static(const gcvo_grid *target, const float *src_xyz, const float *src_cov,
                                        const float *src_feat, int64_t n_src, const double T[16], void *cuda_stream,
                                        double *f, double g[6], double H[36]) {
    if (!target || !src_xyz || !src_feat || !T || !f || !g || !H) return GCVO_ERR_INVALID_ARG;
    if (target->kp.kernel_mode == 0 && !src_cov) return GCVO_ERR_INVALID_ARG;
    if (target->kp.feat_dim > 3) return GCVO_ERR_INVALID_ARG;   // the scratch holds 3 feature channels
    if (n_src < 1) return GCVO_ERR_INVALID_ARG;
    if (n_src > NA_MAX_SRC) return GCVO_ERR_CAPACITY;   // beyond the static scratch
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(T[k])) return GCVO_ERR_NONFINITE;
    const int dev = target->device;
    if (dev < 0 || dev >= 64) return GCVO_ERR_INVALID_ARG;
    // inputs must already be on the grid's device (a copy would need a buffer)
    for (const float *p : {src_xyz, src_cov, src_feat}) {
        if (!p) continue;
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return GCVO_ERR_INVALID_ARG;
        }
        if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return GCVO_ERR_INVALID_ARG;
        if (at.type == cudaMemoryTypeDevice && at.device != dev) return GCVO_ERR_INVALID_ARG;
    }
    GCVO_CUDA(cudaSetDevice(dev));
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lk(g_na_mutex);
        if (!g_na_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                set_last_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __LINE__);
                return GCVO_ERR_CUDA;
            }
            g_na_addr[dev] = static_cast<unsigned char *>(p);
        }
        base = g_na_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int n = (int)n_src;
    const int n_items = (n + NA_ITEM - 1) / NA_ITEM;
    const bool iso = target->kp.kernel_mode == 1;
    const int fd = target->kp.feat_dim;
    // the array keeps the previous call's contents: zero the counters
    GCVO_CUDA(cudaMemsetAsync(base + NA_WORDS, 0, 256, s));
    GCVO_CUDA(cudaMemcpyAsync(base + NA_GRID, &target->store.d, sizeof(GridDev), cudaMemcpyHostToDevice, s));
    k_na_pack<<<(n + 255) / 256, 256, 0, s>>>(src_xyz, iso ? nullptr : src_cov, src_feat, fd, n, iso ? 1 : 0, base);
    NaSetup su{};
    memcpy(su.T, T, sizeof(su.T));
    su.cutoff = target->kp.cutoff;
    su.sigma2 = target->kp.sigma2;
    su.iso_ell = target->kp.iso_ell;
    su.kernel_mode = target->kp.kernel_mode;
    su.n_src = n;
    su.n_items = n_items;
    k_na_setup<<<1, 1, 0, s>>>(su, base);
    count_launches(2);
    GCVO_CUDA(cudaGetLastError());
    int *words = reinterpret_cast<int *>(base + NA_WORDS);
    FinalizeArgs fa{};
    fa.probs = reinterpret_cast<ProbDev *>(base + NA_PROB);
    fa.grids = reinterpret_cast<const GridDev *>(base + NA_GRID);
    fa.part = reinterpret_cast<const float *>(base + NA_PART);
    fa.counts = reinterpret_cast<const long long *>(base + NA_COUNTS);
    fa.chunk = reinterpret_cast<double *>(base + NA_CHUNK);
    fa.chunk_cnt = reinterpret_cast<long long *>(base + NA_CHUNKCNT);
    fa.n_chunks = words + 5;
    fa.evalout = reinterpret_cast<EvalOut *>(base + NA_EVAL);
    fa.logs = nullptr;
    fa.n_active = words + 4;
    fa.n_problems = 1;
    fa.k_max = 1;
    fa.mode = FIN_POSE;
    GCVO_CUDA(launch_finalize(fa, s));
    // the source in the grid's frame at T, in place
    TransformArgs ta{};
    ta.spos = ta.tpos = reinterpret_cast<float4 *>(base + NA_SPOS);
    ta.sca = ta.tca = reinterpret_cast<float4 *>(base + NA_SCA);
    ta.scb = ta.tcb = reinterpret_cast<float4 *>(base + NA_SCB);
    ta.tlo = reinterpret_cast<float4 *>(base + NA_TLO);
    ta.sfx = nullptr;
    ta.tfx = nullptr;
    ta.pprob = nullptr;
    ta.probs = fa.probs;
    ta.n = n;
    ta.iso = iso ? 1 : 0;
    GCVO_CUDA(launch_transform(ta, s));
    PairArgs pa{};
    pa.tpos = ta.tpos;
    pa.tca = ta.tca;
    pa.tcb = ta.tcb;
    pa.tlo = ta.tlo;
    pa.tfx = nullptr;
    pa.items = reinterpret_cast<const int *>(base + NA_ITEMS);
    pa.item_prob = reinterpret_cast<const int *>(base + NA_IPROB);
    pa.n_items = words + 1;
    pa.probs = fa.probs;
    pa.grids = fa.grids;
    pa.part = reinterpret_cast<float *>(base + NA_PART);
    pa.counts = reinterpret_cast<long long *>(base + NA_COUNTS);
    pa.work = words;
    pa.status_word = reinterpret_cast<unsigned *>(words + 3);
    pa.ls_literal = 0;
    int sm = 0;
    GCVO_CUDA(cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = pair_blocks_per_sm(PAIR_EVAL, iso, fd, NA_SUB);
    int grid = std::max(1, std::min(n_items, std::max(1, per_sm) * sm));
    GCVO_CUDA(launch_pair(pa, PAIR_EVAL, iso, fd, NA_SUB, grid, s));
    fa.mode = FIN_EVAL;
    fa.reduce_blocks = std::max(1, sm) * 8;
    GCVO_CUDA(launch_finalize(fa, s));
    EvalOut e;
    unsigned st = 0;
    GCVO_CUDA(cudaMemcpyAsync(&e, base + NA_EVAL, sizeof(EvalOut), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaMemcpyAsync(&st, words + 3, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    if (st & DEV_ERR_NONFINITE) return GCVO_ERR_NONFINITE;
    if (st & DEV_ERR_TIMEOUT) return GCVO_ERR_TIMEOUT;
    bool fin = std::isfinite(e.f);
    for (int k = 0; k < 6; ++k) fin = fin && std::isfinite(e.g[k]);
    if (!fin) return GCVO_ERR_NONFINITE;
    *f = e.f;
    memcpy(g, e.g, 6 * sizeof(double));
    memcpy(H, e.H, 36 * sizeof(double));
    return GCVO_OK;
}
