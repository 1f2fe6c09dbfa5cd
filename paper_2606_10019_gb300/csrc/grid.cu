// Per-point kNN covariances (gcvo_estimate_covariances, Eq. 7b and the
// eigenvalue bound that follows it) and the voxel-hash primitives they use.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "knn.cuh"

namespace gcvo {
namespace {

__global__ void k_heads(const unsigned long long *keys, int64_t n, int *head) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_cells(const unsigned long long *keys, const int *incl, int64_t n, int *cell_start,
                        unsigned long long *hkeys, int *hval, unsigned long long hmask) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long k = keys[i];
    if (i == 0 || k != keys[i - 1]) {
        int c = incl[i] - 1;
        cell_start[c] = (int)i;
        unsigned long long s = hash_key(k) & hmask;
        for (;;) {
            unsigned long long prev = atomicCAS(hkeys + s, EMPTY_KEY, k);
            if (prev == EMPTY_KEY || prev == k) {
                hval[s] = c;
                break;
            }
            s = (s + 1) & hmask;
        }
    }
    if (i == n - 1) cell_start[incl[i]] = (int)n;
}

__global__ void k_fill_u64(unsigned long long *p, int64_t n, unsigned long long v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace

// ---------------------------------------------------------------------------
// kNN covariances of a batch of clouds (Eq. 7b and the eigenvalue bound that
// follows it) in one set of launches.  The points of all clouds are gathered
// into one array; every cloud keeps its own voxel box and voxel size, and its
// voxel keys are offset by the voxel counts of the clouds before it, so that
// one sort, one voxel list and one hash table serve the whole batch.  Each
// point then searches its own cloud: shells of voxels around its voxel,
// stopping once the knn-th distance is within the shells' reach.  Three
// grids per cloud, voxel edges h, 3h and 9h: every point first searches two
// shells of the fine grid (one thread per point); the points whose
// neighbours lie farther away (sparse parts of a LiDAR frame) search two
// shells of the middle grid, and the few left one warp per point on the
// coarse grid without a shell limit.  The neighbour list is ordered by
// (squared distance, index in the cloud), so the result depends neither on
// the voxel sizes, nor on the pass that finds it, nor on the other clouds of
// the batch.
//
// Host syncs per batch: the key widths (after the voxel sizes are set) and
// the number of points left after each pass (the middle and coarse grids are
// built only when there are some), then the status.
// ---------------------------------------------------------------------------
namespace {

using namespace knn;

constexpr int KC_CHUNK = 4096;      // points per block of the gather
constexpr int KC_BOX = 8;           // ints per cloud: enc min xyz, enc max xyz, bad, occupied voxels
constexpr int KC_AXIS_MAX = 1 << 20;
constexpr double KC_PROD_MAX = 1099511627776.0;   // 2^40 voxels per cloud and grid
constexpr int KC_OCC_SHIFT = 50;                   // occupancy keys: cloud << 50 | voxel
constexpr int64_t KC_GROUP_POINTS = (int64_t)1 << 24;
constexpr int KC_SETUP_THREADS = 256;
constexpr int KC_MID = 3, KC_COARSE = 9;           // voxel edges of the second and third grids, in fine voxels
constexpr int KC_GROUP_CLOUDS = 1 << (63 - KC_OCC_SHIFT);

__device__ __forceinline__ int kc_enc(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float kc_dec(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

// the voxel of point p in grid g, clamped to the grid
__device__ __forceinline__ unsigned long long kc_voxel(const GridDev &g, float4 p) {
    float pc[3] = {p.x, p.y, p.z};
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int q = (int)floorf((pc[a] - g.corner[a]) * g.inv_h);
        c[a] = min(max(q, 0), g.dims[a] - 1);
    }
    return ((unsigned long long)c[0] * g.dims[1] + c[1]) * g.dims[2] + c[2];
}

// Box and occupancy counters to their identities, the occupancy set empty.
__global__ void k_kc_init(int *box, int n_clouds, unsigned long long *hset, int64_t H) {
    const int64_t nb = (int64_t)n_clouds * KC_BOX;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < max(H, nb);
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < H) hset[i] = EMPTY_KEY;
        if (i < nb) {
            const int k = (int)(i % KC_BOX);
            box[i] = k < 3 ? 0x7fffffff : (k < 6 ? (int)0x80000000 : 0);
        }
    }
}

// One block per chunk of one cloud: copies the points into the gathered array
// (the cloud's index in w) and folds them into the cloud's box.
__global__ void k_kc_gather(const KnnCloud *cl, const int2 *chunks, float4 *P, int *box) {
    const int2 ch = chunks[blockIdx.x];
    const KnnCloud c = cl[ch.x];
    const int64_t i0 = (int64_t)ch.y * KC_CHUNK;
    const int64_t i1 = min(c.n, i0 + KC_CHUNK);
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        float v[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            v[a] = c.xyz[a * c.n + i];
            if (!isfinite(v[a])) bad = 1;
            mn[a] = fminf(mn[a], v[a]);
            mx[a] = fmaxf(mx[a], v[a]);
        }
        P[c.off + i] = make_float4(v[0], v[1], v[2], __int_as_float(ch.x));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        int *b = box + (int64_t)ch.x * KC_BOX;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (mn[a] <= mx[a]) {
                atomicMin(b + a, kc_enc(mn[a]));
                atomicMax(b + 3 + a, kc_enc(mx[a]));
            }
        }
        if (bad) atomicOr(b + 6, 1);
    }
}

// Voxel size h, box corner and dims of cloud c's grid: the axis counts are
// kept within KC_AXIS_MAX and their product within prod_max by doubling h
// (the search is exact at any voxel size).  False for a cloud with a
// non-finite box.
__device__ bool kc_grid(const int *b, double h, double prod_max, GridDev &g, double &prod) {
    float mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
        mn[a] = kc_dec(b[a]);
        mx[a] = kc_dec(b[3 + a]);
    }
    double ext[3];
    for (int a = 0; a < 3; ++a) {
        ext[a] = (double)mx[a] - (double)mn[a];
        if (!(ext[a] >= 0.0) || !isfinite(ext[a])) return false;
    }
    if (!(h > 0.0) || !isfinite(h)) h = 1.0;
    for (int it = 0; it < 400; ++it) {
        prod = 1.0;
        bool fits = true;
        for (int a = 0; a < 3; ++a) {
            const double d = floor(ext[a] / h) + 2.0;
            fits = fits && d <= (double)KC_AXIS_MAX;
            prod *= d;
        }
        if (fits && prod <= prod_max) break;
        h *= 2.0;
    }
    g.h = (float)h;
    g.inv_h = (float)(1.0 / h);
    prod = 1.0;
    for (int a = 0; a < 3; ++a) {
        g.corner[a] = mn[a];
        g.dims[a] = (int)fmin(floor(ext[a] / h) + 2.0, (double)KC_AXIS_MAX);
        prod *= g.dims[a];
    }
    return prod <= prod_max;
}

// One thread per cloud: the voxel size from the kernel range (or from the
// box: about two mean point spacings) and the grid for counting occupied
// voxels.
__global__ void k_kc_grid0(const KnnCloud *cl, int n_clouds, int *box, GridDev *gf) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_clouds) return;
    int *b = box + (int64_t)c * KC_BOX;
    double h = cl[c].cell0;
    if (!(h > 0.0)) {
        double vol = 1.0;
        int nz = 0;
        for (int a = 0; a < 3; ++a) {
            const double e = (double)kc_dec(b[3 + a]) - (double)kc_dec(b[a]);
            if (e > 0) {
                vol *= e;
                ++nz;
            }
        }
        h = nz > 0 ? pow(vol / (double)cl[c].n, 1.0 / nz) * 2.0 : 1.0;
    }
    GridDev g{};
    double prod = 0.0;
    if (b[6] || !kc_grid(b, h, (double)(1ull << KC_OCC_SHIFT), g, prod)) {
        b[6] = 1;
        g.h = 1.f;
        g.inv_h = 1.f;
        g.dims[0] = g.dims[1] = g.dims[2] = 1;
    }
    gf[c] = g;
}

// Occupied voxels of each cloud at the first voxel size: insertion into a
// set of (cloud, voxel) keys, counting the new ones.
__global__ void k_kc_occupancy(const float4 *P, int64_t N, const GridDev *gf, unsigned long long *hset,
                               unsigned long long hmask, int *box) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = P[i];
        const int c = cloud_of(p);
        const unsigned long long key = ((unsigned long long)c << KC_OCC_SHIFT) | kc_voxel(gf[c], p);
        unsigned long long s = hash_key(key) & hmask;
        for (unsigned long long probe = 0; probe <= hmask; ++probe) {
            const unsigned long long prev = atomicCAS(hset + s, EMPTY_KEY, key);
            if (prev == EMPTY_KEY) {
                atomicAdd(box + (int64_t)c * KC_BOX + 7, 1);
                break;
            }
            if (prev == key) break;
            s = (s + 1) & hmask;
        }
    }
}

// One block: the three search grids of every cloud and their key offsets.
// A voxel from the kernel range can hold hundreds of points of a dense
// cloud, and every query would sort all of them; so the fine voxel shrinks
// towards about knn / 2 points per occupied voxel (points on surfaces: the
// count scales with the square of the edge), at most 16-fold.  The middle
// grid (KC_MID fine voxels per edge) serves the points whose neighbours lie
// beyond the fine grid's two shells, the coarse grid (KC_COARSE) those
// beyond the middle grid's.  tot: key ranges of the three grids, and
// whether any cloud had a non-finite point.
__global__ void __launch_bounds__(KC_SETUP_THREADS)
    k_kc_setup(const KnnCloud *cl, int n_clouds, int *box, const GridDev ta, const GridDev tb, GridDev *gf,
               GridDev *gm, GridDev *gc, unsigned long long *tot) {
    __shared__ unsigned long long sp[3][KC_SETUP_THREADS];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    GridDev *const out[3] = {gf, gm, gc};
    const double scale[3] = {1.0, (double)KC_MID, (double)KC_COARSE};
    const int per = (n_clouds + blockDim.x - 1) / blockDim.x;
    const int c0 = threadIdx.x * per, c1 = min(n_clouds, c0 + per);
    unsigned long long acc[3] = {0ull, 0ull, 0ull};
    for (int c = c0; c < c1; ++c) {
        int *b = box + (int64_t)c * KC_BOX;
        GridDev g[3] = {ta, tb, ta};   // the coarse grid reuses the fine grid's storage
        double pr[3] = {1.0, 1.0, 1.0};
        bool ok = !b[6];
        if (ok) {
            double h = gf[c].h;
            const int knn = cl[c].knn;
            const double occ = (double)cl[c].n / (double)max(1, b[7]);
            if (occ > 2.0 * knn) h *= fmax(1.0 / 16.0, sqrt(0.5 * knn / occ));
            for (int l = 0; l < 3 && ok; ++l) ok = kc_grid(b, scale[l] * h, KC_PROD_MAX, g[l], pr[l]);
        }
        if (!ok) {
            b[6] = 1;
            sbad = 1;
            for (int l = 0; l < 3; ++l) {
                g[l].h = g[l].inv_h = 1.f;
                g[l].dims[0] = g[l].dims[1] = g[l].dims[2] = 1;
                pr[l] = 1.0;
            }
        }
        for (int l = 0; l < 3; ++l) {
            g[l].n = (int)cl[c].n;
            out[l][c] = g[l];
            acc[l] += (unsigned long long)pr[l];
        }
    }
    for (int l = 0; l < 3; ++l) sp[l][threadIdx.x] = acc[l];
    __syncthreads();
    // inclusive scan over the threads' sums (Hillis-Steele)
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        unsigned long long v[3];
        for (int l = 0; l < 3; ++l) v[l] = threadIdx.x >= o ? sp[l][threadIdx.x - o] : 0ull;
        __syncthreads();
        for (int l = 0; l < 3; ++l) sp[l][threadIdx.x] += v[l];
        __syncthreads();
    }
    for (int l = 0; l < 3; ++l) {
        unsigned long long base = sp[l][threadIdx.x] - acc[l];
        for (int c = c0; c < c1; ++c) {
            GridDev &g = out[l][c];
            g.key_base = base;
            base += (unsigned long long)g.dims[0] * g.dims[1] * g.dims[2];
        }
    }
    if (threadIdx.x == blockDim.x - 1)
        for (int l = 0; l < 3; ++l) tot[l] = sp[l][threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) tot[3] = sbad;
}

__global__ void k_kc_keys(const float4 *P, int64_t N, const GridDev *g, unsigned long long *keys, int *vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 p = P[i];
    const GridDev &gc = g[cloud_of(p)];
    keys[i] = gc.key_base + kc_voxel(gc, p);
    vals[i] = (int)i;
}

__global__ void k_kc_reorder(const float4 *P, const int *vals, int64_t N, const KnnCloud *cl, float4 *pos,
                             int *orig) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int j = vals[i];
    const float4 p = P[j];
    pos[i] = p;
    orig[i] = (int)(j - cl[cloud_of(p)].off);
}

// The search in shells 1 and 2 of grid g[cloud], one thread per point:
// list == null takes every sorted point of grid g (pass 1, queries in voxel
// order), otherwise the points of list (indices into the gathered array P).
// Points whose neighbours lie farther away are queued in out (gathered
// indices) for the next grid.
__global__ void k_knn_cov(const GridDev *g, const KnnCloud *cl, const float4 *P, const int *list, const int *n_list,
                          int64_t N, int *out, int *n_out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (list ? (int64_t)*n_list : N)) return;
    float4 q;
    int j;
    if (list) {
        j = list[t];
        q = P[j];
    } else {
        q = g[0].pos[t];
        j = (int)(cl[cloud_of(q)].off + g[0].orig[t]);
    }
    const int c = cloud_of(q);
    const KnnCloud &k = cl[c];
    KnnList L;
    if (knn_search(g[c], q, k.knn, 2, L))
        knn_write_cov<true>(g[c], q, L, k.knn, k.eig_max, k.eig_ratio, k.n, (int)(j - k.off), k.cov);
    else
        out[atomicAdd(n_out, 1)] = j;
}

}  // namespace

void launch_knn_far(const GridDev *gc, const KnnCloud *cl, const float4 *P, const int *list, const int *n_list,
                    int *next, unsigned *status, int sm_count, int64_t m_max, cudaStream_t s);

size_t knn_meta_bytes(int64_t n_points, int n_clouds) {
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t C = (size_t)std::max(n_clouds, 1);
    const size_t chunks = (size_t)(n_points / KC_CHUNK) + C;
    return al(C * sizeof(KnnCloud)) + 3 * al(C * sizeof(GridDev)) + al(C * KC_BOX * sizeof(int)) +
           al(chunks * sizeof(int2)) + al(4 * sizeof(unsigned long long));
}

namespace {

// Sorted points, voxel ranges and hash table of the grids g[0 .. C-1] into
// store (pos, orig, cell_start, hkeys, hval); P is the gathered array.
gcvo_status kc_build(gcvo_ctx *ctx, const float4 *P, int64_t N, const KnnCloud *cl, const GridDev *g,
                     unsigned long long key_range, unsigned long long H, GridStore &st) {
    cudaStream_t s = ctx->stream;
    int bits = 1;
    while (bits < 62 && (1ull << bits) < key_range) ++bits;
    auto *keys = ctx->sort_keys.as<unsigned long long>();
    int *vals = ctx->sort_vals.as<int>();
    int *incl = vals + ((N + 63) / 64) * 64;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    k_kc_keys<<<blocks, 256, 0, s>>>(P, N, g, keys, vals);
    count_launches(1);
    GCVO_CUDA(cudaGetLastError());
    GCVO_TRY(radix_sort_pairs(keys, vals, N, bits, ctx->sort_tmp.ptr, ctx->sort_tmp.bytes, s));
    k_heads<<<blocks, 256, 0, s>>>(keys, N, incl);
    count_launches(1);
    GCVO_TRY(scan_inclusive_sum(incl, N, ctx->scan_tmp.ptr, s));
    k_fill_u64<<<(unsigned)((H + 255) / 256), 256, 0, s>>>(st.hkeys.as<unsigned long long>(), (int64_t)H, EMPTY_KEY);
    k_cells<<<blocks, 256, 0, s>>>(keys, incl, N, st.cell_start.as<int>(), st.hkeys.as<unsigned long long>(),
                                   st.hval.as<int>(), H - 1);
    k_kc_reorder<<<blocks, 256, 0, s>>>(P, vals, N, cl, st.pos.as<float4>(), st.orig.as<int>());
    count_launches(3);
    GCVO_CUDA(cudaGetLastError());
    return GCVO_OK;
}

}  // namespace

namespace {

gcvo_status knn_cov_group(gcvo_ctx *ctx, int n_clouds, const KnnJob *jobs) {
    cudaStream_t s = ctx->stream;
    const int C = n_clouds;
    std::vector<KnnCloud> cl(C);
    std::vector<int2> chunks;
    int64_t N = 0;
    for (int c = 0; c < C; ++c) {
        const KnnJob &j = jobs[c];
        const gcvo_kernel_params &kp = *j.kp;
        if (j.n < kp.knn || j.n > ((int64_t)1 << 28)) return GCVO_ERR_INVALID_ARG;
        KnnCloud &k = cl[c];
        k.xyz = j.xyz;
        k.cov = j.cov;
        k.n = j.n;
        k.off = N;
        k.eig_max = kp.eig_max;
        k.eig_ratio = kp.eig_ratio;
        // the kernel range when an eigenvalue bound is given; otherwise a
        // size from the box (the shell search adapts)
        k.cell0 = kp.eig_max > 0 ? (kp.cutoff > 0 ? kp.cutoff : 3.0) * std::sqrt(2.0 * kp.eig_max) * 0.5 : 0.0;
        k.knn = kp.knn;
        k.pad = 0;
        for (int64_t q = 0; q * KC_CHUNK < j.n; ++q) chunks.push_back(make_int2(c, (int)q));
        N += j.n;
    }
    unsigned long long H = 64;
    while (H < 2ull * (unsigned long long)N) H <<= 1;

    // scratch
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    GCVO_TRY(ctx->knn_meta.ensure(knn_meta_bytes(N, C), s));
    char *m = static_cast<char *>(ctx->knn_meta.ptr);
    auto *d_cl = reinterpret_cast<KnnCloud *>(m);
    m += al(C * sizeof(KnnCloud));
    GridDev *d_g[3];
    for (auto &p : d_g) {
        p = reinterpret_cast<GridDev *>(m);
        m += al(C * sizeof(GridDev));
    }
    int *d_box = reinterpret_cast<int *>(m);
    m += al((size_t)C * KC_BOX * sizeof(int));
    auto *d_chunks = reinterpret_cast<int2 *>(m);
    m += al(((size_t)(N / KC_CHUNK) + C) * sizeof(int2));
    auto *d_tot = reinterpret_cast<unsigned long long *>(m);
    GridStore &sa = ctx->knn_grid;    // fine, then coarse
    GridStore &sb = ctx->knn_grid2;   // middle
    GCVO_TRY(sa.ca.ensure(N * sizeof(float4), s));   // the gathered points
    for (GridStore *st : {&sa, &sb}) {
        GCVO_TRY(st->pos.ensure(N * sizeof(float4), s));
        GCVO_TRY(st->orig.ensure(N * sizeof(int), s));
        GCVO_TRY(st->cell_start.ensure((N + 1) * sizeof(int), s));
        GCVO_TRY(st->hkeys.ensure(H * sizeof(unsigned long long), s));
        GCVO_TRY(st->hval.ensure(H * sizeof(int), s));
    }
    GCVO_TRY(ctx->sort_keys.ensure(N * sizeof(unsigned long long), s));
    GCVO_TRY(ctx->sort_vals.ensure(N * sizeof(int) * 2 + 1024, s));
    GCVO_TRY(ctx->sort_tmp.ensure(radix_sort_scratch_bytes(N), s));
    GCVO_TRY(ctx->scan_tmp.ensure(scan_scratch_bytes(N) + 1024, s));
    GCVO_TRY(ctx->status_word.ensure(256, s));
    GCVO_TRY(ctx->knn_retry.ensure(2 * N * sizeof(int) + 256, s));
    float4 *P = sa.ca.as<float4>();
    int *list1 = ctx->knn_retry.as<int>();
    int *list2 = list1 + N;
    unsigned *stw = ctx->status_word.as<unsigned>();
    // [0]: points left after the fine grid, [1]: after the middle grid,
    // [2]: work counter of the coarse pass
    int *n_list = reinterpret_cast<int *>(stw + 1);
    GCVO_CUDA(cudaMemcpyAsync(d_cl, cl.data(), C * sizeof(KnnCloud), cudaMemcpyHostToDevice, s));
    GCVO_CUDA(cudaMemcpyAsync(d_chunks, chunks.data(), chunks.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    GCVO_CUDA(cudaMemsetAsync(stw, 0, 4 * sizeof(unsigned), s));

    // gather, boxes, voxel sizes
    auto *hset = sb.hkeys.as<unsigned long long>();   // free until the middle grid is built
    const int sm = std::max(1, ctx->sm_count);
    const unsigned fill_blocks = (unsigned)std::min<unsigned long long>((H + 255) / 256, (unsigned long long)sm * 8);
    k_kc_init<<<fill_blocks, 256, 0, s>>>(d_box, C, hset, (int64_t)H);
    k_kc_gather<<<(unsigned)chunks.size(), 256, 0, s>>>(d_cl, d_chunks, P, d_box);
    k_kc_grid0<<<(unsigned)((C + 127) / 128), 128, 0, s>>>(d_cl, C, d_box, d_g[0]);
    const unsigned pt_blocks = (unsigned)std::min<int64_t>((N + 255) / 256, (int64_t)sm * 16);
    k_kc_occupancy<<<pt_blocks, 256, 0, s>>>(P, N, d_g[0], hset, H - 1, d_box);
    GridDev ta{}, tb{};
    for (int v = 0; v < 2; ++v) {
        GridStore &st = v ? sb : sa;
        GridDev &t = v ? tb : ta;
        t.pos = st.pos.as<float4>();
        t.orig = st.orig.as<int>();
        t.cell_start = st.cell_start.as<int>();
        t.hkeys = st.hkeys.as<unsigned long long>();
        t.hval = st.hval.as<int>();
        t.hmask = H - 1;
    }
    k_kc_setup<<<1, KC_SETUP_THREADS, 0, s>>>(d_cl, C, d_box, ta, tb, d_g[0], d_g[1], d_g[2], d_tot);
    count_launches(5);
    GCVO_CUDA(cudaGetLastError());
    unsigned long long tot[4];
    GCVO_CUDA(cudaMemcpyAsync(tot, d_tot, sizeof(tot), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    if (tot[3]) return GCVO_ERR_NONFINITE;

    // pass 1: every point on the fine grids, shells 1 and 2
    GCVO_TRY(kc_build(ctx, P, N, d_cl, d_g[0], tot[0], H, sa));
    k_knn_cov<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(d_g[0], d_cl, P, nullptr, nullptr, N, list1, n_list);
    count_launches(1);
    GCVO_CUDA(cudaGetLastError());
    int m1 = 0;
    GCVO_CUDA(cudaMemcpyAsync(&m1, n_list, sizeof(int), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    if (m1 == 0) return GCVO_OK;

    // pass 2: the points left, on the middle grids, shells 1 and 2
    GCVO_TRY(kc_build(ctx, P, N, d_cl, d_g[1], tot[1], H, sb));
    k_knn_cov<<<(unsigned)((m1 + 127) / 128), 128, 0, s>>>(d_g[1], d_cl, P, list1, n_list, N, list2, n_list + 1);
    count_launches(1);
    GCVO_CUDA(cudaGetLastError());
    int m2 = 0;
    GCVO_CUDA(cudaMemcpyAsync(&m2, n_list + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    if (m2 == 0) return GCVO_OK;

    // pass 3: the rest, one warp per point on the coarse grids, no shell limit
    GCVO_TRY(kc_build(ctx, P, N, d_cl, d_g[2], tot[2], H, sa));
    launch_knn_far(d_g[2], d_cl, P, list2, n_list + 1, n_list + 2, stw, sm, m2, s);
    count_launches(1);
    GCVO_CUDA(cudaGetLastError());
    unsigned hs = 0;
    GCVO_CUDA(cudaMemcpyAsync(&hs, stw, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    if (hs & DEV_ERR_CAPACITY) return GCVO_ERR_INVALID_ARG;
    return GCVO_OK;
}

}  // namespace

gcvo_status knn_covariances(gcvo_ctx *ctx, int n_clouds, const KnnJob *jobs) {
    if (n_clouds < 1 || !jobs) return GCVO_ERR_INVALID_ARG;
    // groups of at most KC_GROUP_CLOUDS clouds with at most KC_GROUP_POINTS
    // points together (the scans' capacity); a larger cloud forms a group of
    // its own
    int c0 = 0;
    while (c0 < n_clouds) {
        int c1 = c0 + 1;
        int64_t n = jobs[c0].n;
        while (c1 < n_clouds && c1 - c0 < KC_GROUP_CLOUDS && n + jobs[c1].n <= KC_GROUP_POINTS) n += jobs[c1++].n;
        GCVO_TRY(knn_cov_group(ctx, c1 - c0, jobs + c0));
        c0 = c1;
    }
    return GCVO_OK;
}

}  // namespace gcvo
