// Pass 3 of the kNN covariances: the points whose neighbours lie beyond the
// fine and middle grids' two shells (a separate translation unit so that it
// compiles in parallel with grid.cu).
#include <algorithm>

#include "common.cuh"
#include "knn.cuh"

namespace gcvo {
namespace {

using namespace knn;

// Pass 3: one warp per queued point, searching its cloud's coarse grid shell
// by shell without a limit.  The lanes split each shell's voxels and keep
// private sorted lists; after every shell the warp merges them (repeated
// warp-wide minimum over each lane's next entry) into the knn nearest so
// far, and stops once the knn-th distance is within the shells' reach.
// The searches differ in length by orders of magnitude (one shell or
// dozens), so each warp takes its next point from a counter as it finishes.
__global__ void k_knn_cov_far(const GridDev *gcs, const KnnCloud *cl, const float4 *P, const int *list,
                              const int *n_list, int *next, unsigned *status) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int m = *n_list;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(next, 1);
        t = __shfl_sync(FULL, t, 0);
        if (t >= m) break;
        const int j = list[t];
        const float4 q = P[j];
        const int cloud = cloud_of(q);
        const GridDev &coarse = gcs[cloud];
        const KnnCloud &kc = cl[cloud];
        const int knn = kc.knn;
        const int maxR = max(coarse.dims[0], max(coarse.dims[1], coarse.dims[2]));
        int cq[3];
        {
            float qc[3] = {q.x, q.y, q.z};
            for (int a = 0; a < 3; ++a) {
                int c = (int)floorf((qc[a] - coarse.corner[a]) * coarse.inv_h);
                cq[a] = min(max(c, 0), coarse.dims[a] - 1);
            }
        }
        KnnList L;   // this lane's private list
#pragma unroll
        for (int k = 0; k < KNN_MAX; ++k) {
            L.d[k] = INFINITY;
            L.i[k] = 0x7fffffff;
            L.k[k] = -1;
        }
        float wd = INFINITY;
        int wi = 0x7fffffff;
        KnnList M;   // merged result (identical in every lane)
        bool done = false;
        for (int R = 1; R <= maxR && !done; ++R) {
            const int side = 2 * R + 1;
            const int cube = side * side * side;
            for (int v = lane; v < cube; v += 32) {
                int dx = v / (side * side) - R, dy = (v / side) % side - R, dz = v % side - R;
                if (R > 1 && max(abs(dx), max(abs(dy), abs(dz))) != R) continue;   // shell only
                int cx = cq[0] + dx, cy = cq[1] + dy, cz = cq[2] + dz;
                if (cx < 0 || cy < 0 || cz < 0 || cx >= coarse.dims[0] || cy >= coarse.dims[1] ||
                    cz >= coarse.dims[2])
                    continue;
                unsigned long long key =
                    coarse.key_base + ((unsigned long long)cx * coarse.dims[1] + cy) * coarse.dims[2] + cz;
                int c = grid_lookup(coarse, key);
                if (c < 0) continue;
                for (int k = coarse.cell_start[c], k1 = coarse.cell_start[c + 1]; k < k1; ++k) {
                    float4 y = coarse.pos[k];
                    float ex = y.x - q.x, ey = y.y - q.y, ez = y.z - q.z;
                    float d2 = ex * ex + ey * ey + ez * ez;
                    if (d2 > wd) continue;
                    int oi = coarse.orig[k];
                    if (d2 == wd && oi >= wi) continue;
                    float cd = d2;
                    int ci = oi, ck = k;
#pragma unroll
                    for (int mm = 0; mm < KNN_MAX; ++mm) {
                        if (mm < knn) {
                            bool less = cd < L.d[mm] || (cd == L.d[mm] && ci < L.i[mm]);
                            if (less) {
                                float td = L.d[mm];
                                int ti = L.i[mm], tk = L.k[mm];
                                L.d[mm] = cd;
                                L.i[mm] = ci;
                                L.k[mm] = ck;
                                cd = td;
                                ci = ti;
                                ck = tk;
                            }
                        }
                    }
#pragma unroll
                    for (int mm = 0; mm < KNN_MAX; ++mm)
                        if (mm == knn - 1) {
                            wd = L.d[mm];
                            wi = L.i[mm];
                        }
                }
            }
            // merge: knn rounds of a warp-wide minimum over (d, index)
            int head = 0;
            for (int r = 0; r < knn; ++r) {
                float hd = INFINITY;
                int hi = 0x7fffffff, hk = -1;
#pragma unroll
                for (int mm = 0; mm < KNN_MAX; ++mm)
                    if (mm == head) {
                        hd = L.d[mm];
                        hi = L.i[mm];
                        hk = L.k[mm];
                    }
                float bd = hd;
                int bi = hi;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    float od = __shfl_xor_sync(FULL, bd, o);
                    int oi = __shfl_xor_sync(FULL, bi, o);
                    if (od < bd || (od == bd && oi < bi)) {
                        bd = od;
                        bi = oi;
                    }
                }
                const bool mine = (hd == bd && hi == bi && hk >= 0);
                const unsigned who = __ballot_sync(FULL, mine);
                const int src = who ? __ffs(who) - 1 : 0;
                const int bk = __shfl_sync(FULL, hk, src);
                if (lane == src && who) ++head;
#pragma unroll
                for (int mm = 0; mm < KNN_MAX; ++mm)
                    if (mm == r) {
                        M.d[mm] = who ? bd : INFINITY;
                        M.i[mm] = who ? bi : 0x7fffffff;
                        M.k[mm] = who ? bk : -1;
                    }
            }
            // every lane prunes with the merged knn-th distance from now on
            float md = INFINITY;
            int mi = 0x7fffffff, mk = -1;
#pragma unroll
            for (int mm = 0; mm < KNN_MAX; ++mm)
                if (mm == knn - 1) {
                    md = M.d[mm];
                    mi = M.i[mm];
                    mk = M.k[mm];
                }
            if (mk >= 0 && (md < wd || (md == wd && mi < wi))) {
                wd = md;
                wi = mi;
            }
            const float reach = (float)R * coarse.h;
            done = mk >= 0 && md <= reach * reach * 0.999f;
        }
        bool full = true;
#pragma unroll
        for (int mm = 0; mm < KNN_MAX; ++mm)
            if (mm < knn && M.k[mm] < 0) full = false;
        if (!full) {
            if (lane == 0) atomicOr(status, DEV_ERR_CAPACITY);
            continue;
        }
        if (lane == 0) knn_write_cov<false>(coarse, q, M, knn, kc.eig_max, kc.eig_ratio, kc.n, (int)(j - kc.off), kc.cov);
    }
}

}  // namespace

// One resident wave: as many blocks of 4 warps as fit on the GPU, at most
// one warp per queued point (m_max).  next: zeroed work counter.
void launch_knn_far(const GridDev *gc, const KnnCloud *cl, const float4 *P, const int *list, const int *n_list,
                    int *next, unsigned *status, int sm_count, int64_t m_max, cudaStream_t s) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_knn_cov_far, 128, 0) != cudaSuccess || b < 1) b = 1;
        per_sm = b;
    }
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((m_max + 3) / 4, (int64_t)per_sm * sm_count));
    k_knn_cov_far<<<(unsigned)blocks, 128, 0, s>>>(gc, cl, P, list, n_list, next, status);
}

}  // namespace gcvo
