// Learned initial-pose proposal: a point-set network that maps a (source,
// target) pair of clouds to a twist, so that Algorithm 1 can start closer to
// the optimum.  (The paper has no counterpart; it is the learned-proposal
// extension of the registration path.)
//
//   per point p = ((xyz - c) / s, l) with c, s the target's centroid and RMS
//   radius:  h1 = relu(W1 p + b1) (64), h2 = relu(W2 h1 + b2) (128),
//            h3 = W3 h2 + b3 (256);  cloud feature = max over points of h3
//   u = [feat_src, feat_tgt] (512): z1 = relu(H1 u + c1) (256),
//            z2 = relu(H2 z1 + c2) (128), out = H3 z2 + c3 (6)
//   out is the twist (omega, v / s) of S T S^-1 with S the shift by -c.
//
// Weights are BF16 copies of FP32 master weights (Adam); every product
// accumulates in FP32.  The per-point layers 2 and 3 (the dense part: 82 k
// flop per point) run on the tensor cores with mma.sync m16n8k16 BF16; the
// max-pool is computed by one block per cloud, so the argmax (lowest point
// index on ties) is deterministic.  Backward uses that only each channel's
// argmax point receives gradient from the max-pool.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace gcvo {
namespace prop {

// parameter tensors, in the order of the flat parameter vector
enum { W1, B1, W2, B2, W3, B3, H1, C1, H2, C2, H3, C3, NT };
constexpr int ROWS[NT] = {64, 64, 128, 128, 256, 256, 256, 256, 128, 128, 6, 6};
constexpr int COLS[NT] = {4, 1, 64, 1, 128, 1, 512, 1, 256, 1, 128, 1};

struct Layout {
    int off[NT + 1];
    Layout() {
        off[0] = 0;
        for (int k = 0; k < NT; ++k) off[k + 1] = off[k] + ROWS[k] * COLS[k];
    }
    int n() const { return off[NT]; }
};

struct Net {
    const float *p;               // FP32 master (biases are read from here)
    const __nv_bfloat16 *w;       // BF16 copy, same layout
    int off[NT + 1];
};

constexpr int PT_WARPS = 4;       // per-point kernel: warps per block, 16 points each
constexpr int W2_LD = 64 + 8;     // padded rows in shared memory (bank spread)
constexpr int W3_LD = 128 + 8;

__device__ inline uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ inline void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// Normalisation: one block per pair.  Points of cloud 2b (source) and 2b+1
// (target) are written as float4 (x', y', z', l).
// ---------------------------------------------------------------------------
__global__ void k_prep(int n, const float *sx, const float *sf, int sf_stride, const float *tx, const float *tf,
                       int tf_stride, float4 *pts, float *cs) {
    const int b = blockIdx.x;
    const float *t = tx + (size_t)b * 3 * n;
    const float *s = sx + (size_t)b * 3 * n;
    __shared__ double red[4][256];
    double a0 = 0, a1 = 0, a2 = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a0 += t[i];
        a1 += t[n + i];
        a2 += t[2 * n + i];
    }
    red[0][threadIdx.x] = a0;
    red[1][threadIdx.x] = a1;
    red[2][threadIdx.x] = a2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    const double c0 = red[0][0] / n, c1 = red[1][0] / n, c2 = red[2][0] / n;
    __syncthreads();
    double r2 = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double d0 = t[i] - c0, d1 = t[n + i] - c1, d2 = t[2 * n + i] - c2;
        r2 += d0 * d0 + d1 * d1 + d2 * d2;
    }
    red[3][threadIdx.x] = r2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[3][threadIdx.x] += red[3][threadIdx.x + o];
        __syncthreads();
    }
    const double sc = sqrt(red[3][0] / n) + 1e-6;
    const float is = (float)(1.0 / sc);
    if (threadIdx.x == 0) {
        cs[4 * b + 0] = (float)c0;
        cs[4 * b + 1] = (float)c1;
        cs[4 * b + 2] = (float)c2;
        cs[4 * b + 3] = (float)sc;
    }
    const float f0 = (float)c0, f1 = (float)c1, f2 = (float)c2;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        pts[(size_t)(2 * b) * n + i] = make_float4((s[i] - f0) * is, (s[n + i] - f1) * is, (s[2 * n + i] - f2) * is,
                                                   sf[(size_t)b * sf_stride + i]);
        pts[(size_t)(2 * b + 1) * n + i] = make_float4((t[i] - f0) * is, (t[n + i] - f1) * is,
                                                       (t[2 * n + i] - f2) * is, tf[(size_t)b * tf_stride + i]);
    }
}

// ---------------------------------------------------------------------------
// Per-point MLP and max-pool: one block per cloud, each warp takes tiles of
// 16 points.  Layer 1 (4 -> 64) in FP32; layers 2 and 3 on the tensor cores,
// the output fragments of layer 2 (bias, relu, BF16) being the input
// fragments of layer 3.  feat[cloud][c] = max over points, arg[cloud][c] =
// the point (lowest index on ties).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PT_WARPS * 32) k_point_fwd(Net net, int n, const float4 *pts, float *feat,
                                                            int *arg) {
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16 *w2 = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *w3 = w2 + 128 * W2_LD;
    float *w1 = reinterpret_cast<float *>(w3 + 256 * W3_LD);
    float *b1 = w1 + 256;
    float *b2 = b1 + 64;
    float *b3 = b2 + 128;
    float *wmax = b3 + 256;              // [PT_WARPS][256]
    int *warg = reinterpret_cast<int *>(wmax + PT_WARPS * 256);

    const int cloud = blockIdx.x;
    for (int i = threadIdx.x; i < 128 * 64; i += blockDim.x) w2[(i / 64) * W2_LD + i % 64] = net.w[net.off[W2] + i];
    for (int i = threadIdx.x; i < 256 * 128; i += blockDim.x) w3[(i / 128) * W3_LD + i % 128] = net.w[net.off[W3] + i];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        w1[i] = __bfloat162float(net.w[net.off[W1] + i]);
        b3[i] = net.p[net.off[B3] + i];
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) b1[i] = net.p[net.off[B1] + i];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) b2[i] = net.p[net.off[B2] + i];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    float rmax[64];   // running max for this lane's channels: tile j (32), cols 2t, 2t+1
    int rarg[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) {
        rmax[k] = -INFINITY;
        rarg[k] = 0x7fffffff;
    }
    const float4 *P = pts + (size_t)cloud * n;
    for (int base = warp * 16; base < n; base += PT_WARPS * 16) {
        const int r0 = base + g, r1 = base + g + 8;
        const float4 p0 = P[min(r0, n - 1)], p1 = P[min(r1, n - 1)];
        const bool v0 = r0 < n, v1 = r1 < n;
        // layer 1 straight into the A fragments of layer 2 (K = 64)
        uint32_t a2[4][4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            float h[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int col = 16 * kk + 2 * t + (q & 1) + (q >> 1) * 8;
                const float *wr = w1 + 4 * col;
                h[2 * q] = fmaxf(wr[0] * p0.x + wr[1] * p0.y + wr[2] * p0.z + wr[3] * p0.w + b1[col], 0.f);
                h[2 * q + 1] = fmaxf(wr[0] * p1.x + wr[1] * p1.y + wr[2] * p1.z + wr[3] * p1.w + b1[col], 0.f);
            }
            // h[0,2]: row g cols 2t, 2t+1; h[1,3]: row g+8; h[4..7]: cols + 8
            a2[kk][0] = pack_bf16(h[0], h[2]);
            a2[kk][1] = pack_bf16(h[1], h[3]);
            a2[kk][2] = pack_bf16(h[4], h[6]);
            a2[kk][3] = pack_bf16(h[5], h[7]);
        }
        // layer 2 (64 -> 128): 16 n-tiles
        uint32_t a3[8][4];
#pragma unroll
        for (int jp = 0; jp < 8; ++jp) {
            float c[2][4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = 2 * jp + h;
                c[h][0] = c[h][1] = c[h][2] = c[h][3] = 0.f;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const __nv_bfloat16 *row = w2 + (8 * j + g) * W2_LD + 16 * kk + 2 * t;
                    mma16816(c[h], a2[kk], *reinterpret_cast<const uint32_t *>(row),
                             *reinterpret_cast<const uint32_t *>(row + 8));
                }
                const float bb0 = b2[8 * j + 2 * t], bb1 = b2[8 * j + 2 * t + 1];
                c[h][0] = fmaxf(c[h][0] + bb0, 0.f);
                c[h][1] = fmaxf(c[h][1] + bb1, 0.f);
                c[h][2] = fmaxf(c[h][2] + bb0, 0.f);
                c[h][3] = fmaxf(c[h][3] + bb1, 0.f);
            }
            a3[jp][0] = pack_bf16(c[0][0], c[0][1]);
            a3[jp][1] = pack_bf16(c[0][2], c[0][3]);
            a3[jp][2] = pack_bf16(c[1][0], c[1][1]);
            a3[jp][3] = pack_bf16(c[1][2], c[1][3]);
        }
        // layer 3 (128 -> 256): 32 n-tiles, running max over the points
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const __nv_bfloat16 *row = w3 + (8 * j + g) * W3_LD + 16 * kk + 2 * t;
                mma16816(c, a3[kk], *reinterpret_cast<const uint32_t *>(row),
                         *reinterpret_cast<const uint32_t *>(row + 8));
            }
            const float bb0 = b3[8 * j + 2 * t], bb1 = b3[8 * j + 2 * t + 1];
            const float x00 = v0 ? c[0] + bb0 : -INFINITY, x01 = v0 ? c[1] + bb1 : -INFINITY;
            const float x10 = v1 ? c[2] + bb0 : -INFINITY, x11 = v1 ? c[3] + bb1 : -INFINITY;
            // column 2t: rows r0, r1 (r0 < r1 keeps the lower index on ties)
            if (x00 > rmax[2 * j] || (x00 == rmax[2 * j] && r0 < rarg[2 * j])) {
                rmax[2 * j] = x00;
                rarg[2 * j] = r0;
            }
            if (x10 > rmax[2 * j] || (x10 == rmax[2 * j] && r1 < rarg[2 * j])) {
                rmax[2 * j] = x10;
                rarg[2 * j] = r1;
            }
            if (x01 > rmax[2 * j + 1] || (x01 == rmax[2 * j + 1] && r0 < rarg[2 * j + 1])) {
                rmax[2 * j + 1] = x01;
                rarg[2 * j + 1] = r0;
            }
            if (x11 > rmax[2 * j + 1] || (x11 == rmax[2 * j + 1] && r1 < rarg[2 * j + 1])) {
                rmax[2 * j + 1] = x11;
                rarg[2 * j + 1] = r1;
            }
        }
    }
    // reduce over the 8 lanes sharing t (the g bits), then over the warps
#pragma unroll
    for (int k = 0; k < 64; ++k) {
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
            float om = __shfl_xor_sync(0xffffffffu, rmax[k], o);
            int oa = __shfl_xor_sync(0xffffffffu, rarg[k], o);
            if (om > rmax[k] || (om == rmax[k] && oa < rarg[k])) {
                rmax[k] = om;
                rarg[k] = oa;
            }
        }
    }
    if (g == 0) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ch = 8 * j + 2 * t + h;
                wmax[warp * 256 + ch] = rmax[2 * j + h];
                warg[warp * 256 + ch] = rarg[2 * j + h];
            }
    }
    __syncthreads();
    for (int ch = threadIdx.x; ch < 256; ch += blockDim.x) {
        float m = wmax[ch];
        int a = warg[ch];
        for (int w = 1; w < PT_WARPS; ++w) {
            float om = wmax[w * 256 + ch];
            int oa = warg[w * 256 + ch];
            if (om > m || (om == m && oa < a)) {
                m = om;
                a = oa;
            }
        }
        feat[(size_t)cloud * 256 + ch] = m;
        arg[(size_t)cloud * 256 + ch] = a;
    }
}

size_t point_fwd_smem() {
    return (size_t)(128 * W2_LD + 256 * W3_LD) * 2 + (256 + 64 + 128 + 256) * 4 + PT_WARPS * 256 * 8;
}

// ---------------------------------------------------------------------------
// Head: one block (256 threads) per pair.  z1 = relu(H1 u + c1), z2 =
// relu(H2 z1 + c2), out = H3 z2 + c3; pre-activations y1, y2 kept for
// backward.
// ---------------------------------------------------------------------------
__global__ void k_head_fwd(Net net, const float *feat, float *y1, float *y2, float *out) {
    const int b = blockIdx.x;
    __shared__ float u[512], z1[256], z2[128];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        u[i] = feat[(size_t)(2 * b) * 256 + i];
        u[256 + i] = feat[(size_t)(2 * b + 1) * 256 + i];
    }
    __syncthreads();
    {
        const int o = threadIdx.x;   // 256 outputs
        const __nv_bfloat16 *w = net.w + net.off[H1] + (size_t)o * 512;
        float s = net.p[net.off[C1] + o];
        for (int i = 0; i < 512; i += 2) {
            float2 wf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(w + i));
            s += wf.x * u[i] + wf.y * u[i + 1];
        }
        y1[(size_t)b * 256 + o] = s;
        z1[o] = fmaxf(s, 0.f);
    }
    __syncthreads();
    if (threadIdx.x < 128) {
        const int o = threadIdx.x;
        const __nv_bfloat16 *w = net.w + net.off[H2] + (size_t)o * 256;
        float s = net.p[net.off[C2] + o];
        for (int i = 0; i < 256; i += 2) {
            float2 wf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(w + i));
            s += wf.x * z1[i] + wf.y * z1[i + 1];
        }
        y2[(size_t)b * 128 + o] = s;
        z2[o] = fmaxf(s, 0.f);
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int o = threadIdx.x;
        const __nv_bfloat16 *w = net.w + net.off[H3] + (size_t)o * 128;
        float s = net.p[net.off[C3] + o];
        for (int i = 0; i < 128; ++i) s += __bfloat162float(w[i]) * z2[i];
        out[(size_t)b * 6 + o] = s;
    }
}

// Per-pair backward through the head: deltas of every layer, and d feat.
__global__ void k_head_bwd(Net net, int B, const float *feat, const float *y1, const float *y2, const float *out,
                           const float *label, float *d_out, float *d_y1, float *d_y2, float *d_feat, float *loss) {
    const int b = blockIdx.x;
    __shared__ float dy2[128], dy1[256], sd_out[6];
    if (threadIdx.x < 6) {
        float d = out[(size_t)b * 6 + threadIdx.x] - label[(size_t)b * 6 + threadIdx.x];
        sd_out[threadIdx.x] = 2.0f * d / (float)B;
        d_out[(size_t)b * 6 + threadIdx.x] = 2.0f * d / (float)B;
        atomicAdd(loss, d * d / (float)B);
    }
    __syncthreads();
    if (threadIdx.x < 128) {
        const int i = threadIdx.x;
        float s = 0.f;
        for (int o = 0; o < 6; ++o) s += __bfloat162float(net.w[net.off[H3] + o * 128 + i]) * sd_out[o];
        float d = y2[(size_t)b * 128 + i] > 0.f ? s : 0.f;
        dy2[i] = d;
        d_y2[(size_t)b * 128 + i] = d;
    }
    __syncthreads();
    {
        const int i = threadIdx.x;   // 256
        float s = 0.f;
        for (int o = 0; o < 128; ++o) s += __bfloat162float(net.w[net.off[H2] + o * 256 + i]) * dy2[o];
        float d = y1[(size_t)b * 256 + i] > 0.f ? s : 0.f;
        dy1[i] = d;
        d_y1[(size_t)b * 256 + i] = d;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 512; i += blockDim.x) {
        float s = 0.f;
        for (int o = 0; o < 256; ++o) s += __bfloat162float(net.w[net.off[H1] + o * 512 + i]) * dy1[o];
        // d feat of cloud 2b (i < 256) or 2b+1
        d_feat[(size_t)(2 * b) * 256 + i] = s;
    }
}

// Head weight gradients: one thread per weight, summed over the batch in
// order (deterministic).  dW[o][i] = sum_b delta[b][o] * x[b][i].
__global__ void k_outer_sum(int B, int rows, int cols, const float *delta, int dstride, const float *x, int xstride,
                            int xrelu_from_pre, float *dW, float *db) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < rows * cols) {
        const int o = idx / cols, i = idx % cols;
        float s = 0.f;
        for (int b = 0; b < B; ++b) {
            float xv = x[(size_t)b * xstride + i];
            if (xrelu_from_pre) xv = fmaxf(xv, 0.f);
            s += delta[(size_t)b * dstride + o] * xv;
        }
        dW[idx] += s;
    }
    if (db && idx < rows) {
        float s = 0.f;
        for (int b = 0; b < B; ++b) s += delta[(size_t)b * dstride + idx];
        db[idx] += s;
    }
}

// ---------------------------------------------------------------------------
// Per-point backward: one block (128 threads) per cloud.  For every channel
// c with a gradient g_c, its argmax point p gets d h3[p][c] = g_c; the block
// recomputes h1, h2 of p as the forward did (BF16 inputs to layers 2 and 3),
// and accumulates dW3[c] += g_c h2, dW2 += d2 h1^T with d2 = g_c W3[c] *
// relu'(a2), dW1 += d1 p^T with d1 = (W2^T d2) * relu'(a1) (and the biases).
// Layers 1 and 2 are summed over the block's channels in shared memory first.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_point_bwd(Net net, int n, const float4 *pts, const int *arg,
                                                   const float *d_feat, float *grad) {
    const int cloud = blockIdx.x;
    __shared__ float sW2[128 * 64];   // dW2 partial
    __shared__ float sB2[128], sW1[64 * 4], sB1[64];
    __shared__ float h1[64], a1[64], h2[128], a2[128], d2[128];
    __shared__ float pv[4];
    for (int i = threadIdx.x; i < 128 * 64; i += blockDim.x) sW2[i] = 0.f;
    for (int i = threadIdx.x; i < 128; i += blockDim.x) sB2[i] = 0.f;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sW1[i] = 0.f;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) sB1[i] = 0.f;
    int last_p = -1;
    __syncthreads();
    for (int c = 0; c < 256; ++c) {
        const float gc = d_feat[(size_t)cloud * 256 + c];
        if (gc == 0.f) continue;
        const int p = arg[(size_t)cloud * 256 + c];
        if (p != last_p) {
            if (threadIdx.x == 0) {
                float4 q = pts[(size_t)cloud * n + p];
                pv[0] = q.x;
                pv[1] = q.y;
                pv[2] = q.z;
                pv[3] = q.w;
            }
            __syncthreads();
            if (threadIdx.x < 64) {
                const int o = threadIdx.x;
                float s = net.p[net.off[B1] + o];
                for (int i = 0; i < 4; ++i) s += __bfloat162float(net.w[net.off[W1] + o * 4 + i]) * pv[i];
                a1[o] = s;
                h1[o] = __bfloat162float(__float2bfloat16_rn(fmaxf(s, 0.f)));
            }
            __syncthreads();
            {
                const int o = threadIdx.x;   // 128
                float s = 0.f;
                for (int i = 0; i < 64; ++i) s += __bfloat162float(net.w[net.off[W2] + o * 64 + i]) * h1[i];
                s += net.p[net.off[B2] + o];
                a2[o] = s;
                h2[o] = __bfloat162float(__float2bfloat16_rn(fmaxf(s, 0.f)));
            }
            __syncthreads();
            last_p = p;
        }
        {
            const int o = threadIdx.x;
            atomicAdd(grad + net.off[W3] + c * 128 + o, gc * h2[o]);
            if (o == 0) atomicAdd(grad + net.off[B3] + c, gc);
            float d = a2[o] > 0.f ? gc * __bfloat162float(net.w[net.off[W3] + c * 128 + o]) : 0.f;
            d2[o] = d;
            sB2[o] += d;
            for (int i = 0; i < 64; ++i) sW2[o * 64 + i] += d * h1[i];
        }
        __syncthreads();
        if (threadIdx.x < 64) {
            const int i = threadIdx.x;
            float s = 0.f;
            for (int o = 0; o < 128; ++o) s += __bfloat162float(net.w[net.off[W2] + o * 64 + i]) * d2[o];
            const float d1 = a1[i] > 0.f ? s : 0.f;
            sB1[i] += d1;
            for (int k = 0; k < 4; ++k) sW1[i * 4 + k] += d1 * pv[k];
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < 128 * 64; i += blockDim.x) atomicAdd(grad + net.off[W2] + i, sW2[i]);
    for (int i = threadIdx.x; i < 128; i += blockDim.x) atomicAdd(grad + net.off[B2] + i, sB2[i]);
    for (int i = threadIdx.x; i < 256; i += blockDim.x) atomicAdd(grad + net.off[W1] + i, sW1[i]);
    for (int i = threadIdx.x; i < 64; i += blockDim.x) atomicAdd(grad + net.off[B1] + i, sB1[i]);
}

// Adam (Kingma & Ba) on the FP32 master weights; refreshes the BF16 copy.
__global__ void k_adam(int n, float *p, const float *g, float *m, float *v, __nv_bfloat16 *w, float lr, float b1,
                       float b2, float eps, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    p[i] = pi;
    w[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(int n, const float *p, __nv_bfloat16 *w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = __float2bfloat16_rn(p[i]);
}

}  // namespace prop
}  // namespace gcvo

// ---------------------------------------------------------------------------
// SE(3) helpers for the label / proposal conversion (host, double).
// ---------------------------------------------------------------------------
namespace {

void se3_exp(const double xi[6], double T[16]) {
    const double *w = xi, *v = xi + 3;
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2], th = std::sqrt(th2);
    double A, B, C;
    if (th < 1e-4) {
        A = 1 - th2 / 6 + th2 * th2 / 120;
        B = 0.5 - th2 / 24 + th2 * th2 / 720;
        C = 1.0 / 6 - th2 / 120 + th2 * th2 / 5040;
    } else {
        A = std::sin(th) / th;
        B = (1 - std::cos(th)) / th2;
        C = (th - std::sin(th)) / (th2 * th);
    }
    double W[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0}, W2[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) W2[3 * r + c] = W[3 * r] * W[c] + W[3 * r + 1] * W[3 + c] + W[3 * r + 2] * W[6 + c];
    for (int r = 0; r < 3; ++r) {
        double tr = 0;
        for (int c = 0; c < 3; ++c) {
            double I = r == c ? 1.0 : 0.0;
            T[4 * r + c] = I + A * W[3 * r + c] + B * W2[3 * r + c];
            tr += (I + B * W[3 * r + c] + C * W2[3 * r + c]) * v[c];
        }
        T[4 * r + 3] = tr;
    }
    T[12] = T[13] = T[14] = 0;
    T[15] = 1;
}

// log of a rigid transform: rotation vector from the skew part of R (with
// the symmetric part near pi), translation through the inverse V matrix.
void se3_log(const double T[16], double xi[6]) {
    const double R[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
    double cth = std::min(1.0, std::max(-1.0, (R[0] + R[4] + R[8] - 1.0) / 2.0));
    double th = std::acos(cth);
    double w[3];
    if (th < 1e-6) {
        w[0] = (R[7] - R[5]) / 2;
        w[1] = (R[2] - R[6]) / 2;
        w[2] = (R[3] - R[1]) / 2;
    } else if (M_PI - th < 1e-4) {
        // axis from the diagonal of (R + I) / 2 = n n^T
        double d[3] = {std::sqrt(std::max(0.0, (R[0] + 1) / 2)), std::sqrt(std::max(0.0, (R[4] + 1) / 2)),
                       std::sqrt(std::max(0.0, (R[8] + 1) / 2))};
        int k = d[0] >= d[1] && d[0] >= d[2] ? 0 : (d[1] >= d[2] ? 1 : 2);
        double nrm[3];
        nrm[k] = d[k];
        for (int j = 0; j < 3; ++j)
            if (j != k) nrm[j] = (R[3 * k + j] + R[3 * j + k]) / (4 * d[k]);
        double s = 1.0 / std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
        for (int j = 0; j < 3; ++j) w[j] = nrm[j] * s * th;
    } else {
        double f = th / (2 * std::sin(th));
        w[0] = (R[7] - R[5]) * f;
        w[1] = (R[2] - R[6]) * f;
        w[2] = (R[3] - R[1]) * f;
    }
    // V^-1 t = (I - 1/2 W + (1/th^2)(1 - A / (2B)) W^2) t
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    th = std::sqrt(th2);
    double D;
    if (th < 1e-4) D = 1.0 / 12 + th2 / 720;
    else {
        double A = std::sin(th) / th, B = (1 - std::cos(th)) / th2;
        D = (1 - A / (2 * B)) / th2;
    }
    double W[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0}, W2[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) W2[3 * r + c] = W[3 * r] * W[c] + W[3 * r + 1] * W[3 + c] + W[3 * r + 2] * W[6 + c];
    const double t[3] = {T[3], T[7], T[11]};
    for (int r = 0; r < 3; ++r) {
        double s = 0;
        for (int c = 0; c < 3; ++c) s += ((r == c ? 1.0 : 0.0) - 0.5 * W[3 * r + c] + D * W2[3 * r + c]) * t[c];
        xi[3 + r] = s;
    }
    for (int k = 0; k < 3; ++k) xi[k] = w[k];
}

}  // namespace

using namespace gcvo;

struct gcvo_proposal {
    int device = 0;
    prop::Layout L;
    DevBuf p, g, m, v, w;                // master, grad, Adam moments, BF16 copy
    DevBuf pts, cs, feat, arg, y1, y2, out, label, d_out, d_y1, d_y2, d_feat, loss;
    int step = 0;
    int cap_pairs = 0, cap_points = 0;
};

namespace {

prop::Net net_of(gcvo_proposal *P) {
    prop::Net n;
    n.p = P->p.as<float>();
    n.w = P->w.as<__nv_bfloat16>();
    for (int k = 0; k <= prop::NT; ++k) n.off[k] = P->L.off[k];
    return n;
}

gcvo_status ensure_batch(gcvo_ctx *ctx, gcvo_proposal *P, int B, int n) {
    cudaStream_t s = ctx->stream;
    GCVO_TRY(P->pts.ensure((size_t)2 * B * n * sizeof(float4), s));
    GCVO_TRY(P->cs.ensure((size_t)B * 4 * sizeof(float), s));
    GCVO_TRY(P->feat.ensure((size_t)2 * B * 256 * sizeof(float), s));
    GCVO_TRY(P->arg.ensure((size_t)2 * B * 256 * sizeof(int), s));
    GCVO_TRY(P->y1.ensure((size_t)B * 256 * sizeof(float), s));
    GCVO_TRY(P->y2.ensure((size_t)B * 128 * sizeof(float), s));
    GCVO_TRY(P->out.ensure((size_t)B * 6 * sizeof(float), s));
    GCVO_TRY(P->label.ensure((size_t)B * 6 * sizeof(float), s));
    GCVO_TRY(P->d_out.ensure((size_t)B * 6 * sizeof(float), s));
    GCVO_TRY(P->d_y1.ensure((size_t)B * 256 * sizeof(float), s));
    GCVO_TRY(P->d_y2.ensure((size_t)B * 128 * sizeof(float), s));
    GCVO_TRY(P->d_feat.ensure((size_t)2 * B * 256 * sizeof(float), s));
    GCVO_TRY(P->loss.ensure(256, s));
    return GCVO_OK;
}

// Normalisation and the forward pass of a batch; leaves out, feat, arg, y1,
// y2 on the device.
gcvo_status forward_batch(gcvo_ctx *ctx, gcvo_proposal *P, int B, int n, const float *sx, const float *sf, int sfs,
                          const float *tx, const float *tf, int tfs) {
    cudaStream_t s = ctx->stream;
    GCVO_TRY(ensure_batch(ctx, P, B, n));
    prop::k_prep<<<B, 256, 0, s>>>(n, sx, sf, sfs, tx, tf, tfs, P->pts.as<float4>(), P->cs.as<float>());
    static bool attr = false;
    if (!attr) {
        GCVO_CUDA(cudaFuncSetAttribute(prop::k_point_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)prop::point_fwd_smem()));
        attr = true;
    }
    prop::Net net = net_of(P);
    prop::k_point_fwd<<<2 * B, prop::PT_WARPS * 32, prop::point_fwd_smem(), s>>>(
        net, n, P->pts.as<float4>(), P->feat.as<float>(), P->arg.as<int>());
    prop::k_head_fwd<<<B, 256, 0, s>>>(net, P->feat.as<float>(), P->y1.as<float>(), P->y2.as<float>(),
                                      P->out.as<float>());
    count_launches(3);
    GCVO_CUDA(cudaGetLastError());
    return GCVO_OK;
}

bool valid_batch(int B, int n) { return B >= 1 && B <= 65535 && n >= 1 && n <= (1 << 24); }

}  // namespace

extern "C" {

gcvo_status gcvo_proposal_create(gcvo_ctx *ctx, gcvo_proposal **out) {
    if (!ctx || !out) return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    gcvo_proposal *P = new (std::nothrow) gcvo_proposal();
    if (!P) return GCVO_ERR_WORKSPACE;
    P->device = ctx->device;
    const size_t n = P->L.n();
    cudaStream_t s = ctx->stream;
    gcvo_status st = GCVO_OK;
    for (DevBuf *b : {&P->p, &P->g, &P->m, &P->v})
        if (st == GCVO_OK) st = b->ensure(n * sizeof(float), s);
    if (st == GCVO_OK) st = P->w.ensure(n * sizeof(__nv_bfloat16), s);
    if (st == GCVO_OK) {
        for (DevBuf *b : {&P->p, &P->g, &P->m, &P->v, &P->w})
            if (cudaMemsetAsync(b->ptr, 0, b->bytes, s) != cudaSuccess) st = GCVO_ERR_CUDA;
    }
    if (st != GCVO_OK) {
        gcvo_proposal_destroy(P);
        return st;
    }
    *out = P;
    return GCVO_OK;
}

gcvo_status gcvo_proposal_destroy(gcvo_proposal *P) {
    if (!P) return GCVO_ERR_INVALID_ARG;
    cudaSetDevice(P->device);
    for (DevBuf *b : {&P->p, &P->g, &P->m, &P->v, &P->w, &P->pts, &P->cs, &P->feat, &P->arg, &P->y1, &P->y2,
                      &P->out, &P->label, &P->d_out, &P->d_y1, &P->d_y2, &P->d_feat, &P->loss})
        b->release();
    delete P;
    return GCVO_OK;
}

int64_t gcvo_proposal_n_params(void) { return prop::Layout().n(); }

gcvo_status gcvo_proposal_set_params(gcvo_ctx *ctx, gcvo_proposal *P, const float *params) {
    if (!ctx || !P || !params) return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    const int n = P->L.n();
    cudaStream_t s = ctx->stream;
    GCVO_CUDA(cudaMemcpyAsync(P->p.ptr, params, n * sizeof(float), cudaMemcpyDefault, s));
    GCVO_CUDA(cudaMemsetAsync(P->m.ptr, 0, n * sizeof(float), s));
    GCVO_CUDA(cudaMemsetAsync(P->v.ptr, 0, n * sizeof(float), s));
    prop::k_to_bf16<<<(n + 255) / 256, 256, 0, s>>>(n, P->p.as<float>(), P->w.as<__nv_bfloat16>());
    count_launches(1);
    GCVO_CUDA(cudaGetLastError());
    GCVO_CUDA(cudaStreamSynchronize(s));
    P->step = 0;
    return GCVO_OK;
}

gcvo_status gcvo_proposal_get_params(gcvo_ctx *ctx, const gcvo_proposal *P, float *params_out) {
    if (!ctx || !P || !params_out) return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    GCVO_CUDA(cudaMemcpyAsync(params_out, P->p.ptr, P->L.n() * sizeof(float), cudaMemcpyDefault, ctx->stream));
    GCVO_CUDA(cudaStreamSynchronize(ctx->stream));
    return GCVO_OK;
}

gcvo_status gcvo_proposal_get_state(gcvo_ctx *ctx, const gcvo_proposal *P, float *state_out, int64_t *step_out) {
    if (!ctx || !P || !state_out || !step_out) return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    const size_t n = (size_t)P->L.n();
    const DevBuf *parts[3] = {&P->p, &P->m, &P->v};
    for (int k = 0; k < 3; ++k)
        GCVO_CUDA(cudaMemcpyAsync(state_out + k * n, parts[k]->ptr, n * sizeof(float), cudaMemcpyDefault,
                                  ctx->stream));
    GCVO_CUDA(cudaStreamSynchronize(ctx->stream));
    *step_out = P->step;
    return GCVO_OK;
}

gcvo_status gcvo_proposal_set_state(gcvo_ctx *ctx, gcvo_proposal *P, const float *state, int64_t step) {
    if (!ctx || !P || !state || step < 0 || step > (int64_t)1 << 30) return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    const size_t n = (size_t)P->L.n();
    cudaStream_t s = ctx->stream;
    DevBuf *parts[3] = {&P->p, &P->m, &P->v};
    for (int k = 0; k < 3; ++k)
        GCVO_CUDA(cudaMemcpyAsync(parts[k]->ptr, state + k * n, n * sizeof(float), cudaMemcpyDefault, s));
    prop::k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((int)n, P->p.as<float>(), P->w.as<__nv_bfloat16>());
    count_launches(1);
    GCVO_CUDA(cudaGetLastError());
    GCVO_CUDA(cudaStreamSynchronize(s));
    P->step = (int)step;
    return GCVO_OK;
}

gcvo_status gcvo_proposal_infer(gcvo_ctx *ctx, gcvo_proposal *P, int B, int n, const float *src_xyz,
                                const float *src_feat, int src_feat_stride, const float *tgt_xyz,
                                const float *tgt_feat, int tgt_feat_stride, float *twist_out, double *T0_out) {
    if (!ctx || !P || !src_xyz || !src_feat || !tgt_xyz || !tgt_feat || !valid_batch(B, n)) return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    GCVO_TRY(forward_batch(ctx, P, B, n, src_xyz, src_feat, src_feat_stride, tgt_xyz, tgt_feat, tgt_feat_stride));
    std::vector<float> out((size_t)B * 6), cs((size_t)B * 4);
    GCVO_CUDA(cudaMemcpyAsync(out.data(), P->out.ptr, out.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    GCVO_CUDA(cudaMemcpyAsync(cs.data(), P->cs.ptr, cs.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    GCVO_CUDA(cudaStreamSynchronize(ctx->stream));
    if (twist_out) memcpy(twist_out, out.data(), out.size() * 4);
    if (T0_out) {
        for (int b = 0; b < B; ++b) {
            // xi = (omega, v s) in the centred frame; T = S^-1 exp(xi) S
            double xi[6], Tc[16];
            const double sc = cs[4 * b + 3];
            for (int k = 0; k < 3; ++k) {
                xi[k] = out[6 * b + k];
                xi[3 + k] = out[6 * b + 3 + k] * sc;
            }
            se3_exp(xi, Tc);
            double *T = T0_out + 16 * b;
            memcpy(T, Tc, sizeof(Tc));
            const double c[3] = {cs[4 * b], cs[4 * b + 1], cs[4 * b + 2]};
            for (int r = 0; r < 3; ++r)
                T[4 * r + 3] = Tc[4 * r + 3] + c[r] - (Tc[4 * r] * c[0] + Tc[4 * r + 1] * c[1] + Tc[4 * r + 2] * c[2]);
        }
    }
    return GCVO_OK;
}

gcvo_status gcvo_proposal_train_step(gcvo_ctx *ctx, gcvo_proposal *P, int B, int n, const float *src_xyz,
                                     const float *src_feat, int src_feat_stride, const float *tgt_xyz,
                                     const float *tgt_feat, int tgt_feat_stride, const double *T_label, float lr,
                                     float *loss_out, float *grad_out) {
    if (!ctx || !P || !src_xyz || !src_feat || !tgt_xyz || !tgt_feat || !T_label || !valid_batch(B, n) ||
        !(lr >= 0.f))
        return GCVO_ERR_INVALID_ARG;
    GCVO_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    GCVO_TRY(forward_batch(ctx, P, B, n, src_xyz, src_feat, src_feat_stride, tgt_xyz, tgt_feat, tgt_feat_stride));
    // labels: the twist of S T S^-1 (S the shift by -c), translation / s
    std::vector<float> cs((size_t)B * 4), lab((size_t)B * 6);
    GCVO_CUDA(cudaMemcpyAsync(cs.data(), P->cs.ptr, cs.size() * 4, cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < B; ++b) {
        const double *T = T_label + 16 * b;
        const double c[3] = {cs[4 * b], cs[4 * b + 1], cs[4 * b + 2]};
        double Tc[16];
        memcpy(Tc, T, sizeof(Tc));
        for (int r = 0; r < 3; ++r)
            Tc[4 * r + 3] = T[4 * r + 3] - c[r] + (T[4 * r] * c[0] + T[4 * r + 1] * c[1] + T[4 * r + 2] * c[2]);
        double xi[6];
        se3_log(Tc, xi);
        for (int k = 0; k < 3; ++k) {
            lab[6 * b + k] = (float)xi[k];
            lab[6 * b + 3 + k] = (float)(xi[3 + k] / cs[4 * b + 3]);
        }
    }
    GCVO_CUDA(cudaMemcpyAsync(P->label.ptr, lab.data(), lab.size() * 4, cudaMemcpyHostToDevice, s));
    const int np = P->L.n();
    GCVO_CUDA(cudaMemsetAsync(P->g.ptr, 0, np * sizeof(float), s));
    GCVO_CUDA(cudaMemsetAsync(P->loss.ptr, 0, sizeof(float), s));
    prop::Net net = net_of(P);
    prop::k_head_bwd<<<B, 256, 0, s>>>(net, B, P->feat.as<float>(), P->y1.as<float>(), P->y2.as<float>(),
                                      P->out.as<float>(), P->label.as<float>(), P->d_out.as<float>(),
                                      P->d_y1.as<float>(), P->d_y2.as<float>(), P->d_feat.as<float>(),
                                      P->loss.as<float>());
    float *g = P->g.as<float>();
    const int *off = P->L.off;
    // dH1 = sum_b dy1 u^T (u = the pair's two features), dH2 = dy2 z1^T, dH3 = dout z2^T
    prop::k_outer_sum<<<(256 * 512 + 255) / 256, 256, 0, s>>>(B, 256, 512, P->d_y1.as<float>(), 256,
                                                             P->feat.as<float>(), 512, 0, g + off[prop::H1],
                                                             g + off[prop::C1]);
    prop::k_outer_sum<<<(128 * 256 + 255) / 256, 256, 0, s>>>(B, 128, 256, P->d_y2.as<float>(), 128,
                                                             P->y1.as<float>(), 256, 1, g + off[prop::H2],
                                                             g + off[prop::C2]);
    prop::k_outer_sum<<<(6 * 128 + 255) / 256, 256, 0, s>>>(B, 6, 128, P->d_out.as<float>(), 6, P->y2.as<float>(),
                                                           128, 1, g + off[prop::H3], g + off[prop::C3]);
    prop::k_point_bwd<<<2 * B, 128, 0, s>>>(net, n, P->pts.as<float4>(), P->arg.as<int>(), P->d_feat.as<float>(), g);
    count_launches(5);
    GCVO_CUDA(cudaGetLastError());
    if (grad_out) {
        GCVO_CUDA(cudaMemcpyAsync(grad_out, g, np * sizeof(float), cudaMemcpyDeviceToHost, s));
    }
    if (lr > 0.f) {
        P->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float bc1 = 1.f - std::pow(b1, (float)P->step), bc2 = 1.f - std::pow(b2, (float)P->step);
        prop::k_adam<<<(np + 255) / 256, 256, 0, s>>>(np, P->p.as<float>(), g, P->m.as<float>(), P->v.as<float>(),
                                                     P->w.as<__nv_bfloat16>(), lr, b1, b2, 1e-8f, bc1, bc2);
        count_launches(1);
        GCVO_CUDA(cudaGetLastError());
    }
    float L = 0.f;
    GCVO_CUDA(cudaMemcpyAsync(&L, P->loss.ptr, sizeof(float), cudaMemcpyDeviceToHost, s));
    GCVO_CUDA(cudaStreamSynchronize(s));
    if (loss_out) *loss_out = L;
    return GCVO_OK;
}

}  // extern "C"
