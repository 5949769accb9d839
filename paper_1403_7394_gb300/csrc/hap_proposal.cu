// Learned candidate proposal: exact k nearest neighbours, kNN-distance
// features, a 3-layer MLP (width 128, BF16 weights, FP32 accumulation) with
// forward, backward and Adam kernels, and per-row candidate selection.
//
// None of this is in the paper (§2 is dense); it prunes each row of HAP to K
// candidate exemplars so that large N needs N*K instead of N^2 messages.
// Reductions are in fixed order (per-CTA partials summed in CTA order), so
// training is bitwise reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <vector>

#include "hap.h"
#include "hap_common.cuh"
#include "hap_internal.h"

namespace hap {
namespace {

// ---------------------------------------------------------------------------
// exact kNN: one thread per query row, candidates streamed through shared
// memory in tiles, a stable sorted top-M list per row in shared memory
// ---------------------------------------------------------------------------
constexpr int KNN_ROWS = 128;
constexpr int KNN_TILE = 64;
constexpr int KNN_MAXM = 128;

template <int D>  // padded dimension, the query vector lives in registers
__global__ void __launch_bounds__(KNN_ROWS) knn_kernel(const float* __restrict__ Q, int Nq, const float* __restrict__ C,
                                                       const int32_t* __restrict__ cid, int Nc, int d, int M,
                                                       int32_t* __restrict__ out_idx, float* __restrict__ out_dist) {
    // queries are points 0..Nq-1; candidate j has global id cid[j] (j if cid
    // is NULL); a query never takes itself
    extern __shared__ __align__(16) float ksm[];
    float* ct = ksm;                                      // [KNN_TILE][D]
    float* tdist = ct + KNN_TILE * D;                     // [M][KNN_ROWS]
    int* tidx = reinterpret_cast<int*>(tdist + M * KNN_ROWS);
    const int t = threadIdx.x;
    const int i = blockIdx.x * KNN_ROWS + t;
    const bool valid = i < Nq;
    float q[D];
#pragma unroll
    for (int k = 0; k < D; ++k) q[k] = (valid && k < d) ? Q[(int64_t)i * d + k] : 0.f;
    int cnt = 0;
    float thr = kInf;
    auto insert = [&](float dv, int j) {
        int p = cnt < M ? cnt : M - 1;
        if (cnt < M) ++cnt;
        while (p > 0 && tdist[(p - 1) * KNN_ROWS + t] > dv) {
            tdist[p * KNN_ROWS + t] = tdist[(p - 1) * KNN_ROWS + t];
            tidx[p * KNN_ROWS + t] = tidx[(p - 1) * KNN_ROWS + t];
            --p;
        }
        tdist[p * KNN_ROWS + t] = dv;
        tidx[p * KNN_ROWS + t] = j;
        thr = cnt == M ? tdist[(M - 1) * KNN_ROWS + t] : kInf;
    };
    for (int c0 = 0; c0 < Nc; c0 += KNN_TILE) {
        __syncthreads();
        for (int e = t; e < KNN_TILE * D; e += KNN_ROWS) {
            const int r = e / D, k = e - r * D, j = c0 + r;
            ct[e] = (j < Nc && k < d) ? C[(int64_t)j * d + k] : 0.f;
        }
        __syncthreads();
        if (!valid) continue;
        const int nc = min(KNN_TILE, Nc - c0);
        for (int r = 0; r < nc; r += 4) {  // four candidates in flight, 4 dimensions per load
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            const float4* c = reinterpret_cast<const float4*>(ct + r * D);
#pragma unroll
            for (int k4 = 0; k4 < D / 4; ++k4) {
                const float4 v0 = c[k4], v1 = c[D / 4 + k4], v2 = c[2 * (D / 4) + k4], v3 = c[3 * (D / 4) + k4];
                const float x0 = q[4 * k4], x1 = q[4 * k4 + 1], x2 = q[4 * k4 + 2], x3 = q[4 * k4 + 3];
                float e;
                e = x0 - v0.x; a0 = fmaf(e, e, a0); e = x1 - v0.y; a0 = fmaf(e, e, a0);
                e = x2 - v0.z; a0 = fmaf(e, e, a0); e = x3 - v0.w; a0 = fmaf(e, e, a0);
                e = x0 - v1.x; a1 = fmaf(e, e, a1); e = x1 - v1.y; a1 = fmaf(e, e, a1);
                e = x2 - v1.z; a1 = fmaf(e, e, a1); e = x3 - v1.w; a1 = fmaf(e, e, a1);
                e = x0 - v2.x; a2 = fmaf(e, e, a2); e = x1 - v2.y; a2 = fmaf(e, e, a2);
                e = x2 - v2.z; a2 = fmaf(e, e, a2); e = x3 - v2.w; a2 = fmaf(e, e, a2);
                e = x0 - v3.x; a3 = fmaf(e, e, a3); e = x1 - v3.y; a3 = fmaf(e, e, a3);
                e = x2 - v3.z; a3 = fmaf(e, e, a3); e = x3 - v3.w; a3 = fmaf(e, e, a3);
            }
            const float dv[4] = {a0, a1, a2, a3};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (r + u >= nc) continue;
                const int j = cid ? cid[c0 + r + u] : c0 + r + u;
                if (j != i && (cnt < M || dv[u] < thr)) insert(dv[u], j);
            }
        }
    }
    if (valid)
        for (int m = 0; m < M; ++m) {
            out_idx[(int64_t)i * M + m] = m < cnt ? tidx[m * KNN_ROWS + t] : -1;
            out_dist[(int64_t)i * M + m] = m < cnt ? tdist[m * KNN_ROWS + t] : kInf;
        }
}

__global__ void gather_rows_kernel(const float* __restrict__ X, int64_t d, const int32_t* __restrict__ rows,
                                   float* __restrict__ out) {
    const int64_t r = blockIdx.x;
    const int64_t src = rows[r];
    for (int64_t k = threadIdx.x; k < d; k += blockDim.x) out[r * d + k] = X[src * d + k];
}

// ---------------------------------------------------------------------------
// top-H scores (hubs): bitonic sort of (descending score, ascending index)
// keys packed in 64 bits, padded to a power of two with keys that sort last
// ---------------------------------------------------------------------------
__global__ void hub_keys_kernel(const float* __restrict__ score, int N, int n2, uint64_t* __restrict__ keys) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2) return;
    if (i >= N) { keys[i] = ~0ull; return; }
    // larger score -> smaller key: order-preserving bits of -score
    uint32_t b = __float_as_uint(-score[i]);
    b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    keys[i] = ((uint64_t)b << 32) | (uint32_t)i;
}
__global__ void bitonic_step_kernel(uint64_t* __restrict__ keys, int n2, int j, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2) return;
    const int p = i ^ j;
    if (p > i) {
        const uint64_t a = keys[i], b = keys[p];
        const bool up = (i & k) == 0;
        if ((a > b) == up) { keys[i] = b; keys[p] = a; }
    }
}
__global__ void hub_ids_kernel(const uint64_t* __restrict__ keys, int H, int32_t* __restrict__ hubs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < H) hubs[i] = (int32_t)(keys[i] & 0xffffffffu);
}

// candidates: self, the K_near nearest, then the nearest hubs not yet taken
// (pool entries beyond K_near fill any remainder); sorted by index
__global__ void select_hub_candidates_kernel(const int32_t* __restrict__ pool, int Mp, const int32_t* __restrict__ hubnn,
                                             int Mh, int N, int K, int K_near, int32_t* __restrict__ cand) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int sel[64];
    int ns = 0;
    sel[ns++] = i;
    const int32_t* pi = pool + (int64_t)i * Mp;
    const int32_t* hi = hubnn + (int64_t)i * Mh;
    auto taken = [&](int v) {
        for (int a = 0; a < ns; ++a)
            if (sel[a] == v) return true;
        return false;
    };
    for (int q = 0; q < K_near && ns < K; ++q)
        if (pi[q] >= 0 && !taken(pi[q])) sel[ns++] = pi[q];
    for (int q = 0; q < Mh && ns < K; ++q)
        if (hi[q] >= 0 && !taken(hi[q])) sel[ns++] = hi[q];
    for (int q = K_near; q < Mp && ns < K; ++q)
        if (pi[q] >= 0 && !taken(pi[q])) sel[ns++] = pi[q];
    for (int a = 1; a < ns; ++a) {
        const int v = sel[a];
        int b = a - 1;
        while (b >= 0 && sel[b] > v) { sel[b + 1] = sel[b]; --b; }
        sel[b + 1] = v;
    }
    for (int q = 0; q < K; ++q) cand[(int64_t)i * K + q] = q < ns ? sel[q] : -1;
}

// Distinct exemplars: flag every point chosen as an exemplar, then list the
// flagged points in increasing order (exclusive prefix sum of the flags).
__global__ void mark_points_kernel(const int32_t* __restrict__ e, int64_t n_e, int64_t N, int* __restrict__ flag) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_e) return;
    const int32_t v = e[k];
    if (v >= 0 && v < N) flag[v] = 1;
}
__global__ void compact_points_kernel(const int* __restrict__ flag, const int* __restrict__ off, int64_t N,
                                      int32_t* __restrict__ points, int* __restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (flag[i]) points[off[i]] = (int32_t)i;
    if (i == N - 1) *count = off[i] + flag[i];
}

// mean over rows of log(dist[i][F-1]) in FP64: per-block partials, fixed order
__global__ void log_mean_partial_kernel(const float* __restrict__ dist, int N, int M, int col, double* __restrict__ part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        acc += log(fmax((double)dist[(int64_t)i * M + col], 1e-30));
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void features_kernel(const float* __restrict__ dist, int N, int M, int F, float log_scale,
                                float* __restrict__ feats) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)N * F) return;
    const int64_t i = e / F;
    const int q = (int)(e - i * F);
    feats[e] = logf(fmaxf(dist[i * M + q], 1e-30f)) - log_scale;
}

// ---------------------------------------------------------------------------
// MLP: logits = W3 . relu(W2^T relu(W1^T f + b1) + b2) + b3, width 128
// ---------------------------------------------------------------------------
constexpr int MH = 128;     // width
constexpr int MS = 32;      // samples per tile
constexpr int MAXF = 32;    // input features
constexpr int W2LD = MH + 1;  // padded row stride of W2 in shared memory

// offsets of the flat FP32 parameter vector
struct MLPLayout {
    int F, P, oW1, ob1, oW2, ob2, oW3, ob3;
};
__host__ __device__ inline MLPLayout mlp_layout(int F) {
    MLPLayout y;
    y.F = F;
    y.oW1 = 0;
    y.ob1 = y.oW1 + F * MH;
    y.oW2 = y.ob1 + MH;
    y.ob2 = y.oW2 + MH * MH;
    y.oW3 = y.ob2 + MH;
    y.ob3 = y.oW3 + MH;
    y.P = y.ob3 + 1;
    return y;
}

struct MLPSmem {
    float* W2;   // [MH][W2LD]
    float* W1;   // [MAXF][MH]
    float* x;    // [MS][MAXF]
    float* h1;   // [MS][MH]
    float* red;  // [MS][4] per-warp partials
    float* g;    // [MS]
    float* lq;   // [MS] per-sample loss terms
    float* d2;   // [MS][MH]
    float* dW2;  // [MH][W2LD]
};
__device__ inline MLPSmem mlp_smem(float* base, bool train) {
    MLPSmem m;
    m.W2 = base;
    m.W1 = m.W2 + MH * W2LD;
    m.x = m.W1 + MAXF * MH;
    m.h1 = m.x + MS * MAXF;
    m.red = m.h1 + MS * MH;
    m.g = m.red + MS * 4;
    m.lq = m.g + MS;
    m.d2 = m.lq + MS;
    m.dW2 = train ? m.d2 + MS * MH : nullptr;
    return m;
}
size_t mlp_smem_bytes(bool train) {
    size_t f = (size_t)MH * W2LD + MAXF * MH + MS * MAXF + MS * MH + MS * 4 + 2 * MS + MS * MH;
    if (train) f += (size_t)MH * W2LD;
    return f * sizeof(float);
}

__device__ inline float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// Loads the BF16 weights as FP32 into shared memory (W1, W2).
__device__ void mlp_load_weights(const MLPSmem& s, int F, const __nv_bfloat16* W1h, const __nv_bfloat16* W2h) {
    for (int e = threadIdx.x; e < MH * MH; e += MH) s.W2[(e / MH) * W2LD + (e % MH)] = bf(W2h[e]);
    for (int e = threadIdx.x; e < F * MH; e += MH) s.W1[e] = bf(W1h[e]);
}

// Forward of one tile for thread u: h1 (shared), h2 (registers), logits.
__device__ void mlp_tile_forward(const MLPSmem& s, int F, int ns, const float* b1, const float* b2,
                                 float w3u, float b3, float (&h2)[MS], float (&logit)[MS], bool (&pos1)[MS]) {
    const int u = threadIdx.x, lane = u & 31, warp = u >> 5;
    float a[MS];
#pragma unroll
    for (int q = 0; q < MS; ++q) a[q] = b1[u];
    for (int f = 0; f < F; ++f) {
        const float w = s.W1[f * MH + u];
#pragma unroll
        for (int q = 0; q < MS; ++q) a[q] = fmaf(s.x[q * MAXF + f], w, a[q]);
    }
#pragma unroll
    for (int q = 0; q < MS; ++q) {
        pos1[q] = a[q] > 0.f;
        s.h1[q * MH + u] = fmaxf(a[q], 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MS; ++q) a[q] = b2[u];
    for (int v = 0; v < MH; ++v) {
        const float w = s.W2[v * W2LD + u];
#pragma unroll
        for (int q = 0; q < MS; ++q) a[q] = fmaf(s.h1[q * MH + v], w, a[q]);
    }
#pragma unroll
    for (int q = 0; q < MS; ++q) h2[q] = fmaxf(a[q], 0.f);
    // logits: warp sums then the 4 warps in order
#pragma unroll
    for (int q = 0; q < MS; ++q) {
        float c = h2[q] * w3u;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) s.red[q * 4 + warp] = c;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MS; ++q)
        logit[q] = b3 + ((s.red[q * 4 + 0] + s.red[q * 4 + 1]) + (s.red[q * 4 + 2] + s.red[q * 4 + 3]));
    (void)ns;
}

__device__ void mlp_load_tile(const MLPSmem& s, const float* feats, int64_t n, int F, int64_t s0) {
    for (int e = threadIdx.x; e < MS * MAXF; e += MH) {
        const int q = e / MAXF, f = e - q * MAXF;
        const int64_t r = s0 + q;
        s.x[e] = (r < n && f < F) ? feats[r * F + f] : 0.f;
    }
}

__global__ void __launch_bounds__(MH) mlp_forward_kernel(const float* __restrict__ feats, int64_t n, int F,
                                                        const __nv_bfloat16* __restrict__ W1h, const float* __restrict__ b1,
                                                        const __nv_bfloat16* __restrict__ W2h, const float* __restrict__ b2,
                                                        const __nv_bfloat16* __restrict__ W3h, const float* __restrict__ b3,
                                                        float* __restrict__ out) {
    extern __shared__ __align__(16) float msm[];
    const MLPSmem s = mlp_smem(msm, false);
    mlp_load_weights(s, F, W1h, W2h);
    const float w3u = bf(W3h[threadIdx.x]);
    const float bb3 = b3[0];
    for (int64_t s0 = (int64_t)blockIdx.x * MS; s0 < n; s0 += (int64_t)gridDim.x * MS) {
        __syncthreads();
        mlp_load_tile(s, feats, n, F, s0);
        __syncthreads();
        float h2[MS], logit[MS];
        bool pos1[MS];
        mlp_tile_forward(s, F, 0, b1, b2, w3u, bb3, h2, logit, pos1);
        if (threadIdx.x < MS && s0 + threadIdx.x < n) {
            float v = 0.f;
#pragma unroll
            for (int q = 0; q < MS; ++q)
                if (q == (int)threadIdx.x) v = logit[q];
            out[s0 + threadIdx.x] = v;
        }
    }
}

// Forward + backward over all samples; per-CTA gradient partials [P] and
// loss partial, summed in CTA order by mlp_reduce_kernel.
__global__ void __launch_bounds__(MH) mlp_grad_kernel(const float* __restrict__ feats, const float* __restrict__ labels,
                                                     int64_t n, int F, float pos_weight,
                                                     const __nv_bfloat16* __restrict__ W1h, const float* __restrict__ b1,
                                                     const __nv_bfloat16* __restrict__ W2h, const float* __restrict__ b2,
                                                     const __nv_bfloat16* __restrict__ W3h, const float* __restrict__ b3,
                                                     float* __restrict__ gpart, float* __restrict__ lpart) {
    extern __shared__ __align__(16) float msm[];
    const MLPSmem s = mlp_smem(msm, true);
    const MLPLayout y = mlp_layout(F);
    const int u = threadIdx.x;
    mlp_load_weights(s, F, W1h, W2h);
    for (int e = u; e < MH * W2LD; e += MH) s.dW2[e] = 0.f;
    const float w3u = bf(W3h[u]);
    const float bb3 = b3[0];
    float gW3 = 0.f, gb3 = 0.f, gb2 = 0.f, gb1 = 0.f, loss = 0.f;
    float gW1[MAXF];
#pragma unroll
    for (int f = 0; f < MAXF; ++f) gW1[f] = 0.f;
    const float inv_n = 1.0f / (float)n;
    for (int64_t s0 = (int64_t)blockIdx.x * MS; s0 < n; s0 += (int64_t)gridDim.x * MS) {
        __syncthreads();
        mlp_load_tile(s, feats, n, F, s0);
        __syncthreads();
        float h2[MS], logit[MS];
        bool pos1[MS];
        mlp_tile_forward(s, F, 0, b1, b2, w3u, bb3, h2, logit, pos1);
        // d loss / d logit for the tile's samples (thread q < MS)
        if (u < MS) {
            float z = 0.f;
#pragma unroll
            for (int q = 0; q < MS; ++q)
                if (q == u) z = logit[q];
            const int64_t r = s0 + u;
            float gq = 0.f;
            if (r < n) {
                const float yv = labels[r];
                const float w = yv > 0.5f ? pos_weight : 1.f;
                const float sp = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));  // softplus
                s.lq[u] = w * (sp - yv * z);
                gq = w * (1.f / (1.f + expf(-z)) - yv) * inv_n;
            } else {
                s.lq[u] = 0.f;
            }
            s.g[u] = gq;
        }
        __syncthreads();
        if (u == 0)
            for (int q = 0; q < MS; ++q) loss += s.lq[q];
        // output layer and d2 = g W3 [z2 > 0]
#pragma unroll
        for (int q = 0; q < MS; ++q) {
            const float gq = s.g[q];
            gW3 = fmaf(gq, h2[q], gW3);
            const float d = h2[q] > 0.f ? gq * w3u : 0.f;
            s.d2[q * MH + u] = d;
            gb2 += d;
        }
        if (u == 0)
            for (int q = 0; q < MS; ++q) gb3 += s.g[q];
        __syncthreads();
        // dW2[v][u] += sum_q h1[q][v] d2[q][u]  (thread u owns column u)
        for (int v = 0; v < MH; ++v) {
            float acc = 0.f;
#pragma unroll
            for (int q = 0; q < MS; ++q) acc = fmaf(s.h1[q * MH + v], s.d2[q * MH + u], acc);
            s.dW2[v * W2LD + u] += acc;
        }
        // d1[q][v] = (sum_u d2[q][u] W2[v][u]) [z1 > 0]   (thread v = u)
        const int v = u;
        float d1[MS];
#pragma unroll
        for (int q = 0; q < MS; ++q) d1[q] = 0.f;
        for (int uu = 0; uu < MH; ++uu) {
            const float w = s.W2[v * W2LD + uu];
#pragma unroll
            for (int q = 0; q < MS; ++q) d1[q] = fmaf(s.d2[q * MH + uu], w, d1[q]);
        }
#pragma unroll
        for (int q = 0; q < MS; ++q) {
            const float dq = pos1[q] ? d1[q] : 0.f;
            gb1 += dq;
#pragma unroll
            for (int f = 0; f < MAXF; ++f)
                if (f < F) gW1[f] = fmaf(s.x[q * MAXF + f], dq, gW1[f]);
        }
    }
    __syncthreads();
    float* gp = gpart + (int64_t)blockIdx.x * y.P;
#pragma unroll
    for (int f = 0; f < MAXF; ++f)
        if (f < F) gp[y.oW1 + f * MH + u] = gW1[f];
    gp[y.ob1 + u] = gb1;
    for (int vv = 0; vv < MH; ++vv) gp[y.oW2 + vv * MH + u] = s.dW2[vv * W2LD + u];
    gp[y.ob2 + u] = gb2;
    gp[y.oW3 + u] = gW3;
    if (u == 0) {
        gp[y.ob3] = gb3;
        lpart[blockIdx.x] = loss;
    }
}

__global__ void mlp_reduce_kernel(const float* __restrict__ gpart, const float* __restrict__ lpart, int ncta, int P,
                                  int64_t n, float* __restrict__ grads, float* __restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) {
        float acc = 0.f;
        for (int c = 0; c < ncta; ++c) acc += gpart[(int64_t)c * P + p];
        grads[p] = acc;
    }
    if (p == 0) {
        double l = 0.0;
        for (int c = 0; c < ncta; ++c) l += lpart[c];
        loss[0] = (float)(l / (double)n);
    }
}

// Adam on the FP32 master parameters, then the BF16 weight copies.
__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int P, float lr, float b1, float b2, float eps, float c1,
                            float c2, int F, __nv_bfloat16* __restrict__ W1h, __nv_bfloat16* __restrict__ W2h,
                            __nv_bfloat16* __restrict__ W3h) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const float gp = g[p];
    const float mp = b1 * m[p] + (1.f - b1) * gp;
    const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
    m[p] = mp;
    v[p] = vp;
    const float th = theta[p] - lr * (mp / c1) / (sqrtf(vp / c2) + eps);
    theta[p] = th;
    const MLPLayout y = mlp_layout(F);
    if (p < y.ob1) W1h[p - y.oW1] = __float2bfloat16_rn(th);
    else if (p >= y.oW2 && p < y.ob2) W2h[p - y.oW2] = __float2bfloat16_rn(th);
    else if (p >= y.oW3 && p < y.ob3) W3h[p - y.oW3] = __float2bfloat16_rn(th);
}

__global__ void refresh_bf16_kernel(const float* __restrict__ theta, int P, int F, __nv_bfloat16* __restrict__ W1h,
                                    __nv_bfloat16* __restrict__ W2h, __nv_bfloat16* __restrict__ W3h) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const MLPLayout y = mlp_layout(F);
    const float th = theta[p];
    if (p < y.ob1) W1h[p - y.oW1] = __float2bfloat16_rn(th);
    else if (p >= y.oW2 && p < y.ob2) W2h[p - y.oW2] = __float2bfloat16_rn(th);
    else if (p >= y.oW3 && p < y.ob3) W3h[p - y.oW3] = __float2bfloat16_rn(th);
}

// ---------------------------------------------------------------------------
// candidate selection: self + K_near nearest + highest-scoring pool members
// ---------------------------------------------------------------------------
__global__ void select_candidates_kernel(const int32_t* __restrict__ pool, int N, int M, const float* __restrict__ score,
                                         int K, int K_near, int32_t* __restrict__ cand) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int sel[64];
    int ns = 0;
    sel[ns++] = i;
    const int32_t* pi = pool + (int64_t)i * M;
    if (!score) {
        for (int q = 0; q < K - 1; ++q) sel[ns++] = pi[q];
    } else {
        for (int q = 0; q < K_near; ++q) sel[ns++] = pi[q];
        uint32_t used[4] = {0u, 0u, 0u, 0u};  // pool positions already taken (M <= 128)
        for (int r = 0; r < K - 1 - K_near; ++r) {
            int best = -1;
            float bs = -kInf;
            for (int q = K_near; q < M; ++q) {
                if (used[q >> 5] & (1u << (q & 31))) continue;
                const float sv = score[pi[q]];
                if (best < 0 || sv > bs) { bs = sv; best = q; }
            }
            used[best >> 5] |= 1u << (best & 31);
            sel[ns++] = pi[best];
        }
    }
    for (int a = 1; a < K; ++a) {  // sort by index
        const int v = sel[a];
        int b = a - 1;
        while (b >= 0 && sel[b] > v) { sel[b + 1] = sel[b]; --b; }
        sel[b + 1] = v;
    }
    for (int q = 0; q < K; ++q) cand[(int64_t)i * K + q] = sel[q];
}

}  // namespace
}  // namespace hap

using namespace hap;

#define PCU(x)                          \
    do {                                \
        if ((x) != cudaSuccess) {       \
            cudaGetLastError();         \
            return HAP_ECUDA;           \
        }                               \
    } while (0)

struct hap_mlp {
    int F = 0;
    MLPLayout y{};
    float* theta = nullptr;  // FP32 master parameters [P]
    float* m = nullptr;
    float* v = nullptr;
    float* grads = nullptr;
    float* loss = nullptr;
    __nv_bfloat16* W1h = nullptr;
    __nv_bfloat16* W2h = nullptr;
    __nv_bfloat16* W3h = nullptr;
    float* gpart = nullptr;
    float* lpart = nullptr;
    int ncta = 0;
    int64_t step = 0;
    cudaStream_t stream = nullptr;
};

// kernels launched by the stateless proposal entry points (hap_proposal_launches)
static std::atomic<int64_t> g_launches{0};

extern "C" {

int64_t hap_proposal_launches(void) { return g_launches.load(); }

static int knn_launch(const float* Q, int64_t Nq, const float* C, const int32_t* cid, int64_t Nc, int64_t d, int M,
                      int32_t* idx, float* dist, cudaStream_t st, int method) {
    if (method != HAP_KNN_AUTO && method != HAP_KNN_CUDA_CORES && method != HAP_KNN_TENSOR_CORES) return HAP_EINVAL;
    const int M2 = std::min(M + 16, knn_tc_max_candidates());
    const bool tc_ok = d <= 64 && M + 16 <= knn_tc_max_candidates();
    if (method == HAP_KNN_TENSOR_CORES && !tc_ok) return HAP_EUNSUPPORTED;
    // tensor cores once the N_q x N_c distances dominate (the first pass keeps
    // M + 16 candidates per query for the exact re-rank)
    if (method == HAP_KNN_TENSOR_CORES || (method == HAP_KNN_AUTO && tc_ok && (double)Nq * (double)Nc >= 16e6)) {
        int64_t nl = 0;
        cudaError_t err = launch_knn_tc(Q, Nq, C, cid, Nc, d, M, M2, idx, dist, st, &nl);
        if (err == cudaErrorNotSupported) { cudaGetLastError(); return HAP_EUNSUPPORTED; }
        PCU(err);
        g_launches += nl;
        return HAP_OK;
    }
    const int D = d <= 4 ? 4 : d <= 8 ? 8 : d <= 16 ? 16 : d <= 32 ? 32 : 64;
    const size_t smem = ((size_t)KNN_TILE * D + (size_t)M * KNN_ROWS * 2) * 4;
    const unsigned grid = (unsigned)((Nq + KNN_ROWS - 1) / KNN_ROWS);
#define HAP_KNN_CASE(DD)                                                                                \
    if (D == DD) {                                                                                      \
        PCU(cudaFuncSetAttribute(knn_kernel<DD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        knn_kernel<DD><<<grid, KNN_ROWS, smem, st>>>(Q, (int)Nq, C, cid, (int)Nc, (int)d, M, idx, dist); \
    }
    HAP_KNN_CASE(4) HAP_KNN_CASE(8) HAP_KNN_CASE(16) HAP_KNN_CASE(32) HAP_KNN_CASE(64)
#undef HAP_KNN_CASE
    PCU(cudaGetLastError());
    g_launches += 1;
    return HAP_OK;
}

int hap_knn_with(const float* X, int64_t N, int64_t d, int M, int method, int32_t* idx, float* dist, void* stream) {
    if (!X || !idx || !dist || N < 2 || d < 1 || d > 64 || M < 1 || M > KNN_MAXM || M >= N) return HAP_EINVAL;
    return knn_launch(X, N, X, nullptr, N, d, M, idx, dist, static_cast<cudaStream_t>(stream), method);
}

int hap_knn(const float* X, int64_t N, int64_t d, int M, int32_t* idx, float* dist, void* stream) {
    return hap_knn_with(X, N, d, M, HAP_KNN_AUTO, idx, dist, stream);
}

int hap_knn_subset(const float* X, int64_t N, int64_t d, const int32_t* subset, int64_t Ns, int M, int32_t* idx,
                   float* dist, void* stream) {
    return hap_knn_subset_with(X, N, d, subset, Ns, M, HAP_KNN_AUTO, idx, dist, stream);
}

int hap_knn_subset_with(const float* X, int64_t N, int64_t d, const int32_t* subset, int64_t Ns, int M, int method,
                        int32_t* idx, float* dist, void* stream) {
    if (!X || !subset || !idx || !dist || N < 1 || Ns < 1 || d < 1 || d > 64 || M < 1 || M > KNN_MAXM || M > Ns)
        return HAP_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* C = nullptr;
    PCU(cudaMallocAsync(&C, (size_t)Ns * d * 4, st));
    // gather the subset's points (one row per thread block)
    for (int64_t q = 0; q < Ns; q += 65535) {
        const int64_t nb = Ns - q < 65535 ? Ns - q : 65535;
        gather_rows_kernel<<<(unsigned)nb, 64, 0, st>>>(X, d, subset + q, C + q * d);
        g_launches += 1;
    }
    int rc = knn_launch(X, N, C, subset, Ns, d, M, idx, dist, st, method);
    cudaFreeAsync(C, st);
    return rc;
}

int hap_top_scores(const float* score, int64_t N, int64_t H, int32_t* hubs, void* stream) {
    if (!score || !hubs || N < 1 || H < 1 || H > N || N > (1 << 30)) return HAP_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int n2 = 1;
    while (n2 < N) n2 <<= 1;
    uint64_t* keys = nullptr;
    PCU(cudaMallocAsync(&keys, (size_t)n2 * 8, st));
    const unsigned g = (unsigned)((n2 + 255) / 256);
    hub_keys_kernel<<<g, 256, 0, st>>>(score, (int)N, n2, keys);
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) bitonic_step_kernel<<<g, 256, 0, st>>>(keys, n2, j, k);
    hub_ids_kernel<<<(unsigned)((H + 255) / 256), 256, 0, st>>>(keys, (int)H, hubs);
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) g_launches += 1;
    g_launches += 2;
    cudaError_t err = cudaGetLastError();
    cudaFreeAsync(keys, st);
    PCU(err);
    return HAP_OK;
}

int hap_exemplar_points(const int32_t* e, int64_t n_e, int64_t N, int32_t* points, int64_t* count, void* stream) {
    if (!e || !points || !count || n_e < 1 || N < 1 || N > (1 << 30)) return HAP_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t tiles = scan_tiles(N);
    char* buf = nullptr;
    const size_t fb = ((size_t)N * 4 + 255) / 256 * 256;
    PCU(cudaMallocAsync(reinterpret_cast<void**>(&buf), 2 * fb + (size_t)tiles * 8 + 256, st));
    int* flag = reinterpret_cast<int*>(buf);
    int* off = reinterpret_cast<int*>(buf + fb);
    int64_t* tsum = reinterpret_cast<int64_t*>(buf + 2 * fb);
    int* cnt = reinterpret_cast<int*>(buf + 2 * fb + (size_t)tiles * 8);
    cudaError_t err = cudaMemsetAsync(flag, 0, (size_t)N * 4, st);
    if (err == cudaSuccess) {
        mark_points_kernel<<<(unsigned)((n_e + 255) / 256), 256, 0, st>>>(e, n_e, N, flag);
        err = scan_exclusive(flag, N, off, tsum, st);
    }
    if (err == cudaSuccess) {
        compact_points_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(flag, off, N, points, cnt);
        err = cudaGetLastError();
    }
    int c = 0;
    if (err == cudaSuccess) err = cudaMemcpyAsync(&c, cnt, 4, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    cudaFreeAsync(buf, st);
    PCU(err);
    g_launches += 5;  // mark, three scan launches, compact
    *count = c;
    return HAP_OK;
}

int hap_select_hub_candidates(const int32_t* pool, int64_t N, int Mp, const int32_t* hubnn, int Mh, int K, int K_near,
                              int32_t* cand, void* stream) {
    if (!pool || !hubnn || !cand || N < 2 || K < 2 || K > 64 || K_near < 0 || K_near > Mp || Mh < 0) return HAP_EINVAL;
    select_hub_candidates_kernel<<<(unsigned)((N + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
        pool, Mp, hubnn, Mh, (int)N, K, K_near, cand);
    PCU(cudaGetLastError());
    g_launches += 1;
    return HAP_OK;
}

int hap_knn_features(const float* dist, int64_t N, int M, int F, float* feats, float* log_scale_out, void* stream) {
    if (!dist || !feats || N < 1 || F < 1 || F > M || F > MAXF) return HAP_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nb = 64;
    std::vector<double> part(nb);
    double* dpart = nullptr;
    PCU(cudaMallocAsync(&dpart, nb * sizeof(double), st));
    log_mean_partial_kernel<<<nb, 256, 0, st>>>(dist, (int)N, M, F - 1, dpart);
    PCU(cudaGetLastError());
    PCU(cudaMemcpyAsync(part.data(), dpart, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    PCU(cudaFreeAsync(dpart, st));
    PCU(cudaStreamSynchronize(st));
    double tot = 0.0;
    for (double x : part) tot += x;
    const float ls = (float)(tot / (double)N);
    if (log_scale_out) *log_scale_out = ls;
    const int64_t n = N * F;
    features_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dist, (int)N, M, F, ls, feats);
    PCU(cudaGetLastError());
    g_launches += 2;
    return HAP_OK;
}

int hap_mlp_create(int F, const float* theta0, hap_mlp** out) {
    if (!out || F < 1 || F > MAXF || !theta0) return HAP_EINVAL;
    hap_mlp* h = new (std::nothrow) hap_mlp();
    if (!h) return HAP_ENOMEM;
    h->F = F;
    h->y = mlp_layout(F);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    h->ncta = sms;
    const size_t P = h->y.P;
    bool ok = cudaMalloc(&h->theta, P * 4) == cudaSuccess && cudaMalloc(&h->m, P * 4) == cudaSuccess &&
              cudaMalloc(&h->v, P * 4) == cudaSuccess && cudaMalloc(&h->grads, P * 4) == cudaSuccess &&
              cudaMalloc(&h->loss, 16) == cudaSuccess && cudaMalloc(&h->W1h, (size_t)F * MH * 2) == cudaSuccess &&
              cudaMalloc(&h->W2h, (size_t)MH * MH * 2) == cudaSuccess && cudaMalloc(&h->W3h, MH * 2) == cudaSuccess &&
              cudaMalloc(&h->gpart, (size_t)h->ncta * P * 4) == cudaSuccess &&
              cudaMalloc(&h->lpart, (size_t)h->ncta * 4) == cudaSuccess;
    if (!ok) { cudaGetLastError(); hap_mlp_destroy(h); return HAP_ENOMEM; }
    cudaMemcpy(h->theta, theta0, P * 4, cudaMemcpyHostToDevice);
    cudaMemset(h->m, 0, P * 4);
    cudaMemset(h->v, 0, P * 4);
    const size_t fsm = mlp_smem_bytes(false), tsm = mlp_smem_bytes(true);
    if (cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm) != cudaSuccess ||
        cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm) != cudaSuccess) {
        cudaGetLastError();
        hap_mlp_destroy(h);
        return HAP_ECUDA;
    }
    refresh_bf16_kernel<<<(unsigned)((P + 255) / 256), 256>>>(h->theta, (int)P, F, h->W1h, h->W2h, h->W3h);
    if (cudaDeviceSynchronize() != cudaSuccess) { cudaGetLastError(); hap_mlp_destroy(h); return HAP_ECUDA; }
    *out = h;
    return HAP_OK;
}

void hap_mlp_destroy(hap_mlp* h) {
    if (!h) return;
    cudaFree(h->theta); cudaFree(h->m); cudaFree(h->v); cudaFree(h->grads); cudaFree(h->loss);
    cudaFree(h->W1h); cudaFree(h->W2h); cudaFree(h->W3h); cudaFree(h->gpart); cudaFree(h->lpart);
    delete h;
}

int hap_mlp_set_stream(hap_mlp* h, void* stream) {
    if (!h) return HAP_EINVAL;
    h->stream = static_cast<cudaStream_t>(stream);
    return HAP_OK;
}

int hap_mlp_num_params(hap_mlp* h, int64_t* P) {
    if (!h || !P) return HAP_EINVAL;
    *P = h->y.P;
    return HAP_OK;
}

int hap_mlp_get_params(hap_mlp* h, float* theta_host) {
    if (!h || !theta_host) return HAP_EINVAL;
    PCU(cudaMemcpyAsync(theta_host, h->theta, (size_t)h->y.P * 4, cudaMemcpyDeviceToHost, h->stream));
    PCU(cudaStreamSynchronize(h->stream));
    return HAP_OK;
}

int hap_mlp_forward(hap_mlp* h, const float* feats, int64_t n, float* logits) {
    if (!h || !feats || !logits || n < 1) return HAP_EINVAL;
    const MLPLayout& y = h->y;
    const int grid = (int)std::min<int64_t>((n + MS - 1) / MS, (int64_t)h->ncta * 4);
    mlp_forward_kernel<<<grid, MH, mlp_smem_bytes(false), h->stream>>>(feats, n, h->F, h->W1h, h->theta + y.ob1, h->W2h,
                                                                       h->theta + y.ob2, h->W3h, h->theta + y.ob3, logits);
    PCU(cudaGetLastError());
    g_launches += 1;
    return HAP_OK;
}

int hap_mlp_gradients(hap_mlp* h, const float* feats, const float* labels, int64_t n, float pos_weight,
                      float* grads_host, float* loss_host) {
    if (!h || !feats || !labels || n < 1) return HAP_EINVAL;
    const MLPLayout& y = h->y;
    mlp_grad_kernel<<<h->ncta, MH, mlp_smem_bytes(true), h->stream>>>(feats, labels, n, h->F, pos_weight, h->W1h,
                                                                     h->theta + y.ob1, h->W2h, h->theta + y.ob2, h->W3h,
                                                                     h->theta + y.ob3, h->gpart, h->lpart);
    PCU(cudaGetLastError());
    mlp_reduce_kernel<<<(unsigned)((y.P + 255) / 256), 256, 0, h->stream>>>(h->gpart, h->lpart, h->ncta, y.P, n,
                                                                           h->grads, h->loss);
    PCU(cudaGetLastError());
    g_launches += 2;
    if (grads_host) PCU(cudaMemcpyAsync(grads_host, h->grads, (size_t)y.P * 4, cudaMemcpyDeviceToHost, h->stream));
    if (loss_host) PCU(cudaMemcpyAsync(loss_host, h->loss, 4, cudaMemcpyDeviceToHost, h->stream));
    if (grads_host || loss_host) PCU(cudaStreamSynchronize(h->stream));
    return HAP_OK;
}

int hap_mlp_train_step(hap_mlp* h, const float* feats, const float* labels, int64_t n, float pos_weight, float lr,
                       float* loss_host) {
    int rc = hap_mlp_gradients(h, feats, labels, n, pos_weight, nullptr, nullptr);
    if (rc) return rc;
    h->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)h->step), c2 = 1.f - powf(b2, (float)h->step);
    adam_kernel<<<(unsigned)((h->y.P + 255) / 256), 256, 0, h->stream>>>(h->theta, h->m, h->v, h->grads, h->y.P, lr, b1,
                                                                        b2, 1e-8f, c1, c2, h->F, h->W1h, h->W2h, h->W3h);
    PCU(cudaGetLastError());
    g_launches += 1;
    if (loss_host) {
        PCU(cudaMemcpyAsync(loss_host, h->loss, 4, cudaMemcpyDeviceToHost, h->stream));
        PCU(cudaStreamSynchronize(h->stream));
    }
    return HAP_OK;
}

int hap_select_candidates(const int32_t* pool, int64_t N, int M, const float* score, int K, int K_near, int32_t* cand,
                          void* stream) {
    if (!pool || !cand || N < 2 || K < 2 || K > 64 || M < K - 1 || M > KNN_MAXM || K_near < 0 || K_near > K - 1)
        return HAP_EINVAL;
    select_candidates_kernel<<<(unsigned)((N + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
        pool, (int)N, M, score, K, K_near, cand);
    PCU(cudaGetLastError());
    g_launches += 1;
    return HAP_OK;
}

}  // extern "C"
