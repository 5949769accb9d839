// Exemplar extraction (Eq. 2.8), FP64 net similarity, state read-out, and the
// similarity input paths (copy, FP32 CUDA-core build of s_ij = -||x_i-x_j||^2).
#include "hap_common.cuh"
#include "hap_internal.h"

namespace hap {

// alpha of the current iteration: the stored (one step behind) value with the
// pending update applied exactly as the row pass applies it.
HAP_DEV float alpha_now(float a, float r, float b, bool diag, bool pending, float lam, float oml) {
    return pending ? damp(a, avail_target(b, r, diag), lam, oml) : a;
}

// Eq. 2.8: one CTA per (l, i), argmax_j(alpha + rho) with the lowest index on ties.
__global__ void exemplars_kernel(const float* __restrict__ A, const float* __restrict__ R,
                                 const float* __restrict__ b, int pending, float lam, float oml,
                                 int64_t N, int64_t ld, int64_t NR, int64_t R0, int32_t* __restrict__ e) {
    __shared__ float sv[32];
    __shared__ int si[32];
    const int64_t rowid = blockIdx.x;  // l * NR + (i - R0): rows R0 .. R0 + NR - 1 are held
    const int64_t l = rowid / NR, i = R0 + rowid - l * NR;
    const float* Ar = A + rowid * ld;
    const float* Rr = R + rowid * ld;
    const float* bl = b + l * ld;
    float best = -kInf;
    int bi = 0x7fffffff;
    for (int64_t j0 = 4LL * threadIdx.x; j0 < N; j0 += 4LL * blockDim.x) {
        const float4 a4 = ld_stream(Ar + j0), r4 = ld_stream(Rr + j0);
        const float4 b4 = pending ? __ldg(reinterpret_cast<const float4*>(bl + j0)) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t j = j0 + q;
            if (j < N) {
                const float r = f4_get(r4, q);
                const float v = __fadd_rn(alpha_now(f4_get(a4, q), r, f4_get(b4, q), j == i, pending != 0, lam, oml), r);
                if (v > best) { best = v; bi = (int)j; }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sv[warp] = best; si[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (sv[w] > best || (sv[w] == best && si[w] < bi)) { best = sv[w]; bi = si[w]; }
        e[rowid] = bi;
    }
}

// alpha of the current iteration into a dense [L][N][N] buffer.
__global__ void materialize_A_kernel(float* __restrict__ dst, const float* __restrict__ A,
                                     const float* __restrict__ R, const float* __restrict__ b,
                                     int pending, float lam, float oml, int64_t N, int64_t ld, int64_t NR,
                                     int64_t R0) {
    const int64_t rowid = blockIdx.x;
    const int64_t l = rowid / NR, i = R0 + rowid - l * NR;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
        const float a = A[rowid * ld + j], r = R[rowid * ld + j];
        dst[rowid * N + j] = alpha_now(a, r, pending ? b[l * ld + j] : 0.f, j == i, pending != 0, lam, oml);
    }
}

// NS^l = sum_i s^l_{i, e_i} in FP64, one CTA per level, fixed-order tree.
template <typename ST>
__global__ void netsim_kernel(const ST* __restrict__ S, int64_t s_level_stride, const float* __restrict__ pref,
                              const int32_t* __restrict__ e, int64_t N, int64_t ld, double* __restrict__ ns) {
    __shared__ double part[1024];
    const int l = blockIdx.x;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const int64_t ej = e[(int64_t)l * N + i];
        double s;
        if (ej == i) s = (double)pref[(int64_t)l * ld + i];
        else s = (double)(float)S[(int64_t)l * s_level_stride + i * ld + ej];
        acc += s;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) ns[l] = part[0];
}

// Acceptance check of an assignment (Eq. 2.8), one CTA per level: points
// whose exemplar is its own exemplar (e_{e_i} = e_i) and exemplars (e_i = i);
// integer counts, exact in any order.
__global__ void acceptance_kernel(const int32_t* __restrict__ e, int64_t N, long long* __restrict__ out) {
    __shared__ long long part[2][1024];
    const int l = blockIdx.x;
    const int32_t* el = e + (int64_t)l * N;
    long long cons = 0, ex = 0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const int32_t ej = el[i];
        cons += (ej >= 0 && ej < N && el[ej] == ej) ? 1 : 0;
        ex += (ej == i) ? 1 : 0;
    }
    part[0][threadIdx.x] = cons;
    part[1][threadIdx.x] = ex;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            part[0][threadIdx.x] += part[0][threadIdx.x + o];
            part[1][threadIdx.x] += part[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[l] = part[0][0];
        out[gridDim.x + l] = part[1][0];
    }
}

// Similarity copy with type conversion (FP32 <-> BF16, round to nearest).
template <typename DT, typename ST>
__global__ void copy_similarity_kernel(DT* __restrict__ dst, int64_t ld, const ST* __restrict__ src,
                                       int64_t ld_src, int64_t N) {
    const int64_t i = blockIdx.x;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
        const float v = (float)src[i * ld_src + j];
        if constexpr (sizeof(DT) == 2) dst[i * ld + j] = __float2bfloat16_rn(v);
        else dst[i * ld + j] = v;
    }
}

// Precondition check of the similarity (§2 admits s_ij down to -inf; the
// library requires finite values): one block per row of one level, the
// off-diagonal entries j < N tested, ST_BOUNDS recorded once per row that
// holds a NaN or an infinity.
template <typename ST>
__global__ void check_finite_kernel(const ST* __restrict__ S, int64_t N, int64_t ld, unsigned* status) {
    const int64_t i = blockIdx.x, l = blockIdx.y;
    const ST* row = S + (l * N + i) * ld;
    bool bad = false;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
        const float v = (float)row[j];
        bad |= (j != i) && !(fabsf(v) <= 3.402823466e38f);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_BOUNDS);
}

// Dense FP32 copy of one level's similarity with the preferences on the diagonal.
template <typename ST>
__global__ void read_similarity_kernel(float* __restrict__ dst, const ST* __restrict__ S,
                                       const float* __restrict__ pref_l, int64_t N, int64_t ld) {
    const int64_t i = blockIdx.x;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x)
        dst[i * N + j] = (j == i) ? pref_l[i] : (float)S[i * ld + j];
}

// FP32 CUDA-core build: s_ij = -sum_k (x_ik - x_jk)^2 in the direct difference
// form, 64 x 64 tile per CTA, 4 x 4 per thread, X staged k-major in shared memory.
template <typename OT>
__global__ void __launch_bounds__(256) sbuild_f32_kernel(const float* __restrict__ X, int64_t N, int64_t d,
                                                        OT* __restrict__ S, int64_t ld) {
    constexpr int BT = 64, BK = 16;
    __shared__ float xi[BK][BT + 4], xj[BK][BT + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t i0 = (int64_t)blockIdx.y * BT, j0 = (int64_t)blockIdx.x * BT;
    float acc[4][4] = {};
    for (int64_t k0 = 0; k0 < d; k0 += BK) {
        for (int q = threadIdx.x; q < BT * BK; q += 256) {
            const int r = q / BK, kk = q % BK;
            const int64_t gi = i0 + r, gj = j0 + r, gk = k0 + kk;
            xi[kk][r] = (gi < N && gk < d) ? X[gi * d + gk] : 0.f;
            xj[kk][r] = (gj < N && gk < d) ? X[gj * d + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[4], bv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = xi[kk][ty * 4 + q]; bv[q] = xj[kk][tx * 4 + q]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float df = a[u] - bv[v];
                    acc[u][v] = fmaf(df, df, acc[u][v]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t gi = i0 + ty * 4 + u;
        if (gi >= N) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t gj = j0 + tx * 4 + v;
            if (gj >= N) continue;
            const float s = -acc[u][v];
            if constexpr (sizeof(OT) == 2) S[gi * ld + gj] = __float2bfloat16_rn(s);
            else S[gi * ld + gj] = s;
        }
    }
}

// ---------------------------------------------------------------------------
cudaError_t launch_exemplars(const float* A, const float* R, const float* b, int pending,
                             float lam, float oml, int64_t N, int64_t ld, int L,
                             int32_t* e, cudaStream_t st, int64_t nrows, int64_t row0) {
    int threads = 256;
    if (N <= 1024) threads = 128;
    const int64_t NR = nrows ? nrows : N;
    exemplars_kernel<<<(unsigned)(L * NR), threads, 0, st>>>(A, R, b, pending, lam, oml, N, ld, NR, row0, e);
    return cudaGetLastError();
}

cudaError_t launch_materialize_A(float* dst, const float* A, const float* R, const float* b,
                                 int pending, float lam, float oml, int64_t N, int64_t ld, int L,
                                 cudaStream_t st, int64_t nrows, int64_t row0) {
    const int64_t NR = nrows ? nrows : N;
    materialize_A_kernel<<<(unsigned)(L * NR), 256, 0, st>>>(dst, A, R, b, pending, lam, oml, N, ld, NR, row0);
    return cudaGetLastError();
}

cudaError_t launch_netsim(const void* S, int s_bf16, int64_t s_level_stride, const float* pref,
                          const int32_t* e, int64_t N, int64_t ld, int L, double* ns, cudaStream_t st) {
    if (s_bf16)
        netsim_kernel<__nv_bfloat16><<<L, 1024, 0, st>>>(static_cast<const __nv_bfloat16*>(S), s_level_stride, pref, e, N, ld, ns);
    else
        netsim_kernel<float><<<L, 1024, 0, st>>>(static_cast<const float*>(S), s_level_stride, pref, e, N, ld, ns);
    return cudaGetLastError();
}

cudaError_t launch_acceptance(const int32_t* e, int64_t N, int L, long long* out, cudaStream_t st) {
    acceptance_kernel<<<L, 1024, 0, st>>>(e, N, out);
    return cudaGetLastError();
}

cudaError_t launch_copy_similarity(void* dst, int dst_bf16, int64_t ld, const void* src,
                                   int src_bf16, int64_t ld_src, int64_t N, cudaStream_t st, int64_t nrows) {
    const unsigned grid = (unsigned)(nrows ? nrows : N);
    if (dst_bf16 && src_bf16)
        copy_similarity_kernel<<<grid, 256, 0, st>>>(static_cast<__nv_bfloat16*>(dst), ld, static_cast<const __nv_bfloat16*>(src), ld_src, N);
    else if (dst_bf16)
        copy_similarity_kernel<<<grid, 256, 0, st>>>(static_cast<__nv_bfloat16*>(dst), ld, static_cast<const float*>(src), ld_src, N);
    else if (src_bf16)
        copy_similarity_kernel<<<grid, 256, 0, st>>>(static_cast<float*>(dst), ld, static_cast<const __nv_bfloat16*>(src), ld_src, N);
    else
        copy_similarity_kernel<<<grid, 256, 0, st>>>(static_cast<float*>(dst), ld, static_cast<const float*>(src), ld_src, N);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const void* S, int s_bf16, int levels, int64_t N, int64_t ld, unsigned* status,
                                cudaStream_t st) {
    const dim3 grid((unsigned)N, (unsigned)levels);
    if (s_bf16)
        check_finite_kernel<<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(S), N, ld, status);
    else
        check_finite_kernel<<<grid, 256, 0, st>>>(static_cast<const float*>(S), N, ld, status);
    return cudaGetLastError();
}

cudaError_t launch_read_similarity(float* dst, const void* S, int s_bf16, const float* pref_l,
                                   int64_t N, int64_t ld, cudaStream_t st) {
    if (s_bf16)
        read_similarity_kernel<<<(unsigned)N, 256, 0, st>>>(dst, static_cast<const __nv_bfloat16*>(S), pref_l, N, ld);
    else
        read_similarity_kernel<<<(unsigned)N, 256, 0, st>>>(dst, static_cast<const float*>(S), pref_l, N, ld);
    return cudaGetLastError();
}

cudaError_t launch_sbuild_f32(const float* X, int64_t N, int64_t d, void* S, int s_bf16, int64_t ld, cudaStream_t st) {
    const dim3 grid((unsigned)((N + 63) / 64), (unsigned)((N + 63) / 64));
    if (s_bf16)
        sbuild_f32_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(X, N, d, static_cast<__nv_bfloat16*>(S), ld);
    else
        sbuild_f32_kernel<float><<<grid, 256, 0, st>>>(X, N, d, static_cast<float*>(S), ld);
    return cudaGetLastError();
}

}  // namespace hap
