// Availability step of Algorithm 1's sequential level loop (Gauss-Seidel
// schedule).  Under that schedule level l's availability must be final before
// level l sends its messages, which the next level uses in the same
// iteration, so it cannot ride one step behind inside the row pass as in the
// data-parallel schedule.  Per level and iteration the library runs the fused
// row pass on level l alone (rho^l with the tau^l the previous level sent),
// the column statistics (b^l, and rho_jj + P_j of level l) and this kernel:
//   alpha^l_ij <- damp(alpha, min(0, b_j - max(0, rho_ij)))   (Eq. 2.2, i != j)
//   alpha^l_jj <- damp(alpha, b_j - rho_jj)                     (Eq. 2.3)
//   c^l_i       = max_j (alpha^l_ij + rho^l_ij)                 (Eq. 2.6)
//   phi^{l-1}_i = max_j (alpha^l_ij + s^l_ij), s^l_ii = pref    (Eq. 2.5)
//   tau^{l+1}_i = c^l_i + rho^l_ii + P^l_i                      (Eq. 2.4)
// One CTA per row (grid-stride over rows), float4 accesses, exact maxima.
#include "hap_common.cuh"
#include "hap_internal.h"

namespace hap {
namespace {

constexpr int kGsThreads = 256;

template <typename ST>
HAP_DEV float4 gs_load_s(const ST* p);
template <>
HAP_DEV float4 gs_load_s<float>(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
template <>
HAP_DEV float4 gs_load_s<__nv_bfloat16>(const __nv_bfloat16* p) {
    return SVec<__nv_bfloat16>::to_f4(__ldcs(reinterpret_cast<const uint2*>(p)));
}

template <typename ST>
__global__ void __launch_bounds__(kGsThreads) gs_availability_kernel(const GsArgs p) {
    __shared__ float red[2][kGsThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t N = p.N, ld = p.ld;
    const float lam = p.lam, oml = p.oml;
    const ST* S = static_cast<const ST*>(p.S);
    const bool want_phi = p.phi_out != nullptr;
    for (int64_t row = blockIdx.x; row < N; row += gridDim.x) {
        const int64_t off = row * ld;
        const float pref_i = p.pref[row];
        float cm = -kInf, pm = -kInf;
        for (int64_t j0 = 4 * (int64_t)tid; j0 < ld; j0 += 4 * kGsThreads) {
            const float4 a4 = ld_stream(p.A + off + j0);
            const float4 r4 = ld_stream(p.R + off + j0);
            const float4 b4 = __ldg(reinterpret_cast<const float4*>(p.b + j0));
            float4 s4 = want_phi ? gs_load_s<ST>(S + off + j0) : f4_splat(0.f);
            float4 an = a4;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t j = j0 + e;
                if (j >= N) continue;  // padding keeps alpha = -inf
                const bool diag = j == row;
                const float v = damp(f4_get(a4, e), avail_target(f4_get(b4, e), f4_get(r4, e), diag), lam, oml);
                f4_set(an, e, v);
                cm = fmaxf(cm, __fadd_rn(v, f4_get(r4, e)));
                if (want_phi) pm = fmaxf(pm, __fadd_rn(v, diag ? pref_i : f4_get(s4, e)));
            }
            st_stream(p.A + off + j0, an);
        }
        // exact block maxima of c and phi
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            cm = fmaxf(cm, __shfl_xor_sync(0xffffffffu, cm, o));
            pm = fmaxf(pm, __shfl_xor_sync(0xffffffffu, pm, o));
        }
        if (lane == 0) {
            red[0][warp] = cm;
            red[1][warp] = pm;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < kGsThreads / 32; ++w) {
                cm = fmaxf(cm, red[0][w]);
                pm = fmaxf(pm, red[1][w]);
            }
            const float cval = p.update_c ? cm : p.c[row];
            if (p.update_c) p.c[row] = cval;
            if (want_phi) p.phi_out[row] = pm;
            if (p.tau_next) p.tau_next[row] = __fadd_rn(cval, p.tp[row]);
        }
        __syncthreads();  // red is reused by the next row
    }
}

}  // namespace

cudaError_t launch_gs_availability(const GsArgs& a, int s_bf16, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    const int64_t want = (int64_t)sms * 8;
    const unsigned grid = (unsigned)(a.N < want ? a.N : want);
    if (s_bf16)
        gs_availability_kernel<__nv_bfloat16><<<grid, kGsThreads, 0, st>>>(a);
    else
        gs_availability_kernel<float><<<grid, kGsThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace hap
