// hap_iterate_noalloc: HAP iterations on caller-owned messages with the
// scratch memory of the row pass in a fixed device array of this library, so
// the call itself allocates nothing.  See include/hap.h for the contract.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "hap.h"
#include "hap_common.cuh"
#include "hap_internal.h"

namespace hap {
namespace {

// Limits of the fixed scratch: at most kMaxLevelCols = L * ld floats per
// vector and kMaxClusters row-pass clusters.
constexpr int64_t kMaxLevelCols = 16384;
constexpr int kMaxClusters = 64;
constexpr size_t kStatusBytes = 256;
constexpr size_t kVecBytes = (size_t)kMaxLevelCols * sizeof(float);
constexpr size_t kScratchBytes = kStatusBytes + 3 * kVecBytes + (size_t)kMaxClusters * kVecBytes;

// The scratch itself: status word, b, tau's column part, rho_jj, and the
// per-cluster column partials.  Every GPU that loads the library holds it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device ordinal, looked up once per
// device with that device current (host code must not use the symbol itself).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

int scratch_for_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return HAP_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HAP_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return HAP_OK;
}

// alpha <- damp(alpha, Eqs. 2.2/2.3 from b and rho) in place on the padded
// [L][N][ld] layout: applies the availability update the row pass leaves
// pending after the last iteration.
__global__ void apply_pending_alpha_kernel(float* __restrict__ A, const float* __restrict__ R,
                                           const float* __restrict__ b, float lam, float oml,
                                           int64_t N, int64_t ld) {
    const int64_t rowid = blockIdx.x;
    const int64_t l = rowid / N, i = rowid - l * N;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
        const int64_t q = rowid * ld + j;
        A[q] = damp(A[q], avail_target(b[l * ld + j], R[q], j == i), lam, oml);
    }
}

}  // namespace
}  // namespace hap

using namespace hap;

extern "C" int hap_iterate_noalloc(int64_t N, int L, float damping, int c_mode, const void* S, int s_dtype,
                                   const float* pref, float* A, float* R, float* c, float* tau, float* phi,
                                   int64_t t0, int n, void* stream) {
    if (N < 2 || L < 1 || n < 0 || t0 < 0 || !S || !pref || !A || !R || !c || !tau || !phi) return HAP_EINVAL;
    if (!(damping > 0.f && damping < 1.f)) return HAP_EINVAL;
    if (c_mode != HAP_C_PAPER && c_mode != HAP_C_FIXED) return HAP_EINVAL;
    if (s_dtype != HAP_S_F32 && s_dtype != HAP_S_BF16) return HAP_EINVAL;
    const int64_t ld = (N + 31) / 32 * 32;
    if ((int64_t)L * ld > kMaxLevelCols) return HAP_EUNSUPPORTED;  // beyond the fixed scratch
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    void* base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    unsigned char* sc = static_cast<unsigned char*>(base);
    unsigned* status = reinterpret_cast<unsigned*>(sc);
    float* b = reinterpret_cast<float*>(sc + kStatusBytes);
    float* tpart = reinterpret_cast<float*>(sc + kStatusBytes + kVecBytes);
    float* rdiag = reinterpret_cast<float*>(sc + kStatusBytes + 2 * kVecBytes);
    float* partials = reinterpret_cast<float*>(sc + kStatusBytes + 3 * kVecBytes);

    // Launch shape: 8 columns per thread, the fewest CTAs per cluster that hold
    // a row and fit in shared memory, at most kMaxClusters clusters.
    int dev = 0, smem_limit = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return HAP_ECUDA;
    }
    LaunchShape sh{0, 0, 2, 0};
    for (int cs = 1; cs <= 16; cs *= 2) {
        const int64_t per = (ld / 4 + 2LL * cs - 1) / (2LL * cs);
        int T = (int)((per + 31) / 32 * 32);
        if (T < 32) T = 32;
        if (T > 512) continue;
        LaunchShape cand{T, cs, 2, 0};
        if (rowpass_smem_bytes(cand, L, s_dtype == HAP_S_BF16) > (size_t)smem_limit) continue;
        sh = cand;
        break;
    }
    if (!sh.T) return HAP_EUNSUPPORTED;
    int maxc = 0;
    if (rowpass_max_clusters(sh, L, s_dtype == HAP_S_BF16, &maxc) != cudaSuccess || maxc < 1) {
        cudaGetLastError();
        return HAP_EUNSUPPORTED;
    }
    int64_t G = maxc < kMaxClusters ? maxc : kMaxClusters;
    if (G > (N + 3) / 4) G = (N + 3) / 4;
    sh.G = (int)(G < 1 ? 1 : G);

#define NA_CU(x)                        \
    do {                                \
        if ((x) != cudaSuccess) {       \
            cudaGetLastError();         \
            return HAP_ECUDA;           \
        }                               \
    } while (0)

    // Calls share the scratch: clear the status word, and rebuild tau's column
    // part from the caller's rho (iteration t0 + 1 reads it when t0 >= 1).
    NA_CU(cudaMemsetAsync(status, 0, kStatusBytes, st));
    NA_CU(cudaMemsetAsync(phi + (int64_t)(L - 1) * ld, 0, (size_t)ld * sizeof(float), st));
    NA_CU(launch_fill_alpha_padding(A, (int64_t)L * N, N, ld, st));
    NA_CU(launch_prepare_from_R(R, sh.G, L, N, ld, rdiag, tpart, st));

    RowPassArgs a;
    a.A = A;
    a.R = R;
    a.S = S;
    a.N = N;
    a.ld = ld;
    a.s_level_stride = 0;
    a.L = L;
    a.pref = pref;
    a.c = c;
    a.tau = tau;
    a.phi = phi;
    a.tpart = tpart;
    a.b = b;
    a.rdiag = rdiag;
    a.partials = partials;
    a.status = status;
    a.lam = damping;
    a.oml = 1.0f - damping;
    for (int it = 0; it < n; ++it) {
        const int64_t t = t0 + it + 1;
        a.pending = it > 0 ? 1 : 0;
        a.update_c = (c_mode == HAP_C_PAPER && t >= 2) ? 1 : 0;
        a.use_tau = t >= 2 ? 1 : 0;
        NA_CU(launch_rowpass(a, sh, s_dtype == HAP_S_BF16, st));
        NA_CU(launch_colstats(partials, sh.G, L, N, ld, c, phi, rdiag, b, tpart, st));
    }
    if (n > 0) {
        apply_pending_alpha_kernel<<<(unsigned)((int64_t)L * N), 256, 0, st>>>(A, R, b, damping, 1.0f - damping, N, ld);
        NA_CU(cudaGetLastError());
    }
    unsigned host_status = 0;
    NA_CU(cudaMemcpyAsync(&host_status, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    NA_CU(cudaStreamSynchronize(st));
#undef NA_CU
    if (host_status & ST_TIMEOUT) return HAP_ETIMEOUT;
    if (host_status) return HAP_EDEVICE;
    return HAP_OK;
}

extern "C" size_t hap_noalloc_scratch_bytes(void) { return kScratchBytes; }
