// Fused HAP row pass and column statistics (one iteration = two launches).
//
// Schedule of one iteration t (the data-parallel MR-HAP schedule of §3: every
// (i, l) is updated from the state at the start of the iteration):
//
//   row pass, per row i, levels l = 0..L-1 in order, by one thread-block
//   cluster that holds the whole row on chip (each CTA a contiguous slice of
//   columns, each thread 4*K columns):
//     1. alpha_{t-1} = damp(alpha_{t-2}, Eqs. 2.2/2.3 from b_{t-1}, rho_{t-1})
//        is applied on the fly and written back (availability is kept one
//        step behind so that A is read and written once per iteration);
//     2. m1, k1, m2 = max / lowest argmax / second max of alpha + s over the
//        row (Eq. 2.1's max_{k != j}), c = max(alpha + rho) (Eq. 2.6), and
//        phi^{l-1}_i = m1 (Eq. 2.5) - one exact warp/CTA/cluster reduction;
//     3. tau^l_i = c^{l-1}_i + rho^{l-1}_ii + P^{l-1}_i (Eq. 2.4) with
//        c^{l-1}_i from the previous level of the same row;
//     4. rho_t = damp(rho_{t-1}, s + min(tau, -max_{k != j})) (Eq. 2.1),
//        written back, and max(0, rho_t) accumulated per column in shared
//        memory for the rows this cluster owns (Eqs. 2.2-2.4 column sums).
//   column statistics, per (l, j): P_j = fixed-order sum of the per-cluster
//   partials, b_j = c_j + phi_j + rho_jj + P_j (used by the next row pass)
//   and rho_jj + P_j (tau of the next iteration).
//
// Every reduction is exact (max) or has a fixed order, so a run is bitwise
// reproducible.  When S is shared by all levels it is read once per row.
#include "hap_common.cuh"
#include "hap_internal.h"

namespace hap {

template <typename ST, int K, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) rowpass_kernel(const RowPassArgs p) {
    using SV = SVec<ST>;
    using raw_t = typename SV::raw;
    extern __shared__ float4 acc_s[];  // [L][K][T] per-thread column sums
    __shared__ float4 red[2][32];      // per-warp partial (m1, m2, c, k1), double-buffered
    __shared__ float4 cred[2];         // per-CTA partial, read by the cluster

    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    const unsigned C = cluster_nctarank(), rank = cluster_ctarank();
    const unsigned g = cluster_id_x(), G = cluster_count_x();
    const int L = p.L;
    const int64_t N = p.N, ld = p.ld;
    const float lam = p.lam, oml = p.oml;
    const bool pending = p.pending != 0;
    const bool s_each_level = p.s_level_stride != 0;
    const ST* Sb = reinterpret_cast<const ST*>(p.S);

    int64_t col[K];
    bool ok[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        col[k] = (int64_t)rank * (4LL * K * T) + 4LL * (k * T + tid);
        ok[k] = col[k] < ld;
    }
    for (int q = tid; q < L * K * T; q += T) acc_s[q] = make_float4(0.f, 0.f, 0.f, 0.f);

    const int64_t my_rows = N > (int64_t)g ? (N - 1 - (int64_t)g) / G + 1 : 0;
    const int64_t nsteps = my_rows * L;

    // Registers of the step being loaded (software pipeline depth 1).
    float4 na[K], nr[K], nb[K];
    raw_t ns[K];
    auto issue = [&](int64_t row, int l, bool load_s) {
        const int64_t off = ((int64_t)l * N + row) * ld;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (ok[k]) {
                na[k] = ld_stream(p.A + off + col[k]);
                nr[k] = ld_stream(p.R + off + col[k]);
                nb[k] = pending ? __ldg(reinterpret_cast<const float4*>(p.b + (int64_t)l * ld + col[k]))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                na[k] = nr[k] = nb[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        if (load_s) {
            const int64_t soff = (int64_t)l * p.s_level_stride + row * ld;
#pragma unroll
            for (int k = 0; k < K; ++k) ns[k] = ok[k] ? SV::load(Sb + soff + col[k]) : SV::zero();
        }
    };

    if (nsteps > 0) issue(g, 0, true);
    raw_t srow[K];
#pragma unroll
    for (int k = 0; k < K; ++k) srow[k] = SV::zero();
    float c_prev = 0.f;
    int64_t row = g;
    int l = 0;

    for (int64_t s = 0; s < nsteps; ++s) {
        float4 a[K], r[K], bb[K];
#pragma unroll
        for (int k = 0; k < K; ++k) { a[k] = na[k]; r[k] = nr[k]; bb[k] = nb[k]; }
        if (s_each_level || l == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) srow[k] = ns[k];
        }
        int64_t nrow = row;
        int nl = l + 1;
        if (nl == L) { nl = 0; nrow += G; }
        if (s + 1 < nsteps) issue(nrow, nl, s_each_level || nl == 0);

        const int64_t i = row;
        const int64_t off = ((int64_t)l * N + row) * ld;
        const int64_t voff = (int64_t)l * ld;
        const float pref_i = p.pref[voff + i];

        // ---- pass 1: pending availability, row statistics --------------------
        float m1 = -kInf, m2 = -kInf, cm = -kInf;
        int k1 = 0x7fffffff;
        float4 sv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float4 s4 = SV::to_f4(srow[k]);
            float4 an = a[k];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t j = col[k] + e;
                const bool diag = (j == i);
                const float sj = diag ? pref_i : f4_get(s4, e);
                f4_set(s4, e, sj);
                float aj = f4_get(a[k], e);
                const float rj = f4_get(r[k], e);
                if (pending) aj = damp(aj, avail_target(f4_get(bb[k], e), rj, diag), lam, oml);
                f4_set(an, e, aj);
                if (j < N) {
                    top2_push(__fadd_rn(aj, sj), (int)j, m1, k1, m2);
                    cm = fmaxf(cm, __fadd_rn(aj, rj));
                }
            }
            sv[k] = s4;
            if (pending && ok[k]) st_stream(p.A + off + col[k], an);
        }

        // ---- exact reduction: warp, CTA, cluster -----------------------------
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float o1 = __shfl_xor_sync(0xffffffffu, m1, o);
            const int ok1 = __shfl_xor_sync(0xffffffffu, k1, o);
            const float o2 = __shfl_xor_sync(0xffffffffu, m2, o);
            const float oc = __shfl_xor_sync(0xffffffffu, cm, o);
            top2_merge(m1, k1, m2, o1, ok1, o2);
            cm = fmaxf(cm, oc);
        }
        const int par = (int)(s & 1);
        if (lane == 0) red[par][warp] = make_float4(m1, m2, cm, __int_as_float(k1));
        __syncthreads();
        m1 = m2 = cm = -kInf;
        k1 = 0x7fffffff;
        for (int w = 0; w < nw; ++w) {
            const float4 v = red[par][w];
            top2_merge(m1, k1, m2, v.x, __float_as_int(v.w), v.y);
            cm = fmaxf(cm, v.z);
        }
        if (C > 1) {
            if (tid == 0) cred[par] = make_float4(m1, m2, cm, __int_as_float(k1));
            cluster_barrier();
            m1 = m2 = cm = -kInf;
            k1 = 0x7fffffff;
            const uint32_t base = smem_addr(&cred[par]);
            for (unsigned q = 0; q < C; ++q) {
                const float4 v = ld_dsmem_f4(map_to_rank(base, q));
                top2_merge(m1, k1, m2, v.x, __float_as_int(v.w), v.y);
                cm = fmaxf(cm, v.z);
            }
        }

        // ---- inter-level messages of (i, l) ----------------------------------
        const float cval = p.update_c ? cm : p.c[voff + i];
        const float tauv = (p.use_tau && l > 0) ? __fadd_rn(c_prev, p.tpart[voff + i]) : kInf;
        c_prev = cval;
        if (rank == 0 && tid == 0) {
            if (p.update_c) p.c[voff + i] = cval;
            p.tau[voff + i] = tauv;
            if (l > 0) p.phi[voff - ld + i] = m1;
        }

        // ---- pass 2: responsibilities and column sums ------------------------
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float4 rn4, add;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t j = col[k] + e;
                const float mx = (j == (int64_t)k1) ? m2 : m1;
                const float rh = __fadd_rn(f4_get(sv[k], e), fminf(tauv, -mx));
                const float rn = damp(f4_get(r[k], e), rh, lam, oml);
                f4_set(rn4, e, rn);
                if (j == i) p.rdiag[voff + i] = rn;
                f4_set(add, e, (j != i && j < N) ? fmaxf(rn, 0.f) : 0.f);
            }
            if (ok[k]) st_stream(p.R + off + col[k], rn4);
            float4& acc = acc_s[(l * K + k) * T + tid];
            acc.x = __fadd_rn(acc.x, add.x);
            acc.y = __fadd_rn(acc.y, add.y);
            acc.z = __fadd_rn(acc.z, add.z);
            acc.w = __fadd_rn(acc.w, add.w);
        }
        row = nrow;
        l = nl;
    }

    // ---- per-cluster column partials ------------------------------------------
    for (int ll = 0; ll < L; ++ll) {
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (ok[k])
                *reinterpret_cast<float4*>(p.partials + ((int64_t)g * L + ll) * ld + col[k]) =
                    acc_s[(ll * K + k) * T + tid];
    }
    // No CTA may leave while a peer can still read its shared memory.
    if (C > 1) cluster_barrier();
}

// P_j as the fixed-order sum of the cluster partials; b and tau's column part.
__global__ void colstats_kernel(const float* __restrict__ partials, int G, int L, int64_t N, int64_t ld,
                                const float* __restrict__ c, const float* __restrict__ phi,
                                const float* __restrict__ rdiag, float* __restrict__ b,
                                float* __restrict__ tpart) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)L * N) return;
    const int l = (int)(idx / N);
    const int64_t j = idx - (int64_t)l * N;
    const float* pp = partials + (int64_t)l * ld + j;
    const int64_t gstride = (int64_t)L * ld;
    float P = 0.f;
#pragma unroll 8
    for (int q = 0; q < G; ++q) P = __fadd_rn(P, pp[q * gstride]);
    const int64_t v = (int64_t)l * ld + j;
    const float rd = rdiag[v];
    b[v] = __fadd_rn(__fadd_rn(__fadd_rn(c[v], phi[v]), rd), P);
    if (l + 1 < L) tpart[v + ld] = __fadd_rn(rd, P);
}

// The same column statistics recomputed from a stored rho (after the state is
// replaced), summing rows in exactly the order the row pass uses: cluster q
// owns rows q, q+G, q+2G, ... and its partial is summed over q in order.
__global__ void prepare_from_R_kernel(const float* __restrict__ R, int G, int L, int64_t N, int64_t ld,
                                      float* __restrict__ rdiag, float* __restrict__ tpart) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)L * N) return;
    const int l = (int)(idx / N);
    const int64_t j = idx - (int64_t)l * N;
    const float* Rl = R + (int64_t)l * N * ld;
    float P = 0.f;
    for (int q = 0; q < G; ++q) {
        float acc = 0.f;
        for (int64_t i = q; i < N; i += G) {
            const float rv = Rl[i * ld + j];
            acc = __fadd_rn(acc, (i != j) ? fmaxf(rv, 0.f) : 0.f);
        }
        P = __fadd_rn(P, acc);
    }
    const float rd = Rl[j * ld + j];
    rdiag[(int64_t)l * ld + j] = rd;
    if (l + 1 < L) tpart[(int64_t)(l + 1) * ld + j] = __fadd_rn(rd, P);
}

// ---------------------------------------------------------------------------
template <typename ST, int K, int MAXT>
static cudaError_t launch_one(const RowPassArgs& a, const LaunchShape& sh, cudaStream_t st) {
    auto kern = rowpass_kernel<ST, K, MAXT>;
    const size_t smem = rowpass_smem_bytes(sh, a.L);
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    if (sh.C > 8) {
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (err != cudaSuccess) return err;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(sh.G * sh.C), 1, 1);
    cfg.blockDim = dim3((unsigned)sh.T, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)sh.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <typename ST, int K, int MAXT>
static cudaError_t max_clusters_one(const LaunchShape& sh, int L, int* out) {
    auto kern = rowpass_kernel<ST, K, MAXT>;
    const size_t smem = rowpass_smem_bytes(sh, L);
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    if (sh.C > 8) {
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (err != cudaSuccess) return err;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)sh.C, 1, 1);
    cfg.blockDim = dim3((unsigned)sh.T, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)sh.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(out, kern, &cfg);
}

size_t rowpass_smem_bytes(const LaunchShape& sh, int L) {
    return (size_t)L * sh.K * sh.T * sizeof(float4);
}

#define HAP_ROWPASS_DISPATCH(FN, ...)                                               \
    do {                                                                            \
        if (s_bf16) {                                                               \
            if (sh.K == 1) return FN<__nv_bfloat16, 1, 1024>(__VA_ARGS__);          \
            if (sh.K == 2) return FN<__nv_bfloat16, 2, 512>(__VA_ARGS__);           \
            if (sh.K == 4) return FN<__nv_bfloat16, 4, 256>(__VA_ARGS__);           \
        } else {                                                                    \
            if (sh.K == 1) return FN<float, 1, 1024>(__VA_ARGS__);                  \
            if (sh.K == 2) return FN<float, 2, 512>(__VA_ARGS__);                   \
            if (sh.K == 4) return FN<float, 4, 256>(__VA_ARGS__);                   \
        }                                                                           \
        return cudaErrorInvalidValue;                                               \
    } while (0)

cudaError_t launch_rowpass(const RowPassArgs& a, const LaunchShape& sh, int s_bf16, cudaStream_t st) {
    HAP_ROWPASS_DISPATCH(launch_one, a, sh, st);
}

cudaError_t rowpass_max_clusters(const LaunchShape& sh, int L, int s_bf16, int* max_clusters) {
    HAP_ROWPASS_DISPATCH(max_clusters_one, sh, L, max_clusters);
}

cudaError_t launch_colstats(const float* partials, int G, int L, int64_t N, int64_t ld,
                            const float* c, const float* phi, const float* rdiag,
                            float* b, float* tpart, cudaStream_t st) {
    const int64_t total = (int64_t)L * N;
    const int threads = 256;
    const unsigned blocks = (unsigned)((total + threads - 1) / threads);
    colstats_kernel<<<blocks, threads, 0, st>>>(partials, G, L, N, ld, c, phi, rdiag, b, tpart);
    return cudaGetLastError();
}

cudaError_t launch_prepare_from_R(const float* R, int G, int L, int64_t N, int64_t ld,
                                  float* rdiag, float* tpart, cudaStream_t st) {
    const int64_t total = (int64_t)L * N;
    const int threads = 128;
    const unsigned blocks = (unsigned)((total + threads - 1) / threads);
    prepare_from_R_kernel<<<blocks, threads, 0, st>>>(R, G, L, N, ld, rdiag, tpart);
    return cudaGetLastError();
}

}  // namespace hap
