// Fused HAP row pass and column statistics (one iteration = two launches).
//
// Schedule of one iteration t (the data-parallel MR-HAP schedule of §3: every
// (i, l) is updated from the state at the start of the iteration):
//
//   row pass, per row i, levels l = 0..L-1 in order, by one thread-block
//   cluster that holds the whole row on chip (each CTA a contiguous slice of
//   columns, each thread 4*K columns; every thread keeps the column sums of
//   its columns for all levels, in shared memory or, in the TMEM variant, in
//   tensor memory so that shared memory holds only the TMA ring):
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
//
// Bounded waits.  Every wait (ring stage, cluster exchange) gives up after
// RowPassArgs::wait_ns and records ST_TIMEOUT.  A warp in which any thread
// gave up leaves the step loop at once (the decision is warp-uniform, so
// every warp-collective instruction still sees a converged warp); its
// missing exchange messages then make every other warp of the cluster give
// up within one more limit.  The ring is refilled only by the issuing thread
// after its own wait on that stage succeeded, so each stage has at most one
// copy in flight; after the loop that thread waits (bounded) for every copy
// it issued and did not consume, so no bulk copy lands in the shared memory
// of a CTA that has left.  The CTA (and, for clusters, the cluster) then
// meets at one barrier before it frees tensor memory and exits, which orders
// every exchange store into its shared memory before the exit.
#include "hap_rowpass_kernel.cuh"

namespace hap {

// Columns j in [N, ld) of alpha hold -inf so that padding never wins the row
// maxima of alpha + s and alpha + rho (no per-element masks in the row pass).
__global__ void fill_alpha_padding_kernel(float* A, int64_t rows, int64_t N, int64_t ld) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
    if (r >= rows) return;
    for (int64_t j = N + threadIdx.x; j < ld; j += blockDim.x) A[r * ld + j] = -kInf;
}

// Fixed summation order of P_j over the G cluster partials: kChunks
// contiguous ranges of clusters [q_lo(w), q_lo(w+1)), each summed in cluster
// order, then the range sums folded in range order.  colstats_kernel and
// prepare_from_R_kernel both follow it, so P (and everything after it) has
// the same bits whether it comes from the row pass or from a stored rho.
constexpr int kChunks = 8;
HAP_DEV int chunk_lo(int w, int G) { return (int)(((int64_t)w * G) / kChunks); }

// P_j from the cluster partials; b and tau's column part.  Block (32, kChunks):
// x picks one of 32 consecutive (l, j), y one range of clusters.
__global__ void __launch_bounds__(32 * kChunks) colstats_kernel(
    const float* __restrict__ partials, int G, int L, int64_t N, int64_t ld, const float* __restrict__ c,
    const float* __restrict__ phi, const float* __restrict__ rdiag, float* __restrict__ b,
    float* __restrict__ tpart, float* __restrict__ tp_level) {
    __shared__ float red[kChunks][32];
    const int x = threadIdx.x, w = threadIdx.y;
    const int64_t idx = (int64_t)blockIdx.x * 32 + x;
    const bool valid = idx < (int64_t)L * N;
    const int l = valid ? (int)(idx / N) : 0;
    const int64_t j = valid ? idx - (int64_t)l * N : 0;
    float acc = 0.f;
    if (valid) {
        const float* pp = partials + (int64_t)l * ld + j;
        const int64_t gstride = (int64_t)L * ld;
        const int q1 = chunk_lo(w + 1, G);
#pragma unroll 4
        for (int q = chunk_lo(w, G); q < q1; ++q) acc = __fadd_rn(acc, pp[q * gstride]);
    }
    red[w][x] = acc;
    __syncthreads();
    if (w != 0 || !valid) return;
    float P = red[0][x];
#pragma unroll
    for (int u = 1; u < kChunks; ++u) P = __fadd_rn(P, red[u][x]);
    const int64_t v = (int64_t)l * ld + j;
    const float rd = rdiag[v];
    b[v] = __fadd_rn(__fadd_rn(__fadd_rn(c[v], phi[v]), rd), P);
    if (l + 1 < L) tpart[v + ld] = __fadd_rn(rd, P);
    if (tp_level) tp_level[v] = __fadd_rn(rd, P);
}

// The same column statistics recomputed from a stored rho (after the state is
// replaced), summing rows in exactly the order the row pass and
// colstats_kernel use: cluster q owns rows q, q+G, q+2G, ... and its sum is
// folded into P in the chunked cluster order above.
__global__ void prepare_from_R_kernel(const float* __restrict__ R, int G, int L, int64_t N, int64_t ld,
                                      float* __restrict__ rdiag, float* __restrict__ tpart) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)L * N) return;
    const int l = (int)(idx / N);
    const int64_t j = idx - (int64_t)l * N;
    const float* Rl = R + (int64_t)l * N * ld;
    float P = 0.f;
    for (int w = 0; w < kChunks; ++w) {
        float part = 0.f;
        for (int q = chunk_lo(w, G); q < chunk_lo(w + 1, G); ++q) {
            float acc = 0.f;
            for (int64_t i = q; i < N; i += G) {
                const float rv = Rl[i * ld + j];
                acc = __fadd_rn(acc, (i != j) ? fmaxf(rv, 0.f) : 0.f);
            }
            part = __fadd_rn(part, acc);
        }
        P = w == 0 ? part : __fadd_rn(P, part);
    }
    const float rd = Rl[j * ld + j];
    rdiag[(int64_t)l * ld + j] = rd;
    if (l + 1 < L) tpart[(int64_t)(l + 1) * ld + j] = __fadd_rn(rd, P);
}

// Row bands.  The column statistics of a row-partitioned problem (§3: the
// availability job keys its messages by column, so it needs every row's
// responsibilities of that column) are exchanged once per iteration: each band
// contributes its rows' part of P_j, summed over its cluster partials in the
// order colstats_kernel uses, and the c, phi and rho_jj of the rows it owns.
__global__ void __launch_bounds__(32 * kChunks) band_summary_kernel(
    const float* __restrict__ partials, int G, int L, int64_t N, int64_t ld, const float* __restrict__ c,
    const float* __restrict__ phi, const float* __restrict__ rdiag, int64_t row0, int64_t nrows,
    float* __restrict__ xch) {
    __shared__ float red[kChunks][32];
    const int x = threadIdx.x, w = threadIdx.y;
    const int64_t idx = (int64_t)blockIdx.x * 32 + x;
    const bool valid = idx < (int64_t)L * N;
    const int l = valid ? (int)(idx / N) : 0;
    const int64_t j = valid ? idx - (int64_t)l * N : 0;
    float acc = 0.f;
    if (valid) {
        const float* pp = partials + (int64_t)l * ld + j;
        const int64_t gstride = (int64_t)L * ld;
        const int q1 = chunk_lo(w + 1, G);
        for (int q = chunk_lo(w, G); q < q1; ++q) acc = __fadd_rn(acc, pp[q * gstride]);
    }
    red[w][x] = acc;
    __syncthreads();
    if (w != 0 || !valid) return;
    float P = red[0][x];
#pragma unroll
    for (int u = 1; u < kChunks; ++u) P = __fadd_rn(P, red[u][x]);
    const int64_t v = (int64_t)l * ld + j, part = (int64_t)L * ld;
    const bool own = j >= row0 && j < row0 + nrows;
    xch[v] = P;
    xch[part + v] = own ? c[v] : 0.f;
    xch[2 * part + v] = own ? phi[v] : 0.f;
    xch[3 * part + v] = own ? rdiag[v] : 0.f;
}

// Every band's exchange buffer in, the column statistics of the whole problem
// out: P_j summed in band order (the same bits on every band), c, phi and
// rho_jj from the band owning column j; b and tau's column part as in
// colstats_kernel.
__global__ void band_columns_kernel(const float* __restrict__ xch_all, int P, const BandBounds bb, int L,
                                    int64_t N, int64_t ld, float* __restrict__ c, float* __restrict__ phi,
                                    float* __restrict__ rdiag, float* __restrict__ b, float* __restrict__ tpart) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)L * N) return;
    const int l = (int)(idx / N);
    const int64_t j = idx - (int64_t)l * N;
    const int64_t v = (int64_t)l * ld + j, part = (int64_t)L * ld, band = 4 * part;
    float Ps = xch_all[v];
    for (int r = 1; r < P; ++r) Ps = __fadd_rn(Ps, xch_all[r * band + v]);
    int o = 0;
    while (o + 1 < P && j >= bb.lo[o + 1]) ++o;
    const float* own = xch_all + o * band;
    const float cv = own[part + v], ph = own[2 * part + v], rd = own[3 * part + v];
    c[v] = cv;
    phi[v] = ph;
    rdiag[v] = rd;
    b[v] = __fadd_rn(__fadd_rn(__fadd_rn(cv, ph), rd), Ps);
    if (l + 1 < L) tpart[v + ld] = __fadd_rn(rd, Ps);
}

template <typename ST, int K, int MAXT, int NST, bool TM>
static cudaError_t max_clusters_one(const LaunchShape& sh, int L, int* out) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cudaError_t err = cluster_config<ST, K, MAXT, NST, TM, false>(sh, L, &cfg, attr);
    if (err != cudaSuccess) return err;
    cfg.gridDim = dim3((unsigned)sh.C, 1, 1);
    return cudaOccupancyMaxActiveClusters(out, rowpass_kernel<ST, K, MAXT, NST, TM, false>, &cfg);
}

template <typename ST, int K, int MAXT, int NST, bool TM>
static cudaError_t blocks_per_sm_one(const LaunchShape& sh, int L, int* out) {
    auto kern = rowpass_kernel<ST, K, MAXT, NST, TM, false>;
    const size_t smem = rowpass_smem_bytes(sh, L, sizeof(ST) == 2);
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kern, sh.T, smem);
}

// The TMEM variant bounds how many of its CTAs share an SM through its
// shared-memory request, so that their TMEM allocations always fit together
// and an allocation never waits for another row-pass CTA (which could itself
// be waiting for a cluster peer blocked in allocation): more than half of an
// SM's 228 KB keeps one CTA per SM (at most 512 columns); more than a third
// keeps two (the dual shape, at most 256 columns each).
constexpr size_t kTmemMinSmem = 116 * 1024;
constexpr size_t kTmemDualMinSmem = 80 * 1024;

size_t rowpass_smem_bytes(const LaunchShape& sh, int L, int s_bf16) {
    const int nst = sh.tm ? sh.nst : kStages;
    const size_t bytes = rowpass_smem_layout(sh.T, sh.K, sh.C, L, s_bf16 ? 2 : 4, nst, sh.tm != 0, nullptr, nullptr);
    if (!sh.tm) return bytes;
    const size_t lo = sh.dual ? kTmemDualMinSmem : kTmemMinSmem;
    return bytes < lo ? lo : bytes;
}

int rowpass_tmem_columns(const LaunchShape& sh, int L) { return sh.tm ? rowpass_tmem_cols(sh.T, sh.K, L) : 0; }

cudaError_t launch_fill_alpha_padding(float* A, int64_t rows, int64_t N, int64_t ld, cudaStream_t st) {
    if (ld == N) return cudaSuccess;
    const dim3 block(32, 8);
    fill_alpha_padding_kernel<<<(unsigned)((rows + 7) / 8), block, 0, st>>>(A, rows, N, ld);
    return cudaGetLastError();
}

cudaError_t launch_rowpass(const RowPassArgs& a, const LaunchShape& sh, int s_bf16, cudaStream_t st) {
    if (a.nrows) return launch_rowpass_band(a, sh, s_bf16, st);
    if (a.debug) return launch_rowpass_checked(a, sh, s_bf16, st);
    HAP_ROWPASS_DISPATCH(launch_plain, a, sh, st);
}

cudaError_t rowpass_max_clusters(const LaunchShape& sh, int L, int s_bf16, int* max_clusters) {
    HAP_ROWPASS_DISPATCH(max_clusters_one, sh, L, max_clusters);
}

cudaError_t rowpass_blocks_per_sm(const LaunchShape& sh, int L, int s_bf16, int* blocks) {
    HAP_ROWPASS_DISPATCH(blocks_per_sm_one, sh, L, blocks);
}

cudaError_t launch_colstats(const float* partials, int G, int L, int64_t N, int64_t ld,
                            const float* c, const float* phi, const float* rdiag,
                            float* b, float* tpart, cudaStream_t st, float* tp_level) {
    const int64_t total = (int64_t)L * N;
    const unsigned blocks = (unsigned)((total + 31) / 32);
    colstats_kernel<<<blocks, dim3(32, kChunks), 0, st>>>(partials, G, L, N, ld, c, phi, rdiag, b, tpart, tp_level);
    return cudaGetLastError();
}

cudaError_t launch_band_summary(const float* partials, int G, int L, int64_t N, int64_t ld, const float* c,
                                const float* phi, const float* rdiag, int64_t row0, int64_t nrows, float* xch,
                                cudaStream_t st) {
    const int64_t total = (int64_t)L * N;
    const unsigned blocks = (unsigned)((total + 31) / 32);
    band_summary_kernel<<<blocks, dim3(32, kChunks), 0, st>>>(partials, G, L, N, ld, c, phi, rdiag, row0, nrows, xch);
    return cudaGetLastError();
}

cudaError_t launch_band_columns(const float* xch_all, int P, const BandBounds& bb, int L, int64_t N, int64_t ld,
                                float* c, float* phi, float* rdiag, float* b, float* tpart, cudaStream_t st) {
    const int64_t total = (int64_t)L * N;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    band_columns_kernel<<<blocks, 256, 0, st>>>(xch_all, P, bb, L, N, ld, c, phi, rdiag, b, tpart);
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
