// Host-side declarations shared by the translation units of libhap.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hap.h"

namespace hap {

// Status-word bits written by kernels (the host maps them to HAP_E* codes).
enum : unsigned {
    ST_TIMEOUT = 1u,  // a bounded wait gave up
    ST_BOUNDS = 2u,   // an index or alignment check failed
    ST_TMEM = 4u,     // tensor-memory allocation failed
};

// One launch of the fused row pass (one HAP iteration, all levels).
struct RowPassArgs {
    float* A;              // [L][N][ld] availabilities alpha (one step behind when pending)
    float* R;              // [L][N][ld] responsibilities rho
    const void* S;         // [Ls][N][ld] similarities (FP32 or BF16)
    int64_t N;
    int64_t ld;            // row stride of A, R, S and of every [L][ld] vector
    int64_t s_level_stride;  // elements between levels of S; 0 = shared by all levels
    int L;
    const float* pref;     // [L][ld]  preferences s_ii^l
    float* c;              // [L][ld]  cluster preference c (Eq. 2.6), in/out
    float* tau;            // [L][ld]  out: tau of this iteration (Eq. 2.4)
    float* phi;            // [L][ld]  out: phi of this iteration (Eq. 2.5); level L-1 stays 0
    const float* tpart;    // [L][ld]  rho^{l-1}_ii + P^{l-1}_i of the previous iteration (level >= 1)
    const float* b;        // [L][ld]  b_j = c_j + phi_j + rho_jj + P_j of the previous iteration
    float* rdiag;          // [L][ld]  out: rho_ii of this iteration
    float* partials;       // [G][L][ld] out: per-cluster column sums of max(0, rho) off the diagonal
    unsigned* status;      // device status word (ST_* bits)
    float lam, oml;        // damping lambda and 1 - lambda
    int pending;           // alpha of the previous iteration still to be applied
    int update_c;          // apply Eq. 2.6 this iteration
    int use_tau;           // tau from Eq. 2.4 this iteration (else +inf)
    const float* tau_in = nullptr;  // [L][ld] tau given per row (sequential level schedule), else computed
    float kappa = 0.f;     // Eq. 2.7 level-wise similarity update (0 = off; shared S only)
    uint64_t wait_ns = 2000000000ull;  // limit of every bounded wait of the row pass
    int debug = 0;         // 1: index checks that record ST_BOUNDS (see hap_options.debug_bounds)
    // Row band: A, R and S hold rows row0 .. row0 + nrows - 1 of an N-point
    // problem ([L][nrows][ld], [nrows][ld]); the [L][ld] vectors keep global
    // indices.  nrows = 0: every row (row0 = 0).  Bands take the band
    // instances of the kernel (no debug_bounds checks there).
    int64_t row0 = 0;
    int64_t nrows = 0;
};

struct LaunchShape {
    int T;   // threads per CTA
    int C;   // CTAs per cluster
    int K;   // float4 groups per thread and row (4*K columns)
    int G;   // clusters in the grid
    int tm;  // 1: column sums in tensor memory (TMEM), 0: in shared memory
    int nst; // TMA ring stages of the TMEM variant (2 or 4; the other has 3)
    int dual = 0;  // TMEM variant: 1 = two CTAs per SM (T <= 256 threads and <= 256
                   // TMEM columns each, so both allocations always fit)
};

// Kernel launchers (return a cudaError_t).
cudaError_t launch_rowpass(const RowPassArgs& a, const LaunchShape& sh, int s_bf16, cudaStream_t st);
// the same with the debug_bounds index checks compiled in (hap_rowpass_dbg.cu)
cudaError_t launch_rowpass_checked(const RowPassArgs& a, const LaunchShape& sh, int s_bf16, cudaStream_t st);
// the same over a band of rows (a.nrows > 0; hap_rowpass_band.cu)
cudaError_t launch_rowpass_band(const RowPassArgs& a, const LaunchShape& sh, int s_bf16, cudaStream_t st);
cudaError_t rowpass_max_clusters(const LaunchShape& sh, int L, int s_bf16, int* max_clusters);
cudaError_t rowpass_blocks_per_sm(const LaunchShape& sh, int L, int s_bf16, int* blocks);
size_t rowpass_smem_bytes(const LaunchShape& sh, int L, int s_bf16);
int rowpass_tmem_columns(const LaunchShape& sh, int L);  // 0 for shared-memory sums
cudaError_t launch_fill_alpha_padding(float* A, int64_t rows, int64_t N, int64_t ld, cudaStream_t st);

// tp_level (may be null) receives rho_jj + P_j at each level's own index.
cudaError_t launch_colstats(const float* partials, int G, int L, int64_t N, int64_t ld,
                            const float* c, const float* phi, const float* rdiag,
                            float* b, float* tpart, cudaStream_t st, float* tp_level = nullptr);

// Nearest neighbours with tensor-core first-pass distances (BF16 hi/lo split)
// and an exact FP32 re-rank of the M2 >= M best candidates per query row.
// Queries Q [Nq][d], candidates C [Nc][d] (global ids cid, null = index);
// a query never takes its own id.  d <= 64, M2 <= knn_tc_max_candidates().
// launches (may be null) is increased by the number of kernels launched.
int knn_tc_max_candidates();
cudaError_t launch_knn_tc(const float* Q, int64_t Nq, const float* C, const int32_t* cid, int64_t Nc, int64_t d, int M,
                          int M2, int32_t* idx, float* dist, cudaStream_t st, int64_t* launches = nullptr);

// One level of the sequential (Gauss-Seidel) schedule after its rho pass and
// column statistics: alpha^l (Eqs. 2.2-2.3, damped), then c^l (Eq. 2.6, when
// update_c), phi^{l-1} (Eq. 2.5, when phi_out) and tau^{l+1} = c^l + tp
// (Eq. 2.4, when tau_next).  A, R, S point at level l; vectors at level l.
struct GsArgs {
    float* A;
    const float* R;
    const void* S;
    const float* b;
    const float* pref;
    float* c;
    const float* tp;
    float* phi_out;
    float* tau_next;
    int64_t N, ld;
    float lam, oml;
    int update_c;
};
cudaError_t launch_gs_availability(const GsArgs& a, int s_bf16, cudaStream_t st);
cudaError_t launch_prepare_from_R(const float* R, int G, int L, int64_t N, int64_t ld,
                                  float* rdiag, float* tpart, cudaStream_t st);

// Row bands (hap_band_*).  band_summary: the band's exchange buffer
// xch [4][L][ld] = (P_j of the band's rows summed over its G cluster partials
// in the column-statistics order, then c, phi and rho_jj of the band's own
// rows j in [row0, row0 + nrows), zero elsewhere).
cudaError_t launch_band_summary(const float* partials, int G, int L, int64_t N, int64_t ld, const float* c,
                                const float* phi, const float* rdiag, int64_t row0, int64_t nrows, float* xch,
                                cudaStream_t st);
// band_columns: from every band's exchange buffer (xch_all [P][4][L][ld], in
// band order; band r owns rows [bounds[r], bounds[r+1])): P_j summed in band
// order, c, phi, rho_jj taken from the band that owns j; writes the full c,
// phi, rdiag vectors, b = c + phi + rho_jj + P and tau's column part.
constexpr int kMaxBands = 64;
struct BandBounds {
    int64_t lo[kMaxBands + 1];
};
cudaError_t launch_band_columns(const float* xch_all, int P, const BandBounds& bb, int L, int64_t N, int64_t ld,
                                float* c, float* phi, float* rdiag, float* b, float* tpart, cudaStream_t st);
// Launch shape of a context or band with nrows rows of an N-point problem;
// option checks shared by both.
int plan_shape(int64_t N, int64_t nrows, int L, const hap_options& o, LaunchShape* sh);
int check_options(const hap_options& o);

// nrows / row0 (band contexts): A, R and e hold rows row0 .. row0 + nrows - 1
// of the N-point problem; nrows = 0 means all N rows.
cudaError_t launch_exemplars(const float* A, const float* R, const float* b, int pending,
                             float lam, float oml, int64_t N, int64_t ld, int L,
                             int32_t* e, cudaStream_t st, int64_t nrows = 0, int64_t row0 = 0);
cudaError_t launch_materialize_A(float* dst, const float* A, const float* R, const float* b,
                                 int pending, float lam, float oml, int64_t N, int64_t ld, int L,
                                 cudaStream_t st, int64_t nrows = 0, int64_t row0 = 0);
// out: [2][L] counts, self-consistent points then exemplars per level
cudaError_t launch_acceptance(const int32_t* e, int64_t N, int L, long long* out, cudaStream_t st);
cudaError_t launch_netsim(const void* S, int s_bf16, int64_t s_level_stride, const float* pref,
                          const int32_t* e, int64_t N, int64_t ld, int L, double* ns,
                          cudaStream_t st);

// Sets ST_BOUNDS in *status if any off-diagonal s_ij (i != j, j < N) of the
// `levels` matrices ([levels][N][ld], level stride N*ld) is not finite.
cudaError_t launch_check_finite(const void* S, int s_bf16, int levels, int64_t N, int64_t ld, unsigned* status,
                                cudaStream_t st);
// nrows rows (0: N) of N similarities each
cudaError_t launch_copy_similarity(void* dst, int dst_bf16, int64_t ld, const void* src,
                                   int src_bf16, int64_t ld_src, int64_t N, cudaStream_t st, int64_t nrows = 0);
cudaError_t launch_read_similarity(float* dst, const void* S, int s_bf16, const float* pref_l,
                                   int64_t N, int64_t ld, cudaStream_t st);
cudaError_t launch_sbuild_f32(const float* X, int64_t N, int64_t d, void* S, int s_bf16,
                              int64_t ld, cudaStream_t st);
// tcgen05 build: scratch must hold 2 * N_pad * Kpad BF16 values plus N floats.
size_t sbuild_tc_scratch_bytes(int64_t N, int64_t d, int split);
cudaError_t launch_sbuild_tc(const float* X, int64_t N, int64_t d, int split, void* S, int s_bf16,
                             int64_t ld, void* scratch, unsigned* status, cudaStream_t st, int* kernels);

// ---- exclusive prefix sums and stable radix sort (hap_sort.cu) ----------
constexpr int kRadixBits = 9;  // digit of one radix pass
// tile sums scan_exclusive needs for n inputs
int64_t scan_tiles(int64_t n);
// out[i] = in[0] + ... + in[i-1]; tsum holds scan_tiles(n) values of scratch
cudaError_t scan_exclusive(const int* in, int64_t n, int* out, int64_t* tsum, cudaStream_t st);
cudaError_t scan_exclusive(const int* in, int64_t n, int64_t* out, int64_t* tsum, cudaStream_t st);
// histogram entries of one radix pass over n keys (hist and hoff each)
int64_t radix_hist_size(int64_t n);
// one stable pass on the 9-bit digit at `shift`: (key_in, val_in; null =
// position) -> (key_out, val_out); tsum holds scan_tiles(radix_hist_size(n))
cudaError_t radix_pass(const int32_t* key_in, const int32_t* val_in, int64_t n, int shift, int* hist, int* hoff,
                       int64_t* tsum, int32_t* key_out, int32_t* val_out, cudaStream_t st);
// stable sort of n keys in [0, 2^bits): key_out the sorted keys, perm[r] the
// input position of the r-th; scratch allocated and freed on the stream
cudaError_t stable_sort_keys(const int32_t* key, int64_t n, int bits, int32_t* key_out, int32_t* perm,
                             cudaStream_t st);

}  // namespace hap
