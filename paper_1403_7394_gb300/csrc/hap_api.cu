// C ABI of libhap: context, workspace carve-up, launch-shape selection and the
// per-iteration launch sequence.  See include/hap.h for the contract.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "hap.h"
#include "hap_internal.h"

using namespace hap;

struct hap_ctx {
    int64_t N = 0;
    int L = 0;
    int64_t ld = 0;
    hap_options opt{};
    float lam = 0.5f;
    cudaStream_t stream = nullptr;
    int device = 0;

    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;

    float* A = nullptr;
    float* R = nullptr;
    void* S = nullptr;
    float *pref = nullptr, *c = nullptr, *c0 = nullptr, *tau = nullptr, *phi = nullptr;
    float *tpart = nullptr, *b = nullptr, *rdiag = nullptr, *partials = nullptr;
    int32_t* e = nullptr;
    double* ns = nullptr;
    long long* acc = nullptr;
    unsigned* status = nullptr;
    int64_t s_level_stride = 0;
    int s_levels = 1;

    LaunchShape sh{};
    int64_t launches = 0;  // kernels launched by this context
    int64_t iter = 0;
    bool pending = false;
    bool e_valid = false;  // e holds Eq. 2.8 of the current messages

    std::vector<cudaEvent_t> ev;  // pairs (start, stop) of timed row-pass launches
    double prof_ms = 0.0;
    int64_t prof_n = 0;
};

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t A, R, xs, S, pref, c, c0, tau, phi, tpart, b, rdiag, partials, e, ns, acc, status, total;
};

// d up to which the tensor-core build always finds operand scratch in the
// alpha and rho storage plus a reserve placed right after rho
constexpr int64_t kBuildMaxD = 256;

int64_t padded_ld(int64_t N) { return (N + 31) / 32 * 32; }

// Largest shared-memory request of which two CTAs fit on one SM (228 KB per
// SM, 1 KB of it reserved per CTA).
constexpr size_t kDualSmemMax = 113 * 1024;

// Row-pass launch shape: one cluster holds a whole row (C CTAs x T threads x
// 4K columns >= ld); then as many clusters as can be resident at once
// (persistent grid).  shape_for gives, for one column-sum variant, the fewest
// CTAs per cluster (1, 2, 4, 8, 16, or o.cluster_size) whose T threads x 4K
// columns cover the row and whose shared memory fits.  dual = 1 asks for the
// TMEM variant with two CTAs per SM (T <= 256 and <= 256 TMEM columns per
// CTA); it fails where that is not possible.
int shape_for(int64_t ld, int L, const hap_options& o, int tm, int K, int dual, int smem_limit, LaunchShape* out) {
    const int64_t q4 = ld / 4;  // float4 columns
    const int maxT = tm ? (dual ? 256 : 512) : (K == 1 ? 1024 : K == 2 ? 512 : 256);
    const int s_bf16 = o.s_dtype == HAP_S_BF16;
    const int sizes[5] = {1, 2, 4, 8, 16};
    if (dual && !tm) return HAP_EINVAL;
    for (int c : sizes) {
        if (o.cluster_size && c != o.cluster_size) continue;
        int T = o.block_threads;
        const int quantum = tm ? 128 : 32;  // TMEM: whole lane quarters per warp group
        if (T == 0) {
            const int64_t per = (q4 + (int64_t)c * K - 1) / ((int64_t)c * K);
            T = (int)((per + quantum - 1) / quantum * quantum);
            if (T < quantum) T = quantum;
            if (T > maxT) continue;
        } else if (T < quantum || T > maxT || T % quantum) {
            return HAP_EINVAL;
        }
        if ((int64_t)c * T * K * 4 < ld) continue;
        LaunchShape sh{T, c, K, 0, tm, tm ? 4 : 0};
        if (dual) {
            // two CTAs of at most 256 threads per SM: the threads of one
            // 512-thread CTA, half the row per CTA, twice the clusters
            sh.nst = 2;
            sh.dual = 1;
            if (rowpass_tmem_columns(sh, L) > 256 || rowpass_smem_bytes(sh, L, s_bf16) > kDualSmemMax)
                return HAP_EUNSUPPORTED;
            *out = sh;
            return HAP_OK;
        }
        if (tm && rowpass_smem_bytes(sh, L, s_bf16) > (size_t)smem_limit) sh.nst = 2;
        if (rowpass_smem_bytes(sh, L, s_bf16) > (size_t)smem_limit) continue;
        if (tm && rowpass_tmem_columns(sh, L) > 512) return HAP_EUNSUPPORTED;
        *out = sh;
        return HAP_OK;
    }
    return HAP_EUNSUPPORTED;
}

int choose_shape(int64_t N, int L, const hap_options& o, LaunchShape* out) {
    const int64_t ld = padded_ld(N);
    if (o.cluster_size < 0 || o.cluster_size > 16) return HAP_EINVAL;
    if (o.col_sums < HAP_COLSUM_AUTO || o.col_sums > HAP_COLSUM_TMEM) return HAP_EINVAL;
    int dev = 0, smem_limit = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return HAP_ECUDA;
    }
    const bool explicit_shape = o.elems_per_thread || o.block_threads || o.cluster_size;
    const int mode = o.col_sums != HAP_COLSUM_AUTO ? o.col_sums
                     : o.ctas_per_sm == 2               ? HAP_COLSUM_TMEM
                     : explicit_shape                   ? HAP_COLSUM_SMEM
                                                        : HAP_COLSUM_AUTO;
    // 8 columns per thread by default with shared-memory sums (enough work per
    // step to amortise the per-row reduction, few enough registers for
    // 512-thread CTAs); 16 with TMEM sums (twice the row per cluster).
    auto K_of = [&](int tm, int* K) {
        *K = o.elems_per_thread ? o.elems_per_thread / 4 : (tm ? 4 : 2);
        if (o.elems_per_thread && o.elems_per_thread != 4 * *K) return HAP_EINVAL;
        if (tm ? (*K != 2 && *K != 4) : (*K != 1 && *K != 2 && *K != 4)) return HAP_EINVAL;
        return HAP_OK;
    };
    if (o.ctas_per_sm < 0 || o.ctas_per_sm > 2) return HAP_EINVAL;
    if (o.ctas_per_sm == 2 && mode == HAP_COLSUM_SMEM) return HAP_EINVAL;
    if (mode != HAP_COLSUM_AUTO || o.ctas_per_sm) {
        const int tm = mode == HAP_COLSUM_SMEM ? 0 : 1;
        int K = 0, rc = K_of(tm, &K);
        if (rc) return rc;
        return shape_for(ld, L, o, tm, K, o.ctas_per_sm == 2, smem_limit, out);
    }
    // automatic: among both variants, every cluster size that holds the row
    // with no CTA left without columns, and one or two CTAs per SM, the shape
    // whose co-resident clusters cover the most SMs (clusters are placed
    // within a GPC, so a size may leave SMs idle: on GB300 four 512-thread
    // CTAs per cluster place 36 clusters on 144 of 152 SMs, and clusters of
    // eight place 15 whether or not two CTAs could share an SM); on a tie the
    // one with fewer CTAs per cluster (a cheaper row exchange), then two CTAs
    // per SM (more threads on each SM), then TMEM sums (16 columns per thread;
    // measured faster on GB300)
    LaunchShape best{};
    int64_t best_sms = -1;
    for (int tm = 1; tm >= 0; --tm) {
        int K = 0;
        if (K_of(tm, &K)) continue;
        for (int c : {1, 2, 4, 8, 16})
        for (int dual = 0; dual <= tm; ++dual) {
            hap_options oc = o;
            oc.cluster_size = c;
            LaunchShape sh{};
            if (shape_for(ld, L, oc, tm, K, dual, smem_limit, &sh) != HAP_OK) continue;
            // every CTA of the cluster must hold columns of the row
            if ((int64_t)(sh.C - 1) * sh.T * sh.K * 4 >= ld) continue;
            int maxc = 0, per_sm = 0;
            if (rowpass_max_clusters(sh, L, o.s_dtype == HAP_S_BF16, &maxc) != cudaSuccess ||
                rowpass_blocks_per_sm(sh, L, o.s_dtype == HAP_S_BF16, &per_sm) != cudaSuccess) {
                cudaGetLastError();
                return HAP_ECUDA;
            }
            if (maxc < 1 || per_sm < 1) continue;
            // SMs the co-resident CTAs occupy (several may share one SM)
            const int64_t ctas = (int64_t)std::min<int64_t>(maxc, (N + 3) / 4) * sh.C;
            const int64_t sms = std::min<int64_t>(n_sm, (ctas + per_sm - 1) / per_sm);
            if (sms > best_sms || (sms == best_sms && sh.C < best.C) ||
                (sms == best_sms && sh.C == best.C && sh.dual && !best.dual)) {
                best = sh;
                best_sms = sms;
            }
        }
    }
    if (best_sms <= 0) return HAP_EUNSUPPORTED;
    *out = best;
    return HAP_OK;
}

int finish_shape(int64_t N, int L, const hap_options& o, LaunchShape* sh) {
    int maxc = 0;
    cudaError_t err = rowpass_max_clusters(*sh, L, o.s_dtype == HAP_S_BF16, &maxc);
    if (err != cudaSuccess) { cudaGetLastError(); return HAP_ECUDA; }
    if (maxc < 1) return HAP_EUNSUPPORTED;
    int64_t G = o.grid_clusters ? o.grid_clusters : maxc;
    // keep a few rows per cluster on small problems (fewer partials to sum)
    const int64_t cap = o.grid_clusters ? N : (N + 3) / 4;
    if (G > cap) G = cap;
    if (G < 1) G = 1;
    sh->G = (int)G;
    return HAP_OK;
}

Layout make_layout(int64_t N, int L, const hap_options& o, const LaunchShape& sh) {
    const int64_t ld = padded_ld(N);
    const size_t mat = (size_t)L * N * ld * sizeof(float);
    const size_t s_elem = o.s_dtype == HAP_S_BF16 ? 2 : 4;
    const int s_levels = o.s_per_level ? L : 1;
    const size_t vec = (size_t)L * ld * sizeof(float);
    Layout y{};
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = align_up(off + bytes); return at; };
    y.A = take(mat);
    y.R = take(mat);
    const size_t need = sbuild_tc_scratch_bytes(N, kBuildMaxD, 1), have = align_up(mat) + mat;
    y.xs = take(need > have ? need - have : 0);
    y.S = take((size_t)s_levels * N * ld * s_elem);
    y.pref = take(vec);
    y.c = take(vec);
    y.c0 = take(vec);
    y.tau = take(vec);
    y.phi = take(vec);
    y.tpart = take(vec);
    y.b = take(vec);
    y.rdiag = take(vec);
    y.partials = take((size_t)sh.G * L * ld * sizeof(float));
    y.e = take((size_t)L * N * sizeof(int32_t));
    y.ns = take((size_t)L * sizeof(double));
    y.acc = take((size_t)2 * L * sizeof(long long));
    y.status = take(4 * sizeof(unsigned));
    y.total = off;
    return y;
}

int check_opts(const hap_options& o) {
    if (o.c_mode != HAP_C_PAPER && o.c_mode != HAP_C_FIXED) return HAP_EINVAL;
    if (o.schedule != HAP_SCHED_JACOBI && o.schedule != HAP_SCHED_GAUSS_SEIDEL) return HAP_EINVAL;
    if (!(o.kappa >= 0.f && o.kappa <= 1.f)) return HAP_EINVAL;
    if (o.kappa != 0.f && (o.schedule != HAP_SCHED_JACOBI || o.s_per_level)) return HAP_EUNSUPPORTED;
    if (o.s_dtype != HAP_S_F32 && o.s_dtype != HAP_S_BF16) return HAP_EINVAL;
    if (o.s_per_level != 0 && o.s_per_level != 1) return HAP_EINVAL;
    if (o.wait_limit_ns < 0 || (o.debug_bounds != 0 && o.debug_bounds != 1)) return HAP_EINVAL;
    return HAP_OK;
}

uint64_t wait_limit(const hap_options& o) {
    return o.wait_limit_ns > 0 ? (uint64_t)o.wait_limit_ns : 2000000000ull;
}

int plan(int64_t N, int L, const hap_options& o, LaunchShape* sh, Layout* y) {
    if (N < 2 || L < 1 || L > 16) return HAP_EINVAL;
    if (N > 65536) return HAP_EUNSUPPORTED;
    int rc = check_opts(o);
    if (rc) return rc;
    rc = choose_shape(N, L, o, sh);
    if (rc) return rc;
    rc = finish_shape(N, L, o, sh);
    if (rc) return rc;
    *y = make_layout(N, L, o, *sh);
    return HAP_OK;
}

}  // namespace

// The row width fixes the shape (one cluster per row); the rows held only cap
// the grid.
int hap::plan_shape(int64_t N, int64_t nrows, int L, const hap_options& o, LaunchShape* sh) {
    if (N < 2 || L < 1 || L > 16 || nrows < 1 || nrows > N) return HAP_EINVAL;
    if (N > 65536) return HAP_EUNSUPPORTED;
    int rc = check_opts(o);
    if (rc) return rc;
    rc = choose_shape(N, L, o, sh);
    if (rc) return rc;
    return finish_shape(nrows, L, o, sh);
}

int hap::check_options(const hap_options& o) { return check_opts(o); }

namespace {

#define CU(x)                                        \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ != cudaSuccess) {                     \
            cudaGetLastError();                      \
            return HAP_ECUDA;                        \
        }                                            \
    } while (0)

// Messages back to Algorithm 1's initial values: alpha = rho = 0, tau = +inf,
// phi = 0, c = c0; clears a reported device error.
int reset_messages(hap_ctx* h) {
    const size_t mat = (size_t)h->L * h->N * h->ld * sizeof(float);
    const size_t vec = (size_t)h->L * h->ld * sizeof(float);
    CU(cudaMemsetAsync(h->status, 0, 4 * sizeof(unsigned), h->stream));
    CU(cudaMemsetAsync(h->A, 0, mat, h->stream));
    CU(launch_fill_alpha_padding(h->A, (int64_t)h->L * h->N, h->N, h->ld, h->stream));
    CU(cudaMemsetAsync(h->R, 0, mat, h->stream));
    CU(cudaMemcpyAsync(h->c, h->c0, vec, cudaMemcpyDeviceToDevice, h->stream));
    CU(cudaMemsetAsync(h->phi, 0, vec, h->stream));
    CU(cudaMemsetAsync(h->tpart, 0, vec, h->stream));
    CU(cudaMemsetAsync(h->b, 0, vec, h->stream));
    CU(cudaMemsetAsync(h->rdiag, 0, vec, h->stream));
    std::vector<float> inf((size_t)h->L * h->ld, __builtin_inff());
    CU(cudaMemcpyAsync(h->tau, inf.data(), vec, cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    h->iter = 0;
    h->pending = false;
    h->e_valid = false;
    return HAP_OK;
}

// Eq. 2.8 of the current messages into h->e, once per change of the messages.
int ensure_exemplars(hap_ctx* h) {
    if (h->e_valid) return HAP_OK;
    CU(launch_exemplars(h->A, h->R, h->b, h->pending, h->lam, 1.0f - h->lam, h->N, h->ld, h->L, h->e, h->stream));
    h->launches += 1;
    h->e_valid = true;
    return HAP_OK;
}

// debug_bounds: every off-diagonal similarity finite, else HAP_EINVAL (the
// status word is cleared again; the messages are reset by the caller).
int check_similarity(hap_ctx* h) {
    if (!h->opt.debug_bounds) return HAP_OK;
    CU(launch_check_finite(h->S, h->opt.s_dtype == HAP_S_BF16, h->s_levels, h->N, h->ld, h->status, h->stream));
    h->launches += 1;
    unsigned st[4] = {0, 0, 0, 0};
    CU(cudaMemcpyAsync(st, h->status, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (st[0] & ST_BOUNDS) {
        CU(cudaMemsetAsync(h->status, 0, 4 * sizeof(unsigned), h->stream));
        CU(cudaStreamSynchronize(h->stream));
        return HAP_EINVAL;
    }
    return HAP_OK;
}

int check_status(hap_ctx* h) {
    unsigned st[4] = {0, 0, 0, 0};
    CU(cudaMemcpyAsync(st, h->status, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (st[0] & ST_TIMEOUT) return HAP_ETIMEOUT;
    if (st[0]) return HAP_EDEVICE;
    return HAP_OK;
}

}  // namespace

extern "C" {

void hap_default_options(hap_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->c_mode = HAP_C_PAPER;
    opt->schedule = HAP_SCHED_JACOBI;
    opt->s_dtype = HAP_S_F32;
}

int hap_workspace_bytes(int64_t N, int L, const hap_options* opt, size_t* bytes) {
    if (!bytes) return HAP_EINVAL;
    hap_options o;
    hap_default_options(&o);
    if (opt) o = *opt;
    LaunchShape sh;
    Layout y;
    int rc = plan(N, L, o, &sh, &y);
    if (rc) return rc;
    *bytes = y.total;
    return HAP_OK;
}

int hap_create(int64_t N, int L, const float* prefs, float damping, const hap_options* opt,
               void* dev_workspace, size_t ws_bytes, hap_ctx** out) {
    if (!out) return HAP_EINVAL;
    *out = nullptr;
    if (!(damping > 0.f && damping < 1.f)) return HAP_EINVAL;
    hap_options o;
    hap_default_options(&o);
    if (opt) o = *opt;
    LaunchShape sh;
    Layout y;
    int rc = plan(N, L, o, &sh, &y);
    if (rc) return rc;
    if (dev_workspace && ((uintptr_t)dev_workspace % kAlign)) return HAP_EINVAL;
    if (dev_workspace && ws_bytes < y.total) return HAP_ENOMEM;

    hap_ctx* h = new (std::nothrow) hap_ctx();
    if (!h) return HAP_ENOMEM;
    h->N = N;
    h->L = L;
    h->ld = padded_ld(N);
    h->opt = o;
    h->lam = damping;
    h->sh = sh;
    cudaGetDevice(&h->device);
    if (dev_workspace) {
        h->ws = dev_workspace;
        h->ws_bytes = ws_bytes;
    } else {
        if (cudaMalloc(&h->ws, y.total) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return HAP_ENOMEM;
        }
        h->ws_bytes = y.total;
        h->own_ws = true;
    }
    char* base = static_cast<char*>(h->ws);
    h->A = reinterpret_cast<float*>(base + y.A);
    h->R = reinterpret_cast<float*>(base + y.R);
    h->S = base + y.S;
    h->pref = reinterpret_cast<float*>(base + y.pref);
    h->c = reinterpret_cast<float*>(base + y.c);
    h->c0 = reinterpret_cast<float*>(base + y.c0);
    h->tau = reinterpret_cast<float*>(base + y.tau);
    h->phi = reinterpret_cast<float*>(base + y.phi);
    h->tpart = reinterpret_cast<float*>(base + y.tpart);
    h->b = reinterpret_cast<float*>(base + y.b);
    h->rdiag = reinterpret_cast<float*>(base + y.rdiag);
    h->partials = reinterpret_cast<float*>(base + y.partials);
    h->e = reinterpret_cast<int32_t*>(base + y.e);
    h->ns = reinterpret_cast<double*>(base + y.ns);
    h->acc = reinterpret_cast<long long*>(base + y.acc);
    h->status = reinterpret_cast<unsigned*>(base + y.status);
    h->s_levels = o.s_per_level ? L : 1;
    h->s_level_stride = o.s_per_level ? N * h->ld : 0;

    const size_t s_bytes = (size_t)h->s_levels * N * h->ld * (o.s_dtype == HAP_S_BF16 ? 2 : 4);
    const size_t vec = (size_t)L * h->ld * sizeof(float);
    int r2 = HAP_OK;
    do {
        if (cudaMemsetAsync(h->S, 0, s_bytes, h->stream) != cudaSuccess) { r2 = HAP_ECUDA; break; }
        if (cudaMemsetAsync(h->c0, 0, vec, h->stream) != cudaSuccess) { r2 = HAP_ECUDA; break; }
        if (cudaMemsetAsync(h->pref, 0, vec, h->stream) != cudaSuccess) { r2 = HAP_ECUDA; break; }
        if (cudaMemsetAsync(h->status, 0, 4 * sizeof(unsigned), h->stream) != cudaSuccess) { r2 = HAP_ECUDA; break; }
        if (cudaMemsetAsync(h->partials, 0, (size_t)sh.G * L * h->ld * sizeof(float), h->stream) != cudaSuccess) { r2 = HAP_ECUDA; break; }
        if (prefs) {
            r2 = hap_set_preferences(h, prefs, 0);
            if (r2) break;
        }
        r2 = reset_messages(h);
    } while (0);
    if (r2) {
        cudaGetLastError();
        hap_destroy(h);
        return r2;
    }
    *out = h;
    return HAP_OK;
}

void hap_destroy(hap_ctx* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    if (h->own_ws && h->ws) cudaFree(h->ws);
    delete h;
}

int hap_set_stream(hap_ctx* h, void* stream) {
    if (!h) return HAP_EINVAL;
    h->stream = static_cast<cudaStream_t>(stream);
    return HAP_OK;
}

int hap_set_preferences(hap_ctx* h, const float* prefs, int per_point) {
    if (!h || !prefs || (per_point != 0 && per_point != 1)) return HAP_EINVAL;
    std::vector<float> host((size_t)h->L * h->ld, 0.f);
    for (int l = 0; l < h->L; ++l)
        for (int64_t i = 0; i < h->N; ++i) {
            const float v = per_point ? prefs[(size_t)l * h->N + i] : prefs[l];
            if (!(v > -__builtin_inff() && v < __builtin_inff())) return HAP_EINVAL;
            host[(size_t)l * h->ld + i] = v;
        }
    CU(cudaMemcpyAsync(h->pref, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return HAP_OK;
}

int hap_set_cluster_preferences(hap_ctx* h, const float* c0) {
    if (!h || !c0) return HAP_EINVAL;
    std::vector<float> host((size_t)h->L * h->ld, 0.f);
    for (int l = 0; l < h->L; ++l)
        for (int64_t i = 0; i < h->N; ++i) host[(size_t)l * h->ld + i] = c0[(size_t)l * h->N + i];
    CU(cudaMemcpyAsync(h->c0, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    return reset_messages(h);
}

int hap_set_similarity(hap_ctx* h, int level, const void* S, int64_t ld, int dtype) {
    if (!h || !S || ld < h->N || (dtype != HAP_S_F32 && dtype != HAP_S_BF16)) return HAP_EINVAL;
    if (level < -1 || level >= h->L) return HAP_EINVAL;
    if (level >= 0 && !h->opt.s_per_level) return HAP_EINVAL;
    const size_t es = h->opt.s_dtype == HAP_S_BF16 ? 2 : 4;
    const int first = level < 0 ? 0 : level;
    const int last = level < 0 ? h->s_levels : level + 1;
    for (int l = first; l < last; ++l) {
        char* dst = static_cast<char*>(h->S) + (size_t)l * h->N * h->ld * es;
        CU(launch_copy_similarity(dst, h->opt.s_dtype == HAP_S_BF16, h->ld, S, dtype == HAP_S_BF16, ld, h->N, h->stream));
        h->launches += 1;
    }
    const int rc = reset_messages(h);
    return rc ? rc : check_similarity(h);
}

int hap_build_similarity(hap_ctx* h, const float* X, int64_t d, int mode) {
    if (!h || !X || d < 1) return HAP_EINVAL;
    if (mode != HAP_SBUILD_F32 && mode != HAP_SBUILD_BF16 && mode != HAP_SBUILD_BF16_SPLIT) return HAP_EINVAL;
    const int s_bf16 = h->opt.s_dtype == HAP_S_BF16;
    const size_t es = s_bf16 ? 2 : 4;
    // Points in host memory are first copied into the end of the alpha and rho
    // storage (the build resets the messages anyway), behind the operand
    // scratch of the tensor-core modes.
    cudaPointerAttributes pa{};
    const cudaError_t pq = cudaPointerGetAttributes(&pa, X);
    if (pq != cudaSuccess) cudaGetLastError();
    if (pq != cudaSuccess || pa.type == cudaMemoryTypeHost || pa.type == cudaMemoryTypeUnregistered) {
        const size_t xbytes = (size_t)h->N * d * sizeof(float);
        const size_t ops = mode == HAP_SBUILD_F32 ? 0 : sbuild_tc_scratch_bytes(h->N, d, mode == HAP_SBUILD_BF16_SPLIT);
        char* lo = reinterpret_cast<char*>(h->A);
        char* end = static_cast<char*>(h->S);
        if ((size_t)(end - lo) < ops + xbytes + 1024) return HAP_EUNSUPPORTED;
        float* stage = reinterpret_cast<float*>(((uintptr_t)(end - xbytes)) & ~(uintptr_t)255);
        CU(cudaMemcpyAsync(stage, X, xbytes, cudaMemcpyHostToDevice, h->stream));
        X = stage;
    }
    if (mode == HAP_SBUILD_F32) {
        CU(launch_sbuild_f32(X, h->N, d, h->S, s_bf16, h->ld, h->stream));
        h->launches += 1;
    } else if (mode == HAP_SBUILD_BF16 || mode == HAP_SBUILD_BF16_SPLIT) {
        const int split = mode == HAP_SBUILD_BF16_SPLIT;
        // the alpha and rho storage and the reserve after it (contiguous, reset
        // after the build) serve as operand scratch
        const size_t need = sbuild_tc_scratch_bytes(h->N, d, split);
        const size_t cap = (size_t)(static_cast<char*>(h->S) - reinterpret_cast<char*>(h->A));
        if (need > cap) return HAP_EUNSUPPORTED;
        int nk = 0;
        cudaError_t err = launch_sbuild_tc(X, h->N, d, split, h->S, s_bf16, h->ld, h->A, h->status, h->stream, &nk);
        if (err == cudaErrorNotSupported) return HAP_EUNSUPPORTED;
        CU(err);
        h->launches += nk;
    } else {
        return HAP_EINVAL;
    }
    for (int l = 1; l < h->s_levels; ++l)
        CU(cudaMemcpyAsync(static_cast<char*>(h->S) + (size_t)l * h->N * h->ld * es, h->S,
                           (size_t)h->N * h->ld * es, cudaMemcpyDeviceToDevice, h->stream));
    int rc = reset_messages(h);
    if (rc) return rc;
    rc = check_similarity(h);
    if (rc) return rc;
    return check_status(h);
}

int hap_get_similarity(hap_ctx* h, int level, float* S) {
    if (!h || !S || level < 0 || level >= h->L) return HAP_EINVAL;
    const int s_bf16 = h->opt.s_dtype == HAP_S_BF16;
    const char* src = static_cast<const char*>(h->S) + (size_t)level * h->s_level_stride * (s_bf16 ? 2 : 4);
    CU(launch_read_similarity(S, src, s_bf16, h->pref + (size_t)level * h->ld, h->N, h->ld, h->stream));
    h->launches += 1;
    return HAP_OK;
}

// Algorithm 1's sequential level loop: per level, the fused row pass on that
// level alone (alpha final, tau^l as the previous level sent it), the column
// statistics (b^l; rho_jj + P_j into tpart's level-l row) and the availability
// step that also sends c^l, phi^{l-1} and tau^{l+1}.
static int iterate_gauss_seidel(hap_ctx* h, RowPassArgs a, int n) {
    const int s_bf16 = h->opt.s_dtype == HAP_S_BF16;
    const int64_t N = h->N, ld = h->ld, L = h->L;
    const int64_t mat = N * ld;
    for (int it = 0; it < n; ++it) {
        for (int64_t l = 0; l < L; ++l) {
            RowPassArgs v = a;
            v.A = h->A + l * mat;
            v.R = h->R + l * mat;
            v.S = static_cast<char*>(h->S) + (size_t)(l * h->s_level_stride) * (s_bf16 ? 2 : 4);
            v.s_level_stride = 0;
            v.L = 1;
            v.pref = h->pref + l * ld;
            v.c = h->c + l * ld;
            v.tau = h->tau + l * ld;
            v.phi = h->phi + l * ld;
            v.tpart = h->tpart + l * ld;
            v.b = h->b + l * ld;
            v.rdiag = h->rdiag + l * ld;
            v.pending = 0;
            v.update_c = 0;
            v.use_tau = 0;
            v.tau_in = l > 0 ? h->tau + l * ld : nullptr;
            v.kappa = 0.f;
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (h->opt.profile) {
                CU(cudaEventCreate(&e0));
                CU(cudaEventCreate(&e1));
                CU(cudaEventRecord(e0, h->stream));
            }
            CU(launch_rowpass(v, h->sh, s_bf16, h->stream));
            if (h->opt.profile) {
                CU(cudaEventRecord(e1, h->stream));
                h->ev.push_back(e0);
                h->ev.push_back(e1);
            }
            CU(launch_colstats(h->partials, h->sh.G, 1, N, ld, v.c, v.phi, v.rdiag, h->b + l * ld, nullptr, h->stream,
                               h->tpart + l * ld));
            GsArgs g;
            g.A = v.A;
            g.R = v.R;
            g.S = v.S;
            g.b = v.b;
            g.pref = v.pref;
            g.c = v.c;
            g.tp = h->tpart + l * ld;
            g.phi_out = l > 0 ? h->phi + (l - 1) * ld : nullptr;
            g.tau_next = l + 1 < L ? h->tau + (l + 1) * ld : nullptr;
            g.N = N;
            g.ld = ld;
            g.lam = a.lam;
            g.oml = a.oml;
            g.update_c = h->opt.c_mode == HAP_C_PAPER ? 1 : 0;
            CU(launch_gs_availability(g, s_bf16, h->stream));
            h->launches += 3;
        }
        h->pending = false;
        h->iter += 1;
        h->e_valid = false;
    }
    return HAP_OK;
}

int hap_iterate(hap_ctx* h, int n) {
    if (!h || n < 0) return HAP_EINVAL;
    RowPassArgs a;
    a.A = h->A;
    a.R = h->R;
    a.S = h->S;
    a.N = h->N;
    a.ld = h->ld;
    a.s_level_stride = h->s_level_stride;
    a.L = h->L;
    a.pref = h->pref;
    a.c = h->c;
    a.tau = h->tau;
    a.phi = h->phi;
    a.tpart = h->tpart;
    a.b = h->b;
    a.rdiag = h->rdiag;
    a.partials = h->partials;
    a.status = h->status;
    a.lam = h->lam;
    a.oml = 1.0f - h->lam;
    a.kappa = h->opt.kappa;
    a.wait_ns = wait_limit(h->opt);
    a.debug = h->opt.debug_bounds;
    const int s_bf16 = h->opt.s_dtype == HAP_S_BF16;
    if (h->opt.schedule == HAP_SCHED_GAUSS_SEIDEL) return iterate_gauss_seidel(h, a, n);
    for (int it = 0; it < n; ++it) {
        const int64_t t = h->iter + 1;
        a.pending = h->pending ? 1 : 0;
        a.update_c = (h->opt.c_mode == HAP_C_PAPER && t >= 2) ? 1 : 0;
        a.use_tau = t >= 2 ? 1 : 0;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->opt.profile) {
            CU(cudaEventCreate(&e0));
            CU(cudaEventCreate(&e1));
            CU(cudaEventRecord(e0, h->stream));
        }
        CU(launch_rowpass(a, h->sh, s_bf16, h->stream));
        if (h->opt.profile) {
            CU(cudaEventRecord(e1, h->stream));
            h->ev.push_back(e0);
            h->ev.push_back(e1);
        }
        CU(launch_colstats(h->partials, h->sh.G, h->L, h->N, h->ld, h->c, h->phi, h->rdiag, h->b, h->tpart, h->stream));
        h->launches += 2;
        h->pending = true;
        h->iter = t;
        h->e_valid = false;
    }
    return HAP_OK;
}

int hap_exemplars(hap_ctx* h, int32_t* e, int on_host) {
    if (!h || !e || (on_host != 0 && on_host != 1)) return HAP_EINVAL;
    const int rc = ensure_exemplars(h);
    if (rc) return rc;
    const size_t bytes = (size_t)h->L * h->N * sizeof(int32_t);
    CU(cudaMemcpyAsync(e, h->e, bytes, on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
    if (on_host) return hap_sync(h);
    return HAP_OK;
}

int hap_net_similarity(hap_ctx* h, double* ns) {
    if (!h || !ns) return HAP_EINVAL;
    const int rc = ensure_exemplars(h);
    if (rc) return rc;
    CU(launch_netsim(h->S, h->opt.s_dtype == HAP_S_BF16, h->s_level_stride, h->pref, h->e, h->N, h->ld, h->L, h->ns, h->stream));
    h->launches += 1;
    CU(cudaMemcpyAsync(ns, h->ns, (size_t)h->L * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return hap_sync(h);
}

int hap_acceptance(hap_ctx* h, int64_t* consistent, int64_t* exemplars) {
    if (!h) return HAP_EINVAL;
    const int rc0 = ensure_exemplars(h);
    if (rc0) return rc0;
    CU(launch_acceptance(h->e, h->N, h->L, h->acc, h->stream));
    h->launches += 1;
    std::vector<long long> host((size_t)2 * h->L);
    CU(cudaMemcpyAsync(host.data(), h->acc, host.size() * sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    int rc = hap_sync(h);
    if (rc) return rc;
    for (int l = 0; l < h->L; ++l) {
        if (consistent) consistent[l] = host[l];
        if (exemplars) exemplars[l] = host[h->L + l];
    }
    return HAP_OK;
}

int hap_get_state(hap_ctx* h, float* A, float* R, float* vecs, int64_t* iter) {
    if (!h) return HAP_EINVAL;
    const int64_t N = h->N, L = h->L, ld = h->ld;
    if (A) {
        CU(launch_materialize_A(A, h->A, h->R, h->b, h->pending, h->lam, 1.0f - h->lam, N, ld, (int)L, h->stream));
        h->launches += 1;
    }
    if (R)
        CU(cudaMemcpy2DAsync(R, N * sizeof(float), h->R, ld * sizeof(float), N * sizeof(float), (size_t)(L * N),
                             cudaMemcpyDeviceToDevice, h->stream));
    if (vecs) {
        const float* src[3] = {h->c, h->tau, h->phi};
        for (int q = 0; q < 3; ++q)
            CU(cudaMemcpy2DAsync(vecs + (size_t)q * L * N, N * sizeof(float), src[q], ld * sizeof(float),
                                 N * sizeof(float), (size_t)L, cudaMemcpyDeviceToDevice, h->stream));
    }
    if (iter) *iter = h->iter;
    return HAP_OK;
}

int hap_set_state(hap_ctx* h, const float* A, const float* R, const float* vecs, int64_t iter) {
    if (!h || !A || !R || !vecs || iter < 0) return HAP_EINVAL;
    const int64_t N = h->N, L = h->L, ld = h->ld;
    CU(cudaMemcpy2DAsync(h->A, ld * sizeof(float), A, N * sizeof(float), N * sizeof(float), (size_t)(L * N),
                         cudaMemcpyDeviceToDevice, h->stream));
    CU(cudaMemcpy2DAsync(h->R, ld * sizeof(float), R, N * sizeof(float), N * sizeof(float), (size_t)(L * N),
                         cudaMemcpyDeviceToDevice, h->stream));
    float* dst[3] = {h->c, h->tau, h->phi};
    for (int q = 0; q < 3; ++q)
        CU(cudaMemcpy2DAsync(dst[q], ld * sizeof(float), vecs + (size_t)q * L * N, N * sizeof(float),
                             N * sizeof(float), (size_t)L, cudaMemcpyDeviceToDevice, h->stream));
    CU(launch_prepare_from_R(h->R, h->sh.G, (int)L, N, ld, h->rdiag, h->tpart, h->stream));
    CU(cudaMemsetAsync(h->status, 0, 4 * sizeof(unsigned), h->stream));
    h->launches += 1;
    h->iter = iter;
    h->pending = false;
    h->e_valid = false;
    return HAP_OK;
}

int hap_set_wait_limit(hap_ctx* h, int64_t ns) {
    if (!h || ns < 0) return HAP_EINVAL;
    h->opt.wait_limit_ns = ns;
    return HAP_OK;
}

int hap_sync(hap_ctx* h) {
    if (!h) return HAP_EINVAL;
    CU(cudaStreamSynchronize(h->stream));
    CU(cudaGetLastError());
    return check_status(h);
}

int hap_query(hap_ctx* h, int key, int64_t* value) {
    if (!h || !value) return HAP_EINVAL;
    switch (key) {
        case HAP_Q_BLOCK_THREADS: *value = h->sh.T; return HAP_OK;
        case HAP_Q_CLUSTER_SIZE: *value = h->sh.C; return HAP_OK;
        case HAP_Q_GRID_CLUSTERS: *value = h->sh.G; return HAP_OK;
        case HAP_Q_LD: *value = h->ld; return HAP_OK;
        case HAP_Q_ITER: *value = h->iter; return HAP_OK;
        case HAP_Q_ELEMS_PER_THREAD: *value = 4 * h->sh.K; return HAP_OK;
        case HAP_Q_LAUNCHES: *value = h->launches; return HAP_OK;
        case HAP_Q_COL_SUMS: *value = h->sh.tm ? HAP_COLSUM_TMEM : HAP_COLSUM_SMEM; return HAP_OK;
        case HAP_Q_STAGES: *value = h->sh.tm ? h->sh.nst : 3; return HAP_OK;
        case HAP_Q_CTAS_PER_SM: *value = h->sh.dual ? 2 : 1; return HAP_OK;
        default: return HAP_EINVAL;
    }
}

int hap_row_pass_time(hap_ctx* h, double* ms, int64_t* launches, int reset) {
    if (!h || !ms || !launches) return HAP_EINVAL;
    CU(cudaStreamSynchronize(h->stream));
    for (size_t q = 0; q + 1 < h->ev.size(); q += 2) {
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, h->ev[q], h->ev[q + 1]));
        h->prof_ms += t;
        h->prof_n += 1;
        cudaEventDestroy(h->ev[q]);
        cudaEventDestroy(h->ev[q + 1]);
    }
    h->ev.clear();
    *ms = h->prof_ms;
    *launches = h->prof_n;
    if (reset) {
        h->prof_ms = 0.0;
        h->prof_n = 0;
    }
    return HAP_OK;
}

const char* hap_strerror(int code) {
    switch (code) {
        case HAP_OK: return "HAP_OK";
        case HAP_EINVAL: return "HAP_EINVAL: invalid argument";
        case HAP_ENOMEM: return "HAP_ENOMEM: workspace too small or allocation failed";
        case HAP_ECUDA: return "HAP_ECUDA: CUDA runtime error";
        case HAP_EDEVICE: return "HAP_EDEVICE: kernel reported an error";
        case HAP_ETIMEOUT: return "HAP_ETIMEOUT: bounded device wait expired";
        case HAP_EUNSUPPORTED: return "HAP_EUNSUPPORTED: unsupported size or mode";
        default: return "unknown HAP status";
    }
}

}  // extern "C"
