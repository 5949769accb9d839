// Row bands of one HAP problem (the row-partitioned decomposition of §3: the
// responsibility job is keyed by node i, the availability job by exemplar j).
// A band holds rows row0 .. row0 + nrows - 1 of S, alpha and rho; its row pass
// is the fused row-pass kernel with a row offset, and the column statistics
// of the whole problem are formed from every band's exchange buffer (its rows'
// part of P_j and the c, phi, rho_jj of the rows it owns), summed in band
// order, so every band computes the same b and tau's column part.
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>
#include <vector>

#include "hap.h"
#include "hap_internal.h"

using namespace hap;

struct hap_band {
    int64_t N = 0, row0 = 0, nrows = 0, ld = 0;
    int L = 0;
    hap_options opt{};
    float lam = 0.5f;
    cudaStream_t stream = nullptr;
    LaunchShape sh{};
    void* ws = nullptr;
    float *A = nullptr, *R = nullptr;
    void* S = nullptr;
    float *pref = nullptr, *c = nullptr, *tau = nullptr, *phi = nullptr, *tpart = nullptr, *b = nullptr,
          *rdiag = nullptr, *partials = nullptr;
    int32_t* e = nullptr;
    unsigned* status = nullptr;
    int64_t iter = 0, launches = 0;
    bool pending = false;
    bool rows_done = false;  // hap_band_rows ran; hap_band_columns completes the iteration
};

namespace {

constexpr size_t kAl = 256;
size_t al(size_t x) { return (x + kAl - 1) / kAl * kAl; }

#define BNDCU(x)                       \
    do {                               \
        if ((x) != cudaSuccess) {      \
            cudaGetLastError();        \
            return HAP_ECUDA;          \
        }                              \
    } while (0)

// Algorithm 1's initial values: alpha = rho = 0 (alpha's padding -inf),
// tau = +inf, phi = 0, c = 0; clears the status word.
int band_reset(hap_band* h) {
    const size_t mat = (size_t)h->L * h->nrows * h->ld * 4, vec = (size_t)h->L * h->ld * 4;
    BNDCU(cudaMemsetAsync(h->status, 0, 4 * sizeof(unsigned), h->stream));
    BNDCU(cudaMemsetAsync(h->A, 0, mat, h->stream));
    BNDCU(launch_fill_alpha_padding(h->A, (int64_t)h->L * h->nrows, h->N, h->ld, h->stream));
    BNDCU(cudaMemsetAsync(h->R, 0, mat, h->stream));
    float* zero[5] = {h->c, h->phi, h->tpart, h->b, h->rdiag};
    for (float* z : zero) BNDCU(cudaMemsetAsync(z, 0, vec, h->stream));
    std::vector<float> inf((size_t)h->L * h->ld, __builtin_inff());
    BNDCU(cudaMemcpyAsync(h->tau, inf.data(), vec, cudaMemcpyHostToDevice, h->stream));
    BNDCU(cudaStreamSynchronize(h->stream));
    h->iter = 0;
    h->pending = false;
    h->rows_done = false;
    return HAP_OK;
}

}  // namespace

extern "C" {

int hap_band_create(int64_t N, int64_t row0, int64_t nrows, int L, const float* prefs, float damping,
                    const hap_options* opt, hap_band** out) {
    if (!out) return HAP_EINVAL;
    *out = nullptr;
    if (!(damping > 0.f && damping < 1.f) || row0 < 0 || nrows < 1 || row0 + nrows > N) return HAP_EINVAL;
    hap_options o;
    hap_default_options(&o);
    if (opt) o = *opt;
    int rc = check_options(o);
    if (rc) return rc;
    if (o.schedule != HAP_SCHED_JACOBI || o.kappa != 0.f || o.s_per_level || o.debug_bounds) return HAP_EUNSUPPORTED;
    LaunchShape sh{};
    rc = plan_shape(N, nrows, L, o, &sh);
    if (rc) return rc;
    hap_band* h = new (std::nothrow) hap_band();
    if (!h) return HAP_ENOMEM;
    h->N = N;
    h->row0 = row0;
    h->nrows = nrows;
    h->L = L;
    h->ld = (N + 31) / 32 * 32;
    h->opt = o;
    h->lam = damping;
    h->sh = sh;
    const size_t mat = al((size_t)L * nrows * h->ld * 4), vec = al((size_t)L * h->ld * 4);
    const size_t sb = al((size_t)nrows * h->ld * (o.s_dtype == HAP_S_BF16 ? 2 : 4));
    const size_t pb = al((size_t)sh.G * L * h->ld * 4), eb = al((size_t)L * nrows * 4);
    const size_t total = 2 * mat + sb + 7 * vec + pb + eb + al(16);
    if (cudaMalloc(&h->ws, total) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return HAP_ENOMEM;
    }
    char* p = static_cast<char*>(h->ws);
    h->A = reinterpret_cast<float*>(p); p += mat;
    h->R = reinterpret_cast<float*>(p); p += mat;
    h->S = p; p += sb;
    float** v[7] = {&h->pref, &h->c, &h->tau, &h->phi, &h->tpart, &h->b, &h->rdiag};
    for (float** q : v) { *q = reinterpret_cast<float*>(p); p += vec; }
    h->partials = reinterpret_cast<float*>(p); p += pb;
    h->e = reinterpret_cast<int32_t*>(p); p += eb;
    h->status = reinterpret_cast<unsigned*>(p);
    rc = HAP_OK;
    if (cudaMemset(h->S, 0, sb) != cudaSuccess || cudaMemset(h->partials, 0, pb) != cudaSuccess ||
        cudaMemset(h->pref, 0, vec) != cudaSuccess)
        rc = HAP_ECUDA;
    if (!rc && prefs) {
        std::vector<float> host((size_t)L * h->ld, 0.f);
        for (int l = 0; l < L && !rc; ++l) {
            if (!(prefs[l] > -__builtin_inff() && prefs[l] < __builtin_inff())) rc = HAP_EINVAL;
            for (int64_t i = 0; i < N; ++i) host[(size_t)l * h->ld + i] = prefs[l];
        }
        if (!rc && cudaMemcpy(h->pref, host.data(), host.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = HAP_ECUDA;
    }
    if (!rc) rc = band_reset(h);
    if (rc) {
        cudaGetLastError();
        hap_band_destroy(h);
        return rc;
    }
    *out = h;
    return HAP_OK;
}

void hap_band_destroy(hap_band* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
    delete h;
}

int hap_band_set_stream(hap_band* h, void* stream) {
    if (!h) return HAP_EINVAL;
    h->stream = static_cast<cudaStream_t>(stream);
    return HAP_OK;
}

int hap_band_set_similarity(hap_band* h, const void* S, int64_t ld_src, int dtype) {
    if (!h || !S || ld_src < h->N || (dtype != HAP_S_F32 && dtype != HAP_S_BF16)) return HAP_EINVAL;
    BNDCU(launch_copy_similarity(h->S, h->opt.s_dtype == HAP_S_BF16, h->ld, S, dtype == HAP_S_BF16, ld_src, h->N,
                                 h->stream, h->nrows));
    h->launches += 1;
    return band_reset(h);
}

int hap_band_exchange_floats(hap_band* h, int64_t* n) {
    if (!h || !n) return HAP_EINVAL;
    *n = 4 * (int64_t)h->L * h->ld;
    return HAP_OK;
}

int hap_band_rows(hap_band* h, float* xch) {
    if (!h || !xch || h->rows_done) return HAP_EINVAL;
    const int64_t t = h->iter + 1;
    RowPassArgs a;
    a.A = h->A;
    a.R = h->R;
    a.S = h->S;
    a.N = h->N;
    a.ld = h->ld;
    a.s_level_stride = 0;
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
    a.pending = h->pending ? 1 : 0;
    a.update_c = (h->opt.c_mode == HAP_C_PAPER && t >= 2) ? 1 : 0;
    a.use_tau = t >= 2 ? 1 : 0;
    a.wait_ns = h->opt.wait_limit_ns > 0 ? (uint64_t)h->opt.wait_limit_ns : 2000000000ull;
    a.row0 = h->row0;
    a.nrows = h->nrows;
    BNDCU(launch_rowpass(a, h->sh, h->opt.s_dtype == HAP_S_BF16, h->stream));
    BNDCU(launch_band_summary(h->partials, h->sh.G, h->L, h->N, h->ld, h->c, h->phi, h->rdiag, h->row0, h->nrows,
                              xch, h->stream));
    h->launches += 2;
    h->rows_done = true;
    return HAP_OK;
}

int hap_band_columns(hap_band* h, const float* xch_all, int P, const int64_t* bounds) {
    if (!h || !xch_all || !bounds || P < 1 || P > kMaxBands || !h->rows_done) return HAP_EINVAL;
    BandBounds bb{};
    bool mine = false;
    if (bounds[0] != 0 || bounds[P] != h->N) return HAP_EINVAL;
    for (int r = 0; r <= P; ++r) {
        if (r > 0 && bounds[r] <= bounds[r - 1]) return HAP_EINVAL;
        bb.lo[r] = bounds[r];
        if (r < P && bounds[r] == h->row0 && bounds[r + 1] == h->row0 + h->nrows) mine = true;
    }
    if (!mine) return HAP_EINVAL;
    BNDCU(launch_band_columns(xch_all, P, bb, h->L, h->N, h->ld, h->c, h->phi, h->rdiag, h->b, h->tpart, h->stream));
    h->launches += 1;
    h->rows_done = false;
    h->pending = true;
    h->iter += 1;
    return HAP_OK;
}

int hap_band_get_state(hap_band* h, float* A, float* R, float* vecs, int64_t* iter) {
    if (!h || h->rows_done) return HAP_EINVAL;
    const int64_t N = h->N, L = h->L, ld = h->ld, nr = h->nrows;
    if (A) {
        BNDCU(launch_materialize_A(A, h->A, h->R, h->b, h->pending, h->lam, 1.0f - h->lam, N, ld, (int)L, h->stream,
                                   nr, h->row0));
        h->launches += 1;
    }
    if (R)
        BNDCU(cudaMemcpy2DAsync(R, N * 4, h->R, ld * 4, N * 4, (size_t)(L * nr), cudaMemcpyDeviceToDevice, h->stream));
    if (vecs) {
        const float* src[3] = {h->c, h->tau, h->phi};
        for (int q = 0; q < 3; ++q)
            BNDCU(cudaMemcpy2DAsync(vecs + (size_t)q * L * N, N * 4, src[q], ld * 4, N * 4, (size_t)L,
                                    cudaMemcpyDeviceToDevice, h->stream));
    }
    if (iter) *iter = h->iter;
    return HAP_OK;
}

int hap_band_exemplars(hap_band* h, int32_t* e, int on_host) {
    if (!h || !e || (on_host != 0 && on_host != 1) || h->rows_done) return HAP_EINVAL;
    BNDCU(launch_exemplars(h->A, h->R, h->b, h->pending, h->lam, 1.0f - h->lam, h->N, h->ld, h->L, h->e, h->stream,
                           h->nrows, h->row0));
    h->launches += 1;
    BNDCU(cudaMemcpyAsync(e, h->e, (size_t)h->L * h->nrows * 4,
                          on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
    return on_host ? hap_band_sync(h) : HAP_OK;
}

int hap_band_sync(hap_band* h) {
    if (!h) return HAP_EINVAL;
    BNDCU(cudaStreamSynchronize(h->stream));
    BNDCU(cudaGetLastError());
    unsigned st = 0;
    BNDCU(cudaMemcpy(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost));
    if (st & ST_TIMEOUT) return HAP_ETIMEOUT;
    if (st) return HAP_EDEVICE;
    return HAP_OK;
}

int hap_band_query(hap_band* h, int key, int64_t* value) {
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

}  // extern "C"
