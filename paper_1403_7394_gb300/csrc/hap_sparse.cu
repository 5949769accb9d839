// Sparse HAP: the messages of §2 (Eqs. 2.1-2.6 with damping, §3 schedule)
// kept only on a candidate graph with K entries per row (row i's candidate
// exemplars, including i itself, sorted by index).  It is exactly HAP on a
// similarity that is -inf outside the graph: such pairs never win a row
// maximum and add max(0, rho) = 0 to every column sum.
//
// Layout: cand [N][K] int32, s [N][K] FP32 (= -||x_i - x_cand||^2, the
// preference on the self entry), alpha and rho [L][N][K], the column terms
// b [N][4 ceil(L/4)] (all levels of a column side by side, so one 16-byte
// gather per candidate brings them).  Row pass: one warp per row walks the L
// levels (alpha kept one step behind exactly as in the dense row pass); the
// next level's alpha and rho load while the current level reduces, and the
// next row's candidates, CSC slots, similarities, per-level scalars and b
// load while the current row runs.  The column index (CSC: for every column
// j the entries (k, q) with cand[k][q] = j, in entry order) is built on the
// GPU by a stable radix sort of the entries by column.  The row pass writes
// each positive off-diagonal responsibility straight to its CSC slot and
// sets the slot's bit in a per-level bitmap zeroed before the pass (most
// responsibilities are negative, so a few scattered writes per row); the
// column statistics read the bitmap and gather the values of set bits alone,
// in a fixed order, so the CSC values are neither zeroed nor swept.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <vector>

#include "hap.h"
#include "hap_common.cuh"
#include "hap_internal.h"

namespace hap {
namespace {

constexpr int SP_MAXK = 64;

struct SparseArgs {
    const int32_t* cand;
    const int32_t* pos;    // [N][K] CSC slot of every entry
    float* cval;           // [L][N*K] max(0, rho) in CSC order, valid where the slot's bit is set
    unsigned* cbits;       // [L][cwords] bit e of level l set iff slot e holds a positive value; zero before the pass
    int64_t cwords;
    const float* s;
    float* A;
    float* R;
    const float* pref;
    float* c;
    float* tau;
    float* phi;
    const float* tpart;
    const float* b;        // [N][Lb]: the levels of one column side by side (Lb = L rounded up to 4)
    float* rdiag;
    unsigned* status;
    int N, L, K, Lb;
    float lam, oml;
    int pending, update_c, use_tau;
};

// one warp per row, all levels of the row in order; lane holds entries
// q = lane and q = lane + 32.  The column terms b of four levels of a
// candidate come in one 16-byte gather (levels 0-3 of the next row's
// candidates during this row's last level, levels 4q..4q+3 four levels
// ahead when kMultiChunk, i.e. L > 4).
// kFull: K = 64, every lane holds two entries (no per-entry predicates:
// 29 % fewer instructions; the pass is issue-bound).
template <bool kMultiChunk, bool kFull>
__global__ void __launch_bounds__(256, 4) sparse_rowpass_kernel(const SparseArgs p) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int K = kFull ? 64 : p.K, L = p.L, N = p.N;
    const int64_t NK = (int64_t)N * K;
    const bool pending = p.pending != 0;
    bool has[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) has[h] = kFull || lane + 32 * h < K;
    // the next row's candidates, CSC slots and similarities load while this
    // row's levels run
    int njq[2] = {0x7fffffff, 0x7fffffff}, npq[2] = {0, 0};
    float nsq[2] = {0.f, 0.f};
    // and so do its per-level scalars: lane t < L holds level t's
    // preference, fixed c and tau part, broadcast by shuffles when needed
    float nsc_pref = 0.f, nsc_c = 0.f, nsc_tp = 0.f;
    auto load_row = [&](int64_t r) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = lane + 32 * h;
            if (has[h] && r < N) {
                njq[h] = p.cand[r * K + q];
                npq[h] = p.pos[r * K + q];
                nsq[h] = p.s[r * K + q];
            }
        }
        if (lane < L && r < N) {
            const int64_t at = (int64_t)lane * N + r;
            nsc_pref = __ldg(p.pref + at);
            if (!p.update_c) nsc_c = p.c[at];
            nsc_tp = p.tpart[at];
        }
    };
    auto gather_b = [&](const int (&j)[2], int chunk, float4 (&out)[2]) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
            out[h] = (has[h] && pending)
                         ? __ldg(reinterpret_cast<const float4*>(p.b + (int64_t)j[h] * p.Lb + 4 * chunk))
                         : f4_splat(0.f);
    };
    float4 bc[2] = {f4_splat(0.f), f4_splat(0.f)};
    load_row(wid);
    if (wid < N) gather_b(njq, 0, bc);
    for (int64_t i = wid; i < N; i += nw) {
        int jq[2], pq[2];
        float sq[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            jq[h] = has[h] ? njq[h] : 0x7fffffff;
            pq[h] = npq[h];
            sq[h] = nsq[h];
        }
        const float sc_pref = nsc_pref, sc_c = nsc_c, sc_tp = nsc_tp;
        load_row(i + nw);
        // level 0's messages; later levels are loaded one level ahead.
        // Al / Rl point at this lane's first entry of the row at level l,
        // vo is level l's offset in the [L][N] vectors
        float* Al = p.A + i * K + lane;
        float* Rl = p.R + i * K + lane;
        int64_t vo = 0;
        float a[2], r[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            a[h] = has[h] ? Al[32 * h] : -kInf;
            r[h] = has[h] ? Rl[32 * h] : 0.f;
        }
        float4 bn[2] = {f4_splat(0.f), f4_splat(0.f)};
        float c_prev = 0.f;
        for (int l = 0; l < L; ++l, Al += NK, Rl += NK, vo += N) {
            if (kMultiChunk) {
                if ((l & 3) == 0 && l > 0) {
                    bc[0] = bn[0];
                    bc[1] = bn[1];
                }
                if ((l & 3) == 0 && l + 4 < L) gather_b(jq, (l >> 2) + 1, bn);
            }
            const float bb[2] = {f4_get(bc[0], l & 3), f4_get(bc[1], l & 3)};
            // bc is spent after the last level's read: the next row's gather
            // goes out while that level runs
            if (l == L - 1 && i + nw < N) gather_b(njq, 0, bc);
            float na[2] = {-kInf, -kInf}, nr[2] = {0.f, 0.f};
            if (l + 1 < L) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (has[h]) {
                        na[h] = Al[NK + 32 * h];
                        nr[h] = Rl[NK + 32 * h];
                    }
                }
            }
            const float pref_i = __shfl_sync(0xffffffffu, sc_pref, l);
            float x[2];
            float m1 = -kInf, m2 = -kInf, cm = -kInf;
            int k1 = 0x7fffffff;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!has[h]) { x[h] = -kInf; continue; }
                const bool diag = jq[h] == (int)i;
                const float sv = diag ? pref_i : sq[h];
                x[h] = sv;
                if (pending) {
                    a[h] = damp(a[h], avail_target(bb[h], r[h], diag), p.lam, p.oml);
                    Al[32 * h] = a[h];
                }
                top2_push(__fadd_rn(a[h], sv), jq[h], m1, k1, m2);
                cm = fmaxf(cm, __fadd_rn(a[h], r[h]));
            }
            warp_top2(m1, k1, m2, cm);
            const float c_fixed = __shfl_sync(0xffffffffu, sc_c, l);
            const float tp_i = __shfl_sync(0xffffffffu, sc_tp, l);
            const float cval = p.update_c ? cm : c_fixed;
            const float tauv = (p.use_tau && l > 0) ? __fadd_rn(c_prev, tp_i) : kInf;
            c_prev = cval;
            if (lane == 0) {
                if (p.update_c) p.c[vo + i] = cval;
                p.tau[vo + i] = tauv;
                if (l > 0) p.phi[vo - N + i] = m1;
            }
            float rnv[2];
            bool wpos[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                wpos[h] = false;
                if (!has[h]) continue;
                const float mx = jq[h] == k1 ? m2 : m1;
                const float rn = damp(r[h], __fadd_rn(x[h], fminf(tauv, -mx)), p.lam, p.oml);
                Rl[32 * h] = rn;
                const bool diag = jq[h] == (int)i;
                if (diag) p.rdiag[vo + i] = rn;
                rnv[h] = rn;
                wpos[h] = !diag && rn > 0.f;
            }
            // only positive off-diagonal responsibilities are written (a few
            // per row), each with its slot's bit; one warp vote skips the
            // common case where no lane has one
            if (__any_sync(0xffffffffu, wpos[0] || wpos[1])) {
                float* cv = p.cval + l * NK;
                unsigned* cb = p.cbits + l * p.cwords;
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (wpos[h]) {
                        cv[pq[h]] = rnv[h];
                        atomicOr(cb + (pq[h] >> 5), 1u << (pq[h] & 31));
                    }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                a[h] = na[h];
                r[h] = nr[h];
            }
        }
    }
}

// P_j = sum over the column's entries (rows k != j) of max(0, rho), read from
// the CSC-ordered values the row pass wrote; a slot whose bit is clear holds
// a zero term and is skipped (adding +0 to a sum of non-negative terms leaves
// it unchanged, so skipping it does not change the result).  Columns with at
// most kShortCol entries (most of them: a point is the candidate of a few
// neighbours) are summed in entry order by one thread; longer ones (hubs,
// thousands of entries) by one warp: lane t sums the set slots of the
// column's bitmap words t, t + 32, ... in slot order, then a fixed
// xor-shuffle tree.  The split depends only on the
// column's length, so every sum has a fixed order.
constexpr int kShortCol = 32;

HAP_DEV void colstats_finish(int64_t j, int l, int L, int N, float P, const float* __restrict__ c,
                             const float* __restrict__ phi, const float* __restrict__ rdiag, float* __restrict__ b,
                             float* __restrict__ tpart) {
    const int64_t idx = (int64_t)l * N + j;
    const float rd = rdiag[idx];
    b[j * ((L + 3) & ~3) + l] = __fadd_rn(__fadd_rn(__fadd_rn(c[idx], phi[idx]), rd), P);
    if (l + 1 < L) tpart[idx + N] = __fadd_rn(rd, P);
}

// P_j of one short column (one thread, slots in order).
HAP_DEV void colstats_short_column(int64_t t, int ncols, const float* __restrict__ cval,
                                   const unsigned* __restrict__ cbits, int64_t cwords,
                                   const int64_t* __restrict__ cptr, const int32_t* __restrict__ cols, int N, int L,
                                   int K, const float* __restrict__ c, const float* __restrict__ phi,
                                   const float* __restrict__ rdiag, float* __restrict__ b, float* __restrict__ tpart) {
    if (t >= (int64_t)L * ncols) return;
    const int l = (int)(t / ncols);
    const int64_t j = cols[t - (int64_t)l * ncols];
    const float* v = cval + (int64_t)l * N * K;
    const unsigned* bits = cbits + l * cwords;
    const int64_t e0 = cptr[j], e1 = cptr[j + 1];
    float P = 0.f;
    if (e0 < e1) {
        const int64_t w0 = e0 >> 5, w1 = (e1 - 1) >> 5;
        for (int64_t w = w0; w <= w1; ++w) {
            unsigned m = bits[w];
            if (w == w0) m &= ~0u << (e0 & 31);
            if (w == w1) m &= (2u << ((e1 - 1) & 31)) - 1u;  // bits up to e1 - 1 (all 32 when it is bit 31)
            while (m) {
                P = __fadd_rn(P, v[w * 32 + __ffs(m) - 1]);
                m &= m - 1u;
            }
        }
    }
    colstats_finish(j, l, L, N, P, c, phi, rdiag, b, tpart);
}

// P_j of one long column (one warp): lane t sums the set slots of the
// column's bitmap words t, t + 32, ... in slot order, four loads in flight,
// then a fixed xor-shuffle tree.
HAP_DEV void colstats_long_column(int64_t w, int lane, int ncols, const float* __restrict__ cval,
                                  const unsigned* __restrict__ cbits, int64_t cwords,
                                  const int64_t* __restrict__ cptr, const int32_t* __restrict__ cols, int N, int L,
                                  int K, const float* __restrict__ c, const float* __restrict__ phi,
                                  const float* __restrict__ rdiag, float* __restrict__ b, float* __restrict__ tpart) {
    if (w >= (int64_t)L * ncols) return;
    const int l = (int)(w / ncols);
    const int64_t j = cols[w - (int64_t)l * ncols];
    const float* v = cval + (int64_t)l * N * K;
    const unsigned* bits = cbits + l * cwords;
    const int64_t e0 = cptr[j], e1 = cptr[j + 1];
    float P = 0.f;
    const int64_t w0 = e0 >> 5, w1 = (e1 - 1) >> 5;
    for (int64_t q = w0 + lane; e0 < e1 && q <= w1; q += 32) {
        unsigned m = bits[q];
        if (q == w0) m &= ~0u << (e0 & 31);
        if (q == w1) m &= (2u << ((e1 - 1) & 31)) - 1u;
        const float* vw = v + q * 32;
        while (m) {
            float x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                x[u] = m ? vw[__ffs(m) - 1] : 0.f;  // +0 leaves the sum unchanged
                m &= m - 1u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) P = __fadd_rn(P, x[u]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) P = __fadd_rn(P, __shfl_xor_sync(0xffffffffu, P, o));
    if (lane == 0) colstats_finish(j, l, L, N, P, c, phi, rdiag, b, tpart);
}

// The column statistics of one iteration in one launch: the first blocks sum
// the long columns (a warp each; scheduled first, they take longest), the
// next the short ones (a thread each), the last clear the bitmap the next
// iteration's row pass will fill (bitmaps alternate between iterations, so
// nothing reads it here).  The split depends only on the column's length, so
// every sum has a fixed order.
struct ColArgs {
    const float* cval;
    const unsigned* cbits;     // this iteration's bitmap [L][cwords]
    unsigned* clear_bits;      // the next iteration's bitmap, zeroed here
    int64_t cwords;            // words per level (a multiple of 4)
    const int64_t* cptr;
    const int32_t* long_cols;
    const int32_t* short_cols;
    int n_long, n_short, N, L, K;
    const float* c;
    const float* phi;
    const float* rdiag;
    float* b;
    float* tpart;
    unsigned long_blocks, short_blocks, clear_blocks;
};
__global__ void __launch_bounds__(256) sparse_colstats_kernel(const ColArgs p) {
    const unsigned blk = blockIdx.x;
    if (blk < p.long_blocks) {
        const int64_t t = (int64_t)blk * blockDim.x + threadIdx.x;
        colstats_long_column(t >> 5, threadIdx.x & 31, p.n_long, p.cval, p.cbits, p.cwords, p.cptr, p.long_cols, p.N,
                             p.L, p.K, p.c, p.phi, p.rdiag, p.b, p.tpart);
    } else if (blk < p.long_blocks + p.short_blocks) {
        const int64_t t = (int64_t)(blk - p.long_blocks) * blockDim.x + threadIdx.x;
        colstats_short_column(t, p.n_short, p.cval, p.cbits, p.cwords, p.cptr, p.short_cols, p.N, p.L, p.K, p.c,
                              p.phi, p.rdiag, p.b, p.tpart);
    } else {
        const int64_t n4 = (int64_t)p.L * p.cwords / 4;
        uint4* z = reinterpret_cast<uint4*>(p.clear_bits);
        for (int64_t q = (int64_t)(blk - p.long_blocks - p.short_blocks) * blockDim.x + threadIdx.x; q < n4;
             q += (int64_t)p.clear_blocks * blockDim.x)
            z[q] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// Column classes: flag[j] = 1 for a long column; after the prefix sums the
// columns of each class are listed in increasing order.
__global__ void column_class_kernel(const int* __restrict__ cnt, int N, int* __restrict__ is_long,
                                    int* __restrict__ is_short) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > N) return;
    const int lg = (j < N && cnt[j] > kShortCol) ? 1 : 0;
    is_long[j] = lg;
    is_short[j] = (j < N) ? 1 - lg : 0;
}
__global__ void column_compact_kernel(const int* __restrict__ is_long, const int* __restrict__ long_pos,
                                      const int* __restrict__ short_pos, int N, int32_t* __restrict__ long_cols,
                                      int32_t* __restrict__ short_cols) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    if (is_long[j]) long_cols[long_pos[j]] = j;
    else short_cols[short_pos[j]] = j;
}

// ---- candidate graph on the GPU: checks, column index (CSC) -----------------
// Every row must be strictly increasing, in range and contain its own index;
// a violation sets ST_BOUNDS.  Also counts the entries of every column.
__global__ void sparse_check_count_kernel(const int32_t* __restrict__ cand, int N, int K, unsigned* status,
                                          int* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N) return;
    bool bad = false, self = false;
    for (int q = lane; q < K; q += 32) {
        const int j = cand[i * K + q];
        const int prev = q > 0 ? cand[i * K + q - 1] : -1;
        if (j < 0 || j >= N || j <= prev) {
            bad = true;
        } else {
            atomicAdd(cnt + j, 1);
            self |= j == (int)i;
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    self = __any_sync(0xffffffffu, self);
    if (lane == 0 && (bad || !self)) atomicOr(status, ST_BOUNDS);
}

// Exclusive prefix sums of int counts (3 launches: tile sums, one-CTA scan of
// the tile sums, tile-local scans plus offsets).
// pos[cent[x]] = x: the CSC slot of every entry
__global__ void inverse_perm_kernel(const int32_t* __restrict__ cent, int64_t n, int32_t* __restrict__ pos) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n) pos[cent[x]] = (int32_t)x;
}

// s_iq = -||x_i - x_cand||^2 (FP32, direct differences); one warp per row
__global__ void sparse_similarity_kernel(const float* __restrict__ X, int64_t d, const int32_t* __restrict__ cand,
                                         int N, int K, float* __restrict__ s) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)N * K) return;
    const int64_t i = e / K;
    const int64_t j = cand[e];
    float acc = 0.f;
    for (int64_t k = 0; k < d; ++k) {
        const float df = X[i * d + k] - X[j * d + k];
        acc = fmaf(df, df, acc);
    }
    s[e] = -acc;
}

__global__ void sparse_exemplars_kernel(const int32_t* __restrict__ cand, const float* __restrict__ A,
                                        const float* __restrict__ R, const float* __restrict__ b, int N, int L, int K,
                                        int pending, float lam, float oml, int32_t* __restrict__ e,
                                        float* __restrict__ A_out) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= (int64_t)L * N) return;
    const int l = (int)(w / N);
    const int64_t i = w - (int64_t)l * N;
    float best = -kInf;
    int bj = 0x7fffffff;
    for (int q = lane; q < K; q += 32) {
        const int64_t at = w * K + q;
        const int j = cand[i * K + q];
        const float r = R[at];
        float a = A[at];
        if (pending) a = damp(a, avail_target(b[(int64_t)j * ((L + 3) & ~3) + l], r, j == i), lam, oml);
        if (A_out) A_out[at] = a;
        const float v = __fadd_rn(a, r);
        if (v > best || (v == best && j < bj)) { best = v; bj = j; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ov > best || (ov == best && oj < bj)) { best = ov; bj = oj; }
    }
    if (e && lane == 0) e[w] = bj;
}

// NS^l = sum_i s(i, e_i) with s = -||x_i - x_e||^2 in FP64 from the points
// (preference on self-assignments); one CTA per level, fixed-order tree
// NS^l = sum_i -||x_i - x_{e_i}||^2 (the preference where e_i = i) in FP64
// from the points: kNsChunks fixed chunks of the points per level, each
// summed by a fixed tree in one CTA, then the chunks in order by one thread
// per level, so the value does not depend on the launch.  ns holds
// L * (kNsChunks + 1) doubles: the chunk sums, then NS^0 .. NS^{L-1}.
constexpr int kNsChunks = 128;

__global__ void __launch_bounds__(256) netsim_points_kernel(const float* __restrict__ X, int64_t d,
                                                            const int32_t* __restrict__ e,
                                                            const float* __restrict__ pref, int N,
                                                            double* __restrict__ ns) {
    __shared__ double part[256];
    const int c = blockIdx.x, l = blockIdx.y;
    const int64_t per = ((int64_t)N + kNsChunks - 1) / kNsChunks;
    const int64_t i0 = (int64_t)c * per, i1 = i0 + per < N ? i0 + per : N;
    double acc = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int64_t j = e[(int64_t)l * N + i];
        if (j == i) { acc += (double)pref[(int64_t)l * N + i]; continue; }
        double sq = 0.0;
        for (int64_t k = 0; k < d; ++k) {
            const double df = (double)X[i * d + k] - (double)X[j * d + k];
            sq += df * df;
        }
        acc -= sq;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) ns[(int64_t)l * kNsChunks + c] = part[0];
}

__global__ void netsim_finish_kernel(double* __restrict__ ns, int L) {
    const int l = threadIdx.x;
    if (l >= L) return;
    double t = 0.0;
    for (int c = 0; c < kNsChunks; ++c) t += ns[(int64_t)l * kNsChunks + c];
    ns[(int64_t)L * kNsChunks + l] = t;
}

cudaError_t launch_netsim_points(const float* X, int64_t d, const int32_t* e, const float* pref, int N, int L,
                                 double* ns, cudaStream_t st) {
    netsim_points_kernel<<<dim3(kNsChunks, (unsigned)L), 256, 0, st>>>(X, d, e, pref, N, ns);
    netsim_finish_kernel<<<1, 32 * ((L + 31) / 32), 0, st>>>(ns, L);
    return cudaGetLastError();
}

}  // namespace
}  // namespace hap

using namespace hap;

#define SCU(x)                          \
    do {                                \
        if ((x) != cudaSuccess) {       \
            cudaGetLastError();         \
            return HAP_ECUDA;           \
        }                               \
    } while (0)

struct hap_sparse {
    int N = 0, L = 0, K = 0;
    float lam = 0.5f;
    int c_mode = HAP_C_PAPER;
    cudaStream_t stream = nullptr;
    int32_t* cand = nullptr;
    float* s = nullptr;
    float *A = nullptr, *R = nullptr;
    float *pref = nullptr, *c = nullptr, *c0 = nullptr, *tau = nullptr, *phi = nullptr, *tpart = nullptr, *b = nullptr,
          *rdiag = nullptr;
    int64_t* cptr = nullptr;
    int32_t* cent = nullptr;
    int32_t* pos = nullptr;       // [N*K] CSC slot of every entry
    float* cval = nullptr;        // [L][N*K] max(0, rho) in CSC order
    unsigned* cbits = nullptr;    // [2][L][cwords] bitmaps of the positive slots, used by alternate iterations
    int64_t cwords = 0;           // words per level, a multiple of 4
    int bm = 0;                   // the bitmap the next row pass fills
    int32_t* tmp[4] = {nullptr, nullptr, nullptr, nullptr};  // radix-sort key / value buffers
    int* cnt = nullptr;           // [N + 1] column counts
    int* cls = nullptr;           // [4][N + 1] column-class flags and positions
    int32_t* long_cols = nullptr; // columns with more than kShortCol entries, increasing
    int32_t* short_cols = nullptr;
    int n_long = 0, n_short = 0;
    int* hist = nullptr;          // radix histograms, then their offsets
    int* hoff = nullptr;
    int64_t* tsum = nullptr;      // scan tile sums
    int32_t* e = nullptr;
    double* ns = nullptr;         // [L][kNsChunks] chunk sums of the net similarity, then [L] totals
    unsigned* status = nullptr;
    const float* X = nullptr;  // points of the last hap_sparse_set_candidates (borrowed for NS)
    int64_t d = 0;
    int64_t iter = 0;
    bool pending = false;
    int64_t launches = 0;
    bool profile = false;
    std::vector<cudaEvent_t> ev;   // per profiled iteration: before the row pass, after it, after the
                                   // column statistics
    double prof_ms[2] = {0, 0};
    int64_t prof_n = 0;
};

namespace {

int sparse_reset(hap_sparse* h) {
    const size_t mat = (size_t)h->L * h->N * h->K * 4, vec = (size_t)h->L * h->N * 4;
    SCU(cudaMemsetAsync(h->A, 0, mat, h->stream));
    SCU(cudaMemsetAsync(h->R, 0, mat, h->stream));
    SCU(cudaMemcpyAsync(h->c, h->c0, vec, cudaMemcpyDeviceToDevice, h->stream));
    SCU(cudaMemsetAsync(h->phi, 0, vec, h->stream));
    SCU(cudaMemsetAsync(h->tpart, 0, vec, h->stream));
    SCU(cudaMemsetAsync(h->b, 0, (size_t)h->N * ((h->L + 3) & ~3) * 4, h->stream));
    SCU(cudaMemsetAsync(h->rdiag, 0, vec, h->stream));
    SCU(cudaMemsetAsync(h->cbits, 0, (size_t)2 * h->L * h->cwords * 4, h->stream));
    h->bm = 0;
    std::vector<float> inf((size_t)h->L * h->N, __builtin_inff());
    SCU(cudaMemcpyAsync(h->tau, inf.data(), vec, cudaMemcpyHostToDevice, h->stream));
    SCU(cudaStreamSynchronize(h->stream));
    h->iter = 0;
    h->pending = false;
    return HAP_OK;
}

}  // namespace

extern "C" {

int hap_sparse_create(int64_t N, int L, int K, const float* prefs, float damping, int c_mode, hap_sparse** out) {
    if (!out || N < 2 || L < 1 || L > 16 || K < 2 || K > SP_MAXK || K > N || !(damping > 0.f && damping < 1.f) ||
        (c_mode != HAP_C_PAPER && c_mode != HAP_C_FIXED) || N * K >= (int64_t)1 << 31)
        return HAP_EINVAL;
    hap_sparse* h = new (std::nothrow) hap_sparse();
    if (!h) return HAP_ENOMEM;
    h->N = (int)N;
    h->L = L;
    h->K = K;
    h->lam = damping;
    h->c_mode = c_mode;
    h->cwords = (int64_t)((N * K + 127) / 128) * 4;
    const size_t nk = (size_t)N * K, mat = nk * L * 4, vec = (size_t)L * N * 4;
    bool ok = cudaMalloc(&h->cand, nk * 4) == cudaSuccess && cudaMalloc(&h->s, nk * 4) == cudaSuccess &&
              cudaMalloc(&h->A, mat) == cudaSuccess && cudaMalloc(&h->R, mat) == cudaSuccess &&
              cudaMalloc(&h->pref, vec) == cudaSuccess && cudaMalloc(&h->c, vec) == cudaSuccess &&
              cudaMalloc(&h->c0, vec) == cudaSuccess && cudaMalloc(&h->tau, vec) == cudaSuccess &&
              cudaMalloc(&h->phi, vec) == cudaSuccess && cudaMalloc(&h->tpart, vec) == cudaSuccess &&
              cudaMalloc(&h->b, (size_t)N * ((L + 3) & ~3) * 4) == cudaSuccess &&
              cudaMalloc(&h->rdiag, vec) == cudaSuccess &&
              cudaMalloc(&h->cptr, (N + 1) * 8) == cudaSuccess && cudaMalloc(&h->cent, nk * 4) == cudaSuccess &&
              cudaMalloc(&h->e, (size_t)L * N * 4) == cudaSuccess && cudaMalloc(&h->ns, (size_t)L * (kNsChunks + 1) * 8) == cudaSuccess &&
              cudaMalloc(&h->status, 16) == cudaSuccess && cudaMalloc(&h->pos, nk * 4) == cudaSuccess &&
              cudaMalloc(&h->cval, mat) == cudaSuccess && cudaMalloc(&h->cnt, (N + 1) * 4) == cudaSuccess &&
              cudaMalloc(&h->cbits, (size_t)2 * L * h->cwords * 4) == cudaSuccess &&
              cudaMalloc(&h->cls, (size_t)4 * (N + 1) * 4) == cudaSuccess &&
              cudaMalloc(&h->long_cols, (size_t)N * 4) == cudaSuccess &&
              cudaMalloc(&h->short_cols, (size_t)N * 4) == cudaSuccess;
    const int64_t nhist = radix_hist_size((int64_t)nk);
    const int64_t ntiles = scan_tiles(std::max<int64_t>(nhist, N + 1));
    for (int q = 0; q < 4 && ok; ++q) ok = cudaMalloc(&h->tmp[q], nk * 4) == cudaSuccess;
    ok = ok && cudaMalloc(&h->hist, nhist * 4) == cudaSuccess && cudaMalloc(&h->hoff, nhist * 4) == cudaSuccess &&
         cudaMalloc(&h->tsum, ntiles * 8) == cudaSuccess;
    if (!ok) { cudaGetLastError(); hap_sparse_destroy(h); return HAP_ENOMEM; }
    cudaMemset(h->c0, 0, vec);
    cudaMemset(h->status, 0, 16);
    std::vector<float> pv((size_t)L * N, 0.f);
    if (prefs)
        for (int l = 0; l < L; ++l)
            for (int64_t i = 0; i < N; ++i) pv[(size_t)l * N + i] = prefs[l];
    cudaMemcpy(h->pref, pv.data(), vec, cudaMemcpyHostToDevice);
    int rc = sparse_reset(h);
    if (rc) { hap_sparse_destroy(h); return rc; }
    *out = h;
    return HAP_OK;
}

void hap_sparse_destroy(hap_sparse* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    cudaFree(h->cand); cudaFree(h->s); cudaFree(h->A); cudaFree(h->R); cudaFree(h->pref); cudaFree(h->c);
    cudaFree(h->c0); cudaFree(h->tau); cudaFree(h->phi); cudaFree(h->tpart); cudaFree(h->b); cudaFree(h->rdiag);
    cudaFree(h->cptr); cudaFree(h->cent); cudaFree(h->e); cudaFree(h->ns); cudaFree(h->status);
    cudaFree(h->pos); cudaFree(h->cval); cudaFree(h->cbits); cudaFree(h->cnt); cudaFree(h->hist); cudaFree(h->hoff); cudaFree(h->tsum);
    cudaFree(h->cls); cudaFree(h->long_cols); cudaFree(h->short_cols);
    for (int q = 0; q < 4; ++q) cudaFree(h->tmp[q]);
    delete h;
}

int hap_sparse_set_profile(hap_sparse* h, int on) {
    if (!h || (on != 0 && on != 1)) return HAP_EINVAL;
    h->profile = on != 0;
    return HAP_OK;
}

int hap_sparse_profile_times(hap_sparse* h, double* ms, int64_t* iterations, int reset) {
    if (!h || !ms || !iterations) return HAP_EINVAL;
    SCU(cudaStreamSynchronize(h->stream));
    for (size_t q = 0; q + 2 < h->ev.size(); q += 3) {
        for (int k = 0; k < 2; ++k) {
            float t = 0.f;
            SCU(cudaEventElapsedTime(&t, h->ev[q + k], h->ev[q + k + 1]));
            h->prof_ms[k] += t;
        }
        h->prof_n += 1;
        for (int k = 0; k < 3; ++k) cudaEventDestroy(h->ev[q + k]);
    }
    h->ev.clear();
    for (int k = 0; k < 2; ++k) ms[k] = h->prof_ms[k];
    *iterations = h->prof_n;
    if (reset) {
        for (double& v : h->prof_ms) v = 0.0;
        h->prof_n = 0;
    }
    return HAP_OK;
}

int hap_sparse_set_stream(hap_sparse* h, void* stream) {
    if (!h) return HAP_EINVAL;
    h->stream = static_cast<cudaStream_t>(stream);
    return HAP_OK;
}

int hap_sparse_set_preferences(hap_sparse* h, const float* prefs, int per_point) {
    if (!h || !prefs) return HAP_EINVAL;
    std::vector<float> pv((size_t)h->L * h->N);
    for (int l = 0; l < h->L; ++l)
        for (int i = 0; i < h->N; ++i) pv[(size_t)l * h->N + i] = per_point ? prefs[(size_t)l * h->N + i] : prefs[l];
    SCU(cudaMemcpyAsync(h->pref, pv.data(), pv.size() * 4, cudaMemcpyHostToDevice, h->stream));
    SCU(cudaStreamSynchronize(h->stream));
    return HAP_OK;
}

int hap_sparse_set_candidates(hap_sparse* h, const int32_t* cand, const float* X, int64_t d) {
    if (!h || !cand || !X || d < 1) return HAP_EINVAL;
    const int64_t N = h->N, K = h->K, nk = N * K;
    cudaStream_t st = h->stream;
    SCU(cudaMemcpyAsync(h->cand, cand, nk * 4, cudaMemcpyDeviceToDevice, st));
    // checks (sorted, distinct, in range, contains the row) and column counts
    SCU(cudaMemsetAsync(h->cnt, 0, (N + 1) * 4, st));
    SCU(cudaMemsetAsync(h->status, 0, 16, st));
    sparse_check_count_kernel<<<(unsigned)((N * 32 + 255) / 256), 256, 0, st>>>(h->cand, (int)N, (int)K, h->status, h->cnt);
    SCU(cudaGetLastError());
    SCU(scan_exclusive(h->cnt, N + 1, h->cptr, h->tsum, st));
    // columns by length class, each list in increasing column order
    int* is_long = h->cls;
    int* is_short = h->cls + (N + 1);
    int* long_pos = h->cls + 2 * (N + 1);
    int* short_pos = h->cls + 3 * (N + 1);
    column_class_kernel<<<(unsigned)((N + 1 + 255) / 256), 256, 0, st>>>(h->cnt, (int)N, is_long, is_short);
    SCU(scan_exclusive(is_long, N + 1, long_pos, h->tsum, st));
    SCU(scan_exclusive(is_short, N + 1, short_pos, h->tsum, st));
    column_compact_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(is_long, long_pos, short_pos, (int)N,
                                                                       h->long_cols, h->short_cols);
    SCU(cudaGetLastError());
    // entries sorted by column, stable: the CSC entry order
    int passes = 1;
    while (passes * kRadixBits < 31 && ((int64_t)1 << (passes * kRadixBits)) < N) ++passes;
    const int32_t* kin = h->cand;
    const int32_t* vin = nullptr;  // first pass: value = entry index
    for (int p = 0; p < passes; ++p) {
        const bool last = p + 1 == passes;
        int32_t* ko = (kin == h->tmp[0]) ? h->tmp[2] : h->tmp[0];
        int32_t* vo = last ? h->cent : ((vin == h->tmp[1]) ? h->tmp[3] : h->tmp[1]);
        SCU(radix_pass(kin, vin, nk, p * kRadixBits, h->hist, h->hoff, h->tsum, ko, vo, st));
        kin = ko;
        vin = vo;
    }
    inverse_perm_kernel<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(h->cent, nk, h->pos);
    sparse_similarity_kernel<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(X, d, h->cand, (int)N, (int)K, h->s);
    SCU(cudaGetLastError());
    h->launches += 6 + 3 * passes + 3 * passes + 8;  // checks, scans, sort passes, classes, inverse map, s
    unsigned stw = 0;
    int nl = 0;
    SCU(cudaMemcpyAsync(&stw, h->status, 4, cudaMemcpyDeviceToHost, st));
    SCU(cudaMemcpyAsync(&nl, long_pos + N, 4, cudaMemcpyDeviceToHost, st));
    SCU(cudaStreamSynchronize(st));
    h->n_long = nl;
    h->n_short = (int)N - nl;
    if (stw & ST_BOUNDS) {
        SCU(cudaMemset(h->status, 0, 16));
        return HAP_EINVAL;
    }
    h->X = X;
    h->d = d;
    return sparse_reset(h);
}

int hap_sparse_iterate(hap_sparse* h, int n) {
    if (!h || n < 0) return HAP_EINVAL;
    SparseArgs a;
    a.cand = h->cand; a.pos = h->pos; a.cval = h->cval; a.cwords = h->cwords;
    a.s = h->s; a.A = h->A; a.R = h->R; a.pref = h->pref; a.c = h->c; a.tau = h->tau;
    a.phi = h->phi; a.tpart = h->tpart; a.b = h->b; a.rdiag = h->rdiag; a.status = h->status;
    a.N = h->N; a.L = h->L; a.K = h->K; a.Lb = (h->L + 3) & ~3; a.lam = h->lam; a.oml = 1.0f - h->lam;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t warps = std::min<int64_t>(h->N, (int64_t)sms * 64);
    const unsigned grid = (unsigned)((warps * 32 + 255) / 256);
    ColArgs ca;
    ca.cval = h->cval; ca.cwords = h->cwords; ca.cptr = h->cptr; ca.long_cols = h->long_cols;
    ca.short_cols = h->short_cols; ca.n_long = h->n_long; ca.n_short = h->n_short; ca.N = h->N; ca.L = h->L;
    ca.K = h->K; ca.c = h->c; ca.phi = h->phi; ca.rdiag = h->rdiag; ca.b = h->b; ca.tpart = h->tpart;
    ca.long_blocks = (unsigned)(((int64_t)h->L * h->n_long * 32 + 255) / 256);
    ca.short_blocks = (unsigned)(((int64_t)h->L * h->n_short + 255) / 256);
    ca.clear_blocks = (unsigned)sms * 2;
    const size_t bm_words = (size_t)h->L * h->cwords;
    for (int it = 0; it < n; ++it) {
        const int64_t t = h->iter + 1;
        a.pending = h->pending ? 1 : 0;
        a.update_c = (h->c_mode == HAP_C_PAPER && t >= 2) ? 1 : 0;
        a.use_tau = t >= 2 ? 1 : 0;
        a.cbits = h->cbits + (size_t)h->bm * bm_words;
        ca.cbits = a.cbits;
        ca.clear_bits = h->cbits + (size_t)(h->bm ^ 1) * bm_words;
        cudaEvent_t ev[3] = {};
        if (h->profile) {
            for (auto& e : ev) SCU(cudaEventCreate(&e));
            SCU(cudaEventRecord(ev[0], h->stream));
        }
        if (h->L > 4)
            sparse_rowpass_kernel<true, false><<<grid, 256, 0, h->stream>>>(a);
        else if (h->K == 64)
            sparse_rowpass_kernel<false, true><<<grid, 256, 0, h->stream>>>(a);
        else
            sparse_rowpass_kernel<false, false><<<grid, 256, 0, h->stream>>>(a);
        SCU(cudaGetLastError());
        if (h->profile) SCU(cudaEventRecord(ev[1], h->stream));
        sparse_colstats_kernel<<<ca.long_blocks + ca.short_blocks + ca.clear_blocks, 256, 0, h->stream>>>(ca);
        SCU(cudaGetLastError());
        if (h->profile) {
            SCU(cudaEventRecord(ev[2], h->stream));
            h->ev.insert(h->ev.end(), ev, ev + 3);
        }
        h->launches += 2;
        h->bm ^= 1;
        h->pending = true;
        h->iter = t;
    }
    return HAP_OK;
}

int hap_sparse_exemplars(hap_sparse* h, int32_t* e, int on_host) {
    if (!h || !e || (on_host != 0 && on_host != 1)) return HAP_EINVAL;
    const int64_t rows = (int64_t)h->L * h->N;
    sparse_exemplars_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, h->stream>>>(
        h->cand, h->A, h->R, h->b, h->N, h->L, h->K, h->pending, h->lam, 1.0f - h->lam, h->e, nullptr);
    SCU(cudaGetLastError());
    h->launches += 1;
    SCU(cudaMemcpyAsync(e, h->e, rows * 4, on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
    if (on_host) SCU(cudaStreamSynchronize(h->stream));
    return HAP_OK;
}

int hap_net_similarity_points(const float* X, int64_t N, int64_t d, int L, const int32_t* e, const float* pref,
                              double* ns_host, void* stream) {
    if (!X || !e || !pref || !ns_host || N < 1 || L < 1) return HAP_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* dns = nullptr;
    SCU(cudaMallocAsync(&dns, (size_t)L * (kNsChunks + 1) * 8, st));
    SCU(launch_netsim_points(X, d, e, pref, (int)N, L, dns, st));
    SCU(cudaMemcpyAsync(ns_host, dns + (size_t)L * kNsChunks, (size_t)L * 8, cudaMemcpyDeviceToHost, st));
    SCU(cudaFreeAsync(dns, st));
    SCU(cudaStreamSynchronize(st));
    return HAP_OK;
}

int hap_sparse_net_similarity(hap_sparse* h, double* ns) {
    if (!h || !ns || !h->X) return HAP_EINVAL;
    const int64_t rows = (int64_t)h->L * h->N;
    sparse_exemplars_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, h->stream>>>(
        h->cand, h->A, h->R, h->b, h->N, h->L, h->K, h->pending, h->lam, 1.0f - h->lam, h->e, nullptr);
    SCU(cudaGetLastError());
    SCU(launch_netsim_points(h->X, h->d, h->e, h->pref, h->N, h->L, h->ns, h->stream));
    h->launches += 3;
    SCU(cudaMemcpyAsync(ns, h->ns + (size_t)h->L * kNsChunks, (size_t)h->L * 8, cudaMemcpyDeviceToHost, h->stream));
    SCU(cudaStreamSynchronize(h->stream));
    return HAP_OK;
}

int hap_sparse_get_state(hap_sparse* h, float* A, float* R, float* vecs, int64_t* iter) {
    if (!h) return HAP_EINVAL;
    const int64_t rows = (int64_t)h->L * h->N, mat = rows * h->K;
    if (A) {
        sparse_exemplars_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, h->stream>>>(
            h->cand, h->A, h->R, h->b, h->N, h->L, h->K, h->pending, h->lam, 1.0f - h->lam, nullptr, A);
        SCU(cudaGetLastError());
        h->launches += 1;
    }
    if (R) SCU(cudaMemcpyAsync(R, h->R, mat * 4, cudaMemcpyDeviceToDevice, h->stream));
    if (vecs) {
        const float* src[3] = {h->c, h->tau, h->phi};
        for (int q = 0; q < 3; ++q)
            SCU(cudaMemcpyAsync(vecs + (size_t)q * rows, src[q], rows * 4, cudaMemcpyDeviceToDevice, h->stream));
    }
    if (iter) *iter = h->iter;
    return HAP_OK;
}

int hap_sparse_query(hap_sparse* h, int key, int64_t* value) {
    if (!h || !value) return HAP_EINVAL;
    if (key == HAP_Q_ITER) { *value = h->iter; return HAP_OK; }
    if (key == HAP_Q_LAUNCHES) { *value = h->launches; return HAP_OK; }
    return HAP_EINVAL;
}

}  // extern "C"
