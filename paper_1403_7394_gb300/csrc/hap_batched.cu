// Batched HAP: many independent instances of uneven N and L advanced by ONE
// persistent row-pass launch per iteration (plus one batched column-statistics
// launch), replayed from a CUDA graph.
//
// Work items are (instance, band) pairs: band g of an instance owns the row
// blocks g, g + G, g + 2G, ... (a block = `rps` consecutive rows, which are
// contiguous in memory, so one TMA bulk copy per tensor moves a whole block).
// A 512-thread CTA (16 warps) is split into rps row groups of g whole warps,
// g = ceil(ld / (32 * 4K)) with 4K columns per thread, rps = floor(16 / g);
// each group holds one row of the block, so instances with small N process
// up to 16 rows per step and every instance keeps at least 15 of 16 warps
// busy for g <= 5.  Groups synchronise only among themselves (a named barrier
// per group); a stage of the TMA ring is refilled once every warp has
// released it (an "empty" mbarrier per stage), so groups never wait for a
// CTA-wide barrier.  Each thread keeps the running column sums of max(0, rho)
// of its columns for all levels of the current item in tensor memory (TMEM),
// so shared memory holds only the ring; at the end of an item every group
// writes its sums as one partial row (band * rps + group) and the batched
// column-statistics kernel sums an instance's partial rows in order
// (fixed-order reductions, bitwise reproducible for a fixed schedule).  The
// equations are those of the single-instance row pass (Eqs. 2.1-2.6 with
// damping, §3 schedule).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "hap.h"
#include "hap_common.cuh"
#include "hap_internal.h"

namespace hap {
namespace {

constexpr int kBT = 512;            // threads per CTA
constexpr int kBW = kBT / 32;       // warps per CTA
constexpr int kBMaxLd = 4096;       // longest row the batched path takes
// 16 columns per thread when every instance has at most 8 levels (TMEM holds
// 4 warp slots x L x 16 columns <= 512), else 8 columns per thread.
__host__ __device__ constexpr int b_stages(int K) { return K == 4 ? 2 : 4; }
__host__ __device__ constexpr int b_stage_elems(int K) { return kBT * 4 * K; }

struct BInst {
    float* A;
    float* R;
    const void* S;
    const float* pref;
    float* c;
    float* tau;
    float* phi;
    float* tpart;
    float* b;
    float* rdiag;
    float* partials;  // [G * rps][L][ld]: one row per (band, row group)
    int N, L, ld, rps, g, G;
};
struct BItem {
    int inst, band, nsteps;
};
struct BatchArgs {
    const BInst* inst;
    const BItem* items;
    int* counter;          // next unclaimed item (zeroed before every launch)
    int n_items;           // items, sorted by decreasing work
    unsigned* status;
    float lam, oml;
    int pending, update_c, use_tau;
    uint64_t wait_ns;      // limit of every bounded wait
};

size_t batched_smem_bytes(int K, int s_elem) {
    const size_t E = (size_t)b_stage_elems(K);
    const size_t stage = 2 * E * 4 + E * s_elem;
    const size_t bytes = b_stages(K) * stage + 2 * kBW * 16 + 2 * b_stages(K) * 8 + 8 + 4 * (b_stages(K) + 2) + 256;
    // more than half an SM's shared memory: one CTA per SM, so its TMEM
    // allocation never waits for another CTA
    return std::max<size_t>(bytes, 116 * 1024);
}

int batched_tmem_cols(int K, int maxL) {
    int n = 32;
    while (n < 4 * maxL * 4 * K) n *= 2;
    return n;
}

HAP_DEV void named_barrier(int id, int threads) {
    asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(threads) : "memory");
}

template <typename ST>
HAP_DEV float4 bload_s(const ST* p);
template <>
HAP_DEV float4 bload_s<float>(const float* p) { return *reinterpret_cast<const float4*>(p); }
template <>
HAP_DEV float4 bload_s<__nv_bfloat16>(const __nv_bfloat16* p) {
    return SVec<__nv_bfloat16>::to_f4(*reinterpret_cast<const uint2*>(p));
}

template <typename ST, int K>
__global__ void __launch_bounds__(kBT, 1) rowpass_batched_kernel(const BatchArgs p, int maxL, int tcols) {
    constexpr int NST = b_stages(K);
    constexpr int E = b_stage_elems(K);
    constexpr uint32_t A_BYTES = E * 4, S_BYTES = E * sizeof(ST);
    constexpr uint32_t STAGE = 2 * A_BYTES + S_BYTES;
    extern __shared__ __align__(128) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float4* red = reinterpret_cast<float4*>(sm + NST * STAGE);  // [2][kBW] warp summaries
    const uint32_t full0 = smem_addr(red + 2 * kBW);            // full[NST] (TMA landed)
    const uint32_t empty0 = full0 + 8 * NST;                    // empty[NST] (every warp released)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(red + 2 * kBW) + 4 * NST;
    // items claimed by the producer, in claim order; -1 = no more work
    constexpr int F = NST + 2;
    int* fifo = reinterpret_cast<int*>(tslot + 2);
    // the current item's descriptors (read from shared memory where used, which
    // keeps them out of registers) and the producer's cursor
    struct BProd {
        int pi, pq, issued, claimed, done;
    };
    BInst* s_in = reinterpret_cast<BInst*>(reinterpret_cast<unsigned char*>(fifo + F) +
                                           ((16 - (reinterpret_cast<uintptr_t>(fifo + F) & 15)) & 15));
    BItem* s_it = reinterpret_cast<BItem*>(s_in + 1);
    BProd* prod = reinterpret_cast<BProd*>(s_it + 1);
    const uint32_t sm0 = smem_addr(sm);
    const float lam = p.lam, oml = p.oml;
    const bool pending = p.pending != 0;

    if (tid == 0) {
        for (int q = 0; q < NST; ++q) {
            mbar_init(full0 + 8 * q, 1);
            mbar_init(empty0 + 8 * q, kBW);
        }
        fence_mbarrier_init();
    }
    if (warp == 0) tmem_alloc(smem_addr(tslot), (uint32_t)tcols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // this thread's sums of level l: lane 32*(warp%4)+lane, columns tq + l*4K ..
    const uint32_t tq = *tslot + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * maxL * 4 * K);
    bool bad = false;

    // ---- producer (thread 0): claims items from the global list (largest
    // first) and streams their steps ahead of the consumers.  Which CTA takes
    // which item does not change any result: every item writes only its own
    // rows and partial rows.
    if (tid == 0) *prod = BProd{-1, 0, 0, 0, 0};
    auto issue_next = [&]() {
        BProd c = *prod;
        if (c.done) return false;
        while (c.pi < 0 || c.pq >= p.items[c.pi].nsteps) {
            c.pi = atomicAdd(p.counter, 1);
            c.pq = 0;
            fifo[c.claimed % F] = c.pi < p.n_items ? c.pi : -1;
            ++c.claimed;
            if (c.pi >= p.n_items) {
                c.done = 1;
                *prod = c;
                return false;
            }
        }
        const int pi = c.pi, pq = c.pq, issued = c.issued;
        const BItem itm = p.items[pi];
        const BInst in = p.inst[itm.inst];
        const int m = pq / in.L, l = pq % in.L;
        const int i0 = (itm.band + m * in.G) * in.rps;
        const int nrows = min(in.rps, in.N - i0);
        const int st = issued % NST;
        // the stage's previous contents (step issued - NST) must be released by every warp
        if (issued >= NST && !bad) bad = !mbar_wait(empty0 + 8 * st, (uint32_t)((issued / NST - 1) & 1), p.status, p.wait_ns);
        // after a wait gave up nothing more is issued (the stage may still be read)
        if (bad) {
            *prod = c;
            return false;
        }
        const uint32_t bar = full0 + 8 * st, dst = sm0 + (uint32_t)st * STAGE;
        const bool load_s = l == 0;
        const uint32_t n = (uint32_t)nrows * (uint32_t)in.ld;
        mbar_arrive_expect_tx(bar, n * (8u + (load_s ? (uint32_t)sizeof(ST) : 0u)));
        const int64_t off = ((int64_t)l * in.N + i0) * in.ld;
        bulk_g2s(dst, in.A + off, n * 4u, bar);
        bulk_g2s(dst + A_BYTES, in.R + off, n * 4u, bar);
        if (load_s) bulk_g2s(dst + 2 * A_BYTES, static_cast<const ST*>(in.S) + (int64_t)i0 * in.ld, n * (uint32_t)sizeof(ST), bar);
        c.pq = pq + 1;
        c.issued = issued + 1;
        *prod = c;
        return true;
    };
    if (tid == 0)
        for (int q = 0; q < NST; ++q)
            if (!issue_next()) break;
    __syncthreads();  // the first claimed item is in fifo[0]

    int step = 0;    // consumer step counter of this CTA (ring position)
    int waited = 0;  // steps whose copies this thread saw land
    for (int kit = 0;; ++kit) {
        // read by every thread after a CTA barrier: the item is CTA-uniform
        const int it = fifo[kit % F];
        if (it < 0) break;
        if (tid == 0) {
            *s_it = p.items[it];
            *s_in = p.inst[s_it->inst];
        }
        __syncthreads();
        const BItem itm = *s_it;
        const BInst& in = *s_in;
        const int g = in.g, tg = 32 * g, rps = in.rps;
        const int r = warp / g;
        const bool active = r < rps;  // warps beyond rps * g only keep the ring in step
        const int t = (warp - r * g) * 32 + lane;
        const int L = in.L, N = in.N;
        const int64_t ld = in.ld;
        int col[K];
        bool ok[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            col[k] = 4 * (k * tg + t);
            ok[k] = active && col[k] < (int)ld;
        }
        {
            float z[4 * K];
#pragma unroll
            for (int q = 0; q < 4 * K; ++q) z[q] = 0.f;
            __syncwarp();
            for (int ll = 0; ll < L; ++ll) tmem_store<4 * K>(tq + (uint32_t)(ll * 4 * K), z);
        }
        float4 srow[K];
#pragma unroll
        for (int k = 0; k < K; ++k) srow[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        float c_prev = 0.f;
        // per-column b and per-row scalars of the next step, loaded ahead
        float4 nb[K];
        float npref = 0.f, nc = 0.f, ntp = 0.f;
        auto prefetch = [&](int q) {
            const int pm = q / L, pl = q % L;
            const int prow = (itm.band + pm * in.G) * rps + r;
            const bool prv = active && prow < N;
            const int64_t pv = (int64_t)pl * ld;
#pragma unroll
            for (int k = 0; k < K; ++k)
                nb[k] = (pending && ok[k] && prv) ? __ldg(reinterpret_cast<const float4*>(in.b + pv + col[k])) : f4_splat(0.f);
            npref = prv ? __ldg(in.pref + pv + prow) : 0.f;
            nc = (!p.update_c && prv) ? in.c[pv + prow] : 0.f;
            ntp = (p.use_tau && pl > 0 && prv) ? __ldg(in.tpart + pv + prow) : 0.f;
        };
        if (itm.nsteps > 0) prefetch(0);
        for (int q = 0; q < itm.nsteps; ++q, ++step) {
            const int m = q / L, l = q % L;
            const int i0 = (itm.band + m * in.G) * rps;
            const int row = i0 + r;
            const bool rv = active && row < N;  // this group's row exists
            const float pref_i = npref, c_fixed = nc, tpart_i = ntp;
            const int st = step % NST;
            const unsigned char* base = sm + (size_t)st * STAGE;
            const int rr0 = active ? r : 0;
            const float* sA = reinterpret_cast<const float*>(base) + (size_t)rr0 * ld;
            const float* sR = reinterpret_cast<const float*>(base + A_BYTES) + (size_t)rr0 * ld;
            const ST* sS = reinterpret_cast<const ST*>(base + 2 * A_BYTES) + (size_t)rr0 * ld;
            if (!bad) {
                bad = !mbar_wait(full0 + 8 * st, (uint32_t)(step / NST) & 1u, p.status, p.wait_ns);
                if (!bad) ++waited;
            }
            const int64_t voff = (int64_t)l * ld;
            const int64_t off = ((int64_t)l * N + row) * ld;

            // ---- pass 1: pending availability (Eqs. 2.2/2.3), row statistics ------
            float m1 = -kInf, m2 = -kInf, cm = -kInf;
            int k1 = 0x7fffffff;
            float4 rr[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float4 a4 = f4_splat(-kInf), r4 = f4_splat(0.f), s4 = f4_splat(0.f);
                const bool live = ok[k] && rv;
                if (live) {
                    a4 = *reinterpret_cast<const float4*>(sA + col[k]);
                    r4 = *reinterpret_cast<const float4*>(sR + col[k]);
                    if (l == 0) srow[k] = bload_s<ST>(sS + col[k]);
                    s4 = srow[k];
                }
                float4 an = a4;
                const float4 b4 = nb[k];
                if (pending) {
                    an.x = damp(a4.x, avail_target(b4.x, r4.x, false), lam, oml);
                    an.y = damp(a4.y, avail_target(b4.y, r4.y, false), lam, oml);
                    an.z = damp(a4.z, avail_target(b4.z, r4.z, false), lam, oml);
                    an.w = damp(a4.w, avail_target(b4.w, r4.w, false), lam, oml);
                }
                const int dd = row - col[k];
                if ((unsigned)dd < 4u) {
                    f4_set(s4, dd, pref_i);
                    if (pending) f4_set(an, dd, damp(f4_get(a4, dd), avail_target(f4_get(b4, dd), f4_get(r4, dd), true), lam, oml));
                }
                if (pending && live && !bad) st_stream(in.A + off + col[k], an);
                top2_push(__fadd_rn(an.x, s4.x), col[k] + 0, m1, k1, m2);
                top2_push(__fadd_rn(an.y, s4.y), col[k] + 1, m1, k1, m2);
                top2_push(__fadd_rn(an.z, s4.z), col[k] + 2, m1, k1, m2);
                top2_push(__fadd_rn(an.w, s4.w), col[k] + 3, m1, k1, m2);
                cm = fmaxf(cm, fmaxf(fmaxf(__fadd_rn(an.x, r4.x), __fadd_rn(an.y, r4.y)),
                                     fmaxf(__fadd_rn(an.z, r4.z), __fadd_rn(an.w, r4.w))));
                rr[k] = r4;
            }
            // this warp has read stage st; b and the row scalars of the next step
            // load while the reductions and pass 2 run
            __syncwarp();
            if (lane == 0) mbar_arrive_local(empty0 + 8 * st);
            if (q + 1 < itm.nsteps) prefetch(q + 1);
            // ---- exact reduction within the row group ----------------------------
            warp_top2(m1, k1, m2, cm);
            const int par = step & 1;
            if (lane == 0) red[par * kBW + warp] = make_float4(m1, m2, cm, __int_as_float(k1));
            if (g == 1) __syncwarp();
            else if (active) named_barrier(1 + r, tg);
            m1 = m2 = cm = -kInf;
            k1 = 0x7fffffff;
            if (active) {
                for (int w = 0; w < g; ++w) {
                    const float4 v = red[par * kBW + r * g + w];
                    top2_merge(m1, k1, m2, v.x, __float_as_int(v.w), v.y);
                    cm = fmaxf(cm, v.z);
                }
            }
            if (tid == 0) issue_next();  // refills stage st once every warp released it
            // ---- inter-level messages (Eqs. 2.4-2.6) ---------------------------
            const float cval = p.update_c ? cm : c_fixed;
            const float tauv = (p.use_tau && l > 0 && rv) ? __fadd_rn(c_prev, tpart_i) : kInf;
            c_prev = cval;
            if (rv && t == 0 && !bad) {
                if (p.update_c) in.c[voff + row] = cval;
                in.tau[voff + row] = tauv;
                if (l > 0) in.phi[voff - ld + row] = m1;
            }
            // ---- responsibilities (Eq. 2.1) and column sums ------------------------
            const float mm1 = fminf(tauv, -m1), mm2 = fminf(tauv, -m2);
            float addv[4 * K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float4 r4 = rr[k];
                float4 s4 = (ok[k] && rv) ? srow[k] : f4_splat(0.f);
                const int dd = row - col[k];
                if ((unsigned)dd < 4u) f4_set(s4, dd, pref_i);
                // min(tau, -max_{k != j}): mm2 at the row's argmax k1, mm1 elsewhere
                const int dk = k1 - col[k];
                float4 rn;
                rn.x = damp(r4.x, __fadd_rn(s4.x, dk == 0 ? mm2 : mm1), lam, oml);
                rn.y = damp(r4.y, __fadd_rn(s4.y, dk == 1 ? mm2 : mm1), lam, oml);
                rn.z = damp(r4.z, __fadd_rn(s4.z, dk == 2 ? mm2 : mm1), lam, oml);
                rn.w = damp(r4.w, __fadd_rn(s4.w, dk == 3 ? mm2 : mm1), lam, oml);
                float4 add = make_float4(fmaxf(rn.x, 0.f), fmaxf(rn.y, 0.f), fmaxf(rn.z, 0.f), fmaxf(rn.w, 0.f));
                if (!(ok[k] && rv)) add = f4_splat(0.f);
                if ((unsigned)dd < 4u) {
                    f4_set(add, dd, 0.f);
                    if (rv && !bad) in.rdiag[voff + row] = f4_get(rn, dd);
                }
                if (ok[k] && rv && !bad) st_stream(in.R + off + col[k], rn);
                addv[4 * k + 0] = add.x;
                addv[4 * k + 1] = add.y;
                addv[4 * k + 2] = add.z;
                addv[4 * k + 3] = add.w;
            }
            __syncwarp();  // tcgen05.ld / st are warp-collective
            float cur[4 * K];
            const uint32_t ta = tq + (uint32_t)(l * 4 * K);
            tmem_load<4 * K>(ta, cur);
#pragma unroll
            for (int q2 = 0; q2 < 4 * K; ++q2) cur[q2] = __fadd_rn(cur[q2], addv[q2]);
            tmem_store<4 * K>(ta, cur);
        }
        // ---- this item's sums: partial row (band * rps + group) -------------------
        for (int ll = 0; ll < L; ++ll) {
            float cur[4 * K];
            __syncwarp();
            tmem_load<4 * K>(tq + (uint32_t)(ll * 4 * K), cur);
            if (active) {
                float* dst = in.partials + ((int64_t)(itm.band * rps + r) * L + ll) * ld;
#pragma unroll
                for (int k = 0; k < K; ++k)
                    if (ok[k])
                        *reinterpret_cast<float4*>(dst + col[k]) =
                            make_float4(cur[4 * k], cur[4 * k + 1], cur[4 * k + 2], cur[4 * k + 3]);
            }
        }
        // The next item may group the warps differently: no warp may reuse a
        // named-barrier id with another thread count while a group of this
        // item still waits on it.  A timed-out wait anywhere ends the CTA's
        // work uniformly (the status word already records it).
        if (__syncthreads_or(bad)) break;
    }
    // After a wait gave up: every bulk copy this CTA issued lands before it
    // leaves (thread 0 issued them all and saw the first `waited` land; each
    // stage has at most one copy in flight, since a stage is re-armed only
    // after its previous copy was consumed).
    if (tid == 0)
        for (int q = waited; q < prod->issued; ++q)
            mbar_wait(full0 + 8 * (q % NST), (uint32_t)(q / NST) & 1u, p.status, kWaitNs);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(*tslot, (uint32_t)tcols);
}

// Column statistics of every instance: one thread per (instance, level, column);
// G is the instance's number of partial rows (bands x row groups).
struct BCol {
    const float* partials;
    const float* c;
    const float* phi;
    const float* rdiag;
    float* b;
    float* tpart;
    int N, L, ld, G;
    int64_t first;  // first flat index of this instance
};
__global__ void colstats_batched_kernel(const BCol* __restrict__ cols, int B, int64_t total) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int lo = 0, hi = B - 1;
    while (lo < hi) {  // last instance whose first index <= idx
        const int mid = (lo + hi + 1) >> 1;
        if (cols[mid].first <= idx) lo = mid; else hi = mid - 1;
    }
    const BCol in = cols[lo];
    const int64_t rel = idx - in.first;
    const int l = (int)(rel / in.N);
    const int64_t j = rel - (int64_t)l * in.N;
    const float* pp = in.partials + (int64_t)l * in.ld + j;
    float P = 0.f;
    for (int q = 0; q < in.G; ++q) P = __fadd_rn(P, pp[(int64_t)q * in.L * in.ld]);
    const int64_t v = (int64_t)l * in.ld + j;
    const float rd = in.rdiag[v];
    in.b[v] = __fadd_rn(__fadd_rn(__fadd_rn(in.c[v], in.phi[v]), rd), P);
    if (l + 1 < in.L) in.tpart[v + in.ld] = __fadd_rn(rd, P);
}

// Eq. 2.8 for every (instance, level, row): one warp per row.
__global__ void exemplars_batched_kernel(const BInst* __restrict__ inst, const int64_t* __restrict__ row_first,
                                         const int64_t* __restrict__ e_first, int B, int64_t total_rows,
                                         int pending, float lam, float oml, int32_t* __restrict__ e) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= total_rows) return;
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row_first[mid] <= gw) lo = mid; else hi = mid - 1;
    }
    const BInst in = inst[lo];
    const int64_t rel = gw - row_first[lo];
    const int l = (int)(rel / in.N);
    const int64_t i = rel - (int64_t)l * in.N;
    const float* Ar = in.A + rel * in.ld;
    const float* Rr = in.R + rel * in.ld;
    float best = -kInf;
    int bi = 0x7fffffff;
    for (int64_t j = lane; j < in.N; j += 32) {
        const float r = Rr[j];
        float a = Ar[j];
        if (pending) a = damp(a, avail_target(in.b[(int64_t)l * in.ld + j], r, j == i), lam, oml);
        const float v = __fadd_rn(a, r);
        if (v > best) { best = v; bi = (int)j; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) e[e_first[lo] + rel] = bi;
}

// NS^l of every (instance, level) in FP64, fixed-order tree per block.
template <typename ST>
__global__ void netsim_batched_kernel(const BInst* __restrict__ inst, const int* __restrict__ lev_inst,
                                      const int* __restrict__ lev_l, const int64_t* __restrict__ e_first,
                                      const int32_t* __restrict__ e, double* __restrict__ ns) {
    __shared__ double part[256];
    const int q = blockIdx.x, b = lev_inst[q], l = lev_l[q];
    const BInst in = inst[b];
    const ST* S = static_cast<const ST*>(in.S);
    double accd = 0.0;
    for (int64_t i = threadIdx.x; i < in.N; i += blockDim.x) {
        const int64_t ej = e[e_first[b] + (int64_t)l * in.N + i];
        accd += (ej == i) ? (double)in.pref[(int64_t)l * in.ld + i] : (double)(float)S[i * in.ld + ej];
    }
    part[threadIdx.x] = accd;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) ns[q] = part[0];
}

}  // namespace
}  // namespace hap

using namespace hap;

struct hap_batch {
    int B = 0;
    std::vector<int64_t> N;
    std::vector<int> L, ld;
    hap_options opt{};
    float lam = 0.5f;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    int s_bf16 = 0;
    int maxL = 1;
    int K = 4;                       // float4 groups per thread (16 columns; 8 when an instance has > 8 levels)
    int tcols = 32;                  // TMEM columns of a row-pass CTA
    float* partials = nullptr;       // all instances' partial rows (sized by the schedule)
    size_t partials_bytes = 0;
    std::vector<BInst> inst;         // host copy of the descriptors
    std::vector<size_t> inst_bytes;  // workspace bytes per instance (before partials)
    BInst* d_inst = nullptr;
    BCol* d_cols = nullptr;
    BItem* d_items = nullptr;
    int* d_counter = nullptr;        // item claim counter of the row pass
    int n_items = 0;
    int64_t* d_row_first = nullptr;
    int64_t* d_e_first = nullptr;
    int* d_lev_inst = nullptr;
    int* d_lev_l = nullptr;
    int32_t* d_e = nullptr;
    double* d_ns = nullptr;
    unsigned* status = nullptr;
    void* build_scratch = nullptr;   // operands of the tensor-core build
    size_t build_scratch_bytes = 0;
    std::vector<float*> c0;          // per instance initial c (device)
    int64_t total_cols = 0, total_rows = 0, total_levels = 0;
    int grid = 0;                    // persistent CTAs
    int items_per_cta = 2;           // scheduling granularity (autotuned)
    int64_t iter = 0;
    bool pending = false;
    cudaGraphExec_t graph = nullptr;
    int64_t launches = 0;
};

namespace {

constexpr size_t kAl = 256;
size_t al(size_t x) { return (x + kAl - 1) / kAl * kAl; }

#define BCU(x)                              \
    do {                                    \
        if ((x) != cudaSuccess) {           \
            cudaGetLastError();             \
            return HAP_ECUDA;               \
        }                                   \
    } while (0)

// Row groups for a row of ld columns at 4K columns per thread: g whole warps
// per row (32 g 4K >= ld), rps = floor(16 / g) rows per step.
void group_shape(int ld, int K, int* rps, int* g) {
    *g = (ld + 32 * 4 * K - 1) / (32 * 4 * K);
    *rps = kBW / *g;
}

// Tile width of the batch's row pass: 4K columns per thread (16 with a 2-stage
// ring of 8192-element steps, or 8 with a 4-stage ring of 4096-element steps),
// with every instance's row groups re-derived from it.  16 columns need
// every instance to have at most 8 levels (TMEM holds 4 warp slots x L x 16
// columns).  The schedule is rebuilt by the caller.
int set_tile(hap_batch* h, int K) {
    if (K != 4 && K != 2) return HAP_EINVAL;
    if (K == 4 && h->maxL > 8) return HAP_EUNSUPPORTED;
    h->K = K;
    h->tcols = batched_tmem_cols(K, h->maxL);
    for (int b = 0; b < h->B; ++b) group_shape(h->ld[b], K, &h->inst[b].rps, &h->inst[b].g);
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return HAP_OK;
}

// Bands per instance (total ~ items_per_cta x grid, proportional to work) and
// a longest-processing-time assignment of items to the persistent CTAs.
int schedule(hap_batch* h) {
    const int B = h->B;
    std::vector<double> work(B);
    double tot = 0;
    for (int b = 0; b < B; ++b) {
        work[b] = (double)h->N[b] * h->N[b] * h->L[b];
        tot += work[b];
    }
    const double target = tot / ((double)h->grid * h->items_per_cta);
    std::vector<BItem> items;
    std::vector<double> iw;
    for (int b = 0; b < B; ++b) {
        const int nblk = (int)((h->N[b] + h->inst[b].rps - 1) / h->inst[b].rps);
        int G = (int)(work[b] / target + 0.5);
        G = std::max(1, std::min(G, nblk));
        h->inst[b].G = G;
        for (int g = 0; g < G; ++g) {
            const int blocks = nblk > g ? (nblk - 1 - g) / G + 1 : 0;
            items.push_back(BItem{b, g, blocks * h->L[b]});
            iw.push_back((double)blocks * h->inst[b].rps * h->N[b] * h->L[b]);
        }
    }
    std::vector<int> order(items.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return iw[a] > iw[b]; });
    // partial rows: G bands x rps groups per instance
    size_t need = 0;
    std::vector<size_t> poff(B);
    for (int b = 0; b < B; ++b) {
        poff[b] = need;
        need += al((size_t)h->inst[b].G * h->inst[b].rps * h->L[b] * h->ld[b] * 4);
    }
    if (need > h->partials_bytes) {
        if (h->partials) cudaFree(h->partials);
        h->partials = nullptr;
        h->partials_bytes = 0;
        BCU(cudaMalloc(&h->partials, need));
        h->partials_bytes = need;
    }
    for (int b = 0; b < B; ++b)
        h->inst[b].partials = reinterpret_cast<float*>(reinterpret_cast<char*>(h->partials) + poff[b]);
    // one list, largest items first: CTAs claim them in this order (dynamic
    // longest-processing-time balancing)
    std::vector<BItem> flat;
    for (int o : order) flat.push_back(items[o]);
    h->n_items = (int)flat.size();
    if (h->d_items) cudaFree(h->d_items);
    BCU(cudaMalloc(&h->d_items, std::max<size_t>(1, flat.size()) * sizeof(BItem)));
    BCU(cudaMemcpy(h->d_items, flat.data(), flat.size() * sizeof(BItem), cudaMemcpyHostToDevice));
    BCU(cudaMemcpy(h->d_inst, h->inst.data(), B * sizeof(BInst), cudaMemcpyHostToDevice));
    std::vector<BCol> cols(B);
    int64_t first = 0;
    for (int b = 0; b < B; ++b) {
        const BInst& in = h->inst[b];
        cols[b] = BCol{in.partials, in.c, in.phi, in.rdiag, in.b, in.tpart, in.N, in.L, in.ld, in.G * in.rps, first};
        first += (int64_t)in.L * in.N;
    }
    BCU(cudaMemcpy(h->d_cols, cols.data(), B * sizeof(BCol), cudaMemcpyHostToDevice));
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return HAP_OK;
}

// Algorithm 1's initial values for every instance; clears a reported device
// error.
int batch_reset(hap_batch* h) {
    BCU(cudaMemsetAsync(h->status, 0, 16, h->stream));
    for (int b = 0; b < h->B; ++b) {
        const BInst& in = h->inst[b];
        const size_t mat = (size_t)in.L * in.N * in.ld * 4, vec = (size_t)in.L * in.ld * 4;
        BCU(cudaMemsetAsync(in.A, 0, mat, h->stream));
        BCU(launch_fill_alpha_padding(in.A, (int64_t)in.L * in.N, in.N, in.ld, h->stream));
        BCU(cudaMemsetAsync(in.R, 0, mat, h->stream));
        BCU(cudaMemcpyAsync(in.c, h->c0[b], vec, cudaMemcpyDeviceToDevice, h->stream));
        BCU(cudaMemsetAsync(in.phi, 0, vec, h->stream));
        BCU(cudaMemsetAsync(in.tpart, 0, vec, h->stream));
        BCU(cudaMemsetAsync(in.b, 0, vec, h->stream));
        BCU(cudaMemsetAsync(in.rdiag, 0, vec, h->stream));
        std::vector<float> inf(in.L * (size_t)in.ld, __builtin_inff());
        BCU(cudaMemcpyAsync(in.tau, inf.data(), vec, cudaMemcpyHostToDevice, h->stream));
        BCU(cudaStreamSynchronize(h->stream));
    }
    h->iter = 0;
    h->pending = false;
    return HAP_OK;
}

cudaError_t launch_batched_iteration(hap_batch* h, int pending, int update_c, int use_tau, cudaStream_t st) {
    BatchArgs a;
    a.inst = h->d_inst;
    a.items = h->d_items;
    a.counter = h->d_counter;
    a.n_items = h->n_items;
    cudaError_t err0 = cudaMemsetAsync(h->d_counter, 0, sizeof(int), st);
    if (err0 != cudaSuccess) return err0;
    a.status = h->status;
    a.wait_ns = h->opt.wait_limit_ns > 0 ? (uint64_t)h->opt.wait_limit_ns : 2000000000ull;
    a.lam = h->lam;
    a.oml = 1.0f - h->lam;
    a.pending = pending;
    a.update_c = update_c;
    a.use_tau = use_tau;
    const size_t smem = batched_smem_bytes(h->K, h->s_bf16 ? 2 : 4);
    if (h->K == 4) {
        if (h->s_bf16)
            rowpass_batched_kernel<__nv_bfloat16, 4><<<h->grid, kBT, smem, st>>>(a, h->maxL, h->tcols);
        else
            rowpass_batched_kernel<float, 4><<<h->grid, kBT, smem, st>>>(a, h->maxL, h->tcols);
    } else {
        if (h->s_bf16)
            rowpass_batched_kernel<__nv_bfloat16, 2><<<h->grid, kBT, smem, st>>>(a, h->maxL, h->tcols);
        else
            rowpass_batched_kernel<float, 2><<<h->grid, kBT, smem, st>>>(a, h->maxL, h->tcols);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const unsigned blocks = (unsigned)((h->total_cols + 255) / 256);
    colstats_batched_kernel<<<blocks, 256, 0, st>>>(h->d_cols, h->B, h->total_cols);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int hap_batch_create(int B, const int64_t* N, const int* L, float damping, const hap_options* opt,
                     hap_batch** out) {
    if (!out || B < 1 || !N || !L || !(damping > 0.f && damping < 1.f)) return HAP_EINVAL;
    *out = nullptr;
    hap_options o;
    hap_default_options(&o);
    if (opt) o = *opt;
    if (o.c_mode != HAP_C_PAPER && o.c_mode != HAP_C_FIXED) return HAP_EINVAL;
    if (o.schedule != HAP_SCHED_JACOBI || o.kappa != 0.f) return HAP_EUNSUPPORTED;
    hap_batch* h = new (std::nothrow) hap_batch();
    if (!h) return HAP_ENOMEM;
    h->B = B;
    h->opt = o;
    h->lam = damping;
    h->s_bf16 = o.s_dtype == HAP_S_BF16;
    h->N.assign(N, N + B);
    h->L.assign(L, L + B);
    size_t total = 0;
    int maxL = 1;
    for (int b = 0; b < B; ++b) {
        if (N[b] < 2 || L[b] < 1 || L[b] > 16) { delete h; return HAP_EINVAL; }
        const int64_t ldb = (N[b] + 31) / 32 * 32;
        if (ldb > kBMaxLd) { delete h; return HAP_EUNSUPPORTED; }
        h->ld.push_back((int)ldb);
        maxL = std::max(maxL, L[b]);
    }
    h->maxL = maxL;
    h->K = maxL <= 8 ? 4 : 2;
    h->tcols = batched_tmem_cols(h->K, maxL);
    int dev = 0, sms = 0, smem_limit = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // the shared-memory opt-in of both tile widths is set here, never inside a
    // stream capture (the autotuner may switch between them)
    for (int K : {4, 2}) {
        if (K == 4 && maxL > 8) continue;
        const size_t smem = batched_smem_bytes(K, h->s_bf16 ? 2 : 4);
        if (smem > (size_t)smem_limit || batched_tmem_cols(K, maxL) > 512) { delete h; return HAP_EUNSUPPORTED; }
        cudaError_t fa = K == 4
            ? cudaFuncSetAttribute(h->s_bf16 ? (const void*)rowpass_batched_kernel<__nv_bfloat16, 4>
                                             : (const void*)rowpass_batched_kernel<float, 4>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
            : cudaFuncSetAttribute(h->s_bf16 ? (const void*)rowpass_batched_kernel<__nv_bfloat16, 2>
                                             : (const void*)rowpass_batched_kernel<float, 2>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (fa != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return HAP_ECUDA;
        }
    }
    h->grid = sms;
    // workspace: per instance A, R, S, 8 vectors (the partial rows are sized
    // by the schedule, in a buffer of their own)
    std::vector<size_t> off(B);
    h->inst.resize(B);
    for (int b = 0; b < B; ++b) {
        int rps, g;
        group_shape(h->ld[b], h->K, &rps, &g);
        h->inst[b].rps = rps;
        h->inst[b].g = g;
        const size_t mat = (size_t)L[b] * N[b] * h->ld[b] * 4;
        const size_t vec = (size_t)L[b] * h->ld[b] * 4;
        const size_t s = (size_t)N[b] * h->ld[b] * (h->s_bf16 ? 2 : 4);
        off[b] = total;
        total += al(mat) * 2 + al(s) + 8 * al(vec);
    }
    int64_t ecount = 0, levels = 0;
    for (int b = 0; b < B; ++b) { ecount += (int64_t)L[b] * N[b]; levels += L[b]; }
    const size_t e_off = total;
    total += al((size_t)ecount * 4) + al((size_t)levels * 8) + al(16);
    size_t xs = 0;
    for (int b = 0; b < B; ++b) xs = std::max(xs, sbuild_tc_scratch_bytes(N[b], 256, 1));
    const size_t xs_off = total;
    total += al(xs);
    if (cudaMalloc(&h->ws, total) != cudaSuccess) { cudaGetLastError(); delete h; return HAP_ENOMEM; }
    h->own_ws = true;
    h->ws_bytes = total;
    char* base = static_cast<char*>(h->ws);
    for (int b = 0; b < B; ++b) {
        BInst& in = h->inst[b];
        const size_t mat = al((size_t)L[b] * N[b] * h->ld[b] * 4), vec = al((size_t)L[b] * h->ld[b] * 4);
        const size_t s = al((size_t)N[b] * h->ld[b] * (h->s_bf16 ? 2 : 4));
        char* p = base + off[b];
        in.A = reinterpret_cast<float*>(p); p += mat;
        in.R = reinterpret_cast<float*>(p); p += mat;
        in.S = p; p += s;
        float* v[8];
        for (int q = 0; q < 8; ++q) { v[q] = reinterpret_cast<float*>(p); p += vec; }
        in.pref = v[0]; in.c = v[1]; in.tau = v[2]; in.phi = v[3]; in.tpart = v[4]; in.b = v[5]; in.rdiag = v[6];
        h->c0.push_back(v[7]);
        in.partials = nullptr;
        in.N = (int)N[b];
        in.L = L[b];
        in.ld = h->ld[b];
        in.G = 1;
    }
    h->d_e = reinterpret_cast<int32_t*>(base + e_off);
    h->d_ns = reinterpret_cast<double*>(base + e_off + al((size_t)ecount * 4));
    h->status = reinterpret_cast<unsigned*>(base + e_off + al((size_t)ecount * 4) + al((size_t)levels * 8));
    h->build_scratch = base + xs_off;
    h->build_scratch_bytes = al(xs);
    h->total_cols = ecount;
    h->total_rows = ecount;
    h->total_levels = levels;
    std::vector<int64_t> row_first(B), e_first(B);
    std::vector<int> lev_inst, lev_l;
    int64_t acc = 0;
    for (int b = 0; b < B; ++b) {
        row_first[b] = acc;
        e_first[b] = acc;
        acc += (int64_t)L[b] * N[b];
        for (int l = 0; l < L[b]; ++l) { lev_inst.push_back(b); lev_l.push_back(l); }
    }
    bool okm = cudaMalloc(&h->d_inst, B * sizeof(BInst)) == cudaSuccess &&
               cudaMalloc(&h->d_cols, B * sizeof(BCol)) == cudaSuccess &&
               cudaMalloc(&h->d_row_first, B * sizeof(int64_t)) == cudaSuccess &&
               cudaMalloc(&h->d_e_first, B * sizeof(int64_t)) == cudaSuccess &&
               cudaMalloc(&h->d_lev_inst, levels * sizeof(int)) == cudaSuccess &&
               cudaMalloc(&h->d_lev_l, levels * sizeof(int)) == cudaSuccess &&
               cudaMalloc(&h->d_counter, sizeof(int)) == cudaSuccess &&
               cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    if (!okm) { cudaGetLastError(); hap_batch_destroy(h); return HAP_ENOMEM; }
    cudaMemcpy(h->d_row_first, row_first.data(), B * sizeof(int64_t), cudaMemcpyHostToDevice);
    cudaMemcpy(h->d_e_first, e_first.data(), B * sizeof(int64_t), cudaMemcpyHostToDevice);
    cudaMemcpy(h->d_lev_inst, lev_inst.data(), levels * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(h->d_lev_l, lev_l.data(), levels * sizeof(int), cudaMemcpyHostToDevice);
    for (int b = 0; b < B; ++b) {
        const BInst& in = h->inst[b];
        const size_t vec = (size_t)in.L * in.ld * 4;
        cudaMemset(const_cast<float*>(in.pref), 0, vec);
        cudaMemset(h->c0[b], 0, vec);
        cudaMemset(const_cast<void*>(in.S), 0, (size_t)in.N * in.ld * (h->s_bf16 ? 2 : 4));
    }
    cudaMemset(h->status, 0, 16);
    int rc = schedule(h);
    if (!rc) rc = batch_reset(h);
    if (rc) { hap_batch_destroy(h); return rc; }
    *out = h;
    return HAP_OK;
}

void hap_batch_destroy(hap_batch* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    cudaFree(h->d_inst);
    cudaFree(h->d_cols);
    cudaFree(h->d_items);
    cudaFree(h->d_counter);
    cudaFree(h->d_row_first);
    cudaFree(h->d_e_first);
    cudaFree(h->d_lev_inst);
    cudaFree(h->d_lev_l);
    cudaFree(h->partials);
    if (h->own_ws) cudaFree(h->ws);
    delete h;
}

int hap_batch_set_stream(hap_batch* h, void* stream) {
    if (!h) return HAP_EINVAL;
    h->stream = static_cast<cudaStream_t>(stream);
    return HAP_OK;
}

int hap_batch_set_preferences(hap_batch* h, const float* prefs) {
    if (!h || !prefs) return HAP_EINVAL;
    int64_t q = 0;
    for (int b = 0; b < h->B; ++b) {
        const BInst& in = h->inst[b];
        std::vector<float> host((size_t)in.L * in.ld, 0.f);
        for (int l = 0; l < in.L; ++l) {
            const float v = prefs[q++];
            if (!(v > -__builtin_inff() && v < __builtin_inff())) return HAP_EINVAL;
            for (int i = 0; i < in.N; ++i) host[(size_t)l * in.ld + i] = v;
        }
        BCU(cudaMemcpyAsync(const_cast<float*>(in.pref), host.data(), host.size() * 4, cudaMemcpyHostToDevice, h->stream));
        BCU(cudaStreamSynchronize(h->stream));
    }
    return HAP_OK;
}

int hap_batch_build_similarity(hap_batch* h, const float* X, int64_t d, int mode) {
    if (!h || !X || d < 1) return HAP_EINVAL;
    // operand scratch of the tensor-core build, reused in stream order
    const size_t scratch_cap = h->build_scratch_bytes;
    int64_t row0 = 0;
    for (int b = 0; b < h->B; ++b) {
        const BInst& in = h->inst[b];
        const float* Xb = X + row0 * d;
        row0 += in.N;
        if (mode == HAP_SBUILD_F32) {
            BCU(launch_sbuild_f32(Xb, in.N, d, const_cast<void*>(in.S), h->s_bf16, in.ld, h->stream));
            h->launches += 1;
        } else if (mode == HAP_SBUILD_BF16 || mode == HAP_SBUILD_BF16_SPLIT) {
            const int split = mode == HAP_SBUILD_BF16_SPLIT;
            if (sbuild_tc_scratch_bytes(in.N, d, split) > scratch_cap) return HAP_EUNSUPPORTED;
            int nk = 0;
            cudaError_t err = launch_sbuild_tc(Xb, in.N, d, split, const_cast<void*>(in.S), h->s_bf16, in.ld,
                                               h->build_scratch, h->status, h->stream, &nk);
            if (err == cudaErrorNotSupported) return HAP_EUNSUPPORTED;
            BCU(err);
            h->launches += nk;
        } else {
            return HAP_EINVAL;
        }
    }
    return batch_reset(h);
}

int hap_batch_set_similarity(hap_batch* h, int b, const void* S, int64_t ld, int dtype) {
    if (!h || b < 0 || b >= h->B || !S || ld < h->N[b] || (dtype != HAP_S_F32 && dtype != HAP_S_BF16)) return HAP_EINVAL;
    const BInst& in = h->inst[b];
    BCU(launch_copy_similarity(const_cast<void*>(in.S), h->s_bf16, in.ld, S, dtype == HAP_S_BF16, ld, in.N, h->stream));
    h->launches += 1;
    return batch_reset(h);
}

int hap_batch_iterate(hap_batch* h, int n) {
    if (!h || n < 0) return HAP_EINVAL;
    for (int it = 0; it < n; ++it) {
        const int64_t t = h->iter + 1;
        const int update_c = (h->opt.c_mode == HAP_C_PAPER && t >= 2) ? 1 : 0;
        if (t >= 2 && h->pending) {
            // steady state: one CUDA graph of (batched row pass, batched column statistics)
            if (!h->graph) {
                cudaGraph_t g = nullptr;
                BCU(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
                cudaError_t err = launch_batched_iteration(h, 1, update_c, 1, h->cap_stream);
                cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
                if (err != cudaSuccess || e2 != cudaSuccess) { cudaGetLastError(); if (g) cudaGraphDestroy(g); return HAP_ECUDA; }
                err = cudaGraphInstantiate(&h->graph, g, 0);
                cudaGraphDestroy(g);
                BCU(err);
            }
            BCU(cudaGraphLaunch(h->graph, h->stream));
        } else {
            BCU(launch_batched_iteration(h, h->pending ? 1 : 0, update_c, t >= 2 ? 1 : 0, h->stream));
        }
        h->launches += 2;
        h->pending = true;
        h->iter = t;
    }
    return HAP_OK;
}

int hap_batch_exemplars(hap_batch* h, int32_t* e, int on_host) {
    if (!h || !e || (on_host != 0 && on_host != 1)) return HAP_EINVAL;
    const unsigned blocks = (unsigned)((h->total_rows * 32 + 255) / 256);
    exemplars_batched_kernel<<<blocks, 256, 0, h->stream>>>(h->d_inst, h->d_row_first, h->d_e_first, h->B, h->total_rows,
                                                           h->pending, h->lam, 1.0f - h->lam, h->d_e);
    BCU(cudaGetLastError());
    h->launches += 1;
    BCU(cudaMemcpyAsync(e, h->d_e, (size_t)h->total_rows * 4, on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                        h->stream));
    if (on_host) BCU(cudaStreamSynchronize(h->stream));
    return HAP_OK;
}

int hap_batch_net_similarity(hap_batch* h, double* ns) {
    if (!h || !ns) return HAP_EINVAL;
    const unsigned blocks = (unsigned)((h->total_rows * 32 + 255) / 256);
    exemplars_batched_kernel<<<blocks, 256, 0, h->stream>>>(h->d_inst, h->d_row_first, h->d_e_first, h->B, h->total_rows,
                                                           h->pending, h->lam, 1.0f - h->lam, h->d_e);
    BCU(cudaGetLastError());
    if (h->s_bf16)
        netsim_batched_kernel<__nv_bfloat16><<<(unsigned)h->total_levels, 256, 0, h->stream>>>(
            h->d_inst, h->d_lev_inst, h->d_lev_l, h->d_e_first, h->d_e, h->d_ns);
    else
        netsim_batched_kernel<float><<<(unsigned)h->total_levels, 256, 0, h->stream>>>(
            h->d_inst, h->d_lev_inst, h->d_lev_l, h->d_e_first, h->d_e, h->d_ns);
    BCU(cudaGetLastError());
    h->launches += 2;
    BCU(cudaMemcpyAsync(ns, h->d_ns, (size_t)h->total_levels * 8, cudaMemcpyDeviceToHost, h->stream));
    BCU(cudaStreamSynchronize(h->stream));
    unsigned st = 0;
    BCU(cudaMemcpy(&st, h->status, 4, cudaMemcpyDeviceToHost));
    if (st & ST_TIMEOUT) return HAP_ETIMEOUT;
    if (st) return HAP_EDEVICE;
    return HAP_OK;
}

int hap_batch_get_state(hap_batch* h, int b, float* A, float* R, float* vecs, int64_t* iter) {
    if (!h || b < 0 || b >= h->B) return HAP_EINVAL;
    const BInst& in = h->inst[b];
    const int64_t N = in.N, L = in.L, ld = in.ld;
    if (A) {
        BCU(launch_materialize_A(A, in.A, in.R, in.b, h->pending, h->lam, 1.0f - h->lam, N, ld, (int)L, h->stream));
        h->launches += 1;
    }
    if (R)
        BCU(cudaMemcpy2DAsync(R, N * 4, in.R, ld * 4, N * 4, (size_t)(L * N), cudaMemcpyDeviceToDevice, h->stream));
    if (vecs) {
        const float* src[3] = {in.c, in.tau, in.phi};
        for (int q = 0; q < 3; ++q)
            BCU(cudaMemcpy2DAsync(vecs + (size_t)q * L * N, N * 4, src[q], ld * 4, N * 4, (size_t)L,
                                  cudaMemcpyDeviceToDevice, h->stream));
    }
    if (iter) *iter = h->iter;
    return HAP_OK;
}

// Autotuner: times one steady-state iteration (CUDA events) for every tile
// width (16 columns per thread and 8192-element steps in a 2-stage ring, or 8
// columns and 4096-element steps in a 4-stage ring: narrow rows fill the
// small steps, e.g. 16 rows of 256 columns, where they fill half a large one)
// and every scheduling granularity in {2, 4, 6, 8, 12, 16} items per CTA
// (finer items balance the dynamic claiming better but cost a CTA barrier,
// TMEM zeroing and partial rows each), and keeps the fastest pair; the
// messages are reset to Algorithm 1's start afterwards.
int hap_batch_tune(hap_batch* h, double* best_ms) {
    if (!h) return HAP_EINVAL;
    const int cands[6] = {2, 4, 6, 8, 12, 16};
    double best = 1e30;
    int best_c = h->items_per_cta, best_k = h->K;
    cudaEvent_t e0, e1;
    BCU(cudaEventCreate(&e0));
    BCU(cudaEventCreate(&e1));
    for (int K : {4, 2}) {
        if (set_tile(h, K) != HAP_OK) continue;
        for (int c : cands) {
            h->items_per_cta = c;
            int rc = schedule(h);
            if (rc) return rc;
            rc = batch_reset(h);
            if (rc) return rc;
            BCU(launch_batched_iteration(h, 0, 0, 0, h->stream));  // warm-up (t = 1)
            BCU(cudaEventRecord(e0, h->stream));
            for (int r = 0; r < 3; ++r) BCU(launch_batched_iteration(h, 1, h->opt.c_mode == HAP_C_PAPER, 1, h->stream));
            BCU(cudaEventRecord(e1, h->stream));
            BCU(cudaEventSynchronize(e1));
            float ms = 0.f;
            BCU(cudaEventElapsedTime(&ms, e0, e1));
            if (ms / 3 < best) {
                best = ms / 3;
                best_c = c;
                best_k = K;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int rc = set_tile(h, best_k);
    h->items_per_cta = best_c;
    if (!rc) rc = schedule(h);
    if (!rc) rc = batch_reset(h);
    if (best_ms) *best_ms = best;
    return rc;
}

int hap_batch_set_tile(hap_batch* h, int elems_per_thread) {
    if (!h || (elems_per_thread != 16 && elems_per_thread != 8)) return HAP_EINVAL;
    int rc = set_tile(h, elems_per_thread / 4);
    if (!rc) rc = schedule(h);
    if (!rc) rc = batch_reset(h);
    return rc;
}

int hap_batch_query(hap_batch* h, int key, int64_t* value) {
    if (!h || !value) return HAP_EINVAL;
    switch (key) {
        case HAP_Q_ITER: *value = h->iter; return HAP_OK;
        case HAP_Q_LAUNCHES: *value = h->launches; return HAP_OK;
        case HAP_Q_GRID_CLUSTERS: *value = h->grid; return HAP_OK;
        case HAP_Q_BATCH_ITEMS_PER_CTA: *value = h->items_per_cta; return HAP_OK;
        case HAP_Q_ELEMS_PER_THREAD: *value = 4 * h->K; return HAP_OK;
        default: return HAP_EINVAL;
    }
}

int hap_batch_set_wait_limit(hap_batch* h, int64_t ns) {
    if (!h || ns < 0) return HAP_EINVAL;
    h->opt.wait_limit_ns = ns;
    if (h->graph) {  // the captured launches carry the old limit
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return HAP_OK;
}

int hap_batch_sync(hap_batch* h) {
    if (!h) return HAP_EINVAL;
    BCU(cudaStreamSynchronize(h->stream));
    unsigned st = 0;
    BCU(cudaMemcpy(&st, h->status, 4, cudaMemcpyDeviceToHost));
    if (st & ST_TIMEOUT) return HAP_ETIMEOUT;
    if (st) return HAP_EDEVICE;
    return HAP_OK;
}

}  // extern "C"
