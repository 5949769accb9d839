// The fused row-pass kernel template (see hap_rowpass.cu for the schedule)
// and its launch helpers, shared by the translation units that instantiate
// it: hap_rowpass.cu (the kernels every iteration runs), hap_rowpass_dbg.cu
// (the debug_bounds variants, whose index checks are compiled in only there,
// so the kernels without them carry no dead branch) and hap_rowpass_band.cu
// (the row-band variants, whose row offset is likewise compiled in only there).
#pragma once

#include "hap_common.cuh"
#include "hap_internal.h"

namespace hap {

constexpr int kStages = 3;  // TMA ring depth of the shared-memory-sums variant

// Shared memory of one row-pass CTA: nst x {A, R, S slices} | per-thread
// column sums [L][K][T] float4 (not in the TMEM variant) | exchange slots
// [2][C][32] float4 | mbarriers full[nst], xfull[2] | TMEM address slot.
__host__ __device__ inline size_t rowpass_smem_layout(int T, int K, int C, int L, int s_elem, int nst, bool tm,
                                                      size_t* stage_bytes, size_t* a_bytes) {
    const size_t W = (size_t)4 * K * T;
    const size_t a = (W * 4 + 127) / 128 * 128;
    const size_t sb = (W * s_elem + 127) / 128 * 128;
    if (stage_bytes) *stage_bytes = 2 * a + sb;
    if (a_bytes) *a_bytes = a;
    return nst * (2 * a + sb) + (tm ? 0 : (size_t)L * W * 4) + (size_t)2 * C * 32 * 16 + (nst + 2) * 8 + 8;
}

// TMEM columns of the TMEM variant: the warps sharing a lane quarter (T/128
// of them) each hold L x 4K consecutive columns; allocation is a power of two
// of at least 32 columns.
__host__ __device__ inline int rowpass_tmem_cols(int T, int K, int L) {
    const int need = (T / 128) * L * 4 * K;
    int n = 32;
    while (n < need) n *= 2;
    return n;
}

template <typename ST>
HAP_DEV float4 load_s_smem(const ST* p);
template <>
HAP_DEV float4 load_s_smem<float>(const float* p) { return *reinterpret_cast<const float4*>(p); }
template <>
HAP_DEV float4 load_s_smem<__nv_bfloat16>(const __nv_bfloat16* p) {
    return SVec<__nv_bfloat16>::to_f4(*reinterpret_cast<const uint2*>(p));
}

// BAND: A, R and S hold a band of rows (RowPassArgs::row0 / nrows); the other
// instances have row0 = 0 and nrows = N folded in at compile time.
template <typename ST, int K, int MAXT, int NST, bool TM, bool DBG, bool BAND = false>
__global__ void __launch_bounds__(MAXT, 1) rowpass_kernel(const RowPassArgs p) {
    static_assert(!TM || K == 2 || K == 4, "TMEM column sums use 8 or 16 columns per thread");
    extern __shared__ __align__(128) unsigned char sm[];
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    const unsigned C = cluster_nctarank(), rank = cluster_ctarank();
    const unsigned g = cluster_id_x(), G = cluster_count_x();
    const int L = p.L;
    const int N = (int)p.N;                            // columns (points)
    const int NR = BAND ? (int)p.nrows : N;            // rows held: R0 .. R0 + NR - 1
    const int R0 = BAND ? (int)p.row0 : 0;
    const int64_t ld = p.ld;
    const float lam = p.lam, oml = p.oml;
    const bool pending = p.pending != 0;
    const bool s_each_level = p.s_level_stride != 0;
    const bool kap = p.kappa != 0.f;  // shared S only (checked on the host)
    const ST* Sb = reinterpret_cast<const ST*>(p.S);

    // ---- shared memory carve-up ------------------------------------------------
    size_t stage_bytes, a_bytes;
    rowpass_smem_layout(T, K, (int)C, L, (int)sizeof(ST), NST, TM, &stage_bytes, &a_bytes);
    float4* acc = reinterpret_cast<float4*>(sm + NST * stage_bytes);    // [L][K][T] (shared-memory sums)
    float4* xbuf = acc + (TM ? 0 : (size_t)L * K * T);                  // [2][C][32]
    const uint32_t bar0 = smem_addr(xbuf + 2 * C * 32);                 // full[NST], xfull[2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(xbuf + 2 * C * 32) + 2 * (NST + 2);
    const uint32_t sm0 = smem_addr(sm);
    // TMEM variant: this thread's sums of level l live in lane 32*(warp%4)+lane,
    // columns tacc + l*4K .. +4K-1.
    const int tcols = TM ? rowpass_tmem_cols(T, K, L) : 0;
    uint32_t tacc = 0;

    // ---- columns of this thread: slice of CTA `rank`, 4 consecutive per group
    const int W = 4 * K * T;
    const int slice0 = (int)rank * W;
    const int slice_len = max(0, min(W, (int)ld - slice0));
    int col[K];
    bool ok[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        col[k] = slice0 + 4 * (k * T + tid);
        ok[k] = col[k] < (int)ld;
    }
    if (!TM)
        for (int q = tid; q < L * K * T; q += T) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (TM && warp == 0) tmem_alloc(smem_addr(tslot), (uint32_t)tcols);
    if (tid == 0) {
        for (int q = 0; q < NST + 2; ++q) mbar_init(bar0 + 8 * q, 1);
        fence_mbarrier_init();
    }
    if (TM) tc_fence_before();
    if (C > 1) cluster_barrier(); else __syncthreads();
    if (TM) {
        tc_fence_after();
        tacc = *tslot + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * L * 4 * K);
        float z[4 * K];
#pragma unroll
        for (int q = 0; q < 4 * K; ++q) z[q] = 0.f;
        for (int ll = 0; ll < L; ++ll) tmem_store<4 * K>(tacc + (uint32_t)(ll * 4 * K), z);
    }

    const int my_rows = NR > (int)g ? (NR - 1 - (int)g) / (int)G + 1 : 0;
    const int nsteps = my_rows * L;

    // One elected thread streams the A, R (and, when needed, S) row slices of
    // step q into ring stage q % NST.
    auto issue = [&](int q) {
        const int row = (int)g + (q / L) * (int)G, l = q % L, st = q % NST;
        const bool load_s = s_each_level || l == 0;
        const uint32_t bar = bar0 + 8 * st;
        const uint32_t dst = sm0 + (uint32_t)(st * stage_bytes);
        const uint32_t bytes = (uint32_t)slice_len * (8u + (load_s ? (uint32_t)sizeof(ST) : 0u));
        const int64_t off = ((int64_t)l * NR + row) * ld + slice0;
        // debug variant: the copied slices must lie inside the messages; a
        // failed check is recorded and the copy skipped (the stage then
        // completes with no bytes)
        const bool in_bounds = !DBG || slice_len == 0 || (row < NR && slice0 + slice_len <= ld &&
                                            off + slice_len <= (int64_t)L * NR * ld &&
                                            (int64_t)(s_each_level ? l : 0) * p.s_level_stride + (int64_t)row * ld +
                                                    slice0 + slice_len <= (s_each_level ? (int64_t)L : 1) * NR * ld);
        if (!in_bounds) atomicOr(p.status, ST_BOUNDS);
        mbar_arrive_expect_tx(bar, in_bounds ? bytes : 0u);
        if (slice_len > 0 && in_bounds) {
            bulk_g2s(dst, p.A + off, (uint32_t)slice_len * 4u, bar);
            bulk_g2s(dst + (uint32_t)a_bytes, p.R + off, (uint32_t)slice_len * 4u, bar);
            if (load_s)
                bulk_g2s(dst + 2u * (uint32_t)a_bytes, Sb + (int64_t)l * p.s_level_stride + (int64_t)row * ld + slice0,
                         (uint32_t)slice_len * (uint32_t)sizeof(ST), bar);
        }
    };
    // issuing thread only: steps issued, and steps whose stage it has waited for
    int issued = 0, consumed = 0;
    if (tid == 0)
        for (; issued < min(NST, nsteps); ++issued) issue(issued);

    float4 srow[K];
#pragma unroll
    for (int k = 0; k < K; ++k) srow[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    float c_prev = 0.f;
    bool bad = false;
    int row = (int)g, l = 0;

    // Per-column b of the pending availability update and per-row scalars
    // (preference, fixed c, tau's column part), loaded one step ahead.
    float4 nb[K];
    float npref = 0.f, nc = 0.f, ntp = 0.f, ntau = kInf;
    auto prefetch = [&](int prow, int pl) {
        const int64_t pv = (int64_t)pl * ld;  // level pl of a [L][ld] vector: b by column,
        const int64_t pr = pv + R0 + prow;    // the row scalars at the row's index in the problem
#pragma unroll
        for (int k = 0; k < K; ++k)
            nb[k] = (pending && ok[k]) ? __ldg(reinterpret_cast<const float4*>(p.b + pv + col[k])) : f4_splat(0.f);
        npref = __ldg(p.pref + pr);
        nc = p.update_c ? 0.f : p.c[pr];
        ntp = (p.use_tau && pl > 0) ? __ldg(p.tpart + pr) : 0.f;
        if (p.tau_in) ntau = p.tau_in[pr];
    };
    if (nsteps > 0) prefetch(row, 0);

    for (int s = 0; s < nsteps; ++s) {
        const int st = s % NST;
        const unsigned char* base = sm + (size_t)st * stage_bytes;
        const float* sA = reinterpret_cast<const float*>(base);
        const float* sR = reinterpret_cast<const float*>(base + a_bytes);
        const ST* sS = reinterpret_cast<const ST*>(base + 2 * a_bytes);
        if (!mbar_wait(bar0 + 8 * st, (uint32_t)(s / NST) & 1u, p.status, p.wait_ns)) bad = true;
        if (__any_sync(0xffffffffu, bad)) { bad = true; break; }
        if (tid == 0) consumed = s + 1;

        const bool new_s = s_each_level || l == 0;
        const int grow = R0 + row;  // this row's index in the problem (its diagonal column)
        const int64_t voff = (int64_t)l * ld;
        const int64_t off = ((int64_t)l * NR + row) * ld;
        float4 bcur[K];
#pragma unroll
        for (int k = 0; k < K; ++k) bcur[k] = nb[k];
        const float pref_i = npref, c_fixed = nc, tpart_i = ntp, tau_given = ntau;
        {
            int prow = row, pl = l + 1;
            if (pl == L) { pl = 0; prow += (int)G; }
            if (s + 1 < nsteps) prefetch(prow, pl);
        }

        // ---- pass 1: pending availability (Eqs. 2.2/2.3), row statistics ------
        float m1 = -kInf, m2 = -kInf, cm = -kInf;
        int k1 = 0x7fffffff;
        float4 rr[K], ss[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int q = k * T + tid;
            float4 a4 = f4_splat(-kInf), r4 = f4_splat(0.f), s4 = f4_splat(0.f);
            if (ok[k]) {
                a4 = reinterpret_cast<const float4*>(sA)[q];
                r4 = reinterpret_cast<const float4*>(sR)[q];
                if (new_s) srow[k] = load_s_smem<ST>(sS + 4 * q);
                s4 = srow[k];
            }
            float4 an = a4;
            const float4 b4 = bcur[k];
            if (pending) {
                an.x = damp(a4.x, avail_target(b4.x, r4.x, false), lam, oml);
                an.y = damp(a4.y, avail_target(b4.y, r4.y, false), lam, oml);
                an.z = damp(a4.z, avail_target(b4.z, r4.z, false), lam, oml);
                an.w = damp(a4.w, avail_target(b4.w, r4.w, false), lam, oml);
            }
            const int dd = grow - col[k];
            if ((unsigned)dd < 4u) {  // this float4 holds the diagonal element
                f4_set(s4, dd, pref_i);
                if (pending) f4_set(an, dd, damp(f4_get(a4, dd), avail_target(f4_get(b4, dd), f4_get(r4, dd), true), lam, oml));
            }
            if (kap) {  // Eq. 2.7: the next level's similarity from this level's start-of-iteration messages
                const float kp = p.kappa;
                srow[k].x = __fadd_rn(srow[k].x, __fmul_rn(kp, __fadd_rn(an.x, r4.x)));
                srow[k].y = __fadd_rn(srow[k].y, __fmul_rn(kp, __fadd_rn(an.y, r4.y)));
                srow[k].z = __fadd_rn(srow[k].z, __fmul_rn(kp, __fadd_rn(an.z, r4.z)));
                srow[k].w = __fadd_rn(srow[k].w, __fmul_rn(kp, __fadd_rn(an.w, r4.w)));
            }
            if (pending && ok[k] && !bad) st_stream(p.A + off + col[k], an);
            top2_push(__fadd_rn(an.x, s4.x), col[k] + 0, m1, k1, m2);
            top2_push(__fadd_rn(an.y, s4.y), col[k] + 1, m1, k1, m2);
            top2_push(__fadd_rn(an.z, s4.z), col[k] + 2, m1, k1, m2);
            top2_push(__fadd_rn(an.w, s4.w), col[k] + 3, m1, k1, m2);
            cm = fmaxf(cm, fmaxf(fmaxf(__fadd_rn(an.x, r4.x), __fadd_rn(an.y, r4.y)),
                                 fmaxf(__fadd_rn(an.z, r4.z), __fadd_rn(an.w, r4.w))));
            rr[k] = r4;
            ss[k] = s4;
        }

        // ---- exact reduction over the cluster: warp redux, then every warp's
        // summary sent to every CTA's shared memory (st.async + mbarrier) ------
        warp_top2(m1, k1, m2, cm);
        const int par = s & 1;
        const uint32_t xbar = bar0 + 8 * (NST + par);
        if (lane == 0) {
            const float4 v = make_float4(m1, m2, cm, __int_as_float(k1));
            const uint32_t slot = smem_addr(xbuf + (par * C + rank) * 32 + warp);
            for (unsigned q = 0; q < C; ++q) st_async_f4(map_to_rank(slot, q), v, map_to_rank(xbar, q));
        }
        if (tid == 0) mbar_arrive_expect_tx(xbar, (uint32_t)(C * nw * 16));
        if (!mbar_wait(xbar, (uint32_t)(s >> 1) & 1u, p.status, p.wait_ns)) bad = true;
        if (__any_sync(0xffffffffu, bad)) { bad = true; break; }
        m1 = m2 = cm = -kInf;
        k1 = 0x7fffffff;
        for (int q = lane; q < (int)C * 32; q += 32) {
            if ((q & 31) < nw) {
                const float4 v = xbuf[par * C * 32 + q];
                top2_merge(m1, k1, m2, v.x, __float_as_int(v.w), v.y);
                cm = fmaxf(cm, v.z);
            }
        }
        warp_top2(m1, k1, m2, cm);
        // debug variant: the row maximum of Eq. 2.1 must sit in a real column
        // (alpha's padding is -inf; a NaN similarity leaves no maximum)
        if constexpr (DBG)
            if (tid == 0 && rank == 0 && (k1 < 0 || k1 >= N)) atomicOr(p.status, ST_BOUNDS);
        // every warp of this CTA has read stage st: refill it
        if (tid == 0 && s + NST < nsteps) issue(issued++);

        // ---- inter-level messages of (i, l): Eqs. 2.4-2.6 --------------------
        const float cval = p.update_c ? cm : c_fixed;
        const float tauv = p.tau_in ? tau_given : (p.use_tau && l > 0) ? __fadd_rn(c_prev, tpart_i) : kInf;
        c_prev = cval;
        if (rank == 0 && tid == 0 && !bad) {
            if (p.update_c) p.c[voff + grow] = cval;
            p.tau[voff + grow] = tauv;
            if (l > 0) p.phi[voff - ld + grow] = m1;
        }

        // ---- pass 2: responsibilities (Eq. 2.1) and column sums -----------------
        float addv[TM ? 4 * K : 1];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int dk = k1 - col[k];
            const float4 r4 = rr[k], s4 = ss[k];
            float4 rn;
            rn.x = damp(r4.x, __fadd_rn(s4.x, fminf(tauv, -(dk == 0 ? m2 : m1))), lam, oml);
            rn.y = damp(r4.y, __fadd_rn(s4.y, fminf(tauv, -(dk == 1 ? m2 : m1))), lam, oml);
            rn.z = damp(r4.z, __fadd_rn(s4.z, fminf(tauv, -(dk == 2 ? m2 : m1))), lam, oml);
            rn.w = damp(r4.w, __fadd_rn(s4.w, fminf(tauv, -(dk == 3 ? m2 : m1))), lam, oml);
            float4 add = make_float4(fmaxf(rn.x, 0.f), fmaxf(rn.y, 0.f), fmaxf(rn.z, 0.f), fmaxf(rn.w, 0.f));
            const int dd = grow - col[k];
            if ((unsigned)dd < 4u) {
                f4_set(add, dd, 0.f);
                if (!bad) p.rdiag[voff + grow] = f4_get(rn, dd);
            }
            if (ok[k] && !bad) st_stream(p.R + off + col[k], rn);
            if constexpr (TM) {
                addv[4 * k + 0] = add.x;
                addv[4 * k + 1] = add.y;
                addv[4 * k + 2] = add.z;
                addv[4 * k + 3] = add.w;
            } else {
                float4& a = acc[(l * K + k) * T + tid];
                a.x = __fadd_rn(a.x, add.x);
                a.y = __fadd_rn(a.y, add.y);
                a.z = __fadd_rn(a.z, add.z);
                a.w = __fadd_rn(a.w, add.w);
            }
        }
        if constexpr (TM) {
            __syncwarp();  // tcgen05.ld / st are warp-collective
            float cur[4 * K];
            const uint32_t ta = tacc + (uint32_t)(l * 4 * K);
            tmem_load<4 * K>(ta, cur);
#pragma unroll
            for (int q = 0; q < 4 * K; ++q) cur[q] = __fadd_rn(cur[q], addv[q]);
            tmem_store<4 * K>(ta, cur);
        }
        if (++l == L) { l = 0; row += (int)G; }
    }

    // ---- after a wait gave up: let this CTA's own bulk copies land ------------
    if (tid == 0)
        for (int q = consumed; q < issued; ++q)
            mbar_wait(bar0 + 8 * (q % NST), (uint32_t)(q / NST) & 1u, p.status, kWaitNs);

    // ---- per-cluster column partials (skipped by warps that gave up) ----------
    for (int ll = 0; ll < L && !bad; ++ll) {
        if constexpr (TM) {
            float cur[4 * K];
            __syncwarp();
            tmem_load<4 * K>(tacc + (uint32_t)(ll * 4 * K), cur);
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (ok[k])
                    *reinterpret_cast<float4*>(p.partials + ((int64_t)g * L + ll) * ld + col[k]) =
                        make_float4(cur[4 * k], cur[4 * k + 1], cur[4 * k + 2], cur[4 * k + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (ok[k])
                    *reinterpret_cast<float4*>(p.partials + ((int64_t)g * L + ll) * ld + col[k]) =
                        acc[(ll * K + k) * T + tid];
        }
    }
    if constexpr (TM) {
        __syncwarp();
        tmem_store_wait();  // a warp that gave up may still have stores in flight
        tc_fence_before();
    }
    __syncthreads();
    if constexpr (TM) {
        tc_fence_after();
        if (warp == 0) tmem_dealloc(*tslot, (uint32_t)tcols);
    }
    // No CTA may leave while a peer can still write into its shared memory.
    if (C > 1) cluster_barrier();
}

template <typename ST, int K, int MAXT, int NST, bool TM, bool DBG, bool BAND = false>
cudaError_t cluster_config(const LaunchShape& sh, int L, cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr) {
    auto kern = rowpass_kernel<ST, K, MAXT, NST, TM, DBG, BAND>;
    const size_t smem = rowpass_smem_bytes(sh, L, sizeof(ST) == 2);
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    if (sh.C > 8) {
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (err != cudaSuccess) return err;
    }
    cfg->blockDim = dim3((unsigned)sh.T, 1, 1);
    cfg->dynamicSmemBytes = smem;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)sh.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg->attrs = attr;
    cfg->numAttrs = 1;
    return cudaSuccess;
}

template <typename ST, int K, int MAXT, int NST, bool TM, bool DBG, bool BAND = false>
cudaError_t launch_one(const RowPassArgs& a, const LaunchShape& sh, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cudaError_t err = cluster_config<ST, K, MAXT, NST, TM, DBG, BAND>(sh, a.L, &cfg, attr);
    if (err != cudaSuccess) return err;
    cfg.gridDim = dim3((unsigned)(sh.G * sh.C), 1, 1);
    cfg.stream = st;
    return cudaLaunchKernelEx(&cfg, rowpass_kernel<ST, K, MAXT, NST, TM, DBG, BAND>, a);
}

template <typename ST, int K, int MAXT, int NST, bool TM>
cudaError_t launch_plain(const RowPassArgs& a, const LaunchShape& sh, cudaStream_t st) {
    return launch_one<ST, K, MAXT, NST, TM, false>(a, sh, st);
}
template <typename ST, int K, int MAXT, int NST, bool TM>
cudaError_t launch_checked(const RowPassArgs& a, const LaunchShape& sh, cudaStream_t st) {
    return launch_one<ST, K, MAXT, NST, TM, true>(a, sh, st);
}
template <typename ST, int K, int MAXT, int NST, bool TM>
cudaError_t launch_band(const RowPassArgs& a, const LaunchShape& sh, cudaStream_t st) {
    return launch_one<ST, K, MAXT, NST, TM, false, true>(a, sh, st);
}

// Instantiated shapes: shared-memory sums with 4, 8 or 16 columns per thread
// and a 3-stage ring; TMEM sums with 8 or 16 columns per thread and a 2- or
// 4-stage ring.
#define HAP_ROWPASS_DISPATCH_ST(ST, FN, ...)                                        \
    do {                                                                            \
        if (!sh.tm) {                                                               \
            if (sh.K == 1) return FN<ST, 1, 1024, kStages, false>(__VA_ARGS__);     \
            if (sh.K == 2) return FN<ST, 2, 512, kStages, false>(__VA_ARGS__);      \
            if (sh.K == 4) return FN<ST, 4, 256, kStages, false>(__VA_ARGS__);      \
        } else if (sh.nst == 2) {                                                   \
            if (sh.K == 2) return FN<ST, 2, 512, 2, true>(__VA_ARGS__);             \
            if (sh.K == 4) return FN<ST, 4, 512, 2, true>(__VA_ARGS__);             \
        } else if (sh.nst == 4) {                                                   \
            if (sh.K == 2) return FN<ST, 2, 512, 4, true>(__VA_ARGS__);             \
            if (sh.K == 4) return FN<ST, 4, 512, 4, true>(__VA_ARGS__);             \
        }                                                                           \
    } while (0)
#define HAP_ROWPASS_DISPATCH(FN, ...)                                               \
    do {                                                                            \
        if (s_bf16) HAP_ROWPASS_DISPATCH_ST(__nv_bfloat16, FN, __VA_ARGS__);        \
        else HAP_ROWPASS_DISPATCH_ST(float, FN, __VA_ARGS__);                       \
        return cudaErrorInvalidValue;                                               \
    } while (0)

}  // namespace hap
