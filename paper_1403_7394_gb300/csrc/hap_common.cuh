// Device helpers shared by the HAP kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "hap_internal.h"

#define HAP_DEV __device__ __forceinline__

namespace hap {

constexpr float kInf = __builtin_inff();

// Damping of §2: lam * old + (1 - lam) * new, with one fixed rounding
// sequence (product, then fused multiply-add) so that every kernel that
// recomputes a damped value obtains the same bits.
HAP_DEV float damp(float old_v, float new_v, float lam, float oml) {
    return __fmaf_rn(lam, old_v, __fmul_rn(oml, new_v));
}

// Availability target of Eqs. 2.2/2.3 given the column term
// b_j = c_j + phi_j + rho_jj + P_j:  min(0, b_j - max(0, rho_ij)) off the
// diagonal, b_j - rho_jj on it.
HAP_DEV float avail_target(float b, float r, bool diag) {
    return diag ? __fsub_rn(b, r) : fminf(0.f, __fsub_rn(b, fmaxf(r, 0.f)));
}

// Running (max, lowest argmax, second max) of a stream visited in
// increasing index order.
HAP_DEV void top2_push(float x, int j, float& m1, int& k1, float& m2) {
    m2 = fmaxf(m2, fminf(x, m1));
    if (x > m1) { m1 = x; k1 = j; }
}

// Merge of two (max, lowest argmax, second max) summaries of disjoint index
// sets; commutative and exact (no rounding), so any merge order gives the
// same bits.
HAP_DEV void top2_merge(float& m1, int& k1, float& m2, float o1, int ok1, float o2) {
    if (o1 > m1 || (o1 == m1 && ok1 < k1)) {
        m2 = fmaxf(m1, o2);
        m1 = o1;
        k1 = ok1;
    } else {
        m2 = fmaxf(m2, o1);
    }
}

// ---- cluster / distributed shared memory (PTX) -------------------------
HAP_DEV unsigned cluster_nctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
HAP_DEV unsigned cluster_ctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
HAP_DEV unsigned cluster_id_x() {
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
HAP_DEV unsigned cluster_count_x() {
    unsigned r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// All threads of all CTAs of the cluster; release/acquire orders the shared
// memory writes before the barrier with the remote reads after it.
HAP_DEV void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
HAP_DEV uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
HAP_DEV uint32_t map_to_rank(uint32_t addr, unsigned rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
HAP_DEV float4 ld_dsmem_f4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr) : "memory");
    return v;
}

// ---- mbarrier, bulk copies (TMA), asynchronous remote stores ---------------
HAP_DEV void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}
HAP_DEV void fence_mbarrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
HAP_DEV void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}
// One arrival (release semantics) on a barrier of this CTA.
HAP_DEV void mbar_arrive_local(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}
HAP_DEV bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    return done != 0;
}
// Non-blocking test of the phase with the given parity.
HAP_DEV bool mbar_test_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    return done != 0;
}
HAP_DEV uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Default limit of a bounded wait.
constexpr uint64_t kWaitNs = 2000000000ull;
// Waits for the phase with the given parity to complete, for at most about
// limit_ns nanoseconds; on expiry records ST_TIMEOUT in the status word and
// returns false so the caller can stop waiting and leave.  Limits of a
// millisecond or more wait with try_wait (the thread may be suspended while
// it waits); shorter ones poll with test_wait, so that the clock is read
// within a few nanoseconds of the limit.
HAP_DEV bool mbar_wait(uint32_t bar, uint32_t parity, unsigned* status, uint64_t limit_ns = kWaitNs) {
    if (mbar_test_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    const bool poll = limit_ns < 1000000ull;
    for (;;) {
        if (poll ? mbar_test_wait(bar, parity) : mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > limit_ns) {
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
    }
}
// Bulk (non-tensor) TMA copy global -> this CTA's shared memory, completing
// `bytes` of transaction count on the mbarrier.  16-byte aligned addresses,
// size a multiple of 16.
HAP_DEV void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
// 16-byte store into a (possibly remote) CTA's shared memory that completes
// 16 bytes of transaction count on that CTA's mbarrier.
HAP_DEV void st_async_f4(uint32_t remote_addr, float4 v, uint32_t remote_bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
                 :: "r"(remote_addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(remote_bar) : "memory");
}

// ---- exact warp reductions -------------------------------------------------
HAP_DEV float redux_max(float v) {
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
// Warp-wide (max, lowest argmax, second max) and plain max, all lanes get
// the result.  Lanes summarise disjoint index sets.
HAP_DEV void warp_top2(float& m1, int& k1, float& m2, float& cm) {
    const float wm1 = redux_max(m1);
    const int wk1 = __reduce_min_sync(0xffffffffu, m1 == wm1 ? k1 : 0x7fffffff);
    const float wm2 = redux_max((m1 == wm1 && k1 == wk1) ? m2 : m1);
    cm = redux_max(cm);
    m1 = wm1;
    k1 = wk1;
    m2 = wm2;
}

// ---- streaming global loads / stores -------------------------------------
// ---- tensor memory (TMEM) -------------------------------------------------
// Allocation by one whole warp; the TMEM address is written to shared memory.
HAP_DEV void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(dst_smem), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
HAP_DEV void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}
HAP_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
HAP_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// N consecutive 32-bit TMEM columns of one lane per thread (shape 32x32b):
// thread t of the warp owns lane (lane field of taddr) + t.  The warp must be
// converged and taddr's lane field must be the warp's lane quarter.
// tmem_load waits for this thread's earlier tmem_store first, so a
// load-modify-store sequence on the same columns is ordered.
template <int N>
HAP_DEV void tmem_load(uint32_t taddr, float (&v)[N]);
template <int N>
HAP_DEV void tmem_store(uint32_t taddr, const float (&v)[N]);

template <>
HAP_DEV void tmem_load<8>(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.wait::st.sync.aligned;\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr) : "memory");
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}
template <>
HAP_DEV void tmem_store<8>(uint32_t taddr, const float (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                    "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                    "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])) : "memory");
}
template <>
HAP_DEV void tmem_load<16>(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.wait::st.sync.aligned;\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, "
                 "%8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr) : "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}
template <>
HAP_DEV void tmem_store<16>(uint32_t taddr, const float (&v)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, "
                 "%9, %10, %11, %12, %13, %14, %15, %16};"
                 :: "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                    "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                    "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                    "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                    "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                    "r"(__float_as_uint(v[15])) : "memory");
}
// Completes this thread's outstanding tmem_store operations.
HAP_DEV void tmem_store_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

HAP_DEV float4 ld_stream(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
HAP_DEV void st_stream(float* p, float4 v) { __stcs(reinterpret_cast<float4*>(p), v); }

// Four similarities as float4, from FP32 or BF16 storage.
template <typename ST> struct SVec;
template <> struct SVec<float> {
    using raw = float4;
    static HAP_DEV raw load(const float* p) { return ld_stream(p); }
    static HAP_DEV float4 to_f4(raw v) { return v; }
    static HAP_DEV raw zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <> struct SVec<__nv_bfloat16> {
    using raw = uint2;
    static HAP_DEV raw load(const __nv_bfloat16* p) { return __ldcs(reinterpret_cast<const uint2*>(p)); }
    static HAP_DEV float4 to_f4(raw v) {
        return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u),
                           __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
    }
    static HAP_DEV raw zero() { return make_uint2(0u, 0u); }
};

HAP_DEV float f4_get(const float4& v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
HAP_DEV float4 f4_splat(float x) { return make_float4(x, x, x, x); }
HAP_DEV void f4_set(float4& v, int e, float x) {
    if (e == 0) v.x = x; else if (e == 1) v.y = x; else if (e == 2) v.z = x; else v.w = x;
}

}  // namespace hap
