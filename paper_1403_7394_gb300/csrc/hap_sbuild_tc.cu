// Tensor-core similarity build: s_ij = 2 x_i.x_j - ||x_i||^2 - ||x_j||^2
// (the negative squared Euclidean distance of §2) with the dot products on
// the 5th-generation tensor cores (tcgen05, BF16 x BF16 -> FP32 in tensor
// memory) and the norms in FP32 from the FP32 points.
//
// Split mode: x = hi + lo with hi = bf16(x), lo = bf16(x - hi); then
// x_i.x_j ~ hi_i.hi_j + hi_i.lo_j + lo_i.hi_j, computed as ONE contraction
// over K' = 3d of A_i = [hi_i, hi_i, lo_i] and B_j = [hi_j, lo_j, hi_j]
// (the dropped lo.lo term is ~2^-16 of the product).
//
// The build kernel (sbuild_sym_kernel, below) contracts only the tiles on and
// above the diagonal and writes each tile twice; the same file holds the
// tensor-core first pass of the exact kNN.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "hap_common.cuh"
#include "hap_internal.h"

namespace hap {
namespace {

constexpr int BM = 128, BK = 64;  // operand rows per tile and K-chunk (64 BF16 = 128 bytes)

// ---- tcgen05 / TMA PTX -------------------------------------------------------
HAP_DEV void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar) : "memory");
}
// D[tmem] (+)= A[smem] x B[smem]^T, both K-major BF16, FP32 accumulation.
HAP_DEV void umma_bf16(uint32_t tmem_d, uint64_t desc_a, uint64_t desc_b, uint32_t idesc, uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(tmem_d), "l"(desc_a), "l"(desc_b), "r"(idesc), "r"(accumulate) : "memory");
}
// Arrives on the mbarrier once every previously issued MMA of this thread is done.
HAP_DEV void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar) : "memory");
}
HAP_DEV void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}
// 32 lanes x 32 consecutive FP32 columns: thread t of the warp receives row
// (lane base + t), columns col .. col+31.
// The same load without the wait: several may be in flight before one
// tcgen05.wait::ld; the registers are valid only after that wait.
HAP_DEV void tmem_ld_32x32b_x32_nowait(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
}

// tcgen05.wait::ld that also marks r as written by it, so no use of the
// loaded registers can be scheduled before the wait; `tie` does only the
// latter for further registers of loads the same wait covered.
HAP_DEV void tmem_wait_ld(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
                   "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :: "memory");
}
HAP_DEV void tmem_tie(uint32_t (&r)[32]) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
                   "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}

// Maximum of 32 values by a pairwise tree (5 dependent steps, exact).
HAP_DEV float max32(const uint32_t (&r)[32]) {
    float m[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) m[q] = fmaxf(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1]));
#pragma unroll
    for (int w = 8; w > 0; w >>= 1)
#pragma unroll
        for (int q = 0; q < w; ++q) m[q] = fmaxf(m[q], m[q + w]);
    return m[0];
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
// Bits: [0,14) start >> 4, [16,30) leading offset >> 4 (unused here),
// [32,46) stride offset >> 4, [46,48) version 1, [61,64) swizzle (2 = 128B).
HAP_DEV uint64_t desc_kmajor_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// ---- symmetric persistent build -----------------------------------------------
// s is symmetric, so of the 128-row strips r and 256-column blocks J of the
// padded N x N matrix only the tiles with 256 J + 255 >= 128 r are
// contracted (M = 128, N = 256 per tcgen05.mma), and each 128 x 128 half
// above the diagonal is written twice, as itself and transposed; a half on
// the diagonal writes its upper triangle both ways (so S is symmetric bit for
// bit) and a half below it (the first half of the first block of an odd
// strip) is skipped.  That is about half the tensor work of the full tiling
// for the same N^2 writes, and the 256-column tiles read 25 % fewer operand
// bytes per output than 128-column ones.
// Tile order: groups of kSyGroup strips, and within a group the blocks J in
// order, each with the group's strips that need it; the persistent CTAs (one
// per SM) take the tiles of that list round-robin.  At any moment the GPU
// then works on a few A strips and B blocks, which stay in L2 (loads hinted
// evict-last, the similarity stores evict-first) while N^2 results stream
// through it; with a contiguous range of tiles per CTA the operands were
// re-read from memory about 16 times.
//   warp 4 (producer): TMA loads of the A and B K-chunks into a ring.
//   warp 5 (MMA issuer): tcgen05.mma into one of two TMEM accumulators
//     (256 columns each), so one tile's products overlap the previous tile's
//     epilogue.
//   warps 0-3 (epilogue; thread = tile row = TMEM lane): read a finished
//     accumulator, hand it back, and write each 128 x 32 column block twice
//     by TMA tensor stores from shared-memory boxes that the four warps fill
//     together (the stores clip at N): as itself (128 rows x 32 columns,
//     staged with the 128-byte (FP32) or 64-byte (BF16) swizzle, so the
//     row-per-lane writes hit every bank) and transposed (32 rows x 128
//     columns, staged row = column, where the 32 lanes of a warp write one
//     contiguous piece).  Plain stores from registers, and 32 x 32 boxes
//     per warp, measured slower.  The warps meet at named barriers, so every
//     decision to stop is taken by all 128 epilogue threads together.
constexpr int SY_THREADS = 192;  // 4 epilogue warps, 1 producer warp, 1 MMA warp
constexpr int SY_BN = 256;       // tile columns
constexpr int SY_RING_MAX = 8;
constexpr int kSyGroup = 16;     // strips per group of the tile order
constexpr uint32_t SY_TMEM_COLS = 2 * SY_BN;
constexpr uint32_t SY_ACHUNK = BM * BK * 2;            // A K-chunk, 16 KB
constexpr uint32_t SY_BCHUNK = SY_BN * BK * 2;         // B K-chunk, 32 KB
constexpr uint32_t SY_BOX = 128 * 32 * 4;              // one staged 128 x 32 box (FP32 size)
constexpr uint32_t SY_STG = 4 * SY_BOX;                // two buffers x {direct, transposed}
constexpr uint32_t kSyIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(SY_BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

// Dynamic shared memory: alignment slack | ring stages [B | A] | staging
// [2][2 boxes].  At least 116 KB: one CTA per SM, so its 512-column TMEM
// allocation never waits.
__host__ __device__ inline size_t sbuild_sym_smem_bytes(int ring) {
    const size_t b = 1024 + (size_t)ring * (SY_BCHUNK + SY_ACHUNK) + (size_t)SY_STG;
    return b < 116 * 1024 ? 116 * 1024 : b;
}

// Tiles of the symmetric build: strip r needs the blocks J = r/2 .. T2-1.
__host__ __device__ inline int64_t sym_tile_count(int T) {
    const int T2 = (T + 1) / 2;
    int64_t n = 0;
    for (int r = 0; r < T; ++r) n += T2 - r / 2;
    return n;
}
// Group g (strips r0 .. r0+n-1, r0 = kSyGroup g): block J (>= r0 / 2) is
// needed by the first c(J) = min(n, 2J + 2 - r0) strips; jf is the first
// block all n need, and sp(J) the tiles of the blocks before J (J <= jf).
struct SymGroup {
    int r0, n, J0, jf;
    __host__ __device__ SymGroup(int g, int T) {
        r0 = g * kSyGroup;
        n = (T - r0 < kSyGroup ? T - r0 : kSyGroup);
        J0 = r0 / 2;
        jf = (n + r0 - 1) / 2;  // ceil((n + r0 - 2) / 2)
        if (jf < J0) jf = J0;
    }
    __host__ __device__ int count(int J) const { return 2 * J + 2 - r0 < n ? 2 * J + 2 - r0 : n; }
    __host__ __device__ int64_t sp(int J) const { return (int64_t)(J - J0) * (2 - r0) + (int64_t)(J - J0) * (J0 + J - 1); }
    __host__ __device__ int64_t total(int T2) const { return sp(jf) + (int64_t)(T2 - jf) * n; }
    __host__ __device__ int64_t offset(int J) const { return J <= jf ? sp(J) : sp(jf) + (int64_t)(J - jf) * n; }
};
// The tile list (r << 16 | J) in that order: block g = group, thread J.
__global__ void sym_order_kernel(int T, int32_t* __restrict__ tiles) {
    const int g = blockIdx.x, J = threadIdx.x, T2 = (T + 1) / 2;
    const SymGroup sg(g, T);
    if (J < sg.J0 || J >= T2) return;
    int64_t base = 0;
    for (int q = 0; q < g; ++q) base += SymGroup(q, T).total(T2);
    const int64_t o = base + sg.offset(J);
    const int c = sg.count(J);
    for (int i = 0; i < c; ++i) tiles[o + i] = ((sg.r0 + i) << 16) | J;
}

template <typename OT>
HAP_DEV void store1(OT* dst, float v);
template <>
HAP_DEV void store1<float>(float* dst, float v) { *dst = v; }
template <>
HAP_DEV void store1<__nv_bfloat16>(__nv_bfloat16* dst, float v) { *dst = __float2bfloat16_rn(v); }

// L2 eviction priorities: the operands (tens of MB, read by every CTA) stay
// in L2 while the N^2 similarities stream through it to memory.
HAP_DEV uint64_t l2_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
HAP_DEV uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// TMA tile load with an L2 cache policy.
HAP_DEV void tma_load_2d_hint(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar), "l"(pol) : "memory");
}
// TMA tensor store of a shared-memory box (bulk-group completion) with an L2
// cache policy.
HAP_DEV void tma_store_2d(const CUtensorMap* map, uint32_t src, int c0, int c1, uint64_t pol) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%1, %2}], [%3], %4;"
                 :: "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(src), "l"(pol) : "memory");
}
HAP_DEV void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most one committed group still reading shared memory
HAP_DEV void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// every committed group complete
HAP_DEV void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
HAP_DEV void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Named barrier of the 128 epilogue threads; the _and form returns whether
// every one of them passed `pred`.
HAP_DEV void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
HAP_DEV bool epi_all(bool pred) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\t"
                 "setp.ne.u32 p, %1, 0;\n\t"
                 "bar.red.and.pred q, 1, 128, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r) : "r"((uint32_t)pred) : "memory");
    return r != 0;
}

// Thread `r`'s 32 values (row r of a 128 x 32 block) into the swizzled box.
template <typename OT>
HAP_DEV void stage_direct(unsigned char* box, int r, const float (&v)[32]);
template <>
HAP_DEV void stage_direct<float>(unsigned char* box, int r, const float (&v)[32]) {
    // 128-byte rows, 16-byte chunk k stored at chunk k ^ (r % 8)
#pragma unroll
    for (int k = 0; k < 8; ++k)
        *reinterpret_cast<float4*>(box + r * 128 + ((k ^ (r & 7)) << 4)) =
            make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}
template <>
HAP_DEV void stage_direct<__nv_bfloat16>(unsigned char* box, int r, const float (&v)[32]) {
    // 64-byte rows, 16-byte chunk k stored at chunk k ^ ((r / 2) % 4)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint4 u;
        __nv_bfloat162 p0 = __floats2bfloat162_rn(v[8 * k + 0], v[8 * k + 1]);
        __nv_bfloat162 p1 = __floats2bfloat162_rn(v[8 * k + 2], v[8 * k + 3]);
        __nv_bfloat162 p2 = __floats2bfloat162_rn(v[8 * k + 4], v[8 * k + 5]);
        __nv_bfloat162 p3 = __floats2bfloat162_rn(v[8 * k + 6], v[8 * k + 7]);
        u.x = *reinterpret_cast<uint32_t*>(&p0);
        u.y = *reinterpret_cast<uint32_t*>(&p1);
        u.z = *reinterpret_cast<uint32_t*>(&p2);
        u.w = *reinterpret_cast<uint32_t*>(&p3);
        *reinterpret_cast<uint4*>(box + r * 64 + ((k ^ ((r >> 1) & 3)) << 4)) = u;
    }
}

template <typename OT>
__global__ void __launch_bounds__(SY_THREADS, 1) sbuild_sym_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                  const __grid_constant__ CUtensorMap tmB,
                                                                  const __grid_constant__ CUtensorMap tmSd,
                                                                  const __grid_constant__ CUtensorMap tmSt,
                                                                  const float* __restrict__ norms,
                                                                  const int32_t* __restrict__ tiles, OT* __restrict__ S,
                                                                  int N, int64_t ld, int kchunks, int ring, int T,
                                                                  int64_t total, unsigned* status) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t stage_bytes = SY_BCHUNK + SY_ACHUNK;
    const uint32_t sR = base;                               // ring: [B | A]
    const uint32_t sS = sR + (uint32_t)ring * stage_bytes;  // staging
    unsigned char* stg_all = smem_raw + (sS - raw);
    // full[R], empty[R], acc_full[2], acc_empty[2], mma_done
    __shared__ uint64_t bars[2 * SY_RING_MAX + 5];
    __shared__ __align__(16) float cnorm[2][SY_BN];  // column norms of the tile (by tile parity)
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t r_full = smem_addr(&bars[0]), r_empty = r_full + 8 * SY_RING_MAX;
    const uint32_t acc_full = r_empty + 8 * SY_RING_MAX, acc_empty = acc_full + 16, mma_done = acc_empty + 16;
    const int R = ring;
    const int64_t t_first = blockIdx.x, t_step = gridDim.x;

    if (tid == 0) {
        for (int q = 0; q < R; ++q) {
            mbar_init(r_full + 8 * q, 1);
            mbar_init(r_empty + 8 * q, 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(acc_full + 8 * q, 1);
            mbar_init(acc_empty + 8 * q, BM);
        }
        mbar_init(mma_done, 1);
        s_abort = 0;
        fence_mbarrier_init();
    }
    if (warp == 0) tmem_alloc(smem_addr(&tmem_slot), SY_TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int* abort_flag = &s_abort;

    if (warp == 4) {
        if (lane == 0) {  // ---- producer
            const uint64_t pol = l2_evict_last();
            int g = 0;
            bool ok = true;
            for (int64_t t = t_first; t < total && ok && !*abort_flag; t += t_step) {
                const int tr = __ldg(tiles + t) >> 16, tJ = __ldg(tiles + t) & 0xffff;
                for (int kc = 0; kc < kchunks; ++kc, ++g) {
                    const int st = g % R;
                    if (g >= R && !(ok = mbar_wait(r_empty + 8 * st, (uint32_t)((g / R - 1) & 1), status))) break;
                    const uint32_t dst = sR + (uint32_t)st * stage_bytes;
                    mbar_arrive_expect_tx(r_full + 8 * st, stage_bytes);
                    tma_load_2d_hint(dst, &tmB, kc * BK, tJ * SY_BN, r_full + 8 * st, pol);
                    tma_load_2d_hint(dst + SY_BCHUNK, &tmA, kc * BK, tr * BM, r_full + 8 * st, pol);
                }
            }
            if (!ok) *abort_flag = 1;
            // no copy may land in shared memory after the CTA has left: wait for
            // every issued copy (each is the last on its barrier)
            for (int q = g > R ? g - R : 0; q < g; ++q) mbar_wait(r_full + 8 * (q % R), (uint32_t)((q / R) & 1), status);
        }
    } else if (warp == 5) {
        if (lane == 0) {  // ---- MMA issuer
            int g = 0, tl = 0;
            bool ok = true;
            for (int64_t t = t_first; t < total && ok && !*abort_flag; t += t_step, ++tl) {
                const int buf = tl & 1;
                if (tl >= 2 && !(ok = mbar_wait(acc_empty + 8 * buf, (uint32_t)((tl / 2 - 1) & 1), status))) break;
                tc_fence_after();
                for (int kc = 0; kc < kchunks; ++kc, ++g) {
                    const int st = g % R;
                    if (!(ok = mbar_wait(r_full + 8 * st, (uint32_t)((g / R) & 1), status))) break;
                    tc_fence_after();
                    const uint32_t stg = sR + (uint32_t)st * stage_bytes;
                    const uint32_t a_s = stg + SY_BCHUNK;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
                        umma_bf16(tmem + (uint32_t)(buf * SY_BN), desc_kmajor_sw128(a_s + 32 * kk),
                                  desc_kmajor_sw128(stg + 32 * kk), kSyIdesc, (kc > 0 || kk > 0) ? 1u : 0u);
                    umma_commit(r_empty + 8 * st);
                }
                if (!ok) break;
                umma_commit(acc_full + 8 * buf);
            }
            if (!ok) *abort_flag = 1;
            // every issued MMA completes before tensor memory is freed
            umma_commit(mma_done);
            mbar_wait(mma_done, 0u, status);
        }
    } else {  // ---- epilogue: warps 0-3, thread = tile row = TMEM lane
        const uint64_t pol = l2_evict_first();
        int tl = 0, ch = 0;
        for (int64_t t = t_first; t < total; t += t_step, ++tl) {
            const int wr = __ldg(tiles + t) >> 16, wJ = __ldg(tiles + t) & 0xffff;
            const int r0 = wr * BM + 32 * warp, row = r0 + lane;
            const float ni = row < N ? __ldg(norms + row) : 0.f;
            // the tile's column norms into shared memory (read as broadcasts
            // below; the buffer of this parity was last read two tiles ago,
            // before the barrier of the previous tile)
            const int buf = tl & 1;
            const int cj = wJ * SY_BN + tid;  // (the norms hold T * 128 values)
            cnorm[buf][tid] = cj < T * BM ? __ldg(norms + cj) : 0.f;
            cnorm[buf][tid + BM] = cj + BM < T * BM ? __ldg(norms + cj + BM) : 0.f;
            // one decision for all 128 epilogue threads (they meet at named
            // barriers below, and the TMEM loads are warp-collective)
            const bool got = *abort_flag == 0 && mbar_wait(acc_full + 8 * buf, (uint32_t)((tl >> 1) & 1), status);
            if (!epi_all(got)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                const int cb = 2 * wJ + h;  // 128-column block of this half
                // the whole half row into registers (four loads, one wait); after
                // the second half the accumulator goes back to the MMA warp
                uint32_t rg[4][32];
                const bool need = cb >= wr && cb < T;
                if (need) {
                    __syncwarp();
                    const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(buf * SY_BN + 128 * h);
#pragma unroll
                    for (int b = 0; b < 4; ++b) tmem_ld_32x32b_x32_nowait(ta + 32 * b, rg[b]);
                    tmem_wait_ld(rg[0]);
#pragma unroll
                    for (int b = 1; b < 4; ++b) tmem_tie(rg[b]);
                }
                if (h == 1) {
                    tc_fence_before();
                    mbar_arrive(acc_empty + 8 * buf);
                }
                if (!need) continue;
                const bool diag = cb == wr;
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const int c0 = cb * 128 + 32 * cc;
                    float v[32];
#pragma unroll
                    for (int q = 0; q < 32; q += 4) {
                        const float4 nj = *reinterpret_cast<const float4*>(&cnorm[buf][128 * h + 32 * cc + q]);
                        v[q + 0] = __fsub_rn(__fsub_rn(2.f * __uint_as_float(rg[cc][q + 0]), ni), nj.x);
                        v[q + 1] = __fsub_rn(__fsub_rn(2.f * __uint_as_float(rg[cc][q + 1]), ni), nj.y);
                        v[q + 2] = __fsub_rn(__fsub_rn(2.f * __uint_as_float(rg[cc][q + 2]), ni), nj.z);
                        v[q + 3] = __fsub_rn(__fsub_rn(2.f * __uint_as_float(rg[cc][q + 3]), ni), nj.w);
                    }
                    const int m0 = wr * BM;
                    if (m0 >= N || c0 >= N) continue;  // no element of this block inside S (uniform)
                    if (!diag) {
                        unsigned char* bd = stg_all + (ch & 1) * (2 * SY_BOX);
                        OT* bt = reinterpret_cast<OT*>(bd + SY_BOX);
                        // the stores issued from these boxes two blocks ago have read them
                        if (tid == 0) bulk_wait_read_1();
                        epi_sync();
                        stage_direct<OT>(bd, tid, v);
#pragma unroll
                        for (int q = 0; q < 32; ++q) store1<OT>(bt + q * BM + tid, v[q]);
                        fence_proxy_async_smem();
                        epi_sync();
                        if (tid == 0) {
                            tma_store_2d(&tmSd, smem_addr(bd), c0, m0, pol);  // rows m0.., columns c0..
                            tma_store_2d(&tmSt, smem_addr(bt), m0, c0, pol);  // rows c0.., columns m0..
                            bulk_commit();
                        }
                        ++ch;
                    } else if (row < N) {
                        // diagonal block: S[row][j] for j >= row and S[j][row] for j > row
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            const int j = c0 + q;
                            if (j < N && j >= row) store1<OT>(S + (int64_t)row * ld + j, v[q]);
                            if (j < N && j > row) store1<OT>(S + (int64_t)j * ld + row, v[q]);
                        }
                    }
                }
            }
        }
        // the last stores must have read shared memory (and completed) before
        // the CTA leaves
        if (tid == 0) bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, SY_TMEM_COLS);
}

// Operands of the contraction (zero-padded to [npad][kpad] BF16; A or B may
// be null) and FP32 row norms (accumulated in FP64 from the FP32 points).
__global__ void pack_operands_kernel(const float* __restrict__ X, int N, int d, int split, int kpad,
                                     __nv_bfloat16* __restrict__ A, __nv_bfloat16* __restrict__ B,
                                     float* __restrict__ norms) {
    const int i = blockIdx.x;
    double acc = 0.0;
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        const float x = X[(int64_t)i * d + k];
        acc += (double)x * (double)x;
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        __nv_bfloat16* a = A ? A + (int64_t)i * kpad : nullptr;
        __nv_bfloat16* b = B ? B + (int64_t)i * kpad : nullptr;
        if (split) {
            const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
            if (a) { a[k] = hi; a[d + k] = hi; a[2 * d + k] = lo; }
            if (b) { b[k] = hi; b[d + k] = lo; b[2 * d + k] = hi; }
        } else {
            if (a) a[k] = hi;
            if (b) b[k] = hi;
        }
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        norms[i] = (float)t;
    }
}

// ---- nearest neighbours with tensor-core candidate distances ----------------
// One CTA per 128 query rows streams every KBN-column tile of candidates
// (KBN = 256 or 128): warp 4 loads the query operand once and the candidate
// K-chunks through a TMA ring, warp 5 issues the tcgen05.mma contractions
// into one of two TMEM accumulators (KBN columns each) so that the next
// tile's products overlap the epilogue of this one, and warps 0-3 (one
// query row per thread, its TMEM lane) turn dot products into squared
// distances
// ||q||^2 + ||c||^2 - 2 q.c and keep the M2 smallest per row in shared
// memory.  The candidate norm enters the contraction as two extra K columns
// (A: 1, 1; B: -||c||^2/2 split into BF16 hi and lo), so the accumulator
// holds v = q.c - ||c||^2/2 and the row's ranking key ||c||^2 - 2 q.c = -2v
// needs no per-candidate arithmetic: a 32-column batch is skipped after one
// max-reduction unless its largest v beats the row's threshold.  With the
// BF16 hi/lo split the keys carry an error of about 2^-16 of the norms; a
// second kernel recomputes the M2 candidates' distances exactly in FP32 and
// keeps the M nearest, so the M2 - M spare candidates absorb the rounding of
// the first pass.
constexpr int KT_RING_MAX = 4;  // candidate K-chunk stages (fewer when shared memory is short)
constexpr int KT_MAXM2 = 80;    // candidates kept per row by the first pass
// per-row buffer of threshold-passing candidates of one 32-column batch (128-wide
// tiles) or of one 16-column half batch (256-wide tiles, where shared memory is short)
__host__ __device__ constexpr int knn_pend(int kbn) { return kbn == 256 ? 16 : 32; }
constexpr int KT_THREADS = 192; // 4 epilogue warps, 1 producer warp, 1 MMA warp
constexpr int KT_HEAP_D = 4;    // arity of the per-row candidate heap
// candidates per tile KBN: 256 (one M = 128, N = 256 MMA per K step) where
// shared memory allows, else 128
__host__ __device__ constexpr uint32_t knn_idesc(int kbn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kbn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

struct KnnTcArgs {
    const int32_t* cid;   // candidate c's global id (null: c)
    const int32_t* qperm; // operand row r holds query qperm[r] (null: r)
    const int32_t* cperm; // operand column j holds candidate cperm[j] (null: j)
    const int32_t* qkey;  // [Nq] spatial bucket of operand row r, increasing (null: no rotation)
    const int32_t* ckey;  // [Nc] spatial bucket of operand column j, increasing
    const int32_t* self_col;  // [Nq] operand column holding query r's own point, -1 none (null: see exclude_self)
    int Nq, Nc, M2, kchunks, ring;
    int exclude_self;     // without self_col: drop column r for row r (queries and candidates in the same order)
    int32_t* cand;        // out [Nq][M2] candidate indices per query, -1 where fewer
    unsigned* status;
};

// at least 116 KB: one CTA per SM, so its 2 KBN-column TMEM allocation never waits
size_t knn_tc_smem_bytes(int kchunks, int ring, int M2, int kbn) {
    const size_t b = 1024 + (size_t)kchunks * BM * BK * 2 + (size_t)ring * kbn * BK * 2 + (size_t)M2 * BM * 8 +
                     (size_t)knn_pend(kbn) * BM * 8;
    return b < 116 * 1024 ? 116 * 1024 : b;
}

template <int KBN>
__global__ void __launch_bounds__(KT_THREADS, 1) knn_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                              const __grid_constant__ CUtensorMap tmB,
                                                              const KnnTcArgs p) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t sA = base;                                          // kchunks x [128][64] BF16
    const uint32_t sB = sA + (uint32_t)p.kchunks * BM * BK * 2;        // ring x [256][64] BF16
    const int R = p.ring;
    float* tdist = reinterpret_cast<float*>(smem_raw + (sB + R * KBN * BK * 2 - raw));  // heap [M2][128]
    int* tidx = reinterpret_cast<int*>(tdist + p.M2 * BM);                                   // [M2][128]
    constexpr int PEND = knn_pend(KBN);
    float* pdist = reinterpret_cast<float*>(tidx + p.M2 * BM);  // [PEND][128]
    int* pidx = reinterpret_cast<int*>(pdist + PEND * BM);      // [PEND][128]
    __shared__ uint64_t bars[1 + 2 * KT_RING_MAX + 4];  // a_full, b_full[R], b_empty[R], acc_full[2], acc_empty[2]
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t a_full = smem_addr(&bars[0]);
    const uint32_t b_full = a_full + 8, b_empty = b_full + 8 * KT_RING_MAX;
    const uint32_t acc_full = b_empty + 8 * KT_RING_MAX, acc_empty = acc_full + 16;
    const int m0 = blockIdx.x * BM;
    const int ntiles = (p.Nc + KBN - 1) / KBN;
    // With queries and candidates sorted by spatial bucket, candidate tiles
    // are visited from the one holding the first candidate of this query
    // tile's first bucket (wrapping), so the nearest candidates come first
    // and the row thresholds tighten at once (the bucket before it in the
    // sorted order is no nearer in space than any other).  Without buckets every CTA
    // scans from tile 0, in step with the others, sharing tiles in L2.
    int t0 = 0;
    if (p.qkey) {
        const int key = p.qkey[m0 < p.Nq ? m0 : p.Nq - 1];
        int lo = 0, hi = p.Nc;  // first column whose bucket is >= key
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (p.ckey[mid] < key) lo = mid + 1; else hi = mid;
        }
        t0 = (lo < p.Nc ? lo : p.Nc - 1) / KBN;
    }
    if (tid == 0) {
        mbar_init(a_full, 1);
        for (int q = 0; q < R; ++q) {
            mbar_init(b_full + 8 * q, 1);
            mbar_init(b_empty + 8 * q, 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(acc_full + 8 * q, 1);
            mbar_init(acc_empty + 8 * q, BM);
        }
        s_abort = 0;
        fence_mbarrier_init();
    }
    if (warp == 0) tmem_alloc(smem_addr(&tmem_slot), 2 * KBN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int* abort_flag = &s_abort;

    if (warp == 4) {
        if (lane == 0) {  // ---- producer
            mbar_arrive_expect_tx(a_full, (uint32_t)p.kchunks * BM * BK * 2);
            for (int kc = 0; kc < p.kchunks; ++kc) tma_load_2d(sA + (uint32_t)kc * BM * BK * 2, &tmA, kc * BK, m0, a_full);
            const int total = ntiles * p.kchunks;
            for (int g = 0; g < total && !*abort_flag; ++g) {
                const int st = g % R;
                if (g >= R && !mbar_wait(b_empty + 8 * st, (uint32_t)((g / R - 1) & 1), p.status)) {
                    *abort_flag = 1;
                    break;
                }
                const int t = g / p.kchunks, kc = g - t * p.kchunks;
                const int tt = t0 + t < ntiles ? t0 + t : t0 + t - ntiles;
                mbar_arrive_expect_tx(b_full + 8 * st, KBN * BK * 2);
                tma_load_2d(sB + (uint32_t)st * KBN * BK * 2, &tmB, kc * BK, tt * KBN, b_full + 8 * st);
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {  // ---- MMA issuer
            bool ok = mbar_wait(a_full, 0u, p.status);
            for (int t = 0; t < ntiles && ok && !*abort_flag; ++t) {
                const int buf = t & 1;
                if (t >= 2 && !(ok = mbar_wait(acc_empty + 8 * buf, (uint32_t)((t / 2 - 1) & 1), p.status))) break;
                tc_fence_after();
                for (int kc = 0; kc < p.kchunks; ++kc) {
                    const int g = t * p.kchunks + kc, st = g % R;
                    if (!(ok = mbar_wait(b_full + 8 * st, (uint32_t)((g / R) & 1), p.status))) break;
                    tc_fence_after();
                    const uint32_t a_s = sA + (uint32_t)kc * BM * BK * 2, b_s = sB + (uint32_t)st * KBN * BK * 2;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
                        umma_bf16(tmem + (uint32_t)(buf * KBN), desc_kmajor_sw128(a_s + 32 * kk),
                                  desc_kmajor_sw128(b_s + 32 * kk), knn_idesc(KBN), (kc > 0 || kk > 0) ? 1u : 0u);
                    umma_commit(b_empty + 8 * st);
                }
                if (!ok) break;
                umma_commit(acc_full + 8 * buf);
            }
            if (!ok) *abort_flag = 1;
        }
    } else {  // ---- epilogue: warps 0-3, thread = query row = TMEM lane
        const int row = m0 + tid;
        const int qrow = row < p.Nq ? (p.qperm ? p.qperm[row] : row) : -1;
        // the column never taken by this row (its own point), -1 none; the
        // heap keeps operand columns, mapped to candidates on output
        const int skip = p.self_col ? (row < p.Nq ? p.self_col[row] : -1) : (p.exclude_self ? row : -1);
        // the M2 smallest first-pass keys ||c||^2 - 2 q.c of this row as a
        // KT_HEAP_D-ary max-heap in shared memory (root = current threshold); columns below
        // the threshold are first appended to a short buffer (cheap even when
        // few lanes of the warp take the branch) and then pushed into the
        // heap by all lanes with pending candidates together
        int cnt = 0;
        float thr = kInf, vthr = -kInf;  // key < thr  <=>  v > vthr = -thr / 2
        const int M2 = p.M2;
        auto heap_push = [&](float dv, int j) {
            // KT_HEAP_D-ary max-heap: children of node c are D c + 1 .. D c + D,
            // so a sift passes fewer levels than in a binary heap and the
            // child loads of a level are independent
            if (cnt < M2) {  // sift up
                int c = cnt++;
                while (c > 0) {
                    const int par = (c - 1) / KT_HEAP_D;
                    const float pd = tdist[par * BM + tid];
                    if (pd >= dv) break;
                    tdist[c * BM + tid] = pd;
                    tidx[c * BM + tid] = tidx[par * BM + tid];
                    c = par;
                }
                tdist[c * BM + tid] = dv;
                tidx[c * BM + tid] = j;
            } else if (dv < tdist[tid]) {  // replace the root, sift down
                int c = 0;
                for (;;) {
                    const int ch0 = KT_HEAP_D * c + 1;
                    if (ch0 >= M2) break;
                    float cd = tdist[ch0 * BM + tid];
                    int ch = ch0;
#pragma unroll
                    for (int u = 1; u < KT_HEAP_D; ++u) {
                        if (ch0 + u < M2) {
                            const float x = tdist[(ch0 + u) * BM + tid];
                            if (x > cd) { cd = x; ch = ch0 + u; }
                        }
                    }
                    if (cd <= dv) break;
                    tdist[c * BM + tid] = cd;
                    tidx[c * BM + tid] = tidx[ch * BM + tid];
                    c = ch;
                }
                tdist[c * BM + tid] = dv;
                tidx[c * BM + tid] = j;
            }
            thr = cnt == M2 ? tdist[tid] : kInf;
            vthr = -0.5f * thr;
        };
        for (int t = 0; t < ntiles; ++t) {
            // warp-uniform decisions: the TMEM loads below are warp-collective
            if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
            const int buf = t & 1;
            const bool got = mbar_wait(acc_full + 8 * buf, (uint32_t)((t >> 1) & 1), p.status);
            if (!__all_sync(0xffffffffu, got)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int tt = t0 + t < ntiles ? t0 + t : t0 + t - ntiles;
            const bool full_tile = (tt + 1) * KBN <= p.Nc;
            // 128 columns per round: four TMEM loads in flight, one wait (the
            // epilogue warp is alone on its sub-partition, so the load
            // latency is paid once per round); the accumulator goes back to
            // the MMA warp as soon as the last round's values are in registers
            constexpr int RC = KBN < 128 ? KBN : 128;  // columns per round
#pragma unroll 1
            for (int hh = 0; hh < KBN / RC; ++hh) {
                uint32_t r[RC / 32][32];
                __syncwarp();
                const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(buf * KBN + RC * hh);
#pragma unroll
                for (int b = 0; b < RC / 32; ++b) tmem_ld_32x32b_x32_nowait(ta + 32 * b, r[b]);
                tmem_wait_ld(r[0]);
#pragma unroll
                for (int b = 1; b < RC / 32; ++b) tmem_tie(r[b]);
                if (hh == KBN / RC - 1) {
                    tc_fence_before();
                    mbar_arrive(acc_empty + 8 * buf);
                }
#pragma unroll
                for (int b = 0; b < RC / 32; ++b) {
                    const int jb = tt * KBN + RC * hh + 32 * b;
                    if (max32(r[b]) > vthr) {
                        // PEND columns at a time, each part buffered then
                        // pushed (a later part sees the tightened threshold)
#pragma unroll
                        for (int hq = 0; hq < 32 / PEND; ++hq) {
                            int np = 0;
#pragma unroll
                            for (int q = PEND * hq; q < PEND * hq + PEND; ++q) {
                                const float v = __uint_as_float(r[b][q]);
                                if (v > vthr && (full_tile || jb + q < p.Nc)) {
                                    pdist[np * BM + tid] = -2.f * v;
                                    pidx[np * BM + tid] = jb + q;
                                    ++np;
                                }
                            }
                            for (int k = 0; k < np; ++k) {
                                const int j = pidx[k * BM + tid];
                                if (j != skip) heap_push(pdist[k * BM + tid], j);
                            }
                        }
                    }
                }
            }
        }
        if (qrow >= 0)
            for (int m = 0; m < M2; ++m) {
                const int j = m < cnt ? tidx[m * BM + tid] : -1;
                p.cand[(int64_t)qrow * M2 + m] = (j >= 0 && p.cperm) ? p.cperm[j] : j;
            }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 2 * KBN);
}

// Exact re-rank of the first pass's candidates: one warp per query row,
// FP32 direct-difference distances accumulated in dimension order (the
// CUDA-core kNN's arithmetic), the M nearest by (distance, global index).
// (distance, global index) lexicographic order of two candidates
HAP_DEV bool cand_less(float da, int ga, float db, int gb) { return da < db || (da == db && ga < gb); }

// Bitonic sort of the warp's 32 R candidates into ascending order, element
// e = R * lane + r in register r of lane e / R: partners R or more elements
// apart are exchanged by shuffles, nearer ones within the lane.  Then the
// first M elements go out (index -1 and an infinite distance past the last
// valid candidate).
template <int R, int PER>
HAP_DEV void rerank_emit(const float (&dv)[PER], const int (&gv)[PER], int64_t i, int M,
                         int32_t* __restrict__ out_idx, float* __restrict__ out_dist) {
    const int lane = threadIdx.x & 31;
    float d[R];
    int g[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        d[r] = r < PER ? dv[r] : kInf;
        g[r] = r < PER ? gv[r] : 0x7fffffff;
    }
#pragma unroll
    for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= R) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int e = R * lane + r;
                    const float od = __shfl_xor_sync(0xffffffffu, d[r], j / R);
                    const int og = __shfl_xor_sync(0xffffffffu, g[r], j / R);
                    const bool keep_small = ((e & j) == 0) == ((e & k) == 0);
                    const bool other_less = cand_less(od, og, d[r], g[r]);
                    if (keep_small == other_less) {
                        d[r] = od;
                        g[r] = og;
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int r2 = r ^ j;
                    if (r2 > r) {
                        const int e = R * lane + r;
                        const bool ascending = (e & k) == 0;
                        if (cand_less(d[r2], g[r2], d[r], g[r]) == ascending) {
                            const float td = d[r];
                            const int tg = g[r];
                            d[r] = d[r2];
                            g[r] = g[r2];
                            d[r2] = td;
                            g[r2] = tg;
                        }
                    }
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int m = R * lane + r;
        if (m < M) {
            out_idx[i * M + m] = g[r] == 0x7fffffff ? -1 : g[r];
            out_dist[i * M + m] = d[r];
        }
    }
}

__global__ void knn_rerank_kernel(const float* __restrict__ Q, const float* __restrict__ C,
                                  const int32_t* __restrict__ cid, int Nq, int d, int M2, int M,
                                  const int32_t* __restrict__ cand, const unsigned* __restrict__ status,
                                  int32_t* __restrict__ out_idx, float* __restrict__ out_dist) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= Nq) return;
    if (*status) {  // the first pass gave up waiting: no result
        for (int m = lane; m < M; m += 32) {
            out_idx[i * M + m] = -1;
            out_dist[i * M + m] = __int_as_float(0x7fc00000);
        }
        return;
    }
    constexpr int PER = (KT_MAXM2 + 31) / 32;
    float dv[PER];
    int gv[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int q = lane + 32 * u;
        const int j = q < M2 ? cand[i * M2 + q] : -1;
        dv[u] = kInf;
        gv[u] = 0x7fffffff;
        if (j >= 0) {
            float acc = 0.f;
            for (int k = 0; k < d; ++k) {
                const float e = Q[i * d + k] - C[(int64_t)j * d + k];
                acc = fmaf(e, e, acc);
            }
            dv[u] = acc;
            gv[u] = cid ? cid[j] : j;
        }
    }
    // ascending (distance, global index) order of all candidates by one
    // warp-wide bitonic sort; element m is then the m-th nearest
    if (M2 <= 32) rerank_emit<1>(dv, gv, i, M, out_idx, out_dist);
    else if (M2 <= 64) rerank_emit<2>(dv, gv, i, M, out_idx, out_dist);
    else rerank_emit<4>(dv, gv, i, M, out_idx, out_dist);
}

// Operands of the nearest-neighbour contraction (zero-padded to [npad][kpad]
// BF16): queries A = [hi, hi, lo, 1, 1], candidates B = [hi, lo, hi, h, l]
// with h + l = -||c||^2 / 2 (BF16 hi and lo; the norm accumulated in FP64).
__global__ void pack_knn_kernel(const float* __restrict__ X, const int32_t* __restrict__ perm, int N, int d,
                                int kpad, int is_b, __nv_bfloat16* __restrict__ out) {
    const int i = blockIdx.x;
    const int64_t src = perm ? perm[i] : i;
    __nv_bfloat16* o = out + (int64_t)i * kpad;
    double acc = 0.0;
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        const float x = X[src * d + k];
        acc += (double)x * (double)x;
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
        o[k] = hi;
        o[d + k] = is_b ? lo : hi;
        o[2 * d + k] = is_b ? hi : lo;
    }
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        if (is_b) {
            const float h = (float)(-0.5 * t);
            const __nv_bfloat16 bh = __float2bfloat16_rn(h);
            o[3 * d] = bh;
            o[3 * d + 1] = __float2bfloat16_rn((float)(-0.5 * t - (double)__bfloat162float(bh)));
        } else {
            o[3 * d] = __float2bfloat16_rn(1.f);
            o[3 * d + 1] = __float2bfloat16_rn(1.f);
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    return fn;
}

bool encode_operand_map(CUtensorMap* map, void* ptr, int64_t rows, int64_t kpad, int box_rows = BM) {
    auto enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// Tensor map of S (N x N, row stride ld) for the build's TMA stores: direct
// boxes of 128 rows x 32 columns staged with the 128-byte (FP32 rows) or
// 64-byte (BF16) swizzle, transposed boxes of 32 rows x 128 columns staged
// plain.  Stores clip at N.
bool encode_s_map(CUtensorMap* map, void* S, int64_t N, int64_t ld, int s_bf16, bool swizzled) {
    auto enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * (s_bf16 ? 2 : 4)};
    const cuuint32_t box[2] = {swizzled ? 32u : 128u, swizzled ? 128u : 32u};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapSwizzle sw = !swizzled ? CU_TENSOR_MAP_SWIZZLE_NONE
                                  : s_bf16  ? CU_TENSOR_MAP_SWIZZLE_64B
                                            : CU_TENSOR_MAP_SWIZZLE_128B;
    return enc(map, s_bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, S, dims, strides,
               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct Scratch {
    int64_t npad, kpad;
    size_t a_off, b_off, n_off, t_off, total;  // operands, norms, tile list of the symmetric build
};
Scratch scratch_layout(int64_t N, int64_t d, int split) {
    Scratch s;
    s.kpad = ((split ? 3 * d : d) + BK - 1) / BK * BK;
    s.npad = (N + BM - 1) / BM * BM;
    const size_t op = (size_t)s.npad * s.kpad * 2;
    s.a_off = 0;
    s.b_off = (op + 1023) / 1024 * 1024;
    s.n_off = s.b_off + (op + 1023) / 1024 * 1024;
    s.t_off = (s.n_off + (size_t)s.npad * 4 + 255) / 256 * 256;
    s.total = s.t_off + (size_t)sym_tile_count((int)(s.npad / BM)) * 4 + 2048;
    return s;
}

}  // namespace

size_t sbuild_tc_scratch_bytes(int64_t N, int64_t d, int split) { return scratch_layout(N, d, split).total; }

cudaError_t launch_sbuild_tc(const float* X, int64_t N, int64_t d, int split, void* S, int s_bf16, int64_t ld,
                             void* scratch, unsigned* status, cudaStream_t st, int* kernels) {
    *kernels = 0;
    const Scratch sl = scratch_layout(N, d, split);
    // operand tiles 1024-byte aligned (the layout reserves the slack)
    char* base = reinterpret_cast<char*>(((uintptr_t)scratch + 1023) & ~(uintptr_t)1023);
    __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(base + sl.a_off);
    __nv_bfloat16* B = reinterpret_cast<__nv_bfloat16*>(base + sl.b_off);
    float* norms = reinterpret_cast<float*>(base + sl.n_off);
    cudaError_t err = cudaMemsetAsync(base, 0, sl.n_off + (size_t)sl.npad * 4, st);
    if (err != cudaSuccess) return err;
    pack_operands_kernel<<<(unsigned)N, 64, 0, st>>>(X, (int)N, (int)d, split, (int)sl.kpad, A, B, norms);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    *kernels = 1;
    CUtensorMap mA;
    if (!encode_operand_map(&mA, A, sl.npad, sl.kpad)) return cudaErrorNotSupported;
    const int kchunks = (int)(sl.kpad / BK);
    // the symmetric persistent kernel (a ring of at least two stages fits on
    // every GPU this targets; otherwise the build is not supported)
    int dev = 0, smem_optin = 0, n_sm = 0;
    err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    const size_t room = (size_t)smem_optin - 4096;  // the kernel's static shared memory (2.2 KB)
    int ring = SY_RING_MAX;
    while (ring >= 2 && sbuild_sym_smem_bytes(ring) > room) --ring;
    CUtensorMap mBw, mSd, mSt;
    if (ring >= 2 && encode_operand_map(&mBw, B, sl.npad, sl.kpad, SY_BN) && encode_s_map(&mSd, S, N, ld, s_bf16, true) &&
        encode_s_map(&mSt, S, N, ld, s_bf16, false)) {
        const int T = (int)(sl.npad / BM), T2 = (T + 1) / 2;
        const int64_t tiles = sym_tile_count(T);
        int32_t* tlist = reinterpret_cast<int32_t*>(base + sl.t_off);
        sym_order_kernel<<<(unsigned)((T + kSyGroup - 1) / kSyGroup), (unsigned)T2, 0, st>>>(T, tlist);
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        *kernels = 2;
        const unsigned grid = (unsigned)(tiles < n_sm ? tiles : n_sm);
        const size_t smem = sbuild_sym_smem_bytes(ring);
        if (s_bf16) {
            auto k = sbuild_sym_kernel<__nv_bfloat16>;
            err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) return err;
            k<<<grid, SY_THREADS, smem, st>>>(mA, mBw, mSd, mSt, norms, tlist, static_cast<__nv_bfloat16*>(S), (int)N, ld,
                                               kchunks, ring, T, tiles, status);
        } else {
            auto k = sbuild_sym_kernel<float>;
            err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) return err;
            k<<<grid, SY_THREADS, smem, st>>>(mA, mBw, mSd, mSt, norms, tlist, static_cast<float*>(S), (int)N, ld, kchunks,
                                               ring, T, tiles, status);
        }
        err = cudaGetLastError();
        if (err == cudaSuccess) *kernels = 3;
        return err;
    }
    return cudaErrorNotSupported;
}


int knn_tc_max_candidates() { return KT_MAXM2; }

// Spatial order of one kNN problem: operand row r / column j hold query
// qperm[r] / candidate cperm[j], with bucket keys qkey / ckey increasing.
struct KnnOrder {
    const int32_t *qperm = nullptr, *cperm = nullptr, *qkey = nullptr, *ckey = nullptr;
};

// rerank 0: the first pass alone, its M2 candidates per query straight into
// idx [Nq][M2] (unordered, BF16-split keys; dist unused)
// wide: 256 candidates per tile where they fit (the MMA stream bounds the
// kNN of a set among itself); else 128 (a subset search is bound by the heap
// inserts of its first tiles, which wider tiles only make longer)
static cudaError_t knn_tc_core(const float* Q, int64_t Nq, const float* C, const int32_t* cid, int64_t Nc, int64_t d,
                               int M, int M2, int32_t* idx, float* dist, const KnnOrder& ord, int exclude_self,
                               const int32_t* self_col, int rerank, bool wide, cudaStream_t st) {
    if (M2 > KT_MAXM2 || M2 < M || d > 64) return cudaErrorInvalidValue;
    const int64_t kpad = (3 * d + 2 + BK - 1) / BK * BK;
    // tile width and ring: 256 candidates per tile when at least three
    // K-chunk stages fit beside the query operand and the heaps, else 128
    int dev = 0, smem_limit = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int kchunks = (int)(kpad / BK);
    auto ring_for = [&](int kbn) {
        int r = KT_RING_MAX;
        while (r > 2 && knn_tc_smem_bytes(kchunks, r, M2, kbn) > (size_t)smem_limit) --r;
        return r;
    };
    int KBN = 256, ring = ring_for(256);
    if (!wide || ring < 3 || knn_tc_smem_bytes(kchunks, ring, M2, 256) > (size_t)smem_limit) {
        KBN = 128;
        ring = ring_for(128);
    }
    const size_t smem = knn_tc_smem_bytes(kchunks, ring, M2, KBN);
    if (smem > (size_t)smem_limit) return cudaErrorNotSupported;
    const int64_t qpad = (Nq + BM - 1) / BM * BM, cpad = (Nc + KBN - 1) / KBN * KBN;
    const size_t aB = (size_t)qpad * kpad * 2, bB = (size_t)cpad * kpad * 2;
    const size_t off_b = (aB + 1023) / 1024 * 1024;
    const size_t off_cand = off_b + (bB + 1023) / 1024 * 1024;
    const size_t off_status = off_cand + ((size_t)Nq * M2 * 4 + 255) / 256 * 256;
    const size_t total = off_status + 256 + 1024;
    char* raw = nullptr;
    cudaError_t err = cudaMallocAsync(reinterpret_cast<void**>(&raw), total, st);
    if (err != cudaSuccess) return err;
    char* base = reinterpret_cast<char*>(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(base);
    __nv_bfloat16* B = reinterpret_cast<__nv_bfloat16*>(base + off_b);
    int32_t* cand = reinterpret_cast<int32_t*>(base + off_cand);
    unsigned* status = reinterpret_cast<unsigned*>(base + off_status);
    do {
        if ((err = cudaMemsetAsync(base, 0, off_cand, st)) != cudaSuccess) break;
        if ((err = cudaMemsetAsync(status, 0, 16, st)) != cudaSuccess) break;
        pack_knn_kernel<<<(unsigned)Nq, 64, 0, st>>>(Q, ord.qperm, (int)Nq, (int)d, (int)kpad, 0, A);
        pack_knn_kernel<<<(unsigned)Nc, 64, 0, st>>>(C, ord.cperm, (int)Nc, (int)d, (int)kpad, 1, B);
        if ((err = cudaGetLastError()) != cudaSuccess) break;
        CUtensorMap mA, mB;
        if (!encode_operand_map(&mA, A, qpad, kpad) || !encode_operand_map(&mB, B, cpad, kpad, KBN)) {
            err = cudaErrorNotSupported;
            break;
        }
        KnnTcArgs a;
        a.cid = cid;
        a.qperm = ord.qperm;
        a.cperm = ord.cperm;
        a.qkey = ord.qkey;
        a.ckey = ord.ckey;
        a.exclude_self = exclude_self;
        a.self_col = self_col;
        a.Nq = (int)Nq;
        a.Nc = (int)Nc;
        a.M2 = M2;
        a.kchunks = (int)(kpad / BK);
        a.cand = rerank ? cand : idx;
        a.status = status;
        a.ring = ring;
        auto kern = KBN == 256 ? knn_tc_kernel<256> : knn_tc_kernel<128>;
        if ((err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            break;
        kern<<<(unsigned)(qpad / BM), KT_THREADS, smem, st>>>(mA, mB, a);
        if ((err = cudaGetLastError()) != cudaSuccess || !rerank) break;
        knn_rerank_kernel<<<(unsigned)((Nq * 32 + 255) / 256), 256, 0, st>>>(Q, C, cid, (int)Nq, (int)d, M2, M, cand,
                                                                            status, idx, dist);
        err = cudaGetLastError();
    } while (0);
    cudaError_t e2 = cudaFreeAsync(raw, st);
    return err != cudaSuccess ? err : e2;
}

// inv[cid[j]] = j for the candidates whose global id is a query index
__global__ void inverse_subset_kernel(const int32_t* __restrict__ cid, int64_t Nc, int64_t Nq,
                                      int32_t* __restrict__ inv) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < Nc && cid[j] >= 0 && cid[j] < Nq) inv[cid[j]] = (int32_t)j;
}

__global__ void pivot_rows_kernel(const float* __restrict__ C, int64_t d, int64_t step, float* __restrict__ out) {
    const int64_t i = blockIdx.x;
    for (int64_t k = threadIdx.x; k < d; k += blockDim.x) out[i * d + k] = C[i * step * d + k];
}

// The first pass prunes a 32-column batch unless it beats a row's current
// threshold, which is cheap only once the threshold is close to its final
// value.  So for the kNN of a point set among itself the points are first
// sorted by their nearest of P pivots (every 128th point: buckets of about
// one tile; the bucket search is the first pass alone with one candidate),
// and each query tile scans the candidates from its own bucket on.  The
// result does not depend on the order: the re-rank sorts by (distance,
// index).  Queries against another set (hubs) keep the input order: there
// the heap inserts of the first tiles dominate (M2 = 80 for M = 64), and
// buckets of one or four tiles of hubs measured no faster.
cudaError_t launch_knn_tc(const float* Q, int64_t Nq, const float* C, const int32_t* cid, int64_t Nc, int64_t d, int M,
                          int M2, int32_t* idx, float* dist, cudaStream_t st, int64_t* launches) {
    if (M2 > KT_MAXM2 || M2 < M || d > 64) return cudaErrorInvalidValue;
    const bool self = Q == C && cid == nullptr && Nq == Nc;
    const int64_t P = Nc / 128;
    if (!self) {
        // queries Q are the N points, candidates their subset cid: the
        // column holding a query's own point comes from the inverse of cid
        int32_t* inv = nullptr;
        cudaError_t err = cudaMallocAsync(reinterpret_cast<void**>(&inv), (size_t)Nq * 4, st);
        if (err != cudaSuccess) return err;
        do {
            if ((err = cudaMemsetAsync(inv, 0xff, (size_t)Nq * 4, st)) != cudaSuccess) break;
            if (cid) {
                inverse_subset_kernel<<<(unsigned)((Nc + 255) / 256), 256, 0, st>>>(cid, Nc, Nq, inv);
                if ((err = cudaGetLastError()) != cudaSuccess) break;
            }
            err = knn_tc_core(Q, Nq, C, cid, Nc, d, M, M2, idx, dist, KnnOrder{}, 0, inv, 1, false, st);
        } while (0);
        if (launches) *launches += (cid ? 1 : 0) + 4;  // inverse map; two operand packs, first pass, re-rank
        cudaError_t e2 = cudaFreeAsync(inv, st);
        return err != cudaSuccess ? err : e2;
    }
    if (P < 8) {
        if (launches) *launches += 4;  // two operand packs, the first pass, the re-rank
        return knn_tc_core(Q, Nq, C, cid, Nc, d, M, M2, idx, dist, KnnOrder{}, 1, nullptr, 1, true, st);
    }
    int bits = 1;
    while (((int64_t)1 << bits) < P) ++bits;
    // pivots; the bucket search (two packs and a first pass); the sort (5
    // kernels per 9-bit pass); the ordered search
    if (launches) *launches += 1 + 3 + 5 * ((bits + kRadixBits - 1) / kRadixBits) + 4;
    // scratch: pivots, and per point its bucket, the sorted buckets and the
    // permutation
    const size_t bytes = (size_t)P * d * 4 + (size_t)Nq * 12 + 1024;
    char* raw = nullptr;
    cudaError_t err = cudaMallocAsync(reinterpret_cast<void**>(&raw), bytes, st);
    if (err != cudaSuccess) return err;
    float* piv = reinterpret_cast<float*>(raw);
    int32_t* bkt = reinterpret_cast<int32_t*>(piv + P * d);
    int32_t* key = bkt + Nq;
    int32_t* perm = key + Nq;
    do {
        pivot_rows_kernel<<<(unsigned)P, 64, 0, st>>>(C, d, Nc / P, piv);
        if ((err = cudaGetLastError()) != cudaSuccess) break;
        // the approximately nearest pivot (first-pass keys) is bucket enough
        if ((err = knn_tc_core(Q, Nq, piv, nullptr, P, d, 1, 1, bkt, nullptr, KnnOrder{}, 0, nullptr, 0, true, st)) !=
            cudaSuccess)
            break;
        if ((err = stable_sort_keys(bkt, Nq, bits, key, perm, st)) != cudaSuccess) break;
        KnnOrder ord;
        ord.qperm = ord.cperm = perm;
        ord.qkey = ord.ckey = key;
        err = knn_tc_core(Q, Nq, C, cid, Nc, d, M, M2, idx, dist, ord, 1, nullptr, 1, true, st);
    } while (0);
    cudaError_t e2 = cudaFreeAsync(raw, st);
    return err != cudaSuccess ? err : e2;
}
}  // namespace hap
