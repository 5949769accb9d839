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
// Kernel layout: one CTA (4 warps) per 128 x 128 output tile.  Thread 0
// streams 128 x 64 BF16 K-chunks of A and B with TMA (128-byte swizzle) into
// a shared-memory ring and issues the tcgen05.mma instructions (M = N = 128,
// K = 16) accumulating in 128 TMEM columns; tcgen05.commit frees a ring stage
// once the MMAs reading it finish.  The 4 warps then read their 32 TMEM
// lanes (rows) with tcgen05.ld and write s to global memory.  The kernel is
// bound by the N^2 output writes for d <= 192.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "hap_common.cuh"
#include "hap_internal.h"

namespace hap {
namespace {

constexpr int BM = 128, BN = 128, BK = 64;  // tile and K-chunk (64 BF16 = 128 bytes)
constexpr int kRing = 3;                     // K-chunk stages in shared memory
constexpr uint32_t kChunkBytes = (BM + BN) * BK * 2;
constexpr uint32_t kTmemCols = 128;

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
HAP_DEV void tmem_ld_32x32b_x32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
// Bits: [0,14) start >> 4, [16,30) leading offset >> 4 (unused here),
// [32,46) stride offset >> 4, [46,48) version 1, [61,64) swizzle (2 = 128B).
HAP_DEV uint64_t desc_kmajor_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

template <typename OT>
HAP_DEV void store_row32(OT* dst, const float (&v)[32]);
template <>
HAP_DEV void store_row32<float>(float* dst, const float (&v)[32]) {
#pragma unroll
    for (int q = 0; q < 32; q += 4) *reinterpret_cast<float4*>(dst + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
}
template <>
HAP_DEV void store_row32<__nv_bfloat16>(__nv_bfloat16* dst, const float (&v)[32]) {
#pragma unroll
    for (int q = 0; q < 32; q += 8) {
        uint4 u;
        __nv_bfloat162 p0 = __floats2bfloat162_rn(v[q], v[q + 1]), p1 = __floats2bfloat162_rn(v[q + 2], v[q + 3]);
        __nv_bfloat162 p2 = __floats2bfloat162_rn(v[q + 4], v[q + 5]), p3 = __floats2bfloat162_rn(v[q + 6], v[q + 7]);
        u.x = *reinterpret_cast<uint32_t*>(&p0);
        u.y = *reinterpret_cast<uint32_t*>(&p1);
        u.z = *reinterpret_cast<uint32_t*>(&p2);
        u.w = *reinterpret_cast<uint32_t*>(&p3);
        *reinterpret_cast<uint4*>(dst + q) = u;
    }
}

template <typename OT>
__global__ void __launch_bounds__(128, 1) sbuild_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB,
                                                          const float* __restrict__ norms, OT* __restrict__ S,
                                                          int N, int64_t ld, int kchunks, unsigned* status) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned base for the 128-byte swizzled tiles
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    __shared__ uint64_t bars[2 * kRing + 1];  // full[kRing], empty[kRing], done
    __shared__ uint32_t tmem_base_slot;
    __shared__ float col_norm[BN];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const uint32_t bar_full = smem_addr(&bars[0]), bar_empty = smem_addr(&bars[kRing]), bar_done = smem_addr(&bars[2 * kRing]);

    if (tid == 0) {
        for (int q = 0; q < 2 * kRing + 1; ++q) mbar_init(smem_addr(&bars[q]), 1);
        fence_mbarrier_init();
    }
    if (warp == 0) tmem_alloc(smem_addr(&tmem_base_slot), kTmemCols);
    col_norm[tid] = (n0 + tid < N) ? norms[n0 + tid] : 0.f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_slot;

    bool ok = true;
    if (tid == 0) {
        auto load_chunk = [&](int k) {
            const int st = k % kRing;
            const uint32_t sa = base + (uint32_t)st * kChunkBytes, sb = sa + BM * BK * 2;
            mbar_arrive_expect_tx(bar_full + 8 * st, kChunkBytes);
            tma_load_2d(sa, &tmA, k * BK, m0, bar_full + 8 * st);
            tma_load_2d(sb, &tmB, k * BK, n0, bar_full + 8 * st);
        };
        for (int k = 0; k < kchunks && k < kRing; ++k) load_chunk(k);
        for (int k = 0; k < kchunks && ok; ++k) {
            const int st = k % kRing;
            ok = mbar_wait(bar_full + 8 * st, (uint32_t)(k / kRing) & 1u, status);
            if (!ok) break;
            tc_fence_after();
            const uint32_t sa = base + (uint32_t)st * kChunkBytes, sb = sa + BM * BK * 2;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)  // 16 BF16 = 32 bytes per MMA along K
                umma_bf16(tmem, desc_kmajor_sw128(sa + 32 * kk), desc_kmajor_sw128(sb + 32 * kk), kIdesc,
                          (k > 0 || kk > 0) ? 1u : 0u);
            umma_commit(bar_empty + 8 * st);
            if (k + kRing < kchunks) {
                ok = mbar_wait(bar_empty + 8 * st, (uint32_t)(k / kRing) & 1u, status);
                if (ok) load_chunk(k + kRing);
            }
        }
        if (ok) umma_commit(bar_done);
        else mbar_arrive(bar_done);  // release the epilogue; results are flagged invalid
    }
    __syncwarp();
    mbar_wait(bar_done, 0u, status);
    __syncwarp();  // tcgen05.ld below is warp-collective
    tc_fence_after();

    // ---- epilogue: warp w owns TMEM lanes (tile rows) 32w .. 32w+31 ---------
    const int row = m0 + 32 * warp + lane;
    const float ni = row < N ? norms[row] : 0.f;
#pragma unroll 1
    for (int cc = 0; cc < BN / 32; ++cc) {
        float v[32];
        tmem_ld_32x32b_x32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * cc), v);
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = __fsub_rn(__fsub_rn(2.f * v[q], ni), col_norm[32 * cc + q]);
        const int c0 = n0 + 32 * cc;
        if (row < N) {
            OT* dst = S + (int64_t)row * ld + c0;
            if (c0 + 32 <= N) {
                store_row32<OT>(dst, v);
            } else {
#pragma unroll
                for (int q = 0; q < 32; ++q)
                    if (c0 + q < N) dst[q] = (OT)v[q];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// Operands of the contraction (zero-padded to [npad][kpad] BF16) and FP32
// row norms (accumulated in FP64 from the FP32 points).
__global__ void pack_operands_kernel(const float* __restrict__ X, int N, int d, int split, int kpad,
                                     __nv_bfloat16* __restrict__ A, __nv_bfloat16* __restrict__ B,
                                     float* __restrict__ norms) {
    const int i = blockIdx.x;
    double acc = 0.0;
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        const float x = X[(int64_t)i * d + k];
        acc += (double)x * (double)x;
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        __nv_bfloat16* a = A + (int64_t)i * kpad;
        __nv_bfloat16* b = B + (int64_t)i * kpad;
        if (split) {
            const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
            a[k] = hi; a[d + k] = hi; a[2 * d + k] = lo;
            b[k] = hi; b[d + k] = lo; b[2 * d + k] = hi;
        } else {
            a[k] = hi;
            b[k] = hi;
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

bool encode_operand_map(CUtensorMap* map, void* ptr, int64_t rows, int64_t kpad) {
    auto enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

struct Scratch {
    int64_t npad, kpad;
    size_t a_off, b_off, n_off, total;
};
Scratch scratch_layout(int64_t N, int64_t d, int split) {
    Scratch s;
    s.kpad = ((split ? 3 * d : d) + BK - 1) / BK * BK;
    s.npad = (N + BM - 1) / BM * BM;
    const size_t op = (size_t)s.npad * s.kpad * 2;
    s.a_off = 0;
    s.b_off = (op + 1023) / 1024 * 1024;
    s.n_off = s.b_off + (op + 1023) / 1024 * 1024;
    s.total = s.n_off + (size_t)s.npad * 4 + 2048;
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
    CUtensorMap mA, mB;
    if (!encode_operand_map(&mA, A, sl.npad, sl.kpad) || !encode_operand_map(&mB, B, sl.npad, sl.kpad))
        return cudaErrorNotSupported;
    const int kchunks = (int)(sl.kpad / BK);
    const size_t smem = (size_t)kRing * kChunkBytes + 1024;
    const dim3 grid((unsigned)(sl.npad / BN), (unsigned)(sl.npad / BM));
    if (s_bf16) {
        auto k = sbuild_tc_kernel<__nv_bfloat16>;
        err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        k<<<grid, 128, smem, st>>>(mA, mB, norms, static_cast<__nv_bfloat16*>(S), (int)N, ld, kchunks, status);
    } else {
        auto k = sbuild_tc_kernel<float>;
        err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        k<<<grid, 128, smem, st>>>(mA, mB, norms, static_cast<float*>(S), (int)N, ld, kchunks, status);
    }
    err = cudaGetLastError();
    if (err == cudaSuccess) *kernels = 2;
    return err;
}

}  // namespace hap
