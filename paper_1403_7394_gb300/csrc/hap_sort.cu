// Exclusive prefix sums and a stable radix sort of int32 keys, shared by the
// sparse column index (entries sorted by column) and the spatial order of the
// nearest-neighbour search (points sorted by their nearest pivot).
#include <cuda_runtime.h>
#include <stdint.h>

#include "hap_common.cuh"
#include "hap_internal.h"

namespace hap {
namespace {

constexpr int kScanT = 256, kScanPer = 8, kScanTile = kScanT * kScanPer;

HAP_DEV int64_t block_exclusive_scan(int64_t v, int64_t* warp_sums, int64_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const int64_t t = warp_sums[w];
            warp_sums[w] = run;
            run += t;
        }
        *total = run;
    }
    __syncthreads();
    const int64_t out = x - v + warp_sums[warp];
    __syncthreads();
    return out;
}

__global__ void scan_tile_sums_kernel(const int* __restrict__ in, int64_t n, int64_t* __restrict__ tsum) {
    __shared__ int64_t ws[kScanT / 32];
    __shared__ int64_t tot;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int64_t v = 0;
    for (int u = 0; u < kScanPer; ++u) v += (base + u < n) ? in[base + u] : 0;
    block_exclusive_scan(v, ws, &tot);
    if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

__global__ void scan_tile_offsets_kernel(int64_t* __restrict__ tsum, int64_t ntiles) {
    __shared__ int64_t ws[kScanT / 32];
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < ntiles; b0 += kScanT) {
        const int64_t k = b0 + threadIdx.x;
        const int64_t v = k < ntiles ? tsum[k] : 0;
        const int64_t ex = block_exclusive_scan(v, ws, &tot);
        if (k < ntiles) tsum[k] = carry + ex;
        carry += tot;
        __syncthreads();
    }
}

template <typename OT>
__global__ void scan_apply_kernel(const int* __restrict__ in, int64_t n, const int64_t* __restrict__ toff,
                                  OT* __restrict__ out) {
    __shared__ int64_t ws[kScanT / 32];
    __shared__ int64_t tot;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int64_t v = 0;
    for (int u = 0; u < kScanPer; ++u) v += (base + u < n) ? in[base + u] : 0;
    int64_t run = block_exclusive_scan(v, ws, &tot) + toff[blockIdx.x];
    for (int u = 0; u < kScanPer; ++u) {
        if (base + u < n) {
            out[base + u] = (OT)run;
            run += in[base + u];
        }
    }
}

// Stable least-significant-digit radix sort of (key, value) pairs, 9-bit
// digits, chunks of kRadixChunk consecutive elements per CTA.  Pass p orders
// by digit p with ties kept in their current order, so after the last pass
// equal keys keep their input order.
constexpr int kRadixBins = 1 << kRadixBits, kRadixT = 256, kRadixRounds = 16;
constexpr int kRadixChunk = kRadixT * kRadixRounds;

__global__ void radix_hist_kernel(const int32_t* __restrict__ key, int64_t n, int shift, int nchunks,
                                  int* __restrict__ hist) {
    __shared__ int h[kRadixBins];
    for (int d = threadIdx.x; d < kRadixBins; d += kRadixT) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixChunk;
    for (int r = 0; r < kRadixRounds; ++r) {
        const int64_t idx = base + (int64_t)r * kRadixT + threadIdx.x;
        if (idx < n) atomicAdd(&h[(key[idx] >> shift) & (kRadixBins - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadixBins; d += kRadixT) hist[(int64_t)d * nchunks + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(kRadixT) radix_scatter_kernel(
    const int32_t* __restrict__ key, const int32_t* __restrict__ val, int64_t n, int shift, int nchunks,
    const int* __restrict__ off, int32_t* __restrict__ okey, int32_t* __restrict__ oval) {
    __shared__ int running[kRadixBins];
    __shared__ int wcnt[kRadixT / 32][kRadixBins];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int d = tid; d < kRadixBins; d += kRadixT) {
        running[d] = 0;
        for (int w = 0; w < kRadixT / 32; ++w) wcnt[w][d] = 0;
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixChunk;
    for (int r = 0; r < kRadixRounds; ++r) {
        const int64_t idx = base + (int64_t)r * kRadixT + tid;
        const bool valid = idx < n;
        const int32_t k = valid ? key[idx] : 0;
        const int32_t v = valid ? (val ? val[idx] : (int32_t)idx) : 0;
        const int d = valid ? ((k >> shift) & (kRadixBins - 1)) : kRadixBins;  // invalid: own class
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int before = running[d] + rank;
            for (int w = 0; w < warp; ++w) before += wcnt[w][d];
            const int64_t pos = (int64_t)off[(int64_t)d * nchunks + blockIdx.x] + before;
            okey[pos] = k;
            oval[pos] = v;
        }
        __syncthreads();
        for (int d2 = tid; d2 < kRadixBins; d2 += kRadixT) {
            int sum = 0;
            for (int w = 0; w < kRadixT / 32; ++w) {
                sum += wcnt[w][d2];
                wcnt[w][d2] = 0;
            }
            running[d2] += sum;
        }
        __syncthreads();
    }
}


}  // namespace

int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

template <typename OT>
static cudaError_t scan_exclusive_t(const int* in, int64_t n, OT* out, int64_t* tsum, cudaStream_t st) {
    const int64_t tiles = scan_tiles(n);
    scan_tile_sums_kernel<<<(unsigned)tiles, kScanT, 0, st>>>(in, n, tsum);
    scan_tile_offsets_kernel<<<1, kScanT, 0, st>>>(tsum, tiles);
    scan_apply_kernel<OT><<<(unsigned)tiles, kScanT, 0, st>>>(in, n, tsum, out);
    return cudaGetLastError();
}

cudaError_t scan_exclusive(const int* in, int64_t n, int* out, int64_t* tsum, cudaStream_t st) {
    return scan_exclusive_t<int>(in, n, out, tsum, st);
}

cudaError_t scan_exclusive(const int* in, int64_t n, int64_t* out, int64_t* tsum, cudaStream_t st) {
    return scan_exclusive_t<int64_t>(in, n, out, tsum, st);
}

int64_t radix_chunks(int64_t n) { return (n + kRadixChunk - 1) / kRadixChunk; }

int64_t radix_hist_size(int64_t n) { return (int64_t)kRadixBins * radix_chunks(n); }

cudaError_t radix_pass(const int32_t* key_in, const int32_t* val_in, int64_t n, int shift, int* hist, int* hoff,
                       int64_t* tsum, int32_t* key_out, int32_t* val_out, cudaStream_t st) {
    const int nchunks = (int)radix_chunks(n);
    radix_hist_kernel<<<nchunks, kRadixT, 0, st>>>(key_in, n, shift, nchunks, hist);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    if ((err = scan_exclusive(hist, (int64_t)kRadixBins * nchunks, hoff, tsum, st)) != cudaSuccess) return err;
    radix_scatter_kernel<<<nchunks, kRadixT, 0, st>>>(key_in, val_in, n, shift, nchunks, hoff, key_out, val_out);
    return cudaGetLastError();
}

cudaError_t stable_sort_keys(const int32_t* key, int64_t n, int bits, int32_t* key_out, int32_t* perm,
                             cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int passes = 1;
    while (passes * kRadixBits < bits) ++passes;
    const int64_t nh = radix_hist_size(n), nt = scan_tiles(nh);
    // scratch: histogram and offsets, tile sums, and one ping-pong pair of keys and values
    const size_t bytes = (size_t)nh * 8 + (size_t)nt * 8 + (size_t)n * 8 + 256;
    char* raw = nullptr;
    cudaError_t err = cudaMallocAsync(reinterpret_cast<void**>(&raw), bytes, st);
    if (err != cudaSuccess) return err;
    int* hist = reinterpret_cast<int*>(raw);
    int* hoff = hist + nh;
    int64_t* tsum = reinterpret_cast<int64_t*>(raw + (((size_t)nh * 8 + 7) & ~(size_t)7));
    int32_t* tk = reinterpret_cast<int32_t*>(tsum + nt);
    int32_t* tv = tk + n;
    // pass p writes the final outputs when (passes - 1 - p) is even, the
    // scratch pair otherwise, so the last pass lands in key_out / perm
    const int32_t* kin = key;
    const int32_t* vin = nullptr;  // first pass: value = position
    for (int p = 0; p < passes && err == cudaSuccess; ++p) {
        const bool to_out = ((passes - 1 - p) & 1) == 0;
        int32_t* ko = to_out ? key_out : tk;
        int32_t* vo = to_out ? perm : tv;
        err = radix_pass(kin, vin, n, p * kRadixBits, hist, hoff, tsum, ko, vo, st);
        kin = ko;
        vin = vo;
    }
    cudaError_t e2 = cudaFreeAsync(raw, st);
    return err != cudaSuccess ? err : e2;
}

}  // namespace hap
