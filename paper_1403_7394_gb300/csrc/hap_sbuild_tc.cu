// Tensor-core (tcgen05) similarity build - placeholder until the kernel lands.
#include "hap_common.cuh"
#include "hap_internal.h"

namespace hap {

size_t sbuild_tc_scratch_bytes(int64_t N, int64_t d, int split) {
    const int64_t kpad = ((split ? 3 * d : d) + 63) / 64 * 64;
    const int64_t npad = (N + 127) / 128 * 128;
    return (size_t)(2 * npad * kpad * 2 + npad * 4 + 1024);
}

cudaError_t launch_sbuild_tc(const float*, int64_t, int64_t, int, void*, int, int64_t, void*, unsigned*,
                             cudaStream_t, int*) {
    return cudaErrorNotSupported;
}

}  // namespace hap
