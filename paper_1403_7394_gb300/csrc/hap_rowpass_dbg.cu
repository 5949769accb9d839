// The row pass with the debug_bounds index checks compiled in (every bulk
// copy inside the messages; the row maximum of Eq. 2.1 in a real column),
// selected at run time by RowPassArgs::debug.  Failed checks record
// ST_BOUNDS in the status word and skip the access; nothing traps.
#include "hap_rowpass_kernel.cuh"

namespace hap {

cudaError_t launch_rowpass_checked(const RowPassArgs& a, const LaunchShape& sh, int s_bf16, cudaStream_t st) {
    HAP_ROWPASS_DISPATCH(launch_checked, a, sh, st);
}

}  // namespace hap
