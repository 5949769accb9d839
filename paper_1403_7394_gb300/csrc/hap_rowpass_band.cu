// The row pass over a band of rows (RowPassArgs::row0 / nrows: A, R and S
// hold rows row0 .. row0 + nrows - 1; the [L][ld] vectors keep the rows'
// indices in the problem), selected at run time by a nonzero nrows.  The
// offsets are compiled in only here, so the kernels every unbanded iteration
// runs are unchanged.
#include "hap_rowpass_kernel.cuh"

namespace hap {

cudaError_t launch_rowpass_band(const RowPassArgs& a, const LaunchShape& sh, int s_bf16, cudaStream_t st) {
    HAP_ROWPASS_DISPATCH(launch_band, a, sh, st);
}

}  // namespace hap
