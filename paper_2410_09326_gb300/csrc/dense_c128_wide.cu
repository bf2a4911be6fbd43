// Dense fused-block launches for complex128 states, 5 and 6 targets (matrix
// in device memory, staged in shared memory).
#include "kernels_common.cuh"

namespace qs {
namespace kern {

cudaError_t run_dense_c128_wide(double2 *a, int n, const Block &b, const void *dev_mat, cudaStream_t s, int threads) {
  switch (b.k) {
    case 5: return run_dense_smem<double2, 5>(a, n, b, (const double2 *)dev_mat, s, threads);
    case 6: return run_dense_smem<double2, 6>(a, n, b, (const double2 *)dev_mat, s, threads);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kern
}  // namespace qs
