// Dense fused-block launches for complex128 states (FP64 accumulation).
#include "kernels_common.cuh"

namespace qs {
namespace kern {

cudaError_t run_dense_c128(double2 *a, int n, const Block &b, const void *dev_mat, cudaStream_t s, int threads) {
  switch (b.k) {
    case 1: return run_dense_param<double2, 1>(a, n, b, s, threads);
    case 2: return run_dense_param<double2, 2>(a, n, b, s, threads);
    case 3: return run_dense_param<double2, 3>(a, n, b, s, threads);
    case 4: return run_dense_param<double2, 4>(a, n, b, s, threads);
    case 5: return run_dense_smem<double2, 5>(a, n, b, (const double2 *)dev_mat, s, threads);
    case 6: return run_dense_smem<double2, 6>(a, n, b, (const double2 *)dev_mat, s, threads);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kern
}  // namespace qs
