// Dense fused-block launches for complex128 states (FP64 accumulation),
// 1..4 targets; 5 and 6 targets are in dense_c128_wide.cu.
#include "kernels_common.cuh"

namespace qs {
namespace kern {

cudaError_t run_dense_c128_wide(double2 *a, int n, const Block &b, const void *dev_mat, cudaStream_t s, int threads);

cudaError_t run_dense_c128(double2 *a, int n, const Block &b, const void *dev_mat, cudaStream_t s, int threads) {
  switch (b.k) {
    case 1: return run_dense_param<double2, 1>(a, n, b, s, threads);
    case 2: return run_dense_param<double2, 2>(a, n, b, s, threads);
    case 3: return run_dense_param<double2, 3>(a, n, b, s, threads);
    case 4: return run_dense_param<double2, 4>(a, n, b, s, threads);
    case 5:
    case 6: return run_dense_c128_wide(a, n, b, dev_mat, s, threads);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kern
}  // namespace qs
