// Dense fused-block launches for complex64 states, 5 and 6 targets.
#include "kernels_common.cuh"

namespace qs {
namespace kern {

cudaError_t run_dense_c64_wide(float2 *a, int n, const Block &b, const void *dev_mat, cudaStream_t s, int threads) {
  switch (b.k) {
    case 5: return run_dense_param<float2, 5>(a, n, b, s, threads);
    case 6: return run_dense_smem<float2, 6>(a, n, b, (const float2 *)dev_mat, s, threads);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kern
}  // namespace qs
