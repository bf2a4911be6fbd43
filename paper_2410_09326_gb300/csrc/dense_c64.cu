// Dense fused-block launches for complex64 states (FP32 accumulation),
// 1..4 targets; 5 and 6 targets are in dense_c64_wide.cu (a translation unit
// of their own, so the two compile in parallel).
#include "kernels_common.cuh"

namespace qs {
namespace kern {

cudaError_t run_dense_c64_wide(float2 *a, int n, const Block &b, const void *dev_mat, cudaStream_t s, int threads);

cudaError_t run_dense_c64(float2 *a, int n, const Block &b, const void *dev_mat, cudaStream_t s, int threads) {
  if (b.k <= 3 && b.shuffles) {
    bool used = false;
    const cudaError_t e = run_dense_shfl_c64(a, n, b, s, used);
    if (used || e != cudaSuccess) return e;
  }
  switch (b.k) {
    case 1: return run_dense_param<float2, 1>(a, n, b, s, threads);
    case 2: return run_dense_param<float2, 2>(a, n, b, s, threads);
    case 3: return run_dense_param<float2, 3>(a, n, b, s, threads);
    case 4: return run_dense_param<float2, 4>(a, n, b, s, threads);
    case 5:
    case 6: return run_dense_c64_wide(a, n, b, dev_mat, s, threads);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kern
}  // namespace qs
