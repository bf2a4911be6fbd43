// Pieces shared by the FP16 tensor-core kernels (tc16.cu: thread-per-group
// gathers; tc16x.cu: lane-exchange gathers): the kind::f16 instruction
// descriptor and MMA, the FP16 hi/lo row split, 16-byte cp.async, and the
// shared-memory size of the operands.
#pragma once
#include <cstdint>

#include <cuda_fp16.h>

#include "tc_common.cuh"

namespace qs {
namespace kern {

// kind::f16 instruction descriptor: D = F32 (bits 4-5 = 1), A = B = F16
// (format 0 in bits 7-9 and 10-12), both K-major, N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t make_idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

// The same MMA with the A operand in tensor memory (tmem_a: lane m = row m,
// K packed two FP16 values per 32-bit column, 8 columns per K step of 16).
__device__ __forceinline__ void mma_f16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ uint32_t pack_half2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// One 16-byte core-matrix row of A from four scaled complex amplitudes
// (re, im interleaved): hi = fp16(x), lo = fp16(x - hi).
__device__ __forceinline__ void split_row(const float (&x)[8], uint4 &hi, uint4 &lo) {
  uint32_t *hp = reinterpret_cast<uint32_t *>(&hi), *lp = reinterpret_cast<uint32_t *>(&lo);
#pragma unroll
  for (int u = 0; u < 4; u++) {
    const __half2 hh = __floats2half2_rn(x[2 * u], x[2 * u + 1]);
    const float2 hf = __half22float2(hh);
    hp[u] = *reinterpret_cast<const uint32_t *>(&hh);
    lp[u] = pack_half2(x[2 * u] - hf.x, x[2 * u + 1] - hf.y);
  }
}

// A (hi, lo) for 128 rows and B (hi, lo), K = 4..6 targets.
template <int K> size_t tc16_smem_bytes() {
  constexpr size_t KR = 2 << K;
  return 2 * 128 * KR * 2 + 2 * KR * KR * 2;
}

// The lane-exchange kernels (tc16x.cu) for a block the planner marked for
// them (b.tc_xg); B must have been built in slot order (tc16_build_b does).
cudaError_t run_dense_tc16x(float2 *a, int n, const Block &b, const void *dev_b, int *err, cudaStream_t s,
                            LaunchShape *shape);

}  // namespace kern
}  // namespace qs
