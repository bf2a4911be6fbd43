// Device helpers and the dense fused-block kernels (included by the dense
// translation units, one per amplitude type, so they compile in parallel).
#pragma once
#include <cstdint>

#include "qs_internal.h"

namespace qs {
namespace kern {

__device__ __forceinline__ uint64_t insert_zeros(uint64_t j, const int *fixed, int nf) {
  for (int i = 0; i < nf; i++) {
    const int p = fixed[i];
    j = ((j >> p) << (p + 1)) | (j & ((1ull << p) - 1));
  }
  return j;
}

template <typename T> struct Real;
template <> struct Real<float2> { using type = float; };
template <> struct Real<double2> { using type = double; };

template <typename T, int K> struct DenseParam {
  T m[1 << (2 * K)];          // row-major (2^K)^2
  long long n_groups;         // 2^(n - K - controls)
  unsigned long long cmask;   // control bits, all set
  int nf;                     // number of fixed bits (targets + controls)
  int fixed[kMaxFixed];       // ascending
  int tq[K];                  // targets ascending
};

struct DenseIdx {
  long long n_groups;
  unsigned long long cmask;
  int nf;
  int fixed[kMaxFixed];
  int tq[QS_MAX_FUSE];
};

template <typename T, int K, bool PAIR = false>
__device__ __forceinline__ void group_apply(T *__restrict__ a, uint64_t base, const uint64_t *d,
                                            const T *m) {
  using R = typename Real<T>::type;
  constexpr int D = 1 << K;
  T v[D];
  if constexpr (PAIR) {
    // bit 0 is a target (complex64): elements s and s+1 share one 16-byte access
#pragma unroll
    for (int s = 0; s < D; s += 2) {
      uint64_t off = 0;
#pragma unroll
      for (int j = 1; j < K; j++)
        if ((s >> j) & 1) off += d[j];
      const float4 x = *reinterpret_cast<const float4 *>(a + base + off);
      v[s].x = x.x;
      v[s].y = x.y;
      v[s + 1].x = x.z;
      v[s + 1].y = x.w;
    }
  } else {
#pragma unroll
    for (int s = 0; s < D; s++) {
      uint64_t off = 0;
#pragma unroll
      for (int j = 0; j < K; j++)
        if ((s >> j) & 1) off += d[j];
      v[s] = a[base + off];
    }
  }
  // The store addresses are recomputed from an opaque copy of the base
  // instead of keeping 2^K 64-bit load addresses live across the mat-vec.
  uint64_t base2 = base;
  asm volatile("" : "+l"(base2));
  T y[2];
#pragma unroll
  for (int r = 0; r < D; r++) {
    R re = 0, im = 0;
#pragma unroll
    for (int c = 0; c < D; c++) {
      const T w = m[r * D + c];
      re = fma(w.x, v[c].x, re);
      re = fma(-w.y, v[c].y, re);
      im = fma(w.x, v[c].y, im);
      im = fma(w.y, v[c].x, im);
    }
    y[r & 1].x = re;
    y[r & 1].y = im;
    if constexpr (PAIR) {
      if (r & 1) {
        uint64_t off = 0;
#pragma unroll
        for (int j = 1; j < K; j++)
          if ((r >> j) & 1) off += d[j];
        *reinterpret_cast<float4 *>(a + base2 + off) = make_float4(y[0].x, y[0].y, y[1].x, y[1].y);
      }
    } else {
      uint64_t off = 0;
#pragma unroll
      for (int j = 0; j < K; j++)
        if ((r >> j) & 1) off += d[j];
      a[base2 + off] = y[r & 1];
    }
  }
}

// Minimum resident CTAs of 256 threads per SM: caps registers so that enough
// loads stay in flight for HBM (64 regs at 4, 128 at 2, 255 at 1); each
// thread keeps 2^K independent loads in flight, so 1-2 CTAs suffice.
template <typename T, int K> struct DenseOcc {
  static constexpr int value = sizeof(T) == 8 ? (K <= 3 ? 4 : (K == 4 ? 2 : 1))
                                              : (K <= 2 ? 4 : (K == 3 ? 2 : 1));
};

template <typename T, int K>
__global__ void __launch_bounds__(256, DenseOcc<T, K>::value) k_dense_param(T *__restrict__ a,
                                                     const __grid_constant__ DenseParam<T, K> p) {
  uint64_t d[K];
#pragma unroll
  for (int j = 0; j < K; j++) d[j] = 1ull << p.tq[j];
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (sizeof(T) == 8 && K >= 1 && p.tq[0] == 0) {
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < p.n_groups; g += stride) {
      const uint64_t base = insert_zeros((uint64_t)g, p.fixed, p.nf) | p.cmask;
      group_apply<T, K, sizeof(T) == 8>(a, base, d, p.m);
    }
    return;
  }
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < p.n_groups; g += stride) {
    const uint64_t base = insert_zeros((uint64_t)g, p.fixed, p.nf) | p.cmask;
    group_apply<T, K>(a, base, d, p.m);
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(256, DenseOcc<T, K>::value) k_dense_smem(T *__restrict__ a, const T *__restrict__ mat,
                                                    const __grid_constant__ DenseIdx p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *m = reinterpret_cast<T *>(smem_raw);
  constexpr int D = 1 << K;
  for (int i = threadIdx.x; i < D * D; i += blockDim.x) m[i] = mat[i];
  __syncthreads();
  uint64_t d[K];
#pragma unroll
  for (int j = 0; j < K; j++) d[j] = 1ull << p.tq[j];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < p.n_groups; g += stride) {
    const uint64_t base = insert_zeros((uint64_t)g, p.fixed, p.nf) | p.cmask;
    group_apply<T, K>(a, base, d, m);
  }
}


int grid_for(long long work, int threads);
// CTAs of `func` that fit on one SM (registers, shared memory, threads).
int resident_ctas(const void *func, int threads, size_t dyn_smem);

inline void fill_fixed(const Block &b, int *fixed, int &nf) {
  uint64_t m = b.cmask;
  if (b.kind == BK_DENSE)
    for (int j = 0; j < b.k; j++) m |= 1ull << b.q[j];
  nf = 0;
  for (int q = 0; q < 64; q++)
    if ((m >> q) & 1) fixed[nf++] = q;
}

template <typename T> T to_dev(cd z) {
  T t;
  t.x = (typename Real<T>::type)z.real();
  t.y = (typename Real<T>::type)z.imag();
  return t;
}

template <typename T, int K>
cudaError_t run_dense_param(T *a, int n, const Block &b, cudaStream_t s, int threads) {
  static thread_local DenseParam<T, K> p;  // large: kept off the stack; the launch copies it
  constexpr int D = 1 << K;
  for (int i = 0; i < D * D; i++) p.m[i] = to_dev<T>(b.mat[i]);
  p.n_groups = 1ll << (n - K - b.nctrl);
  p.cmask = b.cmask;
  fill_fixed(b, p.fixed, p.nf);
  for (int j = 0; j < K; j++) p.tq[j] = b.q[j];
  k_dense_param<T, K><<<grid_for(p.n_groups, threads), threads, 0, s>>>(a, p);
  return cudaGetLastError();
}

template <typename T, int K>
cudaError_t run_dense_smem(T *a, int n, const Block &b, const T *dev_mat, cudaStream_t s, int threads) {
  DenseIdx p;
  p.n_groups = 1ll << (n - K - b.nctrl);
  p.cmask = b.cmask;
  fill_fixed(b, p.fixed, p.nf);
  for (int j = 0; j < K; j++) p.tq[j] = b.q[j];
  const size_t smem = sizeof(T) << (2 * K);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_dense_smem<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_dense_smem<T, K><<<grid_for(p.n_groups, threads), threads, smem, s>>>(a, dev_mat, p);
  return cudaGetLastError();
}

// Tensor-core path (tc_dense.cu): dense blocks with 4 or 5 targets, c64.
// dev_b holds tc_b_floats(k) floats written by tc_build_b; err is a device
// error word set to 1 when a bounded wait expires.
size_t tc_b_floats(int k);
void tc_build_b(const Block &b, float *out);
cudaError_t run_dense_tc(float2 *a, int n, const Block &b, const void *dev_b, int *err, cudaStream_t s,
                         LaunchShape *shape);
// FP16-operand variant (tc16.cu), k = 4..6: dev_b holds tc16_b_bytes(k) bytes
// written by tc16_build_b.
size_t tc16_b_bytes(int k);
void tc16_build_b(const Block &b, void *out);
cudaError_t run_dense_tc16(float2 *a, int n, const Block &b, const void *dev_b, int *err, cudaStream_t s,
                           LaunchShape *shape);

// Cache-blocked passes (tile.cu): a BK_TILE block's descriptor (header,
// member matrices and tables, member descriptors) lives in device memory.
size_t tile_desc_bytes(const Block &b, bool c128);
size_t tile_smem_bytes(const Block &b, bool c128);
void tile_fill_desc(const Block &b, bool c128, void *out);
cudaError_t run_tile(void *a, int n, bool c128, const Block &b, const void *dev_desc, cudaStream_t s);

// Phase-polynomial diagonal blocks (phase.cu), n > 10: factor table and
// chunk terms in device memory.
size_t phase_desc_bytes(const Block &b, bool c128);
void phase_fill_desc(const Block &b, bool c128, void *out);
cudaError_t run_phase(void *a, int n, bool c128, const Block &b, const void *dev_desc, cudaStream_t s,
                      LaunchShape *shape);

// Warp-shuffle variant for 1..3 targets with one among bits 1..5 (dense_shfl.cu);
// used = false when the block does not qualify (nothing launched).
cudaError_t run_dense_shfl_c64(float2 *a, int n, const Block &b, cudaStream_t s, bool &used);

cudaError_t run_dense_c64(float2 *a, int n, const Block &b, const void *dev_mat, cudaStream_t s, int threads);
cudaError_t run_dense_c128(double2 *a, int n, const Block &b, const void *dev_mat, cudaStream_t s, int threads);

}  // namespace kern
}  // namespace qs
