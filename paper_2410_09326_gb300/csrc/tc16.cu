// Dense fused blocks on the tensor cores with FP16 operands (tcgen05
// kind::f16, FP32 accumulation), K = 4, 5, 6 targets.
//
// Same real GEMM as the TF32 kernel (tc_dense.cu): group m of a 128-group
// tile is row m of A (its 2^K amplitudes as interleaved re/im, K-major), the
// real embedding of the block matrix is B, D = A B^T lands in TMEM with lane
// m = group m. Operands are split in two FP16 halves, hi = fp16(x) and
// lo = fp16(x - hi), each with an 11-bit significand, and
// D = A_hi B_hi + A_hi B_lo + A_lo B_hi keeps ~22 bits of the product (the
// same as 3 x TF32, at twice the tensor rate and half the shared memory).
// FP16's range is narrow: every row of A is scaled by a power of two so its
// largest component lies in [0.5, 1) before the split. Matrix entries are at
// most 1 in magnitude and need no scaling. In the epilogue the large and the
// small products (kept in separate TMEM columns, because the accumulation
// rounds toward zero) are summed in registers and each group is rescaled to
// its input norm -- a fused block is unitary -- which also undoes the row
// scale exactly.
//
// This file holds the thread-per-group kernel (each thread gathers its own
// group, coalesced across the warp when the targets sit above the lowest
// free bits), the B builder and the dispatch; the lane-exchange kernels for
// low targets are in tc16x.cu.
//
// Shared memory per CTA: A hi/lo 2 x 128 x 2^(K+1) x 2 B and B hi/lo
// 2 x 4^(K+1) x 2 B: 20 KB (K=4), 48 KB (K=5), 128 KB (K=6).
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "tc16_common.cuh"

namespace qs {
namespace kern {

namespace {

// TPR threads share one row of A (one group): thread (h, r), r = tid % 128,
// h = tid / 128, gathers and converts the amplitudes s in [h D/TPR,
// (h+1) D/TPR) of group r and later reads the matching TMEM columns of lane r
// (warps w and w + 4 see the same lane quadrant). The row's scale and norms
// are combined through shared memory. Six targets take two threads per group:
// one thread would need more registers than exist (measured on GB300: 3.0-3.5
// vs 5.1-5.7 TB/s). The next tile is gathered into registers while the
// current tile's MMAs run. Resident CTAs per SM: 4 (K = 4), 3 (K = 5), 1 (K = 6).
template <int K> struct Tc16Occ {
  static constexpr int value = K <= 4 ? 4 : (K == 5 ? 3 : 1);
};
template <int K> constexpr int tc16_rows() { return K >= 6 ? 2 : 1; }

template <int K>
__global__ void __launch_bounds__(kTcThreads * tc16_rows<K>(), Tc16Occ<K>::value)
    k_dense_tc16(float2 *__restrict__ a, const uint4 *__restrict__ bmat, const __grid_constant__ TcParam p,
                 int *__restrict__ err) {
  constexpr int TPR = tc16_rows<K>();
  constexpr int NT = kTcThreads * TPR;
  constexpr int D = 1 << K;                    // amplitudes per group
  constexpr int DH = D / TPR;                  // amplitudes per thread
  constexpr int KR = 2 * D;                    // real K = N of the GEMM
  constexpr uint32_t A_BYTES = 128u * KR * 2u;
  constexpr uint32_t B_BYTES = (uint32_t)KR * KR * 2u;
  constexpr uint32_t SBO = (KR / 8) * 128u;    // 8-row groups
  constexpr uint32_t LBO = 128u;               // K-adjacent core matrices
  constexpr uint32_t NCOLS = 2 * KR;           // large and small accumulators
  constexpr uint32_t IDESC = make_idesc_f16(128, KR);
  static_assert(DH % 4 == 0, "a thread converts whole 16-byte core-matrix rows");

  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *sA_hi = smem;
  unsigned char *sA_lo = smem + A_BYTES;
  unsigned char *sB = smem + 2 * A_BYTES;  // hi then lo
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ float red_in[TPR > 1 ? 2 * NT : 1];   // (row max, row norm) partials of the inputs
  __shared__ float red_out[TPR > 1 ? NT : 1];      // row norm partials of the outputs

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int r = tid & 127;   // row of A = TMEM lane
  const int h = tid >> 7;    // which part of the row
  const int s0 = h * DH;     // first amplitude of this thread's part

  for (int i = tid; i < (int)(2 * B_BYTES / 16); i += NT) reinterpret_cast<uint4 *>(sB)[i] = bmat[i];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(NCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t mbar_a = smem_addr(&mbar);
  const uint32_t a_hi = smem_addr(sA_hi), a_lo = smem_addr(sA_lo);
  const uint32_t b_hi = smem_addr(sB), b_lo = smem_addr(sB + B_BYTES);

  uint64_t d[K];
#pragma unroll
  for (int j = 0; j < K; j++) d[j] = 1ull << p.tq[j];
  const bool pair = p.tq[0] == 0;
  // this thread's row of A: 8-row group (r / 8), row (r % 8) of each core matrix
  const uint32_t row_off = (uint32_t)(r >> 3) * SBO + (uint32_t)(r & 7) * 16u;
  uint32_t phase = 0;
  bool aborted = false;

  auto offset = [&](int s) {
    uint64_t off = 0;
#pragma unroll
    for (int j = 0; j < K; j++)
      if ((s >> j) & 1) off += d[j];
    return off;
  };

  long long tile = blockIdx.x;
  float2 v[DH];
  uint64_t base = 0;
  bool valid = false;
  auto gather = [&](long long t) {
    const long long g = t * kTcThreads + r;
    valid = t < p.n_tiles && g < p.n_groups;
    base = valid ? (insert_zeros((uint64_t)g, p.fixed, p.nf) | p.cmask) : 0;
    if (pair) {
#pragma unroll
      for (int u = 0; u < DH; u += 2) {
        const float4 x =
            valid ? *reinterpret_cast<const float4 *>(a + base + offset(s0 + u)) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[u] = make_float2(x.x, x.y);
        v[u + 1] = make_float2(x.z, x.w);
      }
    } else {
#pragma unroll
      for (int u = 0; u < DH; u++) v[u] = valid ? a[base + offset(s0 + u)] : make_float2(0.f, 0.f);
    }
  };
  gather(tile);

  for (; tile < p.n_tiles; tile += gridDim.x) {
    // row scale: largest component into [0.5, 1); max and norm in four
    // independent chains
    float m4[4] = {0.f, 0.f, 0.f, 0.f}, s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < DH; u++) {
      m4[u & 3] = fmaxf(m4[u & 3], fmaxf(fabsf(v[u].x), fabsf(v[u].y)));
      s4[u & 3] = fmaf(v[u].x, v[u].x, fmaf(v[u].y, v[u].y, s4[u & 3]));
    }
    float mx = fmaxf(fmaxf(m4[0], m4[1]), fmaxf(m4[2], m4[3]));
    float nin = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    if constexpr (TPR > 1) {
      red_in[2 * tid] = mx;
      red_in[2 * tid + 1] = nin;
      __syncthreads();
#pragma unroll
      for (int o = 1; o < TPR; o++) {
        const int pt = (tid + o * kTcThreads) % NT;
        mx = fmaxf(mx, red_in[2 * pt]);
        nin += red_in[2 * pt + 1];
      }
    }
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    const float sc = ldexpf(1.f, -e);
    // hi/lo rows: amplitudes 4c..4c+3 fill the 16-byte row of core matrix c
#pragma unroll
    for (int cl = 0; cl < DH / 4; cl++) {
      const int c = s0 / 4 + cl;
      float x[8];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        x[2 * u] = v[4 * cl + u].x * sc;
        x[2 * u + 1] = v[4 * cl + u].y * sc;
      }
      uint4 hi, lo;
      split_row(x, hi, lo);
      *reinterpret_cast<uint4 *>(sA_hi + row_off + c * LBO) = hi;
      *reinterpret_cast<uint4 *>(sA_lo + row_off + c * LBO) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < KR / 16; ks++) {
        const uint32_t koff = (uint32_t)ks * 2u * LBO;
        const uint64_t dah = make_desc(a_hi + koff, LBO, SBO);
        const uint64_t dal = make_desc(a_lo + koff, LBO, SBO);
        const uint64_t dbh = make_desc(b_hi + koff, LBO, SBO);
        const uint64_t dbl = make_desc(b_lo + koff, LBO, SBO);
        const uint32_t acc = ks > 0 ? 1u : 0u;
        mma_f16(tmem, dah, dbh, IDESC, acc);
        mma_f16(tmem + KR, dah, dbl, IDESC, acc);
        mma_f16(tmem + KR, dal, dbh, IDESC, 1u);
      }
      if (!p.withhold_commit) mma_commit(mbar_a);
    }
    const uint64_t cur_base = base;
    const bool cur_valid = valid;
    gather(tile + gridDim.x);  // next tile, in flight during the MMAs
    const bool ok = mbar_wait(mbar_a, phase);
    phase ^= 1;
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicExch(err, 1);
      aborted = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const uint32_t col0 = (uint32_t)(2 * s0);  // this thread's first column
    // pass 1: norm of the computed group (large + small products), 16
    // columns (8 amplitudes) at a time to keep registers free
    float o4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int hh = 0; hh < 2 * DH / 16; hh++) {
      uint32_t rb[16], rs[16];
      TmemLd<16>::run(lane_base + col0 + 16 * hh, rb);
      TmemLd<16>::run(lane_base + KR + col0 + 16 * hh, rs);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int i = 0; i < 16; i++) {
        const float y = __uint_as_float(rb[i]) + __uint_as_float(rs[i]);
        o4[i & 3] = fmaf(y, y, o4[i & 3]);
      }
    }
    float nout = (o4[0] + o4[1]) + (o4[2] + o4[3]);
    if constexpr (TPR > 1) {
      red_out[tid] = nout;
      __syncthreads();
#pragma unroll
      for (int o = 1; o < TPR; o++) nout += red_out[(tid + o * kTcThreads) % NT];
    }
    // unitary block: the group keeps its input norm (this also undoes the row scale)
    const float f = nout > 0.f ? sqrtf(nin / nout) : 1.f;
    // pass 2: scale and store, 8 amplitudes per chunk
#pragma unroll
    for (int hh = 0; hh < 2 * DH / 16; hh++) {
      uint32_t rb[16], rs[16];
      TmemLd<16>::run(lane_base + col0 + 16 * hh, rb);
      TmemLd<16>::run(lane_base + KR + col0 + 16 * hh, rs);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (cur_valid) {
        if (pair) {
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const int sl = s0 + 8 * hh + 2 * u;
            float y[4];
#pragma unroll
            for (int q = 0; q < 4; q++) y[q] = (__uint_as_float(rb[4 * u + q]) + __uint_as_float(rs[4 * u + q])) * f;
            *reinterpret_cast<float4 *>(a + cur_base + offset(sl)) = make_float4(y[0], y[1], y[2], y[3]);
          }
        } else {
#pragma unroll
          for (int u = 0; u < 8; u++)
            a[cur_base + offset(s0 + 8 * hh + u)] =
                make_float2((__uint_as_float(rb[2 * u]) + __uint_as_float(rs[2 * u])) * f,
                            (__uint_as_float(rb[2 * u + 1]) + __uint_as_float(rs[2 * u + 1])) * f);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (aborted) {
    // MMAs may still be in flight: make sure their completion is signalled,
    // give them a bounded chance to land, then return the columns
    if (tid == 0) mma_commit(mbar_a);
    mbar_wait(mbar_a, phase ^ 1);
  }
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
}

template <int K>
cudaError_t run_tc16(float2 *a, int n, const Block &b, const void *dev_b, int *err, cudaStream_t s,
                     LaunchShape *shape) {
  constexpr int NT = kTcThreads * tc16_rows<K>();
  TcParam p;
  p.n_groups = 1ll << (n - K - b.nctrl);
  p.n_tiles = (p.n_groups + kTcThreads - 1) / kTcThreads;
  p.cmask = b.cmask;
  p.withhold_commit = b.withhold_commit ? 1 : 0;
  fill_fixed(b, p.fixed, p.nf);
  for (int j = 0; j < K; j++) p.tq[j] = b.q[j];
  const size_t smem = tc16_smem_bytes<K>();
  // per device: opt in to the shared memory and size one wave of resident
  // CTAs; TMEM columns stay within 512 per SM (4 x 64, 3 x 128, 1 x 256)
  static thread_local int configured = -1;
  static thread_local int per_sm = 1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    cudaError_t e = cudaFuncSetAttribute(k_dense_tc16<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int occ = resident_ctas((const void *)k_dense_tc16<K>, NT, smem);
    const int tmem_cap = 512 / (4 << K);
    per_sm = occ > Tc16Occ<K>::value ? Tc16Occ<K>::value : occ;
    if (per_sm > tmem_cap) per_sm = tmem_cap;
    configured = dev;
  }
  const int grid = tc_grid((long long)dev_info().sms * per_sm, p.n_tiles, b.tc_max_ctas);
  if (shape) {
    shape->tiles = p.n_tiles;
    shape->ctas = grid;
  }
  k_dense_tc16<K><<<grid, NT, smem, s>>>(a, (const uint4 *)dev_b, p, err);
  return cudaGetLastError();
}

}  // namespace

size_t tc16_b_bytes(int k) { return 2u * (size_t)(2 << k) * (size_t)(2 << k) * 2u; }

// B = real embedding of U, split into FP16 hi/lo, in the 16-bit core-matrix
// layout (row r, column c at (r/8) * (KR/8) * 64 + (c/8) * 64 + (r%8) * 8 + c%8 halves).
void tc16_build_b(const Block &b, void *out) {
  const int D = 1 << b.k, KR = 2 * D;
  const size_t n = (size_t)KR * KR;
  __half *h = (__half *)out;
  // lane-exchange blocks take the matrix with rows and columns in slot
  // order: entry (rho, sigma) = U(pi(rho), pi(sigma)), pi(rho) = sum over the
  // slot bits set of 1 << (their target's position). The layout depends on the
  // targets and controls only (the planner checked that n admits it), so any
  // n above the fixed bits gives the same slots.
  std::vector<cd> slot_mat;
  const std::vector<cd> *m = &b.mat;
  TcXLayout x;
  if (b.tc_xg && tc_exchange_layout(64, b, x)) {
    auto pi = [&](int rho) {
      int s = 0;
      for (int j = 0; j < b.k; j++)
        if ((rho >> j) & 1) s |= 1 << x.slot_mat[j];
      return s;
    };
    slot_mat.resize((size_t)D * D);
    for (int r = 0; r < D; r++)
      for (int c = 0; c < D; c++) slot_mat[(size_t)r * D + c] = b.mat[(size_t)pi(r) * D + pi(c)];
    m = &slot_mat;
  }
  auto at = [&](int row, int col) {
    return (size_t)(row >> 3) * (KR / 8) * 64 + (size_t)(col >> 3) * 64 + (row & 7) * 8 + (col & 7);
  };
  for (int r = 0; r < D; r++)
    for (int s = 0; s < D; s++) {
      const cd u = (*m)[(size_t)r * D + s];
      const float vals[2][2] = {{(float)u.real(), (float)-u.imag()}, {(float)u.imag(), (float)u.real()}};
      for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) {
          const float x = vals[i][j];
          const __half hi = __float2half_rn(x);
          const __half lo = __float2half_rn(x - __half2float(hi));
          h[at(2 * r + i, 2 * s + j)] = hi;
          h[n + at(2 * r + i, 2 * s + j)] = lo;
        }
    }
}

cudaError_t run_dense_tc16(float2 *a, int n, const Block &b, const void *dev_b, int *err, cudaStream_t s,
                           LaunchShape *shape) {
  if (b.tc_xg) return run_dense_tc16x(a, n, b, dev_b, err, s, shape);  // B in slot order: only they take it
  switch (b.k) {
    case 4: return run_tc16<4>(a, n, b, dev_b, err, s, shape);
    case 5: return run_tc16<5>(a, n, b, dev_b, err, s, shape);
    case 6: return run_tc16<6>(a, n, b, dev_b, err, s, shape);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kern
}  // namespace qs
