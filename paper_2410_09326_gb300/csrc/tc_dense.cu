// Dense fused blocks on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// A block with K targets maps each group of 2^K amplitudes to a row of a
// real GEMM: with x_s = (re, im) interleaved, the group's 2^(K+1) reals form
// row m of A (M = 128 groups per tile, K-major), and the real embedding of
// the block matrix U,
//   B[2r][2s] = Re U_rs,  B[2r][2s+1] = -Im U_rs,
//   B[2r+1][2s] = Im U_rs, B[2r+1][2s+1] = Re U_rs,
// is B (N = 2^(K+1) rows, K-major), so D = A B^T holds the outputs in the
// same interleaved order: TMEM lane m = group m, column 2r(+1) = Re(Im) y_r.
//
// FP32 accuracy from TF32 inputs: every operand is split as hi = tf32(x),
// lo = tf32(x - hi) (round to nearest), and D = A_hi B_hi + A_hi B_lo +
// A_lo B_hi (the 3xTF32 scheme of Ootomo and Yokota, "Recovering single
// precision accuracy from Tensor Cores while surpassing the FP32 theoretical
// peak performance", 2022). The tensor core's FP32 accumulation rounds toward
// zero, which shrinks every amplitude a little on each pass; two measures
// keep that bias out of long circuits: the large A_hi B_hi term accumulates
// in its own TMEM columns (KR/8 roundings instead of 3 KR/8), the small terms
// in separate ones, the two summed in registers with round-to-nearest; and,
// since a fused block is unitary and therefore preserves the norm of each
// group exactly, every computed group is rescaled to its input norm.
//
// One CTA = 128 threads = 4 warps; thread m owns group m of the tile: it
// gathers the group's amplitudes from HBM (coalesced across the warp for
// targets above bit 4), writes its hi/lo row into shared memory in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix,
// K-adjacent core matrices 128 B apart, 8-row groups 2^(K+1)/4 * 128 B
// apart), one elected thread issues the MMAs and commits to an mbarrier, and
// warp w reads TMEM lanes 32w..32w+31 back with tcgen05.ld.
//
// Every mbarrier wait is bounded; on expiry the kernel records the failure
// in the caller's error word and leaves the tile loop, then frees its TMEM.
#include <cstdint>
#include <cstring>

#include "tc_common.cuh"

namespace qs {
namespace kern {

namespace {

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Instruction descriptor for kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9 and 10-12 = 2), both K-major, N >> 3 in bits 17-22, M >> 4 in
// bits 24-28.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

// K = targets (4 or 5). bmat: B_hi then B_lo, each N x N floats already in
// the core-matrix layout (built on the host). err: error word (0 = fine).
// Resident CTAs per SM the register budget is sized for (shared memory
// allows 4 at K = 4 and 2 at K = 5).
template <int K> struct TcOcc {
  static constexpr int value = K <= 4 ? 4 : 2;
};

template <int K, bool SPLIT, bool RENORM>
__global__ void __launch_bounds__(kTcThreads, TcOcc<K>::value)
    k_dense_tc(float2 *__restrict__ a, const float4 *__restrict__ bmat, const __grid_constant__ TcParam p,
               int *__restrict__ err) {
  constexpr int D = 1 << K;             // amplitudes per group
  constexpr int KR = 2 * D;             // real K = N of the GEMM
  constexpr uint32_t A_BYTES = 128u * KR * 4u;
  constexpr uint32_t B_BYTES = (uint32_t)KR * KR * 4u;
  constexpr uint32_t SBO_A = (KR / 4) * 128u;  // 8-row groups of A
  constexpr uint32_t SBO_B = (KR / 4) * 128u;
  constexpr uint32_t LBO = 128u;
  // SPLIT: columns [0, KR) accumulate A_hi B_hi, [KR, 2KR) the two small
  // correction products, so the tensor core's accumulation rounding of the
  // large term happens KR/8 times instead of 3 KR/8 times.
  constexpr uint32_t NCOLS = (SPLIT ? 2 * KR : KR) < 32 ? 32 : (SPLIT ? 2 * KR : KR);
  constexpr uint32_t IDESC = make_idesc(128, KR);

  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *sA_hi = smem;
  unsigned char *sA_lo = smem + A_BYTES;
  unsigned char *sB = smem + 2 * A_BYTES;  // hi then lo
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;

  // B (constant for the launch) into shared memory
  for (int i = tid; i < (int)(2 * B_BYTES / 16); i += kTcThreads)
    reinterpret_cast<float4 *>(sB)[i] = bmat[i];
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
  // this thread's row of A: 8-row group (tid / 8), row (tid % 8) of each core matrix
  const uint32_t row_off = (uint32_t)(tid >> 3) * SBO_A + (uint32_t)(tid & 7) * 16u;
  uint32_t phase = 0;
  bool aborted = false;

  // Software pipeline: the amplitudes of the next tile are loaded into
  // registers while the tensor cores work on the current one.
  long long tile = blockIdx.x;
  float2 v[D];
  uint64_t base = 0;
  bool valid = false;
  auto gather = [&](long long t, uint64_t &b, bool &ok) {
    const long long g = t * kTcThreads + tid;
    ok = t < p.n_tiles && g < p.n_groups;
    b = ok ? (insert_zeros((uint64_t)g, p.fixed, p.nf) | p.cmask) : 0;
    if (pair) {
      // bit 0 is a target: elements s and s+1 are adjacent, one 16-byte load
#pragma unroll
      for (int s = 0; s < D; s += 2) {
        uint64_t off = 0;
#pragma unroll
        for (int j = 1; j < K; j++)
          if ((s >> j) & 1) off += d[j];
        const float4 x = ok ? *reinterpret_cast<const float4 *>(a + b + off) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[s] = make_float2(x.x, x.y);
        v[s + 1] = make_float2(x.z, x.w);
      }
    } else {
#pragma unroll
      for (int s = 0; s < D; s++) {
        uint64_t off = 0;
#pragma unroll
        for (int j = 0; j < K; j++)
          if ((s >> j) & 1) off += d[j];
        v[s] = ok ? a[b + off] : make_float2(0.f, 0.f);
      }
    }
  };
  gather(tile, base, valid);

  for (; tile < p.n_tiles; tile += gridDim.x) {
    // hi/lo rows: amplitudes 2c, 2c+1 fill the 16-byte row of core matrix c
#pragma unroll
    for (int c = 0; c < D / 2; c++) {
      float4 hi, lo;
      hi.x = tf32_rn(v[2 * c].x);
      hi.y = tf32_rn(v[2 * c].y);
      hi.z = tf32_rn(v[2 * c + 1].x);
      hi.w = tf32_rn(v[2 * c + 1].y);
      lo.x = tf32_rn(v[2 * c].x - hi.x);
      lo.y = tf32_rn(v[2 * c].y - hi.y);
      lo.z = tf32_rn(v[2 * c + 1].x - hi.z);
      lo.w = tf32_rn(v[2 * c + 1].y - hi.w);
      *reinterpret_cast<float4 *>(sA_hi + row_off + c * LBO) = hi;
      *reinterpret_cast<float4 *>(sA_lo + row_off + c * LBO) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < KR / 8; ks++) {
        const uint32_t koff = (uint32_t)ks * 2u * LBO;
        const uint64_t dah = make_desc(a_hi + koff, LBO, SBO_A);
        const uint64_t dal = make_desc(a_lo + koff, LBO, SBO_A);
        const uint64_t dbh = make_desc(b_hi + koff, LBO, SBO_B);
        const uint64_t dbl = make_desc(b_lo + koff, LBO, SBO_B);
        if (SPLIT) {
          mma_tf32(tmem, dah, dbh, IDESC, ks > 0 ? 1u : 0u);
          mma_tf32(tmem + KR, dah, dbl, IDESC, ks > 0 ? 1u : 0u);
          mma_tf32(tmem + KR, dal, dbh, IDESC, 1u);
        } else {
          mma_tf32(tmem, dah, dbh, IDESC, ks > 0 ? 1u : 0u);
          mma_tf32(tmem, dah, dbl, IDESC, 1u);
          mma_tf32(tmem, dal, dbh, IDESC, 1u);
        }
      }
      if (!p.withhold_commit) mma_commit(mbar_a);
    }
    const uint64_t cur_base = base;
    const bool cur_valid = valid;
    float nin_cur = 0.f;
    if (RENORM) {
#pragma unroll
      {
        // squared norm in four independent chains
        float s4[4] = {0.f, 0.f, 0.f, 0.f};
        for (int s = 0; s < D; s++) s4[s & 3] = fmaf(v[s].x, v[s].x, fmaf(v[s].y, v[s].y, s4[s & 3]));
        nin_cur = (s4[0] + s4[1]) + (s4[2] + s4[3]);
      }
    }
    gather(tile + gridDim.x, base, valid);  // next tile, in flight during the MMAs
    const bool ok = mbar_wait(mbar_a, phase);
    phase ^= 1;
    // every thread reaches this vote (the wait is bounded), so the whole CTA
    // leaves the loop together when any wait expired
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicExch(err, 1);
      aborted = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    uint32_t r[KR];
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    TmemLd<KR>::run(lane_base, r);
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    if (SPLIT) {
#pragma unroll
      for (int h = 0; h < KR / 32; h++) {
        uint32_t t[32];
        TmemLd<32>::run(lane_base + KR + 32 * h, t);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int i = 0; i < 32; i++)
          r[32 * h + i] = __float_as_uint(__uint_as_float(r[32 * h + i]) + __uint_as_float(t[i]));
      }
    }
    if (RENORM) {
      // A unitary block preserves the norm of every group exactly; rescaling
      // the computed group to its input norm removes the shrinkage left by
      // the tensor core's round-toward-zero accumulation.
      const float nin = nin_cur;
      float o4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < KR; i++) o4[i & 3] = fmaf(__uint_as_float(r[i]), __uint_as_float(r[i]), o4[i & 3]);
      const float nout = (o4[0] + o4[1]) + (o4[2] + o4[3]);
      const float f = nout > 0.f ? sqrtf(nin / nout) : 1.f;
#pragma unroll
      for (int i = 0; i < KR; i++) r[i] = __float_as_uint(__uint_as_float(r[i]) * f);
    }
    if (cur_valid) {
      if (pair) {
#pragma unroll
        for (int s = 0; s < D; s += 2) {
          uint64_t off = 0;
#pragma unroll
          for (int j = 1; j < K; j++)
            if ((s >> j) & 1) off += d[j];
          *reinterpret_cast<float4 *>(a + cur_base + off) =
              make_float4(__uint_as_float(r[2 * s]), __uint_as_float(r[2 * s + 1]), __uint_as_float(r[2 * s + 2]),
                          __uint_as_float(r[2 * s + 3]));
        }
      } else {
#pragma unroll
        for (int s = 0; s < D; s++) {
          uint64_t off = 0;
#pragma unroll
          for (int j = 0; j < K; j++)
            if ((s >> j) & 1) off += d[j];
          a[cur_base + off] = make_float2(__uint_as_float(r[2 * s]), __uint_as_float(r[2 * s + 1]));
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
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
  }
}

// Rounds to TF32 (nearest, ties away from zero), as cvt.rna.tf32.f32 does.
float tf32_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return x;
  u += 0x1000u;
  u &= 0xFFFFE000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// B = real embedding of U, split hi/lo, in the core-matrix layout.
void build_tc_b(const Block &b, float *out) {
  const int D = 1 << b.k, KR = 2 * D;
  const size_t n = (size_t)KR * KR;
  auto at = [&](int row, int col) {
    return (size_t)(row >> 3) * (KR / 4) * 32 + (size_t)(col >> 2) * 32 + (row & 7) * 4 + (col & 3);
  };
  for (int r = 0; r < D; r++)
    for (int s = 0; s < D; s++) {
      const cd u = b.mat[(size_t)r * D + s];
      const float vals[2][2] = {{(float)u.real(), (float)-u.imag()}, {(float)u.imag(), (float)u.real()}};
      for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) {
          const float x = vals[i][j];
          const float hi = tf32_host(x);
          const float lo = tf32_host(x - hi);
          out[at(2 * r + i, 2 * s + j)] = hi;
          out[n + at(2 * r + i, 2 * s + j)] = lo;
        }
    }
}

template <int K> size_t tc_smem_bytes() {
  constexpr int KR = 2 << K;
  return 2u * 128u * KR * 4u + 2u * KR * KR * 4u;
}

template <int K, bool SPLIT, bool RENORM>
cudaError_t run_tc(float2 *a, int n, const Block &b, const void *dev_b, int *err, cudaStream_t s,
                   LaunchShape *shape) {
  TcParam p;
  p.n_groups = 1ll << (n - K - b.nctrl);
  p.n_tiles = (p.n_groups + kTcThreads - 1) / kTcThreads;
  p.cmask = b.cmask;
  p.withhold_commit = b.withhold_commit ? 1 : 0;
  fill_fixed(b, p.fixed, p.nf);
  for (int j = 0; j < K; j++) p.tq[j] = b.q[j];
  const size_t smem = tc_smem_bytes<K>();
  // per device: opt in to the shared memory, then size one wave of resident
  // CTAs (registers and shared memory decide how many; TMEM columns stay
  // within 512 per SM: at most 4 CTAs x 64 or 2 x 128)
  static thread_local int configured = -1;
  static thread_local int per_sm = 1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    cudaError_t e = cudaFuncSetAttribute(k_dense_tc<K, SPLIT, RENORM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int occ = resident_ctas((const void *)k_dense_tc<K, SPLIT, RENORM>, kTcThreads, smem);
    per_sm = occ > TcOcc<K>::value ? TcOcc<K>::value : occ;
    configured = dev;
  }
  const int grid = tc_grid((long long)dev_info().sms * per_sm, p.n_tiles, b.tc_max_ctas);
  if (shape) {
    shape->tiles = p.n_tiles;
    shape->ctas = grid;
  }
  k_dense_tc<K, SPLIT, RENORM><<<grid, kTcThreads, smem, s>>>(a, (const float4 *)dev_b, p, err);
  return cudaGetLastError();
}

}  // namespace

size_t tc_b_floats(int k) { return 2u * (size_t)(2 << k) * (size_t)(2 << k); }

void tc_build_b(const Block &b, float *out) { build_tc_b(b, out); }

cudaError_t run_dense_tc(float2 *a, int n, const Block &b, const void *dev_b, int *err, cudaStream_t s,
                         LaunchShape *shape) {
  switch (b.k) {
    case 4: return run_tc<4, true, true>(a, n, b, dev_b, err, s, shape);
    case 5: return run_tc<5, true, true>(a, n, b, dev_b, err, s, shape);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kern
}  // namespace qs
