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
// Shared memory per CTA: A hi/lo 2 x 128 x 2^(K+1) x 2 B and B hi/lo
// 2 x 4^(K+1) x 2 B: 20 KB (K=4), 48 KB (K=5), 128 KB (K=6).
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#include <cuda_fp16.h>

#include "tc16_common.cuh"

namespace qs {
namespace kern {

namespace {

// Resident CTAs per SM the register budget is sized for (TPR threads per row).
// PFD = tiles gathered ahead into registers (0, 1 or 2). Without the
// prefetch a thread needs fewer registers, so more CTAs fit and they hide
// each other's gathers; two tiles ahead keep loads in flight across a whole
// tile at the price of registers.
template <int K, int TPR, int PFD = 1, bool SK = false> struct Tc16Occ {
  static constexpr int value =
      SK ? 2 : PFD == 3 ? (K <= 4 ? 4 : 2) : TPR == 4 ? 1
               : (PFD == 1 ? (K <= 4 ? 4 : (K == 5 ? 3 : 1))
                           : (PFD == 0 ? (K <= 4 ? 6 : (K == 5 ? 4 : 1)) : (K <= 4 ? 3 : (K == 5 ? 2 : 1))));
};

// TPR threads share one row of A (one group): thread (h, r), r = tid % 128,
// h = tid / 128, gathers and converts the amplitudes s in [h D/TPR,
// (h+1) D/TPR) of group r and later reads the matching TMEM columns of lane r
// (warps w and w + 4 see the same lane quadrant). The row's scale and norms
// are combined through shared memory. More threads per row means fewer
// registers per thread and more warps per SM to hide the gather latency.
// SK (split K, with TPR = 2): the A buffers hold one half of the K columns at
// a time -- thread half h is exactly K half h -- so the MMAs run in two
// rounds (half 0, wait, half 1) and the shared memory of 6-target blocks
// drops from 128 KB to 96 KB: two CTAs fit per SM.
// PFD = 3 (one thread per group, 4 or 5 targets; opt-in): each thread copies
// its group's amplitudes with cp.async two tiles ahead into one of two
// shared-memory staging areas ([amplitude][thread], 8-byte elements, or
// 16-byte pairs when bit 0 is a target) and reads them back at the top of the
// tile: no registers hold tiles in flight. Measured on GB300 the 8-byte
// copies cost more than they hide (4.6-5.9 vs 5.6-6.3 TB/s), except for
// 16-byte pairs at 5 targets; the exchange kernel's 16-byte staging is the
// default instead.
template <int K, int TPR, int PFD, bool SK = false>
__global__ void __launch_bounds__(kTcThreads * TPR, Tc16Occ<K, TPR, PFD, SK>::value)
    k_dense_tc16(float2 *__restrict__ a, const uint4 *__restrict__ bmat, const __grid_constant__ TcParam p,
                 int *__restrict__ err) {
  constexpr int NT = kTcThreads * TPR;
  constexpr int D = 1 << K;                    // amplitudes per group
  constexpr int DH = D / TPR;                  // amplitudes per thread
  constexpr int KR = 2 * D;                    // real K = N of the GEMM
  constexpr int KA = SK ? KR / 2 : KR;         // K columns held in the A buffers
  constexpr uint32_t A_BYTES = 128u * KA * 2u;
  constexpr uint32_t B_BYTES = (uint32_t)KR * KR * 2u;
  constexpr uint32_t SBO = (KR / 8) * 128u;    // 8-row groups of B
  constexpr uint32_t SBO_A = (KA / 8) * 128u;  // 8-row groups of A
  constexpr uint32_t LBO = 128u;               // K-adjacent core matrices
  constexpr uint32_t NCOLS = 2 * KR;           // large and small accumulators
  constexpr uint32_t IDESC = make_idesc_f16(128, KR);
  static_assert(DH % 4 == 0, "a thread converts whole 16-byte core-matrix rows");
  static_assert(!SK || TPR == 2, "split K pairs each thread half with a K half");

  static_assert(PFD != 3 || (TPR == 1 && !SK), "staged copies: one thread per group");
  constexpr uint32_t STAGE_BYTES = (uint32_t)DH * kTcThreads * 8u;

  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *sA_hi = smem;
  unsigned char *sA_lo = smem + A_BYTES;
  unsigned char *sB = smem + 2 * A_BYTES;  // hi then lo
  unsigned char *sStage = sB + 2 * B_BYTES;  // PFD = 3: two staging areas
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
  const uint32_t row_off = (uint32_t)(r >> 3) * SBO_A + (uint32_t)(r & 7) * 16u;
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
  float2 v[DH], v2[PFD == 2 ? DH : 1];
  uint64_t base = 0, base2 = 0;
  bool valid = false, valid2 = false;
  auto gather = [&](long long t, uint64_t &b, bool &ok, float2 *v) {
    const long long g = t * kTcThreads + r;
    ok = t < p.n_tiles && g < p.n_groups;
    b = ok ? (insert_zeros((uint64_t)g, p.fixed, p.nf) | p.cmask) : 0;
    if (pair) {
#pragma unroll
      for (int u = 0; u < DH; u += 2) {
        const float4 x = ok ? *reinterpret_cast<const float4 *>(a + b + offset(s0 + u)) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[u] = make_float2(x.x, x.y);
        v[u + 1] = make_float2(x.z, x.w);
      }
    } else {
#pragma unroll
      for (int u = 0; u < DH; u++) v[u] = ok ? a[b + offset(s0 + u)] : make_float2(0.f, 0.f);
    }
  };
  // PFD = 3: tile t into staging area u, one commit group per tile
  uint64_t sbase0 = 0, sbase1 = 0;
  bool svalid0 = false, svalid1 = false;
  auto stage_in = [&](long long t, int u) {
    const long long g = t * kTcThreads + r;
    const bool ok = t < p.n_tiles && g < p.n_groups;
    const uint64_t b = ok ? (insert_zeros((uint64_t)g, p.fixed, p.nf) | p.cmask) : 0;
    if (u) {
      sbase1 = b;
      svalid1 = ok;
    } else {
      sbase0 = b;
      svalid0 = ok;
    }
    if (ok) {
      const uint32_t dst = smem_addr(sStage) + (uint32_t)u * STAGE_BYTES;
      if (pair) {
#pragma unroll
        for (int w = 0; w < DH / 2; w++)
          cp_async16(dst + ((uint32_t)w * kTcThreads + (uint32_t)tid) * 16u, a + b + offset(2 * w));
      } else {
#pragma unroll
        for (int w = 0; w < DH; w++)
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst + ((uint32_t)w * kTcThreads +
                                                                                  (uint32_t)tid) * 8u),
                       "l"(a + b + offset(w))
                       : "memory");
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (PFD == 3) {
    stage_in(tile, 0);
    stage_in(tile + gridDim.x, 1);
  }
  if (PFD == 1 || PFD == 2) gather(tile, base, valid, v);
  if (PFD == 2) gather(tile + gridDim.x, base2, valid2, v2);

  for (int it = 0; tile < p.n_tiles; tile += gridDim.x, it++) {
    if (PFD == 0) gather(tile, base, valid, v);
    if constexpr (PFD == 3) {
      // this tile's group has landed once at most the next one is pending
      asm volatile("cp.async.wait_group 1;" ::: "memory");
      const int u = it & 1;
      const unsigned char *src = sStage + (uint32_t)u * STAGE_BYTES;
      base = u ? sbase1 : sbase0;
      valid = u ? svalid1 : svalid0;
      if (pair) {
#pragma unroll
        for (int w = 0; w < DH / 2; w++) {
          const float4 x = valid ? *reinterpret_cast<const float4 *>(src + ((uint32_t)w * kTcThreads + tid) * 16u)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
          v[2 * w] = make_float2(x.x, x.y);
          v[2 * w + 1] = make_float2(x.z, x.w);
        }
      } else {
#pragma unroll
        for (int w = 0; w < DH; w++)
          v[w] = valid ? *reinterpret_cast<const float2 *>(src + ((uint32_t)w * kTcThreads + tid) * 8u)
                       : make_float2(0.f, 0.f);
      }
    }
    // row scale: largest component into [0.5, 1)
    float mx = 0.f, nin = 0.f;
#pragma unroll
    for (int u = 0; u < DH; u++) {
      mx = fmaxf(mx, fmaxf(fabsf(v[u].x), fabsf(v[u].y)));
      nin = fmaf(v[u].x, v[u].x, fmaf(v[u].y, v[u].y, nin));
    }
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
    auto convert = [&]() {
#pragma unroll
    for (int cl = 0; cl < DH / 4; cl++) {
      const int c = SK ? cl : s0 / 4 + cl;
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
    };
    // MMAs over K steps [k0, k0 + nks) of 16 columns; A holds them from step 0
    auto issue = [&](int k0, int nks) {
      if (tid == 0) {
#pragma unroll
        for (int ks = 0; ks < KA / 16; ks++) {
          if (ks >= nks) break;
          const uint32_t aoff = (uint32_t)ks * 2u * LBO;
          const uint32_t boff = (uint32_t)(k0 + ks) * 2u * LBO;
          const uint64_t dah = make_desc(a_hi + aoff, LBO, SBO_A);
          const uint64_t dal = make_desc(a_lo + aoff, LBO, SBO_A);
          const uint64_t dbh = make_desc(b_hi + boff, LBO, SBO);
          const uint64_t dbl = make_desc(b_lo + boff, LBO, SBO);
          const uint32_t acc = (k0 + ks) > 0 ? 1u : 0u;
          mma_f16(tmem, dah, dbh, IDESC, acc);
          mma_f16(tmem + KR, dah, dbl, IDESC, acc);
          mma_f16(tmem + KR, dal, dbh, IDESC, 1u);
        }
        if (!p.withhold_commit) mma_commit(mbar_a);
      }
    };
    auto publish = [&]() {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
    };
    if constexpr (SK) {
      // K half 0 from thread half 0; its MMAs must finish reading A before
      // thread half 1 overwrites it with K half 1
      if (h == 0) convert();
      publish();
      issue(0, KR / 32);
      const bool ok0 = mbar_wait(mbar_a, phase);
      phase ^= 1;
      if (!__syncthreads_and(ok0)) {
        if (tid == 0) atomicExch(err, 1);
        aborted = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (h == 1) convert();
      publish();
      issue(KR / 32, KR / 32);
    } else {
      convert();
      publish();
      issue(0, KR / 16);
    }
    const uint64_t cur_base = base;
    const bool cur_valid = valid;
    if (PFD == 3) stage_in(tile + 2 * (long long)gridDim.x, it & 1);  // the area just read
    if (PFD == 1) gather(tile + gridDim.x, base, valid, v);  // next tile, in flight during the MMAs
    if (PFD == 2) {
      // the tile after next goes in flight; the next one (loaded during the
      // previous tile) moves into place
#pragma unroll
      for (int u = 0; u < DH; u++) v[u] = v2[u];
      base = base2;
      valid = valid2;
      gather(tile + 2 * (long long)gridDim.x, base2, valid2, v2);
    }
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
    float nout = 0.f;
#pragma unroll
    for (int hh = 0; hh < 2 * DH / 16; hh++) {
      uint32_t rb[16], rs[16];
      TmemLd<16>::run(lane_base + col0 + 16 * hh, rb);
      TmemLd<16>::run(lane_base + KR + col0 + 16 * hh, rs);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int i = 0; i < 16; i++) {
        const float y = __uint_as_float(rb[i]) + __uint_as_float(rs[i]);
        nout = fmaf(y, y, nout);
      }
    }
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
  if constexpr (PFD == 3) asm volatile("cp.async.wait_all;" ::: "memory");  // copies still in flight
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

// Staged variant (K = 4, 5; bit 0 not a control): a tile of 128 groups is
// the sub-cube of the index space spanned by the 7 lowest free bits and the
// K targets (the other bits fixed per tile). Bits 0..6 always lie in it, so
// in address order the tile is made of contiguous runs of at least 1 KiB,
// whatever the targets: the CTA copies it into shared memory with 16-byte
// cp.async in address order, two tiles ahead (two staging buffers, so two
// tiles' loads are in flight per CTA without holding registers), each thread
// then reads its group's row from a layout in which consecutive rows are
// consecutive words, and stores its results directly. Element e of the tile (its
// local index, bit j = j-th lowest bit of the sub-cube) sits at global offset
// dep_lo[e & 63] + dep_hi[e >> 6] from the tile base and at staging slot
// slot_lo[e & 63] + slot_hi[e >> 6], slot(r, s) = 128 s + r, or
// 256 (s >> 1) + 2 r + (s & 1) when bit 0 is a target (pairs stay adjacent).
struct TcStageParam {
  long long n_tiles;
  unsigned long long cmask;
  int nhi;                        // free bits above the 7 lowest: the tile index
  int hi_pos[40];
  int pair;                       // bit 0 is target 0
  int withhold_commit;
  int low7[7];                    // the 7 lowest free bits (row r's bits, in order)
  int tq[QS_MAX_FUSE];            // targets ascending (matrix bit order)
  unsigned long long dep_lo[64], dep_hi[64];
  unsigned short slot_lo[64], slot_hi[64];
};


template <int K>
__global__ void __launch_bounds__(kTcThreads, 2)
    k_dense_tc16s(float2 *__restrict__ a, const uint4 *__restrict__ bmat, const __grid_constant__ TcStageParam p,
                  int *__restrict__ err) {
  constexpr int D = 1 << K;
  constexpr int KR = 2 * D;
  constexpr int ELEMS = 128 * D;                 // amplitudes per tile
  constexpr int LB = 7 + K;                      // local index bits
  constexpr uint32_t A_BYTES = 128u * KR * 2u;
  constexpr uint32_t B_BYTES = (uint32_t)KR * KR * 2u;
  constexpr uint32_t SBO = (KR / 8) * 128u;
  constexpr uint32_t LBO = 128u;
  constexpr uint32_t NCOLS = 2 * KR;
  constexpr uint32_t IDESC = make_idesc_f16(128, KR);
  constexpr uint32_t IN_BYTES = (uint32_t)ELEMS * 8u;

  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *sA_hi = smem;
  unsigned char *sA_lo = smem + A_BYTES;
  unsigned char *sB = smem + 2 * A_BYTES;                     // hi then lo
  float2 *sIn0 = reinterpret_cast<float2 *>(smem + 2 * A_BYTES + 2 * B_BYTES);  // two staging buffers
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  for (int i = tid; i < (int)(2 * B_BYTES / 16); i += kTcThreads) reinterpret_cast<uint4 *>(sB)[i] = bmat[i];
  // the copies of thread tid are the elements e = 2 tid + 256 j: their low
  // 6 bits are the thread's own, their high bits (tid / 32 + 4 j) are the
  // same across a warp, so the high tables are read from the parameter bank
  // as broadcasts and shared memory stays free for the two staging buffers
  const unsigned long long my_dep = p.dep_lo[(2 * tid) & 63];
  const uint32_t my_slot = p.slot_lo[(2 * tid) & 63];
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
  const uint32_t in_addr0 = smem_addr(sIn0);
  const int r = tid;
  const uint32_t row_off = (uint32_t)(r >> 3) * SBO + (uint32_t)(r & 7) * 16u;
  const bool pair = p.pair != 0;

  auto tile_base = [&](long long t) {
    uint64_t b = p.cmask;
    for (int j = 0; j < p.nhi; j++) b |= (uint64_t)((t >> j) & 1) << p.hi_pos[j];
    return b;
  };
  // one commit group per tile slot, empty past the last tile, so that
  // "all but the newest group" always means "the tile about to be used"
  auto issue_loads = [&](long long t, int buf) {
    if (t < p.n_tiles) {
      const uint64_t tb = tile_base(t);
      const uint32_t dst = in_addr0 + (uint32_t)buf * IN_BYTES;
#pragma unroll 4
      for (int e = 2 * tid; e < ELEMS; e += 2 * kTcThreads) {
        const uint64_t off = tb + my_dep + p.dep_hi[e >> 6];
        const uint32_t slot = my_slot + p.slot_hi[e >> 6];
        cp_async16(dst + slot * 8u, a + off);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // this thread's group base within a tile, and target offsets
  uint64_t rbase = 0;
#pragma unroll
  for (int j = 0; j < 7; j++) rbase |= (uint64_t)((r >> j) & 1) << p.low7[j];
  uint64_t d[K];
#pragma unroll
  for (int j = 0; j < K; j++) d[j] = 1ull << p.tq[j];
  auto offset = [&](int s) {
    uint64_t off = 0;
#pragma unroll
    for (int j = 0; j < K; j++)
      if ((s >> j) & 1) off += d[j];
    return off;
  };

  uint32_t phase = 0;
  bool aborted = false;
  long long tile = blockIdx.x;
  issue_loads(tile, 0);
  issue_loads(tile + gridDim.x, 1);
  int buf = 0;
  for (; tile < p.n_tiles; tile += gridDim.x, buf ^= 1) {
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();
    const float2 *sIn = sIn0 + (size_t)buf * ELEMS;
    // this thread's group (row r) out of the staged tile
    float2 v[D];
    if (pair) {
#pragma unroll
      for (int s = 0; s < D; s += 2) {
        const float4 x = *reinterpret_cast<const float4 *>(sIn + (s >> 1) * 256 + 2 * r);
        v[s] = make_float2(x.x, x.y);
        v[s + 1] = make_float2(x.z, x.w);
      }
    } else {
#pragma unroll
      for (int s = 0; s < D; s++) v[s] = sIn[s * 128 + r];
    }
    float mx = 0.f, nin = 0.f;
#pragma unroll
    for (int s = 0; s < D; s++) {
      mx = fmaxf(mx, fmaxf(fabsf(v[s].x), fabsf(v[s].y)));
      nin = fmaf(v[s].x, v[s].x, fmaf(v[s].y, v[s].y, nin));
    }
    int ex = 0;
    if (mx > 0.f) frexpf(mx, &ex);
    const float sc = ldexpf(1.f, -ex);
#pragma unroll
    for (int c = 0; c < D / 4; c++) {
      float x[8];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        x[2 * u] = v[4 * c + u].x * sc;
        x[2 * u + 1] = v[4 * c + u].y * sc;
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
        mma_f16(tmem, dah, dbh, IDESC, ks > 0 ? 1u : 0u);
        mma_f16(tmem + KR, dah, dbl, IDESC, ks > 0 ? 1u : 0u);
        mma_f16(tmem + KR, dal, dbh, IDESC, 1u);
      }
      if (!p.withhold_commit) mma_commit(mbar_a);
    }
    // every row has been read out of this staging buffer: refill it with
    // the tile after next
    const uint64_t cur_base = tile_base(tile) + rbase;
    issue_loads(tile + 2 * (long long)gridDim.x, buf);
    const bool ok = mbar_wait(mbar_a, phase);
    phase ^= 1;
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicExch(err, 1);
      aborted = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    float nout = 0.f;
#pragma unroll
    for (int h = 0; h < KR / 16; h++) {
      uint32_t rb[16], rs[16];
      TmemLd<16>::run(lane_base + 16 * h, rb);
      TmemLd<16>::run(lane_base + KR + 16 * h, rs);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int i = 0; i < 16; i++) {
        const float y = __uint_as_float(rb[i]) + __uint_as_float(rs[i]);
        nout = fmaf(y, y, nout);
      }
    }
    const float f = nout > 0.f ? sqrtf(nin / nout) : 1.f;
    // scale and store, 8 amplitudes per chunk
#pragma unroll
    for (int h = 0; h < KR / 16; h++) {
      uint32_t rb[16], rs[16];
      TmemLd<16>::run(lane_base + 16 * h, rb);
      TmemLd<16>::run(lane_base + KR + 16 * h, rs);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (pair) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int sl = 8 * h + 2 * u;
          float y[4];
#pragma unroll
          for (int q = 0; q < 4; q++) y[q] = (__uint_as_float(rb[4 * u + q]) + __uint_as_float(rs[4 * u + q])) * f;
          *reinterpret_cast<float4 *>(a + cur_base + offset(sl)) = make_float4(y[0], y[1], y[2], y[3]);
        }
      } else {
#pragma unroll
        for (int u = 0; u < 8; u++)
          a[cur_base + offset(8 * h + u)] =
              make_float2((__uint_as_float(rb[2 * u]) + __uint_as_float(rs[2 * u])) * f,
                          (__uint_as_float(rb[2 * u + 1]) + __uint_as_float(rs[2 * u + 1])) * f);
      }
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (aborted) {
    if (tid == 0) mma_commit(mbar_a);
    mbar_wait(mbar_a, phase ^ 1);
  }
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
  (void)LB;
}

// Host tables of the staged kernel; false when the block does not qualify
// (bit 0 a control, or fewer than 7 free bits).
bool stage_param(int n, const Block &b, TcStageParam &p) {
  std::memset(&p, 0, sizeof(p));
  uint64_t fixed = b.cmask;
  for (int j = 0; j < b.k; j++) fixed |= 1ull << b.q[j];
  if (b.cmask & 1ull) return false;
  int freep[64], nfree = 0;
  for (int q = 0; q < n; q++)
    if (!((fixed >> q) & 1)) freep[nfree++] = q;
  if (nfree < 7) return false;
  p.pair = b.q[0] == 0 ? 1 : 0;
  // sub-cube bits in ascending order: 7 lowest free bits and the targets
  int pos[16], np = 0, rbit[16], sbit[16];
  uint64_t cube = 0;
  for (int j = 0; j < 7; j++) cube |= 1ull << freep[j];
  for (int j = 0; j < b.k; j++) cube |= 1ull << b.q[j];
  for (int q = 0; q < 64; q++)
    if ((cube >> q) & 1) {
      pos[np] = q;
      rbit[np] = -1;
      sbit[np] = -1;
      for (int j = 0; j < 7; j++)
        if (freep[j] == q) rbit[np] = j;
      for (int j = 0; j < b.k; j++)
        if (b.q[j] == q) sbit[np] = j;
      np++;
    }
  auto slot_of_bit = [&](int j) -> uint32_t {
    if (rbit[j] >= 0) return p.pair ? (2u << rbit[j]) : (1u << rbit[j]);
    const int sb = sbit[j];
    if (!p.pair) return 128u << sb;
    return sb == 0 ? 1u : (256u << (sb - 1));
  };
  for (int x = 0; x < 64; x++) {
    uint64_t dl = 0, dh = 0;
    uint32_t sl = 0, sh = 0;
    for (int j = 0; j < 6 && j < np; j++)
      if ((x >> j) & 1) {
        dl |= 1ull << pos[j];
        sl += slot_of_bit(j);
      }
    for (int j = 6; j < np && j < 12; j++)
      if ((x >> (j - 6)) & 1) {
        dh |= 1ull << pos[j];
        sh += slot_of_bit(j);
      }
    p.dep_lo[x] = dl;
    p.dep_hi[x] = dh;
    p.slot_lo[x] = (unsigned short)sl;
    p.slot_hi[x] = (unsigned short)sh;
  }
  for (int j = 0; j < 7; j++) p.low7[j] = freep[j];
  for (int j = 0; j < b.k; j++) p.tq[j] = b.q[j];
  p.nhi = 0;
  for (int j = 7; j < nfree; j++) p.hi_pos[p.nhi++] = freep[j];
  p.n_tiles = 1ll << p.nhi;
  p.cmask = b.cmask;
  p.withhold_commit = b.withhold_commit ? 1 : 0;
  return true;
}

template <int K> size_t tc16s_smem_bytes() {
  constexpr size_t KR = 2 << K;
  return 2 * 128 * KR * 2 + 2 * KR * KR * 2 + 2 * (size_t)128 * (1 << K) * 8;
}

template <int K>
cudaError_t run_tc16s(float2 *a, const TcStageParam &p, const void *dev_b, int *err, cudaStream_t s) {
  const size_t smem = tc16s_smem_bytes<K>();
  static thread_local int configured = -1;
  static thread_local int per_sm = 1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    cudaError_t e = cudaFuncSetAttribute(k_dense_tc16s<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int occ = resident_ctas((const void *)k_dense_tc16s<K>, kTcThreads, smem);
    // TMEM: 2 x 128 columns (K = 5) or 4 x 64 (K = 4) stay within 512 per SM
    const int cap = K == 5 ? 2 : 4;
    per_sm = occ > cap ? cap : occ;
    configured = dev;
  }
  long long grid = (long long)dev_info().sms * per_sm;
  if (grid > p.n_tiles) grid = p.n_tiles;
  k_dense_tc16s<K><<<(int)grid, kTcThreads, smem, s>>>(a, (const uint4 *)dev_b, p, err);
  return cudaGetLastError();
}

template <int K, int TPR, int PFD = 1, bool SK = false>
cudaError_t run_tc16(float2 *a, int n, const Block &b, const void *dev_b, int *err, cudaStream_t s) {
  TcParam p;
  p.n_groups = 1ll << (n - K - b.nctrl);
  p.n_tiles = (p.n_groups + kTcThreads - 1) / kTcThreads;
  p.cmask = b.cmask;
  p.withhold_commit = b.withhold_commit ? 1 : 0;
  fill_fixed(b, p.fixed, p.nf);
  for (int j = 0; j < K; j++) p.tq[j] = b.q[j];
  const size_t smem = SK ? tc16_smem_bytes<K>() - (size_t)128 * (2 << K) * 2
                          : tc16_smem_bytes<K>() + (PFD == 3 ? 2 * (size_t)(1 << K) * kTcThreads * 8 : 0);
  // per device: opt in to the shared memory and size one wave of resident
  // CTAs; TMEM columns stay within 512 per SM (4 x 64, 3 x 128, 1 x 256)
  static thread_local int configured = -1;
  static thread_local int per_sm = 1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    cudaError_t e =
        cudaFuncSetAttribute(k_dense_tc16<K, TPR, PFD, SK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int occ = resident_ctas((const void *)k_dense_tc16<K, TPR, PFD, SK>, kTcThreads * TPR, smem);
    // TMEM: at most 512 columns per SM (2 x KR columns per CTA)
    const int tmem_cap = 512 / (4 << K);
    per_sm = occ > Tc16Occ<K, TPR, PFD, SK>::value ? Tc16Occ<K, TPR, PFD, SK>::value : occ;
    if (per_sm > tmem_cap) per_sm = tmem_cap;
    configured = dev;
  }
  long long grid = (long long)dev_info().sms * per_sm;
  if (grid > p.n_tiles) grid = p.n_tiles;
  k_dense_tc16<K, TPR, PFD, SK><<<(int)grid, kTcThreads * TPR, smem, s>>>(a, (const uint4 *)dev_b, p, err);
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

cudaError_t run_dense_tc16(float2 *a, int n, const Block &b, const void *dev_b, int *err, cudaStream_t s) {
  if (b.tc_xg) return run_dense_tc16x(a, n, b, dev_b, err, s);  // B in slot order: only they take it
  if (b.tc_staged && (b.k == 4 || b.k == 5)) {
    static thread_local TcStageParam sp;  // large: kept off the stack; the launch copies it
    if (stage_param(n, b, sp)) return b.k == 4 ? run_tc16s<4>(a, sp, dev_b, err, s) : run_tc16s<5>(a, sp, dev_b, err, s);
  }
  if (b.tc_prefetch == 3 && b.tc_rows == 1) {
    if (b.k == 4) return run_tc16<4, 1, 3>(a, n, b, dev_b, err, s);
    if (b.k == 5) return run_tc16<5, 1, 3>(a, n, b, dev_b, err, s);
  }
  if (b.tc_prefetch == 0 && b.tc_rows == 1) {
    if (b.k == 4) return run_tc16<4, 1, 0>(a, n, b, dev_b, err, s);
    if (b.k == 5) return run_tc16<5, 1, 0>(a, n, b, dev_b, err, s);
  }
  if (b.tc_prefetch == 0 && b.tc_rows == 2 && b.k == 6) return run_tc16<6, 2, 0>(a, n, b, dev_b, err, s);
  if (b.tc_prefetch == 2 && b.tc_rows == 1) {
    if (b.k == 4) return run_tc16<4, 1, 2>(a, n, b, dev_b, err, s);
    if (b.k == 5) return run_tc16<5, 1, 2>(a, n, b, dev_b, err, s);
  }
  if (b.tc_prefetch == 2 && b.tc_rows == 2 && b.k == 6) return run_tc16<6, 2, 2>(a, n, b, dev_b, err, s);
  if (b.tc_splitk && b.tc_rows == 2 && b.k == 6) return run_tc16<6, 2, 1, true>(a, n, b, dev_b, err, s);
  switch (b.k * 8 + b.tc_rows) {
    case 4 * 8 + 1: return run_tc16<4, 1>(a, n, b, dev_b, err, s);
    case 4 * 8 + 2: return run_tc16<4, 2>(a, n, b, dev_b, err, s);
    case 5 * 8 + 1: return run_tc16<5, 1>(a, n, b, dev_b, err, s);
    case 5 * 8 + 2: return run_tc16<5, 2>(a, n, b, dev_b, err, s);
    case 5 * 8 + 4: return run_tc16<5, 4>(a, n, b, dev_b, err, s);
    case 6 * 8 + 1: return run_tc16<6, 1>(a, n, b, dev_b, err, s);
    case 6 * 8 + 2: return run_tc16<6, 2>(a, n, b, dev_b, err, s);
    case 6 * 8 + 4: return run_tc16<6, 4>(a, n, b, dev_b, err, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kern
}  // namespace qs
