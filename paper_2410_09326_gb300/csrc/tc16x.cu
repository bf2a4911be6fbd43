// Dense fused blocks of 4..6 targets on the tensor cores (FP16 operand
// halves, as in tc16.cu) with lane-exchange gathers: a warp loads the
// sub-cube spanned by a block's targets and its five lowest free bits in
// address order and exchanges bits between lanes, registers and the 16-byte
// element (warp shuffles; lane/register exchanges of the loads, where lane
// bit 0 takes no part, by the staging copies' placement) until each lane
// holds one whole group; B is built
// in the same "slot" order (tc16_build_b). The host layout (which bits sit on
// lanes and registers, which exchanges run) is tc_exchange_layout below; the
// planner picks these kernels where tc_exchange_pays.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <type_traits>

#include "tc16_common.cuh"

namespace qs {
namespace kern {

namespace {

// Lane-exchange variant (K = 4, 5; one thread per group; later tiles in
// flight during the MMAs). Where targets sit among the lowest bits, the
// thread-per-group gather above reads short runs per load instruction (16 or
// 32 bytes when bit 1 or 2 is a target), so a warp touches many sectors per
// instruction. Here warp w of a tile owns the sub-cube of its 32 groups
// (targets + the five lowest free bits; the other bits fixed per warp item)
// and loads it in address order: 16-byte loads whose element bit is bit 0,
// lanes over the next five bits, registers over the rest. Warp shuffles then
// exchange position bits -- the element bit with a lane bit (half of every
// register moves), lane bits with register bits (half of the registers
// move) -- until each lane holds one whole group, its amplitudes in slot
// order (slot bit 0 = element bit, 1 + j = register bit j). B is built on the
// host with its rows and columns in the same slot order, so the product comes
// out in slot order, the same exchanges (involutions on disjoint bit pairs)
// restore the load layout 8 slots at a time, and the warp stores as it loaded.
struct TcXParam {
  long long n_tiles;          // tiles of 128 groups = 4 warp items of 32
  unsigned long long cmask;
  int nf;                     // fixed bits of the warp item index
  int fixed[kMaxFixed];
  int lbit[5];                // physical bit of lane bit i (load layout)
  int rbit[5];                // physical bit of register bit j (load layout)
  int la;                     // lane bit exchanged with the element bit, -1: none
  int nswb;                   // lane bits lb[i] exchanged with register bits i
  int lb[2];
  int part_bit[2];            // 6 targets: the target bits thread part h fixes (bit j of h -> part_bit[j])
  int stage_xch;              // bit i: lane/register exchange i of the loads done by the staging copies
  int withhold_commit;
};

// The exchanges of the lane-exchange kernels, on N consecutive 16-byte
// registers starting at a multiple of 4 (register bits 0 and 1 of the pairs
// lie inside any such run): first the element bit with lane bit la -- half
// of every register crosses: lane bit 0 keeps the element-0 half and trades
// its element-1 half for the partner's element-0 half, lane bit 1 the other
// way round -- then lane bit lb[i] with register bit i (half of the
// registers cross). Each is an involution on its own pair of bits and the
// pairs are disjoint, so running them again restores the load layout.
struct LaneExchange {
  int la, nswb, lb0, lb1, lane;
  __device__ __forceinline__ LaneExchange(const TcXParam &p, int lane_)
      : la(p.la), nswb(p.nswb), lb0(p.lb[0]), lb1(p.lb[1]), lane(lane_) {}
  template <int N> __device__ __forceinline__ void run(float4 *w) const {
    element<N>(w);
    lanes<N>(w);
  }
  template <int N> __device__ __forceinline__ void element(float4 *w) const {
    if (la >= 0) {
      const bool up = (lane >> la) & 1;
      const unsigned m = 1u << la;
#pragma unroll
      for (int q = 0; q < N; q++) {
        const float s0 = up ? w[q].x : w[q].z, s1 = up ? w[q].y : w[q].w;
        const float r0 = __shfl_xor_sync(0xffffffffu, s0, m), r1 = __shfl_xor_sync(0xffffffffu, s1, m);
        if (up) {
          w[q].x = r0;
          w[q].y = r1;
        } else {
          w[q].z = r0;
          w[q].w = r1;
        }
      }
    }
  }
  // the lane/register exchanges, but for those in skip (bit i: exchange i)
  template <int N> __device__ __forceinline__ void lanes(float4 *w, int skip = 0) const {
#pragma unroll
    for (int i = 0; i < 2; i++) {
      if (i >= nswb) break;
      if ((skip >> i) & 1) continue;
      const int lbi = i == 0 ? lb0 : lb1;
      const bool up = (lane >> lbi) & 1;
#pragma unroll
      for (int q = 0; q < N; q++) {
        if ((q >> i) & 1) continue;
        const int q2 = q | (1 << i);
        const float4 snd = up ? w[q] : w[q2];
        float4 rcv;
        rcv.x = __shfl_xor_sync(0xffffffffu, snd.x, 1u << lbi);
        rcv.y = __shfl_xor_sync(0xffffffffu, snd.y, 1u << lbi);
        rcv.z = __shfl_xor_sync(0xffffffffu, snd.z, 1u << lbi);
        rcv.w = __shfl_xor_sync(0xffffffffu, snd.w, 1u << lbi);
        if (up) w[q] = rcv;
        else w[q2] = rcv;
      }
    }
  }
};

// The loads go to shared memory by cp.async, two tiles ahead (two staging
// areas, [register][thread] 16-byte slots); each thread reads back its own
// slots, which lanes of its own warp filled (staging_slots below), so a
// __syncwarp is all that guards an area. Without registers held for tiles in flight the SM keeps four
// tiles (128 KB at 5 targets) on the way: the n = 30 benchmark step's
// dominant kernel went from 5.95 (one tile ahead in registers) to 6.36 TB/s
// on GB300. Resident CTAs per SM: 4 (K = 4), 2 (K = 5).
template <int K> constexpr int tc16x_occ() { return K <= 4 ? 4 : 2; }

// The lane/register exchanges i of the loads with bit i of p.stage_xch set
// happen in the staging copies: after them, lane L's register q holds what
// the load layout puts at lane L with bit lb[i] set to bit i of q and
// register q with bit i set to bit lb[i] of L, so the copy of load-layout register q goes
// straight to the staging row of the register that holds it after the
// exchange. Only register bits 0 and 1 take part. Within row r the slots
// are swizzled: lane L's slot is L ^ S(r), S(r) = sum_i (bit i of r) << lb[i],
// which keeps both the copies of one instruction and the read-back of one
// row free of bank conflicts (without it, copies whose lanes differ only in
// bits lb[i] < 3 hit one bank group: the 5-target kernel fell to 4.0 TB/s
// with targets 0..4). wdst[q & 3] + (q & ~3) * stride is where this lane's
// copy of register q goes, rdst[r & 3] + (r & ~3) * stride the slot it
// reads for register r. Threads read chunks other lanes of their warp
// copied, so a __syncwarp follows the wait for the copies (and precedes a
// refill of the area). Measured on GB300 (n = 28, random states) against
// the shuffles: 6 to 12% faster with lb[i] >= 1 (the copies of one 32-byte
// sector stay together), but 6 to 22% slower where lane bit 0 takes part
// (each sector split over two rows), and slower too where a load's runs are
// shorter than 256 bytes and the staged pieces shorter than 64 bytes
// (targets 1, 2, 3, 4, 20: 4993 -> 4710 GB/s; 0, 1, 2, 3, 4 with lane bit
// 0's exchange left to the shuffles: 5225 -> 4750; but 2, 3, 4, 9, 27, whose
// staged bit 3 leaves 64-byte pieces: 5600 -> 5900), so the host stages the
// exchanges with lb[i] >= 1 where bits 0..4 are the element and lane bits or
// the exchanged bit is 3 or above, and leaves the rest to the shuffles.
__device__ __forceinline__ void staging_slots(const TcXParam &p, int warp, int lane, uint32_t stride,
                                              uint32_t wdst[4], uint32_t rdst[4]) {
#pragma unroll
  for (int c = 0; c < 4; c++) {
    int rl = c, sw = 0;
#pragma unroll
    for (int i = 0; i < 2; i++) {
      if (i >= p.nswb) break;
      if (!((p.stage_xch >> i) & 1)) continue;
      const int lb = p.lb[i];
      rl = (rl & ~(1 << i)) | (((lane >> lb) & 1) << i);
      sw |= ((c >> i) & 1) << lb;
    }
    wdst[c] = (uint32_t)rl * stride + (uint32_t)(warp * 32 + (lane ^ sw)) * 16u;
    rdst[c] = (uint32_t)c * stride + (uint32_t)(warp * 32 + (lane ^ sw)) * 16u;
  }
}

// STAGED: some lane/register exchanges are done by the staging copies
// (p.stage_xch != 0); the other instantiation keeps plain per-thread slots
template <int K, bool STAGED>
__global__ void __launch_bounds__(kTcThreads, tc16x_occ<K>())
    k_dense_tc16x(float2 *__restrict__ a, const uint4 *__restrict__ bmat, const __grid_constant__ TcXParam p,
                  int *__restrict__ err) {
  constexpr int D = 1 << K;
  constexpr int NV = D / 2;    // 16-byte registers per lane
  constexpr uint32_t STAGE_BYTES = (uint32_t)NV * kTcThreads * 16u;
  constexpr int RB = K - 1;    // register bits
  constexpr int KR = 2 * D;
  constexpr uint32_t A_BYTES = 128u * KR * 2u;
  constexpr uint32_t B_BYTES = (uint32_t)KR * KR * 2u;
  constexpr uint32_t SBO = (KR / 8) * 128u;
  constexpr uint32_t LBO = 128u;
  constexpr uint32_t NCOLS = 2 * KR;
  constexpr uint32_t IDESC = make_idesc_f16(128, KR);

  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *sA_hi = smem;
  unsigned char *sA_lo = smem + A_BYTES;
  unsigned char *sB = smem + 2 * A_BYTES;  // hi then lo
  unsigned char *sStage = sB + 2 * B_BYTES;  // two staging areas
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  for (int i = tid; i < (int)(2 * B_BYTES / 16); i += kTcThreads) reinterpret_cast<uint4 *>(sB)[i] = bmat[i];
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
  const uint32_t row_off = (uint32_t)(tid >> 3) * SBO + (uint32_t)(tid & 7) * 16u;

  uint64_t lane_off = 0;
#pragma unroll
  for (int i = 0; i < 5; i++)
    if ((lane >> i) & 1) lane_off += 1ull << p.lbit[i];
  uint64_t roff[RB];
#pragma unroll
  for (int j = 0; j < RB; j++) roff[j] = 1ull << p.rbit[j];
  auto offset = [&](int rr) {
    uint64_t o = lane_off;
#pragma unroll
    for (int j = 0; j < RB; j++)
      if ((rr >> j) & 1) o += roff[j];
    return o;
  };
  const LaneExchange xch(p, lane);
  uint32_t wdst[4] = {0, 0, 0, 0}, rdst[4] = {0, 0, 0, 0};
  if constexpr (STAGED) staging_slots(p, warp, lane, kTcThreads * 16u, wdst, rdst);
  auto wslot = [&](int r) {
    return STAGED ? (uint32_t)(r & ~3) * kTcThreads * 16u + wdst[r & 3] : ((uint32_t)r * kTcThreads + (uint32_t)tid) * 16u;
  };
  auto rslot = [&](int r) {
    return STAGED ? (uint32_t)(r & ~3) * kTcThreads * 16u + rdst[r & 3] : ((uint32_t)r * kTcThreads + (uint32_t)tid) * 16u;
  };

  uint32_t phase = 0;
  bool aborted = false;
  long long tile = blockIdx.x;
  float4 v[NV];
  uint64_t base = 0;
  bool valid = false;
  // tile t into staging area u (one commit group per tile, empty past the end)
  uint64_t sbase0 = 0, sbase1 = 0;
  bool svalid0 = false, svalid1 = false;
  auto stage_in = [&](long long t, int u) {
    const bool ok = t < p.n_tiles;
    const uint64_t b = ok ? (insert_zeros((uint64_t)(t * 4 + warp), p.fixed, p.nf) | p.cmask) : 0;
    if (u) {
      sbase1 = b;
      svalid1 = ok;
    } else {
      sbase0 = b;
      svalid0 = ok;
    }
    if (ok) {
      const uint32_t dst = smem_addr(sStage) + (uint32_t)u * STAGE_BYTES;
#pragma unroll
      for (int r = 0; r < NV; r++)
        cp_async16(dst + wslot(r), a + b + offset(r));
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  stage_in(tile, 0);
  stage_in(tile + gridDim.x, 1);

  for (int it = 0; tile < p.n_tiles; tile += gridDim.x, it++) {
    {
      // this tile's group has landed once at most the next one is pending
      asm volatile("cp.async.wait_group 1;" ::: "memory");
      if constexpr (STAGED) __syncwarp();
      const int u = it & 1;
      const unsigned char *src = sStage + (uint32_t)u * STAGE_BYTES;
#pragma unroll
      for (int r = 0; r < NV; r++) v[r] = *reinterpret_cast<const float4 *>(src + rslot(r));
      base = u ? sbase1 : sbase0;
      valid = u ? svalid1 : svalid0;
    }
    if constexpr (STAGED) {
      xch.element<NV>(v);
      xch.lanes<NV>(v, p.stage_xch);
    } else {
      xch.run<NV>(v);
    }
    // row max and squared norm in four independent chains
    float m4[4] = {0.f, 0.f, 0.f, 0.f}, s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int r = 0; r < NV; r++) {
      m4[r & 3] = fmaxf(m4[r & 3], fmaxf(fmaxf(fabsf(v[r].x), fabsf(v[r].y)), fmaxf(fabsf(v[r].z), fabsf(v[r].w))));
      s4[r & 3] = fmaf(v[r].x, v[r].x, fmaf(v[r].y, v[r].y, fmaf(v[r].z, v[r].z, fmaf(v[r].w, v[r].w, s4[r & 3]))));
    }
    const float mx = fmaxf(fmaxf(m4[0], m4[1]), fmaxf(m4[2], m4[3]));
    const float nin = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    const float sc = ldexpf(1.f, -e);
    // slots 4c..4c+3 (registers 2c, 2c + 1) fill the 16-byte row of core matrix c
#pragma unroll
    for (int c = 0; c < D / 4; c++) {
      const float x[8] = {v[2 * c].x * sc,     v[2 * c].y * sc,     v[2 * c].z * sc,     v[2 * c].w * sc,
                          v[2 * c + 1].x * sc, v[2 * c + 1].y * sc, v[2 * c + 1].z * sc, v[2 * c + 1].w * sc};
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
    // refill the area just read (this thread's own chunks). Refilling it
    // right after the read instead measured 0.5-1.8% slower on GB300.
    stage_in(tile + 2 * (long long)gridDim.x, it & 1);
    const bool ok = mbar_wait(mbar_a, phase);
    phase ^= 1;
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicExch(err, 1);
      aborted = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    float o4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int hh = 0; hh < KR / 16; hh++) {
      uint32_t rb[16], rs[16];
      TmemLd<16>::run(lane_base + 16 * hh, rb);
      TmemLd<16>::run(lane_base + KR + 16 * hh, rs);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int i = 0; i < 16; i++) {
        const float y = __uint_as_float(rb[i]) + __uint_as_float(rs[i]);
        o4[i & 3] = fmaf(y, y, o4[i & 3]);
      }
    }
    const float nout = (o4[0] + o4[1]) + (o4[2] + o4[3]);
    const float f = nout > 0.f ? sqrtf(nin / nout) : 1.f;
    // 8 slots (4 registers) at a time: scale, exchange back, store
#pragma unroll
    for (int hh = 0; hh < KR / 16; hh++) {
      uint32_t rb[16], rs[16];
      TmemLd<16>::run(lane_base + 16 * hh, rb);
      TmemLd<16>::run(lane_base + KR + 16 * hh, rs);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      float4 y[4];
#pragma unroll
      for (int q = 0; q < 4; q++)
        y[q] = make_float4((__uint_as_float(rb[4 * q]) + __uint_as_float(rs[4 * q])) * f,
                           (__uint_as_float(rb[4 * q + 1]) + __uint_as_float(rs[4 * q + 1])) * f,
                           (__uint_as_float(rb[4 * q + 2]) + __uint_as_float(rs[4 * q + 2])) * f,
                           (__uint_as_float(rb[4 * q + 3]) + __uint_as_float(rs[4 * q + 3])) * f);
      xch.run<4>(y);
      if (cur_valid) {
#pragma unroll
        for (int q = 0; q < 4; q++) *reinterpret_cast<float4 *>(a + cur_base + offset(4 * hh + q)) = y[q];
      }
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");  // copies still in flight
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (aborted) {
    if (tid == 0) mma_commit(mbar_a);
    mbar_wait(mbar_a, phase ^ 1);
  }
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
}

// Six targets: the same lane exchange with two threads per group. Thread
// (h, r), h = tid / 128, holds the 32 amplitudes of group r whose highest
// target equals h: warp w and warp w + 4 load the same 32 groups' two halves,
// each exactly as a 5-target exchange warp (the highest target fixed per
// half; slot bit 5 = the highest target). The row's scale and norms are
// combined over the two halves through shared memory.
//
// Operand placement. A 6-target tile's A (hi and lo, 64 KB) and B (64 KB)
// would fill shared memory and leave no room to stage loads, so A lives in
// tensor memory instead: the MMA reads its A operand from TMEM (lane m = row
// m, K packed two FP16 values per 32-bit column, 8 columns per K step of
// 16), written by the converting threads with tcgen05.st (thread (h, r)
// writes lane r, columns [32 h, 32 h + 32) of each half). The three
// products accumulate into one FP32 accumulator of 128 columns, so TMEM
// holds two accumulators and two A buffers (4 x 128 columns). Shared memory
// holds B and two 64 KB staging areas.
//
// Warp roles (one CTA per SM). Warps 0..7 convert and store: iteration i
// waits for tile i's products (mbarrier done[i % 2]), rescales, exchanges
// back and stores them, converts tile i + 2 -- read back from its staging area, which is
// refilled with tile i + 4 by cp.async -- into the A buffer tile i used, and
// arrives on ready[i % 2]. Warp 8 issues the MMAs: tile i once ready[i % 2]
// says its A is written and its accumulator read out, with completion on
// done[i % 2]. The converting warps never wait for an MMA issue, and a
// group's two threads (warps w and w + 4) synchronise only with each other,
// on named barrier 1 + w: the four warp pairs run independently between
// the tile-wide mbarriers. Measured on GB300 from random states at n = 28,
// high targets: one A buffer in shared memory, register gathers 5.1 TB/s;
// A in TMEM with staging 5.3; both double-buffered, one thread issuing 4.7;
// warp roles 5.56 (four threads per group instead of two: 5.37); the row
// reductions in independent chains, with results stored as 8-byte slot
// halves where no lane/register exchange had to be undone, 5.87; barriers
// per warp pair 6.01; 16-byte stores after the exchange back in every
// layout instead of those 8-byte ones 6.26.
namespace x6 {
constexpr int kConv = 2 * kTcThreads;  // converting threads, two per group
constexpr int kThreads = kConv + 32;   // + the MMA warp
// The two threads of a group sit in warps w and w + 4 (w = warp % 4): such a
// pair of warps synchronises on its own named barrier 1 + w (64 threads).
__device__ __forceinline__ void pair_sync(int w) { asm volatile("bar.sync %0, 64;" ::"r"(1 + w) : "memory"); }
// AND of a predicate over the pair of warps
__device__ __forceinline__ bool pair_and(int w, bool v) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, %2, 64, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(out)
      : "r"((uint32_t)v), "r"(1 + w)
      : "memory");
  return out != 0;
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
}  // namespace x6

// STAGED as in k_dense_tc16x (the unstaged instantiation measured 5% faster
// than one kernel addressing its slots at run time, for layouts without
// staged exchanges)
template <bool STAGED>
__global__ void __launch_bounds__(x6::kThreads, 1)
    k_dense_tc16x6(float2 *__restrict__ a, const uint4 *__restrict__ bmat, const __grid_constant__ TcXParam p,
                   int *__restrict__ err) {
  constexpr int NT = x6::kConv;  // converting threads
  constexpr int NV = 16;        // 16-byte registers per thread (32 amplitudes)
  constexpr int RB = 4;         // register bits
  constexpr int KR = 128;       // real K = N
  constexpr uint32_t B_BYTES = (uint32_t)KR * KR * 2u;
  constexpr uint32_t STAGE_BYTES = (uint32_t)NV * NT * 16u;  // one tile
  constexpr uint32_t SBO = (KR / 8) * 128u;
  constexpr uint32_t LBO = 128u;
  constexpr uint32_t NCOLS = 512;
  // accumulator u at 128 u, A buffer u (hi, then lo 64 columns after) at 256 + 128 u
  constexpr uint32_t COL_A = 256;
  constexpr uint32_t IDESC = make_idesc_f16(128, KR);

  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *sB = smem;                   // hi then lo
  unsigned char *sStage = smem + 2 * B_BYTES; // two staging areas
  __shared__ __align__(8) uint64_t done[2];   // tile's MMAs complete (one arrival: the commit)
  __shared__ __align__(8) uint64_t ready[2];  // A written, accumulator read out (NT arrivals)
  __shared__ __align__(8) uint64_t drain;     // final commit of the MMA thread
  __shared__ uint32_t tmem_slot;
  __shared__ float red_in[2][2 * NT];         // per A buffer: the prologue converts two tiles back to back
  __shared__ float red_out[2][NT];            // per accumulator: consecutive read-outs alternate
  __shared__ float nin_row[2][kTcThreads];    // input norm of each group, per A buffer

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  for (int i = tid; i < (int)(2 * B_BYTES / 16); i += x6::kThreads) reinterpret_cast<uint4 *>(sB)[i] = bmat[i];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(NCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int u = 0; u < 2; u++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&done[u])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&ready[u])), "n"(NT));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&drain)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // B was written by ordinary stores: make it visible to the tensor cores
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const long long G = gridDim.x;

  if (warp == NT / 32) {
    // ---- the MMA warp: one thread issues, tile after tile ----
    if (lane == 0) {
      const uint32_t b_hi = smem_addr(sB), b_lo = smem_addr(sB + B_BYTES);
      uint32_t pr0 = 0, pr1 = 0;
      int it = 0;
      for (long long t = blockIdx.x; t < p.n_tiles; t += G, it++) {
        const int u = it & 1;
        if (!mbar_wait(smem_addr(&ready[u]), u ? pr1 : pr0)) {
          atomicExch(err, 1);
          break;
        }
        if (u) pr1 ^= 1;
        else pr0 ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t d = tmem + 128u * (uint32_t)u;
        const uint32_t a_hi = tmem + COL_A + 128u * (uint32_t)u, a_lo = a_hi + 64u;
#pragma unroll
        for (int ks = 0; ks < KR / 16; ks++) {
          const uint32_t koff = (uint32_t)ks * 2u * LBO;
          const uint64_t dbh = make_desc(b_hi + koff, LBO, SBO);
          const uint64_t dbl = make_desc(b_lo + koff, LBO, SBO);
          mma_f16_ta(d, a_hi + 8u * ks, dbh, IDESC, ks > 0 ? 1u : 0u);
          mma_f16_ta(d, a_hi + 8u * ks, dbl, IDESC, 1u);
          mma_f16_ta(d, a_lo + 8u * ks, dbh, IDESC, 1u);
        }
        if (!p.withhold_commit) mma_commit(smem_addr(&done[u]));
      }
      // every MMA this thread issued has completed once this commit arrives
      mma_commit(smem_addr(&drain));
      mbar_wait(smem_addr(&drain), 0);
    }
  } else {
    // ---- the converting warps ----
    const int h = tid >> 7;
    const int r = tid & 127;
    // this thread's TMEM lane (row r of A and D) in column 0
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    uint64_t lane_off = h ? (1ull << p.part_bit[0]) : 0ull;
#pragma unroll
    for (int i = 0; i < 5; i++)
      if ((lane >> i) & 1) lane_off += 1ull << p.lbit[i];
    uint64_t roff[RB];
#pragma unroll
    for (int j = 0; j < RB; j++) roff[j] = 1ull << p.rbit[j];
    auto offset = [&](int rr) {
      uint64_t o = lane_off;
#pragma unroll
      for (int j = 0; j < RB; j++)
        if ((rr >> j) & 1) o += roff[j];
      return o;
    };
    auto tile_base = [&](long long t) {
      return insert_zeros((uint64_t)(t * 4 + (warp & 3)), p.fixed, p.nf) | p.cmask;
    };
    const LaneExchange xch(p, lane);
    uint32_t wdst[4] = {0, 0, 0, 0}, rdst[4] = {0, 0, 0, 0};
    if constexpr (STAGED) staging_slots(p, warp, lane, NT * 16u, wdst, rdst);
    auto wslot = [&](int q) {
      return STAGED ? (uint32_t)(q & ~3) * NT * 16u + wdst[q & 3] : ((uint32_t)q * NT + (uint32_t)tid) * 16u;
    };
    auto rslot = [&](int q) {
      return STAGED ? (uint32_t)(q & ~3) * NT * 16u + rdst[q & 3] : ((uint32_t)q * NT + (uint32_t)tid) * 16u;
    };

    // tile t into staging area u: this thread's 16 chunks, one commit group
    // per tile (empty past the last tile, so the group count stays uniform)
    auto stage_in = [&](long long t, int u) {
      if (t < p.n_tiles) {
        const uint64_t b = tile_base(t);
        const uint32_t dst = smem_addr(sStage) + (uint32_t)u * STAGE_BYTES;
#pragma unroll
        for (int q = 0; q < NV; q++) cp_async16(dst + wslot(q), a + b + offset(q));
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // tile t (staged in area u) -> A buffer u: exchange, row scale, FP16
    // hi/lo split, tcgen05.st; refills area u with tile t + 2 G; the row's
    // input norm (both halves) goes to nin_row[u]; then arrives on ready[u]
    auto convert = [&](long long t, int u) {
      asm volatile("cp.async.wait_group 1;" ::: "memory");
      if constexpr (STAGED) __syncwarp();
      float4 v[NV];
      const unsigned char *src = sStage + (uint32_t)u * STAGE_BYTES;
#pragma unroll
      for (int q = 0; q < NV; q++) v[q] = *reinterpret_cast<const float4 *>(src + rslot(q));
      if constexpr (STAGED) {
        xch.element<NV>(v);
        xch.lanes<NV>(v, p.stage_xch);
        __syncwarp();  // every lane of the warp has read its slots
      } else {
        xch.run<NV>(v);
      }
      // refill the area with tile t + 2 G
      stage_in(t + 2 * G, u);
      // row max and squared norm in four independent chains
      float m4[4] = {0.f, 0.f, 0.f, 0.f}, s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < NV; q++) {
        m4[q & 3] = fmaxf(m4[q & 3], fmaxf(fmaxf(fabsf(v[q].x), fabsf(v[q].y)), fmaxf(fabsf(v[q].z), fabsf(v[q].w))));
        s4[q & 3] = fmaf(v[q].x, v[q].x, fmaf(v[q].y, v[q].y, fmaf(v[q].z, v[q].z, fmaf(v[q].w, v[q].w, s4[q & 3]))));
      }
      float mx = fmaxf(fmaxf(m4[0], m4[1]), fmaxf(m4[2], m4[3]));
      float nin = (s4[0] + s4[1]) + (s4[2] + s4[3]);
      red_in[u][2 * tid] = mx;
      red_in[u][2 * tid + 1] = nin;
      x6::pair_sync(warp & 3);
      mx = fmaxf(mx, red_in[u][2 * (tid ^ kTcThreads)]);
      nin += red_in[u][2 * (tid ^ kTcThreads) + 1];
      if (h == 0) nin_row[u][r] = nin;
      int e = 0;
      if (mx > 0.f) frexpf(mx, &e);
      const float sc = ldexpf(1.f, -e);
      // slot 2 q + c (register q, element c) holds K = 64 h + 4 q + 2 c (re)
      // and + 1 (im): column 32 h + 2 q + c of its half
      uint32_t hi[32], lo[32];
#pragma unroll
      for (int q = 0; q < NV; q++) {
        const float x[4] = {v[q].x * sc, v[q].y * sc, v[q].z * sc, v[q].w * sc};
#pragma unroll
        for (int c = 0; c < 2; c++) {
          const __half2 hh = __floats2half2_rn(x[2 * c], x[2 * c + 1]);
          const float2 hf = __half22float2(hh);
          hi[2 * q + c] = *reinterpret_cast<const uint32_t *>(&hh);
          lo[2 * q + c] = pack_half2(x[2 * c] - hf.x, x[2 * c + 1] - hf.y);
        }
      }
      const uint32_t acol = lane_base + COL_A + 128u * (uint32_t)u + 32u * (uint32_t)h;
      TmemSt<32>::run(acol, hi);
      TmemSt<32>::run(acol + 64, lo);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;");
      x6::mbar_arrive(smem_addr(&ready[u]));
    };

    uint32_t pd0 = 0, pd1 = 0;  // parity each accumulator's barrier waits for next
    long long tile = blockIdx.x;
    stage_in(tile, 0);
    stage_in(tile + G, 1);
    if (tile < p.n_tiles) convert(tile, 0);
    if (tile + G < p.n_tiles) convert(tile + G, 1);
    for (int it = 0; tile < p.n_tiles; tile += G, it++) {
      const int u = it & 1;
      const bool ok = mbar_wait(smem_addr(&done[u]), u ? pd1 : pd0);
      if (u) pd1 ^= 1;
      else pd0 ^= 1;
      // a pair that gives up stops arriving on ready[]: the MMA warp's and
      // the other pairs' bounded waits then run out as well
      if (!x6::pair_and(warp & 3, ok)) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      uint32_t y32[64];
      TmemLd<64>::run(lane_base + 128u * (uint32_t)u + 64u * (uint32_t)h, y32);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      float o4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < 64; i++) o4[i & 3] = fmaf(__uint_as_float(y32[i]), __uint_as_float(y32[i]), o4[i & 3]);
      float nout = (o4[0] + o4[1]) + (o4[2] + o4[3]);
      red_out[u][tid] = nout;
      x6::pair_sync(warp & 3);
      nout += red_out[u][tid ^ kTcThreads];
      const float nin = nin_row[u][r];
      const float f = nout > 0.f ? sqrtf(nin / nout) : 1.f;
      const uint64_t cur_base = tile_base(tile);
      // 8 slots (4 registers) at a time: scale, exchange back, store
#pragma unroll
      for (int hh = 0; hh < 4; hh++) {
        float4 y[4];
#pragma unroll
        for (int q = 0; q < 4; q++)
          y[q] = make_float4(__uint_as_float(y32[16 * hh + 4 * q]) * f, __uint_as_float(y32[16 * hh + 4 * q + 1]) * f,
                             __uint_as_float(y32[16 * hh + 4 * q + 2]) * f,
                             __uint_as_float(y32[16 * hh + 4 * q + 3]) * f);
        xch.run<4>(y);
#pragma unroll
        for (int q = 0; q < 4; q++) *reinterpret_cast<float4 *>(a + cur_base + offset(4 * hh + q)) = y[q];
      }
      // tile + 2 G into the A buffer (and, for the MMA warp, the accumulator)
      // this tile has finished with
      if (tile + 2 * G < p.n_tiles) convert(tile + 2 * G, u);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // copies still in flight
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
}

void fill_xparam(int K, int n, const Block &b, const TcXLayout &x, TcXParam &p) {
  std::memset(&p, 0, sizeof(p));
  p.n_tiles = (1ll << (n - K - b.nctrl)) / kTcThreads;
  p.cmask = b.cmask;
  p.nf = x.nf;
  for (int i = 0; i < x.nf; i++) p.fixed[i] = x.fixed[i];
  for (int i = 0; i < 5; i++) p.lbit[i] = x.lbit[i];
  for (int j = 0; j < (K == 6 ? 4 : K - 1); j++) p.rbit[j] = x.rbit[j];
  p.la = x.la;
  p.nswb = x.nswb;
  // staged exchanges (see staging_slots): those with lb[i] >= 1, where a
  // load's runs cover 256 bytes (bits 0..4 on the element and lane bits) or
  // the exchanged bit is 3 or above (the staged pieces stay >= 64 bytes)
  uint64_t eml = 1;
  for (int i = 0; i < 5; i++) eml |= 1ull << x.lbit[i];
  const bool long_runs = (eml & 0x1Full) == 0x1Full;
  p.stage_xch = 0;
  for (int i = 0; i < x.nswb; i++) {
    p.lb[i] = x.lb[i];
    if (x.lb[i] >= 1 && (long_runs || x.lbit[x.lb[i]] >= 3)) p.stage_xch |= 1 << i;
  }
  p.part_bit[0] = x.part_bit[0];
  p.part_bit[1] = x.part_bit[1];
  p.withhold_commit = b.withhold_commit ? 1 : 0;
}

template <int K>
cudaError_t run_tc16x(float2 *a, int n, const Block &b, const TcXLayout &x, const void *dev_b, int *err,
                      cudaStream_t s, LaunchShape *shape) {
  TcXParam p;
  fill_xparam(K, n, b, x, p);
  // two staging areas of one tile (2^(K-1) 16-byte chunks per thread)
  const size_t smem = tc16_smem_bytes<K>() + 2 * (size_t)(1 << (K - 1)) * kTcThreads * 16;
  static thread_local int configured = -1;
  static thread_local int per_sm = 1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    int occ = 1 << 30;
    for (const void *f : {(const void *)k_dense_tc16x<K, false>, (const void *)k_dense_tc16x<K, true>}) {
      cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      occ = std::min(occ, resident_ctas(f, kTcThreads, smem));
    }
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int tmem_cap = 512 / (4 << K);
    per_sm = occ > tc16x_occ<K>() ? tc16x_occ<K>() : occ;
    if (per_sm > tmem_cap) per_sm = tmem_cap;
    configured = dev;
  }
  const int grid = tc_grid((long long)dev_info().sms * per_sm, p.n_tiles, b.tc_max_ctas);
  if (shape) {
    shape->tiles = p.n_tiles;
    shape->ctas = grid;
  }
  if (p.stage_xch) k_dense_tc16x<K, true><<<grid, kTcThreads, smem, s>>>(a, (const uint4 *)dev_b, p, err);
  else k_dense_tc16x<K, false><<<grid, kTcThreads, smem, s>>>(a, (const uint4 *)dev_b, p, err);
  return cudaGetLastError();
}

cudaError_t run_tc16x6(float2 *a, int n, const Block &b, const TcXLayout &x, const void *dev_b, int *err,
                       cudaStream_t s, LaunchShape *shape) {
  TcXParam p;
  fill_xparam(6, n, b, x, p);
  // B (hi + lo) of 64 KB, two 64 KB staging areas (A lives in TMEM)
  const size_t smem = 2 * (size_t)128 * 128 * 2 + 2 * (size_t)16 * 2 * kTcThreads * 16;
  static thread_local int configured = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    for (const void *f : {(const void *)k_dense_tc16x6<false>, (const void *)k_dense_tc16x6<true>}) {
      cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      if (resident_ctas(f, x6::kThreads, smem) < 1) return cudaErrorInvalidConfiguration;
    }
    configured = dev;
  }
  const int grid = tc_grid((long long)dev_info().sms, p.n_tiles, b.tc_max_ctas);  // one CTA per SM
  if (shape) {
    shape->tiles = p.n_tiles;
    shape->ctas = grid;
  }
  if (p.stage_xch) k_dense_tc16x6<true><<<grid, x6::kThreads, smem, s>>>(a, (const uint4 *)dev_b, p, err);
  else k_dense_tc16x6<false><<<grid, x6::kThreads, smem, s>>>(a, (const uint4 *)dev_b, p, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t run_dense_tc16x(float2 *a, int n, const Block &b, const void *dev_b, int *err, cudaStream_t s,
                            LaunchShape *shape) {
  TcXLayout x;
  if (!tc_exchange_layout(n, b, x)) return cudaErrorInvalidValue;
  switch (b.k) {
    case 4: return run_tc16x<4>(a, n, b, x, dev_b, err, s, shape);
    case 5: return run_tc16x<5>(a, n, b, x, dev_b, err, s, shape);
    case 6: return run_tc16x6(a, n, b, x, dev_b, err, s, shape);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kern

bool tc_exchange_pays(const Block &b) {
  if (b.kind != BK_DENSE || b.k < 4 || b.k > 6) return false;
  // measured on GB300 from random states at n = 28: with 5 targets the
  // exchange kernel is ahead for every placement (5.77-6.01 vs 5.56-5.72 TB/s
  // with at most one low target, 4.87-5.79 vs 3.21-4.96 with two or three);
  // with 4 targets only where two or more targets lie among bits 1..3
  // (4.89-5.34 vs 3.41-5.29 TB/s), elsewhere the plain gather is ahead
  // (5.84-6.29 vs 5.59-5.87); with 6 targets (two threads per group) where
  // any target lies among bits 1..3 (4.40-5.13 vs 3.17-5.02 TB/s), not for
  // high targets (5.10-5.51 vs 5.50-5.54)
  if (b.k == 5) return true;
  int low = 0;
  for (int j = 0; j < b.k; j++) low += (b.q[j] >= 1 && b.q[j] <= 3) ? 1 : 0;
  return b.k == 6 ? low >= 1 : low >= 2;
}

bool tc_exchange_layout(int n, const Block &b, TcXLayout &x) {
  if (b.kind == BK_DENSE && b.k == 6 && !(b.cmask & 1ull)) {
    // two threads per group: each part is a 5-target exchange over the five
    // lower targets with the highest fixed (like a control) per part
    Block b5;
    b5.kind = BK_DENSE;
    b5.k = 5;
    for (int j = 0; j < 5; j++) b5.q[j] = b.q[j];
    b5.cmask = b.cmask | (1ull << b.q[5]);
    b5.nctrl = b.nctrl + 1;
    if (!tc_exchange_layout(n, b5, x)) return false;
    x.part_bit[0] = b.q[5];
    x.part_bit[1] = -1;
    x.slot_mat[5] = 5;
    return true;
  }
  x.part_bit[0] = x.part_bit[1] = -1;
  if (b.kind != BK_DENSE || (b.k != 4 && b.k != 5) || (b.cmask & 1ull)) return false;
  const int K = b.k;
  if (n - K - b.nctrl < 7) return false;  // whole tiles of 128 groups
  uint64_t tmask = 0;
  for (int j = 0; j < K; j++) tmask |= 1ull << b.q[j];
  const uint64_t used = tmask | b.cmask;
  uint64_t cube = tmask;  // the warp's sub-cube: targets + the five lowest free bits
  for (int q = 0, nfree = 0; q < 64 && nfree < 5; q++)
    if (!((used >> q) & 1)) {
      cube |= 1ull << q;
      nfree++;
    }
  if (!(cube & 1ull) || __builtin_popcountll(cube) != K + 5) return false;
  auto is_t = [&](int q) { return ((tmask >> q) & 1) != 0; };
  // lane bits: the five lowest bits of the sub-cube above bit 0 (longest
  // runs per load); the rest are register bits
  uint64_t lanes = 0;
  for (int q = 1, nl = 0; q < 64 && nl < 5; q++)
    if ((cube >> q) & 1) {
      lanes |= 1ull << q;
      nl++;
    }
  // targets left on lane bits once the element bit (if free) has taken the
  // lowest one; above two, the highest of them trade places with the lowest
  // free register bits (shorter runs per load, fewer exchanges)
  auto lane_targets = [&]() { return __builtin_popcountll(lanes & tmask) - (is_t(0) ? 0 : 1); };
  while (lane_targets() > 2) {
    const uint64_t lt = lanes & tmask, fr = cube & ~lanes & ~tmask & ~1ull;
    if (!fr) return false;
    const int hi_t = 63 - __builtin_clzll(lt), lo_f = __builtin_ctzll(fr);
    lanes = (lanes & ~(1ull << hi_t)) | (1ull << lo_f);
  }
  // targets on lane bits above bit 3 (past a load's first 128-byte run),
  // other than the element bit's partner, trade places with free register
  // bits too: each load still reads whole 128-byte lines and the lane/
  // register exchange they would need is saved. Measured on GB300 from
  // random states at n = 28 (5 targets 2, 4, 5, 13, 18): 5683 GB/s with the
  // exchanges, 6520 without; moving targets on bits 1..3 as well (runs of
  // 16 to 64 bytes) measured 5 to 48% slower.
  for (;;) {
    uint64_t lt = lanes & tmask & ~0xFull;
    if (!is_t(0)) {
      const uint64_t all = lanes & tmask;
      lt &= ~(all & (~all + 1));  // the element bit's partner: the lowest lane target
    }
    const uint64_t fr = cube & ~lanes & ~tmask & ~1ull;
    if (!lt || !fr) break;
    const int hi_t = 63 - __builtin_clzll(lt), lo_f = __builtin_ctzll(fr);
    lanes = (lanes & ~(1ull << hi_t)) | (1ull << lo_f);
  }
  int nl = 0;
  for (int q = 0; q < 64; q++)
    if ((lanes >> q) & 1) x.lbit[nl++] = q;
  int lpost[5];
  for (int i = 0; i < 5; i++) lpost[i] = x.lbit[i];
  // element bit free: exchange it with the lowest lane bit holding a target
  // (one exists: K targets, K - 1 register bits)
  x.la = -1;
  int epost = 0;
  if (!is_t(0)) {
    for (int i = 0; i < 5 && x.la < 0; i++)
      if (is_t(x.lbit[i])) x.la = i;
    if (x.la < 0) return false;
    epost = x.lbit[x.la];
    lpost[x.la] = 0;
  }
  // lane bits still holding targets <-> register bits holding free bits
  // (equally many); the latter become register bits 0, 1
  int tl[5], ntl = 0, fr[4], nfr = 0, tr[4], ntr = 0;
  for (int i = 0; i < 5; i++)
    if (is_t(lpost[i])) tl[ntl++] = i;
  for (int q = 1; q < 64; q++)
    if (((cube & ~lanes) >> q) & 1) {
      if (is_t(q)) {
        if (ntr < 4) tr[ntr] = q;
        ntr++;
      } else {
        if (nfr < 4) fr[nfr] = q;
        nfr++;
      }
    }
  if (ntr + nfr != K - 1 || ntl != nfr || ntl > 2) return false;
  x.nswb = ntl;
  int rb = 0;
  for (int i = 0; i < nfr; i++) x.rbit[rb++] = fr[i];
  for (int i = 0; i < ntr; i++) x.rbit[rb++] = tr[i];
  for (int i = 0; i < ntl; i++) x.lb[i] = tl[i];
  // the target each slot bit holds once the exchanges are done
  int slot_phys[6];
  slot_phys[0] = epost;
  for (int j = 0; j < K - 1; j++) slot_phys[1 + j] = j < ntl ? lpost[tl[j]] : x.rbit[j];
  for (int s = 0; s < K; s++) {
    x.slot_mat[s] = -1;
    for (int t = 0; t < K; t++)
      if (b.q[t] == slot_phys[s]) x.slot_mat[s] = t;
    if (x.slot_mat[s] < 0) return false;
  }
  const uint64_t fixedm = cube | b.cmask;
  if (__builtin_popcountll(fixedm) > kMaxFixed) return false;
  x.nf = 0;
  for (int q = 0; q < 64; q++)
    if ((fixedm >> q) & 1) x.fixed[x.nf++] = q;
  return true;
}

}  // namespace qs
