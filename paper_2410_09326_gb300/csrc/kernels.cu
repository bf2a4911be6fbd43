// CUDA kernels of the simulator core (sm_103a).
//
// Every kernel is one HBM pass over the amplitudes a block changes:
//  - k_dense_param / k_dense_smem: a fused block with K targets (the 2^K x 2^K
//    product matrix of Sec. III-D's merged gates). One thread owns one group
//    of 2^K amplitudes at a time; consecutive threads own groups whose bases
//    differ in the lowest free bits, so a warp's loads for one matrix column
//    are contiguous whenever the targets sit above bit 4. The matrix of
//    blocks with K <= 5 (c64) / K <= 4 (c128) travels in the kernel's
//    parameter space, so the fully unrolled mat-vec reads its entries as
//    constant-bank operands of the FMAs and costs no loads.
//  - k_diag: a diagonal block of up to QS_MAX_DIAG qubits: one multiply by a
//    phase looked up in shared memory.
//  - k_permute: exchange of two physical bits (a plain SWAP, Sec. III-D; also
//    used to restore logical order).
//  - k_probs / k_probs_reduce: FP64 marginal probabilities (Sec. II-B, "final
//    probability distribution") with per-CTA shared-memory histograms and a
//    fixed-order cross-CTA sum.
// Control bits never enter the index space: only the 2^(n - controls)
// amplitudes whose control bits are 1 are read and written.
#include <cstring>
#include <mutex>
#include <string>

#include "kernels_common.cuh"

namespace qs {
namespace kern {

int resident_ctas(const void *func, int threads, size_t dyn_smem) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, func) != cudaSuccess) return 1;
  int dev = 0;
  cudaGetDevice(&dev);
  int regs_sm = 65536, smem_sm = 228 * 1024, thr_sm = 2048, reserved = 1024;
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  const int warps = (threads + 31) / 32;
  const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;  // 256-register allocation units
  int by_regs = regs_warp > 0 ? regs_sm / (regs_warp * warps) : 64;
  int by_smem = (int)(smem_sm / (fa.sharedSizeBytes + dyn_smem + reserved));
  int by_thr = thr_sm / threads;
  int r = by_regs < by_smem ? by_regs : by_smem;
  if (by_thr < r) r = by_thr;
  return r < 1 ? 1 : r;
}

int grid_for(long long work, int threads) {
  const DevInfo &di = dev_info();
  long long want = (work + threads - 1) / threads;
  long long cap = (long long)di.sms * (di.max_threads_per_sm / threads) * 4;
  if (cap < 1) cap = 1;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

template <typename T> struct DiagParam {
  T tab[1 << QS_MAX_DIAG];
  long long n_amps;  // 2^(n - controls)
  unsigned long long cmask;
  int nf;
  int fixed[kMaxFixed];  // control positions ascending
  int k;
  int tq[QS_MAX_DIAG];
};

template <typename T>
__global__ void __launch_bounds__(256) k_diag(T *__restrict__ a, const __grid_constant__ DiagParam<T> p) {
  using R = typename Real<T>::type;
  __shared__ T tab[1 << QS_MAX_DIAG];
  const int tn = 1 << p.k;
  for (int i = threadIdx.x; i < tn; i += blockDim.x) tab[i] = p.tab[i];
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < p.n_amps; j += stride) {
    const uint64_t idx = insert_zeros((uint64_t)j, p.fixed, p.nf) | p.cmask;
    int l = 0;
    for (int b = 0; b < p.k; b++) l |= (int)((idx >> p.tq[b]) & 1) << b;
    const T w = tab[l];
    const T v = a[idx];
    T y;
    y.x = fma((R)w.x, v.x, -(R)w.y * v.y);
    y.y = fma((R)w.x, v.y, (R)w.y * v.x);
    a[idx] = y;
  }
}

// Chunked diagonal pass, used when no control bit lies below bit kChunkBits:
// the compacted index space splits into chunks of 2^kChunkBits amplitudes
// that are contiguous in memory. The table index of an amplitude is
// (index bits of the chunk base on table qubits >= kChunkBits) OR
// lo_tab[offset within the chunk], so the per-amplitude work is one shared
// load, one table load and a complex multiply; each thread moves 16 bytes
// per access.
constexpr int kChunkBits = 10;

template <typename T>
__global__ void __launch_bounds__(256) k_diag_chunk(T *__restrict__ a, const __grid_constant__ DiagParam<T> p) {
  using R = typename Real<T>::type;
  constexpr int CH = 1 << kChunkBits;
  constexpr int PER = sizeof(T) == 8 ? 2 : 1;  // amplitudes per 16-byte access
  constexpr int LANES = CH / PER;              // accesses per chunk
  __shared__ T tab[1 << QS_MAX_DIAG];
  __shared__ uint16_t lo_tab[CH];
  const int tn = 1 << p.k;
  for (int i = threadIdx.x; i < tn; i += blockDim.x) tab[i] = p.tab[i];
  for (int o = threadIdx.x; o < CH; o += blockDim.x) {
    int l = 0;
    for (int b = 0; b < p.k; b++)
      if (p.tq[b] < kChunkBits) l |= ((o >> p.tq[b]) & 1) << b;
    lo_tab[o] = (uint16_t)l;
  }
  __syncthreads();
  const long long n_chunks = p.n_amps >> kChunkBits;
  const long long total = n_chunks * LANES;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    const long long chunk = t / LANES;
    const int o = (int)(t - chunk * LANES) * PER;
    const uint64_t cbase = insert_zeros((uint64_t)chunk << kChunkBits, p.fixed, p.nf) | p.cmask;
    int lhi = 0;
    for (int b = 0; b < p.k; b++)
      if (p.tq[b] >= kChunkBits) lhi |= (int)((cbase >> p.tq[b]) & 1) << b;
    T *ptr = a + cbase + o;
    if constexpr (PER == 2) {
      float4 v = *reinterpret_cast<const float4 *>(ptr);
      const T w0 = tab[lhi | lo_tab[o]], w1 = tab[lhi | lo_tab[o + 1]];
      float4 y;
      y.x = fmaf(w0.x, v.x, -w0.y * v.y);
      y.y = fmaf(w0.x, v.y, w0.y * v.x);
      y.z = fmaf(w1.x, v.z, -w1.y * v.w);
      y.w = fmaf(w1.x, v.w, w1.y * v.z);
      *reinterpret_cast<float4 *>(ptr) = y;
    } else {
      const T v = *ptr;
      const T w = tab[lhi | lo_tab[o]];
      T y;
      y.x = fma((R)w.x, v.x, -(R)w.y * v.y);
      y.y = fma((R)w.x, v.y, (R)w.y * v.x);
      *ptr = y;
    }
  }
}

// Exchange of physical bits qa < qb: the amplitudes with (bit qa, bit qb) =
// (1, 0) and (0, 1) trade places. Each thread keeps kPermUnroll exchanges in
// flight (all loads before the stores). With complex64 and qa >= 1 the two
// amplitudes that differ only in bit 0 move together as one 16-byte access,
// so bit 0 joins the fixed bits and every access is a full 16 bytes.
constexpr int kPermUnroll = 4;

template <typename V>
__global__ void __launch_bounds__(256) k_permute(V *__restrict__ a, long long n_items, int nf, int f0, int f1,
                                                 int f2, unsigned long long da, unsigned long long db) {
  const int fixed[3] = {f0, f1, f2};
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; j + (kPermUnroll - 1) * stride < n_items; j += kPermUnroll * stride) {
    V x[kPermUnroll], y[kPermUnroll];
    uint64_t i0[kPermUnroll];
#pragma unroll
    for (int u = 0; u < kPermUnroll; u++) {
      i0[u] = insert_zeros((uint64_t)(j + u * stride), fixed, nf);
      x[u] = a[i0[u] + da];
      y[u] = a[i0[u] + db];
    }
#pragma unroll
    for (int u = 0; u < kPermUnroll; u++) {
      a[i0[u] + da] = y[u];
      a[i0[u] + db] = x[u];
    }
  }
  for (; j < n_items; j += stride) {
    const uint64_t i0 = insert_zeros((uint64_t)j, fixed, nf);
    const V x = a[i0 + da], y = a[i0 + db];
    a[i0 + da] = y;
    a[i0 + db] = x;
  }
}

template <typename T> __global__ void k_set_one(T *a, uint64_t idx) {
  T one;
  one.x = 1;
  one.y = 0;
  a[idx] = one;
}

constexpr int kProbsSmemBits = 12;  // shared histogram up to 4096 bins
constexpr int kMaxProbBits = 26;

struct ProbsParam {
  long long n_amps;
  int m;
  int pos[kMaxProbBits];
};

__device__ __forceinline__ int extract_bits(uint64_t i, const int *pos, int m) {
  int b = 0;
  for (int j = 0; j < m; j++) b |= (int)((i >> pos[j]) & 1) << j;
  return b;
}

template <typename T>
__global__ void __launch_bounds__(256) k_probs(const T *__restrict__ a, const __grid_constant__ ProbsParam p,
                                               double *__restrict__ partial) {
  // each thread keeps UNROLL 16-byte loads in flight per trip (two complex64
  // amplitudes or one complex128 amplitude per load)
  constexpr int PER = sizeof(T) == 8 ? 2 : 1;
  constexpr int UNROLL = 4;
  extern __shared__ double hist[];
  const int nb = 1 << p.m;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0.0;
  __syncthreads();
  const unsigned lane = threadIdx.x & 31;
  const long long n_vec = p.n_amps / PER;
  const long long S = (long long)gridDim.x * blockDim.x;
  // every lane runs the same trip count so the warp collectives stay converged
  const long long trips = (n_vec + S * UNROLL - 1) / (S * UNROLL);
  const long long j0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long t = 0; t < trips; t++) {
    double v[UNROLL * PER];
    int bin[UNROLL * PER];
#pragma unroll
    for (int u = 0; u < UNROLL; u++) {
      const long long j = j0 + (t * UNROLL + u) * S;
      if (j < n_vec) {
        if constexpr (PER == 2) {
          const float4 x = *reinterpret_cast<const float4 *>(a + 2 * j);
          v[2 * u] = (double)x.x * x.x + (double)x.y * x.y;
          v[2 * u + 1] = (double)x.z * x.z + (double)x.w * x.w;
        } else {
          const T x = a[j];
          v[u] = (double)x.x * x.x + (double)x.y * x.y;
        }
      } else {
#pragma unroll
        for (int e = 0; e < PER; e++) v[u * PER + e] = 0.0;
      }
#pragma unroll
      for (int e = 0; e < PER; e++) bin[u * PER + e] = extract_bits((uint64_t)(j * PER + e), p.pos, p.m);
    }
#pragma unroll
    for (int e = 0; e < UNROLL * PER; e++) {
      const int b0 = __shfl_sync(0xffffffffu, bin[e], 0);
      if (__all_sync(0xffffffffu, bin[e] == b0)) {
        double s = v[e];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && s != 0.0) atomicAdd(&hist[b0], s);
      } else if (v[e] != 0.0) {
        atomicAdd(&hist[bin[e]], v[e]);
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nb; k += blockDim.x) partial[(size_t)blockIdx.x * nb + k] = hist[k];
}

__global__ void k_probs_reduce(const double *__restrict__ partial, int nblocks, int nb,
                               double *__restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nb) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; b++) s += partial[(size_t)b * nb + k];
  out[k] = s;
}

// Wide histograms: one thread per bin, looping over the summed-out bits.
template <typename T>
__global__ void __launch_bounds__(256) k_probs_wide(const T *__restrict__ a, const __grid_constant__ ProbsParam p,
                                                    int n, double *__restrict__ out) {
  const long long nb = 1ll << p.m;
  const long long per = 1ll << (n - p.m);
  int rest[64];
  int nr = 0;
  for (int q = 0; q < n; q++) {
    bool used = false;
    for (int j = 0; j < p.m; j++) used |= (p.pos[j] == q);
    if (!used) rest[nr++] = q;
  }
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += stride) {
    uint64_t base = 0;
    for (int j = 0; j < p.m; j++) base |= (uint64_t)((b >> j) & 1) << p.pos[j];
    double s = 0.0;
    for (long long r = 0; r < per; r++) {
      uint64_t idx = base;
      for (int j = 0; j < nr; j++) idx |= (uint64_t)((r >> j) & 1) << rest[j];
      const T x = a[idx];
      s += (double)x.x * (double)x.x + (double)x.y * (double)x.y;
    }
    out[b] = s;
  }
}

template <typename T>
cudaError_t run_block(T *a, int n, const Block &b, const void *dev_mat, cudaStream_t s, int threads) {
  if (b.kind == BK_PERMUTE) {
    const int qa = b.q[0], qb = b.q[1];  // qa < qb
    if (sizeof(T) == 8 && qa >= 1) {
      // 16-byte pairs over bit 0: indices in units of two amplitudes
      const long long items = 1ll << (n - 3);
      k_permute<float4><<<grid_for(items / kPermUnroll, threads), threads, 0, s>>>(
          (float4 *)a, items, 2, qa - 1, qb - 1, 0, 1ull << (qa - 1), 1ull << (qb - 1));
    } else {
      const long long items = 1ll << (n - 2);
      k_permute<T><<<grid_for(items / kPermUnroll, threads), threads, 0, s>>>(a, items, 2, qa, qb, 0, 1ull << qa,
                                                                            1ull << qb);
    }
    return cudaGetLastError();
  }
  if (b.kind == BK_DIAG) {
    static thread_local DiagParam<T> p;
    const int tn = 1 << b.k;
    for (int i = 0; i < tn; i++) p.tab[i] = to_dev<T>(b.mat[i]);
    p.n_amps = 1ll << (n - b.nctrl);
    p.cmask = b.cmask;
    fill_fixed(b, p.fixed, p.nf);
    p.k = b.k;
    for (int j = 0; j < b.k; j++) p.tq[j] = b.q[j];
    const bool chunked = (b.cmask & ((1ull << kChunkBits) - 1)) == 0 && n - b.nctrl >= kChunkBits;
    if (chunked) {
      const long long accesses = p.n_amps / (sizeof(T) == 8 ? 2 : 1);
      k_diag_chunk<T><<<grid_for(accesses, threads), threads, 0, s>>>(a, p);
    } else {
      k_diag<T><<<grid_for(p.n_amps, threads), threads, 0, s>>>(a, p);
    }
    return cudaGetLastError();
  }
  if constexpr (sizeof(T) == 8) return run_dense_c64((float2 *)a, n, b, dev_mat, s, threads);
  else return run_dense_c128((double2 *)a, n, b, dev_mat, s, threads);
}

}  // namespace kern

using namespace kern;

const DevInfo &dev_info() {
  static thread_local DevInfo di;
  static thread_local int dev_cached = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != dev_cached) {
    cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&di.max_threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (di.sms <= 0) di.sms = 1;
    if (di.max_threads_per_sm <= 0) di.max_threads_per_sm = 1024;
    dev_cached = dev;
  }
  return di;
}

bool block_needs_dev_matrix(const Block &b, bool c128) {
  if (b.kind == BK_TILE || b.kind == BK_PHASE) return true;
  if (b.kind != BK_DENSE) return false;
  if (b.tc && !c128) return true;
  return b.k == 6 || (c128 && b.k == 5);
}

size_t block_dev_matrix_bytes(const Block &b, bool c128) {
  if (!block_needs_dev_matrix(b, c128)) return 0;
  if (b.kind == BK_TILE) return tile_desc_bytes(b, c128);
  if (b.kind == BK_PHASE) return phase_desc_bytes(b, c128);
  if (b.tc && !c128) return b.tc_tf32 ? tc_b_floats(b.k) * sizeof(float) : tc16_b_bytes(b.k);
  return b.mat.size() * (c128 ? 16 : 8);
}

void fill_dev_matrix(const Block &b, bool c128, void *host_out) {
  if (b.kind == BK_TILE) {
    tile_fill_desc(b, c128, host_out);
    return;
  }
  if (b.kind == BK_PHASE) {
    phase_fill_desc(b, c128, host_out);
    return;
  }
  if (b.tc && !c128) {
    if (b.tc_tf32) tc_build_b(b, (float *)host_out);
    else tc16_build_b(b, host_out);
    return;
  }
  for (size_t k = 0; k < b.mat.size(); k++) {
    if (c128) {
      double v[2] = {b.mat[k].real(), b.mat[k].imag()};
      std::memcpy((char *)host_out + k * 16, v, 16);
    } else {
      float v[2] = {(float)b.mat[k].real(), (float)b.mat[k].imag()};
      std::memcpy((char *)host_out + k * 8, v, 8);
    }
  }
}

cudaError_t launch_block_with_matrix(void *amps, int n, bool c128, const Block &b, const void *dev_mat,
                                     int *err, cudaStream_t s, int threads, LaunchShape *shape) {
  if (threads <= 0) threads = 256;
  if (b.kind == BK_TILE) return run_tile(amps, n, c128, b, dev_mat, s);
  if (b.kind == BK_PHASE) return run_phase(amps, n, c128, b, dev_mat, s, shape);
  if (b.kind == BK_DENSE && b.tc && !c128)
    return b.tc_tf32 ? run_dense_tc((float2 *)amps, n, b, dev_mat, err, s, shape)
                     : run_dense_tc16((float2 *)amps, n, b, dev_mat, err, s, shape);
  if (c128) return run_block<double2>((double2 *)amps, n, b, dev_mat, s, threads);
  return run_block<float2>((float2 *)amps, n, b, dev_mat, s, threads);
}

cudaError_t launch_block(void *amps, int n, bool c128, const Block &b, cudaStream_t s, int threads) {
  return launch_block_with_matrix(amps, n, c128, b, nullptr, nullptr, s, threads);
}

// Marginals with more than 12 measured bits. The state is cut into chunks
// of 2^12 contiguous amplitudes; within a chunk the measured bits above bit
// 11 are constant (they give the high part of the bin) and the measured bits
// below bit 12 index a shared-memory sub-histogram. Chunks are visited in an
// order whose fastest-varying bits are the summed-out high bits, so a CTA
// walking a contiguous range of that order flushes its sub-histogram (FP64
// global atomics into the zeroed output) only when the high part changes.
constexpr int kProbChunkBits = 12;

struct ProbsChunkParam {
  int m_lo;                      // measured bits below kProbChunkBits
  int lo_pos[kProbChunkBits];    // their positions
  int lo_j[kProbChunkBits];      // their bin bit
  int n_sum_hi;                  // summed-out bits >= kProbChunkBits
  int sum_hi_pos[64];
  int m_hi;                      // measured bits >= kProbChunkBits
  int hi_pos[kMaxProbBits];
  int hi_j[kMaxProbBits];
  long long n_chunks;
};

__device__ __forceinline__ void chunk_of(long long cp, const ProbsChunkParam &p, uint64_t &chunk_base,
                                         unsigned &hi_bin) {
  // cp = (measured-high bits, summed-high bits fastest) -> amplitude index of
  // the chunk start and the high part of its bin
  uint64_t base = 0;
  int b = 0;
  for (int i = 0; i < p.n_sum_hi; i++, b++) base |= (uint64_t)((cp >> b) & 1) << p.sum_hi_pos[i];
  unsigned hb = 0;
  for (int i = 0; i < p.m_hi; i++, b++) {
    const unsigned bit = (unsigned)((cp >> b) & 1);
    base |= (uint64_t)bit << p.hi_pos[i];
    hb |= bit << p.hi_j[i];
  }
  chunk_base = base;
  hi_bin = hb;
}

template <typename T>
__global__ void __launch_bounds__(256) k_probs_chunk(const T *__restrict__ a, const __grid_constant__ ProbsChunkParam p,
                                                     double *__restrict__ out) {
  // Thread t always reads the same NSLOT offsets of every chunk, so the low
  // part of each slot's bin never changes: the squares accumulate in
  // registers and meet (warp reduction, shared histogram, FP64 atomics into
  // `out`) only when the chunk's high part of the bin changes.
  constexpr int CH = 1 << kProbChunkBits;
  constexpr int PER = sizeof(T) == 8 ? 2 : 1;  // amplitudes per 16-byte load
  constexpr int NLD = CH / (256 * PER);        // loads per thread per chunk
  constexpr int NSLOT = NLD * PER;
  __shared__ double hist[CH];
  const int nsub = 1 << p.m_lo;
  for (int s = threadIdx.x; s < nsub; s += blockDim.x) hist[s] = 0.0;
  int sub[NSLOT];
#pragma unroll
  for (int u = 0; u < NLD; u++)
#pragma unroll
    for (int e = 0; e < PER; e++) {
      const int o = (threadIdx.x + u * 256) * PER + e;
      int s = 0;
      for (int i = 0; i < p.m_lo; i++) s |= ((o >> p.lo_pos[i]) & 1) << i;
      sub[u * PER + e] = s;
    }
  auto lo_bin = [&](int s) {
    unsigned b = 0;
    for (int i = 0; i < p.m_lo; i++) b |= (unsigned)((s >> i) & 1) << p.lo_j[i];
    return b;
  };
  __syncthreads();
  const unsigned lane = threadIdx.x & 31;
  // complex64: each slot sums |a|^2 in compensated FP32 (Kahan) and meets
  // FP64 at the flush; GB300's FP64 rate could not keep up with one FP64
  // operation per amplitude at HBM speed. complex128: FP64 throughout.
  using Acc = typename Real<T>::type;
  Acc acc[NSLOT], comp[NSLOT];
#pragma unroll
  for (int e = 0; e < NSLOT; e++) acc[e] = comp[e] = 0;
  // when every slot of every thread in the CTA lands in the same bin (no
  // measured bit below bit 12), the slots are summed in the thread first
  bool same = true;
#pragma unroll
  for (int e = 1; e < NSLOT; e++) same &= sub[e] == sub[0];
  const bool one_bin = __syncthreads_and(same && sub[0] == 0);
  auto flush = [&](unsigned hb) {
    if (one_bin) {
      double v = 0.0;
#pragma unroll
      for (int e = 0; e < NSLOT; e++) {
        v += (double)acc[e] - (double)comp[e];
        acc[e] = comp[e] = 0;
      }
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0 && v != 0.0) atomicAdd(&hist[0], v);
      __syncthreads();
      if (threadIdx.x == 0) {
        if (hist[0] != 0.0) atomicAdd(&out[hb], hist[0]);
        hist[0] = 0.0;
      }
      __syncthreads();
      return;
    }
#pragma unroll
    for (int e = 0; e < NSLOT; e++) {
      const int b0 = __shfl_sync(0xffffffffu, sub[e], 0);
      double v = (double)acc[e] - (double)comp[e];
      acc[e] = comp[e] = 0;
      if (__all_sync(0xffffffffu, sub[e] == b0)) {
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0 && v != 0.0) atomicAdd(&hist[b0], v);
      } else if (v != 0.0) {
        atomicAdd(&hist[sub[e]], v);
      }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < nsub; s += blockDim.x) {
      const double v = hist[s];
      if (v != 0.0) atomicAdd(&out[hb | lo_bin(s)], v);
      hist[s] = 0.0;
    }
    __syncthreads();
  };
  // contiguous range of the chunk order for this CTA
  const long long per = (p.n_chunks + gridDim.x - 1) / gridDim.x;
  const long long c0 = (long long)blockIdx.x * per;
  const long long c1 = c0 + per < p.n_chunks ? c0 + per : p.n_chunks;
  unsigned cur_hi = 0;
  bool dirty = false;
  for (long long cp = c0; cp < c1; cp++) {
    uint64_t base;
    unsigned hb;
    chunk_of(cp, p, base, hb);
    if (dirty && hb != cur_hi) flush(cur_hi);
    cur_hi = hb;
    dirty = true;
    T xs[NSLOT];
#pragma unroll
    for (int u = 0; u < NLD; u++) {
      const int o = (threadIdx.x + u * 256) * PER;
      if constexpr (PER == 2) {
        const float4 x = *reinterpret_cast<const float4 *>(a + base + o);
        xs[2 * u].x = x.x;
        xs[2 * u].y = x.y;
        xs[2 * u + 1].x = x.z;
        xs[2 * u + 1].y = x.w;
      } else {
        xs[u] = a[base + o];
      }
    }
#pragma unroll
    for (int e = 0; e < NSLOT; e++) {
      if constexpr (sizeof(T) == 8) {
        const float y = fmaf(xs[e].x, xs[e].x, xs[e].y * xs[e].y) - comp[e];
        const float t = acc[e] + y;
        comp[e] = (t - acc[e]) - y;
        acc[e] = t;
      } else {
        acc[e] += xs[e].x * xs[e].x + xs[e].y * xs[e].y;
      }
    }
  }
  if (__syncthreads_or(dirty)) flush(cur_hi);
}

// sum |a_i - b_i|^2 over i, one FP64 partial per CTA (fixed-order reduce)
template <typename Ta, typename Tb>
__global__ void __launch_bounds__(256) k_distance(const Ta *__restrict__ a, const Tb *__restrict__ b, long long N,
                                                  double *__restrict__ partial) {
  __shared__ double red[256];
  double s = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    const double dx = (double)a[i].x - (double)b[i].x, dy = (double)a[i].y - (double)b[i].y;
    s += dx * dx + dy * dy;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

template <typename T> size_t param_bytes_t(const Block &b) {
  if (b.kind == BK_TILE) return 2 * sizeof(T *) + sizeof(long long) + tile_desc_bytes(b, sizeof(T) == 16);
  if (b.kind == BK_PHASE) return 2 * sizeof(T *) + sizeof(long long) + phase_desc_bytes(b, sizeof(T) == 16);
  if (b.kind == BK_PERMUTE) return sizeof(T *) + sizeof(long long) + 2 * sizeof(int);
  if (b.kind == BK_DIAG) return sizeof(T *) + sizeof(DiagParam<T>);
  switch (b.k) {
    case 1: return sizeof(T *) + sizeof(DenseParam<T, 1>);
    case 2: return sizeof(T *) + sizeof(DenseParam<T, 2>);
    case 3: return sizeof(T *) + sizeof(DenseParam<T, 3>);
    case 4: return sizeof(T *) + sizeof(DenseParam<T, 4>);
    case 5:
      if (sizeof(T) == 8) return sizeof(T *) + sizeof(DenseParam<T, 5>);
      return 2 * sizeof(T *) + sizeof(DenseIdx) + (sizeof(T) << 10);
    default: return 2 * sizeof(T *) + sizeof(DenseIdx) + (sizeof(T) << 12);
  }
}

size_t block_param_bytes(const Block &b, bool c128) {
  return c128 ? param_bytes_t<double2>(b) : param_bytes_t<float2>(b);
}

cudaError_t launch_permute(void *amps, int n, bool c128, int qa, int qb, cudaStream_t s) {
  Block b;
  b.kind = BK_PERMUTE;
  b.q[0] = qa < qb ? qa : qb;
  b.q[1] = qa < qb ? qb : qa;
  return launch_block(amps, n, c128, b, s, 256);
}

cudaError_t launch_set_basis(void *amps, int n, bool c128, uint64_t idx, cudaStream_t s) {
  const size_t bytes = (size_t)(c128 ? 16 : 8) << n;
  cudaError_t e = cudaMemsetAsync(amps, 0, bytes, s);
  if (e != cudaSuccess) return e;
  if (c128) k_set_one<double2><<<1, 1, 0, s>>>((double2 *)amps, idx);
  else k_set_one<float2><<<1, 1, 0, s>>>((float2 *)amps, idx);
  return cudaGetLastError();
}

int distance_grid() { return dev_info().sms * 4; }

cudaError_t launch_distance(const void *a, bool a128, const void *b, bool b128, int n, double *partial,
                            cudaStream_t s) {
  const long long N = 1ll << n;
  const int grid = distance_grid();
  if (!a128 && !b128) k_distance<float2, float2><<<grid, 256, 0, s>>>((const float2 *)a, (const float2 *)b, N, partial);
  else if (!a128 && b128) k_distance<float2, double2><<<grid, 256, 0, s>>>((const float2 *)a, (const double2 *)b, N, partial);
  else if (a128 && !b128) k_distance<double2, float2><<<grid, 256, 0, s>>>((const double2 *)a, (const float2 *)b, N, partial);
  else k_distance<double2, double2><<<grid, 256, 0, s>>>((const double2 *)a, (const double2 *)b, N, partial);
  return cudaGetLastError();
}

int probs_grid(int n) {
  const long long N = 1ll << n;
  return grid_for(N, 256);
}

size_t probs_scratch_doubles(int n, int m) {
  if (m > kProbsSmemBits || n >= kProbChunkBits) return 0;
  return (size_t)probs_grid(n) << m;
}

cudaError_t launch_probs(const void *amps, int n, bool c128, const int *pos, int m, double *partial,
                         double *out, cudaStream_t s) {
  if (m < 0 || m > kMaxProbBits || m > n) return cudaErrorInvalidValue;
  ProbsParam p;
  p.n_amps = 1ll << n;
  p.m = m;
  for (int j = 0; j < m; j++) p.pos[j] = pos[j];
  if (m <= kProbsSmemBits && n < kProbChunkBits) {
    const int grid = probs_grid(n);
    const size_t smem = sizeof(double) << m;
    if (c128) k_probs<double2><<<grid, 256, smem, s>>>((const double2 *)amps, p, partial);
    else k_probs<float2><<<grid, 256, smem, s>>>((const float2 *)amps, p, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nb = 1 << m;
    k_probs_reduce<<<(nb + 255) / 256, 256, 0, s>>>(partial, grid, nb, out);
    return cudaGetLastError();
  }
  const long long nb = 1ll << m;
  if (n >= kProbChunkBits) {
    ProbsChunkParam c;
    std::memset(&c, 0, sizeof(c));
    bool used[64] = {false};
    for (int j = 0; j < m; j++) {
      used[pos[j]] = true;
      if (pos[j] < kProbChunkBits) {
        c.lo_pos[c.m_lo] = pos[j];
        c.lo_j[c.m_lo++] = j;
      }
    }
    for (int q = kProbChunkBits; q < n; q++) {
      if (used[q]) continue;
      c.sum_hi_pos[c.n_sum_hi++] = q;
    }
    // measured high bits in ascending position order
    for (int q = kProbChunkBits; q < n; q++)
      for (int j = 0; j < m; j++)
        if (pos[j] == q) {
          c.hi_pos[c.m_hi] = q;
          c.hi_j[c.m_hi++] = j;
        }
    c.n_chunks = 1ll << (n - kProbChunkBits);
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * (size_t)nb, s);
    if (e != cudaSuccess) return e;
    // one wave of resident CTAs
    const int occ = c128 ? resident_ctas((const void *)k_probs_chunk<double2>, 256, 0)
                         : resident_ctas((const void *)k_probs_chunk<float2>, 256, 0);
    long long grid = (long long)dev_info().sms * occ;
    if (grid > c.n_chunks) grid = c.n_chunks;
    if (c128) k_probs_chunk<double2><<<(int)grid, 256, 0, s>>>((const double2 *)amps, c, out);
    else k_probs_chunk<float2><<<(int)grid, 256, 0, s>>>((const float2 *)amps, c, out);
    return cudaGetLastError();
  }
  const int grid = grid_for(nb, 256);
  if (c128) k_probs_wide<double2><<<grid, 256, 0, s>>>((const double2 *)amps, p, n, out);
  else k_probs_wide<float2><<<grid, 256, 0, s>>>((const float2 *)amps, p, n, out);
  return cudaGetLastError();
}

}  // namespace qs

// ---------------------------------------------------------------------------
// Marginal probabilities without any allocation
// ---------------------------------------------------------------------------
// Some callers cannot let a library call cudaMalloc: a serving process that
// reserved all of its device memory up front through its own pool, or a
// caller that must not risk the device-wide synchronisation cudaMalloc and
// cudaFree may imply. For them, states of fewer than 12 qubits keep the
// per-CTA partial histograms of the probability reduction in this fixed
// array instead of state-owned scratch (at most 8 CTAs x 2^11 bins); larger
// states take the chunked kernel, which accumulates with FP64 atomics
// straight into the caller's output after zeroing it and needs no scratch
// (the per-CTA kernel ran 25-30x slower than it on a 30-qubit state on
// GB300). Every GPU that loads the library keeps these 128 KiB until exit.
namespace qs {
std::string &last_error_ref();
}

namespace {

constexpr int kNoAllocScratchDoubles = 1 << 14;  // 128 KiB
static __device__ __align__(256) double g_probs_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

qs_status noalloc_fail(qs_status s, const char *msg) {
  qs::last_error_ref() = msg;
  return s;
}

}  // namespace

extern "C" qs_status qs_probs_noalloc(const void *dev_amps, int n, qs_dtype dtype, const int *phys_bits, int m,
                                      double *dev_out, void *cuda_stream) {
  using namespace qs;
  using namespace qs::kern;
  if (!dev_amps || !dev_out || (m > 0 && !phys_bits))
    return noalloc_fail(QS_EINVAL, "qs_probs_noalloc: null argument");
  if (dtype != QS_C64 && dtype != QS_C128) return noalloc_fail(QS_EINVAL, "qs_probs_noalloc: unknown dtype");
  const int nmax = dtype == QS_C64 ? QS_MAX_N_C64 : QS_MAX_N_C128;
  if (n < 1 || n > nmax) return noalloc_fail(QS_EINVAL, "qs_probs_noalloc: qubit count out of range");
  if (m < 0 || m > n || m > kMaxProbBits)
    return noalloc_fail(QS_EINVAL, "qs_probs_noalloc: m must be in 0..min(n, 26)");
  if (((uintptr_t)dev_amps & 15) != 0 || ((uintptr_t)dev_out & 7) != 0)
    return noalloc_fail(QS_EINVAL, "qs_probs_noalloc: misaligned device pointer");
  int pos[kMaxProbBits];
  for (int j = 0; j < m; j++) {
    if (phys_bits[j] < 0 || phys_bits[j] >= n) return noalloc_fail(QS_EINVAL, "qs_probs_noalloc: bit out of range");
    for (int i = 0; i < j; i++)
      if (phys_bits[i] == phys_bits[j]) return noalloc_fail(QS_EINVAL, "qs_probs_noalloc: duplicate bit");
    pos[j] = phys_bits[j];
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(QS_ECUDA, "qs_probs_noalloc: cudaGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(QS_EUNSUPPORTED, "qs_probs_noalloc: device ordinal too large");
  double *scratch = nullptr;
  {
    // first call on this device: resolve the array's device address once,
    // with the device current (the host-side name is only a stand-in)
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      void *addr = nullptr;
      e = cudaGetSymbolAddress(&addr, g_probs_scratch);
      if (e != cudaSuccess || !addr) return noalloc_fail(QS_ECUDA, "qs_probs_noalloc: cudaGetSymbolAddress failed");
      g_scratch_ptr[dev] = (double *)addr;
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (n >= kProbChunkBits) {
    // the chunked kernel: zeroes dev_out (an asynchronous memset, no
    // allocation), then FP64 atomics into it; no scratch
    e = launch_probs(dev_amps, n, dtype == QS_C128, pos, m, nullptr, dev_out, s);
    if (e != cudaSuccess) return noalloc_fail(QS_ECUDA, "qs_probs_noalloc: launch failed");
    return QS_OK;
  }
  ProbsParam p;
  p.n_amps = 1ll << n;
  p.m = m;
  for (int j = 0; j < m; j++) p.pos[j] = pos[j];
  // every partial slot the reduce kernel reads is written by this call, so
  // nothing in the array has to start at zero (at most 8 CTAs x 2^11 bins
  // below 12 qubits; the cap only guards the array's bounds)
  int grid = probs_grid(n);
  const int cap = kNoAllocScratchDoubles >> m;
  if (grid > cap) grid = cap;
  const size_t smem = sizeof(double) << m;
  if (dtype == QS_C128) k_probs<double2><<<grid, 256, smem, s>>>((const double2 *)dev_amps, p, scratch);
  else k_probs<float2><<<grid, 256, smem, s>>>((const float2 *)dev_amps, p, scratch);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    const int nb = 1 << m;
    k_probs_reduce<<<(nb + 255) / 256, 256, 0, s>>>(scratch, grid, nb, dev_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return noalloc_fail(QS_ECUDA, "qs_probs_noalloc: launch failed");
  return QS_OK;
}
