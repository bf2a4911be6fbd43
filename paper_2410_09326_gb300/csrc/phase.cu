// Diagonal runs of any width as phase polynomials (BK_PHASE).
//
// Every diagonal gate of the IR (T, S, Z, RZ, U1, CPhase, CZ, CRZ, RZZ, ...)
// acts on at most two qubits, so any run of them multiplies amplitude x by
// exp(i phi(x)) with phi a quadratic polynomial in the bits of x: a constant,
// one angle per qubit and one per qubit pair. The kernel needs no 2^k table
// (so the run may span all n qubits, e.g. the controlled-phase ladders of a
// QFT, where the paper notes CPhase gates on slow qubits are costly, Sec.
// IV-C) and stays one read and one write of the state:
//   the state is cut into chunks of 2^10 contiguous amplitudes (bits 0..9 of
//   the index vary inside a chunk, the rest are fixed). Terms among bits
//   0..9 form a 1024-entry factor table L (built on the host in FP64). For a
//   chunk, every term touching a higher bit either is a chunk-wide factor
//   (all its bits above 9) or multiplies by exp(i b) exactly when one chunk
//   bit s is 1 (a pair of bit s and a higher bit that is set in the chunk):
//   one warp folds those into E_0..E_9 and a chunk factor C, then
//     w(o) = L[o] * C * prod_{s < 5, o_s = 1} E_s * prod_{5 <= s < 10, o_s = 1} E_s
//   where the first product depends only on the lane (each lane reads fixed
//   offsets mod 32) and the second one on the load step (shared across the
//   warp by shuffles).
#include <algorithm>
#include <cstring>

#include "kernels_common.cuh"

namespace qs {
namespace kern {

namespace {

constexpr int kPhaseThreads = 256;
constexpr int kPhaseChunkBits = 10;
constexpr int kPhaseSlots = kPhaseChunkBits + 1;  // E_0..E_9, then C

struct PhaseHdr {
  int off[kPhaseSlots + 1];  // terms of slot s: [off[s], off[s + 1])
  int pad[4];
};
static_assert(sizeof(PhaseHdr) % 16 == 0, "header alignment");

template <typename T> struct alignas(16) PhaseTerm {
  unsigned long long mask;  // bits that must all be set in the chunk base
  unsigned long long pad;
  T f;                      // factor exp(i angle)
};

template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  T r;
  r.x = fma(a.x, b.x, -a.y * b.y);
  r.y = fma(a.x, b.y, a.y * b.x);
  return r;
}

template <typename T>
__global__ void __launch_bounds__(kPhaseThreads) k_phase(T *__restrict__ a, const unsigned char *__restrict__ desc,
                                                         long long n_chunks) {
  extern __shared__ __align__(16) unsigned char smem[];
  using Term = PhaseTerm<T>;
  const PhaseHdr *hdr = reinterpret_cast<const PhaseHdr *>(desc);
  __shared__ int off[kPhaseSlots + 1];
  if (threadIdx.x <= kPhaseSlots) off[threadIdx.x] = hdr->off[threadIdx.x];
  T *ltab = reinterpret_cast<T *>(smem);
  const Term *terms = reinterpret_cast<const Term *>(ltab + (1 << kPhaseChunkBits));
  {
    const int nt = hdr->off[kPhaseSlots];
    const int words = (int)(((sizeof(T) << kPhaseChunkBits) + nt * sizeof(Term)) / 16);
    const uint4 *src = reinterpret_cast<const uint4 *>(desc + sizeof(PhaseHdr));
    uint4 *dst = reinterpret_cast<uint4 *>(smem);
    for (int i = threadIdx.x; i < words; i += kPhaseThreads) dst[i] = src[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (kPhaseThreads / 32);
  for (long long c = ((long long)blockIdx.x * kPhaseThreads + threadIdx.x) >> 5; c < n_chunks; c += nwarps) {
    const uint64_t cbase = (uint64_t)c << kPhaseChunkBits;
    T *chunk = a + cbase;
    // complex64: the chunk's loads go out first, so that they are in flight
    // while the warp folds the chunk's terms (which depend on cbase only).
    // Staging each warp's next chunk in shared memory by cp.async instead
    // (8 KB per warp, 122 registers) measured 8% slower on GB300.
    float4 v4[sizeof(T) == 8 ? 16 : 1];
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int it = 0; it < 16; it++) v4[it] = *reinterpret_cast<const float4 *>(chunk + 2 * lane + 64 * it);
    }
    // the warp folds the terms together: lane l takes terms l, l + 32, ...
    // of each slot, then a butterfly over the lanes multiplies the partial
    // products (every lane ends with the whole product)
    T e[kPhaseSlots];
#pragma unroll
    for (int s = 0; s < kPhaseSlots; s++) {
      T acc;
      acc.x = 1;
      acc.y = 0;
      for (int t = off[s] + lane; t < off[s + 1]; t += 32) {
        const unsigned long long mk = terms[t].mask;
        if ((cbase & mk) == mk) acc = cmul(acc, terms[t].f);
      }
      e[s] = acc;
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
#pragma unroll
      for (int s = 0; s < kPhaseSlots; s++) {
        T o;
        o.x = __shfl_xor_sync(0xffffffffu, e[s].x, d);
        o.y = __shfl_xor_sync(0xffffffffu, e[s].y, d);
        e[s] = cmul(e[s], o);
      }
    }
    // second factor: lane l holds the one for bits 5..9 equal to l
    T fb;
    fb.x = 1;
    fb.y = 0;
#pragma unroll
    for (int i = 0; i < 5; i++)
      if ((lane >> i) & 1) fb = cmul(fb, e[5 + i]);
    if constexpr (sizeof(T) == 8) {
      // lane reads offsets 2 lane + 64 it (+1): bits 0..4 are (2 lane) mod 32
      // (+1), bits 5..9 are (lane >> 4) + 2 it
      T fa0 = e[kPhaseChunkBits];
#pragma unroll
      for (int i = 1; i < 5; i++)
        if (((2 * lane) >> i) & 1) fa0 = cmul(fa0, e[i]);
      const T fa1 = cmul(fa0, e[0]);
      const float4 *v = v4;
#pragma unroll
      for (int it = 0; it < 16; it++) {
        const int src = (lane >> 4) + 2 * it;
        T g;
        g.x = __shfl_sync(0xffffffffu, fb.x, src);
        g.y = __shfl_sync(0xffffffffu, fb.y, src);
        const int o = 2 * lane + 64 * it;
        // the two table entries of this lane's pair in one 16-byte load
        const float4 lt = *reinterpret_cast<const float4 *>(ltab + o);
        const T w0 = cmul(cmul(make_float2(lt.x, lt.y), fa0), g), w1 = cmul(cmul(make_float2(lt.z, lt.w), fa1), g);
        float4 y;
        y.x = fmaf(w0.x, v[it].x, -w0.y * v[it].y);
        y.y = fmaf(w0.x, v[it].y, w0.y * v[it].x);
        y.z = fmaf(w1.x, v[it].z, -w1.y * v[it].w);
        y.w = fmaf(w1.x, v[it].w, w1.y * v[it].z);
        *reinterpret_cast<float4 *>(chunk + 2 * lane + 64 * it) = y;
      }
    } else {
      // lane reads offsets lane + 32 it: bits 0..4 are the lane, bits 5..9 are it
      T fa = e[kPhaseChunkBits];
#pragma unroll
      for (int i = 0; i < 5; i++)
        if ((lane >> i) & 1) fa = cmul(fa, e[i]);
#pragma unroll
      for (int half = 0; half < 2; half++) {
        T v[16];
#pragma unroll
        for (int it = 0; it < 16; it++) v[it] = chunk[lane + 32 * (16 * half + it)];
#pragma unroll
        for (int it = 0; it < 16; it++) {
          const int step = 16 * half + it;
          T g;
          g.x = __shfl_sync(0xffffffffu, fb.x, step);
          g.y = __shfl_sync(0xffffffffu, fb.y, step);
          const int o = lane + 32 * step;
          chunk[o] = cmul(cmul(cmul(ltab[o], fa), g), v[it]);
        }
      }
    }
  }
}

template <typename T> struct PhaseLayout {
  std::vector<int> slot;
  std::vector<unsigned long long> mask;
  std::vector<double> angle;
};

// Terms of the block that touch bits above the chunk, by slot.
template <typename T> void collect_terms(const Block &b, PhaseLayout<T> &L) {
  const int k = b.k;
  auto add = [&](int s, unsigned long long m, double ang) {
    if (ang == 0.0) return;
    L.slot.push_back(s);
    L.mask.push_back(m);
    L.angle.push_back(ang);
  };
  for (int j = 0; j < k; j++)
    if (b.ph_q[j] >= kPhaseChunkBits) add(kPhaseChunkBits, 1ull << b.ph_q[j], b.ph_a[j]);
  for (int j = 0; j < k; j++)
    for (int l = j + 1; l < k; l++) {
      const int qj = b.ph_q[j], ql = b.ph_q[l];  // qj < ql
      const double ang = b.ph_b[tri_index(j, l, k)];
      if (ql < kPhaseChunkBits) continue;  // in the table
      if (qj < kPhaseChunkBits) add(qj, 1ull << ql, ang);
      else add(kPhaseChunkBits, (1ull << qj) | (1ull << ql), ang);
    }
}

template <typename T> size_t desc_bytes_t(const Block &b) {
  PhaseLayout<T> L;
  collect_terms(b, L);
  return sizeof(PhaseHdr) + (sizeof(T) << kPhaseChunkBits) + L.slot.size() * sizeof(PhaseTerm<T>);
}

template <typename T> void fill_desc_t(const Block &b, unsigned char *out) {
  using R = typename Real<T>::type;
  PhaseLayout<T> L;
  collect_terms(b, L);
  std::memset(out, 0, desc_bytes_t<T>(b));
  PhaseHdr *h = reinterpret_cast<PhaseHdr *>(out);
  T *ltab = reinterpret_cast<T *>(out + sizeof(PhaseHdr));
  PhaseTerm<T> *terms = reinterpret_cast<PhaseTerm<T> *>(ltab + (1 << kPhaseChunkBits));
  // table of the terms among chunk bits (constant included), in FP64
  const int k = b.k;
  for (int o = 0; o < (1 << kPhaseChunkBits); o++) {
    double ang = b.ph_c;
    for (int j = 0; j < k; j++) {
      const int qj = b.ph_q[j];
      if (qj >= kPhaseChunkBits || !((o >> qj) & 1)) continue;
      ang += b.ph_a[j];
      for (int l = j + 1; l < k; l++) {
        const int ql = b.ph_q[l];
        if (ql < kPhaseChunkBits && ((o >> ql) & 1)) ang += b.ph_b[tri_index(j, l, k)];
      }
    }
    ltab[o].x = (R)std::cos(ang);
    ltab[o].y = (R)std::sin(ang);
  }
  // counting sort by slot
  int cnt[kPhaseSlots] = {0};
  for (int s : L.slot) cnt[s]++;
  h->off[0] = 0;
  for (int s = 0; s < kPhaseSlots; s++) h->off[s + 1] = h->off[s] + cnt[s];
  int pos[kPhaseSlots];
  for (int s = 0; s < kPhaseSlots; s++) pos[s] = h->off[s];
  for (size_t i = 0; i < L.slot.size(); i++) {
    PhaseTerm<T> &t = terms[pos[L.slot[i]]++];
    t.mask = L.mask[i];
    t.f.x = (R)std::cos(L.angle[i]);
    t.f.y = (R)std::sin(L.angle[i]);
  }
}

template <typename T> cudaError_t run_phase_t(T *a, int n, const Block &b, const void *dev_desc, size_t desc_bytes,
                                              cudaStream_t s, LaunchShape *shape) {
  const size_t smem = desc_bytes - sizeof(PhaseHdr);
  static thread_local int configured = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    int maxs = 0;
    cudaDeviceGetAttribute(&maxs, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_phase<T>);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_phase<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    configured = dev;
  }
  const long long n_chunks = 1ll << (n - kPhaseChunkBits);
  const long long warps = (long long)dev_info().sms * resident_ctas((const void *)k_phase<T>, kPhaseThreads, smem) *
                          (kPhaseThreads / 32);
  long long grid = (std::min(warps, n_chunks) + kPhaseThreads / 32 - 1) / (kPhaseThreads / 32);
  if (b.tc_max_ctas > 0 && grid > b.tc_max_ctas) grid = b.tc_max_ctas;  // test hook: several chunks per warp
  if (grid < 1) grid = 1;
  if (shape) {
    shape->tiles = n_chunks;  // chunks of 1024 amplitudes, one warp each at a time
    shape->ctas = (int)grid;
  }
  k_phase<T><<<(int)grid, kPhaseThreads, smem, s>>>(a, (const unsigned char *)dev_desc, n_chunks);
  return cudaGetLastError();
}

}  // namespace

size_t phase_desc_bytes(const Block &b, bool c128) {
  return c128 ? desc_bytes_t<double2>(b) : desc_bytes_t<float2>(b);
}

void phase_fill_desc(const Block &b, bool c128, void *out) {
  if (c128) fill_desc_t<double2>(b, (unsigned char *)out);
  else fill_desc_t<float2>(b, (unsigned char *)out);
}

cudaError_t run_phase(void *a, int n, bool c128, const Block &b, const void *dev_desc, cudaStream_t s,
                      LaunchShape *shape) {
  if (!dev_desc || n <= kPhaseChunkBits) return cudaErrorInvalidValue;
  const size_t bytes = phase_desc_bytes(b, c128);
  if (c128) return run_phase_t<double2>((double2 *)a, n, b, dev_desc, bytes, s, shape);
  return run_phase_t<float2>((float2 *)a, n, b, dev_desc, bytes, s, shape);
}

}  // namespace kern
}  // namespace qs
