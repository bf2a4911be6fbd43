// Fused blocks with low targets on the CUDA cores (complex64, 1..3 targets,
// bit 0 free and at most one free bit among bits 0..3, i.e. targets 1, 2, 3):
// warp-wide loads and shuffles.
//
// A warp owns 64 consecutive amplitudes per load (lane l holds amplitudes
// 2l and 2l + 1 in one 16-byte access, so every load instruction of the warp
// reads 512 contiguous bytes), times 2^R such spans at the offsets of R
// further bits: the targets above bit 5 and, for every target t in bits
// 1..5, one free bit f above bit 5. A target t in the lane bits is then
// swapped with its free bit f across the warp -- lanes that differ in lane
// bit t - 1 exchange the halves of their registers that differ in f (one
// __shfl_xor_sync per value) -- after which every lane holds whole groups in
// registers: the mat-vec runs on them with the matrix as constant-bank
// operands (its rows and columns reordered on the host to the register
// order), the swaps are undone and the warp stores as it loaded.
#include <cstring>

#include "kernels_common.cuh"

namespace qs {
namespace kern {

namespace {

template <int K> struct ShflParam {
  float2 m[1 << (2 * K)];     // matrix in register order (row-major)
  long long n_items;          // warp work items
  unsigned long long cmask;   // controls (all above bit 5)
  int nf;                     // fixed bits of the item index: 0..5, the R bits, the controls
  int fixed[kMaxFixed];
  int nswap;                  // targets among bits 1..5
  int lane_bit[3];            // lane bit (target - 1) of swap i; swap i pairs it with register bit i
  unsigned long long roff[3]; // address offset of register bit j (1 << its bit)
};

template <int K, bool T0>
__global__ void __launch_bounds__(256, 2) k_dense_shfl(float2 *__restrict__ a, const __grid_constant__ ShflParam<K> p) {
  constexpr int R = T0 ? K - 1 : K;   // register index bits
  constexpr int NV = 1 << R;          // 16-byte loads per lane
  constexpr int D = 1 << K;
  const int lane = threadIdx.x & 31;
  uint64_t off[NV];
#pragma unroll
  for (int r = 0; r < NV; r++) {
    uint64_t o = (uint64_t)lane << 1;
#pragma unroll
    for (int j = 0; j < R; j++)
      if ((r >> j) & 1) o += p.roff[j];
    off[r] = o;
  }
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long it = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < p.n_items; it += warps) {
    const uint64_t base = insert_zeros((uint64_t)it, p.fixed, p.nf) | p.cmask;
    float4 v[NV];
#pragma unroll
    for (int r = 0; r < NV; r++) v[r] = *reinterpret_cast<const float4 *>(a + base + off[r]);
    auto swaps = [&]() {
#pragma unroll
      for (int i = 0; i < R; i++) {
        if (i >= p.nswap) break;
        const int lb = p.lane_bit[i];
        const bool up = (lane >> lb) & 1;
#pragma unroll
        for (int r = 0; r < NV; r++) {
          if ((r >> i) & 1) continue;
          const int r2 = r | (1 << i);
          float4 send = up ? v[r] : v[r2];
          float4 recv;
          recv.x = __shfl_xor_sync(0xffffffffu, send.x, 1 << lb);
          recv.y = __shfl_xor_sync(0xffffffffu, send.y, 1 << lb);
          recv.z = __shfl_xor_sync(0xffffffffu, send.z, 1 << lb);
          recv.w = __shfl_xor_sync(0xffffffffu, send.w, 1 << lb);
          if (up) v[r] = recv;
          else v[r2] = recv;
        }
      }
    };
    swaps();
    // register order: amplitude rho = (bit 0 of the 16-byte access) | (r << 1)
    auto get = [&](int rho) {
      const float4 &x = v[rho >> 1];
      return (rho & 1) ? make_float2(x.z, x.w) : make_float2(x.x, x.y);
    };
    auto put = [&](int rho, float2 y) {
      float4 &x = v[rho >> 1];
      if (rho & 1) {
        x.z = y.x;
        x.w = y.y;
      } else {
        x.x = y.x;
        x.y = y.y;
      }
    };
    constexpr int G = T0 ? 1 : 2;  // groups per lane: bit 0 free -> two
#pragma unroll
    for (int g = 0; g < G; g++) {
      float2 in[D];
#pragma unroll
      for (int s = 0; s < D; s++) in[s] = get(T0 ? s : (g | (s << 1)));
#pragma unroll
      for (int row = 0; row < D; row++) {
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int c = 0; c < D; c++) {
          const float2 w = p.m[row * D + c];
          re = fmaf(w.x, in[c].x, re);
          re = fmaf(-w.y, in[c].y, re);
          im = fmaf(w.x, in[c].y, im);
          im = fmaf(w.y, in[c].x, im);
        }
        put(T0 ? row : (g | (row << 1)), make_float2(re, im));
      }
    }
    // the swaps are involutions: applying them again (same order is fine,
    // they act on disjoint bit pairs) restores the load layout
    swaps();
#pragma unroll
    for (int r = 0; r < NV; r++) *reinterpret_cast<float4 *>(a + base + off[r]) = v[r];
  }
}

template <int K, bool T0>
cudaError_t launch_shfl(float2 *a, const ShflParam<K> &p, cudaStream_t s) {
  const long long want = (p.n_items + 7) / 8;  // 8 warps per CTA
  long long cap = (long long)dev_info().sms * 2 * 4;
  long long grid = want < cap ? want : cap;
  if (grid < 1) grid = 1;
  k_dense_shfl<K, T0><<<(int)grid, 256, 0, s>>>(a, p);
  return cudaGetLastError();
}

template <int K> cudaError_t run_shfl_k(float2 *a, int n, const Block &b, cudaStream_t s, bool &used) {
  used = false;
  // targets in the warp's 6 low bits, others; controls must lie above bit 5
  if (b.cmask & 63ull) return cudaSuccess;
  bool t0 = false;
  int lane_t[6], nl = 0, hi_t[6], nh = 0;
  uint64_t tmask = 0;
  for (int j = 0; j < K; j++) {
    const int q = b.q[j];
    tmask |= 1ull << q;
    if (q == 0) t0 = true;
    else if (q <= 5) lane_t[nl++] = q;
    else hi_t[nh++] = q;
  }
  if (nl == 0) return cudaSuccess;
  // Only where the thread-per-group kernel reads badly: without bit 0 as a
  // target its lanes step through the lowest free bits, and with at most one
  // free bit among bits 0..3 a warp's load touches 16 lines for 256 bytes
  // (targets 1, 2, 3: 4.4 TB/s there, 5.7 TB/s here); with two or more free
  // low bits, or bit 0 a target (16-byte pairs), it reads at 6.2-6.6 TB/s and
  // stays faster than the shuffles (5.7-6.2 TB/s on GB300).
  if (t0 || __builtin_popcountll(~tmask & 15ull) > 1) return cudaSuccess;
  // one free bit above bit 5 per lane target
  int freeb[6], nfree = 0;
  for (int q = 6; q < n && nfree < nl; q++)
    if (!((tmask | b.cmask) >> q & 1)) freeb[nfree++] = q;
  if (nfree < nl) return cudaSuccess;
  static thread_local ShflParam<K> p;
  std::memset(&p, 0, sizeof(p));
  // register bits: the free partners first (swap i pairs lane target i with
  // register bit i), then the high targets
  int rbit_addr[6], rb = 0;
  for (int i = 0; i < nl; i++) rbit_addr[rb++] = freeb[i];
  for (int i = 0; i < nh; i++) rbit_addr[rb++] = hi_t[i];
  const int R = rb;  // = K - t0
  for (int j = 0; j < R; j++) p.roff[j] = 1ull << rbit_addr[j];
  p.nswap = nl;
  for (int i = 0; i < nl; i++) p.lane_bit[i] = lane_t[i] - 1;
  // after the swaps, register bit j carries: lane target j (j < nl) or
  // high target j - nl; register order index s' -> address bit of each bit
  int sbit_addr[8], ns = 0;
  if (t0) sbit_addr[ns++] = 0;
  for (int j = 0; j < R; j++) sbit_addr[ns++] = j < nl ? lane_t[j] : rbit_addr[j];
  // s' bit -> position in the block's ascending target list (matrix index)
  int sbit_mat[8];
  for (int j = 0; j < ns; j++)
    for (int t = 0; t < K; t++)
      if (b.q[t] == sbit_addr[j]) sbit_mat[j] = t;
  constexpr int D = 1 << K;
  auto to_mat = [&](int sp) {
    int sidx = 0;
    for (int j = 0; j < K; j++)
      if ((sp >> j) & 1) sidx |= 1 << sbit_mat[j];
    return sidx;
  };
  for (int r = 0; r < D; r++)
    for (int c = 0; c < D; c++) p.m[r * D + c] = to_dev<float2>(b.mat[(size_t)to_mat(r) * D + to_mat(c)]);
  // item index: every bit except 0..5, the register bits and the controls
  uint64_t fixedm = 63ull | b.cmask;
  for (int j = 0; j < R; j++) fixedm |= 1ull << rbit_addr[j];
  if (__builtin_popcountll(fixedm) > kMaxFixed || (fixedm >> n) != 0) return cudaSuccess;
  p.nf = 0;
  for (int q = 0; q < n; q++)
    if ((fixedm >> q) & 1) p.fixed[p.nf++] = q;
  p.n_items = 1ll << (n - p.nf);
  p.cmask = b.cmask;
  used = true;
  return t0 ? launch_shfl<K, true>(a, p, s) : launch_shfl<K, false>(a, p, s);
}

}  // namespace

cudaError_t run_dense_shfl_c64(float2 *a, int n, const Block &b, cudaStream_t s, bool &used) {
  used = false;
  if (n < 9) return cudaSuccess;
  switch (b.k) {
    case 1: return run_shfl_k<1>(a, n, b, s, used);
    case 2: return run_shfl_k<2>(a, n, b, s, used);
    case 3: return run_shfl_k<3>(a, n, b, s, used);
    default: return cudaSuccess;
  }
}

}  // namespace kern
}  // namespace qs
