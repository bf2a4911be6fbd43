// Cache-blocked passes (QS_TILE): several member blocks in one HBM pass.
//
// The chunk segment of the paper's simulator (Sec. III-D: amplitudes whose
// qubits are "fast" stay in the buffer while a run of gates is applied to
// them) becomes, on the GPU, a tile of 2^m amplitudes in shared memory: the
// tile spans m physical qubits (bits 0..kTileLowBits-1, so every load reads
// contiguous runs of at least 128 bytes, plus m - kTileLowBits others chosen
// by the planner) and one tile exists for every value of the other n - m bits.
// Each CTA takes tiles from a grid-stride loop; per tile it
//   1. gathers the 2^m amplitudes into shared memory (16-byte cp.async),
//   2. applies every member block in order -- a dense block (<= 4 targets,
//      all inside the tile) as a group mat-vec per thread, a diagonal block
//      (any qubits) as one phase per amplitude, where table qubits outside the
//      tile are constant for the tile; controls outside the tile decide, for
//      the whole tile, whether a member runs at all,
//   3. scatters the tile back.
// Member matrices, phase tables and descriptors are staged in shared memory
// once per CTA.
#include <cstring>

#include "kernels_common.cuh"

namespace qs {
namespace kern {

namespace {

constexpr int kTileThreads = 256;

struct TileHdr {
  int m;          // tile qubits
  int n_ops;      // member blocks
  int pool_len;   // matrix / phase entries (amplitude type), a multiple of 2
  int pad;
  int tile_q[16]; // physical positions ascending; tile_q[j] = j for j < kTileLowBits
};

struct TileOp {
  int kind;                   // 0 dense, 1 diagonal
  int k;                      // dense targets / table qubits
  int nf;                     // local fixed positions (dense: targets + local controls; diagonal: local controls)
  int pool_off;               // first entry of the matrix / table in the pool
  unsigned long long gcmask;  // control bits outside the tile (physical)
  unsigned lcmask;            // control bits inside the tile (local positions)
  int pad;
  int fixed[16];              // local positions, ascending
  int tq[QS_MAX_DIAG];        // dense: local target positions; diagonal: local position of table bit j,
                              // or -1 - physical position when it lies outside the tile
  int pad2[2];
};
static_assert(sizeof(TileHdr) % 16 == 0, "header alignment");
static_assert(sizeof(TileOp) % 16 == 0, "descriptor alignment");

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T, int K>
__device__ __forceinline__ void tile_dense(T *tile, int m, const TileOp &op, const T *mat) {
  constexpr int D = 1 << K;
  uint64_t d[K];
#pragma unroll
  for (int j = 0; j < K; j++) d[j] = 1ull << op.tq[j];
  const int groups = 1 << (m - op.nf);
  if constexpr (K <= 2) {
    // the whole matrix in registers for the op
    T mr[D * D];
#pragma unroll
    for (int i = 0; i < D * D; i++) mr[i] = mat[i];
    if (sizeof(T) == 8 && op.tq[0] == 0) {
      for (int g = threadIdx.x; g < groups; g += kTileThreads) {
        const uint64_t base = insert_zeros((uint64_t)g, op.fixed, op.nf) | op.lcmask;
        group_apply<T, K, sizeof(T) == 8>(tile, base, d, mr);
      }
    } else {
      for (int g = threadIdx.x; g < groups; g += kTileThreads) {
        const uint64_t base = insert_zeros((uint64_t)g, op.fixed, op.nf) | op.lcmask;
        group_apply<T, K>(tile, base, d, mr);
      }
    }
  } else {
    if (sizeof(T) == 8 && op.tq[0] == 0) {
      for (int g = threadIdx.x; g < groups; g += kTileThreads) {
        const uint64_t base = insert_zeros((uint64_t)g, op.fixed, op.nf) | op.lcmask;
        group_apply<T, K, sizeof(T) == 8>(tile, base, d, mat);
      }
    } else {
      for (int g = threadIdx.x; g < groups; g += kTileThreads) {
        const uint64_t base = insert_zeros((uint64_t)g, op.fixed, op.nf) | op.lcmask;
        group_apply<T, K>(tile, base, d, mat);
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void tile_diag(T *tile, int m, const TileOp &op, const T *tab, uint64_t tbase) {
  using R = typename Real<T>::type;
  int lhi = 0;  // table bits outside the tile: fixed for this tile
  for (int j = 0; j < op.k; j++)
    if (op.tq[j] < 0) lhi |= (int)((tbase >> (-1 - op.tq[j])) & 1) << j;
  const int amps = 1 << (m - op.nf);
  for (int j = threadIdx.x; j < amps; j += kTileThreads) {
    const uint32_t e = (uint32_t)insert_zeros((uint64_t)j, op.fixed, op.nf) | op.lcmask;
    int l = lhi;
    for (int b = 0; b < op.k; b++)
      if (op.tq[b] >= 0) l |= (int)((e >> op.tq[b]) & 1) << b;
    const T w = tab[l];
    const T v = tile[e];
    T y;
    y.x = fma((R)w.x, v.x, -(R)w.y * v.y);
    y.y = fma((R)w.x, v.y, (R)w.y * v.x);
    tile[e] = y;
  }
}

template <typename T>
__global__ void __launch_bounds__(kTileThreads) k_tile(T *__restrict__ a, const unsigned char *__restrict__ desc,
                                                       long long n_tiles) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int PER = 16 / (int)sizeof(T);  // amplitudes per 16-byte copy
  const TileHdr *hdr = reinterpret_cast<const TileHdr *>(desc);
  const int m = hdr->m, n_ops = hdr->n_ops, pool_len = hdr->pool_len;
  const int tsize = 1 << m;
  T *tile = reinterpret_cast<T *>(smem);
  T *pool = tile + tsize;
  TileOp *ops = reinterpret_cast<TileOp *>(pool + pool_len);
  uint64_t *dep = reinterpret_cast<uint64_t *>(ops + n_ops);
  __shared__ int tq[16];
  if (threadIdx.x < 16) tq[threadIdx.x] = hdr->tile_q[threadIdx.x];
  {
    // pool and descriptors follow the header contiguously in both places
    const uint4 *src = reinterpret_cast<const uint4 *>(desc + sizeof(TileHdr));
    uint4 *dst = reinterpret_cast<uint4 *>(pool);
    const int words = (int)((pool_len * sizeof(T) + n_ops * sizeof(TileOp)) / 16);
    for (int i = threadIdx.x; i < words; i += kTileThreads) dst[i] = src[i];
  }
  __syncthreads();
  // offset of every run of 2^kTileLowBits contiguous amplitudes in the tile
  const int nhi = m - kTileLowBits;
  for (int h = threadIdx.x; h < (1 << nhi); h += kTileThreads) {
    uint64_t off = 0;
    for (int j = 0; j < nhi; j++) off |= (uint64_t)((h >> j) & 1) << tq[kTileLowBits + j];
    dep[h] = off;
  }
  __syncthreads();
  constexpr uint32_t lowmask = (1u << kTileLowBits) - 1;
  for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const uint64_t tbase = insert_zeros((uint64_t)t, tq, m);
    for (int i = threadIdx.x; i < tsize / PER; i += kTileThreads) {
      const uint32_t e = (uint32_t)i * PER;
      cp_async16(tile + e, a + tbase + dep[e >> kTileLowBits] + (e & lowmask));
    }
    cp_async_wait_all();
    __syncthreads();
    for (int o = 0; o < n_ops; o++) {
      const TileOp &op = ops[o];
      if ((tbase & op.gcmask) != op.gcmask) continue;  // same for the whole CTA
      const T *mat = pool + op.pool_off;
      if (op.kind == 1) {
        tile_diag<T>(tile, m, op, mat, tbase);
      } else {
        switch (op.k) {
          case 1: tile_dense<T, 1>(tile, m, op, mat); break;
          case 2: tile_dense<T, 2>(tile, m, op, mat); break;
          case 3: tile_dense<T, 3>(tile, m, op, mat); break;
          case 4: tile_dense<T, 4>(tile, m, op, mat); break;
          default: break;
        }
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < tsize / PER; i += kTileThreads) {
      const uint32_t e = (uint32_t)i * PER;
      *reinterpret_cast<uint4 *>(a + tbase + dep[e >> kTileLowBits] + (e & lowmask)) =
          *reinterpret_cast<const uint4 *>(tile + e);
    }
    __syncthreads();
  }
}

template <typename T> size_t pool_entries(const Block &b) {
  size_t e = 0;
  for (const Block &s : b.sub) e += s.mat.size();
  return (e + 1) & ~(size_t)1;
}

template <typename T> size_t desc_bytes_t(const Block &b) {
  return sizeof(TileHdr) + pool_entries<T>(b) * sizeof(T) + b.sub.size() * sizeof(TileOp);
}

template <typename T> size_t smem_bytes_t(const Block &b) {
  return ((size_t)1 << b.k) * sizeof(T) + desc_bytes_t<T>(b) - sizeof(TileHdr) +
         ((size_t)1 << (b.k - kTileLowBits)) * sizeof(uint64_t);
}

int local_pos(const Block &t, int q) {
  for (int j = 0; j < t.k; j++)
    if (t.tile_q[j] == q) return j;
  return -1;
}

template <typename T> void fill_desc_t(const Block &b, unsigned char *out) {
  std::memset(out, 0, desc_bytes_t<T>(b));
  TileHdr *h = reinterpret_cast<TileHdr *>(out);
  h->m = b.k;
  h->n_ops = (int)b.sub.size();
  h->pool_len = (int)pool_entries<T>(b);
  for (int j = 0; j < b.k; j++) h->tile_q[j] = b.tile_q[j];
  T *pool = reinterpret_cast<T *>(out + sizeof(TileHdr));
  TileOp *ops = reinterpret_cast<TileOp *>(pool + h->pool_len);
  int off = 0;
  for (size_t i = 0; i < b.sub.size(); i++) {
    const Block &s = b.sub[i];
    TileOp &op = ops[i];
    op.kind = s.kind == BK_DIAG ? 1 : 0;
    op.k = s.k;
    op.pool_off = off;
    for (size_t e = 0; e < s.mat.size(); e++) pool[off + e] = to_dev<T>(s.mat[e]);
    off += (int)s.mat.size();
    uint32_t fixed_mask = 0;
    for (int q = 0; q < 64; q++) {
      if (!((s.cmask >> q) & 1)) continue;
      const int lp = local_pos(b, q);
      if (lp >= 0) {
        op.lcmask |= 1u << lp;
        fixed_mask |= 1u << lp;
      } else {
        op.gcmask |= 1ull << q;
      }
    }
    for (int j = 0; j < s.k; j++) {
      const int lp = local_pos(b, s.q[j]);
      if (s.kind == BK_DENSE) {
        op.tq[j] = lp;  // inside the tile by construction
        fixed_mask |= 1u << lp;
      } else {
        op.tq[j] = lp >= 0 ? lp : -1 - s.q[j];
      }
    }
    op.nf = 0;
    for (int j = 0; j < b.k; j++)
      if ((fixed_mask >> j) & 1) op.fixed[op.nf++] = j;
  }
}

template <typename T> cudaError_t run_tile_t(T *a, int n, const Block &b, const void *dev_desc, cudaStream_t s) {
  const size_t smem = smem_bytes_t<T>(b);
  static thread_local int configured = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    // dynamic shared memory up to the opt-in limit minus the static part
    int maxs = 0;
    cudaDeviceGetAttribute(&maxs, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_tile<T>);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tile<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    configured = dev;
  }
  const long long n_tiles = 1ll << (n - b.k);
  long long grid = (long long)dev_info().sms * resident_ctas((const void *)k_tile<T>, kTileThreads, smem);
  if (grid > n_tiles) grid = n_tiles;
  k_tile<T><<<(int)grid, kTileThreads, smem, s>>>(a, (const unsigned char *)dev_desc, n_tiles);
  return cudaGetLastError();
}

}  // namespace

size_t tile_desc_bytes(const Block &b, bool c128) {
  return c128 ? desc_bytes_t<double2>(b) : desc_bytes_t<float2>(b);
}

size_t tile_smem_bytes(const Block &b, bool c128) {
  return c128 ? smem_bytes_t<double2>(b) : smem_bytes_t<float2>(b);
}

void tile_fill_desc(const Block &b, bool c128, void *out) {
  if (c128) fill_desc_t<double2>(b, (unsigned char *)out);
  else fill_desc_t<float2>(b, (unsigned char *)out);
}

cudaError_t run_tile(void *a, int n, bool c128, const Block &b, const void *dev_desc, cudaStream_t s) {
  if (!dev_desc || b.k < kTileLowBits + 1 || b.k > kMaxTileBits || b.k >= n) return cudaErrorInvalidValue;
  if (c128) return run_tile_t<double2>((double2 *)a, n, b, dev_desc, s);
  return run_tile_t<float2>((float2 *)a, n, b, dev_desc, s);
}

}  // namespace kern
}  // namespace qs
