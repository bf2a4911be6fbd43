// Batched simulation: many circuits of uneven width in one persistent launch,
// captured as a CUDA graph (the paper's repeated-run use case, Sec. IV-E:
// a QAOA circuit simulated again and again).
//
// Every circuit is planned on the host (virtual swap + fusion) and its blocks
// are uploaded once as descriptors plus a pool of matrices. The kernel runs
// one CTA per circuit, taken from a work queue ordered by decreasing cost
// (2^n x blocks), so CTAs never wait on one another:
//  - circuits with n <= kSmemBits live in shared memory for the whole run:
//    the CTA writes |0...0> there, applies every block in shared memory, and
//    writes the final state to the circuit's buffer once;
//  - wider circuits are reset and updated in their own global buffer (L2
//    resident for the widths of this use case), block after block.
// A block's matrix or phase table is staged in shared memory before use.
// Each run starts every circuit from |0...0>.
//
// The autotuner times candidate (fusion width, threads per CTA) pairs on the
// batch itself and keeps the fastest; the chosen launch (queue reset + kernel)
// is captured once as a CUDA graph, and qs_batch_run replays it.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "kernels_common.cuh"

namespace qs {
std::string &last_error_ref();
}

namespace qs {
namespace kern {
namespace {

constexpr int kSmemBits = 14;                        // 2^14 c64 amplitudes = 128 KiB
constexpr int kMatFloats2 = 1 << (2 * QS_MAX_FUSE);  // 64 x 64 complex entries
constexpr int kMaxBatchN = 26;

struct BBlock {
  int kind;  // 0 dense, 1 diagonal, 2 exchange
  int k;
  int nf;
  int fixed[kMaxFixed];
  int tq[QS_MAX_DIAG];
  unsigned long long cmask;
  long long mat_off;  // into the matrix pool (float2 entries)
};

struct BCircuit {
  float2 *amps;
  int n;
  int first_block;
  int n_blocks;
};

template <int K>
__device__ __forceinline__ void dense_cta(float2 *a, int n, const BBlock &b, const float2 *m) {
  uint64_t d[K];
#pragma unroll
  for (int j = 0; j < K; j++) d[j] = 1ull << b.tq[j];
  const long long groups = 1ll << (n - K - __popcll(b.cmask));
  for (long long g = threadIdx.x; g < groups; g += blockDim.x) {
    const uint64_t base = insert_zeros((uint64_t)g, b.fixed, b.nf) | b.cmask;
    group_apply<float2, K>(a, base, d, m);
  }
}

// MAXT caps the registers: the 5- and 6-target mat-vecs only exist in the
// 256-thread variant (255 registers), which the host picks for k >= 5.
template <int MAXT>
__device__ void apply_block_cta(float2 *a, int n, const BBlock &b, const float2 *m) {
  if (b.kind == 2) {
    const int fixed[2] = {b.tq[0], b.tq[1]};
    const long long pairs = 1ll << (n - 2);
    for (long long j = threadIdx.x; j < pairs; j += blockDim.x) {
      const uint64_t base = insert_zeros((uint64_t)j, fixed, 2);
      const uint64_t i0 = base | (1ull << b.tq[0]), i1 = base | (1ull << b.tq[1]);
      const float2 x = a[i0], y = a[i1];
      a[i0] = y;
      a[i1] = x;
    }
    return;
  }
  if (b.kind == 1) {
    const long long amps = 1ll << (n - __popcll(b.cmask));
    for (long long j = threadIdx.x; j < amps; j += blockDim.x) {
      const uint64_t idx = insert_zeros((uint64_t)j, b.fixed, b.nf) | b.cmask;
      int l = 0;
      for (int t = 0; t < b.k; t++) l |= (int)((idx >> b.tq[t]) & 1) << t;
      const float2 w = m[l], v = a[idx];
      a[idx] = make_float2(fmaf(w.x, v.x, -w.y * v.y), fmaf(w.x, v.y, w.y * v.x));
    }
    return;
  }
  switch (b.k) {
    case 1: dense_cta<1>(a, n, b, m); break;
    case 2: dense_cta<2>(a, n, b, m); break;
    case 3: dense_cta<3>(a, n, b, m); break;
    case 4: dense_cta<4>(a, n, b, m); break;
    case 5:
      if constexpr (MAXT <= 256) dense_cta<5>(a, n, b, m);
      break;
    case 6:
      if constexpr (MAXT <= 256) dense_cta<6>(a, n, b, m);
      break;
    default: break;
  }
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
    k_batch(const BCircuit *__restrict__ circs, const int *__restrict__ order, int count,
            const BBlock *__restrict__ blocks, const float2 *__restrict__ pool, int *__restrict__ queue) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2 *mat = reinterpret_cast<float2 *>(smem);
  float2 *st = reinterpret_cast<float2 *>(smem + sizeof(float2) * kMatFloats2);
  __shared__ int next;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(queue, 1);
    __syncthreads();
    const int c = next;
    __syncthreads();
    if (c >= count) break;
    const BCircuit C = circs[order[c]];
    const long long N = 1ll << C.n;
    float2 *a = C.n <= kSmemBits ? st : C.amps;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) a[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
    __syncthreads();
    for (int bi = 0; bi < C.n_blocks; bi++) {
      const BBlock &b = blocks[C.first_block + bi];
      const int entries = b.kind == 0 ? (1 << (2 * b.k)) : (b.kind == 1 ? (1 << b.k) : 0);
      for (int i = threadIdx.x; i < entries; i += blockDim.x) mat[i] = pool[b.mat_off + i];
      __syncthreads();
      apply_block_cta<MAXT>(a, C.n, b, mat);
      __syncthreads();
    }
    if (C.n <= kSmemBits) {
      float4 *dst = reinterpret_cast<float4 *>(C.amps);
      const float4 *src = reinterpret_cast<const float4 *>(st);
      for (long long i = threadIdx.x; i < N / 2; i += blockDim.x) dst[i] = src[i];
      if (N == 1 && threadIdx.x == 0) C.amps[0] = st[0];
      __syncthreads();
    }
  }
}

}  // namespace
}  // namespace kern
}  // namespace qs

using namespace qs;
using namespace qs::kern;

struct qs_state;
namespace qs {
// accessors into the opaque state (api.cpp)
void *state_amps(qs_state *st);
int state_n(const qs_state *st);
bool state_c64(const qs_state *st);
int8_t *state_perm(qs_state *st);
cudaStream_t state_stream(const qs_state *st);
}  // namespace qs

struct qs_batch {
  std::vector<qs_state *> states;
  std::vector<std::vector<qs_gate>> gates;
  uint64_t flags = 0;
  qs_opts opts;
  cudaStream_t stream = nullptr;
  int device = 0;
  // device data of the chosen plan
  BCircuit *d_circs = nullptr;
  int *d_order = nullptr;
  BBlock *d_blocks = nullptr;
  float2 *d_pool = nullptr;
  int *d_queue = nullptr;
  std::vector<std::vector<int8_t>> final_perm;
  int k_chosen = 0, threads = 0, grid = 0, total_blocks = 0;
  size_t smem = 0;
  double tune_ms[16] = {0};
  int tune_k[16] = {0}, tune_threads[16] = {0}, n_tune = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t own_stream = nullptr;
};

namespace {

qs_status bfail(qs_status s, const std::string &m) {
  qs::last_error_ref() = m;
  return s;
}

void free_plan(qs_batch *b) {
  qs::dev_free(b->d_circs);
  qs::dev_free(b->d_order);
  qs::dev_free(b->d_blocks);
  qs::dev_free(b->d_pool);
  b->d_circs = nullptr;
  b->d_order = nullptr;
  b->d_blocks = nullptr;
  b->d_pool = nullptr;
}

// Plans every circuit with the given flags and uploads the descriptors.
qs_status upload_plan(qs_batch *bt, uint64_t flags) {
  free_plan(bt);
  std::vector<BCircuit> circs(bt->states.size());
  std::vector<BBlock> blocks;
  std::vector<float2> pool;
  std::vector<double> cost(bt->states.size());
  bt->final_perm.assign(bt->states.size(), {});
  for (size_t c = 0; c < bt->states.size(); c++) {
    const int n = state_n(bt->states[c]);
    std::vector<Block> plan;
    PlanStats stats;
    std::string err;
    int8_t perm[QS_MAX_QUBITS];
    for (int q = 0; q < n; q++) perm[q] = (int8_t)q;
    qs_status s = build_plan(n, bt->gates[c].data(), bt->gates[c].size(), flags & ~(uint64_t)(QS_TC | QS_TILE), bt->opts,
                             perm, plan, stats, err, false, /*allow_phase=*/false);
    if (s != QS_OK) return bfail(s, "qs_batch: circuit " + std::to_string(c) + ": " + err);
    bt->final_perm[c].assign(perm, perm + n);
    circs[c].amps = (float2 *)state_amps(bt->states[c]);
    circs[c].n = n;
    circs[c].first_block = (int)blocks.size();
    circs[c].n_blocks = (int)plan.size();
    cost[c] = std::ldexp(1.0, n) * (double)(plan.size() + 1);
    for (const Block &b : plan) {
      BBlock d;
      std::memset(&d, 0, sizeof(d));
      d.kind = (int)b.kind;
      d.k = b.k;
      d.cmask = b.cmask;
      if (b.kind == BK_PERMUTE) {
        d.tq[0] = b.q[0];
        d.tq[1] = b.q[1];
      } else {
        fill_fixed(b, d.fixed, d.nf);
        for (int j = 0; j < b.k; j++) d.tq[j] = b.q[j];
      }
      d.mat_off = (long long)pool.size();
      for (const cd &z : b.mat) pool.push_back(make_float2((float)z.real(), (float)z.imag()));
      blocks.push_back(d);
    }
  }
  std::vector<int> order(circs.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  if (pool.empty()) pool.push_back(make_float2(0.f, 0.f));
  if (blocks.empty()) blocks.push_back(BBlock());
  cudaError_t e = qs::dev_malloc((void **)&bt->d_circs, sizeof(BCircuit) * circs.size());
  if (e == cudaSuccess) e = qs::dev_malloc((void **)&bt->d_order, sizeof(int) * order.size());
  if (e == cudaSuccess) e = qs::dev_malloc((void **)&bt->d_blocks, sizeof(BBlock) * blocks.size());
  if (e == cudaSuccess) e = qs::dev_malloc((void **)&bt->d_pool, sizeof(float2) * pool.size());
  if (e != cudaSuccess) return bfail(QS_ENOMEM, "qs_batch: descriptor allocation failed");
  e = cudaMemcpy(bt->d_circs, circs.data(), sizeof(BCircuit) * circs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(bt->d_order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(bt->d_blocks, blocks.data(), sizeof(BBlock) * blocks.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(bt->d_pool, pool.data(), sizeof(float2) * pool.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bfail(QS_ECUDA, std::string("qs_batch: upload failed: ") + cudaGetErrorString(e));
  bt->total_blocks = (int)blocks.size();
  return QS_OK;
}

cudaError_t launch_batch(qs_batch *bt, int threads) {
  cudaError_t e = cudaMemsetAsync(bt->d_queue, 0, sizeof(int), bt->stream);
  if (e != cudaSuccess) return e;
  const int count = (int)bt->states.size();
  int grid = dev_info().sms;  // one CTA per SM: 160 KB of shared memory each
  if (grid > count) grid = count;
  bt->grid = grid;
  if (threads == 256)
    k_batch<256><<<grid, 256, bt->smem, bt->stream>>>(bt->d_circs, bt->d_order, count, bt->d_blocks, bt->d_pool,
                                                      bt->d_queue);
  else if (threads == 1024)
    k_batch<1024><<<grid, 1024, bt->smem, bt->stream>>>(bt->d_circs, bt->d_order, count, bt->d_blocks, bt->d_pool,
                                                        bt->d_queue);
  else
    k_batch<512><<<grid, 512, bt->smem, bt->stream>>>(bt->d_circs, bt->d_order, count, bt->d_blocks, bt->d_pool,
                                                      bt->d_queue);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

qs_status qs_batch_create(qs_state *const *states, const qs_gate *const *gates, const size_t *n_gates, int count,
                          uint64_t flags, const qs_opts *opts, void *cuda_stream, qs_batch **out) {
  if (!out || !states || !gates || !n_gates || count <= 0) return bfail(QS_EINVAL, "qs_batch_create: bad arguments");
  *out = nullptr;
  if (opts && opts->n_global != 0)
    return bfail(QS_EUNSUPPORTED, "qs_batch_create: global bits (opts.n_global) are for qs_plan only");
  qs_batch *bt = new (std::nothrow) qs_batch();
  if (!bt) return bfail(QS_ENOMEM, "qs_batch_create: host allocation failed");
  if (opts) bt->opts = *opts;
  else qs_default_opts(&bt->opts);
  bt->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&bt->device);
  for (int c = 0; c < count; c++) {
    if (!states[c] || (n_gates[c] && !gates[c])) {
      delete bt;
      return bfail(QS_EINVAL, "qs_batch_create: null state or gate list");
    }
    if (!state_c64(states[c]) || state_n(states[c]) > kMaxBatchN) {
      delete bt;
      return bfail(QS_EUNSUPPORTED, "qs_batch_create: batches take complex64 states of at most 26 qubits");
    }
    for (int d = 0; d < c; d++)
      if (state_amps(states[d]) == state_amps(states[c])) {
        delete bt;
        return bfail(QS_EINVAL, "qs_batch_create: two entries share one state");
      }
    bt->states.push_back(states[c]);
    bt->gates.emplace_back(gates[c], gates[c] + n_gates[c]);
  }
  bt->smem = sizeof(float2) * (kMatFloats2 + (1 << kSmemBits));
  cudaError_t e = cudaFuncSetAttribute(k_batch<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt->smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt->smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt->smem);
  if (!bt->stream && e == cudaSuccess) {
    // the legacy stream cannot be captured: the batch runs on its own stream
    e = cudaStreamCreateWithFlags(&bt->own_stream, cudaStreamDefault);  // ordered with the legacy stream
    bt->stream = bt->own_stream;
  }
  if (e == cudaSuccess) e = qs::dev_malloc((void **)&bt->d_queue, sizeof(int));
  if (e != cudaSuccess) {
    qs_batch_free(bt);
    return bfail(QS_ECUDA, std::string("qs_batch_create: ") + cudaGetErrorString(e));
  }
  // fixed width, or autotune (fusion width x threads) on the batch itself
  std::vector<int> ks, ths = {256, 512, 1024};
  const int kfix = (flags & QS_FUSE) ? QS_FUSE_K_OF(flags) : 0;
  if (kfix) ks = {kfix};
  else ks = {2, 3, 4};
  if (bt->opts.threads > 0) ths = {bt->opts.threads};
  if (kfix >= 5) ths = {256};  // the wide mat-vecs need the 256-thread register budget
  const uint64_t base = (flags & (QS_VSWAP | QS_DIAG)) | QS_FUSE;
  double best = 1e300;
  int best_k = ks[0], best_t = ths[0];
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int k : ks) {
    qs_status s = upload_plan(bt, base | QS_FUSE_K(k));
    if (s != QS_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      qs_batch_free(bt);
      return s;
    }
    for (int t : ths) {
      float ms = 0;
      if (ks.size() * ths.size() > 1) {
        e = launch_batch(bt, t);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, bt->stream);
        if (e == cudaSuccess) e = launch_batch(bt, t);
        if (e == cudaSuccess) e = cudaEventRecord(e1, bt->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          qs_batch_free(bt);
          return bfail(QS_ECUDA, std::string("qs_batch_create: tuning launch failed: ") + cudaGetErrorString(e));
        }
        if (bt->n_tune < 16) {
          bt->tune_ms[bt->n_tune] = ms;
          bt->tune_k[bt->n_tune] = k;
          bt->tune_threads[bt->n_tune] = t;
          bt->n_tune++;
        }
      }
      if (ms < best) {
        best = ms;
        best_k = k;
        best_t = t;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  qs_status s = upload_plan(bt, base | QS_FUSE_K(best_k));
  if (s != QS_OK) {
    qs_batch_free(bt);
    return s;
  }
  bt->k_chosen = best_k;
  bt->threads = best_t;
  bt->flags = base | QS_FUSE_K(best_k);
  // capture queue reset + kernel once; runs replay the graph
  e = cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t le = launch_batch(bt, bt->threads);
    e = cudaStreamEndCapture(bt->stream, &bt->graph);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&bt->exec, bt->graph, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (bt->graph) cudaGraphDestroy(bt->graph);
    bt->graph = nullptr;
    bt->exec = nullptr;  // direct launches instead (still one kernel per run)
  }
  *out = bt;
  return QS_OK;
}

qs_status qs_batch_run(qs_batch *bt) {
  if (!bt) return bfail(QS_EINVAL, "qs_batch_run: null batch");
  cudaError_t e = bt->exec ? cudaGraphLaunch(bt->exec, bt->stream) : launch_batch(bt, bt->threads);
  if (e != cudaSuccess) return bfail(QS_ECUDA, std::string("qs_batch_run: ") + cudaGetErrorString(e));
  for (size_t c = 0; c < bt->states.size(); c++)
    std::memcpy(state_perm(bt->states[c]), bt->final_perm[c].data(), bt->final_perm[c].size());
  return QS_OK;
}

qs_status qs_batch_sync(qs_batch *bt) {
  if (!bt) return bfail(QS_EINVAL, "qs_batch_sync: null batch");
  cudaError_t e = cudaStreamSynchronize(bt->stream);
  if (e != cudaSuccess) return bfail(QS_ECUDA, std::string("qs_batch_sync: ") + cudaGetErrorString(e));
  return QS_OK;
}

qs_status qs_batch_info(const qs_batch *bt, qs_batch_info_t *out) {
  if (!bt || !out) return bfail(QS_EINVAL, "qs_batch_info: null argument");
  std::memset(out, 0, sizeof(*out));
  out->count = (int)bt->states.size();
  out->fuse_k = bt->k_chosen;
  out->threads = bt->threads;
  out->grid = bt->grid;
  out->total_blocks = bt->total_blocks;
  out->graph = bt->exec != nullptr;
  out->n_tuned = bt->n_tune;
  for (int i = 0; i < bt->n_tune; i++) {
    out->tuned_k[i] = bt->tune_k[i];
    out->tuned_threads[i] = bt->tune_threads[i];
    out->tuned_ms[i] = bt->tune_ms[i];
  }
  return QS_OK;
}

void qs_batch_free(qs_batch *bt) {
  if (!bt) return;
  if (bt->stream) cudaStreamSynchronize(bt->stream);
  else cudaDeviceSynchronize();
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  free_plan(bt);
  qs::dev_free(bt->d_queue);
  if (bt->own_stream) cudaStreamDestroy(bt->own_stream);
  delete bt;
}

qs_status qs_apply_batch(qs_state *const *states, const qs_gate *const *gates, const size_t *n_gates, int count,
                         uint64_t flags, const qs_opts *opts) {
  qs_batch *bt = nullptr;
  qs_status s = qs_batch_create(states, gates, n_gates, count, flags, opts, nullptr, &bt);
  if (s != QS_OK) return s;
  s = qs_batch_run(bt);
  if (s == QS_OK) s = qs_batch_sync(bt);
  const std::string err = s == QS_OK ? std::string() : qs::last_error_ref();
  qs_batch_free(bt);
  if (s != QS_OK) qs::last_error_ref() = err;
  return s;
}

}  // extern "C"
