// C ABI of the simulator core: state handles, the apply pipeline (ingest
// counters -> virtual swap -> fusion -> launches), profiling and reductions.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "qs_internal.h"

namespace qs {

std::string &last_error_ref() {
  static thread_local std::string msg;
  return msg;
}

}  // namespace qs

using namespace qs;

struct qs_state {
  int n = 0;
  qs_dtype dtype = QS_C64;
  void *amps = nullptr;
  bool owned = false;
  cudaStream_t stream = nullptr;
  int device = 0;
  int8_t perm[QS_MAX_QUBITS] = {0};
  bool bad = false;
  // device scratch for reductions and wide matrices, grown on demand
  double *d_partial = nullptr;
  size_t partial_cap = 0;
  double *d_out = nullptr;
  size_t out_cap = 0;
  void *d_mats = nullptr;
  size_t mats_cap = 0;
  void *h_mats = nullptr;  // pinned staging for d_mats
  size_t h_mats_cap = 0;
  cudaEvent_t mats_copied = nullptr;
  int *d_err = nullptr;  // set by kernels whose bounded waits expired
  // profiling (Sec. III-C): counters per logical qubit and gate type, the
  // longest run of consecutive one-qubit gates per qubit, per-block records
  int64_t counters[QS_MAX_QUBITS][QS_N_GATE_TYPES] = {{0}};
  int32_t run_1q[QS_MAX_QUBITS] = {0};
  int32_t max_run_1q[QS_MAX_QUBITS] = {0};
  int64_t gates_seen = 0;
  std::vector<cudaEvent_t> events;
  std::vector<qs_block_record> recs;
  bool recs_timed = false;
  bool recs_resolved = false;
  uint64_t flags_used = 0;
  PlanStats last_stats;
  double h2d_bytes = 0;
  std::vector<int> rec_class;  // kernel class of each record (measured-profile table)
  qs_class_table classes = {};
};

namespace qs {
void *state_amps(qs_state *st) { return st->amps; }
int state_n(const qs_state *st) { return st->n; }
bool state_c64(const qs_state *st) { return st->dtype == QS_C64; }
int8_t *state_perm(qs_state *st) { return st->perm; }
cudaStream_t state_stream(const qs_state *st) { return st->stream; }
}  // namespace qs

namespace {

int amp_bytes(const qs_state *st) { return st->dtype == QS_C128 ? 16 : 8; }

qs_status fail(qs_status s, const std::string &msg) {
  last_error_ref() = msg;
  return s;
}

qs_status cuda_fail(qs_state *st, cudaError_t e, const char *where) {
  if (st) st->bad = true;
  return fail(QS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// After a stream synchronisation: a kernel that gave up a bounded wait left
// 1 in the error word; report it once and clear it.
qs_status check_device_error(qs_state *st) {
  if (!st->d_err) return QS_OK;
  int h = 0;
  cudaError_t e = cudaMemcpy(&h, st->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return QS_ECUDA;
  if (h) {
    cudaMemset(st->d_err, 0, sizeof(int));
    last_error_ref() = "a device-side wait timed out; results of the last apply are not valid";
    return QS_ETIMEOUT;
  }
  return QS_OK;
}

// Resolves the CUDA-event times of the last apply call's blocks (waiting for
// them when `wait`) and adds them to the per-class throughput table once.
qs_status resolve_records(qs_state *st, bool wait) {
  if (!st->recs_timed || st->recs_resolved || st->recs.empty()) return QS_OK;
  cudaEvent_t last = st->events[st->recs.size()];
  if (!wait && cudaEventQuery(last) != cudaSuccess) {
    cudaGetLastError();  // not ready is not an error
    return QS_OK;
  }
  cudaError_t e = cudaEventSynchronize(last);
  if (e != cudaSuccess) return QS_ECUDA;
  for (size_t i = 0; i < st->recs.size(); i++) {
    float t0 = 0, dt = 0;
    e = cudaEventElapsedTime(&t0, st->events[0], st->events[i]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&dt, st->events[i], st->events[i + 1]);
    if (e != cudaSuccess) return QS_ECUDA;
    st->recs[i].t_start_ms = t0;
    st->recs[i].ms = dt;
    const int c = st->rec_class[i];
    st->classes.bytes[c] += st->recs[i].bytes;
    st->classes.ms[c] += dt;
    st->classes.count[c] += 1;
  }
  st->recs_resolved = true;
  return QS_OK;
}

qs_status fold_records(qs_state *st, bool wait) { return resolve_records(st, wait); }

// Undoes the relabelling with physical bit exchanges (one per cycle step),
// leaving perm = identity.
cudaError_t to_logical_order(qs_state *st) {
  for (int l = 0; l < st->n; l++) {
    if (st->perm[l] == l) continue;
    int other = -1;
    for (int k = 0; k < st->n; k++)
      if (st->perm[k] == l) other = k;
    cudaError_t e = launch_permute(st->amps, st->n, st->dtype == QS_C128, st->perm[l], l, st->stream);
    if (e != cudaSuccess) return e;
    st->perm[other] = st->perm[l];
    st->perm[l] = (int8_t)l;
  }
  return cudaSuccess;
}

qs_status check_state(const qs_state *st) {
  if (!st) return fail(QS_EINVAL, "null state");
  if (st->bad) return fail(QS_ESTATE, "state invalid after an earlier CUDA error");
  return QS_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

template <typename T> cudaError_t grow(T *&ptr, size_t &cap, size_t need) {
  if (need <= cap) return cudaSuccess;
  dev_free(ptr);
  ptr = nullptr;
  cap = 0;
  cudaError_t e = dev_malloc((void **)&ptr, need * sizeof(T));
  if (e == cudaSuccess) cap = need;
  return e;
}

qs_status make_state(int n, qs_dtype dtype, void *stream, qs_state **out) {
  if (!out) return fail(QS_EINVAL, "null output handle");
  *out = nullptr;
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_EINVAL, "unknown dtype");
  const int nmax = dtype == QS_C64 ? QS_MAX_N_C64 : QS_MAX_N_C128;
  if (n < 1 || n > nmax) return fail(QS_EUNSUPPORTED, "qubit count out of range for this dtype");
  qs_state *st = new (std::nothrow) qs_state();
  if (!st) return fail(QS_ENOMEM, "host allocation failed");
  st->n = n;
  st->dtype = dtype;
  st->stream = (cudaStream_t)stream;
  cudaGetDevice(&st->device);
  for (int q = 0; q < n; q++) st->perm[q] = (int8_t)q;
  *out = st;
  return QS_OK;
}

void record_counters(qs_state *st, const qs_gate *gates, size_t n_gates) {
  for (size_t i = 0; i < n_gates; i++) {
    const qs_gate &g = gates[i];
    for (int j = 0; j < g.nq; j++) st->counters[g.q[j]][g.op]++;
    if (g.nq == 1) {
      int q = g.q[0];
      st->run_1q[q]++;
      st->max_run_1q[q] = std::max(st->max_run_1q[q], st->run_1q[q]);
    } else {
      for (int j = 0; j < g.nq; j++) st->run_1q[g.q[j]] = 0;
    }
  }
  st->gates_seen += (int64_t)n_gates;
}

}  // namespace

extern "C" {

void qs_default_opts(qs_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->merge_run = 5;
  o->t_ratio = 0.10;
  o->low_bits = 5;
  o->reloc_share = 0.25;
  o->diag_max = QS_MAX_DIAG;
  o->threads = 0;
  o->peak_gbs = 6688.8;
  o->fuse_lookahead = 60;
}

const char *qs_last_error(void) { return last_error_ref().c_str(); }

qs_status qs_alloc_state(int n, qs_dtype dtype, void *cuda_stream, qs_state **out) {
  qs_status s = make_state(n, dtype, cuda_stream, out);
  if (s != QS_OK) return s;
  qs_state *st = *out;
  const size_t bytes = (size_t)amp_bytes(st) << n;
  cudaError_t e = dev_malloc(&st->amps, bytes);
  if (e != cudaSuccess) {
    delete st;
    *out = nullptr;
    return fail(QS_ENOMEM, dev_refused_by_budget() ? std::string("state allocation refused by the memory budget")
                                                   : std::string("device allocation of the state failed: ") +
                                                         cudaGetErrorString(e));
  }
  st->owned = true;
  e = launch_set_basis(st->amps, n, dtype == QS_C128, 0, st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "qs_alloc_state");
  return QS_OK;
}

qs_status qs_attach_state(void *dev_ptr, int n, qs_dtype dtype, void *cuda_stream, qs_state **out) {
  if (!dev_ptr) return fail(QS_EINVAL, "null device pointer");
  if (((uintptr_t)dev_ptr & 15) != 0) return fail(QS_EINVAL, "device pointer not 16-byte aligned");
  qs_status s = make_state(n, dtype, cuda_stream, out);
  if (s != QS_OK) return s;
  (*out)->amps = dev_ptr;
  (*out)->owned = false;
  return QS_OK;
}

void qs_free_state(qs_state *st) {
  if (!st) return;
  DeviceGuard g(st->device);
  if (st->stream) cudaStreamSynchronize(st->stream);
  else cudaDeviceSynchronize();
  if (st->owned) dev_free(st->amps);
  dev_free(st->d_partial);
  dev_free(st->d_out);
  dev_free(st->d_mats);
  if (st->h_mats) cudaFreeHost(st->h_mats);
  if (st->mats_copied) cudaEventDestroy(st->mats_copied);
  dev_free(st->d_err);
  for (cudaEvent_t e : st->events) cudaEventDestroy(e);
  delete st;
}

qs_status qs_set_basis(qs_state *st, uint64_t x) {
  qs_status s = check_state(st);
  if (s != QS_OK) return s;
  if (st->n < 64 && (x >> st->n) != 0) return fail(QS_EINVAL, "basis index out of range");
  DeviceGuard g(st->device);
  for (int q = 0; q < st->n; q++) st->perm[q] = (int8_t)q;
  cudaError_t e = launch_set_basis(st->amps, st->n, st->dtype == QS_C128, x, st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "qs_set_basis");
  return QS_OK;
}

qs_status qs_get_perm(const qs_state *st, int8_t *perm_out) {
  if (!st || !perm_out) return fail(QS_EINVAL, "null argument");
  std::memcpy(perm_out, st->perm, st->n);
  return QS_OK;
}

qs_status qs_device_ptr(const qs_state *st, void **out) {
  if (!st || !out) return fail(QS_EINVAL, "null argument");
  *out = st->amps;
  return QS_OK;
}

qs_status qs_apply_circuit(qs_state *st, const qs_gate *gates, size_t n_gates, uint64_t flags,
                           const qs_opts *opts) {
  qs_status s = check_state(st);
  if (s != QS_OK) return s;
  if (n_gates && !gates) return fail(QS_EINVAL, "null gate list");
  qs_opts o;
  if (opts) o = *opts;
  else qs_default_opts(&o);
  if (o.n_global != 0)
    return fail(QS_EUNSUPPORTED, "qs_apply_circuit: global bits (opts.n_global) need a sharded runner; "
                                 "qs_plan plans their exchanges");
  DeviceGuard dg(st->device);
  // fold the timings of an earlier profiled call that has finished
  fold_records(st, false);
  if (flags & QS_PGO_MEASURED) {
    std::string err;
    uint64_t f = 0;
    s = measured_select(st->n, st->dtype == QS_C128, gates, n_gates, o, &st->classes, flags, &f, nullptr, err);
    if (s != QS_OK) return fail(s, "qs_apply_circuit: " + err);
    // a first call has no measurements yet: profile it so the next one has
    flags = f | QS_PROFILE;
  } else if (flags & QS_PGO_RULES) {
    flags = rules_select(st->n, gates, n_gates, o, flags);
  }

  std::vector<Block> plan;
  PlanStats stats;
  std::string err;
  int8_t perm[QS_MAX_QUBITS];
  std::memcpy(perm, st->perm, sizeof(perm));
  s = build_plan(st->n, gates, n_gates, flags, o, perm, plan, stats, err, st->dtype == QS_C128);
  if (s != QS_OK) return fail(s, "qs_apply_circuit: " + err);
  record_counters(st, gates, n_gates);

  const bool c128 = st->dtype == QS_C128;
  const int ab = amp_bytes(st);
  // matrices of wide dense blocks: one pinned staging buffer, one copy
  size_t mat_bytes = 0;
  std::vector<size_t> mat_off(plan.size(), (size_t)-1);
  for (size_t i = 0; i < plan.size(); i++)
    if (block_needs_dev_matrix(plan[i], c128)) {
      mat_off[i] = mat_bytes;
      mat_bytes += (block_dev_matrix_bytes(plan[i], c128) + 255) & ~(size_t)255;
    }
  bool any_tc = false;
  for (const Block &b : plan) any_tc |= b.tc && !c128;
  cudaError_t e;
  if (mat_bytes) {
    if (st->mats_copied) {
      e = cudaEventSynchronize(st->mats_copied);  // staging buffer free again
      if (e != cudaSuccess) return cuda_fail(st, e, "qs_apply_circuit");
    } else {
      e = cudaEventCreateWithFlags(&st->mats_copied, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(st, e, "qs_apply_circuit");
    }
    if (mat_bytes > st->h_mats_cap) {
      if (st->h_mats) cudaFreeHost(st->h_mats);
      st->h_mats = nullptr;
      st->h_mats_cap = 0;
      e = cudaMallocHost(&st->h_mats, mat_bytes);
      if (e != cudaSuccess) return fail(QS_ENOMEM, "pinned staging allocation failed");
      st->h_mats_cap = mat_bytes;
    }
    size_t cap_bytes = st->mats_cap;
    unsigned char *dm = (unsigned char *)st->d_mats;
    if (mat_bytes > cap_bytes) {
      dev_free(dm);
      dm = nullptr;
      st->d_mats = nullptr;
      st->mats_cap = 0;
      e = dev_malloc((void **)&dm, mat_bytes);
      if (e != cudaSuccess) return fail(QS_ENOMEM, "matrix buffer allocation failed");
      st->d_mats = dm;
      st->mats_cap = mat_bytes;
    }
    parallel_blocks(plan.size(), [&](size_t i) {
      if (mat_off[i] != (size_t)-1) fill_dev_matrix(plan[i], c128, (unsigned char *)st->h_mats + mat_off[i]);
    });
    e = cudaMemcpyAsync(st->d_mats, st->h_mats, mat_bytes, cudaMemcpyHostToDevice, st->stream);
    if (e != cudaSuccess) return cuda_fail(st, e, "qs_apply_circuit");
    e = cudaEventRecord(st->mats_copied, st->stream);
    if (e != cudaSuccess) return cuda_fail(st, e, "qs_apply_circuit");
  }

  if (any_tc && !st->d_err) {
    e = dev_malloc((void **)&st->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(st->d_err, 0, sizeof(int), st->stream);
    if (e != cudaSuccess) return fail(QS_ENOMEM, "error word allocation failed");
  }
  const bool prof = flags & QS_PROFILE;
  if (prof) {
    while (st->events.size() < plan.size() + 1) {
      cudaEvent_t ev;
      e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return cuda_fail(st, e, "qs_apply_circuit");
      st->events.push_back(ev);
    }
    e = cudaEventRecord(st->events[0], st->stream);
    if (e != cudaSuccess) return cuda_fail(st, e, "qs_apply_circuit");
  }
  st->recs.clear();
  st->rec_class.clear();
  st->recs.reserve(plan.size());
  st->h2d_bytes = 0;
  for (size_t i = 0; i < plan.size(); i++) {
    const Block &b = plan[i];
    const void *dm = mat_off[i] == (size_t)-1 ? nullptr : (const unsigned char *)st->d_mats + mat_off[i];
    LaunchShape shape;
    e = launch_block_with_matrix(st->amps, st->n, c128, b, dm, st->d_err, st->stream, o.threads, &shape);
    if (e != cudaSuccess) return cuda_fail(st, e, "qs_apply_circuit launch");
    if (prof) {
      e = cudaEventRecord(st->events[i + 1], st->stream);
      if (e != cudaSuccess) return cuda_fail(st, e, "qs_apply_circuit");
    }
    qs_block_record r;
    fill_record(b, (int)i, st->n, ab, r);
    r.tiles = shape.tiles;
    r.ctas = shape.ctas;
    st->rec_class.push_back(block_class(b));
    st->h2d_bytes += (double)block_param_bytes(b, c128);
    st->recs.push_back(r);
  }
  std::memcpy(st->perm, perm, sizeof(perm));
  st->recs_timed = prof;
  st->recs_resolved = false;
  st->flags_used = flags;
  st->last_stats = stats;
  return QS_OK;
}

qs_status qs_profile(qs_state *st, qs_profile_summary *out, qs_block_record *recs, size_t cap,
                     size_t *n_recs) {
  qs_status s = check_state(st);
  if (s != QS_OK) return s;
  if (!out) return fail(QS_EINVAL, "null summary");
  DeviceGuard dg(st->device);
  if (resolve_records(st, true) != QS_OK) return cuda_fail(st, cudaGetLastError(), "qs_profile");
  std::memset(out, 0, sizeof(*out));
  out->n_qubits = st->n;
  out->n_blocks = (int)st->recs.size();
  out->gates_seen = st->gates_seen;
  out->flags_used = st->flags_used;
  out->swaps_absorbed = st->last_stats.swaps_absorbed;
  out->gates_last = st->last_stats.gates_in;
  std::memcpy(out->counters, st->counters, sizeof(st->counters));
  std::memcpy(out->max_1q_run, st->max_run_1q, sizeof(st->max_run_1q));
  double tot_ms = 0, tot_b = 0;
  for (const auto &r : st->recs) {
    tot_b += r.bytes;
    if (r.ms >= 0) tot_ms += r.ms;
  }
  out->total_ms = st->recs_timed ? tot_ms : -1;
  out->total_bytes = tot_b;
  out->h2d_bytes = st->h2d_bytes;
  if (n_recs) *n_recs = st->recs.size();
  if (recs) {
    size_t k = std::min(cap, st->recs.size());
    std::memcpy(recs, st->recs.data(), k * sizeof(qs_block_record));
  }
  return QS_OK;
}

qs_status qs_profile_classes(const qs_state *st, qs_class_table *out) {
  if (!st || !out) return fail(QS_EINVAL, "null argument");
  *out = st->classes;
  return QS_OK;
}

qs_status qs_pgo_select(int n, qs_dtype dtype, const qs_gate *gates, size_t n_gates, const qs_class_table *table,
                        const qs_opts *opts, uint64_t *flags_out, double *predicted_ms) {
  if (!flags_out || (n_gates && !gates)) return fail(QS_EINVAL, "null argument");
  if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_EINVAL, "qubit count out of range");
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_EINVAL, "unknown dtype");
  qs_opts o;
  if (opts) o = *opts;
  else qs_default_opts(&o);
  std::string err;
  qs_status s = measured_select(n, dtype == QS_C128, gates, n_gates, o, table, 0, flags_out, predicted_ms, err);
  if (s != QS_OK) return fail(s, "qs_pgo_select: " + err);
  return QS_OK;
}

qs_status qs_pgo_predict(int n, qs_dtype dtype, const qs_gate *gates, size_t n_gates, uint64_t flags,
                         const qs_class_table *table, const qs_opts *opts, double *predicted_ms) {
  if (!predicted_ms || (n_gates && !gates)) return fail(QS_EINVAL, "qs_pgo_predict: null argument");
  if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_EINVAL, "qs_pgo_predict: qubit count out of range");
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_EINVAL, "qs_pgo_predict: unknown dtype");
  if (flags & (QS_PGO_RULES | QS_PGO_MEASURED)) return fail(QS_EINVAL, "qs_pgo_predict: give explicit pass flags");
  qs_opts o;
  if (opts) o = *opts;
  else qs_default_opts(&o);
  std::vector<Block> plan;
  PlanStats stats;
  std::string err;
  int8_t perm[QS_MAX_QUBITS];
  for (int q = 0; q < n; q++) perm[q] = (int8_t)q;
  qs_status s = build_plan(n, gates, n_gates, flags, o, perm, plan, stats, err, dtype == QS_C128);
  if (s != QS_OK) return fail(s, "qs_pgo_predict: " + err);
  *predicted_ms = predict_plan_ms(plan, n, dtype == QS_C128 ? 16 : 8, table, o.peak_gbs > 0 ? o.peak_gbs : 6688.8);
  return QS_OK;
}

qs_status qs_fold_rotations(int n, const qs_gate *in, size_t n_in, qs_gate *out, size_t cap, size_t *n_out) {
  if (n < 1 || n > QS_MAX_QUBITS || (n_in && !in) || !n_out) return fail(QS_EINVAL, "qs_fold_rotations: bad arguments");
  std::vector<Block> plan;
  PlanStats stats;
  std::string err;
  int8_t perm[QS_MAX_QUBITS];
  for (int q = 0; q < n; q++) perm[q] = (int8_t)q;
  qs_opts o;
  qs_default_opts(&o);
  // validation of the input gates
  qs_status s = build_plan(n, in, n_in, QS_PLAIN, o, perm, plan, stats, err);
  if (s != QS_OK) return fail(s, "qs_fold_rotations: " + err);
  std::vector<qs_gate> f = fold_rotations(n, in, n_in);
  *n_out = f.size();
  if (f.size() > cap) return fail(QS_EINVAL, "qs_fold_rotations: output buffer too small");
  if (!f.empty()) std::memcpy(out, f.data(), f.size() * sizeof(qs_gate));
  return QS_OK;
}

qs_status qs_block_features(int n, qs_dtype dtype, const qs_block_record *recs, size_t count, float *out) {
  if ((count && (!recs || !out)) || n < 1 || n > QS_MAX_QUBITS) return fail(QS_EINVAL, "qs_block_features: bad arguments");
  for (size_t i = 0; i < count; i++) record_features(recs[i], n, dtype == QS_C128, out + i * QS_MLP_FEATURES);
  return QS_OK;
}

qs_status qs_pgo_select_mlp(qs_mlp *m, int n, qs_dtype dtype, const qs_gate *gates, size_t n_gates,
                            const qs_opts *opts, uint64_t *flags_out, double *predicted_ms) {
  if (!m || !flags_out || (n_gates && !gates)) return fail(QS_EINVAL, "qs_pgo_select_mlp: null argument");
  if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_EINVAL, "qs_pgo_select_mlp: qubit count out of range");
  qs_opts o;
  if (opts) o = *opts;
  else qs_default_opts(&o);
  std::string err;
  qs_status s = mlp_select(m, n, dtype == QS_C128, gates, n_gates, o, flags_out, predicted_ms, err);
  if (s != QS_OK) return fail(s, "qs_pgo_select_mlp: " + err);
  return QS_OK;
}

qs_status qs_profile_reset(qs_state *st) {
  if (!st) return fail(QS_EINVAL, "null state");
  std::memset(&st->classes, 0, sizeof(st->classes));
  std::memset(st->counters, 0, sizeof(st->counters));
  std::memset(st->run_1q, 0, sizeof(st->run_1q));
  std::memset(st->max_run_1q, 0, sizeof(st->max_run_1q));
  st->gates_seen = 0;
  st->recs.clear();
  return QS_OK;
}

qs_status qs_tc_exchange_layout(int n, int k, const int *targets, uint64_t cmask, qs_exchange_layout *out) {
  if (!targets || !out) return fail(QS_EINVAL, "null argument");
  if (n < 1 || n > QS_MAX_QUBITS || k < 4 || k > 6) return fail(QS_EINVAL, "n or k out of range");
  Block b;
  b.kind = BK_DENSE;
  b.k = k;
  uint64_t tmask = 0;
  for (int j = 0; j < k; j++) {
    if (targets[j] < 0 || targets[j] >= n || (j > 0 && targets[j] <= targets[j - 1]))
      return fail(QS_EINVAL, "targets must be distinct, ascending and below n");
    b.q[j] = targets[j];
    tmask |= 1ull << targets[j];
  }
  if ((cmask & tmask) || (n < 64 && (cmask >> n))) return fail(QS_EINVAL, "bad control mask");
  b.cmask = cmask;
  b.nctrl = __builtin_popcountll(cmask);
  std::memset(out, 0, sizeof(*out));
  TcXLayout x;
  if (!tc_exchange_layout(n, b, x)) return QS_OK;
  out->applies = 1;
  for (int i = 0; i < 5; i++) out->lane_bits[i] = x.lbit[i];
  const int rb = k == 6 ? 4 : k - 1;
  for (int j = 0; j < 4; j++) out->reg_bits[j] = j < rb ? x.rbit[j] : -1;
  out->la = x.la;
  out->nswb = x.nswb;
  for (int i = 0; i < 2; i++) out->lb[i] = i < x.nswb ? x.lb[i] : -1;
  for (int s = 0; s < 6; s++) out->slot_target[s] = s < k ? x.slot_mat[s] : -1;
  out->part_bits[0] = x.part_bit[0];
  out->part_bits[1] = x.part_bit[1];
  return QS_OK;
}

qs_status qs_plan(int n, const qs_gate *gates, size_t n_gates, uint64_t flags, const qs_opts *opts,
                  int8_t *perm_inout, qs_block_record *recs, size_t cap, size_t *n_blocks, double *mats,
                  size_t mats_cap, size_t *mats_len) {
  if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_EINVAL, "qubit count out of range");
  if (!perm_inout || (n_gates && !gates)) return fail(QS_EINVAL, "null argument");
  qs_opts o;
  if (opts) o = *opts;
  else qs_default_opts(&o);
  if (flags & QS_PGO_RULES) flags = rules_select(n, gates, n_gates, o, flags);
  std::vector<Block> plan;
  PlanStats stats;
  std::string err;
  int8_t perm[QS_MAX_QUBITS];
  std::memcpy(perm, perm_inout, n);
  qs_status s = build_plan(n, gates, n_gates, flags, o, perm, plan, stats, err);
  if (s != QS_OK) return fail(s, "qs_plan: " + err);
  std::memcpy(perm_inout, perm, n);
  size_t mlen = 0, nr = 0;
  auto put = [&](double re, double im) {
    if (mats && mlen < mats_cap) {
      mats[2 * mlen] = re;
      mats[2 * mlen + 1] = im;
    }
    mlen++;
  };
  auto emit = [&](const Block &b, int index) {
    if (recs && nr < cap) fill_record(b, index, n, 8, recs[nr]);
    nr++;
    for (const cd &z : b.mat) put(z.real(), z.imag());
    if (b.kind == BK_PHASE) {
      for (int j = 0; j < b.k; j++) put((double)b.ph_q[j], b.ph_a[j]);
      put(b.ph_c, 0.0);
      for (double x : b.ph_b) put(x, 0.0);
    }
  };
  for (size_t i = 0; i < plan.size(); i++) {
    emit(plan[i], (int)i);
    for (const Block &m : plan[i].sub) emit(m, (int)i);  // a tile pass's members, in order
  }
  if (n_blocks) *n_blocks = nr;
  if (mats_len) *mats_len = mlen;
  return QS_OK;
}

qs_status qs_measure_probs(qs_state *st, const int *logical_qubits, int m, double *host_out) {
  qs_status s = check_state(st);
  if (s != QS_OK) return s;
  if (!host_out || (m > 0 && !logical_qubits)) return fail(QS_EINVAL, "null argument");
  if (m < 0 || m > st->n || m > 26) return fail(QS_EINVAL, "m out of range");
  int pos[32];
  for (int j = 0; j < m; j++) {
    int l = logical_qubits[j];
    if (l < 0 || l >= st->n) return fail(QS_EINVAL, "qubit out of range");
    for (int i = 0; i < j; i++)
      if (logical_qubits[i] == l) return fail(QS_EINVAL, "duplicate qubit");
    pos[j] = st->perm[l];
  }
  DeviceGuard dg(st->device);
  const size_t nb = (size_t)1 << m;
  cudaError_t e = grow(st->d_partial, st->partial_cap, std::max<size_t>(1, probs_scratch_doubles(st->n, m)));
  if (e == cudaSuccess) e = grow(st->d_out, st->out_cap, nb);
  if (e != cudaSuccess) return fail(QS_ENOMEM, "scratch allocation failed");
  e = launch_probs(st->amps, st->n, st->dtype == QS_C128, pos, m, st->d_partial, st->d_out, st->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, st->d_out, nb * sizeof(double), cudaMemcpyDeviceToHost, st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "qs_measure_probs");
  return check_device_error(st);
}

qs_status qs_norm(qs_state *st, double *host_out) { return qs_measure_probs(st, nullptr, 0, host_out); }

qs_status qs_read_state(qs_state *st, void *host_out, int logical_order) {
  qs_status s = check_state(st);
  if (s != QS_OK) return s;
  if (!host_out) return fail(QS_EINVAL, "null argument");
  DeviceGuard dg(st->device);
  cudaError_t e = cudaSuccess;
  if (logical_order) {
    e = to_logical_order(st);
    if (e != cudaSuccess) return cuda_fail(st, e, "qs_read_state");
  }
  e = cudaMemcpyAsync(host_out, st->amps, (size_t)amp_bytes(st) << st->n, cudaMemcpyDeviceToHost, st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "qs_read_state");
  return check_device_error(st);
}

qs_status qs_state_distance(qs_state *a, qs_state *b, double *out) {
  qs_status s = check_state(a);
  if (s == QS_OK) s = check_state(b);
  if (s != QS_OK) return s;
  if (!out || a == b) return fail(QS_EINVAL, "qs_state_distance: bad arguments");
  if (a->n != b->n || a->device != b->device) return fail(QS_EINVAL, "qs_state_distance: states differ in size or device");
  DeviceGuard dg(a->device);
  cudaError_t e = cudaSuccess;
  if (std::memcmp(a->perm, b->perm, a->n) != 0) {
    e = to_logical_order(a);
    if (e == cudaSuccess) e = to_logical_order(b);
    if (e != cudaSuccess) return cuda_fail(a, e, "qs_state_distance");
  }
  // b's stream waits for a's work; the reduction runs on b's stream
  if (a->stream != b->stream) {
    e = cudaStreamSynchronize(a->stream);
    if (e != cudaSuccess) return cuda_fail(a, e, "qs_state_distance");
  }
  const int grid = distance_grid();
  e = grow(b->d_partial, b->partial_cap, (size_t)grid);
  if (e != cudaSuccess) return fail(QS_ENOMEM, "scratch allocation failed");
  e = launch_distance(a->amps, a->dtype == QS_C128, b->amps, b->dtype == QS_C128, a->n, b->d_partial, b->stream);
  std::vector<double> part(grid);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(part.data(), b->d_partial, sizeof(double) * grid, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "qs_state_distance");
  double sum = 0;
  for (double v : part) sum += v;
  *out = std::sqrt(sum);
  return QS_OK;
}

qs_status qs_write_state(qs_state *st, const void *host_in) {
  qs_status s = check_state(st);
  if (s != QS_OK) return s;
  if (!host_in) return fail(QS_EINVAL, "null argument");
  DeviceGuard dg(st->device);
  cudaError_t e = cudaMemcpyAsync(st->amps, host_in, (size_t)amp_bytes(st) << st->n, cudaMemcpyHostToDevice, st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "qs_write_state");
  return QS_OK;
}

}  // extern "C"
