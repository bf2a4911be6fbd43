// Profile-guided pass selection (Sec. III-A "PGO compilation flow", Sec.
// III-D activation rules).
//
// Rule-based activator: the paper's counter rules, one decision per
// optimisation, from the counters of the circuit at hand.
//
// Measured-profile activator: the paper leaves the mapping from profile data
// to optimisation flags open (Sec. III-A, "PGO design considerations"). Here
// the profile of earlier runs is a per-kernel-class throughput table (bytes and
// device time of every profiled block, grouped by kernel kind, width, tensor
// cores and whether bits 0 and 1 are both targets); each candidate
// flag set is planned on the host and its time predicted as the sum over its
// blocks of bytes / class throughput. Classes without measurements use
// compiled-in fractions of the HBM peak measured for these kernels on GB300.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "qs_internal.h"

namespace qs {

int block_class(const Block &b) {
  // phase polynomials share the diagonal kind with the "low" bit set, which
  // only dense classes use otherwise
  if (b.kind == BK_PHASE) return 64 + 8 * BK_DIAG + 7;
  // global-bit exchanges (planning only) likewise take an unused "low" class
  if (b.kind == BK_GLOBAL) return 64 + 8 * BK_PERMUTE + 2;
  // "low": bits 0 and 1 are both targets, so a thread's group is a run of
  // >= 4 contiguous amplitudes and a warp's accesses are strided
  int low = 0;
  if (b.kind == BK_DENSE && b.k > 1 && b.q[0] == 0 && b.q[1] == 1) low = 1;
  const int kind = (int)b.kind;  // 0 dense, 1 diag, 2 permute
  const int k = std::min(b.k, 7);
  return kind * 8 + k + (b.tc ? 32 : 0) + low * 64;
}

double class_prior_fraction(int cls) {
  const int kind = (cls % 32) / 8, k = cls % 8;
  const bool tc = (cls & 32) != 0, low = (cls & 64) != 0;
  double f;
  if (kind == 3) f = 0.15;  // tile pass: bound by the member blocks' arithmetic, not by HBM
  else if (kind == 2) f = 0.80;
  else if (kind == 1) f = 0.85;
  else if (tc) f = k <= 4 ? 0.90 : (k == 5 ? 0.86 : 0.74);
  else {
    static const double dense[8] = {0.95, 0.98, 0.97, 0.97, 0.64, 0.34, 0.10, 0.05};
    f = dense[k];
  }
  if (low && kind == 0) f *= tc ? 0.75 : 0.95;
  return f;
}

double predict_plan_ms(const std::vector<Block> &plan, int n, int amp_bytes, const qs_class_table *t,
                       double peak_gbs) {
  // scale the priors by what this device achieved relative to them
  // (byte-weighted mean of measured / prior throughput over measured classes)
  double scale = 1.0;
  if (t) {
    double num = 0, den = 0;
    for (int c = 0; c < QS_N_CLASSES; c++)
      if (t->count[c] > 0 && t->ms[c] > 0) {
        const double g = t->bytes[c] / (t->ms[c] * 1e-3) / 1e9;
        num += g / (class_prior_fraction(c) * peak_gbs) * t->bytes[c];
        den += t->bytes[c];
      }
    if (den > 0) scale = num / den;
  }
  double ms = 0;
  for (const Block &b : plan) {
    const int c = block_class(b);
    const double bytes = block_bytes(b, n, amp_bytes);
    double gbs;
    if (t && t->count[c] > 0 && t->ms[c] > 0) gbs = t->bytes[c] / (t->ms[c] * 1e-3) / 1e9;
    else gbs = class_prior_fraction(c) * peak_gbs * scale;
    ms += bytes / (gbs * 1e9) * 1e3 + 0.004;  // + launch gap
  }
  return ms;
}

// Rule-based activator (Sec. III-A "PGO compilation flow", Sec. III-D):
// one decision per optimisation from the counters of the circuit at hand.
uint64_t rules_select(int n, const qs_gate *gates, size_t n_gates, const qs_opts &o, uint64_t base) {
  int run[QS_MAX_QUBITS] = {0}, max_run = 0;
  int64_t swaps = 0, two_q_low = 0, t_count = 0, dense = 0;
  for (size_t i = 0; i < n_gates; i++) {
    const qs_gate &g = gates[i];
    if (g.op == QS_SWAP) swaps++;
    if (g.op == QS_T || g.op == QS_TDG) t_count++;
    if (!op_info(g.op).diagonal) dense++;
    if (g.nq == 1) {
      max_run = std::max(max_run, ++run[g.q[0]]);
    } else {
      for (int j = 0; j < g.nq; j++) run[g.q[j]] = 0;
      if ((g.op == QS_CX || g.op == QS_CPHASE || g.op == QS_CU1 || g.op == QS_CZ) &&
          (g.q[g.nq - 1] < o.low_bits))
        two_q_low++;
    }
  }
  (void)n;
  uint64_t f = base & ~(uint64_t)(QS_VSWAP | QS_FUSE | QS_DIAG | QS_FOLD | QS_RELOCATE | QS_TILE | (15ull << 16));
  // rotation folding: T gates above the threshold share of all gates
  if (n_gates && (double)t_count / (double)n_gates > o.t_ratio) f |= QS_FOLD;
  // virtual swap: SWAP gates present, or two-qubit gates hitting the fast
  // segment (the paper's CPhase/CNOT counter rule)
  if (swaps > 0 || two_q_low > 0) f |= QS_VSWAP;
  // relocation: the planner moves bits 0 and 1 out of the way when their
  // share of multi-qubit gates passes opts.reloc_share
  if (two_q_low > 0) f |= QS_RELOCATE;
  // merging: a run of consecutive one-qubit gates above the threshold, or
  // (GPU reading) any circuit with more than one gate, since each fused gate
  // saves a full pass over the state
  if (max_run > o.merge_run || n_gates > 1) f |= QS_FUSE | QS_FUSE_K(5) | QS_DIAG | QS_TC;
  (void)dense;
  return f;
}


void record_features(const qs_block_record &r, int n, bool c128, float *f) {
  for (int i = 0; i < QS_MLP_FEATURES; i++) f[i] = 0.f;
  int k = r.kind == BK_PERMUTE ? 2 : r.k;
  int tmin = 64, tmax = -1, low5 = 0, high = 0;
  bool bit[64] = {false};
  for (int j = 0; j < k && j < QS_MAX_DIAG; j++) {
    const int q = r.qubits[j];
    if (q < 0) continue;
    bit[q] = true;
    tmin = std::min(tmin, q);
    tmax = std::max(tmax, q);
    if (q < 5) low5++;
    if (q >= n - 6) high++;
  }
  f[0] = n / 32.f;
  f[1] = k / 6.f;
  f[2] = r.nctrl / 8.f;
  f[3] = r.kind == BK_DENSE;
  f[4] = r.kind == BK_DIAG || r.kind == BK_PHASE;
  f[5] = r.kind == BK_PERMUTE;
  f[6] = r.tc ? 1.f : 0.f;
  f[7] = (r.kind == BK_DENSE && bit[0] && bit[1]) ? 1.f : 0.f;
  f[8] = tmax >= 0 ? tmin / (float)n : 0.f;
  f[9] = tmax >= 0 ? tmax / (float)n : 0.f;
  f[10] = low5 / 6.f;
  f[11] = high / 6.f;
  f[12] = std::log2((float)r.n_gates + 1.f) / 8.f;
  f[13] = (float)(std::log2(r.bytes > 1 ? r.bytes : 1.0) / 40.0);
  for (int j = 0; j < 5; j++) f[14 + j] = bit[j] ? 1.f : 0.f;
  for (int q = 5; q < 64; q++)
    if (bit[q]) {
      if (q < 10) f[19] = 1.f;
      else if (q < 20) f[20] = 1.f;
      else f[21] = 1.f;
    }
  f[22] = c128 ? 1.f : 0.f;
  f[23] = r.meta == 4 ? 1.f : 0.f;
}

namespace {

// The flag sets both activators choose among: plain, virtual swap alone,
// fusion k = 1..6 with diagonal runs (tensor cores for k >= 4, c64), and
// cache-blocked tile passes when the state is wider than one tile.
std::vector<uint64_t> candidate_flags(int n, const qs_gate *gates, size_t n_gates, bool c128, const qs_opts &o) {
  bool has_swap = false;
  for (size_t i = 0; i < n_gates; i++) has_swap |= gates[i].op == QS_SWAP;
  std::vector<uint64_t> cands;
  const uint64_t vs = has_swap ? QS_VSWAP : 0;
  cands.push_back(QS_PLAIN);
  if (has_swap) cands.push_back(QS_VSWAP);
  for (int k = 1; k <= 6; k++) {
    cands.push_back(vs | QS_FUSE | QS_FUSE_K(k) | QS_DIAG);
    if (k >= 4 && !c128) cands.push_back(vs | QS_FUSE | QS_FUSE_K(k) | QS_DIAG | QS_TC);
  }
  if (n > tile_bits_of(o, c128)) cands.push_back(vs | QS_TILE);
  return cands;
}

}  // namespace

qs_status mlp_select(qs_mlp *mm, int n, bool c128, const qs_gate *gates, size_t n_gates, const qs_opts &o,
                     uint64_t *flags_out, double *pred_ms, std::string &err) {
  const std::vector<uint64_t> cands = candidate_flags(n, gates, n_gates, c128, o);
  std::vector<float> feats;
  std::vector<size_t> first(cands.size() + 1, 0);
  std::vector<Block> plan;
  PlanStats stats;
  for (size_t c = 0; c < cands.size(); c++) {
    int8_t perm[QS_MAX_QUBITS];
    for (int q = 0; q < n; q++) perm[q] = (int8_t)q;
    qs_status s = build_plan(n, gates, n_gates, cands[c], o, perm, plan, stats, err, c128);
    if (s != QS_OK) return s;
    first[c] = feats.size() / QS_MLP_FEATURES;
    for (size_t i = 0; i < plan.size(); i++) {
      qs_block_record r;
      fill_record(plan[i], (int)i, n, c128 ? 16 : 8, r);
      feats.resize(feats.size() + QS_MLP_FEATURES);
      record_features(r, n, c128, feats.data() + feats.size() - QS_MLP_FEATURES);
    }
  }
  first[cands.size()] = feats.size() / QS_MLP_FEATURES;
  const int total = (int)first[cands.size()];
  std::vector<float> y(total > 0 ? total : 1);
  if (total > 0) {
    qs_status s = qs_mlp_predict(mm, feats.data(), total, y.data());
    if (s != QS_OK) {
      err = "cost-model prediction failed";
      return s;
    }
  }
  double best = 1e300;
  uint64_t best_f = cands[0];
  for (size_t c = 0; c < cands.size(); c++) {
    double ms = 0;
    for (size_t i = first[c]; i < first[c + 1]; i++) ms += std::exp((double)y[i]) + 0.004;
    if (ms < best * 0.999) {
      best = ms;
      best_f = cands[c];
    }
  }
  *flags_out = best_f;
  if (pred_ms) *pred_ms = best;
  return QS_OK;
}

qs_status measured_select(int n, bool c128, const qs_gate *gates, size_t n_gates, const qs_opts &o,
                          const qs_class_table *t, uint64_t base, uint64_t *flags_out, double *pred_ms,
                          std::string &err) {
  const uint64_t keep = base & ~(uint64_t)(QS_VSWAP | QS_FUSE | QS_DIAG | QS_TC | QS_TILE | (15ull << 16) |
                                           QS_PGO_RULES | QS_PGO_MEASURED);
  const std::vector<uint64_t> cands = candidate_flags(n, gates, n_gates, c128, o);
  const double peak = o.peak_gbs > 0 ? o.peak_gbs : 6688.8;
  double best = 1e300;
  uint64_t best_f = cands[0];
  std::vector<Block> plan;
  PlanStats stats;
  for (uint64_t f : cands) {
    int8_t perm[QS_MAX_QUBITS];
    for (int q = 0; q < n; q++) perm[q] = (int8_t)q;
    qs_status s = build_plan(n, gates, n_gates, f, o, perm, plan, stats, err, c128);
    if (s != QS_OK) return s;
    const double ms = predict_plan_ms(plan, n, c128 ? 16 : 8, t, peak);
    if (ms < best * 0.999) {
      best = ms;
      best_f = f;
    }
  }
  *flags_out = keep | best_f;
  if (pred_ms) *pred_ms = best;
  return QS_OK;
}

}  // namespace qs
