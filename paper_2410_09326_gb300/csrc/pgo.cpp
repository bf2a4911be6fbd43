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
  if (kind == 2) f = 0.80;
  else if (kind == 1) f = 0.85;
  else if (tc) f = k <= 4 ? 0.85 : 0.76;
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
  uint64_t f = base & ~(uint64_t)(QS_VSWAP | QS_FUSE | QS_DIAG | (15ull << 16));
  // virtual swap: SWAP gates present, or two-qubit gates hitting the fast
  // segment (the paper's CPhase/CNOT counter rule)
  if (swaps > 0 || two_q_low > 0) f |= QS_VSWAP;
  // merging: a run of consecutive one-qubit gates above the threshold, or
  // (GPU reading) any circuit with more than one gate, since each fused gate
  // saves a full pass over the state
  if (max_run > o.merge_run || n_gates > 1) f |= QS_FUSE | QS_FUSE_K(5) | QS_DIAG | QS_TC;
  (void)t_count;
  (void)dense;
  return f;
}


qs_status measured_select(int n, bool c128, const qs_gate *gates, size_t n_gates, const qs_opts &o,
                          const qs_class_table *t, uint64_t base, uint64_t *flags_out, double *pred_ms,
                          std::string &err) {
  const uint64_t keep = base & ~(uint64_t)(QS_VSWAP | QS_FUSE | QS_DIAG | QS_TC | (15ull << 16) |
                                           QS_PGO_RULES | QS_PGO_MEASURED);
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
  const double peak = o.peak_gbs > 0 ? o.peak_gbs : 6688.8;
  double best = 1e300;
  uint64_t best_f = cands[0];
  std::vector<Block> plan;
  PlanStats stats;
  for (uint64_t f : cands) {
    int8_t perm[QS_MAX_QUBITS];
    for (int q = 0; q < n; q++) perm[q] = (int8_t)q;
    qs_status s = build_plan(n, gates, n_gates, f, o, perm, plan, stats, err);
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
