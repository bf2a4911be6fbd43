// Rotation folding and peephole cancellation (Sec. III-D "Rotation folding":
// phase rotations are combined through the commutation rules of Clifford and
// Pauli gates, e.g. T . T -> S, and pairs such as CNOT . CNOT cancel, Sec.
// III-C).
//
// Phase-polynomial view: inside a run of CNOT, X, SWAP and diagonal gates,
// every wire holds a parity (XOR of input variables, plus a constant) and
// every phase gate diag(1, e^{ia}) multiplies the state by e^{ia P} for the
// parity P of its wire. Two phase gates with the same parity merge into the
// first one as long as the parity stays available, i.e. stays in the GF(2)
// span of the values the wires still hold: a gate outside that set (H, RX, a
// general U3, ...) on wire w takes w's value out of the span and gives w a
// fresh variable; terms whose parity leaves the span are closed. Diagonal
// gates that are not linear phases (CPhase, CZ, CRZ) pass through untouched:
// they change no wire value and commute with every phase term.
//
// RZ(t) = e^{-it/2} diag(1, e^{it}) takes part with its global phase
// tracked; a nonzero total is emitted at the end as U1(2g) RZ(-2g) = e^{ig}
// on qubit 0, so amplitudes stay exact. RZZ and the other two-qubit phases
// pass through unchanged.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "qs_internal.h"

namespace qs {

namespace {

using Bits = std::vector<uint64_t>;  // set of variables as a bitset

struct Wire {
  Bits par;
  int cst = 0;
};

struct Term {
  size_t out_index;  // position of the emitted gate in the output list
  int wire;
  int cst;           // constant of the wire at the first occurrence
  double angle;      // phase e^{i angle P}
  bool open = true;
};

bool phase_angle(const qs_gate &g, double &a, double &gphase) {
  gphase = 0;
  switch (g.op) {
    case QS_T: a = M_PI / 4; return true;
    case QS_TDG: a = -M_PI / 4; return true;
    case QS_S: a = M_PI / 2; return true;
    case QS_SDG: a = -M_PI / 2; return true;
    case QS_Z: a = M_PI; return true;
    case QS_U1: a = g.p[0]; return true;
    case QS_RZ: a = g.p[0]; gphase = -g.p[0] / 2; return true;
    default: return false;
  }
}

double wrap(double a) {
  a = std::fmod(a, 2 * M_PI);
  if (a > M_PI) a -= 2 * M_PI;
  if (a <= -M_PI) a += 2 * M_PI;
  return a;
}

// One-qubit phase gate diag(1, e^{ia}) on q, by name where one fits.
qs_gate phase_gate(int q, double a) {
  qs_gate g;
  std::memset(&g, 0, sizeof(g));
  g.nq = 1;
  g.q[0] = (uint8_t)q;
  const double w = wrap(a);
  auto near = [&](double x) { return std::fabs(w - x) < 1e-12; };
  if (near(M_PI / 4)) g.op = QS_T;
  else if (near(-M_PI / 4)) g.op = QS_TDG;
  else if (near(M_PI / 2)) g.op = QS_S;
  else if (near(-M_PI / 2)) g.op = QS_SDG;
  else if (near(M_PI) || near(-M_PI)) g.op = QS_Z;
  else {
    g.op = QS_U1;
    g.p[0] = w;
  }
  return g;
}

// Is target in the GF(2) span of rows (Gaussian elimination on copies)?
bool in_span(std::vector<Bits> rows, Bits target) {
  const size_t words = target.size();
  for (size_t wi = 0; wi < words; wi++)
    for (int bit = 63; bit >= 0; bit--) {
      const uint64_t m = 1ull << bit;
      int piv = -1;
      for (size_t r = 0; r < rows.size(); r++)
        if (rows[r][wi] & m) {
          piv = (int)r;
          break;
        }
      if (piv < 0) continue;
      Bits p = rows[piv];
      rows.erase(rows.begin() + piv);
      for (auto &r : rows)
        if (r[wi] & m)
          for (size_t k = 0; k < words; k++) r[k] ^= p[k];
      if (target[wi] & m)
        for (size_t k = 0; k < words; k++) target[k] ^= p[k];
    }
  for (uint64_t w : target)
    if (w) return false;
  return true;
}

bool same_qubits(const qs_gate &a, const qs_gate &b) {
  if (a.op != b.op || a.nq != b.nq) return false;
  for (int j = 0; j < a.nq; j++)
    if (a.q[j] != b.q[j]) return false;
  return true;
}

bool self_inverse(int op) {
  return op == QS_H || op == QS_X || op == QS_Y || op == QS_Z || op == QS_CX || op == QS_CZ || op == QS_CY ||
         op == QS_SWAP || op == QS_CCX || op == QS_CSWAP || op == QS_CH || op == QS_ID;
}

// Removes adjacent equal self-inverse gates (nothing in between touches
// their qubits) and identity gates, until nothing changes.
std::vector<qs_gate> cancel_pairs(std::vector<qs_gate> g) {
  bool changed = true;
  while (changed) {
    changed = false;
    std::vector<int> last(64, -1);  // last kept gate per qubit
    std::vector<char> dead(g.size(), 0);
    for (size_t i = 0; i < g.size(); i++) {
      if (g[i].op == QS_ID) {
        dead[i] = 1;
        changed = true;
        continue;
      }
      int prev = last[g[i].q[0]];
      bool ok = prev >= 0 && self_inverse(g[i].op) && same_qubits(g[prev], g[i]);
      for (int j = 0; ok && j < g[i].nq; j++) ok = last[g[i].q[j]] == prev;
      if (ok) {
        dead[i] = dead[prev] = 1;
        changed = true;
        for (int j = 0; j < g[i].nq; j++) last[g[i].q[j]] = -1;
        // the qubits' previous gates are unknown now: be conservative
        continue;
      }
      for (int j = 0; j < g[i].nq; j++) last[g[i].q[j]] = (int)i;
    }
    std::vector<qs_gate> out;
    out.reserve(g.size());
    for (size_t i = 0; i < g.size(); i++)
      if (!dead[i]) out.push_back(g[i]);
    g.swap(out);
  }
  return g;
}

}  // namespace

std::vector<qs_gate> fold_rotations(int n, const qs_gate *in, size_t n_in) {
  const size_t words = (size_t)(n + n_in + 63) / 64 + 1;  // one variable per wire opening
  std::vector<Wire> wire(n);
  int next_var = 0;
  auto fresh = [&](int w) {
    wire[w].par.assign(words, 0);
    wire[w].par[next_var / 64] |= 1ull << (next_var % 64);
    wire[w].cst = 0;
    next_var++;
  };
  for (int w = 0; w < n; w++) fresh(w);
  std::vector<qs_gate> out;
  std::vector<char> drop;
  std::map<Bits, int> open_term;  // parity -> index into terms
  std::vector<Term> terms;
  double gphase = 0;

  auto close_lost = [&](int w) {
    // w's value leaves the span: close the terms whose parity no longer fits
    std::vector<Bits> rows;
    for (int x = 0; x < n; x++)
      if (x != w) rows.push_back(wire[x].par);
    for (auto it = open_term.begin(); it != open_term.end();) {
      if (!in_span(rows, it->first)) {
        terms[it->second].open = false;
        it = open_term.erase(it);
      } else {
        ++it;
      }
    }
  };

  for (size_t i = 0; i < n_in; i++) {
    const qs_gate &g = in[i];
    double a, gp;
    if (g.nq == 1 && phase_angle(g, a, gp)) {
      const int w = g.q[0];
      gphase += gp;
      const Wire &W = wire[w];
      double ang = W.cst ? -a : a;  // e^{ia(P^1)} = e^{ia} e^{-iaP}
      if (W.cst) gphase += a;
      auto it = open_term.find(W.par);
      if (it != open_term.end()) {
        terms[it->second].angle += ang;
        continue;
      }
      Term t;
      t.out_index = out.size();
      t.wire = w;
      t.cst = W.cst;
      t.angle = ang;
      open_term[W.par] = (int)terms.size();
      terms.push_back(t);
      out.push_back(g);  // replaced at the end by the merged gate
      continue;
    }
    if (g.op == QS_RZZ) {
      // e^{-it/2} e^{it (x_a ^ x_b)}: a phase on the XOR of two wires; it is
      // kept as a gate (nothing to merge it into unless a wire holds that
      // parity), but it changes no wire value
      out.push_back(g);
      continue;
    }
    if (g.op == QS_CX) {
      const int c = g.q[0], t = g.q[1];
      for (size_t k = 0; k < words; k++) wire[t].par[k] ^= wire[c].par[k];
      wire[t].cst ^= wire[c].cst;
      out.push_back(g);
      continue;
    }
    if (g.op == QS_X) {
      wire[g.q[0]].cst ^= 1;
      out.push_back(g);
      continue;
    }
    if (g.op == QS_SWAP) {
      std::swap(wire[g.q[0]], wire[g.q[1]]);
      out.push_back(g);
      continue;
    }
    if (op_info(g.op).diagonal) {  // CPhase, CZ, CRZ, CU1, ID, two-qubit phases
      out.push_back(g);
      continue;
    }
    // any other gate: its wires get fresh variables after their current
    // values leave the span
    for (int j = 0; j < g.nq; j++) {
      close_lost(g.q[j]);
      fresh(g.q[j]);
    }
    out.push_back(g);
  }
  // write the merged phases at their first occurrences; drop zero angles
  drop.assign(out.size(), 0);
  for (const Term &t : terms) {
    // on a wire holding P ^ 1 the gate diag(1, e^{-iA}) gives e^{-iA} e^{iAP}:
    // the missing e^{iA} joins the global phase correction
    const double emit = t.cst ? -t.angle : t.angle;
    if (t.cst) gphase += t.angle;
    if (std::fabs(wrap(emit)) < 1e-12) {
      drop[t.out_index] = 1;
      continue;
    }
    out[t.out_index] = phase_gate(t.wire, emit);
  }
  std::vector<qs_gate> res;
  for (size_t i = 0; i < out.size(); i++)
    if (!drop[i]) res.push_back(out[i]);
  res = cancel_pairs(res);
  const double gw = wrap(gphase);
  if (std::fabs(gw) > 1e-12 && n > 0) {
    qs_gate u;
    std::memset(&u, 0, sizeof(u));
    u.op = QS_U1;
    u.nq = 1;
    u.p[0] = 2 * gw;
    qs_gate r = u;
    r.op = QS_RZ;
    r.p[0] = -2 * gw;
    res.push_back(u);
    res.push_back(r);
  }
  return res;
}

}  // namespace qs
