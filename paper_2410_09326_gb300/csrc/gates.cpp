// Gate table and OpenQASM-2 subset parser of the library (IR ingest).
//
// The paper names its gates (Sec. III-C counters: H, S, T, X, U, CPhase, CU1,
// SWAP, ...) but does not define them; the matrices here are the OpenQASM 2
// qelib1 definitions, RZ(t) = diag(e^{-it/2}, e^{it/2}).
#include <cctype>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "qs_internal.h"

namespace qs {

static const OpInfo kOps[QS_N_GATE_TYPES] = {
    {"h", 1, 0, 0, false},     {"s", 1, 0, 0, true},      {"t", 1, 0, 0, true},
    {"x", 1, 0, 0, false},     {"y", 1, 0, 0, false},     {"z", 1, 0, 0, true},
    {"sdg", 1, 0, 0, true},    {"tdg", 1, 0, 0, true},    {"rx", 1, 1, 0, false},
    {"ry", 1, 1, 0, false},    {"rz", 1, 1, 0, true},     {"cp", 2, 1, 1, true},
    {"cu1", 2, 1, 1, true},    {"swap", 2, 0, 0, false},  {"cx", 2, 0, 1, false},
    {"cz", 2, 0, 1, true},     {"cy", 2, 0, 1, false},    {"ch", 2, 0, 1, false},
    {"crx", 2, 1, 1, false},   {"cry", 2, 1, 1, false},   {"crz", 2, 1, 1, true},
    {"u1", 1, 1, 0, true},     {"u2", 1, 2, 0, false},    {"u3", 1, 3, 0, false},
    {"sx", 1, 0, 0, false},    {"sxdg", 1, 0, 0, false},  {"id", 1, 0, 0, true},
    {"rzz", 2, 1, 0, true},    {"rxx", 2, 1, 0, false},   {"ryy", 2, 1, 0, false},
    {"ccx", 3, 0, 2, false},   {"cswap", 3, 0, 1, false}, {"cu3", 2, 3, 1, false},
};

const OpInfo &op_info(int op) { return kOps[op]; }

int op_by_name(const char *name) {
  for (int i = 0; i < QS_N_GATE_TYPES; i++)
    if (!std::strcmp(kOps[i].name, name)) return i;
  return -1;
}

namespace {

cd expi(double a) { return cd(std::cos(a), std::sin(a)); }

// 2x2 target matrix of a one-target op (after stripping controls).
void one_target(int op, const double *p, cd u[4]) {
  const double r = 1.0 / std::sqrt(2.0);
  const cd I(0, 1);
  u[0] = u[1] = u[2] = u[3] = 0;
  switch (op) {
    case QS_H: case QS_CH: u[0] = r; u[1] = r; u[2] = r; u[3] = -r; break;
    case QS_X: case QS_CX: case QS_CCX: u[1] = 1; u[2] = 1; break;
    case QS_Y: case QS_CY: u[1] = -I; u[2] = I; break;
    case QS_Z: case QS_CZ: u[0] = 1; u[3] = -1; break;
    case QS_ID: u[0] = 1; u[3] = 1; break;
    case QS_S: u[0] = 1; u[3] = I; break;
    case QS_SDG: u[0] = 1; u[3] = -I; break;
    case QS_T: u[0] = 1; u[3] = expi(M_PI / 4); break;
    case QS_TDG: u[0] = 1; u[3] = expi(-M_PI / 4); break;
    case QS_SX: u[0] = cd(.5, .5); u[1] = cd(.5, -.5); u[2] = cd(.5, -.5); u[3] = cd(.5, .5); break;
    case QS_SXDG: u[0] = cd(.5, -.5); u[1] = cd(.5, .5); u[2] = cd(.5, .5); u[3] = cd(.5, -.5); break;
    case QS_RX: case QS_CRX: {
      double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
      u[0] = c; u[1] = -I * s; u[2] = -I * s; u[3] = c;
      break;
    }
    case QS_RY: case QS_CRY: {
      double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
      u[0] = c; u[1] = -s; u[2] = s; u[3] = c;
      break;
    }
    case QS_RZ: case QS_CRZ: u[0] = expi(-p[0] / 2); u[3] = expi(p[0] / 2); break;
    case QS_U1: case QS_CPHASE: case QS_CU1: u[0] = 1; u[3] = expi(p[0]); break;
    case QS_U2: case QS_U3: case QS_CU3: {
      double th = op == QS_U2 ? M_PI / 2 : p[0];
      double ph = op == QS_U2 ? p[0] : p[1];
      double la = op == QS_U2 ? p[1] : p[2];
      double c = std::cos(th / 2), s = std::sin(th / 2);
      u[0] = c; u[1] = -expi(la) * s; u[2] = expi(ph) * s; u[3] = expi(ph + la) * c;
      break;
    }
    default: break;
  }
}

}  // namespace

void gate_full_matrix(const qs_gate &g, std::vector<cd> &out) {
  const OpInfo &info = kOps[g.op];
  const int nq = info.nq, nc = info.nctrl, d = 1 << nq;
  out.assign((size_t)d * d, cd(0, 0));
  // two-target ops: local target index l = bit(t0) + 2 bit(t1)
  cd t2[16];
  int nt = nq - nc;
  if (nt == 2) {
    for (auto &z : t2) z = 0;
    if (g.op == QS_SWAP || g.op == QS_CSWAP) {
      t2[0] = 1; t2[1 * 4 + 2] = 1; t2[2 * 4 + 1] = 1; t2[15] = 1;
    } else if (g.op == QS_RZZ) {
      cd a = expi(-g.p[0] / 2), b = expi(g.p[0] / 2);
      t2[0] = a; t2[5] = b; t2[10] = b; t2[15] = a;
    } else if (g.op == QS_RXX || g.op == QS_RYY) {
      double c = std::cos(g.p[0] / 2), s = std::sin(g.p[0] / 2);
      for (int l = 0; l < 4; l++) t2[l * 5] = c;
      // exp(-i t/2 P(x)P) = cos - i sin P(x)P; XX flips both bits with +1,
      // YY does so with -1 when the bits are equal and +1 otherwise.
      for (int l = 0; l < 4; l++) {
        int f = l ^ 3;
        double sign = (g.op == QS_RXX) ? 1.0 : ((l == 0 || l == 3) ? -1.0 : 1.0);
        t2[f * 4 + l] = cd(0, -s * sign);
      }
    }
  } else {
    cd u[4];
    one_target(g.op, g.p, u);
    for (int i = 0; i < 4; i++) t2[i] = u[i];
  }
  const int dt = 1 << nt;
  const int cm = (1 << nc) - 1;
  for (int col = 0; col < d; col++) {
    if ((col & cm) != cm) {
      out[(size_t)col * d + col] = 1;
      continue;
    }
    int tc = col >> nc;
    for (int tr = 0; tr < dt; tr++) out[(size_t)((tr << nc) | cm) * d + col] = t2[tr * dt + tc];
  }
}

bool gate_diag_on(const qs_gate &g, int j) {
  const OpInfo &info = kOps[g.op];
  return info.diagonal || j < info.nctrl;
}

}  // namespace qs

// ---------------------------------------------------------------------------
// Parser
// ---------------------------------------------------------------------------
namespace {

struct Cursor {
  const char *s;
  int line = 1;
  void ws() {
    for (;;) {
      while (*s && std::isspace((unsigned char)*s)) {
        if (*s == '\n') line++;
        s++;
      }
      if (s[0] == '/' && s[1] == '/') {
        while (*s && *s != '\n') s++;
        continue;
      }
      return;
    }
  }
  bool eat(char c) {
    ws();
    if (*s != c) return false;
    s++;
    return true;
  }
  bool qref(long *q) {
    ws();
    if (*s != 'q') return false;
    s++;
    if (!eat('[')) return false;
    ws();
    char *end;
    long v = std::strtol(s, &end, 10);
    if (end == s) return false;
    s = end;
    if (!eat(']')) return false;
    *q = v;
    return true;
  }
};

}  // namespace

namespace qs {
std::string &last_error_ref();
}

extern "C" qs_status qs_parse_qasm(const char *text, int *n_qubits, qs_gate *gates, size_t cap,
                                   size_t *n_gates) {
  using namespace qs;
  if (!text || !n_qubits || !n_gates) {
    last_error_ref() = "qs_parse_qasm: null argument";
    return QS_EINVAL;
  }
  Cursor c{text};
  long n = -1;
  size_t cnt = 0;
  auto fail = [&](const char *what) {
    last_error_ref() = std::string("qs_parse_qasm: line ") + std::to_string(c.line) + ": " + what;
    return QS_EINVAL;
  };
  for (;;) {
    c.ws();
    if (!*c.s) break;
    char name[16];
    int len = 0;
    while (*c.s && (std::isalnum((unsigned char)*c.s) || *c.s == '_' || *c.s == '.')) {
      if (len < 15) name[len++] = (char)std::tolower((unsigned char)*c.s);
      c.s++;
    }
    name[len] = 0;
    if (!len) return fail("expected a statement");
    if (!std::strcmp(name, "openqasm") || !std::strcmp(name, "include")) {
      while (*c.s && *c.s != ';') c.s++;
      if (!c.eat(';')) return fail("missing ';'");
      continue;
    }
    if (!std::strcmp(name, "qreg")) {
      if (!c.qref(&n)) return fail("bad qreg");
      if (!c.eat(';')) return fail("missing ';'");
      if (n <= 0 || n > QS_MAX_QUBITS) return fail("register size out of range");
      continue;
    }
    int op = op_by_name(name);
    if (op < 0) return fail("unknown gate");
    const OpInfo &info = op_info(op);
    qs_gate g;
    std::memset(&g, 0, sizeof(g));
    g.op = (uint8_t)op;
    g.nq = (uint8_t)info.nq;
    int np = 0;
    c.ws();
    if (*c.s == '(') {
      c.s++;
      for (;;) {
        c.ws();
        char *end;
        double v = std::strtod(c.s, &end);
        if (end == c.s) return fail("bad parameter");
        if (np >= 3) return fail("too many parameters");
        g.p[np++] = v;
        c.s = end;
        if (c.eat(',')) continue;
        if (c.eat(')')) break;
        return fail("bad parameter list");
      }
    }
    if (np != info.nparams) return fail("wrong parameter count");
    if (n < 0) return fail("gate before qreg");
    for (int j = 0; j < info.nq; j++) {
      long q;
      if (j && !c.eat(',')) return fail("expected ','");
      if (!c.qref(&q)) return fail("bad qubit reference");
      if (q < 0 || q >= n) return fail("qubit out of range");
      for (int i = 0; i < j; i++)
        if (g.q[i] == q) return fail("duplicate qubit");
      g.q[j] = (uint8_t)q;
    }
    if (!c.eat(';')) return fail("missing ';'");
    if (gates && cnt < cap) gates[cnt] = g;
    cnt++;
  }
  if (n < 0) return fail("no qreg");
  *n_qubits = (int)n;
  *n_gates = cnt;
  if (cnt > cap) {
    last_error_ref() = "qs_parse_qasm: buffer too small";
    return QS_EINVAL;
  }
  return QS_OK;
}
