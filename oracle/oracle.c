/*
 * FP64 CPU oracle for the state-vector simulator -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load this file's library. The product path never calls it, and it
 * shares no code with the CUDA library: it has its own parser, its own gate
 * table and its own apply loop.
 *
 * What it computes is the plain definition of Schroedinger-style (full-state)
 * simulation, Sec. II-B: the 2^n complex amplitudes are kept in memory and
 * updated gate by gate, psi <- G_k psi, in the circuit's order, in complex128.
 * SWAP gates are applied as real amplitude exchanges. Alongside, the oracle
 * composes the SWAP transpositions into the logical->physical qubit map that
 * the virtual-swap optimisation (Sec. III-D, "Virtual swap") must report.
 *
 * Conventions (readings of the paper, which never defines them):
 *  - qubit q_i is bit i of the basis index (little-endian);
 *  - gate matrices follow the OpenQASM 2 qelib1 definitions; RZ is
 *    exp(-i theta Z / 2) (global phase kept), U1 = diag(1, e^{i lambda});
 *  - in "name(p) q[a],q[b],..." controls come first, then targets;
 *  - within a multi-target gate the local index is sum_j bit(t_j) << j.
 */
#include <ctype.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double re, im; } cplx;

#define OR_MAX_Q 3
#define OR_MAX_N 40

typedef struct {
  int nc, nt;             /* controls, targets */
  int q[OR_MAX_Q];        /* controls then targets */
  cplx u[16];             /* target unitary, row-major, (2^nt)^2 */
  int is_swap;
} ogate;

static cplx C(double re, double im) { cplx z = {re, im}; return z; }
static cplx cexp_i(double a) { return C(cos(a), sin(a)); }

/* Target unitary of a named gate. Returns 0 on success. */
static int gate_table(const char *name, const double *p, int *nc, int *nt, cplx *u) {
  const double r2 = 1.0 / sqrt(2.0);
  memset(u, 0, sizeof(cplx) * 16);
  *nc = 0; *nt = 1;
  /* one-qubit bases; controlled variants reuse them */
  const char *base = name;
  if (!strcmp(name, "cp") || !strcmp(name, "cu1")) { *nc = 1; base = "u1"; }
  else if (!strcmp(name, "cx")) { *nc = 1; base = "x"; }
  else if (!strcmp(name, "cy")) { *nc = 1; base = "y"; }
  else if (!strcmp(name, "cz")) { *nc = 1; base = "z"; }
  else if (!strcmp(name, "ch")) { *nc = 1; base = "h"; }
  else if (!strcmp(name, "crx")) { *nc = 1; base = "rx"; }
  else if (!strcmp(name, "cry")) { *nc = 1; base = "ry"; }
  else if (!strcmp(name, "crz")) { *nc = 1; base = "rz"; }
  else if (!strcmp(name, "cu3")) { *nc = 1; base = "u3"; }
  else if (!strcmp(name, "ccx")) { *nc = 2; base = "x"; }
  else if (!strcmp(name, "cswap")) { *nc = 1; base = "swap"; }

  if (!strcmp(base, "h")) { u[0] = C(r2, 0); u[1] = C(r2, 0); u[2] = C(r2, 0); u[3] = C(-r2, 0); }
  else if (!strcmp(base, "x")) { u[1] = C(1, 0); u[2] = C(1, 0); }
  else if (!strcmp(base, "y")) { u[1] = C(0, -1); u[2] = C(0, 1); }
  else if (!strcmp(base, "z")) { u[0] = C(1, 0); u[3] = C(-1, 0); }
  else if (!strcmp(base, "id")) { u[0] = C(1, 0); u[3] = C(1, 0); }
  else if (!strcmp(base, "s")) { u[0] = C(1, 0); u[3] = C(0, 1); }
  else if (!strcmp(base, "sdg")) { u[0] = C(1, 0); u[3] = C(0, -1); }
  else if (!strcmp(base, "t")) { u[0] = C(1, 0); u[3] = cexp_i(M_PI / 4); }
  else if (!strcmp(base, "tdg")) { u[0] = C(1, 0); u[3] = cexp_i(-M_PI / 4); }
  else if (!strcmp(base, "sx")) { u[0] = C(.5, .5); u[1] = C(.5, -.5); u[2] = C(.5, -.5); u[3] = C(.5, .5); }
  else if (!strcmp(base, "sxdg")) { u[0] = C(.5, -.5); u[1] = C(.5, .5); u[2] = C(.5, .5); u[3] = C(.5, -.5); }
  else if (!strcmp(base, "rx")) {
    double c = cos(p[0] / 2), s = sin(p[0] / 2);
    u[0] = C(c, 0); u[1] = C(0, -s); u[2] = C(0, -s); u[3] = C(c, 0);
  } else if (!strcmp(base, "ry")) {
    double c = cos(p[0] / 2), s = sin(p[0] / 2);
    u[0] = C(c, 0); u[1] = C(-s, 0); u[2] = C(s, 0); u[3] = C(c, 0);
  } else if (!strcmp(base, "rz")) { u[0] = cexp_i(-p[0] / 2); u[3] = cexp_i(p[0] / 2); }
  else if (!strcmp(base, "u1")) { u[0] = C(1, 0); u[3] = cexp_i(p[0]); }
  else if (!strcmp(base, "u2") || !strcmp(base, "u3")) {
    double th, ph, la;
    if (!strcmp(base, "u2")) { th = M_PI / 2; ph = p[0]; la = p[1]; }
    else { th = p[0]; ph = p[1]; la = p[2]; }
    double c = cos(th / 2), s = sin(th / 2);
    cplx el = cexp_i(la), ep = cexp_i(ph), epl = cexp_i(ph + la);
    u[0] = C(c, 0);
    u[1] = C(-el.re * s, -el.im * s);
    u[2] = C(ep.re * s, ep.im * s);
    u[3] = C(epl.re * c, epl.im * c);
  } else if (!strcmp(base, "swap")) {
    *nt = 2;
    u[0 * 4 + 0] = C(1, 0); u[1 * 4 + 2] = C(1, 0); u[2 * 4 + 1] = C(1, 0); u[3 * 4 + 3] = C(1, 0);
  } else if (!strcmp(base, "rzz")) {
    *nt = 2;
    cplx a = cexp_i(-p[0] / 2), b = cexp_i(p[0] / 2);
    u[0] = a; u[5] = b; u[10] = b; u[15] = a;
  } else if (!strcmp(base, "rxx")) {
    *nt = 2;
    double c = cos(p[0] / 2), s = sin(p[0] / 2);
    for (int l = 0; l < 4; l++) { u[l * 4 + l] = C(c, 0); u[l * 4 + (l ^ 3)] = C(0, -s); }
  } else if (!strcmp(base, "ryy")) {
    *nt = 2;
    double c = cos(p[0] / 2), s = sin(p[0] / 2);
    for (int l = 0; l < 4; l++) u[l * 4 + l] = C(c, 0);
    u[0 * 4 + 3] = C(0, s); u[3 * 4 + 0] = C(0, s);
    u[1 * 4 + 2] = C(0, -s); u[2 * 4 + 1] = C(0, -s);
  } else {
    return -1;
  }
  return 0;
}

static int n_params_of(const char *name) {
  static const char *one[] = {"rx", "ry", "rz", "cp", "cu1", "crx", "cry", "crz", "u1", "rzz", "rxx", "ryy"};
  for (size_t i = 0; i < sizeof(one) / sizeof(one[0]); i++) if (!strcmp(name, one[i])) return 1;
  if (!strcmp(name, "u2")) return 2;
  if (!strcmp(name, "u3") || !strcmp(name, "cu3")) return 3;
  return 0;
}

/* ---- parser: OpenQASM-2 subset, one gate per statement ---- */

static const char *skip_ws(const char *s) {
  for (;;) {
    while (*s && isspace((unsigned char)*s)) s++;
    if (s[0] == '/' && s[1] == '/') { while (*s && *s != '\n') s++; continue; }
    return s;
  }
}

/* Parses "q[<int>]"; returns pointer after it or NULL. */
static const char *parse_qref(const char *s, int *q) {
  s = skip_ws(s);
  if (*s != 'q') return NULL;
  s = skip_ws(s + 1);
  if (*s != '[') return NULL;
  char *end;
  long v = strtol(s + 1, &end, 10);
  if (end == s + 1) return NULL;
  s = skip_ws(end);
  if (*s != ']') return NULL;
  *q = (int)v;
  return s + 1;
}

/* Parses the whole text. gates may be NULL (count only). Returns 0 or -line. */
static int parse(const char *text, int *n_out, ogate *gates, int cap, int *count) {
  const char *s = text;
  int n = -1, cnt = 0, line = 0;
  while (1) {
    s = skip_ws(s);
    if (!*s) break;
    line++;
    char name[16];
    int len = 0;
    while (*s && (isalnum((unsigned char)*s) || *s == '_' || *s == '.')) {
      if (len < 15) name[len++] = (char)tolower((unsigned char)*s);
      s++;
    }
    name[len] = 0;
    if (len == 0) return -line;
    if (!strcmp(name, "openqasm")) { while (*s && *s != ';') s++; if (*s) s++; continue; }
    if (!strcmp(name, "include")) { while (*s && *s != ';') s++; if (*s) s++; continue; }
    if (!strcmp(name, "qreg")) {
      int v;
      const char *t = parse_qref(s, &v);
      if (!t) return -line;
      s = skip_ws(t);
      if (*s != ';') return -line;
      s++;
      n = v;
      continue;
    }
    double p[3] = {0, 0, 0};
    int np = 0;
    s = skip_ws(s);
    if (*s == '(') {
      s++;
      while (1) {
        char *end;
        s = skip_ws(s);
        double v = strtod(s, &end);
        if (end == s) return -line;
        if (np >= 3) return -line;
        p[np++] = v;
        s = skip_ws(end);
        if (*s == ',') { s++; continue; }
        if (*s == ')') { s++; break; }
        return -line;
      }
    }
    if (np != n_params_of(name)) return -line;
    ogate g;
    memset(&g, 0, sizeof(g));
    if (gate_table(name, p, &g.nc, &g.nt, g.u)) return -line;
    g.is_swap = !strcmp(name, "swap");
    int nq = g.nc + g.nt, got = 0;
    while (got < nq) {
      int q;
      const char *t = parse_qref(s, &q);
      if (!t) return -line;
      if (n < 0 || q < 0 || q >= n) return -line;
      for (int j = 0; j < got; j++) if (g.q[j] == q) return -line;
      g.q[got++] = q;
      s = skip_ws(t);
      if (got < nq) { if (*s != ',') return -line; s++; }
    }
    if (*s != ';') return -line;
    s++;
    if (gates) { if (cnt >= cap) return -line; gates[cnt] = g; }
    cnt++;
  }
  if (n <= 0 || n > OR_MAX_N) return -1;
  *n_out = n;
  *count = cnt;
  return 0;
}

/* psi <- G psi for one gate: every index with all target bits 0 and all
 * control bits 1 is the base of one group of 2^nt amplitudes. */
static void apply_gate(cplx *psi, int n, const ogate *g) {
  const long long N = 1LL << n;
  long long tmask = 0, cmask = 0;
  for (int j = 0; j < g->nc; j++) cmask |= 1LL << g->q[j];
  for (int j = 0; j < g->nt; j++) tmask |= 1LL << g->q[g->nc + j];
  const int d = 1 << g->nt;
#pragma omp parallel for schedule(static)
  for (long long i = 0; i < N; i++) {
    if ((i & tmask) != 0 || (i & cmask) != cmask) continue;
    long long idx[4];
    cplx v[4], w[4];
    for (int l = 0; l < d; l++) {
      long long k = i;
      for (int j = 0; j < g->nt; j++) if ((l >> j) & 1) k |= 1LL << g->q[g->nc + j];
      idx[l] = k;
      v[l] = psi[k];
    }
    for (int r = 0; r < d; r++) {
      double re = 0, im = 0;
      for (int c = 0; c < d; c++) {
        cplx m = g->u[r * d + c];
        re += m.re * v[c].re - m.im * v[c].im;
        im += m.re * v[c].im + m.im * v[c].re;
      }
      w[r] = C(re, im);
    }
    for (int l = 0; l < d; l++) psi[idx[l]] = w[l];
  }
}

/* ---- exported entry points ---- */

/* Number of qubits and gates in a circuit text; 0 on success. */
int oracle_count(const char *text, int *n_out, int *gates_out) {
  return parse(text, n_out, NULL, 0, gates_out);
}

/* Simulates `text`. out: 2*2^n doubles (re, im interleaved), logical order.
 * init: optional initial state (same layout); NULL means |0...0>.
 * perm_out: n ints, logical qubit -> physical bit after absorbing every SWAP
 * as a relabelling (composition of the SWAP transpositions).
 * nthreads <= 0 keeps the OpenMP default; a positive count holds for this call
 * only. Returns 0 or a negative error. */
int oracle_simulate(const char *text, int n_expected, const double *init, double *out,
                    int *perm_out, int nthreads) {
  int n = 0, count = 0;
  int rc = parse(text, &n, NULL, 0, &count);
  if (rc) return rc;
  if (n != n_expected) return -1000;
  ogate *gates = (ogate *)malloc(sizeof(ogate) * (count ? count : 1));
  if (!gates) return -1001;
  rc = parse(text, &n, gates, count, &count);
  if (rc) { free(gates); return rc; }
#ifdef _OPENMP
  const int prev_threads = omp_get_max_threads();
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  const long long N = 1LL << n;
  cplx *psi = (cplx *)out;
  if (init) memcpy(psi, init, sizeof(cplx) * N);
  else {
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < N; i++) psi[i] = C(0, 0);
    psi[0] = C(1, 0);
  }
  int perm[OR_MAX_N];
  for (int q = 0; q < n; q++) perm[q] = q;
  for (int k = 0; k < count; k++) {
    apply_gate(psi, n, &gates[k]);
    if (gates[k].is_swap) {
      int a = gates[k].q[0], b = gates[k].q[1];
      int t = perm[a]; perm[a] = perm[b]; perm[b] = t;
    }
  }
  if (perm_out) for (int q = 0; q < n; q++) perm_out[q] = perm[q];
  free(gates);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(prev_threads);  /* the count applies to this call only */
#endif
  return 0;
}

/* Target unitary of one named gate: out = (2^nt)^2 complex (row-major,
 * re/im interleaved). Returns 0, or -1 for an unknown name. */
int oracle_gate_matrix(const char *name, const double *params, double *out, int *n_ctrl,
                       int *n_targ) {
  double p[3] = {0, 0, 0};
  int np = n_params_of(name);
  for (int i = 0; i < np; i++) p[i] = params[i];
  cplx u[16];
  int nc, nt;
  if (gate_table(name, p, &nc, &nt, u)) return -1;
  int d = 1 << nt;
  for (int i = 0; i < d * d; i++) { out[2 * i] = u[i].re; out[2 * i + 1] = u[i].im; }
  *n_ctrl = nc;
  *n_targ = nt;
  return 0;
}

/* Marginal probabilities of m logical qubits: out[b] = sum over i whose bit
 * qubits[j] equals bit j of b, of |psi_i|^2 (2^m doubles). */
int oracle_probs(const double *state, int n, const int *qubits, int m, double *out) {
  const long long N = 1LL << n;
  const cplx *psi = (const cplx *)state;
  for (long long b = 0; b < (1LL << m); b++) out[b] = 0.0;
  for (long long i = 0; i < N; i++) {
    long long b = 0;
    for (int j = 0; j < m; j++) b |= ((i >> qubits[j]) & 1LL) << j;
    out[b] += psi[i].re * psi[i].re + psi[i].im * psi[i].im;
  }
  return 0;
}

/* Threads the OpenMP runtime would use (for reporting). */
int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
