// Host passes: virtual swap, k-qubit fusion and block classification.
//
// Virtual swap (Sec. III-D): a SWAP gate exchanges two qubits' roles; instead
// of moving 2^(n-1) amplitudes, the pass swaps the two entries of the
// logical->physical map and later gates are renamed through it.
//
// Fusion generalises single-qubit gate merging (Sec. III-D, Z-Y
// decomposition: consecutive one-qubit gates collapse into one unitary) and
// QCOR's two-qubit block merging (Sec. IV, "all-on" set) to blocks of up to k
// qubits whose product matrix is formed in FP64 on the host.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>

#include "qs_internal.h"

namespace qs {

namespace {

constexpr double kEps = 1e-14;

bool is_one(cd z) { return std::abs(z - cd(1, 0)) <= kEps; }
bool is_zero(cd z) { return std::abs(z) <= kEps; }

int popcount64(uint64_t x) { return __builtin_popcountll(x); }

// Position of physical qubit q inside the sorted list qs[0..w).
int pos_of(const int *qs, int w, int q) {
  for (int i = 0; i < w; i++)
    if (qs[i] == q) return i;
  return -1;
}

// Applies a gate's full matrix G (on local positions pos[0..m)) from the left
// to every column of the block matrix M (2^w x 2^w, row-major).
void left_multiply(std::vector<cd> &M, int w, const std::vector<cd> &G, const int *pos, int m) {
  const int d = 1 << w, dg = 1 << m;
  int gmask = 0;
  for (int j = 0; j < m; j++) gmask |= 1 << pos[j];
  std::vector<cd> v(dg), r(dg);
  for (int col = 0; col < d; col++) {
    for (int base = 0; base < d; base++) {
      if (base & gmask) continue;
      for (int l = 0; l < dg; l++) {
        int idx = base;
        for (int j = 0; j < m; j++)
          if ((l >> j) & 1) idx |= 1 << pos[j];
        v[l] = M[(size_t)idx * d + col];
      }
      for (int a = 0; a < dg; a++) {
        cd acc = 0;
        for (int b = 0; b < dg; b++) acc += G[(size_t)a * dg + b] * v[b];
        r[a] = acc;
      }
      for (int l = 0; l < dg; l++) {
        int idx = base;
        for (int j = 0; j < m; j++)
          if ((l >> j) & 1) idx |= 1 << pos[j];
        M[(size_t)idx * d + col] = r[l];
      }
    }
  }
}

// Runs f(0..n) on up to 16 host threads when the work is large enough to pay
// for them (block products are independent once the grouping is fixed).
template <typename F> void parallel_for(size_t n, F f) {
  unsigned nt = std::min(16u, std::max(1u, std::thread::hardware_concurrency()));
  if (n < 16 || nt <= 1) {
    for (size_t i = 0; i < n; i++) f(i);
    return;
  }
  if (nt > n / 4) nt = (unsigned)std::max<size_t>(1, n / 4);
  std::atomic<size_t> next{0};
  std::vector<std::thread> th;
  th.reserve(nt);
  for (unsigned t = 0; t < nt; t++)
    th.emplace_back([&] {
      for (size_t i; (i = next.fetch_add(1)) < n;) f(i);
    });
  for (auto &x : th) x.join();
}

// f(0..n) for a handful of independent tasks, one host thread each.
template <typename F> void run_tasks(size_t n, F f) {
  std::vector<std::thread> th;
  for (size_t i = 1; i < n; i++) th.emplace_back([&f, i] { f(i); });
  if (n > 0) f(0);
  for (auto &t : th) t.join();
}

struct Pending {
  std::vector<int> members;  // indices into the physical gate list
  uint64_t qmask = 0;
  bool all_diag = true;
  uint64_t tmask = 0;       // qubits some member acts on non-diagonally
  uint64_t out_union = 0;   // tile sub-groups: member qubits outside the tile
  uint64_t cl_and = ~0ull;  // tile sub-groups: qubits every member is the identity on when 0
};

// Commuting greedy grouping of the gates pg[idx[..]] (ascending list order):
// a gate may join any group at or after the last group it cannot commute
// past (two gates commute when both act diagonally on every qubit they
// share); it joins the first such group `fits` accepts, else a new one.
struct NoJoin {
  void operator()(Pending &, int, uint64_t) const {}
};

template <typename Fits, typename Joined = NoJoin>
void greedy_groups(const std::vector<qs_gate> &pg, const std::vector<int> &idx, std::vector<Pending> &groups,
                   Fits fits, Joined joined = Joined()) {
  std::vector<int> last_any(64, -1), last_nd(64, -1);
  for (int i : idx) {
    const qs_gate &g = pg[i];
    uint64_t gmask = 0, gt = 0;
    int lower = -1;
    for (int j = 0; j < g.nq; j++) {
      const int q = g.q[j];
      gmask |= 1ull << q;
      if (!gate_diag_on(g, j)) gt |= 1ull << q;
      lower = std::max(lower, gate_diag_on(g, j) ? last_nd[q] : last_any[q]);
    }
    const bool gdiag = op_info(g.op).diagonal;
    int chosen = -1;
    for (int b = std::max(lower, 0); b < (int)groups.size(); b++)
      if (fits(groups[b], i, gmask, gt, gdiag)) {
        chosen = b;
        break;
      }
    if (chosen < 0) {
      groups.emplace_back();
      chosen = (int)groups.size() - 1;
    }
    Pending &p = groups[chosen];
    p.members.push_back(i);
    p.qmask |= gmask;
    p.tmask |= gt;
    p.all_diag = p.all_diag && gdiag;
    joined(p, i, gmask);
    for (int j = 0; j < g.nq; j++) {
      const int q = g.q[j];
      last_any[q] = std::max(last_any[q], chosen);
      if (!gate_diag_on(g, j)) last_nd[q] = std::max(last_nd[q], chosen);
    }
  }
}

// Fusion with a roll-out look-ahead (a pilot method): where a gate could join
// several blocks (the first four that fit) or open a new one, each choice is
// followed by `horizon` gates of plain first-fit placement, and the choice
// whose roll-out ends with the fewest blocks -- then the narrowest recent
// blocks -- is kept; ties keep the earliest candidate (first fit). Placement
// obeys the same commutation rule and width limits as greedy_groups.
// limit(all_diag_block_and_gate) is the width bound.
template <typename Limit>
void lookahead_groups(const std::vector<qs_gate> &pg, const std::vector<int> &idx, std::vector<Pending> &groups,
                      Limit limit, int horizon, int tail_blocks = 6) {
  struct LG {
    uint64_t qmask;
    bool all_diag;
  };
  struct GI {
    uint64_t gmask;
    bool gdiag;
    int nq;
    int q[6];
    bool dq[6];
  };
  const int N = (int)idx.size();
  std::vector<GI> info(N);
  for (int i = 0; i < N; i++) {
    const qs_gate &g = pg[idx[i]];
    GI &x = info[i];
    x.gmask = 0;
    x.gdiag = op_info(g.op).diagonal;
    x.nq = g.nq;
    for (int j = 0; j < g.nq; j++) {
      x.q[j] = g.q[j];
      x.dq[j] = gate_diag_on(g, j);
      x.gmask |= 1ull << g.q[j];
    }
  }
  auto lower_of = [](const GI &x, const int *la, const int *ln) {
    int lower = -1;
    for (int j = 0; j < x.nq; j++) lower = std::max(lower, x.dq[j] ? ln[x.q[j]] : la[x.q[j]]);
    return lower;
  };
  auto fits = [&](const LG &b, const GI &x) {
    return popcount64(b.qmask | x.gmask) <= limit(b.all_diag && x.gdiag);
  };
  auto place = [](std::vector<LG> &G, int *la, int *ln, const GI &x, int ch) {
    if (ch == (int)G.size()) G.push_back({0, true});
    G[ch].qmask |= x.gmask;
    G[ch].all_diag = G[ch].all_diag && x.gdiag;
    for (int j = 0; j < x.nq; j++) {
      la[x.q[j]] = std::max(la[x.q[j]], ch);
      if (!x.dq[j]) ln[x.q[j]] = std::max(ln[x.q[j]], ch);
    }
  };
  std::vector<LG> G, G2;
  int la[64], ln[64], la2[64], ln2[64];
  for (int q = 0; q < 64; q++) la[q] = ln[q] = -1;
  for (int i = 0; i < N; i++) {
    const GI &x = info[i];
    const int lower = std::max(lower_of(x, la, ln), 0);
    int cand[5], nc = 0;
    for (int b = lower; b < (int)G.size() && nc < 4; b++)
      if (fits(G[b], x)) cand[nc++] = b;
    cand[nc++] = (int)G.size();
    int ch = cand[0];
    if (nc > 1 && horizon > 0) {
      long best_blocks = -1, best_tail = 0;
      for (int c = 0; c < nc; c++) {
        G2 = G;
        std::memcpy(la2, la, sizeof(la));
        std::memcpy(ln2, ln, sizeof(ln));
        place(G2, la2, ln2, x, cand[c]);
        const int end = std::min(N, i + 1 + horizon);
        for (int j = i + 1; j < end; j++) {
          const GI &y = info[j];
          int b = std::max(lower_of(y, la2, ln2), 0);
          while (b < (int)G2.size() && !fits(G2[b], y)) b++;
          place(G2, la2, ln2, y, b);
        }
        long tail = 0;
        for (int b = std::max(0, (int)G2.size() - tail_blocks); b < (int)G2.size(); b++)
          tail += popcount64(G2[b].qmask);
        if (best_blocks < 0 || (long)G2.size() < best_blocks ||
            ((long)G2.size() == best_blocks && tail < best_tail)) {
          best_blocks = (long)G2.size();
          best_tail = tail;
          ch = cand[c];
        }
      }
    }
    place(G, la, ln, x, ch);
    if (ch == (int)groups.size()) groups.emplace_back();
    Pending &p = groups[ch];
    p.members.push_back(idx[i]);
    p.qmask |= x.gmask;
    p.all_diag = p.all_diag && x.gdiag;
  }
}

// Qubits on which the gate is the identity whenever that qubit is 0 (the
// controls of a controlled gate; both qubits of CZ / CPhase; the qubit of a
// phase gate diag(1, e^{ia})). A block made only of such gates on a qubit has
// that qubit as a detected control.
uint64_t ctrl_like_mask(const qs_gate &g) {
  const OpInfo &oi = op_info(g.op);
  uint64_t m = 0;
  if (!oi.diagonal) {
    for (int j = 0; j < oi.nctrl; j++) m |= 1ull << g.q[j];
    return m;
  }
  std::vector<cd> G;
  gate_full_matrix(g, G);
  const int d = 1 << g.nq;
  for (int j = 0; j < g.nq; j++) {
    bool ok = true;
    for (int l = 0; l < d && ok; l++)
      if (!((l >> j) & 1) && !is_one(G[(size_t)l * d + l])) ok = false;
    if (ok) m |= 1ull << g.q[j];
  }
  return m;
}

// Turns a group of gates into a classified Block (dense/diag/permute);
// returns false when the product is the identity (nothing to launch).
double wrap_angle(double a) {
  a = std::remainder(a, 2 * M_PI);  // [-pi, pi]
  return a <= -M_PI ? a + 2 * M_PI : a;
}

// Phase polynomial of a run of diagonal gates (each on at most two qubits):
// gate g contributes arg g(00) + (arg g(10) - arg g(00)) x_0 +
// (arg g(01) - arg g(00)) x_1 + (arg g(11) - arg g(10) - arg g(01) +
// arg g(00)) x_0 x_1, which equals arg g(x) on all four inputs. Returns false
// when the product is the identity.
bool phase_block(const std::vector<qs_gate> &pg, const Pending &p, const int *qs, int w, Block &out) {
  std::vector<double> a(w, 0.0), b((size_t)w * (w - 1) / 2, 0.0);
  double c = 0;
  std::vector<cd> G;
  for (int gi : p.members) {
    const qs_gate &g = pg[gi];
    gate_full_matrix(g, G);
    const int d = 1 << g.nq;
    double ph[4] = {0, 0, 0, 0};
    for (int l = 0; l < d; l++) ph[l] = std::arg(G[(size_t)l * d + l]);
    const int j0 = pos_of(qs, w, g.q[0]);
    c += ph[0];
    a[j0] += ph[1] - ph[0];
    if (g.nq == 2) {
      const int j1 = pos_of(qs, w, g.q[1]);
      a[j1] += ph[2] - ph[0];
      const double x = ph[3] - ph[1] - ph[2] + ph[0];
      b[j0 < j1 ? tri_index(j0, j1, w) : tri_index(j1, j0, w)] += x;
    }
  }
  // keep the qubits that still carry a term
  auto zero = [](double v) { return std::fabs(wrap_angle(v)) <= kEps; };
  std::vector<char> used(w, 0);
  for (int j = 0; j < w; j++) {
    if (!zero(a[j])) used[j] = 1;
    for (int l = j + 1; l < w; l++)
      if (!zero(b[tri_index(j, l, w)])) used[j] = used[l] = 1;
  }
  std::vector<int> keep;
  for (int j = 0; j < w; j++)
    if (used[j]) keep.push_back(j);
  const int k = (int)keep.size();
  if (k == 0 && zero(c)) return false;
  out.kind = BK_PHASE;
  out.k = k;
  out.ph_c = wrap_angle(c);
  out.ph_q.resize(k);
  out.ph_a.resize(k);
  out.ph_b.assign(k > 1 ? (size_t)k * (k - 1) / 2 : 0, 0.0);
  for (int j = 0; j < k; j++) {
    out.ph_q[j] = qs[keep[j]];
    out.ph_a[j] = wrap_angle(a[keep[j]]);
    for (int l = j + 1; l < k; l++) out.ph_b[tri_index(j, l, k)] = wrap_angle(b[tri_index(keep[j], keep[l], w)]);
  }
  for (int j = 0; j < std::min(k, QS_MAX_DIAG); j++) out.q[j] = out.ph_q[j];
  return true;
}

// table_max: widest diagonal run kept as a phase table; wider all-diagonal
// groups become phase polynomials when phase_ok.
bool finish_block(const std::vector<qs_gate> &pg, const Pending &p, bool allow_permute, Block &out,
                  int table_max = QS_MAX_DIAG, bool phase_ok = false) {
  int qs[64], w = 0;
  for (int q = 0; q < 64; q++)
    if ((p.qmask >> q) & 1) qs[w++] = q;
  out = Block();
  out.n_gates = (int)p.members.size();
  const qs_gate &g0 = pg[p.members[0]];
  if (out.n_gates == 1) {
    out.first_op = g0.op;
    out.meta = g0.op == QS_SWAP ? 3 : (op_info(g0.op).nq == 1 ? 0 : 1);
  }
  if (allow_permute && out.n_gates == 1 && g0.op == QS_SWAP) {
    out.kind = BK_PERMUTE;
    out.k = 2;
    out.q[0] = std::min(g0.q[0], g0.q[1]);
    out.q[1] = std::max(g0.q[0], g0.q[1]);
    return true;
  }
  std::vector<cd> G;
  if (p.all_diag && phase_ok && w > table_max) {
    const int first_op = out.first_op, meta = out.meta, ng = out.n_gates;
    if (!phase_block(pg, p, qs, w, out)) return false;
    out.first_op = first_op;
    out.meta = meta;
    out.n_gates = ng;
    return true;
  }
  if (p.all_diag) {
    // diagonal table over the w qubits: product of every member's diagonal
    std::vector<cd> tab((size_t)1 << w, cd(1, 0));
    for (int gi : p.members) {
      const qs_gate &g = pg[gi];
      gate_full_matrix(g, G);
      int m = g.nq, dg = 1 << m;
      int pos[8];
      for (int j = 0; j < m; j++) pos[j] = pos_of(qs, w, g.q[j]);
      for (size_t l = 0; l < tab.size(); l++) {
        int lg = 0;
        for (int j = 0; j < m; j++) lg |= (int)((l >> pos[j]) & 1) << j;
        tab[l] *= G[(size_t)lg * dg + lg];
      }
    }
    // a qubit whose 0 half carries phase 1 everywhere acts as a control
    uint64_t cmask = 0;
    int keep[64], nk = 0;
    for (int j = 0; j < w; j++) {
      bool ctrl = true;
      for (size_t l = 0; l < tab.size() && ctrl; l++)
        if (!((l >> j) & 1) && !is_one(tab[l])) ctrl = false;
      if (ctrl) cmask |= 1ull << qs[j];
      else keep[nk++] = j;
    }
    int cbits = 0;
    for (int j = 0; j < w; j++)
      if ((cmask >> qs[j]) & 1) cbits |= 1 << j;
    std::vector<cd> t2((size_t)1 << nk);
    bool identity = true;
    for (size_t l2 = 0; l2 < t2.size(); l2++) {
      int l = cbits;
      for (int j = 0; j < nk; j++)
        if ((l2 >> j) & 1) l |= 1 << keep[j];
      t2[l2] = tab[l];
      if (!is_one(t2[l2])) identity = false;
    }
    if (identity) return false;
    out.kind = BK_DIAG;
    out.k = nk;
    for (int j = 0; j < nk; j++) out.q[j] = qs[keep[j]];
    out.cmask = cmask;
    out.nctrl = popcount64(cmask);
    out.mat = std::move(t2);
    return true;
  }
  // dense product over the w qubits
  const int d = 1 << w;
  std::vector<cd> M((size_t)d * d, cd(0, 0));
  for (int i = 0; i < d; i++) M[(size_t)i * d + i] = 1;
  for (int gi : p.members) {
    const qs_gate &g = pg[gi];
    gate_full_matrix(g, G);
    int pos[8];
    for (int j = 0; j < g.nq; j++) pos[j] = pos_of(qs, w, g.q[j]);
    left_multiply(M, w, G, pos, g.nq);
  }
  // control detection: block-diagonal in bit j with identity on the 0 half
  uint64_t cmask = 0;
  int keep[64], nk = 0;
  for (int j = 0; j < w; j++) {
    bool ctrl = true;
    for (int r = 0; r < d && ctrl; r++)
      for (int c = 0; c < d && ctrl; c++) {
        cd z = M[(size_t)r * d + c];
        int br = (r >> j) & 1, bc = (c >> j) & 1;
        if (br != bc) { if (!is_zero(z)) ctrl = false; }
        else if (br == 0) { if (r == c ? !is_one(z) : !is_zero(z)) ctrl = false; }
      }
    if (ctrl) cmask |= 1ull << qs[j];
    else keep[nk++] = j;
  }
  int cbits = 0;
  for (int j = 0; j < w; j++)
    if ((cmask >> qs[j]) & 1) cbits |= 1 << j;
  const int dk = 1 << nk;
  std::vector<cd> R((size_t)dk * dk);
  bool diag = true, identity = true;
  auto expand = [&](int l2) {
    int l = cbits;
    for (int j = 0; j < nk; j++)
      if ((l2 >> j) & 1) l |= 1 << keep[j];
    return l;
  };
  for (int r = 0; r < dk; r++)
    for (int c = 0; c < dk; c++) {
      cd z = M[(size_t)expand(r) * d + expand(c)];
      R[(size_t)r * dk + c] = z;
      if (r != c && !is_zero(z)) diag = false, identity = false;
      if (r == c && !is_one(z)) identity = false;
    }
  if (identity) return false;
  out.cmask = cmask;
  out.nctrl = popcount64(cmask);
  out.k = nk;
  for (int j = 0; j < nk; j++) out.q[j] = qs[keep[j]];
  if (diag && nk <= QS_MAX_DIAG) {
    out.kind = BK_DIAG;
    out.mat.resize(dk);
    for (int i = 0; i < dk; i++) out.mat[i] = R[(size_t)i * dk + i];
  } else {
    out.kind = BK_DENSE;
    out.mat = std::move(R);
  }
  return true;
}

void push_exchanges(const std::vector<std::pair<int, int>> &reloc, std::vector<Block> &plan) {
  for (auto &pr : reloc) {  // the exchanges run first
    Block b;
    b.kind = BK_PERMUTE;
    b.k = 2;
    b.q[0] = std::min(pr.first, pr.second);
    b.q[1] = std::max(pr.first, pr.second);
    b.n_gates = 0;
    b.meta = 3;
    plan.push_back(std::move(b));
  }
}

constexpr int kTileMaxOps = 64;     // member blocks of one tile pass
constexpr int kTilePool = 2048;     // matrix + phase-table entries of one tile pass

// Cache-blocked passes (the GPU analogue of the chunk segment that virtual
// swap keeps hot qubits in, Sec. III-D): gates are grouped, with the same
// commutation rule as fusion, into passes whose non-diagonal qubits fit one
// tile of m qubits that always contains bits 0..kTileLowBits-1. A pass then
// costs one HBM read and write: each CTA loads a tile of 2^m amplitudes
// into shared memory, applies the pass's member blocks there, and stores it.
// Inside a pass the gates are fused again, at most tile_k qubits wide; a
// qubit outside the tile may only be a control or sit in a diagonal block.
qs_status tile_plan(int n, const std::vector<qs_gate> &pg, const std::vector<int> &all, const qs_opts &opts,
                    bool c128, std::vector<Block> &out, std::string &err) {
  const int m = tile_bits_of(opts, c128);
  const int kin = tile_k_of(opts);
  const int D = std::max(1, std::min(opts.diag_max, QS_MAX_DIAG));
  const uint64_t low = (1ull << kTileLowBits) - 1;
  std::vector<Pending> passes;
  greedy_groups(pg, all, passes, [&](const Pending &p, int, uint64_t, uint64_t gt, bool) {
    return popcount64(p.tmask | low | gt) <= m;
  });
  // tile qubits of every pass: its non-diagonal qubits, padded with the
  // lowest free bits (longer contiguous runs per load)
  std::vector<uint64_t> tmask(passes.size());
  for (size_t pi = 0; pi < passes.size(); pi++) {
    uint64_t t = passes[pi].tmask | low;
    for (int q = 0; q < n && popcount64(t) < m; q++) t |= 1ull << q;
    tmask[pi] = t;
  }
  std::vector<uint64_t> cl(pg.size(), 0);
  parallel_for(pg.size(), [&](size_t i) { cl[i] = ctrl_like_mask(pg[i]); });
  // member blocks of every pass
  std::vector<Pending> subs;
  std::vector<int> sub_pass;
  for (size_t pi = 0; pi < passes.size(); pi++) {
    const uint64_t T = tmask[pi];
    std::vector<Pending> sg;
    greedy_groups(
        pg, passes[pi].members, sg,
        [&](const Pending &p, int i, uint64_t gmask, uint64_t, bool gdiag) {
          const int width = popcount64(p.qmask | gmask);
          if (p.all_diag && gdiag) return width <= D;
          // a non-diagonal block may reach outside the tile only through
          // qubits that are controls of every member: then they are
          // detected as controls of the product
          const uint64_t out = p.out_union | (gmask & ~T);
          return width <= kin && (out & ~(p.cl_and & cl[i])) == 0;
        },
        [&](Pending &p, int i, uint64_t gmask) {
          p.out_union |= gmask & ~T;
          p.cl_and &= cl[i];
        });
    for (Pending &p : sg) {
      subs.push_back(std::move(p));
      sub_pass.push_back((int)pi);
    }
  }
  std::vector<Block> done(subs.size());
  std::vector<char> keep(subs.size(), 0);
  parallel_for(subs.size(), [&](size_t i) { keep[i] = finish_block(pg, subs[i], false, done[i]) ? 1 : 0; });
  (void)err;
  size_t si = 0;
  for (size_t pi = 0; pi < passes.size(); pi++) {
    const uint64_t T = tmask[pi];
    std::vector<Block> members;
    for (; si < subs.size() && sub_pass[si] == (int)pi; si++)
      if (keep[si]) members.push_back(std::move(done[si]));
    bool ok = true;
    for (const Block &b : members) {
      if (b.kind == BK_DENSE) {
        ok = ok && b.k <= 4;
        for (int j = 0; j < b.k; j++) ok = ok && ((T >> b.q[j]) & 1);
      } else if (b.kind != BK_DIAG) {
        ok = false;
      }
    }
    if (!ok) {  // cannot happen by construction; the members stay valid alone
      for (Block &b : members) out.push_back(std::move(b));
      continue;
    }
    // split at the shared-memory limits of one pass
    size_t b0 = 0;
    while (b0 < members.size()) {
      size_t b1 = b0;
      int pool = 0;
      while (b1 < members.size() && (int)(b1 - b0) < kTileMaxOps) {
        const Block &b = members[b1];
        const int ent = b.kind == BK_DENSE ? (1 << (2 * b.k)) : (1 << b.k);
        if (b1 > b0 && pool + ent > kTilePool) break;
        pool += ent;
        b1++;
      }
      if (b1 - b0 == 1) {
        out.push_back(std::move(members[b0]));
      } else {
        Block t;
        t.kind = BK_TILE;
        t.k = m;
        int w = 0;
        for (int q = 0; q < 64; q++)
          if ((T >> q) & 1) t.tile_q[w++] = q;
        t.meta = 5;
        t.n_gates = 0;
        for (size_t j = b0; j < b1; j++) {
          t.n_gates += members[j].n_gates;
          t.sub.push_back(std::move(members[j]));
        }
        out.push_back(std::move(t));
      }
      b0 = b1;
    }
  }
  return QS_OK;
}

// Fusion and classification of the physical gates pg[idx...] (one segment
// of the circuit between global-tier exchanges); appends the blocks.
qs_status plan_segment(int n, const std::vector<qs_gate> &pg, const std::vector<int> &all, uint64_t flags,
                       const qs_opts &opts, int D, int K, bool c128, bool allow_phase, std::vector<Block> &plan,
                       std::string &err) {
  const bool fuse = flags & QS_FUSE;
  const bool dfuse = flags & QS_DIAG;
  std::vector<Pending> groups;
  const bool tiled = (flags & QS_TILE) && n > tile_bits_of(opts, c128);
  if (tiled) {
    std::vector<Block> tplan;
    qs_status ts = tile_plan(n, pg, all, opts, c128, tplan, err);
    if (ts != QS_OK) return ts;
    for (Block &b : tplan) plan.push_back(std::move(b));
    return QS_OK;
  }
  if (!fuse && !dfuse) {
    groups.resize(all.size());
    for (size_t i = 0; i < all.size(); i++) {
      const qs_gate &g = pg[all[i]];
      groups[i].members.push_back(all[i]);
      for (int j = 0; j < g.nq; j++) groups[i].qmask |= 1ull << g.q[j];
      groups[i].all_diag = op_info(g.op).diagonal;
    }
  } else {
    // diagonal runs: up to D qubits as a phase table, any width as a phase
    // polynomial (states of at least 11 qubits, which the kernel needs)
    const bool phase_ok = dfuse && allow_phase && n > QS_MAX_DIAG;
    const int dlimit = phase_ok ? 64 : D;
    auto limit = [&](bool nd) { return nd ? (dfuse ? dlimit : std::max(K, 1)) : K; };
    if (opts.fuse_lookahead > 0) {
      // the roll-out heuristic usually saves blocks but is not guaranteed
      // to, and its best horizon and tie-break vary: plain first fit and
      // roll-outs of L, 4L/3 and 5L/3 gates (ties broken by the width of the
      // last 6 or 12 blocks) run side by side on host threads, and the
      // grouping with the fewest blocks is launched (earliest on a tie)
      constexpr int kVariants = 6;
      std::vector<Pending> alt[kVariants];
      const int L = opts.fuse_lookahead;
      const int horizons[kVariants] = {0, L, L, L + L / 3, L + L / 3, L + 2 * L / 3};
      const int tails[kVariants] = {0, 6, 12, 6, 12, 6};
      run_tasks(kVariants, [&](size_t v) {
        if (v == 0)
          greedy_groups(pg, all, alt[0], [&](const Pending &p, int, uint64_t gmask, uint64_t, bool gdiag) {
            return popcount64(p.qmask | gmask) <= limit(p.all_diag && gdiag);
          });
        else
          lookahead_groups(pg, all, alt[v], limit, horizons[v], tails[v]);
      });
      int best = 0;
      for (int v = 1; v < kVariants; v++)
        if (alt[v].size() < alt[best].size()) best = v;
      groups.swap(alt[best]);
    } else {
      greedy_groups(pg, all, groups, [&](const Pending &p, int, uint64_t gmask, uint64_t, bool gdiag) {
        return popcount64(p.qmask | gmask) <= limit(p.all_diag && gdiag);
      });
    }
  }

  // (3) products and classification
  std::vector<Block> done(groups.size());
  std::vector<char> keep(groups.size(), 0);
  const bool phase_ok = dfuse && allow_phase && n > QS_MAX_DIAG;
  parallel_for(groups.size(), [&](size_t i) {
    if (!groups[i].members.empty()) keep[i] = finish_block(pg, groups[i], true, done[i], D, phase_ok) ? 1 : 0;
  });
  for (size_t i = 0; i < groups.size(); i++)
    if (keep[i]) plan.push_back(std::move(done[i]));
  return QS_OK;
}

}  // namespace

void parallel_blocks(size_t n, const std::function<void(size_t)> &f) { parallel_for(n, f); }

int tile_bits_of(const qs_opts &o, bool c128) {
  if (o.tile_bits > 0) return std::min(o.tile_bits, c128 ? kMaxTileBits - 1 : kMaxTileBits);
  return c128 ? 12 : 13;  // 64 KiB of amplitudes
}

int tile_k_of(const qs_opts &o) { return o.tile_k > 0 ? std::min(o.tile_k, 4) : 3; }

void fill_record(const Block &b, int index, int n, int amp_bytes, qs_block_record &r) {
  std::memset(&r, 0, sizeof(r));
  r.index = (int32_t)index;
  r.kind = (uint8_t)b.kind;
  r.k = (uint8_t)b.k;
  r.nctrl = (uint8_t)b.nctrl;
  r.tc = b.tc ? (b.tc_xg ? 2 : 1) : 0;
  for (int j = 0; j < QS_MAX_DIAG; j++) r.qubits[j] = j < b.k ? (int8_t)b.q[j] : (int8_t)-1;
  if (b.kind == BK_TILE)
    for (int j = 0; j < QS_MAX_DIAG; j++)
      r.qubits[j] = kTileLowBits + j < b.k ? (int8_t)b.tile_q[kTileLowBits + j] : (int8_t)-1;
  r.meta = (uint8_t)b.meta;
  r.op = b.n_gates == 1 ? (uint8_t)b.first_op : (uint8_t)255;
  r.n_gates = b.n_gates;
  r.cmask = b.cmask;
  r.bytes = block_bytes(b, n, amp_bytes);
  r.t_start_ms = -1;
  r.ms = -1;
}

double block_bytes(const Block &b, int n, int amp_bytes) {
  double amps = std::ldexp(1.0, n - b.nctrl);
  if (b.kind == BK_PERMUTE || b.kind == BK_GLOBAL) amps = std::ldexp(1.0, n - 1);
  return 2.0 * amps * amp_bytes;
}

qs_status build_plan(int n, const qs_gate *gates, size_t n_gates, uint64_t flags,
                     const qs_opts &opts, int8_t *perm, std::vector<Block> &plan,
                     PlanStats &stats, std::string &err, bool c128, bool allow_phase) {
  plan.clear();
  stats = PlanStats();
  stats.gates_in = (int)n_gates;
  // validation first: a bad gate leaves perm untouched
  for (size_t i = 0; i < n_gates; i++) {
    const qs_gate &g = gates[i];
    if (g.op >= QS_N_GATE_TYPES) {
      err = "gate " + std::to_string(i) + ": unknown op";
      return QS_EINVAL;
    }
    if (g.nq != op_info(g.op).nq) {
      err = "gate " + std::to_string(i) + ": qubit count does not match the op";
      return QS_EINVAL;
    }
    for (int j = 0; j < g.nq; j++) {
      if (g.q[j] >= n) {
        err = "gate " + std::to_string(i) + ": qubit out of range";
        return QS_EINVAL;
      }
      for (int k = 0; k < j; k++)
        if (g.q[k] == g.q[j]) {
          err = "gate " + std::to_string(i) + ": duplicate qubit";
          return QS_EINVAL;
        }
    }
    for (int j = 0; j < op_info(g.op).nparams; j++)
      if (!std::isfinite(g.p[j])) {
        err = "gate " + std::to_string(i) + ": non-finite angle";
        return QS_EINVAL;
      }
  }
  const bool vswap = flags & QS_VSWAP;
  const bool fuse = flags & QS_FUSE;
  int K = fuse ? QS_FUSE_K_OF(flags) : 0;
  if (fuse && K == 0) K = 4;
  if (K > QS_MAX_FUSE) {
    err = "fusion width above QS_MAX_FUSE";
    return QS_EUNSUPPORTED;
  }
  int D = std::max(1, std::min(opts.diag_max, QS_MAX_DIAG));
  if (opts.tc_exchange < 0 || opts.tc_exchange > 2) {
    err = "opts.tc_exchange out of range (0..2)";
    return QS_EINVAL;
  }
  if (opts.tc_max_ctas < 0) {
    err = "opts.tc_max_ctas must not be negative";
    return QS_EINVAL;
  }
  if (opts.n_global < 0 || opts.n_global > n - 1 || (opts.n_global > 0 && n - opts.n_global < 2)) {
    err = "opts.n_global out of range (0..n-2 global bits, two local bits at least)";
    return QS_EINVAL;
  }
  if (flags & QS_TILE) {
    const int tmax = c128 ? kMaxTileBits - 1 : kMaxTileBits;
    if (opts.tile_bits != 0 && (opts.tile_bits < 8 || opts.tile_bits > tmax)) {
      err = "opts.tile_bits out of range";
      return QS_EINVAL;
    }
    if (opts.tile_k < 0 || opts.tile_k > 4) {
      err = "opts.tile_k out of range (0..4)";
      return QS_EINVAL;
    }
  }

  // (0) rotation folding (an IR rewrite; exact)
  std::vector<qs_gate> folded;
  if (flags & QS_FOLD) {
    folded = fold_rotations(n, gates, n_gates);
    stats.gates_removed = (int)n_gates - (int)folded.size();
    gates = folded.data();
    n_gates = folded.size();
  }

  // (1) virtual swap and renaming to physical qubits
  std::vector<qs_gate> pg;
  pg.reserve(n_gates);
  for (size_t i = 0; i < n_gates; i++) {
    qs_gate g = gates[i];
    if (vswap && g.op == QS_SWAP) {
      std::swap(perm[g.q[0]], perm[g.q[1]]);
      stats.swaps_absorbed++;
      continue;
    }
    for (int j = 0; j < g.nq; j++) g.q[j] = (uint8_t)perm[g.q[j]];
    pg.push_back(g);
  }

  // (1b) relocation (Sec. III-D: move hot qubits out of the slow segment).
  // Here the slow positions are physical bits 0 and 1: a block whose targets
  // include both gathers 8-byte elements at 32-byte strides. When the share
  // of multi-qubit non-diagonal gates touching them exceeds reloc_share and
  // twice the share a random qubit pair would have, each
  // hot low bit is exchanged once, up front, with the high bit that carries
  // the fewest such gates, and every gate is renamed.
  std::vector<std::pair<int, int>> reloc;
  if ((flags & QS_RELOCATE) && n >= 6) {
    std::vector<double> heat(64, 0.0);
    double total = 0, low = 0;
    for (const qs_gate &g : pg) {
      if (op_info(g.op).diagonal || g.nq < 2) continue;
      total += 1;
      bool touches_low = false;
      for (int j = 0; j < g.nq; j++) {
        heat[g.q[j]] += 1;
        touches_low |= g.q[j] < 2;
      }
      if (touches_low) low += 1;
    }
    // "hot" means well above the share a random pair of qubits would have
    const double uniform = 1.0 - (double)(n - 2) * (n - 3) / ((double)n * (n - 1));
    if (total > 0 && low / total > std::max(opts.reloc_share, 2.0 * uniform)) {
      std::vector<int> used;
      for (int lowq = 0; lowq < 2; lowq++) {
        if (heat[lowq] == 0) continue;
        int best = -1;
        for (int q = n - 1 - opts.n_global; q >= 5; q--) {
          if (std::find(used.begin(), used.end(), q) != used.end()) continue;
          if (best < 0 || heat[q] < heat[best]) best = q;
        }
        if (best < 0 || heat[best] >= heat[lowq]) continue;
        used.push_back(best);
        reloc.push_back({lowq, best});
      }
      for (auto &pr : reloc) {
        const int a = pr.first, b = pr.second;
        for (qs_gate &g : pg)
          for (int j = 0; j < g.nq; j++) {
            if (g.q[j] == a) g.q[j] = (uint8_t)b;
            else if (g.q[j] == b) g.q[j] = (uint8_t)a;
          }
        for (int l = 0; l < n; l++) {
          if (perm[l] == a) perm[l] = (int8_t)b;
          else if (perm[l] == b) perm[l] = (int8_t)a;
        }
      }
      stats.relocations = (int)reloc.size();
    }
  }

  // (1c) global tier: the top n_global physical bits are held by other
  // ranks (one shard per value of those bits). A gate acting non-diagonally
  // on a global bit first needs that bit exchanged with a local one (a
  // virtual swap of the two bits: a pairwise half-shard exchange between the
  // ranks that differ in the global bit); the plan records the exchange and
  // every later gate, and perm, follow the relabelling. The local bit taken
  // is the one whose next non-diagonal use lies furthest ahead (never used
  // again first; ties: the highest bit), so that exchanges stay rare. Gates
  // that are diagonal on a global bit (controls, phases) need no exchange: a
  // shard knows its global bits.
  std::vector<size_t> cuts;                   // segment starts in pg
  std::vector<std::pair<int, int>> gswaps;    // (local, global) exchanged at each cut
  const int nloc = n - opts.n_global;
  if (opts.n_global > 0) {
    auto next_use = [&](size_t from, int q) {
      for (size_t i = from; i < pg.size(); i++)
        for (int j = 0; j < pg[i].nq; j++)
          if (pg[i].q[j] == q && !gate_diag_on(pg[i], j)) return i;
      return pg.size();
    };
    for (size_t i = 0; i < pg.size(); i++) {
      for (int j = 0; j < pg[i].nq; j++) {
        const int G = pg[i].q[j];
        if (G < nloc || gate_diag_on(pg[i], j)) continue;
        int L = -1;
        size_t far = 0;
        for (int q = nloc - 1; q >= 0; q--) {
          bool in_gate = false;
          for (int jj = 0; jj < pg[i].nq; jj++) in_gate |= pg[i].q[jj] == q;
          if (in_gate) continue;
          const size_t u = next_use(i, q);
          if (L < 0 || u > far) {
            L = q;
            far = u;
          }
        }
        if (L < 0) {
          err = "global tier: no local bit free for an exchange";
          return QS_EUNSUPPORTED;
        }
        for (size_t k2 = i; k2 < pg.size(); k2++)
          for (int jj = 0; jj < pg[k2].nq; jj++) {
            if (pg[k2].q[jj] == G) pg[k2].q[jj] = (uint8_t)L;
            else if (pg[k2].q[jj] == L) pg[k2].q[jj] = (uint8_t)G;
          }
        for (int l = 0; l < n; l++) {
          if (perm[l] == G) perm[l] = (int8_t)L;
          else if (perm[l] == L) perm[l] = (int8_t)G;
        }
        cuts.push_back(i);
        gswaps.push_back({L, G});
      }
    }
  }

  push_exchanges(reloc, plan);
  size_t seg_begin = 0;
  for (size_t sgi = 0; sgi <= cuts.size(); sgi++) {
    const size_t seg_end = sgi < cuts.size() ? cuts[sgi] : pg.size();
    std::vector<int> idx;
    for (size_t i = seg_begin; i < seg_end; i++) idx.push_back((int)i);
    qs_status st = plan_segment(n, pg, idx, flags, opts, D, K, c128, allow_phase, plan, err);
    if (st != QS_OK) return st;
    if (sgi < cuts.size()) {
      Block b;
      b.kind = BK_GLOBAL;
      b.k = 2;
      b.q[0] = gswaps[sgi].first;
      b.q[1] = gswaps[sgi].second;
      b.n_gates = 0;
      b.meta = 3;
      plan.push_back(std::move(b));
    }
    seg_begin = seg_end;
  }
  const bool tf32 = opts.tc_precision == 1;
  for (Block &b : plan) {
    b.tc = (flags & QS_TC) && b.kind == BK_DENSE && b.k >= 4 && b.k <= (tf32 ? 5 : 6);
    b.tc_tf32 = b.tc && tf32;
    b.shuffles = opts.no_shuffles == 0;
    // lane-exchange gathers where they measured faster (tc_exchange_pays),
    // or everywhere the layout allows with tc_exchange = 2
    TcXLayout xl;
    b.tc_xg = b.tc && !tf32 && opts.tc_exchange != 1 && (opts.tc_exchange == 2 || tc_exchange_pays(b)) &&
              tc_exchange_layout(n, b, xl);
    b.withhold_commit = b.tc && opts.test_wait_timeout != 0;
    b.tc_max_ctas = (b.tc || b.kind == BK_PHASE) ? opts.tc_max_ctas : 0;
  }
  return QS_OK;
}

}  // namespace qs
