// Internal declarations shared by the host runtime and the CUDA kernels.
#pragma once

#include <complex>
#include <functional>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "qs.h"

namespace qs {

using cd = std::complex<double>;

// ---------------------------------------------------------------------------
// Gate table (OpenQASM 2 qelib1 definitions)
// ---------------------------------------------------------------------------
struct OpInfo {
  const char *name;
  int nq;        // controls + targets
  int nparams;
  int nctrl;     // leading control qubits
  bool diagonal; // the whole gate is diagonal in the computational basis
};

const OpInfo &op_info(int op);
int op_by_name(const char *name);  // -1 if unknown

// Full matrix of a gate on its own qubits (controls embedded), local index
// l = sum_j bit(q_j) << j over the gate's qubit order; (2^nq)^2 row-major.
void gate_full_matrix(const qs_gate &g, std::vector<cd> &out);

// True when the gate acts diagonally on its j-th qubit (a control qubit, or
// any qubit of a diagonal gate): it then commutes with every other gate that
// is diagonal on that qubit.
bool gate_diag_on(const qs_gate &g, int j);

// ---------------------------------------------------------------------------
// Plan: the list of kernels one qs_apply_circuit call launches
// ---------------------------------------------------------------------------
// BK_GLOBAL: an exchange of a local with a global physical bit (opts.n_global
// > 0, qs_plan only): q[0] the local bit, q[1] the global one.
enum BlockKind : uint8_t { BK_DENSE = 0, BK_DIAG = 1, BK_PERMUTE = 2, BK_TILE = 3, BK_PHASE = 4, BK_GLOBAL = 5 };

constexpr int kMaxFixed = 24;  // targets + controls handled by the index insert
constexpr int kMaxTileBits = 14;  // widest shared-memory tile (QS_TILE)
constexpr int kTileLowBits = 4;   // contiguous low bits every tile includes (128-byte c64 runs)

struct Block {
  BlockKind kind = BK_DENSE;
  int k = 0;                      // dense: targets; diag: table qubits; permute: 2
  int q[QS_MAX_DIAG] = {0};       // physical qubits ascending (permute: a < b)
  uint64_t cmask = 0;             // physical control bits (all must be 1)
  int nctrl = 0;
  std::vector<cd> mat;            // dense (2^k)^2 row-major; diag 2^k phases
  int n_gates = 0;
  int first_op = -1;              // op of a single-gate block
  int meta = 4;                   // 0 one-qubit, 1 two-qubit, 3 swap, 4 fused
  bool tc = false;
  bool tc_tf32 = false;           // tensor-core operands: 3 x TF32 instead of 2 x FP16
  bool shuffles = true;           // CUDA-core blocks with low targets: warp-shuffle kernel
  bool tc_xg = false;             // 4..6-target tensor-core blocks: lane-exchange gathers (tc16x.cu)
  bool withhold_commit = false;   // test hook (qs_opts.test_wait_timeout)
  int tc_max_ctas = 0;            // test hook (qs_opts.tc_max_ctas): cap on tensor-core and phase CTAs
  // tile pass (BK_TILE): k = tile qubits, tile_q their physical positions
  // ascending (0..kTileLowBits-1 first); sub = the member blocks in order,
  // dense targets inside the tile, diagonal qubits and controls anywhere
  int tile_q[kMaxTileBits] = {0};
  std::vector<Block> sub;
  // phase polynomial (BK_PHASE): the block multiplies amplitude x by
  // exp(i (ph_c + sum_j ph_a[j] x_{ph_q[j]} + sum_{j<l} ph_b[j,l] x_{ph_q[j]} x_{ph_q[l]})),
  // k = ph_q.size(), ph_b upper triangle in row order, angles in (-pi, pi]
  std::vector<int> ph_q;
  std::vector<double> ph_a, ph_b;
  double ph_c = 0;
};

// Lane-exchange layout of a 4-, 5- or 6-target FP16 tensor-core block
// (tc16x.cu; 6 targets: two threads per group, each part laid out as a
// 5-target block with the highest target fixed).
// A warp owns the sub-cube of 32 groups spanned by the targets and the five
// lowest free bits. It loads it in address order -- element bit of each
// 16-byte load = bit 0, lane bits = the next five bits of the sub-cube
// (where that would leave more than two targets on lane bits after the
// element bit's exchange, the highest of them trade places with the lowest
// free register bits), register bits = the rest -- and then exchanges bits
// between positions with
// warp shuffles until the lane bits hold the free bits and the element and
// register bits hold the targets, i.e. every lane holds one whole group in
// "slot" order (slot bit 0 = element, slot bit 1 + j = register bit j).
struct TcXLayout {
  int lbit[5];       // physical bit of lane bit i, as loaded
  int rbit[5];       // physical bit of register bit j, as loaded (k - 1 used)
  int la;            // lane bit exchanged with the element bit, -1 if bit 0 is a target
  int nswb;          // lane bits lb[i] exchanged with register bits i (i < nswb <= 2)
  int lb[2];
  int slot_mat[6];   // slot bit -> position of its target in the block's ascending list
  int part_bit[2];   // 6 targets: part_bit[0] = the sixth target, fixed per thread part h (h = 1
                     // sets it; slot bit 5), part_bit[1] = -1; else both -1
  int nf;            // targets, controls and the five lowest free bits, ascending
  int fixed[kMaxFixed];
};
// False when the block cannot take the layout: not 4..6 targets, bit 0 a
// control, fewer than 7 free bits among n (whole tiles of 128 groups), or
// too many fixed bits.
bool tc_exchange_layout(int n, const Block &b, TcXLayout &x);
// True where the exchange kernel measured faster than the plain
// thread-per-group gather: every 5-target block, 4-target blocks with two
// or more targets among bits 1..3, 6-target blocks with one or more.
bool tc_exchange_pays(const Block &b);

// Index of the pair (j, l), j < l < w, in a row-order upper triangle.
inline size_t tri_index(int j, int l, int w) { return (size_t)j * (2 * w - j - 1) / 2 + (l - j - 1); }

struct PlanStats {
  int gates_in = 0;
  int swaps_absorbed = 0;
  int relocations = 0;
  int gates_removed = 0;  // by rotation folding
};

// Virtual swap + fusion + classification. Gates are logical; perm is the
// state's logical->physical map, updated in place for absorbed SWAPs.
// Returns QS_OK or QS_EINVAL (message in err).
// c128 selects the amplitude size the default tile width is computed for.
qs_status build_plan(int n, const qs_gate *gates, size_t n_gates, uint64_t flags,
                     const qs_opts &opts, int8_t *perm, std::vector<Block> &plan,
                     PlanStats &stats, std::string &err, bool c128 = false, bool allow_phase = true);

// Tile width QS_TILE uses for these options and amplitude type.
int tile_bits_of(const qs_opts &o, bool c128);
int tile_k_of(const qs_opts &o);

double block_bytes(const Block &b, int n, int amp_bytes);

// The public record of a planned block (passes.cpp).
void fill_record(const Block &b, int index, int n, int amp_bytes, qs_block_record &r);

// Cost-model features of a block record (pgo.cpp).
void record_features(const qs_block_record &r, int n, bool c128, float *f);

// f(0..n) on a few host threads (passes.cpp).
void parallel_blocks(size_t n, const std::function<void(size_t)> &f);

// Rotation folding + peephole cancellation (fold.cpp): an equivalent gate
// list (exact, global phase included).
std::vector<qs_gate> fold_rotations(int n, const qs_gate *in, size_t n_in);

// Profile-guided selection (pgo.cpp).
uint64_t rules_select(int n, const qs_gate *gates, size_t n_gates, const qs_opts &o, uint64_t base);
int block_class(const Block &b);
double predict_plan_ms(const std::vector<Block> &plan, int n, int amp_bytes, const qs_class_table *t,
                       double peak_gbs);
qs_status measured_select(int n, bool c128, const qs_gate *gates, size_t n_gates, const qs_opts &o,
                          const qs_class_table *t, uint64_t base, uint64_t *flags_out, double *pred_ms,
                          std::string &err);
qs_status mlp_select(qs_mlp *mm, int n, bool c128, const qs_gate *gates, size_t n_gates, const qs_opts &o,
                     uint64_t *flags_out, double *pred_ms, std::string &err);

// Device allocations counted against the budget of qs_set_memory_limit
// (devmem.cpp); dev_free takes null.
cudaError_t dev_malloc(void **p, size_t bytes);
void dev_free(void *p);
// True when this thread's last dev_malloc was refused by the budget.
bool dev_refused_by_budget();

// ---------------------------------------------------------------------------
// Kernel launchers (kernels.cu). All asynchronous on `s`.
// ---------------------------------------------------------------------------
// Launch shape of a tensor-core block: tiles of 128 groups and CTAs launched
// (each CTA loops over tiles blockIdx.x, blockIdx.x + gridDim.x, ...).
struct LaunchShape {
  long long tiles = 0;
  int ctas = 0;
};

struct DevInfo {
  int sms = 0;
  int max_threads_per_sm = 0;
};
const DevInfo &dev_info();

cudaError_t launch_block(void *amps, int n, bool c128, const Block &b, cudaStream_t s, int threads);
// Dense blocks too wide for the parameter space (k = 6, or k = 5 in c128)
// read their matrix from device memory (row-major, the state's dtype).
// Tensor-core blocks read their split real embedding from device memory too.
bool block_needs_dev_matrix(const Block &b, bool c128);
size_t block_dev_matrix_bytes(const Block &b, bool c128);
void fill_dev_matrix(const Block &b, bool c128, void *host_out);
// Bytes of gate data one block ships to the device: its kernel parameters
// (matrix or phase table included) plus any matrix upload.
size_t block_param_bytes(const Block &b, bool c128);
// err: device error word for kernels with bounded waits (tensor-core path);
// shape (may be null) receives a tensor-core launch's tiles and CTAs.
cudaError_t launch_block_with_matrix(void *amps, int n, bool c128, const Block &b, const void *dev_mat,
                                     int *err, cudaStream_t s, int threads, LaunchShape *shape = nullptr);
cudaError_t launch_permute(void *amps, int n, bool c128, int a, int b, cudaStream_t s);
cudaError_t launch_set_basis(void *amps, int n, bool c128, uint64_t idx, cudaStream_t s);

// Marginal probabilities over m physical bits pos[0..m) (bin bit j = pos[j]).
// partial: device scratch of probs_scratch_doubles(n, m) doubles; out: 2^m
// doubles on the device.
size_t probs_scratch_doubles(int n, int m);
// sum |a_i - b_i|^2 into distance_grid() FP64 partials
int distance_grid();
cudaError_t launch_distance(const void *a, bool a128, const void *b, bool b128, int n, double *partial,
                            cudaStream_t s);
cudaError_t launch_probs(const void *amps, int n, bool c128, const int *pos, int m,
                         double *partial, double *out, cudaStream_t s);

}  // namespace qs
