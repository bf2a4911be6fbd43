/*
 * qs.h -- C ABI of the GB300 state-vector simulator core.
 *
 * The library applies a compiled gate list to a 2^n-amplitude state vector
 * held in GPU memory (full-state, Schroedinger-style simulation, Sec. II-B of
 * arXiv 2410.09326 "QOPS"), with the paper's profile-guided optimisations:
 * virtual swap (Sec. III-D), gate merging generalised to k-qubit fusion
 * (Sec. III-D "Single-qubit gate merging"), and a pass activator driven by
 * per-gate counters and per-block timings (Sec. III-A "PGO compilation flow",
 * Sec. III-C "QOPS Profiling Library").
 *
 * Conventions
 *  - Qubit q_i is bit i of the basis index (little-endian). The paper's
 *    storage example puts q_0 in the most significant ("file") segment; this
 *    library does not.
 *  - Amplitudes are interleaved complex: QS_C64 = {float re, im} (8 bytes),
 *    QS_C128 = {double re, im} (16 bytes). Gate matrices follow the OpenQASM 2
 *    qelib1 definitions; RZ(t) = diag(e^{-it/2}, e^{it/2}).
 *  - A state carries a logical->physical qubit map `perm` (perm[l] = the
 *    physical bit that holds logical qubit l). Gates name logical qubits.
 *    Amplitude a_phys[P(i)] equals the logical amplitude a[i] where
 *    P(i) = sum_l bit_l(i) << perm[l].
 *  - Every call returns a qs_status; on failure qs_last_error() gives a
 *    message (thread-local, valid until the next call on that thread).
 *    Nothing aborts the process.
 *  - Calls that launch work are asynchronous on the state's stream, except
 *    qs_measure_probs, qs_norm and qs_read_state, which synchronise it.
 *  - A CUDA error seen by a call marks the state invalid; later calls on it
 *    return QS_ESTATE.
 */
#ifndef QS_ABI_H_
#define QS_ABI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QS_OK = 0,
  QS_EINVAL = 1,        /* bad argument (qubit out of range, duplicate, ...) */
  QS_ENOMEM = 2,        /* device or host allocation failed */
  QS_ECUDA = 3,         /* a CUDA call failed; the state is now invalid */
  QS_EUNSUPPORTED = 4,  /* valid request the library does not handle */
  QS_ETIMEOUT = 5,      /* a bounded device-side wait ran out */
  QS_ESTATE = 6         /* the state is invalid after an earlier CUDA error */
} qs_status;

typedef enum { QS_C64 = 0, QS_C128 = 1 } qs_dtype;

/*
 * Gate types. The paper's counter-based profiler (Sec. III-C) keeps 33 gate
 * counters per qubit, naming H first, S second, T third, CPhase, CU1 and SWAP
 * among them and using 0 for H and 11 for CPhase in its context records. The
 * full list is in a missing figure, so the ids below are this library's own:
 * H=0, S=1, T=2, CPHASE=11, CU1=12, SWAP=13 follow the text, the rest fill
 * the gaps.
 */
typedef enum {
  QS_H = 0, QS_S = 1, QS_T = 2, QS_X = 3, QS_Y = 4, QS_Z = 5, QS_SDG = 6,
  QS_TDG = 7, QS_RX = 8, QS_RY = 9, QS_RZ = 10, QS_CPHASE = 11, QS_CU1 = 12,
  QS_SWAP = 13, QS_CX = 14, QS_CZ = 15, QS_CY = 16, QS_CH = 17, QS_CRX = 18,
  QS_CRY = 19, QS_CRZ = 20, QS_U1 = 21, QS_U2 = 22, QS_U3 = 23, QS_SX = 24,
  QS_SXDG = 25, QS_ID = 26, QS_RZZ = 27, QS_RXX = 28, QS_RYY = 29,
  QS_CCX = 30, QS_CSWAP = 31, QS_CU3 = 32,
  QS_N_GATE_TYPES = 33
} qs_op;

#define QS_MAX_QUBITS 40   /* the paper's profiler supports 40 qubits */
#define QS_MAX_N_C64 34    /* 2^34 * 8 B = 128 GiB of HBM */
#define QS_MAX_N_C128 33   /* 2^33 * 16 B = 128 GiB of HBM */
#define QS_MAX_FUSE 6      /* widest dense fused block */
#define QS_MAX_DIAG 10     /* widest diagonal fused block (phase table 2^10) */

/* One gate: q[0..nc-1] are controls, then targets (logical qubits). 32 B. */
typedef struct {
  uint8_t op;    /* qs_op */
  uint8_t nq;    /* controls + targets, must match the op */
  uint8_t q[6];
  double p[3];   /* angles in radians; unused entries ignored */
} qs_gate;

/* Flags of qs_apply_circuit. */
#define QS_PLAIN ((uint64_t)0)              /* one kernel per gate, SWAP moves data */
#define QS_VSWAP ((uint64_t)1 << 0)         /* SWAPs become relabellings of perm */
#define QS_FUSE ((uint64_t)1 << 1)          /* k-qubit fusion, k from QS_FUSE_K */
#define QS_DIAG ((uint64_t)1 << 2)          /* diagonal runs fuse, any width */
#define QS_TC ((uint64_t)1 << 3)            /* dense k>=4 blocks on tensor cores (opts->tc_precision) */
#define QS_PROFILE ((uint64_t)1 << 4)       /* time every block with CUDA events */
#define QS_RELOCATE ((uint64_t)1 << 5)      /* profile-guided hot-qubit relocation */
#define QS_FOLD ((uint64_t)1 << 6)          /* rotation folding + pair cancellation first */
#define QS_TILE ((uint64_t)1 << 7)          /* cache-blocked passes: runs of blocks whose targets fit one
                                               shared-memory tile (opts->tile_bits qubits, the lowest
                                               bits included) share one HBM pass */
#define QS_PGO_RULES ((uint64_t)1 << 8)     /* pick flags with the paper's counter rules */
#define QS_PGO_MEASURED ((uint64_t)1 << 9)  /* pick flags from a measured block profile */
#define QS_FUSE_K(k) ((uint64_t)((k) & 15) << 16)
#define QS_FUSE_K_OF(f) ((int)(((f) >> 16) & 15))

/* Tunables; pass NULL for defaults (qs_default_opts). */
typedef struct {
  int merge_run;        /* 1q-merge activation: longest 1q run > this (paper: e.g. five) */
  double t_ratio;       /* rotation-folding activation: T count / gates (paper: e.g. 10%) */
  int low_bits;         /* physical bits below this are "fast" (chunk-segment analogue) */
  double reloc_share;   /* relocate a high qubit carrying >= this share of block time */
  int diag_max;         /* widest diagonal phase table, 1..QS_MAX_DIAG (wider runs: polynomials) */
  int threads;          /* launch override: threads per CTA (0 = tuned default) */
  double peak_gbs;      /* HBM copy bandwidth the cost model scales its priors by */
  int tc_precision;     /* QS_TC operands: 0 = two FP16 halves (k = 4..6), 1 = 3 x TF32 (k = 4, 5) */
  int test_wait_timeout; /* test hook, 0 in normal use: tensor-core blocks withhold their
                            completion signal, so their bounded (1 s) wait runs out and the
                            next synchronising call returns QS_ETIMEOUT; results invalid */
  int tile_bits;        /* QS_TILE: qubits per shared-memory tile, 0 = 64 KiB of amplitudes
                           (13 for c64, 12 for c128); 8..14 c64, 8..13 c128 */
  int tile_k;           /* QS_TILE: fusion width inside a tile, 0 = 3; 1..4 */
  int fuse_lookahead;   /* fusion: where a gate could join several blocks or open a new one,
                           each choice is followed by this many gates of first-fit placement
                           and the one leaving the fewest blocks is taken; 0 = first fit
                           (qs_default_opts: 60) */
  int no_shuffles;      /* 1: CUDA-core blocks whose targets cover bits 1, 2, 3 (bit 0 free) keep
                           the thread-per-group kernel instead of warp-wide loads and shuffles (c64) */
  int tc_exchange;      /* 4- to 6-target tensor-core blocks (FP16 halves): the thread-per-group
                           kernel (each thread gathers its own group) or the lane-exchange kernel
                           (a warp loads its groups' sub-cube in address order and hands each
                           lane its group by warp shuffles):
                           0 = lane exchange where it measured faster (every 5-target block,
                           4-target blocks with two or more targets among bits 1..3, 6-target
                           blocks with one or more); 1 = never; 2 = wherever the layout allows
                           (bit 0 not a control, whole tiles of 128 groups) */
  int tc_max_ctas;      /* test hook, 0 in normal use: at most this many CTAs per tensor-core
                           or phase-polynomial launch (normally one wave of resident CTAs, no
                           more than there are tiles or chunks), so that every CTA loops over
                           several tiles (every warp over several 1024-amplitude chunks) even
                           on a small state; the block records report tiles (chunks) and CTAs */
  int n_global;         /* sharding tier (qs_plan only; 0 elsewhere): the top n_global physical
                           bits are global -- a state sharded over 2^n_global ranks, one shard per
                           value of those bits (Sec. II-B's file segment, across ranks). The plan
                           then acts on global bits only diagonally (controls, phases: a shard
                           knows its own global bits) and, before a gate that acts on a global
                           bit non-diagonally, exchanges that bit with the local bit whose next
                           non-diagonal use lies furthest ahead (a virtual swap of the two bits,
                           Sec. III-D: ranks differing in the global bit swap half of their
                           shards); records of kind 5 mark those exchanges and perm follows
                           them. Blocks may still name global bits: their matrices are then
                           block-diagonal in them. 0..n-2; qs_apply_circuit and batches
                           return QS_EUNSUPPORTED for n_global > 0 (one GPU, no sharded runner) */
} qs_opts;

void qs_default_opts(qs_opts *out);

typedef struct qs_state qs_state;

/*
 * Sec. II-B (full-state, Schroedinger-style simulation): the simulator keeps
 * all 2^n complex amplitudes of an n-qubit system in memory and updates them
 * gate by gate. This allocates that state vector in HBM.
 * Allocates a state of n qubits in library-owned device memory on the
 * current device and sets it to |0...0> with perm = identity. cuda_stream is
 * a cudaStream_t (NULL = legacy default stream) that all work on the state is
 * ordered on. n must be 1..QS_MAX_N_C64 (c64) or 1..QS_MAX_N_C128 (c128).
 */
qs_status qs_alloc_state(int n, qs_dtype dtype, void *cuda_stream, qs_state **out);

/*
 * Sec. II-B: the same 2^n-amplitude state vector, in memory the caller owns.
 * Wraps caller-owned device memory (for example a torch tensor) of
 * 2^n amplitudes of the given dtype, 16-byte aligned. The contents are left
 * as they are (perm = identity); qs_free_state does not free the memory.
 */
qs_status qs_attach_state(void *dev_ptr, int n, qs_dtype dtype, void *cuda_stream, qs_state **out);

/* Sec. II-B: releases the state vector's handle (and the amplitudes when
 * library-owned). NULL is a no-op. */
void qs_free_state(qs_state *st);

/* Sec. II-B: sets the state to the logical basis state |x> (the state a
 * simulation starts from) and perm to identity. Asynchronous on the state's
 * stream. */
qs_status qs_set_basis(qs_state *st, uint64_t x);

/*
 * IR ingest (the simulator's input format, Sec. III-A: the compiler emits
 * OpenQASM). Parses the OpenQASM-2 subset "qreg q[N]; name(p..) q[a],q[b];"
 * with the gate names of qs_op (lower case: h s t x y z sdg tdg rx ry rz cp
 * cu1 swap cx cz cy ch crx cry crz u1 u2 u3 sx sxdg id rzz rxx ryy ccx cswap
 * cu3). Writes up to `cap` gates; *n_gates receives the total count and
 * *n_qubits the register size. Returns QS_EINVAL with the line number in
 * qs_last_error on a syntax error, or when the text holds more than cap gates
 * (*n_gates is still set, so a caller can size a buffer with cap = 0).
 */
qs_status qs_parse_qasm(const char *text, int *n_qubits, qs_gate *gates, size_t cap, size_t *n_gates);

/*
 * Applies gates[0..n_gates) in order. flags select the passes: QS_PLAIN runs
 * one kernel per gate; QS_VSWAP absorbs SWAPs into perm (Sec. III-D "Virtual
 * swap"); QS_FUSE | QS_FUSE_K(k) groups gates into dense blocks of at most k
 * qubits, commuting gates past each other only where they act diagonally on
 * every shared qubit; QS_DIAG lets diagonal runs grow: up to opts->diag_max
 * qubits as a phase table, wider (any width, states of more than 10 qubits)
 * as a phase polynomial exp(i(c + sum a_j x_j + sum b_jl x_j x_l)); QS_TC runs dense blocks with 4..6 targets on the tensor cores;
 * QS_TILE groups gates (same commutation rule) into passes whose non-diagonal
 * qubits fit a tile of opts->tile_bits qubits and applies each pass -- its
 * gates fused again, at most opts->tile_k wide -- in shared memory during one
 * read and one write of the state (QS_TILE is ignored when n <= tile bits);
 * QS_PGO_RULES / QS_PGO_MEASURED replace the pass flags by the activator's
 * choice (see qs_pgo_select). gates is copied during the call; the launches
 * are asynchronous on the state's stream.
 */
qs_status qs_apply_circuit(qs_state *st, const qs_gate *gates, size_t n_gates, uint64_t flags,
                           const qs_opts *opts);

/*
 * Profiling (Sec. III-C). Counter-based: every applied gate increments
 * counters[q][op] for each logical qubit q it touches, and the longest run of
 * consecutive one-qubit gates per qubit is kept (the activator's merge
 * counter, Sec. III-D). Context-based: the paper records one tuple per gate
 * (meta type 0 = one-qubit, 1 = two-qubit, 3 = SWAP; qubits; gate type;
 * timestamp); here one record per launched block of the last apply call,
 * with meta 4 for a fused block, its physical qubits, and -- when the call
 * had QS_PROFILE -- its start time and device time from CUDA events.
 */
typedef struct {
  int32_t index;     /* launch order within the last apply call */
  uint8_t kind;      /* 0 dense block, 1 diagonal block, 2 physical bit exchange,
                        3 tile pass (QS_TILE: several blocks in one HBM pass),
                        4 phase polynomial (a diagonal run wider than opts->diag_max),
                        5 exchange of a local bit (qubits[0]) with a global one (qubits[1])
                          (qs_plan with opts->n_global > 0) */
  uint8_t k;         /* targets (dense) / table qubits (diagonal) / 2 (exchange) /
                        tile qubits (tile pass) */
  uint8_t nctrl;     /* control bits that must be 1: only 2^(n-nctrl) amplitudes move */
  uint8_t tc;        /* 1 if it ran on the tensor cores, 2 if so with lane-exchange gathers */
  int8_t qubits[QS_MAX_DIAG]; /* physical qubits ascending, -1 padded; for a tile pass the
                                 tile's qubits above its contiguous low bits */
  uint8_t meta;      /* 0 one-qubit gate, 1 two-qubit gate, 3 swap, 4 fused block,
                        5 tile pass */
  uint8_t op;        /* qs_op of a single-gate block, 255 for a fused block */
  int32_t n_gates;   /* gates merged into the block */
  uint64_t cmask;    /* physical control bits (the block acts where all are 1) */
  double bytes;      /* algorithmic bytes: 2 x amplitudes changed x amplitude size */
  double t_start_ms; /* start relative to the first block (QS_PROFILE), else -1 */
  double ms;         /* device time (QS_PROFILE), else -1 */
  int64_t tiles;     /* blocks of an apply call: tensor-core blocks, tiles of 128 groups;
                        phase polynomials, chunks of 1024 amplitudes; else 0 */
  int32_t ctas;      /* the same blocks: CTAs launched (each loops over tiles ctas apart;
                        each of a phase CTA's 8 warps over chunks 8 ctas apart); else 0 */
  int32_t reserved;
} qs_block_record;

typedef struct {
  int32_t n_qubits;
  int32_t n_blocks;           /* blocks launched by the last apply call */
  int64_t gates_seen;         /* gates counted since the last reset */
  int32_t gates_last;         /* gates in the last apply call */
  int32_t swaps_absorbed;     /* SWAPs the last call turned into relabellings */
  uint64_t flags_used;        /* flags the last call ran with (after PGO) */
  int64_t counters[QS_MAX_QUBITS][QS_N_GATE_TYPES];
  int32_t max_1q_run[QS_MAX_QUBITS];
  double total_ms;            /* sum of block times of the last call, -1 if untimed */
  double total_bytes;         /* sum of algorithmic bytes of the last call */
  double h2d_bytes;           /* gate data the last call shipped to the device
                                 (kernel parameters and matrix uploads) */
} qs_profile_summary;

/*
 * Fills *out and up to cap block records of the last apply call (*n_recs gets
 * the total). With QS_PROFILE timings this waits for the last block's event.
 */
qs_status qs_profile(qs_state *st, qs_profile_summary *out, qs_block_record *recs, size_t cap,
                     size_t *n_recs);

/* Clears the counters, records and class table (start of a new profiling run). */
qs_status qs_profile_reset(qs_state *st);

/*
 * Measured profile as a throughput table: bytes, device time and launch count
 * of every profiled block so far, by kernel class
 *   class = kind * 8 + min(k, 7) + 32 * (tensor cores) + 64 * (a dense
 *           block whose targets include bits 0 and 1),
 * kind 0 dense, 1 diagonal, 2 exchange.
 */
#define QS_N_CLASSES 128
typedef struct {
  double bytes[QS_N_CLASSES];
  double ms[QS_N_CLASSES];
  int64_t count[QS_N_CLASSES];
} qs_class_table;

qs_status qs_profile_classes(const qs_state *st, qs_class_table *out);

/*
 * Measured-profile activator (the mapping from profile to flags that the
 * paper leaves open, Sec. III-A). Plans every candidate flag set {plain,
 * virtual swap, fusion k = 1..6 with diagonal runs, tensor cores for k >= 4}
 * on the host and predicts its time as the sum over blocks of bytes / class
 * throughput from `table` (NULL = compiled-in GB300 priors only, scaled to
 * opts->peak_gbs). Host only; returns the fastest candidate's flags and its
 * predicted milliseconds. qs_apply_circuit with QS_PGO_MEASURED does the
 * same with the state's own table and profiles the run it launches.
 */
qs_status qs_pgo_select(int n, qs_dtype dtype, const qs_gate *gates, size_t n_gates, const qs_class_table *table,
                        const qs_opts *opts, uint64_t *flags_out, double *predicted_ms);

/*
 * The same model for one given flag set (Sec. III-A: the profile's estimate
 * of what a set of passes would cost): plans `flags` on the host and writes
 * the predicted device milliseconds (sum over blocks of bytes / class
 * throughput from `table`, or the compiled-in priors where NULL or
 * unmeasured, plus a launch gap per block). Host only.
 */
qs_status qs_pgo_predict(int n, qs_dtype dtype, const qs_gate *gates, size_t n_gates, uint64_t flags,
                         const qs_class_table *table, const qs_opts *opts, double *predicted_ms);

/*
 * The host passes alone (virtual swap, fusion, classification), without a
 * GPU: the plan qs_apply_circuit would launch for a state of n qubits whose
 * map is *perm_inout (n entries, updated for absorbed SWAPs). Fills up to cap
 * records (ms = -1) and, when mats is not NULL, the blocks' matrices in FP64
 * as interleaved (re, im) pairs, block after block: (2^k)^2 entries for a
 * dense block (row-major over the block's ascending physical qubits, local
 * index sum_j bit(q_j) << j), 2^k phases for a diagonal block, none for an
 * exchange or a tile pass; for a phase polynomial (kind 4) its k qubits as
 * (physical qubit, linear angle) pairs, then (constant angle, 0), then
 * (pair angle, 0) for every qubit pair j < l in row order. A tile pass's record is followed by the records
 * (and matrices) of its member blocks in the order the pass applies them;
 * they carry the pass's index. *n_blocks (records) and *mats_len (complex
 * entries) receive the totals.
 */
qs_status qs_plan(int n, const qs_gate *gates, size_t n_gates, uint64_t flags, const qs_opts *opts,
                  int8_t *perm_inout, qs_block_record *recs, size_t cap, size_t *n_blocks,
                  double *mats, size_t mats_cap, size_t *mats_len);

/*
 * Device-memory budget for the library's own allocations (states from
 * qs_alloc_state, reduction and matrix scratch, batch plans, cost-model
 * buffers; borrowed states do not count). 0 = no budget (the default). An
 * allocation that would take the library's live device bytes above the
 * budget fails with QS_ENOMEM before any CUDA call; lowering the budget
 * frees nothing. Process wide and thread-safe. qs_memory_in_use returns the
 * library's live device bytes.
 */
void qs_set_memory_limit(uint64_t bytes);
uint64_t qs_memory_in_use(void);

/*
 * Lane-exchange layout of the FP16 tensor-core kernels (introspection for
 * tests and tools; host only, no GPU). A warp of those kernels owns the
 * sub-cube spanned by a block's targets and its five lowest free bits (6
 * targets: two threads per group; the five lower targets, the sixth fixed
 * per thread part),
 * loads it with 16-byte accesses (element bit = bit 0) whose lane bits and
 * register bits are given below, and exchanges bits between positions with
 * warp shuffles until every lane holds one group: first the element bit with
 * lane bit la (if la >= 0), then lane bit lb[i] with register bit i for
 * i < nswb. Slot bit 0 is then the element bit, slot bit 1 + j register bit j
 * (slot bit 5 = part_bits[0] for 6 targets); slot_target[s] is the position, in
 * the ascending target list, of the target slot bit s holds.
 * targets: k (4..6) distinct ascending physical bits < n; cmask: controls,
 * disjoint from them. Returns QS_EINVAL for bad arguments; *out->applies = 0
 * when the block cannot take the layout (bit 0 a control, fewer than 7 free
 * bits, too many fixed bits).
 */
typedef struct {
  int32_t applies;
  int32_t lane_bits[5];    /* physical bit of lane bit i, as loaded */
  int32_t reg_bits[4];     /* physical bit of register bit j, as loaded (k - 1 used, 4 for k = 6) */
  int32_t la;              /* lane bit exchanged with the element bit, -1 if none */
  int32_t nswb;            /* lane/register exchanges (0..2) */
  int32_t lb[2];           /* their lane bits */
  int32_t slot_target[6];  /* slot bit -> index in the ascending target list */
  int32_t part_bits[2];    /* 6 targets: part_bits[0] = the physical bit fixed per thread part
                              (the sixth target; the second part has it set), part_bits[1] = -1;
                              else both -1 */
} qs_exchange_layout;

qs_status qs_tc_exchange_layout(int n, int k, const int *targets, uint64_t cmask, qs_exchange_layout *out);

/*
 * Rotation folding (Sec. III-D): phase rotations (T, T^dagger, S, S^dagger,
 * Z, U1, RZ) on the same parity of a CNOT/X/SWAP/diagonal region merge into
 * the first of them (e.g. T . T -> S), then adjacent equal self-inverse gates
 * cancel (CNOT . CNOT, H . H, ...). The result is the same unitary, global
 * phase included (a nonzero phase is appended as U1, RZ on qubit 0). Host
 * only. Writes up to cap gates; *n_out receives the count (QS_EINVAL when it
 * exceeds cap).
 */
qs_status qs_fold_rotations(int n, const qs_gate *in, size_t n_in, qs_gate *out, size_t cap, size_t *n_out);

/* Sec. III-D (virtual swap): a SWAP gate is not executed but relabels qubits;
 * this returns the resulting logical->physical map: perm_out[l] = physical
 * bit of logical qubit l (n entries, host memory the caller owns). */
qs_status qs_get_perm(const qs_state *st, int8_t *perm_out);

/*
 * Sec. II-B: a full-state simulation ends in the final probability
 * distribution of the measured qubits; this is that distribution.
 * Marginal probabilities of m logical qubits (FP64 accumulation on the GPU):
 * host_out[b] = sum of |a_i|^2 over logical indices i whose bit
 * logical_qubits[j] equals bit j of b; 2^m doubles, m in 0..min(n, 26).
 * m = 0 gives the squared norm. Synchronises the stream.
 */
qs_status qs_measure_probs(qs_state *st, const int *logical_qubits, int m, double *host_out);

/*
 * Marginal probabilities without any allocation. The paper has no
 * counterpart: this is for callers that cannot let the library allocate
 * device memory -- a process that reserved all of its HBM through its own
 * pool, or one that must not risk the device-wide synchronisation that
 * cudaMalloc/cudaFree may imply. Same result as qs_measure_probs, but on raw
 * pointers: dev_amps holds 2^n amplitudes of `dtype` in device memory
 * (16-byte aligned), phys_bits (host, m entries) names PHYSICAL bit
 * positions (bin bit j = phys_bits[j]; map logical qubits through perm
 * first), and dev_out receives 2^m doubles in device memory (8-byte
 * aligned), m in 0..min(n, 26); larger m returns QS_EINVAL. The work is
 * enqueued on cuda_stream (a cudaStream_t; NULL = legacy stream) and the
 * call returns without synchronising.
 * Scratch: states of 12 or more qubits need none -- the call zeroes dev_out
 * with an asynchronous memset and the kernel accumulates into it. Smaller
 * states keep per-CTA partial sums in a fixed 128 KiB array inside the
 * library (kept by every GPU that loads it until exit). The call makes no
 * cudaMalloc, cudaFree or other allocating call. The first call on a device
 * resolves the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture. All calls
 * on states below 12 qubits share the one array: such calls whose work
 * overlaps on the GPU (different streams, or several host threads) race and
 * may corrupt each other's results; order them on one stream.
 */
qs_status qs_probs_noalloc(const void *dev_amps, int n, qs_dtype dtype, const int *phys_bits, int m,
                           double *dev_out, void *cuda_stream);

/* Sec. II-B: the total probability (squared norm sum |a_i|^2) of the state
 * vector in FP64. Synchronises the stream. */
qs_status qs_norm(qs_state *st, double *host_out);

/*
 * Sec. II-B (full-state simulation can expose the intermediate or final
 * state) and Sec. III-D (the relabelling of virtual swap, undone on request).
 * Copies the amplitudes to host memory (2^n of the state's dtype). With
 * logical_order != 0 the state is first brought to perm = identity on the
 * GPU by physical bit exchanges (which changes the device layout and perm);
 * with 0 the physical layout is copied as it is. Synchronises the stream.
 */
qs_status qs_read_state(qs_state *st, void *host_out, int logical_order);

/*
 * L2 distance sqrt(sum_i |a_i - b_i|^2) between two states of the same width
 * (any dtypes, FP64 accumulation on the GPU) in logical order: when their
 * maps differ both are first brought to perm = identity on the GPU. For
 * validating a complex64 run against a complex128 one without copying the
 * states to the host. Synchronises both streams.
 */
qs_status qs_state_distance(qs_state *a, qs_state *b, double *out);

/* Copies 2^n amplitudes from host memory into the state (physical layout). */
qs_status qs_write_state(qs_state *st, const void *host_in);

/* Device pointer of the amplitudes (for callers that share the buffer). */
qs_status qs_device_ptr(const qs_state *st, void **out);

/*
 * Learned cost model. The paper leaves the mapping from profile data to
 * optimisation flags open (Sec. III-A); here a 2 x 64 ReLU MLP predicts the
 * natural log of a fused block's device time in ms from QS_MLP_FEATURES
 * features of the block (qs_block_features), trained on block profiles the
 * simulator records (QS_PROFILE). It replaces profiling runs: candidate plans
 * are scored by their summed predicted block times.
 *
 * Parameters form one flat FP32 vector of QS_MLP_PARAMS values: W1 (64 x 24,
 * row-major, out x in), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1);
 * y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3. Training (qs_mlp_train)
 * standardises inputs and targets with the training set's mean and standard
 * deviation and runs Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the mean
 * squared error, with the library's own forward, backward and update kernels
 * on the GPU. qs_mlp_gradient returns the gradient of the mean squared error
 * on the inputs exactly as given (no standardisation), for checking.
 */
#define QS_MLP_FEATURES 24
#define QS_MLP_HIDDEN 64
#define QS_MLP_PARAMS (64 * 24 + 64 + 64 * 64 + 64 + 64 + 1)
typedef struct qs_mlp qs_mlp;

/* Features of profiled or planned blocks: count x QS_MLP_FEATURES floats. */
qs_status qs_block_features(int n, qs_dtype dtype, const qs_block_record *recs, size_t count, float *out);
qs_status qs_mlp_create(uint64_t seed, void *cuda_stream, qs_mlp **out);
void qs_mlp_free(qs_mlp *m);
/* Reads (host_out) and/or writes (host_in) the flat parameter vector. */
qs_status qs_mlp_params(qs_mlp *m, float *host_out, const float *host_in);
qs_status qs_mlp_gradient(qs_mlp *m, const float *x, const float *y, int n, float *grad_out, float *loss_out);
/* Trains on n samples (host arrays); loss_out: last batch's loss in standardised units. */
qs_status qs_mlp_train(qs_mlp *m, const float *x, const float *y, int n, int epochs, int batch, float lr,
                       uint64_t seed, float *loss_out);
/* Predicted log-milliseconds of n feature rows. */
qs_status qs_mlp_predict(qs_mlp *m, const float *x, int n, float *y_out);
/* Learned activator: the candidate flag set of qs_pgo_select with the least
 * summed predicted block time; host planning + one batched prediction. */
qs_status qs_pgo_select_mlp(qs_mlp *m, int n, qs_dtype dtype, const qs_gate *gates, size_t n_gates,
                            const qs_opts *opts, uint64_t *flags_out, double *predicted_ms);

/*
 * Batches: many circuits of uneven width in one persistent launch, replayed
 * as a CUDA graph (the paper's repeated runs of one circuit, Sec. IV-E, e.g.
 * QAOA). qs_batch_create plans circuit c for states[c] (complex64, at most 26
 * qubits, distinct buffers) and uploads every block once. Without QS_FUSE in
 * flags the autotuner times fusion widths k = 2..4 x CTA sizes {256, 512,
 * 1024} (opts->threads fixes the size) on the batch itself and keeps the
 * fastest; QS_FUSE | QS_FUSE_K(k) fixes k (k >= 5 runs 256-thread CTAs).
 * QS_VSWAP and QS_DIAG pass through to the planner. The chosen launch is captured as a CUDA
 * graph on cuda_stream (NULL: a stream owned by the batch). Each
 * qs_batch_run applies every circuit to its state starting from |0...0>
 * (one CTA per circuit; states of <= 14 qubits stay in shared memory for the
 * whole circuit), asynchronously, and sets each state's perm to its circuit's
 * final logical->physical map. The states must outlive the batch.
 */
typedef struct qs_batch qs_batch;

typedef struct {
  int32_t count;          /* circuits */
  int32_t fuse_k;         /* fusion width in use */
  int32_t threads;        /* threads per CTA in use */
  int32_t grid;           /* CTAs launched */
  int32_t total_blocks;   /* fused blocks over all circuits */
  int32_t graph;          /* 1 if runs replay a CUDA graph */
  int32_t n_tuned;        /* autotuner trials recorded below */
  int32_t tuned_k[16];
  int32_t tuned_threads[16];
  double tuned_ms[16];
} qs_batch_info_t;

qs_status qs_batch_create(qs_state *const *states, const qs_gate *const *gates, const size_t *n_gates, int count,
                          uint64_t flags, const qs_opts *opts, void *cuda_stream, qs_batch **out);
qs_status qs_batch_run(qs_batch *b);
qs_status qs_batch_sync(qs_batch *b);   /* waits for the batch's stream */
qs_status qs_batch_info(const qs_batch *b, qs_batch_info_t *out);
void qs_batch_free(qs_batch *b);

/*
 * Sec. IV-E (many simulation runs of one circuit family, e.g. QAOA).
 * One-shot batch: qs_batch_create + one qs_batch_run + qs_batch_sync +
 * qs_batch_free with the same arguments (NULL stream: the batch's own). Each
 * state is set to |0...0> and its circuit applied in one persistent launch;
 * returns after the results are in the states. For repeated runs keep the
 * qs_batch handle instead (planning, upload and autotuning happen once).
 */
qs_status qs_apply_batch(qs_state *const *states, const qs_gate *const *gates, const size_t *n_gates, int count,
                         uint64_t flags, const qs_opts *opts);

const char *qs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QS_ABI_H_ */
