"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (absolute L2 over all 2^n amplitudes, after placing the oracle's
logical-order state through the reported permutation): 1e-5 for complex64
(FP32 accumulation) and 1e-12 for complex128. The permutation must match the
oracle's composed SWAP transpositions bit for bit whenever SWAPs are absorbed.
At n = 30 the oracle cannot run whole: the cases here use properties that
hold at any size (GHZ marginals, norm, circuit x inverse = |0...0>); the
whole-state comparisons at n = 24 (oracle) and n = 30, 32 (complex128 GPU
runs) are in test_gpu_bench_parity.py.
"""

import math

import numpy as np
import pytest

import circuitgen as cg
import oracle
import paper_2410_09326_gb300 as qs
from lane_exchange_rule import lane_exchange_expected

pytestmark = pytest.mark.gpu

TOL = {qs.QS_C64: 1e-5, qs.QS_C128: 1e-12}

FLAGS = {
    "plain": qs.QS_PLAIN,
    "vswap": qs.QS_VSWAP,
    "diag": qs.QS_DIAG,
    "pgo_rules": qs.QS_PGO_RULES,
    "pgo_measured": qs.QS_PGO_MEASURED,
    "fold_vswap_k4_diag": qs.QS_FOLD | qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(4) | qs.QS_DIAG,
    "fold_plain": qs.QS_FOLD,
    "relocate_k4_tc": qs.QS_RELOCATE | qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(4) | qs.QS_TC | qs.QS_DIAG,
    **{f"vswap_k{k}": qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k) for k in range(1, 7)},
    **{f"vswap_k{k}_diag": qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_DIAG for k in range(1, 7)},
    **{f"vswap_k{k}_tc": qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_TC for k in (4, 5, 6)},
    **{f"vswap_k{k}_tc_diag": qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_TC | qs.QS_DIAG for k in (4, 5)},
}


@pytest.fixture(scope="module", autouse=True)
def lib():
    return qs.load(build_if_missing=True)


def gpu_run(n, gates, flags, dtype, init=None, logical=False):
    st = qs.qs_alloc_state(n, dtype)
    try:
        if init is not None:
            qs.qs_write_state(st, init.astype(np.complex64 if dtype == qs.QS_C64 else np.complex128))
        qs.qs_apply_circuit(st, gates, flags)
        perm = qs.qs_get_perm(st, n)
        psi = qs.qs_read_state(st, n, dtype, logical_order=logical)
        if logical:
            assert list(qs.qs_get_perm(st, n)) == list(range(n))
        return psi.astype(np.complex128), perm
    finally:
        qs.qs_free_state(st)


def planned_perm(n, arr, flags, dtype):
    """The map the host passes predict for these flags (the measured-profile
    activator of a fresh state has no measurements: its choice is the priors')."""
    if flags & qs.QS_PGO_MEASURED:
        flags, _ = qs.qs_pgo_select(n, arr, dtype=dtype)
    return [int(x) for x in qs.qs_plan(n, arr, flags)[2]]


def check(n, gates, flags, dtype, init=None):
    text = cg.to_qasm(n, gates)
    want, operm = oracle.simulate(text, init=init)
    arr = qs.gates_to_array(gates)
    got, perm = gpu_run(n, arr, flags, dtype, init=init)
    pgo = qs.QS_PGO_RULES | qs.QS_PGO_MEASURED | qs.QS_RELOCATE
    # bit-exact against the host plan's map under every flag set (relocation
    # and activator choices included), and against the oracle's composed
    # SWAP transpositions where only virtual swap relabels
    assert list(perm) == planned_perm(n, arr, flags, dtype), (list(perm), hex(flags))
    if flags & qs.QS_VSWAP and not flags & pgo and any(g[0] == "swap" for g in gates):
        assert list(perm) == list(operm), (list(perm), list(operm))
    elif not flags & (qs.QS_VSWAP | pgo):
        assert list(perm) == list(range(n))
    assert sorted(perm) == list(range(n))
    err = np.linalg.norm(got - oracle.to_physical(want, perm))
    assert err <= TOL[dtype], (err, flags)
    return err


@pytest.mark.parametrize("name", sorted(FLAGS))
@pytest.mark.parametrize("index", [0, 1, 2])
def test_layered_swaps_n12_c128(name, index):
    """n=12 complex128 layered random circuit with 10 SWAPs."""
    n, gates = cg.layered_swaps_circuit(index)
    check(n, gates, FLAGS[name], qs.QS_C128)


@pytest.mark.parametrize("name", sorted(FLAGS))
@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("n", [2, 5, 9, 14])
def test_all_gate_types(name, dtype, n):
    """Every gate type, targets low/high/mixed, controls above and below."""
    rng = cg.SplitMix64(9000 + n)
    gates = cg.all_gate_types_circuit(n, 120 if n > 9 else 200, rng)
    init = None
    if n == 9:
        init = np.array([rng.uniform(-1, 1) + 1j * rng.uniform(-1, 1) for _ in range(1 << n)])
        init /= np.linalg.norm(init)
    check(n, gates, FLAGS[name], dtype, init=init)


@pytest.mark.parametrize("tc", [0, qs.QS_TC])
@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_dense_block_every_target_class(dtype, k, tc):
    """One dense k-qubit block per target placement class at n=13."""
    n = 13
    rng = cg.SplitMix64(31 * k)
    placements = [list(range(k)), list(range(n - k, n)), [0] + list(range(n - k + 1, n)),
                  sorted(rng.shuffle(list(range(n)))[:k])]
    for qubits in placements:
        gates = []
        for _ in range(3):
            for q in qubits:
                gates.append(("u3", [q], [rng.uniform(0, 6.28) for _ in range(3)]))
            for a, b in zip(qubits[:-1], qubits[1:]):
                gates.append(("cx", [a, b]))
        # a control outside the block exercises the controlled subspace
        check(n, gates, qs.QS_FUSE | qs.QS_FUSE_K(k) | tc, dtype)
        outside = [q for q in range(n) if q not in qubits][0]
        gates2 = [("h", [outside])] + [("ccx", [outside, qubits[0], qubits[-1]])] if k > 1 else gates
        check(n, gates + gates2, qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_DIAG | tc, dtype)


def random_state(n, rng):
    init = np.array([rng.uniform(-1, 1) + 1j * rng.uniform(-1, 1) for _ in range(1 << n)])
    return init / np.linalg.norm(init)


def block_gates(qubits, rng, ctrl=None, reps=2):
    """Two layers of U3 on every target and a CX (CCX with a control) chain:
    one dense block on `qubits` (controlled by `ctrl`)."""
    gates = []
    for _ in range(reps):
        if ctrl is None:
            gates += [("u3", [q], [rng.uniform(0, 6.28) for _ in range(3)]) for q in qubits]
            gates += [("cx", [a, b]) for a, b in zip(qubits[:-1], qubits[1:])]
        else:
            gates += [("cu3", [ctrl, q], [rng.uniform(0, 6.28) for _ in range(3)]) for q in qubits]
            gates += [("ccx", [ctrl, a, b]) for a, b in zip(qubits[:-1], qubits[1:])]
    return gates


def run_tc_block(n, gates, width, init, opts):
    st = qs.qs_alloc_state(n, qs.QS_C64)
    try:
        qs.qs_write_state(st, init.astype(np.complex64))
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), qs.QS_FUSE | qs.QS_FUSE_K(width) | qs.QS_TC, opts)
        _, recs = qs.qs_profile(st)
        got = qs.qs_read_state(st, n, qs.QS_C64).astype(np.complex128)
    finally:
        qs.qs_free_state(st)
    return got, recs


@pytest.mark.parametrize("max_ctas", [3, 5])
@pytest.mark.parametrize("exchange", [1, 2])
@pytest.mark.parametrize("k", [4, 5, 6])
def test_tc_steady_state_loop(k, exchange, max_ctas):
    """Every tensor-core kernel through its steady-state tile loop: the
    launch is capped at 3 or 5 CTAs (opts.tc_max_ctas), so each CTA runs at
    least three tiles -- the next tile's gather or cp.async staging while the
    current tile's MMAs run, the alternation of the two staging areas, the
    mbarrier phase flips -- and a ragged last round (tiles not a multiple of
    the CTAs). Thread-per-group (exchange 1) and lane-exchange (exchange 2)
    kernels, high, low, bit-0 and mixed targets, with and without a control,
    n = 17, from a random state, against the oracle element by element; the
    record shows tiles >= 3 x CTAs."""
    n = 17
    rng = cg.SplitMix64(4000 + 10 * k + exchange + max_ctas)
    init = random_state(n, rng)
    o = qs.qs_default_opts()
    o.tc_exchange = exchange
    o.tc_max_ctas = max_ctas
    patterns = [([12, 13, 14, 15, 16, 11], None), ([0, 1, 2, 3, 4, 5], None), ([1, 2, 8, 9, 10, 11], None),
                ([0, 3, 7, 12, 14, 16], None), ([2, 3, 9, 10, 11], 6), ([0, 5, 9, 13, 15], 16)]
    for pattern, ctrl in patterns:
        if ctrl is not None and k == 6:
            continue  # 7 fused qubits
        qubits = sorted(pattern[:k])
        gates = block_gates(qubits, rng, ctrl)
        width = k + (0 if ctrl is None else 1)
        want, _ = oracle.simulate(cg.to_qasm(n, gates), init=init)
        got, recs = run_tc_block(n, gates, width, init, o)
        blk = [r for r in recs if r.kind == 0 and r.k == k]
        assert len(blk) == 1 and blk[0].tc in (1, 2), (qubits, ctrl)
        assert blk[0].ctas <= max_ctas and blk[0].tiles >= 3 * blk[0].ctas, (blk[0].tiles, blk[0].ctas)
        if exchange == 2:
            assert blk[0].tc == 2, (qubits, ctrl)
        assert np.linalg.norm(got - want) <= 1e-5, (qubits, ctrl)


@pytest.mark.parametrize("max_ctas", [0, 3])
@pytest.mark.parametrize("k", [4, 5])
def test_tc_tf32_operands(k, max_ctas):
    """The 3 x TF32 tensor-core kernel (opts.tc_precision = 1, the precision
    option beside the default FP16 halves): high, low, bit-0 and mixed
    targets, with and without a control, one wave of CTAs or 3 CTAs looping
    over the tiles, n = 17 from a random state, against the oracle."""
    n = 17
    rng = cg.SplitMix64(6100 + 10 * k + max_ctas)
    init = random_state(n, rng)
    o = qs.qs_default_opts()
    o.tc_precision = 1
    o.tc_max_ctas = max_ctas
    for pattern, ctrl in (([12, 13, 14, 15, 16], None), ([0, 1, 2, 3, 4], None), ([1, 2, 8, 9, 10], None),
                          ([0, 5, 9, 13, 15], 16)):
        qubits = sorted(pattern[:k])
        gates = block_gates(qubits, rng, ctrl)
        want, _ = oracle.simulate(cg.to_qasm(n, gates), init=init)
        got, recs = run_tc_block(n, gates, k + (0 if ctrl is None else 1), init, o)
        blk = [r for r in recs if r.kind == 0 and r.k == k]
        assert len(blk) == 1 and blk[0].tc == 1, (qubits, ctrl)
        if max_ctas:
            assert blk[0].ctas <= max_ctas and blk[0].tiles >= 3 * blk[0].ctas
        assert np.linalg.norm(got - want) <= 1e-5, (qubits, ctrl)


@pytest.mark.parametrize("max_ctas", [0, 4])
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("k,ctrl", [(4, None), (4, 5), (4, 0), (5, None), (5, 5), (5, 0), (6, None)])
@pytest.mark.parametrize("n", [12, 17])
def test_tc_lane_exchange(n, k, ctrl, mode, max_ctas):
    """4-, 5- and 6-target (two threads per group; a controlled one would
    need 7 fused qubits) tensor-core blocks with lane-exchange gathers
    (opts.tc_exchange: 0 automatic, 1 never, 2 wherever the layout allows)
    on low-bit target patterns (no exchange, the element bit's exchange, one
    or two lane/register exchanges, targets moved from lane to register bits
    to keep two or because they lie past the first 128-byte run), without a
    control, with a control on bit 5 and with bit 0 a control (no exchange
    layout), one tile (n = 12) and many (n = 17), one
    wave of CTAs or at most 4 CTAs looping over the tiles, from a random
    state; the record's tc field says which kernel ran (2 = lane exchange)."""
    rng = cg.SplitMix64(1300 + 10 * k + n + (ctrl or 0))
    o = qs.qs_default_opts()
    o.tc_exchange = mode
    o.tc_max_ctas = max_ctas
    init = np.array([rng.uniform(-1, 1) + 1j * rng.uniform(-1, 1) for _ in range(1 << n)])
    init /= np.linalg.norm(init)
    patterns = ([7, 8, 9, 10, 11], [1, 7, 8, 9, 10], [2, 7, 8, 9, 10], [3, 7, 8, 9, 10], [0, 7, 8, 9, 10],
                [0, 1, 8, 9, 10], [1, 2, 8, 9, 10], [2, 3, 8, 9, 10], [1, 2, 3, 9, 10], [0, 1, 2, 3, 9],
                [0, 1, 2, 3, 4], [1, 2, 3, 4, 5], [1, 4, 9, 10, 11], [0, 2, 5, 9, 10])
    kinds = set()
    for pattern in patterns:
        # 6 targets: the pattern plus the lowest qubit above it
        qubits = pattern[:k] if k <= 5 else pattern + [max(pattern) + 1]
        if ctrl is not None and ctrl in qubits or max(qubits) >= n:
            continue
        ctrls = [] if ctrl is None else [ctrl]
        if ctrl is None:
            gates = []
            for _ in range(2):
                gates += [("u3", [q], [rng.uniform(0, 6.28) for _ in range(3)]) for q in qubits]
                gates += [("cx", [a, b]) for a, b in zip(qubits[:-1], qubits[1:])]
        else:
            gates = []  # the random state already spreads over the control's values
            for _ in range(2):
                gates += [("cu3", [ctrl, q], [rng.uniform(0, 6.28) for _ in range(3)]) for q in qubits]
                gates += [("ccx", [ctrl, a, b]) for a, b in zip(qubits[:-1], qubits[1:])]
        want, _ = oracle.simulate(cg.to_qasm(n, gates), init=init)
        st = qs.qs_alloc_state(n, qs.QS_C64)
        try:
            qs.qs_write_state(st, init.astype(np.complex64))
            qs.qs_apply_circuit(st, qs.gates_to_array(gates), qs.QS_FUSE | qs.QS_FUSE_K(k + len(ctrls)) | qs.QS_TC, o)
            _, recs = qs.qs_profile(st)
            blk = [r for r in recs if r.kind == 0 and r.k == k]
            assert len(blk) == 1 and [int(x) for x in blk[0].qubits[:k]] == qubits and blk[0].nctrl == len(ctrls)
            fits, pays = lane_exchange_expected(n, qubits, ctrls)
            expect = fits and (mode == 2 or (mode == 0 and pays))
            assert blk[0].tc == (2 if expect else 1), (qubits, ctrl, mode, blk[0].tc)
            if max_ctas:
                assert blk[0].ctas <= max_ctas
            kinds.add(int(blk[0].tc))
            got = qs.qs_read_state(st, n, qs.QS_C64).astype(np.complex128)
        finally:
            qs.qs_free_state(st)
        assert np.linalg.norm(got - want) <= 1e-5, (qubits, ctrl, mode)
    if mode == 2 and ctrl != 0 and n == 17:
        assert 2 in kinds
    if k == 5 and ctrl is None:
        # both ways of doing the lane/register exchanges run above: in the
        # staging copies (exchanged lane bit >= 1, and bits 0..4 on the
        # element and lane bits or the exchanged bit >= 3) and by shuffles
        staged = []
        for pattern in patterns:
            x = qs.qs_tc_exchange_layout(n, pattern)
            if x.applies and x.nswb:
                lanes = [int(b) for b in x.lane_bits]
                long_runs = {1, 2, 3, 4} <= set(lanes)
                staged += [int(x.lb[i]) >= 1 and (long_runs or lanes[int(x.lb[i])] >= 3) for i in range(x.nswb)]
        assert any(staged) and not all(staged), staged


@pytest.mark.parametrize("shuffles", [0, 1])
@pytest.mark.parametrize("n", [9, 12, 16])
def test_low_target_warp_shuffle_kernel(n, shuffles):
    """3-target blocks on bits 1, 2, 3 (bit 0 free): the warp-shuffle kernel
    (default) and the thread-per-group kernel (opts.no_shuffles = 1), with and
    without a control above bit 5, from a random state."""
    rng = cg.SplitMix64(900 + n)
    o = qs.qs_default_opts()
    o.no_shuffles = shuffles
    init = np.array([rng.uniform(-1, 1) + 1j * rng.uniform(-1, 1) for _ in range(1 << n)])
    init /= np.linalg.norm(init)
    for extra in ([], [("h", [n - 1]), ("ccx", [n - 1, 1, 3])]):
        gates = []
        for _ in range(2):
            gates += [("u3", [q], [rng.uniform(0, 6.28) for _ in range(3)]) for q in (1, 2, 3)]
            gates += [("cx", [1, 2]), ("cx", [3, 1])]
        gates += extra
        want, _ = oracle.simulate(cg.to_qasm(n, gates), init=init)
        st = qs.qs_alloc_state(n, qs.QS_C64)
        try:
            qs.qs_write_state(st, init.astype(np.complex64))
            qs.qs_apply_circuit(st, qs.gates_to_array(gates), qs.QS_FUSE | qs.QS_FUSE_K(3), o)
            _, recs = qs.qs_profile(st)
            assert any(r.kind == 0 and r.k == 3 and [int(x) for x in r.qubits[:3]] == [1, 2, 3] for r in recs)
            got = qs.qs_read_state(st, n, qs.QS_C64).astype(np.complex128)
        finally:
            qs.qs_free_state(st)
        assert np.linalg.norm(got - want) <= 1e-5


@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny_registers(n):
    rng = cg.SplitMix64(77 + n)
    gates = cg.all_gate_types_circuit(n, 50, rng)
    for name in ("plain", "vswap_k6_diag", "vswap_k2"):
        check(n, gates, FLAGS[name], qs.QS_C64)
        check(n, gates, FLAGS[name], qs.QS_C128)


def test_empty_circuit_and_identity():
    for dtype in (qs.QS_C64, qs.QS_C128):
        got, perm = gpu_run(6, qs.gates_to_array([]), qs.QS_PLAIN, dtype)
        assert got[0] == 1 and np.count_nonzero(got) == 1
        got, perm = gpu_run(6, qs.gates_to_array([("h", [2]), ("h", [2])]), FLAGS["vswap_k4_diag"], dtype)
        assert got[0] == 1 and np.count_nonzero(got) == 1


# ---------------------------------------------------------------------------
# Closed forms at larger n
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["plain", "vswap", "vswap_k4_diag", "vswap_k6_diag"])
def test_ghz_n24(name):
    n = 24
    got, perm = gpu_run(n, qs.gates_to_array(cg.ghz(n)), FLAGS[name], qs.QS_C64)
    want = np.zeros(1 << n)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert np.linalg.norm(got - want) < 1e-5


@pytest.mark.parametrize("name", ["plain", "vswap", "vswap_k2_diag", "vswap_k5_diag"])
@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_qft_closed_form_n18(name, dtype):
    n = 18
    gates, x = cg.qft(n, x=123457)
    got, perm = gpu_run(n, qs.gates_to_array(gates), FLAGS[name], dtype, logical=True)
    y = np.arange(1 << n, dtype=np.int64)
    # reduce x*y mod 2^n first: the FP64 phase argument stays exact
    want = np.exp(2j * np.pi * ((x * y) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)
    assert np.linalg.norm(got - want) < TOL[dtype]


def test_benchmark_random_n20_vs_oracle():
    """The 30-layer random circuit with 5% SWAPs of the n=28 workload, at n=20."""
    c = cg.benchmark_circuits(n=20)
    n, gates = c["random"]
    for name in ("plain", "vswap", "vswap_k3_diag", "vswap_k5_diag", "vswap_k4_tc_diag", "vswap_k5_tc_diag"):
        check(n, gates, FLAGS[name], qs.QS_C64)


@pytest.mark.parametrize("flags,exchange", [("vswap_k4_tc", 1)])
def test_relocation_speeds_up_a_low_heavy_circuit(flags, exchange):
    """Blocks whose targets include bits 0 and 1 gather at a 32-byte stride
    on the thread-per-group tensor-core kernel (opts.tc_exchange = 1);
    moving those bits up front (two half-state exchanges) pays off there.
    The exchange kernels read such blocks in whole sectors and the 3-target
    CUDA-core kernels lose little on them, which leaves relocation about
    neutral there (measured within 1%; not asserted)."""
    from tests.test_host import low_heavy_circuit
    n = 26
    gates = low_heavy_circuit(n, reps=60, seed=5, swaps=False)
    arr = qs.gates_to_array(gates)
    o = qs.qs_default_opts()
    o.tc_exchange = exchange
    st = qs.qs_alloc_state(n, qs.QS_C64)
    try:
        t = {}
        for name, f in (("base", FLAGS[flags]), ("reloc", FLAGS[flags] | qs.QS_RELOCATE)):
            best = 1e9
            for _ in range(3):
                qs.qs_set_basis(st, 0)
                qs.qs_apply_circuit(st, arr, f | qs.QS_PROFILE, o)
                summ, _ = qs.qs_profile(st, with_records=False)
                best = min(best, summ.total_ms)
            t[name] = best
        assert t["reloc"] < t["base"], t
    finally:
        qs.qs_free_state(st)


def test_tc_blocks_really_run_on_tensor_cores():
    n = 16
    rng = cg.SplitMix64(12)
    gates = cg.random_layered(n, 8, rng, one_q=("u3",), two_q=("cx", "cz"))
    st = qs.qs_alloc_state(n, qs.QS_C64)
    try:
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), FLAGS["vswap_k5_tc_diag"] | qs.QS_PROFILE)
        summ, recs = qs.qs_profile(st)
        assert any(r.tc for r in recs) and all(bool(r.tc) == (r.kind == 0 and r.k in (4, 5)) for r in recs)
    finally:
        qs.qs_free_state(st)


# ---------------------------------------------------------------------------
# Reductions
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_probs_and_norm(dtype):
    n = 14
    rng = cg.SplitMix64(5)
    gates = cg.random_layered(n, 6, rng, n_swaps=5)
    text = cg.to_qasm(n, gates)
    want, _ = oracle.simulate(text)
    st = qs.qs_alloc_state(n, dtype)
    try:
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), FLAGS["vswap_k4_diag"])
        tol = 1e-6 if dtype == qs.QS_C64 else 1e-13
        assert abs(qs.qs_norm(st) - 1.0) < tol
        for qubits in ([0], [13], [3, 7], [12, 0, 5], list(range(10)), list(range(12)),
                       list(range(13)), list(range(n)), [], [13, 12, 11, 10, 9, 8, 7, 6, 5, 4, 3, 2, 1, 0]):
            got = qs.qs_measure_probs(st, qubits)
            ref = oracle.probs(want, qubits) if qubits else np.array([1.0])
            assert np.abs(got - ref).max() < tol, qubits
    finally:
        qs.qs_free_state(st)


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_wide_marginals_n20(dtype):
    """More than 12 measured qubits: the chunked kernel, low/high/mixed bits."""
    n = 20
    rng = cg.SplitMix64(8)
    gates = cg.random_layered(n, 5, rng, n_swaps=6)
    want, _ = oracle.simulate(cg.to_qasm(n, gates))
    st = qs.qs_alloc_state(n, dtype)
    try:
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), FLAGS["vswap_k3_diag"])
        subsets = [list(range(16)), list(range(4, 20)), list(range(19, 3, -1)),
                   sorted(rng.shuffle(list(range(n)))[:14]), list(range(n))[::-1], list(range(13))]
        tol = 1e-6 if dtype == qs.QS_C64 else 1e-13
        for qubits in subsets:
            got = qs.qs_measure_probs(st, qubits)
            ref = oracle.probs(want, qubits)
            assert np.abs(got - ref).max() < tol, (qubits, np.abs(got - ref).max())
            assert abs(got.sum() - 1) < 10 * tol
    finally:
        qs.qs_free_state(st)


def test_measured_pgo_regret():
    """The measured-profile activator, fed by profiled runs of the candidate
    flag sets on this GPU, picks a set whose measured time is within 15% of
    the best candidate's (brute force over the same candidates)."""
    n = 24
    c = cg.benchmark_circuits(n=n)
    _, gates = c["random"]
    arr = qs.gates_to_array(gates)
    st = qs.qs_alloc_state(n, qs.QS_C64)
    try:
        times = {}
        cands = [qs.QS_PLAIN, qs.QS_VSWAP] + [qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_DIAG
                                             for k in range(1, 7)] + \
                [qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_DIAG | qs.QS_TC for k in (4, 5, 6)]
        for f in cands:
            best = 1e9
            for _ in range(2):
                qs.qs_set_basis(st, 0)
                qs.qs_apply_circuit(st, arr, f | qs.QS_PROFILE)
                summ, _ = qs.qs_profile(st, with_records=False)
                best = min(best, summ.total_ms)
            times[f] = best
        table = qs.qs_profile_classes(st)
        chosen, pred = qs.qs_pgo_select(n, arr, table=table)
        qs.qs_set_basis(st, 0)
        qs.qs_apply_circuit(st, arr, chosen | qs.QS_PROFILE)
        summ, _ = qs.qs_profile(st, with_records=False)
        t_chosen = min(summ.total_ms, times.get(chosen, 1e9))
        assert t_chosen <= 1.15 * min(times.values()), (hex(chosen), t_chosen, sorted(times.values())[:3])
        # QS_PGO_MEASURED inside apply uses the same table and stays correct
        qs.qs_set_basis(st, 0)
        qs.qs_apply_circuit(st, arr, qs.QS_PGO_MEASURED)
        summ, _ = qs.qs_profile(st, with_records=False)
        assert summ.flags_used & qs.QS_FUSE
    finally:
        qs.qs_free_state(st)


# ---------------------------------------------------------------------------
# API behaviour
# ---------------------------------------------------------------------------

def test_errors_leave_state_usable():
    st = qs.qs_alloc_state(5, qs.QS_C64)
    try:
        bad = qs.gates_to_array([("h", [0])])
        bad[0]["q"][0] = 7
        with pytest.raises(qs.QsError) as e:
            qs.qs_apply_circuit(st, bad, qs.QS_PLAIN)
        assert e.value.status == qs.QS_EINVAL
        with pytest.raises(qs.QsError):
            qs.qs_measure_probs(st, [5])
        with pytest.raises(qs.QsError):
            qs.qs_measure_probs(st, [1, 1])
        qs.qs_apply_circuit(st, qs.gates_to_array([("x", [4])]), qs.QS_PLAIN)
        assert np.allclose(qs.qs_measure_probs(st, [4]), [0, 1])
    finally:
        qs.qs_free_state(st)
    with pytest.raises(qs.QsError) as e:
        qs.qs_alloc_state(35, qs.QS_C64)
    assert e.value.status == qs.QS_EUNSUPPORTED


@pytest.mark.parametrize("k,exchange,precision", [(4, 1, 0), (4, 2, 0), (5, 0, 0), (5, 1, 0), (6, 2, 0), (6, 1, 0),
                                                   (5, 0, 1)])
def test_bounded_wait_times_out_and_state_recovers(k, exchange, precision):
    """Failure detection without a GPU fault: the test hook withholds the
    tensor cores' completion signal, the kernel's 1 s wait runs out, the CTA
    frees its TMEM and returns, and the next synchronising call reports
    QS_ETIMEOUT. The state stays usable. Lane-exchange kernels (4, 5 targets
    staged by cp.async, 6 targets), the thread-per-group ones and the 3 x TF32
    one."""
    n = 14
    gates = [("u3", [q], [0.1 * q, 0.2, 0.3]) for q in range(k)] + [("cx", [q, q + 1]) for q in range(0, k - 1, 2)]
    gates += [("cx", [k - 2, k - 1])]
    arr = qs.gates_to_array(gates)
    st = qs.qs_alloc_state(n, qs.QS_C64)
    try:
        opts = qs.qs_default_opts()
        opts.test_wait_timeout = 1
        opts.tc_exchange = exchange
        opts.tc_precision = precision
        qs.qs_apply_circuit(st, arr, qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_TC, opts)
        _, recs = qs.qs_profile(st)
        assert [r.tc for r in recs if r.kind == 0 and r.k == k] == [1 if exchange == 1 or precision else 2]
        with pytest.raises(qs.QsError) as e:
            qs.qs_norm(st)
        assert e.value.status == qs.QS_ETIMEOUT
        # the error is reported once; the state can be reset and used again
        opts.test_wait_timeout = 0
        qs.qs_set_basis(st, 0)
        qs.qs_apply_circuit(st, arr, qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_TC, opts)
        want, _ = oracle.simulate(cg.to_qasm(n, gates))
        got = qs.qs_read_state(st, n, qs.QS_C64).astype(np.complex128)
        assert np.linalg.norm(got - want) < 1e-5
    finally:
        qs.qs_free_state(st)


def test_apply_rejects_global_bits():
    """The global-bit tier (opts.n_global) is planned by qs_plan only: a
    single-GPU apply call refuses it before launching anything."""
    st = qs.qs_alloc_state(10, qs.QS_C64)
    try:
        o = qs.qs_default_opts()
        o.n_global = 1
        with pytest.raises(qs.QsError) as e:
            qs.qs_apply_circuit(st, qs.gates_to_array([("h", [9])]), qs.QS_PLAIN, o)
        assert e.value.status == qs.QS_EUNSUPPORTED
        assert qs.qs_measure_probs(st, [9])[0] == 1.0
    finally:
        qs.qs_free_state(st)


def test_chrome_trace_of_a_profiled_call(tmp_path):
    """A profiled apply call (QS_PROFILE) exported as a Chrome trace: one
    event per launched block, durations summing to the profile's device time,
    starts in launch order."""
    import json

    from paper_2410_09326_gb300 import trace
    n = 16
    gates = cg.random_layered(n, 6, cg.SplitMix64(88), n_swaps=3)
    st = qs.qs_alloc_state(n, qs.QS_C64)
    try:
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), qs.QS_PGO_RULES | qs.QS_PROFILE)
        summ, recs = qs.qs_profile(st)
        path = tmp_path / "trace.json"
        assert trace.write_chrome_trace(st, str(path)) == len(recs) > 0
    finally:
        qs.qs_free_state(st)
    ev = json.loads(path.read_text())["traceEvents"]
    assert abs(sum(e["dur"] for e in ev) / 1e3 - summ.total_ms) < 1e-6 * max(1.0, summ.total_ms)
    starts = [e["ts"] for e in ev]
    assert starts == sorted(starts)


def test_memory_budget_on_device():
    """The device-memory budget counts the state and the scratch the library
    allocates: with room for the state only, a 6-qubit block (its matrix goes
    through a device buffer) is refused with QS_ENOMEM before anything runs;
    without the budget the same call runs and matches the oracle; freeing the
    state returns the live byte count to where it was."""
    n = 16
    base = qs.qs_memory_in_use()
    qs.qs_set_memory_limit(base + (8 << n) + 4096)
    gates = [("u3", [q], [0.1 * q, 0.2, 0.3]) for q in range(6)] + [("cx", [q, q + 1]) for q in range(5)]
    arr = qs.gates_to_array(gates)
    try:
        st = qs.qs_alloc_state(n, qs.QS_C64)
        try:
            assert qs.qs_memory_in_use() == base + (8 << n)
            with pytest.raises(qs.QsError) as e:
                qs.qs_apply_circuit(st, arr, qs.QS_FUSE | qs.QS_FUSE_K(6))
            assert e.value.status == qs.QS_ENOMEM
            qs.qs_set_memory_limit(0)
            qs.qs_apply_circuit(st, arr, qs.QS_FUSE | qs.QS_FUSE_K(6))
            want, _ = oracle.simulate(cg.to_qasm(n, gates))
            got = qs.qs_read_state(st, n, qs.QS_C64).astype(np.complex128)
            assert np.linalg.norm(got - want) < 1e-5
        finally:
            qs.qs_free_state(st)
        assert qs.qs_memory_in_use() == base
    finally:
        qs.qs_set_memory_limit(0)


def test_attach_torch_tensor_and_stream():
    torch = pytest.importorskip("torch")
    n = 12
    buf = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    buf[0] = 1
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    st = qs.qs_attach_state(buf.data_ptr(), n, qs.QS_C64, stream=s)
    try:
        gates = cg.ghz(n)
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), FLAGS["vswap_k3_diag"])
        s.synchronize()
        out = buf.cpu().numpy()
        assert abs(out[0] - 1 / math.sqrt(2)) < 1e-6 and abs(out[-1] - 1 / math.sqrt(2)) < 1e-6
    finally:
        qs.qs_free_state(st)
    assert buf.is_cuda  # memory stays the caller's


def test_set_basis_and_profile_records():
    n = 16
    st = qs.qs_alloc_state(n, qs.QS_C64)
    try:
        qs.qs_set_basis(st, 0b1011)
        p = qs.qs_measure_probs(st, [0, 1, 2, 3])
        assert p[0b1011] == 1.0
        gates, x = cg.qft(n, x=99)
        qs.qs_profile_reset(st)
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), FLAGS["vswap_k2_diag"] | qs.QS_PROFILE)
        summ, recs = qs.qs_profile(st)
        assert summ.n_blocks == len(recs) > 0 and summ.swaps_absorbed == n // 2
        assert all(r.ms > 0 for r in recs) and summ.total_ms > 0
        assert summ.gates_seen == len(gates)
        # counter table: H on every qubit once, CPhase on q_j j times as target
        hcol = [summ.counters[q][0] for q in range(n)]
        assert hcol == [1] * n
        assert sum(summ.counters[q][11] for q in range(n)) == 2 * (n * (n - 1) // 2)
        assert sum(r.n_gates for r in recs) <= len(gates)
    finally:
        qs.qs_free_state(st)


# ---------------------------------------------------------------------------
# Benchmark sizes: closed forms at sampled indices, properties at any size
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["plain", "pgo"])
def test_bench_size_n30_ghz_marginals(name):
    """GHZ at n = 30: the whole probability mass on |0..0> and |1..1> (the
    whole-state comparisons of the benchmark circuits against a complex128
    run are in test_gpu_bench_parity.py)."""
    import bench
    n = 30
    flags = bench.PLAIN_FLAGS if name == "plain" else bench.OPT_FLAGS
    st = qs.qs_alloc_state(n, qs.QS_C64)
    try:
        qs.qs_apply_circuit(st, qs.gates_to_array(cg.ghz(n)), flags)
        p = qs.qs_measure_probs(st, [0, n - 1])
        assert abs(p[0] - 0.5) < 1e-5 and abs(p[3] - 0.5) < 1e-5 and p[1] + p[2] < 1e-10
        assert abs(qs.qs_norm(st) - 1) < 1e-5
    finally:
        qs.qs_free_state(st)


def test_bench_size_n30_random_times_inverse():
    import bench
    from tests.test_oracle_pins import _inverse
    n = 30
    c = cg.benchmark_circuits(n=n)
    _, gates = c["random"]
    st = qs.qs_alloc_state(n, qs.QS_C64)
    try:
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), bench.OPT_FLAGS)
        assert abs(qs.qs_norm(st) - 1) < 1e-5
        qs.qs_apply_circuit(st, qs.gates_to_array(_inverse(gates)), bench.OPT_FLAGS)
        p = qs.qs_measure_probs(st, list(range(12)))
        # back to |0...0>: amplitude error e gives 1 - p0 <= e^2 and p0 >= (1 - e)^2
        assert p[0] > (1 - 1e-5) ** 2
    finally:
        qs.qs_free_state(st)
