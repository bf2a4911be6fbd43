"""GPU parity at the benchmark's flags and sizes.

At n = 24 the oracle runs whole in seconds, and a launch of the tensor-core
kernels still spans many tiles per CTA (at k = 5, 4096 tiles over about 300
resident CTAs), so every amplitude the benchmark's kernels write in their
steady-state loop is compared with the FP64 oracle: the three benchmark
circuit families under the rule activator (the benchmark's own flags) and
under 6-qubit tensor-core fusion (the measured-profile activator's choice),
and the 40-layer U3 + CX/CZ workload at k = 4, 5, 6 on the tensor cores.
The permutation is compared bit for bit with the one the host passes
predict (qs_plan), and with the oracle's composed SWAPs where nothing was
relocated.

At n = 30 and n = 32 the oracle cannot run whole; there the complex64
result is compared over the whole state with a complex128 run of the same
circuit on the GPU (plain per-gate kernels for the benchmark circuits;
those are pinned to the oracle at 1e-12 by the tests at smaller n), with
qs_state_distance (FP64 accumulation, both states brought to logical
order). Tolerance: L2 <= 1e-5 over all 2^n amplitudes.
"""

import math

import numpy as np
import pytest

import circuitgen as cg
import oracle
import paper_2410_09326_gb300 as qs

pytestmark = pytest.mark.gpu

TOL64 = 1e-5
RULES = qs.QS_PGO_RULES
K6_TC = qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(6) | qs.QS_DIAG | qs.QS_TC

_oracle_cache = {}


@pytest.fixture(scope="module", autouse=True)
def lib():
    return qs.load(build_if_missing=True)


def oracle_state(text):
    if text not in _oracle_cache:
        _oracle_cache.clear()  # one 2^24 state at a time (256 MB)
        _oracle_cache[text] = oracle.simulate(text)
    return _oracle_cache[text]


def circuit(name, n):
    if name == "u3":
        return cg.u3_entangler_circuit(n=n, layers=40)[1]
    c = cg.benchmark_circuits(n=n)
    return c[name][1]


def check_full_state(n, gates, flags, opts=None):
    text = cg.to_qasm(n, gates)
    want, operm = oracle_state(text)
    arr = qs.gates_to_array(gates)
    _, _, plan_perm = qs.qs_plan(n, arr, flags, opts=opts)
    st = qs.qs_alloc_state(n, qs.QS_C64)
    try:
        qs.qs_apply_circuit(st, arr, flags, opts)
        summ, recs = qs.qs_profile(st)
        perm = qs.qs_get_perm(st, n)
        got = qs.qs_read_state(st, n, qs.QS_C64).astype(np.complex128)
    finally:
        qs.qs_free_state(st)
    assert list(perm) == list(plan_perm), (list(perm), list(plan_perm))
    if not any(r.kind == 2 and r.n_gates == 0 for r in recs):  # no relocation exchange in the plan
        assert list(perm) == list(operm), (list(perm), list(operm))
    tc = [r for r in recs if r.tc]
    for r in tc:
        assert r.tiles >= 3 * r.ctas, (r.k, r.tiles, r.ctas)
    err = np.linalg.norm(got - oracle.to_physical(want, perm))
    assert err <= TOL64, err
    return err, tc


@pytest.mark.parametrize("flags", ["rules", "k6_tc"])
@pytest.mark.parametrize("name", ["ghz", "qft", "random"])
def test_benchmark_circuits_n24_vs_oracle(name, flags):
    """The benchmark's three circuit families at n = 24, every amplitude
    against the oracle, under the benchmark's flags (rule activator) and
    under 6-qubit tensor-core fusion."""
    n = 24
    err, tc = check_full_state(n, circuit(name, n), RULES if flags == "rules" else K6_TC)
    if name == "random":
        assert tc, "the random circuit runs tensor-core blocks"
        if flags == "k6_tc":
            assert any(r.k == 6 for r in tc)


@pytest.mark.parametrize("exchange", [0, 1])
@pytest.mark.parametrize("k", [4, 5, 6])
def test_u3_layers_n24_tensor_cores_vs_oracle(k, exchange):
    """40 layers of U3 + CX/CZ at n = 24 fused into k-qubit tensor-core
    blocks (lane-exchange kernels where they pay, or thread-per-group only),
    every amplitude against the oracle."""
    n = 24
    o = qs.qs_default_opts()
    o.tc_exchange = exchange
    flags = qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_DIAG | qs.QS_TC
    err, tc = check_full_state(n, circuit("u3", n), flags, o)
    assert any(r.k == k for r in tc)
    if exchange == 1:
        assert all(r.tc == 1 for r in tc)


def fp64_reference(n, gates, flags=qs.QS_PLAIN):
    ref = qs.qs_alloc_state(n, qs.QS_C128)
    qs.qs_apply_circuit(ref, qs.gates_to_array(gates), flags)
    return ref


@pytest.mark.parametrize("name", ["ghz", "qft", "random"])
def test_bench_size_n30_whole_state_vs_fp64_gpu(name):
    """The benchmark workload itself (n = 30, the benchmark's flags): the
    whole complex64 state against a complex128 run of the plain per-gate
    kernels, L2 <= 1e-5; for the QFT the complex128 run is also checked
    against the closed form exp(2 pi i x y / 2^n) / 2^(n/2) at sampled
    indices to 1e-12."""
    import bench
    n = 30
    if name == "qft":
        gates, x = cg.qft(n, rng=cg.SplitMix64(cg.seed_of(1, 0)))
    else:
        gates = circuit(name, n)
    st = qs.qs_alloc_state(n, qs.QS_C64)
    ref = None
    try:
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), bench.OPT_FLAGS)
        ref = fp64_reference(n, gates)
        if name == "qft":
            perm = qs.qs_get_perm(ref, n)
            psi = qs.qs_read_state(ref, n, qs.QS_C128)
            rng = cg.SplitMix64(17)
            ys = np.array([rng.next() & ((1 << n) - 1) for _ in range(4096)] + [0, (1 << n) - 1])
            phys = np.zeros_like(ys)
            for l in range(n):
                phys |= ((ys >> l) & 1) << int(perm[l])
            want = np.exp(2j * np.pi * ((x * ys) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)
            assert np.abs(psi[phys] - want).max() < 1e-12
            del psi
        if name == "ghz":
            p = qs.qs_measure_probs(ref, [0, n - 1])
            assert abs(p[0] - 0.5) < 1e-12 and abs(p[3] - 0.5) < 1e-12
        dist = qs.qs_state_distance(st, ref)
        assert dist <= TOL64, dist
    finally:
        qs.qs_free_state(st)
        if ref is not None:
            qs.qs_free_state(ref)


def test_u3_layers_n32_tensor_cores_vs_fp64_gpu():
    """The n = 32 workload (32 GiB complex64): 40 layers of U3 + CX/CZ fused
    into 5- and 6-qubit tensor-core blocks, each against one complex128 run
    (64 GiB) of the same circuit on the CUDA cores in FP64 (3-qubit fusion),
    L2 <= 1e-5 over all 2^32 amplitudes."""
    n = 32
    gates = circuit("u3", n)
    arr = qs.gates_to_array(gates)
    st = qs.qs_alloc_state(n, qs.QS_C64)
    ref = None
    try:
        ref = fp64_reference(n, gates, qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(3) | qs.QS_DIAG)
        for k in (5, 6):
            qs.qs_set_basis(st, 0)
            qs.qs_apply_circuit(st, arr, qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_DIAG | qs.QS_TC)
            dist = qs.qs_state_distance(st, ref)
            print(f"n=32 k={k}: L2 vs FP64 GPU run = {dist:.3e} (bound 1e-5)")
            assert dist <= TOL64, (k, dist)
    finally:
        qs.qs_free_state(st)
        if ref is not None:
            qs.qs_free_state(ref)
