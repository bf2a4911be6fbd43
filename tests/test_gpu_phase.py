"""GPU parity of phase-polynomial diagonal blocks against the FP64 oracle.

The kernel splits every term of exp(i phi(x)) by where its bits lie: both
below bit 10 (the chunk's factor table), one below and one above (a per-chunk
factor of that chunk bit), or all above (a chunk-wide factor). The cases
below put terms in each of those places, use random initial states (so every
amplitude matters), the smallest state the kernel takes (n = 11), several
chunks per warp, and both amplitude types, with the usual tolerances
(absolute L2: 1e-5 complex64, 1e-12 complex128).
"""

import math

import numpy as np
import pytest

import circuitgen as cg
import oracle
import paper_2410_09326_gb300 as qs
from tests.test_host import diagonal_circuit

pytestmark = pytest.mark.gpu

TOL = {qs.QS_C64: 1e-5, qs.QS_C128: 1e-12}
FLAGS = qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(4) | qs.QS_DIAG


@pytest.fixture(scope="module", autouse=True)
def lib():
    return qs.load(build_if_missing=True)


def random_state(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


def run(n, gates, dtype, init, flags=FLAGS):
    st = qs.qs_alloc_state(n, dtype)
    try:
        qs.qs_write_state(st, init.astype(np.complex64 if dtype == qs.QS_C64 else np.complex128))
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), flags)
        _, recs = qs.qs_profile(st)
        perm = qs.qs_get_perm(st, n)
        return qs.qs_read_state(st, n, dtype).astype(np.complex128), perm, recs
    finally:
        qs.qs_free_state(st)


def check(n, gates, dtype, seed):
    init = random_state(n, seed)
    want, _ = oracle.simulate(cg.to_qasm(n, gates), init=init)
    got, perm, recs = run(n, gates, dtype, init)
    assert any(r.kind == 4 for r in recs), "no phase polynomial was planned"
    err = np.linalg.norm(got - oracle.to_physical(want, perm))
    assert err <= TOL[dtype], err


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("n", [11, 12, 16, 20])
def test_random_diagonal_runs(dtype, n):
    check(n, diagonal_circuit(n, 300, 7000 + n), dtype, n)


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_terms_in_every_place(dtype):
    n = 14
    gates = [("cp", [2, 5], [0.7]), ("cp", [3, 12], [1.1]), ("cp", [11, 13], [-0.4]), ("rz", [4], [0.9]),
             ("rz", [12], [-1.3]), ("rzz", [0, 13], [0.5]), ("crz", [13, 1], [2.1]), ("t", [10], []),
             ("s", [9], []), ("cz", [10, 11], []), ("u1", [0], [0.2]), ("cu1", [9, 10], [1.7]),
             ("rzz", [5, 6], [-2.2]), ("z", [13], [])]
    check(n, gates, dtype, 3)


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_mixed_with_dense_gates(dtype):
    n = 16
    check(n, diagonal_circuit(n, 500, 7100, dense_every=30), dtype, 4)


def test_qft_closed_form_n22():
    n = 22
    gates, x = cg.qft(n, rng=cg.SplitMix64(cg.seed_of(1, 9)))
    st = qs.qs_alloc_state(n, qs.QS_C64)
    try:
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(5) | qs.QS_DIAG)
        _, recs = qs.qs_profile(st)
        assert any(r.kind == 4 for r in recs)
        perm = qs.qs_get_perm(st, n)
        psi = qs.qs_read_state(st, n, qs.QS_C64).astype(np.complex128)
    finally:
        qs.qs_free_state(st)
    ys = np.arange(1 << n, dtype=np.int64)
    phys = np.zeros_like(ys)
    for l in range(n):
        phys |= ((ys >> l) & 1) << int(perm[l])
    want = np.exp(2j * np.pi * ((x * ys) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)
    assert np.linalg.norm(psi[phys] - want) <= 1e-5


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("ctas", [1, 3])
def test_several_chunks_per_warp(dtype, ctas):
    """The phase kernel's chunk loop (complex64: the next chunk staged in
    shared memory while the current one is applied) over many chunks per
    warp: the launch capped to 1 or 3 CTAs of 8 warps on n = 17 (128
    chunks), against the oracle."""
    n = 17
    gates = diagonal_circuit(n, 300, 7200 + ctas)
    init = random_state(n, 11 + ctas)
    want, _ = oracle.simulate(cg.to_qasm(n, gates), init=init)
    o = qs.qs_default_opts()
    o.tc_max_ctas = ctas
    st = qs.qs_alloc_state(n, dtype)
    try:
        qs.qs_write_state(st, init.astype(np.complex64 if dtype == qs.QS_C64 else np.complex128))
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), FLAGS, opts=o)
        _, recs = qs.qs_profile(st)
        perm = qs.qs_get_perm(st, n)
        got = qs.qs_read_state(st, n, dtype).astype(np.complex128)
    finally:
        qs.qs_free_state(st)
    ph = [r for r in recs if r.kind == 4]
    assert ph and all(r.ctas == ctas and r.tiles == 1 << (n - 10) for r in ph)
    assert all(r.tiles >= 3 * 8 * r.ctas for r in ph)  # several chunks per warp
    err = np.linalg.norm(got - oracle.to_physical(want, perm))
    assert err <= TOL[dtype], err
