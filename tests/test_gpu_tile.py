"""GPU parity of cache-blocked passes (QS_TILE) against the FP64 oracle.

A tile pass gathers 2^m amplitudes spanning the tile's qubits into shared
memory, applies its member blocks there and scatters them back, so the cases
cover: tiles of every width the options allow (m = 8..14, several tiles per
state and a single tile row), member fusion widths 1..4, controls and
diagonal qubits outside the tile, circuits with every gate type, the QFT's
long diagonal runs, and both amplitude types. Tolerances are the ones of the
other parity tests (absolute L2: 1e-5 complex64, 1e-12 complex128); the
permutation must equal the oracle's composed SWAP transpositions exactly.
"""

import math

import numpy as np
import pytest

import circuitgen as cg
import oracle
import paper_2410_09326_gb300 as qs

pytestmark = pytest.mark.gpu

TOL = {qs.QS_C64: 1e-5, qs.QS_C128: 1e-12}
TILE = qs.QS_VSWAP | qs.QS_TILE


@pytest.fixture(scope="module", autouse=True)
def lib():
    return qs.load(build_if_missing=True)


def random_state(n, seed):
    rng = cg.SplitMix64(seed)
    v = np.array([rng.uniform(-1, 1) + 1j * rng.uniform(-1, 1) for _ in range(1 << n)])
    return v / np.linalg.norm(v)


def opts(bits=0, k=0):
    o = qs.qs_default_opts()
    o.tile_bits = bits
    o.tile_k = k
    return o


def run(n, gates, flags, dtype, o, init=None):
    st = qs.qs_alloc_state(n, dtype)
    try:
        if init is not None:
            qs.qs_write_state(st, init.astype(np.complex64 if dtype == qs.QS_C64 else np.complex128))
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), flags, o)
        _, recs = qs.qs_profile(st)
        perm = qs.qs_get_perm(st, n)
        psi = qs.qs_read_state(st, n, dtype).astype(np.complex128)
        return psi, perm, recs
    finally:
        qs.qs_free_state(st)


def check(n, gates, dtype, o, flags=TILE, init=None, want_tiles=True):
    want, operm = oracle.simulate(cg.to_qasm(n, gates), init=init)
    got, perm, recs = run(n, gates, flags, dtype, o, init=init)
    if flags & qs.QS_VSWAP:
        assert list(perm) == list(operm)
    err = np.linalg.norm(got - oracle.to_physical(want, perm))
    assert err <= TOL[dtype], err
    tiles = [r for r in recs if r.kind == 3]
    if want_tiles:
        assert tiles, "no tile pass was planned"
        for r in tiles:
            assert r.k == (o.tile_bits or (12 if dtype == qs.QS_C128 else 13)) and r.meta == 5
    return err, len(tiles)


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("bits,k", [(8, 1), (8, 2), (9, 3), (10, 4), (12, 3), (13, 2)])
def test_random_layered_vs_oracle(dtype, bits, k):
    if dtype == qs.QS_C128 and bits > 13:
        pytest.skip("c128 tiles are at most 13 qubits")
    n = 16
    gates = cg.random_layered(n, 8, cg.SplitMix64(cg.seed_of(0, 700 + bits + k)), n_swaps=4)
    check(n, gates, dtype, opts(bits, k))


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("n", [9, 12, 15])
def test_every_gate_type(dtype, n):
    gates = cg.all_gate_types_circuit(n, 150, cg.SplitMix64(cg.seed_of(0, 800 + n)))
    check(n, gates, dtype, opts(8, 3))


def test_single_row_of_tiles_and_widest_tile():
    # n = m + 1: two tiles; m = 14: 128 KiB tiles (c64)
    n = 15
    gates = cg.random_layered(n, 6, cg.SplitMix64(cg.seed_of(0, 901)), n_swaps=2)
    check(n, gates, qs.QS_C64, opts(14, 3))
    check(n, gates, qs.QS_C128, opts(13, 3))


def test_controls_and_phases_outside_the_tile():
    # high-qubit controls (CX, CCX, CU3, CSWAP targets low) and diagonal
    # gates on qubits no tile holds: they must act per tile, not be dropped
    n = 16
    rng = np.random.default_rng(3)
    gates = []
    for layer in range(6):
        for q in range(4):
            gates.append(("u3", [q], [float(x) for x in rng.uniform(0, 2 * np.pi, 3)]))
        hi = [int(x) for x in rng.choice(np.arange(9, 16), 4, replace=False)]
        gates += [("cx", [hi[0], layer % 4], []), ("ccx", [hi[1], hi[2], (layer + 1) % 4], []),
                  ("cu3", [hi[3], (layer + 2) % 4], [0.3, 1.1, -0.4]),
                  ("cswap", [hi[0], 1, 2], []),
                  ("rz", [hi[1]], [0.7]), ("rzz", [hi[2], hi[3]], [1.3]), ("cp", [hi[0], 3], [0.9]),
                  ("crz", [hi[3], 0], [-0.6]), ("t", [hi[2]], []), ("cz", [hi[1], hi[0]], [])]
    init = random_state(n, cg.seed_of(0, 902))
    for dtype in (qs.QS_C64, qs.QS_C128):
        check(n, gates, dtype, opts(8, 2), init=init)


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_qft_closed_form(dtype):
    n = 18
    gates, x = cg.qft(n, rng=cg.SplitMix64(cg.seed_of(1, 5)))
    got, perm, recs = run(n, gates, TILE, dtype, opts(10, 3))
    assert any(r.kind == 3 for r in recs)
    ys = np.arange(1 << n, dtype=np.int64)
    phys = np.zeros_like(ys)
    for l in range(n):
        phys |= ((ys >> l) & 1) << int(perm[l])
    want = np.exp(2j * np.pi * ((x * ys) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)
    err = np.linalg.norm(got[phys] - want)
    assert err <= TOL[dtype] * 4, err


def test_ghz_and_tile_flag_ignored_when_state_fits_one_tile():
    for n in (13, 20):
        got, perm, recs = run(n, cg.ghz(n), TILE, qs.QS_C64, opts())
        assert (any(r.kind == 3 for r in recs)) == (n > 13)
        assert abs(got[0] - 1 / math.sqrt(2)) < 1e-6 and abs(got[(1 << n) - 1] - 1 / math.sqrt(2)) < 1e-6
    check(12, cg.random_layered(12, 5, cg.SplitMix64(cg.seed_of(0, 903))), qs.QS_C64, opts(), want_tiles=False)


def test_tiles_with_fold_relocation_and_fusion_flags():
    n = 17
    gates = cg.random_layered(n, 10, cg.SplitMix64(cg.seed_of(0, 904)), n_swaps=5)
    for extra in (qs.QS_FOLD, qs.QS_RELOCATE, qs.QS_FUSE | qs.QS_FUSE_K(5) | qs.QS_DIAG | qs.QS_TC):
        want, operm = oracle.simulate(cg.to_qasm(n, gates))
        got, perm, _ = run(n, gates, TILE | extra, qs.QS_C64, opts(9, 3))
        assert np.linalg.norm(got - oracle.to_physical(want, perm)) <= 1e-5


def test_bench_size_n30_tiles_times_inverse():
    from tests.test_oracle_pins import _inverse
    n = 30
    _, gates = cg.benchmark_circuits(n=n)["random"]
    st = qs.qs_alloc_state(n, qs.QS_C64)
    try:
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), TILE)
        _, recs = qs.qs_profile(st)
        assert sum(r.kind == 3 for r in recs) >= 10
        assert abs(qs.qs_norm(st) - 1) < 1e-5
        qs.qs_apply_circuit(st, qs.gates_to_array(_inverse(gates)), TILE)
        p = qs.qs_measure_probs(st, list(range(12)))
        assert p[0] > (1 - 1e-5) ** 2
    finally:
        qs.qs_free_state(st)
