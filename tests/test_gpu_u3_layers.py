"""U3 + CX/CZ layers (the n=32 tensor-core workload) at oracle-sized n, and
the device-side distance used to validate the n=32 run against FP64."""

import numpy as np
import pytest

import circuitgen as cg
import oracle
import paper_2410_09326_gb300 as qs

pytestmark = pytest.mark.gpu

V = qs.QS_VSWAP | qs.QS_FUSE | qs.QS_DIAG
VARIANTS = {"cuda_k4": V | qs.QS_FUSE_K(4), "cuda_k5": V | qs.QS_FUSE_K(5), "cuda_k6": V | qs.QS_FUSE_K(6),
            "tc_k4": V | qs.QS_FUSE_K(4) | qs.QS_TC, "tc_k5": V | qs.QS_FUSE_K(5) | qs.QS_TC}


@pytest.fixture(scope="module", autouse=True)
def lib():
    return qs.load(build_if_missing=True)


@pytest.fixture(scope="module")
def u3_layers_n20():
    n, gates = cg.u3_entangler_circuit(n=20, layers=40)
    want, _ = oracle.simulate(cg.to_qasm(n, gates))
    return n, gates, want


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_u3_layers_n20_vs_oracle(name, u3_layers_n20):
    n, gates, want = u3_layers_n20
    st = qs.qs_alloc_state(n, qs.QS_C64)
    try:
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), VARIANTS[name] | qs.QS_PROFILE)
        summ, recs = qs.qs_profile(st)
        if "tc" in name:
            assert any(r.tc for r in recs)
        got = qs.qs_read_state(st, n, qs.QS_C64, logical_order=True).astype(np.complex128)
        err = np.linalg.norm(got - want)
        assert err < 1e-5, (name, err)
    finally:
        qs.qs_free_state(st)


def test_state_distance_matches_host():
    n = 14
    rng = cg.SplitMix64(21)
    gates = cg.random_layered(n, 8, rng, n_swaps=7)
    arr = qs.gates_to_array(gates)
    a = qs.qs_alloc_state(n, qs.QS_C64)
    b = qs.qs_alloc_state(n, qs.QS_C128)
    try:
        qs.qs_apply_circuit(a, arr, qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(4) | qs.QS_TC)
        qs.qs_apply_circuit(b, arr, qs.QS_PLAIN)
        d = qs.qs_state_distance(a, b)  # different maps: both go to logical order
        ha = qs.qs_read_state(a, n, qs.QS_C64).astype(np.complex128)
        hb = qs.qs_read_state(b, n, qs.QS_C128)
        assert list(qs.qs_get_perm(a, n)) == list(range(n))
        assert abs(d - np.linalg.norm(ha - hb)) < 1e-12
        assert 0 < d < 1e-5
        want, _ = oracle.simulate(cg.to_qasm(n, gates))
        assert np.linalg.norm(hb - want) < 1e-12
    finally:
        qs.qs_free_state(a)
        qs.qs_free_state(b)
