"""Batched persistent launch (many circuits of uneven width, one kernel,
replayed as a CUDA graph) against the FP64 oracle, circuit by circuit."""

import numpy as np
import pytest

import circuitgen as cg
import oracle
import paper_2410_09326_gb300 as qs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    return qs.load(build_if_missing=True)


def make_batch_inputs():
    circuits = cg.qaoa_batch(count=18, index=7)
    rng = cg.SplitMix64(4040)
    for n in (8, 13, 15, 17):  # random circuits with SWAPs: virtual swap inside the batch
        circuits.append((n, cg.random_layered(n, 6, rng, n_swaps=5)))
    circuits.append((3, cg.all_gate_types_circuit(3, 40, rng)))
    return circuits


@pytest.mark.parametrize("flags", [qs.QS_VSWAP | qs.QS_DIAG, qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(5) | qs.QS_DIAG,
                                   qs.QS_FUSE | qs.QS_FUSE_K(1)])
def test_batch_matches_oracle_and_replays(flags):
    circuits = make_batch_inputs()
    states = [qs.qs_alloc_state(n, qs.QS_C64) for n, _ in circuits]
    arrays = [qs.gates_to_array(g) for _, g in circuits]
    b = qs.qs_batch_create(states, arrays, flags)
    try:
        info = qs.qs_batch_info(b)
        assert info.count == len(circuits) and info.graph == 1
        if not flags & qs.QS_FUSE:
            assert info.n_tuned == 9 and info.fuse_k in (2, 3, 4)
        first = []
        for rep in range(2):
            # scribble over the states: every run must start from |0...0>
            for (n, _), st in zip(circuits, states):
                qs.qs_set_basis(st, (1 << n) - 1)
            qs.qs_batch_run(b)
            qs.qs_batch_sync(b)
            for i, ((n, gates), st) in enumerate(zip(circuits, states)):
                got = qs.qs_read_state(st, n, qs.QS_C64).astype(np.complex128)
                perm = qs.qs_get_perm(st, n)
                want, operm = oracle.simulate(cg.to_qasm(n, gates))
                if flags & qs.QS_VSWAP:
                    assert list(perm) == list(operm)
                err = np.linalg.norm(got - oracle.to_physical(want, perm))
                assert err < 1e-5, (i, n, err)
                if rep == 0:
                    first.append(got)
                else:
                    assert np.array_equal(got, first[i])  # graph replay is deterministic
    finally:
        qs.qs_batch_free(b)
        for st in states:
            qs.qs_free_state(st)


def test_batch_rejects_bad_inputs():
    st = qs.qs_alloc_state(4, qs.QS_C128)
    try:
        with pytest.raises(qs.QsError) as e:
            qs.qs_batch_create([st], [qs.gates_to_array([("h", [0])])])
        assert e.value.status == qs.QS_EUNSUPPORTED
    finally:
        qs.qs_free_state(st)
    st = qs.qs_alloc_state(4, qs.QS_C64)
    try:
        with pytest.raises(qs.QsError) as e:
            qs.qs_batch_create([st, st], [qs.gates_to_array([("h", [0])])] * 2)
        assert e.value.status == qs.QS_EINVAL
    finally:
        qs.qs_free_state(st)


def test_one_shot_apply_batch():
    """qs_apply_batch: create, one run, sync and free in one call; every state
    ends at its own circuit's result from |0...0>."""
    circuits = make_batch_inputs()[:10]
    states = [qs.qs_alloc_state(n, qs.QS_C64) for n, _ in circuits]
    try:
        for (n, _), st in zip(circuits, states):
            qs.qs_set_basis(st, 1)
        qs.qs_apply_batch(states, [qs.gates_to_array(g) for _, g in circuits], qs.QS_VSWAP | qs.QS_DIAG)
        for (n, gates), st in zip(circuits, states):
            want, operm = oracle.simulate(cg.to_qasm(n, gates))
            perm = qs.qs_get_perm(st, n)
            assert list(perm) == list(operm)
            got = qs.qs_read_state(st, n, qs.QS_C64).astype(np.complex128)
            assert np.linalg.norm(got - oracle.to_physical(want, perm)) < 1e-5
        with pytest.raises(qs.QsError) as e:
            qs.qs_apply_batch([states[0], states[0]], [qs.gates_to_array([("h", [0])])] * 2)
        assert e.value.status == qs.QS_EINVAL
    finally:
        for st in states:
            qs.qs_free_state(st)
