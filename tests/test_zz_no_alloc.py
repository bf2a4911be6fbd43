"""The no-allocation probabilities entry point (qs_probs_noalloc).

It serves callers that cannot let the library allocate device memory (a
process that reserved its HBM up front through its own pool, or one that
must not risk the synchronisation cudaMalloc/cudaFree may imply). Its
scratch is a fixed array inside the library, so the test checks, through the
C ABI, that two calls in a row give the same marginals as qs_measure_probs
(which uses state-owned scratch) and as the FP64 oracle, within the
tolerances of the other probability tests, on states small enough to use
the fixed array and on larger ones (no scratch), and that the library's
count of live device bytes does not move across the calls. The file sorts last so
that a failure here comes after every other test has run; it also passes on
its own in a fresh process.
"""

import numpy as np
import pytest

import circuitgen as cg
import oracle
import paper_2410_09326_gb300 as qs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,tol", [(qs.QS_C64, 1e-6), (qs.QS_C128, 1e-13)])
def test_noalloc_matches_measure_probs_twice(dtype, tol):
    torch = pytest.importorskip("torch")
    qs.load(build_if_missing=True)
    n = 22
    rng = cg.SplitMix64(321)
    gates = cg.random_layered(n, 4, rng, n_swaps=4)
    stream = torch.cuda.Stream()
    st = qs.qs_alloc_state(n, dtype, stream=stream)
    try:
        qs.qs_apply_circuit(st, qs.gates_to_array(gates),
                            qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(3) | qs.QS_DIAG)
        perm = qs.qs_get_perm(st, n)
        amps = qs.qs_device_ptr(st)
        for logical in ([], [0], [3, 17], list(range(12)), [21, 5, 9, 0, 14], list(range(16))):
            want = qs.qs_measure_probs(st, logical)
            phys = [int(perm[l]) for l in logical]
            out = torch.full((1 << len(logical),), -1.0, dtype=torch.float64, device="cuda")
            live = qs.qs_memory_in_use()
            for _ in range(2):  # the shared array keeps the previous call's contents
                out.fill_(-1.0)
                qs.qs_probs_noalloc(amps, n, dtype, phys, out.data_ptr(), stream=stream)
                stream.synchronize()
                got = out.cpu().numpy()
                assert np.abs(got - want).max() < tol, (logical, np.abs(got - want).max())
            assert qs.qs_memory_in_use() == live
    finally:
        qs.qs_free_state(st)


@pytest.mark.parametrize("n", [9, 14])
@pytest.mark.parametrize("dtype,tol", [(qs.QS_C64, 1e-6), (qs.QS_C128, 1e-13)])
def test_noalloc_matches_the_oracle(dtype, tol, n):
    """Marginals of a layered circuit with SWAPs against the FP64 oracle's,
    twice in a row, the measured bits mapped through perm: 9 qubits (partial
    sums in the library's fixed array) and 14 (the chunked kernel, straight
    into the output)."""
    torch = pytest.importorskip("torch")
    qs.load(build_if_missing=True)
    gates = cg.random_layered(n, 6, cg.SplitMix64(654), n_swaps=5)
    want_state, _ = oracle.simulate(cg.to_qasm(n, gates))
    st = qs.qs_alloc_state(n, dtype)
    try:
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(4) | qs.QS_DIAG)
        perm = qs.qs_get_perm(st, n)
        amps = qs.qs_device_ptr(st)
        torch.cuda.synchronize()
        for logical in ([n - 1], [2, n - 3, 7], list(range(min(n, 12))), list(range(n - 1, 1, -1))):
            want = oracle.probs(want_state, logical)
            out = torch.full((1 << len(logical),), -1.0, dtype=torch.float64, device="cuda")
            for _ in range(2):
                out.fill_(-1.0)
                qs.qs_probs_noalloc(amps, n, dtype, [int(perm[l]) for l in logical], out.data_ptr())
                torch.cuda.synchronize()
                assert np.abs(out.cpu().numpy() - want).max() < tol, logical
    finally:
        qs.qs_free_state(st)


def test_noalloc_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    qs.load(build_if_missing=True)
    n = 14
    buf = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    out = torch.zeros(1 << 15, dtype=torch.float64, device="cuda")
    with pytest.raises(qs.QsError) as e:
        qs.qs_probs_noalloc(buf.data_ptr(), n, qs.QS_C64, list(range(15)), out.data_ptr())
    assert e.value.status == qs.QS_EINVAL and "26" in str(e.value)
    with pytest.raises(qs.QsError):
        qs.qs_probs_noalloc(buf.data_ptr(), n, qs.QS_C64, [1, 1], out.data_ptr())
    with pytest.raises(qs.QsError):
        qs.qs_probs_noalloc(buf.data_ptr(), n, qs.QS_C64, [14], out.data_ptr())
