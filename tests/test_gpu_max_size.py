"""The largest states the library accepts: n = 34 complex64 and n = 33
complex128 (128 GiB each), planned by the rule activator (virtual swap,
5-qubit tensor-core fusion, phase polynomials). The oracle cannot hold these
states, so the checks are closed forms at sampled indices and properties that
hold at any size: GHZ marginals, QFT of a basis state (modulus 2^(-n/2) and
phase exp(2 pi i x y / 2^n)), the norm."""

import math

import numpy as np
import pytest

import circuitgen as cg
import paper_2410_09326_gb300 as qs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    return qs.load(build_if_missing=True)


def ghz_marginals(n, dtype):
    st = qs.qs_alloc_state(n, dtype)
    try:
        qs.qs_apply_circuit(st, qs.gates_to_array(cg.ghz(n)), qs.QS_PGO_RULES)
        p = qs.qs_measure_probs(st, [0, n // 2, n - 1])
        assert abs(p[0] - 0.5) < 1e-5 and abs(p[7] - 0.5) < 1e-5
        assert p[1:7].sum() < 1e-10
        assert abs(qs.qs_norm(st) - 1) < 1e-5
    finally:
        qs.qs_free_state(st)


def test_ghz_n34_c64():
    ghz_marginals(34, qs.QS_C64)


def test_ghz_n33_c128():
    ghz_marginals(33, qs.QS_C128)


def test_qft_n34_c64_sampled_closed_form():
    torch = pytest.importorskip("torch")
    n = 34
    gates, x = cg.qft(n, rng=cg.SplitMix64(cg.seed_of(1, 34)))
    buf = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    st = qs.qs_attach_state(buf.data_ptr(), n, qs.QS_C64)
    try:
        qs.qs_set_basis(st, 0)
        qs.qs_apply_circuit(st, qs.gates_to_array(gates), qs.QS_PGO_RULES)
        _, recs = qs.qs_profile(st)
        assert any(r.kind == 4 for r in recs)  # the controlled-phase ladders ran as phase polynomials
        perm = qs.qs_get_perm(st, n)
        norm = qs.qs_norm(st)
    finally:
        qs.qs_free_state(st)
    rng = cg.SplitMix64(3434)
    ys = np.array([rng.next() & ((1 << n) - 1) for _ in range(8192)] + [0, (1 << n) - 1], dtype=np.int64)
    phys = np.zeros_like(ys)
    for l in range(n):
        phys |= ((ys >> l) & 1) << int(perm[l])
    got = buf[torch.from_numpy(phys).cuda()].cpu().numpy().astype(np.complex128)
    del buf
    torch.cuda.empty_cache()
    # x * y mod 2^n without overflow: split y into 17-bit halves
    lo, hi = ys & ((1 << 17) - 1), ys >> 17
    xy = ((x * lo) % (1 << n) + ((x * hi) % (1 << (n - 17))) * (1 << 17)) % (1 << n)
    want = np.exp(2j * np.pi * (xy / float(1 << n))) / math.sqrt(float(1 << n))
    scale = math.sqrt(float(1 << n))
    assert np.abs(got - want).max() * scale < 1e-3
    assert abs(norm - 1) < 1e-5
