"""Learned cost model: GPU forward/backward against the FP64 network
reference, training, and what the trained network gains in pass selection."""

import math

import numpy as np
import pytest

import circuitgen as cg
import paper_2410_09326_gb300 as qs
from oracle import mlp as ref
from paper_2410_09326_gb300 import costmodel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    return qs.load(build_if_missing=True)


@pytest.mark.parametrize("seed", [1, 2])
def test_gradient_matches_fp64_reference(seed):
    m = qs.qs_mlp_create(seed)
    try:
        rng = np.random.default_rng(seed)
        p = qs.qs_mlp_params(m)
        for trial in range(2):
            x = rng.normal(size=(300, qs.QS_MLP_FEATURES)).astype(np.float32)
            y = rng.normal(size=300).astype(np.float32)
            g, loss = qs.qs_mlp_gradient(m, x, y)
            g_ref = ref.gradient(p.astype(np.float64), x.astype(np.float64), y.astype(np.float64))
            l_ref = ref.loss(p.astype(np.float64), x.astype(np.float64), y.astype(np.float64))
            rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
            assert rel < 1e-4, rel
            assert abs(loss - l_ref) <= 1e-5 * l_ref
            # parameters written through the ABI are the ones used
            p = (p * 0.7 + rng.normal(scale=0.05, size=p.size)).astype(np.float32)
            qs.qs_mlp_params(m, p)
    finally:
        qs.qs_mlp_free(m)


def test_training_fits_a_known_function():
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, size=(4096, qs.QS_MLP_FEATURES)).astype(np.float32)
    y = (np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2] + 0.5 * np.abs(x[:, 3])).astype(np.float32)
    m = qs.qs_mlp_create(3)
    try:
        before = np.mean((qs.qs_mlp_predict(m, x) - y) ** 2)
        qs.qs_mlp_train(m, x, y, epochs=60, batch=256, lr=3e-3, seed=1)
        after = np.mean((qs.qs_mlp_predict(m, x) - y) ** 2)
        assert after < 0.05 * before and after < 0.02, (before, after)
    finally:
        qs.qs_mlp_free(m)


def low_heavy(n, layers, rng):
    """Layers of U3 on qubits 0..5, a CX chain among them and one CX from a
    low qubit to a random high one: nearly every gate on the lowest bits."""
    g = []
    for _ in range(layers):
        g += [("u3", [q], [rng.uniform(0, 6.28) for _ in range(3)]) for q in range(6)]
        g += [("cx", [q, q + 1]) for q in range(5)]
        g.append(("cx", [rng.randint(6), 6 + rng.randint(n - 6)]))
    return g


def ctrl_heavy(n, layers, rng):
    """Layers of RY on every qubit and n/3 CCX / CSWAP / CU3 on random qubits."""
    g = []
    for _ in range(layers):
        g += [("ry", [q], [rng.uniform(0, 6.28)]) for q in range(n)]
        for _ in range(n // 3):
            a, b, c = rng.shuffle(list(range(n)))[:3]
            nm = ["ccx", "cswap", "cu3"][rng.randint(3)]
            g.append((nm, [a, b], [rng.uniform(0, 6.28) for _ in range(3)]) if nm == "cu3" else (nm, [a, b, c]))
    return g


def test_learned_selection_gains_over_the_priors():
    """What the trained network gains over the selector without it (the
    compiled-in per-class priors, Sec. III-A's open profile-to-flags mapping).
    Train on profiled blocks of seeded layered-random, QFT, GHZ and QAOA
    circuits (n = 18..26), then pick flags for circuit families it has not
    seen -- low-target-heavy layers, controlled-gate-heavy layers, a random
    circuit and QAOA, n = 24..26 -- without running them, against brute force
    over the 12 candidate flag sets measured on this GPU. The priors charge
    a tile pass a fixed fraction of HBM bandwidth whatever its gate count and
    so choose tile passes for the low-target-heavy circuits (measured 2-3x
    slower than the best); the network, which sees the gate count, does not.
    Asserted: the network's mean regret is below the priors' by at least
    0.15, its worst regret within 25% of brute force, and its predictions of
    the candidates' device times are closer to the measured ones."""
    train = costmodel.training_circuits(40, n_lo=18, n_hi=26, index0=100)
    x, y = costmodel.build_dataset(train)
    assert len(y) > 20000
    m = qs.qs_mlp_create(11)
    try:
        qs.qs_mlp_train(m, x, y, epochs=40, batch=256, lr=2e-3, seed=2)
        rng = cg.SplitMix64(777)
        held = {}
        for n in (24, 25, 26):
            held[f"low_heavy_n{n}"] = (n, low_heavy(n, 40, rng))
        held["ctrl_heavy_n24"] = (24, ctrl_heavy(24, 6, rng))
        held["random_n25"] = (25, cg.random_layered(25, 20, rng, swap_frac=0.05))
        held["qaoa_n24"] = (24, cg.qaoa_maxcut(24, 3, rng)[0])
        held["qaoa_n26"] = (26, cg.qaoa_maxcut(26, 3, rng)[0])
        cands = [qs.QS_PLAIN, qs.QS_VSWAP] + \
                [qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_DIAG for k in range(1, 7)] + \
                [qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_DIAG | qs.QS_TC for k in (4, 5, 6)] + \
                [qs.QS_VSWAP | qs.QS_TILE]
        report = {}
        for name, (n, gates) in held.items():
            arr = qs.gates_to_array(gates)
            meas = costmodel.measure_candidates(n, gates, cands, repeats=2)
            best = min(meas.values())

            def regret(f):
                t = meas.get(f)
                if t is None:
                    t = costmodel.measure_candidates(n, gates, [f])[f]
                return t / best

            err_mlp = np.mean([abs(math.log(costmodel.mlp_plan_ms(m, n, gates, f) / meas[f])) for f in cands])
            err_pri = np.mean([abs(math.log(qs.qs_pgo_predict(n, arr, f) / meas[f])) for f in cands])
            report[name] = {"mlp": regret(qs.qs_pgo_select_mlp(m, n, arr)[0]),
                            "priors": regret(qs.qs_pgo_select(n, arr)[0]),
                            "plan_log_err_mlp": float(err_mlp), "plan_log_err_priors": float(err_pri)}
        print(report)
        r_mlp = [r["mlp"] for r in report.values()]
        r_pri = [r["priors"] for r in report.values()]
        assert np.mean(r_mlp) <= np.mean(r_pri) - 0.15, report
        assert max(r_mlp) <= 1.25, report
        assert np.mean([r["plan_log_err_mlp"] for r in report.values()]) < \
            np.mean([r["plan_log_err_priors"] for r in report.values()]), report
    finally:
        qs.qs_mlp_free(m)
