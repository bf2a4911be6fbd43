"""Rotation folding (Sec. III-D) on the host: exactness against the oracle,
the paper's worked example, and the T-ratio activation rule."""

import os

import numpy as np
import pytest

import circuitgen as cg
import oracle
import paper_2410_09326_gb300 as qs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rotation_folding_ham15_fragment.txt")


@pytest.fixture(scope="module", autouse=True)
def lib():
    return qs.load(build_if_missing=True)


def read_golden():
    parts, cur = {}, None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = line.strip("[]")
            parts[cur] = []
            continue
        name, qubits = line.split()
        parts[cur].append((name, [int(q) for q in qubits.split(",")]))
    return parts


def unitary_distance(n, a, b, trials=3):
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(trials):
        init = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
        init /= np.linalg.norm(init)
        sa, _ = oracle.simulate(cg.to_qasm(n, a), init=init)
        sb, _ = oracle.simulate(cg.to_qasm(n, b), init=init)
        worst = max(worst, np.linalg.norm(sa - sb))
    return worst


def test_paper_listings_are_equivalent_and_folding_reproduces_them():
    g = read_golden()
    n = 20
    assert unitary_distance(n, g["before"], g["after"], trials=1) < 1e-12
    folded = qs.array_to_gates(qs.qs_fold_rotations(n, qs.gates_to_array(g["before"])))
    assert sorted((name, tuple(q)) for name, q, _ in folded) == sorted((name, tuple(q)) for name, q in g["after"])
    assert len(folded) == 6 and len(g["before"]) == 11


@pytest.mark.parametrize("seed", range(6))
def test_folding_is_exact_on_clifford_t(seed):
    rng = cg.SplitMix64(500 + seed)
    n = 6
    names = ["t", "tdg", "s", "sdg", "z", "x", "h", "cx", "cx", "t", "swap", "rz", "u1", "cp"]
    gates = []
    for _ in range(300):
        name = names[rng.randint(len(names))]
        nq, npar = cg.GATES[name]
        qubits = rng.shuffle(list(range(n)))[:nq]
        gates.append((name, qubits, [rng.uniform(-3, 3) for _ in range(npar)]))
    folded = qs.array_to_gates(qs.qs_fold_rotations(n, qs.gates_to_array(gates)))
    assert len(folded) < len(gates)
    assert unitary_distance(n, gates, folded) < 1e-11


@pytest.mark.parametrize("seed", range(3))
def test_folding_is_exact_on_every_gate_type(seed):
    rng = cg.SplitMix64(900 + seed)
    n = 5
    gates = cg.all_gate_types_circuit(n, 250, rng)
    folded = qs.array_to_gates(qs.qs_fold_rotations(n, qs.gates_to_array(gates)))
    assert len(folded) <= len(gates) + 2
    assert unitary_distance(n, gates, folded) < 1e-11


def test_global_phase_of_rz_is_kept():
    # RZ(a) RZ(b) on the same wire merge; the folded circuit keeps the phase
    gates = [("x", [0]), ("rz", [0], [0.3]), ("cx", [0, 1]), ("cx", [0, 1]), ("rz", [0], [0.4])]
    folded = qs.array_to_gates(qs.qs_fold_rotations(2, qs.gates_to_array(gates)))
    assert unitary_distance(2, gates, folded) < 1e-12
    assert sum(1 for g in folded if g[0] == "cx") == 0


def test_t_ratio_rule_activates_folding():
    g = read_golden()
    arr = qs.gates_to_array(g["before"])
    recs, _, _ = qs.qs_plan(20, arr, qs.QS_PGO_RULES)
    # T gates are 5 of 11 (> 10%): folding ran, so fewer gates reached the blocks
    assert sum(r.n_gates for r in recs) <= 6
    recs_plain, _, _ = qs.qs_plan(20, arr, qs.QS_PLAIN)
    assert len(recs_plain) == 11
    # a circuit without T gates is not folded (the QFT of Sec. III-D is the paper's counterexample)
    gates, _ = cg.qft(6, x=3)
    arr = qs.gates_to_array(gates)
    f_rules = qs.qs_plan(6, arr, qs.QS_PGO_RULES)[0]
    assert sum(r.n_gates for r in f_rules) == len(gates) - 3  # only the 3 SWAPs left the list (virtual swap)
