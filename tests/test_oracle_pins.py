"""Pins of the FP64 oracle to facts outside itself (CPU only).

Every check here compares the oracle with something the mathematics fixes:
textbook gate identities, closed-form states (GHZ, QFT of basis states),
invariants (norm, circuit x inverse = |0...0>), and brute force on tiny
inputs (an einsum contraction written independently of the oracle's index
loops). A dropped term, a wrong sign, a swapped index or a transposed
operand in the oracle fails at least one of them.
"""

import math

import numpy as np
import pytest

import circuitgen as cg
import oracle

I2 = np.eye(2)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.diag([1, -1]).astype(complex)
H = np.array([[1, 1], [1, -1]], dtype=complex) / math.sqrt(2)


def U(name, *p):
    return oracle.gate_matrix(name, p)[0]


# ---------------------------------------------------------------------------
# Gate table (the paper names the gates, Sec. III-C; matrices follow qelib1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", sorted(cg.GATES))
def test_every_gate_unitary(name):
    rng = cg.SplitMix64(7)
    p = [rng.uniform(-7, 7) for _ in range(cg.GATES[name][1])]
    u, nc, nt = oracle.gate_matrix(name, p)
    assert nc + nt == cg.GATES[name][0]
    assert np.allclose(u.conj().T @ u, np.eye(u.shape[0]), atol=1e-15)


def test_pauli_and_clifford_identities():
    assert np.allclose(U("x"), X) and np.allclose(U("y"), Y) and np.allclose(U("z"), Z)
    assert np.allclose(U("h"), H)
    assert np.allclose(U("h") @ U("x") @ U("h"), U("z"))
    assert np.allclose(U("y"), 1j * U("x") @ U("z"))
    assert np.allclose(U("s") @ U("s"), U("z"))
    assert np.allclose(U("t") @ U("t"), U("s"))
    assert np.allclose(U("sdg"), U("s").conj().T)
    assert np.allclose(U("tdg"), U("t").conj().T)
    assert np.allclose(U("sx") @ U("sx"), U("x"))
    assert np.allclose(U("sxdg"), U("sx").conj().T)
    assert np.allclose(U("id"), I2)


def test_rotation_closed_forms():
    th = 0.7321
    c, s = math.cos(th / 2), math.sin(th / 2)
    # RY(theta)|0> = cos|0> + sin|1>  (a transposed RY would give -sin)
    assert np.allclose(U("ry", th) @ [1, 0], [c, s])
    # RX(theta)|0> = cos|0> - i sin|1>
    assert np.allclose(U("rx", th) @ [1, 0], [c, -1j * s])
    # RZ(theta) = diag(e^{-i theta/2}, e^{i theta/2})
    assert np.allclose(U("rz", th), np.diag([np.exp(-0.5j * th), np.exp(0.5j * th)]))
    assert np.allclose(U("rz", 0.3) @ U("rz", 0.4), U("rz", 0.7))
    assert np.allclose(U("rx", math.pi), -1j * X)
    assert np.allclose(U("ry", math.pi), -1j * Y)
    assert np.allclose(U("u1", th), np.exp(0.5j * th) * U("rz", th))


def test_u3_reductions():
    th, ph, la = 0.4, 1.3, -2.2
    assert np.allclose(U("u3", th, 0, 0), U("ry", th))
    assert np.allclose(U("u3", th, -math.pi / 2, math.pi / 2), U("rx", th))
    assert np.allclose(U("u3", 0, 0, la), U("u1", la))
    assert np.allclose(U("u2", ph, la), U("u3", math.pi / 2, ph, la))
    # U3 = e^{i(ph+la)/2} RZ(ph) RY(th) RZ(la)  (Z-Y decomposition, Sec. III-D)
    zyz = np.exp(0.5j * (ph + la)) * U("rz", ph) @ U("ry", th) @ U("rz", la)
    assert np.allclose(U("u3", th, ph, la), zyz)


def test_two_qubit_targets():
    th = 1.234
    # local index l = bit(t0) + 2 bit(t1); kron(A on t1, B on t0)
    zz = np.kron(Z, Z)
    xx = np.kron(X, X)
    yy = np.kron(Y, Y)
    expm = lambda m: math.cos(th / 2) * np.eye(4) - 1j * math.sin(th / 2) * m
    assert np.allclose(U("rzz", th), expm(zz))
    assert np.allclose(U("rxx", th), expm(xx))
    assert np.allclose(U("ryy", th), expm(yy))
    sw = U("swap")
    for a in range(2):
        for b in range(2):
            v = np.zeros(4)
            v[a + 2 * b] = 1
            assert np.allclose(sw @ v, np.eye(4)[b + 2 * a])


def test_controlled_bases():
    for cname, base, p in [("cx", "x", ()), ("cy", "y", ()), ("cz", "z", ()), ("ch", "h", ()),
                           ("crx", "rx", (0.3,)), ("cry", "ry", (0.3,)), ("crz", "rz", (0.3,)),
                           ("cp", "u1", (0.3,)), ("cu1", "u1", (0.3,)), ("cu3", "u3", (0.3, 0.2, 0.1))]:
        u, nc, nt = oracle.gate_matrix(cname, p)
        assert (nc, nt) == (1, 1)
        assert np.allclose(u, U(base, *p))
    u, nc, nt = oracle.gate_matrix("ccx")
    assert (nc, nt) == (2, 1) and np.allclose(u, X)
    u, nc, nt = oracle.gate_matrix("cswap")
    assert (nc, nt) == (1, 2) and np.allclose(u, U("swap"))


# ---------------------------------------------------------------------------
# Brute force on tiny inputs: an einsum contraction, independent of oracle.c
# ---------------------------------------------------------------------------

def _full_gate(name, qubits, params):
    """Gate on (controls + targets) as a (2^k x 2^k) matrix whose local index
    is sum_j bit(qubits[j]) << j, built block-wise from the target unitary."""
    u, nc, nt = oracle.gate_matrix(name, params)
    k = nc + nt
    d = 1 << k
    m = np.zeros((d, d), dtype=complex)
    cmask = (1 << nc) - 1
    for col in range(d):
        if col & cmask != cmask:
            m[col, col] = 1.0
            continue
        tc = col >> nc
        for tr in range(1 << nt):
            m[(tr << nc) | cmask, col] = u[tr, tc]
    return m


def _einsum_apply(psi, n, name, qubits, params):
    """Contract a gate into the state viewed as an n-axis tensor.
    Axis a of reshape([2]*n) is qubit n-1-a (C order, little-endian index)."""
    m = _full_gate(name, qubits, params)
    k = len(qubits)
    t = psi.reshape([2] * n)
    # gate tensor: out bits (most significant local bit first), then in bits
    g = m.reshape([2] * (2 * k))
    # local bit j of the row index is axis k-1-j of the reshaped matrix
    in_axes = [n - 1 - qubits[j] for j in range(k)]
    g_in = [2 * k - 1 - j for j in range(k)]
    out = np.tensordot(g, t, axes=(g_in, in_axes))
    # out's first k axes are out bits for local bits k-1..0
    src = list(range(k))
    dst = [n - 1 - qubits[k - 1 - a] for a in range(k)]
    out = np.moveaxis(out, src, dst)
    return out.reshape(-1)


def _brute(n, gates, init=None):
    psi = np.zeros(1 << n, dtype=complex) if init is None else init.copy()
    if init is None:
        psi[0] = 1
    for name, qs, *rest in gates:
        psi = _einsum_apply(psi, n, name, qs, rest[0] if rest else ())
    return psi


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_all_gate_types(n, seed):
    rng = cg.SplitMix64(1000 + 17 * n + seed)
    gates = cg.all_gate_types_circuit(n, 60, rng)
    text = cg.to_qasm(n, gates)
    got, _ = oracle.simulate(text)
    want = _brute(n, gates)
    assert np.linalg.norm(got - want) < 1e-12
    init = np.array([rng.uniform(-1, 1) + 1j * rng.uniform(-1, 1) for _ in range(1 << n)])
    init /= np.linalg.norm(init)
    got, _ = oracle.simulate(text, init=init)
    assert np.linalg.norm(got - _brute(n, gates, init)) < 1e-12


def test_dense_unitary_product_n4():
    """Columns of the oracle's map equal the dense 2^n matrix product of
    kron-embedded gates (adjacent-qubit gates only, kron order explicit)."""
    n = 4
    gates = [("h", [0]), ("cx", [0, 1]), ("ry", [2], [0.3]), ("rzz", [2, 3], [0.9]),
             ("u3", [3], [0.1, 0.2, 0.3]), ("swap", [1, 2]), ("cp", [2, 3], [0.77])]

    def embed(m2, lo, width):
        # operator on qubits lo..lo+width-1; kron puts the highest qubit first
        return np.kron(np.kron(np.eye(1 << (n - lo - width)), m2), np.eye(1 << lo))

    dense = np.eye(1 << n, dtype=complex)
    for name, qs, *rest in gates:
        lo = min(qs)
        width = len(qs)
        m = _full_gate(name, qs, rest[0] if rest else ())
        if qs != list(range(lo, lo + width)):  # reorder local bits to ascending qubits
            order = np.argsort(qs)
            d = 1 << width
            p = np.zeros((d, d))
            for l in range(d):
                l2 = sum(((l >> j) & 1) << int(np.where(order == j)[0][0]) for j in range(width))
                p[l2, l] = 1
            m = p @ m @ p.T
        dense = embed(m, lo, width) @ dense
    text = cg.to_qasm(n, gates)
    for col in range(1 << n):
        init = np.zeros(1 << n, dtype=complex)
        init[col] = 1
        got, _ = oracle.simulate(text, init=init)
        assert np.allclose(got, dense[:, col], atol=1e-13)


# ---------------------------------------------------------------------------
# Closed-form whole states
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 7, 12])
def test_ghz_closed_form(n):
    psi, perm = oracle.simulate(cg.to_qasm(n, cg.ghz(n)))
    want = np.zeros(1 << n, dtype=complex)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert np.linalg.norm(psi - want) < 1e-14
    assert list(perm) == list(range(n))


def qft_closed_form(n, x):
    y = np.arange(1 << n)
    return np.exp(2j * np.pi * x * y / (1 << n)) / math.sqrt(1 << n)


def bit_reverse(v, n):
    return int(format(v, f"0{n}b")[::-1], 2)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8])
def test_qft_of_basis_states(n):
    xs = range(1 << n) if n <= 4 else [0, 1, 5, (1 << n) - 1, 37 % (1 << n)]
    for x in xs:
        gates, _ = cg.qft(n, x=x, swaps=True)
        psi, perm = oracle.simulate(cg.to_qasm(n, gates))
        assert np.linalg.norm(psi - qft_closed_form(n, x)) < 1e-12
        # the swap network as a relabelling is the bit reversal
        assert list(perm) == [n - 1 - q for q in range(n)]
        # without the swaps the output comes out bit-reversed
        gates, _ = cg.qft(n, x=x, swaps=False)
        psi2, _ = oracle.simulate(cg.to_qasm(n, gates))
        rev = np.array([bit_reverse(i, n) for i in range(1 << n)])
        assert np.linalg.norm(psi2[rev] - qft_closed_form(n, x)) < 1e-12


def _inverse(gates):
    inv = {"s": "sdg", "sdg": "s", "t": "tdg", "tdg": "t", "sx": "sxdg", "sxdg": "sx"}
    neg1 = {"rx", "ry", "rz", "u1", "cp", "cu1", "crx", "cry", "crz", "rzz", "rxx", "ryy"}
    out = []
    for name, qs, *rest in reversed(gates):
        p = list(rest[0]) if rest else []
        if name in inv:
            out.append((inv[name], qs, []))
        elif name in neg1:
            out.append((name, qs, [-p[0]]))
        elif name in ("u3", "cu3"):
            out.append((name, qs, [-p[0], -p[2], -p[1]]))
        elif name == "u2":
            out.append(("u3", qs, [-math.pi / 2, -p[1], -p[0]]))
        else:
            out.append((name, qs, p))
    return out


@pytest.mark.parametrize("n", [3, 6, 10])
def test_circuit_times_inverse_is_identity(n):
    rng = cg.SplitMix64(55 + n)
    gates = cg.all_gate_types_circuit(n, 200, rng)
    psi, perm = oracle.simulate(cg.to_qasm(n, gates + _inverse(gates)))
    want = np.zeros(1 << n, dtype=complex)
    want[0] = 1
    assert np.linalg.norm(psi - want) < 1e-12


@pytest.mark.parametrize("index", range(3))
def test_norm_preserved_layered_swaps(index):
    n, gates = cg.layered_swaps_circuit(index)
    psi, perm = oracle.simulate(cg.to_qasm(n, gates))
    assert abs(np.vdot(psi, psi).real - 1) < 1e-13
    assert sorted(perm) == list(range(n))


# ---------------------------------------------------------------------------
# The logical->physical map (virtual swap, Sec. III-D)
# ---------------------------------------------------------------------------

def test_perm_matches_data_that_never_moved():
    """A SWAP-only circuit on |x>: the oracle moves data, a relabelling moves
    none, so placing the oracle's state through perm gives back |x>."""
    n = 7
    rng = cg.SplitMix64(99)
    for trial in range(20):
        x = rng.randint(1 << n)
        gates = [("x", [q]) for q in range(n) if (x >> q) & 1]
        prep = len(gates)
        for _ in range(1 + rng.randint(12)):
            a, b = cg.random_pair(rng, n)
            gates.append(("swap", [a, b]))
        psi, perm = oracle.simulate(cg.to_qasm(n, gates))
        phys = oracle.to_physical(psi, perm)
        assert np.argmax(np.abs(phys)) == x and abs(abs(phys[x]) - 1) < 1e-15
        assert prep >= 0


def test_probs_marginals():
    n = 5
    psi, _ = oracle.simulate(cg.to_qasm(n, cg.ghz(n)))
    assert np.allclose(oracle.probs(psi, [0]), [0.5, 0.5])
    assert np.allclose(oracle.probs(psi, [0, 3]), [0.5, 0, 0, 0.5])
    assert np.allclose(oracle.probs(psi, list(range(n))), np.abs(psi) ** 2)
    # product state: marginal of RY(th)|0> on q2 is (cos^2, sin^2)
    th = 0.9
    psi, _ = oracle.simulate(cg.to_qasm(n, [("ry", [2], [th]), ("h", [4])]))
    assert np.allclose(oracle.probs(psi, [2]), [math.cos(th / 2) ** 2, math.sin(th / 2) ** 2])
    assert np.allclose(oracle.probs(psi, [4, 2]), np.outer([math.cos(th / 2) ** 2, math.sin(th / 2) ** 2], [0.5, 0.5]).reshape(-1))


def test_parser_rejects_bad_input():
    for bad in ["qreg q[2];\nh q[2];\n", "qreg q[2];\ncx q[0],q[0];\n", "qreg q[2];\nrz q[0];\n",
                "qreg q[2];\nfoo q[0];\n", "h q[0];\n", "qreg q[2];\nh q[0]\n"]:
        with pytest.raises(ValueError):
            oracle.simulate(bad)


# ---------------------------------------------------------------------------
# Cost-model network reference (oracle/mlp.py)
# ---------------------------------------------------------------------------

def test_mlp_gradient_matches_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(3)
    p = rng.normal(scale=0.3, size=mlp.N_PARAMS)
    x = rng.normal(size=(7, mlp.F))
    t = rng.normal(size=7)
    g = mlp.gradient(p, x, t)
    h = 1e-6
    for i in list(range(0, mlp.N_PARAMS, 97)) + [mlp.N_PARAMS - 1, mlp.N_PARAMS - 2]:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, x, t) - mlp.loss(p - e, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_mlp_linear_regime_closed_form():
    """With every pre-activation positive the network is one affine map."""
    from oracle import mlp
    rng = np.random.default_rng(4)
    w = {"W1": rng.uniform(0.1, 1, (mlp.H, mlp.F)), "b1": rng.uniform(0.1, 1, mlp.H),
         "W2": rng.uniform(0.1, 1, (mlp.H, mlp.H)), "b2": rng.uniform(0.1, 1, mlp.H),
         "w3": rng.normal(size=mlp.H), "b3": np.array([0.5])}
    x = rng.uniform(0, 1, (5, mlp.F))
    y, _ = mlp.forward(mlp.pack(w), x)
    want = ((x @ w["W1"].T + w["b1"]) @ w["W2"].T + w["b2"]) @ w["w3"] + 0.5
    assert np.allclose(y, want, rtol=1e-13)
    assert mlp.N_PARAMS == 64 * 24 + 64 + 64 * 64 + 64 + 64 + 1


def test_thread_count_applies_to_one_call_only():
    """A thread count passed to one oracle call does not change the next
    call's default (the OpenMP setting is restored), and the result does not
    depend on the thread count."""
    before = oracle.max_threads()
    n, gates = cg.layered_swaps_circuit(3)
    text = cg.to_qasm(n, gates)
    one, perm1 = oracle.simulate(text, nthreads=1)
    assert oracle.max_threads() == before
    many, perm2 = oracle.simulate(text)
    assert np.array_equal(perm1, perm2)
    assert np.abs(one - many).max() < 1e-13


def test_oracle_timing_helper_extrapolates_by_gate_count():
    """The benchmark's oracle timing helper: a short circuit is timed whole,
    a longer one on its first gates (at least three) and extrapolated by
    gate count."""
    import bench
    n, gates = cg.layered_swaps_circuit(0)
    text = cg.to_qasm(n, gates)
    secs, timed, total, extrapolated = bench.time_oracle_sampled(text, 1, 1e-3)
    assert total == len(gates) and 3 <= timed <= total and secs > 0
    assert extrapolated == (timed < total)
    secs, timed, total, extrapolated = bench.time_oracle_sampled(text, 1, 1e3)
    assert timed == total and not extrapolated
