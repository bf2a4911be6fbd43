"""Seeded synthetic circuit generators (OpenQASM-2 text).

This module is the one piece of code that both the FP64 oracle and the GPU
path consume: it only draws random numbers and prints gate lines. It contains
none of the simulation arithmetic (no matrices, no amplitudes, no fusion).

The paper's benchmark circuits (QCOR suite, Sec. IV, Table "tab:allonresult")
are not available, so seeded stand-ins with the same shapes are used:
GHZ, QFT of a basis state with its final SWAP network (Sec. IV-C, Table
"tab:virtual swap number"), layered random circuits, and QAOA Max-Cut
ansaetze on random 3-regular graphs (Sec. IV-E, Table "tab:large scale").

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds. Uniform doubles take the top 53 bits.

Text format (a subset of OpenQASM 2.0, one gate per line):
    OPENQASM 2.0;
    qreg q[N];
    name(p0,p1,p2) q[a],q[b];
Controls are listed first, then targets. Angles are printed with 17
significant digits, so every parser reads back the exact double.
"""

import math

MASK64 = (1 << 64) - 1

# Gate names understood by both consumers, with (n_qubits, n_params).
GATES = {
    "h": (1, 0), "s": (1, 0), "t": (1, 0), "x": (1, 0), "y": (1, 0),
    "z": (1, 0), "sdg": (1, 0), "tdg": (1, 0), "rx": (1, 1), "ry": (1, 1),
    "rz": (1, 1), "cp": (2, 1), "cu1": (2, 1), "swap": (2, 0), "cx": (2, 0),
    "cz": (2, 0), "cy": (2, 0), "ch": (2, 0), "crx": (2, 1), "cry": (2, 1),
    "crz": (2, 1), "u1": (1, 1), "u2": (1, 2), "u3": (1, 3), "sx": (1, 0),
    "sxdg": (1, 0), "id": (1, 0), "rzz": (2, 1), "rxx": (2, 1),
    "ryy": (2, 1), "ccx": (3, 0), "cswap": (3, 0), "cu3": (2, 3),
}


class SplitMix64:
    """SplitMix64 stream; `next()` returns a 64-bit unsigned integer."""

    def __init__(self, seed):
        self.state = seed & MASK64

    def next(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo=0.0, hi=1.0):
        """Uniform double in [lo, hi) from the top 53 bits."""
        return lo + (hi - lo) * ((self.next() >> 11) * (1.0 / 9007199254740992.0))

    def randint(self, m):
        """Integer in [0, m) by multiply-shift on the top 32 bits."""
        return ((self.next() >> 32) * m) >> 32

    def shuffle(self, xs):
        for i in range(len(xs) - 1, 0, -1):
            j = self.randint(i + 1)
            xs[i], xs[j] = xs[j], xs[i]
        return xs


def seed_of(family, index):
    """Seed rule for the stand-in workloads: family id x 1000 + circuit index
    (0 layered + SWAPs, 1 benchmark circuits, 2 U3 layers, 3 QAOA batch,
    4 cost-model training)."""
    return family * 1000 + index


def fmt_gate(name, qubits, params=()):
    if name not in GATES:
        raise ValueError(f"unknown gate {name}")
    nq, npar = GATES[name]
    if len(qubits) != nq or len(params) != npar:
        raise ValueError(f"{name}: wrong arity")
    qs = ",".join(f"q[{q}]" for q in qubits)
    if npar:
        ps = ",".join(repr(float(p)) for p in params)
        return f"{name}({ps}) {qs};"
    return f"{name} {qs};"


def to_qasm(n, gates):
    """gates: list of (name, qubits, params)."""
    lines = ["OPENQASM 2.0;", f"qreg q[{n}];"]
    lines += [fmt_gate(g[0], g[1], g[2] if len(g) > 2 else ()) for g in gates]
    return "\n".join(lines) + "\n"


# ---------------------------------------------------------------------------
# Workload shapes
# ---------------------------------------------------------------------------

def ghz(n):
    """H on q0, then a CX chain q_i -> q_{i+1}."""
    gates = [("h", [0])]
    gates += [("cx", [i, i + 1]) for i in range(n - 1)]
    return gates


def qft(n, x=None, swaps=True, rng=None):
    """QFT of the basis state |x> (x drawn from rng when None).

    X gates prepare |x> (little-endian: q_i is bit i of x). Then for
    j = n-1 .. 0: H(q_j) followed by CP(pi / 2^(j-i)) with control q_i and
    target q_j for every i < j; then the SWAP network SWAP(q_i, q_{n-1-i}).
    With this orientation the result is
        2^(-n/2) sum_y exp(2 pi i x y / 2^n) |y>.
    """
    if x is None:
        rng = rng or SplitMix64(0)
        x = rng.next() & ((1 << n) - 1)
    gates = [("x", [i]) for i in range(n) if (x >> i) & 1]
    for j in range(n - 1, -1, -1):
        gates.append(("h", [j]))
        for i in range(j - 1, -1, -1):
            gates.append(("cp", [i, j], [math.pi / (1 << (j - i))]))
    if swaps:
        for i in range(n // 2):
            gates.append(("swap", [i, n - 1 - i]))
    return gates, x


def random_matching(rng, n):
    perm = rng.shuffle(list(range(n)))
    return [(perm[2 * i], perm[2 * i + 1]) for i in range(n // 2)]


def random_pair(rng, n):
    a = rng.randint(n)
    b = rng.randint(n - 1)
    if b >= a:
        b += 1
    return a, b


def random_layered(n, layers, rng, one_q=("h", "x", "rx", "ry", "rz"),
                   two_q=("cx",), n_swaps=0, swap_frac=None):
    """Layers of a random 1q gate on every qubit, then 2q gates on a matching.

    SWAPs on random pairs are inserted at uniformly random positions, either
    `n_swaps` of them or enough to make `swap_frac` of the final list.
    """
    gates = []
    for _ in range(layers):
        for q in range(n):
            name = one_q[rng.randint(len(one_q))]
            npar = GATES[name][1]
            params = [rng.uniform(0.0, 2.0 * math.pi) for _ in range(npar)]
            gates.append((name, [q], params))
        for a, b in random_matching(rng, n):
            name = two_q[rng.randint(len(two_q))]
            gates.append((name, [a, b], []))
    if swap_frac is not None:
        n_swaps = int(round(len(gates) * swap_frac / (1.0 - swap_frac)))
    for _ in range(n_swaps):
        pos = rng.randint(len(gates) + 1)
        a, b = random_pair(rng, n)
        gates.insert(pos, ("swap", [a, b], []))
    return gates


def random_3_regular(n, rng, max_tries=1000):
    """Random simple 3-regular graph on n (even) nodes by the pairing model."""
    if n % 2:
        raise ValueError("3-regular graphs need an even node count")
    for _ in range(max_tries):
        stubs = rng.shuffle([v for v in range(n) for _ in range(3)])
        edges = set()
        ok = True
        for i in range(0, len(stubs), 2):
            a, b = stubs[i], stubs[i + 1]
            if a == b or (min(a, b), max(a, b)) in edges:
                ok = False
                break
            edges.add((min(a, b), max(a, b)))
        if ok:
            return sorted(edges)
    raise RuntimeError("no simple 3-regular pairing found")


def qaoa_maxcut(n, p, rng):
    """QAOA Max-Cut ansatz: H on all, then p x (RZZ(gamma) on edges, RX(beta))."""
    edges = random_3_regular(n, rng)
    gates = [("h", [q]) for q in range(n)]
    for _ in range(p):
        gamma = rng.uniform(0.0, math.pi)
        beta = rng.uniform(0.0, math.pi)
        gates += [("rzz", [a, b], [gamma]) for a, b in edges]
        gates += [("rx", [q], [beta]) for q in range(n)]
    return gates, edges


# ---------------------------------------------------------------------------
# The five workload families
# ---------------------------------------------------------------------------

def layered_swaps_circuit(index=0, n=12, layers=20, n_swaps=10):
    """Plain per-gate case: random 1q layers + CX matching + 10 random SWAPs."""
    rng = SplitMix64(seed_of(0, index))
    return n, random_layered(n, layers, rng, n_swaps=n_swaps)


def benchmark_circuits(n=28, layers=30, index=0):
    """GHZ, QFT of a random basis state with swaps, 30-layer random + 5% SWAP."""
    rng = SplitMix64(seed_of(1, index))
    q, x = qft(n, rng=rng)
    return {
        "ghz": (n, ghz(n)),
        "qft": (n, q, x),
        "random": (n, random_layered(n, layers, rng, swap_frac=0.05)),
    }


def u3_entangler_circuit(n=32, layers=40, index=0):
    """U3 layers (angles in [0, 2pi)) + CX/CZ (p = 1/2) on a random matching."""
    rng = SplitMix64(seed_of(2, index))
    return n, random_layered(n, layers, rng, one_q=("u3",), two_q=("cx", "cz"))


def qaoa_batch(count=512, index=0, widths=(10, 12, 14, 16, 18, 20)):
    """QAOA circuits of even width in [10, 20], p uniform in 1..4."""
    rng = SplitMix64(seed_of(3, index))
    out = []
    for _ in range(count):
        n = widths[rng.randint(len(widths))]
        p = 1 + rng.randint(4)
        gates, _ = qaoa_maxcut(n, p, rng)
        out.append((n, gates))
    return out


def training_circuit(index, n_lo=20, n_hi=30, depth_lo=5, depth_hi=30):
    """Cost-model training circuits: layered random circuits (random one-qubit
    gates on every qubit, then CX on a random matching) of random n and depth."""
    rng = SplitMix64(seed_of(4, index))
    n = n_lo + rng.randint(n_hi - n_lo + 1)
    depth = depth_lo + rng.randint(depth_hi - depth_lo + 1)
    return n, random_layered(n, depth, rng, n_swaps=rng.randint(n))


def all_gate_types_circuit(n, length, rng):
    """Every gate type at random positions (test coverage of the gate table)."""
    names = sorted(GATES)
    gates = []
    for _ in range(length):
        name = names[rng.randint(len(names))]
        nq, npar = GATES[name]
        if nq > n:
            continue
        qs = rng.shuffle(list(range(n)))[:nq]
        params = [rng.uniform(-2.0 * math.pi, 2.0 * math.pi) for _ in range(npar)]
        gates.append((name, qs, params))
    return gates
