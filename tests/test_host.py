"""Host-side checks of the library (no GPU): exported symbols, the IR parser,
and the virtual-swap / fusion passes.

The passes are checked by applying the planned blocks' FP64 matrices to a
state in numpy (a contraction written here, independent of both the CUDA
kernels and the oracle's loops) and comparing with the oracle. Every fusion
is a valid answer as long as the product matches; no partition is assumed.
"""

import ctypes
import json
import math
import re
import subprocess

import numpy as np
import pytest

import circuitgen as cg
import oracle
import paper_2410_09326_gb300 as qs
from paper_2410_09326_gb300 import build as qbuild
from lane_exchange_rule import lane_exchange_expected


@pytest.fixture(scope="module", autouse=True)
def lib():
    return qs.load(build_if_missing=True)


def header_functions():
    text = open(qbuild.INC + "/qs.h").read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qs_[a-z_0-9]+)\s*\(", text)) - {"QS_FUSE_K"})


def test_every_declared_symbol_is_exported():
    names = header_functions()
    assert "qs_apply_circuit" in names and "qs_measure_probs" in names
    out = subprocess.run(["nm", "-D", "--defined-only", qs.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(qs.load(), n)


def test_binding_struct_layouts_match_the_header(tmp_path):
    """The ctypes structures of the binding have the sizes and field offsets
    the C compiler gives the header's structs (a mismatch would silently pass
    wrong options or misread records)."""
    structs = {"qs_opts": qs.qs_opts, "qs_block_record": qs.qs_block_record,
               "qs_profile_summary": qs.qs_profile_summary, "qs_class_table": qs.qs_class_table,
               "qs_batch_info_t": qs.qs_batch_info_t, "qs_exchange_layout": qs.qs_exchange_layout}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "qs.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", qbuild.INC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        name, field, value = line.split()
        cls = structs[name]
        got = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert got == int(value), (name, field, got, value)


def test_library_built_for_sm_103a():
    out = subprocess.run(["cuobjdump", "--list-elf", qs.library_path()], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_parser_matches_generator():
    rng = cg.SplitMix64(3)
    gates = cg.all_gate_types_circuit(7, 300, rng)
    n, arr = qs.qs_parse_qasm(cg.to_qasm(7, gates))
    assert n == 7 and arr.size == len(gates)
    for g, a in zip(gates, arr):
        assert qs.OPS[a["op"]] == g[0]
        assert list(a["q"][: a["nq"]]) == list(g[1])
        ps = g[2] if len(g) > 2 else []
        assert list(a["p"][: len(ps)]) == list(ps)  # exact round trip of 17 digits


@pytest.mark.parametrize("bad", ["qreg q[2];\nh q[2];\n", "qreg q[2];\ncx q[0],q[0];\n",
                                 "qreg q[2];\nrz q[0];\n", "qreg q[2];\nfoo q[0];\n", "h q[0];\n",
                                 "qreg q[2];\nh q[0]\n", "qreg q[41];\n"])
def test_parser_rejects(bad):
    with pytest.raises(qs.QsError) as e:
        qs.qs_parse_qasm(bad)
    assert e.value.status == qs.QS_EINVAL


def test_ids_follow_the_paper():
    # Sec. III-C: H is type 0 and CPhase type 11 in the context records
    assert qs.OPS.index("h") == 0 and qs.OPS.index("cp") == 11
    assert qs.OPS[:3] == ["h", "s", "t"] and len(qs.OPS) == 33


# ---------------------------------------------------------------------------
# Passes
# ---------------------------------------------------------------------------

def apply_block(psi, n, rec, mat):
    """Applies one planned block to a physical-order state (numpy, FP64)."""
    idx = np.arange(1 << n, dtype=np.int64)
    if rec.kind == 2:  # exchange of physical bits a, b
        a, b = rec.qubits[0], rec.qubits[1]
        flip = ((idx >> a) & 1) ^ ((idx >> b) & 1)
        return psi[idx ^ (flip << a) ^ (flip << b)]
    if rec.kind == 4:  # phase polynomial
        q = mat["qubits"]
        bits = [((idx >> int(x)) & 1).astype(float) for x in q]
        ang = np.full(1 << n, mat["c"])
        for j in range(len(q)):
            ang += mat["a"][j] * bits[j]
            for l in range(j + 1, len(q)):
                ang += mat["b"][j, l] * bits[j] * bits[l]
        return psi * np.exp(1j * ang)
    qubits = [int(rec.qubits[j]) for j in range(rec.k)]
    cm = int(rec.cmask)
    on = (idx & cm) == cm
    out = psi.copy()
    if rec.kind == 1:
        local = np.zeros(1 << n, dtype=np.int64)
        for j, q in enumerate(qubits):
            local |= ((idx >> q) & 1) << j
        out[on] = psi[on] * mat[local[on]]
        return out
    d = 1 << rec.k
    tmask = sum(1 << q for q in qubits)
    bases = idx[((idx & tmask) == 0) & on]
    offs = np.array([sum(((l >> j) & 1) << q for j, q in enumerate(qubits)) for l in range(d)],
                    dtype=np.int64)
    sel = bases[:, None] + offs[None, :]
    out[sel] = psi[sel] @ mat.T
    return out


def plan_state(n, gates, flags, init=None, opts=None):
    recs, mats, perm = qs.qs_plan(n, qs.gates_to_array(gates), flags, opts=opts)
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1
    if init is not None:
        psi = init.copy()
    for r, m in zip(recs, mats):
        if r.kind == 3:
            continue  # a tile pass: its member blocks follow
        psi = apply_block(psi, n, r, m)
    return psi, perm, recs


ALL_FLAGS = [qs.QS_PLAIN, qs.QS_VSWAP, qs.QS_DIAG, qs.QS_VSWAP | qs.QS_DIAG] + [
    qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k) | d for k in range(1, 7) for d in (0, qs.QS_DIAG)] + [
    qs.QS_FUSE | qs.QS_FUSE_K(4), qs.QS_PGO_RULES]


@pytest.mark.parametrize("flags", ALL_FLAGS)
def test_plan_reproduces_oracle_all_gate_types(flags):
    n = 7
    rng = cg.SplitMix64(4242)
    gates = cg.all_gate_types_circuit(n, 250, rng)
    want, operm = oracle.simulate(cg.to_qasm(n, gates))
    got, perm, recs = plan_state(n, gates, flags)
    if flags & qs.QS_VSWAP:
        assert list(perm) == list(operm)
    elif flags & qs.QS_PGO_RULES:
        assert sorted(perm) == list(range(n))  # the rules may also relocate
    else:
        assert list(perm) == list(range(n))
    assert np.linalg.norm(got - oracle.to_physical(want, perm)) < 1e-12


@pytest.mark.parametrize("flags", ALL_FLAGS[::3])
def test_plan_reproduces_oracle_qft_and_layered_swaps(flags):
    n = 8
    gates, x = cg.qft(n, x=77)
    want, operm = oracle.simulate(cg.to_qasm(n, gates))
    got, perm, _ = plan_state(n, gates, flags)
    assert np.linalg.norm(got - oracle.to_physical(want, perm)) < 1e-12
    n, gates = cg.layered_swaps_circuit(1)
    want, operm = oracle.simulate(cg.to_qasm(n, gates))
    got, perm, _ = plan_state(n, gates, flags)
    assert np.linalg.norm(got - oracle.to_physical(want, perm)) < 1e-12


def test_fusion_reduces_blocks():
    n, gates = cg.layered_swaps_circuit(0)
    arr = qs.gates_to_array(gates)
    counts = {k: len(qs.qs_plan(n, arr, qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k))[0]) for k in range(1, 7)}
    plain = len(qs.qs_plan(n, arr, qs.QS_PLAIN)[0])
    assert plain == len(gates)
    assert counts[1] < plain and all(counts[k + 1] <= counts[k] for k in range(1, 6))


def test_diagonal_runs_fuse_wide():
    # QFT: the CPhase ladder after each H is one diagonal run
    n = 12
    gates, _ = cg.qft(n, x=5, swaps=False)
    recs, mats, _ = qs.qs_plan(n, qs.gates_to_array(gates), qs.QS_FUSE | qs.QS_FUSE_K(1) | qs.QS_DIAG)
    diag = [r for r in recs if r.kind == 1]
    assert diag and max(r.k + r.nctrl for r in diag) >= 8


def test_controls_are_detected():
    recs, mats, _ = qs.qs_plan(5, qs.gates_to_array([("ccx", [0, 3, 1]), ("cp", [2, 4], [0.3])]), qs.QS_PLAIN)
    assert recs[0].kind == 0 and recs[0].k == 1 and recs[0].cmask == 0b1001 and recs[0].qubits[0] == 1
    # CPhase acts only where both bits are 1: a one-entry table with two controls
    assert recs[1].kind == 1 and recs[1].k == 0 and recs[1].cmask == 0b10100
    assert np.isclose(mats[1][0], np.exp(0.3j))


def test_identity_products_are_dropped():
    recs, _, _ = qs.qs_plan(3, qs.gates_to_array([("cx", [0, 1]), ("cx", [0, 1]), ("h", [2]), ("h", [2])]),
                            qs.QS_FUSE | qs.QS_FUSE_K(2))
    assert recs == []


def test_plan_rejects_bad_gates():
    arr = qs.gates_to_array([("h", [0])])
    arr[0]["q"][0] = 9
    with pytest.raises(qs.QsError) as e:
        qs.qs_plan(4, arr, qs.QS_PLAIN)
    assert e.value.status == qs.QS_EINVAL
    arr = qs.gates_to_array([("cx", [0, 1])])
    arr[0]["nq"] = 1
    with pytest.raises(qs.QsError):
        qs.qs_plan(4, arr, qs.QS_PLAIN)
    with pytest.raises(qs.QsError) as e:
        qs.qs_plan(4, qs.gates_to_array([("h", [0])]), qs.QS_FUSE | qs.QS_FUSE_K(7))
    assert e.value.status == qs.QS_EUNSUPPORTED


@pytest.mark.parametrize("flags", [qs.QS_PLAIN, qs.QS_VSWAP, qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(3),
                                   qs.QS_FUSE | qs.QS_FUSE_K(2) | qs.QS_DIAG])
def test_plan_perm_and_counts(flags):
    n, gates = cg.layered_swaps_circuit(0)
    arr = qs.gates_to_array(gates)
    recs, mats, perm = qs.qs_plan(n, arr, flags)
    _, operm = oracle.simulate(cg.to_qasm(n, gates))
    if flags & qs.QS_VSWAP:
        assert list(perm) == list(operm)
    else:
        assert list(perm) == list(range(n))
    assert sum(r.n_gates for r in recs) <= len(gates)
    k_max = (flags >> 16) & 15 if flags & qs.QS_FUSE else 3
    for r, m in zip(recs, mats):
        if r.kind == 0:
            assert r.k <= max(k_max, 3)
            assert np.allclose(m.conj().T @ m, np.eye(1 << r.k), atol=1e-12)
        elif r.kind == 1:
            assert r.k <= qs.QS_MAX_DIAG and np.allclose(np.abs(m), 1, atol=1e-12)


def test_swaps_absorbed_count():
    n = 6
    gates = [("h", [0]), ("swap", [0, 5]), ("cx", [5, 1]), ("swap", [1, 2])]
    recs, mats, perm = qs.qs_plan(n, qs.gates_to_array(gates), qs.QS_VSWAP)
    assert len(recs) == 2 and all(r.kind != 2 for r in recs)
    assert list(perm) == [5, 2, 1, 3, 4, 0]
    # the CX on logical (5 -> 1) runs on physical (0 -> 1)... after the
    # first swap logical 5 lives at physical 0
    assert recs[1].qubits[0] == 1 and recs[1].nctrl == 1
    recs, mats, perm = qs.qs_plan(n, qs.gates_to_array(gates), qs.QS_PLAIN)
    assert [r.kind for r in recs] == [0, 2, 0, 2]


# ---------------------------------------------------------------------------
# Profile-guided selection (host side)
# ---------------------------------------------------------------------------

def test_rules_select_follows_the_paper_rules():
    # a SWAP present -> virtual swap; more than one gate -> fusion
    n, gates = cg.layered_swaps_circuit(0)
    recs, _, perm = qs.qs_plan(n, qs.gates_to_array(gates), qs.QS_PGO_RULES)
    _, operm = oracle.simulate(cg.to_qasm(n, gates))
    assert list(perm) == list(operm)  # SWAPs were absorbed
    assert len(recs) < len(gates) // 2  # and gates were merged


def test_chrome_trace_of_block_records():
    """The Chrome-trace export: one complete event per timed record (start
    and duration in microseconds, the kernel class as the name, qubits without
    the -1 padding, GB/s from bytes and time), untimed records skipped, and
    the result serialisable as JSON."""
    from paper_2410_09326_gb300 import trace
    recs = []
    for i, (kind, k, tc, start, ms) in enumerate([(0, 5, 2, 0.0, 2.9), (4, 12, 0, 2.9, 2.8), (0, 3, 0, -1.0, -1.0)]):
        r = qs.qs_block_record()
        r.index, r.kind, r.k, r.tc, r.n_gates = i, kind, k, tc, 7
        for j in range(len(r.qubits)):
            r.qubits[j] = j if j < k else -1
        r.bytes = 17179869184.0
        r.t_start_ms, r.ms = start, ms
        recs.append(r)
    tr = json.loads(json.dumps(trace.chrome_trace(recs)))
    ev = tr["traceEvents"]
    assert len(ev) == 2 and all(e["ph"] == "X" for e in ev)
    assert ev[0]["name"] == "dense k=5 tensor cores lane exchange" and ev[1]["name"] == "phase polynomial k=12"
    assert ev[0]["ts"] == 0.0 and abs(ev[0]["dur"] - 2900.0) < 1e-9 and abs(ev[1]["ts"] - 2900.0) < 1e-9
    assert ev[0]["args"]["qubits"] == [0, 1, 2, 3, 4] and ev[0]["args"]["gates"] == 7
    assert abs(ev[0]["args"]["GB/s"] - 17179869184.0 / 2.9 / 1e6) < 1e-6


def test_memory_budget_refuses_before_any_cuda_call():
    """A state larger than the device-memory budget is refused with
    QS_ENOMEM by the budget itself (no CUDA call is made, so this holds
    without a GPU); the live byte count is unchanged."""
    before = qs.qs_memory_in_use()
    qs.qs_set_memory_limit(1 << 20)
    try:
        with pytest.raises(qs.QsError) as e:
            qs.qs_alloc_state(20, qs.QS_C64)  # 8 MiB
        assert e.value.status == qs.QS_ENOMEM and "memory budget" in str(e.value)
        assert qs.qs_memory_in_use() == before
    finally:
        qs.qs_set_memory_limit(0)


def exchange_emulation(lay, k):
    """Offsets (from the warp's base) of the amplitudes each lane of a
    lane-exchange warp loads, as a (32 lanes, registers, 2 elements) array,
    and the kernel's exchange step on such an array: the element bit with lane
    bit la (the lane whose la bit is 1 takes the partner's element-1 half into
    its element-0 half, the other lane the partner's element-0 half into its
    element-1 half), then lane bit lb[i] with register bit i (the lane whose
    lb bit is 1 takes the partner's register q2 = q | 2^i into its register q,
    the other the partner's register q into its register q2)."""
    nv = 16 if k == 6 else 1 << (k - 1)
    nrb = 4 if k == 6 else k - 1
    lanes = np.arange(32, dtype=np.int64)
    regs = np.arange(nv, dtype=np.int64)
    lane_off = sum(((lanes >> i) & 1) << int(lay.lane_bits[i]) for i in range(5))
    reg_off = sum(((regs >> j) & 1) << int(lay.reg_bits[j]) for j in range(nrb))
    off = lane_off[:, None, None] + reg_off[None, :, None] + np.arange(2, dtype=np.int64)[None, None, :]

    def run(w):
        w = w.copy()
        n_regs = w.shape[1]
        if lay.la >= 0:
            up = ((lanes >> lay.la) & 1) == 1
            partner = lanes ^ (1 << lay.la)
            old = w.copy()
            w[up, :, 0] = old[partner[up], :, 1]
            w[~up, :, 1] = old[partner[~up], :, 0]
        for i in range(lay.nswb):
            up = ((lanes >> lay.lb[i]) & 1) == 1
            partner = lanes ^ (1 << lay.lb[i])
            old = w.copy()
            for q in range(n_regs):
                if (q >> i) & 1:
                    continue
                q2 = q | (1 << i)
                w[up, q, :] = old[partner[up], q2, :]
                w[~up, q2, :] = old[partner[~up], q, :]
        return w

    return off, run


def test_lane_exchange_layout_index_arithmetic():
    """The tensor-core lane-exchange layout (qs_tc_exchange_layout), checked
    by emulating a warp on the CPU for 3000 random blocks (4..6 targets,
    biased to low bits, 0..2 controls, n up to 34) and 1000 6-target blocks
    with uniformly placed bits: the element, lane and
    register bits are exactly the warp's sub-cube (targets + five lowest free
    bits), so every amplitude of a sub-cube is loaded once; after the
    exchanges every lane holds one group -- one assignment of the free bits
    -- in slot order (slot bit s -> target slot_target[s]); the exchanges run
    again 4 registers at a time (as the kernels' stores do) restore the load
    layout; no target but the element bit's partner sits on a lane bit
    above bit 3; the layout applies exactly when bit 0 is not a control and
    7 or more free bits remain."""
    rng = cg.SplitMix64(4242)
    applied = 0
    for trial in range(4000):
        # the last 1000: 6-target blocks with uniformly placed bits
        k = 6 if trial >= 3000 else 4 + rng.randint(3)
        nctrl = rng.randint(3)
        n = min(34, k + nctrl + 5 + rng.randint(12))
        chosen = []
        while len(chosen) < k + nctrl:
            q = rng.randint(n) if trial >= 3000 or rng.randint(3) == 0 else rng.randint(min(n, 8))
            if q not in chosen:
                chosen.append(q)
        targets = sorted(chosen[:k])
        ctrls = chosen[k:]
        cmask = sum(1 << c for c in ctrls)
        lay = qs.qs_tc_exchange_layout(n, targets, cmask)
        assert bool(lay.applies) == (0 not in ctrls and n - k - nctrl >= 7), (n, targets, ctrls)
        if not lay.applies:
            continue
        applied += 1
        inner = targets[:5]
        free5 = [q for q in range(64) if q not in targets and q not in ctrls][:5]
        cube = sorted(set(inner) | set(free5))
        nrb = 4 if k == 6 else k - 1
        pos = [0] + list(lay.lane_bits) + list(lay.reg_bits[:nrb])
        assert sorted(pos) == cube, (targets, ctrls, pos, cube)
        if k == 6:
            assert list(lay.part_bits) == [targets[5], -1] and lay.slot_target[5] == 5
        else:
            assert list(lay.part_bits) == [-1, -1]
        assert 0 <= lay.nswb <= 2
        # loads read whole 128-byte lines where they can: no target sits on
        # a lane bit above bit 3 but the element bit's partner
        lane_t = [b for b in lay.lane_bits if b in inner]
        partner = [] if 0 in inner else [min(lane_t)]
        assert all(b <= 3 for b in lane_t if b not in partner), (targets, list(lay.lane_bits))
        off, run = exchange_emulation(lay, k)
        after = run(off)
        tmask = sum(1 << t for t in inner)
        nv = off.shape[1]
        rho = (np.arange(2)[None, :] + 2 * np.arange(nv)[:, None])   # slot of (register, element)
        slot_off = np.zeros_like(rho)
        for sb in range(len(inner)):
            slot_off += ((rho >> sb) & 1) << targets[lay.slot_target[sb]]
        groups = after[:, 0, 0]
        assert np.all(groups & tmask == 0)
        assert sorted(groups.tolist()) == sorted(sum(((g >> i) & 1) << free5[i] for i in range(5)) for g in range(32))
        assert np.array_equal(after, groups[:, None, None] + slot_off[None, :, :])
        back = np.concatenate([run(after[:, c:c + 4, :]) for c in range(0, nv, 4)], axis=1)
        assert np.array_equal(back, off)
    assert applied > 2500


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_lane_exchange_choice_on_benchmark_circuits(mode):
    """The planner marks a 4/5/6-target tensor-core block for lane-exchange
    gathers (record tc = 2) exactly where the rule says: automatic mode where
    the plain gather reads short runs, never with mode 1, wherever the layout
    fits with mode 2. Checked on every block of the n = 30 benchmark circuits
    and of 40 random circuits at n = 12..20."""
    o = qs.qs_default_opts()
    o.tc_exchange = mode
    cases = []
    c = cg.benchmark_circuits(n=30)
    cases += [(30, c["ghz"][1]), (30, c["qft"][1]), (30, c["random"][1])]
    for i in range(40):
        rng = cg.SplitMix64(7000 + i)
        n = 12 + i % 9
        gates = cg.random_layered(n, 4, rng, one_q=("u3",), two_q=("cx", "cz"))
        for _ in range(3 * n):  # controlled gates: blocks with controls
            q = rng.shuffle(list(range(n)))[:3]
            gates.append(("ccx", q) if rng.randint(2) else ("cu3", q[:2], [rng.uniform(0, 6.28) for _ in range(3)]))
        cases.append((n, gates))
    seen = {1: 0, 2: 0}
    for n, gates in cases:
        for k in (4, 5, 6):
            recs, _, _ = qs.qs_plan(n, qs.gates_to_array(gates), qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_TC,
                                    opts=o)
            for r in recs:
                if r.kind != 0 or r.k not in (4, 5, 6):
                    continue
                qubits = [int(x) for x in r.qubits[:r.k]]
                ctrls = [q for q in range(n) if (r.cmask >> q) & 1]
                fits, pays = lane_exchange_expected(n, qubits, ctrls)
                expect = fits and (mode == 2 or (mode == 0 and pays))
                assert r.tc == (2 if expect else 1), (n, qubits, ctrls, mode)
                seen[r.tc] += 1
    assert seen[1] > 0 and (mode == 1 or seen[2] > 0)


def test_measured_select_with_priors_prefers_wide_tensor_core_blocks():
    c = cg.benchmark_circuits(n=30)
    n, gates = c["random"]
    flags, ms = qs.qs_pgo_select(n, qs.gates_to_array(gates))
    assert flags & qs.QS_VSWAP and flags & qs.QS_FUSE and flags & qs.QS_TC
    assert (flags >> 16) & 15 in (4, 5, 6)
    assert 100 < ms < 5000
    # GHZ has no SWAP: no virtual swap in the choice
    n, gates = c["ghz"]
    flags, _ = qs.qs_pgo_select(n, qs.gates_to_array(gates))
    assert not flags & qs.QS_VSWAP and flags & qs.QS_FUSE


def test_pgo_predict_matches_the_selectors_estimate():
    """qs_pgo_predict of the flag set qs_pgo_select chose reproduces the
    selector's own predicted time (priors and a class table), and no
    candidate the selector considered is predicted faster."""
    n = 24
    gates = qs.gates_to_array(cg.benchmark_circuits(n=n)["random"][1])
    t = qs.qs_class_table()
    for c in range(qs.QS_N_CLASSES):
        t.bytes[c], t.ms[c], t.count[c] = (3e9 if c % 3 else 5e9), 1.0, 1
    for table in (None, t):
        f, ms = qs.qs_pgo_select(n, gates, table=table)
        assert qs.qs_pgo_predict(n, gates, f, table=table) == pytest.approx(ms, rel=1e-12)
        others = [qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_DIAG | tc
                  for k in range(1, 7) for tc in ((0, qs.QS_TC) if k >= 4 else (0,))]
        assert all(qs.qs_pgo_predict(n, gates, g, table=table) >= ms * 0.999 for g in others)
    with pytest.raises(qs.QsError):
        qs.qs_pgo_predict(n, gates, qs.QS_PGO_RULES)


def test_measured_select_follows_the_table():
    """A table in which every tensor-core class ran slowly steers the choice
    away from the tensor cores; one in which wide CUDA-core blocks ran fast
    steers it to them."""
    c = cg.benchmark_circuits(n=26)
    n, gates = c["random"]
    arr = qs.gates_to_array(gates)
    t = qs.qs_class_table()
    for cls in range(qs.QS_N_CLASSES):
        kind, k, tc = (cls % 32) // 8, cls % 8, bool(cls & 32)
        gbs = 6000.0
        if tc or kind == 3:
            gbs = 300.0
        elif kind == 0 and k >= 4:
            gbs = 500.0
        t.bytes[cls] = gbs * 1e9 * 1e-3  # bytes moved in 1 ms at that rate
        t.ms[cls] = 1.0
        t.count[cls] = 1
    flags, _ = qs.qs_pgo_select(n, arr, table=t)
    assert not flags & qs.QS_TC and (flags >> 16) & 15 <= 3
    for cls in range(qs.QS_N_CLASSES):
        kind, k = (cls % 32) // 8, cls % 8
        if kind == 0 and k == 6 and not cls & 32:
            t.bytes[cls] = 7000.0 * 1e6
    flags, _ = qs.qs_pgo_select(n, arr, table=t)
    assert (flags >> 16) & 15 == 6 and not flags & qs.QS_TC


def low_heavy_circuit(n, reps=30, seed=3, swaps=True):
    rng = cg.SplitMix64(seed)
    gates = []
    for _ in range(reps):
        gates.append(("u3", [0], [rng.uniform(0, 6) for _ in range(3)]))
        gates.append(("u3", [1], [rng.uniform(0, 6) for _ in range(3)]))
        gates.append(("cx", [0, 1]))
        gates.append(("cx", [1, 2 + rng.randint(n - 2)]))
        if swaps:
            gates.append(("swap", [2 + rng.randint(n - 2), 2 + rng.randint(n - 2)]))
            if gates[-1][1][0] == gates[-1][1][1]:
                gates.pop()
    return gates


@pytest.mark.parametrize("flags", [qs.QS_RELOCATE, qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(4) | qs.QS_RELOCATE,
                                   qs.QS_PGO_RULES])
def test_relocation_moves_hot_low_bits_and_stays_exact(flags):
    n = 14
    gates = low_heavy_circuit(n)
    want, _ = oracle.simulate(cg.to_qasm(n, gates))
    got, perm, recs = plan_state(n, gates, flags)
    assert np.linalg.norm(got - oracle.to_physical(want, perm)) < 1e-12
    exchanges = [r for r in recs if r.kind == 2 and r.n_gates == 0]
    assert len(exchanges) == 2 and {min(r.qubits[0], r.qubits[1]) for r in exchanges} == {0, 1}
    # after relocation no dense block targets both bits 0 and 1
    assert not any(r.kind == 0 and r.k >= 2 and r.qubits[0] == 0 and r.qubits[1] == 1 for r in recs)


def test_relocation_leaves_balanced_circuits_alone():
    n, gates = cg.layered_swaps_circuit(0)
    recs, _, _ = qs.qs_plan(n, qs.gates_to_array(gates), qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(4) | qs.QS_RELOCATE)
    assert not any(r.kind == 2 and r.n_gates == 0 for r in recs)


def tile_opts(bits, k=0):
    o = qs.qs_default_opts()
    o.tile_bits = bits
    o.tile_k = k
    return o


def tile_groups(recs):
    """(tile record, [member records]) for every tile pass of a plan."""
    out = []
    for r in recs:
        if r.kind == 3:
            out.append((r, []))
        elif out and r.index == out[-1][0].index:
            out[-1][1].append(r)
    return out


@pytest.mark.parametrize("bits,k", [(8, 1), (8, 2), (8, 3), (9, 4), (11, 3)])
def test_tile_plan_reproduces_oracle(bits, k):
    """Cache-blocked passes: applying every pass's member blocks in order (the
    work one tile pass does per tile) gives the oracle's state; dense members
    only touch the tile's qubits, and each pass has at least two members."""
    o = tile_opts(bits, k)
    cases = [(12, cg.all_gate_types_circuit(12, 300, cg.SplitMix64(77 + bits + k))),
             (13, cg.random_layered(13, 6, cg.SplitMix64(78 + k), n_swaps=6)),
             (12, cg.qft(12, x=1234)[0])]
    for n, gates in cases:
        want, operm = oracle.simulate(cg.to_qasm(n, gates))
        got, perm, recs = plan_state(n, gates, qs.QS_VSWAP | qs.QS_TILE, opts=o)
        assert list(perm) == list(operm)
        assert np.linalg.norm(got - oracle.to_physical(want, perm)) < 1e-12
        groups = tile_groups(recs)
        assert groups
        for t, members in groups:
            assert t.k == bits and t.meta == 5 and len(members) >= 2
            tile = set(range(4)) | {int(q) for q in t.qubits if q >= 0}
            assert len(tile) == min(bits, 4 + 10)
            assert t.n_gates == sum(m.n_gates for m in members)
            for m in members:
                if m.kind == 0:
                    # one gate alone may be wider than tile_k (a CX at tile_k = 1)
                    assert m.k <= max(k, 2) and {int(m.qubits[j]) for j in range(m.k)} <= tile
                else:
                    assert m.kind == 1


def test_tile_plan_options_and_small_states():
    arr = qs.gates_to_array(cg.random_layered(12, 3, cg.SplitMix64(5)))
    for bad in (tile_opts(7), tile_opts(15), tile_opts(9, 5)):
        with pytest.raises(qs.QsError):
            qs.qs_plan(12, arr, qs.QS_TILE, opts=bad)
    # a state no wider than one tile runs without tile passes
    recs, _, _ = qs.qs_plan(12, arr, qs.QS_TILE, opts=tile_opts(12))
    assert not any(r.kind == 3 for r in recs)
    recs, _, _ = qs.qs_plan(12, arr, qs.QS_TILE, opts=tile_opts(11))
    assert any(r.kind == 3 for r in recs)


def test_tile_passes_cut_hbm_passes_at_n30():
    """At the benchmark width the tile planner needs far fewer passes over
    the state than 5-qubit fusion (the point of cache blocking) on circuits
    of dense gates."""
    c = cg.benchmark_circuits(n=30)
    fused = qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(5) | qs.QS_DIAG
    for name in ("ghz", "random"):
        arr = qs.gates_to_array(c[name][1])
        top_fused = [r for r in qs.qs_plan(30, arr, fused)[0]]
        top_tiled = [r for r in qs.qs_plan(30, arr, qs.QS_VSWAP | qs.QS_TILE)[0] if not tile_member(r)]
        assert len(top_tiled) < 0.5 * len(top_fused), (name, len(top_tiled), len(top_fused))


def tile_member(r, _last=[None]):
    # records after a tile record that carry its index are its members
    if r.kind == 3:
        _last[0] = r.index
        return False
    return r.index == _last[0]


def diagonal_circuit(n, count, seed, dense_every=0):
    """Random diagonal gates of every kind (optionally with an H now and then)."""
    rng = cg.SplitMix64(seed)
    names = [("t", 1, 0), ("s", 1, 0), ("z", 1, 0), ("sdg", 1, 0), ("tdg", 1, 0), ("rz", 1, 1), ("u1", 1, 1),
             ("cp", 2, 1), ("cu1", 2, 1), ("cz", 2, 0), ("crz", 2, 1), ("rzz", 2, 1), ("id", 1, 0)]
    gates = []
    for i in range(count):
        if dense_every and i % dense_every == dense_every - 1:
            gates.append(("h", [rng.randint(n)], []))
            continue
        name, nq, npar = names[rng.randint(len(names))]
        qs_ = rng.shuffle(list(range(n)))[:nq]
        gates.append((name, qs_, [rng.uniform(-2 * math.pi, 2 * math.pi) for _ in range(npar)]))
    return gates


@pytest.mark.parametrize("n,seed,dense_every", [(11, 1, 0), (12, 2, 0), (13, 3, 25), (14, 4, 40)])
def test_phase_polynomial_blocks_reproduce_oracle(n, seed, dense_every):
    """Diagonal runs wider than the phase table become one phase polynomial
    (kind 4): applying its constant, linear and pair angles gives the
    oracle's state in FP64."""
    gates = diagonal_circuit(n, 400, 600 + seed, dense_every)
    want, _ = oracle.simulate(cg.to_qasm(n, gates))
    got, perm, recs = plan_state(n, gates, qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(4) | qs.QS_DIAG)
    assert any(r.kind == 4 and r.k > 10 for r in recs)
    assert np.linalg.norm(got - oracle.to_physical(want, perm)) < 1e-12


def test_qft_diagonal_ladders_become_polynomials():
    n = 14
    gates, x = cg.qft(n, x=4321)
    want, _ = oracle.simulate(cg.to_qasm(n, gates))
    got, perm, recs = plan_state(n, gates, qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(5) | qs.QS_DIAG)
    assert np.linalg.norm(got - oracle.to_physical(want, perm)) < 1e-12
    narrow = qs.qs_plan(n, qs.gates_to_array(gates), qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(5) | qs.QS_DIAG)[0]
    assert any(r.kind == 4 for r in narrow)
    # states of at most 10 qubits keep phase tables
    recs10 = qs.qs_plan(10, qs.gates_to_array(cg.qft(10, x=5)[0]), qs.QS_FUSE | qs.QS_FUSE_K(5) | qs.QS_DIAG)[0]
    assert not any(r.kind == 4 for r in recs10)


def test_measured_select_picks_tile_passes_when_they_measured_fast():
    """Cache-blocked passes are a candidate of the measured-profile activator:
    chosen when the table says tile passes move bytes at HBM speed, not with
    the compiled-in priors (their CUDA-core arithmetic is the bound)."""
    c = cg.benchmark_circuits(n=30)
    n, gates = c["random"]
    arr = qs.gates_to_array(gates)
    flags, _ = qs.qs_pgo_select(n, arr)
    assert not flags & qs.QS_TILE
    t = qs.qs_class_table()
    for cls in range(qs.QS_N_CLASSES):
        kind = (cls % 32) // 8
        t.bytes[cls] = (6500.0 if kind == 3 else 5000.0) * 1e6
        t.ms[cls] = 1.0
        t.count[cls] = 1
    flags, ms = qs.qs_pgo_select(n, arr, table=t)
    assert flags & qs.QS_TILE and flags & qs.QS_VSWAP


def test_lookahead_fusion_never_adds_blocks_and_saves_them_on_layered_circuits():
    """The roll-out search keeps first fit's grouping unless it finds one with
    fewer blocks; on the layered random circuits it does (the measured step
    time follows the block count, each block being one HBM pass)."""
    c = cg.benchmark_circuits(n=30)
    arr = qs.gates_to_array(c["random"][1])
    first = qs.qs_default_opts()
    first.fuse_lookahead = 0
    for k in (4, 5, 6):
        flags = qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(k) | qs.QS_DIAG
        base = len(qs.qs_plan(30, arr, flags, opts=first)[0])
        searched = len(qs.qs_plan(30, arr, flags)[0])
        assert searched <= base
        if k >= 5:
            assert searched <= 0.9 * base, (k, searched, base)
    for name in ("ghz", "qft"):
        arr = qs.gates_to_array(c[name][1])
        flags = qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(5) | qs.QS_DIAG
        assert len(qs.qs_plan(30, arr, flags)[0]) <= len(qs.qs_plan(30, arr, flags, opts=first)[0])
