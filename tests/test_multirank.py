"""The benchmark's multi-rank host logic on CPU with gloo, world size 2:
barrier, max over ranks of the per-rank time, and the whole-job aggregate of
independent replicas (weak scaling)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, _, w = bench.dist_env()
    assert (r, w) == (rank, world)
    bench.barrier(world)
    mx = bench.max_over_ranks(100.0 + 50.0 * rank, world)
    val = bench.aggregate_value(17.18e9, mx, world)
    out[rank] = (mx, val)
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 150.0  # the slowest rank's time
    # two replicas of 17.18 GB each in 150 ms
    assert out[0][1] == pytest.approx(2 * 17.18e9 / 0.150 / 1e9)


# ---------------------------------------------------------------------------
# Global-bit tier: a sharded execution of the host plan on gloo ranks
# ---------------------------------------------------------------------------

def _apply_shard(shard, n, g, rank, rec, mat):
    """One planned block on this rank's shard (numpy, FP64). The shard holds
    the amplitudes whose top g physical bits equal `rank`; a block may name
    global bits only where its matrix is block-diagonal in them (asserted)."""
    import numpy as np
    nl = n - g
    loc = np.arange(1 << nl, dtype=np.int64)
    full = loc | (rank << nl)
    if rec.kind == 4:  # phase polynomial over full indices
        bits = [((full >> int(x)) & 1).astype(float) for x in mat["qubits"]]
        ang = np.full(1 << nl, mat["c"])
        for j in range(len(bits)):
            ang += mat["a"][j] * bits[j]
            for l in range(j + 1, len(bits)):
                ang += mat["b"][j, l] * bits[j] * bits[l]
        return shard * np.exp(1j * ang)
    qubits = [int(rec.qubits[j]) for j in range(rec.k)]
    if rec.kind == 2:  # exchange of two local bits
        a, b = qubits
        assert a < nl and b < nl
        flip = ((loc >> a) & 1) ^ ((loc >> b) & 1)
        return shard[loc ^ (flip << a) ^ (flip << b)]
    cm = int(rec.cmask)
    if ((rank << nl) & cm) != (cm & ~((1 << nl) - 1)):
        return shard  # a global control is 0 on this shard
    cml = cm & ((1 << nl) - 1)
    on = (loc & cml) == cml
    gj = [j for j, q in enumerate(qubits) if q >= nl]
    lj = [j for j, q in enumerate(qubits) if q < nl]
    fixed = sum(((rank >> (qubits[j] - nl)) & 1) << j for j in gj)
    gmask = sum(1 << j for j in gj)
    d = 1 << rec.k
    keep = [l for l in range(d) if (l & gmask) == fixed]
    out = shard.copy()
    if rec.kind == 1:
        sub = mat[keep]
        local = np.zeros(1 << nl, dtype=np.int64)
        for i, j in enumerate(lj):
            local |= ((loc >> qubits[j]) & 1) << i
        out[on] = shard[on] * sub[local[on]]
        return out
    other = [l for l in range(d) if (l & gmask) != fixed]
    if other:
        assert np.abs(mat[np.ix_(keep, other)]).max() < 1e-14, "block not diagonal in a global bit"
    sub = mat[np.ix_(keep, keep)]
    lq = [qubits[j] for j in lj]
    tmask = sum(1 << q for q in lq)
    bases = loc[((loc & tmask) == 0) & on]
    offs = np.array([sum(((l >> i) & 1) << q for i, q in enumerate(lq)) for l in range(len(keep))],
                    dtype=np.int64)
    sel = bases[:, None] + offs[None, :]
    out[sel] = shard[sel] @ sub.T
    return out


def _exchange(shard, n, g, rank, local_bit, global_bit):
    """Virtual swap of a local with a global bit: this rank and the rank that
    differs in the global bit trade the halves of their shards whose local
    bit differs from their own global bit."""
    import numpy as np
    import torch
    import torch.distributed as dist
    nl = n - g
    gb = global_bit - nl
    partner = rank ^ (1 << gb)
    mine = (rank >> gb) & 1
    loc = np.arange(1 << nl, dtype=np.int64)
    half = loc[((loc >> local_bit) & 1) != mine]
    send = torch.from_numpy(np.ascontiguousarray(shard[half])).view(torch.float64)
    recv = torch.empty_like(send)
    reqs = [dist.isend(send, partner), dist.irecv(recv, partner)]
    for r in reqs:
        r.wait()
    out = shard.copy()
    out[half] = recv.view(torch.complex128).numpy()
    return out


def _sharded_worker(rank, world, port, n, flag_list, out):
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import circuitgen as cg
    import paper_2410_09326_gb300 as qs
    g = world.bit_length() - 1
    nl = n - g
    rng = cg.SplitMix64(7100 + n)
    gates = cg.all_gate_types_circuit(n, 160, rng) + cg.random_layered(n, 4, rng, n_swaps=4)
    res = {}
    for flags in flag_list:
        o = qs.qs_default_opts()
        o.n_global = g
        recs, mats, perm = qs.qs_plan(n, qs.gates_to_array(gates), flags, opts=o)
        shard = np.zeros(1 << nl, dtype=np.complex128)
        if rank == 0:
            shard[0] = 1
        exchanges = 0
        for r, m in zip(recs, mats):
            if r.kind == 5:
                assert r.qubits[0] < nl <= r.qubits[1]
                shard = _exchange(shard, n, g, rank, int(r.qubits[0]), int(r.qubits[1]))
                exchanges += 1
            else:
                shard = _apply_shard(shard, n, g, rank, r, m)
        parts = [torch.empty(2 << nl, dtype=torch.float64) for _ in range(world)] if rank == 0 else None
        dist.gather(torch.from_numpy(shard).view(torch.float64), parts, dst=0)
        if rank == 0:
            psi = np.concatenate([p.view(torch.complex128).numpy() for p in parts])
            res[flags] = (psi, [int(x) for x in perm], exchanges)
    if rank == 0:
        out["res"] = {f: (v[0].tobytes(), v[1], v[2]) for f, v in res.items()}
        out["gates"] = gates
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_plan_with_global_bits_matches_the_oracle(world):
    """The global-bit tier of the planner (opts.n_global), executed by
    `world` gloo ranks on the CPU: each rank holds the shard of its global
    bits' value, applies the plan's blocks in FP64 with those bits fixed
    (a block names a global bit only where its matrix is block-diagonal in
    it), and performs each planned exchange of a local with a global bit as
    a pairwise half-shard send/recv. The gathered state, placed through the
    plan's perm, equals the oracle's to 1e-12 for plain, virtual-swap,
    fused and rule-activated plans, with exchanges planned."""
    import numpy as np
    import circuitgen as cg
    import oracle
    import paper_2410_09326_gb300 as qs
    n = 8
    flag_list = [qs.QS_PLAIN, qs.QS_VSWAP, qs.QS_VSWAP | qs.QS_FUSE | qs.QS_FUSE_K(3) | qs.QS_DIAG,
                 qs.QS_FUSE | qs.QS_FUSE_K(4) | qs.QS_DIAG, qs.QS_PGO_RULES]
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, world, port, n, flag_list, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    want, _ = oracle.simulate(cg.to_qasm(n, out["gates"]))
    for flags, (buf, perm, exchanges) in out["res"].items():
        psi = np.frombuffer(buf, dtype=np.complex128)
        assert exchanges > 0, hex(flags)
        assert sorted(perm) == list(range(n))
        err = np.linalg.norm(psi - oracle.to_physical(want, perm))
        assert err < 1e-12, (hex(flags), err)
