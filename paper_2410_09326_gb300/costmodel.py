"""Cost-model workflow over the C ABI: profile blocks, train, select.

Data: every block the simulator launches under QS_PROFILE becomes one sample
(qs_block_features row, natural log of its event-timed milliseconds).
Training and prediction run in the library (qs_mlp_train / qs_mlp_predict);
this module only drives the calls and holds no simulation arithmetic.
"""

import math

import numpy as np

import circuitgen as cg

from . import (QS_C64, QS_DIAG, QS_FUSE, QS_FUSE_K, QS_PROFILE, QS_TC, QS_TILE, QS_VSWAP, gates_to_array,
               qs_alloc_state, qs_apply_circuit, qs_block_features, qs_free_state, qs_mlp_predict, qs_plan,
               qs_profile, qs_set_basis)

# flag sets profiled for training: every kernel class the selector can choose
TRAIN_FLAGS = [0, QS_VSWAP] + [QS_VSWAP | QS_FUSE | QS_FUSE_K(k) | QS_DIAG for k in (2, 3, 4, 5, 6)] + \
              [QS_VSWAP | QS_FUSE | QS_FUSE_K(k) | QS_DIAG | QS_TC for k in (4, 5, 6)] + [QS_VSWAP | QS_TILE]


def profile_blocks(n, gates, flags, state=None, repeats=1):
    """(features, log_ms) of every block of one run (the last of `repeats`)."""
    own = state is None
    st = qs_alloc_state(n, QS_C64) if own else state
    try:
        arr = gates_to_array(gates)
        for _ in range(repeats):
            qs_set_basis(st, 0)
            qs_apply_circuit(st, arr, flags | QS_PROFILE)
            summ, recs = qs_profile(st)
        recs = [r for r in recs if r.ms > 0]
        feats = qs_block_features(n, recs)
        y = np.array([math.log(r.ms) for r in recs], dtype=np.float32)
        return feats, y, summ.total_ms
    finally:
        if own:
            qs_free_state(st)


def build_dataset(circuits, flag_sets=TRAIN_FLAGS, max_n=None):
    """Profiles every circuit under every flag set; returns (X, y)."""
    xs, ys = [], []
    states = {}
    try:
        for n, gates in circuits:
            if max_n and n > max_n:
                continue
            if n not in states:
                states[n] = qs_alloc_state(n, QS_C64)
            for f in flag_sets:
                x, y, _ = profile_blocks(n, gates, f, state=states[n])
                xs.append(x)
                ys.append(y)
    finally:
        for st in states.values():
            qs_free_state(st)
    return np.concatenate(xs), np.concatenate(ys)


def training_circuits(count, n_lo=20, n_hi=30, index0=0):
    """Seeded training circuits of random width in [n_lo, n_hi]: mostly
    layered random circuits, plus QFTs of random basis states, GHZ
    chains and QAOA ansaetze, so that wide diagonal blocks and chains are in
    the training distribution too."""
    out = []
    for i in range(count):
        kind = i % 10
        rng = cg.SplitMix64(cg.seed_of(4, 100000 + index0 + i))
        n = n_lo + rng.randint(n_hi - n_lo + 1)
        if kind < 6:
            out.append(cg.training_circuit(index0 + i, n_lo=n_lo, n_hi=n_hi))
        elif kind < 8:
            gates, _ = cg.qft(n, rng=rng)
            out.append((n, gates))
        elif kind == 8:
            out.append((n, cg.ghz(n)))
        else:
            n -= n % 2
            gates, _ = cg.qaoa_maxcut(n, 1 + rng.randint(4), rng)
            out.append((n, gates))
    return out


def mlp_plan_ms(m, n, gates, flags):
    """The network's prediction of one flag set's device time: the planned
    blocks' predicted times plus the activator's launch gap per block."""
    recs, _, _ = qs_plan(n, gates_to_array(gates), flags)
    # a tile pass's member blocks follow it with its index; only the pass runs
    seen = set()
    recs = [r for r in recs if not (r.index in seen or seen.add(r.index))]
    if not recs:
        return 0.0
    y = qs_mlp_predict(m, qs_block_features(n, recs))
    return float(np.exp(y.astype(np.float64)).sum() + 0.004 * len(recs))


def measure_candidates(n, gates, candidates, repeats=2):
    """Measured total block time of each candidate flag set (brute force)."""
    st = qs_alloc_state(n, QS_C64)
    try:
        out = {}
        for f in candidates:
            best = float("inf")
            for _ in range(repeats):
                _, _, ms = profile_blocks(n, gates, f, state=st)
                best = min(best, ms)
            out[f] = best
        return out
    finally:
        qs_free_state(st)
