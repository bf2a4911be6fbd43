"""Chrome-trace export of a profiled apply call (the analogue of the
paper's timeline view of the context profile, Sec. III-C): one complete
event per launched block with its device start and duration from the
block records of qs_profile (calls made with QS_PROFILE), named for the
kernel class that ran it, with the block's qubits, gate count and bytes as
arguments. Open the file in a Chrome-trace viewer."""

import json

KINDS = {0: "dense", 1: "diagonal", 2: "bit exchange", 3: "tile pass", 4: "phase polynomial"}


def block_name(rec):
    """Kernel class of a block record."""
    name = f"{KINDS.get(rec.kind, 'block')} k={rec.k}"
    if rec.kind == 0 and rec.tc:
        name += " tensor cores" + (" lane exchange" if rec.tc == 2 else "")
    if rec.nctrl:
        name += f" ctrl={rec.nctrl}"
    return name


def chrome_trace(records, label="qs"):
    """Trace-event dict for timed block records (untimed ones are skipped)."""
    events = []
    for r in records:
        if r.ms < 0 or r.t_start_ms < 0:
            continue
        qubits = [int(q) for q in r.qubits if q >= 0]  # records pad with -1
        events.append({"name": block_name(r), "ph": "X", "pid": label, "tid": "stream",
                       "ts": r.t_start_ms * 1e3, "dur": r.ms * 1e3,
                       "args": {"index": int(r.index), "qubits": qubits, "gates": int(r.n_gates),
                                "bytes": float(r.bytes), "GB/s": float(r.bytes / r.ms / 1e6) if r.ms > 0 else None}})
    return {"traceEvents": events, "displayTimeUnit": "ms"}


def write_chrome_trace(state, path, label="qs"):
    """Writes the last profiled apply call of `state` as a Chrome trace;
    returns the number of events."""
    from . import qs_profile
    _, recs = qs_profile(state)
    tr = chrome_trace(recs, label)
    with open(path, "w") as f:
        json.dump(tr, f)
    return len(tr["traceEvents"])
