"""Python binding of the GB300 state-vector simulator core (libqs.so).

Argument marshalling only: every step of the simulation (parsing, virtual
swap, fusion, the kernels, the reductions) runs in the native library
declared in `include/qs.h`. Function names match the C ABI. Import fails
loudly when the library has not been built (see `build.py`); there is no
CPU fallback.
"""

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

QS_OK, QS_EINVAL, QS_ENOMEM, QS_ECUDA, QS_EUNSUPPORTED, QS_ETIMEOUT, QS_ESTATE = range(7)
QS_C64, QS_C128 = 0, 1

QS_PLAIN = 0
QS_VSWAP = 1 << 0
QS_FUSE = 1 << 1
QS_DIAG = 1 << 2
QS_TC = 1 << 3
QS_PROFILE = 1 << 4
QS_RELOCATE = 1 << 5
QS_FOLD = 1 << 6
QS_TILE = 1 << 7
QS_PGO_RULES = 1 << 8
QS_PGO_MEASURED = 1 << 9


def QS_FUSE_K(k):
    return (k & 15) << 16


QS_N_GATE_TYPES = 33
QS_N_CLASSES = 128
QS_MLP_FEATURES = 24
QS_MLP_HIDDEN = 64
QS_MLP_PARAMS = 64 * 24 + 64 + 64 * 64 + 64 + 64 + 1
QS_MAX_QUBITS = 40
QS_MAX_DIAG = 10

OPS = ["h", "s", "t", "x", "y", "z", "sdg", "tdg", "rx", "ry", "rz", "cp", "cu1", "swap",
       "cx", "cz", "cy", "ch", "crx", "cry", "crz", "u1", "u2", "u3", "sx", "sxdg", "id",
       "rzz", "rxx", "ryy", "ccx", "cswap", "cu3"]

GATE_DTYPE = np.dtype([("op", "u1"), ("nq", "u1"), ("q", "u1", (6,)), ("p", "<f8", (3,))])
assert GATE_DTYPE.itemsize == 32


class QsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"qs status {status}: {msg}")
        self.status = status


class qs_opts(ctypes.Structure):
    _fields_ = [("merge_run", ctypes.c_int), ("t_ratio", ctypes.c_double),
                ("low_bits", ctypes.c_int), ("reloc_share", ctypes.c_double),
                ("diag_max", ctypes.c_int), ("threads", ctypes.c_int),
                ("peak_gbs", ctypes.c_double), ("tc_precision", ctypes.c_int),
                ("test_wait_timeout", ctypes.c_int), ("tile_bits", ctypes.c_int),
                ("tile_k", ctypes.c_int), ("fuse_lookahead", ctypes.c_int),
                ("no_shuffles", ctypes.c_int), ("tc_exchange", ctypes.c_int), ("tc_max_ctas", ctypes.c_int),
                ("n_global", ctypes.c_int)]


class qs_class_table(ctypes.Structure):
    _fields_ = [("bytes", ctypes.c_double * QS_N_CLASSES), ("ms", ctypes.c_double * QS_N_CLASSES),
                ("count", ctypes.c_int64 * QS_N_CLASSES)]


class qs_batch_info_t(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("fuse_k", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("total_blocks", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("n_tuned", ctypes.c_int32), ("tuned_k", ctypes.c_int32 * 16),
                ("tuned_threads", ctypes.c_int32 * 16), ("tuned_ms", ctypes.c_double * 16)]


class qs_block_record(ctypes.Structure):
    _fields_ = [("index", ctypes.c_int32), ("kind", ctypes.c_uint8), ("k", ctypes.c_uint8),
                ("nctrl", ctypes.c_uint8), ("tc", ctypes.c_uint8),
                ("qubits", ctypes.c_int8 * QS_MAX_DIAG), ("meta", ctypes.c_uint8),
                ("op", ctypes.c_uint8), ("n_gates", ctypes.c_int32), ("cmask", ctypes.c_uint64),
                ("bytes", ctypes.c_double),
                ("t_start_ms", ctypes.c_double), ("ms", ctypes.c_double),
                ("tiles", ctypes.c_int64), ("ctas", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class qs_exchange_layout(ctypes.Structure):
    _fields_ = [("applies", ctypes.c_int32), ("lane_bits", ctypes.c_int32 * 5), ("reg_bits", ctypes.c_int32 * 4),
                ("la", ctypes.c_int32), ("nswb", ctypes.c_int32), ("lb", ctypes.c_int32 * 2),
                ("slot_target", ctypes.c_int32 * 6), ("part_bits", ctypes.c_int32 * 2)]


class qs_profile_summary(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_blocks", ctypes.c_int32),
                ("gates_seen", ctypes.c_int64), ("gates_last", ctypes.c_int32),
                ("swaps_absorbed", ctypes.c_int32), ("flags_used", ctypes.c_uint64),
                ("counters", (ctypes.c_int64 * QS_N_GATE_TYPES) * QS_MAX_QUBITS),
                ("max_1q_run", ctypes.c_int32 * QS_MAX_QUBITS),
                ("total_ms", ctypes.c_double), ("total_bytes", ctypes.c_double),
                ("h2d_bytes", ctypes.c_double)]


def library_path():
    return _build.LIB


def load(build_if_missing=False):
    """Loads libqs.so; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libqs.so is not built ({path}); run paper_2410_09326_gb300/build.py")
    lib = ctypes.CDLL(path)
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    sigs = {
        "qs_default_opts": (None, [ctypes.POINTER(qs_opts)]),
        "qs_alloc_state": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]),
        "qs_attach_state": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]),
        "qs_free_state": (None, [vp]),
        "qs_set_basis": (ctypes.c_int, [vp, ctypes.c_uint64]),
        "qs_parse_qasm": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int), vp, sz,
                                         ctypes.POINTER(sz)]),
        "qs_apply_circuit": (ctypes.c_int, [vp, vp, sz, ctypes.c_uint64, ctypes.POINTER(qs_opts)]),
        "qs_profile": (ctypes.c_int, [vp, ctypes.POINTER(qs_profile_summary),
                                      ctypes.POINTER(qs_block_record), sz, ctypes.POINTER(sz)]),
        "qs_profile_reset": (ctypes.c_int, [vp]),
        "qs_profile_classes": (ctypes.c_int, [vp, ctypes.POINTER(qs_class_table)]),
        "qs_pgo_select": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, sz, ctypes.POINTER(qs_class_table),
                                         ctypes.POINTER(qs_opts), ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(ctypes.c_double)]),
        "qs_pgo_predict": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, sz, ctypes.c_uint64,
                                          ctypes.POINTER(qs_class_table), ctypes.POINTER(qs_opts),
                                          ctypes.POINTER(ctypes.c_double)]),
        "qs_get_perm": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int8)]),
        "qs_measure_probs": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_double)]),
        "qs_norm": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double)]),
        "qs_read_state": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "qs_write_state": (ctypes.c_int, [vp, vp]),
        "qs_state_distance": (ctypes.c_int, [vp, vp, ctypes.POINTER(ctypes.c_double)]),
        "qs_fold_rotations": (ctypes.c_int, [ctypes.c_int, vp, sz, vp, sz, ctypes.POINTER(sz)]),
        "qs_device_ptr": (ctypes.c_int, [vp, ctypes.POINTER(vp)]),
        "qs_last_error": (ctypes.c_char_p, []),
        "qs_block_features": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(qs_block_record), sz,
                                             ctypes.POINTER(ctypes.c_float)]),
        "qs_mlp_create": (ctypes.c_int, [ctypes.c_uint64, vp, ctypes.POINTER(vp)]),
        "qs_mlp_free": (None, [vp]),
        "qs_mlp_params": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
        "qs_mlp_gradient": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                           ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                           ctypes.POINTER(ctypes.c_float)]),
        "qs_mlp_train": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_float)]),
        "qs_mlp_predict": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_float)]),
        "qs_pgo_select_mlp": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, sz, ctypes.POINTER(qs_opts),
                                             ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)]),
        "qs_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(sz),
                                           ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(qs_opts), vp,
                                           ctypes.POINTER(vp)]),
        "qs_batch_run": (ctypes.c_int, [vp]),
        "qs_batch_sync": (ctypes.c_int, [vp]),
        "qs_batch_info": (ctypes.c_int, [vp, ctypes.POINTER(qs_batch_info_t)]),
        "qs_batch_free": (None, [vp]),
        "qs_apply_batch": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(sz),
                                          ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(qs_opts)]),
        "qs_probs_noalloc": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                            ctypes.c_int, vp, vp]),
        "qs_set_memory_limit": (None, [ctypes.c_uint64]),
        "qs_memory_in_use": (ctypes.c_uint64, []),
        "qs_tc_exchange_layout": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                 ctypes.c_uint64, ctypes.POINTER(qs_exchange_layout)]),
        "qs_plan": (ctypes.c_int, [ctypes.c_int, vp, sz, ctypes.c_uint64, ctypes.POINTER(qs_opts),
                                   ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(qs_block_record), sz,
                                   ctypes.POINTER(sz), ctypes.POINTER(ctypes.c_double), sz,
                                   ctypes.POINTER(sz)]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != QS_OK:
        raise QsError(status, _lib.qs_last_error().decode(errors="replace"))


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def qs_default_opts():
    o = qs_opts()
    load().qs_default_opts(ctypes.byref(o))
    return o


def qs_alloc_state(n, dtype=QS_C64, stream=None):
    h = ctypes.c_void_p()
    _check(load().qs_alloc_state(n, dtype, _stream_handle(stream), ctypes.byref(h)))
    return h


def qs_attach_state(dev_ptr, n, dtype=QS_C64, stream=None):
    h = ctypes.c_void_p()
    _check(load().qs_attach_state(ctypes.c_void_p(dev_ptr), n, dtype, _stream_handle(stream),
                                  ctypes.byref(h)))
    return h


def qs_free_state(st):
    load().qs_free_state(st)


def qs_set_basis(st, x):
    _check(load().qs_set_basis(st, x))


def qs_parse_qasm(text):
    """Returns (n_qubits, gates) with gates a GATE_DTYPE array."""
    lib = load()
    raw = text.encode() if isinstance(text, str) else text
    n = ctypes.c_int(0)
    cnt = ctypes.c_size_t(0)
    st = lib.qs_parse_qasm(raw, ctypes.byref(n), None, 0, ctypes.byref(cnt))
    if st != QS_OK and cnt.value == 0:
        _check(st)
    gates = np.zeros(cnt.value, dtype=GATE_DTYPE)
    _check(lib.qs_parse_qasm(raw, ctypes.byref(n), gates.ctypes.data_as(ctypes.c_void_p),
                             cnt.value, ctypes.byref(cnt)))
    return n.value, gates


def qs_apply_circuit(st, gates, flags=QS_PLAIN, opts=None):
    gates = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    _check(load().qs_apply_circuit(st, gates.ctypes.data_as(ctypes.c_void_p), gates.size, flags,
                                   ctypes.byref(opts) if opts is not None else None))


def qs_profile(st, with_records=True):
    """Returns (summary, list of block records)."""
    lib = load()
    s = qs_profile_summary()
    n = ctypes.c_size_t(0)
    _check(lib.qs_profile(st, ctypes.byref(s), None, 0, ctypes.byref(n)))
    recs = []
    if with_records and n.value:
        arr = (qs_block_record * n.value)()
        _check(lib.qs_profile(st, ctypes.byref(s), arr, n.value, ctypes.byref(n)))
        recs = list(arr)
    return s, recs


def qs_profile_classes(st):
    t = qs_class_table()
    _check(load().qs_profile_classes(st, ctypes.byref(t)))
    return t


def qs_pgo_select(n, gates, dtype=QS_C64, table=None, opts=None):
    """Host-only measured-profile activator: returns (flags, predicted_ms)."""
    gates = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    f = ctypes.c_uint64(0)
    ms = ctypes.c_double(0)
    _check(load().qs_pgo_select(n, dtype, gates.ctypes.data_as(ctypes.c_void_p), gates.size,
                                ctypes.byref(table) if table is not None else None,
                                ctypes.byref(opts) if opts is not None else None, ctypes.byref(f),
                                ctypes.byref(ms)))
    return f.value, ms.value


def qs_pgo_predict(n, gates, flags, dtype=QS_C64, table=None, opts=None):
    """Host-only plan-time prediction (ms) of one flag set from a class table
    (None: the compiled-in priors)."""
    gates = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    ms = ctypes.c_double(0)
    _check(load().qs_pgo_predict(n, dtype, gates.ctypes.data_as(ctypes.c_void_p), gates.size, flags,
                                 ctypes.byref(table) if table is not None else None,
                                 ctypes.byref(opts) if opts is not None else None, ctypes.byref(ms)))
    return ms.value


def qs_profile_reset(st):
    _check(load().qs_profile_reset(st))


def qs_get_perm(st, n):
    out = (ctypes.c_int8 * n)()
    _check(load().qs_get_perm(st, out))
    return np.array(list(out), dtype=np.int64)


def qs_measure_probs(st, logical_qubits):
    q = np.ascontiguousarray(logical_qubits, dtype=np.int32)
    out = np.empty(1 << len(q), dtype=np.float64)
    _check(load().qs_measure_probs(st, q.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(q),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def qs_probs_noalloc(dev_amps, n, dtype, phys_bits, dev_out, stream=None):
    """No-allocation marginal probabilities on raw device pointers (asynchronous;
    dev_out must hold 2^len(phys_bits) doubles on the device)."""
    q = np.ascontiguousarray(phys_bits, dtype=np.int32)
    _check(load().qs_probs_noalloc(ctypes.c_void_p(dev_amps), n, dtype,
                                   q.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(q),
                                   ctypes.c_void_p(dev_out), _stream_handle(stream)))


def qs_norm(st):
    out = ctypes.c_double(0)
    _check(load().qs_norm(st, ctypes.byref(out)))
    return out.value


def qs_read_state(st, n, dtype=QS_C64, logical_order=False, out=None):
    npdt = np.complex64 if dtype == QS_C64 else np.complex128
    if out is None:
        out = np.empty(1 << n, dtype=npdt)
    _check(load().qs_read_state(st, out.ctypes.data_as(ctypes.c_void_p), 1 if logical_order else 0))
    return out


def qs_fold_rotations(n, gates):
    """Rotation folding + pair cancellation (host only): returns the new gate array."""
    gates = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    cap = gates.size + 2
    out = np.zeros(cap, dtype=GATE_DTYPE)
    cnt = ctypes.c_size_t(0)
    _check(load().qs_fold_rotations(n, gates.ctypes.data_as(ctypes.c_void_p), gates.size,
                                    out.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(cnt)))
    return out[: cnt.value].copy()


def array_to_gates(arr):
    """GATE_DTYPE array -> (name, qubits, params) tuples (for printing as text)."""
    out = []
    for a in arr:
        name = OPS[a["op"]]
        nq = int(a["nq"])
        npar = {"rx": 1, "ry": 1, "rz": 1, "cp": 1, "cu1": 1, "crx": 1, "cry": 1, "crz": 1, "u1": 1,
                "rzz": 1, "rxx": 1, "ryy": 1, "u2": 2, "u3": 3, "cu3": 3}.get(name, 0)
        out.append((name, [int(x) for x in a["q"][:nq]], [float(x) for x in a["p"][:npar]]))
    return out


def qs_state_distance(a, b):
    out = ctypes.c_double(0)
    _check(load().qs_state_distance(a, b, ctypes.byref(out)))
    return out.value


def qs_write_state(st, host):
    host = np.ascontiguousarray(host)
    _check(load().qs_write_state(st, host.ctypes.data_as(ctypes.c_void_p)))


def qs_device_ptr(st):
    p = ctypes.c_void_p()
    _check(load().qs_device_ptr(st, ctypes.byref(p)))
    return p.value


def qs_set_memory_limit(nbytes):
    """Device-memory budget for the library's own allocations (0 = none)."""
    load().qs_set_memory_limit(int(nbytes))


def qs_memory_in_use():
    """The library's live device bytes."""
    return int(load().qs_memory_in_use())


def qs_tc_exchange_layout(n, targets, cmask=0):
    """The lane-exchange layout of a tensor-core block (qs_exchange_layout)."""
    t = (ctypes.c_int * len(targets))(*[int(x) for x in targets])
    out = qs_exchange_layout()
    _check(load().qs_tc_exchange_layout(n, len(targets), t, cmask, ctypes.byref(out)))
    return out


def qs_plan(n, gates, flags=QS_PLAIN, opts=None, perm=None):
    """Host passes only. Returns (records, matrices, perm): matrices[i] is the
    block's complex128 matrix ((2^k, 2^k) dense, (2^k,) diagonal, None exchange
    or tile pass) or, for a phase polynomial, a dict of its qubits, linear
    angles a, constant c and pair angles b (upper triangle)."""
    lib = load()
    gates = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    pm = (ctypes.c_int8 * n)(*(range(n) if perm is None else [int(x) for x in perm]))
    nb = ctypes.c_size_t(0)
    ml = ctypes.c_size_t(0)
    args = lambda recs, cap, mats, mcap: (n, gates.ctypes.data_as(ctypes.c_void_p), gates.size, flags,
                                          ctypes.byref(opts) if opts is not None else None, pm, recs,
                                          cap, ctypes.byref(nb), mats, mcap, ctypes.byref(ml))
    perm0 = (ctypes.c_int8 * n)(*pm)
    _check(lib.qs_plan(*args(None, 0, None, 0)))
    ctypes.memmove(pm, perm0, n)
    recs = (qs_block_record * max(1, nb.value))()
    mats = np.zeros(2 * max(1, ml.value), dtype=np.float64)
    _check(lib.qs_plan(*args(recs, nb.value, mats.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             ml.value)))
    cm = mats.view(np.complex128)
    out, off = [], 0
    for r in list(recs)[: nb.value]:
        if r.kind == 0:
            d = 1 << r.k
            out.append(cm[off: off + d * d].reshape(d, d).copy())
            off += d * d
        elif r.kind == 1:
            d = 1 << r.k
            out.append(cm[off: off + d].copy())
            off += d
        elif r.kind == 4:
            k = r.k
            qa = cm[off: off + k]
            c = cm[off + k].real
            b = np.zeros((k, k))
            iu = np.triu_indices(k, 1)
            b[iu] = cm[off + k + 1: off + k + 1 + len(iu[0])].real
            out.append({"qubits": qa.real.astype(np.int64), "a": qa.imag.copy(), "c": c, "b": b})
            off += k + 1 + len(iu[0])
        else:
            out.append(None)
    return list(recs)[: nb.value], out, np.array(list(pm), dtype=np.int64)


def qs_batch_create(states, gate_arrays, flags=0, opts=None, stream=None):
    """states: list of state handles; gate_arrays: list of GATE_DTYPE arrays."""
    lib = load()
    count = len(states)
    arrs = [np.ascontiguousarray(g, dtype=GATE_DTYPE) for g in gate_arrays]
    st = (ctypes.c_void_p * count)(*[s.value for s in states])
    gp = (ctypes.c_void_p * count)(*[a.ctypes.data for a in arrs])
    ng = (ctypes.c_size_t * count)(*[a.size for a in arrs])
    h = ctypes.c_void_p()
    _check(lib.qs_batch_create(st, gp, ng, count, flags, ctypes.byref(opts) if opts is not None else None,
                               _stream_handle(stream), ctypes.byref(h)))
    h._keep = arrs  # the library copies the gates; keep the arrays alive for the call only
    return h


def qs_apply_batch(states, gate_arrays, flags=0, opts=None):
    """One-shot batch: every state set to |0...0> and its circuit applied in
    one persistent launch; returns when the results are in the states."""
    count = len(states)
    arrs = [np.ascontiguousarray(g, dtype=GATE_DTYPE) for g in gate_arrays]
    st = (ctypes.c_void_p * count)(*[s.value for s in states])
    gp = (ctypes.c_void_p * count)(*[a.ctypes.data for a in arrs])
    ng = (ctypes.c_size_t * count)(*[a.size for a in arrs])
    _check(load().qs_apply_batch(st, gp, ng, count, flags, ctypes.byref(opts) if opts is not None else None))


def qs_batch_run(b):
    _check(load().qs_batch_run(b))


def qs_batch_sync(b):
    _check(load().qs_batch_sync(b))


def qs_batch_info(b):
    info = qs_batch_info_t()
    _check(load().qs_batch_info(b, ctypes.byref(info)))
    return info


def qs_batch_free(b):
    load().qs_batch_free(b)


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def qs_block_features(n, recs, dtype=QS_C64):
    """Feature rows (len(recs) x QS_MLP_FEATURES float32) of block records."""
    arr = (qs_block_record * max(1, len(recs)))(*recs)
    out = np.zeros((len(recs), QS_MLP_FEATURES), dtype=np.float32)
    _check(load().qs_block_features(n, dtype, arr, len(recs), _fptr(out)))
    return out


def qs_mlp_create(seed=0, stream=None):
    h = ctypes.c_void_p()
    _check(load().qs_mlp_create(seed, _stream_handle(stream), ctypes.byref(h)))
    return h


def qs_mlp_free(m):
    load().qs_mlp_free(m)


def qs_mlp_params(m, new=None):
    """Returns the flat FP32 parameters; writes `new` first when given."""
    out = np.zeros(QS_MLP_PARAMS, dtype=np.float32)
    src = None
    if new is not None:
        src = np.ascontiguousarray(new, dtype=np.float32)
        assert src.size == QS_MLP_PARAMS
    _check(load().qs_mlp_params(m, _fptr(out), _fptr(src) if src is not None else None))
    return out


def qs_mlp_gradient(m, x, y):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    g = np.zeros(QS_MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_float(0)
    _check(load().qs_mlp_gradient(m, _fptr(x), _fptr(y), len(y), _fptr(g), ctypes.byref(loss)))
    return g, loss.value


def qs_mlp_train(m, x, y, epochs=30, batch=256, lr=1e-3, seed=0):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    loss = ctypes.c_float(0)
    _check(load().qs_mlp_train(m, _fptr(x), _fptr(y), len(y), epochs, batch, lr, seed, ctypes.byref(loss)))
    return loss.value


def qs_mlp_predict(m, x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.zeros(len(x), dtype=np.float32)
    _check(load().qs_mlp_predict(m, _fptr(x), len(x), _fptr(y)))
    return y


def qs_pgo_select_mlp(m, n, gates, dtype=QS_C64, opts=None):
    gates = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    f = ctypes.c_uint64(0)
    ms = ctypes.c_double(0)
    _check(load().qs_pgo_select_mlp(m, n, dtype, gates.ctypes.data_as(ctypes.c_void_p), gates.size,
                                    ctypes.byref(opts) if opts is not None else None, ctypes.byref(f),
                                    ctypes.byref(ms)))
    return f.value, ms.value


def gates_to_array(gates):
    """(name, qubits, params) tuples -> GATE_DTYPE array (no parsing of text)."""
    arr = np.zeros(len(gates), dtype=GATE_DTYPE)
    for i, g in enumerate(gates):
        name, qs = g[0], g[1]
        ps = g[2] if len(g) > 2 else ()
        arr[i]["op"] = OPS.index(name)
        arr[i]["nq"] = len(qs)
        arr[i]["q"][: len(qs)] = qs
        arr[i]["p"][: len(ps)] = ps
    return arr
