"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package. The CUDA library never loads it and the
two share no code (the oracle has its own parser and gate table, in
`oracle.c`).

`simulate` is the plain definition of full-state simulation (Sec. II-B): the
state is updated gate by gate in the circuit's order in complex128, SWAPs are
real amplitude exchanges, and the SWAP transpositions are composed into the
logical->physical map that the virtual-swap pass (Sec. III-D) must report.
"""

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force=False):
    """Compiles oracle.c with gcc + OpenMP into _build/liboracle.so."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_simulate.argtypes = [ctypes.c_char_p, ctypes.c_int, dp, dp, ip, ctypes.c_int]
        lib.oracle_count.argtypes = [ctypes.c_char_p, ip, ip]
        lib.oracle_gate_matrix.argtypes = [ctypes.c_char_p, dp, dp, ip, ip]
        lib.oracle_probs.argtypes = [dp, ctypes.c_int, ip, ctypes.c_int, dp]
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def count(text):
    """(n_qubits, n_gates) of a circuit text; raises ValueError on a parse error."""
    lib = _load()
    n = ctypes.c_int(0)
    g = ctypes.c_int(0)
    rc = lib.oracle_count(text.encode(), ctypes.byref(n), ctypes.byref(g))
    if rc:
        raise ValueError(f"oracle parse error (code {rc})")
    return n.value, g.value


def simulate(text, init=None, nthreads=0):
    """Returns (state complex128 in logical order, perm int array).

    init: optional complex128 initial state (default |0...0>).
    perm[l] = physical bit that holds logical qubit l once every SWAP is
    absorbed as a relabelling.
    """
    lib = _load()
    n, _ = count(text)
    out = np.empty(1 << n, dtype=np.complex128)
    perm = np.empty(n, dtype=np.int32)
    ip = None
    if init is not None:
        init = np.ascontiguousarray(init, dtype=np.complex128)
        if init.shape != (1 << n,):
            raise ValueError("init has the wrong size")
        ip = _dptr(init.view(np.float64))
    rc = lib.oracle_simulate(text.encode(), n, ip, _dptr(out.view(np.float64)), _iptr(perm), nthreads)
    if rc:
        raise ValueError(f"oracle error (code {rc})")
    return out, perm


def gate_matrix(name, params=()):
    """(U, n_controls, n_targets) for one named gate; U acts on the targets."""
    lib = _load()
    p = np.zeros(3, dtype=np.float64)
    p[: len(params)] = params
    out = np.zeros(32, dtype=np.float64)
    nc = ctypes.c_int(0)
    nt = ctypes.c_int(0)
    if lib.oracle_gate_matrix(name.encode(), _dptr(p), _dptr(out), ctypes.byref(nc), ctypes.byref(nt)):
        raise ValueError(f"unknown gate {name}")
    d = 1 << nt.value
    u = out[: 2 * d * d].view(np.complex128).reshape(d, d).copy()
    return u, nc.value, nt.value


def probs(state, qubits):
    """Marginal probabilities of the listed qubits (bit j of the bin = qubits[j])."""
    lib = _load()
    state = np.ascontiguousarray(state, dtype=np.complex128)
    n = int(np.log2(state.size))
    q = np.asarray(qubits, dtype=np.int32)
    out = np.empty(1 << len(q), dtype=np.float64)
    lib.oracle_probs(_dptr(state.view(np.float64)), n, _iptr(q), len(q), _dptr(out))
    return out


def max_threads():
    return _load().oracle_max_threads()


def to_physical(state_logical, perm):
    """Places a logical-order state in physical order: phys[P(i)] = logical[i],
    P(i) = sum_l bit_l(i) << perm[l]."""
    n = len(perm)
    idx = np.arange(1 << n, dtype=np.int64)
    p = np.zeros_like(idx)
    for l in range(n):
        p |= ((idx >> l) & 1) << int(perm[l])
    out = np.empty_like(state_logical)
    out[p] = state_logical
    return out
