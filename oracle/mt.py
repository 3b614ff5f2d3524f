"""Original Mersenne Twister oracle -- TEST INFRASTRUCTURE ONLY.

ctypes access to the plain sequential C oracle in ``mt_oracle.c``: the
comparison generator of the paper's Sec. 5.3 (the original MT of Matsumoto
and Nishimura 1998, run at the same period as MTGP through tests 35 and 100).
Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product path never does and shares no code
with it.

* ``params_mt19937`` -- the parameter set printed in the 1998 paper.
* ``params_generate`` -- a seed-generated set for another exponent (the
  paper's sets came from MT's dynamic creator, which is not rebuilt).
* ``init_state`` / ``generate`` / ``generate_many`` -- the generator.

Pins: ``tests/test_mt_oracle.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mt_oracle.c")
_HDR = os.path.join(_HERE, "mt_oracle.h")
_LIB = os.path.join(_HERE, "libmt_oracle.so")
_lock = threading.Lock()
_lib = None

U32, F32_12, F32_01 = 0, 1, 2
FIELDS = ("p", "n", "m", "r", "a", "u", "s", "t", "l", "b", "c")


class MtParams(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint32) for f in FIELDS]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f in FIELDS}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, -O2, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(_HDR)):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC,
                               "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # MT_ORACLE_LIB loads a prebuilt variant instead (used by the
            # mutation test to check that the pins reject planted mistakes).
            lib = ctypes.CDLL(os.environ.get("MT_ORACLE_LIB") or build())
            P = ctypes.POINTER(MtParams)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.omt_params_complete.argtypes = [P]
            lib.omt_params_mt19937.argtypes = [P]
            lib.omt_params_mt19937.restype = None
            lib.omt_params_generate.argtypes = [ctypes.c_uint32, ctypes.c_uint64, P]
            lib.omt_init_state.argtypes = [P, ctypes.c_uint32, u32p]
            lib.omt_init_state.restype = None
            lib.omt_generate.argtypes = [P, u32p, ctypes.c_uint64, ctypes.c_int, u32p]
            lib.omt_generate_many.argtypes = [P, u32p, ctypes.c_uint32, u32p, u64p,
                                              ctypes.c_uint32, ctypes.c_int, u32p, ctypes.c_int]
            _lib = lib
    return _lib


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def params_mt19937() -> MtParams:
    q = MtParams()
    _load().omt_params_mt19937(ctypes.byref(q))
    return q


def params_generate(p: int, seed: int) -> MtParams:
    q = MtParams()
    if _load().omt_params_generate(p, seed, ctypes.byref(q)) != 0:
        raise ValueError("oracle: unusable exponent %d" % p)
    return q


def params_from_fields(**fields) -> MtParams:
    """Any subset of FIELDS; n = 0 derives n and r from p."""
    q = MtParams()
    for f, v in fields.items():
        setattr(q, f, int(v) & 0xFFFFFFFF)
    if _load().omt_params_complete(ctypes.byref(q)) != 0:
        raise ValueError("oracle: parameter fields out of range")
    return q


def init_state(q: MtParams, seed: int) -> np.ndarray:
    st = np.zeros(q.n, dtype=np.uint32)
    _load().omt_init_state(ctypes.byref(q), seed & 0xFFFFFFFF, _u32p(st))
    return st


def generate(q: MtParams, state: np.ndarray, count: int, fmt: int = U32):
    """Returns (outputs as uint32 bit patterns, advanced state)."""
    st = np.ascontiguousarray(state, dtype=np.uint32).copy()
    assert st.shape == (q.n,)
    out = np.zeros(max(count, 1), dtype=np.uint32)
    if _load().omt_generate(ctypes.byref(q), _u32p(st), count, fmt, _u32p(out)) != 0:
        raise RuntimeError("oracle: generate failed")
    return out[:count], st


def generate_many(q: MtParams, states: np.ndarray, ids, counts, fmt: int = U32,
                  n_threads: int = 1):
    """Requests (ids[j], counts[j]) in order; returns (out, advanced states)."""
    st = np.ascontiguousarray(states, dtype=np.uint32).copy()
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    total = int(counts.sum()) if counts.size else 0
    out = np.zeros(max(total, 1), dtype=np.uint32)
    rc = _load().omt_generate_many(ctypes.byref(q), _u32p(st), st.shape[0], _u32p(ids),
                                   counts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                   ids.size, fmt, _u32p(out), n_threads)
    if rc != 0:
        raise RuntimeError("oracle: generate_many failed")
    return out[:total], st
