"""MTGP32 oracle -- TEST INFRASTRUCTURE ONLY.

Python access (ctypes + NumPy) to the plain sequential C oracle in
``mtgp_oracle.c``.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_1501_07701_gb300``) never does and shares no code with it.

What each function follows in the paper (Passerat-Palmbach et al., ESM 2010):

* ``params_generate`` / ``params_from_fields`` -- the parameterized status of
  Sec. 3.1 (the generator's signature, with the precomputed tables of a
  "fast" status).  The paper prints no parameter set, so sets are
  seed-generated (SplitMix64) or given field by field.
* ``init_state`` -- the seed status of Sec. 3.1 / Sec. 5.1, expanded by the
  MT-family seeding recurrence.  Parity against the MTGP release's own seeding
  is unpinned (its extra parameter-derived fill is omitted on purpose).
* ``generate`` / ``generate_many`` -- the generator of Sec. 2 / Sec. 3.2, one
  independent status per stream.

Pins: ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mtgp_oracle.c")
_LIB = os.path.join(_HERE, "libmtgp_oracle.so")
_lock = threading.Lock()
_lib = None

U32, F32_12, F32_01 = 0, 1, 2


class Params(ctypes.Structure):
    _fields_ = [
        ("mexp", ctypes.c_uint32),
        ("n", ctypes.c_uint32),
        ("pos", ctypes.c_uint32),
        ("sh1", ctypes.c_uint32),
        ("sh2", ctypes.c_uint32),
        ("mask", ctypes.c_uint32),
        ("rec_basis", ctypes.c_uint32 * 4),
        ("tmp_basis", ctypes.c_uint32 * 4),
        ("rec_tbl", ctypes.c_uint32 * 16),
        ("tmp_tbl", ctypes.c_uint32 * 16),
    ]

    def as_dict(self) -> dict:
        return {
            "mexp": self.mexp, "n": self.n, "pos": self.pos, "sh1": self.sh1,
            "sh2": self.sh2, "mask": self.mask,
            "rec_basis": list(self.rec_basis), "tmp_basis": list(self.tmp_basis),
            "rec_tbl": list(self.rec_tbl), "tmp_tbl": list(self.tmp_tbl),
        }


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, -O2, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mtgp_oracle.h"))):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC,
                               "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # MTGP_ORACLE_LIB loads a prebuilt variant instead (used by the
            # mutation test to check that the pins reject planted mistakes).
            path = os.environ.get("MTGP_ORACLE_LIB")
            if not path:
                path = build()
            lib = ctypes.CDLL(path)
            P = ctypes.POINTER(Params)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.omtgp_params_complete.argtypes = [P]
            lib.omtgp_params_generate.argtypes = [ctypes.c_uint32, ctypes.c_uint64, P]
            lib.omtgp_init_state.argtypes = [P, ctypes.c_uint32, u32p]
            lib.omtgp_init_state.restype = None
            lib.omtgp_generate.argtypes = [P, u32p, ctypes.c_uint64, ctypes.c_int, u32p]
            lib.omtgp_generate_many.argtypes = [P, u32p, ctypes.c_uint32, u32p, u64p,
                                                ctypes.c_uint32, ctypes.c_int, u32p, ctypes.c_int]
            lib.omtgp_gap_histogram.argtypes = [u32p, ctypes.c_uint64, ctypes.c_uint, ctypes.c_uint,
                                                ctypes.c_uint, u64p]
            lib.omtgp_hamming_pairs.argtypes = [u32p, ctypes.c_uint64, ctypes.c_uint, ctypes.c_uint,
                                                ctypes.c_uint, u32p, ctypes.c_uint, u64p]
            _lib = lib
    return _lib


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _u64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def params_generate(mexp: int, seed: int) -> Params:
    p = Params()
    if _load().omtgp_params_generate(mexp, seed, ctypes.byref(p)) != 0:
        raise ValueError("oracle: unusable Mexp %d" % mexp)
    return p


def params_from_fields(mexp, pos, sh1, sh2, rec_basis, tmp_basis, n=0, mask=0) -> Params:
    p = Params()
    p.mexp, p.n, p.pos, p.sh1, p.sh2, p.mask = mexp, n, pos, sh1, sh2, mask
    for b in range(4):
        p.rec_basis[b] = rec_basis[b] & 0xFFFFFFFF
        p.tmp_basis[b] = tmp_basis[b] & 0xFFFFFFFF
    if _load().omtgp_params_complete(ctypes.byref(p)) != 0:
        raise ValueError("oracle: parameter fields out of range")
    return p


def init_state(p: Params, seed: int) -> np.ndarray:
    st = np.zeros(p.n, dtype=np.uint32)
    _load().omtgp_init_state(ctypes.byref(p), seed & 0xFFFFFFFF, _u32p(st))
    return st


def generate(p: Params, state: np.ndarray, count: int, fmt: int = U32):
    """Returns (outputs as uint32 bit patterns, advanced state)."""
    st = np.ascontiguousarray(state, dtype=np.uint32).copy()
    assert st.shape == (p.n,)
    out = np.zeros(max(count, 1), dtype=np.uint32)
    if _load().omtgp_generate(ctypes.byref(p), _u32p(st), count, fmt, _u32p(out)) != 0:
        raise RuntimeError("oracle: generate failed")
    return out[:count], st


def generate_many(p: Params, states: np.ndarray, ids, counts, fmt: int = U32,
                  n_threads: int = 1):
    """Requests (ids[j], counts[j]) in order; returns (out, advanced states)."""
    st = np.ascontiguousarray(states, dtype=np.uint32).copy()
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    total = int(counts.sum()) if counts.size else 0
    out = np.zeros(max(total, 1), dtype=np.uint32)
    rc = _load().omtgp_generate_many(ctypes.byref(p), _u32p(st), st.shape[0], _u32p(ids),
                                     _u64p(counts), ids.size, fmt, _u32p(out), n_threads)
    if rc != 0:
        raise RuntimeError("oracle: generate_many failed")
    return out[:total], st


def gap_histogram(x, r: int = 25, b: int = 5, t: int = 128) -> np.ndarray:
    """Gap-length histogram (Sec. 4.2, test 35): t + 1 counts."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    hist = np.zeros(t + 1, dtype=np.uint64)
    if _load().omtgp_gap_histogram(_u32p(x), x.size, r, b, t, _u64p(hist)) != 0:
        raise ValueError("oracle: bad gap-test arguments")
    return hist


def hamming_pairs(x, r: int = 25, s: int = 5, L: int = 1200, bounds=()) -> np.ndarray:
    """Table of weight classes of successive block pairs (Sec. 4.2, test 100):
    C x C counts, C = len(bounds) + 1."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    bnd = np.ascontiguousarray(bounds, dtype=np.uint32)
    C = bnd.size + 1
    table = np.zeros(C * C, dtype=np.uint64)
    if _load().omtgp_hamming_pairs(_u32p(x), x.size, r, s, L, _u32p(bnd), bnd.size,
                                   _u64p(table)) != 0:
        raise ValueError("oracle: bad Hamming-test arguments")
    return table.reshape(C, C)
