"""Python binding of libmtgp (ctypes): argument marshalling only.

Every function keeps the name of the C entry point it calls (include/mtgp.h).
Device buffers are torch CUDA tensors (any 4-byte dtype) or raw integer
pointers; streams are torch.cuda.Stream objects, raw cudaStream_t integers,
or None for torch's current stream.  All generation work runs in the CUDA
kernels of libmtgp.so; if the library is missing this module raises instead
of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmtgp.so")

MTGP_U32, MTGP_F32_12, MTGP_F32_01 = 0, 1, 2
STATUS_NAMES = {0: "MTGP_OK", 1: "MTGP_EINVAL", 2: "MTGP_ENOMEM", 3: "MTGP_ECUDA",
                4: "MTGP_ETIMEOUT", 5: "MTGP_EBUSY", 6: "MTGP_EIO", 7: "MTGP_EDEVICE"}

_lib = None
_lock = threading.Lock()


class MtgpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class ParamsDesc(ctypes.Structure):
    _fields_ = [("mexp", ctypes.c_uint32), ("n", ctypes.c_uint32), ("pos", ctypes.c_uint32),
                ("sh1", ctypes.c_uint32), ("sh2", ctypes.c_uint32), ("mask", ctypes.c_uint32),
                ("rec_tbl", ctypes.c_uint32 * 16), ("tmp_tbl", ctypes.c_uint32 * 16)]


class LaunchConfig(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("words_per_lane", ctypes.c_uint32), ("kernel", ctypes.c_uint32),
                ("coop_percent", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PlanInfo(ctypes.Structure):
    _fields_ = [("total_numbers", ctypes.c_uint64), ("n_items", ctypes.c_uint32),
                ("kernel_launches", ctypes.c_uint32), ("config", LaunchConfig),
                ("grid_ctas", ctypes.c_uint32), ("n_coop", ctypes.c_uint32),
                ("regs_per_thread", ctypes.c_uint32), ("resident_ctas_per_sm", ctypes.c_uint32),
                ("max_piece", ctypes.c_uint64), ("n_split_streams", ctypes.c_uint32),
                ("n_jumps", ctypes.c_uint32), ("n_pieces", ctypes.c_uint32), ("stats", ctypes.c_uint32)]


class StatsConfig(ctypes.Structure):
    """mtgp_stats_config (include/mtgp.h)."""
    _fields_ = [(f, ctypes.c_uint32) for f in ("gap_r", "gap_b", "gap_t", "ham_r", "ham_s", "ham_L",
                                                "n_bounds")] + [("bounds", ctypes.c_uint32 * 15)]


class MtParams(ctypes.Structure):
    """mtgp_mt_params (include/mtgp_mt.h)."""
    _fields_ = [(f, ctypes.c_uint32) for f in ("p", "n", "m", "r", "a", "u", "s", "t", "l", "b", "c")]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("max_tick_requests", ctypes.c_uint32), ("tick_timeout_s", ctypes.c_double),
                ("max_piece", ctypes.c_uint64)]


class Completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("count", ctypes.c_uint64),
                ("arena_offset", ctypes.c_uint64), ("fmt", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("submit_time", ctypes.c_double), ("done_time", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("numbers", ctypes.c_uint64),
                ("ticks", ctypes.c_uint64), ("elapsed", ctypes.c_double),
                ("busy_wait", ctypes.c_double), ("launch_host_s", ctypes.c_double),
                ("jumps", ctypes.c_uint64)]


_VP = ctypes.c_void_p
_U32P = ctypes.POINTER(ctypes.c_uint32)
_U64P = ctypes.POINTER(ctypes.c_uint64)

# name -> argtypes (restype int status unless listed in _STR)
_SIGS = {
    "mtgp_params_load": [ctypes.c_char_p, ctypes.POINTER(_VP)],
    "mtgp_params_generate": [ctypes.c_uint32, ctypes.c_uint64, ctypes.POINTER(_VP)],
    "mtgp_params_create": [ctypes.POINTER(ParamsDesc), ctypes.POINTER(_VP)],
    "mtgp_params_get": [_VP, ctypes.POINTER(ParamsDesc)],
    "mtgp_params_free": [_VP],
    "mtgp_init_statuses": [_VP, _U32P, ctypes.c_uint32, _VP, ctypes.POINTER(_VP)],
    "mtgp_jump": [_VP, _U32P, _U64P, ctypes.c_uint32, _VP],
    "mtgp_params_minpoly": [_VP, _U64P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32)],
    "mtgp_params_period_check": [_VP, _VP, ctypes.POINTER(ctypes.c_int32)],
    "mtgp_gap_histogram": [_VP, _U64P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                           _U64P, _VP],
    "mtgp_hamming_pairs": [_VP, _U64P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                           _U32P, ctypes.c_uint32, _U64P, _VP],
    "mtgp_init_statuses_multi": [ctypes.POINTER(_VP), ctypes.c_uint32, _U32P, _U32P, ctypes.c_uint32,
                                 _VP, ctypes.POINTER(_VP)],
    "mtgp_set_statuses": [_VP, _U32P, _VP],
    "mtgp_get_statuses": [_VP, _U32P, _VP],
    "mtgp_streams_info": [_VP, _U32P, _U32P],
    "mtgp_generate_u32": [_VP, _U32P, _U64P, ctypes.c_uint32, _VP, _VP],
    "mtgp_generate_f32": [_VP, _U32P, _U64P, ctypes.c_uint32, ctypes.c_int, _VP, _VP],
    "mtgp_generate_to_host": [_VP, _U32P, _U64P, ctypes.c_uint32, ctypes.c_int, _VP,
                              ctypes.c_uint64, _VP],
    "mtgp_generate_noalloc": [_VP, _U32P, _U64P, ctypes.c_uint32, ctypes.c_int, _VP, _VP],
    "mtgp_check": [_VP, _VP],
    "mtgp_streams_free": [_VP],
    "mtgp_get_launch_config": [_VP, ctypes.POINTER(LaunchConfig)],
    "mtgp_set_launch_config": [_VP, ctypes.POINTER(LaunchConfig)],
    "mtgp_autotune": [_VP, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                      ctypes.POINTER(LaunchConfig)],
    "mtgp_plan_create": [_VP, _U32P, _U64P, ctypes.c_uint32, ctypes.c_int, _VP,
                         ctypes.POINTER(_VP)],
    "mtgp_plan_launch": [_VP, _VP],
    "mtgp_plan_set_split": [_VP, ctypes.c_uint64],
    "mtgp_plan_set_stats": [_VP, ctypes.POINTER(StatsConfig)],
    "mtgp_plan_read_stats": [_VP, _U64P, _U64P, _VP],
    "mtgp_plan_autotune": [_VP, ctypes.POINTER(LaunchConfig)],
    "mtgp_plan_get_info": [_VP, ctypes.POINTER(PlanInfo)],
    "mtgp_plan_set_trace": [_VP, ctypes.c_int],
    "mtgp_plan_read_trace": [_VP, _U64P],
    "mtgp_plan_free": [_VP],
    "mtgp_server_create": [_VP, ctypes.POINTER(ServerConfig), ctypes.POINTER(_VP)],
    "mtgp_server_submit": [_VP, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64],
    "mtgp_server_progress": [_VP, ctypes.POINTER(Completion), ctypes.c_uint32, _U32P],
    "mtgp_server_release": [_VP, ctypes.c_uint64, ctypes.c_uint64],
    "mtgp_server_arena": [_VP, ctypes.POINTER(_VP)],
    "mtgp_server_read": [_VP, ctypes.c_uint64, ctypes.c_uint64, _VP],
    "mtgp_server_run_trace": [_VP, ctypes.POINTER(ctypes.c_double), _U32P, _U64P,
                              ctypes.POINTER(ctypes.c_int32), ctypes.c_uint32, ctypes.c_uint32,
                              ctypes.POINTER(ctypes.c_double), _U64P, ctypes.POINTER(ServerStats)],
    "mtgp_server_debug_hold": [_VP, ctypes.c_int],
    "mtgp_server_free": [_VP],
    "mtgp_mt_params_mt19937": [ctypes.POINTER(MtParams)],
    "mtgp_mt_params_generate": [ctypes.c_uint32, ctypes.c_uint64, ctypes.POINTER(MtParams)],
    "mtgp_mt_init": [ctypes.POINTER(MtParams), _U32P, ctypes.c_uint32, _VP, ctypes.POINTER(_VP)],
    "mtgp_mt_init_multi": [ctypes.POINTER(MtParams), ctypes.c_uint32, _U32P, _U32P, ctypes.c_uint32,
                           _VP, ctypes.POINTER(_VP)],
    "mtgp_mt_set_statuses": [_VP, _U32P, _VP],
    "mtgp_mt_get_statuses": [_VP, _U32P, _VP],
    "mtgp_mt_generate": [_VP, _U32P, _U64P, ctypes.c_uint32, ctypes.c_int, _VP, _VP],
    "mtgp_mt_check": [_VP, _VP],
    "mtgp_mt_params_minpoly": [ctypes.POINTER(MtParams), _U64P, ctypes.c_uint32,
                               ctypes.POINTER(ctypes.c_int32)],
    "mtgp_mt_params_period_check": [ctypes.POINTER(MtParams), _VP, ctypes.POINTER(ctypes.c_int32)],
    "mtgp_mt_free": [_VP],
    "mtgp_last_error": [],
    "mtgp_version": [],
}
_STR = {"mtgp_last_error", "mtgp_version"}


def load_library(path: str | None = None):
    """Loads libmtgp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError("libmtgp.so not found at %s; build it with "
                                   "paper_1501_07701_gb300.build.build()" % p)
            lib = ctypes.CDLL(p)
            for name, args in _SIGS.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ctypes.c_char_p if name in _STR else ctypes.c_int
            _lib = lib
    return _lib


def _call(name, *args):
    lib = load_library()
    st = getattr(lib, name)(*args)
    if st != 0:
        raise MtgpError(st, lib.mtgp_last_error().decode())


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev_ptr(buf, min_elems: int = 0):
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    import torch
    if not isinstance(buf, torch.Tensor) or not buf.is_cuda:
        raise TypeError("device buffer must be a CUDA tensor or an integer pointer")
    if buf.element_size() != 4 or not buf.is_contiguous():
        raise TypeError("device buffer must be contiguous with 4-byte elements")
    if buf.numel() < min_elems:
        raise ValueError("device buffer holds %d elements, %d needed" % (buf.numel(), min_elems))
    return buf.data_ptr()


def _req_arrays(ids, counts):
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    if ids.shape != counts.shape or ids.ndim != 1:
        raise ValueError("stream_ids and counts must be 1-D arrays of equal length")
    return ids, counts


def _p32(a):
    return a.ctypes.data_as(_U32P)


def _p64(a):
    return a.ctypes.data_as(_U64P)


class Params:
    """Owning wrapper of an mtgp_params_t."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            _call("mtgp_params_free", self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Streams:
    """Owning wrapper of an mtgp_streams_t."""

    def __init__(self, handle):
        self.handle = handle

    @property
    def n_streams(self):
        return mtgp_streams_info(self)[0]

    @property
    def n_words(self):
        return mtgp_streams_info(self)[1]

    def close(self):
        if self.handle:
            _call("mtgp_streams_free", self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owning wrapper of an mtgp_plan_t (keeps its Streams alive)."""

    def __init__(self, handle, streams, out, n_req=0):
        self.handle = handle
        self.streams = streams
        self.out = out
        self.n_req = n_req
        self.stats = None   # (gap t or 0, weight classes C or 0) while statistics are on

    def close(self):
        if self.handle:
            _call("mtgp_plan_free", self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mtgp_version():
    return load_library().mtgp_version().decode()


def mtgp_params_load(path: str) -> Params:
    h = _VP()
    _call("mtgp_params_load", path.encode(), ctypes.byref(h))
    return Params(h)


def mtgp_params_generate(mexp: int, seed: int) -> Params:
    h = _VP()
    _call("mtgp_params_generate", mexp, seed, ctypes.byref(h))
    return Params(h)


def mtgp_params_create(mexp, pos, sh1, sh2, rec_tbl, tmp_tbl, n=0, mask=0) -> Params:
    d = ParamsDesc()
    d.mexp, d.n, d.pos, d.sh1, d.sh2, d.mask = mexp, n, pos, sh1, sh2, mask
    for i in range(16):
        d.rec_tbl[i] = int(rec_tbl[i]) & 0xFFFFFFFF
        d.tmp_tbl[i] = int(tmp_tbl[i]) & 0xFFFFFFFF
    h = _VP()
    _call("mtgp_params_create", ctypes.byref(d), ctypes.byref(h))
    return Params(h)


def mtgp_params_get(params: Params) -> dict:
    d = ParamsDesc()
    _call("mtgp_params_get", params.handle, ctypes.byref(d))
    return {"mexp": d.mexp, "n": d.n, "pos": d.pos, "sh1": d.sh1, "sh2": d.sh2, "mask": d.mask,
            "rec_tbl": list(d.rec_tbl), "tmp_tbl": list(d.tmp_tbl)}


def mtgp_init_statuses(params: Params, seeds, stream=None) -> Streams:
    seeds = np.ascontiguousarray(seeds, dtype=np.uint32)
    h = _VP()
    _call("mtgp_init_statuses", params.handle, _p32(seeds), seeds.size, _stream_handle(stream),
          ctypes.byref(h))
    return Streams(h)


def mtgp_init_statuses_multi(params_list, set_of_stream, seeds, stream=None) -> Streams:
    """One parameter set per stream: stream s uses params_list[set_of_stream[s]]."""
    seeds = np.ascontiguousarray(seeds, dtype=np.uint32)
    set_of = np.ascontiguousarray(set_of_stream, dtype=np.uint32)
    if set_of.shape != seeds.shape:
        raise ValueError("set_of_stream and seeds must have the same length")
    arr = (_VP * len(params_list))(*[p.handle for p in params_list])
    h = _VP()
    _call("mtgp_init_statuses_multi", arr, len(params_list), _p32(set_of), _p32(seeds), seeds.size,
          _stream_handle(stream), ctypes.byref(h))
    return Streams(h)


def mtgp_streams_info(streams: Streams):
    n, w = ctypes.c_uint32(), ctypes.c_uint32()
    _call("mtgp_streams_info", streams.handle, ctypes.byref(n), ctypes.byref(w))
    return n.value, w.value


def mtgp_set_statuses(streams: Streams, states, stream=None):
    n, w = mtgp_streams_info(streams)
    states = np.ascontiguousarray(states, dtype=np.uint32)
    if states.shape != (n, w):
        raise ValueError("states must have shape (%d, %d)" % (n, w))
    _call("mtgp_set_statuses", streams.handle, _p32(states), _stream_handle(stream))


def mtgp_get_statuses(streams: Streams, stream=None) -> np.ndarray:
    n, w = mtgp_streams_info(streams)
    out = np.zeros((n, w), np.uint32)
    _call("mtgp_get_statuses", streams.handle, _p32(out), _stream_handle(stream))
    return out


def mtgp_generate_u32(streams: Streams, stream_ids, counts, out, stream=None):
    ids, counts = _req_arrays(stream_ids, counts)
    total = int(counts.sum()) if counts.size else 0
    _call("mtgp_generate_u32", streams.handle, _p32(ids), _p64(counts), ids.size,
          _dev_ptr(out, total), _stream_handle(stream))


def mtgp_generate_f32(streams: Streams, stream_ids, counts, fmt, out, stream=None):
    ids, counts = _req_arrays(stream_ids, counts)
    total = int(counts.sum()) if counts.size else 0
    _call("mtgp_generate_f32", streams.handle, _p32(ids), _p64(counts), ids.size, int(fmt),
          _dev_ptr(out, total), _stream_handle(stream))


def mtgp_generate_to_host(streams: Streams, stream_ids, counts, fmt, host_out, chunk_bytes=0,
                          stream=None):
    """host_out: a NumPy array or a CPU torch tensor (pinned for full speed)."""
    ids, counts = _req_arrays(stream_ids, counts)
    total = int(counts.sum()) if counts.size else 0
    if isinstance(host_out, np.ndarray):
        if host_out.itemsize != 4 or not host_out.flags.c_contiguous or host_out.size < total:
            raise ValueError("host_out must be a contiguous 4-byte array of >= %d elements" % total)
        ptr = host_out.ctypes.data
    else:
        if host_out.is_cuda or host_out.element_size() != 4 or host_out.numel() < total:
            raise ValueError("host_out must be a CPU tensor of >= %d 4-byte elements" % total)
        ptr = host_out.data_ptr()
    _call("mtgp_generate_to_host", streams.handle, _p32(ids), _p64(counts), ids.size, int(fmt),
          ptr, int(chunk_bytes), _stream_handle(stream))


def mtgp_generate_noalloc(streams: Streams, stream_ids, counts, fmt, out, stream=None):
    """mtgp_generate_u32/_f32 without any allocation (work table in a static
    device array; at most 1024 requests; calls on one device must not
    overlap on the GPU)."""
    ids, counts = _req_arrays(stream_ids, counts)
    total = int(counts.sum()) if counts.size else 0
    _call("mtgp_generate_noalloc", streams.handle, _p32(ids), _p64(counts), ids.size, int(fmt),
          _dev_ptr(out, total), _stream_handle(stream))


def mtgp_check(streams: Streams, stream=None):
    _call("mtgp_check", streams.handle, _stream_handle(stream))


def mtgp_get_launch_config(streams: Streams) -> dict:
    c = LaunchConfig()
    _call("mtgp_get_launch_config", streams.handle, ctypes.byref(c))
    return c.as_dict()


def mtgp_set_launch_config(streams: Streams, warps_per_cta=4, ctas_per_sm=0, words_per_lane=8,
                           kernel=0, coop_percent=100):
    c = LaunchConfig(warps_per_cta, ctas_per_sm, words_per_lane, kernel, coop_percent)
    _call("mtgp_set_launch_config", streams.handle, ctypes.byref(c))


def mtgp_autotune(streams: Streams, fmt=MTGP_U32, sample_streams=0, sample_count=0) -> dict:
    c = LaunchConfig()
    _call("mtgp_autotune", streams.handle, int(fmt), sample_streams, sample_count, ctypes.byref(c))
    return c.as_dict()


def mtgp_plan_create(streams: Streams, stream_ids, counts, fmt, out) -> Plan:
    ids, counts = _req_arrays(stream_ids, counts)
    total = int(counts.sum()) if counts.size else 0
    h = _VP()
    _call("mtgp_plan_create", streams.handle, _p32(ids), _p64(counts), ids.size, int(fmt),
          _dev_ptr(out, total), ctypes.byref(h))
    return Plan(h, streams, out, ids.size)


def mtgp_plan_launch(plan: Plan, stream=None):
    _call("mtgp_plan_launch", plan.handle, _stream_handle(stream))


def mtgp_plan_set_split(plan: Plan, max_piece: int):
    _call("mtgp_plan_set_split", plan.handle, int(max_piece))


def mtgp_plan_set_stats(plan: Plan, gap=None, hamming=None):
    """Fuse the statistics of tests 35 and 100 (Sec. 4.2) into the plan's
    launches, per request: gap = (r, b, t) or None, hamming = (r, s, L,
    bounds) or None; both None turns them off."""
    if gap is None and hamming is None:
        _call("mtgp_plan_set_stats", plan.handle, None)
        plan.stats = None
        return
    c = StatsConfig()
    if gap is not None:
        c.gap_r, c.gap_b, c.gap_t = (int(v) for v in gap)
    if hamming is not None:
        r, s, L, bounds = hamming
        bnd = [int(b) for b in bounds]
        if len(bnd) > 15:
            raise ValueError("at most 15 bounds")
        c.ham_r, c.ham_s, c.ham_L, c.n_bounds = int(r), int(s), int(L), len(bnd)
        for i, b in enumerate(bnd):
            c.bounds[i] = b
    _call("mtgp_plan_set_stats", plan.handle, ctypes.byref(c))
    plan.stats = (c.gap_t, (c.n_bounds + 1) if c.ham_L else 0)


def mtgp_plan_read_stats(plan: Plan, stream=None):
    """Counts of the plan's last launch: (hist (n_req, t+1) or None,
    table (n_req, C, C) or None)."""
    if plan.stats is None:
        raise MtgpError(1, "the plan computes no statistics")
    t, C = plan.stats
    hist = np.zeros((plan.n_req, t + 1), np.uint64) if t else None
    tab = np.zeros((plan.n_req, C, C), np.uint64) if C else None
    _call("mtgp_plan_read_stats", plan.handle, _p64(hist) if hist is not None else None,
          _p64(tab) if tab is not None else None, _stream_handle(stream))
    return hist, tab


def mtgp_plan_autotune(plan: Plan) -> dict:
    c = LaunchConfig()
    _call("mtgp_plan_autotune", plan.handle, ctypes.byref(c))
    return c.as_dict()


def mtgp_plan_set_trace(plan: Plan, enable: bool = True):
    _call("mtgp_plan_set_trace", plan.handle, int(bool(enable)))


def mtgp_plan_read_trace(plan: Plan) -> np.ndarray:
    """(n_items, 4) uint64: start ns, end ns, SM, numbers -- table order."""
    n = mtgp_plan_get_info(plan)["n_items"]
    out = np.zeros((max(n, 1), 4), np.uint64)
    _call("mtgp_plan_read_trace", plan.handle, _p64(out))
    return out[:n]


def mtgp_plan_get_info(plan: Plan) -> dict:
    i = PlanInfo()
    _call("mtgp_plan_get_info", plan.handle, ctypes.byref(i))
    return {"total_numbers": i.total_numbers, "n_items": i.n_items,
            "kernel_launches": i.kernel_launches, "config": i.config.as_dict(),
            "grid_ctas": i.grid_ctas, "n_coop": i.n_coop, "regs_per_thread": i.regs_per_thread,
            "resident_ctas_per_sm": i.resident_ctas_per_sm, "max_piece": i.max_piece,
            "n_split_streams": i.n_split_streams, "n_jumps": i.n_jumps, "n_pieces": i.n_pieces,
            "stats": bool(i.stats)}


class Server:
    """Owning wrapper of an mtgp_server_t (keeps its Streams alive)."""

    def __init__(self, handle, streams):
        self.handle = handle
        self.streams = streams

    def close(self):
        if self.handle:
            _call("mtgp_server_free", self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mtgp_server_create(streams: Streams, arena_bytes=0, max_inflight=0, max_tick_requests=0,
                       tick_timeout_s=0.0, max_piece=0):
    c = ServerConfig(arena_bytes, max_inflight, max_tick_requests, tick_timeout_s, max_piece)
    h = _VP()
    _call("mtgp_server_create", streams.handle, ctypes.byref(c), ctypes.byref(h))
    return Server(h, streams)


def mtgp_server_submit(server: Server, stream_id, count, fmt, tag):
    _call("mtgp_server_submit", server.handle, int(stream_id), int(count), int(fmt), int(tag))


def mtgp_server_progress(server: Server, max_out=1024):
    """Returns a list of completion dicts."""
    buf = (Completion * max_out)()
    n = ctypes.c_uint32()
    _call("mtgp_server_progress", server.handle, buf, max_out, ctypes.byref(n))
    return [{"tag": c.tag, "count": c.count, "arena_offset": c.arena_offset, "fmt": c.fmt,
             "submit_time": c.submit_time, "done_time": c.done_time} for c in buf[:n.value]]


def mtgp_server_debug_hold(server: Server, hold: bool = True):
    _call("mtgp_server_debug_hold", server.handle, int(bool(hold)))


def mtgp_server_release(server: Server, arena_offset, count):
    _call("mtgp_server_release", server.handle, int(arena_offset), int(count))


def mtgp_server_arena(server: Server) -> int:
    h = _VP()
    _call("mtgp_server_arena", server.handle, ctypes.byref(h))
    return h.value


def mtgp_server_read(server: Server, arena_offset, count) -> np.ndarray:
    """Copies a result out of the arena (uint32 bit patterns)."""
    out = np.zeros(max(int(count), 1), np.uint32)
    _call("mtgp_server_read", server.handle, int(arena_offset), int(count), out.ctypes.data)
    return out[:int(count)]


def mtgp_server_run_trace(server: Server, t_arrival, ids, counts, fmts, mode=0, record=False):
    """Returns (latency seconds array, arena offsets or None, stats dict)."""
    t = np.ascontiguousarray(t_arrival, dtype=np.float64)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    fmts = np.ascontiguousarray(fmts, dtype=np.int32)
    n = t.size
    if not (ids.size == counts.size == fmts.size == n):
        raise ValueError("trace arrays must have equal length")
    lat = np.zeros(n, np.float64)
    offs = np.zeros(n, np.uint64) if record else None
    st = ServerStats()
    _call("mtgp_server_run_trace", server.handle,
          t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _p32(ids), _p64(counts),
          fmts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n, int(mode),
          lat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
          _p64(offs) if record else None, ctypes.byref(st))
    return lat, offs, {"requests": st.requests, "numbers": st.numbers, "ticks": st.ticks,
                       "elapsed": st.elapsed, "busy_wait": st.busy_wait,
                       "launch_host_s": st.launch_host_s, "jumps": st.jumps}


# ---------------------------------------------------------------------------
# Quality statistics (Sec. 4.2, tests 35 and 100) over device sequences
# ---------------------------------------------------------------------------
def mtgp_gap_histogram(values, counts, r=25, b=5, t=128, stream=None) -> np.ndarray:
    """Gap-length histograms of the device sequences in `values` (back to
    back, lengths `counts`): array (n_seq, t + 1)."""
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    hist = np.zeros((counts.size, t + 1), dtype=np.uint64)
    _call("mtgp_gap_histogram", _dev_ptr(values, int(counts.sum())), _p64(counts), counts.size, r, b, t,
          _p64(hist), _stream_handle(stream))
    return hist


def mtgp_hamming_pairs(values, counts, r=25, s=5, L=1200, bounds=(), stream=None) -> np.ndarray:
    """Tables of successive block-weight classes: array (n_seq, C, C)."""
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    bnd = np.ascontiguousarray(bounds, dtype=np.uint32)
    C = bnd.size + 1
    table = np.zeros((counts.size, C, C), dtype=np.uint64)
    _call("mtgp_hamming_pairs", _dev_ptr(values, int(counts.sum())), _p64(counts), counts.size, r, s, L,
          _p32(bnd) if bnd.size else None, bnd.size, _p64(table), _stream_handle(stream))
    return table


# ---------------------------------------------------------------------------
# Jump-ahead
# ---------------------------------------------------------------------------
def mtgp_jump(streams: Streams, stream_ids, jumps, stream=None):
    """Advance each listed stream by its jump (numbers skipped, exactly)."""
    ids = np.ascontiguousarray(stream_ids, dtype=np.uint32)
    js = np.ascontiguousarray(jumps, dtype=np.uint64)
    if ids.shape != js.shape or ids.ndim != 1:
        raise ValueError("stream_ids and jumps must be 1-D arrays of the same length")
    _call("mtgp_jump", streams.handle, _p32(ids), _p64(js), ids.size, _stream_handle(stream))


def mtgp_params_minpoly(params: Params) -> np.ndarray:
    """Coefficients (uint8, index = power of t) of the jump polynomial mu."""
    d = ctypes.c_int32()
    _call("mtgp_params_minpoly", params.handle, None, 0, ctypes.byref(d))
    words = np.zeros(d.value // 64 + 1, dtype=np.uint64)
    _call("mtgp_params_minpoly", params.handle, _p64(words), words.size, ctypes.byref(d))
    bits = np.unpackbits(words.view(np.uint8), bitorder="little")
    return bits[:d.value + 1].copy()


def mtgp_params_period_check(params: Params, stream=None) -> bool:
    """True if the transition polynomial has degree Mexp and is irreducible
    (for a Mersenne-prime Mexp: period 2^Mexp - 1)."""
    r = ctypes.c_int32()
    _call("mtgp_params_period_check", params.handle, _stream_handle(stream), ctypes.byref(r))
    return bool(r.value)


# ---------------------------------------------------------------------------
# The original Mersenne Twister (comparison generator, include/mtgp_mt.h)
# ---------------------------------------------------------------------------
class MtStreams:
    """Owning wrapper of an mtgp_mt_t."""

    def __init__(self, handle, params: MtParams, n_streams: int):
        self.handle = handle
        self.params = params
        self.n_streams = n_streams

    def close(self):
        if self.handle:
            _call("mtgp_mt_free", self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mtgp_mt_params_mt19937() -> MtParams:
    q = MtParams()
    _call("mtgp_mt_params_mt19937", ctypes.byref(q))
    return q


def mtgp_mt_params_generate(p: int, seed: int) -> MtParams:
    q = MtParams()
    _call("mtgp_mt_params_generate", p, seed, ctypes.byref(q))
    return q


def mtgp_mt_init(params: MtParams, seeds, stream=None) -> MtStreams:
    seeds = np.ascontiguousarray(seeds, dtype=np.uint32)
    h = _VP()
    q = MtParams(*[getattr(params, f) for f, _ in MtParams._fields_])
    _call("mtgp_mt_init", ctypes.byref(q), _p32(seeds), seeds.size, _stream_handle(stream),
          ctypes.byref(h))
    return MtStreams(h, q, seeds.size)


def mtgp_mt_init_multi(params_list, set_of_stream, seeds, stream=None) -> MtStreams:
    """One parameter set per stream: stream s uses params_list[set_of_stream[s]]."""
    seeds = np.ascontiguousarray(seeds, dtype=np.uint32)
    set_of = np.ascontiguousarray(set_of_stream, dtype=np.uint32)
    if set_of.shape != seeds.shape:
        raise ValueError("set_of_stream and seeds must have the same length")
    arr = (MtParams * len(params_list))(
        *[MtParams(*[getattr(q, f) for f, _ in MtParams._fields_]) for q in params_list])
    h = _VP()
    _call("mtgp_mt_init_multi", arr, len(params_list), _p32(set_of), _p32(seeds), seeds.size,
          _stream_handle(stream), ctypes.byref(h))
    return MtStreams(h, arr[0], seeds.size)


def mtgp_mt_set_statuses(mt: MtStreams, states, stream=None):
    states = np.ascontiguousarray(states, dtype=np.uint32)
    if states.shape != (mt.n_streams, mt.params.n):
        raise ValueError("states must have shape (%d, %d)" % (mt.n_streams, mt.params.n))
    _call("mtgp_mt_set_statuses", mt.handle, _p32(states), _stream_handle(stream))


def mtgp_mt_get_statuses(mt: MtStreams, stream=None) -> np.ndarray:
    out = np.zeros((mt.n_streams, mt.params.n), np.uint32)
    _call("mtgp_mt_get_statuses", mt.handle, _p32(out), _stream_handle(stream))
    return out


def mtgp_mt_generate(mt: MtStreams, stream_ids, counts, fmt, out, stream=None):
    ids, counts = _req_arrays(stream_ids, counts)
    total = int(counts.sum()) if counts.size else 0
    _call("mtgp_mt_generate", mt.handle, _p32(ids), _p64(counts), ids.size, int(fmt),
          _dev_ptr(out, total), _stream_handle(stream))


def mtgp_mt_check(mt: MtStreams, stream=None):
    _call("mtgp_mt_check", mt.handle, _stream_handle(stream))


def mtgp_mt_params_minpoly(params: MtParams) -> np.ndarray:
    """Coefficients (uint8, index = power of t) of the set's transition polynomial."""
    q = MtParams(*[getattr(params, f) for f, _ in MtParams._fields_])
    d = ctypes.c_int32()
    _call("mtgp_mt_params_minpoly", ctypes.byref(q), None, 0, ctypes.byref(d))
    words = np.zeros(d.value // 64 + 1, dtype=np.uint64)
    _call("mtgp_mt_params_minpoly", ctypes.byref(q), _p64(words), words.size, ctypes.byref(d))
    bits = np.unpackbits(words.view(np.uint8), bitorder="little")
    return bits[:d.value + 1].copy()


def mtgp_mt_params_period_check(params: MtParams, stream=None) -> bool:
    """True if the set's transition polynomial has degree p and is irreducible
    (for a Mersenne-prime p: period 2^p - 1)."""
    q = MtParams(*[getattr(params, f) for f, _ in MtParams._fields_])
    r = ctypes.c_int32()
    _call("mtgp_mt_params_period_check", ctypes.byref(q), _stream_handle(stream), ctypes.byref(r))
    return bool(r.value)
