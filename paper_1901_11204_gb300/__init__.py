"""Python binding of the cc C ABI (include/cc.h): argument marshalling only.

Every step of the pair counting runs in the CUDA kernels of libcc.so; this module only
turns torch tensors into device pointers and streams into handles. There is no CPU
fallback: if libcc.so is missing or fails to load, every call raises.

The functions named cc_* mirror the C entry points one to one. The convenience helpers
(count_pairs, interaction_sum, count_pairs_batched, Plan, Server) take torch CUDA tensors
and return torch tensors that live on the device.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcc.so")

CC_OK = 0
CC_ERR_INVALID_ARG = 1
CC_ERR_RANGE = 2
CC_ERR_NOMEM = 3
CC_ERR_CUDA = 4
CC_ERR_TIMEOUT = 5
CC_ERR_BUSY = 6
CC_ERR_NOT_FOUND = 7
CC_I32 = 0
CC_F32 = 1
CC_OP_COUNT = 0
CC_OP_SUM = 1
CC_COUNT_INVALID = 0xFFFFFFFFFFFFFFFF


class CCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_STATUS_NAMES = {0: "CC_OK", 1: "CC_ERR_INVALID_ARG", 2: "CC_ERR_RANGE", 3: "CC_ERR_NOMEM",
                 4: "CC_ERR_CUDA", 5: "CC_ERR_TIMEOUT", 6: "CC_ERR_BUSY", 7: "CC_ERR_NOT_FOUND"}


class cc_points(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("z", ctypes.c_void_p), ("r", ctypes.c_void_p)]


class cc_result(ctypes.Structure):
    _fields_ = [("req_id", ctypes.c_uint64), ("set_id", ctypes.c_int32), ("op", ctypes.c_int32),
                ("status", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("count", ctypes.c_ulonglong), ("sum", ctypes.c_float), ("pad2", ctypes.c_float),
                ("t_arrive_s", ctypes.c_double), ("t_done_s", ctypes.c_double)]


_lib = None
_lock = threading.Lock()

_VP = ctypes.c_void_p
_PTS = ctypes.POINTER(cc_points)
_SIGS = {
    "cc_count_pairs": ([_PTS, ctypes.c_int64, ctypes.c_uint32, _VP, _VP], ctypes.c_int),
    "cc_count_pairs_straightforward": ([_PTS, ctypes.c_int64, ctypes.c_uint32, _VP, _VP], ctypes.c_int),
    "cc_count_same_site": ([_PTS, ctypes.c_int64, _VP, _VP], ctypes.c_int),
    "cc_count_contacts": ([_PTS, ctypes.c_int64, _VP, _VP], ctypes.c_int),
    "cc_count_pairs_noalloc": ([_PTS, ctypes.c_int64, ctypes.c_uint32, _VP, _VP], ctypes.c_int),
    "cc_interaction_sum": ([_PTS, ctypes.c_int64, ctypes.c_uint32, _VP, _VP, _VP], ctypes.c_int),
    "cc_validate_points": ([_PTS, ctypes.c_int64, _VP], ctypes.c_int),
    "cc_reserve": ([ctypes.c_int64, _VP], ctypes.c_int),
    "cc_release": ([_VP], ctypes.c_int),
    "cc_stream_status": ([_VP], ctypes.c_int),
    "cc_stream_mode": ([_VP, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "cc_set_tensor_cores": ([ctypes.c_int32], ctypes.c_int),
    "cc_plan_create": ([ctypes.POINTER(_VP), ctypes.c_char_p, ctypes.c_int32, ctypes.c_int64], ctypes.c_int),
    "cc_plan_destroy": ([_VP], None),
    "cc_count_pairs_batched": ([_VP, _PTS, _VP, ctypes.c_int32, ctypes.c_uint32, _VP, _VP, _VP], ctypes.c_int),
    "cc_plan_last_items": ([_VP, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "cc_server_create": ([ctypes.POINTER(_VP), ctypes.c_size_t, ctypes.c_int32], ctypes.c_int),
    "cc_server_create_tuned": ([ctypes.POINTER(_VP), ctypes.c_size_t, ctypes.c_int32, ctypes.c_char_p], ctypes.c_int),
    "cc_server_register_set": ([_VP, _PTS, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "cc_server_unregister_set": ([_VP, ctypes.c_int32], ctypes.c_int),
    "cc_server_submit": ([_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64], ctypes.c_int),
    "cc_server_poll": ([_VP, ctypes.POINTER(cc_result), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "cc_server_drain": ([_VP, ctypes.c_double], ctypes.c_int),
    "cc_server_stats": ([_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "cc_server_destroy": ([_VP], None),
    "cc_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "cc_last_error": ([], ctypes.c_char_p),
    "cc_version": ([], ctypes.c_char_p),
    "cc_set_wait_limit_ns": ([ctypes.c_uint64], None),
    "cc_debug_stall_copies": ([ctypes.c_int], None),
    "cc_profile_enable": ([ctypes.c_int], None),
    "cc_profile_read": ([ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
}


def lib():
    """The loaded libcc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libcc.so not built ({LIB_PATH}); run __graft_entry__.build() "
                                   "or python paper_1901_11204_gb300/builder.py")
            L = ctypes.CDLL(LIB_PATH)
            for name, (argt, rest) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = argt
                f.restype = rest
            _lib = L
        return _lib


def build(force: bool = False, verbose: bool = False) -> str:
    from . import builder
    return builder.build(force=force, verbose=verbose)


def _check(status: int):
    if status != CC_OK:
        raise CCError(status, lib().cc_last_error().decode())


# ---- thin 1:1 wrappers over the C ABI (raw pointers / handles) -------------------------

def cc_count_pairs(points: cc_points, n: int, r2: int, d_count: int, stream: int) -> int:
    return lib().cc_count_pairs(ctypes.byref(points), n, r2, d_count, stream)


def cc_interaction_sum(points: cc_points, n: int, r2: int, d_sum: int, d_count: int, stream: int) -> int:
    return lib().cc_interaction_sum(ctypes.byref(points), n, r2, d_sum, d_count, stream)


def cc_validate_points(points: cc_points, n: int, stream: int) -> int:
    return lib().cc_validate_points(ctypes.byref(points), n, stream)


def cc_count_pairs_batched(plan: int, points: cc_points, d_offsets: int, n_sets: int, r2: int,
                           d_counts: int, d_sums: int, stream: int) -> int:
    return lib().cc_count_pairs_batched(plan, ctypes.byref(points), d_offsets, n_sets, r2,
                                        d_counts, d_sums, stream)


def cc_stream_status(stream: int) -> int:
    return lib().cc_stream_status(stream)


# ---- torch helpers ---------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _stream_handle(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def make_points(x, y, z, r=None) -> cc_points:
    """cc_points over device tensors (int32 x/y/z, or float32 x/y/z/r)."""
    torch = _torch()
    for t in (x, y, z) + ((r,) if r is not None else ()):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("coordinates must be contiguous CUDA tensors")
    if x.dtype == torch.int32:
        return cc_points(CC_I32, x.data_ptr(), y.data_ptr(), z.data_ptr(), None)
    if x.dtype == torch.float32:
        if r is None or r.dtype != torch.float32:
            raise ValueError("FP32 spheres need float32 radii")
        return cc_points(CC_F32, x.data_ptr(), y.data_ptr(), z.data_ptr(), r.data_ptr())
    raise ValueError(f"unsupported dtype {x.dtype}")


def count_pairs(x, y, z, r2: int = 0, r=None, out=None, stream=None):
    """Exact colliding-pair count of one set; returns a 1-element uint64 (int64 view)
    device tensor. Asynchronous on `stream` (default: torch's current stream)."""
    torch = _torch()
    pts = make_points(x, y, z, r)
    if out is None:
        out = torch.empty(1, dtype=torch.int64, device=x.device)
    _check(cc_count_pairs(pts, x.numel(), int(r2), out.data_ptr(), _stream_handle(stream)))
    return out


def count_pairs_straightforward(x, y, z, r2: int = 0, r=None, out=None, stream=None):
    """Same count with the straightforward schedule of the paper's comparison (each group
    of 1024 objects against all later ones); for measuring the balance effect."""
    torch = _torch()
    pts = make_points(x, y, z, r)
    if out is None:
        out = torch.empty(1, dtype=torch.int64, device=x.device)
    _check(lib().cc_count_pairs_straightforward(ctypes.byref(pts), x.numel(), int(r2), out.data_ptr(),
                                                _stream_handle(stream)))
    return out


def count_same_site(x, y, z, out=None, stream=None):
    """Algorithm 1 (Section 3): same-site bead pairs in linear time (int32 points)."""
    torch = _torch()
    pts = make_points(x, y, z)
    if out is None:
        out = torch.empty(1, dtype=torch.int64, device=x.device)
    _check(lib().cc_count_same_site(ctypes.byref(pts), x.numel(), out.data_ptr(), _stream_handle(stream)))
    return out


def count_contacts(x, y, z, out=None, stream=None):
    """Algorithm 2 (Section 3): face-adjacent bead pairs in linear time (int32 points)."""
    torch = _torch()
    pts = make_points(x, y, z)
    if out is None:
        out = torch.empty(1, dtype=torch.int64, device=x.device)
    _check(lib().cc_count_contacts(ctypes.byref(pts), x.numel(), out.data_ptr(), _stream_handle(stream)))
    return out


def interaction_sum(x, y, z, r2: int = 0, r=None, out_sum=None, out_count=None, stream=None):
    """(sum, count) device tensors: FP32 sum of 1/max(d, 1e-6) over colliding pairs and
    their number."""
    torch = _torch()
    pts = make_points(x, y, z, r)
    if out_sum is None:
        out_sum = torch.empty(1, dtype=torch.float32, device=x.device)
    if out_count is None:
        out_count = torch.empty(1, dtype=torch.int64, device=x.device)
    _check(cc_interaction_sum(pts, x.numel(), int(r2), out_sum.data_ptr(), out_count.data_ptr(),
                              _stream_handle(stream)))
    return out_sum, out_count


def validate_points(x, y, z, r=None, stream=None) -> int:
    """Synchronous range check; returns the cc_status (CC_OK or CC_ERR_RANGE)."""
    pts = make_points(x, y, z, r)
    return cc_validate_points(pts, x.numel(), _stream_handle(stream))


def stream_status(stream=None) -> int:
    return cc_stream_status(_stream_handle(stream))


# Pair kernel chosen by the device for the last single-set call on a stream
# (cc_stream_mode): the CC_MODE_* values of cc.h.
MODE_FP32_EXACT, MODE_INT_WIDE, MODE_RANGE_ERROR, MODE_FP32_SPHERES, MODE_TENSOR = 0, 1, 2, 3, 4
MODE_TENSOR_SPHERES = 5


def set_tensor_cores(enable: bool) -> None:
    """Enable (default) or disable the tensor-core pair kernel for later counts."""
    _check(lib().cc_set_tensor_cores(1 if enable else 0))


def stream_mode(stream=None) -> int:
    m = ctypes.c_int32(-1)
    _check(lib().cc_stream_mode(_stream_handle(stream), ctypes.byref(m)))
    return int(m.value)


def reserve(max_n: int, stream=None):
    _check(lib().cc_reserve(int(max_n), _stream_handle(stream)))


def set_wait_limit_ns(ns: int):
    lib().cc_set_wait_limit_ns(int(ns))


def debug_stall_copies(on: bool):
    lib().cc_debug_stall_copies(1 if on else 0)


def profile_enable(on: bool):
    """Bracket every single-set pair-kernel launch with CUDA events (benchmarking)."""
    lib().cc_profile_enable(1 if on else 0)


def profile_read():
    """(total kernel milliseconds, launches) since the previous read."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(lib().cc_profile_read(ctypes.byref(ms), ctypes.byref(n)))
    return float(ms.value), int(n.value)


def version() -> str:
    return lib().cc_version().decode()


def as_u64(t) -> int:
    """Python int of a 1-element int64 tensor holding an unsigned 64-bit count."""
    v = int(t.item())
    return v & 0xFFFFFFFFFFFFFFFF


# ---- batched sets ----------------------------------------------------------------------

class Plan:
    """Batching plan (cc_plan): band table + device work queue + captured graph."""

    def __init__(self, max_sets: int, max_points: int, tune_table_json: str | None = None):
        h = ctypes.c_void_p()
        js = tune_table_json.encode() if tune_table_json else None
        _check(lib().cc_plan_create(ctypes.byref(h), js, int(max_sets), int(max_points)))
        self.handle = h.value

    def count_pairs_batched(self, x, y, z, offsets, r2: int = 0, r=None, want_sum=False,
                            counts=None, sums=None, stream=None):
        """Per-set counts (int64 view of uint64) and, with want_sum, FP32 sums, for the
        sets [offsets[k], offsets[k+1]) of the concatenated coordinates."""
        torch = _torch()
        pts = make_points(x, y, z, r)
        if offsets.dtype != torch.int64 or not offsets.is_cuda:
            raise ValueError("offsets must be an int64 CUDA tensor")
        n_sets = offsets.numel() - 1
        if counts is None:
            counts = torch.empty(max(n_sets, 1), dtype=torch.int64, device=x.device)
        if want_sum and sums is None:
            sums = torch.empty(max(n_sets, 1), dtype=torch.float32, device=x.device)
        _check(cc_count_pairs_batched(self.handle, pts, offsets.data_ptr(), n_sets, int(r2),
                                      counts.data_ptr(), sums.data_ptr() if want_sum else None,
                                      _stream_handle(stream)))
        return counts[:n_sets], (sums[:n_sets] if want_sum else None)

    def last_items(self) -> int:
        v = ctypes.c_int64()
        _check(lib().cc_plan_last_items(self.handle, ctypes.byref(v)))
        return int(v.value)

    def close(self):
        if getattr(self, "handle", None):
            lib().cc_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- serving ---------------------------------------------------------------------------

TUNE_TABLE_PATH = os.path.join(_HERE, "tune_gb300.json")


def default_tune_table() -> str | None:
    """The band table the autotuner measured on GB300 (tune_gb300.json), or None."""
    if os.path.exists(TUNE_TABLE_PATH):
        with open(TUNE_TABLE_PATH) as f:
            return f.read()
    return None


class Server:
    """Continuous-batching server (cc_server) over device-resident sets. Its batching
    plans use tune_table_json (default: the packaged GB300 table; None: built-in)."""

    def __init__(self, mem_budget_bytes: int, max_slots: int, tune_table_json: str | None = "default"):
        h = ctypes.c_void_p()
        if tune_table_json == "default":
            tune_table_json = default_tune_table()
        js = tune_table_json.encode() if tune_table_json else None
        _check(lib().cc_server_create_tuned(ctypes.byref(h), int(mem_budget_bytes), int(max_slots), js))
        self.handle = h.value
        self._keep = []

    def register_set(self, x, y, z, r=None) -> int:
        """Copies a set (numpy arrays on the host or CUDA tensors) into device memory."""
        import numpy as np

        def ptr(a):
            if hasattr(a, "data_ptr"):
                return a.data_ptr()
            a = np.ascontiguousarray(a)
            self._keep.append(a)
            return a.ctypes.data

        is_f32 = str(getattr(x, "dtype", "")).endswith("float32")
        pts = cc_points(CC_F32 if is_f32 else CC_I32, ptr(x), ptr(y), ptr(z),
                        ptr(r) if r is not None else None)
        sid = ctypes.c_int32()
        _check(lib().cc_server_register_set(self.handle, ctypes.byref(pts), len(x), ctypes.byref(sid)))
        self._keep.clear()
        return int(sid.value)

    def unregister_set(self, set_id: int):
        _check(lib().cc_server_unregister_set(self.handle, int(set_id)))

    def submit(self, set_id: int, op: int, r2: int, req_id: int):
        _check(lib().cc_server_submit(self.handle, int(set_id), int(op), int(r2), int(req_id)))

    def poll(self, max_results: int = 4096):
        buf = (cc_result * max_results)()
        n = ctypes.c_int32()
        _check(lib().cc_server_poll(self.handle, buf, max_results, ctypes.byref(n)))
        return [dict(req_id=b.req_id, set_id=b.set_id, op=b.op, status=b.status, count=b.count,
                     sum=b.sum, t_arrive=b.t_arrive_s, t_done=b.t_done_s) for b in buf[:n.value]]

    def drain(self, timeout_s: float = 60.0):
        _check(lib().cc_server_drain(self.handle, float(timeout_s)))

    def stats(self):
        v = [ctypes.c_int64() for _ in range(4)]
        _check(lib().cc_server_stats(self.handle, *[ctypes.byref(t) for t in v]))
        return dict(batches=v[0].value, admitted=v[1].value, peak_inflight=v[2].value,
                    peak_bytes=v[3].value)

    def close(self):
        if getattr(self, "handle", None):
            lib().cc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
