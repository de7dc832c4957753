"""CPU oracle (test infrastructure only).

Loads the plain C reference in ``cc_oracle.c`` through ctypes. Only the tests, the smoke
check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this
package; the product package never does, and nothing here imports the product package.

Every function states the passage of the paper it follows (Saldanha and de Souza,
arXiv 1901.11204): the standard pairwise loop of Section 4 is the definition the counts
are checked against; the proposed cyclic order of Section 4 and Algorithms 1 and 2 of
Section 3 are independent cross-checks. Parity of the FP32 interaction *sum* against the
GPU is a tolerance check (1e-5 relative), not bit parity.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libcc_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
          "-std=c11", "-Wall"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/libcc_oracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(path: str):
    lib = ctypes.CDLL(path)
    i32p = ctypes.POINTER(ctypes.c_int32)
    f32p = ctypes.POINTER(ctypes.c_float)
    i64p = ctypes.POINTER(ctypes.c_int64)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    f64p = ctypes.POINTER(ctypes.c_double)
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_get_threads.restype = ctypes.c_int
    lib.oracle_count_i32.argtypes = [i32p, i32p, i32p, ctypes.c_int64, ctypes.c_uint32]
    lib.oracle_count_i32.restype = ctypes.c_uint64
    lib.oracle_count_i32_cyclic.argtypes = [i32p, i32p, i32p, ctypes.c_int64, ctypes.c_uint32]
    lib.oracle_count_i32_cyclic.restype = ctypes.c_uint64
    lib.oracle_sum_i32.argtypes = [i32p, i32p, i32p, ctypes.c_int64, ctypes.c_uint32, f64p]
    lib.oracle_sum_i32.restype = ctypes.c_uint64
    lib.oracle_count_f32.argtypes = [f32p, f32p, f32p, f32p, ctypes.c_int64, f64p]
    lib.oracle_count_f32.restype = ctypes.c_uint64
    lib.oracle_count_i32_sets.argtypes = [i32p, i32p, i32p, i64p, ctypes.c_int64,
                                          ctypes.c_uint32, u64p]
    lib.oracle_count_f32_sets.argtypes = [f32p, f32p, f32p, f32p, i64p, ctypes.c_int64,
                                          u64p, f64p]
    lib.oracle_collide_f32.argtypes = [ctypes.c_float] * 8
    lib.oracle_collide_f32.restype = ctypes.c_int
    lib.oracle_cyclic_schedule.argtypes = [ctypes.c_int64, i64p, i64p, ctypes.c_int64]
    lib.oracle_cyclic_schedule.restype = ctypes.c_int64
    lib.oracle_cyclic_work.argtypes = [ctypes.c_int64, ctypes.c_int64]
    lib.oracle_cyclic_work.restype = ctypes.c_int64
    lib.oracle_count_colls.argtypes = [i32p, i32p, i32p, ctypes.c_int64]
    lib.oracle_count_colls.restype = ctypes.c_uint64
    lib.oracle_count_contacts.argtypes = [i32p, i32p, i32p, ctypes.c_int64]
    lib.oracle_count_contacts.restype = ctypes.c_uint64
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB_PATH)
        return _lib


def use_library(path: str | None) -> None:
    """Point this module at another build of cc_oracle.c (None: the default build).
    The mutation tests use this to check that planted mistakes fail the pins."""
    global _lib
    with _lock:
        _lib = None if path is None else _bind(path)


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def set_threads(t: int) -> None:
    """Number of OpenMP threads for the loops below (0 = all available)."""
    _load().oracle_set_threads(int(t))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def count_i32(x, y, z, r2: int) -> int:
    """Standard algorithm (Section 4): pairs i<j with integer squared distance <= r2."""
    x, y, z = _i32(x), _i32(y), _i32(z)
    n = len(x)
    assert len(y) == n and len(z) == n
    return int(_load().oracle_count_i32(_p(x, ctypes.c_int32), _p(y, ctypes.c_int32),
                                        _p(z, ctypes.c_int32), n, int(r2)))


def sum_i32(x, y, z, r2: int) -> tuple[int, float]:
    """Standard algorithm over integer points: (count, FP64 sum of 1/max(d,1e-6))."""
    x, y, z = _i32(x), _i32(y), _i32(z)
    s = ctypes.c_double(0.0)
    c = _load().oracle_sum_i32(_p(x, ctypes.c_int32), _p(y, ctypes.c_int32),
                               _p(z, ctypes.c_int32), len(x), int(r2), ctypes.byref(s))
    return int(c), float(s.value)


def count_i32_cyclic(x, y, z, r2: int) -> int:
    """Proposed algorithm (Section 4) with the even-N extra step: same pairs, other order."""
    x, y, z = _i32(x), _i32(y), _i32(z)
    return int(_load().oracle_count_i32_cyclic(_p(x, ctypes.c_int32), _p(y, ctypes.c_int32),
                                               _p(z, ctypes.c_int32), len(x), int(r2)))


def count_f32(x, y, z, r) -> tuple[int, float]:
    """Standard algorithm over FP32 spheres: (count, FP64 sum of 1/max(d,1e-6))."""
    x, y, z, r = _f32(x), _f32(y), _f32(z), _f32(r)
    s = ctypes.c_double(0.0)
    c = _load().oracle_count_f32(_p(x, ctypes.c_float), _p(y, ctypes.c_float),
                                 _p(z, ctypes.c_float), _p(r, ctypes.c_float), len(x),
                                 ctypes.byref(s))
    return int(c), float(s.value)


def count_i32_sets(x, y, z, offsets, r2: int) -> np.ndarray:
    """Per-set counts: the standard loop inside every [offsets[k], offsets[k+1])."""
    x, y, z = _i32(x), _i32(y), _i32(z)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    out = np.zeros(len(off) - 1, dtype=np.uint64)
    _load().oracle_count_i32_sets(_p(x, ctypes.c_int32), _p(y, ctypes.c_int32),
                                  _p(z, ctypes.c_int32), _p(off, ctypes.c_int64),
                                  len(off) - 1, int(r2), _p(out, ctypes.c_uint64))
    return out


def count_f32_sets(x, y, z, r, offsets) -> tuple[np.ndarray, np.ndarray]:
    x, y, z, r = _f32(x), _f32(y), _f32(z), _f32(r)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    cnt = np.zeros(len(off) - 1, dtype=np.uint64)
    sm = np.zeros(len(off) - 1, dtype=np.float64)
    _load().oracle_count_f32_sets(_p(x, ctypes.c_float), _p(y, ctypes.c_float),
                                  _p(z, ctypes.c_float), _p(r, ctypes.c_float),
                                  _p(off, ctypes.c_int64), len(off) - 1,
                                  _p(cnt, ctypes.c_uint64), _p(sm, ctypes.c_double))
    return cnt, sm


def collide_f32(a, b) -> bool:
    """The FP32 sphere predicate for one pair; a and b are (x, y, z, r)."""
    return bool(_load().oracle_collide_f32(*[float(v) for v in a], *[float(v) for v in b]))


def cyclic_schedule(n: int) -> tuple[np.ndarray, np.ndarray]:
    """The (i, j) pairs of the proposed algorithm in evaluation order (Section 4)."""
    lib = _load()
    total = int(lib.oracle_cyclic_schedule(int(n), None, None, 0))
    pi = np.zeros(max(total, 1), dtype=np.int64)
    pj = np.zeros(max(total, 1), dtype=np.int64)
    lib.oracle_cyclic_schedule(int(n), _p(pi, ctypes.c_int64), _p(pj, ctypes.c_int64), total)
    return pi[:total], pj[:total]


def cyclic_work(n: int, i: int) -> int:
    """Evaluations performed by object i under the proposed algorithm."""
    return int(_load().oracle_cyclic_work(int(n), int(i)))


def count_colls(x, y, z) -> int:
    """Algorithm 1 (Section 3): same-site collisions through a space array of counts."""
    x, y, z = _i32(x), _i32(y), _i32(z)
    v = int(_load().oracle_count_colls(_p(x, ctypes.c_int32), _p(y, ctypes.c_int32),
                                       _p(z, ctypes.c_int32), len(x)))
    if v == 2 ** 64 - 1:
        raise ValueError("space array too large for Algorithm 1")
    return v


def count_contacts(x, y, z) -> int:
    """Algorithm 2 (Section 3): pairs on face-adjacent sites, via the space array."""
    x, y, z = _i32(x), _i32(y), _i32(z)
    v = int(_load().oracle_count_contacts(_p(x, ctypes.c_int32), _p(y, ctypes.c_int32),
                                          _p(z, ctypes.c_int32), len(x)))
    if v == 2 ** 64 - 1:
        raise ValueError("space array too large for Algorithm 2")
    return v
