"""ctypes wrapper around the CPU oracle (test infrastructure only).

Arrays are numpy.  A cloud is any C-contiguous array of n 16-byte records,
for example the ``(n, 4)`` int32 arrays the scene generators produce.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

VOIDP = C.c_void_p
U64 = C.c_uint64
U32 = C.c_uint32
INT = C.c_int
FLT = C.c_float


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            L.oracle_project.argtypes = [VOIDP, INT, INT, FLT, FLT, FLT, C.POINTER(U32), C.POINTER(FLT)]
            L.oracle_project.restype = INT
            L.oracle_key.argtypes = [FLT, U32]
            L.oracle_key.restype = U64
            L.oracle_clear_keys.argtypes = [VOIDP, C.c_size_t]
            L.oracle_clear_hq.argtypes = [VOIDP, VOIDP, VOIDP, C.c_size_t]
            L.oracle_render_basic.argtypes = [VOIDP, U64, VOIDP, INT, INT, VOIDP]
            L.oracle_hq_depth.argtypes = [VOIDP, U64, VOIDP, INT, INT, VOIDP]
            L.oracle_hq_color.argtypes = [VOIDP, U64, VOIDP, INT, INT, FLT, VOIDP, VOIDP, VOIDP]
            L.oracle_hq_channel_sums.argtypes = [VOIDP, U64, VOIDP, INT, INT, FLT, VOIDP, VOIDP, VOIDP,
                                                 VOIDP, VOIDP]
            L.oracle_resolve_basic.argtypes = [VOIDP, C.c_size_t, VOIDP, U64, U32, VOIDP]
            L.oracle_resolve_hq.argtypes = [VOIDP, VOIDP, C.c_size_t, U32, VOIDP]
            L.oracle_render_basic_threads.argtypes = [VOIDP, U64, VOIDP, INT, INT, VOIDP, INT]
            L.oracle_render_basic_threads.restype = INT
            L.oracle_resolve_basic_threads.argtypes = [VOIDP, C.c_size_t, VOIDP, U64, U32, VOIDP, INT]
            L.oracle_resolve_basic_threads.restype = INT
            L.oracle_key_rgb.argtypes = [FLT, U32]
            L.oracle_key_rgb.restype = U64
            L.oracle_render_rgb.argtypes = [VOIDP, U64, VOIDP, INT, INT, VOIDP]
            L.oracle_resolve_rgb.argtypes = [VOIDP, C.c_size_t, U32, VOIDP]
            L.oracle_morton_codes63.argtypes = [VOIDP, U64, VOIDP]
            L.oracle_aabb.argtypes = [VOIDP, U64, VOIDP, VOIDP]
            L.oracle_morton_codes.argtypes = [VOIDP, U64, VOIDP]
            L.oracle_splitmix64.argtypes = [U64, U64]
            L.oracle_splitmix64.restype = U64
            L.oracle_counter_keys.argtypes = [U64, U64, VOIDP]
            L.oracle_reorder.argtypes = [VOIDP, U64, U64, INT, U32, VOIDP]
            L.oracle_reorder.restype = INT
            L.oracle_gather.argtypes = [VOIDP, U64, VOIDP, VOIDP]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(VOIDP)


def _cloud(pts: np.ndarray) -> tuple[np.ndarray, int]:
    pts = np.ascontiguousarray(pts)
    assert pts.nbytes % 16 == 0
    return pts, pts.nbytes // 16


def _mat(m) -> np.ndarray:
    m = np.ascontiguousarray(np.asarray(m, dtype=np.float32).reshape(16))
    return m


def project(m, width: int, height: int, x: float, y: float, z: float):
    """Returns (pixel, w) or None when culled."""
    mm = _mat(m)
    p = U32()
    w = FLT()
    ok = lib().oracle_project(_ptr(mm), width, height, FLT(x), FLT(y), FLT(z), C.byref(p), C.byref(w))
    return (p.value, w.value) if ok else None


def key(w: float, index: int) -> int:
    return int(lib().oracle_key(FLT(w), index))


def splitmix64(seed: int, k: int) -> int:
    return int(lib().oracle_splitmix64(seed & ((1 << 64) - 1), k))


def counter_keys(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint32)
    lib().oracle_counter_keys(seed & ((1 << 64) - 1), count, _ptr(out))
    return out


def clear_keys(npx: int) -> np.ndarray:
    k = np.empty(npx, dtype=np.uint64)
    lib().oracle_clear_keys(_ptr(k), npx)
    return k


def render_basic(pts: np.ndarray, m, width: int, height: int, keys: np.ndarray | None = None) -> np.ndarray:
    pts, n = _cloud(pts)
    if keys is None:
        keys = clear_keys(width * height)
    assert keys.dtype == np.uint64 and keys.size == width * height
    lib().oracle_render_basic(_ptr(pts), n, _ptr(_mat(m)), width, height, _ptr(keys))
    return keys


def key_rgb(w: float, rgba: int) -> int:
    return int(lib().oracle_key_rgb(FLT(w), rgba & 0xFFFFFFFF))


def render_rgb(pts: np.ndarray, m, width: int, height: int, keys: np.ndarray | None = None) -> np.ndarray:
    """Colour-payload keys (depth bits << 24 | rgb)."""
    pts, n = _cloud(pts)
    if keys is None:
        keys = clear_keys(width * height)
    assert keys.dtype == np.uint64 and keys.size == width * height
    lib().oracle_render_rgb(_ptr(pts), n, _ptr(_mat(m)), width, height, _ptr(keys))
    return keys


def resolve_rgb(keys: np.ndarray, background: int = 0) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    out = np.empty(keys.size, dtype=np.uint32)
    lib().oracle_resolve_rgb(_ptr(keys), keys.size, background, _ptr(out))
    return out


def render_basic_threads(pts: np.ndarray, m, width: int, height: int, threads: int = 0,
                         keys: np.ndarray | None = None):
    """render_basic on several host threads; returns (keys, threads used)."""
    pts, n = _cloud(pts)
    if keys is None:
        keys = clear_keys(width * height)
    used = lib().oracle_render_basic_threads(_ptr(pts), n, _ptr(_mat(m)), width, height, _ptr(keys), threads)
    return keys, used


def resolve_basic_threads(keys: np.ndarray, pts: np.ndarray, background: int = 0, threads: int = 0):
    pts, n = _cloud(pts)
    out = np.empty(keys.size, dtype=np.uint32)
    used = lib().oracle_resolve_basic_threads(_ptr(keys), keys.size, _ptr(pts), n, background, _ptr(out), threads)
    return out, used


def clear_hq(npx: int):
    d = np.empty(npx, dtype=np.uint32)
    rg = np.empty(npx, dtype=np.uint64)
    ba = np.empty(npx, dtype=np.uint64)
    lib().oracle_clear_hq(_ptr(d), _ptr(rg), _ptr(ba), npx)
    return d, rg, ba


def render_hq(pts: np.ndarray, m, width: int, height: int, depth_factor: float = 1.01, bufs=None):
    """Depth pass then colour pass; returns (depth u32, rg u64, ba u64)."""
    pts, n = _cloud(pts)
    if bufs is None:
        bufs = clear_hq(width * height)
    d, rg, ba = bufs
    mm = _mat(m)
    lib().oracle_hq_depth(_ptr(pts), n, _ptr(mm), width, height, _ptr(d))
    lib().oracle_hq_color(_ptr(pts), n, _ptr(mm), width, height, FLT(depth_factor), _ptr(d), _ptr(rg), _ptr(ba))
    return d, rg, ba


def hq_channel_sums(pts: np.ndarray, m, width: int, height: int, depth: np.ndarray, depth_factor: float = 1.01):
    pts, n = _cloud(pts)
    npx = width * height
    out = [np.zeros(npx, dtype=np.uint64) for _ in range(4)]
    lib().oracle_hq_channel_sums(_ptr(pts), n, _ptr(_mat(m)), width, height, FLT(depth_factor), _ptr(depth),
                                 *[_ptr(o) for o in out])
    return tuple(out)


def resolve_basic(keys: np.ndarray, pts: np.ndarray, background: int = 0) -> np.ndarray:
    pts, n = _cloud(pts)
    out = np.empty(keys.size, dtype=np.uint32)
    lib().oracle_resolve_basic(_ptr(keys), keys.size, _ptr(pts), n, background, _ptr(out))
    return out


def resolve_hq(rg: np.ndarray, ba: np.ndarray, background: int = 0) -> np.ndarray:
    out = np.empty(rg.size, dtype=np.uint32)
    lib().oracle_resolve_hq(_ptr(rg), _ptr(ba), rg.size, background, _ptr(out))
    return out


def aabb(pts: np.ndarray):
    pts, n = _cloud(pts)
    lo = np.empty(3, dtype=np.float32)
    hi = np.empty(3, dtype=np.float32)
    lib().oracle_aabb(_ptr(pts), n, _ptr(lo), _ptr(hi))
    return lo, hi


def morton_codes(pts: np.ndarray) -> np.ndarray:
    pts, n = _cloud(pts)
    codes = np.empty(n, dtype=np.uint32)
    lib().oracle_morton_codes(_ptr(pts), n, _ptr(codes))
    return codes


def morton_codes63(pts: np.ndarray) -> np.ndarray:
    pts, n = _cloud(pts)
    codes = np.empty(n, dtype=np.uint64)
    lib().oracle_morton_codes63(_ptr(pts), n, _ptr(codes))
    return codes


MORTON, MORTON_SHUFFLE, SHUFFLE, MORTON63, MORTON63_SHUFFLE = 0, 1, 2, 3, 4


def reorder(pts: np.ndarray, seed: int, mode: int, batch: int = 128) -> np.ndarray:
    """perm[new] = old."""
    pts, n = _cloud(pts)
    perm = np.empty(n, dtype=np.uint32)
    rc = lib().oracle_reorder(_ptr(pts), n, seed & ((1 << 64) - 1), mode, batch, _ptr(perm))
    if rc != 0:
        raise ValueError("oracle_reorder rejected its arguments")
    return perm


def gather(pts: np.ndarray, perm: np.ndarray) -> np.ndarray:
    pts, n = _cloud(pts)
    perm = np.ascontiguousarray(perm, dtype=np.uint32)
    out = np.empty_like(pts)
    lib().oracle_gather(_ptr(pts), n, _ptr(perm), _ptr(out))
    return out
