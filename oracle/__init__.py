"""CPU oracle for the exact isotropic median / percentile filter.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
``cpu_baseline`` / ``--impl reference`` legs are the only users. The CUDA product path
(``paper_2505_22938_gb300``) never imports this package, and this package never imports
it; the two share no code. Inputs for both come from ``datagen``.

Parts:
  * kernel rasterisers (own code, independent of the library's host geometry):
    disk (Eq. 3), axis-aligned ellipse, convex polygon (Sec. 6.2.3), explicit row spans;
  * the filter itself (``fim_oracle.cpp``): clamp gather + ``std::nth_element``;
  * tile-footprint geometry used to pin the Fig. 10 counts.

Every function states the passage it follows. Where the paper is silent or ambiguous this
package reads it as follows: the circle is dx^2 + dy^2 <= r^2 (Eq. 3 on the lattice; the
figures' counts use r^2 + r, available as a disk limit); an even tap count takes the lower
median (rank (n - 1) // 2); floats are ordered by IEEE totalOrder (-0 < +0); borders clamp
to the edge; polygon boundaries are inclusive with a 1e-9 tolerance; a spatially varying
percentile (Fig. 14) is a float32 map with one percentile per output pixel, clamped to
[0, 100] with NaN counted as 0, and rounded to a rank like a single percentile.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fim_oracle.cpp")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libfim_oracle.so")
_lock = threading.Lock()
_lib = None

DTYPE_CODE = {"u8": 0, "u16": 1, "f32": 2}
NP_DTYPE = {"u8": np.uint8, "u16": np.uint16, "f32": np.float32}


def dtype_name(a: np.ndarray) -> str:
    for k, v in NP_DTYPE.items():
        if a.dtype == v:
            return k
    raise TypeError(f"unsupported dtype {a.dtype}")


# --------------------------------------------------------------------------------------
# Build / load
# --------------------------------------------------------------------------------------

def build(force: bool = False) -> str:
    """Compile the C++ oracle into ``oracle/_build/libfim_oracle.so`` (g++, OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.fim_oracle_filter.restype = ctypes.c_int
            lib.fim_oracle_filter.argtypes = [
                ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t,
                ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                ctypes.c_int, ctypes.c_int]
            lib.fim_oracle_points.restype = ctypes.c_int
            lib.fim_oracle_points.argtypes = [
                ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
            lib.fim_oracle_filter_ranks.restype = ctypes.c_int
            lib.fim_oracle_filter_ranks.argtypes = [
                ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t,
                ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                ctypes.c_void_p, ctypes.c_int]
            lib.fim_oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().fim_oracle_max_threads())


# --------------------------------------------------------------------------------------
# Kernel shapes: offset sets K as (dx, dy) int32 arrays, row-major in (dy, dx).
# --------------------------------------------------------------------------------------

def disk_offsets(r: int) -> np.ndarray:
    """Eq. 3 on the integer lattice: all (dx, dy) with dx^2 + dy^2 <= r^2."""
    return disk_limit_offsets(r, r * r)


def disk_limit_offsets(r: int, limit: int) -> np.ndarray:
    """All (dx, dy) with |dx|,|dy| <= r and dx^2 + dy^2 <= limit (limit = r^2 + r gives the
    slightly fuller disk whose counts match Fig. 3b and Fig. 10)."""
    pts = [(dx, dy) for dy in range(-r, r + 1) for dx in range(-r, r + 1) if dx * dx + dy * dy <= limit]
    return np.asarray(pts, dtype=np.int32).reshape(-1, 2)


def ellipse_offsets(a: int, b: int) -> np.ndarray:
    """Axis-aligned ellipse, semi-axis a along x and b along y: (dx/a)^2 + (dy/b)^2 <= 1,
    tested exactly in integers as dx^2 b^2 + dy^2 a^2 <= a^2 b^2."""
    pts = [(dx, dy) for dy in range(-b, b + 1) for dx in range(-a, a + 1)
           if dx * dx * b * b + dy * dy * a * a <= a * a * b * b]
    return np.asarray(pts, dtype=np.int32).reshape(-1, 2)


def regular_polygon_vertices(sides: int, circumradius: float, phase_deg: float = 0.0) -> np.ndarray:
    """Counter-clockwise vertices at angles phase + 360k/sides degrees."""
    ang = np.deg2rad(phase_deg + 360.0 * np.arange(sides) / sides)
    return np.stack([circumradius * np.cos(ang), circumradius * np.sin(ang)], axis=1)


def polygon_offsets(verts: np.ndarray, eps: float = 1e-9) -> np.ndarray:
    """Lattice points inside or on a convex polygon given counter-clockwise (Sec. 6.2.3: a
    polygon kernel replaces the circle test of Eq. 3 by a point-in-polygon test).
    A point p is inside iff cross(v[i+1]-v[i], p-v[i]) >= -eps for every edge i."""
    v = np.asarray(verts, dtype=np.float64)
    m = len(v)
    x0, x1 = int(math.floor(v[:, 0].min())) - 1, int(math.ceil(v[:, 0].max())) + 1
    y0, y1 = int(math.floor(v[:, 1].min())) - 1, int(math.ceil(v[:, 1].max())) + 1
    pts = []
    for dy in range(y0, y1 + 1):
        for dx in range(x0, x1 + 1):
            ok = True
            for i in range(m):
                ax, ay = v[i]
                bx, by = v[(i + 1) % m]
                if (bx - ax) * (dy - ay) - (by - ay) * (dx - ax) < -eps:
                    ok = False
                    break
            if ok:
                pts.append((dx, dy))
    return np.asarray(pts, dtype=np.int32).reshape(-1, 2)


def spans_offsets(lo, hi, dy0: int) -> np.ndarray:
    """Kernel given row by row: row dy0+i covers dx in [lo[i], hi[i]]."""
    pts = []
    for i, (a, b) in enumerate(zip(lo, hi)):
        for dx in range(int(a), int(b) + 1):
            pts.append((dx, dy0 + i))
    return np.asarray(pts, dtype=np.int32).reshape(-1, 2)


def median_rank(n: int) -> int:
    """0-based rank of the median of n values; the lower median when n is even (Sec. 3.1)."""
    return (n - 1) // 2


def percentile_rank(n: int, pct: float) -> int:
    """0-based rank for a percentile in [0, 100]: round(pct/100 * (n-1)), half away from zero."""
    t = pct / 100.0 * (n - 1)
    return int(math.floor(t + 0.5))


def percentile_rank_map(n: int, pct: np.ndarray) -> np.ndarray:
    """Per-pixel 0-based ranks for a map of percentiles (a spatially varying percentile,
    Fig. 14): each value is clamped to [0, 100] (NaN counts as 0), widened to fp64, and
    rounded as in percentile_rank: floor(p / 100 * (n - 1) + 1/2), evaluated in that order."""
    p = np.asarray(pct, dtype=np.float32).astype(np.float64)
    p = np.where(np.isnan(p), 0.0, np.clip(p, 0.0, 100.0))
    t = p / 100.0 * float(n - 1)
    return np.floor(t + 0.5).astype(np.int32)


# --------------------------------------------------------------------------------------
# The filter
# --------------------------------------------------------------------------------------

def median_filter(img: np.ndarray, offsets: np.ndarray, rank: int | None = None, nthreads: int = 0) -> np.ndarray:
    """Rank-order filter of a 2-D image (clamp-to-edge), rank defaults to the median."""
    img = np.ascontiguousarray(img)
    assert img.ndim == 2
    dt = dtype_name(img)
    off = np.ascontiguousarray(offsets, dtype=np.int32)
    n = off.shape[0]
    k = median_rank(n) if rank is None else int(rank)
    dx = np.ascontiguousarray(off[:, 0])
    dy = np.ascontiguousarray(off[:, 1])
    out = np.empty_like(img)
    h, w = img.shape
    rc = _load().fim_oracle_filter(DTYPE_CODE[dt], img.ctypes.data, img.strides[0], out.ctypes.data,
                                   out.strides[0], w, h, dx.ctypes.data, dy.ctypes.data, n, k, nthreads)
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return out


def rank_map_filter(img: np.ndarray, offsets: np.ndarray, ranks: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """Rank-order filter with its own 0-based rank at every pixel (ranks: same shape as img)."""
    img = np.ascontiguousarray(img)
    assert img.ndim == 2 and ranks.shape == img.shape
    dt = dtype_name(img)
    off = np.ascontiguousarray(offsets, dtype=np.int32)
    n = off.shape[0]
    dx = np.ascontiguousarray(off[:, 0])
    dy = np.ascontiguousarray(off[:, 1])
    rk = np.ascontiguousarray(ranks, dtype=np.int32)
    out = np.empty_like(img)
    h, w = img.shape
    rc = _load().fim_oracle_filter_ranks(DTYPE_CODE[dt], img.ctypes.data, img.strides[0], out.ctypes.data,
                                         out.strides[0], w, h, dx.ctypes.data, dy.ctypes.data, n,
                                         rk.ctypes.data, nthreads)
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return out


def median_points(img: np.ndarray, offsets: np.ndarray, xs, ys, rank: int | None = None,
                  nthreads: int = 0) -> np.ndarray:
    """The same definition evaluated only at pixels (xs[i], ys[i])."""
    img = np.ascontiguousarray(img)
    dt = dtype_name(img)
    off = np.ascontiguousarray(offsets, dtype=np.int32)
    n = off.shape[0]
    k = median_rank(n) if rank is None else int(rank)
    dx = np.ascontiguousarray(off[:, 0])
    dy = np.ascontiguousarray(off[:, 1])
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    vals = np.empty(xs.shape[0], dtype=img.dtype)
    h, w = img.shape
    rc = _load().fim_oracle_points(DTYPE_CODE[dt], img.ctypes.data, img.strides[0], w, h, xs.ctypes.data,
                                   ys.ctypes.data, xs.shape[0], dx.ctypes.data, dy.ctypes.data, n, k,
                                   vals.ctypes.data, nthreads)
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return vals


# --------------------------------------------------------------------------------------
# Tile geometry (Sec. 4.1, Fig. 10)
# --------------------------------------------------------------------------------------

def tile_footprint_size(offsets: np.ndarray, tile_w: int, tile_h: int) -> int:
    """Number of input pixels read by at least one window of a tile_w x tile_h output tile:
    the union of (p + K) over the tile's pixels p (Fig. 10's rounded rectangle)."""
    off = np.asarray(offsets, dtype=np.int64)
    xmin, ymin = off.min(axis=0)
    xmax, ymax = off.max(axis=0)
    W = tile_w + int(xmax - xmin)
    H = tile_h + int(ymax - ymin)
    cover = np.zeros((H, W), dtype=bool)
    for dx, dy in off:
        cover[dy - ymin: dy - ymin + tile_h, dx - xmin: dx - xmin + tile_w] = True
    return int(cover.sum())


def candidate_median_ranks(n_taps: int, footprint: int) -> int:
    """How many ranks of a footprint can be the median of some window inside it (Fig. 10):
    a window holds n of the N footprint values, so its median rank k = (n-1)/2 within the
    window is at least k and at most N-1-(n-1-k) within the footprint."""
    k = median_rank(n_taps)
    return (footprint - 1 - (n_taps - 1 - k)) - k + 1
