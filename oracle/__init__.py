"""RASTER oracle -- TEST INFRASTRUCTURE ONLY.

Python access to the plain single-threaded CPU oracle in ``raster_oracle.cpp``
(Alg. 1 of the paper, written out).  Only ``tests/``, the package's smoke check
and the benchmark's CPU-baseline leg may import this module; the CUDA library
and its binding never do.

Also holds two independent restatements used to pin the oracle on tiny inputs:
``brute_force`` (all-pairs Chebyshev adjacency + union-find, a different
algorithm from the oracle's neighbour search) and ``project_exact`` (exact
rational arithmetic, then IEEE round-to-nearest, then floor).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "raster_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "libraster_oracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
E_RANGE = 2
NOISE = np.iinfo(np.int64).min
CHEBYSHEV, MANHATTAN = 0, 1  # neighbourhood metrics of Sect. 3.2


def build(force: bool = False) -> str:
    """Compile the oracle: -O2, no fused multiply-add, no fast-math."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        compile_source(_SRC, tmp)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def compile_source(src: str, out: str) -> str:
    """Compile an oracle source file (the real one, or a deliberately broken
    copy made by a test) with the oracle's flags."""
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", src, "-o", out])
    return out


_PR_SRC = os.path.join(_HERE, "praster.cpp")
_PR_LIB_PATH = os.path.join(_HERE, "_build", "libraster_praster.so")
_pr_lib = None


def build_praster(force: bool = False) -> str:
    """Compile the multi-threaded P-RASTER baseline (same flags, plus threads)."""
    os.makedirs(os.path.dirname(_PR_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_PR_LIB_PATH) or os.path.getmtime(_PR_LIB_PATH) < os.path.getmtime(_PR_SRC):
        tmp = _PR_LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-pthread",
                               "-fPIC", "-shared", _PR_SRC, "-o", tmp])
        os.replace(tmp, _PR_LIB_PATH)
    return _PR_LIB_PATH


def _load_praster():
    global _pr_lib
    with _lock:
        if _pr_lib is None:
            L = ctypes.CDLL(build_praster())
            vp, i64, u32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
            L.praster_create.restype = vp
            L.praster_create.argtypes = [dbl, u32, u32, ctypes.c_int]
            L.praster_free.argtypes = [vp]
            L.praster_run.restype = ctypes.c_int
            L.praster_run.argtypes = [vp, vp, i64]
            L.praster_labels.restype = ctypes.c_int
            L.praster_labels.argtypes = [vp, vp, i64, vp]
            for name in ("praster_n_tiles", "praster_n_significant", "praster_n_clusters", "praster_n_kept"):
                getattr(L, name).restype = i64
                getattr(L, name).argtypes = [vp]
            L.praster_copy_kept.argtypes = [vp, vp, vp, vp]
            L.praster_times.argtypes = [vp, vp]
            _pr_lib = L
    return _pr_lib


def praster(xy, precision: float, tau: int, mu: int, threads: int, with_labels: bool = False, sort: bool = True):
    """P-RASTER (Sect. 3.5, Alg. 2-3) on `threads` host threads: per-thread
    maps, join, tau filter, per-slice clustering, border joins right to left,
    then (optionally) labels.  Returns (Result, labels or None, seconds as
    {contract, agglomerate, labels}).  The rows come cluster by cluster;
    sort=True puts them in (ix, iy) order, like the oracle's."""
    a = _xy(xy)
    assert a.shape[1] == 2
    L = _load_praster()
    h = L.praster_create(scale_of(precision), tau, mu, int(threads))
    try:
        st = L.praster_run(h, a.ctypes.data, a.shape[0])
        k = L.praster_n_kept(h)
        key, cnt, cid = np.empty(k, np.int64), np.empty(k, np.uint64), np.empty(k, np.int64)
        L.praster_copy_kept(h, key.ctypes.data, cnt.ctypes.data, cid.ctypes.data)
        lab = None
        if with_labels:
            lab = np.empty(a.shape[0], np.int64)
            L.praster_labels(h, a.ctypes.data, a.shape[0], lab.ctypes.data)
        t = np.zeros(3)
        L.praster_times(h, t.ctypes.data)
        if sort and k:
            o = tile_order(key)
            key, cnt, cid = key[o], cnt[o], cid[o]
        res = Result(status=st, points=int(a.shape[0]), n_tiles=L.praster_n_tiles(h),
                     n_significant=L.praster_n_significant(h), n_clusters=L.praster_n_clusters(h),
                     key=key, count=cnt, cid=cid)
        return res, lab, {"contract": float(t[0]), "agglomerate": float(t[1]), "labels": float(t[2])}
    finally:
        L.praster_free(h)


def load_library(path: str):
    """Load an oracle shared library and declare its entry points."""
    L = ctypes.CDLL(path)
    _declare(L)
    return L


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = load_library(_LIB_PATH)
    return _lib


def _declare(L):
    vp, i64, u32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
    L.oracle_create.restype = vp
    L.oracle_create.argtypes = [dbl, u32, u32]
    L.oracle_create_ex.restype = vp
    L.oracle_create_ex.argtypes = [dbl, u32, u32, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.oracle_free.argtypes = [vp]
    L.oracle_add.restype = ctypes.c_int
    L.oracle_add.argtypes = [vp, vp, i64]
    L.oracle_finish.restype = ctypes.c_int
    L.oracle_finish.argtypes = [vp]
    for name in ("oracle_points", "oracle_n_tiles", "oracle_n_significant", "oracle_n_kept",
                 "oracle_n_clusters"):
        getattr(L, name).restype = i64
        getattr(L, name).argtypes = [vp]
    L.oracle_status.restype = ctypes.c_int
    L.oracle_status.argtypes = [vp]
    L.oracle_copy_tiles.argtypes = [vp, vp, vp]
    L.oracle_copy_kept.argtypes = [vp, vp, vp, vp]
    L.oracle_labels.restype = ctypes.c_int
    L.oracle_labels.argtypes = [vp, vp, i64, vp]
    L.oracle_project.argtypes = [vp, i64, dbl, vp, vp, ctypes.c_int]
    L.oracle_count_keys.argtypes = [vp, i64, dbl, vp, i64, vp, ctypes.c_int]
    L.oracle_point_groups.restype = i64
    L.oracle_point_groups.argtypes = [vp, vp, i64, vp, vp, i64]


def scale_of(precision: float) -> float:
    """s = 10^precision as one double: exact for integer precisions 0..22,
    otherwise the host C library's pow(10, precision)."""
    if precision == int(precision) and 0 <= precision <= 22:
        return float(10 ** int(precision))
    return 10.0 ** float(precision)


def _xy(xy) -> np.ndarray:
    a = np.ascontiguousarray(xy, dtype=np.float64)
    assert a.ndim == 2 and a.shape[1] in (2, 3)
    return a


@dataclass
class Result:
    status: int
    points: int
    n_tiles: int          # D: distinct tiles
    n_significant: int    # S: tiles with count >= tau
    n_clusters: int
    key: np.ndarray       # kept tiles, (ix, iy) order
    count: np.ndarray
    cid: np.ndarray


class Oracle:
    """Chunked oracle session: add() per chunk, then finish()."""

    def __init__(self, precision: float, tau: int, mu: int, scale: float | None = None, lib=None,
                 metric: int = 0, delta: int = 1, groups: bool = False, dims: int = 2):
        """dims: coordinates per point, 2 or 3 (Sect. 3.6, higher dimensions);
        the 2 x 2 group rule applies to two coordinates only."""
        assert dims in (2, 3) and not (groups and dims == 3)
        self.L = lib if lib is not None else _load()
        self.scale = scale_of(precision) if scale is None else scale
        self.dims = dims
        if metric == CHEBYSHEV and delta == 1 and not groups and dims == 2:
            self.h = self.L.oracle_create(self.scale, tau, mu)
        else:
            self.h = self.L.oracle_create_ex(self.scale, tau, mu, metric, delta, 1 if groups else 0, dims)

    def __del__(self):
        if getattr(self, "h", None):
            self.L.oracle_free(self.h)
            self.h = None

    def add(self, xy) -> int:
        a = _xy(xy)
        assert a.shape[1] == self.dims
        return self.L.oracle_add(self.h, a.ctypes.data, a.shape[0])

    def finish(self) -> Result:
        st = self.L.oracle_finish(self.h)
        k = self.L.oracle_n_kept(self.h)
        key = np.empty(k, np.int64)
        cnt = np.empty(k, np.uint64)
        cid = np.empty(k, np.int64)
        self.L.oracle_copy_kept(self.h, key.ctypes.data, cnt.ctypes.data, cid.ctypes.data)
        return Result(status=st, points=self.L.oracle_points(self.h), n_tiles=self.L.oracle_n_tiles(self.h),
                      n_significant=self.L.oracle_n_significant(self.h),
                      n_clusters=self.L.oracle_n_clusters(self.h), key=key, count=cnt, cid=cid)

    def tiles(self) -> tuple[np.ndarray, np.ndarray]:
        d = self.L.oracle_n_tiles(self.h)
        key = np.empty(d, np.int64)
        cnt = np.empty(d, np.uint64)
        self.L.oracle_copy_tiles(self.h, key.ctypes.data, cnt.ctypes.data)
        return key, cnt

    def point_groups(self, xy) -> tuple[np.ndarray, np.ndarray]:
        """RASTER' (Sect. 3.4): (row_start, point_index) over the kept tiles in
        the order of finish()'s rows, indices increasing within a row."""
        a = _xy(xy)
        assert a.shape[1] == self.dims
        k = self.L.oracle_n_kept(self.h)
        row_start = np.empty(k + 1, np.int64)
        idx = np.empty(max(a.shape[0], 1), np.int64)
        m = self.L.oracle_point_groups(self.h, a.ctypes.data, a.shape[0], row_start.ctypes.data, idx.ctypes.data,
                                       idx.shape[0])
        return row_start, idx[:m]

    def labels(self, xy) -> tuple[int, np.ndarray]:
        a = _xy(xy)
        assert a.shape[1] == self.dims
        out = np.empty(a.shape[0], np.int64)
        st = self.L.oracle_labels(self.h, a.ctypes.data, a.shape[0], out.ctypes.data)
        return st, out


def raster(xy, precision: float, tau: int, mu: int, scale: float | None = None, chunks: int = 1,
           with_labels: bool = False, lib=None, metric: int = 0, delta: int = 1, groups: bool = False):
    """Run the oracle on one point set; optionally in ``chunks`` contiguous chunks.
    ``metric``/``delta`` choose neighbors(u, delta) (Sect. 3.2; default Chebyshev 1)
    and ``groups`` adds the 2 x 2 group rule of Sect. 3.6."""
    a = _xy(xy)
    o = Oracle(precision, tau, mu, scale, lib=lib, metric=metric, delta=delta, groups=groups, dims=a.shape[1])
    n = a.shape[0]
    for c in range(chunks):
        o.add(a[n * c // chunks: n * (c + 1) // chunks])
    r = o.finish()
    if with_labels:
        st, lab = o.labels(a)
        return r, lab, o
    return r, o


def project(xy, scale: float) -> tuple[np.ndarray, np.ndarray]:
    a = _xy(xy)
    keys = np.empty(a.shape[0], np.int64)
    ok = np.empty(a.shape[0], np.uint8)
    _load().oracle_project(a.ctypes.data, a.shape[0], scale, keys.ctypes.data, ok.ctypes.data, a.shape[1])
    return keys, ok.astype(bool)


def count_keys(xy, scale: float, keys, lib=None) -> np.ndarray:
    """Exact number of points in each of the given tiles (range-error points
    count nowhere); one pass over the points, used to check sampled outputs."""
    a = _xy(xy)
    k = np.ascontiguousarray(keys, dtype=np.int64)
    out = np.empty(k.shape[0], np.uint64)
    (lib if lib is not None else _load()).oracle_count_keys(a.ctypes.data, a.shape[0], scale, k.ctypes.data, k.shape[0], out.ctypes.data,
                              a.shape[1])
    return out


# ---------------------------------------------------------------------------
# Key helpers (plain definitions of the packing convention).
def pack(ix, iy):
    ix = np.asarray(ix, dtype=np.int64)
    iy = np.asarray(iy, dtype=np.int64)
    return ((ix << 32) | (iy & 0xFFFFFFFF)).astype(np.int64)


def unpack(key):
    key = np.asarray(key, dtype=np.int64)
    return (key >> 32).astype(np.int64), (key & 0xFFFFFFFF).astype(np.uint32).astype(np.int32).astype(np.int64)


BIAS3 = 1 << 20  # three coordinates: 21-bit fields, each index offset by 2^20


def pack3(ix, iy, iz):
    ix, iy, iz = (np.asarray(v, dtype=np.int64) for v in (ix, iy, iz))
    return ((ix + BIAS3) << 42) | ((iy + BIAS3) << 21) | (iz + BIAS3)


def unpack3(key):
    key = np.asarray(key, dtype=np.int64)
    return tuple(((key >> sh) & 0x1FFFFF) - BIAS3 for sh in (42, 21, 0))


def tile_order(key) -> np.ndarray:
    """Indices that sort keys in (ix, iy) lexicographic order."""
    ix, iy = unpack(key)
    return np.lexsort((iy, ix))


# ---------------------------------------------------------------------------
# Independent restatements used only to pin the oracle on small inputs.
def project_exact(x: float, scale: float):
    """floor(RN(x * s)) by exact rational arithmetic: the product of the two
    binary64 values is formed exactly, rounded once to the nearest double
    (ties to even, which is what float(Fraction) does), then floored.
    Returns None when the result is not a valid tile index."""
    import math
    if not (math.isfinite(x) and math.isfinite(scale)):
        return None
    exact = Fraction(x) * Fraction(scale)
    try:
        q = float(exact)  # correctly rounded
    except OverflowError:
        return None
    if not math.isfinite(q):
        return None
    f = math.floor(q)
    if f < -(2**31 - 1) or f > 2**31 - 2:
        return None
    return f


def brute_force(keys, counts, tau: int, mu: int, metric: int = CHEBYSHEV, delta: int = 1, significant=None,
                dims: int = 2):
    """RASTER agglomeration by all-pairs adjacency: tiles with count >= tau (or
    those of the boolean mask ``significant``) are joined when their Chebyshev
    (largest coordinate difference) or Manhattan (sum of differences) distance
    is at most ``delta``, via union-find; components with at least mu tiles are
    kept; the id is the lexicographically smallest member.  O(T^2); tiny T."""
    keys = np.asarray(keys, dtype=np.int64)
    counts = np.asarray(counts)
    sig = keys[np.asarray(significant, dtype=bool)] if significant is not None else keys[counts >= tau]
    coords = np.stack(unpack3(sig) if dims == 3 else unpack(sig), axis=1).astype(np.int64)
    t = len(sig)
    parent = list(range(t))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    def near(a, b):
        d = np.abs(coords[a] - coords[b])
        return int(d.max() if metric == CHEBYSHEV else d.sum()) <= delta

    for a in range(t):
        for b in range(a + 1, t):
            if near(a, b):
                ra, rb = find(a), find(b)
                if ra != rb:
                    parent[rb] = ra
    comps: dict[int, list[int]] = {}
    for a in range(t):
        comps.setdefault(find(a), []).append(a)
    rows = []
    n_clusters = 0
    for members in comps.values():
        if len(members) < mu:
            continue
        n_clusters += 1
        best = min(members, key=lambda m: tuple(int(c) for c in coords[m]))
        for m in members:
            rows.append((int(sig[m]), int(sig[best])))
    rows.sort(key=lambda r: r[0] if dims == 3 else (r[0] >> 32, np.int32(np.uint32(r[0] & 0xFFFFFFFF))))
    cnt_of = {int(k): int(c) for k, c in zip(keys, counts)}
    key = np.array([r[0] for r in rows], dtype=np.int64)
    cid = np.array([r[1] for r in rows], dtype=np.int64)
    cnt = np.array([cnt_of[int(k)] for k in key], dtype=np.uint64)
    return key, cnt, cid, n_clusters
