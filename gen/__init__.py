"""Seeded synthetic workloads for RASTER (inputs only; no clustering arithmetic).

The paper's own generator and data are not available.  Its workload -- clusters
of uniform points around random centres, shuffled (Sect. 4.2, "Data") -- is
stood in for by the square-cluster-plus-noise recipes below, generated by the
C routine in ``raster_gen.c`` (a pure function of seed and position, so any
slice can be produced on its own).

Both the CPU oracle and the CUDA path read the arrays this module returns.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, asdict

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "raster_gen.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libraster_gen.so")
_lock = threading.Lock()
_lib = None

HALF_WIDTH = 0.05  # clusters are 0.1 x 0.1 squares


def build(force: bool = False) -> str:
    """Compile the generator (plain C, IEEE arithmetic without contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.gen_points_range.restype = ctypes.c_int
            lib.gen_points_range.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                             ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                                             ctypes.c_uint64, ctypes.c_int]
            lib.gen_rng_at.restype = ctypes.c_uint64
            lib.gen_rng_at.argtypes = [ctypes.c_uint64] * 3
            lib.gen_perm_apply.restype = ctypes.c_uint64
            lib.gen_perm_apply.argtypes = [ctypes.c_uint64] * 3
            _lib = lib
    return _lib


@dataclass(frozen=True)
class Workload:
    """One clustering problem: points plus the RASTER parameters to run it with."""
    n: int
    clusters: int
    cluster_points: int
    canvas: float
    precision: float
    tau: int
    mu: int
    seed: int
    shuffle: bool = True

    def asdict(self):
        return asdict(self)


# Plain-RASTER workloads (2-D FP64, p = 2, tau = 5, mu = 4).
C1_1M = Workload(n=1_000_000, clusters=1_000, cluster_points=900_000, canvas=100.0,
                 precision=2, tau=5, mu=4, seed=1)
C2_50M = Workload(n=50_000_000, clusters=100_000, cluster_points=45_000_000, canvas=1000.0,
                  precision=2, tau=5, mu=4, seed=2)
C3_500M = Workload(n=500_000_000, clusters=1_000_000, cluster_points=475_000_000, canvas=3000.0,
                   precision=2, tau=5, mu=4, seed=3)
NAMED = {"1m": C1_1M, "50m": C2_50M, "500m": C3_500M}


def nthreads_default() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def points_into(out, w: Workload, lo: int = 0, hi: int | None = None, nthreads: int | None = None):
    """Write positions [lo, hi) of workload ``w`` into ``out`` (a C-contiguous
    float64 buffer of shape (hi-lo, 2): numpy array or pinned CPU tensor)."""
    lib = _load()
    hi = w.n if hi is None else hi
    if isinstance(out, np.ndarray):
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.shape == (hi - lo, 2)
        ptr = out.ctypes.data
    else:  # torch CPU tensor
        assert out.dtype.__str__() == "torch.float64" and out.is_contiguous() and tuple(out.shape) == (hi - lo, 2)
        ptr = out.data_ptr()
    rc = lib.gen_points_range(ptr, w.n, w.clusters, w.cluster_points, float(w.canvas), HALF_WIDTH,
                              w.seed, 1 if w.shuffle else 0, lo, hi, nthreads or nthreads_default())
    if rc != 0:
        raise ValueError("generator rejected arguments")
    return out


def points(w: Workload, lo: int = 0, hi: int | None = None, nthreads: int | None = None) -> np.ndarray:
    hi = w.n if hi is None else hi
    out = np.empty((hi - lo, 2), dtype=np.float64)
    return points_into(out, w, lo, hi, nthreads)


def rng_at(seed: int, stream: int, ctr: int) -> int:
    return int(_load().gen_rng_at(seed & (2**64 - 1), stream, ctr))


def u01(seed: int, stream: int, ctr: int) -> float:
    return (rng_at(seed, stream, ctr) >> 11) * 2.0 ** -53


def perm_apply(n: int, seed: int, i: int) -> int:
    return int(_load().gen_perm_apply(n, seed, i))


# Per-instance parameter choices for the batched and served workloads.
PRECISIONS = (1, 2, 3)
TAUS = (3, 5, 8)
MUS = (2, 4)
_ST_SIZE, _ST_PARAM, _ST_SEED, _ST_ARRIVAL, _ST_CHUNKS = 11, 12, 13, 14, 15


def _log_uniform_size(seed: int, i: int, lo: int, hi: int) -> int:
    u = u01(seed, _ST_SIZE, i)
    return int(math.floor(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))))


def _instance(seed: int, i: int, size: int, noise_frac: float) -> Workload:
    clusters = max(1, size // 500)
    noise = int(size * noise_frac)
    canvas = 100.0 * math.sqrt(size / 1e6) + 1.0
    r = rng_at(seed, _ST_PARAM, i)
    p = PRECISIONS[r % 3]
    tau = TAUS[(r >> 8) % 3]
    mu = MUS[(r >> 16) % 2]
    inst_seed = rng_at(seed, _ST_SEED, i)
    return Workload(n=size, clusters=clusters, cluster_points=size - noise, canvas=canvas,
                    precision=p, tau=tau, mu=mu, seed=inst_seed)


def batch_instances(count: int = 4096, seed: int = 4, lo: int = 1_000, hi: int = 2_000_000) -> list[Workload]:
    """The batched workload: ``count`` independent instances, sizes log-uniform in
    [lo, hi), size/500 square clusters plus 10% noise on [0, 100*sqrt(size/1e6)+1)^2,
    per-instance p in {1,2,3}, tau in {3,5,8}, mu in {2,4}."""
    return [_instance(seed, i, _log_uniform_size(seed, i, lo, hi), 0.10) for i in range(count)]


@dataclass(frozen=True)
class Request:
    """A served clustering request: a workload, its arrival time and its chunking."""
    rid: int
    arrival_s: float
    work: Workload
    chunks: int


def serve_requests(rate_per_s: float, duration_s: float, seed: int = 5, lo: int = 10_000,
                   hi: int = 20_000_000, max_chunks: int = 8) -> list[Request]:
    """Poisson arrivals at ``rate_per_s`` for ``duration_s``; sizes log-uniform in
    [lo, hi), each sent as 1..max_chunks chunks; per-request p/tau/mu as for the
    batched workload."""
    out, t, i = [], 0.0, 0
    while True:
        u = u01(seed, _ST_ARRIVAL, i)
        t += -math.log1p(-u) / rate_per_s
        if t >= duration_s:
            break
        w = _instance(seed, i, _log_uniform_size(seed, i, lo, hi), 0.10)
        chunks = 1 + rng_at(seed, _ST_CHUNKS, i) % max_chunks
        out.append(Request(rid=i, arrival_s=t, work=w, chunks=int(chunks)))
        i += 1
    return out


def chunk_bounds(n: int, chunks: int) -> list[tuple[int, int]]:
    """Split [0, n) into ``chunks`` nearly equal contiguous ranges."""
    return [(n * c // chunks, n * (c + 1) // chunks) for c in range(chunks)]


# ---------------------------------------------------------------------------
# Three-coordinate points: cubes of uniform points (centres uniform in the
# canvas cube) plus uniform noise, shuffled.  numpy's seeded generator; the
# same arrays on any machine.

CUBES_100M = dict(n_clusters=100_000, per=900, side=0.1, canvas=100.0, noise=10_000_000, seed=21)


def cubes3(n_clusters: int, per: int, side: float, canvas: float, noise: int, seed: int) -> np.ndarray:
    g = np.random.default_rng(seed)
    centres = g.uniform(0.0, canvas, (n_clusters, 3))
    out = np.empty((n_clusters * per + noise, 3), dtype=np.float64)
    out[:n_clusters * per] = (centres[:, None, :] + g.uniform(-side / 2, side / 2, (n_clusters, per, 3))).reshape(-1, 3)
    out[n_clusters * per:] = g.uniform(0.0, canvas, (noise, 3))
    return out[g.permutation(out.shape[0])]
