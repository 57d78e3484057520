"""GB300-native RASTER (contraction clustering) -- Python binding.

Thin wrapper over the C ABI in ``include/raster.h`` (libraster.so): argument
marshalling only; every step of the clustering runs in the CUDA kernels.
PyTorch supplies device memory and streams.

    r = Raster(precision=2, tau=5, mu=4)
    r.contract(xy_cuda)            # (n, 2) float64 CUDA tensor; callable per chunk
    res = r.agglomerate()          # kept tiles: key, count, cid (CUDA tensors)
    labels = r.point_labels(xy_cuda)
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _native
from ._native import CHEBYSHEV, INVALID_KEY, MANHATTAN, NOISE, RasterError, check, lib

__all__ = ["Raster", "Result", "RasterError", "NOISE", "CHEBYSHEV", "MANHATTAN", "lib", "build", "pack", "unpack",
           "pack3", "unpack3"]


def build(force: bool = False) -> str:
    from . import builder as _b
    return _b.build(force=force)


def pack(ix: torch.Tensor, iy: torch.Tensor) -> torch.Tensor:
    return (ix.to(torch.int64) << 32) | (iy.to(torch.int64) & 0xFFFFFFFF)


def unpack(key: torch.Tensor):
    return key >> 32, (key & 0xFFFFFFFF).to(torch.int32).to(torch.int64)


BIAS3 = 1 << 20  # three coordinates: 21-bit index fields, each offset by 2^20


def pack3(ix: torch.Tensor, iy: torch.Tensor, iz: torch.Tensor) -> torch.Tensor:
    ix, iy, iz = (t.to(torch.int64) for t in (ix, iy, iz))
    return ((ix + BIAS3) << 42) | ((iy + BIAS3) << 21) | (iz + BIAS3)


def unpack3(key: torch.Tensor):
    return tuple(((key >> sh) & 0x1FFFFF) - BIAS3 for sh in (42, 21, 0))


class _DeviceArray:
    """Wraps a device pointer owned by the library for torch.as_tensor."""

    def __init__(self, ptr: int, n: int, typestr: str, device: torch.device):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr or 0, False),
                                         "version": 3, "strides": None}
        self.device = device


def _view(ptr: int, n: int, dtype: torch.dtype, device: torch.device) -> torch.Tensor:
    if n == 0:
        return torch.empty(0, dtype=dtype, device=device)
    typestr = {torch.int64: "<i8", torch.int32: "<i4"}[dtype]
    return torch.as_tensor(_DeviceArray(ptr, n, typestr, device), device=device)


@dataclass
class Result:
    """Tiles of kept clusters (one row per tile) and run statistics."""
    key: torch.Tensor     # int64 packed tile keys
    count: torch.Tensor   # int64 points per tile
    cid: torch.Tensor     # int64 cluster id (key of the cluster's (ix, iy)-smallest tile)
    n_clusters: int
    n_distinct: int
    n_significant: int
    n_points: int
    status: int
    dims: int = 2  # coordinates per point of the handle that produced it

    def sorted(self) -> "Result":
        """Rows in (ix, iy[, iz]) order (the library's row order is unspecified)."""
        if self.key.numel() == 0:
            return self
        if self.dims == 3:  # integer key order is (ix, iy, iz) order
            order = torch.argsort(self.key, stable=True)
        else:
            ix, iy = unpack(self.key)
            order = torch.argsort(iy, stable=True)
            order = order[torch.argsort(ix[order], stable=True)]
        return Result(self.key[order], self.count[order], self.cid[order], self.n_clusters, self.n_distinct,
                      self.n_significant, self.n_points, self.status, self.dims)


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_points(xy: torch.Tensor, where: str, dims: int = 2):
    if not (xy.is_cuda and xy.dtype == torch.float64 and xy.dim() == 2 and xy.shape[1] == dims and xy.is_contiguous()):
        raise ValueError(f"{where}: expected a contiguous (n, {dims}) float64 CUDA tensor")


class Raster:
    """One RASTER problem (precision, tau, mu) with a device-resident tile table."""

    def __init__(self, precision: float, tau: int, mu: int, metric: int = CHEBYSHEV, delta: int = 1,
                 groups: bool = False, dims: int = 2):
        """metric/delta: neighbors(u, delta) (Sect. 3.2; default Chebyshev 1);
        groups: the 2 x 2 group rule of Sect. 3.6; dims: coordinates per
        point, 2 or 3 (Sect. 3.6, higher dimensions)."""
        self._L = lib()
        self.dims = int(dims)
        h = ctypes.c_void_p()
        if metric == CHEBYSHEV and delta == 1 and not groups and dims == 2:
            check(self._L.raster_create(float(precision), int(tau), int(mu), ctypes.byref(h)), "raster_create")
        else:
            p = _native.Params(float(precision), int(tau), int(mu), int(metric), int(delta), 1 if groups else 0,
                               int(dims))
            check(self._L.raster_create_ex(ctypes.byref(p), ctypes.byref(h)), "raster_create_ex")
        self._h = h
        self.precision, self.tau, self.mu = precision, tau, mu
        self.metric, self.delta, self.groups = metric, delta, groups
        self.device = torch.device("cuda", torch.cuda.current_device())

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._L.raster_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    @property
    def scale(self) -> float:
        return self._L.raster_get_scale(self._h)

    @property
    def capacity(self) -> int:
        return self._L.raster_table_capacity(self._h)

    # -- hot path ------------------------------------------------------------
    def reserve(self, n_tiles: int):
        check(self._L.raster_reserve(self._h, int(n_tiles)), "raster_reserve")

    def contract(self, xy: torch.Tensor, stream=None):
        _check_points(xy, "contract", self.dims)
        check(self._L.raster_contract(self._h, ctypes.c_void_p(xy.data_ptr()), xy.shape[0], _stream_ptr(stream)),
              "raster_contract")

    def contract_keys(self, xy: torch.Tensor, keys: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """contract(xy), also writing each point's tile key (CUDA int64, n
        entries; INVALID_KEY for a point that does not project) for
        key_labels."""
        _check_points(xy, "contract_keys", self.dims)
        if keys is None:
            keys = torch.empty(xy.shape[0], dtype=torch.int64, device=xy.device)
        assert keys.is_cuda and keys.dtype == torch.int64 and keys.is_contiguous() and keys.numel() == xy.shape[0]
        check(self._L.raster_contract_keys(self._h, ctypes.c_void_p(xy.data_ptr()), xy.shape[0],
                                           ctypes.c_void_p(keys.data_ptr()), _stream_ptr(stream)),
              "raster_contract_keys")
        return keys

    def contract_tiles(self, key: torch.Tensor, count: torch.Tensor, stream=None):
        """Add count[i] points to tile key[i] (CUDA int64 keys, CUDA int32 or
        uint32-valued counts): the join of partial tile counts."""
        assert key.is_cuda and key.dtype == torch.int64 and key.is_contiguous()
        assert count.is_cuda and count.dtype == torch.int32 and count.is_contiguous()
        assert key.numel() == count.numel()
        check(self._L.raster_contract_tiles(self._h, ctypes.c_void_p(key.data_ptr()),
                                            ctypes.c_void_p(count.data_ptr()), key.numel(), _stream_ptr(stream)),
              "raster_contract_tiles")

    def contract_host(self, xy, stream=None):
        """xy: host (n, 2) float64 (pinned torch tensor or numpy array)."""
        ptr, n = _host_ptr(xy, cols=self.dims)
        check(self._L.raster_contract_host(self._h, ctypes.c_void_p(ptr), n, _stream_ptr(stream)),
              "raster_contract_host")

    def agglomerate(self, copy: bool = True, allow_range_error: bool = False, raw: bool = False) -> Result:
        """copy=False returns views of the library's arrays; raw=True also keeps
        the counts as the library's uint32 bits (an int32 view) so that no
        torch kernel runs."""
        out = _native.Clusters()
        st = self._L.raster_agglomerate(self._h, ctypes.byref(out))
        if st != _native.OK and not (allow_range_error and st == _native.E_RANGE):
            raise RasterError(st, "raster_agglomerate")
        n = out.n_tiles
        key = _view(out.key, n, torch.int64, self.device)
        cnt = _view(out.count, n, torch.int32, self.device)
        cid = _view(out.cid, n, torch.int64, self.device)
        if copy:
            key, cid = key.clone(), cid.clone()
        if not raw:
            cnt = cnt.to(torch.int64) & 0xFFFFFFFF
        return Result(key, cnt, cid, out.n_clusters, out.n_distinct, out.n_significant, out.n_points, st, self.dims)

    def _result(self, out, st, copy: bool, raw: bool) -> Result:
        n = out.n_tiles
        key = _view(out.key, n, torch.int64, self.device)
        cnt = _view(out.count, n, torch.int32, self.device)
        cid = _view(out.cid, n, torch.int64, self.device)
        if copy:
            key, cid = key.clone(), cid.clone()
        if not raw:
            cnt = cnt.to(torch.int64) & 0xFFFFFFFF
        return Result(key, cnt, cid, out.n_clusters, out.n_distinct, out.n_significant, out.n_points, st, self.dims)

    def cluster_host(self, xy, out=None, copy: bool = True, allow_range_error: bool = False, raw: bool = False,
                     stream=None):
        """The whole method on host points in one call: contraction (one copy of
        the points to the device), agglomeration, and the label of every point
        back in host memory.  Returns (Result, labels)."""
        ptr, n = _host_ptr(xy, cols=self.dims)
        if out is None:
            out = torch.empty(n, dtype=torch.int64, pin_memory=torch.cuda.is_available())
        optr, on = _host_ptr(out, cols=None)
        assert on == n
        res = _native.Clusters()
        st = self._L.raster_cluster_host(self._h, ctypes.c_void_p(ptr), n, ctypes.c_void_p(optr), ctypes.byref(res),
                                         _stream_ptr(stream))
        if st != _native.OK and not (allow_range_error and st == _native.E_RANGE):
            raise RasterError(st, "raster_cluster_host")
        return self._result(res, st, copy, raw), out

    def point_labels(self, xy: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        _check_points(xy, "point_labels", self.dims)
        if out is None:
            out = torch.empty(xy.shape[0], dtype=torch.int64, device=xy.device)
        assert out.is_cuda and out.dtype == torch.int64 and out.is_contiguous() and out.numel() == xy.shape[0]
        check(self._L.raster_point_labels(self._h, ctypes.c_void_p(xy.data_ptr()), xy.shape[0],
                                          ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
              "raster_point_labels")
        return out

    def key_labels(self, keys: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Labels of the points whose tile keys contract_keys wrote: the same
        as point_labels of those points."""
        assert keys.is_cuda and keys.dtype == torch.int64 and keys.is_contiguous()
        if out is None:
            out = torch.empty(keys.numel(), dtype=torch.int64, device=keys.device)
        assert out.is_cuda and out.dtype == torch.int64 and out.is_contiguous() and out.numel() == keys.numel()
        check(self._L.raster_key_labels(self._h, ctypes.c_void_p(keys.data_ptr()), keys.numel(),
                                        ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
              "raster_key_labels")
        return out

    def point_labels_host(self, xy, out=None, stream=None):
        ptr, n = _host_ptr(xy, cols=self.dims)
        if out is None:
            out = torch.empty(n, dtype=torch.int64)
        optr, on = _host_ptr(out, cols=None)
        assert on == n
        check(self._L.raster_point_labels_host(self._h, ctypes.c_void_p(ptr), n, ctypes.c_void_p(optr),
                                               _stream_ptr(stream)), "raster_point_labels_host")
        return out

    def point_groups(self, xy: torch.Tensor, n_tiles: int, out=None, stream=None):
        """RASTER' output: (row_start int64[n_tiles+1], point_index int64[m]) --
        the indices of the points of each kept tile, rows in the order of the
        last agglomerate() result (n_tiles = its number of rows).  `out` may
        give (row_start, point_index) buffers of n_tiles+1 and n entries."""
        _check_points(xy, "point_groups", self.dims)
        n = xy.shape[0]
        if out is None:
            out = (torch.empty(n_tiles + 1, dtype=torch.int64, device=xy.device),
                   torch.empty(max(n, 1), dtype=torch.int64, device=xy.device))  # at most n grouped points
        row_start, idx = out
        for t, size in ((row_start, n_tiles + 1), (idx, n)):
            assert t.is_cuda and t.dtype == torch.int64 and t.is_contiguous() and t.numel() >= size
        m = ctypes.c_int64()
        check(self._L.raster_point_groups(self._h, ctypes.c_void_p(xy.data_ptr()), n,
                                          ctypes.c_void_p(row_start.data_ptr()), ctypes.c_void_p(idx.data_ptr()),
                                          idx.numel(), ctypes.byref(m), _stream_ptr(stream)), "raster_point_groups")
        return row_start[:n_tiles + 1], idx[:m.value]

    def table_stats(self) -> dict:
        """Occupancy and probe lengths of the tile table (diagnostics)."""
        t = _native.TableStats()
        check(self._L.raster_table_stats(self._h, ctypes.byref(t)), "raster_table_stats")
        occ = t.occupied
        return {"capacity": t.capacity, "occupied": occ, "load": occ / t.capacity if t.capacity else 0.0,
                "mean_probe": t.probe_sum / occ if occ else 0.0, "max_probe": t.probe_max}

    def export_tiles(self):
        """All tiles with at least one point: (key int64, count int64) CUDA tensors."""
        n = ctypes.c_int64()
        self._L.raster_export_tiles(self._h, None, None, 0, ctypes.byref(n))
        d = n.value
        key = torch.empty(max(d, 1), dtype=torch.int64, device=self.device)
        cnt = torch.empty(max(d, 1), dtype=torch.int32, device=self.device)
        check(self._L.raster_export_tiles(self._h, ctypes.c_void_p(key.data_ptr()), ctypes.c_void_p(cnt.data_ptr()),
                                          max(d, 1), ctypes.byref(n)), "raster_export_tiles")
        return key[:d], cnt[:d].to(torch.int64) & 0xFFFFFFFF

    def reset(self, stream=None):
        check(self._L.raster_reset(self._h, _stream_ptr(stream)), "raster_reset")

    def status(self) -> int:
        return self._L.raster_status(self._h)


def _host_ptr(a, cols=2):
    import numpy as np
    if isinstance(a, np.ndarray):
        if cols is None:
            assert a.dtype == np.int64 and a.flags.c_contiguous and a.ndim == 1
            return a.ctypes.data, a.shape[0]
        assert a.dtype == np.float64 and a.flags.c_contiguous and a.ndim == 2 and a.shape[1] == cols
        return a.ctypes.data, a.shape[0]
    assert not a.is_cuda and a.is_contiguous()
    if cols is None:
        assert a.dtype == torch.int64 and a.dim() == 1
    else:
        assert a.dtype == torch.float64 and a.dim() == 2 and a.shape[1] == cols
    return a.data_ptr(), a.shape[0]
