"""Batched form: many independent RASTER instances in one graph launch.

    b = RasterBatch([(xy_0, p_0, tau_0, mu_0), ...])   # xy_i: (n_i, 2) float64 CUDA tensors
    b.run(); b.wait()
    res = b.result(i)                                  # same fields as Raster.agglomerate()

The xy tensors must stay alive and keep their addresses while the batch lives
(the graph holds their pointers); new data is run by writing into them.
"""
from __future__ import annotations

import ctypes

import torch

from . import _native
from ._native import RasterError, check, lib
from . import Result, _view, _stream_ptr


class RasterBatch:
    def __init__(self, instances, load: float = 0.0, block: int = 0, width: int = 0, preagg: int = -1):
        self._L = lib()
        self._xy = []
        arr = (_native.Instance * max(len(instances), 1))()
        for i, (xy, p, tau, mu) in enumerate(instances):
            if not (xy.is_cuda and xy.dtype == torch.float64 and xy.dim() == 2 and xy.shape[1] == 2
                    and xy.is_contiguous()):
                raise ValueError("instance points must be contiguous (n, 2) float64 CUDA tensors")
            self._xy.append(xy)
            arr[i] = _native.Instance(xy.data_ptr() if xy.numel() else 0, xy.shape[0], float(p), int(tau), int(mu))
        cfg = _native.BatchConfig(float(load), int(block), int(width), int(preagg))
        h = ctypes.c_void_p()
        check(self._L.raster_batch_create(arr, len(instances), ctypes.byref(cfg), ctypes.byref(h)),
              "raster_batch_create")
        self._h = h
        self.count = len(instances)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def run(self, stream=None):
        check(self._L.raster_batch_run(self._h, _stream_ptr(stream)), "raster_batch_run")

    def wait(self, allow_range_error: bool = False) -> int:
        st = self._L.raster_batch_wait(self._h)
        if st != _native.OK and not (allow_range_error and st == _native.E_RANGE):
            raise RasterError(st, "raster_batch_wait")
        return st

    def counts(self, i: int) -> _native.Clusters:
        out = _native.Clusters()
        self._L.raster_batch_result(self._h, i, ctypes.byref(out))
        return out

    def result(self, i: int, copy: bool = True) -> Result:
        out = _native.Clusters()
        st = self._L.raster_batch_result(self._h, i, ctypes.byref(out))
        n = out.n_tiles
        key = _view(out.key, n, torch.int64, self.device)
        cnt = _view(out.count, n, torch.int32, self.device)
        cid = _view(out.cid, n, torch.int64, self.device)
        if copy:
            key, cid = key.clone(), cid.clone()
        cnt = cnt.to(torch.int64) & 0xFFFFFFFF
        return Result(key, cnt, cid, out.n_clusters, out.n_distinct, out.n_significant, out.n_points, st)

    @property
    def device_bytes(self) -> int:
        return self._L.raster_batch_device_bytes(self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._L.raster_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
