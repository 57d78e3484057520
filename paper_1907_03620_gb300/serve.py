"""Served form: client side of the continuous-batching engine (libraster.so).

    srv = RasterServer(max_active=4096, reserve_bytes=4 << 30)
    srv.submit(rid, precision, tau, mu, n_total, n_chunks)
    srv.push(rid, chunk_xy)            # CUDA (n, 2) float64; kept alive until done
    rid, res, latency_ms = srv.poll()  # a completed request (Result), or None
    srv.release(rid)

The engine's worker thread does all scheduling and GPU work; this module only
marshals arguments and keeps chunk tensors alive until their request is done.
"""
from __future__ import annotations

import ctypes

import torch

from . import Result, _view
from . import _native
from ._native import check, lib


class RasterServer:
    def __init__(self, max_active: int = 4096, reserve_bytes: int = 1 << 30, table_slots: int = 0,
                 result_rows: int = 0):
        """Requests are admitted while free device memory, less reserve_bytes,
        covers their tables and rows; table_slots and result_rows optionally
        bound what the engine holds at once (0: no bound beyond the device)."""
        self._L = lib()
        h = ctypes.c_void_p()
        cfg = _native.ServerConfig(int(table_slots), int(result_rows), int(max_active), int(reserve_bytes))
        check(self._L.raster_server_create(ctypes.byref(cfg), ctypes.byref(h)), "raster_server_create")
        self._h = h
        self._alive: dict[int, list] = {}
        self.device = torch.device("cuda", torch.cuda.current_device())

    def submit(self, rid: int, precision: float, tau: int, mu: int, n_total: int, n_chunks: int):
        check(self._L.raster_server_submit(self._h, int(rid), float(precision), int(tau), int(mu), int(n_total),
                                           int(n_chunks)), "raster_server_submit")
        self._alive[int(rid)] = []

    def push(self, rid: int, xy: torch.Tensor):
        assert xy.is_cuda and xy.dtype == torch.float64 and xy.dim() == 2 and xy.is_contiguous()
        self._alive[int(rid)].append(xy)
        check(self._L.raster_server_push(self._h, int(rid), ctypes.c_void_p(xy.data_ptr() if xy.numel() else 0),
                                         xy.shape[0]), "raster_server_push")

    def poll(self, wait_ms: int = 0, copy: bool = True, rows: bool = True):
        """A completed request as (id, Result, latency_ms), or None.  rows=False
        skips building the result tensors (no torch work): the Result then
        holds the counts and status only, with empty tensors."""
        rid = ctypes.c_int64()
        out = _native.Clusters()
        lat = ctypes.c_double()
        st = self._L.raster_server_poll(self._h, int(wait_ms), ctypes.byref(rid), ctypes.byref(out),
                                        ctypes.byref(lat))
        if st == _native.E_STATE:
            return None
        if st not in (_native.OK, _native.E_RANGE, _native.E_TABLE_FULL, _native.E_INTERNAL, _native.E_OOM):
            raise _native.RasterError(st, "raster_server_poll")
        if not rows:
            none = torch.empty(0, dtype=torch.int64)
            return rid.value, Result(none, none, none, out.n_clusters, out.n_distinct, out.n_significant,
                                     out.n_points, st), lat.value
        n = out.n_tiles
        key = _view(out.key, n, torch.int64, self.device)
        cnt = _view(out.count, n, torch.int32, self.device)
        cid = _view(out.cid, n, torch.int64, self.device)
        if copy:
            key, cid = key.clone(), cid.clone()
        cnt = cnt.to(torch.int64) & 0xFFFFFFFF
        return rid.value, Result(key, cnt, cid, out.n_clusters, out.n_distinct, out.n_significant, out.n_points,
                                 st), lat.value

    def release(self, rid: int):
        check(self._L.raster_server_release(self._h, int(rid)), "raster_server_release")
        self._alive.pop(int(rid), None)

    def stats(self) -> dict:
        s = _native.ServerStats()
        st = self._L.raster_server_stats(self._h, ctypes.byref(s))
        d = {n: getattr(s, n) for n, _ in _native.ServerStats._fields_}
        d["status"] = st
        return d

    def close(self):
        if getattr(self, "_h", None):
            self._L.raster_server_destroy(self._h)
            self._h = None
            self._alive.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
