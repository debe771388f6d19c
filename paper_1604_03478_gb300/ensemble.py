"""Batch of independent cavities advanced by one persistent kernel launch
(``lbm_ensemble_*`` in include/lbm_melt.h); argument marshalling only."""
from __future__ import annotations

import ctypes as C

from . import _abi
from .cavity import Cavity, LbmError, make_args


class Ensemble:
    """cases: list of dicts with the Cavity arguments (nx, ny, nz, face,
    precision, Ra, Pr, Ste, Th, Tc, Tm, Ma, s0, s_nu, s_alpha, derive, rates)."""

    def __init__(self, cases, stream=None):
        L = _abi.load()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        arr = (_abi.lbm_melt_case * len(cases))()
        self._dims = []
        for k, c in enumerate(cases):
            c = dict(c)
            nx, ny, nz = c.pop("nx"), c.pop("ny"), c.pop("nz")
            face = c.pop("face", 0)
            grid, rates = make_args(nx, ny, nz, face, c.pop("precision", 0), c.pop("Ma", 0.1), c.pop("s0", 1.0),
                                    c.pop("s_nu", 1.0), c.pop("s_alpha", 1.0), c.pop("derive", False),
                                    **c.pop("rates", {}))
            arr[k].grid = grid
            arr[k].rates = rates
            arr[k].Ra = c.pop("Ra", 0.0)
            arr[k].Pr = c.pop("Pr", 1.0)
            arr[k].Ste = c.pop("Ste", 0.1)
            arr[k].Th = c.pop("Th", 1.0)
            arr[k].Tc = c.pop("Tc", 0.0)
            arr[k].Tm = c.pop("Tm", 0.0)
            if c:
                raise TypeError("unknown case keys: %s" % sorted(c))
            self._dims.append((nx, ny, nz, face))
        h = C.c_void_p()
        st = L.lbm_ensemble_create(len(cases), arr, C.c_void_p(stream), C.byref(h))
        if st != 0:
            raise LbmError(st, "lbm_ensemble_create failed")
        self._h = h
        self.n = len(cases)

    def _check(self, st):
        if st != 0:
            raise LbmError(st, _abi.load().lbm_ensemble_last_error(self._h).decode())

    def step(self, n=1):
        self._check(_abi.load().lbm_ensemble_step(self._h, int(n)))

    def sync(self):
        self._check(_abi.load().lbm_ensemble_sync(self._h))

    def set_launch(self, block=128, nodes_per_thread=2, graph_steps=8):
        self._check(_abi.load().lbm_ensemble_set_launch(self._h, int(block), int(nodes_per_thread),
                                                        int(graph_steps)))

    def set_barrier_timeout(self, spins):
        self._check(_abi.load().lbm_ensemble_set_barrier_timeout(self._h, int(spins)))

    def inject_barrier_fault(self, block=0):
        self._check(_abi.load().lbm_ensemble_inject_barrier_fault(self._h, int(block)))

    def info(self):
        n, g, b, k = C.c_longlong(), C.c_int(), C.c_int(), C.c_int()
        self._check(_abi.load().lbm_ensemble_info(self._h, C.byref(n), C.byref(g), C.byref(b), C.byref(k)))
        return dict(nodes=n.value, grid=g.value, block=b.value, nodes_per_thread=k.value)

    def phase_times(self, reset=False):
        """Mean microseconds per step of the stream-collide, front and flip
        phases (each with its closing grid barrier) since creation or the
        last reset, and the number of steps timed."""
        us = (C.c_double * 3)()
        n = C.c_longlong()
        self._check(_abi.load().lbm_ensemble_phase_times(self._h, 1 if reset else 0, us, C.byref(n)))
        return dict(stream_collide_us=us[0], front_us=us[1], flip_us=us[2], steps=n.value)

    def member(self, i):
        h = _abi.load().lbm_ensemble_member(self._h, int(i))
        if not h:
            raise IndexError(i)
        nx, ny, nz, face = self._dims[i]
        return Cavity._member(h, nx, ny, nz, face)

    def close(self):
        if getattr(self, "_h", None):
            _abi.load().lbm_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
