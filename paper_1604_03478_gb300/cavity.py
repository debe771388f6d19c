"""Convenience wrapper of one cavity handle of the C ABI.

Every method is argument marshalling around one ``lbm_melt_*`` call.  Host
results come back as numpy arrays; ``get_device`` returns torch CUDA tensors
filled by the library through device pointers.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi

DEFAULT_RATES = dict(s_e=1.19, s_eps=1.4, s_q=1.2, s_pi=1.4, s_m=1.98, s_g4=1.0, s_g5=1.0)


def default_rates():
    return dict(DEFAULT_RATES)


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_abi.STATUS_NAMES.get(status, status), msg))
        self.status = status


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return C.c_void_p(a.ctypes.data)
    return C.c_void_p(a.data_ptr())  # torch tensor


def make_args(nx, ny, nz, face=0, precision=0, Ma=0.1, s0=1.0, s_nu=1.0, s_alpha=1.0, derive=False, **rates):
    r = dict(DEFAULT_RATES)
    r.update(rates)
    grid = _abi.lbm_melt_grid(nx, ny, nz, face, precision, Ma, s0)
    rr = _abi.lbm_melt_rates(s_nu, r["s_e"], r["s_eps"], r["s_q"], r["s_pi"], r["s_m"], s_alpha,
                             r["s_g4"], r["s_g5"], 1 if derive else 0)
    return grid, rr


class Cavity:
    """One cavity on the current CUDA device.

    Arguments follow ``lbm_melt_create``: the grid (nx, ny, nz), heated face
    (0: y = 0, 1: z = 0), storage precision (0 fp32, 1 fp16), Ma, initial
    front s0, Ra, Pr, Ste, Th, Tc, Tm and the rates (``derive`` takes s_nu,
    s_alpha from Ra, Pr, Ma and H).  ``stream`` is a cudaStream_t as int
    (default: torch's current stream).  ``solid=1`` turns on heat conduction
    in the solid with conductivity ratio ``ks_kl`` = k_s / k_l
    (lbm_melt_set_solid_conduction).
    """

    def __init__(self, nx, ny, nz, face=0, precision=0, Ra=0.0, Pr=1.0, Ste=0.1, Th=1.0, Tc=0.0, Tm=0.0,
                 Ma=0.1, s0=1.0, s_nu=1.0, s_alpha=1.0, derive=False, stream=None, solid=0, ks_kl=1.0,
                 **rates):
        L = _abi.load()
        self.grid, self.rates = make_args(nx, ny, nz, face, precision, Ma, s0, s_nu, s_alpha, derive, **rates)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = C.c_void_p()
        st = L.lbm_melt_create(C.byref(self.grid), Ra, Pr, Ste, Th, Tc, Tm, C.byref(self.rates),
                               C.c_void_p(stream), C.byref(h))
        if st != 0:
            msg = L.lbm_melt_derive_error(C.byref(self.grid), Ra, Pr, Ste, Th, Tc, Tm, C.byref(self.rates))
            raise LbmError(st, (msg or b"").decode() or "lbm_melt_create failed")
        self._h = h
        self._owned = True
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.face = face
        self.H = ny if face == 0 else nz
        self.cols_shape = (nz, nx) if face == 0 else (ny, nx)
        self.ncols = self.cols_shape[0] * self.cols_shape[1]
        if solid:
            self.set_solid_conduction(ks_kl)

    @classmethod
    def _member(cls, handle, nx, ny, nz, face):
        """View of a cavity owned by an ensemble (never destroyed here)."""
        obj = cls.__new__(cls)
        obj._h = C.c_void_p(handle)
        obj._owned = False
        obj.shape = (nz, ny, nx)
        obj.N = nx * ny * nz
        obj.face = face
        obj.H = ny if face == 0 else nz
        obj.cols_shape = (nz, nx) if face == 0 else (ny, nx)
        obj.ncols = obj.cols_shape[0] * obj.cols_shape[1]
        return obj

    # -- lifetime
    def close(self):
        if not getattr(self, "_owned", True):
            self._h = None
            return
        if getattr(self, "_h", None):
            _abi.load().lbm_melt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise LbmError(st, _abi.load().lbm_melt_last_error(self._h).decode())

    # -- calls
    def step(self, n=1):
        self._check(_abi.load().lbm_melt_step(self._h, int(n)))

    def sync(self):
        self._check(_abi.load().lbm_melt_sync(self._h))

    def get(self, T=True, u=True, S=True, lf=True):
        Ta = np.zeros(self.shape, np.float32) if T else None
        ua = np.zeros(self.shape + (3,), np.float32) if u else None
        Sa = np.zeros(self.cols_shape, np.float64) if S else None
        la = np.zeros(1, np.float64) if lf else None
        self._check(_abi.load().lbm_melt_get(self._h, _ptr(Ta), _ptr(ua), _ptr(Sa), _ptr(la), 0))
        return Ta, ua, Sa, (float(la[0]) if lf else None)

    TOTAL_KEYS = ("liquid_fraction", "sum_T_minus_Tm", "sum_rho_minus_1", "n_liquid", "max_u", "sum_S",
                  "nusselt_mean")

    def totals(self):
        """FP64 totals of the current state (see lbm_melt_totals)."""
        out = np.zeros(len(self.TOTAL_KEYS), np.float64)
        self._check(_abi.load().lbm_melt_totals(self._h, _ptr(out), 0))
        return dict(zip(self.TOTAL_KEYS, out.tolist()))

    def nusselt(self):
        """Heat-surface Nusselt number per column (cols_shape) and its mean
        over the heated wall (see lbm_melt_get_nusselt)."""
        nu = np.zeros(self.cols_shape, np.float64)
        m = np.zeros(1, np.float64)
        self._check(_abi.load().lbm_melt_get_nusselt(self._h, _ptr(nu), _ptr(m), 0))
        return nu, float(m[0])

    def set_report(self, every, capacity=4096):
        self._check(_abi.load().lbm_melt_set_report(self._h, int(every), int(capacity)))

    def get_report(self, max_rows=1 << 20):
        """Recorded rows: columns steps, then the seven totals."""
        n = C.c_longlong()
        self._check(_abi.load().lbm_melt_get_report(self._h, None, 0, C.byref(n)))
        rows = np.zeros((min(n.value, max_rows), 8), np.float64)
        self._check(_abi.load().lbm_melt_get_report(self._h, _ptr(rows), rows.shape[0], C.byref(n)))
        return rows

    def get_device(self, T=None, u=None, S=None, lf=None):
        """Fill caller-owned torch CUDA tensors (any may be None)."""
        self._check(_abi.load().lbm_melt_get(self._h, _ptr(T), _ptr(u), _ptr(S), _ptr(lf), 1))

    def get_state(self):
        f = np.zeros((19, self.N), np.float32)
        g = np.zeros((7, self.N), np.float32)
        s = np.zeros(self.ncols, np.float64)
        self._check(_abi.load().lbm_melt_get_state(self._h, _ptr(f), _ptr(g), _ptr(s), 0))
        return f, g, s

    def set_state(self, f=None, g=None, s=None):
        f = None if f is None else np.ascontiguousarray(f, np.float32).reshape(19, self.N)
        g = None if g is None else np.ascontiguousarray(g, np.float32).reshape(7, self.N)
        s = None if s is None else np.ascontiguousarray(s, np.float64).reshape(self.ncols)
        self._check(_abi.load().lbm_melt_set_state(self._h, _ptr(f), _ptr(g), _ptr(s), 0))

    def set_hot_wall(self, Thw, ptr_kind=None):
        if ptr_kind is None:
            ptr_kind = 0 if isinstance(Thw, np.ndarray) else 1
        if ptr_kind == 0:
            Thw = np.ascontiguousarray(Thw, np.float32).reshape(self.ncols)
        self._check(_abi.load().lbm_melt_set_hot_wall(self._h, _ptr(Thw), ptr_kind))

    def info(self):
        i = _abi.lbm_melt_info()
        self._check(_abi.load().lbm_melt_get_info(self._h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in i._fields_}

    PARAM_KEYS = ("Ra", "s_nu", "s_alpha", "coef", "gbeta")

    def tape_forward(self, steps, ckpt_every=0):
        """Advance `steps` steps recording checkpoints for tape_backward."""
        self._check(_abi.load().lbm_melt_tape_forward(self._h, int(steps), int(ckpt_every)))

    def tape_backward(self, seed):
        """dL/d(heated-wall field) per column and the parameter sensitivities
        for dL/dS = seed of the final front."""
        seed = np.ascontiguousarray(seed, np.float64).reshape(self.ncols)
        dth = np.zeros(self.ncols, np.float64)
        dpar = np.zeros(5, np.float64)
        self._check(_abi.load().lbm_melt_tape_backward(self._h, _ptr(seed), _ptr(dth), _ptr(dpar), 0))
        return dth.reshape(self.cols_shape), dict(zip(self.PARAM_KEYS, dpar.tolist()))

    def tape_clear(self):
        self._check(_abi.load().lbm_melt_tape_clear(self._h))

    def set_launch(self, bx=0, by=0):
        self._check(_abi.load().lbm_melt_set_launch(self._h, int(bx), int(by)))

    def set_timing(self, on=True):
        self._check(_abi.load().lbm_melt_set_timing(self._h, 1 if on else 0))

    def set_node_pairs(self, mode):
        """Nodes per thread of the stream-collide: -1 choose, 0 one, 1 two
        (lbm_melt_set_node_pairs)."""
        self._check(_abi.load().lbm_melt_set_node_pairs(self._h, int(mode)))

    def set_solid_conduction(self, ks_kl):
        """Heat conduction in the solid with k_s / k_l = ks_kl (0: off);
        before the first step, re-initialises the state."""
        self._check(_abi.load().lbm_melt_set_solid_conduction(self._h, float(ks_kl)))

    def set_graph_steps(self, steps):
        """Steps per CUDA-graph replay in step() (0: step by step)."""
        self._check(_abi.load().lbm_melt_set_graph_steps(self._h, int(steps)))

    def kernel_time(self, reset=True):
        ms = C.c_double()
        n = C.c_longlong()
        self._check(_abi.load().lbm_melt_kernel_time(self._h, C.byref(ms), C.byref(n), 1 if reset else 0))
        return ms.value, n.value
