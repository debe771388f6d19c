"""Python access to the CPU FP64 oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this module; the CUDA library and its
binding never import it.

The oracle is the plain double-buffered restatement of the double-MRT
lattice Boltzmann method with interfacial tracking (Li, Yang & Zhang,
arXiv:1604.03478, section 2, Eqs. 1-6).  See ``lbm_oracle.c`` for the step,
the readings of the paper it takes, and the layout.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
_LIB_CS = os.path.join(_HERE, "liblbm_oracle_cs.so")

# Non-hydrodynamic D3Q19 rates of d'Humieres et al. (2002) and inert D3Q7
# higher-order rates; the hydrodynamic ones come from the case.
DEFAULT_RATES = dict(s_e=1.19, s_eps=1.4, s_q=1.2, s_pi=1.4, s_m=1.98, s_g4=1.0, s_g5=1.0)


def _compile(out, extra):
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC",
                           "-shared"] + extra + ["-o", tmp, _SRC, "-lm"])
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` into ``liblbm_oracle.so`` (FP64) and
    ``liblbm_oracle_cs.so`` (the same source in double _Complex, for
    complex-step tangent-linear derivatives); gcc, OpenMP, -O2."""
    if force:
        for p in (_LIB, _LIB_CS):
            if os.path.exists(p):
                os.remove(p)
    _compile(_LIB, [])
    _compile(_LIB_CS, ["-DORC_COMPLEX"])
    return _LIB


class _Cfg(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("face", C.c_int),
                ("Ra", C.c_double), ("Pr", C.c_double), ("Ste", C.c_double), ("Th", C.c_double),
                ("Tc", C.c_double), ("Tm", C.c_double), ("Ma", C.c_double), ("s0", C.c_double),
                ("s_nu", C.c_double), ("s_e", C.c_double), ("s_eps", C.c_double), ("s_q", C.c_double),
                ("s_pi", C.c_double), ("s_m", C.c_double), ("s_alpha", C.c_double),
                ("s_g4", C.c_double), ("s_g5", C.c_double), ("derive", C.c_int),
                ("solid", C.c_int), ("ks_kl", C.c_double)]


_lib = None
_lib_cs = None


def _declare(L):
    dp = C.POINTER(C.c_double)
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.POINTER(_Cfg), C.c_char_p, C.c_int]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_step.restype = C.c_int
    L.orc_step.argtypes = [C.c_void_p, C.c_long]
    L.orc_get.argtypes = [C.c_void_p, dp, dp, dp, dp]
    L.orc_get_state.argtypes = [C.c_void_p, dp, dp, dp]
    L.orc_set_state.argtypes = [C.c_void_p, dp, dp, dp]
    L.orc_set_hot_wall.argtypes = [C.c_void_p, dp]
    L.orc_nusselt.argtypes = [C.c_void_p, dp, dp]
    L.orc_info.argtypes = [C.c_void_p, dp]
    L.orc_error.restype = C.c_char_p
    L.orc_error.argtypes = [C.c_void_p]
    L.orc_num_threads.restype = C.c_int
    L.orc_set_num_threads.argtypes = [C.c_int]


def lib_cs() -> C.CDLL:
    """The complex-step build (tangent-linear derivatives)."""
    global _lib_cs
    if _lib_cs is None:
        build()
        L = C.CDLL(_LIB_CS)
        _declare(L)
        dp = C.POINTER(C.c_double)
        L.orc_cs_perturb.restype = C.c_int
        L.orc_cs_perturb.argtypes = [C.c_void_p, C.c_double, dp]
        L.orc_cs_get_s.argtypes = [C.c_void_p, dp, dp, dp, dp]
        _lib_cs = L
    return _lib_cs


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        _declare(L)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.orc_neumann_lambda.restype = C.c_double
        L.orc_neumann_lambda.argtypes = [C.c_double]
        L.orc_front_gradient.restype = C.c_double
        L.orc_front_gradient.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double]
        L.orc_ghost_T.restype = C.c_double
        L.orc_ghost_T.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double]
        L.orc_solid_gradient.restype = C.c_double
        L.orc_solid_gradient.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double]
        L.orc_solid_ghost_T.restype = C.c_double
        L.orc_solid_ghost_T.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double]
        L.orc_neumann_lambda2.restype = C.c_double
        L.orc_neumann_lambda2.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_lattice19.argtypes = [ip, ip, ip, dp, ip]
        L.orc_lattice7.argtypes = [ip, ip, ip, dp, ip]
        L.orc_matrices.argtypes = [dp, dp, dp, dp]
        L.orc_feq19.argtypes = [C.c_double, dp, dp]
        L.orc_geq7.argtypes = [C.c_double, dp, dp]
        L.orc_guo19.argtypes = [dp, dp, dp]
        L.orc_collide_f.argtypes = [dp, dp, dp, dp, dp]
        L.orc_collide_g.argtypes = [dp, dp, dp, dp]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


# ------------------------------------------------------------ unit functions

def lattice19():
    ex, ey, ez, opp = (np.zeros(19, np.int32) for _ in range(4))
    w = np.zeros(19)
    lib().orc_lattice19(_ip(ex), _ip(ey), _ip(ez), _p(w), _ip(opp))
    return np.stack([ex, ey, ez], 1), w, opp


def lattice7():
    ex, ey, ez, opp = (np.zeros(7, np.int32) for _ in range(4))
    w = np.zeros(7)
    lib().orc_lattice7(_ip(ex), _ip(ey), _ip(ez), _p(w), _ip(opp))
    return np.stack([ex, ey, ez], 1), w, opp


def matrices():
    M, Mi, N, Ni = np.zeros((19, 19)), np.zeros((19, 19)), np.zeros((7, 7)), np.zeros((7, 7))
    lib().orc_matrices(_p(M), _p(Mi), _p(N), _p(Ni))
    return M, Mi, N, Ni


def feq19(rho, u):
    out = np.zeros(19)
    lib().orc_feq19(float(rho), _p(np.asarray(u, float)), _p(out))
    return out


def geq7(T, u):
    out = np.zeros(7)
    lib().orc_geq7(float(T), _p(np.asarray(u, float)), _p(out))
    return out


def guo19(u, F):
    out = np.zeros(19)
    lib().orc_guo19(_p(np.asarray(u, float)), _p(np.asarray(F, float)), _p(out))
    return out


def collide_f(f, S19, F):
    f = np.ascontiguousarray(f, float)
    out, u = np.zeros(19), np.zeros(3)
    lib().orc_collide_f(_p(f), _p(np.ascontiguousarray(S19, float)), _p(np.asarray(F, float)), _p(out), _p(u))
    return out, u


def collide_g(g, Q7, u):
    out = np.zeros(7)
    lib().orc_collide_g(_p(np.ascontiguousarray(g, float)), _p(np.ascontiguousarray(Q7, float)),
                        _p(np.asarray(u, float)), _p(out))
    return out


def neumann_lambda(Ste):
    return lib().orc_neumann_lambda(float(Ste))


def front_gradient(Tcol, s, Tw, Tm):
    Tcol = np.ascontiguousarray(Tcol, float)
    return lib().orc_front_gradient(_p(Tcol), len(Tcol), float(s), float(Tw), float(Tm))


def ghost_T(Tcol, s, Tw, Tm):
    Tcol = np.ascontiguousarray(Tcol, float)
    return lib().orc_ghost_T(_p(Tcol), len(Tcol), float(s), float(Tw), float(Tm))


def solid_gradient(Tcol, s, Tc, Tm):
    Tcol = np.ascontiguousarray(Tcol, float)
    return lib().orc_solid_gradient(_p(Tcol), len(Tcol), float(s), float(Tc), float(Tm))


def solid_ghost_T(Tcol, s, Tc, Tm):
    Tcol = np.ascontiguousarray(Tcol, float)
    return lib().orc_solid_ghost_T(_p(Tcol), len(Tcol), float(s), float(Tc), float(Tm))


def neumann_lambda2(Ste, theta, kappa):
    """Two-phase Neumann front constant: s = 2 lambda sqrt(alpha_l t) for a
    solid initially at Tc, theta = (Tm - Tc) / (Th - Tm), kappa = k_s / k_l."""
    return lib().orc_neumann_lambda2(float(Ste), float(theta), float(kappa))


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(n):
    """Threads of the oracle's OpenMP loops from now on (timing only)."""
    lib().orc_set_num_threads(int(n))


# ---------------------------------------------------------------- simulator

INFO_KEYS = ("nu", "alpha", "gbeta", "lambda", "t0", "s_nu", "s_alpha", "H", "steps",
             "q_hot", "q_cold", "mass", "n_liquid", "sum_T_liquid", "sum_T_solid", "alpha_s")


class OracleError(RuntimeError):
    pass


class Oracle:
    """One cavity advanced by the FP64 oracle.

    Arguments mirror the library's create call: grid (nx, ny, nz), heated face
    (0: y = 0, 1: z = 0), Ra, Pr, Ste, Th, Tc, Tm, Ma, initial front s0, and
    the relaxation rates.  With ``derive`` the rates s_nu and s_alpha follow
    from Ra, Pr, Ma and H; otherwise pass them explicitly.  ``solid`` = 1
    turns on heat conduction in the solid (conductivity ratio ``ks_kl`` =
    k_s / k_l), the k_s term of Eq. 6.
    """

    def __init__(self, nx, ny, nz, face=0, Ra=0.0, Pr=1.0, Ste=0.1, Th=1.0, Tc=0.0, Tm=0.0,
                 Ma=0.1, s0=1.0, s_nu=1.0, s_alpha=1.0, derive=False, solid=0, ks_kl=1.0, _lib=None,
                 **rates):
        self._L = _lib if _lib is not None else lib()
        r = dict(DEFAULT_RATES)
        r.update(rates)
        cfg = _Cfg(nx, ny, nz, face, Ra, Pr, Ste, Th, Tc, Tm, Ma, s0, s_nu, r["s_e"], r["s_eps"],
                   r["s_q"], r["s_pi"], r["s_m"], s_alpha, r["s_g4"], r["s_g5"], 1 if derive else 0,
                   int(solid), float(ks_kl))
        err = C.create_string_buffer(256)
        h = self._L.orc_create(C.byref(cfg), err, 256)
        if not h:
            raise OracleError(err.value.decode())
        self._h = h
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.face = face
        self.H = ny if face == 0 else nz
        self.cols_shape = (nz, nx) if face == 0 else (ny, nx)
        self.ncols = self.cols_shape[0] * self.cols_shape[1]

    def close(self):
        if self._h:
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        st = self._L.orc_step(self._h, int(n))
        if st != 0:
            raise OracleError("orc_step: %s" % self._L.orc_error(self._h).decode())

    def get(self):
        T = np.zeros(self.N)
        u = np.zeros(3 * self.N)
        s = np.zeros(self.ncols)
        lf = np.zeros(1)
        self._L.orc_get(self._h, _p(T), _p(u), _p(s), _p(lf))
        return T.reshape(self.shape), u.reshape(self.shape + (3,)), s.reshape(self.cols_shape), float(lf[0])

    def get_state(self):
        f = np.zeros((19, self.N))
        g = np.zeros((7, self.N))
        s = np.zeros(self.ncols)
        self._L.orc_get_state(self._h, _p(f), _p(g), _p(s))
        return f, g, s

    def set_state(self, f=None, g=None, s=None):
        f = None if f is None else np.ascontiguousarray(f, float).reshape(19, self.N)
        g = None if g is None else np.ascontiguousarray(g, float).reshape(7, self.N)
        s = None if s is None else np.ascontiguousarray(s, float).reshape(self.ncols)
        self._L.orc_set_state(self._h, _p(f), _p(g), _p(s))

    def set_hot_wall(self, Thw):
        Thw = np.ascontiguousarray(Thw, float).reshape(self.ncols)
        self._L.orc_set_hot_wall(self._h, _p(Thw))

    def nusselt(self):
        """Local Nusselt number on the heated wall per column (cols_shape)
        and its mean over the wall, from the last step's wall flux."""
        nu = np.zeros(self.ncols)
        m = np.zeros(1)
        self._L.orc_nusselt(self._h, _p(nu), _p(m))
        return nu.reshape(self.cols_shape), float(m[0])

    def info(self):
        v = np.zeros(len(INFO_KEYS))
        self._L.orc_info(self._h, _p(v))
        return dict(zip(INFO_KEYS, v.tolist()))


def tangent(nx, ny, nz, steps, dRa=0.0, dThw=None, h=1e-20, wall=None, **kw):
    """Directional derivative by complex step: run the oracle in complex
    arithmetic with Ra -> Ra + i h dRa and the heated-wall field -> Th +
    i h dThw (per column), and return (S, dS, lf, dlf): the final front
    heights, the liquid fraction and their derivatives along the direction.
    ``wall`` (per column) replaces the scalar Th as the real part of the
    heated-wall field before the run.  The phase flags are those of the
    unperturbed run (branches on real parts).
    """
    o = Oracle(nx, ny, nz, _lib=lib_cs(), **kw)
    if wall is not None:
        o.set_hot_wall(wall)
    dT = None if dThw is None else np.ascontiguousarray(np.asarray(dThw, float).reshape(o.ncols) * h)
    st = o._L.orc_cs_perturb(o._h, float(dRa) * h, _p(dT))
    if st != 0:
        raise OracleError("orc_cs_perturb failed")
    o.step(steps)
    re, im = np.zeros(o.ncols), np.zeros(o.ncols)
    lre, lim = np.zeros(1), np.zeros(1)
    o._L.orc_cs_get_s(o._h, _p(re), _p(im), _p(lre), _p(lim))
    o.close()
    return re.reshape(o.cols_shape), (im / h).reshape(o.cols_shape), float(lre[0]), float(lim[0] / h)
