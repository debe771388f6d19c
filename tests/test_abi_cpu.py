"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/lbm_melt.h declares, and validates arguments and
derives the lattice parameters (section 1, Eq. 7) before touching CUDA."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def abi():
    from paper_1604_03478_gb300 import build, _abi
    build.build()
    return _abi


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(lbm_\w+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_function(abi):
    L = C.CDLL(abi.library_path())
    names = _declared()
    assert "lbm_melt_create" in names and "lbm_melt_step" in names and "lbm_melt_get" in names
    for n in names:
        assert hasattr(L, n), n
    assert abi.load().lbm_melt_version().startswith(b"lbm_melt")


def _derive(abi, grid_kw=None, Ra=0.0, Pr=1.0, Ste=0.1, Th=1.0, Tc=0.0, Tm=0.0, **rk):
    from paper_1604_03478_gb300.cavity import make_args
    g = dict(nx=8, ny=16, nz=8, face=0, precision=0, Ma=0.1, s0=1.0)
    g.update(grid_kw or {})
    r = dict(s_nu=1.25, s_alpha=2 / 3, derive=False)
    r.update(rk)
    grid, rates = make_args(g["nx"], g["ny"], g["nz"], g["face"], g["precision"], g["Ma"], g["s0"], **r)
    info = abi.lbm_melt_info()
    st = abi.load().lbm_melt_derive(C.byref(grid), Ra, Pr, Ste, Th, Tc, Tm, C.byref(rates), C.byref(info))
    msg = abi.load().lbm_melt_derive_error(C.byref(grid), Ra, Pr, Ste, Th, Tc, Tm, C.byref(rates))
    return st, info, msg.decode()


@pytest.mark.parametrize("case", [
    dict(grid_kw=dict(ny=3)), dict(grid_kw=dict(nx=0)), dict(grid_kw=dict(face=2)),
    dict(grid_kw=dict(precision=3)), dict(Th=0.0), dict(Tc=0.5), dict(Ste=-0.1), dict(Ra=-1.0),
    dict(Ra=0.0, derive=True), dict(Ra=1e5, Pr=0.02, derive=True, grid_kw=dict(Ma=0.5)),
    dict(s_nu=1.9999), dict(s_alpha=2.5), dict(grid_kw=dict(s0=20.0)), dict(grid_kw=dict(s0=0.2)),
    dict(s_e=2.5),
])
def test_create_rejects_bad_arguments(abi, case):
    st, info, msg = _derive(abi, **case)
    assert st == abi.LBM_EINVAL and msg


def test_create_rejects_before_touching_cuda(abi):
    """lbm_melt_create validates first: a bad argument returns EINVAL on a
    machine without a GPU."""
    from paper_1604_03478_gb300.cavity import make_args
    grid, rates = make_args(8, 3, 8)
    h = C.c_void_p()
    st = abi.load().lbm_melt_create(C.byref(grid), 0.0, 1.0, 0.1, 1.0, 0.0, 0.0, C.byref(rates), None, C.byref(h))
    assert st == abi.LBM_EINVAL and not h.value


@pytest.mark.parametrize("Ra,Pr,Ma,H", [(1e5, 0.02, 0.1, 128), (1e6, 0.02, 0.1, 256), (25000, 0.02, 0.1, 64),
                                        (1e4, 0.7, 0.2, 32)])
def test_derived_parameters_match_oracle(abi, orc, Ra, Pr, Ma, H):
    st, info, msg = _derive(abi, grid_kw=dict(nx=4, ny=H, nz=4, Ma=Ma), Ra=Ra, Pr=Pr, Ste=0.1, derive=True)
    assert st == abi.LBM_OK, msg
    o = orc.Oracle(4, H, 4, Ra=Ra, Pr=Pr, Ma=Ma, Ste=0.1, derive=True).info()
    for k in ("nu", "alpha", "gbeta", "s_nu", "s_alpha", "t0"):
        assert getattr(info, k) == pytest.approx(o[k], rel=1e-13), k
    assert info.lambda_ == pytest.approx(o["lambda"], rel=1e-13)
    # Eq. 7: Fo = t Ma / (H sqrt(3 Ra Pr)) = alpha t / H^2
    assert info.alpha / H ** 2 == pytest.approx(Ma / (H * np.sqrt(3 * Ra * Pr)), rel=1e-13)


def test_workload_lattice_parameters(abi):
    """Lattice viscosities of the workloads (128^3, Ra 1e5, Pr 0.02, Ma 0.1:
    nu = 3.30e-3; 256^3, Ra 1e6: nu = 2.09e-3)."""
    st, i128, _ = _derive(abi, grid_kw=dict(nx=128, ny=128, nz=128), Ra=1e5, Pr=0.02, derive=True)
    st2, i256, _ = _derive(abi, grid_kw=dict(nx=256, ny=256, nz=256), Ra=1e6, Pr=0.02, derive=True)
    assert st == st2 == abi.LBM_OK
    assert i128.nu == pytest.approx(3.30e-3, rel=3e-3) and i128.tau_nu == pytest.approx(0.5099, abs=1e-4)
    assert i256.nu == pytest.approx(2.09e-3, rel=3e-3) and i256.tau_nu == pytest.approx(0.5063, abs=1e-4)


NULL_HANDLE_CALLS = [
    ("lbm_melt_step", (1,)), ("lbm_melt_sync", ()), ("lbm_melt_totals", (None, 0)),
    ("lbm_melt_set_report", (0, 0)), ("lbm_melt_get_report", (None, 0, None)),
    ("lbm_melt_get", (None, None, None, None, 0)), ("lbm_melt_get_async", (None, None, 0)),
    ("lbm_melt_get_noalloc", (None, None, None, None, 0)), ("lbm_melt_get_state", (None, None, None, 0)),
    ("lbm_melt_set_state", (None, None, None, 0)), ("lbm_melt_set_hot_wall", (None, 0)),
    ("lbm_melt_get_nusselt", (None, None, 0)), ("lbm_melt_get_info", (None,)), ("lbm_melt_set_launch", (128, 1)),
    ("lbm_melt_set_graph_steps", (16,)), ("lbm_melt_set_node_pairs", (0,)),
    ("lbm_melt_set_solid_conduction", (1.0,)), ("lbm_melt_set_timing", (1,)),
    ("lbm_melt_kernel_time", (None, None, 0)), ("lbm_melt_tape_forward", (10, 0)), ("lbm_melt_tape_clear", ()),
    ("lbm_melt_tape_backward", (None, None, None, 0)),
    ("lbm_ensemble_step", (1,)), ("lbm_ensemble_sync", ()), ("lbm_ensemble_set_launch", (128, 2, 8)),
    ("lbm_ensemble_set_barrier_timeout", (1000,)), ("lbm_ensemble_inject_barrier_fault", (0,)),
    ("lbm_ensemble_phase_times", (0, None, None)), ("lbm_ensemble_info", (None, None, None, None)),
]


@pytest.mark.parametrize("name,args", NULL_HANDLE_CALLS, ids=[c[0] for c in NULL_HANDLE_CALLS])
def test_null_handle_is_rejected(abi, name, args):
    """Every entry point that takes a handle answers LBM_EINVAL for a NULL one
    and touches nothing else (no GPU needed)."""
    fn = getattr(abi.load(), name)
    assert fn(None, *args) == abi.LBM_EINVAL
