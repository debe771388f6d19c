"""GPU parity at the full sizes of the benchmark workloads, in the launch
configuration that bench.py times (default block shapes, the stream-collide
grid cut at the height bound): the 256^3 side-heated cavity at Ra 1e6 with
the front at 0.4 H (with the solid held at Tm, and with a subcooled,
conducting solid) and the 128^3 convection-melting cavity at Ra 1e5.

A few steps from the initial state (both AA phases) are compared field by
field with the FP64 oracle run at the same size; a longer 256^3 run is held
to a property that holds at any size: the cavity, its walls and gravity are
mirror-symmetric in x, so T, u_y, u_z and S are even in x and u_x is odd
(FP32 rounding aside: mirrored nodes sum their directions in another order)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_T, TOL_LF = 1e-4, 1e-3
FULL = {
    "256^3 Ra 1e6 front at 0.4 H": (256, dict(face=0, Ra=1e6, Pr=0.02, Ste=0.05, Ma=0.1, s0=0.4 * 256, derive=True)),
    "128^3 Ra 1e5 from s0 = 1": (128, dict(face=0, Ra=1e5, Pr=0.02, Ste=0.1, Ma=0.1, s0=1.0, derive=True)),
    # the subcooled workload of bench.py's solid leg (heat conduction in the solid)
    "256^3 Ra 1e6 front at 0.4 H, solid at Tc = -0.25": (
        256, dict(face=0, Ra=1e6, Pr=0.02, Ste=0.05, Ma=0.1, s0=0.4 * 256, derive=True, Tc=-0.25, solid=1,
                  ks_kl=1.0)),
}


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1604_03478_gb300 import build, Cavity
    build.build()
    return Cavity


@pytest.mark.parametrize("name", sorted(FULL))
def test_full_size_against_oracle(lib, orc, name):
    n, kw = FULL[name]
    gpu = lib(n, n, n, **kw)
    gpu.step(5)
    Tg, ug, Sg, lfg = gpu.get()
    gpu.close()
    o = orc.Oracle(n, n, n, **kw)
    o.step(5)
    To, uo, So, lfo = o.get()
    del o
    assert np.abs(Tg - To).max() <= TOL_T
    assert np.abs(ug - uo).max() <= TOL_T
    assert np.abs(Sg - So).max() <= 1e-6
    assert abs(lfg - lfo) <= 1e-6


def test_full_size_mirror_symmetry(lib):
    n, kw = FULL["256^3 Ra 1e6 front at 0.4 H"]
    gpu = lib(n, n, n, **kw)
    gpu.step(300)
    T, u, S, lf = gpu.get()
    gpu.close()
    Tm = T[:, :, ::-1]
    um = u[:, :, ::-1, :]
    assert np.abs(T - Tm).max() <= 1e-5
    assert np.abs(u[..., 0] + um[..., 0]).max() <= 1e-6
    assert np.abs(u[..., 1:] - um[..., 1:]).max() <= 1e-6
    assert np.abs(S - S[:, ::-1]).max() <= 1e-6
    assert np.abs(u).max() > 1e-4  # the flow has started


def test_full_ensemble_members_match_single_cavities():
    """The 48-cavity workload of bench.py (71.2 M nodes, sizes 48..160,
    seeded Ra, Ste and heated face), as autotuned there: every member after
    10 steps against the same cavity run on its own (FP32 rounding)."""
    import torch
    assert torch.cuda.is_available()
    from paper_1604_03478_gb300 import Cavity, Ensemble, inputs
    draws = inputs.ensemble(48, 2016)
    cases = [dict(nx=d["n"], ny=d["n"], nz=d["n"], face=d["face"], Ra=d["Ra"], Pr=0.02, Ste=d["Ste"], Ma=0.1,
                  s0=0.4 * d["n"], derive=True) for d in draws]
    ens = Ensemble(cases)
    ens.set_launch(128, 4, 8)
    ens.step(10)
    ens.sync()
    for k, c in enumerate(cases):
        single = Cavity(c["nx"], c["ny"], c["nz"], **{kk: v for kk, v in c.items() if kk not in ("nx", "ny", "nz")})
        single.step(10)
        a = ens.member(k).get()
        b = single.get()
        single.close()
        assert np.abs(a[0] - b[0]).max() <= 1e-5, k
        assert np.abs(a[1] - b[1]).max() <= 1e-5, k
        assert np.abs(a[2] - b[2]).max() <= 1e-6, k
    ens.close()


def test_adjoint_96cube_against_tangent_oracle(lib, orc):
    """The adjoint workload's cavity (96^3, Ra 1e5, Pr 0.02, Ste 0.1, front
    from s0 = 1), over 40 steps with sqrt(N) checkpoints: the gradient of the
    final liquid fraction along Ra and along a seeded wall-field direction
    against the complex-step tangent-linear oracle, 1e-3 relative."""
    from paper_1604_03478_gb300 import inputs
    n, steps = 96, 40
    kw = dict(face=0, Ra=1e5, Pr=0.02, Ste=0.1, Ma=0.1, s0=1.0, derive=True)
    cav = lib(n, n, n, **kw)
    cav.set_hot_wall(np.full(cav.ncols, 1.0, np.float32))
    cav.tape_forward(steps)
    dth, par = cav.tape_backward(np.full(cav.ncols, 1.0 / (cav.H * cav.ncols)))
    cav.close()
    _, _, _, dlf_ra = orc.tangent(n, n, n, steps, dRa=1.0, **kw)
    assert par["Ra"] == pytest.approx(dlf_ra, rel=1e-3)
    v = inputs.gaussian_field(n * n, 1.0, 7)
    _, _, _, dlf_v = orc.tangent(n, n, n, steps, dThw=v, **kw)
    assert float(dth.ravel() @ v) == pytest.approx(dlf_v, rel=1e-3)


def _golden_adjoint():
    import os
    from conftest import GOLDEN
    g = {}
    with open(os.path.join(GOLDEN, "adjoint_96cube_4000steps.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()
                g[k] = float(v)
    return g


def test_adjoint_96cube_4000_steps_against_golden(lib):
    """The adjoint workload as the benchmark runs it: 96^3, Ra 1e5, Pr 0.02,
    Ste 0.1, front from s0 = 1, 4000 steps with sqrt(N) checkpoints, heated
    wall 1 + N(0, 0.01^2) per column (seed 5).  The gradient of the final
    liquid fraction along Ra and along two seeded wall directions, and of
    the L2 mismatch to the final front of a run with wall seed 11, against
    the FP64 oracle's complex-step tangent-linear values (stored by
    oracle/make_golden_adjoint.py; central differences agree with them to
    1e-4), 1e-3 relative."""
    from paper_1604_03478_gb300 import inputs
    g = _golden_adjoint()
    n, steps = 96, 4000
    kw = dict(face=0, Ra=1e5, Pr=0.02, Ste=0.1, Ma=0.1, s0=1.0, derive=True)
    wall = (1.0 + inputs.gaussian_field(n * n, 0.01, 5)).astype(np.float32)
    target = lib(n, n, n, **kw)
    target.set_hot_wall((1.0 + inputs.gaussian_field(n * n, 0.01, 11)).astype(np.float32))
    target.step(steps)
    S_target = target.get(T=False, u=False)[2].ravel()
    target.close()
    cav = lib(n, n, n, **kw)
    cav.set_hot_wall(wall)
    cav.tape_forward(steps)
    _, _, S, lf = cav.get(T=False, u=False)
    assert lf == pytest.approx(g["liquid_fraction"], rel=1e-4)
    dth, par = cav.tape_backward(np.full(cav.ncols, 1.0 / (cav.H * cav.ncols)))
    v1 = inputs.gaussian_field(n * n, 1.0, 7)
    v2 = inputs.gaussian_field(n * n, 1.0, 8)
    assert par["Ra"] == pytest.approx(g["dlf_dRa"], rel=1e-3)
    assert float(dth.ravel() @ v1) == pytest.approx(g["dlf_dv1"], rel=1e-3)
    assert float(dth.ravel() @ v2) == pytest.approx(g["dlf_dv2"], rel=1e-3)
    r = S.ravel() - S_target
    assert float(r @ r) == pytest.approx(g["mismatch_L2"], rel=1e-3)
    dth2, par2 = cav.tape_backward(2.0 * r)
    assert float(dth2.ravel() @ v1) == pytest.approx(g["dL2_dv1"], rel=1e-3)
    assert par2["Ra"] == pytest.approx(g["dL2_dRa"], rel=1e-3)
    cav.close()
