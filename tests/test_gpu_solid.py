"""GPU parity of heat conduction in the solid (the k_s dT_s/da term of Eq. 6
with a subcooled solid, Tc < Tm; lbm_melt_set_solid_conduction) against the
FP64 oracle's conduction build on the same seeded inputs, and against what
the mathematics fixes (a held front's linear profiles, zero subcooling
reducing to the held-solid method).  Tolerances as for the plain method:
max |dT| <= 1e-4 and |d liquid fraction| <= 1e-3 over a run; every
distribution within 2e-6 after a few steps from a given state."""
import ctypes as C

import numpy as np
import pytest

from paper_1604_03478_gb300 import inputs

pytestmark = pytest.mark.gpu

W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
W7 = np.array([1 / 4] + [1 / 8] * 6)
TOL_T, TOL_LF = 1e-4, 1e-3


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1604_03478_gb300 import build, Cavity
    build.build()
    return Cavity


def _pair(lib, orc, shape, pairs=-1, **kw):
    gpu = lib(*shape, **kw)
    gpu.set_node_pairs(pairs)  # -1: the default choice (one node per thread at these sizes); 1: two
    return gpu, orc.Oracle(*shape, **kw)


def _compare(gpu, o, tol_T=TOL_T, tol_lf=TOL_LF, tol_u=1e-4):
    Tg, ug, Sg, lfg = gpu.get()
    To, uo, So, lfo = o.get()
    dT = np.abs(Tg - To).max()
    du = np.abs(ug - uo).max()
    dS = np.abs(Sg - So).max()
    assert dT <= tol_T, ("T", dT)
    assert abs(lfg - lfo) <= tol_lf, ("lf", lfg, lfo)
    assert du <= tol_u, ("u", du)
    assert dS <= tol_lf, ("S", dS)
    return dT, du, dS, abs(lfg - lfo)


@pytest.mark.parametrize("face,shape", [(0, (33, 40, 5)), (1, (5, 33, 40))])
@pytest.mark.parametrize("kappa", [0.5, 2.0])
def test_subcooled_conduction_melting(lib, orc, face, shape, kappa):
    """Ra = 0, a solid initially at the two-phase Neumann profile above a
    front one cell deep, cold wall at Tc = -0.5 < Tm: 600 steps, every T
    (both phases) and the front."""
    kw = dict(face=face, Ra=0.0, Ste=0.5, Th=1.0, Tc=-0.5, Tm=0.0, s_nu=1.25, s_alpha=2 / 3, solid=1,
              ks_kl=kappa)
    gpu, o = _pair(lib, orc, shape, **kw)
    ig, io = gpu.info(), o.info()
    assert ig["lambda_"] == pytest.approx(io["lambda"], rel=1e-12)
    assert ig["t0"] == pytest.approx(io["t0"], rel=1e-12)
    _compare(gpu, o, tol_u=1e-6)  # the initial state
    gpu.step(600)
    o.step(600)
    dT, _, dS, _ = _compare(gpu, o, tol_u=1e-6)
    Tg = gpu.get()[0]
    assert Tg.min() < -0.1  # the solid is subcooled, not held at Tm


@pytest.mark.parametrize("face,shape", [(0, (40, 24, 20)), (1, (36, 20, 26))])
@pytest.mark.parametrize("steps", [150, 151])
@pytest.mark.parametrize("pairs", [-1, 1])
def test_subcooled_convection_melting(lib, orc, face, shape, steps, pairs):
    """Ra > 0 with a subcooled solid, both heated faces, both AA phases, a
    ragged x extent."""
    kw = dict(face=face, Ra=1e5, Pr=0.1, Ste=1.0, Ma=0.2, s0=3.0, derive=True, Tc=-0.5, Tm=0.0, solid=1,
              ks_kl=1.5)
    gpu, o = _pair(lib, orc, shape, pairs, **kw)
    gpu.step(steps)
    o.step(steps)
    _compare(gpu, o)


@pytest.mark.parametrize("face", [0, 1])
@pytest.mark.parametrize("pairs", [-1, 1])
def test_refreezing_front(lib, orc, face, pairs):
    """A front started near the cold wall recedes (the solid's conduction
    flux exceeds the liquid's): nodes refreeze every few steps in both AA
    phases."""
    shape = (10, 32, 7) if face == 0 else (10, 7, 32)
    kw = dict(face=face, Ra=0.0, Ste=1.0, Th=1.0, Tc=-1.0, Tm=0.0, s0=28.0, s_nu=1.25, s_alpha=1.0, solid=1,
              ks_kl=1.0)
    gpu, o = _pair(lib, orc, shape, pairs, **kw)
    gpu.step(301)
    o.step(301)
    _compare(gpu, o, tol_u=1e-6)
    assert o.get()[2].max() < 26.0  # several layers refroze


def _random_state(o, seed, s_lo, s_hi, Tc, amp=2e-3):
    """Perturbed populations in both phases (the solid's g now matters): T
    linear from the heated wall to Tm at the front in the liquid and from Tm
    to Tc at the cold wall in the solid."""
    nz, ny, nx = o.shape
    H = o.H
    s = inputs.uniform(o.ncols, s_lo, s_hi, seed)
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    col = (Z * nx + X) if o.face == 0 else (Y * nx + X)
    ax = (Y if o.face == 0 else Z) + 0.5
    sc = s[col]
    liq = (ax < sc).reshape(-1)
    T = np.where(ax < sc, 1.0 - ax / sc, Tc * (ax - sc) / (H - sc)).reshape(-1)
    f = inputs.noisy(np.tile(W19[:, None], (1, o.N)), amp, seed + 1)
    f[:, ~liq] = 0.0
    g = W7[:, None] * T[None, :] + amp * 0.1 * inputs.uniform((7, o.N), -1.0, 1.0, seed + 2)
    return f.astype(np.float32), g.astype(np.float32), s


@pytest.mark.parametrize("face", [0, 1])
@pytest.mark.parametrize("nsteps", [1, 2, 3])
@pytest.mark.parametrize("pairs", [-1, 1])
def test_steps_from_random_state(lib, orc, face, nsteps, pairs):
    """A non-flat front and perturbed populations in both phases: after 1,
    2, 3 steps every distribution agrees (liquid f; g of every node)."""
    shape = (14, 10, 9) if face == 0 else (14, 9, 10)
    kw = dict(face=face, Ra=2e4, Pr=0.5, Ste=0.3, Ma=0.15, derive=True, Tc=-0.6, Tm=0.0, solid=1, ks_kl=1.8)
    gpu, o = _pair(lib, orc, shape, pairs, **kw)
    f, g, s = _random_state(o, 7 + face, 2.2, 7.8, -0.6)
    o.set_state(f.astype(np.float64), g.astype(np.float64), s)
    gpu.set_state(f, g, s)
    gpu.step(nsteps)
    o.step(nsteps)
    fg, gg, sg = gpu.get_state()
    fo, go, so = o.get_state()
    np.testing.assert_allclose(sg, so, atol=1e-7, rtol=0)
    np.testing.assert_allclose(gg, go, atol=2e-6, rtol=0)
    np.testing.assert_allclose(fg, fo, atol=2e-6, rtol=0)
    _compare(gpu, o, tol_u=2e-6)


@pytest.mark.parametrize("face", [0, 1])
@pytest.mark.parametrize("direction", ["melt", "freeze"])
@pytest.mark.parametrize("pairs", [-1, 1])
def test_flips_after_even_and_odd_steps(lib, orc, face, direction, pairs):
    """Fronts placed just below node centres (melting) or just above them
    under a strongly subcooled solid (refreezing), so that nodes change
    phase in the first (even, values in flight) and second (odd) steps."""
    shape = (12, 10, 11) if face == 0 else (12, 11, 10)
    Tc = -0.2 if direction == "melt" else -4.0
    kw = dict(face=face, Ra=0.0, Ste=1.0, Tc=Tc, Tm=0.0, s_nu=1.3, s_alpha=1.5, solid=1, ks_kl=1.0)
    gpu, o = _pair(lib, orc, shape, pairs, **kw)
    f, g, s = _random_state(o, 21 + face, 2.0, 6.0, Tc)
    if direction == "melt":
        s = np.floor(s) + 0.5 - inputs.uniform(s.shape, 0.01, 0.03, 5)
    else:
        s = np.floor(s) + 0.5 + inputs.uniform(s.shape, 0.01, 0.03, 5)
    o.set_state(f.astype(np.float64), g.astype(np.float64), s)
    gpu.set_state(f, g, s)
    js0 = np.ceil(s - 0.5)
    # the front moves by FP32 gradients of temperatures up to |Tc|
    tol_s = 1e-7 * max(1.0, abs(Tc))
    for n in range(1, 5):
        gpu.step(1)
        o.step(1)
        fg, gg, sg = gpu.get_state()
        fo, go, so = o.get_state()
        np.testing.assert_allclose(sg, so, atol=tol_s, rtol=0)
        np.testing.assert_allclose(fg, fo, atol=2e-6, rtol=0)
        np.testing.assert_allclose(gg, go, atol=2e-6, rtol=0)
        _compare(gpu, o, tol_u=2e-6)
        if n == 1:
            moved = np.ceil(so - 0.5) - js0
            # a good share of the columns changed phase in the even step (0.47-0.61 of them)
            assert ((moved > 0) if direction == "melt" else (moved < 0)).mean() > 0.4


@pytest.mark.parametrize("kappa", [1.0, 3.0])
def test_held_front_gives_linear_profiles(lib, kappa):
    """Against the closed form, not the oracle: Ste = 0 holds the front, and
    both phases come to the linear conduction profiles between their
    Dirichlet ends (Th at the wall and Tm at s in the liquid, Tm at s and Tc
    at the cold wall in the solid).  The FP32 fixed point lies off the exact
    one by the per-step rounding of the populations times the diffusion time
    of the segment (~1e-8 x L^2 / alpha): 2.5e-6 observed, bar 1e-5; a wrong
    ghost or crossing rule is off by O(1e-2)."""
    H, s0, Th, Tc, Tm = 24, 8.5, 1.0, -1.0, 0.0
    gpu = lib(3, H, 3, Ra=0.0, Ste=0.0, Th=Th, Tc=Tc, Tm=Tm, s0=s0, s_nu=1.25, s_alpha=1.0, solid=1, ks_kl=kappa)
    gpu.step(int(6000 / min(kappa, 1.0)))
    T, u, S, _ = gpu.get()
    a = np.arange(H) + 0.5
    ex = np.where(a < s0, Th + (Tm - Th) * a / s0, Tm + (Tc - Tm) * (a - s0) / (H - s0))
    np.testing.assert_allclose(T, ex[None, :, None] * np.ones(T.shape), atol=1e-5)
    assert np.all(S == s0)


@pytest.mark.parametrize("face", [0, 1])
def test_no_subcooling_is_the_held_solid_method(lib, face):
    """Tc = Tm: the solid stays at Tm exactly, so until the first node
    changes phase the conduction kernels give the held-solid method's
    results (FP32 storage).  The held-solid kernels collide two nodes per
    thread in packed FP32x2 arithmetic and the conduction kernels one, so
    the two agree to FP32 rounding rather than bit for bit."""
    kw = dict(face=face, Ra=5e4, Pr=0.02, Ste=0.1, Ma=0.1, s0=3.0, derive=True, Tc=0.0, Tm=0.0)
    shape = (12, 16, 10) if face == 0 else (12, 10, 16)
    a = lib(*shape, **kw)
    b = lib(*shape, solid=1, ks_kl=2.5, **kw)
    a.step(250)
    b.step(250)
    Ta, ua, Sa, _ = a.get()
    Tb, ub, Sb, _ = b.get()
    assert Sa.min() > 3.2 and Sa.max() < 3.5  # moved, no flip yet
    np.testing.assert_allclose(Sa, Sb, atol=1e-7, rtol=0)  # 1.3e-8 measured
    np.testing.assert_allclose(Ta, Tb, atol=1e-6, rtol=0)
    np.testing.assert_allclose(ua, ub, atol=1e-7, rtol=0)
    # the solid stays at Tm exactly in both
    solid = Ta == 0.0
    assert solid.sum() > 0 and np.all(Tb[solid] == 0.0)


def test_fp16_storage_error(lib, orc):
    """Shifted-FP16 storage with a subcooled solid: the error against the
    FP64 oracle, by phase.  The solid's slow diffusion changes a population
    per step by about its FP16 rounding step (stagnation), so FP16 is far
    less accurate here than with the solid held at Tm (1.8e-4): measured
    3.8e-3 in the liquid, 1.3e-2 in the solid, 5e-4 in the liquid fraction
    after 200 steps; the bars are about twice that.  FP32 storage is the one
    to use with conduction in the solid."""
    kw = dict(face=0, Ra=1e5, Pr=0.1, Ste=1.0, Ma=0.2, s0=3.0, derive=True, Tc=-0.5, Tm=0.0, solid=1, ks_kl=1.5)
    gpu = lib(24, 20, 16, precision=1, **kw)
    o = orc.Oracle(24, 20, 16, **kw)
    gpu.step(200)
    o.step(200)
    Tg, ug, Sg, lfg = gpu.get()
    To, uo, So, lfo = o.get()
    fo = o.get_state()[0]
    liq = fo.any(axis=0).reshape(To.shape)
    dTl, dTs = np.abs(Tg - To)[liq].max(), np.abs(Tg - To)[~liq].max()
    dlf = abs(lfg - lfo)
    print("fp16 storage, subcooled solid: max|dT| liquid %.3g, solid %.3g, |dlf| = %.3g" % (dTl, dTs, dlf))
    assert dTl < 8e-3 and dTs < 3e-2 and dlf < 1e-3


def test_rejections(lib):
    """Conduction is chosen before the first step; the adjoint and the
    ensemble keep the solid at Tm."""
    from paper_1604_03478_gb300 import _abi
    from paper_1604_03478_gb300.cavity import LbmError
    from paper_1604_03478_gb300.ensemble import Ensemble
    gpu = lib(8, 12, 8, Ra=0.0, Ste=0.5, Tc=-0.5, s_nu=1.25, s_alpha=1.0)
    gpu.step(1)
    with pytest.raises(LbmError):
        gpu.set_solid_conduction(1.0)
    g2 = lib(8, 12, 8, Ra=0.0, Ste=0.5, Tc=-0.5, s_nu=1.25, s_alpha=1.0)
    with pytest.raises(LbmError):
        g2.set_solid_conduction(-1.0)
    g2.set_solid_conduction(1.0)
    with pytest.raises(LbmError):
        g2.tape_forward(4)
    ens = Ensemble([dict(nx=16, ny=16, nz=16, Ra=1e4, Pr=0.02, Ste=0.1, face=0, derive=True, Ma=0.1)])
    m = ens.member(0)
    st = _abi.load().lbm_melt_set_solid_conduction(m._h, C.c_double(1.0))
    assert st == _abi.LBM_EINVAL
