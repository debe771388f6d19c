"""GPU parity of the two-nodes-per-thread stream-collide (lbm_melt_set_node_pairs
mode 1: x-adjacent nodes as the lanes of packed FP32x2 arithmetic) at small
sizes, where the default chooses one node per thread: against the FP64
oracle with the plain method's tolerances, and against the one-node kernels
to FP32 rounding.  Pairs at x = 0 and x = nx - 1, at the interface (one-node
fallback per node), across flips in the even and the odd step, and FP16
storage are covered."""
import numpy as np
import pytest

from paper_1604_03478_gb300 import inputs

pytestmark = pytest.mark.gpu

W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
W7 = np.array([1 / 4] + [1 / 8] * 6)


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1604_03478_gb300 import build, Cavity
    build.build()
    return Cavity


def _pairs(lib, shape, **kw):
    c = lib(*shape, **kw)
    c.set_node_pairs(1)
    return c


def _compare(gpu, o, tol_T=1e-4, tol_lf=1e-3, tol_u=1e-4):
    Tg, ug, Sg, lfg = gpu.get()
    To, uo, So, lfo = o.get()
    assert np.abs(Tg - To).max() <= tol_T
    assert np.abs(ug - uo).max() <= tol_u
    assert np.abs(Sg - So).max() <= tol_lf
    assert abs(lfg - lfo) <= tol_lf


def _random_state(o, seed, s_lo, s_hi, amp=2e-3):
    nz, ny, nx = o.shape
    s = inputs.uniform(o.ncols, s_lo, s_hi, seed)
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    col = (Z * nx + X) if o.face == 0 else (Y * nx + X)
    ax = (Y if o.face == 0 else Z) + 0.5
    sc = s[col]
    liq = (ax < sc).reshape(-1)
    T = np.where(ax < sc, 1.0 - ax / sc, 0.0).reshape(-1)
    f = inputs.noisy(np.tile(W19[:, None], (1, o.N)), amp, seed + 1)
    f[:, ~liq] = 0.0
    g = inputs.noisy(W7[:, None] * T[None, :], amp, seed + 2)
    return f.astype(np.float32), g.astype(np.float32), s


@pytest.mark.parametrize("face,shape", [(0, (40, 24, 20)), (1, (36, 20, 26))])
@pytest.mark.parametrize("steps", [150, 151])
def test_convection_melting(lib, orc, face, shape, steps):
    kw = dict(face=face, Ra=1e5, Pr=0.1, Ste=1.0, Ma=0.2, s0=3.0, derive=True)
    gpu, o = _pairs(lib, shape, **kw), orc.Oracle(*shape, **kw)
    gpu.step(steps)
    o.step(steps)
    _compare(gpu, o)


@pytest.mark.parametrize("face", [0, 1])
@pytest.mark.parametrize("nsteps", [1, 2, 3])
def test_steps_from_random_state(lib, orc, face, nsteps):
    """Every distribution after 1, 2, 3 steps from a perturbed, non-flat
    state (the interior pairs, the x-wall pairs, the pairs split by the
    front)."""
    shape = (14, 10, 9) if face == 0 else (14, 9, 10)
    kw = dict(face=face, Ra=2e4, Pr=0.5, Ste=0.3, Ma=0.15, derive=True)
    gpu, o = _pairs(lib, shape, **kw), orc.Oracle(*shape, **kw)
    f, g, s = _random_state(o, 7 + face, 2.2, 7.8)
    o.set_state(f.astype(np.float64), g.astype(np.float64), s)
    gpu.set_state(f, g, s)
    gpu.step(nsteps)
    o.step(nsteps)
    fg, gg, sg = gpu.get_state()
    fo, go, so = o.get_state()
    liq = fo.any(axis=0)
    np.testing.assert_allclose(sg, so, atol=1e-7, rtol=0)
    np.testing.assert_allclose(gg[:, liq], go[:, liq], atol=2e-6, rtol=0)
    np.testing.assert_allclose(fg, fo, atol=2e-6, rtol=0)


@pytest.mark.parametrize("face", [0, 1])
def test_flips_after_even_and_odd_steps(lib, orc, face):
    shape = (12, 10, 11) if face == 0 else (12, 11, 10)
    kw = dict(face=face, Ra=0.0, Ste=1.0, s_nu=1.3, s_alpha=1.5)
    gpu, o = _pairs(lib, shape, **kw), orc.Oracle(*shape, **kw)
    f, g, s = _random_state(o, 21 + face, 2.0, 6.0)
    s = np.floor(s) + 0.5 - inputs.uniform(s.shape, 0.01, 0.03, 5)
    o.set_state(f.astype(np.float64), g.astype(np.float64), s)
    gpu.set_state(f, g, s)
    for n in range(1, 5):
        gpu.step(1)
        o.step(1)
        fg, gg, sg = gpu.get_state()
        fo, go, so = o.get_state()
        liq = fo.any(axis=0)
        np.testing.assert_allclose(sg, so, atol=1e-7, rtol=0)
        np.testing.assert_allclose(fg, fo, atol=2e-6, rtol=0)
        np.testing.assert_allclose(gg[:, liq], go[:, liq], atol=2e-6, rtol=0)


def test_pairs_and_single_nodes_agree(lib):
    """Both variants of the same run, FP32 storage: FP32 rounding apart."""
    kw = dict(face=0, Ra=5e4, Pr=0.2, Ste=0.5, Ma=0.15, s0=2.5, derive=True)
    a = lib(32, 18, 16, **kw)
    a.set_node_pairs(0)
    b = _pairs(lib, (32, 18, 16), **kw)
    a.step(200)
    b.step(200)
    Ta, ua, Sa, la = a.get()
    Tb, ub, Sb, lb = b.get()
    np.testing.assert_allclose(Ta, Tb, atol=2e-6, rtol=0)
    np.testing.assert_allclose(ua, ub, atol=2e-7, rtol=0)
    np.testing.assert_allclose(Sa, Sb, atol=1e-6, rtol=0)


def test_fp16_storage_error(lib, orc):
    """Shifted-FP16 storage on the pair kernels against the FP64 oracle
    (1.5e-4 measured; the one-node kernels' bar)."""
    kw = dict(face=0, Ra=1e5, Pr=0.1, Ste=1.0, Ma=0.2, s0=3.0, derive=True)
    gpu = _pairs(lib, (24, 20, 16), precision=1, **kw)
    o = orc.Oracle(24, 20, 16, **kw)
    gpu.step(200)
    o.step(200)
    Tg, _, _, lfg = gpu.get()
    To, _, _, lfo = o.get()
    dT = np.abs(Tg - To).max()
    print("fp16 pairs: max|dT| = %.3g" % dT)
    assert dT < 5e-4 and abs(lfg - lfo) < 1e-5


def test_mode_checks(lib):
    from paper_1604_03478_gb300.cavity import LbmError
    c = lib(13, 10, 9, Ra=0.0, Ste=0.5, s_nu=1.25, s_alpha=1.0)
    with pytest.raises(LbmError):
        c.set_node_pairs(1)  # odd nx
    with pytest.raises(LbmError):
        c.set_node_pairs(2)
    c.set_node_pairs(0)
    c.set_node_pairs(-1)
