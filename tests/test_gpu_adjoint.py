"""GPU tests of the hand-written adjoint (lbm_melt_tape_forward/backward):
gradients of the final liquid fraction and of an L2 front mismatch, with
respect to Ra and to the heated-wall temperature field, against the
complex-step tangent-linear FP64 oracle and central finite differences of
the FP64 oracle (flags held: no node changes phase between the perturbed
runs), within 1e-3 relative."""
import numpy as np
import pytest

from paper_1604_03478_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = {
    0: dict(face=0, Ra=2e4, Pr=0.3, Ste=0.5, Ma=0.15, s0=3.0),
    1: dict(face=1, Ra=3e4, Pr=0.5, Ste=0.4, Ma=0.15, s0=2.6),
}
SHAPES = {0: (10, 12, 8), 1: (9, 8, 12)}
STEPS = 60
REL = 1e-3


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1604_03478_gb300 import build, Cavity
    build.build()
    return Cavity


def _gpu(lib, face, seed_fn, ckpt=8, steps=STEPS):
    cav = lib(*SHAPES[face], derive=True, **CASES[face])
    cav.set_hot_wall(np.full(cav.ncols, 1.0, np.float32))
    cav.tape_forward(steps, ckpt)
    S = cav.get(T=False, u=False)[2]
    dth, par = cav.tape_backward(seed_fn(S, cav))
    return cav, S, dth, par


def _lf_seed(S, cav):
    return np.full(cav.ncols, 1.0 / (cav.H * cav.ncols))


@pytest.mark.parametrize("face", [0, 1])
def test_liquid_fraction_gradient_vs_tangent_oracle(lib, orc, face):
    cav, S, dth, par = _gpu(lib, face, _lf_seed)
    ncols = cav.ncols
    _, _, _, dlf_ra = orc.tangent(*SHAPES[face], STEPS, dRa=1.0, derive=True, **CASES[face])
    assert par["Ra"] == pytest.approx(dlf_ra, rel=REL)
    for k in range(3):
        v = inputs.gaussian_field(ncols, 1.0, 100 + k)
        _, _, _, dlf_v = orc.tangent(*SHAPES[face], STEPS, dThw=v, derive=True, **CASES[face])
        assert float(dth.ravel() @ v) == pytest.approx(dlf_v, rel=REL)
    cav.close()


def test_front_mismatch_gradient(lib, orc):
    """L = sum (S - S*)^2 with S* the final front of a run whose wall is
    perturbed by a seeded Gaussian field (sigma 0.01): a reachable target."""
    face = 0
    ncols = SHAPES[face][0] * SHAPES[face][2]
    o = orc.Oracle(*SHAPES[face], derive=True, **CASES[face])
    o.set_hot_wall(1.0 + inputs.gaussian_field(ncols, 0.01, 7))
    o.step(STEPS)
    S_target = o.get()[2].ravel()
    cav, S, dth, par = _gpu(lib, face, lambda S, c: 2.0 * (S.ravel() - S_target))
    resid = S.ravel() - S_target
    v = inputs.gaussian_field(ncols, 1.0, 9)
    _, dS_v, _, _ = orc.tangent(*SHAPES[face], STEPS, dThw=v, derive=True, **CASES[face])
    assert float(dth.ravel() @ v) == pytest.approx(float(2.0 * resid @ dS_v.ravel()), rel=REL)
    _, dS_ra, _, _ = orc.tangent(*SHAPES[face], STEPS, dRa=1.0, derive=True, **CASES[face])
    assert par["Ra"] == pytest.approx(float(2.0 * resid @ dS_ra.ravel()), rel=REL)
    cav.close()


def test_gradient_vs_central_differences(lib, orc):
    """Central differences of the FP64 oracle along Ra and along a wall
    direction, with eps small enough that no node changes phase."""
    face = 0
    cav, S, dth, par = _gpu(lib, face, _lf_seed)
    res = []
    for sgn in (1, -1):
        kw = dict(CASES[face])
        kw["Ra"] += sgn * 2.0
        oo = orc.Oracle(*SHAPES[face], derive=True, **kw)
        oo.step(STEPS)
        res.append((oo.get()[3], oo.info()["n_liquid"]))
    assert res[0][1] == res[1][1]
    assert par["Ra"] == pytest.approx((res[0][0] - res[1][0]) / 4.0, rel=REL)
    v = inputs.gaussian_field(cav.ncols, 1.0, 5)
    res = []
    for sgn in (1, -1):
        oo = orc.Oracle(*SHAPES[face], derive=True, **CASES[face])
        oo.set_hot_wall(1.0 + sgn * 1e-4 * v)
        oo.step(STEPS)
        res.append((oo.get()[3], oo.info()["n_liquid"]))
    assert res[0][1] == res[1][1]
    assert float(dth.ravel() @ v) == pytest.approx((res[0][0] - res[1][0]) / 2e-4, rel=REL)
    cav.close()


def test_fp16_storage_gradient(lib):
    """Shifted FP16 storage (FP32 arithmetic): the recorded run and its
    snapshots are FP16-rounded, the adjoint itself is FP32; the gradient stays
    within the 1e-3 relative bar of the FP32-storage one."""
    out = {}
    for prec in (0, 1):
        cav = lib(*SHAPES[0], precision=prec, derive=True, **CASES[0])
        cav.set_hot_wall(np.full(cav.ncols, 1.0, np.float32))
        cav.tape_forward(STEPS, 8)
        out[prec] = cav.tape_backward(_lf_seed(None, cav))
        cav.close()
    (d32, p32), (d16, p16) = out[0], out[1]
    assert p16["Ra"] == pytest.approx(p32["Ra"], rel=REL)
    v = inputs.gaussian_field(d32.size, 1.0, 100)
    assert float(d16.ravel() @ v) == pytest.approx(float(d32.ravel() @ v), rel=REL)


def test_checkpoint_spacing_does_not_change_the_gradient(lib):
    out = [_gpu(lib, 0, _lf_seed, ckpt=c) for c in (1, 7, STEPS)]
    for cav, S, dth, par in out[1:]:
        np.testing.assert_array_equal(dth, out[0][2])
        assert par == out[0][3]
    for o in out:
        o[0].close()


def test_backward_leaves_the_final_state(lib):
    cav = lib(*SHAPES[0], derive=True, **CASES[0])
    cav.tape_forward(25, 6)
    before = cav.get()
    f0, g0, s0 = cav.get_state()
    cav.tape_backward(np.ones(cav.ncols))
    after = cav.get()
    f1, g1, s1 = cav.get_state()
    for a, b in zip(before[:3], after[:3]):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(f0, f1)
    np.testing.assert_array_equal(s0, s1)
    cav.step(3)  # still steps
    cav.close()


def test_autograd_function(lib):
    import torch
    from paper_1604_03478_gb300.autograd import melt_front
    face = 0
    spec = dict(nx=SHAPES[face][0], ny=SHAPES[face][1], nz=SHAPES[face][2], **{k: v for k, v in CASES[face].items()
                                                                              if k != "Ra"})
    ncols = SHAPES[face][0] * SHAPES[face][2]
    dTh = torch.zeros(ncols, dtype=torch.float64, device="cuda", requires_grad=True)
    Ra = torch.tensor(CASES[face]["Ra"], dtype=torch.float64, device="cuda", requires_grad=True)
    S = melt_front(dTh, Ra, spec, STEPS, 8)
    loss = S.sum() / (SHAPES[face][1] * ncols)
    loss.backward()
    cav, S2, dth, par = _gpu(lib, face, _lf_seed)
    np.testing.assert_allclose(dTh.grad.cpu().numpy(), dth.ravel(), rtol=1e-6, atol=1e-12)
    assert float(Ra.grad) == pytest.approx(par["Ra"], rel=1e-6)
    cav.close()
