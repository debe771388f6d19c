"""Pins of the complex-step tangent-linear oracle (the FP64 oracle source
built in double _Complex): its directional derivatives of the final front
and liquid fraction, with respect to Ra and to the heated-wall field, agree
with central finite differences of the FP64 oracle while no node changes
phase, are linear in the direction, and reproduce the derivative of the
analytic conduction-melting solution."""
import numpy as np
import pytest
from scipy.special import erf

from paper_1604_03478_gb300 import inputs

CASE = dict(face=0, Ra=2e4, Pr=0.3, Ste=0.5, Ma=0.15, s0=3.0, derive=True)
SHAPE = (10, 12, 8)
STEPS = 60


def _fd(orc, eps, dRa=0.0, dThw=None, case=CASE, shape=SHAPE, steps=STEPS):
    out = []
    for sgn in (1, -1):
        kw = dict(case)
        kw["Ra"] = case["Ra"] + sgn * eps * dRa
        o = orc.Oracle(*shape, **kw)
        if dThw is not None:
            o.set_hot_wall(case.get("Th", 1.0) + sgn * eps * np.asarray(dThw))
        o.step(steps)
        T, u, S, lf = o.get()
        out.append((S, lf, o.info()["n_liquid"]))
    (Sp, lp, np_), (Sm, lm, nm) = out
    assert np_ == nm, "a node changed phase between the +eps and -eps runs"
    return (Sp - Sm) / (2 * eps), (lp - lm) / (2 * eps)


def test_tangent_ra_matches_central_fd(orc):
    S, dS, lf, dlf = orc.tangent(*SHAPE, STEPS, dRa=1.0, **CASE)
    dS_fd, dlf_fd = _fd(orc, eps=2.0, dRa=1.0)
    scale = np.abs(dS).max()
    assert scale > 0
    np.testing.assert_allclose(dS, dS_fd, atol=1e-5 * scale, rtol=0)
    assert dlf == pytest.approx(dlf_fd, rel=1e-5)


def test_tangent_wall_field_matches_central_fd(orc):
    ncols = SHAPE[0] * SHAPE[2]
    v = inputs.gaussian_field(ncols, 1.0, 11)
    S, dS, lf, dlf = orc.tangent(*SHAPE, STEPS, dThw=v, **CASE)
    dS_fd, dlf_fd = _fd(orc, eps=1e-4, dThw=v)
    scale = np.abs(dS).max()
    np.testing.assert_allclose(dS, dS_fd, atol=1e-5 * scale, rtol=0)
    assert dlf == pytest.approx(dlf_fd, rel=1e-5)


def test_tangent_is_linear_in_the_direction(orc):
    ncols = SHAPE[0] * SHAPE[2]
    v1 = inputs.gaussian_field(ncols, 1.0, 1)
    v2 = inputs.gaussian_field(ncols, 1.0, 2)
    a = orc.tangent(*SHAPE, 20, dRa=3.0, dThw=v1, **CASE)[3]
    b = orc.tangent(*SHAPE, 20, dRa=-1.0, dThw=v2, **CASE)[3]
    c = orc.tangent(*SHAPE, 20, dRa=2.0 * 3.0 - 1.0, dThw=2 * v1 + v2, **CASE)[3]
    assert c == pytest.approx(2 * a + b, rel=1e-10)


def test_tangent_conduction_closed_form(orc):
    """Ra = 0: raising the whole heated wall by dT raises the effective
    Stefan number Ste (Th + dT - Tm)/(Th - Tm); the analytic front is
    s = 2 lambda(Ste') sqrt(alpha t), so ds/dT = 2 sqrt(alpha t) lambda'(Ste)
    Ste / (Th - Tm).  The discrete front's derivative tracks it within a few
    percent (the start from a one-cell front is the same for both signs)."""
    Ste, n, steps = 0.5, 48, 2500
    kw = dict(face=0, Ra=0.0, Ste=Ste, s_nu=1 / 0.8, s_alpha=2 / 3)
    S, dS, lf, dlf = orc.tangent(1, n, 1, steps, dThw=np.ones(1), **kw)
    info = orc.Oracle(1, n, 1, **kw).info()
    lam, a, t = info["lambda"], info["alpha"], info["t0"] + steps
    F1 = np.exp(lam ** 2) * erf(lam) * (1 + 2 * lam ** 2) + 2 * lam / np.sqrt(np.pi)
    dlam = (1 / np.sqrt(np.pi)) / F1
    ds_exact = 2 * np.sqrt(a * t) * dlam * Ste / 1.0
    assert float(dS.ravel()[0]) == pytest.approx(ds_exact, rel=0.05)


def test_golden_adjoint_values_are_consistent():
    """The stored gradients of the 96^3 x 4000-step adjoint workload
    (tests/golden/adjoint_96cube_4000steps.txt, written from the oracle by
    oracle/make_golden_adjoint.py): the complex-step derivative along the
    seed-7 wall direction agrees with the central differences of the real
    oracle (no column ended with another liquid count), to the accuracy a
    difference quotient with eps = 1e-9 allows."""
    from conftest import GOLDEN
    import os
    g = {}
    with open(os.path.join(GOLDEN, "adjoint_96cube_4000steps.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()
                g[k] = float(v)
    assert g["fd_count_changes"] == 0
    assert g["fd_dlf_dv1"] == pytest.approx(g["dlf_dv1"], rel=2e-4)
    assert 0.05 < g["liquid_fraction"] < 0.2
    assert g["dlf_dRa"] < 0 and g["dL2_dv1"] < 0
