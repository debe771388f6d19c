"""Pins of the oracle's interfacial tracking (paper Eq. 6, section 3.1).

The gradient and ghost rules are exact for polynomials they are built on;
the Neumann root is checked against an independent root finder and its
small-Stefan asymptote; a held front gives the exact linear conduction
profile; a moving front follows the analytic conduction-melting solution
(zero subcooling) within a tolerance that shrinks under refinement.
"""
import numpy as np
import pytest
from scipy.optimize import brentq
from scipy.special import erf

# roots of lambda exp(lambda^2) erf(lambda) = Ste / sqrt(pi), six decimals
TABULATED_LAMBDA = {0.05: 0.156821, 0.1: 0.220016, 0.2: 0.306424, 0.5: 0.464786, 1.0: 0.620063}


@pytest.mark.parametrize("Ste", sorted(TABULATED_LAMBDA))
def test_neumann_lambda(orc, Ste):
    lam = orc.neumann_lambda(Ste)
    ref = brentq(lambda l: l * np.exp(l * l) * erf(l) - Ste / np.sqrt(np.pi), 1e-9, 5, xtol=1e-15)
    assert lam == pytest.approx(ref, abs=1e-12)
    assert lam == pytest.approx(TABULATED_LAMBDA[Ste], abs=1e-6)


def test_neumann_lambda_small_ste(orc):
    for Ste in (1e-4, 1e-3):
        assert orc.neumann_lambda(Ste) == pytest.approx(np.sqrt(Ste / 2), rel=Ste)


@pytest.mark.parametrize("s", [1.0, 1.3, 1.9, 2.0, 2.4, 3.7, 5.5, 9.99])
def test_gradient_exact_for_quadratic(orc, s):
    # T(y) = Tm + b (y - s) + c (y - s)^2, so T(s) = Tm and T'(s) = b
    Tm, b, c = 0.2, -0.7, 0.05
    n = 12
    y = np.arange(n) + 0.5
    T = Tm + b * (y - s) + c * (y - s) ** 2
    Tw = Tm + b * (0 - s) + c * s ** 2
    assert orc.front_gradient(T, s, Tw, Tm) == pytest.approx(b, abs=1e-12)


@pytest.mark.parametrize("s", [0.5, 0.75, 0.99])
def test_gradient_linear_below_one_cell(orc, s):
    T = np.zeros(8)
    assert orc.front_gradient(T, s, 1.0, 0.0) == pytest.approx(-1.0 / s, abs=1e-14)


@pytest.mark.parametrize("s", [0.6, 1.0, 1.2, 2.5, 2.51, 4.9, 7.0])
def test_ghost_exact_for_linear(orc, s):
    Tm, b, n = 0.1, -0.3, 10
    y = np.arange(n) + 0.5
    T = Tm + b * (y - s)
    Tw = Tm + b * (0 - s)
    js = int(np.sum(y < s))
    assert orc.ghost_T(T, s, Tw, Tm) == pytest.approx(Tm + b * (js + 0.5 - s), abs=1e-13)


def test_node_at_front_is_solid(orc):
    o = orc.Oracle(2, 8, 2, Ra=0, Ste=0.0, s0=2.5, s_nu=1.2, s_alpha=1.0)
    o.step(3)
    T, u, s, lf = o.get()
    # node centres 0.5, 1.5 liquid; 2.5 (== s) solid and reported at Tm
    assert o.info()["n_liquid"] == 2 * 2 * 2
    assert T[0, 2, 0] == 0.0 and T[0, 1, 0] > 0.0


@pytest.mark.parametrize("s0", [3.0, 8.3, 8.5, 8.7])
def test_held_front_gives_linear_profile(orc, s0):
    """Ste = 0 holds the front; the steady state is T = Th - (Th - Tm) a / s0
    between the heated wall and the front."""
    o = orc.Oracle(1, 16, 1, Ra=0, Ste=0.0, s0=s0, s_nu=1 / 0.8, s_alpha=2 / 3)
    o.step(8000)
    T, u, s, lf = o.get()
    y = np.arange(16) + 0.5
    want = np.where(y < s0, 1 - y / s0, 0.0)
    np.testing.assert_allclose(T.ravel(), want, atol=1e-10)


@pytest.mark.parametrize("Tc", [0.0, -0.5])
def test_all_liquid_wall_to_wall_profile(orc, Tc):
    o = orc.Oracle(2, 12, 2, Ra=0, Ste=0.0, Th=1.0, Tc=Tc, Tm=0.0, s0=12.0, s_nu=1 / 0.8, s_alpha=1.2)
    o.step(6000)
    T, u, s, lf = o.get()
    y = np.arange(12) + 0.5
    np.testing.assert_allclose(T[0, :, 0], 1 + (Tc - 1) * y / 12, atol=1e-10)


def _neumann_run(orc, Ste, n, face=0, lateral=2):
    shape = (lateral, n, lateral) if face == 0 else (lateral, lateral, n)
    o = orc.Oracle(*shape, face=face, Ra=0.0, Ste=Ste, s_nu=1 / 0.8, s_alpha=2 / 3)
    info = o.info()
    steps = int(round(1000 * (n / 32) ** 2))
    o.step(steps)
    t = info["t0"] + steps
    T, u, s, lf = o.get()
    lam, a = info["lambda"], info["alpha"]
    s_exact = 2 * lam * np.sqrt(a * t)
    y = np.arange(n) + 0.5
    Tcol = T[0, :, 0] if face == 0 else T[:, 0, 0]
    T_exact = np.where(y < s.flat[0], 1 - erf(y / (2 * np.sqrt(a * t))) / erf(lam), 0.0)
    return o, s, lf, s_exact / n, np.abs(Tcol - T_exact).max(), u


@pytest.mark.parametrize("Ste", [0.1, 0.5, 1.0])
def test_conduction_melting_matches_neumann(orc, Ste):
    """Section 3.1: conduction melting against the analytic solution, 32 cells
    along the heating axis, 1000 steps from a front one cell deep."""
    o, s, lf, lf_exact, dT, u = _neumann_run(orc, Ste, 32)
    assert abs(lf - lf_exact) / lf_exact < 0.01
    assert dT < 0.01
    assert np.ptp(s) < 1e-12           # the front stays flat without convection
    assert np.abs(u).max() < 1e-12     # and nothing moves


def test_conduction_melting_bottom_heated(orc):
    o, s, lf, lf_exact, dT, u = _neumann_run(orc, 0.5, 32, face=1)
    assert abs(lf - lf_exact) / lf_exact < 0.01 and dT < 0.01


@pytest.mark.parametrize("Ste", [0.5, 1.0])
def test_conduction_error_shrinks_under_refinement(orc, Ste):
    errs = []
    for n in (16, 32, 64):
        o, s, lf, lf_exact, dT, u = _neumann_run(orc, Ste, n, lateral=1)
        errs.append((abs(lf - lf_exact) / lf_exact, dT))
    assert errs[0][0] > errs[1][0] > errs[2][0]
    assert errs[0][1] > errs[1][1] > errs[2][1]


def test_receding_front_refreezes_a_node(orc):
    """Refreezing (R11: flips both ways).  A liquid layer colder than Tm
    below a flat front makes dT/da > 0 at the front, so Eq. 6 moves it back
    towards the heated wall; the layer it leaves becomes solid: its f is
    dropped (reported 0, T reported Tm), and on the next step every link
    pointing down from it into the liquid bounces back, so the node below
    receives its own post-collision value in the opposite direction."""
    n, s0 = 8, 5.51                                   # layer 5 (centre 5.5) just below the front
    o = orc.Oracle(4, n, 3, face=0, Ra=0, Ste=1.0, Th=1.0, Tm=0.0, s0=s0, s_nu=1.2, s_alpha=1.0)
    e, w, opp = orc.lattice19()
    e7, w7, _ = orc.lattice7()
    nz, ny, nx = o.shape
    y = (np.arange(ny) + 0.5)[None, :, None] * np.ones(o.shape)
    # liquid from Th at the wall down to -0.4 just below the front (colder than Tm = 0)
    T = np.where(y < s0, 1.0 - 1.4 * y / 5.5, 0.0)
    f0 = np.tile(w[:, None], (1, o.N))
    o.set_state(f0, w7[:, None] * T.reshape(1, -1), np.full(o.ncols, s0))
    o.step(1)
    _, _, s1, _ = o.get()
    assert np.all(s1 < 5.5) and np.all(s1 > 5.0)    # the front receded over layer 5
    f1, g1, _ = o.get_state()
    T1 = o.get()[0]
    f1 = f1.reshape((19,) + o.shape)
    assert np.all(f1[:, :, 5, :] == 0.0)              # dropped
    assert np.all(T1[:, 5, :] == 0.0)                 # reported at Tm
    # the next step: node (x, 4, z) pulls the directions with e_y = -1 from
    # layer 5, now solid, so it gets back its own post-collision f_opp(i)
    S19 = np.array([1.0, 1.19, 1.4, 1.0, 1.2, 1.0, 1.2, 1.0, 1.2, 1.2, 1.4, 1.2, 1.4, 1.2, 1.2, 1.2,
                    1.98, 1.98, 1.98])
    x, z = 1, 1
    fstar, _ = orc.collide_f(f1[:, z, 4, x], S19, [0.0, 0.0, 0.0])
    o.step(1)
    f2 = o.get_state()[0].reshape((19,) + o.shape)
    down = [i for i in range(19) if e[i, 1] == -1]
    assert len(down) == 5
    for i in down:
        assert f2[i, z, 4, x] == pytest.approx(fstar[opp[i]], abs=1e-15)
