"""Pins of the oracle's solid-phase conduction (the k_s term of Eq. 6 with a
subcooled solid, Tc < Tm; section 1 allows Tc <= Tm, the paper solves only
Tc = Tm).

Reading of the method: the solid runs the D3Q7 collision at u = 0 with
alpha_s = (k_s / k_l) alpha (equal rho c); the interface is the mirror of the
liquid-side ghost rule on the solid side; Eq. 6 takes
kappa dT_s/da - dT_l/da.  Pinned here against what the mathematics fixes:

* the solid-side stencils are exact on the polynomials they are built on;
* the two-phase Neumann constant equals an independent root of the textbook
  transcendental equation, and theta = 0 gives the one-phase root;
* with Tc = Tm the method is the zero-subcooling one, bit for bit;
* a held front gives the exact linear profiles on both sides;
* a moving front comes to rest where the two conduction fluxes balance,
  s* = H (Th - Tm) / ((Th - Tm) + kappa (Tm - Tc)), from below (melting) and
  from above (refreezing);
* the transient follows the two-phase Neumann solution within a tolerance
  that shrinks under refinement;
* the heat balance (wall heat = sensible + latent) closes to first order;
* a side-heated convection case keeps its mirror symmetry.
"""
import numpy as np
import pytest
from scipy.optimize import brentq
from scipy.special import erf, erfc


def _lambda2(Ste, theta, kappa):
    """Root of the interface balance of the classical two-phase Neumann
    solution (a semi-infinite solid at Tc melted from a wall at Th; Carslaw &
    Jaeger, Conduction of Heat in Solids): with the front s = 2 lambda
    sqrt(alpha_l t), the liquid erf profile and the solid erfc profile,
        lambda sqrt(pi) / Ste = e^{-lambda^2} / erf(lambda)
            - theta (k_s/k_l) sqrt(alpha_l/alpha_s) e^{-lambda^2 alpha_l/alpha_s}
              / erfc(lambda sqrt(alpha_l/alpha_s)),
    theta = (Tm - Tc)/(Th - Tm); here alpha_s / alpha_l = kappa = k_s / k_l
    (equal rho c)."""
    ratio = 1.0 / kappa                  # alpha_l / alpha_s
    nu = np.sqrt(ratio)

    def F(lam):
        liquid = np.exp(-lam * lam) / erf(lam)
        solid = theta * kappa * nu * np.exp(-lam * lam * ratio) / erfc(lam * nu)
        return lam * np.sqrt(np.pi) / Ste - liquid + solid

    return brentq(F, 1e-9, 10.0, xtol=1e-15)


@pytest.mark.parametrize("Ste,theta,kappa", [(0.1, 0.5, 1.0), (0.5, 0.5, 1.0), (1.0, 1.0, 2.0),
                                             (0.5, 0.3, 0.5), (0.2, 2.0, 1.5)])
def test_two_phase_neumann_lambda(orc, Ste, theta, kappa):
    lam = orc.neumann_lambda2(Ste, theta, kappa)
    assert lam == pytest.approx(_lambda2(Ste, theta, kappa), abs=1e-12)
    # subcooling slows the front
    assert lam < orc.neumann_lambda(Ste)


@pytest.mark.parametrize("Ste", [0.1, 0.5, 1.0])
def test_two_phase_lambda_without_subcooling_is_one_phase(orc, Ste):
    assert orc.neumann_lambda2(Ste, 0.0, 2.0) == pytest.approx(orc.neumann_lambda(Ste), abs=1e-12)


# ------------------------------------------------------------- stencils

@pytest.mark.parametrize("s", [3.2, 4.0, 4.5, 4.99, 6.7])
def test_solid_gradient_exact_for_quadratics(orc, s):
    """Quadratic through (s, Tm): the stencil nodes k = ceil(s), k + 1."""
    n, Tm, Tc = 12, 0.3, -2.0
    a = np.arange(n) + 0.5
    T = Tm + 0.7 * (a - s) - 0.05 * (a - s) ** 2
    assert orc.solid_gradient(T, s, Tc, Tm) == pytest.approx(0.7, abs=1e-12)
    # a solid at Tm gives exactly zero, whatever Tc is (Tc only enters at the wall)
    assert orc.solid_gradient(np.full(n, Tm), s, Tc, Tm) == 0.0


def test_solid_gradient_wall_stands_in(orc):
    n, Tm, Tc = 8, 0.0, -1.0
    a = np.arange(n) + 0.5
    for s in (6.2, 6.9):                 # guarded node 7 = n - 1: the wall (n, Tc) is the second point
        slope = (Tc - Tm) / (n - s)
        T = Tm + slope * (a - s)
        assert orc.solid_gradient(T, s, Tc, Tm) == pytest.approx(slope, abs=1e-12)
    # no node at least half a cell above s: linear through (s, Tm) and (n, Tc)
    for s in (7.1, 7.5):
        T = np.zeros(n)
        T[7] = 123.0                     # the only solid node is not used
        assert orc.solid_gradient(T, s, Tc, Tm) == pytest.approx((Tc - Tm) / (n - s), abs=1e-12)


@pytest.mark.parametrize("s", [3.2, 4.0, 4.5, 6.6, 7.3])
def test_solid_ghost_temperature_on_a_line(orc, s):
    """The solid side's ghost sits at the last liquid node (centre js - 1/2)
    and lies on the line through (s, Tm) and the guarded solid node."""
    n, Tm, Tc = 8, 0.2, -1.0
    a = np.arange(n) + 0.5
    js = int(np.ceil(s - 0.5))
    if np.ceil(s) >= n:                  # wall line
        slope = (Tc - Tm) / (n - s)
    else:
        slope = -0.4
    T = Tm + slope * (a - s)
    assert orc.solid_ghost_T(T, s, Tc, Tm) == pytest.approx(Tm + slope * (js - 0.5 - s), abs=1e-12)


def test_solid_ghost_without_a_side_is_tm(orc):
    T = np.linspace(1, -1, 8)
    assert orc.solid_ghost_T(T, 0.5, -1.0, 0.0) == 0.0     # no liquid node
    assert orc.solid_ghost_T(T, 7.8, -1.0, 0.0) == 0.0     # no solid node


# -------------------------------------------------------------- runs

@pytest.mark.parametrize("face", [0, 1])
def test_no_subcooling_reduces_to_held_solid(orc, face):
    """Tc = Tm: the solid stays at Tm exactly, so while no node changes phase
    the conduction build is the zero-subcooling method bit for bit
    (convection, moving fronts, ghost nodes on both sides).  A node that
    melts carries its own populations into the liquid in both builds; they
    are the solid's (at Tm) here and the values streamed into the ghost node
    there, so after the first flip the two differ within the discretisation
    error (next test)."""
    kw = dict(face=face, Ra=5e4, Pr=0.02, Ste=0.1, Ma=0.1, s0=3.0, derive=True, Tc=0.0, Tm=0.0)
    shape = (12, 16, 10) if face == 0 else (12, 10, 16)
    a = orc.Oracle(*shape, **kw)
    b = orc.Oracle(*shape, solid=1, ks_kl=2.5, **kw)
    a.step(250)
    b.step(250)
    Ta, ua, Sa, la = a.get()
    Tb, ub, Sb, lb = b.get()
    assert Sa.min() > 3.2 and Sa.max() < 3.5      # moved, no flip yet
    np.testing.assert_array_equal(Sa, Sb)
    np.testing.assert_array_equal(Ta, Tb)
    np.testing.assert_array_equal(ua, ub)
    fa, ga, _ = a.get_state()
    fb, gb, _ = b.get_state()
    np.testing.assert_array_equal(fa, fb)
    liq = (fa != 0).any(0)
    np.testing.assert_array_equal(ga[:, liq], gb[:, liq])


@pytest.mark.parametrize("Ste", [0.1, 1.0])
def test_no_subcooling_matches_one_phase_neumann(orc, Ste):
    """Tc = Tm with fronts crossing many layers: the conduction build
    follows the one-phase Neumann solution as closely as the held-solid
    build (both first order)."""
    errs = []
    for solid in (0, 1):
        o = orc.Oracle(1, 32, 1, Ra=0.0, Ste=Ste, s_nu=1 / 0.8, s_alpha=2 / 3, solid=solid, ks_kl=1.7)
        info = o.info()
        o.step(1000)
        t = info["t0"] + 1000
        _, _, S, _ = o.get()
        s_exact = 2 * info["lambda"] * np.sqrt(info["alpha"] * t)
        errs.append(abs(S.flat[0] - s_exact) / s_exact)
    assert errs[1] < 0.01 and errs[1] < 2 * errs[0] + 1e-3


@pytest.mark.parametrize("kappa", [1.0, 3.0])
def test_held_front_gives_linear_profiles(orc, kappa):
    """Ste = 0 holds the front; both phases reach the linear conduction
    profiles between their Dirichlet ends: Th at the wall and Tm at s in the
    liquid, Tm at s and Tc at the cold wall in the solid."""
    H, s0, Th, Tc, Tm = 24, 8.5, 1.0, -1.0, 0.0
    o = orc.Oracle(3, H, 3, Ra=0, Ste=0.0, Th=Th, Tc=Tc, Tm=Tm, s0=s0, s_alpha=1.0, solid=1, ks_kl=kappa)
    o.step(int(6000 / min(kappa, 1.0)))
    T, u, S, _ = o.get()
    a = np.arange(H) + 0.5
    ex = np.where(a < s0, Th + (Tm - Th) * a / s0, Tm + (Tc - Tm) * (a - s0) / (H - s0))
    np.testing.assert_allclose(T, ex[None, :, None] * np.ones(o.shape), atol=1e-6)
    assert np.all(S == s0)


@pytest.mark.parametrize("kappa,Tc,s0", [(1.0, -1.0, 4.0), (2.0, -1.0, 4.0), (0.5, -0.5, 4.0),
                                         (1.0, -1.0, 28.0)])
def test_front_comes_to_rest_where_fluxes_balance(orc, kappa, Tc, s0):
    """Steady state of Eq. 6 in one dimension: linear profiles on both sides
    and k_l (Th - Tm) / s = k_s (Tm - Tc) / (H - s).  From s0 = 28 the front
    recedes (refreezing) to the same height."""
    H, Th, Tm = 32, 1.0, 0.0
    o = orc.Oracle(3, H, 3, Ra=0, Ste=1.0, Th=Th, Tc=Tc, Tm=Tm, s0=s0, s_alpha=1.0, solid=1, ks_kl=kappa)
    o.step(40000)
    _, _, S, _ = o.get()
    s_star = H * (Th - Tm) / ((Th - Tm) + kappa * (Tm - Tc))
    np.testing.assert_allclose(S, s_star, atol=1e-7)


def _two_phase_run(orc, Ste, theta, kappa, n, depth=2):
    H = depth * n
    o = orc.Oracle(1, H, 1, Ra=0, Ste=Ste, Th=1.0, Tc=-theta, Tm=0.0, s0=1.0, s_nu=1 / 0.8, s_alpha=2 / 3,
                   solid=1, ks_kl=kappa)
    info = o.info()
    steps = int(round(1000 * (n / 32) ** 2))
    o.step(steps)
    t = info["t0"] + steps
    T, _, S, _ = o.get()
    lam = _lambda2(Ste, theta, kappa)
    a, a_s = info["alpha"], info["alpha_s"]
    assert a_s == pytest.approx(kappa * a, rel=1e-14)
    s_exact = 2 * lam * np.sqrt(a * t)
    y = np.arange(H) + 0.5
    T_exact = np.where(y < s_exact, 1 - erf(y / (2 * np.sqrt(a * t))) / erf(lam),
                       -theta + theta * erfc(y / (2 * np.sqrt(a_s * t))) / erfc(lam / np.sqrt(kappa)))
    return abs(S.flat[0] - s_exact) / s_exact, np.abs(T[0, :, 0] - T_exact).max()


@pytest.mark.parametrize("Ste,theta,kappa,depth", [(0.5, 0.5, 1.0, 2), (1.0, 1.0, 2.0, 4), (0.5, 0.3, 0.5, 2)])
def test_subcooled_conduction_melting_matches_two_phase_neumann(orc, Ste, theta, kappa, depth):
    """1000 steps from a front one cell deep, 32 cells to the front's scale;
    the cavity is deep enough that the cold wall is not felt (semi-infinite
    solid)."""
    ds, dT = _two_phase_run(orc, Ste, theta, kappa, 32, depth)
    assert ds < 0.02 and dT < 0.02


def test_two_phase_error_shrinks_under_refinement(orc):
    errs = [_two_phase_run(orc, 0.5, 0.5, 1.0, n) for n in (16, 32, 64)]
    assert errs[0][0] > errs[1][0] > errs[2][0]
    assert errs[0][1] > errs[1][1] > errs[2][1]


@pytest.mark.parametrize("kappa", [1.0, 2.0])
def test_energy_balance_with_solid_conduction(orc, kappa):
    """Heat through the two isothermal walls = sensible heat of both phases
    (equal rho c) + latent heat (Th - Tm)/Ste per melted volume; the
    imbalance is first-order and shrinks with refinement."""
    rel = []
    for n in (16, 32):
        o = orc.Oracle(2, n, 2, Ra=0, Ste=0.5, Th=1.0, Tc=-0.5, Tm=0.0, s_nu=1 / 0.8, s_alpha=2 / 3, solid=1,
                       ks_kl=kappa)
        i0 = o.info()
        lf0 = o.get()[3]
        o.step(int(1000 * (n / 32) ** 2))
        i1 = o.info()
        lf1 = o.get()[3]
        assert i1["q_cold"] < 0                          # heat leaves through the cold wall
        q = i1["q_hot"] + i1["q_cold"]
        sensible = (i1["sum_T_liquid"] + i1["sum_T_solid"]) - (i0["sum_T_liquid"] + i0["sum_T_solid"])
        latent = (1.0 / 0.5) * (lf1 - lf0) * n * 4
        rel.append(abs(q - sensible - latent) / i1["q_hot"])
    assert rel[0] < 0.05 and rel[1] < rel[0]


def test_subcooled_convection_mirror_symmetry(orc):
    """Side heating with a subcooled solid: the problem is symmetric about
    the mid x plane, and so must be T, s and the mirrored velocity."""
    o = orc.Oracle(10, 12, 10, face=0, Ra=2e4, Pr=0.02, Ste=0.2, Ma=0.1, s0=3.5, derive=True, Tc=-0.5, Tm=0.0,
                   solid=1, ks_kl=1.5)
    o.step(300)
    T, u, s, _ = o.get()
    assert np.ptp(s) > 0.01 and T.min() < -0.1
    np.testing.assert_allclose(T, T[:, :, ::-1], atol=1e-12)
    np.testing.assert_allclose(u[..., 0], -u[:, :, ::-1, 0], atol=1e-12)
    np.testing.assert_allclose(u[..., 1:], u[:, :, ::-1, 1:], atol=1e-12)
    np.testing.assert_allclose(s, s[:, ::-1], atol=1e-12)


def test_subcooling_slows_convection_melting(orc):
    kw = dict(face=0, Ra=2e4, Pr=0.02, Ste=0.2, Ma=0.1, s0=3.5, derive=True, Tm=0.0)
    lf = []
    for Tc, solid in ((0.0, 0), (-0.5, 1), (-1.0, 1)):
        o = orc.Oracle(8, 12, 8, Tc=Tc, solid=solid, **kw)
        o.step(300)
        lf.append(o.get()[3])
    assert lf[0] > lf[1] > lf[2]


def test_phase_crossing_links_one_step(orc):
    """One step from a stepped, held front (Ste = 0), checked link by link.
    Column x = 1 has its front at 2.4 (liquid nodes 0, 1), its neighbours at
    6.3 (liquid nodes 0..5).  After the streaming:
    * a solid node of column 1 whose lateral neighbour is liquid but not that
      column's last liquid node receives the rest state at Tm, w_i Tm;
    * a liquid node whose lateral neighbour in column 1 is solid but not
      column 1's first solid node receives w_i Tm as well;
    * along a column, the first solid node receives from the last liquid
      node the solid side's ghost population, and the last liquid node from
      the first solid node the liquid side's (each built from the state
      before the step: an extrapolated temperature plus the non-equilibrium
      part of the neighbour on its own side); a solid node beside a last
      liquid node receives that node's solid-side ghost population too."""
    nx, H, nz, Tm, Tc = 4, 8, 3, 0.3, -0.7
    o = orc.Oracle(nx, H, nz, face=0, Ra=0.0, Ste=0.0, Th=1.0, Tc=Tc, Tm=Tm, s0=6.3, s_alpha=1.3,
                   solid=1, ks_kl=1.7)
    e7, w7, opp7 = orc.lattice7()
    rng = np.random.default_rng(3)
    g0 = w7[:, None] * rng.uniform(-0.5, 1.0, o.N)[None, :] + 0.01 * rng.standard_normal((7, o.N))
    f0 = np.tile(orc.feq19(1.0, [0, 0, 0])[:, None], (1, o.N))
    s = np.full(o.cols_shape, 6.3)
    s[:, 1] = 2.4
    o.set_state(f0, g0, s)
    o.step(1)
    g1 = o.get_state()[1]
    idx = lambda x, y, z: (z * H + y) * nx + x                  # noqa: E731
    px = next(i for i in range(7) if tuple(e7[i]) == (1, 0, 0))   # streams from x - 1
    mx = next(i for i in range(7) if tuple(e7[i]) == (-1, 0, 0))  # streams from x + 1
    up = next(i for i in range(7) if tuple(e7[i]) == (0, 1, 0))
    dn = next(i for i in range(7) if tuple(e7[i]) == (0, -1, 0))
    for z in range(nz):
        for y in (3, 4):          # solid in column 1, not its first solid node; liquid, not last, at x = 0, 2
            assert g1[px, idx(1, y, z)] == w7[px] * Tm
            assert g1[mx, idx(1, y, z)] == w7[mx] * Tm
            assert g1[mx, idx(0, y, z)] == w7[mx] * Tm          # from column 1's solid node at x = 1
            assert g1[px, idx(2, y, z)] == w7[px] * Tm
    # along column (x = 0, z = 1): nodes 5 (last liquid) and 6 (first solid)
    T0 = g0.sum(0)
    x, z = 0, 1
    Tcol = np.array([T0[idx(x, j, z)] for j in range(H)])
    zero = np.zeros(3)
    Q7s = np.array([1.0] + [1.0 / (1.7 * 0.25 * (1 / 1.3 - 0.5) / 0.25 + 0.5)] * 3 + [1.0, 1.0, 1.0])
    Tgs = orc.solid_ghost_T(Tcol, 6.3, Tc, Tm)
    spost = orc.geq7(Tgs, zero) + orc.collide_g(g0[:, idx(x, 6, z)], Q7s, zero) - orc.geq7(Tcol[6], zero)
    np.testing.assert_allclose(g1[up, idx(x, 6, z)], spost[up], rtol=0, atol=1e-14)
    # laterally, the same ghost feeds column 1's solid node beside it
    np.testing.assert_allclose(g1[px, idx(1, 5, z)], spost[px], rtol=0, atol=1e-14)
    assert Tgs == pytest.approx(Tm + (Tcol[7] - Tm) * (5.5 - 6.3) / (7.5 - 6.3), abs=1e-14)
    Tg = orc.ghost_T(Tcol, 6.3, 1.0, Tm)
    fL = f0[:, idx(x, 5, z)]
    _, uL = orc.collide_f(fL, np.ones(19), [0.0, 0.0, 0.0])
    Q7l = np.array([1.0, 1.3, 1.3, 1.3, 1.0, 1.0, 1.0])
    gpost = orc.geq7(Tg, zero) + orc.collide_g(g0[:, idx(x, 5, z)], Q7l, uL) - orc.geq7(Tcol[5], uL)
    np.testing.assert_allclose(g1[dn, idx(x, 5, z)], gpost[dn], rtol=0, atol=1e-14)
