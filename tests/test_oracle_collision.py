"""Pins of the oracle's MRT collisions (paper Eqs. 1, 2, 4) and forcing.

MRT with every rate equal must reduce to BGK; equilibria are fixed points;
mass is conserved and momentum changes by exactly the force; the Guo source
has the moments that define it.  The BGK reference here is written from the
textbook single-relaxation-time formula, not from the oracle.
"""
import numpy as np
import pytest

W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
W7 = np.array([1 / 4] + [1 / 8] * 6)


def _lat(orc):
    e, w, opp = orc.lattice19()
    np.testing.assert_allclose(w, W19)
    return e.astype(float)


def _bgk_feq(e, rho, u):
    eu = e @ u
    return W19 * (rho + 3 * eu + 4.5 * eu ** 2 - 1.5 * (u @ u))


def _guo(e, u, F):
    return W19 * (3 * ((e - u) @ F) + 9 * (e @ u) * (e @ F))


def _rand_f(rng, e):
    rho = 1 + 0.05 * rng.standard_normal()
    u = 0.05 * rng.standard_normal(3)
    return _bgk_feq(e, rho, u) + 1e-3 * rng.standard_normal(19)


def test_equilibrium_is_fixed_point(orc):
    e = _lat(orc)
    rng = np.random.default_rng(10)
    rates = rng.uniform(0.5, 1.9, 19)
    for _ in range(10):
        rho = 1 + 0.05 * rng.standard_normal()
        u = 0.05 * rng.standard_normal(3)
        fe = _bgk_feq(e, rho, u)
        out, uo = orc.collide_f(fe, rates, [0, 0, 0])
        np.testing.assert_allclose(out, fe, atol=1e-15)
        np.testing.assert_allclose(uo, u, atol=1e-15)


@pytest.mark.parametrize("force", [False, True])
def test_mrt_reduces_to_bgk(orc, force):
    e = _lat(orc)
    rng = np.random.default_rng(11)
    for _ in range(10):
        tau = rng.uniform(0.51, 2.0)
        f = _rand_f(rng, e)
        F = 1e-3 * rng.standard_normal(3) if force else np.zeros(3)
        rho = f.sum()
        u = f @ e + F / 2
        want = f - (f - _bgk_feq(e, rho, u)) / tau + (1 - 0.5 / tau) * _guo(e, u, F)
        out, _ = orc.collide_f(f, np.full(19, 1 / tau), F)
        np.testing.assert_allclose(out, want, atol=1e-15)


def test_collision_conserves_mass_and_adds_force(orc):
    e = _lat(orc)
    rng = np.random.default_rng(12)
    for _ in range(10):
        f = _rand_f(rng, e)
        F = 1e-3 * rng.standard_normal(3)
        rates = rng.uniform(0.3, 1.95, 19)
        out, _ = orc.collide_f(f, rates, F)
        assert out.sum() == pytest.approx(f.sum(), abs=1e-14)
        np.testing.assert_allclose(out @ e, f @ e + F, atol=1e-15)


def test_guo_source_moments(orc):
    e = _lat(orc)
    rng = np.random.default_rng(13)
    for _ in range(10):
        u = 0.05 * rng.standard_normal(3)
        F = rng.standard_normal(3)
        Fi = orc.guo19(u, F)
        np.testing.assert_allclose(Fi, _guo(e, u, F), atol=1e-15)
        assert abs(Fi.sum()) < 1e-14
        np.testing.assert_allclose(Fi @ e, F, atol=1e-14)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", Fi, e, e),
                                   np.outer(u, F) + np.outer(F, u), atol=1e-14)


def test_d3q7_bgk_and_conservation(orc):
    e7, w7, _ = orc.lattice7()
    np.testing.assert_allclose(w7, W7)
    rng = np.random.default_rng(14)
    for _ in range(10):
        T = rng.uniform(0, 1)
        u = 0.05 * rng.standard_normal(3)
        ge = W7 * T * (1 + 4 * (e7 @ u))
        np.testing.assert_allclose(orc.geq7(T, u), ge, atol=1e-15)
        g = ge + 1e-3 * rng.standard_normal(7)
        Tg = g.sum()
        tau = rng.uniform(0.51, 2)
        want = g - (g - W7 * Tg * (1 + 4 * (e7 @ u))) / tau
        np.testing.assert_allclose(orc.collide_g(g, np.full(7, 1 / tau), u), want, atol=1e-15)
        out = orc.collide_g(g, rng.uniform(0.3, 1.9, 7), u)
        assert out.sum() == pytest.approx(Tg, abs=1e-15)
        # equilibrium is a fixed point
        np.testing.assert_allclose(orc.collide_g(ge, rng.uniform(0.3, 1.9, 7), u), ge, atol=1e-15)
