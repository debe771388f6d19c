"""Pins of the oracle's lattices, transforms and equilibria (paper Eqs. 2-5).

These check the oracle against what the paper prints (the velocity sets of
Eqs. 3 and 5) and against closed forms of the moment bases it defers to
(d'Humieres et al. 2002 for D3Q19; the orthogonal D3Q7 basis), so that a
wrong row, sign or index in the oracle fails here.
"""
import itertools

import numpy as np
import pytest

from conftest import load_golden

D3Q19_NORMS = [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8]
D3Q7_NORMS = [7, 2, 2, 2, 42, 12, 4]


def test_d3q19_velocities_match_eq3(orc):
    e, w, opp = orc.lattice19()
    printed = load_golden("eq3_d3q19_velocities.txt").astype(int)
    assert printed.shape == (3, 19)
    np.testing.assert_array_equal(e.T, printed)


def test_d3q7_velocities_match_eq5(orc):
    e, w, opp = orc.lattice7()
    printed = load_golden("eq5_d3q7_velocities.txt").astype(int)
    np.testing.assert_array_equal(e.T, printed)


def test_opposites(orc):
    e, w, opp = orc.lattice19()
    np.testing.assert_array_equal(e[opp], -e)
    assert list(opp) == [0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 14, 13, 12, 11, 18, 17, 16, 15]
    e7, w7, opp7 = orc.lattice7()
    np.testing.assert_array_equal(e7[opp7], -e7)


def test_d3q19_weights_isotropy(orc):
    e, w, _ = orc.lattice19()
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    d = np.eye(3)
    for a, b in itertools.product(range(3), repeat=2):
        assert np.sum(w * e[:, a] * e[:, b]) == pytest.approx(d[a, b] / 3, abs=1e-15)
    for a, b, c in itertools.product(range(3), repeat=3):
        assert abs(np.sum(w * e[:, a] * e[:, b] * e[:, c])) < 1e-15
    for a, b, c, dd in itertools.product(range(3), repeat=4):
        want = (d[a, b] * d[c, dd] + d[a, c] * d[b, dd] + d[a, dd] * d[b, c]) / 9
        assert np.sum(w * e[:, a] * e[:, b] * e[:, c] * e[:, dd]) == pytest.approx(want, abs=1e-15)


def test_d3q7_weights(orc):
    e, w, _ = orc.lattice7()
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    # second moment c_sT^2 delta with c_sT^2 = 1/4
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, e, e), np.eye(3) / 4, atol=1e-15)


def test_M_rows_orthogonal_with_dhumieres_norms(orc):
    M, Minv, N, Ninv = orc.matrices()
    G = M @ M.T
    np.testing.assert_allclose(np.diag(G), D3Q19_NORMS, atol=1e-12)
    np.testing.assert_allclose(G - np.diag(np.diag(G)), 0, atol=1e-12)
    np.testing.assert_allclose(Minv @ M, np.eye(19), atol=1e-13)
    # for orthogonal rows the inverse is M^T D^-1
    np.testing.assert_allclose(Minv, M.T / np.array(D3Q19_NORMS), atol=1e-14)


def test_N_rows_orthogonal(orc):
    M, Minv, N, Ninv = orc.matrices()
    G = N @ N.T
    np.testing.assert_allclose(np.diag(G), D3Q7_NORMS, atol=1e-13)
    np.testing.assert_allclose(G - np.diag(np.diag(G)), 0, atol=1e-13)
    np.testing.assert_allclose(Ninv @ N, np.eye(7), atol=1e-14)


def _meq_dhumieres(rho, j):
    """Closed-form D3Q19 moment equilibria (d'Humieres et al. 2002),
    incompressible form with rho0 = 1 and the "stable" choices
    w_eps = 3, w_epsj = -11/2, w_xx = -1/2."""
    jx, jy, jz = j
    jj = jx * jx + jy * jy + jz * jz
    pxx = 2 * jx * jx - jy * jy - jz * jz
    pww = jy * jy - jz * jz
    return np.array([rho, -11 * rho + 19 * jj, 3 * rho - 5.5 * jj,
                     jx, -2 / 3 * jx, jy, -2 / 3 * jy, jz, -2 / 3 * jz,
                     pxx, -0.5 * pxx, pww, -0.5 * pww,
                     jx * jy, jy * jz, jx * jz, 0, 0, 0])


def test_meq_is_M_times_feq(orc):
    rng = np.random.default_rng(1)
    M, *_ = orc.matrices()
    for _ in range(20):
        rho = 1 + 0.1 * rng.standard_normal()
        u = 0.1 * rng.standard_normal(3)
        np.testing.assert_allclose(M @ orc.feq19(rho, u), _meq_dhumieres(rho, u), atol=2e-15)


def test_feq_moments(orc):
    e, w, _ = orc.lattice19()
    rng = np.random.default_rng(2)
    for _ in range(10):
        rho = 1 + 0.1 * rng.standard_normal()
        u = 0.1 * rng.standard_normal(3)
        fe = orc.feq19(rho, u)
        assert fe.sum() == pytest.approx(rho, abs=1e-15)
        np.testing.assert_allclose(fe @ e, u, atol=1e-15)
        # incompressible: Pi = rho/3 I + u u (rho0 = 1)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", fe, e, e),
                                   rho / 3 * np.eye(3) + np.outer(u, u), atol=1e-15)


def test_neq_closed_form(orc):
    M, Minv, N, Ninv = orc.matrices()
    rng = np.random.default_rng(3)
    for _ in range(10):
        T = rng.uniform(-1, 2)
        u = 0.1 * rng.standard_normal(3)
        want = np.array([T, u[0] * T, u[1] * T, u[2] * T, 0.75 * T, 0, 0])
        np.testing.assert_allclose(N @ orc.geq7(T, u), want, atol=1e-15)
