"""Pins of the oracle's streaming and boundary rules (paper section 1 and
Eqs. 1, 4), by brute force on tiny cavities with the collision switched off
(every relaxation rate 0 makes the collision the identity when F = 0)."""
import numpy as np
import pytest

ZERO_RATES = dict(s_nu=0.0, s_alpha=0.0, s_e=0.0, s_eps=0.0, s_q=0.0, s_pi=0.0, s_m=0.0,
                  s_g4=0.0, s_g5=0.0)


def _free(orc, nx, ny, nz, s0, face=0):
    return orc.Oracle(nx, ny, nz, face=face, Ra=0.0, Ste=0.0, Th=1.0, Tc=0.0, Tm=0.0, s0=s0, **ZERO_RATES)


def _idx(o, x, y, z):
    nz, ny, nx = o.shape
    return (z * ny + y) * nx + x


@pytest.mark.parametrize("i", range(1, 19))
def test_f_delta_streams_one_link(orc, i):
    e, w, opp = orc.lattice19()
    o = _free(orc, 5, 6, 7, s0=6.0)  # all liquid
    f = np.tile(w[:, None], (1, o.N))
    g = np.zeros((7, o.N))
    x0 = (2, 3, 3)
    f[i, _idx(o, *x0)] += 0.01
    o.set_state(f, g)
    o.step(1)
    f1, _, _ = o.get_state()
    want = np.tile(w[:, None], (1, o.N))
    dst = tuple(np.add(x0, e[i]))
    want[i, _idx(o, *dst)] += 0.01
    np.testing.assert_allclose(f1, want, atol=1e-15)


@pytest.mark.parametrize("i", range(1, 19))
def test_f_bounce_back_at_walls(orc, i):
    e, w, opp = orc.lattice19()
    o = _free(orc, 3, 4, 3, s0=4.0)
    for x0 in [(0, 0, 0), (2, 3, 2), (1, 0, 2), (0, 3, 1)]:
        dst = np.add(x0, e[i])
        if (dst >= 0).all() and (dst < [3, 4, 3]).all():
            continue
        f = np.tile(w[:, None], (1, o.N))
        f[i, _idx(o, *x0)] += 0.01
        o.set_state(f, np.zeros((7, o.N)), np.full(o.ncols, 4.0))
        o.step(1)
        f1, _, _ = o.get_state()
        want = np.tile(w[:, None], (1, o.N))
        want[opp[i], _idx(o, *x0)] += 0.01
        np.testing.assert_allclose(f1, want, atol=1e-15)


def test_f_bounce_back_at_solid_node(orc):
    e, w, opp = orc.lattice19()
    o = _free(orc, 4, 6, 4, s0=3.0)  # nodes y = 0, 1, 2 liquid
    for i in (3, 7, 8, 15, 17):      # directions with +y component
        f = np.tile(w[:, None], (1, o.N))
        f[i, _idx(o, 1, 2, 1)] += 0.01
        o.set_state(f, np.zeros((7, o.N)), np.full(o.ncols, 3.0))
        o.step(1)
        f1, _, _ = o.get_state()
        assert f1[opp[i], _idx(o, 1, 2, 1)] == pytest.approx(w[opp[i]] + 0.01, abs=1e-15)


def test_g_anti_bounce_back_and_adiabatic(orc):
    """All liquid, g = 0: after one step the heated-wall nodes hold 2 w T_h in
    the population entering from the wall, the cold-wall nodes 2 w T_c = 0,
    and a delta aimed at an adiabatic wall comes back unchanged."""
    o = _free(orc, 3, 5, 4, s0=5.0)
    e7, w7, opp7 = orc.lattice7()
    g = np.zeros((7, o.N))
    g[1, _idx(o, 2, 2, 1)] = 0.3   # +x at the x = nx-1 adiabatic wall
    g[4, _idx(o, 1, 0, 2)] = 0.2   # -y at the heated wall y = 0
    o.set_state(np.tile(orc.lattice19()[1][:, None], (1, o.N)), g)
    o.step(1)
    _, g1, _ = o.get_state()
    want = np.zeros((7, o.N))
    for x in range(3):
        for z in range(4):
            want[3, _idx(o, x, 0, z)] = 2 * w7[3] * 1.0
    want[2, _idx(o, 2, 2, 1)] = 0.3
    want[3, _idx(o, 1, 0, 2)] += -0.2
    np.testing.assert_allclose(g1, want, atol=1e-15)


def test_g_bottom_heated_walls(orc):
    """Heated face z = 0: the Dirichlet walls are z = 0 and z = H."""
    o = _free(orc, 3, 4, 5, s0=5.0, face=1)
    e7, w7, _ = orc.lattice7()
    o.set_state(np.tile(orc.lattice19()[1][:, None], (1, o.N)), np.zeros((7, o.N)))
    o.step(1)
    _, g1, _ = o.get_state()
    g1 = g1.reshape(7, 5, 4, 3)
    np.testing.assert_allclose(g1[5, 0], 2 * w7[5], atol=1e-15)
    g1[5, 0] = 0
    np.testing.assert_allclose(g1, 0, atol=1e-15)
