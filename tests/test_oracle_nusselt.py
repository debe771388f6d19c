"""Pins of the oracle's heat-surface Nusselt number (section 3.2, Figs. 4(b)
and 5: Nu on the heated wall, its 3-D distribution and its dependence on
Ra).  Nu = -H (dT/da at the wall) / (Th - Tm), from the flux the last
streaming carried through the wall links.

Closed forms fix it: a held front between the heated wall and Tm gives the
exact linear profile, so Nu = H / s0 to round-off; conduction melting follows
the Neumann solution, whose wall gradient gives Nu(t) = H / (sqrt(pi alpha t)
erf(lambda)), met to first order (the error shrinks under refinement).  The
convection findings of section 3.2 are checked on a small cavity."""
import numpy as np
import pytest
from scipy.special import erf


@pytest.mark.parametrize("face", [0, 1])
@pytest.mark.parametrize("s0", [3.0, 5.5, 8.3, 10.5])
def test_nusselt_held_front_is_exact(orc, face, s0):
    shape = (3, 16, 4) if face == 0 else (3, 4, 16)
    o = orc.Oracle(*shape, face=face, Ra=0, Ste=0.0, Th=1.7, Tm=0.2, Tc=0.2, s0=s0, s_nu=1.2, s_alpha=1.0)
    o.step(3000)
    nu, mean = o.nusselt()
    np.testing.assert_allclose(nu, 16.0 / s0, rtol=1e-10)
    assert mean == pytest.approx(16.0 / s0, rel=1e-10)


def _neumann_nu(orc, Ste, n):
    o = orc.Oracle(2, n, 2, Ra=0, Ste=Ste, s_nu=1.2, s_alpha=2 / 3, s0=1.0)
    info = o.info()
    steps = int(1000 * (n / 32) ** 2)
    o.step(steps)
    _, mean = o.nusselt()
    t = info["t0"] + steps
    ref = n / (np.sqrt(np.pi * info["alpha"] * t) * erf(info["lambda"]))
    return abs(mean - ref) / ref


@pytest.mark.parametrize("Ste", [0.1, 0.5, 1.0])
def test_nusselt_conduction_melting_matches_neumann(orc, Ste):
    assert _neumann_nu(orc, Ste, 32) < 0.01


@pytest.mark.parametrize("Ste", [0.5, 1.0])
def test_nusselt_error_shrinks_under_refinement(orc, Ste):
    e = [_neumann_nu(orc, Ste, n) for n in (16, 32, 64)]
    assert e[2] < e[1] < e[0]


def test_nusselt_convection_findings(orc):
    """Section 3.2: with convection the heated wall's Nu is largest at mid x
    (the no-slip side walls slow the flow near them), and a lower Ra gives a
    lower Nu at the same Fourier number (case 2 against case 1)."""
    means = []
    for Ra in (1e5, 1e4):
        o = orc.Oracle(11, 16, 16, face=0, Ra=Ra, Pr=0.1, Ste=1.0, Ma=0.2, s0=3.0, derive=True)
        info = o.info()
        steps = int(round(0.1 * 16 ** 2 / info["alpha"]))
        o.step(steps)
        nu, mean = o.nusselt()
        means.append(mean)
        if Ra == 1e5:
            over_x = nu.mean(axis=0)  # columns are (z, x): average over height
            assert over_x[5] > over_x[0] and over_x[5] > over_x[-1]
            np.testing.assert_allclose(over_x, over_x[::-1], rtol=1e-10)  # mirror symmetry in x
    assert means[0] > means[1]
