"""Pins of the oracle's quadrature and rational filter (Sec. 2.1, Sec. 2.3, eq. rational)."""
import numpy as np
import pytest

from oracle.contour import alpha, contour_nodes, inside, rho_a, trapezoid_nodes
from paper_1506_04463_gb300.workloads import Contour


@pytest.mark.parametrize("ne", [4, 8, 16])
def test_circle_filter_closed_form(ne):
    # Half-offset trapezoid nodes are the roots of s^ne = -1 scaled onto the
    # circle, so the quadrature of the Cauchy integral sums to 1/(1+s^ne).
    c, r = 0.3 - 1.2j, 0.7
    z, w = trapezoid_nodes(c, r, 1.0, 0.0, ne)
    rng = np.random.default_rng(5)
    s = rng.uniform(-1.6, 1.6, 20) + 1j * rng.uniform(-1.6, 1.6, 20)
    s = np.concatenate([s, [0, 0.625, 1.25, 0.625j]])
    got = rho_a(c + r * s, z, w)
    assert np.max(np.abs(got - 1.0 / (1.0 + s ** ne))) < 1e-13


def test_nodes_on_contour_and_weight_moments():
    z, w = trapezoid_nodes(1 + 1j, 2.0, 0.5, 0.3, 16)
    u = np.exp(-0.3j) * (z - (1 + 1j))
    assert np.allclose((u.real / 2.0) ** 2 + (u.imag / 1.0) ** 2, 1.0, atol=1e-14)
    # (1/2 pi i) oint z^k dz = 0 for k >= 0: the trapezoid rule is exact for
    # low-degree trigonometric polynomials.
    for k in range(4):
        assert abs(np.sum(w * z ** k)) < 1e-13
    # the nodes run counter-clockwise: the signed area is positive
    area = 0.5 * np.sum(z.real * np.roll(z.imag, -1) - np.roll(z.real, -1) * z.imag)
    assert area > 0


def test_ellipse_reduces_to_circle():
    z1, w1 = trapezoid_nodes(2.0, 0.5, 1.0, 0.0, 8)
    con = Contour(1, 2.0, 0.5, ratio=1.0, angle=0.0, ne=8)
    z2, w2 = contour_nodes(con)
    assert np.allclose(z1, z2, atol=0) and np.allclose(w1, w2, atol=0)
    assert np.allclose(z1, 2.0 + 0.5 * np.exp(1j * np.pi * (2 * np.arange(1, 9) - 1) / 8))
    assert np.allclose(w1, 0.5 * np.exp(1j * np.pi * (2 * np.arange(1, 9) - 1) / 8) / 8)


def test_ellipse_exponential_convergence():
    # Sec. 2.3: the trapezoid rule converges exponentially in ne; inside ->1, outside ->0.
    c, a, ratio, phi = 1 + 1j, 2.0, 0.5, 0.3
    errs_in, errs_out = [], []
    p_out = c + 1.5 * a * np.exp(1j * phi)
    for ne in (8, 16, 32):
        z, w = trapezoid_nodes(c, a, ratio, phi, ne)
        errs_in.append(abs(rho_a(c, z, w) - 1))
        errs_out.append(abs(rho_a(p_out, z, w)))
    assert errs_in[0] > 10 * errs_in[1] > 100 * errs_in[2]
    assert errs_out[0] > 10 * errs_out[1] > 100 * errs_out[2]
    assert errs_in[2] < 1e-6 and errs_out[2] < 1e-7


def test_inside_and_alpha():
    con = Contour(1, 1.0 + 0j, 2.0, ratio=0.5, angle=0.0, ne=8)
    pts = np.array([1.0, 2.9, 3.1, 1 + 0.9j, 1 + 1.1j, np.inf, np.nan])
    assert list(inside(pts, con)) == [True, True, False, True, False, False, False]
    assert alpha(con) == pytest.approx(3.0)
    assert alpha(Contour(0, 3j, 0.5)) == pytest.approx(3.5)
