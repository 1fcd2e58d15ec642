"""Quadrature nodes/weights and the rational filter (oracle; test infrastructure only).

Readings of the paper used here (it prints no trapezoid formula):
  * nodes theta_j = pi (2j-1)/ne, j = 1..ne (half-offset, counter-clockwise);
  * ellipse z(theta) = c + e^{i phi} (a cos theta + i b sin theta), b = ratio*a;
  * weight w_j = (1/(2 pi i)) z'(theta_j) (2 pi/ne), so that
    rho_a(z) = sum_j w_j/(z_j - z) approximates the Cauchy integral (eq. cauchy).
"""
from __future__ import annotations

import numpy as np


def trapezoid_nodes(center: complex, a: float, ratio: float = 1.0, angle: float = 0.0, ne: int = 8):
    """Trapezoidal rule on a circle/ellipse (Sec. 2.1 contour parameters, Sec. 2.3 rule).

    Returns (z, w), complex arrays of length ne.
    """
    j = np.arange(1, ne + 1)
    theta = np.pi * (2 * j - 1) / ne
    b = ratio * a
    rot = np.exp(1j * angle)
    z = center + rot * (a * np.cos(theta) + 1j * b * np.sin(theta))
    # dz/dtheta = rot*(-a sin + i b cos); w = dz/dtheta * (2pi/ne) / (2 pi i)
    dz = rot * (-a * np.sin(theta) + 1j * b * np.cos(theta))
    w = dz / (1j * ne)
    return z.astype(np.complex128), w.astype(np.complex128)


def contour_nodes(con):
    """Nodes/weights of a Contour (kind 0 circle, 1 ellipse, 2 custom)."""
    if con.kind == 2:
        return np.asarray(con.z, np.complex128), np.asarray(con.w, np.complex128)
    ratio = 1.0 if con.kind == 0 else con.ratio
    angle = 0.0 if con.kind == 0 else con.angle
    return trapezoid_nodes(con.center, con.r, ratio, angle, con.ne)


def rho_a(lam, z, w):
    """Rational filter rho_a(lambda) = sum_j w_j / (z_j - lambda) (eq. rational)."""
    lam = np.asarray(lam, np.complex128)
    out = np.zeros(lam.shape, np.complex128)
    for zj, wj in zip(z, w):
        out += wj / (zj - lam)
    return out


def inside(lam, con):
    """Closed inside test of the search contour (circle or ellipse).  Custom
    contours use the polygon through the nodes (even-odd rule)."""
    lam = np.asarray(lam, np.complex128)
    ok = np.isfinite(lam)
    if con.kind == 2:
        z = np.asarray(con.z)
        x, y = lam.real, lam.imag
        res = np.zeros(lam.shape, bool)
        for k in range(len(z)):
            x1, y1 = z[k].real, z[k].imag
            x2, y2 = z[(k + 1) % len(z)].real, z[(k + 1) % len(z)].imag
            cond = (y1 > y) != (y2 > y)
            with np.errstate(divide="ignore", invalid="ignore"):
                xc = x1 + (y - y1) * (x2 - x1) / (y2 - y1)
            res ^= cond & (x < xc)
        return res & ok
    ratio = 1.0 if con.kind == 0 else con.ratio
    angle = 0.0 if con.kind == 0 else con.angle
    u = np.exp(-1j * angle) * (np.where(ok, lam, 0) - con.center)
    a, b = con.r, ratio * con.r
    return ok & ((u.real / a) ** 2 + (u.imag / b) ** 2 <= 1.0)


def alpha(con):
    """alpha of eq. (res): |lambda_mid| + r (ellipse: the larger semi-axis)."""
    if con.kind == 2:
        z = np.asarray(con.z)
        c = np.mean(z)
        return abs(c) + np.max(np.abs(z - c))
    ratio = 1.0 if con.kind == 0 else con.ratio
    return abs(con.center) + con.r * max(1.0, ratio)
