"""Closed-form chi for a static spherically symmetric source (Sec. 2.7, Eq. analytical, Eq. Ar).

TEST INFRASTRUCTURE ONLY (part of the oracle package).

In code units the chi equation is nu L(chi) - kappa q2(chi) = xi S with
S = (3/2)(G_eff/G) a Omega_m0 delta.  For a spherical field write X = chi'/r.
Then L(chi) = (r^3 X)'/r^2 and the screening bracket (L chi)^2 - chi_ij chi^ij
equals (2/r^2)(r^3 X^2)'.  Integrating once from the centre gives the algebraic
relation  nu X - 2 kappa X^2 = xi y_N,  where y_N(r) = r^-3 int_0^r s^2 S(s) ds.
This is Eq. analytical with A = y_N/(E^2 a^4) and x = X/(E^2 a^4).  Its root
continuous with the linear solution is
    X = 2 xi y_N / (nu + sgn(nu) sqrt(nu^2 - 8 kappa xi y_N)),
and chi(r) = -int_r^inf s X(s) ds (chi -> 0 at infinity, as in Sec. 3.6.1).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

_GL_X, _GL_W = np.polynomial.legendre.leggauss(48)


def _X_of_y(y, nu, kappa, xi):
    s = 1.0 if nu >= 0 else -1.0
    disc = nu * nu - 8.0 * kappa * xi * y
    if np.any(disc < 0):
        raise ValueError("source too strong: no real solution (Sec. 3.3 condition)")
    return 2.0 * xi * y / (nu + s * np.sqrt(disc))


def tophat_yN(r, S0, R):
    """y_N for a top-hat S = S0 (r < R), 0 outside: S0/3 inside, S0 R^3/(3 r^3) outside."""
    r = np.asarray(r, dtype=float)
    return np.where(r <= R, S0 / 3.0, S0 * R ** 3 / (3.0 * np.maximum(r, 1e-300) ** 3))


def gauss_yN(r, S0, s):
    """y_N for S = S0 exp(-r^2/(2 s^2)) (closed-form enclosed integral with erf)."""
    r = np.asarray(r, dtype=float)
    rr = np.maximum(r, 1e-300)
    q = rr / s
    enc = S0 * s ** 3 * (np.sqrt(np.pi / 2.0) * erf(q / np.sqrt(2.0)) - q * np.exp(-0.5 * q * q))
    small = S0 / 3.0 * (1.0 - 0.3 * q * q)  # series near the centre, avoids cancellation
    return np.where(q < 1e-3, small, enc / rr ** 3)


def tophat_profile(r, S0, R, nu, kappa, xi):
    """chi(r) for the top-hat source: closed form inside R, quadrature of X outside."""
    r = np.asarray(r, dtype=float)
    Xin = _X_of_y(S0 / 3.0, nu, kappa, xi)
    # outside: y_N = A t^3 with A = S0 R^3 / (3 r^3); integrand is smooth in t
    def outside(rv):
        rv = np.maximum(rv, R)
        t = 0.5 * (_GL_X + 1.0)
        w = 0.5 * _GL_W
        rv = rv[..., None]
        y = S0 * R ** 3 / (3.0 * rv ** 3) * t ** 3
        X = _X_of_y(y, nu, kappa, xi)
        return -np.sum(w * rv ** 2 * X / t ** 3, axis=-1)
    chiR = outside(np.array(R))
    inside = chiR - Xin * (R * R - r * r) / 2.0
    return np.where(r <= R, inside, outside(r))


def gauss_profile(r, S0, s, nu, kappa, xi):
    """chi(r) for a Gaussian source; the integrand of the t-quadrature is smooth everywhere."""
    r = np.asarray(r, dtype=float)
    # integrate from r outward in pieces: [r, r + 12 s] with Gauss-Legendre, tail via t-substitution
    a = r[..., None]
    b = a + 12.0 * s
    x = 0.5 * (_GL_X + 1.0)
    w = 0.5 * _GL_W
    pieces = 8
    total = np.zeros(r.shape)
    for k in range(pieces):
        lo = a + (b - a) * k / pieces
        hi = a + (b - a) * (k + 1) / pieces
        sv = lo + (hi - lo) * x
        X = _X_of_y(gauss_yN(sv, S0, s), nu, kappa, xi)
        total += np.sum(w * (hi - lo) * sv * X, axis=-1)
    # tail beyond b: the enclosed integral has saturated, y_N = M_tot / r^3
    Mtot = S0 * s ** 3 * np.sqrt(np.pi / 2.0)
    rb = b[..., 0]
    t = x
    svt = rb[..., None] / t
    X = _X_of_y(Mtot / svt ** 3, nu, kappa, xi)
    total += np.sum(w * rb[..., None] ** 2 * X / t ** 3, axis=-1)
    return -total


def radial_derivative_ratio(yN_val, nu, kappa, xi):
    """Psi'/Psi'_GR = (y_N + xi X)/y_N (Eq. analytical, y row), the quantity of Fig. spher-ana."""
    X = _X_of_y(yN_val, nu, kappa, xi)
    return (yN_val + xi * X) / yN_val
