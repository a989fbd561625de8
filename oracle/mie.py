"""Closed-form solutions for the sound-soft unit sphere (test infrastructure).

Series from the addition theorem for Phi (the paper's sphere results cite the
Mie series of Bowman et al.; Section 5.1).  For the combined-field operator
A = 1/2 + D - i eta S on the unit sphere every spherical harmonic of degree n
is an eigenfunction:

    S[Y_n] = i k j_n(k) h_n(k) Y_n,    D[Y_n] = (i k^2 j_n'(k) h_n(k) - 1/2) Y_n,
    A Y_n = lambda_n Y_n,   lambda_n = i k h_n(k) (k j_n'(k) - i eta j_n(k)),

h_n = j_n + i y_n the spherical Hankel function of the first kind.  The plane
wave e^{i k d.x} = sum_n i^n (2n+1) j_n(k|x|) P_n(xhat.d), so the solution of
A phi = -u^i (Eq. CombLayIE) is phi = -sum_n i^n (2n+1) j_n(k) / lambda_n P_n,
and the far field of the scattered wave in the normalisation of Eq. FarField is
u_inf(xhat) = (i/k) sum_n (2n+1) (j_n(k) / h_n(k)) P_n(xhat.d).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import eval_legendre, spherical_jn, spherical_yn


def _nmax(k: float) -> int:
    return int(k + 40)


def hankel1(n, z):
    return spherical_jn(n, z) + 1j * spherical_yn(n, z)


def eigenvalue(n, k: float, eta: float):
    """lambda_n of A = 1/2 + D - i eta S on the unit sphere."""
    return 1j * k * hankel1(n, k) * (k * spherical_jn(n, k, derivative=True) - 1j * eta * spherical_jn(n, k))


def single_layer_eigenvalue(n, k):
    return 1j * k * spherical_jn(n, k) * hankel1(n, k)


def double_layer_eigenvalue(n, k):
    return 1j * k * k * spherical_jn(n, k, derivative=True) * hankel1(n, k) - 0.5


def density(points, k: float, eta: float, d=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Exact CFIE density on the unit sphere for incidence u^i = exp(i k d.x)."""
    x = np.asarray(points, dtype=np.float64)
    xh = x / np.linalg.norm(x, axis=1, keepdims=True)
    c = xh @ np.asarray(d, dtype=np.float64)
    phi = np.zeros(x.shape[0], dtype=np.complex128)
    for n in range(_nmax(k) + 1):
        phi -= (1j ** n) * (2 * n + 1) * spherical_jn(n, k) / eigenvalue(n, k, eta) * eval_legendre(n, c)
    return phi


def far_field(xhat, k: float, d=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Exact far-field pattern (Eq. FarField normalisation) of the sound-soft unit sphere."""
    xh = np.asarray(xhat, dtype=np.float64)
    c = xh @ np.asarray(d, dtype=np.float64)
    u = np.zeros(xh.shape[0], dtype=np.complex128)
    for n in range(_nmax(k) + 1):
        u += (2 * n + 1) * (spherical_jn(n, k) / hankel1(n, k)) * eval_legendre(n, c)
    return (1j / k) * u


def scattered_field(x, k: float, d=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Exact scattered field of the sound-soft unit sphere at exterior points |x| > 1 for
    incidence e^{i k d.x}: u^s(x) = -sum_n i^n (2n+1) (j_n(k) / h_n(k)) h_n(k|x|) P_n(xhat.d),
    the outgoing expansion whose boundary values cancel the plane wave's on |x| = 1."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    r = np.linalg.norm(x, axis=1)
    c = (x / r[:, None]) @ np.asarray(d, dtype=np.float64)
    u = np.zeros(x.shape[0], dtype=np.complex128)
    for n in range(_nmax(k) + 1):
        u -= (1j ** n) * (2 * n + 1) * (spherical_jn(n, k) / hankel1(n, k)) * hankel1(n, k * r) * eval_legendre(n, c)
    return u


def far_field_quadrature(points, normals, weights, phi, k: float, eta: float, xhat) -> np.ndarray:
    """Eq. FarField evaluated with the surface quadrature:
    u_inf(xhat) = (1/4pi) sum_m [-i k (xhat.nu_m) - i eta] exp(-i k xhat.y_m) phi_m w_m."""
    y = np.asarray(points)
    nu = np.asarray(normals)
    xh = np.asarray(xhat)
    ph = np.exp(-1j * k * (xh @ y.T))
    kern = (-1j * k * (xh @ nu.T) - 1j * eta) * ph
    return kern @ (np.asarray(phi) * np.asarray(weights)) / (4 * math.pi)


def sphere_grid(Nphi: int, Ntheta: int) -> np.ndarray:
    """Uniform direction grid of Eq. SphereGrid (polar angle in [0, pi], azimuth in [0, 2 pi])."""
    pol = np.linspace(0.0, math.pi, Nphi)
    az = np.linspace(0.0, 2 * math.pi, Ntheta)
    P, A = np.meshgrid(pol, az, indexing="ij")
    return np.stack([np.sin(P) * np.cos(A), np.sin(P) * np.sin(A), np.cos(P)], -1).reshape(-1, 3)


def far_field_error(u_exact, u_approx) -> float:
    """Eq. FarFieldRelErr: max relative error of the far-field modulus."""
    return float(np.max(np.abs(np.abs(u_exact) - np.abs(u_approx)) / np.abs(u_exact)))


def real_ylm(l: int, m: int, points) -> np.ndarray:
    """Real spherical harmonic (unnormalised orthogonal basis) evaluated at directions of points."""
    from scipy.special import lpmv

    x = np.asarray(points)
    xh = x / np.linalg.norm(x, axis=1, keepdims=True)
    th = np.arccos(np.clip(xh[:, 2], -1, 1))
    ph = np.arctan2(xh[:, 1], xh[:, 0])
    P = lpmv(abs(m), l, np.cos(th))
    if m > 0:
        return P * np.cos(m * ph)
    if m < 0:
        return P * np.sin(-m * ph)
    return P
