"""Pins of the oracle's sphere closed forms and of the rectangular-polar correction.

* The Mie far field (closed form) equals Eq. FarField integrated over the exact
  Mie density with the surface quadrature (two independent routes).
* The corrected discrete operator (direct sum + RP correction, Section 4.2)
  reproduces the eigen-relations A Y_n = lambda_n Y_n of the unit sphere.
* The exact Mie density solves the corrected discrete CFIE to the same accuracy.
"""
import math

import numpy as np
import pytest

from oracle import mie
from workloads import cube_sphere


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_mie_far_field_two_routes():
    s = cube_sphere(32, 8)
    for k in (math.pi, 4.0):
        eta = k
        phi = mie.density(s.points, k, eta)
        xh = mie.sphere_grid(21, 21)
        uq = mie.far_field_quadrature(s.points, s.normals, s.weights, phi, k, eta, xh)
        ue = mie.far_field(xh, k)
        assert rel(uq, ue) < 1e-7
        assert mie.far_field_error(ue, uq) < 1e-6


def test_mie_low_frequency_limit():
    """Static limit: for k -> 0 the far field of the sound-soft unit sphere tends to -1
    (the capacity of the unit sphere), independent of direction."""
    k = 1e-4
    u = mie.far_field(mie.sphere_grid(5, 5), k)
    assert np.allclose(u, -1.0, atol=2e-4)


@pytest.fixture(scope="module")
def corrected_sphere(oracle_lib):
    n, m, k = 32, 8, 2 * math.pi  # 2 wavelengths across, N = 6,144
    s = cube_sphere(n, m)
    rp, col, val = oracle_lib.rp_correction_sphere(s.points, s.normals, s.weights, n, m, 1.0, k, k)
    return s, k, rp, col, val


def corrected_apply(oracle_lib, s, k, rp, col, val, sig):
    y = oracle_lib.direct(s.points, s.normals, s.weights, k, k, sig, cI=0.5)
    return y + oracle_lib.csr_apply(rp, col, val, sig)


def test_rp_eigen_relations(oracle_lib, corrected_sphere):
    s, k, rp, col, val = corrected_sphere
    assert 500 < rp[-1] / s.N < 700  # own patch and its neighbours (8 x 8 nodes each)
    for l, m in ((0, 0), (1, 1), (2, -1), (4, 3), (7, 2), (10, -5)):
        Y = mie.real_ylm(l, m, s.points)[None, :].astype(complex)
        lam = mie.eigenvalue(l, k, k)
        y = corrected_apply(oracle_lib, s, k, rp, col, val, Y)
        assert rel(y, lam * Y) < 3e-5, (l, m)
        y0 = oracle_lib.direct(s.points, s.normals, s.weights, k, k, Y, cI=0.5)
        assert rel(y0, lam * Y) > 1e-2  # the uncorrected quadrature is far off


def test_mie_density_solves_corrected_system(oracle_lib, corrected_sphere):
    s, k, rp, col, val = corrected_sphere
    phi = mie.density(s.points, k, k)[None, :]
    ui = np.exp(1j * k * s.points[:, 2])[None, :]
    r = corrected_apply(oracle_lib, s, k, rp, col, val, phi) + ui
    assert np.linalg.norm(r) / np.linalg.norm(ui) < 3e-5
