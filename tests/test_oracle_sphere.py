"""Pins of the oracle's sphere closed forms and of the rectangular-polar correction.

* The Mie far field (closed form) equals Eq. FarField integrated over the exact
  Mie density with the surface quadrature (two independent routes).
* The corrected discrete operator (direct sum + RP correction, Section 4.2)
  reproduces the eigen-relations A Y_n = lambda_n Y_n of the unit sphere.
* The single- and double-layer sums alone (layers 2 and 1), with their shares of the
  correction, reproduce the eigenvalues of S and D on the unit sphere.
* The exact Mie density solves the corrected discrete CFIE to the same accuracy.
* The off-surface combined-layer potential of the exact Mie density matches the
  closed-form exterior field, and tends to the far-field pattern as |x| grows.
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


def test_single_and_double_layer_eigen_relations(oracle_lib, corrected_sphere):
    """The oracle's double-layer and single-layer direct sums (layers 1 and 2), each with its
    share of the rectangular-polar correction (C is linear in eta: C_D = C(0) and
    C_S = i (C(k) - C(0)) / k), reproduce the unit sphere's eigenvalues
    D[Y_n] = (i k^2 j_n' h_n - 1/2) Y_n and S[Y_n] = i k j_n h_n Y_n."""
    s, k, rp, col, val = corrected_sphere
    n, m = 32, 8
    rp0, col0, val0 = oracle_lib.rp_correction_sphere(s.points, s.normals, s.weights, n, m, 1.0, k, 0.0)
    for l, mm in ((1, 1), (3, 2), (7, -4)):  # (k = 2 pi is a zero of j_0: S has the eigenvalue 0 there)
        Y = mie.real_ylm(l, mm, s.points)[None, :].astype(complex)
        cD = oracle_lib.csr_apply(rp0, col0, val0, Y)
        cS = 1j * (oracle_lib.csr_apply(rp, col, val, Y) - cD) / k
        D = oracle_lib.direct(s.points, s.normals, s.weights, k, 0.0, Y, layer=1) + cD
        S = oracle_lib.direct(s.points, s.normals, s.weights, k, 0.0, Y, layer=2) + cS
        assert rel(D, mie.double_layer_eigenvalue(l, k) * Y) < 3e-5, l
        assert rel(S, mie.single_layer_eigenvalue(l, k) * Y) < 3e-5, l


def test_mie_density_solves_corrected_system(oracle_lib, corrected_sphere):
    s, k, rp, col, val = corrected_sphere
    phi = mie.density(s.points, k, k)[None, :]
    ui = np.exp(1j * k * s.points[:, 2])[None, :]
    r = corrected_apply(oracle_lib, s, k, rp, col, val, phi) + ui
    assert np.linalg.norm(r) / np.linalg.norm(ui) < 3e-5


# ---- off-surface field and far field (Eq. CombinedLayer, Eq. FarField) ----------------

def test_field_matches_exterior_mie_series(oracle_lib):
    """The combined-layer potential of the exact Mie density, summed with the surface
    quadrature at exterior points, equals the closed-form scattered field; the error is the
    quadrature's and shrinks with the distance from the surface and with refinement."""
    rng = np.random.default_rng(7)
    dirs = rng.normal(size=(40, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    s = cube_sphere(32, 8)
    for k, bars in ((math.pi, ((1.25, 5e-6), (1.5, 2e-7), (3.0, 2e-8))), (2 * math.pi, ((1.5, 5e-6), (3.0, 5e-6)))):
        phi = mie.density(s.points, k, k)
        for R, bar in bars:
            u = oracle_lib.field(s.points, s.normals, s.weights, k, k, phi, dirs * R)[0]
            assert rel(u, mie.scattered_field(dirs * R, k)) < bar, (k, R)
    coarse = cube_sphere(16, 8)
    phi = mie.density(coarse.points, math.pi, math.pi)
    u = oracle_lib.field(coarse.points, coarse.normals, coarse.weights, math.pi, math.pi, phi, dirs * 1.5)[0]
    assert rel(u, mie.scattered_field(dirs * 1.5, math.pi)) > 1e-6  # the coarse grid is visibly worse


def test_field_tends_to_far_field(oracle_lib):
    """u(R xhat) R e^{-ikR} -> u_inf(xhat) with an O(1/R) error, for the discrete sums and
    for the closed forms alike (fixes the far-field normalisation and the sign of its phase)."""
    from workloads import random_density

    rng = np.random.default_rng(8)
    dirs = rng.normal(size=(30, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    s = cube_sphere(16, 8)
    k = 2 * math.pi
    sig = random_density(s.N, 2, 5)
    uf = oracle_lib.far_field(s.points, s.normals, s.weights, k, k, sig, dirs)
    errs = []
    for R in (1e5, 1e6):
        u = oracle_lib.field(s.points, s.normals, s.weights, k, k, sig, dirs * R) * R * np.exp(-1j * k * R)
        errs.append(rel(u, uf))
        um = mie.scattered_field(dirs * R, k) * R * np.exp(-1j * k * R)
        assert rel(um, mie.far_field(dirs, k)) < 30.0 / R
    assert errs[1] < 1e-5
    assert 9.0 < errs[0] / errs[1] < 11.0


def test_field_brute_force_against_layer_kernels(oracle_lib):
    """Tiny case: the vectorised off-surface sum equals a loop over the C oracle's kernel
    (pinned separately by reciprocity and a finite-difference normal derivative); a target
    on a source point drops that pair."""
    rng = np.random.default_rng(9)
    N, M, k, eta = 23, 7, 3.7, 1.3
    x = rng.normal(size=(N, 3))
    nu = rng.normal(size=(N, 3))
    nu /= np.linalg.norm(nu, axis=1, keepdims=True)
    w = rng.uniform(0.1, 1.0, N)
    sig = rng.normal(size=(2, N)) + 1j * rng.normal(size=(2, N))
    t = rng.normal(size=(M, 3)) * 2.0
    t[3] = x[5]
    ref = np.zeros((2, M), dtype=complex)
    for j in range(M):
        for m in range(N):
            if j == 3 and m == 5:
                continue
            Phi, dPhi = oracle_lib.layer_kernels(k, t[j], x[m], nu[m])
            ref[:, j] += (dPhi - 1j * eta * Phi) * w[m] * sig[:, m]
    assert rel(oracle_lib.field(x, nu, w, k, eta, sig, t), ref) < 1e-13
    ff = oracle_lib.far_field(x, nu, w, k, eta, sig, t / np.linalg.norm(t, axis=1, keepdims=True))
    assert ff.shape == (2, M) and np.all(np.isfinite(ff))
