"""The library's rectangular-polar correction (``ifgf_rp_correction``, host only) against the
oracle's and against facts of the continuous operators:

* cube-sphere: the same sparsity as the oracle's RP correction (which uses the exact sphere
  map; the library interpolates each patch from its nodes), the products C phi agree, and
  the corrected discrete operator reproduces the sphere's eigen-relations
  A Y_n = lambda_n Y_n as closely as the oracle's does;
* ellipsoid (no closed form): Gauss's law for the double layer, (1/2 + D)[1] = 0 on a closed
  surface in the static limit, holds to 3e-5 with the correction and only to 1e-2 without;
* argument validation.
"""
import math

import numpy as np
import pytest

from oracle import mie
from workloads import cube_sphere, ellipsoid, patch_node_index, random_density


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def B():
    from paper_2112_06316_gb300 import binding
    from paper_2112_06316_gb300 import build as _b

    _b.build()
    return binding


def test_rp_matches_oracle_and_eigen_relations(B, oracle_lib):
    n, m, k = 32, 8, 2 * math.pi
    s = cube_sphere(n, m)
    delta = math.pi / (2 * (n // m))  # one nominal sub-patch side, the oracle's default
    ro, co, vo = oracle_lib.rp_correction_sphere(s.points, s.normals, s.weights, n, m, 1.0, k, k,
                                                 delta=delta, Nbeta=48, dgrade=5.0)
    rl, cl, vl = B.rp_correction(s.points, s.normals, s.weights, patch_node_index(s), m, k, k, delta=delta,
                                 n_beta=48, d_grade=5.0)
    assert np.array_equal(np.diff(rl), np.diff(ro))
    sig = random_density(s.N, 2, 1)
    assert rel(oracle_lib.csr_apply(rl, cl, vl, sig), oracle_lib.csr_apply(ro, co, vo, sig)) < 3e-5
    for l, mm in ((0, 0), (2, 1), (5, -3), (9, 4)):
        Y = mie.real_ylm(l, mm, s.points)[None, :].astype(complex)
        lam = mie.eigenvalue(l, k, k)
        y0 = oracle_lib.direct(s.points, s.normals, s.weights, k, k, Y, cI=0.5)
        el = rel(y0 + oracle_lib.csr_apply(rl, cl, vl, Y), lam * Y)
        eo = rel(y0 + oracle_lib.csr_apply(ro, co, vo, Y), lam * Y)
        assert el < 3e-5 and el < 1.05 * eo + 1e-7, (l, mm, el, eo)


def test_rp_gauss_law_on_an_ellipsoid(B, oracle_lib):
    s = ellipsoid(32, 8, (1.0, 1.5, 2.0))
    k = 1e-8  # static limit
    delta = 1.5 * math.pi / 8
    rl, cl, vl = B.rp_correction(s.points, s.normals, s.weights, patch_node_index(s), 8, k, 0.0, delta=delta)
    one = np.ones((1, s.N), dtype=complex)
    y0 = oracle_lib.direct(s.points, s.normals, s.weights, k, 0.0, one, cI=0.5)
    y = y0 + oracle_lib.csr_apply(rl, cl, vl, one)
    assert np.abs(y0).max() > 1e-2
    assert np.abs(y).max() < 3e-5 and np.sqrt(np.mean(np.abs(y) ** 2)) < 5e-6


def test_rp_validation(B):
    s = cube_sphere(8, 8)
    pn = patch_node_index(s)
    args = (s.points, s.normals, s.weights)
    with pytest.raises(B.IFGFError, match="permutation"):
        bad = pn.copy()
        bad[1] = bad[0]
        B.rp_correction(*args, bad, 8, 1.0, delta=0.3)
    with pytest.raises(B.IFGFError, match="multiple of m"):
        B.rp_correction(*args, pn, 7, 1.0, delta=0.3)
    with pytest.raises(B.IFGFError, match="EINVAL"):
        B.rp_correction(*args, pn, 8, -1.0, delta=0.3)
    with pytest.raises(B.IFGFError, match="EINVAL"):
        B.rp_correction(*args, pn, 8, 1.0, delta=0.3, n_beta=1)
    rp, col, val = B.rp_correction(*args, pn, 8, 1.0, delta=0.0)  # own patches only
    assert rp[-1] == s.N * 64 and np.all(np.isfinite(val))


def test_single_layer_from_two_couplings(B, oracle_lib):
    """With c_I = 0 the corrected operator is D - i eta S, so S = i (A_{eta=1} - A_{eta=0}); on the
    unit sphere that reproduces S[Y_n] = i k j_n(k) h_n(k) Y_n and D[Y_n] = (i k^2 j_n' h_n - 1/2) Y_n."""
    n, m, k = 32, 8, 2 * math.pi
    s = cube_sphere(n, m)
    pn = patch_node_index(s)
    delta = math.pi / (2 * (n // m))

    def A(eta, Y):
        rp, col, val = B.rp_correction(s.points, s.normals, s.weights, pn, m, k, eta, delta=delta)
        return oracle_lib.direct(s.points, s.normals, s.weights, k, eta, Y, cI=0.0) + oracle_lib.csr_apply(rp, col, val, Y)

    # (k = 2 pi is a zero of j_0, where S has the eigenvalue 0: start at degree 1)
    for l, mm in ((1, 1), (3, 2), (7, -4)):
        Y = mie.real_ylm(l, mm, s.points)[None, :].astype(complex)
        D = A(0.0, Y)
        S = 1j * (A(1.0, Y) - D)
        assert rel(S, mie.single_layer_eigenvalue(l, k) * Y) < 3e-5, l
        assert rel(D, mie.double_layer_eigenvalue(l, k) * Y) < 3e-5, l


def test_rp_quadrature_self_convergence(B, oracle_lib):
    """Doubling the RP quadrature points (Eq. BetaCov) shrinks the change of C phi by more
    than ten: 24 -> 48 -> 96 points per direction."""
    s = cube_sphere(16, 8)
    pn = patch_node_index(s)
    sig = random_density(s.N, 1, 2)
    out = {}
    for nb in (24, 48, 96):
        rp, col, val = B.rp_correction(s.points, s.normals, s.weights, pn, 8, 2 * math.pi, delta=math.pi / 4,
                                       n_beta=nb)
        out[nb] = oracle_lib.csr_apply(rp, col, val, sig)
    e24, e48 = rel(out[24], out[96]), rel(out[48], out[96])
    assert e48 < 0.1 * e24 and e48 < 1e-3, (e24, e48)
