"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a finite
difference, a symmetry, a textbook integral, a brute-force loop over the
oracle's single-pair kernel, polynomial exactness, the paper's printed level
counts, or convergence of the IFGF approximation to the direct sum.
"""
import json
import math
import os

import numpy as np
import pytest

from workloads import cube_sphere, fejer_nodes, fejer_weights, random_density, sphere_workload

HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# ---------------------------------------------------------------- quadrature inputs (Section 4)
def test_fejer_exactness():
    """Fejer's first rule (Eq. FejersWeights) integrates x^j exactly for j < J."""
    for J in (5, 8, 26):
        x, w = fejer_nodes(J), fejer_weights(J)
        assert abs(w.sum() - 2.0) < 1e-14
        for j in range(J):
            exact = 0.0 if j % 2 else 2.0 / (j + 1)
            assert abs((w * x ** j).sum() - exact) < 1e-13


def test_sphere_area_weights():
    """Equiangular cube-sphere area weights sum to 4 pi (unit sphere)."""
    for n, m in ((26, 26), (64, 8)):
        s = cube_sphere(n, m)
        assert abs(s.weights.sum() - 4 * math.pi) < 1e-12
        assert np.allclose(np.linalg.norm(s.points, axis=1), 1.0, atol=1e-15)


# ---------------------------------------------------------------- kernel (Eq. GreenFunction, Eq. double_layer)
def test_kernel_reciprocity_and_normal_derivative(oracle_lib):
    rng = np.random.default_rng(7)
    for _ in range(20):
        k = rng.uniform(0.5, 30)
        x, y = rng.normal(size=3), rng.normal(size=3)
        nu = rng.normal(size=3)
        nu /= np.linalg.norm(nu)
        phi_xy, dphi = oracle_lib.layer_kernels(k, x, y, nu)
        phi_yx, _ = oracle_lib.layer_kernels(k, y, x, nu)
        assert abs(phi_xy - phi_yx) <= 1e-14 * abs(phi_xy)
        # d/dnu(y) by a central difference of Phi along nu at y
        h = 1e-5
        fp, _ = oracle_lib.layer_kernels(k, x, y + h * nu, nu)
        fm, _ = oracle_lib.layer_kernels(k, x, y - h * nu, nu)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - dphi) <= 1e-7 * max(1.0, abs(dphi))
        # combined kernel = dPhi/dnu - i eta Phi
        eta = rng.uniform(0, 40)
        K = oracle_lib.kernel(k, eta, x, y, nu)
        assert abs(K - (dphi - 1j * eta * phi_xy)) <= 1e-13 * abs(K)


def test_gauss_and_shell_potential_static_limit(oracle_lib):
    """k -> 0 on the unit sphere: the double layer of 1 is -1/2 (Gauss) and the single
    layer of 1 is 1 (uniform shell); the plain quadrature without singular correction
    is only O(h) accurate, so the bound is loose.  Pins sign and 4 pi normalisation."""
    s = cube_sphere(26)
    one = np.ones((1, s.N), complex)
    ydl = oracle_lib.direct(s.points, s.normals, s.weights, 1e-9, 0.0, one)
    assert abs(np.median(ydl.real) + 0.5) < 2e-2
    ysl = oracle_lib.direct(s.points, s.normals, s.weights, 1e-9, 1.0, one)  # -i * S[1]
    assert abs(np.median(-ysl.imag) - 1.0) < 5e-2


def test_direct_sum_brute_force(oracle_lib):
    """Assembly of Eq. field1 (m != l, weights, identity term, multiple rhs, row subset)
    against a Python loop over the single-pair kernel."""
    rng = np.random.default_rng(3)
    N, k, eta, cI = 37, 4.0, 2.5, 0.5
    x = rng.normal(size=(N, 3))
    nu = rng.normal(size=(N, 3))
    nu /= np.linalg.norm(nu, axis=1, keepdims=True)
    w = rng.uniform(0.1, 1.0, N)
    sig = random_density(N, 2, 11)
    ref = np.zeros((2, N), complex)
    for l in range(N):
        for m in range(N):
            if m != l:
                ref[:, l] += oracle_lib.kernel(k, eta, x[l], x[m], nu[m]) * w[m] * sig[:, m]
    ref += cI * sig
    got = oracle_lib.direct(x, nu, w, k, eta, sig, cI=cI)
    assert rel(got, ref) < 1e-14
    rows = np.array([5, 0, 36, 17])
    assert rel(oracle_lib.direct(x, nu, w, k, eta, sig, cI=cI, rows=rows), ref[:, rows]) < 1e-14
    # conjugate transpose: <A s, g> = <s, A^H g>
    g = random_density(N, 2, 12)
    lhs = np.vdot(g, got)
    rhs = np.vdot(oracle_lib.direct_adjoint(x, nu, w, k, eta, g, cI=cI), sig)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # the single and double layers alone (layers 2 and 1) against the loop over Phi and dPhi/dnu
    for layer in (1, 2):
        ref = cI * sig.copy()
        for l in range(N):
            for m in range(N):
                if m != l:
                    phi, dphi = oracle_lib.layer_kernels(k, x[l], x[m], nu[m])
                    ref[:, l] += (dphi if layer == 1 else phi) * w[m] * sig[:, m]
        got = oracle_lib.direct(x, nu, w, k, eta, sig, cI=cI, layer=layer)
        assert rel(got, ref) < 1e-14, layer
        lhs = np.vdot(g, got)
        rhs = np.vdot(oracle_lib.direct_adjoint(x, nu, w, k, eta, g, cI=cI, layer=layer), sig)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# ---------------------------------------------------------------- Chebyshev (Eq. ChebyPoly, ChebyNodes)
def test_chebyshev_exact_for_low_degree(oracle_lib):
    rng = np.random.default_rng(5)
    for n in (3, 5, 7, 9):
        xk = np.cos((2 * np.arange(n) + 1) * np.pi / (2 * n))
        for deg in range(n):
            c = rng.normal(size=deg + 1)
            vals = np.polyval(c, xk)
            for t in rng.uniform(-1, 1, 5):
                assert abs(oracle_lib.cheb_interp_1d(vals, t) - np.polyval(c, t)) < 1e-12
        # degree n is not reproduced (the interpolant has degree n-1)
        vals = xk ** n
        errs = [abs(oracle_lib.cheb_interp_1d(vals, t) - t ** n) for t in (0.3, 0.77)]
        assert max(errs) > 1e-6


# ---------------------------------------------------------------- factorisation (Eq. hgn2, double_layer_fact, w23)
def test_factorisation_identity(oracle_lib):
    """E(x; y0) * W(x, y; y0) reproduces K(x, y) for both factor modes; the
    cancellation-free phase equals the literal phase."""
    rng = np.random.default_rng(9)
    for _ in range(30):
        k, eta, H = rng.uniform(1, 60), rng.uniform(0, 60), rng.uniform(0.05, 2)
        y0 = rng.normal(size=3)
        h = math.sqrt(3) / 2 * H
        y = y0 + rng.uniform(-H / 2, H / 2, 3)
        nu = rng.normal(size=3)
        nu /= np.linalg.norm(nu)
        d = rng.normal(size=3)
        x = y0 + d / np.linalg.norm(d) * rng.uniform(1.5 * H, 40 * H)
        r = np.linalg.norm(x - y0)
        E1 = np.exp(1j * k * r) / (4 * math.pi * r)
        E2 = E1 / r
        K = oracle_lib.kernel(k, eta, x, y, nu)
        (Wc,) = oracle_lib.wfactors(k, eta, x, y0, h, y, nu, split=False)
        W2, W13 = oracle_lib.wfactors(k, eta, x, y0, h, y, nu, split=True)
        assert abs(E1 * Wc - K) < 1e-11 * abs(K)
        assert abs(E2 * W2 + E1 * W13 - K) < 1e-11 * abs(K)
        (Wl,) = oracle_lib.wfactors(k, eta, x, y0, h, y, nu, split=False, literal=True)
        assert abs(Wl - Wc) < 1e-8 * abs(Wc)


# ---------------------------------------------------------------- IFGF oracle (Algorithm 1)
@pytest.fixture(scope="module")
def sphere1():
    s = cube_sphere(26)
    k = math.pi
    sig = random_density(s.N, 1, 1)
    return s, k, sig


def test_ifgf_oracle_counts_config1(oracle_lib, sphere1):
    s, k, sig = sphere1
    _, info = oracle_lib.ifgf(s.points, s.normals, s.weights, oracle_lib.IFGFParams(k=k, levels=3), sig)
    assert info["nbox"][3] == 56
    assert info["nrc"][3] == 344
    assert info["cousin_evals"][3] == 184224
    assert info["leaf_evals"] == 1819800


def test_ifgf_oracle_converges_to_direct(oracle_lib, sphere1):
    s, k, sig = sphere1
    yd = oracle_lib.direct(s.points, s.normals, s.weights, k, k, sig, cI=0.5)
    errs = []
    for ps, pa in ((3, 5), (5, 7), (7, 9), (9, 11)):
        p = oracle_lib.IFGFParams(k=k, levels=3, Ps=ps, Pang=pa, identity_coef=0.5)
        yi, _ = oracle_lib.ifgf(s.points, s.normals, s.weights, p, sig)
        errs.append(rel(yi, yd))
    assert errs[0] < 3e-3
    assert all(errs[i + 1] < 0.3 * errs[i] for i in range(3)), errs
    assert errs[-1] < 2e-6


def test_ifgf_oracle_multilevel_all_modes(oracle_lib):
    """4-wavelength sphere (N = 13,824, D = 4 as in Table 1): two levels of recursion,
    propagation through split and combined factors; all modes converge to the direct sum."""
    s, k = sphere_workload(48, 6, 4.0)
    sig = random_density(s.N, 2, 4)
    rows = np.random.default_rng(0).choice(s.N, 600, replace=False)
    yd = oracle_lib.direct(s.points, s.normals, s.weights, k, k, sig, rows=rows)
    for fm in (0, 1, 2):
        e = []
        for ps, pa in ((3, 5), (6, 8)):
            p = oracle_lib.IFGFParams(k=k, levels=4, Ps=ps, Pang=pa, factor_mode=fm)
            yi, info = oracle_lib.ifgf(s.points, s.normals, s.weights, p, sig)
            e.append(rel(yi[:, rows], yd))
        assert e[0] < 5e-3 and e[1] < 1e-4, (fm, e)
    assert info["nrc"][3] > 0 and info["prop_evals"][3] > 0


def test_ifgf_oracle_levels_match_table1(oracle_lib):
    """Automatic level count reproduces Table 1's levels for the sphere sizes there."""
    rows = json.load(open(os.path.join(HERE, "golden", "paper_table1_spheres.json")))["rows"]
    for r in rows[:3]:
        n = int(round(math.sqrt(r["N"] / 6)))
        s, k = sphere_workload(n, 8 if n % 8 == 0 else 6, float(r["diameter_wavelengths"]))
        assert s.N == r["N"]
        assert oracle_lib.auto_levels(s.points) == r["levels"], r


def _fig3_errors(oracle_lib, HL, eta, Ps=3, npts=100):
    """Section 3.3 / Fig. 3 set-up: interpolate the analytic factors along one ray x = y0 + (h/s) u
    over the cone segment closest to the source box (s in [eta0 - eta0/n_s, eta0], n_s of the
    size rule), Ps first-kind Chebyshev points; max error of the reconstructed kernel over
    the segment, relative to max |K|, for the combined factor and for the split pair."""
    k = 2 * math.pi
    H = HL * 1.0
    h = math.sqrt(3) / 2 * H
    y0 = np.zeros(3)
    y = np.array([0.4, -0.3, 0.45]) * H
    u = np.array([1.0, 0.7, 0.4]) / np.linalg.norm([1.0, 0.7, 0.4])
    nu = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    ns = 2 ** max(0, math.ceil(math.log2(2 * H)))
    e0 = math.sqrt(3) / 3
    a, b = e0 - e0 / ns, e0
    nodes = a + (np.cos((2 * np.arange(Ps) + 1) * math.pi / (2 * Ps)) + 1) / 2 * (b - a)
    vc = np.array([oracle_lib.wfactors(k, eta, y0 + h / s * u, y0, h, y, nu, split=False)[0] for s in nodes])
    vs = np.array([oracle_lib.wfactors(k, eta, y0 + h / s * u, y0, h, y, nu, split=True) for s in nodes])

    def interp(v, t):
        return oracle_lib.cheb_interp_1d(v.real, t) + 1j * oracle_lib.cheb_interp_1d(v.imag, t)

    ec, es, kk = [], [], []
    for s in np.linspace(a, b, npts + 1)[1:]:
        t = 2 * (s - a) / (b - a) - 1
        x = y0 + h / s * u
        r = h / s
        E1 = np.exp(1j * k * r) / (4 * math.pi * r)
        K = oracle_lib.kernel(k, eta, x, y, nu)
        ec.append(abs(E1 * interp(vc, t) - K))
        es.append(abs(E1 / r * interp(vs[:, 0], t) + E1 * interp(vs[:, 1], t) - K))
        kk.append(abs(K))
    return max(ec) / max(kk), max(es) / max(kk)


@pytest.mark.parametrize("eta", [0.0, 2 * math.pi])
def test_fig3_factor_interpolation_level_independent(oracle_lib, eta):
    """For H >= lambda the combined factor and the split pair interpolate equally well (Fig. 3
    text), and with the segment size halved as H doubles (Remark cone_seg_size) the error
    stays bounded as the box grows 8-fold; a factor carrying the unfactored oscillation
    e^{ik|x - y|} would fail both."""
    errs = [_fig3_errors(oracle_lib, HL, eta) for HL in (1.0, 2.0, 4.0, 8.0)]
    for c, s in errs:
        assert 0.9 < c / s < 1.25, errs
        assert c < 1e-2, errs
    assert max(c for c, _ in errs[1:]) < 4 * min(c for c, _ in errs[1:]), errs


def test_ifgf_oracle_reaches_direct_sum_to_rounding(oracle_lib):
    """With fine cone segments and high orders the interpolation error vanishes and
    Algorithm 1 reproduces the direct sum to rounding: one level (cousin interpolation
    only) to 1e-13, two levels (propagation through split and combined factors) to 2e-8."""
    k = math.pi
    s = cube_sphere(12, 12)  # N = 864
    sig = random_density(s.N, 1, 3)
    yd = oracle_lib.direct(s.points, s.normals, s.weights, k, k, sig, cI=0.5)
    for (ps, pa, nc0, ns0), bar in (((7, 9, 4, 2), 1e-8), ((11, 12, 8, 4), 1e-13)):
        p = oracle_lib.IFGFParams(k=k, levels=3, Ps=ps, Pang=pa, nC0=nc0, nS0=ns0, identity_coef=0.5)
        y, _ = oracle_lib.ifgf(s.points, s.normals, s.weights, p, sig)
        assert rel(y, yd) < bar, (ps, pa, rel(y, yd))
    s = cube_sphere(24, 12)  # N = 3,456, D = 4
    sig = random_density(s.N, 1, 3)
    yd = oracle_lib.direct(s.points, s.normals, s.weights, k, k, sig, cI=0.5)
    for fm in (0, 1, 2):
        p = oracle_lib.IFGFParams(k=k, levels=4, Ps=7, Pang=9, nC0=4, nS0=2, identity_coef=0.5, factor_mode=fm)
        y, info = oracle_lib.ifgf(s.points, s.normals, s.weights, p, sig)
        assert info["prop_evals"][3] > 0
        assert rel(y, yd) < 2e-8, (fm, rel(y, yd))


# ---------------------------------------------------------------- cone grid per level (Remark cone_seg_size)
def _cone_grid(oracle_lib, s, k, levels, cone_rule=0):
    sig = random_density(s.N, 1, 5)
    _, info = oracle_lib.ifgf(s.points, s.normals, s.weights,
                              oracle_lib.IFGFParams(k=k, levels=levels, cone_rule=cone_rule), sig)
    assert info["D"] == levels
    return {d: (info["ns"][d], info["nC"][d]) for d in range(3, levels + 1)}, info


def test_cone_grid_size_rule_16_wavelength_sphere(oracle_lib):
    """Per-level (n_s, n_C) under the size rule (reading of Remark cone_seg_size and the
    Fig. 3 text: constant segments while H <= lambda/2, then n_s and n_C double each time the
    box side doubles), derived by hand for the 16-wavelength unit sphere (k = 16 pi, so
    lambda = 1/8) with six levels.  The root box side is the point cloud's largest extent, a
    hair under 2, so H_d = L / 2^(d-1) gives H_d / lambda just under 4, 2, 1, 1/2 for d = 3..6:
    the leaf (d = 6) keeps (n_S0, n_C0) = (1, 2) and every coarser level doubles both:
    (2, 4), (4, 8), (8, 16).  With k 1% larger every H_d / lambda moves just above those
    powers of two, so every level gets one more doubling: (2, 4) at the leaf up to (16, 32).
    A doubling that fires one level early or late, or an exponent rounded down instead of up
    (floor instead of ceiling of log2(2 H_d / lambda)), fails one of the two cases."""
    s = cube_sphere(32, 8)  # N = 6,144; the cone grid depends on H_d and k only
    grid, info = _cone_grid(oracle_lib, s, 16 * math.pi, 6)
    assert 1.99 < info["root_side"] < 2.0
    assert grid == {3: (8, 16), 4: (4, 8), 5: (2, 4), 6: (1, 2)}, grid
    grid, _ = _cone_grid(oracle_lib, s, 16 * math.pi * 1.01, 6)
    assert grid == {3: (16, 32), 4: (8, 16), 5: (4, 8), 6: (2, 4)}, grid


def test_cone_grid_literal_rule(oracle_lib):
    """cone_rule = 1, the remark read literally: the leaf level D keeps (n_S0, n_C0) = (1, 2)
    and n_s, n_C double on the way from level d to d - 1 exactly when k H_d > 1/2.  Unit
    sphere, root side L = 1.9955 (the Fejer nodes stop short of the poles), five levels:
    H_5 = L/16 = 0.1247, H_4 = L/8 = 0.2494.
    * k = pi:     k H_5 = 0.392 (no doubling into level 4), k H_4 = 0.784 (doubling into 3)
                  -> levels 5, 4, 3 = (1, 2), (1, 2), (2, 4);
    * k = 1.5 pi: k H_5 = 0.588, k H_4 = 1.175 -> (1, 2), (2, 4), (4, 8).
    The size rule gives (1, 2) at every level for k = pi (lambda = 2: all H_d <= lambda/2),
    so the two rules are told apart; at the 16-wavelength sphere (k H_6 = 3.1 > 1/2 at every
    level) the literal rule coincides with the size rule above."""
    s = cube_sphere(26)  # N = 4,056
    grid, info = _cone_grid(oracle_lib, s, math.pi, 5, cone_rule=1)
    assert abs(info["root_side"] - 1.9955) < 1e-4
    assert grid == {3: (2, 4), 4: (1, 2), 5: (1, 2)}, grid
    grid, _ = _cone_grid(oracle_lib, s, 1.5 * math.pi, 5, cone_rule=1)
    assert grid == {3: (4, 8), 4: (2, 4), 5: (1, 2)}, grid
    grid, _ = _cone_grid(oracle_lib, s, math.pi, 5, cone_rule=0)
    assert grid == {3: (1, 2), 4: (1, 2), 5: (1, 2)}, grid
    grid, _ = _cone_grid(oracle_lib, cube_sphere(32, 8), 16 * math.pi, 6, cone_rule=1)
    assert grid == {3: (8, 16), 4: (4, 8), 5: (2, 4), 6: (1, 2)}, grid


def test_relevant_cones_per_level_roughly_constant(oracle_lib):
    """Section 3.5: with the cone refinement of Remark cone_seg_size the number of relevant
    cone segments per level stays roughly constant while the number of boxes grows about
    fourfold per level on a surface.  8-wavelength sphere (N = 55,296, automatic depth 5 as in
    Table 1): boxes grow ~20x from level 3 to 5, relevant cones stay within a factor 2.5.  One
    missing or extra doubling at any level would move that level's count by ~8x."""
    s, k = sphere_workload(96, 8, 8.0)
    sig = random_density(s.N, 1, 5)
    _, info = oracle_lib.ifgf(s.points, s.normals, s.weights, oracle_lib.IFGFParams(k=k), sig)
    assert info["D"] == 5
    nb = [info["nbox"][d] for d in (3, 4, 5)]
    nrc = [info["nrc"][d] for d in (3, 4, 5)]
    assert nb[2] / nb[0] > 15, nb
    assert max(nrc) / min(nrc) < 2.5, nrc


# ---------------------------------------------------------------- IFGF far field (Eq. FarField, Section 3.4)
@pytest.mark.parametrize("fm", [0, 1])
def test_ifgf_far_field_mie(oracle_lib, fm):
    """The far-field pattern taken from the level-3 interpolants at s = 0, for the exact Mie
    density of a sound-soft unit sphere (k = pi), against the closed-form far field.  With
    factor_mode 0 level 3 stores the split pair (its W13 member is the one that survives the
    limit); factor_mode 1 the combined factor.  The error falls with the interpolation orders
    to the size of the IFGF error of an apply."""
    from oracle import mie

    s = cube_sphere(24, 6)
    k = math.pi
    phi = mie.density(s.points, k, k)
    xh = mie.sphere_grid(11, 11)
    ue = mie.far_field(xh, k)
    errs = {}
    for ps, pa, lev in ((3, 5, 3), (5, 8, 3), (5, 8, 4)):
        out, info = oracle_lib.ifgf_far_field(
            s.points, s.normals, s.weights,
            oracle_lib.IFGFParams(k=k, Ps=ps, Pang=pa, levels=lev, factor_mode=fm), phi, xh)
        assert info["split"][3] == (1 if fm == 0 else 0)
        errs[(ps, pa, lev)] = rel(out[0], ue)
    assert errs[(3, 5, 3)] < 1e-3
    assert errs[(5, 8, 3)] < 1e-5 and errs[(5, 8, 4)] < 3e-5  # combined factor at H < lambda/2: less accurate
    assert errs[(5, 8, 3)] < errs[(3, 5, 3)] / 30


def test_ifgf_far_field_converges_to_sum(oracle_lib):
    """A 3-wavelength sphere with random densities (two right-hand sides), D = 4: the IFGF far
    field approaches the plain quadrature sum of Eq. FarField as the orders grow, for every
    direction (max-modulus error), with the combined factor at level 3."""
    s, k = sphere_workload(24, 6, 3.0)
    sig = random_density(s.N, 2, 31)
    rng = np.random.default_rng(32)
    xh = rng.normal(size=(60, 3))
    xh /= np.linalg.norm(xh, axis=1)[:, None]
    ref = oracle_lib.far_field(s.points, s.normals, s.weights, k, k, sig, xh)
    e = []
    for ps, pa in ((3, 5), (5, 7), (6, 8)):
        out, info = oracle_lib.ifgf_far_field(s.points, s.normals, s.weights,
                                              oracle_lib.IFGFParams(k=k, Ps=ps, Pang=pa, levels=4), sig, xh)
        assert info["split"][3] == 0 and info["D"] == 4
        e.append(float(np.abs(out - ref).max() / np.abs(ref).max()))
    assert e[0] < 5e-3 and e[2] < 1e-4
    assert e[0] > e[1] > e[2]


@pytest.mark.parametrize("layer", [1, 2])
def test_ifgf_oracle_layers_converge_to_direct(oracle_lib, layer):
    """The IFGF apply with the double layer alone (1) or the single layer alone (2): 3-wavelength
    sphere, D = 4, split factors below lambda/2 and the combined factor above (the single layer's
    q = 2 factor is zero); the error against the direct sum of that layer falls with the orders."""
    s, k = sphere_workload(24, 6, 3.0)
    sig = random_density(s.N, 1, 33)
    ref = oracle_lib.direct(s.points, s.normals, s.weights, k, k, sig, cI=0.5, layer=layer)
    e = []
    for ps, pa in ((3, 5), (5, 8)):
        y, info = oracle_lib.ifgf(s.points, s.normals, s.weights,
                                  oracle_lib.IFGFParams(k=k, Ps=ps, Pang=pa, levels=4, identity_coef=0.5,
                                                        layer=layer), sig)
        assert info["split"][4] == 1 and info["split"][3] == 0
        e.append(rel(y, ref))
    assert e[0] < 5e-3 and e[1] < 1e-4 and e[1] < e[0] / 10


# ---------------------------------------------------------------- adaptive octree (leaves at several levels)
def _two_spheres():
    """A unit sphere (1,536 points) and a sphere of radius 0.15 centred at (1.6, 0, 0) with 3,456
    points: a point density 20x higher in one corner of the root box."""
    from workloads import two_spheres

    s = two_spheres()
    return s.points, s.normals, s.weights


def test_adaptive_tree_reduces_to_uniform(oracle_lib):
    """With a leaf budget above every box's point count every level-3 box is a leaf, and the
    adaptive apply is the uniform three-level apply (up to rounding order in the near field)."""
    pts, nrm, w = _two_spheres()
    k = 2 * math.pi
    sig = random_density(pts.shape[0], 2, 41)
    P = lambda **kw: oracle_lib.IFGFParams(k=k, identity_coef=0.5, **kw)
    y3, _ = oracle_lib.ifgf(pts, nrm, w, P(levels=3), sig)
    ya, _ = oracle_lib.ifgf(pts, nrm, w, P(levels=6, leaf_max=10 ** 9), sig)
    assert rel(ya, y3) < 1e-13


def test_adaptive_tree_converges_to_direct(oracle_lib):
    """Adaptive tree on the two-sphere set (levels up to 6, leaves of at most 64 points): the error
    against the direct sum falls with the orders to 3e-8 (every pair enters exactly once: through
    one cousin interpolation or through the near field at the coarser of the two leaf levels), and
    the relevant cone segments are a fraction of the uniform tree's."""
    pts, nrm, w = _two_spheres()
    k = 2 * math.pi
    sig = random_density(pts.shape[0], 1, 42)
    ref = oracle_lib.direct(pts, nrm, w, k, k, sig, cI=0.5)
    P = lambda **kw: oracle_lib.IFGFParams(k=k, identity_coef=0.5, levels=6, **kw)
    e = []
    for kw in (dict(Ps=3, Pang=5), dict(Ps=5, Pang=8), dict(Ps=6, Pang=8, nC0=4, nS0=2)):
        y, info = oracle_lib.ifgf(pts, nrm, w, P(leaf_max=64, **kw), sig)
        e.append(rel(y, ref))
    assert e[0] < 1e-3 and e[1] < 1e-5 and e[2] < 1e-7, e
    _, iu = oracle_lib.ifgf(pts, nrm, w, P(Ps=5, Pang=8), sig)
    _, ia = oracle_lib.ifgf(pts, nrm, w, P(Ps=5, Pang=8, leaf_max=64), sig)
    assert sum(ia["nrc"]) < sum(iu["nrc"]) / 5


def test_adaptive_near_pairs_brute_force(oracle_lib):
    """The adaptive near field visits exactly the pairs of the rule it implements: a point's leaf is its
    first box from level 3 down holding at most leaf_max points (level D at the latest), and two points
    interact directly when their boxes at the coarser of their two leaf levels are neighbours.  Counted
    here by brute force over all pairs of a small two-density cloud from the root box the oracle reports;
    a pair missing or counted twice changes the count."""
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.normal(size=(450, 3)) * 0.04 + 0.3, rng.uniform(-1, 1, (250, 3))])
    nrm = rng.normal(size=x.shape)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    w = rng.uniform(0.5, 1.5, x.shape[0])
    D, lm = 6, 12
    _, info = oracle_lib.ifgf(x, nrm, w, oracle_lib.IFGFParams(k=3.0, levels=D, leaf_max=lm), random_density(len(x), 1, 6))
    lo = np.asarray(info["root_center"]) - info["root_side"] / 2
    cell = {d: np.clip(np.floor((x - lo) / (info["root_side"] / 2 ** (d - 1))).astype(np.int64), 0, 2 ** (d - 1) - 1)
            for d in range(3, D + 1)}
    lev = np.full(len(x), D)
    done = np.zeros(len(x), bool)
    for d in range(3, D):
        _, inv, cnt = np.unique(cell[d], axis=0, return_inverse=True, return_counts=True)
        m = ~done & (cnt[inv.ravel()] <= lm)
        lev[m] = d
        done |= m
    assert len(set(lev.tolist())) >= 3  # leaves at several levels
    mlev = np.minimum(lev[:, None], lev[None, :])
    near = np.zeros((len(x), len(x)), bool)
    for d in range(3, D + 1):
        dd = np.abs(cell[d][:, None, :] - cell[d][None, :, :]).max(axis=2) <= 1
        near |= (mlev == d) & dd
    np.fill_diagonal(near, False)
    assert info["near_pairs"] == int(near.sum())
