"""GPU: sparse RP correction inside the apply, and GMRES (the solve of Eq. CombLayIE).

The correction matrix comes from the oracle (host precompute); the apply, the
correction product and GMRES run in the library.  Results are checked against
closed forms of the sound-soft unit sphere (eigen-relations, Mie density and far
field) and against the true residual of the returned iterate.
"""
import math

import numpy as np
import pytest

from oracle import mie
from workloads import cube_sphere, ellipsoid, random_density

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_06316_gb300 import binding
    from paper_2112_06316_gb300 import build as _b

    _b.build()
    return binding


@pytest.fixture(scope="module")
def sphere_plan(B, oracle_lib):
    n, m, k = 32, 8, 2 * math.pi  # unit sphere 2 wavelengths across, N = 6,144
    s = cube_sphere(n, m)
    rp, col, val = oracle_lib.rp_correction_sphere(s.points, s.normals, s.weights, n, m, 1.0, k, k)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, Ps=5, Pang=8))
    plan.set_correction(rp, col, val)
    return s, k, plan


def test_corrected_apply_eigen_relations(B, sphere_plan):
    s, k, plan = sphere_plan
    for l, m in ((0, 0), (2, 1), (5, -3), (9, 4)):
        Y = mie.real_ylm(l, m, s.points).astype(np.complex128)
        lam = mie.eigenvalue(l, k, k)
        y64 = plan.apply(torch.from_numpy(Y).cuda()).cpu().numpy()
        y32 = plan.apply(torch.from_numpy(Y.astype(np.complex64)).cuda()).cpu().numpy()
        assert rel(y64, lam * Y) < 1e-4, (l, m)
        assert rel(y32, lam * Y) < 1e-4, (l, m)
    assert plan.missed_lookups() == 0


@pytest.mark.parametrize("prec,tol", [(0, 1e-8), (1, 1e-5)])
def test_gmres_sphere_against_mie(B, sphere_plan, prec, tol):
    """Plane wave along z; Eq. CombLayIE with eta = k; compare the density with the Mie
    series and the far field on the (200 x 200) grid of Eq. SphereGrid."""
    s, k, plan = sphere_plan
    ui = np.exp(1j * k * s.points[:, 2])
    rhs = torch.from_numpy(-ui).cuda()
    x, ok, it, hist = plan.gmres(rhs, restart=40, maxit=200, tol=tol, precision=prec)
    assert ok, hist[-5:]
    assert it < 60
    assert np.all(np.diff(hist[1:]) <= 1e-12)  # GMRES residual estimates never increase
    phi = x.cpu().numpy()
    phi_ex = mie.density(s.points, k, k)
    assert rel(phi, phi_ex) < 1e-4
    xh = mie.sphere_grid(200, 200)
    uf = mie.far_field_quadrature(s.points, s.normals, s.weights, phi, k, k, xh)
    assert mie.far_field_error(mie.far_field(xh, k), uf) < 1e-4
    # true residual of the returned iterate
    r = plan.apply(x).cpu().numpy() + ui
    assert np.linalg.norm(r) / np.linalg.norm(ui) < (3 * tol if prec == 0 else 1e-4)


def test_gmres_restart_and_nonsphere(B):
    """Ellipsoid without correction (the bare quadrature operator is still a valid
    linear system): short restarts converge and the true residual matches tol."""
    e = ellipsoid(24, 8, (1.0, 1.5, 2.0))
    k = 5.0
    plan = B.Plan(e.points, e.normals, e.weights, B.Params(k=k))
    b = torch.from_numpy(random_density(e.N, 1, 3)[0]).cuda()
    x, ok, it, hist = plan.gmres(b, restart=8, maxit=400, tol=1e-9)
    assert ok
    r = plan.apply(x) - b
    assert (torch.linalg.norm(r) / torch.linalg.norm(b)).item() < 3e-9


def test_gmres_edge_cases(B):
    s = cube_sphere(8, 8)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=2.0))
    z = torch.zeros(s.N, dtype=torch.complex128, device="cuda")
    x, ok, it, hist = plan.gmres(z)
    assert ok and it == 0 and torch.count_nonzero(x).item() == 0
    b = torch.from_numpy(random_density(s.N, 1, 1)[0]).cuda()
    x, ok, it, hist = plan.gmres(b, maxit=0, tol=1e-8)
    assert not ok and it == 0
    with pytest.raises(B.IFGFError, match="EINVAL"):
        plan.gmres(b, restart=0)


def test_library_rp_correction_on_the_gpu_apply(B):
    """The product path end to end: the library's own host RP correction
    (ifgf_rp_correction) attached to a plan and applied on the GPU reproduces the sphere's
    eigen-relations like the oracle's correction does."""
    from workloads import patch_node_index

    n, m, k = 32, 8, 2 * math.pi
    s = cube_sphere(n, m)
    rp, col, val = B.rp_correction(s.points, s.normals, s.weights, patch_node_index(s), m, k, k,
                                   delta=math.pi / (2 * (n // m)))
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, Ps=5, Pang=8))
    plan.set_correction(rp, col, val)
    for l, mm in ((0, 0), (2, 1), (5, -3), (9, 4)):
        Y = mie.real_ylm(l, mm, s.points).astype(np.complex128)
        lam = mie.eigenvalue(l, k, k)
        assert rel(plan.apply(torch.from_numpy(Y).cuda()).cpu().numpy(), lam * Y) < 1e-4, (l, mm)
        assert rel(plan.apply(torch.from_numpy(Y.astype(np.complex64)).cuda()).cpu().numpy(), lam * Y) < 1e-4
    assert plan.missed_lookups() == 0
    plan.close()


@pytest.mark.parametrize("shape", ["sphere", "ellipsoid"])
def test_rp_correction_gpu_matches_host(B, shape):
    """ifgf_rp_correction_gpu (quadrature on the device) gives the host builder's correction:
    the same sparsity and entry order, values equal to FP64 rounding."""
    from parity import check
    from workloads import patch_node_index

    n, m = 32, 8
    s = cube_sphere(n, m) if shape == "sphere" else ellipsoid(n, m, (1.0, 1.5, 2.0))
    k = 2 * math.pi
    delta = math.pi / (2 * (n // m))
    host = B.rp_correction(s.points, s.normals, s.weights, patch_node_index(s), m, k, k, delta=delta)
    dev = B.rp_correction(s.points, s.normals, s.weights, patch_node_index(s), m, k, k, delta=delta, device=True)
    assert np.array_equal(host[0], dev[0]) and np.array_equal(host[1], dev[1])
    check(dev[2], host[2], 1e-12, shape)
    with pytest.raises(B.IFGFError, match="EUNSUPPORTED"):
        B.rp_correction(s.points, s.normals, s.weights, patch_node_index(s), m, k, k, delta=delta, n_beta=96,
                        device=True)


@pytest.mark.slow
def test_mie_solve_full_size_16_wavelengths(B):
    """Sound-soft sphere 16 wavelengths across (k = 16 pi, cube-sphere 6 x 256 x 256, N = 393,216):
    the correction built on the GPU (ifgf_rp_correction_gpu, about 600 entries per row), the
    headline apply (orders (5, 8, 8), combined factor, mixed precision) with the correction in
    every GMRES iteration (FP64 Arnoldi), plane wave along z.  The density is compared with the
    Mie series and the far field (ifgf_far_field, and ifgf_far_field_ifgf from the level-3
    interpolants) on the 200 x 200 grid of Eq. SphereGrid with the error of Eq. FarFieldRelErr;
    the paper's Table 1 reports far-field errors of order 1e-4 for spheres of this size."""
    import time

    from workloads import patch_node_index, sphere_workload

    s, k = sphere_workload(256, 8, 16.0)
    t = time.perf_counter()
    rp, col, val = B.rp_correction(s.points, s.normals, s.weights, patch_node_index(s), 8, k, k,
                                   delta=math.pi / (2 * 32), device=True)
    t_rp = time.perf_counter() - t
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, Ps=5, Pang=8, factor_mode=1))
    plan.set_correction(rp, col, val)
    del col, val
    ui = np.exp(1j * k * s.points[:, 2])
    x, ok, it, hist = plan.gmres(torch.from_numpy(-ui).cuda(), restart=60, maxit=120, tol=1e-5, precision=1)
    assert ok, hist[-5:]
    phi = x.cpu().numpy()
    e_phi = rel(phi, mie.density(s.points, k, k))
    xh = mie.sphere_grid(200, 200)
    uf = plan.far_field(x, torch.from_numpy(xh).cuda()).cpu().numpy()
    e_far = mie.far_field_error(mie.far_field(xh, k), uf)
    print(f"RP on the GPU {t_rp:.1f} s ({rp[-1]} entries), GMRES {it} iterations, density rel err {e_phi:.2e}, "
          f"far-field err {e_far:.2e}")
    assert e_phi < 5e-4, e_phi
    assert e_far < 5e-4, e_far
    assert plan.missed_lookups() == 0
    plan.close()
    # the same far field from the level-3 interpolants (a plan with the far-field cone segments)
    pf = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, Ps=5, Pang=8, factor_mode=1, far_field=1))
    ui_f = pf.far_field_ifgf(x, torch.from_numpy(xh).cuda()).cpu().numpy()
    e_far_ifgf = mie.far_field_error(mie.far_field(xh, k), ui_f)
    print(f"far-field err from the level-3 interpolants {e_far_ifgf:.2e}")
    assert e_far_ifgf < 5e-4, e_far_ifgf
    assert pf.missed_lookups() == 0
    pf.close()
