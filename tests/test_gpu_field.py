"""GPU: off-surface potential (Eq. CombinedLayer) and far-field pattern (Eq. FarField).

``ifgf_field`` / ``ifgf_far_field`` through the C ABI against the oracle's plain
numpy sums, element by element (FP64 <= 1e-12 relative l2, mixed <= 1e-5), against
the closed-form scattered field and far field of the sound-soft sphere for the
exact Mie density, at the bench's 16-wavelength sphere on sampled targets, and on
the edge cases (no targets, no right-hand sides, invalid arguments).
"""
import ctypes
import math

import numpy as np
import pytest

from oracle import mie
from parity import check
from workloads import cube_sphere, random_density, sphere_workload

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


def unit(v):
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@pytest.fixture(scope="module")
def small(B):
    s = cube_sphere(16, 8)  # N = 1,536, unit sphere two wavelengths across (k = 2 pi)
    k = 2 * math.pi
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, levels=4))
    return s, k, plan


def run(plan, fn, sig, tgt, dtype):
    out = getattr(plan, fn)(torch.from_numpy(sig.astype(dtype)).cuda(), torch.from_numpy(tgt).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("nrhs", [1, 3, 6])
def test_far_field_vs_oracle(B, oracle_lib, small, nrhs):
    s, k, plan = small
    rng = np.random.default_rng(11)
    xh = unit(rng.normal(size=(333, 3)))  # ragged over the 128-thread blocks
    sig = random_density(s.N, nrhs, 12)
    ref = oracle_lib.far_field(s.points, s.normals, s.weights, k, k, sig, xh)
    y64 = run(plan, "far_field", sig, xh, np.complex128)
    y32 = run(plan, "far_field", sig, xh, np.complex64)
    assert y64.shape == ref.shape and y32.shape == ref.shape
    check(y64, ref, 1e-12)
    check(y32, ref, 1e-5)
    for q in range(nrhs):  # every column on its own, not only the stacked norm
        assert rel(y32[q], ref[q]) < 1e-5


@pytest.mark.parametrize("nrhs", [1, 5])
def test_potential_vs_oracle(B, oracle_lib, small, nrhs):
    s, k, plan = small
    rng = np.random.default_rng(13)
    x = unit(rng.normal(size=(201, 3))) * rng.uniform(1.05, 4.0, size=(201, 1))
    x[7] = [0.0, 0.0, 0.0]        # the centre of the sphere (inside: the interior value of the representation)
    x[8] = [30.0, -20.0, 10.0]    # far outside the root box
    sig = random_density(s.N, nrhs, 14)
    ref = oracle_lib.field(s.points, s.normals, s.weights, k, k, sig, x)
    y64 = run(plan, "field", sig, x, np.complex128)
    y32 = run(plan, "field", sig, x, np.complex64)
    check(y64, ref, 1e-12)
    check(y32, ref, 1e-5)
    # FP64: a target on a source point drops that pair, as the oracle does
    x1 = s.points[[5, 900]] * 1.0
    ref1 = oracle_lib.field(s.points, s.normals, s.weights, k, k, sig, x1)
    check(run(plan, "field", sig, x1, np.complex128), ref1, 1e-12)


def test_fp64_deterministic(B, small):
    s, k, plan = small
    rng = np.random.default_rng(15)
    xh = unit(rng.normal(size=(77, 3)))
    sig = random_density(s.N, 2, 16)
    a = run(plan, "far_field", sig, xh, np.complex128)
    b = run(plan, "far_field", sig, xh, np.complex128)
    assert np.array_equal(a, b)


def test_mie_scattered_and_far_field(B):
    """Exact Mie density on the unit sphere: the GPU sums reproduce the closed-form
    scattered field (|x| = 1.5, 3) and far field (the paper's far-field error, Eq.
    FarFieldRelErr, over a spherical grid of Eq. SphereGrid)."""
    s = cube_sphere(32, 8)
    k = math.pi
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k))
    phi = mie.density(s.points, k, k)
    xh = mie.sphere_grid(21, 21)
    ue = mie.far_field(xh, k)
    u64 = run(plan, "far_field", phi, xh, np.complex128)
    u32 = run(plan, "far_field", phi, xh, np.complex64)
    assert rel(u64, ue) < 1e-7 and mie.far_field_error(ue, u64) < 1e-6
    assert rel(u32, ue) < 5e-6 and mie.far_field_error(ue, u32) < 5e-5
    rng = np.random.default_rng(17)
    d = unit(rng.normal(size=(40, 3)))
    for R, bar in ((1.5, 2e-7), (3.0, 2e-8)):
        x = d * R
        us = mie.scattered_field(x, k)
        assert rel(run(plan, "field", phi, x, np.complex128), us) < bar
        assert rel(run(plan, "field", phi, x, np.complex64), us) < 5e-6


def test_bench_sphere_sampled(B, oracle_lib):
    """The 16-wavelength sphere of the bench (N = 393,216): far field on the 200 x 200
    grid of Eq. SphereGrid and on 160,000 directions (one leaf-box chunk), potential on
    a 100 x 100 plane of Eq. PlanarGrid; sampled outputs against the oracle."""
    s, k = sphere_workload(256, 8, 16.0)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, Ps=5, Pang=8, factor_mode=1))
    sig = random_density(s.N, 1, 18)
    rng = np.random.default_rng(19)
    xh = mie.sphere_grid(200, 200)
    pick = rng.choice(xh.shape[0], 48, replace=False)
    ref = oracle_lib.far_field(s.points, s.normals, s.weights, k, k, sig, xh[pick])
    y32 = run(plan, "far_field", sig, xh, np.complex64)
    check(y32[:, pick], ref, 1e-5)
    xh2 = unit(rng.normal(size=(160000, 3)))
    pick2 = rng.choice(xh2.shape[0], 32, replace=False)
    y2 = run(plan, "far_field", sig, xh2, np.complex64)
    check(y2[:, pick2], oracle_lib.far_field(s.points, s.normals, s.weights, k, k, sig, xh2[pick2]), 1e-5)
    g = np.linspace(-3.0, 3.0, 100)
    X, Y = np.meshgrid(g, g, indexing="ij")
    plane = np.stack([X.ravel(), Y.ravel(), np.full(X.size, 1.5)], -1)
    pick3 = rng.choice(plane.shape[0], 48, replace=False)
    y3 = run(plan, "field", sig, plane, np.complex64)
    check(y3[:, pick3], oracle_lib.field(s.points, s.normals, s.weights, k, k, sig, plane[pick3]), 1e-5)


def test_edge_cases(B, small):
    s, k, plan = small
    sig = torch.from_numpy(random_density(s.N, 2, 20)).cuda()
    none = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    assert plan.far_field(sig, none).shape == (2, 0)
    assert plan.field(sig[:0], torch.ones((4, 3), dtype=torch.float64, device="cuda") * 2).shape == (0, 4)
    t = torch.ones((4, 3), dtype=torch.float64, device="cuda") * 2
    out = torch.empty((2, 4), dtype=torch.complex128, device="cuda")
    lib = B.lib()
    h = plan.handle
    VP = ctypes.c_void_p
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.ifgf_field(h, VP(sig.data_ptr()), VP(t.data_ptr()), ctypes.c_int64(-1), VP(out.data_ptr()), 2, 0, st) == -1
    assert lib.ifgf_far_field(h, VP(sig.data_ptr()), None, ctypes.c_int64(4), VP(out.data_ptr()), 2, 0, st) == -1
    assert lib.ifgf_field(h, VP(sig.data_ptr()), VP(t.data_ptr()), ctypes.c_int64(4), VP(sig.data_ptr()), 2, 0, st) == -1
    assert b"alias" in lib.ifgf_last_error()
    assert lib.ifgf_field(h, VP(sig.data_ptr()), VP(t.data_ptr()), ctypes.c_int64(4), VP(out.data_ptr()), 2, 7, st) == -1
    assert lib.ifgf_far_field(None, VP(sig.data_ptr()), VP(t.data_ptr()), ctypes.c_int64(4), VP(out.data_ptr()), 2, 0,
                              st) == -1
    with pytest.raises(TypeError):
        plan.far_field(sig.real.contiguous(), t)


def test_operator_wrapper_is_the_plan(B, small):
    """IFGFOperator(points, normals, weights, k, params) builds the same plan as Plan(..., Params(k))."""
    s, k, plan = small
    op = B.IFGFOperator(s.points, s.normals, s.weights, k, B.Params(k=0.0, levels=4))
    assert op.params.k == k and op.info()["nrc"] == plan.info()["nrc"]
    sig = torch.from_numpy(random_density(s.N, 1, 21)).cuda()
    assert torch.equal(op.apply(sig), plan.apply(sig))
    op.close()


# ---------------------------------------------------------------- far field from the IFGF interpolants
FAR_CASES = {
    # name: (geometry, params, nrhs, tensor-core fill)
    "sphere1_D3_split_3x5": (lambda: (cube_sphere(24, 6), math.pi), dict(levels=3), 2, None),
    "sphere3_D4_combined_5x8": (lambda: sphere_workload(24, 6, 3.0), dict(levels=4, Ps=5, Pang=8), 1, None),
    "sphere4_D5_split_tc_5x8": (lambda: sphere_workload(48, 6, 4.0), dict(levels=5, Ps=5, Pang=8, factor_mode=2),
                                3, 0.0),
    "sphere3_D4_6x8": (lambda: sphere_workload(32, 8, 3.0), dict(levels=4, Ps=6, Pang=8), 1, None),
}


@pytest.mark.parametrize("case", list(FAR_CASES))
def test_far_field_ifgf_vs_oracle(B, oracle_lib, case):
    """ifgf_far_field_ifgf against the oracle's far field from the level-3 interpolants,
    element by element (FP64 <= 1e-10, mixed <= 1e-5), and against the plain quadrature sum
    of Eq. FarField within the IFGF error of the orders used; repeatable bit for bit; an
    ordinary apply on the same plan afterwards is unchanged."""
    geo, kw, nrhs, fill = FAR_CASES[case]
    s, k = geo()
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, far_field=1, **kw))
    if fill is not None:
        plan.set_tc_fill(fill)
    sig = random_density(s.N, nrhs, 41)
    rng = np.random.default_rng(42)
    xh = unit(rng.normal(size=(333, 3)))
    xh[:6] = [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0]]  # cone-grid poles and seams
    ref, info = oracle_lib.ifgf_far_field(s.points, s.normals, s.weights,
                                          oracle_lib.IFGFParams(k=k, **kw), sig, xh)
    assert info["D"] == plan.info()["D"]
    y64 = run(plan, "far_field_ifgf", sig, xh, np.complex128)
    y32 = run(plan, "far_field_ifgf", sig, xh, np.complex64)
    assert plan.missed_lookups() == 0
    check(y64, ref, 1e-10, "fp64")
    check(y32, ref, 1e-5, "mixed")
    direct = oracle_lib.far_field(s.points, s.normals, s.weights, k, k, sig, xh)
    bound = 3e-3 if kw.get("Ps", 3) == 3 else 1e-4
    assert rel(y64, direct) < bound
    assert np.array_equal(run(plan, "far_field_ifgf", sig, xh, np.complex64), y32)
    # the upward-only pass leaves the plan's apply as it was
    sg = torch.from_numpy(sig.astype(np.complex128)).cuda()
    ya = plan.apply(sg).cpu().numpy()
    yr, _ = oracle_lib.ifgf(s.points, s.normals, s.weights, oracle_lib.IFGFParams(k=k, identity_coef=0.5, **kw), sig)
    check(ya, yr, 1e-10, "apply after far field")
    plan.close()


def test_far_field_ifgf_mie(B):
    """Exact Mie density on the unit sphere (k = pi): the IFGF far field on a grid of Eq.
    SphereGrid against the closed form (Eq. FarFieldRelErr), at orders (5, 8)."""
    s = cube_sphere(32, 8)
    k = math.pi
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, Ps=5, Pang=8, far_field=1))
    phi = mie.density(s.points, k, k)
    xh = mie.sphere_grid(41, 41)
    ue = mie.far_field(xh, k)
    u64 = run(plan, "far_field_ifgf", phi, xh, np.complex128)
    u32 = run(plan, "far_field_ifgf", phi, xh, np.complex64)
    assert mie.far_field_error(ue, u64) < 2e-5 and mie.far_field_error(ue, u32) < 3e-5
    plan.close()


def test_far_field_ifgf_edge_cases(B):
    s = cube_sphere(16, 8)
    k = 2 * math.pi
    lib = B.lib()
    plain = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, levels=3))
    sig = torch.from_numpy(random_density(s.N, 1, 43)).cuda()
    xh = torch.from_numpy(unit(np.random.default_rng(44).normal(size=(5, 3)))).cuda()
    out = torch.zeros((1, 5), dtype=torch.complex128, device="cuda")
    # a plan without the far-field segments is refused
    st = lib.ifgf_far_field_ifgf(plain.handle, ctypes.c_void_p(sig.data_ptr()), ctypes.c_void_p(xh.data_ptr()),
                                 ctypes.c_int64(5), ctypes.c_void_p(out.data_ptr()), ctypes.c_int(1), ctypes.c_int(0),
                                 ctypes.c_void_p(0))
    assert st == -1 and "far_field" in lib.ifgf_last_error().decode()
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, levels=3, far_field=1))
    # no directions / no right-hand sides: nothing to do
    for M, nrhs in ((0, 1), (5, 0)):
        st = lib.ifgf_far_field_ifgf(plan.handle, ctypes.c_void_p(sig.data_ptr()), ctypes.c_void_p(xh.data_ptr()),
                                     ctypes.c_int64(M), ctypes.c_void_p(out.data_ptr()), ctypes.c_int(nrhs),
                                     ctypes.c_int(0), ctypes.c_void_p(0))
        assert st == 0
    # invalid precision, aliasing output
    st = lib.ifgf_far_field_ifgf(plan.handle, ctypes.c_void_p(sig.data_ptr()), ctypes.c_void_p(xh.data_ptr()),
                                 ctypes.c_int64(5), ctypes.c_void_p(out.data_ptr()), ctypes.c_int(1), ctypes.c_int(7),
                                 ctypes.c_void_p(0))
    assert st == -1
    st = lib.ifgf_far_field_ifgf(plan.handle, ctypes.c_void_p(sig.data_ptr()), ctypes.c_void_p(xh.data_ptr()),
                                 ctypes.c_int64(5), ctypes.c_void_p(sig.data_ptr()), ctypes.c_int(1), ctypes.c_int(0),
                                 ctypes.c_void_p(0))
    assert st == -1
    plain.close()
    plan.close()


# ---------------------------------------------------------------- potential at targets inside the octree
def _targets(rng):
    g = np.linspace(-2.0, 2.0, 30)
    X, Y = np.meshgrid(g, g, indexing="ij")
    plane = np.stack([X.ravel(), Y.ravel(), np.full(X.size, 1.5)], -1)  # a plane of Eq. PlanarGrid
    d = unit(rng.normal(size=(200, 3)))
    return np.concatenate([plane, d * rng.uniform(1.2, 3.0, (200, 1))])


@pytest.mark.parametrize("layer,orders", [(0, (3, 5)), (0, (5, 8)), (2, (5, 8))])
def test_field_ifgf_vs_oracle(B, oracle_lib, layer, orders):
    """ifgf_field_ifgf: the targets join the octree as zero-weight points; against the oracle's IFGF
    on the same point set (element by element: FP64 <= 1e-10, mixed <= 1e-5) and against the plain
    quadrature sum of Eq. CombinedLayer within the IFGF error of the orders."""
    s, k = sphere_workload(24, 6, 3.0)
    rng = np.random.default_rng(61)
    tg = _targets(rng)
    M = tg.shape[0]
    ps, pa = orders
    kw = dict(levels=5, Ps=ps, Pang=pa, layer=layer)
    plan = B.Plan.with_targets(s.points, s.normals, s.weights, tg, B.Params(k=k, **kw))
    assert plan.n_targets == M and plan.N == s.N + M
    sig = random_density(s.N, 2, 62)
    xa = np.concatenate([s.points, tg])
    na = np.concatenate([s.normals, np.zeros_like(tg)])
    wa = np.concatenate([s.weights, np.zeros(M)])
    sa = np.concatenate([sig, np.zeros((2, M), complex)], axis=1)
    ya, info = oracle_lib.ifgf(xa, na, wa, oracle_lib.IFGFParams(k=k, identity_coef=0.5, **kw), sa)
    ref = ya[:, s.N:]
    assert info["D"] == plan.info()["D"]
    for dt, tol in ((np.complex128, 1e-10), (np.complex64, 1e-5)):
        y = plan.field_ifgf(torch.from_numpy(sig.astype(dt)).cuda())
        torch.cuda.synchronize()
        check(y.cpu().numpy(), ref, tol, str(dt))
    assert plan.missed_lookups() == 0
    direct = oracle_lib.field(s.points, s.normals, s.weights, k, k, sig, tg, layer=layer)
    assert rel(ref, direct) < (5e-3 if ps == 3 else 2e-4)
    plan.close()


def test_field_ifgf_edge_cases(B):
    s = cube_sphere(16, 8)
    k = 2 * math.pi
    plain = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, levels=3))
    sig = torch.from_numpy(random_density(s.N, 1, 63)).cuda()
    out = torch.zeros((1, 4), dtype=torch.complex128, device="cuda")
    lib = B.lib()
    st = lib.ifgf_field_ifgf(plain.handle, ctypes.c_void_p(sig.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                             ctypes.c_int(1), ctypes.c_int(0), ctypes.c_void_p(0))
    assert st == -1 and "targets" in lib.ifgf_last_error().decode()
    bad = np.array([[2.0, 0.0, 0.0], [np.nan, 0.0, 0.0]])
    with pytest.raises(B.IFGFError):
        B.Plan.with_targets(s.points, s.normals, s.weights, bad, B.Params(k=k, levels=3))
    with pytest.raises(B.IFGFError):
        B.Plan.with_targets(s.points, s.normals, s.weights, np.zeros((0, 3)), B.Params(k=k, levels=3))
    plan = B.Plan.with_targets(s.points, s.normals, s.weights, np.array([[3.0, 0.0, 0.0]]),
                               B.Params(k=k, levels=3))
    assert plan.field_ifgf(sig[:0]).shape == (0, 1)
    plain.close()
    plan.close()
