"""GPU parity of the C-ABI apply against the FP64 oracle (element by element).

Bars: FP64 path vs the oracle's Algorithm 1 with identical parameters <= 1e-10
relative l2; mixed path <= 1e-5; IFGF vs the direct sum at the accuracy the
interpolation orders reach.  Every apply also checks that no point fell outside
the plan's relevant cone segments.
"""
import math

import numpy as np
import pytest

from parity import check, rel
from workloads import cube_sphere, ellipsoid, random_density, sphere_workload, star_body

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_06316_gb300 import binding
    from paper_2112_06316_gb300 import build as _b

    _b.build()
    return binding


def gpu_apply(plan, sig, dtype):
    t = torch.from_numpy(sig.astype(dtype)).cuda()
    y = plan.apply(t)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def run_case(lib, oracle_lib, x, n, w, k, prm_kw, nrhs=1, seed=1, tol64=1e-10, tol32=1e-5):
    sig = random_density(x.shape[0], nrhs, seed)
    okw = {kk: v for kk, v in prm_kw.items() if kk != "cone_band"}
    ref, oinfo = oracle_lib.ifgf(x, n, w, oracle_lib.IFGFParams(k=k, identity_coef=0.5, **okw), sig)
    plan = lib.Plan(x, n, w, lib.Params(k=k, **prm_kw))
    y64 = gpu_apply(plan, sig, np.complex128)
    y32 = gpu_apply(plan, sig, np.complex64)
    assert plan.missed_lookups() == 0
    e64 = check(y64, ref, tol64, "fp64")
    e32 = check(y32, ref, tol32, "mixed")
    info = plan.info()
    assert info["D"] == oinfo["D"]
    plan.close()
    return e64, e32, ref, sig


def test_config1_sphere_1lambda(lib, oracle_lib):
    """Unit sphere 1 wavelength across (k = pi), 6 x 26 x 26 points, D = 3, orders (3, 5, 5)."""
    s = cube_sphere(26)
    k = math.pi
    e64, e32, ref, sig = run_case(lib, oracle_lib, s.points, s.normals, s.weights, k, {"levels": 3})
    yd = oracle_lib.direct(s.points, s.normals, s.weights, k, k, sig, cI=0.5)
    assert rel(ref, yd) < 3e-3  # IFGF at (3,5,5) vs the direct sum


@pytest.mark.parametrize("fm", [0, 1, 2])
def test_multilevel_factor_modes(lib, oracle_lib, fm):
    """4-wavelength sphere, D = 4: split / combined factors and their conversion in propagation."""
    s, k = sphere_workload(48, 6, 4.0)
    run_case(lib, oracle_lib, s.points, s.normals, s.weights, k, {"levels": 4, "factor_mode": fm}, nrhs=2)


@pytest.mark.parametrize("ps,pa", [(4, 6), (5, 7), (5, 8), (6, 8)])
def test_higher_orders(lib, oracle_lib, ps, pa):
    s, k = sphere_workload(32, 8, 3.0)
    run_case(lib, oracle_lib, s.points, s.normals, s.weights, k, {"levels": 4, "Ps": ps, "Pang": pa})


def test_literal_cone_rule_and_more_rhs(lib, oracle_lib):
    s, k = sphere_workload(64, 8, 6.0)
    run_case(lib, oracle_lib, s.points, s.normals, s.weights, k, {"levels": 5, "cone_rule": 1}, nrhs=5)


def test_ellipsoid_and_star_body(lib, oracle_lib):
    e = ellipsoid(40, 8, (1.0, 1.6, 2.4))
    run_case(lib, oracle_lib, e.points, e.normals, e.weights, 12.0, {"levels": 5})
    t = star_body(32, 8, 4)
    run_case(lib, oracle_lib, t.points, t.normals, t.weights, 15.0, {})


def test_uneven_cloud_ragged_boxes(lib, oracle_lib):
    """Clustered random points: boxes with 1..hundreds of points, empty neighbours, ragged tails."""
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(size=(2000, 3)) * 0.05, rng.uniform(-1, 1, (1001, 3))])
    n = rng.normal(size=x.shape)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    w = rng.uniform(0.5, 1.5, x.shape[0])
    run_case(lib, oracle_lib, x, n, w, 20.0, {"levels": 6}, nrhs=3)


def test_tiny_inputs(lib, oracle_lib):
    """N = 1 (no interactions: y = sigma / 2), N = 2 and 9 (cousins of each other or
    neighbours), and nrhs = 0 (no-op)."""
    for N in (1, 2, 9):
        rng = np.random.default_rng(N)
        x = rng.uniform(-1, 1, (N, 3))
        n = rng.normal(size=(N, 3))
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        w = np.ones(N)
        sig = random_density(N, 1, 3)
        plan = lib.Plan(x, n, w, lib.Params(k=3.0))
        y = gpu_apply(plan, sig, np.complex128)
        ref, _ = oracle_lib.ifgf(x, n, w, oracle_lib.IFGFParams(k=3.0, identity_coef=0.5), sig)
        check(y, ref, 1e-12)
        if N == 1:
            assert np.allclose(y, 0.5 * sig, rtol=0, atol=1e-15)
        z = torch.zeros((0, N), dtype=torch.complex128, device="cuda")
        assert plan.apply(z).shape == (0, N)


def test_fp64_bitwise_deterministic(lib):
    s, k = sphere_workload(48, 6, 4.0)
    plan = lib.Plan(s.points, s.normals, s.weights, lib.Params(k=k))
    sig = random_density(s.N, 1, 9)
    a = gpu_apply(plan, sig, np.complex128)
    b = gpu_apply(plan, sig, np.complex128)
    assert np.array_equal(a, b)
    a = gpu_apply(plan, sig, np.complex64)
    b = gpu_apply(plan, sig, np.complex64)
    assert np.array_equal(a, b)


def test_sparse_correction(lib, oracle_lib):
    """K5: y(with C) - y(without C) equals the plain CSR product C sigma."""
    s, k = sphere_workload(32, 8, 3.0)
    rng = np.random.default_rng(4)
    N = s.N
    counts = rng.integers(0, 40, N)
    counts[::7] = 0  # empty rows
    rowptr = np.concatenate([[0], np.cumsum(counts)])
    col = rng.integers(0, N, rowptr[-1]).astype(np.int32)
    val = rng.normal(size=rowptr[-1]) + 1j * rng.normal(size=rowptr[-1])
    plan = lib.Plan(s.points, s.normals, s.weights, lib.Params(k=k))
    sig = random_density(N, 2, 5)
    y0 = gpu_apply(plan, sig, np.complex128)
    y0m = gpu_apply(plan, sig, np.complex64)
    plan.set_correction(rowptr, col, val)
    assert plan.info()["correction_nnz"] == rowptr[-1]
    y1 = gpu_apply(plan, sig, np.complex128)
    y1m = gpu_apply(plan, sig, np.complex64)
    ref = oracle_lib.csr_apply(rowptr, col, val, sig)
    check(y1 - y0, ref, 1e-13)
    check(y1m - y0m, ref, 1e-5)
    plan.set_correction(np.zeros(N + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, complex))
    assert np.array_equal(gpu_apply(plan, sig, np.complex128), y0)


@pytest.mark.slow
def test_config2_full_size(lib, oracle_lib):
    """Sphere 16 wavelengths across, 6 x 256 x 256 points (N = 393,216), auto D = 6, orders (3, 5, 5)."""
    s, k = sphere_workload(256, 8, 16.0)
    e64, e32, ref, sig = run_case(lib, oracle_lib, s.points, s.normals, s.weights, k, {}, seed=2)
    rows = np.random.default_rng(0).choice(s.N, 2000, replace=False)
    yd = oracle_lib.direct(s.points, s.normals, s.weights, k, k, sig, cI=0.5, rows=rows)
    assert rel(ref[:, rows], yd) < 6e-3


@pytest.mark.slow
def test_config2_qualified_orders_vs_direct(lib, oracle_lib):
    """Orders (5, 8, 8) on the 16-wavelength sphere reach <= 1e-4 against the direct sum
    (sampled rows), in FP64 and in mixed precision."""
    s, k = sphere_workload(256, 8, 16.0)
    sig = random_density(s.N, 1, 2)
    rows = np.random.default_rng(0).choice(s.N, 2000, replace=False)
    yd = oracle_lib.direct(s.points, s.normals, s.weights, k, k, sig, cI=0.5, rows=rows)
    plan = lib.Plan(s.points, s.normals, s.weights, lib.Params(k=k, Ps=5, Pang=8))
    y64 = gpu_apply(plan, sig, np.complex128)
    y32 = gpu_apply(plan, sig, np.complex64)
    assert plan.missed_lookups() == 0
    assert rel(y64[:, rows], yd) < 1e-4
    assert rel(y32[:, rows], yd) < 1e-4
    check(y32, y64, 1e-5)


@pytest.mark.parametrize("engine", [2, 1, 0])
@pytest.mark.parametrize("fm", [0, 1, 2])
@pytest.mark.parametrize("ps", [5, 6])
def test_tensor_core_propagation_modes(lib, oracle_lib, ps, fm, engine):
    """Orders with Pang = 8 propagate through the tensor cores on the mixed path (engine 2:
    tcgen05 over the K = 8 c-contraction per (node run, pair), the b- and a-contractions on CUDA
    cores; engine 1: tcgen05 with TMEM accumulators over the K = 64 angular contraction; engine 0:
    warp mma.sync over K = P; all with a three-term TF32 split), forced on at every level (fill
    threshold 0);
    two propagation levels (D = 5) in every factor-mode combination (split -> split,
    split -> combined, combined -> combined), two right-hand sides.  The result matches the
    oracle to the mixed bar and the CUDA-core propagation (threshold > 1) to 2e-6."""
    s, k = sphere_workload(64, 8, 6.0)
    sig = random_density(s.N, 2, 4)
    ref, _ = oracle_lib.ifgf(s.points, s.normals, s.weights,
                             oracle_lib.IFGFParams(k=k, identity_coef=0.5, levels=5, Ps=ps, Pang=8,
                                                   factor_mode=fm), sig)
    plan = lib.Plan(s.points, s.normals, s.weights, lib.Params(k=k, levels=5, Ps=ps, Pang=8, factor_mode=fm))
    plan.set_tc_engine(engine)
    plan.set_tc_fill(0.0)
    y_tc = gpu_apply(plan, sig, np.complex64)
    assert plan.missed_lookups() == 0
    plan.set_tc_fill(2.0)
    y_cc = gpu_apply(plan, sig, np.complex64)
    check(y_tc, ref, 1e-5, "tensor cores vs oracle")
    check(y_tc, y_cc, 2e-6, "tensor cores vs CUDA cores")
    plan.close()


def test_tensor_core_propagation_full_size_level_choice(lib):
    """16-wavelength sphere at orders (5, 8): the default fill threshold puts the fine
    propagation levels on the tensor cores; the result equals the all-CUDA-core one to
    2e-6 and the FP64 apply to 1e-5."""
    s, k = sphere_workload(256, 8, 16.0)
    sig = random_density(s.N, 1, 8)
    plan = lib.Plan(s.points, s.normals, s.weights, lib.Params(k=k, Ps=5, Pang=8))
    y_def = gpu_apply(plan, sig, np.complex64)
    plan.set_tc_fill(2.0)
    y_cc = gpu_apply(plan, sig, np.complex64)
    y64 = gpu_apply(plan, sig, np.complex128)
    assert plan.missed_lookups() == 0
    check(y_def, y_cc, 2e-6, "default vs CUDA-core propagation")
    check(y_def, y64, 1e-5, "mixed vs fp64")
    plan.close()


@pytest.mark.parametrize("prec", [np.complex64, np.complex128])
def test_concurrent_stages_match_single_stream(lib, prec):
    """The near field and the cousin interpolation run on the plan's auxiliary stream beside the
    leaf/propagation chain; with profiling on everything runs on the caller's stream.  Both orders
    of execution give bitwise-identical fields (every kernel is output-stationary, and the field's
    writers run in the same order on either schedule)."""
    s, k = sphere_workload(64, 8, 6.0)
    sig = random_density(s.N, 2, 12)
    plan = lib.Plan(s.points, s.normals, s.weights, lib.Params(k=k, levels=5, Ps=5, Pang=8))
    y_par = gpu_apply(plan, sig, prec)
    plan.set_profiling(True)
    y_seq = gpu_apply(plan, sig, prec)
    assert len(plan.stage_times()) > 0
    plan.set_profiling(False)
    assert plan.missed_lookups() == 0
    assert np.array_equal(y_par, y_seq)
    plan.close()


@pytest.mark.slow
def test_bench_configuration_full_size_vs_oracle(lib, oracle_lib):
    """The timed configuration itself against the oracle over all N: 16-wavelength sphere
    (6 x 256 x 256 points, N = 393,216, automatic depth 6), orders (5, 8, 8), the combined
    factor on every level (factor mode 1) and the default tensor-core fill threshold, so the
    two finest propagation steps run on the tensor cores.  FP64 <= 1e-10 and mixed <= 1e-5
    against the oracle's Algorithm 1 with identical parameters, in l2 and element-wise."""
    s, k = sphere_workload(256, 8, 16.0)
    prm = {"Ps": 5, "Pang": 8, "factor_mode": 1}
    sig = random_density(s.N, 1, 2)
    ref, oinfo = oracle_lib.ifgf(s.points, s.normals, s.weights,
                                 oracle_lib.IFGFParams(k=k, identity_coef=0.5, **prm), sig)
    plan = lib.Plan(s.points, s.normals, s.weights, lib.Params(k=k, **prm))
    info = plan.info()
    assert info["D"] == oinfo["D"] == 6
    y64 = gpu_apply(plan, sig, np.complex128)
    y32 = gpu_apply(plan, sig, np.complex64)
    assert plan.missed_lookups() == 0
    plan.set_profiling(True)
    gpu_apply(plan, sig, np.complex64)
    kinds = {kd for kd, _, _ in plan.stage_times()}
    plan.set_profiling(False)
    assert "prop_tc" in kinds  # the tensor-core propagation ran
    check(y64, ref, 1e-10, "fp64")
    check(y32, ref, 1e-5, "mixed")
    plan.close()


@pytest.mark.parametrize("fm", [0, 1, 2])
def test_interp_engines(lib, oracle_lib, fm):
    """Both mixed CUDA-core interpolation engines (cone-stationary: cousin lists and grouped
    propagation, the default; point-stationary: kept for plans of 2^24 points or more) against
    the oracle, with split, combined and mixed factor levels, three right-hand sides, the
    propagation on CUDA cores (tensor-core fill threshold above 1); the two agree to FP32
    rounding.  Both are bitwise reproducible (fixed summation order)."""
    s, k = sphere_workload(64, 8, 6.0)
    sig = random_density(s.N, 3, 41)
    prm = dict(levels=5, Ps=5, Pang=8, factor_mode=fm)
    ref, _ = oracle_lib.ifgf(s.points, s.normals, s.weights, oracle_lib.IFGFParams(k=k, identity_coef=0.5, **prm), sig)
    plan = lib.Plan(s.points, s.normals, s.weights, lib.Params(k=k, **prm))
    plan.set_tc_fill(2.0)
    y1 = gpu_apply(plan, sig, np.complex64)
    assert np.array_equal(y1, gpu_apply(plan, sig, np.complex64))
    plan.set_profiling(True)
    gpu_apply(plan, sig, np.complex64)
    kinds = [kd for kd, _, _ in plan.stage_times()]
    plan.set_profiling(False)
    assert "prop_cs" in kinds and "cousin_sum" in kinds, kinds
    plan.set_interp_engine(0)
    y0 = gpu_apply(plan, sig, np.complex64)
    assert plan.missed_lookups() == 0
    check(y1, ref, 1e-5, "cone-stationary")
    check(y0, ref, 1e-5, "point-stationary")
    check(y1, y0, 2e-6, "engines")
    plan.close()
