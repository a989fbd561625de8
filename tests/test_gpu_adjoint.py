"""GPU adjoint A^H of the discrete operator (conjugate transpose of every stage).

* FP64: <A s, g> = <s, A^H g> to 1e-12 relative (exact identity of a linear map).
* Tiny surface: A^H g equals the conjugate transpose of the oracle's Algorithm 1
  matrix (built column by column from the oracle) to 1e-10.
* Mixed adjoint vs FP64 adjoint <= 1e-5; dense oracle adjoint (direct sum) on
  sampled columns within the interpolation error.
"""
import math

import numpy as np
import pytest

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


def cu(a, dt=np.complex128):
    return torch.from_numpy(np.ascontiguousarray(a.astype(dt))).cuda()


@pytest.mark.parametrize("fm", [0, 1, 2])
def test_dot_product_identity_fp64(B, oracle_lib, fm):
    s, k = sphere_workload(48, 6, 4.0)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, levels=4, factor_mode=fm))
    # a random sparse correction makes C^H part of the test
    rng = np.random.default_rng(3)
    counts = rng.integers(0, 20, s.N)
    rowptr = np.concatenate([[0], np.cumsum(counts)])
    col = rng.integers(0, s.N, rowptr[-1]).astype(np.int32)
    val = (rng.normal(size=rowptr[-1]) + 1j * rng.normal(size=rowptr[-1])) * 1e-3
    plan.set_correction(rowptr, col, val)
    sig = random_density(s.N, 2, 1)
    g = random_density(s.N, 2, 2)
    As = plan.apply(cu(sig)).cpu().numpy()
    Ahg = plan.adjoint(cu(g)).cpu().numpy()
    lhs = np.vdot(g, As)
    rhs = np.vdot(Ahg, sig)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    Ahg32 = plan.adjoint(cu(g, np.complex64)).cpu().numpy()
    check(Ahg32, Ahg, 1e-5)
    assert plan.missed_lookups() == 0


@pytest.mark.parametrize("orders", [(3, 5), (4, 6), (5, 8)])
@pytest.mark.parametrize("fm", [0, 1, 2])
def test_mixed_adjoint_orders_and_factors(B, orders, fm):
    """The FP32 anterpolation owns one (Pang odd), two (Pang = 6) or four (Pang = 8) output
    columns per thread, with one or two factors per cone: each layout, two right-hand
    sides, matches the FP64 adjoint (which the oracle pins above and below)."""
    s, k = sphere_workload(48, 6, 4.0)
    plan = B.Plan(s.points, s.normals, s.weights,
                  B.Params(k=k, Ps=orders[0], Pang=orders[1], levels=4, factor_mode=fm))
    g = random_density(s.N, 2, 4)
    a64 = plan.adjoint(cu(g)).cpu().numpy()
    a32 = plan.adjoint(cu(g, np.complex64)).cpu().numpy()
    check(a32, a64, 1e-5)
    assert plan.missed_lookups() == 0


def test_adjoint_matches_oracle_matrix_transpose(B, oracle_lib):
    """Tiny 4-level surface: the oracle's Algorithm 1 applied to every unit vector gives
    the discrete IFGF matrix M; the GPU adjoint must equal M^H g."""
    s = cube_sphere(8, 8)  # N = 384
    k = 9.0
    prm = dict(k=k, levels=4)
    N = s.N
    M = np.zeros((N, N), dtype=np.complex128)
    E = np.eye(N, dtype=np.complex128)
    for c0 in range(0, N, 64):
        y, _ = oracle_lib.ifgf(s.points, s.normals, s.weights,
                               oracle_lib.IFGFParams(identity_coef=0.5, **prm), E[c0:c0 + 64])
        M[:, c0:c0 + 64] = y.T
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(**prm))
    g = random_density(N, 3, 7)
    ref = (M.conj().T @ g.T).T
    got = plan.adjoint(cu(g)).cpu().numpy()
    check(got, ref, 1e-10)
    got32 = plan.adjoint(cu(g, np.complex64)).cpu().numpy()
    check(got32, ref, 1e-5)


def test_adjoint_vs_dense_direct_adjoint(B, oracle_lib):
    """Columns of the exact (direct-sum) adjoint on a sample: the IFGF adjoint agrees to the
    accuracy of the interpolation orders."""
    s, k = sphere_workload(64, 8, 6.0)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, Ps=5, Pang=8))
    g = random_density(s.N, 1, 5)
    rows = np.random.default_rng(1).choice(s.N, 4096, replace=False)  # 4,096 dense columns
    ref = oracle_lib.direct_adjoint(s.points, s.normals, s.weights, k, k, g, cI=0.5, rows=rows)
    got = plan.adjoint(cu(g)).cpu().numpy()[:, rows]
    assert rel(got, ref) < 1e-4
    got32 = plan.adjoint(cu(g, np.complex64)).cpu().numpy()[:, rows]
    assert rel(got32, ref) < 1e-4


@pytest.mark.slow
def test_mixed_adjoint_full_size(B):
    """16-wavelength sphere (N = 393,216) at orders (5, 8, 8): the FP32 classification of
    anterpolation entries may differ from the host lists near cone boundaries; the local
    coordinates are then re-expressed in the list's cone.  No real misses, and the
    mixed adjoint matches the FP64 adjoint."""
    s, k = sphere_workload(256, 8, 16.0)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, Ps=5, Pang=8))
    g = random_density(s.N, 1, 9)
    a64 = plan.adjoint(cu(g)).cpu().numpy()
    a32 = plan.adjoint(cu(g, np.complex64)).cpu().numpy()
    assert plan.missed_lookups() == 0
    check(a32, a64, 1e-5)
