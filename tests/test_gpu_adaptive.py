"""GPU: the adaptive octree (ifgf_params.leaf_max > 0) for non-uniform point densities.

A box of level 3..D-1 holding at most leaf_max points is a leaf: its factor F at its relevant cone
nodes comes from its points directly (the FP64 leaf kernel on a list of cones, the mixed k_leaf32a),
no boxes exist below it, and only points that still have a box at level d take level-d cousin
interpolation.  Points of two leaves interact directly when their boxes neighbour at the coarser of
the two leaf levels.  Checked element by element against the oracle's adaptive IFGF (FP64 <= 1e-10,
mixed <= 1e-5) on the two-sphere set (point density 20x higher in one corner) and a 3:1 ellipsoid
(a stretched cube-sphere grid: points three times denser at the tips than around the waist), with
the orders (3, 5) and (5, 8), the split and combined factors, the tcgen05 propagation, both mixed
cousin engines and one and two right-hand sides; against the direct sum on sampled rows; a leaf budget
above every box's count reproduces the uniform three-level plan; far field from the level-3
interpolants and potential at targets on adaptive plans; chunks of leaves with long near-source
lists run as one block each; the adjoint (against the forward by the inner-product identity) and
the k-gradient against central differences, and the density gradient through autograd.
"""
import numpy as np
import pytest

from parity import check, rel
from workloads import ellipsoid, random_density, two_spheres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

K = 2 * np.pi  # the unit sphere is two wavelengths across


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_06316_gb300 import binding
    from paper_2112_06316_gb300 import build as _b

    _b.build()
    return binding


@pytest.fixture(scope="module")
def geo():
    return two_spheres()


def cu(a, dt=np.complex128):
    return torch.from_numpy(np.ascontiguousarray(a.astype(dt))).cuda()


def apply(plan, sig, dt):
    y = plan.apply(cu(sig, dt))
    torch.cuda.synchronize()
    return y.cpu().numpy()


# (plan parameters, tensor-core fill threshold or None, mixed cousin engine or None)
CASES = {
    "leaf64_3x5": (dict(levels=6, leaf_max=64), None, None),
    "leaf64_5x8": (dict(levels=6, leaf_max=64, Ps=5, Pang=8), None, None),
    "leaf64_5x8_tc": (dict(levels=6, leaf_max=64, Ps=5, Pang=8), 0.0, None),
    "leaf64_5x8_chunked_cousins": (dict(levels=6, leaf_max=64, Ps=5, Pang=8), None, 0),
    "leaf16_D7_split": (dict(levels=7, leaf_max=16, factor_mode=2), None, None),
    "leaf16_D7_combined": (dict(levels=7, leaf_max=16, factor_mode=1), None, None),
    "ellipsoid_3to1_leaf32": (dict(levels=6, leaf_max=32, Ps=5, Pang=8), None, None),
}


@pytest.mark.parametrize("case", list(CASES))
def test_adaptive_apply_vs_oracle(B, oracle_lib, geo, case):
    kw, fill, engine = CASES[case]
    s = ellipsoid(32, 8, (1.0, 1.0, 3.0)) if case.startswith("ellipsoid") else geo
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=K, **kw))
    if fill is not None:
        plan.set_tc_fill(fill)
    if engine is not None:
        plan.set_interp_engine(engine)
    sig = random_density(s.N, 2, 71)
    ref, oinfo = oracle_lib.ifgf(s.points, s.normals, s.weights, oracle_lib.IFGFParams(k=K, identity_coef=0.5, **kw),
                                 sig)
    info = plan.info()
    # same tree; the library's relevant cones are the oracle's plus those within the FP32 classification
    # band (cone_band) of a marked point
    assert info["D"] == oinfo["D"] and info["cousin_evals"] == oinfo["cousin_evals"]
    assert all(o <= g <= 1.1 * o for g, o in zip(info["nrc"], oinfo["nrc"]))
    check(apply(plan, sig, np.complex128), ref, 1e-10, "fp64")
    check(apply(plan, sig, np.complex64), ref, 1e-5, "mixed")
    # one right-hand side: the source-pair leaf and near kernels at level D
    check(apply(plan, sig[:1], np.complex128), ref[:1], 1e-10, "fp64 nrhs 1")
    check(apply(plan, sig[:1], np.complex64), ref[:1], 1e-5, "mixed nrhs 1")
    assert plan.missed_lookups() == 0
    rows = np.random.default_rng(72).choice(s.N, 300, replace=False)
    yd = oracle_lib.direct(s.points, s.normals, s.weights, K, K, sig, cI=0.5, rows=rows)
    assert rel(ref[:, rows], yd) < (5e-3 if kw.get("Ps", 3) == 3 else 1e-4)
    plan.close()


def test_adaptive_near_block_chunks(B, oracle_lib):
    """Leaves whose near-source lists are long (small level-3 leaves beside dense boxes) run their
    near field as one block per chunk (warps split the sources, summed in warp order): the mixed
    apply, one and two right-hand sides, against the oracle."""
    s = two_spheres(48, 32, 0.1, 1.6)
    kw = dict(levels=7, leaf_max=64)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=K, **kw))
    assert plan.info()["near_block_chunks"] > 0
    sig = random_density(s.N, 2, 77)
    ref, _ = oracle_lib.ifgf(s.points, s.normals, s.weights, oracle_lib.IFGFParams(k=K, identity_coef=0.5, **kw), sig)
    check(apply(plan, sig, np.complex64), ref, 1e-5, "mixed")
    check(apply(plan, sig[:1], np.complex64), ref[:1], 1e-5, "mixed nrhs 1")
    check(apply(plan, sig, np.complex128), ref, 1e-10, "fp64")
    assert plan.missed_lookups() == 0
    plan.close()


def test_adaptive_tree_has_coarse_leaves(B, geo):
    """The two-sphere set's adaptive plan keeps far fewer relevant cones than the uniform one and
    has leaves above level D (so the coarse-leaf kernels are exercised by the parity cases)."""
    s = geo
    pu = B.dry_run(s.points, s.normals, s.weights, B.Params(k=K, levels=6, Ps=5, Pang=8))
    pa = B.dry_run(s.points, s.normals, s.weights, B.Params(k=K, levels=6, Ps=5, Pang=8, leaf_max=64))
    assert sum(pa["nrc"]) < sum(pu["nrc"]) / 5
    # level-3 boxes (side L / 8) of at most 64 points: leaves five levels above D
    lo = np.asarray(pa["root_center"]) - pa["root_side"] / 2
    ijk = np.clip(np.floor((s.points - lo) / (pa["root_side"] / 8)).astype(int), 0, 7)
    _, counts = np.unique(ijk, axis=0, return_counts=True)
    assert (counts <= 64).any() and (counts > 64).any()


def test_leaf_budget_above_every_box_is_the_three_level_plan(B, geo):
    """leaf_max >= N: every level-3 box is a leaf and the plan of depth 6 computes the uniform
    three-level apply (coarse-leaf kernels and near lists built from level-6 boxes against the level-3
    plan's own kernels: equal to rounding)."""
    s = geo
    sig = random_density(s.N, 2, 73)
    p3 = B.Plan(s.points, s.normals, s.weights, B.Params(k=K, levels=3))
    pa = B.Plan(s.points, s.normals, s.weights, B.Params(k=K, levels=6, leaf_max=10 ** 9))
    y3 = apply(p3, sig, np.complex128)
    check(apply(pa, sig, np.complex128), y3, 1e-12, "fp64")
    check(apply(pa, sig, np.complex64), y3, 1e-5, "mixed")
    p3.close()
    pa.close()


def test_adaptive_far_field_and_targets(B, oracle_lib, geo):
    """Far field from the level-3 interpolants and the potential at targets inside the octree, both
    on adaptive plans, against the oracle's adaptive IFGF on the same trees."""
    s = geo
    kw = dict(levels=6, leaf_max=64, Ps=5, Pang=8)
    sig = random_density(s.N, 2, 74)
    rng = np.random.default_rng(75)
    xh = rng.normal(size=(129, 3))
    xh /= np.linalg.norm(xh, axis=1)[:, None]
    pf = B.Plan(s.points, s.normals, s.weights, B.Params(k=K, far_field=1, **kw))
    fi_ref, _ = oracle_lib.ifgf_far_field(s.points, s.normals, s.weights, oracle_lib.IFGFParams(k=K, **kw), sig, xh)
    for dt, tol in ((np.complex128, 1e-10), (np.complex64, 1e-5)):
        fi = pf.far_field_ifgf(cu(sig, dt), torch.from_numpy(xh).cuda()).cpu().numpy()
        check(fi, fi_ref, tol, "IFGF far field")
    ff = oracle_lib.far_field(s.points, s.normals, s.weights, K, K, sig, xh)
    assert rel(fi_ref, ff) < 1e-4
    assert pf.missed_lookups() == 0
    pf.close()
    # targets: between the spheres and beside the small one (inside the root box)
    tg = np.concatenate([np.array([[1.3, 0.0, 0.0], [1.6, 0.3, 0.0], [1.6, 0.0, -0.25]]),
                         np.array([1.6, 0.0, 0.0]) + 0.2 * xh[:40]])
    M = tg.shape[0]
    pt = B.Plan.with_targets(s.points, s.normals, s.weights, tg, B.Params(k=K, **kw))
    xa = np.concatenate([s.points, tg])
    na = np.concatenate([s.normals, np.zeros_like(tg)])
    wa = np.concatenate([s.weights, np.zeros(M)])
    sa = np.concatenate([sig, np.zeros((2, M), complex)], axis=1)
    ya, info = oracle_lib.ifgf(xa, na, wa, oracle_lib.IFGFParams(k=K, identity_coef=0.5, **kw), sa)
    assert info["D"] == pt.info()["D"]
    for dt, tol in ((np.complex128, 1e-10), (np.complex64, 1e-5)):
        y = pt.field_ifgf(cu(sig, dt))
        torch.cuda.synchronize()
        check(y.cpu().numpy(), ya[:, s.N:], tol, str(dt))
    direct = oracle_lib.field(s.points, s.normals, s.weights, K, K, sig, tg)
    assert rel(ya[:, s.N:], direct) < 2e-4
    assert pt.missed_lookups() == 0
    pt.close()


ADJ_CASES = {
    "leaf64_3x5": (dict(levels=6, leaf_max=64), None),
    "leaf64_5x8_tc": (dict(levels=6, leaf_max=64, Ps=5, Pang=8), 0.0),
    "leaf16_D7_split": (dict(levels=7, leaf_max=16, factor_mode=2), None),
}


@pytest.mark.parametrize("case", list(ADJ_CASES))
def test_adaptive_adjoint(B, geo, case):
    """The adjoint of an adaptive plan (anterpolation at every level, the transposed leaf evaluation
    at every level's leaves, the transposed near field on the adaptive near lists): the FP64 adjoint
    satisfies <A s, g> = <s, A^H g> to rounding (A is parity-checked against the oracle above), the
    mixed adjoint matches it to 1e-5, the vector-Jacobian product without the k-derivative equals the
    adjoint, and its k-derivative Re <g, dA/dk s> (coarse leaves included) matches a central
    difference of Re <g, A(k) s> over plans at k +- h with the same tree and eta (FP64 to 1e-6, the
    mixed one to 1e-4)."""
    kw, fill = ADJ_CASES[case]
    s = geo
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=K, **kw))
    if fill is not None:
        plan.set_tc_fill(fill)
    sig = random_density(s.N, 2, 78)
    g = random_density(s.N, 2, 79)
    As = apply(plan, sig, np.complex128)
    Ahg = plan.adjoint(cu(g)).cpu().numpy()
    lhs, rhs = np.vdot(g, As), np.vdot(Ahg, sig)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs), (lhs, rhs)
    Ahg32 = plan.adjoint(cu(g, np.complex64)).cpu().numpy()
    check(Ahg32, Ahg, 1e-5, "mixed adjoint")
    gs, dk0 = plan.vjp(cu(sig), cu(g), with_dk=False)
    check(gs.cpu().numpy(), Ahg, 1e-13, "vjp without dk")
    assert dk0 == 0.0
    gs, dk = plan.vjp(cu(sig), cu(g))
    check(gs.cpu().numpy(), Ahg, 1e-13, "vjp")
    _, dk32 = plan.vjp(cu(sig, np.complex64), cu(g, np.complex64))
    h = 1e-4
    pp = B.Plan(s.points, s.normals, s.weights, B.Params(k=K + h, eta=K, **kw))
    pm = B.Plan(s.points, s.normals, s.weights, B.Params(k=K - h, eta=K, **kw))
    fd = (np.vdot(g, apply(pp, sig, np.complex128)).real - np.vdot(g, apply(pm, sig, np.complex128)).real) / (2 * h)
    assert abs(dk - fd) <= 1e-6 * abs(fd), (dk, fd)
    assert abs(dk32 - dk) <= 1e-4 * abs(dk), (dk32, dk)
    assert plan.missed_lookups() == 0
    for q in (plan, pp, pm):
        q.close()


def test_adaptive_autograd_density_gradient(B, geo):
    """torch autograd through an adaptive plan: the gradient in the density (no k-gradient asked)
    equals A^H of the output gradient."""
    from paper_2112_06316_gb300 import ifgf_apply

    s = geo
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=K, levels=6, leaf_max=64))
    sig = cu(random_density(s.N, 1, 80)[0]).requires_grad_(True)
    w = cu(random_density(s.N, 1, 81)[0])
    k = torch.tensor(K, dtype=torch.float64)
    y = ifgf_apply(sig, k, plan)
    (y * w.conj()).real.sum().backward()
    ref = plan.adjoint(w).cpu().numpy()
    check(sig.grad.cpu().numpy(), ref, 1e-12, "density gradient")
    plan.close()
