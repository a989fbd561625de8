"""CPU tests of the C-ABI library: symbol exports, argument validation and the
host plan (octree, cousins, relevant cone segments) against the oracle's counts.
No GPU is touched: plans are built with ifgf_plan_dry_run."""
import math
import os
import re

import numpy as np
import pytest

from workloads import cube_sphere, ellipsoid, random_density, sphere_workload, two_spheres

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2112_06316_gb300 import binding
    from paper_2112_06316_gb300 import build as _b

    _b.build()
    return binding


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ifgf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ifgf_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(B):
    import ctypes

    lib = ctypes.CDLL(B.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    # and the binding wraps each of them
    assert set(names) <= set(B.exported_symbols()), set(names) - set(B.exported_symbols())


def _sphere():
    s = cube_sphere(26)
    return s, math.pi


def test_validation_errors(B):
    s, k = _sphere()
    x, n, w = s.points, s.normals, s.weights
    with pytest.raises(B.IFGFError, match="EINVAL"):
        B.dry_run(x[:0], n[:0], w[:0], B.Params(k=k))
    bad = x.copy()
    bad[3, 1] = np.nan
    with pytest.raises(B.IFGFError, match="EINVAL"):
        B.dry_run(bad, n, w, B.Params(k=k))
    nb = n.copy()
    nb[7] *= 1.01
    with pytest.raises(B.IFGFError, match="not unit"):
        B.dry_run(x, nb, w, B.Params(k=k))
    wb = w.copy()
    wb[0] = 0.0
    with pytest.raises(B.IFGFError, match="weight"):
        B.dry_run(x, n, wb, B.Params(k=k))
    with pytest.raises(B.IFGFError, match="EINVAL"):
        B.dry_run(x, n, w, B.Params(k=-1.0))
    with pytest.raises(B.IFGFError, match="EINVAL"):
        B.dry_run(x, n, w, B.Params(k=k, levels=2))
    with pytest.raises(B.IFGFError, match="EUNSUPPORTED"):
        B.dry_run(x, n, w, B.Params(k=k, Ps=2, Pang=2))


@pytest.mark.parametrize("case", ["sphere1", "sphere4", "ellipsoid", "cloud"])
def test_plan_counts_match_oracle(B, oracle_lib, case):
    rng = np.random.default_rng(1)
    if case == "sphere1":
        s, k = _sphere()
        x, n, w, D = s.points, s.normals, s.weights, 3
    elif case == "sphere4":
        s, k = sphere_workload(48, 6, 4.0)
        x, n, w, D = s.points, s.normals, s.weights, 4
    elif case == "ellipsoid":
        s = ellipsoid(32, 8, (1.0, 2.0, 3.0))
        k, x, n, w, D = 6.0, s.points, s.normals, s.weights, 5
    else:  # clustered random cloud with random unit normals
        x = np.concatenate([rng.normal(size=(1500, 3)) * 0.1, rng.uniform(-1, 1, (1500, 3))])
        n = rng.normal(size=x.shape)
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        w = rng.uniform(0.5, 1.5, x.shape[0])
        k, D = 9.0, 5
    for fm, cr in ((0, 0), (1, 1), (2, 0)):
        sig = random_density(x.shape[0], 1, 0)
        _, oi = oracle_lib.ifgf(x, n, w, oracle_lib.IFGFParams(k=k, levels=D, factor_mode=fm, cone_rule=cr), sig)
        pi = B.dry_run(x, n, w, B.Params(k=k, levels=D, factor_mode=fm, cone_rule=cr, cone_band=0.0))
        for key in ("nbox", "ns", "nC", "split", "nrc", "cousin_evals", "prop_evals"):
            assert pi[key][3:] == oi[key][3:], (case, key, pi[key], oi[key])
        assert pi["leaf_evals"] == oi["leaf_evals"]
        assert pi["near_pairs"] == oi["near_pairs"] + x.shape[0]  # the plan counts the l == m slots
        assert abs(pi["root_side"] - oi["root_side"]) == 0.0
        # the default band only adds cone segments
        pb = B.dry_run(x, n, w, B.Params(k=k, levels=D, factor_mode=fm, cone_rule=cr))
        assert all(a >= b for a, b in zip(pb["nrc"], pi["nrc"]))


def test_auto_levels_match_oracle_rule(B, oracle_lib):
    for n, m, wl in ((26, 26, 1.0), (48, 6, 4.0), (96, 8, 8.0), (64, 8, 2.0)):
        s, k = sphere_workload(n, m, wl)
        pi = B.dry_run(s.points, s.normals, s.weights, B.Params(k=k))
        assert pi["D"] == oracle_lib.auto_levels(s.points)


def test_entry_points_reject_a_null_plan_without_a_gpu(B):
    """Every call that takes a plan checks it before any device work: a null plan gives
    IFGF_EINVAL and a message, on a machine without a GPU too."""
    import ctypes

    lib = B.lib()
    dk = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    info = B.CInfo()
    calls = {
        "ifgf_apply": lambda: lib.ifgf_apply(None, None, None, 1, B.MIXED, None),
        "ifgf_apply_adjoint": lambda: lib.ifgf_apply_adjoint(None, None, None, 1, B.MIXED, None),
        "ifgf_apply_vjp": lambda: lib.ifgf_apply_vjp(None, None, None, None, 1, ctypes.byref(dk), B.MIXED, None),
        "ifgf_apply_noalloc": lambda: lib.ifgf_apply_noalloc(None, None, None, 1, B.MIXED, None),
        "ifgf_field": lambda: lib.ifgf_field(None, None, None, ctypes.c_int64(4), None, 1, B.MIXED, None),
        "ifgf_far_field": lambda: lib.ifgf_far_field(None, None, None, ctypes.c_int64(4), None, 1, B.MIXED, None),
        "ifgf_gmres": lambda: lib.ifgf_gmres(None, None, None, 10, 10, 1e-6, B.FP64, ctypes.byref(it), None, None),
        "ifgf_plan_info": lambda: lib.ifgf_plan_info(None, ctypes.byref(info)),
        "ifgf_plan_set_correction": lambda: lib.ifgf_plan_set_correction(None, None, None, None, ctypes.c_int64(0)),
    }
    for name, call in calls.items():
        assert call() == -1, name
        assert lib.ifgf_last_error(), name
    lib.ifgf_plan_destroy(None)  # a no-op


@pytest.mark.parametrize("case", ["two_spheres", "two_spheres_5x8", "ellipsoid_3to1", "cloud"])
def test_adaptive_plan_counts_match_oracle(B, oracle_lib, case):
    """Adaptive octree (leaf_max > 0): the library's planner builds the oracle's tree (boxes, cone grids,
    relevant cones, cousin and propagation evaluations, leaf evaluations at every level's leaves, and
    the near pairs of the coarser-leaf-level rule), without a GPU."""
    rng = np.random.default_rng(2)
    kw = {}
    if case.startswith("two_spheres"):
        s = two_spheres()
        x, n, w, k, D, lm = s.points, s.normals, s.weights, 2 * np.pi, 6, 64
        if case.endswith("5x8"):
            kw = dict(Ps=5, Pang=8)
    elif case == "ellipsoid_3to1":
        s = ellipsoid(32, 8, (1.0, 1.0, 3.0))
        x, n, w, k, D, lm = s.points, s.normals, s.weights, 2 * np.pi, 6, 32
    else:  # a dense cluster inside a sparse cloud, random unit normals
        x = np.concatenate([rng.normal(size=(2000, 3)) * 0.05, rng.uniform(-1, 1, (1000, 3))])
        n = rng.normal(size=x.shape)
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        w = rng.uniform(0.5, 1.5, x.shape[0])
        k, D, lm = 9.0, 7, 16
    sig = random_density(x.shape[0], 1, 0)
    _, oi = oracle_lib.ifgf(x, n, w, oracle_lib.IFGFParams(k=k, levels=D, leaf_max=lm, **kw), sig)
    pi = B.dry_run(x, n, w, B.Params(k=k, levels=D, leaf_max=lm, cone_band=0.0, **kw))
    for key in ("nbox", "ns", "nC", "split", "nrc", "cousin_evals", "prop_evals"):
        assert pi[key][3:] == oi[key][3:], (case, key, pi[key], oi[key])
    assert pi["leaf_evals"] == oi["leaf_evals"]
    assert pi["near_pairs"] == oi["near_pairs"] + x.shape[0]
    # fewer relevant cones than the uniform tree of the same depth
    pu = B.dry_run(x, n, w, B.Params(k=k, levels=D, cone_band=0.0, **kw))
    assert sum(pi["nrc"]) < sum(pu["nrc"])
