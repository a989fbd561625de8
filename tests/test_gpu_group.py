"""Batched apply of many scatterers as one CUDA graph (ifgf_group_*): equal to the
per-plan applies bit for bit (output-stationary kernels), replayable, re-captured
when buffers change; autotuned; each body checked against the oracle."""
import math

import numpy as np
import pytest

from parity import check
from workloads import random_density, scatterer_batch, sphere_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_06316_gb300 import binding
    from paper_2112_06316_gb300 import build as _b

    _b.build()
    return binding


def make(B, bodies, nrhs, dtype, seed0=30):
    plans = [B.Plan(s.points, s.normals, s.weights, B.Params(k=k)) for s, k in bodies]
    sig = [torch.from_numpy(random_density(s.N, nrhs, seed0 + i).astype(dtype)).cuda() for i, (s, k) in enumerate(bodies)]
    return plans, sig


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_group_equals_per_plan(B, dtype):
    bodies = scatterer_batch(seed=3, count=6, n_min=16, n_max=40, d_max=6.0)
    plans, sig = make(B, bodies, 4, dtype)
    ref = [p.apply(s) for p, s in zip(plans, sig)]
    g = B.Group(plans, nstreams=3)
    outs = [torch.empty_like(s) for s in sig]
    for _ in range(2):  # capture, then replay
        for o in outs:
            o.fill_(float("nan"))
        g.apply(sig, outs)
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert torch.equal(o, r)
    outs2 = [torch.empty_like(s) for s in sig]  # new buffers -> new capture
    g.apply(sig, outs2)
    torch.cuda.synchronize()
    for o, r in zip(outs2, ref):
        assert torch.equal(o, r)
    g.set_streams(1)
    g.apply(sig, outs2)
    torch.cuda.synchronize()
    for o, r in zip(outs2, ref):
        assert torch.equal(o, r)
    g.close()


def test_group_bodies_vs_oracle_and_autotune(B, oracle_lib, tmp_path):
    from paper_2112_06316_gb300.autotune import Autotuner, gpu_timer, tune_key

    bodies = scatterer_batch(seed=5, count=4, n_min=16, n_max=32, d_max=5.0)
    plans, sig = make(B, bodies, 2, np.complex128)
    g = B.Group(plans)
    outs = [torch.empty_like(s) for s in sig]
    g.apply(sig, outs)
    torch.cuda.synchronize()
    for (s, k), o, sg in zip(bodies, outs, sig):
        ref, _ = oracle_lib.ifgf(s.points, s.normals, s.weights, oracle_lib.IFGFParams(k=k, identity_coef=0.5),
                                 sg.cpu().numpy())
        assert np.linalg.norm(o.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-10
    tuner = Autotuner(str(tmp_path / "tune.json"))
    key = tune_key(torch.cuda.get_device_name(), "fp64", sum(s.N for s, _ in bodies), 2)
    r = tuner.tune(key, gpu_timer(g, plans, sig, outs), reps=2)
    assert r.config in [c for c, _ in r.table]
    # the tuned configuration still gives identical results
    g.set_streams(r.config["nstreams"])
    for p in plans:
        p.set_rhs_block(r.config["rhs_block"])
    g.apply(sig, outs)
    torch.cuda.synchronize()
    for o, p, s in zip(outs, plans, sig):
        assert torch.equal(o, p.apply(s))


@pytest.mark.slow
def test_config3_full_batch(B):
    """24 scatterers (spheres and ellipsoids, 2-24 wavelengths, 24k-393k points), 4 complex64
    right-hand sides each, one captured graph; equal to the per-plan applies."""
    bodies = scatterer_batch(seed=3)
    plans, sig = make(B, bodies, 4, np.complex64)
    g = B.Group(plans)
    outs = [torch.empty_like(s) for s in sig]
    g.apply(sig, outs)
    torch.cuda.synchronize()
    for o, p, s in zip(outs, plans, sig):
        assert torch.equal(o, p.apply(s))
    assert all(p.missed_lookups() == 0 for p in plans)


def test_group_recaptures_on_kernel_settings(B):
    """The per-plan settings that choose kernels (right-hand-side blocking, tensor-core fill
    threshold and engine) are baked into a captured graph: changing one must trigger a new
    capture, and the replayed result must equal a per-plan apply under the new setting."""
    bodies = scatterer_batch(seed=5, count=3, n_min=24, n_max=40, d_max=5.0)
    plans = [B.Plan(s.points, s.normals, s.weights, B.Params(k=k, Ps=5, Pang=8)) for s, k in bodies]
    sig = [torch.from_numpy(random_density(s.N, 4, 50 + i).astype(np.complex64)).cuda()
           for i, (s, k) in enumerate(bodies)]
    g = B.Group(plans, nstreams=2)
    outs = [torch.empty_like(s) for s in sig]

    def run_and_compare():
        g.apply(sig, outs)
        torch.cuda.synchronize()
        for p, s, o in zip(plans, sig, outs):
            assert torch.equal(o, p.apply(s))

    run_and_compare()
    assert g.captures() == 1
    run_and_compare()  # replay
    assert g.captures() == 1
    # each step changes one plan's setting away from its current value
    changes = [(0, lambda p: p.set_rhs_block(1)), (1, lambda p: p.set_tc_fill(0.0)),
               (2, lambda p: p.set_tc_engine(0)), (1, lambda p: p.set_tc_fill(2.0)),
               (0, lambda p: p.set_rhs_block(4))]
    for i, (j, change) in enumerate(changes):
        change(plans[j])
        run_and_compare()
        assert g.captures() == 2 + i
    plans[0].set_rhs_block(4)  # unchanged value: the graph stays
    run_and_compare()
    assert g.captures() == 1 + len(changes)
    g.close()


def test_tune_plan_kernel_choices(B, oracle_lib, tmp_path):
    """tune_plan times the plan's kernel choices (tensor-core fill threshold and engine, interpolation
    engine), caches the fastest and leaves the plan configured with it; the tuned apply still matches
    the oracle element by element, and a second tuner reads the cache without timing."""
    from paper_2112_06316_gb300.autotune import Autotuner, PLAN_CANDIDATES, tune_plan

    s, k = sphere_workload(48, 6, 4.0)
    kw = dict(levels=5, Ps=5, Pang=8)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, **kw))
    sig = random_density(s.N, 1, 71)
    st = torch.from_numpy(sig.astype(np.complex64)).cuda()
    r = tune_plan(plan, st, Autotuner(str(tmp_path / "t.json")), reps=2)
    assert not r.cached and len(r.table) == len(PLAN_CANDIDATES)
    assert r.ms == min(t for _, t in r.table)
    y = plan.apply(st)
    torch.cuda.synchronize()
    ref, _ = oracle_lib.ifgf(s.points, s.normals, s.weights, oracle_lib.IFGFParams(k=k, identity_coef=0.5, **kw), sig)
    check(y.cpu().numpy(), ref, 1e-5, str(r.config))
    assert plan.missed_lookups() == 0
    r2 = tune_plan(plan, st, Autotuner(str(tmp_path / "t.json")))
    assert r2.cached and r2.config == r.config
    plan.close()
