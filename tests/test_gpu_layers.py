"""GPU: the single-layer and double-layer operators alone (ifgf_params.layer).

The plan's kernel is the combined field dPhi/dnu - i eta Phi (layer 0, Eq. CombinedLayer), the
double layer dPhi/dnu alone (layer 1) or the single layer Phi alone (layer 2).  Every evaluation of
the plan follows it.  Checked against the oracle's IFGF with the same layer, element by element
(FP64 <= 1e-10, mixed <= 1e-5), and against the oracle's direct sums of that layer:

* apply on the 1-wavelength sphere (D = 3, orders (3,5)), a 4-wavelength sphere (D = 4, split and
  combined factors) and the tcgen05 propagation path (orders (5,8), every level on the tensor cores);
* the double layer equals the combined field at eta = 0 bit for bit;
* adjoint: <A s, g> = <s, A^H g> and the oracle's direct adjoint on sampled rows;
* k-gradient of the single layer against central differences;
* off-surface potential and far field (direct), and the far field from the level-3 interpolants.
"""
import math

import numpy as np
import pytest

from parity import check, rel
from workloads import cube_sphere, random_density, sphere_workload

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


def cu(a, dt=np.complex128):
    return torch.from_numpy(np.ascontiguousarray(a.astype(dt))).cuda()


def apply(plan, sig, dt):
    y = plan.apply(cu(sig, dt))
    torch.cuda.synchronize()
    return y.cpu().numpy()


CASES = {
    "sphere1_D3_3x5": (lambda: (cube_sphere(26), math.pi), dict(levels=3), None),
    "sphere4_D4_split": (lambda: sphere_workload(48, 6, 4.0), dict(levels=4, factor_mode=2), None),
    "sphere4_D4_combined": (lambda: sphere_workload(48, 6, 4.0), dict(levels=4, factor_mode=1), None),
    "sphere4_D5_5x8_tc": (lambda: sphere_workload(48, 6, 4.0), dict(levels=5, Ps=5, Pang=8), 0.0),
}


@pytest.mark.parametrize("layer", [1, 2])
@pytest.mark.parametrize("case", list(CASES))
def test_layer_apply_vs_oracle(B, oracle_lib, case, layer):
    geo, kw, fill = CASES[case]
    s, k = geo()
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, layer=layer, **kw))
    if fill is not None:
        plan.set_tc_fill(fill)
    sig = random_density(s.N, 2, 51)
    ref, oinfo = oracle_lib.ifgf(s.points, s.normals, s.weights,
                                 oracle_lib.IFGFParams(k=k, identity_coef=0.5, layer=layer, **kw), sig)
    y64 = apply(plan, sig, np.complex128)
    y32 = apply(plan, sig, np.complex64)
    assert plan.missed_lookups() == 0 and plan.info()["D"] == oinfo["D"]
    check(y64, ref, 1e-10, "fp64")
    check(y32, ref, 1e-5, "mixed")
    rows = np.random.default_rng(52).choice(s.N, 200, replace=False)
    yd = oracle_lib.direct(s.points, s.normals, s.weights, k, k, sig, cI=0.5, rows=rows, layer=layer)
    assert rel(y64[:, rows], yd) < (5e-3 if kw.get("Ps", 3) == 3 else 1e-4)
    plan.close()


def test_double_layer_is_combined_field_at_eta_zero(B):
    s, k = sphere_workload(32, 8, 3.0)
    pd = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, levels=4, layer=1))
    p0 = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, eta=0.0, levels=4))
    sig = random_density(s.N, 1, 53)
    for dt in (np.complex128, np.complex64):
        assert np.array_equal(apply(pd, sig, dt), apply(p0, sig, dt))
    pd.close()
    p0.close()


@pytest.mark.parametrize("layer", [1, 2])
def test_layer_adjoint(B, oracle_lib, layer):
    s, k = sphere_workload(48, 6, 4.0)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, levels=4, layer=layer))
    sig = random_density(s.N, 2, 54)
    g = random_density(s.N, 2, 55)
    As = plan.apply(cu(sig)).cpu().numpy()
    Ahg = plan.adjoint(cu(g)).cpu().numpy()
    assert abs(np.vdot(g, As) - np.vdot(Ahg, sig)) <= 1e-12 * abs(np.vdot(g, As))
    Ahg32 = plan.adjoint(cu(g, np.complex64)).cpu().numpy()
    check(Ahg32, Ahg, 1e-5, "mixed adjoint")
    rows = np.random.default_rng(56).choice(s.N, 100, replace=False)
    ref = oracle_lib.direct_adjoint(s.points, s.normals, s.weights, k, k, g, cI=0.5, rows=rows, layer=layer)
    assert rel(Ahg[:, rows], ref) < 5e-3
    plan.close()


def test_single_layer_k_gradient(B):
    from paper_2112_06316_gb300 import ifgf_apply

    s, k0 = sphere_workload(48, 6, 4.0)
    kw = dict(levels=4, layer=2)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k0, **kw))
    sig = torch.from_numpy(random_density(s.N, 1, 57)[0]).cuda()
    b = torch.from_numpy(random_density(s.N, 1, 58)[0]).cuda()
    k = torch.tensor(k0, dtype=torch.float64, requires_grad=True)
    y = ifgf_apply(sig, k, plan)
    ((y - b).abs() ** 2).sum().backward()
    h = 1e-4
    pp = B.Plan(s.points, s.normals, s.weights, B.Params(k=k0 + h, **kw))
    pm = B.Plan(s.points, s.normals, s.weights, B.Params(k=k0 - h, **kw))

    def loss(p):
        return float(((p.apply(sig) - b).abs() ** 2).sum().item())

    with torch.no_grad():
        fd = (loss(pp) - loss(pm)) / (2 * h)
    assert abs(fd - float(k.grad)) <= 1e-6 * abs(fd), (fd, float(k.grad))
    for p in (plan, pp, pm):
        p.close()


@pytest.mark.parametrize("layer", [1, 2])
def test_layer_off_surface(B, oracle_lib, layer):
    s, k = sphere_workload(32, 8, 3.0)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, levels=4, layer=layer, far_field=1))
    sig = random_density(s.N, 2, 59)
    rng = np.random.default_rng(60)
    xh = rng.normal(size=(257, 3))
    xh /= np.linalg.norm(xh, axis=1)[:, None]
    tg = xh * 1.7
    ff_ref = oracle_lib.far_field(s.points, s.normals, s.weights, k, k, sig, xh, layer=layer)
    nf_ref = oracle_lib.field(s.points, s.normals, s.weights, k, k, sig, tg, layer=layer)
    for dt, tol in ((np.complex128, 1e-12), (np.complex64, 1e-5)):
        ff = plan.far_field(cu(sig, dt), torch.from_numpy(xh).cuda()).cpu().numpy()
        nf = plan.field(cu(sig, dt), torch.from_numpy(tg).cuda()).cpu().numpy()
        check(ff, ff_ref, tol, "far field")
        check(nf, nf_ref, tol, "potential")
    fi_ref, _ = oracle_lib.ifgf_far_field(s.points, s.normals, s.weights,
                                          oracle_lib.IFGFParams(k=k, levels=4, layer=layer), sig, xh)
    for dt, tol in ((np.complex128, 1e-10), (np.complex64, 1e-5)):
        fi = plan.far_field_ifgf(cu(sig, dt), torch.from_numpy(xh).cuda()).cpu().numpy()
        check(fi, fi_ref, tol, "IFGF far field")
    assert rel(fi_ref, ff_ref) < 1e-2  # orders (3, 5): the IFGF error of an apply, a few 1e-3
    assert plan.missed_lookups() == 0
    plan.close()
