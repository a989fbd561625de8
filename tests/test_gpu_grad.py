"""Hand-written backward through torch.autograd: gradients of L = |A(k) sigma - b|^2
with respect to the density sigma and the wavenumber k, checked against central
finite differences (step 1e-4) on the FP64 form with the plan structure frozen
(eta held fixed; the plans at k +- h have the same octree and cone segments)."""
import math

import numpy as np
import pytest

from workloads import random_density, sphere_workload

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


def loss_of(plan, sig, b):
    y = plan.apply(sig)
    return float(((y - b).abs() ** 2).sum().item())


@pytest.mark.parametrize("fm", [0, 1, 2])
def test_grad_sigma_and_k_vs_finite_differences(B, fm):
    from paper_2112_06316_gb300 import ifgf_apply

    s, k0 = sphere_workload(48, 6, 4.0)  # N = 13,824, D = 4
    eta = k0
    kw = dict(eta=eta, levels=4, factor_mode=fm)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k0, **kw))
    sig = torch.from_numpy(random_density(s.N, 1, 1)[0]).cuda().requires_grad_(True)
    b = torch.from_numpy(random_density(s.N, 1, 2)[0]).cuda()
    k = torch.tensor(k0, dtype=torch.float64, requires_grad=True)
    y = ifgf_apply(sig, k, plan)
    L = ((y - b).abs() ** 2).sum()
    L.backward()
    gs, gk = sig.grad.detach(), float(k.grad)
    # density direction (L is quadratic in sigma: central differences are exact up to rounding)
    d = torch.from_numpy(random_density(s.N, 1, 3)[0]).cuda()
    eps = 1e-4
    with torch.no_grad():
        fd = (loss_of(plan, sig + eps * d, b) - loss_of(plan, sig - eps * d, b)) / (2 * eps)
    an = float(torch.real(torch.vdot(gs, d)).item())
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
    # wavenumber
    h = 1e-4
    pp = B.Plan(s.points, s.normals, s.weights, B.Params(k=k0 + h, **kw))
    pm = B.Plan(s.points, s.normals, s.weights, B.Params(k=k0 - h, **kw))
    assert pp.info()["nrc"] == plan.info()["nrc"] == pm.info()["nrc"]
    with torch.no_grad():
        fdk = (loss_of(pp, sig, b) - loss_of(pm, sig, b)) / (2 * h)
    assert abs(fdk - gk) <= 1e-6 * abs(gk), (fdk, gk)


@pytest.mark.parametrize("orders", [(3, 5), (5, 8)])
def test_vjp_density_part_is_the_adjoint(B, orders):
    s, k = sphere_workload(32, 8, 3.0)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, Ps=orders[0], Pang=orders[1]))
    sig = torch.from_numpy(random_density(s.N, 2, 4)).cuda()
    g = torch.from_numpy(random_density(s.N, 2, 5)).cuda()
    gs, dk = plan.vjp(sig, g)
    assert torch.allclose(gs, plan.adjoint(g), rtol=0, atol=0)
    gs32, dk32 = plan.vjp(sig.to(torch.complex64), g.to(torch.complex64))
    assert abs(dk32 - dk) <= 1e-4 * abs(dk)


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
def test_vjp_from_saved_forward_state(B, dtype):
    """ifgf_apply_ws leaves the forward state in a caller-owned workspace; ifgf_apply_vjp_ws
    on it gives the same gradient and k-derivative as ifgf_apply_vjp (which re-runs the
    forward apply), bit for bit, even after other applies of the plan -- the autograd
    backward therefore needs no second forward apply.  A workspace that is too small is
    refused."""
    s, k = sphere_workload(32, 8, 3.0)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, Ps=5, Pang=8, levels=4))
    plan.set_tc_fill(0.0)
    sig = torch.from_numpy(random_density(s.N, 2, 6).astype(dtype)).cuda()
    g = torch.from_numpy(random_density(s.N, 2, 7).astype(dtype)).cuda()
    y_ref = plan.apply(sig).clone()
    y, state = plan.apply_with_state(sig)
    torch.cuda.synchronize()
    assert torch.equal(y, y_ref)
    gs_ref, dk_ref = plan.vjp(sig, g)
    plan.apply(torch.from_numpy(random_density(s.N, 2, 8).astype(dtype)).cuda())  # other state in the plan
    gs, dk = plan.vjp_from_state(state, g)
    assert torch.equal(gs, gs_ref)
    assert dk == dk_ref
    with pytest.raises(B.IFGFError):
        plan.vjp_from_state(state[: state.numel() // 2], g)
    plan.close()
