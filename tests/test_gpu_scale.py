"""GPU: the two largest workloads of the suite, at full size.

* 128-wavelength sphere (k = 128 pi, cube-sphere 6 x 1024 x 1024 with 8 x 8 Fejer
  sub-patches, N = 6,291,456, automatic depth D = 8), orders (3, 5, 5), two complex64
  right-hand sides: mixed apply against the FP64 apply (<= 1e-5) and against direct-sum
  rows (4,000 of them; the accuracy of the orders), then 20 GMRES iterations with FP64 Arnoldi and the
  mixed apply.
* 32-wavelength star-shaped body r = 1 + 0.2 sum a_lm Y_lm (6 x 512 x 512, N = 1,572,864),
  orders (5, 8, 8): mixed forward, gradients of L = |A(k) sigma - b|^2 in sigma and k
  from the hand-written backward against central differences of the FP64 form (step
  1e-4, plan structure frozen), the adjoint against columns of the dense direct-sum
  adjoint, and the adjoint / forward time ratio.
"""
import math

import numpy as np
import pytest

from parity import check
from workloads import random_density, sphere_workload, star_body

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

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


def test_sphere_128_wavelengths(B, oracle_lib):
    s, k = sphere_workload(1024, 8, 128.0)
    assert s.N == 6291456
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k))
    info = plan.info()
    assert info["D"] == 8
    sig = random_density(s.N, 2, 5)
    y32 = plan.apply(torch.from_numpy(sig.astype(np.complex64)).cuda()).cpu().numpy()
    y64 = plan.apply(torch.from_numpy(sig).cuda()).cpu().numpy()
    assert plan.missed_lookups() == 0
    check(y32, y64, 1e-5)
    rows = np.random.default_rng(5).choice(s.N, 4000, replace=False)  # ~1 min of oracle time on 16 cores
    ref = oracle_lib.direct(s.points, s.normals, s.weights, k, k, sig, cI=0.5, rows=rows)
    e64 = rel(y64[:, rows], ref)
    print(f"128-wavelength sphere: IFGF (3,5,5) vs direct rows {e64:.2e}")
    assert e64 < 1e-2, e64  # orders (3, 5, 5): a few 1e-3 on every sphere of the suite
    assert rel(y32[:, rows], ref) < 1.01 * e64 + 1e-5
    # GMRES(20), 20 iterations, plane wave along z (Eq. CombLayIE without the singular correction)
    b = torch.from_numpy(-np.exp(1j * k * s.points[:, 2])).cuda()
    x, conv, its, hist = plan.gmres(b, restart=20, maxit=20, tol=0.0, precision=B.MIXED)
    assert its == 20 and not conv
    h = np.asarray(hist[: its + 1])
    print("GMRES residual history", h)
    assert np.all(np.diff(h) <= 1e-12) and h[-1] < 0.1 * h[0], h
    r = (b - plan.apply(x.to(torch.complex64)).to(torch.complex128)).norm() / b.norm()
    assert abs(float(r) - h[-1]) <= 0.05 * h[-1] + 1e-4, (float(r), h[-1])
    plan.close()


def loss_of(plan, sig, b):
    y = plan.apply(sig)
    return float(((y - b).abs() ** 2).sum().item())


def test_star_body_32_wavelengths_gradients(B, oracle_lib):
    from paper_2112_06316_gb300 import ifgf_apply

    s = star_body(512, 8, 4)
    assert s.N == 1572864
    k0 = 2 * math.pi * 32 / (2 * np.linalg.norm(s.points, axis=1).max())
    kw = dict(eta=k0, Ps=5, Pang=8)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k0, **kw))
    sig_np = random_density(s.N, 1, 41)[0]
    # mixed forward against FP64
    y32 = plan.apply(torch.from_numpy(sig_np.astype(np.complex64)).cuda()).cpu().numpy()
    y64 = plan.apply(torch.from_numpy(sig_np).cuda()).cpu().numpy()
    check(y32, y64, 1e-5)
    # gradients from the hand-written backward (FP64 form)
    sig = torch.from_numpy(sig_np).cuda().requires_grad_(True)
    b = torch.from_numpy(random_density(s.N, 1, 42)[0]).cuda()
    k = torch.tensor(k0, dtype=torch.float64, requires_grad=True)
    L = ((ifgf_apply(sig, k, plan) - b).abs() ** 2).sum()
    L.backward()
    gs, gk = sig.grad.detach(), float(k.grad)
    d = torch.from_numpy(random_density(s.N, 1, 43)[0]).cuda()
    eps = 1e-4
    with torch.no_grad():
        fd = (loss_of(plan, sig + eps * d, b) - loss_of(plan, sig - eps * d, b)) / (2 * eps)
    an = float(torch.real(torch.vdot(gs, d)).item())
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
    h = 1e-4
    pp = B.Plan(s.points, s.normals, s.weights, B.Params(k=k0 + h, **kw))
    pm = B.Plan(s.points, s.normals, s.weights, B.Params(k=k0 - h, **kw))
    assert pp.info()["nrc"] == plan.info()["nrc"] == pm.info()["nrc"]
    with torch.no_grad():
        fdk = (loss_of(pp, sig, b) - loss_of(pm, sig, b)) / (2 * h)
    assert abs(fdk - gk) <= 1e-6 * abs(gk), (fdk, gk)
    pp.close()
    pm.close()
    # adjoint against the dense direct-sum adjoint on sampled columns
    g = random_density(s.N, 1, 44)
    cols = np.random.default_rng(44).choice(s.N, 1024, replace=False)
    ref = oracle_lib.direct_adjoint(s.points, s.normals, s.weights, k0, k0, g, cI=0.5, rows=cols)
    g64 = torch.from_numpy(g).cuda()
    g32 = g64.to(torch.complex64)
    a64 = plan.adjoint(g64).cpu().numpy()
    a32 = plan.adjoint(g32).cpu().numpy()
    e64 = rel(a64[:, cols], ref)
    print(f"star body: adjoint vs dense adjoint columns {e64:.2e}")
    assert e64 < 3e-4  # orders (5, 8, 8) reach ~6e-5 on the spheres; the star body is rougher
    assert rel(a32[:, cols], ref) < 1.01 * e64 + 1e-5
    check(a32, a64, 1e-5)
    assert plan.missed_lookups() == 0
    # adjoint / forward device time (mixed), CUDA events, warm
    s32 = torch.from_numpy(sig_np.astype(np.complex64)).cuda().reshape(1, -1)
    yo, ao = torch.empty_like(s32), torch.empty_like(g32)

    def t(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ratio = t(lambda: plan.adjoint(g32, out=ao)) / t(lambda: plan.apply(s32, out=yo))
    assert ratio <= 2.5, ratio
    plan.close()
