"""The allocation-free apply (ifgf_apply_noalloc) against the ordinary apply.

Some callers cannot call cudaMalloc when they apply the operator: their device
memory is reserved up front by the host application (or a pool that must not be
bypassed), or they run on a path where the implicit device synchronisation of
cudaMalloc/cudaFree would stall other work.  ifgf_apply_noalloc serves them by
keeping the apply's workspace in a fixed device array inside the library.

These tests call it through the C ABI and check its output against ifgf_apply's:
* twice in a row on one plan, for each precision;
* after a call on a different, deeper plan with another density (so that the
  shared array holds stale propagation values and cone values of another
  layout), on a plan with propagation on the tensor cores and a sparse
  correction -- the result must equal ifgf_apply bit for bit, and ifgf_apply on
  the plan's own workspace must still give the same result afterwards;
* a request whose workspace is larger than the fixed array is refused with a
  clear error.
"""
import ctypes
import math

import numpy as np
import pytest

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


def _noalloc(B, plan, sig, out, prec):
    stream = torch.cuda.current_stream().cuda_stream
    return B.lib().ifgf_apply_noalloc(plan.handle, ctypes.c_void_p(sig.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_int(sig.shape[0]), ctypes.c_int(prec), ctypes.c_void_p(stream))


def _run_noalloc(B, plan, sig, prec):
    out = torch.full_like(sig, complex("nan"))
    st = _noalloc(B, plan, sig, out, prec)
    assert st == 0, B.lib().ifgf_last_error().decode()
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("prec,dtype,tol", [(0, np.complex128, 1e-10), (1, np.complex64, 1e-5)])
def test_noalloc_matches_apply(B, prec, dtype, tol):
    s = cube_sphere(26)  # unit sphere, N = 4,056, one wavelength across
    k = math.pi
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, levels=3))
    sig = torch.from_numpy(random_density(s.N, 2, 1).astype(dtype)).cuda()
    ref = plan.apply(sig)
    for _ in range(2):  # two calls in a row share (and overwrite) the fixed array
        out = _run_noalloc(B, plan, sig, prec)
        assert rel(out.cpu().numpy(), ref.cpu().numpy()) <= tol
        assert torch.equal(out, ref)
    assert plan.missed_lookups() == 0
    plan.close()


@pytest.mark.parametrize("prec,dtype", [(0, np.complex128), (1, np.complex64)])
def test_noalloc_after_another_plan(B, prec, dtype):
    # plan A: 4-wavelength sphere, five levels (three propagation steps), orders (5, 8), the
    # combined factor on every level (its FP64 workspace, 57 MiB, fits the 64 MiB array), every
    # propagation level forced onto the tensor cores
    sa, ka = sphere_workload(48, 6, 4.0)
    plan_a = B.Plan(sa.points, sa.normals, sa.weights, B.Params(k=ka, levels=5, Ps=5, Pang=8, factor_mode=1))
    plan_a.set_tc_fill(0.0)
    sig_a = torch.from_numpy(random_density(sa.N, 1, 21).astype(dtype)).cuda()
    # plan B (under test): 3-wavelength sphere, four levels, orders (5, 8), split factors at the
    # leaf level and the combined one above, tensor-core propagation, a sparse correction with
    # empty and full rows, two right-hand sides
    sb, kb = sphere_workload(32, 8, 3.0)
    plan_b = B.Plan(sb.points, sb.normals, sb.weights, B.Params(k=kb, levels=4, Ps=5, Pang=8))
    plan_b.set_tc_fill(0.0)
    rng = np.random.default_rng(22)
    counts = rng.integers(0, 30, sb.N)
    counts[::5] = 0
    rowptr = np.concatenate([[0], np.cumsum(counts)])
    col = rng.integers(0, sb.N, rowptr[-1]).astype(np.int32)
    val = (rng.normal(size=rowptr[-1]) + 1j * rng.normal(size=rowptr[-1])) * 1e-2
    plan_b.set_correction(rowptr, col, val)
    sig_b = torch.from_numpy(random_density(sb.N, 2, 23).astype(dtype)).cuda()

    ref_b = plan_b.apply(sig_b).clone()
    ref_a = plan_a.apply(sig_a).clone()
    torch.cuda.synchronize()
    out_a = _run_noalloc(B, plan_a, sig_a, prec)  # leaves plan A's values in the shared array
    assert torch.equal(out_a, ref_a)
    for _ in range(2):
        out_b = _run_noalloc(B, plan_b, sig_b, prec)
        assert torch.equal(out_b, ref_b)
    # the plan's own workspace is untouched by the allocation-free calls
    again = plan_b.apply(sig_b)
    torch.cuda.synchronize()
    assert torch.equal(again, ref_b)
    assert plan_a.missed_lookups() == 0 and plan_b.missed_lookups() == 0
    plan_a.close()
    plan_b.close()


def test_noalloc_rejects_oversized_workspace(B):
    s = cube_sphere(26)
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=math.pi, levels=3))
    nrhs = 2048  # w*sigma and u alone need 2 x 2048 x 4056 x 16 B = 266 MB > 64 MiB
    sig = torch.zeros((nrhs, s.N), dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(sig)
    st = _noalloc(B, plan, sig, out, 0)
    assert st == -1  # IFGF_EINVAL
    msg = B.lib().ifgf_last_error().decode()
    assert "exceeds" in msg and "scratch" in msg
    plan.close()
