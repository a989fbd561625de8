"""The allocation-free apply (ifgf_apply_noalloc) against the ordinary apply.

Some callers cannot call cudaMalloc when they apply the operator: their device
memory is reserved up front by the host application (or a pool that must not be
bypassed), or they run on a path where the implicit device synchronisation of
cudaMalloc/cudaFree would stall other work.  ifgf_apply_noalloc serves them by
keeping the apply's workspace in a fixed device array inside the library.  This
test calls it through the C ABI twice in a row for each precision and checks
its output against ifgf_apply's, and checks that a request whose workspace is
larger than the fixed array is refused with a clear error.
"""
import ctypes
import math

import numpy as np
import pytest

from workloads import cube_sphere, random_density

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


@pytest.mark.parametrize("prec,dtype,tol", [(0, np.complex128, 1e-10), (1, np.complex64, 1e-5)])
def test_noalloc_matches_apply(B, prec, dtype, tol):
    s = cube_sphere(26)  # unit sphere, N = 4,056, one wavelength across
    k = math.pi
    plan = B.Plan(s.points, s.normals, s.weights, B.Params(k=k, levels=3))
    sig = torch.from_numpy(random_density(s.N, 2, 1).astype(dtype)).cuda()
    ref = plan.apply(sig)
    for _ in range(2):  # two calls in a row share (and overwrite) the fixed array
        out = torch.full_like(sig, complex("nan"))
        st = _noalloc(B, plan, sig, out, prec)
        assert st == 0, B.lib().ifgf_last_error().decode()
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), ref.cpu().numpy()) <= tol
    assert plan.missed_lookups() == 0
    plan.close()


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
