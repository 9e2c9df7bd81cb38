"""GPU test of the allocation-free split-precision product.

zt_zgemm_skew_split_noalloc serves callers that cannot call cudaMalloc: a
serving process that reserved the device memory for resident simulation state
at start-up, a host application whose own allocator owns the device, or a
time-critical loop that must not pay the device synchronisation of an
allocation.  It keeps its scratch in a static device array instead.  Here it
is called through the C ABI twice in a row (a larger N first, then a smaller
one, so that leftovers of the first call would show up in the second), and
each result is compared with the plan-based split product, zt_zgemm_skew on a
ZT_PRECISION_SPLIT plan, at the 1e-12 relative tolerance of the split-product
tests.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2206_05466_gb300.inputs import vorticity_w0

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2206_05466_gb300 import zeitlin as z  # noqa: E402

MAX_N = 256


def _noalloc():
    L = z.load()
    f = L.zt_zgemm_skew_split_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _inputs(N, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    Y = vorticity_w0(N, seed=seed + 1)
    return (torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())


def _plan_product(N, Xd, Yd):
    plan = z.Plan(N, z.PRECISION_SPLIT)
    Cd = torch.empty_like(Xd)
    z.zt_zgemm_skew(plan, Xd, Yd, Cd)
    torch.cuda.synchronize()
    out = Cd.cpu().numpy()
    plan.close()
    return out


def test_noalloc_matches_plan_product_on_consecutive_calls():
    f = _noalloc()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for N, seed in ((MAX_N, 11), (97, 12)):
        Xd, Yd = _inputs(N, seed)
        Cd = torch.full((N, N), float("nan"), dtype=torch.complex128, device="cuda")
        rc = f(N, ctypes.c_void_p(Xd.data_ptr()), ctypes.c_void_p(Yd.data_ptr()), ctypes.c_void_p(Cd.data_ptr()),
               stream)
        assert rc == z.ZT_OK, z.load().zt_last_error().decode()
        got = Cd.cpu().numpy()
        want = _plan_product(N, Xd, Yd)
        assert _rel(got, want) < 1e-12, (N, _rel(got, want))
        assert _rel(got, Xd.cpu().numpy() @ Yd.cpu().numpy()) < 1e-12


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    f = _noalloc()
    N = MAX_N + 1
    Xd, Yd = _inputs(N, 3)
    Cd = torch.empty_like(Xd)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = f(N, ctypes.c_void_p(Xd.data_ptr()), ctypes.c_void_p(Yd.data_ptr()), ctypes.c_void_p(Cd.data_ptr()), stream)
    assert rc == z.ZT_EINVAL
    assert b"static scratch" in z.load().zt_last_error()
