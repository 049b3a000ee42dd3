"""The allocation-free residual entry point, metos3d_residual_static.

Some callers cannot allocate device memory at the moment they need the residual norm
|| a - b ||_2: a process whose device memory is all owned by another allocator with a
fixed budget has none to spare, and a caller without a library context has no
context-owned scratch to use.
metos3d_residual_static keeps its partial sums in a static device array instead.  Here it
is called through the C ABI and compared with the context-based metos3d_residual, within
the tolerance the other reduction tests use, on two calls in a row (the second call must
not see the first call's leftovers).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import m3d_inputs as mi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-13   # relative, as in the residual and mass checks of the parity tests


@pytest.fixture(scope="module")
def m3d():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1410_0204_gb300 as m
    m.load()
    return m


def _static_residual(L, a, b, out, stream):
    return L.metos3d_residual_static(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                     ctypes.c_longlong(a.numel()), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))


def test_static_residual_matches_context_residual_twice(m3d):
    L = m3d.load()
    prob = mi.make_problem("ndop_64x32x8")
    ctx = m3d.Context.from_problem(prob, model=m3d.MODEL_NDOP, ntracer=2, nparam=7)
    stream = torch.cuda.current_stream()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    pairs = [(mi.random_state(prob, seed=1), mi.random_state(prob, seed=2)),
             (mi.random_state(prob, seed=3), mi.random_state(prob, seed=3) * (1 + 1e-3))]
    for a_h, b_h in pairs:
        a = torch.from_numpy(a_h).cuda()
        b = torch.from_numpy(b_h).cuda()
        assert _static_residual(L, a, b, out, stream) == m3d.M3D_OK, L.metos3d_residual_static_error()
        torch.cuda.synchronize()
        got = float(out.item())
        want = ctx.residual(a, b)
        assert abs(got - want) <= TOL * want, (got, want)
        assert abs(got - np.linalg.norm(a_h - b_h)) <= TOL * want
    ctx.close()


def test_static_residual_edge_sizes_and_limit(m3d):
    L = m3d.load()
    stream = torch.cuda.current_stream()
    out = torch.empty((1,), dtype=torch.float64, device="cuda")
    r = np.random.default_rng(5)
    for n in (0, 1, 2047, 2048, 2049, 300001):
        a = torch.from_numpy(r.standard_normal(n)).cuda()
        b = torch.from_numpy(r.standard_normal(n)).cuda()
        assert _static_residual(L, a, b, out, stream) == m3d.M3D_OK
        torch.cuda.synchronize()
        want = float(np.linalg.norm(a.cpu().numpy() - b.cpu().numpy()))
        assert abs(float(out.item()) - want) <= TOL * max(want, 1e-300)
    # beyond the static array: rejected before any device work (the pointers are never read)
    small = torch.zeros(4, dtype=torch.float64, device="cuda")
    too_many = ctypes.c_longlong(65536 * 2048 + 1)
    st = L.metos3d_residual_static(ctypes.c_void_p(small.data_ptr()), ctypes.c_void_p(small.data_ptr()), too_many,
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert st == m3d.M3D_ERR_ARG
    assert b"exceed the maximum" in L.metos3d_residual_static_error()
