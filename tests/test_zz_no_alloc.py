"""The allocation-free entry point kkt_solve_noalloc, called through the C
interface, against the handle-based path (kkt_create / kkt_factor /
kkt_solve) on the same inputs, for two calls in a row.

It exists for callers that cannot allocate device memory where they solve
(inside a graph-capture region, a real-time loop, a plugin whose host owns
the allocator); it keeps its factor in a fixed library-owned device buffer
that every call reuses. This file runs last so that a failure here leaves
every other test already run.
"""
import ctypes

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kkt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_00946_gb300 as k
    return k


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def handle_solve(kkt, D, E, G, R, b, P):
    import torch
    N, n, _ = D.shape
    m = R.shape[0]
    h = kkt.kkt_create(N, n, m, P)
    try:
        bd = dev(b)
        kkt.kkt_factor(h, dev(D), dev(E), dev(G) if m else None, dev(R) if m else None)
        kkt.kkt_solve(h, bd)
        torch.cuda.synchronize()
        return bd.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)


def test_noalloc_matches_handle_path_twice(kkt):
    import torch
    lib = ctypes.CDLL(kkt.LIB_PATH)
    fn = lib.kkt_solve_noalloc
    fn.restype = ctypes.c_int
    vp = ctypes.c_void_p
    fn.argtypes = [ctypes.c_int] * 4 + [vp] * 5 + [ctypes.c_int, ctypes.c_int, vp, vp]
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(256, 32, 8, 16, 0), (200, 12, 4, 9, 1)]   # two calls in a row, different shapes
    outs = []
    for N, n, m, P, seed in cases:
        D, E, G, R = gen.ipm(N, n, m, seed=seed)
        b = gen.rhs(N * n + m, 3, seed=seed + 10)
        Dd, Ed, Gd, Rd, bd = dev(D), dev(E), dev(G), dev(R), dev(b)
        info = torch.full((4,), 7, dtype=torch.int32, device="cuda")
        st = fn(N, n, m, P, Dd.data_ptr(), Ed.data_ptr(), Gd.data_ptr(), Rd.data_ptr(), bd.data_ptr(),
                3, 3, info.data_ptr(), stream)
        assert st == 0, kkt.status_string(st)
        torch.cuda.synchronize()
        assert info.cpu().tolist() == [0, 0, 0, 0]
        outs.append((bd.cpu().numpy(), handle_solve(kkt, D, E, G, R, b, P)))
    for x_noalloc, x_ref in outs:
        np.testing.assert_allclose(x_noalloc, x_ref, rtol=0, atol=1e-11 * np.abs(x_ref).max())


def test_noalloc_rejects_too_large(kkt):
    import torch
    N, n, m = 1024, 32, 8
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(kkt.KKTError) as ei:
        kkt.kkt_solve_noalloc(N, n, m, 4, z, z, z, z, z, nrhs=1, ldb=1)
    assert ei.value.status == kkt.KKT_ERR_CAPACITY
