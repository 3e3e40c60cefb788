"""The allocation-free entry point kkt_solve_noalloc, called through the C
interface, against the handle-based path (kkt_create / kkt_factor /
kkt_solve) on the same inputs for two calls in a row, and against the FP64
oracle.

It exists for callers that cannot allocate device memory where they solve
(a real-time loop that must not touch an allocator, a plugin whose host
framework owns every allocation); it keeps its factor in a fixed
library-owned device buffer that every call reuses. This file runs last so
that a failure here leaves every other test already run.
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


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="module")
def noalloc(kkt):
    """The C entry point itself (plain ctypes, no Python wrapper)."""
    lib = ctypes.CDLL(kkt.LIB_PATH)
    fn = lib.kkt_solve_noalloc
    fn.restype = ctypes.c_int
    vp = ctypes.c_void_p
    fn.argtypes = [ctypes.c_int] * 4 + [vp] * 5 + [ctypes.c_int, ctypes.c_int, vp, vp]
    return fn


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def ptr(t):
    return t.data_ptr() if t is not None else None


def handle_solve(kkt, D, E, G, R, b, P):
    import torch
    N, n, _ = D.shape
    m = R.shape[0]
    h = kkt.kkt_create(N, n, m, P)
    try:
        bd = dev(b)
        kkt.kkt_factor(h, dev(D), dev(E) if N > 1 else None, dev(G) if m else None, dev(R) if m else None)
        kkt.kkt_solve(h, bd)
        torch.cuda.synchronize()
        return bd.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)


def call(noalloc, N, n, m, P, D, E, G, R, b, nrhs):
    """One call through the C interface; returns (status, x, info record)."""
    import torch
    Dd, bd = dev(D), dev(b)
    Ed = dev(E) if N > 1 else None
    Gd, Rd = (dev(G), dev(R)) if m else (None, None)
    info = torch.full((4,), 7, dtype=torch.int32, device="cuda")
    st = noalloc(N, n, m, P, ptr(Dd), ptr(Ed), ptr(Gd), ptr(Rd), ptr(bd), nrhs, nrhs, ptr(info),
                 torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, bd.cpu().numpy(), info.cpu().tolist()


def test_noalloc_matches_handle_path_twice(kkt, noalloc):
    cases = [(256, 32, 8, 16, 0), (200, 12, 4, 9, 1)]   # two calls in a row, different shapes
    outs = []
    for N, n, m, P, seed in cases:
        D, E, G, R = gen.ipm(N, n, m, seed=seed)
        b = gen.rhs(N * n + m, 3, seed=seed + 10)
        st, x, info = call(noalloc, N, n, m, P, D, E, G, R, b, 3)
        assert st == 0, kkt.status_string(st)
        assert info == [0, 0, 0, 0]
        outs.append((x, handle_solve(kkt, D, E, G, R, b, P)))
    for x_noalloc, x_ref in outs:
        np.testing.assert_allclose(x_noalloc, x_ref, rtol=0, atol=1e-11 * np.abs(x_ref).max())


# (N, n, m, P, nrhs): the sequential method without an arrow, more right-hand
# sides than one substitution chunk (16 columns), a block size the handle
# path runs one warp per task (here the CTA kernel), and a two-level case
@pytest.mark.parametrize("N,n,m,P,nrhs", [(40, 24, 0, 1, 2), (96, 16, 4, 6, 20), (300, 6, 2, 12, 1),
                                          (128, 32, 8, 8, 1)])
def test_noalloc_matches_oracle(kkt, orc, noalloc, N, n, m, P, nrhs):
    """x against the FP64 oracle's sequential solve on moderately conditioned
    inputs (Sigma over +-2 decades): |x - x_oracle| <= 1e-10 |x_oracle| and a
    normwise backward error of a few units of roundoff; two calls in a row
    give the same x bit for bit."""
    D, E, G, R = gen.ipm(N, n, m, seed=N + n, sigma_decades=2.0)
    b = gen.rhs(N * n + m, nrhs, seed=N + 1)
    st, x, info = call(noalloc, N, n, m, P, D, E, G, R, b, nrhs)
    assert st == 0, kkt.status_string(st)
    assert info == [0, 0, 0, 0]
    F = orc.seq_factor(D, E, G, R)
    xo = orc.seq_solve(F, b)
    err = np.abs(x - xo).max() / np.abs(xo).max()
    assert err <= 1e-10, f"forward difference {err:.3e}"
    for c in range(nrhs):
        eta = orc.block_backward_error(D, E, G, R, x[:, c] if x.ndim == 2 else x, b[:, c] if b.ndim == 2 else b)
        assert eta <= 1e-14, f"column {c}: backward error {eta:.3e}"
    st2, x2, _ = call(noalloc, N, n, m, P, D, E, G, R, b, nrhs)
    assert st2 == 0 and np.array_equal(x, x2)


@pytest.mark.parametrize("P,bad_stage", [(1, 5), (4, 9), (4, 7)])
def test_noalloc_reports_breakdown(kkt, noalloc, P, bad_stage):
    """A negated diagonal block (made on the host) comes back in the caller's
    info record as KKT_ERR_NOT_SPD with its natural stage; a following call on
    SPD input clears the record."""
    N, n, m = 16, 4, 2
    D, E, G, R, _ = gen.known_factor(N, n, m, seed=0)
    b = gen.rhs(N * n + m, 1, seed=3)
    Dbad = D.copy()
    Dbad[bad_stage] = -Dbad[bad_stage]
    st, _, info = call(noalloc, N, n, m, P, Dbad, E, G, R, b, 1)
    assert st == 0
    # stage 7 separates segments 1 and 2 of the partition [7, 2, 2, 2]: its
    # pivot block is factored in the reduced system (level 2)
    level = 2 if (P, bad_stage) == (4, 7) else 1
    assert info == [kkt.KKT_ERR_NOT_SPD, 0, bad_stage, level], info
    st, _, info = call(noalloc, N, n, m, P, D, E, G, R, b, 1)
    assert st == 0 and info == [0, 0, 0, 0]


def test_noalloc_rejects_too_large(kkt):
    import torch
    N, n, m = 1024, 32, 8
    z = torch.zeros(N * n * n, dtype=torch.float64, device="cuda")
    zb = torch.zeros(N * n + m, dtype=torch.float64, device="cuda")
    with pytest.raises(kkt.KKTError) as ei:
        kkt.kkt_solve_noalloc(N, n, m, 4, z, z, z, z, zb, nrhs=1, ldb=1)
    assert ei.value.status == kkt.KKT_ERR_CAPACITY


def test_noalloc_wrapper_checks_sizes(kkt):
    """The Python wrapper refuses tensors smaller than the shape needs (the
    kernels would access them out of bounds) before calling the library."""
    import torch
    N, n, m = 16, 4, 2
    z = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        kkt.kkt_solve_noalloc(N, n, m, 2, z, z, z, z, z, nrhs=1, ldb=1)
