"""The one-warp substitution of systems solved by the sequential method (one
level, P = 1) with one right-hand side, which kkt_solve and
kkt_solve_refined choose for such systems: one warp per system runs the
forward sweep (Algorithm 2), the corner of Eq. (7) and the backward sweep
(Algorithm 3), the stage blocks streamed by bulk copies into a double
buffer.

Checked through the C interface against the FP64 oracle (backward error
<= 1e-14, residual within 10x the oracle's, forward difference within
10 u kappa_est) and against the multi-column substitution on the same
factor (two equal columns run the CTA kernels). Shapes cover one and two
rows per lane, arrow widths 0 to 16, N = 1, 2, 3 and longer horizons, odd
block sizes and FP32 blocks whose m n is not a multiple of 4 (the bulk
copies cannot take them; the CTA kernels run), FP64 and mixed precision,
uneven batches, and the bordered descriptors a fused factor-and-solve
leaves behind (the arrow carries one more row).
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


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


def gates(orc, D, E, G, R, x, b, xo, fwd=True):
    eta = orc.block_backward_error(D, E, G, R, x, b)
    assert eta <= 1e-14, f"backward error {eta:.3e}"
    r = np.linalg.norm(b - orc.block_matvec(D, E, G, R, x))
    ro = np.linalg.norm(b - orc.block_matvec(D, E, G, R, xo))
    assert r <= max(1e-10 * np.linalg.norm(b), 10 * ro), (r, ro)
    if fwd:
        kap = orc.cond_est(D, E, G, R)
        err = np.abs(x - xo).max() / np.abs(xo).max()
        assert err <= 10 * U * kap, f"forward difference {err:.3e} > 10 u kappa = {10 * U * kap:.3e}"


def inputs(N, n, m, seed):
    D, E, G, R = gen.ipm(N, n, m, seed=seed, sigma_decades=3.0)
    b = gen.rhs(N * n + m, 1, seed=seed + 1)
    return D, E, G, R, b


def dev_blocks(D, E, G, R, N, m):
    return dev(D), dev(E) if N > 1 else None, dev(G) if m else None, dev(R) if m else None


@pytest.mark.parametrize("N,n,m", [
    (1, 8, 4), (2, 6, 2), (3, 12, 0), (40, 2, 1), (64, 24, 4), (50, 32, 8), (30, 34, 16), (25, 48, 16),
    (33, 48, 0), (200, 16, 5), (20, 7, 3), (15, 45, 2)])
def test_seq_solve_fp64(kkt, orc, N, n, m):
    """FP64: x (one column) against the oracle, and against the same
    factor's two-column substitution within the forward-error bound."""
    import torch
    D, E, G, R, b = inputs(N, n, m, seed=10 * N + n + m)
    h = kkt.kkt_create_plan(N, n, m, [1], kkt.KKT_PARTITION_BALANCED, kkt.KKT_FP64)
    try:
        Dd, Ed, Gd, Rd = dev_blocks(D, E, G, R, N, m)
        kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
        x1 = dev(b)
        kkt.kkt_solve(h, x1)
        x2 = dev(np.stack([b, b], axis=1))
        kkt.kkt_solve(h, x2, nrhs=2, ldb=2)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        x1, x2 = x1.cpu().numpy(), x2.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)
    xo = orc.seq_solve(orc.seq_factor(D, E, G, R), b)
    gates(orc, D, E, G, R, x1, b, xo)
    kap = orc.cond_est(D, E, G, R)
    np.testing.assert_allclose(x1, x2[:, 0], rtol=0, atol=10 * U * kap * np.abs(x2[:, 0]).max())
    np.testing.assert_array_equal(x2[:, 0], x2[:, 1])


@pytest.mark.parametrize("N,n,m", [(64, 24, 4), (40, 48, 4), (50, 32, 8), (30, 6, 2), (20, 2, 1), (3, 12, 0),
                                   (1, 16, 4)])
def test_seq_solve_mixed_refined(kkt, orc, N, n, m):
    """Mixed precision: FP32 factor and one-column FP32 substitutions, FP64
    refinement to the rounding floor; the FP64 gates hold against the oracle.
    (20, 2, 1): m n = 2, not a multiple of 4: the FP32 blocks go through the
    CTA kernels."""
    import torch
    D, E, G, R, b = inputs(N, n, m, seed=3 * N + n)
    h = kkt.kkt_create_plan(N, n, m, [1], kkt.KKT_PARTITION_BALANCED, kkt.KKT_MIXED_FP32_ALL)
    try:
        Dd, Ed, Gd, Rd = dev_blocks(D, E, G, R, N, m)
        kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
        x = torch.zeros(N * n + m, dtype=torch.float64, device="cuda")
        kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, dev(b), x, sweeps=10, tol=1e-16)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        x = x.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)
    xo = orc.seq_solve(orc.seq_factor(D, E, G, R), b)
    gates(orc, D, E, G, R, x, b, xo, fwd=False)


@pytest.mark.parametrize("precision", [0, 2])
def test_seq_solve_uneven_batch(kkt, orc, precision):
    """An uneven batch of sequential systems (block sizes 6, 7, 12, 24, 48;
    arrows 0, 3, 4): launch groups per block size, odd n on the CTA kernels;
    every system against the oracle (FP64 directly, mixed after refinement)."""
    import torch
    rng = np.random.default_rng(5)
    shapes = [(int(rng.integers(1, 60)), int(n), int(m)) for n, m in
              zip(rng.choice([6, 7, 12, 24, 48], size=14), rng.choice([0, 3, 4], size=14))]
    systems = [gen.ipm(N, n, m, seed=40 + i, sigma_decades=3.0) for i, (N, n, m) in enumerate(shapes)]
    bs = [gen.rhs(N * n + m, 1, seed=60 + i) for i, (N, n, m) in enumerate(shapes)]
    Ns, ns, ms = zip(*shapes)
    cat = lambda i: dev(np.concatenate([s[i].ravel() for s in systems] + [np.zeros(1)]))
    D, E, G, R = cat(0), cat(1), cat(2), cat(3)
    b = dev(np.concatenate(bs))
    h = kkt.kkt_batch_create(list(Ns), list(ns), list(ms), [1] * len(shapes), precision)
    try:
        kkt.kkt_factor(h, D, E, G, R)
        if precision:
            x = torch.zeros_like(b)
            kkt.kkt_solve_refined(h, D, E, G, R, b, x, sweeps=10, tol=1e-16)
        else:
            x = b.clone()
            kkt.kkt_solve(h, x)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        off = kkt.kkt_batch_offsets(h, len(shapes))["b"]
        x = x.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)
    for i, s in enumerate(systems):
        xi = x[off[i]:off[i + 1]]
        xo = orc.seq_solve(orc.seq_factor(*s), bs[i])
        gates(orc, *s, xi, bs[i], xo, fwd=not precision)


@pytest.mark.parametrize("N,n,m", [(40, 24, 4), (30, 32, 0), (12, 48, 15)])
def test_seq_solve_after_bordered_factorization(kkt, orc, N, n, m):
    """kkt_factor_solve (the bordered pass) leaves descriptors whose arrow has
    one more row; a following kkt_solve on another right-hand side runs the
    one-warp substitution on them (the extra row's x is not part of the
    corner) and meets the gates."""
    import torch
    D, E, G, R, b = inputs(N, n, m, seed=N + 7)
    b2 = gen.rhs(N * n + m, 1, seed=N + 8)
    h = kkt.kkt_create_plan(N, n, m, [1], kkt.KKT_PARTITION_BALANCED, kkt.KKT_FP64)
    try:
        Dd, Ed, Gd, Rd = dev_blocks(D, E, G, R, N, m)
        x1 = dev(b)
        kkt.kkt_factor_solve(h, Dd, Ed, Gd, Rd, x1)
        x2 = dev(b2)
        kkt.kkt_solve(h, x2)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        x1, x2 = x1.cpu().numpy(), x2.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)
    F = orc.seq_factor(D, E, G, R)
    gates(orc, D, E, G, R, x1, b, orc.seq_solve(F, b))
    gates(orc, D, E, G, R, x2, b2, orc.seq_solve(F, b2))


def test_seq_solve_wait_runs_out_and_reports(kkt, orc):
    """Every stage expecting 16 bytes more than its copies deliver
    (kkt_set_wait_limit with unmet): each system's first wait runs out after
    the short limit, the call completes, kkt_get_info reports
    KKT_ERR_TIMEOUT at level 1; with the real counts restored the next solve
    on the same factor is correct."""
    import torch
    N, n, m = 30, 12, 4
    D, E, G, R, b = inputs(N, n, m, seed=77)
    h = kkt.kkt_create_plan(N, n, m, [1], kkt.KKT_PARTITION_BALANCED, kkt.KKT_FP64)
    try:
        Dd, Ed, Gd, Rd = dev_blocks(D, E, G, R, N, m)
        kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        kkt.kkt_set_wait_limit(h, 1 << 16, unmet=True)
        x = dev(b)
        kkt.kkt_solve(h, x)
        torch.cuda.synchronize()
        info = kkt.kkt_get_info(h)
        assert info["status"] == kkt.KKT_ERR_TIMEOUT and info["level"] == 1, info
        kkt.kkt_set_wait_limit(h, 1 << 31, unmet=False)
        x = dev(b)
        kkt.kkt_solve(h, x)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        x = x.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)
    gates(orc, D, E, G, R, x, b, orc.seq_solve(orc.seq_factor(D, E, G, R), b))
