"""The backward substitution of every level below the top in one launch
(k_backward_chain; Algorithm 3's parallel phase of each level, top down):
CTAs take (task, column group) items by ticket, request their stage's factor
blocks, wait (bounded) for the level above's counter and release their own.
Through the C interface:
* bitwise the per-level launches (kkt_set_backward_chain(h, 0)) for the
  bordered factor-and-solve pass, the two-pass solve with one right-hand
  side and with 3 and 16 (chunks of several columns run the per-level
  launches either way), mixed precision with refinement, and plans with
  multi-stage segments on every level;
* the oracle's gates on the chained result;
* kkt_launch_counts: one backward launch instead of L - 1;
* a wait that cannot be met (kkt_set_wait_limit with unmet) runs out, the
  call completes and kkt_get_info reports KKT_ERR_TIMEOUT; with the real
  counts restored the next solve is correct.
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


def halving(P1):
    lv = [P1]
    while lv[-1] > 1:
        lv.append(lv[-1] // 2)
    return lv


def run(kkt, chain, N, n, m, levels, D, E, G, R, b, mode, precision=0):
    import torch
    h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED, precision)
    try:
        kkt.kkt_set_backward_chain(h, chain)
        counts = kkt.kkt_launch_counts(h)
        Dd, Ed, Gd, Rd = dev(D), dev(E), dev(G) if m else None, dev(R) if m else None
        if mode == "bordered":
            x = dev(b[:, 0])
            kkt.kkt_factor_solve(h, Dd, Ed, Gd, Rd, x)
        elif mode == "refined":
            x = torch.zeros(b.shape[0], dtype=torch.float64, device="cuda")
            kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
            kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, dev(b[:, 0]), x, sweeps=6, tol=1e-16)
        else:
            x = dev(b)
            kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
            kkt.kkt_solve(h, x, nrhs=b.shape[1], ldb=b.shape[1])
        torch.cuda.synchronize()
        info = kkt.kkt_get_info(h)
        assert info["status"] == 0, info
        return x.cpu().numpy(), counts
    finally:
        kkt.kkt_destroy(h)


CASES = [
    (1024, 32, 8, halving(256), "bordered", 1, 0),
    (1024, 32, 8, halving(256), "two-pass", 1, 0),
    (1024, 32, 8, halving(256), "two-pass", 3, 0),
    (1024, 32, 8, halving(256), "two-pass", 16, 0),
    (600, 24, 6, [60, 12, 3, 1], "two-pass", 2, 0),
    (600, 24, 6, [60, 12, 3, 1], "bordered", 1, 0),
    (300, 17, 0, [32, 8, 2, 1], "bordered", 1, 0),
    (400, 32, 8, [40, 10, 3, 1], "refined", 1, 2),
]


@pytest.mark.parametrize("N,n,m,levels,mode,nrhs,precision", CASES)
def test_chain_bitwise_and_oracle(kkt, orc, N, n, m, levels, mode, nrhs, precision):
    D, E, G, R = gen.ipm(N, n, m, seed=7 * N + n, sigma_decades=3.0)
    b = gen.rhs(N * n + m, nrhs, seed=N + 3).reshape(N * n + m, nrhs)
    xc, cc = run(kkt, True, N, n, m, levels, D, E, G, R, b, mode, precision)
    xl, cl = run(kkt, False, N, n, m, levels, D, E, G, R, b, mode, precision)
    L = len(levels)
    assert cl[1] - cc[1] == (L - 1) - 1, (cc, cl)  # one group per level here
    np.testing.assert_array_equal(xc, xl)
    x0 = xc if xc.ndim == 1 else xc[:, 0]
    b0 = b[:, 0]
    assert orc.block_backward_error(D, E, G, R, x0, b0) <= 1e-14
    xr = orc.seq_solve(orc.seq_factor(D, E, G, R), b0)
    kap = orc.cond_est(D, E, G, R)
    err = np.abs(x0 - xr).max() / np.abs(xr).max()
    assert err <= (100 if precision else 10) * U * kap, f"forward difference {err:.3e}"


def test_chain_not_used_for_two_levels(kkt):
    """Two levels leave one backward level: one launch either way."""
    h = kkt.kkt_create_plan(500, 32, 8, [40, 1], kkt.KKT_PARTITION_BALANCED, kkt.KKT_FP64)
    try:
        a = kkt.kkt_launch_counts(h)
        kkt.kkt_set_backward_chain(h, False)
        assert kkt.kkt_launch_counts(h) == a
    finally:
        kkt.kkt_destroy(h)


def test_chain_wait_runs_out_and_reports(kkt, orc):
    """Every chained wait expects one item more than its level has: each
    item below the first chained level gives up after the short limit, the
    solve completes, kkt_get_info reports KKT_ERR_TIMEOUT; with the real
    counts restored the next solve on the same factor is correct."""
    import torch
    N, n, m = 1024, 32, 8
    levels = halving(256)
    D, E, G, R = gen.ipm(N, n, m, seed=5, sigma_decades=3.0)
    b = gen.rhs(N * n + m, 1, seed=6)
    h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED, kkt.KKT_FP64)
    try:
        Dd, Ed, Gd, Rd = dev(D), dev(E), dev(G), dev(R)
        kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        kkt.kkt_set_wait_limit(h, 1 << 16, unmet=True)
        x = dev(b)
        kkt.kkt_solve(h, x)
        torch.cuda.synchronize()
        info = kkt.kkt_get_info(h)
        assert info["status"] == kkt.KKT_ERR_TIMEOUT, info
        kkt.kkt_set_wait_limit(h, 1 << 31, unmet=False)
        x = dev(b)
        kkt.kkt_solve(h, x)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        x = x.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)
    assert orc.block_backward_error(D, E, G, R, x, b) <= 1e-14


def test_code_warmup_same_bits_eager_and_graph(kkt, orc):
    """kkt_set_code_warmup: the companion system's pass on the forked side
    stream leaves this call's result bit for bit unchanged, eagerly and
    replayed from a captured graph (fork and join inside the capture)."""
    import torch
    N, n, m = 1024, 32, 8
    levels = halving(256)
    D, E, G, R = gen.ipm(N, n, m, seed=21, sigma_decades=3.0)
    b = gen.rhs(N * n + m, 1, seed=22)
    Dd, Ed, Gd, Rd, bsrc = dev(D), dev(E), dev(G), dev(R), dev(b)
    outs = []
    for warm in (False, True):
        h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED, kkt.KKT_FP64)
        try:
            kkt.kkt_set_code_warmup(h, warm)
            x = bsrc.clone()
            kkt.kkt_factor_solve(h, Dd, Ed, Gd, Rd, x)
            torch.cuda.synchronize()
            assert kkt.kkt_get_info(h)["status"] == 0
            outs.append(x.cpu().numpy())
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(s):
                xg = bsrc.clone()
                with torch.cuda.graph(g, stream=s):
                    kkt.kkt_factor_solve(h, Dd, Ed, Gd, Rd, xg, stream=s.cuda_stream)
            torch.cuda.current_stream().wait_stream(s)
            for _ in range(2):
                xg.copy_(bsrc)
                g.replay()
            torch.cuda.synchronize()
            assert kkt.kkt_get_info(h)["status"] == 0
            outs.append(xg.cpu().numpy())
            kkt.kkt_set_code_warmup(h, False)  # releases the companion
        finally:
            kkt.kkt_destroy(h)
    for o in outs[1:]:
        np.testing.assert_array_equal(outs[0], o)
    assert orc.block_backward_error(D, E, G, R, outs[0], b) <= 1e-14
