"""The persistent schedule of the factorization (kkt_set_persistent): one
launch whose CTAs take segment tasks of every level by ticket, in
topological and longest-first order, a reduced-system task waiting on the
ready counters of the tasks that feed it. Checked through the C interface:
bitwise the results of the per-level launches (the same operations per
element), the FP64 oracle's solution, CUDA-graph capture, and the bounded
waits (an injected unsatisfiable dependency makes every wait run out: the
call returns, kkt_get_info reports KKT_ERR_TIMEOUT, nothing hangs)."""
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


def packed(systems):
    cat = lambda i: dev(np.concatenate([s[i].ravel() for s in systems] + [np.zeros(1)]))
    return cat(0), cat(1), cat(2), cat(3)


def factor_solve(kkt, h, D, E, G, R, b):
    import torch
    x = b.clone()
    kkt.kkt_factor(h, D, E, G, R)
    kkt.kkt_solve(h, x)
    torch.cuda.synchronize()
    return x.cpu().numpy(), kkt.kkt_get_info(h)


def batch_case(kind):
    """(systems, right-hand sides, N, n, m, P per system)"""
    if kind == "uneven_seq":      # the uneven workload's kind of batch, sequential plans
        sy = gen.uneven_batch(40, seed=4, N_range=(8, 70))
        Ps = [1] * len(sy)
    elif kind == "uneven_two_level":
        sy = gen.uneven_batch(16, seed=6, N_range=(10, 60))
        Ps = [max(1, min(1 + i % 4, (s[0].shape[0] + 1) // 2)) for i, s in enumerate(sy)]
    else:
        raise ValueError(kind)
    Ns = [s[0].shape[0] for s in sy]
    ns = [s[0].shape[1] for s in sy]
    ms = [s[3].shape[0] for s in sy]
    bs = [gen.rhs(N * n + m, 1, seed=50 + i) for i, (N, n, m) in enumerate(zip(Ns, ns, ms))]
    return sy, bs, Ns, ns, ms, Ps


@pytest.mark.parametrize("kind", ["uneven_seq", "uneven_two_level"])
@pytest.mark.parametrize("precision", [0, 2])
def test_persistent_batch_bitwise_and_oracle(kkt, orc, kind, precision):
    sy, bs, Ns, ns, ms, Ps = batch_case(kind)
    D, E, G, R = packed(sy)
    b = dev(np.concatenate(bs))
    h = kkt.kkt_batch_create(Ns, ns, ms, Ps, precision)
    try:
        x_lv, info = factor_solve(kkt, h, D, E, G, R, b)
        assert info["status"] == 0
        kkt.kkt_set_persistent(h, True)
        assert kkt.kkt_launch_counts(h)[0] == 1
        x_p, info = factor_solve(kkt, h, D, E, G, R, b)
        assert info["status"] == 0, info
        x_p2, _ = factor_solve(kkt, h, D, E, G, R, b)
        off = kkt.kkt_batch_offsets(h, len(sy))["b"]
    finally:
        kkt.kkt_destroy(h)
    np.testing.assert_array_equal(x_p, x_lv)
    np.testing.assert_array_equal(x_p2, x_p)
    if precision == 0:
        for i, s in enumerate(sy):
            xi = x_p[off[i]:off[i + 1]]
            assert orc.block_backward_error(*s, xi, bs[i]) <= 1e-14


@pytest.mark.parametrize("N,n,m,levels,precision", [(300, 24, 4, [30, 6, 1], 0), (2048, 6, 2, [64, 8, 1], 0),
                                                    (2048, 6, 2, [64, 8, 1], 2), (1024, 32, 8, [152, 38, 10, 1], 0),
                                                    (500, 48, 4, [50, 10, 2, 1], 2)])
def test_persistent_multi_level_bitwise(kkt, orc, N, n, m, levels, precision):
    """Recursive plans (every level in the one launch, reduced-system tasks
    released by their feeders): bitwise the per-level result, and the
    oracle's solution to its backward-error gate."""
    kind = gen.raceline if n <= 8 else gen.ipm
    Dh, Eh, Gh, Rh = kind(N, n, m, seed=9)
    bh = gen.rhs(N * n + m, 1, seed=10)
    D, E, G, R, b = dev(Dh), dev(Eh), dev(Gh), dev(Rh), dev(bh)
    h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED, precision)
    try:
        x_lv, info = factor_solve(kkt, h, D, E, G, R, b)
        assert info["status"] == 0
        kkt.kkt_set_persistent(h, True)
        x_p, info = factor_solve(kkt, h, D, E, G, R, b)
        assert info["status"] == 0, info
    finally:
        kkt.kkt_destroy(h)
    np.testing.assert_array_equal(x_p, x_lv)
    if precision == 0:
        assert orc.block_backward_error(Dh, Eh, Gh, Rh, x_p, bh) <= 1e-14


def test_persistent_graph_capture(kkt):
    import torch
    sy, bs, Ns, ns, ms, Ps = batch_case("uneven_two_level")
    D, E, G, R = packed(sy)
    b0 = dev(np.concatenate(bs))
    h = kkt.kkt_batch_create(Ns, ns, ms, Ps)
    try:
        kkt.kkt_set_persistent(h, True)
        x_ref, _ = factor_solve(kkt, h, D, E, G, R, b0)
        x = b0.clone()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                kkt.kkt_factor(h, D, E, G, R)
                kkt.kkt_solve(h, x)
        torch.cuda.current_stream().wait_stream(s)
        for _ in range(2):
            x.copy_(b0)
            g.replay()
            torch.cuda.synchronize()
            np.testing.assert_array_equal(x.cpu().numpy(), x_ref)
        assert kkt.kkt_get_info(h)["status"] == 0
    finally:
        kkt.kkt_destroy(h)


def test_persistent_wait_runs_out_and_reports(kkt, orc):
    """An injected dependency that no task releases: every reduced-system
    task's wait runs out after the (short) limit; the call completes,
    kkt_get_info reports KKT_ERR_TIMEOUT at a reduced level; with the real
    counts restored the next factorization is correct again."""
    import torch
    N, n, m = 200, 24, 4
    Dh, Eh, Gh, Rh = gen.ipm(N, n, m, seed=2, sigma_decades=2.0)
    bh = gen.rhs(N * n + m, 1, seed=3)
    D, E, G, R, b = dev(Dh), dev(Eh), dev(Gh), dev(Rh), dev(bh)
    h = kkt.kkt_create_plan(N, n, m, [20, 4, 1], kkt.KKT_PARTITION_BALANCED)
    try:
        kkt.kkt_set_persistent(h, True)
        kkt.kkt_set_wait_limit(h, 1 << 16, unmet=True)
        kkt.kkt_factor(h, D, E, G, R)
        torch.cuda.synchronize()
        info = kkt.kkt_get_info(h)
        assert info["status"] == kkt.KKT_ERR_TIMEOUT, info
        assert info["level"] >= 2
        kkt.kkt_set_wait_limit(h, 1 << 31, unmet=False)
        x, info = factor_solve(kkt, h, D, E, G, R, b)
        assert info["status"] == 0, info
    finally:
        kkt.kkt_destroy(h)
    xo = orc.seq_solve(orc.seq_factor(Dh, Eh, Gh, Rh), bh)
    assert np.abs(x - xo).max() <= 1e-10 * np.abs(xo).max()


def test_persistent_keeps_refine_fallback_buffers(kkt, orc):
    """The refinement fallback's buffers survive enabling the persistent
    schedule after them: a mixed handle with the fallback set first and the
    persistent schedule second refines a stalling system (Sigma over 20
    decades) to the same x, bit for bit, as a handle with the fallback alone,
    meets the FP64 backward-error gate, and is destroyed cleanly."""
    import torch
    N, n, m = 2048, 6, 2
    D, E, G, R = gen.raceline(N, n, m, seed=5, sigma_decades=10.0)
    b = gen.rhs(N * n + m, 1, seed=6)
    Dd, Ed, Gd, Rd, bd = dev(D), dev(E), dev(G), dev(R), dev(b)
    xs = {}
    for persist in (False, True):
        h = kkt.kkt_create_plan(N, n, m, [1], kkt.KKT_PARTITION_BALANCED, kkt.KKT_MIXED_FP32_ALL)
        try:
            kkt.kkt_set_refine_fallback(h, 12)
            if persist:
                kkt.kkt_set_persistent(h, True)
                assert kkt.kkt_launch_counts(h)[0] == 1
            kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
            x = torch.zeros(N * n + m, dtype=torch.float64, device="cuda")
            kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, bd, x, sweeps=10, tol=1e-16)
            torch.cuda.synchronize()
            assert kkt.kkt_get_info(h)["status"] == 0
            xs[persist] = x.cpu().numpy()
        finally:
            kkt.kkt_destroy(h)
    np.testing.assert_array_equal(xs[True], xs[False])
    assert orc.block_backward_error(D, E, G, R, xs[True], b) <= 1e-14
