"""Factor tasks of one-stage segments on clusters of 2, 4 or 8 CTAs: the
deep levels of recursive plans whose every segment is a single stage with
fill-in rows (Alg. 1 on the reduced systems of Eq. (7)), which the automatic
pairing policy runs with k_factor_clus. Each CTA of a cluster factors the
pivot block, solves a band of the panel rows and updates a band of the
Schur trapezoid; the operations per element are those of the one- and
two-CTA layouts, so the solution must agree bit for bit with
KKT_PAIR_AUTO_PAIRS (pairs) and KKT_PAIR_OFF (one CTA per task), for the
two-pass solve (several right-hand sides) and the bordered factor-and-solve
pass alike; and it meets the oracle's gates.

Shapes: the single-system benchmark shape (N = 1024, n = 32, m = 8) with
its halving plan, odd block sizes just above the one-warp kernels' limit,
no arrow (m = 0), the largest blocks with a wide arrow (n = 48, m = 15, so
that the bordered arrow has 16 rows), and a plan whose levels 2 and 3 have
segments of several stages (they keep the one- and two-CTA layouts) above
a level of single stages.
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


SHAPES = [
    (1024, 32, 8, halving(256)),
    (255, 17, 3, halving(64)),
    (300, 24, 0, halving(64)),
    (200, 48, 15, halving(32)),
    (130, 33, 5, [40, 12, 4, 2, 1]),
]


def run_policy(kkt, policy, N, n, m, levels, D, E, G, R, b, bordered):
    import torch
    h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED, kkt.KKT_FP64)
    try:
        kkt.kkt_set_pairing(h, policy)
        ctas = [kkt.kkt_factor_ctas_per_task(h, l) for l in range(len(levels))]
        Dd, Ed, Gd, Rd = dev(D), dev(E), dev(G) if m else None, dev(R) if m else None
        if bordered:
            x = dev(b[:, 0])
            kkt.kkt_factor_solve(h, Dd, Ed, Gd, Rd, x)
        else:
            x = dev(b)
            kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
            kkt.kkt_solve(h, x, nrhs=b.shape[1], ldb=b.shape[1])
        torch.cuda.synchronize()
        info = kkt.kkt_get_info(h)
        assert info["status"] == 0, info
        return x.cpu().numpy(), ctas
    finally:
        kkt.kkt_destroy(h)


@pytest.mark.parametrize("bordered", [False, True])
@pytest.mark.parametrize("N,n,m,levels", SHAPES)
def test_cluster_layout_bitwise_and_oracle(kkt, orc, N, n, m, levels, bordered):
    D, E, G, R = gen.ipm(N, n, m, seed=N + n + m, sigma_decades=3.0)
    b = gen.rhs(N * n + m, 3, seed=N + 1).reshape(N * n + m, 3)
    xa, ca = run_policy(kkt, kkt.KKT_PAIR_AUTO, N, n, m, levels, D, E, G, R, b, bordered)
    xp, cp = run_policy(kkt, kkt.KKT_PAIR_AUTO_PAIRS, N, n, m, levels, D, E, G, R, b, bordered)
    xo, co = run_policy(kkt, kkt.KKT_PAIR_OFF, N, n, m, levels, D, E, G, R, b, bordered)
    # the deep levels (one-stage segments) run on clusters under the automatic policy
    assert max(ca[1:-1]) >= 4, ca
    assert max(cp) <= 2 and max(co) == 1, (cp, co)
    np.testing.assert_array_equal(xa, xp)
    np.testing.assert_array_equal(xa, xo)
    # gates against the FP64 oracle on the first column
    x0 = xa if bordered else xa[:, 0]
    b0 = b[:, 0]
    eta = orc.block_backward_error(D, E, G, R, x0, b0)
    assert eta <= 1e-14, f"backward error {eta:.3e}"
    xr = orc.seq_solve(orc.seq_factor(D, E, G, R), b0)
    kap = orc.cond_est(D, E, G, R)
    err = np.abs(x0 - xr).max() / np.abs(xr).max()
    assert err <= 10 * U * kap, f"forward difference {err:.3e} > 10 u kappa = {10 * U * kap:.3e}"


def test_ctas_per_task_query(kkt):
    """kkt_factor_ctas_per_task: argument checks and the layouts it reports
    (the multi-stage first level one CTA per task, forced pairs 2)."""
    levels = halving(256)
    h = kkt.kkt_create_plan(1024, 32, 8, levels, kkt.KKT_PARTITION_BALANCED, kkt.KKT_FP64)
    try:
        assert kkt.kkt_factor_ctas_per_task(h, 0) == 1
        with pytest.raises(kkt.KKTError):
            kkt.kkt_factor_ctas_per_task(h, len(levels))
        with pytest.raises(kkt.KKTError):
            kkt.kkt_factor_ctas_per_task(h, -1)
        kkt.kkt_set_pairing(h, kkt.KKT_PAIR_ON)
        assert all(kkt.kkt_factor_ctas_per_task(h, l) == 2 for l in range(len(levels)))
    finally:
        kkt.kkt_destroy(h)



@pytest.mark.parametrize("precision", [1, 2])
def test_cluster_layout_mixed_levels(kkt, orc, precision):
    """KKT_MIXED_FP32 (level 1 in FP32 panels, the deeper levels FP64: the
    deep levels run on clusters, the backward levels one launch per level
    since their precisions differ) and KKT_MIXED_FP32_ALL (every level mixed:
    no clusters, the backward levels in one launch): the refined solution
    agrees bit for bit with the pair layout's and meets the gates."""
    import torch
    N, n, m = 255, 32, 8
    levels = halving(64)
    D, E, G, R = gen.ipm(N, n, m, seed=77, sigma_decades=3.0)
    b = gen.rhs(N * n + m, 1, seed=78)
    Dd, Ed, Gd, Rd, bd = dev(D), dev(E), dev(G), dev(R), dev(b)
    outs, ctas = [], []
    for policy in (kkt.KKT_PAIR_AUTO, kkt.KKT_PAIR_AUTO_PAIRS):
        h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED, precision)
        try:
            kkt.kkt_set_pairing(h, policy)
            ctas.append([kkt.kkt_factor_ctas_per_task(h, l) for l in range(len(levels))])
            x = torch.zeros_like(bd)
            kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
            kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, bd, x, sweeps=8, tol=1e-16)
            torch.cuda.synchronize()
            assert kkt.kkt_get_info(h)["status"] == 0
            outs.append(x.cpu().numpy())
        finally:
            kkt.kkt_destroy(h)
    if precision == 1:
        assert max(ctas[0][1:-1]) >= 4, ctas[0]
    else:
        assert max(ctas[0]) <= 2, ctas[0]
    np.testing.assert_array_equal(outs[0], outs[1])
    assert orc.block_backward_error(D, E, G, R, outs[0], b) <= 1e-14
