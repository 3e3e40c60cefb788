"""Host-side checks of the C interface that need no GPU: the library loads,
exports every symbol include/kkt.h declares, its partition rule and flop
model agree with the oracle's, and invalid arguments return status codes."""
import os
import re

import numpy as np
import pytest

import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def kkt():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_2511_00946_gb300 as k
    return k


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "kkt.h")).read()
    return sorted(set(re.findall(r"^\s*(?:kkt_status|const char\*)\s+(kkt_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(kkt):
    import ctypes
    lib = ctypes.CDLL(kkt.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(kkt.EXPORTED) == names


def test_partition_rule_matches_oracle(kkt, orc):
    for N in list(range(1, 80)) + [1024, 2356, 8192]:
        for P in sorted({1, 2, 3, 4, 7, 16, 152, 512, (N + 1) // 2, (N + 1) // 2 + 1}):
            try:
                want = orc.partition(N, P)
            except ValueError:
                with pytest.raises(kkt.KKTError) as ei:
                    kkt.kkt_partition_rule(N, P)
                assert ei.value.status == kkt.KKT_ERR_PARTITION
                continue
            assert kkt.kkt_partition_rule(N, P) == want, (N, P)


@pytest.mark.parametrize("N,n,m,P", [(16, 8, 4, 4), (40, 5, 2, 7), (30, 3, 0, 5), (20, 4, 3, 1),
                                     (64, 6, 2, 16), (33, 7, 1, 17)])
def test_flop_model_matches_oracle_counters(kkt, orc, N, n, m, P):
    """The library's algorithmic flop counts (the roofline numerators) equal
    what the oracle's instrumented primitives count, standard convention."""
    D, E, G, R, _ = gen.known_factor(N, n, m, seed=1)
    F = orc.par_factor(D, E, G, R, P=P, flops=True)
    _, fp, fs = orc.par_solve(F, gen.rhs(N * n + m, 1, seed=2), flops=True)
    orc.flops_reset()
    orc.seq_factor(D, E, G, R)
    _, seq_std = orc.flops_get()
    got = kkt.kkt_plan_flops(N, n, m, [P, 1] if P > 1 else [1], kkt.KKT_PARTITION_PAPER)
    assert got["factor"] == pytest.approx(F["flops_std"].sum(), rel=1e-12)
    assert got["solve"] == pytest.approx(fs.sum(), rel=1e-12)
    assert got["sequential_factor"] == pytest.approx(seq_std, rel=1e-12)


@pytest.mark.parametrize("paired", [False, True])
@pytest.mark.parametrize("N,n,m,P", [(1024, 32, 8, 152), (1024, 32, 8, 304), (151, 32, 8, 38), (8192, 6, 2, 2048),
                                     (50, 4, 0, 25), (16, 8, 4, 4), (37, 32, 8, 10), (5, 3, 0, 3)])
def test_balanced_partition(kkt, N, n, m, P, paired):
    """Balanced mode: same constraint as Eq. (13), every segment >= 1 stage,
    the other segments within one stage of each other, and a maximum segment
    cost (under the stage costs of the layout) never above the paper rule's.
    A paired segment's stage costs 1.05 first-segment stages (the fill-in
    rows run on the other CTA of the pair)."""
    seg = kkt.kkt_partition_balanced(N, n, m, P, paired)
    assert len(seg) == P and min(seg) >= 1
    assert sum(seg) + P - 1 == N
    if P > 2:
        assert max(seg[1:]) - min(seg[1:]) <= 1
    w = lambda R: n ** 3 / 3 + n * n / 2 + n / 6 + R * n * n + R * (R + 1) * n + 5 * n ** 3
    w2 = 1.05 * w(n + m) if paired else w(2 * n + m)
    cost = lambda s: max([s[0] * w(n + m)] + [x * w2 for x in s[1:]])
    paper = kkt.kkt_partition_rule(N, P)
    assert cost(seg) <= cost(paper) + 1e-9
    if paired and P > 2:
        assert abs(seg[0] - seg[1]) <= 1 + seg[1] // 10   # nearly equal lengths


def test_plan_flops_follow_pairing(kkt):
    """The paired levels of a plan depend on the SM count only through
    2 x tasks <= SMs; with no SMs nothing is paired."""
    plan = [152, 38, 10, 1]
    a = kkt.kkt_plan_flops(1024, 32, 8, plan, kkt.KKT_PARTITION_BALANCED, sms=0)
    b = kkt.kkt_plan_flops(1024, 32, 8, plan, kkt.KKT_PARTITION_BALANCED, sms=152)
    c = kkt.kkt_plan_flops(1024, 32, 8, plan, kkt.KKT_PARTITION_BALANCED, sms=75)
    assert a["sequential_factor"] == b["sequential_factor"]
    assert a["factor"] != b["factor"]        # level 2 (38 tasks) is paired on 152 SMs
    assert c["factor"] != b["factor"]        # on 75 SMs level 2 is not paired
    d = kkt.kkt_plan_flops(1024, 32, 8, plan, kkt.KKT_PARTITION_PAPER, sms=152)
    e = kkt.kkt_plan_flops(1024, 32, 8, plan, kkt.KKT_PARTITION_PAPER, sms=0)
    assert d == e                            # the paper rule ignores the layout


def test_invalid_arguments(kkt):
    with pytest.raises(kkt.KKTError) as ei:
        kkt.kkt_plan_flops(10, 4, 0, [6, 1])
    assert ei.value.status == kkt.KKT_ERR_PARTITION
    with pytest.raises(kkt.KKTError) as ei:
        kkt.kkt_plan_flops(10, 4, 0, [2, 2])      # last level must be sequential
    assert ei.value.status in (kkt.KKT_ERR_ARG, kkt.KKT_ERR_PARTITION)
    with pytest.raises(kkt.KKTError):
        kkt.kkt_plan_flops(0, 4, 0, [1])
    assert kkt.status_string(kkt.KKT_ERR_NOT_SPD).startswith("pivot")
    for setter, args in ((kkt.kkt_set_refine_tol, (1e-16,)), (kkt.kkt_set_refine_fallback, (4,)),
                         (kkt.kkt_set_persistent, (True,)), (kkt.kkt_set_wait_limit, (1 << 20,)),
                         (kkt.kkt_set_backward_chain, (True,)), (kkt.kkt_set_pairing, (kkt.KKT_PAIR_AUTO_PAIRS,)),
                         (kkt.kkt_set_code_warmup, (True,))):
        with pytest.raises(kkt.KKTError) as ei:   # no handle: refused before any device work
            setter(None, *args)
        assert ei.value.status == kkt.KKT_ERR_ARG
    with pytest.raises(kkt.KKTError) as ei:
        kkt.kkt_factor_ctas_per_task(None, 0)
    assert ei.value.status == kkt.KKT_ERR_ARG


def test_recursive_plan_flops(kkt):
    """Level sizes chain: N_{l+1} = P_l - 1; the flop total grows with the
    fill-in of every partitioned level."""
    one = kkt.kkt_plan_flops(1024, 32, 8, [1])
    two = kkt.kkt_plan_flops(1024, 32, 8, [152, 1])
    three = kkt.kkt_plan_flops(1024, 32, 8, [152, 38, 1])
    assert one["factor"] == one["sequential_factor"]
    assert one["factor"] < two["factor"] < three["factor"] < 2.5 * one["factor"]


def test_bench_launch_names_with_the_backward_chain(kkt, monkeypatch):
    """The bench's per-launch split of a fused step: border copy, one factor
    launch per level (the top one with the corner solve and its backward
    sweep), then either one backward launch per level below the top or one
    launch for all of them, carrying their summed flops."""
    import bench
    monkeypatch.setattr(bench, "device_sms", lambda: 152)
    plan = [256, 128, 64, 32, 16, 8, 4, 2, 1]
    part = kkt.KKT_PARTITION_BALANCED
    n_lv, f_lv = bench.per_launch_flops(kkt, plan, part, 1, chain=False)
    n_ch, f_ch = bench.per_launch_flops(kkt, plan, part, 1, chain=True)
    L = len(plan)
    assert len(n_lv) == 1 + L + (L - 1) and len(n_ch) == 1 + L + 1
    assert n_ch[:1 + L] == n_lv[:1 + L] and f_ch[:1 + L] == f_lv[:1 + L]
    assert n_ch[-1] == f"k_backward_chain (levels {L - 1}..1)"
    assert f_ch[-1] == pytest.approx(sum(f_lv[1 + L:]), rel=1e-12)
    assert all(f > 0 for f in f_lv[1:])
