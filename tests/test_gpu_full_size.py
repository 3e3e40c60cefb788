"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times: the whole 4096-system uneven batch and the whole
512-system differentiable batch, drawn on the device by the benchmark's own
generator (gen.device, the same seeds), planned by the autotuner, factored
with the persistent schedule or per-level launches and solved (FP64) or
refined to the FP64 path's accuracy (FP32 mixed). The outputs of sampled
systems, one or more of every block-size class, are copied back together
with their inputs and checked against the FP64 oracle one by one:
* backward error (the oracle's block definition) <= 1e-14;
* relative residual within 10x the oracle's own on the same input;
* |x - x_oracle| <= 10 u kappa_est |x_oracle| (Hager-Higham estimate);
* for the differentiable batch, bbar and every block gradient against the
  oracle's FP64 adjoint on the same x, within 10 u kappa_est of each
  output's largest entry.
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


def host_system(D, E, G, R, off, s, N, n, m):
    """System s's blocks from the packed device arrays, as the oracle takes them."""
    return (D[off["D"][s]:off["D"][s + 1]].cpu().numpy().reshape(N, n, n),
            E[off["E"][s]:off["E"][s + 1]].cpu().numpy().reshape(max(N - 1, 0), n, n),
            G[off["G"][s]:off["G"][s + 1]].cpu().numpy().reshape(N, m, n),
            R[off["R"][s]:off["R"][s + 1]].cpu().numpy().reshape(m, m))


def gates(orc, sy, x, b):
    D, E, G, R = sy
    eta = orc.block_backward_error(D, E, G, R, x, b)
    assert eta <= 1e-14, f"backward error {eta:.3e}"
    xo = orc.seq_solve(orc.seq_factor(D, E, G, R), b)
    r = np.linalg.norm(b - orc.block_matvec(D, E, G, R, x))
    ro = np.linalg.norm(b - orc.block_matvec(D, E, G, R, xo))
    assert r <= max(1e-10 * np.linalg.norm(b), 10 * ro), (r, ro)
    kap = orc.cond_est(D, E, G, R)
    err = np.abs(x - xo).max() / np.abs(xo).max()
    assert err <= 10 * U * kap, f"forward difference {err:.3e} > 10 u kappa = {10 * U * kap:.3e}"
    return kap


def sample_per_class(Ns, ns, ms, per_class=2):
    idx = {}
    for i, key in enumerate(zip(ns, ms)):
        idx.setdefault(key, [])
        if len(idx[key]) < per_class:
            idx[key].append(i)
    # the longest system too (its chain is the longest)
    return sorted({i for v in idx.values() for i in v} | {int(np.argmax(Ns))})


@pytest.mark.parametrize("path", ["fp64", "mixed_persist"])
def test_uneven4096_full_batch(kkt, orc, path):
    import torch
    import bench
    import gen.device as gdev
    spec = bench.BATCHES["uneven4096"]
    Ns, ns, ms = bench.batch_shapes("uneven4096")
    count = len(Ns)
    D, E, G, R = gdev.batch(Ns, ns, ms, seed=bench.rank_seed(11, 0), kind=spec["kind"],
                            sigma_decades=spec["sigma"], psd_couplings=spec["psd"])
    off = gdev.offsets(Ns, ns, ms)
    b = gdev.rhs(int(off["b"][-1]), 1, seed=bench.rank_seed(12, 0))
    mixed = path.startswith("mixed")
    prec = kkt.KKT_MIXED_FP32_ALL if mixed else kkt.KKT_FP64
    h, lv = kkt.kkt_batch_create_tuned(Ns, ns, ms, prec)
    try:
        if path.endswith("_persist"):
            kkt.kkt_set_persistent(h, True)
        kkt.kkt_factor(h, D, E, G, R)
        if mixed:
            x = torch.zeros_like(b)
            kkt.kkt_solve_refined(h, D, E, G, R, b, x, sweeps=8, tol=1e-16)
        else:
            x = b.clone()
            kkt.kkt_solve(h, x)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        assert kkt.kkt_batch_offsets(h, count)["b"][-1] == off["b"][-1]
    finally:
        kkt.kkt_destroy(h)
    for s in sample_per_class(Ns, ns, ms):
        N, n, m = Ns[s], ns[s], ms[s]
        sy = host_system(D, E, G, R, off, s, N, n, m)
        gates(orc, sy, x[off["b"][s]:off["b"][s + 1]].cpu().numpy(), b[off["b"][s]:off["b"][s + 1]].cpu().numpy())


@pytest.mark.parametrize("path", ["fp64", "mixed"])
def test_adjoint512_full_batch(kkt, orc, path):
    import torch
    import bench
    import gen.device as gdev
    spec = bench.BATCHES["adjoint512"]
    Ns, ns, ms = bench.batch_shapes("adjoint512")
    count = len(Ns)
    D, E, G, R = gdev.batch(Ns, ns, ms, seed=bench.rank_seed(11, 0), kind=spec["kind"],
                            sigma_decades=spec["sigma"])
    off = gdev.offsets(Ns, ns, ms)
    b = gdev.rhs(int(off["b"][-1]), 1, seed=bench.rank_seed(12, 0))
    mixed = path == "mixed"
    prec = kkt.KKT_MIXED_FP32_ALL if mixed else kkt.KKT_FP64
    h, lv = kkt.kkt_batch_create_tuned(Ns, ns, ms, prec)
    try:
        kkt.kkt_factor(h, D, E, G, R)
        if mixed:
            x = torch.zeros_like(b)
            kkt.kkt_solve_refined(h, D, E, G, R, b, x, sweeps=8, tol=1e-16)
            kkt.kkt_set_refine_tol(h, 1e-16)
        else:
            x = b.clone()
            kkt.kkt_solve(h, x)
        bb = torch.empty_like(b)
        gD, gE, gG, gR = (torch.empty_like(t) for t in (D, E, G, R))
        kkt.kkt_solve_adjoint(h, x, x, bb, gD, gE, gG, gR, D=D, E=E, G=G, R=R, sweeps=8 if mixed else 1)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
    finally:
        kkt.kkt_destroy(h)
    for s in (0, 255, 511):
        N, n, m = Ns[s], ns[s], ms[s]
        sy = host_system(D, E, G, R, off, s, N, n, m)
        xs = x[off["b"][s]:off["b"][s + 1]].cpu().numpy()
        kap = gates(orc, sy, xs, b[off["b"][s]:off["b"][s + 1]].cpu().numpy())
        ref = orc.adjoint(*sy, xs, xs)
        got = dict(bbar=bb[off["b"][s]:off["b"][s + 1]], dD=gD[off["D"][s]:off["D"][s + 1]],
                   dE=gE[off["E"][s]:off["E"][s + 1]], dG=gG[off["G"][s]:off["G"][s + 1]],
                   dR=gR[off["R"][s]:off["R"][s + 1]])
        for name, r in zip(("bbar", "dD", "dE", "dG", "dR"), ref):
            g = got[name].cpu().numpy().reshape(r.shape)
            err = np.abs(g - r).max() / np.abs(r).max()
            assert err <= 10 * U * kap, f"system {s} {name}: {err:.3e} > {10 * U * kap:.3e}"
