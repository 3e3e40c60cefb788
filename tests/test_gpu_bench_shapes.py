"""Parity at the benchmark workloads' shapes and plans.

The batched workloads of the benchmark (race line, uneven batch,
differentiable solve) run here through the level plans the benchmark uses,
with inputs drawn on the host by `gen` (the same recipes the benchmark draws
on the device) so that the FP64 oracle sees the same values. Every system is
checked against the oracle:
* G1: normwise backward error (oracle's block definition) <= 1e-14;
* G2: relative residual within 10x the oracle's own on the same input (or
  1e-10);
* G3: |x - x_oracle| <= 10 u kappa_est |x_oracle| on sampled systems, kappa_est
  the oracle's Hager-Higham estimate of kappa_1(Psi).
The device's own backward error (kkt_refine_eta, which scales by row sums of
|Psi| formed from 20-bit truncated entries) is compared with the oracle's on
the same x.
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


def pack(systems):
    """Device arrays of a batch in the packed layout (system after system)."""
    cat = lambda i: dev(np.concatenate([s[i].ravel() for s in systems] + [np.zeros(1)]))
    return cat(0), cat(1), cat(2), cat(3)


def check_system(orc, s, x, b, xo=None, kappa=None):
    D, E, G, R = s
    eta = orc.block_backward_error(D, E, G, R, x, b)
    assert eta <= 1e-14, f"backward error {eta:.3e}"
    if xo is not None:
        rg = np.linalg.norm(b - orc.block_matvec(D, E, G, R, x)) / np.linalg.norm(b)
        ro = np.linalg.norm(b - orc.block_matvec(D, E, G, R, xo)) / np.linalg.norm(b)
        assert rg <= max(1e-10, 10 * ro), (rg, ro)
    if kappa is not None:
        err = np.abs(x - xo).max() / np.abs(xo).max()
        assert err <= 10 * U * kappa, f"forward difference {err:.3e} > 10 u kappa = {10 * U * kappa:.3e}"
    return eta


def run_batch(kkt, h, systems, bs, path, sweeps=8, tol=1e-16):
    """One benchmark step of `path` on handle h: the FP64 path factors and
    solves, the mixed path factors and refines to the FP64 path's accuracy
    (eta <= 1e-16 or until eta stops falling), as the benchmark does."""
    import torch
    D, E, G, R = pack(systems)
    b = dev(np.concatenate(bs))
    kkt.kkt_factor(h, D, E, G, R)
    if path == "mixed":
        x = torch.zeros_like(b)
        kkt.kkt_solve_refined(h, D, E, G, R, b, x, sweeps=sweeps, tol=tol)
    else:
        x = b.clone()
        kkt.kkt_solve(h, x)
    torch.cuda.synchronize()
    info = kkt.kkt_get_info(h)
    assert info["status"] == 0, info
    return x.cpu().numpy(), (D, E, G, R, b)


def split(kkt, h, x, count):
    off = kkt.kkt_batch_offsets(h, count)["b"]
    return [x[off[i]:off[i + 1]] for i in range(count)]


# ------------------------------------------------------------ race line (64 x N = 8192, n = 6, m = 2)

@pytest.mark.parametrize("path", ["fp64", "mixed"])
def test_raceline_batch_on_the_tuned_plan(kkt, orc, path):
    """The race-line workload: 64 systems of N = 8192 stages, n = 6, m = 2,
    Sigma over 16 decades, on the plan the autotuner picks for exactly these
    shapes (a multi-level plan with thousands of level-1 segments); FP64, and
    FP32 mixed with FP64 refinement to the FP64 path's accuracy (G1 and G2
    both hold: a refinement stopped at eta <= 1e-14 leaves a residual about
    100x the FP64 one and fails G2)."""
    count, N, n, m = 64, 8192, 6, 2
    systems = [gen.raceline(N, n, m, seed=s, sigma_decades=8.0) for s in range(count)]
    bs = [gen.rhs(N * n + m, 1, seed=1000 + s) for s in range(count)]
    prec = kkt.KKT_MIXED_FP32_ALL if path == "mixed" else kkt.KKT_FP64
    h, lv = kkt.kkt_batch_create_tuned([N] * count, [n] * count, [m] * count, prec)
    try:
        assert min(lv) >= 3, lv          # the recursive plan, not the sequential method
        P1 = sum(len(kkt.kkt_partition(h, s, 1)) for s in range(count))
        assert P1 >= 1000, P1
        x, _ = run_batch(kkt, h, systems, bs, path)
        xs = split(kkt, h, x, count)
        eta_dev = kkt.kkt_refine_eta(h, 7, count) if path == "mixed" else None
    finally:
        kkt.kkt_destroy(h)
    for s in range(count):
        sample = s in (0, 21, 63)
        xo = orc.seq_solve(orc.seq_factor(*systems[s]), bs[s]) if sample else None
        kap = orc.cond_est(*systems[s]) if sample else None
        check_system(orc, systems[s], xs[s], bs[s], xo, kap)
    if eta_dev is not None:
        assert eta_dev.max() <= 2e-15


# ------------------------------------------------------------ uneven batch (slice of the 4096 shapes)

def uneven_shapes():
    """The uneven workload's shapes (4096 systems), as the benchmark draws them."""
    import bench
    return bench.batch_shapes("uneven4096")


def test_uneven_batch_tuner_picks_the_sequential_method(kkt):
    """On the full 4096-system uneven batch the tuner keeps every system
    sequential (P = 1), which is the plan the slices below run."""
    Ns, ns, ms = uneven_shapes()
    for prec in (kkt.KKT_FP64, kkt.KKT_MIXED_FP32_ALL):
        h, lv = kkt.kkt_batch_create_tuned(Ns, ns, ms, prec)
        kkt.kkt_destroy(h)
        assert max(lv) == 1, prec


@pytest.mark.parametrize("path", ["fp64", "mixed"])
def test_uneven_batch_slice(kkt, orc, path):
    """A slice of the uneven workload covering every (n, m) class, 16 systems
    each, in the sequential plan (P = 1), with the workload's generator
    (Sigma over +-6 decades, PSD-embedded couplings)."""
    Ns, ns, ms = uneven_shapes()
    idx = []
    for n in (12, 24, 48):
        for m in (0, 4):
            idx += [i for i in range(len(Ns)) if ns[i] == n and ms[i] == m][:16]
    systems = [gen.ipm(Ns[i], ns[i], ms[i], seed=i, sigma_decades=6.0, psd_couplings=True) for i in idx]
    bs = [gen.rhs(Ns[i] * ns[i] + ms[i], 1, seed=5000 + i) for i in idx]
    sN, sn, sm = [Ns[i] for i in idx], [ns[i] for i in idx], [ms[i] for i in idx]
    prec = kkt.KKT_MIXED_FP32_ALL if path == "mixed" else kkt.KKT_FP64
    h = kkt.kkt_batch_create(sN, sn, sm, [1] * len(idx), prec)
    try:
        x, _ = run_batch(kkt, h, systems, bs, path)
        xs = split(kkt, h, x, len(idx))
    finally:
        kkt.kkt_destroy(h)
    for k in range(len(idx)):
        sample = k % 8 == 0
        xo = orc.seq_solve(orc.seq_factor(*systems[k]), bs[k])
        kap = orc.cond_est(*systems[k]) if sample else None
        check_system(orc, systems[k], xs[k], bs[k], xo, kap)


# ------------------------------------------------------------ differentiable solve (N = 256, n = 32, m = 8)

@pytest.mark.parametrize("path", ["fp64", "mixed"])
def test_adjoint_bench_shape_full_sigma(kkt, orc, path):
    """The differentiable workload's systems (N = 256, n = 32, m = 8, Sigma
    over 16 decades, kappa ~ 1e9) in the sequential plan the tuner picks for
    that batch, loss 1/2 ||x||^2 (xbar = x): bbar and every block gradient
    against the oracle's FP64 adjoint on the same x, within 10 u kappa_est of
    each output's largest entry. The mixed path (FP32 factor, both solves
    refined to the rounding floor, as the benchmark runs it) meets the same
    bound as the FP64 path."""
    import torch
    count, N, n, m = 4, 256, 32, 8
    prec = kkt.KKT_MIXED_FP32_ALL if path == "mixed" else kkt.KKT_FP64
    h, lv = kkt.kkt_batch_create_tuned([N] * 512, [n] * 512, [m] * 512, prec)
    kkt.kkt_destroy(h)
    assert max(lv) == 1
    systems = [gen.ipm(N, n, m, seed=300 + s, sigma_decades=8.0) for s in range(count)]
    bs = [gen.rhs(N * n + m, 1, seed=400 + s) for s in range(count)]
    h = kkt.kkt_batch_create([N] * count, [n] * count, [m] * count, [1] * count, prec)
    try:
        x, (D, E, G, R, b) = run_batch(kkt, h, systems, bs, path)
        kkt.kkt_set_refine_tol(h, 1e-16)   # the adjoint stops where the forward solve does
        xd = dev(x)
        bbar = torch.empty_like(xd)
        gD, gE, gG, gR = (torch.empty_like(t) for t in (D, E, G, R))
        kkt.kkt_solve_adjoint(h, xd, xd, bbar, gD, gE, gG, gR, D, E, G, R, sweeps=8 if path == "mixed" else 1)
        torch.cuda.synchronize()
        off = kkt.kkt_batch_offsets(h, count)
        got = dict(bbar=bbar.cpu().numpy(), dD=gD.cpu().numpy(), dE=gE.cpu().numpy(), dG=gG.cpu().numpy(),
                   dR=gR.cpu().numpy())
    finally:
        kkt.kkt_destroy(h)
    xs = [x[off["b"][s]:off["b"][s + 1]] for s in range(count)]
    for s in range(count):
        Ds, Es, Gs, Rs = systems[s]
        kap = orc.cond_est(Ds, Es, Gs, Rs)
        check_system(orc, systems[s], xs[s], bs[s])
        ref = orc.adjoint(Ds, Es, Gs, Rs, xs[s], xs[s])
        sl = dict(bbar=got["bbar"][off["b"][s]:off["b"][s + 1]],
                  dD=got["dD"][off["D"][s]:off["D"][s + 1]].reshape(Ds.shape),
                  dE=got["dE"][off["E"][s]:off["E"][s + 1]].reshape(Es.shape),
                  dG=got["dG"][off["G"][s]:off["G"][s + 1]].reshape(Gs.shape),
                  dR=got["dR"][off["R"][s]:off["R"][s + 1]].reshape(Rs.shape))
        for name, r in zip(("bbar", "dD", "dE", "dG", "dR"), ref):
            g = sl[name].reshape(r.shape)
            err = np.abs(g - r).max() / np.abs(r).max()
            assert err <= 10 * U * kap, f"system {s} {name}: {err:.3e} > {10 * U * kap:.3e}"


# ------------------------------------------------------------ the device's backward error against the oracle's

@pytest.mark.parametrize("N,n,m,kind", [(256, 32, 8, "ipm"), (120, 48, 4, "ipm"), (2048, 6, 2, "raceline"),
                                        (300, 12, 0, "ipm")])
def test_device_eta_matches_oracle(kkt, orc, N, n, m, kind):
    """kkt_refine_eta after one refinement sweep of a mixed factor (x is the
    raw FP32-factor solution, eta ~ 1e-8, far above rounding) equals the
    oracle's backward error on the same x to 2e-5 relative: the device scales
    by row sums of |Psi| built from entries truncated to 20 mantissa bits and
    summed in FP32, so it may read up to a few parts in 1e6 high. With the
    FP64 factor both are at rounding level and agree to within the rounding
    of the residual itself (2 gamma_K, K terms per row)."""
    import torch
    gen_fn = gen.ipm if kind == "ipm" else gen.raceline
    D, E, G, R = gen_fn(N, n, m, seed=N + n, sigma_decades=6.0)
    b = gen.rhs(N * n + m, 1, seed=77)
    for prec in (kkt.KKT_MIXED_FP32_ALL, kkt.KKT_FP64):
        h = kkt.kkt_create_plan(N, n, m, [1], kkt.KKT_PARTITION_BALANCED, prec)
        try:
            Dd, Ed = dev(D), dev(E)
            Gd, Rd = (dev(G), dev(R)) if m else (None, None)
            kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
            x = torch.zeros(N * n + m, dtype=torch.float64, device="cuda")
            kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, dev(b), x, sweeps=1, tol=0.0)
            torch.cuda.synchronize()
            eta_dev = float(kkt.kkt_refine_eta(h, 0)[0])
            xh = x.cpu().numpy()
        finally:
            kkt.kkt_destroy(h)
        eta_orc = orc.block_backward_error(D, E, G, R, xh, b)
        if prec == kkt.KKT_FP64:
            K = 3 * n + m + 1
            gam = K * U / (1 - K * U)
            assert abs(eta_dev - eta_orc) <= 2 * gam, (eta_dev, eta_orc)
        else:
            assert eta_orc > 1e-12            # far above rounding
            assert abs(eta_dev - eta_orc) <= 2e-5 * eta_orc, (eta_dev, eta_orc)
            assert eta_dev >= eta_orc * (1 - 1e-9)   # the truncated norm never reads low
