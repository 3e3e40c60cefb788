"""The adjoint kernel (kkt_solve_adjoint) and the autograd function against
the FP64 oracle's adjoint and against central finite differences."""
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


@pytest.mark.parametrize("N,n,m,levels,precision,nrhs", [
    (16, 8, 4, [4, 1], 0, 1), (64, 12, 3, [8, 3, 1], 0, 2), (40, 6, 0, [1], 0, 1),
    (128, 32, 8, [16, 1], 1, 1), (100, 16, 4, [10, 1], 2, 3)])
def test_adjoint_matches_oracle(kkt, orc, N, n, m, levels, precision, nrhs):
    import torch
    D, E, G, R = gen.ipm(N, n, m, seed=7, sigma_decades=3.0)
    b = gen.rhs(N * n + m, nrhs, seed=8)
    xbar = gen.rhs(N * n + m, nrhs, seed=9)
    h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED, precision)
    try:
        Dd, Ed, Gd, Rd = dev(D), dev(E), dev(G) if m else None, dev(R) if m else None
        kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
        x = torch.zeros_like(dev(b))
        kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, dev(b), x, sweeps=6, tol=0.0)
        bbar = torch.empty_like(x)
        dD, dE = torch.empty_like(Dd), torch.empty_like(Ed)
        dG = torch.empty_like(Gd) if m else None
        dR = torch.empty_like(Rd) if m else None
        kkt.kkt_solve_adjoint(h, x, dev(xbar), bbar, dD, dE, dG, dR, Dd, Ed, Gd, Rd, sweeps=6)
        torch.cuda.synchronize()
        got = [bbar.cpu().numpy(), dD.cpu().numpy(), dE.cpu().numpy()]
        if m:
            got += [dG.cpu().numpy(), dR.cpu().numpy()]
    finally:
        kkt.kkt_destroy(h)
    xo = orc.seq_solve(orc.seq_factor(D, E, G, R), b)
    ref = orc.adjoint(D, E, G, R, xo, xbar)
    ref = [ref[0], ref[1], ref[2]] + ([ref[3], ref[4]] if m else [])
    for name, g, r in zip(("bbar", "dD", "dE", "dG", "dR"), got, ref):
        np.testing.assert_allclose(g.reshape(r.shape), r, rtol=0, atol=1e-9 * max(1.0, np.abs(r).max()),
                                   err_msg=name)


@pytest.mark.parametrize("sigma,levels,abs_tol", [(1.0, [16, 1], 1e-6), (8.0, [1], 1e-5)])
def test_autograd_function_and_finite_differences(kkt, sigma, levels, abs_tol):
    """L = 1/2 ||x||^2 through the differentiable solve (the differentiable-MPC
    workload shape: N = 256, n = 32, m = 8): autograd gradients against
    central differences (h = 1e-6) of the same GPU forward on 64 sampled
    entries of D (lower), E, G, R and b. With Sigma over 16 decades (the
    workload's, kappa ~ 1e9) the rounding of the forward solve moves L by
    far more than h^2 terms do, and the central difference itself is only
    good to a few 1e-6 absolute (measured with the FP64 oracle's forward
    on the same samples: at most 3.2e-6, where Richardson extrapolation does
    not help, so it is noise, not truncation); the exact check at that
    conditioning is the comparison with the oracle's adjoint
    (test_gpu_bench_shapes)."""
    import torch
    N, n, m = 256, 32, 8
    D, E, G, R = gen.ipm(N, n, m, seed=3, sigma_decades=sigma)
    b = gen.rhs(N * n + m, 1, seed=4)
    solver = kkt.KKTSolver(N, n, m, levels=levels)
    try:
        Dd, Ed, Gd, Rd, bd = (dev(a).requires_grad_() for a in (D, E, G, R, b))
        x = kkt.kkt_solve_differentiable(solver, Dd, Ed, Gd, Rd, bd)
        loss = 0.5 * (x * x).sum()
        loss.backward()
        grads = [t.grad.cpu().numpy() for t in (Dd, Ed, Gd, Rd, bd)]

        def L(arrs):
            with torch.no_grad():
                xx = kkt.kkt_solve_differentiable(solver, *[dev(a) for a in arrs])
                return 0.5 * float((xx * xx).sum())

        rng = np.random.default_rng(1)
        base = [D, E, G, R, b]
        hstep = 1e-6
        L0 = L(base)
        for s in range(64):
            which = s % 5
            a = base[which]
            if which == 0:
                j, r = rng.integers(N), rng.integers(n)
                pos = (j, r, rng.integers(r + 1))
            elif which == 3:
                r = rng.integers(m)
                pos = (r, rng.integers(r + 1))
            else:
                pos = tuple(rng.integers(k) for k in a.shape)
            plus = [c.copy() for c in base]
            minus = [c.copy() for c in base]
            plus[which][pos] += hstep
            minus[which][pos] -= hstep
            fd = (L(plus) - L(minus)) / (2 * hstep)
            g = grads[which][pos]
            assert fd == pytest.approx(g, rel=1e-4, abs=abs_tol * max(1.0, abs(L0))), (which, pos, fd, g)
    finally:
        solver.close()
