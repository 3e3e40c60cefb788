"""Mixed precision (FP64 pivots and Schur accumulators, FP32 panel trsm and
Schur dot products, or TF32/BF16 Schur products on the tensor cores, FP32
substitutions) with FP64 iterative refinement, through the C interface,
against the FP64 oracle.

The gate is the FP64 one: after refinement the normwise backward error is
<= 1e-14 and the solution agrees with the oracle's to the accuracy the
conditioning allows; the unrefined (raw FP32-factor) error is reported and
bounded loosely.
"""
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


def eta(orc, D, E, G, R, x, b):
    r = b - orc.block_matvec(D, E, G, R, x)
    A = orc.assemble_dense(D, E, G, R) if D.shape[0] * D.shape[1] <= 4000 else None
    if A is not None:
        nrm = np.abs(A).sum(axis=1).max()
    else:
        Ds = np.tril(D) + np.swapaxes(np.tril(D, -1), 1, 2)
        rows = np.abs(Ds).sum(axis=2)
        rows[1:] += np.abs(E).sum(axis=2)
        rows[:-1] += np.abs(E).sum(axis=1)
        if G.size:
            rows += np.abs(G).sum(axis=1)
        nrm = rows.max()
        if G.size:
            nrm = max(nrm, (np.abs(G).sum(axis=(0, 2)) + np.abs(np.tril(R) + np.tril(R, -1).T).sum(axis=1)).max())
    return np.abs(r).max() / (nrm * np.abs(x).max() + np.abs(b).max())


def run(kkt, D, E, G, R, b, levels, precision, sweeps, tol=1e-15, pair_off=False):
    import torch
    N, n, _ = D.shape
    m = R.shape[0]
    h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED, precision)
    try:
        if pair_off:   # whole-CTA segment tasks (paired tasks keep the CUDA-core products)
            kkt.kkt_set_pairing(h, kkt.KKT_PAIR_OFF)
        Dd, Ed, Gd, Rd = dev(D), dev(E), dev(G) if m else None, dev(R) if m else None
        kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
        bd = dev(b)
        xd = torch.zeros_like(bd)
        kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, bd, xd, sweeps=sweeps, tol=tol)
        raw = dev(b)
        kkt.kkt_solve(h, raw)          # the unrefined solution with the same factor
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        etas = [float(kkt.kkt_refine_eta(h, s)[0]) for s in range(sweeps)]
        np.testing.assert_array_equal(bd.cpu().numpy(), b)   # b is read-only
        return xd.cpu().numpy(), raw.cpu().numpy(), etas
    finally:
        kkt.kkt_destroy(h)


@pytest.mark.parametrize("name,N,n,m,levels,kind", [
    ("ipm n32 m8", 256, 32, 8, [16, 1], "ipm8"),
    ("ipm n32 m8 deep", 512, 32, 8, [64, 16, 4, 1], "ipm8"),
    ("ipm n12 m0", 150, 12, 0, [1], "ipm6"),
    ("ipm n24 m4", 120, 24, 4, [8, 1], "ipm6"),
    ("ipm n48 m4", 60, 48, 4, [6, 1], "ipm6"),
    ("raceline n6 m2", 2048, 6, 2, [64, 8, 1], "race"),
])
@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_refinement_reaches_fp64(kkt, orc, name, N, n, m, levels, kind, precision):
    if kind == "race":
        D, E, G, R = gen.raceline(N, n, m, seed=3)
    else:
        D, E, G, R = gen.ipm(N, n, m, seed=3, sigma_decades=8.0 if kind == "ipm8" else 6.0)
    b = gen.rhs(N * n + m, 1, seed=4)
    x, raw, etas = run(kkt, D, E, G, R, b, levels, precision, sweeps=10, tol=0.0)
    e = eta(orc, D, E, G, R, x, b)
    assert e <= 1e-14, (name, e, etas)
    assert etas[-1] <= 1e-14, etas
    e_raw = eta(orc, D, E, G, R, raw, b)
    assert e_raw <= 1e-5, e_raw                 # raw FP32-factor solve: loose bound, reported
    xo = orc.seq_solve(orc.seq_factor(D, E, G, R), b)
    ro = b - orc.block_matvec(D, E, G, R, xo)
    r = b - orc.block_matvec(D, E, G, R, x)
    assert np.linalg.norm(r) <= max(1e-10 * np.linalg.norm(b), 10 * np.linalg.norm(ro))
    assert np.abs(x - xo).max() <= 1e-5 * np.abs(xo).max()


def test_refinement_multiple_rhs_and_early_stop(kkt, orc):
    """17 right-hand sides (two chunks); once converged the remaining sweeps
    leave x unchanged on the device."""
    import torch
    N, n, m = 128, 16, 4
    D, E, G, R = gen.ipm(N, n, m, seed=8)
    b = gen.rhs(N * n + m, 17, seed=9)
    h = kkt.kkt_create_plan(N, n, m, [8, 1], kkt.KKT_PARTITION_BALANCED, kkt.KKT_MIXED_FP32)
    try:
        Dd, Ed, Gd, Rd, bd = dev(D), dev(E), dev(G), dev(R), dev(b)
        kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
        x8 = torch.zeros_like(bd)
        kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, bd, x8, sweeps=8, tol=1e-13)
        etas8 = [kkt.kkt_refine_eta(h, s, 1)[0] for s in range(8)]
        x3 = torch.zeros_like(bd)
        kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, bd, x3, sweeps=3, tol=1e-13)
        torch.cuda.synchronize()
        x8, x3 = x8.cpu().numpy(), x3.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)
    np.testing.assert_array_equal(x8, x3)          # converged within 3 sweeps, then stopped
    # after convergence the recorded eta stays that of the converging sweep
    conv = next(s for s in range(8) if etas8[s] <= 1e-13)
    assert 0.0 < etas8[conv] <= 1e-13
    assert all(etas8[s] == etas8[conv] for s in range(conv, 8))
    assert all(etas8[s] > 1e-13 for s in range(conv))
    for c in range(17):
        assert eta(orc, D, E, G, R, x8[:, c], b[:, c]) <= 1e-13


def test_fp64_handle_refinement(kkt, orc):
    """With an FP64 factor one correction sweep is the plain solve plus a
    residual check, and refinement keeps the backward error at the floor."""
    N, n, m = 200, 24, 4
    D, E, G, R = gen.ipm(N, n, m, seed=12)
    b = gen.rhs(N * n + m, 1, seed=13)
    x, raw, etas = run(kkt, D, E, G, R, b, [13, 1], 0, sweeps=2)
    np.testing.assert_allclose(x, raw, rtol=0, atol=1e-9 * np.abs(raw).max())
    assert eta(orc, D, E, G, R, x, b) <= 1e-14


def test_mixed_uneven_batch(kkt, orc):
    import torch
    sy = gen.uneven_batch(10, seed=5, N_range=(20, 60))
    Ns = [s[0].shape[0] for s in sy]
    ns = [s[0].shape[1] for s in sy]
    ms = [s[3].shape[0] for s in sy]
    h = kkt.kkt_batch_create(Ns, ns, ms, None, kkt.KKT_MIXED_FP32)
    try:
        off = kkt.kkt_batch_offsets(h, len(sy))
        cat = lambda i: dev(np.concatenate([s[i].ravel() for s in sy] + [np.zeros(1)]))
        bs = [gen.rhs(N * n + m, 1, seed=i) for i, (N, n, m) in enumerate(zip(Ns, ns, ms))]
        Dd, Ed, Gd, Rd = cat(0), cat(1), cat(2), cat(3)
        b = dev(np.concatenate(bs))
        x = torch.zeros_like(b)
        kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
        kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, b, x, sweeps=6, tol=1e-15)
        torch.cuda.synchronize()
        x = x.cpu().numpy()
        etas = kkt.kkt_refine_eta(h, 5, len(sy))
    finally:
        kkt.kkt_destroy(h)
    for i, s in enumerate(sy):
        xi = x[off["b"][i]:off["b"][i + 1]]
        assert eta(orc, *s, xi, bs[i]) <= 1e-14, (i, etas)


def test_refinement_multiple_rhs_cta_blocks(kkt, orc):
    """Mixed factor, CTA-size blocks and 20 right-hand sides (two chunks): the
    FP32 correction solves split a chunk's columns over several CTAs per task
    on the reduced levels; every column reaches the FP64 gate and agrees, bit
    for bit, with its own single-column refinement (every sweep run: tol < 0,
    so that no stop decision, which looks at a chunk's columns together,
    differs between the two)."""
    import torch
    N, n, m = 150, 24, 4
    D, E, G, R = gen.ipm(N, n, m, seed=21, sigma_decades=4.0)
    b = gen.rhs(N * n + m, 20, seed=22).reshape(N * n + m, 20)
    h = kkt.kkt_create_plan(N, n, m, [15, 3, 1], kkt.KKT_PARTITION_BALANCED, kkt.KKT_MIXED_FP32_ALL)
    try:
        Dd, Ed, Gd, Rd = dev(D), dev(E), dev(G), dev(R)
        kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
        x = torch.zeros((N * n + m, 20), dtype=torch.float64, device="cuda")
        kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, dev(b), x, sweeps=5, tol=-1.0)
        x1 = torch.zeros(N * n + m, dtype=torch.float64, device="cuda")
        kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, dev(np.ascontiguousarray(b[:, 13])), x1, sweeps=5, tol=-1.0)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        x, x1 = x.cpu().numpy(), x1.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)
    np.testing.assert_array_equal(x[:, 13], x1)
    for c in (0, 13, 19):
        r = b[:, c] - orc.block_matvec(D, E, G, R, x[:, c])
        xo = orc.seq_solve(orc.seq_factor(D, E, G, R), b[:, c])
        assert np.abs(x[:, c] - xo).max() <= 1e-5 * np.abs(xo).max()
        assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(b[:, c])


@pytest.mark.parametrize("N,n,m,levels", [(128, 32, 8, [1]), (90, 48, 4, [1]), (120, 48, 4, [8, 1]),
                                          (100, 40, 0, [1])])
@pytest.mark.parametrize("precision", [3, 4])
def test_tensor_core_schur_products(kkt, orc, N, n, m, levels, precision):
    """KKT_MIXED_TF32 / KKT_MIXED_BF16: the Schur products of blocks n >= 32
    on the tensor cores. The unrefined solution differs from the FP32
    CUDA-core path's (a different product arithmetic ran) and is as accurate
    as the operand rounding allows; after refinement the FP64 gates hold."""
    D, E, G, R = gen.ipm(N, n, m, seed=31, sigma_decades=6.0)
    b = gen.rhs(N * n + m, 1, seed=32)
    x, raw, etas = run(kkt, D, E, G, R, b, levels, precision, sweeps=12, tol=1e-16, pair_off=True)
    _, raw32, _ = run(kkt, D, E, G, R, b, levels, kkt.KKT_MIXED_FP32, sweeps=1, tol=1e-16, pair_off=True)
    assert not np.array_equal(raw, raw32)
    e_raw = eta(orc, D, E, G, R, raw, b)
    assert e_raw <= (1e-3 if precision == 4 else 1e-4), e_raw
    e = eta(orc, D, E, G, R, x, b)
    assert e <= 1e-14, (e, etas)
    xo = orc.seq_solve(orc.seq_factor(D, E, G, R), b)
    r = b - orc.block_matvec(D, E, G, R, x)
    ro = b - orc.block_matvec(D, E, G, R, xo)
    assert np.linalg.norm(r) <= max(1e-10 * np.linalg.norm(b), 10 * np.linalg.norm(ro)), etas


@pytest.mark.parametrize("kind,N,n,m,sigma", [("race", 2048, 6, 2, 10.0), ("ipm", 200, 48, 4, 11.0),
                                              ("ipm", 200, 32, 8, 12.0)])
def test_refinement_stall_falls_back_to_pcg(kkt, orc, kind, N, n, m, sigma):
    """Barrier scaling beyond the workloads' (Sigma over 20-24 decades): the
    stationary refinement with the FP32 factor stalls well above the FP64
    level (its residual stays far more than 10x the oracle's); with the
    fallback enabled the stalled systems continue with conjugate gradients
    preconditioned by the same factor and reach the FP64 gates."""
    import torch
    gen_fn = gen.raceline if kind == "race" else gen.ipm
    D, E, G, R = gen_fn(N, n, m, seed=5, sigma_decades=sigma)
    b = gen.rhs(N * n + m, 1, seed=6)
    xo = orc.seq_solve(orc.seq_factor(D, E, G, R), b)
    ro = np.linalg.norm(b - orc.block_matvec(D, E, G, R, xo))
    ratios = {}
    for cg in (0, 12):
        h = kkt.kkt_create_plan(N, n, m, [1], kkt.KKT_PARTITION_BALANCED, kkt.KKT_MIXED_FP32_ALL)
        try:
            if cg:
                kkt.kkt_set_refine_fallback(h, cg)
            Dd, Ed, Gd, Rd = dev(D), dev(E), dev(G), dev(R)
            kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
            x = torch.zeros(N * n + m, dtype=torch.float64, device="cuda")
            kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, dev(b), x, sweeps=10, tol=1e-16)
            torch.cuda.synchronize()
            assert kkt.kkt_get_info(h)["status"] == 0
            eta_dev = float(kkt.kkt_refine_eta(h, 9)[0])
            x = x.cpu().numpy()
        finally:
            kkt.kkt_destroy(h)
        ratios[cg] = np.linalg.norm(b - orc.block_matvec(D, E, G, R, x)) / ro
        if cg:
            assert orc.block_backward_error(D, E, G, R, x, b) <= 1e-14
            assert eta_dev <= 1e-14
    assert ratios[0] > 10.0, ratios      # the classic sweeps stall
    assert ratios[12] <= 10.0, ratios    # the fallback reaches the FP64 path's residual


@pytest.mark.parametrize("N,n,m,levels", [(60, 6, 2, [6, 1]), (80, 12, 4, [8, 1]), (30, 16, 0, [3, 1]),
                                          (40, 48, 4, [4, 1]), (50, 33, 3, [5, 1])])
def test_one_column_residual_matches_chunked(kkt, orc, N, n, m, levels):
    """A one-column refinement (the residual kernel that stages the blocks in
    shared memory) and the same column inside a chunk of three (the kernel
    for several columns) run the same substitutions on plans with fill-in
    rows and the same residual arithmetic term for term: x and every sweep's
    eta agree bit for bit, for packed small blocks (several stages per warp),
    two rows per lane (n > 32) and m = 0."""
    import torch
    D, E, G, R = gen.ipm(N, n, m, seed=N + n, sigma_decades=4.0)
    b = gen.rhs(N * n + m, 3, seed=5).reshape(N * n + m, 3)
    h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED, kkt.KKT_MIXED_FP32_ALL)
    try:
        Dd, Ed = dev(D), dev(E)
        Gd, Rd = (dev(G), dev(R)) if m else (None, None)
        kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
        x3 = torch.zeros((N * n + m, 3), dtype=torch.float64, device="cuda")
        kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, dev(b), x3, sweeps=4, tol=-1.0)
        x1 = torch.zeros(N * n + m, dtype=torch.float64, device="cuda")
        kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, dev(np.ascontiguousarray(b[:, 1])), x1, sweeps=4, tol=-1.0)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        x3, x1 = x3.cpu().numpy(), x1.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)
    np.testing.assert_array_equal(x3[:, 1], x1)
    assert orc.block_backward_error(D, E, G, R, x1, b[:, 1]) <= 1e-14


def test_one_column_residual_uneven_batch(kkt, orc):
    """The one-column residual on an uneven batch (block sizes 6 to 48, one
    launch over every system's chunks) against the chunked kernel, bit for
    bit, and the oracle's backward error."""
    import torch
    shapes = [(40, 6, 2, 4), (33, 12, 0, 3), (25, 48, 4, 3), (60, 24, 4, 6), (17, 33, 3, 2), (9, 16, 1, 2)]
    systems = [gen.ipm(N, n, m, seed=70 + i, sigma_decades=4.0) for i, (N, n, m, _) in enumerate(shapes)]
    Ns, ns, ms, Ps = (list(v) for v in zip(*shapes))
    cat = lambda i: dev(np.concatenate([s[i].ravel() for s in systems] + [np.zeros(1)]))
    D, E, G, R = cat(0), cat(1), cat(2), cat(3)
    rows = sum(N * n + m for N, n, m, _ in shapes)
    b = gen.rhs(rows, 3, seed=9).reshape(rows, 3)
    h = kkt.kkt_batch_create(Ns, ns, ms, Ps, kkt.KKT_MIXED_FP32_ALL)
    try:
        kkt.kkt_factor(h, D, E, G, R)
        x3 = torch.zeros((rows, 3), dtype=torch.float64, device="cuda")
        kkt.kkt_solve_refined(h, D, E, G, R, dev(b), x3, sweeps=4, tol=-1.0)
        x1 = torch.zeros(rows, dtype=torch.float64, device="cuda")
        kkt.kkt_solve_refined(h, D, E, G, R, dev(np.ascontiguousarray(b[:, 2])), x1, sweeps=4, tol=-1.0)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        off = kkt.kkt_batch_offsets(h, len(shapes))["b"]
        x3, x1 = x3.cpu().numpy(), x1.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)
    np.testing.assert_array_equal(x3[:, 2], x1)
    for i, s in enumerate(systems):
        xi, bi = x1[off[i]:off[i + 1]], b[off[i]:off[i + 1], 2]
        assert orc.block_backward_error(*s, xi, bi) <= 1e-14
