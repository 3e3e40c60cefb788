"""Parity of the CUDA path (through the C interface) with the FP64 oracle.

Tolerances (derived from FP64 arithmetic, see the design notes):
* factor blocks on well-conditioned inputs: |L_gpu - L_oracle| <= 1e-12 * max|L|
  (both are the unique Cholesky factor; only the rounding order differs);
* solutions on well-conditioned inputs: |x_gpu - x_oracle| <= 1e-11 * max|x|;
* every input: normwise backward error of the GPU solution <= 1e-14 (a
  backward-stable Cholesky solve gives a few units of roundoff) and the
  relative residual within 10x the oracle's own on the same input (or 1e-10);
* ill-conditioned inputs: |x_gpu - x_oracle| <= 10 * u * kappa_est * max|x|, with
  kappa_est the oracle's estimate of kappa_1(Psi) (Hager-Higham).
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


PAIRINGS = ["off", "on"]


def gpu_solve(kkt, D, E, G, R, b, P=1, levels=None, want_factor=False, balanced=False, pairing=None):
    import torch
    N, n = D.shape[0], D.shape[1]
    m = 0 if R is None or np.size(R) == 0 else R.shape[0]
    if balanced:
        h = kkt.kkt_create_plan(N, n, m, levels or ([P, 1] if P > 1 else [1]), kkt.KKT_PARTITION_BALANCED)
    elif levels:
        h = kkt.kkt_create_levels(N, n, m, levels)
    else:
        h = kkt.kkt_create(N, n, m, P)
    try:
        if pairing is not None:
            kkt.kkt_set_pairing(h, {"off": kkt.KKT_PAIR_OFF, "on": kkt.KKT_PAIR_ON,
                                    "auto": kkt.KKT_PAIR_AUTO}[pairing])
        Ed = dev(E) if N > 1 else None
        Gd = dev(G) if m else None
        Rd = dev(R) if m else None
        bd = dev(b)
        kkt.kkt_factor(h, dev(D), Ed, Gd, Rd)
        kkt.kkt_solve(h, bd)
        torch.cuda.synchronize()
        info = kkt.kkt_get_info(h)
        assert info["status"] == 0, info
        F = kkt.kkt_get_factor(h, N, n, m) if want_factor else None
        if F is not None:
            F["seg"] = kkt.kkt_partition(h, 0, 1)     # the handle's level-1 segment lengths
        return bd.cpu().numpy(), F
    finally:
        kkt.kkt_destroy(h)


def check_solution(orc, D, E, G, R, x, b, xo=None, fwd_tol=None):
    A_mv = orc.block_matvec(D, E, G, R, x)
    r = b - A_mv
    Ainf = None
    # normwise backward error with ||Psi||_inf from the blocks
    N, n = D.shape[0], D.shape[1]
    Ds = np.tril(D) + np.swapaxes(np.tril(D, -1), 1, 2)
    rows = np.abs(Ds).sum(axis=2)
    if N > 1:
        rows[1:] += np.abs(E).sum(axis=2)
        rows[:-1] += np.abs(E).sum(axis=1)
    if G.size:
        rows += np.abs(G).sum(axis=1)[:, :]
        grows = np.abs(G).sum(axis=(0, 2)) + np.abs(np.tril(R) + np.tril(R, -1).T).sum(axis=1)
        Ainf = max(rows.max(), grows.max())
    else:
        Ainf = rows.max()
    eta = np.abs(r).max() / (Ainf * np.abs(x).max() + np.abs(b).max())
    assert eta <= 1e-14, f"backward error {eta:.3e}"
    if xo is not None:
        ro = b - orc.block_matvec(D, E, G, R, xo)
        rel_gpu = np.linalg.norm(r) / np.linalg.norm(b)
        rel_orc = np.linalg.norm(ro) / np.linalg.norm(b)
        assert rel_gpu <= max(1e-10, 10 * rel_orc), (rel_gpu, rel_orc)
        if fwd_tol == "kappa":   # the forward-error bound of a backward-stable solve
            fwd_tol = 10 * U * orc.cond_est(D, E, G, R)
        if fwd_tol is not None:
            err = np.abs(x - xo).max() / np.abs(xo).max()
            assert err <= fwd_tol, f"forward difference {err:.3e} > {fwd_tol:.3e}"
    return eta


# ------------------------------------------------------------- config 1

@pytest.mark.parametrize("pairing", PAIRINGS)
@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 8])
def test_known_factor_blocks_and_solution(kkt, orc, P, pairing):
    """N = 16 stages of n = 8, arrow m = 4, Psi = L L^T: factor blocks equal
    the oracle's Algorithm 1 blocks; at P = 1 they equal the generating L.
    Both factor layouts (one CTA per segment, or a pair of CTAs)."""
    D, E, G, R, Lf = gen.known_factor(16, 8, 4, seed=0)
    b = gen.rhs(16 * 8 + 4, 1, seed=1)
    x, F = gpu_solve(kkt, D, E, G, R, b, P=P, want_factor=True, pairing=pairing)
    Fo = orc.par_factor(D, E, G, R, P=P)
    xo = orc.par_solve(Fo, b)
    for key in ("Ld", "Le", "Lw", "Lh", "Lg", "Lr"):
        scale = max(1.0, np.abs(Fo[key]).max() if Fo[key].size else 1.0)
        np.testing.assert_allclose(F[key], Fo[key], rtol=0, atol=1e-12 * scale, err_msg=key)
    if P == 1:
        for key in ("Ld", "Le", "Lg", "Lr"):
            np.testing.assert_allclose(F[key], Lf[key], rtol=0, atol=1e-12)
    np.testing.assert_allclose(x, xo, rtol=0, atol=1e-11 * np.abs(xo).max())
    check_solution(orc, D, E, G, R, x, b, xo)


# ------------------------------------------------------------- edge cases

@pytest.mark.parametrize("N,n,m,P", [
    (1, 8, 4, 1), (2, 8, 0, 1), (3, 1, 0, 2), (3, 1, 1, 2), (5, 3, 2, 3), (9, 5, 0, 5),
    (17, 7, 3, 9), (11, 2, 16, 4), (24, 48, 4, 3), (30, 12, 0, 7), (7, 6, 2, 4), (64, 13, 5, 31),
    (20, 48, 16, 4)])
@pytest.mark.parametrize("pairing", PAIRINGS)
def test_edge_shapes(kkt, orc, N, n, m, P, pairing):
    """Single stage, no arrow, odd and tiny blocks, an arrow wider than the
    block, the largest block, P at its feasibility limit (all segments of
    one stage). Blocks larger than 16 use the IPM generator with a mild
    barrier spread: a random triangular factor of that size is numerically
    singular in FP64 (the oracle breaks down on it too)."""
    if n <= 16:
        D, E, G, R, _ = gen.known_factor(N, n, m, seed=N + n + m)
    else:
        D, E, G, R = gen.ipm(N, n, m, seed=N + n + m, sigma_decades=1.0)
    b = gen.rhs(N * n + m, 1, seed=3)
    x, F = gpu_solve(kkt, D, E, G, R, b, P=P, want_factor=True, pairing=pairing)
    Fo = orc.par_factor(D, E, G, R, P=P)
    xo = orc.par_solve(Fo, b)
    for key in ("Ld", "Le", "Lw", "Lh", "Lg", "Lr"):
        scale = max(1.0, np.abs(Fo[key]).max() if Fo[key].size else 1.0)
        np.testing.assert_allclose(F[key], Fo[key], rtol=0, atol=1e-12 * scale, err_msg=key)
    np.testing.assert_allclose(x, xo, rtol=0, atol=1e-11 * np.abs(xo).max())


@pytest.mark.parametrize("nrhs,ldb", [(1, 1), (3, 3), (16, 16), (17, 20), (40, 40)])
def test_multiple_rhs(kkt, orc, nrhs, ldb):
    """Several right-hand sides (chunks of 16, a leading dimension above nrhs)."""
    import torch
    N, n, m, P = 40, 8, 3, 6
    D, E, G, R, _ = gen.known_factor(N, n, m, seed=2)
    b = gen.rhs(N * n + m, ldb, seed=7).reshape(N * n + m, ldb)
    h = kkt.kkt_create(N, n, m, P)
    try:
        bd = dev(b)
        kkt.kkt_factor(h, dev(D), dev(E), dev(G), dev(R))
        kkt.kkt_solve(h, bd, nrhs=nrhs, ldb=ldb)
        torch.cuda.synchronize()
        x = bd.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)
    Fo = orc.par_factor(D, E, G, R, P=P)
    xo = orc.par_solve(Fo, b[:, :nrhs])
    np.testing.assert_allclose(x[:, :nrhs], xo, rtol=0, atol=1e-11 * np.abs(xo).max())
    np.testing.assert_array_equal(x[:, nrhs:], b[:, nrhs:])   # untouched columns


@pytest.mark.parametrize("N,n,m,levels,nrhs,ldb", [
    (200, 24, 4, [20, 4, 1], 16, 16),   # columns split over four CTAs per task on the deep levels
    (120, 32, 8, [12, 1], 17, 20),      # two chunks (16 + 1), a leading dimension above nrhs
    (90, 20, 0, [9, 2, 1], 40, 40),     # three chunks
])
def test_multiple_rhs_column_split(kkt, orc, N, n, m, levels, nrhs, ldb):
    """Several right-hand sides with CTA-size blocks: a level with few
    segment tasks spreads the columns of a chunk over several CTAs. Each
    column's arithmetic is its own, so the columns agree bit for bit with
    single-column solves, and with the oracle to the parity tolerance."""
    import torch
    D, E, G, R = gen.ipm(N, n, m, seed=91)
    b = gen.rhs(N * n + m, ldb, seed=92).reshape(N * n + m, ldb)
    h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED)
    try:
        Dd, Ed, Gd, Rd = dev(D), dev(E), dev(G) if m else None, dev(R) if m else None
        kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
        bd = dev(b)
        kkt.kkt_solve(h, bd, nrhs=nrhs, ldb=ldb)
        cols = []
        for c in (0, nrhs // 2, nrhs - 1):
            bc = dev(np.ascontiguousarray(b[:, c]))
            kkt.kkt_solve(h, bc)
            cols.append((c, bc))
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        x = bd.cpu().numpy()
        cols = [(c, v.cpu().numpy()) for c, v in cols]
    finally:
        kkt.kkt_destroy(h)
    for c, v in cols:
        np.testing.assert_array_equal(x[:, c], v)
    np.testing.assert_array_equal(x[:, nrhs:], b[:, nrhs:])   # untouched columns
    F = orc.seq_factor(D, E, G, R)
    xo = orc.seq_solve(F, np.ascontiguousarray(b[:, :nrhs]))
    for c in range(0, nrhs, 7):
        check_solution(orc, D, E, G, R, x[:, c], b[:, c], xo[:, c], fwd_tol="kappa")


# ------------------------------------------------------------- IPM-shaped

@pytest.mark.parametrize("pairing", PAIRINGS)
@pytest.mark.parametrize("N,n,m,P", [(128, 32, 8, 1), (128, 32, 8, 16), (200, 24, 4, 13), (96, 12, 0, 20)])
def test_ipm_shaped(kkt, orc, N, n, m, P, pairing):
    """Barrier-scaled blocks (Sigma over 16 decades): backward error at the
    FP64 floor, residual and forward difference as the oracle's."""
    D, E, G, R = gen.ipm(N, n, m, seed=11)
    b = gen.rhs(N * n + m, 1, seed=12)
    x, _ = gpu_solve(kkt, D, E, G, R, b, P=P, pairing=pairing)
    xo = orc.par_solve(orc.par_factor(D, E, G, R, P=P), b)
    check_solution(orc, D, E, G, R, x, b, xo, fwd_tol="kappa")


def test_ipm_full_size_two_levels(kkt, orc):
    """N = 1024 stages of n = 32 with arrow m = 8 (the single-system IPM
    workload), P = 64: complete comparison with the oracle."""
    N, n, m, P = 1024, 32, 8, 64
    D, E, G, R = gen.ipm(N, n, m, seed=0)
    b = gen.rhs(N * n + m, 1, seed=1)
    x, _ = gpu_solve(kkt, D, E, G, R, b, P=P)
    xo = orc.seq_solve(orc.seq_factor(D, E, G, R), b)
    check_solution(orc, D, E, G, R, x, b, xo, fwd_tol="kappa")


# ------------------------------------------------------------- recursion

@pytest.mark.parametrize("pairing", PAIRINGS)
@pytest.mark.parametrize("N,levels", [(16, [4, 2, 1]), (64, [16, 4, 1]), (200, [40, 10, 3, 1]),
                                      (100, [50, 25, 12, 6, 3, 1])])
def test_recursive_levels(kkt, orc, N, levels, pairing):
    """The reduced system partitioned again (same block-tridiagonal-arrow
    form): the solution is unchanged up to rounding."""
    n, m = 6, 2
    D, E, G, R, _ = gen.known_factor(N, n, m, seed=5)
    b = gen.rhs(N * n + m, 2, seed=6)
    x, _ = gpu_solve(kkt, D, E, G, R, b, levels=levels, pairing=pairing)
    xo = orc.seq_solve(orc.seq_factor(D, E, G, R), b)
    np.testing.assert_allclose(x, xo, rtol=0, atol=1e-11 * np.abs(xo).max())


@pytest.mark.parametrize("N,n,m,levels", [(1024, 32, 8, [152, 38, 10, 1]), (300, 12, 4, [60, 12, 1]),
                                           (100, 8, 2, [40, 1]), (64, 6, 0, [20, 6, 1])])
def test_balanced_partition_solution(kkt, orc, N, n, m, levels):
    """Balanced segment lengths (not Eq. (13)) give the same solution."""
    D, E, G, R = gen.ipm(N, n, m, seed=21)
    b = gen.rhs(N * n + m, 1, seed=22)
    x, _ = gpu_solve(kkt, D, E, G, R, b, levels=levels, balanced=True)
    xo = orc.seq_solve(orc.seq_factor(D, E, G, R), b)
    check_solution(orc, D, E, G, R, x, b, xo, fwd_tol="kappa")


def test_balanced_two_level_blocks(kkt, orc):
    """Two balanced levels: the factor blocks are Algorithm 1's on the
    oracle's run with the same segment lengths."""
    N, n, m, P = 40, 5, 2, 9
    D, E, G, R, _ = gen.known_factor(N, n, m, seed=3)
    b = gen.rhs(N * n + m, 1, seed=4)
    x, F = gpu_solve(kkt, D, E, G, R, b, P=P, want_factor=True, balanced=True)
    seg = F["seg"]
    assert seg in (kkt.kkt_partition_balanced(N, n, m, P, False), kkt.kkt_partition_balanced(N, n, m, P, True))
    Fo = orc.par_factor(D, E, G, R, seg_len=seg)
    for key in ("Ld", "Le", "Lw", "Lh", "Lg", "Lr"):
        scale = max(1.0, np.abs(Fo[key]).max() if Fo[key].size else 1.0)
        np.testing.assert_allclose(F[key], Fo[key], rtol=0, atol=1e-12 * scale, err_msg=key)
    np.testing.assert_allclose(x, orc.par_solve(Fo, b), rtol=0, atol=1e-11 * np.abs(x).max())


def test_recursive_factor_is_nested_cholesky(kkt, orc):
    """With three levels the factor is chol of the doubly permuted matrix:
    compare the top-level corner with the dense Cholesky (unique)."""
    import torch
    N, n, m = 25, 3, 2
    levels = [6, 2, 1]
    D, E, G, R, _ = gen.known_factor(N, n, m, seed=8)
    A = orc.assemble_dense(D, E, G, R)
    L = orc.dense_chol(A)
    h = kkt.kkt_create_levels(N, n, m, levels)
    try:
        kkt.kkt_factor(h, dev(D), dev(E), dev(G), dev(R))
        torch.cuda.synchronize()
        with pytest.raises(kkt.KKTError):
            kkt.kkt_get_factor(h, N, n, m)   # only two-level layouts export blocks
    finally:
        kkt.kkt_destroy(h)
    # the corner block of any symmetric permutation that keeps g last is the
    # same: R-hat R-hat^T = Schur complement of the stage part
    x, _ = gpu_solve(kkt, D, E, G, R, np.eye(N * n + m)[:, -m:].copy(), levels=levels)
    S = np.linalg.inv(x[-m:, :])          # (Psi^{-1})_gg^{-1} = Schur complement
    np.testing.assert_allclose(S, L[-m:, -m:] @ L[-m:, -m:].T, rtol=1e-10, atol=1e-12)


# ------------------------------------------------------------- batches

def test_uniform_batch(kkt, orc):
    import torch
    count, N, n, m = 6, 30, 8, 2
    sy = [gen.ipm(N, n, m, seed=s) for s in range(count)]
    Ps = [1, 2, 3, 4, 5, 1]
    h = kkt.kkt_batch_create([N] * count, [n] * count, [m] * count, Ps)
    try:
        D = dev(np.concatenate([s[0].ravel() for s in sy]))
        E = dev(np.concatenate([s[1].ravel() for s in sy]))
        G = dev(np.concatenate([s[2].ravel() for s in sy]))
        R = dev(np.concatenate([s[3].ravel() for s in sy]))
        bs = [gen.rhs(N * n + m, 1, seed=100 + s) for s in range(count)]
        b = dev(np.concatenate(bs))
        kkt.kkt_factor(h, D, E, G, R)
        kkt.kkt_solve(h, b)
        torch.cuda.synchronize()
        x = b.cpu().numpy().reshape(count, N * n + m)
    finally:
        kkt.kkt_destroy(h)
    for s in range(count):
        xo = orc.seq_solve(orc.seq_factor(*sy[s]), bs[s])
        check_solution(orc, *sy[s], x[s], bs[s], xo, fwd_tol=1e-6)


def test_uneven_batch(kkt, orc):
    import torch
    sy = gen.uneven_batch(12, seed=3, N_range=(5, 40))
    Ns = [s[0].shape[0] for s in sy]
    ns = [s[0].shape[1] for s in sy]
    ms = [s[3].shape[0] for s in sy]
    Ps = [max(1, min(4, (N + 1) // 2)) for N in Ns]
    h = kkt.kkt_batch_create(Ns, ns, ms, Ps)
    try:
        off = kkt.kkt_batch_offsets(h, len(sy))
        assert off["D"][-1] == sum(N * n * n for N, n in zip(Ns, ns))
        cat = lambda i: dev(np.concatenate([s[i].ravel() for s in sy] + [np.zeros(1)]))
        bs = [gen.rhs(N * n + m, 1, seed=i) for i, (N, n, m) in enumerate(zip(Ns, ns, ms))]
        b = dev(np.concatenate(bs))
        kkt.kkt_factor(h, cat(0), cat(1), cat(2), cat(3))
        kkt.kkt_solve(h, b)
        torch.cuda.synchronize()
        x = b.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)
    for i, s in enumerate(sy):
        xi = x[off["b"][i]:off["b"][i + 1]]
        xo = orc.seq_solve(orc.seq_factor(*s), bs[i])
        check_solution(orc, *s, xi, bs[i], xo, fwd_tol=1e-6)


# ------------------------------------------------------------- failure, determinism, graphs

@pytest.mark.parametrize("pairing", PAIRINGS)
@pytest.mark.parametrize("P,bad_stage", [(1, 5), (4, 9), (4, 7), (4, 8)])
def test_not_spd_reported(kkt, P, bad_stage, pairing):
    """A negated diagonal block (made on the host) is reported as
    KKT_ERR_NOT_SPD with its natural stage; nothing traps."""
    import torch
    N, n, m = 16, 4, 2
    D, E, G, R, _ = gen.known_factor(N, n, m, seed=0)
    D = D.copy()
    D[bad_stage] = -D[bad_stage]
    h = kkt.kkt_create(N, n, m, P)
    try:
        kkt.kkt_set_pairing(h, kkt.KKT_PAIR_OFF if pairing == "off" else kkt.KKT_PAIR_ON)
        kkt.kkt_factor(h, dev(D), dev(E), dev(G), dev(R))
        torch.cuda.synchronize()
        info = kkt.kkt_get_info(h)
        assert info["status"] == kkt.KKT_ERR_NOT_SPD
        assert info["stage"] == bad_stage and info["system"] == 0
        assert kkt.kkt_get_info(h)["status"] == 0   # cleared
    finally:
        kkt.kkt_destroy(h)


def test_nan_input_reported(kkt):
    import torch
    D, E, G, R, _ = gen.known_factor(8, 3, 1, seed=0)
    D = D.copy()
    D[0, 0, 0] = np.nan
    h = kkt.kkt_create(8, 3, 1, 2)
    try:
        kkt.kkt_factor(h, dev(D), dev(E), dev(G), dev(R))
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == kkt.KKT_ERR_NOT_SPD
    finally:
        kkt.kkt_destroy(h)


def test_bad_arguments(kkt):
    with pytest.raises(kkt.KKTError) as ei:
        kkt.kkt_create(10, 4, 0, 6)
    assert ei.value.status == kkt.KKT_ERR_PARTITION
    with pytest.raises(kkt.KKTError) as ei:
        kkt.kkt_create(10, 49, 0, 1)
    assert ei.value.status == kkt.KKT_ERR_ARG
    h = kkt.kkt_create(10, 4, 0, 2)
    try:
        import torch
        b = torch.zeros(40, dtype=torch.float64, device="cuda")
        with pytest.raises(kkt.KKTError) as ei:
            kkt.kkt_solve(h, b)
        assert ei.value.status == kkt.KKT_ERR_STATE
    finally:
        kkt.kkt_destroy(h)


def test_deterministic_and_graph_capturable(kkt):
    """Fixed summation orders: two runs agree bit for bit; factor + solve
    captured in a CUDA graph and replayed gives the same bits."""
    import torch
    N, n, m, P = 200, 16, 4, 12
    D, E, G, R = gen.ipm(N, n, m, seed=4)
    b = gen.rhs(N * n + m, 1, seed=5)
    h = kkt.kkt_create(N, n, m, P)
    try:
        Dd, Ed, Gd, Rd = dev(D), dev(E), dev(G), dev(R)
        outs = []
        for _ in range(2):
            bd = dev(b)
            kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
            kkt.kkt_solve(h, bd)
            torch.cuda.synchronize()
            outs.append(bd.cpu().numpy())
        np.testing.assert_array_equal(outs[0], outs[1])
        bd = dev(b)
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                kkt.kkt_factor(h, Dd, Ed, Gd, Rd, stream=s)
                kkt.kkt_solve(h, bd, stream=s)
        bd.copy_(dev(b))
        g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(bd.cpu().numpy(), outs[0])
    finally:
        kkt.kkt_destroy(h)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_factor_layouts_bitwise_identical(kkt, precision):
    """The three factor layouts (whole CTA, warp-split CTA, CTA pair) assign
    the same per-element arithmetic to different threads: the factor and
    the (refined, for mixed precision) solution agree bit for bit."""
    import torch
    N, n, m = 600, 24, 6
    levels = [60, 12, 3, 1]
    D, E, G, R = gen.ipm(N, n, m, seed=31)
    b = gen.rhs(N * n + m, 3, seed=32).reshape(N * n + m, 3)
    Dd, Ed, Gd, Rd = dev(D), dev(E), dev(G), dev(R)
    outs = []
    for policy in (kkt.KKT_PAIR_OFF, kkt.KKT_PAIR_ON, kkt.KKT_PAIR_AUTO):
        h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED, precision)
        try:
            kkt.kkt_set_pairing(h, policy)
            bd = dev(b)
            if precision == 0:
                kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
                kkt.kkt_solve(h, bd, nrhs=3, ldb=3)
                x = bd
            else:
                x = torch.zeros_like(bd)
                kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
                kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, bd, x, nrhs=3, sweeps=4, tol=0.0)
            torch.cuda.synchronize()
            assert kkt.kkt_get_info(h)["status"] == 0
            outs.append(x.cpu().numpy())
        finally:
            kkt.kkt_destroy(h)
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])


# ------------------------------------------------------------- autotuned batches

def test_tuned_uneven_batch(kkt, orc):
    """The autotuner's plan (timed on the device) solves an uneven batch like
    the oracle; every chosen level plan is a valid hierarchy."""
    import torch
    sy = gen.uneven_batch(10, seed=9, N_range=(8, 60))
    Ns = [s[0].shape[0] for s in sy]
    ns = [s[0].shape[1] for s in sy]
    ms = [s[3].shape[0] for s in sy]
    h, lv = kkt.kkt_batch_create_tuned(Ns, ns, ms)
    try:
        assert len(lv) == len(sy) and min(lv) >= 1
        for i, N in enumerate(Ns):
            Nl = N
            for l in range(1, lv[i] + 1):
                seg = kkt.kkt_partition(h, i, l)
                assert sum(seg) + len(seg) - 1 == Nl and min(seg) >= 1
                Nl = len(seg) - 1
            assert len(kkt.kkt_partition(h, i, lv[i])) == 1     # sequential top level
        off = kkt.kkt_batch_offsets(h, len(sy))
        cat = lambda i: dev(np.concatenate([s[i].ravel() for s in sy] + [np.zeros(1)]))
        bs = [gen.rhs(N * n + m, 1, seed=40 + i) for i, (N, n, m) in enumerate(zip(Ns, ns, ms))]
        b = dev(np.concatenate(bs))
        kkt.kkt_factor(h, cat(0), cat(1), cat(2), cat(3))
        kkt.kkt_solve(h, b)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        x = b.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)
    for i, s in enumerate(sy):
        xi = x[off["b"][i]:off["b"][i + 1]]
        xo = orc.seq_solve(orc.seq_factor(*s), bs[i])
        check_solution(orc, *s, xi, bs[i], xo, fwd_tol=1e-6)


def test_tuned_plans_follow_the_batch(kkt):
    """Many short systems fill the GPU on their own: the tuner keeps them
    sequential (no fill-in). A single long system gets a partitioned plan."""
    h, lv = kkt.kkt_batch_create_tuned([40] * 2048, [8] * 2048, [2] * 2048)
    kkt.kkt_destroy(h)
    assert max(lv) == 1
    h, lv = kkt.kkt_batch_create_tuned([4096], [16], [4])
    try:
        assert lv[0] >= 2 and len(kkt.kkt_partition(h, 0, 1)) > 1
    finally:
        kkt.kkt_destroy(h)


# ------------------------------------------------------------- fused factor + solve

@pytest.mark.parametrize("pairing", PAIRINGS)
@pytest.mark.parametrize("N,n,m,levels", [(16, 8, 4, [4, 1]), (128, 32, 8, [16, 4, 1]), (200, 24, 4, [20, 5, 1]),
                                          (64, 6, 2, [16, 4, 1]), (40, 12, 0, [6, 1]), (30, 20, 3, [1]),
                                          (1024, 32, 8, [152, 38, 10, 3, 1])])
def test_factor_solve_fused(kkt, orc, N, n, m, levels, pairing):
    """The right-hand side bordered onto the arrow: one pass gives the
    solution of factor + solve (to rounding), and the factor it leaves
    solves further right-hand sides and refines like kkt_factor's."""
    import torch
    D, E, G, R = gen.ipm(N, n, m, seed=41)
    b = gen.rhs(N * n + m, 1, seed=42)
    b2 = gen.rhs(N * n + m, 1, seed=43)
    h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED)
    try:
        kkt.kkt_set_pairing(h, kkt.KKT_PAIR_OFF if pairing == "off" else kkt.KKT_PAIR_ON)
        Dd, Ed, Gd, Rd = dev(D), dev(E) if N > 1 else None, dev(G) if m else None, dev(R) if m else None
        x_two = dev(b)
        kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
        kkt.kkt_solve(h, x_two)
        x_one = dev(b)
        kkt.kkt_factor_solve(h, Dd, Ed, Gd, Rd, x_one)
        x_again = dev(b2)
        kkt.kkt_solve(h, x_again)                     # the fused pass's factor, a new right-hand side
        xr = torch.zeros_like(x_again)
        kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, dev(b2), xr, sweeps=1, tol=0.0)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        with pytest.raises(kkt.KKTError):
            kkt.kkt_get_factor(h, N, n, m)            # blocks of the bordered pass are not exported
    finally:
        kkt.kkt_destroy(h)
    x_two, x_one, x_again, xr = (t.cpu().numpy() for t in (x_two, x_one, x_again, xr))
    xo = orc.seq_solve(orc.seq_factor(D, E, G, R), b)
    check_solution(orc, D, E, G, R, x_one, b, xo, fwd_tol="kappa")
    np.testing.assert_allclose(x_one, x_two, rtol=0, atol=1e-9 * np.abs(x_two).max())
    xo2 = orc.seq_solve(orc.seq_factor(D, E, G, R), b2)
    check_solution(orc, D, E, G, R, x_again, b2, xo2, fwd_tol="kappa")
    check_solution(orc, D, E, G, R, xr, b2, xo2, fwd_tol="kappa")


def test_factor_solve_fused_batch(kkt, orc):
    """Uneven batch, systems of different depths and block sizes."""
    import torch
    sy = gen.uneven_batch(9, seed=12, N_range=(6, 50))
    Ns = [s[0].shape[0] for s in sy]
    ns = [s[0].shape[1] for s in sy]
    ms = [s[3].shape[0] for s in sy]
    Ps = [max(1, min(5, (N + 1) // 2)) if i % 3 else 1 for i, N in enumerate(Ns)]
    h = kkt.kkt_batch_create(Ns, ns, ms, Ps)
    try:
        off = kkt.kkt_batch_offsets(h, len(sy))
        cat = lambda i: dev(np.concatenate([s[i].ravel() for s in sy] + [np.zeros(1)]))
        bs = [gen.rhs(N * n + m, 1, seed=70 + i) for i, (N, n, m) in enumerate(zip(Ns, ns, ms))]
        b = dev(np.concatenate(bs))
        kkt.kkt_factor_solve(h, cat(0), cat(1), cat(2), cat(3), b)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
        x = b.cpu().numpy()
    finally:
        kkt.kkt_destroy(h)
    for i, s in enumerate(sy):
        xi = x[off["b"][i]:off["b"][i + 1]]
        xo = orc.seq_solve(orc.seq_factor(*s), bs[i])
        check_solution(orc, *s, xi, bs[i], xo, fwd_tol=1e-6)


def test_factor_solve_reports_breakdown(kkt):
    """A bordered pass reports a non-SPD pivot block like kkt_factor."""
    import torch
    N, n, m = 16, 4, 2
    D, E, G, R, _ = gen.known_factor(N, n, m, seed=0)
    D = D.copy()
    D[9] = -D[9]
    h = kkt.kkt_create(N, n, m, 4)
    try:
        kkt.kkt_factor_solve(h, dev(D), dev(E), dev(G), dev(R), dev(gen.rhs(N * n + m, 1, seed=1)))
        torch.cuda.synchronize()
        info = kkt.kkt_get_info(h)
        assert info["status"] == kkt.KKT_ERR_NOT_SPD and info["stage"] == 9
    finally:
        kkt.kkt_destroy(h)


@pytest.mark.parametrize("N,n,m,levels,nrhs", [
    (120, 24, 6, [12, 3, 1], 1),     # one system, bordered pass: chunked transfer, 4 level-1 streams
    (40, 20, 3, [3, 1], 1),          # fewer segments than chunks
    (60, 8, 4, [6, 1], 1),           # warp-per-task blocks
    (50, 17, 0, [1], 1),             # one level: the plain path
    (90, 24, 6, [9, 1], 3),          # several right-hand sides: the plain path
])
def test_factor_solve_host_matches_device(kkt, orc, N, n, m, levels, nrhs):
    """kkt_factor_solve from host buffers (page-locked torch tensors, read in
    place by the factorization, and plain NumPy arrays, copied in chunks)
    returns, bit for bit, what kkt_factor_solve returns on device copies of
    the same inputs: the chunked transfer only reorders launches of
    independent segments."""
    import torch
    D, E, G, R = gen.ipm(N, n, m, seed=81)
    b = gen.rhs(N * n + m, nrhs, seed=82).reshape(N * n + m, -1) if nrhs > 1 else gen.rhs(N * n + m, 1, seed=82)
    h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED)
    try:
        bd = dev(b)
        kkt.kkt_factor_solve(h, dev(D), dev(E) if N > 1 else None, dev(G) if m else None, dev(R) if m else None, bd)
        torch.cuda.synchronize()
        x_dev = bd.cpu().numpy()
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hb = pin(b)
        kkt.kkt_factor_solve_host(h, pin(D), pin(E) if N > 1 else None, pin(G) if m else None,
                                  pin(R) if m else None, hb)
        torch.cuda.synchronize()
        x_pinned = hb.numpy().copy()
        nb = np.ascontiguousarray(b).copy()
        kkt.kkt_factor_solve_host(h, np.ascontiguousarray(D), np.ascontiguousarray(E) if N > 1 else None,
                                  np.ascontiguousarray(G) if m else None, np.ascontiguousarray(R) if m else None, nb)
        torch.cuda.synchronize()
        assert kkt.kkt_get_info(h)["status"] == 0
    finally:
        kkt.kkt_destroy(h)
    np.testing.assert_array_equal(x_pinned, x_dev)
    np.testing.assert_array_equal(nb, x_dev)
    for c in range(nrhs):
        bc = b.reshape(b.shape[0], -1)[:, c]
        xc = x_dev.reshape(x_dev.shape[0], -1)[:, c]
        check_solution(orc, D, E, G, R, xc, bc, orc.seq_solve(orc.seq_factor(D, E, G, R), bc), fwd_tol="kappa")


def test_factor_solve_host_other_handles(kkt, orc):
    """The host entry point on handles without the chunked transfer: a batch,
    a mixed-precision handle (no bordered pass) and a system of one stage;
    each returns what kkt_factor_solve returns on device copies."""
    import torch
    sy = gen.uneven_batch(5, seed=31, N_range=(6, 40))
    Ns = [s[0].shape[0] for s in sy]
    ns = [s[0].shape[1] for s in sy]
    ms = [s[3].shape[0] for s in sy]
    cat = lambda i: np.concatenate([s[i].ravel() for s in sy] + [np.zeros(1)])
    bs = np.concatenate([gen.rhs(N * n + m, 1, seed=90 + i) for i, (N, n, m) in enumerate(zip(Ns, ns, ms))])
    cases = [(kkt.kkt_batch_create(Ns, ns, ms, [max(1, min(3, (N + 1) // 2)) for N in Ns]),
              [cat(0), cat(1), cat(2), cat(3)], bs)]
    D, E, G, R = gen.ipm(64, 24, 4, seed=33)
    cases.append((kkt.kkt_create_plan(64, 24, 4, [8, 1], kkt.KKT_PARTITION_BALANCED, kkt.KKT_MIXED_FP32),
                  [D, E, G, R], gen.rhs(64 * 24 + 4, 1, seed=34)))
    D1, E1, G1, R1 = gen.ipm(1, 20, 3, seed=35)
    cases.append((kkt.kkt_create(1, 20, 3, 1), [D1, None, G1, R1], gen.rhs(23, 1, seed=36)))
    for h, arrs, b in cases:
        try:
            bd = dev(b)
            kkt.kkt_factor_solve(h, *[dev(a) if a is not None else None for a in arrs], bd)
            torch.cuda.synchronize()
            hb = np.ascontiguousarray(b).copy()
            kkt.kkt_factor_solve_host(h, *[np.ascontiguousarray(a) if a is not None else None for a in arrs], hb)
            torch.cuda.synchronize()
            assert kkt.kkt_get_info(h)["status"] == 0
            np.testing.assert_array_equal(hb, bd.cpu().numpy())
        finally:
            kkt.kkt_destroy(h)


def test_bench_workload_every_candidate_plan(kkt, orc):
    """The single-system workload exactly as the benchmark times it: its
    seeds and shapes, every level plan its search may pick, kkt_factor_solve
    captured into a CUDA graph and replayed after an L2-evicting write. Each
    plan's x against the oracle's sequential solution, and two replays
    bitwise equal."""
    import torch
    import bench
    D, E, G, R, b = bench.workload(0)
    xo = orc.seq_solve(orc.seq_factor(D, E, G, R), b)
    Dd, Ed, Gd, Rd, b0 = (dev(a) for a in (D, E, G, R, b))
    flush = torch.empty(bench.L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    part = kkt.KKT_PARTITION_BALANCED
    plans = bench.candidate_plans(kkt, part)
    assert plans
    for plan in plans:
        h = kkt.kkt_create_plan(bench.N_STAGES, bench.N_BLOCK, bench.M_ARROW, plan, part)
        try:
            bd = b0.clone()
            for _ in range(2):
                bd.copy_(b0)
                kkt.kkt_factor_solve(h, Dd, Ed, Gd, Rd, bd)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            cap = torch.cuda.Stream()
            cap.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(cap):
                with torch.cuda.graph(g, stream=cap):
                    kkt.kkt_factor_solve(h, Dd, Ed, Gd, Rd, bd)
            torch.cuda.current_stream().wait_stream(cap)
            xs = []
            for _ in range(2):
                bd.copy_(b0)
                flush.zero_()
                g.replay()
                torch.cuda.synchronize()
                xs.append(bd.cpu().numpy())
            assert kkt.kkt_get_info(h)["status"] == 0, plan
            np.testing.assert_array_equal(xs[0], xs[1])
            check_solution(orc, D, E, G, R, xs[0], b, xo, fwd_tol="kappa")
        finally:
            kkt.kkt_destroy(h)


@pytest.mark.parametrize("N,n,m,levels", [(120, 24, 6, [12, 3, 1]), (60, 8, 4, [6, 1]), (50, 17, 0, [1])])
def test_factor_solve_host_page_locked_graph(kkt, N, n, m, levels):
    """Page-locked inputs read in place, captured into a CUDA graph: two
    replays give the device path's x bit for bit. With only some inputs
    page-locked the call falls back to copying, with the same result."""
    import torch
    D, E, G, R = gen.ipm(N, n, m, seed=83)
    b = gen.rhs(N * n + m, 1, seed=84)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED)
    try:
        bd = dev(b)
        kkt.kkt_factor_solve(h, dev(D), dev(E) if N > 1 else None, dev(G) if m else None, dev(R) if m else None, bd)
        torch.cuda.synchronize()
        x_dev = bd.cpu().numpy()
        hD, hE, hG, hR = pin(D), pin(E) if N > 1 else None, pin(G) if m else None, pin(R) if m else None
        hb0, hb = pin(b), pin(b)
        kkt.kkt_factor_solve_host(h, hD, hE, hG, hR, hb)      # eager, before capture
        torch.cuda.synchronize()
        np.testing.assert_array_equal(hb.numpy(), x_dev)
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        cap.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cap):
            with torch.cuda.graph(g, stream=cap):
                kkt.kkt_factor_solve_host(h, hD, hE, hG, hR, hb)
        torch.cuda.current_stream().wait_stream(cap)
        for _ in range(2):
            hb.copy_(hb0)
            g.replay()
            torch.cuda.synchronize()
            np.testing.assert_array_equal(hb.numpy(), x_dev)
        del g
        # D page-locked, the rest pageable: the copy path
        nb = np.ascontiguousarray(b).copy()
        kkt.kkt_factor_solve_host(h, hD, np.ascontiguousarray(E) if N > 1 else None,
                                  np.ascontiguousarray(G) if m else None, np.ascontiguousarray(R) if m else None, nb)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(nb, x_dev)
        assert kkt.kkt_get_info(h)["status"] == 0
    finally:
        kkt.kkt_destroy(h)


def test_factor_solve_host_page_locked_allocates_no_input_copies(kkt):
    """With page-locked inputs the host entry point keeps only a device copy
    of b: the device's free memory drops by far less than the 19 MB of D, E,
    G, R (a copy of them is made only by a call that needs one)."""
    import torch
    N, n, m = 1024, 32, 8
    D, E, G, R = gen.ipm(N, n, m, seed=85)
    b = gen.rhs(N * n + m, 1, seed=86)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h = kkt.kkt_create_plan(N, n, m, [152, 38, 10, 1], kkt.KKT_PARTITION_BALANCED)
    try:
        bd = dev(b)
        kkt.kkt_factor_solve(h, dev(D), dev(E), dev(G), dev(R), bd)   # modules loaded, handle warm
        torch.cuda.synchronize()
        hD, hE, hG, hR, hb = pin(D), pin(E), pin(G), pin(R), pin(b)
        free0 = torch.cuda.mem_get_info()[0]
        kkt.kkt_factor_solve_host(h, hD, hE, hG, hR, hb)
        torch.cuda.synchronize()
        drop = free0 - torch.cuda.mem_get_info()[0]
        inputs = sum(a.nbytes for a in (D, E, G, R))
        assert inputs > 16 << 20
        assert drop <= 8 << 20, (drop, inputs)
        np.testing.assert_array_equal(hb.numpy(), bd.cpu().numpy())
        assert kkt.kkt_get_info(h)["status"] == 0
    finally:
        kkt.kkt_destroy(h)
