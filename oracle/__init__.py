"""FP64 CPU oracle for the block-tridiagonal-arrow KKT solve (arXiv 2511.00946).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline may import this package; the product library never does. It shares
no code with the CUDA path. The arithmetic lives in ``kkt_oracle.c`` (plain C
loops, FP64); this module compiles it with gcc, loads it with ctypes and adds
the definitions the tests need around it:

* ``assemble_dense`` writes out Psi of Eq. (3) from its blocks;
* ``permutation`` is the reordering of Sec. 3.1 (segment stages first, then
  the separators, then the global variable), as a list of stage indices;
* ``dense_factor_blocks`` reads the blocks of a dense lower factor of the
  permuted matrix back into the natural-order block arrays that
  ``par_factor`` returns, so the two can be compared block by block.

Parity pins (see tests/test_oracle_pins.py): dense Cholesky against closed
forms and brute force, recovery of a known generating factor, equality of the
partitioned factor with the dense Cholesky of the permuted matrix, the flop
counts of Table 1, the speedup table (Table 2) and the backward error.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kkt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libkkt_oracle.so")
_lib = None
_lock = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 into oracle/_build (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.orc_dense_chol.argtypes = [ctypes.c_int, _dp, _dp]
            L.orc_dense_solve.argtypes = [ctypes.c_int, _dp, _dp]
            L.orc_partition.argtypes = [ctypes.c_int, ctypes.c_int, _ip]
            L.orc_seq_factor.argtypes = [ctypes.c_int] * 3 + [_dp] * 8
            L.orc_seq_solve.argtypes = [ctypes.c_int] * 3 + [_dp] * 5 + [ctypes.c_int]
            L.orc_par_factor.argtypes = [ctypes.c_int] * 4 + [_ip] + [_dp] * 11
            L.orc_par_solve.argtypes = [ctypes.c_int] * 4 + [_ip] + [_dp] * 7 + [ctypes.c_int, _dp]
            L.orc_seq_batch.argtypes = [ctypes.c_int] * 7 + [_dp] * 5 + [_ip]
            L.orc_flops_reset.argtypes = []
            L.orc_flops_get.argtypes = [_dp, _dp]
            _lib = L
    return _lib


def _p(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _nonempty(a: np.ndarray) -> np.ndarray:
    # ctypes needs a valid pointer even for zero-sized blocks (m = 0, N = 1).
    return a if a.size else np.zeros(1)


# --------------------------------------------------------------------------
# definitions written out (Eq. (3) and the permutation of Sec. 3.1)
# --------------------------------------------------------------------------

def assemble_dense(D, E, G, R) -> np.ndarray:
    """Psi of Eq. (3): stage blocks on the diagonal, Psi_{j+1,j} = E[j] below
    it, the arrow row Psi_{g,j} = G[j] and the corner Psi_gg = R; symmetric."""
    N, n, _ = D.shape
    m = 0 if R is None else R.shape[0]
    dim = N * n + m
    A = np.zeros((dim, dim))
    for j in range(N):
        A[j * n:(j + 1) * n, j * n:(j + 1) * n] = np.tril(D[j]) + np.tril(D[j], -1).T
        if j + 1 < N:
            A[(j + 1) * n:(j + 2) * n, j * n:(j + 1) * n] = E[j]
            A[j * n:(j + 1) * n, (j + 1) * n:(j + 2) * n] = E[j].T
        if m:
            A[N * n:, j * n:(j + 1) * n] = G[j]
            A[j * n:(j + 1) * n, N * n:] = G[j].T
    if m:
        A[N * n:, N * n:] = np.tril(R) + np.tril(R, -1).T
    return A


def segment_starts(seg_len) -> list[int]:
    """First stage of every segment; the separator of segment k >= 1 is the
    stage right before it."""
    f = [0]
    for k in range(1, len(seg_len)):
        f.append(f[-1] + seg_len[k - 1] + 1)
    return f


def permutation(N: int, seg_len) -> list[int]:
    """Stage order of the permuted matrix P Psi P^T (Sec. 3.1): every
    segment's stages in segment order, then the separators s_2..s_P; the
    global block goes last (not listed)."""
    f = segment_starts(seg_len)
    order = []
    for k, L in enumerate(seg_len):
        order += list(range(f[k], f[k] + L))
    order += [f[k] - 1 for k in range(1, len(seg_len))]
    assert sorted(order) == list(range(N))
    return order


def permute_dense(A: np.ndarray, N: int, n: int, seg_len) -> tuple[np.ndarray, np.ndarray]:
    """Return (P A P^T, idx) where idx lists the natural row of each permuted row."""
    idx = np.concatenate([np.arange(j * n, (j + 1) * n) for j in permutation(N, seg_len)]
                         + [np.arange(N * n, A.shape[0])]).astype(np.int64)
    return A[np.ix_(idx, idx)], idx


def dense_factor_blocks(Lp: np.ndarray, N: int, n: int, m: int, seg_len) -> dict:
    """Read a dense lower factor of P Psi P^T into the natural-order block
    arrays of ``par_factor`` (Ld, Le, Lw, Lh, Lg, Lr)."""
    order = permutation(N, seg_len)
    pos = {j: t for t, j in enumerate(order)}  # stage -> block row in permuted order
    f = segment_starts(seg_len)
    P = len(seg_len)

    def blk(rj, cj):  # block of L-hat at (row stage, column stage), permuted positions
        r, c = pos[rj], pos[cj]
        return Lp[r * n:(r + 1) * n, c * n:(c + 1) * n].copy()

    out = {k: np.zeros((N, n, n)) for k in ("Ld", "Lw", "Lh")}
    out["Le"] = np.zeros((max(N - 1, 0), n, n))
    out["Lg"] = np.zeros((N, m, n))
    for j in range(N):
        out["Ld"][j] = blk(j, j)
        if m:
            c = pos[j]
            out["Lg"][j] = Lp[N * n:, c * n:(c + 1) * n]
    for k in range(P):
        fk, lk = f[k], f[k] + seg_len[k] - 1
        for j in range(fk, lk):
            out["Le"][j] = blk(j + 1, j)
        if k < P - 1:
            out["Le"][lk] = blk(lk + 1, lk)          # F-hat_k
        if k >= 1:
            for j in range(fk, lk + 1):
                out["Lw"][j] = blk(fk - 1, j)        # W = L-hat(s_k, j)
        if 1 <= k < P - 1:
            out["Lh"][fk - 1] = blk(f[k + 1] - 1, fk - 1)  # H_k = L-hat(s_{k+1}, s_k)
    out["Lr"] = Lp[N * n:, N * n:].copy()
    return out


# --------------------------------------------------------------------------
# wrappers over the C oracle
# --------------------------------------------------------------------------

def dense_chol(A) -> np.ndarray:
    """O1: textbook dense Cholesky. Raises on breakdown."""
    A = _f64(A)
    L = np.zeros_like(A)
    st = lib().orc_dense_chol(A.shape[0], _p(A), _p(L))
    if st:
        raise np.linalg.LinAlgError(f"dense Cholesky breakdown at column {st - 1}")
    return L


def dense_solve(L, b) -> np.ndarray:
    """O1: x = (L L^T)^{-1} b for each column of b."""
    L = _f64(L)
    b = _f64(b)
    cols = b.reshape(b.shape[0], -1)
    out = np.empty_like(cols)
    for c in range(cols.shape[1]):
        v = np.ascontiguousarray(cols[:, c])
        lib().orc_dense_solve(L.shape[0], _p(L), _p(v))
        out[:, c] = v
    return out.reshape(b.shape)


def partition(N: int, P: int) -> list[int]:
    """Eq. (13) with the balance ratio 19/7 (Sec. 3.3). Raises ValueError when
    no partition exists (P > floor((N+1)/2))."""
    seg = (ctypes.c_int * max(P, 1))()
    st = lib().orc_partition(N, P, seg)
    if st:
        raise ValueError(f"no partition of N={N} into P={P} segments")
    return list(seg[:P])


def _shapes(D, E, G, R):
    D = _f64(D)
    N, n, _ = D.shape
    E = _f64(E) if N > 1 else np.zeros((0, n, n))
    m = 0 if R is None else np.asarray(R).shape[0]
    G = _f64(G) if m else np.zeros((N, 0, n))
    R = _f64(R) if m else np.zeros((0, 0))
    return D, E, G, R, N, n, m


def seq_factor(D, E, G, R) -> dict:
    """O2: sequential block Cholesky in natural order. Raises on breakdown."""
    D, E, G, R, N, n, m = _shapes(D, E, G, R)
    out = dict(Ld=np.zeros((N, n, n)), Le=np.zeros((max(N - 1, 0), n, n)),
               Lg=np.zeros((N, m, n)), Lr=np.zeros((m, m)))
    st = lib().orc_seq_factor(N, n, m, _p(D), _p(_nonempty(E)), _p(_nonempty(G)), _p(_nonempty(R)),
                              _p(out["Ld"]), _p(_nonempty(out["Le"])), _p(_nonempty(out["Lg"])),
                              _p(_nonempty(out["Lr"])))
    if st:
        raise np.linalg.LinAlgError(f"sequential factor breakdown, code {st}")
    out.update(N=N, n=n, m=m)
    return out


def seq_solve(F: dict, b) -> np.ndarray:
    """O2: x = Psi^{-1} b with a ``seq_factor`` result; b is (dim,) or (dim, nrhs)."""
    b = _f64(b)
    x = np.ascontiguousarray(b.reshape(b.shape[0], -1).copy())
    lib().orc_seq_solve(F["N"], F["n"], F["m"], _p(F["Ld"]), _p(_nonempty(F["Le"])),
                        _p(_nonempty(F["Lg"])), _p(_nonempty(F["Lr"])), _p(x), x.shape[1])
    return x.reshape(b.shape)


def par_factor(D, E, G, R, P: int | None = None, seg_len=None, flops: bool = False) -> dict:
    """O3: Algorithm 1 on the partition of Eq. (13) (or the given segment
    lengths). Returns the natural-order block arrays (see kkt_oracle.c) plus
    ``seg_len`` and, if asked, per-segment and sequential-phase flops."""
    D, E, G, R, N, n, m = _shapes(D, E, G, R)
    if seg_len is None:
        seg_len = partition(N, P)
    P = len(seg_len)
    segs = (ctypes.c_int * P)(*seg_len)
    out = dict(Ld=np.zeros((N, n, n)), Le=np.zeros((max(N - 1, 0), n, n)), Lw=np.zeros((N, n, n)),
               Lh=np.zeros((N, n, n)), Lg=np.zeros((N, m, n)), Lr=np.zeros((m, m)))
    fl = np.zeros(2 * (P + 1))
    st = lib().orc_par_factor(N, n, m, P, segs, _p(D), _p(_nonempty(E)), _p(_nonempty(G)),
                              _p(_nonempty(R)), _p(out["Ld"]), _p(_nonempty(out["Le"])),
                              _p(out["Lw"]), _p(out["Lh"]), _p(_nonempty(out["Lg"])),
                              _p(_nonempty(out["Lr"])), _p(fl))
    if st:
        raise np.linalg.LinAlgError(f"partitioned factor breakdown, code {st}")
    out.update(N=N, n=n, m=m, seg_len=list(seg_len))
    if flops:
        out["flops_paper"] = fl[0::2].copy()    # [seg 0 .. seg P-1, sequential phase]
        out["flops_std"] = fl[1::2].copy()
    return out


def par_solve(F: dict, b, flops: bool = False):
    """O3: Algorithms 2 and 3 with a ``par_factor`` result."""
    b = _f64(b)
    x = np.ascontiguousarray(b.reshape(b.shape[0], -1).copy())
    P = len(F["seg_len"])
    segs = (ctypes.c_int * P)(*F["seg_len"])
    fl = np.zeros(2 * (P + 1))
    lib().orc_par_solve(F["N"], F["n"], F["m"], P, segs, _p(F["Ld"]), _p(_nonempty(F["Le"])),
                        _p(F["Lw"]), _p(F["Lh"]), _p(_nonempty(F["Lg"])), _p(_nonempty(F["Lr"])),
                        _p(x), x.shape[1], _p(fl))
    x = x.reshape(b.shape)
    if flops:
        return x, fl[0::2].copy(), fl[1::2].copy()
    return x


def seq_batch(D, E, G, R, b, nthreads: int = 1, shared_matrix: bool = False) -> np.ndarray:
    """O2 factor+solve of a batch of same-shape systems over POSIX threads.
    D is (count, N, n, n) (or (N, n, n) with shared_matrix), b is
    (count, dim, nrhs). Returns the solutions."""
    b = _f64(b)
    count, dim, nrhs = b.shape
    D = _f64(D)
    N, n = D.shape[-3], D.shape[-1]
    m = 0 if R is None else np.asarray(R).shape[-1]
    E = _f64(E) if N > 1 else np.zeros(1)
    G = _f64(G) if m else np.zeros(1)
    R = _f64(R) if m else np.zeros(1)
    x = b.copy()
    status = (ctypes.c_int * count)()
    st = lib().orc_seq_batch(count, N, n, m, nrhs, 0 if shared_matrix else 1, nthreads, _p(D),
                             _p(_nonempty(E)), _p(_nonempty(G)), _p(_nonempty(R)), _p(x), status)
    if st:
        raise np.linalg.LinAlgError(f"batch factor breakdown, code {st}")
    return x


def flops_reset():
    lib().orc_flops_reset()


def flops_get() -> tuple[float, float]:
    p, s = ctypes.c_double(), ctypes.c_double()
    lib().orc_flops_get(ctypes.byref(p), ctypes.byref(s))
    return p.value, s.value


def backward_error(A: np.ndarray, x: np.ndarray, b: np.ndarray) -> float:
    """Normwise backward error ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    r = b - A @ x
    return float(np.abs(r).max() / (np.abs(A).sum(axis=1).max() * np.abs(x).max() + np.abs(b).max()))


def block_matvec(D, E, G, R, x):
    """y = Psi x computed block by block (the product with the matrix of
    Eq. (3)); x is (dim,) or (dim, nrhs). Used for residuals."""
    N, n, _ = D.shape
    m = 0 if R is None or np.size(R) == 0 else R.shape[0]
    X = x.reshape(x.shape[0], -1)
    Xs = X[:N * n].reshape(N, n, -1)
    Ds = np.tril(D) + np.swapaxes(np.tril(D, -1), 1, 2)
    Y = np.einsum("jab,jbr->jar", Ds, Xs)
    if N > 1:
        Y[1:] += np.einsum("jab,jbr->jar", E, Xs[:-1])
        Y[:-1] += np.einsum("jba,jbr->jar", E, Xs[1:])
    out = np.empty_like(X)
    out[:N * n] = Y.reshape(N * n, -1)
    if m:
        xg = X[N * n:]
        Rs = np.tril(R) + np.tril(R, -1).T
        out[:N * n] += np.einsum("jba,br->jar", G, xg).reshape(N * n, -1)
        out[N * n:] = np.einsum("jab,jbr->ar", G, Xs) + Rs @ xg
    return out.reshape(x.shape)


def adjoint(D, E, G, R, x, xbar):
    """Adjoint of x = Psi^{-1} b (definition): bbar = Psi^{-1} xbar (Psi is
    symmetric) with the O2 solve, and dL/dPsi = -bbar x^T restricted to the
    stored blocks, a symmetric pair of entries counted as one parameter
    (dD, dR lower-triangular), summed over the columns of x."""
    D = _f64(D)
    N, n, _ = D.shape
    m = 0 if R is None or np.size(R) == 0 else np.asarray(R).shape[0]
    bbar = seq_solve(seq_factor(D, E, G, R), xbar)
    X = np.asarray(x, dtype=np.float64).reshape(x.shape[0], -1)
    B = bbar.reshape(bbar.shape[0], -1)
    Xs, Bs = X[:N * n].reshape(N, n, -1), B[:N * n].reshape(N, n, -1)
    full = -np.einsum("jrq,jcq->jrc", Bs, Xs)
    dD = np.tril(full + np.swapaxes(full, 1, 2))
    idx = np.arange(n)
    dD[:, idx, idx] = full[:, idx, idx]
    dE = -(np.einsum("jrq,jcq->jrc", Bs[1:], Xs[:-1]) + np.einsum("jrq,jcq->jrc", Xs[1:], Bs[:-1]))
    dG = np.zeros((N, m, n))
    dR = np.zeros((m, m))
    if m:
        xg, bg = X[N * n:], B[N * n:]
        dG = -(np.einsum("rq,jcq->jrc", bg, Xs) + np.einsum("rq,jcq->jrc", xg, Bs))
        fr = -bg @ xg.T
        dR = np.tril(fr + fr.T)
        dR[np.arange(m), np.arange(m)] = np.diag(fr)
    return bbar, dD, dE, dG, dR


def block_norm_inf(D, E, G, R) -> float:
    """||Psi||_inf (largest row sum of |Psi|) from the blocks of Eq. (3); Psi
    is symmetric, so this is also ||Psi||_1."""
    D = _f64(D)
    N, n, _ = D.shape
    m = 0 if R is None or np.size(R) == 0 else np.asarray(R).shape[0]
    Ds = np.tril(D) + np.swapaxes(np.tril(D, -1), 1, 2)
    rows = np.abs(Ds).sum(axis=2)
    if N > 1:
        E = _f64(E)
        rows[1:] += np.abs(E).sum(axis=2)      # E_{j-1} in stage row j
        rows[:-1] += np.abs(E).sum(axis=1)     # E_j^T in stage row j
    norm = rows.max()
    if m:
        G = _f64(G)
        Rs = np.tril(R) + np.tril(R, -1).T
        rows = rows + np.abs(G).sum(axis=1)    # G_j^T in stage row j
        grows = np.abs(G).sum(axis=(0, 2)) + np.abs(Rs).sum(axis=1)
        norm = max(rows.max(), grows.max())
    return float(norm)


def block_backward_error(D, E, G, R, x, b) -> float:
    """Normwise backward error ||b - Psi x||_inf / (||Psi||_inf ||x||_inf +
    ||b||_inf) with the product and the norm taken block by block (Eq. (3));
    for several columns the maxima run over all of them together."""
    x = np.asarray(x, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    r = b - block_matvec(D, E, G, R, x)
    return float(np.abs(r).max() / (block_norm_inf(D, E, G, R) * np.abs(x).max() + np.abs(b).max()))


def cond_est(D, E, G, R, F: dict | None = None) -> float:
    """Estimate of kappa_1(Psi) = ||Psi||_1 ||Psi^{-1}||_1: the 1-norm of the
    inverse by Hager's method (SIAM J. Sci. Stat. Comput. 5, 1984) with
    Higham's safeguards (ACM TOMS 14, 1988): at most five steps of
    x -> y = Psi^{-1} x, z = Psi^{-1} sign(y) (Psi^{-1} is symmetric), moving x
    to the unit vector of the largest |z_j| until ||z||_inf <= z^T x; the
    estimate is the larger of ||y||_1 and 2 ||Psi^{-1} v||_1 / (3 dim) for the
    alternating vector v_i = (-1)^i (1 + i / (dim - 1)). A lower bound on the
    true value, usually within a factor of a few. The solves use the O2
    factor F (computed when not given)."""
    if F is None:
        F = seq_factor(D, E, G, R)
    N, n, m = F["N"], F["n"], F["m"]
    dim = N * n + m
    solve = lambda v: seq_solve(F, v)
    x = np.full(dim, 1.0 / dim)
    est = 0.0
    j_prev = -1
    for it in range(5):
        y = solve(x)
        est_new = float(np.abs(y).sum())
        if it > 0 and est_new <= est:
            est = max(est, est_new)
            break
        est = est_new
        xi = np.where(y >= 0, 1.0, -1.0)
        z = solve(xi)
        j = int(np.argmax(np.abs(z)))
        if np.abs(z).max() <= z @ x or j == j_prev:
            break
        x = np.zeros(dim)
        x[j] = 1.0
        j_prev = j
    i = np.arange(dim)
    v = np.where(i % 2 == 0, 1.0, -1.0) * (1.0 + i / max(dim - 1, 1))
    est = max(est, 2.0 * float(np.abs(solve(v)).sum()) / (3.0 * dim))
    return block_norm_inf(D, E, G, R) * est

