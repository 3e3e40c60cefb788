"""Seeded synthetic inputs for the block-tridiagonal-arrow KKT solve.

Shared by the oracle side (tests, CPU baseline) and the GPU side (tests,
benchmark). It holds no arithmetic of the method: only random draws and the
matrix products that build an SPD matrix of the right shape. Every generator
takes a seed and returns NumPy FP64 arrays in the layout of the C interface:

  D [N][n][n]   Psi_{j,j}        E [N-1][n][n]  Psi_{j+1,j}
  G [N][m][n]   Psi_{g,j}        R [m][m]       Psi_{g,g}

Workloads (shapes and value distributions of the paper's multistage KKT
systems, Sec. 2 and Sec. 4; the paper's own benchmark problems need models and
track data that are not available, so these stand in for them):

* ``known_factor``  Psi = L L^T from a known block-bidiagonal-arrow L (the
  generating factor is returned too);
* ``ipm``           interior-point-shaped stage blocks Q + G^T Sigma G with a
  barrier scaling Sigma spanning many decades, random dynamics couplings;
* ``raceline``      long horizon, tiny blocks, tridiagonal couplings embedded
  as a PSD pair so the matrix stays SPD;
* ``uneven_batch``  a list of ``ipm`` systems of mixed sizes.
"""
from __future__ import annotations

import numpy as np


def _arrow(rng, N, n, m, D):
    """Arrow blocks T_j ~ N(0, 1/n) with a PSD embedding: the matrix
    [[I, T^T], [T, I + T T^T]] is PSD (its Schur complement is I), so adding
    I to every D_j and using R = I + sum_j T_j T_j^T keeps Psi SPD."""
    if m == 0:
        return np.zeros((N, 0, n)), np.zeros((0, 0))
    T = rng.normal(0.0, 1.0 / np.sqrt(n), size=(N, m, n))
    D += np.eye(n)[None]
    R = np.eye(m) + np.einsum("jab,jcb->ac", T, T)
    return T, R


def known_factor(N=16, n=8, m=4, seed=0):
    """Psi = L L^T for a block-bidiagonal-arrow L: diagonal blocks L_jj
    lower-triangular with diagonal U[1,2] and strictly-lower entries
    N(0, 0.3^2); couplings L_{j+1,j}, arrow blocks L_{g,j} N(0, 0.3^2);
    corner L_gg like a diagonal block. Returns (D, E, G, R, Lfac) with Lfac the
    generating blocks (Ld, Le, Lg, Lr)."""
    rng = np.random.default_rng(seed)

    def tri(k):
        M = np.tril(rng.normal(0.0, 0.3, size=(k, k)), -1)
        M[np.diag_indices(k)] = rng.uniform(1.0, 2.0, size=k)
        return M

    Ld = np.stack([tri(n) for _ in range(N)])
    Le = rng.normal(0.0, 0.3, size=(max(N - 1, 0), n, n))
    Lg = rng.normal(0.0, 0.3, size=(N, m, n))
    Lr = tri(m) if m else np.zeros((0, 0))
    D = np.einsum("jab,jcb->jac", Ld, Ld)
    D[1:] += np.einsum("jab,jcb->jac", Le, Le)
    E = np.einsum("jab,jcb->jac", Le, Ld[:N - 1])
    G = np.einsum("jab,jcb->jac", Lg, Ld)
    if N > 1 and m:
        G[1:] += np.einsum("jab,jcb->jac", Lg[:-1], Le)
    R = np.einsum("jab,jcb->ac", Lg, Lg) + Lr @ Lr.T if m else np.zeros((0, 0))
    return D, E, G, R, dict(Ld=Ld, Le=Le, Lg=Lg, Lr=Lr)


def ipm(N=1024, n=32, m=8, seed=0, sigma_decades=8.0, g_rows=None, reg=1e-8, psd_couplings=False):
    """Interior-point-shaped KKT matrix: D_j = Q_j + G_j^T Sigma_j G_j + reg I
    with Q_j = R_j R_j^T (R_j ~ N(0,1), n x n), constraint rows G_j ~ N(0,1)
    (g_rows x n, default 2n), Sigma_j diagonal log-uniform in
    [10^-d, 10^d]; couplings E_j ~ N(0, 1/n) (random dynamics); arrow as in
    ``_arrow``. With ``psd_couplings`` every coupling is embedded as the PSD
    pair [[C^T C, C^T], [C, I]] on stages (j, j+1) (E_j = C_j, D_j += C_j^T C_j,
    D_{j+1} += I), which keeps Psi SPD for any draw: without it small blocks
    (n = 12, no arrow) can give an indefinite matrix."""
    rng = np.random.default_rng(seed)
    g_rows = 2 * n if g_rows is None else g_rows
    Rq = rng.normal(size=(N, n, n))
    Gc = rng.normal(size=(N, g_rows, n))
    sig = 10.0 ** rng.uniform(-sigma_decades, sigma_decades, size=(N, g_rows))
    D = np.einsum("jab,jcb->jac", Rq, Rq) + np.einsum("jra,jr,jrb->jab", Gc, sig, Gc)
    D += reg * np.eye(n)[None]
    E = rng.normal(0.0, 1.0 / np.sqrt(n), size=(max(N - 1, 0), n, n))
    if psd_couplings and N > 1:
        D[:-1] += np.einsum("jab,jac->jbc", E, E)
        D[1:] += np.eye(n)[None]
    G, R = _arrow(rng, N, n, m, D)
    return D, E, G, R


def raceline(N=8192, n=6, m=2, seed=0, sigma_decades=8.0, g_rows=4, reg=1e-2, coupling=0.1):
    """Long-horizon, tiny-block KKT matrix: D_j = reg I + G_j^T Sigma_j G_j
    (G_j ~ N(0,1), g_rows x n; Sigma_j log-uniform in [10^-d, 10^d]) and
    couplings C_j ~ N(0, coupling^2) embedded as the PSD pair
    [[C^T C, -C^T], [-C, I]] on stages (j, j+1): E_j = -C_j, D_j += C_j^T C_j,
    D_{j+1} += I. Arrow as in ``_arrow``."""
    rng = np.random.default_rng(seed)
    Gc = rng.normal(size=(N, g_rows, n))
    sig = 10.0 ** rng.uniform(-sigma_decades, sigma_decades, size=(N, g_rows))
    D = np.einsum("jra,jr,jrb->jab", Gc, sig, Gc) + reg * np.eye(n)[None]
    C = rng.normal(0.0, coupling, size=(max(N - 1, 0), n, n))
    E = -C
    if N > 1:
        D[:-1] += np.einsum("jab,jac->jbc", C, C)
        D[1:] += np.eye(n)[None]
    G, R = _arrow(rng, N, n, m, D)
    return D, E, G, R


def uneven_batch(count=4096, seed=0, N_range=(20, 200), n_choices=(12, 24, 48), m_choices=(0, 4),
                 sigma_decades=6.0):
    """A batch of independent ``ipm`` systems with PSD-embedded couplings:
    N uniform in N_range, n and m drawn from the given choices, Sigma
    log-uniform over +-sigma_decades. Returns a list of (D, E, G, R)."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        N = int(rng.integers(N_range[0], N_range[1] + 1))
        n = int(rng.choice(n_choices))
        m = int(rng.choice(m_choices))
        out.append(ipm(N, n, m, seed=int(rng.integers(2**31)), sigma_decades=sigma_decades, psd_couplings=True))
    return out


def rhs(dim, nrhs=1, seed=0):
    """Right-hand side b ~ N(0, 1), shape (dim,) for nrhs = 1 else (dim, nrhs)."""
    rng = np.random.default_rng(seed)
    b = rng.normal(size=(dim, nrhs))
    return b[:, 0].copy() if nrhs == 1 else b
