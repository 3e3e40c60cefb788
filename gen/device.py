"""Seeded synthetic batches built on the GPU, for the batched workloads.

The recipes are those of ``gen.ipm`` and ``gen.raceline`` (same shapes, value
distributions and SPD embedding), drawn from a seeded torch CUDA generator
instead of NumPy's: the values are not bitwise those of the NumPy generators,
which serve the oracle comparisons on smaller cases. Building the largest
batch (4096 systems, about 7 GB of blocks) on the host would take minutes;
here it takes a few batched matrix products per block size.

Like ``gen`` this holds no arithmetic of the method, only random draws and the
products that build an SPD matrix. Outputs are flat FP64 CUDA tensors in the
packed batch layout of the C interface (system after system):

  D  sum_s N_s n_s^2        E  sum_s (N_s - 1) n_s^2
  G  sum_s N_s m_s n_s      R  sum_s m_s^2         b  sum_s (N_s n_s + m_s)
"""
from __future__ import annotations

import numpy as np
import torch


def offsets(Ns, ns, ms):
    """Start offsets (elements; rows for b) of every system's blocks."""
    Ns, ns, ms = (np.asarray(v, dtype=np.int64) for v in (Ns, ns, ms))
    size = dict(D=Ns * ns * ns, E=np.maximum(Ns - 1, 0) * ns * ns, G=Ns * ms * ns, R=ms * ms, b=Ns * ns + ms)
    return {k: np.concatenate([[0], np.cumsum(v)]) for k, v in size.items()}


def _draw_blocks(gen, S, n, kind, sigma_decades, g_rows, reg, dev):
    """S stage blocks D of size n x n for one recipe, in chunks."""
    out = torch.empty((S, n, n), dtype=torch.float64, device=dev)
    chunk = max(1, (1 << 27) // (8 * n * max(g_rows, n)))
    eye = torch.eye(n, dtype=torch.float64, device=dev)
    for a in range(0, S, chunk):
        c = min(chunk, S - a)
        Gc = torch.randn((c, g_rows, n), generator=gen, dtype=torch.float64, device=dev)
        u = torch.rand((c, g_rows), generator=gen, dtype=torch.float64, device=dev)
        sig = torch.pow(10.0, (2.0 * u - 1.0) * sigma_decades)
        Dc = torch.einsum("jra,jr,jrb->jab", Gc, sig, Gc)
        if kind == "ipm":
            Rq = torch.randn((c, n, n), generator=gen, dtype=torch.float64, device=dev)
            Dc += Rq @ Rq.transpose(1, 2)
        out[a:a + c] = Dc + reg * eye
    return out


def batch(Ns, ns, ms, seed=0, kind="ipm", sigma_decades=None, g_rows=None, reg=None, coupling=0.1,
          psd_couplings=False, device="cuda"):
    """Packed (D, E, G, R) of independent systems with N_s stages of size n_s
    and arrow m_s. kind = "ipm" (gen.ipm: D = R R^T + G^T Sigma G + reg I,
    couplings N(0, 1/n), PSD-embedded with ``psd_couplings``) or "raceline"
    (gen.raceline: D = reg I + G^T Sigma G, PSD-embedded couplings
    N(0, coupling^2)); arrow as gen._arrow."""
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    Ns, ns, ms = (np.asarray(v, dtype=np.int64) for v in (Ns, ns, ms))
    off = offsets(Ns, ns, ms)
    if sigma_decades is None:
        sigma_decades = 8.0
    if reg is None:
        reg = 1e-8 if kind == "ipm" else 1e-2
    D = torch.empty(int(off["D"][-1]), dtype=torch.float64, device=dev)
    E = torch.empty(max(int(off["E"][-1]), 1), dtype=torch.float64, device=dev)
    G = torch.zeros(max(int(off["G"][-1]), 1), dtype=torch.float64, device=dev)
    R = torch.zeros(max(int(off["R"][-1]), 1), dtype=torch.float64, device=dev)
    for n in sorted(set(ns.tolist())):
        sel = np.nonzero(ns == n)[0]
        S = int(Ns[sel].sum())
        gr = g_rows if g_rows is not None else (2 * n if kind == "ipm" else 4)
        Dn = _draw_blocks(gen, S, n, kind, sigma_decades, gr, reg, dev)
        eye = torch.eye(n, dtype=torch.float64, device=dev)
        at = 0
        for s in sel:
            N, m = int(Ns[s]), int(ms[s])
            Ds = Dn[at:at + N]
            at += N
            if N > 1:
                if kind == "ipm":
                    Es = torch.randn((N - 1, n, n), generator=gen, dtype=torch.float64, device=dev) / np.sqrt(n)
                    if psd_couplings:
                        Ds[:-1] += Es.transpose(1, 2) @ Es
                        Ds[1:] += eye
                else:
                    C = coupling * torch.randn((N - 1, n, n), generator=gen, dtype=torch.float64, device=dev)
                    Es = -C
                    Ds[:-1] += C.transpose(1, 2) @ C
                    Ds[1:] += eye
                E[int(off["E"][s]):int(off["E"][s + 1])] = Es.reshape(-1)
            if m:
                T = torch.randn((N, m, n), generator=gen, dtype=torch.float64, device=dev) / np.sqrt(n)
                Ds += eye
                G[int(off["G"][s]):int(off["G"][s + 1])] = T.reshape(-1)
                Rs = torch.eye(m, dtype=torch.float64, device=dev) + torch.einsum("jab,jcb->ac", T, T)
                R[int(off["R"][s]):int(off["R"][s + 1])] = Rs.reshape(-1)
            D[int(off["D"][s]):int(off["D"][s + 1])] = Ds.reshape(-1)
    return D, E, G, R


def rhs(rows, nrhs=1, seed=0, device="cuda"):
    """b ~ N(0, 1) of shape (rows,) or (rows, nrhs), FP64 on the device."""
    gen = torch.Generator(device=torch.device(device))
    gen.manual_seed(int(seed))
    shape = (rows,) if nrhs == 1 else (rows, nrhs)
    return torch.randn(shape, generator=gen, dtype=torch.float64, device=device)
