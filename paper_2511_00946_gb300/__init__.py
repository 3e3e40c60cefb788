"""GB300-native partitioned block Cholesky solver for SPD block-tridiagonal-arrow
KKT systems (arXiv 2511.00946, Algorithms 1-3).

Thin Python binding over the C interface of ``libkkt.so`` (include/kkt.h).
The functions keep the C names and only marshal arguments: every step of the
factorization and the solve runs in the library's CUDA kernels. PyTorch is
used for device memory and streams only. There is no CPU fallback: if the
library is missing, importing this package raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# KKT_DEBUG=1 in the environment loads the debug build (index checks on every
# task, reported as KKT_ERR_BOUNDS; build.py --debug builds it)
DEBUG = os.environ.get("KKT_DEBUG", "0") not in ("", "0")
LIB_PATH = os.path.join(_HERE, "_build_debug" if DEBUG else "_build", "libkkt.so")

(KKT_OK, KKT_ERR_ARG, KKT_ERR_PARTITION, KKT_ERR_NOT_SPD, KKT_ERR_CUDA, KKT_ERR_TIMEOUT, KKT_ERR_STATE,
 KKT_ERR_CAPACITY, KKT_ERR_BOUNDS) = range(9)
KKT_FP64, KKT_MIXED_FP32, KKT_MIXED_FP32_ALL, KKT_MIXED_TF32, KKT_MIXED_BF16 = 0, 1, 2, 3, 4
KKT_PARTITION_PAPER, KKT_PARTITION_BALANCED = 0, 1
KKT_PAIR_AUTO, KKT_PAIR_OFF, KKT_PAIR_ON, KKT_PAIR_AUTO_PAIRS = 0, 1, 2, 3
RHS_CHUNK = 16

EXPORTED = [
    "kkt_create", "kkt_create_levels", "kkt_create_plan", "kkt_batch_create", "kkt_batch_create_tuned", "kkt_destroy",
    "kkt_partition", "kkt_partition_rule", "kkt_partition_balanced", "kkt_batch_offsets", "kkt_factor", "kkt_solve", "kkt_factor_solve", "kkt_factor_solve_host", "kkt_solve_refined", "kkt_solve_adjoint", "kkt_refine_eta", "kkt_set_refine_tol",
    "kkt_get_info",
    "kkt_get_factor", "kkt_set_pairing", "kkt_set_launch_events", "kkt_launch_counts", "kkt_factor_ctas_per_task", "kkt_flops", "kkt_plan_flops", "kkt_solve_noalloc", "kkt_status_string",
    "kkt_set_persistent", "kkt_set_backward_chain", "kkt_set_code_warmup", "kkt_set_wait_limit",
    "kkt_set_refine_fallback",
]


class KKTError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
        "(the solver has no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)
_vp = ctypes.c_void_p
_ip = ctypes.POINTER(ctypes.c_int)
_dp = ctypes.POINTER(ctypes.c_double)
_szp = ctypes.POINTER(ctypes.c_size_t)
_i = ctypes.c_int

_sig = {
    "kkt_create": [_i, _i, _i, _i, _i, ctypes.POINTER(_vp)],
    "kkt_create_levels": [_i, _i, _i, _i, _ip, _i, ctypes.POINTER(_vp)],
    "kkt_create_plan": [_i, _i, _i, _i, _ip, _i, _i, ctypes.POINTER(_vp)],
    "kkt_batch_create": [_i, _ip, _ip, _ip, _ip, _i, ctypes.POINTER(_vp)],
    "kkt_batch_create_tuned": [_i, _ip, _ip, _ip, _i, _ip, ctypes.POINTER(_vp)],
    "kkt_partition_balanced": [_i, _i, _i, _i, _i, _ip],
    "kkt_destroy": [_vp],
    "kkt_partition": [_vp, _i, _i, _ip, _ip],
    "kkt_partition_rule": [_i, _i, _ip],
    "kkt_batch_offsets": [_vp, _szp, _szp, _szp, _szp, _szp],
    "kkt_factor": [_vp, _vp, _vp, _vp, _vp, _vp],
    "kkt_solve": [_vp, _vp, _i, _i, _vp],
    "kkt_factor_solve": [_vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _vp],
    "kkt_factor_solve_host": [_vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _vp],
    "kkt_solve_refined": [_vp, _vp, _vp, _vp, _vp, _vp, _i, _vp, _i, _i, _i, ctypes.c_double, _vp],
    "kkt_refine_eta": [_vp, _i, _dp],
    "kkt_solve_adjoint": [_vp, _vp, _vp, _vp, _vp, _vp, _i, _vp, _i, _vp, _i, _i, _vp, _vp, _vp, _vp, _i, _vp],
    "kkt_get_info": [_vp, _ip, _i],
    "kkt_get_factor": [_vp, _i, _dp, _dp, _dp, _dp, _dp, _dp],
    "kkt_set_pairing": [_vp, _i],
    "kkt_set_launch_events": [_vp, ctypes.POINTER(_vp), _i],
    "kkt_launch_counts": [_vp, _ip, _ip],
    "kkt_factor_ctas_per_task": [_vp, ctypes.c_int, _ip],
    "kkt_flops": [_vp, _dp, _dp, _dp],
    "kkt_plan_flops": [_i, _i, _i, _i, _ip, _i, _i, _dp, _dp, _dp],
    "kkt_solve_noalloc": [_i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp, _i, _i, _vp, _vp],
    "kkt_status_string": [_i],
    "kkt_set_persistent": [_vp, _i],
    "kkt_set_backward_chain": [_vp, _i],
    "kkt_set_code_warmup": [_vp, _i],
    "kkt_set_wait_limit": [_vp, ctypes.c_longlong, _i],
    "kkt_set_refine_fallback": [_vp, _i],
    "kkt_set_refine_tol": [_vp, ctypes.c_double],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_char_p if _name == "kkt_status_string" else ctypes.c_int


def status_string(status: int) -> str:
    return _lib.kkt_status_string(int(status)).decode()


kkt_status_string = status_string


def _check(st: int, what: str):
    if st != KKT_OK:
        raise KKTError(st, what)


def _ints(v):
    arr = (ctypes.c_int * len(v))(*[int(x) for x in v])
    return arr


def _ptr(x):
    """Device pointer of a torch CUDA tensor (FP64, contiguous) or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError("expected a torch CUDA tensor or a raw device pointer")
    if not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- C names

def kkt_create(N: int, n: int, m: int, P: int, precision: int = KKT_FP64) -> int:
    h = _vp()
    _check(_lib.kkt_create(N, n, m, P, precision, ctypes.byref(h)), "kkt_create")
    return h.value


def kkt_create_levels(N: int, n: int, m: int, P_levels, precision: int = KKT_FP64) -> int:
    h = _vp()
    _check(_lib.kkt_create_levels(N, n, m, len(P_levels), _ints(P_levels), precision, ctypes.byref(h)),
           "kkt_create_levels")
    return h.value


def kkt_create_plan(N: int, n: int, m: int, P_levels, partition: int = KKT_PARTITION_BALANCED,
                    precision: int = KKT_FP64) -> int:
    h = _vp()
    _check(_lib.kkt_create_plan(N, n, m, len(P_levels), _ints(P_levels), partition, precision,
                                ctypes.byref(h)), "kkt_create_plan")
    return h.value


def kkt_batch_create(N, n, m, P=None, precision: int = KKT_FP64) -> int:
    """Batch of independent systems (packed inputs, see kkt_batch_offsets)."""
    count = len(N)
    h = _vp()
    _check(_lib.kkt_batch_create(count, _ints(N), _ints(n), _ints(m), _ints(P) if P is not None else None,
                                 precision, ctypes.byref(h)), "kkt_batch_create")
    return h.value


def kkt_batch_create_tuned(N, n, m, precision: int = KKT_FP64):
    """Batch handle whose level plans are picked by timing candidates on the
    device (see the C header); returns (handle, levels per system)."""
    c = len(N)
    h = _vp()
    lv = (ctypes.c_int * c)()
    _check(_lib.kkt_batch_create_tuned(c, _ints(N), _ints(n), _ints(m), precision, lv, ctypes.byref(h)),
           "kkt_batch_create_tuned")
    return h.value, list(lv)


def kkt_destroy(h: int):
    _check(_lib.kkt_destroy(h), "kkt_destroy")


def kkt_partition(h: int, system: int = 0, level: int = 1) -> list[int]:
    P = ctypes.c_int()
    _check(_lib.kkt_partition(h, system, level, ctypes.byref(P), None), "kkt_partition")
    seg = (ctypes.c_int * P.value)()
    _check(_lib.kkt_partition(h, system, level, None, seg), "kkt_partition")
    return list(seg)


def kkt_partition_rule(N: int, P: int) -> list[int]:
    seg = (ctypes.c_int * max(P, 1))()
    _check(_lib.kkt_partition_rule(N, P, seg), "kkt_partition_rule")
    return list(seg[:P])


def kkt_partition_balanced(N: int, n: int, m: int, P: int, paired: bool = False) -> list[int]:
    seg = (ctypes.c_int * max(P, 1))()
    _check(_lib.kkt_partition_balanced(N, n, m, P, int(bool(paired)), seg), "kkt_partition_balanced")
    return list(seg[:P])


def kkt_batch_offsets(h: int, count: int) -> dict:
    arrs = {k: (ctypes.c_size_t * (count + 1))() for k in ("D", "E", "G", "R", "b")}
    _check(_lib.kkt_batch_offsets(h, arrs["D"], arrs["E"], arrs["G"], arrs["R"], arrs["b"]),
           "kkt_batch_offsets")
    return {k: np.array(list(v), dtype=np.int64) for k, v in arrs.items()}


def kkt_factor(h: int, D, E, G, R, stream=None):
    _check(_lib.kkt_factor(h, _ptr(D), _ptr(E), _ptr(G), _ptr(R), _stream(stream)), "kkt_factor")


def kkt_solve(h: int, b, nrhs: int | None = None, ldb: int | None = None, stream=None):
    if nrhs is None:
        nrhs = 1 if b.dim() == 1 else b.shape[1]
    if ldb is None:
        ldb = 1 if b.dim() == 1 else b.shape[1]
    _check(_lib.kkt_solve(h, _ptr(b), nrhs, ldb, _stream(stream)), "kkt_solve")


def kkt_factor_solve(h: int, D, E, G, R, b, nrhs: int | None = None, ldb: int | None = None, stream=None):
    """Factor and solve in one pass (the right-hand side bordered onto the
    arrow, see the C header); b is overwritten with x."""
    if nrhs is None:
        nrhs = 1 if b.dim() == 1 else b.shape[1]
    if ldb is None:
        ldb = 1 if b.dim() == 1 else b.shape[1]
    _check(_lib.kkt_factor_solve(h, _ptr(D), _ptr(E), _ptr(G), _ptr(R), _ptr(b), nrhs, ldb, _stream(stream)),
           "kkt_factor_solve")


def _host_ptr(x):
    """Host pointer of a contiguous float64 CPU tensor or NumPy array (None
    passes through); page-locked torch tensors let the copies run async."""
    if x is None:
        return None
    import numpy as _np
    if isinstance(x, _np.ndarray):
        if x.dtype != _np.float64 or not x.flags.c_contiguous:
            raise TypeError("expected a C-contiguous float64 array")
        return x.ctypes.data
    import torch
    if not isinstance(x, torch.Tensor) or x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
        raise TypeError("expected a contiguous float64 host tensor or array")
    return x.data_ptr()


def kkt_factor_solve_host(h: int, D, E, G, R, b, nrhs: int | None = None, ldb: int | None = None, stream=None):
    """kkt_factor_solve from host buffers (see the C header): the transfer of
    the stage blocks overlaps the level-1 factorization; b (host) receives x
    when `stream` reaches the end of the call."""
    if nrhs is None:
        nrhs = 1 if b.ndim == 1 else b.shape[1]
    if ldb is None:
        ldb = 1 if b.ndim == 1 else b.shape[1]
    _check(_lib.kkt_factor_solve_host(h, _host_ptr(D), _host_ptr(E), _host_ptr(G), _host_ptr(R), _host_ptr(b),
                                      nrhs, ldb, _stream(stream)), "kkt_factor_solve_host")


def kkt_solve_refined(h: int, D, E, G, R, b, x, nrhs: int | None = None, ldb: int | None = None,
                      ldx: int | None = None, sweeps: int = 3, tol: float = 1e-15, stream=None):
    """Iterative refinement with the current (mixed or FP64) factor; b is
    read-only, x receives the solution (see include/kkt.h)."""
    if nrhs is None:
        nrhs = 1 if b.dim() == 1 else b.shape[1]
    if ldb is None:
        ldb = 1 if b.dim() == 1 else b.shape[1]
    if ldx is None:
        ldx = 1 if x.dim() == 1 else x.shape[1]
    _check(_lib.kkt_solve_refined(h, _ptr(D), _ptr(E), _ptr(G), _ptr(R), _ptr(b), ldb, _ptr(x), ldx, nrhs,
                                  sweeps, float(tol), _stream(stream)), "kkt_solve_refined")


def kkt_solve_adjoint(h: int, x, xbar, bbar, dD, dE, dG, dR, D=None, E=None, G=None, R=None,
                      sweeps: int = 4, stream=None):
    """bbar = Psi^{-1} xbar and the block gradients of a loss with x = Psi^{-1} b
    (see include/kkt.h); x, xbar, bbar are (rows,) or (rows, nrhs) tensors."""
    nrhs = 1 if x.dim() == 1 else x.shape[1]
    ld = lambda t: 1 if t.dim() == 1 else t.shape[1]
    _check(_lib.kkt_solve_adjoint(h, _ptr(D), _ptr(E), _ptr(G), _ptr(R), _ptr(x), ld(x), _ptr(xbar), ld(xbar),
                                  _ptr(bbar), ld(bbar), nrhs, _ptr(dD), _ptr(dE), _ptr(dG), _ptr(dR), sweeps,
                                  _stream(stream)), "kkt_solve_adjoint")


def kkt_refine_eta(h: int, sweep: int, count: int = 1) -> np.ndarray:
    out = np.zeros(count)
    _check(_lib.kkt_refine_eta(h, sweep, out.ctypes.data_as(_dp)), "kkt_refine_eta")
    return out


def kkt_get_info(h: int, clear: bool = True) -> dict:
    buf = (ctypes.c_int * 4)()
    _check(_lib.kkt_get_info(h, buf, int(clear)), "kkt_get_info")
    return dict(status=buf[0], system=buf[1], stage=buf[2], level=buf[3])


def kkt_get_factor(h: int, N: int, n: int, m: int, system: int = 0) -> dict:
    out = dict(Ld=np.zeros((N, n, n)), Le=np.zeros((max(N - 1, 0), n, n)), Lw=np.zeros((N, n, n)),
               Lh=np.zeros((N, n, n)), Lg=np.zeros((N, m, n)), Lr=np.zeros((m, m)))
    p = {k: (v.ctypes.data_as(_dp) if v.size else None) for k, v in out.items()}
    _check(_lib.kkt_get_factor(h, system, p["Ld"], p["Le"], p["Lw"], p["Lh"], p["Lg"], p["Lr"]),
           "kkt_get_factor")
    return out


def kkt_set_pairing(h: int, policy: int) -> None:
    """KKT_PAIR_AUTO (default), KKT_PAIR_OFF, KKT_PAIR_ON or
    KKT_PAIR_AUTO_PAIRS: whether factor tasks run on one CTA, a pair of CTAs
    or (the deep levels' one-stage segments, automatic policy only) a
    cluster of up to eight (see the C header)."""
    _check(_lib.kkt_set_pairing(h, int(policy)), "kkt_set_pairing")


def kkt_set_launch_events(h: int, events) -> None:
    """events: list of torch.cuda.Event (created with enable_timing=True and
    already recorded once so that they own a CUDA event) or raw handles."""
    handles = []
    for ev in events or []:  # None: no event after that launch
        handles.append(None if ev is None else ev if isinstance(ev, int) else ev.cuda_event)
    arr = (_vp * max(len(handles), 1))(*handles)
    _check(_lib.kkt_set_launch_events(h, arr if handles else None, len(handles)), "kkt_set_launch_events")


def kkt_set_persistent(h: int, on: bool = True) -> None:
    """One persistent launch for the whole factorization (ticket queue in
    topological, longest-first order; see the C header)."""
    _check(_lib.kkt_set_persistent(h, int(bool(on))), "kkt_set_persistent")


def kkt_set_backward_chain(h: int, on: bool = True) -> None:
    """The backward substitution of every level below the top in one launch
    (default where it applies) or one launch per level (see the C header)."""
    _check(_lib.kkt_set_backward_chain(h, int(bool(on))), "kkt_set_backward_chain")


def kkt_set_code_warmup(h: int, on: bool = True) -> None:
    """Instruction warm-up of kkt_factor_solve: a companion system's bordered
    pass on a forked side stream (see the C header)."""
    _check(_lib.kkt_set_code_warmup(h, int(bool(on))), "kkt_set_code_warmup")


def kkt_set_wait_limit(h: int, cycles: int, unmet: bool = False) -> None:
    """Clock-cycle bound of the persistent schedule's dependency waits and of
    the one-warp substitution's bulk-copy waits; `unmet` makes every such
    wait run out (tests the timeout path)."""
    _check(_lib.kkt_set_wait_limit(h, int(cycles), int(bool(unmet))), "kkt_set_wait_limit")


def kkt_set_refine_tol(h: int, tol: float) -> None:
    """Refinement tolerance of kkt_solve_adjoint on a mixed factor (0: until
    eta stops falling)."""
    _check(_lib.kkt_set_refine_tol(h, float(tol)), "kkt_set_refine_tol")


def kkt_set_refine_fallback(h: int, cg_iters: int) -> None:
    """Preconditioned conjugate-gradient fallback of kkt_solve_refined for
    systems whose refinement stalls (cg_iters = 0 disables it)."""
    _check(_lib.kkt_set_refine_fallback(h, int(cg_iters)), "kkt_set_refine_fallback")


def kkt_factor_ctas_per_task(h: int, level: int) -> int:
    """CTAs per segment task of level `level`'s per-level factor launches:
    1, 2 (pairs), 4 or 8 (clusters of one-stage segments)."""
    c = ctypes.c_int(0)
    _check(_lib.kkt_factor_ctas_per_task(h, int(level), ctypes.byref(c)), "kkt_factor_ctas_per_task")
    return c.value


def kkt_launch_counts(h: int) -> tuple[int, int]:
    f, s = ctypes.c_int(), ctypes.c_int()
    _check(_lib.kkt_launch_counts(h, ctypes.byref(f), ctypes.byref(s)), "kkt_launch_counts")
    return f.value, s.value


def kkt_flops(h: int) -> dict:
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.kkt_flops(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "kkt_flops")
    return dict(factor=a.value, solve=b.value, sequential_factor=c.value)


def kkt_plan_flops(N: int, n: int, m: int, P_levels, partition: int = KKT_PARTITION_PAPER, sms: int = 0) -> dict:
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.kkt_plan_flops(N, n, m, len(P_levels), _ints(P_levels), partition, int(sms), ctypes.byref(a),
                               ctypes.byref(b), ctypes.byref(c)), "kkt_plan_flops")
    return dict(factor=a.value, solve=b.value, sequential_factor=c.value)


def kkt_solve_noalloc(N: int, n: int, m: int, P: int, D, E, G, R, b, nrhs: int | None = None,
                      ldb: int | None = None, info=None, stream=None):
    """Factor and solve one system in the library's fixed device buffer (no
    allocation; see include/kkt.h). `info`: optional int32 CUDA tensor of 4."""
    if nrhs is None:
        nrhs = 1 if b.dim() == 1 else b.shape[1]
    if ldb is None:
        ldb = 1 if b.dim() == 1 else b.shape[1]
    # the kernels read and write every element of these extents: a smaller
    # tensor would be accessed out of bounds
    need = {"D": (D, N * n * n), "E": (E, (N - 1) * n * n), "G": (G, N * m * n), "R": (R, m * m),
            "b": (b, ((N * n + m - 1) * ldb + nrhs) if N * n + m > 0 else 0)}
    for name, (t, count) in need.items():
        if count > 0 and (t is None or t.numel() < count):
            raise ValueError(f"kkt_solve_noalloc: {name} needs at least {count} elements for N={N}, n={n}, "
                             f"m={m}, nrhs={nrhs}, ldb={ldb}")
    ip = None
    if info is not None:
        import torch
        if not (info.is_cuda and info.dtype == torch.int32 and info.numel() >= 4):
            raise TypeError("info must be an int32 CUDA tensor of 4 elements")
        ip = info.data_ptr()
    _check(_lib.kkt_solve_noalloc(N, n, m, P, _ptr(D), _ptr(E), _ptr(G), _ptr(R), _ptr(b), nrhs, ldb, ip,
                                  _stream(stream)), "kkt_solve_noalloc")


# ---------------------------------------------------------------- differentiable solve

def _autograd_function():
    import torch

    class KKTSolveFunction(torch.autograd.Function):
        """x = Psi^{-1} b through the solver's handle: forward = kkt_factor +
        kkt_solve (kkt_solve_refined for a mixed handle), backward =
        kkt_solve_adjoint with the stored factor. The handle must not be
        refactored between the forward and the backward pass."""

        @staticmethod
        def forward(ctx, D, E, G, R, b, solver):
            kkt_factor(solver.h, D, E, G, R)
            x = torch.empty_like(b)
            if solver.mixed:
                kkt_solve_refined(solver.h, D, E, G, R, b, x, sweeps=solver.sweeps, tol=solver.tol)
            else:
                x.copy_(b)
                kkt_solve(solver.h, x)
            ctx.save_for_backward(D, E, G, R, x)
            ctx.solver = solver
            return x

        @staticmethod
        def backward(ctx, xbar):
            D, E, G, R, x = ctx.saved_tensors
            solver = ctx.solver
            xbar = xbar.contiguous()
            bbar = torch.empty_like(x)
            dD = torch.empty_like(D)
            dE = torch.empty_like(E) if E is not None else None
            dG = torch.empty_like(G) if G is not None else None
            dR = torch.empty_like(R) if R is not None else None
            kkt_solve_adjoint(solver.h, x, xbar, bbar, dD, dE, dG, dR, D, E, G, R, sweeps=solver.sweeps)
            return dD, dE, dG, dR, bbar, None

    return KKTSolveFunction


_KKTSolveFunction = None


def kkt_solve_differentiable(solver, D, E, G, R, b):
    """x = Psi^{-1} b, differentiable with respect to D, E, G, R and b (FP64
    CUDA tensors in the layout of include/kkt.h; the upper triangles of D and
    R are not read and receive zero gradient)."""
    global _KKTSolveFunction
    if _KKTSolveFunction is None:
        _KKTSolveFunction = _autograd_function()
    return _KKTSolveFunction.apply(D, E, G, R, b, solver)


# ---------------------------------------------------------------- convenience

class KKTSolver:
    """Owns one handle. ``factor(D, E, G, R)`` and ``solve(b)`` take float64
    CUDA tensors in the layout of include/kkt.h and enqueue on the current
    torch stream."""

    def __init__(self, N, n, m, P=1, precision=KKT_FP64, levels=None, partition=KKT_PARTITION_BALANCED,
                 sweeps=4, tol=0.0):
        self.N, self.n, self.m = N, n, m
        self.mixed = precision != KKT_FP64
        self.sweeps = sweeps
        self.tol = tol  # refinement tolerance of the forward and adjoint solves (mixed)
        if levels is not None:
            self.h = kkt_create_plan(N, n, m, levels, partition, precision)
        else:
            self.h = kkt_create(N, n, m, P, precision)
        kkt_set_refine_tol(self.h, tol)

    def factor(self, D, E, G=None, R=None, stream=None):
        kkt_factor(self.h, D, E, G, R, stream)

    def solve(self, b, stream=None):
        kkt_solve(self.h, b, stream=stream)
        return b

    def info(self, clear=True):
        return kkt_get_info(self.h, clear)

    def close(self):
        if self.h:
            kkt_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
