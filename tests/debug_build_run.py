"""Run by tests/test_gpu_debug_build.py in a process of its own with
KKT_DEBUG=1 (the index-checking build of the library): tiny shapes through
every kernel family (segment factor tasks in the whole-CTA, split, paired and
warp layouts, the recursive levels, the persistent schedule, the bordered
pass, the substitutions, mixed refinement with its fallback, the residual,
the adjoint, the allocation-free entry point), each result checked against
the FP64 oracle and every kkt_get_info record required to be clean (a failed
index check would read KKT_ERR_BOUNDS). Prints one line per case and "ok"."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import gen  # noqa: E402
import oracle  # noqa: E402
import paper_2511_00946_gb300 as kkt  # noqa: E402

assert kkt.DEBUG and "_build_debug" in kkt.LIB_PATH, kkt.LIB_PATH


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def clean(h, what):
    info = kkt.kkt_get_info(h)
    assert info["status"] == 0, (what, info)


def check(D, E, G, R, x, b, what):
    eta = oracle.block_backward_error(D, E, G, R, x, b)
    assert eta <= 1e-14, (what, eta)
    print(f"{what}: eta {eta:.2e}", flush=True)


def single(N, n, m, levels, precision=0, pairing=None, persistent=False, fused=False, refine=0, kind="ipm"):
    D, E, G, R = (gen.raceline if kind == "race" else gen.ipm)(N, n, m, seed=N + n, sigma_decades=4.0)
    b = gen.rhs(N * n + m, 1, seed=1)
    h = kkt.kkt_create_plan(N, n, m, levels, kkt.KKT_PARTITION_BALANCED, precision)
    what = f"N={N} n={n} m={m} levels={levels} prec={precision} pair={pairing} persist={persistent} fused={fused}"
    try:
        if pairing:
            kkt.kkt_set_pairing(h, {"off": kkt.KKT_PAIR_OFF, "on": kkt.KKT_PAIR_ON}[pairing])
        if persistent:
            kkt.kkt_set_persistent(h, True)
        if refine:
            kkt.kkt_set_refine_fallback(h, refine)
        Dd, Ed, Gd, Rd = dev(D), dev(E), dev(G) if m else None, dev(R) if m else None
        bd = dev(b)
        if fused:
            kkt.kkt_factor_solve(h, Dd, Ed, Gd, Rd, bd)
            x = bd
        elif precision:
            kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
            x = torch.zeros_like(bd)
            kkt.kkt_solve_refined(h, Dd, Ed, Gd, Rd, bd, x, sweeps=8, tol=1e-16)
        else:
            kkt.kkt_factor(h, Dd, Ed, Gd, Rd)
            kkt.kkt_solve(h, bd)
            x = bd
        torch.cuda.synchronize()
        clean(h, what)
        if not precision:
            xb = torch.empty_like(x)
            gD, gE = torch.empty_like(Dd), torch.empty_like(Ed)
            gG = torch.empty_like(Gd) if m else None
            gR = torch.empty_like(Rd) if m else None
            kkt.kkt_solve_adjoint(h, x, x, xb, gD, gE, gG, gR, Dd, Ed, Gd, Rd, sweeps=1)
            torch.cuda.synchronize()
            clean(h, what + " adjoint")
        check(D, E, G, R, x.cpu().numpy(), b, what)
    finally:
        kkt.kkt_destroy(h)


for P in (1, 2, 3, 4):
    for pairing in ("off", "on"):
        single(16, 8, 4, [P, 1] if P > 1 else [1], pairing=pairing)
single(64, 24, 4, [8, 3, 1])
single(64, 24, 4, [8, 3, 1], persistent=True)
single(64, 24, 4, [8, 3, 1], fused=True)
single(200, 6, 2, [20, 5, 1], kind="race")
single(200, 6, 2, [20, 5, 1], kind="race", persistent=True)
single(96, 32, 8, [12, 3, 1], fused=True)
single(80, 48, 4, [1], precision=kkt.KKT_MIXED_FP32_ALL, refine=4)
single(80, 48, 4, [8, 1], precision=kkt.KKT_MIXED_TF32)
single(60, 12, 0, [6, 1], precision=kkt.KKT_MIXED_FP32_ALL)

# a small uneven batch, sequential and two-level plans
sy = gen.uneven_batch(12, seed=3, N_range=(5, 30))
Ns = [s[0].shape[0] for s in sy]
ns = [s[0].shape[1] for s in sy]
ms = [s[3].shape[0] for s in sy]
for Ps in ([1] * len(sy), [max(1, min(3, (N + 1) // 2)) for N in Ns]):
    h = kkt.kkt_batch_create(Ns, ns, ms, Ps)
    try:
        cat = lambda i: dev(np.concatenate([s[i].ravel() for s in sy] + [np.zeros(1)]))
        bs = [gen.rhs(N * n + m, 1, seed=i) for i, (N, n, m) in enumerate(zip(Ns, ns, ms))]
        b = dev(np.concatenate(bs))
        kkt.kkt_factor(h, cat(0), cat(1), cat(2), cat(3))
        kkt.kkt_solve(h, b)
        torch.cuda.synchronize()
        clean(h, f"batch P={Ps[:3]}")
        off = kkt.kkt_batch_offsets(h, len(sy))["b"]
        x = b.cpu().numpy()
        for i, s in enumerate(sy):
            check(*s, x[off[i]:off[i + 1]], bs[i], f"batch system {i}")
    finally:
        kkt.kkt_destroy(h)

# the allocation-free entry point
N, n, m, P = 40, 16, 4, 4
D, E, G, R = gen.ipm(N, n, m, seed=2, sigma_decades=2.0)
b = gen.rhs(N * n + m, 1, seed=3)
bd = dev(b)
info = torch.zeros(4, dtype=torch.int32, device="cuda")
kkt.kkt_solve_noalloc(N, n, m, P, dev(D), dev(E), dev(G), dev(R), bd, info=info)
torch.cuda.synchronize()
assert info.cpu().tolist() == [0, 0, 0, 0]
check(D, E, G, R, bd.cpu().numpy(), b, "noalloc")
print("ok")
