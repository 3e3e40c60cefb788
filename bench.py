"""Benchmark: KKT factor + solve throughput on one GB300.

Workload (one step = the whole hot path, Algorithms 1-3, on one system):
an interior-point-shaped SPD block-tridiagonal-arrow KKT matrix with N = 1024
stage blocks of n = 32, arrow width m = 8, FP64, stage blocks
Q + G^T Sigma G + 1e-8 I with Sigma log-uniform over [1e-8, 1e8], random
dynamics couplings, one right-hand side b ~ N(0, 1). Every step factors the
matrix and solves for b from inputs resident in HBM (kkt_factor_solve: the
right-hand side bordered onto the arrow, so the factorization carries the
forward substitution); L2 is flushed (a 256 MiB write) before every timed
step. The level plan (segments per level of the recursive partition) is
picked on the device among a few candidates before the warm-up.

In the same run the line's `batched` object measures the comparison the
metric names on the uneven 4096-system batch: the plain FP64 path against the
FP32-mixed path refined to the FP64 path's accuracy (eta <= 1e-16 or the
rounding floor; residuals of 64 sampled systems checked on the host against
the FP64 path's), each with per-level launches and with the persistent
schedule, plus the dominant batched launch's roofline.

`--impl reference` times the FP64 CPU oracle (the sequential block method)
on the host cores instead, on a bounded sample of the same workload.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = "KKT factor+solve systems/sec at stated error vs plain FP64 GPU; % FLOP roofline"
UNIT = "systems/s"
N_STAGES, N_BLOCK, M_ARROW = 1024, 32, 8
WORKLOAD = f"ipm-shaped KKT, one system: N={N_STAGES}, n={N_BLOCK}, m={M_ARROW}, FP64, nrhs={{nrhs}}"
# FP64 peak from unit counts and clocks: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
L2_FLUSH_BYTES = 256 << 20


# --- one process per GPU (torchrun). Every workload partitions into
# independent systems, so ranks exchange no data: rank r solves its own share
# of the global batch, and the only collectives are the barriers around the
# timed region and one MAX reduction of the per-rank step times.

def rank_env():
    """(world, rank, local_rank) from the torchrun environment; (1, 0, 0) alone."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init_ranks(backend: str = "nccl"):
    """Join the process group when launched with more than one rank."""
    world, rank, local = rank_env()
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world, rank, local


def _grouped() -> bool:
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def barrier():
    if _grouped():
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(values):
    """Elementwise maximum over all ranks of a list of floats (the slowest
    rank's times); the list itself when running alone."""
    vals = [float(v) for v in values]
    if not _grouped():
        return vals
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(vals, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu().tolist()]


def whole_job_rate(systems_per_rank: int, ms_max: float, world: int) -> float:
    """Systems per second of the whole job: every rank solves systems_per_rank
    systems per step, and a step takes the slowest rank's time ms_max."""
    return world * systems_per_rank * 1000.0 / ms_max


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank's share of the global batch (distinct systems per rank)."""
    return base + 7919 * rank


def step_stats(ms_list):
    """Mean, standard deviation, median and extremes of the per-step times (ms)."""
    return {"mean": statistics.mean(ms_list), "std": statistics.pstdev(ms_list),
            "median": statistics.median(ms_list), "min": min(ms_list), "max": max(ms_list), "n": len(ms_list)}


# Arm cores report an implementer and a part number instead of a model name
ARM_PARTS = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd49": "Arm Neoverse N2",
             "0xd0c": "Arm Neoverse N1", "0xd8e": "Arm Neoverse N3", "0xd84": "Arm Neoverse V3"}


def host_cpu(cpuinfo: str = "/proc/cpuinfo") -> str:
    """Model name of the host CPU (as /proc/cpuinfo or the platform reports it)."""
    part = None
    try:
        with open(cpuinfo) as f:
            for ln in f:
                k, _, v = ln.partition(":")
                k, v = k.strip(), v.strip()
                if k in ("model name", "Model") and v:
                    return v
                if k == "CPU part" and v and part is None:
                    part = v.lower()
    except OSError:
        pass
    if part:
        return ARM_PARTS.get(part, f"Arm CPU part {part}")
    import platform
    return platform.processor() or platform.machine()


def finish_ranks():
    if _grouped():
        import torch.distributed as dist
        dist.destroy_process_group()


def backward_error(D, E, G, R, x, b):
    """||b - Psi x||_inf / (||Psi||_inf ||x||_inf + ||b||_inf), blocks of Eq. (3)."""
    N, n, _ = D.shape
    m = R.shape[0]
    Ds = np.tril(D) + np.swapaxes(np.tril(D, -1), 1, 2)
    xs = x[:N * n].reshape(N, n)
    y = np.einsum("jab,jb->ja", Ds, xs)
    y[1:] += np.einsum("jab,jb->ja", E, xs[:-1])
    y[:-1] += np.einsum("jba,jb->ja", E, xs[1:])
    y = y.reshape(-1)
    xg = x[N * n:]
    Rs = np.tril(R) + np.tril(R, -1).T
    y += np.einsum("jba,b->ja", G, xg).reshape(-1)
    yg = np.einsum("jab,jb->a", G, xs) + Rs @ xg
    r = b - np.concatenate([y, yg])
    rows = np.abs(Ds).sum(axis=2)
    rows[1:] += np.abs(E).sum(axis=2)
    rows[:-1] += np.abs(E).sum(axis=1)
    rows += np.abs(G).sum(axis=1)
    grows = np.abs(G).sum(axis=(0, 2)) + np.abs(Rs).sum(axis=1)
    norm = max(rows.max(), grows.max()) if m else rows.max()
    return float(np.abs(r).max() / (norm * np.abs(x).max() + np.abs(b).max())), \
        float(np.linalg.norm(r) / np.linalg.norm(b))


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled every 2 ms during the
    timed region through NVML's read-only queries (ctypes; nvidia-smi's 200 ms
    loop as a fallback)."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index: int, period_s: float = 0.002):
        self.cuda_index = cuda_index
        self.period = period_s
        self.samples = []       # (sm_mhz, max_mhz, reasons_bitmask)
        self.stop = threading.Event()
        self.nvml = None
        self.proc = None

    def _nvml_handle(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        handle = ctypes.c_void_p()
        try:
            import torch
            p = torch.cuda.get_device_properties(self.cuda_index)
            bus = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0".encode()
            if lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(handle)) != 0:
                raise RuntimeError
        except Exception:
            if lib.nvmlDeviceGetHandleByIndex_v2(self.cuda_index, ctypes.byref(handle)) != 0:
                return None
        fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        return lib, handle, fn

    def _loop(self):
        import ctypes
        lib, handle, reasons_fn = self.nvml
        mhz, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        lib.nvmlDeviceGetMaxClockInfo(handle, 1, ctypes.byref(mx))
        while not self.stop.is_set():
            if lib.nvmlDeviceGetClockInfo(handle, 1, ctypes.byref(mhz)) == 0 and \
                    reasons_fn(handle, ctypes.byref(rs)) == 0:
                self.samples.append((float(mhz.value), float(mx.value), int(rs.value)))
            time.sleep(self.period)

    def _smi(self):
        for line in self.proc.stdout:
            p = [v.strip() for v in line.split(",")]
            try:
                bits = 0
                for name_bit, v in zip((0x8, 0x40, 0x20, 0x4), p[3:7]):
                    if v.lower() == "active":
                        bits |= name_bit
                self.samples.append((float(p[1]), float(p[2]), bits))
            except (ValueError, IndexError):
                pass

    def __enter__(self):
        try:
            self.nvml = self._nvml_handle()
        except OSError:
            self.nvml = None
        if self.nvml:
            self.t = threading.Thread(target=self._loop, daemon=True)
        else:
            fields = ("index,clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                      "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                      "clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={fields}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._smi, daemon=True)
        self.t.start()
        return self

    def __exit__(self, *exc):
        self.stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.t.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = set()
        for _, _, bits in self.samples:
            for bit, name in self.REASONS.items():
                if bits & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(v[0] for v in self.samples),
                "sm_max_mhz": max(v[1] for v in self.samples), "reasons": sorted(reasons),
                "samples": len(self.samples), "source": "nvml" if self.nvml else "nvidia-smi"}


def read_traffic(kernel_src_sha: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None when that summary was taken on other kernel source."""
    path = os.path.join(ROOT, "profiles", "k_factor_level1_ipm1024.md")
    if not os.path.exists(path):
        return None
    sha, traffic = None, None
    for line in open(path):
        if line.startswith("kernel_source_sha256:"):
            sha = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch:"):
            traffic = float(line.split(":", 1)[1].strip())
    return traffic if sha == kernel_src_sha else None


def kernel_source_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("kkt_kernels.cu", "kkt_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2511_00946_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def workload(seed: int, nrhs: int = 1):
    D, E, G, R = gen.ipm(N_STAGES, N_BLOCK, M_ARROW, seed=seed)
    b = gen.rhs(N_STAGES * N_BLOCK + M_ARROW, nrhs, seed=seed + 1)
    return D, E, G, R, b


def cpu_oracle_rate(D, E, G, R, b, budget_s: float):
    """The FP64 oracle's sequential factor + solve on one host core, timed on
    as many copies of the system as fit in about `budget_s` seconds."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    F = oracle.seq_factor(D, E, G, R)
    oracle.seq_solve(F, b)
    one = time.perf_counter() - t0
    reps = max(1, int(budget_s / max(one, 1e-6)))
    t0 = time.perf_counter()
    for _ in range(reps):
        F = oracle.seq_factor(D, E, G, R)
        oracle.seq_solve(F, b)
    dt = time.perf_counter() - t0
    return reps / dt, reps, dt


def run_reference(args):
    _, rank, _ = rank_env()
    if rank != 0:
        return
    D, E, G, R, b = workload(0, args.nrhs)
    per_step = []
    total_sys = 0
    for _ in range(args.warmup):
        cpu_oracle_rate(D, E, G, R, b, budget_s=0.0)
    for _ in range(args.steps):
        rate, reps, dt = cpu_oracle_rate(D, E, G, R, b, budget_s=args.ref_seconds)
        per_step.append(dt / reps)
        total_sys += reps
    ms = 1000.0 * statistics.mean(per_step)
    value = 1000.0 / ms
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD.format(nrhs=args.nrhs), "method": "FP64 CPU oracle, sequential block Cholesky"},
        "ms_stats": step_stats([1000.0 * t for t in per_step]),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": host_cpu(),
                         "sample": f"{total_sys} factor+solve runs of the workload system, "
                                   f"{args.steps} steps of about {args.ref_seconds:.0f} s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def graph_bracket():
    """Two timing events recorded inside a captured graph, around the step
    (external event-record nodes): a host delay between the timer's start and
    the replay's launch (a thread switch, a driver query of the clock
    sampler) then never lands in a step's time. None where this PyTorch has
    no external events; the caller then records around the replay."""
    import torch
    try:
        return (torch.cuda.Event(enable_timing=True, external=True),
                torch.cuda.Event(enable_timing=True, external=True))
    except TypeError:
        return None


def device_sms() -> int:
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def per_launch_flops(kkt, plan, partition, nrhs=1, chain=False):
    """Names and algorithmic FP64 flops (standard convention, as executed) of
    the launches of one factor-and-solve step, in launch order. With one
    right-hand side (kkt_factor_solve, the right-hand side bordered onto the
    arrow): factor levels 1..L with the flop model of m + 1 arrow rows (the
    factorization plus the forward substitution it carries; the top level's
    launch also runs the corner solve and the top level's backward sweep),
    backward levels L-1..1. With several (the two
    passes): factor levels 1..L, forward levels 1..L (the top one also solves
    the corner and runs its backward sweep), backward levels L-1..1 (with
    `chain`, the backward levels L-1..1 in one launch)."""
    L = len(plan)
    Ns = [N_STAGES]
    for p in plan[:-1]:
        Ns.append(p - 1)
    sms = device_sms()
    fused = nrhs == 1
    ma = M_ARROW + 1 if fused else M_ARROW
    sufb = [kkt.kkt_plan_flops(Ns[l], N_BLOCK, ma, plan[l:], partition, sms) for l in range(L)]
    suf = [kkt.kkt_plan_flops(Ns[l], N_BLOCK, M_ARROW, plan[l:], partition, sms) for l in range(L)]
    fac = [sufb[l]["factor"] - (sufb[l + 1]["factor"] if l + 1 < L else 0.0) for l in range(L)]
    sol = [nrhs * (suf[l]["solve"] - (suf[l + 1]["solve"] if l + 1 < L else 0.0)) for l in range(L)]
    names, flops = [], []
    if fused:
        names.append("k_border (bordered arrow copy)")
        flops.append(0.0)
    tag = " (+forward)" if fused else ""
    names += [f"k_factor level {l + 1}{tag}" for l in range(L)]
    flops += list(fac)
    if not fused:
        for l in range(L - 1):
            names.append(f"k_forward level {l + 1}")
            flops.append(sol[l] / 2.0)
        names.append(f"k_forward level {L} (forward, corner, backward)")
        flops.append(sol[L - 1])
    else:
        names[-1] = f"k_factor level {L} (+forward, corner, corner solve, backward)"
        flops[-1] += sol[L - 1] / 2.0
    if chain:
        names.append(f"k_backward_chain (levels {L - 1}..1)")
        flops.append(sum(sol[l] / 2.0 for l in range(L - 1)))
    else:
        for l in range(L - 2, -1, -1):
            names.append(f"k_backward level {l + 1}")
            flops.append(sol[l] / 2.0)
    return names, flops


def candidate_plans(kkt, partition):
    # four-fold reductions per level, and halving ones (more levels, two stages per deep segment)
    plans = [[304, 76, 19, 6, 2, 1], [256, 64, 16, 4, 1], [304, 76, 19, 5, 1], [256, 64, 16, 4, 2, 1],
             [304, 76, 19, 9, 3, 1], [304, 76, 25, 8, 2, 1], [152, 38, 10, 3, 1], [228, 57, 14, 3, 1],
             [256, 128, 64, 32, 16, 8, 4, 2, 1], [288, 144, 72, 36, 18, 9, 4, 2, 1],
             [320, 160, 80, 40, 20, 10, 5, 2, 1], [256, 128, 64, 32, 16, 8, 4, 1],
             [304, 152, 76, 38, 19, 9, 4, 2, 1], [304, 152, 76, 38, 19, 9, 4, 1],
             [304, 152, 76, 38, 19, 9, 3, 1], [256, 64, 32, 16, 8, 4, 2, 1]]
    ok = []
    for p in plans:
        try:
            kkt.kkt_plan_flops(N_STAGES, N_BLOCK, M_ARROW, p, partition)
            ok.append(p)
        except kkt.KKTError:
            pass
    return ok


# ------------------------------------------------------------------ batches
# The batched workloads (one line each, selected with --workload): the same
# JSON contract; `value` is the fastest path that meets the stated error.
BATCHES = {
    "uneven4096": dict(
        desc="4096 independent ipm-shaped KKT systems (PSD-embedded couplings), N uniform in [20, 200], "
             "n in {12, 24, 48}, m in {0, 4}, Sigma log-uniform over [1e-6, 1e6]; FP64 vs mixed precision "
             "(FP32, or TF32/BF16 tensor-core Schur products for n = 48) + FP64 refinement",
        kind="ipm", sigma=6.0, psd=True,
        paths=("fp64", "fp64_persist", "mixed", "mixed_persist", "mixed_tf32", "mixed_bf16")),
    "adjoint512": dict(
        desc="512 ipm-shaped KKT systems N=256, n=32, m=8; loss 1/2 ||x||^2: factor + solve + adjoint "
             "(dL/db and every block gradient), FP64 vs FP32 mixed with both solves refined in FP64",
        kind="ipm", sigma=8.0, paths=("fp64_adjoint", "mixed_adjoint")),
    "raceline64": dict(
        desc="64 race-line-shaped KKT systems N=8192, n=6, m=2; FP64 vs FP32 mixed + FP64 refinement",
        kind="raceline", sigma=8.0, paths=("fp64", "fp64_persist", "mixed")),
}


def batch_shapes(name: str, seed: int = 0):
    rng = np.random.default_rng(seed)
    if name == "uneven4096":
        c = 4096
        return (rng.integers(20, 201, size=c).tolist(), rng.choice([12, 24, 48], size=c).tolist(),
                rng.choice([0, 4], size=c).tolist())
    if name == "adjoint512":
        return [256] * 512, [32] * 512, [8] * 512
    if name == "raceline64":
        return [8192] * 64, [6] * 64, [2] * 64
    raise ValueError(name)


def batch_cpu_baseline(name: str, Ns, ns, ms, budget_s: float):
    """The oracle's sequential factor + solve over the host cores (one system
    per thread at a time) on a bounded sample of the batch's systems,
    generated on the host with the same recipe (gen); for the differentiable
    workload also the oracle's adjoint (which factors the system again)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    oracle.build()
    spec = BATCHES[name]
    rng = np.random.default_rng(7)
    idx = rng.permutation(len(Ns))
    cores = os.cpu_count() or 1
    systems = []
    for i in idx[: max(2 * cores, 8)]:
        N, n, m = int(Ns[i]), int(ns[i]), int(ms[i])
        if spec["kind"] == "ipm":
            sy = gen.ipm(N, n, m, seed=int(i), sigma_decades=spec["sigma"], psd_couplings=spec.get("psd", False))
        else:
            sy = gen.raceline(N, n, m, seed=int(i), sigma_decades=spec["sigma"])
        systems.append((sy, gen.rhs(N * n + m, 1, seed=int(i) + 1)))

    adjoint = name == "adjoint512"

    def one(sy):
        (D, E, G, R), b = sy
        x = oracle.seq_solve(oracle.seq_factor(D, E, G, R), b)
        if adjoint:     # the same step as the GPU's: loss 1/2 ||x||^2, xbar = x
            oracle.adjoint(D, E, G, R, x, x)

    with ThreadPoolExecutor(max_workers=cores) as ex:
        t0 = time.perf_counter()
        list(ex.map(one, systems))
        first = time.perf_counter() - t0
        reps = max(1, int(budget_s / max(first, 1e-6)))
        t0 = time.perf_counter()
        for _ in range(reps):
            list(ex.map(one, systems))
        dt = time.perf_counter() - t0
    return dict(value=reps * len(systems) / dt, unit=UNIT, cores=cores, kind="oracle", cpu=host_cpu(),
                sample=f"{reps} x {len(systems)} systems drawn from the batch on {cores} threads ({dt:.1f} s)"
                + ("; factor + solve + oracle.adjoint (a second factorization)" if adjoint else ""))


def _plan_is_sequential(kkt, h, count):
    return all(len(kkt.kkt_partition(h, s, 1)) == 1 for s in range(count))


def _factor_launch_groups(Ns, ns, ms):
    """Factor launches of a batch whose systems are all sequential (P = 1),
    in launch order: one per block size, small blocks (one warp per system)
    first, each with the indices of its systems."""
    groups = {}
    for s, n in enumerate(ns):
        groups.setdefault(n, []).append(s)
    return [(n, groups[n]) for n in sorted(groups)]


def measure_batch(name, args, world, rank, local, host_check=64, paths=None):
    """Time one batched workload, FP64 and (where listed) mixed, each step a
    CUDA graph of factor + solve (FP64) or factor + refinement (mixed).
    Returns (results per path, shapes). Besides the step time: the device's
    eta; a host FP64 check of the residual of `host_check` sampled systems
    for both paths on the same inputs; and, on sequential plans, the time of
    every factor launch over diagnostic replays and of the dominant one over
    the timed steps (two event nodes in the timed graph)."""
    import torch
    import paper_2511_00946_gb300 as kkt
    import gen.device as gdev
    spec = BATCHES[name]
    Ns, ns, ms = batch_shapes(name)
    count = len(Ns)
    # rank r holds systems [r * count, (r + 1) * count) of the global batch:
    # the same shapes, its own draws
    D, E, G, R = gdev.batch(Ns, ns, ms, seed=rank_seed(11, rank), kind=spec["kind"],
                            sigma_decades=spec["sigma"], psd_couplings=spec.get("psd", False))
    off = gdev.offsets(Ns, ns, ms)
    b0 = gdev.rhs(int(off["b"][-1]), 1, seed=rank_seed(12, rank))
    stream = torch.cuda.current_stream()
    sample = sorted(np.random.default_rng(3).choice(count, size=min(host_check, count), replace=False).tolist())
    host_blocks = []
    for s in sample:
        N, n, m = Ns[s], ns[s], ms[s]
        host_blocks.append((D[off["D"][s]:off["D"][s + 1]].cpu().numpy().reshape(N, n, n),
                            E[off["E"][s]:off["E"][s + 1]].cpu().numpy().reshape(max(N - 1, 0), n, n),
                            G[off["G"][s]:off["G"][s + 1]].cpu().numpy().reshape(N, m, n),
                            R[off["R"][s]:off["R"][s + 1]].cpu().numpy().reshape(m, m),
                            b0[off["b"][s]:off["b"][s + 1]].cpu().numpy()))
    results = {}
    for path in (paths or (args.paths.split(",") if args.paths else spec["paths"])):
        persist = path.endswith("_persist")
        base = path[:-len("_persist")] if persist else path
        adjoint = base.endswith("_adjoint")
        prec = {"mixed": kkt.KKT_MIXED_FP32_ALL, "mixed_tf32": kkt.KKT_MIXED_TF32,
                "mixed_bf16": kkt.KKT_MIXED_BF16}.get(base.replace("_adjoint", ""), kkt.KKT_FP64)
        mixed = path.startswith("mixed")
        t0 = time.perf_counter()
        if args.P:
            # the paper's two-phase method with P segments in every system
            h = kkt.kkt_batch_create(Ns, ns, ms, [args.P] * count, prec)
            lv = [2 if args.P > 1 else 1] * count
        else:
            h, lv = kkt.kkt_batch_create_tuned(Ns, ns, ms, prec)
        tune_s = time.perf_counter() - t0
        if persist:     # one persistent launch for the factorization (ticket queue, longest first)
            kkt.kkt_set_persistent(h, True)
        if mixed and adjoint:   # the adjoint's refinement stops at the forward solve's tolerance
            kkt.kkt_set_refine_tol(h, args.tol)
        b = b0.clone()
        x = torch.zeros_like(b0)
        bb = torch.empty_like(b0)
        gD, gE, gG, gR = (torch.empty_like(t) for t in (D, E, G, R))
        seq = _plan_is_sequential(kkt, h, count)
        fgroups = _factor_launch_groups(Ns, ns, ms) if seq and not persist else []

        def launch_step():
            kkt.kkt_factor(h, D, E, G, R)
            if mixed:
                kkt.kkt_solve_refined(h, D, E, G, R, b, x, sweeps=args.sweeps, tol=args.tol)
            else:
                kkt.kkt_solve(h, b)
            if adjoint:
                # loss 1/2 ||x||^2: xbar = x; on a mixed factor bbar is refined
                # like x (to the rounding floor, at most `sweeps` sweeps)
                xs_ = x if mixed else b
                kkt.kkt_solve_adjoint(h, xs_, xs_, bb, gD, gE, gG, gR, D=D, E=E, G=G, R=R,
                                      sweeps=args.sweeps if mixed else 1)

        def reset():
            if not mixed:
                b.copy_(b0)

        def capture(events, bracket=None):
            kkt.kkt_set_launch_events(h, events)
            for _ in range(2):
                reset()
                launch_step()
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            cap = torch.cuda.Stream()
            cap.wait_stream(stream)
            with torch.cuda.stream(cap):
                with torch.cuda.graph(g, stream=cap):
                    if bracket:
                        bracket[0].record(cap)
                    launch_step()
                    if bracket:
                        bracket[1].record(cap)
            stream.wait_stream(cap)
            torch.cuda.synchronize()
            return g

        def new_events(k):
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
            for ev in evs:
                ev.record()
            torch.cuda.synchronize()
            return evs

        # diagnostic replays: an event after every factor launch
        split, dom = None, None
        if fgroups:
            nf = len(fgroups)
            diag = new_events(nf)
            graph = capture(diag)
            per = [[] for _ in range(nf)]
            for it in range(8):
                reset()
                e0 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                graph.replay()
                torch.cuda.synchronize()
                if it >= 2:
                    prev = e0
                    for i, ev in enumerate(diag):
                        per[i].append(prev.elapsed_time(ev))
                        prev = ev
            split = [statistics.mean(v) for v in per]
            dom = int(np.argmax(split))
            del graph
        dom_ev = new_events(2) if dom is not None else None
        evs = None
        if dom is not None:
            evs = [None] * len(fgroups)
            if dom > 0:
                evs[dom - 1] = dom_ev[0]
            evs[dom] = dom_ev[1]
        br = graph_bracket()
        graph = capture(evs or [], br)
        for _ in range(max(args.warmup, 3)):
            reset()
            graph.replay()
        torch.cuda.synchronize()
        ms_list, dom_ms = [], []
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            for _ in range(args.steps):
                reset()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                graph.replay()
                e1.record(stream)
                e1.synchronize()
                t0 = br[0] if br else e0
                ms_list.append(t0.elapsed_time(br[1] if br else e1))
                if dom is not None:
                    dom_ms.append((dom_ev[0] if dom > 0 else t0).elapsed_time(dom_ev[1]))
        barrier()
        kkt.kkt_set_launch_events(h, [])
        info = kkt.kkt_get_info(h)
        if info["status"] != 0:
            raise RuntimeError(f"{name}/{path}: factorization failed: {info}")
        # error of the returned solution: the device's eta per system, and a
        # host FP64 residual of the sampled systems
        xs = (x if mixed else b).cpu().numpy()
        if mixed and adjoint:
            # the step's last refinement is the adjoint's: refine x once more
            # on its own (same factor and input, the same sweeps) for x's eta
            x1 = torch.zeros_like(b0)
            kkt.kkt_solve_refined(h, D, E, G, R, b0, x1, sweeps=args.sweeps, tol=args.tol)
            eta_dev = kkt.kkt_refine_eta(h, args.sweeps - 1, count)
            eta_raw = kkt.kkt_refine_eta(h, 0, count)
        elif mixed:
            eta_dev = kkt.kkt_refine_eta(h, args.sweeps - 1, count)
            eta_raw = kkt.kkt_refine_eta(h, 0, count)
        else:
            x1 = torch.zeros_like(b0)
            kkt.kkt_solve_refined(h, D, E, G, R, b0, x1, sweeps=1, tol=0.0)
            eta_dev = kkt.kkt_refine_eta(h, 0, count)
            eta_raw = eta_dev
        host, host_adj, grads = [], [], []
        if adjoint:
            bbs = bb.cpu().numpy()
            gh = [t.cpu().numpy() for t in (gD, gE, gG, gR)]
        for s, (Dh, Eh, Gh, Rh, bh) in zip(sample, host_blocks):
            xsl = xs[off["b"][s]:off["b"][s + 1]]
            host.append(backward_error(Dh, Eh, Gh, Rh, xsl, bh))
            if adjoint:
                # the adjoint solve Psi bbar = xbar (= x) and the sampled
                # system's block gradients
                host_adj.append(backward_error(Dh, Eh, Gh, Rh, bbs[off["b"][s]:off["b"][s + 1]], xsl))
                grads.append([g[off[k][s]:off[k][s + 1]] for g, k in zip(gh, ("D", "E", "G", "R"))])
        fl = kkt.kkt_flops(h)
        t_ms, max_eta = max_over_ranks([statistics.median(ms_list), float(np.max(eta_dev))])
        P1 = [len(kkt.kkt_partition(h, s, 1)) for s in range(count)]
        r = dict(ms_per_step=t_ms, ms_stats=step_stats(ms_list), value=whole_job_rate(count, t_ms, world),
                 max_eta=max_eta, max_eta_unrefined=float(np.max(eta_raw)),
                 host_check={"systems": len(sample), "max_backward_error": max(e for e, _ in host),
                             "relres": [rr for _, rr in host]},
                 levels_max=int(max(lv)), level1_segments_total=int(sum(P1)), tune_s=tune_s,
                 factor_flops=fl["factor"], sequential_factor_flops=fl["sequential_factor"],
                 clocks=clk.summary())
        if adjoint:
            r["host_check"]["adjoint_max_backward_error"] = max(e for e, _ in host_adj)
            r["host_check"]["adjoint_relres"] = [rr for _, rr in host_adj]
            r["_grads"] = grads     # sampled gradients, compared across paths and then dropped
        if mixed:
            r["refinement"] = {"sweeps_max": args.sweeps, "tol": args.tol,
                               "stop": "eta <= tol, or eta <= 4 u and a sweep that cuts it by less than 10 % (rounding floor)"}
        if split is not None:
            names = [f"{'k_factor_w' if n <= 16 else 'k_factor'} n={n} ({len(sy)} systems)" for n, sy in fgroups]
            r["factor_launch_ms"] = {nm: round(v, 4) for nm, v in zip(names, split)}
            dom_avg = statistics.mean(dom_ms)
            r["dominant_factor_launch"] = {"kernel": names[dom], "launch_ms": dom_avg}
            if not mixed:
                flops = 0.0
                cache = {}
                for s in fgroups[dom][1]:
                    key = (Ns[s], ns[s], ms[s])
                    if key not in cache:
                        cache[key] = kkt.kkt_plan_flops(*key, [1])["factor"]
                    flops += cache[key]
                ach = flops / (dom_avg * 1e-3) / 1e12
                peak = FP64_PEAK_GFLOPS / 1000.0
                r["roofline"] = {"bound": "alu", "kernel": names[dom], "launch_ms": dom_avg, "achieved": ach,
                                 "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                                 "flops_per_launch": flops, "traffic": None,
                                 "note": "FP64 sequential factor flops of the launch's systems (standard "
                                         "convention) over its event-timed duration in the timed graph"}
        results[path] = r
        kkt.kkt_destroy(h)
        del graph
        torch.cuda.synchronize()
    return results, (Ns, ns, ms)


def compare_paths(results):
    """Equal-accuracy comparison of each mixed path with the FP64 path on the
    same inputs: the ratio of the sampled systems' relative residuals (mixed
    over FP64; worst and median system) and of the step rates. `best` is the
    fastest mixed path at equal accuracy (residuals within 10x the FP64
    path's, eta <= 1e-14)."""
    fp = {p: r for p, r in results.items() if p.startswith("fp64")}
    grads = {p: r.pop("_grads", None) for p, r in results.items()}
    if not fp:
        return None
    ref, a = min(fp.items(), key=lambda kv: kv[1]["ms_per_step"])   # the faster plain FP64 schedule
    out = {"fp64_reference_path": ref}
    for p, m in results.items():
        if not p.startswith("mixed"):
            continue
        ratios = [rm / ra for rm, ra in zip(m["host_check"]["relres"], a["host_check"]["relres"])]
        out[p] = {"rate_over_fp64": m["value"] / a["value"], "ms_fp64": a["ms_per_step"],
                  "ms_mixed": m["ms_per_step"], "worst_relres_ratio_over_fp64": max(ratios),
                  "median_relres_ratio_over_fp64": statistics.median(ratios),
                  "max_eta_fp64": a["max_eta"], "max_eta_mixed": m["max_eta"]}
        equal = max(ratios) <= 10.0 and m["max_eta"] <= 1e-14
        if "adjoint_relres" in m["host_check"] and "adjoint_relres" in a["host_check"]:
            # the adjoint solve at equal accuracy too; the gradients' largest
            # difference from the FP64 path's, relative to their largest entry
            ar = [rm / ra for rm, ra in zip(m["host_check"]["adjoint_relres"], a["host_check"]["adjoint_relres"])]
            out[p]["worst_adjoint_relres_ratio_over_fp64"] = max(ar)
            out[p]["adjoint_max_backward_error"] = m["host_check"]["adjoint_max_backward_error"]
            equal = equal and max(ar) <= 10.0 and m["host_check"]["adjoint_max_backward_error"] <= 1e-14
            if grads.get(p) and grads.get(ref):
                out[p]["gradient_max_rel_diff_vs_fp64"] = {
                    k: max(float(np.abs(gm[i] - gf[i]).max() / max(np.abs(gf[i]).max(), 1e-300))
                           for gm, gf in zip(grads[p], grads[ref]) if gf[i].size)
                    for i, k in enumerate(("dD", "dE", "dG", "dR"))}
        out[p]["equal_accuracy"] = bool(equal)
    if len(out) == 1:
        return None
    ok = [p for p, c in out.items() if p != "fp64_reference_path" and c["equal_accuracy"]]
    best = max(ok, key=lambda p: out[p]["rate_over_fp64"]) if ok else None
    return {"paths": out, "best_mixed_at_equal_accuracy": best,
            "best_rate_over_fp64": out[best]["rate_over_fp64"] if best else None}


def run_batch(args):
    import torch
    name = args.workload
    spec = BATCHES[name]
    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    init_ranks("nccl")
    results, (Ns, ns, ms) = measure_batch(name, args, world, rank, local)
    count = len(Ns)
    # value: the fastest path that meets the error gates (eta <= 1e-14 and,
    # for the mixed path, residuals within 10x the FP64 path's)
    cmp_ = compare_paths(results)
    ok = {p: r for p, r in results.items()
          if r["max_eta"] <= 1e-14 and (not p.startswith("mixed") or (cmp_ and cmp_["paths"][p]["equal_accuracy"]))}
    best = min(ok.items(), key=lambda kv: kv[1]["ms_per_step"]) if ok else min(
        results.items(), key=lambda kv: kv[1]["ms_per_step"])
    bp, br = best
    if rank != 0:
        finish_ranks()
        return
    line = {
        "metric": METRIC, "value": br["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": br["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if not bp.startswith("mixed") else
        {"mixed": "f32+f64", "mixed_tf32": "tf32+f32+f64", "mixed_bf16": "bf16+f32+f64"}[
            bp.replace("_persist", "").replace("_adjoint", "")],
        "data": "synthetic",
        "config": {"workload": spec["desc"], "name": name, "path": bp, "systems": count * world,
                   "systems_per_rank": count,
                   "plan": f"two levels, P = {args.P} per system" if args.P else "autotuned per system",
                   "refinement": {"sweeps_max": args.sweeps, "tol": args.tol}
                   if any(p.startswith("mixed") for p in spec["paths"]) else None,
                   "l2": "inputs larger than L2", "graph": "one CUDA graph per step"},
        "error": {"max_backward_error": br["max_eta"], "gate": 1e-14},
        "paths": results,
        "comparison": cmp_,
        "roofline": next((r["roofline"] for r in results.values() if r.get("roofline")), None),
        "clocks": br["clocks"],
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline(name, Ns, ns, ms, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    finish_ranks()


# Small cases of the batched kernels for ncu captures (inputs larger than L2,
# about 1 GB on the device): two runs of the path, nothing timed.
PROFILE_CASES = {
    "mixed48": "304 ipm-shaped systems N=60, n=48, m=4 (Sigma +-6 decades, PSD couplings), FP32 mixed, "
               "sequential plan: factor + 2 refinement sweeps",
    "fp64_48": "the same systems, FP64: factor + solve",
    "adjoint128": "128 ipm-shaped systems N=256, n=32, m=8 (Sigma +-8 decades), FP64: factor + solve + adjoint",
    "adjoint128_mixed": "the same systems, FP32 mixed: factor + refined solve + refined adjoint (tol 1e-16, "
                        "at most 8 sweeps each)",
    "adjoint512_mixed": "the differentiable workload's 512 systems, FP32 mixed: factor + refined solve + refined "
                        "adjoint (tol 1e-16, at most 8 sweeps each)",
    "uneven512": "512 systems of the uneven workload's shapes, FP64, persistent factorization + solve",
    "uneven4096_mixed": "the uneven workload's 4096 systems, FP32 mixed, persistent factorization + refined "
                        "solve (tol 1e-16, at most 8 sweeps)",
}


def run_profile_case(name):
    import torch
    import paper_2511_00946_gb300 as kkt
    import gen.device as gdev
    torch.cuda.set_device(0)
    if name in ("mixed48", "fp64_48"):
        c = 304
        Ns, ns, ms = [60] * c, [48] * c, [4] * c
        D, E, G, R = gdev.batch(Ns, ns, ms, seed=1, kind="ipm", sigma_decades=6.0, psd_couplings=True)
    elif name in ("adjoint128", "adjoint128_mixed", "adjoint512_mixed"):
        c = 512 if name == "adjoint512_mixed" else 128
        Ns, ns, ms = [256] * c, [32] * c, [8] * c
        D, E, G, R = gdev.batch(Ns, ns, ms, seed=1, kind="ipm", sigma_decades=8.0)
    elif name in ("uneven512", "uneven4096_mixed"):
        Ns, ns, ms = (v[:512] if name == "uneven512" else v for v in batch_shapes("uneven4096"))
        c = len(Ns)
        D, E, G, R = gdev.batch(Ns, ns, ms, seed=1, kind="ipm", sigma_decades=6.0, psd_couplings=True)
    else:
        raise ValueError(name)
    b = gdev.rhs(int(sum(N * n + m for N, n, m in zip(Ns, ns, ms))), 1, seed=2)
    prec = (kkt.KKT_MIXED_FP32_ALL if name in ("mixed48", "adjoint128_mixed", "adjoint512_mixed", "uneven4096_mixed")
            else kkt.KKT_FP64)
    h = kkt.kkt_batch_create(Ns, ns, ms, [1] * c, prec)
    if name in ("uneven512", "uneven4096_mixed"):
        kkt.kkt_set_persistent(h, True)
    x = torch.zeros_like(b)
    gD, gE, gG, gR = (torch.empty_like(t) for t in (D, E, G, R))
    bb = torch.empty_like(b)
    for _ in range(2):
        kkt.kkt_factor(h, D, E, G, R)
        if name == "mixed48":
            kkt.kkt_solve_refined(h, D, E, G, R, b, x, sweeps=2, tol=0.0)
        elif name == "uneven4096_mixed":
            kkt.kkt_solve_refined(h, D, E, G, R, b, x, sweeps=8, tol=1e-16)
        elif name in ("adjoint128_mixed", "adjoint512_mixed"):
            kkt.kkt_solve_refined(h, D, E, G, R, b, x, sweeps=8, tol=1e-16)
            kkt.kkt_set_refine_tol(h, 1e-16)
            kkt.kkt_solve_adjoint(h, x, x, bb, gD, gE, gG, gR, D=D, E=E, G=G, R=R, sweeps=8)
        else:
            x.copy_(b)
            kkt.kkt_solve(h, x)
            if name == "adjoint128":
                kkt.kkt_solve_adjoint(h, x, x, bb, gD, gE, gG, gR, D=D, E=E, G=G, R=R, sweeps=1)
    torch.cuda.synchronize()
    info = kkt.kkt_get_info(h)
    kkt.kkt_destroy(h)
    print(json.dumps({"profile_case": name, "desc": PROFILE_CASES[name], "info": info}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--levels", default=None, help="comma-separated segments per level (skips the search)")
    ap.add_argument("--ref-seconds", type=float, default=3.0)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched FP64-vs-mixed comparison in the default line")
    ap.add_argument("--workload", default="ipm1024", choices=["ipm1024"] + sorted(BATCHES),
                    help="ipm1024: the single-system workload (default); the others are the batched ones")
    ap.add_argument("--sweeps", type=int, default=8, help="refinement sweeps of the mixed path (at most)")
    ap.add_argument("--nrhs", type=int, default=1, help="right-hand sides per step (ipm1024)")
    ap.add_argument("--paths", default=None,
                    help="batched workloads: comma-separated subset of the workload's paths (default: all)")
    ap.add_argument("--P", type=int, default=0,
                    help="batched workloads: the two-level method with P segments per system (default: tuned)")
    ap.add_argument("--partition", default="balanced", choices=["balanced", "paper"],
                    help="segment lengths: pairing-aware balanced, or Eq. (13) of the paper")
    ap.add_argument("--tol", type=float, default=1e-16,
                    help="refinement stop of the mixed path: a system stops once its eta is below this (or "
                         "once it is at the rounding floor); 1e-16 gives residuals within a few times the "
                         "FP64 path's")
    ap.add_argument("--profile-case", default=None, choices=sorted(PROFILE_CASES),
                    help="run one small case of the batched kernels twice, untimed (for ncu captures)")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "ipm1024":
        run_batch(args)
        return

    import torch
    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    init_ranks("nccl")
    import paper_2511_00946_gb300 as kkt

    D, E, G, R, b = workload(rank, args.nrhs)
    part = kkt.KKT_PARTITION_BALANCED if args.partition == "balanced" else kkt.KKT_PARTITION_PAPER
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Dd, Ed, Gd, Rd, b0 = dev(D), dev(E), dev(G), dev(R), dev(b)
    bd = b0.clone()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # --- level plan: fastest of a few candidates (untimed)
    search = {}
    if args.levels:
        plan = [int(v) for v in args.levels.split(",")]
    else:
        best = None
        for p in candidate_plans(kkt, part):
            h = kkt.kkt_create_plan(N_STAGES, N_BLOCK, M_ARROW, p, part)
            kkt.kkt_set_code_warmup(h, True)
            ts = []
            for it in range(9):
                bd.copy_(b0)
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                kkt.kkt_factor_solve(h, Dd, Ed, Gd, Rd, bd)
                e1.record()
                torch.cuda.synchronize()
                if it:
                    ts.append(e0.elapsed_time(e1))
            kkt.kkt_destroy(h)
            t = statistics.median(ts)
            search[",".join(map(str, p))] = round(t, 4)
            if best is None or t < best[0]:
                best = (t, p)
        plan = best[1]
    h = kkt.kkt_create_plan(N_STAGES, N_BLOCK, M_ARROW, plan, part)
    # the code of the kernels that run once per step is brought into L2 by a
    # companion system's pass on a forked side stream (kkt_set_code_warmup)
    kkt.kkt_set_code_warmup(h, True)
    # the companion's launches per step: its border copy, two factor levels,
    # its top level and one backward launch
    hw = kkt.kkt_create_plan(7, N_BLOCK, M_ARROW, [4, 2, 1], part)
    warm_launches = 1 + kkt.kkt_launch_counts(hw)[0] + 1
    kkt.kkt_destroy(hw)
    fl = kkt.kkt_flops(h)
    # one group per level: L forward launches, then one backward launch per
    # level below the top or a single one for all of them
    chain = kkt.kkt_launch_counts(h)[1] == len(plan) + 1 and len(plan) >= 3 and args.nrhs == 1
    launch_names, launch_flops = per_launch_flops(kkt, plan, part, args.nrhs, chain)
    nl = len(launch_names)

    def launch_step():
        # factor + solve: with one right-hand side in one pass (bordered onto
        # the arrow), with several the factorization and then the solve
        kkt.kkt_factor_solve(h, Dd, Ed, Gd, Rd, bd)

    cap = torch.cuda.Stream()

    def capture(events, bracket=None):
        """One step (factor + solve, every level) captured into a CUDA graph,
        with an event recorded after each launch whose entry is not None (and
        the bracket's two events around the step)."""
        kkt.kkt_set_launch_events(h, events)
        for _ in range(2):
            bd.copy_(b0)
            launch_step()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        cap.wait_stream(stream)
        with torch.cuda.stream(cap):
            with torch.cuda.graph(g, stream=cap):
                if bracket:
                    bracket[0].record(cap)
                launch_step()
                if bracket:
                    bracket[1].record(cap)
        stream.wait_stream(cap)
        torch.cuda.synchronize()
        return g

    def new_events(k):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        for ev in evs:
            ev.record()
        torch.cuda.synchronize()
        return evs

    # diagnostic replays (not the timed steps): an event after every launch
    # gives the per-launch split and picks the dominant launch; each event
    # record is a graph node of its own and costs a few microseconds, so the
    # timed graph records only the two events around the dominant launch
    diag_ev = new_events(nl)
    graph = capture(diag_ev)
    launch_ms = [[] for _ in range(nl)]
    for it in range(30):
        bd.copy_(b0)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        diag_ev[-1].synchronize()
        if it >= 3:
            prev = e0
            for i, ev in enumerate(diag_ev):
                launch_ms[i].append(prev.elapsed_time(ev))
                prev = ev
    diag_avg = [statistics.mean(v) for v in launch_ms]
    dom = int(np.argmax([a if f > 0 else -1.0 for a, f in zip(diag_avg, launch_flops)]))  # largest compute launch
    del graph

    dom_ev = new_events(2)  # after launch dom-1 (its start) and after launch dom
    evs = [None] * nl
    if dom > 0:
        evs[dom - 1] = dom_ev[0]
    evs[dom] = dom_ev[1]
    br = graph_bracket()
    graph = capture(evs, br)

    def step():
        graph.replay()

    for _ in range(max(args.warmup, 3)):
        bd.copy_(b0)
        step()
    torch.cuda.synchronize()
    info = kkt.kkt_get_info(h)
    if info["status"] != 0:
        raise RuntimeError(f"factorization failed: {info}")

    step_ms, dom_ms = [], []
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            bd.copy_(b0)
            flush.zero_()       # evict L2 before the timed step
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            t0 = br[0] if br else e0
            step_ms.append(t0.elapsed_time(br[1] if br else e1))
            dom_ms.append((dom_ev[0] if dom > 0 else t0).elapsed_time(dom_ev[1]))
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    barrier()
    ms = max_over_ranks([statistics.mean(step_ms)])[0]
    value = whole_job_rate(1, ms, world)
    x = bd.cpu().numpy()
    errs = [backward_error(D, E, G, R, x.reshape(x.shape[0], -1)[:, c], b.reshape(b.shape[0], -1)[:, c])
            for c in range(args.nrhs)]
    eta, relres = max(e[0] for e in errs), max(e[1] for e in errs)

    # --- end to end through the public API with host buffers (pinned): the
    # host entry point reads the inputs from host memory (the factor launches
    # load the page-locked blocks in place; b is copied in), factors, solves
    # and copies x back; the call is captured once into a CUDA graph and
    # replayed
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hD, hE, hG, hR, hb = pin(D), pin(E), pin(G), pin(R), pin(b)
    hx = hb.clone().pin_memory()
    h2d = sum(t.numel() * 8 for t in (hD, hE, hG, hR, hb))
    d2h = hx.numel() * 8
    kkt.kkt_set_launch_events(h, [])

    def e2e_step():
        kkt.kkt_factor_solve_host(h, hD, hE, hG, hR, hx)

    for _ in range(2):
        hx.copy_(hb)
        e2e_step()
    torch.cuda.synchronize()
    e2e_graph = torch.cuda.CUDAGraph()
    ebr = graph_bracket()
    cap.wait_stream(stream)
    with torch.cuda.stream(cap):
        with torch.cuda.graph(e2e_graph, stream=cap):
            if ebr:
                ebr[0].record(cap)
            e2e_step()
            if ebr:
                ebr[1].record(cap)
    stream.wait_stream(cap)
    torch.cuda.synchronize()
    e2e_ms = []
    barrier()
    for it in range(args.steps + 2):
        hx.copy_(hb)            # host copy of b: x overwrites it
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_graph.replay()
        e1.record(stream)
        e1.synchronize()
        if it >= 2:
            e2e_ms.append((ebr[0] if ebr else e0).elapsed_time(ebr[1] if ebr else e1))
    barrier()
    e2e_val = whole_job_rate(1, max_over_ranks([statistics.mean(e2e_ms)])[0], world)
    e2e_same = bool(np.array_equal(hx.numpy(), x))  # the device path's solution, bit for bit
    del e2e_graph
    # the same call made eagerly (no graph): the host work of every call
    # (pointer queries, chunk plan, launches) is paid each step; host wall
    # clock from the call to the synchronization that makes x readable
    for _ in range(3):
        hx.copy_(hb)
        e2e_step()
        torch.cuda.synchronize()
    eager_ms = []
    barrier()
    for _ in range(args.steps):
        hx.copy_(hb)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        stream.synchronize()
        eager_ms.append(1000.0 * (time.perf_counter() - t0))
    barrier()
    eager_val = whole_job_rate(1, max_over_ranks([statistics.mean(eager_ms)])[0], world)
    eager_same = bool(np.array_equal(hx.numpy(), x))

    # --- roofline of the dominant kernel (largest share of the step), timed
    # live over the timed steps
    names = launch_names
    dom_avg = statistics.mean(dom_ms)
    achieved = launch_flops[dom] / (dom_avg * 1e-3) / 1e12
    peak = FP64_PEAK_GFLOPS / 1000.0
    traffic = read_traffic(kernel_source_sha())

    # the batched comparison the metric names (mixed precision against the
    # plain FP64 path at equal accuracy), measured in the same run
    batched = None
    if not args.no_batched:
        # FP64 and FP32 mixed, each with per-level launches and with the
        # persistent schedule (the tensor-core variants are in the
        # --workload uneven4096 line)
        bres, (bN, bn, bm) = measure_batch("uneven4096", args, world, rank, local,
                                           paths=("fp64", "fp64_persist", "mixed", "mixed_persist"))
        batched = {"workload": BATCHES["uneven4096"]["desc"], "systems": len(bN) * world,
                   "paths": bres, "comparison": compare_paths(bres),
                   "roofline": next((r["roofline"] for r in bres.values() if r.get("roofline")), None)}
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            batched["cpu_baseline"] = batch_cpu_baseline("uneven4096", bN, bn, bm, args.cpu_seconds / 2)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, reps, dt = cpu_oracle_rate(D, E, G, R, b, budget_s=args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": host_cpu(),
               "sample": f"{reps} sequential FP64 factor+solve runs of the workload system ({dt:.1f} s)"}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "ms_stats": step_stats(step_ms),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.format(nrhs=args.nrhs), "levels": plan, "partition": args.partition,
                       "precision": "fp64",
                       "l2": "flushed before every timed step (256 MiB write)",
                       "timer": "CUDA events recorded inside the captured graph around the step (external "
                                "event-record nodes), read after each replay",
                       "code_warmup": "on: each step forks a side stream on which a 7-stage companion system "
                                      "runs its bordered pass, bringing the code of the once-per-step kernels "
                                      "into L2 (its launches are counted in gpu_launches)",
                       "replicas": world,
                       "plan_search_ms": search or None},
            "error": {"backward_error": eta, "relative_residual": relres},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "kkt_factor_solve_host (page-locked host buffers, graph replay): the factor "
                           "launches read D, E, G, R from host memory over the host link, b is copied in and "
                           "x copied out; the byte counts are every input and output crossing per step",
                    "same_x_as_device_path": e2e_same,
                    "eager": {"value": eager_val, "unit": UNIT, "ms_mean": statistics.mean(eager_ms),
                              "ms_median": statistics.median(eager_ms),
                              "how": "the same call without a graph, host wall clock from the call to the "
                                     "stream synchronization that makes x readable (L2 flushed before)",
                              "same_x_as_device_path": eager_same}},
            "gpu_launches": args.steps * (nl + warm_launches),
            "launches_per_step": {names[i] if i < len(names) else f"launch {i}": round(a, 4)
                                  for i, a in enumerate(diag_avg)},
            "launches_per_step_note": "ms per launch from 27 diagnostic graph replays with an event after "
                                      "every launch (those event nodes add about 5 us each); the timed steps "
                                      "record only the two events around the dominant launch",
            "roofline": {"bound": "alu", "kernel": names[dom], "launch_ms": dom_avg, "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                         "traffic": traffic, "peak_note": "FP64 FMA: 152 SMs x 2/clk x 2 flop x 2.07 GHz"},
            "flops_per_step": {"factor": fl["factor"], "solve": fl["solve"],
                               "sequential_factor": fl["sequential_factor"]},
            "clocks": clk.summary(),
            "wall_s_timed": wall,
        }
        if cpu:
            out["cpu_baseline"] = cpu
        if batched:
            out["batched"] = batched
        print(json.dumps(out), flush=True)
    kkt.kkt_destroy(h)
    finish_ranks()


if __name__ == "__main__":
    main()
