"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Every workload partitions into independent systems (one system per rank, or
one batch of systems per rank), so the ranks exchange no data: the multi-rank
logic is the barrier around the timed region, the MAX reduction of the
per-rank step times, the whole-job rate computed from the slowest rank, and
distinct draws per rank. These tests run that logic with world_size 2 over
gloo, and launch the reference arm under torchrun to check that rank 0 alone
prints the one JSON line.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    import gen.device as gdev

    w, r, local = bench.init_ranks("gloo")
    bench.barrier()
    # per-rank step times: the slowest rank differs per entry
    times = [1.0 + r, 5.0 - 2.0 * r, 0.25 * (r + 1)]
    got = bench.max_over_ranks(times)
    # this rank's share of a small batch: same shapes on every rank, own draws
    Ns, ns, ms = [3, 5], [4, 6], [2, 0]
    D, E, G, R = gdev.batch(Ns, ns, ms, seed=bench.rank_seed(11, r), device="cpu")
    rate = bench.whole_job_rate(len(Ns), got[0], w)
    bench.barrier()
    bench.finish_ranks()
    np.savez(os.path.join(out_dir, f"rank{r}.npz"), world=w, local=local, got=np.array(got), rate=rate,
             D=D.numpy(), E=E.numpy(), G=G.numpy(), R=R.numpy())


@pytest.fixture(scope="module")
def two_ranks(tmp_path_factory):
    import torch.multiprocessing as mp
    out = tmp_path_factory.mktemp("ranks")
    mp.start_processes(_rank_main, args=(2, _free_port(), str(out)), nprocs=2, join=True,
                       start_method="spawn")
    return [dict(np.load(out / f"rank{r}.npz")) for r in range(2)]


def test_world_and_local_rank(two_ranks):
    for r, res in enumerate(two_ranks):
        assert int(res["world"]) == 2 and int(res["local"]) == r


def test_max_over_ranks_takes_slowest_rank(two_ranks):
    expect = [max(1.0 + r for r in range(2)), max(5.0 - 2.0 * r for r in range(2)),
              max(0.25 * (r + 1) for r in range(2))]
    for res in two_ranks:
        assert res["got"].tolist() == expect


def test_whole_job_rate_counts_every_rank(two_ranks):
    # 2 ranks x 2 systems per step, slowest step 2 ms -> 2000 systems/s
    for res in two_ranks:
        assert float(res["rate"]) == pytest.approx(2 * 2 * 1000.0 / 2.0)


def test_ranks_draw_distinct_systems_of_equal_shape(two_ranks):
    a, b = two_ranks
    for k in "DEGR":
        assert a[k].shape == b[k].shape
    assert not np.array_equal(a["D"], b["D"])
    assert not np.array_equal(a["G"], b["G"])


def test_single_rank_is_identity():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.5, 1.0]) == [3.5, 1.0]
    assert bench.whole_job_rate(4096, 80.0, 1) == pytest.approx(4096 * 1000.0 / 80.0)
    assert bench.rank_seed(11, 0) == 11 and bench.rank_seed(11, 1) != bench.rank_seed(11, 0)


def test_reference_arm_under_torchrun_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-seconds", "0.2"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["cpu_baseline"]["kind"] == "oracle"


def test_host_cpu_names_x86_and_arm(tmp_path):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    x86 = tmp_path / "x86"
    x86.write_text("processor\t: 0\nmodel name\t: Some Xeon @ 2.70GHz\nflags\t\t: fpu\n")
    arm = tmp_path / "arm"
    arm.write_text("processor\t: 0\nCPU implementer\t: 0x41\nCPU part\t: 0xd4f\n\nprocessor\t: 1\nCPU part\t: 0xd4f\n")
    odd = tmp_path / "odd"
    odd.write_text("processor\t: 0\nCPU part\t: 0xabc\n")
    assert bench.host_cpu(str(x86)) == "Some Xeon @ 2.70GHz"
    assert bench.host_cpu(str(arm)) == "Arm Neoverse V2"
    assert bench.host_cpu(str(odd)) == "Arm CPU part 0xabc"
    assert bench.host_cpu(str(tmp_path / "missing"))      # falls back to the platform's name
