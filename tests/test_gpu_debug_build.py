"""The debug build (KKT_DEBUG: index checks on entry to every segment task and
residual task, failures reported as KKT_ERR_BOUNDS, never a trap) on tiny
shapes through every kernel family, against the FP64 oracle, in a process of
its own (tests/debug_build_run.py)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_tiny_shapes_clean():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, ROOT)
    import importlib.util
    spec = importlib.util.spec_from_file_location("kkt_build", os.path.join(ROOT, "paper_2511_00946_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build(debug=True)
    env = dict(os.environ, KKT_DEBUG="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_build_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert r.stdout.strip().splitlines()[-1] == "ok"
