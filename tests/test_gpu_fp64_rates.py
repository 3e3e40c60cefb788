"""The FP64 rates the kernels' design rests on, measured on the device by a
small helper compiled from tests/csrc/fp64_rate_probe.cu: FP64 FMA
throughput over every SM, the cycles one warp waits for a dependent FP64
FMA, the FP64 warp-level matrix multiply-accumulate (mma.sync m8n8k4) and
FP32 FMA throughput. The test checks that each figure is a plausible
measurement (finite, positive, the FP64 rates below the FP32 one) and
prints them; the design's choices (CUDA-core FP64 FMAs, no FP64 tensor-core
path) rest on the FP64 matrix rate being of the order of the FMA rate.
"""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fp64_rates():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libfp64_rate_probe.so")
    src = os.path.join(HERE, "csrc", "fp64_rate_probe.cu")
    if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared",
                               "-Xcompiler", "-fPIC", "-o", lib, src])
    L = ctypes.CDLL(lib)
    L.fp64_rates.argtypes = [ctypes.c_void_p]
    L.fp64_rates.restype = ctypes.c_int
    out = np.zeros(6)
    assert L.fp64_rates(out.ctypes.data) == 0
    dfma, lat, dmma, ffma, sms, mhz = out
    print(f"\nFP64 FMA {dfma:.3f} TFLOP/s, dependent FP64 FMA {lat:.1f} cycles, FP64 mma.sync {dmma:.3f} TFLOP/s, "
          f"FP32 FMA {ffma:.1f} TFLOP/s, {int(sms)} SMs, {mhz:.0f} MHz reported")
    for v in out:
        assert math.isfinite(v) and v > 0
    assert dfma < ffma and dmma < ffma
