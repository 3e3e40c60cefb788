"""The device arithmetic helpers of the factor and residual kernels against
exact references, run on the GPU through a small test helper compiled from
tests/csrc/numerics_probe.cu (it includes the library's kkt_numerics.cuh):

* pivot_rsqrt(d), the pivot reciprocal square root (hardware FP32 estimate
  plus one Halley step, with the exponent split off by integer operations),
  against 1/sqrt(d) evaluated to 50 significant digits: at most 2 units in
  the last place over every binary exponent, a dense sweep of the mantissa
  range [1, 4) and the boundaries of the fast path; NaN for d <= 0, NaN and
  infinity;
* abs_lo(v), |v| as a float cut to 20 mantissa bits (the |Psi| row sums that
  scale the backward error): never above |v|, within 2^-20 relative below it
  over the float range, 0 below it and the largest float above it.
"""
import ctypes
import os
import shutil
import subprocess
from decimal import Decimal, getcontext

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libnumerics_probe.so")
    src = os.path.join(HERE, "csrc", "numerics_probe.cu")
    hdr = os.path.join(os.path.dirname(HERE), "paper_2511_00946_gb300", "csrc", "kkt_numerics.cuh")
    if not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(src), os.path.getmtime(hdr)):
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared",
                               "-Xcompiler", "-fPIC", "-o", lib, src])
    L = ctypes.CDLL(lib)
    L.numerics_probe.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong]
    L.numerics_probe.restype = ctypes.c_int

    def run(what, values):
        x = torch.from_numpy(np.ascontiguousarray(values, dtype=np.float64)).cuda()
        y = torch.empty_like(x)
        assert L.numerics_probe(what, x.data_ptr(), y.data_ptr(), x.numel()) == 0
        return y.cpu().numpy()
    return run


def _ulp_err(d, r):
    """|r - 1/sqrt(d)| in units in the last place of the exact value."""
    getcontext().prec = 50
    errs = np.empty(len(d))
    for i, (dv, rv) in enumerate(zip(d, r)):
        exact = 1 / Decimal(float(dv)).sqrt()
        ulp = Decimal(float(np.spacing(float(exact))))
        errs[i] = float(abs(Decimal(float(rv)) - exact) / ulp)
    return errs


def test_pivot_rsqrt_within_two_ulp(probe):
    rng = np.random.default_rng(0)
    vals = []
    # every binary exponent of the normal range (fast path 2 <= ef <= 2045 and
    # both boundaries), four mantissas each
    for e in range(-1022, 1024):
        vals += list(np.ldexp(rng.uniform(1.0, 2.0, 4), e))
        vals.append(np.ldexp(1.0, e))
    # a dense sweep of d' in [1, 4) at exponent 0 and a large one
    vals += list(rng.uniform(1.0, 4.0, 20000))
    vals += list(np.ldexp(rng.uniform(1.0, 4.0, 2000), 600))
    # the ends of [1, 4) and of the double range, subnormals
    vals += [1.0, np.nextafter(1.0, 2.0), np.nextafter(4.0, 0.0), 2.0, 3.0, np.nextafter(2.0, 0.0),
             np.finfo(np.float64).max, np.finfo(np.float64).tiny, np.nextafter(np.finfo(np.float64).tiny, 1.0),
             5e-324, 1e-310, 2.0 ** -1021, 2.0 ** 1023, np.nextafter(2.0 ** 1023, np.inf)]
    d = np.array(vals)
    r = probe(0, d)
    errs = _ulp_err(d, r)
    worst = int(np.argmax(errs))
    assert errs.max() <= 2.0, f"max error {errs.max():.3f} ulp at d = {d[worst]!r}"


def test_pivot_rsqrt_not_positive_is_nan(probe):
    bad = np.array([0.0, -0.0, -1.0, -1e-300, -np.inf, np.inf, np.nan, -5e-324])
    r = probe(0, bad)
    assert np.isnan(r).all(), r
    flags = probe(2, np.concatenate([bad, [1.0, 5e-324, np.finfo(np.float64).max]]))
    assert flags.tolist() == [1.0] * len(bad) + [0.0, 0.0, 0.0]


def test_abs_lo_truncates_to_20_bits(probe):
    rng = np.random.default_rng(1)
    e = rng.integers(-126, 128, 50000)
    v = np.ldexp(rng.uniform(1.0, 2.0, e.size), e) * rng.choice([-1.0, 1.0], e.size)
    v = np.concatenate([v, [1.0, -1.0, 2.0 ** -126, np.finfo(np.float32).max]])
    a = probe(1, v)
    av = np.abs(v)
    assert (a <= av).all()
    assert (a >= av * (1 - 2.0 ** -20)).all(), np.max((av - a) / av)
    # the float32 value keeps at most 20 mantissa bits
    mant = a.astype(np.float32).view(np.uint32) & 0x7FFFFF
    assert (mant & 0x7).max() == 0
    # below the float range: 0; above it: the largest float
    tiny = np.array([2.0 ** -127, 1e-40, 1e-300, 0.0, -1e-45])
    assert (probe(1, tiny) == 0.0).all()
    big = np.array([2.0 ** 128, 1e39, 1e300, -1e300, np.inf])
    assert (probe(1, big) == float(np.finfo(np.float32).max)).all()
