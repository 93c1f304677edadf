"""The device FP64 reciprocal used by the solves' pivots and the barycentric coordinates
(recip64: two Newton-Raphson steps from the FP32 reciprocal, IEEE division outside
[1e-30, 1e30]) against IEEE 1/x, on random inputs over the whole range, both signs, and
edge cases: powers of two, values next to 1, the ends of the Newton range and beyond it,
subnormals, infinities. The stated bound: within 1 ulp of the correctly rounded 1/x."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from tests._helpers import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    need_gpu()
    from paper_2510_18838_gb300 import build
    out = tmp_path_factory.mktemp("recip64") / "librecip64.so"
    cmd = [build.nvcc(), *build.ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "--expt-relaxed-constexpr", "-I", build.INCLUDE, "-I", build.CSRC,
           os.path.join(ROOT, "tests", "gpu_kernels", "recip64.cu"), "-o", str(out)]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(str(out))
    L.recip64_run.restype = ctypes.c_int
    L.recip64_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    return L


def test_recip64_within_one_ulp_of_ieee(lib):
    import torch
    rng = np.random.default_rng(64)
    x = np.concatenate([
        10.0 ** rng.uniform(-35, 35, 400_000) * rng.choice([-1.0, 1.0], 400_000),
        1.0 + rng.integers(-2000, 2000, 4000) * np.finfo(np.float64).eps,
        np.ldexp(1.0, np.arange(-1060, 1020)), -np.ldexp(1.0, np.arange(-1060, 1020)),
        np.nextafter(1e-30, 0.0) * np.array([1.0, -1.0]), np.nextafter(1e30, np.inf) * np.array([1.0, -1.0]),
        np.array([1e-30, 1e30, -1e-30, -1e30, 3e-310, -3e-310, np.inf, -np.inf, 1.5, 3.0, 7.0]),
        rng.uniform(1.0, 2.0, 100_000),
    ])
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    st = lib.recip64_run(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), x.size,
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    with np.errstate(divide="ignore", over="ignore"):
        ref = 1.0 / x
    fin = np.isfinite(ref) & (ref != 0)
    assert np.array_equal(y[~fin], ref[~fin])       # infinities and zeros as IEEE division
    ulp = np.spacing(np.abs(ref[fin]))
    err = np.abs(y[fin] - ref[fin]) / ulp
    assert err.max() <= 1.0, (err.max(), x[fin][np.argmax(err)])
    # most results are the correctly rounded reciprocal
    assert (err == 0).mean() > 0.9
