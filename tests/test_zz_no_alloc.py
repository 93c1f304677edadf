"""pcms_apply_map_noalloc: the operator apply for callers that may not allocate device memory
while they run (a solver's time-step loop with a fixed footprint after set-up, or code that
shares the GPU with an application whose allocator owns the free memory). It must give the
same result as pcms_apply_map, call after call, using only the library's fixed scratch
array, and refuse maps whose scratch would not fit.

This file is collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2510_18838_gb300 import workloads as W
from tests._helpers import TOL_FP64, TOL_MIXED, need_gpu, normwise_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    from paper_2510_18838_gb300 import build, pcms
    build.build()
    return torch, pcms


def _noalloc(pcms, torch, m, fields):
    out = torch.empty((fields.shape[0], m.n_tgt), dtype=fields.dtype, device=fields.device)
    st = pcms.lib().pcms_apply_map_noalloc(m.handle, ctypes.c_void_p(fields.data_ptr()),
                                           fields.shape[0], ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


@pytest.mark.parametrize("dim,deg,prec,nf", [(2, 2, "mixed", 16), (3, 1, "fp64", 3),
                                             (2, 1, "mixed", 1)])
def test_noalloc_apply_matches_apply_on_two_calls(env, dim, deg, prec, nf):
    torch, pcms = env
    dev = torch.device("cuda", 0)
    src = torch.from_numpy(W.uniform_points(60000, dim, 910 + dim)).to(dev)
    tgt = torch.from_numpy(W.uniform_points(40000, dim, 920 + dim)).to(dev)
    r = 0.02 if dim == 2 else 0.06
    m = pcms.create_map(src, tgt, deg, r, precision=prec)
    dt = torch.float32 if prec == "mixed" else torch.float64
    tol = TOL_MIXED if prec == "mixed" else TOL_FP64
    g = torch.Generator(device=dev).manual_seed(5)
    for call in range(2):                       # two calls in a row share the scratch array
        f = torch.rand((nf, 60000), generator=g, device=dev, dtype=torch.float64).to(dt)
        ref = m.apply(f).cpu().numpy()
        st, out = _noalloc(pcms, torch, m, f)
        assert st == pcms.OK, pcms.lib().pcms_last_error()
        got = out.cpu().numpy()
        ok = np.isfinite(ref).all(axis=0)
        assert np.array_equal(np.isfinite(got).all(axis=0), ok)
        assert normwise_err(got, ref, ok) <= tol, call
    m.destroy()


def test_noalloc_refuses_maps_beyond_the_fixed_scratch(env):
    torch, pcms = env
    dev = torch.device("cuda", 0)
    src = torch.from_numpy(W.uniform_points(400000, 2, 930)).to(dev)
    tgt = torch.from_numpy(W.uniform_points(200000, 2, 931)).to(dev)
    m = pcms.create_map(src, tgt, 1, 0.004, precision="mixed")
    f = torch.rand((16, 400000), device=dev, dtype=torch.float32)
    st, _ = _noalloc(pcms, torch, m, f)
    assert st == pcms.CAPACITY
    assert b"bytes of scratch" in pcms.lib().pcms_last_error()
    st, out = _noalloc(pcms, torch, m, f[:1].contiguous())   # one field fits
    assert st == pcms.OK
    ref = m.apply(f[:1].contiguous()).cpu().numpy()
    ok = np.isfinite(ref).all(axis=0)
    assert normwise_err(out.cpu().numpy(), ref, ok) <= TOL_MIXED
    m.destroy()
