"""GPU test of fx_state_init_equilibrium_noalloc, the initialisation entry point for callers
that cannot allocate device memory (code inside a host application that owns the allocator).

It goes through the C ABI, writes into a caller-owned device buffer, and must agree with
fx_state_init_equilibrium (which stages its input in the bound workspace) on two calls in a row
with different inputs.  Kept in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from paper_1806_07390_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_L1 = 1e-10


@pytest.fixture(scope="module")
def fxmod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_07390_gb300 import build, fx
    build.build()
    return fx


def reference_state(fxmod, pb, prim):
    g = fxmod.Grid(pb)
    g.init_equilibrium(prim)
    out = g.download(precision=fxmod.FX_FP64 if pb.precision == "fp64" else fxmod.FX_FP32)
    g.close()
    return out.astype(np.float64)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_init_matches_workspace_init_twice(fxmod, precision):
    import torch

    L = fxmod.lib()
    pb, prim_a = W.kh_2d(nx=40, ny=36, ngroups=16, seed=1, precision=precision)
    _, prim_b = W.kh_2d(nx=40, ny=36, ngroups=16, seed=2, precision=precision)
    prim_b = prim_b.copy()
    prim_b[-1] *= 1.3  # a different radiation temperature, so stale contents cannot pass
    ref_a = reference_state(fxmod, pb, prim_a)
    ref_b = reference_state(fxmod, pb, prim_b)

    h = fxmod.Grid(pb, bind=False)  # no workspace: the call must not need one
    dtype = torch.float64 if precision == "fp64" else torch.float32
    prec = fxmod.FX_FP64 if precision == "fp64" else fxmod.FX_FP32
    out = torch.empty(h.nelem, dtype=dtype, device="cuda")
    stream = torch.cuda.current_stream()
    for prim, ref in ((prim_a, ref_a), (prim_b, ref_b)):
        p = np.ascontiguousarray(prim, dtype=np.float64)
        out.fill_(float("nan"))
        st = L.fx_state_init_equilibrium_noalloc(h.h, p.ctypes.data_as(ctypes.c_void_p),
                                                 ctypes.c_void_p(out.data_ptr()), prec,
                                                 ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, L.fx_last_error(h.h).decode()
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        err = np.sum(np.abs(got - ref)) / np.sum(np.abs(ref))
        assert err <= FP64_L1, err
    h.close()


def test_noalloc_init_rejects_inputs_beyond_its_array(fxmod):
    import torch

    L = fxmod.lib()
    pb, _ = W.kh_2d(nx=16, ny=16, ngroups=4)
    pb.n = (4096, 1024, 1)  # 5 x 4M doubles of primitives: more than the 64 MiB array
    h = fxmod.Grid(pb, bind=False)
    prim = np.empty((5, 4096 * 1024))  # correctly sized input; it is rejected before any copy
    out = torch.empty(h.nelem, dtype=torch.float64, device="cuda")
    st = L.fx_state_init_equilibrium_noalloc(h.h, prim.ctypes.data_as(ctypes.c_void_p),
                                             ctypes.c_void_p(out.data_ptr()), fxmod.FX_FP64, None)
    assert st == -7
    assert b"exceed" in L.fx_last_error(h.h)
    h.close()
