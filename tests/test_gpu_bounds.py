"""Index checks of the debug build (FX_BOUNDS_CHECK; the stand-in for the closed memory sanitizer).

The debug build checks every kernel index that the sources mark (FXI, FXP, FXPR) against its
buffer's extent and reports the first index outside it as FX_ERR_BOUNDS with its site, instead
of accessing it.  Here:
  - a positive control: a probe kernel whose stated extent is smaller than its real buffer must
    report an index in the gap, with the right site, index and extent, and read element 0;
  - every kernel path of the stage update (tests/bounds_cases.py) runs through the debug build
    with no index outside its buffer, and gives the normal build's results: the states bit for
    bit, the sums that use floating-point atomics (budgets, the objective, the adjoint) to their
    rounding;
  - so do one step of the full-size kh2d and lognormal3d workloads (states compared by digest).
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, HERE)
import bounds_cases  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def test_probe_reports_the_first_index_outside_the_stated_extent(torch_cuda, tmp_path):
    torch = torch_cuda
    src = os.path.join(HERE, "cuda", "bounds_probe.cu")
    so = str(tmp_path / "probe.so")
    from paper_1806_07390_gb300 import build as B
    cmd = [B._nvcc(), *B.ARCH, "-O3", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
           "-shared", "-I", B.CSRC, src, "-o", so]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(so)
    L.fx_probe.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int]
    L.fx_probe_tag.restype = ctypes.c_uint
    buf = torch.arange(1, 65, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    status = torch.zeros(6, dtype=torch.int32, device="cuda")

    def probe(n, i):
        status.zero_()
        assert L.fx_probe(status.data_ptr(), buf.data_ptr(), out.data_ptr(), n, i) == 0
        return status.cpu().numpy().view(np.uint32), float(out.item())

    w, v = probe(64, 10)  # inside: read through, nothing recorded
    assert v == 11.0 and not w.any()
    w, v = probe(32, 40)  # outside the stated extent (inside the real buffer)
    line = next(k + 1 for k, s in enumerate(open(src)) if "the checked read" in s)
    assert w[0] == 8  # ST_BOUNDS
    assert w[1] == (L.fx_probe_tag() << 16 | line)
    assert w[2:4].view(np.int64)[0] == 40 and w[4:6].view(np.int64)[0] == 32
    assert v == 1.0  # the access went to element 0
    w, v = probe(32, -3)
    assert w[0] == 8 and w[2:4].view(np.int64)[0] == -3 and v == 1.0


def _compare(name, key, a, b):
    if key in ("state", "sha256"):
        assert a.dtype == b.dtype and np.array_equal(a, b), f"{name}: states differ"
        return
    # sums over blocks with floating-point atomics: equal to their rounding
    tol = 1e-10 if a.dtype == np.float64 and "fp32" not in name else 1e-4
    scale = max(np.max(np.abs(b)), 1e-300)
    assert np.max(np.abs(a - b)) <= tol * scale, f"{name}/{key}: {np.max(np.abs(a - b)) / scale:.2e}"


def _check_debug_build(tmp_path, cases, full):
    from paper_1806_07390_gb300 import build as B
    lib_bc = B.build(bounds_check=True)
    out = str(tmp_path / "bc.npz")
    env = dict(os.environ, FX_LIBRARY=lib_bc)
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py"), out] + (["--full"] if full else []),
                       env=env, capture_output=True, text=True, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "libfx_bc.so" in r.stdout
    bc = np.load(out)
    for name in cases:
        st = int(bc[f"{name}/status"][0])
        assert st == 0, f"{name}: debug build status {st}"
        st_n, ref = cases[name]()
        assert st_n == 0, f"{name}: normal build status {st_n}"
        keys = sorted(k.split("/", 1)[1] for k in bc.files if k.startswith(name + "/") and not k.endswith("/status"))
        assert keys == sorted(ref), (name, keys, sorted(ref))
        for k in keys:
            _compare(name, k, bc[f"{name}/{k}"], np.asarray(ref[k]))


def test_every_kernel_path_stays_inside_its_buffers(torch_cuda, tmp_path):
    _check_debug_build(tmp_path, bounds_cases.CASES, full=False)


def test_full_size_workloads_stay_inside_their_buffers(torch_cuda, tmp_path):
    # one step of kh2d 1024^2 x 16 and lognormal3d 256^3 x 12 (FP32 + FP64 Newton) in the
    # benchmark's launch configuration: the largest state offsets and the most blocks
    _check_debug_build(tmp_path, bounds_cases.FULL_CASES, full=True)
