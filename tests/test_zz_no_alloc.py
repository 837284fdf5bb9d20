"""The allocation-free least-squares entry point (tk_sketched_ls_static) against the regular
one (tk_sketched_ls), through the C ABI, on two calls in a row with different sizes.

It exists for callers that may not allocate device memory after start-up; its workspace is
a fixed device array of the library, shared by every call.  This file is collected last so
that a run stopping at its first failure has already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_static_workspace_least_squares_matches_regular_entry_point():
    import torch
    assert torch.cuda.is_available()
    import paper_2608_11091_b300 as P
    rng = np.random.default_rng(2024)
    for s, k in [(300, 97), (64, 20)]:          # second call smaller: stale contents must not leak
        M = P.to_fortran(rng.standard_normal((s, k)), "cuda")
        b = P.to_fortran(rng.standard_normal(s), "cuda")
        y_ref, res_ref = P.tk_sketched_ls(M, b)
        y, res = P.tk_sketched_ls_static(M, b)
        torch.cuda.synchronize()
        yr, yd = y_ref.cpu().numpy(), y.cpu().numpy()
        assert np.allclose(yd, yr, rtol=1e-12, atol=1e-14)
        assert np.isclose(res.item(), res_ref.item(), rtol=1e-12)
        ynp = np.linalg.lstsq(M.cpu().numpy(), b.cpu().numpy(), rcond=None)[0]
        assert np.allclose(yd, ynp, rtol=1e-10, atol=1e-12)


def test_static_workspace_rejects_sizes_beyond_its_limits():
    import torch
    import paper_2608_11091_b300 as P
    for s, k in [(600, 10), (300, 200), (20, 20)]:
        M = P.to_fortran(np.ones((s, k)), "cuda")
        b = P.to_fortran(np.ones(s), "cuda")
        with pytest.raises(P.TuckerError):
            P.tk_sketched_ls_static(M, b)


_FRESH_PROCESS = r"""
import ctypes, sys
import numpy as np
lib = ctypes.CDLL(sys.argv[1])                 # the library (and through it the CUDA runtime)
rt = ctypes.CDLL("libcudart.so.13")
vp, sz = ctypes.c_void_p, ctypes.c_size_t
assert rt.cudaSetDevice(0) == 0 and rt.cudaFree(None) == 0      # context, modules loaded eagerly
rng = np.random.default_rng(5)
s, k = 200, 60
host = {"M": np.asfortranarray(rng.standard_normal((s, k))), "b": rng.standard_normal(s),
        "y": np.zeros(k), "res": np.zeros(1)}
dev = {}
for name, a in host.items():
    p = vp()
    assert rt.cudaMalloc(ctypes.byref(p), sz(a.nbytes)) == 0
    assert rt.cudaMemcpy(p, a.ctypes.data_as(vp), sz(a.nbytes), 1) == 0          # host to device
    dev[name] = p
h = vp()
assert lib.tk_create(ctypes.byref(h), 0) == 0
# the regular entry point first: its launch reserves what the least-squares kernel needs (and
# its handle allocates its own workspace), so what follows isolates the static entry point
assert lib.tk_sketched_ls(h, dev["M"], dev["b"], s, k, dev["y"], dev["res"], None) == 0
assert rt.cudaDeviceSynchronize() == 0
free, total = sz(), sz()
assert rt.cudaMemGetInfo(ctypes.byref(free), ctypes.byref(total)) == 0
free0 = free.value
for _ in range(3):
    assert lib.tk_sketched_ls_static(dev["M"], dev["b"], s, k, dev["y"], dev["res"], None) == 0
assert rt.cudaDeviceSynchronize() == 0
assert rt.cudaMemGetInfo(ctypes.byref(free), ctypes.byref(total)) == 0
print("FREE", free0, free.value)
"""


def test_static_workspace_allocates_nothing_in_a_fresh_process():
    """In a new process without PyTorch, with the library's device image loaded eagerly at
    context creation, the first calls of the static entry point leave the device's free memory
    unchanged: the entry point allocates nothing itself."""
    import os
    import subprocess
    import sys
    import paper_2608_11091_b300 as P
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    out = subprocess.run([sys.executable, "-c", _FRESH_PROCESS, P.LIB_PATH], capture_output=True, text=True,
                         env=env, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = [ln for ln in out.stdout.splitlines() if ln.startswith("FREE")][-1]
    free0, free1 = (int(v) for v in line.split()[1:])
    assert free1 == free0, (free0, free1)
