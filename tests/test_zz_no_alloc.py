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
