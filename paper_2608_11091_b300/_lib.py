"""ctypes declarations of the C ABI in include/tuckersgmres.h.

Loading fails loudly: there is no fallback implementation of any entry point.
"""
from __future__ import annotations

import ctypes
import os

TK_MAX_D = 8
HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtuckersgmres.so")

TK_OK, TK_NOT_CONVERGED, TK_BREAKDOWN, TK_SKETCH_EXHAUSTED, TK_SUSPENDED = 0, 1, 2, 3, 4
TK_EINVAL, TK_ENOMEM, TK_ECUDA, TK_EINTERNAL = -1, -2, -3, -4
TK_IDENTITY, TK_BANDED, TK_DENSE = 0, 1, 2
TK_RHOSVD_SGMRES, TK_MLN_SGMRES, TK_RHOSVD_GMRES = 0, 1, 2
TK_FP64, TK_MIXED = 0, 1

EXPORTS = ["tk_create", "tk_destroy", "tk_last_error", "tk_solve", "tk_apply", "tk_roundsum",
           "tk_kron_sketch", "tk_inner", "tk_residual", "tk_gaussian", "tk_philox",
           "tk_sketched_ls", "tk_mln_roundsum", "tk_profile", "tk_profile_report",
           "tk_sketched_ls_static", "tk_sum_norm", "tk_adjoint_grads", "tk_solve_precond",
           "tk_expsum_laplacian", "tk_checkpoint_save", "tk_checkpoint_load", "tk_set_workspace_limit",
           "tk_fma_peak", "tk_solve_expsum", "tk_solve_concurrent", "tk_selftest_qr_wait"]


class tk_tucker(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32),
                ("n", ctypes.c_int64 * TK_MAX_D),
                ("r", ctypes.c_int64 * TK_MAX_D),
                ("core", ctypes.c_void_p),
                ("factor", ctypes.c_void_p * TK_MAX_D)]


class tk_modemat(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("kl", ctypes.c_int32), ("ku", ctypes.c_int32),
                ("n", ctypes.c_int64), ("data", ctypes.c_void_p)]


class tk_operator(ctypes.Structure):
    _fields_ = [("nterms", ctypes.c_int32), ("d", ctypes.c_int32),
                ("theta", ctypes.POINTER(ctypes.c_double)),
                ("mats", ctypes.POINTER(tk_modemat))]


class tk_opts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("rank_cap", ctypes.c_int32),
                ("sketch_s", ctypes.c_int32), ("oversample_p", ctypes.c_int32),
                ("ktrunc", ctypes.c_int32), ("maxit", ctypes.c_int32),
                ("adaptive_rank", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("transpose", ctypes.c_int32), ("mln_r_sol", ctypes.c_int32),
                ("mln_p_sol", ctypes.c_int32), ("gcv_tikhonov", ctypes.c_int32),
                ("gcv_rows", ctypes.c_int32), ("stop_after", ctypes.c_int32),
                ("resume", ctypes.c_int32), ("true_residual", ctypes.c_int32),
                ("tol", ctypes.c_double), ("eta", ctypes.c_double),
                ("round_tol", ctypes.c_double), ("seed", ctypes.c_uint64)]


class tk_solve_job(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p), ("op", ctypes.c_void_p), ("precond", ctypes.c_void_p),
                ("expsum_q", ctypes.c_int32), ("b", ctypes.c_void_p), ("opts", ctypes.c_void_p),
                ("x_out", ctypes.c_void_p), ("report", ctypes.c_void_p), ("stream", ctypes.c_void_p),
                ("status", ctypes.c_int32)]


class tk_report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("sketched_res", ctypes.c_double),
                ("res_hist", ctypes.POINTER(ctypes.c_double)),
                ("res_hist_len", ctypes.c_int32),
                ("out_rank", ctypes.c_int32 * TK_MAX_D),
                ("ms_total", ctypes.c_double),
                ("workspace_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64),
                ("true_res", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} not found: build the CUDA library first "
            "(python -m paper_2608_11091_b300.build); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, i32, i64, u64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, P(ctypes.c_double)
    sig = {
        "tk_create": (ctypes.c_int, [P(vp), ctypes.c_int]),
        "tk_destroy": (ctypes.c_int, [vp]),
        "tk_last_error": (ctypes.c_char_p, [vp]),
        "tk_solve": (ctypes.c_int, [vp, P(tk_operator), P(tk_tucker), P(tk_opts), P(tk_tucker), P(tk_report), vp]),
        "tk_apply": (ctypes.c_int, [vp, P(tk_operator), P(tk_tucker), i32, P(vp), vp]),
        "tk_roundsum": (ctypes.c_int, [vp, i32, P(tk_tucker), dp, P(tk_opts), u64, P(tk_tucker), P(i32), vp]),
        "tk_kron_sketch": (ctypes.c_int, [vp, P(tk_tucker), P(vp), i32, vp, vp]),
        "tk_inner": (ctypes.c_int, [vp, P(tk_tucker), P(tk_tucker), dp, vp]),
        "tk_residual": (ctypes.c_int, [vp, P(tk_operator), P(tk_tucker), P(tk_tucker), i32, dp, vp]),
        "tk_gaussian": (ctypes.c_int, [vp, u64, u64, i64, i32, vp, vp]),
        "tk_philox": (ctypes.c_int, [vp, u64, u64, u64, i64, vp, vp]),
        "tk_sketched_ls": (ctypes.c_int, [vp, vp, vp, i32, i32, vp, vp, vp]),
        "tk_mln_roundsum": (ctypes.c_int, [vp, i32, P(tk_tucker), dp, P(vp), i32, i32, P(tk_tucker), vp]),
        "tk_profile": (ctypes.c_int, [vp, i32]),
        "tk_profile_report": (ctypes.c_char_p, [vp]),
        "tk_sketched_ls_static": (ctypes.c_int, [vp, vp, i32, i32, vp, vp, vp]),
        "tk_sum_norm": (ctypes.c_int, [vp, i32, P(tk_tucker), dp, dp, vp]),
        "tk_adjoint_grads": (ctypes.c_int, [vp, P(tk_operator), P(tk_tucker), P(tk_tucker), P(tk_tucker), dp, vp, P(vp), vp]),
        "tk_solve_precond": (ctypes.c_int, [vp, P(tk_operator), P(tk_operator), P(tk_tucker), P(tk_opts), P(tk_tucker),
                                            P(tk_report), vp]),
        "tk_expsum_laplacian": (ctypes.c_int, [vp, i64, i32, P(vp), dp, vp]),
        "tk_checkpoint_save": (ctypes.c_int, [vp, vp, i64, P(i64)]),
        "tk_checkpoint_load": (ctypes.c_int, [vp, vp, i64]),
        "tk_set_workspace_limit": (ctypes.c_int, [vp, i64]),
        "tk_fma_peak": (ctypes.c_int, [vp, i32, dp, vp]),
        "tk_selftest_qr_wait": (ctypes.c_int, [vp, i32, vp]),
        "tk_solve_expsum": (ctypes.c_int, [vp, P(tk_operator), i32, P(tk_tucker), P(tk_opts), P(tk_tucker),
                                           P(tk_report), vp]),
        "tk_solve_concurrent": (ctypes.c_int, [i32, P(tk_solve_job)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib
