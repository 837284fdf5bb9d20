"""Whole-solver parity cases shared by the GPU parity tests and the sensitivity script.
name -> (workload builder, solver parameters (None: the workload's own), transpose)."""
import workloads as W

CASES = {
    "poisson3d_n32_full": (lambda: W.workload("poisson3d_n32"), None, False),
    "poisson3d_n20_r12": (lambda: W.poisson3d(20, 1, 3, None, "p20"),
                          W.SolverParams('rhosvd', 12, 64, 5, 40, 1e-9, seed=4), False),
    "convdiff3d_n64": (lambda: W.convdiff3d(64, 1, None), W.SolverParams('rhosvd', 16, 96, 5, 25, 1e-8, seed=2), False),
    "deblur3d_n48": (lambda: W.deblur3d(48, 2, None), W.SolverParams('rhosvd', 16, 128, 5, 8, 1e-8, seed=5), False),
    "convdiff_ragged": (lambda: W.convdiff3d(37, 3, None, rhs_rank=2),
                        W.SolverParams('rhosvd', 7, 33, 6, 20, 1e-8, ktrunc=3, seed=6), False),
    "mln_varcoef4d_n16": (lambda: W.varcoef4d(16, 1, None), W.SolverParams('mln', 6, 0, 6, 10, 1e-8, seed=7), False),
    "mln_convdiff_n40": (lambda: W.convdiff3d(40, 2, None), W.SolverParams('mln', 10, 0, 12, 16, 1e-8, seed=8), False),
    "adjoint_convdiff_n30": (lambda: W.convdiff3d(30, 4, None), W.SolverParams('rhosvd', 10, 64, 5, 15, 1e-8, seed=9), True),
    "exhaustion_convdiff_n16": (lambda: W.convdiff3d(16, 5, None), W.SolverParams('rhosvd', 4, 10, 5, 40, 1e-14, seed=1), False),
    "point_source_n64": (lambda: W.poisson3d_point(64, None, 8, "p64"),
                         W.SolverParams('rhosvd', 32, 64, 5, 6, 1e-8, eta=0.4, ktrunc=1, seed=2), False),
    # MLN memory-efficient variant (Section 3.3): stored sketches cut to r_sol + p_sol
    "mln_save_varcoef4d_n16": (lambda: W.varcoef4d(16, 1, None),
                               W.SolverParams('mln', 6, 0, 6, 10, 1e-8, seed=7, r_sol=4, p_sol=4), False),
    "mln_save_convdiff_n40": (lambda: W.convdiff3d(40, 2, None),
                              W.SolverParams('mln', 10, 0, 12, 16, 1e-8, ktrunc=3, seed=8, r_sol=8, p_sol=8), False),
    # projected Tikhonov with the GCV parameter (Section 4.3), noisy deblurring
    "tik_sgmres_deblur_n24": (lambda: W.deblur3d_noisy(24, 3, None),
                              W.SolverParams('rhosvd', 12, 64, 5, 20, 1e-8, seed=3, tikhonov=True), False),
    "tik_sgmres_deblur_n24_sketchrows": (lambda: W.deblur3d_noisy(24, 3, None),
                                         W.SolverParams('rhosvd', 12, 64, 5, 20, 1e-8, seed=3, tikhonov=True,
                                                        gcv_rows="sketch"), False),
    "tik_gmres_deblur_n16": (lambda: W.deblur3d_noisy(16, 4, None),
                             W.SolverParams('gmres', 10, 0, 5, 15, 1e-8, seed=4, tikhonov=True), False),
    "tik_mln_deblur_n16": (lambda: W.deblur3d_noisy(16, 5, None),
                           W.SolverParams('mln', 8, 0, 16, 12, 1e-8, seed=5, tikhonov=True), False),
    # effective-rank RoundSum sketch size (Section 3.1): rank-1 right-hand side, so the early
    # Krylov tensors have low rank and the estimate is below rank_cap + p
    "adaptive_poisson3d_n20": (lambda: W.poisson3d(20, 1, 3, None, "p20"),
                               W.SolverParams('rhosvd', 12, 64, 5, 10, 1e-9, seed=4, adaptive_rank=True), False),
    "adaptive_gmres_convdiff_ragged": (lambda: W.convdiff3d(37, 3, None, rhs_rank=2),
                                       W.SolverParams('gmres', 7, 0, 6, 10, 1e-8, seed=6, adaptive_rank=True), False),
    # Algorithm 1 (full Arnoldi through RoundSum)
    "gmres_poisson3d_n20_r12": (lambda: W.poisson3d(20, 1, 3, None, "p20"),
                                W.SolverParams('gmres', 12, 0, 5, 30, 1e-9, seed=4), False),
    "gmres_convdiff_ragged": (lambda: W.convdiff3d(37, 3, None, rhs_rank=2),
                              W.SolverParams('gmres', 7, 0, 6, 15, 1e-8, seed=6), False),
    "gmres_adjoint_convdiff_n30": (lambda: W.convdiff3d(30, 4, None), W.SolverParams('gmres', 10, 0, 5, 12, 1e-8, seed=9),
                                   True),
}


# Mixed-precision parity cases: (builder, parameters); RoundSum sketches rounded to BF16.
MIXED_CASES = {
    "poisson3d_n20_r12": (lambda: W.poisson3d(20, 1, 3, None, "p20"), W.SolverParams('rhosvd', 12, 64, 5, 25, 1e-9, seed=4)),
    "convdiff3d_n48": (lambda: W.convdiff3d(48, 1, None), W.SolverParams('rhosvd', 12, 96, 5, 15, 1e-8, seed=2)),
    "deblur3d_n40": (lambda: W.deblur3d(40, 2, None), W.SolverParams('rhosvd', 12, 128, 5, 8, 1e-8, seed=5)),
    "convdiff3d_n256_prefix": (lambda: W.workload("convdiff3d_n256"), W.SolverParams('rhosvd', 32, 128, 5, 10, 1e-6, seed=0)),
}


# Preconditioned (flexible) parity cases: (builder, parameters, q of the exponential sum).
PRECOND_CASES = {
    "poisson3d_n32_q8": (lambda: W.workload("poisson3d_n32"), W.SolverParams('rhosvd', 12, 64, 5, 20, 3e-7, seed=3), 8),
    "poisson3d_n32_q8_r16": (lambda: W.workload("poisson3d_n32"), W.SolverParams('rhosvd', 16, 64, 5, 20, 2e-8, seed=3), 8),
    "point_n203_q4": (lambda: W.poisson3d_point(203, None, 4, "p203"),
                      W.SolverParams('rhosvd', 17, 40, 9, 12, 1e-6, eta=0.4, ktrunc=2, seed=11), 4),
    "poisson3d_point_n1000": (lambda: W.workload("poisson3d_point_n1000"), None, 8),
}
