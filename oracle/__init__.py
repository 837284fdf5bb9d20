"""FP64 CPU oracle for the Tucker-format sketched GMRES solvers.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
baseline leg may import this package.  The product path (the CUDA library and its
Python binding) never imports it and shares no code with it; the two meet only in
the seeded input generators of the `workloads` module.

Plain, slow and written to be checked against the paper by eye:
  tensor.py    Section 2.2-2.3   unfoldings, TTM, Khatri-Rao, MTTKRP, Tucker inner products
  operators.py Section 1 Eq.(1.2) separable operators applied to Tucker tensors
  rhosvd.py    Section 3.1       RoundSum: Khatri-Rao sketched randomized HOSVD + ST-HOSVD
  mln.py       Section 3.3       MLN_Sketch / MLN_Sum / MLN_Recovery (Algorithms 3-5)
  sgmres.py    Algorithms 1, 2, 6   RHOSVD-Tucker GMRES and sGMRES, MLN-Tucker sGMRES (with the
               memory-efficient sketches); dense sGMRES (Eq. 2.8); Section 4.3 projected
               Tikhonov with the GCV parameter
  precond.py   Section 3.4       exponential-sum inverse Laplacian, the flexible iteration's preconditioner
  residual.py  Algorithm 1-2 output contract   true relative residual in Tucker form
  adjoint.py   (no counterpart in the paper)   gradients of a loss through the solve

Every function is FP64.  Library primitives (matmul, LAPACK QR, SVD, least squares)
serve as single steps; there is no blocking, fusion or reordering beyond the
algorithms as the paper states them.  Parity is pinned by tests/test_oracle_pins.py
against closed forms, brute force on small dense problems and invariants; no
function here is parity-unpinned.
"""
