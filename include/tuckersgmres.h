/*
 * tuckersgmres.h - C ABI of the B300 (sm_103a) Tucker-format sketched GMRES library.
 *
 * Solves L(X) = B (Section 1, Eq. (1.1)-(1.2)) with B and X Tucker tensors
 * (Section 2.3, Eq. (2.3)) and L = sum_t theta_t A_1^(t) x ... x A_d^(t) given as a list of
 * per-mode matrix tuples, by RHOSVD-Tucker sGMRES (Algorithm 2) or MLN-Tucker sGMRES
 * (Algorithm 6).  Every step runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions (all entry points):
 *   - Tensors are column-major: a core G in R^{r_1 x ... x r_d} stores G[i_1,..,i_d] at
 *     i_1 + r_1 (i_2 + r_2 (...)); a factor U_k in R^{n_k x r_k} stores U[i,j] at i + n_k j.
 *     The operator is applied in mode-product form L(X) = sum_t theta_t X x_1 A_1^(t) .. x_d A_d^(t),
 *     i.e. vec(L(X)) = sum_t theta_t (A_d^(t) kron ... kron A_1^(t)) vec(X), vec column-major.
 *   - "device" pointers are CUDA device memory of the handle's device; "host" pointers are
 *     ordinary host memory.  Inputs are borrowed: the caller keeps them alive and unchanged
 *     until the work on `stream` has completed.  Outputs are caller-allocated.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Entry points that return a
 *     value through a host pointer synchronize that stream; the others only enqueue work.
 *   - Every entry point returns a tk_status; 0 is success.  Negative values are errors; the
 *     handle's message is then available from tk_last_error().  Errors leave outputs undefined.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef TUCKERSGMRES_H
#define TUCKERSGMRES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TK_MAX_D 8

typedef enum {
    TK_OK = 0,                  /* converged: sketched residual < eta * tol                  */
    TK_NOT_CONVERGED = 1,       /* maxit iterations ran; x is the last iterate                */
    TK_BREAKDOWN = 2,           /* ||W|| ~ 0: the Krylov space is invariant; x is final       */
    TK_SKETCH_EXHAUSTED = 3,    /* the iteration count reached sketch size - 1                */
    TK_SUSPENDED = 4,           /* opts->stop_after iterations ran; the Krylov state is held  */
                                /* by the handle (tk_checkpoint_save), x is not written       */
    TK_EINVAL = -1,             /* invalid argument (shape, kind, null pointer, size limit)   */
    TK_ENOMEM = -2,             /* device allocation failed                                   */
    TK_ECUDA = -3,              /* a CUDA runtime call or kernel launch failed                 */
    TK_EINTERNAL = -4           /* a device-side check failed (non-finite value, bad state)   */
} tk_status;

/* Tucker tensor (Section 2.3): core (device, column-major r_1 x..x r_d) and factors
 * (device, column-major n_k x r_k with leading dimension n_k). */
typedef struct {
    int32_t d;
    int64_t n[TK_MAX_D];
    int64_t r[TK_MAX_D];
    double *core;
    double *factor[TK_MAX_D];
} tk_tucker;

/* One mode matrix A in R^{n x n} (Eq. (1.2)).
 *   TK_IDENTITY: data unused.
 *   TK_BANDED:   kl sub- and ku super-diagonals in LAPACK band layout, device memory,
 *                data[(ku + i - j) + (kl + ku + 1) j] = A[i, j]; covers diagonal, bidiagonal,
 *                tridiagonal and banded Toeplitz blur matrices.
 *   TK_DENSE:    device, column-major n x n. */
typedef enum { TK_IDENTITY = 0, TK_BANDED = 1, TK_DENSE = 2 } tk_kind;

typedef struct {
    int32_t kind;
    int32_t kl, ku;
    int64_t n;
    const double *data;
} tk_modemat;

/* L = sum_t theta[t] * A_1^(t) x ... x A_d^(t) (Eq. (1.2)); theta is host memory,
 * mats is a host array of nterms*d mode matrices, mats[t*d + k] = A_{k+1}^(t). */
typedef struct {
    int32_t nterms;
    int32_t d;
    const double *theta;
    const tk_modemat *mats;
} tk_operator;

/* TK_RHOSVD_GMRES: Algorithm 1 (full Arnoldi, least squares on the Hessenberg matrix; the
 * comparator of the paper's experiments; sketch_s, ktrunc and eta unused, stops at res < tol). */
enum { TK_RHOSVD_SGMRES = 0, TK_MLN_SGMRES = 1, TK_RHOSVD_GMRES = 2 };
enum { TK_FP64 = 0, TK_MIXED = 1 };

/* Solver options (Algorithm 2 inputs; Algorithm 6 inputs). */
typedef struct {
    int32_t variant;        /* TK_RHOSVD_SGMRES, TK_MLN_SGMRES or TK_RHOSVD_GMRES                 */
    int32_t rank_cap;       /* RHOSVD: multilinear rank cap; MLN: Nystrom target rank r           */
    int32_t sketch_s;       /* RHOSVD: Krylov sketch size s (MLN uses r + p)                      */
    int32_t oversample_p;   /* RHOSVD: RoundSum oversampling (paper: 5); MLN: Nystrom p            */
    int32_t ktrunc;         /* short-recurrence window k_trunc >= 1                               */
    int32_t maxit;          /* N_max                                                               */
    int32_t adaptive_rank;  /* RHOSVD: 1 = effective-rank sketch size (Section 3.1): each RoundSum */
                            /* uses min(max_k r~_k, rank_cap) + p columns, r~_k the smallest r   */
                            /* whose tail of the eigenvalues of V_k^T V_k, V_k = [|c_i| ||G_i||   */
                            /* U_k^(i)]_i, is <= round_tol^2 of their sum (formed when V_k has   */
                            /* <= 96 rows or columns, else r~_k = rank_cap); 0 = rank_cap + p;    */
                            /* ignored by the MLN variant, which has no RoundSum                  */
    int32_t precision;      /* TK_FP64 or TK_MIXED                                                 */
    int32_t transpose;      /* 1 = solve the adjoint system L^T(X) = B                            */
    int32_t mln_r_sol;      /* MLN memory-efficient variant (Section 3.3): 0 = off; else the     */
    int32_t mln_p_sol;      /* solution rank r_sol <= rank_cap and p_sol, r_sol + p_sol <= r + p:  */
                            /* stored sketches leaving the window are cut to r_sol + p_sol, the   */
                            /* solution is recovered at rank r_sol (x_out zero-padded)            */
    int32_t gcv_tikhonov;   /* 1: projected Tikhonov in every least-squares step, the parameter    */
                            /* chosen by GCV over sigma_max 10^(-12+12g/120), g = 0..120          */
                            /* (Section 4.3); needs at most 96 iterations                          */
    int32_t gcv_rows;       /* rows m in GCV's trace(I - A_lambda) for the sketched variants:     */
                            /* 0 = k + 1 (the dimension of span[M_k, S b], where the sketched     */
                            /* residual lives; the count Algorithm 1 uses for its k + 1 x k        */
                            /* Hessenberg matrix), 1 = every row of the sketch (s, or r + p)      */
    int32_t stop_after;     /* > 0: suspend after this many iterations of this call if the solve  */
                            /* has not ended (status TK_SUSPENDED; the handle keeps the Krylov    */
                            /* state); 0 = run to the end                                          */
    int32_t resume;         /* 1: continue the solve suspended in this handle (same operator, b,   */
                            /* preconditioner and options apart from stop_after / resume /        */
                            /* true_residual); the continued iterations are bit-for-bit those of  */
                            /* an uninterrupted solve                                              */
    int32_t true_residual;  /* 1: report->true_res = ||L(x) - b|| / ||b|| of the returned x       */
    double tol;             /* tolerance                                                           */
    double eta;             /* sketched correction factor: stop when res_k < eta * tol             */
    double round_tol;       /* ST-HOSVD tolerance epsilon (RoundSum)                               */
    uint64_t seed;          /* key of the Gaussian sketch stream                                   */
} tk_opts;

/* Solve report.  res_hist is caller-owned host memory of res_hist_len doubles (may be NULL). */
typedef struct {
    int32_t iters;
    int32_t status;                 /* TK_OK, TK_NOT_CONVERGED, TK_BREAKDOWN, TK_SKETCH_EXHAUSTED */
    double sketched_res;            /* final ||M y - b_s|| / ||b_s||                            */
    double *res_hist;
    int32_t res_hist_len;
    int32_t out_rank[TK_MAX_D];     /* multilinear rank of x (x is zero-padded beyond it)        */
    double ms_total;                /* device time of the solve (CUDA events)                   */
    int64_t workspace_bytes;        /* device workspace held by the handle after the solve       */
    int64_t kernel_launches;        /* kernels the library launched for this call                */
    double true_res;                /* ||L(x) - b|| / ||b|| when opts->true_residual, else -1      */
} tk_report;

typedef struct tk_handle tk_handle;

/* Create a handle bound to CUDA device `device`.  The handle owns a growable device
 * workspace (cudaMalloc on first need) released by tk_destroy. */
int tk_create(tk_handle **h, int device);
int tk_destroy(tk_handle *h);
/* Message of the last error on this handle (valid until the next call). */
const char *tk_last_error(const tk_handle *h);

/* tk_profile: enable (1) or disable (0) per-kernel device timing on this handle.  When
 * enabled, every kernel the library launches is bracketed by two CUDA events recorded on the
 * launching stream (a few microseconds of host overhead per launch).  The paper has no
 * counterpart; this is measurement plumbing. */
int tk_profile(tk_handle *h, int32_t enable);
/* tk_profile_report: per-kernel totals since the last report, one line per kernel name:
 * "<name> <launches> <total_ms> <algorithmic_flops> <algorithmic_bytes>\n" (flops counted from
 * the shapes for the GEMM, QR, SVD and contraction kernels; bytes, each operand read once and each
 * result written once, for the streaming kernels; 0 where not defined); resets the totals.  Synchronizes on the recorded events.
 * The returned string is owned by the handle and valid until the next call on it. */
const char *tk_profile_report(tk_handle *h);

/* tk_fma_peak: measured FMA throughput of the handle's device in TFLOP/s (fp64 = 1: FP64 DFMA,
 * 0: FP32 FFMA), written to *tflops_host: 8 independent FMA chains per thread over 8 CTAs of
 * 256 threads per SM, best of three timed launches after a warm-up launch (CUDA events).  The
 * paper has no counterpart; it is the denominator of the library's ALU rooflines.
 * Synchronizes. */
int tk_fma_peak(tk_handle *h, int32_t fp64, double *tflops_host, void *stream);

/* tk_solve: RHOSVD-Tucker sGMRES (Algorithm 2), MLN-Tucker sGMRES (Algorithm 6) or
 * RHOSVD-Tucker GMRES (Algorithm 1, opts->variant) for L(X) = B (or L^T(X) = B when
 * opts->transpose).  x_out is caller-allocated with
 * x_out->r[k] = rank_cap for every mode (core rank_cap^d, factors n_k x rank_cap); the
 * solution is written zero-padded and report->out_rank holds its multilinear rank.
 * Synchronizes `stream`.  Returns TK_OK / TK_NOT_CONVERGED / TK_BREAKDOWN /
 * TK_SKETCH_EXHAUSTED (all successful, x_out valid) or a negative error. */
int tk_solve(tk_handle *h, const tk_operator *op, const tk_tucker *b, const tk_opts *opts,
             tk_tucker *x_out, tk_report *report, void *stream);

/* tk_solve_precond: RHOSVD-Tucker sGMRES with flexible preconditioning (Section 3.4): each
 * iteration forms Z_k = RoundSum(M(V_k)) with the separable operator `precond` (same layout as
 * `op`), sketches RoundSum(L(Z_k)), and the solution is RoundSum(sum_i y_i Z_i).  Otherwise as
 * tk_solve; TK_EINVAL for the MLN variant or a NULL precond. */
int tk_solve_precond(tk_handle *h, const tk_operator *op, const tk_operator *precond, const tk_tucker *b,
                     const tk_opts *opts, tk_tucker *x_out, tk_report *report, void *stream);

/* tk_solve_expsum: tk_solve_precond with the exponential-sum inverse of the Laplacian of
 * tk_expsum_laplacian (Section 3.4: 2q+1 terms c_h E_h x .. x E_h, E_h = exp(-t_h T_{n_k}) in
 * mode k, c_h = eta t_h, t_h = exp(h eta), eta = pi / sqrt(q)) applied as the paper applies it,
 * through the sine eigenbasis V_k of T_{n_k} (the DST-I): with U^_k = V_k^T U_k the terms of M(X)
 * are [c_h G; diag(w_h) U^_1, ..] in that basis (w_h = exp(-t_h lambda)), RoundSum draws its
 * Gaussian sketches S_k as usual and applies them rotated (V_k^T S_k), and the compressed
 * factors are rotated back by V_k.  In exact arithmetic this is RoundSum(M(V_k)) with the
 * sketches S_k, i.e. tk_solve_precond with the dense E_h; it needs three n_k x n_k products per
 * mode per application instead of 2q+1.  Builds V_k and the weights on the device (n_k <= 16384);
 * q = 1..64.  Otherwise as tk_solve_precond. */
int tk_solve_expsum(tk_handle *h, const tk_operator *op, int32_t q, const tk_tucker *b, const tk_opts *opts,
                    tk_tucker *x_out, tk_report *report, void *stream);

/* tk_solve_concurrent: independent solves run at the same time, each on its own host thread,
 * handle and stream, so that their kernels overlap on the GPU (a single solve is a chain of
 * small dependent launches that leaves most SMs idle; the forward and adjoint solves of a
 * gradient are independent).  The paper has no counterpart.  Job i is what tk_solve
 * (precond == NULL, expsum_q == 0), tk_solve_precond (precond set) or tk_solve_expsum
 * (expsum_q > 0) would do with the same arguments; its return value is stored in jobs[i].status.
 * Every job needs its own handle (TK_EINVAL otherwise; a handle is used by one thread at a time)
 * and should have its own stream.  Returns TK_OK when every job succeeded (status >= 0), else the
 * first negative status.  Synchronizes every job's stream.  The mixed form's tensor-core timeout
 * flag is shared by the library, so a timeout may be reported by another concurrent mixed job. */
typedef struct {
    tk_handle *h;
    const tk_operator *op;
    const tk_operator *precond;
    int32_t expsum_q;
    const tk_tucker *b;
    const tk_opts *opts;
    tk_tucker *x_out;
    tk_report *report;
    void *stream;
    int32_t status;
} tk_solve_job;
int tk_solve_concurrent(int32_t count, tk_solve_job *jobs);

/* tk_checkpoint_save / tk_checkpoint_load: the Krylov state of a solve suspended by
 * opts->stop_after (status TK_SUSPENDED) as an opaque byte string in host memory, so that a
 * long solve can stop and continue later, in another handle or another process (the paper
 * has no counterpart; the state is the loop variables of Algorithms 1, 2 and 6 after
 * iteration k).  Contents: the Krylov tensors the remaining iterations and the final sum
 * read (Algorithm 2: V_1..V_{k+1}, and Z_1..Z_k in the flexible form; Algorithm 1: V_1..V_{k+1}
 * with the Hessenberg matrix; Algorithm 6: the window's tensors and every stored sketch, cut
 * or full), the sketched columns M and b_s, the least-squares factorisation (reflectors, tau,
 * Q^T b, the compact WY factor), the residual history and the RoundSum call counter; the
 * Gaussian sketch matrices are regenerated from the seed.  The string also records the
 * problem's shape and options, and a resume with different ones fails with TK_EINVAL.
 *   save: with buf == NULL writes only the size to *size_out; otherwise copies the state into
 *         buf (host, cap bytes; TK_EINVAL when cap is too small or no solve is suspended).
 *   load: replaces the handle's suspended state by buf (host, size bytes; the format is
 *         checked, TK_EINVAL if it is not a checkpoint of this library).
 * A following tk_solve / tk_solve_precond with opts->resume = 1 continues the solve; its
 * iterations and result are bit-for-bit those of the uninterrupted solve.  Synchronizes. */
int tk_checkpoint_save(tk_handle *h, void *buf, int64_t cap, int64_t *size_out);
int tk_checkpoint_load(tk_handle *h, const void *buf, int64_t size);

/* tk_set_workspace_limit: cap the device workspace the handle may hold (bytes; 0 = no cap).
 * A call that would need more fails with TK_ENOMEM before launching work that depends on the
 * missing memory, and the handle stays usable.  The paper has no counterpart; this is the hook
 * through which callers (and the tests) bound the library's device memory. */
int tk_set_workspace_limit(tk_handle *h, int64_t bytes);

/* tk_selftest_qr_wait: failure detection of the multi-cluster QR without a fault.  Runs one
 * R-only QR of a 2560 x 50 matrix on two 16-CTA clusters (the path the ST-HOSVD of tall
 * unfoldings takes) with one exchange made to go missing: mode 1, the CTAs of cluster 0 expect 8
 * bytes more than their peers push at the first step; mode 2, CTA 0 does not publish its first
 * step's sums to the other cluster.  The waiting CTAs give up after their bound (~0.3 s), set the
 * library's QR error flag and run to the end, so the context stays usable.  The paper has no
 * counterpart.  Returns TK_OK when the lost exchange was detected (the flag is then cleared),
 * TK_EINTERNAL when it was not, TK_EINVAL for another mode.  Synchronizes `stream`. */
int tk_selftest_qr_wait(tk_handle *h, int32_t mode, void *stream);

/* tk_expsum_laplacian: the exponential-sum approximation of the inverse Laplacian
 * (Section 3.4): Delta_d^{-1} ~ sum_{h=-q}^{q} c_h E_h x ... x E_h with E_h = exp(-t_h T_n),
 * T_n = tridiag(-1, 2, -1), t_h = exp(h eta), c_h = eta t_h, eta = pi / sqrt(q) (the printed
 * exp(+t_h Delta_1) read with the minus sign that makes the sum approximate the inverse).
 * E_h is formed on the GPU through the sine eigenpairs of T_n: V exp(-t_h Lambda) V^T.
 * mats: 2q+1 caller-allocated device n x n column-major outputs, mats[h+q] = E_h;
 * coef_host: 2q+1 doubles, coef_host[h+q] = c_h.  Build a tk_operator from them with
 * TK_DENSE mode matrices (the same E_h in every mode).  Synchronizes. */
int tk_expsum_laplacian(tk_handle *h, int64_t n, int32_t q, double *const *mats, double *coef_host, void *stream);

/* tk_apply: the Tucker matvec of Section 3.1 without recompression.  For every term t and
 * mode k writes A_k^(t) U_k (or its transpose) into out_factors[t*d + k] (device,
 * n_k x r_k, caller-allocated); the terms share x's core scaled by theta_t.  For identity
 * modes U_k is copied.  Enqueues only. */
int tk_apply(tk_handle *h, const tk_operator *op, const tk_tucker *x, int32_t transpose,
             double *const *out_factors, void *stream);

/* tk_roundsum: RoundSum (Section 3.1) of sum_i coef[i] X_i (coef host memory) with the
 * Gaussian matrices of stream (seed, purpose 2, call_index, mode).  Output rank is capped at
 * rank_cap with ST-HOSVD tolerance round_tol; sketch size rank_cap + oversample_p (or the
 * effective-rank estimate when adaptive_rank).  out is caller-allocated with r[k] = rank_cap;
 * written zero-padded; out_rank (host, d entries) receives the ranks.  Synchronizes. */
int tk_roundsum(tk_handle *h, int32_t nterms, const tk_tucker *xs, const double *coef,
                const tk_opts *opts, uint64_t call_index, tk_tucker *out, int32_t *out_rank,
                void *stream);

/* tk_kron_sketch: Kronecker-structured sketch (Algorithm 2, b_s and M columns):
 * out[l] = X x_1 S_1[:,l]^T ... x_d S_d[:,l]^T for l < s, S_k device n_k x s column-major,
 * out device (s doubles).  Enqueues only. */
int tk_kron_sketch(tk_handle *h, const tk_tucker *x, const double *const *S, int32_t s,
                   double *out, void *stream);

/* tk_inner: <X, Y>_F (Section 2.2) written to *out_host.  Synchronizes. */
int tk_inner(tk_handle *h, const tk_tucker *x, const tk_tucker *y, double *out_host, void *stream);

/* tk_residual: true relative residual ||L(X) - B||_F / ||B||_F in Tucker form (QR of the
 * concatenated factors, no n_1 x .. x n_d tensor formed), written to *rel_host.  Synchronizes. */
int tk_residual(tk_handle *h, const tk_operator *op, const tk_tucker *x, const tk_tucker *b,
                int32_t transpose, double *rel_host, void *stream);

/* tk_sum_norm: ||sum_i coef[i] X_i||_F (coef host memory) written to *out_host, in Tucker form:
 * QR of the concatenated distinct factors of each mode, then the norm of the small projected
 * core, so differences of nearly equal tensors keep their relative accuracy.  The
 * concatenated rank per mode must be <= 256.  Synchronizes. */
int tk_sum_norm(tk_handle *h, int32_t nterms, const tk_tucker *xs, const double *coef, double *out_host,
                void *stream);

/* tk_adjoint_grads: gradients of a loss l(x) through the solve x = L^{-1}(b), given the adjoint
 * solution mu of L^T(mu) = dl/dx (tk_solve with opts->transpose = 1).  The paper has no
 * counterpart; these are the adjoint contractions of the differentiable form:
 *   dtheta_host[t] = dl/dtheta_t = -<mu, A_1^(t) x ... x A_d^(t) applied to x>   (host, nterms)
 *   dcore_b        = dl/dG_b  = mu x_1 U_b1^T ... x_d U_bd^T        (device, r_b1 x .. x r_bd)
 *   dfactor_b[k]   = dl/dU_bk = mu_(k) (kron_{j != k} U_bj) G_b(k)^T  (device, n_k x r_bk)
 * for b = [G_b; U_b1, ..., U_bd].  Any output pointer may be NULL to skip it.  Synchronizes. */
int tk_adjoint_grads(tk_handle *h, const tk_operator *op, const tk_tucker *mu, const tk_tucker *x,
                     const tk_tucker *b, double *dtheta_host, double *dcore_b, double *const *dfactor_b,
                     void *stream);

/* tk_gaussian: `count` values of the N(0,1) stream (seed, stream_id) - Philox4x32-10 with
 * Box-Muller, element e from counter (e/2, stream_id) - into out (device).  bf16_round = 1
 * rounds each value to the nearest bfloat16 (ties to even).  Enqueues only. */
int tk_gaussian(tk_handle *h, uint64_t seed, uint64_t stream_id, int64_t count,
                int32_t bf16_round, double *out, void *stream);

/* tk_philox: raw Philox4x32-10 words of counter blocks [first, first + nblocks) for
 * stream_id and key seed: out[4*i + w] (device, uint32).  Enqueues only. */
int tk_philox(tk_handle *h, uint64_t seed, uint64_t stream_id, uint64_t first, int64_t nblocks,
              uint32_t *out, void *stream);

/* tk_sketched_ls: y = argmin ||M y - b||_2 for M (device, s x k column-major, lda = s),
 * b (device, s), via Householder QR (Algorithm 2 least-squares step; the reflectors applied in
 * compact WY form for k <= 256, one at a time beyond); writes y (device, k)
 * and the residual norm ||M y - b|| to *res (device).  Enqueues only.  Requires k < s <= 1024. */
int tk_sketched_ls(tk_handle *h, const double *M, const double *b, int32_t s, int32_t k,
                   double *y, double *res, void *stream);

/* tk_sketched_ls_static: the same least-squares solve as tk_sketched_ls, for callers that
 * must not allocate device memory after start-up (an application that reserves the GPU's
 * memory up front for its own allocator, or a latency-critical loop that cannot accept
 * cudaMalloc's implicit device synchronisation).  The paper has no counterpart; this is an
 * interface for such callers.  It takes no handle and allocates nothing: its workspace is a
 * fixed 645 KiB array in the library's device image (reflectors s x k, tau, Q^T b and the
 * k x k compact-WY factor at s <= 512, k <= 128), resident on every GPU that loads the library until the process exits.
 * M (device, s x k column-major), b (device, s), y (device, k) and res (device, 1) belong to
 * the caller.  Sizes with k < 1, k >= s, s > 512 or k > 128 return TK_EINVAL; a CUDA failure
 * returns TK_ECUDA (no message: there is no handle).  The first call on a device looks up the
 * array's device address on that device (cudaGetSymbolAddress, with the device current); make
 * that first call before any stream capture.  The address is kept for the life of the process:
 * after cudaDeviceReset of a device it no longer names the array, so do not call this entry
 * point on a device that has been reset.  Every call shares the one array and it keeps the
 * last call's contents, so calls that may overlap on the GPU (different streams, or devices
 * sharing a context) race: serialise them.  Enqueues only. */
int tk_sketched_ls_static(const double *M, const double *b, int32_t s, int32_t k, double *y,
                          double *res, void *stream);

/* tk_mln_roundsum: MLN_Sketch + MLN_Sum + MLN_Recovery (Algorithms 3-5) of
 * sum_i coef[i] X_i with Psi_k (device, n_k x (r+p)); out caller-allocated with r[k] = r.
 * Enqueues only. */
int tk_mln_roundsum(tk_handle *h, int32_t nterms, const tk_tucker *xs, const double *coef,
                    const double *const *psi, int32_t r, int32_t p, tk_tucker *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TUCKERSGMRES_H */
