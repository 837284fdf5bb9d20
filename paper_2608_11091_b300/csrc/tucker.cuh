// Tucker-level routines shared by the solvers and the C ABI.
#pragma once

#include "tk_internal.cuh"

namespace tk {

struct Dims {
    int d;
    int n[TK_MAX_D];
};

// One Tucker term coef * (*coef_dev if set) * [core; f_1, ..., f_d] of a sum; f_k is n_k x r_k.
struct TTerm {
    const double *core = nullptr;
    const double *f[TK_MAX_D] = {};
    int r[TK_MAX_D] = {};
    double coef = 1.0;
    const double *coef_dev = nullptr;
};

// Output buffers of a compression: core R^d, factors n_k x R (ld n_k), ranks (device, d ints).
struct TOut {
    double *core;
    double *f[TK_MAX_D];
    int *rank_dev;
};

struct MttJob {
    const double *core;
    int r[TK_MAX_D];
    const double *P[TK_MAX_D];
    int ldp[TK_MAX_D];
    int keep;
    double *out;
};
// tensor_cores: the leading GEMM runs on tcgen05 (mixed-precision form, gemm_oz), the row-wise
// Hadamard contractions in FP64
void mttkrp_batch(Ctx &c, int d, int s, const std::vector<MttJob> &jobs, bool tensor_cores = false);

struct TtmJob {
    const double *core;
    int r[TK_MAX_D];
    const double *P[TK_MAX_D];   // s_k x r_k
    int ldp[TK_MAX_D];
    double coef;
    const double *coef_dev;
};
struct TtmGroup {
    int sdims[TK_MAX_D];
    std::vector<TtmJob> jobs;
    double *out;
    double beta;
};
// tc: the mode products on tensor cores (mixed-precision form)
void ttm_groups(Ctx &c, int d, const std::vector<TtmGroup> &groups, bool tc = false);

struct InnerJob {
    TTerm x, y;
    double *out;
};
void inner_batch(Ctx &c, const Dims &pb, const std::vector<InnerJob> &jobs);

void kron_sketch_batch(Ctx &c, const Dims &pb, const std::vector<TTerm> &xs, const double *const *S,
                       int s, double *const *outs);

struct OpDesc {
    int nterms;
    std::vector<double> theta;
    std::vector<tk_modemat> mats;   // nterms * d
};
// tc: dense mode matrices applied on tensor cores (mixed-precision form)
std::vector<TTerm> apply_operator(Ctx &c, const Dims &pb, const OpDesc &op, const TTerm &x, int transpose,
                                  bool tc = false);

struct RSConfig {
    int sr;             // sketch size (columns of S_k)
    int R;              // rank cap; output padded to R
    double eps;         // ST-HOSVD tolerance
    uint64_t seed;
    uint64_t call;      // RoundSum call index (stream id)
    int bf16_sketch;    // mixed-precision form: Gaussian matrices rounded to bfloat16 and the
                        // range finder's products (factor sketches U^T S, the MTTKRP, rotated
                        // sketches) on tensor cores (gemm_oz): they only choose the subspace,
                        // the FP64 projection onto it keeps the result exact
    // mixed form, flexible preconditioner application only: every product of the compression
    // on tensor cores (any Z_k is a valid preconditioned direction, Section 3.4)
    int tc_all = 0;
    // optional orthogonal n_k x n_k matrices Q_k (device): the terms are given in the basis Q_k
    // (term factors Q_k^T U), so the sketches are rotated into it (S_k <- Q_k^T S_k) and the
    // output factors rotated back (U <- Q_k U): the result is RoundSum of the terms Q_k U with
    // the sketches S_k, computed without forming Q_k U
    const double *const *rot = nullptr;
    // adaptive sketch size (Section 3.1): when adaptive_p >= 0, sr is replaced by
    // min(max_k r~_k, R) + adaptive_p, r~_k from the Gram eigenvalues of the energy-weighted
    // concatenated factors at relative threshold rank_tol
    int adaptive_p = -1;
    double rank_tol = 0.0;
    int *sr_used = nullptr;   // optional host output: the sketch size this call used
};
// The effective-rank sketch size of a sum (Section 3.1); see RSConfig::adaptive_p.
int effective_sketch_size(Ctx &c, const Dims &pb, const std::vector<TTerm> &terms, int cap, int p,
                          double rank_tol);
void roundsum(Ctx &c, const Dims &pb, const std::vector<TTerm> &terms, const RSConfig &cfg, const TOut &out);

// Exponential-sum preconditioner (Section 3.4) in the sine eigenbasis of T_n: per mode the
// basis V_k (n_k x n_k, symmetric orthogonal) and the weights w[h][i] = exp(-t_h lambda_i).
struct ExpSumPC {
    int q = 0, nh = 0;
    std::vector<double> coef;              // c_h = eta t_h, h = -q..q
    const double *V[TK_MAX_D] = {};
    const double *w[TK_MAX_D] = {};        // nh x n_k, row h contiguous
};
// Terms of M(X) in the sine basis: [c_h G; diag(w_h) V_1^T U_1, ..., diag(w_h) V_d^T U_d]
std::vector<TTerm> expsum_terms(Ctx &c, const Dims &pb, const ExpSumPC &es, const TTerm &x, bool tc = false);

// tc: the sketched core's TTM chain on tensor cores (mixed-precision form); mln_recovery's tc is
// accepted for symmetry and unused (its products feed R^+ and the representation: FP64)
void mln_sketch_sum(Ctx &c, const Dims &pb, const std::vector<TTerm> &terms, const double *const *psi,
                    int r, int p, double *gpsi, double *const *F, double beta, bool tc = false);
void mln_recovery(Ctx &c, const Dims &pb, const double *gpsi, const double *const *F,
                  const double *const *psi, int r, int p, const TOut &out, bool tc = false);

}  // namespace tk
