// Internal declarations of the Tucker sGMRES CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tuckersgmres.h"

namespace tk {

// ------------------------------------------------------------------------------------------
// Errors
// ------------------------------------------------------------------------------------------
struct Error {
    int code;
    std::string msg;
};

#define TK_CUDA(call)                                                                           \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            throw ::tk::Error{TK_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};    \
    } while (0)

#define TK_REQUIRE(cond, msg)                                                                   \
    do {                                                                                        \
        if (!(cond)) throw ::tk::Error{TK_EINVAL, std::string(msg)};                            \
    } while (0)

// ------------------------------------------------------------------------------------------
// Device workspace: chunked bump allocator.  Chunks persist for the handle's lifetime, so
// after the first call of a given size no further cudaMalloc happens.
// ------------------------------------------------------------------------------------------
class Arena {
public:
    struct Mark { size_t chunk, off; };
    ~Arena();
    double *alloc(size_t n_doubles) { return static_cast<double *>(alloc_bytes(n_doubles * 8)); }
    int *alloc_int(size_t n) { return static_cast<int *>(alloc_bytes(n * 4)); }
    void *alloc_bytes(size_t bytes);
    Mark mark() const { return Mark{cur_, off_}; }
    void release(Mark m) { cur_ = m.chunk; off_ = m.off; }
    void reset() { cur_ = 0; off_ = 0; }
    size_t capacity() const;
    // cap on the device memory the arena may hold (0: none); a growth beyond it throws TK_ENOMEM
    void set_limit(size_t bytes) { limit_ = bytes; }

private:
    struct Chunk { char *base; size_t size; };
    std::vector<Chunk> chunks_;
    size_t cur_ = 0, off_ = 0;
    size_t limit_ = 0;
};

struct ScopedMark {
    Arena &a;
    Arena::Mark m;
    explicit ScopedMark(Arena &ar) : a(ar), m(ar.mark()) {}
    ~ScopedMark() { a.release(m); }
};

// Opt-in per-kernel device timing: CUDA events recorded on the launching stream around each
// launch; collected after the call has synchronized.
class Profiler {
public:
    ~Profiler();
    void begin(cudaStream_t st);
    void end(cudaStream_t st, const char *name, double flops, double bytes = 0.0);
    void collect();                       // requires the recorded work to have completed
    std::string report_and_reset();       // "name launches total_ms" lines
private:
    cudaEvent_t get();
    std::vector<cudaEvent_t> pool_;
    size_t used_ = 0;
    struct Rec { const char *name; cudaEvent_t a, b; double flops, bytes; };
    std::vector<Rec> recs_;
    cudaEvent_t open_ = nullptr;
    struct Tot { long long n = 0; double ms = 0.0, flops = 0.0, bytes = 0.0; };
    std::vector<std::pair<std::string, Tot>> tot_;
};

// Per-call context.
struct Ctx {
    cudaStream_t st;
    Arena *arena;
    int64_t launches = 0;
    int num_sms = 148;
    Profiler *prof = nullptr;
    void pre_launch() { if (prof) prof->begin(st); }
    // `flops`: algorithmic operations of the launch, `bytes`: algorithmic memory traffic (each
    // operand read once, each result written once); 0 where not defined
    void check_launch(const char *what, double flops = 0.0, double bytes = 0.0);
};

// ------------------------------------------------------------------------------------------
// Grouped FP64 GEMM:  C_p = beta_p C_p + sum_s coef_s op(A_s) op(B_s)   for each problem p,
// each problem optionally strided-batched.  op(A) is M x K (ta = 1: A stored K x M),
// op(B) is K x N (tb = 1: B stored N x K).  All column-major.
// ------------------------------------------------------------------------------------------
constexpr int GEMM_MAXSEG = 8;
constexpr int GEMM_MAXPROB = 16;

struct GSeg {
    const double *A, *B;
    const double *coef_dev;   // optional device scalar multiplying coef
    double coef;
    int K, lda, ldb;
};

struct GProb {
    int M, N, ta, tb, ldc, batch, nseg;
    long long sA, sB, sC;
    double *C;
    double beta;
    int tiles_m, tiles_n, tile_begin;
    GSeg seg[GEMM_MAXSEG];
};

struct GGroup {
    int nprob, total;
    GProb p[GEMM_MAXPROB];
};

// Host-side builder that chunks problems/segments into launches.
class Gemm {
public:
    // `tag`: the profiler's name for this builder's launches (the contraction it serves);
    // `tc`: run the problems on tensor cores (gemm_oz: sliced BF16 products, exact FP32
    // accumulation, ~2^-40 relative accuracy) where their shape allows, FP64 otherwise
    explicit Gemm(Ctx &c, const char *tag = "gemm", bool tc = false) : c_(c), tag_(tag), tc_(tc) {}
    // C = beta C + sum coef_s op(A_s) op(B_s).  Segments beyond GEMM_MAXSEG are chunked.
    struct Seg {
        const double *A; int lda;
        const double *B; int ldb;
        int K; double coef; const double *coef_dev;
    };
    void add(int M, int N, int ta, int tb, double *C, int ldc, double beta,
             const std::vector<Seg> &segs, int batch = 1, long long sA = 0, long long sB = 0,
             long long sC = 0);
    void add1(int M, int N, int K, int ta, int tb, const double *A, int lda, const double *B,
              int ldb, double *C, int ldc, double beta = 0.0, double coef = 1.0,
              const double *coef_dev = nullptr, int batch = 1, long long sA = 0,
              long long sB = 0, long long sC = 0) {
        add(M, N, ta, tb, C, ldc, beta, {Seg{A, lda, B, ldb, K, coef, coef_dev}}, batch, sA, sB, sC);
    }
    void run();   // launches everything added so far (problems may run concurrently)
    ~Gemm() {}

private:
    Ctx &c_;
    const char *tag_;
    bool tc_;
    std::vector<GProb> pending_;
    void flush_group(std::vector<GProb> &probs, int ksplit);
};

// ------------------------------------------------------------------------------------------
// Tensor-core GEMM of the mixed-precision form (k_gemm_oz.cu): the grouped problems of Gemm
// with FP64 operands sliced into BF16 digit planes, products on tcgen05 with exact FP32
// accumulation per 256-long chunk, FP64 accumulation across chunks.
// ------------------------------------------------------------------------------------------
bool oz_supported(const GProb &p);
void gemm_oz(Ctx &c, const std::vector<GProb> &probs, const char *tag);
// 1 if a tensor-core GEMM gave up waiting for its copies or MMAs since the last reset
int oz_error_flag(bool reset);
// Nonzero when a clustered SVD's replay of the FP32 rotations gave up waiting (reset clears it).
int svd_error_flag(bool reset);
// Nonzero when a multi-cluster QR gave up waiting for another cluster's sums (reset clears it).
int qr_error_flag(bool reset);
// Self-test of the multi-cluster QR's bounded waits (inject 1 or 2): 1 when the lost exchange was
// detected (kernel finished, flag set and cleared), 0 otherwise.
int qr_wait_selftest(Ctx &c, int inject);

// ------------------------------------------------------------------------------------------
// Small dense linear algebra (FP64)
// ------------------------------------------------------------------------------------------
struct QRJob {
    double *A;        // m x s column-major, lda = m; overwritten by R (upper) and reflectors
    double *tau;      // min(m, s)
    double *Q;        // optional: explicit m x s orthonormal factor (ldq = m), zero columns >= m
    int m, s;
    int *perm;        // optional: column pivoting (largest remaining norm first); column j of R
                      // belongs to input column perm[j]
};
void qr_householder(Ctx &c, const std::vector<QRJob> &jobs);

struct SVDJob {
    const double *R;  // s x s upper triangle (ld = ldr)
    int ldr, s;
    double *W;        // out: s x wcols, leading right singular vectors of R, zero-padded
    int wcols;
    double *sigma;    // out: s singular values, descending
    int *rank;        // out: kept rank (tail-energy criterion), may be null
    const double *normsq;   // device: ||C||^2 for the threshold eps^2 ||C||^2 / d (may be null)
    double eps2_over_d;
    int rank_cap;
    const int *perm;  // set: R comes from a column-pivoted QR of C^T and W receives the leading
                      // left singular vectors of C = P R^T Q^T (Jacobi on R^T, rows of W permuted)
};
void svd_jacobi(Ctx &c, const std::vector<SVDJob> &jobs);

// Incremental Householder least squares.  State arrays live in workspace.
struct LSState {
    double *H;        // s x kmax reflectors (column j holds v_j in rows j..s-1)
    double *tau;      // kmax
    double *qtb;      // s: Q^T b (rows updated incrementally)
    double *y;        // kmax
    double *res;      // 1: ||M y - b||
    double *T;        // optional, kmax x kmax (ld ldt): the compact WY factor of the reflectors
    int ldt;
};
// Compact WY least squares (T set, s <= LSW_MAXS rows, k <= LSW_MAXK columns).
constexpr int LSW_MAXS = 1024, LSW_MAXK = 256;
// Processes columns [c0, k) of M (s x k, lda = s) and solves for y_k.
void ls_update(Ctx &c, const double *M, const double *b, int s, int c0, int k, const LSState &st,
               int init_qtb);
// Projected Tikhonov with the GCV-chosen parameter on the current least-squares state (k columns,
// R in st.H with leading dimension ldr, m rows of the problem): overwrites st.y and *st.res.
void tikhonov_gcv(Ctx &c, const LSState &st, int ldr, int k, int m, double *lambda_out);

// ------------------------------------------------------------------------------------------
// Elementwise / structured kernels
// ------------------------------------------------------------------------------------------
struct BandJob {
    const double *band;   // (kl+ku+1) x n band layout
    const double *U;      // n x r
    double *out;          // n x r
    int n, r, kl, ku, trans;
};
void band_apply(Ctx &c, const std::vector<BandJob> &jobs);

// out[i, mm, l] = sum_j T[i, j, mm, l] P[j, l]  with T dims (a, b, cc, s)
struct HadJob {
    const double *T, *P;
    double *out;
    int a, b, cc, s, ldp;
};
void hadamard_contract(Ctx &c, const std::vector<HadJob> &jobs);

// out[rho + c m] = C[(rho % a) + c a + (rho / a) a sk]: transpose of the mode unfolding
void gather_unfold_t(Ctx &c, const double *C, double *out, long long a, int sk, long long rest);

void gaussian(Ctx &c, uint64_t seed, const uint64_t *sids, const long long *counts,
              double *const *outs, int nmat, int bf16);
void philox_raw(Ctx &c, uint64_t seed, uint64_t sid, uint64_t first, long long nblocks, uint32_t *out);

// out = sum_i x_i y_i  (deterministic single-CTA reduction), optionally scaled by alpha
void dot(Ctx &c, const double *x, const double *y, long long n, double *out);
struct DotJob { const double *x, *y; long long n; double *out; };
void dots(Ctx &c, const std::vector<DotJob> &jobs);

void fill(Ctx &c, double *p, long long n, double v);
void copy(Ctx &c, double *dst, const double *src, long long n);
// y = x * (*s) or (1 / *s) when inv
void scale_by(Ctx &c, double *y, const double *x, long long n, const double *s, int inv);
// copy a column-major block (rows x cols) between leading dimensions, zero-filling dst extra
void copy_pad(Ctx &c, double *dst, int ld_dst, int rows_dst, int cols_dst, const double *src,
              int ld_src, int rows_src, int cols_src);
// copy a tensor core with dims r_src into dims r_dst (zero padded), d modes
void copy_core_pad(Ctx &c, double *dst, const int *rdst, const double *src, const int *rsrc, int d);
// extract the superdiagonal G[i,..,i] of a cube with side m, d modes: out[i]
void superdiag(Ctx &c, const double *G, int m, int d, double *out, double scale_host,
               const double *scale_dev);
// dst (n x r, ld n) = |coef * (*cd or 1)| * sqrt(*normsq) * src (n x r, ld n), many jobs per launch
struct WeightedCopyJob { const double *src; double *dst; const double *cd, *normsq; double coef; int n, r; };
void weighted_copy(Ctx &c, const std::vector<WeightedCopyJob> &jobs);
// out[i + n j] = w[i] in[i + n j]  (n x r), many jobs per launch
struct RowScaleJob { const double *in, *w; double *out; int n, r; };
void row_scale(Ctx &c, const std::vector<RowScaleJob> &jobs);
// w[h n + i] = exp(-t_h lambda_i), lambda_i = 2 - 2 cos((i + 1) pi / (n + 1)), t_h = exp((h - q) eta)
void expsum_weights(Ctx &c, double *w, int n, int q, double eta);
// scalar helpers for the solver control flow
void sqrt_scalar(Ctx &c, const double *in, double *out);
// V (n x n) = sine eigenvectors of tridiag(-1,2,-1), columns scaled by exp(-t lambda_j) if t != 0
void sine_basis(Ctx &c, double *V, int n, double t);
// p = I (n x n)
void set_identity(Ctx &c, double *p, int n);
// measured FMA rate of the device in TFLOP/s (fp64 = 1: FP64, 0: FP32)
double fma_peak_tflops(Ctx &c, int fp64);
// dst (cols x rows, ld ldd) = src(rows x cols, ld lds)^T
void transpose_block(Ctx &c, double *dst, int ldd, const double *src, int lds, int rows, int cols);
// upper triangle (rows x cols) of src into dst, zeros below the diagonal
void triu_copy(Ctx &c, double *dst, int ldd, const double *src, int lds, int rows, int cols);
// pseudo-inverses of n small square matrices through their Jacobi SVD, singular values
// <= rcond * sigma_max dropped
void pinv_small(Ctx &c, const double *const *R, const int *ldr, int s, double *const *out, int n,
                double rcond);

}  // namespace tk
