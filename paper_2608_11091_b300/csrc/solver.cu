// Solver drivers (Algorithms 2 and 6) and the C ABI.
#include <cmath>
#include <cstring>
#include <map>
#include <thread>

#include "tucker.cuh"

struct tk_handle {
    int device = 0;
    int num_sms = 148;
    tk::Arena arena;
    std::string err;
    double *pinned = nullptr;   // small host staging area for scalars read back per iteration
    tk::Profiler prof;
    bool prof_on = false;
    std::string prof_text;
    std::vector<char> ckpt;     // Krylov state of a suspended solve (empty: none)
};

namespace tk {

constexpr int SC_BETA2 = 0, SC_BETA = 1, SC_BS2 = 2, SC_BS = 3, SC_NW0SQ = 4, SC_NWSQ = 5,
              SC_NW = 6, SC_RES = 7, SC_H = 8, SC_N = 8 + 64;

static long long prodi(const int *v, int d) {
    long long p = 1;
    for (int i = 0; i < d; ++i) p *= v[i];
    return p;
}

static Dims dims_of(const tk_tucker *t) {
    Dims D{};
    D.d = t->d;
    for (int k = 0; k < t->d; ++k) D.n[k] = (int)t->n[k];
    return D;
}

static void check_tucker(const tk_tucker *t, const char *what) {
    TK_REQUIRE(t != nullptr, std::string(what) + ": null tensor");
    TK_REQUIRE(t->d >= 2 && t->d <= TK_MAX_D, std::string(what) + ": order d must be 2..8");
    TK_REQUIRE(t->core != nullptr, std::string(what) + ": null core");
    for (int k = 0; k < t->d; ++k) {
        TK_REQUIRE(t->n[k] >= 1 && t->n[k] <= (1 << 24), std::string(what) + ": bad mode size");
        TK_REQUIRE(t->r[k] >= 1 && t->r[k] <= 1024, std::string(what) + ": bad rank");
        TK_REQUIRE(t->factor[k] != nullptr, std::string(what) + ": null factor");
    }
}

static TTerm term_of(const tk_tucker *t, double coef = 1.0) {
    TTerm T;
    T.core = t->core;
    for (int k = 0; k < t->d; ++k) { T.f[k] = t->factor[k]; T.r[k] = (int)t->r[k]; }
    T.coef = coef;
    return T;
}

static OpDesc op_of(const tk_operator *op, const Dims &pb) {
    TK_REQUIRE(op != nullptr && op->mats != nullptr && op->theta != nullptr, "operator: null");
    TK_REQUIRE(op->nterms >= 1 && op->nterms <= 64, "operator: nterms must be 1..64");
    TK_REQUIRE(op->d == pb.d, "operator: order differs from the tensor's");
    OpDesc D;
    D.nterms = op->nterms;
    for (int t = 0; t < op->nterms; ++t) {
        D.theta.push_back(op->theta[t]);
        for (int k = 0; k < pb.d; ++k) {
            const tk_modemat &m = op->mats[t * pb.d + k];
            TK_REQUIRE(m.kind == TK_IDENTITY || m.kind == TK_BANDED || m.kind == TK_DENSE, "operator: bad kind");
            TK_REQUIRE(m.n == pb.n[k], "operator: mode matrix size differs from the tensor's");
            if (m.kind != TK_IDENTITY) TK_REQUIRE(m.data != nullptr, "operator: null matrix data");
            if (m.kind == TK_BANDED) TK_REQUIRE(m.kl >= 0 && m.ku >= 0 && m.kl + m.ku < 65536, "operator: bad band");
            D.mats.push_back(m);
        }
    }
    return D;
}

struct SolveOut {
    int iters = 0;
    int status = TK_NOT_CONVERGED;
    double sres = 0.0;
    std::vector<double> hist;
    int ranks[TK_MAX_D] = {};
};

static void readback(Ctx &c, double *host, const double *dev, int n) {
    TK_CUDA(cudaMemcpyAsync(host, dev, n * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    TK_CUDA(cudaStreamSynchronize(c.st));
}

// Tucker tensor stored at rank R in every mode (zero-padded)
struct Slot {
    double *core;
    double *f[TK_MAX_D];
    int *rank;
    TTerm term(const Dims &pb, int R) const {
        TTerm T;
        T.core = core;
        for (int k = 0; k < pb.d; ++k) { T.f[k] = f[k]; T.r[k] = R; }
        return T;
    }
    TOut out(const Dims &pb) const {
        TOut o{};
        o.core = core;
        for (int k = 0; k < pb.d; ++k) o.f[k] = f[k];
        o.rank_dev = rank;
        return o;
    }
};

static Slot alloc_slot(Ctx &c, const Dims &pb, int R) {
    Slot s{};
    int rr[TK_MAX_D];
    for (int k = 0; k < pb.d; ++k) rr[k] = R;
    s.core = c.arena->alloc(prodi(rr, pb.d));
    for (int k = 0; k < pb.d; ++k) s.f[k] = c.arena->alloc((size_t)pb.n[k] * R);
    s.rank = c.arena->alloc_int(TK_MAX_D);
    return s;
}

// RoundSum settings of a solve: fixed sketch size rank_cap + p, or the effective-rank estimate
// (Section 3.1) at the relative threshold round_tol when adaptive_rank is set
static RSConfig rs_cfg(const tk_opts &o, int sr, int R, uint64_t call, int bf16) {
    RSConfig rc{sr, R, o.round_tol, o.seed, call, bf16};
    if (o.adaptive_rank) {
        rc.adaptive_p = o.oversample_p;
        rc.rank_tol = o.round_tol;
    }
    return rc;
}

// ------------------------------------------------------------------------------------------
// Suspended solves: the loop state after iteration k as a byte string (host memory).  A
// suspension copies the device state out; a resume allocates the same buffers and copies it
// back, then the loop continues with the same kernels on the same values.
// ------------------------------------------------------------------------------------------
struct BlobW {
    std::vector<char> &b;
    void host(const void *p, size_t n) {
        const char *q = static_cast<const char *>(p);
        b.insert(b.end(), q, q + n);
    }
    template <class T> void val(const T &v) { host(&v, sizeof(T)); }
    void dev(Ctx &c, const void *d, size_t n) {
        const size_t o = b.size();
        b.resize(o + n);
        if (n) {
            TK_CUDA(cudaMemcpyAsync(b.data() + o, d, n, cudaMemcpyDeviceToHost, c.st));
            TK_CUDA(cudaStreamSynchronize(c.st));
        }
    }
    void devd(Ctx &c, const double *d, long long n) { dev(c, d, (size_t)n * sizeof(double)); }
};

struct BlobR {
    const std::vector<char> &b;
    size_t pos;
    void host(void *p, size_t n) {
        TK_REQUIRE(pos + n <= b.size(), "checkpoint: truncated state");
        std::memcpy(p, b.data() + pos, n);
        pos += n;
    }
    template <class T> T val() {
        T v;
        host(&v, sizeof(T));
        return v;
    }
    void dev(Ctx &c, void *d, size_t n) {
        TK_REQUIRE(pos + n <= b.size(), "checkpoint: truncated state");
        if (n) TK_CUDA(cudaMemcpyAsync(d, b.data() + pos, n, cudaMemcpyHostToDevice, c.st));
        pos += n;
    }
    void devd(Ctx &c, double *d, long long n) { dev(c, d, (size_t)n * sizeof(double)); }
};

// Where a solve takes its state from (resume) and puts it (suspension).
struct Ckpt {
    const std::vector<char> *in = nullptr;
    size_t in_pos = 0;
    std::vector<char> *out = nullptr;
    int stop_after = 0;
};

static void put_slot(BlobW &w, Ctx &c, const Dims &pb, int R, const Slot &sl) {
    int rr[TK_MAX_D];
    for (int k = 0; k < pb.d; ++k) rr[k] = R;
    w.devd(c, sl.core, prodi(rr, pb.d));
    for (int k = 0; k < pb.d; ++k) w.devd(c, sl.f[k], (long long)pb.n[k] * R);
    w.dev(c, sl.rank, sizeof(int) * TK_MAX_D);
}

static Slot get_slot(BlobR &r, Ctx &c, const Dims &pb, int R) {
    Slot sl = alloc_slot(c, pb, R);
    int rr[TK_MAX_D];
    for (int k = 0; k < pb.d; ++k) rr[k] = R;
    r.devd(c, sl.core, prodi(rr, pb.d));
    for (int k = 0; k < pb.d; ++k) r.devd(c, sl.f[k], (long long)pb.n[k] * R);
    r.dev(c, sl.rank, sizeof(int) * TK_MAX_D);
    return sl;
}

static void put_ls(BlobW &w, Ctx &c, const LSState &ls, int rows, int kmax) {
    w.devd(c, ls.H, (long long)rows * kmax);
    w.devd(c, ls.tau, kmax);
    w.devd(c, ls.qtb, rows);
    w.devd(c, ls.y, kmax);
    w.devd(c, ls.T, (long long)kmax * kmax);
}

static void get_ls(BlobR &r, Ctx &c, const LSState &ls, int rows, int kmax) {
    r.devd(c, ls.H, (long long)rows * kmax);
    r.devd(c, ls.tau, kmax);
    r.devd(c, ls.qtb, rows);
    r.devd(c, ls.y, kmax);
    r.devd(c, ls.T, (long long)kmax * kmax);
}

// ------------------------------------------------------------------------------------------
// RHOSVD-Tucker sGMRES (Algorithm 2)
// ------------------------------------------------------------------------------------------
static void solve_rhosvd(Ctx &c, const Dims &pb, const OpDesc &op, const tk_tucker *b,
                         const tk_opts &o, tk_tucker *x, SolveOut &so, double *pinned,
                         const OpDesc *precond, Ckpt &ck, const ExpSumPC *es = nullptr) {
    ScopedMark solve_mark(*c.arena);
    const int d = pb.d, R = o.rank_cap, s = o.sketch_s, sr = o.rank_cap + o.oversample_p;
    const int kmax = std::min(o.maxit, s - 1);
    TK_REQUIRE(sr <= 96, "RoundSum sketch size rank_cap + p must be <= 96");
    TK_REQUIRE(o.ktrunc >= 1 && o.ktrunc <= 64, "ktrunc must be 1..64");
    const int bf16 = o.precision == TK_MIXED ? 1 : 0;
    double *sc = c.arena->alloc(SC_N);
    fill(c, sc, SC_N, 0.0);
    // Krylov sketch S_k (n_k x s): stream (seed, purpose 1, call 0, mode k)
    double *S[TK_MAX_D];
    {
        uint64_t sids[TK_MAX_D];
        long long cnt[TK_MAX_D];
        for (int k = 0; k < d; ++k) {
            S[k] = c.arena->alloc((size_t)pb.n[k] * s);
            sids[k] = (uint64_t(1) << 48) | uint64_t(k);
            cnt[k] = (long long)pb.n[k] * s;
        }
        gaussian(c, o.seed, sids, cnt, S, d, 0);
    }
    const TTerm B = term_of(b);
    std::vector<TTerm> V;
    double *bs = c.arena->alloc(s);
    double *M = c.arena->alloc((size_t)s * kmax);
    LSState ls{};
    ls.H = c.arena->alloc((size_t)s * kmax);
    ls.tau = c.arena->alloc(kmax);
    ls.qtb = c.arena->alloc(s);
    ls.y = c.arena->alloc(kmax);
    ls.T = c.arena->alloc((size_t)kmax * kmax);
    ls.ldt = kmax;
    ls.res = sc + SC_RES;
    // V_1 = B / beta  (own core copy, factors borrowed from B)
    TTerm v1 = B;
    double *v1core = c.arena->alloc(prodi(B.r, d));
    v1.core = v1core;
    V.push_back(v1);
    std::vector<int *> vrank{nullptr}, zrank;   // rank arrays of the slots behind V and Z
    int k0 = 0;
    uint64_t call = 0;
    std::vector<TTerm> Z;   // flexible preconditioning (Section 3.4): Z_k = RoundSum(M(V_k))
    double beta_s;
    if (ck.in) {
        BlobR r{*ck.in, ck.in_pos};
        k0 = r.val<int>();
        call = r.val<uint64_t>();
        so.hist.resize(k0);
        r.host(so.hist.data(), sizeof(double) * k0);
        r.devd(c, sc, SC_N);
        r.devd(c, v1core, prodi(B.r, d));
        r.devd(c, bs, s);
        r.devd(c, M, (long long)s * kmax);
        get_ls(r, c, ls, s, kmax);
        for (int j = 2; j <= k0 + 1; ++j) {
            const Slot sl = get_slot(r, c, pb, R);
            V.push_back(sl.term(pb, R));
            vrank.push_back(sl.rank);
        }
        if (precond)
            for (int j = 1; j <= k0; ++j) {
                const Slot sl = get_slot(r, c, pb, R);
                Z.push_back(sl.term(pb, R));
                zrank.push_back(sl.rank);
            }
        TK_REQUIRE(r.pos == ck.in->size(), "checkpoint: state does not match this solve");
        readback(c, pinned, sc, 4);
        beta_s = pinned[SC_BS];
    } else {
        inner_batch(c, pb, {InnerJob{B, B, sc + SC_BETA2}});
        sqrt_scalar(c, sc + SC_BETA2, sc + SC_BETA);
        scale_by(c, v1core, b->core, prodi(B.r, d), sc + SC_BETA, 1);
        kron_sketch_batch(c, pb, {B}, S, s, &bs);
        dot(c, bs, bs, s, sc + SC_BS2);
        sqrt_scalar(c, sc + SC_BS2, sc + SC_BS);
        readback(c, pinned, sc, 4);
        beta_s = pinned[SC_BS];
        TK_REQUIRE(std::isfinite(pinned[SC_BETA]) && pinned[SC_BETA] > 0.0, "right-hand side is zero or not finite");
        TK_REQUIRE(std::isfinite(beta_s) && beta_s > 0.0, "sketch of the right-hand side is zero or not finite");
    }
    auto suspend = [&](int k) {
        BlobW w{*ck.out};
        w.val(k);
        w.val(call);
        w.host(so.hist.data(), sizeof(double) * k);
        w.devd(c, sc, SC_N);
        w.devd(c, v1core, prodi(B.r, d));
        w.devd(c, bs, s);
        w.devd(c, M, (long long)s * kmax);
        put_ls(w, c, ls, s, kmax);
        for (int j = 2; j <= k + 1; ++j) {
            Slot sl{};
            sl.core = const_cast<double *>(V[j - 1].core);
            for (int kk = 0; kk < d; ++kk) sl.f[kk] = const_cast<double *>(V[j - 1].f[kk]);
            sl.rank = vrank[j - 1];
            put_slot(w, c, pb, R, sl);
        }
        if (precond)
            for (int j = 1; j <= k; ++j) {
                Slot sl{};
                sl.core = const_cast<double *>(Z[j - 1].core);
                for (int kk = 0; kk < d; ++kk) sl.f[kk] = const_cast<double *>(Z[j - 1].f[kk]);
                sl.rank = zrank[j - 1];
                put_slot(w, c, pb, R, sl);
            }
    };

    so.status = kmax < o.maxit ? TK_SKETCH_EXHAUSTED : TK_NOT_CONVERGED;
    int k = 0;
    for (k = k0 + 1; k <= kmax; ++k) {
        Slot vn = alloc_slot(c, pb, R);
        if (precond) {
            Slot zs = alloc_slot(c, pb, R);
            ScopedMark it(*c.arena);
            if (es) {
                // Section 3.4: the terms of M(V_k) in the sine eigenbasis, RoundSum with the sketches
                // rotated into that basis and the factors rotated back (the DST-I application)
                std::vector<TTerm> mterms = expsum_terms(c, pb, *es, V.back(), bf16 != 0);
                RSConfig rc = rs_cfg(o, sr, R, call++, bf16);
                rc.rot = es->V;
                rc.tc_all = bf16;      // mixed form: the whole preconditioner application
                roundsum(c, pb, mterms, rc, zs.out(pb));
            } else {
                std::vector<TTerm> mterms = apply_operator(c, pb, *precond, V.back(), o.transpose, bf16 != 0);
                RSConfig rc = rs_cfg(o, sr, R, call++, bf16);
                rc.tc_all = bf16;
                roundsum(c, pb, mterms, rc, zs.out(pb));
            }
            Z.push_back(zs.term(pb, R));
            zrank.push_back(zs.rank);
        }
        {
            ScopedMark it(*c.arena);
            std::vector<TTerm> terms = apply_operator(c, pb, op, precond ? Z.back() : V.back(), o.transpose);
            Slot wmv = alloc_slot(c, pb, R);
            roundsum(c, pb, terms, rs_cfg(o, sr, R, call++, bf16), wmv.out(pb));
            const TTerm W = wmv.term(pb, R);
            dot(c, W.core, W.core, prodi(W.r, d), sc + SC_NW0SQ);
            double *mcol = M + (size_t)(k - 1) * s;
            kron_sketch_batch(c, pb, {W}, S, s, &mcol);
            const int j0 = std::max(1, k - o.ktrunc + 1);
            std::vector<InnerJob> ij;
            for (int j = j0; j <= k; ++j) ij.push_back(InnerJob{V[j - 1], W, sc + SC_H + (j - j0)});
            inner_batch(c, pb, ij);
            std::vector<TTerm> orth{W};
            for (int j = j0; j <= k; ++j) {
                TTerm t = V[j - 1];
                t.coef = -1.0;
                t.coef_dev = sc + SC_H + (j - j0);
                orth.push_back(t);
            }
            roundsum(c, pb, orth, rs_cfg(o, sr, R, call++, bf16), vn.out(pb));
            const long long csz = prodi(W.r, d);
            dot(c, vn.core, vn.core, csz, sc + SC_NWSQ);
            sqrt_scalar(c, sc + SC_NWSQ, sc + SC_NW);
            ls_update(c, M, bs, s, k - 1, k, ls, k == 1);
            if (o.gcv_tikhonov) tikhonov_gcv(c, ls, s, k, o.gcv_rows ? s : k + 1, nullptr);
            scale_by(c, vn.core, vn.core, csz, sc + SC_NW, 1);
            readback(c, pinned, sc, 8);
        }
        const double res = pinned[SC_RES] / beta_s;
        TK_REQUIRE(std::isfinite(res), "sketched residual is not finite (non-finite input or overflow)");
        so.hist.push_back(res);
        so.sres = res;
        if (std::sqrt(std::max(pinned[SC_NWSQ], 0.0)) <= 1e-14 * std::sqrt(std::max(pinned[SC_NW0SQ], 0.0))) {
            so.status = TK_BREAKDOWN;
            break;
        }
        V.push_back(vn.term(pb, R));
        vrank.push_back(vn.rank);
        if (res < o.eta * o.tol) {
            so.status = TK_OK;
            break;
        }
        if (ck.stop_after > 0 && k - k0 >= ck.stop_after && k < kmax) {
            suspend(k);
            so.status = TK_SUSPENDED;
            so.iters = k;
            return;
        }
    }
    if (k > kmax) k = kmax;
    so.iters = k;
    if (!so.hist.empty()) so.sres = so.hist.back();
    // X~ = RoundSum(sum_i y_i V_i)  (flexible form: sum_i y_i Z_i)
    std::vector<TTerm> fin;
    for (int i = 0; i < k; ++i) {
        TTerm t = precond ? Z[i] : V[i];
        t.coef = 1.0;
        t.coef_dev = ls.y + i;
        fin.push_back(t);
    }
    TOut xo{};
    xo.core = x->core;
    for (int kk = 0; kk < d; ++kk) xo.f[kk] = x->factor[kk];
    int *rk = c.arena->alloc_int(TK_MAX_D);
    xo.rank_dev = rk;
    roundsum(c, pb, fin, rs_cfg(o, sr, R, call++, bf16), xo);
    int hr[TK_MAX_D];
    TK_CUDA(cudaMemcpyAsync(hr, rk, sizeof(int) * d, cudaMemcpyDeviceToHost, c.st));
    TK_CUDA(cudaStreamSynchronize(c.st));
    for (int kk = 0; kk < d; ++kk) so.ranks[kk] = hr[kk];
}

// ------------------------------------------------------------------------------------------
// RHOSVD-Tucker GMRES (Algorithm 1): full Arnoldi, every sum through RoundSum, least squares on
// the Hessenberg matrix (the incremental Householder kernel with M = H, b = beta e_1)
// ------------------------------------------------------------------------------------------
static void solve_gmres(Ctx &c, const Dims &pb, const OpDesc &op, const tk_tucker *b, const tk_opts &o,
                        tk_tucker *x, SolveOut &so, double *pinned, Ckpt &ck) {
    ScopedMark solve_mark(*c.arena);
    const int d = pb.d, R = o.rank_cap, sr = o.rank_cap + o.oversample_p;
    const int kmax = o.maxit, ld = kmax + 1;
    TK_REQUIRE(sr <= 96, "RoundSum sketch size rank_cap + p must be <= 96");
    TK_REQUIRE(kmax <= 4095, "maxit must be <= 4095");
    const int bf16 = o.precision == TK_MIXED ? 1 : 0;
    double *sc = c.arena->alloc(SC_N);
    fill(c, sc, SC_N, 0.0);
    const TTerm B = term_of(b);
    std::vector<TTerm> V;
    std::vector<int *> vrank{nullptr};
    TTerm v1 = B;
    double *v1core = c.arena->alloc(prodi(B.r, d));
    v1.core = v1core;
    V.push_back(v1);
    // Hessenberg matrix H ((kmax + 1) x kmax, column-major) and beta e_1
    double *H = c.arena->alloc((size_t)ld * kmax);
    double *e1 = c.arena->alloc(ld);
    LSState ls{};
    ls.H = c.arena->alloc((size_t)ld * kmax);
    ls.tau = c.arena->alloc(kmax);
    ls.qtb = c.arena->alloc(ld);
    ls.y = c.arena->alloc(kmax);
    ls.T = c.arena->alloc((size_t)kmax * kmax);
    ls.ldt = kmax;
    ls.res = sc + SC_RES;
    int k0 = 0;
    uint64_t call = 0;
    double beta;
    if (ck.in) {
        BlobR r{*ck.in, ck.in_pos};
        k0 = r.val<int>();
        call = r.val<uint64_t>();
        so.hist.resize(k0);
        r.host(so.hist.data(), sizeof(double) * k0);
        r.devd(c, sc, SC_N);
        r.devd(c, v1core, prodi(B.r, d));
        r.devd(c, H, (long long)ld * kmax);
        r.devd(c, e1, ld);
        get_ls(r, c, ls, ld, kmax);
        for (int j = 2; j <= k0 + 1; ++j) {
            const Slot sl = get_slot(r, c, pb, R);
            V.push_back(sl.term(pb, R));
            vrank.push_back(sl.rank);
        }
        TK_REQUIRE(r.pos == ck.in->size(), "checkpoint: state does not match this solve");
        readback(c, pinned, sc, 4);
        beta = pinned[SC_BETA];
    } else {
        inner_batch(c, pb, {InnerJob{B, B, sc + SC_BETA2}});
        sqrt_scalar(c, sc + SC_BETA2, sc + SC_BETA);
        scale_by(c, v1core, b->core, prodi(B.r, d), sc + SC_BETA, 1);
        fill(c, H, (long long)ld * kmax, 0.0);
        fill(c, e1, ld, 0.0);
        copy(c, e1, sc + SC_BETA, 1);
        readback(c, pinned, sc, 4);
        beta = pinned[SC_BETA];
        TK_REQUIRE(std::isfinite(beta) && beta > 0.0, "right-hand side is zero or not finite");
    }
    auto suspend = [&](int k) {
        BlobW w{*ck.out};
        w.val(k);
        w.val(call);
        w.host(so.hist.data(), sizeof(double) * k);
        w.devd(c, sc, SC_N);
        w.devd(c, v1core, prodi(B.r, d));
        w.devd(c, H, (long long)ld * kmax);
        w.devd(c, e1, ld);
        put_ls(w, c, ls, ld, kmax);
        for (int j = 2; j <= k + 1; ++j) {
            Slot sl{};
            sl.core = const_cast<double *>(V[j - 1].core);
            for (int kk = 0; kk < d; ++kk) sl.f[kk] = const_cast<double *>(V[j - 1].f[kk]);
            sl.rank = vrank[j - 1];
            put_slot(w, c, pb, R, sl);
        }
    };

    so.status = TK_NOT_CONVERGED;
    int k = 0;
    for (k = k0 + 1; k <= kmax; ++k) {
        Slot vn = alloc_slot(c, pb, R);
        {
            ScopedMark it(*c.arena);
            std::vector<TTerm> terms = apply_operator(c, pb, op, V.back(), o.transpose);
            Slot wmv = alloc_slot(c, pb, R);
            roundsum(c, pb, terms, rs_cfg(o, sr, R, call++, bf16), wmv.out(pb));
            const TTerm W = wmv.term(pb, R);
            dot(c, W.core, W.core, prodi(W.r, d), sc + SC_NW0SQ);
            double *hcol = H + (size_t)(k - 1) * ld;
            std::vector<InnerJob> ij;
            for (int j = 1; j <= k; ++j) ij.push_back(InnerJob{V[j - 1], W, hcol + (j - 1)});
            inner_batch(c, pb, ij);
            std::vector<TTerm> orth{W};
            for (int j = 1; j <= k; ++j) {
                TTerm t = V[j - 1];
                t.coef = -1.0;
                t.coef_dev = hcol + (j - 1);
                orth.push_back(t);
            }
            roundsum(c, pb, orth, rs_cfg(o, sr, R, call++, bf16), vn.out(pb));
            const long long csz = prodi(W.r, d);
            dot(c, vn.core, vn.core, csz, sc + SC_NWSQ);
            sqrt_scalar(c, sc + SC_NWSQ, sc + SC_NW);
            copy(c, hcol + k, sc + SC_NW, 1);                      // h_{k+1,k} = ||W||
            ls_update(c, H, e1, ld, k - 1, k, ls, k == 1);
            if (o.gcv_tikhonov) tikhonov_gcv(c, ls, ld, k, k + 1, nullptr);
            scale_by(c, vn.core, vn.core, csz, sc + SC_NW, 1);
            readback(c, pinned, sc, 8);
        }
        const double res = pinned[SC_RES] / beta;
        TK_REQUIRE(std::isfinite(res), "residual is not finite (non-finite input or overflow)");
        so.hist.push_back(res);
        so.sres = res;
        if (std::sqrt(std::max(pinned[SC_NWSQ], 0.0)) <= 1e-14 * std::sqrt(std::max(pinned[SC_NW0SQ], 0.0))) {
            so.status = TK_BREAKDOWN;
            break;
        }
        V.push_back(vn.term(pb, R));
        vrank.push_back(vn.rank);
        if (res < o.tol) {
            so.status = TK_OK;
            break;
        }
        if (ck.stop_after > 0 && k - k0 >= ck.stop_after && k < kmax) {
            suspend(k);
            so.status = TK_SUSPENDED;
            so.iters = k;
            return;
        }
    }
    if (k > kmax) k = kmax;
    so.iters = k;
    if (!so.hist.empty()) so.sres = so.hist.back();
    std::vector<TTerm> fin;
    for (int i = 0; i < k; ++i) {
        TTerm t = V[i];
        t.coef = 1.0;
        t.coef_dev = ls.y + i;
        fin.push_back(t);
    }
    TOut xo{};
    xo.core = x->core;
    for (int kk = 0; kk < d; ++kk) xo.f[kk] = x->factor[kk];
    int *rk = c.arena->alloc_int(TK_MAX_D);
    xo.rank_dev = rk;
    roundsum(c, pb, fin, rs_cfg(o, sr, R, call++, bf16), xo);
    int hr[TK_MAX_D];
    TK_CUDA(cudaMemcpyAsync(hr, rk, sizeof(int) * d, cudaMemcpyDeviceToHost, c.st));
    TK_CUDA(cudaStreamSynchronize(c.st));
    for (int kk = 0; kk < d; ++kk) so.ranks[kk] = hr[kk];
}

// ------------------------------------------------------------------------------------------
// MLN-Tucker sGMRES (Algorithm 6, without the memory-saving truncation)
// ------------------------------------------------------------------------------------------
struct Sk {
    double *g;
    double *F[TK_MAX_D];
};

static Sk alloc_sk(Ctx &c, const Dims &pb, int r, int rp) {
    Sk s{};
    long long gs = 1;
    for (int k = 0; k < pb.d; ++k) gs *= rp;
    s.g = c.arena->alloc(gs);
    for (int k = 0; k < pb.d; ++k) s.F[k] = c.arena->alloc((size_t)pb.n[k] * r);
    return s;
}

void axpy_list(Ctx &c, double *y, long long n, double beta, const std::vector<const double *> &xs,
               const std::vector<double> &coef, const std::vector<const double *> &coef_dev);

static void solve_mln(Ctx &c, const Dims &pb, const OpDesc &op, const tk_tucker *b, const tk_opts &o,
                      tk_tucker *x, SolveOut &so, double *pinned, Ckpt &ck) {
    ScopedMark solve_mark(*c.arena);
    const int d = pb.d, r = o.rank_cap, p = o.oversample_p, rp = r + p;
    const int kmax = std::min(o.maxit, rp - 1);
    TK_REQUIRE(r >= 1 && p >= 0 && r <= 96, "MLN: rank must be 1..96");
    TK_REQUIRE(o.ktrunc >= 1 && o.ktrunc <= 64, "ktrunc must be 1..64");
    // mixed form: the sketch of L(V_i) (MLN_Sketch of the operator terms, the dominant TTM
    // chains) on tensor cores (gemm_oz); the recoveries, the sketches of the basis tensors,
    // inner products, sketch sums and least squares stay FP64
    const bool tc = o.precision == TK_MIXED;
    long long gsz = 1, csz = 1;
    for (int k = 0; k < d; ++k) { gsz *= rp; csz *= r; }
    double *sc = c.arena->alloc(SC_N);
    fill(c, sc, SC_N, 0.0);
    double *psi[TK_MAX_D];
    {
        uint64_t sids[TK_MAX_D];
        long long cnt[TK_MAX_D];
        for (int k = 0; k < d; ++k) {
            psi[k] = c.arena->alloc((size_t)pb.n[k] * rp);
            sids[k] = (uint64_t(1) << 48) | uint64_t(k);
            cnt[k] = (long long)pb.n[k] * rp;
        }
        gaussian(c, o.seed, sids, cnt, psi, d, 0);
    }
    const TTerm B = term_of(b);
    std::vector<TTerm> V;
    std::vector<int *> vrank{nullptr};
    TTerm v1 = B;
    double *v1core = c.arena->alloc(prodi(B.r, d));
    v1.core = v1core;
    V.push_back(v1);
    // Stored sketches.  Default: every sketch kept at full size.  Memory-efficient variant
    // (Section 3.3): full-size sketches live in a ring of ktrunc + 1 slots; the sketch of V_m is
    // cut to (r_sol + p_sol)^d and n x r_sol just before its slot is reused (it has left the
    // window by then), into a compact store.
    const bool save = o.mln_r_sol > 0;
    const int rs = o.mln_r_sol, rts = o.mln_r_sol + o.mln_p_sol, K = o.ktrunc;
    if (save) TK_REQUIRE(rs <= r && o.mln_p_sol >= 0 && rts <= rp, "MLN: need r_sol <= r and r_sol + p_sol <= r + p");
    long long gcut = 1;
    for (int k = 0; k < d; ++k) gcut *= rts;
    std::vector<Sk> sks;                 // index m: sketch of V_{m+1} (full size, or its ring slot)
    std::vector<Sk> ring;
    std::vector<Sk> cut;                 // compact sketches (save), index m
    std::vector<char> is_cut;
    auto alloc_cut = [&](int m) -> Sk & {
        Sk t{};
        t.g = c.arena->alloc(gcut);
        for (int k = 0; k < d; ++k) t.F[k] = c.arena->alloc((size_t)pb.n[k] * rs);
        if ((int)cut.size() <= m) { cut.resize(m + 1); is_cut.resize(m + 1, 0); }
        cut[m] = t;
        is_cut[m] = 1;
        return cut[m];
    };
    auto cut_sketch = [&](int m) {
        Sk &t = alloc_cut(m);
        int rd[TK_MAX_D], rsrc[TK_MAX_D];
        for (int k = 0; k < d; ++k) { rd[k] = rts; rsrc[k] = rp; }
        copy_core_pad(c, t.g, rd, sks[m].g, rsrc, d);
        for (int k = 0; k < d; ++k) copy(c, t.F[k], sks[m].F[k], (long long)pb.n[k] * rs);
    };
    if (save)
        for (int q = 0; q <= K; ++q) ring.push_back(alloc_sk(c, pb, r, rp));
    double *bs = c.arena->alloc(rp);
    double *M = c.arena->alloc((size_t)rp * kmax);
    LSState ls{};
    ls.H = c.arena->alloc((size_t)rp * kmax);
    ls.tau = c.arena->alloc(kmax);
    ls.qtb = c.arena->alloc(rp);
    ls.y = c.arena->alloc(kmax);
    ls.T = c.arena->alloc((size_t)kmax * kmax);
    ls.ldt = kmax;
    ls.res = sc + SC_RES;
    int i0 = 0;
    double beta_s;
    auto full_sk = [&](int m) { return save ? ring[m % (K + 1)] : alloc_sk(c, pb, r, rp); };
    if (ck.in) {
        BlobR rd{*ck.in, ck.in_pos};
        i0 = rd.val<int>();
        so.hist.resize(i0);
        rd.host(so.hist.data(), sizeof(double) * i0);
        rd.devd(c, sc, SC_N);
        rd.devd(c, bs, rp);
        rd.devd(c, M, (long long)rp * kmax);
        get_ls(rd, c, ls, rp, kmax);
        // the window of iteration i0 + 1: V_{j0} .. V_{i0+1}
        const int j0 = std::max(1, i0 + 1 - o.ktrunc + 1);
        if (j0 == 1) rd.devd(c, v1core, prodi(B.r, d));
        for (int j = 2; j <= i0 + 1; ++j) {
            if (j < j0) {               // outside every later window: never read again
                V.push_back(TTerm{});
                vrank.push_back(nullptr);
                continue;
            }
            const Slot sl = get_slot(rd, c, pb, r);
            V.push_back(sl.term(pb, r));
            vrank.push_back(sl.rank);
        }
        for (int m = 0; m <= i0; ++m) {
            const char isc = rd.val<char>();
            if (isc) {
                Sk &t = alloc_cut(m);
                rd.devd(c, t.g, gcut);
                for (int k = 0; k < d; ++k) rd.devd(c, t.F[k], (long long)pb.n[k] * rs);
                sks.push_back(Sk{});     // its ring slot has been reused
            } else {
                Sk t = full_sk(m);
                rd.devd(c, t.g, gsz);
                for (int k = 0; k < d; ++k) rd.devd(c, t.F[k], (long long)pb.n[k] * r);
                sks.push_back(t);
            }
        }
        TK_REQUIRE(rd.pos == ck.in->size(), "checkpoint: state does not match this solve");
        readback(c, pinned, sc, 4);
        beta_s = pinned[SC_BS];
    } else {
        inner_batch(c, pb, {InnerJob{B, B, sc + SC_BETA2}});
        sqrt_scalar(c, sc + SC_BETA2, sc + SC_BETA);
        scale_by(c, v1core, b->core, prodi(B.r, d), sc + SC_BETA, 1);
        sks.push_back(full_sk(0));
        mln_sketch_sum(c, pb, {V[0]}, psi, r, p, sks[0].g, sks[0].F, 0.0);
        superdiag(c, sks[0].g, rp, d, bs, 1.0, sc + SC_BETA);
        dot(c, bs, bs, rp, sc + SC_BS2);
        sqrt_scalar(c, sc + SC_BS2, sc + SC_BS);
        readback(c, pinned, sc, 4);
        beta_s = pinned[SC_BS];
        TK_REQUIRE(std::isfinite(pinned[SC_BETA]) && pinned[SC_BETA] > 0.0, "right-hand side is zero or not finite");
        TK_REQUIRE(std::isfinite(beta_s) && beta_s > 0.0, "sketch of the right-hand side is zero or not finite");
    }
    auto suspend = [&](int i) {
        BlobW w{*ck.out};
        w.val(i);
        w.host(so.hist.data(), sizeof(double) * i);
        w.devd(c, sc, SC_N);
        w.devd(c, bs, rp);
        w.devd(c, M, (long long)rp * kmax);
        put_ls(w, c, ls, rp, kmax);
        const int j0 = std::max(1, i + 1 - o.ktrunc + 1);
        if (j0 == 1) w.devd(c, v1core, prodi(B.r, d));
        for (int j = std::max(2, j0); j <= i + 1; ++j) {
            Slot sl{};
            sl.core = const_cast<double *>(V[j - 1].core);
            for (int k = 0; k < d; ++k) sl.f[k] = const_cast<double *>(V[j - 1].f[k]);
            sl.rank = vrank[j - 1];
            put_slot(w, c, pb, r, sl);
        }
        for (int m = 0; m <= i; ++m) {
            const char isc = (m < (int)is_cut.size() && is_cut[m]) ? 1 : 0;
            w.val(isc);
            if (isc) {
                w.devd(c, cut[m].g, gcut);
                for (int k = 0; k < d; ++k) w.devd(c, cut[m].F[k], (long long)pb.n[k] * rs);
            } else {
                w.devd(c, sks[m].g, gsz);
                for (int k = 0; k < d; ++k) w.devd(c, sks[m].F[k], (long long)pb.n[k] * r);
            }
        }
    };

    so.status = kmax < o.maxit ? TK_SKETCH_EXHAUSTED : TK_NOT_CONVERGED;
    int i = 0;
    for (i = i0 + 1; i <= kmax; ++i) {
        Slot vn = alloc_slot(c, pb, r);
        Sk skn;
        if (save) {
            // the slot for the sketch of V_{i+1} holds that of V_{i-K}, outside every later window
            if (i - K - 1 >= 0) cut_sketch(i - K - 1);
            skn = ring[i % (K + 1)];
        } else {
            skn = alloc_sk(c, pb, r, rp);
        }
        {
            ScopedMark it(*c.arena);
            std::vector<TTerm> terms = apply_operator(c, pb, op, V.back(), o.transpose);
            Sk gw = alloc_sk(c, pb, r, rp);
            mln_sketch_sum(c, pb, terms, psi, r, p, gw.g, gw.F, 0.0, tc);
            superdiag(c, gw.g, rp, d, M + (size_t)(i - 1) * rp, 1.0, nullptr);
            Slot w = alloc_slot(c, pb, r);
            mln_recovery(c, pb, gw.g, gw.F, psi, r, p, w.out(pb));
            const TTerm W = w.term(pb, r);
            inner_batch(c, pb, {InnerJob{W, W, sc + SC_NW0SQ}});
            const int j0 = std::max(1, i - o.ktrunc + 1);
            std::vector<InnerJob> ij;
            for (int j = j0; j <= i; ++j) ij.push_back(InnerJob{V[j - 1], W, sc + SC_H + (j - j0)});
            inner_batch(c, pb, ij);
            // MLN_Sum(gw, sketches of the window, {1, -h_j})
            std::vector<const double *> xs, cd;
            std::vector<double> cf;
            for (int j = j0; j <= i; ++j) { xs.push_back(sks[j - 1].g); cf.push_back(-1.0); cd.push_back(sc + SC_H + (j - j0)); }
            axpy_list(c, gw.g, gsz, 1.0, xs, cf, cd);
            for (int k = 0; k < d; ++k) {
                std::vector<const double *> fx;
                for (int j = j0; j <= i; ++j) fx.push_back(sks[j - 1].F[k]);
                axpy_list(c, gw.F[k], (long long)pb.n[k] * r, 1.0, fx, cf, cd);
            }
            mln_recovery(c, pb, gw.g, gw.F, psi, r, p, vn.out(pb));
            const TTerm Wn = vn.term(pb, r);
            inner_batch(c, pb, {InnerJob{Wn, Wn, sc + SC_NWSQ}});
            sqrt_scalar(c, sc + SC_NWSQ, sc + SC_NW);
            ls_update(c, M, bs, rp, i - 1, i, ls, i == 1);
            if (o.gcv_tikhonov) tikhonov_gcv(c, ls, rp, i, o.gcv_rows ? rp : i + 1, nullptr);
            scale_by(c, vn.core, vn.core, csz, sc + SC_NW, 1);
            mln_sketch_sum(c, pb, {Wn}, psi, r, p, skn.g, skn.F, 0.0);
            readback(c, pinned, sc, 8);
        }
        const double res = pinned[SC_RES] / beta_s;
        TK_REQUIRE(std::isfinite(res), "sketched residual is not finite (non-finite input or overflow)");
        so.hist.push_back(res);
        so.sres = res;
        if (std::sqrt(std::max(pinned[SC_NWSQ], 0.0)) <= 1e-14 * std::sqrt(std::max(pinned[SC_NW0SQ], 0.0))) {
            so.status = TK_BREAKDOWN;
            break;
        }
        V.push_back(vn.term(pb, r));
        vrank.push_back(vn.rank);
        sks.push_back(skn);
        if (res < o.eta * o.tol) {
            so.status = TK_OK;
            break;
        }
        if (ck.stop_after > 0 && i - i0 >= ck.stop_after && i < kmax) {
            suspend(i);
            so.status = TK_SUSPENDED;
            so.iters = i;
            return;
        }
    }
    if (i > kmax) i = kmax;
    so.iters = i;
    if (!so.hist.empty()) so.sres = so.hist.back();
    if (save) {
        // X~ = MLN_Recovery(MLN_Sum(cut sketches 1..i, y)) at rank r_sol with the leading
        // r_sol + p_sol columns of each Psi_k, zero-padded into x_out
        for (int m = 0; m < i; ++m)
            if ((int)is_cut.size() <= m || !is_cut[m]) cut_sketch(m);
        Sk sol{};
        sol.g = c.arena->alloc(gcut);
        for (int k = 0; k < d; ++k) sol.F[k] = c.arena->alloc((size_t)pb.n[k] * rs);
        std::vector<const double *> xs, cd;
        std::vector<double> cf;
        for (int m = 0; m < i; ++m) { xs.push_back(cut[m].g); cf.push_back(1.0); cd.push_back(ls.y + m); }
        axpy_list(c, sol.g, gcut, 0.0, xs, cf, cd);
        for (int k = 0; k < d; ++k) {
            std::vector<const double *> fx;
            for (int m = 0; m < i; ++m) fx.push_back(cut[m].F[k]);
            axpy_list(c, sol.F[k], (long long)pb.n[k] * rs, 0.0, fx, cf, cd);
        }
        TOut tmp{};
        long long cs = 1;
        for (int k = 0; k < d; ++k) cs *= rs;
        tmp.core = c.arena->alloc(cs);
        for (int k = 0; k < d; ++k) tmp.f[k] = c.arena->alloc((size_t)pb.n[k] * rs);
        tmp.rank_dev = nullptr;
        mln_recovery(c, pb, sol.g, sol.F, psi, rs, o.mln_p_sol, tmp);
        int rd[TK_MAX_D], rsrc[TK_MAX_D];
        for (int k = 0; k < d; ++k) { rd[k] = r; rsrc[k] = rs; }
        copy_core_pad(c, x->core, rd, tmp.core, rsrc, d);
        for (int k = 0; k < d; ++k)
            copy_pad(c, x->factor[k], pb.n[k], pb.n[k], r, tmp.f[k], pb.n[k], pb.n[k], rs);
        TK_CUDA(cudaStreamSynchronize(c.st));
        for (int k = 0; k < d; ++k) so.ranks[k] = rs;
        return;
    }
    // X~ = MLN_Recovery(MLN_Sum(sketches 1..i, y))
    Sk sol = alloc_sk(c, pb, r, rp);
    {
        std::vector<const double *> xs, cd;
        std::vector<double> cf;
        for (int m = 0; m < i; ++m) { xs.push_back(sks[m].g); cf.push_back(1.0); cd.push_back(ls.y + m); }
        axpy_list(c, sol.g, gsz, 0.0, xs, cf, cd);
        for (int k = 0; k < d; ++k) {
            std::vector<const double *> fx;
            for (int m = 0; m < i; ++m) fx.push_back(sks[m].F[k]);
            axpy_list(c, sol.F[k], (long long)pb.n[k] * r, 0.0, fx, cf, cd);
        }
    }
    TOut xo{};
    xo.core = x->core;
    for (int k = 0; k < d; ++k) xo.f[k] = x->factor[k];
    xo.rank_dev = nullptr;
    mln_recovery(c, pb, sol.g, sol.F, psi, r, p, xo);
    TK_CUDA(cudaStreamSynchronize(c.st));
    for (int k = 0; k < d; ++k) so.ranks[k] = r;
}

// ------------------------------------------------------------------------------------------
// ||sum_i c_i X_i|| in Tucker form: QR of the concatenated distinct factors per mode, then the
// norm of the small dense core sum_i c_i G_i x_k R_k[:, block_i] (no cancellation between terms)
// ------------------------------------------------------------------------------------------
static double sum_norm(Ctx &c, const Dims &pb, const std::vector<TTerm> &terms) {
    ScopedMark mark(*c.arena);
    const int d = pb.d;
    double *Rk[TK_MAX_D];
    int rows[TK_MAX_D];
    std::vector<std::vector<int>> off(terms.size(), std::vector<int>(d));
    std::vector<QRJob> qj;
    for (int k = 0; k < d; ++k) {
        std::map<const double *, int> seen;
        int width = 0;
        for (size_t i = 0; i < terms.size(); ++i) {
            auto it = seen.find(terms[i].f[k]);
            if (it != seen.end()) { off[i][k] = it->second; continue; }
            seen[terms[i].f[k]] = width;
            off[i][k] = width;
            width += terms[i].r[k];
        }
        TK_REQUIRE(width <= 256, "sum norm: concatenated rank above 256");
        double *U = c.arena->alloc((size_t)pb.n[k] * width);
        for (auto &kv : seen) {
            int rr = 0;
            for (size_t i = 0; i < terms.size(); ++i)
                if (terms[i].f[k] == kv.first) rr = terms[i].r[k];
            copy(c, U + (size_t)kv.second * pb.n[k], kv.first, (long long)pb.n[k] * rr);
        }
        qj.push_back(QRJob{U, c.arena->alloc(width), nullptr, pb.n[k], width, nullptr});
        rows[k] = std::min(pb.n[k], width);
        Rk[k] = c.arena->alloc((size_t)rows[k] * width);
    }
    qr_householder(c, qj);
    for (int k = 0; k < d; ++k) triu_copy(c, Rk[k], rows[k], qj[k].A, pb.n[k], rows[k], qj[k].s);
    TtmGroup G{};
    long long cs = 1;
    for (int k = 0; k < d; ++k) { G.sdims[k] = rows[k]; cs *= rows[k]; }
    double *core = c.arena->alloc(cs);
    G.out = core;
    G.beta = 0.0;
    for (size_t i = 0; i < terms.size(); ++i) {
        TtmJob J{};
        J.core = terms[i].core;
        for (int k = 0; k < d; ++k) {
            J.r[k] = terms[i].r[k];
            J.P[k] = Rk[k] + (size_t)off[i][k] * rows[k];
            J.ldp[k] = rows[k];
        }
        J.coef = terms[i].coef;
        J.coef_dev = terms[i].coef_dev;
        G.jobs.push_back(J);
    }
    ttm_groups(c, d, {G});
    double *sc = c.arena->alloc(1);
    dot(c, core, core, cs, sc);
    double h;
    TK_CUDA(cudaMemcpyAsync(&h, sc, sizeof(double), cudaMemcpyDeviceToHost, c.st));
    TK_CUDA(cudaStreamSynchronize(c.st));
    return std::sqrt(std::max(h, 0.0));
}

// True relative residual ||L(X) - B|| / ||B|| (output contract of Algorithms 2 and 6)
static double true_residual(Ctx &c, const Dims &pb, const OpDesc &op, const tk_tucker *x,
                            const tk_tucker *b, int transpose) {
    ScopedMark mark(*c.arena);
    std::vector<TTerm> terms = apply_operator(c, pb, op, term_of(x), transpose);
    terms.push_back(term_of(b, -1.0));
    const double num = sum_norm(c, pb, terms);
    const double den = sum_norm(c, pb, {term_of(b)});
    return num / den;
}

// ------------------------------------------------------------------------------------------
// Adjoint contractions.  With mu the adjoint solution (L^T mu = dl/dx) and x the forward
// solution:  dl/dtheta_t = -<mu, L_t(x)>,  dl/dG_b = mu x_k U_bk^T = G_mu x_k (U_bk^T U_mu,k),
// dl/dU_bk = U_mu,k [G_mu x_{j != k} (U_bj^T U_mu,j)]_(k) G_b(k)^T.
// ------------------------------------------------------------------------------------------
static void adjoint_grads(Ctx &c, const Dims &pb, const OpDesc &op, const tk_tucker *mu, const tk_tucker *x,
                          const tk_tucker *b, double *dtheta_host, double *dcore, double *const *dfac) {
    ScopedMark mark(*c.arena);
    const int d = pb.d;
    const TTerm M = term_of(mu), X = term_of(x), Bt = term_of(b);
    double *dth = c.arena->alloc(op.nterms);
    if (dtheta_host) {
        OpDesc unit = op;
        for (auto &t : unit.theta) t = 1.0;
        std::vector<TTerm> lx = apply_operator(c, pb, unit, X, 0);
        std::vector<InnerJob> ij;
        for (int t = 0; t < op.nterms; ++t) ij.push_back(InnerJob{M, lx[t], dth + t});
        inner_batch(c, pb, ij);
    }
    // P_k = U_bk^T U_mu,k  (r_b x r_mu)
    double *P[TK_MAX_D];
    {
        Gemm g(c);
        for (int k = 0; k < d; ++k) {
            P[k] = c.arena->alloc((size_t)Bt.r[k] * M.r[k]);
            g.add1(Bt.r[k], M.r[k], pb.n[k], 1, 0, Bt.f[k], pb.n[k], M.f[k], pb.n[k], P[k], Bt.r[k]);
        }
        g.run();
    }
    if (dcore) {
        TtmGroup G{};
        for (int k = 0; k < d; ++k) G.sdims[k] = Bt.r[k];
        G.out = dcore;
        G.beta = 0.0;
        TtmJob J{};
        J.core = M.core;
        for (int k = 0; k < d; ++k) { J.r[k] = M.r[k]; J.P[k] = P[k]; J.ldp[k] = Bt.r[k]; }
        J.coef = 1.0;
        G.jobs.push_back(J);
        ttm_groups(c, d, {G});
    }
    if (dfac) {
        // H_k = G_mu x_{j != k} P_j  (identity in mode k), then dU_bk = U_mu,k H_k(k) G_b(k)^T
        std::vector<TtmGroup> groups(d);
        std::vector<double *> Hk(d);
        std::vector<double *> eye(d);
        for (int k = 0; k < d; ++k) {
            eye[k] = c.arena->alloc((size_t)M.r[k] * M.r[k]);
            set_identity(c, eye[k], M.r[k]);
        }
        for (int k = 0; k < d; ++k) {
            TtmGroup &G = groups[k];
            long long sz = 1;
            for (int j = 0; j < d; ++j) { G.sdims[j] = j == k ? M.r[j] : Bt.r[j]; sz *= G.sdims[j]; }
            Hk[k] = c.arena->alloc(sz);
            G.out = Hk[k];
            G.beta = 0.0;
            TtmJob J{};
            J.core = M.core;
            for (int j = 0; j < d; ++j) {
                J.r[j] = M.r[j];
                J.P[j] = j == k ? eye[k] : P[j];
                J.ldp[j] = j == k ? M.r[j] : Bt.r[j];
            }
            J.coef = 1.0;
            G.jobs.push_back(J);
        }
        ttm_groups(c, d, groups);
        // T_k (r_mu,k x r_b,k) = H_k(k) G_b(k)^T : contraction over all modes but k
        for (int k = 0; k < d; ++k) {
            const long long a = [&]() { long long p = 1; for (int j = 0; j < k; ++j) p *= Bt.r[j]; return p; }();
            const long long rest = [&]() { long long p = 1; for (int j = k + 1; j < d; ++j) p *= Bt.r[j]; return p; }();
            double *Ht = c.arena->alloc((size_t)M.r[k] * a * rest);
            double *Gt = c.arena->alloc((size_t)Bt.r[k] * a * rest);
            // unfoldings as (a*rest) x r transposes
            gather_unfold_t(c, Hk[k], Ht, a, M.r[k], rest);
            gather_unfold_t(c, Bt.core, Gt, a, Bt.r[k], rest);
            double *T = c.arena->alloc((size_t)M.r[k] * Bt.r[k]);
            Gemm g(c);
            g.add1(M.r[k], Bt.r[k], (int)(a * rest), 1, 0, Ht, (int)(a * rest), Gt, (int)(a * rest), T, M.r[k]);
            g.run();
            Gemm g2(c);
            g2.add1(pb.n[k], Bt.r[k], M.r[k], 0, 0, M.f[k], pb.n[k], T, M.r[k], dfac[k], pb.n[k]);
            g2.run();
        }
    }
    if (dtheta_host) {
        TK_CUDA(cudaMemcpyAsync(dtheta_host, dth, sizeof(double) * op.nterms, cudaMemcpyDeviceToHost, c.st));
        TK_CUDA(cudaStreamSynchronize(c.st));
        for (int t = 0; t < op.nterms; ++t) dtheta_host[t] = -dtheta_host[t];
    } else {
        TK_CUDA(cudaStreamSynchronize(c.st));
    }
}

}  // namespace tk

// ==========================================================================================
// C ABI
// ==========================================================================================
using namespace tk;

template <class F>
static int guarded(tk_handle *h, F &&f) {
    if (!h) return TK_EINVAL;
    h->err.clear();
    try {
        TK_CUDA(cudaSetDevice(h->device));
        return f();
    } catch (const Error &e) {
        h->err = e.msg;
        return e.code;
    } catch (const std::exception &e) {
        h->err = e.what();
        return TK_EINTERNAL;
    }
}

static Ctx make_ctx(tk_handle *h, void *stream) {
    Ctx c;
    c.st = (cudaStream_t)stream;
    c.arena = &h->arena;
    c.num_sms = h->num_sms;
    c.prof = h->prof_on ? &h->prof : nullptr;
    return c;
}

extern "C" {

int tk_create(tk_handle **out, int device) {
    if (!out) return TK_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return TK_ECUDA;
    }
    tk_handle *h = new tk_handle();
    h->device = device;
    if (cudaSetDevice(device) != cudaSuccess) { delete h; return TK_ECUDA; }
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMallocHost(&h->pinned, 256 * sizeof(double)) != cudaSuccess) { delete h; return TK_ENOMEM; }
    *out = h;
    return TK_OK;
}

int tk_destroy(tk_handle *h) {
    if (!h) return TK_EINVAL;
    cudaSetDevice(h->device);
    if (h->pinned) cudaFreeHost(h->pinned);
    delete h;
    return TK_OK;
}

const char *tk_last_error(const tk_handle *h) { return h ? h->err.c_str() : "null handle"; }

int tk_profile(tk_handle *h, int32_t enable) {
    return guarded(h, [&]() -> int {
        h->prof_on = enable != 0;
        return TK_OK;
    });
}

const char *tk_profile_report(tk_handle *h) {
    if (!h) return "";
    try {
        TK_CUDA(cudaSetDevice(h->device));
        h->prof_text = h->prof.report_and_reset();
    } catch (const Error &e) {
        h->err = e.msg;
        h->prof_text.clear();
    }
    return h->prof_text.c_str();
}

// The problem a checkpoint belongs to: shapes and options (stop_after, resume and
// true_residual excluded).  A resume must present the same.
struct CkFinger {
    uint32_t magic, version;
    int32_t d, precond, nterms, pc_nterms;
    int64_t n[TK_MAX_D], br[TK_MAX_D];
    tk_opts o;
};
constexpr uint32_t CK_MAGIC = 0x4b434b54u;   // "TKCK"
constexpr uint32_t CK_VERSION = 1;

static CkFinger finger_of(const tk_tucker *b, const tk_opts &o, const OpDesc &od, const OpDesc *pd) {
    CkFinger f;
    std::memset(&f, 0, sizeof f);
    f.magic = CK_MAGIC;
    f.version = CK_VERSION;
    f.d = b->d;
    f.precond = pd != nullptr;
    f.nterms = od.nterms;
    f.pc_nterms = pd ? pd->nterms : 0;
    for (int k = 0; k < b->d; ++k) { f.n[k] = b->n[k]; f.br[k] = b->r[k]; }
    f.o = o;
    f.o.stop_after = 0;
    f.o.resume = 0;
    f.o.true_residual = 0;
    return f;
}

static int solve_entry(tk_handle *h, const tk_operator *op, const tk_operator *pc, const tk_tucker *b,
                       const tk_opts *opts, tk_tucker *x_out, tk_report *report, void *stream,
                       int expsum_q = 0) {
    return guarded(h, [&]() -> int {
        TK_REQUIRE(opts != nullptr && report != nullptr, "solve: null opts or report");
        check_tucker(b, "b");
        check_tucker(x_out, "x_out");
        const Dims pb = dims_of(b);
        const OpDesc od = op_of(op, pb);
        const tk_opts o = *opts;
        TK_REQUIRE(x_out->d == b->d, "x_out: order differs from b");
        for (int k = 0; k < pb.d; ++k) {
            TK_REQUIRE(x_out->n[k] == b->n[k], "x_out: mode size differs from b");
            TK_REQUIRE(x_out->r[k] == o.rank_cap, "x_out: every rank must equal rank_cap");
        }
        TK_REQUIRE(o.variant == TK_RHOSVD_SGMRES || o.variant == TK_MLN_SGMRES || o.variant == TK_RHOSVD_GMRES,
                   "unknown variant");
        TK_REQUIRE(o.rank_cap >= 1 && o.oversample_p >= 0 && o.maxit >= 1, "bad rank_cap / p / maxit");
        TK_REQUIRE(o.precision == TK_FP64 || o.precision == TK_MIXED, "bad precision");
        TK_REQUIRE(o.adaptive_rank == 0 || o.adaptive_rank == 1, "adaptive_rank must be 0 or 1");
        TK_REQUIRE(o.gcv_tikhonov == 0 || o.gcv_tikhonov == 1, "gcv_tikhonov must be 0 or 1");
        TK_REQUIRE(o.gcv_rows == 0 || o.gcv_rows == 1, "gcv_rows must be 0 or 1");
        TK_REQUIRE(!o.gcv_tikhonov || o.maxit <= 96, "Tikhonov/GCV: maxit must be <= 96");
        TK_REQUIRE(o.tol > 0.0 && o.eta > 0.0 && o.round_tol >= 0.0, "bad tolerances");
        TK_REQUIRE(o.stop_after >= 0 && (o.resume == 0 || o.resume == 1), "bad stop_after / resume");
        if (o.variant == TK_RHOSVD_SGMRES) TK_REQUIRE(o.sketch_s >= 2 && o.sketch_s <= 4096, "sketch_s must be 2..4096");
        OpDesc pd;
        if (pc) {
            TK_REQUIRE(o.variant == TK_RHOSVD_SGMRES, "preconditioning is available for RHOSVD-Tucker sGMRES");
            pd = op_of(pc, pb);
        }
        if (expsum_q) {
            TK_REQUIRE(o.variant == TK_RHOSVD_SGMRES, "preconditioning is available for RHOSVD-Tucker sGMRES");
            TK_REQUIRE(expsum_q >= 1 && expsum_q <= 64, "expsum: q must be 1..64");
            for (int k = 0; k < pb.d; ++k) TK_REQUIRE(pb.n[k] <= 16384, "expsum: mode size must be <= 16384");
            pd.nterms = 2 * expsum_q + 1;   // recorded in the checkpoint fingerprint
        }
        CkFinger fp = finger_of(b, o, od, (pc || expsum_q) ? &pd : nullptr);
        if (expsum_q) fp.precond = 2;
        Ckpt ck;
        std::vector<char> next;
        if (o.resume) {
            TK_REQUIRE(h->ckpt.size() >= sizeof(CkFinger), "resume: no suspended solve in this handle");
            TK_REQUIRE(std::memcmp(h->ckpt.data(), &fp, sizeof(CkFinger)) == 0,
                       "resume: the suspended solve had another shape, variant or options");
            ck.in = &h->ckpt;
            ck.in_pos = sizeof(CkFinger);
        }
        if (o.stop_after > 0) {
            ck.stop_after = o.stop_after;
            next.resize(sizeof(CkFinger));
            std::memcpy(next.data(), &fp, sizeof(CkFinger));
            ck.out = &next;
        }
        Ctx c = make_ctx(h, stream);
        cudaEvent_t e0, e1;
        TK_CUDA(cudaEventCreate(&e0));
        TK_CUDA(cudaEventCreate(&e1));
        TK_CUDA(cudaEventRecord(e0, c.st));
        SolveOut so;
        ScopedMark pc_mark(h->arena);
        ExpSumPC es;
        if (expsum_q) {
            // sine eigenbasis and exponential weights per distinct mode size (Section 3.4)
            es.q = expsum_q;
            es.nh = 2 * expsum_q + 1;
            const double eta = M_PI / std::sqrt((double)expsum_q);
            for (int hh = -expsum_q; hh <= expsum_q; ++hh) es.coef.push_back(eta * std::exp(hh * eta));
            for (int k = 0; k < pb.d; ++k) {
                int same = -1;
                for (int j = 0; j < k; ++j)
                    if (pb.n[j] == pb.n[k]) { same = j; break; }
                if (same >= 0) { es.V[k] = es.V[same]; es.w[k] = es.w[same]; continue; }
                double *Vk = c.arena->alloc((size_t)pb.n[k] * pb.n[k]);
                double *wk = c.arena->alloc((size_t)pb.n[k] * es.nh);
                sine_basis(c, Vk, pb.n[k], 0.0);
                expsum_weights(c, wk, pb.n[k], expsum_q, eta);
                es.V[k] = Vk;
                es.w[k] = wk;
            }
        }
        if (o.variant == TK_RHOSVD_SGMRES)
            solve_rhosvd(c, pb, od, b, o, x_out, so, h->pinned, (pc || expsum_q) ? &pd : nullptr, ck,
                         expsum_q ? &es : nullptr);
        else if (o.variant == TK_RHOSVD_GMRES)
            solve_gmres(c, pb, od, b, o, x_out, so, h->pinned, ck);
        else
            solve_mln(c, pb, od, b, o, x_out, so, h->pinned, ck);
        TK_CUDA(cudaEventRecord(e1, c.st));
        TK_CUDA(cudaEventSynchronize(e1));
        if (o.precision == TK_MIXED && oz_error_flag(true) != 0)
            throw Error{TK_EINTERNAL, "a tensor-core GEMM gave up waiting for its copies or MMAs"};
        if (svd_error_flag(true) != 0)
            throw Error{TK_EINTERNAL, "a clustered SVD gave up waiting for its FP32 sweeps"};
        if (qr_error_flag(true) != 0)
            throw Error{TK_EINTERNAL, "a multi-cluster QR gave up waiting for another cluster's sums"};
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (so.status == TK_SUSPENDED) h->ckpt.swap(next);
        else if (o.resume) h->ckpt.clear();
        report->iters = so.iters;
        report->status = so.status;
        report->sketched_res = so.sres;
        if (report->res_hist)
            for (int i = 0; i < std::min<int>(report->res_hist_len, (int)so.hist.size()); ++i)
                report->res_hist[i] = so.hist[i];
        for (int k = 0; k < TK_MAX_D; ++k) report->out_rank[k] = k < pb.d ? so.ranks[k] : 0;
        report->ms_total = ms;
        report->workspace_bytes = (int64_t)h->arena.capacity();
        report->kernel_launches = c.launches;
        report->true_res = -1.0;
        if (o.true_residual && so.status != TK_SUSPENDED)
            report->true_res = true_residual(c, pb, od, x_out, b, o.transpose);
        return so.status;
    });
}

int tk_solve(tk_handle *h, const tk_operator *op, const tk_tucker *b, const tk_opts *opts,
             tk_tucker *x_out, tk_report *report, void *stream) {
    return solve_entry(h, op, nullptr, b, opts, x_out, report, stream);
}

int tk_solve_precond(tk_handle *h, const tk_operator *op, const tk_operator *precond, const tk_tucker *b,
                     const tk_opts *opts, tk_tucker *x_out, tk_report *report, void *stream) {
    if (!precond) return TK_EINVAL;
    return solve_entry(h, op, precond, b, opts, x_out, report, stream);
}

int tk_solve_expsum(tk_handle *h, const tk_operator *op, int32_t q, const tk_tucker *b, const tk_opts *opts,
                    tk_tucker *x_out, tk_report *report, void *stream) {
    if (q < 1) {
        if (h) h->err = "expsum: q must be >= 1";
        return TK_EINVAL;
    }
    return solve_entry(h, op, nullptr, b, opts, x_out, report, stream, q);
}

int tk_solve_concurrent(int32_t count, tk_solve_job *jobs) {
    if (count < 1 || !jobs) return TK_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!jobs[i].h) return TK_EINVAL;
        for (int j = 0; j < i; ++j)
            if (jobs[j].h == jobs[i].h) {
                jobs[i].h->err = "solve_concurrent: every job needs its own handle";
                return TK_EINVAL;
            }
    }
    auto run = [jobs](int i) {
        tk_solve_job &J = jobs[i];
        if (J.expsum_q > 0)
            J.status = tk_solve_expsum(J.h, J.op, J.expsum_q, J.b, J.opts, J.x_out, J.report, J.stream);
        else if (J.precond)
            J.status = tk_solve_precond(J.h, J.op, J.precond, J.b, J.opts, J.x_out, J.report, J.stream);
        else
            J.status = tk_solve(J.h, J.op, J.b, J.opts, J.x_out, J.report, J.stream);
    };
    std::vector<std::thread> th;
    int next = 1;
    try {
        for (; next < count; ++next) th.emplace_back(run, next);
    } catch (const std::exception &) {
        // no more threads: the remaining jobs run in this thread after the first
    }
    run(0);
    for (int i = next; i < count; ++i) run(i);
    for (auto &t : th) t.join();
    for (int i = 0; i < count; ++i)
        if (jobs[i].status < 0) return jobs[i].status;
    return TK_OK;
}

int tk_checkpoint_save(tk_handle *h, void *buf, int64_t cap, int64_t *size_out) {
    return guarded(h, [&]() -> int {
        TK_REQUIRE(!h->ckpt.empty(), "checkpoint_save: no suspended solve in this handle");
        if (size_out) *size_out = (int64_t)h->ckpt.size();
        if (!buf) return TK_OK;
        TK_REQUIRE(cap >= (int64_t)h->ckpt.size(), "checkpoint_save: buffer too small");
        std::memcpy(buf, h->ckpt.data(), h->ckpt.size());
        return TK_OK;
    });
}

int tk_checkpoint_load(tk_handle *h, const void *buf, int64_t size) {
    return guarded(h, [&]() -> int {
        TK_REQUIRE(buf != nullptr && size >= (int64_t)sizeof(CkFinger), "checkpoint_load: no state given");
        CkFinger f;
        std::memcpy(&f, buf, sizeof f);
        TK_REQUIRE(f.magic == CK_MAGIC && f.version == CK_VERSION, "checkpoint_load: not a checkpoint of this library");
        const char *p = static_cast<const char *>(buf);
        h->ckpt.assign(p, p + size);
        return TK_OK;
    });
}

int tk_fma_peak(tk_handle *h, int32_t fp64, double *tflops_host, void *stream) {
    return guarded(h, [&]() -> int {
        TK_REQUIRE(tflops_host != nullptr, "fma_peak: null output");
        Ctx c = make_ctx(h, stream);
        ScopedMark mark(h->arena);
        *tflops_host = fma_peak_tflops(c, fp64 ? 1 : 0);
        return TK_OK;
    });
}

int tk_selftest_qr_wait(tk_handle *h, int32_t mode, void *stream) {
    return guarded(h, [&]() -> int {
        TK_REQUIRE(mode == 1 || mode == 2, "selftest_qr_wait: mode 1 or 2");
        Ctx c = make_ctx(h, stream);
        ScopedMark mark(h->arena);
        if (!qr_wait_selftest(c, mode))
            throw Error{TK_EINTERNAL, "selftest_qr_wait: the lost exchange was not detected"};
        return TK_OK;
    });
}

int tk_set_workspace_limit(tk_handle *h, int64_t bytes) {
    return guarded(h, [&]() -> int {
        TK_REQUIRE(bytes >= 0, "workspace limit must be >= 0");
        h->arena.set_limit((size_t)bytes);
        return TK_OK;
    });
}

int tk_expsum_laplacian(tk_handle *h, int64_t n, int32_t q, double *const *mats, double *coef_host, void *stream) {
    return guarded(h, [&]() -> int {
        TK_REQUIRE(n >= 1 && n <= 16384 && q >= 1 && q <= 64 && mats && coef_host, "expsum: bad arguments");
        Ctx c = make_ctx(h, stream);
        ScopedMark mark(h->arena);
        const int nn = (int)n;
        double *V = c.arena->alloc((size_t)nn * nn);
        double *B = c.arena->alloc((size_t)nn * nn);
        sine_basis(c, V, nn, 0.0);
        const double eta = M_PI / std::sqrt((double)q);
        for (int hh = -q; hh <= q; ++hh) {
            const double t = std::exp(hh * eta);
            coef_host[hh + q] = eta * t;
            TK_REQUIRE(mats[hh + q] != nullptr, "expsum: null output matrix");
            sine_basis(c, B, nn, t);                      // V diag(exp(-t lambda))
            Gemm g(c);
            g.add1(nn, nn, nn, 0, 1, B, nn, V, nn, mats[hh + q], nn);   // (V D) V^T
            g.run();
        }
        TK_CUDA(cudaStreamSynchronize(c.st));
        return TK_OK;
    });
}

int tk_apply(tk_handle *h, const tk_operator *op, const tk_tucker *x, int32_t transpose,
             double *const *out_factors, void *stream) {
    return guarded(h, [&]() -> int {
        check_tucker(x, "x");
        TK_REQUIRE(out_factors != nullptr, "apply: null outputs");
        const Dims pb = dims_of(x);
        const OpDesc od = op_of(op, pb);
        Ctx c = make_ctx(h, stream);
        std::vector<BandJob> bj;
        Gemm g(c);
        for (int t = 0; t < od.nterms; ++t)
            for (int k = 0; k < pb.d; ++k) {
                const tk_modemat &m = od.mats[t * pb.d + k];
                double *o = out_factors[t * pb.d + k];
                TK_REQUIRE(o != nullptr, "apply: null output factor");
                const int n = pb.n[k], r = (int)x->r[k];
                if (m.kind == TK_IDENTITY) copy(c, o, x->factor[k], (long long)n * r);
                else if (m.kind == TK_BANDED) bj.push_back(BandJob{m.data, x->factor[k], o, n, r, m.kl, m.ku, transpose});
                else g.add1(n, r, n, transpose, 0, m.data, n, x->factor[k], n, o, n);
            }
        band_apply(c, bj);
        g.run();
        return TK_OK;
    });
}

int tk_roundsum(tk_handle *h, int32_t nterms, const tk_tucker *xs, const double *coef,
                const tk_opts *opts, uint64_t call_index, tk_tucker *out, int32_t *out_rank,
                void *stream) {
    return guarded(h, [&]() -> int {
        TK_REQUIRE(nterms >= 1 && xs != nullptr && coef != nullptr && opts != nullptr, "roundsum: bad arguments");
        check_tucker(out, "out");
        const Dims pb = dims_of(out);
        std::vector<TTerm> terms;
        for (int i = 0; i < nterms; ++i) {
            check_tucker(&xs[i], "term");
            TK_REQUIRE(xs[i].d == pb.d, "roundsum: order mismatch");
            for (int k = 0; k < pb.d; ++k) TK_REQUIRE(xs[i].n[k] == pb.n[k], "roundsum: mode size mismatch");
            terms.push_back(term_of(&xs[i], coef[i]));
        }
        const int R = opts->rank_cap;
        for (int k = 0; k < pb.d; ++k) TK_REQUIRE(out->r[k] == R, "roundsum: out ranks must equal rank_cap");
        TK_REQUIRE(opts->adaptive_rank == 0 || opts->adaptive_rank == 1, "roundsum: adaptive_rank must be 0 or 1");
        const int sr = R + opts->oversample_p;
        TK_REQUIRE(sr <= 96, "roundsum: rank_cap + p must be <= 96");
        Ctx c = make_ctx(h, stream);
        ScopedMark mark(h->arena);
        TOut o{};
        o.core = out->core;
        for (int k = 0; k < pb.d; ++k) o.f[k] = out->factor[k];
        o.rank_dev = c.arena->alloc_int(TK_MAX_D);
        roundsum(c, pb, terms, rs_cfg(*opts, sr, R, call_index, opts->precision == TK_MIXED ? 1 : 0), o);
        int hr[TK_MAX_D];
        TK_CUDA(cudaMemcpyAsync(hr, o.rank_dev, sizeof(int) * pb.d, cudaMemcpyDeviceToHost, c.st));
        TK_CUDA(cudaStreamSynchronize(c.st));
        if (svd_error_flag(true) != 0)
            throw Error{TK_EINTERNAL, "a clustered SVD gave up waiting for its FP32 sweeps"};
        if (qr_error_flag(true) != 0)
            throw Error{TK_EINTERNAL, "a multi-cluster QR gave up waiting for another cluster's sums"};
        if (out_rank) for (int k = 0; k < pb.d; ++k) out_rank[k] = hr[k];
        return TK_OK;
    });
}

int tk_kron_sketch(tk_handle *h, const tk_tucker *x, const double *const *S, int32_t s, double *out,
                   void *stream) {
    return guarded(h, [&]() -> int {
        check_tucker(x, "x");
        TK_REQUIRE(S != nullptr && out != nullptr && s >= 1, "kron_sketch: bad arguments");
        const Dims pb = dims_of(x);
        Ctx c = make_ctx(h, stream);
        ScopedMark mark(h->arena);
        kron_sketch_batch(c, pb, {term_of(x)}, S, s, &out);
        return TK_OK;
    });
}

int tk_inner(tk_handle *h, const tk_tucker *x, const tk_tucker *y, double *out_host, void *stream) {
    return guarded(h, [&]() -> int {
        check_tucker(x, "x");
        check_tucker(y, "y");
        TK_REQUIRE(out_host != nullptr && x->d == y->d, "inner: bad arguments");
        for (int k = 0; k < x->d; ++k) TK_REQUIRE(x->n[k] == y->n[k], "inner: mode size mismatch");
        const Dims pb = dims_of(x);
        Ctx c = make_ctx(h, stream);
        ScopedMark mark(h->arena);
        double *o = c.arena->alloc(1);
        inner_batch(c, pb, {InnerJob{term_of(x), term_of(y), o}});
        TK_CUDA(cudaMemcpyAsync(h->pinned, o, sizeof(double), cudaMemcpyDeviceToHost, c.st));
        TK_CUDA(cudaStreamSynchronize(c.st));
        *out_host = h->pinned[0];
        return TK_OK;
    });
}

int tk_residual(tk_handle *h, const tk_operator *op, const tk_tucker *x, const tk_tucker *b,
                int32_t transpose, double *rel_host, void *stream) {
    return guarded(h, [&]() -> int {
        check_tucker(x, "x");
        check_tucker(b, "b");
        TK_REQUIRE(rel_host != nullptr && x->d == b->d, "residual: bad arguments");
        for (int k = 0; k < x->d; ++k) TK_REQUIRE(x->n[k] == b->n[k], "residual: mode size mismatch");
        const Dims pb = dims_of(x);
        const OpDesc od = op_of(op, pb);
        Ctx c = make_ctx(h, stream);
        *rel_host = true_residual(c, pb, od, x, b, transpose);
        return TK_OK;
    });
}

int tk_sum_norm(tk_handle *h, int32_t nterms, const tk_tucker *xs, const double *coef, double *out_host,
                void *stream) {
    return guarded(h, [&]() -> int {
        TK_REQUIRE(nterms >= 1 && xs && coef && out_host, "sum_norm: bad arguments");
        check_tucker(&xs[0], "term");
        const Dims pb = dims_of(&xs[0]);
        std::vector<TTerm> terms;
        for (int i = 0; i < nterms; ++i) {
            check_tucker(&xs[i], "term");
            TK_REQUIRE(xs[i].d == pb.d, "sum_norm: order mismatch");
            for (int k = 0; k < pb.d; ++k) TK_REQUIRE(xs[i].n[k] == pb.n[k], "sum_norm: mode size mismatch");
            terms.push_back(term_of(&xs[i], coef[i]));
        }
        Ctx c = make_ctx(h, stream);
        *out_host = sum_norm(c, pb, terms);
        return TK_OK;
    });
}

int tk_adjoint_grads(tk_handle *h, const tk_operator *op, const tk_tucker *mu, const tk_tucker *x,
                     const tk_tucker *b, double *dtheta_host, double *dcore_b, double *const *dfactor_b,
                     void *stream) {
    return guarded(h, [&]() -> int {
        check_tucker(mu, "mu");
        check_tucker(x, "x");
        check_tucker(b, "b");
        const Dims pb = dims_of(mu);
        for (int k = 0; k < pb.d; ++k)
            TK_REQUIRE(x->n[k] == pb.n[k] && b->n[k] == pb.n[k], "adjoint_grads: mode size mismatch");
        TK_REQUIRE(x->d == pb.d && b->d == pb.d, "adjoint_grads: order mismatch");
        const OpDesc od = op_of(op, pb);
        Ctx c = make_ctx(h, stream);
        adjoint_grads(c, pb, od, mu, x, b, dtheta_host, dcore_b, dfactor_b);
        return TK_OK;
    });
}

int tk_gaussian(tk_handle *h, uint64_t seed, uint64_t stream_id, int64_t count, int32_t bf16_round,
                double *out, void *stream) {
    return guarded(h, [&]() -> int {
        TK_REQUIRE(out != nullptr && count >= 0, "gaussian: bad arguments");
        if (count == 0) return TK_OK;
        Ctx c = make_ctx(h, stream);
        long long cnt = count;
        gaussian(c, seed, &stream_id, &cnt, &out, 1, bf16_round);
        return TK_OK;
    });
}

int tk_philox(tk_handle *h, uint64_t seed, uint64_t stream_id, uint64_t first, int64_t nblocks,
              uint32_t *out, void *stream) {
    return guarded(h, [&]() -> int {
        TK_REQUIRE(out != nullptr && nblocks >= 0, "philox: bad arguments");
        if (nblocks == 0) return TK_OK;
        Ctx c = make_ctx(h, stream);
        philox_raw(c, seed, stream_id, first, nblocks, out);
        return TK_OK;
    });
}

int tk_sketched_ls(tk_handle *h, const double *M, const double *b, int32_t s, int32_t k, double *y,
                   double *res, void *stream) {
    return guarded(h, [&]() -> int {
        TK_REQUIRE(M && b && y && res, "sketched_ls: null pointer");
        TK_REQUIRE(k >= 1 && k < s && s <= 1024, "sketched_ls: need 1 <= k < s <= 1024");
        Ctx c = make_ctx(h, stream);
        ScopedMark mark(h->arena);
        LSState st{};
        st.H = c.arena->alloc((size_t)s * k);
        st.tau = c.arena->alloc(k);
        st.qtb = c.arena->alloc(s);
        if (k <= LSW_MAXK) {
            st.T = c.arena->alloc((size_t)k * k);
            st.ldt = k;
        }
        st.y = y;
        st.res = res;
        ls_update(c, M, b, s, 0, k, st, 1);
        TK_CUDA(cudaStreamSynchronize(c.st));   // workspace is released on return
        return TK_OK;
    });
}

int tk_mln_roundsum(tk_handle *h, int32_t nterms, const tk_tucker *xs, const double *coef,
                    const double *const *psi, int32_t r, int32_t p, tk_tucker *out, void *stream) {
    return guarded(h, [&]() -> int {
        TK_REQUIRE(nterms >= 1 && xs && coef && psi && r >= 1 && p >= 0 && r <= 96, "mln_roundsum: bad arguments");
        check_tucker(out, "out");
        const Dims pb = dims_of(out);
        for (int k = 0; k < pb.d; ++k) TK_REQUIRE(out->r[k] == r, "mln_roundsum: out ranks must equal r");
        std::vector<TTerm> terms;
        for (int i = 0; i < nterms; ++i) {
            check_tucker(&xs[i], "term");
            TK_REQUIRE(xs[i].d == pb.d, "mln_roundsum: order mismatch");
            terms.push_back(term_of(&xs[i], coef[i]));
        }
        Ctx c = make_ctx(h, stream);
        ScopedMark mark(h->arena);
        Sk sk = alloc_sk(c, pb, r, r + p);
        mln_sketch_sum(c, pb, terms, psi, r, p, sk.g, sk.F, 0.0);
        TOut o{};
        o.core = out->core;
        for (int k = 0; k < pb.d; ++k) o.f[k] = out->factor[k];
        o.rank_dev = nullptr;
        mln_recovery(c, pb, sk.g, sk.F, psi, r, p, o);
        TK_CUDA(cudaStreamSynchronize(c.st));
        return TK_OK;
    });
}

}  // extern "C"
