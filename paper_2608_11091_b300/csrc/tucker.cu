// Tucker-level building blocks on top of the kernels: MTTKRP (Definition 2.3), TTM chains
// (Definition 2.2), Tucker inner products (Section 2.2), the Kronecker-structured sketch
// (Algorithm 2), the separable-operator apply (Eq. (1.2)), RoundSum (Section 3.1) and the
// multilinear Nystrom routines (Algorithms 3-5).
#include <algorithm>
#include <map>

#include "tucker.cuh"

namespace tk {

static long long prod(const int *v, int a, int b) {
    long long p = 1;
    for (int i = a; i < b; ++i) p *= v[i];
    return p;
}

// ------------------------------------------------------------------------------------------
// MTTKRP / Khatri-Rao contraction of a core with per-mode matrices P_j (r_j x s):
//   keep >= 0:  out (r_keep x s) = G_(keep) (KR_{j != keep} P_j)      (Definition 2.3)
//   keep <  0:  out (s)          with out[l] = sum_a G[a] prod_j P_j[a_j, l]
// One GEMM contracts an outer mode, then row-wise Hadamard contractions remove the rest.
// ------------------------------------------------------------------------------------------
void mttkrp_batch(Ctx &c, int d, int s, const std::vector<MttJob> &jobs, bool tensor_cores) {
    struct St { std::vector<int> dims, modes; const double *T; };
    std::vector<St> st(jobs.size());
    Gemm g(c, "gemm_mttkrp", tensor_cores);
    for (size_t i = 0; i < jobs.size(); ++i) {
        const MttJob &J = jobs[i];
        const int nleft = (J.keep >= 0) ? d - 2 : d - 1;   // contractions after the GEMM
        if (J.keep != d - 1) {
            const long long rest = prod(J.r, 0, d - 1);
            double *T = nleft == 0 ? J.out : c.arena->alloc(rest * s);
            g.add1((int)rest, s, J.r[d - 1], 0, 0, J.core, (int)rest, J.P[d - 1], J.ldp[d - 1], T, (int)rest);
            for (int k = 0; k < d - 1; ++k) { st[i].dims.push_back(J.r[k]); st[i].modes.push_back(k); }
            st[i].T = T;
        } else {
            const long long rest = prod(J.r, 1, d);
            double *T = nleft == 0 ? J.out : c.arena->alloc(rest * s);
            g.add1((int)rest, s, J.r[0], 1, 0, J.core, J.r[0], J.P[0], J.ldp[0], T, (int)rest);
            for (int k = 1; k < d; ++k) { st[i].dims.push_back(J.r[k]); st[i].modes.push_back(k); }
            st[i].T = T;
        }
    }
    g.run();
    for (;;) {
        std::vector<HadJob> hj;
        for (size_t i = 0; i < jobs.size(); ++i) {
            const MttJob &J = jobs[i];
            St &S = st[i];
            int pos = -1, remaining = 0;
            for (int p = 0; p < (int)S.modes.size(); ++p)
                if (S.modes[p] != J.keep) { pos = p; ++remaining; }
            if (pos < 0) continue;
            long long a = 1, cc = 1;
            for (int p = 0; p < pos; ++p) a *= S.dims[p];
            for (int p = pos + 1; p < (int)S.dims.size(); ++p) cc *= S.dims[p];
            double *out = remaining == 1 ? J.out : c.arena->alloc(a * cc * s);
            const int m = S.modes[pos];
            hj.push_back(HadJob{S.T, J.P[m], out, (int)a, S.dims[pos], (int)cc, s, J.ldp[m]});
            S.dims.erase(S.dims.begin() + pos);
            S.modes.erase(S.modes.begin() + pos);
            S.T = out;
        }
        if (hj.empty()) break;
        hadamard_contract(c, hj);
    }
}

// ------------------------------------------------------------------------------------------
// Sums of TTM chains:  out_g = beta_g out_g + sum_j coef_j G_j x_1 P_1j ... x_d P_dj
// (P_kj is s_k x r_kj with leading dimension ldp).  Levels are batched across groups; the
// last mode sums the terms of a group as GEMM segments (no atomics).
// ------------------------------------------------------------------------------------------
void ttm_groups(Ctx &c, int d, const std::vector<TtmGroup> &groups, bool tc) {
    struct St { const double *X; int dims[TK_MAX_D]; };
    std::vector<std::vector<St>> st(groups.size());
    for (size_t gi = 0; gi < groups.size(); ++gi)
        for (const TtmJob &J : groups[gi].jobs) {
            St s{};
            s.X = J.core;
            for (int k = 0; k < d; ++k) s.dims[k] = J.r[k];
            st[gi].push_back(s);
        }
    for (int k = 0; k < d - 1; ++k) {
        Gemm g(c, "gemm_ttm", tc);
        for (size_t gi = 0; gi < groups.size(); ++gi) {
            const TtmGroup &G = groups[gi];
            for (size_t ji = 0; ji < G.jobs.size(); ++ji) {
                const TtmJob &J = G.jobs[ji];
                St &S = st[gi][ji];
                const long long a = prod(S.dims, 0, k), b = prod(S.dims, k + 1, d);
                const int rk = S.dims[k], sk = G.sdims[k];
                double *Y = c.arena->alloc(a * sk * b);
                if (k == 0)
                    g.add1(sk, (int)b, rk, 0, 0, J.P[0], J.ldp[0], S.X, rk, Y, sk);
                else
                    g.add1((int)a, sk, rk, 0, 1, S.X, (int)a, J.P[k], J.ldp[k], Y, (int)a, 0.0, 1.0,
                           nullptr, (int)b, a * rk, 0, a * sk);
                S.X = Y;
                S.dims[k] = sk;
            }
        }
        g.run();
    }
    Gemm g(c, "gemm_ttm", tc);
    const int k = d - 1;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const TtmGroup &G = groups[gi];
        if (G.jobs.empty()) continue;
        const long long a = prod(G.sdims, 0, k);
        const int sk = G.sdims[k];
        std::vector<Gemm::Seg> segs;
        for (size_t ji = 0; ji < G.jobs.size(); ++ji) {
            const TtmJob &J = G.jobs[ji];
            if (k == 0)
                segs.push_back(Gemm::Seg{J.P[0], J.ldp[0], st[gi][ji].X, st[gi][ji].dims[0],
                                         st[gi][ji].dims[0], J.coef, J.coef_dev});
            else
                segs.push_back(Gemm::Seg{st[gi][ji].X, (int)a, J.P[k], J.ldp[k], st[gi][ji].dims[k],
                                         J.coef, J.coef_dev});
        }
        if (k == 0)
            g.add(sk, 1, 0, 0, G.out, sk, G.beta, segs);   // order-1 tensors
        else
            g.add((int)a, sk, 0, 1, G.out, (int)a, G.beta, segs);
    }
    g.run();
}

// ------------------------------------------------------------------------------------------
// Inner products <X, Y> = <G_X, G_Y x_k (U_k^T W_k)>
// ------------------------------------------------------------------------------------------
void inner_batch(Ctx &c, const Dims &pb, const std::vector<InnerJob> &jobs) {
    const int d = pb.d;
    Gemm g(c, "gemm_inner");
    std::vector<std::vector<double *>> P(jobs.size());
    for (size_t i = 0; i < jobs.size(); ++i) {
        const InnerJob &J = jobs[i];
        for (int k = 0; k < d; ++k) {
            double *p = c.arena->alloc((size_t)J.x.r[k] * J.y.r[k]);
            g.add1(J.x.r[k], J.y.r[k], pb.n[k], 1, 0, J.x.f[k], pb.n[k], J.y.f[k], pb.n[k], p, J.x.r[k]);
            P[i].push_back(p);
        }
    }
    g.run();
    std::vector<TtmGroup> groups(jobs.size());
    std::vector<double *> tmp(jobs.size());
    for (size_t i = 0; i < jobs.size(); ++i) {
        const InnerJob &J = jobs[i];
        TtmGroup &G = groups[i];
        TtmJob t{};
        t.core = J.y.core;
        for (int k = 0; k < d; ++k) {
            t.r[k] = J.y.r[k];
            t.P[k] = P[i][k];
            t.ldp[k] = J.x.r[k];
            G.sdims[k] = J.x.r[k];
        }
        t.coef = 1.0;
        G.jobs.push_back(t);
        tmp[i] = c.arena->alloc(prod(J.x.r, 0, d));
        G.out = tmp[i];
        G.beta = 0.0;
    }
    ttm_groups(c, d, groups);
    std::vector<DotJob> dj;
    for (size_t i = 0; i < jobs.size(); ++i) dj.push_back(DotJob{jobs[i].x.core, tmp[i], prod(jobs[i].x.r, 0, d), jobs[i].out});
    dots(c, dj);
}

// ------------------------------------------------------------------------------------------
// Kronecker-structured sketch: out[l] = X x_1 S_1[:,l]^T ... x_d S_d[:,l]^T
// ------------------------------------------------------------------------------------------
void kron_sketch_batch(Ctx &c, const Dims &pb, const std::vector<TTerm> &xs,
                       const double *const *S, int s, double *const *outs) {
    const int d = pb.d;
    Gemm g(c, "gemm_sketch");
    std::vector<MttJob> mj(xs.size());
    for (size_t i = 0; i < xs.size(); ++i) {
        MttJob &J = mj[i];
        J.core = xs[i].core;
        J.keep = -1;
        J.out = outs[i];
        for (int k = 0; k < d; ++k) {
            J.r[k] = xs[i].r[k];
            double *p = c.arena->alloc((size_t)xs[i].r[k] * s);
            g.add1(xs[i].r[k], s, pb.n[k], 1, 0, xs[i].f[k], pb.n[k], S[k], pb.n[k], p, xs[i].r[k]);
            J.P[k] = p;
            J.ldp[k] = xs[i].r[k];
        }
    }
    g.run();
    mttkrp_batch(c, d, s, mj);
}

// ------------------------------------------------------------------------------------------
// Operator apply (Eq. (1.2)): term t of L(X) is [theta_t G; A_1^(t) U_1, ..., A_d^(t) U_d].
// Identity modes share X's factor; banded modes run the band kernel; dense modes a GEMM.
// ------------------------------------------------------------------------------------------
std::vector<TTerm> apply_operator(Ctx &c, const Dims &pb, const OpDesc &op, const TTerm &x,
                                  int transpose, bool tc) {
    const int d = pb.d;
    std::vector<TTerm> out(op.nterms);
    std::vector<BandJob> bj;
    Gemm g(c, "gemm_apply", tc);
    // distinct (matrix, mode) pairs produce one factor each
    std::map<std::pair<const void *, int>, double *> made;
    for (int t = 0; t < op.nterms; ++t) {
        TTerm &T = out[t];
        T.core = x.core;
        T.coef = op.theta[t] * x.coef;
        T.coef_dev = x.coef_dev;
        for (int k = 0; k < d; ++k) {
            T.r[k] = x.r[k];
            const tk_modemat &m = op.mats[t * d + k];
            if (m.kind == TK_IDENTITY) {
                T.f[k] = x.f[k];
                continue;
            }
            auto key = std::make_pair((const void *)m.data, k + 16 * m.kind + 64 * m.kl + 8192 * m.ku);
            auto it = made.find(key);
            if (it != made.end()) { T.f[k] = it->second; continue; }
            double *buf = c.arena->alloc((size_t)pb.n[k] * x.r[k]);
            if (m.kind == TK_BANDED)
                bj.push_back(BandJob{m.data, x.f[k], buf, pb.n[k], x.r[k], m.kl, m.ku, transpose});
            else
                g.add1(pb.n[k], x.r[k], pb.n[k], transpose, 0, m.data, pb.n[k], x.f[k], pb.n[k], buf, pb.n[k]);
            made[key] = buf;
            T.f[k] = buf;
        }
    }
    band_apply(c, bj);
    g.run();
    return out;
}

// ------------------------------------------------------------------------------------------
// RoundSum (Section 3.1): Khatri-Rao sketched randomized HOSVD of sum_i c_i X_i followed by
// ST-HOSVD of the projected core.  Output zero-padded to rank R.
// ------------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------------
// Effective-rank sketch size (Section 3.1): V_k = [|c_i| ||G^(i)||_F U_k^(i)]_i, its squared
// singular values are the eigenvalues lambda of V_k^T V_k; r~_k is the smallest r with
// sum_{j > r} lambda_j <= rank_tol^2 sum_j lambda_j and s = min(max_k r~_k, cap) + p.  Formed
// when V_k has at most 96 columns or rows (pivoted QR of V_k or V_k^T, Jacobi SVD of its R);
// beyond that r~_k = cap.  One read-back of the singular values per call.
// ------------------------------------------------------------------------------------------
int effective_sketch_size(Ctx &c, const Dims &pb, const std::vector<TTerm> &terms, int cap, int p,
                          double rank_tol) {
    ScopedMark mark(*c.arena);
    const int d = pb.d, N = (int)terms.size();
    constexpr int GMAX = 96;
    double *ns = c.arena->alloc(N);
    {
        std::vector<DotJob> dj;
        for (int i = 0; i < N; ++i) dj.push_back(DotJob{terms[i].core, terms[i].core, prod(terms[i].r, 0, d), ns + i});
        dots(c, dj);
    }
    int width[TK_MAX_D], cols[TK_MAX_D];
    bool formed[TK_MAX_D];
    std::vector<QRJob> qj;
    std::vector<SVDJob> sj;
    double *sig = c.arena->alloc((size_t)d * GMAX);
    fill(c, sig, (long long)d * GMAX, 0.0);
    std::vector<WeightedCopyJob> wj;
    double *Vk[TK_MAX_D];
    for (int k = 0; k < d; ++k) {
        width[k] = 0;
        for (int i = 0; i < N; ++i) width[k] += terms[i].r[k];
        formed[k] = std::min(pb.n[k], width[k]) <= GMAX;
        if (!formed[k]) continue;
        Vk[k] = c.arena->alloc((size_t)pb.n[k] * width[k]);
        int off = 0;
        for (int i = 0; i < N; ++i) {
            wj.push_back(WeightedCopyJob{terms[i].f[k], Vk[k] + (size_t)off * pb.n[k], terms[i].coef_dev, ns + i,
                                         terms[i].coef, pb.n[k], terms[i].r[k]});
            off += terms[i].r[k];
        }
    }
    weighted_copy(c, wj);
    for (int k = 0; k < d; ++k) {
        if (!formed[k]) continue;
        // columns of the QR: the smaller side (V_k or its transpose)
        double *A = Vk[k];
        int m = pb.n[k];
        cols[k] = width[k];
        if (width[k] > pb.n[k]) {
            A = c.arena->alloc((size_t)pb.n[k] * width[k]);
            transpose_block(c, A, width[k], Vk[k], pb.n[k], pb.n[k], width[k]);
            m = width[k];
            cols[k] = pb.n[k];
        }
        int *perm = c.arena->alloc_int(cols[k]);
        qj.push_back(QRJob{A, c.arena->alloc(cols[k]), nullptr, m, cols[k], perm});
        SVDJob s{};
        s.perm = perm;
        s.R = A; s.ldr = m; s.s = std::min(m, cols[k]); s.W = nullptr; s.wcols = 0;
        s.sigma = sig + (size_t)k * GMAX; s.rank = nullptr; s.normsq = nullptr; s.eps2_over_d = 0.0;
        s.rank_cap = s.s;
        sj.push_back(s);
    }
    if (!qj.empty()) {
        qr_householder(c, qj);
        svd_jacobi(c, sj);
    }
    std::vector<double> hs((size_t)d * GMAX);
    TK_CUDA(cudaMemcpyAsync(hs.data(), sig, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, c.st));
    TK_CUDA(cudaStreamSynchronize(c.st));
    int rmax = 1;
    for (int k = 0; k < d; ++k) {
        int rk = cap;
        if (formed[k]) {
            const int q = std::min(pb.n[k], width[k]);
            std::vector<double> lam(q);
            double total = 0.0;
            for (int j = 0; j < q; ++j) { lam[j] = hs[(size_t)k * GMAX + j] * hs[(size_t)k * GMAX + j]; total += lam[j]; }
            // tail[r] = sum_{j >= r} lambda_j (descending order); smallest r >= 1 with tail <= thr
            const double thr = rank_tol * rank_tol * total;
            double tail = 0.0;
            rk = q;
            std::vector<double> suffix(q + 1, 0.0);
            for (int j = q - 1; j >= 0; --j) { tail += lam[j]; suffix[j] = tail; }
            for (int r = 1; r <= q; ++r)
                if (suffix[r] <= thr) { rk = r; break; }
        }
        rmax = std::max(rmax, rk);
    }
    return std::min(rmax, cap) + p;
}

void roundsum(Ctx &c, const Dims &pb, const std::vector<TTerm> &terms, const RSConfig &cfg,
              const TOut &out) {
    ScopedMark mark(*c.arena);
    const int N = (int)terms.size();
    TK_REQUIRE(N >= 1, "roundsum: no terms");
    const int d = pb.d, R = cfg.R;
    const int sr = cfg.adaptive_p >= 0 ? effective_sketch_size(c, pb, terms, R, cfg.adaptive_p, cfg.rank_tol) : cfg.sr;
    if (cfg.sr_used) *cfg.sr_used = sr;
    // 1. Gaussian S_k (n_k x sr), stream (seed, purpose 2, call, k)
    double *S[TK_MAX_D];
    {
        uint64_t sids[TK_MAX_D];
        long long cnt[TK_MAX_D];
        for (int k = 0; k < d; ++k) {
            S[k] = c.arena->alloc((size_t)pb.n[k] * sr);
            sids[k] = (uint64_t(2) << 48) | (cfg.call << 8) | uint64_t(k);
            cnt[k] = (long long)pb.n[k] * sr;
        }
        gaussian(c, cfg.seed, sids, cnt, S, d, cfg.bf16_sketch);
    }
    const bool mixed = cfg.bf16_sketch != 0;            // range finder on tensor cores
    const bool all_tc = mixed && cfg.tc_all != 0;        // representation too (preconditioner)
    if (cfg.rot) {
        // terms given in the bases Q_k: rotate the sketches, S_k <- Q_k^T S_k
        Gemm g(c, "gemm_rotate", mixed);
        for (int k = 0; k < d; ++k) {
            double *Sr = c.arena->alloc((size_t)pb.n[k] * sr);
            g.add1(pb.n[k], sr, pb.n[k], 1, 0, cfg.rot[k], pb.n[k], S[k], pb.n[k], Sr, pb.n[k]);
            S[k] = Sr;
        }
        g.run();
    }
    // 2. factor sketches M_j^(i) = U_j^(i)T S_j, shared between terms with the same factor
    // (mixed form: on tensor cores, gemm_oz)
    std::vector<std::vector<const double *>> M(N, std::vector<const double *>(d));
    {
        Gemm g(c, "gemm_factor_sketch", mixed);
        std::map<const double *, double *> made[TK_MAX_D];
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < d; ++j) {
                auto it = made[j].find(terms[i].f[j]);
                if (it != made[j].end()) { M[i][j] = it->second; continue; }
                double *m = c.arena->alloc((size_t)terms[i].r[j] * sr);
                g.add1(terms[i].r[j], sr, pb.n[j], 1, 0, terms[i].f[j], pb.n[j], S[j], pb.n[j], m, terms[i].r[j]);
                made[j][terms[i].f[j]] = m;
                M[i][j] = m;
            }
        g.run();
    }
    // 3. Z_k^(i) = G_(k)^(i) (KR_{j != k} M_j^(i))   (r_k x sr)
    std::vector<std::vector<double *>> Z(N, std::vector<double *>(d));
    {
        std::vector<MttJob> mj;
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < d; ++k) {
                MttJob J{};
                J.core = terms[i].core;
                J.keep = k;
                for (int j = 0; j < d; ++j) { J.r[j] = terms[i].r[j]; J.P[j] = M[i][j]; J.ldp[j] = terms[i].r[j]; }
                Z[i][k] = c.arena->alloc((size_t)terms[i].r[k] * sr);
                J.out = Z[i][k];
                mj.push_back(J);
            }
        mttkrp_batch(c, d, sr, mj, mixed);
    }
    // 4. Y_k = sum_i c_i U_k^(i) Z_k^(i)   (n_k x sr)
    double *Y[TK_MAX_D], *Q[TK_MAX_D];
    {
        Gemm g(c, "gemm_range", all_tc);
        for (int k = 0; k < d; ++k) {
            Y[k] = c.arena->alloc((size_t)pb.n[k] * sr);
            std::vector<Gemm::Seg> segs;
            for (int i = 0; i < N; ++i)
                segs.push_back(Gemm::Seg{terms[i].f[k], pb.n[k], Z[i][k], terms[i].r[k], terms[i].r[k],
                                         terms[i].coef, terms[i].coef_dev});
            g.add(pb.n[k], sr, 0, 0, Y[k], pb.n[k], 0.0, segs);
        }
        g.run();
    }
    // 5. economy QR of every Y_k -> orthonormal U^_k (n_k x sr; zero columns beyond n_k)
    {
        std::vector<QRJob> qj;
        for (int k = 0; k < d; ++k) {
            Q[k] = c.arena->alloc((size_t)pb.n[k] * sr);
            double *tau = c.arena->alloc(sr);
            qj.push_back(QRJob{Y[k], tau, Q[k], pb.n[k], sr, nullptr});
        }
        qr_householder(c, qj);
    }
    // 6. projections P_k^(i) = U^_k^T U_k^(i)   (sr x r_k^(i))
    std::vector<std::vector<const double *>> P(N, std::vector<const double *>(d));
    {
        Gemm g(c, "gemm_proj", all_tc);
        std::map<const double *, double *> made[TK_MAX_D];
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < d; ++k) {
                auto it = made[k].find(terms[i].f[k]);
                if (it != made[k].end()) { P[i][k] = it->second; continue; }
                double *p = c.arena->alloc((size_t)sr * terms[i].r[k]);
                g.add1(sr, terms[i].r[k], pb.n[k], 1, 0, Q[k], pb.n[k], terms[i].f[k], pb.n[k], p, sr);
                made[k][terms[i].f[k]] = p;
                P[i][k] = p;
            }
        g.run();
    }
    // 7. core projection C^ = sum_i c_i G^(i) x_1 P_1^(i) ... x_d P_d^(i)   (sr^d)
    long long csize = 1;
    for (int k = 0; k < d; ++k) csize *= sr;
    double *C = c.arena->alloc(csize);
    {
        TtmGroup G{};
        for (int k = 0; k < d; ++k) G.sdims[k] = sr;
        G.out = C;
        G.beta = 0.0;
        for (int i = 0; i < N; ++i) {
            TtmJob J{};
            J.core = terms[i].core;
            for (int k = 0; k < d; ++k) { J.r[k] = terms[i].r[k]; J.P[k] = P[i][k]; J.ldp[k] = sr; }
            J.coef = terms[i].coef;
            J.coef_dev = terms[i].coef_dev;
            G.jobs.push_back(J);
        }
        ttm_groups(c, d, {G}, all_tc);
    }
    // 8. ST-HOSVD of C^: per mode QR of the transposed unfolding, Jacobi SVD of R, truncate
    double *normsq = c.arena->alloc(1);
    dot(c, C, C, csize, normsq);
    int cur[TK_MAX_D];
    for (int k = 0; k < d; ++k) cur[k] = sr;
    double *W[TK_MAX_D];
    for (int k = 0; k < d; ++k) {
        const long long a = prod(cur, 0, k), rest = prod(cur, k + 1, d);
        const long long m = a * rest;
        const int sk = cur[k];
        double *Ut = c.arena->alloc(m * sk);
        gather_unfold_t(c, C, Ut, a, sk, rest);
        double *tau = c.arena->alloc(sk);
        int *perm = c.arena->alloc_int(sk);
        qr_householder(c, {QRJob{Ut, tau, nullptr, (int)m, sk, perm}});
        W[k] = c.arena->alloc((size_t)sk * R);
        SVDJob sj{};
        sj.perm = perm;
        sj.R = Ut; sj.ldr = (int)m; sj.s = sk; sj.W = W[k]; sj.wcols = R; sj.sigma = nullptr;
        sj.rank = out.rank_dev ? out.rank_dev + k : nullptr;
        sj.normsq = normsq; sj.eps2_over_d = cfg.eps * cfg.eps / d; sj.rank_cap = R;
        svd_jacobi(c, {sj});
        double *Cn = (k == d - 1) ? out.core : c.arena->alloc(a * R * rest);
        Gemm g(c, "gemm_hosvd", all_tc);
        if (k == 0)
            g.add1(R, (int)rest, sk, 1, 0, W[k], sk, C, sk, Cn, R);
        else
            g.add1((int)a, R, sk, 0, 0, C, (int)a, W[k], sk, Cn, (int)a, 0.0, 1.0, nullptr, (int)rest,
                   a * sk, 0, a * R);
        g.run();
        C = Cn;
        cur[k] = R;
    }
    // 9. output factors U^_k W_k   (n_k x R), rotated back by Q_k when the terms were rotated
    {
        Gemm g(c, "gemm_factors", all_tc);
        double *tmp[TK_MAX_D];
        for (int k = 0; k < d; ++k) {
            tmp[k] = cfg.rot ? c.arena->alloc((size_t)pb.n[k] * R) : out.f[k];
            g.add1(pb.n[k], R, sr, 0, 0, Q[k], pb.n[k], W[k], sr, tmp[k], pb.n[k]);
        }
        g.run();
        if (cfg.rot) {
            Gemm g2(c, "gemm_rotate", all_tc);
            for (int k = 0; k < d; ++k)
                g2.add1(pb.n[k], R, pb.n[k], 0, 0, cfg.rot[k], pb.n[k], tmp[k], pb.n[k], out.f[k], pb.n[k]);
            g2.run();
        }
    }
}

// ------------------------------------------------------------------------------------------
// Exponential-sum preconditioner applied in the sine eigenbasis (Section 3.4: the DST-I of the
// factor matrices): E_h U = V diag(w_h) V^T U, so the 2q+1 terms of M(X) are, in the basis V,
// [c_h G; diag(w_h) V^T U_1, ...]: one product V^T U_k per mode and row scalings.
// ------------------------------------------------------------------------------------------
std::vector<TTerm> expsum_terms(Ctx &c, const Dims &pb, const ExpSumPC &es, const TTerm &x, bool tc) {
    const int d = pb.d;
    double *Uh[TK_MAX_D];
    {
        Gemm g(c, "gemm_sine", tc);
        for (int k = 0; k < d; ++k) {
            Uh[k] = c.arena->alloc((size_t)pb.n[k] * x.r[k]);
            g.add1(pb.n[k], x.r[k], pb.n[k], 1, 0, es.V[k], pb.n[k], x.f[k], pb.n[k], Uh[k], pb.n[k]);
        }
        g.run();
    }
    std::vector<TTerm> out(es.nh);
    std::vector<RowScaleJob> jobs;
    for (int h = 0; h < es.nh; ++h) {
        TTerm &T = out[h];
        T.core = x.core;
        T.coef = es.coef[h] * x.coef;
        T.coef_dev = x.coef_dev;
        for (int k = 0; k < d; ++k) {
            T.r[k] = x.r[k];
            double *f = c.arena->alloc((size_t)pb.n[k] * x.r[k]);
            jobs.push_back(RowScaleJob{Uh[k], es.w[k] + (size_t)h * pb.n[k], f, pb.n[k], x.r[k]});
            T.f[k] = f;
        }
    }
    row_scale(c, jobs);
    return out;
}

// ------------------------------------------------------------------------------------------
// Multilinear Nystrom (Algorithms 3-5)
// ------------------------------------------------------------------------------------------
// MLN_Sketch of a sum of terms, accumulated (MLN_Sum) into gpsi ((r+p)^d) and F_k (n_k x r):
//   G_Psi += c_i G^(i) x_k (Psi_k^T U_k^(i)),  F_k += c_i U_k^(i) MTTKRP(G^(i), {Ubar^T}, k)
void mln_sketch_sum(Ctx &c, const Dims &pb, const std::vector<TTerm> &terms, const double *const *psi,
                    int r, int p, double *gpsi, double *const *F, double beta, bool tc) {
    ScopedMark mark(*c.arena);
    const int d = pb.d, rp = r + p, N = (int)terms.size();
    // U_Psi,k^(i) = Psi_k^T U_k^(i)  ((r+p) x r_k); Ubar^T = first r rows, transposed on use
    std::vector<std::vector<const double *>> UP(N, std::vector<const double *>(d));
    {
        Gemm g(c, "gemm_mln");
        std::map<const double *, double *> made[TK_MAX_D];
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < d; ++k) {
                auto it = made[k].find(terms[i].f[k]);
                if (it != made[k].end()) { UP[i][k] = it->second; continue; }
                double *u = c.arena->alloc((size_t)rp * terms[i].r[k]);
                g.add1(rp, terms[i].r[k], pb.n[k], 1, 0, psi[k], pb.n[k], terms[i].f[k], pb.n[k], u, rp);
                made[k][terms[i].f[k]] = u;
                UP[i][k] = u;
            }
        g.run();
    }
    // sketched core: sum_i c_i G^(i) x_k U_Psi,k^(i) (mixed form: this TTM chain, the dominant
    // (r+p)^d work, on tensor cores; the factor contributions below, which MLN_Recovery applies
    // R^+ to, stay FP64)
    {
        TtmGroup G{};
        for (int k = 0; k < d; ++k) G.sdims[k] = rp;
        G.out = gpsi;
        G.beta = beta;
        for (int i = 0; i < N; ++i) {
            TtmJob J{};
            J.core = terms[i].core;
            for (int k = 0; k < d; ++k) { J.r[k] = terms[i].r[k]; J.P[k] = UP[i][k]; J.ldp[k] = rp; }
            J.coef = terms[i].coef;
            J.coef_dev = terms[i].coef_dev;
            G.jobs.push_back(J);
        }
        ttm_groups(c, d, {G}, tc);
    }
    // factor contributions: T_k^(i) = MTTKRP(G^(i), {Ubar_l^T}, k) (r_k x r); F_k = sum c_i U_k T_k
    // Ubar_l^T (r_l x r) is the transpose of the first r rows of U_Psi,l: materialise it.
    std::vector<std::vector<double *>> UbT(N, std::vector<double *>(d));
    {
        std::map<const double *, double *> made[TK_MAX_D];
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < d; ++k) {
                auto it = made[k].find(UP[i][k]);
                if (it != made[k].end()) { UbT[i][k] = it->second; continue; }
                double *u = c.arena->alloc((size_t)terms[i].r[k] * r);
                transpose_block(c, u, terms[i].r[k], UP[i][k], rp, r, terms[i].r[k]);
                made[k][UP[i][k]] = u;
                UbT[i][k] = u;
            }
    }
    std::vector<std::vector<double *>> T(N, std::vector<double *>(d));
    {
        std::vector<MttJob> mj;
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < d; ++k) {
                MttJob J{};
                J.core = terms[i].core;
                J.keep = k;
                for (int j = 0; j < d; ++j) { J.r[j] = terms[i].r[j]; J.P[j] = UbT[i][j]; J.ldp[j] = terms[i].r[j]; }
                T[i][k] = c.arena->alloc((size_t)terms[i].r[k] * r);
                J.out = T[i][k];
                mj.push_back(J);
            }
        mttkrp_batch(c, d, r, mj);
    }
    {
        Gemm g(c, "gemm_mln");
        for (int k = 0; k < d; ++k) {
            std::vector<Gemm::Seg> segs;
            for (int i = 0; i < N; ++i)
                segs.push_back(Gemm::Seg{terms[i].f[k], pb.n[k], T[i][k], terms[i].r[k], terms[i].r[k],
                                         terms[i].coef, terms[i].coef_dev});
            g.add(pb.n[k], r, 0, 0, F[k], pb.n[k], beta, segs);
        }
        g.run();
    }
}

// MLN_Recovery (Algorithm 5): Q_k R_k = qr(Psi_k^T F_k); U~_k = F_k R_k^+; G~ = G_Psi x_k Q_k^T
void mln_recovery(Ctx &c, const Dims &pb, const double *gpsi, const double *const *F,
                  const double *const *psi, int r, int p, const TOut &out, bool tc) {
    ScopedMark mark(*c.arena);
    const int d = pb.d, rp = r + p;
    double *PF[TK_MAX_D], *Qk[TK_MAX_D], *Rp[TK_MAX_D];
    {
        Gemm g(c, "gemm_mln");
        for (int k = 0; k < d; ++k) {
            PF[k] = c.arena->alloc((size_t)rp * r);
            g.add1(rp, r, pb.n[k], 1, 0, psi[k], pb.n[k], F[k], pb.n[k], PF[k], rp);
        }
        g.run();
    }
    {
        std::vector<QRJob> qj;
        for (int k = 0; k < d; ++k) {
            Qk[k] = c.arena->alloc((size_t)rp * r);
            qj.push_back(QRJob{PF[k], c.arena->alloc(r), Qk[k], rp, r, nullptr});
        }
        qr_householder(c, qj);
    }
    {
        const double *Rs[TK_MAX_D];
        int ld[TK_MAX_D];
        for (int k = 0; k < d; ++k) {
            Rp[k] = c.arena->alloc((size_t)r * r);
            Rs[k] = PF[k];
            ld[k] = rp;
        }
        pinv_small(c, Rs, ld, r, Rp, d, r * 0x1p-52);
    }
    {
        Gemm g(c, "gemm_mln");
        for (int k = 0; k < d; ++k) g.add1(pb.n[k], r, r, 0, 0, F[k], pb.n[k], Rp[k], r, out.f[k], pb.n[k]);
        g.run();
    }
    {
        TtmGroup G{};
        for (int k = 0; k < d; ++k) G.sdims[k] = r;
        G.out = out.core;
        G.beta = 0.0;
        TtmJob J{};
        J.core = gpsi;
        for (int k = 0; k < d; ++k) {
            J.r[k] = rp;
            // Q_k^T (r x (r+p)) as the TTM matrix: materialise the transpose
            double *qt = c.arena->alloc((size_t)r * rp);
            transpose_block(c, qt, r, Qk[k], rp, rp, r);
            J.P[k] = qt;
            J.ldp[k] = r;
        }
        J.coef = 1.0;
        G.jobs.push_back(J);
        ttm_groups(c, d, {G});
    }
}

}  // namespace tk
