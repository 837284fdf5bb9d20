// Small dense FP64 linear algebra of the RoundSum and least-squares steps:
//  * Householder QR of a tall-skinny matrix (the range finder's economy QR, Section 3.1;
//    the QR of a core unfolding inside ST-HOSVD; MLN_Recovery's QR, Algorithm 5).  One
//    thread-block cluster per matrix; the rows are split across the cluster's CTAs and each
//    reflector's two reductions go through distributed shared memory in fixed rank order.
//  * One-sided (Hestenes) Jacobi SVD of a small square matrix, one CTA per matrix, used for
//    the ST-HOSVD truncation (left singular vectors of the unfolding) and for R^+ in
//    MLN_Recovery.
//  * Incremental Householder least squares for y_k = argmin ||M y - b_s|| (Algorithm 2).
#include <cooperative_groups.h>

#include <algorithm>

#include "tk_internal.cuh"

namespace cg = cooperative_groups;

namespace tk {

constexpr int QR_MAXS = 256;
constexpr int SVD_MAXS = 112;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block, result returned to every thread.  `scratch` holds >= 33 doubles.
__device__ double block_sum(double v, double *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += scratch[w];
    return t;
}

// Householder vector in LAPACK dlarfg form: given alpha and sigma2 = ||x||^2 of the part
// below, returns tau, beta (new diagonal) and the scale 1 / (alpha - beta) for v.
__device__ __forceinline__ void householder(double alpha, double sigma2, double &tau, double &beta,
                                            double &scal) {
    if (sigma2 == 0.0) {
        tau = 0.0;
        beta = alpha;
        scal = 0.0;
        return;
    }
    const double nrm = sqrt(alpha * alpha + sigma2);
    beta = alpha >= 0.0 ? -nrm : nrm;
    tau = (beta - alpha) / beta;
    scal = 1.0 / (alpha - beta);
}

// ------------------------------------------------------------------------------------------
// Cluster Householder QR
// ------------------------------------------------------------------------------------------
struct QRJobs {
    int n;
    QRJob j[TK_MAX_D];
};

__global__ void __launch_bounds__(256) k_qr(const __grid_constant__ QRJobs jobs) {
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int q = (int)cl.block_rank();
    const QRJob &J = jobs.j[blockIdx.y];
    const int m = J.m, s = J.s, kmax = min(m, s);
    const int rb = (m + C - 1) / C;
    const int r0 = min(m, q * rb), r1 = min(m, r0 + rb);
    double *A = J.A;

    __shared__ double red[2][QR_MAXS + 2];
    __shared__ double wsum[QR_MAXS + 2];
    __shared__ double taus[QR_MAXS];
    __shared__ double scratch[40];
    __shared__ double bc[4];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    int buf = 0;
    for (int j = 0; j < kmax; ++j) {
        double ps = 0.0;
        for (int i = max(r0, j + 1) + tid; i < r1; i += blockDim.x) {
            const double v = A[i + (long long)j * m];
            ps = fma(v, v, ps);
        }
        ps = block_sum(ps, scratch);
        if (tid == 0) {
            red[buf][0] = ps;
            red[buf][1] = (j >= r0 && j < r1) ? A[j + (long long)j * m] : 0.0;
        }
        cl.sync();
        if (tid == 0) {
            double s2 = 0.0, al = 0.0;
            for (int qq = 0; qq < C; ++qq) {
                s2 += cl.map_shared_rank(&red[buf][0], qq)[0];
                al += cl.map_shared_rank(&red[buf][1], qq)[0];
            }
            double tau, beta, scal;
            householder(al, s2, tau, beta, scal);
            bc[0] = tau;
            bc[1] = scal;
            bc[2] = beta;
            taus[j] = tau;
        }
        buf ^= 1;
        __syncthreads();
        const double tau = bc[0], scal = bc[1], beta = bc[2];
        for (int i = max(r0, j + 1) + tid; i < r1; i += blockDim.x) A[i + (long long)j * m] *= scal;
        if (tid == 0 && j >= r0 && j < r1) A[j + (long long)j * m] = beta;
        __syncthreads();
        if (tau == 0.0) continue;   // uniform across the cluster
        const int ib = max(r0, j);
        for (int c = j + 1 + warp; c < s; c += nw) {
            double p = 0.0;
            for (int i = ib + lane; i < r1; i += 32) {
                const double v = (i == j) ? 1.0 : A[i + (long long)j * m];
                p = fma(v, A[i + (long long)c * m], p);
            }
            p = warp_sum(p);
            if (lane == 0) red[buf][c] = p;
        }
        cl.sync();
        for (int c = j + 1 + tid; c < s; c += blockDim.x) {
            double w = 0.0;
            for (int qq = 0; qq < C; ++qq) w += cl.map_shared_rank(&red[buf][c], qq)[0];
            wsum[c] = w * tau;
        }
        buf ^= 1;
        __syncthreads();
        const int nrows = r1 - ib, ncols = s - j - 1;
        if (nrows > 0) {
            for (int e = tid; e < nrows * ncols; e += blockDim.x) {
                const int i = ib + e % nrows, c = j + 1 + e / nrows;
                const double v = (i == j) ? 1.0 : A[i + (long long)j * m];
                A[i + (long long)c * m] -= v * wsum[c];
            }
        }
        __syncthreads();
    }
    if (J.tau && q == 0)
        for (int j = tid; j < kmax; j += blockDim.x) J.tau[j] = taus[j];
    if (J.Q) {
        double *Q = J.Q;
        const int nr = r1 - r0;
        for (int e = tid; e < nr * s; e += blockDim.x) {
            const int i = r0 + e % nr, c = e / nr;
            Q[i + (long long)c * m] = (i == c) ? 1.0 : 0.0;
        }
        __syncthreads();
        for (int j = kmax - 1; j >= 0; --j) {
            const double tau = taus[j];
            if (tau == 0.0) continue;
            const int ib = max(r0, j);
            for (int c = j + warp; c < s; c += nw) {
                double p = 0.0;
                for (int i = ib + lane; i < r1; i += 32) {
                    const double v = (i == j) ? 1.0 : A[i + (long long)j * m];
                    p = fma(v, Q[i + (long long)c * m], p);
                }
                p = warp_sum(p);
                if (lane == 0) red[buf][c] = p;
            }
            cl.sync();
            for (int c = j + tid; c < s; c += blockDim.x) {
                double w = 0.0;
                for (int qq = 0; qq < C; ++qq) w += cl.map_shared_rank(&red[buf][c], qq)[0];
                wsum[c] = w * tau;
            }
            buf ^= 1;
            __syncthreads();
            const int nrows = r1 - ib, ncols = s - j;
            if (nrows > 0) {
                for (int e = tid; e < nrows * ncols; e += blockDim.x) {
                    const int i = ib + e % nrows, c = j + e / nrows;
                    const double v = (i == j) ? 1.0 : A[i + (long long)j * m];
                    Q[i + (long long)c * m] -= v * wsum[c];
                }
            }
            __syncthreads();
        }
    }
    cl.sync();   // keep this CTA's shared memory alive until every peer finished reading it
}

void qr_householder(Ctx &c, const std::vector<QRJob> &jobs) {
    if (jobs.empty()) return;
    for (size_t base = 0; base < jobs.size(); base += TK_MAX_D) {
        QRJobs J{};
        J.n = (int)std::min<size_t>(TK_MAX_D, jobs.size() - base);
        int mmax = 0;
        for (int i = 0; i < J.n; ++i) {
            J.j[i] = jobs[base + i];
            TK_REQUIRE(J.j[i].s <= QR_MAXS, "QR: more than 256 columns");
            mmax = std::max(mmax, J.j[i].m);
        }
        // cluster size: enough rows per CTA to amortise the per-step cluster barriers
        int C = 1;
        while (C < 8 && mmax / (C * 2) >= 32) C *= 2;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)C, (unsigned)J.n, 1);
        cfg.blockDim = dim3(256, 1, 1);
        cfg.stream = c.st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        TK_CUDA(cudaLaunchKernelEx(&cfg, k_qr, J));
        c.check_launch("qr");
    }
}

// ------------------------------------------------------------------------------------------
// One-sided Jacobi SVD of a small square matrix (one CTA each)
// ------------------------------------------------------------------------------------------
struct SVDJobs {
    int n;
    SVDJob j[TK_MAX_D];
    double *pinv[TK_MAX_D];   // optional s x s pseudo-inverse outputs
    double rcond;
};

__global__ void __launch_bounds__(512) k_svd(const __grid_constant__ SVDJobs jobs) {
    extern __shared__ double sm[];
    const SVDJob &J = jobs.j[blockIdx.x];
    const int s = J.s;
    double *A = sm;
    double *V = sm + s * s;
    __shared__ double sig[SVD_MAXS];
    __shared__ int order[SVD_MAXS];
    __shared__ int rotated;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int e = tid; e < s * s; e += blockDim.x) {
        const int i = e % s, c = e / s;
        A[e] = (i <= c && i < J.ldr) ? J.R[i + (long long)c * J.ldr] : 0.0;
        V[e] = (i == c) ? 1.0 : 0.0;
    }
    const int sp = s + (s & 1);
    const double tol = 1e-15;
    __syncthreads();
    for (int sweep = 0; sweep < 40 && sp > 1; ++sweep) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int round = 0; round < sp - 1; ++round) {
            for (int pr = warp; pr < sp / 2; pr += nw) {
                int p, qq;
                if (pr == 0) { p = round; qq = sp - 1; }
                else { p = (round + pr) % (sp - 1); qq = (round - pr + (sp - 1)) % (sp - 1); }
                if (p >= s || qq >= s) continue;
                if (p > qq) { const int t = p; p = qq; qq = t; }
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = lane; i < s; i += 32) {
                    const double a = A[i + p * s], b = A[i + qq * s];
                    al = fma(a, a, al);
                    be = fma(b, b, be);
                    ga = fma(a, b, ga);
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                if (ga != 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
                    const double zeta = (be - al) / (2.0 * ga);
                    const double t = copysign(1.0, zeta) / (fabs(zeta) + hypot(1.0, zeta));
                    const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                    for (int i = lane; i < s; i += 32) {
                        const double a = A[i + p * s], b = A[i + qq * s];
                        A[i + p * s] = cs * a - sn * b;
                        A[i + qq * s] = sn * a + cs * b;
                        const double va = V[i + p * s], vb = V[i + qq * s];
                        V[i + p * s] = cs * va - sn * vb;
                        V[i + qq * s] = sn * va + cs * vb;
                    }
                    if (lane == 0) rotated = 1;
                }
            }
            __syncthreads();
        }
        const int any = rotated;
        __syncthreads();
        if (!any) break;
    }
    // singular values and descending order (ties by index)
    for (int c = warp; c < s; c += nw) {
        double t = 0.0;
        for (int i = lane; i < s; i += 32) t = fma(A[i + c * s], A[i + c * s], t);
        t = warp_sum(t);
        if (lane == 0) sig[c] = sqrt(t);
    }
    __syncthreads();
    for (int c = tid; c < s; c += blockDim.x) {
        int pos = 0;
        for (int o = 0; o < s; ++o)
            if (sig[o] > sig[c] || (sig[o] == sig[c] && o < c)) ++pos;
        order[pos] = c;
    }
    __syncthreads();
    __shared__ int kept;
    if (tid == 0) {
        int r = min(s, J.rank_cap);
        if (J.normsq) {
            const double thr = J.eps2_over_d * (*J.normsq);
            double tail = 0.0;
            int rr = s;
            // smallest rr with sum_{pos >= rr} sig^2 <= thr
            for (int pos = s - 1; pos >= 1; --pos) {
                const double v = sig[order[pos]];
                tail += v * v;
                if (tail <= thr) rr = pos; else break;
            }
            r = min(rr, J.rank_cap);
        }
        r = max(r, 1);
        kept = r;
        if (J.rank) *J.rank = r;
    }
    __syncthreads();
    const int r = kept;
    if (J.sigma)
        for (int c = tid; c < s; c += blockDim.x) J.sigma[c] = sig[order[c]];
    if (J.W)
        for (int e = tid; e < s * J.wcols; e += blockDim.x) {
            const int i = e % s, c = e / s;
            J.W[e] = (c < r) ? V[i + order[c] * s] : 0.0;
        }
    double *P = jobs.pinv[blockIdx.x];
    if (P) {
        // R = U S V^T with U S = A (final);  R^+ = sum_c V[:,c] A[:,c]^T / sig_c^2
        const double smax = sig[order[0]];
        const double cut = jobs.rcond * smax;
        for (int e = tid; e < s * s; e += blockDim.x) {
            const int i = e % s, jj = e / s;
            double t = 0.0;
            for (int c = 0; c < s; ++c) {
                const double sc = sig[c];
                if (sc > cut && sc > 0.0) t += V[i + c * s] * A[jj + c * s] / (sc * sc);
            }
            P[i + (long long)jj * s] = t;
        }
    }
}

static void svd_launch(Ctx &c, SVDJobs &J, int smax) {
    const size_t smem = 2 * (size_t)smax * smax * sizeof(double);
    static bool attr_set = false;
    if (!attr_set) {
        TK_CUDA(cudaFuncSetAttribute(k_svd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     2 * SVD_MAXS * SVD_MAXS * (int)sizeof(double)));
        attr_set = true;
    }
    k_svd<<<J.n, 512, smem, c.st>>>(J);
    c.check_launch("svd");
}

void svd_jacobi(Ctx &c, const std::vector<SVDJob> &jobs) {
    for (size_t base = 0; base < jobs.size(); base += TK_MAX_D) {
        SVDJobs J{};
        J.n = (int)std::min<size_t>(TK_MAX_D, jobs.size() - base);
        int smax = 1;
        for (int i = 0; i < J.n; ++i) {
            J.j[i] = jobs[base + i];
            TK_REQUIRE(J.j[i].s <= SVD_MAXS && J.j[i].s >= 1, "SVD: size must be 1..112");
            smax = std::max(smax, J.j[i].s);
            J.pinv[i] = nullptr;
        }
        J.rcond = 0.0;
        svd_launch(c, J, smax);
    }
}

// Pseudo-inverse of small square matrices through the Jacobi SVD (MLN_Recovery's R^+).
void pinv_small(Ctx &c, const double *const *R, const int *ldr, int s, double *const *out, int n,
                double rcond) {
    SVDJobs J{};
    J.n = n;
    for (int i = 0; i < n; ++i) {
        SVDJob &j = J.j[i];
        j.R = R[i]; j.ldr = ldr[i]; j.s = s; j.W = nullptr; j.wcols = 0; j.sigma = nullptr;
        j.rank = nullptr; j.normsq = nullptr; j.eps2_over_d = 0.0; j.rank_cap = s;
        J.pinv[i] = out[i];
    }
    J.rcond = rcond;
    TK_REQUIRE(s <= SVD_MAXS, "pinv: size must be <= 112");
    svd_launch(c, J, s);
}

// ------------------------------------------------------------------------------------------
// Incremental Householder least squares (one CTA)
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_ls(const double *M, const double *b, int s, int c0, int k,
                                            LSState st, int init_qtb) {
    __shared__ double scratch[40];
    __shared__ double bc[4];
    const int tid = threadIdx.x, nt = blockDim.x;
    double *H = st.H;
    if (init_qtb)
        for (int i = tid; i < s; i += nt) st.qtb[i] = b[i];
    for (int col = c0; col < k; ++col) {
        double *h = H + (long long)col * s;
        for (int i = tid; i < s; i += nt) h[i] = M[i + (long long)col * s];
        __syncthreads();
        for (int j = 0; j < col; ++j) {
            const double *v = H + (long long)j * s;
            double p = 0.0;
            for (int i = j + tid; i < s; i += nt) p = fma(i == j ? 1.0 : v[i], h[i], p);
            p = block_sum(p, scratch);
            const double f = st.tau[j] * p;
            for (int i = j + tid; i < s; i += nt) h[i] -= (i == j ? 1.0 : v[i]) * f;
            __syncthreads();
        }
        double p = 0.0;
        for (int i = col + 1 + tid; i < s; i += nt) p = fma(h[i], h[i], p);
        p = block_sum(p, scratch);
        if (tid == 0) {
            double tau, beta, scal;
            householder(h[col], p, tau, beta, scal);
            bc[0] = tau; bc[1] = scal; bc[2] = beta;
            st.tau[col] = tau;
        }
        __syncthreads();
        const double tau = bc[0], scal = bc[1], beta = bc[2];
        for (int i = col + 1 + tid; i < s; i += nt) h[i] *= scal;
        __syncthreads();
        if (tid == 0) h[col] = beta;
        // apply the new reflector to Q^T b
        double q = 0.0;
        for (int i = col + tid; i < s; i += nt) q = fma(i == col ? 1.0 : h[i], st.qtb[i], q);
        __syncthreads();
        q = block_sum(q, scratch);
        const double f = tau * q;
        for (int i = col + tid; i < s; i += nt) st.qtb[i] -= (i == col ? 1.0 : h[i]) * f;
        __syncthreads();
    }
    // back substitution R y = (Q^T b)[0:k], column oriented; y holds the running rhs
    for (int i = tid; i < k; i += nt) st.y[i] = st.qtb[i];
    __syncthreads();
    for (int j = k - 1; j >= 0; --j) {
        if (tid == 0) {
            const double rjj = H[j + (long long)j * s];
            st.y[j] = rjj != 0.0 ? st.y[j] / rjj : 0.0;
        }
        __syncthreads();
        const double yj = st.y[j];
        for (int i = tid; i < j; i += nt) st.y[i] -= H[i + (long long)j * s] * yj;
        __syncthreads();
    }
    double r = 0.0;
    for (int i = k + tid; i < s; i += nt) r = fma(st.qtb[i], st.qtb[i], r);
    r = block_sum(r, scratch);
    if (tid == 0) *st.res = sqrt(r);
}

void ls_update(Ctx &c, const double *M, const double *b, int s, int c0, int k, const LSState &st,
               int init_qtb) {
    TK_REQUIRE(s >= 1 && s <= 4096 && k >= 1 && k < s + 1, "least squares: bad size");
    k_ls<<<1, 512, 0, c.st>>>(M, b, s, c0, k, st, init_qtb);
    c.check_launch("ls");
}

}  // namespace tk
