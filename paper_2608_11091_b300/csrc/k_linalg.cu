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

#include <atomic>
#include <type_traits>

#include "tk_internal.cuh"

namespace cg = cooperative_groups;

namespace tk {

constexpr int QR_MAXS = 256;
constexpr int SVD_MAXS = 96;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block, result returned to every thread.  `scratch` holds >= 33 doubles.  The
// warp partials are combined once by warp 0 (an FP64 warp instruction costs the same whatever
// its lanes hold, so every thread re-adding them would cost nw times as much).
__device__ double block_sum(double v, double *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < nw ? scratch[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) scratch[32] = t;
    }
    __syncthreads();
    return scratch[32];
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
    // with G > 1 clusters per job (n = 1): every CTA's exchange slot in global memory, two per CTA
    // (by exchange parity), each xs values of two tagged words (zeroed before the launch)
    int xs;
    // receive area in dynamic shared memory: [2 parities][C senders][rxs] doubles from rx_off
    int rx_off, rxs;
    // self-test of the bounded waits (0 in every solve): 1 = cluster 0 expects 8 bytes more than
    // its peers push at the first exchange, 2 = CTA 0 does not publish the first exchange to the
    // other clusters; the waiting CTAs run out their limit, set g_qr_error and finish
    int inject;
    unsigned long long *xw[TK_MAX_D];
};
constexpr int QR_GMAX = 3;
constexpr int QR_DSMEM = 200 * 1024;   // dynamic shared memory of a QR CTA at most (rows + receive area)
// bounded waits of the cross-cluster exchange (a step takes ~10 us; the limit is ~0.1 s or more),
// after which g_qr_error is set and the kernel carries on with zeros for the missing sums
__device__ int g_qr_error;
constexpr long QR_SPIN = 1L << 18;
// A value crosses clusters as two 64-bit words, each a 32-bit half of the double under the
// 32-bit exchange number X: an aligned 64-bit access is single-copy atomic, so a reader that
// sees X in both words holds the value of exchange X, with no flag, fence or second round trip
// (slots start zeroed and X >= 1).
__device__ __forceinline__ void xw_put(unsigned long long *w, double v, unsigned X) {
    const unsigned long long t = (unsigned long long)X << 32;
    const unsigned long long a = t | (unsigned)__double2loint(v), b = t | (unsigned)__double2hiint(v);
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(w), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void xw_load(const unsigned long long *w, unsigned long long &a, unsigned long long &b) {
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(w) : "memory");
}
__device__ __forceinline__ bool xw_ok(unsigned long long a, unsigned long long b, unsigned X) {
    return (unsigned)(a >> 32) == X && (unsigned)(b >> 32) == X;
}
__device__ __forceinline__ double xw_val(unsigned long long a, unsigned long long b) {
    return __hiloint2double((int)(unsigned)b, (int)(unsigned)a);
}
// Inside a cluster a CTA pushes its exchange buffer into every peer's shared memory with
// st.async, each store counted (in bytes) on the peer's mbarrier of that exchange's parity; the
// receiver posts the bytes it expects and waits for the phase, so no cluster barrier or remote
// load is on a step's path.  An mbarrier's transaction count may run below zero while stores
// land before the expectation is posted; the phase cannot complete before the receiver's arrive.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned cluster_addr(unsigned a, int rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void push2(unsigned dst, double a, double b, unsigned mb) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];"
                 ::"r"(dst), "d"(a), "d"(b), "r"(mb) : "memory");
}
__device__ __forceinline__ void push1(unsigned dst, double a, unsigned mb) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];"
                 ::"r"(dst), "d"(a), "r"(mb) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned mb, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
}
// waits for the phase of the given parity, suspended at most ~1 us per call
__device__ __forceinline__ bool mbar_try(unsigned mb, unsigned parity) {
    unsigned ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok) : "r"(mb), "r"(parity), "r"(1000) : "memory");
    return ok != 0;
}
int qr_error_flag(bool reset) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_qr_error, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (reset && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_qr_error, &z, sizeof(int));
    }
    return v;
}

// One reflector per step, one cluster-wide exchange per step.  With x = A[j:, j], alpha = x_0,
// sigma2 = ||x_1:||^2, nrm = (alpha^2 + sigma2)^(1/2), beta = -sign(alpha) nrm, the reflector
// is LAPACK's H = I - tau v v^T, v = (x - beta e_0) / (alpha - beta) (v_0 = 1), tau =
// (beta - alpha) / beta in [1, 2].  (The unnormalised v = x - beta e_0 would need
// tau = 1 / (nrm (nrm + |alpha|)), which overflows once the columns left after an exact
// low-rank block are rounding noise and each step shrinks them further.)  For every trailing
// column c, v^T A[j:, c] = P_c + (D_c - alpha P_c) / (alpha - beta) with D_c = x^T A[j:, c] and
// P_c = A[j, c], so a step needs, from every CTA over its own rows, the partial sigma2 and
// D_c, and from the CTA owning row j its row (alpha, P_c): one exchange per step (below).  On this part an FP64 warp instruction holds an
// SMSP's FP64 pipe for ~64 cycles whatever the active lanes, so the scalar work is kept off
// the FP64 pipe where it can be: pivoting (largest remaining norm first) uses FP32 norms,
// scaled once by the largest initial column norm and downdated by the new row of R each step
// (a pivot only has to grade R, it does not enter the result); the argmax is one warp of
// FP32 shuffles; peer sums use two or four threads per column.
// The two FP64 passes of a step (partial sums D_c, trailing update) cost one FP64 FMA per element
// and run at the FP64 pipe's rate only if every warp carries the same number of them with all
// lanes active: the CTA's (column, row) elements are split into equal contiguous ranges, one per
// thread, in column-major order (odd range length, so that the lanes of a warp fall on distinct
// banks), walked as two independent streams (the two halves) with one uniform trip count, so
// that a column change inside a range costs no partially active FP64 instruction.  A stream's
// partial sum of a column goes to its half of slot (thread + column) of `pp`; the slots of a
// column's contributors (the threads whose ranges meet it, a contiguous run) are added in thread
// order, by one thread when there are at most 8, else by a warp.  The kernel leaves R and the
// reflectors; qr_form_q builds an explicit Q from them.
// Rows live in shared memory when they fit (SMEM = true), else in global memory.  On one
// cluster the peers' exchange buffers are read through distributed shared memory after a cluster
// barrier; the buffers alternate by a running exchange count, so a buffer is rewritten only after
// every peer has passed the next barrier.  A tall single unfolding runs on G <= 3 clusters: each
// CTA pushes its exchange buffer into its cluster peers' receive areas (st.async counted on an
// mbarrier per exchange parity), writes it to a global slot as tagged words (xw_put) for the
// other clusters, and reads all of them locally or from the slots.  A receive area or slot of
// exchange X is rewritten at X + 2, which no CTA reaches before every CTA has read X (it needs
// every CTA's sums of X + 1, formed after reading X).
constexpr int QR_THREADS = 256;
template <bool SMEM, int G>
__global__ void __launch_bounds__(QR_THREADS, 1) k_qr(const __grid_constant__ QRJobs jobs, int rb_cap) {
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int q = (int)cl.block_rank();
    const int g = (int)blockIdx.x / C, qg = (int)blockIdx.x;   // cluster, CTA over the job
    const QRJob &J = jobs.j[blockIdx.y];
    const int m = J.m, s = J.s, kmax = min(m, s);
    const int rb = (m + G * C - 1) / (G * C);
    const int r0 = min(m, qg * rb), r1 = min(m, r0 + rb), nr = r1 - r0;
    extern __shared__ __align__(16) double dyn[];
    double *Al = dyn;                              // nr x s, ld rb_cap
    // the exchange inside the cluster: pushes into the peers' receive areas (several clusters:
    // the barrier's latency would add to the other clusters' round trip), or one cluster barrier
    // and distributed-shared-memory loads of the peers' buffers (one cluster: ncu 400 vs 420 us
    // for the range finder's 1024 x 69 QRs, pushes 616 vs 630 us for the 4761 x 69 unfolding on
    // three clusters)
    constexpr bool PUSH = G > 1;
    double *const rx = dyn + jobs.rx_off;          // [2][C][rxs]: the peers' exchange buffers
    __shared__ __align__(8) unsigned long long mbar[2];   // one per exchange parity
    __shared__ double red[2][2 * QR_MAXS];         // [0, nc1): partial sums, [nc1, 2 nc1): owner's row
    __shared__ double wv[QR_MAXS];
    __shared__ double prow[QR_MAXS];               // owner's row j of the step (local copy)
    __shared__ double taus[QR_MAXS];
    __shared__ float nrmf[QR_MAXS];
    __shared__ int permv[QR_MAXS];
    __shared__ double bc[4];
    __shared__ double pp[2 * (QR_THREADS + QR_MAXS)];  // per-thread partial sums (two per slot thread + column)
    __shared__ int pivot;
    const bool piv = J.perm != nullptr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    auto A = [&](int i, int c) -> double & {
        return SMEM ? Al[(i - r0) + (size_t)c * rb_cap] : J.A[i + (long long)c * m];
    };
    if (SMEM)
        for (int e = tid; e < nr * s; e += nt) {
            const int i = r0 + e % nr, c = e / nr;
            A(i, c) = J.A[i + (long long)c * m];
        }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cl.sync();     // every peer's mbarriers initialised before the first push
    int xch = 0;   // exchanges so far (selects the buffer)
    bool xgive = false;   // this thread gave up a wait (the error flag is set; results are void)
    // the exchange buffer that CTA `from` (cluster rank) pushed here for exchange parity P
    auto rxb = [&](int P, int from) { return rx + (size_t)(P * C + from) * jobs.rxs; };
    // entry e of cluster peer `peer`'s exchange buffer of exchange X (own: rd): pushed here
    // (PUSH), else read through distributed shared memory after the cluster barrier
    auto peer_val = [&](const double *rd, int X, int peer, int e) -> double {
        if (PUSH) return peer == q ? rd[e] : rxb(X & 1, peer)[e];
        return cl.map_shared_rank(rd, peer)[e];
    };
    // threads of a pass: a short pass (at most 3200 elements: small unfoldings, the last steps)
    // is bound by its combine and latency rather than the FP64 pipe, so it takes four warps (one
    // per sub-partition) and leaves each column half as many partial sums to combine
    auto pass_threads = [&](int T) { return T > 3200 ? nt : min(nt, 128); };
    // the column sums out[cc] from the partials in pp (slot thread + column, two halves); ends
    // with out[] visible to the CTA
    auto combine = [&](int T, int nrows, int E, int nc, double *out) {
        // the partials of column cc are pp[2 (tlo + cc) .. 2 (thi + cc) + 1]: up to 8 contributors
        // one thread adds them in order; more (the last steps, few columns) go to a group of L
        // lanes each, strided over them and a shuffle tree, with L chosen so that every warp takes
        // its columns in one round (one column per warp at a time cost up to ~3k cycles a step)
        const int ncmax = T > 0 ? (nrows + E - 2) / E + 1 : 0;
        if (ncmax <= 8) {
            for (int cc = tid; cc < nc; cc += nt) {
                double acc = 0.0;
                if (T > 0) {
                    const int tlo = (cc * nrows) / E, thi = ((cc + 1) * nrows - 1) / E;
                    for (int t = tlo; t <= thi; ++t) acc += pp[2 * (t + cc)] + pp[2 * (t + cc) + 1];
                }
                out[cc] = acc;
            }
        } else {
            const int nw = nt >> 5, cpw = (nc + nw - 1) / nw;   // columns per warp
            const int L = cpw <= 1 ? 32 : cpw <= 2 ? 16 : cpw <= 4 ? 8 : cpw <= 8 ? 4 : 2;
            const int gpw = 32 / L, grp = lane / L, gl = lane & (L - 1);
            for (int base = warp * gpw; base < nc; base += nw * gpw) {   // warp-uniform trip count
                const int cc = base + grp;
                double acc = 0.0;
                if (cc < nc) {
                    const int tlo = (cc * nrows) / E, thi = ((cc + 1) * nrows - 1) / E;
                    const int b0 = 2 * (tlo + cc), nv = 2 * (thi - tlo + 1);
                    for (int k = gl; k < nv; k += L) acc += pp[b0 + k];
                }
                for (int o = L >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (cc < nc && gl == 0) out[cc] = acc;
            }
        }
        __syncthreads();
    };
    // sum over rows [ib, r1) of x * y for columns cc = 0 .. nc - 1 into out[cc], where
    // xy(i, cc, x, y) gives the two factors of element (i, cc); ends with out[] complete and
    // visible to the whole CTA.  Every thread runs the same trip count (all but the last few), so
    // the FMAs issue with full warps; a column change stores the two partial chains (no FP64
    // instruction on the divergent path) and the combine adds them.
    auto flat_sums = [&](int ib, int nc, auto xy, double *out) {
        const int nrows = r1 - ib;
        const int T = nrows > 0 ? nrows * nc : 0;
        const int na = pass_threads(T);
        const int E = T > 0 ? (((T + na - 1) / na) | 1) : 1;
        const int e0 = tid < na ? min(T, tid * E) : T, cnt = min(T, e0 + E) - e0;
        if (cnt > 0) {
            // two streams over the two halves of the range; stream A's partial of a column goes
            // to pp[2 (tid + cc)], stream B's to pp[2 (tid + cc) + 1] (both zeroed first: a column
            // may be met by one stream only)
            const int h = cnt >> 1;
            const int cf = e0 / nrows, cl_ = (e0 + cnt - 1) / nrows;
            for (int cc = cf; cc <= cl_; ++cc) {
                pp[2 * (tid + cc)] = 0.0;
                pp[2 * (tid + cc) + 1] = 0.0;
            }
            int cA = cf, iA = ib + (e0 - cA * nrows);
            int cB = (e0 + h) / nrows, iB = ib + (e0 + h - cB * nrows);
            double sA = 0.0, sB = 0.0;
            for (int k = 0; k < h; ++k) {
                double xa, ya, xb, yb;
                xy(iA, cA, xa, ya);
                xy(iB, cB, xb, yb);
                sA = fma(xa, ya, sA);
                sB = fma(xb, yb, sB);
                if (++iA == r1) { pp[2 * (tid + cA)] = sA; sA = 0.0; iA = ib; ++cA; }
                if (++iB == r1) { pp[2 * (tid + cB) + 1] = sB; sB = 0.0; iB = ib; ++cB; }
            }
            if (cnt & 1) {                                          // the last element: stream B's next
                double xb, yb;
                xy(iB, cB, xb, yb);
                sB = fma(xb, yb, sB);
                if (++iB == r1) { pp[2 * (tid + cB) + 1] = sB; sB = 0.0; iB = ib; ++cB; }
            }
            if (iA != ib) pp[2 * (tid + cA)] = sA;                  // stream A ended inside column cA
            if (iB != ib) pp[2 * (tid + cB) + 1] = sB;
        }
        __syncthreads();
        combine(T, nrows, E, nc, out);
    };
    // M(i, c0 + cc) -= v(i) * wc[cc] for rows [ib, r1), cc = 0 .. nc - 1 (M = A or Q); one
    // uniform loop per thread as in flat_sums
    auto flat_update = [&](int ib, int c0, int nc, auto v, const double *wc, auto M) {
        const int nrows = r1 - ib;
        const int T = nrows > 0 ? nrows * nc : 0;
        if (T == 0) return;
        const int E = ((T + nt - 1) / nt) | 1;
        const int e0 = min(T, tid * E), cnt = min(T, e0 + E) - e0;
        // two independent streams over the two halves of the range, loads issued before the
        // stores in each iteration (the compiler cannot reorder them across a store itself)
        const int h = cnt >> 1;
        int cA = e0 / nrows, iA = ib + (e0 - cA * nrows);
        int cB = (e0 + h) / nrows, iB = ib + (e0 + h - cB * nrows);
        double wA = h > 0 ? wc[cA] : 0.0, wB = cnt > h ? wc[cB] : 0.0;
        for (int k = 0; k < h; ++k) {
            double &a = M(iA, c0 + cA), &b = M(iB, c0 + cB);
            const double va = v(iA), vb = v(iB), xa = a, xb = b;
            a = fma(-va, wA, xa);
            b = fma(-vb, wB, xb);
            if (++iA == r1) { iA = ib; ++cA; wA = wc[cA]; }      // cA stays < nc: stream A ends at e0 + h
            if (++iB == r1) { iB = ib; ++cB; if (k + 1 < h || (cnt & 1)) wB = wc[cB]; }
        }
        if (cnt & 1) {                                          // the last element: stream B's next
            double &b = M(iB, c0 + cB);
            b = fma(-v(iB), wB, b);
        }
    };
    // Step j's trailing update and step j + 1's partial sums in one pass over rows [ib, r1) and
    // positions c = j + 1 + cc, cc = 0 .. nc - 1: position j + 1 holds the next column x (already
    // reflected; its element only adds x_i^2 for i > j + 1, the sigma2 part), every other position
    // takes a' = a - v_i w_c (v_j = 1) and adds x_i a' for i >= j + 1 (D_c part).  Two FP64 FMAs
    // per element, both streams' loads issued before their stores; partials and combine as in
    // flat_sums, the combine writing out[cc].
    auto fused_pass = [&](int j, int p, int ib, int nc, double *out) {
        const int nrows = r1 - ib;
        const int T = nrows > 0 ? nrows * nc : 0;
        const int na = pass_threads(T);
        const int E = T > 0 ? (((T + na - 1) / na) | 1) : 1;
        const int e0 = tid < na ? min(T, tid * E) : T, cnt = min(T, e0 + E) - e0;
        const int c0 = j + 1;
        if (cnt > 0) {
            const int h = cnt >> 1;
            const int cf = e0 / nrows, cl_ = (e0 + cnt - 1) / nrows;
            for (int cc = cf; cc <= cl_; ++cc) {
                pp[2 * (tid + cc)] = 0.0;
                pp[2 * (tid + cc) + 1] = 0.0;
            }
            int cA = cf, iA = ib + (e0 - cA * nrows);
            int cB = (e0 + h) / nrows, iB = ib + (e0 + h - cB * nrows);
            // w of position j + 1 + cc (0 for the x column itself)
            auto wat = [&](int cc) { return (cc == 0 || cc >= nc) ? 0.0 : wv[(j + 1 + cc == p) ? 1 : cc + 1]; };
            double wA = wat(cA), wB = wat(cB);
            double sA = 0.0, sB = 0.0;
            for (int k = 0; k < h; ++k) {
                double &a = A(iA, c0 + cA), &b = A(iB, c0 + cB);
                const double aa = a, bb = b;
                const double va = (iA == j) ? 1.0 : A(iA, j), vb = (iB == j) ? 1.0 : A(iB, j);
                const double xa = A(iA, c0), xb = A(iB, c0);
                const double na = fma(-va, wA, aa), nb = fma(-vb, wB, bb);
                if (cA != 0) a = na;
                if (cB != 0) b = nb;
                sA = fma(iA > (cA == 0 ? j + 1 : j) ? xa : 0.0, na, sA);
                sB = fma(iB > (cB == 0 ? j + 1 : j) ? xb : 0.0, nb, sB);
                if (++iA == r1) { pp[2 * (tid + cA)] = sA; sA = 0.0; iA = ib; ++cA; wA = wat(cA); }
                if (++iB == r1) { pp[2 * (tid + cB) + 1] = sB; sB = 0.0; iB = ib; ++cB; wB = wat(cB); }
            }
            if (cnt & 1) {                                          // the last element: stream B's next
                double &b = A(iB, c0 + cB);
                const double bb = b;
                const double vb = (iB == j) ? 1.0 : A(iB, j), xb = A(iB, c0);
                const double nb = fma(-vb, wB, bb);
                if (cB != 0) b = nb;
                sB = fma(iB > (cB == 0 ? j + 1 : j) ? xb : 0.0, nb, sB);
                if (++iB == r1) { pp[2 * (tid + cB) + 1] = sB; sB = 0.0; iB = ib; ++cB; }
            }
            if (iA != ib) pp[2 * (tid + cA)] = sA;
            if (iB != ib) pp[2 * (tid + cB) + 1] = sB;
        }
        __syncthreads();
        combine(T, nrows, E, nc, out);
    };
    // G > 1: after its cluster barrier's arrive every CTA writes its exchange buffer to its global
    // slot as tagged words; after the barrier's wait it reads its own cluster's buffers through
    // distributed shared memory and the other clusters' slots from global memory (bounded waits on
    // the tags).  A cluster's sum is formed with the same reduction tree wherever it is read and
    // the clusters' sums are added in cluster order, so every CTA holds the same doubles.
    unsigned long long *const xw = G > 1 ? jobs.xw[blockIdx.y] : nullptr;
    auto xslot = [&](int X, int cta) { return xw + (size_t)((X & 1) * G * C + cta) * jobs.xs * 2; };
    // exchange X: push rdb[0 .. n) into every peer's receive area (and, when G > 1, into this
    // CTA's global slot as tagged words), then wait until the bytes_in expected from the peers
    // have landed here (bounded)
    auto xsync = [&](const double *rdb, int n, int X, unsigned bytes_in) {
        if (!PUSH) {
            cl.sync();
            return;
        }
        const int P = X & 1;
        const unsigned mb = smem_u32(&mbar[P]);
        __syncthreads();                              // rdb complete
        // (after a wait gave up no more arrivals: a phase that did not complete takes no second one)
        if (tid == 0 && !xgive) mbar_expect(mb, bytes_in + (jobs.inject == 1 && X == 1 && g == 0 ? 8u : 0u));
        const int npair = (n + 1) >> 1;
        const unsigned src = smem_u32(rxb(P, q));     // this CTA's slot, at the same offset in every peer
        for (int k = tid; k < (C - 1) * npair; k += nt) {
            const int pi = k / npair, e2 = k - pi * npair, peer = pi + (pi >= q);
            const unsigned dst = cluster_addr(src + 16u * e2, peer), rmb = cluster_addr(mb, peer);
            if (2 * e2 + 1 < n) push2(dst, rdb[2 * e2], rdb[2 * e2 + 1], rmb);
            else push1(dst, rdb[2 * e2], rmb);
        }
        if (G > 1 && !(jobs.inject == 2 && X == 1 && qg == 0)) {
            unsigned long long *dst = xslot(X, qg);
            for (int e = tid; e < n; e += nt) xw_put(dst + 2 * e, rdb[e], (unsigned)X);
        }
        const unsigned par = ((X - 1) >> 1) & 1;       // completions of this mbarrier so far, mod 2
        for (long it = 0; !xgive && !mbar_try(mb, par); ++it)
            if (it >= QR_SPIN) { atomicExch(&g_qr_error, 1); xgive = true; }   // no further waits
    };
    // sum over every cluster's peers of rd[lo .. hi) into dst[lo .. hi): TPC threads per entry
    // (4, or 2 when four would take the threads a second round: every load of a thread is then in
    // flight at once, one round trip), each over the peers q = gq + TPC u of every cluster (C <=
    // 16), combined by shuffles within the group.  Per peer slot u the clusters' values are added
    // in cluster order, then one tree over u: the same doubles in every CTA.  Optionally the
    // group's first thread also copies the owner's row entry into rowdst[cc], from rowsh
    // (distributed shared memory) or from value rowoff + cc of CTA rowcta's slot.
    auto peer_sums_t = [&](auto tpc, const double *rd, int lo, int hi, int t0, int nthr, double *dst, int X,
                           const double *rowsh, int rowcta, int rowoff, double *rowdst) {
        constexpr int TPC = decltype(tpc)::value, PPT = 16 / TPC, NO = G > 1 ? G - 1 : 1;
        const int nT = (hi - lo) * TPC;
        for (int e = tid - t0; e >= 0 && e < ((nT + 31) & ~31); e += nthr) {
            const int cc = lo + e / TPC, gq = e % TPC;
            const bool act = e < nT;
            double v[PPT], o[NO][PPT];          // own cluster; the others (k: cluster k + (k >= g))
            unsigned long long wa[NO][PPT], wb[NO][PPT], ra = 0, rb2 = 0;
            unsigned long long need = 0;
            double rowv = 0.0;
#pragma unroll
            for (int u = 0; u < PPT; ++u) {
                v[u] = 0.0;
#pragma unroll
                for (int k = 0; k < NO; ++k) {
                    o[k][u] = 0.0;
                    if (act && k < G - 1 && gq + TPC * u < C) need |= 1ull << (PPT * k + u);
                }
            }
            if (act) {
                if (rowdst && gq == 0) {
                    if (rowsh) rowv = rowsh[cc];
                    else need |= 1ull << 40;
                }
#pragma unroll
                for (int u = 0; u < PPT; ++u)
                    if (gq + TPC * u < C) v[u] = peer_val(rd, X, gq + TPC * u, cc);
            }
            for (long it = 0; need && !xgive; ++it) {
#pragma unroll
                for (int k = 0; k < NO; ++k)
#pragma unroll
                    for (int u = 0; u < PPT; ++u)
                        if (need >> (PPT * k + u) & 1ull)
                            xw_load(xslot(X, (k + (k >= g)) * C + gq + TPC * u) + 2 * cc, wa[k][u], wb[k][u]);
                if (need >> 40 & 1ull) xw_load(xslot(X, rowcta) + 2 * (rowoff + cc), ra, rb2);
#pragma unroll
                for (int k = 0; k < NO; ++k)
#pragma unroll
                    for (int u = 0; u < PPT; ++u)
                        if ((need >> (PPT * k + u) & 1ull) && xw_ok(wa[k][u], wb[k][u], (unsigned)X)) {
                            o[k][u] = xw_val(wa[k][u], wb[k][u]);
                            need &= ~(1ull << (PPT * k + u));
                        }
                if ((need >> 40 & 1ull) && xw_ok(ra, rb2, (unsigned)X)) {
                    rowv = xw_val(ra, rb2);
                    need &= ~(1ull << 40);
                }
                if (need) {
                    if (it >= QR_SPIN) { atomicExch(&g_qr_error, 1); xgive = true; break; }
                    __nanosleep(32);
                }
            }
            if (act && rowdst && gq == 0) rowdst[cc] = rowv;
            double x[PPT];
#pragma unroll
            for (int u = 0; u < PPT; ++u) {
                x[u] = v[u];
                if (G > 1) {
                    // cluster c's value: own (c == g), else o[c - (c > g)]
                    x[u] = g == 0 ? v[u] : o[0][u];
#pragma unroll
                    for (int c2 = 1; c2 < G; ++c2)
                        x[u] += c2 == g ? v[u] : (c2 > g ? o[c2 - 1][u] : o[c2 < NO ? c2 : 0][u]);
                }
            }
            double tot;
            if (PPT == 4) {
                tot = (x[0] + x[1]) + (x[2] + x[3]);
            } else {
                tot = ((x[0] + x[1]) + (x[2] + x[3])) + ((x[4 % PPT] + x[5 % PPT]) + (x[6 % PPT] + x[7 % PPT]));
            }
#pragma unroll
            for (int sh = 1; sh < TPC; sh <<= 1) tot += __shfl_xor_sync(0xffffffffu, tot, sh);
            if (act && gq == 0) dst[cc] = tot;
        }
    };
    auto peer_sums = [&](const double *rd, int lo, int hi, int t0, int nthr, double *dst, int X,
                         const double *rowsh, int rowcta, int rowoff, double *rowdst) {
        if ((hi - lo) * 4 <= nthr)
            peer_sums_t(std::integral_constant<int, 4>{}, rd, lo, hi, t0, nthr, dst, X, rowsh, rowcta, rowoff, rowdst);
        else
            peer_sums_t(std::integral_constant<int, 2>{}, rd, lo, hi, t0, nthr, dst, X, rowsh, rowcta, rowoff, rowdst);
    };
    double sc2 = 1.0, scr = 1.0;   // pivot-norm scaling (1 / largest initial squared norm)
    if (piv) {
        for (int c = tid; c < s; c += nt) permv[c] = c;
        double *rd = red[xch & 1];
        flat_sums(r0, s, [&](int i, int c, double &x, double &y) { x = y = A(i, c); }, rd);
        xsync(rd, s, xch + 1, 8u * (C - 1) * s);
        ++xch;
        peer_sums(rd, 0, s, 0, nt, wv, xch, nullptr, 0, 0, nullptr);
        __syncthreads();
        if (warp == 0) {                 // largest squared column norm: one warp of shuffles
            double mxn = 0.0;
            for (int c = lane; c < s; c += 32) mxn = fmax(mxn, wv[c]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mxn = fmax(mxn, __shfl_xor_sync(0xffffffffu, mxn, o));
            if (lane == 0) bc[0] = mxn > 0.0 ? 1.0 / mxn : 1.0;
        }
        __syncthreads();
        sc2 = bc[0];
        scr = sqrt(sc2);
        for (int c = tid; c < s; c += nt) nrmf[c] = (float)(wv[c] * sc2);
        __syncthreads();
    }
    // warp 0: column of largest FP32 norm among j0 .. s-1 (ties: lowest index) into `pivot`
    auto argmax_pivot = [&](int j0) {
        float bv = -1.f;
        int bi = j0;
        for (int c = j0 + lane; c < s; c += 32) {
            const float v = nrmf[c];
            if (v > bv) { bv = v; bi = c; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (lane == 0) pivot = bi;
        return bi;                                  // the same in every lane after the butterfly
    };
    // step j + 1's partial sums are formed in the same pass as step j's trailing update
    // (fused_pass below); step 0's here: pivot, then the plain sums
    if (piv) {
        if (warp == 0) argmax_pivot(0);
        __syncthreads();
        const int p0 = pivot;
        if (p0 != 0) {
            for (int i = r0 + tid; i < r1; i += nt) {
                const double t = A(i, 0);
                A(i, 0) = A(i, p0);
                A(i, p0) = t;
            }
            if (tid == 0) {
                const float t = nrmf[0]; nrmf[0] = nrmf[p0]; nrmf[p0] = t;
                const int u = permv[0]; permv[0] = permv[p0]; permv[p0] = u;
            }
        }
        __syncthreads();
    }
    if (kmax > 0) {
        double *rd = red[xch & 1];
        // rd[0] = sigma2 part (rows > 0), rd[cc] = D_cc part; the owner of row 0 adds its row
        flat_sums(r0, s, [&](int i, int cc, double &x, double &y) {
            y = A(i, cc);
            x = (cc == 0 && i == 0) ? 0.0 : A(i, 0);
        }, rd);
        if (qg == 0)
            for (int cc = tid; cc < s; cc += nt) rd[s + cc] = A(0, cc);
    }
    for (int j = 0; j < kmax; ++j) {
        const int nc1 = s - j;              // columns j .. s-1
        const int own = j / rb;              // CTA holding row j (over the job)
        const bool owner = (qg == own);
        const int og = own / C, orank = own % C;   // its cluster and rank there
        const bool here = (og == g);
        const int ib = max(r0, j);
        double *rd = red[xch & 1];
        // partial sums [0, nc1), the owner's row [nc1, 2 nc1)
        xsync(rd, owner ? 2 * nc1 : nc1, xch + 1, 8u * ((C - 1) * nc1 + (here && !owner ? nc1 : 0)));
        ++xch;
        const double *ro = !here ? nullptr                       // the owner's buffer
                           : PUSH ? (orank == q ? rd : rxb(xch & 1, orank)) : cl.map_shared_rank(rd, orank);
        if (warp == 0) {
            // sigma2 over the peers (lane = peer, C <= 16) of every cluster, alpha from the owner,
            // the scalars
            double s2 = lane >= C ? 0.0 : peer_val(rd, xch, lane, 0);
            double so[G];
            unsigned long long wa[G], wb[G], aa = 0, ab = 0;
            unsigned need = 0;
            double al = 0.0;
#pragma unroll
            for (int c2 = 0; c2 < G; ++c2) {
                so[c2] = 0.0;
                if (c2 != g && lane < C) need |= 1u << c2;
            }
            if (here) al = ro[nc1];                   // beside the sigma2 loads
            else if (lane == 0) need |= 1u << 8;
            for (long it = 0; need && !xgive; ++it) {
#pragma unroll
                for (int c2 = 0; c2 < G; ++c2)
                    if (need >> c2 & 1u) xw_load(xslot(xch, c2 * C + lane), wa[c2], wb[c2]);
                if (need >> 8 & 1u) xw_load(xslot(xch, own) + 2 * nc1, aa, ab);
#pragma unroll
                for (int c2 = 0; c2 < G; ++c2)
                    if ((need >> c2 & 1u) && xw_ok(wa[c2], wb[c2], (unsigned)xch)) {
                        so[c2] = xw_val(wa[c2], wb[c2]);
                        need &= ~(1u << c2);
                    }
                if ((need >> 8 & 1u) && xw_ok(aa, ab, (unsigned)xch)) {
                    al = xw_val(aa, ab);
                    need &= ~(1u << 8);
                }
                if (need) {
                    if (it >= QR_SPIN) { atomicExch(&g_qr_error, 1); xgive = true; break; }
                    __nanosleep(32);
                }
            }
            // per peer (lane) the clusters in order, then one tree over the peers: the same
            // doubles in every CTA
            double x = g == 0 ? s2 : so[0];
#pragma unroll
            for (int c2 = 1; c2 < G; ++c2) x += c2 == g ? s2 : so[c2];
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            s2 = x;
            if (lane == 0) {
                // with nrm = (alpha^2 + sigma2)^(1/2) and a = |alpha|: tau = (beta - alpha) / beta
                // = 1 + a / nrm and 1 / (alpha - beta) = sign(alpha) / (a + nrm); one reciprocal
                // square root and one reciprocal in the dependent chain
                double tau = 0.0, beta = al, scal = 0.0;
                if (s2 > 0.0) {
                    const double x2 = fma(al, al, s2), rn = rsqrt(x2), nrm = x2 * rn, a = fabs(al);
                    beta = al >= 0.0 ? -nrm : nrm;
                    tau = fma(a, rn, 1.0);
                    scal = (al >= 0.0 ? 1.0 : -1.0) / (a + nrm);
                }
                bc[0] = tau; bc[1] = beta; bc[2] = scal; bc[3] = al;
                taus[j] = tau;
            }
        } else {
            peer_sums(rd, 1, nc1, 32, nt - 32, wv, xch, here ? ro + nc1 : nullptr, own, nc1, prow);
        }
        __syncthreads();
        const double tau = bc[0], beta = bc[1], scal = bc[2], al = bc[3];
        // w_c = tau v^T A_c = tau (P_c + (D_c - alpha P_c) / (alpha - beta)); pivot norms lose
        // the new row of R, R_jc = P_c - w_c; v stored in place: x_i / (alpha - beta)
        for (int cc = 1 + tid; cc < nc1; cc += nt) {
            const double Pc = prow[cc];
            const double w = tau * fma(scal, fma(-al, Pc, wv[cc]), Pc);
            wv[cc] = w;
            if (piv) {
                const float rf = (float)((Pc - w) * scr);
                nrmf[j + cc] = fmaxf(nrmf[j + cc] - rf * rf, 0.f);
            }
        }
        for (int i = max(r0, j + 1) + tid; i < r1; i += nt) A(i, j) *= scal;
        if (owner && tid == 0) A(j, j) = beta;
        __syncthreads();
        if (j + 1 == kmax) {
            // last reflector: columns beyond kmax (m < s) still take it
            if (tau != 0.0)
                flat_update(ib, j + 1, nc1 - 1, [&](int i) { return (i == j) ? 1.0 : A(i, j); }, wv + 1,
                            [&](int i, int c) -> double & { return A(i, c); });
            __syncthreads();
            break;
        }
        // pivot of step j + 1 (every warp finds the same), then that column takes reflector j and
        // moves to position j + 1; the old column j + 1 goes to position p
        int p = j + 1;
        if (piv) p = argmax_pivot(j + 1);
        for (int i = r0 + tid; i < r1; i += nt) {
            const double v = (i == j) ? 1.0 : A(i, j);
            const double wp = (i >= ib) ? wv[p - j] : 0.0;
            const double xp = fma(-v, wp, A(i, p));
            if (p != j + 1) A(i, p) = A(i, j + 1);
            A(i, j + 1) = xp;
        }
        __syncthreads();
        // reflector j on columns j + 2 .. s - 1 and step j + 1's partial sums in one pass (the
        // column now at position p is the old column j + 1: it takes w of position j + 1)
        double *rn = red[xch & 1];
        fused_pass(j, p, ib, nc1 - 1, rn);
        if (qg == (j + 1) / rb)
            for (int cc = tid; cc < nc1 - 1; cc += nt) rn[nc1 - 1 + cc] = A(j + 1, j + 1 + cc);
        if (tid == 0 && p != j + 1) {                // FP32 norm and index follow the move
            const float f = nrmf[j + 1]; nrmf[j + 1] = nrmf[p]; nrmf[p] = f;
            const int u = permv[j + 1]; permv[j + 1] = permv[p]; permv[p] = u;
        }
    }
    if (J.tau && qg == 0)
        for (int j = tid; j < kmax; j += nt) J.tau[j] = taus[j];
    if (piv && qg == 0)
        for (int c = tid; c < s; c += nt) J.perm[c] = permv[c];
    if (SMEM) {
        for (int e = tid; e < nr * s; e += nt) {
            const int i = r0 + e % nr, c = e / nr;
            J.A[i + (long long)c * m] = A(i, c);
        }
    }
    cl.sync();   // keep this CTA's shared memory alive until every peer finished reading it
}

using QRKernel = void (*)(QRJobs, int);
static QRKernel qr_kernel(bool smem, int G) {
    static const QRKernel k[2][QR_GMAX] = {{k_qr<false, 1>, k_qr<false, 2>, k_qr<false, 3>},
                                           {k_qr<true, 1>, k_qr<true, 2>, k_qr<true, 3>}};
    return k[smem ? 1 : 0][G - 1];
}

static void qr_reflectors(Ctx &c, const std::vector<QRJob> &jobs, int inject = 0) {
    if (jobs.empty()) return;
    static std::atomic<bool> attr_set{false};   // set once; idempotent if two threads race
    if (!attr_set) {
        for (int G = 1; G <= QR_GMAX; ++G) {
            TK_CUDA(cudaFuncSetAttribute(qr_kernel(true, G), cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            TK_CUDA(cudaFuncSetAttribute(qr_kernel(false, G), cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            TK_CUDA(cudaFuncSetAttribute(qr_kernel(true, G), cudaFuncAttributeMaxDynamicSharedMemorySize, QR_DSMEM));
            TK_CUDA(cudaFuncSetAttribute(qr_kernel(false, G), cudaFuncAttributeMaxDynamicSharedMemorySize, QR_DSMEM));
        }
        attr_set = true;
    }
    for (size_t base = 0; base < jobs.size(); base += TK_MAX_D) {
        QRJobs J{};
        J.inject = inject;
        J.n = (int)std::min<size_t>(TK_MAX_D, jobs.size() - base);
        int mmax = 0, smax = 0;
        for (int i = 0; i < J.n; ++i) {
            J.j[i] = jobs[base + i];
            TK_REQUIRE(J.j[i].s <= QR_MAXS, "QR: more than 256 columns");
            TK_REQUIRE(J.j[i].Q == nullptr, "QR kernel: Q is formed by qr_form_q");
            mmax = std::max(mmax, J.j[i].m);
            smax = std::max(smax, J.j[i].s);
        }
        // cluster of up to 16 CTAs with >= 48 rows each, shrunk until the device can place it;
        // a single tall unfolding (the FP64 pass dominates its steps) is split over G <= 3 clusters
        // of >= 64 rows per CTA that add their per-step sums through global memory.  Clusters wait
        // only for their own job's clusters, so a job can stall only if it cannot have all G
        // resident: with one other such job running concurrently, 2 G - 1 co-resident clusters
        // guarantee that one of the two has all of its clusters
        int C = std::max(1, std::min(16, (mmax + 47) / 48));
        int G = J.n == 1 ? std::max(1, std::min(QR_GMAX, mmax / (16 * 64))) : 1;
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr[1];
        int rb = 0;
        bool use_smem = false;
        for (;;) {
            // dynamic shared memory: the rows (when they fit) and the receive area
            rb = (mmax + G * C - 1) / (G * C);
            const size_t rows = (size_t)rb * smax * sizeof(double);
            const size_t rxbytes = G > 1 ? (size_t)2 * C * 2 * smax * sizeof(double) : 0;
            use_smem = rows + rxbytes <= QR_DSMEM;
            J.rxs = 2 * smax;
            J.rx_off = use_smem ? (rb * smax + 1) & ~1 : 0;   // 16-byte aligned
            cfg = cudaLaunchConfig_t{};
            cfg.gridDim = dim3((unsigned)(G * C), (unsigned)J.n, 1);
            cfg.blockDim = dim3(QR_THREADS, 1, 1);
            cfg.dynamicSmemBytes = (size_t)J.rx_off * sizeof(double) + rxbytes;
            cfg.stream = c.st;
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = C;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            if (C == 1 && G == 1) break;
            int nclusters = 0;
            const cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, qr_kernel(use_smem, G), &cfg);
            if (e != cudaSuccess) cudaGetLastError();
            if (e == cudaSuccess && nclusters >= 2 * G - 1) break;
            if (G > 1) --G;
            else C = C > 8 ? 8 : C / 2;
        }
        ScopedMark mark(*c.arena);
        if (G > 1) {                  // two slots per CTA of xs values, two words each, zeroed
            J.xs = 2 * smax;
            const size_t words = (size_t)2 * G * C * J.xs * 2;
            J.xw[0] = static_cast<unsigned long long *>(c.arena->alloc_bytes(sizeof(unsigned long long) * words));
            TK_CUDA(cudaMemsetAsync(J.xw[0], 0, sizeof(unsigned long long) * words, c.st));
        }
        c.pre_launch();
        TK_CUDA(cudaLaunchKernelEx(&cfg, qr_kernel(use_smem, G), J, rb));
        double flops = 0.0;   // Householder R: 2 m s^2 - 2 s^3 / 3
        for (int i = 0; i < J.n; ++i) {
            const double m = J.j[i].m, s = std::min(J.j[i].m, J.j[i].s);
            flops += 2.0 * m * s * s - 2.0 * s * s * s / 3.0;
        }
        c.check_launch("qr", flops);
    }
}

// Explicit Q from the reflectors in compact WY form (Schreiber and Van Loan's representation,
// with T from the UT transform of Joffrain, Low, Quintana-Orti and van de Geijn): with
// k = min(m, s), V (m x k) unit lower trapezoidal (v_j(j) = 1, v_j(i) = A(i, j) below, zero above)
// and tau, H_0 ... H_{k-1} = I - V T V^T where T^{-1} = S = diag(1 / tau) + the strict upper
// part of V^T V (an algebraic identity for any tau; a reflector with tau = 0 is the identity and
// its column of V is set to zero, with S_jj = 1).  Q = E - V X with S X = V_1^T, V_1 = V[0:k, :],
// E = [I_s; 0] (or [I_m, 0] when m < s, columns >= m of Q zero).  The k reflector steps that
// the backward accumulation would take, each with a cluster exchange, become two FP64 GEMMs over m
// and a triangular solve of order k whose columns are independent.
struct QRWY {
    int n, k[TK_MAX_D], m[TK_MAX_D], s[TK_MAX_D];
    const double *A[TK_MAX_D], *tau[TK_MAX_D], *W[TK_MAX_D];
    double *V[TK_MAX_D], *Q[TK_MAX_D], *X[TK_MAX_D];
};

__global__ void k_qr_wy_init(const __grid_constant__ QRWY J) {
    const int b = blockIdx.y, m = J.m[b], s = J.s[b], k = J.k[b];
    const long long n = (long long)m * s;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), c = (int)(e / m);
        if (c < k) {
            const double v = (i > c) ? J.A[b][e] : (i == c ? 1.0 : 0.0);
            J.V[b][e] = J.tau[b][c] == 0.0 ? 0.0 : v;
        }
        J.Q[b][e] = (i == c && c < k) ? 1.0 : 0.0;
    }
}

// S X = V_1^T for columns [c0, c0 + QWY_CPB) of X: S (upper triangle from W = V^T V and tau) in
// shared memory, right-looking back substitution (row j of X, then the rank-1 update of the rows
// above it), the block's columns side by side
constexpr int QWY_CPB = 8;
__global__ void __launch_bounds__(256) k_qr_wy_solve(const __grid_constant__ QRWY J) {
    const int b = blockIdx.y, k = J.k[b], m = J.m[b];
    const int c0 = blockIdx.x * QWY_CPB;
    if (c0 >= k) return;
    const int nc = min(QWY_CPB, k - c0);
    extern __shared__ double wsh[];
    double *S = wsh;                                  // k x k (upper triangle used)
    double *Bs = wsh + (size_t)k * k;                 // k x QWY_CPB
    const int tid = threadIdx.x, nt = blockDim.x;
    const double *W = J.W[b], *V = J.V[b], *tau = J.tau[b];
    for (int e = tid; e < k * k; e += nt) S[e] = W[e];
    for (int e = tid; e < k * nc; e += nt) {
        const int j = e % k, cc = e / k;
        Bs[j + cc * k] = V[(c0 + cc) + (long long)j * m];      // V_1^T[j, c] = V[c, j]
    }
    __syncthreads();
    for (int j = k - 1; j >= 0; --j) {
        const double dj = tau[j] == 0.0 ? 1.0 : tau[j];          // 1 / S_jj
        if (tid < nc) Bs[j + tid * k] *= dj;
        __syncthreads();
        for (int e = tid; e < j * nc; e += nt) {
            const int i = e % j, cc = e / j;
            Bs[i + cc * k] = fma(-S[i + j * k], Bs[j + cc * k], Bs[i + cc * k]);
        }
        __syncthreads();
    }
    for (int e = tid; e < k * nc; e += nt) {
        const int j = e % k, cc = e / k;
        J.X[b][j + (long long)(c0 + cc) * k] = Bs[j + cc * k];
    }
}

static void qr_form_q(Ctx &c, const std::vector<QRJob> &jobs) {
    for (size_t base = 0; base < jobs.size(); base += TK_MAX_D) {
        QRWY J{};
        J.n = (int)std::min<size_t>(TK_MAX_D, jobs.size() - base);
        int kmax = 0;
        long long nmax = 0;
        for (int i = 0; i < J.n; ++i) {
            const QRJob &q = jobs[base + i];
            TK_REQUIRE(q.tau != nullptr, "QR: the explicit Q needs tau");
            J.m[i] = q.m;
            J.s[i] = q.s;
            J.k[i] = std::min(q.m, q.s);
            J.A[i] = q.A;
            J.tau[i] = q.tau;
            J.Q[i] = q.Q;
            J.V[i] = c.arena->alloc((size_t)q.m * J.k[i]);
            J.W[i] = J.X[i] = nullptr;
            kmax = std::max(kmax, J.k[i]);
            nmax = std::max(nmax, (long long)q.m * q.s);
        }
        double *Wb[TK_MAX_D];
        for (int i = 0; i < J.n; ++i) {
            Wb[i] = c.arena->alloc((size_t)J.k[i] * J.k[i]);
            J.W[i] = Wb[i];
            J.X[i] = c.arena->alloc((size_t)J.k[i] * J.k[i]);
        }
        c.pre_launch();
        k_qr_wy_init<<<dim3((unsigned)std::min<long long>((nmax + 255) / 256, 592), (unsigned)J.n), 256, 0, c.st>>>(J);
        double bytes = 0.0;
        for (int i = 0; i < J.n; ++i) bytes += 8.0 * ((double)J.m[i] * J.k[i] * 2 + (double)J.m[i] * J.s[i]);
        c.check_launch("qr_wy_init", 0.0, bytes);
        {
            Gemm g(c, "gemm_qr");
            for (int i = 0; i < J.n; ++i)
                g.add1(J.k[i], J.k[i], J.m[i], 1, 0, J.V[i], J.m[i], J.V[i], J.m[i], Wb[i], J.k[i]);
            g.run();
        }
        constexpr int WY_SMEM_MAX = 227 * 1024;
        static std::atomic<bool> attr_set{false};
        if (!attr_set) {
            TK_CUDA(cudaFuncSetAttribute(k_qr_wy_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, WY_SMEM_MAX));
            attr_set = true;
        }
        const size_t smem = sizeof(double) * ((size_t)kmax * kmax + (size_t)kmax * QWY_CPB);
        TK_REQUIRE(smem <= (size_t)WY_SMEM_MAX, "QR: an explicit Q of more than 165 columns");
        c.pre_launch();
        k_qr_wy_solve<<<dim3((unsigned)((kmax + QWY_CPB - 1) / QWY_CPB), (unsigned)J.n), 256, smem, c.st>>>(J);
        double flops = 0.0;
        for (int i = 0; i < J.n; ++i) flops += (double)J.k[i] * J.k[i] * J.k[i];
        c.check_launch("qr_wy_solve", flops);
        {
            Gemm g(c, "gemm_qr");
            for (int i = 0; i < J.n; ++i)
                g.add1(J.m[i], J.k[i], J.k[i], 0, 0, J.V[i], J.m[i], J.X[i], J.k[i], J.Q[i], J.m[i], 1.0, -1.0);
            g.run();
        }
    }
}

// Self-test of the multi-cluster QR's bounded waits: one R-only QR of a 2560 x 50 matrix (zeros:
// the values do not matter) on two clusters with an exchange made to go missing (inject 1 or 2,
// see QRJobs::inject).  Returns 1 when the kernel gave up waiting, set the error flag and
// finished (the flag is cleared), 0 otherwise.
int qr_wait_selftest(Ctx &c, int inject) {
    TK_REQUIRE(inject == 1 || inject == 2, "QR self-test: mode 1 or 2");
    const int m = 2560, s = 50;
    double *A = c.arena->alloc((size_t)m * s);
    double *tau = c.arena->alloc(s);
    TK_CUDA(cudaMemsetAsync(A, 0, sizeof(double) * m * s, c.st));
    qr_error_flag(true);
    qr_reflectors(c, {QRJob{A, tau, nullptr, m, s, nullptr}}, inject);
    TK_CUDA(cudaStreamSynchronize(c.st));
    return qr_error_flag(true) != 0 ? 1 : 0;
}

void qr_householder(Ctx &c, const std::vector<QRJob> &jobs) {
    if (jobs.empty()) return;
    // the kernel leaves R and the reflectors; an explicit Q is formed from them afterwards
    std::vector<QRJob> rj = jobs;
    bool wantq = false;
    for (QRJob &j : rj) {
        wantq = wantq || j.Q != nullptr;
        j.Q = nullptr;
    }
    qr_reflectors(c, rj);
    if (!wantq) return;
    std::vector<QRJob> qj;
    for (const QRJob &j : jobs)
        if (j.Q) qj.push_back(j);
    ScopedMark mark(*c.arena);
    qr_form_q(c, qj);
}

// ------------------------------------------------------------------------------------------
// One-sided Jacobi SVD of a small square matrix (one CTA each)
// ------------------------------------------------------------------------------------------
struct SVDJobs {
    int n;
    SVDJob j[TK_MAX_D];
    double *pinv[TK_MAX_D];   // optional s x s pseudo-inverse outputs
    double rcond;
    float2 *rlog[TK_MAX_D];   // k_svd_cl: rotation log of the FP32 sweeps (SVD_LOG_SWEEPS sweeps)
    unsigned long long *prog[TK_MAX_D];   // k_svd_cl: progress word of the FP32 phase
    unsigned long long tag;               // k_svd_cl: this launch's id << 32
};
constexpr int SVD_LOG_SWEEPS = 20;

// Sweep counts of the last k_svd launch (per block: FP32 phase, FP64 phase); diagnostics.
__device__ int g_svd_sweeps[2 * TK_MAX_D];

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide reductions with a single combining warp.  On this part an FP64 warp instruction
// occupies the SMSP's FP64 pipe for ~64 cycles however many lanes are active, so partials are
// combined once by warp 0, never re-added by every thread.  `scratch` holds >= 33 elements.
__device__ float block_sum_f(float v, float *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_t(v);
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (warp == 0) {
        float t = lane < nw ? scratch[lane] : 0.f;
        t = warp_sum_t(t);
        if (lane == 0) scratch[32] = t;
    }
    __syncthreads();
    const float r = scratch[32];
    __syncthreads();
    return r;
}

__device__ int block_max_i(int v, int *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int t = lane < nw ? scratch[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = max(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (lane == 0) scratch[32] = t;
    }
    __syncthreads();
    const int r = scratch[32];
    __syncthreads();
    return r;
}

// Round-robin tournament: in round `round` of a sweep over sp (even) columns, pair `pr` joins
// columns p < q; every column appears in exactly one pair per round.
__device__ __forceinline__ void rr_pair(int round, int pr, int sp, int &p, int &q) {
    if (pr == 0) { p = round; q = sp - 1; }
    else {
        // (round + pr) mod (sp - 1) and (round - pr) mod (sp - 1), both arguments in
        // (-(sp - 1), 2 (sp - 1)): one conditional correction each, no integer division
        p = round + pr;
        if (p >= sp - 1) p -= sp - 1;
        q = round - pr;
        if (q < 0) q += sp - 1;
    }
    if (p > q) { const int t = p; p = q; q = t; }
}

// FP32 one-sided (Hestenes) Jacobi on the columns of A (s x s, column-major, shared memory),
// rotations accumulated into V.  A round of the sweep is latency bound (dot product, butterfly,
// rotation, barrier, s - 1 rounds in a row), so each pair takes a group of G lanes with up to
// J32R rows per lane held in registers: 32 / G pairs share a warp and only ceil(np G / 32) warps
// issue the round, synchronised by a named barrier.  The butterfly leaves a_p . a_q in every lane
// of the group and every lane forms the rotation itself, with fast FP32 intrinsics: this phase
// only has to bring the columns close to orthogonal, the FP64 phase finishes.  A pair is rotated
// when |a_p . a_q| > tol ||a_p|| ||a_q|| and both squared norms exceed `floor2`.  Convergence is
// checked after every sweep on the full Gram matrix A^T A (one dot product per thread), which
// replaces a final rotation-free sweep.  Column squared norms are kept in `nrm2` (Rutishauser's
// updates inside a sweep, exact from the Gram check between sweeps).  Returns the number of sweeps.
// LOG: V is not touched; the rotation of every live pair of every round is written to `rlog`
// instead, (cos, sin) as a float2 at [(sweep (s' - 1) + round) np + pair] ((1, 0) when the pair is
// not rotated), for replay_rotations (the round is bound by moving columns through shared
// memory, and V's columns are half of that traffic).
constexpr int J32R = 5;
__device__ __forceinline__ float dot_rows(const float *x, const float *y, int s) {
    float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
    int i = 0;
    for (; i + 3 < s; i += 4) {
        t0 = fmaf(x[i], y[i], t0);
        t1 = fmaf(x[i + 1], y[i + 1], t1);
        t2 = fmaf(x[i + 2], y[i + 2], t2);
        t3 = fmaf(x[i + 3], y[i + 3], t3);
    }
    for (; i < s; ++i) t0 = fmaf(x[i], y[i], t0);
    return (t0 + t1) + (t2 + t3);
}
// Progress word of a logged FP32 phase (global memory): tag (the launch's id << 32) | sweeps
// logged | SVD_PROG_DONE once the phase has ended; written with release semantics after the
// block's barrier, so every log entry of the announced sweeps is visible to a reader that
// acquires it.
constexpr unsigned long long SVD_PROG_DONE = 1ULL << 16;
__device__ __forceinline__ void svd_publish(unsigned long long *prog, unsigned long long v) {
    __threadfence();
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(prog), "l"(v) : "memory");
}
template <int G, bool LOG>
__device__ int jacobi32_g(float *A, float *V, float *nrm2, int s, float tol, float floor2, int max_sweeps,
                          int *flag, float2 *rlog, unsigned long long *prog, unsigned long long tag) {
    constexpr int PPW = 32 / G;                      // pairs per warp
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5, nt = blockDim.x;
    const int gl = lane & (G - 1), slot = lane / G;
    const int sp = s + (s & 1), np = sp / 2;
    const int nact = min(nw, (np + PPW - 1) / PPW);  // warps holding a pair
    int sweeps = 0;
    for (;;) {
        // Gram check: squared norms first, then every pair p < q
        for (int c = tid; c < s; c += nt) nrm2[c] = dot_rows(A + c * s, A + c * s, s);
        if (tid == 0) *flag = 0;
        __syncthreads();
        for (int e = tid; e < s * s; e += nt) {
            const int p = e % s, q = e / s;
            if (p >= q) continue;
            const float al = nrm2[p], be = nrm2[q];
            if (al <= floor2 || be <= floor2) continue;
            const float g = dot_rows(A + p * s, A + q * s, s);
            // 4x the rotation tolerance: the check's dot product is summed in another order
            // than the sweep's, and a pair between the two must not keep the loop alive
            if (fabsf(g) > 4.f * tol * __fsqrt_rn(al) * __fsqrt_rn(be)) *flag = 1;
        }
        __syncthreads();
        const int more = *flag;
        __syncthreads();
        if (!more || sweeps >= max_sweeps || sp < 2) break;
        ++sweeps;
        if (warp < nact) {
            for (int round = 0; round < sp - 1; ++round) {
                // every lane of the warp runs the same trip count, so the butterfly below is
                // warp-uniform; a group without a live pair carries zeros through it
                for (int base = warp * PPW; base < np; base += nw * PPW) {
                    const int pr = base + slot;
                    int p = 0, q = 0;
                    bool live = pr < np;
                    if (live) {
                        rr_pair(round, pr, sp, p, q);
                        live = q < s;
                    }
                    float a[J32R], b[J32R], va[J32R], vb[J32R];
#pragma unroll
                    for (int k = 0; k < J32R; ++k) {
                        const int i = gl + G * k;
                        a[k] = b[k] = va[k] = vb[k] = 0.f;
                        if (live && i < s) {
                            a[k] = A[i + p * s];
                            b[k] = A[i + q * s];
                            if (!LOG) {
                                va[k] = V[i + p * s];
                                vb[k] = V[i + q * s];
                            }
                        }
                    }
                    const float al = live ? nrm2[p] : 0.f, be = live ? nrm2[q] : 0.f;
                    float ga = 0.f;
#pragma unroll
                    for (int k = 0; k < J32R; ++k) ga = fmaf(a[k], b[k], ga);
#pragma unroll
                    for (int o = G / 2; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
                    if (!live) continue;
                    float2 *lg = LOG ? rlog + ((size_t)(sweeps - 1) * (sp - 1) + round) * np + pr : nullptr;
                    // norms above floor2 = 2^-100 or a positive fraction of ||A||_F^2: normal
                    // numbers, so x * rsqrt(x) is a safe square root
                    if (al <= floor2 || be <= floor2 || !(fabsf(ga) > tol * (al * rsqrtf(al)) * (be * rsqrtf(be)))) {
                        if (LOG && gl == 0) *lg = make_float2(1.f, 0.f);
                        continue;
                    }
                    const float zeta = __fdividef(be - al, 2.f * ga);
                    const float az = fabsf(zeta), z1 = fmaf(zeta, zeta, 1.f);
                    const float t = az < 1e18f ? __fdividef(copysignf(1.f, zeta), az + z1 * rsqrtf(z1))
                                               : __fdividef(0.5f, zeta);
                    const float cs = rsqrtf(fmaf(t, t, 1.f)), sn = cs * t;
                    if (LOG && gl == 0) *lg = make_float2(cs, sn);
#pragma unroll
                    for (int k = 0; k < J32R; ++k) {
                        const int i = gl + G * k;
                        if (i < s) {
                            A[i + p * s] = cs * a[k] - sn * b[k];
                            A[i + q * s] = sn * a[k] + cs * b[k];
                            if (!LOG) {
                                V[i + p * s] = cs * va[k] - sn * vb[k];
                                V[i + q * s] = sn * va[k] + cs * vb[k];
                            }
                        }
                    }
                    if (gl == 0) {
                        nrm2[p] = fmaxf(al - t * ga, 0.f);
                        nrm2[q] = be + t * ga;
                    }
                }
                asm volatile("bar.sync 1, %0;" ::"r"(nact * 32) : "memory");
            }
        }
        __syncthreads();
        // this sweep's log is complete (the barrier above): announce it
        if (LOG && tid == 0) svd_publish(prog, tag | (unsigned long long)sweeps);
    }
    if (LOG && tid == 0) svd_publish(prog, tag | (unsigned long long)sweeps | SVD_PROG_DONE);
    return sweeps;
}
// s <= G J32R rows per group; SVD_MAXS = 96 needs G = 32 at most
template <bool LOG>
__device__ int jacobi32(float *A, float *V, float *nrm2, int s, float tol, float floor2, int max_sweeps,
                        int *flag, float2 *rlog = nullptr, unsigned long long *prog = nullptr,
                        unsigned long long tag = 0) {
    if (s <= 4 * J32R) return jacobi32_g<4, LOG>(A, V, nrm2, s, tol, floor2, max_sweeps, flag, rlog, prog, tag);
    if (s <= 8 * J32R) return jacobi32_g<8, LOG>(A, V, nrm2, s, tol, floor2, max_sweeps, flag, rlog, prog, tag);
    if (s <= 16 * J32R) return jacobi32_g<16, LOG>(A, V, nrm2, s, tol, floor2, max_sweeps, flag, rlog, prog, tag);
    return jacobi32_g<32, LOG>(A, V, nrm2, s, tol, floor2, max_sweeps, flag, rlog, prog, tag);
}

// Bounded waits of the replay for the FP32 phase's progress (a sweep takes ~100 us; the limit
// is ~0.1 s), after which g_svd_error is set and the replay stops.
__device__ int g_svd_error;
constexpr long SVD_SPIN = 1L << 17;

// V = the product of the rotations jacobi32<true> logs (V starts as the identity), rows [r0, r1)
// only, in shared memory row-major with leading dimension s + 1, replayed sweep by sweep while
// the FP32 phase runs on another CTA: before sweep k the block waits (bounded) until the progress
// word announces it or the end of the phase.  A row changes only under column rotations, so rows
// are independent, and the pairs of a round touch disjoint columns: one thread per (row, pair), a
// barrier over those threads' warps per round; each sweep's log is first staged in shared memory
// (`stage`, (s' - 1) np float2) by the whole block.  The same products in the same order as
// rotating V inline.
__device__ void replay_rotations(const float2 *rlog, const unsigned long long *prog, unsigned long long tag,
                                 int s, float *Vrows, int r0, int r1, float2 *stage) {
    __shared__ unsigned long long prog_s;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int sp = s + (s & 1), np = sp / 2, R = sp - 1, ld = s + 1, nrow = r1 - r0;
    const int ntask = nrow * np, nwt = (ntask + 31) / 32;        // warps holding a task
    const int row = tid / np, pr = tid % np;
    for (int e = tid; e < nrow * ld; e += nt) {
        const int lr = e / ld, c = e % ld;
        Vrows[e] = (c == r0 + lr) ? 1.f : 0.f;
    }
    for (int sw = 0;; ++sw) {
        if (tid == 0) {
            unsigned long long v = 0;
            for (long it = 0;; ++it) {
                asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(prog) : "memory");
                if ((v & 0xFFFFFFFF00000000ULL) == tag && ((v & 0xFFFFULL) > (unsigned long long)sw || (v & SVD_PROG_DONE)))
                    break;
                if (it >= SVD_SPIN) {                                  // give up: no further sweep
                    atomicExch(&g_svd_error, 1);
                    v = tag | SVD_PROG_DONE;
                    break;
                }
                __nanosleep(256);
            }
            prog_s = v;
        }
        __syncthreads();
        if ((prog_s & 0xFFFFULL) <= (unsigned long long)sw) break;       // the phase ended before sweep sw
        const float2 *src = rlog + (size_t)sw * R * np;
        for (int e = tid; e < R * np; e += nt) stage[e] = __ldcg(src + e);   // written by another SM
        __syncthreads();
        if (tid < nwt * 32) {
            float *v = Vrows + row * ld;
            for (int round = 0; round < R; ++round) {
                if (tid < ntask) {
                    int p, q;
                    rr_pair(round, pr, sp, p, q);
                    if (q < s) {
                        const float2 r = stage[round * np + pr];
                        const float a = v[p], b = v[q];
                        v[p] = r.x * a - r.y * b;
                        v[q] = r.y * a + r.x * b;
                    }
                }
                asm volatile("bar.sync 2, %0;" ::"r"(nwt * 32) : "memory");
            }
        }
        __syncthreads();
    }
}

int svd_error_flag(bool reset) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_svd_error, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (reset && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_svd_error, &z, sizeof(int));
    }
    return v;
}

// FP64 phase of the one-sided Jacobi SVD.  Every FP64 warp instruction occupies an SMSP's FP64
// pipe for ~64 cycles on this part whatever the active lanes, so the work is organised by
// FP64 instruction count.  Each step starts with a Gram check: H = A^T A (one FP64 dot per
// thread, packed upper triangle in `gram`), diagonal into `nrm2`; a pair (p, q) still needs
// work when H_pq^2 > (4 tol)^2 H_pp H_qq with both squared norms above `floor2`.  Then:
//
//  * correction step (graded mode, when every such pair is well separated,
//    |H_pq| <= 1e-3 |H_qq - H_pp|): all rotations at once, A <- A (I + T + T^2 / 2) with the
//    skew first-order angles T_pq = H_pq / (H_qq - H_pp) (pairs below tolerance: 0).  The
//    off-diagonal left is second order in the angles (quadratic convergence) and
//    I + T + T^2 / 2 is orthogonal to third order; T^2 is formed in FP32 (its entries are
//    squares of the angles).  One FP64 GEMM instead of s - 1 sequential rounds.
//  * otherwise a full sweep of round-robin rotations: (1) partial dot products over JNP row
//    blocks, warp = row block, lane = pair; (2) one thread per pair, spread over four warps
//    (one per SMSP), sums the parts, tests, and forms the rotation: angle from FP32 arithmetic,
//    cos = (1 + t^2)^(-1/2) refined by two FP64 Newton steps so that the rotation is
//    orthogonal to FP64 rounding; (3) one thread per (pair, row) rotates.
//
// The loop ends at the first Gram check with no pair left (or after max_steps steps).
// Scratch for the correction step (graded mode only): `tmat` s x s FP64, `tf` 2 s^2 floats
// (may alias `gram`, which is dead once T is formed).
constexpr int JNP = 4;
constexpr int SVD_REGS = 9;   // outputs per thread held in registers by an in-place GEMM (s^2 / threads)
template <bool ACC>
__device__ int jacobi64(double *A, double *V, double *nrm2, int s, double tol, double floor2, int max_steps,
                        int *flag, double *gpart, double *cpar, double *spar, int *act, double *gram,
                        double *tmat, float *tf, int *nsweeps) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    const int sp = s + (s & 1), np = sp / 2;
    const int wpp = (np + 31) / 32;             // warps per row block in sweep step (1)
    const int rbk = (s + JNP - 1) / JNP;
    const int nps = s * (s + 1) / 2;
    const double chk2 = 16.0 * tol * tol;
    __shared__ int sep_bad;
    int steps = 0, sweeps = 0;
    auto unpack = [](int e, int &p, int &q) {
        q = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
        while (q * (q + 1) / 2 > e) --q;
        while ((q + 1) * (q + 2) / 2 <= e) ++q;
        p = e - q * (q + 1) / 2;
    };
    for (;;) {
        // Gram check
        for (int e = tid; e < nps; e += nt) {
            int p, q;
            unpack(e, p, q);
            double g = 0.0;
            for (int i = 0; i < s; ++i) g = fma(A[i + p * s], A[i + q * s], g);
            gram[e] = g;
            if (p == q) nrm2[p] = g;
        }
        if (tid == 0) { *flag = 0; sep_bad = 0; }
        __syncthreads();
        for (int e = tid; e < nps; e += nt) {
            int p, q;
            unpack(e, p, q);
            if (p == q) continue;
            const double al = nrm2[p], be = nrm2[q], g = gram[e];
            if (al > floor2 && be > floor2 && g * g > chk2 * al * be) {
                *flag = 1;
                if (!(fabs(g) <= 1e-3 * fabs(be - al))) sep_bad = 1;
            }
        }
        __syncthreads();
        const int more = *flag, simultaneous = (tmat != nullptr) && !sep_bad;
        __syncthreads();
        if (!more || steps >= max_steps || sp < 2) break;
        ++steps;
        if (simultaneous) {
            // T (skew) into tmat, and an FP32 copy into tf[0 .. s^2)
            for (int e = tid; e < s * s; e += nt) {
                const int p = e % s, q = e / s;
                double t = 0.0;
                if (p != q) {
                    const int lo = min(p, q), hi = max(p, q);
                    const double al = nrm2[lo], be = nrm2[hi], g = gram[lo + hi * (hi + 1) / 2];
                    if (al > floor2 && be > floor2 && g * g > chk2 * al * be) {
                        const double tl = g / (be - al);      // T[lo, hi]
                        t = (p == lo) ? tl : -tl;
                    }
                }
                tmat[e] = t;
            }
            __syncthreads();
            for (int e = tid; e < s * s; e += nt) tf[e] = (float)tmat[e];
            __syncthreads();
            // D = T + T^2 / 2 (T^2 in FP32 into tf[s^2 ..)), then in place into tmat
            float *t2 = tf + s * s;
            for (int e = tid; e < s * s; e += nt) {
                const int i = e % s, j = e / s;
                float acc = 0.f;
                for (int k = 0; k < s; ++k) acc = fmaf(tf[i + k * s], tf[k + j * s], acc);
                t2[e] = acc;
            }
            __syncthreads();
            for (int e = tid; e < s * s; e += nt) tmat[e] += 0.5 * (double)t2[e];
            __syncthreads();
            // A <- A + A D, outputs held in registers until every thread has read A
            double r[SVD_REGS];
#pragma unroll
            for (int k = 0; k < SVD_REGS; ++k) {
                const int e = tid + k * nt;
                if (e < s * s) {
                    const int i = e % s, j = e / s;
                    double acc = A[e];
                    for (int kk = 0; kk < s; ++kk) acc = fma(A[i + kk * s], tmat[kk + j * s], acc);
                    r[k] = acc;
                }
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < SVD_REGS; ++k) {
                const int e = tid + k * nt;
                if (e < s * s) A[e] = r[k];
            }
            __syncthreads();
            continue;
        }
        ++sweeps;
        for (int round = 0; round < sp - 1; ++round) {
            // (1) partial dots: warp = (part, pair block), lane = pair
            for (int w = warp; w < JNP * wpp; w += nt >> 5) {
                const int part = w / wpp, pr = (w % wpp) * 32 + lane;
                if (pr >= np) continue;
                int p, q;
                rr_pair(round, pr, sp, p, q);
                double g = 0.0;
                if (q < s) {
                    const int i1 = min(s, (part + 1) * rbk);
                    for (int i = part * rbk; i < i1; ++i) g = fma(A[i + p * s], A[i + q * s], g);
                }
                gpart[part * np + pr] = g;
            }
            __syncthreads();
            // (2) rotation per pair: pair pr on warp pr % 4, lane pr / 4
            if (warp < 4) {
                for (int pr = lane * 4 + warp; pr < np; pr += 128) {
                    int p, q;
                    rr_pair(round, pr, sp, p, q);
                    int doit = 0;
                    if (q < s) {
                        const double al = nrm2[p], be = nrm2[q];
                        double ga = gpart[pr];
#pragma unroll
                        for (int part = 1; part < JNP; ++part) ga += gpart[part * np + pr];
                        if (al > floor2 && be > floor2 && ga * ga > tol * tol * al * be) {
                            // zeta = (be - al) / (2 ga) in FP32 after a power-of-two scaling
                            // that brings 2 ga to [1, 2) (no FP64 divide)
                            const double g2 = 2.0 * ga;
                            const int eg = (__double2hiint(g2) >> 20) & 0x7ff;
                            const double sc = __hiloint2double((2046 - eg) << 20, 0);
                            const float zf = __fdividef((float)((be - al) * sc), (float)(g2 * sc));
                            const float az = fabsf(zf);
                            const float tf32 = az < 1e18f ? copysignf(1.f, zf) / (az + __fsqrt_rn(fmaf(zf, zf, 1.f)))
                                                          : 0.5f / zf;
                            const double t = (double)tf32;
                            const double x = fma(t, t, 1.0), hx = -0.5 * x;
                            double c = (double)rsqrtf((float)x);
                            c = c * fma(hx * c, c, 1.5);
                            c = c * fma(hx * c, c, 1.5);
                            const double sn = c * t, tg = t * ga;
                            cpar[pr] = c;
                            spar[pr] = sn;
                            // Rutishauser's updates (approximate for the FP32 angle; the next
                            // Gram check recomputes the norms exactly)
                            nrm2[p] = fmax(al - tg, 0.0);
                            nrm2[q] = be + tg;
                            doit = tf32 != 0.f;
                        }
                    }
                    act[pr] = doit;
                }
            }
            __syncthreads();
            // (3) rotations
            for (int e = tid; e < np * s; e += nt) {
                const int pr = e / s, i = e - pr * s;
                if (!act[pr]) continue;
                int p, q;
                rr_pair(round, pr, sp, p, q);
                const double c = cpar[pr], sn = spar[pr];
                const double a = A[i + p * s], b = A[i + q * s];
                A[i + p * s] = c * a - sn * b;
                A[i + q * s] = sn * a + c * b;
                if (ACC) {
                    const double va = V[i + p * s], vb = V[i + q * s];
                    V[i + p * s] = c * va - sn * vb;
                    V[i + q * s] = sn * va + c * vb;
                }
            }
            __syncthreads();
        }
    }
    if (nsweeps) *nsweeps = sweeps;
    return steps;
}

// One step of the polar iteration with its second-order term: X = Y (I + E)^(-1/2) ~
// Y (I - E / 2 + 3 E^2 / 8) with Y = double(V32), E = Y^T Y - I (|E| ~ s 2^-24 for an FP32
// product of rotations, so the E^3 term is below FP64 rounding; E^2 in FP32).  Y, Z: s x s FP64
// scratch; X receives the result and may hold V32 itself (V32 is copied out before X is used
// for the FP32 copies of E and E^2).
__device__ void polar_step(const float *V32, double *X, double *Y, double *Z, int s) {
    const int tid = threadIdx.x, nt = blockDim.x, ss = s * s;
    for (int e = tid; e < ss; e += nt) Y[e] = (double)V32[e];
    __syncthreads();
    float *ef = reinterpret_cast<float *>(X), *e2f = ef + ss;
    for (int e = tid; e < ss; e += nt) {
        const int i = e % s, j = e / s;
        if (i > j) continue;
        double t = 0.0;
        for (int k = 0; k < s; ++k) t = fma(Y[k + i * s], Y[k + j * s], t);
        const double ev = t - ((i == j) ? 1.0 : 0.0);
        Z[i + j * s] = ev;
        Z[j + i * s] = ev;
        ef[i + j * s] = (float)ev;
        ef[j + i * s] = (float)ev;
    }
    __syncthreads();
    for (int e = tid; e < ss; e += nt) {
        const int i = e % s, j = e / s;
        float acc = 0.f;
        for (int k = 0; k < s; ++k) acc = fmaf(ef[i + k * s], ef[k + j * s], acc);
        e2f[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < ss; e += nt) {
        const int i = e % s, j = e / s;
        Z[e] = ((i == j) ? 1.0 : 0.0) - 0.5 * Z[e] + 0.375 * (double)e2f[e];
    }
    __syncthreads();
    for (int e = tid; e < ss; e += nt) {
        const int i = e % s, j = e / s;
        double t = 0.0;
        for (int k = 0; k < s; ++k) t = fma(Y[i + k * s], Z[k + j * s], t);
        X[e] = t;   // X's FP32 contents were last read before the previous barrier
    }
    __syncthreads();
}

// SVD of a small square matrix R (upper triangle read) to FP64 accuracy.  Two modes:
//
// ST-HOSVD (J.perm set): R comes from the column-pivoted QR C^T P = Q R of a core unfolding;
// one-sided Jacobi runs on the columns of R^T (row-graded R: high relative accuracy and few
// sweeps, after Drmac and Veselic).  R^T V = U S needs no V: the left singular vectors of
// C = P R^T Q^T are P times the normalised final columns U.
//
// Pseudo-inverse (jobs.pinv set; R from an unpivoted QR): Jacobi on R with V accumulated;
// R^+ = sum_c V[:,c] A[:,c]^T / sigma_c^2 over sigma_c > rcond sigma_max.
//
// Both: the bulk of the Jacobi work runs in FP32 (~60x the FP64 rate on this part) on B
// scaled by a power of two; two Newton-Schulz steps V <- V (3 I - V^T V) / 2 in FP64 restore
// the orthonormality of the FP32 V (error e -> 1.5 e^2); FP64 sweeps on A = B V finish.
// Shared memory: three s x s FP64 regions X | Y | Z (X holds the FP32 A and V in phase 1,
// Z the packed Gram matrix in phase 4).
__global__ void __launch_bounds__(1024) k_svd(const __grid_constant__ SVDJobs jobs) {
    extern __shared__ double sm[];
    const SVDJob &J = jobs.j[blockIdx.x];
    const int s = J.s, ss = s * s;
    double *X = sm, *Y = sm + ss, *Z = sm + 2 * ss;
    __shared__ double sig[SVD_MAXS];
    __shared__ double rsig[SVD_MAXS];
    __shared__ long long skey[SVD_MAXS];
    __shared__ int order[SVD_MAXS];
    __shared__ int flag;
    __shared__ float fscr[40];
    __shared__ int iscr[40];
    __shared__ double nrm64[SVD_MAXS];
    __shared__ float nrm32[SVD_MAXS];
    __shared__ double gpart[JNP * (SVD_MAXS / 2 + 1)];
    __shared__ double cpar[SVD_MAXS / 2 + 1], spar[SVD_MAXS / 2 + 1];
    __shared__ int act[SVD_MAXS / 2 + 1];
    __shared__ int kept;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    auto Rat = [&](int i, int c) -> double {
        return (i <= c && i < J.ldr) ? J.R[i + (long long)c * J.ldr] : 0.0;
    };
    const bool graded = J.perm != nullptr;
    // B = R^T (graded) or R
    auto Bat = [&](int i, int c) -> double { return graded ? Rat(c, i) : Rat(i, c); };
    float *A32 = reinterpret_cast<float *>(X), *V32 = A32 + ss;
    // power-of-two scale from the largest biased exponent (integer work only)
    int emax = 0;
    for (int e = tid; e < ss; e += nt) emax = max(emax, (__double2hiint(Bat(e % s, e / s)) >> 20) & 0x7ff);
    emax = min(block_max_i(emax, iscr), 2044);
    const double inv = __hiloint2double((2045 - emax) << 20, 0);       // 2^(1022 - emax)
    const double mx = __hiloint2double((emax + 1) << 20, 0);           // 2^(emax - 1022)
    for (int e = tid; e < ss; e += nt) {
        A32[e] = (float)(Bat(e % s, e / s) * inv);
        V32[e] = (e % s == e / s) ? 1.f : 0.f;
    }
    float frop = 0.f;
    for (int e = tid; e < ss; e += nt) frop = fmaf(A32[e], A32[e], frop);
    __syncthreads();
    const float fro = block_sum_f(frop, fscr);
    // phase 1: FP32 sweeps.  On the graded R^T they resolve singular values far below the
    // largest with relative accuracy; columns below 2^-100 (scaled) are left to FP64.
    const int n32 = jacobi32<false>(A32, V32, nrm32, s, 8.0f * sqrtf((float)s) * 0x1p-24f,
                             graded ? 0x1p-100f : fro * 0x1p-40f, 20, &flag);
    if (tid == 0) g_svd_sweeps[2 * blockIdx.x] = n32;
    // phase 2: V = double(V32), orthonormalised (polar step) into X
    polar_step(V32, X, Y, Z, s);
    // phase 3: A = B V into Y (B triangular: R^T lower, R upper)
    for (int e = tid; e < ss; e += nt) {
        const int i = e % s, j = e / s;
        double t = 0.0;
        if (graded)
            for (int k = 0; k <= i; ++k) t = fma(Bat(i, k), X[k + j * s], t);
        else
            for (int k = i; k < s; ++k) t = fma(Bat(i, k), X[k + j * s], t);
        Y[e] = t;
    }
    __syncthreads();
    // phase 4: FP64 sweeps (V accumulated only when R^+ needs it)
    double *A = Y, *V = graded ? nullptr : X;
    const double fro_r = (double)fro * mx * mx;
    const double floor2 = fro_r * (double)s * s * 0x1p-106;
    const double tol64 = 4.0 * sqrt((double)s) * 0x1p-53;
    // graded mode: X (V no longer needed) holds T, the FP32 scratch aliases the Gram region Z
    int nsw = 0;
    const int n64 = graded
        ? jacobi64<false>(A, nullptr, nrm64, s, tol64, floor2, 16, &flag, gpart, cpar, spar, act, Z, X,
                          reinterpret_cast<float *>(Z), &nsw)
        : jacobi64<true>(A, X, nrm64, s, tol64, floor2, 16, &flag, gpart, cpar, spar, act, Z, nullptr,
                         nullptr, &nsw);
    if (tid == 0) g_svd_sweeps[2 * blockIdx.x + 1] = n64 * 100 + nsw;
    // singular values from the final Gram check's diagonal; descending order by the integer
    // image of the (non-negative) doubles, ties by index
    for (int c = tid; c < s; c += nt) {
        const double v = sqrt(nrm64[c]);
        sig[c] = v;
        skey[c] = __double_as_longlong(v);
        rsig[c] = v > 0.0 ? 1.0 / v : 0.0;
    }
    __syncthreads();
    for (int c = tid; c < s; c += nt) {
        int pos = 0;
        const long long kc = skey[c];
        for (int o = 0; o < s; ++o)
            if (skey[o] > kc || (skey[o] == kc && o < c)) ++pos;
        order[pos] = c;
    }
    __syncthreads();
    // kept rank: smallest r with sum_{pos >= r} sigma_pos^2 <= eps^2 ||C||^2 / d (suffix sums
    // by one warp, SVD_MAXS <= 96 = 3 x 32 positions)
    if (warp == 0) {
        int r = min(s, J.rank_cap);
        if (J.normsq) {
            const double thr = J.eps2_over_d * (*J.normsq);
            double e2[3], suf[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int pos = k * 32 + lane;
                e2[k] = pos < s ? nrm64[order[pos]] : 0.0;
            }
            // suffix sums: within each 32-block by shuffles, then block carries
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                double v = e2[k];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const double u = __shfl_down_sync(0xffffffffu, v, o);
                    if (lane + o < 32) v += u;
                }
                suf[k] = v;
            }
            const double c2 = __shfl_sync(0xffffffffu, suf[2], 0);
            const double c1 = __shfl_sync(0xffffffffu, suf[1], 0) + c2;
            suf[1] += c2;
            suf[0] += c1;
            // candidate r = pos (pos >= 1) when tail[pos] <= thr; smallest such pos
            int best = s;
#pragma unroll
            for (int k = 2; k >= 0; --k) {
                const int pos = k * 32 + lane;
                const unsigned m = __ballot_sync(0xffffffffu, pos >= 1 && pos < s && suf[k] <= thr);
                if (m) best = k * 32 + __ffs(m) - 1;
            }
            r = min(best, J.rank_cap);
        }
        r = max(r, 1);
        if (lane == 0) {
            kept = r;
            if (J.rank) *J.rank = r;
        }
    }
    __syncthreads();
    const int r = kept;
    if (J.sigma)
        for (int c = tid; c < s; c += nt) J.sigma[c] = sig[order[c]];
    if (J.W) {
        if (graded) {
            // W[perm[i], c] = U[i, order[c]], U = A / sigma; columns at rounding level dropped
            const double fl = sqrt(floor2);
            for (int e = tid; e < s * J.wcols; e += nt) {
                const int i = e % s, c = e / s;
                double v = 0.0;
                if (c < r) {
                    const int o = order[c];
                    if (sig[o] > fl) v = A[i + o * s] * rsig[o];
                }
                J.W[J.perm[i] + (long long)c * s] = v;
            }
        } else {
            for (int e = tid; e < s * J.wcols; e += nt) {
                const int i = e % s, c = e / s;
                J.W[e] = (c < r) ? V[i + order[c] * s] : 0.0;
            }
        }
    }
    double *P = jobs.pinv[blockIdx.x];
    if (P && V) {
        // R = U S V^T with U S = A (final):  R^+ = sum_c V[:,c] A[:,c]^T / sig_c^2
        const double cut = jobs.rcond * sig[order[0]];
        for (int e = tid; e < ss; e += nt) {
            const int i = e % s, jj = e / s;
            double t = 0.0;
            for (int c = 0; c < s; ++c) {
                const double sc = sig[c];
                if (sc > cut && sc > 0.0) t += V[i + c * s] * A[jj + c * s] * (rsig[c] * rsig[c]);
            }
            P[i + (long long)jj * s] = t;
        }
    }
}

// Projected Tikhonov with the GCV parameter (Section 4.3) on the least-squares state of k_ls:
// M = Q R (R k x k upper triangle of st.H, ld ldr), Q^T b = st.qtb, rho = ||tail of Q^T b|| =
// *st.res.  SVD of R (the same FP32 sweeps, polar step and FP64 sweeps as k_svd, V kept):
// A = R V has columns sigma_j u_j, so t_j = a_j^T c = sigma_j (U^T b)_j.  GCV over
// lambda_g = sigma_max 10^(-12 + 12 g / 120), g = 0..120 (Golub, Heath and Wahba):
//   G(lambda) = [sum_j (lambda^2 t_j / (sigma_j (sigma_j^2 + lambda^2)))^2 + rho^2]
//               / (m - sum_j sigma_j^2 / (sigma_j^2 + lambda^2))^2,
// smallest value (ties: the smaller lambda).  Then y = V diag(1 / (sigma^2 + lambda^2)) t
// overwrites st.y and ||M y - b|| = (||R y - c||^2 + rho^2)^(1/2) overwrites *st.res.
constexpr int GCV_POINTS = 121;
__global__ void __launch_bounds__(1024) k_tikhonov(LSState st, int ldr, int k, int m, double *lambda_out) {
    extern __shared__ double sm[];
    const int s = k, ss = s * s;
    double *X = sm, *Y = sm + ss, *Z = sm + 2 * ss;
    __shared__ double sig[SVD_MAXS], tv[SVD_MAXS], cvec[SVD_MAXS], yv[SVD_MAXS];
    __shared__ double gval[GCV_POINTS];
    __shared__ double nrm64[SVD_MAXS];
    __shared__ float nrm32[SVD_MAXS];
    __shared__ double gpart[JNP * (SVD_MAXS / 2 + 1)];
    __shared__ double cpar[SVD_MAXS / 2 + 1], spar[SVD_MAXS / 2 + 1];
    __shared__ int act[SVD_MAXS / 2 + 1];
    __shared__ int flag;
    __shared__ float fscr[40];
    __shared__ int iscr[40];
    __shared__ double scr[40];
    __shared__ double lam_s, rho2_s;
    const int tid = threadIdx.x, nt = blockDim.x;
    auto Rat = [&](int i, int c) -> double { return i <= c ? st.H[i + (long long)c * ldr] : 0.0; };
    if (tid == 0) { const double r = *st.res; rho2_s = r * r; }
    for (int i = tid; i < s; i += nt) cvec[i] = st.qtb[i];
    // SVD of R: scaled FP32 sweeps with V, polar step, A = R V, FP64 sweeps with V
    int emax = 0;
    for (int e = tid; e < ss; e += nt) emax = max(emax, (__double2hiint(Rat(e % s, e / s)) >> 20) & 0x7ff);
    emax = min(block_max_i(emax, iscr), 2044);
    const double inv = __hiloint2double((2045 - emax) << 20, 0);
    const double mx = __hiloint2double((emax + 1) << 20, 0);
    float *A32 = reinterpret_cast<float *>(X), *V32 = A32 + ss;
    for (int e = tid; e < ss; e += nt) {
        A32[e] = (float)(Rat(e % s, e / s) * inv);
        V32[e] = (e % s == e / s) ? 1.f : 0.f;
    }
    float frop = 0.f;
    for (int e = tid; e < ss; e += nt) frop = fmaf(A32[e], A32[e], frop);
    __syncthreads();
    const float fro = block_sum_f(frop, fscr);
    jacobi32<false>(A32, V32, nrm32, s, 8.0f * sqrtf((float)s) * 0x1p-24f, fro * 0x1p-40f, 20, &flag);
    polar_step(V32, X, Y, Z, s);
    for (int e = tid; e < ss; e += nt) {
        const int i = e % s, j = e / s;
        double t = 0.0;
        for (int kk = i; kk < s; ++kk) t = fma(Rat(i, kk), X[kk + j * s], t);
        Y[e] = t;
    }
    __syncthreads();
    const double fro_r = (double)fro * mx * mx;
    const double floor2 = fro_r * (double)s * s * 0x1p-106;
    int nsw = 0;
    jacobi64<true>(Y, X, nrm64, s, 4.0 * sqrt((double)s) * 0x1p-53, floor2, 16, &flag, gpart, cpar, spar, act,
                   Z, nullptr, nullptr, &nsw);
    // singular values, t_j = a_j^T c
    for (int j = tid; j < s; j += nt) {
        sig[j] = sqrt(nrm64[j]);
        double t = 0.0;
        for (int i = 0; i < s; ++i) t = fma(Y[i + j * s], cvec[i], t);
        tv[j] = t;
    }
    __syncthreads();
    double smax = 0.0;
    for (int j = 0; j < s; ++j) smax = fmax(smax, sig[j]);
    const double rho2 = rho2_s;
    for (int g = tid; g < GCV_POINTS; g += nt) {
        const double lam = smax * pow(10.0, -12.0 + 12.0 * g / (GCV_POINTS - 1));
        const double l2 = lam * lam;
        double num = rho2, tr = (double)m;
        for (int j = 0; j < s; ++j) {
            const double s2 = sig[j] * sig[j], den = s2 + l2;
            if (sig[j] > 0.0) {
                const double q = l2 * tv[j] / (sig[j] * den);
                num = fma(q, q, num);
                tr -= s2 / den;
            }
        }
        gval[g] = num / (tr * tr);
    }
    __syncthreads();
    if (tid == 0) {
        int best = 0;
        for (int g = 1; g < GCV_POINTS; ++g)
            if (gval[g] < gval[best]) best = g;
        lam_s = smax * pow(10.0, -12.0 + 12.0 * best / (GCV_POINTS - 1));
        if (lambda_out) *lambda_out = lam_s;
    }
    __syncthreads();
    const double l2 = lam_s * lam_s;
    for (int i = tid; i < s; i += nt) {
        double t = 0.0;
        for (int j = 0; j < s; ++j) {
            const double den = sig[j] * sig[j] + l2;
            if (den > 0.0) t = fma(X[i + j * s], tv[j] / den, t);
        }
        yv[i] = t;
        st.y[i] = t;
    }
    __syncthreads();
    double r2 = 0.0;
    for (int i = tid; i < s; i += nt) {
        double t = -cvec[i];
        for (int l = i; l < s; ++l) t = fma(Rat(i, l), yv[l], t);
        r2 = fma(t, t, r2);
    }
    r2 = block_sum(r2, scr);
    if (tid == 0) *st.res = sqrt(r2 + rho2);
}

void tikhonov_gcv(Ctx &c, const LSState &st, int ldr, int k, int m, double *lambda_out) {
    TK_REQUIRE(k >= 1 && k <= SVD_MAXS, "Tikhonov/GCV: at most 96 least-squares columns");
    static std::atomic<bool> attr_set{false};   // set once; idempotent if two threads race
    if (!attr_set) {
        TK_CUDA(cudaFuncSetAttribute(k_tikhonov, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     3 * SVD_MAXS * SVD_MAXS * (int)sizeof(double)));
        attr_set = true;
    }
    c.pre_launch();
    k_tikhonov<<<1, 1024, 3 * (size_t)k * k * sizeof(double), c.st>>>(st, ldr, k, m, lambda_out);
    c.check_launch("tikhonov", 12.0 * k * (double)k * k);
}

// ST-HOSVD SVD (graded mode) on a cluster of SCL CTAs.  The FP32 sweeps are a chain of
// barrier-separated rounds and stay on CTA 0; the FP64 phase after them is dense matrix work
// (polar step, A = B V, Gram checks, first-order corrections), which on one SM runs at one SM's
// FP64 rate.  Here every CTA owns a block of cb = ceil(s / SCL) columns and computes those
// columns of E = Y^T Y - I, of V = Y Z, of A = B V, of H = A^T A, of T and of A (I + D), reading
// the full operand it needs from its peers' shared memory after a cluster barrier.  The control
// decisions (converged, separated) are made identically by every CTA from the gathered flags, so
// all CTAs pass the same cluster barriers.  A check that finds a non-separated pair hands the
// current A to CTA 0, which finishes with sweeps exactly as the single-CTA kernel does.
// Shared memory per CTA: X | Y | Z, s x s doubles each:
//   X: CTA 0's FP32 A and V during the sweeps; afterwards [0, s cb) this CTA's columns (V, then
//      A) and, behind them, an FP32 publish area (s cb floats: columns of E, then of T);
//   Y: full copies (Y = double(V32), then the gathered A);
//   Z: [0, s cb) work columns (E, Z, H, T, D) and, behind them, FP32 full gathers (s^2 floats).
constexpr int SCL = 16;
__global__ void __launch_bounds__(1024) k_svd_cl(const __grid_constant__ SVDJobs jobs) {
    cg::cluster_group cl = cg::this_cluster();
    const int q = (int)cl.block_rank();
    const SVDJob &J = jobs.j[blockIdx.x / SCL];
    extern __shared__ double sm[];
    const int s = J.s, ss = s * s;
    double *X = sm, *Y = sm + ss, *Z = sm + 2 * ss;
    const int cb = (s + SCL - 1) / SCL;
    const int c0 = min(s, q * cb), c1 = min(s, c0 + cb), nc = c1 - c0;
    double *Acol = X;                                            // s x cb (this CTA's columns)
    float *pub = reinterpret_cast<float *>(X + (size_t)s * cb);  // s x cb floats
    double *W_ = Z;                                              // s x cb work columns
    float *full32 = reinterpret_cast<float *>(Z + (size_t)s * cb);   // s x s floats
    __shared__ double dcol[SVD_MAXS], dall[SVD_MAXS];
    __shared__ double sig[SVD_MAXS], rsig[SVD_MAXS];
    __shared__ long long skey[SVD_MAXS];
    __shared__ int order[SVD_MAXS];
    __shared__ int flag, kept, fl_more, fl_bad;
    __shared__ int cflags[2];                                    // published: more, bad
    __shared__ float fscr[40];
    __shared__ int iscr[40];
    __shared__ double nrm64[SVD_MAXS];
    __shared__ float nrm32[SVD_MAXS];
    __shared__ double gpart[JNP * (SVD_MAXS / 2 + 1)];
    __shared__ double cpar[SVD_MAXS / 2 + 1], spar[SVD_MAXS / 2 + 1];
    __shared__ int act[SVD_MAXS / 2 + 1];
    __shared__ double scal[2];                                   // CTA 0: mx, fro
    float2 *const rlog = jobs.rlog[blockIdx.x / SCL];
    unsigned long long *const prog = jobs.prog[blockIdx.x / SCL];
    const int rpc = (s + SCL - 2) / (SCL - 1);                   // rows of V per replaying CTA
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    auto Bat = [&](int i, int c) -> double {                     // B = R^T (lower triangle)
        return (c <= i && c < J.ldr) ? J.R[c + (long long)i * J.ldr] : 0.0;
    };
    auto owner = [&](int col) { return col / cb; };
    // ---- phase 1: CTA 0 runs the scaled FP32 sweeps on A and logs the rotations; CTA q >= 1
    // replays them on rows [(q - 1) rpc, q rpc) of V (in its Z, row-major, ld s + 1) as each
    // sweep is announced, staging the sweep's log in its Y.  The progress word is cleared
    // before any CTA reads it.
    if (q == 0 && tid == 0) *prog = 0ULL;
    cl.sync();
    if (q > 0) {
        const int r0 = min(s, (q - 1) * rpc), r1 = min(s, r0 + rpc);
        replay_rotations(rlog, prog, jobs.tag, s, reinterpret_cast<float *>(Z), r0, r1,
                         reinterpret_cast<float2 *>(Y));
    } else {
        float *A32 = reinterpret_cast<float *>(X);
        int emax = 0;
        // walked in R's storage order (c fastest: coalesced reads of R's rows)
        for (int e = tid; e < ss; e += nt) emax = max(emax, (__double2hiint(Bat(e / s, e % s)) >> 20) & 0x7ff);
        emax = min(block_max_i(emax, iscr), 2044);
        const double inv = __hiloint2double((2045 - emax) << 20, 0);
        float frop = 0.f;                                         // ||A32||_F^2 from the values written
        for (int e = tid; e < ss; e += nt) {
            const int i = e / s, c = e % s;
            const float a = (float)(Bat(i, c) * inv);
            A32[i + c * s] = a;
            frop = fmaf(a, a, frop);
        }
        __syncthreads();
        const float fro = block_sum_f(frop, fscr);
        const int n32 = jacobi32<true>(A32, nullptr, nrm32, s, 8.0f * sqrtf((float)s) * 0x1p-24f, 0x1p-100f,
                                       SVD_LOG_SWEEPS, &flag, rlog, prog, jobs.tag);
        if (tid == 0) {
            g_svd_sweeps[2 * (blockIdx.x / SCL)] = n32;
            scal[0] = __hiloint2double((emax + 1) << 20, 0);
            scal[1] = (double)fro;
        }
    }
    cl.sync();                                                                    // (1) V's rows ready
    // ---- phase 2: Y = double(V) everywhere, each row from the CTA that replayed it; E columns
    {
        for (int e = tid; e < ss; e += nt) {
            const int r = e % s, c = e / s, o = r / rpc;
            Y[e] = (double)reinterpret_cast<const float *>(cl.map_shared_rank(Z, 1 + o))[(r - o * rpc) * (s + 1) + c];
        }
        if (tid < 2) scal[tid] = cl.map_shared_rank(scal, 0)[tid];
    }
    cl.sync();                                                                    // (2) peers' Z free
    const double mx = scal[0], fro = scal[1];
    for (int e = tid; e < s * nc; e += nt) {
        const int i = e % s, jl = e / s, j = c0 + jl;
        double t = 0.0;
        for (int k = 0; k < s; ++k) t = fma(Y[k + i * s], Y[k + j * s], t);
        const double ev = t - (i == j ? 1.0 : 0.0);
        W_[i + jl * s] = ev;
        pub[i + jl * s] = (float)ev;
    }
    cl.sync();                                                                    // (3)
    for (int e = tid; e < ss; e += nt) {                          // gather E (FP32) in full
        const int i = e % s, k = e / s, o = owner(k);
        full32[e] = reinterpret_cast<const float *>(cl.map_shared_rank(X + (size_t)s * cb, o))[i + (k - o * cb) * s];
    }
    __syncthreads();
    for (int e = tid; e < s * nc; e += nt) {                      // Z = I - E / 2 + 3 E^2 / 8
        const int i = e % s, jl = e / s, j = c0 + jl;
        float acc = 0.f;
        for (int k = 0; k < s; ++k) acc = fmaf(full32[i + k * s], full32[k + j * s], acc);
        W_[i + jl * s] = (i == j ? 1.0 : 0.0) - 0.5 * W_[i + jl * s] + 0.375 * (double)acc;
    }
    __syncthreads();
    for (int e = tid; e < s * nc; e += nt) {                      // V columns = Y Z, then A = B V
        const int i = e % s, jl = e / s;
        double t = 0.0;
        for (int k = 0; k < s; ++k) t = fma(Y[i + k * s], W_[k + jl * s], t);
        Acol[i + jl * s] = t;
    }
    __syncthreads();
    for (int e = tid; e < s * nc; e += nt) {
        const int i = e % s, jl = e / s;
        double t = 0.0;
        for (int k = 0; k <= i; ++k) t = fma(Bat(i, k), Acol[k + jl * s], t);
        W_[i + jl * s] = t;
    }
    __syncthreads();
    for (int e = tid; e < s * nc; e += nt) Acol[e] = W_[e];
    // ---- phase 3: Gram checks and first-order corrections, column-parallel
    const double fro_r = fro * mx * mx;
    const double floor2 = fro_r * (double)s * s * 0x1p-106;
    const double tol = 4.0 * sqrt((double)s) * 0x1p-53, chk2 = 16.0 * tol * tol;
    bool sweep_fallback = false;
    for (int step = 0; step <= 16; ++step) {
        cl.sync();                                                                // A columns final
        for (int e = tid; e < ss; e += nt) {                      // gather A in full into Y
            const int i = e % s, k = e / s, o = owner(k);
            Y[e] = cl.map_shared_rank(Acol, o)[i + (k - o * cb) * s];
        }
        __syncthreads();
        for (int e = tid; e < s * nc; e += nt) {                  // H columns
            const int i = e % s, jl = e / s, j = c0 + jl;
            double t = 0.0;
            for (int r = 0; r < s; ++r) t = fma(Y[r + i * s], Y[r + j * s], t);
            W_[i + jl * s] = t;
            if (i == j) dcol[jl] = t;
        }
        __syncthreads();
        cl.sync();                                                                // diagonals published
        for (int j = tid; j < s; j += nt) {
            const int o = owner(j);
            dall[j] = cl.map_shared_rank(dcol, o)[j - o * cb];
        }
        if (tid == 0) { fl_more = 0; fl_bad = 0; }
        __syncthreads();
        for (int e = tid; e < s * nc; e += nt) {                  // T columns and flags
            const int i = e % s, jl = e / s, j = c0 + jl;
            double t = 0.0;
            if (i != j) {
                const double di = dall[i], dj = dall[j], g = W_[i + jl * s];
                if (di > floor2 && dj > floor2 && g * g > chk2 * di * dj) {
                    fl_more = 1;
                    if (fabs(g) <= 1e-3 * fabs(dj - di)) t = g / (dj - di);
                    else fl_bad = 1;
                }
            }
            W_[i + jl * s] = t;
            pub[i + jl * s] = (float)t;
        }
        __syncthreads();
        if (tid == 0) { cflags[0] = fl_more; cflags[1] = fl_bad; }
        cl.sync();                                                                // flags, T published
        int more = 0, bad = 0;
        for (int o = 0; o < SCL; ++o) {
            const int *cf = cl.map_shared_rank(cflags, o);
            more |= cf[0];
            bad |= cf[1];
        }
        if (!more || step == 16) break;
        if (bad) { sweep_fallback = true; break; }
        for (int e = tid; e < ss; e += nt) {                      // gather T (FP32) in full
            const int i = e % s, k = e / s, o = owner(k);
            full32[e] = reinterpret_cast<const float *>(cl.map_shared_rank(X + (size_t)s * cb, o))[i + (k - o * cb) * s];
        }
        __syncthreads();
        for (int e = tid; e < s * nc; e += nt) {                  // D = T + T^2 / 2
            const int i = e % s, jl = e / s, j = c0 + jl;
            float acc = 0.f;
            for (int k = 0; k < s; ++k) acc = fmaf(full32[i + k * s], full32[k + j * s], acc);
            W_[i + jl * s] += 0.5 * (double)acc;
        }
        __syncthreads();
        double r[SVD_REGS];
#pragma unroll
        for (int k = 0; k < SVD_REGS; ++k) {                      // A columns <- A + A D
            const int e = tid + k * nt;
            r[k] = 0.0;
            if (e < s * nc) {
                const int i = e % s, jl = e / s;
                double acc = Acol[e];
                for (int kk = 0; kk < s; ++kk) acc = fma(Y[i + kk * s], W_[kk + jl * s], acc);
                r[k] = acc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < SVD_REGS; ++k) {
            const int e = tid + k * nt;
            if (e < s * nc) Acol[e] = r[k];
        }
    }
    // ---- tail on CTA 0 (Y holds the gathered A of the last check)
    if (q == 0) {
        if (sweep_fallback) {
            int nsw = 0;
            jacobi64<false>(Y, nullptr, nrm64, s, tol, floor2, 16, &flag, gpart, cpar, spar, act, Z, nullptr,
                            nullptr, &nsw);
            for (int j = tid; j < s; j += nt) dall[j] = nrm64[j];
            __syncthreads();
        }
        for (int c = tid; c < s; c += nt) {
            const double v = sqrt(fmax(dall[c], 0.0));
            sig[c] = v;
            skey[c] = __double_as_longlong(v);
            rsig[c] = v > 0.0 ? 1.0 / v : 0.0;
        }
        __syncthreads();
        for (int c = tid; c < s; c += nt) {
            int pos = 0;
            const long long kc = skey[c];
            for (int o = 0; o < s; ++o)
                if (skey[o] > kc || (skey[o] == kc && o < c)) ++pos;
            order[pos] = c;
        }
        __syncthreads();
        if (warp == 0) {
            int r = min(s, J.rank_cap);
            if (J.normsq) {
                const double thr = J.eps2_over_d * (*J.normsq);
                double suf[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int pos = k * 32 + lane;
                    double v = pos < s ? fmax(dall[order[pos]], 0.0) : 0.0;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const double u = __shfl_down_sync(0xffffffffu, v, o);
                        if (lane + o < 32) v += u;
                    }
                    suf[k] = v;
                }
                const double c2 = __shfl_sync(0xffffffffu, suf[2], 0);
                const double c1 = __shfl_sync(0xffffffffu, suf[1], 0) + c2;
                suf[1] += c2;
                suf[0] += c1;
                int best = s;
#pragma unroll
                for (int k = 2; k >= 0; --k) {
                    const int pos = k * 32 + lane;
                    const unsigned msk = __ballot_sync(0xffffffffu, pos >= 1 && pos < s && suf[k] <= thr);
                    if (msk) best = k * 32 + __ffs(msk) - 1;
                }
                r = min(best, J.rank_cap);
            }
            r = max(r, 1);
            if (lane == 0) {
                kept = r;
                if (J.rank) *J.rank = r;
            }
        }
        __syncthreads();
        const int r = kept;
        if (J.sigma)
            for (int c = tid; c < s; c += nt) J.sigma[c] = sig[order[c]];
        if (J.W) {
            const double fl = sqrt(floor2);
            for (int e = tid; e < s * J.wcols; e += nt) {
                const int i = e % s, c = e / s;
                double v = 0.0;
                if (c < r) {
                    const int o = order[c];
                    if (sig[o] > fl) v = Y[i + o * s] * rsig[o];
                }
                J.W[J.perm[i] + (long long)c * s] = v;
            }
        }
    }
    cl.sync();   // keep shared memory alive until every peer has finished reading it
}

static void svd_launch(Ctx &c, SVDJobs &J, int smax) {
    const size_t smem = 3 * (size_t)smax * smax * sizeof(double);
    static std::atomic<bool> attr_set{false};   // set once; idempotent if two threads race
    if (!attr_set) {
        TK_CUDA(cudaFuncSetAttribute(k_svd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     3 * SVD_MAXS * SVD_MAXS * (int)sizeof(double)));
        attr_set = true;
    }
    c.pre_launch();
    // 1024 threads: enough for one Gram-check dot product per thread and for every FP32 pair
    // group (at most 48 pairs at s = 96)
    k_svd<<<J.n, 1024, smem, c.st>>>(J);
    // algorithmic work: Golub and Van Loan's count for the singular values and one set of
    // singular vectors of an s x s matrix, 12 s^3
    double flops = 0.0;
    for (int i = 0; i < J.n; ++i) flops += 12.0 * J.j[i].s * (double)J.j[i].s * J.j[i].s;
    c.check_launch("svd", flops);
}

static void svd_cl_launch(Ctx &c, SVDJobs &J, int smax) {
    const size_t smem = 3 * (size_t)smax * smax * sizeof(double);
    // rotation logs of the FP32 phase (released with the mark: later work on this stream runs
    // after the kernel)
    ScopedMark mark(*c.arena);
    for (int i = 0; i < J.n; ++i) {
        const int sp = J.j[i].s + (J.j[i].s & 1);
        J.rlog[i] = static_cast<float2 *>(
            c.arena->alloc_bytes((size_t)SVD_LOG_SWEEPS * (sp - 1) * (sp / 2) * sizeof(float2)));
        J.prog[i] = static_cast<unsigned long long *>(c.arena->alloc_bytes(sizeof(unsigned long long)));
    }
    // a progress word left by an earlier launch carries another id (ids repeat after 2^32 launches)
    static std::atomic<unsigned> launch_id{0};
    J.tag = (unsigned long long)(launch_id.fetch_add(1) + 1) << 32;
    static std::atomic<bool> attr_set{false};   // set once; idempotent if two threads race
    if (!attr_set) {
        TK_CUDA(cudaFuncSetAttribute(k_svd_cl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     3 * SVD_MAXS * SVD_MAXS * (int)sizeof(double)));
        TK_CUDA(cudaFuncSetAttribute(k_svd_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        attr_set = true;
    }
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)(SCL * J.n), 1, 1);
    cfg.blockDim = dim3(1024, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = SCL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    c.pre_launch();
    TK_CUDA(cudaLaunchKernelEx(&cfg, k_svd_cl, J));
    double flops = 0.0;
    for (int i = 0; i < J.n; ++i) flops += 12.0 * J.j[i].s * (double)J.j[i].s * J.j[i].s;
    c.check_launch("svd", flops);
}

void svd_jacobi(Ctx &c, const std::vector<SVDJob> &jobs) {
    // graded (ST-HOSVD) jobs of at least 2 SCL columns: the clustered kernel
    bool all_graded = !jobs.empty();
    for (const SVDJob &j : jobs) all_graded = all_graded && j.perm != nullptr && j.s >= 16;
    if (all_graded) {
        for (size_t base = 0; base < jobs.size(); base += TK_MAX_D) {
            SVDJobs J{};
            J.n = (int)std::min<size_t>(TK_MAX_D, jobs.size() - base);
            int smax = 1;
            for (int i = 0; i < J.n; ++i) {
                J.j[i] = jobs[base + i];
                TK_REQUIRE(J.j[i].s <= SVD_MAXS, "SVD: size must be 1..96");
                smax = std::max(smax, J.j[i].s);
            }
            svd_cl_launch(c, J, smax);
        }
        return;
    }
    for (size_t base = 0; base < jobs.size(); base += TK_MAX_D) {
        SVDJobs J{};
        J.n = (int)std::min<size_t>(TK_MAX_D, jobs.size() - base);
        int smax = 1;
        for (int i = 0; i < J.n; ++i) {
            J.j[i] = jobs[base + i];
            TK_REQUIRE(J.j[i].s <= SVD_MAXS && J.j[i].s >= 1, "SVD: size must be 1..96");
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
        j.rank = nullptr; j.normsq = nullptr; j.eps2_over_d = 0.0; j.rank_cap = s; j.perm = nullptr;
        J.pinv[i] = out[i];
    }
    J.rcond = rcond;
    TK_REQUIRE(s <= SVD_MAXS, "pinv: size must be <= 96");
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

// Incremental Householder least squares in compact WY form (Schreiber and Van Loan): the
// product H_0 ... H_{c-1} of the stored reflectors is I - V T V^T, V unit lower trapezoidal
// (column j: 1 in row j, v_j below), T upper triangular, grown by one column per reflector:
// T[0:c, c] = -tau_c T[0:c, 0:c] (V^T v_c), T[c][c] = tau_c.  A new column h is reduced as
// Q^T h = h - V (T^T (V^T h)): three matrix-vector products whose loads are all independent,
// instead of c reflector steps each waiting on the previous one.  Reflectors, tau and Q^T b are
// stored exactly as by the sequential form, so either form may continue the other's state.
// Back substitution (k <= LSW_BSK): R packed into shared memory, one warp, rows across lanes.
constexpr int LSW_BSK = 96;
constexpr int LSW_SHM = LSW_BSK * (LSW_BSK + 1) / 2;           // >= LSW_MAXS + 2 LSW_MAXK
static_assert(LSW_SHM >= LSW_MAXS + 2 * LSW_MAXK, "shared work area too small");
__global__ void __launch_bounds__(512) k_ls_wy(const double *M, const double *b, int s, int c0, int k,
                                               LSState st, int init_qtb) {
    __shared__ double shm[LSW_SHM];
    __shared__ double scratch[40];
    __shared__ double bc[4];
    double *hs = shm, *z = shm + LSW_MAXS, *u = z + LSW_MAXK;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5, nt = blockDim.x;
    double *H = st.H, *T = st.T;
    const long long ldt = st.ldt;
    if (init_qtb)
        for (int i = tid; i < s; i += nt) st.qtb[i] = b[i];
    for (int col = c0; col < k; ++col) {
        for (int i = tid; i < s; i += nt) hs[i] = M[i + (long long)col * s];
        __syncthreads();
        if (col > 0) {
            // z = V^T h: a warp per reflector, rows across lanes (v_j: 1 in row j, stored below)
            for (int j = warp; j < col; j += nw) {
                const double *v = H + (long long)j * s;
                double p = 0.0;
                for (int i = j + lane; i < s; i += 32) p = fma(i == j ? 1.0 : v[i], hs[i], p);
                p = warp_sum(p);
                if (lane == 0) z[j] = p;
            }
            __syncthreads();
            // u = T^T z
            for (int j = tid; j < col; j += nt) {
                const double *tc = T + j * ldt;
                double a = 0.0;
                for (int i = 0; i <= j; ++i) a = fma(tc[i], z[i], a);
                u[j] = a;
            }
            __syncthreads();
            // h -= V u
            for (int i = tid; i < s; i += nt) {
                const int jm = min(i, col - 1);
                double a = 0.0;
                for (int j = 0; j <= jm; ++j) a = fma(j == i ? 1.0 : H[i + (long long)j * s], u[j], a);
                hs[i] -= a;
            }
            __syncthreads();
        }
        // reflector of h[col:]
        double p = 0.0;
        for (int i = col + 1 + tid; i < s; i += nt) p = fma(hs[i], hs[i], p);
        p = block_sum(p, scratch);
        if (tid == 0) {
            double tau, beta, scal;
            householder(hs[col], p, tau, beta, scal);
            bc[0] = tau; bc[1] = scal; bc[2] = beta;
            st.tau[col] = tau;
        }
        __syncthreads();
        const double tau = bc[0], scal = bc[1], beta = bc[2];
        for (int i = col + 1 + tid; i < s; i += nt) hs[i] *= scal;
        __syncthreads();
        for (int i = tid; i < s; i += nt) H[i + (long long)col * s] = (i == col) ? beta : hs[i];
        // new column of T from y = V^T v_col (rows >= col of the earlier reflectors)
        if (col > 0) {
            for (int j = warp; j < col; j += nw) {
                const double *v = H + (long long)j * s;
                double q = 0.0;
                for (int i = col + lane; i < s; i += 32) q = fma(v[i], i == col ? 1.0 : hs[i], q);
                q = warp_sum(q);
                if (lane == 0) z[j] = q;
            }
            __syncthreads();
            for (int i = tid; i < col; i += nt) {
                double a = 0.0;
                for (int l = i; l < col; ++l) a = fma(T[i + l * ldt], z[l], a);
                T[i + col * ldt] = -tau * a;
            }
        }
        if (tid == 0) T[col + col * ldt] = tau;
        // Q^T b: the new reflector
        double q = 0.0;
        for (int i = col + tid; i < s; i += nt) q = fma(i == col ? 1.0 : hs[i], st.qtb[i], q);
        q = block_sum(q, scratch);
        const double f = tau * q;
        for (int i = col + tid; i < s; i += nt) st.qtb[i] -= (i == col ? 1.0 : hs[i]) * f;
        __syncthreads();
    }
    // back substitution R y = (Q^T b)[0:k]
    if (k <= LSW_BSK) {
        double *Rp = shm;                                        // packed upper triangle
        for (int e = tid; e < k * k; e += nt) {
            const int i = e % k, j = e / k;
            if (i <= j) Rp[j * (j + 1) / 2 + i] = H[i + (long long)j * s];
        }
        __syncthreads();
        if (warp == 0) {
            constexpr int RPL = (LSW_BSK + 31) / 32;             // rows per lane
            double cv[RPL], dr[RPL];
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const int i = lane + 32 * r;
                cv[r] = i < k ? st.qtb[i] : 0.0;
                const double d = i < k ? Rp[i * (i + 1) / 2 + i] : 0.0;
                dr[r] = d != 0.0 ? 1.0 / d : 0.0;               // a zero pivot gives y_j = 0
            }
            for (int j = k - 1; j >= 0; --j) {
                const int rj = j >> 5;
                double own = 0.0;
#pragma unroll
                for (int r = 0; r < RPL; ++r)
                    if (r == rj) own = cv[r] * dr[r];
                const double yj = __shfl_sync(0xffffffffu, own, j & 31);
                if (lane == (j & 31)) st.y[j] = yj;
                const double *rc = Rp + j * (j + 1) / 2;
#pragma unroll
                for (int r = 0; r < RPL; ++r) {
                    const int i = lane + 32 * r;
                    if (i < j) cv[r] = fma(-rc[i], yj, cv[r]);
                }
            }
        }
    } else {
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
    }
    double r = 0.0;
    for (int i = k + tid; i < s; i += nt) r = fma(st.qtb[i], st.qtb[i], r);
    r = block_sum(r, scratch);
    if (tid == 0) *st.res = sqrt(r);
}

void ls_update(Ctx &c, const double *M, const double *b, int s, int c0, int k, const LSState &st,
               int init_qtb) {
    TK_REQUIRE(s >= 1 && s <= 4096 && k >= 1 && k < s + 1, "least squares: bad size");
    c.pre_launch();
    if (st.T && s <= LSW_MAXS && k <= LSW_MAXK && k <= st.ldt)
        k_ls_wy<<<1, 512, 0, c.st>>>(M, b, s, c0, k, st, init_qtb);
    else
        k_ls<<<1, 512, 0, c.st>>>(M, b, s, c0, k, st, init_qtb);
    // new columns c0 .. k-1: each takes the earlier reflectors (4 s j flops) and its own
    c.check_launch("ls", 2.0 * s * ((double)k * k - (double)c0 * c0) + 4.0 * s * (k - c0));
}

}  // namespace tk
