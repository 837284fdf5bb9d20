// Grouped FP64 GEMM for the Tucker contractions (factor sketches U^T S, the range finder
// Y_k = sum_i U_k^(i) Z_k^(i), projections U^_k^T U_k^(i), mode products of the core).
//
// One launch runs up to GEMM_MAXPROB problems, each a sum over up to GEMM_MAXSEG segments
// (so a sum of Tucker terms reduces over the concatenated K without atomics).  Tiles are
// 32 x 32 with 256 threads, 2 x 2 FP64 outputs per thread (warps outside a partial tile idle).  Problems whose reduction
// dimension is long relative to their tile count split K over a thread-block cluster of
// up to 8 CTAs (the factor chosen per problem, so that small grids still occupy the SMs); the
// partial tiles are summed through distributed shared memory in a fixed rank order, so results
// are deterministic run to run.
#include <cooperative_groups.h>

#include <algorithm>

#include "tk_internal.cuh"

namespace cg = cooperative_groups;

namespace tk {

constexpr int BM = 32, BN = 32, BK = 16;

__global__ void __launch_bounds__(256) k_gemm_group(const __grid_constant__ GGroup g, int ksplit) {
    const int blk = blockIdx.x / ksplit;
    const int part = blockIdx.x % ksplit;
    int pi = 0;
    while (pi + 1 < g.nprob && blk >= g.p[pi + 1].tile_begin) ++pi;
    const GProb &P = g.p[pi];
    int t = blk - P.tile_begin;
    const int per_batch = P.tiles_m * P.tiles_n;
    const int b = t / per_batch;
    t -= b * per_batch;
    const int m0 = (t % P.tiles_m) * BM;
    const int n0 = (t / P.tiles_m) * BN;

    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    __shared__ double red[BM][BN + 1];

    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    // Every thread owns a 2 x 2 block.  A warp spans either 4 rows x 32 columns (rows split
    // across warps) or 32 rows x 4 columns; the tile takes the split along its shorter valid
    // extent, and a warp whose rows (columns) all lie outside C skips the FMAs: an FP64 warp
    // instruction costs the same whatever its lanes hold, and the sketch width r + p rarely
    // fills the last tile (37 = 32 + 5).
    const int mv = min(BM, P.M - m0), nv = min(BN, P.N - n0);
    const bool colsplit = nv < mv;
    const int r0 = colsplit ? tx * 2 : ty * 2, c0 = colsplit ? ty * 2 : tx * 2;
    const bool active = (colsplit ? (tid >> 5) * 4 < nv : (tid >> 5) * 4 < mv);
    double acc00 = 0, acc01 = 0, acc10 = 0, acc11 = 0;

    // split-K: part `part` of `ksplit` takes an equal share of the concatenated reduction
    // (all segments end to end), so short segments are not cut into mostly empty slabs
    int ktot = 0;
    for (int si = 0; si < P.nseg; ++si) ktot += P.seg[si].K;
    const int kcs = (ktot + ksplit - 1) / ksplit;
    const int kg0 = part * kcs, kg1 = min(ktot, kg0 + kcs);
    int koff = 0;
    for (int si = 0; si < P.nseg; ++si) {
        const GSeg &S = P.seg[si];
        const int kb = max(kg0 - koff, 0), ke = min(kg1 - koff, S.K);
        koff += S.K;
        if (kb >= ke) continue;   // uniform across the CTA
        const double cf = S.coef * (S.coef_dev ? *S.coef_dev : 1.0);
        const double *A = S.A + (long long)b * P.sA;
        const double *B = S.B + (long long)b * P.sB;
        for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
            for (int rep = 0; rep < 2; ++rep) {
                const int e = tid + rep * 256;
                int mm, kk;
                if (P.ta == 0) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
                const int gm = m0 + mm, gk = k0 + kk;
                double v = 0.0;
                if (gm < P.M && gk < ke)
                    v = P.ta == 0 ? A[gm + (long long)gk * S.lda] : A[gk + (long long)gm * S.lda];
                As[kk][mm] = v * cf;
                int nn;
                if (P.tb == 0) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
                const int gn = n0 + nn, gk2 = k0 + kk;
                double w = 0.0;
                if (gn < P.N && gk2 < ke)
                    w = P.tb == 0 ? B[gk2 + (long long)gn * S.ldb] : B[gn + (long long)gk2 * S.ldb];
                Bs[kk][nn] = w;
            }
            __syncthreads();
            if (active) {
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    const double a0 = As[kk][r0], a1 = As[kk][r0 + 1];
                    const double b0 = Bs[kk][c0], b1 = Bs[kk][c0 + 1];
                    acc00 = fma(a0, b0, acc00);
                    acc01 = fma(a0, b1, acc01);
                    acc10 = fma(a1, b0, acc10);
                    acc11 = fma(a1, b1, acc11);
                }
            }
            __syncthreads();
        }
    }

    double *C = P.C + (long long)b * P.sC;
    if (ksplit == 1) {
        const double acc[2][2] = {{acc00, acc01}, {acc10, acc11}};
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int gm = m0 + r0 + i, gn = n0 + c0 + j;
                if (gm < P.M && gn < P.N) {
                    double *c = C + gm + (long long)gn * P.ldc;
                    *c = P.beta == 0.0 ? acc[i][j] : fma(P.beta, *c, acc[i][j]);
                }
            }
        return;
    }
    // split-K: reduce partial tiles across the cluster in rank order
    cg::cluster_group cl = cg::this_cluster();
    red[r0][c0] = acc00;
    red[r0][c0 + 1] = acc01;
    red[r0 + 1][c0] = acc10;
    red[r0 + 1][c0 + 1] = acc11;
    cl.sync();
    const int rows = BM / ksplit;
    for (int e = tid; e < rows * BN; e += 256) {
        const int row = part * rows + e / BN, col = e % BN;
        double s = 0.0;
        for (int q = 0; q < ksplit; ++q) s += cl.map_shared_rank(&red[row][col], q)[0];
        const int gm = m0 + row, gn = n0 + col;
        if (gm < P.M && gn < P.N) {
            double *c = C + gm + (long long)gn * P.ldc;
            *c = P.beta == 0.0 ? s : fma(P.beta, *c, s);
        }
    }
    cl.sync();
}

void Gemm::add(int M, int N, int ta, int tb, double *C, int ldc, double beta,
               const std::vector<Seg> &segs, int batch, long long sA, long long sB, long long sC) {
    if (M <= 0 || N <= 0 || batch <= 0) return;
    // chunk segments: first chunk uses beta, later chunks accumulate (beta = 1)
    size_t i = 0;
    bool first = true;
    do {
        GProb p{};
        p.M = M; p.N = N; p.ta = ta; p.tb = tb; p.ldc = ldc;
        p.batch = batch; p.sA = sA; p.sB = sB; p.sC = sC; p.C = C;
        p.beta = first ? beta : 1.0;
        p.nseg = 0;
        for (; i < segs.size() && p.nseg < GEMM_MAXSEG; ++i) {
            if (segs[i].K <= 0) continue;
            GSeg &g = p.seg[p.nseg++];
            g.A = segs[i].A; g.B = segs[i].B; g.K = segs[i].K;
            g.lda = segs[i].lda; g.ldb = segs[i].ldb;
            g.coef = segs[i].coef; g.coef_dev = segs[i].coef_dev;
        }
        p.tiles_m = (M + BM - 1) / BM;
        p.tiles_n = (N + BN - 1) / BN;
        if (!first && p.nseg == 0) break;
        pending_.push_back(p);   // later chunks of the same C run in later waves (see run())
        first = false;
    } while (i < segs.size());
}

void Gemm::flush_group(std::vector<GProb> &probs, int ksplit) {
    if (probs.empty()) return;
    for (size_t base = 0; base < probs.size(); base += GEMM_MAXPROB) {
        GGroup g{};
        g.nprob = (int)std::min<size_t>(GEMM_MAXPROB, probs.size() - base);
        int tiles = 0;
        for (int j = 0; j < g.nprob; ++j) {
            g.p[j] = probs[base + j];
            g.p[j].tile_begin = tiles;
            tiles += g.p[j].tiles_m * g.p[j].tiles_n * g.p[j].batch;
        }
        g.total = tiles;
        double flops = 0.0;
        for (int j = 0; j < g.nprob; ++j)
            for (int q = 0; q < g.p[j].nseg; ++q)
                flops += 2.0 * g.p[j].M * (double)g.p[j].N * g.p[j].seg[q].K * g.p[j].batch;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)(tiles * ksplit), 1, 1);
        cfg.blockDim = dim3(256, 1, 1);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = c_.st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = ksplit;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        c_.pre_launch();
        TK_CUDA(cudaLaunchKernelEx(&cfg, k_gemm_group, g, ksplit));
        c_.check_launch(tag_, flops);
    }
    probs.clear();
}

void Gemm::run() {
    // Problems writing the same C (segment chunks) must run in order: split the pending list
    // into waves where no C repeats.
    std::vector<std::vector<GProb>> waves(1);
    std::vector<double *> seen;
    for (const GProb &p : pending_) {
        if (std::find(seen.begin(), seen.end(), p.C) != seen.end()) {
            waves.emplace_back();
            seen.clear();
        }
        seen.push_back(p.C);
        waves.back().push_back(p);
    }
    for (const std::vector<GProb> &wave : waves) {
        if (tc_) {
            std::vector<GProb> oz, rest;
            for (const GProb &p : wave) (oz_supported(p) ? oz : rest).push_back(p);
            gemm_oz(c_, oz, tag_);
            if (rest.empty()) continue;
            flush_group(rest, 1);
            continue;
        }
        // a small grid runs each tile's BK-slab chain on an otherwise idle SM: split K (powers
        // of two, BM divisible by the factor) while the wave's grid stays within two CTAs per
        // SM, each problem only as far as every part keeps at least 8 of its reduction
        long long tiles = 0;
        for (const GProb &p : wave) tiles += (long long)p.tiles_m * p.tiles_n * p.batch;
        int wmax = 0;
        while (wmax < 3 && tiles * (2LL << wmax) <= 2LL * c_.num_sms) ++wmax;
        std::vector<GProb> by_split[4];            // split factors 1, 2, 4, 8
        for (const GProb &p : wave) {
            long long ktot = 0;
            for (int s = 0; s < p.nseg; ++s) ktot += p.seg[s].K;
            int w = 0;
            while (w < wmax && ktot >= 8LL * (2 << w)) ++w;
            by_split[w].push_back(p);
        }
        for (int w = 3; w >= 0; --w) flush_group(by_split[w], 1 << w);
    }
    pending_.clear();
}

}  // namespace tk
