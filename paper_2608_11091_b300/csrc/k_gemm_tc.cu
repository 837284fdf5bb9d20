// Tensor-core GEMM of the mixed-precision form (tcgen05, sm_103a): C = beta C + coef op(A) op(B)
// with FP64 operands, BF16 products and FP32 accumulation in tensor memory.
//
// Each FP64 operand is split on the fly into up to three BF16 pieces x = hi + mid + lo (8 bits
// each, 24 bits together), and the products hi*hi, hi*mid, mid*hi, ... whose scale is within
// 2^-24 of the leading one are accumulated, so the result carries about FP32 accuracy.  The
// Gaussian sketch matrices of the mixed form are rounded to BF16 when drawn, so they need one
// piece.  Operands are converted by the CTA's threads straight into shared memory in the
// K-major, no-swizzle canonical layout (core matrices of 8 rows x 16 bytes; K-adjacent core
// matrices 128 B apart, row-adjacent 256 B apart); one thread issues the MMAs (M = 128,
// N <= 128, K = 16 each) and commits them to an mbarrier; the 128 threads read the FP32
// accumulator back from tensor memory (one row per thread).  Long reductions split K over a
// cluster of up to 8 CTAs and sum the partial tiles through distributed shared memory in
// rank order (deterministic).  Every mbarrier wait is bounded: on timeout the kernel records
// an error in g_tc_error, skips the tensor-memory reads and still frees its tensor memory.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>

#include <atomic>

#include "tk_internal.cuh"

namespace cg = cooperative_groups;

namespace tk {

__device__ int g_tc_error;

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 32, TC_KSTEPS = TC_BK / 16;
constexpr int TC_TILE_A = 128 * 16 * 2;             // bytes of one 128 x 16 BF16 sub-tile
constexpr int TC_TILE_B = TC_BN * 16 * 2;
constexpr int TC_PIECE_A = TC_KSTEPS * TC_TILE_A;   // bytes per BF16 piece of the A chunk
constexpr int TC_PIECE_B = TC_KSTEPS * TC_TILE_B;
constexpr int TC_SMEM_OPS = 3 * TC_PIECE_A + 3 * TC_PIECE_B;
constexpr int TC_SMEM_RED = TC_BM * (TC_BN + 1) * 4;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
    return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;    // leading (K) byte offset
    d |= (uint64_t)(256 >> 4) << 32;    // stride (row) byte offset
    d |= (uint64_t)1 << 46;             // tcgen05 descriptor version; no swizzle
    return d;
}

// x = hi + mid + lo in BF16 (from the FP32 rounding of x)
__device__ __forceinline__ void split3(double x, __nv_bfloat16 &hi, __nv_bfloat16 &mid, __nv_bfloat16 &lo) {
    const float xf = (float)x;
    hi = __float2bfloat16_rn(xf);
    const float r1 = xf - __bfloat162float(hi);
    mid = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(mid);
    lo = __float2bfloat16_rn(r2);
}

struct TcGroup {
    int nprob;
    TcProb p[GEMM_MAXPROB];
};

__global__ void __launch_bounds__(128) k_gemm_tc(const __grid_constant__ TcGroup g, int ksplit) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char *sA = tc_smem;
    unsigned char *sB = tc_smem + 3 * TC_PIECE_A;
    float *red = reinterpret_cast<float *>(tc_smem + TC_SMEM_OPS);
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t taddr_s;
    __shared__ int failed_s;

    const int blk = blockIdx.x / ksplit, part = blockIdx.x % ksplit;
    int pi = 0;
    while (pi + 1 < g.nprob && blk >= g.p[pi + 1].tile_begin) ++pi;
    const TcProb &P = g.p[pi];
    const int t = blk - P.tile_begin;
    const int m0 = (t % P.tiles_m) * TC_BM, n0 = (t / P.tiles_m) * TC_BN;
    const int nmma = min(TC_BN, ((min(TC_BN, P.N - n0) + 15) / 16) * 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)), "r"(TC_BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        failed_s = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = taddr_s;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nmma >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);

    const int kc = (P.K + ksplit - 1) / ksplit;
    const int kb = part * kc, ke = min(P.K, kb + kc);
    uint32_t phase = 0;
    bool any = false;
    for (int k0 = kb; k0 < ke; k0 += TC_BK) {
        // A chunk: rows m0..m0+127, k0..k0+31
        for (int e = tid; e < TC_BM * TC_BK; e += 128) {
            int row, kk;
            if (P.ta) { kk = e % TC_BK; row = e / TC_BK; } else { row = e % TC_BM; kk = e / TC_BM; }
            const int gm = m0 + row, gk = k0 + kk;
            double v = 0.0;
            if (gm < P.M && gk < ke) v = P.ta ? P.A[gk + (long long)gm * P.lda] : P.A[gm + (long long)gk * P.lda];
            __nv_bfloat16 h, m, l;
            split3(v * P.coef, h, m, l);
            const uint32_t off = (kk >> 4) * TC_TILE_A + kmajor_off(row, kk & 15);
            *reinterpret_cast<__nv_bfloat16 *>(sA + off) = h;
            if (P.na > 1) *reinterpret_cast<__nv_bfloat16 *>(sA + TC_PIECE_A + off) = m;
            if (P.na > 2) *reinterpret_cast<__nv_bfloat16 *>(sA + 2 * TC_PIECE_A + off) = l;
        }
        // B chunk (as N x K K-major): columns n0..n0+127, k0..k0+31
        for (int e = tid; e < TC_BN * TC_BK; e += 128) {
            int col, kk;
            if (P.tb) { col = e % TC_BN; kk = e / TC_BN; } else { kk = e % TC_BK; col = e / TC_BK; }
            const int gn = n0 + col, gk = k0 + kk;
            double v = 0.0;
            if (gn < P.N && gk < ke) v = P.tb ? P.B[gn + (long long)gk * P.ldb] : P.B[gk + (long long)gn * P.ldb];
            __nv_bfloat16 h, m, l;
            split3(v, h, m, l);
            const uint32_t off = (kk >> 4) * TC_TILE_B + kmajor_off(col, kk & 15);
            *reinterpret_cast<__nv_bfloat16 *>(sB + off) = h;
            if (P.nb > 1) *reinterpret_cast<__nv_bfloat16 *>(sB + TC_PIECE_B + off) = m;
            if (P.nb > 2) *reinterpret_cast<__nv_bfloat16 *>(sB + 2 * TC_PIECE_B + off) = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const int npc = max(P.na, P.nb);
            for (int ks = 0; ks < TC_KSTEPS; ++ks)
                for (int ia = 0; ia < P.na; ++ia)
                    for (int ib = 0; ib < P.nb; ++ib) {
                        if (ia + ib >= npc) continue;
                        const uint64_t da = smem_desc(smem_u32(sA + ia * TC_PIECE_A + ks * TC_TILE_A));
                        const uint64_t db = smem_desc(smem_u32(sB + ib * TC_PIECE_B + ks * TC_TILE_B));
                        const uint32_t acc = any ? 1u : 0u;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
                                     "l"(da), "l"(db), "r"(idesc), "r"(acc));
                        any = true;
                    }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar)));
        }
        any = true;
        // bounded wait for the MMAs of this chunk (frees the shared-memory operands)
        int ok = 0;
        for (long it = 0; it < (1L << 22); ++it) {
            uint32_t done;
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(done) : "r"(smem_u32(&mbar)), "r"(phase));
            if (done) { ok = 1; break; }
        }
        if (!ok) failed_s = 1;
        phase ^= 1;
        __syncthreads();
        if (failed_s) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = warp * 32 + lane;
    const bool have = any && !failed_s;
    if (failed_s && tid == 0) atomicExch(&g_tc_error, 1);
    double *C = P.C;
    if (ksplit == 1) {
        for (int c0 = 0; c0 < nmma; c0 += 8) {
            uint32_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (have) {
                const uint32_t a = taddr + ((uint32_t)(warp * 32) << 16) + c0;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7]) : "r"(a));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            }
            const int gm = m0 + row;
            for (int j = 0; j < 8; ++j) {
                const int gn = n0 + c0 + j;
                if (gm < P.M && gn < P.N) {
                    double *c = C + gm + (long long)gn * P.ldc;
                    const double v = (double)__uint_as_float(r[j]);
                    *c = P.beta == 0.0 ? v : fma(P.beta, *c, v);
                }
            }
        }
    } else {
        cg::cluster_group cl = cg::this_cluster();
        for (int c0 = 0; c0 < TC_BN; c0 += 8) {
            uint32_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (have && c0 < nmma) {
                const uint32_t a = taddr + ((uint32_t)(warp * 32) << 16) + c0;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7]) : "r"(a));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            }
            for (int j = 0; j < 8; ++j) red[row * (TC_BN + 1) + c0 + j] = __uint_as_float(r[j]);
        }
        cl.sync();
        const int rows = TC_BM / ksplit;
        for (int e = tid; e < rows * TC_BN; e += 128) {
            const int rr = part * rows + e / TC_BN, col = e % TC_BN;
            double s = 0.0;
            for (int q = 0; q < ksplit; ++q) s += (double)cl.map_shared_rank(red, q)[rr * (TC_BN + 1) + col];
            const int gm = m0 + rr, gn = n0 + col;
            if (gm < P.M && gn < P.N) {
                double *c = C + gm + (long long)gn * P.ldc;
                *c = P.beta == 0.0 ? s : fma(P.beta, *c, s);
            }
        }
        cl.sync();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_BN));
}

void gemm_tc(Ctx &c, const std::vector<TcProb> &probs) {
    if (probs.empty()) return;
    static std::atomic<bool> attr_set{false};   // set once; idempotent if two threads race
    if (!attr_set) {
        TK_CUDA(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_OPS + TC_SMEM_RED));
        attr_set = true;
    }
    // long reductions with few tiles split K over a cluster; others run one CTA per tile
    std::vector<TcProb> split, plain;
    for (TcProb p : probs) {
        p.tiles_m = (p.M + TC_BM - 1) / TC_BM;
        p.tiles_n = (p.N + TC_BN - 1) / TC_BN;
        if (p.K >= 256 && p.tiles_m * p.tiles_n * 8 <= 4 * c.num_sms) split.push_back(p); else plain.push_back(p);
    }
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<TcProb> &v = pass == 0 ? split : plain;
        const int ksplit = pass == 0 ? 8 : 1;
        for (size_t base = 0; base < v.size(); base += GEMM_MAXPROB) {
            TcGroup G{};
            G.nprob = (int)std::min<size_t>(GEMM_MAXPROB, v.size() - base);
            int tiles = 0;
            double flops = 0.0;
            for (int j = 0; j < G.nprob; ++j) {
                G.p[j] = v[base + j];
                G.p[j].tile_begin = tiles;
                tiles += G.p[j].tiles_m * G.p[j].tiles_n;
                flops += 2.0 * G.p[j].M * (double)G.p[j].N * G.p[j].K;
            }
            cudaLaunchConfig_t cfg{};
            cfg.gridDim = dim3((unsigned)(tiles * ksplit), 1, 1);
            cfg.blockDim = dim3(128, 1, 1);
            cfg.dynamicSmemBytes = TC_SMEM_OPS + (ksplit > 1 ? TC_SMEM_RED : 0);
            cfg.stream = c.st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = ksplit;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            c.pre_launch();
            TK_CUDA(cudaLaunchKernelEx(&cfg, k_gemm_tc, G, ksplit));
            c.check_launch("gemm_tc", flops);
        }
    }
}

int tc_error_flag(bool reset) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (reset && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
    }
    return v;
}

}  // namespace tk
