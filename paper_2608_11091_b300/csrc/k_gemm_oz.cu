// Tensor-core GEMM of the mixed-precision form (tcgen05 + TMA, sm_103a):
//   C = beta C + sum_s coef_s op(A_s) op(B_s)      (FP64 operands and result)
// computed from BF16 products with FP32 accumulation, exactly, on integer slices of the
// operands (the splitting of Ozaki, Ogita, Oishi and Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012), restated here for BF16 tensor cores:
//
//  * Slicing (k_oz_split).  Per row m of an operand and per chunk c of 256 reduction indices,
//    e = the exponent with max_k |x_mk| < 2^e.  x = 2^(e - 7) (d_0 + d_1 2^-8 + ... + d_4 2^-32)
//    + O(2^(e - 40)) with integer digits |d_p| <= 128 (the balanced base-256 expansion of the
//    nearest integer to x 2^(39 - e)), each exactly representable in BF16.  Digits are written as
//    five BF16 planes, K contiguous.
//  * Products.  For digit planes p of A and q of B, sum_k d_p g_q over a chunk of 256 is an
//    integer; grouping the products by level L = p + q (<= 4, 15 products), each level's sum
//    is at most (L + 1) 256 2^14 <= 2^24 in magnitude, so the FP32 accumulation in tensor memory
//    is exact.  Products with p + q > 4 are dropped: the error is about 2^-40 relative to
//    max|A row| max|B column| per reduction index.  One MMA per A plane p and 16-wide K step
//    covers every level at once: B's planes q = 0..4-p are one operand of N = 32 (5 - p) rows,
//    and the accumulator starts at level p's columns, so plane q's block lands on level p + q.
//  * Accumulation.  Per chunk the epilogue combines the levels exactly in 64-bit integers,
//    sum_L S_L 2^(8(4 - L)), and forms 2^(e_m + f_n - 46) times it as an FP64 value with integer
//    operations (the FP64 pipe of this part is slow), adding it to the output in FP64 registers
//    when a CTA has more than one chunk; then C = beta C + acc.
//
// Pipeline (k_gemm_oz, one 128 x 32 output tile per CTA or a cluster of up to 8 CTAs splitting
// its reduction, 18 warps): warp 16 lane 0 issues the TMA loads (five A planes 128 x 64 and five
// B planes 32 x 64 per K slab of 64, 128-byte swizzle) into a two-stage ring; warp 17 lane 0
// issues the tcgen05.mma (M 128, K 16, five per K step) into two alternating sets of five
// accumulators in tensor memory; warps 0-15 read a finished set back (tcgen05.ld, a quarter of
// the columns each) while the next chunk is multiplied; a split reduction pushes each rank's
// partial rows into the ring of the rank that adds them.  mbarriers: full / empty per stage,
// accumulator full / empty per set.  Every wait has an iteration limit: on expiry the kernel
// records an error in g_oz_error and all roles stop issuing work; the CTA waits (bounded) for
// its own copies and MMAs before freeing its tensor memory.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "tk_internal.cuh"

namespace tk {

__device__ int g_oz_error;

constexpr int OZ_S = 5;                               // digit planes per operand
constexpr int OZ_L = OZ_S;                            // accumulator levels L = p + q = 0..4
constexpr int OZ_BM = 128, OZ_BN = 32, OZ_BK = 64;    // tile and K slab
constexpr int OZ_CHUNK = 256;                         // reduction indices per exact chunk
constexpr int OZ_SLABS = OZ_CHUNK / OZ_BK;            // slabs per chunk
constexpr int OZ_MAXCHUNK = 16;                       // K <= 4096
constexpr int OZ_A_TILE = OZ_BM * OZ_BK * 2;          // 16 KB
constexpr int OZ_B_TILE = OZ_BN * OZ_BK * 2;          // 4 KB
constexpr int OZ_STAGE = OZ_S * (OZ_A_TILE + OZ_B_TILE);
constexpr int OZ_STAGES = 2;
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE + 1024;  // + alignment slack
constexpr int OZ_TMEM_COLS = 512;                     // 2 sets x 5 levels x 32 columns
constexpr int OZ_SET_COLS = OZ_L * OZ_BN;
constexpr int OZ_EPI_WARPS = 16;                      // epilogue: TMEM lane quarter x column quarter
constexpr int OZ_EPI_THREADS = 32 * OZ_EPI_WARPS;
constexpr int OZ_THREADS = OZ_EPI_THREADS + 64;       // then the TMA producer warp and the MMA warp
constexpr int OZ_WARP_TMA = OZ_EPI_WARPS, OZ_WARP_MMA = OZ_EPI_WARPS + 1;
constexpr long OZ_SPIN = 1L << 20;                    // bounded waits

// ------------------------------------------------------------------------------------------
// Slicing
// ------------------------------------------------------------------------------------------
struct OzSeg {
    const double *p, *cd;
    double coef;
    int K, ld, koff;
};

// One operand side: `rows` logical rows (A: M x batch folded, B: N) by the concatenated K of
// the segments; element (m, k) of segment s at local index kk is, with i = m % a, b = m / a,
// p[i + ld kk + bstride b] (trans = 0) or p[kk + ld i + bstride b] (trans = 1), times coef (and
// *cd when set).
struct OzSide {
    int rows, a, trans, nseg, Kpad, Rpad;
    long long bstride;
    OzSeg seg[GEMM_MAXSEG];
    __nv_bfloat16 *planes;   // [OZ_S][Rpad][Kpad]
    short *exps;             // [nchunk][Rpad]
};

constexpr int OZ_MAXSIDES = 24;
struct OzSides {
    int n;
    OzSide s[OZ_MAXSIDES];
};

// grid (row blocks of 32, chunks, sides); 256 threads; tile 32 rows x (up to) 256 in dynamic
// shared memory (row stride OZ_CHUNK + 1), chunk c covering [256 c, min(256 c + 256, Kpad)).
// Integer arithmetic on the FP64 bit patterns throughout (the FP64 pipe is slow on this part):
// e = the largest exponent field of the row's chunk minus 1022 (so |v| < 2^e); X = the nearest
// integer to v 2^(39 - e), |X| < 2^39, from the 53-bit significand by a rounding shift; the
// digits are X's balanced base-256 expansion, X = d_0 2^32 + d_1 2^24 + ... + d_4, |d_p| <= 128.
constexpr int OZ_SPLIT_LD = OZ_CHUNK + 1;
constexpr int OZ_SPLIT_SMEM = 32 * OZ_SPLIT_LD * 8;
__global__ void __launch_bounds__(256) k_oz_split(const __grid_constant__ OzSides S) {
    const OzSide &D = S.s[blockIdx.z];
    const int r0 = blockIdx.x * 32, c = blockIdx.y, k0 = c * OZ_CHUNK;
    if (r0 >= D.Rpad || k0 >= D.Kpad) return;
    const int W = min(OZ_CHUNK, D.Kpad - k0);        // a multiple of 64
    extern __shared__ long long oz_tile[];
    auto t = [&](int r, int kk) -> long long & { return oz_tile[r * OZ_SPLIT_LD + kk]; };
    __shared__ int er[32];                           // row index i within its batch, later the exponents
    __shared__ long long rowoff[32];                  // per row: bstride b (+ i when not transposed)
    __shared__ double segscale[GEMM_MAXSEG];         // per segment: coef (* *cd)
    __shared__ int segunit[GEMM_MAXSEG];             // per segment: the scale is 1 (no FP64 multiply)
    __shared__ short segk[OZ_CHUNK];                 // per reduction index of the chunk: its segment, -1 past K
    const int tid = threadIdx.x;
    // the row offsets and the segment scales once per block, not per element (integer division
    // and FP64 multiplies are slow per element on this part)
    if (tid < 32) {
        const int m = r0 + tid;
        const int i = m % D.a, b = m / D.a;
        rowoff[tid] = (long long)b * D.bstride + (D.trans ? 0LL : (long long)i);
        er[tid] = i;
    }
    if (tid < D.nseg) {
        const double sc = D.seg[tid].coef * (D.seg[tid].cd ? *D.seg[tid].cd : 1.0);
        segscale[tid] = sc;
        segunit[tid] = sc == 1.0;
    }
    for (int kk = tid; kk < OZ_CHUNK; kk += 256) {
        const int k = k0 + kk;
        int sg = -1;
        for (int s = 0; s < D.nseg; ++s)
            if (k >= D.seg[s].koff && k < D.seg[s].koff + D.seg[s].K) sg = s;
        segk[kk] = (short)sg;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    // source of element (r, kk) and its segment, or null (padding)
    auto src_of = [&](int r, int kk, int &sg) -> const double * {
        sg = 0;
        if (r0 + r >= D.rows || kk >= W) return nullptr;
        const int s = segk[kk];
        if (s < 0) return nullptr;
        sg = s;
        const OzSeg &g = D.seg[s];
        const int kl = k0 + kk - g.koff;
        const double *src = g.p + rowoff[r];
        return D.trans ? src + kl + (long long)g.ld * er[r] : src + (long long)g.ld * kl;
    };
    // a batch of eight elements per thread: every address first, then the eight loads together
    // (the segment search would otherwise keep one load in flight), then scale and store
    auto batch = [&](const int (&rr)[8], const int (&kc)[8]) {
        const double *src[8];
        int sg[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) src[u] = src_of(rr[u], kc[u], sg[u]);
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = src[u] ? *src[u] : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (kc[u] >= W) continue;
            if (src[u] && !segunit[sg[u]]) v[u] *= segscale[sg[u]];
            t(rr[u], kc[u]) = __double_as_longlong(v[u]);
        }
    };
    // coalesced: a warp walks a row along the reduction index (transposed storage) or the 32
    // rows of one reduction index (rows contiguous)
    if (D.trans) {
        for (int r = warp; r < 32; r += 8) {
            int rr[8], kc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) { rr[u] = r; kc[u] = lane + 32 * u; }
            batch(rr, kc);
        }
    } else {
        for (int kk0 = warp; kk0 < W; kk0 += 64) {
            int rr[8], kc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) { rr[u] = lane; kc[u] = kk0 + 8 * u; }
            batch(rr, kc);
        }
    }
    __syncthreads();
    {
        // er[] now takes the exponents: every read of it as a row index happened before the barrier
        for (int r = warp; r < 32; r += 8) {
            int ef = 0;
            for (int kk = lane; kk < W; kk += 32) ef = max(ef, (int)((t(r, kk) >> 52) & 0x7FF));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ef = max(ef, __shfl_xor_sync(0xffffffffu, ef, o));
            // exponent field E: |v| < 2^(E - 1022) for every v of the row (0 for an all-zero
            // or subnormal row, whose digits are then 0)
            if (lane == 0) {
                er[r] = ef;
                D.exps[(long long)c * D.Rpad + r0 + r] = (short)(ef > 0 ? ef - 1022 : 0);
            }
        }
    }
    __syncthreads();
    // digits, two adjacent reduction indices per thread (one packed BF16 pair per plane).  X is
    // signed, |X| <= 2^39 (a 53-bit significand shifted right by at least 14).  With
    // Y = X + 0x80808080 the bytes of Y's low word are d_p + 128 for p = 4, 3, 2, 1 (byte 0 up;
    // the balanced digits, in [-128, 127]) and Y >> 32 is d_0 (|d_0| <= 128): adding 128 at every
    // digit position turns the balanced expansion into Y's plain one.  A byte permutation puts
    // byte u into the float 2^23 + u, and one exact subtraction of 2^23 + 128 gives the digit
    const long long plane = (long long)D.Rpad * D.Kpad;
    auto digits = [&](long long bits, int ew, float (&d)[OZ_S]) {
        const int ef = (int)((unsigned long long)bits >> 52) & 0x7FF;
        long long X = 0;
        if (ef > 0) {
            // |v| 2^(39 - e) = m 2^(ef - 1075 + 39 - e) with m the significand, e = E - 1022:
            // a right shift by E + 14 - ef >= 14 with rounding to nearest
            const long long m = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
            const int sh = ew + 14 - ef;
            if (sh < 63) X = (m + (1LL << (sh - 1))) >> sh;
            if (bits < 0) X = -X;
        }
        const long long Y = X + 0x80808080LL;
        const unsigned lo = (unsigned)Y;
        d[0] = (float)(int)(Y >> 32);
#pragma unroll
        for (int p = 1; p < OZ_S; ++p)
            d[p] = __uint_as_float(__byte_perm(lo, 0x4B000000u, 0x7540u + (unsigned)(OZ_S - 1 - p))) - 8388736.f;
    };
    const int Wh = W >> 1;
    for (int e = tid; e < 32 * Wh; e += 256) {
        const int r = e / Wh, kk = 2 * (e % Wh);
        float da[OZ_S], db[OZ_S];
        digits(t(r, kk), er[r], da);
        digits(t(r, kk + 1), er[r], db);
        __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>(D.planes + (long long)(r0 + r) * D.Kpad + k0 + kk);
#pragma unroll
        for (int p = 0; p < OZ_S; ++p)
            dst[(p * plane) >> 1] = __floats2bfloat162_rn(da[p], db[p]);
    }
}

// ------------------------------------------------------------------------------------------
// Main kernel
// ------------------------------------------------------------------------------------------
struct OzProb {                                       // CUtensorMap carries its own alignment
    CUtensorMap tmA, tmB;                            // 3-D: (K, rows, plane), BF16, 128-B swizzle
    const short *expA, *expB;
    double *C;
    double beta;
    long long sC;
    int M, N, a, ldc, RpadA, RpadB, nslab, nchunk;
    int tiles_m, tiles_n, tile_begin;
};

constexpr int OZ_MAXPROB = 12;
struct OzGroup {
    OzProb p[OZ_MAXPROB];
    int nprob;
    int ks;                                           // K split: CTAs per tile (one cluster)
};

__device__ __forceinline__ uint32_t oz_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t parity) {
    for (long it = 0; it < OZ_SPIN; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// RN(x) 2^ex for an integer |x| < 2^62, built with integer operations (the FP64 pipe is slow on
// this part): the same value as RN((double)x) * 2^ex, which is exact, whenever the result is a
// normal number; outside that range the library path (never inlined, so the common path stays
// branch-free)
__device__ __noinline__ double oz_scaled_slow(long long x, int ex) { return ldexp((double)x, ex); }
__device__ __forceinline__ double oz_scaled(long long x, int ex) {
    if (x == 0) return 0.0;
    const unsigned long long sgn = (unsigned long long)x & (1ULL << 63);
    const unsigned long long u = x < 0 ? 0ULL - (unsigned long long)x : (unsigned long long)x;
    const int lz = __clzll((long long)u);
    const int E = 63 - lz + ex + 1023;                  // biased exponent of the leading bit
    if (E < 1 || E > 2045) return oz_scaled_slow(x, ex);
    const unsigned long long t = u << lz;                // leading bit at 63
    const unsigned long long hi = t >> 11, rem = t & 0x7FFULL;
    // to nearest, ties to even; a carry to 2^53 moves into the exponent field below
    const unsigned long long mnt = hi + ((rem + 0x3FFULL + (hi & 1ULL)) >> 11);
    return __longlong_as_double((long long)(sgn | (((unsigned long long)(E - 1) << 52) + mnt)));
}

// K-major operand tile in shared memory with 128-byte swizzle (8 rows x 128 B atoms)
__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;      // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                // descriptor version
    d |= (uint64_t)2 << 61;                // 128-byte swizzle
    return d;
}

__global__ void __launch_bounds__(OZ_THREADS, 1) k_gemm_oz(const __grid_constant__ OzGroup g) {
    extern __shared__ unsigned char oz_dyn[];
    __shared__ __align__(8) uint64_t bar_full[OZ_STAGES], bar_empty[OZ_STAGES], bar_accf[2], bar_acce[2];
    __shared__ uint32_t taddr_s;
    __shared__ int stop_s;
    __shared__ int fex[OZ_MAXCHUNK][OZ_BN];   // column exponents f_n per chunk

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // a tile's reduction is split over the g.ks CTAs of its cluster: rank r takes the chunks
    // [r nchunk / ks, (r + 1) nchunk / ks) (possibly none) and the partial tiles are added in rank
    // order at the end
    const int ks = g.ks, tile_id = (int)blockIdx.x / ks, rank = (int)blockIdx.x % ks;
    int pi = 0;
    while (pi + 1 < g.nprob && tile_id >= g.p[pi + 1].tile_begin) ++pi;
    const OzProb &P = g.p[pi];
    // the output's parameters in registers: P lives in parameter space behind a dynamic index,
    // and a load through it could otherwise be repeated after every store to C
    double *const Cout = P.C;
    const double beta = P.beta;
    const long long sC = P.sC;
    const int Mout = P.M, Nout = P.N, afold = P.a, ldc = P.ldc, RpadA = P.RpadA;
    const short *const expA = P.expA;
    const int t = tile_id - P.tile_begin;
    const int m0 = (t % P.tiles_m) * OZ_BM, n0 = (t / P.tiles_m) * OZ_BN;
    const int c_lo = (rank * P.nchunk) / ks, c_hi = ((rank + 1) * P.nchunk) / ks;
    const int k_lo = c_lo * OZ_SLABS, nk = max(0, min(c_hi * OZ_SLABS, P.nslab) - k_lo);
    const uint32_t base = (oz_smem(oz_dyn) + 1023u) & ~1023u;   // 1024-aligned stage ring

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(oz_smem(&taddr_s)), "r"(OZ_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < OZ_STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_smem(&bar_full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_smem(&bar_empty[s])));
        }
        for (int s = 0; s < 2; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_smem(&bar_accf[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(oz_smem(&bar_acce[s])), "r"(OZ_EPI_THREADS));
        }
        stop_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = tid; e < P.nchunk * OZ_BN; e += blockDim.x) {
        const int c = e / OZ_BN, j = e % OZ_BN;
        fex[c][j] = P.expB[(long long)c * P.RpadB + n0 + j];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = taddr_s;
    int issued_slabs = 0;       // producer / MMA progress, for the bounded drain at exit

    // epilogue role (warps 0-15): one output row and 8 columns per thread (a warp reads the TMEM
    // lanes of its quarter, warp & 3, and the column quarter warp >> 2)
    constexpr int NH = OZ_BN / (OZ_EPI_WARPS / 4);       // columns per epilogue thread
    static_assert(NH == 8, "the epilogue's tensor-memory loads are .x8");
    const int q4 = warp & 3, h = (warp >> 2) % (OZ_EPI_WARPS / 4);
    const int row = q4 * 32 + lane, m = m0 + row;
    double acc[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) acc[j] = 0.0;
    if (warp == OZ_WARP_TMA) {
        // ---------------- TMA producer
        if (lane == 0) {
            for (int kl = 0; kl < nk; ++kl) {
                const int s = kl % OZ_STAGES, k = k_lo + kl;
                if (kl >= OZ_STAGES && !oz_wait(oz_smem(&bar_empty[s]), ((kl / OZ_STAGES) - 1) & 1)) {
                    stop_s = 1;
                    break;
                }
                if (*(volatile int *)&stop_s) break;
                const uint32_t fb = oz_smem(&bar_full[s]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(OZ_STAGE) : "memory");
                const uint32_t st = base + s * OZ_STAGE;
                for (int p = 0; p < OZ_S; ++p) {
                    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                                 ::"r"(st + p * OZ_A_TILE), "l"((uint64_t)&P.tmA), "r"(k * OZ_BK), "r"(m0), "r"(p), "r"(fb)
                                 : "memory");
                    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                                 ::"r"(st + OZ_S * OZ_A_TILE + p * OZ_B_TILE), "l"((uint64_t)&P.tmB), "r"(k * OZ_BK),
                                   "r"(n0), "r"(p), "r"(fb)
                                 : "memory");
                }
                issued_slabs = kl + 1;
            }
            // drain: wait (bounded) until every issued copy has landed before the CTA exits
            for (int k = max(0, issued_slabs - OZ_STAGES); k < issued_slabs; ++k)
                oz_wait(oz_smem(&bar_full[k % OZ_STAGES]), (k / OZ_STAGES) & 1);
        }
    } else if (warp == OZ_WARP_MMA) {
        // ---------------- MMA issuer.  One MMA per A digit plane p and 16-wide K step: B's planes
        // q = 0..4-p lie one after another in shared memory (32 rows each, the same 1024-byte
        // row-group stride), so together they are one operand of N = 32 (5 - p) rows, and with D
        // starting at level p's columns the product block of plane q lands on level p + q.  Five
        // wide MMAs instead of fifteen of N = 32 (a small MMA costs its issue, not its math)
        if (lane == 0) {
            uint32_t idesc[OZ_S];
#pragma unroll
            for (int p = 0; p < OZ_S; ++p)
                idesc[p] = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((OZ_BN * (OZ_S - p)) >> 3) << 17) |
                           ((uint32_t)(OZ_BM >> 4) << 24);
            bool ok = true;
            for (int kl = 0; kl < nk && ok; ++kl) {
                const int s = kl % OZ_STAGES, c = kl / OZ_SLABS, set = c & 1;   // c: local chunk
                if (kl % OZ_SLABS == 0 && c >= 2 && !oz_wait(oz_smem(&bar_acce[set]), ((c / 2) - 1) & 1)) ok = false;
                if (ok && !oz_wait(oz_smem(&bar_full[s]), (kl / OZ_STAGES) & 1)) ok = false;
                if (!ok || *(volatile int *)&stop_s) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t st = base + s * OZ_STAGE;
                // descriptors of the stage's first A and B tiles; every other operand is a
                // constant byte offset from them, added to the start-address field (address >> 4,
                // 14 bits: shared addresses stay below 256 KB, so the field cannot carry)
                const uint64_t dA0 = oz_desc(st), dB0 = oz_desc(st + OZ_S * OZ_A_TILE);
                const uint32_t d0 = taddr + set * OZ_SET_COLS;
                const uint32_t first = (kl % OZ_SLABS == 0) ? 1u : 0u;   // first slab of a chunk
#pragma unroll
                for (int kk = 0; kk < OZ_BK / 16; ++kk)
#pragma unroll
                    for (int p = 0; p < OZ_S; ++p) {
                        const uint64_t da = dA0 + (uint64_t)((p * OZ_A_TILE + kk * 32) >> 4);
                        const uint64_t db = dB0 + (uint64_t)((kk * 32) >> 4);
                        // the first MMA of a chunk (p = 0 covers every level) overwrites
                        const uint32_t acc = (kk == 0 && p == 0) ? (first ^ 1u) : 1u;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                     ::"r"(d0 + (uint32_t)(p * OZ_BN)), "l"(da), "l"(db), "r"(idesc[p]), "r"(acc));
                    }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(oz_smem(&bar_empty[s])) : "memory");
                if (kl % OZ_SLABS == OZ_SLABS - 1 || kl == nk - 1)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 ::"r"(oz_smem(&bar_accf[set])) : "memory");
                issued_slabs = kl + 1;
            }
            if (!ok) stop_s = 1;
            // drain: the last commit tracks every MMA issued; wait (bounded) for it
            if (issued_slabs > 0) {
                const int kl = issued_slabs - 1;
                oz_wait(oz_smem(&bar_empty[kl % OZ_STAGES]), (kl / OZ_STAGES) & 1);
            }
        }
    } else {
        // ---------------- epilogue.  The levels of a chunk combine exactly in 64-bit integers
        // (S_L integer, |S_L| < 2^24: sum_L S_L 2^(8(4-L)) < 2^59); the chunk value is formed
        // with integer operations
        bool ok = true;
        for (int cl = 0; cl < c_hi - c_lo; ++cl) {
            const int set = cl & 1, c = c_lo + cl;
            // warp-uniform outcome: the tensor-memory loads below are .sync.aligned
            const bool arrived = __all_sync(0xffffffffu, oz_wait(oz_smem(&bar_accf[set]), (cl / 2) & 1));
            if (!arrived) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int em = expA[(long long)c * RpadA + m];
            // the five level loads issued together, one wait
            uint32_t r[OZ_L][NH];
#pragma unroll
            for (int L = 0; L < OZ_L; ++L) {
                const uint32_t a = taddr + ((uint32_t)(q4 * 32) << 16) + set * OZ_SET_COLS + L * OZ_BN + h * NH;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(r[L][0]), "=r"(r[L][1]), "=r"(r[L][2]), "=r"(r[L][3]), "=r"(r[L][4]), "=r"(r[L][5]),
                               "=r"(r[L][6]), "=r"(r[L][7])
                             : "r"(a));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(oz_smem(&bar_acce[set])) : "memory");
#pragma unroll
            for (int j = 0; j < NH; ++j) {
                long long ai = 0;
#pragma unroll
                for (int L = 0; L < OZ_L; ++L)
                    ai += (long long)__float2int_rn(__uint_as_float(r[L][j])) << (8 * (OZ_L - 1 - L));
                // chunk value 2^(e_m + f_n) 2^-32 ai with the final 2^-14: 2^(e_m + f_n - 46) ai; the
                // first chunk of the CTA is its value, later ones one FP64 addition
                const double v = oz_scaled(ai, em + fex[c][h * NH + j] - 46);
                acc[j] = cl == 0 ? v : acc[j] + v;
            }
        }
        if (!ok) stop_s = 1;
        if (ks == 1) {
            // folded rows: m = i + a b  ->  C + i + ldc n + sC b; a warp stores 32 consecutive
            // rows of a column.  With beta != 0 every old value is loaded before the first store,
            // so the loads are in flight together
            if (ok && m < Mout) {
                const int i = m % afold, b = m / afold;
                double *Cr = Cout + i + (long long)b * sC + (long long)ldc * (n0 + h * NH);
                const int nn = min(NH, Nout - n0 - h * NH);
                if (beta != 0.0) {
#pragma unroll
                    for (int j = 0; j < NH; ++j)
                        if (j < nn) acc[j] = fma(beta, Cr[(long long)ldc * j], acc[j]);
                }
#pragma unroll
                for (int j = 0; j < NH; ++j)
                    if (j < nn) Cr[(long long)ldc * j] = acc[j];
            }
        }
    }
    if (ks > 1) {
        // split reduction: rank o adds rows [o nr, (o + 1) nr), nr = BM / ks.  Each rank pushes
        // the partial rows into the stage ring of the rank that adds them (remote stores do not
        // wait), slot `rank` of a [ks][BN][nr] buffer; the owner then adds its ks slots in rank
        // order from its own shared memory
        namespace cg = cooperative_groups;
        cg::cluster_group cl = cg::this_cluster();
        const int nr = OZ_BM / ks;
        cl.sync();                        // every rank is past its main loop: the rings are free
        if (warp < OZ_EPI_WARPS) {
            const int o = row / nr, lr = row - o * nr;
#pragma unroll
            for (int j = 0; j < NH; ++j) {
                const uint32_t off = (uint32_t)(((rank * OZ_BN + h * NH + j) * nr + lr) * 8);
                uint32_t ra;
                asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(base + off), "r"(o));
                asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(acc[j]) : "memory");
            }
        }
        cl.sync();                        // every partial has arrived
        const double *buf = reinterpret_cast<const double *>(oz_dyn + (base - oz_smem(oz_dyn)));
        const bool live = !*(volatile int *)&stop_s;
        for (int e = tid; e < nr * OZ_BN; e += OZ_THREADS) {
            const int lr = e % nr, j = e / nr, mm = m0 + rank * nr + lr, n = n0 + j;
            double v = buf[j * nr + lr];
            for (int r = 1; r < ks; ++r) v += buf[(r * OZ_BN + j) * nr + lr];
            if (live && mm < Mout && n < Nout) {
                const int i = mm % afold, b = mm / afold;
                double *cp = Cout + i + (long long)b * sC + (long long)ldc * n;
                *cp = beta == 0.0 ? v : fma(beta, *cp, v);
            }
        }
    }
    __syncthreads();
    if (tid == 0 && stop_s) atomicExch(&g_oz_error, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(OZ_TMEM_COLS));
}

// ------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 oz_encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    TK_REQUIRE(fn != nullptr, "tensor-core GEMM: cuTensorMapEncodeTiled is unavailable");
    return fn;
}

// 3-D map over [OZ_S][rows][Kpad] BF16 planes, box (64, box_rows, 1), 128-byte swizzle
static void oz_tensor_map(CUtensorMap *m, const __nv_bfloat16 *planes, int Kpad, int Rpad, int box_rows) {
    const cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)Rpad, (cuuint64_t)OZ_S};
    const cuuint64_t strides[2] = {(cuuint64_t)Kpad * 2, (cuuint64_t)Kpad * 2 * (cuuint64_t)Rpad};
    const cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = oz_encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(planes), dims,
                                      strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    TK_REQUIRE(r == CUDA_SUCCESS, "tensor-core GEMM: tensor map encoding failed");
}

bool oz_supported(const GProb &p) {
    long long kt = 0;
    for (int s = 0; s < p.nseg; ++s) kt += p.seg[s].K;
    return kt >= 1 && kt <= (long long)OZ_MAXCHUNK * OZ_CHUNK && p.M >= 1 && p.N >= 1 &&
           (p.batch == 1 || p.sB == 0) && (long long)p.M * p.batch < (1LL << 30);
}

// Descriptor of an operand side without its output buffers: two sides with equal keys slice to
// the same planes (the same sketch matrix or basis used by many problems of a call)
static std::string oz_key(const OzSide &S) {
    OzSide k;
    std::memset(&k, 0, sizeof k);               // padding bytes included: the key is the bytes
    k.rows = S.rows; k.a = S.a; k.trans = S.trans; k.nseg = S.nseg; k.Kpad = S.Kpad; k.Rpad = S.Rpad;
    k.bstride = S.bstride;
    for (int i = 0; i < S.nseg; ++i) {
        k.seg[i].p = S.seg[i].p; k.seg[i].cd = S.seg[i].cd; k.seg[i].coef = S.seg[i].coef;
        k.seg[i].K = S.seg[i].K; k.seg[i].ld = S.seg[i].ld; k.seg[i].koff = S.seg[i].koff;
    }
    return std::string(reinterpret_cast<const char *>(&k), sizeof(OzSide));
}

// clusters of `size` CTAs of k_gemm_oz that can be resident at once on this device (queried
// once per device and size; 0 when the query fails, which keeps the reduction unsplit)
static int oz_resident_clusters(const Ctx &c, cudaLaunchConfig_t cfg, int size) {
    constexpr int MAXDEV = 64;
    static std::atomic<int> cache[MAXDEV][4];        // sizes 1, 2, 4, 8; 0 = not yet queried
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return 0;
    const int slot = size == 1 ? 0 : size == 2 ? 1 : size == 4 ? 2 : 3;
    int v = cache[dev][slot].load();
    if (v != 0) return v > 0 ? v : 0;
    cudaLaunchAttribute a[1];
    a[0].id = cudaLaunchAttributeClusterDimension;
    a[0].val.clusterDim.x = (unsigned)size;
    a[0].val.clusterDim.y = 1;
    a[0].val.clusterDim.z = 1;
    cfg.attrs = a;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)(size * c.num_sms), 1, 1);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (const void *)k_gemm_oz, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    cache[dev][slot].store(n > 0 ? n : -1);
    return n > 0 ? n : 0;
}

void gemm_oz(Ctx &c, const std::vector<GProb> &probs, const char *tag) {
    (void)tag;
    if (probs.empty()) return;
    static std::atomic<bool> attr_set{false};   // set once; idempotent if two threads race
    if (!attr_set) {
        TK_CUDA(cudaFuncSetAttribute(k_gemm_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
        TK_CUDA(cudaFuncSetAttribute(k_oz_split, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SPLIT_SMEM));
        attr_set = true;
    }
    // 1. operand sides of every problem; each distinct side is sliced once
    const size_t np = probs.size();
    std::vector<OzSide> A(np), B(np);
    std::vector<OzSide> uniq;
    std::map<std::string, size_t> seen;
    auto place = [&](OzSide &S) {
        const std::string key = oz_key(S);
        auto it = seen.find(key);
        if (it != seen.end()) {
            S.planes = uniq[it->second].planes;
            S.exps = uniq[it->second].exps;
            return;
        }
        const int nch = (S.Kpad + OZ_CHUNK - 1) / OZ_CHUNK;
        S.planes = reinterpret_cast<__nv_bfloat16 *>(c.arena->alloc_bytes((size_t)OZ_S * S.Rpad * S.Kpad * 2));
        S.exps = reinterpret_cast<short *>(c.arena->alloc_bytes((size_t)nch * S.Rpad * 2));
        seen[key] = uniq.size();
        uniq.push_back(S);
    };
    for (size_t j = 0; j < np; ++j) {
        const GProb &p = probs[j];
        TK_REQUIRE(oz_supported(p), "tensor-core GEMM: unsupported shape");
        long long kt = 0;
        for (int s = 0; s < p.nseg; ++s) kt += p.seg[s].K;
        // chunks of 256; a reduction of at most 256 is padded only to the slab width
        const int Kpad = kt <= OZ_CHUNK ? (int)((kt + OZ_BK - 1) / OZ_BK) * OZ_BK
                                        : (int)((kt + OZ_CHUNK - 1) / OZ_CHUNK) * OZ_CHUNK;
        const int rowsA = p.M * p.batch;
        OzSide &a = A[j], &b = B[j];
        a = OzSide{};
        b = OzSide{};
        a.rows = rowsA; a.a = p.M; a.trans = p.ta; a.nseg = p.nseg; a.bstride = p.sA; a.Kpad = Kpad;
        a.Rpad = (rowsA + OZ_BM - 1) / OZ_BM * OZ_BM;
        b.rows = p.N; b.a = p.N; b.trans = p.tb ? 0 : 1; b.nseg = p.nseg; b.bstride = 0; b.Kpad = Kpad;
        b.Rpad = (p.N + OZ_BN - 1) / OZ_BN * OZ_BN;
        int koff = 0;
        for (int s = 0; s < p.nseg; ++s) {
            const GSeg &q = p.seg[s];
            a.seg[s] = OzSeg{q.A, q.coef_dev, q.coef, q.K, q.lda, koff};
            b.seg[s] = OzSeg{q.B, nullptr, 1.0, q.K, q.ldb, koff};
            koff += q.K;
        }
        place(a);
        place(b);
    }
    // 2. slicing of the distinct sides
    for (size_t base = 0; base < uniq.size(); base += OZ_MAXSIDES) {
        OzSides S{};
        S.n = (int)std::min<size_t>(OZ_MAXSIDES, uniq.size() - base);
        int maxRb = 0, maxCh = 0;
        double bytes = 0.0;   // the operand read once, the digit planes and exponents written once
        for (int i = 0; i < S.n; ++i) {
            S.s[i] = uniq[base + i];
            maxRb = std::max(maxRb, S.s[i].Rpad / 32);
            const int nch = (S.s[i].Kpad + OZ_CHUNK - 1) / OZ_CHUNK;
            maxCh = std::max(maxCh, nch);
            long long kt = 0;
            for (int g = 0; g < S.s[i].nseg; ++g) kt += S.s[i].seg[g].K;
            bytes += 8.0 * S.s[i].rows * (double)kt + 2.0 * OZ_S * S.s[i].Rpad * (double)S.s[i].Kpad +
                     2.0 * nch * S.s[i].Rpad;
        }
        c.pre_launch();
        k_oz_split<<<dim3((unsigned)maxRb, (unsigned)maxCh, (unsigned)S.n), 256, OZ_SPLIT_SMEM, c.st>>>(S);
        c.check_launch("oz_split", 0.0, bytes);
    }
    // 3. products, OZ_MAXPROB per launch
    for (size_t base = 0; base < np; base += OZ_MAXPROB) {
        OzGroup G{};
        G.nprob = (int)std::min<size_t>(OZ_MAXPROB, np - base);
        int tiles = 0;
        double flops = 0.0, bytes = 0.0;
        for (int j = 0; j < G.nprob; ++j) {
            const GProb &p = probs[base + j];
            const OzSide &a = A[base + j], &b = B[base + j];
            long long kt = 0;
            for (int s = 0; s < p.nseg; ++s) kt += p.seg[s].K;
            OzProb &P = G.p[j];
            oz_tensor_map(&P.tmA, a.planes, a.Kpad, a.Rpad, OZ_BM);
            oz_tensor_map(&P.tmB, b.planes, b.Kpad, b.Rpad, OZ_BN);
            P.expA = a.exps; P.expB = b.exps; P.C = p.C; P.beta = p.beta; P.sC = p.sC;
            P.M = a.rows; P.N = p.N; P.a = p.M; P.ldc = p.ldc; P.RpadA = a.Rpad; P.RpadB = b.Rpad;
            P.nslab = a.Kpad / OZ_BK; P.nchunk = (a.Kpad + OZ_CHUNK - 1) / OZ_CHUNK;
            P.tiles_m = a.Rpad / OZ_BM; P.tiles_n = b.Rpad / OZ_BN; P.tile_begin = tiles;
            tiles += P.tiles_m * P.tiles_n;
            flops += 2.0 * p.M * (double)p.N * kt * p.batch;
            bytes += 8.0 * ((double)a.rows * kt + (double)p.N * kt + (p.beta != 0.0 ? 2.0 : 1.0) * a.rows * (double)p.N);
        }
        // split the reduction over a cluster while the grid stays within one wave and every
        // split gets at least one chunk.  One CTA per SM (the tile takes all of tensor memory)
        // and a cluster's CTAs on one GPC: the clusters of a size that fit at once are fewer
        // than SMs / size (36 clusters of 4 ran as two waves, each SM busy half the launch)
        int maxch = 1;
        for (int j = 0; j < G.nprob; ++j) maxch = std::max(maxch, G.p[j].nchunk);
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr[1];
        cfg.blockDim = dim3(OZ_THREADS, 1, 1);
        cfg.dynamicSmemBytes = OZ_SMEM;
        cfg.stream = c.st;
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int ks = 1;
        // (and leaves the SMs of two 16-CTA clusters free: a concurrent solve's QR or SVD must
        // not wait behind a split that only shortens this product)
        while (ks < 8 && 2 * ks <= maxch && tiles <= oz_resident_clusters(c, cfg, 2 * ks) &&
               tiles * 2 * ks <= c.num_sms - 32)
            ks *= 2;
        G.ks = ks;
        cfg.gridDim = dim3((unsigned)(tiles * ks), 1, 1);
        attr[0].val.clusterDim.x = (unsigned)ks;
        c.pre_launch();
        TK_CUDA(cudaLaunchKernelEx(&cfg, k_gemm_oz, G));
        c.check_launch("gemm_tc", flops, bytes);   // one profiler entry for every tensor-core product
    }
}

int oz_error_flag(bool reset) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_oz_error, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (reset && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_oz_error, &z, sizeof(int));
    }
    return v;
}

}  // namespace tk
