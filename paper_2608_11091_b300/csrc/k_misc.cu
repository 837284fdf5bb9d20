// Structured and elementwise kernels of the Tucker sGMRES hot path.
#include <algorithm>

#include <cooperative_groups.h>

#include "tk_internal.cuh"

namespace cg = cooperative_groups;

namespace tk {

void Ctx::check_launch(const char *what, double flops, double bytes) {
    ++launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        throw Error{TK_ECUDA, std::string("launch of ") + what + ": " + cudaGetErrorString(e)};
    if (prof) prof->end(st, what, flops, bytes);
}

// ------------------------------------------------------------------------------------------
// Profiler
// ------------------------------------------------------------------------------------------
Profiler::~Profiler() {
    for (cudaEvent_t e : pool_) cudaEventDestroy(e);
}

cudaEvent_t Profiler::get() {
    if (used_ == pool_.size()) {
        cudaEvent_t e;
        TK_CUDA(cudaEventCreate(&e));
        pool_.push_back(e);
    }
    return pool_[used_++];
}

void Profiler::begin(cudaStream_t st) {
    open_ = get();
    TK_CUDA(cudaEventRecord(open_, st));
}

void Profiler::end(cudaStream_t st, const char *name, double flops, double bytes) {
    cudaEvent_t b = get();
    TK_CUDA(cudaEventRecord(b, st));
    recs_.push_back(Rec{name, open_, b, flops, bytes});
}

void Profiler::collect() {
    for (const Rec &r : recs_) {
        float ms = 0.f;
        TK_CUDA(cudaEventSynchronize(r.b));
        TK_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        bool found = false;
        for (auto &t : tot_)
            if (t.first == r.name) {
                t.second.n += 1; t.second.ms += ms; t.second.flops += r.flops; t.second.bytes += r.bytes;
                found = true;
                break;
            }
        if (!found) { Tot t; t.n = 1; t.ms = ms; t.flops = r.flops; t.bytes = r.bytes; tot_.push_back({r.name, t}); }
    }
    recs_.clear();
    used_ = 0;
}

std::string Profiler::report_and_reset() {
    collect();
    std::string s;
    for (auto &t : tot_)
        s += t.first + " " + std::to_string(t.second.n) + " " + std::to_string(t.second.ms) + " " +
             std::to_string(t.second.flops) + " " + std::to_string(t.second.bytes) + "\n";
    tot_.clear();
    return s;
}

// ------------------------------------------------------------------------------------------
// Arena
// ------------------------------------------------------------------------------------------
Arena::~Arena() {
    for (auto &c : chunks_) cudaFree(c.base);
}

void *Arena::alloc_bytes(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    while (cur_ < chunks_.size()) {
        if (off_ + bytes <= chunks_[cur_].size) {
            void *p = chunks_[cur_].base + off_;
            off_ += bytes;
            return p;
        }
        ++cur_;
        off_ = 0;
    }
    size_t sz = std::max(bytes, size_t(256) << 20);
    if (limit_) {
        const size_t held = capacity();
        if (held + bytes > limit_)
            throw Error{TK_ENOMEM, "device workspace limit of " + std::to_string(limit_) + " bytes reached"};
        sz = std::min(sz, limit_ - held);
    }
    char *p = nullptr;
    if (cudaMalloc(&p, sz) != cudaSuccess) {
        cudaGetLastError();
        throw Error{TK_ENOMEM, "device workspace allocation of " + std::to_string(sz) + " bytes failed"};
    }
    chunks_.push_back(Chunk{p, sz});
    cur_ = chunks_.size() - 1;
    off_ = bytes;
    return p;
}

size_t Arena::capacity() const {
    size_t t = 0;
    for (auto &c : chunks_) t += c.size;
    return t;
}

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) + Box-Muller
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k.x += W0; k.y += W1; }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ double round_bf16(double x) {
    if (x == 0.0) return 0.0;
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long lsb = (b >> 45) & 1ull;
    b = ((b + (1ull << 44) - 1ull + lsb) >> 45) << 45;
    return __longlong_as_double((long long)b);
}

struct GaussJobs {
    int n;
    uint64_t sid[TK_MAX_D * 2];
    long long count[TK_MAX_D * 2];
    double *out[TK_MAX_D * 2];
};

__global__ void k_gaussian(uint64_t seed, const __grid_constant__ GaussJobs J, int bf16) {
    const int job = blockIdx.y;
    const long long cnt = J.count[job];
    const long long npair = (cnt + 1) / 2;
    const uint64_t sid = J.sid[job];
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < npair;
         b += (long long)gridDim.x * blockDim.x) {
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)b, (uint32_t)((unsigned long long)b >> 32), (uint32_t)sid,
                       (uint32_t)(sid >> 32)),
            key);
        const unsigned long long m1 = (unsigned long long)(w.x >> 5) * 67108864ull + (w.y >> 6);
        const unsigned long long m2 = (unsigned long long)(w.z >> 5) * 67108864ull + (w.w >> 6);
        const double u1 = ((double)m1 + 1.0) * 0x1p-53;
        const double u2 = (double)m2 * 0x1p-53;
        const double rad = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincos(2.0 * 3.141592653589793 * u2, &sn, &cs);
        double z0 = rad * cs, z1 = rad * sn;
        if (bf16) { z0 = round_bf16(z0); z1 = round_bf16(z1); }
        J.out[job][2 * b] = z0;
        if (2 * b + 1 < cnt) J.out[job][2 * b + 1] = z1;
    }
}

void gaussian(Ctx &c, uint64_t seed, const uint64_t *sids, const long long *counts,
              double *const *outs, int nmat, int bf16) {
    for (int base = 0; base < nmat; base += TK_MAX_D * 2) {
        GaussJobs J{};
        J.n = std::min(TK_MAX_D * 2, nmat - base);
        long long mx = 1, total = 0;
        for (int i = 0; i < J.n; ++i) {
            J.sid[i] = sids[base + i];
            J.count[i] = counts[base + i];
            J.out[i] = outs[base + i];
            mx = std::max(mx, (counts[base + i] + 1) / 2);
            total += counts[base + i];
        }
        const int threads = 256;
        const long long blocks = std::min<long long>((mx + threads - 1) / threads, 4096);
        c.pre_launch();
        k_gaussian<<<dim3((unsigned)blocks, J.n), threads, 0, c.st>>>(seed, J, bf16);
        c.check_launch("gaussian", 0.0, 8.0 * (double)total);   // every value written once
    }
}

__global__ void k_philox_raw(uint64_t seed, uint64_t sid, uint64_t first, long long nb, uint32_t *out) {
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb;
         i += (long long)gridDim.x * blockDim.x) {
        const uint64_t b = first + (uint64_t)i;
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)b, (uint32_t)(b >> 32), (uint32_t)sid, (uint32_t)(sid >> 32)), key);
        out[4 * i] = w.x; out[4 * i + 1] = w.y; out[4 * i + 2] = w.z; out[4 * i + 3] = w.w;
    }
}

void philox_raw(Ctx &c, uint64_t seed, uint64_t sid, uint64_t first, long long nb, uint32_t *out) {
    const long long blocks = std::min<long long>((nb + 255) / 256, 4096);
    c.pre_launch();
    k_philox_raw<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, c.st>>>(seed, sid, first, nb, out);
    c.check_launch("philox", 0.0, 16.0 * (double)nb);
}

// ------------------------------------------------------------------------------------------
// Banded mode-matrix apply: out = A U (or A^T U), A in LAPACK band layout
// ------------------------------------------------------------------------------------------
struct BandJobs {
    int n;
    BandJob j[32];
};

__global__ void k_band(const __grid_constant__ BandJobs J) {
    const BandJob &B = J.j[blockIdx.y];
    const long long total = (long long)B.n * B.r;
    const int ld = B.kl + B.ku + 1;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % B.n);
        const long long j = e / B.n;
        const double *u = B.U + j * B.n;
        double acc = 0.0;
        if (!B.trans) {
            const int c0 = max(0, i - B.kl), c1 = min(B.n - 1, i + B.ku);
            for (int c = c0; c <= c1; ++c) acc = fma(B.band[B.ku + i - c + (long long)c * ld], u[c], acc);
        } else {
            const int c0 = max(0, i - B.ku), c1 = min(B.n - 1, i + B.kl);
            for (int c = c0; c <= c1; ++c) acc = fma(B.band[B.ku + c - i + (long long)i * ld], u[c], acc);
        }
        B.out[e] = acc;
    }
}

void band_apply(Ctx &c, const std::vector<BandJob> &jobs) {
    for (size_t base = 0; base < jobs.size(); base += 32) {
        BandJobs J{};
        J.n = (int)std::min<size_t>(32, jobs.size() - base);
        long long mx = 1;
        double bytes = 0.0;
        for (int i = 0; i < J.n; ++i) {
            J.j[i] = jobs[base + i];
            const BandJob &b = J.j[i];
            mx = std::max(mx, (long long)b.n * b.r);
            bytes += 8.0 * ((double)b.n * b.r * 2 + (double)(b.kl + b.ku + 1) * b.n);
        }
        const long long blocks = std::min<long long>((mx + 255) / 256, 2048);
        c.pre_launch();
        k_band<<<dim3((unsigned)blocks, J.n), 256, 0, c.st>>>(J);
        c.check_launch("band", 0.0, bytes);
    }
}

// ------------------------------------------------------------------------------------------
// Khatri-Rao (row-wise Hadamard) contraction: out[i, mm, l] = sum_j T[i, j, mm, l] P[j, l]
// ------------------------------------------------------------------------------------------
struct HadJobs {
    int n;
    HadJob j[32];
};

__global__ void k_hadamard(const __grid_constant__ HadJobs J) {
    const HadJob &H = J.j[blockIdx.y];
    const long long total = (long long)H.a * H.cc * H.s;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e % H.a;
        const long long rest = e / H.a;          // mm + cc * l
        const long long mm = rest % H.cc, l = rest / H.cc;
        const double *t = H.T + i + (long long)H.a * H.b * (mm + (long long)H.cc * l);
        const double *p = H.P + l * H.ldp;
        double acc = 0.0;
        for (int j = 0; j < H.b; ++j) acc = fma(t[(long long)j * H.a], p[j], acc);
        H.out[e] = acc;
    }
}

void hadamard_contract(Ctx &c, const std::vector<HadJob> &jobs) {
    for (size_t base = 0; base < jobs.size(); base += 32) {
        HadJobs J{};
        J.n = (int)std::min<size_t>(32, jobs.size() - base);
        long long mx = 1;
        double bytes = 0.0, flops = 0.0;
        for (int i = 0; i < J.n; ++i) {
            J.j[i] = jobs[base + i];
            const HadJob &h = J.j[i];
            mx = std::max(mx, (long long)h.a * h.cc * h.s);
            bytes += 8.0 * ((double)h.a * h.b * h.cc * h.s + (double)h.b * h.s + (double)h.a * h.cc * h.s);
            flops += 2.0 * h.a * h.b * h.cc * (double)h.s;
        }
        const long long blocks = std::min<long long>((mx + 255) / 256, 4096);
        c.pre_launch();
        k_hadamard<<<dim3((unsigned)blocks, J.n), 256, 0, c.st>>>(J);
        c.check_launch("hadamard", flops, bytes);
    }
}

// ------------------------------------------------------------------------------------------
// Transposed mode unfolding gather
// ------------------------------------------------------------------------------------------
__global__ void k_gather_unfold_t(const double *C, double *out, long long a, int sk, long long rest) {
    const long long m = a * rest;
    const long long total = m * sk;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long rho = e % m, col = e / m;
        out[e] = C[(rho % a) + col * a + (rho / a) * a * sk];
    }
}

void gather_unfold_t(Ctx &c, const double *C, double *out, long long a, int sk, long long rest) {
    const long long total = a * rest * sk;
    const long long blocks = std::min<long long>((total + 255) / 256, 4096);
    c.pre_launch();
    k_gather_unfold_t<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, c.st>>>(C, out, a, sk, rest);
    c.check_launch("gather", 0.0, 16.0 * (double)total);
}

// ------------------------------------------------------------------------------------------
// Deterministic reductions
// ------------------------------------------------------------------------------------------
struct DotJobs {
    int n;
    DotJob j[32];
};

// One 8-CTA cluster per dot product: each CTA sums a contiguous eighth (one SM's FP64 pipe
// would otherwise take every FMA), warp 0 combines its warps, and CTA 0 adds the eight
// partials in rank order, so the result depends only on n, never on the batching.
constexpr int DOT_CL = 8;
__global__ void __launch_bounds__(1024) k_dots(const __grid_constant__ DotJobs J) {
    cg::cluster_group cl = cg::this_cluster();
    const int q = (int)cl.block_rank();
    const DotJob &D = J.j[blockIdx.x / DOT_CL];
    const long long chunk = (D.n + DOT_CL - 1) / DOT_CL;
    const long long i0 = q * chunk, i1 = min(D.n, i0 + chunk);
    double acc = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc = fma(D.x[i], D.y[i], acc);
    __shared__ double sh[33];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        double t = lane < nw ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[32] = t;
    }
    cl.sync();
    if (q == 0 && threadIdx.x == 0) {
        double t = 0.0;
        for (int r = 0; r < DOT_CL; ++r) t += cl.map_shared_rank(sh, r)[32];
        *D.out = t;
    }
    cl.sync();   // keep every CTA's partial alive until CTA 0 has read it
}

void dots(Ctx &c, const std::vector<DotJob> &jobs) {
    for (size_t base = 0; base < jobs.size(); base += 32) {
        DotJobs J{};
        J.n = (int)std::min<size_t>(32, jobs.size() - base);
        double bytes = 0.0;
        for (int i = 0; i < J.n; ++i) {
            J.j[i] = jobs[base + i];
            bytes += 16.0 * (double)J.j[i].n;
        }
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)(J.n * DOT_CL), 1, 1);
        cfg.blockDim = dim3(1024, 1, 1);
        cfg.stream = c.st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = DOT_CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        c.pre_launch();
        TK_CUDA(cudaLaunchKernelEx(&cfg, k_dots, J));
        c.check_launch("dots", 0.0, bytes);
    }
}

void dot(Ctx &c, const double *x, const double *y, long long n, double *out) {
    dots(c, {DotJob{x, y, n, out}});
}

// ------------------------------------------------------------------------------------------
// Elementwise helpers
// ------------------------------------------------------------------------------------------
__global__ void k_fill(double *p, long long n, double v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

void fill(Ctx &c, double *p, long long n, double v) {
    if (n <= 0) return;
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    c.pre_launch();
    k_fill<<<(unsigned)blocks, 256, 0, c.st>>>(p, n, v);
    c.check_launch("fill", 0.0, 8.0 * (double)n);
}

__global__ void k_scale_by(double *y, const double *x, long long n, const double *s, int inv) {
    const double f = inv ? 1.0 / *s : *s;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = x[i] * f;
}

void scale_by(Ctx &c, double *y, const double *x, long long n, const double *s, int inv) {
    if (n <= 0) return;
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    c.pre_launch();
    k_scale_by<<<(unsigned)blocks, 256, 0, c.st>>>(y, x, n, s, inv);
    c.check_launch("scale", 0.0, 16.0 * (double)n);
}

void copy(Ctx &c, double *dst, const double *src, long long n) {
    if (n <= 0) return;
    TK_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
}

__global__ void k_copy_pad(double *dst, int ldd, int rd, int cd, const double *src, int lds, int rs, int cs) {
    const long long total = (long long)rd * cd;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % rd), j = (int)(e / rd);
        dst[i + (long long)j * ldd] = (i < rs && j < cs) ? src[i + (long long)j * lds] : 0.0;
    }
}

void copy_pad(Ctx &c, double *dst, int ld_dst, int rows_dst, int cols_dst, const double *src,
              int ld_src, int rows_src, int cols_src) {
    const long long total = (long long)rows_dst * cols_dst;
    if (total <= 0) return;
    const long long blocks = std::min<long long>((total + 255) / 256, 4096);
    c.pre_launch();
    k_copy_pad<<<(unsigned)blocks, 256, 0, c.st>>>(dst, ld_dst, rows_dst, cols_dst, src, ld_src,
                                                   rows_src, cols_src);
    c.check_launch("copy_pad", 0.0, 8.0 * ((double)total + (double)std::min(rows_src, rows_dst) * std::min(cols_src, cols_dst)));
}

struct CoreDims { int d; int rd[TK_MAX_D]; int rs[TK_MAX_D]; };

__global__ void k_copy_core_pad(double *dst, const double *src, CoreDims D, long long total) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long rem = e, soff = 0, sstride = 1;
        bool inside = true;
        for (int k = 0; k < D.d; ++k) {
            const int idx = (int)(rem % D.rd[k]);
            rem /= D.rd[k];
            if (idx >= D.rs[k]) inside = false;
            soff += idx * sstride;
            sstride *= D.rs[k];
        }
        dst[e] = inside ? src[soff] : 0.0;
    }
}

void copy_core_pad(Ctx &c, double *dst, const int *rdst, const double *src, const int *rsrc, int d) {
    CoreDims D{};
    D.d = d;
    long long total = 1;
    for (int k = 0; k < d; ++k) { D.rd[k] = rdst[k]; D.rs[k] = rsrc[k]; total *= rdst[k]; }
    const long long blocks = std::min<long long>((total + 255) / 256, 4096);
    c.pre_launch();
    k_copy_core_pad<<<(unsigned)blocks, 256, 0, c.st>>>(dst, src, D, total);
    c.check_launch("copy_core_pad", 0.0, 16.0 * (double)total);
}

__global__ void k_superdiag(const double *G, int m, int d, double *out, double sh, const double *sd) {
    long long stride = 0, p = 1;
    for (int k = 0; k < d; ++k) { stride += p; p *= m; }
    const double f = sh * (sd ? *sd : 1.0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        out[i] = f * G[(long long)i * stride];
}

void superdiag(Ctx &c, const double *G, int m, int d, double *out, double scale_host,
               const double *scale_dev) {
    c.pre_launch();
    k_superdiag<<<(m + 255) / 256, 256, 0, c.st>>>(G, m, d, out, scale_host, scale_dev);
    c.check_launch("superdiag", 0.0, 16.0 * (double)m);
}

__global__ void k_transpose(double *dst, int ldd, const double *src, int lds, int rows, int cols) {
    const long long total = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % rows), j = (int)(e / rows);
        dst[j + (long long)i * ldd] = src[i + (long long)j * lds];
    }
}

void transpose_block(Ctx &c, double *dst, int ldd, const double *src, int lds, int rows, int cols) {
    const long long total = (long long)rows * cols;
    if (total <= 0) return;
    const long long blocks = std::min<long long>((total + 255) / 256, 4096);
    c.pre_launch();
    k_transpose<<<(unsigned)blocks, 256, 0, c.st>>>(dst, ldd, src, lds, rows, cols);
    c.check_launch("transpose", 0.0, 16.0 * (double)total);
}

__global__ void k_triu(double *dst, int ldd, const double *src, int lds, int rows, int cols) {
    const long long total = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % rows), j = (int)(e / rows);
        dst[i + (long long)j * ldd] = (i <= j) ? src[i + (long long)j * lds] : 0.0;
    }
}

void triu_copy(Ctx &c, double *dst, int ldd, const double *src, int lds, int rows, int cols) {
    const long long total = (long long)rows * cols;
    if (total <= 0) return;
    const long long blocks = std::min<long long>((total + 255) / 256, 4096);
    c.pre_launch();
    k_triu<<<(unsigned)blocks, 256, 0, c.st>>>(dst, ldd, src, lds, rows, cols);
    c.check_launch("triu", 0.0, 16.0 * (double)total);
}

// Sine eigenvectors of tridiag(-1, 2, -1) (the DST-I basis, Section 3.4), column-major:
// V[i, j] = sqrt(2/(n+1)) sin((i+1)(j+1) pi / (n+1)); optionally scaled per column by
// exp(-t lambda_j), lambda_j = 2 - 2 cos((j+1) pi / (n+1)).
__global__ void k_sine_basis(double *V, int n, double t) {
    const long long total = (long long)n * n;
    const double sc = sqrt(2.0 / (n + 1));
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e % n, j = e / n;
        const long long prod = ((i + 1) * (j + 1)) % (2 * (n + 1));   // sin is 2(n+1)-periodic here
        double v = sc * sinpi((double)prod / (n + 1));
        if (t != 0.0) v *= exp(-t * (2.0 - 2.0 * cospi((double)(j + 1) / (n + 1))));
        V[e] = v;
    }
}

void sine_basis(Ctx &c, double *V, int n, double t) {
    const long long total = (long long)n * n;
    const long long blocks = std::min<long long>((total + 255) / 256, 4096);
    c.pre_launch();
    k_sine_basis<<<(unsigned)blocks, 256, 0, c.st>>>(V, n, t);
    c.check_launch("sine_basis", 0.0, 8.0 * (double)total);
}

// ------------------------------------------------------------------------------------------
// Row scalings of the exponential-sum preconditioner in the sine basis (memory bound)
// ------------------------------------------------------------------------------------------
constexpr int RS_MAXJ = 128;
struct RowScaleJobs {
    int n;
    RowScaleJob j[RS_MAXJ];
};

__global__ void k_row_scale(const __grid_constant__ RowScaleJobs J) {
    const RowScaleJob &R = J.j[blockIdx.y];
    const long long total = (long long)R.n * R.r;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        R.out[e] = R.w[e % R.n] * R.in[e];
}

void row_scale(Ctx &c, const std::vector<RowScaleJob> &jobs) {
    for (size_t base = 0; base < jobs.size(); base += RS_MAXJ) {
        RowScaleJobs J{};
        J.n = (int)std::min<size_t>(RS_MAXJ, jobs.size() - base);
        long long mx = 1;
        double bytes = 0.0;
        for (int i = 0; i < J.n; ++i) {
            J.j[i] = jobs[base + i];
            const long long e = (long long)J.j[i].n * J.j[i].r;
            mx = std::max(mx, e);
            bytes += 16.0 * e + 8.0 * J.j[i].n;
        }
        const long long blocks = std::min<long long>((mx + 255) / 256, 512);
        c.pre_launch();
        k_row_scale<<<dim3((unsigned)blocks, J.n), 256, 0, c.st>>>(J);
        c.check_launch("row_scale", 0.0, bytes);
    }
}

constexpr int WC_MAXJ = 56;   // 56 x 48 bytes of parameters per launch
struct WeightedCopyJobs {
    int n;
    WeightedCopyJob j[WC_MAXJ];
};

__global__ void k_weighted_copy(const __grid_constant__ WeightedCopyJobs J) {
    const WeightedCopyJob &W = J.j[blockIdx.y];
    const double w = fabs(W.coef * (W.cd ? *W.cd : 1.0)) * sqrt(fmax(*W.normsq, 0.0));
    const long long total = (long long)W.n * W.r;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        W.dst[e] = w * W.src[e];
}

void weighted_copy(Ctx &c, const std::vector<WeightedCopyJob> &jobs) {
    for (size_t base = 0; base < jobs.size(); base += WC_MAXJ) {
        WeightedCopyJobs J{};
        J.n = (int)std::min<size_t>(WC_MAXJ, jobs.size() - base);
        long long mx = 1;
        double bytes = 0.0;
        for (int i = 0; i < J.n; ++i) {
            J.j[i] = jobs[base + i];
            mx = std::max(mx, (long long)J.j[i].n * J.j[i].r);
            bytes += 16.0 * J.j[i].n * (double)J.j[i].r;   // each factor entry read and written once
        }
        const long long blocks = std::min<long long>((mx + 255) / 256, 256);
        c.pre_launch();
        k_weighted_copy<<<dim3((unsigned)blocks, J.n), 256, 0, c.st>>>(J);
        c.check_launch("weighted_copy", 0.0, bytes);
    }
}

__global__ void k_expsum_weights(double *w, int n, int q, double eta) {
    const long long total = (long long)n * (2 * q + 1);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e % n, h = e / n;
        const double lam = 2.0 - 2.0 * cospi((double)(i + 1) / (n + 1));
        w[e] = exp(-exp((double)(h - q) * eta) * lam);
    }
}

void expsum_weights(Ctx &c, double *w, int n, int q, double eta) {
    const long long total = (long long)n * (2 * q + 1);
    const long long blocks = std::min<long long>((total + 255) / 256, 1024);
    c.pre_launch();
    k_expsum_weights<<<(unsigned)blocks, 256, 0, c.st>>>(w, n, q, eta);
    c.check_launch("expsum_weights", 0.0, 8.0 * (double)total);
}

__global__ void k_set_identity(double *p, int n) {
    const long long total = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        p[e] = (e % n == e / n) ? 1.0 : 0.0;
}

void set_identity(Ctx &c, double *p, int n) {
    const long long total = (long long)n * n;
    if (total <= 0) return;
    const long long blocks = std::min<long long>((total + 255) / 256, 1024);
    c.pre_launch();
    k_set_identity<<<(unsigned)blocks, 256, 0, c.st>>>(p, n);
    c.check_launch("identity", 0.0, 8.0 * (double)total);
}

__global__ void k_sqrt_scalar(const double *in, double *out) { *out = sqrt(fmax(*in, 0.0)); }

void sqrt_scalar(Ctx &c, const double *in, double *out) {
    c.pre_launch();
    k_sqrt_scalar<<<1, 1, 0, c.st>>>(in, out);
    c.check_launch("sqrt", 0.0, 16.0);
}

}  // namespace tk

namespace tk {

// ------------------------------------------------------------------------------------------
// MLN_Sum streaming axpy (Algorithm 4): y = beta y + sum_j coef_j (*coef_dev_j) x_j
// 128-bit vector loads when every pointer is 16-byte aligned.
// ------------------------------------------------------------------------------------------
constexpr int AXPY_MAX = 16;
struct AxpyJobs {
    int n;
    const double *x[AXPY_MAX];
    double coef[AXPY_MAX];
    const double *cd[AXPY_MAX];
};

__global__ void __launch_bounds__(256) k_axpy_list(double *y, long long n, double beta,
                                                   const __grid_constant__ AxpyJobs J, int vec) {
    double cf[AXPY_MAX];
#pragma unroll
    for (int j = 0; j < AXPY_MAX; ++j) cf[j] = j < J.n ? J.coef[j] * (J.cd[j] ? *J.cd[j] : 1.0) : 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (vec) {
        const long long n2 = n / 2;
        double2 *y2 = reinterpret_cast<double2 *>(y);
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n2; e += stride) {
            double2 acc = beta == 0.0 ? make_double2(0.0, 0.0) : y2[e];
            if (beta != 0.0 && beta != 1.0) { acc.x *= beta; acc.y *= beta; }
            for (int j = 0; j < J.n; ++j) {
                const double2 v = reinterpret_cast<const double2 *>(J.x[j])[e];
                acc.x = fma(cf[j], v.x, acc.x);
                acc.y = fma(cf[j], v.y, acc.y);
            }
            y2[e] = acc;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) {
            const long long e = n - 1;
            double acc = beta == 0.0 ? 0.0 : beta * y[e];
            for (int j = 0; j < J.n; ++j) acc = fma(cf[j], J.x[j][e], acc);
            y[e] = acc;
        }
        return;
    }
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += stride) {
        double acc = beta == 0.0 ? 0.0 : beta * y[e];
        for (int j = 0; j < J.n; ++j) acc = fma(cf[j], J.x[j][e], acc);
        y[e] = acc;
    }
}

void axpy_list(Ctx &c, double *y, long long n, double beta, const std::vector<const double *> &xs,
               const std::vector<double> &coef, const std::vector<const double *> &coef_dev) {
    if (n <= 0) return;
    if (xs.empty()) {
        if (beta == 0.0) fill(c, y, n, 0.0);
        else if (beta != 1.0) TK_REQUIRE(false, "axpy_list: scaling without terms");
        return;
    }
    for (size_t base = 0; base < xs.size(); base += AXPY_MAX) {
        AxpyJobs J{};
        J.n = (int)std::min<size_t>(AXPY_MAX, xs.size() - base);
        bool aligned = ((uintptr_t)y % 16) == 0;
        for (int j = 0; j < J.n; ++j) {
            J.x[j] = xs[base + j];
            J.coef[j] = coef[base + j];
            J.cd[j] = coef_dev[base + j];
            aligned = aligned && ((uintptr_t)J.x[j] % 16) == 0;
        }
        const long long work = aligned ? n / 2 : n;
        const long long blocks = std::max<long long>(1, std::min<long long>((work + 255) / 256, (long long)c.num_sms * 8));
        c.pre_launch();
        k_axpy_list<<<(unsigned)blocks, 256, 0, c.st>>>(y, n, base == 0 ? beta : 1.0, J, aligned ? 1 : 0);
        // x_j read, y written, and y read unless it is overwritten (beta = 0 in the first chunk)
        const double reads_y = (base == 0 && beta == 0.0) ? 0.0 : 1.0;
        c.check_launch("axpy_list", 2.0 * J.n * (double)n, 8.0 * (double)n * (J.n + 1 + reads_y));
    }
}

// ------------------------------------------------------------------------------------------
// FMA-rate probe: the denominator of the FP64 (and FP32) ALU rooflines, measured on the device
// the library runs on.  Every thread runs 8 independent FMA chains (x <- x a + b, |a| < 1 keeps
// them bounded) for `iters` steps; the grid covers every SM with several CTAs so the pipes are
// the limit, not latency.  Algorithmic flops: 2 x 8 x iters per thread.
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T *out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
    }
    T acc = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) acc += x[j];
    if (acc == (T)-1.2345) out[blockIdx.x] = acc;   // never true; keeps the chains live
}

double fma_peak_tflops(Ctx &c, int fp64) {
    const int blocks = c.num_sms * 8, threads = 256, iters = fp64 ? 2048 : 65536;
    void *out = c.arena->alloc(blocks);
    cudaEvent_t e0, e1;
    TK_CUDA(cudaEventCreate(&e0));
    TK_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {   // the first launch warms the clocks; best of the rest
        TK_CUDA(cudaEventRecord(e0, c.st));
        if (fp64)
            k_fma_peak<double><<<blocks, threads, 0, c.st>>>((double *)out, iters, 0.999999, 1e-7);
        else
            k_fma_peak<float><<<blocks, threads, 0, c.st>>>((float *)out, iters, 0.999999f, 1e-7f);
        TK_CUDA(cudaGetLastError());
        TK_CUDA(cudaEventRecord(e1, c.st));
        TK_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        TK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
    return flops / (best * 1e-3) / 1e12;
}

}  // namespace tk
