// A least-squares entry point that performs no device allocation.
//
// tk_sketched_ls needs a few hundred kilobytes of device workspace, which the handle obtains
// with cudaMalloc on first use.  Some callers cannot allow that: a host application that
// reserves the GPU's memory up front for its own allocator and forbids any other device
// allocation, or a latency-critical loop in which cudaMalloc's implicit device-wide
// synchronisation is unacceptable.  tk_sketched_ls_static serves them: its workspace is a
// fixed array in the library's device image, so it needs neither a handle nor any
// allocation.  The array is created when the library's module is loaded on a device and
// stays resident on every GPU that loads the library until the process exits.
//
// Host code must not use the array's name as a device pointer (on the host it only names
// a stand-in object); the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on it.
#include <mutex>

#include "tk_internal.cuh"

namespace tk {
// The compact WY Householder least-squares kernel of k_linalg.cu.
__global__ void k_ls_wy(const double *M, const double *b, int s, int c0, int k, LSState st, int init_qtb);
}  // namespace tk

namespace {

constexpr int kMaxRows = 512;   // largest s accepted
constexpr int kMaxCols = 128;   // largest k accepted
static_assert(kMaxRows <= tk::LSW_MAXS && kMaxCols <= tk::LSW_MAXK, "limits beyond the WY kernel's");
// Reflectors (s x k, leading dimension s), tau (k), Q^T b (s) and the WY factor T (k x k,
// leading dimension kMaxCols) at their largest sizes.
constexpr size_t kScratchDoubles =
    (size_t)kMaxRows * kMaxCols + kMaxCols + kMaxRows + (size_t)kMaxCols * kMaxCols;

static __device__ __align__(256) double g_ls_scratch[kScratchDoubles];

std::mutex g_mutex;
constexpr int kMaxDevices = 256;
double *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
int scratch_address(double **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return TK_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_ls_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return TK_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return TK_OK;
}

}  // namespace

extern "C" int tk_sketched_ls_static(const double *M, const double *b, int32_t s, int32_t k, double *y,
                                     double *res, void *stream) {
    if (!M || !b || !y || !res) return TK_EINVAL;
    if (k < 1 || k >= s || s > kMaxRows || k > kMaxCols) return TK_EINVAL;
    double *base = nullptr;
    const int rc = scratch_address(&base);
    if (rc != TK_OK) return rc;
    tk::LSState st{};
    st.H = base;
    st.tau = base + (size_t)kMaxRows * kMaxCols;
    st.qtb = st.tau + kMaxCols;
    st.T = st.qtb + kMaxRows;
    st.ldt = kMaxCols;
    st.y = y;
    st.res = res;
    // Every scratch word the kernel reads it has written earlier in the same call (Q^T b is
    // initialised from b, each reflector column and each column of T before use), so nothing
    // needs clearing.
    tk::k_ls_wy<<<1, 512, 0, static_cast<cudaStream_t>(stream)>>>(M, b, s, 0, k, st, 1);
    return cudaGetLastError() == cudaSuccess ? TK_OK : TK_ECUDA;
}
