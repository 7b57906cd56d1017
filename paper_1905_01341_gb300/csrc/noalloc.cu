// Allocation-free variant of the direct (all-pairs) operator product.
//
// Some callers cannot allocate device memory when they need a product: code that runs
// inside another framework's fixed memory pool or budget, or a latency-critical loop in which
// a device allocation (which synchronises the device) is not acceptable. This entry point
// serves them: the caller passes inputs and outputs, and the one scratch buffer the direct
// FP32 kernel needs (the hi + lo split of the coordinates) is a file-scope __device__ array
// of fixed size, so the call allocates nothing.
#include "internal.h"

namespace bem {
namespace {

constexpr int64_t kNoAllocMaxN = 262144;  // largest N this entry point accepts
constexpr int kMaxDevices = 64;

// hi[3][N] followed by lo[3][N], for N <= kNoAllocMaxN (6 MiB per device, held until exit).
__device__ __align__(256) float g_split_scratch[6 * kNoAllocMaxN];

// Device address of g_split_scratch on each device, looked up once per device. In host code
// the symbol itself is a host-side stand-in, not a device address.
float *g_split_addr[kMaxDevices] = {};

__global__ void k_split_noalloc(int64_t n, const double *__restrict__ x, float *__restrict__ hi,
                                float *__restrict__ lo) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h = (float)x[i];
    hi[i] = h;
    lo[i] = (float)(x[i] - (double)h);
}

__global__ void k_diag_noalloc(int64_t N, double f, const double *__restrict__ xL, double g,
                               const double *__restrict__ xM, const double *__restrict__ ld,
                               const double *__restrict__ md, double *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double v = out[i];
    if (f != 0.0) v += f * ld[i] * xL[i];
    if (g != 0.0) v += g * md[i] * xM[i];
    out[i] = v;
}

}  // namespace

}  // namespace bem

using namespace bem;

extern "C" int bem_apply_direct_noalloc(int64_t N, const double *xyz, const double *s, const double *n,
                                        const double *ldiag, const double *mdiag, double f, const double *xL,
                                        double g, const double *xM, double *out, void *stream) {
    try {
        if (N < 2 || N > kNoAllocMaxN)
            fail(BEM_ERR_ARG, "bem_apply_direct_noalloc: N must be in 2.." + std::to_string(kNoAllocMaxN) +
                                  " (got " + std::to_string(N) + ")");
        if (!xyz || !s || !n || !ldiag || !mdiag || !out) fail(BEM_ERR_ARG, "bem_apply_direct_noalloc: null array");
        if ((f != 0.0 && !xL) || (g != 0.0 && !xM))
            fail(BEM_ERR_ARG, "bem_apply_direct_noalloc: null input with a non-zero coefficient");
        int dev = 0;
        BEM_CUDA(cudaGetDevice(&dev));
        if (dev < 0 || dev >= kMaxDevices) fail(BEM_ERR_ARG, "bem_apply_direct_noalloc: device index too large");
        if (!g_split_addr[dev]) {
            // first call on this device (the current one): look up the array's device address
            void *p = nullptr;
            BEM_CUDA(cudaGetSymbolAddress(&p, g_split_scratch));
            g_split_addr[dev] = static_cast<float *>(p);
        }
        float *hi = g_split_addr[dev];
        float *lo = hi + 3 * N;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        k_split_noalloc<<<div_up(3 * N, 256), 256, 0, st>>>(3 * N, xyz, hi, lo);
        BEM_LAUNCH_CHECK();
        launch_direct32_raw(N, hi, lo, s, n, f, xL, g, xM, out, st);
        k_diag_noalloc<<<div_up(N, 256), 256, 0, st>>>(N, f, xL, g, xM, ldiag, mdiag, out);
        BEM_LAUNCH_CHECK();
        return BEM_OK;
    } catch (const Error &e) {
        g_create_error = e.msg;  // reported by bem_last_error(NULL)
        return e.code;
    }
}
