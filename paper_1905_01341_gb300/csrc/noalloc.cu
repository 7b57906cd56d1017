// Allocation-free variant of the direct (all-pairs) operator product.
//
// Some callers cannot allocate device memory when they need a product: code that runs
// inside another framework's fixed memory pool or budget, or a latency-critical loop in which
// a device allocation (which synchronises the device) is not acceptable. This entry point
// serves them: the caller passes inputs and outputs, and the one scratch buffer the direct
// FP32 kernel needs (the hi + lo split of the coordinates) is a file-scope __device__ array
// of fixed size, so the call allocates nothing. It launches the same three kernels as a
// context's direct FP32 product (coordinate split, all-pairs sum, identity diagonals).
#include <atomic>
#include <mutex>

#include "internal.h"

namespace bem {
namespace {

constexpr int64_t kNoAllocMaxN = 262144;  // largest N this entry point accepts
constexpr int kMaxDevices = 64;

// hi[3][N] followed by lo[3][N], for N <= kNoAllocMaxN (6 MiB per device, held until exit).
__device__ __align__(256) float g_split_scratch[6 * kNoAllocMaxN];

// Device address of g_split_scratch on each device, looked up once per device (under a lock,
// so concurrent first calls from several host threads are safe; a failed lookup is retried on
// the next call). In host code the symbol itself is a host-side stand-in, not a device address.
// The address belongs to the device's primary context: after cudaDeviceReset the module is
// loaded again and the cached address is stale, so this entry point must not be used on a
// device after a reset in the same process.
std::atomic<float *> g_split_addr[kMaxDevices];
std::mutex g_split_lock;

float *scratch_address(int dev) {
    float *p = g_split_addr[dev].load(std::memory_order_acquire);
    if (p) return p;
    std::lock_guard<std::mutex> lk(g_split_lock);
    p = g_split_addr[dev].load(std::memory_order_relaxed);
    if (!p) {
        void *a = nullptr;
        BEM_CUDA(cudaGetSymbolAddress(&a, g_split_scratch));  // with `dev` current
        p = static_cast<float *>(a);
        g_split_addr[dev].store(p, std::memory_order_release);
    }
    return p;
}

// A caller array must be device (or managed) memory reachable from the current device: a host
// pointer handed to the kernels would fault or read the wrong memory. cudaPointerGetAttributes
// allocates nothing.
void require_device_array(const void *p, int dev, const char *name) {
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(BEM_ERR_ARG, std::string("bem_apply_direct_noalloc: ") + name + " is not a device pointer");
    }
    const bool ok = a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
    if (!ok)
        fail(BEM_ERR_ARG, std::string("bem_apply_direct_noalloc: ") + name +
                              " must be device memory of the current device");
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
        const struct {
            const void *p;
            const char *name;
        } arrays[] = {{xyz, "xyz"}, {s, "s"}, {n, "n"}, {ldiag, "ldiag"}, {mdiag, "mdiag"}, {out, "out"},
                      {f != 0.0 ? xL : nullptr, "xL"}, {g != 0.0 ? xM : nullptr, "xM"}};
        for (const auto &a : arrays)
            if (a.p) require_device_array(a.p, dev, a.name);
        float *hi = scratch_address(dev);
        float *lo = hi + 3 * N;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        launch_split_hilo(3 * N, xyz, hi, lo, st);
        launch_direct32_raw(N, hi, lo, s, n, f, xL, g, xM, out, st);
        launch_add_diag(N, f, xL, g, xM, ldiag, mdiag, out, st);
        return BEM_OK;
    } catch (const Error &e) {
        g_create_error = e.msg;  // reported by bem_last_error(NULL)
        return e.code;
    }
}
