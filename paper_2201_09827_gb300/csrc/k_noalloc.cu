// w = A^T v without any allocation by the library.
//
// Some callers cannot allocate device memory at the point where they call this: code running
// under a custom memory allocator that forbids cudaMalloc during its hot loop, real-time
// control loops with no room for allocation latency, and hosts that hand the library a fixed
// memory budget. gir_gemv(trans = 1) allocates a buffer of partial sums on every call; this
// entry point runs the same two kernels (column partial sums per row chunk, then their sum)
// with the partial sums placed in a fixed array that lives in the library's device image.
//
// The array holds GIR_NOALLOC_SCRATCH = 2^19 doubles (4 MiB); a call needs ceil(n / 256) * n of
// them, so n is limited to 11520 (45 * 11520 = 518400 fit; n = 11521 would need 46 * 11521 =
// 529966). Every GPU that loads the library keeps the array until the process exits.
// All calls share it: two calls whose kernels overlap on the GPU (different streams, or
// different host threads) race on it and must not be issued. Nothing in it needs to start at
// zero, because every partial sum is written before it is read.
#include <atomic>
#include <cstdio>

#include "gir_internal.cuh"

#define GIR_NOALLOC_SCRATCH (1 << 19)
#define GIR_NOALLOC_MAX_DEVICES 64
#define GIR_NOALLOC_MAX_N 11520

namespace gir {

static __device__ __align__(256) double g_noalloc_scratch[GIR_NOALLOC_SCRATCH];

// Host-side copies of the array's device address, one per device, filled by the first call
// made with that device current. Host threads may race on the first fill; they all store the
// same address, and the atomics make that race well defined. A cudaDeviceReset unloads the
// module and invalidates the cached address: after one, call nothing of this library on that
// device in the same process.
static std::atomic<double*> g_noalloc_ptr[GIR_NOALLOC_MAX_DEVICES] = {};

static gir_status noalloc_scratch(double** out) {
    int dev = 0;
    GIR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= GIR_NOALLOC_MAX_DEVICES) return GIR_UNSUPPORTED;
    double* cached = g_noalloc_ptr[dev].load(std::memory_order_relaxed);
    if (!cached) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            fprintf(stderr, "gir: cudaGetSymbolAddress of the fixed scratch array failed: %s\n",
                    cudaGetErrorString(e));
            return GIR_CUDA_ERROR;
        }
        cached = static_cast<double*>(p);
        g_noalloc_ptr[dev].store(cached, std::memory_order_relaxed);
    }
    *out = cached;
    return GIR_OK;
}

}  // namespace gir

extern "C" gir_status gir_gemv_t_noalloc(const double* A, int64_t n, int64_t lda, const double* v, double* w,
                                         void* stream) {
    if (!A || !v || !w || n < 1 || lda < n) return GIR_INVALID_ARG;
    const int64_t need = ((n + 255) / 256) * n;
    if (n > GIR_NOALLOC_MAX_N || need > GIR_NOALLOC_SCRATCH) {
        fprintf(stderr,
                "gir_gemv_t_noalloc: n = %lld needs %lld scratch doubles, the fixed array holds %d (n <= %d)\n",
                (long long)n, (long long)need, GIR_NOALLOC_SCRATCH, GIR_NOALLOC_MAX_N);
        return GIR_INVALID_ARG;
    }
    double* scratch = nullptr;
    GIR_TRY(gir::noalloc_scratch(&scratch));
    return gir::launch_gemv(A, n, lda, v, w, 1, scratch, (cudaStream_t)stream);
}
