// Internal declarations of the GB300 GMRES-IR library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>

#include "../../include/gir.h"

#define GIR_CUDA_TRY(expr)                                                        \
    do {                                                                          \
        cudaError_t e_ = (expr);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            fprintf(stderr, "gir: CUDA error %s at %s:%d: %s\n", #expr, __FILE__, \
                    __LINE__, cudaGetErrorString(e_));                            \
            return GIR_CUDA_ERROR;                                                \
        }                                                                         \
    } while (0)

#define GIR_TRY(expr)                       \
    do {                                    \
        gir_status s_ = (expr);             \
        if (s_ != GIR_OK) return s_;        \
    } while (0)

namespace gir {

// Raises a kernel's dynamic shared-memory limit once per device. Safe from several host threads
// (the batch solve's workers): a race only repeats the idempotent call.
inline cudaError_t ensure_dyn_smem(const void* fn, int bytes, std::atomic<unsigned>& done) {
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned bit = 1u << (dev & 31);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// Host-side count of kernel launches made by this library (all streams, all handles).
void count_launch();
unsigned long long launch_count();

// Device-side status flags (bit mask in a global int).
enum : int {
    DEV_SINGULAR = 1,
    DEV_NONFINITE = 2,
    DEV_TIMEOUT = 4,
};

// Bounded spin budget for every device-side wait (about a second of polling).
constexpr long long SPIN_LIMIT = 20000000LL;

constexpr int WARP = 32;

template <typename T>
__host__ __device__ __forceinline__ T gmin(T a, T b) { return a < b ? a : b; }
template <typename T>
__host__ __device__ __forceinline__ T gmax(T a, T b) { return a > b ? a : b; }

// ----------------------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ----------------------------------------------------------------------------- float-float
// Unevaluated pair (hi, lo) of FP32 numbers; Knuth TwoSum and FMA-based TwoProduct keep
// about 48 significand bits. Used where GB300's FP64 rate (1/64 of FP32) would make an
// FP64-accurate stream ALU-bound.
struct ff { float h, l; };

__device__ __forceinline__ ff ff_from_double(double a) {
    float h = __double2float_rn(a);
    float l = __double2float_rn(a - (double)h);
    return {h, l};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.h + (double)a.l; }

// acc += x * y with x exact in FP32 (e.g. a bf16/fp16 value) and y = (yh, yl).
__device__ __forceinline__ void ff_acc_prod1(float& sh, float& sl, float x, float yh, float yl) {
    float p = x * yh;
    float e = fmaf(x, yh, -p);
    e = fmaf(x, yl, e);
    float s = sh + p;
    float bb = s - sh;
    float t = (sh - (s - bb)) + (p - bb);
    sh = s;
    sl += t + e;
}
// acc += (xh, xl) * (yh, yl)
__device__ __forceinline__ void ff_acc_prod2(float& sh, float& sl, float xh, float xl, float yh, float yl) {
    float p = xh * yh;
    float e = fmaf(xh, yh, -p);
    e = fmaf(xh, yl, e);
    e = fmaf(xl, yh, e);
    float s = sh + p;
    float bb = s - sh;
    float t = (sh - (s - bb)) + (p - bb);
    sh = s;
    sl += t + e;
}
// acc += (xh, xl)
__device__ __forceinline__ void ff_acc_add(float& sh, float& sl, float xh, float xl) {
    float s = sh + xh;
    float bb = s - sh;
    float t = (sh - (s - bb)) + (xh - bb);
    sh = s;
    sl += t + xl;
}
__device__ __forceinline__ ff ff_norm(float h, float l) {
    float s = h + l;
    float e = l - (s - h);
    return {s, e};
}

// ----------------------------------------------------------------------------- factor format
// Factors are stored as 16-bit patterns: bf16 or fp16 (u_f). FP8-E4M3 factors (values
// RN_e4m3(x s) / s with a power-of-two scale s per 128 x 128 tile) have at most 4 significant
// bits and are stored exactly as bf16 patterns, so they use FF_BF16 from the factorization on.
enum FactorFmt : int { FF_BF16 = 0, FF_FP16 = 1 };

__device__ __forceinline__ float uf_to_float(uint16_t v, int fmt) {
    if (fmt == FF_BF16) return __bfloat162float(__ushort_as_bfloat16(v));
    return __half2float(__ushort_as_half(v));
}
__device__ __forceinline__ uint16_t float_to_uf(float x, int fmt) {
    if (fmt == FF_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return __half_as_ushort(__float2half_rn(x));
}

// ----------------------------------------------------------------------------- launchers
// vector / tall-skinny kernels (k_vec.cu)
// r = b - A x in FP64 (dd = 0) or double-double (dd = 1); with omega != nullptr also the
// componentwise backward error max_i |r_i| / (|A||x| + |b|)_i into the device scalar *omega
gir_status launch_residual(const double* A, int64_t n, int64_t lda, const double* x, const double* b,
                           double* r, int dd, cudaStream_t s, double* omega = nullptr);
gir_status launch_gemv(const double* A, int64_t n, int64_t lda, const double* v, double* w,
                       int trans, double* scratch, cudaStream_t s);
// out[c] = sum_i X[i, c] * y[i] for c < ncols (X column-major, stride ldx); partial sums in scratch
gir_status launch_multidot(const double* X, int64_t ldx, int ncols, const double* y, int64_t n,
                           double* out, double* scratch, cudaStream_t s);
// G = X^T Y (p x q, column-major with leading dimension ldg) for X n x p, Y n x q column-major
gir_status launch_gemm_tn(const double* X, int64_t ldx, int p, const double* Y, int64_t ldy, int q,
                          int64_t n, double* G, int ldg, double* scratch, cudaStream_t s);
// Y[:, c] = beta * Y[:, c] + alpha * sum_j X[:, j] * Cf[j + c*ldc] for c < q (X n x p);
// coefficients on the device; round32 rounds the results to FP32.
gir_status launch_gemm_nn(const double* X, int64_t ldx, int p, const double* Cf, int ldc, int q,
                          double* Y, int64_t ldy, double alpha, double beta, int64_t n, int round32,
                          cudaStream_t s);
gir_status launch_norm2(const double* x, int64_t n, double* out, double* scratch, cudaStream_t s);
// w = A v in float-float from the FP32 split A = A_hi + A_lo (leading dimension ldf, a multiple
// of 4; 16-byte aligned); vsplit: scratch of 2 * ceil4(n) floats
// A_hi = RN32(A), A_lo = RN32(A - A_hi) (ldf: row pitch of the FP32 halves, even), on at most
// max_ctas CTAs
gir_status launch_split_matrix(const double* A, int64_t n, int64_t lda, float* Ah, float* Al, int64_t ldf,
                               int max_ctas, cudaStream_t s);
gir_status launch_gemv_ff(const float* Ah, const float* Al, int64_t ldf, int64_t n, const double* v, double* w,
                          float* vsplit, cudaStream_t s);
// G = alpha u v^T (n x n, row-major)
gir_status launch_outer(const double* u, const double* v, int64_t n, double alpha, double* G, int64_t ldg,
                        cudaStream_t s);
gir_status launch_norminf(const double* x, int64_t n, double* out, cudaStream_t s);
gir_status launch_matrix_norminf(const double* A, int64_t n, int64_t lda, double* out, double* scratch,
                                 cudaStream_t s);

// LU (k_lu.cu)
struct LUPlan;
// TRSV (k_trsv.cu)
struct TrsvPlan;

}  // namespace gir
