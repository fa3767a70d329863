// Bandwidth-bound kernels of the solve path: residual (Algorithm 4), the FP64
// matrix-vector products inside A~ (the correction equation), and the tall-skinny products of GCRO-DR
// (Algorithm 3: projections against [C_k V], solution/residual/recycle updates).
//
// Layouts: A is FP64 row-major with leading dimension lda; the Krylov/recycle bases are
// column-major n x p blocks (column stride ldx), so every column is a contiguous vector.
#include "gir_internal.cuh"

namespace gir {

// ------------------------------------------------------------------ row dot products
// MODE 0: w_i = sum_j a_ij v_j            (FP64 FMA)
// MODE 1: r_i = b_i - sum_j a_ij x_j      (FP64 FMA)
// MODE 2: r_i = b_i - sum_j a_ij x_j      (double-double: exact FMA products, TwoSum accumulation)
// One warp per row, 16-byte loads along the row when the row start is 16-byte aligned.
// CW (MODE 1, 2): also den_i = sum_j |a_ij| |x_j| + |b_i| and the componentwise backward error
// omega = max_i |r_i| / den_i (0/0 = 0, r/0 = inf), merged into *omax as the bit pattern of a
// non-negative double (those order like unsigned integers).
template <int MODE, bool VEC, bool CW>
__global__ void __launch_bounds__(256) k_rowdot(const double* __restrict__ A, int64_t n, int64_t lda,
                                                const double* __restrict__ x, const double* __restrict__ b,
                                                double* __restrict__ out, unsigned long long* __restrict__ omax) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    double qmax = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps_total) {
        const double* row = A + i * lda;
        double sh = 0.0, sl = 0.0, den = 0.0;
        if (VEC) {
            const double2* row2 = reinterpret_cast<const double2*>(row);
            const double2* x2 = reinterpret_cast<const double2*>(x);
            int64_t n2 = n >> 1;
#pragma unroll 4
            for (int64_t j = lane; j < n2; j += 32) {
                double2 a = __ldcs(row2 + j);
                double2 v = __ldg(x2 + j);
                if (CW) den = fma(fabs(a.x), fabs(v.x), fma(fabs(a.y), fabs(v.y), den));
                if (MODE == 2) {
                    double p = a.x * v.x, e = fma(a.x, v.x, -p);
                    double s = sh + p, bb = s - sh, t = (sh - (s - bb)) + (p - bb);
                    sh = s; sl += t + e;
                    p = a.y * v.y; e = fma(a.y, v.y, -p);
                    s = sh + p; bb = s - sh; t = (sh - (s - bb)) + (p - bb);
                    sh = s; sl += t + e;
                } else {
                    sh = fma(a.x, v.x, sh);
                    sl = fma(a.y, v.y, sl);
                }
            }
            if ((n & 1) && lane == 0) {
                double a = row[n - 1], v = x[n - 1];
                if (CW) den = fma(fabs(a), fabs(v), den);
                if (MODE == 2) {
                    double p = a * v, e = fma(a, v, -p);
                    double s = sh + p, bb = s - sh, t = (sh - (s - bb)) + (p - bb);
                    sh = s; sl += t + e;
                } else {
                    sh = fma(a, v, sh);
                }
            }
        } else {
#pragma unroll 4
            for (int64_t j = lane; j < n; j += 32) {
                double a = __ldcs(row + j), v = __ldg(x + j);
                if (CW) den = fma(fabs(a), fabs(v), den);
                if (MODE == 2) {
                    double p = a * v, e = fma(a, v, -p);
                    double s = sh + p, bb = s - sh, t = (sh - (s - bb)) + (p - bb);
                    sh = s; sl += t + e;
                } else {
                    sh = fma(a, v, sh);
                }
            }
        }
        double ri = 0.0;
        if (MODE != 2) {
            double s = warp_sum(sh + sl);
            if (lane == 0) {
                ri = (MODE == 0) ? s : (b[i] - s);
                out[i] = ri;
            }
        } else {
            // double-double butterfly reduction of (sh, sl)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double oh = __shfl_xor_sync(0xffffffffu, sh, o);
                double ol = __shfl_xor_sync(0xffffffffu, sl, o);
                double s = sh + oh, bb = s - sh, t = (sh - (s - bb)) + (oh - bb);
                t += sl + ol;
                sh = s + t;
                sl = t - (sh - s);
            }
            if (lane == 0) {
                // r = b - (sh + sl), in double-double then rounded
                double bi = b[i];
                double s = bi - sh, bb = s - bi, t = (bi - (s - bb)) + (-sh - bb);
                t -= sl;
                ri = s + t;
                out[i] = ri;
            }
        }
        if (CW) {
            den = warp_sum(den);
            if (lane == 0) {
                const double d = den + fabs(b[i]);
                const double q = (d > 0.0) ? fabs(ri) / d : (ri == 0.0 ? 0.0 : __longlong_as_double(0x7ff0000000000000ll));
                // NaN compares false: keep it visible by taking its (largest) bit pattern
                qmax = (q >= qmax || !(q == q)) ? q : qmax;
            }
        }
    }
    if (CW) {
        __shared__ unsigned long long wmax[8];
        const unsigned long long qb = (unsigned long long)__double_as_longlong(fabs(qmax));
        if (lane == 0) wmax[threadIdx.x >> 5] = qb;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long m = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = wmax[w] > m ? wmax[w] : m;
            atomicMax(omax, m);
        }
    }
}

static int grid_for_rows(int64_t n) {
    int64_t g = (n + 7) / 8;  // 8 warps per block
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

static bool aligned16(const void* p, int64_t ld) {
    return ((uintptr_t)p % 16 == 0) && (ld % 2 == 0);
}

gir_status launch_residual(const double* A, int64_t n, int64_t lda, const double* x, const double* b,
                           double* r, int dd, cudaStream_t s, double* omega) {
    if (n <= 0) return GIR_OK;
    int g = grid_for_rows(n);
    bool v = aligned16(A, lda) && ((uintptr_t)x % 16 == 0);
    unsigned long long* om = reinterpret_cast<unsigned long long*>(omega);
    if (om) GIR_CUDA_TRY(cudaMemsetAsync(om, 0, sizeof(double), s));
#define GIR_ROWDOT(M, V)                                                                      \
    if (om) count_launch(), k_rowdot<M, V, true><<<g, 256, 0, s>>>(A, n, lda, x, b, r, om);  \
    else count_launch(), k_rowdot<M, V, false><<<g, 256, 0, s>>>(A, n, lda, x, b, r, nullptr)
    if (dd) {
        if (v) { GIR_ROWDOT(2, true); } else { GIR_ROWDOT(2, false); }
    } else {
        if (v) { GIR_ROWDOT(1, true); } else { GIR_ROWDOT(1, false); }
    }
#undef GIR_ROWDOT
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

// ------------------------------------------------------------------ A^T v
// Block (row chunk rc, column chunk cc): partial[rc][j] = sum_{i in rc} a_ij v_i.
constexpr int GT_ROWS = 256;
constexpr int GT_COLS = 512;  // 256 threads x 2 columns

__global__ void __launch_bounds__(256) k_gemv_t_partial(const double* __restrict__ A, int64_t n, int64_t lda,
                                                        const double* __restrict__ v, double* __restrict__ part) {
    const int64_t i0 = (int64_t)blockIdx.y * GT_ROWS;
    const int64_t j = (int64_t)blockIdx.x * GT_COLS + threadIdx.x * 2;
    const int64_t i1 = min(n, i0 + GT_ROWS);
    double a0 = 0.0, a1 = 0.0;
    for (int64_t i = i0; i < i1; ++i) {
        double vi = __ldg(v + i);
        const double* row = A + i * lda;
        if (j < n) a0 = fma(__ldcs(row + j), vi, a0);
        if (j + 1 < n) a1 = fma(__ldcs(row + j + 1), vi, a1);
    }
    double* p = part + (int64_t)blockIdx.y * n;
    if (j < n) p[j] = a0;
    if (j + 1 < n) p[j + 1] = a1;
}

__global__ void k_sum_rows(const double* __restrict__ part, int nparts, int64_t n, double* __restrict__ out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < nparts; ++q) s += part[(int64_t)q * n + j];
        out[j] = s;
    }
}

gir_status launch_gemv(const double* A, int64_t n, int64_t lda, const double* v, double* w, int trans,
                       double* scratch, cudaStream_t s) {
    if (n <= 0) return GIR_OK;
    if (!trans) {
        int g = grid_for_rows(n);
        if (aligned16(A, lda) && ((uintptr_t)v % 16 == 0)) count_launch(), k_rowdot<0, true, false><<<g, 256, 0, s>>>(A, n, lda, v, nullptr, w, nullptr);
        else count_launch(), k_rowdot<0, false, false><<<g, 256, 0, s>>>(A, n, lda, v, nullptr, w, nullptr);
    } else {
        dim3 grid((unsigned)((n + GT_COLS - 1) / GT_COLS), (unsigned)((n + GT_ROWS - 1) / GT_ROWS));
        count_launch(), k_gemv_t_partial<<<grid, 256, 0, s>>>(A, n, lda, v, scratch);
        count_launch(), k_sum_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(scratch, (int)grid.y, n, w);
    }
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

// ------------------------------------------------------------------ tall-skinny X^T Y
// G[c + t*p] = sum_i X[i, c] Y[i, t]. Block (b, g) covers rows [b TS_CHUNK, (b+1) TS_CHUNK) for
// the pairs (c, t) with index 8 g .. 8 g + 7, one warp per pair: the FP64 products (one warp
// instruction per 64 cycles of an SM sub-partition on this GPU) spread over every SM rather
// than over one CTA per row chunk. Partial sums per chunk go to part[b * pairs + pair].
constexpr int TS_CHUNK = 1024;
constexpr int TS_PAIRS = 8;   // pairs per CTA (one per warp)

__global__ void __launch_bounds__(256) k_gemm_tn_partial(const double* __restrict__ X, int64_t ldx, int p,
                                                         const double* __restrict__ Y, int64_t ldy, int q,
                                                         int64_t n, double* __restrict__ part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * TS_CHUNK;
    const int64_t i1 = min(n, i0 + TS_CHUNK);
    const int pairs = p * q;
    const int pq = (int)blockIdx.y * TS_PAIRS + warp;
    if (pq >= pairs) return;   // the warp's pair does not exist (no CTA barrier follows)
    const int c = pq % p, t = pq / p;
    const double* xc = X + (int64_t)c * ldx;
    const double* yt = Y + (int64_t)t * ldy;
    double acc = 0.0;
#pragma unroll 8
    for (int64_t i = i0 + lane; i < i1; i += 32) acc = fma(xc[i], yt[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) part[(int64_t)blockIdx.x * pairs + pq] = acc;
}

__global__ void k_sum_parts(const double* __restrict__ part, int nparts, int p, int cnt, int ldg,
                            double* __restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < nparts; ++q) s += part[(int64_t)q * cnt + e];
        out[(e % p) + (int64_t)(e / p) * ldg] = s;
    }
}

gir_status launch_gemm_tn(const double* X, int64_t ldx, int p, const double* Y, int64_t ldy, int q, int64_t n,
                          double* G, int ldg, double* scratch, cudaStream_t s) {
    if (p <= 0 || q <= 0) return GIR_OK;
    int nb = (int)((n + TS_CHUNK - 1) / TS_CHUNK);
    if (nb < 1) nb = 1;
    int cnt = p * q;
    const dim3 grid((unsigned)nb, (unsigned)((cnt + TS_PAIRS - 1) / TS_PAIRS), 1);
    count_launch(), k_gemm_tn_partial<<<grid, 256, 0, s>>>(X, ldx, p, Y, ldy, q, n, scratch);
    count_launch(), k_sum_parts<<<(cnt + 127) / 128, 128, 0, s>>>(scratch, nb, p, cnt, ldg, G);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

gir_status launch_multidot(const double* X, int64_t ldx, int ncols, const double* y, int64_t n, double* out,
                           double* scratch, cudaStream_t s) {
    return launch_gemm_tn(X, ldx, ncols, y, n, 1, n, out, ncols, scratch, s);
}

// ------------------------------------------------------------------ Y = beta Y + X Cf
// Thread per row (128-thread CTAs, so that the rows of n = 16384 reach 128 SMs); coefficients
// staged in shared memory; outputs in groups of 8 columns. Each row's sum runs over c in order;
// the loads of 8 columns are issued ahead of their products.
constexpr int NN_THREADS = 128;
__global__ void __launch_bounds__(NN_THREADS) k_gemm_nn(const double* __restrict__ X, int64_t ldx, int p,
                                                 const double* __restrict__ Cf, int ldc, int q,
                                                 double* __restrict__ Y, int64_t ldy, double alpha, double beta,
                                                 int64_t n, int round32) {
    extern __shared__ double sc[];
    for (int e = threadIdx.x; e < p * q; e += blockDim.x) {
        int c = e % p, t = e / p;
        sc[e] = Cf[c + (int64_t)t * ldc];
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int t0 = 0; t0 < q; t0 += 8) {
            double acc[8];
#pragma unroll
            for (int tt = 0; tt < 8; ++tt) acc[tt] = 0.0;
            int c = 0;
            for (; c + 8 <= p; c += 8) {
                double xv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) xv[u] = X[i + (int64_t)(c + u) * ldx];
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int tt = 0; tt < 8; ++tt)
                        if (t0 + tt < q) acc[tt] = fma(xv[u], sc[c + u + (t0 + tt) * p], acc[tt]);
            }
            for (; c < p; ++c) {
                const double xv = X[i + (int64_t)c * ldx];
#pragma unroll
                for (int tt = 0; tt < 8; ++tt)
                    if (t0 + tt < q) acc[tt] = fma(xv, sc[c + (t0 + tt) * p], acc[tt]);
            }
#pragma unroll
            for (int tt = 0; tt < 8; ++tt) {
                if (t0 + tt < q) {
                    double* y = Y + i + (int64_t)(t0 + tt) * ldy;
                    double v = (beta == 0.0) ? alpha * acc[tt] : fma(beta, *y, alpha * acc[tt]);
                    if (round32) v = (double)__double2float_rn(v);
                    *y = v;
                }
            }
        }
    }
}

gir_status launch_gemm_nn(const double* X, int64_t ldx, int p, const double* Cf, int ldc, int q, double* Y,
                          int64_t ldy, double alpha, double beta, int64_t n, int round32, cudaStream_t s) {
    if (q <= 0 || n <= 0) return GIR_OK;
    if (p <= 0) {
        // Y = beta Y
        if (beta == 0.0) {
            for (int t = 0; t < q; ++t) GIR_CUDA_TRY(cudaMemsetAsync(Y + (int64_t)t * ldy, 0, n * sizeof(double), s));
            return GIR_OK;
        }
        if (beta == 1.0) return GIR_OK;
    }
    size_t smem = (size_t)p * q * sizeof(double);
    if (smem > 48 * 1024) {
        static std::atomic<unsigned> attr_done{0};
        GIR_CUDA_TRY(ensure_dyn_smem((const void*)k_gemm_nn, 200 * 1024, attr_done));
        if (smem > 200 * 1024) return GIR_INVALID_ARG;
    }
    int g = (int)gmin<int64_t>((n + NN_THREADS - 1) / NN_THREADS, 152 * 16);
    count_launch(), k_gemm_nn<<<g, NN_THREADS, smem, s>>>(X, ldx, p, Cf, ldc, q, Y, ldy, alpha, beta, n, round32);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

// ------------------------------------------------------------------ norms
__global__ void __launch_bounds__(256) k_sumsq_partial(const double* __restrict__ x, int64_t n,
                                                       double* __restrict__ part) {
    __shared__ double sw[8];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = fma(x[i], x[i], acc);
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < 8 ? sw[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

__global__ void k_finish_norm2(const double* __restrict__ part, int nparts, double* __restrict__ out) {
    double acc = 0.0;
    for (int q = threadIdx.x; q < nparts; q += 32) acc += part[q];
    acc = warp_sum(acc);
    if (threadIdx.x == 0) *out = sqrt(acc);
}

gir_status launch_norm2(const double* x, int64_t n, double* out, double* scratch, cudaStream_t s) {
    int g = (int)gmin<int64_t>((n + 255) / 256, 256);
    if (g < 1) g = 1;
    count_launch(), k_sumsq_partial<<<g, 256, 0, s>>>(x, n, scratch);
    count_launch(), k_finish_norm2<<<1, 32, 0, s>>>(scratch, g, out);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

__global__ void __launch_bounds__(256) k_absmax(const double* __restrict__ x, int64_t n, unsigned long long* out) {
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = fabs(x[i]);
        if (!(v <= m)) m = v;  // propagates NaN
    }
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

gir_status launch_norminf(const double* x, int64_t n, double* out, cudaStream_t s) {
    GIR_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), s));
    int g = (int)gmin<int64_t>((n + 255) / 256, 256);
    if (g < 1) g = 1;
    count_launch(), k_absmax<<<g, 256, 0, s>>>(x, n, reinterpret_cast<unsigned long long*>(out));
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

// ||A||_inf = max_i sum_j |a_ij|: one warp per row.
__global__ void __launch_bounds__(256) k_rowabs(const double* __restrict__ A, int64_t n, int64_t lda,
                                                double* __restrict__ rs) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps_total) {
        double acc = 0.0;
        for (int64_t j = lane; j < n; j += 32) acc += fabs(A[i * lda + j]);
        acc = warp_sum(acc);
        if (lane == 0) rs[i] = acc;
    }
}

gir_status launch_matrix_norminf(const double* A, int64_t n, int64_t lda, double* out, double* scratch,
                                 cudaStream_t s) {
    count_launch(), k_rowabs<<<grid_for_rows(n), 256, 0, s>>>(A, n, lda, scratch);
    GIR_CUDA_TRY(cudaGetLastError());
    return launch_norminf(scratch, n, out, s);
}


// G = alpha * u v^T (n x n, row-major, leading dimension ldg): the gradient dA = -lambda x^T of a
// loss of x = A^-1 b. Each CTA writes whole rows with 16-byte stores where the row pitch allows.
__global__ void __launch_bounds__(256) k_outer(const double* __restrict__ u, const double* __restrict__ v, int64_t n,
                                               double alpha, double* __restrict__ G, int64_t ldg) {
    const bool vec = ((ldg & 1) == 0) && ((reinterpret_cast<uintptr_t>(G) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(v) & 15) == 0);
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const double ui = alpha * u[i];
        double* g = G + i * ldg;
        if (vec) {
            for (int64_t j = 2 * (int64_t)threadIdx.x; j + 1 < n; j += 2 * (int64_t)blockDim.x) {
                const double2 vv = *reinterpret_cast<const double2*>(v + j);
                *reinterpret_cast<double2*>(g + j) = make_double2(ui * vv.x, ui * vv.y);
            }
            if ((n & 1) && threadIdx.x == 0) g[n - 1] = ui * v[n - 1];
        } else {
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x) g[j] = ui * v[j];
        }
    }
}

gir_status launch_outer(const double* u, const double* v, int64_t n, double alpha, double* G, int64_t ldg,
                        cudaStream_t s) {
    const int g = (int)gmin<int64_t>(n, 152 * 16);
    count_launch(), k_outer<<<g, 256, 0, s>>>(u, v, n, alpha, G, ldg);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}


// ------------------------------------------------------------------ float-float A v
// w = A v with A held as two FP32 matrices (A_hi = RN32(a), A_lo = RN32(a - A_hi), so
// A_hi + A_lo carries 48 significand bits of each FP64 entry) and v split the same way, in
// float-float arithmetic: exact products by FMA (TwoProduct) accumulated with TwoSum. The
// operator M^-1 A of the correction solves is then applied at one precision (the triangular
// solves are float-float as well), and the matrix-vector product streams 8 bytes per entry at
// FP32 arithmetic rates instead of being limited by the FP64 pipe.
__global__ void k_split_ff(const double* __restrict__ v, int64_t n, float* __restrict__ vh, float* __restrict__ vl) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double a = v[i];
        const float h = __double2float_rn(a);
        vh[i] = h;
        vl[i] = __double2float_rn(a - (double)h);
    }
}

__device__ __forceinline__ void ff_mac(float& sh, float& sl, float ah, float al, float vh, float vl) {
    const float p = ah * vh;
    float e = fmaf(ah, vh, -p);
    e = fmaf(ah, vl, e);
    e = fmaf(al, vh, e);
    const float s = sh + p;
    const float bb = s - sh;
    const float t = (sh - (s - bb)) + (p - bb);
    sh = s;
    sl += t + e;
}

// one warp per row; ldf % 4 == 0 and 16-byte aligned A_hi, A_lo, vh, vl (float4 loads)
__global__ void __launch_bounds__(256) k_gemv_ff(const float* __restrict__ Ah, const float* __restrict__ Al,
                                                 int64_t ldf, int64_t n, const float* __restrict__ vh,
                                                 const float* __restrict__ vl, double* __restrict__ w) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t n4 = n >> 2;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps_total) {
        const float4* rh = reinterpret_cast<const float4*>(Ah + i * ldf);
        const float4* rl = reinterpret_cast<const float4*>(Al + i * ldf);
        const float4* xh = reinterpret_cast<const float4*>(vh);
        const float4* xl = reinterpret_cast<const float4*>(vl);
        float sh = 0.0f, sl = 0.0f;
#pragma unroll 2
        for (int64_t j = lane; j < n4; j += 32) {
            const float4 a = __ldcs(rh + j), b = __ldcs(rl + j);
            const float4 c = __ldg(xh + j), d = __ldg(xl + j);
            ff_mac(sh, sl, a.x, b.x, c.x, d.x);
            ff_mac(sh, sl, a.y, b.y, c.y, d.y);
            ff_mac(sh, sl, a.z, b.z, c.z, d.z);
            ff_mac(sh, sl, a.w, b.w, c.w, d.w);
        }
        for (int64_t j = n4 * 4 + lane; j < n; j += 32)
            ff_mac(sh, sl, Ah[i * ldf + j], Al[i * ldf + j], vh[j], vl[j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, sh, o);
            const float ol = __shfl_xor_sync(0xffffffffu, sl, o);
            const float s2 = sh + oh, bb = s2 - sh, t = (sh - (s2 - bb)) + (oh - bb);
            sh = s2;
            sl += t + ol;
        }
        if (lane == 0) w[i] = (double)sh + (double)sl;
    }
}

// A_hi = RN32(A), A_lo = RN32(A - A_hi), row by row (16-byte loads where A allows)
__global__ void __launch_bounds__(256) k_split_matrix(const double* __restrict__ A, int64_t n, int64_t lda,
                                                      float* __restrict__ Ah, float* __restrict__ Al, int64_t ldf) {
    const bool vec = ((lda & 1) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const double* a = A + i * lda;
        float* h = Ah + i * ldf;
        float* l = Al + i * ldf;
        if (vec) {
            for (int64_t j = 2 * (int64_t)threadIdx.x; j + 1 < n; j += 2 * (int64_t)blockDim.x) {
                const double2 v = *reinterpret_cast<const double2*>(a + j);
                const float h0 = __double2float_rn(v.x), h1 = __double2float_rn(v.y);
                *reinterpret_cast<float2*>(h + j) = make_float2(h0, h1);
                *reinterpret_cast<float2*>(l + j) =
                    make_float2(__double2float_rn(v.x - (double)h0), __double2float_rn(v.y - (double)h1));
            }
            if ((n & 1) && threadIdx.x == 0) {
                const float h0 = __double2float_rn(a[n - 1]);
                h[n - 1] = h0;
                l[n - 1] = __double2float_rn(a[n - 1] - (double)h0);
            }
        } else {
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
                const float h0 = __double2float_rn(a[j]);
                h[j] = h0;
                l[j] = __double2float_rn(a[j] - (double)h0);
            }
        }
    }
}

gir_status launch_split_matrix(const double* A, int64_t n, int64_t lda, float* Ah, float* Al, int64_t ldf,
                               int max_ctas, cudaStream_t s) {
    count_launch(), k_split_matrix<<<(unsigned)gmin<int64_t>(n, max_ctas), 256, 0, s>>>(A, n, lda, Ah, Al, ldf);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

gir_status launch_gemv_ff(const float* Ah, const float* Al, int64_t ldf, int64_t n, const double* v, double* w,
                          float* vsplit, cudaStream_t s) {
    if (n <= 0) return GIR_OK;
    float* vh = vsplit;
    float* vl = vsplit + ((n + 3) / 4) * 4;
    count_launch(), k_split_ff<<<(unsigned)gmin<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(v, n, vh, vl);
    count_launch(), k_gemv_ff<<<grid_for_rows(n), 256, 0, s>>>(Ah, Al, ldf, n, vh, vl, w);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

}  // namespace gir
