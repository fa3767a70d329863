// The preconditioned operator A~ = M^-1 A applied in double-double (unit roundoff about
// 2^-106): the paper's u_a = u^2 for the working precision u = FP64 (Algorithm 4, the correction equation; the
// paper simulates quad precision, double-double keeps the u^2 level). The product A v, both
// substitutions with the u_f factors and the diagonal-block inverses are carried in
// double-double without an intermediate rounding; only the result is rounded to u.
//
// Arithmetic: Knuth's TwoSum and the FMA form of Dekker's TwoProduct (p + e = a b exactly with
// e = fma(a, b, -p)); sums accumulate as (hi, lo) with one TwoSum per term, so their error is
// of order 2^-106 times the sum of the absolute terms; the division by a pivot takes two
// correction quotients from exact remainders.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so this path is ALU-bound and several
// times slower than the float-float default; it exists for the accuracy regime that needs it.
//
// Triangular solves: the ticketed persistent scheme of k_trsv.cu with 32-row blocks (a block's
// last tile and its diagonal product, on the critical path, cost 2 x 1024 double-double
// multiply-adds on one SM). Block results are published with a per-block epoch flag written
// with release semantics after the block's stores; consumers poll it with acquire loads, with
// a bounded wait that raises the abort flag.
#include "k_dd.cuh"
#include "trace.cuh"

namespace gir {

constexpr int DB = DD_BLOCK;
constexpr int DT = 4 * DB;  // threads per CTA: row r = tid / 4, columns 8 q .. 8 q + 7, q = tid % 4

// ------------------------------------------------------------------ double-double helpers
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    e = b - (s - a);
}
// (sh, sl) += ph + pl, with (ph, pl) a double-double term; (sh, sl) stays normalised
__device__ __forceinline__ void dd_acc(double& sh, double& sl, double ph, double pl) {
    double s, t;
    two_sum(sh, ph, s, t);
    t += sl + pl;
    fast_two_sum(s, t, sh, sl);
}
// (sh, sl) += a (yh + yl) for an FP64 a
__device__ __forceinline__ void dd_mac_d(double& sh, double& sl, double a, double yh, double yl) {
    const double p = a * yh;
    double e = fma(a, yh, -p);
    e = fma(a, yl, e);
    dd_acc(sh, sl, p, e);
}
// (sh, sl) += (ah + al)(bh + bl)
__device__ __forceinline__ void dd_mac_dd(double& sh, double& sl, double ah, double al, double bh, double bl) {
    const double p = ah * bh;
    double e = fma(ah, bh, -p);
    e = fma(ah, bl, e);
    e = fma(al, bh, e);
    dd_acc(sh, sl, p, e);
}
// (ah + al) / b for an FP64 b: quotient q1 plus two corrections from exact remainders
__device__ __forceinline__ void dd_div_d(double ah, double al, double b, double& qh, double& ql) {
    const double q1 = ah / b;
    double p = q1 * b, pe = fma(q1, b, -p);
    double rh = ah, rl = al;
    dd_acc(rh, rl, -p, -pe);
    const double q2 = rh / b;
    p = q2 * b;
    pe = fma(q2, b, -p);
    dd_acc(rh, rl, -p, -pe);
    const double q3 = rh / b;
    double s, e;
    fast_two_sum(q1, q2, s, e);
    dd_acc(s, e, q3, 0.0);
    qh = s;
    ql = e;
}
// sum of (sh, sl) over the 4 lanes of a row group (lanes xor 1, 2)
__device__ __forceinline__ void dd_quad_reduce(double& sh, double& sl) {
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        const double oh = __shfl_xor_sync(0xffffffffu, sh, o);
        const double ol = __shfl_xor_sync(0xffffffffu, sl, o);
        dd_acc(sh, sl, oh, ol);
    }
}
__device__ __forceinline__ void dd_warp_reduce(double& sh, double& sl) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double oh = __shfl_xor_sync(0xffffffffu, sh, o);
        const double ol = __shfl_xor_sync(0xffffffffu, sl, o);
        dd_acc(sh, sl, oh, ol);
    }
}

// ------------------------------------------------------------------ A v and A^T v
// w_i = sum_j a_ij v_j: one warp per row, exact products, double-double sums
__global__ void __launch_bounds__(256) k_gemv_dd(const double* __restrict__ A, int64_t n, int64_t lda,
                                                 const double* __restrict__ v, double2* __restrict__ w) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const double* row = A + i * lda;
        double sh = 0.0, sl = 0.0;
        // high parts summed by TwoSum; product and sum errors collected in sl, normalised once
        for (int64_t j = lane; j < n; j += 32) {
            const double a = __ldcs(row + j), x = __ldg(v + j);
            const double p = a * x;
            double hs, ht;
            two_sum(sh, p, hs, ht);
            sh = hs;
            sl += ht + fma(a, x, -p);
        }
        fast_two_sum(sh, sl, sh, sl);
        dd_warp_reduce(sh, sl);
        if (lane == 0) w[i] = make_double2(sh, sl);
    }
}
// part[c][j] = sum over rows i of chunk c of a_ij v_i (each thread one column j)
__global__ void __launch_bounds__(256) k_gemv_t_dd_partial(const double* __restrict__ A, int64_t n, int64_t lda,
                                                           const double* __restrict__ v, double2* __restrict__ part) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * DD_TROWS;
    const int64_t i1 = gmin<int64_t>(n, i0 + DD_TROWS);
    if (j >= n) return;
    double sh = 0.0, sl = 0.0;
    for (int64_t i = i0; i < i1; ++i) {
        const double a = __ldcs(A + i * lda + j), x = __ldg(v + i);
        const double p = a * x;
        double hs, ht;
        two_sum(sh, p, hs, ht);
        sh = hs;
        sl += ht + fma(a, x, -p);
    }
    fast_two_sum(sh, sl, sh, sl);
    part[(int64_t)blockIdx.y * n + j] = make_double2(sh, sl);
}
__global__ void k_sum_parts_dd(const double2* __restrict__ part, int nparts, int64_t n, double2* __restrict__ w) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double sh = 0.0, sl = 0.0;
        for (int c = 0; c < nparts; ++c) {
            const double2 p = part[(int64_t)c * n + j];
            dd_acc(sh, sl, p.x, p.y);
        }
        w[j] = make_double2(sh, sl);
    }
}

// r_j = fl64(b_j - sum_c part[c][j]): the transposed residual with A^T x summed in double-double
// (the residual of the adjoint solve in u_r = double-double), one rounding at the end
__global__ void k_resid_t_dd(const double2* __restrict__ part, int nparts, int64_t n, const double* __restrict__ b,
                             double* __restrict__ r) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double sh = 0.0, sl = 0.0;
        for (int c = 0; c < nparts; ++c) {
            const double2 p = part[(int64_t)c * n + j];
            dd_acc(sh, sl, p.x, p.y);
        }
        double rh, rl;
        two_sum(b[j], -sh, rh, rl);
        r[j] = rh + (rl - sl);
    }
}

size_t dd_part_len(int64_t n) { return (size_t)((n + DD_TROWS - 1) / DD_TROWS) * (size_t)n; }

gir_status residual_t_dd(const double* A, int64_t n, int64_t lda, const double* x, const double* b, double* r,
                         double2* part, cudaStream_t s) {
    const dim3 grid((unsigned)((n + 255) / 256), (unsigned)((n + DD_TROWS - 1) / DD_TROWS));
    count_launch(), k_gemv_t_dd_partial<<<grid, 256, 0, s>>>(A, n, lda, x, part);
    count_launch(), k_resid_t_dd<<<(unsigned)gmin<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(part, (int)grid.y, n,
                                                                                               b, r);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

static int rows_grid(int64_t n) { return (int)gmax<int64_t>(1, gmin<int64_t>((n + 7) / 8, 152 * 16)); }

gir_status gemv_dd(DdState& dd, const double* A, int64_t n, int64_t lda, const double* v, int trans, cudaStream_t s) {
    if (!trans) {
        count_launch(), k_gemv_dd<<<rows_grid(n), 256, 0, s>>>(A, n, lda, v, dd.w);
    } else {
        const dim3 grid((unsigned)((n + 255) / 256), (unsigned)((n + DD_TROWS - 1) / DD_TROWS));
        count_launch(), k_gemv_t_dd_partial<<<grid, 256, 0, s>>>(A, n, lda, v, dd.part);
        count_launch(), k_sum_parts_dd<<<(unsigned)gmin<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(
            dd.part, (int)grid.y, n, dd.w);
    }
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

// ------------------------------------------------------------------ diagonal-block inverses
// D[I] = inv(T_II) in double-double for T = L (unit lower, upper = 0) or U (upper = 1), row-major
// DB x DB per block; thread c solves T x = e_c by substitution. Rows/columns beyond n are the
// identity.
__global__ void __launch_bounds__(DB) k_diag_inv_dd(const uint16_t* __restrict__ LU, int64_t ldl, int64_t n, int fmt,
                                                    int upper, double2* __restrict__ D) {
    __shared__ double T[DB][DB + 1];
    __shared__ double Xh[DB][DB + 1], Xl[DB][DB + 1];
    const int64_t base = (int64_t)blockIdx.x * DB;
    const int c = threadIdx.x;
    for (int i = 0; i < DB; ++i) {
        const int64_t gi = base + i, gc = base + c;
        double v;
        if (gi < n && gc < n) {
            v = (double)uf_to_float(LU[gi * ldl + gc], fmt);
            if (!upper) v = (c < i) ? v : (c == i ? 1.0 : 0.0);
            else v = (c >= i) ? v : 0.0;
        } else {
            v = (i == c) ? 1.0 : 0.0;
        }
        T[i][c] = v;
    }
    __syncthreads();
    if (!upper) {
        for (int i = 0; i < DB; ++i) {
            double sh = (i == c) ? 1.0 : 0.0, sl = 0.0;
            for (int q = 0; q < i; ++q) dd_mac_d(sh, sl, -T[i][q], Xh[q][c], Xl[q][c]);
            Xh[i][c] = sh;
            Xl[i][c] = sl;
        }
    } else {
        for (int i = DB - 1; i >= 0; --i) {
            double sh = (i == c) ? 1.0 : 0.0, sl = 0.0;
            for (int q = i + 1; q < DB; ++q) dd_mac_d(sh, sl, -T[i][q], Xh[q][c], Xl[q][c]);
            double qh, ql;
            dd_div_d(sh, sl, T[i][i], qh, ql);
            Xh[i][c] = qh;
            Xl[i][c] = ql;
        }
    }
    __syncthreads();
    for (int i = 0; i < DB; ++i) D[(base + i) * DB + c] = make_double2(Xh[i][c], Xl[i][c]);
}

// ------------------------------------------------------------------ persistent block solve
__device__ __forceinline__ int dd_ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void dd_st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// LOWER: forward order (block I depends on blocks J < I), else backward (J > I).
// TRANS: tile (I, J) is the transpose of the stored tile (J, I) and the diagonal product uses D^T.
template <bool LOWER, bool TRANS>
__global__ void __launch_bounds__(DT) k_trsv_dd(const uint16_t* __restrict__ LU, int64_t ldl, int fmt,
                                                const double2* __restrict__ D, int64_t n, int nblk,
                                                const double2* __restrict__ zin, double2* yout,
                                                int* ready, int epoch,
                                                unsigned long long* __restrict__ ticket_ctr, unsigned long long base,
                                                int* __restrict__ abort_flag, int* __restrict__ flags,
                                                long long spin_limit) {
    __shared__ double2 yj[2][DB];
    __shared__ double2 accs[DB];
    __shared__ int s_ticket, s_abort;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_ticket = (int)(atomicAdd(ticket_ctr, 1ULL) - base);
        s_abort = 0;
    }
    __syncthreads();
    const int t = s_ticket;
    if (t < 0 || t >= nblk) {
        if (tid == 0) { atomicOr(flags, DEV_TIMEOUT); atomicExch(abort_flag, 1); }
        return;
    }
    const int I = LOWER ? t : (nblk - 1 - t);
    const int64_t r0 = (int64_t)I * DB;
    const int r = tid >> 2, q = tid & 3;
    const int64_t gi = r0 + r;
    double ah = 0.0, al = 0.0;
    if (gi < n) {
        const double2 z = zin[gi];
        ah = z.x;
        al = z.y;
    }
    const int ndep = LOWER ? I : (nblk - 1 - I);
    double tv[8];
    auto load_tile = [&](int J) {
        const int64_t c0 = (int64_t)J * DB + q * 8;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int64_t gc = c0 + c;
            double v = 0.0;
            if (gi < n && gc < n) v = (double)uf_to_float(TRANS ? LU[gc * ldl + gi] : LU[gi * ldl + gc], fmt);
            tv[c] = v;
        }
    };
    for (int step = 0; step < ndep; ++step) {
        const int J = LOWER ? step : (nblk - 1 - step);
        const int buf = step & 1;
        load_tile(J);  // independent of y: issued before the wait
        if (tid < DB) {
            const int64_t gc = (int64_t)J * DB + tid;
            double2 v = make_double2(0.0, 0.0);
            if (gc < n) {
                long long spins = 0;
                bool ok = true;
                while (dd_ld_acquire(ready + J) != epoch) {
                    if (((spins & 1023) == 0) && dd_ld_acquire(abort_flag)) { ok = false; break; }
                    if (++spins > spin_limit) {
                        atomicOr(flags, DEV_TIMEOUT);
                        atomicExch(abort_flag, 1);
                        ok = false;
                        break;
                    }
                }
                if (ok) v = __ldcg(yout + gc);
                else s_abort = 1;
            }
            yj[buf][tid] = v;
        }
        __syncthreads();
        if (s_abort) break;
        // 8 terms: exact high products summed by TwoSum, the low parts collected unnormalised
        double sh = 0.0, sl = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const double2 y = yj[buf][q * 8 + c];
            const double a = tv[c];
            const double p = a * y.x;
            double e = fma(a, y.x, -p);
            e = fma(a, y.y, e);
            double hs, ht;
            two_sum(sh, p, hs, ht);
            sh = hs;
            sl += ht + e;
        }
        fast_two_sum(sh, sl, sh, sl);
        dd_quad_reduce(sh, sl);
        dd_acc(ah, al, -sh, -sl);
    }
    // y_I = D_I acc (TRANS: D_I^T acc)
    if (q == 0) accs[r] = make_double2(ah, al);
    __syncthreads();
    double ph = 0.0, pl = 0.0;
    const double2* Dblk = D + (int64_t)I * DB * DB;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int cc = q * 8 + c;
        const double2 d = TRANS ? Dblk[cc * DB + r] : Dblk[r * DB + cc];
        const double2 a = accs[cc];
        dd_mac_dd(ph, pl, d.x, d.y, a.x, a.y);
    }
    dd_quad_reduce(ph, pl);
    if (q == 0 && gi < n) {
        yout[gi] = s_abort ? make_double2(0.0, 0.0) : make_double2(ph, pl);
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        dd_st_release(ready + I, epoch);
    }
}

// The solve CTAs reserve more than half of an SM's shared memory so that each runs alone on its
// SM: the FP64 pipe is the bottleneck, and a CTA on the critical path (the block next in the
// chain) must not share it with CTAs that are working ahead on off-diagonal tiles. CTAs beyond
// the SM count start as earlier ones finish and draw later tickets.
static int solo_smem_bytes() {
    int dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    return per_sm / 2 + 1024;
}

gir_status dd_setup(DdState& dd, const TrsvState& st, cudaStream_t s) {
    dd.solo_smem = solo_smem_bytes();
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_trsv_dd<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dd.solo_smem));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_trsv_dd<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dd.solo_smem));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_trsv_dd<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dd.solo_smem));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_trsv_dd<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dd.solo_smem));
    count_launch(), k_diag_inv_dd<<<dd.nblk, DB, 0, s>>>(st.LU, st.ldl, st.n, st.fmt, 0, dd.DL);
    count_launch(), k_diag_inv_dd<<<dd.nblk, DB, 0, s>>>(st.LU, st.ldl, st.n, st.fmt, 1, dd.DU);
    GIR_CUDA_TRY(cudaMemsetAsync(dd.ready, 0, (size_t)dd.nblk * sizeof(int), s));
    dd.epoch = 0;
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

// ------------------------------------------------------------------ pre/post scaling
// forward: z[i] = R[p] w[p], p = perm[i] (both parts; the low part is 0 for an FP64 input)
__global__ void k_pre_dd(const double2* __restrict__ w2, const double* __restrict__ w64, const int* __restrict__ perm,
                         const double* __restrict__ R, int64_t n, double2* __restrict__ z) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = perm[i];
        double2 v = w64 ? make_double2(w64[p], 0.0) : w2[p];
        if (R) v = make_double2(R[p] * v.x, R[p] * v.y);
        z[i] = v;
    }
}
// transpose: z = S w
__global__ void k_pre_t_dd(const double2* __restrict__ w2, const double* __restrict__ w64,
                           const double* __restrict__ S, int64_t n, double2* __restrict__ z) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = w64 ? make_double2(w64[i], 0.0) : w2[i];
        if (S) v = make_double2(S[i] * v.x, S[i] * v.y);
        z[i] = v;
    }
}
// forward: out[i] = fl_u((mu S[i]) (yh + yl))
__global__ void k_post_dd(const double2* __restrict__ y, const double* __restrict__ S, double mu, int64_t n,
                          int round32, double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = y[i].x + y[i].y;
        if (S) v = (mu * S[i]) * v;
        if (round32) v = (double)__double2float_rn(v);
        out[i] = v;
    }
}
// transpose: out[perm[i]] = fl_u((mu R[perm[i]]) (yh + yl))
__global__ void k_post_t_dd(const double2* __restrict__ y, const int* __restrict__ perm, const double* __restrict__ R,
                            double mu, int64_t n, int round32, double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = perm[i];
        double v = y[i].x + y[i].y;
        if (R) v = (mu * R[p]) * v;
        if (round32) v = (double)__double2float_rn(v);
        out[p] = v;
    }
}

template <bool LOWER, bool TRANS>
static gir_status run_trsv_dd(DdState& dd, TrsvState& st, const double2* D, const double2* z, double2* y,
                              int* flags, cudaStream_t s) {
    const unsigned long long base = st.tickets;
    st.tickets += (unsigned long long)dd.nblk;
    const int epoch = ++dd.epoch;
    const int tslot = trace_begin(s, "trsv dd");
    count_launch(), k_trsv_dd<LOWER, TRANS><<<dd.nblk, DT, dd.solo_smem, s>>>(st.LU, st.ldl, st.fmt, D, st.n, dd.nblk, z, y,
                                                                   dd.ready, epoch, st.ticket_ctr, base,
                                                                   st.abort_flag, flags, SPIN_LIMIT);
    trace_end(tslot, "trsv dd", s);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

gir_status apply_minv_dd(DdState& dd, TrsvState& st, const double* w64, double* out, const double* R,
                         const double* S, double mu, int trans, int round32, int* flags, cudaStream_t s) {
    const int64_t n = st.n;
    const int g = (int)gmin<int64_t>((n + 255) / 256, 1024);
    if (!trans) {
        count_launch(), k_pre_dd<<<g, 256, 0, s>>>(dd.w, w64, st.perm, R, n, dd.z);
        GIR_TRY((run_trsv_dd<true, false>(dd, st, dd.DL, dd.z, dd.y1, flags, s)));
        GIR_TRY((run_trsv_dd<false, false>(dd, st, dd.DU, dd.y1, dd.y2, flags, s)));
        count_launch(), k_post_dd<<<g, 256, 0, s>>>(dd.y2, S, mu, n, round32, out);
    } else {
        count_launch(), k_pre_t_dd<<<g, 256, 0, s>>>(dd.w, w64, S, n, dd.z);
        // M^-T = mu R P^T L^-T U^-T S: U^T first (lower), then L^T (upper, unit)
        GIR_TRY((run_trsv_dd<true, true>(dd, st, dd.DU, dd.z, dd.y1, flags, s)));
        GIR_TRY((run_trsv_dd<false, true>(dd, st, dd.DL, dd.y1, dd.y2, flags, s)));
        count_launch(), k_post_t_dd<<<g, 256, 0, s>>>(dd.y2, st.perm, R, mu, n, round32, out);
    }
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

}  // namespace gir

// A bounded wait that runs out: one CTA of the double-double solve takes ticket 1 of a 2-block
// lower solve whose block 0 never runs, so it polls a publication flag that nothing sets. After
// spin_limit polls it raises the timeout flag and the abort flag, publishes its block and returns.
extern "C" gir_status gir_selftest_wait_timeout(long long spin_limit, void* stream) {
    using namespace gir;
    if (spin_limit < 1 || spin_limit > SPIN_LIMIT) return GIR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = 2 * DB;
    // one allocation: LU (n x n u16) | D (2 blocks) | z | y | ready | flags, abort | ticket
    const size_t off_D = (size_t)n * n * sizeof(uint16_t);
    const size_t off_z = off_D + 2 * DB * DB * sizeof(double2);
    const size_t off_y = off_z + n * sizeof(double2);
    const size_t off_r = off_y + n * sizeof(double2);
    const size_t off_t = off_r + 8 * sizeof(int);
    const size_t bytes = off_t + sizeof(unsigned long long);
    char* buf = nullptr;
    GIR_CUDA_TRY(cudaMalloc(&buf, bytes));
    gir_status st = GIR_OK;
    int hflags = 0;
    if (cudaMemsetAsync(buf, 0, bytes, s) != cudaSuccess) st = GIR_CUDA_ERROR;
    int* ready = reinterpret_cast<int*>(buf + off_r);
    int* flags = ready + 2;
    int* abort_flag = ready + 4;
    unsigned long long* ticket = reinterpret_cast<unsigned long long*>(buf + off_t);
    if (st == GIR_OK) {
        // base = -1: the single CTA draws ticket 1, i.e. block 1, which depends on block 0
        k_trsv_dd<true, false><<<1, DT, 0, s>>>(reinterpret_cast<const uint16_t*>(buf), n, FF_BF16,
                                                reinterpret_cast<const double2*>(buf + off_D), n, 2,
                                                reinterpret_cast<const double2*>(buf + off_z),
                                                reinterpret_cast<double2*>(buf + off_y), ready, 1, ticket,
                                                ~0ULL, abort_flag, flags, spin_limit);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) st = GIR_CUDA_ERROR;
    }
    if (st == GIR_OK && cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = GIR_CUDA_ERROR;
    if (cudaStreamSynchronize(s) != cudaSuccess && st == GIR_OK) st = GIR_CUDA_ERROR;
    cudaFree(buf);
    if (st != GIR_OK) return st;
    return (hflags & DEV_TIMEOUT) ? GIR_TIMEOUT : GIR_OK;
}
