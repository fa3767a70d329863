// Batches of independent systems as ONE persistent kernel launch.
//
// Every CTA (one per SM) takes systems from a device-side queue, longest first, and runs the whole
// of Algorithm 4 on each one by itself, with no host round trip: the scaling of the input, the
// u_f LU with partial pivoting (the block-column model of the factorization: w = 32 columns per
// panel, FP32 GEPP on the panel, stored L and U rounded to u_f, U12 by FP32 substitution with the
// rounded L11, FP32 trailing update with the rounded operands), x0 = M^-1 b, and the refinement
// steps, each with its residual in u_r and a GCRO-DR(m, k) correction (Algorithm 3: Arnoldi with
// CGS2 over [C V], the Givens least-squares update, the cycle end with the harmonic Ritz recycle
// space, and the carry of U_k, C_k to the next step). The stop tests, restart lengths and recycle
// ranks are decided on the device, by the CTA that owns the system; the per-system state lives in
// a workspace slot owned by the CTA. The batch's work is dominated by the streaming of A in the
// Arnoldi products, so a grid of one CTA per SM keeps HBM busy while small and large systems run
// side by side; no CTA ever waits on another.
//
// Arithmetic, per system (the same formats as the single-system path):
//  * A v of A~ in float-float from the split A = A_hi + A_lo (made once per system, after the LU,
//    in the slot memory the LU's FP32 work matrix used; the halves interleaved by groups of four
//    columns, so each row is one HBM stream);
//  * both triangular solves of M^-1 in float-float on the u_f factors, 32-row blocks (two rows per
//    warp for the off-diagonal part; the diagonal block through its float-float inverse, made once
//    per system, with one refinement step);
//  * the residual in FP64 or double-double; CGS2, norms and the small dense algebra in FP64 (the
//    Givens step, cycle end and Cholesky QR are the same device functions the single-system path
//    launches as kernels).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#define GIR_SMALL_DEVICE_ONLY
#include "k_small.cu"
#undef GIR_SMALL_DEVICE_ONLY

#include "gir_persist.cuh"
#include "trace.cuh"

namespace gir {
namespace pb {

constexpr int NT = 512;             // threads per CTA
constexpr int NW = NT / 32;         // warps per CTA
constexpr int PW = 32;              // panel width w of the block-column LU
constexpr int TM = 128;             // trailing-update tile (TM x TM outputs per CTA pass)
constexpr int DYN_BYTES = 200 * 1024;

// One system of the batch (host-filled, device-resident).
struct Sys {
    const double* A;
    const double* b;
    double* x;
    int64_t n, lda;
};

// Workspace of one CTA, sized for the largest order of the batch (nmax).
struct Slot {
    float* F;          // 2 nmax ldwmax floats: the LU's FP32 work matrix W, then A_hi and A_lo interleaved
    uint16_t* LU;      // nmax ldlmax u_f patterns: L strictly lower, U upper
    float* P;          // panel (column-major) when it does not fit in shared memory
    int* perm;
    double* R;         // FP16 scaling (powers of two)
    double* S;
    double* basis;     // [C region (KB columns) | V (m + 1 columns)], column stride n of the system
    double* Uc;        // working U (n x KB)
    double* Ct;
    double* Ut;
    double* rU;        // recycle space kept between refinement steps
    double* rC;
    double* vtmp;
    double* r;
    double* d;
    double* c;
    double* rr;
    SmallState* st;
    double* qh;        // cycle-end scratch: Qh | Pbuf | Gq
    float2* Dinv;      // float-float inverses of the 32 x 32 diagonal blocks: L blocks, then U blocks
};

struct Batch {
    const Sys* sys;
    gir_info* info;
    const int* order;  // systems by decreasing n
    int nsys;
    int* next;         // queue head
    const Slot* slots;
    gir_params p;
    int KB;            // columns reserved for C (largest recycle dimension)
    unsigned long long* prof;  // with tracing on: per CTA, NPH phase times (ns) then NPH counts
};

// Phases timed on the device clock when tracing is on (CTA time, summed over the CTAs).
enum { PH_FACTOR = 0, PH_SPLIT, PH_GEMV, PH_MINV, PH_CGS2, PH_CLOSE, PH_RESID, PH_TOTAL, PH_MINV_DIAG, NPH };

// Per-system state shared by the CTA's threads (one copy in shared memory).
struct Ctx {
    int n;
    int64_t lda, ldw, ldl;
    const double* A;
    const double* b;
    double* x;
    const float* Af;   // A_hi and A_lo interleaved (see split_matrix)
    const uint16_t* LU;
    const int* perm;
    const double* R;
    const double* S;
    double mu;
    int fmt, scaled, r32, rbasis, eig64;
    double normA, binf;
    int rc_k, rc_valid, k_run, k_open;
    unsigned long long* prof;
    Slot sl;
};

// Carve-up of the CTA's dynamic shared memory in the refinement phase (np = n rounded up to 8).
struct Smem {
    float2* ys;     // float-float y of the triangular solves (np)
    float* vh;      // float-float split of the A v input (np each)
    float* vl;
    double* close;  // cycle-end workspace (overlaps all of the above)
    int close_doubles;
};

// ------------------------------------------------------------------ block-level helpers
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Phase clock: every thread reads the start (cheap); thread 0 adds the interval after the phase's
// closing barrier.
__device__ __forceinline__ unsigned long long ph_start(const Ctx& cx) { return cx.prof ? gtimer() : 0ull; }
__device__ __forceinline__ void ph_end(const Ctx& cx, int ph, unsigned long long t0) {
    if (cx.prof && threadIdx.x == 0) {
        cx.prof[ph] += gtimer() - t0;
        cx.prof[NPH + ph] += 1;
    }
}

__device__ __forceinline__ double blk_sum(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = (l < NW) ? red[l] : 0.0;
    return warp_sum(t);   // identical in every thread (commutative butterfly)
}

__device__ __forceinline__ double blk_max(double v, double* red) {
    v = warp_max(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = (l < NW) ? red[l] : 0.0;
    return warp_max(t);
}

// max |x_i| with NaN kept visible (returns NaN if any x_i is NaN)
__device__ double blk_norminf(const double* x, int n, double* red) {
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) {
        const double a = fabs(x[i]);
        m = (a > m || a != a) ? a : m;
    }
    const int bad = __syncthreads_or(m != m);
    const double r = blk_max(m, red);
    return bad ? __longlong_as_double(0x7ff8000000000000ll) : r;
}

__device__ double blk_norm2(const double* x, int n, double* red) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) s = fma(x[i], x[i], s);
    return sqrt(blk_sum(s, red));
}

__device__ __forceinline__ void blk_copy(double* dst, const double* src, int64_t count) {
    for (int64_t i = threadIdx.x; i < count; i += NT) dst[i] = src[i];
}

__device__ __forceinline__ double rnd32(double v, int on) { return on ? (double)__double2float_rn(v) : v; }

// G[a + b ldg] = sum_i X[i + a ldx] Y[i + b ldy], a < p, b < q: a warp per (a, b)
__device__ void blk_gemm_tn(const double* X, int64_t ldx, int p, const double* Y, int64_t ldy, int q, int n,
                            double* G, int ldg) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int e = w; e < p * q; e += NW) {
        const int a = e % p, bcol = e / p;
        const double* xa = X + (int64_t)a * ldx;
        const double* yb = Y + (int64_t)bcol * ldy;
        double t = 0.0;
        for (int i = l; i < n; i += 32) t = fma(xa[i], yb[i], t);
        t = warp_sum(t);
        if (l == 0) G[a + bcol * ldg] = t;
    }
    __syncthreads();
}

// Y[:, c] = beta Y[:, c] + alpha sum_j X[:, j] Cf[j + c ldc], c < q: a thread per row
__device__ void blk_gemm_nn(const double* X, int64_t ldx, int p, const double* Cf, int ldc, int q, double* Y,
                            int64_t ldy, double alpha, double beta, int n, int round32) {
    for (int i = threadIdx.x; i < n; i += NT) {
        for (int c = 0; c < q; ++c) {
            double acc = 0.0;
            for (int j = 0; j < p; ++j) acc = fma(X[i + (int64_t)j * ldx], Cf[j + c * ldc], acc);
            double* y = Y + i + (int64_t)c * ldy;
            double v = (beta == 0.0) ? alpha * acc : fma(beta, *y, alpha * acc);
            *y = rnd32(v, round32);
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------ S1: scaling and the FP32 copy
// W = fl32(mu R A S) (R, S, mu: FP16 only), ||A||_inf in FP64; returns DEV_NONFINITE on Inf/NaN.
__device__ __noinline__ int scale_load(Ctx& cx, float* W, double* red) {
    const int n = cx.n, w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const double* A = cx.A;
    const int64_t lda = cx.lda, ldw = cx.ldw;
    int bad = 0;
    if (cx.scaled) {
        double* R = cx.sl.R;
        double* S = cx.sl.S;
        for (int i = w; i < n; i += NW) {
            double m = 0.0;
            for (int j = l; j < n; j += 32) {
                const double v = fabs(A[(int64_t)i * lda + j]);
                bad |= !(v <= 1.7976931348623157e308);
                m = fmax(m, v);
            }
            m = warp_max(m);
            if (l == 0) {
                int e;
                frexp(m, &e);
                R[i] = (m > 0.0) ? ldexp(1.0, -e) : 1.0;
            }
        }
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += NT) {
            double m = 0.0;
            for (int i = 0; i < n; ++i) m = fmax(m, fabs(A[(int64_t)i * lda + j] * R[i]));
            int e;
            frexp(m, &e);
            S[j] = (m > 0.0) ? ldexp(1.0, -e) : 1.0;
        }
        __syncthreads();
    }
    const double mu = cx.mu;
    double rowmax = 0.0;
    for (int i = w; i < n; i += NW) {
        double rs = 0.0;
        const double ri = cx.scaled ? cx.sl.R[i] : 1.0;
        for (int j = l; j < n; j += 32) {
            double v = A[(int64_t)i * lda + j];
            rs += fabs(v);
            if (cx.scaled) v *= ri * cx.sl.S[j] * mu;
            const float f = __double2float_rn(v);
            bad |= !(fabsf(f) <= 3.4028234663852886e38f);
            W[(int64_t)i * ldw + j] = f;
        }
        rs = warp_sum(rs);
        rowmax = (rs > rowmax || rs != rs) ? rs : rowmax;
    }
    bad = __syncthreads_or(bad);
    const double nA = blk_max(rowmax, red);
    if (threadIdx.x == 0) cx.normA = nA;
    __syncthreads();
    return bad ? DEV_NONFINITE : 0;
}

// ------------------------------------------------------------------ S2: the u_f LU
// (max |v|, its signed value, lowest row on ties) over the CTA; NaN entries are never chosen.
__device__ void blk_argmax(float best, float val, int idx, float* fred, float* vred, int* ired, float& ob, float& ov,
                           int& oi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float b2 = __shfl_xor_sync(0xffffffffu, best, o);
        const float v2 = __shfl_xor_sync(0xffffffffu, val, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (b2 > best || (b2 == best && i2 < idx)) { best = b2; val = v2; idx = i2; }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) { fred[w] = best; vred[w] = val; ired[w] = idx; }
    __syncthreads();
    best = (l < NW) ? fred[l] : -1.0f;
    val = (l < NW) ? vred[l] : 0.0f;
    idx = (l < NW) ? ired[l] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float b2 = __shfl_xor_sync(0xffffffffu, best, o);
        const float v2 = __shfl_xor_sync(0xffffffffu, val, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (b2 > best || (b2 == best && i2 < idx)) { best = b2; val = v2; idx = i2; }
    }
    ob = best;
    ov = val;
    oi = idx;
}

// Block-column LU of W (n x n FP32, row-major, ldw) into LU (u_f, ldl) and perm; returns 0,
// DEV_SINGULAR or DEV_NONFINITE. dyn: the CTA's dynamic shared memory.
__device__ __noinline__ int lu_factor(Ctx& cx, float* W, uint16_t* LU, int* perm, float* Pg, float* dyn) {
    const int n = cx.n, fmt = cx.fmt;
    const int64_t ldw = cx.ldw, ldl = cx.ldl;
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    __shared__ float L11[PW][PW + 1];
    __shared__ int lpiv[PW];
    __shared__ float fred[NW], vred[NW];
    __shared__ int ired[NW];
    for (int i = tid; i < n; i += NT) perm[i] = i;
    int flag = 0;
    for (int c0 = 0; c0 < n; c0 += PW) {
        const int wd = min(PW, n - c0), h = n - c0, c1 = c0 + wd;
        const int ldp = h | 1;  // odd: the column-major panel is bank-conflict free in shared memory
        float* P = ((int64_t)ldp * PW * 4 <= DYN_BYTES) ? dyn : Pg;
        for (int i = w; i < h; i += NW)
            if (l < wd) P[l * ldp + i] = W[(int64_t)(c0 + i) * ldw + c0 + l];
        __syncthreads();
        // GEPP on the panel: FP32 quotients, fused updates of the panel's later columns
        for (int k = 0; k < wd; ++k) {
            float best = -1.0f, val = 0.0f;
            int bi = 0x7fffffff;
            for (int i = k + tid; i < h; i += NT) {
                const float v = P[k * ldp + i];
                if (fabsf(v) > best) { best = fabsf(v); val = v; bi = i; }
            }
            float ob, piv;
            int p;
            blk_argmax(best, val, bi, fred, vred, ired, ob, piv, p);
            if (p == 0x7fffffff) return DEV_NONFINITE;   // the whole column is NaN
            if (piv == 0.0f) return DEV_SINGULAR;
            if (tid < wd && p != k) {
                const float t = P[tid * ldp + k];
                P[tid * ldp + k] = P[tid * ldp + p];
                P[tid * ldp + p] = t;
            }
            if (tid == 0) lpiv[k] = p;
            __syncthreads();
            for (int i = k + 1 + tid; i < h; i += NT) {
                const float lv = __fdiv_rn(P[k * ldp + i], piv);
                P[k * ldp + i] = lv;
                for (int c = k + 1; c < wd; ++c) P[c * ldp + i] = fmaf(-lv, P[c * ldp + k], P[c * ldp + i]);
            }
            __syncthreads();
        }
        if (tid == 0) {
            for (int k = 0; k < wd; ++k) {
                const int a = c0 + k, b = c0 + lpiv[k];
                const int t = perm[a];
                perm[a] = perm[b];
                perm[b] = t;
            }
        }
        // stored factors: L (below the diagonal) and U11, rounded to u_f; the rounded L11 for U12
        for (int e = tid; e < h * PW; e += NT) {
            const int i = e >> 5, c = e & 31;
            if (c >= wd) continue;
            const uint16_t q = float_to_uf(P[c * ldp + i], fmt);
            const float qf = uf_to_float(q, fmt);
            flag |= !(fabsf(qf) <= 3.4028234663852886e38f);
            LU[(int64_t)(c0 + i) * ldl + c0 + c] = q;
            if (i < PW && c < i) L11[i][c] = qf;
        }
        // the panel's interchanges on the other columns: L of earlier panels (u_f) and W right of it
        for (int j = tid; j < n - wd; j += NT) {
            const int col = (j < c0) ? j : j + wd;
            if (col < c0) {
                for (int k = 0; k < wd; ++k) {
                    const int p = lpiv[k];
                    if (p == k) continue;
                    uint16_t* a = LU + (int64_t)(c0 + k) * ldl + col;
                    uint16_t* bq = LU + (int64_t)(c0 + p) * ldl + col;
                    const uint16_t t = *a;
                    *a = *bq;
                    *bq = t;
                }
            } else {
                for (int k = 0; k < wd; ++k) {
                    const int p = lpiv[k];
                    if (p == k) continue;
                    float* a = W + (int64_t)(c0 + k) * ldw + col;
                    float* bq = W + (int64_t)(c0 + p) * ldw + col;
                    const float t = *a;
                    *a = *bq;
                    *bq = t;
                }
            }
        }
        flag = __syncthreads_or(flag);
        if (flag) return DEV_NONFINITE;
        if (c1 >= n) break;
        // U12 = L11^-1 W12 by FP32 substitution with the rounded L11, then rounded to u_f
        for (int j = c1 + tid; j < n; j += NT) {
            float xv[PW];
#pragma unroll
            for (int r = 0; r < PW; ++r) xv[r] = W[(int64_t)(c0 + r) * ldw + j];
#pragma unroll
            for (int r = 1; r < PW; ++r) {
                float t = xv[r];
#pragma unroll
                for (int q = 0; q < r; ++q) t = fmaf(-L11[r][q], xv[q], t);
                xv[r] = t;
            }
#pragma unroll
            for (int r = 0; r < PW; ++r) {
                const uint16_t q = float_to_uf(xv[r], fmt);
                flag |= !(fabsf(uf_to_float(q, fmt)) <= 3.4028234663852886e38f);
                LU[(int64_t)(c0 + r) * ldl + j] = q;
            }
        }
        flag = __syncthreads_or(flag);
        if (flag) return DEV_NONFINITE;
        // W22 -= L21 U12 with the rounded operands, FP32 fused multiply-adds in column order
        float* Ls = dyn;             // [PW][TM]: L21 tile, k-major
        float* Us = dyn + PW * TM;   // [PW][TM]: U12 tile
        const int m2 = n - c1;
        const int tiles = (m2 + TM - 1) / TM;
        const int ty = tid >> 5, tx = tid & 31;   // rows ty*8 .. +7, columns tx*4 .. +3
        for (int t = 0; t < tiles * tiles; ++t) {
            const int r0 = c1 + (t / tiles) * TM, q0 = c1 + (t % tiles) * TM;
            for (int e = tid; e < TM * PW; e += NT) {
                const int r = e >> 5, k = e & 31;
                Ls[k * TM + r] = (r0 + r < n) ? uf_to_float(LU[(int64_t)(r0 + r) * ldl + c0 + k], fmt) : 0.0f;
            }
            for (int e = tid; e < TM * PW; e += NT) {
                const int k = e / TM, q = e % TM;
                Us[k * TM + q] = (q0 + q < n) ? uf_to_float(LU[(int64_t)(c0 + k) * ldl + q0 + q], fmt) : 0.0f;
            }
            __syncthreads();
            float acc[8][4];
            const int rb = r0 + ty * 8, qb = q0 + tx * 4;
            const bool full = (qb + 3 < n);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                if (rb + r < n) {
                    const float* wp = W + (int64_t)(rb + r) * ldw + qb;
                    if (full) {
                        const float4 v = *reinterpret_cast<const float4*>(wp);
                        acc[r][0] = v.x; acc[r][1] = v.y; acc[r][2] = v.z; acc[r][3] = v.w;
                    } else {
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[r][c] = (qb + c < n) ? wp[c] : 0.0f;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0f;
                }
            }
#pragma unroll 4
            for (int k = 0; k < PW; ++k) {
                const float4 a0 = *reinterpret_cast<const float4*>(Ls + k * TM + ty * 8);
                const float4 a1 = *reinterpret_cast<const float4*>(Ls + k * TM + ty * 8 + 4);
                const float4 bv = *reinterpret_cast<const float4*>(Us + k * TM + tx * 4);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bw[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(-av[r], bw[c], acc[r][c]);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                if (rb + r >= n) continue;
                float* wp = W + (int64_t)(rb + r) * ldw + qb;
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (qb + c < n) flag |= !(fabsf(acc[r][c]) <= 3.4028234663852886e38f);
                if (full) {
                    *reinterpret_cast<float4*>(wp) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (qb + c < n) wp[c] = acc[r][c];
                }
            }
            __syncthreads();
        }
        flag = __syncthreads_or(flag);
        if (flag) return DEV_NONFINITE;
    }
    // zero padding columns [n, ldl) of the factors: the bulk copies of the solves take whole 16-byte units
    for (int64_t e = tid; e < (int64_t)n * (ldl - n); e += NT) {
        const int64_t i = e / (ldl - n), j = n + e % (ldl - n);
        LU[i * ldl + j] = 0;
    }
    __syncthreads();
    return 0;
}

// A = A_hi + A_lo (FP32 halves) into the slot's float region, row i at 2 i ldw, the halves interleaved
// by groups of four columns
__device__ __noinline__ void split_matrix(Ctx& cx) {
    const unsigned long long t0 = ph_start(cx);
    const int n = cx.n, w = threadIdx.x >> 5, l = threadIdx.x & 31;
    float* F = cx.sl.F;
    for (int i = w; i < n; i += NW) {
        const double* a = cx.A + (int64_t)i * cx.lda;
        float* row = F + (int64_t)i * 2 * cx.ldw;
        for (int j = l; j < (int)cx.ldw; j += 32) {
            const double v = (j < n) ? a[j] : 0.0;   // zero padding to whole groups of 4
            const float hv = __double2float_rn(v);
            const int g = j >> 2, k = j & 3;
            row[8 * g + k] = hv;                                   // A_hi of columns 4g .. 4g+3
            row[8 * g + 4 + k] = __double2float_rn(v - (double)hv);  // then their A_lo
        }
    }
    __syncthreads();
    ph_end(cx, PH_SPLIT, t0);
}

// ------------------------------------------------------------------ S5: A~ = M^-1 A
__device__ __forceinline__ void ff_mac4(float& sh, float& sl, float ah, float al, float vh, float vl) {
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

__device__ __forceinline__ void ff_fold4(float* sh, float* sl) {
    ff_acc_add(sh[0], sl[0], sh[1], sl[1]);
    ff_acc_add(sh[2], sl[2], sh[3], sl[3]);
    ff_acc_add(sh[0], sl[0], sh[2], sl[2]);
}

__device__ __forceinline__ void ff_warp_sum(float& sh, float& sl) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, sh, o);
        const float ol = __shfl_xor_sync(0xffffffffu, sl, o);
        const float s2 = sh + oh, bb = s2 - sh, t = (sh - (s2 - bb)) + (oh - bb);
        sh = s2;
        sl += t + ol;
    }
}

// w = A v in float-float from A_hi, A_lo (interleaved by groups of four columns, rows of 2 ldw floats with
// ldw = n rounded up to 4, zero padded; one stream per row instead of two): a warp
// takes two rows at a time, each lane keeping GV_U 16-byte loads per half and row in flight, and four
// independent float-float accumulators per row (the TwoSum chains are latency-bound, and the CTA has
// only four warps per scheduler to hide them).
constexpr int GV_U = 2;
constexpr int TR_U = 2;             // triangular solves: 16-byte loads per row in flight per lane
__device__ __noinline__ void gemv_ff(const Ctx& cx, const double* v, double* out, const Smem& sm) {
    const unsigned long long t0 = ph_start(cx);
    const int n = cx.n, w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int ldw = (int)cx.ldw, n4 = ldw >> 2;
    for (int j = threadIdx.x; j < ldw; j += NT) {
        const double x = (j < n) ? v[j] : 0.0;
        const float hv = __double2float_rn(x);
        sm.vh[j] = hv;
        sm.vl[j] = __double2float_rn(x - (double)hv);
    }
    __syncthreads();
    const float4* xh = reinterpret_cast<const float4*>(sm.vh);
    const float4* xl = reinterpret_cast<const float4*>(sm.vl);
    for (int i0 = 2 * w; i0 < n; i0 += 2 * NW) {
        const bool two = i0 + 1 < n;
        // rows interleave A_hi and A_lo by groups of four columns: float4 2j is hi, 2j+1 is lo
        const float4* ra_h = reinterpret_cast<const float4*>(cx.Af + (int64_t)i0 * 2 * ldw);
        const float4* ra_l = ra_h + 1;
        const float4* rb_h = ra_h + 2 * (ldw >> 2);
        const float4* rb_l = rb_h + 1;
        float ah[4] = {0.0f, 0.0f, 0.0f, 0.0f}, al[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        float bh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, bl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int j0 = l; j0 < n4; j0 += 32 * GV_U) {
            float4 a1[GV_U], a2[GV_U], b1[GV_U], b2[GV_U];
#pragma unroll
            for (int u = 0; u < GV_U; ++u) {
                const int j = j0 + 32 * u;
                if (j < n4) {
                    a1[u] = __ldcs(ra_h + 2 * j);
                    a2[u] = __ldcs(ra_l + 2 * j);
                    if (two) {
                        b1[u] = __ldcs(rb_h + 2 * j);
                        b2[u] = __ldcs(rb_l + 2 * j);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < GV_U; ++u) {
                const int j = j0 + 32 * u;
                if (j < n4) {
                    const float4 c = xh[j], d = xl[j];
                    ff_mac4(ah[0], al[0], a1[u].x, a2[u].x, c.x, d.x);
                    ff_mac4(ah[1], al[1], a1[u].y, a2[u].y, c.y, d.y);
                    ff_mac4(ah[2], al[2], a1[u].z, a2[u].z, c.z, d.z);
                    ff_mac4(ah[3], al[3], a1[u].w, a2[u].w, c.w, d.w);
                    if (two) {
                        ff_mac4(bh[0], bl[0], b1[u].x, b2[u].x, c.x, d.x);
                        ff_mac4(bh[1], bl[1], b1[u].y, b2[u].y, c.y, d.y);
                        ff_mac4(bh[2], bl[2], b1[u].z, b2[u].z, c.z, d.z);
                        ff_mac4(bh[3], bl[3], b1[u].w, b2[u].w, c.w, d.w);
                    }
                }
            }
        }
        ff_fold4(ah, al);
        ff_warp_sum(ah[0], al[0]);
        if (l == 0) out[i0] = (double)ah[0] + (double)al[0];
        if (two) {
            ff_fold4(bh, bl);
            ff_warp_sum(bh[0], bl[0]);
            if (l == 0) out[i0 + 1] = (double)bh[0] + (double)bl[0];
        }
    }
    __syncthreads();
    ph_end(cx, PH_GEMV, t0);
}

__device__ __forceinline__ float ufv(uint16_t v, int fmt) { return uf_to_float(v, fmt); }

// sum over the 8 u_f values packed in q of L[c + t] y[c + t] (y: 8 float-float values), into four
// independent float-float accumulators (sh[t % 4], sl[t % 4]): their TwoSum chains overlap
__device__ __forceinline__ void ff_dot8(float* sh, float* sl, uint4 q, const float2* y, int fmt) {
    const float4 y0 = *reinterpret_cast<const float4*>(y);
    const float4 y1 = *reinterpret_cast<const float4*>(y + 2);
    const float4 y2 = *reinterpret_cast<const float4*>(y + 4);
    const float4 y3 = *reinterpret_cast<const float4*>(y + 6);
    ff_acc_prod1(sh[0], sl[0], ufv((uint16_t)(q.x & 0xffffu), fmt), y0.x, y0.y);
    ff_acc_prod1(sh[1], sl[1], ufv((uint16_t)(q.x >> 16), fmt), y0.z, y0.w);
    ff_acc_prod1(sh[2], sl[2], ufv((uint16_t)(q.y & 0xffffu), fmt), y1.x, y1.y);
    ff_acc_prod1(sh[3], sl[3], ufv((uint16_t)(q.y >> 16), fmt), y1.z, y1.w);
    ff_acc_prod1(sh[0], sl[0], ufv((uint16_t)(q.z & 0xffffu), fmt), y2.x, y2.y);
    ff_acc_prod1(sh[1], sl[1], ufv((uint16_t)(q.z >> 16), fmt), y2.z, y2.w);
    ff_acc_prod1(sh[2], sl[2], ufv((uint16_t)(q.w & 0xffffu), fmt), y3.x, y3.y);
    ff_acc_prod1(sh[3], sl[3], ufv((uint16_t)(q.w >> 16), fmt), y3.z, y3.w);
}

// Float-float inverses of the diagonal blocks of L (unit lower) and U (upper) for the solves: one
// warp per block, lane j solves D x = e_j by substitution (the block staged in shared memory);
// rows and columns past n act as the identity. Stored row by row: element (r, q) of block I of
// triangle t at Dinv[((t nb + I) 32 + r) 32 + q].
__device__ __noinline__ void diag_inverses(const Ctx& cx, float* dyn) {
    const int n = cx.n, fmt = cx.fmt, w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int nb = (n + PW - 1) / PW;
    float* D = dyn + (size_t)w * PW * (PW + 1);
    for (int task = w; task < 2 * nb; task += NW) {
        const int t = task / nb, I = task % nb, r0 = I * PW, rows = min(PW, n - r0);
        for (int i = 0; i < PW; ++i) {
            float v = (i == l) ? 1.0f : 0.0f;
            if (i < rows && l < rows) v = ufv(cx.LU[(int64_t)(r0 + i) * cx.ldl + r0 + l], fmt);
            if (t == 0 && l == i) v = 1.0f;   // unit diagonal of L
            D[i * (PW + 1) + l] = v;
        }
        __syncwarp();
        float xh[PW], xl[PW];
        if (t == 0) {
#pragma unroll
            for (int i = 0; i < PW; ++i) {
                float ah = (i == l) ? 1.0f : 0.0f, al = 0.0f;
#pragma unroll
                for (int q = 0; q < i; ++q) ff_acc_prod1(ah, al, -D[i * (PW + 1) + q], xh[q], xl[q]);
                const ff y = ff_norm(ah, al);
                xh[i] = y.h;
                xl[i] = y.l;
            }
        } else {
#pragma unroll
            for (int i = PW - 1; i >= 0; --i) {
                float ah = (i == l) ? 1.0f : 0.0f, al = 0.0f;
#pragma unroll
                for (int q = i + 1; q < PW; ++q) ff_acc_prod1(ah, al, -D[i * (PW + 1) + q], xh[q], xl[q]);
                const float ud = D[i * (PW + 1) + i];
                const float yh = __fdiv_rn(ah, ud);
                const float rem = fmaf(-yh, ud, ah) + al;
                const ff y = ff_norm(yh, __fdiv_rn(rem, ud));
                xh[i] = y.h;
                xl[i] = y.l;
            }
        }
        float2* out = cx.sl.Dinv + ((size_t)t * nb + I) * PW * PW;
#pragma unroll
        for (int i = 0; i < PW; ++i) out[i * PW + l] = make_float2(xh[i], xl[i]);
        __syncwarp();
    }
    __syncthreads();
}

// out = fl_u(mu S U^-1 L^-1 P R w) in float-float, by blocks of 32 rows (L in order, then U in
// reverse order): the block's off-diagonal sums (warp w takes rows w and w + 16), then its diagonal
// block through the precomputed inverse with one refinement step.
__device__ __noinline__ void apply_minv(const Ctx& cx, const double* win, double* out, const Smem& sm) {
    __shared__ float2 accs[PW], y1s[PW], ress[PW];
    __shared__ float2 DinvS[PW * PW];   // the diagonal block's inverse, row-major
    __shared__ float Dg[PW][PW + 1];    // the diagonal block (unit diagonal for L, zero outside the triangle)
    const unsigned long long t0 = ph_start(cx);
    const int n = cx.n, fmt = cx.fmt, w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int ldl = (int)cx.ldl;
    const uint16_t* LU = cx.LU;
    float2* ys = sm.ys;
    const int nb = (n + PW - 1) / PW;
    for (int j = n + threadIdx.x; j < ldl; j += NT) ys[j] = make_float2(0.0f, 0.0f);
    __syncthreads();
    for (int t = 0; t < 2; ++t) {
        for (int bk = 0; bk < nb; ++bk) {
            const int I = (t == 0) ? bk : nb - 1 - bk;
            const int r0 = I * PW, rows = min(PW, n - r0);
            const bool ha = w < rows, hb = w + 16 < rows;
            // the diagonal block's inverse, loaded while the strip streams
            const float2* di = cx.sl.Dinv + ((size_t)t * nb + I) * PW * PW;
            const float2 dv0 = di[threadIdx.x], dv1 = di[threadIdx.x + NT];
            float ah[4] = {0.0f, 0.0f, 0.0f, 0.0f}, al[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            float bh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, bl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            // rows w and w + 16 of the strip; off-diagonal columns [0, r0) of L, [r0 + 32, ldl) of U
            // (both multiples of 8 apart), 8 per lane at a time with TR_U 16-byte loads per row in flight
            const uint16_t* rowa = LU + (int64_t)(r0 + w) * ldl;
            const uint16_t* rowb = LU + (int64_t)(r0 + w + 16) * ldl;
            const int c_lo = (t == 0) ? 0 : min(r0 + PW, ldl), c_hi = (t == 0) ? r0 : ldl;
            if (ha) {
                for (int c0 = c_lo + l * 8; c0 < c_hi; c0 += 256 * TR_U) {
                    uint4 qa[TR_U], qb[TR_U];
#pragma unroll
                    for (int u = 0; u < TR_U; ++u) {
                        const int c = c0 + 256 * u;
                        if (c < c_hi) {
                            qa[u] = __ldg(reinterpret_cast<const uint4*>(rowa + c));
                            if (hb) qb[u] = __ldg(reinterpret_cast<const uint4*>(rowb + c));
                        }
                    }
#pragma unroll
                    for (int u = 0; u < TR_U; ++u) {
                        const int c = c0 + 256 * u;
                        if (c < c_hi) {
                            ff_dot8(ah, al, qa[u], ys + c, fmt);
                            if (hb) ff_dot8(bh, bl, qb[u], ys + c, fmt);
                        }
                    }
                }
            }
            // the diagonal block, masked to its triangle; rows past n are identity rows
            {
                const int ra = w, rb = w + 16;
                const bool in_a = (t == 0) ? (l < ra) : (l >= ra), in_b = (t == 0) ? (l < rb) : (l >= rb);
                Dg[ra][l] = (ha && l < rows) ? (in_a ? ufv(rowa[r0 + l], fmt) : (l == ra ? 1.0f : 0.0f))
                                             : (l == ra ? 1.0f : 0.0f);
                Dg[rb][l] = (hb && l < rows) ? (in_b ? ufv(rowb[r0 + l], fmt) : (l == rb ? 1.0f : 0.0f))
                                             : (l == rb ? 1.0f : 0.0f);
            }
            const unsigned long long td = ph_start(cx);
            DinvS[threadIdx.x] = dv0;
            DinvS[threadIdx.x + NT] = dv1;
            if (ha) {
                ff_fold4(ah, al);
                ff_fold4(bh, bl);
                ff_warp_sum(ah[0], al[0]);
                ff_warp_sum(bh[0], bl[0]);
                if (l == 0) {
                    const int ra = r0 + w, rb = r0 + w + 16;
                    ff a, bq;
                    if (t == 0) {
                        const int pa = cx.perm[ra];
                        a = ff_from_double(cx.scaled ? cx.R[pa] * win[pa] : win[pa]);
                        if (hb) {
                            const int pb = cx.perm[rb];
                            bq = ff_from_double(cx.scaled ? cx.R[pb] * win[pb] : win[pb]);
                        }
                    } else {
                        a = ff{ys[ra].x, ys[ra].y};
                        if (hb) bq = ff{ys[rb].x, ys[rb].y};
                    }
                    ff_acc_add(a.h, a.l, -ah[0], -al[0]);
                    accs[w] = make_float2(a.h, a.l);
                    if (hb) {
                        ff_acc_add(bq.h, bq.l, -bh[0], -bl[0]);
                        accs[w + 16] = make_float2(bq.h, bq.l);
                    } else {
                        accs[w + 16] = make_float2(0.0f, 0.0f);
                    }
                }
            } else if (l == 0) {
                accs[w] = make_float2(0.0f, 0.0f);
                accs[w + 16] = make_float2(0.0f, 0.0f);
            }
            __syncthreads();
            // diagonal block: y1 = Dinv acc, then one refinement step y = y1 + Dinv (acc - D y1), which
            // brings the explicit inverse to the accuracy of a substitution. Warp w takes rows w and
            // w + 16, lane q the products with column q, the warp sums (float-float).
            {
                const int ra = w, rb = w + 16;
                const float2 aq = accs[l];
                const float2 ia = DinvS[ra * PW + l], ib = DinvS[rb * PW + l];
                float pa = ia.x * aq.x, ea = fmaf(ia.x, aq.x, -pa);
                ea = fmaf(ia.x, aq.y, fmaf(ia.y, aq.x, ea));
                float pb = ib.x * aq.x, eb = fmaf(ib.x, aq.x, -pb);
                eb = fmaf(ib.x, aq.y, fmaf(ib.y, aq.x, eb));
                ff_warp_sum(pa, ea);
                ff_warp_sum(pb, eb);
                const ff ya = ff_norm(pa, ea), yb = ff_norm(pb, eb);
                if (l == 0) {
                    y1s[ra] = make_float2(ya.h, ya.l);
                    y1s[rb] = make_float2(yb.h, yb.l);
                }
                __syncthreads();
                // residual acc - D y1: lane q forms -D[r][q] y1[q]; lane 0 adds acc[r]
                const float2 yq = y1s[l];
                float ha_ = 0.0f, la_ = 0.0f, hb_ = 0.0f, lb_ = 0.0f;
                ff_acc_prod1(ha_, la_, -Dg[ra][l], yq.x, yq.y);
                ff_acc_prod1(hb_, lb_, -Dg[rb][l], yq.x, yq.y);
                if (l == 0) {
                    ff_acc_add(ha_, la_, accs[ra].x, accs[ra].y);
                    ff_acc_add(hb_, lb_, accs[rb].x, accs[rb].y);
                }
                ff_warp_sum(ha_, la_);
                ff_warp_sum(hb_, lb_);
                if (l == 0) {
                    const ff ra_ = ff_norm(ha_, la_), rb_ = ff_norm(hb_, lb_);
                    ress[ra] = make_float2(ra_.h, ra_.l);
                    ress[rb] = make_float2(rb_.h, rb_.l);
                }
                __syncthreads();
                const float2 rq = ress[l];
                float qa = ia.x * rq.x, fa = fmaf(ia.x, rq.x, -qa);
                fa = fmaf(ia.x, rq.y, fmaf(ia.y, rq.x, fa));
                float qb = ib.x * rq.x, fb = fmaf(ib.x, rq.x, -qb);
                fb = fmaf(ib.x, rq.y, fmaf(ib.y, rq.x, fb));
                if (l == 0) {
                    ff_acc_add(qa, fa, ya.h, ya.l);
                    ff_acc_add(qb, fb, yb.h, yb.l);
                }
                ff_warp_sum(qa, fa);
                ff_warp_sum(qb, fb);
                if (l == 0) {
                    const ff za = ff_norm(qa, fa), zb = ff_norm(qb, fb);
                    if (ra < rows) ys[r0 + ra] = make_float2(za.h, za.l);
                    if (rb < rows) ys[r0 + rb] = make_float2(zb.h, zb.l);
                }
            }
            __syncthreads();
            ph_end(cx, PH_MINV_DIAG, td);
        }
    }
    for (int i = threadIdx.x; i < n; i += NT) {
        double v = (double)ys[i].x + (double)ys[i].y;
        if (cx.scaled) v *= cx.S[i] * cx.mu;
        out[i] = rnd32(v, cx.r32);
    }
    __syncthreads();
    ph_end(cx, PH_MINV, t0);
}

// ------------------------------------------------------------------ S4: residual in u_r
// rr = b - A x in FP64 (dd = 0) or double-double (dd = 1), stored in u
__device__ __noinline__ void residual(const Ctx& cx, int dd, double* rr) {
    const unsigned long long t0 = ph_start(cx);
    const int n = cx.n, w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int i = w; i < n; i += NW) {
        const double* row = cx.A + (int64_t)i * cx.lda;
        double sh = 0.0, sl = 0.0;
        if (!dd) {
            for (int j = l; j < n; j += 32) sh = fma(row[j], cx.x[j], sh);
            sh = warp_sum(sh);
            if (l == 0) rr[i] = rnd32(cx.b[i] - sh, cx.r32);
        } else {
            for (int j = l; j < n; j += 32) {
                const double a = row[j], v = cx.x[j];
                const double p = a * v, e = fma(a, v, -p);
                const double s = sh + p, bb = s - sh, t = (sh - (s - bb)) + (p - bb);
                sh = s;
                sl += t + e;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double oh = __shfl_xor_sync(0xffffffffu, sh, o);
                const double ol = __shfl_xor_sync(0xffffffffu, sl, o);
                const double s = sh + oh, bb = s - sh;
                double t = (sh - (s - bb)) + (oh - bb);
                t += sl + ol;
                sh = s + t;
                sl = t - (sh - s);
            }
            if (l == 0) {
                const double bi = cx.b[i];
                const double s = bi - sh, bb = s - bi;
                double t = (bi - (s - bb)) + (-sh - bb);
                t -= sl;
                rr[i] = rnd32(s + t, cx.r32);
            }
        }
    }
    __syncthreads();
    ph_end(cx, PH_RESID, t0);
}

// ------------------------------------------------------------------ S6-S11: GCRO-DR
__device__ __forceinline__ double* Vcol(const Ctx& cx, const Batch& B, int j) {
    return cx.sl.basis + (int64_t)(B.KB + j) * cx.n;
}
__device__ __forceinline__ double* Creg(const Ctx& cx, const Batch& B, int kc) {
    return cx.sl.basis + (int64_t)(B.KB - kc) * cx.n;
}

__device__ void apply_atilde(const Ctx& cx, const double* v, double* out, const Smem& sm) {
    gemv_ff(cx, v, cx.sl.vtmp, sm);
    apply_minv(cx, cx.sl.vtmp, out, sm);
}

// One Arnoldi step j over [C V] with CGS2 (two projection passes), the norm, the Givens update
// and the normalisation of v_{j+1}.
__device__ __noinline__ void arnoldi_step(const Ctx& cx, const Batch& B, int j, int kc, const Smem& sm, double* red) {
    const int n = cx.n;
    SmallState* st = cx.sl.st;
    double* w = Vcol(cx, B, j + 1);
    apply_atilde(cx, Vcol(cx, B, j), w, sm);
    const unsigned long long t0 = ph_start(cx);
    const double* basis = Creg(cx, B, kc);
    const int p = kc + j + 1;
    blk_gemm_tn(basis, n, p, w, n, 1, n, st->s1, p);
    blk_gemm_nn(basis, n, p, st->s1, p, 1, w, n, -1.0, 1.0, n, cx.r32);
    blk_gemm_tn(basis, n, p, w, n, 1, n, st->s2, p);
    blk_gemm_nn(basis, n, p, st->s2, p, 1, w, n, -1.0, 1.0, n, cx.r32);
    const double hn = blk_norm2(w, n, red);
    if (threadIdx.x == 0) {
        st->hnorm = hn;
        givens_step_dev(st);
    }
    __syncthreads();
    const double f = (hn != 0.0) ? 1.0 / hn : 0.0;
    for (int i = threadIdx.x; i < n; i += NT) w[i] = rnd32(w[i] * f, cx.rbasis);
    __syncthreads();
    ph_end(cx, PH_CGS2, t0);
}

// Arnoldi steps of one cycle from v_1 = r / beta until convergence or `steps`; returns the steps taken.
__device__ __noinline__ int run_cycle(const Ctx& cx, const Batch& B, int kc, int first, double beta, double tol, int steps,
                         const Smem& sm, double* red) {
    const int n = cx.n;
    SmallState* st = cx.sl.st;
    double* v0 = Vcol(cx, B, 0);
    const double f = (beta != 0.0) ? 1.0 / beta : 0.0;
    for (int i = threadIdx.x; i < n; i += NT) v0[i] = rnd32(cx.sl.r[i] * f, cx.rbasis);
    if (threadIdx.x == 0) {
        st->eig64 = cx.eig64;
        st->j = 0;
        st->kc = kc;
        st->converged = 0;
        st->breakdown = 0;
        st->knew = 0;
        st->first = first;
        st->k_target = cx.k_run;
        st->m = B.p.m;
        st->beta = beta;
        st->tol = tol;
        st->est = beta;
        st->g[0] = beta;
    }
    __syncthreads();
    int j = 0;
    for (; j < steps; ++j) {
        arnoldi_step(cx, B, j, kc, sm, red);
        if (st->status) break;
        if (st->converged) { ++j; break; }
    }
    __syncthreads();
    return j;
}

__device__ __noinline__ void cycle_close(const Ctx& cx, const Smem& sm) {
    SmallState* st = cx.sl.st;
    double* Qh = cx.sl.qh;
    double* Pbuf = Qh + SM_DMAX * SM_DMAX;
    double* Gq = Pbuf + SM_DMAX * (SM_KMAX + 2);
    const unsigned long long t0 = ph_start(cx);
    if (threadIdx.x < CLOSE_THREADS) cycle_close_dev(st, Qh, Pbuf, Gq, sm.close, sm.close_doubles);
    __syncthreads();
    ph_end(cx, PH_CLOSE, t0);
}

// GCRO-DR(m, k) for A~ d = c from d = 0 (Algorithm 3), with the recycle space of the previous
// refinement step (Ctx rc_k, rc_valid; slot rU, rC). Returns a DEV_* mask (0 = no error).
__device__ __noinline__ int gcrodr(Ctx& cx, const Batch& B, const Smem& sm, double* red, int* its_out, int* capp_out,
                      int* cycles, int* conv_out) {
    const int n = cx.n, m = B.p.m;
    const Slot& sl = cx.sl;
    SmallState* st = sl.st;
    int k = cx.k_run;
    const int max_its = B.p.max_its > 0 ? B.p.max_its : 20 * m;
    const int r32 = cx.r32, rb = cx.rbasis;
    int its = 0;
    *capp_out = 0;
    const double normc = blk_norm2(sl.c, n, red);
    const double tol = B.p.tau * normc;
    for (int i = threadIdx.x; i < n; i += NT) sl.d[i] = 0.0;
    __syncthreads();
    if (normc == 0.0) {
        *its_out = 0;
        *conv_out = 1;
        return 0;
    }
    blk_copy(sl.r, sl.c, n);
    __syncthreads();
    int kc = (k > 0) ? cx.rc_k : 0;
    if (kc > 0) {
        blk_copy(sl.Uc, sl.rU, (int64_t)kc * n);
        if (B.p.carry_mode == 1 && cx.rc_valid) {
            blk_copy(Creg(cx, B, kc), sl.rC, (int64_t)kc * n);
            __syncthreads();
        } else {
            __syncthreads();
            // Z = A~ Y (Y = previous U_k), QR(Z) by Cholesky QR twice: C = Q, U = Y R^-1
            for (int i = 0; i < kc; ++i) apply_atilde(cx, sl.Uc + (int64_t)i * n, sl.Ct + (int64_t)i * n, sm);
            *capp_out = kc;
            blk_gemm_tn(sl.Ct, n, kc, sl.Ct, n, kc, n, st->G2, kc);
            if (threadIdx.x == 0) chol_gram_dev(st, kc, 0);
            __syncthreads();
            blk_gemm_nn(sl.Ct, n, kc, st->Ccoef, SM_LDG, kc, sl.Ut, n, 1.0, 0.0, n, 0);
            blk_gemm_tn(sl.Ut, n, kc, sl.Ut, n, kc, n, st->G2, kc);
            if (threadIdx.x == 0) chol_gram_dev(st, kc, 1);
            __syncthreads();
            if (st->knew == kc) {
                blk_gemm_nn(sl.Ut, n, kc, st->Ccoef, SM_LDG, kc, Creg(cx, B, kc), n, 1.0, 0.0, n, rb);
                blk_gemm_nn(sl.Uc, n, kc, st->Rinv, SM_KMAX, kc, sl.Ut, n, 1.0, 0.0, n, rb);
                blk_copy(sl.Uc, sl.Ut, (int64_t)kc * n);
                __syncthreads();
            } else {
                kc = 0;  // the Gram matrix lost definiteness: start again with a GMRES cycle
            }
        }
        if (kc > 0) {
            // d = U C^T r ; r = r - C C^T r
            blk_gemm_tn(Creg(cx, B, kc), n, kc, sl.r, n, 1, n, st->s1, kc);
            blk_gemm_nn(sl.Uc, n, kc, st->s1, kc, 1, sl.d, n, 1.0, 0.0, n, r32);
            blk_gemm_nn(Creg(cx, B, kc), n, kc, st->s1, kc, 1, sl.r, n, -1.0, 1.0, n, r32);
        }
    }
    int ncyc = 0;
    if (kc == 0) {
        // first cycle: GMRES(m) from v1 = r / ||r||, then the harmonic Ritz recycle space
        const double nr = blk_norm2(sl.r, n, red);
        const int j = run_cycle(cx, B, 0, 1, nr, tol, min(m, max_its), sm, red);
        its += j;
        ++ncyc;
        if (st->status) return st->status;
        if (cx.k_open) {
            // Section 5: k = its_1 - 1 when the first GMRES cycle converged
            __syncthreads();
            if (threadIdx.x == 0) {
                cx.k_open = 0;
                if (st->converged && j >= 1) {
                    cx.k_run = min(j - 1, SM_KMAX);
                    st->k_target = cx.k_run;
                }
            }
            __syncthreads();
            k = cx.k_run;
        }
        cycle_close(cx, sm);
        blk_gemm_nn(Vcol(cx, B, 0), n, j, st->ycoef, j, 1, sl.d, n, 1.0, 0.0, n, r32);
        blk_gemm_nn(Vcol(cx, B, 0), n, j + 1, st->zcoef, j + 1, 1, sl.r, n, 1.0, 0.0, n, r32);
        const int knew = st->knew;
        if (knew > 0) {
            blk_gemm_nn(Vcol(cx, B, 0), n, j + 1, st->Ccoef, SM_LDG, knew, Creg(cx, B, knew), n, 1.0, 0.0, n, rb);
            blk_gemm_nn(Vcol(cx, B, 0), n, j, st->Ucoef, SM_LDG, knew, sl.Uc, n, 1.0, 0.0, n, rb);
        }
        kc = knew;
    }
    double rn = blk_norm2(sl.r, n, red);
    while (rn > tol && its < max_its) {
        if (!(rn == rn)) return DEV_NONFINITE;
        const int steps = max(1, min(m - kc, max_its - its));
        const int j = run_cycle(cx, B, kc, 0, rn, tol, steps, sm, red);
        its += j;
        ++ncyc;
        if (st->status) return st->status;
        if (kc > 0) {
            blk_gemm_tn(Creg(cx, B, kc), n, kc + j + 1, sl.Uc, n, kc, n, st->WtU, SM_LDG);
            blk_gemm_tn(sl.Uc, n, kc, sl.Uc, n, kc, n, st->UtU, kc);
        }
        cycle_close(cx, sm);
        const int d_dim = kc + j;
        // d += [U V_j] ycoef ; r -= [C V_{j+1}] zcoef
        if (kc > 0) blk_gemm_nn(sl.Uc, n, kc, st->ycoef, d_dim, 1, sl.d, n, 1.0, 1.0, n, 0);
        blk_gemm_nn(Vcol(cx, B, 0), n, j, st->ycoef + kc, d_dim, 1, sl.d, n, 1.0, 1.0, n, r32);
        blk_gemm_nn(Creg(cx, B, kc), n, kc + j + 1, st->zcoef, d_dim + 1, 1, sl.r, n, -1.0, 1.0, n, r32);
        const int knew = (k > 0) ? st->knew : 0;
        if (knew > 0) {
            blk_gemm_nn(Creg(cx, B, kc), n, kc + j + 1, st->Ccoef, SM_LDG, knew, sl.Ct, n, 1.0, 0.0, n, rb);
            blk_gemm_nn(Vcol(cx, B, 0), n, j, st->Ucoef + kc, SM_LDG, knew, sl.Ut, n, 1.0, 0.0, n, 0);
            if (kc > 0) blk_gemm_nn(sl.Uc, n, kc, st->Ucoef, SM_LDG, knew, sl.Ut, n, 1.0, 1.0, n, 0);
            if (rb) {
                for (int64_t i = threadIdx.x; i < (int64_t)knew * n; i += NT) sl.Ut[i] = rnd32(sl.Ut[i], 1);
                __syncthreads();
            }
            blk_copy(Creg(cx, B, knew), sl.Ct, (int64_t)knew * n);
            blk_copy(sl.Uc, sl.Ut, (int64_t)knew * n);
            __syncthreads();
        }
        kc = knew;
        rn = blk_norm2(sl.r, n, red);
    }
    // keep the recycle space for the next refinement step (Algorithm 3 ends with Y~ = U_k)
    const int rk = (k > 0) ? kc : 0;
    if (rk > 0) {
        blk_copy(sl.rU, sl.Uc, (int64_t)rk * n);
        blk_copy(sl.rC, Creg(cx, B, rk), (int64_t)rk * n);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cx.rc_k = rk;
        cx.rc_valid = rk > 0;
    }
    __syncthreads();
    *its_out = its;
    *cycles += ncyc;
    *conv_out = (rn <= tol);
    if (!(rn == rn)) return DEV_NONFINITE;
    return 0;
}

__device__ gir_status dev_status(int f) {
    if (f & DEV_TIMEOUT) return GIR_TIMEOUT;
    if (f & DEV_NONFINITE) return GIR_NONFINITE;
    if (f & DEV_SINGULAR) return GIR_SINGULAR;
    return GIR_OK;
}

// Algorithm 4 on one system, by the whole CTA.
__device__ void solve_one(const Batch& B, const Slot& sl, int sidx, unsigned char* dyn, Ctx& cx, double* red) {
    const Sys sy = B.sys[sidx];
    gir_info* info = B.info + sidx;
    const int n = (int)sy.n;
    const unsigned long long t0 = gtimer();
    if (threadIdx.x == 0) {
        cx.n = n;
        cx.lda = sy.lda;
        cx.ldw = ((int64_t)n + 3) & ~(int64_t)3;
        cx.ldl = ((int64_t)n + 7) & ~(int64_t)7;
        cx.A = sy.A;
        cx.b = sy.b;
        cx.x = sy.x;
        cx.Af = sl.F;
        cx.LU = sl.LU;
        cx.perm = sl.perm;
        cx.R = sl.R;
        cx.S = sl.S;
        cx.fmt = (B.p.uf == GIR_FP16) ? FF_FP16 : FF_BF16;
        cx.scaled = (B.p.uf == GIR_FP16);
        cx.mu = cx.scaled ? exp2(floor(log2(0.1 * 65504.0 / sqrt((double)n)))) : 1.0;
        cx.r32 = (B.p.u == GIR_FP32);
        cx.rbasis = cx.r32 || (B.p.flags & GIR_FLAG_BASIS_FP32) != 0;
        cx.eig64 = (B.p.flags & GIR_FLAG_EIG_FP64) ? 1 : 0;
        cx.rc_k = 0;
        cx.rc_valid = 0;
        cx.k_run = B.p.k;
        cx.k_open = (B.p.flags & GIR_FLAG_ADAPTIVE_K) != 0;
        cx.prof = B.prof ? B.prof + (size_t)blockIdx.x * 2 * NPH : nullptr;
        cx.sl = sl;
        info->status = GIR_NOT_CONVERGED;
        for (int i = 0; i <= GIR_MAX_IR; ++i) info->cw_berr[i] = -1.0;
        info->final_cw_berr = -1.0;
    }
    // a fresh small state (status, counters) for this system
    for (int i = threadIdx.x; i < (int)(sizeof(SmallState) / 4); i += NT) reinterpret_cast<int*>(sl.st)[i] = 0;
    __syncthreads();
    Smem sm;
    const int np = (n + 7) & ~7;
    sm.ys = reinterpret_cast<float2*>(dyn);
    sm.vh = reinterpret_cast<float*>(dyn + (size_t)8 * np);
    sm.vl = sm.vh + np;
    sm.close = reinterpret_cast<double*>(dyn);
    sm.close_doubles = DYN_BYTES / 8;

    // S1 + S2: scaling, FP32 copy, LU
    int f = scale_load(cx, sl.F, red);
    if (!f) f = lu_factor(cx, sl.F, sl.LU, sl.perm, sl.P, reinterpret_cast<float*>(dyn));
    __syncthreads();
    const unsigned long long t1 = gtimer();
    ph_end(cx, PH_FACTOR, t0);
    if (f) {
        if (threadIdx.x == 0) {
            info->status = dev_status(f);
            info->ms_factor = (float)((t1 - t0) * 1e-6);
        }
        __syncthreads();
        return;
    }
    split_matrix(cx);
    diag_inverses(cx, reinterpret_cast<float*>(dyn));
    const double binf = blk_norminf(cx.b, n, red);
    // x0 = M^-1 b (Algorithm 4, initial solve), stored in u
    apply_minv(cx, cx.b, cx.x, sm);
    const double u = (B.p.u == GIR_FP32) ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
    const double target = (B.p.target_berr < 0.0) ? 2.0 * u : B.p.target_berr;
    gir_status status = GIR_NOT_CONVERGED;
    int ir_steps = 0, total = 0, cycles = 0;
    const int dd = (B.p.ur == GIR_DD);
    for (int i = 0; i <= B.p.imax; ++i) {
        // r_i = b - A x_i in u_r, stored in u
        residual(cx, dd, sl.rr);
        const double rinf = blk_norminf(sl.rr, n, red);
        const double xinf = blk_norminf(cx.x, n, red);
        const double eta = rinf / (cx.normA * xinf + binf);
        if (threadIdx.x == 0) {
            info->berr[i] = eta;
            info->final_berr = eta;
        }
        if (!(eta == eta) || !(xinf <= 1.7976931348623157e308)) { status = GIR_NONFINITE; break; }
        if (eta <= target) { status = GIR_OK; break; }
        if (i == B.p.imax) break;
        // r^ = fl_u(r / ||r||_inf) ; c = M^-1 r^
        const double fs = (rinf != 0.0) ? 1.0 / rinf : 0.0;
        for (int q = threadIdx.x; q < n; q += NT) sl.rr[q] = rnd32(sl.rr[q] * fs, cx.r32);
        __syncthreads();
        apply_minv(cx, sl.rr, sl.c, sm);
        int its = 0, capp = 0, conv = 0;
        const int e = gcrodr(cx, B, sm, red, &its, &capp, &cycles, &conv);
        if (e) { status = dev_status(e); break; }
        if (threadIdx.x == 0) {
            info->its[i] = its;
            info->carry_applies[i] = capp;
        }
        total += its;
        ir_steps = i + 1;
        // x_{i+1} = fl_u(x_i + ||r_i||_inf d)
        for (int q = threadIdx.x; q < n; q += NT) cx.x[q] = rnd32(fma(rinf, sl.d[q], cx.x[q]), cx.r32);
        __syncthreads();
    }
    const unsigned long long t2 = gtimer();
    __syncthreads();
    if (threadIdx.x == 0) {
        info->status = status;
        info->ir_steps = ir_steps;
        info->total_its = total;
        info->cycles = cycles;
        info->k_eff = cx.rc_k;
        info->ms_factor = (float)((t1 - t0) * 1e-6);
        info->ms_solve = (float)((t2 - t1) * 1e-6);
    }
    ph_end(cx, PH_TOTAL, t0);
    __syncthreads();
}

__global__ void __launch_bounds__(NT, 1) k_batch_persistent(const Batch B) {
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ Ctx cx;
    __shared__ double red[NW];
    __shared__ int s_q;
    const Slot sl = B.slots[blockIdx.x];
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(B.next, 1);
        __syncthreads();
        const int q = s_q;
        __syncthreads();
        if (q >= B.nsys) break;
        solve_one(B, sl, B.order[q], dyn, cx, red);
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace pb

bool persistent_batch_supported(int nsys, const int64_t* n, const int64_t* lda, const gir_params* p) {
    if (nsys < 1 || !p) return false;
    if (p->flags & (GIR_FLAG_BATCH_STREAMS | GIR_FLAG_CW_BERR | GIR_FLAG_SIR)) return false;
    if (p->uf != GIR_BF16 && p->uf != GIR_FP16) return false;
    if (p->ua != GIR_FP64) return false;
    if (p->m > PERSIST_MAX_M) return false;
    for (int i = 0; i < nsys; ++i)
        if (n[i] < 1 || n[i] > PERSIST_NMAX || lda[i] < n[i]) return false;
    return true;
}

bool persistent_batch_preferred(int nsys, const int64_t* n) {
    // one CTA per system against the whole GPU per system (gir.h states the model and its constants)
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
        cudaGetLastError();
        nsm = 152;
    }
    double t1max = 0.0, t1sum = 0.0, tstreams = 0.0;
    for (int i = 0; i < nsys; ++i) {
        const double m = (double)n[i];
        const double t1 = 8.7e-9 * m * m * m + 1.8e-5 * m * m;
        t1max = t1 > t1max ? t1 : t1max;
        t1sum += t1;
        tstreams += 2.1 + 4.0e-7 * m * m;
    }
    const double tpers = t1max > t1sum / nsm ? t1max : t1sum / nsm;
    return tpers <= tstreams;
}

gir_status persistent_batch_solve(int nsys, const int64_t* n, const double* const* A, const int64_t* lda,
                                  const double* const* b, double* const* x, const gir_params* p, gir_info* infos,
                                  cudaStream_t s) {
    using namespace pb;
    if (p->m < 1 || p->m > PERSIST_MAX_M || p->k < 0 || p->k >= p->m || p->k > GIR_MAX_K || p->imax < 0 ||
        p->imax >= GIR_MAX_IR || !(p->tau >= 0.0) || (p->carry_mode != 0 && p->carry_mode != 1) ||
        (p->u != GIR_FP64 && p->u != GIR_FP32) || (p->ur != GIR_FP64 && p->ur != GIR_DD) ||
        (p->flags & ~(GIR_FLAG_AUTOTUNE | GIR_FLAG_ADAPTIVE_K | GIR_FLAG_EIG_FP64 | GIR_FLAG_BASIS_FP32 |
                      GIR_FLAG_BATCH_PERSISTENT)) != 0)
        return GIR_INVALID_ARG;
    for (int i = 0; i < nsys; ++i)
        if (!A[i] || !b[i] || !x[i]) return GIR_INVALID_ARG;
    int dev = 0;
    GIR_CUDA_TRY(cudaGetDevice(&dev));
    int nsm = 0;
    GIR_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    static std::atomic<unsigned> attr_done{0};
    GIR_CUDA_TRY(ensure_dyn_smem((const void*)k_batch_persistent, DYN_BYTES, attr_done));
    int occ = 0;
    GIR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_persistent, NT, DYN_BYTES));
    if (occ < 1) return GIR_UNSUPPORTED;
    const int64_t nmax = *std::max_element(n, n + nsys);
    // C columns: k, plus one where the conjugate-pair rule of the harmonic Ritz selection takes a
    // whole pair at the k-th place (the selection caps the total at SM_KMAX)
    const int KB = (p->flags & GIR_FLAG_ADAPTIVE_K) ? SM_KMAX : std::max(1, std::min(p->k + 1, SM_KMAX));
    const int m = p->m;
    const int64_t ldw = (nmax + 3) & ~3, ldl = (nmax + 7) & ~7;
    // per-slot workspace
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    const size_t oF = take(sizeof(float) * 2 * nmax * ldw);
    const size_t oLU = take(sizeof(uint16_t) * nmax * ldl);
    const size_t oP = take(sizeof(float) * PW * (nmax + 1));
    const size_t oDinv = take(sizeof(float2) * 2 * ((nmax + PW - 1) / PW) * PW * PW);
    const size_t oPerm = take(sizeof(int) * nmax);
    const size_t oR = take(sizeof(double) * nmax), oS = take(sizeof(double) * nmax);
    const size_t oBasis = take(sizeof(double) * nmax * (KB + m + 1));
    const size_t oUc = take(sizeof(double) * nmax * KB), oCt = take(sizeof(double) * nmax * KB),
                 oUt = take(sizeof(double) * nmax * KB), orU = take(sizeof(double) * nmax * KB),
                 orC = take(sizeof(double) * nmax * KB);
    size_t ov[5];
    for (int i = 0; i < 5; ++i) ov[i] = take(sizeof(double) * nmax);
    const size_t oSt = take(sizeof(SmallState));
    const size_t oQh = take(sizeof(double) * (SM_DMAX * SM_DMAX + SM_DMAX * (SM_KMAX + 2) + (SM_DMAX + 1) * (SM_KMAX + 2)));
    const size_t slot_bytes = off;
    size_t free_b = 0, total_b = 0;
    GIR_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    int nslots = std::min(nsm * occ, nsys);
    const size_t budget = free_b / 10 * 8;
    if ((size_t)nslots * slot_bytes > budget) nslots = (int)std::max<size_t>(1, budget / slot_bytes);
    // descriptors
    std::vector<Sys> hsys(nsys);
    for (int i = 0; i < nsys; ++i) hsys[i] = Sys{A[i], b[i], x[i], n[i], lda[i]};
    std::vector<int> order(nsys);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return n[a] > n[c]; });
    const size_t oSys = 0;
    size_t doff = align256(sizeof(Sys) * nsys);
    const size_t oInfo = doff;
    doff += align256(sizeof(gir_info) * nsys);
    const size_t oOrder = doff;
    doff += align256(sizeof(int) * nsys);
    const size_t oNext = doff;
    doff += 256;
    const size_t oSlots = doff;
    doff += align256(sizeof(Slot) * nslots);
    const bool prof = trace_on();
    const size_t oProf = doff;
    if (prof) doff += align256(sizeof(unsigned long long) * 2 * NPH * nslots);
    const size_t oWork = doff;
    const size_t total = doff + slot_bytes * nslots;
    unsigned char* base = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&base, total, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return (e == cudaErrorMemoryAllocation) ? GIR_OOM : GIR_CUDA_ERROR;
    }
    std::vector<Slot> hsl(nslots);
    for (int c = 0; c < nslots; ++c) {
        unsigned char* w = base + oWork + slot_bytes * c;
        Slot& q = hsl[c];
        q.F = reinterpret_cast<float*>(w + oF);
        q.LU = reinterpret_cast<uint16_t*>(w + oLU);
        q.P = reinterpret_cast<float*>(w + oP);
        q.Dinv = reinterpret_cast<float2*>(w + oDinv);
        q.perm = reinterpret_cast<int*>(w + oPerm);
        q.R = reinterpret_cast<double*>(w + oR);
        q.S = reinterpret_cast<double*>(w + oS);
        q.basis = reinterpret_cast<double*>(w + oBasis);
        q.Uc = reinterpret_cast<double*>(w + oUc);
        q.Ct = reinterpret_cast<double*>(w + oCt);
        q.Ut = reinterpret_cast<double*>(w + oUt);
        q.rU = reinterpret_cast<double*>(w + orU);
        q.rC = reinterpret_cast<double*>(w + orC);
        q.vtmp = reinterpret_cast<double*>(w + ov[0]);
        q.r = reinterpret_cast<double*>(w + ov[1]);
        q.d = reinterpret_cast<double*>(w + ov[2]);
        q.c = reinterpret_cast<double*>(w + ov[3]);
        q.rr = reinterpret_cast<double*>(w + ov[4]);
        q.st = reinterpret_cast<SmallState*>(w + oSt);
        q.qh = reinterpret_cast<double*>(w + oQh);
    }
    gir_status st = GIR_OK;
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    do {
        if (cudaMemcpyAsync(base + oSys, hsys.data(), sizeof(Sys) * nsys, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(base + oOrder, order.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(base + oSlots, hsl.data(), sizeof(Slot) * nslots, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(base + oInfo, 0, sizeof(gir_info) * nsys, s) != cudaSuccess ||
            (prof && cudaMemsetAsync(base + oProf, 0, sizeof(unsigned long long) * 2 * NPH * nslots, s) != cudaSuccess)) {
            st = GIR_CUDA_ERROR;
            break;
        }
        Batch Bt;
        Bt.sys = reinterpret_cast<const Sys*>(base + oSys);
        Bt.info = reinterpret_cast<gir_info*>(base + oInfo);
        Bt.order = reinterpret_cast<const int*>(base + oOrder);
        Bt.nsys = nsys;
        Bt.next = reinterpret_cast<int*>(base + oNext);
        Bt.slots = reinterpret_cast<const Slot*>(base + oSlots);
        Bt.p = *p;
        Bt.KB = KB;
        Bt.prof = prof ? reinterpret_cast<unsigned long long*>(base + oProf) : nullptr;
        // the queue reset and the persistent launch, captured once into a graph and launched from it
        // on the caller's stream (captured on a private stream: the legacy stream cannot capture)
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            st = GIR_CUDA_ERROR;
            break;
        }
        cudaMemsetAsync(Bt.next, 0, sizeof(int), cs);
        count_launch(), k_batch_persistent<<<nslots, NT, DYN_BYTES, cs>>>(Bt);
        if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || !graph ||
            cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess || cudaGraphLaunch(exec, s) != cudaSuccess) {
            st = GIR_CUDA_ERROR;
            break;
        }
        std::vector<gir_info> hinfo(nsys);
        if (cudaMemcpyAsync(hinfo.data(), base + oInfo, sizeof(gir_info) * nsys, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = GIR_CUDA_ERROR;
            break;
        }
        if (prof) {
            std::vector<unsigned long long> hp((size_t)2 * NPH * nslots);
            if (cudaMemcpy(hp.data(), base + oProf, hp.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost) ==
                cudaSuccess) {
                static const char* names[NPH] = {"batch: scale + LU", "batch: split A", "batch: A v",
                                                 "batch: M^-1",       "batch: CGS2 + Givens", "batch: cycle end",
                                                 "batch: residual",   "batch: whole system",
                                                 "batch: M^-1, diagonal blocks"};
                for (int ph = 0; ph < NPH; ++ph) {
                    double ns = 0.0;
                    long long cnt = 0;
                    for (int c = 0; c < nslots; ++c) {
                        ns += (double)hp[(size_t)c * 2 * NPH + ph];
                        cnt += (long long)hp[(size_t)c * 2 * NPH + NPH + ph];
                    }
                    trace_add(names[ph], ns * 1e-6, cnt);
                }
            }
        }
        gir_status worst = GIR_OK;
        for (int i = 0; i < nsys; ++i) {
            if (infos) infos[i] = hinfo[i];
            if (hinfo[i].status != GIR_OK && (worst == GIR_OK || hinfo[i].status > worst)) worst = hinfo[i].status;
        }
        st = worst;
    } while (0);
    cudaGetLastError();
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    cudaFreeAsync(base, s);
    return st;
}

}  // namespace gir
