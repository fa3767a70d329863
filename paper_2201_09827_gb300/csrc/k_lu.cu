// Precision-u_f LU with partial pivoting (Algorithm 4, the factorization step) for GB300.
//
// Numerical model (block fused multiply-add): the Schur complement W is FP32; a panel of
// width w is factored by GEPP in FP32 arithmetic; the stored factors are the u_f-rounded
// panel values; U12 = L11^-1 W12 by FP32 substitution with the rounded L11 and is rounded
// to u_f; the trailing update takes the u_f operands with FP32 accumulation.
//
// Structure: outer blocks of NB columns (trailing update with K = NB, the tensor-core GEMM);
// inside an outer block, panels of w columns are factored by one thread-block cluster each
// (the whole panel lives in the cluster's distributed shared memory; one cluster barrier
// per column carries the pivot search), followed by the in-block TRSM/GEMM updates.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "gir_internal.cuh"
#include "k_lu.cuh"
#include "trace.cuh"

namespace gir {

// ------------------------------------------------------------------ input scaling (S1)
// Row maxima of |A| -> R_i = 2^-E (|A| row max = f 2^E, f in [0.5, 1)).
__global__ void __launch_bounds__(256) k_row_scale(const double* __restrict__ A, int64_t n, int64_t lda,
                                                   double* __restrict__ R, int* flags) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * 8;
    for (int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); i < n; i += warps_total) {
        double m = 0.0;
        bool bad = false;
        const double* a = A + i * lda;
        int64_t j0 = 0;
        if (((lda & 1) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0)) {
            // 16-byte loads, four per lane in flight (the maximum does not depend on the order)
            const int64_t n2 = n >> 1;
#pragma unroll 4
            for (int64_t j = lane; j < n2; j += 32) {
                const double2 v = __ldcs(reinterpret_cast<const double2*>(a) + j);
                const double x = fabs(v.x), y = fabs(v.y);
                bad |= !(x <= 1.7976931348623157e308) || !(y <= 1.7976931348623157e308);
                m = fmax(m, fmax(x, y));
            }
            j0 = 2 * n2;
        }
        for (int64_t j = j0 + lane; j < n; j += 32) {
            double v = fabs(a[j]);
            bad |= !(v <= 1.7976931348623157e308);
            m = fmax(m, v);
        }
        m = warp_max(m);
        bad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
            int e;
            frexp(m, &e);
            R[i] = (m > 0.0) ? ldexp(1.0, -e) : 1.0;
            if (bad) atomicOr(flags, DEV_NONFINITE);
        }
    }
}

// Column maxima of |R A| (atomicMax on the bit pattern of non-negative doubles).
__global__ void __launch_bounds__(256) k_col_absmax(const double* __restrict__ A, int64_t n, int64_t lda,
                                                    const double* __restrict__ R, unsigned long long* colmax) {
    const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * 256;
    const int64_t i1 = min(n, i0 + 256);
    if (j >= n) return;
    double m = 0.0;
#pragma unroll 8
    for (int64_t i = i0; i < i1; ++i) m = fmax(m, fabs(A[i * lda + j] * R[i]));
    atomicMax(colmax + j, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_col_scale(const unsigned long long* __restrict__ colmax, int64_t n, double* __restrict__ S) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double m = __longlong_as_double((long long)colmax[j]);
        int e;
        frexp(m, &e);
        S[j] = (m > 0.0) ? ldexp(1.0, -e) : 1.0;
    }
}

// W = fl32(mu R A S) (R, S may be null = identity).
__global__ void __launch_bounds__(256) k_quantize(const double* __restrict__ A, int64_t n, int64_t lda,
                                                  const double* __restrict__ R, const double* __restrict__ S,
                                                  double mu, float* __restrict__ W, int64_t ldw, int* flags) {
    // rows in a grid-stride loop, columns by the CTA's threads (two per thread with 16-byte loads
    // where both row pitches and base addresses allow)
    bool bad = false;
    const bool vec = ((lda & 1) == 0) && ((ldw & 1) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(W) & 7) == 0);
    const bool vec4 = vec && ((ldw & 3) == 0) && ((reinterpret_cast<uintptr_t>(W) & 15) == 0);
    auto cvt = [&](double v, int64_t i, int64_t j) {
        if (R) v *= R[i] * S[j] * mu;
        const float f = __double2float_rn(v);
        bad |= !(fabsf(f) <= 3.4028234663852886e38f);
        return f;
    };
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const double* a = A + i * lda;
        float* w = W + i * ldw;
        if (vec4) {
            // four columns per thread: two 16-byte loads, one 16-byte store, two groups in flight
            const int64_t n4 = n >> 2;
#pragma unroll 2
            for (int64_t q = threadIdx.x; q < n4; q += blockDim.x) {
                const int64_t j = 4 * q;
                const double2 v0 = __ldcs(reinterpret_cast<const double2*>(a + j));
                const double2 v1 = __ldcs(reinterpret_cast<const double2*>(a + j + 2));
                *reinterpret_cast<float4*>(w + j) =
                    make_float4(cvt(v0.x, i, j), cvt(v0.y, i, j + 1), cvt(v1.x, i, j + 2), cvt(v1.y, i, j + 3));
            }
            for (int64_t j = 4 * n4 + threadIdx.x; j < n; j += blockDim.x) w[j] = cvt(a[j], i, j);
        } else if (vec) {
            for (int64_t j = 2 * (int64_t)threadIdx.x; j + 1 < n; j += 2 * (int64_t)blockDim.x) {
                const double2 v = *reinterpret_cast<const double2*>(a + j);
                *reinterpret_cast<float2*>(w + j) = make_float2(cvt(v.x, i, j), cvt(v.y, i, j + 1));
            }
            if ((n & 1) && threadIdx.x == 0) w[n - 1] = cvt(a[n - 1], i, n - 1);
        } else {
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x) w[j] = cvt(a[j], i, j);
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, DEV_NONFINITE);
}

// ------------------------------------------------------------------ cluster panel GEPP
// One cluster of C CTAs factors the panel W[r0:n, c0:c0+WC) in place (r0 == c0). CTA q of
// the cluster holds panel rows [q*rpc, (q+1)*rpc) in shared memory. Per column: local
// argmax -> candidate (value, row, row values) written into every CTA's receive slot
// through distributed shared memory -> one cluster barrier -> every thread picks the same
// winner (largest |value|, lowest row on ties) -> swap and rank-1 update of own rows.
// Receive slots are double-buffered by column parity, so one barrier per column suffices.

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_nctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t map_shared(const void* p, uint32_t rank) {
    uint32_t local = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
    return remote;
}
__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_s32(uint32_t addr, int v) {
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

constexpr long long PANEL_WAIT_LIMIT = 4000000LL;   // polls of one column's message barrier
__device__ __forceinline__ void pn_mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void pn_mbar_expect(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(bar)),
                 "r"(bytes)
                 : "memory");
}
// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool pn_mbar_wait(unsigned long long* bar, uint32_t parity) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    for (long long it = 0; it < PANEL_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void pn_st_async_v4(uint32_t addr, float a, float b, float c, float d, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(addr),
                 "f"(a), "f"(b), "f"(c), "f"(d), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void pn_st_async_v2(uint32_t addr, uint32_t a, uint32_t b, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b32 [%0], {%1, %2}, [%3];" ::"r"(addr),
                 "r"(a), "r"(b), "r"(bar)
                 : "memory");
}

constexpr int PANEL_THREADS = 512;
constexpr int PANEL_MAXC = 16;

template <int WC>
struct PanelShared {
    unsigned long long bar[2];                       // message barriers of the two slot buffers
    __align__(16) float cand_rowv[2][PANEL_MAXC][WC];  // [buf][sender]: candidate row values
    __align__(16) float rowj[2][WC];                 // [buf]: row j before the interchange
    __align__(16) uint2 cand_vr[2][PANEL_MAXC];      // [buf][sender]: (|value| bits, row)
    float wbest_val[2][PANEL_THREADS / 32];
    int wbest_row[2][PANEL_THREADS / 32];
    int piv[WC];                      // panel-relative pivot row of each column
    float top[WC][WC + 1];            // final rows 0..wcols-1 of the panel (L11 below the diagonal)
    __align__(16) float ubT[WC][8];   // U rows of the current 8-column mini-panel, column-major
    float l11[WC][WC + 1];            // L11 rounded to u_f (strictly lower part), for the U12 solve
    int ext_row[32];                  // distinct pivot rows below the panel's diagonal block
    int mv_dst[64], mv_src[64];       // net row moves of the panel's interchanges
    int mv_count;
};

// Work the panel kernel does once its columns are factored: store the u_f copy of the panel into
// LU, apply the panel's row interchanges to other columns of W (FP32) and LU (u_f), and solve
// for the U12 rows of the W columns.
struct PanelTail {
    uint16_t* LU;          // null: no u_f store and no LU interchanges
    int64_t ldl;
    int fmt;
    int64_t wcol0, wcol1;  // W columns [wcol0, wcol1) receive the interchanges (and the U12 solve)
    int64_t lcol0, lcol1;  // LU columns [lcol0, lcol1) receive them
    uint16_t* UT;          // U12 transposed (u12_mode 1): UT[col * ldut + i]
    int64_t ldut;
    int64_t w2col0, w2col1;  // further W columns receiving the interchanges only
    int u12_mode;          // 0: none; 1: U12 = fl_uf(L11^-1 W[panel rows, wcol0:wcol1]) by FP32
                           // substitution with the rounded L11, into LU, W and UT; 2: the same in
                           // FP32 with the unrounded L11, into W only (FP8 blocks, rounded later)
};

__device__ __forceinline__ void argmax_merge(float& v, int& r, float ov, int orow) {
    if (ov > v || (ov == v && orow < r)) { v = ov; r = orow; }
}

// Warp-wide argmax of (value, row): the largest value, the lowest row among equal values.
// Values are magnitudes (>= 0), so their bit patterns order like the values; an invalid
// candidate (value < 0) enters as (0, 0x7fffffff) and loses against every valid one.
__device__ __forceinline__ void warp_argmax(float& v, int& row) {
    const bool ok = v >= 0.0f;
    const unsigned vb = ok ? __float_as_uint(v) : 0u;
    const unsigned rb = ok ? (unsigned)row : 0x7fffffffu;
    const unsigned mv = __reduce_max_sync(0xffffffffu, vb);
    const unsigned mr = __reduce_min_sync(0xffffffffu, vb == mv ? rb : 0xffffffffu);
    v = __uint_as_float(mv);
    row = (int)mr;
}

// x / p rounded to nearest, with rp = RN(1/p): Markstein's correction step (q0 = RN(x rp),
// e = x - q0 p exact by FMA, q = RN(q0 + e rp)) gives the correctly rounded quotient when both
// operands are normal and well inside the exponent range; elsewhere the library division.
__device__ __forceinline__ bool div_safe(float v) {
    const uint32_t e = (__float_as_uint(v) >> 23) & 0xffu;
    return e >= 127u - 96u && e <= 127u + 96u;
}
// Rank-1 update of one mini-panel chunk [CB, CB + 8) of two rows (columns > j), returning the
// updated entries of column j + 1; CB is a compile-time start so that only this chunk's code is
// issued (the caller switches on the warp-uniform j / 8).
template <int CB>
__device__ __forceinline__ void chunk_update(float* rowA, float* rowB, const float* pc, float lA, float lB, bool upA,
                                             bool upB, int j, float& nvA, float& nvB) {
#pragma unroll
    for (int c = CB; c < CB + 8; ++c) {
        if (c > j) {
            const float tA = fmaf(-lA, pc[c], rowA[c]);
            const float tB = fmaf(-lB, pc[c], rowB[c]);
            if (upA) rowA[c] = tA;
            if (upB) rowB[c] = tB;
            if (c == j + 1) { nvA = tA; nvB = tB; }
        }
    }
}

__device__ __noinline__ float div_slow(float x, float p) { return __fdiv_rn(x, p); }

// Rank-8 update of one row's columns [CS, WC) by the mini-panel ending at column CS - 1 (its
// multipliers l, its U rows ubT column-major), in step order; returns the new entry of column CS.
template <int CS, int WC>
__device__ __forceinline__ float block_update(float* row, const float (*ubT)[8], const float* l) {
    float nv = 0.0f;
#pragma unroll
    for (int c = CS; c < WC; ++c) {
        const float4 u0 = *reinterpret_cast<const float4*>(&ubT[c][0]);
        const float4 u1 = *reinterpret_cast<const float4*>(&ubT[c][4]);
        float x = row[c];
        x = fmaf(-l[0], u0.x, x);
        x = fmaf(-l[1], u0.y, x);
        x = fmaf(-l[2], u0.z, x);
        x = fmaf(-l[3], u0.w, x);
        x = fmaf(-l[4], u1.x, x);
        x = fmaf(-l[5], u1.y, x);
        x = fmaf(-l[6], u1.z, x);
        x = fmaf(-l[7], u1.w, x);
        row[c] = x;
        if (c == CS) nv = x;
    }
    return nv;
}

__device__ __forceinline__ float div_rn(float x, float p, float rp, bool p_safe) {
    if (x == 0.0f) return __int_as_float((__float_as_int(x) ^ __float_as_int(p)) & (int)0x80000000);
    if (p_safe && div_safe(x)) {
        const float q0 = x * rp;
        const float e = fmaf(-q0, p, x);
        return fmaf(e, rp, q0);
    }
    return __fdiv_rn(x, p);
}

// Work of a panel launch once its columns are factored (sh.top, sh.piv final): the net row moves
// of the panel's interchanges applied to the other columns of W (FP32) and LU (u_f), and the U12
// rows of the block's later W columns (tail.u12_mode). Every CTA of the cluster takes a share.
template <int WC>
__device__ __forceinline__ void panel_tail_work(PanelShared<WC>& sh, float* __restrict__ W, int64_t ldw, int64_t r0,
                                                int wcols, const PanelTail& tail, int C, int rank, int tid,
                                                int lane, int warp) {
    const int64_t ncw = tail.wcol1 - tail.wcol0;
    const int64_t ncw2 = tail.w2col1 - tail.w2col0;
    const int64_t ncl = tail.LU ? tail.lcol1 - tail.lcol0 : 0;
    if (ncw <= 0 && ncw2 <= 0 && ncl <= 0) return;
    // net effect of the interchanges ipiv[r0 .. r0+wcols) as row moves (dst <- src): replay them
    // on slot contents held in one warp's registers (slots 0..31 panel rows, 32.. the distinct
    // pivot rows below the diagonal block, numbered by first use)
    if (warp == 0) {
        const unsigned FULL = 0xffffffffu;
        const int p = (lane < wcols) ? sh.piv[lane] : lane;
        const bool ext = lane < wcols && p >= wcols;
        const unsigned key = ext ? (unsigned)p : (0x80000000u | (unsigned)lane);
        const unsigned same = __match_any_sync(FULL, key);
        const int first = __ffs(same) - 1;
        const unsigned leaders = __ballot_sync(FULL, ext && first == lane);
        const int nlead = __popc(leaders);
        const int slot = ext ? 32 + __popc(leaders & ((1u << first) - 1u)) : p;
        if (ext && first == lane) sh.ext_row[__popc(leaders & ((1u << lane) - 1u))] = p;
        __syncwarp();
        const int rowB = (lane < nlead) ? sh.ext_row[lane] : -1;
        int cA = lane, cB = rowB;
        for (int k = 0; k < wcols; ++k) {
            const int b = __shfl_sync(FULL, slot, k);
            const int va = __shfl_sync(FULL, cA, k);
            const int vbA = __shfl_sync(FULL, cA, b & 31);
            const int vbB = __shfl_sync(FULL, cB, b & 31);
            const int vb = (b < 32) ? vbA : vbB;
            if (lane == k) cA = vb;
            if (b < 32) {
                if (lane == b) cA = va;
            } else if (lane == b - 32) {
                cB = va;
            }
        }
        const bool mA = lane < wcols && cA != lane;
        const bool mB = lane < nlead && cB != rowB;
        const unsigned bA = __ballot_sync(FULL, mA), bB = __ballot_sync(FULL, mB);
        const unsigned lt = (1u << lane) - 1u;
        if (mA) { int i = __popc(bA & lt); sh.mv_dst[i] = lane; sh.mv_src[i] = cA; }
        if (mB) { int i = __popc(bA) + __popc(bB & lt); sh.mv_dst[i] = rowB; sh.mv_src[i] = cB; }
        if (lane == 0) sh.mv_count = __popc(bA) + __popc(bB);
    }
    __syncthreads();
    const int cnt = sh.mv_count;
    const bool trsm = tail.u12_mode != 0;
    if (cnt == 0 && !trsm) return;
    // column chunks (32 FP32 columns of W, 64 u_f columns of LU) spread over the cluster's CTAs;
    // every source of a chunk is read before any destination is written
    const int nchw = (int)((gmax<int64_t>(ncw, 0) + 31) / 32);
    const int nchw2 = (int)((gmax<int64_t>(ncw2, 0) + 31) / 32);
    const int nchl = (int)((gmax<int64_t>(ncl, 0) + 63) / 64);
    if (cnt > 0) {
        for (int ch = rank; ch < nchw + nchw2 + nchl; ch += C) {
            if (ch < nchw + nchw2) {
                const bool second = ch >= nchw;
                const int64_t cbase = second ? tail.w2col0 + (int64_t)(ch - nchw) * 32 : tail.wcol0 + (int64_t)ch * 32;
                const int64_t cend = second ? tail.w2col1 : tail.wcol1;
                float v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int e = tid + k * PANEL_THREADS, m = e >> 5;
                    const int64_t col = cbase + (e & 31);
                    if (m < cnt && col < cend) v[k] = W[(r0 + sh.mv_src[m]) * ldw + col];
                }
                __syncthreads();
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int e = tid + k * PANEL_THREADS, m = e >> 5;
                    const int64_t col = cbase + (e & 31);
                    if (m < cnt && col < cend) W[(r0 + sh.mv_dst[m]) * ldw + col] = v[k];
                }
            } else {
                const int64_t cbase = tail.lcol0 + (int64_t)(ch - nchw - nchw2) * 64;
                uint16_t v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int e = tid + k * PANEL_THREADS, m = e >> 6;
                    const int64_t col = cbase + (e & 63);
                    if (m < cnt && col < tail.lcol1) v[k] = tail.LU[(r0 + sh.mv_src[m]) * tail.ldl + col];
                }
                __syncthreads();
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int e = tid + k * PANEL_THREADS, m = e >> 6;
                    const int64_t col = cbase + (e & 63);
                    if (m < cnt && col < tail.lcol1) tail.LU[(r0 + sh.mv_dst[m]) * tail.ldl + col] = v[k];
                }
            }
            __syncthreads();
        }
    }
    if (trsm && rank < nchw) {
        // U12 rows of this CTA's W chunks, one thread per column: forward substitution with the
        // u_f multipliers, then rounding to u_f (stored in LU, W and UT); in mode 2 the FP32
        // multipliers and no rounding (W only)
        const bool rnd = tail.u12_mode == 1;
        for (int e = tid; e < WC * WC; e += PANEL_THREADS) {
            const int i = e / WC, q = e - (e / WC) * WC;
            const float t = sh.top[i][q];
            sh.l11[i][q] = (q < i) ? (rnd ? uf_to_float(float_to_uf(t, tail.fmt), tail.fmt) : t) : 0.0f;
        }
        __syncthreads();
        const int myw = (nchw - rank + C - 1) / C;
        for (int t = tid; t < myw * 32; t += PANEL_THREADS) {
            const int64_t col = tail.wcol0 + (int64_t)(rank + (t >> 5) * C) * 32 + (t & 31);
            if (col >= tail.wcol1) continue;
            float x[WC];
#pragma unroll
            for (int i = 0; i < WC; ++i) x[i] = (i < wcols) ? W[(r0 + i) * ldw + col] : 0.0f;
#pragma unroll
            for (int i = 1; i < WC; ++i) {
                float acc = x[i];
#pragma unroll
                for (int q = 0; q < WC; ++q)
                    if (q < i) acc = fmaf(-sh.l11[i][q], x[q], acc);
                x[i] = acc;
            }
#pragma unroll
            for (int i = 0; i < WC; ++i) {
                if (i < wcols) {
                    if (rnd) {
                        const uint16_t u = float_to_uf(x[i], tail.fmt);
                        tail.LU[(r0 + i) * tail.ldl + col] = u;
                        W[(r0 + i) * ldw + col] = uf_to_float(u, tail.fmt);
                        tail.UT[col * tail.ldut + i] = u;
                    } else {
                        W[(r0 + i) * ldw + col] = x[i];
                    }
                }
            }
        }
    }
}

// GEPP of one FP32 panel (rows r0..n-1, wcols <= WC columns) by a cluster of C CTAs, each holding
// rpc consecutive rows in shared memory. Per column: thread-owned rows give local candidates
// (computed while the previous column's update ran) and one CTA barrier merges them. Every CTA
// then sends its candidate (value, row, row values) and, if it owns row j, row j to every CTA's
// slot with st.async, which counts the bytes on the receiver's mbarrier; each CTA waits only
// for its own barrier (no cluster-wide barrier per column). Every warp then picks the global
// pivot (largest |value|, lowest row on ties) and updates its rows with correctly rounded FP32
// quotients and fused updates: the FP32 Schur complement of the block-FMA model (Section 3).
// Slots are double-buffered by column parity: a CTA sends column j + 1 only after it has read
// everything of column j - 1's slot, so no sender can overwrite a slot still being read.
template <int WC>
__global__ void __launch_bounds__(PANEL_THREADS, 1)
k_panel(float* __restrict__ W, int64_t ldw, int64_t r0, int64_t n, int wcols, int rpc, int* __restrict__ ipiv,
        int* __restrict__ flags, PanelTail tail) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PanelShared<WC>& sh = *reinterpret_cast<PanelShared<WC>*>(smem_raw);
    // rows padded to WC + 1 floats so that a warp reading one column of 32 rows hits 32 banks
    constexpr int TS = WC + 1;
    constexpr int NW = PANEL_THREADS / 32;
    constexpr int NONE = 0x7fffffff;
    float* tile = reinterpret_cast<float*>(smem_raw + sizeof(PanelShared<WC>));  // [rpc][TS]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int C = (int)cluster_nctarank();
    const int rank = C > 1 ? (int)cluster_ctarank() : 0;
    const int64_t h = n - r0;
    const int g0 = rank * rpc;                              // first panel row of this CTA
    const int myrows = (int)gmax<int64_t>(0, gmin<int64_t>(rpc, h - g0));

    for (int e = tid; e < myrows * WC; e += PANEL_THREADS) {
        int lr = e / WC, c = e - lr * WC;
        tile[lr * TS + c] = (c < wcols) ? W[(r0 + g0 + lr) * ldw + r0 + c] : 0.0f;
    }
    __syncthreads();
    int local_flag = 0;
    float bv = -1.0f;
    int bi = NONE;
    for (int lr = tid; lr < myrows; lr += PANEL_THREADS) {
        float v = fabsf(tile[lr * TS]);
        if (v != v) { local_flag |= DEV_NONFINITE; v = -1.0f; }
        argmax_merge(bv, bi, v, g0 + lr);
    }
    if (tid == 0) {
        pn_mbar_init(&sh.bar[0], 1);
        pn_mbar_init(&sh.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    cluster_barrier();   // every CTA's barriers exist before the first remote message
    const uint32_t col_bytes = (uint32_t)(C * (8 + 4 * WC) + 4 * WC);
    bool dead = false;   // a message wait timed out: skip later waits, flag, finish the launch

    for (int j = 0; j < wcols; ++j) {
        const int buf = j & 1;
        if (tid == 0) pn_mbar_expect(&sh.bar[buf], col_bytes);
        warp_argmax(bv, bi);
        if (lane == 0) { sh.wbest_val[buf][warp] = bv; sh.wbest_row[buf][warp] = bi; }
        __syncthreads();
        // this CTA's candidate, merged redundantly by every warp
        float cv = (lane < NW) ? sh.wbest_val[buf][lane] : -1.0f;
        int cr = (lane < NW) ? sh.wbest_row[buf][lane] : NONE;
        warp_argmax(cv, cr);
        {
            // lane l of warp q sends to CTA q: l < WC/4 a 16-byte chunk of the candidate row,
            // l == WC/4 the (value, row) pair, the next WC/4 lanes row j (its owner only)
            constexpr int NCH = WC / 4;
            const int q = warp, l = lane;
            if (q < C && l <= 2 * NCH) {
                const uint32_t rbar = map_shared(&sh.bar[buf], q);
                if (l < NCH) {
                    const float* src = (cr != NONE) ? tile + (cr - g0) * TS + 4 * l : nullptr;
                    pn_st_async_v4(map_shared(&sh.cand_rowv[buf][rank][4 * l], q), src ? src[0] : 0.0f,
                                   src ? src[1] : 0.0f, src ? src[2] : 0.0f, src ? src[3] : 0.0f, rbar);
                } else if (l == NCH) {
                    pn_st_async_v2(map_shared(&sh.cand_vr[buf][rank], q), __float_as_uint(cv), (uint32_t)cr, rbar);
                } else if (j >= g0 && j < g0 + myrows) {
                    const int k = l - NCH - 1;
                    const float* src = tile + (j - g0) * TS + 4 * k;
                    pn_st_async_v4(map_shared(&sh.rowj[buf][4 * k], q), src[0], src[1], src[2], src[3], rbar);
                }
            }
        }
        // the senders have read their tile rows before any thread updates a row (a thread's own
        // message wait does not cover this CTA's sends to the other CTAs)
        __syncthreads();
        if (!dead && !pn_mbar_wait(&sh.bar[buf], (uint32_t)((j >> 1) & 1))) {
            dead = true;
            local_flag |= DEV_TIMEOUT;
        }
        // global pivot, merged redundantly by every warp
        float pv = -1.0f;
        int pr = NONE;
        if (lane < C) {
            const uint2 vr = sh.cand_vr[buf][lane];
            pv = __uint_as_float(vr.x);
            pr = (int)vr.y;
        }
        const unsigned own = (lane < C) ? __float_as_uint(pv) : 0xffffffffu;
        const int own_row = pr;
        warp_argmax(pv, pr);
        int pq = __ffs(__ballot_sync(0xffffffffu, own == __float_as_uint(pv) && own_row == pr)) - 1;
        if (pr == NONE || pr < j || (int64_t)pr >= h) {
            // no finite candidate in the column (all NaN), or (after a timed-out wait) no valid
            // message: keep the row order, flag, divide by nothing
            local_flag |= (pr == NONE) ? DEV_NONFINITE : DEV_TIMEOUT;
            pr = j;
            pv = 0.0f;
            pq = 0;
        }
        if (pq < 0 || pq >= C) pq = 0;
        const float* prow = sh.cand_rowv[buf][pq];
        const float* rj = sh.rowj[buf];
        const float piv = prow[j];
        if (tid < WC) sh.top[j][tid] = prow[tid];   // row j of the panel is final from here on
        if (tid == 0) {
            sh.piv[j] = pr;
            if (rank == 0) ipiv[r0 + j] = (int)(r0 + pr);
            if (pv == 0.0f) local_flag |= DEV_SINGULAR;
        }
        float pc[WC];
#pragma unroll
        for (int k = 0; k < WC / 4; ++k) {
            const float4 v = reinterpret_cast<const float4*>(prow)[k];
            pc[4 * k] = v.x;
            pc[4 * k + 1] = v.y;
            pc[4 * k + 2] = v.z;
            pc[4 * k + 3] = v.w;
        }
        // columns are processed in mini-panels of 8: a pivot step updates only the rest of its
        // mini-panel; the later columns get the mini-panel's rank-8 update after its last step
        // (same FP32 operations in the same order as rank-1 updates, far less shared-memory traffic)
        const bool next = j + 1 < wcols && (j & 7) != 7;
        const float rp = (piv != 0.0f) ? __frcp_rn(piv) : 0.0f;
        const bool p_safe = div_safe(piv);
        bv = -1.0f;
        bi = NONE;
        // rows in pairs (lr, lr + PANEL_THREADS): the two rows' quotient and update chains are
        // independent and interleave
        for (int lr0 = tid; lr0 < myrows; lr0 += 2 * PANEL_THREADS) {
            const int lr1 = lr0 + PANEL_THREADS;
            const bool has1 = lr1 < myrows;
            float* rowA = tile + lr0 * TS;
            float* rowB = tile + (has1 ? lr1 : lr0) * TS;
            const int gA = g0 + lr0, gB = g0 + lr1;
            if (gA == j) {
#pragma unroll
                for (int c = 0; c < WC; ++c) rowA[c] = pc[c];
            } else if (gA == pr) {
#pragma unroll
                for (int c = 0; c < WC; ++c) rowA[c] = rj[c];
            }
            if (has1) {
                if (gB == j) {
#pragma unroll
                    for (int c = 0; c < WC; ++c) rowB[c] = pc[c];
                } else if (gB == pr) {
#pragma unroll
                    for (int c = 0; c < WC; ++c) rowB[c] = rj[c];
                }
            }
            const bool upA = gA > j, upB = has1 && gB > j;
            if (!upA && !upB) continue;
            // quotients: Markstein's correction of x RN(1/p) where it is exact, else the library
            const float xA = rowA[j], xB = rowB[j];
            float lA = 0.0f, lB = 0.0f;
            if (piv != 0.0f) {
                const float qA = xA * rp, qB = xB * rp;
                lA = fmaf(fmaf(-qA, piv, xA), rp, qA);
                lB = fmaf(fmaf(-qB, piv, xB), rp, qB);
                const bool okA = p_safe && (div_safe(xA) || xA == 0.0f);
                const bool okB = p_safe && (div_safe(xB) || xB == 0.0f);
                if (xA == 0.0f) lA = __int_as_float((__float_as_int(xA) ^ __float_as_int(piv)) & (int)0x80000000);
                if (xB == 0.0f) lB = __int_as_float((__float_as_int(xB) ^ __float_as_int(piv)) & (int)0x80000000);
                // rare (operands near the exponent limits): an out-of-line call, so a real branch
                if (!okA) lA = div_slow(xA, piv);
                if (!okB) lB = div_slow(xB, piv);
            }
            if (!upA) lA = 0.0f;
            if (!upB) lB = 0.0f;
            if (upA) rowA[j] = lA;
            if (upB) rowB[j] = lB;
            float nvA = 0.0f, nvB = 0.0f;   // the updated entries of column j + 1
            switch (j >> 3) {
                case 0: chunk_update<0>(rowA, rowB, pc, lA, lB, upA, upB, j, nvA, nvB); break;
                case 1: chunk_update<8>(rowA, rowB, pc, lA, lB, upA, upB, j, nvA, nvB); break;
                case 2: if (WC > 16) chunk_update<16 % WC>(rowA, rowB, pc, lA, lB, upA, upB, j, nvA, nvB); break;
                default: if (WC > 16) chunk_update<24 % WC>(rowA, rowB, pc, lA, lB, upA, upB, j, nvA, nvB); break;
            }
            if (next) {
                if (upA) {
                    float v = fabsf(nvA);
                    if (v != v) { local_flag |= DEV_NONFINITE; v = -1.0f; }
                    argmax_merge(bv, bi, v, gA);
                }
                if (upB) {
                    float v = fabsf(nvB);
                    if (v != v) { local_flag |= DEV_NONFINITE; v = -1.0f; }
                    argmax_merge(bv, bi, v, gB);
                }
            }
        }
        if ((j & 7) == 7 && j + 1 < wcols) {
            const int j0 = j - 7;
            __syncthreads();   // the mini-panel's pivot rows (sh.top) and multipliers are in place
            // its U rows for the later columns: the pivot rows (as sent, before this mini-panel's
            // updates) take the updates of the earlier pivot rows in step order
            if (tid < WC && tid > j) {
                const int c = tid;
                float u[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    float x = sh.top[j0 + k][c];
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (q < k) x = fmaf(-sh.top[j0 + k][j0 + q], u[q], x);
                    u[k] = x;
                    sh.top[j0 + k][c] = x;
                    sh.ubT[c][k] = x;
                }
            }
            __syncthreads();
            for (int lr = tid; lr < myrows; lr += PANEL_THREADS) {
                const int g = g0 + lr;
                float* row = tile + lr * TS;
                if (g >= j0 && g <= j) {
                    // a pivot row of this mini-panel: its final U values
#pragma unroll
                    for (int c = 0; c < WC; ++c)
                        if (c > j) row[c] = sh.ubT[c][g - j0];
                } else if (g > j) {
                    float l[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) l[q] = row[j0 + q];
                    float nv = 0.0f;
                    switch (j >> 3) {   // j + 1 is 8, 16 or 24
                        case 0: nv = block_update<8, WC>(row, sh.ubT, l); break;
                        case 1: nv = block_update<(16 < WC ? 16 : WC), WC>(row, sh.ubT, l); break;
                        default: nv = block_update<(24 < WC ? 24 : WC), WC>(row, sh.ubT, l); break;
                    }
                    float v = fabsf(nv);
                    if (v != v) { local_flag |= DEV_NONFINITE; v = -1.0f; }
                    argmax_merge(bv, bi, v, g);
                }
            }
        }
    }
    // no CTA leaves while messages to it could still be in flight (only possible after a timeout)
    cluster_barrier();
    for (int e = tid; e < myrows * WC; e += PANEL_THREADS) {
        int lr = e / WC, c = e - lr * WC;
        if (c < wcols) {
            const float v = tile[lr * TS + c];
            W[(r0 + g0 + lr) * ldw + r0 + c] = v;
            if (tail.LU) tail.LU[(r0 + g0 + lr) * tail.ldl + r0 + c] = float_to_uf(v, tail.fmt);
        }
    }
    if (local_flag) atomicOr(flags, local_flag);

    panel_tail_work<WC>(sh, W, ldw, r0, wcols, tail, C, rank, tid, lane, warp);
}

// ------------------------------------------------------------------ swaps, TRSM

// ------------------------------------------------------------------ row permutations
// The interchanges k in [k0, k1) (rows k <-> ipiv[k], applied in order) form one permutation
// of at most 2 (k1 - k0) rows. k_swap_plan simulates them on row labels (slot table in shared
// memory, O(1) per interchange) and emits (dst, src) row pairs; k_permute_rows then moves the
// rows of a column range with coalesced loads and stores (all sources read before any write).
constexpr int PERM_MAXN = 50000;        // rows addressable by the shared slot table
constexpr int PERM_MAXK = 256;          // interchanges per plan (outer block width)

__global__ void __launch_bounds__(256) k_swap_plan(const int* __restrict__ ipiv, int64_t k0, int64_t k1,
                                                   int* __restrict__ plan, int* __restrict__ count,
                                                   int* __restrict__ perm) {
    extern __shared__ int slot_of[];            // indexed by row - k1 for rows >= k1
    __shared__ int content[2 * PERM_MAXK];
    __shared__ int rowof[2 * PERM_MAXK];
    __shared__ int piv_s[PERM_MAXK];
    __shared__ int slot_s[PERM_MAXK];
    __shared__ int scan_s[2 * PERM_MAXK];
    __shared__ int warp_tot[8];
    const int nk = (int)(k1 - k0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = tid; k < nk; k += 256) {
        int p = ipiv[k0 + k];
        piv_s[k] = p;
        if (p >= k1) slot_of[p - k1] = 0x7fffffff;
    }
    __syncthreads();
    // the first interchange that names a row below the block owns that row's slot
    for (int k = tid; k < nk; k += 256) {
        int p = piv_s[k];
        if (p >= k1) atomicMin(&slot_of[p - k1], k);
    }
    __syncthreads();
    // number the distinct rows below the block in order of first use (block scan of leader flags)
    auto block_scan = [&](int* flag, int len) -> int {   // exclusive scan in place, returns total
        const int per = (len + 255) / 256;               // contiguous items per thread
        int local = 0;
        for (int i = 0; i < per; ++i) { int k = tid * per + i; if (k < len) local += flag[k]; }
        int incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) { int t = __shfl_up_sync(0xffffffffu, incl, o); if (lane >= o) incl += t; }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        int wbase = 0, total = 0;
        for (int w2 = 0; w2 < 8; ++w2) { if (w2 < warp) wbase += warp_tot[w2]; total += warp_tot[w2]; }
        int run = wbase + incl - local;
        for (int i = 0; i < per; ++i) {
            int k = tid * per + i;
            if (k < len) { int f = flag[k]; flag[k] = run; run += f; }
        }
        __syncthreads();
        return total;
    };
    for (int k = tid; k < nk; k += 256) {
        int p = piv_s[k];
        scan_s[k] = (p >= k1 && slot_of[p - k1] == k) ? 1 : 0;
    }
    __syncthreads();
    const int next = block_scan(scan_s, nk);
    const int ns = nk + next;
    for (int k = tid; k < nk; k += 256) {
        content[k] = (int)(k0 + k);
        rowof[k] = (int)(k0 + k);
        int p = piv_s[k];
        if (p >= k1 && slot_of[p - k1] == k) {
            content[nk + scan_s[k]] = p;
            rowof[nk + scan_s[k]] = p;
        }
    }
    __syncthreads();
    for (int k = tid; k < nk; k += 256) {
        int p = piv_s[k];
        slot_s[k] = (p < k1) ? (int)(p - k0) : nk + scan_s[slot_of[p - k1]];
    }
    __syncthreads();
    // replay the interchanges in order on the slot contents (slot k is final after step k)
    if (tid == 0) {
        for (int k = 0; k < nk; ++k) {
            const int sb = slot_s[k];
            const int t = content[k];
            content[k] = content[sb];
            content[sb] = t;
        }
    }
    __syncthreads();
    // emit the moves dst <- src of the slots whose content changed
    for (int sidx = tid; sidx < ns; sidx += 256) scan_s[sidx] = (content[sidx] != rowof[sidx]) ? 1 : 0;
    __syncthreads();
    const int c = block_scan(scan_s, ns);
    for (int sidx = tid; sidx < ns; sidx += 256) {
        if (content[sidx] != rowof[sidx]) {
            plan[2 * scan_s[sidx]] = rowof[sidx];
            plan[2 * scan_s[sidx] + 1] = content[sidx];
        }
    }
    if (tid == 0) *count = c;
    // the same moves applied to the row permutation (perm[i] = original row now at position i)
    if (perm) {
        __shared__ int tmp_s[2 * PERM_MAXK];
        for (int sidx = tid; sidx < ns; sidx += 256)
            if (content[sidx] != rowof[sidx]) tmp_s[sidx] = perm[content[sidx]];
        __syncthreads();
        for (int sidx = tid; sidx < ns; sidx += 256)
            if (content[sidx] != rowof[sidx]) perm[rowof[sidx]] = tmp_s[sidx];
    }
}

__global__ void k_iota(int* __restrict__ v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (int)i;
}

constexpr int PERM_THREADS = 1024;
constexpr int PERM_CW = 32;                                   // columns per CTA
constexpr int PERM_PER = 2 * PERM_MAXK * PERM_CW / PERM_THREADS;  // staged values per thread
template <typename T>
__global__ void __launch_bounds__(PERM_THREADS) k_permute_rows(T* __restrict__ M, int64_t ld,
                                                               const int* __restrict__ plan,
                                                               const int* __restrict__ count, int64_t col0,
                                                               int64_t col1) {
    __shared__ int dst_s[2 * PERM_MAXK], src_s[2 * PERM_MAXK];
    const int cnt = *count;
    const int64_t c0 = col0 + (int64_t)blockIdx.x * PERM_CW;
    if (c0 >= col1 || cnt == 0) return;
    for (int i = threadIdx.x; i < cnt; i += PERM_THREADS) {
        dst_s[i] = plan[2 * i];
        src_s[i] = plan[2 * i + 1];
    }
    __syncthreads();
    const int width = (int)gmin<int64_t>(PERM_CW, col1 - c0);
    const int c = threadIdx.x % PERM_CW, r0 = threadIdx.x / PERM_CW;
    constexpr int RSTEP = PERM_THREADS / PERM_CW;
    T v[PERM_PER];
    // every source row of this column chunk is read (into registers) before any row is written
#pragma unroll
    for (int k = 0; k < PERM_PER; ++k) {
        const int r = r0 + k * RSTEP;
        if (r < cnt && c < width) v[k] = M[(int64_t)src_s[r] * ld + c0 + c];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PERM_PER; ++k) {
        const int r = r0 + k * RSTEP;
        if (r < cnt && c < width) M[(int64_t)dst_s[r] * ld + c0 + c] = v[k];
    }
}

// Outer TRSM of one block row band: X = L11^-1 W[r0:r0+nb, cols] with L11 the stored unit-lower
// u_f block (nb <= 256), computed block by block as the per-panel model does: for each 32-row
// block b, X_b = fl32(L_bb^-1 X_b) by FP32 substitution, U_b = fl_uf(X_b) (stored in LU, UT and
// used from then on), and the rows below are updated with the u_f operands L[.., b] and U_b
// (FP32 accumulation from zero over the 32 terms, then one FP32 subtraction).
// One CTA per TBC columns: the column slab lives in shared memory; L11 is staged one 32-column
// block at a time (double-buffered, the next block fetched into registers during this one).
constexpr int TB_MAXNB = 256;
constexpr int TB_LS = 34;   // u16 row stride of a staged L block column

template <int TBC>
constexpr size_t trsm_band_smem() {
    return (size_t)TB_MAXNB * (TBC + 1) * sizeof(float) + 2 * (size_t)TB_MAXNB * TB_LS * sizeof(uint16_t);
}

template <int TBC, bool RND>
__global__ void __launch_bounds__(256) k_trsm_band(uint16_t* __restrict__ LU, int64_t ldl, float* __restrict__ W,
                                                   int64_t ldw, int64_t r0, int nb, int64_t col0, int64_t col1,
                                                   int fmt, uint16_t* __restrict__ UT, int64_t ldut) {
    constexpr int XS = TBC + 1;
    constexpr int CPW = TBC / 8;                // columns per warp in the diagonal block
    static_assert(TBC % 8 == 0, "the diagonal block's columns are spread over 8 warps");
    constexpr int CG = TBC / 4;                 // column groups of 4 in the update
    constexpr int RG = 256 / CG;                // row groups
    constexpr int MAXR = (TB_MAXNB - 32 + RG - 1) / RG;
    constexpr int PF = TB_MAXNB * 32 / 256;     // prefetched L values per thread
    extern __shared__ __align__(16) unsigned char tb_raw[];
    float* X = reinterpret_cast<float*>(tb_raw);                                              // [nb][XS]
    uint16_t* Lb = reinterpret_cast<uint16_t*>(tb_raw + (size_t)TB_MAXNB * XS * sizeof(float));  // [2][nb][LS]
    const int tid = threadIdx.x;
    const int64_t c0 = col0 + (int64_t)blockIdx.x * TBC;
    const int width = (int)gmin<int64_t>(TBC, col1 - c0);
    for (int e = tid; e < nb * TBC; e += 256) {
        int i = e / TBC, c = e - i * TBC;
        X[i * XS + c] = (c < width) ? W[(r0 + i) * ldw + c0 + c] : 0.0f;
    }
    // block column b of L11 (rows b0..nb-1, columns b0..b0+31; zero on and above the diagonal)
    uint16_t pre[PF];
    auto fetch = [&](int b0) {
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            const int e = tid + k * 256, i = b0 + (e >> 5), q = e & 31;
            pre[k] = (i < nb && b0 + q < nb && q < i - b0) ? LU[(r0 + i) * ldl + r0 + b0 + q] : (uint16_t)0;
        }
    };
    auto stash = [&](int b0, uint16_t* L) {
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            const int e = tid + k * 256, i = b0 + (e >> 5), q = e & 31;
            if (i < nb) L[i * TB_LS + q] = pre[k];
        }
    };
    fetch(0);
    stash(0, Lb);
    __syncthreads();
    for (int b0 = 0, step = 0; b0 < nb; b0 += 32, ++step) {
        const int wb = min(32, nb - b0);
        const uint16_t* L = Lb + (step & 1) * TB_MAXNB * TB_LS;
        const bool more = b0 + 32 < nb;
        if (more) fetch(b0 + 32);
        {
            // forward substitution in the diagonal block: lane i of a warp holds row b0 + i (its
            // 32 multipliers in registers) for the warp's columns wp, wp + 8, ...; at step q lane q
            // holds the final x_q, which the lanes below take by shuffle: row i gets
            // x_i - L_i0 x_0 - L_i1 x_1 - ... by FMAs in ascending q, one dependent FMA per step
            const int lane = tid & 31, wp = tid >> 5;
            uint32_t lr[16];   // L[b0 + lane][0..31] as u16 pairs (zero on and above the diagonal)
            const uint32_t* Lrow = reinterpret_cast<const uint32_t*>(L + (b0 + lane) * TB_LS);
#pragma unroll
            for (int k = 0; k < 16; ++k) lr[k] = (lane < wb) ? Lrow[k] : 0u;
            float x[CPW];
#pragma unroll
            for (int j = 0; j < CPW; ++j) x[j] = (lane < wb) ? X[(b0 + lane) * XS + wp + 8 * j] : 0.0f;
#pragma unroll
            for (int q = 0; q < 31; ++q) {
                const uint32_t pair = lr[q >> 1];
                const float lq = uf_to_float((uint16_t)((q & 1) ? (pair >> 16) : (pair & 0xffffu)), fmt);
#pragma unroll
                for (int j = 0; j < CPW; ++j) {
                    const float xq = __shfl_sync(0xffffffffu, x[j], q);
                    if (lane > q) x[j] = fmaf(-lq, xq, x[j]);
                }
            }
            if (lane < wb) {
                const int i = lane;
#pragma unroll
                for (int j = 0; j < CPW; ++j) {
                    const int c = wp + 8 * j;
                    if (RND) {
                        const uint16_t u = float_to_uf(x[j], fmt);
                        const float uv = uf_to_float(u, fmt);
                        X[(b0 + i) * XS + c] = uv;
                        if (c < width) {
                            W[(r0 + b0 + i) * ldw + c0 + c] = uv;
                            LU[(r0 + b0 + i) * ldl + c0 + c] = u;
                            UT[(c0 + c) * ldut + b0 + i] = u;
                        }
                    } else {
                        // FP8 blocks: FP32 values throughout, rounded tile by tile afterwards
                        X[(b0 + i) * XS + c] = x[j];
                        if (c < width) W[(r0 + b0 + i) * ldw + c0 + c] = x[j];
                    }
                }
            }
        }
        __syncthreads();
        // rows below the block: X[i] -= sum_q L[i, b0+q] U_b[q]
        const int rb = b0 + wb;
        if (rb < nb) {
            const int tx = tid % CG, ty = tid / CG;
            float acc[MAXR][4];
#pragma unroll
            for (int m = 0; m < MAXR; ++m)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[m][k] = 0.0f;
            for (int q = 0; q < wb; ++q) {
                float u[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) u[k] = X[(b0 + q) * XS + tx * 4 + k];
#pragma unroll
                for (int m = 0; m < MAXR; ++m) {
                    const int i = rb + ty + m * RG;
                    if (i < nb) {
                        const float l = uf_to_float(L[i * TB_LS + q], fmt);
#pragma unroll
                        for (int k = 0; k < 4; ++k) acc[m][k] = fmaf(l, u[k], acc[m][k]);
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < MAXR; ++m) {
                const int i = rb + ty + m * RG;
                if (i < nb) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) X[i * XS + tx * 4 + k] -= acc[m][k];
                }
            }
        }
        if (more) stash(b0 + 32, Lb + ((step + 1) & 1) * TB_MAXNB * TB_LS);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ FP8-E4M3 operand tiles
// Rounding of an operand region to e4m3 with one power-of-two scale per 128 x 128 tile of the
// global tile grid: s = 2^floor(log2(448 / max|tile|)) (1 for an all-zero tile), value =
// RN_sat_e4m3(x s) / s. The value has at most 4 significant bits, so it is stored exactly as a
// bf16 bit pattern in LU (and transposed in UT): the bf16 tensor-core update then multiplies
// exactly the e4m3 operands the block-scaled FP8 model prescribes, with FP32 accumulation.
// part: TILE_FULL every entry; TILE_LOWER entries below the diagonal (row > col);
// TILE_UPPER entries on and above it. One CTA per tile.
enum { TILE_FULL = 0, TILE_LOWER = 1, TILE_UPPER = 2 };
constexpr int FP8_TILE = 128;

__global__ void __launch_bounds__(256) k_quant_tiles(const float* __restrict__ W, int64_t ldw, uint16_t* __restrict__ LU,
                                                     int64_t ldl, uint16_t* __restrict__ UT, int64_t ldut,
                                                     int64_t ut_row0, int64_t r0, int64_t nrows, int64_t c0,
                                                     int64_t ncols, int part) {
    __shared__ float wmax[8];
    const int tid = threadIdx.x;
    // tile (tr, tc) of the global grid that intersects the region
    const int64_t tr0 = (r0 / FP8_TILE + blockIdx.y) * FP8_TILE;
    const int64_t tc0 = (c0 / FP8_TILE + blockIdx.x) * FP8_TILE;
    const int64_t rb = gmax<int64_t>(tr0, r0), re = gmin<int64_t>(tr0 + FP8_TILE, r0 + nrows);
    const int64_t cb = gmax<int64_t>(tc0, c0), ce = gmin<int64_t>(tc0 + FP8_TILE, c0 + ncols);
    if (rb >= re || cb >= ce) return;
    const int64_t h = re - rb, w = ce - cb;
    auto inside = [&](int64_t i, int64_t j) {
        return part == TILE_FULL || (part == TILE_LOWER ? i > j : i <= j);
    };
    float m = 0.0f;
    for (int64_t e = tid; e < h * w; e += 256) {
        const int64_t i = rb + e / w, j = cb + e % w;
        if (inside(i, j)) m = fmaxf(m, fabsf(W[i * ldw + j]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) wmax[tid >> 5] = m;
    __syncthreads();
    m = wmax[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) m = fmaxf(m, wmax[k]);
    double sc = 1.0;
    if (m > 0.0f) {
        int ex = 0;
        frexp(448.0 / (double)m, &ex);   // 448 / m = f 2^ex with f in [0.5, 1)
        sc = ldexp(1.0, ex - 1);
    }
    const float s = (float)sc, inv = (float)(1.0 / sc);
    for (int64_t e = tid; e < h * w; e += 256) {
        const int64_t i = rb + e / w, j = cb + e % w;
        if (!inside(i, j)) continue;
        const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(W[i * ldw + j] * s, __NV_SATFINITE, __NV_E4M3);
        const __half_raw hr = __nv_cvt_fp8_to_halfraw(q, __NV_E4M3);
        const float v = __half2float(__half(hr)) * inv;
        const uint16_t b = __bfloat16_as_ushort(__float2bfloat16_rn(v));
        LU[i * ldl + j] = b;
        if (UT) UT[j * ldut + (i - ut_row0)] = b;
    }
}

static void quantize_tiles(const float* W, int64_t ldw, uint16_t* LU, int64_t ldl, uint16_t* UT, int64_t ldut,
                           int64_t r0, int64_t nrows, int64_t c0, int64_t ncols, int part, cudaStream_t s) {
    if (nrows <= 0 || ncols <= 0) return;
    const unsigned gx = (unsigned)((c0 + ncols - 1) / FP8_TILE - c0 / FP8_TILE + 1);
    const unsigned gy = (unsigned)((r0 + nrows - 1) / FP8_TILE - r0 / FP8_TILE + 1);
    count_launch(), k_quant_tiles<<<dim3(gx, gy), 256, 0, s>>>(W, ldw, LU, ldl, UT, ldut, r0, r0, nrows, c0, ncols, part);
}

// ------------------------------------------------------------------ SIMT trailing update
// C[M x N] -= A[M x K] * B[K x N] with u_f operands (16-bit, row-major) and FP32 accumulation.
// 128 x 128 tile, BK = 16, 256 threads, 8 x 8 outputs per thread.
template <typename T>
__device__ __forceinline__ float operand_value(T v, int fmt);
template <>
__device__ __forceinline__ float operand_value<uint16_t>(uint16_t v, int fmt) { return uf_to_float(v, fmt); }
template <>
__device__ __forceinline__ float operand_value<float>(float v, int) { return v; }

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_sub_simt(float* __restrict__ Cm, int64_t ldc,
                                                       const T* __restrict__ Am, int64_t lda,
                                                       const T* __restrict__ Bm, int64_t ldb, int M, int N,
                                                       int K, int fmt) {
    __shared__ float As[16][128 + 4];
    __shared__ float Bs[16][128 + 4];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * 128, n0 = blockIdx.x * 128;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
    for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int e = tid + t * 256;           // 0..2047
            int mi = e >> 4, kk = e & 15;    // A: 128 rows x 16 k
            int gm = m0 + mi, gk = k0 + kk;
            As[kk][mi] = (gm < M && gk < K) ? operand_value<T>(Am[(int64_t)gm * lda + gk], fmt) : 0.0f;
            int kb = e >> 7, ni = e & 127;   // B: 16 k x 128 cols
            int gkb = k0 + kb, gn = n0 + ni;
            Bs[kb][ni] = (gkb < K && gn < N) ? operand_value<T>(Bm[(int64_t)gkb * ldb + gn], fmt) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[8], b[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) { a[q] = As[kk][ty * 8 + q]; b[q] = Bs[kk][tx * 8 + q]; }
#pragma unroll
            for (int p = 0; p < 8; ++p)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        int gm = m0 + ty * 8 + p;
        if (gm >= M) continue;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            int gn = n0 + tx * 8 + q;
            if (gn < N) Cm[(int64_t)gm * ldc + gn] -= acc[p][q];
        }
    }
}

// ------------------------------------------------------------------ host driver
// GIR_DEBUG_LU=1: synchronise after every stage and report the first stage that raises a flag.
static int debug_lu_env() {
    const char* e = getenv("GIR_DEBUG_LU");
    return (e && e[0] == '1') ? 1 : 0;
}
static int debug_lu() {
    static const int v = debug_lu_env();
    return v;
}
static gir_status debug_check(const char* stage, int64_t a, int64_t b, int* flags, cudaStream_t s) {
    if (!debug_lu()) return GIR_OK;
    GIR_CUDA_TRY(cudaStreamSynchronize(s));
    int f = 0;
    GIR_CUDA_TRY(cudaMemcpy(&f, flags, sizeof(int), cudaMemcpyDeviceToHost));
    static int last = 0;
    if (f != last) {
        fprintf(stderr, "gir LU debug: flags %d -> %d after %s (%lld, %lld)\n", last, f, stage, (long long)a,
                (long long)b);
        last = f;
    }
    return GIR_OK;
}

// C -= A B with FP32 operands (inside an FP8 block column, before its operands are rounded).
static gir_status gemm_sub_f32(float* C, int64_t ldc, const float* A, int64_t lda, const float* B, int64_t ldb,
                               int64_t M, int64_t N, int64_t K, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return GIR_OK;
    dim3 grid((unsigned)((N + 127) / 128), (unsigned)((M + 127) / 128));
    count_launch(), k_gemm_sub_simt<float><<<grid, 256, 0, s>>>(C, ldc, A, lda, B, ldb, (int)M, (int)N, (int)K, 0);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

static gir_status gemm_sub(float* C, int64_t ldc, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb,
                           const uint16_t* Bt, int64_t ldbt, int64_t M, int64_t N, int64_t K, int fmt,
                           const LUPlan& plan, int* flags, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return GIR_OK;
    if (plan.use_tc && Bt && tc_gemm_supported(M, N, K, lda, ldbt, ldc)) {
        gir_status st = launch_tc_gemm_sub(C, ldc, A, lda, Bt, ldbt, M, N, K, fmt, flags, s);
        if (st != GIR_UNSUPPORTED) return st;
    }
    dim3 grid((unsigned)((N + 127) / 128), (unsigned)((M + 127) / 128));
    count_launch(), k_gemm_sub_simt<uint16_t><<<grid, 256, 0, s>>>(C, ldc, A, lda, B, ldb, (int)M, (int)N, (int)K, fmt);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

struct SwapScratch {
    int* plan = nullptr;   // 2 * 2 * PERM_MAXK ints
    int* count = nullptr;
};

static gir_status make_plan(const int* ipiv, int64_t k0, int64_t k1, int64_t n, const SwapScratch& sw, int* perm,
                            cudaStream_t s) {
    if (k1 - k0 > PERM_MAXK || n - k1 > PERM_MAXN) return GIR_UNSUPPORTED;
    size_t smem = (size_t)gmax<int64_t>(1, n - k1) * sizeof(int);
    count_launch(), k_swap_plan<<<1, 256, smem, s>>>(ipiv, k0, k1, sw.plan, sw.count, perm);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

template <typename T>
static gir_status permute_rows(T* M, int64_t ld, int64_t col0, int64_t col1, const SwapScratch& sw, cudaStream_t s) {
    if (col1 <= col0) return GIR_OK;
    count_launch(), k_permute_rows<T><<<(unsigned)((col1 - col0 + PERM_CW - 1) / PERM_CW), PERM_THREADS, 0, s>>>(
        M, ld, sw.plan, sw.count, col0, col1);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

static gir_status launch_panel(float* W, int64_t ldw, int64_t c0, int64_t n, int wc, int* ipiv, int* flags,
                               const LUPlan& plan, const PanelTail& tail, cudaStream_t s) {
    const int64_t h = n - c0;
    const int64_t budget = plan.panel_smem_budget;
    const int WC = plan.w;
    int64_t bytes_per_row = (int64_t)(WC + 1) * 4;  // padded rows (see k_panel)
    // cluster size: enough CTAs for the panel to fit the shared-memory budget, and (where the
    // cluster limit allows) at most two rows per thread
    int C = (int)((h * bytes_per_row + budget - 1) / budget);
    if (C < 1) C = 1;
    if (C > plan.max_cluster) return GIR_UNSUPPORTED;
    if (!plan.forced_cluster) {
        int64_t by_rows = (h + 2 * PANEL_THREADS - 1) / (2 * PANEL_THREADS);
        C = (int)gmax<int64_t>(C, gmin<int64_t>(by_rows, plan.max_cluster));
    }
    int rpc = (int)((h + C - 1) / C);
    while (!plan.forced_cluster && (int64_t)rpc * bytes_per_row > budget && C < plan.max_cluster) {
        ++C;
        rpc = (int)((h + C - 1) / C);
    }
    if ((int64_t)rpc * bytes_per_row > (plan.forced_cluster ? LUPlan().panel_smem_budget : budget))
        return GIR_UNSUPPORTED;
    size_t smem = (WC == 32 ? sizeof(PanelShared<32>) : sizeof(PanelShared<16>)) + (size_t)rpc * bytes_per_row;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(PANEL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch();
    if (WC == 32) {
        GIR_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_panel<32>, W, ldw, c0, n, wc, rpc, ipiv, flags, tail));
    } else {
        GIR_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_panel<16>, W, ldw, c0, n, wc, rpc, ipiv, flags, tail));
    }
    return GIR_OK;
}

gir_status lu_panel_only(float* W, int64_t ldw, int64_t m, int w, int* ipiv, int cluster, int* flags,
                         cudaStream_t s) {
    LUPlan plan;
    GIR_TRY(lu_prepare(plan));
    if (w < 1 || w > 32) return GIR_INVALID_ARG;
    plan.w = (w <= 16) ? 16 : 32;
    if (cluster > 0) {
        // force the given cluster size through the shared-memory budget
        int64_t bytes = m * (int64_t)(plan.w + 1) * 4;
        plan.panel_smem_budget = (bytes + cluster - 1) / cluster;
        if (plan.panel_smem_budget < 4) plan.panel_smem_budget = 4;
        plan.forced_cluster = 1;
    }
    PanelTail tail = {nullptr, 0, 0, 0, 0, 0, 0, nullptr, 0, 0, 0, 0};
    return launch_panel(W, ldw, 0, m, w, ipiv, flags, plan, tail, s);
}

gir_status lu_update_only(float* C, int64_t ldc, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb,
                          const uint16_t* Bt, int64_t ldbt, int64_t M, int64_t N, int64_t K, int fmt, int use_tc,
                          int* flags, cudaStream_t s) {
    LUPlan plan;
    plan.use_tc = use_tc;
    return gemm_sub(C, ldc, A, lda, B, ldb, Bt, ldbt, M, N, K, fmt, plan, flags, s);
}

gir_status lu_prepare(LUPlan& plan) {
    int dev;
    GIR_CUDA_TRY(cudaGetDevice(&dev));
    const size_t max_smem = sizeof(PanelShared<32>) + (size_t)plan.panel_smem_budget;
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_panel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_panel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_panel<32>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_panel<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_trsm_band<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)trsm_band_smem<8>()));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_trsm_band<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)trsm_band_smem<64>()));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_trsm_band<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)trsm_band_smem<8>()));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_trsm_band<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)trsm_band_smem<64>()));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_swap_plan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(PERM_MAXN * sizeof(int))));
    const char* e = getenv("GIR_NO_TC");
    if (e && e[0] == '1') plan.use_tc = 0;  // CUDA-core trailing update (for A/B comparisons)
    return GIR_OK;
}

gir_status lu_scale_quantize(const double* A, int64_t n, int64_t lda, int uf, double* R, double* S, double* mu,
                             float* W, int64_t ldw, unsigned long long* colmax, int* flags, cudaStream_t s) {
    const double* Rp = nullptr;
    const double* Sp = nullptr;
    *mu = 1.0;
    if (uf == GIR_FP16) {
        int g = (int)gmin<int64_t>((n + 7) / 8, 152 * 16);
        count_launch(), k_row_scale<<<g, 256, 0, s>>>(A, n, lda, R, flags);
        GIR_CUDA_TRY(cudaMemsetAsync(colmax, 0, n * sizeof(unsigned long long), s));
        dim3 grid((unsigned)((n + 255) / 256), (unsigned)((n + 255) / 256));
        count_launch(), k_col_absmax<<<grid, 256, 0, s>>>(A, n, lda, R, colmax);
        count_launch(), k_col_scale<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(colmax, n, S);
        // largest power of two <= 0.1 * 65504 / sqrt(n): headroom for the growth of partial pivoting
        *mu = exp2(floor(log2(0.1 * 65504.0 / sqrt((double)n))));
        Rp = R;
        Sp = S;
    }
    int g = (int)gmin<int64_t>(n, 152 * 16);
    count_launch(), k_quantize<<<g, 256, 0, s>>>(A, n, lda, Rp, Sp, *mu, W, ldw, flags);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

// Look-ahead schedule: block k's trailing update is split into (a) the next block's columns,
// on the main stream, and (b) all later columns, on a side stream, so (b) runs while the next
// block's panels (a few SMs) are factored. Events keep every W update, row interchange and
// UT access ordered: (b)_k finishes before block k+1's end-of-block interchanges and (a)_{k+1}.
gir_status lu_factor(float* W, int64_t ldw, uint16_t* LU, int64_t ldl, int* ipiv, int* perm, int64_t n, int fmt,
                     const LUPlan& plan, uint16_t* UT, int* flags, cudaStream_t s_user) {
    const int w = plan.w;
    const int NB = plan.nb;
    const int64_t ldut = NB;
    if (NB > PERM_MAXK || NB > TB_MAXNB) return GIR_UNSUPPORTED;
    if (plan.fp8 && (NB != FP8_TILE || w != 32)) return GIR_UNSUPPORTED;
    const bool fp8 = plan.fp8 != 0;
    SwapScratch sw;
    // The critical path (panels, interchanges, next-block update) runs on a highest-priority
    // stream so that its small kernels get SMs ahead of the side stream's bulk trailing update.
    // Streams and events are released on every return path (queued work completes first).
    struct Streams {
        cudaStream_t s = nullptr, s2 = nullptr;
        cudaEvent_t ev_swapped = nullptr, ev_b = nullptr, ev_io = nullptr;
        ~Streams() {
            if (ev_swapped) cudaEventDestroy(ev_swapped);
            if (ev_b) cudaEventDestroy(ev_b);
            if (ev_io) cudaEventDestroy(ev_io);
            if (s2) cudaStreamDestroy(s2);
            if (s) cudaStreamDestroy(s);
        }
    } ss_;
    int prio_least = 0, prio_greatest = 0;
    GIR_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
    GIR_CUDA_TRY(cudaStreamCreateWithPriority(&ss_.s, cudaStreamNonBlocking, prio_greatest));
    GIR_CUDA_TRY(cudaStreamCreateWithPriority(&ss_.s2, cudaStreamNonBlocking, prio_least));
    GIR_CUDA_TRY(cudaEventCreateWithFlags(&ss_.ev_swapped, cudaEventDisableTiming));
    GIR_CUDA_TRY(cudaEventCreateWithFlags(&ss_.ev_b, cudaEventDisableTiming));
    GIR_CUDA_TRY(cudaEventCreateWithFlags(&ss_.ev_io, cudaEventDisableTiming));
    cudaStream_t s = ss_.s;
    cudaStream_t s2 = ss_.s2;
    cudaEvent_t ev_swapped = ss_.ev_swapped, ev_b = ss_.ev_b;
    // join: the factorization starts after the caller's earlier work and ends before its later work
    GIR_CUDA_TRY(cudaEventRecord(ss_.ev_io, s_user));
    GIR_CUDA_TRY(cudaStreamWaitEvent(s, ss_.ev_io, 0));
    GIR_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&sw.plan), 4 * PERM_MAXK * sizeof(int), s));
    GIR_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&sw.count), sizeof(int), s));
    if (perm) count_launch(), k_iota<<<(unsigned)gmin<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(perm, n);
    bool b_pending = false;  // a (b) part is running on s2
    gir_status st = GIR_OK;
    // wide column slabs for the bulk (two CTAs per SM), narrow ones for the next block's 256
    // columns on the critical path (32 CTAs of 8 columns: the solve is latency-bound there)
    auto trsm_band = [&](int64_t C0, int64_t NBc, int64_t col0, int64_t col1, bool narrow, cudaStream_t ss) {
        if (col1 <= col0) return;
        if (narrow) {
            if (fp8)
                count_launch(), k_trsm_band<8, false><<<(unsigned)((col1 - col0 + 7) / 8), 256, trsm_band_smem<8>(), ss>>>(
                    LU, ldl, W, ldw, C0, (int)NBc, col0, col1, fmt, UT, ldut);
            else
                count_launch(), k_trsm_band<8, true><<<(unsigned)((col1 - col0 + 7) / 8), 256, trsm_band_smem<8>(), ss>>>(
                    LU, ldl, W, ldw, C0, (int)NBc, col0, col1, fmt, UT, ldut);
        } else {
            if (fp8)
                count_launch(), k_trsm_band<64, false><<<(unsigned)((col1 - col0 + 63) / 64), 256, trsm_band_smem<64>(), ss>>>(
                    LU, ldl, W, ldw, C0, (int)NBc, col0, col1, fmt, UT, ldut);
            else
                count_launch(), k_trsm_band<64, true><<<(unsigned)((col1 - col0 + 63) / 64), 256, trsm_band_smem<64>(), ss>>>(
                    LU, ldl, W, ldw, C0, (int)NBc, col0, col1, fmt, UT, ldut);
        }
        // FP8: U12 of these columns rounded 128 x 128 tile by tile (LU, UT)
        if (fp8) quantize_tiles(W, ldw, LU, ldl, UT, ldut, C0, NBc, col0, col1 - col0, TILE_FULL, ss);
    };
    for (int64_t C0 = 0; C0 < n && st == GIR_OK; C0 += NB) {
        const int64_t NBc = gmin<int64_t>(NB, n - C0);
        const int64_t Cend = C0 + NBc;
        for (int64_t c0 = C0; c0 < Cend; c0 += w) {
            const int wc = (int)gmin<int64_t>(w, Cend - c0);
            int t_ = trace_begin(s, "lu panel");
            // GIR_TRACE_DETAIL=1: the panel phase also reported per panel-height class
            const int td_ = trace_detail() ? trace_begin(s, nullptr) : -1;
            {
                // the panel kernel also stores the u_f panel, applies its interchanges to the
                // block's later columns of W and earlier columns of LU, and solves for U12
                PanelTail tail = {LU, ldl, fmt, c0 + wc, Cend, C0, c0, UT + (c0 - C0), ldut, 0, 0, 1};
                if (fp8) {
                    // inside an FP8 block column everything stays FP32 in W: the earlier panels'
                    // multipliers take the interchanges there, and U12 is solved unrounded
                    tail = PanelTail{nullptr, ldl, fmt, c0 + wc, Cend, 0, 0, nullptr, 0, C0, c0, 2};
                }
                GIR_TRY(launch_panel(W, ldw, c0, n, wc, ipiv, flags, plan, tail, s));
            }
            trace_end(t_, "lu panel", s);
            if (td_ >= 0) {
                const int64_t h_ = n - c0;
                trace_end(td_, h_ > 8192 ? "panel h>8192" : h_ > 2048 ? "panel 2048<h<=8192" :
                               h_ > 512 ? "panel 512<h<=2048" : "panel h<=512", s);
            }
            GIR_TRY(debug_check("panel", C0, c0, flags, s));
            if (c0 + wc < Cend) {
                int64_t ncols = Cend - (c0 + wc);
                t_ = trace_begin(s, "lu inner gemm");
                if (fp8) {
                    GIR_TRY(gemm_sub_f32(W + (c0 + wc) * ldw + (c0 + wc), ldw, W + (c0 + wc) * ldw + c0, ldw,
                                         W + c0 * ldw + (c0 + wc), ldw, n - (c0 + wc), ncols, wc, s));
                } else {
                    GIR_TRY(gemm_sub(W + (c0 + wc) * ldw + (c0 + wc), ldw, LU + (c0 + wc) * ldl + c0, ldl,
                                     LU + c0 * ldl + (c0 + wc), ldl, UT + (c0 + wc) * ldut + (c0 - C0), ldut,
                                     n - (c0 + wc), ncols, wc, fmt, plan, flags, s));
                }
                trace_end(t_, "lu inner gemm", s);
                GIR_TRY(debug_check("inner gemm", C0, c0, flags, s));
            }
        }
        if (fp8) {
            // the block column's factors, rounded to e4m3 tile by tile: L below the diagonal and U11
            quantize_tiles(W, ldw, LU, ldl, nullptr, 0, C0, n - C0, C0, NBc, TILE_LOWER, s);
            quantize_tiles(W, ldw, LU, ldl, nullptr, 0, C0, NBc, C0, NBc, TILE_UPPER, s);
        }
        // the previous block's (b) part touches the trailing W columns and reads L rows of that
        // block: it must finish before this block's interchanges move those rows
        if (b_pending) {
            GIR_CUDA_TRY(cudaStreamWaitEvent(s, ev_b, 0));
            b_pending = false;
        }
        int t_ = trace_begin(s, "lu outer swaps");
        GIR_TRY(make_plan(ipiv, C0, Cend, n, sw, perm, s));
        GIR_TRY(permute_rows<float>(W, ldw, Cend, n, sw, s));
        trace_end(t_, "lu outer swaps", s);
        if (C0 > 0) {
            // the earlier blocks' L columns take the interchanges on the side stream: nothing on the
            // critical path reads them, and the side stream runs them after the previous block's
            // (b) part, which reads those rows; the next block's plan waits for ev_b
            GIR_CUDA_TRY(cudaEventRecord(ev_swapped, s));
            GIR_CUDA_TRY(cudaStreamWaitEvent(s2, ev_swapped, 0));
            GIR_TRY(permute_rows<uint16_t>(LU, ldl, 0, C0, sw, s2));
            GIR_CUDA_TRY(cudaEventRecord(ev_b, s2));
            b_pending = true;
        }
        if (Cend < n) {
            const int64_t ntr = n - Cend;
            const int64_t Ca = gmin<int64_t>(n, Cend + NB);  // (a): columns [Cend, Ca)
            // (a) on the main stream: the next block's columns
            t_ = trace_begin(s, "lu outer trsm");
            trsm_band(C0, NBc, Cend, Ca, true, s);
            trace_end(t_, "lu outer trsm", s);
            GIR_TRY(debug_check("outer trsm a", C0, Cend, flags, s));
            t_ = trace_begin(s, "lu outer gemm");
            GIR_TRY(gemm_sub(W + Cend * ldw + Cend, ldw, LU + Cend * ldl + C0, ldl, LU + C0 * ldl + Cend, ldl,
                             UT + Cend * ldut, ldut, ntr, Ca - Cend, NBc, fmt, plan, flags, s));
            trace_end(t_, "lu outer gemm", s);
            if (Ca < n) {
                // (b) on the side stream, after this block's interchanges
                GIR_CUDA_TRY(cudaEventRecord(ev_swapped, s));
                GIR_CUDA_TRY(cudaStreamWaitEvent(s2, ev_swapped, 0));
                int tb = trace_begin(s2, "lu outer trsm");
                trsm_band(C0, NBc, Ca, n, false, s2);
                trace_end(tb, "lu outer trsm", s2);
                tb = trace_begin(s2, "lu outer gemm");
                GIR_TRY(gemm_sub(W + Cend * ldw + Ca, ldw, LU + Cend * ldl + C0, ldl, LU + C0 * ldl + Ca, ldl,
                                 UT + Ca * ldut, ldut, ntr, n - Ca, NBc, fmt, plan, flags, s2));
                trace_end(tb, "lu outer gemm", s2);
                GIR_CUDA_TRY(cudaEventRecord(ev_b, s2));
                b_pending = true;
            }
            GIR_TRY(debug_check("outer gemm", C0, Cend, flags, s));
        }
    }
    if (b_pending) GIR_CUDA_TRY(cudaStreamWaitEvent(s, ev_b, 0));
    cudaFreeAsync(sw.plan, s);
    cudaFreeAsync(sw.count, s);
    GIR_CUDA_TRY(cudaEventRecord(ss_.ev_io, s));
    GIR_CUDA_TRY(cudaStreamWaitEvent(s_user, ss_.ev_io, 0));
    GIR_CUDA_TRY(cudaGetLastError());
    return st;
}

}  // namespace gir
