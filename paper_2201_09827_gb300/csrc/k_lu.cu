// Precision-u_f LU with partial pivoting (Algorithm 4, line 1) for GB300.
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
        for (int64_t j = lane; j < n; j += 32) {
            double v = fabs(A[i * lda + j]);
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
    const int64_t total = n * n;
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / n, j = e - i * n;
        double v = A[i * lda + j];
        if (R) v *= R[i] * S[j] * mu;
        float f = __double2float_rn(v);
        bad |= !(fabsf(f) <= 3.4028234663852886e38f);
        W[i * ldw + j] = f;
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

constexpr int PANEL_THREADS = 512;
constexpr int PANEL_MAXC = 16;

template <int WC>
struct PanelShared {
    float cand_val[2][PANEL_MAXC];
    int cand_row[2][PANEL_MAXC];
    float cand_rowv[2][PANEL_MAXC][WC];
    float rowj[2][WC];
    float wbest_val[2][PANEL_THREADS / 32];
    int wbest_row[2][PANEL_THREADS / 32];
};

template <int WC>
__global__ void __launch_bounds__(PANEL_THREADS, 1)
k_panel(float* __restrict__ W, int64_t ldw, int64_t r0, int64_t n, int wcols, int rpc, int* __restrict__ ipiv,
        int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PanelShared<WC>& sh = *reinterpret_cast<PanelShared<WC>*>(smem_raw);
    // rows padded to WC + 1 floats so that a warp reading one column of 32 rows hits 32 banks
    constexpr int TS = WC + 1;
    float* tile = reinterpret_cast<float*>(smem_raw + sizeof(PanelShared<WC>));  // [rpc][TS]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rank = (int)cluster_nctarank() > 1 ? (int)cluster_ctarank() : 0;
    const int C = (int)cluster_nctarank();
    const int64_t h = n - r0;
    const int g0 = rank * rpc;                              // first panel row of this CTA
    const int myrows = (int)gmax<int64_t>(0, gmin<int64_t>(rpc, h - g0));

    // load own rows (zero-fill columns beyond wcols)
    for (int e = tid; e < myrows * WC; e += PANEL_THREADS) {
        int lr = e / WC, c = e - lr * WC;
        tile[lr * TS + c] = (c < wcols) ? W[(r0 + g0 + lr) * ldw + r0 + c] : 0.0f;
    }
    __syncthreads();
    cluster_barrier();

    int local_flag = 0;
    for (int j = 0; j < wcols; ++j) {
        const int buf = j & 1;
        // local argmax over own rows with panel row >= j
        float bv = -1.0f;
        int bi = 0x7fffffff;
        for (int lr = tid; lr < myrows; lr += PANEL_THREADS) {
            int g = g0 + lr;
            if (g >= j) {
                float v = fabsf(tile[lr * TS + j]);
                if (v != v) { local_flag |= DEV_NONFINITE; v = -1.0f; }
                if (v > bv || (v == bv && g < bi)) { bv = v; bi = g; }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (lane == 0) { sh.wbest_val[buf][warp] = bv; sh.wbest_row[buf][warp] = bi; }
        __syncthreads();
        if (warp == 0) {
            float v = (lane < PANEL_THREADS / 32) ? sh.wbest_val[buf][lane] : -1.0f;
            int r = (lane < PANEL_THREADS / 32) ? sh.wbest_row[buf][lane] : 0x7fffffff;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                float ov = __shfl_xor_sync(0xffffffffu, v, o);
                int oi = __shfl_xor_sync(0xffffffffu, r, o);
                if (ov > v || (ov == v && oi < r)) { v = ov; r = oi; }
            }
            // candidate (value, row) to every CTA's slot [rank]
            if (lane < C) {
                st_cluster_f32(map_shared(&sh.cand_val[buf][rank], lane), v);
                st_cluster_s32(map_shared(&sh.cand_row[buf][rank], lane), r);
            }
            const int clr = (r != 0x7fffffff) ? r - g0 : -1;
            const bool own_j = (j >= g0 && j < g0 + myrows);
            for (int e = lane; e < C * WC; e += 32) {
                int q = e / WC, c = e - q * WC;
                float val = (clr >= 0) ? tile[clr * TS + c] : 0.0f;
                st_cluster_f32(map_shared(&sh.cand_rowv[buf][rank][c], q), val);
                if (own_j) st_cluster_f32(map_shared(&sh.rowj[buf][c], q), tile[(j - g0) * TS + c]);
            }
        }
        cluster_barrier();
        // global winner
        float pv = -1.0f;
        int pr = 0x7fffffff, pq = 0;
        for (int q = 0; q < C; ++q) {
            float v = sh.cand_val[buf][q];
            int r = sh.cand_row[buf][q];
            if (v > pv || (v == pv && r < pr)) { pv = v; pr = r; pq = q; }
        }
        if (pr == 0x7fffffff) {
            // no finite candidate in the column (all NaN): keep the row order, flag, divide by nothing
            pr = j;
            pv = 0.0f;
            local_flag |= DEV_NONFINITE;
        }
        const float* prow = sh.cand_rowv[buf][pq];
        const float* rj = sh.rowj[buf];
        const float piv = prow[j];
        if (tid == 0 && rank == 0) {
            ipiv[r0 + j] = (int)(r0 + pr);
            if (pv == 0.0f) local_flag |= DEV_SINGULAR;
        }
        for (int lr = tid; lr < myrows; lr += PANEL_THREADS) {
            int g = g0 + lr;
            float* row = tile + lr * TS;
            if (g == j) {
#pragma unroll
                for (int c = 0; c < WC; ++c) row[c] = prow[c];
            } else if (g == pr) {
#pragma unroll
                for (int c = 0; c < WC; ++c) row[c] = rj[c];
            }
            if (g > j) {
                float l = (piv != 0.0f) ? __fdiv_rn(row[j], piv) : 0.0f;
                row[j] = l;
#pragma unroll
                for (int c = 0; c < WC; ++c)
                    if (c > j) row[c] = fmaf(-l, prow[c], row[c]);
            }
        }
        __syncthreads();
    }
    cluster_barrier();
    for (int e = tid; e < myrows * WC; e += PANEL_THREADS) {
        int lr = e / WC, c = e - lr * WC;
        if (c < wcols) W[(r0 + g0 + lr) * ldw + r0 + c] = tile[lr * TS + c];
    }
    if (local_flag) atomicOr(flags, local_flag);
}

// ------------------------------------------------------------------ stores, swaps, TRSM
// LU16[r][c0 + c] = fl_uf(W[r][c0 + c]) for panel rows r in [c0, n), c < wc.
__global__ void k_store_panel(const float* __restrict__ W, int64_t ldw, uint16_t* __restrict__ LU, int64_t ldl,
                              int64_t c0, int wc, int64_t n, int fmt) {
    const int64_t rows = n - c0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * wc; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = c0 + e / wc;
        int c = (int)(e % wc);
        LU[r * ldl + c0 + c] = float_to_uf(W[r * ldw + c0 + c], fmt);
    }
}

// Apply interchanges k in [k0, k1) (rows k <-> ipiv[k]) to W columns [col0, col1).
__global__ void k_laswp_f32(float* __restrict__ W, int64_t ldw, const int* __restrict__ ipiv, int64_t k0,
                            int64_t k1, int64_t col0, int64_t col1) {
    const int64_t j = col0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= col1) return;
    for (int64_t k = k0; k < k1; ++k) {
        int64_t p = ipiv[k];
        if (p != k) {
            float a = W[k * ldw + j], b = W[p * ldw + j];
            W[k * ldw + j] = b;
            W[p * ldw + j] = a;
        }
    }
}

// Row interchanges of later panels applied to the stored L columns: column j (panel
// [j/w*w, j/w*w + w)) sees the interchanges k in [max(kbeg, (j/w + 1) w), kend).
// Within an outer block this runs before the block's L21 feeds the outer update; the final
// pass covers the interchanges of later outer blocks.
__global__ void k_laswp_lower(uint16_t* __restrict__ LU, int64_t ldl, const int* __restrict__ ipiv, int64_t col0,
                              int64_t col1, int w, int64_t kbeg, int64_t kend, int per_outer, int64_t nb) {
    const int64_t j = col0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= col1) return;
    int64_t k0 = per_outer ? (j / nb + 1) * nb : (j / w + 1) * w;
    if (k0 < kbeg) k0 = kbeg;
    for (int64_t k = k0; k < kend; ++k) {
        int64_t p = ipiv[k];
        if (p != k) {
            uint16_t a = LU[k * ldl + j], b = LU[p * ldl + j];
            LU[k * ldl + j] = b;
            LU[p * ldl + j] = a;
        }
    }
}

// ------------------------------------------------------------------ row permutations
// The interchanges k in [k0, k1) (rows k <-> ipiv[k], applied in order) form one permutation
// of at most 2 (k1 - k0) rows. k_swap_plan simulates them on row labels (slot table in shared
// memory, O(1) per interchange) and emits (dst, src) row pairs; k_permute_rows then moves the
// rows of a column range with coalesced loads and stores (all sources read before any write).
constexpr int PERM_MAXN = 50000;        // rows addressable by the shared slot table
constexpr int PERM_MAXK = 512;          // interchanges per plan

__global__ void __launch_bounds__(256) k_swap_plan(const int* __restrict__ ipiv, int64_t k0, int64_t k1,
                                                   int* __restrict__ plan, int* __restrict__ count) {
    extern __shared__ int slot_of[];            // indexed by row - k1 for rows >= k1
    __shared__ int content[2 * PERM_MAXK];
    __shared__ int rowof[2 * PERM_MAXK];
    __shared__ int piv_s[PERM_MAXK];
    const int nk = (int)(k1 - k0);
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        int p = ipiv[k0 + k];
        piv_s[k] = p;
        if (p >= k1) slot_of[p - k1] = -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int ns = nk;
        for (int s = 0; s < nk; ++s) { content[s] = (int)(k0 + s); rowof[s] = (int)(k0 + s); }
        for (int k = 0; k < nk; ++k) {
            int p = piv_s[k];
            if (p >= k1 && slot_of[p - k1] < 0) {
                slot_of[p - k1] = ns;
                content[ns] = p;
                rowof[ns] = p;
                ++ns;
            }
        }
        for (int k = 0; k < nk; ++k) {
            int p = piv_s[k];
            int sa = k, sb = (p < k1) ? (int)(p - k0) : slot_of[p - k1];
            int t = content[sa];
            content[sa] = content[sb];
            content[sb] = t;
        }
        int c = 0;
        for (int s = 0; s < ns; ++s) {
            if (content[s] != rowof[s]) {
                plan[2 * c] = rowof[s];
                plan[2 * c + 1] = content[s];
                ++c;
            }
        }
        *count = c;
    }
}

template <typename T, int CW>
__global__ void __launch_bounds__(256) k_permute_rows(T* __restrict__ M, int64_t ld, const int* __restrict__ plan,
                                                      const int* __restrict__ count, int64_t col0, int64_t col1) {
    extern __shared__ __align__(16) unsigned char prow_raw[];
    T* buf = reinterpret_cast<T*>(prow_raw);   // [count][CW]
    const int cnt = *count;
    const int64_t c0 = col0 + (int64_t)blockIdx.x * CW;
    if (c0 >= col1) return;
    const int width = (int)gmin<int64_t>(CW, col1 - c0);
    for (int e = threadIdx.x; e < cnt * CW; e += blockDim.x) {
        int r = e / CW, c = e - r * CW;
        if (c < width) buf[e] = M[(int64_t)plan[2 * r + 1] * ld + c0 + c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * CW; e += blockDim.x) {
        int r = e / CW, c = e - r * CW;
        if (c < width) M[(int64_t)plan[2 * r] * ld + c0 + c] = buf[e];
    }
}

// X = L11^-1 W[r0:r0+w, col0:col1] with L11 the stored unit-lower u_f block at (r0, r0);
// FP32 substitution; the result is rounded to u_f and written to LU16 (and W).
// The rounded rows are also written transposed into UT (UT[j * ldut + i], K-major operand).
template <int WMAX>
__global__ void __launch_bounds__(256) k_trsm_rows(const uint16_t* __restrict__ LU, int64_t ldl, float* __restrict__ W,
                                                   int64_t ldw, int64_t r0, int w, int64_t col0, int64_t col1, int fmt,
                                                   uint16_t* __restrict__ LUout, uint16_t* __restrict__ UT,
                                                   int64_t ldut) {
    __shared__ float Ls[WMAX][WMAX];
    for (int e = threadIdx.x; e < WMAX * WMAX; e += blockDim.x) {
        int i = e / WMAX, q = e % WMAX;
        Ls[i][q] = (i < w && q < i) ? uf_to_float(LU[(r0 + i) * ldl + r0 + q], fmt) : 0.0f;
    }
    __syncthreads();
    const int64_t j = col0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= col1) return;
    float x[WMAX];
#pragma unroll
    for (int i = 0; i < WMAX; ++i) x[i] = (i < w) ? W[(r0 + i) * ldw + j] : 0.0f;
#pragma unroll
    for (int i = 1; i < WMAX; ++i) {
        float acc = x[i];
#pragma unroll
        for (int q = 0; q < WMAX; ++q)
            if (q < i) acc = fmaf(-Ls[i][q], x[q], acc);
        x[i] = acc;
    }
#pragma unroll
    for (int i = 0; i < WMAX; ++i) {
        if (i < w) {
            uint16_t u = float_to_uf(x[i], fmt);
            LUout[(r0 + i) * ldl + j] = u;
            W[(r0 + i) * ldw + j] = uf_to_float(u, fmt);
            if (UT) UT[j * ldut + i] = u;
        }
    }
}

// Outer TRSM of one block row band: X = L11^-1 W[r0:r0+nb, cols] with L11 the stored unit-lower
// u_f block (nb <= 256), computed block by block as the per-panel model does: for each 32-row
// block b, X_b = fl32(L_bb^-1 X_b) by FP32 substitution, U_b = fl_uf(X_b) (stored in LU, UT and
// used from then on), and the rows below are updated with the u_f operands L[.., b] and U_b
// (FP32 accumulation). One CTA per 64 columns; L11 and the column slab live in shared memory.
constexpr int TB_COLS = 64;
constexpr int TB_MAXNB = 256;

__global__ void __launch_bounds__(256) k_trsm_band(const uint16_t* __restrict__ LU, int64_t ldl, float* __restrict__ W,
                                                   int64_t ldw, int64_t r0, int nb, int w, int64_t col0, int64_t col1,
                                                   int fmt, uint16_t* __restrict__ LUout, uint16_t* __restrict__ UT,
                                                   int64_t ldut) {
    extern __shared__ __align__(16) unsigned char tb_raw[];
    uint16_t* Ls = reinterpret_cast<uint16_t*>(tb_raw);                            // [nb][nb]
    float* X = reinterpret_cast<float*>(tb_raw + (size_t)TB_MAXNB * TB_MAXNB * 2); // [nb][TB_COLS + 1]
    constexpr int XS = TB_COLS + 1;
    const int tid = threadIdx.x;
    const int64_t c0 = col0 + (int64_t)blockIdx.x * TB_COLS;
    const int width = (int)gmin<int64_t>(TB_COLS, col1 - c0);
    for (int e = tid; e < nb * nb; e += 256) {
        int i = e / nb, q = e - i * nb;
        Ls[e] = (q < i) ? LU[(r0 + i) * ldl + r0 + q] : (uint16_t)0;
    }
    for (int e = tid; e < nb * TB_COLS; e += 256) {
        int i = e / TB_COLS, c = e - i * TB_COLS;
        X[i * XS + c] = (c < width) ? W[(r0 + i) * ldw + c0 + c] : 0.0f;
    }
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += w) {
        const int wb = min(w, nb - b0);
        // substitution inside the block: thread per column (FP32 fused updates)
        if (tid < TB_COLS) {
            const int c = tid;
            for (int i = 1; i < wb; ++i) {
                float acc = X[(b0 + i) * XS + c];
                for (int q = 0; q < i; ++q) acc = fmaf(-uf_to_float(Ls[(b0 + i) * nb + b0 + q], fmt), X[(b0 + q) * XS + c], acc);
                X[(b0 + i) * XS + c] = acc;
            }
        }
        __syncthreads();
        // round the block to u_f: stored factor, transposed operand, and the value used below
        for (int e = tid; e < wb * TB_COLS; e += 256) {
            int i = e / TB_COLS, c = e - i * TB_COLS;
            uint16_t u = float_to_uf(X[(b0 + i) * XS + c], fmt);
            float uv = uf_to_float(u, fmt);
            X[(b0 + i) * XS + c] = uv;
            if (c < width) {
                LUout[(r0 + b0 + i) * ldl + c0 + c] = u;
                W[(r0 + b0 + i) * ldw + c0 + c] = uv;
                UT[(c0 + c) * ldut + b0 + i] = u;
            }
        }
        __syncthreads();
        // rows below the block: X[i] -= L[i, b0:b0+wb] U_b
        const int rows_below = nb - (b0 + wb);
        for (int e = tid; e < rows_below * TB_COLS; e += 256) {
            int i = b0 + wb + e / TB_COLS, c = e % TB_COLS;
            float acc = 0.0f;
            for (int q = 0; q < wb; ++q) acc = fmaf(uf_to_float(Ls[i * nb + b0 + q], fmt), X[(b0 + q) * XS + c], acc);
            X[i * XS + c] -= acc;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ SIMT trailing update
// C[M x N] -= A[M x K] * B[K x N] with u_f operands (16-bit, row-major) and FP32 accumulation.
// 128 x 128 tile, BK = 16, 256 threads, 8 x 8 outputs per thread.
__global__ void __launch_bounds__(256) k_gemm_sub_simt(float* __restrict__ Cm, int64_t ldc,
                                                       const uint16_t* __restrict__ Am, int64_t lda,
                                                       const uint16_t* __restrict__ Bm, int64_t ldb, int M, int N,
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
            As[kk][mi] = (gm < M && gk < K) ? uf_to_float(Am[(int64_t)gm * lda + gk], fmt) : 0.0f;
            int kb = e >> 7, ni = e & 127;   // B: 16 k x 128 cols
            int gkb = k0 + kb, gn = n0 + ni;
            Bs[kb][ni] = (gkb < K && gn < N) ? uf_to_float(Bm[(int64_t)gkb * ldb + gn], fmt) : 0.0f;
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
static int debug_lu() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("GIR_DEBUG_LU");
        v = (e && e[0] == '1') ? 1 : 0;
    }
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

static gir_status gemm_sub(float* C, int64_t ldc, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb,
                           const uint16_t* Bt, int64_t ldbt, int64_t M, int64_t N, int64_t K, int fmt,
                           const LUPlan& plan, int* flags, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return GIR_OK;
    if (plan.use_tc && Bt && tc_gemm_supported(M, N, K, lda, ldbt, ldc)) {
        gir_status st = launch_tc_gemm_sub(C, ldc, A, lda, Bt, ldbt, M, N, K, fmt, flags, s);
        if (st != GIR_UNSUPPORTED) return st;
    }
    dim3 grid((unsigned)((N + 127) / 128), (unsigned)((M + 127) / 128));
    count_launch(), k_gemm_sub_simt<<<grid, 256, 0, s>>>(C, ldc, A, lda, B, ldb, (int)M, (int)N, (int)K, fmt);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

struct SwapScratch {
    int* plan = nullptr;   // 2 * 2 * PERM_MAXK ints
    int* count = nullptr;
};

static gir_status make_plan(const int* ipiv, int64_t k0, int64_t k1, int64_t n, const SwapScratch& sw, cudaStream_t s) {
    if (k1 - k0 > PERM_MAXK || n - k1 > PERM_MAXN) return GIR_UNSUPPORTED;
    size_t smem = (size_t)gmax<int64_t>(1, n - k1) * sizeof(int);
    count_launch(), k_swap_plan<<<1, 256, smem, s>>>(ipiv, k0, k1, sw.plan, sw.count);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

static gir_status permute_f32(float* W, int64_t ldw, int64_t col0, int64_t col1, int64_t maxrows, const SwapScratch& sw,
                              cudaStream_t s) {
    if (col1 <= col0) return GIR_OK;
    constexpr int CW = 32;
    size_t smem = (size_t)maxrows * CW * sizeof(float);
    count_launch(), k_permute_rows<float, CW><<<(unsigned)((col1 - col0 + CW - 1) / CW), 256, smem, s>>>(
        W, ldw, sw.plan, sw.count, col0, col1);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

static gir_status permute_u16(uint16_t* LU, int64_t ldl, int64_t col0, int64_t col1, int64_t maxrows,
                              const SwapScratch& sw, cudaStream_t s) {
    if (col1 <= col0) return GIR_OK;
    constexpr int CW = 64;
    size_t smem = (size_t)maxrows * CW * sizeof(uint16_t);
    count_launch(), k_permute_rows<uint16_t, CW><<<(unsigned)((col1 - col0 + CW - 1) / CW), 256, smem, s>>>(
        LU, ldl, sw.plan, sw.count, col0, col1);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

static gir_status launch_panel(float* W, int64_t ldw, int64_t c0, int64_t n, int wc, int* ipiv, int* flags,
                               const LUPlan& plan, cudaStream_t s) {
    const int64_t h = n - c0;
    // cluster size: smallest C such that the panel fits the shared-memory budget per CTA
    const int64_t budget = plan.panel_smem_budget;
    const int WC = plan.w;
    int64_t bytes_per_row = (int64_t)(WC + 1) * 4;  // padded rows (see k_panel)
    int C = (int)((h * bytes_per_row + budget - 1) / budget);
    if (C < 1) C = 1;
    if (C > plan.max_cluster) return GIR_UNSUPPORTED;
    int rpc = (int)((h + C - 1) / C);
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
        GIR_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_panel<32>, W, ldw, c0, n, wc, rpc, ipiv, flags));
    } else {
        GIR_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_panel<16>, W, ldw, c0, n, wc, rpc, ipiv, flags));
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
    }
    return launch_panel(W, ldw, 0, m, w, ipiv, flags, plan, s);
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
    const size_t max_smem = 200 * 1024;
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_panel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_panel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_panel<32>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_panel<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    plan.panel_smem_budget = 160 * 1024;
    plan.max_cluster = 16;
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_trsm_band, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TB_MAXNB * TB_MAXNB * 2 + TB_MAXNB * (TB_COLS + 1) * 4));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_swap_plan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(PERM_MAXN * sizeof(int))));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_permute_rows<float, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      2 * PERM_MAXK * 32 * (int)sizeof(float)));
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_permute_rows<uint16_t, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      2 * PERM_MAXK * 64 * (int)sizeof(uint16_t)));
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
    int g = (int)gmin<int64_t>((n * n + 255) / 256, 152 * 32);
    count_launch(), k_quantize<<<g, 256, 0, s>>>(A, n, lda, Rp, Sp, *mu, W, ldw, flags);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

// Look-ahead schedule: block k's trailing update is split into (a) the next block's columns,
// on the main stream, and (b) all later columns, on a side stream, so (b) runs while the next
// block's panels (a few SMs) are factored. Events keep every W update, row interchange and
// UT access ordered: (b)_k finishes before block k+1's end-of-block interchanges and (a)_{k+1}.
gir_status lu_factor(float* W, int64_t ldw, uint16_t* LU, int64_t ldl, int* ipiv, int64_t n, int fmt,
                     const LUPlan& plan, uint16_t* UT, int* flags, cudaStream_t s) {
    const int w = plan.w;
    const int NB = plan.nb;
    const int64_t ldut = NB;
    if (NB > PERM_MAXK || NB > TB_MAXNB) return GIR_UNSUPPORTED;
    SwapScratch sw;
    // side stream and events, released on every return path (work still queued completes first)
    struct Side {
        cudaStream_t s2 = nullptr;
        cudaEvent_t ev_swapped = nullptr, ev_b = nullptr;
        ~Side() {
            if (ev_swapped) cudaEventDestroy(ev_swapped);
            if (ev_b) cudaEventDestroy(ev_b);
            if (s2) cudaStreamDestroy(s2);
        }
    } side;
    cudaStream_t& s2 = side.s2;
    cudaEvent_t& ev_swapped = side.ev_swapped;
    cudaEvent_t& ev_b = side.ev_b;
    GIR_CUDA_TRY(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    GIR_CUDA_TRY(cudaEventCreateWithFlags(&ev_swapped, cudaEventDisableTiming));
    GIR_CUDA_TRY(cudaEventCreateWithFlags(&ev_b, cudaEventDisableTiming));
    GIR_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&sw.plan), 4 * PERM_MAXK * sizeof(int), s));
    GIR_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&sw.count), sizeof(int), s));
    bool b_pending = false;  // a (b) part is running on s2
    gir_status st = GIR_OK;
    auto trsm_band = [&](int64_t C0, int64_t NBc, int64_t col0, int64_t col1, cudaStream_t ss) {
        if (col1 <= col0) return;
        const size_t smem = (size_t)TB_MAXNB * TB_MAXNB * 2 + (size_t)NBc * (TB_COLS + 1) * 4;
        count_launch(), k_trsm_band<<<(unsigned)((col1 - col0 + TB_COLS - 1) / TB_COLS), 256, smem, ss>>>(
            LU, ldl, W, ldw, C0, (int)NBc, w, col0, col1, fmt, LU, UT, ldut);
    };
    for (int64_t C0 = 0; C0 < n && st == GIR_OK; C0 += NB) {
        const int64_t NBc = gmin<int64_t>(NB, n - C0);
        const int64_t Cend = C0 + NBc;
        for (int64_t c0 = C0; c0 < Cend; c0 += w) {
            const int wc = (int)gmin<int64_t>(w, Cend - c0);
            {
                int t_ = trace_begin(s);
                GIR_TRY(launch_panel(W, ldw, c0, n, wc, ipiv, flags, plan, s));
                trace_end(t_, "lu panel", s);
            }
            GIR_TRY(debug_check("panel", C0, c0, flags, s));
            int t_ = trace_begin(s);
            {
                int64_t tot = (n - c0) * wc;
                int g = (int)gmin<int64_t>((tot + 255) / 256, 152 * 8);
                count_launch(), k_store_panel<<<g, 256, 0, s>>>(W, ldw, LU, ldl, c0, wc, n, fmt);
            }
            GIR_TRY(make_plan(ipiv, c0, c0 + wc, n, sw, s));
            GIR_TRY(permute_f32(W, ldw, c0 + wc, Cend, 2 * wc, sw, s));
            GIR_TRY(permute_u16(LU, ldl, C0, c0, 2 * wc, sw, s));
            trace_end(t_, "lu store+swaps", s);
            if (c0 + wc < Cend) {
                int64_t ncols = Cend - (c0 + wc);
                t_ = trace_begin(s);
                count_launch(), k_trsm_rows<32><<<(unsigned)((ncols + 255) / 256), 256, 0, s>>>(LU, ldl, W, ldw, c0, wc,
                                                                                                 c0 + wc, Cend, fmt, LU,
                                                                                                 UT + (c0 - C0), ldut);
                trace_end(t_, "lu inner trsm", s);
                GIR_TRY(debug_check("inner trsm", C0, c0, flags, s));
                t_ = trace_begin(s);
                GIR_TRY(gemm_sub(W + (c0 + wc) * ldw + (c0 + wc), ldw, LU + (c0 + wc) * ldl + c0, ldl,
                                 LU + c0 * ldl + (c0 + wc), ldl, UT + (c0 + wc) * ldut + (c0 - C0), ldut,
                                 n - (c0 + wc), ncols, wc, fmt, plan, flags, s));
                trace_end(t_, "lu inner gemm", s);
                GIR_TRY(debug_check("inner gemm", C0, c0, flags, s));
            }
        }
        // the previous block's (b) part touches the trailing W columns and reads L rows of that
        // block: it must finish before this block's interchanges move those rows
        if (b_pending) {
            GIR_CUDA_TRY(cudaStreamWaitEvent(s, ev_b, 0));
            b_pending = false;
        }
        int t_ = trace_begin(s);
        GIR_TRY(make_plan(ipiv, C0, Cend, n, sw, s));
        GIR_TRY(permute_f32(W, ldw, Cend, n, 2 * NBc, sw, s));
        GIR_TRY(permute_u16(LU, ldl, 0, C0, 2 * NBc, sw, s));
        trace_end(t_, "lu outer swaps", s);
        if (Cend < n) {
            const int64_t ntr = n - Cend;
            const int64_t Ca = gmin<int64_t>(n, Cend + NB);  // (a): columns [Cend, Ca)
            // (a) on the main stream: the next block's columns
            t_ = trace_begin(s);
            trsm_band(C0, NBc, Cend, Ca, s);
            trace_end(t_, "lu outer trsm", s);
            GIR_TRY(debug_check("outer trsm a", C0, Cend, flags, s));
            t_ = trace_begin(s);
            GIR_TRY(gemm_sub(W + Cend * ldw + Cend, ldw, LU + Cend * ldl + C0, ldl, LU + C0 * ldl + Cend, ldl,
                             UT + Cend * ldut, ldut, ntr, Ca - Cend, NBc, fmt, plan, flags, s));
            trace_end(t_, "lu outer gemm", s);
            if (Ca < n) {
                // (b) on the side stream, after this block's interchanges
                GIR_CUDA_TRY(cudaEventRecord(ev_swapped, s));
                GIR_CUDA_TRY(cudaStreamWaitEvent(s2, ev_swapped, 0));
                int tb = trace_begin(s2);
                trsm_band(C0, NBc, Ca, n, s2);
                trace_end(tb, "lu outer trsm", s2);
                tb = trace_begin(s2);
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
    GIR_CUDA_TRY(cudaGetLastError());
    return st;
}

}  // namespace gir
