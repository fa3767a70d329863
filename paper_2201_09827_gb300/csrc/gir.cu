// C ABI and host orchestration of RGMRES-IR (Algorithm 4) with GCRO-DR (Algorithm 3).
//
// Every arithmetic step runs in the kernels of k_lu.cu (factorization), k_trsv.cu (M^-1),
// k_vec.cu (residual, A v, tall-skinny products) and k_small.cu (Givens, least squares,
// harmonic Ritz, QR). The host only sequences launches on the caller's stream and reads
// back a few scalars per Arnoldi step (convergence flag) and per refinement step (norms).
#include <atomic>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "gir_batch.cuh"
#include "gir_internal.cuh"
#include "k_lu.cuh"
#include "k_small.cuh"
#include "k_trsv.cuh"
#include "k_dd.cuh"
#include "trace.cuh"

using namespace gir;

namespace {

constexpr int KMAX = SM_KMAX;
constexpr int MMAX = SM_MMAX;

// device scalar slots
enum { SC_RINF = 0, SC_XINF, SC_BINF, SC_AINF, SC_NRM2, SC_ONE, SC_S, SC_OMEGA, SC_COUNT = 16 };

struct Recycle {
    double* U = nullptr;  // n x KMAX
    double* C = nullptr;  // n x KMAX
    int k = 0;
    bool c_valid = false;  // A~ U = C holds (set by every GCRO-DR exit)
};

}  // namespace

struct gir_handle {
    int64_t n = 0;
    gir_params p{};
    int fmt = FF_BF16;
    int round32 = 0;
    int rbasis = 0;          // store the Krylov and recycle basis vectors rounded to FP32 (u = FP32 or GIR_FLAG_BASIS_FP32)
    int dev = 0;
    // factors
    uint16_t* LU = nullptr;
    int64_t ldl = 0;
    int* ipiv = nullptr;
    double* R = nullptr;
    double* S = nullptr;
    double mu = 1.0;
    bool scaled = false;
    TrsvState trsv;
    // norms of A (cached per matrix pointer)
    const double* normA_ptr = nullptr;
    double normA = 0.0;
    const double* normAT_ptr = nullptr;
    double normAT = 0.0;
    // Krylov basis [C region (KMAX cols) | V (MMAX + 1 cols)], column-major, stride ldb
    double* Wb = nullptr;
    int64_t ldb = 0;
    Recycle fwd, adj;
    double* Ucur = nullptr;  // n x KMAX working U
    double* Ctmp = nullptr;  // n x KMAX
    double* Utmp = nullptr;  // n x KMAX
    double* vtmp = nullptr;  // n
    float* Ahi = nullptr;    // float-float split of A (A_hi + A_lo), n x ldf, for the Arnoldi products
    float* Alo = nullptr;
    int64_t ldf = 0;
    float* vsplit = nullptr;  // 2 * ldf
    double* r = nullptr;     // n (GCRO-DR residual)
    double* dvec = nullptr;  // n (GCRO-DR solution)
    double* cvec = nullptr;  // n (preconditioned rhs)
    double* rr = nullptr;    // n (refinement residual)
    double* scratch = nullptr;
    size_t scratch_len = 0;
    SmallState* st = nullptr;
    double* qh = nullptr;
    double* dsc = nullptr;   // device scalars
    int* dflags = nullptr;
    double* hsc = nullptr;   // pinned host mirror of dsc
    float ms_factor = 0.f;   // device time of the factorization, reported in every gir_info
    bool dd = false;         // u_a = double-double (the paper's u^2 for u = FP64)
    DdState ddst;            // buffers of the double-double operator
    double2* respart = nullptr;  // partial sums of the adjoint's double-double residual (u_r = dd, u_a != dd)
    int k_run = 0;           // recycle dimension in use (params k, or its_1 - 1 with GIR_FLAG_ADAPTIVE_K)
    bool k_open = false;     // GIR_FLAG_ADAPTIVE_K: k is fixed by the next first GMRES cycle
    SmallState* hst = nullptr;  // pinned host mirror of the SmallState header
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    LUPlan plan;
};

namespace {

gir_status dalloc(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return (e == cudaErrorMemoryAllocation) ? GIR_OOM : GIR_CUDA_ERROR;
    }
    return GIR_OK;
}

template <typename T>
gir_status dalloc_t(T** p, size_t count) {
    return dalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

// Handles and factorization temporaries come from the device's stream-ordered pool, which is
// told to keep freed memory (release threshold = max) so that repeated factorizations reuse
// it without new allocations from the CUDA driver.
gir_status pool_alloc(void** p, size_t bytes, cudaStream_t s) {
    static std::atomic<int> configured_dev{-1};
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev.load() != dev) {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
        configured_dev = dev;
    }
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return (e == cudaErrorMemoryAllocation) ? GIR_OOM : GIR_CUDA_ERROR;
    }
    return GIR_OK;
}

template <typename T>
gir_status pool_alloc_t(T** p, size_t count, cudaStream_t s) {
    return pool_alloc(reinterpret_cast<void**>(p), count * sizeof(T), s);
}

// Frees the handle's memory on stream s; the caller guarantees that no kernel that uses it is
// still queued anywhere else (free_handle synchronises the device for that).
void free_handle_on(gir_handle* h, cudaStream_t s) {
    if (!h) return;
    void* ptrs[] = {h->LU, h->ipiv, h->R, h->S, h->trsv.DL, h->trsv.DU, h->trsv.EL, h->trsv.EU, h->trsv.EUt, h->trsv.ELt, h->trsv.perm, h->trsv.z, h->trsv.y1,
                    h->trsv.y2, h->trsv.ticket_ctr, h->trsv.abort_flag, h->Wb, h->fwd.U, h->fwd.C,
                    h->adj.U, h->adj.C, h->Ucur, h->Ctmp, h->Utmp, h->vtmp, h->r, h->dvec, h->cvec, h->rr,
                    h->scratch, h->st, h->qh, h->dsc, h->dflags, h->Ahi, h->Alo, h->vsplit,
                    h->ddst.DL, h->ddst.DU, h->ddst.z, h->ddst.y1, h->ddst.y2, h->ddst.w, h->ddst.part,
                    h->ddst.ready, h->respart};
    for (void* q : ptrs)
        if (q) cudaFreeAsync(q, s);
    if (h->hsc) cudaFreeHost(h->hsc);
    if (h->hst) cudaFreeHost(h->hst);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    delete h;
}

void free_handle(gir_handle* h) {
    if (!h) return;
    cudaDeviceSynchronize();   // no kernel of any stream may still use the handle's memory
    free_handle_on(h, 0);
}

double unit_roundoff(gir_prec p) {
    switch (p) {
        case GIR_FP32: return 5.9604644775390625e-08;
        case GIR_FP64: return 1.1102230246251565e-16;
        default: return 1.1102230246251565e-16;
    }
}

gir_status validate(int64_t n, int64_t lda, const gir_params* p) {
    if (!p || n < 1 || lda < n) return GIR_INVALID_ARG;
    if (n > (int64_t)1 << 30) return GIR_INVALID_ARG;
    if (p->m < 1 || p->m > GIR_MAX_M) return GIR_INVALID_ARG;
    if (p->k < 0 || p->k >= p->m || p->k > GIR_MAX_K) return GIR_INVALID_ARG;
    if (p->imax < 0 || p->imax >= GIR_MAX_IR) return GIR_INVALID_ARG;
    if (!(p->tau >= 0.0)) return GIR_INVALID_ARG;
    if ((p->flags & ~(GIR_FLAG_AUTOTUNE | GIR_FLAG_CW_BERR | GIR_FLAG_SIR | GIR_FLAG_ADAPTIVE_K | GIR_FLAG_EIG_FP64 |
                      GIR_FLAG_BASIS_FP32 | GIR_FLAG_BATCH_STREAMS | GIR_FLAG_BATCH_PERSISTENT)) != 0)
        return GIR_INVALID_ARG;
    if (p->uf != GIR_BF16 && p->uf != GIR_FP16 && p->uf != GIR_FP8_E4M3) return GIR_UNSUPPORTED;
    if (p->u != GIR_FP64 && p->u != GIR_FP32) return GIR_UNSUPPORTED;
    if (p->ur != GIR_FP64 && p->ur != GIR_DD) return GIR_UNSUPPORTED;
    if (p->ua != GIR_FP64 && p->ua != GIR_DD) return GIR_UNSUPPORTED;
    if (p->carry_mode != 0 && p->carry_mode != 1) return GIR_INVALID_ARG;
    return GIR_OK;
}

// ---------------------------------------------------------------- small device kernels
__global__ void k_fill(double* x, int64_t n, double v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}
__global__ void k_round32(double* x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = (double)__double2float_rn(x[i]);
}
// x = fl_u(x + s d), s read from device memory
__global__ void k_axpy_dev(double* __restrict__ x, const double* __restrict__ d, const double* __restrict__ s,
                           int64_t n, int round32) {
    double a = *s;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = fma(a, d[i], x[i]);
        if (round32) v = (double)__double2float_rn(v);
        x[i] = v;
    }
}
// r = b - t (for the transposed residual)
__global__ void k_sub(const double* __restrict__ b, const double* __restrict__ t, double* __restrict__ r, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = b[i] - t[i];
}
// The recycle dimension of the next cycle close (set once the first cycle's length is known).
__global__ void k_set_ktarget(SmallState* st, int k) {
    if (threadIdx.x == 0) st->k_target = k;
}
// Initialise the small state for a new cycle: beta from device memory, tol, counters.
__global__ void k_cycle_init(SmallState* st, const double* beta, double tol, int kc, int first, int k, int m,
                             int eig64) {
    if (threadIdx.x != 0) return;
    st->eig64 = eig64;
    st->j = 0;
    st->kc = kc;
    st->converged = 0;
    st->breakdown = 0;
    st->knew = 0;
    st->first = first;
    st->k_target = k;
    st->m = m;
    st->beta = *beta;
    st->tol = tol;
    st->est = *beta;
    st->g[0] = *beta;
}
__global__ void k_u16_to_f32(const uint16_t* __restrict__ in, int64_t ldi, float* __restrict__ out, int64_t n,
                             int fmt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / n, j = e - i * n;
        out[e] = uf_to_float(in[i * ldi + j], fmt);
    }
}

int grid1(int64_t n) { return (int)gmin<int64_t>((n + 255) / 256, 2048); }

double* V(gir_handle* h, int j) { return h->Wb + (int64_t)(KMAX + j) * h->ldb; }
double* Cregion(gir_handle* h, int kc) { return h->Wb + (int64_t)(KMAX - kc) * h->ldb; }

#define ST_PTR(h, field) (reinterpret_cast<double*>(reinterpret_cast<char*>((h)->st) + offsetof(SmallState, field)))

gir_status read_header(gir_handle* h, cudaStream_t s) {
    GIR_CUDA_TRY(cudaMemcpyAsync(h->hst, h->st, offsetof(SmallState, cs), cudaMemcpyDeviceToHost, s));
    GIR_CUDA_TRY(cudaStreamSynchronize(s));
    return GIR_OK;
}

gir_status read_scalars(gir_handle* h, cudaStream_t s) {
    GIR_CUDA_TRY(cudaMemcpyAsync(h->hsc, h->dsc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    GIR_CUDA_TRY(cudaStreamSynchronize(s));
    return GIR_OK;
}

int read_flags(gir_handle* h, cudaStream_t s) {
    int f = 0;
    cudaMemcpyAsync(&h->hsc[SC_COUNT - 1], h->dflags, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    memcpy(&f, &h->hsc[SC_COUNT - 1], sizeof(int));
    return f;
}

gir_status flags_status(int f) {
    if (f & DEV_TIMEOUT) return GIR_TIMEOUT;
    if (f & DEV_NONFINITE) return GIR_NONFINITE;
    if (f & DEV_SINGULAR) return GIR_SINGULAR;
    return GIR_OK;
}

// w = M^-1 A v (trans: M^-T A^T v), rounded to u
// A v for the correction equation: float-float from the split of A for A~ = M^-1 A (the triangular
// solves are float-float too); FP64 for the transposed operator of the adjoint solve
// The product of A~ = M^-1 A: float-float (A_hi + A_lo) v, FP64 A^T v, or with u_a = dd the
// double-double product kept unrounded in ddst.w for the substitutions (w is then unused).
gir_status launch_op_gemv(gir_handle* h, const double* A, int64_t lda, const double* v, double* w, int trans,
                          cudaStream_t s) {
    if (h->dd) return gemv_dd(h->ddst, A, h->n, lda, v, trans, s);
    if (!trans) return launch_gemv_ff(h->Ahi, h->Alo, h->ldf, h->n, v, w, h->vsplit, s);
    return launch_gemv(A, h->n, lda, v, w, trans, h->scratch, s);
}

// M^-1 (or M^-T) applied to the output of launch_op_gemv
gir_status apply_minv_op(gir_handle* h, double* w, int trans, cudaStream_t s) {
    const double* R = h->scaled ? h->R : nullptr;
    const double* S = h->scaled ? h->S : nullptr;
    if (h->dd) return apply_minv_dd(h->ddst, h->trsv, nullptr, w, R, S, h->mu, trans, h->round32, h->dflags, s);
    return apply_minv(h->trsv, h->vtmp, w, R, S, h->mu, trans, h->round32, h->dflags, s);
}

gir_status apply_atilde(gir_handle* h, const double* A, int64_t lda, const double* v, double* w, int trans,
                        cudaStream_t s) {
    GIR_TRY(launch_op_gemv(h, A, lda, v, h->vtmp, trans, s));
    return apply_minv_op(h, w, trans, s);
}

gir_status apply_minv_h(gir_handle* h, const double* v, double* w, int trans, cudaStream_t s) {
    const double* R = h->scaled ? h->R : nullptr;
    const double* S = h->scaled ? h->S : nullptr;
    if (h->dd) return apply_minv_dd(h->ddst, h->trsv, v, w, R, S, h->mu, trans, h->round32, h->dflags, s);
    return apply_minv(h->trsv, v, w, R, S, h->mu, trans, h->round32, h->dflags, s);
}

// One Arnoldi step j of (I - C C^T) A~ with CGS2 (Algorithm 3: the Arnoldi process of each cycle; plain GMRES in the first).
gir_status arnoldi_step(gir_handle* h, const double* A, int64_t lda, int trans, int j, int kc, cudaStream_t s) {
    const int64_t n = h->n;
    double* vj = V(h, j);
    double* w = V(h, j + 1);
    { const char* ph_ = trans ? "gemv adjoint" : "gemv";
    int tslot_ = trace_begin(s, ph_);
    GIR_TRY(launch_op_gemv(h, A, lda, vj, h->vtmp, trans, s));
    trace_end(tslot_, ph_, s); }
    { int tslot_ = trace_begin(s, "minv");
    GIR_TRY(apply_minv_op(h, w, trans, s));
    trace_end(tslot_, "minv", s); }
    { int tslot_ = trace_begin(s, "cgs2+givens");
    double* basis = Cregion(h, kc);
    const int p = kc + j + 1;
    GIR_TRY(launch_gemm_tn(basis, h->ldb, p, w, h->ldb, 1, n, ST_PTR(h, s1), p, h->scratch, s));
    GIR_TRY(launch_gemm_nn(basis, h->ldb, p, ST_PTR(h, s1), p, 1, w, h->ldb, -1.0, 1.0, n, h->round32, s));
    GIR_TRY(launch_gemm_tn(basis, h->ldb, p, w, h->ldb, 1, n, ST_PTR(h, s2), p, h->scratch, s));
    GIR_TRY(launch_gemm_nn(basis, h->ldb, p, ST_PTR(h, s2), p, 1, w, h->ldb, -1.0, 1.0, n, h->round32, s));
    GIR_TRY(launch_norm2(w, n, ST_PTR(h, hnorm), h->scratch, s));
    GIR_TRY(launch_givens_step(h->st, s));
    GIR_TRY(launch_scale_by(w, n, ST_PTR(h, hnorm), 1, h->rbasis, s));
    trace_end(tslot_, "cgs2+givens", s); }
    return GIR_OK;
}

// Arnoldi steps of one cycle until convergence or `steps`; returns the number taken.
gir_status run_cycle(gir_handle* h, const double* A, int64_t lda, int trans, int kc, int first, double tol, int steps,
                     int* taken, cudaStream_t s) {
    // v_1 = r / ||r||  (||r|| is in dsc[SC_NRM2])
    GIR_CUDA_TRY(cudaMemcpyAsync(V(h, 0), h->r, h->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    GIR_TRY(launch_scale_by(V(h, 0), h->n, h->dsc + SC_NRM2, 1, h->rbasis, s));
    count_launch(), k_cycle_init<<<1, 32, 0, s>>>(h->st, h->dsc + SC_NRM2, tol, kc, first, h->k_run, h->p.m,
                                                   (h->p.flags & GIR_FLAG_EIG_FP64) ? 1 : 0);
    int j = 0;
    for (; j < steps; ++j) {
        GIR_TRY(arnoldi_step(h, A, lda, trans, j, kc, s));
        { int tslot_ = trace_begin(s, "step sync");
        GIR_TRY(read_header(h, s));
        trace_end(tslot_, "step sync", s); }
        if (h->hst->status) break;
        if (h->hst->converged) { ++j; break; }
    }
    *taken = j;
    return GIR_OK;
}

// GCRO-DR(m, k) for A~ d = c, d0 = 0 (Algorithm 3). rc: the recycle space (in/out).
gir_status gcrodr(gir_handle* h, const double* A, int64_t lda, int trans, Recycle& rc, const double* c, double* d,
                  int* its_out, int* carry_applies, int* cycles, int* converged, cudaStream_t s) {
    const int64_t n = h->n;
    const int m = h->p.m;
    int k = h->k_run;
    const int max_its = h->p.max_its > 0 ? h->p.max_its : 20 * m;
    const int r32 = h->round32;
    const int rb = h->rbasis;   // rounding of stored basis vectors (C, U, V)
    int its = 0;
    *carry_applies = 0;
    GIR_TRY(launch_norm2(c, n, h->dsc + SC_NRM2, h->scratch, s));
    GIR_TRY(read_scalars(h, s));
    const double normc = h->hsc[SC_NRM2];
    const double tol = h->p.tau * normc;
    GIR_CUDA_TRY(cudaMemsetAsync(d, 0, n * sizeof(double), s));
    if (normc == 0.0) {
        *its_out = 0;
        *converged = 1;
        return GIR_OK;
    }
    GIR_CUDA_TRY(cudaMemcpyAsync(h->r, c, n * sizeof(double), cudaMemcpyDeviceToDevice, s));

    int kc = (k > 0) ? rc.k : 0;
    if (kc > 0) {
        // active U in Ucur, C in the C region of the basis
        GIR_CUDA_TRY(cudaMemcpyAsync(h->Ucur, rc.U, (size_t)kc * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (h->p.carry_mode == 1 && rc.c_valid) {
            GIR_CUDA_TRY(
                cudaMemcpyAsync(Cregion(h, kc), rc.C, (size_t)kc * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        } else {
            // Z = A~ Y (Y = previous U_k), QR(Z) by Cholesky QR twice: C = Q, U = Y R^-1
            for (int i = 0; i < kc; ++i) GIR_TRY(apply_atilde(h, A, lda, h->Ucur + i * n, h->Ctmp + i * n, trans, s));
            *carry_applies = kc;
            GIR_TRY(launch_gemm_tn(h->Ctmp, n, kc, h->Ctmp, n, kc, n, ST_PTR(h, G2), kc, h->scratch, s));
            GIR_TRY(launch_chol_gram(h->st, kc, s));
            GIR_TRY(launch_gemm_nn(h->Ctmp, n, kc, ST_PTR(h, Ccoef), SM_LDG, kc, h->Utmp, n, 1.0, 0.0, n, 0, s));
            GIR_TRY(launch_gemm_tn(h->Utmp, n, kc, h->Utmp, n, kc, n, ST_PTR(h, G2), kc, h->scratch, s));
            GIR_TRY(launch_chol_gram(h->st, -kc, s));
            GIR_TRY(read_header(h, s));
            if (h->hst->knew == kc) {
                GIR_TRY(launch_gemm_nn(h->Utmp, n, kc, ST_PTR(h, Ccoef), SM_LDG, kc, Cregion(h, kc), h->ldb, 1.0, 0.0,
                                       n, rb, s));
                GIR_TRY(launch_gemm_nn(h->Ucur, n, kc, ST_PTR(h, Rinv), SM_KMAX, kc, h->Utmp, n, 1.0, 0.0, n, rb, s));
                GIR_CUDA_TRY(
                    cudaMemcpyAsync(h->Ucur, h->Utmp, (size_t)kc * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            } else {
                kc = 0;  // the Gram matrix lost definiteness: start again with a GMRES cycle
            }
        }
        if (kc > 0) {
            // d = U C^T r ; r = r - C C^T r
            GIR_TRY(launch_gemm_tn(Cregion(h, kc), h->ldb, kc, h->r, n, 1, n, ST_PTR(h, s1), kc, h->scratch, s));
            GIR_TRY(launch_gemm_nn(h->Ucur, n, kc, ST_PTR(h, s1), kc, 1, d, n, 1.0, 0.0, n, r32, s));
            GIR_TRY(launch_gemm_nn(Cregion(h, kc), h->ldb, kc, ST_PTR(h, s1), kc, 1, h->r, n, -1.0, 1.0, n, r32, s));
        }
    }
    int ncyc = 0;
    if (kc == 0) {
        // first cycle: GMRES(m) from v1 = r / ||r||, then the harmonic Ritz recycle space
        GIR_TRY(launch_norm2(h->r, n, h->dsc + SC_NRM2, h->scratch, s));
        int j = 0;
        GIR_TRY(run_cycle(h, A, lda, trans, 0, 1, tol, min(m, max_its), &j, s));
        its += j;
        ++ncyc;
        if (h->hst->status) return flags_status(h->hst->status | read_flags(h, s));
        if (h->k_open) {
            // Section 5: the fewest iterations came from recycling the whole first-step subspace,
            // k = its_1 - 1; it applies when the first GMRES cycle converged
            h->k_open = false;
            if (h->hst->converged && j >= 1) {
                h->k_run = k = min(j - 1, KMAX);
                count_launch(), k_set_ktarget<<<1, 32, 0, s>>>(h->st, k);
            }
        }
        { int tslot_ = trace_begin(s, "cycle close");
        GIR_TRY(launch_cycle_close(h->st, h->qh, s));
        trace_end(tslot_, "cycle close", s); }
        GIR_TRY(launch_gemm_nn(V(h, 0), h->ldb, j, ST_PTR(h, ycoef), j, 1, d, n, 1.0, 0.0, n, r32, s));
        GIR_TRY(launch_gemm_nn(V(h, 0), h->ldb, j + 1, ST_PTR(h, zcoef), j + 1, 1, h->r, n, 1.0, 0.0, n, r32, s));
        GIR_TRY(read_header(h, s));
        const int knew = h->hst->knew;
        if (knew > 0) {
            GIR_TRY(launch_gemm_nn(V(h, 0), h->ldb, j + 1, ST_PTR(h, Ccoef), SM_LDG, knew, Cregion(h, knew), h->ldb,
                                   1.0, 0.0, n, rb, s));
            GIR_TRY(launch_gemm_nn(V(h, 0), h->ldb, j, ST_PTR(h, Ucoef), SM_LDG, knew, h->Ucur, n, 1.0, 0.0, n, rb, s));
        }
        kc = knew;
    }
    GIR_TRY(launch_norm2(h->r, n, h->dsc + SC_NRM2, h->scratch, s));
    GIR_TRY(read_scalars(h, s));
    double rn = h->hsc[SC_NRM2];
    while (rn > tol && its < max_its) {
        if (!(rn == rn)) return GIR_NONFINITE;
        const int steps = max(1, min(m - kc, max_its - its));
        int j = 0;
        GIR_TRY(run_cycle(h, A, lda, trans, kc, 0, tol, steps, &j, s));
        its += j;
        ++ncyc;
        if (h->hst->status) return flags_status(h->hst->status | read_flags(h, s));
        if (kc > 0) {
            GIR_TRY(launch_gemm_tn(Cregion(h, kc), h->ldb, kc + j + 1, h->Ucur, n, kc, n, ST_PTR(h, WtU), SM_LDG,
                                   h->scratch, s));
            GIR_TRY(launch_gemm_tn(h->Ucur, n, kc, h->Ucur, n, kc, n, ST_PTR(h, UtU), kc, h->scratch, s));
        }
        { int tslot_ = trace_begin(s, "cycle close");
        GIR_TRY(launch_cycle_close(h->st, h->qh, s));
        trace_end(tslot_, "cycle close", s); }
        const int d_dim = kc + j;
        // d += [U V_j] ycoef ; r -= [C V_{j+1}] zcoef
        if (kc > 0) GIR_TRY(launch_gemm_nn(h->Ucur, n, kc, ST_PTR(h, ycoef), d_dim, 1, d, n, 1.0, 1.0, n, 0, s));
        GIR_TRY(launch_gemm_nn(V(h, 0), h->ldb, j, ST_PTR(h, ycoef) + kc, d_dim, 1, d, n, 1.0, 1.0, n, r32, s));
        GIR_TRY(launch_gemm_nn(Cregion(h, kc), h->ldb, kc + j + 1, ST_PTR(h, zcoef), d_dim + 1, 1, h->r, n, -1.0, 1.0,
                               n, r32, s));
        GIR_TRY(read_header(h, s));
        const int knew = (k > 0) ? h->hst->knew : 0;
        if (knew > 0) {
            // C_new = [C V_{j+1}] Ccoef -> Ctmp ; U_new = U Ucoef_top + V_j Ucoef_bot -> Utmp
            GIR_TRY(launch_gemm_nn(Cregion(h, kc), h->ldb, kc + j + 1, ST_PTR(h, Ccoef), SM_LDG, knew, h->Ctmp, n, 1.0,
                                   0.0, n, rb, s));
            GIR_TRY(launch_gemm_nn(V(h, 0), h->ldb, j, ST_PTR(h, Ucoef) + kc, SM_LDG, knew, h->Utmp, n, 1.0, 0.0, n, 0,
                                   s));
            if (kc > 0)
                GIR_TRY(launch_gemm_nn(h->Ucur, n, kc, ST_PTR(h, Ucoef), SM_LDG, knew, h->Utmp, n, 1.0, 1.0, n, 0, s));
            if (rb) count_launch(), k_round32<<<grid1((int64_t)knew * n), 256, 0, s>>>(h->Utmp, (int64_t)knew * n);
            GIR_CUDA_TRY(cudaMemcpyAsync(Cregion(h, knew), h->Ctmp, (size_t)knew * n * sizeof(double),
                                         cudaMemcpyDeviceToDevice, s));
            GIR_CUDA_TRY(
                cudaMemcpyAsync(h->Ucur, h->Utmp, (size_t)knew * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        kc = knew;
        GIR_TRY(launch_norm2(h->r, n, h->dsc + SC_NRM2, h->scratch, s));
        GIR_TRY(read_scalars(h, s));
        rn = h->hsc[SC_NRM2];
    }
    // keep the recycle space for the next system (Algorithm 3 ends with Y~ = U_k)
    rc.k = (k > 0) ? kc : 0;
    rc.c_valid = rc.k > 0;
    if (rc.k > 0) {
        GIR_CUDA_TRY(cudaMemcpyAsync(rc.U, h->Ucur, (size_t)rc.k * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        GIR_CUDA_TRY(
            cudaMemcpyAsync(rc.C, Cregion(h, rc.k), (size_t)rc.k * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    *its_out = its;
    *cycles += ncyc;
    *converged = (rn <= tol);
    if (!(rn == rn)) return GIR_NONFINITE;
    return GIR_OK;
}

// Refinement loop of Algorithm 4 (initial solve, then residual, correction and update); trans solves the adjoint system.
gir_status refine(gir_handle* h, const double* A, int64_t lda, const double* b, double* x, gir_info* info, int trans,
                  cudaStream_t s) {
    const int64_t n = h->n;
    gir_info loc;
    memset(&loc, 0, sizeof(loc));
    const int r32 = h->round32;
    Recycle& rc = trans ? h->adj : h->fwd;
    if (trans && h->adj.k == 0 && h->fwd.k > 0 && h->k_run > 0) {
        // seed the adjoint recycle space with the forward U_k (any Y~ is a valid start of Algorithm 3)
        h->adj.k = h->fwd.k;
        GIR_CUDA_TRY(cudaMemcpyAsync(h->adj.U, h->fwd.U, (size_t)h->fwd.k * n * sizeof(double), cudaMemcpyDeviceToDevice,
                                     s));
        // C is not yet consistent with U for the adjoint operator: the next carry is literal
        h->adj.c_valid = false;
    }
    cudaEventRecord(h->ev0, s);
    // norms of A (cached per matrix pointer) and b
    if (!trans && h->normA_ptr != A) {
        GIR_TRY(launch_matrix_norminf(A, n, lda, h->dsc + SC_AINF, h->scratch, s));
        GIR_TRY(read_scalars(h, s));
        h->normA = h->hsc[SC_AINF];
        h->normA_ptr = A;
    }
    GIR_TRY(launch_norminf(b, n, h->dsc + SC_BINF, s));
    // x0 = M^-1 b (Algorithm 4, initial solve), stored in u
    GIR_TRY(apply_minv_h(h, b, x, trans, s));
    const int imax = h->p.imax;
    double target = h->p.target_berr;
    if (target < 0.0) target = 2.0 * unit_roundoff(h->p.u);
    loc.status = GIR_NOT_CONVERGED;
    for (int i = 0; i <= GIR_MAX_IR; ++i) loc.cw_berr[i] = -1.0;
    loc.final_cw_berr = -1.0;
    const bool cw = (h->p.flags & GIR_FLAG_CW_BERR) && !trans;
    const bool sir = (h->p.flags & GIR_FLAG_SIR) != 0;
    for (int i = 0; i <= imax; ++i) {
        // r_i = b - A x_i in u_r (Algorithm 4, residual), stored in u
        { int tslot_ = trace_begin(s, "residual");
        if (!trans) {
            GIR_TRY(launch_residual(A, n, lda, x, b, h->rr, h->p.ur == GIR_DD, s, cw ? h->dsc + SC_OMEGA : nullptr));
        } else if (h->p.ur == GIR_DD) {
            GIR_TRY(residual_t_dd(A, n, lda, x, b, h->rr, h->dd ? h->ddst.part : h->respart, s));
        } else {
            GIR_TRY(launch_gemv(A, n, lda, x, h->vtmp, 1, h->scratch, s));
            count_launch(), k_sub<<<grid1(n), 256, 0, s>>>(b, h->vtmp, h->rr, n);
        }
        if (r32) count_launch(), k_round32<<<grid1(n), 256, 0, s>>>(h->rr, n);
        trace_end(tslot_, "residual", s); }
        GIR_TRY(launch_norminf(h->rr, n, h->dsc + SC_RINF, s));
        GIR_TRY(launch_norminf(x, n, h->dsc + SC_XINF, s));
        GIR_TRY(read_scalars(h, s));
        const double rinf = h->hsc[SC_RINF], xinf = h->hsc[SC_XINF], binf = h->hsc[SC_BINF];
        const double nA = trans ? h->normAT : h->normA;
        const double eta = rinf / (nA * xinf + binf);
        loc.berr[i] = eta;
        loc.final_berr = eta;
        const double omega = cw ? h->hsc[SC_OMEGA] : -1.0;
        loc.cw_berr[i] = omega;
        loc.final_cw_berr = omega;
        if (!(eta == eta) || !(xinf <= 1.7976931348623157e308)) {
            loc.status = GIR_NONFINITE;
            break;
        }
        if (eta <= target && (!cw || omega <= target)) {
            loc.status = GIR_OK;
            break;
        }
        if (i == imax) break;
        // r^ = fl_u(r / ||r||_inf) ; c = M^-1 r^ (right-hand side of the correction equation)
        GIR_TRY(launch_scale_by(h->rr, n, h->dsc + SC_RINF, 1, r32, s));
        int its = 0, capp = 0, conv = 0;
        if (sir) {
            // Algorithm 1: the correction by substitution with the factors, d = M^-1 r^
            GIR_TRY(apply_minv_h(h, h->rr, h->dvec, trans, s));
        } else {
            GIR_TRY(apply_minv_h(h, h->rr, h->cvec, trans, s));
            gir_status gs = gcrodr(h, A, lda, trans, rc, h->cvec, h->dvec, &its, &capp, &loc.cycles, &conv, s);
            if (gs != GIR_OK) {
                loc.status = gs;
                break;
            }
        }
        loc.its[i] = its;
        loc.carry_applies[i] = capp;
        loc.total_its += its;
        loc.ir_steps = i + 1;
        // x_{i+1} = fl_u(x_i + ||r_i||_inf d) (Algorithm 4, update)
        count_launch(), k_axpy_dev<<<grid1(n), 256, 0, s>>>(x, h->dvec, h->dsc + SC_RINF, n, r32);
    }
    cudaEventRecord(h->ev1, s);
    cudaEventSynchronize(h->ev1);
    cudaEventElapsedTime(&loc.ms_solve, h->ev0, h->ev1);
    {
        const char* e = getenv("GIR_TRACE");
        if (e && e[0] == '1') {
            static char buf[8192];
            gir_trace_report(buf, sizeof(buf));
            fprintf(stderr, "gir trace (phase, ms, calls):\n%s", buf);
        }
    }
    loc.k_eff = rc.k;
    int f = read_flags(h, s);
    if (f & (DEV_TIMEOUT | DEV_NONFINITE)) loc.status = flags_status(f);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) loc.status = GIR_CUDA_ERROR;
    if (info) {
        float mf = info->ms_factor;
        *info = loc;
        info->ms_factor = mf;
    }
    return loc.status;
}

// column sums of |A| (= ||A||_1 = ||A^T||_inf) ; one thread per column
__global__ void k_colabs(const double* __restrict__ A, int64_t n, int64_t lda, double* __restrict__ cs) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += fabs(A[i * lda + j]);
    cs[j] = s;
}

}  // namespace

void gir::release_handle_on(gir_handle* h, cudaStream_t s) { free_handle_on(h, s); }

// ====================================================================== C ABI
extern "C" {

const char* gir_status_string(gir_status s) {
    switch (s) {
        case GIR_OK: return "GIR_OK";
        case GIR_NOT_CONVERGED: return "GIR_NOT_CONVERGED";
        case GIR_SINGULAR: return "GIR_SINGULAR";
        case GIR_NONFINITE: return "GIR_NONFINITE";
        case GIR_INVALID_ARG: return "GIR_INVALID_ARG";
        case GIR_TIMEOUT: return "GIR_TIMEOUT";
        case GIR_CUDA_ERROR: return "GIR_CUDA_ERROR";
        case GIR_OOM: return "GIR_OOM";
        case GIR_UNSUPPORTED: return "GIR_UNSUPPORTED";
    }
    return "GIR_UNKNOWN";
}

int64_t gir_handle_n(const gir_handle* h) { return h ? h->n : 0; }

void gir_free(gir_handle* h) {
    if (h) cudaDeviceSynchronize();
    free_handle(h);
}

gir_status gir_factor(const double* A, int64_t n, int64_t lda, const gir_params* params, void* stream,
                      gir_handle** out) {
    if (!out || !A) return GIR_INVALID_ARG;
    *out = nullptr;
    GIR_TRY(validate(n, lda, params));
    cudaStream_t s = (cudaStream_t)stream;
    gir_handle* h = new (std::nothrow) gir_handle();
    if (!h) return GIR_OOM;
    h->n = n;
    h->p = *params;
    h->k_run = params->k;
    h->k_open = (params->flags & GIR_FLAG_ADAPTIVE_K) != 0;
    h->fmt = (params->uf == GIR_FP16) ? FF_FP16 : FF_BF16;
    h->round32 = (params->u == GIR_FP32);
    h->rbasis = h->round32 || (params->flags & GIR_FLAG_BASIS_FP32) != 0;
    h->scaled = (params->uf == GIR_FP16);
    h->dd = (params->ua == GIR_DD);
    cudaGetDevice(&h->dev);
    gir_status st = GIR_OK;
#define ALLOC(ptr, cnt)                                                             \
    do {                                                                            \
        st = pool_alloc_t(&(ptr), (size_t)(cnt), s);                                \
        if (st != GIR_OK) { free_handle(h); return st; }                            \
    } while (0)
    h->ldl = (n + 7) / 8 * 8;
    const int64_t ldw = (n + 7) / 8 * 8;
    ALLOC(h->LU, (size_t)n * h->ldl);
    ALLOC(h->ipiv, n);
    ALLOC(h->R, n);
    ALLOC(h->S, n);
    const int nblk = (int)((n + TRSV_BLOCK - 1) / TRSV_BLOCK);
    ALLOC(h->trsv.DL, (size_t)nblk * TRSV_BLOCK * TRSV_BLOCK);
    ALLOC(h->trsv.DU, (size_t)nblk * TRSV_BLOCK * TRSV_BLOCK);
    ALLOC(h->trsv.EL, (size_t)nblk * TRSV_BLOCK * TRSV_BLOCK);
    ALLOC(h->trsv.EU, (size_t)nblk * TRSV_BLOCK * TRSV_BLOCK);
    ALLOC(h->trsv.EUt, (size_t)nblk * TRSV_BLOCK * TRSV_BLOCK);
    ALLOC(h->trsv.ELt, (size_t)nblk * TRSV_BLOCK * TRSV_BLOCK);
    ALLOC(h->trsv.perm, n);
    ALLOC(h->trsv.z, n);
    ALLOC(h->trsv.y1, n);
    ALLOC(h->trsv.y2, n);
    ALLOC(h->trsv.ticket_ctr, 1);
    ALLOC(h->trsv.abort_flag, 1);
    h->ldb = (n + 1) / 2 * 2;
    ALLOC(h->Wb, (size_t)h->ldb * (KMAX + MMAX + 1));
    ALLOC(h->fwd.U, (size_t)n * KMAX);
    ALLOC(h->fwd.C, (size_t)n * KMAX);
    ALLOC(h->adj.U, (size_t)n * KMAX);
    ALLOC(h->adj.C, (size_t)n * KMAX);
    ALLOC(h->Ucur, (size_t)n * KMAX);
    ALLOC(h->Ctmp, (size_t)n * KMAX);
    ALLOC(h->Utmp, (size_t)n * KMAX);
    ALLOC(h->vtmp, n);
    h->ldf = (n + 3) / 4 * 4;
    if (h->dd) {
        DdState& d = h->ddst;
        d.nblk = (int)((n + DD_BLOCK - 1) / DD_BLOCK);
        ALLOC(d.DL, (size_t)d.nblk * DD_BLOCK * DD_BLOCK);
        ALLOC(d.DU, (size_t)d.nblk * DD_BLOCK * DD_BLOCK);
        ALLOC(d.z, n);
        ALLOC(d.y1, n);
        ALLOC(d.y2, n);
        ALLOC(d.w, n);
        ALLOC(d.part, dd_part_len(n));
        ALLOC(d.ready, d.nblk);
    } else {
        // the float-float split of A, used only by the float-float operator
        ALLOC(h->Ahi, (size_t)n * h->ldf);
        ALLOC(h->Alo, (size_t)n * h->ldf);
        ALLOC(h->vsplit, (size_t)2 * h->ldf);
    }
    if (params->ur == GIR_DD && !h->dd) ALLOC(h->respart, dd_part_len(n));
    ALLOC(h->r, n);
    ALLOC(h->dvec, n);
    ALLOC(h->cvec, n);
    ALLOC(h->rr, n);
    h->scratch_len = (size_t)gmax<int64_t>(((n + 255) / 256) * n, 1 << 20);
    ALLOC(h->scratch, h->scratch_len);
    {
        void* p = nullptr;
        st = pool_alloc(&p, sizeof(SmallState), s);
        if (st != GIR_OK) { free_handle(h); return st; }
        h->st = reinterpret_cast<SmallState*>(p);
    }
    ALLOC(h->qh, (size_t)SM_DMAX * SM_DMAX + (size_t)SM_DMAX * (KMAX + 2) + (size_t)(SM_DMAX + 1) * (KMAX + 2));
    ALLOC(h->dsc, SC_COUNT);
    ALLOC(h->dflags, 4);
    if (cudaMallocHost(&h->hsc, SC_COUNT * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&h->hst, sizeof(SmallState)) != cudaSuccess) {
        free_handle(h);
        return GIR_OOM;
    }
    cudaEventCreate(&h->ev0);
    cudaEventCreate(&h->ev1);
    {
        const char* e = getenv("GIR_TRACE");
        if (e && e[0] == '1' && !trace_on()) gir_trace_enable(1);
    }
    float* W = nullptr;
    unsigned long long* colmax = nullptr;
    uint16_t* UT = nullptr;
    st = lu_prepare(h->plan);
    if (params->uf == GIR_FP8_E4M3) {
        h->plan.fp8 = 1;     // block columns are the 128-wide scale tiles of the FP8 model
        h->plan.nb = 128;
    } else {
        const int nb = params->lu_nb > 0 ? params->lu_nb : tuned_lu_nb(n);
        if (nb > 0) h->plan.nb = (nb + h->plan.w - 1) / h->plan.w * h->plan.w;
    }
    if (st == GIR_OK) st = pool_alloc_t(&W, (size_t)n * ldw, s);
    if (st == GIR_OK) st = pool_alloc_t(&colmax, (size_t)n, s);
    if (st == GIR_OK) st = pool_alloc_t(&UT, (size_t)n * h->plan.nb + 64, s);
    if (st != GIR_OK) {
        if (W) cudaFreeAsync(W, s);
        if (colmax) cudaFreeAsync(colmax, s);
        if (UT) cudaFreeAsync(UT, s);
        free_handle(h);
        return st;
    }
    cudaMemsetAsync(h->dflags, 0, 4 * sizeof(int), s);
    cudaMemsetAsync(h->trsv.ticket_ctr, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(h->trsv.abort_flag, 0, sizeof(int), s);
    cudaMemsetAsync(h->st, 0, sizeof(SmallState), s);
    cudaMemsetAsync(h->Wb, 0, (size_t)h->ldb * (KMAX + MMAX + 1) * sizeof(double), s);
    count_launch(), k_fill<<<1, 32, 0, s>>>(h->dsc + SC_ONE, 1, 1.0);
    cudaEventRecord(h->ev0, s);
    if (st == GIR_OK) {
        double mu = 1.0;
        st = lu_scale_quantize(A, n, lda, params->uf, h->R, h->S, &mu, W, ldw, colmax, h->dflags, s);
        h->mu = mu;
    }
    // the float-float split of A for the correction solves, on a low-priority stream beside the
    // (latency-bound) factorization, on few CTAs so that the panel clusters still find free SMs
    cudaStream_t s_aux = nullptr;
    cudaEvent_t ev_aux = nullptr;
    if (st == GIR_OK && !h->dd) {
        int lo_prio = 0, hi_prio = 0;
        cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
        if (cudaStreamCreateWithPriority(&s_aux, cudaStreamNonBlocking, lo_prio) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev_aux, cudaEventDisableTiming) != cudaSuccess) {
            st = GIR_CUDA_ERROR;
        } else {
            cudaEventRecord(ev_aux, s);
            cudaStreamWaitEvent(s_aux, ev_aux, 0);
            st = launch_split_matrix(A, n, lda, h->Ahi, h->Alo, h->ldf, 24, s_aux);
            cudaEventRecord(ev_aux, s_aux);
        }
    }
    if (st == GIR_OK)
        st = lu_factor(W, ldw, h->LU, h->ldl, h->ipiv, h->trsv.perm, n, h->fmt, h->plan, UT, h->dflags, s);
    if (ev_aux) {
        cudaStreamWaitEvent(s, ev_aux, 0);
        cudaEventDestroy(ev_aux);
    }
    if (s_aux) cudaStreamDestroy(s_aux);
    if (st == GIR_OK) st = trsv_setup(h->trsv, h->LU, h->ldl, n, h->fmt, s);
    if (st == GIR_OK && h->dd) st = dd_setup(h->ddst, h->trsv, s);
    cudaFreeAsync(W, s);
    cudaFreeAsync(colmax, s);
    cudaFreeAsync(UT, s);
    cudaEventRecord(h->ev1, s);
    cudaEventSynchronize(h->ev1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    if (st == GIR_OK) {
        int f = read_flags(h, s);
        st = flags_status(f);
        if (cudaGetLastError() != cudaSuccess) st = GIR_CUDA_ERROR;
    }
    if (st != GIR_OK) {
        free_handle(h);
        return st;
    }
    h->ms_factor = ms;
    *out = h;
    return GIR_OK;
}

gir_status gir_solve(gir_handle* h, const double* A, int64_t lda, const double* b, double* x, gir_info* info,
                     void* stream) {
    if (!h || !A || !b || !x || lda < h->n) return GIR_INVALID_ARG;
    if (info) info->ms_factor = h->ms_factor;
    return refine(h, A, lda, b, x, info, 0, (cudaStream_t)stream);
}

gir_status gir_solve_adjoint(gir_handle* h, const double* A, int64_t lda, const double* g, double* lambda,
                             gir_info* info, void* stream) {
    if (!h || !A || !g || !lambda || lda < h->n) return GIR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->normAT_ptr != A) {
        count_launch(), k_colabs<<<(unsigned)((h->n + 255) / 256), 256, 0, s>>>(A, h->n, lda, h->vtmp);
        GIR_TRY(launch_norminf(h->vtmp, h->n, h->dsc + SC_AINF, s));
        GIR_TRY(read_scalars(h, s));
        h->normAT = h->hsc[SC_AINF];
        h->normAT_ptr = A;
    }
    if (info) info->ms_factor = h->ms_factor;
    return refine(h, A, lda, g, lambda, info, 1, s);
}

gir_status gir_residual(const double* A, int64_t n, int64_t lda, const double* x, const double* b, double* r,
                        gir_prec prec, void* stream) {
    if (!A || !x || !b || !r || n < 1 || lda < n) return GIR_INVALID_ARG;
    if (prec != GIR_FP64 && prec != GIR_DD) return GIR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    GIR_TRY(launch_residual(A, n, lda, x, b, r, prec == GIR_DD, s));
    GIR_CUDA_TRY(cudaStreamSynchronize(s));
    return GIR_OK;
}

gir_status gir_backward_errors(const double* A, int64_t n, int64_t lda, const double* x, const double* b,
                               gir_prec prec, double* eta, double* omega, void* stream) {
    if (!A || !x || !b || n < 1 || lda < n) return GIR_INVALID_ARG;
    if (prec != GIR_FP64 && prec != GIR_DD) return GIR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    // workspace: r (n) | row sums of |A| (n) | ||A||, ||x||, ||b||, ||r||, omega
    double* w = nullptr;
    GIR_TRY(dalloc_t(&w, (size_t)2 * n + 5));
    double* r = w;
    double* sc = w + 2 * n;
    gir_status st = launch_residual(A, n, lda, x, b, r, prec == GIR_DD, s, sc + 4);
    if (st == GIR_OK) st = launch_matrix_norminf(A, n, lda, sc + 0, w + n, s);
    if (st == GIR_OK) st = launch_norminf(x, n, sc + 1, s);
    if (st == GIR_OK) st = launch_norminf(b, n, sc + 2, s);
    if (st == GIR_OK) st = launch_norminf(r, n, sc + 3, s);
    double hs[5] = {0, 0, 0, 0, 0};
    if (st == GIR_OK && cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = GIR_CUDA_ERROR;
    if (cudaStreamSynchronize(s) != cudaSuccess && st == GIR_OK) st = GIR_CUDA_ERROR;
    cudaFree(w);
    if (st != GIR_OK) return st;
    if (eta) eta[0] = hs[3] / (hs[0] * hs[1] + hs[2]);
    if (omega) omega[0] = hs[4];
    return GIR_OK;
}

gir_status gir_gemv(const double* A, int64_t n, int64_t lda, const double* v, double* w, int trans, void* stream) {
    if (!A || !v || !w || n < 1 || lda < n) return GIR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double* scratch = nullptr;
    if (trans) GIR_TRY(dalloc_t(&scratch, (size_t)((n + 255) / 256) * n));
    gir_status st = launch_gemv(A, n, lda, v, w, trans, scratch, s);
    cudaStreamSynchronize(s);
    if (scratch) cudaFree(scratch);
    return st;
}

gir_status gir_adjoint_grad_a(const double* lambda, const double* x, int64_t n, double* dA, int64_t ldda,
                              void* stream) {
    if (!lambda || !x || !dA || n < 1 || ldda < n) return GIR_INVALID_ARG;
    return launch_outer(lambda, x, n, -1.0, dA, ldda, (cudaStream_t)stream);
}

gir_status gir_export_factors(const gir_handle* h, float* LU, int32_t* ipiv, double* R, double* S, double* mu,
                              void* stream) {
    if (!h) return GIR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = h->n;
    if (LU) count_launch(), k_u16_to_f32<<<grid1(n * n), 256, 0, s>>>(h->LU, h->ldl, LU, n, h->fmt);
    if (ipiv) GIR_CUDA_TRY(cudaMemcpyAsync(ipiv, h->ipiv, n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    if (R) {
        if (h->scaled) GIR_CUDA_TRY(cudaMemcpyAsync(R, h->R, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        else count_launch(), k_fill<<<grid1(n), 256, 0, s>>>(R, n, 1.0);
    }
    if (S) {
        if (h->scaled) GIR_CUDA_TRY(cudaMemcpyAsync(S, h->S, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        else count_launch(), k_fill<<<grid1(n), 256, 0, s>>>(S, n, 1.0);
    }
    if (mu) *mu = h->mu;
    GIR_CUDA_TRY(cudaStreamSynchronize(s));
    return GIR_OK;
}

gir_status gir_apply_minv(gir_handle* h, const double* v, double* w, int trans, void* stream) {
    if (!h || !v || !w) return GIR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    GIR_TRY(apply_minv_h(h, v, w, trans, s));
    GIR_CUDA_TRY(cudaStreamSynchronize(s));
    return flags_status(read_flags(h, s));
}

gir_status gir_apply_atilde(gir_handle* h, const double* A, int64_t lda, const double* v, double* w, int trans,
                            void* stream) {
    if (!h || !A || !v || !w || lda < h->n) return GIR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    GIR_TRY(apply_atilde(h, A, lda, v, w, trans, s));
    GIR_CUDA_TRY(cudaStreamSynchronize(s));
    return flags_status(read_flags(h, s));
}

gir_status gir_gcrodr(gir_handle* h, const double* A, int64_t lda, const double* c, double* d, int* its_out,
                      void* stream) {
    if (!h || !A || !c || !d || lda < h->n) return GIR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int its = 0, capp = 0, cyc = 0, conv = 0;
    gir_status st = gcrodr(h, A, lda, 0, h->fwd, c, d, &its, &capp, &cyc, &conv, s);
    cudaStreamSynchronize(s);
    if (its_out) *its_out = its;
    if (st != GIR_OK) return st;
    st = flags_status(read_flags(h, s));
    if (st != GIR_OK) return st;
    return conv ? GIR_OK : GIR_NOT_CONVERGED;
}

gir_status gir_export_recycle(const gir_handle* h, int adjoint, double* U, double* C, int kcap, int* k_out,
                              void* stream) {
    if (!h) return GIR_INVALID_ARG;
    const Recycle& rc = adjoint ? h->adj : h->fwd;
    cudaStream_t s = (cudaStream_t)stream;
    int k = rc.k < kcap ? rc.k : kcap;
    if (U && k > 0) GIR_CUDA_TRY(cudaMemcpyAsync(U, rc.U, (size_t)k * h->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (C && k > 0) GIR_CUDA_TRY(cudaMemcpyAsync(C, rc.C, (size_t)k * h->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    GIR_CUDA_TRY(cudaStreamSynchronize(s));
    if (k_out) *k_out = rc.k;
    return GIR_OK;
}

gir_status gir_reset_recycle(gir_handle* h) {
    if (!h) return GIR_INVALID_ARG;
    h->fwd.k = 0;
    h->adj.k = 0;
    return GIR_OK;
}

gir_status gir_small_eig(const double* M, int d, int k, int largest, int mcap, double* wr, double* wi, double* P,
                         int kcap, int* k_out, gir_prec eig_prec) {
    if (!M || !wr || !wi || !P || !k_out || d < 1 || d > SM_DMAX || k < 0 || k > kcap) return GIR_INVALID_ARG;
    if (eig_prec != GIR_FP32 && eig_prec != GIR_FP64) return GIR_INVALID_ARG;
    double *dM = nullptr, *dwr = nullptr, *dwi = nullptr, *dP = nullptr, *scr = nullptr;
    int* dk = nullptr;
    gir_status st = GIR_OK;
    if ((st = dalloc_t(&dM, (size_t)d * d)) != GIR_OK) return st;
    dalloc_t(&dwr, d);
    dalloc_t(&dwi, d);
    dalloc_t(&dP, (size_t)d * (kcap + 2));
    dalloc_t(&scr, (size_t)d * d);
    dalloc_t(&dk, 1);
    if (!dwr || !dwi || !dP || !scr || !dk) st = GIR_OOM;
    if (st == GIR_OK) {
        cudaMemcpy(dM, M, (size_t)d * d * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemset(dP, 0, (size_t)d * (kcap + 2) * sizeof(double));
        st = launch_small_eig(dM, d, k, largest, mcap, eig_prec == GIR_FP64, dwr, dwi, dP, kcap, dk, scr, 0);
        if (st == GIR_OK) {
            if (cudaDeviceSynchronize() != cudaSuccess) st = GIR_CUDA_ERROR;
        }
        if (st == GIR_OK) {
            int kk = 0;
            cudaMemcpy(&kk, dk, sizeof(int), cudaMemcpyDeviceToHost);
            int cols = kk < 0 ? -kk - 1 : kk;
            if (cols > kcap + 2) cols = kcap + 2;
            cudaMemcpy(wr, dwr, d * sizeof(double), cudaMemcpyDeviceToHost);
            cudaMemcpy(wi, dwi, d * sizeof(double), cudaMemcpyDeviceToHost);
            cudaMemcpy(P, dP, (size_t)d * (cols < kcap ? cols : kcap) * sizeof(double), cudaMemcpyDeviceToHost);
            *k_out = kk;
        }
    }
    cudaFree(dM);
    cudaFree(dwr);
    cudaFree(dwi);
    cudaFree(dP);
    cudaFree(scr);
    cudaFree(dk);
    return st;
}

gir_status gir_lu_panel(float* W, int64_t ldw, int64_t m, int w, int32_t* ipiv, int cluster, void* stream) {
    if (!W || !ipiv || m < 1 || w < 1 || w > 32 || ldw < w || m < w || cluster < 0 || cluster > 16)
        return GIR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int* flags = nullptr;
    GIR_TRY(dalloc_t(&flags, 1));
    cudaMemsetAsync(flags, 0, sizeof(int), s);
    gir_status st = lu_panel_only(W, ldw, m, w, ipiv, cluster, flags, s);
    int f = 0;
    if (st == GIR_OK) {
        if (cudaStreamSynchronize(s) != cudaSuccess) st = GIR_CUDA_ERROR;
        cudaMemcpy(&f, flags, sizeof(int), cudaMemcpyDeviceToHost);
        if (st == GIR_OK) st = flags_status(f);
    }
    cudaFree(flags);
    return st;
}

gir_status gir_lu_update(float* C, int64_t ldc, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb,
                         const uint16_t* Bt, int64_t ldbt, int64_t M, int64_t N, int64_t K, gir_prec fmt, int use_tc,
                         void* stream) {
    if (!C || !A || !B || !Bt || M < 0 || N < 0 || K < 0) return GIR_INVALID_ARG;
    if (fmt != GIR_BF16 && fmt != GIR_FP16) return GIR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    int* flags = nullptr;
    GIR_TRY(dalloc_t(&flags, 1));
    cudaMemsetAsync(flags, 0, sizeof(int), s);
    gir_status st = lu_update_only(C, ldc, A, lda, B, ldb, Bt, ldbt, M, N, K, fmt == GIR_BF16 ? FF_BF16 : FF_FP16,
                                   use_tc, flags, s);
    int f = 0;
    if (st == GIR_OK) {
        if (cudaStreamSynchronize(s) != cudaSuccess) st = GIR_CUDA_ERROR;
        cudaMemcpy(&f, flags, sizeof(int), cudaMemcpyDeviceToHost);
        if (st == GIR_OK) st = flags_status(f);
    }
    cudaFree(flags);
    return st;
}

}  // extern "C"
