/*
 * gir.h -- C ABI of the GB300 (sm_103a) recycled mixed-precision GMRES-IR solver.
 *
 * The method is RGMRES-IR (Oktay & Carson, "Mixed Precision GMRES-based Iterative
 * Refinement with Recycling", Algorithm 4): a low-precision (u_f) LU factorization with
 * partial pivoting, refinement steps whose residual r_i = b - A x_i is computed in
 * precision u_r, and a correction equation U^-1 L^-1 A d = U^-1 L^-1 r_i solved by
 * GCRO-DR(m, k) (Algorithm 3), whose recycle space U_k, C_k is carried from one
 * refinement step to the next. With k = 0 the same code is GMRES-IR (Algorithm 2).
 *
 * Conventions shared by every entry point:
 *  - Matrix and vector pointers are DEVICE pointers owned by the caller unless a
 *    parameter says otherwise; matrices are FP64, row-major, leading dimension lda >= n.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). All work
 *    is enqueued on it; entry points that return numbers to the host (gir_info, status)
 *    synchronise that stream before returning.
 *  - Errors are returned as gir_status, never thrown across the ABI. On any status other
 *    than GIR_OK / GIR_NOT_CONVERGED the output buffers are unspecified.
 *  - Not thread-safe per handle: one call at a time per gir_handle.
 */
#ifndef GIR_H
#define GIR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Precisions (Table 1; bf16 and fp8-e4m3 are the formats Section 3 mentions as
 * alternatives to the IEEE ones; GIR_DD is double-double, standing in for quad). */
typedef enum {
    GIR_FP64 = 0,
    GIR_FP32 = 1,
    GIR_FP16 = 2,
    GIR_BF16 = 3,
    GIR_FP8_E4M3 = 4,
    GIR_DD = 5
} gir_prec;

typedef enum {
    GIR_OK = 0,
    GIR_NOT_CONVERGED = 1,  /* i_max refinement steps without meeting the stop test (the paper's "-") */
    GIR_SINGULAR = 2,       /* a zero pivot in the u_f factorization */
    GIR_NONFINITE = 3,      /* Inf/NaN in the input, the factors or an iterate */
    GIR_INVALID_ARG = 4,
    GIR_TIMEOUT = 5,        /* a bounded device-side wait gave up (no hang) */
    GIR_CUDA_ERROR = 6,
    GIR_OOM = 7,
    GIR_UNSUPPORTED = 8     /* a precision combination this build does not implement */
} gir_status;

/* Arguments of Algorithm 4's "Require" line plus the readings the paper leaves open. */
typedef struct {
    gir_prec uf;        /* factorization precision u_f: GIR_FP16 (scaled), GIR_BF16, GIR_FP8_E4M3 */
    gir_prec u;         /* working precision u (storage of x, d, Krylov vectors): GIR_FP64 or GIR_FP32 */
    gir_prec ur;        /* residual precision u_r: GIR_FP64 or GIR_DD */
    gir_prec ua;        /* precision of the A~ = M^-1 A application: GIR_FP64 (float-float A v and
                           substitutions, about 2^-46: Section 4.3.1's uniform-precision reading
                           for u = FP64, u^2 for u = FP32) or GIR_DD (double-double product and
                           substitutions, about 2^-106: Algorithm 4's u^2 for u = FP64; ALU-bound
                           on GB300's FP64 units and several times slower) */
    int m;              /* GCRO-DR restart length (maximum subspace size), 1 <= m <= GIR_MAX_M */
    int k;              /* recycle dimension, 0 <= k < m; k = 0 gives GMRES-IR(m) */
    double tau;         /* inner tolerance on the relative preconditioned residual */
    int imax;           /* maximum number of refinement steps */
    double target_berr; /* stop when ||r||_inf / (||A||_inf ||x||_inf + ||b||_inf) <= target_berr;
                           a negative value selects 2*u; 0 runs exactly imax steps */
    int carry_mode;     /* 0: recompute QR(A~ Y~) at each new refinement step (the start of Algorithm 3);
                           1: reuse (U_k, C_k), which satisfy A~ U_k = C_k already */
    int max_its;        /* cap on Arnoldi steps per GCRO-DR call (<= 0: 20*m) */
    int lu_nb;          /* LU outer block width (<= 0: the tuned value for this size class, if
                           gir_autotune has measured one, else 256) */
    unsigned flags;     /* GIR_FLAG_* bits; other bits must be 0 */
} gir_params;

/* gir_batch_solve: measure (gir_autotune) the size classes of the batch that have no tuned
 * values yet before solving. */
#define GIR_FLAG_AUTOTUNE 0x1u
/* Also compute the componentwise backward error omega_i = max_j |r_j| / (|A||x_i| + |b|)_j of
 * every iterate (Table 2, middle column; fused into the residual pass, which then does one more
 * FP64 multiply-add per matrix entry) and stop only when eta_i and omega_i both meet
 * target_berr. Forward solves only: gir_solve_adjoint reports omega_i = -1. */
#define GIR_FLAG_CW_BERR 0x2u
/* Comparator: general iterative refinement (Algorithm 1, SIR) with the correction d = U^-1 L^-1 r
 * by substitution with the u_f factors (applied as M^-1 is for GCRO-DR), in place of GCRO-DR.
 * m, k, tau and carry_mode are ignored; its[i] = 0. */
#define GIR_FLAG_SIR 0x4u
/* Recycle dimension from the first refinement step (Section 5): when the first GMRES cycle of
 * the handle's first GCRO-DR call converges after its_1 steps, k becomes min(its_1 - 1,
 * GIR_MAX_K) -- the whole first-step subspace is recycled -- for that cycle's extraction and every
 * later step and solve. If that cycle does not converge, params.k stays. info.k_eff reports it. */
#define GIR_FLAG_ADAPTIVE_K 0x8u
/* Harmonic Ritz eigenvalues (Algorithm 3, the eigenproblems at the end of each cycle) by FP64
 * Hessenberg QR instead of the default FP32 one. The eigenvalues decide which k eigenvectors are
 * recycled and seed the FP64 inverse iteration that computes them; FP32 is enough unless
 * |theta| values within about 1e-6 relative of each other straddle the k-th place. The FP64
 * iteration takes several times longer on GB300 (its dependent FP64 chains). */
#define GIR_FLAG_EIG_FP64 0x10u
/* Low-precision basis storage inside GCRO-DR (Section 5 names mixed precision within the
 * recycling solver as future work): the Arnoldi vectors v_j and the recycle vectors C_k, U_k are
 * rounded to FP32 when they are formed; the vector being orthogonalised, d, r and all inner
 * products stay in u. The vectors are still held in FP64 arrays (the numerics of FP32 storage;
 * the halved basis traffic is not built). */
#define GIR_FLAG_BASIS_FP32 0x20u
/* gir_batch_solve only: run the batch on the pool of worker streams even where the persistent
 * kernel could take it (see gir_batch_solve). */
#define GIR_FLAG_BATCH_STREAMS 0x40u
/* gir_batch_solve only: run the batch as the persistent kernel whenever the kernel implements the
 * parameters and sizes (GIR_UNSUPPORTED otherwise), whatever the cost model below prefers. */
#define GIR_FLAG_BATCH_PERSISTENT 0x80u

#define GIR_MAX_M 112
#define GIR_MAX_K 64
#define GIR_MAX_IR 64

typedef struct {
    gir_status status;
    int ir_steps;               /* number of GCRO-DR calls (refinement steps) */
    int total_its;              /* sum of Arnoldi steps over all refinement steps */
    int its[GIR_MAX_IR];        /* Arnoldi steps per refinement step (the paper's per-step counts) */
    int carry_applies[GIR_MAX_IR];
    double berr[GIR_MAX_IR + 1];/* eta_i = ||r_i||_inf / (||A||_inf ||x_i||_inf + ||b||_inf), i = 0..ir_steps */
    double final_berr;
    int cycles;                 /* GCRO-DR restart cycles over all steps */
    int k_eff;                  /* recycle dimension at exit */
    float ms_factor;            /* device time of gir_factor (CUDA events) */
    float ms_solve;             /* device time of the refinement loop */
    double cw_berr[GIR_MAX_IR + 1]; /* omega_i with GIR_FLAG_CW_BERR (forward solves), else -1 */
    double final_cw_berr;
} gir_info;

typedef struct gir_handle gir_handle;

/* Algorithm 4, the factorization step: factor P (mu R A S) = L U in precision u_f with partial pivoting.
 * A: device, n x n row-major, lda >= n; read only, not retained.
 * Allocates the handle (factors, pivots, scalings, recycle space, workspaces); *out owns it.
 * Returns GIR_SINGULAR on a zero pivot, GIR_NONFINITE on overflow, GIR_OOM. Synchronises. */
gir_status gir_factor(const double* A, int64_t n, int64_t lda, const gir_params* params,
                      void* stream, gir_handle** out);

/* Algorithm 4 after the factorization: x0 = M^-1 b, then refinement steps with GCRO-DR corrections.
 * A: the same FP64 matrix that was factored (needed for the residual in u_r).
 * b: device n-vector; x: device n-vector (output). info: host struct (may be NULL).
 * The recycle space persists in the handle: later calls with new b start from it (Section 2).
 * Returns GIR_OK, GIR_NOT_CONVERGED (x holds the last iterate), GIR_NONFINITE, GIR_TIMEOUT. */
gir_status gir_solve(gir_handle* h, const double* A, int64_t lda, const double* b, double* x,
                     gir_info* info, void* stream);

/* Adjoint solve A^T lambda = g by the same refinement, left-preconditioned with M^T
 * (operator M^-T A^T), reusing the factors of gir_factor. Keeps its own recycle space,
 * seeded from the forward U_k when the adjoint one is empty. The residual g - A^T lambda is
 * computed in the handle's u_r (FP64, or double-double: exact products, dd sums). Not in the
 * paper (used for gradients: db = lambda, dA = -lambda x^T). Same arguments and statuses as
 * gir_solve. */
gir_status gir_solve_adjoint(gir_handle* h, const double* A, int64_t lda, const double* g,
                             double* lambda, gir_info* info, void* stream);

/* Batch of independent systems A_i x_i = b_i of different sizes n[i] (host array), each
 * solved by Algorithm 4 with its own factorization and recycle space. A, b, x: host arrays of
 * device pointers (lda: host array). infos: host array of nsys entries (may be NULL).
 * Two engines, same results up to rounding:
 *  - the persistent kernel (where it applies: u_f GIR_BF16 or GIR_FP16, ua GIR_FP64, neither
 *    GIR_FLAG_CW_BERR nor GIR_FLAG_SIR, every n <= 8192, m <= 100; chosen when a cost model of the
 *    two engines on GB300 prefers it, or forced by GIR_FLAG_BATCH_PERSISTENT): ONE kernel launch,
 *    captured in a CUDA graph that is launched on `stream`, whose CTAs (one per SM) take the
 *    systems from a device queue, largest n first, and each run all of Algorithm 4 on a system
 *    with no host round trip (the stop tests, restart sizes and recycle ranks are decided on the
 *    device). Its LU is the block-column model with 32-column panels (factors equal in model to
 *    gir_factor's, not bit for bit). The per-system ms_factor / ms_solve are device-clock
 *    intervals of the CTA that ran the system. Workspace: about 10 n_max^2 bytes per CTA, fewer
 *    CTAs if device memory is short;
 *    A CTA factors and solves its system alone, so a batch of few large systems is faster on the
 *    worker streams, where each system has the whole GPU. The cost model (gir_batch_engine)
 *    compares the kernel's makespan, max(T1(n_max), sum T1(n_i) / CTAs) with the one-CTA time
 *    T1(n) = 8.7e-9 n^3 + 1.8e-5 n^2 ms, against sum (2.1 + 4.0e-7 n_i^2) ms for the streams (both
 *    measured on GB300 for well-conditioned systems; iteration-heavy batches favour the kernel
 *    further);
 *  - the pool of worker streams (otherwise, or with GIR_FLAG_BATCH_STREAMS): each system through
 *    gir_factor + gir_solve on one of the worker streams (one host thread each); the pool size
 *    and each system's LU block width come from the autotuner's table (gir_autotune;
 *    GIR_FLAG_AUTOTUNE tunes missing size classes first) or from defaults.
 * Both start after the work already enqueued on `stream` and synchronise it. Returns GIR_OK,
 * else the worst status of a system (GIR_INVALID_ARG for invalid parameters). Not in the paper. */
gir_status gir_batch_solve(int nsys, const int64_t* n, const double* const* A, const int64_t* lda,
                           const double* const* b, double* const* x, const gir_params* params,
                           gir_info* infos, void* stream);

/* Which engine gir_batch_solve would use for these sizes (n, lda: host arrays of nsys entries) and
 * parameters: 1 = the persistent kernel, 0 = the worker-stream engine, -1 = nsys < 1, a NULL
 * pointer, or GIR_FLAG_BATCH_PERSISTENT for a batch the kernel cannot take. Host logic only (reads
 * the current device's SM count, 152 if there is no device; no allocation); does not validate the
 * parameters otherwise (gir_batch_solve reports GIR_INVALID_ARG). Not in the paper. */
int gir_batch_engine(int nsys, const int64_t* n, const int64_t* lda, const gir_params* params);

/* Autotuner (not in the paper). For each size class (n in (2^(c-1), 2^c]) of the count sizes in
 * n (host array), times gir_factor on a synthetic matrix of the class's largest order with LU
 * outer block widths 64, 128 and 256, and times a synthetic batch of factorizations of the
 * median size with 2, 4, 8 and 16 concurrent workers; the fastest choices go into a process-wide
 * table used by gir_factor (when params->lu_nb <= 0) and gir_batch_solve. Allocates temporary
 * device memory; synchronises. Classes already in the table are not measured again. */
gir_status gir_autotune(const int64_t* n, int count, void* stream);

/* Writes the tuned table as text lines ("class c: n <= N, lu_nb B, ms T" and "workers K") into
 * buf (host, buflen bytes, NUL-terminated) and returns the full length needed. */
int gir_tune_report(char* buf, int buflen);

/* Gradient of a loss L(x) of x = A^-1 b with respect to A, given lambda = A^-T dL/dx from
 * gir_solve_adjoint: dA = -lambda x^T (n x n, row-major, leading dimension ldda >= n). All
 * device pointers; enqueued on stream. Not in the paper (the differentiable-solve pattern). */
gir_status gir_adjoint_grad_a(const double* lambda, const double* x, int64_t n, double* dA, int64_t ldda,
                              void* stream);

void gir_free(gir_handle* h);
const char* gir_status_string(gir_status s);
int64_t gir_handle_n(const gir_handle* h);

/* ----- single steps of the hot path, exposed for parity testing and benchmarking ----- */

/* The residual of Algorithm 4: r = b - A x in precision prec (GIR_FP64 or GIR_DD), rounded to FP64.
 * All device pointers; r must not alias x or b. */
gir_status gir_residual(const double* A, int64_t n, int64_t lda, const double* x, const double* b,
                        double* r, gir_prec prec, void* stream);

/* Backward errors of an approximate solution x (the stop test of Algorithm 4 and the
 * two backward-error columns of Table 2): with r = b - A x in precision prec (GIR_FP64 or GIR_DD),
 *   *eta   = ||r||_inf / (||A||_inf ||x||_inf + ||b||_inf)          (normwise)
 *   *omega = max_i |r_i| / (|A| |x| + |b|)_i, with 0/0 = 0          (componentwise).
 * A, x, b: device (A n x n row-major, lda >= n); eta, omega: host, either may be NULL.
 * Allocates a small workspace; synchronises the stream. */
gir_status gir_backward_errors(const double* A, int64_t n, int64_t lda, const double* x, const double* b,
                               gir_prec prec, double* eta, double* omega, void* stream);

/* Failure-detection check of the bounded device waits: runs one block of a triangular solve
 * whose dependency is never published, so its wait gives up after spin_limit polls
 * (1 <= spin_limit <= 2e7; about 1e5 polls take a fraction of a second). Returns GIR_TIMEOUT when
 * the kernel reported the timeout and returned (the expected outcome; the context stays
 * usable), GIR_OK if it did not, GIR_INVALID_ARG or GIR_CUDA_ERROR. Synchronises the stream. */
gir_status gir_selftest_wait_timeout(long long spin_limit, void* stream);

/* w = A v (trans = 0) or w = A^T v (trans = 1) in FP64 arithmetic (device pointers). */
gir_status gir_gemv(const double* A, int64_t n, int64_t lda, const double* v, double* w,
                    int trans, void* stream);

/* Copy the factors out of a handle. LU: device n x n row-major float buffer receiving the
 * u_f values of L (strictly lower, unit diagonal implied) and U (upper, incl. diagonal);
 * ipiv: device int[n], rows k and ipiv[k] were interchanged at step k (0-based);
 * R, S: device double[n] scalings; mu: host double. Any pointer may be NULL. */
gir_status gir_export_factors(const gir_handle* h, float* LU, int32_t* ipiv, double* R, double* S,
                              double* mu, void* stream);

/* w = M^-1 v (trans = 0) or w = M^-T v (trans = 1), M^-1 = mu S U^-1 L^-1 P R (device pointers). */
gir_status gir_apply_minv(gir_handle* h, const double* v, double* w, int trans, void* stream);

/* w = M^-1 A v (trans = 0) or M^-T A^T v (trans = 1): one application of the preconditioned
 * operator of Algorithm 4's correction equation (device pointers). */
gir_status gir_apply_atilde(gir_handle* h, const double* A, int64_t lda, const double* v, double* w,
                            int trans, void* stream);

/* Algorithm 3 alone: d = GCRO-DR(m, k) solution of A~ d = c from d0 = 0, using and updating
 * the handle's recycle space (forward operator). its_out (host, may be NULL) receives the
 * number of Arnoldi steps; returns GIR_NOT_CONVERGED if max_its was reached. */
gir_status gir_gcrodr(gir_handle* h, const double* A, int64_t lda, const double* c, double* d,
                      int* its_out, void* stream);

/* Copy the recycle space out: U, C device n x kcap column-major (column stride n); returns
 * the current recycle dimension in *k_out (host). Forward (adjoint = 0) or adjoint space. */
gir_status gir_export_recycle(const gir_handle* h, int adjoint, double* U, double* C, int kcap,
                              int* k_out, void* stream);

/* Drop the recycle spaces held by the handle (the next solve starts with a GMRES cycle). */
gir_status gir_reset_recycle(gir_handle* h);

/* Eigenvalues and selected real eigenbasis of a small dense matrix by the single-block solver
 * used for the harmonic Ritz step (Algorithm 3, the eigenproblems at the end of each cycle):
 * FP64 Hessenberg reduction, eigenvalues by Hessenberg QR in eig_prec (GIR_FP32, the solver's
 * default, or GIR_FP64), eigenvectors by FP64 inverse iteration. M: host d x d column-major
 * (d <= GIR_MAX_M); wr, wi: host double[d] eigenvalues; P: host d x kcap column-major receiving
 * a real basis of the eigenvectors of the k eigenvalues of largest (largest != 0) or smallest
 * (largest == 0) magnitude with the conjugate-pair rule; *k_out receives the number of columns
 * written (-cols-1 if the QR iteration ran out of steps). Runs on the GPU; for testing. */
gir_status gir_small_eig(const double* M, int d, int k, int largest, int mcap, double* wr, double* wi,
                         double* P, int kcap, int* k_out, gir_prec eig_prec);

/* GEPP of one panel (Algorithm 4's factorization, the column-by-column pivot search): factor the
 * m x w FP32 block W (device, row-major, leading dimension ldw, w <= 32) in place with
 * partial pivoting in FP32 arithmetic; ipiv (device int[w]) receives the 0-based pivot rows.
 * cluster > 0 forces the number of cooperating CTAs (1..16), 0 chooses it from m.
 * Returns GIR_SINGULAR on a zero pivot. For testing the panel kernel in isolation. */
gir_status gir_lu_panel(float* W, int64_t ldw, int64_t m, int w, int32_t* ipiv, int cluster, void* stream);

/* Trailing update of the factorization: C -= A B with A (M x K, leading dimension lda) and
 * Bt = B^T (N x K, leading dimension ldbt) 16-bit u_f matrices (fmt GIR_BF16 or GIR_FP16,
 * row-major, K contiguous), B itself (K x N, leading dimension ldb) for the CUDA-core path,
 * C FP32 (M x N, ldc); exact products, FP32 accumulation. use_tc selects the tcgen05 tensor
 * core path (1) or CUDA cores (0). All device pointers. For testing the update in isolation. */
gir_status gir_lu_update(float* C, int64_t ldc, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb,
                         const uint16_t* Bt, int64_t ldbt, int64_t M, int64_t N, int64_t K, gir_prec fmt,
                         int use_tc, void* stream);

/* w = A^T v (FP64, device pointers, A row-major with leading dimension lda) for callers that
 * cannot allocate device memory when they call it (an allocator that forbids cudaMalloc in
 * a hot loop, a real-time loop, a fixed memory budget). The paper has no counterpart: this is
 * gir_gemv(trans = 1) with its scratch of partial sums taken from a fixed array in the
 * library's device image instead of cudaMalloc; the library allocates nothing in this call.
 * Limit: ceil(n / 256) * n <= 524288 scratch doubles, i.e. n <= 11520; larger n returns
 * GIR_INVALID_ARG with a message on stderr. The first call on each device looks up the
 * array's address (cudaGetSymbolAddress) with that device current, so make that first call
 * before any stream capture. All calls share the array: calls whose kernels could overlap on
 * the GPU (other streams, other host threads) race on it. Enqueued on `stream`; returns
 * before the kernels finish. Every GPU that loads the library keeps the 4 MiB array until exit.
 * A cudaDeviceReset invalidates the address looked up at the first call. */
gir_status gir_gemv_t_noalloc(const double* A, int64_t n, int64_t lda, const double* v, double* w,
                              void* stream);

/* Instrumentation (not in the paper). gir_trace_enable(1) records CUDA events on the
 * launching stream around each phase of the factorization and of the solve (no added
 * synchronisation); gir_trace_report writes "phase\tms\tcalls" lines into buf (host,
 * buflen bytes, NUL-terminated), clears the totals and returns the full length needed;
 * with buf == NULL it only returns the length and keeps the totals.
 * gir_launch_count returns the number of kernels this library has launched so far. */
void gir_trace_enable(int on);
int gir_trace_report(char* buf, int buflen);
/* Restrict the timing to the phases named in a comma-separated list (NULL or "": all phases).
 * Unselected phases record no events, so their launches run back to back as without timing. */
void gir_trace_select(const char* names);
unsigned long long gir_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* GIR_H */
