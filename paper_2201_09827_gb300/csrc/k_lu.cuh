// Internal interface of the u_f LU (k_lu.cu) and its tensor-core trailing update (k_gemm_tc.cu).
#pragma once
#include "gir_internal.cuh"

namespace gir {

struct LUPlan {
    int w = 32;                       // panel width (one cluster factors w columns)
    int nb = 256;                     // outer block width (K of the big trailing update)
    int use_tc = 1;                   // tcgen05 trailing update when the shape allows it
    int64_t panel_smem_budget = 200 * 1024;  // panel rows held per CTA, bytes
    int max_cluster = 16;             // CTAs per panel cluster (non-portable size)
    int forced_cluster = 0;           // test hook: cluster size fixed by the budget alone
    int fp8 = 0;                      // FP8-E4M3 model: 128-wide FP32 block columns, operands
                                      // rounded per 128 x 128 tile (nb must be 128)
};

gir_status lu_prepare(LUPlan& plan);
gir_status lu_scale_quantize(const double* A, int64_t n, int64_t lda, int uf, double* R, double* S, double* mu,
                             float* W, int64_t ldw, unsigned long long* colmax, int* flags, cudaStream_t s);
// UT: scratch of n x plan.nb 16-bit elements (U12 transposed, K-major operand of the tensor-core update).
// perm (may be null): receives the row permutation, perm[i] = original row now at position i.
gir_status lu_factor(float* W, int64_t ldw, uint16_t* LU, int64_t ldl, int* ipiv, int* perm, int64_t n, int fmt,
                     const LUPlan& plan, uint16_t* UT, int* flags, cudaStream_t s);

// Test hooks: one panel factorization of an m x w FP32 block (rows 0..m) with a forced
// cluster size (0 = automatic), and one trailing update through the chosen path.
gir_status lu_panel_only(float* W, int64_t ldw, int64_t m, int w, int* ipiv, int cluster, int* flags, cudaStream_t s);
gir_status lu_update_only(float* C, int64_t ldc, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb,
                          const uint16_t* Bt, int64_t ldbt, int64_t M, int64_t N, int64_t K, int fmt, int use_tc,
                          int* flags, cudaStream_t s);

// tcgen05 trailing update C[M x N] (FP32) -= A[M x K] Bt[N x K]^T with 16-bit u_f operands,
// both K-major (row pitch lda / ldbt elements, multiples of 8).
bool tc_gemm_supported(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldbt, int64_t ldc);
gir_status launch_tc_gemm_sub(float* C, int64_t ldc, const uint16_t* A, int64_t lda, const uint16_t* Bt, int64_t ldbt,
                              int64_t M, int64_t N, int64_t K, int fmt, int* flags, cudaStream_t s);

}  // namespace gir
