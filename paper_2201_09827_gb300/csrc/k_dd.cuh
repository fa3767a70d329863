// Internal interface of the double-double application of A~ = M^-1 A (k_dd.cu).
#pragma once
#include "gir_internal.cuh"
#include "k_trsv.cuh"

namespace gir {

constexpr int DD_BLOCK = 32;   // rows per block of the double-double triangular solves
constexpr int DD_TROWS = 256;  // rows per partial sum of the transposed product

// Buffers of the double-double operator of one factorization (allocated by the handle).
struct DdState {
    int nblk = 0;                 // ceil(n / DD_BLOCK)
    double2* DL = nullptr;        // inverses of the unit-lower diagonal blocks, double-double
    double2* DU = nullptr;        // inverses of the upper diagonal blocks
    double2* z = nullptr;         // scaled/permuted input
    double2* y1 = nullptr;        // intermediate and final solutions
    double2* y2 = nullptr;
    double2* w = nullptr;         // A v (or A^T v) before the substitutions
    double2* part = nullptr;      // partial sums of A^T v: ceil(n / DD_TROWS) x n
    int* ready = nullptr;         // per-block publication epochs of the solves
    int epoch = 0;
    int solo_smem = 0;            // dynamic shared memory of a solve CTA (one CTA per SM)
};

size_t dd_part_len(int64_t n);
// r = fl64(b - A^T x) with exact products and double-double sums (the adjoint residual in
// u_r = double-double); part: dd_part_len(n) double2 of scratch.
gir_status residual_t_dd(const double* A, int64_t n, int64_t lda, const double* x, const double* b, double* r,
                         double2* part, cudaStream_t s);
// Diagonal-block inverses of L and U in double-double (once per factorization).
gir_status dd_setup(DdState& dd, const TrsvState& st, cudaStream_t s);
// w = A v (trans = 0) or A^T v (trans = 1) with exact products and double-double sums.
gir_status gemv_dd(DdState& dd, const double* A, int64_t n, int64_t lda, const double* v, int trans, cudaStream_t s);
// out = fl_u(M^-1 w) (trans = 0) or fl_u(M^-T w) (trans = 1), every step in double-double.
// The input is dd.w when w64 is null, else the FP64 vector w64 (low part zero).
gir_status apply_minv_dd(DdState& dd, TrsvState& st, const double* w64, double* out, const double* R,
                         const double* S, double mu, int trans, int round32, int* flags, cudaStream_t s);

}  // namespace gir
