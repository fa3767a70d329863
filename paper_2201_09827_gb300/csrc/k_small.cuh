// Internal interface of the small dense FP64 kernels of GCRO-DR (k_small.cu).
#pragma once
#include "gir_internal.cuh"

namespace gir {

constexpr int SM_MMAX = GIR_MAX_M;        // restart length cap
constexpr int SM_KMAX = GIR_MAX_K;        // recycle dimension cap
constexpr int SM_LDH = SM_MMAX + 1;       // leading dimension of H (column-major)
constexpr int SM_DMAX = SM_MMAX;          // kc + j <= m
constexpr int SM_LDG = SM_DMAX + 1;       // leading dimension of (d+1) x * matrices

// Device-resident state of one GCRO-DR solve (lives in global memory; one warp works on it).
struct SmallState {
    int j;              // Arnoldi steps taken in the current cycle
    int kc;             // recycle dimension of the current cycle
    int converged;      // Givens estimate <= tol
    int breakdown;      // h_{j+1,j} == 0
    int knew;           // recycle dimension produced by the last cycle end
    int status;         // bit mask of DEV_* flags
    int k_target;       // requested k
    int m;              // restart length
    int first;          // 1 in a first (plain GMRES) cycle
    int eig64;          // harmonic Ritz eigenvalues by FP64 (1) or FP32 (0) Hessenberg QR
    double beta;        // ||r|| at the cycle start
    double tol;         // tau * ||c||
    double est;         // Givens residual estimate |g_{j+1}|
    double hinv;        // 1 / h_{j+1,j} (0 on breakdown)
    double cs[SM_MMAX], sn[SM_MMAX], g[SM_MMAX + 1];
    double H[SM_LDH * SM_MMAX];         // Hessenberg H (j+1) x j, column-major ld SM_LDH
    double Hr[SM_LDH * SM_MMAX];        // H after the Givens rotations (upper triangular part)
    double B[SM_KMAX * SM_MMAX];        // B = C^T A~ V, column-major ld SM_KMAX
    double s1[SM_KMAX + SM_MMAX + 1];   // projection coefficients of the two CGS passes
    double s2[SM_KMAX + SM_MMAX + 1];
    double hnorm;                       // ||w|| after the second pass
    double dk[SM_KMAX];                 // D_k = diag(1 / ||u_i||)
    double WtU[SM_LDG * SM_KMAX];       // [C V_{j+1}]^T U, column-major ld SM_LDG
    double UtU[SM_KMAX * SM_KMAX];
    double ycoef[SM_KMAX + SM_MMAX];    // d += [U V_j] ycoef  (D folded into the U part)
    double zcoef[SM_KMAX + SM_MMAX + 1];// r -= [C V_{j+1}] zcoef  (first cycle: r = V_{j+1} zcoef)
    double Ccoef[SM_LDG * SM_KMAX];     // C_new = [C V_{j+1}] Ccoef, column-major ld SM_LDG
    double Ucoef[SM_LDG * SM_KMAX];     // U_new = [U V_j] Ucoef
    double Rinv[SM_KMAX * SM_KMAX];     // carry: R^-1 of QR(A~ Y)
    double G2[SM_KMAX * SM_KMAX];       // carry: Gram matrix
    double eig_wr[SM_DMAX], eig_wi[SM_DMAX];
};

// After the two CGS passes and the norm: assemble column j of H and B, apply Givens, update
// the estimate and convergence flag, and 1/h for the normalisation.
gir_status launch_givens_step(SmallState* st, cudaStream_t s);
// End of a cycle: least squares, residual/solution coefficients, harmonic Ritz vectors,
// QR(G P_k), coefficients of the new C_k and U_k. Uses Qh scratch (global, SM_DMAX^2 doubles).
gir_status launch_cycle_close(SmallState* st, double* qh_scratch, cudaStream_t s);
// Carry (Algorithm 3, the QR of A~ Y~ at the start) by Cholesky QR: from the Gram matrix G2 = Z^T Z (k x k)
// compute R (upper, chol) and Rinv; returns rank in st->knew.
gir_status launch_chol_gram(SmallState* st, int k, cudaStream_t s);
// w *= hinv (rounded to u): normalisation of the new Arnoldi vector.
gir_status launch_scale_by(double* w, int64_t n, const double* factor, int invert, int round32, cudaStream_t s);
// Standalone eigen-solver (testing): M d x d column-major in device memory.
gir_status launch_small_eig(const double* M, int d, int k, int largest, int mcap, int eig64, double* wr,
                            double* wi, double* P, int kcap, int* kout, double* scratch, cudaStream_t s);

}  // namespace gir
