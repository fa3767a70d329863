// Internal interface of the preconditioner application (k_trsv.cu).
#pragma once
#include "gir_internal.cuh"

namespace gir {

constexpr int TRSV_BLOCK = 64;

// Device buffers and counters of the persistent block triangular solves of one factorization.
struct TrsvState {
    int64_t n = 0;
    int nblk = 0;
    int fmt = 0;
    const uint16_t* LU = nullptr;
    int64_t ldl = 0;
    float2* DL = nullptr;            // inverses of the unit-lower diagonal blocks (float-float)
    float2* DU = nullptr;            // inverses of the upper diagonal blocks
    float2* EL = nullptr;            // DL[I] L[I, I-1] (float-float), the last step of the L solve
    float2* EU = nullptr;            // DU[I] U[I, I+1], the last step of the U solve
    float2* EUt = nullptr;           // DU[I]^T U[I-1, I]^T, the last step of the U^T solve (M^-T)
    float2* ELt = nullptr;           // DL[I]^T L[I+1, I]^T, the last step of the L^T solve
    bool et_ready = false;           // EUt, ELt hold the current factors (formed on first use)
    int* perm = nullptr;             // row permutation P (from the interchanges)
    double* z = nullptr;             // scaled/permuted input (FP64)
    float2* y1 = nullptr;            // intermediate and final solutions (float-float)
    float2* y2 = nullptr;
    unsigned long long* ticket_ctr = nullptr;
    int* abort_flag = nullptr;
    unsigned long long tickets = 0;  // host mirror of the ticket counter
    int calls = 0;
    int cluster = 16;                // CTAs per cluster of the forward solves (16, or 8 where 16 cannot run)
};

gir_status trsv_setup(TrsvState& st, const uint16_t* LU, int64_t ldl, int64_t n, int fmt, cudaStream_t s);
// out = fl_u(M^-1 w) (trans = 0) or fl_u(M^-T w) (trans = 1); out may alias w.
gir_status apply_minv(TrsvState& st, const double* w, double* out, const double* R, const double* S, double mu,
                      int trans, int round32, int* flags, cudaStream_t s);

}  // namespace gir
