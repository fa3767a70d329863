// Internal interface of the persistent batch kernel (k_persist.cu) for gir_batch_solve (batch.cu).
#pragma once
#include "gir_internal.cuh"

namespace gir {

// Largest order and restart length the persistent kernel takes (its per-CTA shared memory holds
// 16 n bytes of the triangular solves and the cycle end's (m+1) m workspace).
constexpr int64_t PERSIST_NMAX = 8192;
constexpr int PERSIST_MAX_M = 100;

// True if the persistent kernel implements these parameters and sizes: u_f BF16 or FP16, u_a
// float-float, no componentwise stop or SIR comparator, every n <= PERSIST_NMAX, m <= PERSIST_MAX_M,
// and GIR_FLAG_BATCH_STREAMS not set.
bool persistent_batch_supported(int nsys, const int64_t* n, const int64_t* lda, const gir_params* p);

// True if the persistent kernel's modelled makespan on this device does not exceed the worker
// streams' (the model and its GB300 constants are in gir.h, at gir_batch_solve).
bool persistent_batch_preferred(int nsys, const int64_t* n);

// The whole batch in one persistent launch (captured in a CUDA graph, launched on s); fills infos
// and returns the worst status. Synchronises s.
gir_status persistent_batch_solve(int nsys, const int64_t* n, const double* const* A, const int64_t* lda,
                                  const double* const* b, double* const* x, const gir_params* p, gir_info* infos,
                                  cudaStream_t s);

}  // namespace gir
