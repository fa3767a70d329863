// Internal interface between the solver's C ABI (gir.cu) and the batch scheduler and
// autotuner (batch.cu).
#pragma once
#include "gir_internal.cuh"

struct gir_handle;

namespace gir {

// LU outer block width measured for the size class of order n, or 0 if none was measured.
int tuned_lu_nb(int64_t n);

// Frees a handle whose work has completed on stream s, without a device-wide synchronisation.
void release_handle_on(gir_handle* h, cudaStream_t s);

}  // namespace gir
