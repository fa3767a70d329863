// Phase timing hooks (trace.cu). Off unless gir_trace_enable(1) or GIR_TRACE=1.
#pragma once
#include <cuda_runtime.h>

namespace gir {
bool trace_on();
int trace_begin(cudaStream_t s, const char* name);
void trace_end(int slot, const char* name, cudaStream_t s);
// GIR_TRACE_DETAIL=1 (with tracing on): extra per-class phases for diagnosis
bool trace_detail();
// Adds a total measured elsewhere (device clocks of the persistent kernel) to the report.
void trace_add(const char* name, double ms, long long cnt);
}  // namespace gir
