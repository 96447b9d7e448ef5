// internal.h -- host-side helpers shared by the C ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/giga.h"
#include "common.cuh"

namespace giga {

// Thread-local error detail; returns `status` for convenient `return fail(...)`.
giga_status_t fail(giga_status_t status, const std::string& detail);
giga_status_t cuda_fail(cudaError_t e, const char* where);
void clear_error();

// Autotuner (autotune.cu).
enum TuneOp { TUNE_FWD = 0, TUNE_BWD_INPUT = 1, TUNE_BWD_FILTER = 2, TUNE_BWD_FUSED = 3 };
int tune_mode();
int tune_candidates(int op);
DwConfig tune_config(int op, int id, const DwArgs& a);
// Cached choice for (op, problem class); -1 if none.
int tune_lookup(int op, const DwArgs& a);
void tune_store(int op, const DwArgs& a, int id);
// Run one depthwise op with candidate `id` (used by the autotuner).
giga_status_t run_dw_op(int op, const DwArgs& a, const DwConfig& cfg, cudaStream_t st);
// Benchmark all candidates of `op` on these buffers and store the fastest.
giga_status_t tune_dw_op(int op, const DwArgs& a, cudaStream_t st);
// GIGA_LOG is set (to anything but "0"): tuning decisions go to standard error.
bool tune_log_enabled();

// Dense 3 x 3, 64 -> 64 channel path (dense.cu).
size_t dense_workspace_bytes(bool input_grad);
cudaError_t dense_launch(const void* x, const void* w, void* y, int64_t N, int64_t H, int64_t W,
                         bool input_grad, void* ws, cudaStream_t st);
cudaError_t dense_take_error(cudaStream_t st, int* code);
size_t dense_filter_workspace_bytes();
cudaError_t dense_wgrad_launch(const void* x, const void* dy, float* dw, int64_t N, int64_t H,
                               int64_t W, void* ws, cudaStream_t st);

}  // namespace giga
