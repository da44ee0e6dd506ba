// Host-side helpers shared by the C-ABI entry points.
#pragma once

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "device.cuh"
#include "ppeel.h"

namespace pp {

void set_error(const char *fmt, ...);
pp_status fail(pp_status s, const char *fmt, ...);
pp_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define PP_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return ::pp::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

// Multiprocessors of the current device.
int sm_count();

// Options with defaults filled in.
pp_options resolve_options(const pp_options *opt);

// Per-table constants: seeds s_0..s_r are SplitMix64 outputs 1..r+1 from
// `seed`; sub-table j holds floor(n/r) + [j < n mod r] cells.
void make_table_args(TableArgs &a, uint64_t n_cells, uint32_t r, uint64_t seed, uint32_t base);

// cudaStream_t from the ABI's void*.
inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Grid of a persistent kernel: resident CTAs per SM x SMs (at least 1 per SM).
int persistent_grid(const void *fn, int block, size_t smem, uint32_t ctas_per_sm);

// Lets fn take as much dynamic shared memory as the device allows a block
// beside fn's static shared memory.
void allow_max_dynamic_smem(const void *fn);

}  // namespace pp
