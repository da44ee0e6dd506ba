#pragma once

#include <cuda_runtime.h>

#include "device.cuh"
#include "ppeel.h"

namespace pp {

// Bytes of temporary device memory exclusive_scan needs for n values.
size_t exclusive_scan_temp_bytes(u64 n);

// out[i] = in[0] + ... + in[i-1] for i = 0..n (out has n+1 entries).
pp_status exclusive_scan(const u32 *in, u32 *out, u64 n, void *temp, cudaStream_t s);

}  // namespace pp
