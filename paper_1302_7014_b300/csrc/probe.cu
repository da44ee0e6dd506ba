// Measurement helper: the rate of scattered whole-cell accesses (pp_probe_scatter).
//
// The IBLT rounds touch cells at random: a recovered key reads and writes
// 32-byte cells spread over a table far larger than L2.  This kernel does the
// same accesses with nothing else around them -- for each index, a 256-bit
// load of the cell, a 256-bit store of it, or both -- so that the decode's
// speed can be set against what the memory system gives for that pattern.
#include "host.cuh"

using namespace pp;

namespace {

constexpr int kProbeBlock = 256;
constexpr int kProbePer = 8;   // indices per thread in flight

__global__ void __launch_bounds__(kProbeBlock) k_probe(Cell *__restrict__ cells, u64 n_cells,
                                                       const u32 *__restrict__ idx, u64 m, int mode,
                                                       u64 *__restrict__ sink) {
  u64 acc = 0;
  const u64 stride = (u64)gridDim.x * kProbeBlock * kProbePer;
  for (u64 b = (u64)blockIdx.x * kProbeBlock * kProbePer + threadIdx.x; b < m; b += stride) {
    u32 c[kProbePer];
    bool v[kProbePer];
#pragma unroll
    for (int k = 0; k < kProbePer; ++k) {
      const u64 i = b + (u64)k * kProbeBlock;
      c[k] = i < m ? __ldcs(idx + i) : 0u;
      v[k] = i < m && c[k] < n_cells;  // an index past the table is skipped
    }
    u64 key[kProbePer], chk[kProbePer];
    int cnt[kProbePer];
#pragma unroll
    for (int k = 0; k < kProbePer; ++k) {
      key[k] = chk[k] = c[k];
      cnt[k] = 1;
      if (v[k] && mode != 2) ld_cell_cg(cells + c[k], key[k], chk[k], cnt[k]);
    }
#pragma unroll
    for (int k = 0; k < kProbePer; ++k) {
      if (!v[k]) continue;
      if (mode == 1) acc += key[k] ^ chk[k] ^ (u64)cnt[k];
      else st_cell_cs(cells + c[k], key[k] ^ 1ull, chk[k], cnt[k] - 1);
    }
  }
  if (acc == 0x5bd1e995ull) *sink = acc;  // keeps the loads of mode 1 alive
}

}  // namespace

extern "C" pp_status pp_probe_scatter(pp_cell *d_cells, uint64_t n_cells, const uint32_t *d_idx, uint64_t m, int mode,
                                      void *stream) {
  if (!d_cells || (m && !d_idx) || mode < 0 || mode > 2)
    return fail(PP_ERR_INVALID_ARG, "pp_probe_scatter: NULL pointer or mode outside 0..2");
  if (reinterpret_cast<uintptr_t>(d_cells) % 32 != 0)
    return fail(PP_ERR_INVALID_ARG, "pp_probe_scatter: cells must be 32-byte aligned");
  if (m == 0) return PP_OK;
  cudaStream_t s = as_stream(stream);
  const int grid = sm_count() * 8;
  u64 *sink = reinterpret_cast<u64 *>(d_cells);  // never written: acc cannot reach the marker
  k_probe<<<grid, kProbeBlock, 0, s>>>(reinterpret_cast<Cell *>(d_cells), n_cells, d_idx, m, mode, sink);
  PP_CUDA(cudaGetLastError());
  return PP_OK;
}
