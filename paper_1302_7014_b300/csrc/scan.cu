// Device-wide exclusive prefix sum of uint32 (used to turn vertex degrees into
// incidence-list offsets).  Tiles of 4096 values: per-tile sums, a recursive
// scan of the sums, then a per-tile scan with the tile's offset added.
#include "host.cuh"
#include "scan.cuh"

namespace pp {

namespace {

constexpr int kScanBlock = 1024;
constexpr int kPer = 4;
constexpr u64 kTile = (u64)kScanBlock * kPer;

__device__ __forceinline__ u32 block_exclusive(u32 v, u32 *warp_tot, u32 &total) {
  const u32 lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  u32 inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 y = __shfl_up_sync(kFull, inc, o);
    if (lane >= (u32)o) inc += y;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    u32 w = lane < kScanBlock / 32 ? warp_tot[lane] : 0;
    u32 wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 y = __shfl_up_sync(kFull, wi, o);
      if (lane >= (u32)o) wi += y;
    }
    if (lane < kScanBlock / 32) warp_tot[lane] = wi - w;
    if (lane == 31) warp_tot[32] = wi;
  }
  __syncthreads();
  total = warp_tot[32];
  const u32 r = warp_tot[warp] + inc - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanBlock) k_tile_sums(const u32 *__restrict__ in, u64 n,
                                                          u32 *__restrict__ sums) {
  __shared__ u32 wt[33];
  const u64 base = (u64)blockIdx.x * kTile + (u64)threadIdx.x * kPer;
  u32 s = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j)
    if (base + j < n) s += in[base + j];
  u32 total;
  block_exclusive(s, wt, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanBlock) k_tile_scan(const u32 *__restrict__ in, u64 n,
                                                          const u32 *__restrict__ tile_off,
                                                          u32 *__restrict__ out) {
  __shared__ u32 wt[33];
  const u64 base = (u64)blockIdx.x * kTile + (u64)threadIdx.x * kPer;
  u32 v[kPer];
  u32 s = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    v[j] = base + j < n ? in[base + j] : 0u;
    s += v[j];
  }
  u32 total;
  u32 run = block_exclusive(s, wt, total) + (tile_off ? tile_off[blockIdx.x] : 0u);
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    if (base + j < n) {
      out[base + j] = run;
      if (base + j == n - 1) out[n] = run + v[j];
    }
    run += v[j];
  }
}

}  // namespace

size_t exclusive_scan_temp_bytes(u64 n) {
  size_t b = 0;
  while (n > kTile) {
    n = (n + kTile - 1) / kTile;
    b += 2 * (n + 1) * sizeof(u32) + 256;
  }
  return b + 256;
}

pp_status exclusive_scan(const u32 *in, u32 *out, u64 n, void *temp, cudaStream_t s) {
  if (n == 0) {
    PP_CUDA(cudaMemsetAsync(out, 0, sizeof(u32), s));
    return PP_OK;
  }
  const u64 tiles = (n + kTile - 1) / kTile;
  if (tiles == 1) {
    k_tile_scan<<<1, kScanBlock, 0, s>>>(in, n, nullptr, out);
    PP_CUDA(cudaGetLastError());
    return PP_OK;
  }
  u32 *sums = static_cast<u32 *>(temp);
  u32 *sums_scan = sums + tiles + 1;
  char *next = reinterpret_cast<char *>(sums_scan + tiles + 1);
  next += (256 - ((uintptr_t)next & 255)) & 255;
  k_tile_sums<<<(unsigned)tiles, kScanBlock, 0, s>>>(in, n, sums);
  PP_CUDA(cudaGetLastError());
  pp_status st = exclusive_scan(sums, sums_scan, tiles, next, s);
  if (st != PP_OK) return st;
  k_tile_scan<<<(unsigned)tiles, kScanBlock, 0, s>>>(in, n, sums_scan, out);
  PP_CUDA(cudaGetLastError());
  return PP_OK;
}

}  // namespace pp
