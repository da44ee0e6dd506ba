// Tiled scatter of the k-core incidence lists (CSR).
//
// After the degree histogram and its exclusive scan, vertex v's incidences go
// to inc[off[v] ..].  Scattering them with one global atomic per incidence on
// a cursor array of n vertices is bound by random atomics.  Here the
// incidences are sorted by vertex first, as the IBLT build sorts its updates:
//   k_vbin       one record (v, e) per incidence into the bin of v's slab of
//                2^21 vertices (per-block histogram, one atomic per slab per
//                block, runs written contiguously);
//   k_vtile_step launch s sorts slab s's records into 128 tiles of 2^14
//                vertices ("bin" role) while every tile of slab s-1 is
//                scattered with its 2^14 cursors in shared memory ("apply"
//                role: the cursors start at off[], each incidence takes the
//                next slot of its vertex, the final cursors go back to global
//                memory).  A tile whose list is full sends its extra records to
//                the slab's overflow list, which launch s + 2 scatters with
//                global atomics on the cursors the tiles left behind.
// The order of a vertex's incidences differs from the atomic scatter's, which
// is arbitrary too: nothing the peel computes depends on it.
#pragma once

#include "device.cuh"

namespace pp {

constexpr int kVSlabShift = 21;                              // 2^21 vertices per slab
constexpr u32 kVSlabVerts = 1u << kVSlabShift;
constexpr int kVTileShift = 14;                              // 2^14 vertices (64 KB of cursors) per tile
constexpr u32 kVTileVerts = 1u << kVTileShift;
constexpr u32 kVTilesPerSlab = kVSlabVerts >> kVTileShift;   // 128
constexpr int kVThreads = 512;
constexpr int kVBinEdges = 512;                              // edges per k_vbin step
constexpr int kVChunk = 4096;                                // records per bin-role step
constexpr int kVItems = kVChunk / kVThreads;                 // 8

struct VBinArgs {
  u32 *rec_v, *rec_e;   // slab-major, cap records per slab
  u32 *count;           // per slab
  u32 *overflow;        // set when a slab's list is full (the caller falls back)
  u32 cap;
  u32 n_slabs;
};

struct VTileArgs {
  u32 *tv, *te;         // tile-sorted records: two sets, set_stride apart
  u32 *tcount;          // per tile, two sets of kVTilesPerSlab
  u64 set_stride;       // kVTilesPerSlab * cap
  u32 cap;
  u32 o_cap;
  u32 *ov, *oe;         // overflow: three sets, o_cap apart
  u32 *o_count;         // per slab
};

// Dynamic shared memory: kVBinEdges * r records (v, e) + 3 * n_slabs u32.
__global__ void __launch_bounds__(kVThreads) k_vbin(const u32 *__restrict__ edges, u64 m, u32 r, u32 n,
                                                    VBinArgs b) {
  extern __shared__ __align__(16) unsigned char smem[];
  const u32 CAP = kVBinEdges * r;
  u32 *s_v = reinterpret_cast<u32 *>(smem);
  u32 *s_e = s_v + CAP;
  u32 *s_hist = s_e + CAP;
  u32 *s_scan = s_hist + b.n_slabs;
  u32 *s_base = s_scan + b.n_slabs;
  __shared__ u32 s_wt[kVThreads / 32];
  __shared__ u32 s_total;
  const u32 tid = threadIdx.x, ns = b.n_slabs;
  for (u64 e0 = (u64)blockIdx.x * kVBinEdges; e0 < m; e0 += (u64)gridDim.x * kVBinEdges) {
    for (u32 i = tid; i < ns; i += kVThreads) s_hist[i] = 0;
    __syncthreads();
    const u32 ne = (u32)(e0 + kVBinEdges <= m ? kVBinEdges : m - e0);
    // the block's incidences, row-major, coalesced; rank within the slab
    u32 v[kVBinEdges * PP_MAX_R / kVThreads], rk[kVBinEdges * PP_MAX_R / kVThreads];
#pragma unroll
    for (int it = 0; it < kVBinEdges * PP_MAX_R / kVThreads; ++it) {
      const u32 i = (u32)it * kVThreads + tid;
      v[it] = 0xffffffffu;
      rk[it] = 0;
      if (i < ne * r) {
        const u32 x = __ldcs(edges + e0 * r + i);
        if (x < n) {
          v[it] = x;
          rk[it] = atomicAdd(s_hist + (x >> kVSlabShift), 1u);
        }
      }
    }
    __syncthreads();
    const u32 per = (ns + kVThreads - 1) / kVThreads;
    const u32 lo = tid * per, hi = lo + per < ns ? lo + per : ns;
    u32 own = 0;
    for (u32 k = lo; k < hi; ++k) own += s_hist[k];
    u32 inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 y = __shfl_up_sync(kFull, inc, o);
      if ((int)lane_id() >= o) inc += y;
    }
    if (lane_id() == 31) s_wt[tid >> 5] = inc;
    __syncthreads();
    if (tid < 32) {
      const u32 w = tid < kVThreads / 32 ? s_wt[tid] : 0;
      u32 wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(kFull, wi, o);
        if ((int)tid >= o) wi += y;
      }
      if (tid < kVThreads / 32) s_wt[tid] = wi - w;
      if (tid == 31) s_total = wi;
    }
    __syncthreads();
    u32 run = s_wt[tid >> 5] + inc - own;
    for (u32 k = lo; k < hi; ++k) {
      s_scan[k] = run;
      const u32 h = s_hist[k];
      s_base[k] = h ? atomicAdd(b.count + k, h) : 0u;
      run += h;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kVBinEdges * PP_MAX_R / kVThreads; ++it) {
      if (v[it] != 0xffffffffu) {
        const u32 i = (u32)it * kVThreads + tid;
        const u32 pos = s_scan[v[it] >> kVSlabShift] + rk[it];
        s_v[pos] = v[it];
        s_e[pos] = (u32)(e0 + i / r);
      }
    }
    __syncthreads();
    const u32 total = s_total;
    for (u32 p = tid; p < total; p += kVThreads) {
      const u32 sl = s_v[p] >> kVSlabShift;
      const u32 slot = s_base[sl] + (p - s_scan[sl]);
      if (slot < b.cap) {
        const u64 dst = (u64)sl * b.cap + slot;
        b.rec_v[dst] = s_v[p];
        b.rec_e[dst] = s_e[p];
      } else {
        *b.overflow = 1u;
      }
    }
    __syncthreads();
  }
}

// Role "bin": slab `slab`'s records into its 128 tiles.
__device__ __forceinline__ void vtile_bin(unsigned char *smem, const VBinArgs &b, const VTileArgs &ta, u32 slab,
                                          u32 bi, u32 nb) {
  u32 *s_v = reinterpret_cast<u32 *>(smem);   // kVChunk
  u32 *s_e = s_v + kVChunk;                    // kVChunk
  __shared__ u32 s_hist[kVTilesPerSlab], s_scan[kVTilesPerSlab], s_base[kVTilesPerSlab];
  const u32 tid = threadIdx.x;
  const u64 keep = l2_evict_last_policy();
  const u32 set = slab & 1u;
  u32 *tv = ta.tv + set * ta.set_stride, *te = ta.te + set * ta.set_stride;
  u32 *tcount = ta.tcount + set * kVTilesPerSlab;
  const u64 oset = (u64)(slab % 3u) * ta.o_cap;
  const u32 cnt = b.count[slab];
  const u32 n = cnt < b.cap ? cnt : b.cap;
  const u64 src = (u64)slab * b.cap;
  const u32 vbase = slab << kVSlabShift;
  for (u32 c0 = bi * (u32)kVChunk; c0 < n; c0 += nb * (u32)kVChunk) {
    if (tid < kVTilesPerSlab) s_hist[tid] = 0;
    __syncthreads();
    const u32 c1 = c0 + kVChunk < n ? c0 + kVChunk : n;
    u32 v[kVItems], e[kVItems], rk[kVItems];
#pragma unroll
    for (int it = 0; it < kVItems; ++it) {
      const u32 i = c0 + (u32)it * kVThreads + tid;
      const bool ok = i < c1;
      v[it] = ok ? __ldcs(b.rec_v + src + i) : 0xffffffffu;
      e[it] = ok ? __ldcs(b.rec_e + src + i) : 0u;
    }
#pragma unroll
    for (int it = 0; it < kVItems; ++it)
      rk[it] = v[it] != 0xffffffffu ? atomicAdd(s_hist + ((v[it] - vbase) >> kVTileShift), 1u) : 0u;
    __syncthreads();
    if (tid < 32) {
      // 128 entries, 4 per lane
      u32 h[4], own = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) own += (h[q] = s_hist[tid * 4 + q]);
      u32 inc = own;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(kFull, inc, o);
        if ((int)tid >= o) inc += y;
      }
      u32 run = inc - own;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        s_scan[tid * 4 + q] = run;
        s_base[tid * 4 + q] = h[q] ? atomicAdd(tcount + tid * 4 + q, h[q]) : 0u;
        run += h[q];
      }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kVItems; ++it) {
      if (v[it] != 0xffffffffu) {
        const u32 pos = s_scan[(v[it] - vbase) >> kVTileShift] + rk[it];
        s_v[pos] = v[it];
        s_e[pos] = e[it];
      }
    }
    __syncthreads();
    for (u32 p = tid; p < c1 - c0; p += kVThreads) {
      const u32 tile = (s_v[p] - vbase) >> kVTileShift;
      const u32 slot = s_base[tile] + (p - s_scan[tile]);
      if (slot < ta.cap) {
        const u64 dst = (u64)tile * ta.cap + slot;
        st_l2_policy(tv + dst, s_v[p], keep);
        st_l2_policy(te + dst, s_e[p], keep);
      } else {
        const u32 q = atomicAdd(ta.o_count + slab, 1u);
        if (q < ta.o_cap) {
          ta.ov[oset + q] = s_v[p];
          ta.oe[oset + q] = s_e[p];
        }
      }
    }
    __syncthreads();
  }
}

// Role "apply": tile `tile` of slab `slab`, cursors in shared memory.
__device__ __forceinline__ void vtile_apply(unsigned char *smem, const VTileArgs &ta, u32 *cursor,
                                            u32 *__restrict__ inc, u32 slab, u32 tile, u32 n) {
  u32 *s_cur = reinterpret_cast<u32 *>(smem);  // kVTileVerts
  const u64 base = ((u64)slab << kVSlabShift) + ((u64)tile << kVTileShift);
  if (base >= n) return;  // uniform per block
  const u32 nv = (u32)(base + kVTileVerts <= n ? kVTileVerts : n - base);
  const u32 set = slab & 1u;
  const u64 src = set * ta.set_stride + (u64)tile * ta.cap;
  u32 *tcount = ta.tcount + set * kVTilesPerSlab;
  for (u32 i = threadIdx.x; i < nv; i += kVThreads) s_cur[i] = cursor[base + i];
  __syncthreads();
  const u32 cnt = tcount[tile];
  const u32 nr = cnt < ta.cap ? cnt : ta.cap;
  for (u32 i0 = 0; i0 < nr; i0 += kVThreads * kVItems) {
    u32 v[kVItems], e[kVItems];
#pragma unroll
    for (int it = 0; it < kVItems; ++it) {
      const u32 i = i0 + (u32)it * kVThreads + threadIdx.x;
      const bool ok = i < nr;
      v[it] = ok ? __ldcs(ta.tv + src + i) : 0xffffffffu;
      e[it] = ok ? __ldcs(ta.te + src + i) : 0u;
    }
#pragma unroll
    for (int it = 0; it < kVItems; ++it)
      if (v[it] != 0xffffffffu) inc[atomicAdd(s_cur + (u32)(v[it] - base), 1u)] = e[it];
  }
  __syncthreads();
  if (threadIdx.x == 0) tcount[tile] = 0;  // ready for slab + 2
  for (u32 i = threadIdx.x; i < nv; i += kVThreads) cursor[base + i] = s_cur[i];
  for (u32 l = threadIdx.x; l < (nr * 4 + 127) / 128; l += kVThreads) {
    l2_discard(ta.tv + src + l * 32);
    l2_discard(ta.te + src + l * 32);
  }
}

// Launch s (0 <= s <= n_slabs + 1): the overflow of slab s - 2 and the tiles of
// slab s - 1 (apply role, n_apply blocks), the sort of slab s (bin role,
// n_bin blocks), roles interleaved by block index.
__global__ void __launch_bounds__(kVThreads, 2) k_vtile_step(VBinArgs b, VTileArgs ta, u32 *cursor,
                                                             u32 *__restrict__ inc, u32 s, u32 n_apply,
                                                             u32 n_bin, u32 n) {
  extern __shared__ __align__(16) unsigned char smem[];
  const u32 both = n_apply < n_bin ? n_apply : n_bin;
  const u32 blk = blockIdx.x;
  bool apply;
  u32 idx;
  if (blk < 2 * both) {
    apply = (blk & 1u) == 0;
    idx = blk >> 1;
  } else {
    apply = n_apply > n_bin;
    idx = blk - both;
  }
  if (!apply) {
    vtile_bin(smem, b, ta, s, idx, n_bin);
    return;
  }
  if (s >= 2) {
    // the overflow of slab s - 2: its tiles wrote their cursors back in launch s - 1
    const u32 os = s - 2;
    const u64 oset = (u64)(os % 3u) * ta.o_cap;
    const u32 no = min(ta.o_count[os], ta.o_cap);
    for (u32 i = idx * kVThreads + threadIdx.x; i < no; i += n_apply * kVThreads)
      inc[atomicAdd(cursor + ta.ov[oset + i], 1u)] = ta.oe[oset + i];
  }
  if (s >= 1 && s - 1 < b.n_slabs) vtile_apply(smem, ta, cursor, inc, s - 1, idx, n);
}

}  // namespace pp
