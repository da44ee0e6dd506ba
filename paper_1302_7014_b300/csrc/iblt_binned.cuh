// Slab-binned IBLT build.
//
// Random cell updates spread over a table much larger than L2 run at the rate
// at which HBM can open rows for scattered 32-byte sectors.  The binned build
// first sorts every (cell, key) update of the batch into slabs of 2^21 cells
// (64 MB, half of L2) and then applies one slab at a time, so each slab's
// updates are read back from L2 and each cell is written to HBM once.
//
// Pass 1, k_bin: each block takes 256 keys, computes their r cells, counts
// them per slab in shared memory, reserves a run in each slab's record list
// with one atomic per slab, orders its records by slab in shared memory and
// writes every run contiguously.
// Pass 2 (iblt_tiles.cuh) applies one slab at a time, tile by tile in shared
// memory.
#pragma once

#include "iblt_types.cuh"


namespace pp {

template <int R>
__device__ __forceinline__ void apply_touch(Cell *cells, u32 c, u64 x, u64 cs, int sign) {
  touch_cell_nr(cells, c, x, cs, sign);
}

// Dynamic shared memory: 3 * n_slabs u32 (histogram, scan, base) + the staged
// records of one step (kBinKeys * NR * (8 + 4 [+ 4]) bytes).  Registers capped for 5
// resident CTAs per SM (2.99 -> 2.91 ms for the 2^26-cell build).
template <int R, bool BATCH>
__global__ void __launch_bounds__(kBlock, PP_BIN_CTAS) k_bin(Cell *__restrict__ cells, const TableArgs tab0,
                                                const TableArgs *__restrict__ tabs,
                                                const Chunk *__restrict__ chunks, u32 n_chunks,
                                                const u64 *__restrict__ keys, u64 m, int sign, BinArgs b) {
  constexpr int NR = nr_of<R>();
  constexpr int CAP = kBinKeys * NR;
  extern __shared__ __align__(16) unsigned char smem[];
  u64 *s_key = reinterpret_cast<u64 *>(smem);                 // CAP
  u32 *s_cell = reinterpret_cast<u32 *>(s_key + CAP);         // CAP
  u32 *s_tab = s_cell + CAP;                                  // CAP (batch)
  u32 *s_hist = s_tab + (BATCH ? CAP : 0);                    // n_slabs
  u32 *s_scan = s_hist + b.n_slabs;                           // n_slabs
  u32 *s_base = s_scan + b.n_slabs;                           // n_slabs
  __shared__ u32 s_wt[33];
  __shared__ u32 s_total;
  const u32 tid = threadIdx.x;
  const u32 ns = b.n_slabs;
  // work items: plain = key ranges of kBinKeys; batch = the insert chunks (one table each)
  const u64 n_items = BATCH ? n_chunks : (m + kBinKeys - 1) / kBinKeys;
  for (u64 item = blockIdx.x; item < n_items; item += gridDim.x) {
    u64 k0, k1;
    u32 tb = 0;
    if (BATCH) {
      const Chunk ch = chunks[item];
      k0 = ch.begin, k1 = ch.end, tb = ch.table;
    } else {
      k0 = item * kBinKeys;
      k1 = k0 + kBinKeys < m ? k0 + kBinKeys : m;
    }
    const TableArgs &T = BATCH ? tabs[tb] : tab0;
    const int r = rank_of<R>(T);
    // a batch chunk may hold more than kBinKeys keys: walk it in steps
    for (u64 s0 = k0; s0 < k1; s0 += kBinKeys) {
      for (u32 i = tid; i < ns; i += kBlock) s_hist[i] = 0;
      __syncthreads();
      u64 x[kBinItems];
      u32 c[kBinItems][NR], rank[kBinItems][NR];
      bool valid[kBinItems];
#pragma unroll
      for (int it = 0; it < kBinItems; ++it) {
        const u64 ki = s0 + (u64)it * kBlock + tid;
        valid[it] = ki < k1;
        x[it] = valid[it] ? __ldcs(keys + ki) : 0ull;
      }
#pragma unroll
      for (int it = 0; it < kBinItems; ++it) {
        cells_of<NR>(x[it], T, c[it]);
#pragma unroll
        for (int j = 0; j < NR; ++j)
          rank[it][j] = (valid[it] && j < r) ? atomicAdd(s_hist + (c[it][j] >> kSlabShift), 1u) : 0u;
      }
      __syncthreads();
      // exclusive scan of the histogram: thread t owns slabs [t*per, (t+1)*per)
      const u32 per = (ns + kBlock - 1) / kBlock;
      const u32 lo = tid * per, hi = lo + per < ns ? lo + per : ns;
      u32 own = 0;
      for (u32 i = lo; i < hi; ++i) own += s_hist[i];
      u32 inc = own;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(kFull, inc, o);
        if ((int)lane_id() >= o) inc += y;
      }
      if (lane_id() == 31) s_wt[tid >> 5] = inc;
      __syncthreads();
      if (tid < 32) {
        const u32 w = tid < kBlock / 32 ? s_wt[tid] : 0;
        u32 wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const u32 y = __shfl_up_sync(kFull, wi, o);
          if ((int)tid >= o) wi += y;
        }
        if (tid < kBlock / 32) s_wt[tid] = wi - w;
        if (tid == 31) s_total = wi;
      }
      __syncthreads();
      u32 run = s_wt[tid >> 5] + inc - own;
      for (u32 i = lo; i < hi; ++i) {
        s_scan[i] = run;
        const u32 h = s_hist[i];
        s_base[i] = h ? atomicAdd(b.count + i, h) : 0u;
        run += h;
      }
      __syncthreads();
#pragma unroll
      for (int it = 0; it < kBinItems; ++it) {
        if (valid[it]) {
#pragma unroll
          for (int j = 0; j < NR; ++j) {
            if (j < r) {
              const u32 bn = c[it][j] >> kSlabShift;
              const u32 pos = s_scan[bn] + rank[it][j];
              s_key[pos] = x[it];
              s_cell[pos] = c[it][j];
              if (BATCH) s_tab[pos] = tb;
            }
          }
        }
      }
      __syncthreads();
      const u32 total = s_total;
      for (u32 p = tid; p < total; p += kBlock) {
        const u32 bn = s_cell[p] >> kSlabShift;
        const u32 slot = s_base[bn] + (p - s_scan[bn]);
        if (slot < b.cap) {
          const u64 dst = (u64)bn * b.cap + slot;
          b.rec_key[dst] = s_key[p];
          b.rec_cell[dst] = s_cell[p];
          if (BATCH) b.rec_tab[dst] = s_tab[p];
        } else if (b.direct_overflow) {
          const TableArgs &TT = BATCH ? tabs[s_tab[p]] : tab0;
          const u64 xx = s_key[p];
          apply_touch<R>(cells, s_cell[p], xx, checksum(xx, TT.seed[rank_of<R>(TT)]), sign);
        } else {
          *b.overflow = 1u;
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace pp
