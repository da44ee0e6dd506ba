// Slab-binned IBLT build.
//
// Random cell updates spread over a table much larger than L2 run at the rate
// at which HBM can open rows for scattered 32-byte sectors.  The binned build
// first sorts every (cell, key) update of the batch into slabs of 2^21 cells
// (64 MB, half of L2) and then applies one slab at a time, so all updates of
// a slab land in L2 while the slab is resident.  When the table is built from
// scratch the slab is zero-filled just before its updates: the zero lines are
// then already in L2 and the slab is never read from HBM at all.
//
// Pass 1, k_bin: each block takes 256 keys, computes their r cells, counts
// them per slab in shared memory, reserves a run in each slab's record list
// with one atomic per slab, orders its records by slab in shared memory and
// writes every run contiguously.
// Pass 2, k_apply: all updates of one slab (count += sign, XOR key and
// checksum), one launch per slab.
#pragma once

#include "iblt_types.cuh"

namespace pp {

constexpr int kSlabShift = 21;               // 2^21 cells = 64 MB per slab
constexpr u32 kSlabCells = 1u << kSlabShift;
constexpr int kBinKeys = kBlock;             // keys per block per partition step

// Record lists of a binned build: slab s owns records [s*cap, s*cap + min(count[s], cap)).
struct BinArgs {
  u64 *rec_key;
  u32 *rec_cell;   // global cell id
  u32 *rec_tab;    // table id (batched builds)
  u32 *count;      // records routed to each slab (may exceed cap)
  u32 *overflow;   // set to 1 when a record did not fit and could not be applied directly
  u32 cap;
  u32 n_slabs;
  int direct_overflow;  // 1: apply records that do not fit right away (plain insert)
};

template <int R>
__device__ __forceinline__ void apply_touch(Cell *cells, u32 c, u64 x, u64 cx, int sign) {
  Cell *p = cells + c;
  atomicAdd(&p->count, sign);
  atomicXor(&p->key, x);
  atomicXor(&p->chk, cx);
}

// Dynamic shared memory: 3 * n_slabs u32 (histogram, scan, base) + the staged
// records of one step (kBinKeys * NR * (8 + 4 + 4 [+ 4]) bytes).
template <int R, bool BATCH>
__global__ void __launch_bounds__(kBlock) k_bin(Cell *__restrict__ cells, const TableArgs tab0,
                                                const TableArgs *__restrict__ tabs,
                                                const Chunk *__restrict__ chunks, u32 n_chunks,
                                                const u64 *__restrict__ keys, u64 m, int sign, BinArgs b) {
  constexpr int NR = R ? R : PP_MAX_R;
  constexpr int CAP = kBinKeys * NR;
  extern __shared__ __align__(16) unsigned char smem[];
  u64 *s_key = reinterpret_cast<u64 *>(smem);                 // CAP
  u32 *s_cell = reinterpret_cast<u32 *>(s_key + CAP);         // CAP
  u32 *s_bin = s_cell + CAP;                                  // CAP
  u32 *s_tab = s_bin + CAP;                                   // CAP (batch)
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
    const int r = R ? R : (int)T.r;
    // a batch chunk may hold more than kBinKeys keys: walk it in steps
    for (u64 s0 = k0; s0 < k1; s0 += kBinKeys) {
      for (u32 i = tid; i < ns; i += kBlock) s_hist[i] = 0;
      __syncthreads();
      const u64 ki = s0 + tid;
      const bool valid = ki < k1;
      u64 x = 0;
      u32 c[NR], bin[NR], rank[NR];
      if (valid) x = __ldcs(keys + ki);
      cells_of<NR>(x, T, c);
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        bin[j] = c[j] >> kSlabShift;
        rank[j] = (valid && j < r) ? atomicAdd(s_hist + bin[j], 1u) : 0u;
      }
      __syncthreads();
      // exclusive scan of the histogram: thread t owns slabs [t*per, (t+1)*per)
      const u32 per = (ns + kBlock - 1) / kBlock;
      const u32 lo = tid * per, hi = lo + per < ns ? lo + per : ns;
      u32 own = 0;
      for (u32 i = lo; i < hi; ++i) own += s_hist[i];
      // block-wide exclusive scan of per-thread totals
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
      if (valid) {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (j < r) {
            const u32 pos = s_scan[bin[j]] + rank[j];
            s_key[pos] = x;
            s_cell[pos] = c[j];
            s_bin[pos] = bin[j];
            if (BATCH) s_tab[pos] = tb;
          }
        }
      }
      __syncthreads();
      const u32 total = s_total;
      for (u32 p = tid; p < total; p += kBlock) {
        const u32 bn = s_bin[p];
        const u32 slot = s_base[bn] + (p - s_scan[bn]);
        if (slot < b.cap) {
          const u64 dst = (u64)bn * b.cap + slot;
          b.rec_key[dst] = s_key[p];
          b.rec_cell[dst] = s_cell[p];
          if (BATCH) b.rec_tab[dst] = s_tab[p];
        } else if (b.direct_overflow) {
          const TableArgs &TT = BATCH ? tabs[s_tab[p]] : tab0;
          const u64 xx = s_key[p];
          apply_touch<R>(cells, s_cell[p], xx, mix64(xx ^ TT.seed[R ? R : (int)TT.r]), sign);
        } else {
          *b.overflow = 1u;
        }
      }
      __syncthreads();
    }
  }
}

// All recorded updates of slab `slab`.
template <int R, bool BATCH>
__global__ void __launch_bounds__(kBlock) k_apply(Cell *__restrict__ cells, const TableArgs tab0,
                                                  const TableArgs *__restrict__ tabs, BinArgs b, u32 slab,
                                                  int sign) {
  const u32 cnt = b.count[slab];
  const u32 n = cnt < b.cap ? cnt : b.cap;
  const u64 base = (u64)slab * b.cap;
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const u64 x = __ldcs(b.rec_key + base + i);
    const u32 c = __ldcs(b.rec_cell + base + i);
    const TableArgs &T = BATCH ? tabs[__ldcs(b.rec_tab + base + i)] : tab0;
    apply_touch<R>(cells, c, x, mix64(x ^ T.seed[R ? R : (int)T.r]), sign);
  }
}

}  // namespace pp
