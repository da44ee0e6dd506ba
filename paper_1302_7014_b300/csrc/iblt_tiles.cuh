// Tile pass of the slab-binned IBLT build.
//
// Applying a slab's updates with L2 atomics is bound by the L2's atomic
// throughput: every update is three atomics on one 32-byte cell.  The tile
// pass replaces them with shared-memory atomics, in two roles:
//   bin    sorts a slab's update records into the slab's 512 tiles of 4096
//          cells (per-block histogram in shared memory, one atomic per tile
//          per block, runs written contiguously with an L2 "evict last" hint:
//          the next launch reads them back);
//   apply  one block per tile: the tile's cells in shared memory (zero for a
//          build, loaded for an insert), every update of the tile applied
//          there, the 4096 cells written back coalesced.
// Launch s of k_tile_step runs "bin slab s" and "apply slab s-1" side by side
// (block roles interleaved), so the latency-bound sort of one slab overlaps
// the update of the previous one.  Sorted records alternate between two
// buffer sets (slab s in set s % 2).
// A tile whose list is full sends its extra records to the slab's overflow
// list (three sets, slab s in set s % 3); the apply role of launch s + 2
// applies them with global atomics, after the slab's tiles were written.
// Updates commute, so the cells end up exactly as with any other order.
#pragma once

#include "iblt_types.cuh"

namespace pp {

__device__ __forceinline__ u64 chk_seed_of(const TableArgs &T) { return T.seed[T.r]; }

// Role "bin" for slab `slab`, as block `bi` of `nb` bin blocks.
template <bool BATCH>
__device__ __forceinline__ void tile_bin(unsigned char *smem, const BinArgs &b, const TileArgs &ta, u32 slab,
                                         u32 bi, u32 nb) {
  u64 *s_key = reinterpret_cast<u64 *>(smem);              // kTileBinChunk
  u32 *s_cell = reinterpret_cast<u32 *>(s_key + kTileBinChunk);
  u32 *s_tab = s_cell + kTileBinChunk;                     // (batch)
  __shared__ u32 s_hist[kTilesPerSlab], s_scan[kTilesPerSlab], s_base[kTilesPerSlab];
  __shared__ u32 s_wt[kTileThreads / 32];
  const u32 tid = threadIdx.x;
  const u64 keep = l2_evict_last_policy();
  const u32 set = slab & 1u;
  u64 *tkey = ta.key + set * ta.set_stride;
  u16 *toff = ta.off + set * ta.set_stride;
  u32 *ttab = BATCH ? ta.tab + set * ta.set_stride : nullptr;
  u32 *tcount = ta.count + set * kTilesPerSlab;
  const u64 oset = (u64)(slab % 3u) * ta.o_cap;
  const u32 cnt = b.count[slab];
  const u32 n = cnt < b.cap ? cnt : b.cap;
  const u64 src = (u64)slab * b.cap;
  const u32 cbase = slab << kSlabShift;
  for (u32 c0 = bi * (u32)kTileBinChunk; c0 < n; c0 += nb * (u32)kTileBinChunk) {
    if (tid < kTilesPerSlab) s_hist[tid] = 0;
    __syncthreads();
    const u32 c1 = c0 + kTileBinChunk < n ? c0 + kTileBinChunk : n;
    // this thread's records: every load in flight at once, then their ranks
    // within their tiles (shared-memory histogram)
    u64 x[kTileBinItems];
    u32 c[kTileBinItems], tb[kTileBinItems], rk[kTileBinItems];
#pragma unroll
    for (int it = 0; it < kTileBinItems; ++it) {
      const u32 i = c0 + (u32)it * kTileThreads + tid;
      const bool v = i < c1;
      c[it] = v ? __ldcs(b.rec_cell + src + i) : 0xffffffffu;  // no cell has this index
      x[it] = v ? __ldcs(b.rec_key + src + i) : 0ull;
      tb[it] = (BATCH && v) ? __ldcs(b.rec_tab + src + i) : 0u;
    }
#pragma unroll
    for (int it = 0; it < kTileBinItems; ++it)
      rk[it] = c[it] != 0xffffffffu ? atomicAdd(s_hist + ((c[it] - cbase) >> kTileShift), 1u) : 0u;
    __syncthreads();
    // exclusive scan of the slab's tile histogram: one entry per thread
    const u32 own = tid < kTilesPerSlab ? s_hist[tid] : 0u;
    u32 inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 y = __shfl_up_sync(kFull, inc, o);
      if ((int)lane_id() >= o) inc += y;
    }
    if (lane_id() == 31) s_wt[tid >> 5] = inc;
    __syncthreads();
    if (tid < 32) {
      const u32 w = tid < kTileThreads / 32 ? s_wt[tid] : 0;
      u32 wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(kFull, wi, o);
        if ((int)tid >= o) wi += y;
      }
      if (tid < kTileThreads / 32) s_wt[tid] = wi - w;
    }
    __syncthreads();
    if (tid < kTilesPerSlab) {
      s_scan[tid] = s_wt[tid >> 5] + inc - own;
      s_base[tid] = own ? atomicAdd(tcount + tid, own) : 0u;
    }
    __syncthreads();
    // order the chunk by tile in shared memory
#pragma unroll
    for (int it = 0; it < kTileBinItems; ++it) {
      if (c[it] != 0xffffffffu) {
        const u32 pos = s_scan[(c[it] - cbase) >> kTileShift] + rk[it];
        s_key[pos] = x[it];
        s_cell[pos] = c[it];
        if (BATCH) s_tab[pos] = tb[it];
      }
    }
    __syncthreads();
    // contiguous runs per tile; a full tile spills to the overflow list
    for (u32 p = tid; p < c1 - c0; p += kTileThreads) {
      const u32 tile = (s_cell[p] - cbase) >> kTileShift;
      const u32 slot = s_base[tile] + (p - s_scan[tile]);
      if (slot < ta.cap) {
        const u64 dst = (u64)tile * ta.cap + slot;
        st_l2_policy(tkey + dst, s_key[p], keep);
        st_l2_policy(toff + dst, (u16)(s_cell[p] & (kTileCells - 1)), keep);
        if (BATCH) st_l2_policy(ttab + dst, s_tab[p], keep);
      } else {
        const u32 q = atomicAdd(ta.o_count + slab, 1u);
        if (q < ta.o_cap) {
          ta.o_key[oset + q] = s_key[p];
          ta.o_cell[oset + q] = s_cell[p];
          if (BATCH) ta.o_tab[oset + q] = s_tab[p];
        }
      }
    }
    __syncthreads();
  }
}

// The write-out of a tile that also finds F_1 (PrescanArgs): a pure cell is
// stored empty and pushed into the frontier segment of its tile (one
// reservation on the segment's count per warp), each warp writes the bitmap
// words of its cells, and the tile's count sum and the decode's counters are
// recorded.  The cells' values are the build's, so a cell is pure exactly when
// a scan of the built table would find it pure.
template <bool BATCH>
__device__ __forceinline__ void prescan_write(Cell *cells, u64 c0, u32 nc, const u64 *s_key, const u64 *s_chk,
                                              const int *s_cnt, const PrescanArgs &pre) {
  __shared__ u64 s_red[4][kTileThreads / 32];
  const u32 T = (u32)(c0 >> kTileShift);
  const u32 seg = T % pre.tb.n_seg_d;
  const u64 sbase = (u64)seg * pre.tb.cap_d;
  const u32 lane = lane_id();
  u64 alive = 0, nonempty = 0, pushed = 0;
  long long sum = 0;
  u32 flags = 0;
  // the write-out with every warp's ballots kept, then one reservation per
  // warp in the tile's segment for all its pure cells
  constexpr int K = kTileCells / kTileThreads;
  static_assert(K <= 32, "one lane per step holds the seed of the warp's word");
  // BATCH: the warp's 32 cells of step k are one word of one table; lane k
  // loads that word's seed for the whole warp, all steps' loads at once
  u64 wsd = 0;
  if (BATCH && lane < (u32)K) {
    const u32 iw = lane * kTileThreads + (threadIdx.x & ~31u);
    if (iw < nc) wsd = pre.wseed[(c0 + iw) >> 5];
  }
  u32 balls[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const u32 i = threadIdx.x + (u32)k * kTileThreads;
    const u64 seed = BATCH ? __shfl_sync(kFull, wsd, k) : pre.seed_chk;
    bool pure = false;
    if (i < nc) {
      const u64 key = s_key[i], chk = s_chk[i];
      const int cnt = s_cnt[i];
      pure = cell_pure(cnt, key, chk, seed);
      alive += cnt >= 2;
      nonempty += cnt != 0;
      sum += cnt;
      if (pure) st_cell_cs(cells + c0 + i, 0ull, 0ull, 0);
      else st_cell_cs(cells + c0 + i, key, chk, cnt);
    }
    balls[k] = __ballot_sync(kFull, pure);
    if (lane == 0 && i < nc) pre.bitmap[(c0 + i) >> 5] = balls[k];  // i is the warp's first cell
  }
  u32 tot = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) tot += __popc(balls[k]);
  u32 base = 0;
  if (lane == 0 && tot) base = atomicAdd(pre.tb.fseg + seg, tot);
  base = __shfl_sync(kFull, base, 0);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if ((balls[k] >> lane) & 1u) {
      const u32 i = threadIdx.x + (u32)k * kTileThreads;
      const u32 p = base + __popc(balls[k] & lanemask_lt());
      if (p < pre.tb.cap_d) {
        pre.fkey[sbase + p] = s_key[i];
        pre.fcell[sbase + p] = (u32)(c0 + i);
      } else {
        flags |= FLAG_INTERNAL;  // cannot happen: a segment holds every push of its tiles
      }
      pushed += 1;
    }
    base += __popc(balls[k]);
  }
  // the four figures in one reduction: shuffles within each warp, then thread
  // 0 over the warps (two's-complement sums, so the count sum may be signed)
  u64 v[4] = {(u64)sum, alive, nonempty, pushed};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(kFull, v[k], o);
    if (lane == 0) s_red[k][threadIdx.x >> 5] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t[4] = {0, 0, 0, 0};
    for (int w = 0; w < kTileThreads / 32; ++w)
#pragma unroll
      for (int k = 0; k < 4; ++k) t[k] += s_red[k][w];
    const long long sm = (long long)t[0];
    pre.tb.sum[T] = sm > 0 ? (u32)sm : 0u;
    if (t[1]) atomicAdd(&pre.ctl->alive, t[1]);
    if (t[2]) atomicAdd(&pre.ctl->nonempty, t[2]);
    if (t[3]) {
      atomicAdd(&pre.ctl->emptied, t[3]);
      atomicAdd(&pre.ctl->n_next, (u32)t[3]);
    }
  }
  if (flags) atomicOr(&pre.ctl->flags, flags);
}

// Role "apply" for tile `tile` of slab `slab`.  PRESCAN (a build from empty
// cells, single table): the tile's write-out also finds its cells pure before
// any round (see PrescanArgs), unless overflow records will still change the
// tile, which then goes to the rescan list.
template <bool BATCH, bool PRESCAN = false>
__device__ __forceinline__ void tile_apply(unsigned char *smem, Cell *cells, const TableArgs &tab0,
                                           const TableArgs *tabs, const TileArgs &ta, u32 slab, u32 tile,
                                           u64 n_cells, int sign, int zero, const PrescanArgs &pre) {
  u64 *s_key = reinterpret_cast<u64 *>(smem);                 // kTileCells
  u64 *s_chk = s_key + kTileCells;                            // kTileCells
  int *s_cnt = reinterpret_cast<int *>(s_chk + kTileCells);   // kTileCells
  const u64 c0 = ((u64)slab << kSlabShift) + ((u64)tile << kTileShift);
  if (c0 >= n_cells) return;  // uniform per block
  const u32 nc = (u32)(c0 + kTileCells <= n_cells ? kTileCells : n_cells - c0);
  const u32 set = slab & 1u;
  const u64 src = set * ta.set_stride + (u64)tile * ta.cap;
  u32 *tcount = ta.count + set * kTilesPerSlab;
  for (u32 i = threadIdx.x; i < nc; i += kTileThreads) {
    if (zero) {
      s_key[i] = 0;
      s_chk[i] = 0;
      s_cnt[i] = 0;
    } else {
      u64 k, ch;
      int cnt;
      ld_cell_cs(cells + c0 + i, k, ch, cnt);
      s_key[i] = k;
      s_chk[i] = ch;
      s_cnt[i] = cnt;
    }
  }
  __syncthreads();
  const u32 cnt = tcount[tile];
  const u32 n = cnt < ta.cap ? cnt : ta.cap;
  const u64 seed0 = BATCH ? 0 : chk_seed_of(tab0);
  for (u32 i0 = 0; i0 < n; i0 += kTileThreads * kTileApplyItems) {
    u64 x[kTileApplyItems], seed[kTileApplyItems];
    u32 off[kTileApplyItems];
#pragma unroll
    for (int it = 0; it < kTileApplyItems; ++it) {
      const u32 i = i0 + (u32)it * kTileThreads + threadIdx.x;
      const bool v = i < n;
      x[it] = v ? __ldcs(ta.key + src + i) : 0ull;
      off[it] = v ? (u32)__ldcs(ta.off + src + i) : 0xffffffffu;
      seed[it] = (BATCH && v) ? chk_seed_of(tabs[__ldcs(ta.tab + src + i)]) : seed0;
    }
#pragma unroll
    for (int it = 0; it < kTileApplyItems; ++it) {
      if (off[it] != 0xffffffffu) {
        const u32 o = off[it];
        const u64 cs = checksum(x[it], seed[it]);
        atomicAdd(s_cnt + o, sign);
        smem_xor64(s_chk + o, cs);
        smem_xor64(s_key + o, x[it]);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) tcount[tile] = 0;  // ready for slab + 2
  // the tile's sorted records are dead now: drop their L2 lines unwritten (the
  // tile's region starts on a 128-byte line, cap being a multiple of 64)
  for (u32 l = threadIdx.x; l < (n * 8 + 127) / 128; l += kTileThreads) l2_discard(ta.key + src + l * 16);
  for (u32 l = threadIdx.x; l < (n * 2 + 127) / 128; l += kTileThreads) l2_discard(ta.off + src + l * 64);
  if (BATCH)
    for (u32 l = threadIdx.x; l < (n * 4 + 127) / 128; l += kTileThreads) l2_discard(ta.tab + src + l * 32);
  if constexpr (PRESCAN) {
    if (cnt <= ta.cap) {
      prescan_write<BATCH>(cells, c0, nc, s_key, s_chk, s_cnt, pre);
      return;
    }
    if (threadIdx.x == 0) pre.tb.rescan[atomicAdd(pre.tb.n_rescan, 1u)] = (u32)(c0 >> kTileShift);
  }
  for (u32 i = threadIdx.x; i < nc; i += kTileThreads) st_cell_cs(cells + c0 + i, s_key[i], s_chk[i], s_cnt[i]);
}

// Role "bin" of a batched update taken straight from the keys (no slab
// lists): a batch's keys are ordered by table and its tables by arena
// position, so the tables that overlap slab `slab` own one contiguous range
// of the insert chunks.  Every key of that range is hashed here and those of
// its cells that fall in the slab are sorted into the slab's tiles, exactly as
// tile_bin sorts the slab's records.  A table that straddles two slabs is
// hashed in both passes, each keeping its own cells.
struct TileKeysArgs {
  const u64 *keys;
  const Chunk *chunks;    // key ranges of one table each, in table order
  const u32 *slab_chunk;  // per slab: first and one-past-last chunk of its tables
  u32 n_slabs;
};

template <int R>
__device__ __forceinline__ void tile_bin_keys(unsigned char *smem, const TableArgs *tabs, const TileKeysArgs &ka,
                                              const TileArgs &ta, u32 slab, u32 bi, u32 nb) {
  constexpr int NR = nr_of<R>();
  constexpr int KPT = kTileBinItems / NR > 0 ? kTileBinItems / NR : 1;  // keys per thread per step
  static_assert(KPT * NR * kTileThreads <= kTileBinChunk, "a step's records exceed the staging");
  constexpr u32 KEYS = (u32)KPT * kTileThreads;
  u64 *s_key = reinterpret_cast<u64 *>(smem);  // kTileBinChunk
  u32 *s_cell = reinterpret_cast<u32 *>(s_key + kTileBinChunk);
  __shared__ u32 s_hist[kTilesPerSlab], s_scan[kTilesPerSlab], s_base[kTilesPerSlab];
  __shared__ u32 s_wt[kTileThreads / 32];
  __shared__ u32 s_total;
  const u32 tid = threadIdx.x;
  const u64 keep = l2_evict_last_policy();
  const u32 set = slab & 1u;
  u64 *tkey = ta.key + set * ta.set_stride;
  u16 *toff = ta.off + set * ta.set_stride;
  u32 *ttab = ta.tab + set * ta.set_stride;
  u32 *tcount = ta.count + set * kTilesPerSlab;
  const u64 oset = (u64)(slab % 3u) * ta.o_cap;
  const u32 cbase = slab << kSlabShift;
  const u32 cb = ka.slab_chunk[2 * slab], ce = ka.slab_chunk[2 * slab + 1];
  for (u32 ch = cb + bi; ch < ce; ch += nb) {
    const Chunk k = ka.chunks[ch];
    const TableArgs &T = tabs[k.table];
    const int r = rank_of<R>(T);
    for (u32 k0 = k.begin; k0 < k.end; k0 += KEYS) {
      if (tid < kTilesPerSlab) s_hist[tid] = 0;
      __syncthreads();
      u64 x[KPT];
      u32 c[KPT][NR], rk[KPT][NR];
#pragma unroll
      for (int it = 0; it < KPT; ++it) {
        const u32 i = k0 + (u32)it * kTileThreads + tid;
        x[it] = i < k.end ? __ldcs(ka.keys + i) : 0ull;
      }
#pragma unroll
      for (int it = 0; it < KPT; ++it) {
        const bool v = k0 + (u32)it * kTileThreads + tid < k.end;
        cells_of<NR>(x[it], T, c[it]);
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          const bool in = v && j < r && c[it][j] - cbase < kSlabCells;
          if (!in) c[it][j] = 0xffffffffu;  // no cell has this index
          rk[it][j] = in ? atomicAdd(s_hist + ((c[it][j] - cbase) >> kTileShift), 1u) : 0u;
        }
      }
      __syncthreads();
      // exclusive scan of the slab's tile histogram: one entry per thread
      const u32 own = tid < kTilesPerSlab ? s_hist[tid] : 0u;
      u32 inc = own;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(kFull, inc, o);
        if ((int)lane_id() >= o) inc += y;
      }
      if (lane_id() == 31) s_wt[tid >> 5] = inc;
      __syncthreads();
      if (tid < 32) {
        const u32 w = tid < kTileThreads / 32 ? s_wt[tid] : 0;
        u32 wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const u32 y = __shfl_up_sync(kFull, wi, o);
          if ((int)tid >= o) wi += y;
        }
        if (tid < kTileThreads / 32) s_wt[tid] = wi - w;
      }
      __syncthreads();
      const u32 excl = s_wt[tid >> 5] + inc - own;
      if (tid < kTilesPerSlab) {
        s_scan[tid] = excl;
        s_base[tid] = own ? atomicAdd(tcount + tid, own) : 0u;
      }
      if (tid == kTileThreads - 1) s_total = excl + own;
      __syncthreads();
      // order the step's records by tile in shared memory
#pragma unroll
      for (int it = 0; it < KPT; ++it) {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (c[it][j] != 0xffffffffu) {
            const u32 pos = s_scan[(c[it][j] - cbase) >> kTileShift] + rk[it][j];
            s_key[pos] = x[it];
            s_cell[pos] = c[it][j];
          }
        }
      }
      __syncthreads();
      // contiguous runs per tile; a full tile spills to the overflow list
      const u32 total = s_total;
      for (u32 p = tid; p < total; p += kTileThreads) {
        const u32 tile = (s_cell[p] - cbase) >> kTileShift;
        const u32 slot = s_base[tile] + (p - s_scan[tile]);
        if (slot < ta.cap) {
          const u64 dst = (u64)tile * ta.cap + slot;
          st_l2_policy(tkey + dst, s_key[p], keep);
          st_l2_policy(toff + dst, (u16)(s_cell[p] & (kTileCells - 1)), keep);
          st_l2_policy(ttab + dst, k.table, keep);
        } else {
          const u32 q = atomicAdd(ta.o_count + slab, 1u);
          if (q < ta.o_cap) {  // o_cap bounds the slab's records: always true
            ta.o_key[oset + q] = s_key[p];
            ta.o_cell[oset + q] = s_cell[p];
            ta.o_tab[oset + q] = k.table;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Launch s (0 <= s <= n_slabs + 1):
//   apply role  (s >= 1 and s - 1 < n_slabs): the overflow of slab s - 2, then
//               the tiles of slab s - 1;  for s = n_slabs + 1: the overflow of
//               slab s - 2 only;
//   bin role    (s < n_slabs): slab s.
// n_apply / n_bin blocks of each role, interleaved by block index.
template <bool BATCH, bool PRESCAN = false>
__global__ void __launch_bounds__(kTileThreads, 2) k_tile_step(Cell *__restrict__ cells, const TableArgs tab0,
                                                      const TableArgs *__restrict__ tabs, BinArgs b,
                                                      TileArgs ta, u32 s, u32 n_apply, u32 n_bin,
                                                      u64 n_cells, int sign, int zero, PrescanArgs pre) {
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
    tile_bin<BATCH>(smem, b, ta, s, idx, n_bin);
    return;
  }
  if (s >= 2) {
    // the overflow of slab s - 2: its tiles were written by launch s - 1
    const u32 os = s - 2;
    const u64 oset = (u64)(os % 3u) * ta.o_cap;
    const u32 no = min(ta.o_count[os], (u32)ta.o_cap);
    for (u32 i = idx * kTileThreads + threadIdx.x; i < no; i += n_apply * kTileThreads) {
      const u64 x = ta.o_key[oset + i];
      const TableArgs &T = BATCH ? tabs[ta.o_tab[oset + i]] : tab0;
      touch_cell_nr(cells, ta.o_cell[oset + i], x, checksum(x, chk_seed_of(T)), sign);
    }
  }
  if (s >= 1 && s - 1 < b.n_slabs)
    tile_apply<BATCH, PRESCAN>(smem, cells, tab0, tabs, ta, s - 1, idx, n_cells, sign, zero, pre);
}

// The batched tile step with the bin role taken from the keys (tile_bin_keys);
// the apply role is k_tile_step's.
template <int R, bool PRESCAN = false>
__global__ void __launch_bounds__(kTileThreads, 2) k_tile_step_keys(Cell *__restrict__ cells,
                                                           const TableArgs *__restrict__ tabs, TileKeysArgs ka,
                                                           TileArgs ta, u32 s, u32 n_apply, u32 n_bin,
                                                           u64 n_cells, int sign, int zero, PrescanArgs pre) {
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
    tile_bin_keys<R>(smem, tabs, ka, ta, s, idx, n_bin);
    return;
  }
  if (s >= 2) {
    const u32 os = s - 2;
    const u64 oset = (u64)(os % 3u) * ta.o_cap;
    const u32 no = min(ta.o_count[os], (u32)ta.o_cap);
    for (u32 i = idx * kTileThreads + threadIdx.x; i < no; i += n_apply * kTileThreads) {
      const u64 x = ta.o_key[oset + i];
      const TableArgs &T = tabs[ta.o_tab[oset + i]];
      touch_cell_nr(cells, ta.o_cell[oset + i], x, checksum(x, chk_seed_of(T)), sign);
    }
  }
  const TableArgs t0{};
  if (s >= 1 && s - 1 < ka.n_slabs)
    tile_apply<true, PRESCAN>(smem, cells, t0, tabs, ta, s - 1, idx, n_cells, sign, zero, pre);
}

}  // namespace pp
