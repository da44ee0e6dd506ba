// Tile rounds: the IBLT decode's rounds (Sec. 1 at k = 2 on the hypergraph of
// Sec. 6) with each round's cell updates applied tile by tile.
//
// The table is cut into tiles of 4096 consecutive cells.  Per round:
//   k_tclaim  for every frontier entry (cell c, key x snapshotted when c
//             became pure) decides, as k_claim does, whether c is the
//             lowest-index cell of x that was pure at the round's start.  A
//             winner outputs x, and for each of x's cells that was not pure at
//             the round's start writes one record (x, cell) into the region of
//             the cell's coarse bin (2^bin_tshift tiles, at most 128 bins).
//   k_tsort   sorts each coarse bin's records of the round into its tiles'
//             regions as (x, offset of the cell in its tile).  Two passes keep
//             the claim's shared-memory sort small (128 bins, not 16384 tiles)
//             and give every tile's cursor one atomic per chunk.
//   k_tactive lists the tiles that received records, split into sparse
//             (at most kTSCap records) and dense ones.
//   k_tapply_sparse / k_tapply  one block per tile: the round's records of
//             the tile are folded in shared memory into one update per
//             touched cell (count decrement, key XOR, checksum XOR) -- in a
//             small hash table for sparse tiles, in per-cell arrays for dense
//             ones; then every touched cell is read, updated and written back
//             once with plain 256-bit accesses and no global atomics.  A cell
//             that is pure after the update joins the next frontier right
//             there (key snapshot and bitmap bit), so no separate pass
//             re-reads it.
// A pure cell is written as (0, 0, 0) at the moment it joins the frontier (by
// k_tscan or the apply).  In a table built from insertions only, count 1 means
// the cell holds exactly one key x, so it is (x, checkSum(x), 1); x is
// recovered in the next round, and deleting it leaves (0, 0, 0).  The frontier
// entry keeps x, no record is ever sent to a cell that was pure at its round's
// start, and the claim touches no cell.  A decode that stops with a frontier
// pending (round limit, error) puts (x, checkSum(x), 1) back into each of its
// cells (k_trestore), so the table is left as after its last completed round.
// Records of a tile over the whole decode never exceed the sum of the tile's
// counts at the decode's start (each key leaves each of its cells once), so
// every tile owns a fixed region of that size, filled round after round.  That
// bound holds for tables built from insertions only; the host sends tables
// that saw deletions to the binned rounds instead.
//
// The frontier is kept in segments, one per block of k_tscan / k_tapply /
// k_tapply_sparse: a block writes the cells it finds pure into its own
// segment with a cursor in shared memory (no global atomic per push).
#pragma once

#include "iblt_types.cuh"

namespace pp {

constexpr int kTRShift = 12;
constexpr u32 kTRCells = 1u << kTRShift;     // cells per tile
constexpr int kTRThreads = 512;              // threads per block of k_tscan / k_tapply
constexpr int kTRScanItems = kTRCells / kTRThreads;
static_assert(kTRCells / 32 == kTRWordsPerTile, "the batch's word maps cover whole tiles");
constexpr u32 kTRAlign = 64;                 // records: tile regions start on 128-byte lines
constexpr int kTRPosStride = 8;              // write cursors (u32) one per 32-byte sector
constexpr int kTRCellsPerThread = 4;         // touched cells per thread per step of k_tapply
#ifndef PP_TSPARSE_THREADS
#define PP_TSPARSE_THREADS 256
#endif
constexpr int kTSThreads = PP_TSPARSE_THREADS;  // threads per block of k_tapply_sparse
constexpr u32 kTSCap = 512;                  // records of a sparse tile (at most)
constexpr u32 kTSSlots = 1024;               // hash slots of k_tapply_sparse
constexpr u32 kTSEmpty = 0xffffffffu;
#ifndef PP_TSPARSE_CTAS
#define PP_TSPARSE_CTAS 4
#endif
constexpr int kTSCtas = PP_TSPARSE_CTAS;    // resident blocks per SM of k_tapply_sparse
#ifndef PP_TCLAIM_ITEMS
#define PP_TCLAIM_ITEMS 2
#endif
#ifndef PP_TCLAIM_CTAS
#define PP_TCLAIM_CTAS 2
#endif
#ifndef PP_TCLAIM_THREADS
#define PP_TCLAIM_THREADS 512
#endif
constexpr int kTClaimThreads = PP_TCLAIM_THREADS;        // threads per block of k_tclaim
constexpr int kTClaimItems = PP_TCLAIM_ITEMS;            // frontier entries per thread per chunk
constexpr int kTClaimChunk = kTClaimThreads * kTClaimItems;

// First entry of frontier segment k: the dense segments (cap_d entries each)
// come first, then the sparse ones (cap_s each).
__device__ __forceinline__ u64 seg_start(const TileRoundBufs &tb, u32 k) {
  return k < tb.n_seg_d ? (u64)k * tb.cap_d : (u64)tb.n_seg_d * tb.cap_d + (u64)(k - tb.n_seg_d) * tb.cap_s;
}

// Asynchronous global -> shared copies (cp.async): the next chunk's frontier
// entries are fetched while the current chunk is claimed.
__device__ __forceinline__ void cp_async_8(void *dst_shared, const void *src) {
  const u32 d = (u32)__cvta_generic_to_shared(dst_shared);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_4(void *dst_shared, const void *src) {
  const u32 d = (u32)__cvta_generic_to_shared(dst_shared);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// waits until at most one group (the most recently committed) is pending
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Exclusive prefix of in[0..n) into out[0..n) and the total into out[n], by
// one block of B threads (thread i takes a contiguous share).  in may be
// global or shared; s_wt holds B / 32 words.
template <int B>
__device__ __forceinline__ void block_exclusive_scan(const u32 *in, u32 *out, u32 n, u32 *s_wt) {
  const u32 tid = threadIdx.x;
  const u32 per = (n + B - 1) / B;
  const u32 lo = tid * per, hi = min(lo + per, n);
  u32 own = 0;
  for (u32 k = lo; k < hi; ++k) own += in[k];
  u32 inc = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 y = __shfl_up_sync(kFull, inc, o);
    if ((int)lane_id() >= o) inc += y;
  }
  if (lane_id() == 31) s_wt[tid >> 5] = inc;
  __syncthreads();
  if (tid < 32) {
    const u32 w = tid < B / 32 ? s_wt[tid] : 0;
    u32 wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 y = __shfl_up_sync(kFull, wi, o);
      if ((int)tid >= o) wi += y;
    }
    if (tid < B / 32) s_wt[tid] = wi - w;
    if (tid == B / 32 - 1) out[n] = wi;
  }
  __syncthreads();
  u32 run = s_wt[tid >> 5] + inc - own;
  for (u32 k = lo; k < hi; ++k) {
    const u32 v = in[k];
    out[k] = run;
    run += v;
  }
  __syncthreads();
}

// By one warp: the exclusive prefix of cnt[0..n) into scan[0..n] (scan[n] =
// the total), for every k with cnt[k] > 0 a run of cnt[k] slots reserved at
// *cursor(k) (its first slot into base[k]), and cnt[k] set back to 0 for the
// next chunk.  Lane l takes a contiguous share; the reservations of a lane's
// share (at most 4 when n <= 128) are all in flight at once.  The rest of the
// block needs none of this until the next barrier, so a chunk of a
// partitioning kernel spends two barriers on its histogram, not five.
template <class Cursor>
__device__ __forceinline__ void warp_scan_reserve(u32 *cnt, u32 *scan, u32 *base, u32 n, Cursor cursor) {
  const u32 lane = lane_id();
  const u32 per = (n + 31) / 32;
  const u32 lo = min(lane * per, n), hi = min(lo + per, n);
  u32 own = 0;
  for (u32 k = lo; k < hi; ++k) own += cnt[k];
  u32 inc = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 y = __shfl_up_sync(kFull, inc, o);
    if ((int)lane >= o) inc += y;
  }
  u32 run = inc - own;
  if (per <= 4) {
    u32 c[4], b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] = lo + q < hi ? cnt[lo + q] : 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = c[q] ? atomicAdd(cursor(lo + q), c[q]) : 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (lo + q < hi) {
        scan[lo + q] = run;
        run += c[q];
        base[lo + q] = b[q];
        cnt[lo + q] = 0;
      }
    }
  } else {
    for (u32 k = lo; k < hi; ++k) {
      const u32 c = cnt[k];
      scan[k] = run;
      run += c;
      base[k] = c ? atomicAdd(cursor(k), c) : 0u;
      cnt[k] = 0;
    }
  }
  if (lane == 31) scan[n] = inc;
}

// Initial full scan, one tile per block step: F_1 (cells pure before any
// round) with their bitmap bits, the sum of each tile's counts, and the
// decode's alive / nonempty counters.  Every bitmap word is written here.
// The cells of F_1 are emptied as they are found (see the file comment).
// Runs n_seg_d blocks; block b takes tiles b, b + n_seg_d, ... (at most
// 4096 pushes each) and writes segment b.  BATCH: tab0.n_cells is the arena's
// size, and a cell's checksum seed is its word's (bt.wseed).
template <int R, bool BATCH>
__global__ void __launch_bounds__(kTRThreads, 2) k_tscan(Cell *__restrict__ cells, const TableArgs tab0,
                                                      u64 *__restrict__ fkey, u32 *__restrict__ fcell,
                                                      u32 *__restrict__ bitmap, TileRoundBufs tb,
                                                      DecodeCtl *__restrict__ ctl, TRBatch bt) {
  __shared__ u32 s_seg, s_neg;
  __shared__ u64 s_red[kTRThreads / 32];
  const u32 tid = threadIdx.x;
  const u64 seed0 = BATCH ? 0ull : tab0.seed[rank_of<R>(tab0)];
  const u32 n = tab0.n_cells;
  const u64 seg0 = tb.fstart[blockIdx.x];
  u64 alive = 0, nonempty = 0, emptied = 0;
  if (tid == 0) s_seg = 0, s_neg = 0;
  __syncthreads();
  for (u32 t = blockIdx.x; t < tb.n_tiles; t += gridDim.x) {
    const u32 c0 = t << kTRShift;
    long long sum = 0;
    // every load of the tile is issued before its first store (the cell
    // accesses are volatile asm, kept in program order)
    u64 keys[kTRScanItems], chks[kTRScanItems];
    int cnts[kTRScanItems];
#pragma unroll
    for (int it = 0; it < kTRScanItems; ++it) {
      const u32 c = c0 + (u32)it * kTRThreads + tid;
      keys[it] = chks[it] = 0;
      cnts[it] = 0;
      if (c < n) ld_cell_cs(cells + c, keys[it], chks[it], cnts[it]);
    }
    // BATCH: a warp's 32 cells of item `it` are one word of one table; lane
    // `it` fetches that word's seed for the whole warp
    u64 wseed = 0;
    if (BATCH && lane_id() < (u32)kTRScanItems) {
      const u32 cw = c0 + lane_id() * kTRThreads + (tid & ~31u);
      if (cw < n) wseed = bt.wseed[cw >> 5];
    }
#pragma unroll
    for (int it = 0; it < kTRScanItems; ++it) {
      const u32 c = c0 + (u32)it * kTRThreads + tid;
      const bool valid = c < n;
      bool pure = false;
      const u64 key = keys[it];
      const u64 seed_chk = BATCH ? __shfl_sync(kFull, wseed, it) : seed0;
      if (valid) {
        const int cnt = cnts[it];
        pure = cell_pure(cnt, key, chks[it], seed_chk);
        alive += cnt >= 2;
        nonempty += cnt != 0;
        sum += cnt;
        if (cnt < 0) s_neg = 1;
        if (pure) {
          st_cell_cs(cells + c, 0ull, 0ull, 0);
          emptied += 1;
        }
      }
      const u32 ball = __ballot_sync(kFull, pure);
      const u32 first = c0 + (u32)it * kTRThreads + (tid & ~31u);
      if (lane_id() == 0 && first < n) bitmap[first >> 5] = ball;
      const u32 p = warp_reserve<u32>(pure, &s_seg);
      if (pure && p < tb.cap_d) {
        fkey[seg0 + p] = key;
        fcell[seg0 + p] = c;
      } else if (pure) {
        s_neg = 1;  // cannot happen: a segment holds every push of its block's tiles
      }
    }
    const long long sm = block_sum<long long, kTRThreads>(sum, reinterpret_cast<long long *>(s_red));
    if (tid == 0) tb.sum[t] = sm > 0 ? (u32)sm : 0u;
  }
  const u64 a = block_sum<u64, kTRThreads>(alive, s_red);
  const u64 ne = block_sum<u64, kTRThreads>(nonempty, s_red);
  const u64 em = block_sum<u64, kTRThreads>(emptied, s_red);
  if (tid == 0) {
    if (a) atomicAdd(&ctl->alive, a);
    if (ne) atomicAdd(&ctl->nonempty, ne);
    if (em) atomicAdd(&ctl->emptied, em);
    // a negative count (not an insert-only table) or a full segment
    if (s_neg) atomicOr(&ctl->flags, (u32)FLAG_INTERNAL);
    tb.fseg[blockIdx.x] = s_seg;
    if (s_seg) atomicAdd(&ctl->n_next, s_seg);
  }
}

// The scan of a decode whose build found F_1 (PrescanArgs): only the tiles of
// tb.rescan, which the build's overflow pass changed after their write-out,
// are scanned here, with what k_tscan does per tile; their pure cells join
// the tile's frontier segment (tile % n_seg_d) behind the build's entries.
// Usually the list is empty.  BATCH: a cell's checksum seed is its word's.
template <int R, bool BATCH>
__global__ void __launch_bounds__(kTRThreads, 2) k_trescan(Cell *__restrict__ cells, const TableArgs tab0,
                                                        u64 *__restrict__ fkey, u32 *__restrict__ fcell,
                                                        u32 *__restrict__ bitmap, TileRoundBufs tb,
                                                        DecodeCtl *__restrict__ ctl, TRBatch bt) {
  __shared__ u64 s_red[kTRThreads / 32];
  const u32 nl = *(volatile u32 *)tb.n_rescan;
  if (blockIdx.x >= nl) return;  // uniform
  const u32 tid = threadIdx.x, lane = lane_id();
  const u64 seed0 = BATCH ? 0ull : tab0.seed[rank_of<R>(tab0)];
  const u32 n = tab0.n_cells;
  u64 alive = 0, nonempty = 0, pushed = 0;
  u32 flags = 0;
  for (u32 li = blockIdx.x; li < nl; li += gridDim.x) {
    const u32 t = tb.rescan[li];
    const u32 c0 = t << kTRShift;
    const u32 seg = t % tb.n_seg_d;
    const u64 sbase = (u64)seg * tb.cap_d;
    long long sum = 0;
    u64 keys[kTRScanItems], chks[kTRScanItems];
    int cnts[kTRScanItems];
#pragma unroll
    for (int it = 0; it < kTRScanItems; ++it) {
      const u32 c = c0 + (u32)it * kTRThreads + tid;
      keys[it] = chks[it] = 0;
      cnts[it] = 0;
      if (c < n) ld_cell_cs(cells + c, keys[it], chks[it], cnts[it]);
    }
#pragma unroll
    for (int it = 0; it < kTRScanItems; ++it) {
      const u32 c = c0 + (u32)it * kTRThreads + tid;
      bool pure = false;
      if (c < n) {
        const int cnt = cnts[it];
        pure = cell_pure(cnt, keys[it], chks[it], BATCH ? bt.wseed[c >> 5] : seed0);
        alive += cnt >= 2;
        nonempty += cnt != 0;
        sum += cnt;
        if (pure) st_cell_cs(cells + c, 0ull, 0ull, 0);
      }
      const u32 ball = __ballot_sync(kFull, pure);
      const u32 first = c0 + (u32)it * kTRThreads + (tid & ~31u);
      if (lane == 0 && first < n) bitmap[first >> 5] = ball;
      u32 base = 0;
      if (lane == 0 && ball) base = atomicAdd(tb.fseg + seg, (u32)__popc(ball));
      base = __shfl_sync(kFull, base, 0);
      if (pure) {
        const u32 p = base + __popc(ball & lanemask_lt());
        if (p < tb.cap_d) {
          fkey[sbase + p] = keys[it];
          fcell[sbase + p] = c;
        } else {
          flags |= FLAG_INTERNAL;  // cannot happen: a segment holds every push of its tiles
        }
        pushed += 1;
      }
    }
    const long long sm = block_sum<long long, kTRThreads>(sum, reinterpret_cast<long long *>(s_red));
    if (tid == 0) tb.sum[t] = sm > 0 ? (u32)sm : 0u;
  }
  const u64 a = block_sum<u64, kTRThreads>(alive, s_red);
  const u64 ne = block_sum<u64, kTRThreads>(nonempty, s_red);
  const u64 pu = block_sum<u64, kTRThreads>(pushed, s_red);
  if (tid == 0) {
    if (a) atomicAdd(&ctl->alive, a);
    if (ne) atomicAdd(&ctl->nonempty, ne);
    if (pu) {
      atomicAdd(&ctl->emptied, pu);
      atomicAdd(&ctl->n_next, (u32)pu);
    }
  }
  if (flags) atomicOr(&ctl->flags, flags);
}

// Tile regions: base[t] = sum over t' < t of the tile sums, each rounded up to
// kTRAlign records; cursors at 0; every sparse segment empty.  One block;
// flags FLAG_CAPACITY if the regions exceed the record buffers.  Then F_1
// becomes the current frontier, so that the first loop iteration is round 1
// (unless F_1 is empty or an error was flagged: the loop then runs one
// iteration with round 0, which does nothing but end the decode).
__global__ void __launch_bounds__(1024) k_tprefix(TileRoundBufs tb, DecodeCtl *__restrict__ ctl) {
  __shared__ u64 s_w[33];
  const u32 tid = threadIdx.x;
  constexpr u32 kPer = 4;  // consecutive tiles per thread per pass: 4096 tiles a pass, loads coalesced
  const u32 nt = tb.n_tiles;
  u64 carry = 0;  // region bytes of the tiles before this pass (the same in every thread)
  for (u32 p0 = 0; p0 < nt; p0 += 1024 * kPer) {
    const u32 t0 = p0 + tid * kPer;
    u64 v[kPer], own = 0;
#pragma unroll
    for (u32 q = 0; q < kPer; ++q) {
      v[q] = t0 + q < nt ? (u64)(tb.sum[t0 + q] + kTRAlign - 1) / kTRAlign * kTRAlign : 0ull;
      own += v[q];
    }
    u64 inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 y = __shfl_up_sync(kFull, inc, o);
      if ((int)lane_id() >= o) inc += y;
    }
    if (lane_id() == 31) s_w[tid >> 5] = inc;
    __syncthreads();
    if (tid < 32) {
      const u64 w = s_w[tid];
      u64 wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(kFull, wi, o);
        if ((int)tid >= o) wi += y;
      }
      s_w[tid] = wi - w;
      if (tid == 31) s_w[32] = wi;
    }
    __syncthreads();
    u64 run = carry + s_w[tid >> 5] + inc - own;
#pragma unroll
    for (u32 q = 0; q < kPer; ++q) {
      const u32 t = t0 + q;
      if (t < nt) {
        tb.base[t] = run;
        tb.base64[t] = (u32)(run / kTRAlign);
        tb.pos[(u64)t * kTRPosStride] = 0;
        tb.done[t] = 0;
      }
      run += v[q];
    }
    carry += s_w[32];
    __syncthreads();  // s_w is written again by the next pass
  }
  for (u32 k = tid; k < tb.n_seg_s; k += 1024) tb.fseg[tb.n_seg_d + k] = 0;
  for (u32 k = tid; k < tb.n_bins; k += 1024) {
    tb.cpos[(u64)k * kTRPosStride] = 0;
    tb.cdone[k] = 0;
  }
  if (tid == 0) {
    tb.base[tb.n_tiles] = carry;
    tb.base64[tb.n_tiles] = (u32)(carry / kTRAlign);
    u32 fl = *(volatile u32 *)&ctl->flags;
    if (carry > tb.rec_cap) {
      atomicOr(&ctl->flags, (u32)FLAG_CAPACITY);
      fl |= FLAG_CAPACITY;
    }
    DecodeCtl &c = *ctl;
    const u32 f1 = *(volatile u32 *)&c.n_next;
    if ((fl & (FLAG_CAPACITY | FLAG_INTERNAL)) == 0 && f1 > 0) {
      c.out_round_start = c.n_out;
      c.n_front = f1;
      c.n_next = 0;
      c.n_cand = 0;
      c.round = 1;
    }
  }
}

// After the round loop: a decode that stopped with a frontier pending (round
// limit, error) puts (x, checkSum(x), 1) back into each cell that frontier
// emptied (see the file comment), so the table is left as after its last
// completed round.  The pending frontier is n_front entries in the segments.
template <int R, bool BATCH>
__global__ void __launch_bounds__(kBlock) k_trestore(Cell *__restrict__ cells, const TableArgs tab0,
                                                     const u64 *__restrict__ fkey, const u32 *__restrict__ fcell,
                                                     TileRoundBufs tb, DecodeCtl *__restrict__ ctl, TRBatch bt) {
  __shared__ u64 s_red[kBlock / 32];
  if (*(volatile u32 *)&ctl->n_front == 0) return;  // uniform: the decode finished
  const u64 seed0 = BATCH ? 0ull : tab0.seed[rank_of<R>(tab0)];
  const u32 ns = tb.n_seg_d + tb.n_seg_s;
  u64 put = 0;
  for (u32 sg = blockIdx.x; sg < ns; sg += gridDim.x) {
    const u32 cap = sg < tb.n_seg_d ? tb.cap_d : tb.cap_s;
    const u32 k = min(tb.fseg[sg], cap);
    const u64 a = tb.fstart[sg];
    for (u32 i = threadIdx.x; i < k; i += kBlock) {
      const u64 x = fkey[a + i];
      const u32 c = fcell[a + i];
      st_cell_cs(cells + c, x, checksum(x, BATCH ? bt.wseed[c >> 5] : seed0), 1);
      ++put;
    }
  }
  const u64 p = block_sum<u64, kBlock>(put, s_red);
  if (threadIdx.x == 0 && p) atomicAdd(&ctl->emptied, 0ull - p);
}

// Phase B1 of round t (see the file comment).  The records leave the block
// sorted by coarse bin (2^bin_tshift tiles), in contiguous runs with one cursor
// atomic per bin per chunk; k_tsort then sorts each bin's records into its
// tiles.  Dynamic shared memory: the prefix of the frontier's segment sizes
// (n_seg + 1 u32), the chunk's records (kTClaimChunk * NR keys and cells), per
// bin its count, its offset in the chunk and its run's first slot (3 * n_bins
// + 1 u32), and the bins' region bounds / kTRAlign (n_bins + 1 u32).
// BATCH: an entry's table is its cell's word's (bt.wtab); a table's keys go to
// its own output range, counted per table and round (bt.bc).
template <int R, bool BATCH>
__global__ void __launch_bounds__(kTClaimThreads, PP_TCLAIM_CTAS) k_tclaim(Cell *__restrict__ cells, const TableArgs tab0,
                                                      const u64 *__restrict__ fkey,
                                                      const u32 *__restrict__ fcell,
                                                      const u32 *__restrict__ bitmap, TileRoundBufs tb,
                                                      DecodeCtl *__restrict__ ctl, TRBatch bt) {
  constexpr int NR = nr_of<R>();
  constexpr int CAP = kTClaimChunk * NR;
  extern __shared__ __align__(16) unsigned char smem[];
  const u32 ns = tb.n_seg_d + tb.n_seg_s;
  const u32 nb = tb.n_bins;
  u64 *s_key = reinterpret_cast<u64 *>(smem);           // CAP
  u32 *s_cell = reinterpret_cast<u32 *>(s_key + CAP);   // CAP
  u32 *s_pre = s_cell + CAP;                            // ns + 1
  u32 *s_hist = s_pre + ns + 1;                         // nb
  u32 *s_scan = s_hist + nb;                            // nb + 1
  u32 *s_base = s_scan + nb + 1;                        // nb
  u32 *s_bb = s_base + nb;                              // nb + 1
  __shared__ u64 s_out[2][kTClaimChunk];  // a chunk's recovered keys, two chunks in turn
  __shared__ u64 s_fx[2][kTClaimChunk];   // frontier entries of this chunk and the next
  __shared__ u32 s_fc[2][kTClaimChunk];
  __shared__ u32 s_nout, s_nout_cur, s_wt[kTClaimThreads / 32], s_segn;
  __shared__ u64 s_obase;
  const u32 tid = threadIdx.x;
  const u32 n = *(volatile u32 *)&ctl->n_front;
  if (n == 0) return;  // uniform: nothing to claim
  u64 *out = ctl->out;
  const u64 out_cap = ctl->out_cap;
  const u32 round = *(volatile u32 *)&ctl->round;
  const u32 stats_rounds = BATCH ? ctl->stats_rounds : 0u;
  const u64 keep = l2_evict_last_policy();
  const u32 bsh = kTRShift + tb.bin_tshift;  // cell -> coarse bin
  for (u32 b = tid; b <= nb; b += kTClaimThreads) s_bb[b] = tb.base64[min(b << tb.bin_tshift, tb.n_tiles)];
  for (u32 b = tid; b < nb; b += kTClaimThreads) s_hist[b] = 0;  // then zeroed by warp 0 after each chunk
  if (tid == 0) s_nout = 0;
  block_exclusive_scan<kTClaimThreads>(tb.fseg, s_pre, ns, s_wt);
  // segment of entry c: the last k with s_pre[k] <= c
  auto seg_of = [&](u64 c) -> u32 {
    u32 a = 0, b = ns;
    while (b - a > 1) {
      const u32 mid = (a + b) >> 1;
      if (s_pre[mid] <= (u32)c) a = mid;
      else b = mid;
    }
    return a;
  };
  // copies this thread's frontier entries of the chunk at c into buffer bf
  // (a chunk of a large frontier spans one or two segments; a small frontier
  // can spread it over many, so a longer step is a binary search)
  auto fetch = [&](u64 c, u32 a0, int bf) {
#pragma unroll
    for (int it = 0; it < kTClaimItems; ++it) {
      const u32 i = (u32)(c + (u64)it * kTClaimThreads + tid);
      if (i < n) {
        u32 a = a0;
        if (a + 1 < ns && s_pre[a + 1] <= i) {
          ++a;
          if (a + 1 < ns && s_pre[a + 1] <= i) {
            u32 hi = ns;  // s_pre[a + 1] <= i < s_pre[hi] (s_pre[ns] is the total)
            ++a;
            while (hi - a > 1) {
              const u32 mid = (a + hi) >> 1;
              if (s_pre[mid] <= i) a = mid;
              else hi = mid;
            }
          }
        }
        const u64 src = seg_start(tb, a) + (i - s_pre[a]);
        cp_async_8(&s_fx[bf][it * kTClaimThreads + tid], fkey + src);
        cp_async_4(&s_fc[bf][it * kTClaimThreads + tid], fcell + src);
      }
    }
    cp_async_commit();
  };
  u32 flags = 0;
  const u64 stride = (u64)gridDim.x * kTClaimChunk;
  int buf = 0;
  const u64 first = (u64)blockIdx.x * kTClaimChunk;
  if (first < n) fetch(first, seg_of(first), 0);
  // s_segn: segment of the chunk fetched next (warp 0 finds each chunk's
  // successor's while the chunk is reserved)
  if (tid == 0) s_segn = first + stride < n ? seg_of(first + stride) : 0u;
  __syncthreads();
  for (u64 c0 = first; c0 < n; c0 += stride, buf ^= 1) {
    const u64 c1 = c0 + stride;
    // the next chunk's entries travel while this one is claimed
    if (c1 < n) fetch(c1, s_segn, buf ^ 1);
    else cp_async_commit();  // an empty group keeps the wait below uniform
    cp_async_wait_prev();
    u64 x[kTClaimItems];
    u32 c[kTClaimItems], cj[kTClaimItems][NR], rk[kTClaimItems][NR], tbl[kTClaimItems];
    bool win[kTClaimItems];
    u32 need[kTClaimItems];  // bit j: x's cell in sub-table j gets a record
#pragma unroll
    for (int it = 0; it < kTClaimItems; ++it) {
      const u32 i = (u32)(c0 + (u64)it * kTClaimThreads + tid);
      win[it] = i < n;
      x[it] = win[it] ? s_fx[buf][it * kTClaimThreads + tid] : 0ull;
      c[it] = win[it] ? s_fc[buf][it * kTClaimThreads + tid] : 0u;
      tbl[it] = (BATCH && win[it]) ? __ldg(bt.wtab + (c[it] >> 5)) : 0u;
    }
#pragma unroll
    for (int it = 0; it < kTClaimItems; ++it) {
      const TableArgs &T = BATCH ? bt.tabs[tbl[it]] : tab0;
      const int r = rank_of<R>(T);
      cells_of<NR>(x[it], T, cj[it]);
      int js = -1;
#pragma unroll
      for (int j = NR - 1; j >= 0; --j)
        if (j < r && cj[it][j] == c[it]) js = j;
      if (win[it] && js < 0) {
        flags |= FLAG_INTERNAL;
        win[it] = false;
      }
      // the lowest-index cell of x that was pure at the round's start wins;
      // x's cells that were pure at the round's start are empty already
      u32 pure_at_start = 0;
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        if (win[it] && j < r && j != js) {
          const u32 w = __ldcg(bitmap + (cj[it][j] >> 5));
          if ((w >> (cj[it][j] & 31u)) & 1u) pure_at_start |= 1u << j;
        }
      }
      if (win[it] && (pure_at_start & ((1u << (js < 0 ? 0 : js)) - 1u))) win[it] = false;
      need[it] = win[it] ? (((1u << r) - 1u) & ~pure_at_start & ~(1u << (js < 0 ? 0 : js))) : 0u;
    }
#pragma unroll
    for (int it = 0; it < kTClaimItems; ++it) {
      if constexpr (!BATCH) {
        const u32 p = warp_reserve<u32>(win[it], &s_nout);
        if (win[it]) s_out[buf][p] = x[it];
      } else {
        // the warp's winners of one table take one run of its output range
        const TableArgs &T = bt.tabs[tbl[it]];
        const u32 grp = __match_any_sync(kFull, win[it] ? tbl[it] : 0xffffffffu);
        const int leader = __ffs(grp) - 1;
        u64 base = 0;
        if (win[it] && (int)lane_id() == leader) {
          const u32 gsize = __popc(grp);
          const u32 local = round + 1 - T.start_round;
          base = atomicAdd(bt.bc.recovered + tbl[it], (u64)gsize);
          atomicMax(bt.bc.rounds + tbl[it], local);
          if (local <= stats_rounds)
            atomicAdd(bt.bc.round_rec + (u64)tbl[it] * stats_rounds + (local - 1), gsize);
        }
        base = __shfl_sync(kFull, base, leader);
        if (win[it]) {
          const u64 slot = base + __popc(grp & lanemask_lt());
          if (slot < T.out_cap) bt.out[T.out_base + slot] = x[it];
          else flags |= FLAG_CAPACITY;
        }
      }
      // records for the other cells, counted per coarse bin
#pragma unroll
      for (int j = 0; j < NR; ++j)
        rk[it][j] = ((need[it] >> j) & 1u) ? atomicAdd(s_hist + (cj[it][j] >> bsh), 1u) : 0u;
    }
    __syncthreads();
    // bin offsets and cursor reservations (by warp 0 alone for up to 128
    // bins), the output reservation and the next fetch's segment; the
    // histogram and s_nout start over
    auto cursor = [&](u32 k) { return tb.cpos + (u64)k * kTRPosStride; };
    if (nb > 128) {
      block_exclusive_scan<kTClaimThreads>(s_hist, s_scan, nb, s_wt);
      for (u32 k = tid; k < nb; k += kTClaimThreads) {
        const u32 h = s_hist[k];
        s_base[k] = h ? atomicAdd(cursor(k), h) : 0u;
        s_hist[k] = 0;
      }
    }
    if (tid < 32) {
      u32 no = 0;
      u64 ob = 0;
      if (tid == 0) {
        no = s_nout;
        if (no) ob = atomicAdd(&ctl->n_out, (u64)no);
      }
      if (nb <= 128) warp_scan_reserve(s_hist, s_scan, s_base, nb, cursor);
      if (tid == 0) {
        s_nout_cur = no;
        s_nout = 0;
        s_obase = ob;
        s_segn = c1 + stride < n ? seg_of(c1 + stride) : 0u;
      }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kTClaimItems; ++it) {
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        if ((need[it] >> j) & 1u) {
          const u32 pos = s_scan[cj[it][j] >> bsh] + rk[it][j];
          s_key[pos] = x[it];
          s_cell[pos] = cj[it][j];
        }
      }
    }
    __syncthreads();
    // contiguous runs per coarse bin; the bin's region is its tiles' regions
    const u32 total = s_scan[nb];
    for (u32 p = tid; p < total; p += kTClaimThreads) {
      const u32 bn = s_cell[p] >> bsh;
      const u64 dst = (u64)s_bb[bn] * kTRAlign + s_base[bn] + (p - s_scan[bn]);
      if (dst < (u64)s_bb[bn + 1] * kTRAlign && dst < tb.rec_cap) {
        st_l2_policy(tb.crec_key + dst, s_key[p], keep);
        st_l2_policy(tb.crec_cell + dst, s_cell[p], keep);
      } else {
        flags |= FLAG_INTERNAL;  // more records than the bin's counts allow
      }
    }
    const u32 no = s_nout_cur;
    const u64 ob = s_obase;
    for (u32 q = tid; q < no; q += kTClaimThreads) {
      if (ob + q < out_cap) out[ob + q] = s_out[buf][q];
      else flags |= FLAG_CAPACITY;
    }
    // no barrier here: what the next chunk writes before its first barrier
    // (s_out, the fetch buffers, the histogram) is not read from here on,
    // and the rest is written only after that barrier
  }
  if (flags) atomicOr(&ctl->flags, flags);
}

#ifndef PP_TSORT_THREADS
#define PP_TSORT_THREADS 256
#endif
#ifndef PP_TSORT_CTAS
#define PP_TSORT_CTAS 4
#endif
constexpr int kTSortThreads = PP_TSORT_THREADS;
#ifndef PP_TSORT_PER
#define PP_TSORT_PER 8
#endif
constexpr int kTSortPer = PP_TSORT_PER;
constexpr u32 kTSortChunk = kTSortThreads * kTSortPer;  // coarse records per work item
constexpr u32 kMaxBinTiles = 512;                         // tiles per coarse bin (at most)
static_assert(kMaxBinTiles <= 512 && kTSortChunk <= 2048 && kTRShift == 12 && kTSortPer <= 32,
              "k_tsort packs tile (9 bits), cell offset (12) and rank (11) into one word");

// Dynamic shared memory of k_tsort: the chunk prefix over the bins (n_bins + 1
// u32), per bin the round's first and end record and its region's start /
// kTRAlign (3 n_bins + 1 u32), and the chunk's records sorted by tile
// (kTSortChunk keys and offsets).
__host__ __device__ inline size_t tsort_head_bytes(u32 n_bins) { return ((4 * (size_t)n_bins + 2) * 4 + 15) / 16 * 16; }
inline size_t tsort_smem_bytes(u32 n_bins) { return tsort_head_bytes(n_bins) + (size_t)kTSortChunk * (8 + 2); }

// Phase B1': the round's coarse records of each bin, sorted into its tiles'
// record regions (one cursor atomic per tile per chunk of kTSortChunk records).
__global__ void __launch_bounds__(kTSortThreads, PP_TSORT_CTAS) k_tsort(TileRoundBufs tb, DecodeCtl *__restrict__ ctl) {
  if (*(volatile u32 *)&ctl->round == 0) return;  // round 0: F_1 empty or an error, no work
  extern __shared__ __align__(16) unsigned char smem[];
  const u32 nb = tb.n_bins;
  u32 *s_pre = reinterpret_cast<u32 *>(smem);             // nb + 1: chunks before bin b
  u32 *s_blo = s_pre + nb + 1;                            // nb: the round's first record of bin b
  u32 *s_bhi = s_blo + nb;                                // nb: its end
  u32 *s_bb = s_bhi + nb;                                 // nb: region start of bin b / kTRAlign
  u64 *s_key = reinterpret_cast<u64 *>(smem + tsort_head_bytes(nb));  // kTSortChunk
  u16 *s_off = reinterpret_cast<u16 *>(s_key + kTSortChunk);          // kTSortChunk
  __shared__ u32 s_cnt[kMaxBinTiles], s_scan[kMaxBinTiles + 1], s_tb[kMaxBinTiles];
  __shared__ u32 s_tbase[2][kMaxBinTiles + 1];  // the chunk's bin: region start of each tile / kTRAlign
  __shared__ u32 s_wt[kTSortThreads / 32];
  const u32 tid = threadIdx.x;
  const u64 keep = l2_evict_last_policy();
  const u32 ntile = 1u << tb.bin_tshift;
  // chunk counts per bin into s_scan's space first, then their prefix
  // a bin's records end at its cursor, clamped to its region (the claim
  // flagged any record that did not fit, and wrote none past the region)
  auto bin_end = [&](u32 b) -> u32 {
    const u64 rb = tb.base[(u64)b << tb.bin_tshift];
    const u64 re = tb.base[min((b + 1) << tb.bin_tshift, tb.n_tiles)];
    const u32 p = tb.cpos[(u64)b * kTRPosStride];
    return (u64)p < re - rb ? p : (u32)(re - rb);
  };
  for (u32 i = tid; i < ntile; i += kTSortThreads) s_cnt[i] = 0;  // then zeroed after each chunk's scan
  for (u32 b = tid; b < nb; b += kTSortThreads) {
    const u32 lo = tb.cdone[b], hi = bin_end(b);
    s_pre[b] = hi > lo ? (hi - lo + kTSortChunk - 1) / kTSortChunk : 0u;
    s_blo[b] = lo;
    s_bhi[b] = hi;
    s_bb[b] = tb.base64[b << tb.bin_tshift];
  }
  __syncthreads();
  block_exclusive_scan<kTSortThreads>(s_pre, s_pre, nb, s_wt);
  const u32 total = s_pre[nb];
  u32 flags = 0;
  u32 par = 0;  // s_tbase half of this chunk
  for (u32 ch = blockIdx.x; ch < total; ch += gridDim.x, par ^= 1) {
    // bin of this chunk: the last b with s_pre[b] <= ch
    u32 a = 0, bb = nb;
    while (bb - a > 1) {
      const u32 mid = (a + bb) >> 1;
      if (s_pre[mid] <= ch) a = mid;
      else bb = mid;
    }
    const u32 b = a;
    const u64 rb = (u64)s_bb[b] * kTRAlign;
    const u32 lo = s_blo[b] + (ch - s_pre[b]) * kTSortChunk;
    const u32 hi = min(lo + kTSortChunk, s_bhi[b]);
    const u32 t0 = b << tb.bin_tshift;
    u64 x[kTSortPer];
    // a record's cell, then packed: tile in the bin (9 bits), cell in the
    // tile (12 bits), rank among the chunk's records of its tile (11 bits)
    u32 pk[kTSortPer];
    u32 valid = 0;
#pragma unroll
    for (int k = 0; k < kTSortPer; ++k) {
      const u32 i = lo + (u32)k * kTSortThreads + tid;
      const bool v = i < hi;
      x[k] = v ? __ldcs(tb.crec_key + rb + i) : 0ull;
      pk[k] = v ? __ldcs(tb.crec_cell + rb + i) : 0u;
      valid |= (u32)v << k;
    }
    // the bin's tile bounds, loaded while the records are in flight, into
    // the half that the chunk before the previous one read (every thread is
    // past the previous chunk's first barrier, so those reads are done)
    for (u32 i = tid; i <= ntile; i += kTSortThreads) s_tbase[par][i] = tb.base64[min(t0 + i, tb.n_tiles)];
#pragma unroll
    for (int k = 0; k < kTSortPer; ++k) {
      if ((valid >> k) & 1u) {
        const u32 lt = (pk[k] >> kTRShift) - t0;
        const u32 rk = atomicAdd(s_cnt + lt, 1u);
        pk[k] = lt | (pk[k] & (kTRCells - 1)) << 9 | rk << 21;
      }
    }
    __syncthreads();
    // tile offsets and cursor reservations: warp 0 alone for up to 128 tiles
    auto cursor = [&](u32 i) { return tb.pos + (u64)(t0 + i) * kTRPosStride; };
    if (ntile <= 128) {
      if (tid < 32) warp_scan_reserve(s_cnt, s_scan, s_tb, ntile, cursor);
    } else {
      block_exclusive_scan<kTSortThreads>(s_cnt, s_scan, ntile, s_wt);
      for (u32 i = tid; i < ntile; i += kTSortThreads) {
        const u32 h = s_cnt[i];
        s_tb[i] = h ? atomicAdd(cursor(i), h) : 0u;
        s_cnt[i] = 0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTSortPer; ++k) {
      if ((valid >> k) & 1u) {
        const u32 p = s_scan[pk[k] & 511u] + (pk[k] >> 21);
        s_key[p] = x[k];
        s_off[p] = (u16)((pk[k] >> 9) & (kTRCells - 1));
      }
    }
    __syncthreads();
    const u32 nrec = hi > lo ? hi - lo : 0u;
    for (u32 p = tid; p < nrec; p += kTSortThreads) {
      // tile of slot p: the last tile whose run starts at or before p
      u32 l = 0, h2 = ntile;
      while (h2 - l > 1) {
        const u32 mid = (l + h2) >> 1;
        if (s_scan[mid] <= p) l = mid;
        else h2 = mid;
      }
      const u64 dst = (u64)s_tbase[par][l] * kTRAlign + s_tb[l] + (p - s_scan[l]);
      if (dst < (u64)s_tbase[par][l + 1] * kTRAlign && dst < tb.rec_cap) {
        st_l2_policy(tb.rec_key + dst, s_key[p], keep);
        tb.rec_off[dst] = s_off[p];
      } else {
        flags |= FLAG_INTERNAL;  // more records than the tile's counts allow
      }
    }
    // no barrier here: the next chunk writes the other s_tbase half and the
    // (already zeroed) histogram before its first barrier, the rest after it
  }
  if (flags) atomicOr(&ctl->flags, flags);
}

// The tiles with records in the current round (one thread per tile), split
// into sparse (at most kTSCap records) and dense ones; the listed records
// count as consumed from here on (done[t]).
__global__ void __launch_bounds__(kBlock) k_tactive(TileRoundBufs tb, DecodeCtl *__restrict__ ctl) {
  if (*(volatile u32 *)&ctl->round == 0) return;  // round 0: F_1 empty or an error, no work
  // the coarse records of this round are all in their tiles now
  for (u32 b = blockIdx.x * kBlock + threadIdx.x; b < tb.n_bins; b += gridDim.x * kBlock) {
    const u64 rb = tb.base[(u64)b << tb.bin_tshift];
    const u64 re = tb.base[min((b + 1) << tb.bin_tshift, tb.n_tiles)];
    const u32 p = tb.cpos[(u64)b * kTRPosStride];
    tb.cdone[b] = (u64)p < re - rb ? p : (u32)(re - rb);
  }
  for (u32 t0 = blockIdx.x * kBlock; t0 < tb.n_tiles; t0 += gridDim.x * kBlock) {
    const u32 t = t0 + threadIdx.x;
    u32 lo = 0, hi = 0;
    u64 b = 0;
    if (t < tb.n_tiles) {
      lo = tb.done[t];
      b = tb.base[t];
      const u32 p = tb.pos[(u64)t * kTRPosStride], lim = (u32)(tb.base[t + 1] - b);
      hi = p < lim ? p : lim;
      // more records than the tile's counts allow (only a table with deletions
      // could do that): the extra ones landed in the next region
      if (p > lim) atomicOr(&ctl->flags, (u32)FLAG_INTERNAL);
    }
    const bool any = hi > lo;
    const bool dense = any && hi - lo > kTSCap;
    const u32 kd = warp_reserve<u32>(dense, &ctl->n_act_dense);
    const u32 ks = warp_reserve<u32>(any && !dense, &ctl->n_act);
    if (dense) tb.act_d[kd] = TileAct{b + lo, t, hi - lo};
    else if (any) tb.act[ks] = TileAct{b + lo, t, hi - lo};
    if (any) tb.done[t] = hi;  // this round's apply consumes [lo, hi)
  }
}

// Drops the L2 lines of consumed records unwritten (tile regions start on
// 128-byte lines of both record arrays, so no line holds another tile's).
__device__ __forceinline__ void discard_records(const TileRoundBufs &tb, u64 b, u32 n, u32 tid, u32 nthreads) {
  const u64 k0 = (b * 8) & ~127ull, k1 = ((b + n) * 8 + 127) & ~127ull;
  for (u64 a = k0 + (u64)tid * 128; a < k1; a += (u64)nthreads * 128)
    l2_discard(reinterpret_cast<const unsigned char *>(tb.rec_key) + a);
  const u64 o0 = (b * 2) & ~127ull, o1 = ((b + n) * 2 + 127) & ~127ull;
  for (u64 a = o0 + (u64)tid * 128; a < o1; a += (u64)nthreads * 128)
    l2_discard(reinterpret_cast<const unsigned char *>(tb.rec_off) + a);
}

// Shared memory of k_tapply: per cell of a tile the folded key XOR and
// checksum XOR (u64 each), the record count (u32) and the list of touched
// cells (u16).
constexpr size_t kTApplySmem = (size_t)kTRCells * (8 + 8 + 4 + 2);

// Phase B2 of round t + phase A of round t + 1 for the dense tiles (see the
// file comment).  Runs n_seg_d blocks; block b takes the dense tiles b,
// b + n_seg_d, ... and writes frontier segment b.  BATCH: the checksum seeds
// of the tile's 128 words are read into shared memory first.
template <int R, bool BATCH>
__global__ void __launch_bounds__(kTRThreads, 2) k_tapply(Cell *__restrict__ cells, const TableArgs tab0,
                                                          TileRoundBufs tb, u64 *__restrict__ fkey,
                                                          u32 *__restrict__ fcell, u32 *__restrict__ bitmap,
                                                          DecodeCtl *__restrict__ ctl, TRBatch bt) {
  if (*(volatile u32 *)&ctl->round == 0) return;  // round 0: F_1 empty or an error, no work
  extern __shared__ __align__(16) unsigned char smem[];
  u64 *s_dkey = reinterpret_cast<u64 *>(smem);
  u64 *s_dchk = s_dkey + kTRCells;
  u32 *s_dcnt = reinterpret_cast<u32 *>(s_dchk + kTRCells);
  u16 *s_touch = reinterpret_cast<u16 *>(s_dcnt + kTRCells);
  __shared__ u32 s_nt[2], s_seg;  // touched cells of the current tile: two counters, used in turn
  __shared__ u64 s_red[kTRThreads / 32];
  __shared__ u64 s_wseed[BATCH ? kTRCells / 32 : 1];
  const u32 tid = threadIdx.x;
  const u64 seed0 = BATCH ? 0ull : tab0.seed[rank_of<R>(tab0)];
  const u32 n_act = *(volatile u32 *)&ctl->n_act_dense;
  const u64 seg0 = tb.fstart[blockIdx.x];
  u64 emptied = 0, dropped = 0;
  u32 flags = 0;
  if (blockIdx.x < n_act) {  // uniform: blocks with no dense tile skip the set-up
    for (u32 i = tid; i < kTRCells; i += kTRThreads) {
      s_dkey[i] = 0;
      s_dchk[i] = 0;
      s_dcnt[i] = 0;
    }
  }
  if (tid == 0) s_nt[0] = s_nt[1] = 0, s_seg = 0;
  __syncthreads();
  TileAct nxt{};
  if (blockIdx.x < n_act) nxt = tb.act_d[blockIdx.x];
  u32 par = 0;
  for (u32 ai = blockIdx.x; ai < n_act; ai += gridDim.x, par ^= 1) {
    const TileAct cur = nxt;
    if (ai + gridDim.x < n_act) nxt = tb.act_d[ai + gridDim.x];  // the next tile's entry, early
    const u64 b = cur.lo;
    const u32 nrec = cur.n, t = cur.tile;
    if constexpr (BATCH) {
      // the last tile's reads of these seeds ended at its final barrier
      if (tid < kTRCells / 32) s_wseed[tid] = bt.wseed[((u64)t << (kTRShift - 5)) + tid];
      __syncthreads();
    }
    // fold the records into one update per cell (4 records per thread in flight)
    for (u32 i0 = 0; i0 < nrec; i0 += 4 * kTRThreads) {
      u64 x[4];
      u32 o[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const u32 i = i0 + (u32)k * kTRThreads + tid;
        o[k] = i < nrec ? (u32)__ldcs(tb.rec_off + b + i) : 0xffffffffu;
        x[k] = i < nrec ? __ldcs(tb.rec_key + b + i) : 0ull;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool v = o[k] != 0xffffffffu;
        const u32 off = o[k] & (kTRCells - 1);
        bool first = false;
        if (v) {
          const u64 cs = checksum(x[k], BATCH ? s_wseed[off >> 5] : seed0);
          first = atomicAdd(s_dcnt + off, 1u) == 0;
          smem_xor64(s_dkey + off, x[k]);
          smem_xor64(s_dchk + off, cs);
        }
        const u32 q = warp_reserve<u32>(first, &s_nt[par]);
        if (first) s_touch[q] = (u16)off;
      }
    }
    __syncthreads();
    discard_records(tb, b, nrec, tid, kTRThreads);
    // one read-modify-write per touched cell (the loads of a thread's cells in
    // flight together); pure results join F_{t+1} in this block's segment
    const u32 nt = s_nt[par];
    // the other counter was last read before the barrier above: ready it for the next tile
    if (tid == 0) s_nt[par ^ 1] = 0;
    const u32 c0 = t << kTRShift;
    for (u32 k0 = 0; k0 < nt; k0 += kTRCellsPerThread * kTRThreads) {
      u32 off[kTRCellsPerThread];
      bool v[kTRCellsPerThread];
      u64 key[kTRCellsPerThread], chk[kTRCellsPerThread];
      int cnt[kTRCellsPerThread];
#pragma unroll
      for (int q = 0; q < kTRCellsPerThread; ++q) {
        const u32 k = k0 + (u32)q * kTRThreads + tid;
        v[q] = k < nt;
        off[q] = v[q] ? s_touch[k] : 0u;
        key[q] = chk[q] = 0;
        cnt[q] = 0;
        if (v[q]) ld_cell_cg(cells + c0 + off[q], key[q], chk[q], cnt[q]);
      }
#pragma unroll
      for (int q = 0; q < kTRCellsPerThread; ++q) {
        bool pure = false;
        u64 nk = 0;
        if (v[q]) {
          const u32 c = c0 + off[q];
          const int nc = cnt[q] - (int)s_dcnt[off[q]];
          nk = key[q] ^ s_dkey[off[q]];
          const u64 nchk = chk[q] ^ s_dchk[off[q]];
          pure = cell_pure(nc, nk, nchk, BATCH ? s_wseed[off[q] >> 5] : seed0);
          // a pure cell is stored empty: its one key leaves it next round
          if (pure) st_cell_cs(cells + c, 0ull, 0ull, 0);
          else st_cell_cs(cells + c, nk, nchk, nc);
          emptied += (u64)(long long)((cnt[q] != 0) - (!pure && nc != 0));
          dropped += cnt[q] >= 2 && nc < 2;
          s_dcnt[off[q]] = 0;
          s_dkey[off[q]] = 0;
          s_dchk[off[q]] = 0;
        }
        const u32 p = warp_reserve<u32>(pure, &s_seg);
        if (pure && p < tb.cap_d) {
          const u32 c = c0 + off[q];
          fkey[seg0 + p] = nk;
          fcell[seg0 + p] = c;
          atomicOr(bitmap + (c >> 5), 1u << (c & 31u));
        } else if (pure) {
          flags |= FLAG_INTERNAL;  // cannot happen: a segment holds every push of its block's tiles
        }
      }
    }
    __syncthreads();
  }
  const u64 e = block_sum<u64, kTRThreads>(emptied, s_red);
  const u64 d = block_sum<u64, kTRThreads>(dropped, s_red);
  if (tid == 0) {
    if (e) atomicAdd(&ctl->emptied, e);
    if (d) atomicAdd(&ctl->n_cand, (u32)d);
    tb.fseg[blockIdx.x] = s_seg;
    if (s_seg) atomicAdd(&ctl->n_next, s_seg);
  }
  if (flags) atomicOr(&ctl->flags, flags);
}

// Shared memory of k_tapply_sparse: two hash tables (slot -> cell offset,
// folded key XOR, checksum XOR, record count) and their touched-slot lists.
constexpr size_t kTSSmem = 2 * (size_t)kTSSlots * (4 + 8 + 8 + 4) + 2 * (size_t)kTSCap * 2;

// The same for the sparse tiles, with a small hash table (open addressing on
// the cell offset) in place of the per-cell arrays, so that many tiles are in
// flight per SM; block b takes the sparse tiles b, b + n_seg_s, ... (at most
// kTSCap records, hence pushes, each).  The block keeps two tables: while
// the cells of tile k are loaded from memory, the records of tile k + 1 (in
// registers since the previous step) are folded into the other table, and the
// records of tile k + 2 are fetched; one barrier per tile.  Tile k uses table
// k % 2, touched-slot counter k % 3 and (BATCH) seed buffer k % 3: a counter
// or seed buffer is written again only after the barrier that follows its
// last read.  Runs n_seg_s blocks; block b writes frontier segment n_seg_d + b.
template <int R, bool BATCH>
__global__ void __launch_bounds__(kTSThreads, kTSCtas) k_tapply_sparse(Cell *__restrict__ cells, const TableArgs tab0,
                                                                 TileRoundBufs tb, u64 *__restrict__ fkey,
                                                                 u32 *__restrict__ fcell, u32 *__restrict__ bitmap,
                                                                 DecodeCtl *__restrict__ ctl, TRBatch bt) {
  if (*(volatile u32 *)&ctl->round == 0) return;  // round 0: F_1 empty or an error, no work
  extern __shared__ __align__(16) unsigned char smem[];
  u64 *h_key = reinterpret_cast<u64 *>(smem);            // 2 x kTSSlots
  u64 *h_chk = h_key + 2 * kTSSlots;                     // 2 x kTSSlots
  u32 *h_off = reinterpret_cast<u32 *>(h_chk + 2 * kTSSlots);  // 2 x kTSSlots, kTSEmpty if free
  u32 *h_cnt = h_off + 2 * kTSSlots;                     // 2 x kTSSlots
  u16 *s_slot = reinterpret_cast<u16 *>(h_cnt + 2 * kTSSlots);  // 2 x kTSCap: the slots in use
  __shared__ u32 s_ns[3], s_seg;
  __shared__ u64 s_red[kTSThreads / 32];
  constexpr u32 kW = kTRCells / 32;  // words of a tile
  static_assert(!BATCH || kTSThreads >= (int)kW, "one thread per word of a tile");
  __shared__ u64 s_wseed[BATCH ? 3 : 1][BATCH ? kW : 1];
  const u32 tid = threadIdx.x;
  const u64 seed0 = BATCH ? 0ull : tab0.seed[rank_of<R>(tab0)];
  const u32 n_act = *(volatile u32 *)&ctl->n_act;
  const u64 seg0 = tb.fstart[tb.n_seg_d + blockIdx.x];
  const u32 g = gridDim.x;
  u32 flags = 0;
  for (u32 i = tid; i < 2 * kTSSlots; i += kTSThreads) {
    h_off[i] = kTSEmpty;
    h_key[i] = 0;
    h_chk[i] = 0;
    h_cnt[i] = 0;
  }
  if (tid == 0) s_ns[0] = s_ns[1] = s_ns[2] = 0, s_seg = 0;
  u64 emptied = 0, dropped = 0;
  constexpr int PER = kTSCap / kTSThreads;
  static_assert(kTSCap % kTSThreads == 0, "a sparse tile's records split evenly over the threads");
  auto entry = [&](u32 ai) {
    TileAct a{};
    if (ai < n_act) a = tb.act[ai];
    return a;
  };
  // a tile's records (and BATCH: its word seed for thread tid) into registers
  u64 x[PER];
  u32 o[PER];
  u64 nws = 0;
  auto fetch = [&](const TileAct &a) {
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const u32 i = (u32)k * kTSThreads + tid;
      o[k] = i < a.n ? (u32)__ldcs(tb.rec_off + a.lo + i) : kTSEmpty;
      x[k] = i < a.n ? __ldcs(tb.rec_key + a.lo + i) : 0ull;
    }
    if (BATCH && tid < kW && a.n) nws = bt.wseed[((u64)a.tile << (kTRShift - 5)) + tid];
  };
  // folds the records in registers into table hb (touched slots counted in
  // s_ns[cb], listed in s_slot), checksums with seed buffer sb
  auto fold = [&](u32 hb, u32 cb, u32 sb) {
    u32 *ho = h_off + hb * kTSSlots, *hc = h_cnt + hb * kTSSlots;
    u64 *hk = h_key + hb * kTSSlots, *hx = h_chk + hb * kTSSlots;
    u16 *sl = s_slot + hb * kTSCap;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      bool fresh = false;
      u32 slot = 0;
      u32 ok = o[k];
      if (ok != kTSEmpty) {
        const u32 off = ok & (kTRCells - 1);
        slot = off & (kTSSlots - 1);
        // at most kTSCap of the kTSSlots slots are taken, so a free or matching
        // slot is found within kTSCap + 1 probes
        bool found = false;
        for (u32 probe = 0; probe <= kTSCap; ++probe) {
          const u32 prev = atomicCAS(ho + slot, kTSEmpty, off);
          if (prev == kTSEmpty || prev == off) {
            fresh = prev == kTSEmpty;
            found = true;
            break;
          }
          slot = (slot + 1) & (kTSSlots - 1);
        }
        if (!found) {
          flags |= FLAG_INTERNAL;
          ok = kTSEmpty;
        }
      }
      if (ok != kTSEmpty) {
        const u64 cs = checksum(x[k], BATCH ? s_wseed[sb][(ok & (kTRCells - 1)) >> 5] : seed0);
        atomicAdd(hc + slot, 1u);
        smem_xor64(hk + slot, x[k]);
        smem_xor64(hx + slot, cs);
      }
      const u32 q = warp_reserve<u32>(fresh, &s_ns[cb]);
      if (fresh) sl[q] = (u16)slot;
    }
  };
  // prologue: tile 0 folded into table 0, tile 1's records in registers
  TileAct cur = entry(blockIdx.x), a1 = entry(blockIdx.x + g), a2 = entry(blockIdx.x + 2 * g);
  fetch(cur);
  if (BATCH && tid < kW) s_wseed[0][tid] = nws;
  __syncthreads();  // tables, counters and seeds of tile 0 ready
  if (cur.n) {
    fold(0, 0, 0);
    discard_records(tb, cur.lo, cur.n, tid, kTSThreads);
  }
  fetch(a1);
  if (BATCH && tid < kW) s_wseed[1][tid] = nws;
  __syncthreads();
  u32 k = 0;
  for (u32 ai = blockIdx.x; ai < n_act; ai += g, ++k) {
    const u32 hb = k & 1u, cb = k % 3u;
    const u32 ns = s_ns[cb];
    const u32 c0 = cur.tile << kTRShift;
    const u32 *ho = h_off + hb * kTSSlots, *hc = h_cnt + hb * kTSSlots;
    const u64 *hk = h_key + hb * kTSSlots, *hx = h_chk + hb * kTSSlots;
    const u16 *sl = s_slot + hb * kTSCap;
    // the cells of tile k: every load in flight before any store (the cell
    // accesses are volatile asm, kept in program order)
    u32 slots[PER], cs[PER];
    u64 keys[PER], chks[PER];
    int cnts[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const u32 qq = (u32)q * kTSThreads + tid;
      slots[q] = cs[q] = 0;
      keys[q] = chks[q] = 0;
      cnts[q] = 0;
      if (qq < ns) {
        slots[q] = sl[qq];
        cs[q] = c0 + ho[slots[q]];
        ld_cell_cg(cells + cs[q], keys[q], chks[q], cnts[q]);
      }
    }
    // while they travel: tile k + 1 into the other table, tile k + 2 fetched
    if (a1.n) {
      fold(hb ^ 1u, (k + 1) % 3u, (k + 1) % 3u);
      discard_records(tb, a1.lo, a1.n, tid, kTSThreads);
    }
    const TileAct a3 = entry(ai + 3 * g);
    fetch(a2);
    const u32 sb = k % 3u;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const u32 qq = (u32)q * kTSThreads + tid;
      const bool v = qq < ns;
      const u32 slot = slots[q], c = cs[q];
      u64 key = keys[q], chk = chks[q];
      const int cnt = cnts[q];
      bool pure = false;
      if (v) {
        const int nc = cnt - (int)hc[slot];
        key ^= hk[slot];
        chk ^= hx[slot];
        pure = cell_pure(nc, key, chk, BATCH ? s_wseed[sb][(c - c0) >> 5] : seed0);
        // a pure cell is stored empty: its one key leaves it next round
        if (pure) st_cell_cs(cells + c, 0ull, 0ull, 0);
        else st_cell_cs(cells + c, key, chk, nc);
        emptied += (u64)(long long)((cnt != 0) - (!pure && nc != 0));
        dropped += cnt >= 2 && nc < 2;
        u32 *hom = h_off + hb * kTSSlots, *hcm = h_cnt + hb * kTSSlots;
        u64 *hkm = h_key + hb * kTSSlots, *hxm = h_chk + hb * kTSSlots;
        hom[slot] = kTSEmpty;
        hkm[slot] = 0;
        hxm[slot] = 0;
        hcm[slot] = 0;
      }
      const u32 p = warp_reserve<u32>(pure, &s_seg);
      if (pure && p < tb.cap_s) {
        fkey[seg0 + p] = key;
        fcell[seg0 + p] = c;
        atomicOr(bitmap + (c >> 5), 1u << (c & 31u));
      } else if (pure) {
        flags |= FLAG_INTERNAL;  // cannot happen: a segment holds every push of its block's tiles
      }
    }
    // tile k + 2's seeds and counter: their buffers were last read by tile
    // k - 1, before the previous barrier
    if (BATCH && tid < kW) s_wseed[(k + 2) % 3u][tid] = nws;
    if (tid == 0) s_ns[(k + 2) % 3u] = 0;
    cur = a1;
    a1 = a2;
    a2 = a3;
    __syncthreads();
  }
  const u64 e = block_sum<u64, kTSThreads>(emptied, s_red);
  const u64 d = block_sum<u64, kTSThreads>(dropped, s_red);
  if (tid == 0) {
    if (e) atomicAdd(&ctl->emptied, e);
    if (d) atomicAdd(&ctl->n_cand, (u32)d);
    tb.fseg[tb.n_seg_d + blockIdx.x] = s_seg;
    if (s_seg) atomicAdd(&ctl->n_next, s_seg);
  }
  if (flags) atomicOr(&ctl->flags, flags);
}

}  // namespace pp
