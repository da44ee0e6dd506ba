// Binned decode round: the round of Sec. 1 (at k = 2, on the IBLT hypergraph
// of Sec. 6) split so that its cell updates reach HBM in address order.
//
//   k_claim  (phase B1) for every frontier entry (cell c, key x snapshotted at
//            the round's start): c recovers x iff no lower-sub-table cell of x
//            was pure at the round's start (the same lowest-index rule as
//            k_peel).  A winner writes x to the output and one update record
//            (cell, key) per cell of x into the bin of that cell: bins are
//            2^19 consecutive cells (8 MB).  Records are ordered by bin inside
//            the block and leave it as contiguous runs.
//   k_apply_round (phase B2) walks the records bin by bin: blocks take the next
//            chunk of 2048 records from an atomic counter, so at any moment the
//            whole GPU updates a narrow, moving window of the table and HBM
//            sees near-sequential traffic.  Each update is an atomicAdd on
//            the cell's count and an atomicXor on each of its key and
//            checksum fields; a count that drops from 2 to 1 makes the
//            cell a candidate for the next frontier.
// Updates commute, so the order of application does not change the state at
// the end of the round; the claim decisions are all taken in B1, before any
// update of the round lands.
#pragma once

#include "iblt_types.cuh"

namespace pp {

// Removes key x (checksum cs) taken with sign sg from cell c; returns the
// cell's count before the removal.
__device__ __forceinline__ int remove_key(Cell *cells, u32 c, u64 x, u64 cs, int sg = 1) {
  return touch_cell(cells, c, x, cs, -sg);
}

// A cell becomes a candidate for the next frontier when its count reaches 1
// (2 -> 1 in the plain decode; +-1 from any count in the signed one, where a
// cell may get there more than once and the filter keeps its first entry).
template <bool SIGNED>
__device__ __forceinline__ bool becomes_candidate(int old, int sg) {
  const int now = old - sg;
  return SIGNED ? (now == 1 || now == -1) : old == 2;
}

// Shared memory of k_claim: staged records (keys and cells, plus tables in a
// batch: kClaimChunk*NR each) + the plain decode's output staging (kClaimChunk
// u64) + 3 * n_bins u32.

// Registers capped for 5 resident CTAs per SM for plain tables of rank 3 or 4
// (48 per thread, a few spilled, beat 4 CTAs at 64) and for 4 otherwise (the
// generic and batched instances would take 106-154 registers uncapped).
// CLAIM = false (decode with sub-tables): every frontier entry recovers its key
// -- within one sub-table no key is found twice -- so the bitmap is not read.
// SIGNED (sparse recovery, plain tables): each frontier entry carries the sign
// of its cell's count; the winner outputs it, and its records carry it in bit
// 31 of the cell (signed tables have fewer than 2^31 cells).
template <int R, bool BATCH, bool CLAIM = true, bool SIGNED = false>
__global__ void __launch_bounds__(kBlock, (!BATCH && R >= 3) ? 5 : 4) k_claim(Cell *__restrict__ cells, const TableArgs tab0,
                                                  const TableArgs *__restrict__ tabs,
                                                  const u64 *__restrict__ fkey, const u32 *__restrict__ fcell,
                                                  const u32 *__restrict__ ftab, const u32 *__restrict__ bitmap,
                                                  RoundBins rb, u32 *__restrict__ cand, u32 *__restrict__ ctab,
                                                  u64 *__restrict__ bout, DecodeCtl *__restrict__ ctl,
                                                  BatchCounters bc) {
  constexpr int NR = nr_of<R>();
  constexpr int CAP = kClaimChunk * NR;
  constexpr u32 kCellMask = SIGNED ? 0x7fffffffu : 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem[];
  u64 *s_key = reinterpret_cast<u64 *>(smem);       // CAP
  u64 *s_out = s_key + CAP;                         // kClaimChunk (plain)
  u32 *s_cell = reinterpret_cast<u32 *>(s_out + kClaimChunk);
  u32 *s_tab = s_cell + CAP;                        // CAP (batch)
  u32 *s_hist = s_tab + (BATCH ? CAP : 0);          // n_bins
  u32 *s_scan = s_hist + rb.n_bins;
  u32 *s_base = s_scan + rb.n_bins;
  signed char *s_osign = reinterpret_cast<signed char *>(s_base + rb.n_bins);  // kClaimChunk (signed)
  __shared__ u32 s_wt[33];
  __shared__ u32 s_total, s_nout;
  __shared__ u64 s_obase;
  const u32 tid = threadIdx.x;
  const u32 nb = rb.n_bins;
  const u32 n = *(volatile u32 *)&ctl->n_front;
  const u32 round = *(volatile u32 *)&ctl->round;
  u64 *out = BATCH ? bout : ctl->out;
  const u64 out_cap = BATCH ? 0 : ctl->out_cap;
  const u32 stats_rounds = BATCH ? ctl->stats_rounds : 0;
  u32 flags = 0, n_neg = 0;
  u64 ovf_emptied = 0;
  for (u64 c0 = (u64)blockIdx.x * kClaimChunk; c0 < n; c0 += (u64)gridDim.x * kClaimChunk) {
    for (u32 i = tid; i < nb; i += kBlock) s_hist[i] = 0;
    if (tid == 0) s_nout = 0;
    __syncthreads();
    u64 x[kClaimItems];
    u32 cj[kClaimItems][NR], rank[kClaimItems][NR], tb[kClaimItems];
    bool win[kClaimItems];
    int rr[kClaimItems];
    signed char sg[kClaimItems];
    // load every entry of this thread first (independent loads in flight)
    u32 c[kClaimItems];
#pragma unroll
    for (int it = 0; it < kClaimItems; ++it) {
      const u64 i = c0 + (u64)it * kBlock + tid;
      const bool valid = i < n;
      x[it] = valid ? __ldcs(fkey + i) : 0ull;
      c[it] = valid ? __ldcs(fcell + i) : 0u;
      tb[it] = (BATCH && valid) ? __ldcs(ftab + i) : 0u;
      sg[it] = (SIGNED && valid) ? rb.fsign[i] : (signed char)1;
      win[it] = valid;
    }
#pragma unroll
    for (int it = 0; it < kClaimItems; ++it) {
      const TableArgs &T = BATCH ? tabs[tb[it]] : tab0;
      const int r = rank_of<R>(T);
      rr[it] = r;
      cells_of<NR>(x[it], T, cj[it]);
      int jstar = -1;
#pragma unroll
      for (int j = NR - 1; j >= 0; --j)
        if (j < r && cj[it][j] == c[it]) jstar = j;
      if (win[it] && jstar < 0) {
        flags |= FLAG_INTERNAL;
        win[it] = false;
      }
      // the lowest-index cell of x that was pure at the round's start wins
#pragma unroll
      for (int j = 0; j < NR - 1; ++j) {
        if (CLAIM && win[it] && j < jstar) {
          const u32 w = __ldcg(bitmap + (cj[it][j] >> 5));
          if ((w >> (cj[it][j] & 31u)) & 1u) win[it] = false;
        }
      }
    }
#pragma unroll
    for (int it = 0; it < kClaimItems; ++it) {
      // recovered key
      if constexpr (!BATCH) {
        const u32 p = warp_reserve<u32>(win[it], &s_nout);
        if (win[it]) {
          s_out[p] = x[it];
          if (SIGNED) s_osign[p] = sg[it];
        }
        if (SIGNED) n_neg += win[it] && sg[it] < 0;
      } else {
        const TableArgs &T = tabs[tb[it]];
        const u32 label = win[it] ? tb[it] : 0xffffffffu;
        const u32 grp = __match_any_sync(kFull, label);
        const int leader = __ffs(grp) - 1;
        const u32 gsize = __popc(grp);
        u64 base = 0;
        if (win[it] && (int)lane_id() == leader) {
          const u32 local = round + 1 - T.start_round;
          base = atomicAdd(bc.recovered + tb[it], (u64)gsize);
          atomicMax(bc.rounds + tb[it], local);
          if (local <= stats_rounds)
            atomicAdd(bc.round_rec + (u64)tb[it] * stats_rounds + (local - 1), gsize);
        }
        base = __shfl_sync(kFull, base, leader);
        if (win[it]) {
          const u64 slot = base + __popc(grp & lanemask_lt());
          if (slot < T.out_cap) out[T.out_base + slot] = x[it];
          else flags |= FLAG_CAPACITY;
        }
      }
      // update records, counted per bin
#pragma unroll
      for (int j = 0; j < NR; ++j)
        rank[it][j] = (win[it] && j < rr[it]) ? atomicAdd(s_hist + (cj[it][j] >> rb.shift), 1u) : 0u;
    }
    __syncthreads();
    // exclusive scan of the histogram: thread t owns bins [t*per, (t+1)*per)
    const u32 per = (nb + kBlock - 1) / kBlock;
    const u32 lo = tid * per, hi = lo + per < nb ? lo + per : nb;
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
      const u32 w = tid < kBlock / 32 ? s_wt[tid] : 0;
      u32 wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(kFull, wi, o);
        if ((int)tid >= o) wi += y;
      }
      if (tid < kBlock / 32) s_wt[tid] = wi - w;
      if (tid == 31) s_total = wi;
      if (!BATCH && tid == 0 && s_nout) s_obase = atomicAdd(&ctl->n_out, (u64)s_nout);
    }
    __syncthreads();
    u32 run = s_wt[tid >> 5] + inc - own;
    for (u32 k = lo; k < hi; ++k) {
      s_scan[k] = run;
      const u32 h = s_hist[k];
      s_base[k] = h ? atomicAdd(rb.count + k, h) : 0u;
      run += h;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kClaimItems; ++it) {
      if (win[it]) {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (j < rr[it]) {
            const u32 bn = cj[it][j] >> rb.shift;
            const u32 pos = s_scan[bn] + rank[it][j];
            s_key[pos] = x[it];
            s_cell[pos] = cj[it][j] | ((SIGNED && sg[it] < 0) ? 0x80000000u : 0u);
            if (BATCH) s_tab[pos] = tb[it];
          }
        }
      }
    }
    __syncthreads();
    const u32 total = s_total;
    for (u32 p = tid; p < total; p += kBlock) {
      const u32 bn = (s_cell[p] & kCellMask) >> rb.shift;
      const u32 slot = s_base[bn] + (p - s_scan[bn]);
      if (slot < rb.cap) {
        const u64 dst = (u64)bn * rb.cap + slot;
        rb.rec_key[dst] = s_key[p];
        rb.rec_cell[dst] = s_cell[p];
        if (BATCH) rb.rec_tab[dst] = s_tab[p];
      } else {
        // the bin is full: apply this update right away (updates commute)
        const u32 t2 = BATCH ? s_tab[p] : 0u;
        const u64 seed_chk = BATCH ? bc.chk_seed[t2] : tab0.seed[rank_of<R>(tab0)];
        const u64 xx = s_key[p];
        const u32 cc = s_cell[p] & kCellMask;
        const int sgn = (SIGNED && (s_cell[p] >> 31)) ? -1 : 1;
        const int old = remove_key(cells, cc, xx, checksum(xx, seed_chk), sgn);
        if (becomes_candidate<SIGNED>(old, sgn)) {
          const u32 q = atomicAdd(&ctl->n_cand, 1u);
          if (!SIGNED || q < rb.cand_cap) cand[q] = cc;
          else flags |= FLAG_INTERNAL;
          if (BATCH) ctab[q] = t2;
        }
        if (!BATCH) ovf_emptied += (u64)(long long)((old != 0) - (old - sgn != 0));
      }
    }
    if constexpr (!BATCH) {
      const u32 no = s_nout;
      const u64 ob = s_obase;
      for (u32 q = tid; q < no; q += kBlock) {
        if (ob + q < out_cap) {
          out[ob + q] = s_out[q];
          if (SIGNED && rb.osign) rb.osign[ob + q] = s_osign[q];
        } else {
          flags |= FLAG_CAPACITY;
        }
      }
    }
    __syncthreads();
  }
  if (SIGNED && n_neg) atomicAdd(&ctl->n_neg, n_neg);
  if (ovf_emptied) atomicAdd(&ctl->emptied, ovf_emptied);
  if (flags) atomicOr(&ctl->flags, flags);
}

// Shared memory of k_apply_round: chunk prefix (n_bins + 1 u32) + pushes
// (kApplyChunk cells [+ tables]).
template <int R, bool BATCH, bool SIGNED = false>
__global__ void __launch_bounds__(kBlock) k_apply_round(Cell *__restrict__ cells, const TableArgs tab0,
                                                        const TableArgs *__restrict__ tabs, RoundBins rb,
                                                        u32 *__restrict__ cand, u32 *__restrict__ ctab,
                                                        DecodeCtl *__restrict__ ctl, BatchCounters bc) {
  extern __shared__ __align__(16) unsigned char smem[];
  u32 *s_pre = reinterpret_cast<u32 *>(smem);       // n_bins + 1
  u32 *s_cand = s_pre + rb.n_bins + 1;              // kApplyChunk
  u32 *s_ctab = s_cand + kApplyChunk;               // kApplyChunk (batch)
  __shared__ u32 s_wt[33];
  __shared__ u32 s_chunk, s_ncand, s_cbase;
  __shared__ u64 s_red[kBlock / 32];
  const u32 tid = threadIdx.x;
  const u32 nb = rb.n_bins;
  // chunk prefix over the bins (every block computes it)
  const u32 per = (nb + kBlock - 1) / kBlock;
  const u32 lo = tid * per, hi = lo + per < nb ? lo + per : nb;
  u32 own = 0;
  for (u32 k = lo; k < hi; ++k) {
    const u32 cnt = rb.count[k];
    own += ((cnt < rb.cap ? cnt : rb.cap) + kApplyChunk - 1) / kApplyChunk;
  }
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
    if (tid == 31) s_pre[nb] = wi;
  }
  __syncthreads();
  {
    u32 run = s_wt[tid >> 5] + inc - own;
    for (u32 k = lo; k < hi; ++k) {
      s_pre[k] = run;
      const u32 cnt = rb.count[k];
      run += ((cnt < rb.cap ? cnt : rb.cap) + kApplyChunk - 1) / kApplyChunk;
    }
  }
  if (tid == 0) s_ncand = 0;
  __syncthreads();
  const u32 total = s_pre[nb];
  u64 emptied = 0;
  for (;;) {
    if (tid == 0) s_chunk = atomicAdd(&ctl->apply_next, 1u);
    __syncthreads();
    const u32 chunk = s_chunk;
    if (chunk >= total) break;
    // bin of this chunk: last k with s_pre[k] <= chunk
    u32 a = 0, b = nb;
    while (b - a > 1) {
      const u32 mid = (a + b) >> 1;
      if (s_pre[mid] <= chunk) a = mid;
      else b = mid;
    }
    const u32 bn = a;
    const u32 cnt = rb.count[bn];
    const u32 in_bin = cnt < rb.cap ? cnt : rb.cap;
    const u32 first = (chunk - s_pre[bn]) * kApplyChunk;
    const u64 base = (u64)bn * rb.cap;
    // Loads of every record of this thread first, then every update, then
    // the pushes: kApplyPer records' atomics are in flight at once.
    u64 x[kApplyPer], seed_chk[kApplyPer];
    u32 c[kApplyPer], tb[kApplyPer];
    bool v[kApplyPer];
    int old[kApplyPer], sg[kApplyPer];
#pragma unroll
    for (int k = 0; k < kApplyPer; ++k) {
      const u32 i = first + (u32)k * kBlock + tid;
      v[k] = i < in_bin;
      x[k] = v[k] ? __ldcs(rb.rec_key + base + i) : 0ull;
      c[k] = v[k] ? __ldcs(rb.rec_cell + base + i) : 0u;
      tb[k] = (BATCH && v[k]) ? __ldcs(rb.rec_tab + base + i) : 0u;
      sg[k] = (SIGNED && (c[k] >> 31)) ? -1 : 1;
      if (SIGNED) c[k] &= 0x7fffffffu;
    }
#pragma unroll
    for (int k = 0; k < kApplyPer; ++k)
      seed_chk[k] = BATCH ? (v[k] ? bc.chk_seed[tb[k]] : 0ull) : tab0.seed[rank_of<R>(tab0)];
#pragma unroll
    for (int k = 0; k < kApplyPer; ++k)
      old[k] = v[k] ? remove_key(cells, c[k], x[k], checksum(x[k], seed_chk[k]), sg[k]) : 0;
#pragma unroll
    for (int k = 0; k < kApplyPer; ++k) {
      const bool push = v[k] && becomes_candidate<SIGNED>(old[k], sg[k]);
      const u32 q = warp_reserve<u32>(push, &s_ncand);
      if (push) {
        s_cand[q] = c[k];
        if (BATCH) s_ctab[q] = tb[k];
      }
      // batched decodes count their residue with k_residual afterwards
      if (!BATCH && v[k]) emptied += (u64)(long long)((old[k] != 0) - (old[k] - sg[k] != 0));
    }
    __syncthreads();
    const u32 nc = s_ncand;
    if (tid == 0 && nc) s_cbase = atomicAdd(&ctl->n_cand, nc);
    __syncthreads();
    for (u32 q = tid; q < nc; q += kBlock) {
      if (SIGNED && (u64)s_cbase + q >= rb.cand_cap) {
        atomicOr(&ctl->flags, (u32)FLAG_INTERNAL);
        continue;
      }
      cand[s_cbase + q] = s_cand[q];
      if (BATCH) ctab[s_cbase + q] = s_ctab[q];
    }
    __syncthreads();
    if (tid == 0) s_ncand = 0;
  }
  if (!BATCH) {
    const u64 e = block_sum<u64, kBlock>(emptied, s_red);
    if (tid == 0 && e) atomicAdd(&ctl->emptied, e);
  }
}

// Residue of a batched binned decode: non-empty cells per table, one chunk of
// one table per step (tables that recovered every key and saw no deletion are
// empty by construction and skipped).
__global__ void __launch_bounds__(kBlock) k_residual(const Cell *__restrict__ cells,
                                                     const Chunk *__restrict__ chunks, u32 n_chunks,
                                                     BatchCounters bc) {
  __shared__ u64 s_red[kBlock / 32];
  for (u32 ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const Chunk k = chunks[ch];
    if (bc.skip_full && bc.recovered[k.table] >= bc.items[k.table]) continue;  // uniform per block
    u64 nz = 0;
    for (u32 c = k.begin + threadIdx.x; c < k.end; c += kBlock) nz += cells[c].count != 0;
    const u64 t = block_sum<u64, kBlock>(nz, s_red);
    if (threadIdx.x == 0 && t) atomicAdd(bc.residual + k.table, t);
  }
}

// End of a binned round: clears the bins and the apply work counter for the
// next round.
__global__ void k_bins_reset(RoundBins rb, DecodeCtl *__restrict__ ctl) {
  for (u32 i = threadIdx.x; i < rb.n_bins; i += blockDim.x) rb.count[i] = 0;
  if (threadIdx.x == 0) ctl->apply_next = 0;
}

}  // namespace pp
