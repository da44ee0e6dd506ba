// IBLT kernels: build, initial full scan, per-round peel and frontier filter.
//
// The recovery is the round-synchronous k = 2 peel of Sec. 1 applied to the
// IBLT hypergraph of Sec. 6 (cells = vertices, keys = edges):
//   round t recovers every key that is alone in some cell at the start of the
//   round, exactly once, and deletes it from its r cells.
// Each round is two kernels:
//   peel   (phase B)  for every frontier entry (cell c, key x snapshot taken
//                     at the start of the round) decide whether c is the
//                     lowest-index cell of x that was pure at the round's
//                     start; if so recover x and XOR it out of its r cells.
//                     A cell whose count drops from 2 to 1 becomes a candidate.
//   filter (phase A)  keep the candidates that are pure once the round is
//                     over, snapshot their keys and mark them in the
//                     "pure at round start" bitmap: the next frontier.
// The kernel boundary between the two phases is what makes the snapshot and
// the bitmap describe the round's start.  A cell is pure at the start of at
// most one round in the whole decode (its count then drops to 0 and never
// rises), so the bitmap needs no clearing between rounds.
#pragma once

#include "iblt_types.cuh"

namespace pp {



// --------------------------------------------------------------------------
// Build (Sec. 6 "Motivation"; one thread per key as in Sec. 6 "Implementation
// Details", with fire-and-forget atomics: nothing reads their results).
// --------------------------------------------------------------------------
template <int R, bool BATCH>
__global__ void __launch_bounds__(kBlock) k_insert(Cell *__restrict__ cells, const TableArgs tab0,
                                                   const TableArgs *__restrict__ tabs,
                                                   const Chunk *__restrict__ chunks, u32 n_chunks,
                                                   const u64 *__restrict__ keys, u64 m, int sign) {
  constexpr int NR = nr_of<R>();
  if (!BATCH) {
    const int r = rank_of<R>(tab0);
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
      const u64 x = __ldcs(keys + i);
      u32 c[NR];
      cells_of<NR>(x, tab0, c);
      const u64 cs = checksum(x, tab0.seed[r]);
#pragma unroll
      for (int j = 0; j < NR; ++j)
        if (j < r) touch_cell_nr(cells, c[j], x, cs, sign);
    }
  } else {
    for (u32 ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
      const Chunk k = chunks[ch];
      const TableArgs &T = tabs[k.table];
      const int r = rank_of<R>(T);
      for (u32 i = k.begin + threadIdx.x; i < k.end; i += blockDim.x) {
        const u64 x = __ldcs(keys + i);
        u32 c[NR];
        cells_of<NR>(x, T, c);
        const u64 cs = checksum(x, T.seed[r]);
#pragma unroll
        for (int j = 0; j < NR; ++j)
          if (j < r) touch_cell_nr(cells, c[j], x, cs, sign);
      }
    }
  }
}

// --------------------------------------------------------------------------
// Initial full scan: F_1 = cells pure before any round; sets their bits.
// Every 32-cell bitmap word of the table is written here (whole word per warp),
// so a previous decode's bits never leak into this one.
// --------------------------------------------------------------------------
template <int R, bool BATCH>
__global__ void __launch_bounds__(kBlock) k_scan(const Cell *__restrict__ cells, const TableArgs tab0,
                                                 const TableArgs *__restrict__ tabs,
                                                 const Chunk *__restrict__ chunks, u32 n_chunks,
                                                 u64 *__restrict__ fkey, u32 *__restrict__ fcell,
                                                 u32 *__restrict__ ftab, u32 *__restrict__ bitmap,
                                                 DecodeCtl *__restrict__ ctl, BatchCounters bc) {
  constexpr int CH = kBlock * kScanItems;
  __shared__ u64 s_key[CH];
  __shared__ u32 s_cell[CH];
  __shared__ u32 s_n, s_base;
  __shared__ u64 s_red[kBlock / 32];
  const u32 tid = threadIdx.x;
  u64 alive = 0, nonempty = 0;
  if (tid == 0) s_n = 0;
  __syncthreads();
  for (u32 ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    u32 begin, end, table = 0;
    if (BATCH) {
      const Chunk k = chunks[ch];
      begin = k.begin, end = k.end, table = k.table;
    } else {
      begin = ch * (u32)CH;
      end = min(begin + (u32)CH, tab0.n_cells);
    }
    const TableArgs &T = BATCH ? tabs[table] : tab0;
    const int r = rank_of<R>(T);
    const u64 seed_chk = T.seed[r];
    u64 c_alive = 0, c_nonempty = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
      const u32 c = begin + (u32)it * kBlock + tid;
      const bool valid = c < end;
      bool pure = false;
      u64 key = 0;
      if (valid) {
        u64 chk;
        int cnt;
        ld_cell_cs(cells + c, key, chk, cnt);
        pure = cell_pure(cnt, key, chk, seed_chk);
        c_alive += cnt >= 2;
        c_nonempty += cnt != 0;
      }
      const u32 ball = __ballot_sync(kFull, pure);
      const u32 first = begin + (u32)it * kBlock + (tid & ~31u);
      if (lane_id() == 0 && first < end) bitmap[first >> 5] = ball;
      const u32 p = warp_reserve<u32>(pure, &s_n);
      if (pure) {
        s_key[p] = key;
        s_cell[p] = c;
      }
    }
    alive += c_alive;
    nonempty += c_nonempty;
    __syncthreads();
    const u32 n = s_n;
    if (tid == 0) s_base = atomicAdd(&ctl->n_next, n);
    if (BATCH) {
      const u64 ne = block_sum<u64, kBlock>(c_nonempty, s_red);
      if (tid == 0 && ne) atomicAdd(bc.nonempty + table, ne);
      if (tid == 0 && n && bc.live) atomicAdd(bc.live + table, n);
    }
    __syncthreads();
    const u32 base = s_base;
    for (u32 q = tid; q < n; q += kBlock) {
      fkey[base + q] = s_key[q];
      fcell[base + q] = s_cell[q];
      if (BATCH) ftab[base + q] = table;
    }
    __syncthreads();
    if (tid == 0) s_n = 0;
    __syncthreads();
  }
  const u64 a = block_sum<u64, kBlock>(alive, s_red);
  const u64 ne = block_sum<u64, kBlock>(nonempty, s_red);
  if (tid == 0) {
    if (a) atomicAdd(&ctl->alive, a);
    if (ne) atomicAdd(&ctl->nonempty, ne);
  }
}

// --------------------------------------------------------------------------
// Phase B of round t: claim and recover.
// --------------------------------------------------------------------------
template <int R, bool BATCH>
__global__ void __launch_bounds__(kBlock) k_peel(Cell *__restrict__ cells, const TableArgs tab0,
                                                 const TableArgs *__restrict__ tabs,
                                                 const u64 *__restrict__ fkey, const u32 *__restrict__ fcell,
                                                 const u32 *__restrict__ ftab, const u32 *__restrict__ bitmap,
                                                 u32 *__restrict__ cand, u32 *__restrict__ ctab,
                                                 u64 *__restrict__ bout, DecodeCtl *__restrict__ ctl,
                                                 BatchCounters bc) {
  constexpr int NR = nr_of<R>();
  constexpr int CH = kBlock * kPeelItems;
  extern __shared__ __align__(16) unsigned char smem[];
  u64 *s_out = reinterpret_cast<u64 *>(smem);                    // CH      (plain)
  u32 *s_cand = reinterpret_cast<u32 *>(s_out + (BATCH ? 0 : CH)); // CH * NR
  u32 *s_ctab = s_cand + CH * NR;                                 // CH * NR (batch)
  __shared__ u32 s_nout, s_ncand, s_cbase;
  __shared__ u64 s_obase;
  __shared__ u64 s_red[kBlock / 32];
  const u32 tid = threadIdx.x;
  const u32 n = *(volatile u32 *)&ctl->n_front;
  const u32 round = *(volatile u32 *)&ctl->round;
  u64 *out = BATCH ? bout : ctl->out;
  const u64 out_cap = BATCH ? 0 : ctl->out_cap;
  const u32 stats_rounds = BATCH ? ctl->stats_rounds : 0;
  u64 emptied = 0;
  u32 flags = 0;
  if (tid == 0) s_nout = 0, s_ncand = 0;
  __syncthreads();
  for (u64 c0 = (u64)blockIdx.x * CH; c0 < n; c0 += (u64)gridDim.x * CH) {
#pragma unroll
    for (int it = 0; it < kPeelItems; ++it) {
      const u64 i = c0 + (u64)it * kBlock + tid;
      const bool valid = i < n;
      u64 x = 0;
      u32 c = 0, tb = 0;
      if (valid) {
        x = __ldcs(fkey + i);
        c = __ldcs(fcell + i);
        if (BATCH) tb = __ldcs(ftab + i);
      }
      const TableArgs &T = BATCH ? tabs[tb] : tab0;
      const int r = rank_of<R>(T);
      u32 cj[NR];
      cells_of<NR>(x, T, cj);
      int jstar = -1;
#pragma unroll
      for (int j = NR - 1; j >= 0; --j)
        if (j < r && cj[j] == c) jstar = j;
      bool win = valid;
      if (valid && jstar < 0) {
        flags |= FLAG_INTERNAL;
        win = false;
      }
      // The lowest-index cell of x that was pure at the round's start wins.
      // Sub-tables are laid out in order, so only sub-tables j < jstar matter.
#pragma unroll
      for (int j = 0; j < NR - 1; ++j) {
        if (win && j < jstar) {
          const u32 w = __ldcg(bitmap + (cj[j] >> 5));
          if ((w >> (cj[j] & 31u)) & 1u) win = false;
        }
      }
      int old[NR];
      u32 n_empty = 0;
      if (win) {
        const u64 cs = checksum(x, T.seed[r]);
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          old[j] = 0;
          if (j < r) {
            old[j] = touch_cell(cells, cj[j], x, cs, -1);
            n_empty += (u32)((old[j] == 1) - (old[j] == 0));  // net change of non-zero counts
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < NR; ++j) old[j] = 0;
      }
      emptied += (u64)(long long)(int)n_empty;
      if constexpr (!BATCH) {
        const u32 p = warp_reserve<u32>(win, &s_nout);
        if (win) s_out[p] = x;
      } else {
        // Per-table output slots: lanes of one table share one atomic.
        const u32 label = win ? tb : 0xffffffffu;
        const u32 grp = __match_any_sync(kFull, label);
        const int leader = __ffs(grp) - 1;
        const u32 gsize = __popc(grp);
        const u32 gempty = __reduce_add_sync(grp, n_empty);
        u64 base = 0;
        if (win && (int)lane_id() == leader) {
          const u32 local = round + 1 - T.start_round;  // this table's own round number
          base = atomicAdd(bc.recovered + tb, (u64)gsize);
          if (gempty) atomicAdd(bc.emptied + tb, (u64)(long long)(int)gempty);
          atomicMax(bc.rounds + tb, local);
          if (local <= stats_rounds) atomicAdd(bc.round_rec + (u64)tb * stats_rounds + (local - 1), gsize);
        }
        base = __shfl_sync(kFull, base, leader);
        if (win) {
          const u64 slot = base + __popc(grp & lanemask_lt());
          if (slot < T.out_cap) out[T.out_base + slot] = x;
          else flags |= FLAG_CAPACITY;
        }
      }
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const bool push = win && j < r && old[j] == 2;
        const u32 q = warp_reserve<u32>(push, &s_ncand);
        if (push) {
          s_cand[q] = cj[j];
          if (BATCH) s_ctab[q] = tb;
        }
      }
    }
    __syncthreads();
    const u32 nout = BATCH ? 0 : s_nout;
    const u32 ncand = s_ncand;
    if (tid == 0) {
      if (!BATCH && nout) s_obase = atomicAdd(&ctl->n_out, (u64)nout);
      if (ncand) s_cbase = atomicAdd(&ctl->n_cand, ncand);
    }
    __syncthreads();
    if constexpr (!BATCH) {
      const u64 ob = s_obase;
      for (u32 q = tid; q < nout; q += kBlock) {
        if (ob + q < out_cap) out[ob + q] = s_out[q];
        else flags |= FLAG_CAPACITY;
      }
    }
    const u32 cb = s_cbase;
    for (u32 q = tid; q < ncand; q += kBlock) {
      cand[cb + q] = s_cand[q];
      if (BATCH) ctab[cb + q] = s_ctab[q];
    }
    __syncthreads();
    if (tid == 0) s_nout = 0, s_ncand = 0;
    __syncthreads();
  }
  if (!BATCH) {
    const u64 e = block_sum<u64, kBlock>(emptied, s_red);
    if (tid == 0 && e) atomicAdd(&ctl->emptied, e);
  }
  if (flags) atomicOr(&ctl->flags, flags);
}

// --------------------------------------------------------------------------
// Phase A of round t+1: candidates that are pure now form F_{t+1}.
// --------------------------------------------------------------------------
template <int R, bool BATCH>
__global__ void __launch_bounds__(kBlock) k_filter(const Cell *__restrict__ cells, const TableArgs tab0,
                                                   const TableArgs *__restrict__ tabs,
                                                   const u32 *__restrict__ cand, const u32 *__restrict__ ctab,
                                                   u64 *__restrict__ fkey, u32 *__restrict__ fcell,
                                                   u32 *__restrict__ ftab, u32 *__restrict__ bitmap,
                                                   DecodeCtl *__restrict__ ctl, BatchCounters bc) {
  constexpr int CH = kBlock * kFilterItems;
  __shared__ u64 s_key[CH];
  __shared__ u32 s_cell[CH];
  __shared__ u32 s_tab[BATCH ? CH : 1];
  __shared__ u32 s_n, s_base;
  const u32 tid = threadIdx.x;
  const u32 n = *(volatile u32 *)&ctl->n_cand;
  if (tid == 0) s_n = 0;
  __syncthreads();
  for (u64 c0 = (u64)blockIdx.x * CH; c0 < n; c0 += (u64)gridDim.x * CH) {
#pragma unroll
    for (int it = 0; it < kFilterItems; ++it) {
      const u64 i = c0 + (u64)it * kBlock + tid;
      const bool valid = i < n;
      u32 c = 0, tb = 0;
      bool pure = false;
      u64 key = 0;
      if (valid) {
        c = __ldcs(cand + i);
        if (BATCH) tb = __ldcs(ctab + i);
        u64 chk;
        int cnt;
        ld_cell_cg(cells + c, key, chk, cnt);
        u64 seed_chk;
        if (BATCH && bc.chk_seed) {
          seed_chk = bc.chk_seed[tb];
        } else {
          const TableArgs &T = BATCH ? tabs[tb] : tab0;
          seed_chk = T.seed[rank_of<R>(T)];
        }
        pure = cell_pure(cnt, key, chk, seed_chk);
        if (pure) atomicOr(bitmap + (c >> 5), 1u << (c & 31u));
      }
      const u32 p = warp_reserve<u32>(pure, &s_n);
      if (pure) {
        s_key[p] = key;
        s_cell[p] = c;
        if (BATCH) s_tab[p] = tb;
      }
      if (BATCH && bc.live) {
        const u32 grp = __match_any_sync(kFull, pure ? tb : 0xffffffffu);
        if (pure && (int)lane_id() == __ffs(grp) - 1) atomicAdd(bc.live + tb, (u32)__popc(grp));
      }
    }
    __syncthreads();
    const u32 nn = s_n;
    if (tid == 0 && nn) s_base = atomicAdd(&ctl->n_next, nn);
    __syncthreads();
    const u32 base = s_base;
    for (u32 q = tid; q < nn; q += kBlock) {
      fkey[base + q] = s_key[q];
      fcell[base + q] = s_cell[q];
      if (BATCH) ftab[base + q] = s_tab[q];
    }
    __syncthreads();
    if (tid == 0) s_n = 0;
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// End of a loop iteration: record the finished round, promote F_{t+1} to the
// current frontier, decide whether another round runs.  One thread.
// The first iteration after the scan has an empty frontier and only promotes
// F_1; it is not a round.
// --------------------------------------------------------------------------
// Start of a decode: the control block takes its initial value from the
// launch (a kernel rather than a host-to-device copy, so the decode never
// queues behind a bulk upload on the copy engine).
__global__ void k_ctl_init(DecodeCtl *__restrict__ ctl, DecodeCtl init) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *ctl = init;
}

// Copies n words into mapped pinned host memory with stores from the GPU, so
// that a small result reaches the host without a copy engine (where it would
// queue behind any bulk copy that engine is running).
__global__ void k_to_host(const u64 *__restrict__ src, u64 *__restrict__ dst, u32 n) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
  __threadfence_system();
}

__global__ void k_flag_to_host(const u32 *__restrict__ src, u32 *__restrict__ dst) {
  if (threadIdx.x == 0) *dst = *src;
  __threadfence_system();
}

__global__ void k_round_end(DecodeCtl *__restrict__ ctl, RoundStats st, int set_cond,
                            cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  DecodeCtl &c = *ctl;
  const u32 t = c.round;
  if (c.n_front > 0 && t > 0 && st.recovered) {
    // round t just finished
    st.recovered[t - 1] = c.n_out - c.out_round_start;
    st.alive[t - 1] = c.alive;
    st.front[t - 1] = c.n_front;
    c.alive -= c.n_cand;  // every cell leaving "count >= 2" crossed 2 -> 1 once
  }
  c.out_round_start = c.n_out;
  c.n_front = c.n_next;
  c.n_next = 0;
  c.n_cand = 0;
  c.n_act = 0;
  c.n_act_dense = 0;
  u32 more = c.n_front > 0 && (c.flags & (FLAG_CAPACITY | FLAG_INTERNAL)) == 0;
  if (more && t >= c.max_rounds) {
    c.flags |= FLAG_ROUND_LIMIT;
    more = 0;
  }
  if (more) c.round = t + 1;
  c.more = more;
  if (set_cond) cudaGraphSetConditional(cond, more);
}

}  // namespace pp
