// IBLT recovery with sub-tables (Sec. 6 "Implementation Details"; App. B at
// k = 2): every round visits the r sub-tables in order, and the sub-round of
// sub-table j recovers the key of every cell of sub-table j that is pure at
// the sub-round's start, then deletes that key from its r cells.  A key has
// exactly one cell per sub-table, so no key is found twice in a sub-round and
// no claim step is needed (the reason the paper splits the table).
//
// Each sub-table keeps a queue of its cells that may be pure at its next
// sub-round:
//   k_sscan    (once)   every cell pure before the first sub-round;
//   k_speel    (B)      a cell whose count drops from 2 to 1 is appended to
//                       the queue of its own sub-table.
// Counts only fall during a decode, so a cell enters a queue at most once and
// sub-table j's queue fits in the sub-table's own cells' slots.  A cell that is
// pure at the start of its sub-round is always in the queue: it either was
// pure before the decode or crossed 2 -> 1 since, and it cannot have been
// consumed by an earlier sub-round of its sub-table (it would be empty now, or
// unchanged and still impure).
// Per sub-round:
//   k_sfilter  (A)      the queue entries of the sub-table that are pure now:
//                       their keys are snapshotted (the frontier);
//   k_speel    (B)      every frontier key is output and deleted from its r
//                       cells;
//   k_send              statistics; picks the next sub-round whose sub-table
//                       has queued cells (the idle ones in between keep their
//                       numbers) and sets the graph's while condition.
#pragma once

#include "iblt_types.cuh"

namespace pp {

struct SubDecCtl {
  u64 *out;       // recovered keys (caller's buffer)
  u64 out_cap;
  u64 n_out;      // keys recovered so far
  u64 out_start;  // n_out when the current sub-round started
  u64 nonempty;   // cells with count != 0 when the decode started
  u64 emptied;    // net cells emptied (1 -> 0 minus 0 -> -1), mod 2^64
  u32 sub;        // number of the current sub-round (0 before the first)
  u32 part;       // its sub-table
  u32 fb, fe;     // its queue entries fb .. fe-1
  u32 n_front;    // frontier entries written by the filter
  u32 last;       // last sub-round that recovered a key
  u32 flags;
  u32 max_sub;
  u32 more;
  u32 r;
  u32 head[PP_MAX_R];  // queue entries consumed, per sub-table
  u32 tail[PP_MAX_R];  // queue entries appended, per sub-table
};

constexpr int kSubItems = 2;  // frontier entries per thread per chunk of k_speel

// Sub-table of cell c: the last j < r with off[j] <= c (plain tables: base 0).
__device__ __forceinline__ u32 subtable_of(const TableArgs &T, u32 c) {
  u32 j = 0;
  for (u32 h = 1; h < T.r; ++h) j += c >= T.off[h] ? 1u : 0u;
  return j;
}

// Block staging of queue appends: counts per sub-table in shared memory, one
// global atomic per sub-table per flush.
struct SubStage {
  u32 *cell, *part, *rank;
  u32 *cnt, *base;  // PP_MAX_R each
  u32 *n;
  u32 cap;
};

__device__ __forceinline__ void sub_stage_push(SubStage &S, const TableArgs &T, u32 *queue,
                                               SubDecCtl *ctl, u32 c, u32 j) {
  const u32 q = atomicAdd(S.n, 1u);
  if (q < S.cap) {
    S.cell[q] = c;
    S.part[q] = j;
    S.rank[q] = atomicAdd(S.cnt + j, 1u);
  } else {
    const u32 slot = atomicAdd(&ctl->tail[j], 1u);
    if (slot < T.off[j + 1] - T.off[j]) queue[T.off[j] + slot] = c;
    else atomicOr(&ctl->flags, (u32)FLAG_INTERNAL);
  }
}

__device__ __forceinline__ void sub_stage_flush(SubStage &S, const TableArgs &T, u32 *queue,
                                                SubDecCtl *ctl) {
  __syncthreads();
  if (threadIdx.x < T.r) {
    const u32 c = S.cnt[threadIdx.x];
    S.base[threadIdx.x] = c ? atomicAdd(&ctl->tail[threadIdx.x], c) : 0u;
  }
  __syncthreads();
  const u32 nn = min(*S.n, S.cap);
  for (u32 q = threadIdx.x; q < nn; q += blockDim.x) {
    const u32 j = S.part[q];
    const u32 slot = S.base[j] + S.rank[q];
    if (slot < T.off[j + 1] - T.off[j]) queue[T.off[j] + slot] = S.cell[q];
    else atomicOr(&ctl->flags, (u32)FLAG_INTERNAL);
  }
  __syncthreads();
  if (threadIdx.x < PP_MAX_R) S.cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) *S.n = 0;
  __syncthreads();
}

// The queues before the first sub-round: every cell pure before any recovery.
template <int R>
__global__ void __launch_bounds__(kBlock) k_sscan(const Cell *__restrict__ cells, const TableArgs tab0,
                                                  u32 *__restrict__ queue, SubDecCtl *__restrict__ ctl) {
  constexpr int CH = kBlock * kScanItems;
  __shared__ u32 s_cell[CH], s_part[CH], s_rank[CH];
  __shared__ u32 s_cnt[PP_MAX_R], s_base[PP_MAX_R], s_n;
  __shared__ u64 s_red[kBlock / 32];
  SubStage S{s_cell, s_part, s_rank, s_cnt, s_base, &s_n, (u32)CH};
  if (threadIdx.x < PP_MAX_R) s_cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  const u64 seed_chk = tab0.seed[rank_of<R>(tab0)];
  u64 nonempty = 0;
  for (u64 c0 = (u64)blockIdx.x * CH; c0 < tab0.n_cells; c0 += (u64)gridDim.x * CH) {
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
      const u64 c = c0 + (u64)it * kBlock + threadIdx.x;
      if (c < tab0.n_cells) {
        u64 key, chk;
        int cnt;
        ld_cell_cs(cells + c, key, chk, cnt);
        nonempty += cnt != 0;
        if (cell_pure(cnt, key, chk, seed_chk))
          sub_stage_push(S, tab0, queue, ctl, (u32)c, subtable_of(tab0, (u32)c));
      }
    }
    sub_stage_flush(S, tab0, queue, ctl);
  }
  const u64 ne = block_sum<u64, kBlock>(nonempty, s_red);
  if (threadIdx.x == 0 && ne) atomicAdd(&ctl->nonempty, ne);
}

// Phase A of a sub-round: the queued cells of its sub-table that are pure now.
// front_count: where the frontier's size goes (ctl->n_front, or the round
// control block of the binned sub-rounds).
template <int R>
__global__ void __launch_bounds__(kBlock) k_sfilter(const Cell *__restrict__ cells, const TableArgs tab0,
                                                    const u32 *__restrict__ queue, u64 *__restrict__ fkey,
                                                    u32 *__restrict__ fcell, SubDecCtl *__restrict__ ctl,
                                                    u32 *__restrict__ front_count) {
  constexpr int CH = kBlock * kFilterItems;
  __shared__ u64 s_key[CH];
  __shared__ u32 s_cell[CH];
  __shared__ u32 s_n, s_base;
  const u32 j = *(volatile u32 *)&ctl->part;
  const u32 fb = *(volatile u32 *)&ctl->fb, fe = *(volatile u32 *)&ctl->fe;
  const u32 *q = queue + tab0.off[j];
  const u64 seed_chk = tab0.seed[rank_of<R>(tab0)];
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  for (u64 c0 = (u64)fb + (u64)blockIdx.x * CH; c0 < fe; c0 += (u64)gridDim.x * CH) {
#pragma unroll
    for (int it = 0; it < kFilterItems; ++it) {
      const u64 i = c0 + (u64)it * kBlock + threadIdx.x;
      bool pure = false;
      u64 key = 0;
      u32 c = 0;
      if (i < fe) {
        c = __ldcs(q + i);
        u64 chk;
        int cnt;
        ld_cell_cg(cells + c, key, chk, cnt);
        pure = cell_pure(cnt, key, chk, seed_chk);
      }
      const u32 p = warp_reserve<u32>(pure, &s_n);
      if (pure) {
        s_key[p] = key;
        s_cell[p] = c;
      }
    }
    __syncthreads();
    const u32 nn = s_n;
    if (threadIdx.x == 0 && nn) s_base = atomicAdd(front_count, nn);
    __syncthreads();
    for (u32 p = threadIdx.x; p < nn; p += kBlock) {
      fkey[s_base + p] = s_key[p];
      fcell[s_base + p] = s_cell[p];
    }
    __syncthreads();
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
  }
}

// Phase B of a sub-round: output every frontier key and delete it from its r
// cells; a cell whose count drops from 2 to 1 joins its sub-table's queue.
template <int R>
__global__ void __launch_bounds__(kBlock) k_speel(Cell *__restrict__ cells, const TableArgs tab0,
                                                  const u64 *__restrict__ fkey, const u32 *__restrict__ fcell,
                                                  u32 *__restrict__ queue, SubDecCtl *__restrict__ ctl) {
  constexpr int NR = nr_of<R>();
  constexpr int CH = kBlock * kSubItems;
  constexpr int CAP = CH * (NR < 4 ? NR : 4);  // more pushes than this go straight to global
  __shared__ u64 s_out[CH];
  __shared__ u32 s_cell[CAP], s_part[CAP], s_rank[CAP];
  __shared__ u32 s_cnt[PP_MAX_R], s_base[PP_MAX_R], s_n, s_nout;
  __shared__ u64 s_obase;
  __shared__ u64 s_red[kBlock / 32];
  SubStage S{s_cell, s_part, s_rank, s_cnt, s_base, &s_n, (u32)CAP};
  if (threadIdx.x < PP_MAX_R) s_cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_n = 0, s_nout = 0;
  __syncthreads();
  const int r = rank_of<R>(tab0);
  const u32 j = *(volatile u32 *)&ctl->part;
  const u32 n = *(volatile u32 *)&ctl->n_front;
  u64 *out = ctl->out;
  const u64 out_cap = ctl->out_cap;
  u64 emptied = 0;
  u32 flags = 0;
  for (u64 c0 = (u64)blockIdx.x * CH; c0 < n; c0 += (u64)gridDim.x * CH) {
#pragma unroll
    for (int it = 0; it < kSubItems; ++it) {
      const u64 i = c0 + (u64)it * kBlock + threadIdx.x;
      bool ok = false;
      u64 x = 0;
      u32 cj[NR];
      if (i < n) {
        x = __ldcs(fkey + i);
        const u32 c = __ldcs(fcell + i);
        cells_of<NR>(x, tab0, cj);
#pragma unroll
        for (int h = 0; h < NR; ++h)
          if ((u32)h == j) ok = cj[h] == c;  // the key found in c must hash to c
        if (!ok) flags |= FLAG_INTERNAL;
      }
      if (ok) {
        const u64 cs = checksum(x, tab0.seed[r]);
#pragma unroll
        for (int h = 0; h < NR; ++h) {
          if (h < r) {
            const int old = touch_cell(cells, cj[h], x, cs, -1);
            emptied += (u64)(long long)((old == 1) - (old == 0));
            if (old == 2) sub_stage_push(S, tab0, queue, ctl, cj[h], (u32)h);
          }
        }
      }
      const u32 p = warp_reserve<u32>(ok, &s_nout);
      if (ok) s_out[p] = x;
    }
    __syncthreads();
    const u32 no = s_nout;
    if (threadIdx.x == 0 && no) s_obase = atomicAdd(&ctl->n_out, (u64)no);
    __syncthreads();
    for (u32 q = threadIdx.x; q < no; q += kBlock) {
      if (s_obase + q < out_cap) out[s_obase + q] = s_out[q];
      else flags |= FLAG_CAPACITY;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_nout = 0;
    sub_stage_flush(S, tab0, queue, ctl);
  }
  const u64 e = block_sum<u64, kBlock>(emptied, s_red);
  if (threadIdx.x == 0 && e) atomicAdd(&ctl->emptied, e);
  if (flags) atomicOr(&ctl->flags, flags);
}

// Binned sub-rounds: the candidates that k_apply_round collected (cells whose
// count fell from 2 to 1) join the queues of their sub-tables.
__global__ void __launch_bounds__(kBlock) k_sdistribute(const TableArgs tab0, const u32 *__restrict__ cand,
                                                        const DecodeCtl *__restrict__ rctl, u32 *__restrict__ queue,
                                                        SubDecCtl *__restrict__ ctl) {
  constexpr int CH = kBlock * kScanItems;
  __shared__ u32 s_cell[CH], s_part[CH], s_rank[CH];
  __shared__ u32 s_cnt[PP_MAX_R], s_base[PP_MAX_R], s_n;
  SubStage S{s_cell, s_part, s_rank, s_cnt, s_base, &s_n, (u32)CH};
  if (threadIdx.x < PP_MAX_R) s_cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  const u32 n = *(volatile const u32 *)&rctl->n_cand;
  for (u64 c0 = (u64)blockIdx.x * CH; c0 < n; c0 += (u64)gridDim.x * CH) {
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
      const u64 i = c0 + (u64)it * kBlock + threadIdx.x;
      if (i < n) {
        const u32 c = __ldcs(cand + i);
        sub_stage_push(S, tab0, queue, ctl, c, subtable_of(tab0, c));
      }
    }
    sub_stage_flush(S, tab0, queue, ctl);
  }
}

// End of a binned sub-round (one thread): the sub-round's bookkeeping as in
// k_send, reading the recovered keys from the round control block, then that
// block, the bins and the apply counter reset for the next sub-round.
__global__ void k_send_binned(SubDecCtl *__restrict__ ctl, DecodeCtl *__restrict__ rctl, RoundBins rb,
                              u64 *__restrict__ st_rec, int set_cond, cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  SubDecCtl &c = *ctl;
  DecodeCtl &d = *rctl;
  const u32 t = c.sub;
  if (t > 0) {
    const u64 rec = d.n_out - c.out_start;
    st_rec[t - 1] = rec;
    if (rec) c.last = t;
    c.head[c.part] = c.fe;
  }
  c.out_start = d.n_out;
  c.n_out = d.n_out;
  c.emptied = d.emptied;
  d.n_front = 0;
  d.n_cand = 0;
  d.apply_next = 0;
  for (u32 i = 0; i < rb.n_bins; ++i) rb.count[i] = 0;
  c.flags |= d.flags;
  u32 more = 0, dd = 1;
  for (; dd <= c.r; ++dd) {
    const u32 j = (c.part + dd) % c.r;
    if (c.tail[j] > c.head[j]) {
      more = 1;
      break;
    }
  }
  if (c.flags & (FLAG_CAPACITY | FLAG_INTERNAL)) more = 0;
  if (more && (u64)t + dd > c.max_sub) {
    c.flags |= FLAG_ROUND_LIMIT;
    more = 0;
  }
  if (more) {
    for (u32 q = 1; q < dd; ++q) st_rec[t + q - 1] = 0;  // idle sub-rounds
    const u32 j = (c.part + dd) % c.r;
    c.sub = t + dd;
    c.part = j;
    c.fb = c.head[j];
    c.fe = c.tail[j];
  }
  c.more = more;
  if (set_cond) cudaGraphSetConditional(cond, more);
}

// End of a sub-round (one thread).
__global__ void k_send(SubDecCtl *__restrict__ ctl, u64 *__restrict__ st_rec, int set_cond,
                       cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  SubDecCtl &c = *ctl;
  const u32 t = c.sub;
  if (t > 0) {
    const u64 rec = c.n_out - c.out_start;
    st_rec[t - 1] = rec;
    if (rec) c.last = t;
    c.head[c.part] = c.fe;
  }
  c.out_start = c.n_out;
  c.n_front = 0;
  u32 more = 0, d = 1;
  for (; d <= c.r; ++d) {
    const u32 j = (c.part + d) % c.r;
    if (c.tail[j] > c.head[j]) {
      more = 1;
      break;
    }
  }
  if (c.flags & (FLAG_CAPACITY | FLAG_INTERNAL)) more = 0;
  if (more && (u64)t + d > c.max_sub) {
    c.flags |= FLAG_ROUND_LIMIT;
    more = 0;
  }
  if (more) {
    for (u32 q = 1; q < d; ++q) st_rec[t + q - 1] = 0;  // idle sub-rounds
    const u32 j = (c.part + d) % c.r;
    c.sub = t + d;
    c.part = j;
    c.fb = c.head[j];
    c.fe = c.tail[j];
  }
  c.more = more;
  if (set_cond) cudaGraphSetConditional(cond, more);
}

}  // namespace pp
