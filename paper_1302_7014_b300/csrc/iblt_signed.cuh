// Signed IBLT recovery: the table holds a set difference, keys inserted
// (+1) and keys deleted without having been inserted (-1) -- the sparse
// recovery setting of Sec. 6 "Motivation", where insertion and deletion are
// the same XORs.  A cell is pure when |count| == 1 and its checksum field
// matches its key field; the key comes out with the sign of the count.
// Rounds follow Sec. 1 at k = 2 on the hypergraph of the difference, with the
// same kernel structure as the unsigned decode:
//   k_sgscan    F_1 = the cells pure before any round (key, cell, sign);
//   k_sgpeel    (B) a frontier entry's cell recovers its key iff no cell of
//               the key in a lower sub-table was pure at the round's start;
//               the winner removes (key, sign) from its r cells (count -= sign)
//               and pushes every cell whose count becomes +1 or -1;
//   k_sgfilter  (A) candidates that are pure at the round's end form the next
//               frontier.
// Unlike the unsigned case a count can reach +-1 more than once (0 -> -1 ->
// 0 -> +1 ...), so a cell may be pushed several times; the filter keeps an
// entry only when its atomicOr sets the cell's "pure at round start" bit.  A
// cell is pure at most once in a decode (its one item then leaves it), so the
// bit is set at most once and needs no clearing.
#pragma once

#include "iblt_types.cuh"

namespace pp {

// Pure with sign +1 or -1: count +-1 and the checksum field is that of the key
// field alone (an XOR, the same for an inserted and a deleted key).
__device__ __forceinline__ bool signed_pure(int cnt, u64 key, u64 chk, u64 seed_chk) {
  return (cnt == 1 || cnt == -1) && chk == checksum(key, seed_chk);
}

template <int R>
__global__ void __launch_bounds__(kBlock) k_sgscan(const Cell *__restrict__ cells, const TableArgs tab0,
                                                   u64 *__restrict__ fkey, u32 *__restrict__ fcell,
                                                   signed char *__restrict__ fsign, u32 *__restrict__ bitmap,
                                                   DecodeCtl *__restrict__ ctl) {
  constexpr int CH = kBlock * kScanItems;
  __shared__ u64 s_key[CH];
  __shared__ u32 s_cell[CH];
  __shared__ signed char s_sign[CH];
  __shared__ u32 s_n, s_base;
  __shared__ u64 s_red[kBlock / 32];
  const u32 tid = threadIdx.x;
  const u64 seed_chk = tab0.seed[rank_of<R>(tab0)];
  u64 nonempty = 0;
  if (tid == 0) s_n = 0;
  __syncthreads();
  for (u64 begin = (u64)blockIdx.x * CH; begin < tab0.n_cells; begin += (u64)gridDim.x * CH) {
    const u64 end = begin + CH < tab0.n_cells ? begin + CH : tab0.n_cells;
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
      const u64 c = begin + (u64)it * kBlock + tid;
      bool pure = false;
      u64 key = 0;
      int cnt = 0;
      if (c < end) {
        u64 chk;
        ld_cell_cs(cells + c, key, chk, cnt);
        pure = signed_pure(cnt, key, chk, seed_chk);
        nonempty += cnt != 0;
      }
      const u32 ball = __ballot_sync(kFull, pure);
      const u64 first = begin + (u64)it * kBlock + (tid & ~31u);
      if (lane_id() == 0 && first < end) bitmap[first >> 5] = ball;
      const u32 p = warp_reserve<u32>(pure, &s_n);
      if (pure) {
        s_key[p] = key;
        s_cell[p] = (u32)c;
        s_sign[p] = (signed char)cnt;
      }
    }
    __syncthreads();
    const u32 n = s_n;
    if (tid == 0 && n) s_base = atomicAdd(&ctl->n_next, n);
    __syncthreads();
    for (u32 q = tid; q < n; q += kBlock) {
      fkey[s_base + q] = s_key[q];
      fcell[s_base + q] = s_cell[q];
      fsign[s_base + q] = s_sign[q];
    }
    __syncthreads();
    if (tid == 0) s_n = 0;
    __syncthreads();
  }
  const u64 ne = block_sum<u64, kBlock>(nonempty, s_red);
  if (tid == 0 && ne) atomicAdd(&ctl->nonempty, ne);
}

template <int R>
__global__ void __launch_bounds__(kBlock) k_sgpeel(Cell *__restrict__ cells, const TableArgs tab0,
                                                   const u64 *__restrict__ fkey, const u32 *__restrict__ fcell,
                                                   const signed char *__restrict__ fsign,
                                                   const u32 *__restrict__ bitmap, u32 *__restrict__ cand,
                                                   u64 cand_cap, signed char *__restrict__ out_sign,
                                                   DecodeCtl *__restrict__ ctl) {
  constexpr int NR = nr_of<R>();
  constexpr int CH = kBlock * kPeelItems;
  __shared__ u64 s_out[CH];
  __shared__ signed char s_osign[CH];
  __shared__ u32 s_cand[CH * NR];
  __shared__ u32 s_nout, s_ncand, s_cbase;
  __shared__ u64 s_obase;
  __shared__ u64 s_red[kBlock / 32];
  const u32 tid = threadIdx.x;
  const u32 n = *(volatile u32 *)&ctl->n_front;
  u64 *out = ctl->out;
  const u64 out_cap = ctl->out_cap;
  const int r = rank_of<R>(tab0);
  u64 emptied = 0;
  u32 flags = 0, n_neg = 0;
  if (tid == 0) s_nout = 0, s_ncand = 0;
  __syncthreads();
  for (u64 c0 = (u64)blockIdx.x * CH; c0 < n; c0 += (u64)gridDim.x * CH) {
#pragma unroll
    for (int it = 0; it < kPeelItems; ++it) {
      const u64 i = c0 + (u64)it * kBlock + tid;
      const bool valid = i < n;
      u64 x = 0;
      u32 c = 0;
      int sg = 0;
      if (valid) {
        x = __ldcs(fkey + i);
        c = __ldcs(fcell + i);
        sg = __ldcs(fsign + i);
      }
      u32 cj[NR];
      cells_of<NR>(x, tab0, cj);
      int jstar = -1;
#pragma unroll
      for (int j = NR - 1; j >= 0; --j)
        if (j < r && cj[j] == c) jstar = j;
      bool win = valid;
      if (valid && jstar < 0) {
        flags |= FLAG_INTERNAL;
        win = false;
      }
#pragma unroll
      for (int j = 0; j < NR - 1; ++j) {
        if (win && j < jstar) {
          const u32 w = __ldcg(bitmap + (cj[j] >> 5));
          if ((w >> (cj[j] & 31u)) & 1u) win = false;
        }
      }
      if (win) {
        n_neg += sg < 0;
        const u64 cs = checksum(x, tab0.seed[r]);
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (j < r) {
            const int old = touch_cell(cells, cj[j], x, cs, -sg);
            const int now = old - sg;
            emptied += (u64)(long long)((old != 0) - (now != 0));
            if (now == 1 || now == -1) s_cand[atomicAdd(&s_ncand, 1u)] = cj[j];
          }
        }
      }
      const u32 p = warp_reserve<u32>(win, &s_nout);
      if (win) {
        s_out[p] = x;
        s_osign[p] = (signed char)sg;
      }
    }
    __syncthreads();
    const u32 nout = s_nout, ncand = s_ncand;
    if (tid == 0) {
      if (nout) s_obase = atomicAdd(&ctl->n_out, (u64)nout);
      if (ncand) s_cbase = atomicAdd(&ctl->n_cand, ncand);
    }
    __syncthreads();
    for (u32 q = tid; q < nout; q += kBlock) {
      if (s_obase + q < out_cap) {
        out[s_obase + q] = s_out[q];
        if (out_sign) out_sign[s_obase + q] = s_osign[q];
      } else {
        flags |= FLAG_CAPACITY;
      }
    }
    for (u32 q = tid; q < ncand; q += kBlock) {
      if ((u64)s_cbase + q < cand_cap) cand[s_cbase + q] = s_cand[q];
      else flags |= FLAG_INTERNAL;
    }
    __syncthreads();
    if (tid == 0) s_nout = 0, s_ncand = 0;
    __syncthreads();
  }
  const u64 e = block_sum<u64, kBlock>(emptied, s_red);
  if (tid == 0 && e) atomicAdd(&ctl->emptied, e);
  if (n_neg) atomicAdd(&ctl->n_neg, n_neg);
  if (flags) atomicOr(&ctl->flags, flags);
}

template <int R>
__global__ void __launch_bounds__(kBlock) k_sgfilter(const Cell *__restrict__ cells, const TableArgs tab0,
                                                     const u32 *__restrict__ cand, u64 *__restrict__ fkey,
                                                     u32 *__restrict__ fcell, signed char *__restrict__ fsign,
                                                     u32 *__restrict__ bitmap, DecodeCtl *__restrict__ ctl) {
  constexpr int CH = kBlock * kFilterItems;
  __shared__ u64 s_key[CH];
  __shared__ u32 s_cell[CH];
  __shared__ signed char s_sign[CH];
  __shared__ u32 s_n, s_base;
  const u32 tid = threadIdx.x;
  const u32 n = *(volatile u32 *)&ctl->n_cand;
  const u64 seed_chk = tab0.seed[rank_of<R>(tab0)];
  if (tid == 0) s_n = 0;
  __syncthreads();
  for (u64 c0 = (u64)blockIdx.x * CH; c0 < n; c0 += (u64)gridDim.x * CH) {
#pragma unroll
    for (int it = 0; it < kFilterItems; ++it) {
      const u64 i = c0 + (u64)it * kBlock + tid;
      bool keep = false;
      u64 key = 0;
      u32 c = 0;
      int cnt = 0;
      if (i < n) {
        c = __ldcs(cand + i);
        u64 chk;
        ld_cell_cg(cells + c, key, chk, cnt);
        if (signed_pure(cnt, key, chk, seed_chk)) {
          const u32 bit = 1u << (c & 31u);
          keep = (atomicOr(bitmap + (c >> 5), bit) & bit) == 0;  // first entry of this cell
        }
      }
      const u32 p = warp_reserve<u32>(keep, &s_n);
      if (keep) {
        s_key[p] = key;
        s_cell[p] = c;
        s_sign[p] = (signed char)cnt;
      }
    }
    __syncthreads();
    const u32 nn = s_n;
    if (tid == 0 && nn) s_base = atomicAdd(&ctl->n_next, nn);
    __syncthreads();
    for (u32 q = tid; q < nn; q += kBlock) {
      fkey[s_base + q] = s_key[q];
      fcell[s_base + q] = s_cell[q];
      fsign[s_base + q] = s_sign[q];
    }
    __syncthreads();
    if (tid == 0) s_n = 0;
    __syncthreads();
  }
}

}  // namespace pp
