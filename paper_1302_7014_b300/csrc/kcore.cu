// C-ABI: round-synchronous k-core peeling of an explicit r-uniform hypergraph.
//
// Round t (Sec. 1, Sec. 3.1): every vertex whose degree is < k at the start of
// the round is removed, with every edge touching it.  On the device:
//   build   degree histogram -> exclusive scan -> scatter of edge ids gives
//           each vertex its incidence list (CSR);
//   scan    F_1 = {v : deg(v) < k};
//   peel    for v in F_t and each edge e of v: the first thread to clear e's
//           alive bit removes e and takes one degree from each endpoint; the
//           decrement that takes a degree from k to k-1 pushes that endpoint
//           into F_{t+1} (its degree was >= k at the start of round t, and is
//           < k at its end: exactly the vertices round t+1 removes).
// While the frontier is large the full rounds run edge-centric instead
// (k_eround): one pass over the edges still alive removes those with a vertex
// in F_t (a bitmap), with the same decrements and pushes, and needs no
// incidence lists.  Once the frontier is small against the edges left, the
// lists are built for those edges only and the vertex-centric rounds finish.
// Either way round t removes exactly the edges that touch F_t.
//
// Sub-round mode (App. B, pp_peel_kcore_subrounds): the vertices are split into
// p parts and each round runs one sub-round per part; a sub-round removes the
// part's vertices whose degree is < k at the sub-round's start.  Each part
// keeps a queue of its vertices that are due (degree < k, not yet removed):
// the scan fills it, and the k -> k-1 crossing of a vertex appends the vertex
// to its own part's queue.  A sub-round takes the entries its part's queue
// held when the sub-round started; an entry appended during the sub-round of
// its own part waits for the next round, as the definition requires.  Every
// vertex enters a queue at most once (degrees only fall), so part j's queue
// fits in the part's own n_j slots.  Sub-rounds whose part has nothing due
// are skipped on the device (their statistics are still written).
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "host.cuh"
#include "kcore_csr.cuh"
#include "scan.cuh"

using namespace pp;

namespace pp {

constexpr int kKBlock = 256;
constexpr int kKStage = 2048;  // staged pushes per CTA before spilling to global atomics
// Edge-centric rounds run while the frontier holds at least 1 / frontier_switch
// (pp_options, default 2) vertices per edge left: each such round removes a
// large share of the list.  Below that, a pass over every edge left costs more
// than the incidence lists (their build included): measured at 2^25 vertices,
// r = 4, an edge-centric round is latency-bound at about 0.7 TB/s on the list,
// four random bitmap probes per edge.

struct PeelCtl {
  u64 claimed;  // edges removed in the current round
  u64 s;        // vertices left
  u64 m;        // edges left
  u32 round;    // rounds started
  u32 n_front;
  u32 n_next;
  u32 flags;
  u32 max_rounds;
  u32 more;
  u32 k;
  // edge-centric rounds
  u32 src;       // edge list of the next round: 0 or 1 (compacted), 2 = the caller's array
  u32 compact;   // the next round copies its surviving edges to the other list
  u32 sw;        // hand the rounds over to the incidence lists
  u32 econt;     // another edge-centric round follows
  u32 len_next;  // survivors written by a compacting round
  u64 len;       // entries in the list (removed ones included until it is compacted)
};

struct PeelStats {
  u64 *s;  // vertices left after round t
  u64 *m;  // edges left after round t
};

__global__ void k_kinit(PeelCtl *ctl, u64 n, u64 m, u32 k, u32 max_rounds) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    PeelCtl c;
    memset(&c, 0, sizeof c);
    c.s = n;
    c.m = m;
    c.k = k;
    c.max_rounds = max_rounds;
    c.src = 2;
    c.compact = 1;
    c.len = m;
    *ctl = c;
  }
}

// Degree of every vertex (with multiplicity); zeroes the edge-round output.
__global__ void __launch_bounds__(kKBlock) k_hist(const u32 *__restrict__ edges, u64 m, u32 r, u32 n,
                                                  u32 *__restrict__ deg, int *__restrict__ eround,
                                                  PeelCtl *__restrict__ ctl) {
  u32 bad = 0;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    for (u32 j = 0; j < r; ++j) {
      const u32 v = edges[e * r + j];
      if (v < n) atomicAdd(deg + v, 1u);
      else bad = 1;
    }
    if (eround) eround[e] = 0;
  }
  if (bad) atomicOr(&ctl->flags, (u32)FLAG_BAD_ID);
}

__global__ void __launch_bounds__(kKBlock) k_scatter(const u32 *__restrict__ edges, u64 m, u32 r, u32 n,
                                                     u32 *__restrict__ cursor, u32 *__restrict__ inc) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    for (u32 j = 0; j < r; ++j) {
      const u32 v = edges[e * r + j];
      if (v < n) inc[atomicAdd(cursor + v, 1u)] = (u32)e;
    }
  }
}

// F_1 = {v : deg(v) < k}; writes every vertex's round (1 or 0) and, if fb is
// given, every word of the F_1 bitmap.
__global__ void __launch_bounds__(kKBlock) k_kscan(const u32 *__restrict__ deg, u32 n,
                                                   u32 *__restrict__ f0, int *__restrict__ vround,
                                                   u32 *__restrict__ fb, PeelCtl *__restrict__ ctl) {
  __shared__ u32 s_buf[kKBlock * 4];
  __shared__ u32 s_n, s_base;
  const u32 k = ctl->k;
  const u32 CH = kKBlock * 4;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  for (u64 c0 = (u64)blockIdx.x * CH; c0 < n; c0 += (u64)gridDim.x * CH) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const u64 v = c0 + (u64)it * kKBlock + threadIdx.x;
      const bool valid = v < n;
      const bool low = valid && deg[v] < k;
      if (valid && vround) vround[v] = low ? 1 : 0;
      const u32 ball = __ballot_sync(kFull, low);  // 32 consecutive vertices per warp
      if (fb && lane_id() == 0 && v - lane_id() < n) fb[v >> 5] = ball;
      const u32 p = warp_reserve<u32>(low, &s_n);
      if (low) s_buf[p] = (u32)v;
    }
    __syncthreads();
    const u32 nn = s_n;
    if (threadIdx.x == 0 && nn) s_base = atomicAdd(&ctl->n_next, nn);
    __syncthreads();
    for (u32 q = threadIdx.x; q < nn; q += kKBlock) f0[s_base + q] = s_buf[q];
    __syncthreads();
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
  }
}

// Degrees during the rounds: one u32 per vertex, or (D16, every degree below
// 2^16) two 16-bit halves per u32 word, which halves the array so it stays in
// L2 (64 MB at 2^25 vertices).  A half never underflows -- each incidence is
// removed once -- so subtracting 1 from it never borrows from its neighbour.
template <bool D16>
__device__ __forceinline__ u32 deg_dec(u32 *deg, u32 u) {
  if constexpr (D16) {
    const u32 sh = (u & 1u) << 4;
    return (atomicSub(deg + (u >> 1), 1u << sh) >> sh) & 0xffffu;
  } else {
    return atomicSub(deg + u, 1u);
  }
}

// Largest degree (decides whether the rounds run on 16-bit degrees).
// Degree histogram in 16-bit halves (vertex v in half v & 1 of word v >> 1),
// which are also the degrees the rounds decrement: half the bytes of 32-bit
// counts, so the counters stay in L2.  An increment that finds a half at
// 0xFFFF carried out of it; *ovf is then set and the caller counts in 32 bits
// instead.  Zeroes the edge-round output.
__global__ void __launch_bounds__(kKBlock) k_hist16(const u32 *__restrict__ edges, u64 m, u32 r, u32 n,
                                                    u32 *__restrict__ deg16, int *__restrict__ eround,
                                                    u32 *__restrict__ ovf, PeelCtl *__restrict__ ctl) {
  u32 bad = 0, carry = 0;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    for (u32 j = 0; j < r; ++j) {
      const u32 v = edges[e * r + j];
      if (v < n) {
        const u32 sh = (v & 1u) << 4;
        carry |= ((atomicAdd(deg16 + (v >> 1), 1u << sh) >> sh) & 0xffffu) == 0xffffu;
      } else {
        bad = 1;
      }
    }
    if (eround) eround[e] = 0;
  }
  if (bad) atomicOr(&ctl->flags, (u32)FLAG_BAD_ID);
  if (carry) atomicOr(ovf, 1u);
}

// deg[v] = half v & 1 of deg16[v >> 1] (the CSR build reads 32-bit degrees).
__global__ void __launch_bounds__(kKBlock) k_unpack16(const u32 *__restrict__ deg16, u32 n, u32 *__restrict__ deg) {
  for (u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x; w < ((u64)n + 1) / 2; w += (u64)gridDim.x * blockDim.x) {
    const u32 x = deg16[w];
    deg[2 * w] = x & 0xffffu;
    if (2 * w + 1 < n) deg[2 * w + 1] = x >> 16;
  }
}

// Removal of one frontier vertex v in round t (Sec. 1, step (B)): every edge
// of v still alive is claimed through its alive bit (the first of its
// vertices to get there removes it), its round is recorded, and the degrees
// of its r endpoints are decremented; push(u) for each endpoint whose degree
// falls from k to k - 1.  Up to four incidences are read and claimed at once,
// and a claimed edge's row is read in one load (R = 4: 16 bytes, R = 2: 8
// bytes; rows aligned to that) with its R decrements issued together.  R = 0:
// any r, one endpoint at a time.  eid (if given) maps a row to the caller's
// edge id for the edge-round output.  Returns the number of edges claimed.
template <int R, bool D16, typename Push>
__device__ __forceinline__ u32 remove_edges_of(u32 v, u32 t, const u32 *__restrict__ edges, u32 r, u32 n, u32 k,
                                               const u32 *__restrict__ off, const u32 *__restrict__ inc,
                                               u32 *__restrict__ alive, u32 *__restrict__ deg,
                                               const u32 *__restrict__ eid, int *__restrict__ eround, Push push) {
  u32 claimed = 0;
  const u32 b = off[v], e_end = off[v + 1];
  for (u32 p0 = b; p0 < e_end; p0 += 4) {
    u32 ev[4], old[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) ev[q] = p0 + q < e_end ? inc[p0 + q] : 0xffffffffu;  // edge ids are < 2^31
#pragma unroll
    for (int q = 0; q < 4; ++q)
      old[q] = ev[q] != 0xffffffffu ? atomicAnd(alive + (ev[q] >> 5), ~(1u << (ev[q] & 31u))) : 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (ev[q] == 0xffffffffu || !((old[q] >> (ev[q] & 31u)) & 1u)) continue;  // taken by another vertex
      const u32 e = ev[q];
      ++claimed;
      if (eround) eround[eid ? eid[e] : e] = (int)t;
      if constexpr (R == 0) {
        for (u32 h = 0; h < r; ++h) {
          const u32 u = edges[(u64)e * r + h];
          if (u < n && deg_dec<D16>(deg, u) == k) push(u);
        }
      } else {
        u32 u[R], od[R];
        if constexpr (R == 4) {
          const uint4 w = reinterpret_cast<const uint4 *>(edges)[e];
          u[0] = w.x, u[1] = w.y, u[2] = w.z, u[3] = w.w;
        } else if constexpr (R == 2) {
          const uint2 w = reinterpret_cast<const uint2 *>(edges)[e];
          u[0] = w.x, u[1] = w.y;
        } else {
#pragma unroll
          for (int h = 0; h < R; ++h) u[h] = edges[(u64)e * R + h];
        }
#pragma unroll
        for (int h = 0; h < R; ++h) od[h] = u[h] < n ? deg_dec<D16>(deg, u[h]) : 0u;
#pragma unroll
        for (int h = 0; h < R; ++h)
          if (u[h] < n && od[h] == k) push(u[h]);
      }
    }
  }
  return claimed;
}

// One round: remove F_t and its edges.
template <int R, bool D16>
__global__ void __launch_bounds__(kKBlock) k_kpeel(const u32 *__restrict__ edges, const u32 *__restrict__ eid,
                                                   u32 r, u32 n,
                                                   const u32 *__restrict__ off, const u32 *__restrict__ inc,
                                                   u32 *__restrict__ alive, u32 *__restrict__ deg,
                                                   u32 *__restrict__ f0, u32 *__restrict__ f1,
                                                   int *__restrict__ vround, int *__restrict__ eround,
                                                   PeelCtl *__restrict__ ctl) {
  __shared__ u32 s_buf[kKStage];
  __shared__ u32 s_n, s_base;
  __shared__ u64 s_red[kKBlock / 32];
  const u32 t = *(volatile u32 *)&ctl->round;
  const u32 nf = *(volatile u32 *)&ctl->n_front;
  const u32 k = ctl->k;
  const u32 *fin = (t & 1u) ? f0 : f1;  // round t reads F[(t-1) & 1]
  u32 *fout = (t & 1u) ? f1 : f0;       // and writes F[t & 1]
  u64 claimed = 0;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  for (u64 c0 = (u64)blockIdx.x * kKBlock; c0 < nf; c0 += (u64)gridDim.x * kKBlock) {
    const u64 i = c0 + threadIdx.x;
    if (i < nf) {
      claimed += remove_edges_of<R, D16>(fin[i], t, edges, r, n, k, off, inc, alive, deg, eid, eround, [&](u32 u) {
        if (vround) vround[u] = (int)t + 1;
        const u32 q = atomicAdd(&s_n, 1u);
        if (q < (u32)kKStage) s_buf[q] = u;
        else fout[atomicAdd(&ctl->n_next, 1u)] = u;
      });
    }
    __syncthreads();
    const u32 nn = min(s_n, (u32)kKStage);
    if (threadIdx.x == 0 && nn) s_base = atomicAdd(&ctl->n_next, nn);
    __syncthreads();
    for (u32 q = threadIdx.x; q < nn; q += kKBlock) fout[s_base + q] = s_buf[q];
    __syncthreads();
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
  }
  const u64 c = block_sum<u64, kKBlock>(claimed, s_red);
  if (threadIdx.x == 0 && c) atomicAdd(&ctl->claimed, c);
}

__global__ void k_kround_end(PeelCtl *__restrict__ ctl, PeelStats st, int set_cond,
                             cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  PeelCtl &c = *ctl;
  const u32 t = c.round;
  if (c.n_front > 0 && t > 0) {
    c.s -= c.n_front;
    c.m -= c.claimed;
    st.s[t - 1] = c.s;
    st.m[t - 1] = c.m;
  }
  c.claimed = 0;
  c.n_front = c.n_next;
  c.n_next = 0;
  u32 more = c.n_front > 0;
  if (more && t >= c.max_rounds) {
    c.flags |= FLAG_ROUND_LIMIT;
    more = 0;
  }
  if (more) c.round = t + 1;
  c.more = more;
  if (set_cond) cudaGraphSetConditional(cond, more);
}

// ---- edge-centric full rounds ------------------------------------------------
constexpr u32 kDead = 0xffffffffu;  // id of a list entry whose edge was removed in place
constexpr int kEItems = 4;          // list entries per thread per step

// The edge list of the edge-centric rounds: the caller's array at first (ids
// = positions), then two compacted copies (rows of r vertex ids + the
// caller's edge id of each row).  F_t is bitmap fb[t & 1] and list
// f[(t - 1) & 1], the same list convention as k_kpeel.
struct EdgeLists {
  const u32 *user;
  u32 *rows[2], *ids[2];
  u32 *fb[2];
  u32 *f[2];
};

template <int R>
__device__ __forceinline__ void load_row(const u32 *rows, u64 i, u32 (&u)[R]) {
  if constexpr (R == 4) {
    const uint4 w = __ldcs(reinterpret_cast<const uint4 *>(rows) + i);
    u[0] = w.x, u[1] = w.y, u[2] = w.z, u[3] = w.w;
  } else if constexpr (R == 2) {
    const uint2 w = __ldcs(reinterpret_cast<const uint2 *>(rows) + i);
    u[0] = w.x, u[1] = w.y;
  } else {
#pragma unroll
    for (int h = 0; h < R; ++h) u[h] = __ldcs(rows + i * R + h);
  }
}

template <int R>
__device__ __forceinline__ void store_row(u32 *rows, u64 i, const u32 (&u)[R]) {
  if constexpr (R == 4) {
    reinterpret_cast<uint4 *>(rows)[i] = make_uint4(u[0], u[1], u[2], u[3]);
  } else if constexpr (R == 2) {
    reinterpret_cast<uint2 *>(rows)[i] = make_uint2(u[0], u[1]);
  } else {
#pragma unroll
    for (int h = 0; h < R; ++h) rows[i * R + h] = u[h];
  }
}

// Round t, edge-centric: every listed edge with a vertex in F_t is removed --
// round recorded, one degree taken from each endpoint (with multiplicity), an
// endpoint whose degree falls from k to k - 1 pushed into F_{t+1} (bitmap,
// list, vertex round t + 1).  A compacting round copies the surviving edges to
// the other list; otherwise a removed edge's entry is marked dead in place.
// Entries are read kEItems per thread at once: ids, rows, then the frontier
// bits of every endpoint, so the loads of a step are all in flight together.
template <int R, bool D16>
__global__ void __launch_bounds__(kKBlock) k_eround(EdgeLists L, u32 n, u32 *__restrict__ deg,
                                                    int *__restrict__ vround, int *__restrict__ eround,
                                                    PeelCtl *__restrict__ ctl) {
  __shared__ u32 s_buf[kKStage];
  __shared__ u32 s_n, s_base;
  __shared__ u64 s_red[kKBlock / 32];
  const u32 t = *(volatile u32 *)&ctl->round;
  const u32 nf = *(volatile u32 *)&ctl->n_front;
  if (nf == 0) return;  // the iteration that only promotes F_1 (uniform)
  const u32 k = ctl->k;
  const u32 src = ctl->src;
  const u64 len = ctl->len;
  const bool compact = ctl->compact != 0;
  const u32 *srows = src == 2 ? L.user : L.rows[src];
  u32 *sids = src == 2 ? nullptr : L.ids[src];
  const u32 d = src == 0 ? 1u : 0u;
  u32 *drows = L.rows[d], *dids = L.ids[d];
  const u32 *ft = L.fb[t & 1u];
  u32 *fn = L.fb[(t + 1) & 1u];
  u32 *fout = L.f[t & 1u];
  u64 claimed = 0;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  auto push = [&](u32 v) {
    if (vround) vround[v] = (int)t + 1;
    atomicOr(fn + (v >> 5), 1u << (v & 31u));
    const u32 q = atomicAdd(&s_n, 1u);
    if (q < (u32)kKStage) s_buf[q] = v;
    else fout[atomicAdd(&ctl->n_next, 1u)] = v;
  };
  constexpr u32 CH = kKBlock * kEItems;
  for (u64 c0 = (u64)blockIdx.x * CH; c0 < len; c0 += (u64)gridDim.x * CH) {
    u32 id[kEItems], u[kEItems][R], w[kEItems][R];
#pragma unroll
    for (int it = 0; it < kEItems; ++it) {
      const u64 i = c0 + (u64)it * kKBlock + threadIdx.x;
      id[it] = i < len ? (sids ? __ldcs(sids + i) : (u32)i) : kDead;
    }
#pragma unroll
    for (int it = 0; it < kEItems; ++it) {
      if (id[it] != kDead) {
        load_row<R>(srows, c0 + (u64)it * kKBlock + threadIdx.x, u[it]);
      } else {
#pragma unroll
        for (int h = 0; h < R; ++h) u[it][h] = kDead;
      }
    }
#pragma unroll
    for (int it = 0; it < kEItems; ++it)
#pragma unroll
      for (int h = 0; h < R; ++h) w[it][h] = u[it][h] < n ? __ldcg(ft + (u[it][h] >> 5)) : 0u;
#pragma unroll
    for (int it = 0; it < kEItems; ++it) {
      bool hit = false;
#pragma unroll
      for (int h = 0; h < R; ++h) hit |= u[it][h] < n && ((w[it][h] >> (u[it][h] & 31u)) & 1u);
      if (hit) {
        ++claimed;
        if (eround) eround[id[it]] = (int)t;
        u32 od[R];
#pragma unroll
        for (int h = 0; h < R; ++h) od[h] = u[it][h] < n ? deg_dec<D16>(deg, u[it][h]) : 0u;
#pragma unroll
        for (int h = 0; h < R; ++h)
          if (u[it][h] < n && od[h] == k) push(u[it][h]);
        if (!compact) sids[c0 + (u64)it * kKBlock + threadIdx.x] = kDead;  // src != 2 here
      }
      const bool keep = compact && id[it] != kDead && !hit;
      const u32 pos = warp_reserve<u32>(keep, &ctl->len_next);
      if (keep) {
        store_row<R>(drows, pos, u[it]);
        dids[pos] = id[it];
      }
    }
    __syncthreads();
    const u32 nn = min(s_n, (u32)kKStage);
    if (threadIdx.x == 0 && nn) s_base = atomicAdd(&ctl->n_next, nn);
    __syncthreads();
    for (u32 q = threadIdx.x; q < nn; q += kKBlock) fout[s_base + q] = s_buf[q];
    __syncthreads();
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
  }
  const u64 c = block_sum<u64, kKBlock>(claimed, s_red);
  if (threadIdx.x == 0 && c) atomicAdd(&ctl->claimed, c);
}

// After round t's pass: F_t leaves its bitmap (which holds F_{t+2} next).
__global__ void __launch_bounds__(kKBlock) k_eclear(EdgeLists L, const PeelCtl *__restrict__ ctl) {
  const u32 t = *(volatile const u32 *)&ctl->round;
  const u32 nf = *(volatile const u32 *)&ctl->n_front;
  if (t == 0) return;
  const u32 *fin = L.f[(t - 1) & 1u];
  u32 *fb = L.fb[t & 1u];
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) fb[fin[i] >> 5] = 0;
}

// End of an edge-centric round: the statistics and promotion of k_kround_end,
// then the list (switch to the compacted copy), whether the next round
// compacts (half of the list is dead, or it is still the caller's array), and
// whether the incidence-list rounds take over: F_{t+1} holds fewer than
// 1 / sw_ratio vertices per edge left (sw_ratio = 0: never).
__global__ void k_eround_end(PeelCtl *__restrict__ ctl, PeelStats st, u32 sw_ratio, int set_cond,
                             cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  PeelCtl &c = *ctl;
  const u32 t = c.round;
  if (c.n_front > 0 && t > 0) {
    c.s -= c.n_front;
    c.m -= c.claimed;
    st.s[t - 1] = c.s;
    st.m[t - 1] = c.m;
    if (c.compact) {
      c.src = c.src == 0 ? 1u : 0u;
      c.len = c.len_next;
    }
  }
  c.len_next = 0;
  c.claimed = 0;
  c.n_front = c.n_next;
  c.n_next = 0;
  u32 more = c.n_front > 0;
  if (more && t >= c.max_rounds) {
    c.flags |= FLAG_ROUND_LIMIT;
    more = 0;
  }
  if (more) c.round = t + 1;
  c.compact = c.src == 2 || c.m * 2 <= c.len;
  c.sw = more && sw_ratio && (u64)c.n_front * sw_ratio < c.m;
  c.more = more;
  c.econt = more && !c.sw;
  if (set_cond) cudaGraphSetConditional(cond, c.econt);
}

// Before the hand-over: the live entries of list `from` (len entries) copied
// to the other list.
template <int R>
__global__ void __launch_bounds__(kKBlock) k_ecompact(EdgeLists L, u32 from, u64 len, PeelCtl *__restrict__ ctl) {
  const u32 *srows = L.rows[from], *sids = L.ids[from];
  u32 *drows = L.rows[from ^ 1u], *dids = L.ids[from ^ 1u];
  for (u64 c0 = (u64)blockIdx.x * kKBlock; c0 < len; c0 += (u64)gridDim.x * kKBlock) {
    const u64 i = c0 + threadIdx.x;
    const u32 id = i < len ? sids[i] : kDead;
    u32 u[R];
    if (id != kDead) load_row<R>(srows, i, u);
    const u32 pos = warp_reserve<u32>(id != kDead, &ctl->len_next);
    if (id != kDead) {
      store_row<R>(drows, pos, u);
      dids[pos] = id;
    }
  }
}

// ---------------------------------------------------------------------------
// Sub-round mode
// ---------------------------------------------------------------------------
constexpr int kMaxParts = 64;
constexpr int kSubStage = 2048;

struct Parts {
  u32 off[kMaxParts + 1];  // part j = vertex ids off[j] .. off[j+1]-1
  u32 p;
};

struct SubCtl {
  u64 claimed;  // edges removed in the current sub-round
  u64 s;        // vertices left
  u64 m;        // edges left
  u32 sub;      // number of the current sub-round (0 before the first)
  u32 part;     // its part
  u32 fb, fe;   // its frontier: queue entries fb .. fe-1 of that part
  u32 flags;
  u32 max_sub;
  u32 more;
  u32 k;
  u32 head[kMaxParts];  // entries consumed, per part
  u32 tail[kMaxParts];  // entries appended, per part
};

__device__ __forceinline__ u32 part_of(const Parts &P, u32 v) {
  u32 a = 0, b = P.p;  // the last j with off[j] <= v
  while (b - a > 1) {
    const u32 mid = (a + b) >> 1;
    if (P.off[mid] <= v) a = mid;
    else b = mid;
  }
  return a;
}

// Per-block staging of queue appends: entries are counted per part in shared
// memory and leave the block with one global atomic per part.
struct PartStage {
  u32 *buf;   // kSubStage vertices
  u32 *pt;    // their parts
  u32 *rank;  // their rank within the part in this block
  u32 *cnt;   // per part
  u32 *base;  // per part
  u32 *n;
};

__device__ __forceinline__ void stage_push(PartStage &S, const Parts &P, u32 *queue, SubCtl *ctl, u32 u) {
  const u32 j = part_of(P, u);
  const u32 q = atomicAdd(S.n, 1u);
  if (q < (u32)kSubStage) {
    S.buf[q] = u;
    S.pt[q] = j;
    S.rank[q] = atomicAdd(S.cnt + j, 1u);
  } else {
    const u32 slot = atomicAdd(&ctl->tail[j], 1u);
    if (slot < P.off[j + 1] - P.off[j]) queue[P.off[j] + slot] = u;
    else atomicOr(&ctl->flags, (u32)FLAG_INTERNAL);
  }
}

// Writes the block's staged entries; call with the whole block.
__device__ __forceinline__ void stage_flush(PartStage &S, const Parts &P, u32 *queue, SubCtl *ctl) {
  __syncthreads();
  for (u32 j = threadIdx.x; j < P.p; j += blockDim.x) {
    const u32 c = S.cnt[j];
    S.base[j] = c ? atomicAdd(&ctl->tail[j], c) : 0u;
  }
  __syncthreads();
  const u32 nn = min(*S.n, (u32)kSubStage);
  for (u32 q = threadIdx.x; q < nn; q += blockDim.x) {
    const u32 j = S.pt[q];
    const u32 slot = S.base[j] + S.rank[q];
    if (slot < P.off[j + 1] - P.off[j]) queue[P.off[j] + slot] = S.buf[q];
    else atomicOr(&ctl->flags, (u32)FLAG_INTERNAL);
  }
  __syncthreads();
  for (u32 j = threadIdx.x; j < P.p; j += blockDim.x) S.cnt[j] = 0;
  if (threadIdx.x == 0) *S.n = 0;
  __syncthreads();
}

#define PP_PART_STAGE                                                             \
  __shared__ u32 s_buf[kSubStage], s_pt[kSubStage], s_rank[kSubStage];            \
  __shared__ u32 s_cnt[kMaxParts], s_base[kMaxParts], s_n;                        \
  PartStage S{s_buf, s_pt, s_rank, s_cnt, s_base, &s_n};                          \
  for (u32 j = threadIdx.x; j < kMaxParts; j += blockDim.x) s_cnt[j] = 0;         \
  if (threadIdx.x == 0) s_n = 0;                                                  \
  __syncthreads();

__global__ void k_kinit_sub(SubCtl *ctl, u64 n, u64 m, u32 k, u32 max_sub, u32 p) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    SubCtl c;
    memset(&c, 0, sizeof c);
    c.s = n;
    c.m = m;
    c.k = k;
    c.max_sub = max_sub;
    c.part = p - 1;  // the first sub-round looks at part 0
    *ctl = c;
  }
}

// The queues before the first sub-round: every vertex of degree < k.
__global__ void __launch_bounds__(kKBlock) k_kscan_sub(const u32 *__restrict__ deg, u32 n, const Parts P,
                                                       u32 *__restrict__ queue, int *__restrict__ vround,
                                                       SubCtl *__restrict__ ctl) {
  PP_PART_STAGE
  const u32 k = ctl->k;
  const u32 CH = kKBlock * 4;
  for (u64 c0 = (u64)blockIdx.x * CH; c0 < n; c0 += (u64)gridDim.x * CH) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const u64 v = c0 + (u64)it * kKBlock + threadIdx.x;
      if (v < n) {
        if (vround) vround[v] = 0;
        if (deg[v] < k) stage_push(S, P, queue, ctl, (u32)v);
      }
    }
    stage_flush(S, P, queue, ctl);
  }
}

// One sub-round: remove the frontier of the current part and its edges.
template <int R, bool D16>
__global__ void __launch_bounds__(kKBlock) k_kpeel_sub(const u32 *__restrict__ edges, u32 r, u32 n,
                                                       const u32 *__restrict__ off, const u32 *__restrict__ inc,
                                                       u32 *__restrict__ alive, u32 *__restrict__ deg,
                                                       const Parts P, u32 *__restrict__ queue,
                                                       int *__restrict__ vround, int *__restrict__ eround,
                                                       SubCtl *__restrict__ ctl) {
  PP_PART_STAGE
  __shared__ u64 s_red[kKBlock / 32];
  const u32 t = *(volatile u32 *)&ctl->sub;
  const u32 j = *(volatile u32 *)&ctl->part;
  const u32 fb = *(volatile u32 *)&ctl->fb, fe = *(volatile u32 *)&ctl->fe;
  const u32 k = ctl->k;
  const u32 *front = queue + P.off[j];
  u64 claimed = 0;
  for (u64 c0 = (u64)fb + (u64)blockIdx.x * kKBlock; c0 < fe; c0 += (u64)gridDim.x * kKBlock) {
    const u64 i = c0 + threadIdx.x;
    if (i < fe) {
      const u32 v = front[i];
      if (vround) vround[v] = (int)t;
      claimed += remove_edges_of<R, D16>(v, t, edges, r, n, k, off, inc, alive, deg, nullptr, eround,
                                         [&](u32 u) { stage_push(S, P, queue, ctl, u); });
    }
    stage_flush(S, P, queue, ctl);
  }
  const u64 c = block_sum<u64, kKBlock>(claimed, s_red);
  if (threadIdx.x == 0 && c) atomicAdd(&ctl->claimed, c);
}

// End of a sub-round: statistics, then the next sub-round whose part has
// something due (the idle ones in between keep their numbers and statistics).
__global__ void k_kround_end_sub(SubCtl *__restrict__ ctl, PeelStats st, const Parts P, int set_cond,
                                 cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  SubCtl &c = *ctl;
  const u32 t = c.sub;
  if (t > 0) {
    c.s -= c.fe - c.fb;
    c.m -= c.claimed;
    st.s[t - 1] = c.s;
    st.m[t - 1] = c.m;
    c.head[c.part] = c.fe;
  }
  c.claimed = 0;
  u32 more = 0, d = 1;
  for (; d <= P.p; ++d) {
    const u32 j = (c.part + d) % P.p;
    if (c.tail[j] > c.head[j]) {
      more = 1;
      break;
    }
  }
  if (more && (u64)t + d > c.max_sub) {
    c.flags |= FLAG_ROUND_LIMIT;
    more = 0;
  }
  if (more) {
    for (u32 q = 1; q < d; ++q) {  // idle sub-rounds
      st.s[t + q - 1] = c.s;
      st.m[t + q - 1] = c.m;
    }
    const u32 j = (c.part + d) % P.p;
    c.sub = t + d;
    c.part = j;
    c.fb = c.head[j];
    c.fe = c.tail[j];
  }
  c.more = more;
  if (set_cond) cudaGraphSetConditional(cond, more);
}

}  // namespace pp

namespace {

struct KWork {
  u32 *deg = nullptr, *off = nullptr, *cursor = nullptr, *inc = nullptr, *alive = nullptr;
  u32 *f0 = nullptr, *f1 = nullptr;
  u32 *deg16 = nullptr, *ovf = nullptr;
  void *block = nullptr;  // the buffers below up to scan_tmp live in it
  u32 *rows[2] = {nullptr, nullptr}, *ids[2] = {nullptr, nullptr}, *fb[2] = {nullptr, nullptr};
  PeelCtl *ctl = nullptr;
  SubCtl *sub = nullptr;
  u64 *st_s = nullptr, *st_m = nullptr;
  void *scan_tmp = nullptr;
};

struct KPeelArgs {
  const u32 *edges, *eid;
  u32 r, n;
  const u32 *off, *inc;
  u32 *alive, *deg, *f0, *f1;
  int *vround, *eround;
  PeelCtl *ctl;
  void *p[13];
  void bind() {
    void *q[13] = {&edges, &eid, &r, &n, &off, &inc, &alive, &deg, &f0, &f1, &vround, &eround, &ctl};
    memcpy(p, q, sizeof q);
  }
};

struct KEdgeArgs {
  EdgeLists L;
  u32 n;
  u32 *deg;
  int *vround, *eround;
  PeelCtl *ctl;
  void *p[6], *pc[2];
  void bind() {
    void *q[6] = {&L, &n, &deg, &vround, &eround, &ctl};
    void *qc[2] = {&L, &ctl};
    memcpy(p, q, sizeof q);
    memcpy(pc, qc, sizeof qc);
  }
};

struct KEEndArgs {
  PeelCtl *ctl;
  PeelStats st;
  u32 sw_ratio;
  int set_cond;
  cudaGraphConditionalHandle cond;
  void *p[5];
  void bind() {
    void *q[5] = {&ctl, &st, &sw_ratio, &set_cond, &cond};
    memcpy(p, q, sizeof q);
  }
};

const void *pick_eround(int rk, bool d16) {
  switch (rk) {
    case 2: return d16 ? (const void *)k_eround<2, true> : (const void *)k_eround<2, false>;
    case 3: return d16 ? (const void *)k_eround<3, true> : (const void *)k_eround<3, false>;
    default: return d16 ? (const void *)k_eround<4, true> : (const void *)k_eround<4, false>;
  }
}

const void *pick_ecompact(int rk) {
  switch (rk) {
    case 2: return (const void *)k_ecompact<2>;
    case 3: return (const void *)k_ecompact<3>;
    default: return (const void *)k_ecompact<4>;
  }
}

struct KEndArgs {
  PeelCtl *ctl;
  PeelStats st;
  int set_cond;
  cudaGraphConditionalHandle cond;
  void *p[4];
  void bind() {
    void *q[4] = {&ctl, &st, &set_cond, &cond};
    memcpy(p, q, sizeof q);
  }
};

struct KSubPeelArgs {
  const u32 *edges;
  u32 r, n;
  const u32 *off, *inc;
  u32 *alive, *deg;
  Parts P;
  u32 *queue;
  int *vround, *eround;
  SubCtl *ctl;
  void *p[12];
  void bind() {
    void *q[12] = {&edges, &r, &n, &off, &inc, &alive, &deg, &P, &queue, &vround, &eround, &ctl};
    memcpy(p, q, sizeof q);
  }
};

struct KSubEndArgs {
  SubCtl *ctl;
  PeelStats st;
  Parts P;
  int set_cond;
  cudaGraphConditionalHandle cond;
  void *p[5];
  void bind() {
    void *q[5] = {&ctl, &st, &P, &set_cond, &cond};
    memcpy(p, q, sizeof q);
  }
};

template <int R>
const void *peel_kernel(bool sub, bool d16) {
  if (sub) return d16 ? (const void *)k_kpeel_sub<R, true> : (const void *)k_kpeel_sub<R, false>;
  return d16 ? (const void *)k_kpeel<R, true> : (const void *)k_kpeel<R, false>;
}

// round kernel for rank rk (2, 3, 4, or 0 = any) and the degree width
const void *pick_peel(bool sub, int rk, bool d16) {
  switch (rk) {
    case 2: return peel_kernel<2>(sub, d16);
    case 3: return peel_kernel<3>(sub, d16);
    case 4: return peel_kernel<4>(sub, d16);
    default: return peel_kernel<0>(sub, d16);
  }
}

// Round-loop graphs, instantiated once per thread and kernel/grid set and kept:
// a call only rewrites the kernel nodes' arguments before launching
// (instantiating costs more than a whole peel of a small graph).  Never freed:
// their number is bounded by the kernel variants and the CUDA context may be
// gone by the time the thread exits.
struct LoopGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t peel = nullptr, mid = nullptr, end = nullptr;
  cudaGraphConditionalHandle h = 0;
};

struct LoopKey {
  const void *peel, *mid, *end;
  int grid, mid_grid, dev;
  bool operator<(const LoopKey &o) const {
    return std::tie(peel, mid, end, grid, mid_grid, dev) < std::tie(o.peel, o.mid, o.end, o.grid, o.mid_grid, o.dev);
  }
};

std::map<LoopKey, LoopGraph> &loop_graphs() {
  static thread_local std::map<LoopKey, LoopGraph> *m = new std::map<LoopKey, LoopGraph>();
  return *m;
}

inline cudaKernelNodeParams kernel_node(const void *fn, int grid, int block, void **args) {
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void *>(fn);
  kp.gridDim = dim3((unsigned)grid);
  kp.blockDim = dim3((unsigned)block);
  kp.kernelParams = args;
  return kp;
}

// The round loop: a CUDA graph whose while node runs peel -> [mid ->]
// round_end until round_end clears the condition, or the same kernels driven
// from the host.
template <class EndArgs>
pp_status run_rounds(const void *peel_fn, void **peel_p, const void *end_fn, EndArgs &ea, int grid,
                     bool host_loop, cudaStream_t s, const u32 *d_more, const void *mid_fn = nullptr,
                     void **mid_p = nullptr, int mid_grid = 0) {
  if (host_loop) {
    u32 more = 0;
    for (;;) {
      PP_CUDA(cudaLaunchKernel(peel_fn, dim3(grid), dim3(kKBlock), peel_p, 0, s));
      if (mid_fn) PP_CUDA(cudaLaunchKernel(mid_fn, dim3(mid_grid), dim3(kKBlock), mid_p, 0, s));
      PP_CUDA(cudaLaunchKernel(end_fn, dim3(1), dim3(32), ea.p, 0, s));
      PP_CUDA(cudaMemcpyAsync(&more, d_more, sizeof more, cudaMemcpyDeviceToHost, s));
      PP_CUDA(cudaStreamSynchronize(s));
      if (!more) break;
    }
    return PP_OK;
  }
  int dev = 0;
  PP_CUDA(cudaGetDevice(&dev));
  const LoopKey key{peel_fn, mid_fn, end_fn, grid, mid_fn ? mid_grid : 0, dev};
  auto &cache = loop_graphs();
  auto it = cache.find(key);
  if (it != cache.end()) {
    LoopGraph &lg = it->second;
    ea.set_cond = 1;
    ea.cond = lg.h;
    ea.bind();
    cudaKernelNodeParams kp = kernel_node(peel_fn, grid, kKBlock, peel_p);
    bool ok = cudaGraphExecKernelNodeSetParams(lg.exec, lg.peel, &kp) == cudaSuccess;
    if (ok && mid_fn) {
      kp = kernel_node(mid_fn, mid_grid, kKBlock, mid_p);
      ok = cudaGraphExecKernelNodeSetParams(lg.exec, lg.mid, &kp) == cudaSuccess;
    }
    if (ok) {
      kp = kernel_node(end_fn, 1, 32, ea.p);
      ok = cudaGraphExecKernelNodeSetParams(lg.exec, lg.end, &kp) == cudaSuccess;
    }
    if (ok) {
      PP_CUDA(cudaGraphLaunch(lg.exec, s));
      return PP_OK;
    }
    cudaGetLastError();  // the update was refused: build the graph again
    cudaStreamSynchronize(s);
    cudaGraphExecDestroy(lg.exec);
    cudaGraphDestroy(lg.g);
    cache.erase(it);
  }
  LoopGraph lg;
  cudaGraph_t body;
  cudaGraphNodeParams cp{};
  cudaGraphNode_t n_cond;
  cudaKernelNodeParams kp{};
  pp_status st = PP_OK;
  PP_CUDA(cudaGraphCreate(&lg.g, 0));
  if (cudaGraphConditionalHandleCreate(&lg.h, lg.g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    st = fail(PP_ERR_CUDA, "cudaGraphConditionalHandleCreate failed");
    goto fail_out;
  }
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = lg.h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (cudaGraphAddNode(&n_cond, lg.g, nullptr, nullptr, 0, &cp) != cudaSuccess) {
    st = fail(PP_ERR_CUDA, "cudaGraphAddNode(conditional while) failed");
    goto fail_out;
  }
  body = cp.conditional.phGraph_out[0];
  ea.set_cond = 1;
  ea.cond = lg.h;
  ea.bind();
  kp = kernel_node(peel_fn, grid, kKBlock, peel_p);
  if (cudaGraphAddKernelNode(&lg.peel, body, nullptr, 0, &kp) != cudaSuccess) {
    st = fail(PP_ERR_CUDA, "cudaGraphAddKernelNode(peel) failed");
    goto fail_out;
  }
  if (mid_fn) {
    kp = kernel_node(mid_fn, mid_grid, kKBlock, mid_p);
    if (cudaGraphAddKernelNode(&lg.mid, body, &lg.peel, 1, &kp) != cudaSuccess) {
      st = fail(PP_ERR_CUDA, "cudaGraphAddKernelNode(round middle) failed");
      goto fail_out;
    }
  }
  kp = kernel_node(end_fn, 1, 32, ea.p);
  if (cudaGraphAddKernelNode(&lg.end, body, mid_fn ? &lg.mid : &lg.peel, 1, &kp) != cudaSuccess) {
    st = fail(PP_ERR_CUDA, "cudaGraphAddKernelNode(round_end) failed");
    goto fail_out;
  }
  if (cudaGraphInstantiate(&lg.exec, lg.g, 0) != cudaSuccess) {
    st = fail(PP_ERR_CUDA, "cudaGraphInstantiate failed");
    lg.exec = nullptr;
    goto fail_out;
  }
  if (cudaGraphLaunch(lg.exec, s) != cudaSuccess) {
    st = fail(PP_ERR_CUDA, "cudaGraphLaunch failed");
    cudaStreamSynchronize(s);
    cudaGraphExecDestroy(lg.exec);
    goto fail_out;
  }
  cache.emplace(key, lg);
  return PP_OK;
fail_out:
  cudaGraphDestroy(lg.g);
  return st;
}

}  // namespace

// Workspace of pp_peel_kcore: a memory pool owned by the library (one per
// device), whose freed blocks stay mapped for the next call instead of going
// back to the driver at every synchronisation (the default pool's behaviour,
// which cost about 5 ms per call at 2^25 vertices).
static cudaMemPool_t workspace_pool() {
  static cudaMemPool_t pools[64] = {};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

static cudaError_t ws_alloc(void **p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = workspace_pool();
  return pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
}

// The incidence scatter: tiled (kcore_csr.cuh) for large inputs, with the
// plain atomic scatter as the fallback when a slab's record list is full.
static pp_status scatter_incidences(const u32 *edges, uint64_t m, uint32_t r, uint32_t n, u32 *cursor, u32 *inc,
                                    int egrid, cudaStream_t s) {
  if (m * r < (1ull << 22)) {
    k_scatter<<<egrid, kKBlock, 0, s>>>(edges, m, r, n, cursor, inc);
    PP_CUDA(cudaGetLastError());
    return PP_OK;
  }
  const uint32_t ns = (uint32_t)(((uint64_t)n + kVSlabVerts - 1) / kVSlabVerts);
  const double span = (double)((uint64_t)n < kVSlabVerts ? n : kVSlabVerts);
  const uint64_t cap = (uint64_t)((double)m * r * span / (double)n * 1.1) + 4096;
  const uint64_t tcap = ((uint64_t)((double)cap / kVTilesPerSlab * 1.15) + 256 + 31) / 32 * 32;
  if (cap > 0xFFFFFFF0ull || tcap * kVTilesPerSlab * 2 > 0xFFFFFFFFull) {
    k_scatter<<<egrid, kKBlock, 0, s>>>(edges, m, r, n, cursor, inc);
    PP_CUDA(cudaGetLastError());
    return PP_OK;
  }
  u32 *rec_v = nullptr, *rec_e = nullptr, *count = nullptr, *flag = nullptr, *tv = nullptr, *te = nullptr;
  u32 *tcount = nullptr, *ov = nullptr, *oe = nullptr, *o_count = nullptr;
  cudaError_t e = cudaSuccess;
  auto al = [&](u32 **p, uint64_t words) {
    if (e == cudaSuccess) e = ws_alloc((void **)p, (words ? words : 1) * 4, s);
  };
  al(&rec_v, cap * ns);
  al(&rec_e, cap * ns);
  al(&count, ns);
  al(&flag, 1);
  al(&tv, 2 * tcap * kVTilesPerSlab);
  al(&te, 2 * tcap * kVTilesPerSlab);
  al(&tcount, 2 * kVTilesPerSlab);
  al(&ov, 3 * cap);
  al(&oe, 3 * cap);
  al(&o_count, ns);
  pp_status st = PP_OK;
  uint32_t h_flag = 0;
  if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, ns * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(tcount, 0, 2 * kVTilesPerSlab * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(o_count, 0, ns * 4, s);
  if (e != cudaSuccess) {
    st = cuda_fail(e, "pp_peel_kcore tiled scatter buffers", __FILE__, __LINE__);
  } else {
    VBinArgs vb{rec_v, rec_e, count, flag, (u32)cap, ns};
    const size_t smem_bin = (size_t)kVBinEdges * r * 8 + 3 * (size_t)ns * 4;
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute((const void *)k_vbin, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
      cudaFuncSetAttribute((const void *)k_vtile_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kVTileVerts * 4));
      attr = true;
    }
    const uint64_t steps = (m + kVBinEdges - 1) / kVBinEdges;
    const int pgrid = persistent_grid((const void *)k_vbin, kVThreads, smem_bin, 4);
    const int bgrid = (int)(steps < (uint64_t)pgrid ? steps : (uint64_t)pgrid);
    k_vbin<<<bgrid, kVThreads, smem_bin, s>>>(edges, m, r, n, vb);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(&h_flag, flag, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
      st = cuda_fail(e, "pp_peel_kcore incidence binning", __FILE__, __LINE__);
    } else if (h_flag) {
      // a slab got more incidences than its list holds (skewed degrees)
      k_scatter<<<egrid, kKBlock, 0, s>>>(edges, m, r, n, cursor, inc);
      if ((e = cudaGetLastError()) != cudaSuccess) st = cuda_fail(e, "pp_peel_kcore scatter", __FILE__, __LINE__);
    } else {
      VTileArgs ta{tv, te, tcount, tcap * kVTilesPerSlab, (u32)tcap, (u32)cap, ov, oe, o_count};
      const u32 sms = (u32)sm_count();
      for (u32 step = 0; step <= ns + 1 && st == PP_OK; ++step) {
        const u32 n_bin = step < ns ? 2 * sms : 0u;
        const u32 n_apply = (step >= 1 && step - 1 < ns) ? kVTilesPerSlab : (step == ns + 1 ? 2 * sms : 0u);
        if (n_apply + n_bin == 0) continue;
        k_vtile_step<<<n_apply + n_bin, kVThreads, kVTileVerts * 4, s>>>(vb, ta, cursor, inc, step, n_apply,
                                                                         n_bin, n);
        if ((e = cudaGetLastError()) != cudaSuccess) st = cuda_fail(e, "pp_peel_kcore tile scatter", __FILE__, __LINE__);
      }
    }
  }
  cudaFreeAsync(rec_v, s);
  cudaFreeAsync(rec_e, s);
  cudaFreeAsync(count, s);
  cudaFreeAsync(flag, s);
  cudaFreeAsync(tv, s);
  cudaFreeAsync(te, s);
  cudaFreeAsync(tcount, s);
  cudaFreeAsync(ov, s);
  cudaFreeAsync(oe, s);
  cudaFreeAsync(o_count, s);
  return st;
}

// ---- one-block rounds for small graphs ----------------------------------------
// A graph of at most kSmallV vertices and kSmallE edges peels inside one CTA:
// the degrees and each vertex's removal round live in shared memory, and round
// t is two passes separated by block barriers (Sec. 1's round rule):
//   R_t = the vertices still present whose degree is < k (marked with t);
//   D_t = the edges still present with an endpoint marked t; each is removed
//         and its endpoints lose one degree per incidence.
// Rescanning all n vertices and m edges per round costs less than the
// launches and host round trips of the general path at this size.
constexpr u32 kSmallV = 1u << 14;
constexpr u32 kSmallE = 1u << 16;
constexpr int kSmallThreads = 1024;

static size_t small_peel_smem(u32 n, u32 m) {
  return (size_t)n * 4 + (size_t)((n + 1) & ~1u) * 2 + (size_t)((m + 31) / 32) * 4;
}

__device__ __forceinline__ u32 block_sum_small(u32 v, u32 *acc) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if (lane_id() == 0 && v) atomicAdd(acc, v);
  __syncthreads();
  return *acc;
}

// R = 3 or 4: rows of that rank, unrolled; R = 0: any r <= PP_MAX_R.  Each
// thread loads the rows of B edges before testing them, so B rows per thread
// are in flight at once.
template <int R>
__global__ void __launch_bounds__(kSmallThreads, 1)
    k_small_peel(const u32 *__restrict__ edges, u32 m, u32 r, u32 n, u32 k, u32 max_rounds,
                 int *__restrict__ vround, int *__restrict__ eround, PeelCtl *__restrict__ ctl, PeelStats st) {
  extern __shared__ __align__(16) unsigned char smem[];
  u32 *deg = reinterpret_cast<u32 *>(smem);                                   // n
  unsigned short *vr = reinterpret_cast<unsigned short *>(deg + n);           // n (even count)
  u32 *ealive = reinterpret_cast<u32 *>(vr + ((n + 1) & ~1u));               // (m + 31) / 32
  __shared__ u32 s_acc[3], s_flags;
  const u32 tid = threadIdx.x, lane = lane_id();
  const u32 words = (m + 31) / 32;
  for (u32 v = tid; v < n; v += kSmallThreads) deg[v] = 0, vr[v] = 0;
  for (u32 w = tid; w < words; w += kSmallThreads)
    ealive[w] = (w + 1) * 32 <= m ? kFull : (1u << (m & 31u)) - 1u;
  if (tid == 0) s_flags = 0;
  __syncthreads();
  // degrees with multiplicity; the edge-round output starts at 0 (in the core)
  u32 bad = 0;
  for (u32 e = tid; e < m; e += kSmallThreads) {
    for (u32 j = 0; j < r; ++j) {
      const u32 v = edges[(u64)e * r + j];
      if (v < n) atomicAdd(deg + v, 1u);
      else bad = 1;
    }
    if (eround) eround[e] = 0;
  }
  if (bad) atomicOr(&s_flags, (u32)FLAG_BAD_ID);
  __syncthreads();
  u64 s_left = n, m_left = m;
  u32 t = 1;
  if (!(s_flags & FLAG_BAD_ID)) {
    for (;; ++t) {
      if (tid < 3) s_acc[tid] = 0;
      __syncthreads();
      // past the limit R_t is marked (as the pending frontier of the other
      // paths is) but not removed
      const bool run = t <= max_rounds;
      u32 nr = 0;
      for (u32 v = tid; v < n; v += kSmallThreads) {
        if (vr[v] == 0 && deg[v] < k) {
          ++nr;
          vr[v] = (unsigned short)t;
        }
      }
      const u32 removed = block_sum_small(nr, &s_acc[0]);
      if (removed == 0) break;
      if (!run) {
        if (tid == 0) s_flags |= FLAG_ROUND_LIMIT;
        break;
      }
      // one warp per 32-edge word of the alive bitmap
      constexpr int NR = R ? R : PP_MAX_R;
      constexpr int B = R ? 4 : 2;
      const u32 rr = R ? (u32)R : r;
      u32 ne = 0;
      for (u32 b0 = tid & ~31u; b0 < m; b0 += kSmallThreads * B) {
        u32 row[B][NR], word[B];
#pragma unroll
        for (int q = 0; q < B; ++q) {
          const u32 base = b0 + (u32)q * kSmallThreads, e = base + lane;
          word[q] = base < m ? ealive[base >> 5] : 0u;
          const bool live = e < m && ((word[q] >> lane) & 1u);
#pragma unroll
          for (int j = 0; j < NR; ++j) row[q][j] = (live && (u32)j < rr) ? edges[(u64)e * rr + j] : 0u;
        }
#pragma unroll
        for (int q = 0; q < B; ++q) {
          const u32 base = b0 + (u32)q * kSmallThreads, e = base + lane;
          bool hit = false;
          if (e < m && ((word[q] >> lane) & 1u)) {
#pragma unroll
            for (int j = 0; j < NR; ++j)
              if ((u32)j < rr) hit |= vr[row[q][j]] == t;
            if (hit) {
#pragma unroll
              for (int j = 0; j < NR; ++j)
                if ((u32)j < rr) atomicSub(deg + row[q][j], 1u);
              if (eround) eround[e] = (int)t;
            }
          }
          const u32 ball = __ballot_sync(kFull, hit);
          if (lane == 0 && ball) ealive[base >> 5] = word[q] & ~ball;
          ne += hit;
        }
      }
      const u32 gone = block_sum_small(ne, &s_acc[1]);
      s_left -= removed;
      m_left -= gone;
      if (tid == 0) {
        st.s[t - 1] = s_left;
        st.m[t - 1] = m_left;
      }
      __syncthreads();  // s_acc is reset for the next round
    }
  }
  __syncthreads();
  if (vround && !(s_flags & FLAG_BAD_ID))
    for (u32 v = tid; v < n; v += kSmallThreads) vround[v] = (int)vr[v];
  if (tid == 0) {
    PeelCtl c;
    memset(&c, 0, sizeof c);
    c.s = s_left;
    c.m = m_left;
    c.k = k;
    c.max_rounds = max_rounds;
    c.round = t - 1;
    c.flags = s_flags;
    *ctl = c;
  }
}

// The one-block path's results go to mapped pinned memory owned by the calling
// thread (control block, then s_t and m_t for up to n rounds): the call
// allocates nothing and synchronizes once.  Calls return only after that
// synchronization, so one buffer per thread is never shared by two calls.
static pp_status peel_small(uint32_t n, uint32_t r, uint32_t k, const uint32_t *d_edges, uint64_t m,
                            int32_t *d_vertex_round, int32_t *d_edge_round, pp_peel_result *res,
                            const pp_options &o, cudaStream_t s) {
  struct Stage {
    void *h = nullptr;
    size_t bytes = 0;
    ~Stage() {
      if (h) cudaFreeHost(h);  // at thread exit; an error at process teardown is ignored
    }
  };
  thread_local Stage stage;
  const size_t ctl_bytes = (sizeof(PeelCtl) + 255) & ~(size_t)255;
  const size_t bytes = ctl_bytes + 2 * ((size_t)kSmallV + 1) * 8;
  if (stage.bytes < bytes) {
    void *h = nullptr;
    const cudaError_t e = cudaHostAlloc(&h, bytes, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) return cuda_fail(e, "pp_peel_kcore pinned stage", __FILE__, __LINE__);
    stage.h = h;
    stage.bytes = bytes;
  }
  char *hb = static_cast<char *>(stage.h);
  void *db = nullptr;
  cudaError_t e = cudaHostGetDevicePointer(&db, stage.h, 0);
  if (e != cudaSuccess) return cuda_fail(e, "pp_peel_kcore pinned stage", __FILE__, __LINE__);
  static std::once_flag small_attr;
  const void *fns[3] = {(const void *)k_small_peel<3>, (const void *)k_small_peel<4>,
                        (const void *)k_small_peel<0>};
  std::call_once(small_attr, [&fns] {
    for (const void *f : fns)
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_peel_smem(kSmallV, kSmallE));
  });
  const void *fn = r == 3 ? fns[0] : r == 4 ? fns[1] : fns[2];
  u32 m32 = (u32)m, n32 = n, r32 = r, k32 = k, mr32 = o.max_rounds;
  int *vr_out = d_vertex_round, *er_out = d_edge_round;
  PeelCtl *ctlp = reinterpret_cast<PeelCtl *>(db);
  u64 *ss = reinterpret_cast<u64 *>(static_cast<char *>(db) + ctl_bytes);
  PeelStats pst{ss, ss + kSmallV + 1};
  void *kargs[] = {(void *)&d_edges, &m32, &r32, &n32, &k32, &mr32, &vr_out, &er_out, &ctlp, &pst};
  e = cudaLaunchKernel(fn, dim3(1), dim3(kSmallThreads), kargs, small_peel_smem(n, m32), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "pp_peel_kcore small-graph path", __FILE__, __LINE__);
  PeelCtl hc;
  memcpy(&hc, hb, sizeof hc);
  const u64 *hs = reinterpret_cast<const u64 *>(hb + ctl_bytes);
  const uint32_t T = hc.round;
  const uint32_t ncopy = T < res->round_cap ? T : res->round_cap;
  if (ncopy && res->vertices_left) memcpy(res->vertices_left, hs, (size_t)ncopy * 8);
  if (ncopy && res->edges_left) memcpy(res->edges_left, hs + kSmallV + 1, (size_t)ncopy * 8);
  res->rounds = T;
  res->status_flags = hc.flags;
  res->core_vertices = hc.s;
  res->core_edges = hc.m;
  if (hc.flags & FLAG_BAD_ID) return fail(PP_ERR_INVALID_ARG, "pp_peel_kcore: a vertex id is >= n=%u", n);
  if (hc.flags & FLAG_ROUND_LIMIT)
    return fail(PP_ERR_ROUND_LIMIT, "pp_peel_kcore: stopped after max_rounds=%u (sub-)rounds", o.max_rounds);
  return PP_OK;
}

static pp_status peel_kcore_impl(uint32_t n, uint32_t r, uint32_t k, const uint32_t *d_edges, uint64_t m,
                          const Parts *parts, int32_t *d_vertex_round, int32_t *d_edge_round,
                          pp_peel_result *res, const pp_options *opt, void *stream) {
  if (!res) return fail(PP_ERR_INVALID_ARG, "pp_peel_kcore: NULL result");
  if (k < 1) return fail(PP_ERR_INVALID_ARG, "pp_peel_kcore: k=%u < 1", k);
  if (r < 2 || r > PP_MAX_R) return fail(PP_ERR_INVALID_ARG, "pp_peel_kcore: r=%u outside 2..%d", r, PP_MAX_R);
  if ((uint64_t)n > 0xFFFFFFFFull - 64) return fail(PP_ERR_INVALID_ARG, "pp_peel_kcore: n too large");
  if (m > (0xFFFFFFFFull - 64) / r) return fail(PP_ERR_INVALID_ARG, "pp_peel_kcore: m*r >= 2^32-64");
  if (m && !d_edges) return fail(PP_ERR_INVALID_ARG, "pp_peel_kcore: NULL edges");
  const pp_options o = resolve_options(opt);
  cudaStream_t s = as_stream(stream);
  KWork w;
  const u64 nn = n ? n : 1, mm = m ? m : 1;
  cudaError_t e = cudaSuccess;
  // one workspace block, carved into 256-byte aligned buffers
  struct Part {
    void **p;
    size_t bytes;
  };
  Part parts_list[16];
  int np_ = 0;
  auto al = [&](void **p, size_t b) { parts_list[np_++] = Part{p, (b + 255) & ~(size_t)255}; };
  // small graphs in automatic mode peel in one block (k_small_peel)
  if (!parts && n > 0 && m > 0 && n <= kSmallV && m <= kSmallE && o.kcore_mode == 0 && o.host_loop == 0)
    return peel_small(n, r, k, d_edges, m, d_vertex_round, d_edge_round, res, o, s);
  {
    al((void **)&w.deg, nn * 4);
    al((void **)&w.off, (nn + 1) * 4);
    al((void **)&w.cursor, nn * 4);
    al((void **)&w.inc, mm * r * 4);
    al((void **)&w.alive, ((mm + 31) / 32) * 4);
    al((void **)&w.f0, nn * 4);
    al((void **)&w.f1, nn * 4);
    al((void **)&w.deg16, ((nn + 1) / 2) * 4);
    al((void **)&w.ovf, sizeof(u32));
    al(&w.scan_tmp, exclusive_scan_temp_bytes(nn));
  }
  al((void **)&w.ctl, sizeof(PeelCtl));
  if (parts) al((void **)&w.sub, sizeof(SubCtl));
  al((void **)&w.st_s, (size_t)o.max_rounds * 8);
  al((void **)&w.st_m, (size_t)o.max_rounds * 8);
  {
    size_t total = 0;
    for (int i = 0; i < np_; ++i) total += parts_list[i].bytes;
    e = ws_alloc(&w.block, total, s);
    if (e == cudaSuccess) {
      char *q = static_cast<char *>(w.block);
      for (int i = 0; i < np_; ++i) {
        *parts_list[i].p = q;
        q += parts_list[i].bytes;
      }
    }
  }
  pp_status status = PP_OK;
  PeelCtl hc{};
  SubCtl hsub{};
  uint32_t T = 0, ncopy = 0;
  if (e != cudaSuccess) {
    status = cuda_fail(e, "pp_peel_kcore workspace", __FILE__, __LINE__);
    goto cleanup;
  }
  {
    const int sms = sm_count();
    const u64 eb = (m + kKBlock - 1) / kKBlock;
    const int egrid = (int)(eb < (u64)sms * 16 ? (eb ? eb : 1) : (u64)sms * 16);
    const u64 vb = (nn + kKBlock * 4 - 1) / (kKBlock * 4);
    const int vgrid = (int)(vb < (u64)sms * 8 ? vb : (u64)sms * 8);
    {
    if ((e = cudaMemsetAsync(w.deg16, 0, ((nn + 1) / 2) * 4, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(w.ovf, 0, sizeof(u32), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(w.alive, 0xff, ((mm + 31) / 32) * 4, s)) != cudaSuccess) {
      status = cuda_fail(e, "pp_peel_kcore memset", __FILE__, __LINE__);
      goto cleanup;
    }
    k_kinit<<<1, 32, 0, s>>>(w.ctl, n, m, k, o.max_rounds);
    // degrees in 16-bit counters, which the rounds then decrement in place;
    // a degree above 0xFFFF sends the call to 32-bit counters
    if (m) k_hist16<<<egrid, kKBlock, 0, s>>>(d_edges, m, r, n, w.deg16, d_edge_round, w.ovf, w.ctl);
    uint32_t h_ovf = 0;
    if ((e = cudaMemcpyAsync(&h_ovf, w.ovf, sizeof(u32), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
      status = cuda_fail(e, "pp_peel_kcore degree readback", __FILE__, __LINE__);
      goto cleanup;
    }
    const bool d16 = h_ovf == 0;
    if (d16) {
      if (n) k_unpack16<<<vgrid, kKBlock, 0, s>>>(w.deg16, n, w.deg);
    } else {
      if ((e = cudaMemsetAsync(w.deg, 0, nn * 4, s)) != cudaSuccess) {
        status = cuda_fail(e, "pp_peel_kcore memset", __FILE__, __LINE__);
        goto cleanup;
      }
      k_hist<<<egrid, kKBlock, 0, s>>>(d_edges, m, r, n, w.deg, d_edge_round, w.ctl);
    }
    // rank-specialised rounds where the edge rows allow their vector loads
    const uintptr_t ea = (uintptr_t)d_edges;
    const int rk = (r == 4 && ea % 16 == 0) || (r == 2 && ea % 8 == 0) || r == 3 ? (int)r : 0;
    // edge-centric rounds are possible; they start if F_1 is large (or mode 2).
    // Below 2^20 edges the incidence lists cost little and mode 0 keeps them.
    const bool edge_ok = !parts && rk != 0 && m > 0 && n > 0 &&
                         (o.kcore_mode == 2 || (o.kcore_mode == 0 && m >= (1ull << 20)));
    bool edge_mode = false;
    u32 *rdeg = d16 ? w.deg16 : w.deg;
    // incidence lists of edges[0, me) (row i = edge i), from the current degrees
    auto build_csr = [&](const u32 *edges, uint64_t me) -> pp_status {
      pp_status st = exclusive_scan(w.deg, w.off, n, w.scan_tmp, s);
      if (st != PP_OK) return st;
      if (n && (e = cudaMemcpyAsync(w.cursor, w.off, (size_t)n * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "pp_peel_kcore cursor copy", __FILE__, __LINE__);
      if (me) return scatter_incidences(edges, me, r, n, w.cursor, w.inc, egrid, s);
      return PP_OK;
    };
    // vertex-centric rounds over edges[0, me), eid mapping rows to the caller's edge ids
    auto vertex_rounds = [&](const u32 *edges, const u32 *eid, uint64_t me) -> pp_status {
      if ((e = cudaMemsetAsync(w.alive, 0xff, ((me + 31) / 32 ? (me + 31) / 32 : 1) * 4, s)) != cudaSuccess)
        return cuda_fail(e, "pp_peel_kcore memset", __FILE__, __LINE__);
      KPeelArgs pa{edges, eid, r, n, w.off, w.inc, w.alive, rdeg, w.f0, w.f1, d_vertex_round, d_edge_round,
                   w.ctl, {}};
      pa.bind();
      KEndArgs kea{w.ctl, PeelStats{w.st_s, w.st_m}, 0, 0, {}};
      kea.bind();
      const void *peel = pick_peel(false, rk, d16);
      // no more blocks than a frontier of every vertex needs
      const int pgrid = (int)std::min<uint64_t>((uint64_t)persistent_grid(peel, kKBlock, 0, o.ctas_per_sm),
                                                (nn + kKBlock - 1) / kKBlock);
      return run_rounds(peel, pa.p, (const void *)k_kround_end, kea, pgrid, o.host_loop != 0, s, &w.ctl->more);
    };
    if (edge_ok) {
      const uint64_t words = ((uint64_t)nn + 31) / 32;
      for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = ws_alloc((void **)&w.fb[b], words * 4, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(w.fb[0], 0, words * 4, s);  // k_kscan writes fb[1]
      if (e != cudaSuccess) {
        status = cuda_fail(e, "pp_peel_kcore frontier bitmaps", __FILE__, __LINE__);
        goto cleanup;
      }
    }
    if (parts) {
      k_kinit_sub<<<1, 32, 0, s>>>(w.sub, n, m, k, o.max_rounds, parts->p);
      if (n) k_kscan_sub<<<vgrid, kKBlock, 0, s>>>(w.deg, n, *parts, w.f0, d_vertex_round, w.sub);
    } else if (n) {
      k_kscan<<<vgrid, kKBlock, 0, s>>>(w.deg, n, w.f0, d_vertex_round, edge_ok ? w.fb[1] : nullptr, w.ctl);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) {
      status = cuda_fail(e, "pp_peel_kcore build kernels", __FILE__, __LINE__);
      goto cleanup;
    }
    if (edge_ok) {
      if ((e = cudaMemcpyAsync(&hc, w.ctl, sizeof hc, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
          (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        status = cuda_fail(e, "pp_peel_kcore frontier readback", __FILE__, __LINE__);
        goto cleanup;
      }
      edge_mode = o.kcore_mode == 2 || (uint64_t)hc.n_next * o.frontier_switch >= m;
    }
    if (edge_mode) {
      for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = ws_alloc((void **)&w.rows[b], mm * r * 4, s);
        if (e == cudaSuccess) e = ws_alloc((void **)&w.ids[b], mm * 4, s);
      }
      if (e != cudaSuccess) {
        status = cuda_fail(e, "pp_peel_kcore edge lists", __FILE__, __LINE__);
        goto cleanup;
      }
    } else {
      status = build_csr(d_edges, m);
      if (status != PP_OK) goto cleanup;
    }
    if (parts) {
      KSubPeelArgs pa{d_edges, r, n, w.off, w.inc, w.alive, rdeg, *parts, w.f0, d_vertex_round,
                      d_edge_round, w.sub, {}};
      pa.bind();
      KSubEndArgs kea{w.sub, PeelStats{w.st_s, w.st_m}, *parts, 0, 0, {}};
      kea.bind();
      const void *peel = pick_peel(true, rk, d16);
      const int pgrid = (int)std::min<uint64_t>((uint64_t)persistent_grid(peel, kKBlock, 0, o.ctas_per_sm),
                                                (nn + kKBlock - 1) / kKBlock);
      status = run_rounds(peel, pa.p, (const void *)k_kround_end_sub, kea, pgrid,
                          o.host_loop != 0, s, &w.sub->more);
    } else if (!edge_mode) {
      status = vertex_rounds(d_edges, nullptr, m);
    } else {
      // edge-centric rounds while the frontier is large
      EdgeLists L{d_edges, {w.rows[0], w.rows[1]}, {w.ids[0], w.ids[1]}, {w.fb[0], w.fb[1]}, {w.f0, w.f1}};
      KEdgeArgs ka{L, n, rdeg, d_vertex_round, d_edge_round, w.ctl, {}, {}};
      ka.bind();
      KEEndArgs kea{w.ctl, PeelStats{w.st_s, w.st_m}, o.kcore_mode == 2 ? 0u : o.frontier_switch, 0, 0, {}};
      kea.bind();
      const void *er = pick_eround(rk, d16);
      const int pgrid = (int)std::min<uint64_t>((uint64_t)persistent_grid(er, kKBlock, 0, o.ctas_per_sm),
                                                (mm + kKBlock * kEItems - 1) / (kKBlock * kEItems));
      const int cgrid = (int)std::min<uint64_t>(
          (uint64_t)persistent_grid((const void *)k_eclear, kKBlock, 0, o.ctas_per_sm), (nn + kKBlock - 1) / kKBlock);
      status = run_rounds(er, ka.p, (const void *)k_eround_end, kea, pgrid, o.host_loop != 0, s, &w.ctl->econt,
                          (const void *)k_eclear, ka.pc, cgrid);
      if (status != PP_OK) goto cleanup;
      if ((e = cudaMemcpyAsync(&hc, w.ctl, sizeof hc, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
          (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        status = cuda_fail(e, "pp_peel_kcore readback", __FILE__, __LINE__);
        goto cleanup;
      }
      if (hc.more && hc.sw) {
        // hand-over: incidence lists for the edges left, vertex-centric rounds
        const u32 *edges = d_edges, *eid = nullptr;
        uint64_t me = m;
        if (hc.src != 2) {
          u32 cur = hc.src;
          if (hc.len > hc.m) {  // entries removed in place: copy the live ones
            const int g = (int)((hc.len + kKBlock - 1) / kKBlock < (uint64_t)sm_count() * 8
                                    ? (hc.len + kKBlock - 1) / kKBlock : (uint64_t)sm_count() * 8);
            u32 from = cur;
            u64 len = hc.len;
            PeelCtl *ctl = w.ctl;
            void *cp[4] = {&L, &from, &len, &ctl};
            if ((e = cudaLaunchKernel(pick_ecompact(rk), dim3(g), dim3(kKBlock), cp, 0, s)) != cudaSuccess) {
              status = cuda_fail(e, "pp_peel_kcore list compaction", __FILE__, __LINE__);
              goto cleanup;
            }
            cur ^= 1u;
          }
          edges = w.rows[cur];
          eid = w.ids[cur];
          me = hc.m;
        }
        if (d16 && n) k_unpack16<<<vgrid, kKBlock, 0, s>>>(w.deg16, n, w.deg);
        status = build_csr(edges, me);
        if (status == PP_OK) status = vertex_rounds(edges, eid, me);
      }
    }
    if (status != PP_OK) goto cleanup;
    }  // general path
    if ((e = cudaMemcpyAsync(&hc, w.ctl, sizeof hc, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (parts && (e = cudaMemcpyAsync(&hsub, w.sub, sizeof hsub, cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
      status = cuda_fail(e, "pp_peel_kcore readback", __FILE__, __LINE__);
      goto cleanup;
    }
    if (parts) {
      hc.round = hsub.sub;
      hc.flags |= hsub.flags;
      hc.s = hsub.s;
      hc.m = hsub.m;
    }
    T = hc.round;
    ncopy = T < res->round_cap ? T : res->round_cap;
    if (ncopy && res->vertices_left)
      e = cudaMemcpyAsync(res->vertices_left, w.st_s, ncopy * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && ncopy && res->edges_left)
      e = cudaMemcpyAsync(res->edges_left, w.st_m, ncopy * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      status = cuda_fail(e, "pp_peel_kcore stats readback", __FILE__, __LINE__);
      goto cleanup;
    }
    res->rounds = T;
    res->status_flags = hc.flags;
    res->core_vertices = hc.s;
    res->core_edges = hc.m;
    if (hc.flags & FLAG_BAD_ID) status = fail(PP_ERR_INVALID_ARG, "pp_peel_kcore: a vertex id is >= n=%u", n);
    else if (hc.flags & FLAG_INTERNAL) status = fail(PP_ERR_CUDA, "pp_peel_kcore: a part queue overflowed");
    else if (hc.flags & FLAG_ROUND_LIMIT)
      status = fail(PP_ERR_ROUND_LIMIT, "pp_peel_kcore: stopped after max_rounds=%u (sub-)rounds", o.max_rounds);
  }
cleanup:
  auto fr = [&](void *p) {
    if (p) cudaFreeAsync(p, s);
  };
  for (int b = 0; b < 2; ++b) {
    fr(w.rows[b]);
    fr(w.ids[b]);
    fr(w.fb[b]);
  }
  fr(w.block);
  cudaStreamSynchronize(s);
  return status;
}

extern "C" pp_status pp_peel_kcore(uint32_t n, uint32_t r, uint32_t k, const uint32_t *d_edges,
                                   uint64_t m, int32_t *d_vertex_round, int32_t *d_edge_round,
                                   pp_peel_result *res, const pp_options *opt, void *stream) {
  return peel_kcore_impl(n, r, k, d_edges, m, nullptr, d_vertex_round, d_edge_round, res, opt, stream);
}

extern "C" pp_status pp_peel_kcore_subrounds(uint32_t n, uint32_t r, uint32_t k, const uint32_t *d_edges,
                                             uint64_t m, uint32_t n_parts, const uint32_t *h_part_off,
                                             int32_t *d_vertex_round, int32_t *d_edge_round,
                                             pp_peel_result *res, const pp_options *opt, void *stream) {
  if (n_parts < 1 || n_parts > (uint32_t)kMaxParts)
    return fail(PP_ERR_INVALID_ARG, "pp_peel_kcore_subrounds: n_parts=%u outside 1..%d", n_parts, kMaxParts);
  if (!h_part_off) return fail(PP_ERR_INVALID_ARG, "pp_peel_kcore_subrounds: NULL part offsets");
  if (h_part_off[0] != 0 || h_part_off[n_parts] != n)
    return fail(PP_ERR_INVALID_ARG, "pp_peel_kcore_subrounds: part offsets must run from 0 to n=%u", n);
  Parts P{};
  P.p = n_parts;
  for (uint32_t j = 0; j <= n_parts; ++j) {
    if (j && h_part_off[j] < h_part_off[j - 1])
      return fail(PP_ERR_INVALID_ARG, "pp_peel_kcore_subrounds: part offsets decrease at %u", j);
    P.off[j] = h_part_off[j];
  }
  return peel_kcore_impl(n, r, k, d_edges, m, &P, d_vertex_round, d_edge_round, res, opt, stream);
}
