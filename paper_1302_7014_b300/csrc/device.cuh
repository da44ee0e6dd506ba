// Device-side building blocks shared by the peeling kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ppeel.h"

namespace pp {

typedef unsigned long long u64;
typedef unsigned int u32;
typedef unsigned short u16;

constexpr u32 kFull = 0xffffffffu;
constexpr u64 kGamma = 0x9E3779B97F4A7C15ULL;

// Device-side status flags (DecodeCtl::flags, PeelCtl::flags).
enum : u32 {
  FLAG_CAPACITY = 1u,     // an output index ran past its capacity
  FLAG_ROUND_LIMIT = 2u,  // max_rounds reached with a non-empty frontier
  FLAG_BAD_ID = 4u,       // a vertex id >= n was seen
  FLAG_INTERNAL = 8u      // an invariant failed (frontier cell not among its key's cells)
};

// One IBLT cell (Sec. 6 "Motivation"): the XOR of its keys, the XOR of their
// checksums and their count, padded to one 32-byte DRAM sector so that a
// random touch of a cell costs one sector.
struct __align__(32) Cell {
  u64 key;    // XOR of the keys in the cell
  u64 chk;    // XOR of checkSum(x) over the cell's keys
  int count;  // keys inserted minus keys deleted
  u32 pad0;   // always 0
  u64 pad1;   // always 0
};
static_assert(sizeof(Cell) == 32, "cell must be one 32-byte sector");
static_assert(sizeof(Cell) == sizeof(pp_cell), "public and device cell layouts differ");

// Whole-cell loads and stores: one 256-bit access each.  cs = streaming (read
// or written once), cg = cached in L2 only.
__device__ __forceinline__ void ld_cell_cs(const Cell *p, u64 &key, u64 &chk, int &count) {
  u64 w2;
  asm volatile("ld.global.cs.v4.u64 {%0,%1,%2,_}, [%3];" : "=l"(key), "=l"(chk), "=l"(w2) : "l"(p));
  count = (int)(u32)w2;
}
__device__ __forceinline__ void ld_cell_cg(const Cell *p, u64 &key, u64 &chk, int &count) {
  u64 w2;
  asm volatile("ld.global.cg.v4.u64 {%0,%1,%2,_}, [%3];" : "=l"(key), "=l"(chk), "=l"(w2) : "l"(p));
  count = (int)(u32)w2;
}
__device__ __forceinline__ void st_cell_cs(Cell *p, u64 key, u64 chk, int count) {
  asm volatile("st.global.cs.v4.u64 [%0], {%1,%2,%3,%4};" ::"l"(p), "l"(key), "l"(chk), "l"((u64)(u32)count),
               "l"(0ull)
               : "memory");
}

// SplitMix64 output finaliser (Steele, Lea & Flood 2014): the hash family of
// the IBLT (cell positions and checksums).
__host__ __device__ __forceinline__ u64 mix64(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// checkSum(x) of Sec. 6: mix64(x ^ seed_chk), 64 bits.  A cell holding exactly
// x (inserted or deleted) has chk == checksum(x).
__host__ __device__ __forceinline__ u64 checksum(u64 x, u64 seed_chk) { return mix64(x ^ seed_chk); }

// Pure (holds exactly one key, Sec. 6): count == 1 and chk == checkSum(key).
__host__ __device__ __forceinline__ bool cell_pure(int count, u64 key, u64 chk, u64 seed_chk) {
  return count == 1 && chk == checksum(key, seed_chk);
}

// Adds key x (checksum cs) to cell c with sign sg (+1 insert, -1 delete): the
// count moves by sg, both XOR fields take the key.  Returns the old count.
__device__ __forceinline__ int touch_cell(Cell *cells, u32 c, u64 x, u64 cs, int sg) {
  Cell *p = cells + c;
  const int old = atomicAdd(&p->count, sg);
  atomicXor(&p->key, x);
  atomicXor(&p->chk, cs);
  return old;
}
// The same with nothing read back (fire-and-forget reductions).
__device__ __forceinline__ void touch_cell_nr(Cell *cells, u32 c, u64 x, u64 cs, int sg) {
  Cell *p = cells + c;
  atomicAdd(&p->count, sg);
  atomicXor(&p->key, x);
  atomicXor(&p->chk, cs);
}

// XOR of v into the 64-bit word at p in shared memory: one 64-bit atomic
// (PP_SMEM_XOR64=1) or one 32-bit atomic per half (XOR acts bitwise, so the
// halves are independent).
#ifndef PP_SMEM_XOR64
#define PP_SMEM_XOR64 0
#endif
__device__ __forceinline__ void smem_xor64(u64 *p, u64 v) {
#if PP_SMEM_XOR64
  atomicXor(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
#else
  atomicXor(reinterpret_cast<u32 *>(p), (u32)v);
  atomicXor(reinterpret_cast<u32 *>(p) + 1, (u32)(v >> 32));
#endif
}

// Per-table constants.  Sub-table j is cells base+off[j] .. base+off[j+1]-1.
struct __align__(16) TableArgs {
  u64 seed[PP_MAX_R + 1];  // hash seeds s_0..s_{r-1}, checksum seed at [r]
  u32 off[PP_MAX_R + 1];
  u32 base;                // global id of cell 0 (a multiple of 32)
  u32 n_cells;
  u32 r;
  u32 start_round;         // global round that is this table's round 1 (batch/server)
  u64 out_base;            // batch: first slot of this table's output region
  u64 out_cap;             // batch: slots in that region
};

// Kernels are instantiated per rank R: R > 0 is a fixed r; R = 0 takes r at run
// time (up to PP_MAX_R); R = -4 takes r at run time with r <= 4 (mixed r = 3 / 4
// batches), sizing registers and shared memory for 4.
template <int R>
__host__ __device__ constexpr int nr_of() { return R > 0 ? R : (R < 0 ? -R : PP_MAX_R); }

template <int R>
__device__ __forceinline__ int rank_of(const TableArgs &T) { return R > 0 ? R : (int)T.r; }

// The r cells of key x (one per sub-table).
template <int R>
__device__ __forceinline__ void cells_of(u64 x, const TableArgs &t, u32 (&c)[R]) {
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const u64 h = mix64(x ^ t.seed[j]);
    const u64 size = (u64)(t.off[j + 1] - t.off[j]);
    c[j] = t.base + t.off[j] + (u32)__umul64hi(h, size);
  }
}

__device__ __forceinline__ u32 lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ u32 lanemask_lt() {
  u32 m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Warp-aggregated reservation of slots in a counter: every lane with pred gets
// a distinct index.  All 32 lanes must call it.
template <typename T>
__device__ __forceinline__ T warp_reserve(bool pred, T *counter) {
  const u32 mask = __ballot_sync(kFull, pred);
  T base = 0;
  if (mask) {
    const int leader = __ffs(mask) - 1;
    if ((int)lane_id() == leader) base = atomicAdd(counter, (T)__popc(mask));
    base = __shfl_sync(kFull, base, leader);
  }
  return base + (T)__popc(mask & lanemask_lt());
}

// Sum over a block (all threads call it); result valid in thread 0.
template <typename T, int BLOCK>
__device__ __forceinline__ T block_sum(T v, T *scratch /* BLOCK/32 entries */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  if (lane_id() == 0) scratch[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = 0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < BLOCK / 32; ++w) s += scratch[w];
  }
  __syncthreads();
  return s;
}

// L2 eviction-priority policy "evict last" for the whole access (PTX
// createpolicy), and stores that carry a policy: for data written by one
// kernel and read back by the next.
__device__ __forceinline__ u64 l2_evict_last_policy() {
  u64 p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void st_l2_policy(u64 *a, u64 v, u64 pol) {
  asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(a), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_l2_policy(u32 *a, u32 v, u64 pol) {
  asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_l2_policy(u16 *a, u16 v, u64 pol) {
  asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;" ::"l"(a), "h"(v), "l"(pol) : "memory");
}

// Invalidates the 128-byte L2 line at `a` (128-byte aligned) without writing
// it back: for scratch data that no one reads again.
__device__ __forceinline__ void l2_discard(const void *a) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
}

}  // namespace pp
