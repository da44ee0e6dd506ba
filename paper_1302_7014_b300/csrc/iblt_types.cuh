// Types and launch constants shared by the IBLT kernels and their host code.
#pragma once

#include "device.cuh"

namespace pp {

constexpr int kBlock = 256;       // threads per CTA of the staged kernels
constexpr int kScanItems = 4;     // cells per thread per scan chunk
constexpr int kPeelItems = 2;     // frontier entries per thread per peel chunk
constexpr int kFilterItems = 2;   // candidates per thread per filter chunk

// Decode state on the device.  One instance per decode (plain or batched).
struct DecodeCtl {
  u64 *out;             // plain decode: recovered keys (caller's buffer)
  u64 out_cap;          // plain decode: capacity of out
  u64 n_out;            // keys recovered so far (plain decode)
  u64 out_round_start;  // n_out when the current round started
  u64 alive;            // cells with count >= 2 at the start of the current round
  u64 nonempty;         // cells with count != 0 when the decode started
  u64 emptied;          // cells whose count went from 1 to 0 during the decode
  u32 round;            // rounds started so far
  u32 n_front;          // |F_t|: entries of the current frontier
  u32 n_next;           // entries of F_{t+1} written so far
  u32 n_cand;           // candidates pushed during the current round
  u32 flags;            // FLAG_*
  u32 max_rounds;
  u32 more;             // 1 while another round must run
  u32 stats_rounds;     // batch: per-table per-round counter slots
  u32 apply_next;       // binned rounds: next chunk of update records to apply
  u32 pad_;
};

// Per-round device statistics (index t-1 for round t).
struct RoundStats {
  u64 *recovered;  // keys recovered in round t
  u64 *alive;      // cells with count >= 2 at the start of round t
  u32 *front;      // |F_t|
};

// Per-table device counters of a batched decode.
struct BatchCounters {
  u64 *recovered;      // per table: keys recovered (also the output cursor)
  u64 *nonempty;       // per table: non-empty cells at the start
  u64 *emptied;        // per table: cells emptied during the decode
  u32 *rounds;         // per table: last round that recovered a key
  u32 *round_rec;      // per table x stats_rounds: keys recovered per round
  u32 *live;           // per table: entries it has in the frontier being built (or NULL)
};

// A contiguous range of one table's cells or keys.
struct Chunk {
  u32 table;
  u32 begin;  // global cell id (scan) or key index (insert)
  u32 end;
};

// Entry points of one instantiation of the IBLT kernels (plain or batched).
struct IbltKernels {
  const void *insert, *scan, *peel, *filter;
  const void *bin, *apply;           // slab-binned build
  const void *claim, *apply_round;   // binned decode round
  int nr;  // compile-time rank (PP_MAX_R for the generic instance)
};

// The kernel set for rank r (specialised for r = 3 and r = 4).
IbltKernels iblt_kernels(uint32_t r, bool batch);

// Dynamic shared memory of the peel kernel.
size_t peel_smem_bytes(int nr, bool batch);

// Dynamic shared memory of the binning kernel for n_slabs slabs.
size_t bin_smem_bytes(int nr, bool batch, uint32_t n_slabs);

// Dynamic shared memory of the binned round's claim and apply kernels.
size_t claim_smem_bytes(int nr, uint32_t n_bins);
size_t apply_round_smem_bytes(bool batch, uint32_t n_bins);

// The bin-reset kernel that ends a binned round.
const void *bins_reset_kernel();

// The round_end kernel (one thread; records a round and decides on the next).
const void *round_end_kernel();

}  // namespace pp
