// Types and launch constants shared by the IBLT kernels and their host code.
#pragma once

#include "device.cuh"

namespace pp {

constexpr int kBlock = 256;       // threads per CTA of the staged kernels
constexpr int kScanItems = 4;     // cells per thread per scan chunk
constexpr int kPeelItems = 2;     // frontier entries per thread per peel chunk
#ifndef PP_FILTER_ITEMS
#define PP_FILTER_ITEMS 4
#endif
constexpr int kFilterItems = PP_FILTER_ITEMS;  // candidates per thread per filter chunk

// Decode state on the device.  One instance per decode (plain or batched).
struct DecodeCtl {
  u64 *out;             // plain decode: recovered keys (caller's buffer)
  u64 out_cap;          // plain decode: capacity of out
  u64 n_out;            // keys recovered so far (plain decode)
  u64 out_round_start;  // n_out when the current round started
  u64 alive;            // cells with count >= 2 at the start of the current round
  u64 nonempty;         // cells with count != 0 when the decode started
  u64 emptied;          // net count of cells whose count became 0 (1 -> 0 minus 0 -> -1), mod 2^64
  u32 round;            // rounds started so far
  u32 n_front;          // |F_t|: entries of the current frontier
  u32 n_next;           // entries of F_{t+1} written so far
  u32 n_cand;           // candidates pushed during the current round
  u32 flags;            // FLAG_*
  u32 max_rounds;
  u32 more;             // 1 while another round must run
  u32 stats_rounds;     // batch: per-table per-round counter slots
  u32 apply_next;       // binned rounds: next chunk of update records to apply
  u32 n_neg;            // signed decode: keys recovered with sign -1
  u32 n_act;            // tile rounds: sparse tiles with records in the current round
  u32 n_act_dense;      // tile rounds: dense tiles with records in the current round
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
  u64 *emptied;        // per table: net cells emptied (1 -> 0 minus 0 -> -1), mod 2^64
  u32 *rounds;         // per table: last round that recovered a key
  u32 *round_rec;      // per table x stats_rounds: keys recovered per round
  u32 *live;           // per table: entries it has in the frontier being built (or NULL)
  const u64 *chk_seed; // per table: checksum seed (or NULL: read it from TableArgs)
  u64 *residual;       // per table: non-empty cells counted after a binned decode
  const u64 *items;    // per table: keys before the decode (residual scan skips full decodes)
  u32 skip_full;       // 1: tables with every key recovered have no residue to count
  u32 pad;
};

// A contiguous range of one table's cells or keys.
struct Chunk {
  u32 table;
  u32 begin;  // global cell id (scan) or key index (insert)
  u32 end;
};

// Slab-binned build (iblt_binned.cuh).
#ifndef PP_SLAB_SHIFT
#define PP_SLAB_SHIFT 21
#endif
constexpr int kSlabShift = PP_SLAB_SHIFT;    // 2^21 cells = 64 MB per slab
constexpr u32 kSlabCells = 1u << kSlabShift;
#ifndef PP_BIN_ITEMS
#define PP_BIN_ITEMS 4
#endif
#ifndef PP_BIN_CTAS
#define PP_BIN_CTAS 5
#endif
constexpr int kBinItems = PP_BIN_ITEMS;       // keys per thread per partition step
constexpr int kBinKeys = kBlock * kBinItems; // keys per block per partition step

// Record lists of a binned build: slab s owns records [s*cap, s*cap + min(count[s], cap)).
// Tile pass of the binned build (iblt_tiles.cuh): a slab's updates are
// re-sorted into tiles of 2^12 cells, and each tile is updated in shared
// memory and written out whole.
constexpr int kTileShift = 12;
constexpr u32 kTileCells = 1u << kTileShift;               // 4096 cells, 64 KB of shared state
constexpr u32 kTilesPerSlab = kSlabCells >> kTileShift;    // 512
constexpr int kTileThreads = 512;                          // threads per CTA of both tile kernels
constexpr int kTileBinItems = 8;                           // records per thread per chunk
#ifndef PP_TILE_APPLY_ITEMS
#define PP_TILE_APPLY_ITEMS 8
#endif
constexpr int kTileApplyItems = PP_TILE_APPLY_ITEMS;       // records per thread per step of the apply
constexpr int kTileBinChunk = kTileThreads * kTileBinItems;  // 4096 records per bin step

struct TileArgs {
  u64 *key;         // sorted records: two sets, set_stride records apart
  u16 *off;         // each record's cell within its tile
  u32 *tab;         // batch: table of each record
  u32 *count;       // per tile, two sets of kTilesPerSlab (the apply role resets them)
  u64 set_stride;   // kTilesPerSlab * cap
  u32 cap;          // records per tile
  u32 o_cap;        // records per overflow set (a slab's whole record capacity)
  u64 *o_key;       // overflow: three sets, o_cap records apart
  u32 *o_cell;
  u32 *o_tab;
  u32 *o_count;     // per slab
};

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

// Binned decode rounds (iblt_rounds.cuh).
#ifndef PP_ROUND_SHIFT_MIN
#define PP_ROUND_SHIFT_MIN 19
#endif
constexpr int kRoundShiftMin = PP_ROUND_SHIFT_MIN;  // bins hold at least 2^19 cells
constexpr u32 kMaxRoundBins = 128;         // ... and there are at most this many
// Records per thread per grab of k_apply_round (with its resident CTAs per SM,
// pp_options.apply_ctas, it sets the width of the table window being updated).
#ifndef PP_APPLY_PER
#define PP_APPLY_PER 8
#endif
constexpr int kApplyPer = PP_APPLY_PER;
constexpr int kApplyChunk = kBlock * kApplyPer;

// Record lists of one round: bin b owns records [b*cap, b*cap + min(count[b], cap)).
struct RoundBins {
  u64 *rec_key;
  u32 *rec_cell;  // signed decode: bit 31 set for a key removed with sign -1
  u32 *rec_tab;   // batch only
  u32 *count;
  u32 cap;
  u32 n_bins;
  u32 shift;      // bin of cell c = c >> shift
  u32 pad;
  // signed decode only
  const signed char *fsign = nullptr;  // sign of each frontier entry
  signed char *osign = nullptr;        // sign of each recovered key (may be null)
  u64 cand_cap = 0;                    // candidate list capacity
};

// Bin shift for a table (or arena) of n cells: bins of 2^19 cells or more, at
// most kMaxRoundBins of them (few bins keep each block's runs long).
inline u32 round_bin_shift(uint64_t n) {
  u32 sh = kRoundShiftMin;
  while ((n + (1ull << sh) - 1) >> sh > kMaxRoundBins) ++sh;
  return sh;
}

constexpr int kClaimItems = 2;                  // frontier entries per thread per chunk
constexpr int kClaimChunk = kBlock * kClaimItems;

// Tile-pass buffers of one handle (host side; csrc/tiles.cu).
struct TileBufs {
  u64 *key = nullptr, *o_key = nullptr;
  u16 *off = nullptr;
  u32 *tab = nullptr, *count = nullptr;
  u32 *o_cell = nullptr, *o_tab = nullptr, *o_count = nullptr;
  uint64_t cap = 0, o_cap = 0;  // per tile; per overflow set
  uint32_t o_slabs = 0;
  bool batch = false;
};

// Records per tile for a slab list of slab_cap records, and the bytes of the
// tile-pass buffers (pp_workspace_size reports them).
uint64_t tile_cap_for(uint64_t slab_cap);
uint64_t tile_pass_bytes(uint64_t tile_cap, uint64_t o_cap, uint32_t n_slabs, bool batch);

// Grows the buffers to tile_cap records per tile, o_cap per slab's overflow,
// n_slabs overflow counters.
pp_status ensure_tiles(TileBufs &tb, uint64_t tile_cap, uint64_t o_cap, uint32_t n_slabs, bool batch,
                       cudaStream_t s);
void free_tiles(TileBufs &tb);

// Pass 2 of a binned update: every slab of `ba` through k_tile_bin and
// k_tile_apply (zero = build from empty cells), then the last overflow flush.
struct PrescanArgs;  // below
pp_status tile_apply_pass(Cell *cells, const TableArgs &tab0, const TableArgs *tabs, const BinArgs &ba,
                          TileBufs &tb, uint64_t n_cells, int sign, bool zero, cudaStream_t s,
                          const PrescanArgs *pre = nullptr);
// Batched tile pass with the bin role fed from the keys: slab_chunk (device,
// 2 * n_slabs) holds each slab's range of `chunks`; rank as for iblt_kernels.
// Every record of a slab must fit its overflow set (tb.o_cap).  pre (a build
// from empty cells only): the write-out also finds F_1 (PrescanArgs).
pp_status tile_keys_pass(Cell *cells, const TableArgs *tabs, const u64 *keys, const Chunk *chunks,
                         const u32 *slab_chunk, uint32_t n_slabs, int rank, TileBufs &tb, uint64_t n_cells,
                         int sign, bool zero, cudaStream_t s, const PrescanArgs *pre = nullptr);

// A tile with records in the current round: records [lo, lo + n) (absolute slots).
struct TileAct {
  u64 lo;
  u32 tile;
  u32 n;
};

struct TileRoundBufs {
  u64 *rec_key;   // records: the key
  u16 *rec_off;   // records: cell offset in its tile
  u64 *base;      // per tile: first record slot of its region (n_tiles + 1 entries)
  u32 *base64;    // per tile and one past the last: base / kTRAlign (regions start on multiples of kTRAlign)
  u32 *pos;       // per tile (stride kTRPosStride): records written this decode
  u32 *done;      // per tile: records applied this decode
  u32 *sum;       // per tile: sum of counts at the decode's start (scan output)
  TileAct *act;   // sparse tiles with records this round (n_tiles entries)
  TileAct *act_d; // dense tiles with records this round (n_tiles entries)
  u32 *fseg;      // per frontier segment: entries
  const u64 *fstart;  // per frontier segment: first entry in fkey / fcell
  u64 *crec_key;  // coarse records (claim -> k_tsort): the key
  u32 *crec_cell; // coarse records: the cell
  u32 *cpos;      // per coarse bin (stride kTRPosStride): coarse records written this decode
  u32 *cdone;     // per coarse bin: coarse records sorted into tiles this decode
  u64 rec_cap;    // slots in rec_key / rec_off (and crec_key / crec_cell)
  u32 n_bins;     // coarse bins of 2^bin_tshift tiles each
  u32 bin_tshift;
  u32 n_tiles;
  u32 n_seg_d;    // segments of k_tscan / k_tapply blocks (first)
  u32 n_seg_s;    // segments of k_tapply_sparse blocks (after those)
  u32 cap_d;      // entries of a k_tscan / k_tapply segment: 4096 * ceil(n_tiles / n_seg_d)
  u32 cap_s;      // entries of a k_tapply_sparse segment: kTSCap * ceil(n_tiles / n_seg_s)
  u32 pad;
  u32 *rescan;    // tiles the decode must scan itself (a build that found F_1 could not finish them)
  u32 *n_rescan;
};

// A build whose tile pass also finds F_1 (pp_iblt_build_decode): as it writes
// a tile out, the apply role stores the tile's pure cells empty and pushes
// them into the tile's frontier segment (tile % n_seg_d), writes the tile's
// bitmap words and count sum, and adds to the decode's counters.  A tile whose
// cells the overflow pass changes after that write goes to tb.rescan instead.
struct PrescanArgs {
  TileRoundBufs tb;
  u64 *fkey;
  u32 *fcell, *bitmap;
  DecodeCtl *ctl;
  u64 seed_chk;         // the checksum seed (single table)
  const u64 *wseed;     // batch: the checksum seed of each 32-cell word
};

// 32-cell words per 4096-cell tile of the tile rounds (the batch's word maps
// cover whole tiles).
constexpr u32 kTRWordsPerTile = 128;

// The tables of a batched tile-round decode: one arena of 32-cell-aligned
// tables, so that every 32-cell word of it belongs to one table.  All zero in
// a single-table decode.
struct TRBatch {
  const TableArgs *tabs;  // per table
  const u32 *wtab;        // per 32-cell word of the arena: its table
  const u64 *wseed;       // per 32-cell word: its table's checksum seed
  BatchCounters bc;       // per-table output cursors and statistics
  u64 *out;               // recovered keys (table i writes [out_base, out_base + out_cap))
};

// Entry points of one instantiation of the IBLT kernels (plain or batched).
struct IbltKernels {
  const void *insert, *scan, *peel, *filter;
  const void *bin;                   // slab-binned build (pass 1)
  const void *claim, *apply_round;   // binned decode round
  int nr;  // compile-time rank (PP_MAX_R for the generic instance)
  const void *sub_scan = nullptr, *sub_filter = nullptr, *sub_peel = nullptr;  // sub-rounds (plain only)
  const void *sub_claim = nullptr;  // binned sub-rounds: k_claim without the claim check
  const void *sg_scan = nullptr, *sg_peel = nullptr, *sg_filter = nullptr;     // signed (plain only)
  const void *sg_claim = nullptr, *sg_apply = nullptr;                         // signed, binned rounds
  const void *tscan = nullptr, *tclaim = nullptr, *tapply = nullptr;           // tile rounds (plain only)
  const void *tapply_sparse = nullptr, *trestore = nullptr;
  const void *trescan = nullptr;  // tile rounds after a build that found F_1
};

// The kernel set for a rank code: 3 or 4 = that r; -4 = any r <= 4 (batched
// kernels only); 0 = any r up to PP_MAX_R.
IbltKernels iblt_kernels(int rank, bool batch);

// Host side of the tile rounds (csrc/iblt.cu), shared by the single-table
// handle and the batch: the per-tile and per-bin buffers, the frontier
// segments, the grids of the round kernels.
struct TileRoundEngine {
  TileRoundBufs trb{};
  int grid_tscan = 0, grid_tclaim = 0, grid_tapply = 0, grid_tsparse = 0, grid_tsort = 0, grid_act = 0;
  size_t smem_tclaim = 0, smem_tsort = 0;
  uint64_t front = 0;  // frontier entries the segments span (fkey / fcell must hold them)
};

// Sizes the segments, coarse bins and grids for a table (or arena) of n_cells
// and allocates the per-tile buffers; nothing to do once set up.
pp_status tre_setup(TileRoundEngine &e, const IbltKernels &k, uint64_t n_cells, uint32_t ctas_per_sm);
// Grows the record buffers to `need` records; *moved tells that they were
// reallocated (graphs that hold them must be rebuilt).
pp_status tre_records(TileRoundEngine &e, uint64_t need, cudaStream_t s, bool *moved);
void tre_free(TileRoundEngine &e);
// Record slots for a decode of `updates` cell updates (r per key): the updates
// plus the alignment slack of every tile's region.
uint64_t tre_record_need(const TileRoundEngine &e, uint64_t updates);

// Arguments of one tile-round decode.  tab0: the table (single) or, in a
// batch, any TableArgs whose n_cells is the arena's size; bt: zero for a
// single table.  Kernel parameter arrays point into this object.
struct TileRoundLaunch {
  Cell *cells;
  TableArgs tab0;
  u64 *fkey;
  u32 *fcell, *bitmap;
  const u64 *fkey_c;
  const u32 *fcell_c, *bitmap_c;
  TileRoundBufs tb;
  DecodeCtl *ctl;
  TRBatch bt;
  RoundStats st;
  int set_cond;
  cudaGraphConditionalHandle cond;
  void *scan[8], *prefix[2], *claim[8], *active[2], *apply[8], *sort[2], *restore[7], *end[4];
  void bind();
};
void tre_launch_args(TileRoundLaunch &a, const TileRoundEngine &e, Cell *cells, const TableArgs &tab0, u64 *fkey,
                     u32 *fcell, u32 *bitmap, DecodeCtl *ctl, const RoundStats &st, const TRBatch &bt);
// The decode as a CUDA graph: scan, prefix, a while node over the round
// kernels, restore.
pp_status tre_build_graph(const TileRoundEngine &e, const IbltKernels &k, TileRoundLaunch &a, cudaGraphExec_t *exec,
                          bool prescanned = false);
// The same kernels driven from the host (one synchronisation per round);
// h_more: pinned copy of ctl->more.  prescanned: the build found F_1, so the
// decode starts with k_trescan (the tiles the build could not finish) instead
// of the full scan.
pp_status tre_host_loop(const TileRoundEngine &e, const IbltKernels &k, TileRoundLaunch &a, u32 *h_more,
                        cudaStream_t s, bool prescanned = false);

// Dynamic shared memory of the peel kernel.
size_t peel_smem_bytes(int nr, bool batch);

// Dynamic shared memory of the binning kernel for n_slabs slabs.
size_t bin_smem_bytes(int nr, bool batch, uint32_t n_slabs);

// Dynamic shared memory of the binned round's claim and apply kernels.
size_t claim_smem_bytes(int nr, bool batch, uint32_t n_bins, bool sgn = false);
size_t apply_round_smem_bytes(bool batch, uint32_t n_bins);

// The bin-reset kernel that ends a binned round.
const void *bins_reset_kernel();

// The residue counter of batched binned decodes (k_residual).
const void *residual_kernel();

// The round_end kernel (one thread; records a round and decides on the next).
const void *round_end_kernel();

}  // namespace pp
