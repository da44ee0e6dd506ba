// C-ABI: many IBLTs decoded together (batched form of the round-synchronous
// decode).
//
// All tables live in one device arena (table i starts at a 32-cell-aligned
// global cell id) and share one frontier.  A decode is one CUDA graph launch:
// the full scan covers every table, then each device-side round peels the
// current frontier entries of all tables at once.  Tables never share cells,
// so each table's rounds, recovered keys and residue are exactly those of a
// plain decode of that table alone; a table whose frontier empties simply
// stops contributing entries.  Per-table counters record keys recovered per
// round (the first stats_rounds rounds), the last productive round, and the
// residue size.
//
// A batch built from insertions only decodes in tile rounds over the whole
// arena (csrc/iblt_trounds.cuh): the rounds' updates are folded per 4096-cell
// tile whatever tables the tile's cells belong to.  A per-word table map
// (every 32-cell word belongs to one table) gives the kernels a cell's table
// and checksum seed.  Other batches use the binned or direct-atomic rounds.
#include <string.h>

#include <vector>

#include "host.cuh"
#include "iblt_types.cuh"

using namespace pp;

namespace {

constexpr u32 kScanChunk = kBlock * kScanItems;

}  // namespace

struct pp_batch {
  uint32_t n_tables = 0;
  uint32_t rank = 0;          // 0 = mixed r (generic kernels), else the common r
  uint64_t total_cells = 0;   // arena size (cells), including alignment padding
  pp_options opt{};
  std::vector<TableArgs> h_tabs;
  std::vector<uint64_t> items;  // keys per table (inserted - deleted)
  TableArgs *tabs = nullptr;
  Cell *cells = nullptr;
  u64 *fkey = nullptr;
  u32 *fcell = nullptr, *ftab = nullptr, *cand = nullptr, *ctab = nullptr, *bitmap = nullptr;
  Chunk *scan_chunks = nullptr;
  u32 n_scan_chunks = 0;
  Chunk *ins_chunks = nullptr;
  u32 ins_chunk_cap = 0;
  Chunk *h_ins_chunks = nullptr;  // pinned staging
  DecodeCtl *ctl = nullptr, *h_ctl = nullptr;
  u64 *st_rec = nullptr, *st_alive = nullptr;
  u32 *st_front = nullptr;
  BatchCounters bc{};
  // pinned copies of the per-table counters
  u64 *h_recovered = nullptr, *h_nonempty = nullptr, *h_emptied = nullptr;
  u32 *h_rounds = nullptr, *h_round_rec = nullptr;
  IbltKernels k{};
  int grid_scan = 0, grid_peel = 0, grid_filter = 0, grid_insert = 0;
  size_t smem_peel = 0;
  cudaGraphExec_t exec = nullptr;
  u64 *graph_out = nullptr;  // output buffer the instantiated graph writes to
  cudaGraphExec_t exec_pre = nullptr;  // tile rounds after a build that found F_1
  u64 *graph_out_pre = nullptr;
  uint32_t graph_gen_pre = 0;
  // update records shared by the slab-binned build and the binned rounds
  u64 *rec_key = nullptr;
  u32 *rec_cell = nullptr, *rec_tab = nullptr, *bin_count = nullptr, *bin_overflow = nullptr;
  uint64_t rec_cap_total = 0;
  uint32_t count_cap = 0, rec_gen = 0, graph_gen = 0;
  uint32_t max_r = 0;
  bool binned_rounds = false;
  bool had_deletes = false;   // since the last clear/build
  u64 *h_items = nullptr;     // pinned copy of items[] for upload
  u64 *h_residual = nullptr;
  uint32_t n_bins = 0, bin_cap = 0, n_slabs = 0, bin_shift = 0;
  size_t smem_claim = 0, smem_apply_round = 0, smem_bin = 0;
  int grid_claim = 0, grid_apply_round = 0, grid_bin = 0;
  TileBufs tiles;  // tile pass of the binned build (allocated on first use)
  // tile rounds (allocated on the first decode that uses them)
  TileRoundEngine tre;
  u32 *wtab = nullptr;        // per 32-cell word of the arena: its table
  u64 *wseed = nullptr;       // per word: its table's checksum seed
  uint64_t front_cap = 0;     // entries of fkey / fcell
  bool tile_rounds = false;   // the round kind the graph was built with
  // binned updates fed from the keys (every table lies within two slabs)
  bool keys_tiles = false;
  int krank = 0;                 // kernel rank, as passed to iblt_kernels
  u32 *slab_chunk = nullptr, *h_slab_chunk = nullptr;
  uint32_t slab_chunk_cap = 0;   // slabs
};

namespace {

void free_batch(pp_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->exec_pre) cudaGraphExecDestroy(b->exec_pre);
  cudaFree(b->tabs);
  cudaFree(b->cells);
  cudaFree(b->fkey);
  cudaFree(b->fcell);
  cudaFree(b->ftab);
  cudaFree(b->cand);
  cudaFree(b->ctab);
  cudaFree(b->bitmap);
  cudaFree(b->scan_chunks);
  cudaFree(b->ins_chunks);
  cudaFreeHost(b->h_ins_chunks);
  cudaFree(b->ctl);
  cudaFreeHost(b->h_ctl);
  cudaFree(b->st_rec);
  cudaFree(b->st_alive);
  cudaFree(b->st_front);
  cudaFree(b->bc.recovered);
  cudaFree(b->bc.nonempty);
  cudaFree(b->bc.emptied);
  cudaFree(b->bc.rounds);
  cudaFree(b->bc.round_rec);
  cudaFree((void *)b->bc.chk_seed);
  cudaFree(b->bc.residual);
  cudaFree((void *)b->bc.items);
  cudaFreeHost(b->h_items);
  cudaFreeHost(b->h_residual);
  cudaFreeHost(b->h_recovered);
  cudaFreeHost(b->h_nonempty);
  cudaFreeHost(b->h_emptied);
  cudaFreeHost(b->h_rounds);
  cudaFreeHost(b->h_round_rec);
  cudaFree(b->rec_key);
  cudaFree(b->rec_cell);
  cudaFree(b->rec_tab);
  cudaFree(b->bin_count);
  cudaFree(b->bin_overflow);
  free_tiles(b->tiles);
  tre_free(b->tre);
  cudaFree(b->wtab);
  cudaFree(b->wseed);
  cudaFree(b->slab_chunk);
  cudaFreeHost(b->h_slab_chunk);
  delete b;
}

pp_status ensure_records(pp_batch *b, uint64_t records, uint32_t counts, cudaStream_t s) {
  if (records > b->rec_cap_total) {
    PP_CUDA(cudaStreamSynchronize(s));
    cudaFree(b->rec_key);
    cudaFree(b->rec_cell);
    cudaFree(b->rec_tab);
    b->rec_key = nullptr;
    b->rec_cell = nullptr;
    b->rec_tab = nullptr;
    b->rec_cap_total = 0;
    PP_CUDA(cudaMalloc((void **)&b->rec_key, records * sizeof(u64)));
    PP_CUDA(cudaMalloc((void **)&b->rec_cell, records * sizeof(u32)));
    PP_CUDA(cudaMalloc((void **)&b->rec_tab, records * sizeof(u32)));
    b->rec_cap_total = records;
    ++b->rec_gen;
  }
  if (counts > b->count_cap || !b->bin_overflow) {
    PP_CUDA(cudaStreamSynchronize(s));
    cudaFree(b->bin_count);
    cudaFree(b->bin_overflow);
    b->bin_count = nullptr;
    b->bin_overflow = nullptr;
    PP_CUDA(cudaMalloc((void **)&b->bin_count, (counts ? counts : 1) * sizeof(u32)));
    PP_CUDA(cudaMalloc((void **)&b->bin_overflow, sizeof(u32)));
    b->count_cap = counts;
    ++b->rec_gen;
  }
  return PP_OK;
}

bool use_binned(const pp_batch *b, uint64_t records) {
  if (records == 0 || b->opt.binned == 2) return false;
  if (b->opt.binned == 1) return true;
  return b->total_cells >= (1ull << 23) && records >= b->total_cells / 4;
}

// Bins of the binned rounds over the whole arena (2^19 cells each).  A bin's
// list holds the updates of 0.35 keys per cell at the largest r in the batch;
// fuller bins apply their excess directly.
// Round kind: tile rounds for batches built from insertions only (forced on
// or off by opt.rounds), for arenas of 2^21 cells or more by default.
bool batch_wants_tiles(const pp_batch *b) {
  const bool large = b->total_cells >= (1ull << 21);
  return b->k.tscan && !b->had_deletes &&
         (b->opt.rounds == 2 || (b->opt.rounds == 0 && large && b->opt.binned != 2));
}

pp_status ensure_round_bins(pp_batch *b, cudaStream_t s) {
  const u32 shift = round_bin_shift(b->total_cells);
  const uint32_t nb = (uint32_t)((b->total_cells + (1ull << shift) - 1) >> shift);
  const uint64_t span = b->total_cells < (1ull << shift) ? b->total_cells : (1ull << shift);
  const uint64_t cap = (uint64_t)((double)b->max_r * (double)span * 0.35) + 4096;
  pp_status st = ensure_records(b, cap * nb, nb, s);
  if (st != PP_OK) return st;
  b->n_bins = nb;
  b->bin_cap = (uint32_t)cap;
  b->bin_shift = shift;
  b->smem_claim = claim_smem_bytes(b->k.nr, true, nb);
  b->smem_apply_round = apply_round_smem_bytes(true, nb);
  b->grid_claim = persistent_grid(b->k.claim, kBlock, b->smem_claim, b->opt.ctas_per_sm);
  b->grid_apply_round = persistent_grid(b->k.apply_round, kBlock, b->smem_apply_round, b->opt.apply_ctas);
  return PP_OK;
}

// Tile rounds over the arena: the engine's buffers, frontier arrays that span
// its segments, the word maps, and record regions for every key's updates
// (r keys per table plus kTRAlign slack per tile).
pp_status ensure_batch_tiles(pp_batch *b, cudaStream_t s) {
  if (!b->tre.trb.base) {
    pp_status st = tre_setup(b->tre, b->k, b->total_cells, b->opt.ctas_per_sm);
    if (st != PP_OK) return st;
    ++b->rec_gen;
    PP_CUDA(cudaStreamSynchronize(s));
    if (b->tre.front > b->front_cap) {
      cudaFree(b->fkey);
      cudaFree(b->fcell);
      b->fkey = nullptr;
      b->fcell = nullptr;
      PP_CUDA(cudaMalloc((void **)&b->fkey, b->tre.front * sizeof(u64)));
      PP_CUDA(cudaMalloc((void **)&b->fcell, b->tre.front * sizeof(u32)));
      b->front_cap = b->tre.front;
      if (b->exec) cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    // every word of table i (its padding included) maps to i
    const uint64_t nw = (uint64_t)b->tre.trb.n_tiles * kTRWordsPerTile;
    std::vector<u32> wt(nw, 0);
    std::vector<u64> ws(nw, 0);
    for (uint32_t i = 0; i < b->n_tables; ++i) {
      const TableArgs &t = b->h_tabs[i];
      const u64 seed = t.seed[t.r];
      for (uint64_t w = t.base / 32; w < ((uint64_t)t.base + t.n_cells + 31) / 32; ++w) {
        wt[w] = i;
        ws[w] = seed;
      }
    }
    PP_CUDA(cudaMalloc((void **)&b->wtab, nw * sizeof(u32)));
    PP_CUDA(cudaMalloc((void **)&b->wseed, nw * sizeof(u64)));
    PP_CUDA(cudaMemcpy(b->wtab, wt.data(), nw * sizeof(u32), cudaMemcpyHostToDevice));
    PP_CUDA(cudaMemcpy(b->wseed, ws.data(), nw * sizeof(u64), cudaMemcpyHostToDevice));
  }
  uint64_t updates = 0;
  for (uint32_t i = 0; i < b->n_tables; ++i) updates += (uint64_t)b->h_tabs[i].r * b->items[i];
  bool moved = false;
  pp_status st = tre_records(b->tre, tre_record_need(b->tre, updates), s, &moved);
  if (moved) ++b->rec_gen;
  return st;
}

struct BatchArgs {
  // scan
  Cell *cells;
  TableArgs tab0;
  const TableArgs *tabs;
  const Chunk *chunks;
  u32 n_chunks;
  u64 *fkey;
  u32 *fcell, *ftab, *bitmap;
  DecodeCtl *ctl;
  BatchCounters bc;
  // peel
  const u64 *fkey_c;
  const u32 *fcell_c, *ftab_c, *bitmap_c;
  u32 *cand, *ctab;
  u64 *bout;
  // filter
  const Cell *cells_c;
  const u32 *cand_c, *ctab_c;
  // round end
  RoundStats st;
  int set_cond;
  cudaGraphConditionalHandle cond;
  // binned rounds
  RoundBins rb;
  void *scan_p[11], *peel_p[12], *filter_p[11], *end_p[4], *claim_p[13], *applyr_p[8], *reset_p[2];
  void bind() {
    void *s[11] = {&cells, &tab0, &tabs, &chunks, &n_chunks, &fkey, &fcell, &ftab, &bitmap, &ctl, &bc};
    void *p[12] = {&cells, &tab0, &tabs, &fkey_c, &fcell_c, &ftab_c, &bitmap_c, &cand, &ctab, &bout, &ctl, &bc};
    void *f[11] = {&cells_c, &tab0, &tabs, &cand_c, &ctab_c, &fkey, &fcell, &ftab, &bitmap, &ctl, &bc};
    void *e[4] = {&ctl, &st, &set_cond, &cond};
    memcpy(scan_p, s, sizeof s);
    memcpy(peel_p, p, sizeof p);
    memcpy(filter_p, f, sizeof f);
    memcpy(end_p, e, sizeof e);
    void *c[13] = {&cells, &tab0, &tabs, &fkey_c, &fcell_c, &ftab_c, &bitmap_c, &rb, &cand, &ctab, &bout, &ctl, &bc};
    void *a[8] = {&cells, &tab0, &tabs, &rb, &cand, &ctab, &ctl, &bc};
    void *z[2] = {&rb, &ctl};
    memcpy(claim_p, c, sizeof c);
    memcpy(applyr_p, a, sizeof a);
    memcpy(reset_p, z, sizeof z);
  }
};

void fill(pp_batch *b, BatchArgs &a, u64 *out) {
  memset(&a, 0, sizeof a);
  a.cells = b->cells;
  a.tabs = b->tabs;
  a.chunks = b->scan_chunks;
  a.n_chunks = b->n_scan_chunks;
  a.fkey = b->fkey;
  a.fcell = b->fcell;
  a.ftab = b->ftab;
  a.bitmap = b->bitmap;
  a.ctl = b->ctl;
  a.bc = b->bc;
  a.fkey_c = b->fkey;
  a.fcell_c = b->fcell;
  a.ftab_c = b->ftab;
  a.bitmap_c = b->bitmap;
  a.cand = b->cand;
  a.ctab = b->ctab;
  a.bout = out;
  a.cells_c = b->cells;
  a.cand_c = b->cand;
  a.ctab_c = b->ctab;
  a.st = RoundStats{b->st_rec, b->st_alive, b->st_front};
  a.rb = RoundBins{b->rec_key, b->rec_cell, b->rec_tab, b->bin_count, b->bin_cap, b->n_bins, b->bin_shift, 0};
  a.bind();
}

pp_status add_kernel(cudaGraphNode_t *node, cudaGraph_t g, const cudaGraphNode_t *dep, size_t ndep,
                     const void *fn, int grid, int block, size_t smem, void **args) {
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void *>(fn);
  kp.gridDim = dim3((unsigned)grid);
  kp.blockDim = dim3((unsigned)block);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = args;
  PP_CUDA(cudaGraphAddKernelNode(node, g, dep, ndep, &kp));
  return PP_OK;
}

void fill_tiles(pp_batch *b, TileRoundLaunch &a, u64 *out) {
  TableArgs t0{};
  t0.n_cells = (u32)b->total_cells;  // the tile kernels' bound; tables come from the word map
  const TRBatch bt{b->tabs, b->wtab, b->wseed, b->bc, out};
  tre_launch_args(a, b->tre, b->cells, t0, b->fkey, b->fcell, b->bitmap, b->ctl,
                  RoundStats{b->st_rec, b->st_alive, b->st_front}, bt);
}

// The output pointer is a kernel argument, so the graph is rebuilt when it
// changes (the caller usually decodes into the same buffer every time).
pp_status build_graph(pp_batch *b, u64 *out) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  BatchArgs a;
  fill(b, a, out);
  cudaGraph_t g = nullptr;
  PP_CUDA(cudaGraphCreate(&g, 0));
  pp_status st = PP_OK;
  cudaGraphNode_t n_scan, n_cond, n_peel, n_filter, n_end;
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams cp{};
  cudaGraph_t body;
  st = add_kernel(&n_scan, g, nullptr, 0, b->k.scan, b->grid_scan, kBlock, 0, a.scan_p);
  if (st != PP_OK) goto done;
  if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    st = fail(PP_ERR_CUDA, "cudaGraphConditionalHandleCreate failed");
    goto done;
  }
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (cudaGraphAddNode(&n_cond, g, &n_scan, nullptr, 1, &cp) != cudaSuccess) {
    st = fail(PP_ERR_CUDA, "cudaGraphAddNode(conditional while) failed");
    goto done;
  }
  body = cp.conditional.phGraph_out[0];
  a.set_cond = 1;
  a.cond = h;
  if (b->binned_rounds) {
    cudaGraphNode_t n_apply, n_reset;
    st = add_kernel(&n_peel, body, nullptr, 0, b->k.claim, b->grid_claim, kBlock, b->smem_claim, a.claim_p);
    if (st != PP_OK) goto done;
    st = add_kernel(&n_apply, body, &n_peel, 1, b->k.apply_round, b->grid_apply_round, kBlock,
                    b->smem_apply_round, a.applyr_p);
    if (st != PP_OK) goto done;
    st = add_kernel(&n_filter, body, &n_apply, 1, b->k.filter, b->grid_filter, kBlock, 0, a.filter_p);
    if (st != PP_OK) goto done;
    st = add_kernel(&n_reset, body, &n_filter, 1, bins_reset_kernel(), 1, 256, 0, a.reset_p);
    if (st != PP_OK) goto done;
    st = add_kernel(&n_end, body, &n_reset, 1, round_end_kernel(), 1, 32, 0, a.end_p);
    if (st != PP_OK) goto done;
  } else {
    st = add_kernel(&n_peel, body, nullptr, 0, b->k.peel, b->grid_peel, kBlock, b->smem_peel, a.peel_p);
    if (st != PP_OK) goto done;
    st = add_kernel(&n_filter, body, &n_peel, 1, b->k.filter, b->grid_filter, kBlock, 0, a.filter_p);
    if (st != PP_OK) goto done;
    st = add_kernel(&n_end, body, &n_filter, 1, round_end_kernel(), 1, 32, 0, a.end_p);
    if (st != PP_OK) goto done;
  }
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    st = fail(PP_ERR_CUDA, "cudaGraphInstantiate failed");
    b->exec = nullptr;
  }
  b->graph_gen = b->rec_gen;
done:
  cudaGraphDestroy(g);
  return st;
}

}  // namespace

extern "C" {

pp_status pp_batch_create(pp_batch **out, uint32_t n_tables, const uint64_t *n_cells,
                          const uint32_t *r, const uint64_t *seeds, const pp_options *opt) {
  if (!out) return fail(PP_ERR_INVALID_ARG, "pp_batch_create: out is NULL");
  *out = nullptr;
  if (n_tables == 0 || !n_cells || !r || !seeds)
    return fail(PP_ERR_INVALID_ARG, "pp_batch_create: empty batch or NULL arrays");
  pp_batch *b = new pp_batch();
  b->n_tables = n_tables;
  b->opt = resolve_options(opt);
  // scattered 32-byte cell reads: one sector fetched from DRAM, not two
  if (b->opt.l2_fetch == 1) cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, 32);
  b->h_tabs.resize(n_tables);
  b->items.assign(n_tables, 0);
  uint64_t base = 0;
  uint32_t common_r = r[0];
  std::vector<Chunk> chunks;
  for (uint32_t i = 0; i < n_tables; ++i) {
    if (r[i] < 2 || r[i] > PP_MAX_R || n_cells[i] < r[i] || n_cells[i] > 0xFFFFFFFFull) {
      free_batch(b);
      return fail(PP_ERR_INVALID_ARG, "pp_batch_create: table %u has r=%u, n_cells=%llu", i, r[i],
                  (unsigned long long)n_cells[i]);
    }
    if (r[i] != common_r) common_r = 0;
    if (base + n_cells[i] > 0xFFFFFFFFull - 64) {
      free_batch(b);
      return fail(PP_ERR_INVALID_ARG, "pp_batch_create: more than 2^32-64 cells in total");
    }
    make_table_args(b->h_tabs[i], n_cells[i], r[i], seeds[i], (uint32_t)base);
    for (uint64_t c = 0; c < n_cells[i]; c += kScanChunk) {
      const uint64_t e = c + kScanChunk < n_cells[i] ? c + kScanChunk : n_cells[i];
      chunks.push_back(Chunk{i, (u32)(base + c), (u32)(base + e)});
    }
    base += (n_cells[i] + 31) & ~31ull;
  }
  b->rank = common_r;
  b->total_cells = base;
  b->n_scan_chunks = (u32)chunks.size();
  uint32_t max_r = 0;
  for (uint32_t i = 0; i < n_tables; ++i) max_r = r[i] > max_r ? r[i] : max_r;
  b->krank = common_r ? (int)common_r : (max_r <= 4 ? -4 : 0);
  b->k = iblt_kernels(b->krank, true);
  b->keys_tiles = true;
  for (uint32_t i = 0; i < n_tables; ++i)
    if (n_cells[i] > kSlabCells) b->keys_tiles = false;
  b->smem_peel = peel_smem_bytes(b->k.nr, true);
  const uint64_t N = base;
  const uint32_t mr = b->opt.max_rounds;
  const uint32_t sr = b->opt.stats_rounds;
  b->ins_chunk_cap = 1024;
  cudaError_t e = cudaSuccess;
  auto al = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes ? bytes : 16);
  };
  al((void **)&b->tabs, n_tables * sizeof(TableArgs));
  al((void **)&b->cells, N * sizeof(Cell));
  al((void **)&b->fkey, N * sizeof(u64));
  al((void **)&b->fcell, N * sizeof(u32));
  al((void **)&b->ftab, N * sizeof(u32));
  al((void **)&b->cand, N * sizeof(u32));
  al((void **)&b->ctab, N * sizeof(u32));
  al((void **)&b->bitmap, (N / 32 + 1) * sizeof(u32));
  al((void **)&b->scan_chunks, chunks.size() * sizeof(Chunk));
  al((void **)&b->ins_chunks, b->ins_chunk_cap * sizeof(Chunk));
  al((void **)&b->ctl, sizeof(DecodeCtl));
  al((void **)&b->st_rec, (size_t)mr * sizeof(u64));
  al((void **)&b->st_alive, (size_t)mr * sizeof(u64));
  al((void **)&b->st_front, (size_t)mr * sizeof(u32));
  al((void **)&b->bc.recovered, n_tables * sizeof(u64));
  al((void **)&b->bc.nonempty, n_tables * sizeof(u64));
  al((void **)&b->bc.emptied, n_tables * sizeof(u64));
  al((void **)&b->bc.rounds, n_tables * sizeof(u32));
  al((void **)&b->bc.round_rec, (size_t)n_tables * sr * sizeof(u32));
  al((void **)&b->bc.chk_seed, n_tables * sizeof(u64));
  al((void **)&b->bc.residual, n_tables * sizeof(u64));
  al((void **)&b->bc.items, n_tables * sizeof(u64));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_ctl, sizeof(DecodeCtl));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_ins_chunks, b->ins_chunk_cap * sizeof(Chunk));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_recovered, n_tables * sizeof(u64));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_nonempty, n_tables * sizeof(u64));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_emptied, n_tables * sizeof(u64));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_rounds, n_tables * sizeof(u32));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_round_rec, (size_t)n_tables * sr * sizeof(u32));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_items, n_tables * sizeof(u64));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_residual, n_tables * sizeof(u64));
  if (e == cudaSuccess) {
    std::vector<u64> cs(n_tables);
    for (uint32_t i = 0; i < n_tables; ++i) cs[i] = b->h_tabs[i].seed[b->h_tabs[i].r];
    e = cudaMemcpy((void *)b->bc.chk_seed, cs.data(), n_tables * sizeof(u64), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemcpy(b->tabs, b->h_tabs.data(), n_tables * sizeof(TableArgs), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->scan_chunks, chunks.data(), chunks.size() * sizeof(Chunk), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->cells, 0, N * sizeof(Cell));
  if (e == cudaSuccess) e = cudaMemset(b->bitmap, 0, (N / 32 + 1) * sizeof(u32));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    pp_status st = cuda_fail(e, "pp_batch_create allocation", __FILE__, __LINE__);
    free_batch(b);
    return st;
  }
  b->grid_scan = persistent_grid(b->k.scan, kBlock, 0, b->opt.ctas_per_sm);
  b->grid_peel = persistent_grid(b->k.peel, kBlock, b->smem_peel, b->opt.ctas_per_sm);
  b->grid_filter = persistent_grid(b->k.filter, kBlock, 0, b->opt.ctas_per_sm);
  b->grid_insert = persistent_grid(b->k.insert, kBlock, 0, 8) * 2;
  b->max_r = max_r;
  b->front_cap = N;
  *out = b;
  return PP_OK;
}

pp_status pp_batch_destroy(pp_batch *b) {
  if (!b) return PP_OK;
  cudaDeviceSynchronize();
  free_batch(b);
  return PP_OK;
}

pp_status pp_batch_clear(pp_batch *b, void *stream) {
  if (!b) return fail(PP_ERR_INVALID_ARG, "pp_batch_clear: NULL batch");
  PP_CUDA(cudaMemsetAsync(b->cells, 0, b->total_cells * sizeof(Cell), as_stream(stream)));
  for (auto &x : b->items) x = 0;
  b->had_deletes = false;
  return PP_OK;
}

// Uploads the insert work list (key ranges of at most opt.insert_chunk keys, one table each).
static pp_status upload_chunks(pp_batch *b, const uint64_t *h_key_offsets, cudaStream_t s, u32 *n_chunks,
                               uint64_t *records) {
  std::vector<Chunk> chunks;
  uint64_t rec = 0;
  for (uint32_t i = 0; i < b->n_tables; ++i) {
    const uint64_t k0 = h_key_offsets[i], k1 = h_key_offsets[i + 1];
    if (k1 < k0) return fail(PP_ERR_INVALID_ARG, "pp_batch_insert: key offsets decrease at table %u", i);
    if (k1 > 0xFFFFFFFFull) return fail(PP_ERR_INVALID_ARG, "pp_batch_insert: more than 2^32 keys");
    const uint64_t ck = b->opt.insert_chunk;
    for (uint64_t k = k0; k < k1; k += ck)
      chunks.push_back(Chunk{i, (u32)k, (u32)(k + ck < k1 ? k + ck : k1)});
    rec += (k1 - k0) * b->h_tabs[i].r;
  }
  *n_chunks = (u32)chunks.size();
  *records = rec;
  if (chunks.empty()) return PP_OK;
  if (chunks.size() > b->ins_chunk_cap) {
    PP_CUDA(cudaStreamSynchronize(s));
    cudaFree(b->ins_chunks);
    cudaFreeHost(b->h_ins_chunks);
    b->ins_chunks = nullptr;
    b->h_ins_chunks = nullptr;
    b->ins_chunk_cap = (u32)chunks.size();
    PP_CUDA(cudaMalloc((void **)&b->ins_chunks, b->ins_chunk_cap * sizeof(Chunk)));
    PP_CUDA(cudaMallocHost((void **)&b->h_ins_chunks, b->ins_chunk_cap * sizeof(Chunk)));
  } else {
    // the pinned staging buffer may still feed a previous copy
    PP_CUDA(cudaStreamSynchronize(s));
  }
  memcpy(b->h_ins_chunks, chunks.data(), chunks.size() * sizeof(Chunk));
  PP_CUDA(cudaMemcpyAsync(b->ins_chunks, b->h_ins_chunks, chunks.size() * sizeof(Chunk),
                          cudaMemcpyHostToDevice, s));
  return PP_OK;
}

static pp_status direct_update(pp_batch *b, const uint64_t *d_keys, u32 nch, int sign, cudaStream_t s) {
  Cell *cells = b->cells;
  TableArgs t0{};
  const TableArgs *tabs = b->tabs;
  const Chunk *ch = b->ins_chunks;
  const u64 *keys = reinterpret_cast<const u64 *>(d_keys);
  u64 m = 0;
  void *args[] = {&cells, &t0, &tabs, &ch, &nch, &keys, &m, &sign};
  const int grid = nch < (u32)b->grid_insert ? (int)nch : b->grid_insert;
  PP_CUDA(cudaLaunchKernel(b->k.insert, dim3(grid), dim3(kBlock), args, 0, s));
  return PP_OK;
}

// Pass 1 of a binned batch update: every (cell, key) update into its slab's
// list.  Tables differ in load and r, so each slab's expected share is summed
// from the tables it overlaps.
static pp_status batch_bin_pass(pp_batch *b, const uint64_t *d_keys, const uint64_t *h_key_offsets, u32 nch,
                                int sign, int direct_overflow, cudaStream_t s, BinArgs &ba) {
  const uint32_t ns = (uint32_t)((b->total_cells + kSlabCells - 1) / kSlabCells);
  std::vector<double> expect(ns, 0.0);
  for (uint32_t i = 0; i < b->n_tables; ++i) {
    const TableArgs &t = b->h_tabs[i];
    const double rec = (double)(h_key_offsets[i + 1] - h_key_offsets[i]) * t.r;
    if (rec == 0) continue;
    const uint64_t c0 = t.base, c1 = (uint64_t)t.base + t.n_cells;
    for (uint64_t sl = c0 / kSlabCells; sl * kSlabCells < c1; ++sl) {
      const uint64_t a0 = sl * kSlabCells > c0 ? sl * kSlabCells : c0;
      const uint64_t a1 = (sl + 1) * kSlabCells < c1 ? (sl + 1) * kSlabCells : c1;
      expect[sl] += rec * (double)(a1 - a0) / (double)t.n_cells;
    }
  }
  double mx = 0;
  for (double e : expect) mx = e > mx ? e : mx;
  const uint64_t cap = (uint64_t)(mx * 1.05) + 4096;
  if (cap > 0xFFFFFFF0ull) return fail(PP_ERR_INVALID_ARG, "pp_batch_insert: too many keys for one call");
  pp_status st = ensure_records(b, cap * ns, ns, s);
  if (st != PP_OK) return st;
  if (ns != b->n_slabs) {
    b->n_slabs = ns;
    b->smem_bin = bin_smem_bytes(b->k.nr, true, ns);
    b->grid_bin = persistent_grid(b->k.bin, kBlock, b->smem_bin, b->opt.ctas_per_sm);
  }
  PP_CUDA(cudaMemsetAsync(b->bin_count, 0, ns * sizeof(u32), s));
  PP_CUDA(cudaMemsetAsync(b->bin_overflow, 0, sizeof(u32), s));
  ba = BinArgs{b->rec_key, b->rec_cell, b->rec_tab, b->bin_count, b->bin_overflow, (u32)cap, ns, direct_overflow};
  Cell *cells = b->cells;
  TableArgs t0{};
  const TableArgs *tabs = b->tabs;
  const Chunk *ch = b->ins_chunks;
  const u64 *keys = reinterpret_cast<const u64 *>(d_keys);
  u64 m = 0;
  void *args[] = {&cells, &t0, &tabs, &ch, &nch, &keys, &m, &sign, &ba};
  const int grid = nch < (u32)b->grid_bin ? (int)nch : b->grid_bin;
  PP_CUDA(cudaLaunchKernel(b->k.bin, dim3(grid), dim3(kBlock), args, b->smem_bin, s));
  return PP_OK;
}

// Binned update without slab lists, for batches whose tables each lie within
// two slabs: the tile pass hashes the keys of each slab's tables itself
// (k_tile_step_keys), so no slab list is written or read back.  Tiles are
// sized for the expected records of the fullest slab, the overflow sets for
// the most records a slab can receive (every key of every table it overlaps).
static pp_status batch_keys_pass(pp_batch *b, const uint64_t *d_keys, const uint64_t *h_key_offsets, u32 nch,
                                 int sign, bool zero_fill, cudaStream_t s, const PrescanArgs *pre = nullptr) {
  const uint32_t ns = (uint32_t)((b->total_cells + kSlabCells - 1) / kSlabCells);
  std::vector<double> expect(ns, 0.0);
  std::vector<uint64_t> bound(ns, 0);
  for (uint32_t i = 0; i < b->n_tables; ++i) {
    const TableArgs &t = b->h_tabs[i];
    const uint64_t rec = (h_key_offsets[i + 1] - h_key_offsets[i]) * t.r;
    if (rec == 0) continue;
    const uint64_t c0 = t.base, c1 = (uint64_t)t.base + t.n_cells;
    for (uint64_t sl = c0 / kSlabCells; sl * kSlabCells < c1; ++sl) {
      const uint64_t a0 = sl * kSlabCells > c0 ? sl * kSlabCells : c0;
      const uint64_t a1 = (sl + 1) * kSlabCells < c1 ? (sl + 1) * kSlabCells : c1;
      expect[sl] += (double)rec * (double)(a1 - a0) / (double)t.n_cells;
      bound[sl] += rec;
    }
  }
  double mx = 0;
  uint64_t ocap = 0;
  for (uint32_t sl = 0; sl < ns; ++sl) {
    mx = expect[sl] > mx ? expect[sl] : mx;
    ocap = bound[sl] > ocap ? bound[sl] : ocap;
  }
  // each slab's range of the (table-ordered) chunk list
  if (ns > b->slab_chunk_cap) {
    PP_CUDA(cudaStreamSynchronize(s));
    cudaFree(b->slab_chunk);
    cudaFreeHost(b->h_slab_chunk);
    b->slab_chunk = nullptr;
    b->h_slab_chunk = nullptr;
    b->slab_chunk_cap = 0;
    PP_CUDA(cudaMalloc((void **)&b->slab_chunk, 2 * (size_t)ns * sizeof(u32)));
    PP_CUDA(cudaMallocHost((void **)&b->h_slab_chunk, 2 * (size_t)ns * sizeof(u32)));
    b->slab_chunk_cap = ns;
  }
  u32 *sc = b->h_slab_chunk;  // upload_chunks synchronized the stream: no copy reads it
  for (uint32_t sl = 0; sl < ns; ++sl) sc[2 * sl] = 0xffffffffu, sc[2 * sl + 1] = 0;
  for (u32 ch = 0; ch < nch; ++ch) {
    const TableArgs &t = b->h_tabs[b->h_ins_chunks[ch].table];
    const uint64_t c0 = t.base, c1 = (uint64_t)t.base + t.n_cells;
    for (uint64_t sl = c0 / kSlabCells; sl * kSlabCells < c1; ++sl) {
      if (ch < sc[2 * sl]) sc[2 * sl] = ch;
      sc[2 * sl + 1] = ch + 1;
    }
  }
  for (uint32_t sl = 0; sl < ns; ++sl)
    if (sc[2 * sl] == 0xffffffffu) sc[2 * sl] = 0;
  PP_CUDA(cudaMemcpyAsync(b->slab_chunk, sc, 2 * (size_t)ns * sizeof(u32), cudaMemcpyHostToDevice, s));
  pp_status st = ensure_tiles(b->tiles, tile_cap_for((uint64_t)mx + 1), ocap, ns, true, s);
  if (st != PP_OK) return st;
  return tile_keys_pass(b->cells, b->tabs, reinterpret_cast<const u64 *>(d_keys), b->ins_chunks, b->slab_chunk,
                        ns, b->krank, b->tiles, b->total_cells, sign, zero_fill, s, pre);
}

// Pass 2: slab by slab (zero-filled first when building from scratch).
static pp_status batch_apply_pass(pp_batch *b, BinArgs &ba, int sign, bool zero_fill, cudaStream_t s) {
  pp_status st = ensure_tiles(b->tiles, tile_cap_for(ba.cap), ba.cap, ba.n_slabs, true, s);
  if (st != PP_OK) return st;
  TableArgs t0{};
  return tile_apply_pass(b->cells, t0, b->tabs, ba, b->tiles, b->total_cells, sign, zero_fill, s);
}

static void add_items(pp_batch *b, const uint64_t *h_key_offsets, int sign) {
  for (uint32_t i = 0; i < b->n_tables; ++i) {
    const uint64_t d = h_key_offsets[i + 1] - h_key_offsets[i];
    b->items[i] = sign > 0 ? b->items[i] + d : (b->items[i] >= d ? b->items[i] - d : 0);
  }
}

static pp_status batch_update(pp_batch *b, const uint64_t *d_keys, const uint64_t *h_key_offsets,
                              int sign, void *stream) {
  if (!b || !h_key_offsets) return fail(PP_ERR_INVALID_ARG, "pp_batch_insert: NULL argument");
  cudaStream_t s = as_stream(stream);
  u32 nch = 0;
  uint64_t records = 0;
  pp_status st = upload_chunks(b, h_key_offsets, s, &nch, &records);
  if (st != PP_OK || nch == 0) return st;
  if (!d_keys) return fail(PP_ERR_INVALID_ARG, "pp_batch_insert: NULL keys");
  if (use_binned(b, records) && b->keys_tiles) {
    st = batch_keys_pass(b, d_keys, h_key_offsets, nch, sign, false, s);
  } else if (use_binned(b, records)) {
    BinArgs ba;
    st = batch_bin_pass(b, d_keys, h_key_offsets, nch, sign, 1, s, ba);
    if (st == PP_OK) st = batch_apply_pass(b, ba, sign, false, s);
  } else {
    st = direct_update(b, d_keys, nch, sign, s);
  }
  if (st == PP_OK) add_items(b, h_key_offsets, sign);
  return st;
}

pp_status pp_batch_insert(pp_batch *b, const uint64_t *d_keys, const uint64_t *h_key_offsets,
                          void *stream) {
  return batch_update(b, d_keys, h_key_offsets, +1, stream);
}

pp_status pp_batch_delete(pp_batch *b, const uint64_t *d_keys, const uint64_t *h_key_offsets,
                          void *stream) {
  if (b) b->had_deletes = true;
  return batch_update(b, d_keys, h_key_offsets, -1, stream);
}

pp_status pp_batch_build(pp_batch *b, const uint64_t *d_keys, const uint64_t *h_key_offsets, void *stream) {
  if (!b || !h_key_offsets) return fail(PP_ERR_INVALID_ARG, "pp_batch_build: NULL argument");
  cudaStream_t s = as_stream(stream);
  for (auto &x : b->items) x = 0;
  b->had_deletes = false;
  u32 nch = 0;
  uint64_t records = 0;
  pp_status st = upload_chunks(b, h_key_offsets, s, &nch, &records);
  if (st != PP_OK) return st;
  if (nch && !d_keys) return fail(PP_ERR_INVALID_ARG, "pp_batch_build: NULL keys");
  if (nch == 0 || !use_binned(b, records)) {
    PP_CUDA(cudaMemsetAsync(b->cells, 0, b->total_cells * sizeof(Cell), s));
    if (nch) st = direct_update(b, d_keys, nch, +1, s);
  } else if (b->keys_tiles) {
    st = batch_keys_pass(b, d_keys, h_key_offsets, nch, +1, true, s);
  } else {
    BinArgs ba;
    st = batch_bin_pass(b, d_keys, h_key_offsets, nch, +1, 0, s, ba);
    if (st != PP_OK) return st;
    PP_CUDA(cudaMemcpyAsync(&b->h_ctl->more, b->bin_overflow, sizeof(u32), cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
    if (b->h_ctl->more) {
      // a slab got more updates than its list holds: build the plain way
      PP_CUDA(cudaMemsetAsync(b->cells, 0, b->total_cells * sizeof(Cell), s));
      st = direct_update(b, d_keys, nch, +1, s);
    } else {
      st = batch_apply_pass(b, ba, +1, true, s);
    }
  }
  if (st == PP_OK) add_items(b, h_key_offsets, +1);
  return st;
}

// The decode's first part: the output ranges checked (CAPACITY before
// anything runs), fresh per-table counters and control block, and the round
// kind's buffers (the control block is on the device when this returns).
static pp_status decode_prepare(pp_batch *b, uint64_t *d_out_keys, const uint64_t *h_out_offsets, cudaStream_t s,
                                const char *fn) {
  bool moved = false;
  for (uint32_t i = 0; i < b->n_tables; ++i) {
    const uint64_t o0 = h_out_offsets[i], o1 = h_out_offsets[i + 1];
    if (o1 < o0) return fail(PP_ERR_INVALID_ARG, "%s: output offsets decrease at table %u", fn, i);
    if (o1 - o0 < b->items[i])
      return fail(PP_ERR_CAPACITY, "%s: table %u has %llu keys but %llu output slots", fn, i,
                  (unsigned long long)b->items[i], (unsigned long long)(o1 - o0));
    if (b->h_tabs[i].out_base != o0 || b->h_tabs[i].out_cap != o1 - o0) {
      b->h_tabs[i].out_base = o0;
      b->h_tabs[i].out_cap = o1 - o0;
      moved = true;
    }
  }
  if (h_out_offsets[b->n_tables] && !d_out_keys) return fail(PP_ERR_INVALID_ARG, "%s: NULL output", fn);
  if (moved)
    PP_CUDA(cudaMemcpyAsync(b->tabs, b->h_tabs.data(), b->n_tables * sizeof(TableArgs),
                            cudaMemcpyHostToDevice, s));
  // fresh counters
  const uint32_t n = b->n_tables, sr = b->opt.stats_rounds;
  PP_CUDA(cudaMemsetAsync(b->bc.recovered, 0, n * sizeof(u64), s));
  PP_CUDA(cudaMemsetAsync(b->bc.nonempty, 0, n * sizeof(u64), s));
  PP_CUDA(cudaMemsetAsync(b->bc.emptied, 0, n * sizeof(u64), s));
  PP_CUDA(cudaMemsetAsync(b->bc.rounds, 0, n * sizeof(u32), s));
  PP_CUDA(cudaMemsetAsync(b->bc.round_rec, 0, (size_t)n * sr * sizeof(u32), s));
  memset(b->h_ctl, 0, sizeof(DecodeCtl));
  b->h_ctl->max_rounds = b->opt.max_rounds;
  b->h_ctl->stats_rounds = sr;
  // round kind: tile rounds (batches built from insertions only), binned
  // atomic rounds (other large arenas), direct atomics (small arenas)
  const bool large = b->total_cells >= (1ull << 21);
  const bool want_tiles = batch_wants_tiles(b);
  const bool want_bins = !want_tiles && (b->opt.binned == 1 || (b->opt.binned == 0 && large));
  if (want_tiles) {
    pp_status st = ensure_batch_tiles(b, s);
    if (st != PP_OK) return st;
  }
  if (want_bins) {
    pp_status st = ensure_round_bins(b, s);
    if (st != PP_OK) return st;
    PP_CUDA(cudaMemsetAsync(b->bin_count, 0, b->n_bins * sizeof(u32), s));
  }
  if (b->exec && (want_bins != b->binned_rounds || want_tiles != b->tile_rounds ||
                  ((want_bins || want_tiles) && b->graph_gen != b->rec_gen))) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->binned_rounds = want_bins;
  b->tile_rounds = want_tiles;
  PP_CUDA(cudaMemcpyAsync(b->ctl, b->h_ctl, sizeof(DecodeCtl), cudaMemcpyHostToDevice, s));
  return PP_OK;
}

// The round loop of the kind decode_prepare chose (prescanned: tile rounds
// after a build that found F_1).
static pp_status decode_rounds(pp_batch *b, u64 *out, bool prescanned, cudaStream_t s) {
  if (b->tile_rounds && b->opt.host_loop) {
    TileRoundLaunch a;
    fill_tiles(b, a, out);
    pp_status st = tre_host_loop(b->tre, b->k, a, &b->h_ctl->more, s, prescanned);
    if (st != PP_OK) return st;
  } else if (b->tile_rounds && prescanned) {
    if (b->exec_pre && (b->graph_out_pre != out || b->graph_gen_pre != b->rec_gen)) {
      cudaGraphExecDestroy(b->exec_pre);
      b->exec_pre = nullptr;
    }
    if (!b->exec_pre) {
      TileRoundLaunch a;
      fill_tiles(b, a, out);
      pp_status st = tre_build_graph(b->tre, b->k, a, &b->exec_pre, true);
      if (st != PP_OK) return st;
      b->graph_out_pre = out;
      b->graph_gen_pre = b->rec_gen;
    }
    PP_CUDA(cudaGraphLaunch(b->exec_pre, s));
  } else if (b->tile_rounds) {
    if (!b->exec || b->graph_out != out) {
      if (b->exec) cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
      TileRoundLaunch a;
      fill_tiles(b, a, out);
      pp_status st = tre_build_graph(b->tre, b->k, a, &b->exec);
      if (st != PP_OK) return st;
      b->graph_out = out;
      b->graph_gen = b->rec_gen;
    }
    PP_CUDA(cudaGraphLaunch(b->exec, s));
  } else if (b->opt.host_loop) {
    BatchArgs a;
    fill(b, a, out);
    PP_CUDA(cudaLaunchKernel(b->k.scan, dim3(b->grid_scan), dim3(kBlock), a.scan_p, 0, s));
    for (;;) {
      if (b->binned_rounds) {
        PP_CUDA(cudaLaunchKernel(b->k.claim, dim3(b->grid_claim), dim3(kBlock), a.claim_p, b->smem_claim, s));
        PP_CUDA(cudaLaunchKernel(b->k.apply_round, dim3(b->grid_apply_round), dim3(kBlock), a.applyr_p,
                                 b->smem_apply_round, s));
        PP_CUDA(cudaLaunchKernel(b->k.filter, dim3(b->grid_filter), dim3(kBlock), a.filter_p, 0, s));
        PP_CUDA(cudaLaunchKernel(bins_reset_kernel(), dim3(1), dim3(256), a.reset_p, 0, s));
      } else {
        PP_CUDA(cudaLaunchKernel(b->k.peel, dim3(b->grid_peel), dim3(kBlock), a.peel_p, b->smem_peel, s));
        PP_CUDA(cudaLaunchKernel(b->k.filter, dim3(b->grid_filter), dim3(kBlock), a.filter_p, 0, s));
      }
      PP_CUDA(cudaLaunchKernel(round_end_kernel(), dim3(1), dim3(32), a.end_p, 0, s));
      PP_CUDA(cudaMemcpyAsync(&b->h_ctl->more, &b->ctl->more, sizeof(u32), cudaMemcpyDeviceToHost, s));
      PP_CUDA(cudaStreamSynchronize(s));
      if (!b->h_ctl->more) break;
    }
  } else {
    if (!b->exec || b->graph_out != out) {
      pp_status st = build_graph(b, out);
      if (st != PP_OK) return st;
      b->graph_out = out;
    }
    PP_CUDA(cudaGraphLaunch(b->exec, s));
  }
  return PP_OK;
}

// The residue count and the per-table results; synchronizes s.
static pp_status decode_finish(pp_batch *b, pp_table_result *results, cudaStream_t s, const char *fn) {
  const uint32_t n = b->n_tables, sr = b->opt.stats_rounds;
  const bool scan_residue = b->binned_rounds || b->tile_rounds;
  if (scan_residue) {
    // the binned and tile rounds do not track emptied cells per table: count the residue
    for (uint32_t i = 0; i < n; ++i) b->h_items[i] = b->items[i];
    PP_CUDA(cudaMemcpyAsync((void *)b->bc.items, b->h_items, n * sizeof(u64), cudaMemcpyHostToDevice, s));
    PP_CUDA(cudaMemsetAsync(b->bc.residual, 0, n * sizeof(u64), s));
    BatchCounters bc = b->bc;
    bc.skip_full = b->had_deletes ? 0u : 1u;
    const Cell *cells = b->cells;
    const Chunk *ch = b->scan_chunks;
    u32 nch = b->n_scan_chunks;
    void *args[] = {&cells, &ch, &nch, &bc};
    PP_CUDA(cudaLaunchKernel(residual_kernel(), dim3(b->grid_scan), dim3(kBlock), args, 0, s));
    PP_CUDA(cudaMemcpyAsync(b->h_residual, b->bc.residual, n * sizeof(u64), cudaMemcpyDeviceToHost, s));
  }
  PP_CUDA(cudaMemcpyAsync(b->h_ctl, b->ctl, sizeof(DecodeCtl), cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaMemcpyAsync(b->h_recovered, b->bc.recovered, n * sizeof(u64), cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaMemcpyAsync(b->h_nonempty, b->bc.nonempty, n * sizeof(u64), cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaMemcpyAsync(b->h_emptied, b->bc.emptied, n * sizeof(u64), cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaMemcpyAsync(b->h_rounds, b->bc.rounds, n * sizeof(u32), cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaMemcpyAsync(b->h_round_rec, b->bc.round_rec, (size_t)n * sr * sizeof(u32),
                          cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaStreamSynchronize(s));
  for (uint32_t i = 0; i < n; ++i) {
    pp_table_result &r = results[i];
    r.rounds = b->h_rounds[i];
    r.recovered = b->h_recovered[i];
    r.items_before = b->items[i];
    r.residual_cells = scan_residue ? b->h_residual[i] : b->h_nonempty[i] - b->h_emptied[i];
    const uint32_t nc = r.rounds < r.round_cap ? r.rounds : r.round_cap;
    if (r.recovered_per_round) {
      for (uint32_t t = 0; t < nc; ++t)
        r.recovered_per_round[t] = t < sr ? b->h_round_rec[(size_t)i * sr + t] : 0;
    }
    r.stats_complete = r.rounds <= sr;
    b->items[i] -= r.recovered <= b->items[i] ? r.recovered : b->items[i];
  }
  if (b->h_ctl->flags & FLAG_CAPACITY) return fail(PP_ERR_CAPACITY, "%s: output overflow", fn);
  if (b->h_ctl->flags & FLAG_INTERNAL)
    return fail(PP_ERR_INVALID_ARG, "%s: a pure cell's key does not hash to it", fn);
  if (b->h_ctl->flags & FLAG_ROUND_LIMIT)
    return fail(PP_ERR_ROUND_LIMIT, "%s: stopped after max_rounds=%u rounds", fn, b->opt.max_rounds);
  return PP_OK;
}


pp_status pp_batch_decode(pp_batch *b, uint64_t *d_out_keys, const uint64_t *h_out_offsets,
                          pp_table_result *results, void *stream) {
  if (!b || !h_out_offsets || !results) return fail(PP_ERR_INVALID_ARG, "pp_batch_decode: NULL argument");
  cudaStream_t s = as_stream(stream);
  pp_status st = decode_prepare(b, d_out_keys, h_out_offsets, s, "pp_batch_decode");
  if (st != PP_OK) return st;
  st = decode_rounds(b, reinterpret_cast<u64 *>(d_out_keys), false, s);
  if (st != PP_OK) return st;
  return decode_finish(b, results, s, "pp_batch_decode");
}

pp_status pp_batch_build_decode(pp_batch *b, const uint64_t *d_keys, const uint64_t *h_key_offsets,
                                uint64_t *d_out_keys, const uint64_t *h_out_offsets, pp_table_result *results,
                                void *stream) {
  if (!b || !h_key_offsets || !h_out_offsets || !results)
    return fail(PP_ERR_INVALID_ARG, "pp_batch_build_decode: NULL argument");
  cudaStream_t s = as_stream(stream);
  uint64_t records = 0;
  for (uint32_t i = 0; i < b->n_tables; ++i) {
    if (h_key_offsets[i + 1] < h_key_offsets[i] || h_out_offsets[i + 1] < h_out_offsets[i])
      return fail(PP_ERR_INVALID_ARG, "pp_batch_build_decode: offsets decrease at table %u", i);
    const uint64_t m = h_key_offsets[i + 1] - h_key_offsets[i];
    if (h_out_offsets[i + 1] - h_out_offsets[i] < m)
      return fail(PP_ERR_CAPACITY, "pp_batch_build_decode: table %u gets %llu keys but %llu output slots", i,
                  (unsigned long long)m, (unsigned long long)(h_out_offsets[i + 1] - h_out_offsets[i]));
    records += m * b->h_tabs[i].r;
  }
  // the tile write-out finds F_1 when the build takes the keys' tile pass and
  // the decode the tile rounds; otherwise the two calls
  const bool had = b->had_deletes;
  b->had_deletes = false;
  const bool fused = records && b->keys_tiles && use_binned(b, records) && b->k.trescan && batch_wants_tiles(b);
  b->had_deletes = had;
  if (!fused) {
    pp_status st = pp_batch_build(b, d_keys, h_key_offsets, stream);
    if (st != PP_OK) return st;
    return pp_batch_decode(b, d_out_keys, h_out_offsets, results, stream);
  }
  if (!d_keys) return fail(PP_ERR_INVALID_ARG, "pp_batch_build_decode: NULL keys");
  for (auto &x : b->items) x = 0;
  b->had_deletes = false;
  u32 nch = 0;
  uint64_t rec = 0;
  pp_status st = upload_chunks(b, h_key_offsets, s, &nch, &rec);
  if (st != PP_OK) return st;
  add_items(b, h_key_offsets, +1);  // the record regions of the tile rounds are sized from them
  st = decode_prepare(b, d_out_keys, h_out_offsets, s, "pp_batch_build_decode");
  if (st != PP_OK) return st;
  if (!b->tile_rounds) return fail(PP_ERR_INVALID_ARG, "pp_batch_build_decode: tile rounds expected");
  const TileRoundBufs &tb = b->tre.trb;
  PP_CUDA(cudaMemsetAsync(tb.fseg, 0, (size_t)tb.n_seg_d * sizeof(u32), s));
  PP_CUDA(cudaMemsetAsync(tb.n_rescan, 0, sizeof(u32), s));
  const PrescanArgs pre{tb, b->fkey, b->fcell, b->bitmap, b->ctl, 0ull, b->wseed};
  st = batch_keys_pass(b, d_keys, h_key_offsets, nch, +1, true, s, &pre);
  if (st != PP_OK) return st;
  st = decode_rounds(b, reinterpret_cast<u64 *>(d_out_keys), true, s);
  if (st != PP_OK) return st;
  return decode_finish(b, results, s, "pp_batch_build_decode");
}

pp_status pp_batch_copy_cells(pp_batch *b, uint32_t table, void *dst, int to_host, void *stream) {
  if (!b || !dst || table >= b->n_tables) return fail(PP_ERR_INVALID_ARG, "pp_batch_copy_cells: bad argument");
  cudaStream_t s = as_stream(stream);
  const TableArgs &t = b->h_tabs[table];
  PP_CUDA(cudaMemcpyAsync(dst, b->cells + t.base, (size_t)t.n_cells * sizeof(Cell),
                          to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  PP_CUDA(cudaStreamSynchronize(s));
  return PP_OK;
}

pp_status pp_batch_set_options(pp_batch *b, const pp_options *opt) {
  if (!b) return fail(PP_ERR_INVALID_ARG, "pp_batch_set_options: NULL batch");
  PP_CUDA(cudaDeviceSynchronize());
  const pp_options old = b->opt;
  b->opt = resolve_options(opt);
  // the per-table statistics and round buffers were sized at creation
  b->opt.max_rounds = old.max_rounds;
  b->opt.stats_rounds = old.stats_rounds;
  b->grid_scan = persistent_grid(b->k.scan, kBlock, 0, b->opt.ctas_per_sm);
  b->grid_peel = persistent_grid(b->k.peel, kBlock, b->smem_peel, b->opt.ctas_per_sm);
  b->grid_filter = persistent_grid(b->k.filter, kBlock, 0, b->opt.ctas_per_sm);
  b->n_slabs = 0;  // the binning grid is recomputed on the next binned update
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return PP_OK;
}

pp_status pp_batch_get_options(const pp_batch *b, pp_options *opt) {
  if (!b || !opt) return fail(PP_ERR_INVALID_ARG, "pp_batch_get_options: NULL argument");
  *opt = b->opt;
  return PP_OK;
}

pp_status pp_batch_info(const pp_batch *b, uint32_t *n_tables, uint64_t *total_cells, uint32_t *last_rounds) {
  if (!b) return fail(PP_ERR_INVALID_ARG, "pp_batch_info: NULL batch");
  if (n_tables) *n_tables = b->n_tables;
  if (total_cells) *total_cells = b->total_cells;
  if (last_rounds) *last_rounds = b->h_ctl ? b->h_ctl->round : 0;
  return PP_OK;
}

}  // extern "C"
