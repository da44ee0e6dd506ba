// Host side of the build's tile pass (kernels in iblt_tiles.cuh): buffers and
// the per-slab launch sequence, shared by the single-table and batched paths.
#include "host.cuh"
#include "iblt_tiles.cuh"

namespace pp {

static_assert(kTilesPerSlab <= kTileThreads, "the bin role scans one histogram entry per thread");

void free_tiles(TileBufs &tb) {
  cudaFree(tb.key);
  cudaFree(tb.off);
  cudaFree(tb.tab);
  cudaFree(tb.count);
  cudaFree(tb.o_key);
  cudaFree(tb.o_cell);
  cudaFree(tb.o_tab);
  cudaFree(tb.o_count);
  tb = TileBufs{};
}

// dynamic shared memory of k_tile_step: the larger of the two roles
static size_t tile_step_smem() {
  const size_t bin = (size_t)kTileBinChunk * (8 + 4 + 4 + 4);  // a batch bin step (plain: 4 B less per record)
  const size_t apply = (size_t)kTileCells * (8 + 8 + 4);
  return bin > apply ? bin : apply;
}

static const void *tile_step_fn(bool batch, bool prescan = false) {
  if (prescan) return (const void *)k_tile_step<false, true>;
  return batch ? (const void *)k_tile_step<true> : (const void *)k_tile_step<false>;
}

// rank as for iblt_kernels: 3, 4, -4 (any r <= 4) or 0 (any r); prescan: the
// write-out also finds F_1
static const void *tile_keys_fn(int rank, bool prescan) {
  static bool attr = false;
  const void *f[8] = {(const void *)k_tile_step_keys<3>,        (const void *)k_tile_step_keys<4>,
                      (const void *)k_tile_step_keys<-4>,       (const void *)k_tile_step_keys<0>,
                      (const void *)k_tile_step_keys<3, true>,  (const void *)k_tile_step_keys<4, true>,
                      (const void *)k_tile_step_keys<-4, true>, (const void *)k_tile_step_keys<0, true>};
  if (!attr) {
    for (const void *p : f) cudaFuncSetAttribute(p, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_step_smem());
    attr = true;
  }
  return f[(prescan ? 4 : 0) + (rank == 3 ? 0 : rank == 4 ? 1 : rank == -4 ? 2 : 3)];
}

uint64_t tile_cap_for(uint64_t slab_cap) {
  // a tile's expected share of its slab's list with slack, a multiple of 64
  // records so that every tile's region of 2-byte offsets starts on a
  // 128-byte line (a fuller tile spills to the overflow list, which holds a
  // whole slab)
  const uint64_t c = (uint64_t)((double)slab_cap / kTilesPerSlab * 1.15) + 256;
  return (c + 63) / 64 * 64;
}

uint64_t tile_pass_bytes(uint64_t tile_cap, uint64_t o_cap, uint32_t n_slabs, bool batch) {
  const uint64_t tab = batch ? sizeof(u32) : 0;
  return 2 * tile_cap * kTilesPerSlab * (sizeof(u64) + sizeof(u16) + tab) + 2 * kTilesPerSlab * sizeof(u32) +
         3 * o_cap * (sizeof(u64) + sizeof(u32) + tab) + (uint64_t)n_slabs * sizeof(u32);
}

pp_status ensure_tiles(TileBufs &tb, uint64_t tile_cap, uint64_t o_cap, uint32_t n_slabs, bool batch,
                       cudaStream_t s) {
  if (tile_cap > 0xFFFFFFF0ull || o_cap > 0xFFFFFFF0ull)
    return fail(PP_ERR_INVALID_ARG, "tile pass: too many updates for one call");
  if (tb.key && tile_cap <= tb.cap && o_cap <= tb.o_cap && n_slabs <= tb.o_slabs && batch == tb.batch)
    return PP_OK;
  PP_CUDA(cudaStreamSynchronize(s));
  const uint64_t cap = tile_cap > tb.cap ? tile_cap : tb.cap;  // tile_cap_for: multiples of 64
  const uint64_t ocap = o_cap > tb.o_cap ? o_cap : tb.o_cap;
  const uint32_t ns = n_slabs > tb.o_slabs ? n_slabs : tb.o_slabs;
  free_tiles(tb);
  const uint64_t rec = 2 * cap * kTilesPerSlab;
  cudaError_t e = cudaSuccess;
  auto al = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  al((void **)&tb.key, rec * 8);
  al((void **)&tb.off, rec * 2);
  if (batch) al((void **)&tb.tab, rec * 4);
  al((void **)&tb.count, 2 * kTilesPerSlab * 4);
  al((void **)&tb.o_key, 3 * ocap * 8);
  al((void **)&tb.o_cell, 3 * ocap * 4);
  if (batch) al((void **)&tb.o_tab, 3 * ocap * 4);
  al((void **)&tb.o_count, (size_t)ns * 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(tb.count, 0, 2 * kTilesPerSlab * 4, s);
  if (e != cudaSuccess) {
    free_tiles(tb);
    return cuda_fail(e, "tile pass buffers", __FILE__, __LINE__);
  }
  tb.cap = cap;
  tb.o_cap = ocap;
  tb.o_slabs = ns;
  tb.batch = batch;
  static bool attr[2] = {false, false};
  if (!attr[batch]) {
    cudaFuncSetAttribute(tile_step_fn(batch), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_step_smem());
    if (!batch)
      cudaFuncSetAttribute(tile_step_fn(false, true), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tile_step_smem());
    attr[batch] = true;
  }
  return PP_OK;
}

pp_status tile_apply_pass(Cell *cells, const TableArgs &tab0, const TableArgs *tabs, const BinArgs &ba,
                          TileBufs &tb, uint64_t n_cells, int sign, bool zero, cudaStream_t s,
                          const PrescanArgs *pre) {
  if (pre && (tb.batch || !zero)) return fail(PP_ERR_INVALID_ARG, "tile pass: F_1 is found only by a plain build");
  PP_CUDA(cudaMemsetAsync(tb.o_count, 0, (size_t)ba.n_slabs * 4, s));
  TileArgs ta{tb.key, tb.off, tb.tab, tb.count, tb.cap * kTilesPerSlab, (u32)tb.cap, (u32)tb.o_cap,
              tb.o_key, tb.o_cell, tb.o_tab, tb.o_count};
  Cell *c = cells;
  TableArgs t0 = tab0;
  const TableArgs *tp = tabs;
  BinArgs b = ba;
  u32 step = 0, n_apply = 0, n_bin = 0;
  u64 n = n_cells;
  int sg = sign, z = zero ? 1 : 0;
  PrescanArgs pa = pre ? *pre : PrescanArgs{};
  void *args[] = {&c, &t0, &tp, &b, &ta, &step, &n_apply, &n_bin, &n, &sg, &z, &pa};
  const void *fn = tile_step_fn(tb.batch, pre != nullptr);
  const u32 ns = ba.n_slabs;
  const u32 sms = (u32)sm_count();
  // launch s: sort slab s while slab s - 1 is applied tile by tile
  for (step = 0; step <= ns + 1; ++step) {
    n_bin = step < ns ? 3 * sms : 0u;
    n_apply = (step >= 1 && step - 1 < ns) ? kTilesPerSlab : (step == ns + 1 ? 2 * sms : 0u);
    if (n_apply + n_bin == 0) continue;
    PP_CUDA(cudaLaunchKernel(fn, dim3(n_apply + n_bin), dim3(kTileThreads), args, tile_step_smem(), s));
  }
  return PP_OK;
}

pp_status tile_keys_pass(Cell *cells, const TableArgs *tabs, const u64 *keys, const Chunk *chunks,
                         const u32 *slab_chunk, uint32_t n_slabs, int rank, TileBufs &tb, uint64_t n_cells,
                         int sign, bool zero, cudaStream_t s, const PrescanArgs *pre) {
  if (!tb.batch) return fail(PP_ERR_INVALID_ARG, "tile pass: batch buffers expected");
  if (pre && !zero) return fail(PP_ERR_INVALID_ARG, "tile pass: F_1 is found only by a build");
  PP_CUDA(cudaMemsetAsync(tb.o_count, 0, (size_t)n_slabs * 4, s));
  TileArgs ta{tb.key, tb.off, tb.tab, tb.count, tb.cap * kTilesPerSlab, (u32)tb.cap, (u32)tb.o_cap,
              tb.o_key, tb.o_cell, tb.o_tab, tb.o_count};
  TileKeysArgs ka{keys, chunks, slab_chunk, n_slabs};
  Cell *c = cells;
  const TableArgs *tp = tabs;
  u32 step = 0, n_apply = 0, n_bin = 0;
  u64 n = n_cells;
  int sg = sign, z = zero ? 1 : 0;
  PrescanArgs pa = pre ? *pre : PrescanArgs{};
  void *args[] = {&c, &tp, &ka, &ta, &step, &n_apply, &n_bin, &n, &sg, &z, &pa};
  const void *fn = tile_keys_fn(rank, pre != nullptr);
  const u32 sms = (u32)sm_count();
  for (step = 0; step <= n_slabs + 1; ++step) {
    n_bin = step < n_slabs ? 3 * sms : 0u;
    n_apply = (step >= 1 && step - 1 < n_slabs) ? kTilesPerSlab : (step == n_slabs + 1 ? 2 * sms : 0u);
    if (n_apply + n_bin == 0) continue;
    PP_CUDA(cudaLaunchKernel(fn, dim3(n_apply + n_bin), dim3(kTileThreads), args, tile_step_smem(), s));
  }
  return PP_OK;
}

}  // namespace pp
