// C-ABI: one IBLT on the device (create, insert/delete, decode).
//
// Decode = initial full scan, then rounds of (peel, filter, round_end) until
// the frontier is empty (Sec. 1 rounds at k = 2 on the IBLT hypergraph of
// Sec. 6).  By default the round loop is a single CUDA graph: a while-node
// whose body is the three round kernels; the last one decides on the device
// whether another round runs, so the host neither syncs nor launches per round.
#include <stdlib.h>
#include <string.h>

#include "host.cuh"
#include "iblt_binned.cuh"
#include "iblt_kernels.cuh"
#include "iblt_rounds.cuh"
#include "iblt_subrounds.cuh"
#include "iblt_signed.cuh"
#include "iblt_trounds.cuh"

using namespace pp;

namespace pp {

template <int R, bool B>
static IbltKernels iblt_kernels_t() {
  static bool attr_set = false;
  if (!attr_set) {
    // the binning kernel's staging grows with r and the number of slabs
    cudaFuncSetAttribute((const void *)k_bin<R, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute((const void *)k_claim<R, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    if constexpr (!B) {
      cudaFuncSetAttribute((const void *)k_claim<R, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           200 * 1024);
      if constexpr (R >= 0) {
        cudaFuncSetAttribute((const void *)k_claim<R, false, true, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute((const void *)k_apply_round<R, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      }
    }
    cudaFuncSetAttribute((const void *)k_apply_round<R, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    attr_set = true;
  }
  IbltKernels k{(const void *)k_insert<R, B>, (const void *)k_scan<R, B>, (const void *)k_peel<R, B>,
                (const void *)k_filter<R, B>, (const void *)k_bin<R, B>, (const void *)k_claim<R, B>,
                (const void *)k_apply_round<R, B>, nr_of<R>()};
  if constexpr (!B && R >= 0) {
    k.sub_scan = (const void *)k_sscan<R>;
    k.sub_filter = (const void *)k_sfilter<R>;
    k.sub_peel = (const void *)k_speel<R>;
    k.sub_claim = (const void *)k_claim<R, false, false>;
    k.sg_scan = (const void *)k_sgscan<R>;
    k.sg_peel = (const void *)k_sgpeel<R>;
    k.sg_filter = (const void *)k_sgfilter<R>;
    k.sg_claim = (const void *)k_claim<R, false, true, true>;
    k.sg_apply = (const void *)k_apply_round<R, false, true>;
  }
  if constexpr (R >= 0 || B) {
    // tile rounds: plain for a fixed rank or the generic one, batched for every rank code
    k.tscan = (const void *)k_tscan<R, B>;
    k.tclaim = (const void *)k_tclaim<R, B>;
    k.tapply = (const void *)k_tapply<R, B>;
    k.tapply_sparse = (const void *)k_tapply_sparse<R, B>;
    k.trestore = (const void *)k_trestore<R, B>;
    k.trescan = (const void *)k_trescan<R, B>;
    static bool tattr = false;
    if (!tattr) {
      allow_max_dynamic_smem((const void *)k_tapply<R, B>);
      allow_max_dynamic_smem((const void *)k_tclaim<R, B>);
      allow_max_dynamic_smem((const void *)k_tsort);
      allow_max_dynamic_smem((const void *)k_tapply_sparse<R, B>);
      tattr = true;
    }
  }
  return k;
}

IbltKernels iblt_kernels(int rank, bool batch) {
  if (batch) {
    if (rank == 3) return iblt_kernels_t<3, true>();
    if (rank == 4) return iblt_kernels_t<4, true>();
    if (rank == -4) return iblt_kernels_t<-4, true>();
    return iblt_kernels_t<0, true>();
  }
  const uint32_t r = (uint32_t)rank;
  if (r == 3) return iblt_kernels_t<3, false>();
  if (r == 4) return iblt_kernels_t<4, false>();
  return iblt_kernels_t<0, false>();
}

const void *round_end_kernel() { return (const void *)k_round_end; }

const void *bins_reset_kernel() { return (const void *)k_bins_reset; }

const void *residual_kernel() { return (const void *)k_residual; }

size_t claim_smem_bytes(int nr, bool batch, uint32_t n_bins, bool sgn) {
  const size_t cap = (size_t)kClaimChunk * nr;
  return cap * (8 + 4 + (batch ? 4 : 0)) + (size_t)kClaimChunk * 8 + 3 * (size_t)n_bins * 4 +
         (sgn ? (size_t)kClaimChunk : 0);
}

size_t apply_round_smem_bytes(bool batch, uint32_t n_bins) {
  return ((size_t)n_bins + 1) * 4 + (size_t)kApplyChunk * 4 * (batch ? 2 : 1);
}

size_t bin_smem_bytes(int nr, bool batch, uint32_t n_slabs) {
  const size_t cap = (size_t)kBinKeys * nr;
  return cap * (8 + 4 + (batch ? 4 : 0)) + 3 * (size_t)n_slabs * 4;
}

size_t peel_smem_bytes(int nr, bool batch) {
  const size_t ch = (size_t)kBlock * kPeelItems;
  return (batch ? 0 : ch * sizeof(u64)) + ch * nr * sizeof(u32) * (batch ? 2 : 1);
}

}  // namespace pp

namespace pp {

// One build + decode from host buffers in flight (pp_iblt_submit_host): its
// own device key and output buffers, pinned copies of the decode's control
// block and statistics, and the events that order the copies around it.
constexpr uint32_t kJobStatRounds = 4096;  // per-round statistics kept per job
constexpr uint32_t kHostJobs = 3;          // jobs in flight per table
struct HostJob {
  u64 *d_keys = nullptr, *d_out = nullptr;
  uint64_t cap = 0;                    // keys the device buffers hold
  DecodeCtl *h_ctl = nullptr;          // mapped pinned (d_ctl: its device address)
  u64 *h_stats = nullptr;              // mapped pinned: recovered, then alive, kJobStatRounds each
  u32 *h_flag = nullptr;               // mapped pinned: the build's slab overflow flag
  DecodeCtl *d_ctl = nullptr;
  u64 *d_stats = nullptr;
  u32 *d_flag = nullptr;
  cudaStream_t s = nullptr;            // the caller's stream the job ran on
  cudaEvent_t up = nullptr, built = nullptr, dec = nullptr, done = nullptr;
  const uint64_t *h_keys = nullptr;
  uint64_t *h_out = nullptr;
  uint64_t m = 0, out_cap = 0, ticket = 0;
  bool busy = false, reg_keys = false, reg_out = false;
};

}  // namespace pp

// ---- tile rounds: the host side shared by the single table and the batch ----
namespace pp {

namespace {

pp_status tre_node(cudaGraphNode_t *node, cudaGraph_t g, const cudaGraphNode_t *dep, size_t ndep, const void *fn,
                   int grid, int block, size_t smem, void **args) {
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void *>(fn);
  kp.gridDim = dim3((unsigned)grid);
  kp.blockDim = dim3((unsigned)block);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = args;
  PP_CUDA(cudaGraphAddKernelNode(node, g, dep, ndep, &kp));
  return PP_OK;
}

}  // namespace

// Frontier segments: one per block of k_tscan / k_tapply (n_seg_d, each at
// most 4096 pushes per tile it takes) and of k_tapply_sparse (n_seg_s, at most
// kTSCap pushes per tile).  Coarse bins of the claim: at most 128 when a bin of
// 512 tiles allows it, else as many bins of 512 tiles as the tiles need.
pp_status tre_setup(TileRoundEngine &e, const IbltKernels &k, uint64_t n_cells, uint32_t ctas_per_sm) {
  TileRoundBufs &b = e.trb;
  if (b.base) return PP_OK;
  const uint32_t nt = (uint32_t)((n_cells + kTRCells - 1) / kTRCells);
  e.grid_tapply = persistent_grid(k.tapply, kTRThreads, kTApplySmem, 2);
  e.grid_tsparse = persistent_grid(k.tapply_sparse, kTSThreads, kTSSmem, kTSCtas);
  e.grid_tscan = e.grid_tapply;
  const uint32_t nd = (uint32_t)e.grid_tapply, nsp = (uint32_t)e.grid_tsparse;
  const uint64_t cap_d = (uint64_t)kTRCells * ((nt + nd - 1) / nd);
  const uint64_t cap_s = (uint64_t)kTSCap * ((nt + nsp - 1) / nsp);
  if (cap_d > 0xFFFFFFFFull || cap_s > 0xFFFFFFFFull) return fail(PP_ERR_INVALID_ARG, "tile rounds: table too large");
  uint64_t *h_start = (uint64_t *)malloc((size_t)(nd + nsp) * sizeof(uint64_t));
  if (!h_start) return fail(PP_ERR_OUT_OF_MEMORY, "tile round segment table");
  for (uint32_t s = 0; s < nd + nsp; ++s) h_start[s] = s < nd ? s * cap_d : nd * cap_d + (s - nd) * cap_s;
  u64 *d_start = nullptr;
  uint32_t bsh = 0;
  while (bsh < 9 && ((nt + (1u << bsh) - 1) >> bsh) > 128) ++bsh;
  b.bin_tshift = bsh;
  b.n_bins = (nt + (1u << bsh) - 1) >> bsh;
  cudaError_t err = cudaMalloc((void **)&b.base, ((size_t)nt + 1) * sizeof(u64));
  if (err == cudaSuccess) err = cudaMalloc((void **)&b.pos, (size_t)nt * kTRPosStride * sizeof(u32));
  if (err == cudaSuccess) err = cudaMalloc((void **)&b.base64, ((size_t)nt + 1) * sizeof(u32));
  if (err == cudaSuccess) err = cudaMalloc((void **)&b.done, (size_t)nt * sizeof(u32));
  if (err == cudaSuccess) err = cudaMalloc((void **)&b.sum, (size_t)nt * sizeof(u32));
  if (err == cudaSuccess) err = cudaMalloc((void **)&b.act, (size_t)nt * sizeof(TileAct));
  if (err == cudaSuccess) err = cudaMalloc((void **)&b.act_d, (size_t)nt * sizeof(TileAct));
  if (err == cudaSuccess) err = cudaMalloc((void **)&b.fseg, (size_t)(nd + nsp) * sizeof(u32));
  if (err == cudaSuccess) err = cudaMalloc((void **)&b.rescan, (size_t)nt * sizeof(u32));
  if (err == cudaSuccess) err = cudaMalloc((void **)&b.n_rescan, sizeof(u32));
  if (err == cudaSuccess) err = cudaMalloc((void **)&b.cpos, (size_t)b.n_bins * kTRPosStride * sizeof(u32));
  if (err == cudaSuccess) err = cudaMalloc((void **)&b.cdone, (size_t)b.n_bins * sizeof(u32));
  if (err == cudaSuccess) err = cudaMalloc((void **)&d_start, (size_t)(nd + nsp) * sizeof(u64));
  if (err == cudaSuccess)
    err = cudaMemcpy(d_start, h_start, (size_t)(nd + nsp) * sizeof(u64), cudaMemcpyHostToDevice);
  free(h_start);
  b.fstart = d_start;
  if (err != cudaSuccess) {
    pp_status st = cuda_fail(err, "tile round buffers", __FILE__, __LINE__);
    tre_free(e);
    return st;
  }
  b.n_tiles = nt;
  b.n_seg_d = nd;
  b.n_seg_s = nsp;
  b.cap_d = (u32)cap_d;
  b.cap_s = (u32)cap_s;
  e.front = nd * cap_d + nsp * cap_s;
  e.smem_tclaim = (size_t)kTClaimChunk * k.nr * 12 + ((size_t)nd + nsp + 1) * 4 + (4 * (size_t)b.n_bins + 2) * 4;
  e.grid_tclaim = persistent_grid(k.tclaim, kTClaimThreads, e.smem_tclaim, ctas_per_sm);
  e.smem_tsort = tsort_smem_bytes(b.n_bins);
  e.grid_tsort = persistent_grid((const void *)k_tsort, kTSortThreads, e.smem_tsort, 8);
  e.grid_act = (int)((nt + kBlock - 1) / kBlock);
  return PP_OK;
}

pp_status tre_records(TileRoundEngine &e, uint64_t need, cudaStream_t s, bool *moved) {
  TileRoundBufs &b = e.trb;
  if (moved) *moved = false;
  if (need <= b.rec_cap) return PP_OK;
  PP_CUDA(cudaStreamSynchronize(s));
  cudaFree(b.rec_key);
  cudaFree(b.rec_off);
  cudaFree(b.crec_key);
  cudaFree(b.crec_cell);
  b.rec_key = b.crec_key = nullptr;
  b.rec_off = nullptr;
  b.crec_cell = nullptr;
  b.rec_cap = 0;
  PP_CUDA(cudaMalloc((void **)&b.rec_key, need * sizeof(u64)));
  PP_CUDA(cudaMalloc((void **)&b.rec_off, need * sizeof(u16)));
  PP_CUDA(cudaMalloc((void **)&b.crec_key, need * sizeof(u64)));
  PP_CUDA(cudaMalloc((void **)&b.crec_cell, need * sizeof(u32)));
  b.rec_cap = need;
  if (moved) *moved = true;
  return PP_OK;
}

uint64_t tre_record_need(const TileRoundEngine &e, uint64_t updates) {
  return updates + (uint64_t)kTRAlign * e.trb.n_tiles;
}

void tre_free(TileRoundEngine &e) {
  TileRoundBufs &b = e.trb;
  cudaFree(b.rec_key);
  cudaFree(b.rec_off);
  cudaFree(b.crec_key);
  cudaFree(b.crec_cell);
  cudaFree(b.cpos);
  cudaFree(b.cdone);
  cudaFree(b.base);
  cudaFree(b.pos);
  cudaFree(b.base64);
  cudaFree(b.done);
  cudaFree(b.sum);
  cudaFree(b.act);
  cudaFree(b.act_d);
  cudaFree(b.fseg);
  cudaFree(b.rescan);
  cudaFree(b.n_rescan);
  cudaFree(const_cast<u64 *>(b.fstart));
  e = TileRoundEngine{};
}

void TileRoundLaunch::bind() {
  void *a[8] = {&cells, &tab0, &fkey, &fcell, &bitmap, &tb, &ctl, &bt};
  memcpy(scan, a, sizeof a);
  void *b[2] = {&tb, &ctl};
  memcpy(prefix, b, sizeof b);
  memcpy(active, b, sizeof b);
  memcpy(sort, b, sizeof b);
  void *c[8] = {&cells, &tab0, &fkey_c, &fcell_c, &bitmap_c, &tb, &ctl, &bt};
  memcpy(claim, c, sizeof c);
  void *d[8] = {&cells, &tab0, &tb, &fkey, &fcell, &bitmap, &ctl, &bt};
  memcpy(apply, d, sizeof d);
  void *r[7] = {&cells, &tab0, &fkey_c, &fcell_c, &tb, &ctl, &bt};
  memcpy(restore, r, sizeof r);
  void *x[4] = {&ctl, &st, &set_cond, &cond};
  memcpy(end, x, sizeof x);
}

void tre_launch_args(TileRoundLaunch &a, const TileRoundEngine &e, Cell *cells, const TableArgs &tab0, u64 *fkey,
                     u32 *fcell, u32 *bitmap, DecodeCtl *ctl, const RoundStats &st, const TRBatch &bt) {
  memset(&a, 0, sizeof a);
  a.cells = cells;
  a.tab0 = tab0;
  a.fkey = fkey;
  a.fcell = fcell;
  a.bitmap = bitmap;
  a.fkey_c = fkey;
  a.fcell_c = fcell;
  a.bitmap_c = bitmap;
  a.tb = e.trb;
  a.ctl = ctl;
  a.bt = bt;
  a.st = st;
  a.bind();
}

pp_status tre_build_graph(const TileRoundEngine &e, const IbltKernels &k, TileRoundLaunch &a, cudaGraphExec_t *exec,
                          bool prescanned) {
  *exec = nullptr;
  cudaGraph_t g = nullptr;
  PP_CUDA(cudaGraphCreate(&g, 0));
  pp_status st = PP_OK;
  cudaGraphNode_t n_scan, n_pre, n_cond, n_claim, n_sort, n_act, n_apply[2], n_end, n_restore;
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams cp{};
  cudaGraph_t body;
  st = tre_node(&n_scan, g, nullptr, 0, prescanned ? k.trescan : k.tscan, e.grid_tscan, kTRThreads, 0, a.scan);
  if (st != PP_OK) goto done;
  st = tre_node(&n_pre, g, &n_scan, 1, (const void *)k_tprefix, 1, 1024, 0, a.prefix);
  if (st != PP_OK) goto done;
  if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    st = fail(PP_ERR_CUDA, "cudaGraphConditionalHandleCreate failed");
    goto done;
  }
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (cudaGraphAddNode(&n_cond, g, &n_pre, nullptr, 1, &cp) != cudaSuccess) {
    st = fail(PP_ERR_CUDA, "cudaGraphAddNode(conditional while) failed");
    goto done;
  }
  body = cp.conditional.phGraph_out[0];
  // one block per frontier segment
  st = tre_node(&n_restore, g, &n_cond, 1, k.trestore, e.grid_tapply + e.grid_tsparse, kBlock, 0, a.restore);
  if (st != PP_OK) goto done;
  a.set_cond = 1;
  a.cond = h;
  st = tre_node(&n_claim, body, nullptr, 0, k.tclaim, e.grid_tclaim, kTClaimThreads, e.smem_tclaim, a.claim);
  if (st != PP_OK) goto done;
  st = tre_node(&n_sort, body, &n_claim, 1, (const void *)k_tsort, e.grid_tsort, kTSortThreads, e.smem_tsort,
                a.sort);
  if (st != PP_OK) goto done;
  st = tre_node(&n_act, body, &n_sort, 1, (const void *)k_tactive, e.grid_act, kBlock, 0, a.active);
  if (st != PP_OK) goto done;
  // dense and sparse tiles in two kernels that may run side by side
  st = tre_node(&n_apply[0], body, &n_act, 1, k.tapply, e.grid_tapply, kTRThreads, kTApplySmem, a.apply);
  if (st != PP_OK) goto done;
  st = tre_node(&n_apply[1], body, &n_act, 1, k.tapply_sparse, e.grid_tsparse, kTSThreads, kTSSmem, a.apply);
  if (st != PP_OK) goto done;
  st = tre_node(&n_end, body, n_apply, 2, (const void *)k_round_end, 1, 32, 0, a.end);
  if (st != PP_OK) goto done;
  if (cudaGraphInstantiate(exec, g, 0) != cudaSuccess) {
    st = fail(PP_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(cudaGetLastError()));
    *exec = nullptr;
  }
done:
  cudaGraphDestroy(g);
  return st;
}

pp_status tre_host_loop(const TileRoundEngine &e, const IbltKernels &k, TileRoundLaunch &a, u32 *h_more,
                        cudaStream_t s, bool prescanned) {
  a.set_cond = 0;
  PP_CUDA(cudaLaunchKernel(prescanned ? k.trescan : k.tscan, dim3(e.grid_tscan), dim3(kTRThreads), a.scan, 0, s));
  PP_CUDA(cudaLaunchKernel((const void *)k_tprefix, dim3(1), dim3(1024), a.prefix, 0, s));
  for (;;) {
    PP_CUDA(cudaLaunchKernel(k.tclaim, dim3(e.grid_tclaim), dim3(kTClaimThreads), a.claim, e.smem_tclaim, s));
    PP_CUDA(cudaLaunchKernel((const void *)k_tsort, dim3(e.grid_tsort), dim3(kTSortThreads), a.sort,
                             e.smem_tsort, s));
    PP_CUDA(cudaLaunchKernel((const void *)k_tactive, dim3(e.grid_act), dim3(kBlock), a.active, 0, s));
    PP_CUDA(cudaLaunchKernel(k.tapply, dim3(e.grid_tapply), dim3(kTRThreads), a.apply, kTApplySmem, s));
    PP_CUDA(cudaLaunchKernel(k.tapply_sparse, dim3(e.grid_tsparse), dim3(kTSThreads), a.apply, kTSSmem, s));
    PP_CUDA(cudaLaunchKernel((const void *)k_round_end, dim3(1), dim3(32), a.end, 0, s));
    PP_CUDA(cudaMemcpyAsync(h_more, &a.ctl->more, sizeof(u32), cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
    if (!*h_more) break;
  }
  PP_CUDA(cudaLaunchKernel(k.trestore, dim3(e.grid_tapply + e.grid_tsparse), dim3(kBlock), a.restore, 0, s));
  return PP_OK;
}

}  // namespace pp

struct pp_iblt {
  uint64_t n = 0;
  uint32_t r = 0;
  uint64_t seed = 0;
  pp_options opt{};
  TableArgs args{};
  Cell *cells = nullptr;
  u64 *fkey = nullptr;
  u32 *fcell = nullptr, *cand = nullptr, *bitmap = nullptr;
  DecodeCtl *ctl = nullptr, *h_ctl = nullptr;
  u64 *st_rec = nullptr, *st_alive = nullptr;
  u32 *st_front = nullptr;
  u64 *h_rec = nullptr, *h_alive = nullptr;
  int64_t items = 0;
  IbltKernels k{};
  int grid_scan = 0, grid_peel = 0, grid_filter = 0, grid_insert = 0, grid_bin = 0;
  size_t smem_peel = 0, smem_bin = 0;
  cudaGraphExec_t exec = nullptr;
  cudaGraphExec_t exec_pre = nullptr;  // tile rounds after a build that found F_1
  uint32_t graph_gen_pre = 0;
  // update records shared by the slab-binned build and the binned decode
  // rounds (allocated on first use, grown as needed)
  uint32_t n_slabs = 0;
  u64 *rec_key = nullptr;
  u32 *rec_cell = nullptr, *bin_count = nullptr, *bin_overflow = nullptr;
  uint64_t rec_cap_total = 0;
  uint32_t count_cap = 0;
  uint32_t rec_gen = 0;    // bumped whenever the record or count buffers move
  uint32_t graph_gen = 0;  // rec_gen the instantiated graph was built with
  // binned decode rounds
  bool binned_rounds = false;
  uint32_t n_bins = 0, bin_cap = 0, bin_shift = 0;
  size_t smem_claim = 0, smem_apply_round = 0;
  int grid_claim = 0, grid_apply_round = 0;
  TileBufs tiles;  // tile pass of the binned build (allocated on first use)
  // decode with sub-tables (allocated on first use)
  SubDecCtl *sctl = nullptr, *h_sctl = nullptr;
  u32 *squeue = nullptr;  // the per-sub-table queues (n entries)
  cudaGraphExec_t sub_exec = nullptr, sub_exec_binned = nullptr;
  uint32_t sub_graph_gen = 0;
  int grid_sscan = 0, grid_sfilter = 0, grid_speel = 0, grid_sdist = 0;
  // signed decode (allocated on first use)
  signed char *fsign = nullptr;
  u32 *sg_cand = nullptr;  // r pushes per recovered key at most: r * n entries
  cudaGraphExec_t sg_exec = nullptr;
  int grid_sgscan = 0, grid_sgpeel = 0, grid_sgfilter = 0, grid_sgclaim = 0;
  size_t smem_sgclaim = 0;
  signed char *sg_graph_out = nullptr;  // output sign pointer the graph was built with
  // tile rounds (allocated on first use)
  TileRoundEngine tre;        // tile rounds (buffers allocated on first use)
  bool tile_rounds = false;   // the round kind the graph was built with
  bool has_deletes = false;   // a deletion since the last clear/build: no tile rounds
  uint64_t front_cap = 0;     // entries of fkey / fcell
  // host-buffer jobs: at most two in flight
  HostJob jobs[kHostJobs];
  cudaStream_t up_s = nullptr, down_s = nullptr;  // uploads and downloads: one copy engine each
  u32 *h_flag = nullptr, *d_flag = nullptr;       // mapped pinned word: the build's overflow flag
  uint64_t next_ticket = 1;
  bool sg_graph_built = false;
  bool sg_graph_binned = false;         // the graph's round kind
  uint32_t sg_graph_gen = 0;            // rec_gen the binned graph was built with
};

namespace {

void free_all(pp_iblt *t) {
  if (!t) return;
  if (t->exec) cudaGraphExecDestroy(t->exec);
  if (t->exec_pre) cudaGraphExecDestroy(t->exec_pre);
  if (t->sub_exec) cudaGraphExecDestroy(t->sub_exec);
  if (t->sub_exec_binned) cudaGraphExecDestroy(t->sub_exec_binned);
  cudaFree(t->squeue);
  if (t->sg_exec) cudaGraphExecDestroy(t->sg_exec);
  cudaFree(t->fsign);
  cudaFree(t->sg_cand);
  cudaFree(t->sctl);
  cudaFreeHost(t->h_sctl);
  cudaFree(t->cells);
  cudaFree(t->fkey);
  cudaFree(t->fcell);
  cudaFree(t->cand);
  cudaFree(t->bitmap);
  cudaFree(t->ctl);
  cudaFree(t->st_rec);
  cudaFree(t->st_alive);
  cudaFree(t->st_front);
  cudaFreeHost(t->h_ctl);
  cudaFreeHost(t->h_rec);
  cudaFreeHost(t->h_alive);
  cudaFree(t->rec_key);
  cudaFree(t->rec_cell);
  cudaFree(t->bin_count);
  cudaFree(t->bin_overflow);
  free_tiles(t->tiles);
  for (HostJob &j : t->jobs) {
    cudaFree(j.d_keys);
    cudaFree(j.d_out);
    cudaFreeHost(j.h_ctl);
    cudaFreeHost(j.h_stats);
    cudaFreeHost(j.h_flag);
    if (j.built) cudaEventDestroy(j.built);
    if (j.up) cudaEventDestroy(j.up);
    if (j.dec) cudaEventDestroy(j.dec);
    if (j.done) cudaEventDestroy(j.done);
    if (j.reg_keys) cudaHostUnregister(const_cast<uint64_t *>(j.h_keys));
    if (j.reg_out) cudaHostUnregister(j.h_out);
  }
  cudaFreeHost(t->h_flag);
  if (t->up_s) cudaStreamDestroy(t->up_s);
  if (t->down_s) cudaStreamDestroy(t->down_s);
  tre_free(t->tre);
  delete t;
}

struct ScanArgs {
  Cell *cells;
  TableArgs tab0;
  const TableArgs *tabs;
  const Chunk *chunks;
  u32 n_chunks;
  u64 *fkey;
  u32 *fcell;
  u32 *ftab;
  u32 *bitmap;
  DecodeCtl *ctl;
  BatchCounters bc;
  void *p[11];
  void bind() {
    void *q[11] = {&cells, &tab0, &tabs, &chunks, &n_chunks, &fkey, &fcell, &ftab, &bitmap, &ctl, &bc};
    memcpy(p, q, sizeof q);
  }
};

struct PeelArgs {
  Cell *cells;
  TableArgs tab0;
  const TableArgs *tabs;
  const u64 *fkey;
  const u32 *fcell;
  const u32 *ftab;
  const u32 *bitmap;
  u32 *cand;
  u32 *ctab;
  u64 *bout;
  DecodeCtl *ctl;
  BatchCounters bc;
  void *p[12];
  void bind() {
    void *q[12] = {&cells, &tab0, &tabs, &fkey, &fcell, &ftab, &bitmap, &cand, &ctab, &bout, &ctl, &bc};
    memcpy(p, q, sizeof q);
  }
};

struct FilterArgs {
  const Cell *cells;
  TableArgs tab0;
  const TableArgs *tabs;
  const u32 *cand;
  const u32 *ctab;
  u64 *fkey;
  u32 *fcell;
  u32 *ftab;
  u32 *bitmap;
  DecodeCtl *ctl;
  BatchCounters bc;
  void *p[11];
  void bind() {
    void *q[11] = {&cells, &tab0, &tabs, &cand, &ctab, &fkey, &fcell, &ftab, &bitmap, &ctl, &bc};
    memcpy(p, q, sizeof q);
  }
};

struct EndArgs {
  DecodeCtl *ctl;
  RoundStats st;
  int set_cond;
  cudaGraphConditionalHandle cond;
  void *p[4];
  void bind() {
    void *q[4] = {&ctl, &st, &set_cond, &cond};
    memcpy(p, q, sizeof q);
  }
};

struct ClaimArgs {
  Cell *cells;
  TableArgs tab0;
  const TableArgs *tabs;
  const u64 *fkey;
  const u32 *fcell, *ftab, *bitmap;
  RoundBins rb;
  u32 *cand, *ctab;
  u64 *bout;
  DecodeCtl *ctl;
  BatchCounters bc;
  void *p[13];
  void bind() {
    void *q[13] = {&cells, &tab0, &tabs, &fkey, &fcell, &ftab, &bitmap, &rb, &cand, &ctab, &bout, &ctl, &bc};
    memcpy(p, q, sizeof q);
  }
};

struct ApplyRArgs {
  Cell *cells;
  TableArgs tab0;
  const TableArgs *tabs;
  RoundBins rb;
  u32 *cand, *ctab;
  DecodeCtl *ctl;
  BatchCounters bc;
  void *p[8];
  void bind() {
    void *q[8] = {&cells, &tab0, &tabs, &rb, &cand, &ctab, &ctl, &bc};
    memcpy(p, q, sizeof q);
  }
};

struct ResetArgs {
  RoundBins rb;
  DecodeCtl *ctl;
  void *p[2];
  void bind() {
    void *q[2] = {&rb, &ctl};
    memcpy(p, q, sizeof q);
  }
};

void fill_round_args(pp_iblt *t, ClaimArgs &ca, ApplyRArgs &aa, ResetArgs &ra) {
  BatchCounters bc{};
  RoundBins rb{t->rec_key, t->rec_cell, nullptr, t->bin_count, t->bin_cap, t->n_bins, t->bin_shift, 0};
  ca = ClaimArgs{t->cells, t->args, nullptr, t->fkey, t->fcell, nullptr, t->bitmap, rb, t->cand, nullptr,
                 nullptr, t->ctl, bc, {}};
  aa = ApplyRArgs{t->cells, t->args, nullptr, rb, t->cand, nullptr, t->ctl, bc, {}};
  ra = ResetArgs{rb, t->ctl, {}};
  ca.bind();
  aa.bind();
  ra.bind();
}

void fill_args(pp_iblt *t, ScanArgs &sa, PeelArgs &pa, FilterArgs &fa, EndArgs &ea) {
  BatchCounters bc{};
  sa = ScanArgs{t->cells, t->args, nullptr, nullptr,
                (u32)((t->n + kBlock * kScanItems - 1) / (kBlock * kScanItems)),
                t->fkey, t->fcell, nullptr, t->bitmap, t->ctl, bc, {}};
  pa = PeelArgs{t->cells, t->args, nullptr, t->fkey, t->fcell, nullptr, t->bitmap, t->cand,
                nullptr, nullptr, t->ctl, bc, {}};
  fa = FilterArgs{t->cells, t->args, nullptr, t->cand, nullptr, t->fkey, t->fcell, nullptr,
                  t->bitmap, t->ctl, bc, {}};
  ea = EndArgs{t->ctl, RoundStats{t->st_rec, t->st_alive, t->st_front}, 0, 0, {}};
  sa.bind();
  pa.bind();
  fa.bind();
  ea.bind();
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

// scan -> while (more) { peel -> filter -> round_end }
pp_status build_graph(pp_iblt *t) {
  ScanArgs sa;
  PeelArgs pa;
  FilterArgs fa;
  EndArgs ea;
  ClaimArgs ca;
  ApplyRArgs aa;
  ResetArgs ra;
  fill_args(t, sa, pa, fa, ea);
  if (t->binned_rounds) fill_round_args(t, ca, aa, ra);
  cudaGraph_t g = nullptr;
  PP_CUDA(cudaGraphCreate(&g, 0));
  pp_status st = PP_OK;
  cudaGraphNode_t n_scan, n_cond, n_peel, n_filter, n_end;
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams cp{};
  cudaGraph_t body;
  st = add_kernel(&n_scan, g, nullptr, 0, t->k.scan, t->grid_scan, kBlock, 0, sa.p);
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
  ea.set_cond = 1;
  ea.cond = h;
  if (t->binned_rounds) {
    // claim -> apply (binned) -> filter -> reset bins -> round end
    cudaGraphNode_t n_apply, n_reset;
    st = add_kernel(&n_peel, body, nullptr, 0, t->k.claim, t->grid_claim, kBlock, t->smem_claim, ca.p);
    if (st != PP_OK) goto done;
    st = add_kernel(&n_apply, body, &n_peel, 1, t->k.apply_round, t->grid_apply_round, kBlock,
                    t->smem_apply_round, aa.p);
    if (st != PP_OK) goto done;
    st = add_kernel(&n_filter, body, &n_apply, 1, t->k.filter, t->grid_filter, kBlock, 0, fa.p);
    if (st != PP_OK) goto done;
    st = add_kernel(&n_reset, body, &n_filter, 1, (const void *)k_bins_reset, 1, 256, 0, ra.p);
    if (st != PP_OK) goto done;
    st = add_kernel(&n_end, body, &n_reset, 1, (const void *)k_round_end, 1, 32, 0, ea.p);
    if (st != PP_OK) goto done;
  } else {
    st = add_kernel(&n_peel, body, nullptr, 0, t->k.peel, t->grid_peel, kBlock, t->smem_peel, pa.p);
    if (st != PP_OK) goto done;
    st = add_kernel(&n_filter, body, &n_peel, 1, t->k.filter, t->grid_filter, kBlock, 0, fa.p);
    if (st != PP_OK) goto done;
    st = add_kernel(&n_end, body, &n_filter, 1, (const void *)k_round_end, 1, 32, 0, ea.p);
    if (st != PP_OK) goto done;
  }
  // PPEEL_GRAPH_DOT=<path>: write the decode graph in DOT format (debugging aid)
  if (const char *dot = getenv("PPEEL_GRAPH_DOT")) cudaGraphDebugDotPrint(g, dot, cudaGraphDebugDotFlagsVerbose);
  if (cudaGraphInstantiate(&t->exec, g, 0) != cudaSuccess) {
    st = fail(PP_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(cudaGetLastError()));
    t->exec = nullptr;
  }
  t->graph_gen = t->rec_gen;
done:
  cudaGraphDestroy(g);
  return st;
}

// ---- decode with sub-tables ----------------------------------------------
// Plain:  sscan -> while (more) { sfilter -> speel -> send }
// Binned (tables of 2^21 cells or more, as the full-round decode):
//         sscan -> while (more) { sfilter -> claim without the claim check ->
//                                 apply_round -> sdistribute -> send_binned }
struct SubArgs {
  // k_sscan
  const Cell *cells_c;
  TableArgs tab;
  u32 *queue;
  SubDecCtl *ctl;
  void *scan[4];
  // k_sfilter
  u64 *fkey;
  u32 *fcell;
  u32 *front_count;
  void *filter[7];
  // k_speel
  Cell *cells;
  void *peel[6];
  // k_send / k_send_binned
  u64 *st_rec;
  int set_cond;
  cudaGraphConditionalHandle cond;
  void *end[4];
  // binned: k_sdistribute, k_send_binned (claim and apply take ClaimArgs / ApplyRArgs)
  const u32 *cand_c;
  DecodeCtl *rctl;
  const DecodeCtl *rctl_c;
  RoundBins rb;
  void *dist[5];
  void *end_b[6];
  void bind() {
    void *a[4] = {&cells_c, &tab, &queue, &ctl};
    memcpy(scan, a, sizeof a);
    void *b[7] = {&cells_c, &tab, &queue, &fkey, &fcell, &ctl, &front_count};
    memcpy(filter, b, sizeof b);
    void *c[6] = {&cells, &tab, &fkey, &fcell, &queue, &ctl};
    memcpy(peel, c, sizeof c);
    void *d[4] = {&ctl, &st_rec, &set_cond, &cond};
    memcpy(end, d, sizeof d);
    void *e[5] = {&tab, &cand_c, &rctl_c, &queue, &ctl};
    memcpy(dist, e, sizeof e);
    void *f[6] = {&ctl, &rctl, &rb, &st_rec, &set_cond, &cond};
    memcpy(end_b, f, sizeof f);
  }
};

void fill_sub_args(pp_iblt *t, SubArgs &a, bool binned) {
  a.cells_c = t->cells;
  a.tab = t->args;
  a.queue = t->squeue;
  a.ctl = t->sctl;
  a.fkey = t->fkey;
  a.fcell = t->fcell;
  a.front_count = binned ? &t->ctl->n_front : &t->sctl->n_front;
  a.cells = t->cells;
  a.st_rec = t->st_rec;
  a.set_cond = 0;
  a.cond = 0;
  a.cand_c = t->cand;
  a.rctl = t->ctl;
  a.rctl_c = t->ctl;
  a.rb = RoundBins{t->rec_key, t->rec_cell, nullptr, t->bin_count, t->bin_cap, t->n_bins, t->bin_shift, 0};
  a.bind();
}

pp_status sub_prepare(pp_iblt *t) {
  if (!t->k.sub_scan) return fail(PP_ERR_INVALID_ARG, "decode with sub-tables: no kernels for r=%u", t->r);
  if (!t->sctl) {
    PP_CUDA(cudaMalloc((void **)&t->sctl, sizeof(SubDecCtl)));
    PP_CUDA(cudaMallocHost((void **)&t->h_sctl, sizeof(SubDecCtl)));
    PP_CUDA(cudaMalloc((void **)&t->squeue, t->n * sizeof(u32)));
    t->grid_sscan = persistent_grid(t->k.sub_scan, kBlock, 0, t->opt.ctas_per_sm);
    t->grid_sfilter = persistent_grid(t->k.sub_filter, kBlock, 0, t->opt.ctas_per_sm);
    t->grid_speel = persistent_grid(t->k.sub_peel, kBlock, 0, t->opt.ctas_per_sm);
    t->grid_sdist = persistent_grid((const void *)k_sdistribute, kBlock, 0, t->opt.ctas_per_sm);
  }
  return PP_OK;
}

pp_status sub_host_loop(pp_iblt *t, bool binned, cudaStream_t s) {
  SubArgs a;
  fill_sub_args(t, a, binned);
  ClaimArgs ca;
  ApplyRArgs aa;
  ResetArgs ra;
  if (binned) fill_round_args(t, ca, aa, ra);
  PP_CUDA(cudaLaunchKernel(t->k.sub_scan, dim3(t->grid_sscan), dim3(kBlock), a.scan, 0, s));
  for (;;) {
    PP_CUDA(cudaLaunchKernel(t->k.sub_filter, dim3(t->grid_sfilter), dim3(kBlock), a.filter, 0, s));
    if (binned) {
      PP_CUDA(cudaLaunchKernel(t->k.sub_claim, dim3(t->grid_claim), dim3(kBlock), ca.p, t->smem_claim, s));
      PP_CUDA(cudaLaunchKernel(t->k.apply_round, dim3(t->grid_apply_round), dim3(kBlock), aa.p,
                               t->smem_apply_round, s));
      PP_CUDA(cudaLaunchKernel((const void *)k_sdistribute, dim3(t->grid_sdist), dim3(kBlock), a.dist, 0, s));
      PP_CUDA(cudaLaunchKernel((const void *)k_send_binned, dim3(1), dim3(32), a.end_b, 0, s));
    } else {
      PP_CUDA(cudaLaunchKernel(t->k.sub_peel, dim3(t->grid_speel), dim3(kBlock), a.peel, 0, s));
      PP_CUDA(cudaLaunchKernel((const void *)k_send, dim3(1), dim3(32), a.end, 0, s));
    }
    PP_CUDA(cudaMemcpyAsync(&t->h_sctl->more, &t->sctl->more, sizeof(u32), cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
    if (!t->h_sctl->more) break;
  }
  return PP_OK;
}

// Every pointer the plain graph holds lives as long as the handle, so it is
// built once; the binned one also holds the record buffers and is rebuilt
// when they move.
pp_status sub_graph_launch(pp_iblt *t, bool binned, cudaStream_t s) {
  cudaGraphExec_t &exec = binned ? t->sub_exec_binned : t->sub_exec;
  if (binned && exec && t->sub_graph_gen != t->rec_gen) {
    cudaGraphExecDestroy(exec);
    exec = nullptr;
  }
  if (!exec) {
    SubArgs a;
    fill_sub_args(t, a, binned);
    ClaimArgs ca;
    ApplyRArgs aa;
    ResetArgs ra;
    if (binned) fill_round_args(t, ca, aa, ra);
    cudaGraph_t g = nullptr;
    PP_CUDA(cudaGraphCreate(&g, 0));
    pp_status st = PP_OK;
    cudaGraphNode_t n_scan, n_cond, n_filter, n_peel, n_apply, n_dist, n_end;
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams cp{};
    cudaGraph_t body;
    st = add_kernel(&n_scan, g, nullptr, 0, t->k.sub_scan, t->grid_sscan, kBlock, 0, a.scan);
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
    st = add_kernel(&n_filter, body, nullptr, 0, t->k.sub_filter, t->grid_sfilter, kBlock, 0, a.filter);
    if (st != PP_OK) goto done;
    if (binned) {
      st = add_kernel(&n_peel, body, &n_filter, 1, t->k.sub_claim, t->grid_claim, kBlock, t->smem_claim, ca.p);
      if (st != PP_OK) goto done;
      st = add_kernel(&n_apply, body, &n_peel, 1, t->k.apply_round, t->grid_apply_round, kBlock,
                      t->smem_apply_round, aa.p);
      if (st != PP_OK) goto done;
      st = add_kernel(&n_dist, body, &n_apply, 1, (const void *)k_sdistribute, t->grid_sdist, kBlock, 0, a.dist);
      if (st != PP_OK) goto done;
      st = add_kernel(&n_end, body, &n_dist, 1, (const void *)k_send_binned, 1, 32, 0, a.end_b);
      if (st != PP_OK) goto done;
    } else {
      st = add_kernel(&n_peel, body, &n_filter, 1, t->k.sub_peel, t->grid_speel, kBlock, 0, a.peel);
      if (st != PP_OK) goto done;
      st = add_kernel(&n_end, body, &n_peel, 1, (const void *)k_send, 1, 32, 0, a.end);
      if (st != PP_OK) goto done;
    }
    if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) {
      st = fail(PP_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(cudaGetLastError()));
      exec = nullptr;
    }
    if (binned) t->sub_graph_gen = t->rec_gen;
  done:
    cudaGraphDestroy(g);
    if (st != PP_OK) return st;
  }
  PP_CUDA(cudaGraphLaunch(exec, s));
  return PP_OK;
}

// ---- tile rounds ---------------------------------------------------------
// Buffers: a record region per tile (its counts' sum, rounded up to
// kTRAlign), r * items + kTRAlign * tiles records in all.
pp_status ensure_tile_rounds(pp_iblt *t, cudaStream_t s) {
  if (!t->tre.trb.base) {
    pp_status st = tre_setup(t->tre, t->k, t->n, t->opt.ctas_per_sm);
    if (st != PP_OK) return st;
    ++t->rec_gen;
    // the frontier arrays hold every segment
    if (t->tre.front > t->front_cap) {
      PP_CUDA(cudaStreamSynchronize(s));
      cudaFree(t->fkey);
      cudaFree(t->fcell);
      t->fkey = nullptr;
      t->fcell = nullptr;
      PP_CUDA(cudaMalloc((void **)&t->fkey, t->tre.front * sizeof(u64)));
      PP_CUDA(cudaMalloc((void **)&t->fcell, t->tre.front * sizeof(u32)));
      t->front_cap = t->tre.front;
      // every graph holds the frontier pointers
      if (t->sub_exec) cudaGraphExecDestroy(t->sub_exec);
      if (t->sub_exec_binned) cudaGraphExecDestroy(t->sub_exec_binned);
      if (t->sg_exec) cudaGraphExecDestroy(t->sg_exec);
      t->sub_exec = t->sub_exec_binned = t->sg_exec = nullptr;
    }
  }
  const uint64_t items = t->items > 0 ? (uint64_t)t->items : 0;
  bool moved = false;
  pp_status st = tre_records(t->tre, tre_record_need(t->tre, (uint64_t)t->r * items), s, &moved);
  if (moved) ++t->rec_gen;
  return st;
}

void fill_tile_args(pp_iblt *t, TileRoundLaunch &a) {
  tre_launch_args(a, t->tre, t->cells, t->args, t->fkey, t->fcell, t->bitmap, t->ctl,
                  RoundStats{t->st_rec, t->st_alive, t->st_front}, TRBatch{});
}

pp_status build_tile_graph(pp_iblt *t) {
  TileRoundLaunch a;
  fill_tile_args(t, a);
  pp_status st = tre_build_graph(t->tre, t->k, a, &t->exec);
  if (st == PP_OK) t->graph_gen = t->rec_gen;
  return st;
}

// The tile rounds after a build that found F_1 (k_trescan instead of the scan):
// their own graph, kept beside the plain decode's.
pp_status launch_prescanned_rounds(pp_iblt *t, cudaStream_t s) {
  TileRoundLaunch a;
  fill_tile_args(t, a);
  if (t->opt.host_loop) return tre_host_loop(t->tre, t->k, a, &t->h_ctl->more, s, true);
  if (t->exec_pre && t->graph_gen_pre != t->rec_gen) {
    cudaGraphExecDestroy(t->exec_pre);
    t->exec_pre = nullptr;
  }
  if (!t->exec_pre) {
    pp_status st = tre_build_graph(t->tre, t->k, a, &t->exec_pre, true);
    if (st != PP_OK) return st;
    t->graph_gen_pre = t->rec_gen;
  }
  PP_CUDA(cudaGraphLaunch(t->exec_pre, s));
  return PP_OK;
}

pp_status run_tile_host_loop(pp_iblt *t, cudaStream_t s) {
  TileRoundLaunch a;
  fill_tile_args(t, a);
  return tre_host_loop(t->tre, t->k, a, &t->h_ctl->more, s);
}

pp_status run_host_loop(pp_iblt *t, cudaStream_t s) {
  ScanArgs sa;
  PeelArgs pa;
  FilterArgs fa;
  EndArgs ea;
  fill_args(t, sa, pa, fa, ea);
  ClaimArgs ca;
  ApplyRArgs aa;
  ResetArgs ra;
  if (t->binned_rounds) fill_round_args(t, ca, aa, ra);
  PP_CUDA(cudaLaunchKernel(t->k.scan, dim3(t->grid_scan), dim3(kBlock), sa.p, 0, s));
  for (;;) {
    if (t->binned_rounds) {
      PP_CUDA(cudaLaunchKernel(t->k.claim, dim3(t->grid_claim), dim3(kBlock), ca.p, t->smem_claim, s));
      PP_CUDA(cudaLaunchKernel(t->k.apply_round, dim3(t->grid_apply_round), dim3(kBlock), aa.p,
                               t->smem_apply_round, s));
      PP_CUDA(cudaLaunchKernel(t->k.filter, dim3(t->grid_filter), dim3(kBlock), fa.p, 0, s));
      PP_CUDA(cudaLaunchKernel((const void *)k_bins_reset, dim3(1), dim3(256), ra.p, 0, s));
    } else {
      PP_CUDA(cudaLaunchKernel(t->k.peel, dim3(t->grid_peel), dim3(kBlock), pa.p, t->smem_peel, s));
      PP_CUDA(cudaLaunchKernel(t->k.filter, dim3(t->grid_filter), dim3(kBlock), fa.p, 0, s));
    }
    PP_CUDA(cudaLaunchKernel((const void *)k_round_end, dim3(1), dim3(32), ea.p, 0, s));
    PP_CUDA(cudaMemcpyAsync(&t->h_ctl->more, &t->ctl->more, sizeof(u32), cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
    if (!t->h_ctl->more) break;
  }
  return PP_OK;
}

pp_status launch_insert(pp_iblt *t, const uint64_t *d_keys, uint64_t m, int sign, cudaStream_t s) {
  if (m == 0) return PP_OK;
  TableArgs a = t->args;
  const TableArgs *tabs = nullptr;
  const Chunk *chunks = nullptr;
  u32 nch = 0;
  Cell *cells = t->cells;
  const u64 *keys = reinterpret_cast<const u64 *>(d_keys);
  u64 mm = m;
  void *args[] = {&cells, &a, &tabs, &chunks, &nch, &keys, &mm, &sign};
  const u64 want = (m + kBlock - 1) / kBlock;
  const int grid = (int)(want < (u64)t->grid_insert ? want : (u64)t->grid_insert);
  PP_CUDA(cudaLaunchKernel(t->k.insert, dim3(grid), dim3(kBlock), args, 0, s));
  return PP_OK;
}

bool use_binned(const pp_iblt *t, uint64_t m) {
  if (m == 0 || t->opt.binned == 2) return false;
  if (t->opt.binned == 1) return true;
  return t->n >= (1ull << 23) && m * t->r >= t->n / 4;
}

// Grows the shared update-record buffers to `records` entries and the count
// array to `counts` entries (synchronizes `s` when it reallocates).
pp_status ensure_records(pp_iblt *t, uint64_t records, uint32_t counts, cudaStream_t s) {
  if (records > t->rec_cap_total) {
    PP_CUDA(cudaStreamSynchronize(s));
    cudaFree(t->rec_key);
    cudaFree(t->rec_cell);
    t->rec_key = nullptr;
    t->rec_cell = nullptr;
    t->rec_cap_total = 0;
    PP_CUDA(cudaMalloc((void **)&t->rec_key, records * sizeof(u64)));
    PP_CUDA(cudaMalloc((void **)&t->rec_cell, records * sizeof(u32)));
    t->rec_cap_total = records;
    ++t->rec_gen;
  }
  if (counts > t->count_cap || !t->bin_overflow) {
    PP_CUDA(cudaStreamSynchronize(s));
    cudaFree(t->bin_count);
    cudaFree(t->bin_overflow);
    t->bin_count = nullptr;
    t->bin_overflow = nullptr;
    t->count_cap = 0;
    PP_CUDA(cudaMalloc((void **)&t->bin_count, (counts ? counts : 1) * sizeof(u32)));
    PP_CUDA(cudaMalloc((void **)&t->bin_overflow, sizeof(u32)));
    t->count_cap = counts;
    ++t->rec_gen;
  }
  return PP_OK;
}

// Record capacity of one slab's list for a binned update of m keys: the
// updates are uniform over the cells, so the expected count plus slack.
uint64_t slab_record_cap(uint64_t n, uint32_t r, uint64_t m) {
  const double per = (double)m * r * ((double)kSlabCells / (double)n);
  return (uint64_t)(per * 1.05) + 4096;
}

// Bins of the binned decode rounds: count, capacity per bin (records), shift.
void round_bin_layout(uint64_t n, uint32_t r, uint32_t *nb, uint64_t *cap, u32 *shift) {
  const u32 sh = round_bin_shift(n);
  const uint64_t span = n < (1ull << sh) ? n : (1ull << sh);
  *nb = (uint32_t)((n + (1ull << sh) - 1) >> sh);
  *cap = (uint64_t)((double)r * (double)span * 0.525) + 4096;
  *shift = sh;
}

// Pass 1 of a binned build: route every (cell, key) update into its slab's list.
pp_status bin_pass(pp_iblt *t, const uint64_t *d_keys, uint64_t m, int sign, int direct_overflow,
                   cudaStream_t s, BinArgs &ba) {
  const uint32_t ns = (uint32_t)((t->n + kSlabCells - 1) / kSlabCells);
  const uint64_t cap = slab_record_cap(t->n, t->r, m);
  if (cap > 0xFFFFFFF0ull) return fail(PP_ERR_INVALID_ARG, "pp_iblt_insert: too many keys for one call");
  pp_status st = ensure_records(t, cap * ns, ns, s);
  if (st != PP_OK) return st;
  if (ns != t->n_slabs) {
    t->n_slabs = ns;
    t->smem_bin = bin_smem_bytes(t->k.nr, false, ns);
    t->grid_bin = persistent_grid(t->k.bin, kBlock, t->smem_bin, t->opt.ctas_per_sm);
  }
  PP_CUDA(cudaMemsetAsync(t->bin_count, 0, ns * sizeof(u32), s));
  PP_CUDA(cudaMemsetAsync(t->bin_overflow, 0, sizeof(u32), s));
  ba = BinArgs{t->rec_key, t->rec_cell, nullptr, t->bin_count, t->bin_overflow, (u32)cap, ns, direct_overflow};
  TableArgs a = t->args;
  const TableArgs *tabs = nullptr;
  const Chunk *chunks = nullptr;
  u32 nch = 0;
  Cell *cells = t->cells;
  const u64 *keys = reinterpret_cast<const u64 *>(d_keys);
  u64 mm = m;
  void *args[] = {&cells, &a, &tabs, &chunks, &nch, &keys, &mm, &sign, &ba};
  const u64 items = (m + kBinKeys - 1) / kBinKeys;
  const int grid = (int)(items < (u64)t->grid_bin ? items : (u64)t->grid_bin);
  PP_CUDA(cudaLaunchKernel(t->k.bin, dim3(grid), dim3(kBlock), args, t->smem_bin, s));
  return PP_OK;
}

// Bins of the binned decode rounds: 2^19 cells each; a bin's list holds the
// updates of half its cells' worth of recovered keys (a round recovers far
// fewer; a fuller bin applies the excess directly).
pp_status ensure_round_bins(pp_iblt *t, cudaStream_t s) {
  uint32_t nb;
  uint64_t cap;
  u32 shift;
  round_bin_layout(t->n, t->r, &nb, &cap, &shift);
  pp_status st = ensure_records(t, cap * nb, nb, s);
  if (st != PP_OK) return st;
  t->n_bins = nb;
  t->bin_cap = (uint32_t)cap;
  t->bin_shift = shift;
  t->smem_claim = claim_smem_bytes(t->k.nr, false, nb);
  t->smem_apply_round = apply_round_smem_bytes(false, nb);
  t->grid_claim = persistent_grid(t->k.claim, kBlock, t->smem_claim, t->opt.ctas_per_sm);
  t->grid_apply_round = persistent_grid(t->k.apply_round, kBlock, t->smem_apply_round, t->opt.apply_ctas);
  return PP_OK;
}

// Pass 2: slab by slab (zero-filled first when building from scratch).
pp_status apply_pass(pp_iblt *t, BinArgs &ba, int sign, bool zero_fill, cudaStream_t s,
                     const PrescanArgs *pre = nullptr) {
  pp_status st = ensure_tiles(t->tiles, tile_cap_for(ba.cap), ba.cap, ba.n_slabs, false, s);
  if (st != PP_OK) return st;
  return tile_apply_pass(t->cells, t->args, nullptr, ba, t->tiles, t->n, sign, zero_fill, s, pre);
}

pp_status update(pp_iblt *t, const uint64_t *d_keys, uint64_t m, int sign, cudaStream_t s) {
  if (!use_binned(t, m)) return launch_insert(t, d_keys, m, sign, s);
  BinArgs ba;
  pp_status st = bin_pass(t, d_keys, m, sign, 1, s, ba);
  if (st != PP_OK) return st;
  return apply_pass(t, ba, sign, false, s);
}

}  // namespace

namespace {

// Enqueues a whole decode on s (control block set up, round loop launched);
// nothing is read back.
// Round kind: tile rounds (large tables built from insertions only), binned
// atomic rounds (other large tables), direct atomics (small tables).
bool want_tile_rounds(const pp_iblt *t) {
  const bool large = t->n >= (1ull << 21);
  return t->k.tscan && !t->has_deletes &&
         (t->opt.rounds == 2 || (t->opt.rounds == 0 && large && t->opt.binned != 2));
}

void set_host_ctl(pp_iblt *t, uint64_t *d_out_keys, uint64_t out_cap) {
  memset(t->h_ctl, 0, sizeof(DecodeCtl));
  t->h_ctl->out = reinterpret_cast<u64 *>(d_out_keys);
  t->h_ctl->out_cap = out_cap;
  t->h_ctl->max_rounds = t->opt.max_rounds;
}

pp_status decode_enqueue(pp_iblt *t, uint64_t *d_out_keys, uint64_t out_cap, cudaStream_t s) {
  set_host_ctl(t, d_out_keys, out_cap);
  const bool large = t->n >= (1ull << 21);
  const bool want_tiles = want_tile_rounds(t);
  const bool want_bins = !want_tiles && (t->opt.binned == 1 || (t->opt.binned == 0 && large));
  if (want_tiles) {
    pp_status st = ensure_tile_rounds(t, s);
    if (st != PP_OK) return st;
  }
  if (want_bins) {
    pp_status st = ensure_round_bins(t, s);
    if (st != PP_OK) return st;
    PP_CUDA(cudaMemsetAsync(t->bin_count, 0, t->n_bins * sizeof(u32), s));
  }
  // the graph holds buffer pointers: rebuild it when they moved or the round kind changed
  if (t->exec && (want_bins != t->binned_rounds || want_tiles != t->tile_rounds ||
                  ((want_bins || want_tiles) && t->graph_gen != t->rec_gen))) {
    cudaGraphExecDestroy(t->exec);
    t->exec = nullptr;
  }
  t->binned_rounds = want_bins;
  t->tile_rounds = want_tiles;
  k_ctl_init<<<1, 32, 0, s>>>(t->ctl, *t->h_ctl);
  PP_CUDA(cudaGetLastError());
  if (t->opt.host_loop) {
    pp_status st = want_tiles ? run_tile_host_loop(t, s) : run_host_loop(t, s);
    if (st != PP_OK) return st;
  } else {
    if (!t->exec) {
      pp_status st = want_tiles ? build_tile_graph(t) : build_graph(t);
      if (st != PP_OK) return st;
    }
    PP_CUDA(cudaGraphLaunch(t->exec, s));
  }
  return PP_OK;
}

pp_status ensure_flag(pp_iblt *t) {
  if (!t->h_flag) {
    PP_CUDA(cudaHostAlloc((void **)&t->h_flag, sizeof(u32), cudaHostAllocMapped | cudaHostAllocPortable));
    PP_CUDA(cudaHostGetDevicePointer((void **)&t->d_flag, t->h_flag, 0));
  }
  return PP_OK;
}

// Fills *res from the control block c after a decode and the first ncopy
// per-round statistics.
pp_status decode_collect(const DecodeCtl &c, const u64 *h_rec, const u64 *h_alive, uint32_t ncopy,
                         uint64_t items, uint64_t out_cap, pp_decode_result *res, uint32_t max_rounds,
                         const char *fn) {
  const uint32_t T = c.round;
  ncopy = ncopy < T ? ncopy : T;
  ncopy = ncopy < res->round_cap ? ncopy : res->round_cap;
  uint64_t left = items;
  for (uint32_t i = 0; i < ncopy; ++i) {
    left -= h_rec[i] <= left ? h_rec[i] : left;
    if (res->recovered_per_round) res->recovered_per_round[i] = h_rec[i];
    if (res->remaining_per_round) res->remaining_per_round[i] = left;
    if (res->alive_cells_per_round) res->alive_cells_per_round[i] = h_alive[i];
  }
  res->rounds = T;
  res->status_flags = c.flags;
  res->recovered = c.n_out < out_cap ? c.n_out : out_cap;
  res->items_before = items;
  res->residual_cells = c.nonempty - c.emptied;
  if (c.flags & FLAG_CAPACITY)
    return fail(PP_ERR_CAPACITY, "%s: more keys recovered than out_cap=%llu", fn, (unsigned long long)out_cap);
  if (c.flags & FLAG_INTERNAL)
    return fail(PP_ERR_INVALID_ARG,
                "%s: a pure cell's key does not hash to it, or the table holds a negative count", fn);
  if (c.flags & FLAG_ROUND_LIMIT)
    return fail(PP_ERR_ROUND_LIMIT, "%s: stopped after max_rounds=%u rounds", fn, max_rounds);
  return PP_OK;
}

// Reads a finished decode's control block and statistics back into *res.
pp_status decode_result(pp_iblt *t, uint64_t out_cap, pp_decode_result *res, cudaStream_t s, const char *fn) {
  const uint64_t items = t->items > 0 ? (uint64_t)t->items : 0;
  PP_CUDA(cudaMemcpyAsync(t->h_ctl, t->ctl, sizeof(DecodeCtl), cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaStreamSynchronize(s));
  const DecodeCtl c = *t->h_ctl;
  const uint32_t T = c.round;
  const uint32_t ncopy = T < res->round_cap ? T : res->round_cap;
  if (ncopy && (res->recovered_per_round || res->remaining_per_round || res->alive_cells_per_round)) {
    PP_CUDA(cudaMemcpyAsync(t->h_rec, t->st_rec, ncopy * sizeof(u64), cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaMemcpyAsync(t->h_alive, t->st_alive, ncopy * sizeof(u64), cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
  }
  pp_status st = decode_collect(c, t->h_rec, t->h_alive, ncopy, items, out_cap, res, t->opt.max_rounds, fn);
  t->items -= (int64_t)res->recovered;
  return st;
}

}  // namespace

extern "C" {

pp_status pp_iblt_create(pp_iblt **out, uint64_t n_cells, uint32_t r, uint64_t seed,
                         const pp_options *opt) {
  if (!out) return fail(PP_ERR_INVALID_ARG, "pp_iblt_create: out is NULL");
  *out = nullptr;
  if (r < 2 || r > PP_MAX_R)
    return fail(PP_ERR_INVALID_ARG, "pp_iblt_create: r=%u outside 2..%d", r, PP_MAX_R);
  if (n_cells < r || n_cells > 0xFFFFFFFFull - 64)
    return fail(PP_ERR_INVALID_ARG, "pp_iblt_create: n_cells=%llu outside r..2^32-65",
                (unsigned long long)n_cells);
  pp_iblt *t = new pp_iblt();
  t->n = n_cells;
  t->r = r;
  t->seed = seed;
  t->opt = resolve_options(opt);
  make_table_args(t->args, n_cells, r, seed, 0);
  t->k = iblt_kernels((int)r, false);
  t->smem_peel = peel_smem_bytes(t->k.nr, false);
  const uint64_t words = (n_cells + 31) / 32 + 1;
  const uint32_t mr = t->opt.max_rounds;
  cudaError_t e = cudaSuccess;
  auto al = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes ? bytes : 16);
  };
  al((void **)&t->cells, n_cells * sizeof(Cell));
  al((void **)&t->fkey, n_cells * sizeof(u64));
  t->front_cap = n_cells;
  al((void **)&t->fcell, n_cells * sizeof(u32));
  al((void **)&t->cand, n_cells * sizeof(u32));
  al((void **)&t->bitmap, words * sizeof(u32));
  al((void **)&t->ctl, sizeof(DecodeCtl));
  al((void **)&t->st_rec, (size_t)mr * sizeof(u64));
  al((void **)&t->st_alive, (size_t)mr * sizeof(u64));
  al((void **)&t->st_front, (size_t)mr * sizeof(u32));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&t->h_ctl, sizeof(DecodeCtl));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&t->h_rec, (size_t)mr * sizeof(u64));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&t->h_alive, (size_t)mr * sizeof(u64));
  if (e == cudaSuccess) e = cudaMemset(t->cells, 0, n_cells * sizeof(Cell));
  if (e == cudaSuccess) e = cudaMemset(t->bitmap, 0, words * sizeof(u32));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    pp_status st = cuda_fail(e, "pp_iblt_create allocation", __FILE__, __LINE__);
    free_all(t);
    return st;
  }
  // scattered 32-byte cell reads: one sector fetched from DRAM, not two
  if (t->opt.l2_fetch == 1) cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, 32);
  t->grid_scan = persistent_grid(t->k.scan, kBlock, 0, t->opt.ctas_per_sm);
  t->grid_peel = persistent_grid(t->k.peel, kBlock, t->smem_peel, t->opt.ctas_per_sm);
  t->grid_filter = persistent_grid(t->k.filter, kBlock, 0, t->opt.ctas_per_sm);
  t->grid_insert = persistent_grid(t->k.insert, kBlock, 0, 8) * 4;
  *out = t;
  return PP_OK;
}

pp_status pp_workspace_size(uint64_t n_cells, uint32_t r, uint64_t m_keys, const pp_options *opt,
                            uint64_t *table_bytes, uint64_t *fixed_bytes, uint64_t *peak_bytes) {
  if (r < 2 || r > PP_MAX_R || n_cells < r || n_cells > 0xFFFFFFFFull - 64)
    return fail(PP_ERR_INVALID_ARG, "pp_workspace_size: r=%u or n_cells=%llu out of range", r,
                (unsigned long long)n_cells);
  const pp_options o = resolve_options(opt);
  const uint64_t n = n_cells, mr = o.max_rounds;
  const uint64_t table = n * sizeof(Cell);
  const uint64_t fixed = n * (sizeof(u64) + 2 * sizeof(u32)) + ((n + 31) / 32 + 1) * sizeof(u32) +
                         sizeof(DecodeCtl) + mr * (2 * sizeof(u64) + sizeof(u32));
  // the update records are shared by binned builds and binned rounds: the larger need
  uint64_t records = 0, counts = 0, tiles = 0;
  const uint32_t ns = (uint32_t)((n + kSlabCells - 1) / kSlabCells);
  const bool build_binned = m_keys && o.binned != 2 && (o.binned == 1 || (n >= (1ull << 23) && m_keys * r >= n / 4));
  if (build_binned) {
    const uint64_t cap = slab_record_cap(n, r, m_keys);
    records = cap * ns;
    counts = ns;
    tiles = tile_pass_bytes(tile_cap_for(cap), cap, ns, false);
  }
  // decode rounds for a table of m_keys insertions: tile rounds (their own
  // record regions, r * m_keys + slack) or binned rounds (shared records)
  const bool rounds_tiles = o.rounds == 2 || (o.rounds == 0 && n >= (1ull << 21) && o.binned != 2);
  uint64_t tile_round_bytes = 0;
  if (rounds_tiles) {
    const uint64_t nt = (n + kTRCells - 1) / kTRCells;
    tile_round_bytes = ((uint64_t)r * m_keys + (uint64_t)kTRAlign * nt) * (2 * sizeof(u64) + sizeof(u16) + sizeof(u32)) +
                       (nt + 1) * (sizeof(u64) + sizeof(u32)) + nt * (kTRPosStride * sizeof(u32) + 3 * sizeof(u32) +
                                                      2 * sizeof(TileAct));
  }
  const bool rounds_binned = !rounds_tiles && (o.binned == 1 || (o.binned == 0 && n >= (1ull << 21)));
  if (rounds_binned) {
    uint32_t nb;
    uint64_t cap;
    u32 shift;
    round_bin_layout(n, r, &nb, &cap, &shift);
    if (cap * nb > records) records = cap * nb;
    if (nb > counts) counts = nb;
  }
  const uint64_t rec_bytes = records ? records * (sizeof(u64) + sizeof(u32)) + (counts + 1) * sizeof(u32) : 0;
  if (table_bytes) *table_bytes = table;
  if (fixed_bytes) *fixed_bytes = fixed;
  if (peak_bytes) *peak_bytes = table + fixed + rec_bytes + tiles + tile_round_bytes;
  return PP_OK;
}

pp_status pp_iblt_destroy(pp_iblt *t) {
  if (!t) return PP_OK;
  cudaDeviceSynchronize();
  free_all(t);
  return PP_OK;
}

pp_status pp_iblt_clear(pp_iblt *t, void *stream) {
  if (!t) return fail(PP_ERR_INVALID_ARG, "pp_iblt_clear: NULL table");
  PP_CUDA(cudaMemsetAsync(t->cells, 0, t->n * sizeof(Cell), as_stream(stream)));
  t->items = 0;
  t->has_deletes = false;
  return PP_OK;
}

pp_status pp_iblt_insert(pp_iblt *t, const uint64_t *d_keys, uint64_t m, void *stream) {
  if (!t) return fail(PP_ERR_INVALID_ARG, "pp_iblt_insert: NULL table");
  if (m && !d_keys) return fail(PP_ERR_INVALID_ARG, "pp_iblt_insert: NULL keys");
  pp_status st = update(t, d_keys, m, +1, as_stream(stream));
  if (st == PP_OK) t->items += (int64_t)m;
  return st;
}

pp_status pp_iblt_delete(pp_iblt *t, const uint64_t *d_keys, uint64_t m, void *stream) {
  if (!t) return fail(PP_ERR_INVALID_ARG, "pp_iblt_delete: NULL table");
  if (m && !d_keys) return fail(PP_ERR_INVALID_ARG, "pp_iblt_delete: NULL keys");
  pp_status st = update(t, d_keys, m, -1, as_stream(stream));
  if (st == PP_OK) t->items -= (int64_t)m;
  if (m) t->has_deletes = true;
  return st;
}

pp_status pp_iblt_build(pp_iblt *t, const uint64_t *d_keys, uint64_t m, void *stream) {
  if (!t) return fail(PP_ERR_INVALID_ARG, "pp_iblt_build: NULL table");
  if (m && !d_keys) return fail(PP_ERR_INVALID_ARG, "pp_iblt_build: NULL keys");
  cudaStream_t s = as_stream(stream);
  t->items = 0;
  t->has_deletes = false;
  if (!use_binned(t, m)) {
    PP_CUDA(cudaMemsetAsync(t->cells, 0, t->n * sizeof(Cell), s));
    pp_status st = launch_insert(t, d_keys, m, +1, s);
    if (st == PP_OK) t->items = (int64_t)m;
    return st;
  }
  BinArgs ba;
  pp_status st = bin_pass(t, d_keys, m, +1, 0, s, ba);
  if (st != PP_OK) return st;
  // the flag comes back through mapped memory, not a copy engine that may be
  // busy with another stream's bulk copy
  st = ensure_flag(t);
  if (st != PP_OK) return st;
  k_flag_to_host<<<1, 32, 0, s>>>(t->bin_overflow, t->d_flag);
  PP_CUDA(cudaGetLastError());
  PP_CUDA(cudaStreamSynchronize(s));
  if (*(volatile u32 *)t->h_flag) {
    // a slab got more updates than its list holds: build the plain way
    PP_CUDA(cudaMemsetAsync(t->cells, 0, t->n * sizeof(Cell), s));
    st = launch_insert(t, d_keys, m, +1, s);
  } else {
    st = apply_pass(t, ba, +1, true, s);
  }
  if (st == PP_OK) t->items = (int64_t)m;
  return st;
}

pp_status pp_iblt_decode(pp_iblt *t, uint64_t *d_out_keys, uint64_t out_cap, pp_decode_result *res,
                         void *stream) {
  if (!t || !res) return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode: NULL table or result");
  const uint64_t items = t->items > 0 ? (uint64_t)t->items : 0;
  if (out_cap < items)
    return fail(PP_ERR_CAPACITY, "pp_iblt_decode: out_cap=%llu < %llu keys in the table",
                (unsigned long long)out_cap, (unsigned long long)items);
  if (out_cap && !d_out_keys) return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode: NULL output");
  cudaStream_t s = as_stream(stream);
  pp_status st = decode_enqueue(t, d_out_keys, out_cap, s);
  if (st != PP_OK) return st;
  return decode_result(t, out_cap, res, s, "pp_iblt_decode");
}

pp_status pp_iblt_decode_subrounds(pp_iblt *t, uint64_t *d_out_keys, uint64_t out_cap,
                                   pp_decode_result *res, void *stream) {
  if (!t || !res) return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode_subrounds: NULL table or result");
  const uint64_t items = t->items > 0 ? (uint64_t)t->items : 0;
  if (out_cap < items)
    return fail(PP_ERR_CAPACITY, "pp_iblt_decode_subrounds: out_cap=%llu < %llu keys in the table",
                (unsigned long long)out_cap, (unsigned long long)items);
  if (out_cap && !d_out_keys) return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode_subrounds: NULL output");
  cudaStream_t s = as_stream(stream);
  pp_status st = sub_prepare(t);
  if (st != PP_OK) return st;
  const bool binned = t->opt.binned == 1 || (t->opt.binned == 0 && t->n >= (1ull << 21));
  if (binned) {
    st = ensure_round_bins(t, s);
    if (st != PP_OK) return st;
    PP_CUDA(cudaMemsetAsync(t->bin_count, 0, t->n_bins * sizeof(u32), s));
    // the round kernels' control block: output, counters
    memset(t->h_ctl, 0, sizeof(DecodeCtl));
    t->h_ctl->out = reinterpret_cast<u64 *>(d_out_keys);
    t->h_ctl->out_cap = out_cap;
    t->h_ctl->max_rounds = t->opt.max_rounds;
    k_ctl_init<<<1, 32, 0, s>>>(t->ctl, *t->h_ctl);
    PP_CUDA(cudaGetLastError());
  }
  SubDecCtl &h = *t->h_sctl;
  memset(&h, 0, sizeof h);
  h.out = reinterpret_cast<u64 *>(d_out_keys);
  h.out_cap = out_cap;
  h.max_sub = t->opt.max_rounds;
  h.r = t->r;
  h.part = t->r - 1;  // the first sub-round looks at sub-table 0
  PP_CUDA(cudaMemcpyAsync(t->sctl, t->h_sctl, sizeof(SubDecCtl), cudaMemcpyHostToDevice, s));
  st = t->opt.host_loop ? sub_host_loop(t, binned, s) : sub_graph_launch(t, binned, s);
  if (st != PP_OK) return st;
  PP_CUDA(cudaMemcpyAsync(t->h_sctl, t->sctl, sizeof(SubDecCtl), cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaStreamSynchronize(s));
  const SubDecCtl c = *t->h_sctl;
  const uint32_t S = c.last;
  const uint32_t ncopy = S < res->round_cap ? S : res->round_cap;
  if (ncopy && (res->recovered_per_round || res->remaining_per_round)) {
    PP_CUDA(cudaMemcpyAsync(t->h_rec, t->st_rec, ncopy * sizeof(u64), cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
    uint64_t left = items;
    for (uint32_t i = 0; i < ncopy; ++i) {
      left -= t->h_rec[i] <= left ? t->h_rec[i] : left;
      if (res->recovered_per_round) res->recovered_per_round[i] = t->h_rec[i];
      if (res->remaining_per_round) res->remaining_per_round[i] = left;
    }
  }
  if (ncopy && res->alive_cells_per_round)
    memset(res->alive_cells_per_round, 0, ncopy * sizeof(uint64_t));
  res->rounds = S;
  res->status_flags = c.flags;
  res->recovered = c.n_out < out_cap ? c.n_out : out_cap;
  res->items_before = items;
  res->residual_cells = c.nonempty - c.emptied;
  t->items -= (int64_t)res->recovered;
  if (c.flags & FLAG_CAPACITY)
    return fail(PP_ERR_CAPACITY, "pp_iblt_decode_subrounds: more keys recovered than out_cap=%llu",
                (unsigned long long)out_cap);
  if (c.flags & FLAG_INTERNAL)
    return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode_subrounds: a pure cell's key does not hash to it");
  if (c.flags & FLAG_ROUND_LIMIT)
    return fail(PP_ERR_ROUND_LIMIT, "pp_iblt_decode_subrounds: stopped after max_rounds=%u sub-rounds",
                t->opt.max_rounds);
  return PP_OK;
}

pp_status pp_iblt_decode_signed(pp_iblt *t, uint64_t *d_out_keys, int8_t *d_out_signs, uint64_t out_cap,
                                pp_decode_result *res, void *stream) {
  if (!t || !res) return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode_signed: NULL table or result");
  if (out_cap && !d_out_keys) return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode_signed: NULL output");
  if (!t->k.sg_scan) return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode_signed: no kernels for r=%u", t->r);
  if ((uint64_t)t->r * t->n >= (1ull << 32))
    return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode_signed: r * n_cells must stay below 2^32");
  cudaStream_t s = as_stream(stream);
  if (!t->fsign) {
    PP_CUDA(cudaMalloc((void **)&t->fsign, t->n));
    PP_CUDA(cudaMalloc((void **)&t->sg_cand, (size_t)t->r * t->n * sizeof(u32)));
    t->grid_sgscan = persistent_grid(t->k.sg_scan, kBlock, 0, t->opt.ctas_per_sm);
    t->grid_sgpeel = persistent_grid(t->k.sg_peel, kBlock, 0, t->opt.ctas_per_sm);
    t->grid_sgfilter = persistent_grid(t->k.sg_filter, kBlock, 0, t->opt.ctas_per_sm);
  }
  // binned rounds for large tables, as in the unsigned decode
  const bool binned = t->opt.binned == 1 || (t->opt.binned == 0 && t->n >= (1ull << 21));
  if (binned) {
    pp_status st = ensure_round_bins(t, s);
    if (st != PP_OK) return st;
    PP_CUDA(cudaMemsetAsync(t->bin_count, 0, t->n_bins * sizeof(u32), s));
    t->smem_sgclaim = claim_smem_bytes(t->k.nr, false, t->n_bins, true);
    t->grid_sgclaim = persistent_grid(t->k.sg_claim, kBlock, t->smem_sgclaim, t->opt.ctas_per_sm);
  }
  memset(t->h_ctl, 0, sizeof(DecodeCtl));
  t->h_ctl->out = reinterpret_cast<u64 *>(d_out_keys);
  t->h_ctl->out_cap = out_cap;
  t->h_ctl->max_rounds = t->opt.max_rounds;
  k_ctl_init<<<1, 32, 0, s>>>(t->ctl, *t->h_ctl);
  PP_CUDA(cudaGetLastError());
  // kernel arguments (the output sign pointer is one of them)
  const Cell *cells_c = t->cells;
  Cell *cells = t->cells;
  TableArgs tab = t->args;
  u64 *fkey = t->fkey;
  u32 *fcell = t->fcell, *bitmap = t->bitmap, *cand = t->sg_cand;
  signed char *fsign = t->fsign, *osign = reinterpret_cast<signed char *>(d_out_signs);
  const u64 *fkey_c = t->fkey;
  const u32 *fcell_c = t->fcell, *bitmap_c = t->bitmap, *cand_c = t->sg_cand;
  const signed char *fsign_c = t->fsign;
  u64 cand_cap = (u64)t->r * t->n;
  DecodeCtl *ctl = t->ctl;
  RoundStats rs{t->st_rec, t->st_alive, t->st_front};
  int set_cond = 0;
  cudaGraphConditionalHandle cond = 0;
  void *scan_p[] = {&cells_c, &tab, &fkey, &fcell, &fsign, &bitmap, &ctl};
  void *peel_p[] = {&cells, &tab, &fkey_c, &fcell_c, &fsign_c, &bitmap_c, &cand, &cand_cap, &osign, &ctl};
  void *filt_p[] = {&cells_c, &tab, &cand_c, &fkey, &fcell, &fsign, &bitmap, &ctl};
  void *end_p[] = {&ctl, &rs, &set_cond, &cond};
  // binned rounds: claim (records carry the sign) -> apply -> filter -> reset bins
  ClaimArgs ca;
  ApplyRArgs aa;
  ResetArgs ra;
  if (binned) {
    fill_round_args(t, ca, aa, ra);
    ca.rb.fsign = t->fsign;
    ca.rb.osign = osign;
    ca.rb.cand_cap = cand_cap;
    ca.cand = t->sg_cand;
    aa.rb.cand_cap = cand_cap;
    aa.cand = t->sg_cand;
  }
  if (t->opt.host_loop) {
    PP_CUDA(cudaLaunchKernel(t->k.sg_scan, dim3(t->grid_sgscan), dim3(kBlock), scan_p, 0, s));
    for (;;) {
      if (binned) {
        PP_CUDA(cudaLaunchKernel(t->k.sg_claim, dim3(t->grid_sgclaim), dim3(kBlock), ca.p, t->smem_sgclaim, s));
        PP_CUDA(cudaLaunchKernel(t->k.sg_apply, dim3(t->grid_apply_round), dim3(kBlock), aa.p,
                                 t->smem_apply_round, s));
      } else {
        PP_CUDA(cudaLaunchKernel(t->k.sg_peel, dim3(t->grid_sgpeel), dim3(kBlock), peel_p, 0, s));
      }
      PP_CUDA(cudaLaunchKernel(t->k.sg_filter, dim3(t->grid_sgfilter), dim3(kBlock), filt_p, 0, s));
      if (binned) PP_CUDA(cudaLaunchKernel((const void *)k_bins_reset, dim3(1), dim3(256), ra.p, 0, s));
      PP_CUDA(cudaLaunchKernel((const void *)k_round_end, dim3(1), dim3(32), end_p, 0, s));
      PP_CUDA(cudaMemcpyAsync(&t->h_ctl->more, &t->ctl->more, sizeof(u32), cudaMemcpyDeviceToHost, s));
      PP_CUDA(cudaStreamSynchronize(s));
      if (!t->h_ctl->more) break;
    }
  } else {
    if (t->sg_exec && (t->sg_graph_out != osign || t->sg_graph_binned != binned ||
                       (binned && t->sg_graph_gen != t->rec_gen))) {
      cudaGraphExecDestroy(t->sg_exec);
      t->sg_exec = nullptr;
    }
    if (!t->sg_exec) {
      // sgscan -> while (more) { sgpeel -> sgfilter -> round_end }, or with
      // binned rounds { claim -> apply -> sgfilter -> reset bins -> round_end }
      cudaGraph_t g = nullptr;
      PP_CUDA(cudaGraphCreate(&g, 0));
      pp_status st = PP_OK;
      cudaGraphNode_t n_scan, n_cond, n_peel, n_apply, n_filter, n_reset, n_end;
      cudaGraphNodeParams cp{};
      cudaGraph_t body;
      st = add_kernel(&n_scan, g, nullptr, 0, t->k.sg_scan, t->grid_sgscan, kBlock, 0, scan_p);
      if (st != PP_OK) goto sg_done;
      if (cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
        st = fail(PP_ERR_CUDA, "cudaGraphConditionalHandleCreate failed");
        goto sg_done;
      }
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = cond;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      if (cudaGraphAddNode(&n_cond, g, &n_scan, nullptr, 1, &cp) != cudaSuccess) {
        st = fail(PP_ERR_CUDA, "cudaGraphAddNode(conditional while) failed");
        goto sg_done;
      }
      body = cp.conditional.phGraph_out[0];
      set_cond = 1;
      if (binned) {
        st = add_kernel(&n_peel, body, nullptr, 0, t->k.sg_claim, t->grid_sgclaim, kBlock, t->smem_sgclaim, ca.p);
        if (st != PP_OK) goto sg_done;
        st = add_kernel(&n_apply, body, &n_peel, 1, t->k.sg_apply, t->grid_apply_round, kBlock,
                        t->smem_apply_round, aa.p);
        if (st != PP_OK) goto sg_done;
        st = add_kernel(&n_filter, body, &n_apply, 1, t->k.sg_filter, t->grid_sgfilter, kBlock, 0, filt_p);
        if (st != PP_OK) goto sg_done;
        st = add_kernel(&n_reset, body, &n_filter, 1, (const void *)k_bins_reset, 1, 256, 0, ra.p);
        if (st != PP_OK) goto sg_done;
        st = add_kernel(&n_end, body, &n_reset, 1, (const void *)k_round_end, 1, 32, 0, end_p);
        if (st != PP_OK) goto sg_done;
      } else {
        st = add_kernel(&n_peel, body, nullptr, 0, t->k.sg_peel, t->grid_sgpeel, kBlock, 0, peel_p);
        if (st != PP_OK) goto sg_done;
        st = add_kernel(&n_filter, body, &n_peel, 1, t->k.sg_filter, t->grid_sgfilter, kBlock, 0, filt_p);
        if (st != PP_OK) goto sg_done;
        st = add_kernel(&n_end, body, &n_filter, 1, (const void *)k_round_end, 1, 32, 0, end_p);
        if (st != PP_OK) goto sg_done;
      }
      if (cudaGraphInstantiate(&t->sg_exec, g, 0) != cudaSuccess) {
        st = fail(PP_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(cudaGetLastError()));
        t->sg_exec = nullptr;
      }
      t->sg_graph_out = osign;
      t->sg_graph_binned = binned;
      t->sg_graph_gen = t->rec_gen;
    sg_done:
      cudaGraphDestroy(g);
      if (st != PP_OK) return st;
    }
    PP_CUDA(cudaGraphLaunch(t->sg_exec, s));
  }
  PP_CUDA(cudaMemcpyAsync(t->h_ctl, t->ctl, sizeof(DecodeCtl), cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaStreamSynchronize(s));
  const DecodeCtl c = *t->h_ctl;
  const uint32_t T = c.round;
  const uint32_t ncopy = T < res->round_cap ? T : res->round_cap;
  if (ncopy && res->recovered_per_round) {
    PP_CUDA(cudaMemcpyAsync(t->h_rec, t->st_rec, ncopy * sizeof(u64), cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
    for (uint32_t i = 0; i < ncopy; ++i) res->recovered_per_round[i] = t->h_rec[i];
  }
  if (ncopy && res->remaining_per_round) memset(res->remaining_per_round, 0, ncopy * sizeof(uint64_t));
  if (ncopy && res->alive_cells_per_round) memset(res->alive_cells_per_round, 0, ncopy * sizeof(uint64_t));
  res->rounds = T;
  res->status_flags = c.flags;
  res->recovered = c.n_out < out_cap ? c.n_out : out_cap;
  res->items_before = t->items > 0 ? (uint64_t)t->items : 0;
  res->residual_cells = c.nonempty - c.emptied;
  t->items -= (int64_t)c.n_out - 2 * (int64_t)c.n_neg;  // positives minus negatives
  if (c.flags & FLAG_CAPACITY)
    return fail(PP_ERR_CAPACITY, "pp_iblt_decode_signed: more keys recovered than out_cap=%llu",
                (unsigned long long)out_cap);
  if (c.flags & FLAG_INTERNAL)
    return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode_signed: a pure cell's key does not hash to it");
  if (c.flags & FLAG_ROUND_LIMIT)
    return fail(PP_ERR_ROUND_LIMIT, "pp_iblt_decode_signed: stopped after max_rounds=%u rounds",
                t->opt.max_rounds);
  return PP_OK;
}

// ---- build + decode from host buffers -------------------------------------
namespace {

// Pins a host range for the job unless it is pinned already.
pp_status pin_host(void *p, size_t bytes, bool *registered) {
  *registered = false;
  if (!p || !bytes) return PP_OK;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) == cudaSuccess && a.type == cudaMemoryTypeHost) return PP_OK;
  cudaGetLastError();  // a pageable pointer may leave an error behind
  PP_CUDA(cudaHostRegister(p, bytes, cudaHostRegisterDefault));
  *registered = true;
  return PP_OK;
}

// pp_iblt_build without its flag check: the slab-binned build is enqueued as
// if no slab list overflowed (*binned tells whether the flag is meaningful).
pp_status build_enqueue(pp_iblt *t, const uint64_t *d_keys, uint64_t m, cudaStream_t s, bool *binned) {
  t->items = 0;
  t->has_deletes = false;
  *binned = use_binned(t, m);
  pp_status st;
  if (!*binned) {
    PP_CUDA(cudaMemsetAsync(t->cells, 0, t->n * sizeof(Cell), s));
    st = launch_insert(t, d_keys, m, +1, s);
  } else {
    BinArgs ba;
    st = bin_pass(t, d_keys, m, +1, 0, s, ba);
    if (st == PP_OK) st = apply_pass(t, ba, +1, true, s);
  }
  if (st == PP_OK) t->items = (int64_t)m;
  return st;
}

// A build from m keys and its decode, enqueued on s.  When the build is
// slab-binned and the tile rounds decode the table, the build's tile pass
// also finds F_1 (PrescanArgs) and the decode skips its scan of the table;
// otherwise the two run one after the other.  flag_dst null: the build's
// slab-overflow flag is checked here (a full slab list falls back to the
// direct build); else it is copied to flag_dst and nothing waits for it.
// Events (may be null): `built` is recorded once the build has read d_keys;
// the decode waits for `out_free` before it writes d_out_keys (the build
// writes none of it).
pp_status build_decode_enqueue(pp_iblt *t, const uint64_t *d_keys, uint64_t m, uint64_t *d_out_keys,
                               uint64_t out_cap, cudaStream_t s, u32 *flag_dst, cudaEvent_t built = nullptr,
                               cudaEvent_t out_free = nullptr) {
  t->items = 0;
  t->has_deletes = false;
  const bool fused = use_binned(t, m) && t->k.trescan && want_tile_rounds(t);
  if (!fused) {
    pp_status st;
    if (flag_dst) {
      bool binned = false;
      st = build_enqueue(t, d_keys, m, s, &binned);
      if (st == PP_OK && binned) {
        k_flag_to_host<<<1, 32, 0, s>>>(t->bin_overflow, flag_dst);
        PP_CUDA(cudaGetLastError());
      }
    } else {
      st = pp_iblt_build(t, d_keys, m, s);
    }
    if (st != PP_OK) return st;
    if (built) PP_CUDA(cudaEventRecord(built, s));
    if (out_free) PP_CUDA(cudaStreamWaitEvent(s, out_free, 0));
    return decode_enqueue(t, d_out_keys, out_cap, s);
  }
  BinArgs ba;
  pp_status st = bin_pass(t, d_keys, m, +1, 0, s, ba);
  if (st != PP_OK) return st;
  if (!flag_dst) {
    st = ensure_flag(t);
    if (st != PP_OK) return st;
    k_flag_to_host<<<1, 32, 0, s>>>(t->bin_overflow, t->d_flag);
    PP_CUDA(cudaGetLastError());
    PP_CUDA(cudaStreamSynchronize(s));
    if (*(volatile u32 *)t->h_flag) {
      PP_CUDA(cudaMemsetAsync(t->cells, 0, t->n * sizeof(Cell), s));
      st = launch_insert(t, d_keys, m, +1, s);
      if (st != PP_OK) return st;
      t->items = (int64_t)m;
      if (built) PP_CUDA(cudaEventRecord(built, s));
      if (out_free) PP_CUDA(cudaStreamWaitEvent(s, out_free, 0));
      return decode_enqueue(t, d_out_keys, out_cap, s);
    }
  } else {
    k_flag_to_host<<<1, 32, 0, s>>>(t->bin_overflow, flag_dst);
    PP_CUDA(cudaGetLastError());
  }
  t->items = (int64_t)m;
  st = ensure_tile_rounds(t, s);
  if (st != PP_OK) return st;
  // the decode's counters start before the build adds F_1 to them
  set_host_ctl(t, d_out_keys, out_cap);
  k_ctl_init<<<1, 32, 0, s>>>(t->ctl, *t->h_ctl);
  PP_CUDA(cudaGetLastError());
  const TileRoundBufs &tb = t->tre.trb;
  PP_CUDA(cudaMemsetAsync(tb.fseg, 0, (size_t)tb.n_seg_d * sizeof(u32), s));
  PP_CUDA(cudaMemsetAsync(tb.n_rescan, 0, sizeof(u32), s));
  const PrescanArgs pre{tb, t->fkey, t->fcell, t->bitmap, t->ctl, t->args.seed[t->r], nullptr};
  st = apply_pass(t, ba, +1, true, s, &pre);
  if (st != PP_OK) return st;
  if (built) PP_CUDA(cudaEventRecord(built, s));
  if (out_free) PP_CUDA(cudaStreamWaitEvent(s, out_free, 0));
  return launch_prescanned_rounds(t, s);
}

}  // namespace

pp_status pp_iblt_build_decode(pp_iblt *t, const uint64_t *d_keys, uint64_t m, uint64_t *d_out_keys,
                               uint64_t out_cap, pp_decode_result *res, void *stream) {
  if (!t || !res) return fail(PP_ERR_INVALID_ARG, "pp_iblt_build_decode: NULL table or result");
  if (m && !d_keys) return fail(PP_ERR_INVALID_ARG, "pp_iblt_build_decode: NULL keys");
  if (out_cap < m)
    return fail(PP_ERR_CAPACITY, "pp_iblt_build_decode: out_cap=%llu < %llu keys", (unsigned long long)out_cap,
                (unsigned long long)m);
  if (out_cap && !d_out_keys) return fail(PP_ERR_INVALID_ARG, "pp_iblt_build_decode: NULL output");
  cudaStream_t s = as_stream(stream);
  pp_status st = build_decode_enqueue(t, d_keys, m, d_out_keys, out_cap, s, nullptr);
  if (st != PP_OK) return st;
  return decode_result(t, out_cap, res, s, "pp_iblt_build_decode");
}

pp_status pp_iblt_submit_host(pp_iblt *t, const uint64_t *h_keys, uint64_t m, uint64_t *h_out, uint64_t out_cap,
                              uint64_t *ticket, void *stream) {
  if (!t || !ticket) return fail(PP_ERR_INVALID_ARG, "pp_iblt_submit_host: NULL table or ticket");
  if (m && (!h_keys || !h_out)) return fail(PP_ERR_INVALID_ARG, "pp_iblt_submit_host: NULL keys or output");
  if (out_cap < m)
    return fail(PP_ERR_CAPACITY, "pp_iblt_submit_host: out_cap=%llu < %llu keys", (unsigned long long)out_cap,
                (unsigned long long)m);
  HostJob &j = t->jobs[t->next_ticket % kHostJobs];
  if (j.busy)
    return fail(PP_ERR_INVALID_ARG, "pp_iblt_submit_host: %u jobs in flight; finish one first", kHostJobs);
  cudaStream_t s = as_stream(stream);
  if (!t->up_s) PP_CUDA(cudaStreamCreateWithFlags(&t->up_s, cudaStreamNonBlocking));
  if (!t->down_s) PP_CUDA(cudaStreamCreateWithFlags(&t->down_s, cudaStreamNonBlocking));
  if (!j.up) {
    PP_CUDA(cudaEventCreateWithFlags(&j.up, cudaEventDisableTiming));
    PP_CUDA(cudaEventCreateWithFlags(&j.built, cudaEventDisableTiming));
    PP_CUDA(cudaEventCreateWithFlags(&j.dec, cudaEventDisableTiming));
    PP_CUDA(cudaEventCreateWithFlags(&j.done, cudaEventDisableTiming));
    const unsigned fl = cudaHostAllocMapped | cudaHostAllocPortable;
    PP_CUDA(cudaHostAlloc((void **)&j.h_ctl, sizeof(DecodeCtl), fl));
    PP_CUDA(cudaHostAlloc((void **)&j.h_stats, 2 * (size_t)kJobStatRounds * sizeof(u64), fl));
    PP_CUDA(cudaHostAlloc((void **)&j.h_flag, sizeof(u32), fl));
    PP_CUDA(cudaHostGetDevicePointer((void **)&j.d_ctl, j.h_ctl, 0));
    PP_CUDA(cudaHostGetDevicePointer((void **)&j.d_stats, j.h_stats, 0));
    PP_CUDA(cudaHostGetDevicePointer((void **)&j.d_flag, j.h_flag, 0));
  }
  if (m > j.cap) {
    PP_CUDA(cudaEventSynchronize(j.done));
    cudaFree(j.d_keys);
    cudaFree(j.d_out);
    j.d_keys = j.d_out = nullptr;
    j.cap = 0;
    PP_CUDA(cudaMalloc((void **)&j.d_keys, m * sizeof(u64)));
    PP_CUDA(cudaMalloc((void **)&j.d_out, m * sizeof(u64)));
    j.cap = m;
  }
  pp_status st = pin_host(const_cast<uint64_t *>(h_keys), m * sizeof(u64), &j.reg_keys);
  if (st == PP_OK) st = pin_host(h_out, m * sizeof(u64), &j.reg_out);
  if (st != PP_OK) {
    if (j.reg_keys) cudaHostUnregister(const_cast<uint64_t *>(h_keys));
    j.reg_keys = false;
    return st;
  }
  j.h_keys = h_keys;
  j.h_out = h_out;
  j.m = m;
  j.out_cap = out_cap;
  j.s = s;
  *j.h_flag = 0;
  // Three streams: uploads, the caller's (build and decode), downloads.  The
  // upload into this slot waits only for the slot's previous build (its reader),
  // the decode into the slot's output only for the slot's previous download.
  PP_CUDA(cudaStreamWaitEvent(t->up_s, j.built, 0));
  if (m) PP_CUDA(cudaMemcpyAsync(j.d_keys, h_keys, m * sizeof(u64), cudaMemcpyHostToDevice, t->up_s));
  PP_CUDA(cudaEventRecord(j.up, t->up_s));
  PP_CUDA(cudaStreamWaitEvent(s, j.up, 0));
  // The build is enqueued without waiting for its slab-overflow flag: the flag
  // travels with the job, and pp_iblt_finish_host redoes the job in the rare
  // case it is set.  The decode writes the slot's output: it waits for the
  // slot's previous download.
  st = build_decode_enqueue(t, reinterpret_cast<const uint64_t *>(j.d_keys), m,
                            reinterpret_cast<uint64_t *>(j.d_out), m, s, j.d_flag, j.built, j.done);
  if (st != PP_OK) {
    cudaStreamSynchronize(t->up_s);
    if (j.reg_keys) cudaHostUnregister(const_cast<uint64_t *>(h_keys));
    if (j.reg_out) cudaHostUnregister(h_out);
    j.reg_keys = j.reg_out = false;
    return st;
  }
  const uint32_t ns = t->opt.max_rounds < kJobStatRounds ? t->opt.max_rounds : kJobStatRounds;
  // the decode's results reach the host through mapped memory, never queued
  // behind another job's download on a copy engine
  k_to_host<<<1, 128, 0, s>>>(reinterpret_cast<const u64 *>(t->ctl), reinterpret_cast<u64 *>(j.d_ctl),
                              (u32)(sizeof(DecodeCtl) / sizeof(u64)));
  k_to_host<<<8, 256, 0, s>>>(t->st_rec, j.d_stats, ns);
  k_to_host<<<8, 256, 0, s>>>(t->st_alive, j.d_stats + kJobStatRounds, ns);
  PP_CUDA(cudaGetLastError());
  PP_CUDA(cudaEventRecord(j.dec, s));
  // download every slot a recovered key may use
  PP_CUDA(cudaStreamWaitEvent(t->down_s, j.dec, 0));
  if (m) PP_CUDA(cudaMemcpyAsync(h_out, j.d_out, m * sizeof(u64), cudaMemcpyDeviceToHost, t->down_s));
  PP_CUDA(cudaEventRecord(j.done, t->down_s));
  j.ticket = t->next_ticket++;
  j.busy = true;
  *ticket = j.ticket;
  return PP_OK;
}

pp_status pp_iblt_finish_host(pp_iblt *t, uint64_t ticket, pp_decode_result *res) {
  if (!t || !res) return fail(PP_ERR_INVALID_ARG, "pp_iblt_finish_host: NULL table or result");
  HostJob *j = nullptr;
  for (HostJob &x : t->jobs)
    if (x.busy && x.ticket == ticket) j = &x;
  if (!j) return fail(PP_ERR_INVALID_ARG, "pp_iblt_finish_host: no job with ticket %llu in flight",
                      (unsigned long long)ticket);
  cudaError_t e = cudaEventSynchronize(j->done);
  pp_status st = PP_OK;
  if (e == cudaSuccess && *(volatile u32 *)j->h_flag) {
    // a slab of the build got more updates than its list holds: the job's
    // table was incomplete.  Redo it on its stream (after any later job's
    // work there), with the build that checks the flag, then copy its keys.
    const uint64_t *dk = reinterpret_cast<const uint64_t *>(j->d_keys);
    st = build_decode_enqueue(t, dk, j->m, reinterpret_cast<uint64_t *>(j->d_out), j->m, j->s, nullptr);
    if (st == PP_OK) {
      const uint32_t ns = t->opt.max_rounds < kJobStatRounds ? t->opt.max_rounds : kJobStatRounds;
      k_to_host<<<1, 128, 0, j->s>>>(reinterpret_cast<const u64 *>(t->ctl), reinterpret_cast<u64 *>(j->d_ctl),
                                     (u32)(sizeof(DecodeCtl) / sizeof(u64)));
      k_to_host<<<8, 256, 0, j->s>>>(t->st_rec, j->d_stats, ns);
      k_to_host<<<8, 256, 0, j->s>>>(t->st_alive, j->d_stats + kJobStatRounds, ns);
      e = cudaGetLastError();
      if (e == cudaSuccess && j->m)
        e = cudaMemcpyAsync(j->h_out, j->d_out, j->m * sizeof(u64), cudaMemcpyDeviceToHost, j->s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(j->s);
    }
  }
  if (j->reg_keys) cudaHostUnregister(const_cast<uint64_t *>(j->h_keys));
  if (j->reg_out) cudaHostUnregister(j->h_out);
  j->reg_keys = j->reg_out = false;
  j->busy = false;
  if (st != PP_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "pp_iblt_finish_host", __FILE__, __LINE__);
  const uint32_t ns = t->opt.max_rounds < kJobStatRounds ? t->opt.max_rounds : kJobStatRounds;
  st = decode_collect(*j->h_ctl, j->h_stats, j->h_stats + kJobStatRounds, ns, j->m, j->m, res,
                      t->opt.max_rounds, "pp_iblt_finish_host");
  if (j->ticket + 1 == t->next_ticket) t->items = (int64_t)j->m - (int64_t)res->recovered;  // the latest build
  return st;
}

pp_status pp_iblt_build_decode_host(pp_iblt *t, const uint64_t *h_keys, uint64_t m, uint64_t *h_out,
                                    uint64_t out_cap, pp_decode_result *res, void *stream) {
  if (!res) return fail(PP_ERR_INVALID_ARG, "pp_iblt_build_decode_host: NULL result");
  uint64_t ticket = 0;
  pp_status st = pp_iblt_submit_host(t, h_keys, m, h_out, out_cap, &ticket, stream);
  if (st != PP_OK) return st;
  return pp_iblt_finish_host(t, ticket, res);
}

pp_status pp_iblt_copy_cells(pp_iblt *t, void *dst, uint64_t first, uint64_t count, int to_host,
                             void *stream) {
  if (!t || (!dst && count)) return fail(PP_ERR_INVALID_ARG, "pp_iblt_copy_cells: NULL argument");
  if (first > t->n || count > t->n - first)
    return fail(PP_ERR_INVALID_ARG, "pp_iblt_copy_cells: range outside the table");
  cudaStream_t s = as_stream(stream);
  PP_CUDA(cudaMemcpyAsync(dst, t->cells + first, count * sizeof(Cell),
                          to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  PP_CUDA(cudaStreamSynchronize(s));
  return PP_OK;
}

pp_status pp_iblt_info(const pp_iblt *t, uint64_t *n_cells, uint32_t *r, uint64_t *h_seeds) {
  if (!t) return fail(PP_ERR_INVALID_ARG, "pp_iblt_info: NULL table");
  if (n_cells) *n_cells = t->n;
  if (r) *r = t->r;
  if (h_seeds)
    for (uint32_t j = 0; j <= t->r; ++j) h_seeds[j] = t->args.seed[j];
  return PP_OK;
}

}  // extern "C"
