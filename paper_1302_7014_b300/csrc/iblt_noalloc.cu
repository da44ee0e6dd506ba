// IBLT decode that allocates nothing: pp_iblt_decode_noalloc.
//
// Who needs it: callers that must not allocate device memory while they run.
// Typical cases are a host framework that has already reserved nearly all of
// the GPU's memory for its own pool (so cudaMalloc would fail or steal from
// it), services with a "no allocation after start-up" rule, and latency-bound
// loops where cudaFree's implicit device-wide synchronisation would stall
// every other stream.  Such callers own the table and the output buffer; this
// entry point brings its own working memory.
//
// Where the working memory lives: one file-scope __device__ array of fixed
// size (g_noalloc_scratch below).  It exists on a GPU once the library's
// device code is loaded there, and stays until the process exits.  With the
// CUDA runtime's default lazy module loading, that load happens inside the
// first call of this entry point on each device (the cudaGetSymbolAddress
// below triggers it), and loading does take device memory: the array plus the
// module's code.  So the first call on each device must come at start-up,
// before the caller's framework reserves its memory pool and before any
// stream capture; or the process runs with CUDA_MODULE_LOADING=EAGER, which
// loads the module when the CUDA context is created.  Later calls allocate
// nothing.  Host code cannot use the array's name as a device address (on the
// host it names a stand-in object), so every call looks the current device's
// address up with cudaGetSymbolAddress (cheap once the module is loaded); no
// address is cached, so a cudaDeviceReset between calls leaves nothing stale.
//
// Sharing: every call on a device uses the same array and finds the previous
// call's data in it.  The parts that must start at zero are cleared at the
// start of each call; everything else is written before it is read.  Two calls
// whose GPU work overlaps (different streams, or different host threads on
// the same device) race on the array and give wrong results: serialise them.
//
// The decode itself runs the same scan / peel / filter / round-end kernels as
// pp_iblt_decode, driven from the host one round at a time (no graph is built,
// since instantiating one allocates).
#include <stdint.h>
#include <string.h>

#include "host.cuh"
#include "iblt_types.cuh"

using namespace pp;

namespace {

constexpr uint64_t kMaxCells = PP_NOALLOC_MAX_CELLS;
constexpr uint32_t kMaxRounds = PP_NOALLOC_MAX_ROUNDS;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Layout of the scratch array.
constexpr size_t kOffCtl = 0;                                         // DecodeCtl
constexpr size_t kOffSum = 256;                                       // long long: sum of counts
constexpr size_t kOffRec = 512;                                       // u64[kMaxRounds]
constexpr size_t kOffAlive = kOffRec + 8 * (size_t)kMaxRounds;        // u64[kMaxRounds]
constexpr size_t kOffFront = kOffAlive + 8 * (size_t)kMaxRounds;      // u32[kMaxRounds]
constexpr size_t kOffFkey = align256(kOffFront + 4 * (size_t)kMaxRounds);  // u64[kMaxCells]
constexpr size_t kOffFcell = kOffFkey + 8 * kMaxCells;                // u32[kMaxCells]
constexpr size_t kOffCand = kOffFcell + 4 * kMaxCells;                // u32[kMaxCells]
constexpr size_t kOffBitmap = kOffCand + 4 * kMaxCells;               // u32[kMaxCells/32 + 1]
constexpr size_t kScratchBytes = align256(kOffBitmap + 4 * (kMaxCells / 32 + 1));
static_assert(sizeof(DecodeCtl) <= kOffSum, "DecodeCtl outgrew its slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array on the current device, looked up on
// every call (the first call on a device also loads the module there).
pp_status scratch_for_current_device(unsigned char **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
  *out = static_cast<unsigned char *>(p);
  return PP_OK;
}

// Sum of all cell counts (each key adds r to it), for the capacity check.
__global__ void k_count_sum(const Cell *__restrict__ cells, u64 n, long long *__restrict__ sum) {
  __shared__ long long s_red[kBlock / 32];
  long long v = 0;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
    v += cells[i].count;
  const long long b = block_sum<long long, kBlock>(v, s_red);
  if (threadIdx.x == 0 && b) atomicAdd(reinterpret_cast<unsigned long long *>(sum), (unsigned long long)b);
}

}  // namespace

extern "C" pp_status pp_iblt_decode_noalloc(pp_cell *d_cells, uint64_t n_cells, uint32_t r,
                                            uint64_t seed, uint64_t *d_out_keys, uint64_t out_cap,
                                            pp_decode_result *res, void *stream) {
  if (!d_cells || !res) return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode_noalloc: NULL cells or result");
  if (r < 2 || r > PP_MAX_R)
    return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode_noalloc: r=%u outside 2..%d", r, PP_MAX_R);
  if (n_cells < r || n_cells > kMaxCells)
    return fail(PP_ERR_INVALID_ARG,
                "pp_iblt_decode_noalloc: n_cells=%llu outside r..%llu (the fixed scratch holds at most "
                "PP_NOALLOC_MAX_CELLS cells)",
                (unsigned long long)n_cells, (unsigned long long)kMaxCells);
  if (out_cap && !d_out_keys) return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode_noalloc: NULL output");
  if (reinterpret_cast<uintptr_t>(d_cells) % 32 != 0 || reinterpret_cast<uintptr_t>(d_out_keys) % 8 != 0)
    return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode_noalloc: d_cells must be 32-byte and d_out_keys 8-byte aligned");
  unsigned char *scratch = nullptr;
  pp_status st = scratch_for_current_device(&scratch);
  if (st != PP_OK) return st;
  cudaStream_t s = as_stream(stream);
  DecodeCtl *ctl = reinterpret_cast<DecodeCtl *>(scratch + kOffCtl);
  long long *sum = reinterpret_cast<long long *>(scratch + kOffSum);
  u64 *st_rec = reinterpret_cast<u64 *>(scratch + kOffRec);
  u64 *st_alive = reinterpret_cast<u64 *>(scratch + kOffAlive);
  u32 *st_front = reinterpret_cast<u32 *>(scratch + kOffFront);
  u64 *fkey = reinterpret_cast<u64 *>(scratch + kOffFkey);
  u32 *fcell = reinterpret_cast<u32 *>(scratch + kOffFcell);
  u32 *cand = reinterpret_cast<u32 *>(scratch + kOffCand);
  u32 *bitmap = reinterpret_cast<u32 *>(scratch + kOffBitmap);
  Cell *cells = reinterpret_cast<Cell *>(d_cells);

  // Items in the table: every key adds r to the sum of counts.
  PP_CUDA(cudaMemsetAsync(sum, 0, sizeof(long long), s));
  const int grid_sum = sm_count() * 4;
  k_count_sum<<<grid_sum, kBlock, 0, s>>>(cells, n_cells, sum);
  PP_CUDA(cudaGetLastError());
  long long count_sum = 0;
  PP_CUDA(cudaMemcpyAsync(&count_sum, sum, sizeof count_sum, cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaStreamSynchronize(s));
  const uint64_t items = count_sum > 0 ? (uint64_t)count_sum / r : 0;
  if (out_cap < items)
    return fail(PP_ERR_CAPACITY, "pp_iblt_decode_noalloc: out_cap=%llu < %llu keys in the table",
                (unsigned long long)out_cap, (unsigned long long)items);

  // Fresh control block (the only scratch that must start from zero).
  DecodeCtl hc;
  memset(&hc, 0, sizeof hc);
  hc.out = reinterpret_cast<u64 *>(d_out_keys);
  hc.out_cap = out_cap;
  hc.max_rounds = kMaxRounds;
  PP_CUDA(cudaMemcpyAsync(ctl, &hc, sizeof hc, cudaMemcpyHostToDevice, s));

  TableArgs tab0;
  make_table_args(tab0, n_cells, r, seed, 0);
  const IbltKernels k = iblt_kernels((int)r, false);
  const size_t smem_peel = peel_smem_bytes(k.nr, false);
  const int grid_scan = persistent_grid(k.scan, kBlock, 0, 8);
  const int grid_peel = persistent_grid(k.peel, kBlock, smem_peel, 8);
  const int grid_filter = persistent_grid(k.filter, kBlock, 0, 8);

  const TableArgs *no_tabs = nullptr;
  const Chunk *no_chunks = nullptr;
  u32 *no_u32 = nullptr;
  u64 *no_u64 = nullptr;
  BatchCounters bc{};
  u32 n_chunks = (u32)((n_cells + kBlock * kScanItems - 1) / (kBlock * kScanItems));
  void *scan_args[] = {&cells, &tab0, &no_tabs, &no_chunks, &n_chunks, &fkey, &fcell, &no_u32,
                       &bitmap, &ctl, &bc};
  void *peel_args[] = {&cells, &tab0, &no_tabs, &fkey, &fcell, &no_u32, &bitmap, &cand, &no_u32,
                       &no_u64, &ctl, &bc};
  void *filter_args[] = {&cells, &tab0, &no_tabs, &cand, &no_u32, &fkey, &fcell, &no_u32, &bitmap, &ctl, &bc};
  RoundStats rs{st_rec, st_alive, st_front};
  int set_cond = 0;
  cudaGraphConditionalHandle no_cond = 0;
  void *end_args[] = {&ctl, &rs, &set_cond, &no_cond};

  PP_CUDA(cudaLaunchKernel(k.scan, dim3(grid_scan), dim3(kBlock), scan_args, 0, s));
  for (;;) {
    PP_CUDA(cudaLaunchKernel(k.peel, dim3(grid_peel), dim3(kBlock), peel_args, smem_peel, s));
    PP_CUDA(cudaLaunchKernel(k.filter, dim3(grid_filter), dim3(kBlock), filter_args, 0, s));
    PP_CUDA(cudaLaunchKernel(round_end_kernel(), dim3(1), dim3(32), end_args, 0, s));
    u32 more = 0;
    PP_CUDA(cudaMemcpyAsync(&more, &ctl->more, sizeof more, cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
    if (!more) break;
  }
  PP_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof hc, cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaStreamSynchronize(s));

  // Per-round figures go straight into the caller's arrays.
  const uint32_t T = hc.round;
  const uint32_t ncopy = T < res->round_cap ? T : res->round_cap;
  uint64_t *rec_dst = res->recovered_per_round ? res->recovered_per_round : res->remaining_per_round;
  if (ncopy && rec_dst)
    PP_CUDA(cudaMemcpyAsync(rec_dst, st_rec, ncopy * sizeof(u64), cudaMemcpyDeviceToHost, s));
  if (ncopy && res->alive_cells_per_round)
    PP_CUDA(cudaMemcpyAsync(res->alive_cells_per_round, st_alive, ncopy * sizeof(u64),
                            cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaStreamSynchronize(s));
  if (ncopy && res->remaining_per_round) {
    uint64_t left = items;
    for (uint32_t i = 0; i < ncopy; ++i) {
      const uint64_t got = rec_dst[i];
      left -= got <= left ? got : left;
      res->remaining_per_round[i] = left;
    }
  }
  res->rounds = T;
  res->status_flags = hc.flags;
  res->recovered = hc.n_out < out_cap ? hc.n_out : out_cap;
  res->items_before = items;
  res->residual_cells = hc.nonempty - hc.emptied;
  if (hc.flags & FLAG_CAPACITY)
    return fail(PP_ERR_CAPACITY, "pp_iblt_decode_noalloc: more keys recovered than out_cap=%llu",
                (unsigned long long)out_cap);
  if (hc.flags & FLAG_INTERNAL)
    return fail(PP_ERR_INVALID_ARG, "pp_iblt_decode_noalloc: a pure cell's key does not hash to it");
  if (hc.flags & FLAG_ROUND_LIMIT)
    return fail(PP_ERR_ROUND_LIMIT, "pp_iblt_decode_noalloc: stopped after %u rounds", kMaxRounds);
  return PP_OK;
}
