// C-ABI: a continuous-batching IBLT decode service.
//
// A host thread owns one device arena of cells and one of keys.  Requests wait
// in a FIFO queue until their table and key buffer fit in the arenas (memory-
// based admission) and a slot is free.  The thread runs device iterations; one
// iteration is one round of the round-synchronous decode (Sec. 1 at k = 2, on
// the IBLT hypergraph of Sec. 6) for every admitted table at once:
//   peel   the current frontier of all active tables;
//   filter the candidates into the next frontier;
//   admit  tables that arrived since the last iteration: zero their cells,
//          load (or generate) their keys, insert them, and scan them, which
//          puts their first frontier into the same next frontier;
//   end    promote the next frontier.
// So a request that arrives while others are on the GPU joins them at the next
// round boundary and its rounds overlap theirs.  Tables never share cells, so
// each request's result is the result of decoding it alone.  A table is done
// when it has no entries in the frontier being built; its slot and arena
// ranges are then freed.
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string.h>
#include <thread>
#include <chrono>
#include <unordered_map>
#include <vector>

#include "host.cuh"
#include "iblt_types.cuh"

using namespace pp;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) in units (cells or keys), 32-unit aligned.
class RangeAlloc {
 public:
  explicit RangeAlloc(uint64_t size = 0) { reset(size); }
  void reset(uint64_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  bool alloc(uint64_t n, uint64_t *off) {
    n = (n + 31) & ~31ull;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const uint64_t rest = it->second - n, start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t n) {
    n = (n + 31) & ~31ull;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
 private:
  std::map<uint64_t, uint64_t> free_;
};

struct GenChunk {
  u64 seed;        // SplitMix64 seed of the request's keys
  u32 begin, end;  // key slots in the key arena
  u32 first;       // index of the key at `begin` within the request's stream
  u32 pad;
};

// Synthetic request keys: key i = SplitMix64 output i (mix(seed + (i+1) * gamma)).
__global__ void k_gen_keys(u64 *__restrict__ keys, const GenChunk *__restrict__ chunks, u32 n_chunks) {
  for (u32 ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const GenChunk g = chunks[ch];
    for (u32 i = g.begin + threadIdx.x; i < g.end; i += blockDim.x)
      keys[i] = mix64(g.seed + (u64)(g.first + (i - g.begin) + 1) * kGamma);
  }
}

// Reset the per-table counters of newly admitted slots.
__global__ void k_reset_slots(const u32 *__restrict__ slots, u32 n, BatchCounters bc) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const u32 s = slots[i];
    bc.recovered[s] = 0;
    bc.nonempty[s] = 0;
    bc.emptied[s] = 0;
    bc.rounds[s] = 0;
  }
}

constexpr u32 kChunk = 4096;

struct Job {
  uint64_t ticket = 0;
  pp_request req{};
  double arrival = 0, admitted = 0, done = 0;
  uint32_t slot = 0;
  uint64_t cell_off = 0, key_off = 0;
  int state = 0;  // 0 queued, 1 active, 2 done
  pp_request_result result{};
};

}  // namespace

struct pp_server {
  pp_server_config cfg{};
  IbltKernels k{};
  size_t smem_peel = 0;
  int grid_peel = 0, grid_filter = 0, grid_scan = 0, grid_insert = 0;
  cudaStream_t stream = nullptr;
  // device memory
  Cell *cells = nullptr;
  u64 *keys = nullptr, *fkey = nullptr;
  u32 *fcell = nullptr, *ftab = nullptr, *cand = nullptr, *ctab = nullptr, *bitmap = nullptr;
  TableArgs *tabs = nullptr;
  DecodeCtl *ctl = nullptr;
  BatchCounters bc{};
  Chunk *d_chunks = nullptr;
  GenChunk *d_gen = nullptr;
  u32 *d_slots = nullptr;
  uint32_t chunk_cap = 0, gen_cap = 0;
  // pinned staging
  TableArgs *h_tabs = nullptr;
  Chunk *h_chunks = nullptr;
  GenChunk *h_gen = nullptr;
  u32 *h_slots = nullptr;
  DecodeCtl *h_ctl = nullptr;
  u32 *h_live = nullptr, *h_rounds = nullptr;
  u64 *h_recovered = nullptr, *h_nonempty = nullptr, *h_emptied = nullptr;
  // host state (server thread)
  RangeAlloc cell_alloc, key_alloc;
  std::vector<uint32_t> free_slots;
  std::vector<Job *> active;
  // shared state
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job *> queue;
  std::unordered_map<uint64_t, Job *> jobs;
  uint64_t next_ticket = 1;
  bool stopping = false, drain = true;
  pp_status failed = PP_OK;
  std::string fail_msg;
  pp_server_stats stats{};
  double iter_s = 0, gpu_wait_s = 0;  // server thread only
  std::thread thread;
};

namespace {

pp_status alloc_server(pp_server *s) {
  const uint64_t C = s->cfg.arena_cells, K = s->cfg.arena_keys;
  const uint32_t S = s->cfg.max_slots;
  // per iteration: scan chunks (1024 cells), insert chunks (4096 keys), one partial of each per table
  s->chunk_cap = (uint32_t)(C / (kBlock * kScanItems) + K / kChunk + 2 * (uint64_t)S + 16);
  s->gen_cap = (uint32_t)(K / (1u << 20) + S + 16);
  cudaError_t e = cudaSuccess;
  auto al = [&](void **p, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(p, b ? b : 16);
  };
  auto ah = [&](void **p, size_t b) {
    if (e == cudaSuccess) e = cudaMallocHost(p, b ? b : 16);
  };
  al((void **)&s->cells, C * sizeof(Cell));
  al((void **)&s->keys, K * sizeof(u64));
  al((void **)&s->fkey, C * sizeof(u64));
  al((void **)&s->fcell, C * sizeof(u32));
  al((void **)&s->ftab, C * sizeof(u32));
  al((void **)&s->cand, C * sizeof(u32));
  al((void **)&s->ctab, C * sizeof(u32));
  al((void **)&s->bitmap, (C / 32 + 1) * sizeof(u32));
  al((void **)&s->tabs, S * sizeof(TableArgs));
  al((void **)&s->ctl, sizeof(DecodeCtl));
  al((void **)&s->bc.recovered, S * sizeof(u64));
  al((void **)&s->bc.nonempty, S * sizeof(u64));
  al((void **)&s->bc.emptied, S * sizeof(u64));
  al((void **)&s->bc.rounds, S * sizeof(u32));
  al((void **)&s->bc.live, S * sizeof(u32));
  al((void **)&s->d_chunks, s->chunk_cap * sizeof(Chunk));
  al((void **)&s->d_gen, s->gen_cap * sizeof(GenChunk));
  al((void **)&s->d_slots, S * sizeof(u32));
  ah((void **)&s->h_tabs, S * sizeof(TableArgs));
  ah((void **)&s->h_chunks, s->chunk_cap * sizeof(Chunk));
  ah((void **)&s->h_gen, s->gen_cap * sizeof(GenChunk));
  ah((void **)&s->h_slots, S * sizeof(u32));
  ah((void **)&s->h_ctl, sizeof(DecodeCtl));
  ah((void **)&s->h_live, S * sizeof(u32));
  ah((void **)&s->h_rounds, S * sizeof(u32));
  ah((void **)&s->h_recovered, S * sizeof(u64));
  ah((void **)&s->h_nonempty, S * sizeof(u64));
  ah((void **)&s->h_emptied, S * sizeof(u64));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemset(s->bitmap, 0, (C / 32 + 1) * sizeof(u32));
  if (e == cudaSuccess) memset(s->h_ctl, 0, sizeof(DecodeCtl));
  if (e == cudaSuccess) {
    DecodeCtl c;
    memset(&c, 0, sizeof c);
    c.max_rounds = 0xFFFFFFFFu;
    e = cudaMemcpy(s->ctl, &c, sizeof c, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "pp_server_start allocation", __FILE__, __LINE__);
  return PP_OK;
}

void free_server(pp_server *s) {
  if (s->stream) cudaStreamDestroy(s->stream);
  void *dev[] = {s->cells, s->keys, s->fkey, s->fcell, s->ftab, s->cand, s->ctab, s->bitmap, s->tabs,
                 s->ctl, s->bc.recovered, s->bc.nonempty, s->bc.emptied, s->bc.rounds, s->bc.live,
                 s->d_chunks, s->d_gen, s->d_slots};
  for (void *p : dev) cudaFree(p);
  void *host[] = {s->h_tabs, s->h_chunks, s->h_gen, s->h_slots, s->h_ctl, s->h_live, s->h_rounds,
                  s->h_recovered, s->h_nonempty, s->h_emptied};
  for (void *p : host) cudaFreeHost(p);
  for (auto &kv : s->jobs) delete kv.second;
  delete s;
}

#define SV_CUDA(call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) {                                 \
      err = cuda_fail(e_, #call, __FILE__, __LINE__);        \
      return false;                                          \
    }                                                        \
  } while (0)

// One device iteration.  Returns false on a CUDA error (err set).
bool iterate(pp_server *s, std::vector<Job *> &admit, pp_status &err) {
  cudaStream_t st = s->stream;
  const uint32_t S = s->cfg.max_slots;
  BatchCounters bc = s->bc;
  bc.round_rec = nullptr;
  TableArgs t0{};
  RoundStats rs{nullptr, nullptr, nullptr};
  // current round number (read back last iteration) decides new tables' round 1
  const u32 round_now = s->h_ctl->round;
  SV_CUDA(cudaMemsetAsync(s->bc.live, 0, S * sizeof(u32), st));
  {
    // peel + filter for the tables already in the frontier
    Cell *cells = s->cells;
    const TableArgs *tabs = s->tabs;
    const u64 *fk = s->fkey;
    const u32 *fc = s->fcell, *ft = s->ftab, *bm = s->bitmap;
    u32 *cand = s->cand, *ctab = s->ctab;
    u64 *out = s->keys;
    DecodeCtl *ctl = s->ctl;
    void *pa[] = {&cells, &t0, &tabs, &fk, &fc, &ft, &bm, &cand, &ctab, &out, &ctl, &bc};
    SV_CUDA(cudaLaunchKernel(s->k.peel, dim3(s->grid_peel), dim3(kBlock), pa, s->smem_peel, st));
    const Cell *cc = s->cells;
    const u32 *cd = s->cand, *ct = s->ctab;
    u64 *fkw = s->fkey;
    u32 *fcw = s->fcell, *ftw = s->ftab, *bmw = s->bitmap;
    void *fa[] = {&cc, &t0, &tabs, &cd, &ct, &fkw, &fcw, &ftw, &bmw, &ctl, &bc};
    SV_CUDA(cudaLaunchKernel(s->k.filter, dim3(s->grid_filter), dim3(kBlock), fa, 0, st));
  }
  if (!admit.empty()) {
    // new tables: arguments, counters, zeroed cells, keys, insert, scan
    uint32_t n_gen = 0, n_ins = 0, n_scan = 0, n_slots = 0;
    std::vector<Chunk> ins, scan;
    for (Job *j : admit) {
      const pp_request &q = j->req;
      TableArgs &ta = s->h_tabs[j->slot];
      make_table_args(ta, q.n_cells, q.r, q.table_seed, (uint32_t)j->cell_off);
      ta.start_round = round_now + 1;
      ta.out_base = j->key_off;
      ta.out_cap = q.m;
      SV_CUDA(cudaMemcpyAsync(s->tabs + j->slot, &s->h_tabs[j->slot], sizeof(TableArgs),
                              cudaMemcpyHostToDevice, st));
      SV_CUDA(cudaMemsetAsync(s->cells + j->cell_off, 0, q.n_cells * sizeof(Cell), st));
      s->h_slots[n_slots++] = j->slot;
      if (q.m) {
        if (q.h_keys) {
          SV_CUDA(cudaMemcpyAsync(s->keys + j->key_off, q.h_keys, q.m * sizeof(u64),
                                  cudaMemcpyHostToDevice, st));
        } else {
          for (uint64_t k = 0; k < q.m; k += (1u << 20)) {
            const uint64_t e = k + (1u << 20) < q.m ? k + (1u << 20) : q.m;
            s->h_gen[n_gen++] = GenChunk{q.key_seed, (u32)(j->key_off + k), (u32)(j->key_off + e), (u32)k, 0};
          }
        }
        for (uint64_t k = 0; k < q.m; k += kChunk)
          ins.push_back(Chunk{j->slot, (u32)(j->key_off + k), (u32)(j->key_off + (k + kChunk < q.m ? k + kChunk : q.m))});
      }
      for (uint64_t c = 0; c < q.n_cells; c += kBlock * kScanItems)
        scan.push_back(Chunk{j->slot, (u32)(j->cell_off + c),
                             (u32)(j->cell_off + (c + kBlock * kScanItems < q.n_cells ? c + kBlock * kScanItems : q.n_cells))});
    }
    n_ins = (uint32_t)ins.size();
    n_scan = (uint32_t)scan.size();
    if (n_ins + n_scan > s->chunk_cap) {
      err = fail(PP_ERR_CAPACITY, "server: chunk staging overflow");
      return false;
    }
    memcpy(s->h_chunks, ins.data(), n_ins * sizeof(Chunk));
    memcpy(s->h_chunks + n_ins, scan.data(), n_scan * sizeof(Chunk));
    SV_CUDA(cudaMemcpyAsync(s->d_chunks, s->h_chunks, (n_ins + n_scan) * sizeof(Chunk), cudaMemcpyHostToDevice, st));
    SV_CUDA(cudaMemcpyAsync(s->d_slots, s->h_slots, n_slots * sizeof(u32), cudaMemcpyHostToDevice, st));
    k_reset_slots<<<1, 256, 0, st>>>(s->d_slots, n_slots, s->bc);
    if (n_gen) {
      SV_CUDA(cudaMemcpyAsync(s->d_gen, s->h_gen, n_gen * sizeof(GenChunk), cudaMemcpyHostToDevice, st));
      k_gen_keys<<<s->grid_insert, 256, 0, st>>>(s->keys, s->d_gen, n_gen);
    }
    Cell *cells = s->cells;
    const TableArgs *tabs = s->tabs;
    if (n_ins) {
      const Chunk *ch = s->d_chunks;
      u32 nch = n_ins;
      const u64 *keys = s->keys;
      u64 m = 0;
      int sign = 1;
      void *ia[] = {&cells, &t0, &tabs, &ch, &nch, &keys, &m, &sign};
      SV_CUDA(cudaLaunchKernel(s->k.insert, dim3(nch < (u32)s->grid_insert ? nch : s->grid_insert),
                               dim3(kBlock), ia, 0, st));
    }
    {
      const Chunk *ch = s->d_chunks + n_ins;
      u32 nch = n_scan;
      u64 *fk = s->fkey;
      u32 *fc = s->fcell, *ft = s->ftab, *bm = s->bitmap;
      DecodeCtl *ctl = s->ctl;
      void *sa[] = {&cells, &t0, &tabs, &ch, &nch, &fk, &fc, &ft, &bm, &ctl, &bc};
      SV_CUDA(cudaLaunchKernel(s->k.scan, dim3(nch < (u32)s->grid_scan ? nch : s->grid_scan), dim3(kBlock),
                               sa, 0, st));
    }
  }
  {
    DecodeCtl *ctl = s->ctl;
    int set_cond = 0;
    cudaGraphConditionalHandle cond = 0;
    void *ea[] = {&ctl, &rs, &set_cond, &cond};
    SV_CUDA(cudaLaunchKernel(round_end_kernel(), dim3(1), dim3(32), ea, 0, st));
  }
  SV_CUDA(cudaMemcpyAsync(s->h_ctl, s->ctl, sizeof(DecodeCtl), cudaMemcpyDeviceToHost, st));
  SV_CUDA(cudaMemcpyAsync(s->h_live, s->bc.live, S * sizeof(u32), cudaMemcpyDeviceToHost, st));
  SV_CUDA(cudaMemcpyAsync(s->h_rounds, s->bc.rounds, S * sizeof(u32), cudaMemcpyDeviceToHost, st));
  SV_CUDA(cudaMemcpyAsync(s->h_recovered, s->bc.recovered, S * sizeof(u64), cudaMemcpyDeviceToHost, st));
  SV_CUDA(cudaMemcpyAsync(s->h_nonempty, s->bc.nonempty, S * sizeof(u64), cudaMemcpyDeviceToHost, st));
  SV_CUDA(cudaMemcpyAsync(s->h_emptied, s->bc.emptied, S * sizeof(u64), cudaMemcpyDeviceToHost, st));
  {
    const double w0 = now_s();
    SV_CUDA(cudaStreamSynchronize(st));
    s->gpu_wait_s += now_s() - w0;
  }
  if (s->h_ctl->flags & (FLAG_CAPACITY | FLAG_INTERNAL)) {
    err = fail(PP_ERR_CUDA, "server: device flags 0x%x", s->h_ctl->flags);
    return false;
  }
  return true;
}

void complete_finished(pp_server *s, pp_status &err) {
  std::vector<Job *> still;
  std::vector<Job *> finished;
  for (Job *j : s->active) {
    if (s->h_live[j->slot] == 0) finished.push_back(j);
    else still.push_back(j);
  }
  if (finished.empty()) return;
  bool copies = false;
  for (Job *j : finished) {
    pp_request_result &r = j->result;
    r.rounds = s->h_rounds[j->slot];
    r.recovered = s->h_recovered[j->slot];
    r.residual_cells = s->h_nonempty[j->slot] - s->h_emptied[j->slot];
    r.items_before = j->req.m;
    if (j->req.h_out && r.recovered) {
      const uint64_t n = r.recovered < j->req.out_cap ? r.recovered : j->req.out_cap;
      if (cudaMemcpyAsync(j->req.h_out, s->keys + j->key_off, n * sizeof(u64), cudaMemcpyDeviceToHost,
                          s->stream) != cudaSuccess)
        err = fail(PP_ERR_CUDA, "server: result copy failed");
      copies = true;
    }
  }
  if (copies && cudaStreamSynchronize(s->stream) != cudaSuccess) err = fail(PP_ERR_CUDA, "server: result sync failed");
  const double t = now_s();
  std::lock_guard<std::mutex> lock(s->mu);
  for (Job *j : finished) {
    j->done = t;
    j->result.done_s = t;
    j->result.status = PP_OK;
    j->state = 2;
    s->cell_alloc.release(j->cell_off, j->req.n_cells);
    s->key_alloc.release(j->key_off, j->req.m ? j->req.m : 1);
    s->free_slots.push_back(j->slot);
    s->stats.completed++;
    s->stats.keys_recovered += j->result.recovered;
  }
  s->active.swap(still);
  s->stats.active = s->active.size();
  s->cv_done.notify_all();
}

void server_main(pp_server *s) {
  cudaSetDevice(s->cfg.device);
  pp_status err = PP_OK;
  std::vector<Job *> admit;
  for (;;) {
    admit.clear();
    {
      std::unique_lock<std::mutex> lock(s->mu);
      if (s->active.empty() && s->queue.empty()) {
        if (s->stopping) break;
        s->cv_work.wait_for(lock, std::chrono::microseconds(200));
        if (s->active.empty() && s->queue.empty()) continue;
      }
      if (s->stopping && !s->drain) break;
      // strict FIFO admission by free arena space and slots
      while (!s->queue.empty()) {
        Job *j = s->queue.front();
        uint64_t co = 0, ko = 0;
        if (s->free_slots.empty()) break;
        if (!s->cell_alloc.alloc(j->req.n_cells, &co)) break;
        if (!s->key_alloc.alloc(j->req.m ? j->req.m : 1, &ko)) {
          s->cell_alloc.release(co, j->req.n_cells);
          break;
        }
        j->cell_off = co;
        j->key_off = ko;
        j->slot = s->free_slots.back();
        s->free_slots.pop_back();
        j->state = 1;
        j->admitted = now_s();
        j->result.admit_s = j->admitted;
        s->queue.pop_front();
        admit.push_back(j);
        s->stats.admitted++;
      }
      s->stats.pending = s->queue.size();
    }
    for (Job *j : admit) s->active.push_back(j);
    const double t0 = now_s();
    if (!iterate(s, admit, err)) break;
    complete_finished(s, err);
    {
      std::lock_guard<std::mutex> lock(s->mu);
      s->stats.iterations++;
      s->stats.iteration_us = (uint64_t)((s->iter_s += now_s() - t0) * 1e6);
      s->stats.gpu_wait_us = (uint64_t)(s->gpu_wait_s * 1e6);
    }
    if (err != PP_OK) break;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  if (err != PP_OK) {
    s->failed = err;
    s->fail_msg = pp_last_error();
  }
  // anything left is cancelled
  for (auto &kv : s->jobs) {
    Job *j = kv.second;
    if (j->state != 2) {
      j->state = 2;
      j->result.status = err != PP_OK ? err : PP_ERR_TIMEOUT;
      j->result.done_s = now_s();
    }
  }
  s->cv_done.notify_all();
}

}  // namespace

extern "C" {

double pp_server_now(void) { return now_s(); }

void pp_server_config_default(pp_server_config *c) {
  if (!c) return;
  memset(c, 0, sizeof *c);
  c->arena_cells = 1ull << 26;
  c->arena_keys = 1ull << 26;
  c->max_slots = 4096;
  c->max_queue = 1u << 20;
  c->r = 0;
  c->device = 0;
}

pp_status pp_server_start(pp_server **out, const pp_server_config *cfg, const pp_options *opt) {
  if (!out || !cfg) return fail(PP_ERR_INVALID_ARG, "pp_server_start: NULL argument");
  *out = nullptr;
  if (cfg->arena_cells < 64 || cfg->arena_cells > 0xFFFFFFFFull - 64 || cfg->arena_keys < 32 ||
      cfg->arena_keys > 0xFFFFFFFFull - 64 || cfg->max_slots == 0 || (cfg->r && (cfg->r < 2 || cfg->r > PP_MAX_R)))
    return fail(PP_ERR_INVALID_ARG, "pp_server_start: bad configuration");
  pp_server *s = new pp_server();
  s->cfg = *cfg;
  if (!s->cfg.max_queue) s->cfg.max_queue = 1u << 20;
  const pp_options o = resolve_options(opt);
  cudaError_t e = cudaSetDevice(cfg->device);
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "cudaSetDevice", __FILE__, __LINE__);
  }
  // scattered 32-byte cell reads: one sector fetched from DRAM, not two
  if (o.l2_fetch == 1) cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, 32);
  s->k = iblt_kernels((int)cfg->r, true);
  s->smem_peel = peel_smem_bytes(s->k.nr, true);
  pp_status st = alloc_server(s);
  if (st != PP_OK) {
    free_server(s);
    return st;
  }
  s->grid_peel = persistent_grid(s->k.peel, kBlock, s->smem_peel, o.ctas_per_sm);
  s->grid_filter = persistent_grid(s->k.filter, kBlock, 0, o.ctas_per_sm);
  s->grid_scan = persistent_grid(s->k.scan, kBlock, 0, o.ctas_per_sm);
  s->grid_insert = persistent_grid(s->k.insert, kBlock, 0, 8) * 2;
  s->cell_alloc.reset(cfg->arena_cells);
  s->key_alloc.reset(cfg->arena_keys);
  for (uint32_t i = cfg->max_slots; i > 0; --i) s->free_slots.push_back(i - 1);
  s->thread = std::thread(server_main, s);
  *out = s;
  return PP_OK;
}

pp_status pp_server_submit(pp_server *s, const pp_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket) return fail(PP_ERR_INVALID_ARG, "pp_server_submit: NULL argument");
  const uint32_t r = req->r;
  if (r < 2 || r > PP_MAX_R || (s->cfg.r && r != s->cfg.r) || req->n_cells < r)
    return fail(PP_ERR_INVALID_ARG, "pp_server_submit: r=%u / n_cells=%llu not served", r,
                (unsigned long long)req->n_cells);
  if (((req->n_cells + 31) & ~31ull) > s->cfg.arena_cells || ((req->m + 31) & ~31ull) > s->cfg.arena_keys)
    return fail(PP_ERR_CAPACITY, "pp_server_submit: request larger than the server's arenas");
  if (req->h_out && req->out_cap < req->m)
    return fail(PP_ERR_CAPACITY, "pp_server_submit: out_cap < m");
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->failed != PP_OK) return fail(s->failed, "pp_server_submit: server failed: %s", s->fail_msg.c_str());
  if (s->stopping) return fail(PP_ERR_BUSY, "pp_server_submit: server is stopping");
  if (s->queue.size() >= s->cfg.max_queue) {
    s->stats.rejected++;
    return fail(PP_ERR_BUSY, "pp_server_submit: queue full");
  }
  Job *j = new Job();
  j->ticket = s->next_ticket++;
  j->req = *req;
  j->arrival = req->arrival_s > 0 ? req->arrival_s : now_s();
  j->result.ticket = j->ticket;
  j->result.arrival_s = j->arrival;
  s->jobs[j->ticket] = j;
  s->queue.push_back(j);
  s->stats.submitted++;
  *ticket = j->ticket;
  s->cv_work.notify_one();
  return PP_OK;
}

static pp_status take_result(pp_server *s, uint64_t ticket, pp_request_result *res, double timeout_s) {
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return fail(PP_ERR_NOT_FOUND, "pp_server: unknown ticket %llu", (unsigned long long)ticket);
  Job *j = it->second;
  if (j->state != 2 && timeout_s > 0) {
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    s->cv_done.wait_until(lock, until, [&] { return j->state == 2; });
  }
  if (j->state != 2)
    return timeout_s > 0 ? fail(PP_ERR_TIMEOUT, "pp_server_wait: ticket %llu not done", (unsigned long long)ticket)
                         : PP_ERR_BUSY;
  *res = j->result;
  s->jobs.erase(it);
  delete j;
  return res->status == PP_OK ? PP_OK : (pp_status)res->status;
}

pp_status pp_server_poll(pp_server *s, uint64_t ticket, pp_request_result *res) {
  if (!s || !res) return fail(PP_ERR_INVALID_ARG, "pp_server_poll: NULL argument");
  return take_result(s, ticket, res, 0.0);
}

pp_status pp_server_wait(pp_server *s, uint64_t ticket, double timeout_s, pp_request_result *res) {
  if (!s || !res) return fail(PP_ERR_INVALID_ARG, "pp_server_wait: NULL argument");
  return take_result(s, ticket, res, timeout_s > 0 ? timeout_s : 1e-6);
}

pp_status pp_server_get_stats(pp_server *s, pp_server_stats *out) {
  if (!s || !out) return fail(PP_ERR_INVALID_ARG, "pp_server_get_stats: NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->stats;
  out->pending = s->queue.size();
  return s->failed;
}

pp_status pp_server_stop(pp_server *s, int drain) {
  if (!s) return PP_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stopping = true;
    s->drain = drain != 0;
    s->cv_work.notify_all();
  }
  if (s->thread.joinable()) s->thread.join();
  const pp_status st = s->failed;
  cudaStreamSynchronize(s->stream);
  free_server(s);
  return st;
}

}  // extern "C"
