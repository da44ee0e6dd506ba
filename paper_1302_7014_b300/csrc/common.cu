// Status strings, error messages, options and per-table constants.
#include <string.h>

#include "host.cuh"

namespace pp {

static thread_local std::string g_last_error;

void set_error(const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

pp_status fail(pp_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

pp_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
  set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  return e == cudaErrorMemoryAllocation ? PP_ERR_OUT_OF_MEMORY : PP_ERR_CUDA;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

pp_options resolve_options(const pp_options *opt) {
  pp_options o;
  pp_options_default(&o);
  if (opt) {
    if (opt->block) o.block = opt->block;
    if (opt->ctas_per_sm) o.ctas_per_sm = opt->ctas_per_sm;
    if (opt->max_rounds) o.max_rounds = opt->max_rounds;
    o.host_loop = opt->host_loop;
    if (opt->stats_rounds) o.stats_rounds = opt->stats_rounds;
    o.binned = opt->binned;
    o.kcore_mode = opt->kcore_mode;
    o.rounds = opt->rounds;
    if (opt->apply_ctas) o.apply_ctas = opt->apply_ctas;
    if (opt->frontier_switch) o.frontier_switch = opt->frontier_switch;
    if (opt->insert_chunk) o.insert_chunk = opt->insert_chunk;
    if (opt->l2_fetch) o.l2_fetch = opt->l2_fetch;
  }
  return o;
}

void make_table_args(TableArgs &a, uint64_t n_cells, uint32_t r, uint64_t seed, uint32_t base) {
  memset(&a, 0, sizeof a);
  for (uint32_t j = 0; j <= r; ++j) a.seed[j] = mix64(seed + (uint64_t)(j + 1) * kGamma);
  const uint64_t q = n_cells / r, rem = n_cells % r;
  a.off[0] = 0;
  for (uint32_t j = 0; j < r; ++j) a.off[j + 1] = a.off[j] + (uint32_t)(q + (j < rem ? 1 : 0));
  a.base = base;
  a.n_cells = (uint32_t)n_cells;
  a.r = r;
  a.start_round = 1;
}

void allow_max_dynamic_smem(const void *fn) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa{};
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, fn) != cudaSuccess)
    return;
  const int room = optin - (int)fa.sharedSizeBytes;
  if (room > 0) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, room);
}

int persistent_grid(const void *fn, int block, size_t smem, uint32_t ctas_per_sm) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block, smem) != cudaSuccess || occ < 1)
    occ = 1;
  const int per_sm = (int)ctas_per_sm < occ ? (int)ctas_per_sm : occ;
  return sm_count() * (per_sm > 0 ? per_sm : 1);
}

}  // namespace pp

extern "C" {

void pp_options_default(pp_options *opt) {
  if (!opt) return;
  memset(opt, 0, sizeof *opt);
  opt->block = 256;
  opt->ctas_per_sm = 8;
  opt->max_rounds = 65535;
  opt->host_loop = 0;
  opt->stats_rounds = 128;
  opt->apply_ctas = 3;
  opt->frontier_switch = 2;
  opt->insert_chunk = 4096;
  opt->l2_fetch = 1;
}

const char *pp_status_string(pp_status s) {
  switch (s) {
    case PP_OK: return "PP_OK";
    case PP_ERR_INVALID_ARG: return "PP_ERR_INVALID_ARG";
    case PP_ERR_OUT_OF_MEMORY: return "PP_ERR_OUT_OF_MEMORY";
    case PP_ERR_CAPACITY: return "PP_ERR_CAPACITY";
    case PP_ERR_ROUND_LIMIT: return "PP_ERR_ROUND_LIMIT";
    case PP_ERR_TIMEOUT: return "PP_ERR_TIMEOUT";
    case PP_ERR_CUDA: return "PP_ERR_CUDA";
    case PP_ERR_BUSY: return "PP_ERR_BUSY";
    case PP_ERR_NOT_FOUND: return "PP_ERR_NOT_FOUND";
  }
  return "PP_ERR_UNKNOWN";
}

const char *pp_last_error(void) { return pp::g_last_error.c_str(); }

}  // extern "C"
