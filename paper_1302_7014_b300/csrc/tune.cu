// Autotuner of the batched engine: pp_tune_batch.
//
// The batch's run-time knobs -- resident blocks per SM of the round kernels
// (ctas_per_sm), of the binned apply (apply_ctas), the kind of update and
// round (binned = 1: address-ordered records; 2: direct atomics; rounds = 2:
// tile rounds, 1: binned or direct rounds) and the keys
// per insert work item (insert_chunk, which sets how finely a table's keys are
// spread over blocks) -- are searched on the caller's own batch: every
// candidate builds and decodes the batch `reps` times, timed with CUDA events
// on the caller's stream, and the fastest candidate whose per-table results
// equal those of the first one wins.  The batch keeps the winning options.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "host.cuh"

namespace {

struct Candidate {
  uint32_t ctas_per_sm, apply_ctas, binned, insert_chunk, rounds;
};

// One build + decode of the batch (pp_batch_build_decode); per-table results in res.
pp_status run_once(pp_batch *b, uint32_t n_tables, const uint64_t *d_keys, const uint64_t *h_key_offsets,
                   uint64_t *d_out, const uint64_t *h_out_offsets, std::vector<pp_table_result> &res,
                   cudaStream_t s) {
  res.assign(n_tables, pp_table_result{});
  return pp_batch_build_decode(b, d_keys, h_key_offsets, d_out, h_out_offsets, res.data(), s);
}

bool same_results(const std::vector<pp_table_result> &a, const std::vector<pp_table_result> &b) {
  if (a.size() != b.size()) return false;
  for (size_t i = 0; i < a.size(); ++i)
    if (a[i].rounds != b[i].rounds || a[i].recovered != b[i].recovered || a[i].residual_cells != b[i].residual_cells)
      return false;
  return true;
}

}  // namespace

extern "C" pp_status pp_tune_batch(pp_batch *b, const uint64_t *d_keys, const uint64_t *h_key_offsets,
                                   uint64_t *d_out_keys, const uint64_t *h_out_offsets, uint32_t reps,
                                   pp_options *best, pp_tune_report *report, float *h_ms, void *stream) {
  using namespace pp;
  if (!b || !h_key_offsets || !h_out_offsets || !best || !report)
    return fail(PP_ERR_INVALID_ARG, "pp_tune_batch: NULL argument");
  if (reps == 0 || reps > 64) return fail(PP_ERR_INVALID_ARG, "pp_tune_batch: reps=%u outside 1..64", reps);
  uint32_t n_tables = 0;
  uint64_t total = 0;
  pp_status st = pp_batch_info(b, &n_tables, &total, nullptr);
  if (st != PP_OK) return st;
  pp_options base;
  st = pp_batch_get_options(b, &base);
  if (st != PP_OK) return st;
  cudaStream_t s = as_stream(stream);

  std::vector<Candidate> cands;
  cands.push_back(Candidate{base.ctas_per_sm, base.apply_ctas, base.binned, base.insert_chunk, base.rounds});
  // tile rounds (their grids are fixed; the build's work items vary)
  for (uint32_t k : {1024u, 4096u, 16384u}) cands.push_back(Candidate{base.ctas_per_sm, base.apply_ctas, 1u, k, 2u});
  // binned rounds
  for (uint32_t c : {2u, 4u, 8u})
    for (uint32_t a : {2u, 3u, 4u}) cands.push_back(Candidate{c, a, 1u, base.insert_chunk, 1u});
  // direct-atomic rounds
  for (uint32_t c : {2u, 4u, 8u})
    for (uint32_t k : {1024u, 4096u, 16384u}) cands.push_back(Candidate{c, base.apply_ctas, 2u, k, 1u});
  if (cands.size() > PP_TUNE_MAX_CANDIDATES) cands.resize(PP_TUNE_MAX_CANDIDATES);

  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PP_CUDA(cudaEventCreate(&e0));
  PP_CUDA(cudaEventCreate(&e1));
  std::vector<pp_table_result> ref, got;
  float best_ms = 0.f, first_ms = 0.f;
  int best_i = -1;
  uint32_t mismatches = 0;
  for (size_t i = 0; i < cands.size() && st == PP_OK; ++i) {
    pp_options o = base;
    o.ctas_per_sm = cands[i].ctas_per_sm;
    o.apply_ctas = cands[i].apply_ctas;
    o.binned = cands[i].binned;
    o.insert_chunk = cands[i].insert_chunk;
    o.rounds = cands[i].rounds;
    st = pp_batch_set_options(b, &o);
    if (st != PP_OK) break;
    st = run_once(b, n_tables, d_keys, h_key_offsets, d_out_keys, h_out_offsets, got, s);  // warm-up, graphs
    if (st != PP_OK) break;
    if (i == 0) ref = got;
    const bool same = same_results(ref, got);
    std::vector<float> t;
    for (uint32_t k = 0; k < reps && st == PP_OK; ++k) {
      cudaEventRecord(e0, s);
      st = run_once(b, n_tables, d_keys, h_key_offsets, d_out_keys, h_out_offsets, got, s);
      cudaEventRecord(e1, s);
      if (st != PP_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = fail(PP_ERR_CUDA, "pp_tune_batch: event synchronize failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      t.push_back(ms);
    }
    if (st != PP_OK) break;
    std::sort(t.begin(), t.end());
    const float med = t[t.size() / 2];
    if (h_ms) h_ms[i] = same ? med : -1.f;
    if (i == 0) first_ms = med;
    if (!same) {
      ++mismatches;
      continue;
    }
    if (best_i < 0 || med < best_ms) {
      best_ms = med;
      best_i = (int)i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != PP_OK) {
    pp_batch_set_options(b, &base);
    return st;
  }
  *best = base;
  best->ctas_per_sm = cands[best_i].ctas_per_sm;
  best->apply_ctas = cands[best_i].apply_ctas;
  best->binned = cands[best_i].binned;
  best->insert_chunk = cands[best_i].insert_chunk;
  best->rounds = cands[best_i].rounds;
  report->n_candidates = (uint32_t)cands.size();
  report->best_index = (uint32_t)best_i;
  report->default_ms = first_ms;
  report->best_ms = best_ms;
  report->mismatches = mismatches;
  report->pad = 0;
  return pp_batch_set_options(b, best);
}
