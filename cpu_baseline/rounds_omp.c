/* Round-synchronous IBLT build and decode on every host core (OpenMP).
 *
 * The CPU baseline that the GPU figures are set against: the method of Sec. 1
 * (each round removes every vertex of degree < k at once) applied to the IBLT
 * of Sec. 6 at k = 2, parallelised the obvious way on a multicore host:
 *   build   one key per loop iteration, atomic add / XOR on its r cells;
 *   scan    the cells pure before any round, in parallel;
 *   round   every frontier entry (cell c, key x read at the round's start)
 *           recovers x iff no cell of x in a lower sub-table was pure at the
 *           round's start (so a key pure in several cells is recovered once),
 *           and deletes x from its r cells with atomics; a cell whose count
 *           drops from 2 to 1 is a candidate, and the candidates still pure
 *           once every deletion of the round is done form the next frontier.
 * It is neither the oracle (which is plain and sequential) nor the GPU path,
 * and it shares code with neither.  The cell map and checksum follow the
 * table conventions the library documents (SplitMix64 seeds, multiply-high
 * range map, checkSum(x) = mix64(x ^ seed_r)).  Insert-only tables.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct {
  uint64_t seed[17];
  uint64_t off[17];
  uint32_t r;
} layout_t;

static void make_layout(layout_t *L, uint64_t n, uint32_t r, uint64_t table_seed) {
  L->r = r;
  for (uint32_t j = 0; j <= r; ++j) L->seed[j] = mix64(table_seed + (uint64_t)(j + 1) * GOLDEN);
  const uint64_t q = n / r, rem = n % r;
  L->off[0] = 0;
  for (uint32_t j = 0; j < r; ++j) L->off[j + 1] = L->off[j] + q + (j < rem ? 1 : 0);
}

static inline uint64_t cell(const layout_t *L, uint64_t x, uint32_t j) {
  const uint64_t size = L->off[j + 1] - L->off[j];
  return L->off[j] + (uint64_t)(((unsigned __int128)mix64(x ^ L->seed[j]) * size) >> 64);
}

static inline int pure(int64_t cnt, uint64_t key, uint64_t chk, const layout_t *L) {
  return cnt == 1 && chk == mix64(key ^ L->seed[L->r]);
}

int omp_threads(void) { return omp_get_max_threads(); }

/* count / keyx / chkx: n cells, zeroed by the caller. */
int omp_iblt_build(uint64_t n, uint32_t r, uint64_t table_seed, const uint64_t *keys, uint64_t m,
                   int64_t *count, uint64_t *keyx, uint64_t *chkx, int threads) {
  if (r < 2 || r > 16 || n < r) return 3;
  layout_t L;
  make_layout(&L, n, r, table_seed);
#pragma omp parallel for schedule(static) num_threads(threads)
  for (uint64_t i = 0; i < m; ++i) {
    const uint64_t x = keys[i], cs = mix64(x ^ L.seed[r]);
    for (uint32_t j = 0; j < r; ++j) {
      const uint64_t c = cell(&L, x, j);
      __atomic_fetch_add(&count[c], 1, __ATOMIC_RELAXED);
      __atomic_fetch_xor(&keyx[c], x, __ATOMIC_RELAXED);
      __atomic_fetch_xor(&chkx[c], cs, __ATOMIC_RELAXED);
    }
  }
  return 0;
}

/* Compacts per-thread segments: segment t holds got[t] entries at
 * base[t] of src (element size es); returns the total. */
static uint64_t compact(void *dst, const void *src, const uint64_t *base, const uint64_t *got, int nt, size_t es) {
  uint64_t at = 0;
  for (int t = 0; t < nt; ++t) {
    memmove((char *)dst + at * es, (const char *)src + base[t] * es, got[t] * es);
    at += got[t];
  }
  return at;
}

/* Decodes in place.  out_keys: the keys of round 1, 2, ... (unordered within a
 * round); round_end[t-1] = keys recovered in rounds 1..t; *rounds_out = rounds
 * that recovered a key.  Returns 0, 1 (out_cap too small), 2 (round limit),
 * 3 (invalid), 4 (no memory). */
int omp_iblt_decode(uint64_t n, uint32_t r, uint64_t table_seed, int64_t *count, uint64_t *keyx, uint64_t *chkx,
                    uint32_t max_rounds, uint64_t *out_keys, uint64_t out_cap, uint64_t *round_end,
                    uint32_t *rounds_out, int threads) {
  if (r < 2 || r > 16 || n < r) return 3;
  layout_t L;
  make_layout(&L, n, r, table_seed);
  const int nt = threads > 0 ? threads : omp_get_max_threads();
  const uint64_t words = n / 32 + 1;
  uint32_t *bits = (uint32_t *)calloc(words, 4);
  uint64_t *fkey = (uint64_t *)malloc(n * 8), *tkey = (uint64_t *)malloc(n * 8);
  uint64_t *fcell = (uint64_t *)malloc(n * 8), *tcell = (uint64_t *)malloc(n * 8);
  uint64_t *cand = (uint64_t *)malloc((uint64_t)r * n * 8);
  uint64_t base[1024], got[1024], got2[1024];
  int status = 0;
  if (!bits || !fkey || !tkey || !fcell || !tcell || !cand || nt > 1024) {
    status = 4;
    goto done;
  }
  /* F_1: the cells pure before any round; thread t writes at its own range */
#pragma omp parallel num_threads(nt)
  {
    const int t = omp_get_thread_num();
    const uint64_t lo = n * t / nt, hi = n * (t + 1) / nt;
    uint64_t k = 0;
    base[t] = lo;
    for (uint64_t c = lo; c < hi; ++c) {
      if (pure(count[c], keyx[c], chkx[c], &L)) {
        tkey[lo + k] = keyx[c];
        tcell[lo + k] = c;
        ++k;
        __atomic_fetch_or(&bits[c >> 5], 1u << (c & 31), __ATOMIC_RELAXED);
      }
    }
    got[t] = k;
  }
  uint64_t nf = compact(fkey, tkey, base, got, nt, 8);
  compact(fcell, tcell, base, got, nt, 8);
  uint64_t total = 0;
  uint32_t round = 0;
  while (nf > 0) {
    if (round == max_rounds) {
      status = 2;
      break;
    }
    /* claim and delete; winners go to tkey, 2 -> 1 crossings to cand */
#pragma omp parallel num_threads(nt)
    {
      const int t = omp_get_thread_num();
      const uint64_t lo = nf * t / nt, hi = nf * (t + 1) / nt;
      uint64_t k = 0, q = 0;
      base[t] = lo;
      for (uint64_t i = lo; i < hi; ++i) {
        const uint64_t x = fkey[i], c = fcell[i];
        uint64_t cj[16];
        int js = -1, win = 1;
        for (uint32_t j = 0; j < r; ++j) {
          cj[j] = cell(&L, x, j);
          if (js < 0 && cj[j] == c) js = (int)j;
        }
        for (int j = 0; j < js && win; ++j)
          if ((__atomic_load_n(&bits[cj[j] >> 5], __ATOMIC_RELAXED) >> (cj[j] & 31)) & 1u) win = 0;
        if (js < 0 || !win) continue;
        tkey[lo + k++] = x;
        const uint64_t cs = mix64(x ^ L.seed[r]);
        for (uint32_t j = 0; j < r; ++j) {
          const int64_t old = __atomic_fetch_sub(&count[cj[j]], 1, __ATOMIC_RELAXED);
          __atomic_fetch_xor(&keyx[cj[j]], x, __ATOMIC_RELAXED);
          __atomic_fetch_xor(&chkx[cj[j]], cs, __ATOMIC_RELAXED);
          if (old == 2) cand[(uint64_t)r * lo + q++] = cj[j];
        }
      }
      got[t] = k;
      got2[t] = q;
    }
    uint64_t nw = 0;
    for (int t = 0; t < nt; ++t) nw += got[t];
    if (total + nw > out_cap) {
      status = 1;
      break;
    }
    total += compact(out_keys + total, tkey, base, got, nt, 8);
    round_end[round] = total;
    ++round;
    /* candidates still pure form F_{t+1} */
    for (int t = 0; t < nt; ++t) base[t] *= r;
    const uint64_t ncand = compact(cand, cand, base, got2, nt, 8);
#pragma omp parallel num_threads(nt)
    {
      const int t = omp_get_thread_num();
      const uint64_t lo = ncand * t / nt, hi = ncand * (t + 1) / nt;
      uint64_t k = 0;
      base[t] = lo;
      for (uint64_t i = lo; i < hi; ++i) {
        const uint64_t c = cand[i];
        if (pure(count[c], keyx[c], chkx[c], &L)) {
          tkey[lo + k] = keyx[c];
          tcell[lo + k] = c;
          ++k;
          __atomic_fetch_or(&bits[c >> 5], 1u << (c & 31), __ATOMIC_RELAXED);
        }
      }
      got[t] = k;
    }
    nf = compact(fkey, tkey, base, got, nt, 8);
    compact(fcell, tcell, base, got, nt, 8);
  }
  *rounds_out = round;
done:
  free(bits);
  free(fkey);
  free(tkey);
  free(fcell);
  free(tcell);
  free(cand);
  return status;
}
