/* CPU oracle for round-synchronous parallel peeling (Jiang, Mitzenmacher &
 * Thaler, "Parallel Peeling Algorithms").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the CUDA path computes.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark load it; the library's product path
 * never does, and the two share no code.
 *
 * Contents (each function cites the passage it follows):
 *   - the IBLT cell/checksum convention (Sec. 6, "Motivation": r hash functions
 *     and a pseudorandom checkSum; App. B / Sec. 6 "Implementation Details":
 *     one cell per sub-table);
 *   - IBLT insertion (Sec. 6, "Motivation");
 *   - round-synchronous IBLT recovery (Sec. 6: recovery = peeling at k = 2;
 *     Sec. 1: each round removes all vertices of degree < k at once);
 *   - sequential (queue) IBLT recovery (Sec. 6, the serial recovery);
 *   - round-synchronous k-core peeling on explicit hyperedges (Sec. 1 and
 *     Sec. 3.1), reported per round;
 *   - sequential queue k-core peeler (Sec. 1: the core is unique and does not
 *     depend on the removal order).
 *   - peeling and IBLT recovery with sub-tables (App. B, Sec. 6
 *     "Implementation Details"): one part / sub-table per sub-round.
 *   - signed IBLT recovery of a set difference (Sec. 6 "Motivation":
 *     insertions and deletions are the same XORs): count = +1 or -1 is pure.
 *
 * Conventions the paper leaves open (stated, not derived; parity unpinned for
 * the cell map and the sub-table split, which only the known-answer file
 * freezes):
 *   - mix64 is the SplitMix64 output finaliser (Steele, Lea & Flood 2014);
 *     hash seed j (j = 0..r-1) and the checksum seed (index r) are outputs
 *     1..r+1 of SplitMix64 started at the table seed;
 *   - sub-table j holds floor(n/r) + [j < n mod r] cells, laid out in order;
 *   - cell_j(x) = off_j + floor(mix64(x ^ seed_j) * size_j / 2^64);
 *   - checkSum(x) = mix64(x ^ seed_chk), a 64-bit value;
 *   - a cell is pure iff count == 1 and its checksum field equals
 *     checkSum(key field) (signed recovery: count == +1 or -1 and the same
 *     checksum test).
 *
 * Fixed by the paper, not a convention: the key field and the checksum field
 * are XORs (Sec. 6 "Motivation": an inserted key is XORed into the key field
 * of each of its cells and checkSum(x) into the checksum field; a deletion is
 * the same XORs with the count decremented instead of incremented).
 *   - a vertex's degree counts incidences, so an edge that names a vertex
 *     twice contributes 2 to its degree and takes 2 when it is removed.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_GAMMA 0x9E3779B97F4A7C15ULL

enum { ORC_OK = 0, ORC_CAPACITY = 1, ORC_ROUND_LIMIT = 2, ORC_INVALID = 3, ORC_NOMEM = 4 };

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t orc_mix64(uint64_t z) { return mix64(z); }

/* seeds[0..r-1]: hash seeds h_1..h_r; seeds[r]: checksum seed. */
void orc_hash_seeds(uint64_t table_seed, uint32_t r, uint64_t *seeds) {
  for (uint32_t j = 0; j <= r; ++j) seeds[j] = mix64(table_seed + (uint64_t)(j + 1) * ORC_GAMMA);
}

/* off[0..r]: sub-table j is cells off[j] .. off[j+1]-1 (App. B: r sub-tables). */
void orc_part_offsets(uint64_t n, uint32_t r, uint64_t *off) {
  uint64_t q = n / r, rem = n % r;
  off[0] = 0;
  for (uint32_t j = 0; j < r; ++j) off[j + 1] = off[j] + q + (j < rem ? 1 : 0);
}

static uint64_t cell_of(uint64_t x, uint32_t j, const uint64_t *seeds, const uint64_t *off) {
  uint64_t h = mix64(x ^ seeds[j]);
  uint64_t size = off[j + 1] - off[j];
  return off[j] + (uint64_t)(((unsigned __int128)h * size) >> 64);
}

static uint64_t checksum_of(uint64_t x, const uint64_t *seeds, uint32_t r) {
  return mix64(x ^ seeds[r]);
}

/* The r cells of each key (row-major m x r), for building the key hypergraph. */
void orc_key_cells(uint64_t n, uint32_t r, uint64_t table_seed, const uint64_t *keys,
                   uint64_t m, uint64_t *cells) {
  uint64_t seeds[17], off[17];
  orc_hash_seeds(table_seed, r, seeds);
  orc_part_offsets(n, r, off);
  for (uint64_t i = 0; i < m; ++i)
    for (uint32_t j = 0; j < r; ++j) cells[i * r + j] = cell_of(keys[i], j, seeds, off);
}

uint64_t orc_checksum(uint64_t table_seed, uint32_t r, uint64_t x) {
  uint64_t seeds[17];
  orc_hash_seeds(table_seed, r, seeds);
  return checksum_of(x, seeds, r);
}

/* IBLT insertion (sign = +1) or deletion (sign = -1), Sec. 6 "Motivation":
 * for each of the key's r cells, XOR the key into the key field, XOR
 * checkSum(key) into the checksum field and add sign to the count. */
int orc_iblt_insert(uint64_t n, uint32_t r, uint64_t table_seed, const uint64_t *keys,
                    uint64_t m, int64_t sign, int64_t *count, uint64_t *keyx,
                    uint64_t *chkx) {
  if (r < 2 || r > 16 || n < r) return ORC_INVALID;
  uint64_t seeds[17], off[17];
  orc_hash_seeds(table_seed, r, seeds);
  orc_part_offsets(n, r, off);
  for (uint64_t i = 0; i < m; ++i) {
    uint64_t x = keys[i];
    uint64_t cs = checksum_of(x, seeds, r);
    for (uint32_t j = 0; j < r; ++j) {
      uint64_t c = cell_of(x, j, seeds, off);
      count[c] += sign;
      keyx[c] ^= x;
      chkx[c] ^= cs;
    }
  }
  return ORC_OK;
}

static int is_pure(uint64_t c, const int64_t *count, const uint64_t *keyx, const uint64_t *chkx,
                   const uint64_t *seeds, uint32_t r) {
  return count[c] == 1 && chkx[c] == checksum_of(keyx[c], seeds, r);
}

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Round-synchronous IBLT recovery.
 *
 * Round t (Sec. 1's round rule at k = 2, on the IBLT hypergraph of Sec. 6):
 *   P_t = every cell that is pure at the start of round t;
 *   K_t = the distinct keys found in P_t (a key pure in several cells is
 *         recovered once);
 *   each x in K_t is deleted from all r of its cells.
 * The loop ends at the first round with K_t empty; *rounds_out is the number
 * of rounds that recovered at least one key.
 *
 * out_keys receives K_1, K_2, ... in order, each round sorted ascending;
 * round_end[t-1] = |K_1| + ... + |K_t|.
 * cells_alive[t-1] = #cells with count >= 2 at the start of round t: the
 * vertices of the hypergraph still present after round t (Sec. 3.1: a vertex
 * of degree < 2 at the start of a round is removed in that round).
 * Returns ORC_CAPACITY if out_cap is too small and ORC_ROUND_LIMIT if K_t is
 * still non-empty at t = max_rounds + 1. */
int orc_iblt_decode_rounds(uint64_t n, uint32_t r, uint64_t table_seed, int64_t *count,
                           uint64_t *keyx, uint64_t *chkx, uint32_t max_rounds,
                           uint64_t *out_keys, uint64_t out_cap, uint64_t *round_end,
                           uint64_t *cells_alive, uint32_t *rounds_out) {
  if (r < 2 || r > 16 || n < r) return ORC_INVALID;
  uint64_t seeds[17], off[17];
  orc_hash_seeds(table_seed, r, seeds);
  orc_part_offsets(n, r, off);
  uint64_t *pure_keys = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
  if (!pure_keys) return ORC_NOMEM;
  uint64_t total = 0;
  uint32_t t = 0;
  int status = ORC_OK;
  *rounds_out = 0;
  for (;;) {
    /* P_t: scan every cell at the start of the round. */
    uint64_t np = 0, alive = 0;
    for (uint64_t c = 0; c < n; ++c) {
      if (count[c] >= 2) ++alive;
      if (is_pure(c, count, keyx, chkx, seeds, r)) pure_keys[np++] = keyx[c];
    }
    if (np == 0) break;
    if (t == max_rounds) { status = ORC_ROUND_LIMIT; break; }
    /* K_t: distinct keys of P_t. */
    qsort(pure_keys, np, sizeof(uint64_t), cmp_u64);
    uint64_t nk = 0;
    for (uint64_t i = 0; i < np; ++i)
      if (i == 0 || pure_keys[i] != pure_keys[i - 1]) pure_keys[nk++] = pure_keys[i];
    if (total + nk > out_cap) { status = ORC_CAPACITY; break; }
    /* Delete every key of K_t from its r cells. */
    for (uint64_t i = 0; i < nk; ++i) {
      const uint64_t x = pure_keys[i];
      const uint64_t cs = checksum_of(x, seeds, r);
      for (uint32_t j = 0; j < r; ++j) {
        uint64_t c = cell_of(x, j, seeds, off);
        count[c] -= 1;
        keyx[c] ^= x;
        chkx[c] ^= cs;
      }
      out_keys[total + i] = x;
    }
    total += nk;
    round_end[t] = total;
    cells_alive[t] = alive;
    ++t;
  }
  *rounds_out = t;
  free(pure_keys);
  return status;
}

/* Sequential IBLT recovery (Sec. 6): repeatedly take any pure cell, recover its
 * key and delete it from its r cells, until no pure cell is left.  Keys come out
 * in the order found; the recovered set is order-independent. */
int orc_iblt_decode_queue(uint64_t n, uint32_t r, uint64_t table_seed, int64_t *count,
                          uint64_t *keyx, uint64_t *chkx, uint64_t *out_keys,
                          uint64_t out_cap, uint64_t *n_out) {
  if (r < 2 || r > 16 || n < r) return ORC_INVALID;
  uint64_t seeds[17], off[17];
  orc_hash_seeds(table_seed, r, seeds);
  orc_part_offsets(n, r, off);
  /* each cell is pushed at most once initially and once per count change */
  uint64_t cap = n + 16, top = 0;
  uint64_t *stack = (uint64_t *)malloc(cap * sizeof(uint64_t));
  if (!stack) return ORC_NOMEM;
  for (uint64_t c = 0; c < n; ++c)
    if (is_pure(c, count, keyx, chkx, seeds, r)) stack[top++] = c;
  uint64_t got = 0;
  int status = ORC_OK;
  while (top > 0) {
    uint64_t c = stack[--top];
    if (!is_pure(c, count, keyx, chkx, seeds, r)) continue;
    const uint64_t x = keyx[c];
    const uint64_t cs = checksum_of(x, seeds, r);
    if (got == out_cap) { status = ORC_CAPACITY; break; }
    out_keys[got++] = x;
    for (uint32_t j = 0; j < r; ++j) {
      uint64_t d = cell_of(x, j, seeds, off);
      count[d] -= 1;
      keyx[d] ^= x;
      chkx[d] ^= cs;
      if (count[d] == 1) {
        if (top == cap) {
          cap *= 2;
          uint64_t *ns = (uint64_t *)realloc(stack, cap * sizeof(uint64_t));
          if (!ns) { free(stack); return ORC_NOMEM; }
          stack = ns;
        }
        stack[top++] = d;
      }
    }
  }
  *n_out = got;
  free(stack);
  return status;
}

/* Round-synchronous k-core peeling on explicit hyperedges (Sec. 1, Sec. 3.1).
 *
 * edges: m rows of r vertex ids (row-major).  deg(v) = number of incidences.
 * Round t: R_t = {alive v : deg(v) < k}; D_t = {alive e : e has an endpoint in
 * R_t}; R_t and D_t are removed and each endpoint of each edge in D_t loses one
 * degree per incidence.  Stops at the first t with R_t empty.
 * Outputs: vround[v] = round v was removed in (0 = in the k-core); eround[e]
 * likewise; s_t[t-1] = |V_t|, m_t[t-1] = |E_t| for t = 1..T; *T_out = number of
 * rounds with R_t non-empty. */
int orc_kcore_rounds(uint32_t n, uint32_t r, uint32_t k, const uint32_t *edges, uint64_t m,
                     uint32_t max_rounds, int32_t *vround, int32_t *eround, uint64_t *s_t,
                     uint64_t *m_t, uint32_t *T_out) {
  if (r < 1 || k < 1) return ORC_INVALID;
  for (uint64_t i = 0; i < m * r; ++i)
    if (edges[i] >= n) return ORC_INVALID;
  int64_t *deg = (int64_t *)calloc(n ? n : 1, sizeof(int64_t));
  uint64_t *alive_e = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t));
  uint32_t *removed_now = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
  if (!deg || !alive_e || !removed_now) {
    free(deg); free(alive_e); free(removed_now);
    return ORC_NOMEM;
  }
  for (uint64_t i = 0; i < m * r; ++i) deg[edges[i]] += 1;
  for (uint32_t v = 0; v < n; ++v) vround[v] = 0;
  for (uint64_t e = 0; e < m; ++e) { eround[e] = 0; alive_e[e] = e; }
  uint64_t n_alive_e = m, n_alive_v = n;
  uint32_t t = 0;
  int status = ORC_OK;
  for (;;) {
    uint32_t round = t + 1;
    /* R_t from the degrees at the start of the round. */
    uint64_t nr = 0;
    for (uint32_t v = 0; v < n; ++v)
      if (vround[v] == 0 && deg[v] < (int64_t)k) ++nr;
    if (nr == 0) break;
    if (t == max_rounds) { status = ORC_ROUND_LIMIT; break; }
    for (uint32_t v = 0; v < n; ++v)
      if (vround[v] == 0 && deg[v] < (int64_t)k) vround[v] = (int32_t)round;
    n_alive_v -= nr;
    /* D_t: alive edges with an endpoint in R_t. */
    uint64_t nd = 0, keep = 0;
    for (uint64_t i = 0; i < n_alive_e; ++i) {
      uint64_t e = alive_e[i];
      int hit = 0;
      for (uint32_t j = 0; j < r; ++j)
        if (vround[edges[e * r + j]] == (int32_t)round) hit = 1;
      if (hit) removed_now[nd++] = (uint32_t)e;
      else alive_e[keep++] = e;
    }
    n_alive_e = keep;
    /* Remove D_t: every incidence of a removed edge costs its vertex one degree. */
    for (uint64_t i = 0; i < nd; ++i) {
      uint64_t e = removed_now[i];
      eround[e] = (int32_t)round;
      for (uint32_t j = 0; j < r; ++j) deg[edges[e * r + j]] -= 1;
    }
    s_t[t] = n_alive_v;
    m_t[t] = n_alive_e;
    ++t;
  }
  *T_out = t;
  free(deg); free(alive_e); free(removed_now);
  return status;
}

/* Sequential k-core peeler (Sec. 1): keep removing any vertex of degree < k
 * together with its remaining edges.  v_core[v] = 1 iff v is in the k-core;
 * e_core[e] = 1 iff e survives. */
int orc_kcore_queue(uint32_t n, uint32_t r, uint32_t k, const uint32_t *edges, uint64_t m,
                    uint8_t *v_core, uint8_t *e_core) {
  if (r < 1 || k < 1) return ORC_INVALID;
  for (uint64_t i = 0; i < m * r; ++i)
    if (edges[i] >= n) return ORC_INVALID;
  int64_t *deg = (int64_t *)calloc(n ? n : 1, sizeof(int64_t));
  uint64_t *start = (uint64_t *)calloc((uint64_t)n + 1, sizeof(uint64_t));
  uint64_t *fill = (uint64_t *)calloc((uint64_t)n + 1, sizeof(uint64_t));
  uint64_t *inc = (uint64_t *)malloc((m * r ? m * r : 1) * sizeof(uint64_t));
  uint32_t *stack = (uint32_t *)malloc(((uint64_t)n + 1) * sizeof(uint32_t));
  if (!deg || !start || !fill || !inc || !stack) {
    free(deg); free(start); free(fill); free(inc); free(stack);
    return ORC_NOMEM;
  }
  for (uint64_t i = 0; i < m * r; ++i) deg[edges[i]] += 1;
  for (uint32_t v = 0; v < n; ++v) start[v + 1] = start[v] + (uint64_t)deg[v];
  for (uint32_t v = 0; v < n; ++v) fill[v] = start[v];
  for (uint64_t e = 0; e < m; ++e)
    for (uint32_t j = 0; j < r; ++j) inc[fill[edges[e * r + j]]++] = e;
  for (uint32_t v = 0; v < n; ++v) v_core[v] = 1;
  for (uint64_t e = 0; e < m; ++e) e_core[e] = 1;
  uint64_t top = 0;
  for (uint32_t v = 0; v < n; ++v)
    if (deg[v] < (int64_t)k) stack[top++] = v;
  while (top > 0) {
    uint32_t v = stack[--top];
    if (!v_core[v]) continue;
    v_core[v] = 0;
    for (uint64_t p = start[v]; p < start[v + 1]; ++p) {
      uint64_t e = inc[p];
      if (!e_core[e]) continue;
      e_core[e] = 0;
      for (uint32_t j = 0; j < r; ++j) {
        uint32_t u = edges[e * r + j];
        deg[u] -= 1;
        /* u is pushed once: when its degree first drops below k */
        if (deg[u] == (int64_t)k - 1 && v_core[u]) stack[top++] = u;
      }
    }
  }
  free(deg); free(start); free(fill); free(inc); free(stack);
  return ORC_OK;
}

/* Peeling with sub-tables (App. B; the recovery order of Sec. 6
 * "Implementation Details").
 *
 * The vertices are split into p parts: part j (j = 0..p-1) holds the ids
 * part_off[j] .. part_off[j+1]-1, with part_off[0] = 0 and part_off[p] = n.
 * Each round runs one sub-round per part, in part order.  The sub-round of part
 * j removes every alive vertex of part j whose degree is < k at the start of
 * that sub-round, together with every alive edge touching one of them (each
 * endpoint of such an edge loses one degree per incidence).  Vertices of the
 * other parts wait for their own sub-round, so a removal can enable a removal
 * later in the same round (App. B).
 *
 * Sub-rounds are numbered s = (i-1) p + j + 1 for round i and part j.  The
 * process stops once p consecutive sub-rounds removed nothing; S (*S_out) is
 * the number of the last sub-round that removed a vertex (0 if none).
 * Outputs: vround[v] / eround[e] = the sub-round that removed v / e (0 = in
 * the k-core); s_s[s-1] = |V| and m_s[s-1] = |E| after sub-round s, for
 * s = 1..S.  With p = 1 this is orc_kcore_rounds. */
int orc_kcore_subrounds(uint32_t n, uint32_t r, uint32_t k, const uint32_t *edges, uint64_t m,
                        uint32_t p, const uint32_t *part_off, uint32_t max_subrounds,
                        int32_t *vround, int32_t *eround, uint64_t *s_s, uint64_t *m_s,
                        uint32_t *S_out) {
  if (r < 1 || k < 1 || p < 1) return ORC_INVALID;
  if (part_off[0] != 0 || part_off[p] != n) return ORC_INVALID;
  for (uint32_t j = 0; j < p; ++j)
    if (part_off[j] > part_off[j + 1]) return ORC_INVALID;
  for (uint64_t i = 0; i < m * r; ++i)
    if (edges[i] >= n) return ORC_INVALID;
  int64_t *deg = (int64_t *)calloc(n ? n : 1, sizeof(int64_t));
  if (!deg) return ORC_NOMEM;
  for (uint64_t i = 0; i < m * r; ++i) deg[edges[i]] += 1;
  for (uint32_t v = 0; v < n; ++v) vround[v] = 0;
  for (uint64_t e = 0; e < m; ++e) eround[e] = 0;
  uint64_t n_alive_v = n, n_alive_e = m;
  uint32_t s = 0, idle = 0, S = 0;
  int status = ORC_OK;
  while (idle < p) {
    const uint32_t j = s % p, sub = s + 1;
    /* the vertices of part j with degree < k at the start of the sub-round */
    uint64_t nrem = 0;
    for (uint32_t v = part_off[j]; v < part_off[j + 1]; ++v)
      if (vround[v] == 0 && deg[v] < (int64_t)k) ++nrem;
    if (nrem == 0) {
      if (s < max_subrounds) { s_s[s] = n_alive_v; m_s[s] = n_alive_e; }
      ++idle;
      ++s;
      continue;
    }
    if (s >= max_subrounds) { status = ORC_ROUND_LIMIT; break; }
    idle = 0;
    for (uint32_t v = part_off[j]; v < part_off[j + 1]; ++v)
      if (vround[v] == 0 && deg[v] < (int64_t)k) vround[v] = (int32_t)sub;
    n_alive_v -= nrem;
    /* every alive edge with an endpoint removed now goes too */
    for (uint64_t e = 0; e < m; ++e) {
      if (eround[e] != 0) continue;
      int hit = 0;
      for (uint32_t q = 0; q < r; ++q)
        if (vround[edges[e * r + q]] == (int32_t)sub) hit = 1;
      if (!hit) continue;
      eround[e] = (int32_t)sub;
      --n_alive_e;
      for (uint32_t q = 0; q < r; ++q) deg[edges[e * r + q]] -= 1;
    }
    s_s[s] = n_alive_v;
    m_s[s] = n_alive_e;
    S = sub;
    ++s;
  }
  *S_out = S;
  free(deg);
  return status;
}

/* IBLT recovery with sub-tables (Sec. 6 "Implementation Details"; App. B at
 * k = 2): round i runs r sub-rounds, one per sub-table, in order.  The
 * sub-round of sub-table j takes every cell of sub-table j that is pure at the
 * start of the sub-round, recovers the key found in it and deletes that key
 * from its r cells.  A key has exactly one cell in each sub-table, so no key
 * is found twice within a sub-round; every pure cell's key is deleted as
 * found, with no further de-duplication.
 *
 * Sub-rounds are numbered s = (i-1) r + j + 1; the loop stops once r
 * consecutive sub-rounds recovered nothing, and *S_out is the number of the
 * last sub-round that recovered a key.  out_keys receives the keys of
 * sub-rounds 1, 2, ... in order, each sub-round sorted ascending;
 * sub_end[s-1] = the number of keys recovered in sub-rounds 1..s, s = 1..S.
 * Returns ORC_CAPACITY if out_cap is too small and ORC_ROUND_LIMIT if a
 * sub-round past max_subrounds would recover a key. */
int orc_iblt_decode_subrounds(uint64_t n, uint32_t r, uint64_t table_seed, int64_t *count,
                              uint64_t *keyx, uint64_t *chkx, uint32_t max_subrounds,
                              uint64_t *out_keys, uint64_t out_cap, uint64_t *sub_end,
                              uint32_t *S_out) {
  if (r < 2 || r > 16 || n < r) return ORC_INVALID;
  uint64_t seeds[17], off[17];
  orc_hash_seeds(table_seed, r, seeds);
  orc_part_offsets(n, r, off);
  uint64_t *found = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
  if (!found) return ORC_NOMEM;
  uint64_t total = 0;
  uint32_t s = 0, idle = 0, S = 0;
  int status = ORC_OK;
  while (idle < r) {
    const uint32_t j = s % r;
    /* the pure cells of sub-table j at the start of the sub-round */
    uint64_t nf = 0;
    for (uint64_t c = off[j]; c < off[j + 1]; ++c)
      if (is_pure(c, count, keyx, chkx, seeds, r)) found[nf++] = keyx[c];
    if (nf == 0) {
      if (s < max_subrounds) sub_end[s] = total;
      ++idle;
      ++s;
      continue;
    }
    if (s >= max_subrounds) { status = ORC_ROUND_LIMIT; break; }
    if (total + nf > out_cap) { status = ORC_CAPACITY; break; }
    idle = 0;
    qsort(found, nf, sizeof(uint64_t), cmp_u64);
    for (uint64_t i = 0; i < nf; ++i) {
      const uint64_t x = found[i];
      const uint64_t cs = checksum_of(x, seeds, r);
      out_keys[total + i] = x;
      for (uint32_t q = 0; q < r; ++q) {
        uint64_t c = cell_of(x, q, seeds, off);
        count[c] -= 1;
        keyx[c] ^= x;
        chkx[c] ^= cs;
      }
    }
    total += nf;
    sub_end[s] = total;
    S = s + 1;
    ++s;
  }
  *S_out = S;
  free(found);
  return status;
}

/* Signed IBLT recovery: the table holds a set difference (keys inserted with
 * sign +1 and deleted with sign -1 that were never inserted), as in the sparse
 * recovery use of Sec. 6 "Motivation".  A cell is pure when count == s for
 * s = +1 or -1 and its checksum field equals checkSum(key field) (the field is
 * an XOR, so it does not carry the sign); its key comes out with the sign s.
 *
 * Round t (Sec. 1's round rule at k = 2 on the hypergraph of the difference):
 *   P_t = every cell pure at the start of round t;
 *   K_t = the distinct (key, sign) pairs found in P_t;
 *   each (x, s) in K_t is removed from its r cells: count -= s, XOR x out
 *   of the key field and checkSum(x) out of the checksum field.
 * The loop ends at the first round with K_t empty; *rounds_out counts the
 * rounds that recovered something.  out_keys / out_signs receive K_1, K_2,
 * ... in order, each round sorted by (key, sign); round_end[t-1] = the total
 * after round t.  Returns ORC_CAPACITY or ORC_ROUND_LIMIT like the unsigned
 * recovery. */
typedef struct { uint64_t x; int64_t s; } orc_signed_key;

static int cmp_signed(const void *a, const void *b) {
  const orc_signed_key *p = (const orc_signed_key *)a, *q = (const orc_signed_key *)b;
  if (p->x != q->x) return p->x < q->x ? -1 : 1;
  return p->s < q->s ? -1 : (p->s > q->s ? 1 : 0);
}

int orc_iblt_decode_signed(uint64_t n, uint32_t r, uint64_t table_seed, int64_t *count, uint64_t *keyx,
                           uint64_t *chkx, uint32_t max_rounds, uint64_t *out_keys, int8_t *out_signs,
                           uint64_t out_cap, uint64_t *round_end, uint32_t *rounds_out) {
  if (r < 2 || r > 16 || n < r) return ORC_INVALID;
  uint64_t seeds[17], off[17];
  orc_hash_seeds(table_seed, r, seeds);
  orc_part_offsets(n, r, off);
  orc_signed_key *found = (orc_signed_key *)malloc((n ? n : 1) * sizeof(orc_signed_key));
  if (!found) return ORC_NOMEM;
  uint64_t total = 0;
  uint32_t t = 0;
  int status = ORC_OK;
  *rounds_out = 0;
  for (;;) {
    uint64_t nf = 0;
    for (uint64_t c = 0; c < n; ++c) {
      if ((count[c] == 1 || count[c] == -1) &&
          chkx[c] == checksum_of(keyx[c], seeds, r)) {
        found[nf].x = keyx[c];
        found[nf].s = count[c];
        ++nf;
      }
    }
    if (nf == 0) break;
    if (t == max_rounds) { status = ORC_ROUND_LIMIT; break; }
    qsort(found, nf, sizeof(orc_signed_key), cmp_signed);
    uint64_t nk = 0;
    for (uint64_t i = 0; i < nf; ++i)
      if (i == 0 || found[i].x != found[i - 1].x || found[i].s != found[i - 1].s) found[nk++] = found[i];
    if (total + nk > out_cap) { status = ORC_CAPACITY; break; }
    for (uint64_t i = 0; i < nk; ++i) {
      const uint64_t x = found[i].x;
      const uint64_t cs = checksum_of(x, seeds, r);
      const int64_t sg = found[i].s;
      out_keys[total + i] = x;
      out_signs[total + i] = (int8_t)sg;
      for (uint32_t q = 0; q < r; ++q) {
        const uint64_t c = cell_of(x, q, seeds, off);
        count[c] -= sg;
        keyx[c] ^= x;
        chkx[c] ^= cs;
      }
    }
    total += nk;
    round_end[t] = total;
    ++t;
  }
  *rounds_out = t;
  free(found);
  return status;
}
