/* ppeel -- round-synchronous parallel peeling on one B300 (sm_103a).
 *
 * C ABI of libppeel.so.  The operations follow Jiang, Mitzenmacher & Thaler,
 * "Parallel Peeling Algorithms":
 *   - peeling (Sec. 1): repeatedly remove vertices of degree < k with their
 *     edges; what remains is the k-core, unique and independent of the order;
 *   - the parallel round (Sec. 1, Sec. 3.1): one round removes every vertex
 *     whose degree is < k at the start of the round, all at once, together
 *     with every edge that touches one of them;
 *   - Invertible Bloom Lookup Tables (Sec. 6): each key is XORed, with its
 *     checksum, into one cell of each of r sub-tables (App. B); a pure cell
 *     holds exactly one key; recovery is the k = 2 peel of the hypergraph whose
 *     vertices are cells and whose edges are keys, and succeeds iff that
 *     hypergraph's 2-core is empty.
 *
 * General rules for every entry point:
 *   - Pointers named d_* are device pointers owned by the caller; pointers
 *     named h_* and result structs are host memory owned by the caller.
 *   - Handles (pp_iblt, pp_batch, pp_server) own their device memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is ordered on that stream.  Calls that return results in a
 *     host struct (decode, peel) synchronize that stream before returning;
 *     insert and clear only enqueue work.
 *   - Every call returns a pp_status; no exception or longjmp crosses the ABI.
 *     pp_last_error() gives a one-line message for the calling thread's last
 *     failure.  A status other than PP_OK leaves output buffers unspecified
 *     unless stated otherwise.
 *   - Vertex ids, cell ids and edge ids are 32-bit: n, n_cells and m*r must be
 *     below 2^32 - 64.  1 <= k, 2 <= r <= PP_MAX_R.
 */
#ifndef PPEEL_H
#define PPEEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PP_MAX_R 8

typedef enum pp_status {
  PP_OK = 0,
  PP_ERR_INVALID_ARG = 1,   /* bad size, null pointer, out-of-range id, ... */
  PP_ERR_OUT_OF_MEMORY = 2, /* a device or host allocation failed */
  PP_ERR_CAPACITY = 3,      /* an output buffer is too small */
  PP_ERR_ROUND_LIMIT = 4,   /* max_rounds reached with vertices still peelable */
  PP_ERR_TIMEOUT = 5,       /* a bounded wait ran out (server, batch engine) */
  PP_ERR_CUDA = 6,          /* a CUDA runtime call failed; see pp_last_error */
  PP_ERR_BUSY = 7,          /* server: result not ready / queue full */
  PP_ERR_NOT_FOUND = 8      /* server: unknown ticket */
} pp_status;

/* Tuning knobs.  Zero in any field selects the default. */
typedef struct pp_options {
  uint32_t block;        /* threads per CTA of the round kernels (default 256) */
  uint32_t ctas_per_sm;  /* persistent grid = ctas_per_sm * #SMs, capped by occupancy (default 8) */
  uint32_t max_rounds;   /* stop after this many rounds (default 65535) */
  uint32_t host_loop;    /* 1 = drive rounds from the host (one sync per round);
                            0 (default) = one CUDA graph whose while-node keeps
                            looping on the device until the frontier is empty */
  uint32_t stats_rounds; /* batch: per-table per-round counters kept (default 128) */
  uint32_t binned;       /* IBLT build/insert: 0 = slab-binned when the table is at least
                            2^23 cells (default), 1 = always binned, 2 = never */
  uint32_t kcore_mode;   /* pp_peel_kcore full rounds: 0 = for graphs of 2^20 edges or
                            more, edge-centric rounds while the frontier holds at least
                            half as many vertices as there are edges left, then rounds
                            over incidence lists built for the edges left; graphs of at
                            most 2^14 vertices and 2^16 edges (host_loop 0) run every
                            round inside one thread block; other graphs use incidence
                            lists (default); 1 = incidence lists from round
                            1; 2 = edge-centric rounds to the end.  r > 4 and edge
                            rows that are not 16-byte (r = 4) or 8-byte (r = 2) aligned
                            always use 1. */
  uint32_t rounds;       /* IBLT decode rounds of pp_iblt_decode and pp_batch_decode:
                            0 = tile rounds for tables (batch: arenas) of at least
                            2^21 cells that saw no deletion (each round's updates
                            folded per 4096-cell tile in shared memory), binned
                            atomic rounds for other large ones, direct atomics below
                            2^21 cells (default); 1 = never tile rounds; 2 = tile
                            rounds for any table or batch without deletions */
  uint32_t apply_ctas;   /* resident blocks per SM of the binned rounds' apply kernel
                            (default 3; sets the width of the table window updated at once) */
  uint32_t frontier_switch; /* pp_peel_kcore, kcore_mode 0: edge-centric rounds run while
                            |frontier| * frontier_switch >= edges left (default 2) */
  uint32_t insert_chunk; /* batches: keys per insert work item (default 4096) */
  uint32_t l2_fetch;     /* pp_iblt_create, pp_batch_create, pp_server_start: 1
                            (default) = set this process's L2 fetch
                            granularity limit (cudaLimitMaxL2FetchGranularity, a
                            per-context hint that ends with the process) to 32 bytes,
                            so that a scattered 32-byte cell read fetches one sector
                            instead of two; 2 = leave the limit as it is */
} pp_options;

/* Fills *opt with the defaults above. */
void pp_options_default(pp_options *opt);

/* Human-readable name of a status code (static storage). */
const char *pp_status_string(pp_status s);

/* Message describing the calling thread's most recent failure ("" if none). */
const char *pp_last_error(void);

/* ------------------------------------------------------------------------
 * IBLT (Sec. 6 "Motivation" and "Implementation Details"; App. B layout)
 *
 * Cell layout in device memory (32 bytes, 32-byte aligned, cell i at
 * byte 32*i of the table; one DRAM sector per cell):
 *     uint64 key_xor;    XOR of the keys in the cell
 *     uint64 chk_xor;    XOR of checkSum(x) over the cell's keys
 *     int32  count;      insertions minus deletions
 *     uint32 pad0;       0
 *     uint64 pad1;       0
 * Insertion and deletion are the same two XORs; only the count tells them
 * apart (Sec. 6 "Motivation").
 * Cells are split into r sub-tables, in order; sub-table j holds
 * floor(n/r) + [j < n mod r] cells.  Key x lives in cell
 *     off_j + floor(mix64(x ^ s_j) * size_j / 2^64)   of each sub-table j,
 * and checkSum(x) = mix64(x ^ s_r), where mix64 is the SplitMix64 finaliser
 * and s_0..s_r are outputs 1..r+1 of SplitMix64 started at the table seed.
 * A cell is pure iff count == 1 and chk_xor == checkSum(key_xor); the signed
 * decode also takes count == -1 with the same checksum test.
 * ------------------------------------------------------------------------ */
typedef struct pp_iblt pp_iblt;

typedef struct pp_cell {
  uint64_t key_xor;
  uint64_t chk_xor;
  int32_t count;
  uint32_t pad0;
  uint64_t pad1;
} pp_cell;

/* Result of a decode.  The caller sets round_cap and the three array pointers
 * (host arrays of round_cap entries each, or NULL); the decode fills the rest.
 * Entry t-1 describes round t, for t = 1..min(rounds, round_cap):
 *   recovered_per_round[t-1]   keys recovered in round t;
 *   remaining_per_round[t-1]   keys still in the table after round t;
 *   alive_cells_per_round[t-1] cells holding >= 2 keys at the start of round
 *                              t, i.e. the hypergraph's vertices that survive
 *                              round t (Sec. 3.1's survivors at k = 2). */
typedef struct pp_decode_result {
  uint32_t rounds;          /* rounds that recovered >= 1 key */
  uint32_t status_flags;    /* device-side flags (0 = clean) */
  uint64_t recovered;       /* keys written to d_out_keys */
  uint64_t items_before;    /* keys in the table before the decode */
  uint64_t residual_cells;  /* non-empty cells after the decode (2-core residue) */
  uint32_t round_cap;
  uint32_t pad;
  uint64_t *recovered_per_round;
  uint64_t *remaining_per_round;
  uint64_t *alive_cells_per_round;
} pp_decode_result;

/* Creates an empty (all-zero) table of n_cells cells for r hash functions.
 * Allocates the table (16 B/cell) and the decode workspace (~17 B/cell).
 * Errors: INVALID_ARG (r outside 2..PP_MAX_R, n_cells < r or too large),
 * OUT_OF_MEMORY, CUDA. */
pp_status pp_iblt_create(pp_iblt **out, uint64_t n_cells, uint32_t r, uint64_t seed,
                         const pp_options *opt);

/* Frees the table and its workspace (synchronizes the device first).  NULL is a no-op. */
pp_status pp_iblt_destroy(pp_iblt *t);

/* Device memory of a table of n_cells cells and r hash functions (host only,
 * no device call; opt as for pp_iblt_create, NULL = defaults):
 *   *table_bytes  the cells, 32 B each;
 *   *fixed_bytes  the decode workspace allocated by pp_iblt_create;
 *   *peak_bytes   all the handle holds after pp_iblt_create, a pp_iblt_build
 *                 or pp_iblt_insert of m_keys keys and a pp_iblt_decode: the
 *                 above plus the update records of the slab-binned build and
 *                 of the binned rounds (one shared buffer, sized for the
 *                 larger), the build's tile buffers, and the tile rounds'
 *                 record regions (10 B per key and cell, for a table that saw
 *                 no deletion).
 * Not counted: what pp_iblt_decode_subrounds (a few hundred bytes) and
 * pp_iblt_decode_signed (n_cells + 4 r n_cells bytes) add on first use.
 * Any output pointer may be NULL.  Errors: INVALID_ARG as pp_iblt_create. */
pp_status pp_workspace_size(uint64_t n_cells, uint32_t r, uint64_t m_keys, const pp_options *opt,
                            uint64_t *table_bytes, uint64_t *fixed_bytes, uint64_t *peak_bytes);

/* Zeroes every cell (enqueued on `stream`). */
pp_status pp_iblt_clear(pp_iblt *t, void *stream);

/* Inserts m keys (Sec. 6 "Motivation": XOR the key and its checksum into its r
 * cells and add 1 to their counts).  d_keys: m uint64 on the device.  Keys are
 * a set: inserting a key twice makes both copies unrecoverable.  Enqueued on
 * `stream`; the caller keeps d_keys alive until the stream reaches this work. */
pp_status pp_iblt_insert(pp_iblt *t, const uint64_t *d_keys, uint64_t m, void *stream);

/* Deletes m keys: the same XORs with count -1 (Sec. 6: insertion and deletion
 * are identical XOR operations). */
pp_status pp_iblt_delete(pp_iblt *t, const uint64_t *d_keys, uint64_t m, void *stream);

/* Builds the table from scratch: the result equals pp_iblt_clear followed by
 * pp_iblt_insert.  Large tables are built slab by slab (2^21 cells at a time),
 * each slab zero-filled and updated while it sits in L2.  Synchronizes
 * `stream` once (after sorting the keys' updates into slabs). */
pp_status pp_iblt_build(pp_iblt *t, const uint64_t *d_keys, uint64_t m, void *stream);

/* Round-synchronous recovery (Sec. 6 recovery; Sec. 1 rounds at k = 2).
 * Round t recovers every key that is alone in some cell at the start of round
 * t (each such key once, however many of its cells are pure), then deletes
 * those keys from all their cells.  Stops at the first round that recovers
 * nothing.  The table is decoded in place: afterwards it holds the 2-core
 * residue (all zero iff every key was recovered).
 * d_out_keys: out_cap uint64 on the device; receives the recovered keys grouped
 * by round (round 1 first), in no particular order within a round.
 * out_cap must be >= the number of keys in the table, else CAPACITY (nothing
 * is decoded).  ROUND_LIMIT if opt.max_rounds rounds did not finish; the table
 * is then left after the last completed round and *res describes those rounds.
 * Synchronizes `stream`. */
pp_status pp_iblt_decode(pp_iblt *t, uint64_t *d_out_keys, uint64_t out_cap,
                         pp_decode_result *res, void *stream);

/* pp_iblt_build of the m keys at d_keys followed by pp_iblt_decode into
 * d_out_keys (out_cap >= m, else CAPACITY; nothing is built).  Same table,
 * keys, rounds and *res as the two calls.  When the build is slab-binned and
 * the decode runs tile rounds (both chosen as in those calls), the build's
 * write-out of each tile also finds the tile's pure cells (F_1, Sec. 1
 * round 1), so the decode starts at its first round without reading the
 * table once more; a tile that keys crowd beyond its list is left to the
 * decode to scan.  Synchronizes `stream` twice (after sorting the updates
 * into slabs, and at the end). */
pp_status pp_iblt_build_decode(pp_iblt *t, const uint64_t *d_keys, uint64_t m, uint64_t *d_out_keys,
                               uint64_t out_cap, pp_decode_result *res, void *stream);

/* Build and decode from HOST buffers (Sec. 6: insert the keys, then recover
 * them), with the host<->device copies inside the call: the paper's GPU insert
 * times include the upload of the items.
 *   pp_iblt_submit_host  enqueues, for the m keys at h_keys: their upload (on
 *                        an upload stream the table owns), the build and
 *                        decode of pp_iblt_build_decode, and the
 *                        download of the recovered keys into h_out (on a
 *                        download stream; out_cap >= m, else CAPACITY), then
 *                        returns a ticket without waiting for the GPU.
 *   pp_iblt_finish_host  waits for that job and fills *res as pp_iblt_decode
 *                        does (per-round figures for at most the first 4096
 *                        rounds); h_out[0 .. res->recovered) hold the keys,
 *                        grouped by round.
 * At most three jobs are in flight per table (INVALID_ARG for a fourth): jobs
 * upload while earlier ones decode and download while later ones build and
 * decode; each has its own device buffers (2 m keys, kept for reuse).  Should
 * a slab of a job's build overflow its list (keys crowding one slab far beyond
 * the uniform share), pp_iblt_finish_host rebuilds and decodes that job again,
 * synchronously, before returning.
 * h_keys and h_out stay in use until the job is finished; pinned memory
 * (cudaMallocHost / cudaHostRegister) is copied directly, pageable memory is
 * registered for the job's duration, which costs time.  One cudaMemcpyAsync
 * per copy.  The job's table is decoded in place, as by pp_iblt_decode. */
pp_status pp_iblt_submit_host(pp_iblt *t, const uint64_t *h_keys, uint64_t m, uint64_t *h_out, uint64_t out_cap,
                              uint64_t *ticket, void *stream);
pp_status pp_iblt_finish_host(pp_iblt *t, uint64_t ticket, pp_decode_result *res);

/* pp_iblt_submit_host + pp_iblt_finish_host of one job. */
pp_status pp_iblt_build_decode_host(pp_iblt *t, const uint64_t *h_keys, uint64_t m, uint64_t *h_out,
                                    uint64_t out_cap, pp_decode_result *res, void *stream);

/* Recovery with sub-tables, the order of the paper's GPU implementation
 * (Sec. 6 "Implementation Details"; analysed in App. B): every round visits
 * the r sub-tables in order, and the sub-round of sub-table j recovers the key
 * of every cell of sub-table j that is pure at the start of that sub-round,
 * then deletes it from its r cells before the next sub-round starts.  A key
 * has one cell per sub-table, so no key is found twice in a sub-round.
 * Sub-rounds are numbered s = (i-1) r + j + 1 for round i and sub-table j;
 * sub-rounds whose sub-table has no candidate cell are skipped, keeping their
 * numbers.  The table is decoded in place to the same 2-core residue as
 * pp_iblt_decode, and the same keys come out.
 * d_out_keys: out_cap uint64 on the device; receives the keys grouped by
 * sub-round (sub-round 1 first), in no particular order within a sub-round.
 * *res as for pp_iblt_decode, read per sub-round: res->rounds = S, the last
 * sub-round that recovered a key; recovered_per_round[s-1] and
 * remaining_per_round[s-1] describe sub-round s (0 for a skipped one);
 * alive_cells_per_round is not computed in this order and is zero-filled.
 * opt.max_rounds bounds the number of sub-rounds: ROUND_LIMIT if a sub-round
 * past it still has cells to examine.  CAPACITY as for pp_iblt_decode;
 * INVALID_ARG if a pure cell's key does not hash to that cell.
 * Synchronizes `stream`. */
pp_status pp_iblt_decode_subrounds(pp_iblt *t, uint64_t *d_out_keys, uint64_t out_cap,
                                   pp_decode_result *res, void *stream);

/* Signed recovery of a set difference (the sparse recovery use of Sec. 6
 * "Motivation": insertion and deletion are the same XORs, so a table built by
 * inserting the keys of A and deleting those of B holds A \ B with count
 * contribution +1 and B \ A with -1).  A cell is pure when its count is +1 or
 * -1 and its checksum field matches its key field; its key comes out with the
 * sign of the count and is removed from its r cells with that sign.  Rounds as
 * in pp_iblt_decode (Sec. 1 at k = 2, the lowest-index pure cell of a key
 * recovers it).  The table is decoded in place.
 * d_out_keys: out_cap uint64 on the device, keys grouped by round;
 * d_out_signs: out_cap int8 on the device (+1 / -1 per key), or NULL.
 * res: rounds, status_flags, recovered, residual_cells (cells with a non-zero
 * count) and recovered_per_round as for pp_iblt_decode; remaining_per_round
 * and alive_cells_per_round are zero-filled; items_before is the
 * inserted-minus-deleted count.
 * The size of the difference is not known beforehand: a decode that recovers
 * more than out_cap keys stops after that round with CAPACITY.  Decodes in
 * single kernels per phase (no update binning).  Requires r * n_cells < 2^32
 * (INVALID_ARG).  ROUND_LIMIT as for pp_iblt_decode.  Synchronizes `stream`. */
pp_status pp_iblt_decode_signed(pp_iblt *t, uint64_t *d_out_keys, int8_t *d_out_signs, uint64_t out_cap,
                                pp_decode_result *res, void *stream);

/* Copies `count` cells starting at `first` into dst (device memory if
 * to_host == 0, else host memory), on `stream`, and synchronizes it. */
pp_status pp_iblt_copy_cells(pp_iblt *t, void *dst, uint64_t first, uint64_t count,
                             int to_host, void *stream);

/* Number of cells, r, and the r+1 derived seeds (hash seeds, then checksum seed). */
pp_status pp_iblt_info(const pp_iblt *t, uint64_t *n_cells, uint32_t *r, uint64_t *h_seeds);

/* ------------------------------------------------------------------------
 * k-core peeling of an explicit hypergraph (Sec. 1; Sec. 3.1 round rule)
 * ------------------------------------------------------------------------ */
typedef struct pp_peel_result {
  uint32_t rounds;        /* T: rounds that removed >= 1 vertex */
  uint32_t status_flags;
  uint64_t core_vertices; /* |V_T| */
  uint64_t core_edges;    /* |E_T| */
  uint32_t round_cap;     /* in: entries in the two host arrays below */
  uint32_t pad;
  uint64_t *vertices_left; /* out: s_t = vertices left after round t (may be NULL) */
  uint64_t *edges_left;    /* out: m_t = edges left after round t (may be NULL) */
} pp_peel_result;

/* Peels the r-uniform hypergraph with n vertices and m edges to its k-core.
 * d_edges: m*r uint32 vertex ids, row-major (edge e = d_edges[e*r .. e*r+r-1]).
 * A vertex's degree counts incidences: an edge naming a vertex twice adds 2.
 * Round t removes every vertex whose degree is < k at the start of round t and
 * every edge touching one of them.
 * d_vertex_round (n int32, or NULL): round each vertex was removed in, 0 = in
 * the k-core.  d_edge_round (m int32, or NULL): the same for edges.  When the
 * call stops at opt.max_rounds (ROUND_LIMIT), both hold rounds 1..max_rounds,
 * the vertices that round max_rounds + 1 would remove hold max_rounds + 1, and
 * everything else holds 0.
 * Graphs of at most 2^14 vertices and 2^16 edges peel inside one thread block
 * (automatic mode, rounds on the device) with no device workspace; their
 * statistics come back through a 260 KB pinned buffer that the calling thread
 * keeps for its next call.  Larger graphs use incidence lists or edge-centric
 * rounds.
 * Workspace (~16 B per vertex + 4 B per incidence, plus ~16 B per incidence
 * for the tiled incidence scatter of large inputs) comes from a memory pool
 * the library keeps per device; it goes back to that pool when the call ends
 * and stays mapped for the next call.
 * Errors: INVALID_ARG (k < 1, r outside 2..PP_MAX_R, a vertex id >= n -- the
 * id check runs on the device), ROUND_LIMIT, OUT_OF_MEMORY, CUDA.
 * Synchronizes `stream`. */
pp_status pp_peel_kcore(uint32_t n, uint32_t r, uint32_t k, const uint32_t *d_edges,
                        uint64_t m, int32_t *d_vertex_round, int32_t *d_edge_round,
                        pp_peel_result *res, const pp_options *opt, void *stream);

/* Peeling with sub-tables (App. B): the vertices are split into n_parts parts,
 * part j holding the ids h_part_off[j] .. h_part_off[j+1]-1 (a host array of
 * n_parts + 1 entries running from 0 to n, non-decreasing; 1 <= n_parts <= 64).
 * Every round runs one sub-round per part, in part order; the sub-round of part
 * j removes every vertex of part j whose degree is < k at the start of that
 * sub-round, with every edge touching one of them.  With one part this is
 * pp_peel_kcore.  Sub-rounds are numbered s = (i-1) n_parts + j + 1; sub-rounds
 * whose part has nothing to remove are skipped on the device but keep their
 * numbers and statistics.
 * Outputs as for pp_peel_kcore, read per sub-round: d_vertex_round /
 * d_edge_round hold sub-round numbers, res->rounds = S (the last sub-round that
 * removed a vertex), vertices_left[s-1] / edges_left[s-1] describe sub-round s.
 * opt.max_rounds bounds the number of sub-rounds (ROUND_LIMIT).  Errors as for
 * pp_peel_kcore, plus INVALID_ARG for bad part offsets.  Synchronizes
 * `stream`. */
pp_status pp_peel_kcore_subrounds(uint32_t n, uint32_t r, uint32_t k, const uint32_t *d_edges,
                                  uint64_t m, uint32_t n_parts, const uint32_t *h_part_off,
                                  int32_t *d_vertex_round, int32_t *d_edge_round,
                                  pp_peel_result *res, const pp_options *opt, void *stream);

/* ------------------------------------------------------------------------
 * Batched decode: many IBLTs of uneven size, decoded together.
 *
 * The tables share one device arena and one frontier: a decode is one CUDA
 * graph launch in which each device-side round peels the current frontier of
 * every table at once (Sec. 1 rounds at k = 2, per table).  Tables never share
 * cells, so every table's rounds, recovered keys and residue equal those of a
 * plain pp_iblt_decode of that table alone.  A batch built from insertions
 * only decodes in tile rounds over the whole arena (opt.rounds), others in
 * binned or direct-atomic rounds.
 * ------------------------------------------------------------------------ */
typedef struct pp_batch pp_batch;

/* Per-table outcome of pp_batch_decode.  round_cap / recovered_per_round are
 * set by the caller (host array or NULL). */
typedef struct pp_table_result {
  uint32_t rounds;           /* rounds that recovered >= 1 key of this table */
  uint32_t stats_complete;   /* 1 if every round fit in opt.stats_rounds */
  uint64_t recovered;        /* keys written to this table's output slots */
  uint64_t items_before;     /* keys in this table before the decode */
  uint64_t residual_cells;   /* non-empty cells left (the table's 2-core) */
  uint32_t round_cap;
  uint32_t pad;
  uint64_t *recovered_per_round; /* keys recovered in round t at [t-1] */
} pp_table_result;

/* Creates n_tables empty tables; table i has n_cells[i] cells, r[i] hash
 * functions (2..PP_MAX_R, mixed values allowed) and seed seeds[i] (same
 * convention as pp_iblt_create).  All tables together must hold fewer than
 * 2^32 - 64 cells.  Allocates ~49 B per cell. */
pp_status pp_batch_create(pp_batch **out, uint32_t n_tables, const uint64_t *n_cells,
                          const uint32_t *r, const uint64_t *seeds, const pp_options *opt);

pp_status pp_batch_destroy(pp_batch *b);

/* Zeroes every table (enqueued on `stream`). */
pp_status pp_batch_clear(pp_batch *b, void *stream);

/* Inserts keys: table i receives d_keys[h_key_offsets[i] .. h_key_offsets[i+1]-1].
 * h_key_offsets: host array of n_tables+1 nondecreasing entries (< 2^32).
 * Enqueued on `stream` (the host arrays are copied before return). */
pp_status pp_batch_insert(pp_batch *b, const uint64_t *d_keys, const uint64_t *h_key_offsets,
                          void *stream);

/* Deletes keys, same layout as pp_batch_insert. */
pp_status pp_batch_delete(pp_batch *b, const uint64_t *d_keys, const uint64_t *h_key_offsets,
                          void *stream);

/* Builds every table from scratch: equal to pp_batch_clear followed by
 * pp_batch_insert.  A large arena is built slab by slab (2^21 cells at a time,
 * each zero-filled and updated while in L2).  Synchronizes `stream` once. */
pp_status pp_batch_build(pp_batch *b, const uint64_t *d_keys, const uint64_t *h_key_offsets,
                         void *stream);

/* Decodes every table in place.  Table i's recovered keys go to
 * d_out_keys[h_out_offsets[i] ..], grouped by round, in no order within a
 * round; each table needs at least as many slots as it holds keys, else
 * CAPACITY before anything runs.  results: host array of n_tables entries.
 * Synchronizes `stream`. */
pp_status pp_batch_decode(pp_batch *b, uint64_t *d_out_keys, const uint64_t *h_out_offsets,
                          pp_table_result *results, void *stream);

/* pp_batch_build (keys as there) followed by pp_batch_decode (outputs as
 * there; a table's range must hold the keys it gets, else CAPACITY and
 * nothing is built).  Same tables, keys and results as the two calls.  When
 * every table lies within two 2^21-cell slabs, the batch is large enough to
 * be built slab by slab and the decode runs tile rounds, the build's write-
 * out of each tile also finds the tile's pure cells (F_1, Sec. 1 round 1), so
 * the decode starts at its first round without reading the arena once more.
 * Synchronizes `stream`. */
pp_status pp_batch_build_decode(pp_batch *b, const uint64_t *d_keys, const uint64_t *h_key_offsets,
                                uint64_t *d_out_keys, const uint64_t *h_out_offsets, pp_table_result *results,
                                void *stream);

/* Copies table `table`'s cells to dst (host if to_host, else device). */
pp_status pp_batch_copy_cells(pp_batch *b, uint32_t table, void *dst, int to_host, void *stream);

/* Replaces the batch's run-time options (max_rounds and stats_rounds keep the
 * values given at creation, which sized the statistics buffers).  Synchronizes
 * the device; the next decode rebuilds its graph. */
pp_status pp_batch_set_options(pp_batch *b, const pp_options *opt);

/* The batch's current options. */
pp_status pp_batch_get_options(const pp_batch *b, pp_options *opt);

/* Autotuner of the batched form (the paper has no counterpart: the knobs are
 * this implementation's).  Searches the batch's run-time knobs -- ctas_per_sm,
 * apply_ctas, binned (1 = address-ordered records, 2 = direct atomics),
 * insert_chunk and rounds (2 = tile rounds, 1 = binned or direct rounds) -- on
 * the caller's own batch and keys: each candidate runs
 * pp_batch_build_decode once untimed and `reps` times timed (CUDA
 * events on `stream`, median).  Candidate 0 is the batch's options as they
 * were.  A candidate whose per-table rounds, recovered counts or residues
 * differ from candidate 0's is discarded and counted in report->mismatches.
 * On return the batch holds the fastest candidate's options, also copied to
 * *best; h_ms (host, PP_TUNE_MAX_CANDIDATES floats, or NULL) receives every
 * candidate's median time (-1 for a discarded one).  The batch's tables are
 * left decoded.  d_keys / h_key_offsets as for pp_batch_build, d_out_keys /
 * h_out_offsets as for pp_batch_decode.  INVALID_ARG for NULL arguments or reps
 * outside 1..64; errors of the build or decode are passed through (the batch
 * then gets its previous options back). */
#define PP_TUNE_MAX_CANDIDATES 32u
typedef struct pp_tune_report {
  uint32_t n_candidates;
  uint32_t best_index;
  float default_ms;   /* candidate 0: the options the batch had */
  float best_ms;
  uint32_t mismatches;
  uint32_t pad;
} pp_tune_report;

pp_status pp_tune_batch(pp_batch *b, const uint64_t *d_keys, const uint64_t *h_key_offsets, uint64_t *d_out_keys,
                        const uint64_t *h_out_offsets, uint32_t reps, pp_options *best, pp_tune_report *report,
                        float *h_ms, void *stream);

/* Number of tables, arena cells (with alignment padding), rounds of the last decode. */
pp_status pp_batch_info(const pp_batch *b, uint32_t *n_tables, uint64_t *total_cells,
                        uint32_t *last_rounds);

/* ------------------------------------------------------------------------
 * Decode service with continuous batching.
 *
 * A host thread owns device arenas of cells and keys.  Submitted requests
 * wait in FIFO order until their table (n_cells cells) and keys (m slots) fit
 * in the free arena space and a table slot is free (admission by free HBM).
 * The thread then runs device iterations, each one round of the
 * round-synchronous decode (Sec. 1 at k = 2 on the IBLT of Sec. 6) for every
 * admitted table at once; tables admitted since the previous iteration are
 * built and scanned in it and join the others at the next round boundary.
 * A request completes when its table has no pure cell left; each result equals
 * that of decoding the request alone with pp_iblt_decode.
 * ------------------------------------------------------------------------ */
typedef struct pp_server pp_server;

typedef struct pp_server_config {
  uint64_t arena_cells; /* cells shared by all admitted tables (default 2^26) */
  uint64_t arena_keys;  /* key/output slots shared by admitted requests (default 2^26) */
  uint32_t max_slots;   /* tables on the device at once (default 4096) */
  uint32_t max_queue;   /* waiting requests before submit returns BUSY (default 2^20) */
  uint32_t r;           /* 0 = any r; 3 or 4 = only that r (specialised kernels) */
  int32_t device;       /* CUDA device of the server thread (default 0) */
} pp_server_config;

/* One decode request.  The table is built from m keys: either h_keys (host
 * memory, kept alive by the caller until the request completes) or, when
 * h_keys is NULL, the synthetic keys SplitMix64(key_seed) outputs 1..m.  The
 * table uses r and table_seed as in pp_iblt_create.  If h_out is not NULL the
 * recovered keys are copied there (out_cap >= m entries) before completion. */
typedef struct pp_request {
  uint64_t n_cells;
  uint32_t r;
  uint32_t pad;
  uint64_t table_seed;
  uint64_t m;
  uint64_t key_seed;
  const uint64_t *h_keys;
  uint64_t *h_out;
  uint64_t out_cap;
  double arrival_s;     /* arrival on pp_server_now()'s clock; 0 = time of submit */
} pp_request;

typedef struct pp_request_result {
  uint64_t ticket;
  int32_t status;       /* PP_OK, or PP_ERR_TIMEOUT if cancelled by a non-draining stop */
  uint32_t rounds;      /* rounds that recovered >= 1 key */
  uint64_t recovered;
  uint64_t items_before;
  uint64_t residual_cells;
  double arrival_s, admit_s, done_s;  /* latency = done_s - arrival_s */
} pp_request_result;

typedef struct pp_server_stats {
  uint64_t submitted, admitted, completed, rejected, pending, active, iterations, keys_recovered;
  uint64_t iteration_us;  /* time spent in device iterations (launch to completion handling) */
  uint64_t gpu_wait_us;   /* part of it the server thread spent waiting for the GPU */
} pp_server_stats;

/* Monotonic clock (seconds) used for arrival and completion times. */
double pp_server_now(void);

void pp_server_config_default(pp_server_config *cfg);

/* Allocates the arenas and starts the server thread. */
pp_status pp_server_start(pp_server **out, const pp_server_config *cfg, const pp_options *opt);

/* Queues a request (thread-safe).  INVALID_ARG for an r or size the server
 * cannot serve, CAPACITY if it can never fit in the arenas, BUSY if the queue
 * is full or the server is stopping. */
pp_status pp_server_submit(pp_server *s, const pp_request *req, uint64_t *ticket);

/* Non-blocking: PP_OK and *res if the request finished (the ticket is then
 * released), PP_ERR_BUSY if not yet, PP_ERR_NOT_FOUND for an unknown ticket. */
pp_status pp_server_poll(pp_server *s, uint64_t ticket, pp_request_result *res);

/* Waits up to timeout_s seconds; PP_ERR_TIMEOUT if the request is not done by then. */
pp_status pp_server_wait(pp_server *s, uint64_t ticket, double timeout_s, pp_request_result *res);

pp_status pp_server_get_stats(pp_server *s, pp_server_stats *out);

/* Stops the thread (drain != 0: finish every queued and admitted request
 * first) and frees the server. */
pp_status pp_server_stop(pp_server *s, int drain);

/* ------------------------------------------------------------------------
 * IBLT decode that allocates nothing.  The paper has no counterpart: this is
 * a convenience for callers that may not allocate device memory while they
 * run -- for instance under a host framework that has already reserved nearly
 * all GPU memory for its own pool, under a "no allocation after start-up"
 * rule, or in latency-bound code that cannot afford cudaFree's implicit
 * device-wide synchronisation.
 *
 * Decodes the caller's table in place, exactly as pp_iblt_decode does (same
 * kernels, same rounds, same results); rounds are driven from the host.
 * d_cells: n_cells pp_cell records on the device (layout above, 32-byte
 * aligned), built with the same r and seed.  d_out_keys/out_cap and *res as for pp_iblt_decode;
 * items_before is computed from the cells (sum of counts / r), and out_cap
 * below it returns CAPACITY before anything is decoded.
 *
 * Working memory is one fixed array of about 17 MB in the library's device
 * code, which each GPU that loads the library keeps until the process exits.
 * It holds tables of at most PP_NOALLOC_MAX_CELLS cells and decodes of at
 * most PP_NOALLOC_MAX_ROUNDS rounds; larger tables give INVALID_ARG, longer
 * decodes ROUND_LIMIT.
 * First call on a device: under the CUDA runtime's default lazy module
 * loading, the library's device code (and with it the array) is loaded on a
 * GPU by the first call of this function there, and that load takes device
 * memory.  Make the first call at start-up, before the host framework
 * reserves its memory pool and before any stream capture, or run the process
 * with CUDA_MODULE_LOADING=EAGER.  Every call looks up the array's device
 * address again (cudaGetSymbolAddress), so nothing stale survives a
 * cudaDeviceReset.  After that first load no call allocates: no
 * cudaMalloc/cudaFree or other allocating routine is called.
 * All calls on a device share the array: calls whose GPU work overlaps race
 * and must be serialised.  Misaligned d_cells or d_out_keys: INVALID_ARG.
 * Synchronizes `stream`.
 * ------------------------------------------------------------------------ */
#define PP_NOALLOC_MAX_CELLS (1u << 20)
#define PP_NOALLOC_MAX_ROUNDS 4096u

pp_status pp_iblt_decode_noalloc(pp_cell *d_cells, uint64_t n_cells, uint32_t r, uint64_t seed,
                                 uint64_t *d_out_keys, uint64_t out_cap, pp_decode_result *res,
                                 void *stream);

/* ------------------------------------------------------------------------
 * Measurement helper (no counterpart in the paper): the rate at which this GPU
 * serves scattered whole-cell accesses, the access pattern of the IBLT rounds.
 * For each i < m, cell d_idx[i] of d_cells (n_cells pp_cell records, 32-byte
 * aligned, device) is read with one 256-bit load and written back changed
 * (mode 0), only read (mode 1) or only overwritten (mode 2); indices >= n_cells
 * are skipped.  The cells' contents are scratch afterwards.  Enqueued on
 * `stream`; time it with events on that stream.  INVALID_ARG for NULL pointers,
 * a mode outside 0..2 or misaligned cells.
 * ------------------------------------------------------------------------ */
pp_status pp_probe_scatter(pp_cell *d_cells, uint64_t n_cells, const uint32_t *d_idx, uint64_t m, int mode,
                           void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PPEEL_H */
