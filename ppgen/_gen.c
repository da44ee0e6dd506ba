/* Seeded input streams for the peeling workloads (input generation only).
 *
 * SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) and xorshift64* (Vigna,
 * ACM TOMS 2016), written from their published definitions.  Nothing here
 * hashes keys into cells or peels anything: this file only produces keys and
 * edge endpoints, for the CPU oracle and the CUDA path alike.
 */
#include <stdint.h>
#include <stddef.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Outputs start..start+count-1 of SplitMix64 seeded with `seed`:
 * output i = mix(seed + (i+1) * GAMMA). */
void ppgen_splitmix64(uint64_t seed, uint64_t start, uint64_t count, uint64_t *out) {
  for (uint64_t i = 0; i < count; ++i) out[i] = sm_mix(seed + (start + i + 1) * GAMMA);
}

static uint64_t xs_seed_state(uint64_t seed) {
  uint64_t s = sm_mix(seed + GAMMA);
  return s ? s : GAMMA;
}

/* First `count` outputs of xorshift64* seeded with `seed`. */
void ppgen_xorshift64star(uint64_t seed, uint64_t count, uint64_t *out) {
  uint64_t x = xs_seed_state(seed);
  for (uint64_t i = 0; i < count; ++i) {
    x ^= x >> 12;
    x ^= x << 25;
    x ^= x >> 27;
    out[i] = x * 0x2545F4914F6CDD1DULL;
  }
}

/* m edges, row-major (m x r) uint32: draw e*r+j of xorshift64*(seed) gives
 * endpoint j of edge e.  Partitioned form: endpoint j = off[j] +
 * floor(draw * size[j] / 2^64).  Uniform form (size[j] = n, off[j] = 0 for all
 * j) is the same call with every part set to the whole vertex range. */
void ppgen_edges(uint64_t seed, uint64_t m, uint32_t r, const uint32_t *off,
                 const uint32_t *size, uint32_t *out) {
  uint64_t x = xs_seed_state(seed);
  for (uint64_t e = 0; e < m; ++e) {
    for (uint32_t j = 0; j < r; ++j) {
      x ^= x >> 12;
      x ^= x << 25;
      x ^= x >> 27;
      uint64_t d = x * 0x2545F4914F6CDD1DULL;
      out[e * r + j] = off[j] + (uint32_t)(((unsigned __int128)d * size[j]) >> 64);
    }
  }
}
