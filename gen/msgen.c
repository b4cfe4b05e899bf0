/* Host implementation of the seeded input generator; definitions in msgen.h. */
#include "msgen.h"
#include <string.h>

#define MSGEN_GAMMA 0x9E3779B97F4A7C15ULL

uint64_t msgen_mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ULL;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return z;
}

uint64_t msgen_draw(uint64_t seed, uint64_t k) {
  return msgen_mix64(msgen_mix64(seed) + (k + 1) * MSGEN_GAMMA);
}

uint32_t msgen_thr24(double p) {
  if (!(p > 0.0)) return 0;
  if (p >= 1.0) return 1u << 24;
  return (uint32_t)(p * 16777216.0);
}

void msgen_fill_u8(uint8_t* out, int64_t m, int64_t n, int64_t ld, uint64_t seed, uint32_t thr24) {
  msgen_fill_u8_rows(out, 0, m, n, ld, seed, thr24);
}

void msgen_fill_u8_rows(uint8_t* out, int64_t r0, int64_t r1, int64_t n, int64_t ld,
                        uint64_t seed, uint32_t thr24) {
  const uint64_t key = msgen_mix64(seed);
  for (int64_t i = r0; i < r1; ++i) {
    uint8_t* row = out + (i - r0) * ld;
    uint64_t k = (uint64_t)(i * n);
    for (int64_t j = 0; j < n; ++j, ++k) {
      uint64_t z = msgen_mix64(key + (k + 1) * MSGEN_GAMMA);
      row[j] = (uint8_t)((uint32_t)(z >> 40) < thr24);
    }
  }
}

static int64_t msgen_uniform(uint64_t z, int64_t count) {
  return (int64_t)(((z >> 32) * (uint64_t)count) >> 32);
}

void msgen_plant_pos(uint64_t seed, int64_t m, int64_t n, int64_t s, int64_t* r, int64_t* c) {
  uint64_t base = (uint64_t)(m * n);
  *r = msgen_uniform(msgen_draw(seed, base), m - s + 1);
  *c = msgen_uniform(msgen_draw(seed, base + 1), n - s + 1);
}

void msgen_plant_u8(uint8_t* out, int64_t ld, int64_t r, int64_t c, int64_t s) {
  for (int64_t i = r; i < r + s; ++i) memset(out + i * ld + c, 1, (size_t)s);
}

void msgen_pack_bits(const uint8_t* in, int64_t m, int64_t n, int64_t ld,
                     uint32_t* out, int64_t ldw, int pad_value) {
  for (int64_t i = 0; i < m; ++i) {
    const uint8_t* row = in + i * ld;
    uint32_t* orow = out + i * ldw;
    for (int64_t w = 0; w < ldw; ++w) {
      uint32_t word = 0;
      for (int b = 0; b < 32; ++b) {
        int64_t j = 32 * w + b;
        uint32_t bit = (j < n) ? (row[j] != 0) : (uint32_t)(pad_value != 0);
        word |= bit << b;
      }
      orow[w] = word;
    }
  }
}

void msgen_unpack_bits(const uint32_t* in, int64_t m, int64_t n, int64_t ldw,
                       uint8_t* out, int64_t ld) {
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j)
      out[i * ld + j] = (uint8_t)((in[i * ldw + (j >> 5)] >> (j & 31)) & 1u);
}
