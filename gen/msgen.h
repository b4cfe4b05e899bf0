/*
 * msgen — seeded synthetic 0/1 matrices for tests and benchmarks.
 *
 * This module holds no arithmetic of the maximal-square method: it only draws
 * the input matrices that both the CPU oracle and the CUDA path are fed.  The
 * host (msgen.c) and device (msgen_dev.cu) implementations compute the same
 * function, bit for bit, from the definition below.
 *
 * Generator: SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used counter-style:
 *   gamma   = 0x9E3779B97F4A7C15
 *   mix(z)  = z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
 *             z *= 0x94D049BB133111EB; z ^= z>>31
 *   key     = mix(seed)
 *   draw(k) = mix(key + (k+1)*gamma)          (k-th output of a SplitMix64
 *                                              stream whose state starts at key)
 * Cell (i,j) of an m x n matrix is draw(i*n+j); it is 1 iff
 *   (draw(i*n+j) >> 40) < thr24,   thr24 = floor(p * 2^24)   (0 <= thr24 <= 2^24).
 * The planted-square position uses draws m*n and m*n+1 (see msgen_plant_pos).
 *
 * Bit-packed layout (shared with the library's MS_BITS32 format): row i is
 * ldw uint32 words; bit b (LSB = 0) of word w holds column 32*w+b; bits for
 * columns >= n are padding.
 */
#ifndef MSGEN_H
#define MSGEN_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

uint64_t msgen_mix64(uint64_t z);
uint64_t msgen_draw(uint64_t seed, uint64_t k);
uint32_t msgen_thr24(double p);

/* Bernoulli(thr24 / 2^24) cells into a row-major uint8 matrix (values 0/1). */
void msgen_fill_u8(uint8_t* out, int64_t m, int64_t n, int64_t ld, uint64_t seed, uint32_t thr24);
/* Rows r0 <= i < r1 of the same matrix (any m > i), row i written at
 * out + (i - r0) * ld: disjoint row ranges can be filled concurrently. */
void msgen_fill_u8_rows(uint8_t* out, int64_t r0, int64_t r1, int64_t n, int64_t ld,
                        uint64_t seed, uint32_t thr24);
/* Top-left corner of a planted s x s square, uniform over [0,m-s] x [0,n-s],
 * from draws m*n (row) and m*n+1 (column): r = ((draw>>32) * (m-s+1)) >> 32. */
void msgen_plant_pos(uint64_t seed, int64_t m, int64_t n, int64_t s, int64_t* r, int64_t* c);
/* Set the s x s square with top-left (r,c) to ones. */
void msgen_plant_u8(uint8_t* out, int64_t ld, int64_t r, int64_t c, int64_t s);
/* Pack a uint8 matrix (nonzero = 1) into the MS_BITS32 layout; padding bits
 * are set to pad_value (0 or 1) so tests can check that they are ignored. */
void msgen_pack_bits(const uint8_t* in, int64_t m, int64_t n, int64_t ld,
                     uint32_t* out, int64_t ldw, int pad_value);
/* Unpack MS_BITS32 into uint8 0/1. */
void msgen_unpack_bits(const uint32_t* in, int64_t m, int64_t n, int64_t ldw,
                       uint8_t* out, int64_t ld);

#ifdef __cplusplus
}
#endif
#endif
