/*
 * CPU oracle for maximal all-ones square detection — TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * call this code.  The CUDA library never links, loads or calls it, and it
 * shares no code with the CUDA library: both are fed the same seeded inputs
 * from the generator module (gen/), and nothing else is common.
 *
 * Paper: S. Bhandari, "An Efficient Frequency-Based Approach for Maximal
 * Square Detection in Binary Matrices" (arXiv 2503.18974).
 *
 * Every routine takes a row-major uint8 matrix (m rows, n columns, row stride
 * ld >= n bytes; a nonzero byte is a 1) and reports:
 *   side  = largest k such that some k x k submatrix is all ones
 *           (the paper's Algorithm 1 returns the area side*side),
 *   row/col = bottom-right corner of the first such square in row-major order
 *           of that corner, or -1/-1 when side == 0 (including m == 0 or n == 0).
 * Optionally dp[i*ld_dp + j] = side of the largest all-ones square whose
 * bottom-right corner is (i, j)  (Sec. 1 and Eq. 1).
 *
 * Parity status of each routine (pins live in tests/test_oracle.py):
 *   oracle_dp          pinned: brute force, closed forms, invariants
 *   oracle_dp_rows     pinned: equals oracle_dp on all pinned cases
 *   oracle_freq        pinned: brute force, closed forms, equals oracle_dp
 *   oracle_freq_dpmap  pinned: equals oracle_dp's map, closed forms
 *   oracle_brute       pinned: independent numpy enumeration, closed forms
 *   oracle_erode       pinned: equals [dp >= t], closed forms
 *   oracle_all_max     pinned: brute-force enumeration, closed forms
 *   oracle_cube        pinned: brute-force enumeration, closed forms, slices
 */
#ifndef MS_ORACLE_H
#define MS_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t side, row, col, status;
} oracle_result;

/* Textbook DP (Sec. 1, Eq. 1 of Sec. 2.1): full O(mn) table. dp may be NULL,
 * in which case a private table is allocated.  Returns 0, or -1 on allocation
 * failure. */
int oracle_dp(const uint8_t* v, int64_t m, int64_t n, int64_t ld, int32_t* dp, int64_t ld_dp,
              oracle_result* out);

/* Space-optimised DP (Sec. 2.1 and Sec. 4.9): keeps one dp row, O(n) space. */
int oracle_dp_rows(const uint8_t* v, int64_t m, int64_t n, int64_t ld, oracle_result* out);

/* The paper's frequency-based Algorithm 1 (Sec. 3.2), step for step, with the
 * (row, col) of every successful validation recorded; the last record is the
 * witness.  Returns found_max_width (not its square). */
int oracle_freq(const uint8_t* v, int64_t m, int64_t n, int64_t ld, oracle_result* out);

/* DP map from the frequency array of Algorithm 1: freq[j] after row i is the
 * vertical run of ones ending at (i, j) (Sec. 3.4, frequency invariant), and
 * dp[i][j] = max{k : min(freq[j-k+1..j]) >= k}, searched k = 1, 2, ... */
int oracle_freq_dpmap(const uint8_t* v, int64_t m, int64_t n, int64_t ld, int32_t* dp,
                      int64_t ld_dp, oracle_result* out);

/* Brute force: every (top-left, side) checked cell by cell.  Small inputs only. */
int oracle_brute(const uint8_t* v, int64_t m, int64_t n, int64_t ld, oracle_result* out);

/* Bitmap of bottom-right corners of all-ones t x t squares (t >= 1), by
 * definition: s[i*ld_s + j] = 1 iff every cell of the t x t square ending at
 * (i, j) is one (out-of-range cells count as zero).  Used to check the
 * bit-packed erosion path. */
int oracle_erode(const uint8_t* v, int64_t m, int64_t n, int64_t ld, int64_t t, uint8_t* s,
                 int64_t ld_s);

/* All maximal squares (the paper's "all maximal squares" reading, Sec. 3.4
 * and Sec. 6): the bottom-right corner of every all-ones square of the largest
 * side K, i.e. every (i, j) with dp[i][j] == K, in row-major order.  Writes up
 * to cap (row, col) pairs to corners[2*k], [2*k+1] and the total number to
 * *count (none when K == 0).  Returns 0, or -1 on allocation failure. */
int oracle_all_max(const uint8_t* v, int64_t m, int64_t n, int64_t ld, int32_t* corners,
                   int64_t cap, int64_t* count, oracle_result* out);

/* Largest all-ones cube of a 3-D volume (the paper's future-work extension,
 * Sec. 6): v[z*ld_slice + i*ld + j] for z < d, i < m, j < n.  The 3-D
 * analogue of Eq. 1: c[z][i][j] = 1 + min of the seven neighbours that
 * precede it in z, i or j (0 outside the volume) on a one, 0 on a zero.
 * side = max c; (slice, row, col) = the first corner in (z, i, j) order with
 * c == side, or -1s when side == 0.  Returns 0, or -1 on allocation failure. */
typedef struct {
  int32_t side, slice, row, col;
} oracle_cube_result;
int oracle_cube(const uint8_t* v, int64_t d, int64_t m, int64_t n, int64_t ld, int64_t ld_slice,
                oracle_cube_result* out);

#ifdef __cplusplus
}
#endif
#endif
