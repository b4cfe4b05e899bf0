/*
 * CPU oracle for maximal all-ones square detection — TEST INFRASTRUCTURE ONLY.
 * See oracle.h for the contract, the paper reference and the parity status.
 * Plain single-threaded C, written for checking by eye, not for speed.
 */
#include "oracle.h"
#include <stdlib.h>

#define V(i, j) (v[(int64_t)(i) * ld + (j)] != 0)

static void set_empty(oracle_result* out) {
  out->side = 0;
  out->row = -1;
  out->col = -1;
  out->status = 0;
}

/* Textbook DP, Sec. 1 / Eq. 1 (Sec. 2.1):
 *   dp[i][j] = min(dp[i-1][j], dp[i][j-1], dp[i-1][j-1]) + 1  if v[i][j] = 1,
 *   dp[i][j] = 0                                              if v[i][j] = 0,
 * with dp = 0 outside the matrix.  K = max dp; the witness is the first (i, j)
 * in row-major order with dp[i][j] = K. */
int oracle_dp(const uint8_t* v, int64_t m, int64_t n, int64_t ld, int32_t* dp, int64_t ld_dp,
              oracle_result* out) {
  set_empty(out);
  if (m <= 0 || n <= 0) return 0;
  int32_t* table = dp;
  int64_t ldt = ld_dp;
  if (!table) {
    table = (int32_t*)malloc((size_t)(m * n) * sizeof(int32_t));
    if (!table) return -1;
    ldt = n;
  }
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t j = 0; j < n; ++j) {
      int32_t d = 0;
      if (V(i, j)) {
        int32_t up = (i > 0) ? table[(i - 1) * ldt + j] : 0;
        int32_t left = (j > 0) ? table[i * ldt + j - 1] : 0;
        int32_t diag = (i > 0 && j > 0) ? table[(i - 1) * ldt + j - 1] : 0;
        int32_t mn = up < left ? up : left;
        mn = mn < diag ? mn : diag;
        d = mn + 1;
      }
      table[i * ldt + j] = d;
    }
  }
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j)
      if (table[i * ldt + j] > out->side) {
        out->side = table[i * ldt + j];
        out->row = (int32_t)i;
        out->col = (int32_t)j;
      }
  if (!dp) free(table);
  return 0;
}

/* The same recurrence with one row of dp kept (the O(n)-space variant the
 * paper compares against in Sec. 4.9).  prev[j] holds dp[i-1][j]. */
int oracle_dp_rows(const uint8_t* v, int64_t m, int64_t n, int64_t ld, oracle_result* out) {
  set_empty(out);
  if (m <= 0 || n <= 0) return 0;
  int32_t* prev = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  int32_t* cur = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  if (!prev || !cur) {
    free(prev);
    free(cur);
    return -1;
  }
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t j = 0; j < n; ++j) {
      int32_t d = 0;
      if (V(i, j)) {
        int32_t up = prev[j];
        int32_t left = (j > 0) ? cur[j - 1] : 0;
        int32_t diag = (j > 0) ? prev[j - 1] : 0;
        int32_t mn = up < left ? up : left;
        mn = mn < diag ? mn : diag;
        d = mn + 1;
      }
      cur[j] = d;
      if (d > out->side) {
        out->side = d;
        out->row = (int32_t)i;
        out->col = (int32_t)j;
      }
    }
    int32_t* t = prev;
    prev = cur;
    cur = t;
  }
  free(prev);
  free(cur);
  return 0;
}

/* The frequency-based method of Sec. 3.2 (Algorithm 1).  One pass over the
 * rows keeps, per column, the height of the run of ones ending in the current
 * row (the frequency array; Sec. 3.4's frequency invariant).  Two thresholds,
 * a height and a width, start at one and always grow together: while a row is
 * scanned, a run counts the consecutive columns whose height has reached the
 * height threshold, and once the run is as long as the width threshold a
 * square of that side has been seen, so the best side grows by one, both
 * thresholds grow with it and the run starts again.  A zero, or a column too
 * short for the height threshold, breaks the run.  The paper returns the
 * area; this returns the side, and the place of the last acceptance (the
 * witness: the first corner of a largest square in row-major order). */
int oracle_freq(const uint8_t* v, int64_t m, int64_t n, int64_t ld, oracle_result* out) {
  set_empty(out);
  if (m <= 0 || n <= 0) return 0; /* an empty matrix holds no square */
  int64_t* height = (int64_t*)calloc((size_t)n, sizeof(int64_t));
  if (!height) return -1;
  int64_t best = 0, need_h = 1, need_w = 1;
  for (int64_t i = 0; i < m; ++i) {
    int64_t run = 0;
    for (int64_t j = 0; j < n; ++j) {
      height[j] = V(i, j) ? height[j] + 1 : 0;
      if (height[j] >= need_h) {
        run += 1;
      } else {
        run = 0;
      }
      if (run > 0 && run == need_w) {
        best += 1; /* a square of side need_w ends here */
        need_w += 1;
        need_h += 1;
        run = 0;
        out->row = (int32_t)i;
        out->col = (int32_t)j;
      }
    }
  }
  free(height);
  out->side = (int32_t)best;
  return 0;
}

/* DP map from the frequency array.  After row i, freq[j] is the vertical run of
 * ones ending at (i, j) (the frequency invariant of Sec. 3.4).  A k x k square
 * with bottom-right corner (i, j) is all ones exactly when the k columns
 * j-k+1..j each have a run of at least k, so
 *   dp[i][j] = max{k >= 0 : j-k+1 >= 0 and min(freq[j-k+1..j]) >= k},
 * found here by trying k = 1, 2, ... while the running minimum allows it. */
int oracle_freq_dpmap(const uint8_t* v, int64_t m, int64_t n, int64_t ld, int32_t* dp,
                      int64_t ld_dp, oracle_result* out) {
  set_empty(out);
  if (m <= 0 || n <= 0) return 0;
  int64_t* freq = (int64_t*)calloc((size_t)n, sizeof(int64_t));
  if (!freq) return -1;
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t j = 0; j < n; ++j) freq[j] = V(i, j) ? freq[j] + 1 : 0;
    for (int64_t j = 0; j < n; ++j) {
      int64_t k = 0;
      int64_t run_min = INT64_MAX;
      while (j - k >= 0) {
        int64_t f = freq[j - k];
        run_min = f < run_min ? f : run_min;
        if (run_min < k + 1) break;
        ++k;
      }
      if (dp) dp[i * ld_dp + j] = (int32_t)k;
      if (k > out->side) {
        out->side = (int32_t)k;
        out->row = (int32_t)i;
        out->col = (int32_t)j;
      }
    }
  }
  free(freq);
  return 0;
}

static int square_all_ones(const uint8_t* v, int64_t ld, int64_t r, int64_t c, int64_t s) {
  for (int64_t i = r; i < r + s; ++i)
    for (int64_t j = c; j < c + s; ++j)
      if (!V(i, j)) return 0;
  return 1;
}

/* Brute force over every square: for each side s from the largest possible
 * down, scan the bottom-right corners in row-major order and return the first
 * all-ones one. */
int oracle_brute(const uint8_t* v, int64_t m, int64_t n, int64_t ld, oracle_result* out) {
  set_empty(out);
  if (m <= 0 || n <= 0) return 0;
  int64_t smax = m < n ? m : n;
  for (int64_t s = smax; s >= 1; --s)
    for (int64_t i = s - 1; i < m; ++i)
      for (int64_t j = s - 1; j < n; ++j)
        if (square_all_ones(v, ld, i - s + 1, j - s + 1, s)) {
          out->side = (int32_t)s;
          out->row = (int32_t)i;
          out->col = (int32_t)j;
          return 0;
        }
  return 0;
}

int oracle_erode(const uint8_t* v, int64_t m, int64_t n, int64_t ld, int64_t t, uint8_t* s,
                 int64_t ld_s) {
  if (t < 1) return -1;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      int ok = (i - t + 1 >= 0) && (j - t + 1 >= 0);
      if (ok) ok = square_all_ones(v, ld, i - t + 1, j - t + 1, t);
      s[i * ld_s + j] = (uint8_t)ok;
    }
  return 0;
}

/* K from the O(n)-space recurrence, then a second pass over the same rows
 * collects every cell whose dp equals K, in row-major order. */
int oracle_all_max(const uint8_t* v, int64_t m, int64_t n, int64_t ld, int32_t* corners,
                   int64_t cap, int64_t* count, oracle_result* out) {
  *count = 0;
  if (oracle_dp_rows(v, m, n, ld, out) != 0) return -1;
  const int32_t K = out->side;
  if (K == 0) return 0;
  int32_t* prev = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  int32_t* cur = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  if (!prev || !cur) {
    free(prev);
    free(cur);
    return -1;
  }
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t j = 0; j < n; ++j) {
      int32_t d = 0;
      if (V(i, j)) {
        int32_t up = prev[j];
        int32_t left = (j > 0) ? cur[j - 1] : 0;
        int32_t diag = (j > 0) ? prev[j - 1] : 0;
        int32_t mn = up < left ? up : left;
        mn = mn < diag ? mn : diag;
        d = mn + 1;
      }
      cur[j] = d;
      if (d == K) {
        if (*count < cap) {
          corners[2 * *count] = (int32_t)i;
          corners[2 * *count + 1] = (int32_t)j;
        }
        ++*count;
      }
    }
    int32_t* t = prev;
    prev = cur;
    cur = t;
  }
  free(prev);
  free(cur);
  return 0;
}

/* Two slices of c are kept: prev = slice z-1, cur = slice z (m x n each). */
int oracle_cube(const uint8_t* v, int64_t d, int64_t m, int64_t n, int64_t ld, int64_t ld_slice,
                oracle_cube_result* out) {
  out->side = 0;
  out->slice = out->row = out->col = -1;
  if (d <= 0 || m <= 0 || n <= 0) return 0;
  int32_t* prev = (int32_t*)calloc((size_t)(m * n), sizeof(int32_t));
  int32_t* cur = (int32_t*)calloc((size_t)(m * n), sizeof(int32_t));
  if (!prev || !cur) {
    free(prev);
    free(cur);
    return -1;
  }
#define C(t, i, j) (((i) < 0 || (j) < 0) ? 0 : (t)[(i) * n + (j)])
  for (int64_t z = 0; z < d; ++z) {
    for (int64_t i = 0; i < m; ++i) {
      for (int64_t j = 0; j < n; ++j) {
        int32_t c = 0;
        if (v[z * ld_slice + i * ld + j] != 0) {
          int32_t mn = C(prev, i, j);
          const int32_t nb[6] = {C(prev, i - 1, j), C(prev, i, j - 1), C(prev, i - 1, j - 1),
                                 C(cur, i - 1, j), C(cur, i, j - 1), C(cur, i - 1, j - 1)};
          for (int k = 0; k < 6; ++k) mn = nb[k] < mn ? nb[k] : mn;
          c = mn + 1;
        }
        cur[i * n + j] = c;
        if (c > out->side) {
          out->side = c;
          out->slice = (int32_t)z;
          out->row = (int32_t)i;
          out->col = (int32_t)j;
        }
      }
    }
    int32_t* t = prev;
    prev = cur;
    cur = t;
  }
#undef C
  free(prev);
  free(cur);
  return 0;
}
