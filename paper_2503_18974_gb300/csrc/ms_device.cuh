// Device-side building blocks of libms (sm_103a).
//
// The method: for every cell, dp[i][j] = side of the largest all-ones square
// with bottom-right corner (i, j) (Eq. 1, Sec. 2.1); the answer is max dp and
// the first cell reaching it in row-major order (where the paper's
// Algorithm 1, Sec. 3.2, makes its last validation).
//
// Restatement used on the GPU.  Eq. 1 on a one cell is
//   dp[i][j] = 1 + min(dp[i-1][j], dp[i][j-1], dp[i-1][j-1]),
// and 0 on a zero cell.  In row units A = i + 1 - dp (the top row of the
// largest square ending at the cell) the minimum becomes a maximum:
//   A[i][j] = max(A[i-1][j], A[i-1][j-1], A[i][j-1] - 1)  on a one,
//   A[i][j] = i + 1                                        on a zero,
// because the row index of the neighbours above is one less.  The paper's
// frequency array (the vertical run h, Sec. 3.4) is implicit: A >= i + 1 - h.
// A is a small non-negative integer; two independent tiles share every 32-bit
// register (16x2 SIMD), so one max.u16x2 serves two cells.
#pragma once
#include <cstdint>

#include "../../include/ms.h"

namespace ms {

constexpr uint32_t kBias = 64;             // row offset so that every value stays >= 1
constexpr int kHalo = 32;                  // halo rows above / columns left of a tile
constexpr uint64_t kKeyMask = (1ull << 40) - 1;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kSpinLimit = 1 << 22;        // iteration cap of bounded waits
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // a wait gives up after ~1 s

// ---- per-matrix job description and state ---------------------------------

struct JobState {
  unsigned long long key;  // (side << 40) | (kKeyMask - (row*n + col)), atomicMax
  int32_t box[4];          // unresolved region: row lo, row hi, col lo, col hi
  int32_t status;          // ms_status of device-side problems
  int32_t done;            // tile-pass blocks finished (fused size-only finish)
};

struct Job {
  const void* data;
  int64_t m, n, ld;        // ld in bytes (MS_U8) or words (MS_BITS32)
  int32_t fmt;
  int32_t P;               // columns per lane in a tile (tile width = 32*P)
  int32_t band_rows;       // rows a tile counts
  int32_t bands, strips;
  int32_t aligned;         // U8: data and ld allow 16-byte vector loads
  int64_t tile0;           // index of this job's first tile in its launch group
  int32_t* dp;             // optional dp map (device), may be null
  int64_t ld_dp;
  int32_t dp_aligned;      // dp and ld_dp allow 32-byte (2) or 16-byte (1) vector stores
  int32_t tile_kind;       // size-only tile pass: 0 dp recurrence, 1 bitplane tiles (P = 32)
  ms_result* out;
  JobState* st;
  uint32_t* carry;         // fix-up strip carries (carry_words(m, strips_fix) words, 16-B aligned)
  int32_t* progress;       // fix-up per-strip published row counts
  int32_t strips_fix;      // capacity of carry/progress in strips
  int32_t test_hold;       // test hook: the first fix-up strip never publishes carries
  uint32_t* bits_scratch;  // size-only fix-up bitplanes (3 x m x (ceil(n/32)+2) words), or null
  int32_t* corners;        // all largest squares: (row, col) pairs, or null
  int64_t corners_cap;     // pairs that fit in corners
  unsigned long long* corners_count;  // corners found (may exceed the capacity)
  // Bitplane tiles with fix-up scratch: the first row of tile t holding an
  // S_33 cell (INT_MAX: none); from that row on the tile wrote its rows of
  // S_33 (counted words) into the third scratch plane (row stride
  // ceil(n/32) words), which the fix-up starts from.  Null otherwise.
  int32_t* first33;
};

// Appends (i, c) to the job's list of largest-square corners.
__device__ __forceinline__ void emit_corner(const Job& j, int64_t i, int64_t c) {
  const unsigned long long k = atomicAdd(j.corners_count, 1ull);
  if ((int64_t)k < j.corners_cap) {
    j.corners[2 * k] = (int32_t)i;
    j.corners[2 * k + 1] = (int32_t)c;
  }
}

// Fix-up strip carries: one uint16 per window row and strip, each strip's
// rows padded to a multiple of 8 so that 8 rows load as one 16-byte vector.
__host__ __device__ constexpr int64_t carry_stride16(int64_t m) { return (m + 7) / 8 * 8; }
__host__ __device__ constexpr int64_t carry_words(int64_t m, int64_t strips) {
  return carry_stride16(m) / 2 * strips;
}

// ---- 16x2 SIMD helpers ---------------------------------------------------

__device__ __forceinline__ uint32_t vmax2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t vadd2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("add.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
// (a where mask bits are set) | (b elsewhere): one LOP3
__device__ __forceinline__ uint32_t select_bits(uint32_t a, uint32_t b, uint32_t mask) {
  return (a & mask) | (b & ~mask);
}
// PTX prmt in its default mode, where bit 3 of a selector nibble replicates
// the sign (most significant bit) of the selected byte across the output byte.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
  return r;
}
// Marks each nonzero byte of x with its most significant bit (other bits are junk).
__device__ __forceinline__ uint32_t nonzero_msb(uint32_t x) {
  return ((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x;
}

// A store asking L2 to keep its line (evict-last policy): for the few words
// a kernel hands to the next one, which the streamed input would otherwise
// push out of L2 before they are read.
__device__ __forceinline__ void st_keep_l2(uint32_t* p, uint32_t v) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol)
               : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// ---- input loading --------------------------------------------------------
// A lane owns P consecutive columns of a tile row.  Raw<P, FMT> holds them as
// loaded, with no arithmetic on the loaded value, so that a load issued D
// steps ahead is not waited for until its row is consumed.
// MS_U8: ceil(P/4) words of bytes; MS_BITS32: the 32-bit word holding them.

template <int P, int FMT>
struct Raw;

template <int P>
struct Raw<P, MS_U8> {
  static constexpr int W = (P + 3) / 4;
  uint32_t w[W];
};
template <int P>
struct Raw<P, MS_BITS32> {
  uint32_t word;
};

// Per-lane constants that turn a Raw into cells: for MS_BITS32 the shift of
// the lane's columns inside their word and the mask of columns < n.
struct LaneCols {
  uint32_t shift;
  uint32_t mask;
};
template <int P>
__device__ __forceinline__ LaneCols lane_cols(int64_t col, int64_t n) {
  LaneCols c;
  c.shift = (uint32_t)(col & 31);
  const int64_t valid = n - col;
  const uint32_t full = P >= 32 ? 0xffffffffu : ((1u << (P & 31)) - 1u);
  c.mask = valid <= 0 ? 0u : (valid >= P ? full : ((1u << valid) - 1u));
  return c;
}

// Cells ready for pair_mask: MS_U8 words with each nonzero byte marked in its
// most significant bit, MS_BITS32 the lane's P bits in the low bits.
template <int P, int FMT>
struct Cells;
template <int P>
struct Cells<P, MS_U8> {
  uint32_t w[Raw<P, MS_U8>::W];
};
template <int P>
struct Cells<P, MS_BITS32> {
  uint32_t bits;
};

// Bytes known to be 0 or 1 need no nonzero test: a shift puts each byte's
// bit 0 into its most significant bit.  Every raw word is ORed into `seen`,
// so the caller can tell afterwards whether the assumption held.
template <int P>
__device__ __forceinline__ Cells<P, MS_U8> cells_of01(const Raw<P, MS_U8>& r, uint32_t& seen) {
  Cells<P, MS_U8> c;
#pragma unroll
  for (int i = 0; i < Raw<P, MS_U8>::W; ++i) {
    c.w[i] = r.w[i] << 7;
    seen |= r.w[i];
  }
  return c;
}
template <int P>
__device__ __forceinline__ Cells<P, MS_U8> cells_of(const Raw<P, MS_U8>& r, const LaneCols&) {
  Cells<P, MS_U8> c;
#pragma unroll
  for (int i = 0; i < Raw<P, MS_U8>::W; ++i) c.w[i] = nonzero_msb(r.w[i]);
  return c;
}
template <int P>
__device__ __forceinline__ Cells<P, MS_BITS32> cells_of(const Raw<P, MS_BITS32>& r,
                                                        const LaneCols& lc) {
  Cells<P, MS_BITS32> c;
  c.bits = (r.word >> lc.shift) & lc.mask;
  return c;
}

// 16x2 mask of pair k: low half 0xffff if the low tile's cell is one, high
// half 0xffff if the high tile's cell is one.
template <int P>
__device__ __forceinline__ uint32_t pair_mask(const Cells<P, MS_U8>& lo,
                                              const Cells<P, MS_U8>& hi, int k) {
  const uint32_t b = (uint32_t)(k & 3);
  const uint32_t sel = (8u | b) | ((8u | b) << 4) | ((12u | b) << 8) | ((12u | b) << 12);
  return prmt(lo.w[k >> 2], hi.w[k >> 2], sel);
}
template <int P>
__device__ __forceinline__ uint32_t pair_mask(const Cells<P, MS_BITS32>& lo,
                                              const Cells<P, MS_BITS32>& hi, int k) {
  // cells k of both tiles at bits k and 16 + k of one word (columns 16..31
  // of a 32-column chunk use the upper halves), then shifted to bits 15 and
  // 31 and replicated across their halves
  const uint32_t w = k < 16 ? ((lo.bits & 0xffffu) | (hi.bits << 16))
                            : ((lo.bits >> 16) | (hi.bits & 0xffff0000u));
  return prmt(w << (15 - (k & 15)), 0u, 0xBB99u);
}

// ---- size-only tile pass in dp units (fp16x2) ------------------------------
// Inside a tile's window every dp_w is at most the window's width, 32*P <= 1024
// columns, so the window's dp values themselves are exact in fp16 (whose
// integers are exact up to 2048).  On a one dp = 1 + min(up, left, diag), on a
// zero 0: with v = 1.0 or 0.0 per half that is v * m + v after two packed
// minima m, one fma.f16x2, which issues on the FMA pipe while the minima,
// prmt and lop3 of the row-unit form all share the (half-rate) ALU pipe.
// Non-negative fp16 values order like their bit patterns, so min.u16x2 and
// max.u16x2 on the bits are exact minima and maxima.
constexpr uint32_t kOneH = 0x3C00u;        // fp16 1.0
constexpr uint32_t kHaloH2 = 0x50005000u;  // fp16 32.0 (= kHalo) in both halves
static_assert(kHalo == 32, "kHaloH2 encodes kHalo");

__device__ __forceinline__ uint32_t hfma2(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
__device__ __forceinline__ uint32_t imul(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("mul.lo.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
// The integer held by fp16 bits `h` (a whole number 0..2047): IEEE binary16
// stores 2^(e-15) * (1 + f/1024), so the value is (1024 + f) >> (25 - e).
__device__ __forceinline__ int h16_int(uint32_t h) {
  h &= 0xffffu;
  return h == 0u ? 0 : (int)((1024u | (h & 1023u)) >> (25u - (h >> 10)));
}

// 0/1 bytes scaled to 0x3C (the high byte of fp16 1.0): one multiply per word
// (no carries between bytes while every byte is 0 or 1).  Every raw word is
// ORed into `seen`, so the caller can tell afterwards whether that held.
template <int P>
__device__ __forceinline__ Cells<P, MS_U8> cells_h01(const Raw<P, MS_U8>& r, uint32_t& seen) {
  Cells<P, MS_U8> c;
#pragma unroll
  for (int i = 0; i < Raw<P, MS_U8>::W; ++i) {
    c.w[i] = imul(r.w[i], 0x3Cu);
    seen |= r.w[i];
  }
  return c;
}
// Pair k as fp16x2 ones: byte 1 <- low tile's byte, byte 3 <- high tile's
// byte, bytes 0 and 2 <- their (clear) sign bits replicated.
template <int P>
__device__ __forceinline__ uint32_t pair_one(const Cells<P, MS_U8>& lo, const Cells<P, MS_U8>& hi,
                                             int k) {
  const uint32_t b = (uint32_t)(k & 3);
  const uint32_t sel = (8u | b) | (b << 4) | ((12u | b) << 8) | ((4u | b) << 12);
  return prmt(lo.w[k >> 2], hi.w[k >> 2], sel);
}
// MS_BITS32: columns 0..15 of both tiles interleaved by halves (and the same
// shifted right by 5), then columns 16..31 likewise; pair k is one AND and
// one multiply that moves bit j of each half to the fp16 1.0 pattern
// (0x3C00 = 15 << 10).
struct BitsH {
  uint32_t c[4];
};
template <int P>
__device__ __forceinline__ BitsH bits_h(const Cells<P, MS_BITS32>& lo,
                                        const Cells<P, MS_BITS32>& hi) {
  BitsH h;
  h.c[0] = prmt(lo.bits, hi.bits, 0x5410u);
  h.c[1] = h.c[0] >> 5;
  h.c[2] = prmt(lo.bits, hi.bits, 0x7632u);
  h.c[3] = h.c[2] >> 5;
  return h;
}
__device__ __forceinline__ uint32_t pair_one(const BitsH& h, int k) {
  const int j = k & 15;
  const int g = (k >> 4) * 2 + (j > 10 ? 1 : 0);
  const int s = j > 10 ? j - 5 : j;
  return imul(h.c[g] & (0x00010001u << s), kOneH >> s);
}

// ---- results --------------------------------------------------------------

struct Best {
  int32_t val;  // largest dp seen, its first position
  int32_t row;
  int32_t col;
  int32_t big_r0, big_r1;  // rows holding a dp above the halo (big_r0 = INT_MAX: none)
  int64_t big_c0, big_c1;  // columns of the lane chunks holding one
};

__device__ __forceinline__ unsigned long long make_key(int32_t val, int64_t row, int64_t col,
                                                       int64_t n) {
  if (val <= 0) return 0ull;
  return ((unsigned long long)val << 40) |
         (kKeyMask - (unsigned long long)(row * n + col));
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    unsigned long long o = __shfl_xor_sync(kFull, v, d);
    v = o > v ? o : v;
  }
  return v;
}

}  // namespace ms
