// Size-only tile pass by bitplanes: the largest square side and its witness
// of every tile from the corner bitmaps S_t (Eq. 1 and the threshold test of
// Algorithm 1, Sec. 3.2, restated on bits), 32 cells per 32-bit word.
//
// S_t(i, c) = 1 iff the t x t square with bottom-right corner (i, c) is all
// ones (dp(i, c) >= t, Eq. 1), S_1 = the input.  Four t-squares with the
// corners of a (t+s)-square cover it when s <= t, so
//   S_{t+s}(i, c) = U(i, c) & U(i - s, c),  U(i, c) = S_t(i, c) & S_t(i, c - s),
// which gives S_2, S_4, ..., S_32 by doubling (s = t) and any S_{P+s} from
// S_P (P a power of two, s < P).  Batches can run these tiles too (one per
// task of their persistent launch, `k_batch_tiles` below).
//
// A warp takes one tile of the dp-recurrence tile pass's geometry (1024
// window columns, of which the first 32 are halo unless the strip is the
// matrix's first; `band_rows` counted rows below a 32-row halo).  Lane l owns
// window word l (columns wc0 + 32l ... + 31) and walks the window's rows top
// to bottom.  Per row it packs its 32 cells into a word (bytes: four
// multiplies move 8 cells' 0/1 bytes side by side; packed input: the word
// itself), derives S_2 ... S_32 of the row from the same-row neighbour word
// (one shuffle per level) and the level's rows above (registers for levels
// 1, 2 and 4, else a ring per level in shared memory as deep as the level),
// and stores the row's levels in the rings, which also serve the threshold
// tests below.
//
// Largest side, tile by tile (the method's threshold idea: a tile's best so
// far, K, only ever grows, and a row matters only if it holds a (K+1)-square
// corner): every counted row tests S_{K+1} and raises K while the test holds;
// the first row where K reaches its final value holds the tile's first
// K-corner in row-major order.  Inside the window S_t is exact for every
// counted cell while t <= kHalo + 1 (a (kHalo+1)-square ending on a counted
// cell lies inside the window), so K stops at kHalo + 1: from then on the
// rows holding S_{kHalo+1} cells are flagged into the matrix's box for the
// exact fix-up, as in the dp-recurrence tile pass.
#pragma once
#include "ms_kernels.cuh"

namespace ms {
namespace bt {

constexpr int kWarps = 8;                     // warps per block (at most)
constexpr int kRowWords = 32;                 // ring row: word l = lane l
// ring rows of level 2^p (p >= 1; S_1 needs none: the only test on it, of
// S_1 itself, reads the row's own word): 2^p for p < 5 (the doubling reads
// row r - 2^p, a threshold test rows down to r - 2^p + 1), 2 for level 32
// (tests of S_32 and S_33 read rows r and r - 1 only); level 2^p starts at
// ring row 2^p - 2.  With the 4 KB input ring a warp takes exactly 8 KB.
constexpr int kRingRows = 2 + 4 + 8 + 16 + 2;
__host__ __device__ constexpr int ring_depth(int p) { return p < 5 ? 1 << p : 2; }
constexpr int kRingWords = kRingRows * kRowWords;
constexpr int kInBytes = 4096;                // input ring per warp
constexpr int kWarpBytes = kInBytes + kRingWords * 4;
static_assert(kWarpBytes == 8192, "a bitplane tile warp takes what a dp-recurrence tile warp does");
constexpr int kTop = kHalo + 1;               // largest exact level (33)
static_assert(kHalo == 32, "level rings cover shifts up to 32 rows");

// A slot holds one window row in column order: bytes as 64 chunks of 16
// (chunk c = columns wc0 + 16c ...), packed input as one word per lane.
template <int FMT>
struct InGeom {
  static constexpr int kSlot = FMT == MS_U8 ? 1024 : 128;
  static constexpr int kDepth = kInBytes / kSlot;  // rows in flight
  static_assert((kDepth & (kDepth - 1)) == 0 && kDepth >= 4, "input ring depth");
};

// A chunk of an unaligned matrix: its first `nvalid` bytes by byte loads,
// zeros after them (out of line: only such lanes take it, and the row loop
// stays small for the instruction cache).
static __device__ __noinline__ void fill_chunk(uint32_t d, const uint8_t* p, int nvalid) {
  uint32_t w[4] = {0u, 0u, 0u, 0u};
  for (int b = 0; b < nvalid; ++b) w[b >> 2] |= (uint32_t)__ldg(p + b) << (8 * (b & 3));
  st_shared_chunk<16>(d, w);
}

// Streams the tile's window rows into the warp's ring.  Bytes: lane l copies
// chunks l and 32 + l, so that each of the warp's two 16-byte copies reads
// 512 contiguous bytes and writes them contiguously (cp.async for chunks of
// 16-byte-aligned rows, a ragged last chunk with a partial source size that
// zero-fills the rest; byte loads for unaligned rows; nothing beyond the
// matrix's last column is read).  Packed: lane l copies word l.
template <int FMT, bool RAGGED>
struct Reader {
  using G = InGeom<FMT>;
  const uint8_t* ptr;   // the lane's first chunk (bytes) or word (packed) of window row `row`
  const uint8_t* safe;
  int64_t stride;
  int row, nrows;
  // per chunk: 0 no cells; 1..16 an async copy reading that many bytes (the
  // rest of the 16 zero-filled); 32 + v byte loads of v bytes (unaligned
  // rows).  Without RAGGED every async copy reads 16 bytes (a ragged chunk
  // takes the byte loads), which keeps the copy's size a constant: the
  // variant for matrices whose rows hold whole chunks.
  int mode[2], nvalid[2];
  uint32_t dst;            // the lane's first chunk in slot 0

  __device__ __forceinline__ void init(const Tile& g, int lane, uint32_t ring) {
    row = 0;
    nrows = g.nrows;
    safe = g.base;
    if constexpr (FMT == MS_U8) {
      stride = g.ld;
      dst = ring + 16 * lane;
      ptr = g.base + g.wr0 * g.ld + g.wc0 + 16 * lane;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int64_t valid = g.n - (g.wc0 + 16 * (lane + 32 * k));
        const int v = (int)(valid < 16 ? (valid < 0 ? 0 : valid) : 16);
        if constexpr (RAGGED) {
          mode[k] = v == 0 ? 0 : g.aligned ? v : 32 + v;
        } else {
          nvalid[k] = v;
          mode[k] = v == 0 ? 0 : (v == 16 && g.aligned) ? 1 : 2;
        }
      }
    } else {
      const int64_t col = g.wc0 + 32 * (int64_t)lane;
      stride = g.ld * 4;
      dst = ring + 4 * lane;
      ptr = g.base + (g.wr0 * g.ld + (col >> 5)) * 4;
      nvalid[0] = nvalid[1] = 4;
      mode[0] = col < g.n ? 1 : 0;
      mode[1] = 0;
    }
    const uint32_t zero[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < G::kDepth; ++k) {
      if constexpr (FMT == MS_U8) {
        st_shared_chunk<16>(dst + k * G::kSlot, zero);
        st_shared_chunk<16>(dst + k * G::kSlot + 512, zero);
      } else {
        st_shared_chunk<4>(dst + k * G::kSlot, zero);
      }
    }
  }

  // window row `row` into `slot`, then advance
  __device__ __forceinline__ void issue(int slot) {
    const bool ok = (unsigned)row < (unsigned)nrows;
    const uint32_t d = dst + slot * G::kSlot;
    if constexpr (FMT == MS_U8) {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const uint8_t* p = ptr + 512 * k;
        if constexpr (RAGGED) {
          const int md = mode[k];
          if (md & 32) fill_chunk(d + 512 * k, p, ok ? md - 32 : 0);
          else if (md) cp_async(d + 512 * k, ok ? p : safe, 16, ok ? md : 0);
        } else {
          if (mode[k] == 1) cp_async(d + 512 * k, ok ? p : safe, 16, ok ? 16 : 0);
          else if (mode[k] == 2) fill_chunk(d + 512 * k, p, ok ? nvalid[k] : 0);
        }
      }
    } else {
      if (mode[0]) cp_async(d, ok ? ptr : safe, 4, ok ? 4 : 0);
    }
    ptr += stride;
    ++row;
  }
};

__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
__device__ __forceinline__ uint32_t mad_hi(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

// 32 cells given as 0/1 bytes (r[k] = columns 4k..4k+3, byte i = column
// 4k+i) into one word (bit b = column b).  Per 8 columns: q = r[2m] +
// 16 r[2m+1] holds column 8m+i in bit 8i and column 8m+4+i in bit 8i+4;
// times 0x00204081 (= 2^21 + 2^14 + 2^7 + 1) the product's bits 21..28 are
// columns 8m..8m+7 in order (every partial product lands on its own bit, so
// nothing carries), and a high or low multiply-add moves them to bit 8m.
// The multiplies issue on the FMA pipe.
__device__ __forceinline__ uint32_t pack01(const uint32_t r[8]) {
  uint32_t out = 0u;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const uint32_t q = mad_lo(r[2 * m + 1], 16u, r[2 * m]);
    const uint32_t y = imul(q, 0x00204081u) & 0x1FE00000u;
    out = m < 3 ? mad_hi(y, 1u << (8 * m + 11), out) : mad_lo(y, 8u, out);
  }
  return out;
}

// Shared-memory word address of ring row `slot` of level 2^p (its rows start
// at row 2^p - 1), lane word `w` (w = lane + 1 for the lane's own word, lane
// for its left neighbour's).
__device__ __forceinline__ uint32_t ring_at(uint32_t ring, int p, int slot, int w) {
  return ring + 4u * (uint32_t)((((1 << p) - 2) + slot) * kRowWords + w);
}
__device__ __forceinline__ uint32_t lds(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// The lane's word of S_t on window row ir (t <= 33): U(ir) & U(ir - s) from
// ring level P = 2^p <= t, s = t - P (rows above the window read as zeros:
// their ring slots are not yet written).
__device__ __forceinline__ uint32_t level_word(uint32_t ring, int lane, int ir, int t,
                                               uint32_t s1) {
  if (t == 1) return s1;  // S_1 of the row: the lane's own word
  const int p = 31 - __clz(t);
  const int P = 1 << p, s = t - P;
  const int k0 = ir & (ring_depth(p) - 1), k1 = (ir - s) & (ring_depth(p) - 1);
  const uint32_t a0 = lds(ring_at(ring, p, k0, lane));
  const uint32_t l0 = lane ? lds(ring_at(ring, p, k0, lane - 1)) : 0u;
  const uint32_t a1 = lds(ring_at(ring, p, k1, lane));
  const uint32_t l1 = lane ? lds(ring_at(ring, p, k1, lane - 1)) : 0u;
  return a0 & __funnelshift_l(l0, a0, s) & a1 & __funnelshift_l(l1, a1, s);
}

struct TileOut {
  unsigned long long key;  // (K, first K-corner) key, 0 if the tile holds no one
  int r0, r1, c0, c1;      // box of the cells of S_33 (r1 <= r0: none)
  bool redo;               // B01 pass saw a byte above 1
};

// One tile by one warp.  B01 (bytes only): the bytes are taken to be 0 or 1;
// `redo` reports that some byte was not, and the tile must run again.
// plane33 (or null): where the rows of S_33 go from the tile's first S_33
// row on (row stride pw words).
template <int FMT, bool B01, bool RAGGED>
__device__ __forceinline__ TileOut run_tile(const Tile& g, uint32_t in_ring, uint32_t ring,
                                            uint32_t* plane33, int64_t pw) {
  using G = InGeom<FMT>;
  const int lane = threadIdx.x & 31;
  // rows above the window are zeros: clear the level rings
  for (int k = lane; k < kRingWords; k += 32) sts(ring + 4u * k, 0u);
  Reader<FMT, RAGGED> rd;
  rd.init(g, lane, in_ring);
#pragma unroll
  for (int d = 0; d < G::kDepth; ++d) {
    rd.issue(d);
    cp_async_commit();
  }
  const int64_t col = g.wc0 + 32 * (int64_t)lane;
  const LaneCols lc = lane_cols<32>(col, g.n);
  // counted columns of this lane (the halo word of a later strip counts none)
  const uint32_t cm = col >= g.c0 ? lc.mask : 0u;
  const uint32_t lm = lane == 0 ? 0u : 0xffffffffu;  // lane 0's left is outside
  const uint32_t hoff = (lane & 4) ? 16u : 0u;
  const uint32_t hsel = (lane & 4) ? 0x1032u : 0x3210u;
  uint32_t seen = 0u;
  // G_a(r) = S_a(r) & S_a(r, c - a) of the last a rows for a = 1, 2, 4 (the
  // deeper levels read their rows above from the rings)
  uint32_t g1 = 0u, g2[2] = {0u, 0u}, g4[4] = {0u, 0u, 0u, 0u};
  int K = 0;
  TileOut o{0ull, 0x7fffffff, -1, 0x7fffffff, -1, false};
  __syncwarp();

  // rows go in groups of 4 (the last group runs past the window on the
  // reader's zero rows, untested), so that every ring slot of the levels 1,
  // 2, 4 and 32, and every slot inside a group's block of the levels 8 and
  // 16, is a fixed offset
  const uint32_t own = ring + 4u * (uint32_t)lane;  // the lane's word of ring row 0
  const int ngroups = (g.nrows + 3) >> 2;
#pragma unroll 1
  for (int gi = 0; gi < ngroups; ++gi) {
    const int ir0 = gi << 2;
    const uint32_t r8 = own + 4u * (uint32_t)((6 + (ir0 & 4)) * kRowWords);
    const uint32_t r16 = own + 4u * (uint32_t)((14 + (ir0 & 12)) * kRowWords);
    const uint32_t r32 = own + 4u * (uint32_t)(30 * kRowWords);
    const int dbase = G::kDepth > 4 ? (ir0 & (G::kDepth - 1)) : 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int ir = ir0 + j;
      const int d = (dbase + j) & (G::kDepth - 1);
      cp_async_wait<G::kDepth - 1>();
      uint32_t x;
      if constexpr (FMT == MS_U8) {
        // the lane's 32 bytes (chunks 2l and 2l+1); lanes with bit 2 set read
        // their second 16 bytes first, so that each 16-byte read of the warp
        // meets every bank once per 8 lanes, and swap the packed halves back
        const uint32_t a = in_ring + d * G::kSlot + 32u * lane;
        uint32_t r[8];
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a + hoff) : "memory");
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]) : "r"(a + (16u - hoff))
                     : "memory");
        if constexpr (B01) {
          seen |= r[0] | r[1] | r[2] | r[3] | r[4] | r[5] | r[6] | r[7];
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) r[k] = (nonzero_msb(r[k]) >> 7) & 0x01010101u;
        }
        x = prmt(pack01(r), 0u, hsel);
      } else {
        x = lds(in_ring + d * G::kSlot + 4u * lane) & lc.mask;
      }
      // the slot just read receives the row kDepth ahead
      rd.issue(d);
      cp_async_commit();

      // ring slot of this row for level 2^p (as a byte offset from `own`)
      auto slot = [&](int p) -> uint32_t {
        return p == 3 ? r8 + 4u * (uint32_t)(j * kRowWords)
             : p == 4 ? r16 + 4u * (uint32_t)(j * kRowWords)
             : p == 5 ? r32 + 4u * (uint32_t)((j & 1) * kRowWords)
                      : own + 4u * (uint32_t)((((1 << p) - 2) + (j & ((1 << p) - 1))) * kRowWords);
      };
      // doubling: S_2a(ir) = G_a(ir) & G_a(ir - a)
      uint32_t lv[6], lf[5];  // levels 1..32 of the lane's word; levels 1..16 of its left neighbour's
      lv[0] = x;
#pragma unroll
      for (int p = 0; p < 5; ++p) {
        const int A = 1 << p;
        const uint32_t cur = lv[p];
        const uint32_t left = __shfl_up_sync(kFull, cur, 1) & lm;
        lf[p] = left;
        const uint32_t gc = cur & __funnelshift_l(left, cur, A);
        if (p == 0) {
          lv[1] = gc & g1;
          g1 = gc;
        } else if (p == 1) {
          lv[2] = gc & g2[j & 1];
          g2[j & 1] = gc;
        } else if (p == 2) {
          lv[3] = gc & g4[j & 3];
          g4[j & 3] = gc;
        } else {
          const uint32_t o0 = lds(slot(p)), ol = lane ? lds(slot(p) - 4u) : 0u;
          lv[p + 1] = gc & o0 & __funnelshift_l(ol, o0, A);
        }
      }
      __syncwarp();  // every lane has read the slots about to be overwritten
      // levels 2 and 4 serve only tests of S_t with t < 8: once K >= 7 they
      // are never read again
      if (K < 7) {
        sts(slot(1), lv[1]);
        sts(slot(2), lv[2]);
      }
#pragma unroll
      for (int p = 3; p < 6; ++p) sts(slot(p), lv[p]);
      __syncwarp();  // the row's levels are visible to the whole warp

      if (ir >= g.cnt_ir0 && ir < g.nrows) {
        if (K < kTop) {
          // S_{K+1} = U(ir) & U(ir - s) with U = S_P & S_P(c - s), P the
          // level below K+1: a row whose U(ir) is empty holds no
          // (K+1)-corner (U(ir) from the row's registers; level 32 has no
          // neighbour word here and always takes the full test)
          const int t = K + 1, p = 31 - __clz(t), sh = t - (1 << p);
          uint32_t sp = 0u, sl = 0u;
          switch (p) {
            case 0: sp = lv[0]; sl = lf[0]; break;
            case 1: sp = lv[1]; sl = lf[1]; break;
            case 2: sp = lv[2]; sl = lf[2]; break;
            case 3: sp = lv[3]; sl = lf[3]; break;
            case 4: sp = lv[4]; sl = lf[4]; break;
            default: sp = 0xffffffffu; sl = 0xffffffffu; break;
          }
          if (__any_sync(kFull, (sp & __funnelshift_l(sl, sp, sh) & cm) != 0u)) {
            while (K < kTop) {
              const uint32_t w = level_word(ring, lane, ir, K + 1, lv[0]) & cm;
              const unsigned b = __ballot_sync(kFull, w != 0u);
              if (!b) break;
              ++K;
              const int L = __ffs(b) - 1;
              const uint32_t wl = __shfl_sync(kFull, w, L);
              const int64_t c = g.wc0 + 32 * (int64_t)L + (__ffs(wl) - 1);
              o.key = make_key(K, g.wr0 + ir, c, g.n);
            }
          }
        }
        if (K >= kTop) {
          const uint32_t w = level_word(ring, lane, ir, kTop, lv[0]) & cm;
          if (plane33 && cm) st_keep_l2(plane33 + (g.wr0 + ir) * pw + (g.wc0 >> 5) + lane, w);
          const unsigned b = __ballot_sync(kFull, w != 0u);
          if (b) {
            const int L0 = __ffs(b) - 1, L1 = 31 - __clz(b);
            if (o.r0 == 0x7fffffff) o.r0 = (int)(g.wr0 + ir);
            o.r1 = (int)(g.wr0 + ir + 1);
            o.c0 = min(o.c0, (int)(g.wc0 + 32 * L0));
            o.c1 = max(o.c1, (int)min(g.wc0 + 32 * (int64_t)(L1 + 1), g.n));
          }
        }
      }
    }
  }
  cp_async_wait<0>();
  if constexpr (B01 && FMT == MS_U8) o.redo = __any_sync(kFull, (seen & 0xfefefefeu) != 0u);
  __syncwarp();
  return o;
}

// One tile (number t of job j) by the calling warp, in its 8 KB of the
// block's dynamic shared memory; publishes the tile's key and box.  RAGGED
// false: only for matrices whose aligned rows end on a whole 16-byte chunk.
template <int FMT, bool RAGGED = true>
__device__ __forceinline__ void tile_one(const Job& j, int64_t t) {
  extern __shared__ __align__(16) unsigned char ms_dyn_smem[];
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(ms_dyn_smem) +
                        (threadIdx.x >> 5) * (uint32_t)kWarpBytes;
  const uint32_t in_ring = base, ring = base + kInBytes;
  const Tile g = tile_of(j, t);
  const int64_t pw = (j.n + 31) / 32;
  uint32_t* plane33 = j.first33 ? j.bits_scratch + 2 * j.m * (pw + 2) : nullptr;
  TileOut o;
  if constexpr (FMT == MS_U8) {
    o = run_tile<FMT, true, RAGGED>(g, in_ring, ring, plane33, pw);
    if (o.redo) o = run_tile<FMT, false, RAGGED>(g, in_ring, ring, plane33, pw);
  } else {
    o = run_tile<FMT, false, false>(g, in_ring, ring, plane33, pw);
  }
  if ((threadIdx.x & 31) == 0) {
    if (j.first33) j.first33[t] = o.r1 >= 0 ? o.r0 : 0x7fffffff;
    if (o.key) atomicMax(&j.st->key, o.key);
    if (o.r1 >= 0) {
      atomicMin(&j.st->box[0], o.r0);
      atomicMax(&j.st->box[1], o.r1);
      atomicMin(&j.st->box[2], o.c0);
      atomicMax(&j.st->box[3], o.c1);
    }
  }
}

}  // namespace bt

// Size-only tile pass of one matrix by bitplanes (tile geometry of lane width
// 32); FUSE: the last block also runs the bitplane fix-up of the box and
// writes the result, from its own shared memory when the box fits (small
// matrices; the large ones take the variant without that code, whose tile
// loop then keeps every register to itself).  RAGGED: the rows of an aligned
// byte matrix end in a partial 16-byte chunk (copied asynchronously with a
// partial source size); without it the copies' size is a constant.
template <int FMT, bool FUSE, bool RAGGED>
__global__ void __launch_bounds__(256, 3) k_bitiles_one(const Job job, int64_t ntiles,
                                                         TeamSync* team) {
  grid_dependents_may_launch();
  clear_team(team);
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w < ntiles) bt::tile_one<FMT, RAGGED>(job, w);
  if constexpr (FUSE) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // this block's key and box updates before its ticket
      s_last = atomicAdd(&job.st->done, 1) == (int)gridDim.x - 1;
      if (s_last) __threadfence();
    }
    __syncthreads();
    if (s_last) {
      extern __shared__ __align__(16) unsigned char ms_dyn_smem[];
      fixup_bits_job<FMT>(job, reinterpret_cast<uint32_t*>(ms_dyn_smem),
                          (int64_t)(blockDim.x >> 5) * bt::kWarpBytes / 4, 1, 0, nullptr);
    }
  }
}

// ---- batch: bitplane tiles of many matrices, one persistent launch ---------
//
// Warps take tiles (task.job_a, task.tile_a) of one input format from the
// queue, longest first; three blocks of eight warps per SM, as for a single
// large matrix.
template <int FMT>
__global__ void __launch_bounds__(256, 3) k_batch_bitiles(const Job* __restrict__ jobs,
                                                          const PairTask* __restrict__ tasks,
                                                          int ntasks, int* queue) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(queue, 1);
    t = __shfl_sync(kFull, t, 0);
    if (t >= ntasks) break;
    const PairTask task = tasks[t];
    bt::tile_one<FMT>(jobs[task.job_a], task.tile_a);
  }
}

// ---- batch: one persistent launch over a queue of tasks -------------------
//
// Warps take tasks from an atomic queue until it runs dry: tile pairs of one
// format and lane width (the dp recurrence, at most 16 columns per lane) or
// single bitplane tiles (lane width 32, tile_b unused), groups contiguous and
// longest first.  Both kinds use 8 KB of shared memory per warp.
static __global__ void __launch_bounds__(256, 2) k_batch_tiles(const Job* __restrict__ jobs,
                                                        const PairTask* __restrict__ tasks,
                                                        int ntasks, int* queue) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(queue, 1);
    t = __shfl_sync(kFull, t, 0);
    if (t >= ntasks) break;
    const PairTask task = tasks[t];
    const Job& A = jobs[task.job_a];
    const int key = A.fmt * 64 + A.P;
    switch (key) {
      case MS_U8 * 64 + 1: batch_task<1, MS_U8>(jobs, task); break;
      case MS_U8 * 64 + 2: batch_task<2, MS_U8>(jobs, task); break;
      case MS_U8 * 64 + 4: batch_task<4, MS_U8>(jobs, task); break;
      case MS_U8 * 64 + 8: batch_task<8, MS_U8>(jobs, task); break;
      case MS_U8 * 64 + 16: batch_task<16, MS_U8>(jobs, task); break;
      case MS_U8 * 64 + 32: bt::tile_one<MS_U8>(A, task.tile_a); break;
      case MS_BITS32 * 64 + 1: batch_task<1, MS_BITS32>(jobs, task); break;
      case MS_BITS32 * 64 + 2: batch_task<2, MS_BITS32>(jobs, task); break;
      case MS_BITS32 * 64 + 4: batch_task<4, MS_BITS32>(jobs, task); break;
      case MS_BITS32 * 64 + 8: batch_task<8, MS_BITS32>(jobs, task); break;
      case MS_BITS32 * 64 + 32: bt::tile_one<MS_BITS32>(A, task.tile_a); break;
      default: batch_task<16, MS_BITS32>(jobs, task); break;
    }
  }
}

}  // namespace ms
