// Kernels of libms: the tile pass, the exact fix-up of unresolved regions
// and the result write-out.  See ms_device.cuh for the recurrence.
//
// Tile pass.  A matrix is cut into tiles of `band_rows` counted rows and
// 32*P counted columns.  A warp computes two tiles at once (one per 16-bit
// half of every register).  Each tile is computed on a window that also
// covers kHalo rows above and kHalo columns to its left, started from zero
// carries (as if the window's outside were zeros).  Inside such a window the
// recurrence yields dp_w = min(dp, rows into the window, columns into the
// window), so every counted cell is exact as soon as the tile's largest dp_w
// is at most the halo.  Cells whose value exceeds the halo are "flagged"
// and their bounding box (rows exact, columns rounded out to a lane's chunk)
// is recorded per matrix.  Cells on the matrix's top or left edge are exact
// whatever their values, but they are flagged all the same: the fix-up below
// relies on every unflagged cell having dp <= halo.
//
// Lanes are skewed by one row: at step s lane l works on window row s - l,
// so what lane l needs from lane l-1 (A of lane l-1's last column on this row
// and on the row above) was produced one step earlier and is passed with two
// shuffles; nothing waits inside a step.
//
// Fix-up.  If a matrix has flagged cells, their box [rlo, rhi) x [clo, chi)
// grown by the halo up and left is recomputed exactly as one window: its
// columns are split into strips of kFixW, one warp per strip, and each strip
// takes the exact A of its left neighbour's last column row by row through
// global memory (release/acquire flags, bounded waits).  A square whose
// corner lies in the box and which reached above the grown window would
// contain a square of side > halo ending on the row just above rlo, and that
// cell, whose window value is at least min(dp, halo + 1), would then be
// flagged too (likewise on the left); so every cell of the box is exact.
#pragma once
#include "ms_device.cuh"

namespace ms {

struct Tile {
  const uint8_t* base;
  int64_t ld, m, n;
  int64_t wr0;      // first absolute row of the window
  int32_t nrows;    // rows in the window
  int32_t cnt_ir0;  // first counted row, relative to the window
  int64_t wc0;      // first absolute column of the window
  int64_t c0;       // first counted column
  int32_t aligned;
};

// Geometry of tile `t` of job `j` in the tile pass.
__device__ __forceinline__ Tile tile_of(const Job& j, int64_t t) {
  Tile g;
  const int W = 32 * j.P;
  const int band = (int)(t / j.strips);
  const int strip = (int)(t - (int64_t)band * j.strips);
  g.base = reinterpret_cast<const uint8_t*>(j.data);
  g.ld = j.ld;
  g.m = j.m;
  g.n = j.n;
  const int64_t r0 = (int64_t)band * j.band_rows;
  const int64_t r1 = min(j.m, r0 + j.band_rows);
  g.wr0 = r0 >= kHalo ? r0 - kHalo : 0;  // (bands under kHalo rows: the window starts at row 0)
  g.nrows = (int32_t)(r1 - g.wr0);
  g.cnt_ir0 = (int32_t)(r0 - g.wr0);
  if (strip == 0) {
    g.wc0 = 0;
    g.c0 = 0;
  } else {
    g.c0 = W + (int64_t)(strip - 1) * (W - kHalo);
    g.wc0 = g.c0 - kHalo;
  }
  g.aligned = j.aligned;
  return g;
}

__device__ __forceinline__ Tile empty_tile() {
  Tile g;
  g.base = nullptr;
  g.ld = g.m = g.n = 0;
  g.wr0 = 0;
  g.nrows = 0;
  g.cnt_ir0 = 0;
  g.wc0 = 0;
  g.c0 = 0;
  g.aligned = 0;
  return g;
}

// ---- input staging ---------------------------------------------------------
// Each warp owns a ring of slots in shared memory (kRingWarpBytes); a slot
// holds one row step of both tiles: [tile][lane][kLane bytes].  Lane l copies
// its own column chunk of window row (s - l + depth) into the slot it
// consumes at step s with cp.async (no registers held while the copy is in
// flight), so loads run `depth` steps ahead of use; a ragged last chunk is
// copied with a partial source size, the rest of its slot zero-filled.
// Chunks of unaligned rows, and chunks of fewer than 4 bytes at the edge, are
// loaded synchronously into the same slot.  32-byte chunks (uint8, P = 32) get half as many, twice as large
// slots.
constexpr int kRingWarpBytes = 8192;

template <int P, int FMT>
struct RingGeom {
  // bytes per lane and tile in a slot (16, or 32 for 32-byte chunks; deeper
  // rings for narrow chunks measured no faster)
  static constexpr int kLane = (FMT == MS_U8 && P > 16) ? 32 : 16;
  static constexpr int kSlot = 2 * 32 * kLane;
  static constexpr int kDepth = kRingWarpBytes / kSlot;
  static_assert((kDepth & (kDepth - 1)) == 0 && kDepth >= 2, "ring depth: a power of two");
};

// Zero (or write w[]) the kLane bytes at shared address a.
template <int kLane>
__device__ __forceinline__ void st_shared_chunk(uint32_t a, const uint32_t* w) {
  if constexpr (kLane == 4) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(w[0]) : "memory");
  } else if constexpr (kLane == 8) {
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(a), "r"(w[0]), "r"(w[1]) : "memory");
  } else {
#pragma unroll
    for (int h = 0; h < kLane / 4; h += 4)
      asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a + 4 * h), "r"(w[h]),
                   "r"(w[h + 1]), "r"(w[h + 2]), "r"(w[h + 3]) : "memory");
  }
}

__device__ __forceinline__ void cp_async(uint32_t dst, const void* src, int bytes_copy,
                                         int bytes_src) {
  if (bytes_copy == 16)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(bytes_src) : "memory");
  else if (bytes_copy == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src),
                 "r"(bytes_src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src),
                 "r"(bytes_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Streams one lane's column chunk of a tile down the window into its ring.
template <int P, int FMT>
struct AsyncReader {
  using G = RingGeom<P, FMT>;
  static constexpr int kBytes = FMT == MS_U8 ? P : 4;  // chunk bytes
  const uint8_t* ptr;   // chunk of window row `row`
  const uint8_t* safe;  // a valid address (zero-fill copies read nothing)
  int64_t stride;
  int row, nrows;
  // 0: no cells (slots stay zero); 1..kBytes: an async copy reading that many
  // bytes of the chunk (the rest zero-filled); 64 + v: v bytes by synchronous
  // byte loads
  int mode;
  uint32_t dst;         // this lane's place in slot 0
  uint32_t lshift;      // chunks under 4 bytes: bit offset of the chunk in its copied word

  __device__ __forceinline__ void init(const Tile& g, int lane, int first_row, uint32_t ring,
                                       int half) {
    const int64_t col = g.wc0 + (int64_t)P * lane;
    row = first_row;
    nrows = g.nrows;
    dst = ring + half * (32 * G::kLane) + lane * G::kLane;
    safe = g.base;
    lshift = 0;
    if constexpr (FMT == MS_U8) {
      stride = g.ld;
      const int64_t valid = g.n - col;
      const int nvalid = (int)(valid < P ? (valid < 0 ? 0 : valid) : P);
      if constexpr (P >= 4) {
        // (a ragged last chunk of an aligned matrix is copied asynchronously
        // too: the copy reads its valid bytes and zero-fills the rest)
        ptr = g.base + (g.wr0 + first_row) * g.ld + col;
        mode = nvalid == 0 ? 0 : g.aligned ? nvalid : 64 + nvalid;
      } else {
        // 1- and 2-byte chunks are fetched as the aligned 4-byte word holding
        // them (asynchronously, like the wider chunks), unless that word
        // reaches past the row's last column
        const int64_t col4 = col & ~(int64_t)3;
        const bool word_ok = g.aligned && col4 + 4 <= g.n;
        ptr = g.base + (g.wr0 + first_row) * g.ld + (word_ok ? col4 : col);
        lshift = word_ok ? (uint32_t)(8 * (col - col4)) : 0u;
        mode = nvalid == 0 ? 0 : (nvalid == P && word_ok) ? 4 : 64 + nvalid;
      }
    } else {
      stride = g.ld * 4;
      ptr = g.base + ((g.wr0 + first_row) * g.ld + (col >> 5)) * 4;
      mode = col < g.n ? 4 : 0;
    }
    // slots start as zeros: mode 0 never writes, the others overwrite
    uint32_t zero[G::kLane / 4];
#pragma unroll
    for (int b = 0; b < G::kLane / 4; ++b) zero[b] = 0u;
#pragma unroll
    for (int k = 0; k < G::kDepth; ++k) st_shared_chunk<G::kLane>(dst + k * G::kSlot, zero);
  }

  // copy window row `row` into `slot` and advance
  __device__ __forceinline__ void issue(int slot) {
    const bool ok = (unsigned)row < (unsigned)nrows;
    const uint32_t d = dst + slot * G::kSlot;
    const int md = mode;
    if (md & 64) {
      constexpr int NW = G::kLane / 4;
      uint32_t w[NW];
#pragma unroll
      for (int b = 0; b < NW; ++b) w[b] = 0u;
      if (ok)
        for (int b = 0; b < md - 64; ++b) w[b >> 2] |= (uint32_t)__ldg(ptr + b) << (8 * (b & 3));
      st_shared_chunk<G::kLane>(d, w);
    } else if (md) {
      const uint8_t* src = ok ? ptr : safe;
      if constexpr (kBytes > 16) {
        const int v0 = ok ? min(md, 16) : 0, v1 = ok ? max(md - 16, 0) : 0;
        cp_async(d, src, 16, v0);
        cp_async(d + 16, v1 ? src + 16 : safe, 16, v1);
      } else if constexpr (kBytes < 4) {
        cp_async(d, src, 4, ok ? 4 : 0);
      } else {
        cp_async(d, src, kBytes, ok ? md : 0);
      }
    }
    ptr += stride;
    ++row;
  }

  __device__ __forceinline__ void read(int slot, Raw<P, FMT>& r) const {
    const uint32_t a = dst + slot * G::kSlot;
    if constexpr (FMT == MS_U8) {
      if constexpr (Raw<P, MS_U8>::W == 8) {
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3])
                     : "r"(a) : "memory");
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r.w[4]), "=r"(r.w[5]), "=r"(r.w[6]), "=r"(r.w[7])
                     : "r"(a + 16) : "memory");
      } else if constexpr (Raw<P, MS_U8>::W == 4) {
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3])
                     : "r"(a) : "memory");
      } else if constexpr (Raw<P, MS_U8>::W == 2) {
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r.w[0]), "=r"(r.w[1]) : "r"(a)
                     : "memory");
      } else {
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(r.w[0]) : "r"(a) : "memory");
        if constexpr (P < 4) r.w[0] >>= lshift;
      }
    } else {
      asm volatile("ld.shared.u32 %0, [%1];" : "=r"(r.word) : "r"(a) : "memory");
    }
  }
};

// This warp's ring in the block's dynamic shared memory (warps x kRingWarpBytes).
__device__ __forceinline__ uint32_t warp_ring() {
  extern __shared__ __align__(16) unsigned char ms_dyn_smem[];
  return (uint32_t)__cvta_generic_to_shared(ms_dyn_smem) + (threadIdx.x >> 5) * kRingWarpBytes;
}

// Left-edge carries of a strip in the fix-up (mode 1): A of the left
// strip's last column per window row (16 bits), published 8 rows at a time.
struct StripIO {
  const uint16_t* carry_in;   // null for the first strip (zero boundary); 16-B aligned
  const int32_t* progress_in;
  uint16_t* carry_out;        // null for the last strip
  int32_t* progress_out;
  int32_t* status;
  int32_t hold;               // test hook: never publish (the neighbour's wait must time out)
};

// Writes one lane's dp values of one row (half `hi` of the packed A values).
template <int P, bool HI>
__device__ __forceinline__ void store_dp(int32_t* p, const uint32_t* Ap, uint32_t I, int64_t col,
                                         int64_t n, int aligned) {
  auto val = [&](int k) -> int {
    return (int)I - (int)(HI ? (Ap[k] >> 16) : (Ap[k] & 0xffffu));
  };
  if (aligned == 2 && col + P <= n && (P % 8) == 0) {
    // whole 32-byte sectors per lane: no sector is shared between stores
#pragma unroll
    for (int k = 0; k < P; k += 8)
      asm volatile("st.global.cs.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p + k),
                   "r"(val(k)), "r"(val(k + 1)), "r"(val(k + 2)), "r"(val(k + 3)),
                   "r"(val(k + 4)), "r"(val(k + 5)), "r"(val(k + 6)), "r"(val(k + 7))
                   : "memory");
  } else if (aligned && col + P <= n && (P % 4) == 0) {
#pragma unroll
    for (int k = 0; k < P; k += 4) {
      int4 v;
      v.x = val(k);
      v.y = val(k + 1);
      v.z = val(k + 2);
      v.w = val(k + 3);
      __stcs(reinterpret_cast<int4*>(p + k), v);
    }
  } else {
#pragma unroll
    for (int k = 0; k < P; ++k)
      if (col + k < n) p[k] = val(k);
  }
}

// Two independent tiles (low and high 16-bit halves), lanes skewed by a row.
// Mode 0: tile pass (zero carries on the window edges).  Mode 1: a fix-up
// strip taking its left carries from `io` and publishing its right ones.
//
// EMIT (second pass of the all-largest-squares call, largest side emitK <=
// kHalo known): every counted cell with dp == emitK is appended to ej's list.
//
// B01 (uint8 tile pass): the bytes are taken to be 0 or 1 (cheaper cell
// extraction); returns false if some byte of the tiles was larger, in which
// case the caller computes the tiles again without the assumption.
template <int P, int FMT, bool DPMAP, int MODE, bool EMIT = false, bool B01 = false>
__device__ __forceinline__ bool run_tiles(const Tile& ta, const Tile& tb, int32_t* dpa,
                                          int64_t lda, int dpa_al, int32_t* dpb, int64_t ldb,
                                          int dpb_al, const StripIO& io, Best& ba, Best& bb,
                                          uint32_t ring, const Job* ej = nullptr,
                                          uint32_t emitK = 0) {
  static_assert(!B01 || FMT == MS_U8, "the 0/1 shortcut is for bytes");
  uint32_t seen = 0;  // B01: OR of every raw input word
  const int lane = threadIdx.x & 31;
  constexpr uint32_t kB2 = kBias * 0x10001u;
  // size-only tile pass on cells known to be 0/1: dp units in fp16 (hfma2)
  constexpr bool H = MODE == 0 && !DPMAP && !EMIT && (B01 || FMT == MS_BITS32);
  constexpr uint32_t kInit = H ? 0u : kB2;  // the value above / left of the window
  constexpr uint32_t kHaloCmp2 = H ? kHaloH2 : (uint32_t)kHalo * 0x10001u;
  constexpr int D = RingGeom<P, FMT>::kDepth;  // rows of input in flight per lane
  const int nmax = max(ta.nrows, tb.nrows);
  const int nsteps = nmax + 31;

  uint32_t Ap[P];  // A of the lane's columns on the last row computed
#pragma unroll
  for (int k = 0; k < P; ++k) Ap[k] = kInit;
  uint32_t pubL = kInit, pubD = kInit;  // A of the lane's last column: this row, the row above
  uint32_t carryA_prev = kBias;  // fix-up: A of the left strip's last column, previous row
  uint4 cq = make_uint4(0u, 0u, 0u, 0u);  // fix-up: the next carries, 16 bits per row
  bool gave_up = false;
  ba.val = bb.val = 0;
  ba.row = ba.col = bb.row = bb.col = -1;
  ba.big_r0 = bb.big_r0 = 0x7fffffff;
  ba.big_r1 = bb.big_r1 = -1;
  ba.big_c0 = bb.big_c0 = 0x7fffffffffffffffll;
  ba.big_c1 = bb.big_c1 = -1;
  uint32_t best2 = 0;  // best dp per half so far (packed)
  const int64_t cola = ta.wc0 + (int64_t)P * lane;
  const int64_t colb = tb.wc0 + (int64_t)P * lane;
  // a lane chunk counts when it reaches a counted column: in the fix-up the
  // box edge need not fall on a chunk edge, and the chunk's cells left of it
  // are exact too (the window starts at least kHalo columns further left)
  const uint32_t colmask2 = ((cola + P > ta.c0 && cola < ta.n) ? 0x0000ffffu : 0u) |
                            ((colb + P > tb.c0 && colb < tb.n) ? 0xffff0000u : 0u);
  const LaneCols lca = lane_cols<P>(cola, ta.n);
  const LaneCols lcb = lane_cols<P>(colb, tb.n);
  int32_t* dprow_a = DPMAP && dpa ? dpa + ta.wr0 * lda + cola : nullptr;
  int32_t* dprow_b = DPMAP && dpb ? dpb + tb.wr0 * ldb + colb : nullptr;

  AsyncReader<P, FMT> rda, rdb;
  rda.init(ta, lane, -lane, ring, 0);
  rdb.init(tb, lane, -lane, ring, 1);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    rda.issue(d);
    rdb.issue(d);
    cp_async_commit();
  }

  // one step per iteration, not unrolled: the ring slot is a shared-memory
  // address computed at run time, and a rolled loop keeps the kernel small
  // enough for the instruction cache
#pragma unroll 1
  for (int s = 0; s < nsteps; ++s) {
    {
      const int d = s & (D - 1);
      const int ir = s - lane;
      // A of the left neighbour's last column on this row and the row above
      // (lane l-1 produced both one step earlier, on the same window row)
      uint32_t al = __shfl_up_sync(kFull, pubL, 1);
      uint32_t ad = __shfl_up_sync(kFull, pubD, 1);
      cp_async_wait<D - 1>();
      Raw<P, FMT> rlo, rhi;
      rda.read(d, rlo);
      rdb.read(d, rhi);
      Cells<P, FMT> clo, chi;
      if constexpr (B01 && H) {
        clo = cells_h01<P>(rlo, seen);
        chi = cells_h01<P>(rhi, seen);
      } else if constexpr (B01) {
        clo = cells_of01<P>(rlo, seen);
        chi = cells_of01<P>(rhi, seen);
      } else {
        clo = cells_of<P>(rlo, lca);
        chi = cells_of<P>(rhi, lcb);
      }
      if ((unsigned)ir < (unsigned)nmax) {
        const uint32_t I = (uint32_t)ir + 1u + kBias;
        const uint32_t I2 = I * 0x10001u;
        if (lane == 0) {
          // left window edge: a zero column (dp = 0, so A = I on this row and
          // I - 1 on the row above)
          al = H ? 0u : I2;
          ad = H ? 0u : I2 - 0x10001u;
          if constexpr (MODE == 1) {
            if (io.carry_in) {
              if ((ir & 7) == 0) {
                // the next 8 rows of carries: wait until the left strip has
                // published them (bounded), then one 16-byte load from L2
                const int need = min(ir + 8, ta.nrows);
                if (!gave_up) {
                  int spins = 0;
                  const unsigned long long t0 = global_ns();
                  while (ld_acquire(io.progress_in) < need) {
                    if (++spins > kSpinLimit || global_ns() - t0 > kWaitLimitNs) {
                      gave_up = true;
                      atomicExch(io.status, (int)MS_ERR_TIMEOUT);
                      break;
                    }
                    __nanosleep(64);
                  }
                }
                cq = __ldcg(reinterpret_cast<const uint4*>(io.carry_in + ir));
              }
              const uint32_t c = cq.x & 0xffffu;
              cq.x = __funnelshift_r(cq.x, cq.y, 16);
              cq.y = __funnelshift_r(cq.y, cq.z, 16);
              cq.z = __funnelshift_r(cq.z, cq.w, 16);
              cq.w >>= 16;
              al = (al & 0xffff0000u) | c;
              ad = (ad & 0xffff0000u) | carryA_prev;
              carryA_prev = c;
            }
          }
        }
        // dp = 1 + min(up, left, diagonal) on a one, 0 on a zero; in row
        // units A = I - dp this is A = max(A_up, A_diag, A_left - 1) on a one
        // and I on a zero.  Every A is at least kBias, so the packed
        // decrement by 0x00010001 never borrows across halves.  (Selecting I
        // before the last max would shorten the chain along the row to two
        // operations, but measured slower.)
        uint32_t rbest;  // H: the row's largest dp (fp16 bits), else its smallest A
        if constexpr (H) {
          uint32_t rmax = 0u;
          BitsH hb;
          if constexpr (FMT == MS_BITS32) hb = bits_h<P>(clo, chi);
#pragma unroll
          for (int k = 0; k < P; ++k) {
            uint32_t v;
            if constexpr (FMT == MS_BITS32) v = pair_one(hb, k);
            else v = pair_one<P>(clo, chi, k);
            const uint32_t up = Ap[k];
            const uint32_t mn = vmin2(vmin2(up, ad), al);
            ad = up;
            al = hfma2(v, mn, v);
            Ap[k] = al;
            rmax = vmax2(rmax, al);
          }
          rbest = rmax;
        } else {
          uint32_t rmin = 0xffffffffu;
#pragma unroll
          for (int k = 0; k < P; ++k) {
            const uint32_t msk = pair_mask<P>(clo, chi, k);
            const uint32_t up = Ap[k];
            const uint32_t t = vmax2(vmax2(up, ad), al - 0x00010001u);
            ad = up;
            al = select_bits(t, I2, msk);
            Ap[k] = al;
            rmin = vmin2(rmin, al);
          }
          rbest = rmin;
        }
        pubL = al;
        pubD = ad;  // A of this lane's last column, row above

        if constexpr (MODE == 1) {
          if (lane == 31 && io.carry_out) {
            io.carry_out[ir] = (uint16_t)al;
            // the release orders this lane's carry stores before the count
            if ((((ir + 1) & 7) == 0 || ir + 1 == ta.nrows) && !io.hold)
              st_release(io.progress_out, ir + 1);
          }
        }

        // this row's best dp per half (I >= A, so the packed subtraction is
        // exact), kept only for counted rows and columns; H: as fp16 bits,
        // which order like the values
        const uint32_t rowmask2 = (ir >= ta.cnt_ir0 ? 0x0000ffffu : 0u) |
                                  (ir >= tb.cnt_ir0 ? 0xffff0000u : 0u);
        const uint32_t d2 = (H ? rbest : I2 - rbest) & colmask2 & rowmask2;
        if (vmax2(d2, best2) != best2) {
          const uint32_t dlo = d2 & 0xffffu, dhi = d2 >> 16;
          if (dlo > (best2 & 0xffffu)) {
            ba.val = H ? h16_int(dlo) : (int)dlo;
            ba.row = (int32_t)(ta.wr0 + ir);
            const uint32_t target = H ? dlo : I - dlo;
            int kk = 0;
#pragma unroll
            for (int k = P - 1; k >= 0; --k)
              if ((Ap[k] & 0xffffu) == target) kk = k;
            ba.col = (int32_t)(cola + kk);
          }
          if (dhi > (best2 >> 16)) {
            bb.val = H ? h16_int(dhi) : (int)dhi;
            bb.row = (int32_t)(tb.wr0 + ir);
            const uint32_t target = H ? dhi : I - dhi;
            int kk = 0;
#pragma unroll
            for (int k = P - 1; k >= 0; --k)
              if ((Ap[k] >> 16) == target) kk = k;
            bb.col = (int32_t)(colb + kk);
          }
          best2 = vmax2(d2, best2);
        }
        if constexpr (EMIT) {
          const uint32_t km1 = (emitK - 1u) * 0x10001u;
          if (vmax2(d2, km1) != km1) {  // a counted cell of this row reaches emitK
            const bool elo = (d2 & 0xffffu) >= emitK, ehi = (d2 >> 16) >= emitK;
#pragma unroll
            for (int k = 0; k < P; ++k) {
              const uint32_t dk = I2 - Ap[k];
              if (elo && (dk & 0xffffu) == emitK) emit_corner(*ej, ta.wr0 + ir, cola + k);
              if (ehi && (dk >> 16) == emitK) emit_corner(*ej, tb.wr0 + ir, colb + k);
            }
          }
        }
        // rows and lane chunks holding a value above the halo: the fix-up box
        if (vmax2(d2, kHaloCmp2) != kHaloCmp2) {
          if ((d2 & 0xffffu) > (kHaloCmp2 & 0xffffu)) {
            if (ba.big_r0 == 0x7fffffff) {
              ba.big_r0 = (int32_t)(ta.wr0 + ir);
              ba.big_c0 = cola;
              ba.big_c1 = min(cola + P, ta.n);
            }
            ba.big_r1 = (int32_t)(ta.wr0 + ir + 1);
          }
          if ((d2 >> 16) > (kHaloCmp2 >> 16)) {
            if (bb.big_r0 == 0x7fffffff) {
              bb.big_r0 = (int32_t)(tb.wr0 + ir);
              bb.big_c0 = colb;
              bb.big_c1 = min(colb + P, tb.n);
            }
            bb.big_r1 = (int32_t)(tb.wr0 + ir + 1);
          }
        }

        if constexpr (DPMAP) {
          if ((colmask2 & 0xffffu) && ir >= ta.cnt_ir0 && ir < ta.nrows)
            store_dp<P, false>(dprow_a + (int64_t)ir * lda, Ap, I, cola, ta.n, dpa_al);
          if ((colmask2 >> 16) && ir >= tb.cnt_ir0 && ir < tb.nrows)
            store_dp<P, true>(dprow_b + (int64_t)ir * ldb, Ap, I, colb, tb.n, dpb_al);
        }
      }
      // the slot just consumed receives the row D steps ahead
      rda.issue(d);
      rdb.issue(d);
      cp_async_commit();
    }
  }
  cp_async_wait<0>();
  if constexpr (B01) return __any_sync(kFull, (seen & 0xfefefefeu) != 0u) == 0;
  return true;
}

// Reduce a per-lane best to the tile's key; returns the tile's largest value.
__device__ __forceinline__ unsigned long long tile_key(const Best& b, int64_t n) {
  return warp_max_u64(make_key(b.val, b.row, b.col, n));
}

// ---- programmatic dependent launch ------------------------------------------
// A tile kernel lets the fix-up after it be launched early (its blocks are
// placed as the tile blocks retire); the fix-up waits, before it reads
// anything, for the tile grid to finish and its writes to be visible.  Both
// are no-ops for launches without the programmatic attribute.
__device__ __forceinline__ void grid_dependents_may_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---- tile pass ------------------------------------------------------------

__device__ __forceinline__ int find_job(const Job* jobs, int njobs, int64_t t) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile0 <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One warp, two tiles: compute, then publish each tile's key and the box of
// its cells above the halo to its matrix's state.  jb < 0: no high tile.
template <int P, int FMT, bool DPMAP>
__device__ __forceinline__ void tile_pair(const Job& A, const Tile& ga, const Job& B,
                                          const Tile& gb, bool has_b) {
  StripIO io{nullptr, nullptr, nullptr, nullptr, nullptr, 0};
  Best ba, bb;
  bool done = false;
  if constexpr (FMT == MS_U8)  // most inputs hold only 0/1 bytes
    done = run_tiles<P, FMT, DPMAP, 0, false, true>(ga, gb, A.dp, A.ld_dp, A.dp_aligned, B.dp,
                                                    B.ld_dp, B.dp_aligned, io, ba, bb,
                                                    warp_ring());
  if (!done)
    run_tiles<P, FMT, DPMAP, 0>(ga, gb, A.dp, A.ld_dp, A.dp_aligned, B.dp, B.ld_dp, B.dp_aligned,
                                io, ba, bb, warp_ring());
  const unsigned long long ka = tile_key(ba, ga.n);
  const unsigned long long kb = tile_key(bb, gb.n);
  // the tile's cells above the halo: bounding box over the warp's lanes
  const int ar0 = __reduce_min_sync(kFull, ba.big_r0), ar1 = __reduce_max_sync(kFull, ba.big_r1);
  const int br0 = __reduce_min_sync(kFull, bb.big_r0), br1 = __reduce_max_sync(kFull, bb.big_r1);
  const int ac0 = __reduce_min_sync(kFull, (int)min(ba.big_c0, (int64_t)0x7fffffff));
  const int ac1 = __reduce_max_sync(kFull, (int)ba.big_c1);
  const int bc0 = __reduce_min_sync(kFull, (int)min(bb.big_c0, (int64_t)0x7fffffff));
  const int bc1 = __reduce_max_sync(kFull, (int)bb.big_c1);
  if ((threadIdx.x & 31) == 0) {
    if (ka) atomicMax(&A.st->key, ka);
    if (ar1 >= 0) {
      atomicMin(&A.st->box[0], ar0);
      atomicMax(&A.st->box[1], ar1);
      atomicMin(&A.st->box[2], ac0);
      atomicMax(&A.st->box[3], ac1);
    }
    if (has_b && kb) atomicMax(&B.st->key, kb);
    if (has_b && br1 >= 0) {
      atomicMin(&B.st->box[0], br0);
      atomicMax(&B.st->box[1], br1);
      atomicMin(&B.st->box[2], bc0);
      atomicMax(&B.st->box[3], bc1);
    }
  }
}

// Warp w of a single-matrix launch takes tiles 2w and 2w+1.
template <int P, int FMT, bool DPMAP>
__device__ __forceinline__ void tile_pass_warp(const Job* jobs, int njobs, int64_t ntiles,
                                               int64_t w) {
  const int64_t t_a = 2 * w, t_b = 2 * w + 1;
  if (t_a >= ntiles) return;
  const int ja = find_job(jobs, njobs, t_a);
  const Job& A = jobs[ja];
  const Tile ga = tile_of(A, t_a - A.tile0);
  int jb = -1;
  Tile gb = empty_tile();
  if (t_b < ntiles) {
    jb = find_job(jobs, njobs, t_b);
    gb = tile_of(jobs[jb], t_b - jobs[jb].tile0);
  }
  tile_pair<P, FMT, DPMAP>(A, ga, jobs[jb < 0 ? ja : jb], gb, jb >= 0);
}

// ---- batch: one persistent launch over a queue of tile pairs --------------

struct PairTask {
  int32_t job_a, job_b;  // job_b < 0: the high half is idle
  int32_t tile_a, tile_b;
};

template <int P, int FMT>
__device__ __forceinline__ void batch_task(const Job* jobs, const PairTask& t) {
  const Job& A = jobs[t.job_a];
  const bool has_b = t.job_b >= 0;
  const Job& B = jobs[has_b ? t.job_b : t.job_a];
  const Tile ga = tile_of(A, t.tile_a);
  const Tile gb = has_b ? tile_of(B, t.tile_b) : empty_tile();
  tile_pair<P, FMT, false>(A, ga, B, gb, has_b);
}

// ---- fix-up and result ------------------------------------------------------

constexpr int kFixWarps = 16;
constexpr int kFixP = 8;            // short per-row chains: the fix-up is latency-bound
constexpr int kFixW = 32 * kFixP;  // strip width in the fix-up

// ---- size-only fix-up by bitplane growth inside the box ------------------
//
// S_t = bottom-right corners of all-ones t-squares.  Every cell with dp >= 33
// has a window value above the halo and lies in the flagged box, so S_t for
// t >= 33 lies inside the box.  S_32 is exact everywhere; it is built from the
// input on the box grown by 32 up and left, then squares are grown inside the
// box: S_{a+b-1} = S_a & S_a(i-b+1, j) & S_a(i, j-b+1) & S_a(i-b+1, j-b+1)
// (doubling from 32, then binary search), and the witness is the first set
// bit of S_K.  One CTA per matrix; passes are separated by __syncthreads.

// A bitplane stored over rows [r0, ...) x words [w0, w0 + pitch) and zero
// outside its active box [ar0, ar1) x [aw0, aw1), which lies inside the
// storage.  A plane holds fewer than 2^31 words, so indices fit 32 bits.
struct Plane {
  uint32_t* p;
  int r0, w0, pitch;
  int ar0, ar1, aw0, aw1;
  __device__ __forceinline__ uint32_t get(int i, int w) const {
    return (i >= ar0 && i < ar1 && w >= aw0 && w < aw1) ? p[(i - r0) * pitch + (w - w0)] : 0u;
  }
  __device__ __forceinline__ bool empty() const { return ar1 <= ar0 || aw1 <= aw0; }
};

// A team of `size` blocks sharing one matrix's bitplane passes (size 1: a
// lone block).  Passes spread their cells over all the team's threads and end
// with a team barrier: __syncthreads for one block; for several, an arrival
// counter in global memory (bounded wait: on timeout the matrix's status
// becomes MS_ERR_TIMEOUT and the block stops waiting, so nothing hangs).
// Pass boxes and the witness minimum of several blocks live in global memory.
struct TeamSync {            // one per matrix, zeroed before the launch
  unsigned int arrive;       // barrier arrivals
  unsigned int pad;
  int box[3][4];             // pass boxes (as PassBox slots)
  unsigned long long first;  // witness: smallest row-major index
};
static_assert(sizeof(TeamSync) == 64, "cleared as 16 words");

// Zeroes a single call's team state from the tile kernel before it (the
// fix-up reads it only after waiting for that grid); null: nothing to clear.
__device__ __forceinline__ void clear_team(TeamSync* t) {
  if (t && blockIdx.x == 0 && threadIdx.x < 16) reinterpret_cast<uint32_t*>(t)[threadIdx.x] = 0u;
}
struct Team {
  int size, rank;
  TeamSync* sync;  // null when size == 1
  int32_t* status;
  unsigned int passed;  // barriers passed
  bool gave_up;
  bool cluster;         // the team is one thread-block cluster: hardware barrier
  __device__ __forceinline__ int thread() const { return rank * (int)blockDim.x + (int)threadIdx.x; }
  __device__ __forceinline__ int threads() const { return size * (int)blockDim.x; }
  __device__ __forceinline__ void barrier() {
    if (size > 1 && cluster) {
      // every thread of every block of the cluster; release/acquire order
      // the team's global-memory plane writes before the next pass's reads
      asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                   "barrier.cluster.wait.acquire.aligned;" ::: "memory");
      ++passed;
      return;
    }
    __syncthreads();
    if (size > 1) {
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&sync->arrive, 1u);
        const unsigned int target = (passed + 1) * (unsigned int)size;
        if (!gave_up) {
          int spins = 0;
          const unsigned long long t0 = global_ns();
          while ((unsigned int)ld_acquire(reinterpret_cast<const int32_t*>(&sync->arrive)) <
                 target) {
            if (++spins > kSpinLimit || global_ns() - t0 > kWaitLimitNs) {
              gave_up = true;
              atomicExch(status, (int)MS_ERR_TIMEOUT);
              break;
            }
            __nanosleep(32);
          }
        }
        __threadfence();
      }
      ++passed;
      __syncthreads();
    }
  }
};

// Visits the cells (r, c) of a rows x cols grid, spread over the team's
// threads in row-major order; the row/column step is kept incrementally.
// U cells per thread are unrolled (more for passes whose loads come from
// global memory, so that their latencies overlap).
template <int U = 2, class F>
__device__ __forceinline__ void for_cells(const Team& tm, int rows, int cols, F&& f) {
  if (rows <= 0 || cols <= 0) return;
  const int bd = tm.threads(), t0 = tm.thread();
  const int dr = bd / cols, dc = bd - dr * cols;
  int r = t0 / cols, c = t0 - r * cols;
#pragma unroll U
  for (; r < rows;) {
    f(r, c);
    r += dr;
    c += dc;
    if (c >= cols) {
      c -= cols;
      ++r;
    }
  }
}

// bit k of the result = byte k of x is nonzero (k = 0..3): the byte flags
// sit at bits 0, 8, 16, 24 and one multiply moves them to bits 24..27 without
// carries (every partial product lands on its own bit).
__device__ __forceinline__ uint32_t byte_flags4(uint32_t x) {
  const uint32_t t = (nonzero_msb(x) >> 7) & 0x01010101u;
  return (t * 0x01020408u) >> 24;
}

// 32 cells of input row i starting at column 32*w, as bits (columns >= n: 0).
template <int FMT>
__device__ __forceinline__ uint32_t input_word(const Job& j, int i, int w) {
  const int64_t c = 32 * (int64_t)w;
  if (i < 0 || i >= j.m || w < 0 || c >= j.n) return 0u;
  const int64_t valid = j.n - c;
  if constexpr (FMT == MS_BITS32) {
    const uint32_t mask = valid >= 32 ? 0xffffffffu : ((1u << valid) - 1u);
    return __ldg(reinterpret_cast<const uint32_t*>(j.data) + (int64_t)i * j.ld + w) & mask;
  } else {
    const uint8_t* row = reinterpret_cast<const uint8_t*>(j.data) + (int64_t)i * j.ld + c;
    if (valid >= 32 && j.aligned) {
      const uint4 lo = __ldg(reinterpret_cast<const uint4*>(row));
      const uint4 hi = __ldg(reinterpret_cast<const uint4*>(row) + 1);
      return byte_flags4(lo.x) | byte_flags4(lo.y) << 4 | byte_flags4(lo.z) << 8 |
             byte_flags4(lo.w) << 12 | byte_flags4(hi.x) << 16 | byte_flags4(hi.y) << 20 |
             byte_flags4(hi.z) << 24 | byte_flags4(hi.w) << 28;
    }
    uint32_t bits = 0;
    const int lim = valid >= 32 ? 32 : (int)valid;
    for (int b = 0; b < lim; ++b) bits |= (uint32_t)(__ldg(row + b) != 0) << b;
    return bits;
  }
}

// Per-pass bounding box of the nonzero words a block writes.  Threads reduce
// per warp and fold into slot k % 3 with shared-memory atomics; slot
// (k+1) % 3 is reset during pass k (its last readers finished before the
// barrier of pass k-1), so each pass needs a single __syncthreads.
__device__ __forceinline__ void box_reset(int* b) {
  b[0] = 0x7fffffff;
  b[1] = -1;
  b[2] = 0x7fffffff;
  b[3] = -1;
}
// A team's boxes in global memory are kept so that all-zero bytes mean the
// empty box (the launch's memset prepares pass 0 with no reset that could
// race another block's first fold): 0x7fffffff - min and max + 1, both
// folded with atomicMax.
__device__ __forceinline__ void gbox_reset(int* b) {
  b[0] = 0;
  b[1] = 0;
  b[2] = 0;
  b[3] = 0;
}
struct PassBox {
  int (*part)[32][4];  // shared [2][32][4]: per-warp partial boxes, by pass parity
  int k;
  Team* tm;
  __device__ __forceinline__ void begin() const {
    if (threadIdx.x == 0 && tm->size > 1 && tm->rank == 0) gbox_reset(tm->sync->box[(k + 1) % 3]);
  }
  // all threads of the team; returns [r0, r1) x [w0, w1) (empty: r1 <= r0).
  // Each warp posts its partial box and, after one barrier, folds all of
  // them itself (no shared-memory atomics to serialise on one address).
  __device__ __forceinline__ void end(int rmin, int rmax, int wmin, int wmax, int out[4]) {
    rmin = __reduce_min_sync(kFull, rmin);
    rmax = __reduce_max_sync(kFull, rmax);
    wmin = __reduce_min_sync(kFull, wmin);
    wmax = __reduce_max_sync(kFull, wmax);
    int(*p)[4] = part[k & 1];
    const int lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
    if (lane == 0) {
      int* q = p[threadIdx.x >> 5];
      q[0] = rmin;
      q[1] = rmax;
      q[2] = wmin;
      q[3] = wmax;
    }
    __syncthreads();
    int b0 = 0x7fffffff, b1 = -1, b2 = 0x7fffffff, b3 = -1;
    if (lane < nw) {
      b0 = p[lane][0];
      b1 = p[lane][1];
      b2 = p[lane][2];
      b3 = p[lane][3];
    }
    b0 = __reduce_min_sync(kFull, b0);
    b1 = __reduce_max_sync(kFull, b1);
    b2 = __reduce_min_sync(kFull, b2);
    b3 = __reduce_max_sync(kFull, b3);
    if (tm->size > 1) {
      int* g = tm->sync->box[k % 3];
      if (threadIdx.x == 0 && b1 >= 0) {
        atomicMax(g + 0, 0x7fffffff - b0);
        atomicMax(g + 1, b1 + 1);
        atomicMax(g + 2, 0x7fffffff - b2);
        atomicMax(g + 3, b3 + 1);
      }
      tm->barrier();
      // thread 0 reads the team's box (after its acquire) and shares it
      // through the partials' first row, which every warp has finished with
      if (threadIdx.x == 0) {
        p[0][0] = 0x7fffffff - *reinterpret_cast<volatile int*>(g + 0);
        p[0][1] = *reinterpret_cast<volatile int*>(g + 1) - 1;
        p[0][2] = 0x7fffffff - *reinterpret_cast<volatile int*>(g + 2);
        p[0][3] = *reinterpret_cast<volatile int*>(g + 3) - 1;
      }
      __syncthreads();
      b0 = p[0][0];
      b1 = p[0][1];
      b2 = p[0][2];
      b3 = p[0][3];
    }
    out[0] = b0;
    out[1] = b1 + 1;
    out[2] = b2;
    out[3] = b3 + 1;
    ++k;
  }
};

// O = grow(L, d) = S_{a+d} from L = S_a (0 <= d <= a): bit (i, col) is
// L(i, col) & L(i-d, col) & L(i, col-d) & L(i-d, col-d), columns >= n cleared.
// Only L's active box (clipped to O's storage rows/words) can be nonzero.
// Writes O's words there (if write) and sets O's active box; `first`
// receives the smallest row-major index of a set bit.
__device__ __forceinline__ void grow_pass(const Plane& L, Plane& O, int o_r1, int o_w1, int d,
                                          int64_t n, bool write, unsigned long long* first,
                                          PassBox& pb, const Job* emit = nullptr) {
  const int q = d >> 5, r = d & 31;
  const int r0 = max(L.ar0, O.r0), r1 = min(L.ar1, o_r1);
  const int w0 = max(L.aw0, O.w0), w1 = min(L.aw1, o_w1);
  int rmin = 0x7fffffff, rmax = -1, wmin = 0x7fffffff, wmax = -1;
  unsigned long long f = ~0ull;
  pb.begin();
  // (i, w) runs over L's active box, so only the shifted reads (rows i - d,
  // words w - q and w - q - 1) can fall outside it; the matrix's last word
  // is the only partial one
  const int wlast = (int)((n - 1) >> 5);
  const uint32_t lastmask = (n & 31) ? ((1u << (n & 31)) - 1u) : 0xffffffffu;
  for_cells(*pb.tm, r1 - r0, w1 - w0, [&](int rr, int cc) {
    const int i = r0 + rr, w = w0 + cc;
    const uint32_t* row = L.p + (i - L.r0) * L.pitch - L.w0;
    const bool up_ok = i - d >= L.ar0;
    const uint32_t* up = row - d * L.pitch;
    const int wq = w - q;
    const bool q_ok = wq >= L.aw0, q1_ok = wq - 1 >= L.aw0;
    const uint32_t a0 = row[w];
    const uint32_t a1 = up_ok ? up[w] : 0u;
    uint32_t a2 = q_ok ? row[wq] : 0u;
    uint32_t a3 = (up_ok && q_ok) ? up[wq] : 0u;
    if (r) {
      a2 = (a2 << r) | ((q1_ok ? row[wq - 1] : 0u) >> (32 - r));
      a3 = (a3 << r) | ((up_ok && q1_ok ? up[wq - 1] : 0u) >> (32 - r));
    }
    const uint32_t v = a0 & a1 & a2 & a3 & (w == wlast ? lastmask : 0xffffffffu);
    if (write) O.p[(i - O.r0) * O.pitch + (w - O.w0)] = v;
    if (v) {
      rmin = min(rmin, i);
      rmax = max(rmax, i);
      wmin = min(wmin, w);
      wmax = max(wmax, w);
      if (first) {
        const unsigned long long cand = (unsigned long long)i * (unsigned long long)n +
                                        (unsigned long long)(32 * (int64_t)w) +
                                        (unsigned long long)(__ffs(v) - 1);
        f = cand < f ? cand : f;
      }
      if (emit)
        for (uint32_t b = v; b; b &= b - 1)
          emit_corner(*emit, i, 32 * (int64_t)w + (__ffs(b) - 1));
    }
  });
  if (first) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(kFull, f, o);
      f = v < f ? v : f;
    }
    if ((threadIdx.x & 31) == 0 && f != ~0ull) atomicMin(first, f);
  }
  int box[4];
  pb.end(rmin, rmax, wmin, wmax, box);
  O.ar0 = box[0];
  O.ar1 = box[1];
  O.aw0 = box[2];
  O.aw1 = box[3];
}

// Multi-way test by the team, no plane written: how many of the T (<= 7)
// sides t_k = a + d[k] (ascending, 0 < d[k] <= a) have a corner, from L =
// S_a over its active box clipped to rows [o_r0, o_r1) x words [o_w0, o_w1).
// A corner of a t-square is a corner of every smaller square, so the sides
// with a corner are a prefix: a word tests the sides above its best so far,
// the largest first, and stops at its first hit.
constexpr int kTeamWays = 7;
__device__ __forceinline__ int probe_pass(const Plane& L, int o_r0, int o_w0, int o_r1, int o_w1,
                                          const int (&d)[kTeamWays], int T, int64_t n,
                                          PassBox& pb) {
  const int r0 = max(L.ar0, o_r0), r1 = min(L.ar1, o_r1);
  const int w0 = max(L.aw0, o_w0), w1 = min(L.aw1, o_w1);
  const int wlast = (int)((n - 1) >> 5);
  const uint32_t lastmask = (n & 31) ? ((1u << (n & 31)) - 1u) : 0xffffffffu;
  int found = 0;
  pb.begin();
  for_cells(*pb.tm, r1 - r0, w1 - w0, [&](int rr, int cc) {
    const int i = r0 + rr, w = w0 + cc;
    const uint32_t* row = L.p + (i - L.r0) * L.pitch - L.w0;
    const uint32_t a0 = row[w] & (w == wlast ? lastmask : 0xffffffffu);
    if (!a0) return;
#pragma unroll
    for (int k = kTeamWays - 1; k >= 0; --k) {
      if (k >= T) continue;
      if (k < found) break;
      const int dk = d[k], q = dk >> 5, r = dk & 31;
      if (i - dk < L.ar0) continue;  // the square's top row lies above every set bit
      const uint32_t* up = row - dk * L.pitch;
      const int wq = w - q;
      const bool q_ok = wq >= L.aw0, q1_ok = wq - 1 >= L.aw0;
      uint32_t a2 = q_ok ? row[wq] : 0u;
      uint32_t a3 = q_ok ? up[wq] : 0u;
      if (r) {
        a2 = (a2 << r) | ((q1_ok ? row[wq - 1] : 0u) >> (32 - r));
        a3 = (a3 << r) | ((q1_ok ? up[wq - 1] : 0u) >> (32 - r));
      }
      if (a0 & up[w] & a2 & a3) {
        found = k + 1;
        break;
      }
    }
  });
  int box[4];
  pb.end(0x7fffffff, found - 1, 0x7fffffff, -1, box);
  return box[1];  // the team's largest count
}

// Geometry of the bitplane fix-up of box [rlo, rhi) x [clo, chi): S_32 is
// built on rows [ra, rhi) x words [wa, whi) (the box grown by 32 up and
// left) from input rows [pa, rhi) x words [wa-1, whi).
struct BitGeo {
  int ra, wlo, whi, wa, R1, W1, pa, Wv, RP;
  __device__ __forceinline__ BitGeo(int rlo, int rhi, int clo, int chi) {
    ra = max(0, rlo - kHalo);
    wlo = clo / 32;
    whi = (chi + 31) / 32;
    wa = max(0, clo - kHalo) / 32;
    R1 = rhi - ra;
    W1 = whi - wa;
    pa = max(0, ra - 31);
    Wv = W1 + 1;
    RP = rhi - pa;
  }
};

// S_32 of the geometry into s32buf (R1 x W1 words), through the input buffer
// `in` and the vertical buffer `vb` (RP x Wv words each); returns its plane
// with the active box of its set bits.
template <int FMT>
__device__ __forceinline__ Plane build_s32(const Job& j, const BitGeo& g, uint32_t* in,
                                           uint32_t* vb, uint32_t* s32buf, PassBox& pb) {
  const int RP = g.RP, Wv = g.Wv, R1 = g.R1, W1 = g.W1, ra = g.ra, wa = g.wa, pa = g.pa;
  Team& tm = *pb.tm;
  // 1. input bits of rows [pa, rhi), words [wa-1, whi)
  for_cells<8>(tm, RP, Wv, [&](int rr, int cc) {
    in[rr * Wv + cc] = input_word<FMT>(j, pa + rr, wa - 1 + cc);
  });
  tm.barrier();
  // 2. vertical: V_32(i, w) = AND of the 32 rows ending at i.  Rows are taken
  //    in blocks of 32 counted from pa; one thread per block and word column
  //    stores the running AND from the block's top (prefix, into `vb`) and,
  //    in place, from its bottom (suffix, into `in`).  Then V_32(i) is
  //    suffix(i - 31) & prefix(i), or the block's whole prefix when i ends a
  //    block.  Rows above pa only matter when pa is the matrix top, where
  //    they are zeros.
  const int nb = (RP + 31) / 32;
  for_cells(tm, nb, Wv, [&](int bk, int cc) {
    const int r0 = 32 * bk, rows = min(32, RP - r0);
    uint32_t acc = 0xffffffffu;
    for (int k = 0; k < rows; ++k) {
      acc &= in[(r0 + k) * Wv + cc];
      vb[(r0 + k) * Wv + cc] = acc;
    }
    acc = 0xffffffffu;
    for (int k = rows - 1; k >= 0; --k) {
      acc &= in[(r0 + k) * Wv + cc];
      in[(r0 + k) * Wv + cc] = acc;
    }
  });
  tm.barrier();
  auto v32 = [&](int rr, int cc) -> uint32_t {
    if ((rr & 31) == 31) return vb[rr * Wv + cc];
    if (rr < 31) return 0u;
    return in[(rr - 31) * Wv + cc] & vb[rr * Wv + cc];
  };
  // 3. horizontal: S_32 = AND of 32 consecutive V_32 bits ending at each
  //    cell, on rows [ra, rhi) x words [wa, whi)
  Plane s32{s32buf, ra, wa, W1, 0, 0, 0, 0};
  int rmin = 0x7fffffff, rmax = -1, wmin = 0x7fffffff, wmax = -1;
  pb.begin();
  for_cells(tm, R1, W1, [&](int rr, int cc) {
    const int vr = rr + (ra - pa);  // row of V_32 in its [pa, rhi) layout
    const uint32_t x = v32(vr, cc + 1), y = v32(vr, cc);
    unsigned long long z = ((unsigned long long)x << 32) | y;
    z &= z << 1;
    z &= z << 2;
    z &= z << 4;
    z &= z << 8;
    z &= z << 16;
    const uint32_t v = (uint32_t)(z >> 32);
    s32buf[rr * W1 + cc] = v;
    if (v) {
      rmin = min(rmin, ra + rr);
      rmax = max(rmax, ra + rr);
      wmin = min(wmin, wa + cc);
      wmax = max(wmax, wa + cc);
    }
  });
  int box[4];
  pb.end(rmin, rmax, wmin, wmax, box);
  s32.ar0 = box[0];
  s32.ar1 = box[1];
  s32.aw0 = box[2];
  s32.aw1 = box[3];
  return s32;
}

// S_33 of rows [rlo, rhi) x words [wlo, whi) from the bitplane tiles' rows
// (job.first33 set): a word counts where its tile had reached its first
// S_33 row, and is zero elsewhere (every S_33 cell lies in the flagged box,
// so nothing outside it is needed).  Written to `out` (pitch whi - wlo);
// returns its plane.
__device__ __forceinline__ Plane gather_s33(const Job& j, int rlo, int rhi, int wlo, int whi,
                                            uint32_t* out, PassBox& pb) {
  const int64_t pw = (j.n + 31) / 32;
  const uint32_t* raw = j.bits_scratch + 2 * j.m * (pw + 2);
  const int BW = whi - wlo;
  // bitplane tiles are 1024 columns wide (lane width 32); later strips count
  // 1024 - kHalo of them (constant divisors: no division loops per word)
  constexpr int64_t W = 32 * 32;
  Plane s{out, rlo, wlo, BW, 0, 0, 0, 0};
  int rmin = 0x7fffffff, rmax = -1, wmin = 0x7fffffff, wmax = -1;
  pb.begin();
  for_cells<8>(*pb.tm, rhi - rlo, BW, [&](int rr, int cc) {
    const int i = rlo + rr, w = wlo + cc;
    const int64_t c = 32 * (int64_t)w;
    const int64_t strip = c < W ? 0 : 1 + (c - W) / (W - kHalo);
    const int64_t t = (int64_t)(i / j.band_rows) * j.strips + strip;
    const int f33 = __ldcg(j.first33 + t);
    const uint32_t rv = __ldcg(raw + (int64_t)i * pw + w);
    const uint32_t v = f33 <= i ? rv : 0u;
    out[rr * BW + cc] = v;
    if (v) {
      rmin = min(rmin, i);
      rmax = max(rmax, i);
      wmin = min(wmin, w);
      wmax = max(wmax, w);
    }
  });
  int box[4];
  pb.end(rmin, rmax, wmin, wmax, box);
  s.ar0 = box[0];
  s.ar1 = box[1];
  s.aw0 = box[2];
  s.aw1 = box[3];
  return s;
}

// ---- size-only fix-up by one block with its planes in shared memory -----
//
// The common case (a single call's box, or a batch matrix's, that fits one
// block's shared memory): the growth, search and witness of fixup_bits
// below, specialised for one block.  Passes walk the active box of their
// source plane with per-cell predicates and end with one block barrier; the
// search tests several sides per pass while the plane is small.  The result
// is the same: K = the largest t with S_t non-empty, witness = the first set
// bit of S_K in row-major order.
namespace sbox {

constexpr int kWays = 7;          // sides tested per search pass, at most
constexpr int kProbeBudget = 16;  // word tests per thread a search pass may take

// A plane stored over rows [r0, r0 + rows) x words [w0, w0 + cols) of the
// matrix in shared memory (row pitch `pitch` >= cols, odd so that threads
// walking different rows meet different banks), zero outside its active box
// [ar0, ar1) x [aw0, aw1).
struct SP {
  uint32_t* p;
  int r0, w0, pitch, cols, rows;
  int ar0, ar1, aw0, aw1;
  __device__ __forceinline__ int base(int i) const { return (i - r0) * pitch - w0; }
  __device__ __forceinline__ bool empty() const { return ar1 <= ar0 || aw1 <= aw0; }
};

__host__ __device__ __forceinline__ int odd_pitch(int cols) { return cols | 1; }

// A rows x cols region cut into rows * nseg runs of at most `len`
// consecutive words of one row; the block's threads take the runs with
// stride blockDim (about one each).
struct Runs {
  int rows, cols, nseg, len;
  __device__ __forceinline__ Runs(int r, int c) : rows(r), cols(c), nseg(0), len(0) {
    if (r <= 0 || c <= 0) return;
    nseg = max(1, min(c, (int)blockDim.x / r));
    len = (c + nseg - 1) / nseg;
    nseg = (c + len - 1) / len;
  }
  template <class F>
  __device__ __forceinline__ void each(F&& f) const {
    if (nseg == 0) return;
    // unit u = r * nseg + seg, stepped by blockDim without a division per unit
    const int bd = (int)blockDim.x, dr = bd / nseg, ds = bd - dr * nseg;
    int r = (int)threadIdx.x / nseg, seg = (int)threadIdx.x - r * nseg;
    while (r < rows) {
      const int c0 = seg * len;
      f(r, c0, min(cols, c0 + len));
      r += dr;
      seg += ds;
      if (seg >= nseg) {
        seg -= nseg;
        ++r;
      }
    }
  }
};

// Words [wb, we) (inside L's active box) of row i of S_{a+d} from L = S_a
// (0 <= d <= a): the AND of L at (i, col), (i-d, col), (i, col-d),
// (i-d, col-d) for the words' 32 columns, reads left of or above L's active
// box being zeros.  g(w, v) receives each word in order; the shifted reads of
// one word are reused by the next.
// A word whose own bit of L is clear everywhere yields zero without the
// other reads (the levels of random matrices turn sparse within a few
// doublings); a run of set words reuses the previous word's shifted reads.
template <class G>
__device__ __forceinline__ void grow_run(const SP& L, int i, int wb, int we, int d, G&& g) {
  if (i - d < L.ar0) {  // the square's top row lies above every set bit
    for (int w = wb; w < we; ++w) g(w, 0u);
    return;
  }
  const int q = d >> 5, r = d & 31;
  const uint32_t* __restrict__ p = L.p;
  const int bi = L.base(i), bu = L.base(i - d);
  uint32_t pb = 0u, pc = 0u;
  bool have = false;  // pb, pc hold the shifted reads of word w - 1
  int wq = wb - q;
#pragma unroll 2
  for (int w = wb; w < we; ++w, ++wq) {
    const uint32_t a0 = p[bi + w];
    if (a0 == 0u) {
      have = false;
      g(w, 0u);
      continue;
    }
    if (!have) {
      const bool ok1 = wq - 1 >= L.aw0;
      pb = ok1 ? p[bi + wq - 1] : 0u;
      pc = ok1 ? p[bu + wq - 1] : 0u;
    }
    const bool ok = wq >= L.aw0;
    const uint32_t b = ok ? p[bi + wq] : 0u;
    const uint32_t c = ok ? p[bu + wq] : 0u;
    g(w, a0 & p[bu + w] & __funnelshift_l(pb, b, r) & __funnelshift_l(pc, c, r));
    pb = b;
    pc = c;
    have = true;
  }
}

// Block-wide fold of per-thread boxes through `part` ([32][4] shared ints;
// callers alternate two such buffers between consecutive folds); every
// thread receives [r0, r1) x [w0, w1) (empty: r1 <= r0).
__device__ __forceinline__ void fold_box(int rmin, int rmax, int wmin, int wmax, int (*part)[4],
                                         int out[4]) {
  rmin = __reduce_min_sync(kFull, rmin);
  rmax = __reduce_max_sync(kFull, rmax);
  wmin = __reduce_min_sync(kFull, wmin);
  wmax = __reduce_max_sync(kFull, wmax);
  const int lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
  if (lane == 0) {
    int* q = part[threadIdx.x >> 5];
    q[0] = rmin;
    q[1] = rmax;
    q[2] = wmin;
    q[3] = wmax;
  }
  __syncthreads();
  int b0 = 0x7fffffff, b1 = -1, b2 = 0x7fffffff, b3 = -1;
  if (lane < nw) {
    b0 = part[lane][0];
    b1 = part[lane][1];
    b2 = part[lane][2];
    b3 = part[lane][3];
  }
  out[0] = __reduce_min_sync(kFull, b0);
  out[1] = __reduce_max_sync(kFull, b1) + 1;
  out[2] = __reduce_min_sync(kFull, b2);
  out[3] = __reduce_max_sync(kFull, b3) + 1;
}

// O = S_{a+d} from L = S_a over L's active box clipped to O's storage; sets
// O's active box.
__device__ __forceinline__ void grow_write(const SP& L, SP& O, int d, int (*part)[4]) {
  const int r0 = max(L.ar0, O.r0), r1 = min(L.ar1, O.r0 + O.rows);
  const int w0 = max(L.aw0, O.w0), w1 = min(L.aw1, O.w0 + O.cols);
  int rmin = 0x7fffffff, rmax = -1, wmin = 0x7fffffff, wmax = -1;
  uint32_t* __restrict__ op = O.p;  // (never the plane read)
  Runs(r1 - r0, w1 - w0).each([&](int rr, int cb, int ce) {
    const int i = r0 + rr, ob = O.base(i);
    bool any = false;
    grow_run(L, i, w0 + cb, w0 + ce, d, [&](int w, uint32_t v) {
      op[ob + w] = v;
      if (v) {
        wmin = min(wmin, w);
        wmax = max(wmax, w);
        any = true;
      }
    });
    if (any) {
      rmin = min(rmin, i);
      rmax = max(rmax, i);
    }
  });
  int box[4];
  fold_box(rmin, rmax, wmin, wmax, part, box);
  O.ar0 = box[0];
  O.ar1 = box[1];
  O.aw0 = box[2];
  O.aw1 = box[3];
}

// Bit k of the result (k < T <= kWays): S_{t_k} has a set bit, for the T
// sides t_k = lo + (k+1) * span / (T+1) tested from L = S_a (t_k - a <= a).
// A corner of a t-square is a corner of every smaller square, so each run
// tests the sides from the largest down and stops at its first hit.
__device__ __forceinline__ unsigned probe(const SP& L, int a, int lo, int span, int T,
                                          int (*part)[4]) {
  // (32-bit: span * kWays < 2^31 for every supported side)
  int d[kWays];
  const unsigned q = (unsigned)span / (unsigned)(T + 1), rem = (unsigned)span % (unsigned)(T + 1);
#pragma unroll
  for (int k = 0; k < kWays; ++k)
    d[k] = lo + (int)(q * (k + 1) + (rem * (k + 1)) / (unsigned)(T + 1)) - a;
  unsigned mask = 0u;
  Runs(L.ar1 - L.ar0, L.aw1 - L.aw0).each([&](int rr, int cb, int ce) {
    const int i = L.ar0 + rr;
#pragma unroll
    for (int k = kWays - 1; k >= 0; --k) {
      if (k >= T || (mask >> k & 1u)) continue;
      uint32_t hit = 0u;
      grow_run(L, i, L.aw0 + cb, L.aw0 + ce, d[k], [&](int, uint32_t v) { hit |= v; });
      if (hit) {
        mask |= (2u << k) - 1u;
        break;
      }
    }
  });
  mask = __reduce_or_sync(kFull, mask);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5][0] = (int)mask;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  return __reduce_or_sync(kFull, lane < (int)(blockDim.x >> 5) ? (unsigned)part[lane][0] : 0u);
}

// The first set bit (row-major index i*n + col) of S_{a+d} from L = S_a, or
// ~0; every set bit is appended to the corner list when `emit` is given.
__device__ __forceinline__ unsigned long long first_bit(const SP& L, int d, int64_t n,
                                                        unsigned long long* s_first,
                                                        const Job* emit) {
  unsigned long long f = ~0ull;
  Runs(L.ar1 - L.ar0, L.aw1 - L.aw0).each([&](int rr, int cb, int ce) {
    const int i = L.ar0 + rr;
    grow_run(L, i, L.aw0 + cb, L.aw0 + ce, d, [&](int w, uint32_t v) {
      if (!v) return;
      const unsigned long long cand = (unsigned long long)i * (unsigned long long)n +
                                      (unsigned long long)(32 * (int64_t)w) +
                                      (unsigned long long)(__ffs(v) - 1);
      f = cand < f ? cand : f;
      if (emit)
        for (uint32_t b = v; b; b &= b - 1)
          emit_corner(*emit, i, 32 * (int64_t)w + (__ffs(b) - 1));
    });
  });
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(kFull, f, o);
    f = v < f ? v : f;
  }
  if ((threadIdx.x & 31) == 0 && f != ~0ull) atomicMin(s_first, f);
  __syncthreads();
  return *reinterpret_cast<volatile unsigned long long*>(s_first);
}

// S_33 of rows [rlo, rhi) x words [wlo, whi) from the bitplane tiles' rows
// (job.first33 set: a word counts where its tile had reached its first S_33
// row, zero elsewhere) into `out` (shared, pitch odd_pitch(whi - wlo)).  The
// threads take the cells in row-major order (coalesced reads) and each
// issues the global reads of kBatch of its cells before using any of them.
__device__ __forceinline__ SP gather33(const Job& j, int rlo, int rhi, int wlo, int whi,
                                      uint32_t* out, int (*part)[4]) {
  constexpr int kBatch = 8;
  const int64_t pw = (j.n + 31) / 32;
  const uint32_t* raw = j.bits_scratch + 2 * j.m * (pw + 2);
  const int BW = whi - wlo, rows = rhi - rlo, P = odd_pitch(BW);
  // tiles are 32 words wide; a later strip counts 31 (its first is halo)
  const int br = j.band_rows;
  const float inv_br = 1.0f / (float)br;
  int rmin = 0x7fffffff, rmax = -1, wmin = 0x7fffffff, wmax = -1;
  const int bd = (int)blockDim.x;
  const int dr = bd / BW, dc = bd - dr * BW;
  int r = (int)threadIdx.x / BW, c = (int)threadIdx.x - r * BW;
  while (r < rows) {
    int rk[kBatch], ck[kBatch], f[kBatch];
    uint32_t rv[kBatch];
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      rk[k] = r;
      ck[k] = c;
      f[k] = 0x7fffffff;
      rv[k] = 0u;
      if (r < rows) {
        const int i = rlo + r, w = wlo + c;
        const int strip = w < 32 ? 0 : 1 + (w - 32) / 31;
        int band = (int)((float)i * inv_br);  // then corrected to i / br exactly
        band -= band * br > i;
        band += (band + 1) * br <= i;
        f[k] = __ldcg(j.first33 + (int64_t)band * j.strips + strip);
        rv[k] = __ldcg(raw + (int64_t)i * pw + w);
      }
      r += dr;
      c += dc;
      if (c >= BW) {
        c -= BW;
        ++r;
      }
    }
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      if (rk[k] < rows) {
        const int i = rlo + rk[k], w = wlo + ck[k];
        const uint32_t v = f[k] <= i ? rv[k] : 0u;
        out[rk[k] * P + ck[k]] = v;
        if (v) {
          rmin = min(rmin, i);
          rmax = max(rmax, i);
          wmin = min(wmin, w);
          wmax = max(wmax, w);
        }
      }
    }
  }
  int box[4];
  fold_box(rmin, rmax, wmin, wmax, part, box);
  return SP{out, rlo, wlo, P, BW, rows, box[0], box[1], box[2], box[3]};
}

// The largest side found from some S_a and the row-major index (i*n + col)
// of its first corner (side 0: S_a was empty).
struct Found {
  int side;
  unsigned long long idx;
};

// From cur = S_a: doubling, search and witness.  The level planes alternate
// between f0 and f1, which hold rows [rlo, rhi) x words [wlo, whi) at pitch
// odd_pitch(whi - wlo); f1 may be cur's own buffer when cur has that
// geometry (it is free once the first level is built).  `part`: two fold
// buffers; the caller's last fold used part[1 - par0].  Every thread
// returns the same result.
__device__ __forceinline__ Found solve(const Job& j, SP cur, int a, uint32_t* f0, uint32_t* f1,
                                       int rlo, int rhi, int wlo, int whi, int (*part)[32][4],
                                       int par0) {
  __shared__ unsigned long long s_first;
  if (threadIdx.x == 0) s_first = ~0ull;
  __syncthreads();
  int par = par0;
  const int BW = whi - wlo, P = odd_pitch(BW);
  const int kmax = (int)min(j.m, j.n);
  SP nxt{f0, rlo, wlo, P, BW, rhi - rlo, 0, 0, 0, 0};
  int lo, hi;
  for (;;) {
    if (2 * a > kmax || cur.empty()) {
      lo = a;
      hi = min(2 * a, kmax + 1);
      break;
    }
    grow_write(cur, nxt, a, part[par]);
    par ^= 1;
    if (nxt.empty()) {
      lo = a;
      hi = 2 * a;
      break;
    }
    a *= 2;
    // the levels alternate between f0 and f1 (the starting plane is done with)
    uint32_t* other = nxt.p == f0 ? f1 : f0;
    cur = nxt;
    nxt = SP{other, rlo, wlo, P, BW, rhi - rlo, 0, 0, 0, 0};
  }
  if (cur.empty()) return Found{0, ~0ull};  // S_a itself empty
  // search: several sides per pass while the plane is small, else halving
  const int nw = max(1, (cur.ar1 - cur.ar0) * (cur.aw1 - cur.aw0));
  const int ways = max(1, min(kWays, kProbeBudget * (int)blockDim.x / nw));
  while (hi - lo > 1) {
    const int span = hi - lo;
    const int T = min(ways, span - 1);
    const unsigned m = probe(cur, a, lo, span, T, part[par]);
    par ^= 1;
    // S_t shrinks as t grows: the set bits are a prefix of the sides tested
    const int ok = __popc(m & ((1u << T) - 1u));
    const int nlo = ok ? lo + ok * span / (T + 1) : lo;
    const int nhi = ok < T ? lo + (ok + 1) * span / (T + 1) : hi;
    lo = nlo;
    hi = nhi;
  }
  const unsigned long long idx = first_bit(cur, lo - a, j.n, &s_first, j.corners_count ? &j : nullptr);
  return Found{idx == ~0ull ? 0 : lo, idx};
}

// Folds a found side and corner into the matrix's key (one thread).
__device__ __forceinline__ void publish(const Job& j, const Found& f) {
  if (threadIdx.x == 0 && f.side > 0)
    atomicMax(&j.st->key, make_key((int32_t)f.side, (int64_t)(f.idx / (unsigned long long)j.n),
                                   (int64_t)(f.idx % (unsigned long long)j.n), j.n));
}

}  // namespace sbox

// Size-only, by a team of `team_size` blocks (ranks 0..team_size-1, all
// called with the same box; `sync` may be null only for a team of one).  When
// the three planes fit in `smem_words` words of shared memory, rank 0 works
// alone from shared memory and the other ranks return; otherwise the planes
// live in the job's global scratch and the whole team shares every pass.
template <int FMT>
__device__ __forceinline__ void fixup_bits(const Job& j, int rlo, int rhi, int clo, int chi,
                                           uint32_t* smem, int64_t smem_words, int team_size,
                                           int rank, TeamSync* sync, bool cluster = false) {
  __shared__ unsigned long long s_first;
  __shared__ int s_part[2][32][4];
  const BitGeo g(rlo, rhi, clo, chi);
  const int wlo = g.wlo, whi = g.whi;
  // bitplane tiles hand over S_33 of the box; else S_32 is built from the
  // input on the box grown by the halo
  const bool from33 = j.first33 != nullptr;
  const int64_t box_plane = (int64_t)(rhi - rlo) * sbox::odd_pitch(whi - wlo);
  const bool fits = smem && (from33 ? 3 * box_plane
                                    : 2 * (int64_t)g.RP * g.Wv + (int64_t)g.R1 * g.W1) <= smem_words;
  // (a cluster's other blocks may leave: rank 0 alone never uses the cluster
  // barrier)
  const bool alone = fits || !sync || team_size <= 1;
  if (alone && rank != 0) return;
  if (fits) {
    // one block with every plane in shared memory: the specialised passes
    if (from33) {
      const sbox::SP s33 = sbox::gather33(j, rlo, rhi, wlo, whi, smem, s_part[0]);
      sbox::publish(j, sbox::solve(j, s33, kHalo + 1, smem + box_plane, smem + 2 * box_plane,
                                   rlo, rhi, wlo, whi, s_part, 1));
    } else {
      Team t1{1, 0, nullptr, &j.st->status, 0u, false, false};
      PassBox pb1{s_part, 0, &t1};
      uint32_t* in = smem;                             // input bits, then a level plane
      uint32_t* vb = smem + (int64_t)g.RP * g.Wv;      // V_32, then a level plane
      uint32_t* s32buf = smem + 2 * (int64_t)g.RP * g.Wv;
      const Plane s32 = build_s32<FMT>(j, g, in, vb, s32buf, pb1);
      const sbox::SP cur{s32.p, s32.r0, s32.w0, s32.pitch, s32.pitch, g.R1,
                         s32.ar0, s32.ar1, s32.aw0, s32.aw1};
      sbox::publish(j, sbox::solve(j, cur, 32, vb, in, rlo, rhi, wlo, whi, s_part, pb1.k & 1));
    }
    __syncthreads();
    return;
  }
  Team tm{alone ? 1 : team_size, alone ? 0 : rank, alone ? nullptr : sync, &j.st->status, 0u,
          false, cluster && !alone};
  PassBox pb{s_part, 0, &tm};
  if (threadIdx.x == 0) {
    s_first = ~0ull;
    if (!alone && rank == 0) {
      sync->first = ~0ull;
    }
  }
  unsigned long long* first = alone ? &s_first : &sync->first;
  // planes in the job's global scratch: V_32 then levels / S_32 on the grown
  // box / input then levels (from33: the tiles' S_33 rows sit in the third
  // plane, free again once the box's S_33 is gathered into the second)
  const int64_t cap = j.m * ((j.n + 31) / 32 + 2);
  uint32_t* buf0 = j.bits_scratch;
  uint32_t* buf1 = j.bits_scratch + cap;
  uint32_t* buf2 = j.bits_scratch + 2 * cap;
  const Plane s_a = from33 ? gather_s33(j, rlo, rhi, wlo, whi, buf1, pb)
                           : build_s32<FMT>(j, g, buf2, buf0, buf1, pb);
  // 4. doubling from a = 32 (or 33) inside the box [rlo, rhi) x [wlo, whi),
  //    then binary search; level planes alternate between buf0 and buf2
  const int BW = whi - wlo;
  Plane cur = s_a, nxt{buf0, rlo, wlo, BW, 0, 0, 0, 0};
  uint32_t* spare = buf2;
  int a = from33 ? kHalo + 1 : 32, lo, hi;
  const int kmax = (int)min(j.m, j.n);
  for (;;) {
    if (2 * a > kmax || cur.empty()) {
      lo = a;
      hi = min(2 * a, kmax + 1);
      break;
    }
    grow_pass(cur, nxt, rhi, whi, a, j.n, true, nullptr, pb);
    if (nxt.empty()) {
      lo = a;
      hi = 2 * a;
      break;
    }
    a *= 2;
    uint32_t* freed = cur.p == buf1 ? spare : cur.p;
    cur = nxt;
    nxt = Plane{freed, rlo, wlo, BW, 0, 0, 0, 0};
  }
  Plane probe = nxt;  // tests write nothing
  // search: up to seven sides per pass (fewer team barriers than halving)
  while (hi - lo > 1) {
    const int span = hi - lo, T = min(kTeamWays, span - 1);
    int d[kTeamWays];
#pragma unroll
    for (int k = 0; k < kTeamWays; ++k) d[k] = lo + (k + 1) * span / (T + 1) - a;
    const int ok = probe_pass(cur, probe.r0, probe.w0, rhi, whi, d, T, j.n, pb);
    const int nlo = ok ? lo + ok * span / (T + 1) : lo;
    const int nhi = ok < T ? lo + (ok + 1) * span / (T + 1) : hi;
    lo = nlo;
    hi = nhi;
  }
  // 5. witness: the first set bit of S_lo inside the box (and, for the
  //    all-largest-squares call, every set bit: all of them lie in the box)
  grow_pass(cur, probe, rhi, whi, lo - a, j.n, false, first, pb, j.corners_count ? &j : nullptr);
  if (threadIdx.x == 0 && tm.rank == 0) {
    const unsigned long long idx = *reinterpret_cast<volatile unsigned long long*>(first);
    if (idx != ~0ull)
      atomicMax(&j.st->key, make_key((int32_t)lo, (int64_t)(idx / (unsigned long long)j.n),
                                     (int64_t)(idx % (unsigned long long)j.n), j.n));
  }
  __syncthreads();
}

// ---- dp-map fix-up by bitplane levels -------------------------------------
//
// Cells with dp >= 33 lie in the flagged box, and there dp(i,j) is the
// largest t with S_t(i,j).  Keep the levels L_k = S_{32*2^k} (doubling inside
// the box until a level is empty).  A cell whose top level is k has dp in
// [a, 2a) with a = 32*2^k, and for 0 <= D < a
//   S_{a+D}(i,j) = L_k(i,j) & L_k(i-D,j) & L_k(i,j-D) & L_k(i-D,j-D),
// so a binary search on D (each test three bit reads of one stored level)
// gives dp = a + D exactly.  One block builds the levels in the job's scratch;
// a grid then writes the dp of every box cell whose S_32 bit is set and folds
// the largest into the matrix's key.  Levels that do not fit the scratch
// leave the table empty, and the strip fix-up runs instead.

constexpr int kMaxLevels = 12;  // 32 << 11 exceeds every supported side
struct LevelRec {
  int64_t off;  // words after the table
  int32_t r0, w0, pitch;
  int32_t ar0, ar1, aw0, aw1;
  int32_t pad;
};
struct LevelTab {
  int32_t n;  // levels stored; 0: none (no box, or the strip fix-up runs)
  int32_t pad;
  LevelRec lv[kMaxLevels];
};
constexpr int kTabWords = 256;
static_assert(sizeof(LevelTab) <= kTabWords * 4, "level table too large");

__device__ __forceinline__ uint32_t level_bit(const LevelRec& L, const uint32_t* base, int i,
                                              int c) {
  if (c < 0) return 0u;
  const int w = c >> 5;
  if (i < L.ar0 || i >= L.ar1 || w < L.aw0 || w >= L.aw1) return 0u;
  return (base[L.off + (int64_t)(i - L.r0) * L.pitch + (w - L.w0)] >> (c & 31)) & 1u;
}

// Builds S_32 and the doubling levels of box [rlo, rhi) x [clo, chi).  The
// input and vertical buffers use shared memory when they fit.  A
// thread-block cluster (cluster_size > 1, `sync` cleared before the launch)
// shares every pass, with all planes in global memory.
template <int FMT>
__device__ __forceinline__ void fixup_dp_levels(const Job& j, int rlo, int rhi, int clo, int chi,
                                                uint32_t* smem, int64_t smem_words,
                                                int cluster_size, int rank, TeamSync* sync) {
  __shared__ int s_part[2][32][4];
  const bool cl = cluster_size > 1;
  Team tm{cl ? cluster_size : 1, cl ? rank : 0, cl ? sync : nullptr, &j.st->status, 0u, false,
          cl};
  PassBox pb{s_part, 0, &tm};
  if (cl) smem = nullptr;
  LevelTab* tab = reinterpret_cast<LevelTab*>(j.bits_scratch);
  uint32_t* base = j.bits_scratch + kTabWords;
  const int64_t avail = 3 * j.m * ((j.n + 31) / 32 + 2) - kTabWords;
  const BitGeo g(rlo, rhi, clo, chi);
  const int64_t vw = (int64_t)g.RP * g.Wv;
  uint32_t *in, *vb;
  int64_t off = 0;
  if (smem && 2 * vw <= smem_words) {
    in = smem;
    vb = smem + vw;
  } else {
    in = base;
    vb = base + vw;
    off = 2 * vw;
  }
  if (off + (int64_t)g.R1 * g.W1 > avail) return;  // does not fit: table stays empty
  Plane cur = build_s32<FMT>(j, g, in, vb, base + off, pb);
  const bool writer = threadIdx.x == 0 && tm.rank == 0;
  if (writer)
    tab->lv[0] = LevelRec{off, g.ra, g.wa, g.W1, cur.ar0, cur.ar1, cur.aw0, cur.aw1, 0};
  off += (int64_t)g.R1 * g.W1;
  int nl = 1, a = 32;
  const int kmax = (int)min(j.m, j.n);
  while (!cur.empty() && 2 * a <= kmax && nl < kMaxLevels) {
    // S_2a lies inside S_a's active box and inside the box
    const int r0 = max(cur.ar0, rlo), r1 = cur.ar1;
    const int w0 = max(cur.aw0, g.wlo), w1 = cur.aw1;
    if (r1 <= r0 || w1 <= w0) break;
    const int64_t size = (int64_t)(r1 - r0) * (w1 - w0);
    if (off + size > avail) return;
    Plane nxt{base + off, r0, w0, w1 - w0, 0, 0, 0, 0};
    grow_pass(cur, nxt, r1, w1, a, j.n, true, nullptr, pb);
    if (nxt.empty()) break;
    if (writer)
      tab->lv[nl] = LevelRec{off, r0, w0, w1 - w0, nxt.ar0, nxt.ar1, nxt.aw0, nxt.aw1, 0};
    off += size;
    ++nl;
    a *= 2;
    cur = nxt;
  }
  if (writer) tab->n = nl;
}

// One block, or one thread-block cluster of gridDim.x blocks (`sync` cleared
// before the launch).
template <int FMT>
__global__ void __launch_bounds__(1024, 1) k_fixup_dp_levels(const Job job, int64_t smem_words,
                                                             TeamSync* sync) {
  extern __shared__ __align__(16) unsigned char ms_dyn_smem[];
  grid_dependency_wait();
  __shared__ int32_t sbox[4];
  if (threadIdx.x == 0) {
    if (blockIdx.x == 0) reinterpret_cast<LevelTab*>(job.bits_scratch)->n = 0;
    const volatile int32_t* b = job.st->box;
    sbox[0] = b[0];
    sbox[1] = b[1];
    sbox[2] = b[2];
    sbox[3] = b[3];
  }
  __syncthreads();
  if (sbox[1] > sbox[0] && sbox[3] > sbox[2])
    fixup_dp_levels<FMT>(job, sbox[0], sbox[1], sbox[2], sbox[3],
                         reinterpret_cast<uint32_t*>(ms_dyn_smem), smem_words, (int)gridDim.x,
                         (int)blockIdx.x, sync);
}

// Exact dp of the box cells from the levels (grid-stride over S_32's active
// region inside the box).
static __global__ void __launch_bounds__(256) k_fixup_dp_cells(const Job j) {
  __shared__ LevelRec s_lv[kMaxLevels];
  const LevelTab* tab = reinterpret_cast<const LevelTab*>(j.bits_scratch);
  const int nl = tab->n;
  if (nl <= 0) return;
  if ((int)threadIdx.x < nl) s_lv[threadIdx.x] = tab->lv[threadIdx.x];
  __syncthreads();
  const uint32_t* base = j.bits_scratch + kTabWords;
  const int rlo = j.st->box[0], rhi = j.st->box[1], clo = j.st->box[2], chi = j.st->box[3];
  const LevelRec& L0 = s_lv[0];
  const int r0 = max(rlo, L0.ar0), r1 = min(rhi, L0.ar1);
  const int c0 = max(clo, 32 * L0.aw0), c1 = min(chi, 32 * L0.aw1);
  unsigned long long key = 0;
  if (r1 > r0 && c1 > c0) {
    const int W = c1 - c0;
    const int64_t total = (int64_t)(r1 - r0) * W;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int i = r0 + (int)(e / W), c = c0 + (int)(e % W);
      if (!level_bit(L0, base, i, c)) continue;
      int k = 0;
      while (k + 1 < nl && level_bit(s_lv[k + 1], base, i, c)) ++k;
      const LevelRec& L = s_lv[k];
      int lo = 0, hi = 32 << k;  // S_{a+lo} holds, S_{a+hi} does not
      while (hi - lo > 1) {
        const int d = (lo + hi) >> 1;
        if (level_bit(L, base, i - d, c) & level_bit(L, base, i, c - d) &
            level_bit(L, base, i - d, c - d))
          lo = d;
        else
          hi = d;
      }
      const int dpv = (32 << k) + lo;
      j.dp[(int64_t)i * j.ld_dp + c] = dpv;
      const unsigned long long kk = make_key(dpv, i, c, j.n);
      key = kk > key ? kk : key;
    }
  }
  key = warp_max_u64(key);
  if ((threadIdx.x & 31) == 0 && key) atomicMax(&j.st->key, key);
}

// Writes the matrix's result from its key and leaves its state ready for the
// next call (call after a __syncthreads that follows all updates of the key).
__device__ __forceinline__ void finalize_job(const Job& j) {
  JobState* st = j.st;
  if (threadIdx.x == 0) {
    const unsigned long long key = ld_volatile_u64(&st->key);
    ms_result r;
    r.status = *reinterpret_cast<volatile int32_t*>(&st->status);
    if (key == 0ull) {
      r.side = 0;
      r.row = -1;
      r.col = -1;
    } else {
      const unsigned long long idx = kKeyMask - (key & kKeyMask);
      r.side = (int32_t)(key >> 40);
      r.row = (int32_t)(idx / (unsigned long long)j.n);
      r.col = (int32_t)(idx % (unsigned long long)j.n);
    }
    *j.out = r;
    // leave the state ready for the next call
    st->key = 0ull;
    st->box[0] = 0x7fffffff;
    st->box[1] = -1;
    st->box[2] = 0x7fffffff;
    st->box[3] = -1;
    st->status = 0;
    st->done = 0;
  }
}

template <int FMT, bool DPMAP>
__device__ __forceinline__ void fixup_job(const Job& j, bool after_levels = true) {
  __shared__ int32_t sbox[4];
  JobState* st = j.st;
  if (threadIdx.x == 0) {
    const volatile int32_t* b = st->box;
    sbox[0] = b[0];
    sbox[1] = b[1];
    sbox[2] = b[2];
    sbox[3] = b[3];
  }
  __syncthreads();
  const int rlo = sbox[0], rhi = sbox[1], clo = sbox[2], chi = sbox[3];
  // a dp map already completed from bitplane levels (launched just before
  // this kernel) needs no strips
  const bool done = DPMAP && after_levels && j.bits_scratch &&
                    reinterpret_cast<const LevelTab*>(j.bits_scratch)->n > 0;
  if (rhi > rlo && chi > clo && !done) {
    const int64_t br0 = max(0, rlo - kHalo);
    // rounded down to 32 columns: fix-up chunks must stay inside a packed
    // word and keep vector loads aligned (a wider window is still exact)
    const int64_t bc0 = (int64_t)(max(0, clo - kHalo) & ~31);
    const int nstrips = (int)((chi - bc0 + kFixW - 1) / kFixW);
    const int rows = (int)(rhi - br0);
    const int warp = threadIdx.x >> 5;
    const int nwarps = (int)(blockDim.x >> 5);  // strips go round-robin to the warps
    for (int s = warp; s < nstrips && s < j.strips_fix; s += nwarps) {
      Tile g;
      g.base = reinterpret_cast<const uint8_t*>(j.data);
      g.ld = j.ld;
      g.m = j.m;
      g.n = j.n;
      g.wr0 = br0;
      g.nrows = rows;
      g.cnt_ir0 = (int32_t)(rlo - br0);
      g.wc0 = bc0 + (int64_t)s * kFixW;
      g.c0 = clo;
      g.aligned = j.aligned;
      StripIO io;
      uint16_t* carry16 = reinterpret_cast<uint16_t*>(j.carry);
      const int64_t cs = carry_stride16(j.m);
      io.carry_in = s > 0 ? carry16 + (int64_t)(s - 1) * cs : nullptr;
      io.progress_in = s > 0 ? j.progress + (s - 1) : nullptr;
      io.carry_out = (s + 1 < nstrips) ? carry16 + (int64_t)s * cs : nullptr;
      io.progress_out = j.progress + s;
      io.status = &st->status;
      io.hold = (s == 0) ? j.test_hold : 0;
      Best ba, bb;
      run_tiles<kFixP, FMT, DPMAP, 1>(g, empty_tile(), j.dp, j.ld_dp, j.dp_aligned, nullptr, 0, 0,
                                      io, ba, bb, warp_ring());
      const unsigned long long ka = tile_key(ba, j.n);
      if ((threadIdx.x & 31) == 0 && ka) atomicMax(&st->key, ka);
    }
    if (nstrips > j.strips_fix && threadIdx.x == 0) atomicExch(&st->status, (int)MS_ERR_OOM);
    __syncthreads();
    for (int s = threadIdx.x; s < nstrips && s < j.strips_fix; s += blockDim.x) j.progress[s] = 0;
  }
  __syncthreads();
  finalize_job(j);
}

// Size-only fix-up of one matrix by bitplane growth, then its result.
template <int FMT>
__device__ __forceinline__ void fixup_bits_job(const Job& j, uint32_t* smem, int64_t smem_words,
                                               int team_size, int rank, TeamSync* sync,
                                               bool cluster = false) {
  __shared__ int32_t sbox[4];
  if (threadIdx.x == 0) {
    const volatile int32_t* b = j.st->box;
    sbox[0] = b[0];
    sbox[1] = b[1];
    sbox[2] = b[2];
    sbox[3] = b[3];
  }
  __syncthreads();
  if (sbox[1] > sbox[0] && sbox[3] > sbox[2])
    fixup_bits<FMT>(j, sbox[0], sbox[1], sbox[2], sbox[3], smem, smem_words, team_size, rank,
                    sync, cluster);
  if (rank != 0) return;
  __syncthreads();
  finalize_job(j);
}

// One matrix: a team of gridDim.x blocks (`sync` zeroed before the launch when
// there are several); cluster != 0 when the grid is one thread-block cluster.
template <int FMT>
__global__ void __launch_bounds__(1024, 1) k_fixup_bits_one(const Job job, int64_t smem_words,
                                                            TeamSync* sync, int cluster) {
  extern __shared__ __align__(16) unsigned char ms_dyn_smem[];
  grid_dependency_wait();
  fixup_bits_job<FMT>(job, reinterpret_cast<uint32_t*>(ms_dyn_smem), smem_words, (int)gridDim.x,
                      (int)blockIdx.x, sync, cluster != 0);
}

// Batch: one block per (matrix, rank) task, larger teams first (the
// hardware hands blocks to free SMs, which balances the uneven boxes better
// than blocks that loop over several matrices); matrices without bitplane
// scratch go to the strip fix-up.
struct FixTask {
  int32_t job, rank, size, pad;
};
constexpr int kBitsMixedThreads = 512;
static __global__ void __launch_bounds__(kBitsMixedThreads, 2)
    k_fixup_bits_mixed(const Job* __restrict__ jobs, const FixTask* __restrict__ tasks,
                       TeamSync* syncs, int64_t smem_words) {
  extern __shared__ __align__(16) unsigned char ms_dyn_smem[];
  const FixTask t = tasks[blockIdx.x];
  const Job job = jobs[t.job];
  uint32_t* smem = reinterpret_cast<uint32_t*>(ms_dyn_smem);
  if (job.fmt == MS_U8)
    fixup_bits_job<MS_U8>(job, smem, smem_words, t.size, t.rank, syncs + t.job);
  else
    fixup_bits_job<MS_BITS32>(job, smem, smem_words, t.size, t.rank, syncs + t.job);
}

// after_levels: the dp-map level kernels ran just before (their table says
// whether they completed the map).
template <int FMT, bool DPMAP>
__global__ void __launch_bounds__(kFixWarps * 32, 1) k_fixup_one(const Job job, int after_levels) {
  fixup_job<FMT, DPMAP>(job, after_levels != 0);
}

// Every variant fits 128 registers without spills, so two 256-thread blocks
// share an SM.  Single matrix: the job travels as a kernel parameter.
//
// fuse != 0 (small matrices): the last block to finish also finishes the
// matrix -- the fix-up of its box, if any (size-only: bitplane growth from the
// block's ring memory or the job's scratch; dp map: the strip fix-up over the
// block's warps), then the result -- so that one launch does the whole call.
template <int P, int FMT, bool DPMAP>
__global__ void __launch_bounds__(256, 2) k_tiles_one(const Job job, int64_t ntiles, int fuse,
                                                       TeamSync* team) {
  grid_dependents_may_launch();
  clear_team(team);
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  tile_pass_warp<P, FMT, DPMAP>(&job, 1, ntiles, w);
  if (fuse) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // this block's key and box updates before its ticket
      s_last = atomicAdd(&job.st->done, 1) == (int)gridDim.x - 1;
      if (s_last) __threadfence();
    }
    __syncthreads();
    if (s_last) {
      if constexpr (DPMAP) {
        // the strip fix-up over this block's warps and rings, then the result
        fixup_job<FMT, true>(job, false);
      } else {
        extern __shared__ __align__(16) unsigned char ms_dyn_smem[];
        fixup_bits_job<FMT>(job, reinterpret_cast<uint32_t*>(ms_dyn_smem),
                            (int64_t)(blockDim.x >> 5) * kRingWarpBytes / 4, 1, 0, nullptr);
      }
    }
  }
}

// Second pass of the all-largest-squares call: when the largest side K
// (written by the first pass) is at most the halo, every K-square corner is a
// counted cell of some tile with an exact window value; recompute the tiles
// and list those cells.  (Larger K: the box fix-up of the first pass listed
// them.)  Publishes nothing to the matrix state.
template <int P, int FMT>
__global__ void __launch_bounds__(256, 2) k_tiles_emit(const Job job, int64_t ntiles) {
  const int K = *reinterpret_cast<const volatile int32_t*>(&job.out->side);
  if (K <= 0 || K > kHalo) return;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t t_a = 2 * w, t_b = 2 * w + 1;
  if (t_a >= ntiles) return;
  const Tile ga = tile_of(job, t_a);
  const Tile gb = t_b < ntiles ? tile_of(job, t_b) : empty_tile();
  StripIO io{nullptr, nullptr, nullptr, nullptr, nullptr, 0};
  Best ba, bb;
  run_tiles<P, FMT, false, 0, true>(ga, gb, nullptr, 0, 0, nullptr, 0, 0, io, ba, bb,
                                    warp_ring(), &job, (uint32_t)K);
}

static __global__ void k_init_states(JobState* st, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    st[i].key = 0ull;
    st[i].box[0] = 0x7fffffff;
    st[i].box[1] = -1;
    st[i].box[2] = 0x7fffffff;
    st[i].box[3] = -1;
    st[i].status = 0;
    st[i].done = 0;
  }
}

}  // namespace ms
