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
// is at most the halo.  Tiles whose largest value exceeds the halo are
// "flagged" and their union is recorded as a bounding box per matrix.  Tiles
// on the matrix's top or left edge are exact whatever their values, but they
// are flagged all the same: the fix-up below relies on every unflagged cell
// having dp <= halo.
//
// Lanes are skewed by one row: at step s lane l works on window row s - l,
// so what lane l needs from lane l-1 (the row's horizontal run carry Q and
// the diagonal A of the previous row) was produced one step earlier and is
// passed with two shuffles; nothing waits inside a step.
//
// Fix-up.  If a matrix has unresolved tiles, the box [rlo, rhi) x [clo, chi)
// grown by the halo up and left is recomputed exactly as one window: its
// columns are split into strips of 512, one warp per strip, and each strip
// takes the exact horizontal carry of its left neighbour row by row through
// global memory (release/acquire flags, bounded waits).  A square whose
// corner lies in the box and which reached above the grown window would
// contain a square of side > halo ending on the row just above rlo, whose
// tile would then be flagged too (likewise on the left); so every cell of
// the box is exact.
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
  g.wr0 = band == 0 ? 0 : r0 - kHalo;
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

template <int P, int FMT>
__device__ __forceinline__ void load_row(Raw<P, FMT>& r, const Tile& g, int ir, int lane) {
  const int64_t col = g.wc0 + (int64_t)P * lane;
  if (ir < 0 || ir >= g.nrows) {
    if constexpr (FMT == MS_U8) {
#pragma unroll
      for (int i = 0; i < Raw<P, FMT>::W; ++i) r.w[i] = 0;
    } else {
      r.word = 0;
    }
    return;
  }
  const int64_t row = g.wr0 + ir;
  if constexpr (FMT == MS_U8) {
    load_u8<P>(r, g.base + row * g.ld, col, g.n, g.aligned != 0);
  } else {
    load_bits<P>(r, reinterpret_cast<const uint32_t*>(g.base) + row * g.ld, col, g.n);
  }
}

// Left-edge carries of a strip in the fix-up (mode 1).
struct StripIO {
  const uint32_t* carry_in;   // null for the first strip (zero boundary)
  const int32_t* progress_in;
  uint32_t* carry_out;        // null for the last strip
  int32_t* progress_out;
  int32_t* status;
};

template <int P, int FMT, bool DPMAP, int MODE>
__device__ __forceinline__ void run_tiles(const Tile& ta, const Tile& tb, int32_t* dpa,
                                          int64_t lda, int dpa_al, int32_t* dpb, int64_t ldb,
                                          int dpb_al, const StripIO& io, Best& ba, Best& bb) {
  const int lane = threadIdx.x & 31;
  constexpr uint32_t kB2 = kBias * 0x10001u;
  constexpr uint32_t kClamp2 = (kBias - 1) * 0x10001u;
  constexpr int D = 4;  // rows of input prefetched per lane
  const int nmax = max(ta.nrows, tb.nrows);
  const int nsteps = nmax + 31;

  uint32_t Z[P], Ap[P];
#pragma unroll
  for (int k = 0; k < P; ++k) {
    Z[k] = kB2;
    Ap[k] = kB2;
  }
  uint32_t pubQ = 0, pubA = kB2;
  uint32_t carryA_prev = kBias;  // fix-up: A of the left strip's last column, previous row
  bool gave_up = false;
  ba.val = bb.val = 0;
  ba.row = ba.col = bb.row = bb.col = -1;
  const int64_t cola = ta.wc0 + (int64_t)P * lane;
  const int64_t colb = tb.wc0 + (int64_t)P * lane;
  const bool cnt_cola = cola >= ta.c0 && cola < ta.n;
  const bool cnt_colb = colb >= tb.c0 && colb < tb.n;
  const LaneCols lca = lane_cols<P>(cola, ta.n);
  const LaneCols lcb = lane_cols<P>(colb, tb.n);

  Raw<P, FMT> lo[D], hi[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    load_row<P, FMT>(lo[d], ta, d - lane, lane);
    load_row<P, FMT>(hi[d], tb, d - lane, lane);
  }

  for (int s0 = 0; s0 < nsteps; s0 += D) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int s = s0 + d;
      const int ir = s - lane;
      uint32_t qn = __shfl_up_sync(kFull, pubQ, 1);
      uint32_t an = __shfl_up_sync(kFull, pubA, 1);
      const Cells<P, FMT> clo = cells_of<P>(lo[d], lca);
      const Cells<P, FMT> chi = cells_of<P>(hi[d], lcb);
      load_row<P, FMT>(lo[d], ta, ir + D, lane);
      load_row<P, FMT>(hi[d], tb, ir + D, lane);
      if (ir >= 0 && ir < nmax) {
        const uint32_t I = (uint32_t)ir + 1u + kBias;
        const uint32_t I2 = I * 0x10001u;
        if (lane == 0) {
          // left window edge: a zero column (Q = I, A = I - 1 for dp = 0)
          qn = I2;
          an = I2 - 0x10001u;
          if constexpr (MODE == 1) {
            if (io.carry_in) {
              if (!gave_up) {
                int spins = 0;
                while (ld_acquire(io.progress_in) <= ir) {
                  if (++spins > kSpinLimit) {
                    gave_up = true;
                    atomicExch(io.status, (int)MS_ERR_TIMEOUT);
                    break;
                  }
                  __nanosleep(100);
                }
              }
              const uint32_t c = io.carry_in[ir];
              qn = (qn & 0xffff0000u) | (c & 0xffffu);
              an = (an & 0xffff0000u) | carryA_prev;
              carryA_prev = c >> 16;
            }
          }
        }
        qn = vmax2(qn, kClamp2);
        uint32_t Q = qn, Ad = an, rmin = 0xffffffffu;
#pragma unroll
        for (int k = 0; k < P; ++k) {
          const uint32_t msk = pair_mask<P>(clo, chi, k);
          const uint32_t zk = select_bits(Z[k], I2, msk);
          Z[k] = zk;
          Q = select_bits(vadd2(Q, 0xffffffffu), I2, msk);
          const uint32_t an_k = vmax2(vmax2(Ad, zk), Q);
          Ad = Ap[k];
          Ap[k] = an_k;
          rmin = vmin2(rmin, an_k);
        }
        pubQ = Q;
        pubA = Ad;  // A of this lane's last column, previous row

        if constexpr (MODE == 1) {
          if (lane == 31 && io.carry_out) {
            io.carry_out[ir] = (Q & 0xffffu) | (Ap[P - 1] << 16);
            if (((ir + 1) & 31) == 0 || ir + 1 == ta.nrows) {
              __threadfence();
              st_release(io.progress_out, ir + 1);
            }
          }
        }

        // best value and its first position, per tile
        if (cnt_cola && ir >= ta.cnt_ir0 && ir < ta.nrows) {
          const int v = (int)I - (int)(rmin & 0xffffu);
          if (v > ba.val) {
            ba.val = v;
            ba.row = (int32_t)(ta.wr0 + ir);
            const uint32_t target = rmin & 0xffffu;
            int kk = 0;
#pragma unroll
            for (int k = P - 1; k >= 0; --k)
              if ((Ap[k] & 0xffffu) == target) kk = k;
            ba.col = (int32_t)(cola + kk);
          }
        }
        if (cnt_colb && ir >= tb.cnt_ir0 && ir < tb.nrows) {
          const int v = (int)I - (int)(rmin >> 16);
          if (v > bb.val) {
            bb.val = v;
            bb.row = (int32_t)(tb.wr0 + ir);
            const uint32_t target = rmin >> 16;
            int kk = 0;
#pragma unroll
            for (int k = P - 1; k >= 0; --k)
              if ((Ap[k] >> 16) == target) kk = k;
            bb.col = (int32_t)(colb + kk);
          }
        }

        if constexpr (DPMAP) {
          if (cnt_cola && ir >= ta.cnt_ir0 && ir < ta.nrows) {
            int32_t* p = dpa + (ta.wr0 + ir) * lda + cola;
            if (dpa_al && cola + P <= ta.n && (P % 4) == 0) {
#pragma unroll
              for (int k = 0; k < P; k += 4) {
                int4 v;
                v.x = (int)I - (int)(Ap[k] & 0xffffu);
                v.y = (int)I - (int)(Ap[k + 1] & 0xffffu);
                v.z = (int)I - (int)(Ap[k + 2] & 0xffffu);
                v.w = (int)I - (int)(Ap[k + 3] & 0xffffu);
                __stcs(reinterpret_cast<int4*>(p + k), v);
              }
            } else {
#pragma unroll
              for (int k = 0; k < P; ++k)
                if (cola + k < ta.n) p[k] = (int)I - (int)(Ap[k] & 0xffffu);
            }
          }
          if (cnt_colb && ir >= tb.cnt_ir0 && ir < tb.nrows) {
            int32_t* p = dpb + (tb.wr0 + ir) * ldb + colb;
            if (dpb_al && colb + P <= tb.n && (P % 4) == 0) {
#pragma unroll
              for (int k = 0; k < P; k += 4) {
                int4 v;
                v.x = (int)I - (int)(Ap[k] >> 16);
                v.y = (int)I - (int)(Ap[k + 1] >> 16);
                v.z = (int)I - (int)(Ap[k + 2] >> 16);
                v.w = (int)I - (int)(Ap[k + 3] >> 16);
                __stcs(reinterpret_cast<int4*>(p + k), v);
              }
            } else {
#pragma unroll
              for (int k = 0; k < P; ++k)
                if (colb + k < tb.n) p[k] = (int)I - (int)(Ap[k] >> 16);
            }
          }
        }
      }
    }
  }
}

// Reduce a per-lane best to the tile's key; returns the tile's largest value.
__device__ __forceinline__ unsigned long long tile_key(const Best& b, int64_t n) {
  return warp_max_u64(make_key(b.val, b.row, b.col, n));
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
  const Job& B = jobs[jb < 0 ? ja : jb];
  StripIO io{nullptr, nullptr, nullptr, nullptr, nullptr};
  Best ba, bb;
  run_tiles<P, FMT, DPMAP, 0>(ga, gb, A.dp, A.ld_dp, A.dp_aligned, B.dp, B.ld_dp, B.dp_aligned,
                              io, ba, bb);
  const unsigned long long ka = tile_key(ba, ga.n);
  const unsigned long long kb = tile_key(bb, gb.n);
  if ((threadIdx.x & 31) == 0) {
    if (ka) {
      atomicMax(&A.st->key, ka);
      if ((int)(ka >> 40) > kHalo) {
        const int r0 = (int)(ga.wr0 + ga.cnt_ir0);
        atomicMin(&A.st->box[0], r0);
        atomicMax(&A.st->box[1], (int)(ga.wr0 + ga.nrows));
        atomicMin(&A.st->box[2], (int)ga.c0);
        atomicMax(&A.st->box[3], (int)min(ga.n, ga.wc0 + 32 * P));
      }
    }
    if (jb >= 0 && kb) {
      atomicMax(&B.st->key, kb);
      if ((int)(kb >> 40) > kHalo) {
        const int r0 = (int)(gb.wr0 + gb.cnt_ir0);
        atomicMin(&B.st->box[0], r0);
        atomicMax(&B.st->box[1], (int)(gb.wr0 + gb.nrows));
        atomicMin(&B.st->box[2], (int)gb.c0);
        atomicMax(&B.st->box[3], (int)min(gb.n, gb.wc0 + 32 * P));
      }
    }
  }
}

template <int P, int FMT, bool DPMAP>
__global__ void __launch_bounds__(256) k_tiles(const Job* __restrict__ jobs, int njobs,
                                               int64_t ntiles) {
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  tile_pass_warp<P, FMT, DPMAP>(jobs, njobs, ntiles, w);
}

// Single matrix: the job travels as a kernel parameter.
template <int P, int FMT, bool DPMAP>
__global__ void __launch_bounds__(256) k_tiles_one(const Job job, int64_t ntiles) {
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  tile_pass_warp<P, FMT, DPMAP>(&job, 1, ntiles, w);
}

// ---- fix-up and result ------------------------------------------------------

constexpr int kFixWarps = 8;
constexpr int kFixP = 16;
constexpr int kFixW = 32 * kFixP;  // strip width in the fix-up

template <int FMT, bool DPMAP>
__device__ __forceinline__ void fixup_job(const Job& j) {
  __shared__ int32_t sbox[4];
  JobState* st = j.st;
  if (threadIdx.x == 0) {
    sbox[0] = st->box[0];
    sbox[1] = st->box[1];
    sbox[2] = st->box[2];
    sbox[3] = st->box[3];
  }
  __syncthreads();
  const int rlo = sbox[0], rhi = sbox[1], clo = sbox[2], chi = sbox[3];
  if (rhi > rlo && chi > clo) {
    const int64_t br0 = max(0, rlo - kHalo);
    const int64_t bc0 = max(0, clo - kHalo);
    const int nstrips = (int)((chi - bc0 + kFixW - 1) / kFixW);
    const int rows = (int)(rhi - br0);
    const int warp = threadIdx.x >> 5;
    for (int s = warp; s < nstrips && s < j.strips_fix; s += kFixWarps) {
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
      io.carry_in = s > 0 ? j.carry + (int64_t)(s - 1) * j.m : nullptr;
      io.progress_in = s > 0 ? j.progress + (s - 1) : nullptr;
      io.carry_out = (s + 1 < nstrips) ? j.carry + (int64_t)s * j.m : nullptr;
      io.progress_out = j.progress + s;
      io.status = &st->status;
      Best ba, bb;
      run_tiles<kFixP, FMT, DPMAP, 1>(g, empty_tile(), j.dp, j.ld_dp, j.dp_aligned, nullptr, 0, 0,
                                      io, ba, bb);
      const unsigned long long ka = tile_key(ba, j.n);
      if ((threadIdx.x & 31) == 0 && ka) atomicMax(&st->key, ka);
    }
    if (nstrips > j.strips_fix && threadIdx.x == 0) atomicExch(&st->status, (int)MS_ERR_OOM);
    __syncthreads();
    for (int s = threadIdx.x; s < nstrips && s < j.strips_fix; s += blockDim.x) j.progress[s] = 0;
  }
  __syncthreads();
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
  }
}

template <int FMT, bool DPMAP>
__global__ void __launch_bounds__(kFixWarps * 32) k_fixup(const Job* __restrict__ jobs,
                                                          int njobs) {
  const int j = blockIdx.x;
  if (j >= njobs) return;
  const Job job = jobs[j];
  if (job.fmt != FMT) return;
  fixup_job<FMT, DPMAP>(job);
}

template <int FMT, bool DPMAP>
__global__ void __launch_bounds__(kFixWarps * 32) k_fixup_one(const Job job) {
  fixup_job<FMT, DPMAP>(job);
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
    st[i].pad = 0;
  }
}

}  // namespace ms
