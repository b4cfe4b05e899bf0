// Batch matrices small enough for two bitplanes of the whole matrix in one
// block's shared memory.  The matrix is read once into S_1 (32 cells per
// word) and its largest square and first corner are found on the planes by
// doubling and search (squares grown from smaller ones: four t-squares at the
// corners of a (t+s)-square cover it for s <= t, Sec. 3.4 restated on bits),
// exactly: no tiles, no halo, no fix-up.  A persistent launch whose blocks
// take matrices from a queue, largest first.
#pragma once
#include "ms_bitile.cuh"
#include "ms_kernels.cuh"

namespace ms {
namespace small {

// Words of one plane of an m x n matrix (rows at an odd pitch), rounded up
// to 16 bytes so that the second plane, which also stages the input rows for
// 16-byte asynchronous copies, starts 16-byte aligned.
__host__ __device__ __forceinline__ int64_t plane_words(int64_t m, int64_t n) {
  return (m * (int64_t)sbox::odd_pitch((int)((n + 31) / 32)) + 3) / 4 * 4;
}

// S_1 (the input as bits) of the whole matrix into `a`; returns its plane
// with the active box of its set bits.  Threads take the words in row-major
// order (coalesced reads), each issuing kBatch reads before using them.
template <int FMT>
__device__ __forceinline__ sbox::SP load_s1(const Job& j, uint32_t* a, int (*part)[4]) {
  constexpr int kBatch = 4;
  const int rows = (int)j.m, W = (int)((j.n + 31) / 32), P = sbox::odd_pitch(W);
  int rmin = 0x7fffffff, rmax = -1, wmin = 0x7fffffff, wmax = -1;
  const int bd = (int)blockDim.x, dr = bd / W, dc = bd - dr * W;
  int r = (int)threadIdx.x / W, c = (int)threadIdx.x - r * W;
  while (r < rows) {
    int rk[kBatch], ck[kBatch];
    uint32_t v[kBatch];
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      rk[k] = r;
      ck[k] = c;
      v[k] = r < rows ? input_word<FMT>(j, r, c) : 0u;
      r += dr;
      c += dc;
      if (c >= W) {
        c -= W;
        ++r;
      }
    }
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      if (rk[k] < rows) {
        a[rk[k] * P + ck[k]] = v[k];
        if (v[k]) {
          rmin = min(rmin, rk[k]);
          rmax = max(rmax, rk[k]);
          wmin = min(wmin, ck[k]);
          wmax = max(wmax, ck[k]);
        }
      }
    }
  }
  int box[4];
  sbox::fold_box(rmin, rmax, wmin, wmax, part, box);
  return sbox::SP{a, 0, 0, P, W, rows, box[0], box[1], box[2], box[3]};
}

// S_1 of a 16-byte aligned uint8 matrix whose rows are staged into shared
// memory first: `stage` is a ring of NS slots, each holding a chunk of whole
// rows; asynchronous 16-byte copies (zero-filled past column n) keep NS - 1
// chunks in flight while the block packs the oldest one, so that most of the
// stage is always on its way from memory (the load is latency-bound: the
// copies in flight, not the packing, set its pace).
template <int NS>
__device__ __forceinline__ sbox::SP load_s1_ring(const Job& j, uint32_t* a, uint32_t sbase,
                                                 int slot, int (*part)[4]) {
  const int rows = (int)j.m, W = (int)((j.n + 31) / 32), P = sbox::odd_pitch(W);
  const int rb = 32 * W;  // staged bytes per row: whole words, zeros past column n
  const int rc = slot / rb, nch = (rows + rc - 1) / rc, pieces = 2 * W;
  const uint8_t* src = reinterpret_cast<const uint8_t*>(j.data);
  const int bd = (int)blockDim.x;
  // the thread's first piece (row, 16-byte piece) and first word (row, word)
  // of a chunk, and the steps between its next ones (no divisions per item)
  const int pr0 = (int)threadIdx.x / pieces, pq0 = (int)threadIdx.x - pr0 * pieces;
  const int pdr = bd / pieces, pdq = bd - pdr * pieces;
  const int wr0 = (int)threadIdx.x / W, ww0 = (int)threadIdx.x - wr0 * W;
  const int wdr = bd / W, wdw = bd - wdr * W;
  auto issue = [&](int ch) {
    if (ch < nch) {
      const int r0 = ch * rc, nr = min(rc, rows - r0);
      const uint32_t dst = sbase + (uint32_t)((ch % NS) * slot);
      int r = pr0, q = pq0;
      while (r < nr) {
        const int64_t col = 16 * (int64_t)q;
        const int valid = (int)max((int64_t)0, min((int64_t)16, j.n - col));
        const uint8_t* sp = valid ? src + (int64_t)(r0 + r) * j.ld + col : src;
        cp_async(dst + (uint32_t)(r * rb + 16 * q), sp, 16, valid);
        r += pdr;
        q += pdq;
        if (q >= pieces) {
          q -= pieces;
          ++r;
        }
      }
    }
    cp_async_commit();  // (an empty group past the last chunk)
  };
  int rmin = 0x7fffffff, rmax = -1, wmin = 0x7fffffff, wmax = -1;
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) issue(k);
  for (int ch = 0; ch < nch; ++ch) {
    // the slot packed last round (every thread is past it) takes chunk ch + NS - 1
    issue(ch + NS - 1);
    cp_async_wait<NS - 1>();
    __syncthreads();  // chunk ch is in shared memory for every thread
    const int r0 = ch * rc, nr = min(rc, rows - r0);
    const uint32_t sb = sbase + (uint32_t)((ch % NS) * slot);
    int r = wr0, w = ww0;
    while (r < nr) {
      const uint32_t ad = sb + (uint32_t)(r * rb + 32 * w);
      uint32_t v[8];
      asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "r"(ad) : "memory");
      asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]) : "r"(ad + 16u) : "memory");
      uint32_t x;
      if (((v[0] | v[1] | v[2] | v[3] | v[4] | v[5] | v[6] | v[7]) & 0xfefefefeu) == 0u) {
        x = bt::pack01(v);
      } else {  // some byte above one: any nonzero byte is a one
        x = 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) x |= byte_flags4(v[k]) << (4 * k);
      }
      a[(r0 + r) * P + w] = x;
      if (x) {
        rmin = min(rmin, r0 + r);
        rmax = max(rmax, r0 + r);
        wmin = min(wmin, w);
        wmax = max(wmax, w);
      }
      r += wdr;
      w += wdw;
      if (w >= W) {
        w -= W;
        ++r;
      }
    }
    __syncthreads();  // the slot is refilled by the copies issued next round
  }
  cp_async_wait<0>();  // (only empty groups remain)
  int box[4];
  sbox::fold_box(rmin, rmax, wmin, wmax, part, box);
  return sbox::SP{a, 0, 0, P, W, rows, box[0], box[1], box[2], box[3]};
}

// The staged load with as many ring slots (8, 4 or 2) as `stage_bytes` holds
// rows for; returns false (nothing done) when one staged row exceeds half of
// it, or the matrix or the stage is not 16-byte aligned.
__device__ __forceinline__ bool load_s1_staged(const Job& j, uint32_t* a, uint32_t* stage,
                                               int64_t stage_bytes, int (*part)[4],
                                               sbox::SP& out) {
  const int rb = 32 * (int)((j.n + 31) / 32);
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(stage);
  // (16-byte copies: the stage, the rows of the input and the row stride
  // must all be 16-byte aligned)
  if (!j.aligned || (sbase & 15u) != 0) return false;
  const int64_t s8 = (stage_bytes / 8) & ~(int64_t)15, s4 = (stage_bytes / 4) & ~(int64_t)15,
                s2 = (stage_bytes / 2) & ~(int64_t)15;
  if (rb <= s8)
    out = load_s1_ring<8>(j, a, sbase, (int)s8, part);
  else if (rb <= s4)
    out = load_s1_ring<4>(j, a, sbase, (int)s4, part);
  else if (rb <= s2)
    out = load_s1_ring<2>(j, a, sbase, (int)s2, part);
  else
    return false;
  return true;
}

// One matrix by the whole block, in `smem_words` words of shared memory (at
// least two planes); writes its result.
__device__ __forceinline__ void solve_matrix(const Job& j, uint32_t* smem, int64_t smem_words,
                                             int (*part)[32][4]) {
  if (j.m <= 0 || j.n <= 0) {
    if (threadIdx.x == 0) *j.out = ms_result{0, -1, -1, 0};
    return;
  }
  const int64_t pw = plane_words(j.m, j.n);
  uint32_t* A = smem;
  uint32_t* B = smem + pw;
  // (B and the rest of the block's shared memory are free until the first
  // level is built: they stage the input rows)
  sbox::SP s1;
  if (j.fmt != MS_U8)
    s1 = load_s1<MS_BITS32>(j, A, part[0]);
  else if (!load_s1_staged(j, A, B, 4 * (smem_words - pw), part[0], s1))
    s1 = load_s1<MS_U8>(j, A, part[0]);
  // levels alternate between B and A (S_1's buffer is free once S_2 exists)
  const sbox::Found f =
      sbox::solve(j, s1, 1, B, A, 0, (int)j.m, 0, (int)((j.n + 31) / 32), part, 1);
  if (threadIdx.x == 0) {
    ms_result r{0, -1, -1, 0};
    if (f.side > 0) {
      r.side = f.side;
      r.row = (int32_t)(f.idx / (unsigned long long)j.n);
      r.col = (int32_t)(f.idx % (unsigned long long)j.n);
    }
    *j.out = r;
  }
}

}  // namespace small

// Persistent launch over `count` small matrices (jobs[order[k]], k taken from
// the queue counter, which starts at zero): each fits two planes in the
// block's dynamic shared memory.
//
// Launched per size class with blocks of 64 to 1024 threads (every variant
// fits 64 registers a thread, so the SM holds 1024 of its threads: sixteen
// blocks of the tiniest matrices at once, or one block of the largest).  The
// part of a block's shared memory beyond the two planes stages input rows.
static __global__ void __launch_bounds__(1024, 1)
    k_batch_small(const Job* __restrict__ jobs, const int32_t* __restrict__ order, int count,
                  int* queue) {
  extern __shared__ __align__(16) unsigned char ms_dyn_smem[];
  __shared__ int s_next;
  __shared__ int s_part[2][32][4];
  uint32_t* smem = reinterpret_cast<uint32_t*>(ms_dyn_smem);
  uint32_t dyn_bytes;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
  for (;;) {
    __syncthreads();  // the previous matrix and s_next are done with
    if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
    __syncthreads();
    const int t = s_next;
    if (t >= count) return;
    const Job j = jobs[order[t]];
    small::solve_matrix(j, smem, (int64_t)(dyn_bytes / 4), s_part);
  }
}

}  // namespace ms
