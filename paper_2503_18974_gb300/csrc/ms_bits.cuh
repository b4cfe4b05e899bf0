// Bit-packed size-only search: squares grown by AND-ing shifted bitplanes.
//
// S_t is the bitmap of bottom-right corners of all-ones t x t squares, in the
// MS_BITS32 layout (bit b of word w = column 32w+b), with S_1 = the input.
// A (a+b-1)-square is covered by the four a-squares sharing its corners, so
//   S_{a+b-1}(i,j) = S_a(i,j) & S_a(i-b+1,j) & S_a(i,j-b+1) & S_a(i-b+1,j-b+1)
// for 1 <= b <= a+1 (cells outside the matrix read as 0).  The largest square
// side K is the largest t with S_t non-empty; it is found by doubling
// (S_1 -> S_2 -> S_4 -> ... with b = a+1) until S_2a is empty, then by
// binary search inside [a, 2a) with tests S_{a+x} = grow(S_a, x+1).  The
// witness is the first set bit of S_K in row-major order, which is the first
// cell with dp = K (dp >= K exactly on S_K and no dp exceeds K).
//
// One persistent cooperative kernel runs every pass; passes are separated by
// a grid barrier whose waits are bounded.  A pass walks 32-row x 32-word
// blocks of the output; for each block the four shifted 32-row source tiles
// are staged into shared memory by TMA (cp.async.bulk.tensor) through a
// 3-stage pipeline.  Per-buffer block activity maps let late, sparse levels
// skip blocks whose source is empty (S_{a+b-1} is a subset of S_a).
#pragma once
#include <cuda.h>

#include "ms_device.cuh"

namespace ms {
namespace bits {

constexpr int kBR = 32;        // rows per block
constexpr int kBW = 32;        // words per block (1024 columns)
constexpr int kSW = kBW + 8;   // words of a column-shifted tile
constexpr int kStages = 3;
constexpr int kThreads = 256;
constexpr int kMaxPasses = 64;
constexpr int kTileS = kBR * kSW;  // words of one staged tile (all four share one box)
// one stage: two unshifted tiles (rows 0 and -d) and two column-shifted ones
constexpr int kStageWords = 4 * kTileS;
constexpr size_t kSmemBytes = (size_t)kStages * kStageWords * 4 + 256;

struct State {
  unsigned bar_count;
  unsigned bar_gen;
  int32_t err;
  int32_t passes;
  unsigned nonempty[kMaxPasses];
  unsigned long long first;  // min over set bits of S_K of row*n + col
};

struct Args {
  int64_t m, n;
  int64_t wv;       // valid words per row, ceil(n/32)
  int64_t wp;       // row stride of the level buffers, in words
  uint32_t* buf[3];  // [0] unused (the input is read through its tensor map), [1], [2] levels
  uint8_t* act[3];   // block activity of the level buffers ([0] unused: input all active)
  int nbr, nbw;      // blocks per column, per row
  State* st;
  ms_result* out;
};

// ---- PTX helpers -------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Bounded wait for the phase with the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  uint32_t done = 0;
  for (int i = 0; i < kSpinLimit; ++i) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Grid-wide barrier for a cooperative launch, with bounded waits: on timeout
// it records MS_ERR_TIMEOUT and lets the block go on (results then invalid).
__device__ __forceinline__ void grid_barrier(State* st) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = (unsigned)ld_acquire(reinterpret_cast<const int32_t*>(&st->bar_gen));
    __threadfence();
    if (atomicAdd(&st->bar_count, 1u) == gridDim.x - 1) {
      st->bar_count = 0;
      __threadfence();
      st_release(reinterpret_cast<int32_t*>(&st->bar_gen), (int)(gen + 1));
    } else {
      int spins = 0;
      const unsigned long long t0 = global_ns();
      while ((unsigned)ld_acquire(reinterpret_cast<const int32_t*>(&st->bar_gen)) == gen) {
        if (++spins > kSpinLimit || global_ns() - t0 > kWaitLimitNs) {
          atomicExch(&st->err, (int)MS_ERR_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
  }
  __syncthreads();
}

enum PassKind { kGrow = 0, kTest = 1, kWitness = 2 };

struct Stage {
  int blk;      // block index, -1 = end of pass
  int compute;  // 1: source tiles loaded; 0: only clear the output block
};

// One pass over all blocks: out = grow(src, d = b - 1); kGrow also writes the
// level buffer `dst` and its activity map.
__device__ void run_pass(const CUtensorMap* src_map, int src, int dst, int d, int kind, int pass,
                         const Args& A, uint32_t* smem, uint64_t* bars, Stage* stages) {
  const int nblocks = A.nbr * A.nbw;
  const int tid = threadIdx.x;
  const int q = d >> 5, r = d & 31;
  const uint8_t* act_src = src ? A.act[src] : nullptr;
  const uint8_t* act_dst_old = (kind == kGrow) ? A.act[dst] : nullptr;
  __shared__ int next_blk;

  // the producer (thread 0) walks this block's share of blocks in order
  auto wanted = [&](int b, int& comp) -> bool {
    const bool s_on = act_src ? act_src[b] != 0 : true;
    const bool d_on = act_dst_old ? act_dst_old[b] != 0 : false;
    comp = s_on;
    return s_on || d_on;
  };
  auto issue = [&](int slot) {
    // thread 0 only: pick the next wanted block and start its loads
    int b = next_blk, comp = 0;
    while (b < nblocks && !wanted(b, comp)) b += gridDim.x;
    next_blk = b + (int)gridDim.x;
    Stage& sg = stages[slot];
    uint64_t* bar = &bars[slot];
    if (b >= nblocks) {
      sg.blk = -1;
      sg.compute = 0;
      mbar_arrive(bar);
      return;
    }
    sg.blk = b;
    sg.compute = comp;
    if (!comp) {
      mbar_arrive(bar);
      return;
    }
    const int bi = b / A.nbw, bj = b - (b / A.nbw) * A.nbw;
    const int r0 = bi * kBR, w0 = bj * kBW;
    const int xs = ((w0 - q - 1) >> 2) << 2;  // 16-byte aligned start (floor)
    uint32_t* base = smem + slot * kStageWords;
    mbar_expect_tx(bar, (unsigned)(kStageWords * 4));
    tma_load_2d(base, src_map, w0, r0, bar);
    tma_load_2d(base + kTileS, src_map, w0, r0 - d, bar);
    tma_load_2d(base + 2 * kTileS, src_map, xs, r0, bar);
    tma_load_2d(base + 3 * kTileS, src_map, xs, r0 - d, bar);
  };

  if (tid == 0) {
    for (int sidx = 0; sidx < kStages; ++sidx) mbar_init(&bars[sidx], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    next_blk = blockIdx.x;
  }
  __syncthreads();
  if (tid == 0)
    for (int sidx = 0; sidx < kStages; ++sidx) issue(sidx);
  __syncthreads();

  const int lx = tid & 31;   // word within the block
  const int ly = tid >> 5;   // first row; rows ly, ly+8, ly+16, ly+24
  unsigned long long first = ~0ull;
  bool any_local = false;
  for (int it = 0;; ++it) {
    const int slot = it % kStages;
    const unsigned parity = (unsigned)((it / kStages) & 1);
    if (!mbar_wait(&bars[slot], parity)) {
      if (tid == 0) atomicExch(&A.st->err, (int)MS_ERR_TIMEOUT);
    }
    const Stage sg = stages[slot];
    if (sg.blk < 0) break;
    const int bi = sg.blk / A.nbw, bj = sg.blk - (sg.blk / A.nbw) * A.nbw;
    const int r0 = bi * kBR, w0 = bj * kBW;
    const int64_t w = w0 + lx;
    const bool wvalid = w < A.wv;
    // mask of columns < n in this word
    uint32_t cmask = 0u;
    if (wvalid) {
      const int64_t rem = A.n - 32 * w;
      cmask = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    }
    const uint32_t* base = smem + slot * kStageWords;
    const int xs = ((w0 - q - 1) >> 2) << 2;
    const int ks = (w0 + lx - q) - xs;  // index of word (w - q) in a shifted tile, >= 1
    bool blk_any = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int li = ly + 8 * k;
      const int64_t i = r0 + li;
      uint32_t v = 0;
      if (sg.compute) {
        const uint32_t a0 = base[li * kSW + lx];
        const uint32_t a1 = base[kTileS + li * kSW + lx];
        const uint32_t* s0 = base + 2 * kTileS + li * kSW;
        const uint32_t* s1 = base + 3 * kTileS + li * kSW;
        const uint32_t a2 = r ? ((s0[ks] << r) | (s0[ks - 1] >> (32 - r))) : s0[ks];
        const uint32_t a3 = r ? ((s1[ks] << r) | (s1[ks - 1] >> (32 - r))) : s1[ks];
        v = a0 & a1 & a2 & a3 & cmask;
        if (i >= A.m) v = 0;
      }
      if (kind == kGrow && i < A.m && wvalid) A.buf[dst][i * A.wp + w] = v;
      if (v) {
        blk_any = true;
        if (kind == kWitness) {
          // lowest set bit = lowest column of this word; keep the minimum over
          // everything this thread sees (blocks are not visited in cell order)
          const unsigned long long cand = (unsigned long long)i * (unsigned long long)A.n +
                                          (unsigned long long)(32 * w) +
                                          (unsigned long long)(__ffs(v) - 1);
          first = cand < first ? cand : first;
        }
      }
    }
    any_local |= blk_any;
    const int blk_or = __syncthreads_or(blk_any ? 1 : 0);
    if (tid == 0) {
      if (kind == kGrow) A.act[dst][sg.blk] = blk_or ? 1 : 0;
      issue(slot);
    }
    __syncthreads();
  }
  // make this pass's generic-proxy writes visible to the next pass's TMA reads
  asm volatile("fence.proxy.async.global;" ::: "memory");
  if (kind == kWitness) {
#pragma unroll
    for (int dd = 16; dd > 0; dd >>= 1) {
      const unsigned long long o = __shfl_xor_sync(kFull, first, dd);
      first = o < first ? o : first;
    }
    if ((tid & 31) == 0 && first != ~0ull) atomicMin(&A.st->first, first);
  }
  const int cta_any = __syncthreads_or(any_local ? 1 : 0);
  if (tid == 0 && cta_any) atomicOr(&A.st->nonempty[pass], 1u);
}

__global__ void k_bits_reset(State* st) {
  const int i = threadIdx.x;
  if (i < kMaxPasses) st->nonempty[i] = 0u;
  if (i == 0) {
    st->bar_count = 0u;
    st->bar_gen = 0u;
    st->err = 0;
    st->passes = 0;
    st->first = ~0ull;
  }
}

__global__ void __launch_bounds__(kThreads) k_bits_search(const __grid_constant__ CUtensorMap m0,
                                                         const __grid_constant__ CUtensorMap m1,
                                                         const __grid_constant__ CUtensorMap m2,
                                                         const Args A) {
  extern __shared__ __align__(128) unsigned char dsm[];
  uint32_t* smem = reinterpret_cast<uint32_t*>(
      (reinterpret_cast<uintptr_t>(dsm) + 127) & ~(uintptr_t)127);
  __shared__ uint64_t bars[kStages];
  __shared__ Stage stages[kStages];
  const CUtensorMap* maps[3] = {&m0, &m1, &m2};
  const int64_t kmax = A.m < A.n ? A.m : A.n;

  int64_t a = 1;
  int cur = 0, nxt = 1;
  int pass = 0;
  int64_t lo, hi;
  // doubling: S_a -> S_2a while non-empty
  for (;;) {
    if (2 * a > kmax || pass >= kMaxPasses - 24) {
      lo = a;
      hi = (2 * a > kmax) ? kmax + 1 : 2 * a;
      break;
    }
    run_pass(maps[cur], cur, nxt, (int)a, kGrow, pass, A, smem, bars, stages);
    grid_barrier(A.st);
    const bool ne = ld_acquire(reinterpret_cast<const int32_t*>(&A.st->nonempty[pass])) != 0;
    ++pass;
    if (!ne) {
      lo = a;
      hi = 2 * a;
      break;
    }
    a *= 2;
    const int old = cur;
    cur = nxt;
    nxt = (old == 0) ? 2 : old;
  }
  // binary search for the largest t in [lo, hi) with S_t non-empty (S_lo is)
  while (hi - lo > 1 && pass < kMaxPasses - 1) {
    const int64_t t = (lo + hi) / 2;
    run_pass(maps[cur], cur, 0, (int)(t - a), kTest, pass, A, smem, bars, stages);
    grid_barrier(A.st);
    const bool ne = ld_acquire(reinterpret_cast<const int32_t*>(&A.st->nonempty[pass])) != 0;
    ++pass;
    if (ne) lo = t; else hi = t;
  }
  // witness: first set bit of S_lo (lo = 1 with an empty input means K = 0)
  run_pass(maps[cur], cur, 0, (int)(lo - a), kWitness, pass, A, smem, bars, stages);
  grid_barrier(A.st);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long f = *reinterpret_cast<volatile unsigned long long*>(&A.st->first);
    ms_result res;
    res.status = *reinterpret_cast<volatile int32_t*>(&A.st->err);
    if (f == ~0ull || A.m == 0 || A.n == 0) {
      res.side = 0;
      res.row = -1;
      res.col = -1;
    } else {
      res.side = (int32_t)lo;
      res.row = (int32_t)(f / (unsigned long long)A.n);
      res.col = (int32_t)(f % (unsigned long long)A.n);
    }
    *A.out = res;
    A.st->passes = pass + 1;
  }
}

}  // namespace bits
}  // namespace ms
