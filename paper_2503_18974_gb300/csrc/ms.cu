// libms host side: argument checks, workspace, launch planning and the C ABI
// declared in include/ms.h.  Device code lives in ms_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <cstdlib>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "ms_bitile.cuh"
#include "ms_bits.cuh"
#include "ms_kernels.cuh"
#include "ms_small.cuh"

using ms::Job;
using ms::JobState;

// size classes of the batch's small matrices (solved whole, one block each)
constexpr int kClasses = 5;

struct ms_ctx {
  int device = 0;
  int sms = 1;        // streaming multiprocessors of the device
  int bit_slots = 0;  // bitplane tile warps resident at once on the device
  size_t small_smem[kClasses] = {};  // dynamic shared memory of a small-matrix block, by class
  size_t budget = 0;  // 0 = unlimited
  size_t held = 0;    // bytes of device workspace currently held
  ms_tuning tuning{};

  JobState* d_states = nullptr;
  int64_t states_cap = 0;
  uint32_t* d_carry = nullptr;
  int64_t carry_cap = 0;  // in uint32
  int32_t* d_progress = nullptr;
  int64_t progress_cap = 0;
  uint32_t* d_bitfix = nullptr;  // bitplanes of the size-only fix-up
  int32_t* d_first33 = nullptr;  // bitplane tiles: first S_33 row per tile
  int64_t first33_cap = 0;
  int64_t bitfix_cap = 0;        // uint32 words
  ms::TeamSync* d_sync1 = nullptr;  // barrier of a single matrix's fix-up team
  // streams for the small matrices of a batch, one per size class, forked
  // from and joined back into the caller's stream with events
  static constexpr int kSides = kClasses;
  cudaStream_t side[kSides] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kSides] = {};

  // batch job table: device copy, the host image it was uploaded from, and a
  // pinned staging buffer guarded by an event
  unsigned char* d_table = nullptr;  // [jobs | tasks | queue counter]
  int64_t table_cap = 0;             // bytes
  std::vector<unsigned char> uploaded;
  unsigned char* h_stage = nullptr;
  int64_t stage_cap = 0;
  int batch_grid = 0;
  cudaEvent_t stage_free = nullptr;
  bool stage_pending = false;

  // bit-packed search workspace: two level buffers, their block activity maps
  // and the search state; geometry of the last search (buffers hold zeros
  // outside the blocks their maps mark active, for that geometry)
  uint32_t* d_lvl = nullptr;
  int64_t lvl_cap = 0;  // uint32 words, both buffers
  uint8_t* d_act = nullptr;
  int64_t act_cap = 0;
  ms::bits::State* d_bst = nullptr;
  int64_t bst_cap = 0;
  int64_t bits_geom[3] = {-1, -1, -1};  // m, wp, nbw
  int bits_grid = 0;

  // autotuned choices by workload class (see ms_autotune)
  std::map<uint64_t, ms_tuning> tuned;

  // kernel timing (ms_profile_start / ms_profile_stop)
  struct ProfSlot {
    int kind;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  int prof_max = 0;
  int prof_used = 0;
  std::vector<ProfSlot> prof_pool;
  int64_t prof_count[3] = {0, 0, 0};
  int64_t prof_untimed = 0;
  int64_t prof_bit = 0;  // tile launches that were bitplane tiles
};

namespace {

constexpr int kTileThreads = 256;
enum { kProfTile = 0, kProfFixup = 1, kProfOther = 2 };

// Records an event pair around the launches in its scope while profiling is on.
struct ProfScope {
  ms_ctx* c;
  cudaStream_t s;
  int slot = -1;
  ProfScope(ms_ctx* ctx, cudaStream_t st, int kind) : c(ctx), s(st) {
    if (!c || !c->prof_on) return;
    c->prof_count[kind]++;
    if (c->prof_used >= c->prof_max) {
      c->prof_untimed++;
      return;
    }
    if ((int)c->prof_pool.size() <= c->prof_used) {
      ms_ctx::ProfSlot ps{kind, nullptr, nullptr};
      if (cudaEventCreate(&ps.a) != cudaSuccess || cudaEventCreate(&ps.b) != cudaSuccess) {
        cudaGetLastError();
        c->prof_untimed++;
        return;
      }
      c->prof_pool.push_back(ps);
    }
    slot = c->prof_used++;
    c->prof_pool[slot].kind = kind;
    cudaEventRecord(c->prof_pool[slot].a, s);
  }
  ~ProfScope() {
    if (slot >= 0) cudaEventRecord(c->prof_pool[slot].b, s);
  }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Dynamic shared memory of a tile kernel launch: one input ring per warp.
size_t ring_bytes(int threads) { return (size_t)(threads / 32) * ms::kRingWarpBytes; }

// Raise a kernel's dynamic shared memory limit once per device (the rings
// exceed 48 KB; the attribute belongs to the current device's context).
cudaError_t allow_smem(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaGetLastError();
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(fn, dev);
  auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done[key] = bytes;
  return e;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

int64_t strips_for(int64_t n, int P) {
  const int64_t W = 32 * P;
  if (n <= W) return 1;
  return 1 + (n - W + (W - ms::kHalo) - 1) / (W - ms::kHalo);
}

int64_t fix_strips_for(int64_t n) { return (n + ms::kHalo + ms::kFixW - 1) / ms::kFixW + 1; }

// Rows a tile counts.  A warp walks band_rows + 32 (halo) + 31 (lane skew)
// steps, so tall bands amortise the halo while short bands give more warps.
// Aim for about one wave of resident warps (16 per SM, two tiles each) per
// launch, with bands of at least 32 rows.
int64_t auto_band_rows_for(int64_t work_rows /* sum of m * strips */) {
  const int64_t target_tiles = 152 * 16 * 2;
  int64_t br = (work_rows + target_tiles - 1) / target_tiles;
  br = ((br + 31) / 32) * 32;
  br = std::max<int64_t>(br, 32);
  br = std::min<int64_t>(br, 4096);
  return br;
}

int auto_band_rows(int64_t m, int64_t strips) {
  return (int)std::min<int64_t>(auto_band_rows_for(m * strips), std::max<int64_t>(m, 1));
}

// Estimated cycles of one matrix's tile pass with P columns per lane: the
// steps of a tile (band + 32 halo rows + 31 lane-skew steps) times the cycles
// of one step, which is one warp's latency (about 3 cycles per instruction)
// while few warps share a scheduler and the issue time of all of them when
// many do.  Instructions per warp step: a fixed part (input staging, carries,
// bookkeeping) plus the cells; constants from profiles of this kernel.
double tile_cost(int64_t m, int64_t n, int P, int sms) {
  const int64_t strips = strips_for(n, P);
  const int64_t br = auto_band_rows(m, strips);
  const int64_t bands = (m + br - 1) / br;
  const double warps = (double)((bands * strips + 1) / 2);
  const double waves = std::ceil(warps / (16.0 * sms));  // two 8-warp blocks per SM
  const double per_sched = std::min(4.0, warps / waves / (4.0 * sms));
  const double ipstep = 90.0 + 8.5 * P;
  const double cyc = std::max(3.0 * ipstep, per_sched * ipstep / 0.9);
  return waves * (double)(br + 63) * cyc;
}

// Columns per lane.  Narrow matrices take the narrowest tile covering them;
// the others, alone, the width with the lowest estimated cost (small ones are
// latency-bound and want short steps and many tiles, very large ones want
// few instructions and halo columns per cell).  The dp map stays at 16 or
// below (its stores keep more values live).  A 32-column tile has no room
// for a second strip, so lane width 1 only serves n <= 32.
int choose_P(int64_t m, int64_t n, bool dp, int32_t forced, int max_P, int sms) {
  // sms == 0: a batch, where many matrices share one launch and the widest
  // tile (fewest instructions per cell) is best
  if (forced > 1 || (forced == 1 && n <= 32)) return std::min(forced, max_P);
  if (forced == 1) return 2;
  if (n <= 32) return 1;
  const int top = std::min(dp ? 16 : 32, max_P);
  if (sms == 0) {
    if (n <= 64) return 2;
    if (n <= 128) return 4;
    if (n <= 256) return 8;
    return std::min(16, top);
  }
  int cover = 2;  // the narrowest tile covering the matrix, at most the default
  while (cover < 16 && 32 * cover < n) cover *= 2;
  int best = std::min(cover, top);
  double best_cost = tile_cost(m, n, best, sms);
  for (int P = 2; P <= top; P *= 2) {
    const double c = tile_cost(m, n, P, sms);
    if (c < best_cost * 0.97) {  // prefer the default width on near ties
      best = P;
      best_cost = c;
    }
  }
  return best;
}

// Workload class for the autotune cache: entry point (single / batch),
// format mix, log2 of the total cell count and of the matrix count.
uint64_t tune_class(const ms_matrix* ins, int64_t count, bool batch) {
  int64_t cells = 0;
  int fmts = 0;
  for (int64_t i = 0; i < count; ++i) {
    cells += ins[i].m * ins[i].n;
    fmts |= 1 << (ins[i].fmt & 1);
  }
  int lc = 0, lk = 0;
  while ((1ll << lc) < cells && lc < 62) ++lc;
  while ((1ll << lk) < count && lk < 62) ++lk;
  return ((uint64_t)(batch ? 1 : 0) << 60) | ((uint64_t)fmts << 56) | ((uint64_t)lc << 8) |
         (uint64_t)lk;
}

// The tuning a call uses: an explicit band_rows or lane_cols from
// ms_set_tuning wins, else a
// cached autotune result for the class, else the context's tuning (automatic).
ms_tuning effective_tuning(const ms_ctx* ctx, const ms_matrix* ins, int64_t count, bool batch) {
  if (ctx->tuning.band_rows > 0 || ctx->tuning.lane_cols > 0 || ctx->tuning.tile_kind > 0 ||
      ctx->tuned.empty())
    return ctx->tuning;
  auto it = ctx->tuned.find(tune_class(ins, count, batch));
  return it == ctx->tuned.end() ? ctx->tuning : it->second;
}

ms_status check_matrix(const ms_matrix* in) {
  if (!in) return MS_ERR_INVALID;
  if (in->m < 0 || in->n < 0) return MS_ERR_INVALID;
  if (in->fmt != MS_U8 && in->fmt != MS_BITS32) return MS_ERR_INVALID;
  if (in->reserved != 0) return MS_ERR_INVALID;
  if (in->m == 0 || in->n == 0) return MS_OK;
  if (!in->data) return MS_ERR_INVALID;
  const int64_t row_elems = in->fmt == MS_U8 ? in->n : (in->n + 31) / 32;
  if (in->ld < row_elems) return MS_ERR_INVALID;
  if (in->fmt == MS_BITS32 && (reinterpret_cast<uintptr_t>(in->data) & 3u)) return MS_ERR_INVALID;
  if (in->m > 65000) return MS_ERR_UNSUPPORTED;
  if (std::min(in->m, in->n) > 32768) return MS_ERR_UNSUPPORTED;
  if (in->n > ((int64_t)1 << 40) / in->m) return MS_ERR_UNSUPPORTED;
  // column indices of boxes and tiles are 32-bit
  if (in->n > ((int64_t)1 << 31) - 4096) return MS_ERR_UNSUPPORTED;
  return MS_OK;
}

// Band height of bitplane tiles: one tile per warp, and at most as many
// tiles as the GPU holds warps at once (`slots`), so that no tile waits for
// a second wave; bands as even as the rows allow, and at least the halo's
// height.
int bit_band_rows(int64_t m, int64_t strips, int slots) {
  const int64_t bands = std::max<int64_t>(1, slots / std::max<int64_t>(strips, 1));
  const int64_t br = std::max<int64_t>(ms::kHalo, std::min<int64_t>(16384, (m + bands - 1) / bands));
  return (int)std::max<int64_t>(1, std::min<int64_t>(br, m));
}

// Single size-only calls use bitplane tiles when the tuning leaves the
// choice open (an explicit lane width asks for the dp recurrence) and the
// matrix fills the GPU's resident tile warps with bands of at least 64 rows:
// a bitplane tile's rows cost few instructions but a long dependency chain,
// so smaller matrices (short bands, half their rows halo, few warps) are
// latency-bound and faster on the dp recurrence, which overlaps two tiles.
bool use_bit_tiles(const ms_tuning& t, const ms_matrix* in, int bit_slots) {
  if (t.tile_kind != 0) return t.tile_kind == 2;
  if (t.lane_cols > 0 || in->m <= 0 || in->n <= 0) return false;
  const int64_t strips = strips_for(in->n, 32);
  const int64_t bands = std::max<int64_t>(1, bit_slots / strips);
  return (in->m + bands - 1) / bands >= 64;
}

// bit_slots > 0: bitplane tiles, that many resident tile warps.
Job plan_job(const ms_tuning& tune, const ms_matrix* in, bool dp, int max_P, int sms,
             int bit_slots = 0) {
  const bool bit_tiles = bit_slots > 0;
  Job j;
  std::memset(&j, 0, sizeof(j));
  j.data = in->data;
  j.m = in->m;
  j.n = in->n;
  j.ld = in->ld;
  j.fmt = in->fmt;
  j.P = bit_tiles ? 32 : choose_P(in->m, in->n, dp, tune.lane_cols, max_P, sms);
  j.tile_kind = bit_tiles ? 1 : 0;
  if (in->m > 0 && in->n > 0) {
    j.strips = (int32_t)strips_for(in->n, j.P);
    j.band_rows = tune.band_rows > 0 ? (int32_t)std::min<int64_t>(tune.band_rows, in->m)
                  : bit_tiles        ? bit_band_rows(in->m, j.strips, bit_slots)
                                     : auto_band_rows(in->m, j.strips);
    j.bands = (int32_t)((in->m + j.band_rows - 1) / j.band_rows);
  }
  j.aligned = (in->fmt == MS_U8) && (reinterpret_cast<uintptr_t>(in->data) % 16 == 0) &&
              (in->ld % 16 == 0);
  j.strips_fix = (int32_t)fix_strips_for(in->n);
  j.test_hold = tune.test_hold_carries ? 1 : 0;
  return j;
}

int64_t tiles_of(const Job& j) { return (int64_t)j.bands * j.strips; }

// Blocks sharing one matrix's bitplane fix-up: the box is unknown before the
// tile pass, so size the team by the matrix (a block per 2^23 cells for a
// single call, per 2^18 cells in a batch, where blocks are smaller and many
// matrices share the GPU), at most `cap`.
int fix_team_size(int64_t cells, int cap, int shift = 23) {
  const int64_t t = (cells + ((int64_t)1 << shift) - 1) >> shift;
  return (int)std::max<int64_t>(1, std::min<int64_t>(t, cap));
}

// Words of bitplane scratch the size-only fix-up of a matrix may need (three
// planes over at most the whole matrix), and the pool cap beyond which
// matrices fall back to the strip fix-up.
int64_t bitfix_words(const Job& j) { return j.m > 0 && j.n > 0 ? 3 * j.m * ((j.n + 31) / 32 + 2) : 0; }
constexpr int64_t kBitfixCapWords = (int64_t)1 << 30;  // 4 GiB
constexpr size_t kBitsFixSmemBytes = 200 * 1024;         // planes of small boxes
// Batch matrices solved whole in one block, by size class: two planes of at
// most `words` words each, blocks of `threads` threads, `per_sm` blocks per
// SM (the kernel keeps 1024 of its threads on an SM).
struct SmallClass {
  int64_t words;
  int threads, per_sm;
};
constexpr SmallClass kSmall[kClasses] = {{512, 64, 16}, {2048, 128, 8},     // 16 KB
                                         {6144, 256, 4},     // 48 KB
                                         {14320, 512, 2},    // 112 KB (two blocks fit 228 KB)
                                         {28672, 1024, 1}};  // 224 KB
constexpr int kFixClusterBlocks = 8;  // a single large matrix's fix-up cluster (portable size)



// Launch configuration of a fix-up right after its tile pass: `team` blocks
// of 1024 threads with `smem` bytes of dynamic shared memory each, one
// thread-block cluster when team > 1, launched as a programmatic dependent
// of the tile kernel before it on the stream (its blocks wait for that grid
// with griddepcontrol.wait, so the launch overlaps the tile pass's tail).
// The context's team barrier state must have been cleared before the tile
// pass (stream-ordered).
void fixup_config(int team, size_t smem, cudaStream_t s, cudaLaunchConfig_t& cfg,
                  cudaLaunchAttribute (&attr)[2]) {
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = dim3((unsigned)team);
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0] = cudaLaunchAttribute{};
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1] = cudaLaunchAttribute{};
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = (unsigned)team;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = team > 1 ? 2 : 1;
}

ms_status cuda_status(cudaError_t e) { return e == cudaSuccess ? MS_OK : MS_ERR_CUDA; }

template <typename T>
void release(ms_ctx* ctx, T*& p, int64_t& cap) {
  if (p) {
    cudaFree(p);
    ctx->held -= (size_t)cap * sizeof(T);
  }
  p = nullptr;
  cap = 0;
}

template <typename T>
ms_status grow(ms_ctx* ctx, T*& p, int64_t& cap, int64_t need, bool capture) {
  if (need <= cap) return MS_OK;
  if (capture) return MS_ERR_UNSUPPORTED;  // never allocate inside a stream capture
  int64_t want = std::max<int64_t>(need, cap + cap / 2);
  const size_t extra = (size_t)(want - cap) * sizeof(T);
  if (ctx->budget && ctx->held + extra > ctx->budget) {
    want = need;
    if (ctx->held + (size_t)(want - cap) * sizeof(T) > ctx->budget) return MS_ERR_OOM;
  }
  cudaDeviceSynchronize();  // the old buffer may still be in use
  release(ctx, p, cap);
  T* q = nullptr;
  if (cudaMalloc(&q, (size_t)want * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return MS_ERR_OOM;
  }
  p = q;
  cap = want;
  ctx->held += (size_t)want * sizeof(T);
  return MS_OK;
}

// Device state for `njobs` matrices whose fix-up needs `carry` words and
// `progress` counters in total.
ms_status ensure_workspace(ms_ctx* ctx, int64_t njobs, int64_t carry, int64_t progress,
                           cudaStream_t s) {
  const bool cap = capturing(s);
  const int64_t old_states = ctx->states_cap;
  ms_status st = grow(ctx, ctx->d_states, ctx->states_cap, std::max<int64_t>(njobs, 1), cap);
  if (st != MS_OK) return st;
  if (ctx->states_cap != old_states) {
    const int n = (int)ctx->states_cap;
    ms::k_init_states<<<(n + 255) / 256, 256>>>(ctx->d_states, n);
    if (cudaGetLastError() != cudaSuccess) return MS_ERR_CUDA;
  }
  st = grow(ctx, ctx->d_carry, ctx->carry_cap, std::max<int64_t>(carry, 1), cap);
  if (st != MS_OK) return st;
  const int64_t old_prog = ctx->progress_cap;
  st = grow(ctx, ctx->d_progress, ctx->progress_cap, std::max<int64_t>(progress, 1), cap);
  if (st != MS_OK) return st;
  if (ctx->progress_cap != old_prog) {
    if (cudaMemset(ctx->d_progress, 0, (size_t)ctx->progress_cap * sizeof(int32_t)) != cudaSuccess)
      return MS_ERR_CUDA;
  }
  if (!cap && (ctx->states_cap != old_states || ctx->progress_cap != old_prog)) {
    if (cudaDeviceSynchronize() != cudaSuccess) return MS_ERR_CUDA;
  }
  return MS_OK;
}

// ---- launches --------------------------------------------------------------

// Calls on matrices below this many cells finish inside the tile launch (its
// last block runs the fix-up and writes the result): one launch per call,
// where separate fix-up launches would cost more than the work.  The dp
// map's in-block fix-up is the sequential strip one, hence the lower limit.
constexpr int64_t kFusedFinishCells = (int64_t)1 << 24;
constexpr int64_t kFusedFinishCellsDp = (int64_t)1 << 20;

template <int FMT, bool DPMAP>
cudaError_t launch_one_fmt(ms_ctx* ctx, const Job& j, cudaStream_t s) {
  const int64_t ntiles = tiles_of(j);
  const int fuse = ntiles > 0 && ((!DPMAP && j.bits_scratch && j.m * j.n < kFusedFinishCells) ||
                                   (DPMAP && !j.test_hold && j.m * j.n < kFusedFinishCellsDp))
                       ? 1 : 0;
  // a fix-up cluster after the tile pass: the tile kernel clears its team
  // state, so that the fix-up follows it directly on the stream
  const int team = fix_team_size(j.m * j.n, std::min(kFixClusterBlocks, ctx->sms));
  ms::TeamSync* clear = (!fuse && team > 1 && j.bits_scratch) ? ctx->d_sync1 : nullptr;
  if (ntiles > 0 && !DPMAP && j.tile_kind == 1) {
    // bitplane tiles: one tile per warp
    ProfScope ps(ctx, s, kProfTile);
    if (ctx->prof_on) ctx->prof_bit++;
    const int wpb = (int)std::min<int64_t>(ms::bt::kWarps, (ntiles + ctx->sms - 1) / ctx->sms);
    const unsigned grid = (unsigned)((ntiles + wpb - 1) / wpb);
    const size_t sm = (size_t)wpb * ms::bt::kWarpBytes;
    // aligned byte rows that end in a partial 16-byte chunk take the variant
    // whose copies read a partial chunk asynchronously
    const bool ragged = FMT == MS_U8 && j.aligned && j.n % 16 != 0;
    void (*kern)(const ms::Job, int64_t, ms::TeamSync*) =
        fuse ? (ragged ? ms::k_bitiles_one<FMT, true, FMT == MS_U8>
                       : ms::k_bitiles_one<FMT, true, false>)
             : (ragged ? ms::k_bitiles_one<FMT, false, FMT == MS_U8>
                       : ms::k_bitiles_one<FMT, false, false>);
    if (allow_smem((const void*)kern, sm) != cudaSuccess) return cudaGetLastError();
    kern<<<grid, 32 * wpb, sm, s>>>(j, ntiles, clear);
  } else if (ntiles > 0) {
    ProfScope ps(ctx, s, kProfTile);
    const int64_t warps = (ntiles + 1) / 2;
    // small launches spread their warps over all SMs (one block per SM at
    // most): a lone tile is latency-bound, and packing its warps onto a few
    // SMs would make them share those SMs' ALU pipes
    const int wpb = (int)std::min<int64_t>(kTileThreads / 32, (warps + ctx->sms - 1) / ctx->sms);
    const unsigned grid = (unsigned)((warps + wpb - 1) / wpb);
    const size_t sm = ring_bytes(32 * wpb);
    switch (j.P) {
#define MS_LAUNCH_TILES(PP)                                                             \
  case PP:                                                                              \
    if (allow_smem((const void*)ms::k_tiles_one<PP, FMT, DPMAP>, sm) != cudaSuccess)    \
      return cudaGetLastError();                                                        \
    ms::k_tiles_one<PP, FMT, DPMAP><<<grid, 32 * wpb, sm, s>>>(j, ntiles, fuse, clear); \
    break;
      MS_LAUNCH_TILES(1)
      MS_LAUNCH_TILES(2)
      MS_LAUNCH_TILES(4)
      MS_LAUNCH_TILES(8)
      MS_LAUNCH_TILES(16)
      default:
      MS_LAUNCH_TILES(32)
#undef MS_LAUNCH_TILES
    }
  }
  if (!fuse) {
    ProfScope ps(ctx, s, kProfFixup);
    if (!DPMAP && j.bits_scratch) {
      // size-only: bitplane growth in the flagged box, planes in shared
      // memory when the box is small enough
      // large matrices may have large boxes: a team of blocks (one per SM)
      // then shares every pass
      const size_t sm = kBitsFixSmemBytes;
      if (allow_smem((const void*)ms::k_fixup_bits_one<FMT>, sm) != cudaSuccess)
        return cudaGetLastError();
      // a team of several blocks is one thread-block cluster: the blocks
      // share every pass over planes in global memory and meet at the
      // hardware cluster barrier, unless the box fits one block's shared
      // memory (rank 0 alone)
      cudaLaunchConfig_t cfg;
      cudaLaunchAttribute attr[2];
      fixup_config(team, sm, s, cfg, attr);
      const cudaError_t e =
          cudaLaunchKernelEx(&cfg, ms::k_fixup_bits_one<FMT>, j, (int64_t)(sm / 4),
                             team > 1 ? ctx->d_sync1 : nullptr, team > 1 ? 1 : 0);
      if (e != cudaSuccess) return e;
    } else {
      const bool levels = DPMAP && j.bits_scratch && !j.test_hold;
      if (levels) {
        // dp map: bitplane levels in the box, then every box cell's dp from
        // them; the strip kernel below only finalises unless the levels did
        // not fit the scratch (or the strip test hook is on)
        const size_t smb = kBitsFixSmemBytes;
        if (allow_smem((const void*)ms::k_fixup_dp_levels<FMT>, smb) != cudaSuccess)
          return cudaGetLastError();
        // (a large matrix: one thread-block cluster builds the levels, with
        // its planes in global memory)
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute attr[2];
        fixup_config(team, team > 1 ? 0 : smb, s, cfg, attr);
        const cudaError_t e =
            cudaLaunchKernelEx(&cfg, ms::k_fixup_dp_levels<FMT>, j,
                               (int64_t)(team > 1 ? 0 : smb / 4),
                               team > 1 ? ctx->d_sync1 : nullptr);
        if (e != cudaSuccess) return e;
        ms::k_fixup_dp_cells<<<4 * ctx->sms, 256, 0, s>>>(j);
      }
      const size_t sm = ring_bytes(ms::kFixWarps * 32);
      if (allow_smem((const void*)ms::k_fixup_one<FMT, DPMAP>, sm) != cudaSuccess)
        return cudaGetLastError();
      ms::k_fixup_one<FMT, DPMAP><<<1, ms::kFixWarps * 32, sm, s>>>(j, levels ? 1 : 0);
    }
  }
  return cudaGetLastError();
}

// Second pass of the all-largest-squares call (lists corners when the
// largest side is at most the halo).
cudaError_t launch_emit(ms_ctx* ctx, const Job& j, cudaStream_t s) {
  const int64_t ntiles = tiles_of(j);
  if (ntiles <= 0) return cudaSuccess;
  ProfScope ps(ctx, s, kProfOther);
  const int64_t warps = (ntiles + 1) / 2;
  const int wpb = (int)std::min<int64_t>(kTileThreads / 32, (warps + ctx->sms - 1) / ctx->sms);
  const unsigned grid = (unsigned)((warps + wpb - 1) / wpb);
  const size_t sm = ring_bytes(32 * wpb);
  switch (j.fmt * 64 + j.P) {
#define MS_LAUNCH_EMIT(FF, PP)                                                            \
  case FF * 64 + PP:                                                                      \
    if (allow_smem((const void*)ms::k_tiles_emit<PP, FF>, sm) != cudaSuccess)            \
      return cudaGetLastError();                                                          \
    ms::k_tiles_emit<PP, FF><<<grid, 32 * wpb, sm, s>>>(j, ntiles);                       \
    break;
    MS_LAUNCH_EMIT(MS_U8, 1)
    MS_LAUNCH_EMIT(MS_U8, 2)
    MS_LAUNCH_EMIT(MS_U8, 4)
    MS_LAUNCH_EMIT(MS_U8, 8)
    MS_LAUNCH_EMIT(MS_U8, 16)
    MS_LAUNCH_EMIT(MS_U8, 32)
    MS_LAUNCH_EMIT(MS_BITS32, 1)
    MS_LAUNCH_EMIT(MS_BITS32, 2)
    MS_LAUNCH_EMIT(MS_BITS32, 4)
    MS_LAUNCH_EMIT(MS_BITS32, 8)
    MS_LAUNCH_EMIT(MS_BITS32, 16)
    MS_LAUNCH_EMIT(MS_BITS32, 32)
#undef MS_LAUNCH_EMIT
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---- bit-packed size-only search ---------------------------------------------

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 2-D tensor map over `rows` rows of `words` uint32 words, row stride `stride`
// words, boxes of kSW words x kBR rows, zeros outside.
bool make_map(CUtensorMap* map, const void* base, int64_t words, int64_t rows, int64_t stride) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)words, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)stride * 4};
  const cuuint32_t box[2] = {(cuuint32_t)ms::bits::kSW, (cuuint32_t)ms::bits::kBR};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Whether the bitplane search can take this matrix (TMA needs 16-byte
// aligned rows) and was selected.
bool bits_search_applies(const ms_tuning& tune, const ms_matrix* in) {
  if (in->fmt != MS_BITS32 || tune.packed_path != 1) return false;
  if (in->m <= 0 || in->n <= 0) return false;
  if ((reinterpret_cast<uintptr_t>(in->data) & 15u) || (in->ld & 3)) return false;
  return encode_tiled() != nullptr;
}

ms_status run_bits_search(ms_ctx* ctx, const ms_matrix* in, ms_result* out_dev, cudaStream_t s) {
  namespace B = ms::bits;
  const bool cap = capturing(s);
  const int64_t m = in->m, n = in->n;
  const int64_t wv = (n + 31) / 32;
  const int64_t wp = (wv + 3) / 4 * 4;
  const int nbr = (int)((m + B::kBR - 1) / B::kBR);
  const int nbw = (int)((wv + B::kBW - 1) / B::kBW);
  const int64_t nblocks = (int64_t)nbr * nbw;
  if (nblocks > 0x7fffffff / 2) return MS_ERR_UNSUPPORTED;
  ms_status st = grow(ctx, ctx->d_lvl, ctx->lvl_cap, 2 * m * wp, cap);
  if (st != MS_OK) return st;
  st = grow(ctx, ctx->d_act, ctx->act_cap, 2 * nblocks, cap);
  if (st != MS_OK) return st;
  st = grow(ctx, ctx->d_bst, ctx->bst_cap, 1, cap);
  if (st != MS_OK) return st;
  if (ctx->bits_geom[0] != m || ctx->bits_geom[1] != wp || ctx->bits_geom[2] != nbw) {
    if (cap) return MS_ERR_UNSUPPORTED;
    if (cudaMemsetAsync(ctx->d_lvl, 0, (size_t)(2 * m * wp) * 4, s) != cudaSuccess ||
        cudaMemsetAsync(ctx->d_act, 0, (size_t)(2 * nblocks), s) != cudaSuccess)
      return MS_ERR_CUDA;
    ctx->bits_geom[0] = m;
    ctx->bits_geom[1] = wp;
    ctx->bits_geom[2] = nbw;
  }
  if (ctx->bits_grid == 0) {
    if (cudaFuncSetAttribute(B::k_bits_search, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)B::kSmemBytes) != cudaSuccess)
      return MS_ERR_CUDA;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, B::k_bits_search, B::kThreads,
                                                      B::kSmemBytes) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess ||
        per_sm < 1)
      return MS_ERR_CUDA;
    ctx->bits_grid = per_sm * sms;
  }
  CUtensorMap maps[3];
  uint32_t* bx = ctx->d_lvl;
  uint32_t* by = ctx->d_lvl + m * wp;
  if (!make_map(&maps[0], in->data, wv, m, in->ld) || !make_map(&maps[1], bx, wv, m, wp) ||
      !make_map(&maps[2], by, wv, m, wp))
    return MS_ERR_CUDA;
  B::Args args;
  args.m = m;
  args.n = n;
  args.wv = wv;
  args.wp = wp;
  args.buf[0] = nullptr;
  args.buf[1] = bx;
  args.buf[2] = by;
  args.act[0] = nullptr;
  args.act[1] = ctx->d_act;
  args.act[2] = ctx->d_act + nblocks;
  args.nbr = nbr;
  args.nbw = nbw;
  args.st = ctx->d_bst;
  args.out = out_dev;
  const int grid = (int)std::min<int64_t>(ctx->bits_grid, std::max<int64_t>(nblocks, 1));
  ProfScope ps(ctx, s, kProfOther);
  B::k_bits_reset<<<1, B::kMaxPasses, 0, s>>>(ctx->d_bst);
  void* kargs[] = {&maps[0], &maps[1], &maps[2], &args};
  if (cudaLaunchCooperativeKernel((const void*)B::k_bits_search, dim3(grid), dim3(B::kThreads),
                                  kargs, B::kSmemBytes, s) != cudaSuccess)
    return MS_ERR_CUDA;
  return cuda_status(cudaGetLastError());
}

// Where the all-largest-squares call lists its corners.
struct CornerOut {
  int32_t* corners;
  int64_t cap;
  unsigned long long* count;
};

ms_status run_single(ms_ctx* ctx, const ms_matrix* in, int32_t* dp, int64_t ld_dp,
                     ms_result* out_dev, cudaStream_t s, const CornerOut* co = nullptr) {
  ms_status st = check_matrix(in);
  if (st != MS_OK) return st;
  if (!out_dev) return MS_ERR_INVALID;
  if (dp) {
    if (in->m > 0 && in->n > 0 && ld_dp < in->n) return MS_ERR_INVALID;
  }
  DeviceGuard g(ctx->device);
  const ms_tuning tune = effective_tuning(ctx, in, 1, false);
  if (!dp && !co && bits_search_applies(tune, in)) return run_bits_search(ctx, in, out_dev, s);
  Job j = plan_job(tune, in, dp != nullptr, 32, ctx->sms,
                   !dp && !co && use_bit_tiles(tune, in, ctx->bit_slots) ? ctx->bit_slots : 0);
  st = ensure_workspace(ctx, 1, ms::carry_words(j.m, j.strips_fix), j.strips_fix, s);
  if (st != MS_OK) return st;
  const int64_t bw = bitfix_words(j);
  if (bw > 0 && bw <= kBitfixCapWords &&
      grow(ctx, ctx->d_bitfix, ctx->bitfix_cap, bw, capturing(s)) == MS_OK)
    j.bits_scratch = ctx->d_bitfix;
  // bitplane tiles hand their S_33 rows to the bitplane fix-up
  if (j.tile_kind == 1 && j.bits_scratch &&
      grow(ctx, ctx->d_first33, ctx->first33_cap, std::max<int64_t>(tiles_of(j), 1),
           capturing(s)) == MS_OK)
    j.first33 = ctx->d_first33;
  j.tile0 = 0;
  j.dp = dp;
  j.ld_dp = ld_dp;
  const uintptr_t dpa = reinterpret_cast<uintptr_t>(dp);
  j.dp_aligned = !dp ? 0 : (dpa % 32 == 0 && ld_dp % 8 == 0) ? 2
                           : (dpa % 16 == 0 && ld_dp % 4 == 0) ? 1 : 0;
  j.out = out_dev;
  j.st = ctx->d_states;
  j.carry = ctx->d_carry;
  j.progress = ctx->d_progress;
  if (co) {
    // corners of squares above the halo are listed by the bitplane fix-up
    if (!j.bits_scratch && j.m > 0 && j.n > 0) return MS_ERR_OOM;
    j.corners = co->corners;
    j.corners_cap = co->cap;
    j.corners_count = co->count;
  }
  cudaError_t e;
  if (j.fmt == MS_U8)
    e = dp ? launch_one_fmt<MS_U8, true>(ctx, j, s) : launch_one_fmt<MS_U8, false>(ctx, j, s);
  else
    e = dp ? launch_one_fmt<MS_BITS32, true>(ctx, j, s)
           : launch_one_fmt<MS_BITS32, false>(ctx, j, s);
  if (e == cudaSuccess && co) e = launch_emit(ctx, j, s);
  return cuda_status(e);
}

__global__ void __launch_bounds__(ms::kFixWarps * 32, 1) k_fixup_mixed(const Job* __restrict__ jobs, int njobs) {
  const int j = blockIdx.x;
  if (j >= njobs) return;
  const Job job = jobs[j];
  if (job.bits_scratch || job.tile_kind == 2) return;  // k_fixup_bits_mixed / the small launch
  if (job.fmt == MS_U8)
    ms::fixup_job<MS_U8, false>(job);
  else
    ms::fixup_job<MS_BITS32, false>(job);
}

// Steps a warp spends on tile t of job j (window rows + lane skew).
int tile_steps(const Job& j, int64_t t) {
  const int64_t band = t / j.strips;
  const int64_t r0 = band * j.band_rows;
  const int64_t r1 = std::min<int64_t>(j.m, r0 + j.band_rows);
  // window rows, plus the lane skew of the dp recurrence
  return (int)(r1 - std::max<int64_t>(0, r0 - ms::kHalo)) + (j.tile_kind ? 0 : 31);
}



}  // namespace

extern "C" {

const char* ms_status_string(ms_status st) {
  switch (st) {
    case MS_OK: return "MS_OK";
    case MS_ERR_INVALID: return "MS_ERR_INVALID: invalid argument";
    case MS_ERR_OOM: return "MS_ERR_OOM: device memory or workspace budget exhausted";
    case MS_ERR_CUDA: return "MS_ERR_CUDA: a CUDA runtime call failed";
    case MS_ERR_TIMEOUT: return "MS_ERR_TIMEOUT: a bounded device-side wait gave up";
    case MS_ERR_BUDGET: return "MS_ERR_BUDGET: request exceeds the serving memory budget";
    case MS_ERR_UNSUPPORTED: return "MS_ERR_UNSUPPORTED: outside supported sizes or layouts";
    case MS_ERR_CANCELLED: return "MS_ERR_CANCELLED: request withdrawn before admission";
  }
  return "unknown ms_status";
}

ms_status ms_create(ms_ctx** out, int device, size_t workspace_budget_bytes) {
  if (!out) return MS_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return MS_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return MS_ERR_INVALID;
  ms_ctx* ctx = new (std::nothrow) ms_ctx();
  if (!ctx) return MS_ERR_OOM;
  ctx->device = device;
  ctx->budget = workspace_budget_bytes;
  DeviceGuard g(device);
  if (cudaEventCreateWithFlags(&ctx->stage_free, cudaEventDisableTiming) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->stage_free) cudaEventDestroy(ctx->stage_free);
    delete ctx;
    return MS_ERR_CUDA;
  }
  ctx->sms = std::max(ctx->sms, 1);
  {
    // small-matrix blocks: each class's share of an SM's shared memory (its
    // blocks per SM at once), two planes of its largest matrix at least; what
    // lies beyond the planes stages input rows
    int sm_sm = 0, optin = 0, reserved = 0;
    cudaFuncAttributes fa{};
    const bool ok = cudaDeviceGetAttribute(&sm_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                           device) == cudaSuccess &&
                    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                           device) == cudaSuccess &&
                    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock,
                                           device) == cudaSuccess &&
                    cudaFuncGetAttributes(&fa, ms::k_batch_small) == cudaSuccess;
    if (!ok) cudaGetLastError();
    for (int c = 0; c < kClasses; ++c) {
      const size_t planes = 2 * (size_t)kSmall[c].words * 4;
      size_t share = 0;
      if (ok) {
        const size_t st = fa.sharedSizeBytes, per = (size_t)sm_sm / kSmall[c].per_sm;
        share = per > (size_t)reserved + st ? per - (size_t)reserved - st : 0;
        share = std::min(share, (size_t)optin > st ? (size_t)optin - st : 0) & ~(size_t)15;
      }
      ctx->small_smem[c] = std::max(planes, share);
    }
  }
  {
    // bitplane tiles: blocks of kWarps warps that fit an SM at once (both
    // input formats; the smaller count)
    const size_t sm = (size_t)ms::bt::kWarps * ms::bt::kWarpBytes;
    int b0 = 0, b1 = 0;
    // (the variants without the fused fix-up: the launches that fill the GPU)
    if (allow_smem((const void*)ms::k_bitiles_one<MS_U8, false, false>, sm) != cudaSuccess ||
        allow_smem((const void*)ms::k_bitiles_one<MS_BITS32, false, false>, sm) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, ms::k_bitiles_one<MS_U8, false, false>,
                                                      32 * ms::bt::kWarps, sm) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, ms::k_bitiles_one<MS_BITS32, false, false>,
                                                      32 * ms::bt::kWarps, sm) != cudaSuccess) {
      cudaGetLastError();
      b0 = b1 = 1;
    }
    ctx->bit_slots = ctx->sms * ms::bt::kWarps * std::max(1, std::min(b0, b1));
  }
  if (cudaMalloc(&ctx->d_sync1, sizeof(ms::TeamSync)) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(ctx->stage_free);
    delete ctx;
    return MS_ERR_OOM;
  }
  bool made = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < ms_ctx::kSides && made; ++k)
    made = cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&ctx->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
  if (!made) {
    cudaGetLastError();
    ms_destroy(ctx);
    return MS_ERR_CUDA;
  }
  ms_status st = ensure_workspace(ctx, 64, 1 << 16, 1024, nullptr);
  if (st != MS_OK) {
    ms_destroy(ctx);
    return st;
  }
  *out = ctx;
  return MS_OK;
}

ms_status ms_destroy(ms_ctx* ctx) {
  if (!ctx) return MS_ERR_INVALID;
  {
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    release(ctx, ctx->d_states, ctx->states_cap);
    release(ctx, ctx->d_carry, ctx->carry_cap);
    release(ctx, ctx->d_progress, ctx->progress_cap);
    release(ctx, ctx->d_bitfix, ctx->bitfix_cap);
    release(ctx, ctx->d_first33, ctx->first33_cap);
    release(ctx, ctx->d_table, ctx->table_cap);
    release(ctx, ctx->d_lvl, ctx->lvl_cap);
    release(ctx, ctx->d_act, ctx->act_cap);
    release(ctx, ctx->d_bst, ctx->bst_cap);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->stage_free) cudaEventDestroy(ctx->stage_free);
    if (ctx->d_sync1) cudaFree(ctx->d_sync1);
    for (int k = 0; k < ms_ctx::kSides; ++k) {
      if (ctx->side[k]) cudaStreamDestroy(ctx->side[k]);
      if (ctx->ev_join[k]) cudaEventDestroy(ctx->ev_join[k]);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    for (auto& ps : ctx->prof_pool) {
      cudaEventDestroy(ps.a);
      cudaEventDestroy(ps.b);
    }
  }
  delete ctx;
  return MS_OK;
}

ms_status ms_set_tuning(ms_ctx* ctx, const ms_tuning* t) {
  if (!ctx || !t) return MS_ERR_INVALID;
  if (t->band_rows < 0 || t->band_rows > 16384) return MS_ERR_INVALID;
  if (t->packed_path < 0 || t->packed_path > 1) return MS_ERR_INVALID;
  if (t->test_hold_carries < 0 || t->test_hold_carries > 1) return MS_ERR_INVALID;
  if (t->lane_cols != 0 && t->lane_cols != 1 && t->lane_cols != 2 && t->lane_cols != 4 &&
      t->lane_cols != 8 && t->lane_cols != 16 && t->lane_cols != 32)
    return MS_ERR_INVALID;
  if (t->tile_kind < 0 || t->tile_kind > 2) return MS_ERR_INVALID;
  ctx->tuning = *t;
  return MS_OK;
}

ms_status ms_get_tuning(ms_ctx* ctx, ms_tuning* t) {
  if (!ctx || !t) return MS_ERR_INVALID;
  *t = ctx->tuning;
  return MS_OK;
}

ms_status ms_max_square(ms_ctx* ctx, const ms_matrix* in, ms_result* out_dev, ms_stream_t s) {
  if (!ctx) return MS_ERR_INVALID;
  return run_single(ctx, in, nullptr, 0, out_dev, reinterpret_cast<cudaStream_t>(s));
}

ms_status ms_dp_map(ms_ctx* ctx, const ms_matrix* in, int32_t* dp_dev, int64_t ld_dp,
                    ms_result* out_dev, ms_stream_t s) {
  if (!ctx || !in) return MS_ERR_INVALID;
  if (!dp_dev && in->m > 0 && in->n > 0) return MS_ERR_INVALID;
  return run_single(ctx, in, dp_dev, ld_dp, out_dev, reinterpret_cast<cudaStream_t>(s));
}

// Device of a context (for the 3-D path in its own translation unit; not
// exported from the library).
__attribute__((visibility("hidden"))) int ms_ctx_device(const ms_ctx* ctx) {
  return ctx->device;
}

extern "C" ms_status ms_all_max_squares(ms_ctx* ctx, const ms_matrix* in, int32_t* corners_dev,
                                        int64_t capacity, int64_t* count_dev,
                                        ms_result* out_dev, ms_stream_t s) {
  if (!ctx || !count_dev || capacity < 0 || (capacity > 0 && !corners_dev)) return MS_ERR_INVALID;
  ms_status st = check_matrix(in);
  if (st != MS_OK) return st;
  DeviceGuard g(ctx->device);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
  if (cudaMemsetAsync(count_dev, 0, sizeof(int64_t), cs) != cudaSuccess) return MS_ERR_CUDA;
  const CornerOut co{corners_dev, capacity, reinterpret_cast<unsigned long long*>(count_dev)};
  return run_single(ctx, in, nullptr, 0, out_dev, cs, &co);
}

ms_status ms_batch(ms_ctx* ctx, const ms_matrix* ins_host, int32_t count, ms_result* outs_dev,
                   ms_stream_t stream) {
  if (!ctx || count < 0) return MS_ERR_INVALID;
  if (count == 0) return MS_OK;
  if (!ins_host || !outs_dev) return MS_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int32_t i = 0; i < count; ++i) {
    ms_status st = check_matrix(&ins_host[i]);
    if (st != MS_OK) return st;
  }
  DeviceGuard g(ctx->device);
  const bool cap = capturing(s);

  // Plan.  By default (tile_kind 0) a matrix whose two bitplanes fit one
  // block's shared memory is solved whole by the small-matrix launch, and the
  // larger ones go through bitplane tiles and the box fix-up; tile_kind 2
  // sends every matrix through bitplane tiles, tile_kind 1 (or an explicit
  // lane width) through tile pairs of the dp recurrence.
  const ms_tuning tune = effective_tuning(ctx, ins_host, count, true);
  const int mode = tune.lane_cols > 0 ? 1 : tune.tile_kind;
  std::vector<Job> jobs((size_t)count);
  std::vector<int32_t> small[kClasses];  // matrices for the small-matrix launches, by class
  int64_t carry = 0, progress = 0, work_dp = 0, work_bit = 0;
  for (int32_t i = 0; i < count; ++i) {
    jobs[i] = plan_job(tune, &ins_host[i], false, 16, 0);  // dp recurrence: P <= 16
    Job& j = jobs[i];
    const bool empty = j.m <= 0 || j.n <= 0;
    const int64_t pw = empty ? 0 : ms::small::plane_words(j.m, j.n);
    if (mode == 0 && pw <= kSmall[kClasses - 1].words) {
      j.tile_kind = 2;  // solved whole; no tiles, no fix-up state
      j.strips = j.bands = 0;
      int c = 0;
      while (pw > kSmall[c].words) ++c;
      small[c].push_back(i);
      continue;
    }
    if (mode != 1 && !empty) {
      j.P = 32;
      j.tile_kind = 1;
      j.strips = (int32_t)strips_for(j.n, 32);
      work_bit += j.m * (int64_t)j.strips;
    } else {
      work_dp += j.m * (int64_t)j.strips;
    }
    carry += ms::carry_words(j.m, j.strips_fix);
    progress += j.strips_fix;
  }
  // band heights: dp-recurrence pairs from their total work; bitplane tiles
  // at least 128 rows (the 32-row halo), else as many as fill the GPU's
  // resident tile warps once
  const int64_t br_dp = tune.band_rows > 0 ? tune.band_rows : auto_band_rows_for(work_dp);
  const int64_t br_bit =
      tune.band_rows > 0 ? tune.band_rows
                         : std::min<int64_t>(16384, std::max<int64_t>(
                               128, (work_bit + ctx->bit_slots - 1) / std::max(1, ctx->bit_slots)));
  for (Job& j : jobs) {
    if (j.tile_kind == 2 || j.m <= 0 || j.n <= 0) continue;
    const int64_t br = j.tile_kind == 1 ? br_bit : br_dp;
    j.band_rows = (int32_t)std::min<int64_t>(br, j.m);
    j.bands = (int32_t)((j.m + j.band_rows - 1) / j.band_rows);
  }
  ms_status st = ensure_workspace(ctx, count, std::max<int64_t>(carry, 1),
                                  std::max<int64_t>(progress, 1), s);
  if (st != MS_OK) return st;
  // tiles of one format and lane width form a group; dp-recurrence tiles pair
  // up in a warp, bitplane tiles go one per task; longest first
  struct TileRef { int32_t job, tile, steps; };
  std::vector<std::vector<TileRef>> groups(2 * 64);
  int64_t carry_off = 0, prog_off = 0, bit_need = 0;
  for (int32_t i = 0; i < count; ++i)
    if (jobs[i].tile_kind != 2) bit_need += bitfix_words(jobs[i]);
  bit_need = std::min(bit_need, kBitfixCapWords);
  if (bit_need > 0 && grow(ctx, ctx->d_bitfix, ctx->bitfix_cap, bit_need, cap) != MS_OK)
    bit_need = 0;
  int64_t bit_off = 0;
  bool any_bits = false, any_strip = false;
  // first S_33 row per bitplane tile (for their fix-up's hand-over)
  int64_t f33_need = 0, f33_off = 0;
  for (const Job& j : jobs)
    if (j.tile_kind == 1) f33_need += tiles_of(j);
  const bool f33 = f33_need > 0 &&
                   grow(ctx, ctx->d_first33, ctx->first33_cap, f33_need, cap) == MS_OK;
  for (int32_t i = 0; i < count; ++i) {
    Job& j = jobs[i];
    j.tile0 = 0;
    j.out = outs_dev + i;
    j.st = ctx->d_states + i;
    j.bits_scratch = nullptr;
    j.first33 = nullptr;
    if (j.tile_kind == 2) continue;
    j.carry = ctx->d_carry + carry_off;
    j.progress = ctx->d_progress + prog_off;
    carry_off += ms::carry_words(j.m, j.strips_fix);
    prog_off += j.strips_fix;
    const int64_t bw = bitfix_words(j);
    if (bw > 0 && bit_off + bw <= bit_need) {
      j.bits_scratch = ctx->d_bitfix + bit_off;
      bit_off += bw;
    }
    if (j.bits_scratch) any_bits = true; else any_strip = true;
    const int64_t nt = tiles_of(j);
    if (j.tile_kind == 1 && j.bits_scratch && f33) {
      j.first33 = ctx->d_first33 + f33_off;
      f33_off += nt;
    }
    auto& grp = groups[j.fmt * 64 + j.P];
    for (int64_t t = 0; t < nt; ++t) grp.push_back(TileRef{i, (int32_t)t, tile_steps(j, t)});
  }
  std::vector<ms::PairTask> tasks, bit_tasks;
  std::vector<int> task_steps;
  for (auto& grp : groups) {
    std::stable_sort(grp.begin(), grp.end(),
                     [](const TileRef& x, const TileRef& y) { return x.steps > y.steps; });
    if (!grp.empty() && jobs[grp[0].job].tile_kind == 1) {
      for (const TileRef& r : grp) bit_tasks.push_back(ms::PairTask{r.job, -1, r.tile, 0});
      continue;
    }
    for (size_t k = 0; k < grp.size(); k += 2) {
      ms::PairTask t;
      t.job_a = grp[k].job;
      t.tile_a = grp[k].tile;
      t.job_b = k + 1 < grp.size() ? grp[k + 1].job : -1;
      t.tile_b = k + 1 < grp.size() ? grp[k + 1].tile : 0;
      tasks.push_back(t);
      task_steps.push_back(grp[k].steps);
    }
  }
  // bitplane tiles: one launch per input format (uint8 tiles first), longest
  // first within each
  std::stable_sort(bit_tasks.begin(), bit_tasks.end(), [&](const ms::PairTask& x,
                                                           const ms::PairTask& y) {
    const Job &jx = jobs[x.job_a], &jy = jobs[y.job_a];
    if (jx.fmt != jy.fmt) return jx.fmt < jy.fmt;
    return tile_steps(jx, x.tile_a) > tile_steps(jy, y.tile_a);
  });
  int nbit_u8 = 0;
  while (nbit_u8 < (int)bit_tasks.size() && jobs[bit_tasks[nbit_u8].job_a].fmt == MS_U8) ++nbit_u8;
  {
    // dp-recurrence groups stay contiguous in the queue (warps running at the
    // same time mostly execute one lane-width variant, which keeps the
    // instruction cache warm), the group with the longest tiles first,
    // longest first within each group
    std::vector<size_t> idx(tasks.size());
    for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
    std::vector<int> group_of(tasks.size()), group_max(2 * 64, 0);
    for (size_t k = 0; k < tasks.size(); ++k) {
      const Job& ja = jobs[tasks[k].job_a];
      group_of[k] = ja.fmt * 64 + ja.P;
      group_max[group_of[k]] = std::max(group_max[group_of[k]], task_steps[k]);
    }
    std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
      const int gx = group_of[x], gy = group_of[y];
      if (gx != gy)
        return group_max[gx] != group_max[gy] ? group_max[gx] > group_max[gy] : gx > gy;
      return task_steps[x] > task_steps[y];
    });
    std::vector<ms::PairTask> sorted(tasks.size());
    for (size_t k = 0; k < idx.size(); ++k) sorted[k] = tasks[idx[k]];
    tasks.swap(sorted);
  }
  const int ntasks = (int)tasks.size(), nbit = (int)bit_tasks.size();
  // small matrices largest first within each class
  auto by_cells = [&](int32_t x, int32_t y) { return jobs[x].m * jobs[x].n > jobs[y].m * jobs[y].n; };
  int nsmall = 0;
  for (auto& c : small) {
    std::stable_sort(c.begin(), c.end(), by_cells);
    nsmall += (int)c.size();
  }

  // size-only fix-up blocks: a team per tiled matrix with bitplane scratch,
  // sized by the matrix, larger teams (then larger matrices) first so that
  // the longest fix-ups start early
  std::vector<ms::FixTask> fix;
  {
    std::vector<int32_t> order;
    for (int32_t i = 0; i < count; ++i)
      if (jobs[i].bits_scratch && jobs[i].m > 0 && jobs[i].n > 0) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), by_cells);
    for (int32_t i : order) {
      const int size = fix_team_size(jobs[i].m * jobs[i].n, 16, 18);
      for (int r = 0; r < size; ++r) fix.push_back(ms::FixTask{i, r, size, 0});
    }
  }
  const int nfix = (int)fix.size();

  // table image: [jobs | tasks | bitplane tasks | fix tasks | small order |
  // 8 queue counters | team barriers], 16-byte aligned sections; the last two
  // are cleared before every launch
  auto a16 = [](size_t x) { return (x + 15) / 16 * 16; };
  const size_t jobs_bytes = a16((size_t)count * sizeof(Job));
  const size_t tasks_bytes = a16((size_t)ntasks * sizeof(ms::PairTask));
  const size_t bit_bytes = a16((size_t)nbit * sizeof(ms::PairTask));
  const size_t fix_bytes = a16((size_t)nfix * sizeof(ms::FixTask));
  const size_t order_bytes = a16((size_t)nsmall * sizeof(int32_t));
  const size_t clear_bytes = 32 + (size_t)count * sizeof(ms::TeamSync);
  const size_t o_tasks = jobs_bytes, o_bit = o_tasks + tasks_bytes, o_fix = o_bit + bit_bytes,
               o_order = o_fix + fix_bytes, o_clear = o_order + order_bytes;
  const size_t table_bytes = o_clear + clear_bytes;
  std::vector<unsigned char> image(table_bytes, 0);
  std::memcpy(image.data(), jobs.data(), (size_t)count * sizeof(Job));
  if (ntasks) std::memcpy(image.data() + o_tasks, tasks.data(), (size_t)ntasks * sizeof(ms::PairTask));
  if (nbit) std::memcpy(image.data() + o_bit, bit_tasks.data(), (size_t)nbit * sizeof(ms::PairTask));
  if (nfix) std::memcpy(image.data() + o_fix, fix.data(), (size_t)nfix * sizeof(ms::FixTask));
  {
    size_t off = o_order;
    for (const auto& c : small) {
      if (!c.empty()) std::memcpy(image.data() + off, c.data(), c.size() * sizeof(int32_t));
      off += c.size() * sizeof(int32_t);
    }
  }

  // upload only when it differs from the table already on the device
  if (ctx->uploaded != image) {
    if (cap) return MS_ERR_UNSUPPORTED;  // first run the call once outside capture
    st = grow(ctx, ctx->d_table, ctx->table_cap, (int64_t)table_bytes, false);
    if (st != MS_OK) return st;
    if (ctx->stage_pending) cudaEventSynchronize(ctx->stage_free);
    if (ctx->stage_cap < (int64_t)table_bytes) {
      if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
      ctx->h_stage = nullptr;
      ctx->stage_cap = 0;
      if (cudaMallocHost(&ctx->h_stage, table_bytes) != cudaSuccess) {
        cudaGetLastError();
        return MS_ERR_OOM;
      }
      ctx->stage_cap = (int64_t)table_bytes;
    }
    std::memcpy(ctx->h_stage, image.data(), table_bytes);
    if (cudaMemcpyAsync(ctx->d_table, ctx->h_stage, table_bytes, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return MS_ERR_CUDA;
    cudaEventRecord(ctx->stage_free, s);
    ctx->stage_pending = true;
    ctx->uploaded.swap(image);
  }
  const Job* d_jobs = reinterpret_cast<const Job*>(ctx->d_table);
  const ms::PairTask* d_tasks = reinterpret_cast<const ms::PairTask*>(ctx->d_table + o_tasks);
  const ms::PairTask* d_bit = reinterpret_cast<const ms::PairTask*>(ctx->d_table + o_bit);
  const ms::FixTask* d_fix = reinterpret_cast<const ms::FixTask*>(ctx->d_table + o_fix);
  const int32_t* d_order = reinterpret_cast<const int32_t*>(ctx->d_table + o_order);
  unsigned char* d_clear = ctx->d_table + o_clear;
  // queue counters: tile pairs, uint8 and packed bitplane tiles, the small
  // classes
  static_assert(3 + kClasses <= 8, "eight queue counters");
  int* d_queues = reinterpret_cast<int*>(d_clear);
  ms::TeamSync* d_syncs = reinterpret_cast<ms::TeamSync*>(d_clear + 32);
  if (cudaMemsetAsync(d_clear, 0, clear_bytes, s) != cudaSuccess) return MS_ERR_CUDA;

  // The small matrices run on the context's side streams (one per size
  // class), forked from the caller's after the clear and joined back at the
  // end, so that the classes and the large matrices' tiles and fix-up share
  // the GPU and fill each other's tails (while kernels are timed by
  // ms_profile_*, everything stays on the caller's stream).
  const bool fork = nsmall > 0 && !ctx->prof_on;
  cudaStream_t ss[kClasses];
  for (int c = 0; c < kClasses; ++c) ss[c] = s;
  // joins the side streams back on every way out once they are forked (a
  // capture must not end with a branch left open)
  struct Join {
    ms_ctx* c;
    cudaStream_t s;
    bool on = false;
    bool join() {
      bool ok = true;
      for (int k = 0; k < ms_ctx::kSides; ++k)
        ok = cudaEventRecord(c->ev_join[k], c->side[k]) == cudaSuccess &&
             cudaStreamWaitEvent(s, c->ev_join[k], 0) == cudaSuccess && ok;
      on = false;
      return ok;
    }
    ~Join() {
      if (on) join();
    }
  } join{ctx, s};
  if (fork) {
    if (cudaEventRecord(ctx->ev_fork, s) != cudaSuccess) return MS_ERR_CUDA;
    join.on = true;
    for (int k = 0; k < ms_ctx::kSides; ++k) {
      if (cudaStreamWaitEvent(ctx->side[k], ctx->ev_fork, 0) != cudaSuccess) return MS_ERR_CUDA;
      ss[k] = ctx->side[k];
    }
  }
  {
    ProfScope ps(ctx, s, kProfTile);
    // large matrices first: bitplane tiles (one launch per input format)
    for (int k = 0; k < 2; ++k) {
      const int n = k == 0 ? nbit_u8 : nbit - nbit_u8;
      if (n == 0) continue;
      if (ctx->prof_on) ctx->prof_bit++;
      const size_t sm = (size_t)ms::bt::kWarps * ms::bt::kWarpBytes;
      const void* fn = k == 0 ? (const void*)ms::k_batch_bitiles<MS_U8>
                              : (const void*)ms::k_batch_bitiles<MS_BITS32>;
      if (allow_smem(fn, sm) != cudaSuccess) return MS_ERR_CUDA;
      const int grid = std::max(1, std::min(ctx->bit_slots / ms::bt::kWarps,
                                            (n + ms::bt::kWarps - 1) / ms::bt::kWarps));
      if (k == 0)
        ms::k_batch_bitiles<MS_U8><<<grid, 32 * ms::bt::kWarps, sm, s>>>(d_jobs, d_bit, n,
                                                                         d_queues + 1);
      else
        ms::k_batch_bitiles<MS_BITS32><<<grid, 32 * ms::bt::kWarps, sm, s>>>(
            d_jobs, d_bit + nbit_u8, n, d_queues + 2);
      if (cudaGetLastError() != cudaSuccess) return MS_ERR_CUDA;
    }
    if (ntasks > 0) {
      const size_t sm = ring_bytes(kTileThreads);
      if (allow_smem((const void*)ms::k_batch_tiles, sm) != cudaSuccess) return MS_ERR_CUDA;
      if (ctx->batch_grid == 0) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ms::k_batch_tiles,
                                                          kTileThreads, sm) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) !=
                cudaSuccess)
          return MS_ERR_CUDA;
        ctx->batch_grid = std::max(1, per_sm) * sms;
      }
      const int wpb = kTileThreads / 32;
      const int grid = std::max(1, std::min(ctx->batch_grid, (ntasks + wpb - 1) / wpb));
      ms::k_batch_tiles<<<grid, kTileThreads, sm, s>>>(d_jobs, d_tasks, ntasks, d_queues);
      if (cudaGetLastError() != cudaSuccess) return MS_ERR_CUDA;
    }
    // small matrices solved whole, the largest class first
    int off[kClasses], o = 0;
    for (int c = 0; c < kClasses; ++c) {
      off[c] = o;
      o += (int)small[c].size();
    }
    for (int c = kClasses - 1; c >= 0; --c) {
      const int n = (int)small[c].size();
      if (n == 0) continue;
      const size_t sm = ctx->small_smem[c];
      if (allow_smem((const void*)ms::k_batch_small, sm) != cudaSuccess) return MS_ERR_CUDA;
      const int grid = std::min(n, kSmall[c].per_sm * ctx->sms);
      ms::k_batch_small<<<grid, kSmall[c].threads, sm, ss[c]>>>(d_jobs, d_order + off[c], n,
                                                             d_queues + 3 + c);
      if (cudaGetLastError() != cudaSuccess) return MS_ERR_CUDA;
    }
  }
  {
    ProfScope ps(ctx, s, kProfFixup);
    if (any_bits && nfix > 0) {
      const size_t smb = kBitsFixSmemBytes / 2;  // two blocks per SM
      if (allow_smem((const void*)ms::k_fixup_bits_mixed, smb) != cudaSuccess) return MS_ERR_CUDA;
      ms::k_fixup_bits_mixed<<<nfix, ms::kBitsMixedThreads, smb, s>>>(d_jobs, d_fix, d_syncs,
                                                                      (int64_t)(smb / 4));
    }
    if (any_strip) {
      const size_t smf = ring_bytes(ms::kFixWarps * 32);
      if (allow_smem((const void*)k_fixup_mixed, smf) != cudaSuccess) return MS_ERR_CUDA;
      k_fixup_mixed<<<count, ms::kFixWarps * 32, smf, s>>>(d_jobs, count);
    }
  }
  if (join.on && !join.join()) return MS_ERR_CUDA;
  return cuda_status(cudaGetLastError());
}

ms_status ms_autotune(ms_ctx* ctx, const ms_matrix* ins_host, int32_t count, ms_result* outs_dev,
                      ms_stream_t stream, ms_tuning* chosen) {
  if (!ctx || !ins_host || !outs_dev || count < 1) return MS_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (capturing(s)) return MS_ERR_UNSUPPORTED;
  for (int32_t i = 0; i < count; ++i) {
    ms_status st = check_matrix(&ins_host[i]);
    if (st != MS_OK) return st;
  }
  DeviceGuard g(ctx->device);
  const bool batch = count > 1;
  const bool packed_single = !batch && ins_host[0].fmt == MS_BITS32;
  std::vector<ms_tuning> cands;
  const int rows[] = {0, 32, 64, 128, 256, 512, 1024};
  const int lanes[] = {0, 2, 4, 8, 16, 32};
  // batches also choose how their matrices are tiled: small ones whole and
  // large ones as bitplane tiles (0), everything as dp-recurrence tile pairs
  // (1) or everything as bitplane tiles (2); a single matrix between the
  // automatic choice (0) and bitplane tiles with each band height (2)
  for (int tk = 0; tk <= 2; ++tk)
    for (int pp = 0; pp <= (packed_single ? 1 : 0); ++pp)
      for (int lc : lanes)
        for (int r : rows) {
          // the bitplane search has no band height or lane width; batches use
          // the automatic lane width (at most 16), bitplane tiles have none
          if (pp == 1 && (r != 0 || lc != 0)) continue;
          if (batch && lc != 0) continue;
          if (!batch && (tk == 1 || (tk == 2 && (lc != 0 || pp != 0)))) continue;
          ms_tuning t{};
          t.band_rows = r;
          t.packed_path = pp;
          t.lane_cols = lc;
          t.tile_kind = tk;
          cands.push_back(t);
        }
  const ms_tuning saved = ctx->tuning;
  const auto saved_cache = ctx->tuned;
  ctx->tuned.clear();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // Batches are timed as graph replays on a private stream (ordered after
  // the caller's work): a call's host-side planning, which a caller that
  // captures or repeats the call does not wait for, must not decide the
  // choice.  Single matrices are timed as plain calls on the caller's stream.
  cudaStream_t ts = s;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      (batch && (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess ||
                 cudaEventRecord(e0, s) != cudaSuccess || cudaStreamWaitEvent(ts, e0, 0) != cudaSuccess))) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ts != s) cudaStreamDestroy(ts);
    ctx->tuning = saved;
    ctx->tuned = saved_cache;
    return MS_ERR_CUDA;
  }
  // Every candidate is timed in three interleaved rounds (a slow moment of
  // the GPU then costs each candidate one round at most) and keeps its
  // fastest; a later candidate must beat the best so far by 2% to replace
  // it, so near-ties keep the earlier one (the automatic choice comes first).
  std::vector<float> best_of(cands.size(), 1e30f);
  ms_status err = MS_OK;
  const int reps = 3;
  for (int round = 0; round < 3 && err == MS_OK; ++round) {
    for (size_t c = 0; c < cands.size() && err == MS_OK; ++c) {
      ctx->tuning = cands[c];
      auto run = [&]() -> ms_status {
        return batch ? ms_batch(ctx, ins_host, count, outs_dev, ts)
                     : ms_max_square(ctx, ins_host, outs_dev, ts);
      };
      err = run();  // warm-up (also sizes the workspace and uploads a batch's table)
      if (err != MS_OK) break;
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      if (batch) {
        if (cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
          err = MS_ERR_CUDA;
          break;
        }
        const ms_status ec = run();
        const cudaError_t ee = cudaStreamEndCapture(ts, &graph);
        if (ec != MS_OK || ee != cudaSuccess ||
            cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess ||
            cudaGraphLaunch(exec, ts) != cudaSuccess) {
          err = ec != MS_OK ? ec : MS_ERR_CUDA;
        }
      }
      if (err == MS_OK) {
        cudaEventRecord(e0, ts);
        for (int k = 0; k < reps && err == MS_OK; ++k)
          err = batch ? (cudaGraphLaunch(exec, ts) == cudaSuccess ? MS_OK : MS_ERR_CUDA) : run();
        cudaEventRecord(e1, ts);
        if (err == MS_OK && cudaEventSynchronize(e1) != cudaSuccess) err = MS_ERR_CUDA;
      }
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      if (err != MS_OK) {
        cudaGetLastError();
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best_of[c] = std::min(best_of[c], ms);
    }
  }
  if (ts != s) {
    // the caller's stream resumes after the private one
    cudaEventRecord(e1, ts);
    cudaStreamWaitEvent(s, e1, 0);
    cudaStreamSynchronize(ts);
    cudaStreamDestroy(ts);
  }
  size_t pick = 0;
  for (size_t c = 1; c < cands.size(); ++c)
    if (best_of[c] < 0.98f * best_of[pick]) pick = c;
  const ms_tuning best = cands[pick];
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->tuning = saved;
  ctx->tuned = saved_cache;
  if (err != MS_OK) return err;
  ctx->tuned[tune_class(ins_host, count, batch)] = best;
  if (chosen) *chosen = best;
  return MS_OK;
}

ms_status ms_profile_start(ms_ctx* ctx, int32_t max_launches) {
  if (!ctx || max_launches < 0) return MS_ERR_INVALID;
  ctx->prof_on = true;
  ctx->prof_max = max_launches;
  ctx->prof_used = 0;
  ctx->prof_count[0] = ctx->prof_count[1] = ctx->prof_count[2] = 0;
  ctx->prof_untimed = 0;
  ctx->prof_bit = 0;
  return MS_OK;
}

ms_status ms_profile_stop(ms_ctx* ctx, ms_profile* out) {
  if (!ctx || !out) return MS_ERR_INVALID;
  DeviceGuard g(ctx->device);
  ctx->prof_on = false;
  double ms_sum[3] = {0, 0, 0};
  for (int i = 0; i < ctx->prof_used; ++i) {
    const ms_ctx::ProfSlot& ps = ctx->prof_pool[i];
    if (cudaEventSynchronize(ps.b) != cudaSuccess) return MS_ERR_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ps.a, ps.b) != cudaSuccess) return MS_ERR_CUDA;
    ms_sum[ps.kind] += t;
  }
  out->tile_launches = ctx->prof_count[kProfTile];
  out->tile_ms = ms_sum[kProfTile];
  out->fixup_launches = ctx->prof_count[kProfFixup];
  out->fixup_ms = ms_sum[kProfFixup];
  out->other_launches = ctx->prof_count[kProfOther];
  out->other_ms = ms_sum[kProfOther];
  out->untimed_launches = ctx->prof_untimed;
  out->bit_tile_launches = ctx->prof_bit;
  ctx->prof_used = 0;
  return MS_OK;
}

}  // extern "C"
