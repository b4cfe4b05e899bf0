// ms_max_square_noalloc: largest all-ones square of one matrix without any
// device allocation.
//
// Who needs this: some callers may not call cudaMalloc at all.  Examples are
// plug-ins running inside a host application that hands every byte of device
// memory to its own pool allocator and forbids raw allocations, and
// latency-critical services that must not allocate after start-up because
// cudaMalloc can synchronise the device and take milliseconds.  Such callers
// cannot create an ms_ctx (ms_create allocates the context's workspace), so
// this entry point takes no context.
//
// Where its scratch lives: the per-matrix result state, the fix-up progress
// flags and the fix-up strip carries sit in one file-scope device array,
// g_noalloc_scratch, sized for matrices of up to kNoAllocMaxRows x
// kNoAllocMaxCols cells (see the sizes below, about 0.53 MiB).  Every GPU that
// loads this library holds that array until the process exits.  The caller
// still passes the input matrix and the result buffer.
//
// In host code the array's name is only a host-side stand-in, not a device
// address, so the first call on each device looks up the array's real
// address with cudaGetSymbolAddress (with that device current) and keeps it,
// with the device's context; later calls in that context reuse it, and a
// call in a new context of the device (after cudaDeviceReset) looks it up
// again.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "ms_kernels.cuh"

namespace {

constexpr int64_t kNoAllocMaxRows = 8192;
constexpr int64_t kNoAllocMaxCols = 8192;
constexpr int kNoAllocMaxStrips =
    (int)((kNoAllocMaxCols + ms::kHalo + ms::kFixW - 1) / ms::kFixW + 1);
constexpr size_t kStateBytes = 256;
constexpr size_t kProgressBytes = ((kNoAllocMaxStrips * sizeof(int32_t) + 255) / 256) * 256;
constexpr size_t kCarryBytes =
    (size_t)ms::carry_words(kNoAllocMaxRows, kNoAllocMaxStrips) * sizeof(uint32_t);
constexpr size_t kScratchBytes = kStateBytes + kProgressBytes + kCarryBytes;
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

}  // namespace

// The shared scratch: [state | progress flags | strip carries].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

// Clears what must start at zero before each call.  Device code names the
// array directly.
__global__ void k_noalloc_reset(int nstrips) {
  ms::JobState* st = reinterpret_cast<ms::JobState*>(g_noalloc_scratch);
  int32_t* progress = reinterpret_cast<int32_t*>(g_noalloc_scratch + kStateBytes);
  if (threadIdx.x == 0) {
    st->key = 0ull;
    st->box[0] = 0x7fffffff;
    st->box[1] = -1;
    st->box[2] = 0x7fffffff;
    st->box[3] = -1;
    st->status = 0;
    st->done = 0;
  }
  for (int i = threadIdx.x; i < nstrips; i += blockDim.x) progress[i] = 0;
}

template <int P, int FMT>
__global__ void __launch_bounds__(kThreads) k_noalloc_tiles(const ms::Job job, int64_t ntiles) {
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  ms::tile_pass_warp<P, FMT, false>(&job, 1, ntiles, w);
}

template <int FMT>
__global__ void __launch_bounds__(ms::kFixWarps * 32, 1) k_noalloc_fixup(const ms::Job job) {
  ms::fixup_job<FMT, false>(job);
}

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

// The driver's cuCtxGetCurrent, through the runtime's entry-point query (no
// link-time dependency on the driver library).
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

template <int FMT>
cudaError_t allow_smem_all();

// Per device: the context the set-up was made in, the scratch array's device
// address in it, and whether the kernels' shared-memory limits are raised.
struct DeviceSetup {
  CUcontext ctx = nullptr;
  unsigned char* addr = nullptr;
};
std::mutex g_mu;
DeviceSetup g_setup[kMaxDevices];

// Device address of g_noalloc_scratch on the current device.  The set-up
// (cudaGetSymbolAddress with the device current, and the kernels'
// shared-memory limits) runs on the first call on a device, and again when
// the device's context has changed since (after cudaDeviceReset the module is
// loaded anew and the array may sit at another address).
ms_status scratch_address(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return MS_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return MS_ERR_UNSUPPORTED;
  CtxGetCurrentFn get = ctx_get_current();
  if (!get) return MS_ERR_CUDA;
  // (null before the runtime has made the device's context current in this
  // thread: the set-up below does that)
  CUcontext cur = nullptr;
  if (get(&cur) != CUDA_SUCCESS) cur = nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceSetup& d = g_setup[dev];
  if (!d.addr || !cur || d.ctx != cur) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      d.addr = nullptr;
      return MS_ERR_CUDA;
    }
    if (allow_smem_all<MS_U8>() != cudaSuccess || allow_smem_all<MS_BITS32>() != cudaSuccess) {
      cudaGetLastError();
      d.addr = nullptr;
      return MS_ERR_CUDA;
    }
    if (get(&cur) != CUDA_SUCCESS || !cur) {
      d.addr = nullptr;
      return MS_ERR_CUDA;
    }
    d.addr = static_cast<unsigned char*>(p);
    d.ctx = cur;
  }
  *out = d.addr;
  return MS_OK;
}

int pairs_for(int64_t n) {
  if (n <= 32) return 1;
  if (n <= 64) return 2;
  if (n <= 128) return 4;
  if (n <= 256) return 8;
  return 16;
}

// Raise a kernel's dynamic shared memory limit (its per-warp input rings).
cudaError_t allow_smem(const void* fn, int bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

constexpr int kTileSmem = (kThreads / 32) * ms::kRingWarpBytes;
constexpr int kFixSmem = ms::kFixWarps * ms::kRingWarpBytes;

// Every kernel of one format, for the current device (part of the set-up).
template <int FMT>
cudaError_t allow_smem_all() {
  cudaError_t e = allow_smem((const void*)k_noalloc_tiles<1, FMT>, kTileSmem);
  if (e == cudaSuccess) e = allow_smem((const void*)k_noalloc_tiles<2, FMT>, kTileSmem);
  if (e == cudaSuccess) e = allow_smem((const void*)k_noalloc_tiles<4, FMT>, kTileSmem);
  if (e == cudaSuccess) e = allow_smem((const void*)k_noalloc_tiles<8, FMT>, kTileSmem);
  if (e == cudaSuccess) e = allow_smem((const void*)k_noalloc_tiles<16, FMT>, kTileSmem);
  if (e == cudaSuccess) e = allow_smem((const void*)k_noalloc_fixup<FMT>, kFixSmem);
  return e;
}

// (the kernels' shared-memory limits were raised by the device's set-up)
template <int FMT>
cudaError_t launch(const ms::Job& j, int64_t ntiles, cudaStream_t s) {
  if (ntiles > 0) {
    const int64_t warps = (ntiles + 1) / 2;
    const unsigned grid = (unsigned)((warps + kThreads / 32 - 1) / (kThreads / 32));
    const int sm = kTileSmem;
    switch (j.P) {
#define MS_NOALLOC_TILES(PP)                                                      \
  case PP:                                                                        \
    k_noalloc_tiles<PP, FMT><<<grid, kThreads, sm, s>>>(j, ntiles);               \
    break;
      MS_NOALLOC_TILES(1)
      MS_NOALLOC_TILES(2)
      MS_NOALLOC_TILES(4)
      MS_NOALLOC_TILES(8)
      default:
      MS_NOALLOC_TILES(16)
#undef MS_NOALLOC_TILES
    }
  }
  k_noalloc_fixup<FMT><<<1, ms::kFixWarps * 32, kFixSmem, s>>>(j);
  return cudaGetLastError();
}

}  // namespace

extern "C" ms_status ms_max_square_noalloc(const ms_matrix* in, ms_result* out_dev,
                                           ms_stream_t stream) {
  if (!in || !out_dev) return MS_ERR_INVALID;
  if (in->m < 0 || in->n < 0 || in->reserved != 0) return MS_ERR_INVALID;
  if (in->fmt != MS_U8 && in->fmt != MS_BITS32) return MS_ERR_INVALID;
  if (in->m > 0 && in->n > 0) {
    if (!in->data) return MS_ERR_INVALID;
    const int64_t row_elems = in->fmt == MS_U8 ? in->n : (in->n + 31) / 32;
    if (in->ld < row_elems) return MS_ERR_INVALID;
    if (in->fmt == MS_BITS32 && (reinterpret_cast<uintptr_t>(in->data) & 3u))
      return MS_ERR_INVALID;
  }
  // larger matrices do not fit the fixed scratch array
  if (in->m > kNoAllocMaxRows || in->n > kNoAllocMaxCols) return MS_ERR_UNSUPPORTED;

  unsigned char* scratch = nullptr;
  ms_status st = scratch_address(&scratch);
  if (st != MS_OK) return st;

  ms::Job j;
  std::memset(&j, 0, sizeof(j));
  j.data = in->data;
  j.m = in->m;
  j.n = in->n;
  j.ld = in->ld;
  j.fmt = in->fmt;
  j.P = pairs_for(in->n);
  int64_t ntiles = 0;
  if (in->m > 0 && in->n > 0) {
    const int64_t W = 32 * j.P;
    j.strips = (int32_t)(in->n <= W ? 1 : 1 + (in->n - W + (W - ms::kHalo) - 1) / (W - ms::kHalo));
    int64_t br = (in->m * j.strips + 2 * 152 * 16 - 1) / (2 * 152 * 16);
    br = std::min<int64_t>(std::max<int64_t>((br + 31) / 32 * 32, 32), 4096);
    j.band_rows = (int32_t)std::min<int64_t>(br, in->m);
    j.bands = (int32_t)((in->m + j.band_rows - 1) / j.band_rows);
    ntiles = (int64_t)j.bands * j.strips;
  }
  j.aligned = (in->fmt == MS_U8) && (reinterpret_cast<uintptr_t>(in->data) % 16 == 0) &&
              (in->ld % 16 == 0);
  j.tile0 = 0;
  j.out = out_dev;
  j.st = reinterpret_cast<ms::JobState*>(scratch);
  j.progress = reinterpret_cast<int32_t*>(scratch + kStateBytes);
  j.carry = reinterpret_cast<uint32_t*>(scratch + kStateBytes + kProgressBytes);
  j.strips_fix = kNoAllocMaxStrips;

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_noalloc_reset<<<1, kThreads, 0, s>>>(kNoAllocMaxStrips);
  const cudaError_t e = in->fmt == MS_U8 ? launch<MS_U8>(j, ntiles, s)
                                         : launch<MS_BITS32>(j, ntiles, s);
  return e == cudaSuccess ? MS_OK : MS_ERR_CUDA;
}
