// Largest all-ones cube of a 3-D volume (the paper's future-work extension,
// Sec. 6).  The 3-D analogue of Eq. 1 has the same structure as the square
// case, and so does its bitplane form: with C_t = bitmap of corners (last
// slice, row and column) of all-ones t-cubes,
//   C_{a+s}(z,i,j) = AND over dz, di, dj in {0, s} of C_a(z-dz, i-di, j-dj)
// for 0 <= s <= a (eight a-cubes at the corners of an (a+s)-cube overlap and
// cover it).  Doubling from C_1 (the input) until a level is empty, then a
// binary search, gives the side K; the first set bit of C_K in (z, i, j)
// order is the witness.  Bits are packed 32 per word along j; one launch per
// step over the whole volume, each reporting whether its level is empty.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/ms.h"

struct ms_ctx;
extern "C" int ms_ctx_device(const ms_ctx* ctx);  // ms.cu, library-internal

namespace {

constexpr int kThreads = 256;

struct Vol {
  int64_t d, m, n, W;  // W = words per row
};

__device__ __forceinline__ uint32_t nonzero_msb(uint32_t x) {
  return ((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x;
}
// bit k = byte k of x is nonzero (k = 0..3): the byte flags at bits 0, 8,
// 16, 24 move to bits 24..27 in one carry-free multiply
__device__ __forceinline__ uint32_t byte_flags4(uint32_t x) {
  return (((nonzero_msb(x) >> 7) & 0x01010101u) * 0x01020408u) >> 24;
}

// C_1: the input as bits, and whether any is set.
__global__ void __launch_bounds__(kThreads) k_cube_pack(const uint8_t* __restrict__ v,
                                                        int64_t ld, int64_t ld_slice, Vol g,
                                                        int aligned, uint32_t* __restrict__ out,
                                                        unsigned int* any) {
  const int64_t total = g.d * g.m * g.W;
  bool hit = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = e % g.W, zi = e / g.W;
    const int64_t i = zi % g.m, z = zi / g.m;
    const int64_t c0 = 32 * w, valid = g.n - c0;
    const uint8_t* row = v + z * ld_slice + i * ld + c0;
    uint32_t bits = 0;
    if (valid >= 32 && aligned) {
      const uint4 lo = __ldg(reinterpret_cast<const uint4*>(row));
      const uint4 hi = __ldg(reinterpret_cast<const uint4*>(row) + 1);
      bits = byte_flags4(lo.x) | byte_flags4(lo.y) << 4 | byte_flags4(lo.z) << 8 |
             byte_flags4(lo.w) << 12 | byte_flags4(hi.x) << 16 | byte_flags4(hi.y) << 20 |
             byte_flags4(hi.z) << 24 | byte_flags4(hi.w) << 28;
    } else {
      const int lim = valid >= 32 ? 32 : (int)valid;
      for (int b = 0; b < lim; ++b) bits |= (uint32_t)(__ldg(row + b) != 0) << b;
    }
    out[e] = bits;
    hit |= bits != 0u;
  }
  if (__any_sync(0xffffffffu, hit) && (threadIdx.x & 31) == 0) atomicOr(any, 1u);
}

// Word w of row i of slice z of level L shifted right by s columns (bits of
// columns j - s), zero outside the volume.
__device__ __forceinline__ uint32_t shifted(const uint32_t* __restrict__ L, int64_t base,
                                            int64_t w, int q, int r) {
  const int64_t w0 = w - q, w1 = w - q - 1;
  const uint32_t hi = w0 >= 0 ? L[base + w0] : 0u;
  const uint32_t lo = (r && w1 >= 0) ? L[base + w1] : 0u;
  return r ? (hi << r) | (lo >> (32 - r)) : hi;
}

// C_{a+s} from L = C_a: written to `out` if not null; `any` set if a bit is
// set; `first` (if not null) takes the smallest (z, i, j) index of a set bit.
__global__ void __launch_bounds__(kThreads) k_cube_grow(const uint32_t* __restrict__ L,
                                                        uint32_t* __restrict__ out, Vol g, int s,
                                                        unsigned int* any,
                                                        unsigned long long* first) {
  const int64_t total = g.d * g.m * g.W;
  const int q = s >> 5, r = s & 31;
  bool hit = false;
  unsigned long long f = ~0ull;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = e % g.W, zi = e / g.W;
    const int64_t i = zi % g.m, z = zi / g.m;
    uint32_t v = 0u;
    if (z >= s && i >= s) {
      v = 0xffffffffu;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t zz = z - ((c & 1) ? s : 0), ii = i - ((c & 2) ? s : 0);
        const int64_t base = (zz * g.m + ii) * g.W;
        v &= L[base + w] & shifted(L, base, w, q, r);
      }
      const int64_t valid = g.n - 32 * w;
      if (valid < 32) v &= (1u << valid) - 1u;
    }
    if (out) out[e] = v;
    if (v) {
      hit = true;
      if (first) {
        const unsigned long long idx = ((unsigned long long)(z * g.m + i)) * (unsigned long long)g.n +
                                       (unsigned long long)(32 * w + (__ffs(v) - 1));
        f = idx < f ? idx : f;
      }
    }
  }
  if (__any_sync(0xffffffffu, hit) && (threadIdx.x & 31) == 0) atomicOr(any, 1u);
  if (first) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const unsigned long long t = __shfl_down_sync(0xffffffffu, f, o);
      f = t < f ? t : f;
    }
    if ((threadIdx.x & 31) == 0 && f != ~0ull) atomicMin(first, f);
  }
}

struct Scratch {
  uint32_t* lvl[2] = {nullptr, nullptr};
  unsigned int* any = nullptr;  // [0]: flag, [2..3]: first (64-bit)
};

}  // namespace

extern "C" ms_status ms_max_cube(ms_ctx* ctx, const ms_volume* in, ms_cube_result* out_dev,
                                 ms_stream_t stream) {
  if (!ctx || !in || !out_dev) return MS_ERR_INVALID;
  if (in->d < 0 || in->m < 0 || in->n < 0 || in->fmt != MS_U8 || in->reserved != 0)
    return MS_ERR_INVALID;
  const bool empty = in->d == 0 || in->m == 0 || in->n == 0;
  if (!empty) {
    if (!in->data || in->ld < in->n || in->ld_slice < (in->m - 1) * in->ld + in->n)
      return MS_ERR_INVALID;
    if (in->d >= ((int64_t)1 << 31) || in->m >= ((int64_t)1 << 31) ||
        in->n >= ((int64_t)1 << 31) || in->d > ((int64_t)1 << 62) / in->m / in->n)
      return MS_ERR_UNSUPPORTED;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ms_ctx_device(ctx));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  ms_cube_result res{0, -1, -1, -1, MS_OK, 0};
  ms_status st = MS_OK;
  Scratch sc;
  auto fail = [&](ms_status e) {
    cudaGetLastError();
    st = e;
  };
  if (!empty) {
    Vol g{in->d, in->m, in->n, (in->n + 31) / 32};
    const int64_t words = g.d * g.m * g.W;
    if (cudaMallocAsync(&sc.lvl[0], (size_t)words * 4, s) != cudaSuccess ||
        cudaMallocAsync(&sc.lvl[1], (size_t)words * 4, s) != cudaSuccess ||
        cudaMallocAsync(&sc.any, 16, s) != cudaSuccess) {
      fail(MS_ERR_OOM);
    } else {
      int dev = 0, sms = 1;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const int64_t want = (words + kThreads - 1) / kThreads;
      const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, 8LL * sms));
      unsigned int* any = sc.any;
      unsigned long long* first = reinterpret_cast<unsigned long long*>(sc.any + 2);
      // one step: clear the flag, launch, read the flag back
      auto step = [&](auto launch) -> bool {
        unsigned int h = 0;
        if (cudaMemsetAsync(any, 0, 4, s) != cudaSuccess) return fail(MS_ERR_CUDA), false;
        launch();
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&h, any, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
          return fail(MS_ERR_CUDA), false;
        return h != 0;
      };
      const int aligned = (reinterpret_cast<uintptr_t>(in->data) % 16 == 0) && in->ld % 16 == 0 &&
                          in->ld_slice % 16 == 0;
      const bool any1 = step([&] {
        k_cube_pack<<<grid, kThreads, 0, s>>>(static_cast<const uint8_t*>(in->data), in->ld,
                                              in->ld_slice, g, aligned, sc.lvl[0], any);
      });
      if (st == MS_OK && any1) {
        const int kmax = (int)std::min(g.d, std::min(g.m, g.n));
        int cur = 0, a = 1, lo = 1, hi = 2;
        for (;;) {  // doubling: C_2a from C_a
          if (2 * a > kmax) {
            lo = a;
            hi = kmax + 1;
            break;
          }
          const bool ne = step([&] {
            k_cube_grow<<<grid, kThreads, 0, s>>>(sc.lvl[cur], sc.lvl[1 - cur], g, a, any,
                                                  nullptr);
          });
          if (st != MS_OK) break;
          if (!ne) {
            lo = a;
            hi = 2 * a;
            break;
          }
          cur = 1 - cur;
          a *= 2;
        }
        while (st == MS_OK && hi - lo > 1) {  // binary search on C_t = grow(C_a, t - a)
          const int t = (lo + hi) / 2;
          const bool ne = step([&] {
            k_cube_grow<<<grid, kThreads, 0, s>>>(sc.lvl[cur], nullptr, g, t - a, any, nullptr);
          });
          if (ne) lo = t; else hi = t;
        }
        if (st == MS_OK) {  // witness: the first set bit of C_lo
          unsigned long long idx = ~0ull;
          if (cudaMemsetAsync(first, 0xff, 8, s) != cudaSuccess) fail(MS_ERR_CUDA);
          if (st == MS_OK) {
            step([&] {
              k_cube_grow<<<grid, kThreads, 0, s>>>(sc.lvl[cur], nullptr, g, lo - a, any, first);
            });
          }
          if (st == MS_OK &&
              (cudaMemcpyAsync(&idx, first, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
               cudaStreamSynchronize(s) != cudaSuccess))
            fail(MS_ERR_CUDA);
          if (st == MS_OK && idx != ~0ull) {
            const unsigned long long nn = (unsigned long long)g.n, mm = (unsigned long long)g.m;
            res.side = lo;
            res.col = (int32_t)(idx % nn);
            res.row = (int32_t)((idx / nn) % mm);
            res.slice = (int32_t)(idx / nn / mm);
          }
        }
      }
    }
    for (uint32_t* p : sc.lvl)
      if (p) cudaFreeAsync(p, s);
    if (sc.any) cudaFreeAsync(sc.any, s);
  }
  res.status = st;
  if (st == MS_OK || st == MS_ERR_CUDA) {
    if (cudaMemcpyAsync(out_dev, &res, sizeof(res), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      st = MS_ERR_CUDA;
    }
  }
  cudaSetDevice(prev);
  return st;
}
