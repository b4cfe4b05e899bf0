// Device implementation of the seeded input generator (same function as
// msgen.c, definitions in msgen.h).  Used to create large benchmark inputs in
// HBM without a host round trip; tests check it against the host version.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ULL;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return z;
}

// One thread writes 16 consecutive cells of one row.
__global__ void fill_u8_kernel(uint8_t* out, int64_t m, int64_t n, int64_t ld, uint64_t key,
                               uint32_t thr24) {
  const int64_t chunks = (n + 15) / 16;
  const int64_t total = m * chunks;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / chunks;
    const int64_t j0 = (t - i * chunks) * 16;
    uint8_t* row = out + i * ld;
    uint64_t k = (uint64_t)(i * n + j0);
    for (int b = 0; b < 16 && j0 + b < n; ++b, ++k) {
      uint64_t z = mix64(key + (k + 1) * kGamma);
      row[j0 + b] = (uint8_t)((uint32_t)(z >> 40) < thr24);
    }
  }
}

// One thread writes one 32-column word of one row.
__global__ void fill_bits_kernel(uint32_t* out, int64_t m, int64_t n, int64_t ldw, uint64_t key,
                                 uint32_t thr24, uint32_t pad) {
  const int64_t total = m * ldw;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ldw;
    const int64_t w = t - i * ldw;
    uint32_t word = 0;
    for (int b = 0; b < 32; ++b) {
      const int64_t j = 32 * w + b;
      uint32_t bit;
      if (j < n) {
        uint64_t z = mix64(key + ((uint64_t)(i * n + j) + 1) * kGamma);
        bit = (uint32_t)(z >> 40) < thr24;
      } else {
        bit = pad;
      }
      word |= bit << b;
    }
    out[i * ldw + w] = word;
  }
}

__global__ void plant_u8_kernel(uint8_t* out, int64_t ld, int64_t r, int64_t c, int64_t s) {
  const int64_t total = s * s;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / s, j = t - (t / s) * s;
    out[(r + i) * ld + c + j] = 1;
  }
}

__global__ void plant_bits_kernel(uint32_t* out, int64_t ldw, int64_t r, int64_t c, int64_t s) {
  // one thread per (row, word) overlapping the square
  const int64_t w0 = c >> 5, w1 = (c + s - 1) >> 5;
  const int64_t nw = w1 - w0 + 1;
  const int64_t total = s * nw;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = r + t / nw;
    const int64_t w = w0 + (t - (t / nw) * nw);
    const int64_t lo = (w * 32 > c) ? w * 32 : c;
    const int64_t hi = ((w + 1) * 32 < c + s) ? (w + 1) * 32 : c + s;  // exclusive
    uint32_t mask = 0;
    for (int64_t j = lo; j < hi; ++j) mask |= 1u << (j & 31);
    out[i * ldw + w] |= mask;
  }
}

int grid_for(int64_t work) {
  int64_t g = (work + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

extern "C" {

int msgen_fill_u8_dev(uint8_t* out, int64_t m, int64_t n, int64_t ld, uint64_t seed,
                      uint32_t thr24, cudaStream_t stream) {
  if (m <= 0 || n <= 0) return 0;
  fill_u8_kernel<<<grid_for(m * ((n + 15) / 16)), 256, 0, stream>>>(out, m, n, ld, mix64(seed),
                                                                     thr24);
  return (int)cudaGetLastError();
}

int msgen_fill_bits_dev(uint32_t* out, int64_t m, int64_t n, int64_t ldw, uint64_t seed,
                        uint32_t thr24, int pad_value, cudaStream_t stream) {
  if (m <= 0 || ldw <= 0) return 0;
  fill_bits_kernel<<<grid_for(m * ldw), 256, 0, stream>>>(out, m, n, ldw, mix64(seed), thr24,
                                                          pad_value ? 1u : 0u);
  return (int)cudaGetLastError();
}

int msgen_plant_u8_dev(uint8_t* out, int64_t ld, int64_t r, int64_t c, int64_t s,
                       cudaStream_t stream) {
  if (s <= 0) return 0;
  plant_u8_kernel<<<grid_for(s * s), 256, 0, stream>>>(out, ld, r, c, s);
  return (int)cudaGetLastError();
}

int msgen_plant_bits_dev(uint32_t* out, int64_t ldw, int64_t r, int64_t c, int64_t s,
                         cudaStream_t stream) {
  if (s <= 0) return 0;
  plant_bits_kernel<<<grid_for(s * (s / 32 + 2)), 256, 0, stream>>>(out, ldw, r, c, s);
  return (int)cudaGetLastError();
}

}  // extern "C"
