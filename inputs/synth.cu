// Seeded synthetic inputs on the GPU: the same counter-based SplitMix64 recipes
// as inputs/__init__.py, bit for bit, so that full-size keys can be made in HBM
// directly. This file holds no sorting arithmetic and shares nothing with the
// sort library or with the oracle.
//
// Generator: counter-based SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).
//   S(seed, stream)       = mix64(seed * GAMMA ^ stream * 0xD1B54A32D192ED03)
//   draw(seed, stream, i) = mix64(S + (i + 1) * GAMMA)
// Distributions 0..5: uniform, u16, equal, sorted, reverse, and4 (see the
// Python module for the definitions).
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kStreamMul = 0xD1B54A32D192ED03ull;

__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ inline uint64_t draw(uint64_t s, uint64_t i) { return mix64(s + (i + 1) * kGamma); }

__device__ inline uint64_t sorted_u32(uint64_t s, uint64_t idx, uint64_t n) {
  uint64_t r = draw(s, idx) >> 32;
  return ((idx << 32) + r) / n;
}

__device__ inline uint64_t sorted_u64(uint64_t s, uint64_t idx, int L) {
  uint64_t d = draw(s, idx);
  if (L == 0) return d;
  return (idx << (64 - L)) | (d >> L);
}

template <typename K>
__global__ void k_synth(K* out, int64_t n, int dist, uint64_t s, int L) {
  const bool wide = sizeof(K) == 8;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t v;
    switch (dist) {
      case 0: v = draw(s, i); if (!wide) v >>= 32; break;
      case 1: v = draw(s, i); if (!wide) v >>= 32; v &= 0xFFFFull; break;
      case 2: v = draw(s, 0); if (!wide) v >>= 32; break;
      case 3: v = wide ? sorted_u64(s, i, L) : sorted_u32(s, i, n); break;
      case 4: v = wide ? sorted_u64(s, n - 1 - i, L) : sorted_u32(s, n - 1 - i, n); break;
      default: {
        uint64_t a = draw(s, 4 * i), b = draw(s, 4 * i + 1), c = draw(s, 4 * i + 2),
                 d = draw(s, 4 * i + 3);
        if (!wide) { a >>= 32; b >>= 32; c >>= 32; d >>= 32; }
        v = a & b & c & d;
      }
    }
    out[i] = (K)v;
  }
}

template <typename V>
__global__ void k_iota(V* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (V)i;
}

int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

extern "C" {

// Fills out[0..n) (device memory, 4- or 8-byte elements by key_bits) with the
// distribution `dist` (0..5) drawn from (seed, stream). Returns 0, or a CUDA
// error code (1 for bad arguments).
int synth_keys(void* out, int64_t n, int key_bits, int dist, uint64_t seed, uint64_t stream,
               void* cuda_stream) {
  if (n < 0 || (key_bits != 32 && key_bits != 64) || dist < 0 || dist > 5) return 1;
  if (n == 0) return 0;
  if (!out) return 1;
  uint64_t s = mix64((seed * kGamma) ^ (stream * kStreamMul));
  int L = 0;
  for (uint64_t m = (uint64_t)(n - 1); m; m >>= 1) ++L;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (key_bits == 32)
    k_synth<uint32_t><<<grid_for(n), 256, 0, st>>>((uint32_t*)out, n, dist, s, L);
  else
    k_synth<uint64_t><<<grid_for(n), 256, 0, st>>>((uint64_t*)out, n, dist, s, L);
  return (int)cudaGetLastError();
}

// out[i] = i for i in [0, n), 4- or 8-byte elements by val_bits.
int synth_iota(void* out, int64_t n, int val_bits, void* cuda_stream) {
  if (n < 0 || (val_bits != 32 && val_bits != 64)) return 1;
  if (n == 0) return 0;
  if (!out) return 1;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (val_bits == 32)
    k_iota<uint32_t><<<grid_for(n), 256, 0, st>>>((uint32_t*)out, n);
  else
    k_iota<uint64_t><<<grid_for(n), 256, 0, st>>>((uint64_t*)out, n);
  return (int)cudaGetLastError();
}

}  // extern "C"
