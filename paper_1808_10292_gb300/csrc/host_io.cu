// Copies between host buffers and device memory for the host-buffer sorts
// (isort_keys_host, isort_pairs_host).
//
// By default every copy is a cudaMemcpyAsync: the copy engines move host
// buffers at the host link's rate (about 200 GB/s per direction on GB300, both
// directions at once) without taking SMs from the sorts of other streams. The
// other way, forced with mode 2, is a copy kernel: every SM reads (or writes) a
// page-locked host buffer through its device mapping, 16 bytes per access,
// several accesses in flight per thread. It reaches the same link rate alone
// but holds the SMs while it waits on the link, so the sorts of other streams
// cannot overlap it (measured: 12.9 ms against 7.0 ms per pipelined 2^28-key
// step).
#include <algorithm>

#include "isort_internal.h"

namespace isort {
namespace {

constexpr int kCopyThreads = 512;
constexpr int kCopyUnroll = 4;

// dst[i] = src[i] for i < n16 (16-byte words), grid-stride; each thread keeps
// kCopyUnroll loads in flight before it stores them.
__global__ void __launch_bounds__(kCopyThreads) k_copy16(const uint4* __restrict__ src,
                                                        uint4* __restrict__ dst, int64_t n16) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kCopyUnroll - 1) * stride < n16; i += kCopyUnroll * stride) {
    uint4 v[kCopyUnroll];
#pragma unroll
    for (int u = 0; u < kCopyUnroll; ++u) v[u] = src[i + u * stride];
#pragma unroll
    for (int u = 0; u < kCopyUnroll; ++u) dst[i + u * stride] = v[u];
  }
  for (; i < n16; i += stride) dst[i] = src[i];
}

// The last bytes (fewer than 16; a multiple of 4): one 4-byte word per thread.
__global__ void k_copy4(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, int n4) {
  if ((int)threadIdx.x < n4) dst[threadIdx.x] = src[threadIdx.x];
}

// Whether kernels on the current device may dereference host address p
// itself: p is page-locked host memory whose device mapping is p (as for
// cudaHostAlloc memory under unified addressing). Anything else -- pageable
// memory, device or managed memory, a mapping at another address -- is left
// to the copy engines.
bool kernel_addressable(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // not a sticky error: clear it and take the copy engines
    return false;
  }
  return at.type == cudaMemoryTypeHost && at.devicePointer == p;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

cudaError_t copy_host_io(void* dst, const void* src, size_t bytes, bool to_device, int mode,
                         int num_sms, KernelTimer* timer, cudaStream_t st) {
  if (!bytes) return cudaSuccess;
  // modes 0 (automatic) and 1: copy engines; 2: a kernel where the buffers allow it
  if (mode == 2 && bytes % 4 == 0 && aligned16(src) && aligned16(dst) &&
      kernel_addressable(to_device ? src : dst)) {
    const int64_t n16 = (int64_t)(bytes / 16);
    const int tail = (int)(bytes % 16) / 4;
    if (n16) {
      const int64_t want = (n16 + (int64_t)kCopyThreads * kCopyUnroll - 1) /
                           ((int64_t)kCopyThreads * kCopyUnroll);
      const int blocks = (int)std::min<int64_t>(want, (int64_t)num_sms * 4);
      timer_begin(timer, to_device ? "k_copy_h2d" : "k_copy_d2h", st);
      k_copy16<<<blocks, kCopyThreads, 0, st>>>(static_cast<const uint4*>(src),
                                                static_cast<uint4*>(dst), n16);
      timer_end(timer, st);
    }
    if (tail) {
      timer_begin(timer, to_device ? "k_copy_h2d" : "k_copy_d2h", st);
      k_copy4<<<1, 32, 0, st>>>(
          reinterpret_cast<const uint32_t*>(static_cast<const char*>(src) + n16 * 16),
          reinterpret_cast<uint32_t*>(static_cast<char*>(dst) + n16 * 16), tail);
      timer_end(timer, st);
    }
    return cudaGetLastError();
  }
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st);
}

}  // namespace isort
