// isort_keys_noalloc: the radix-256 keys-only sort of 32-bit keys with its
// scratch memory in a fixed, file-scope device array instead of a workspace.
//
// Who needs this: callers that must not allocate device memory once they are
// running. A host framework that owns every byte of device memory through its
// own pool and forbids hidden allocations; a latency-critical loop, where
// cudaMalloc/cudaFree may synchronise the device and stall other work; code
// that must not meet an out-of-memory failure after start-up. Such a caller
// passes its keys and gets them back sorted; the library uses only the static
// array below, which every GPU that loads the library holds until the process
// exits.
//
// This file adds an entry point and changes no other code path: it carves the
// static array the same way the workspace is carved and calls the same
// launcher as isort_keys, always with the built-in default kernel variant
// (variant 0 of the radix-256 table; the autotuner's choice does not apply).
// Device errors are OR-ed into the caller's word, which is required.
#include <cstdint>
#include <mutex>

#include "isort.h"
#include "isort_internal.h"

using namespace isort;

namespace {

// Scratch for n <= ISORT_NOALLOC_MAX_KEYS 32-bit keys: the alternate key
// buffer (4 MiB), two look-back arrays (one row of 256 digits x 4 B per tile
// each), histograms, digit bases, flags and tile counters, with 256-byte
// alignment padding. 5 MiB covers it with room to spare.
constexpr size_t kScratchBytes = size_t(5) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr uint32_t kSpinLimit = 1u << 22;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices];  // device address of g_noalloc_scratch, per device
int g_sms[kMaxDevices];

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" isort_status isort_keys_noalloc(void* keys, int64_t n, uint32_t* err_out,
                                           void* stream) {
  if (n < 0) return ISORT_EINVAL;
  if (n > ISORT_NOALLOC_MAX_KEYS) return ISORT_ENOMEM;  // beyond the fixed scratch
  if (n <= 1) return ISORT_OK;
  if (!keys || (reinterpret_cast<uintptr_t>(keys) & 3)) return ISORT_EINVAL;
  // Device errors land in the caller's word: nothing else would ever read them.
  if (!err_out || (reinterpret_cast<uintptr_t>(err_out) & 3)) return ISORT_EINVAL;

  const LsdEntry* tab = nullptr;
  if (lsd_variants_k32(0, 8, &tab) <= 0) return ISORT_EUNSUPPORTED;
  const LsdEntry& e = tab[0];

  // Device set-up, once per device, with that device current: the host-side
  // name of the array is not a device address, so ask the runtime for it.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ISORT_ECUDA;
  void* base = nullptr;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return ISORT_ECUDA;
      }
      int v = 0;
      if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
        v = 152;
      g_sms[dev] = v;
      g_scratch_ptr[dev] = p;
    }
    base = g_scratch_ptr[dev];
    sms = g_sms[dev];
  }

  // Carve the array: histograms, bases, flags, counters, the first round's
  // output cursors, the two look-back arrays, the alternate key buffer.
  const int64_t tiles = (n + e.tile - 1) / e.tile;
  size_t off = 0;
  const size_t hist = off;     off = align256(off + sizeof(uint32_t) * e.passes * e.radix);
  const size_t bases = off;    off = align256(off + sizeof(uint32_t) * e.passes * e.radix);
  const size_t skip = off;     off = align256(off + sizeof(uint32_t) * e.passes);
  const size_t counters = off; off = align256(off + sizeof(uint32_t) * e.passes);
  const size_t claim = off;    off = align256(off + sizeof(uint32_t) * e.radix);
  const size_t status0 = off;  off = align256(off + sizeof(uint32_t) * e.status_words_per_tile * tiles);
  const size_t status1 = off;  off = align256(off + sizeof(uint32_t) * e.status_words_per_tile * tiles);
  const size_t alt = off;      off = align256(off + sizeof(uint32_t) * (size_t)n);
  if (off > kScratchBytes) return ISORT_ENOMEM;

  char* b = static_cast<char*>(base);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The array keeps the previous call's contents. The launcher clears the
  // histograms, the tile counters and the first round's cursors (and the first
  // look-back array when the first round looks back); every other piece is
  // written before it is read.

  LsdArgs a;
  a.keys = keys;
  a.vals = nullptr;
  a.alt_keys = b + alt;
  a.alt_vals = nullptr;
  a.n = n;
  a.hist = reinterpret_cast<uint32_t*>(b + hist);
  a.base = reinterpret_cast<uint32_t*>(b + bases);
  a.skip = reinterpret_cast<uint32_t*>(b + skip);
  a.counters = reinterpret_cast<uint32_t*>(b + counters);
  a.claim = reinterpret_cast<uint32_t*>(b + claim);
  a.status[0] = reinterpret_cast<uint32_t*>(b + status0);
  a.status[1] = reinterpret_cast<uint32_t*>(b + status1);
  a.err = err_out;
  a.spin_limit = kSpinLimit;
  a.stall_tile = -1;
  a.num_sms = sms;
  a.timer = nullptr;
  a.prefetch_tiles = (int64_t)sms * 4;
  a.check_mode = 0;
  return e.launch(a, st) == cudaSuccess ? ISORT_OK : ISORT_ECUDA;
}
