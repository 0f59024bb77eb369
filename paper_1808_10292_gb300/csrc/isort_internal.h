// Internal interface between the C-ABI layer (api.cu) and the kernel
// translation units. Not installed; not part of the public header.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace isort {

// Optional per-kernel timing: when enabled, the launchers record a CUDA event on
// the launching stream before and after each kernel they enqueue.
struct KernelTimer {
  static constexpr int kMax = 64;
  cudaEvent_t ev[2 * kMax];
  const char* name[kMax];
  int count;
  bool ready;
};

// Records the "before" event of a kernel named `name` (no-op when t is null).
void timer_begin(KernelTimer* t, const char* name, cudaStream_t st);
// Records the "after" event of the kernel begun last.
void timer_end(KernelTimer* t, cudaStream_t st);

// Device pointers and sizes for one LSD sort (keys-only when vals == nullptr).
struct LsdArgs {
  void* keys;           // caller's keys, sorted in place
  void* vals;           // caller's payloads or nullptr
  void* alt_keys;       // workspace: n keys
  void* alt_vals;       // workspace: n payloads (when vals != nullptr)
  int64_t n;
  uint32_t* hist;       // workspace: passes * R counters (zeroed by the launcher)
  uint32_t* base;       // workspace: passes * R global digit bases
  uint32_t* skip;       // workspace: passes flags (1 = trivial pass)
  uint32_t* counters;   // workspace: passes tile-id counters (zeroed by the launcher)
  uint32_t* claim;      // workspace: R (+256) output cursors of the order-free first round
                        // (keys only; zeroed by the launchers), or null: it looks back
  uint32_t* status[2];  // workspace: tiles * R look-back words each
  uint32_t* err;        // workspace: latched device error word
  uint32_t spin_limit;  // polls before a wait gives up
  int64_t stall_tile;   // test hook (-1 = off)
  int num_sms;
  KernelTimer* timer;   // null unless kernel timing is on
  int64_t prefetch_tiles;     // L2 prefetch distance of the rounds, in tiles (0: off)
  uint32_t check_mode;        // test hook of the ordered keys-only rounds (0: normal)
};

typedef cudaError_t (*LsdLaunchFn)(const LsdArgs&, cudaStream_t);

// Copies `bytes` (a multiple of 4) between a host buffer and device memory on
// `st` (to_device: src is the host buffer). Modes 0 and 1 use cudaMemcpyAsync;
// mode 2 uses a copy kernel when the host buffer is page-locked, mapped into
// the device's address space at its own address and 16-byte aligned, else
// cudaMemcpyAsync.
cudaError_t copy_host_io(void* dst, const void* src, size_t bytes, bool to_device, int mode,
                         int num_sms, KernelTimer* timer, cudaStream_t st);

// One compiled kernel family for (key_bits, val_bits, radix_bits, variant).
struct LsdEntry {
  int key_bits, val_bits, radix_bits;
  int threads, keys_per_thread;
  int64_t tile;         // keys per tile (threads * keys_per_thread)
  int radix;            // 2^radix_bits
  int passes;
  size_t status_words_per_tile;  // look-back words per tile per buffer
  int status_buffers;            // look-back buffers (2: alternate by pass)
  LsdLaunchFn launch;
  int64_t extra_status_rows = 0;  // look-back rows beyond one per tile, per buffer
};

// Variant tables, one per key width (sort_k32.cu, sort_k64.cu).
int lsd_variants_k32(int val_bits, int radix_bits, const LsdEntry** out);
int lsd_variants_k64(int val_bits, int radix_bits, const LsdEntry** out);
// Wide-radix paths (wide_rounds.cu): radix_bits 16 (radix 65536) or 11 (radix
// 2048); one entry per (key_bits, val_bits, radix_bits).
int wide_variants(int key_bits, int val_bits, int radix_bits, const LsdEntry** out);

// ---- segmented sort (segmented.cuh) ----
// Layout of the small counter block (uint32 words).
enum {
  kCntClassLen = 0,      // [4] ranges per class
  kCntCursor = 4,        // [4] pop cursors of the persistent BTN kernels
  kCntTiles = 8,         // tiles of all radix ranges
  kCntPassTiles = 9,     // [passes] tile-id counters of the rounds
  kCntWords = 32
};

struct SegArgs {
  void* keys;
  void* vals;
  void* alt_keys;
  void* alt_vals;
  const int64_t* offsets;
  int64_t nseg;
  int64_t total;
  int64_t btn_max;       // ranges longer than this take the radix path
  int network;           // short-range network: 0 = BTN, 1 = OET
  int64_t max_tiles;     // upper bound on tiles of the radix ranges
  int32_t* lists;        // [4][nseg]
  uint32_t* cnt;         // [kCntWords]
  uint32_t* slot_first;  // [nseg] first tile id of each radix range
  int32_t* tile_slot;    // [max_tiles] radix range (slot) of each tile
  uint32_t* seg_hist;    // [nseg][P][R]
  uint32_t* seg_base;    // [nseg][P][R]
  uint32_t* seg_skip;    // [nseg][P] trivial passes of each radix range
  uint32_t* seg_claim;   // [nseg][R] keys only: the first round's output cursors per range
  uint64_t* tile_info;   // [max_tiles] per radix tile: first key (40 bits) | keys << 40 |
                         // skip of each pass << 56
  uint32_t* status[2];   // [max_tiles][R]
  uint32_t* err;
  uint32_t spin_limit;
  int num_sms;
  KernelTimer* timer;
  uint32_t check_mode;   // test hook of the ordered keys-only rounds (0: normal)
  int agg_top;           // the ranges are narrow in key value (a sample sort's buckets):
                         // the top pass reserves slots per digit value in tiles with few digits
};

// Host side: configuration of one (key, payload) family and its launcher.
struct SegConfig {
  int key_bits, val_bits;
  int warp_m, mid_m, cta_m;  // keys per thread of the three BTN classes
  int64_t tile;              // keys per radix tile
  int passes, radix;
  cudaError_t (*launch)(const SegArgs&, cudaStream_t);
};

// The splitter partition round of the sample sort (sample_sort.cu): sample,
// splitters, bucket counts and offsets, and one count-sort round by bucket
// from keys/vals into out_keys/out_vals.
struct GvrArgs {
  const void* keys;      // caller's keys (input of the round)
  const void* vals;      // caller's payloads or nullptr
  void* out_keys;        // workspace: keys grouped by bucket
  void* out_vals;        // workspace: payloads (when vals != nullptr)
  int64_t n;
  int buckets;           // p, 1..256
  int oversample;        // s, p * s <= 4096
  uint64_t seed;
  void* split;           // [255] keys: splitters, then padding
  void* cell;            // [1024] uint16: bucket range of each top-10-bit key cell
  uint32_t* hist;        // [256] bucket counts
  uint32_t* base;        // [256] bucket bases
  uint32_t* skip;        // [1]
  uint32_t* counter;     // [1] tile-id counter
  uint32_t* status;      // [tiles][256] look-back words (payloads only)
  uint32_t* claim;       // [256] keys only: the split round's output cursors
  int64_t* offsets;      // [buckets + 1] bucket offsets for the segmented sort
  uint32_t* counts_out;  // [buckets] caller's copy of the bucket counts, or nullptr
  uint32_t* err;
  uint32_t spin_limit;
  int num_sms;
  KernelTimer* timer;
};

// GSD merge tiles hold at least this many output keys (sizes the cut array).
constexpr int64_t kGsdMinMergeTile = 2048;

// The sample, split and merge steps of GSD (gsd.cu), after the local sort of
// the p sequences [n*k/p, n*(k+1)/p) in keys/vals.
struct GsdArgs {
  void* keys;            // caller's keys, each sequence sorted; the result ends here
  void* vals;            // caller's payloads or nullptr
  void* alt_keys;        // workspace: n keys
  void* alt_vals;        // workspace: n payloads (when vals != nullptr)
  int64_t n;
  int buckets;           // p, a power of two, 1..64
  int oversample;        // r, r * p * p <= 4096
  void* split;           // [p - 1] keys
  int64_t* bound;        // [p][p + 1] part ends inside each sequence
  int64_t* pre;          // [p][p + 1] part offsets inside each bucket
  int64_t* bucket_off;   // [p + 1]
  int64_t* pair_info;    // [p * p / 2][5] merge pairs of one round
  int64_t* pair_tile;    // [p * p / 2 + 1] first output tile of each pair
  int64_t* cut;          // [n / kGsdMinMergeTile + p * p + 1] merge-path split of each output tile
  uint32_t* counts_out;  // [p] caller's copy of the bucket sizes, or nullptr
  uint32_t* err;
  KernelTimer* timer;
};
cudaError_t gsd_merge_launch(int key_bits, int val_bits, const GsdArgs& a, cudaStream_t st);
cudaError_t gsd_offsets_launch(int64_t n, int p, int64_t* off, cudaStream_t st);

int64_t gvr_tile(int key_bits, int val_bits);  // keys per tile of the round
cudaError_t gvr_split_launch(int key_bits, int val_bits, const GvrArgs& a, cudaStream_t st);

// Segmented sort families (segmented_k32.cu, segmented_k64.cu).
const SegConfig* seg_config_k32(int val_bits);
const SegConfig* seg_config_k64(int val_bits);

}  // namespace isort
