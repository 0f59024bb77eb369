// C-ABI of the isort library: argument checks, per-stream workspaces, kernel
// family selection. Every step of a sort runs in the kernels of sort_k32.cu,
// sort_k64.cu (onesweep.cuh), wide_rounds.cu, segmented_k32.cu / segmented_k64.cu
// (segmented.cuh, btn.cuh), sample_sort.cu, gsd.cu, noalloc.cu and host_io.cu;
// this file only validates, carves scratch memory and enqueues.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <unordered_map>

#include "isort.h"
#include "isort_internal.h"

using namespace isort;

namespace {

constexpr uint32_t kDefaultSpinLimit = 1u << 22;  // polls of an L2-resident word: seconds
constexpr int64_t kMaxN = int64_t(1) << 30;

struct Workspace {
  void* base = nullptr;
  size_t bytes = 0;
  bool owned = false;  // allocated by the library (stream-ordered) vs bound by the caller
};

std::mutex g_mu;
std::unordered_map<cudaStream_t, Workspace> g_ws;
std::map<std::tuple<int, int, int>, int> g_variant;  // (key_bits, val_bits, radix_bits) -> index
uint32_t g_spin_limit = kDefaultSpinLimit;
int64_t g_stall_tile = -1;
std::map<int, int> g_sms;  // device -> SM count
KernelTimer g_timer;
bool g_timing = false;
int64_t g_prefetch = -1;  // L2 prefetch distance in tiles; -1: one wave (SMs x 4)
uint32_t g_check_mode = 0;  // test hook of the ordered keys-only rounds
int g_host_copy = 0;        // host-buffer sorts: 0 auto (copy engines), 1 copy engines, 2 kernels

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int num_sms() {
  int dev = 0;
  cudaGetDevice(&dev);
  auto it = g_sms.find(dev);
  if (it != g_sms.end()) return it->second;
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
    v = 152;
  g_sms[dev] = v;
  return v;
}

int variants(int key_bits, int val_bits, int radix_bits, const LsdEntry** out) {
  if (radix_bits == 16 || radix_bits == 11) return wide_variants(key_bits, val_bits, radix_bits, out);
  if (key_bits == 32) return lsd_variants_k32(val_bits, radix_bits, out);
  if (key_bits == 64) return lsd_variants_k64(val_bits, radix_bits, out);
  return 0;
}

// Automatic choice of radix width and kernel variant per (key_bits, val_bits)
// and size bucket (floor(log2 n)): radix_bits = 0 resolves through it.
struct AutoChoice {
  int radix_bits, variant;
};
// Runtime entries (isort_tune_auto; the Python tuner loads its cache here).
std::map<std::pair<int, int>, std::map<int, AutoChoice>> g_auto;

// Built-in entries: what the autotuner (tune.py) picked on a GB300 for these
// sizes (paper_1808_10292_gb300/tune_cache.json); used when no runtime entry
// exists for the widths. Other widths default to radix 256, variant 0.
struct BuiltinChoice {
  int key_bits, val_bits, bucket, radix_bits, variant;
};
const BuiltinChoice kBuiltinAuto[] = {
    {32, 0, 24, 8, 0},   // 2^24 u32 keys: 256 x 32 (0.233 ms against 0.238 for 512 x 16)
    {32, 0, 28, 8, 0},   // 2^28 u32 keys: 256 x 32 (2.78 ms against 2.88 for 384 x 32)
    {32, 32, 26, 8, 0},  // 2^26 u32 pairs: 256 x 20
    {64, 0, 25, 8, 0},   // 2^25 u64 keys: 256 x 20
};

int size_bucket(int64_t n) {
  int b = 0;
  while (b < 62 && (int64_t(2) << b) <= n) ++b;
  return b;
}

// Nearest bucket of `m` to `bucket` (the lower one on a tie) among entries of
// radix width `radix_bits` (0: any width); null if there is none.
const AutoChoice* nearest(const std::map<int, AutoChoice>& m, int bucket, int radix_bits) {
  const AutoChoice* best = nullptr;
  int dist = 1 << 30;
  for (const auto& kv : m) {
    if (radix_bits && kv.second.radix_bits != radix_bits) continue;
    const int d = kv.first > bucket ? kv.first - bucket : bucket - kv.first;
    if (d < dist) {
      dist = d;
      best = &kv.second;
    }
  }
  return best;
}

// The automatic choice for n keys of these widths, among entries of width
// radix_bits (0: any): a runtime entry, else a built-in one; null if neither.
const AutoChoice* auto_choice(int key_bits, int val_bits, int64_t n, int radix_bits) {
  static std::map<std::pair<int, int>, std::map<int, AutoChoice>> builtin;
  if (builtin.empty())
    for (const BuiltinChoice& b : kBuiltinAuto)
      builtin[{b.key_bits, b.val_bits}][b.bucket] = AutoChoice{b.radix_bits, b.variant};
  const int bucket = size_bucket(n);
  for (auto* table : {&g_auto, &builtin}) {
    auto it = table->find({key_bits, val_bits});
    if (it == table->end()) continue;
    if (const AutoChoice* c = nearest(it->second, bucket, radix_bits)) return c;
  }
  return nullptr;
}

// Radix width and variant of a sort of n keys (caller holds g_mu). radix_bits
// 0: the automatic choice (radix 256, variant 0 when nothing is known).
// Otherwise that width, with the variant fixed by isort_tune_set if any, else
// the variant of the nearest automatic entry of that width, else variant 0.
AutoChoice resolve(int key_bits, int val_bits, int radix_bits, int64_t n) {
  if (radix_bits == 0) {
    const AutoChoice* a = auto_choice(key_bits, val_bits, n, 0);
    radix_bits = a ? a->radix_bits : 8;
  }
  AutoChoice c{radix_bits, 0};
  auto it = g_variant.find({key_bits, val_bits, radix_bits});
  if (it != g_variant.end()) {
    c.variant = it->second;
  } else if (const AutoChoice* a = auto_choice(key_bits, val_bits, n, radix_bits)) {
    c.variant = a->variant;
  }
  return c;
}

const LsdEntry* pick(int key_bits, int val_bits, int radix_bits, int64_t n) {
  const AutoChoice c = resolve(key_bits, val_bits, radix_bits, n);
  const LsdEntry* tab = nullptr;
  int nv = variants(key_bits, val_bits, c.radix_bits, &tab);
  if (nv <= 0) return nullptr;
  int v = c.variant;
  if (v < 0 || v >= nv) v = 0;
  return &tab[v];
}

// Workspace layout of one LSD sort. The error word sits at offset 0 so it
// survives from call to call on the same workspace.
struct Layout {
  size_t err, hist, base, skip, counters, claim, status0, status1, alt_k, alt_v, total;
};

Layout layout_for(const LsdEntry& e, int64_t n) {
  Layout L;
  const int64_t tiles = (n + e.tile - 1) / e.tile + e.extra_status_rows;
  size_t off = 0;
  L.err = off;       off = align256(off + 4);
  L.hist = off;      off = align256(off + sizeof(uint32_t) * e.passes * e.radix);
  L.base = off;      off = align256(off + sizeof(uint32_t) * e.passes * e.radix);
  L.skip = off;      off = align256(off + sizeof(uint32_t) * e.passes);
  L.counters = off;  off = align256(off + sizeof(uint32_t) * e.passes);
  // the first round's cursors: R (plus 256 for a wide radix's two order-free steps)
  L.claim = off;     off = align256(off + sizeof(uint32_t) * (e.radix + 256));
  L.status0 = off;   off = align256(off + sizeof(uint32_t) * e.status_words_per_tile * tiles);
  L.status1 = off;
  if (e.status_buffers > 1)
    off = align256(off + sizeof(uint32_t) * e.status_words_per_tile * tiles);
  L.alt_k = off;     off = align256(off + (size_t)n * (e.key_bits / 8));
  L.alt_v = off;     off = align256(off + (size_t)n * (e.val_bits / 8));
  L.total = off;
  return L;
}

// Returns the stream's workspace with at least `need` bytes (caller holds g_mu).
isort_status acquire(cudaStream_t st, size_t need, void** out) {
  Workspace& w = g_ws[st];
  if (w.base && w.bytes >= need) {
    *out = w.base;
    return ISORT_OK;
  }
  if (w.base && !w.owned) return ISORT_ENOMEM;  // bound by the caller and too small
  size_t want = need + need / 8;                // grow with some slack
  void* p = nullptr;
  if (cudaMallocAsync(&p, want, st) != cudaSuccess) {
    cudaGetLastError();
    return ISORT_ENOMEM;
  }
  if (w.base) {  // carry the latched error word over, then release the old block
    cudaMemcpyAsync(p, w.base, 4, cudaMemcpyDeviceToDevice, st);
    cudaFreeAsync(w.base, st);
  } else {
    cudaMemsetAsync(p, 0, 4, st);
  }
  w.base = p;
  w.bytes = want;
  w.owned = true;
  *out = p;
  return ISORT_OK;
}

bool aligned(const void* p, int bytes) { return (reinterpret_cast<uintptr_t>(p) % bytes) == 0; }

// ---- segmented sort workspace ----
std::map<std::pair<int, int>, int64_t> g_seg_btn_max;  // (key_bits, val_bits) -> threshold
// Keys per segmented batch, exclusive: each radix tile records its first key
// in 40 bits.
constexpr int64_t kSegMaxKeys = int64_t(1) << 40;
std::map<std::pair<int, int>, int> g_seg_network;      // (key_bits, val_bits) -> ISORT_NET_*

// Longest range that takes the BTN path: the tuned threshold, capped by the
// capacity of the 256-thread BTN class (256 threads x cta_m keys).
int64_t seg_btn_max(const SegConfig& c) {
  const int64_t cap = 256LL * c.cta_m;
  auto it = g_seg_btn_max.find({c.key_bits, c.val_bits});
  int64_t v = it == g_seg_btn_max.end() ? cap : it->second;
  if (v > cap) v = cap;
  if (v < 64LL * c.mid_m) v = 64LL * c.mid_m;
  return v;
}

struct SegLayout {
  size_t err, cnt, lists, slot_first, tile_slot, seg_hist, seg_base, seg_skip, seg_claim, tile_info,
      status0, status1,
      alt_k, alt_v, total;
  int64_t max_tiles;
};

SegLayout seg_layout(const SegConfig& c, int64_t nseg, int64_t total, int64_t btn_max) {
  SegLayout L;
  // radix ranges are longer than btn_max, so there are at most total/(btn_max+1)
  int64_t slots = total / (btn_max + 1);
  if (slots > nseg) slots = nseg;
  if (slots < 1) slots = 1;
  L.max_tiles = total / c.tile + slots + 1;
  const size_t per_slot = sizeof(uint32_t) * (size_t)c.passes * c.radix;
  size_t off = 0;
  L.err = off;         off = align256(off + 4);
  L.cnt = off;         off = align256(off + sizeof(uint32_t) * kCntWords);
  L.lists = off;       off = align256(off + sizeof(int32_t) * 4 * (size_t)nseg);
  L.slot_first = off;  off = align256(off + sizeof(uint32_t) * (size_t)nseg);
  L.tile_slot = off;   off = align256(off + sizeof(int32_t) * (size_t)L.max_tiles);
  L.seg_hist = off;    off = align256(off + per_slot * (size_t)nseg);
  L.seg_base = off;    off = align256(off + per_slot * (size_t)nseg);
  L.seg_skip = off;    off = align256(off + sizeof(uint32_t) * (size_t)c.passes * nseg);
  L.seg_claim = off;   off = align256(off + sizeof(uint32_t) * (size_t)c.radix * nseg);
  L.tile_info = off;   off = align256(off + sizeof(uint64_t) * (size_t)L.max_tiles);
  L.status0 = off;     off = align256(off + sizeof(uint32_t) * c.radix * (size_t)L.max_tiles);
  L.status1 = off;     off = align256(off + sizeof(uint32_t) * c.radix * (size_t)L.max_tiles);
  L.alt_k = off;       off = align256(off + (size_t)total * (c.key_bits / 8));
  L.alt_v = off;       off = align256(off + (size_t)total * (c.val_bits / 8));
  L.total = off;
  return L;
}

isort_status check_widths(int key_bits, int val_bits, bool pairs) {
  if (key_bits != 32 && key_bits != 64) return ISORT_EINVAL;
  if (pairs && val_bits != 32 && val_bits != 64) return ISORT_EINVAL;
  return ISORT_OK;
}

isort_status resolve_radix(int radix_bits, int* out) {
  if (radix_bits != 0 && radix_bits != 8 && radix_bits != 11 && radix_bits != 16) {
    if (radix_bits > 0 && radix_bits <= 24) return ISORT_EUNSUPPORTED;
    return ISORT_EINVAL;
  }
  *out = radix_bits;
  return ISORT_OK;
}

// Host buffers of a host-buffer sort: inputs copied to the device, results back.
struct HostIo {
  const void* keys_in;
  const void* vals_in;  // null: keys only
  void* keys_out;
  void* vals_out;
};

// One LSD sort of device keys[0..n) (and vals). With io, keys and vals are
// ignored: the sort runs on device copies of io's inputs, placed in the
// stream's workspace after the sort's own layout, and writes io's outputs.
isort_status run_lsd(void* keys, void* vals, int64_t n, int key_bits, int val_bits,
                     int radix_bits, cudaStream_t st, const HostIo* io = nullptr) {
  std::lock_guard<std::mutex> lock(g_mu);
  const LsdEntry* e = pick(key_bits, val_bits, radix_bits, n);
  if (!e) return ISORT_EUNSUPPORTED;
  Layout L = layout_for(*e, n);
  const size_t kbytes = (size_t)n * (key_bits / 8), vbytes = (size_t)n * (val_bits / 8);
  size_t total = L.total, dev_k = 0, dev_v = 0;
  if (io) {
    dev_k = total;
    total = align256(dev_k + kbytes);
    if (io->vals_in) {
      dev_v = total;
      total = align256(dev_v + vbytes);
    }
  }
  void* ws = nullptr;
  isort_status s = acquire(st, total, &ws);
  if (s != ISORT_OK) return s;
  char* b = static_cast<char*>(ws);
  if (io) {
    keys = b + dev_k;
    vals = io->vals_in ? b + dev_v : nullptr;
  }
  LsdArgs a;
  a.keys = keys;
  a.vals = vals;
  a.alt_keys = b + L.alt_k;
  a.alt_vals = vals ? b + L.alt_v : nullptr;
  a.n = n;
  a.hist = reinterpret_cast<uint32_t*>(b + L.hist);
  a.base = reinterpret_cast<uint32_t*>(b + L.base);
  a.skip = reinterpret_cast<uint32_t*>(b + L.skip);
  a.counters = reinterpret_cast<uint32_t*>(b + L.counters);
  a.claim = reinterpret_cast<uint32_t*>(b + L.claim);
  a.status[0] = reinterpret_cast<uint32_t*>(b + L.status0);
  a.status[1] = reinterpret_cast<uint32_t*>(b + L.status1);
  a.err = reinterpret_cast<uint32_t*>(b + L.err);
  a.spin_limit = g_spin_limit;
  a.stall_tile = g_stall_tile;
  g_stall_tile = -1;  // the stall hook applies to one sort only
  a.num_sms = num_sms();
  a.prefetch_tiles = g_prefetch < 0 ? (int64_t)a.num_sms * 4 : g_prefetch;
  a.check_mode = g_check_mode;
  a.timer = nullptr;
  if (g_timing) {
    if (!g_timer.ready) {
      for (int i = 0; i < 2 * KernelTimer::kMax; ++i) cudaEventCreate(&g_timer.ev[i]);
      g_timer.ready = true;
    }
    g_timer.count = 0;
    a.timer = &g_timer;
  }
  cudaError_t ce = cudaSuccess;
  if (io) {
    ce = copy_host_io(keys, io->keys_in, kbytes, true, g_host_copy, a.num_sms, a.timer, st);
    if (ce == cudaSuccess && vals)
      ce = copy_host_io(vals, io->vals_in, vbytes, true, g_host_copy, a.num_sms, a.timer, st);
  }
  if (ce == cudaSuccess) ce = e->launch(a, st);
  if (io && ce == cudaSuccess) {
    ce = copy_host_io(io->keys_out, keys, kbytes, false, g_host_copy, a.num_sms, a.timer, st);
    if (ce == cudaSuccess && vals)
      ce = copy_host_io(io->vals_out, vals, vbytes, false, g_host_copy, a.num_sms, a.timer, st);
  }
  return ce == cudaSuccess ? ISORT_OK : ISORT_ECUDA;
}

}  // namespace

namespace isort {

std::atomic<int64_t> g_launch_count{0};  // every kernel the library enqueues

void timer_begin(KernelTimer* t, const char* name, cudaStream_t st) {
  g_launch_count.fetch_add(1, std::memory_order_relaxed);  // each launch is preceded by this call
  if (!t || t->count >= KernelTimer::kMax) return;
  t->name[t->count] = name;
  cudaEventRecord(t->ev[2 * t->count], st);
}

void timer_end(KernelTimer* t, cudaStream_t st) {
  if (!t || t->count >= KernelTimer::kMax) return;
  cudaEventRecord(t->ev[2 * t->count + 1], st);
  ++t->count;
}

}  // namespace isort

namespace {

// Segmented-sort arguments over workspace b laid out by L (caller holds g_mu).
SegArgs seg_args(const SegConfig& c, const SegLayout& L, char* b, void* keys, void* vals,
                 const int64_t* offsets, int64_t nseg, int64_t total) {
  SegArgs a;
  a.keys = keys;
  a.vals = vals;
  a.alt_keys = b + L.alt_k;
  a.alt_vals = vals ? b + L.alt_v : nullptr;
  a.offsets = offsets;
  a.nseg = nseg;
  a.total = total;
  a.btn_max = seg_btn_max(c);
  {
    auto it = g_seg_network.find({c.key_bits, c.val_bits});
    a.network = it == g_seg_network.end() ? ISORT_NET_BTN : it->second;
  }
  a.max_tiles = L.max_tiles;
  a.lists = reinterpret_cast<int32_t*>(b + L.lists);
  a.cnt = reinterpret_cast<uint32_t*>(b + L.cnt);
  a.slot_first = reinterpret_cast<uint32_t*>(b + L.slot_first);
  a.tile_slot = reinterpret_cast<int32_t*>(b + L.tile_slot);
  a.seg_hist = reinterpret_cast<uint32_t*>(b + L.seg_hist);
  a.seg_base = reinterpret_cast<uint32_t*>(b + L.seg_base);
  a.seg_skip = reinterpret_cast<uint32_t*>(b + L.seg_skip);
  a.seg_claim = reinterpret_cast<uint32_t*>(b + L.seg_claim);
  a.tile_info = reinterpret_cast<uint64_t*>(b + L.tile_info);
  a.status[0] = reinterpret_cast<uint32_t*>(b + L.status0);
  a.status[1] = reinterpret_cast<uint32_t*>(b + L.status1);
  a.err = reinterpret_cast<uint32_t*>(b + L.err);
  a.spin_limit = g_spin_limit;
  a.num_sms = num_sms();
  a.check_mode = g_check_mode;
  a.agg_top = 0;
  a.timer = nullptr;
  if (g_timing) {
    if (!g_timer.ready) {
      for (int i = 0; i < 2 * KernelTimer::kMax; ++i) cudaEventCreate(&g_timer.ev[i]);
      g_timer.ready = true;
    }
    g_timer.count = 0;
    a.timer = &g_timer;
  }
  return a;
}

// Sample-sort workspace: the segmented-sort layout of the p buckets (error word
// at offset 0), then the bucketed copy of the input and the split round's arrays.
struct GvrLayout {
  SegLayout seg;
  size_t out_k, out_v, split, cell, hist, base, skip, counter, status, claim, offsets, total;
};

GvrLayout gvr_layout(const SegConfig& c, int64_t n, int buckets) {
  GvrLayout G;
  G.seg = seg_layout(c, buckets, n, seg_btn_max(c));
  const int64_t tiles = (n + gvr_tile(c.key_bits, c.val_bits) - 1) / gvr_tile(c.key_bits, c.val_bits);
  size_t off = G.seg.total;
  G.out_k = off;    off = align256(off + (size_t)n * (c.key_bits / 8));
  G.out_v = off;    off = align256(off + (size_t)n * (c.val_bits / 8));
  G.split = off;    off = align256(off + 255 * sizeof(uint64_t));
  G.cell = off;     off = align256(off + 1024 * sizeof(uint16_t));
  G.hist = off;     off = align256(off + 256 * sizeof(uint32_t));
  G.base = off;     off = align256(off + 256 * sizeof(uint32_t));
  G.skip = off;     off = align256(off + sizeof(uint32_t));
  G.counter = off;  off = align256(off + sizeof(uint32_t));
  G.status = off;   off = align256(off + sizeof(uint32_t) * 256 * (size_t)tiles);
  G.claim = off;    off = align256(off + 256 * sizeof(uint32_t));
  G.offsets = off;  off = align256(off + sizeof(int64_t) * (size_t)(buckets + 1));
  G.total = off;
  return G;
}

// GSD workspace: the segmented-sort layout of the p sequences (error word at
// offset 0; its alternate buffers serve the merge rounds too), then the
// sequence offsets, splitters and the split and merge plans.
struct GsdLayout {
  SegLayout seg;
  size_t off, split, bound, pre, bucket_off, pair_info, pair_tile, cut, total;
};

GsdLayout gsd_layout(const SegConfig& c, int64_t n, int p) {
  GsdLayout L;
  L.seg = seg_layout(c, p, n, seg_btn_max(c));
  const size_t pp1 = sizeof(int64_t) * (size_t)p * (p + 1);
  const size_t pairs = (size_t)p * p / 2 + 1;
  size_t o = L.seg.total;
  L.off = o;         o = align256(o + sizeof(int64_t) * (p + 1));
  L.split = o;       o = align256(o + sizeof(uint64_t) * (p > 1 ? p - 1 : 1));
  L.bound = o;       o = align256(o + pp1);
  L.pre = o;         o = align256(o + pp1);
  L.bucket_off = o;  o = align256(o + sizeof(int64_t) * (p + 1));
  L.pair_info = o;   o = align256(o + sizeof(int64_t) * 5 * pairs);
  L.pair_tile = o;   o = align256(o + sizeof(int64_t) * (pairs + 1));
  L.cut = o;         o = align256(o + sizeof(int64_t) * (size_t)(n / kGsdMinMergeTile + (int64_t)p * p + 2));
  L.total = o;
  return L;
}

isort_status check_gsd_args(int64_t n, int key_bits, int val_bits, bool pairs, int buckets,
                            int oversample) {
  isort_status s = check_widths(key_bits, val_bits, pairs);
  if (s != ISORT_OK) return s;
  if (n < 0 || buckets < 1 || buckets > 64 || (buckets & (buckets - 1)) || oversample < 1 ||
      (int64_t)oversample * buckets * buckets > 4096)
    return ISORT_EINVAL;
  if (n > (int64_t(1) << 30)) return ISORT_EUNSUPPORTED;
  return ISORT_OK;
}

isort_status check_sample_args(int64_t n, int key_bits, int val_bits, bool pairs, int buckets,
                               int oversample) {
  isort_status s = check_widths(key_bits, val_bits, pairs);
  if (s != ISORT_OK) return s;
  if (n < 0 || buckets < 1 || buckets > 256 || oversample < 1 ||
      (int64_t)buckets * oversample > 4096)
    return ISORT_EINVAL;
  if (n > (int64_t(1) << 30)) return ISORT_EUNSUPPORTED;
  return ISORT_OK;
}

}  // namespace

extern "C" {

isort_status isort_keys(void* keys, int64_t n, int key_bits, int radix_bits, void* stream) {
  isort_status s = check_widths(key_bits, 0, false);
  if (s != ISORT_OK) return s;
  int rb = 0;
  if ((s = resolve_radix(radix_bits, &rb)) != ISORT_OK) return s;
  if (n < 0) return ISORT_EINVAL;
  if (n > kMaxN) return ISORT_EUNSUPPORTED;
  if (n <= 1) return ISORT_OK;
  if (!keys || !aligned(keys, key_bits / 8)) return ISORT_EINVAL;
  return run_lsd(keys, nullptr, n, key_bits, 0, rb, static_cast<cudaStream_t>(stream));
}

isort_status isort_pairs(void* keys, void* vals, int64_t n, int key_bits, int val_bits,
                         int radix_bits, void* stream) {
  isort_status s = check_widths(key_bits, val_bits, true);
  if (s != ISORT_OK) return s;
  int rb = 0;
  if ((s = resolve_radix(radix_bits, &rb)) != ISORT_OK) return s;
  if (n < 0) return ISORT_EINVAL;
  if (n > kMaxN) return ISORT_EUNSUPPORTED;
  if (n <= 1) return ISORT_OK;
  if (!keys || !vals || !aligned(keys, key_bits / 8) || !aligned(vals, val_bits / 8))
    return ISORT_EINVAL;
  return run_lsd(keys, vals, n, key_bits, val_bits, rb, static_cast<cudaStream_t>(stream));
}

isort_status isort_keys_host(const void* keys_in, void* keys_out, int64_t n, int key_bits,
                             int radix_bits, void* stream) {
  isort_status s = check_widths(key_bits, 0, false);
  if (s != ISORT_OK) return s;
  int rb = 0;
  if ((s = resolve_radix(radix_bits, &rb)) != ISORT_OK) return s;
  if (n < 0) return ISORT_EINVAL;
  if (n > kMaxN) return ISORT_EUNSUPPORTED;
  if (n == 0) return ISORT_OK;
  if (!keys_in || !keys_out || !aligned(keys_in, key_bits / 8) || !aligned(keys_out, key_bits / 8))
    return ISORT_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n == 1) {
    if (keys_in == keys_out) return ISORT_OK;
    return cudaMemcpyAsync(keys_out, keys_in, key_bits / 8, cudaMemcpyDefault, st) == cudaSuccess
               ? ISORT_OK
               : ISORT_ECUDA;
  }
  const HostIo io{keys_in, nullptr, keys_out, nullptr};
  return run_lsd(nullptr, nullptr, n, key_bits, 0, rb, st, &io);
}

isort_status isort_pairs_host(const void* keys_in, const void* vals_in, void* keys_out,
                              void* vals_out, int64_t n, int key_bits, int val_bits,
                              int radix_bits, void* stream) {
  isort_status s = check_widths(key_bits, val_bits, true);
  if (s != ISORT_OK) return s;
  int rb = 0;
  if ((s = resolve_radix(radix_bits, &rb)) != ISORT_OK) return s;
  if (n < 0) return ISORT_EINVAL;
  if (n > kMaxN) return ISORT_EUNSUPPORTED;
  if (n == 0) return ISORT_OK;
  if (!keys_in || !keys_out || !vals_in || !vals_out || !aligned(keys_in, key_bits / 8) ||
      !aligned(keys_out, key_bits / 8) || !aligned(vals_in, val_bits / 8) ||
      !aligned(vals_out, val_bits / 8))
    return ISORT_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n == 1) {
    if (keys_in != keys_out &&
        cudaMemcpyAsync(keys_out, keys_in, key_bits / 8, cudaMemcpyDefault, st) != cudaSuccess)
      return ISORT_ECUDA;
    if (vals_in != vals_out &&
        cudaMemcpyAsync(vals_out, vals_in, val_bits / 8, cudaMemcpyDefault, st) != cudaSuccess)
      return ISORT_ECUDA;
    return ISORT_OK;
  }
  const HostIo io{keys_in, vals_in, keys_out, vals_out};
  return run_lsd(nullptr, nullptr, n, key_bits, val_bits, rb, st, &io);
}

isort_status isort_sample_sort(void* keys, void* vals, int64_t n, int key_bits, int val_bits,
                               int buckets, int oversample, uint64_t seed,
                               uint32_t* bucket_counts, void* stream) {
  if (!vals) val_bits = 0;
  isort_status s = check_sample_args(n, key_bits, val_bits, vals != nullptr, buckets, oversample);
  if (s != ISORT_OK) return s;
  if (n == 0) return ISORT_OK;
  if (!keys || !aligned(keys, key_bits / 8) || (vals && !aligned(vals, val_bits / 8)) ||
      (bucket_counts && !aligned(bucket_counts, 4)))
    return ISORT_EINVAL;
  const SegConfig* c = key_bits == 32 ? seg_config_k32(val_bits) : seg_config_k64(val_bits);
  if (!c) return ISORT_EUNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mu);
  const GvrLayout G = gvr_layout(*c, n, buckets);
  void* ws = nullptr;
  if ((s = acquire(st, G.total, &ws)) != ISORT_OK) return s;
  char* b = static_cast<char*>(ws);
  SegArgs sa = seg_args(*c, G.seg, b, b + G.out_k, vals ? b + G.out_v : nullptr,
                        reinterpret_cast<const int64_t*>(b + G.offsets), buckets, n);
  // inside a bucket of many the top byte takes one or two values
  sa.agg_top = buckets >= 128;
  GvrArgs g;
  g.keys = keys;
  g.vals = vals;
  g.out_keys = b + G.out_k;
  g.out_vals = vals ? b + G.out_v : nullptr;
  g.n = n;
  g.buckets = buckets;
  g.oversample = oversample;
  g.seed = seed;
  g.split = b + G.split;
  g.cell = b + G.cell;
  g.hist = reinterpret_cast<uint32_t*>(b + G.hist);
  g.base = reinterpret_cast<uint32_t*>(b + G.base);
  g.skip = reinterpret_cast<uint32_t*>(b + G.skip);
  g.counter = reinterpret_cast<uint32_t*>(b + G.counter);
  g.status = reinterpret_cast<uint32_t*>(b + G.status);
  g.claim = reinterpret_cast<uint32_t*>(b + G.claim);
  g.offsets = reinterpret_cast<int64_t*>(b + G.offsets);
  g.counts_out = bucket_counts;
  g.err = sa.err;
  g.spin_limit = g_spin_limit;
  g.num_sms = sa.num_sms;
  g.timer = sa.timer;
  if (gvr_split_launch(key_bits, val_bits, g, st) != cudaSuccess) return ISORT_ECUDA;
  // the buckets, each sorted independently, in place in the workspace copy
  if (c->launch(sa, st) != cudaSuccess) return ISORT_ECUDA;
  if (cudaMemcpyAsync(keys, g.out_keys, (size_t)n * (key_bits / 8), cudaMemcpyDeviceToDevice,
                      st) != cudaSuccess)
    return ISORT_ECUDA;
  if (vals && cudaMemcpyAsync(vals, g.out_vals, (size_t)n * (val_bits / 8),
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return ISORT_ECUDA;
  return ISORT_OK;
}

isort_status isort_gsd_sort(void* keys, void* vals, int64_t n, int key_bits, int val_bits,
                            int buckets, int oversample, uint32_t* bucket_counts, void* stream) {
  if (!vals) val_bits = 0;
  isort_status s = check_gsd_args(n, key_bits, val_bits, vals != nullptr, buckets, oversample);
  if (s != ISORT_OK) return s;
  if (n == 0) return ISORT_OK;
  if (!keys || !aligned(keys, key_bits / 8) || (vals && !aligned(vals, val_bits / 8)) ||
      (bucket_counts && !aligned(bucket_counts, 4)))
    return ISORT_EINVAL;
  const SegConfig* c = key_bits == 32 ? seg_config_k32(val_bits) : seg_config_k64(val_bits);
  if (!c) return ISORT_EUNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mu);
  const GsdLayout L = gsd_layout(*c, n, buckets);
  void* ws = nullptr;
  if ((s = acquire(st, L.total, &ws)) != ISORT_OK) return s;
  char* b = static_cast<char*>(ws);
  int64_t* off = reinterpret_cast<int64_t*>(b + L.off);
  // 1. LocalSorting of the p sequences, in place
  if (gsd_offsets_launch(n, buckets, off, st) != cudaSuccess) return ISORT_ECUDA;
  SegArgs sa = seg_args(*c, L.seg, b, keys, vals, off, buckets, n);
  if (c->launch(sa, st) != cudaSuccess) return ISORT_ECUDA;
  // 2-5. sample, splitters, split, lg p merge rounds
  GsdArgs g;
  g.keys = keys;
  g.vals = vals;
  g.alt_keys = b + L.seg.alt_k;
  g.alt_vals = vals ? b + L.seg.alt_v : nullptr;
  g.n = n;
  g.buckets = buckets;
  g.oversample = oversample;
  g.split = b + L.split;
  g.bound = reinterpret_cast<int64_t*>(b + L.bound);
  g.pre = reinterpret_cast<int64_t*>(b + L.pre);
  g.bucket_off = reinterpret_cast<int64_t*>(b + L.bucket_off);
  g.pair_info = reinterpret_cast<int64_t*>(b + L.pair_info);
  g.pair_tile = reinterpret_cast<int64_t*>(b + L.pair_tile);
  g.cut = reinterpret_cast<int64_t*>(b + L.cut);
  g.counts_out = bucket_counts;
  g.err = sa.err;
  g.timer = sa.timer;
  return gsd_merge_launch(key_bits, val_bits, g, st) == cudaSuccess ? ISORT_OK : ISORT_ECUDA;
}

isort_status isort_gsd_sort_workspace_size(int64_t n, int key_bits, int val_bits, int buckets,
                                           int oversample, size_t* bytes) {
  if (!bytes) return ISORT_EINVAL;
  isort_status s = check_gsd_args(n, key_bits, val_bits, val_bits != 0, buckets, oversample);
  if (s != ISORT_OK) return s;
  const SegConfig* c = key_bits == 32 ? seg_config_k32(val_bits) : seg_config_k64(val_bits);
  if (!c) return ISORT_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  *bytes = gsd_layout(*c, n, buckets).total;
  return ISORT_OK;
}

isort_status isort_sample_sort_workspace_size(int64_t n, int key_bits, int val_bits, int buckets,
                                              int oversample, size_t* bytes) {
  if (!bytes) return ISORT_EINVAL;
  isort_status s = check_sample_args(n, key_bits, val_bits, val_bits != 0, buckets, oversample);
  if (s != ISORT_OK) return s;
  const SegConfig* c = key_bits == 32 ? seg_config_k32(val_bits) : seg_config_k64(val_bits);
  if (!c) return ISORT_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  *bytes = gvr_layout(*c, n, buckets).total;
  return ISORT_OK;
}

isort_status isort_segmented(void* keys, void* vals, const int64_t* offsets, int64_t num_segments,
                             int64_t total_keys, int key_bits, int val_bits, int radix_bits,
                             void* stream) {
  if (!vals) val_bits = 0;
  isort_status s = check_widths(key_bits, val_bits, vals != nullptr);
  if (s != ISORT_OK) return s;
  if (radix_bits != 0 && radix_bits != 8)
    return (radix_bits > 0 && radix_bits <= 24) ? ISORT_EUNSUPPORTED : ISORT_EINVAL;
  if (num_segments < 0 || total_keys < 0 || num_segments > INT32_MAX) return ISORT_EINVAL;
  if (total_keys >= kSegMaxKeys) return ISORT_EINVAL;
  if (num_segments == 0 || total_keys == 0) return ISORT_OK;
  if (!offsets || !keys || !aligned(keys, key_bits / 8) ||
      (vals && !aligned(vals, val_bits / 8)) || !aligned(offsets, 8))
    return ISORT_EINVAL;
  const SegConfig* c = key_bits == 32 ? seg_config_k32(val_bits) : seg_config_k64(val_bits);
  if (!c) return ISORT_EUNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mu);
  SegLayout L = seg_layout(*c, num_segments, total_keys, seg_btn_max(*c));
  void* ws = nullptr;
  if ((s = acquire(st, L.total, &ws)) != ISORT_OK) return s;
  SegArgs a = seg_args(*c, L, static_cast<char*>(ws), keys, vals, offsets, num_segments,
                       total_keys);
  return c->launch(a, st) == cudaSuccess ? ISORT_OK : ISORT_ECUDA;
}

isort_status isort_tune_segmented(int key_bits, int val_bits, int64_t btn_max_keys) {
  if (key_bits != 32 && key_bits != 64) return ISORT_EINVAL;
  if (val_bits != 0 && val_bits != 32 && val_bits != 64) return ISORT_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (btn_max_keys < 0) {
    g_seg_btn_max.erase({key_bits, val_bits});
    return ISORT_OK;
  }
  g_seg_btn_max[{key_bits, val_bits}] = btn_max_keys;
  return ISORT_OK;
}

int64_t isort_debug_launch_count(void) {
  return isort::g_launch_count.load(std::memory_order_relaxed);
}

isort_status isort_tune_segmented_network(int key_bits, int val_bits, int network) {
  if (key_bits != 32 && key_bits != 64) return ISORT_EINVAL;
  if (val_bits != 0 && val_bits != 32 && val_bits != 64) return ISORT_EINVAL;
  if (network != ISORT_NET_BTN && network != ISORT_NET_OET) return ISORT_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  g_seg_network[{key_bits, val_bits}] = network;
  return ISORT_OK;
}

isort_status isort_segmented_workspace_size(int64_t num_segments, int64_t total_keys, int key_bits,
                                            int val_bits, size_t* bytes) {
  if (!bytes || num_segments < 0 || total_keys < 0 || total_keys >= kSegMaxKeys)
    return ISORT_EINVAL;
  isort_status s = check_widths(key_bits, val_bits, val_bits != 0);
  if (s != ISORT_OK) return s;
  const SegConfig* c = key_bits == 32 ? seg_config_k32(val_bits) : seg_config_k64(val_bits);
  if (!c) return ISORT_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  *bytes = seg_layout(*c, num_segments, total_keys, seg_btn_max(*c)).total;
  return ISORT_OK;
}

isort_status isort_workspace_size(int64_t n, int key_bits, int val_bits, int radix_bits,
                                  size_t* bytes) {
  if (!bytes) return ISORT_EINVAL;
  isort_status s = check_widths(key_bits, val_bits, val_bits != 0);
  if (s != ISORT_OK) return s;
  int rb = 0;
  if ((s = resolve_radix(radix_bits, &rb)) != ISORT_OK) return s;
  if (n < 0) return ISORT_EINVAL;
  if (n > kMaxN) return ISORT_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  const LsdEntry* e = pick(key_bits, val_bits, rb, n);
  if (!e) return ISORT_EUNSUPPORTED;
  *bytes = layout_for(*e, n).total;
  return ISORT_OK;
}

isort_status isort_set_workspace(void* dev_ptr, size_t bytes, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dev_ptr && (!aligned(dev_ptr, 256) || bytes < 256)) return ISORT_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_ws.find(st);
  if (it != g_ws.end() && it->second.owned && it->second.base)
    cudaFreeAsync(it->second.base, st);
  if (!dev_ptr) {
    g_ws.erase(st);
    return ISORT_OK;
  }
  Workspace w;
  w.base = dev_ptr;
  w.bytes = bytes;
  w.owned = false;
  g_ws[st] = w;
  return cudaMemsetAsync(dev_ptr, 0, 4, st) == cudaSuccess ? ISORT_OK : ISORT_ECUDA;
}

isort_status isort_stream_status(void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return ISORT_ECUDA;
  if (cudaGetLastError() != cudaSuccess) return ISORT_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_ws.find(st);
  if (it == g_ws.end() || !it->second.base) return ISORT_OK;
  uint32_t word = 0;
  if (cudaMemcpy(&word, it->second.base, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ISORT_ECUDA;
  if (word) {
    if (cudaMemset(it->second.base, 0, 4) != cudaSuccess) return ISORT_ECUDA;
    if (word & 1u) return ISORT_ETIMEOUT;  // a bounded wait gave up
    if (word & 4u) return ISORT_EINVAL;    // segment offsets were not a valid partition
    return ISORT_ECUDA;                    // an output index failed its bounds check
  }
  return ISORT_OK;
}

isort_status isort_release_workspaces(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  isort_status s = ISORT_OK;
  for (auto& kv : g_ws) {
    if (kv.second.owned && kv.second.base) {
      if (cudaFreeAsync(kv.second.base, kv.first) != cudaSuccess) s = ISORT_ECUDA;
      if (cudaStreamSynchronize(kv.first) != cudaSuccess) s = ISORT_ECUDA;
    }
  }
  g_ws.clear();
  return s;
}

const char* isort_strerror(isort_status s) {
  switch (s) {
    case ISORT_OK: return "ok";
    case ISORT_EINVAL: return "invalid argument";
    case ISORT_ENOMEM: return "out of device memory or workspace too small";
    case ISORT_ECUDA: return "CUDA runtime error";
    case ISORT_ETIMEOUT: return "bounded device wait gave up";
    case ISORT_EUNSUPPORTED: return "unsupported argument combination";
  }
  return "unknown status";
}

isort_status isort_tune_set(int key_bits, int val_bits, int radix_bits, int variant) {
  std::lock_guard<std::mutex> lock(g_mu);
  const LsdEntry* tab = nullptr;
  if (radix_bits == 0) radix_bits = 8;
  int nv = variants(key_bits, val_bits, radix_bits, &tab);
  if (variant == -1) {
    g_variant.erase({key_bits, val_bits, radix_bits});
    return ISORT_OK;
  }
  if (variant < 0 || variant >= nv) return ISORT_EINVAL;
  g_variant[{key_bits, val_bits, radix_bits}] = variant;
  return ISORT_OK;
}

int isort_tune_num_variants(int key_bits, int val_bits, int radix_bits) {
  const LsdEntry* tab = nullptr;
  if (radix_bits == 0) radix_bits = 8;
  return variants(key_bits, val_bits, radix_bits, &tab);
}

isort_status isort_tune_describe(int key_bits, int val_bits, int radix_bits, int variant,
                                 int* threads, int* keys_per_thread) {
  const LsdEntry* tab = nullptr;
  if (radix_bits == 0) radix_bits = 8;
  int nv = variants(key_bits, val_bits, radix_bits, &tab);
  if (variant < 0 || variant >= nv || !threads || !keys_per_thread) return ISORT_EINVAL;
  *threads = tab[variant].threads;
  *keys_per_thread = tab[variant].keys_per_thread;
  return ISORT_OK;
}

isort_status isort_tune_auto(int key_bits, int val_bits, int size_log2, int radix_bits,
                            int variant) {
  if (key_bits != 32 && key_bits != 64) return ISORT_EINVAL;
  if (val_bits != 0 && val_bits != 32 && val_bits != 64) return ISORT_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (radix_bits < 0) {  // clear one bucket, or every bucket of these widths
    auto it = g_auto.find({key_bits, val_bits});
    if (it == g_auto.end()) return ISORT_OK;
    if (size_log2 < 0)
      g_auto.erase(it);
    else
      it->second.erase(size_log2);
    return ISORT_OK;
  }
  if (size_log2 < 0 || size_log2 > 30) return ISORT_EINVAL;
  if (radix_bits != 8 && radix_bits != 11 && radix_bits != 16) return ISORT_EINVAL;
  const LsdEntry* tab = nullptr;
  const int nv = variants(key_bits, val_bits, radix_bits, &tab);
  if (variant < 0 || variant >= nv) return ISORT_EINVAL;
  g_auto[{key_bits, val_bits}][size_log2] = AutoChoice{radix_bits, variant};
  return ISORT_OK;
}

isort_status isort_tune_resolve(int64_t n, int key_bits, int val_bits, int radix_bits,
                               int* radix_out, int* variant_out) {
  if (!radix_out || !variant_out || n < 0) return ISORT_EINVAL;
  isort_status s = check_widths(key_bits, val_bits, val_bits != 0);
  if (s != ISORT_OK) return s;
  int rb = 0;
  if ((s = resolve_radix(radix_bits, &rb)) != ISORT_OK) return s;
  std::lock_guard<std::mutex> lock(g_mu);
  const AutoChoice c = resolve(key_bits, val_bits, rb, n);
  const LsdEntry* tab = nullptr;
  const int nv = variants(key_bits, val_bits, c.radix_bits, &tab);
  if (nv <= 0) return ISORT_EUNSUPPORTED;
  *radix_out = c.radix_bits;
  *variant_out = (c.variant >= 0 && c.variant < nv) ? c.variant : 0;
  return ISORT_OK;
}

int64_t isort_debug_workspace_bytes(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  int64_t total = 0;
  for (const auto& kv : g_ws)
    if (kv.second.owned && kv.second.base) total += (int64_t)kv.second.bytes;
  return total;
}

isort_status isort_debug_set(int what, int64_t value) {
  std::lock_guard<std::mutex> lock(g_mu);
  switch (what) {
    case ISORT_DEBUG_SPIN_LIMIT:
      if (value < 0 || value > 0xffffffffll) return ISORT_EINVAL;
      g_spin_limit = value ? (uint32_t)value : kDefaultSpinLimit;
      return ISORT_OK;
    case ISORT_DEBUG_STALL_TILE:
      g_stall_tile = value;
      return ISORT_OK;
    case ISORT_DEBUG_KERNEL_TIMING:
      g_timing = value != 0;
      return ISORT_OK;
    case ISORT_DEBUG_PREFETCH_TILES:
      g_prefetch = value;
      return ISORT_OK;
    case ISORT_DEBUG_CHECK_MODE:
      if (value < 0 || value > 2) return ISORT_EINVAL;
      g_check_mode = (uint32_t)value;
      return ISORT_OK;
    case ISORT_DEBUG_HOST_COPY:
      if (value < 0 || value > 2) return ISORT_EINVAL;
      g_host_copy = (int)value;
      return ISORT_OK;
  }
  return ISORT_EINVAL;
}

int isort_debug_kernel_times(const char** names, float* ms, int max) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_timer.ready) return 0;
  int n = g_timer.count < max ? g_timer.count : max;
  for (int i = 0; i < n; ++i) {
    if (names) names[i] = g_timer.name[i];
    if (ms) {
      if (cudaEventSynchronize(g_timer.ev[2 * i + 1]) != cudaSuccess ||
          cudaEventElapsedTime(&ms[i], g_timer.ev[2 * i], g_timer.ev[2 * i + 1]) != cudaSuccess)
        ms[i] = -1.0f;
    }
  }
  return n;
}

}  // extern "C"
