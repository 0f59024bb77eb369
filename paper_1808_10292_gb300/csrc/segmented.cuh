// Segmented sort: every range [offsets[s], offsets[s+1]) sorted independently.
//
// The paper's sample sorts (GSD, GER, GVR; Algorithms 1-3) end by splitting the
// keys into p ranges and sorting each on its own; here the ranges are given by
// the caller and thousands of them of very uneven length are sorted in one
// batch. Short ranges go to the paper's BTN merge-split network (btn.cuh), long
// ones to the radix-256 count-sort passes of onesweep.cuh, all ranges of a class
// in the same launch:
//
//   k_seg_classify  one thread per range: checks the offsets, puts the range on
//                   the list of its class (warp BTN, 64-thread BTN, 256-thread
//                   BTN, radix) and gives each radix range a block of tile ids.
//   k_seg_fill      tile id -> radix range.
//   k_seg_btn<Q,M>  persistent: Q threads with M keys each sort one range at a
//                   time, popped from the class list (Q = 32: one range per warp),
//                   with the BTN network or, if chosen, the OET network.
//   k_seg_hist      digit histograms of every radix range, all passes, one read.
//   k_seg_scan      per range and pass, exclusive digit bases.
//   k_seg_onesweep  one count-sort round over the tiles of ALL radix ranges; the
//                   look-back never crosses a range (the first tile of a range
//                   publishes its counts as inclusive). Keys only: pass 0 is the
//                   order-free round (onesweep_tile_first), later passes the
//                   ordered round (onesweep_tile_ordered).
//   k_seg_copy_back the ranges that executed an odd number of passes end in the
//                   alternate buffers: copied home.
// A pass whose digit is constant on a range is skipped for that range (its
// tiles return at once), so each range keeps its own buffer parity. Offsets
// are checked on the device; a bad range is skipped and flagged in the error
// word.
#pragma once
#include "btn.cuh"
#include "onesweep.cuh"

namespace isort {

constexpr uint32_t kErrOffsets = 4u;  // error bit: offsets not a valid partition

// Classes of ranges.
enum { kSegWarp = 0, kSegMid = 1, kSegCta = 2, kSegRadix = 3, kSegClasses = 4 };

// Per radix tile, one 64-bit word (tile_info): the tile's first key (an index
// into the whole batch, 40 bits), its number of keys (14 bits) and the
// range's skipped passes (bit 56 + q: pass q is skipped).
constexpr int kTileKeysShift = 40, kTileSkipShift = 56;
constexpr uint64_t kTileStartMask = (uint64_t(1) << kTileKeysShift) - 1;
constexpr uint64_t kTileKeysMask = 0x3fff;
constexpr int64_t kSegMaxTotal = int64_t(1) << kTileKeysShift;  // keys per batch, exclusive

__device__ __forceinline__ void seg_range(const int64_t* off, int64_t s, int64_t total,
                                          int64_t& start, int64_t& len) {
  int64_t a = off[s], b = off[s + 1];
  a = a < 0 ? 0 : (a > total ? total : a);
  b = b < a ? a : (b > total ? total : b);
  start = a;
  len = b - a;
}

// ---------------------------------------------------------------------------
template <int TILE>
__global__ void k_seg_classify(const int64_t* __restrict__ off, int64_t nseg, int64_t total,
                               int64_t warp_max, int64_t mid_max, int64_t btn_max,
                               int32_t* __restrict__ lists, uint32_t* __restrict__ cnt,
                               uint32_t* __restrict__ slot_first, uint32_t* err) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const int64_t a = off[s], b = off[s + 1];
  bool bad = b < a || a < 0 || b > total || (s == 0 && a != 0) || (s == nseg - 1 && b != total);
  int64_t start, len;
  seg_range(off, s, total, start, len);
  if (len > (int64_t(1) << 30)) bad = true;  // a range's counts must fit the 30-bit status
  if (bad) {
    atomicOr(err, kErrOffsets);
    return;  // skipped: never read or written
  }
  if (len <= 1) return;
  int c = len <= warp_max ? kSegWarp : len <= mid_max ? kSegMid : len <= btn_max ? kSegCta
                                                                                  : kSegRadix;
  const uint32_t idx = atomicAdd(&cnt[kCntClassLen + c], 1u);
  lists[(size_t)c * nseg + idx] = (int32_t)s;
  if (c == kSegRadix) slot_first[idx] = atomicAdd(&cnt[kCntTiles], (uint32_t)((len + TILE - 1) / TILE));
}

template <int TILE>
__global__ void __launch_bounds__(256) k_seg_fill(const int64_t* __restrict__ off, int64_t nseg,
                                                  int64_t total, const int32_t* __restrict__ lists,
                                                  const uint32_t* __restrict__ cnt,
                                                  const uint32_t* __restrict__ slot_first,
                                                  int32_t* __restrict__ tile_slot) {
  const uint32_t slot = blockIdx.x;
  if (slot >= cnt[kCntClassLen + kSegRadix]) return;
  int64_t start, len;
  seg_range(off, lists[(size_t)kSegRadix * nseg + slot], total, start, len);
  const int64_t tiles = (len + TILE - 1) / TILE;
  const uint32_t first = slot_first[slot];
  for (int64_t i = threadIdx.x; i < tiles; i += 256) tile_slot[first + i] = (int32_t)slot;
}

// ---------------------------------------------------------------------------
// Persistent BTN over one class list. Q = 32: every warp of the CTA sorts its
// own ranges; Q > 32: the CTA (Q threads) sorts one range at a time.
template <typename K, typename V, int Q, int M, int CTA>
struct BtnShape {
  static constexpr bool HV = HasVal<V>::value;
  static constexpr int GROUPS = CTA / Q;  // independent sorters per CTA
  static constexpr int CAP = Q * M;       // keys per range at most
  using VS = typename std::conditional<HV, V, uint32_t>::type;
  static constexpr size_t SMEM = (Q > 32 ? (sizeof(K) + sizeof(uint32_t)) * (size_t)CAP : 0) +
                                 (HV ? sizeof(VS) * (size_t)CAP * GROUPS : 0) + 16;
};

template <typename K, typename V, int Q, int M, int CTA, bool OET = false>
__global__ void __launch_bounds__(CTA) k_seg_btn(K* __restrict__ keys, V* __restrict__ vals,
                                                 const int64_t* __restrict__ off, int64_t nseg,
                                                 int64_t total, const int32_t* __restrict__ list,
                                                 uint32_t* __restrict__ cnt, int cls) {
  using S = BtnShape<K, V, Q, M, CTA>;
  constexpr bool HV = S::HV;
  constexpr bool STABLE = HV;  // keys-only: equal keys are indistinguishable
  extern __shared__ __align__(16) unsigned char smem[];
  K* sk = reinterpret_cast<K*>(smem);
  uint32_t* si = reinterpret_cast<uint32_t*>(smem + (Q > 32 ? sizeof(K) * S::CAP : 0));
  typename S::VS* sv = reinterpret_cast<typename S::VS*>(
      smem + (Q > 32 ? (sizeof(K) + sizeof(uint32_t)) * S::CAP : 0));
  __shared__ uint32_t s_pop;
  const int group = threadIdx.x / Q, t = threadIdx.x % Q;
  typename S::VS* my_sv = sv + (size_t)group * S::CAP;
  (void)my_sv;
  const uint32_t count = cnt[kCntClassLen + cls];
  while (true) {
    uint32_t idx;
    if constexpr (Q == 32) {
      if (t == 0) idx = atomicAdd(&cnt[kCntCursor + cls], 1u);
      idx = __shfl_sync(kFullMask, idx, 0);
    } else {
      if (threadIdx.x == 0) s_pop = atomicAdd(&cnt[kCntCursor + cls], 1u);
      __syncthreads();
      idx = s_pop;
      __syncthreads();
    }
    if (idx >= count) break;
    int64_t start, len;
    seg_range(off, list[idx], total, start, len);
    BtnItem<K, STABLE> x[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const int pos = i * Q + t;  // striped load: coalesced
      if (pos < len) {
        x[i].k = keys[start + pos];
        if constexpr (STABLE) x[i].i = (uint32_t)pos;
        if constexpr (HV) my_sv[pos] = vals[start + pos];
      } else {  // padding sorts after every real item
        x[i].k = ~K(0);
        if constexpr (STABLE) x[i].i = 0xffffffffu;
      }
    }
    btn_local_sort<STABLE>(x);
    if constexpr (OET)
      oet_network<STABLE, K, M, Q>(x, t, sk, si);
    else
      btn_network<STABLE, K, M, Q>(x, t, sk, si);
    if constexpr (HV) {
      if constexpr (Q == 32)
        __syncwarp();
      else
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const int pos = t * M + i;  // thread t holds sorted ranks [t*M, t*M + M)
      if (pos < len) {
        keys[start + pos] = x[i].k;
        if constexpr (HV) vals[start + pos] = my_sv[x[i].i];
      }
    }
    if constexpr (Q == 32)
      __syncwarp();
    else
      __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Digit histograms of the radix ranges: CTA c walks a contiguous run of tiles,
// counting into shared memory and flushing into seg_hist when the range
// changes. Long spans count into counters laid out as k_hist's, [p][d][lane %
// LANES], so one warp's atomics fall in different banks; the flush of those
// 128 KiB then costs little next to the span. A span shorter than kSegShortSpan
// keys counts into a compact [p][d] array instead (bank conflicts, but a flush
// of P*R words), so that many short ranges do not pay a full flush each. Keys
// are read as 16-byte vectors.
constexpr int64_t kSegShortSpan = 65536;

template <typename K, int BITS, int TILE, int LANES>
__global__ void __launch_bounds__(1024) k_seg_hist(const K* __restrict__ keys,
                                                   const int64_t* __restrict__ off, int64_t nseg,
                                                   int64_t total, const int32_t* __restrict__ list,
                                                   const uint32_t* __restrict__ cnt,
                                                   const uint32_t* __restrict__ slot_first,
                                                   const int32_t* __restrict__ tile_slot,
                                                   uint32_t* __restrict__ seg_hist) {
  using L = DigitLayout<K, BITS>;
  constexpr int R = L::R, P = L::PASSES;
  extern __shared__ __align__(16) uint32_t s_cnt[];  // [P][R][LANES], then [P][R]
  uint32_t* s_small = s_cnt + P * R * LANES;
  for (int i = threadIdx.x; i < P * R * (LANES + 1); i += 1024) s_cnt[i] = 0;
  const int64_t T = cnt[kCntTiles];
  const int64_t t0 = T * blockIdx.x / gridDim.x, t1 = T * (blockIdx.x + 1) / gridDim.x;
  uint32_t* my = s_cnt + (threadIdx.x & (LANES - 1));
  auto count = [&](K k) {
#pragma unroll
    for (int p = 0; p < P; ++p)
      atomicAdd(&my[(p * R + digit_of(k, p * BITS, (1u << L::width(p)) - 1)) * LANES], 1u);
  };
  auto count_small = [&](K k) {
#pragma unroll
    for (int p = 0; p < P; ++p)
      atomicAdd(&s_small[p * R + digit_of(k, p * BITS, (1u << L::width(p)) - 1)], 1u);
  };
  int32_t cur = -1;
  __syncthreads();
  auto flush = [&](int32_t slot) {  // the lane columns
    __syncthreads();
    for (int j = threadIdx.x; j < P * R; j += 1024) {
      uint32_t s = 0;
#pragma unroll 8
      for (int b = 0; b < LANES; ++b) {
        const int w = j * LANES + ((b + j) & (LANES - 1));
        s += s_cnt[w];
        s_cnt[w] = 0;
      }
      if (s) atomicAdd(&seg_hist[(size_t)slot * P * R + j], s);
    }
    __syncthreads();
  };
  // A range's tiles have consecutive ids and cover consecutive keys, so each
  // run of this CTA's tiles that belongs to one range is counted as one span
  // (long spans keep many 16-byte loads in flight per thread).
  for (int64_t t = t0; t < t1;) {
    const int32_t slot = tile_slot[t];
    int64_t start, len;
    seg_range(off, list[(size_t)kSegRadix * nseg + slot], total, start, len);
    const int64_t first = slot_first[slot];
    const int64_t t_end = min(t1, first + (len + TILE - 1) / TILE);
    const int64_t lo = start + (t - first) * TILE;
    const int64_t hi = min(start + len, start + (t_end - first) * TILE);
    if (hi - lo < kSegShortSpan) {
      count_keys(keys + lo, hi - lo, threadIdx.x, 1024, count_small);
      __syncthreads();
      for (int j = threadIdx.x; j < P * R; j += 1024) {
        const uint32_t c = s_small[j];
        if (c) {
          atomicAdd(&seg_hist[(size_t)slot * P * R + j], c);
          s_small[j] = 0;
        }
      }
      __syncthreads();
    } else {
      if (slot != cur) {
        if (cur >= 0) flush(cur);
        cur = slot;
      }
      count_keys(keys + lo, hi - lo, threadIdx.x, 1024, count);
    }
    t = t_end > t ? t_end : t + 1;
  }
  if (cur >= 0) flush(cur);
}

// Per radix range: exclusive digit bases (relative to the range) of every
// pass, and the range's trivial passes (one digit holds all its keys: the pass
// is the identity on that range and is skipped for it). Also zeroes the
// range's first-round output cursors (seg_claim, keys only; null otherwise)
// and writes, for each of its tiles, where the tile's keys start, how many
// there are and which passes the range skips (tile_info: the rounds take their
// tile from it, and prefetch the tile one wave ahead with it).
template <int BITS, int PASSES, int TILE>
__global__ void __launch_bounds__(1 << BITS) k_seg_scan(const uint32_t* __restrict__ cnt,
                                                       const uint32_t* __restrict__ seg_hist,
                                                       uint32_t* __restrict__ seg_base,
                                                       uint32_t* __restrict__ seg_skip,
                                                       uint32_t* __restrict__ seg_claim,
                                                       const int64_t* __restrict__ off,
                                                       int64_t nseg, int64_t total,
                                                       const int32_t* __restrict__ list,
                                                       const uint32_t* __restrict__ slot_first,
                                                       uint64_t* __restrict__ tile_info) {
  static_assert(PASSES <= 8 && TILE < 16384, "tile_info packs the start, keys and skip bits");
  constexpr int R = 1 << BITS;
  __shared__ uint32_t s_warp[R / 32];
  const uint32_t slot = blockIdx.x;
  if (slot >= cnt[kCntClassLen + kSegRadix]) return;
  if (seg_claim) seg_claim[(size_t)slot * R + threadIdx.x] = 0;
  uint32_t skips = 0;
  for (int p = 0; p < PASSES; ++p) {
    const size_t row = ((size_t)slot * PASSES + p) * R;
    uint32_t tot;
    const uint32_t c = seg_hist[row + threadIdx.x];
    seg_base[row + threadIdx.x] = block_exclusive_scan<R>(c, s_warp, tot);
    const int trivial = __syncthreads_or(c == tot);
    if (threadIdx.x == 0) seg_skip[(size_t)slot * PASSES + p] = trivial;
    skips |= (uint32_t)trivial << p;
  }
  int64_t start, len;
  seg_range(off, list[(size_t)kSegRadix * nseg + slot], total, start, len);
  const int64_t tiles = (len + TILE - 1) / TILE, first = slot_first[slot];
  for (int64_t lt = threadIdx.x; lt < tiles; lt += R) {
    const int64_t at = start + lt * TILE;  // below 2^40: the host refuses larger batches
    const int64_t n = min((int64_t)TILE, len - lt * TILE);
    tile_info[first + lt] =
        (uint64_t)at | ((uint64_t)n << kTileKeysShift) | ((uint64_t)skips << kTileSkipShift);
  }
}

// Input buffer of a radix range in pass `pass`: the parity of the passes
// executed for it before (0: the caller's arrays).
__device__ __forceinline__ int seg_src(const uint32_t* skip_row, int pass) {
  int src = 0;
  for (int q = 0; q < pass; ++q) src ^= (skip_row[q] == 0);
  return src;
}

// The same from a tile_info word's skip bits (bit q: pass q is skipped).
__device__ __forceinline__ int tile_src(uint32_t skips, int pass) {
  return __popc(~skips & ((1u << pass) - 1u)) & 1;
}

// After the last pass: the ranges that executed an odd number of passes end in
// the alternate buffers; copy them home (one tile per CTA iteration).
template <typename K, typename V, int TILE>
__global__ void __launch_bounds__(256) k_seg_copy_back(K* keys, const K* alt, V* vals,
                                                        const V* valt,
                                                        const int64_t* __restrict__ off,
                                                        int64_t nseg, int64_t total,
                                                        const int32_t* __restrict__ list,
                                                        const uint32_t* __restrict__ cnt,
                                                        const uint32_t* __restrict__ slot_first,
                                                        const int32_t* __restrict__ tile_slot,
                                                        const uint32_t* __restrict__ seg_skip,
                                                        int passes) {
  const int64_t T = cnt[kCntTiles];
  for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
    const int32_t slot = tile_slot[t];
    if (!seg_src(seg_skip + (size_t)slot * passes, passes)) continue;
    int64_t start, len;
    seg_range(off, list[(size_t)kSegRadix * nseg + slot], total, start, len);
    const int64_t lo = start + ((int64_t)t - slot_first[slot]) * TILE;
    const int64_t hi = min(start + len, lo + TILE);
    for (int64_t i = lo + threadIdx.x; i < hi; i += 256) {
      keys[i] = alt[i];
      if constexpr (HasVal<V>::value) vals[i] = valt[i];
    }
  }
}

// ---------------------------------------------------------------------------
struct SegPassParams {
  PassParams p;  // keys/vals buffers, pass, shift, mask, status, counter, err...
  const int64_t* off;
  int64_t nseg;
  int64_t total;
  const int32_t* list;
  const uint32_t* cnt;
  const uint32_t* slot_first;
  const int32_t* tile_slot;
  const uint32_t* seg_base;
  const uint32_t* seg_skip;  // [slots][passes] 1 = the pass is the identity on the range
  uint32_t* seg_claim;       // [slots][R] keys only: the first round's output cursors
  const uint64_t* tile_info;  // [tiles] first key | keys << 40 | skipped passes << 56
  int passes;
};

// One round over the tiles of every radix range: the ordered form, or with
// FIRST (keys only, pass 0) the order-free first round of onesweep_tile_first.
// AGG: the ordered form that reserves slots per digit value in tiles with few
// distinct digits (onesweep_tile_ordered), for passes whose digit is nearly
// constant inside each range.
template <typename K, typename V, int BITS, int THREADS, int KPT, int MINB, bool FIRST = false,
          bool AGG = false>
__global__ void __launch_bounds__(THREADS, MINB) k_seg_onesweep(SegPassParams sp) {
  static_assert(!FIRST || !HasVal<V>::value, "the order-free round is keys-only");
  using S = OnesweepShape<K, V, BITS, THREADS, KPT>;
  constexpr int R = S::R, WARPS = S::WARPS, TILE = S::TILE;
  const PassParams& p = sp.p;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_wcnt = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_misc = FIRST ? s_wcnt + 2 * R : s_wcnt + WARPS * R + R;
  const int tid = threadIdx.x;
  const uint32_t ntiles = sp.cnt[kCntTiles];  // read now, off the tile's chain of loads
  if (p.status_next)
    for (int d = tid; d < R; d += THREADS) p.status_next[(size_t)blockIdx.x * R + d] = 0;
  if (tid == 0) s_misc[0] = atomicAdd(p.counter, 1u);
  zero_words<THREADS>(s_wcnt, FIRST ? R : WARPS * R);
  __syncthreads();
  const uint32_t tile = s_misc[0];
  if (tile >= ntiles) return;  // more CTAs than tiles: nothing left
  // One word gives the tile's first key, its length and the range's skipped
  // passes, so the key loads wait on one load; the range (slot, start, length,
  // bases) is looked up while they are in flight.
  const uint64_t info = sp.tile_info[tile];
  const uint32_t skips = (uint32_t)(info >> kTileSkipShift);
  if ((skips >> p.pass) & 1u) return;  // the digit is constant on this range
  const int32_t slot = sp.tile_slot[tile];
  // The tile one wave ahead: thread 0 copies its tile_info word to shared
  // memory now (cp.async: no register, no wait) and prefetches its keys into
  // L2 when this tile is done.
  uint64_t* s_pf = reinterpret_cast<uint64_t*>(s_misc + 62);
  const uint32_t ahead = tile + (uint32_t)p.prefetch_tiles;
  const bool prefetch = tid == 0 && p.prefetch_tiles && ahead < sp.cnt[kCntTiles];
  if (prefetch) cp_async<8>(s_pf, sp.tile_info + ahead);
  int64_t start, len;
  seg_range(sp.off, sp.list[(size_t)kSegRadix * sp.nseg + slot], sp.total, start, len);
  const int64_t lt = (int64_t)tile - sp.slot_first[slot];  // tile index within the range
  const int64_t tile_base = (int64_t)(info & kTileStartMask);
  const int tile_n = (int)((info >> kTileKeysShift) & kTileKeysMask);
  const int src = tile_src(skips, p.pass);
  const K* kin = static_cast<const K*>(src ? p.keys[1] : p.keys[0]);
  K* kout = static_cast<K*>(src ? p.keys[0] : p.keys[1]) + start;
  const V* vin = static_cast<const V*>(src ? p.vals[1] : p.vals[0]);
  V* vout = static_cast<V*>(src ? p.vals[0] : p.vals[1]);
  if constexpr (HasVal<V>::value) vout += start;
  const uint32_t* base = sp.seg_base + ((size_t)slot * sp.passes + p.pass) * R;
  RadixDigit dig{p};
  if constexpr (FIRST) {
    // the range's tiles take their digit ranges from the range's cursors
    uint32_t* claim = sp.seg_claim + (size_t)slot * R;
    if (tile_n == TILE)
      onesweep_tile_first<K, BITS, THREADS, KPT, true>(p, tile, lt == 0, tile_base, tile_n, kin,
                                                       kout, base, (uint32_t)len, smem, dig,
                                                       claim);
    else
      onesweep_tile_first<K, BITS, THREADS, KPT, false>(p, tile, lt == 0, tile_base, tile_n, kin,
                                                        kout, base, (uint32_t)len, smem, dig,
                                                        claim);
  } else {
    if (tile_n == TILE)
      onesweep_tile_ordered<K, V, BITS, THREADS, KPT, true, RadixDigit, AGG>(
          p, tile, lt == 0, tile_base, tile_n, kin, kout, vin, vout, base, (uint32_t)len, smem,
          dig);
    else
      onesweep_tile_ordered<K, V, BITS, THREADS, KPT, false, RadixDigit, AGG>(
          p, tile, lt == 0, tile_base, tile_n, kin, kout, vin, vout, base, (uint32_t)len, smem,
          dig);
  }
  if (prefetch) {
    cp_async_wait_all();
    const uint64_t w = *s_pf;
    const int64_t at = (int64_t)(w & kTileStartMask);
    const int64_t n = (int64_t)((w >> kTileKeysShift) & kTileKeysMask);
    const uint32_t sk = (uint32_t)(w >> kTileSkipShift);
    if (!((sk >> p.pass) & 1u) && n && at + n <= sp.total) {
      const int s = tile_src(sk, p.pass);  // the buffer holding that tile now
      prefetch_tile(static_cast<const K*>(s ? p.keys[1] : p.keys[0]), at, n);
      if constexpr (HasVal<V>::value)
        prefetch_tile(static_cast<const V*>(s ? p.vals[1] : p.vals[0]), at, n);
    }
  }
}

// ---------------------------------------------------------------------------
template <typename K, typename V, int WM, int MM, int CM, int THREADS, int KPT, int MINB>
cudaError_t seg_launch(const SegArgs& a, cudaStream_t st) {
  using L = DigitLayout<K, 8>;
  using OS = OnesweepShape<K, V, 8, THREADS, KPT>;
  constexpr int R = L::R, P = L::PASSES, TILE = OS::TILE;
  cudaError_t e;
  const int64_t nslots = a.nseg;
  if (a.total >= kSegMaxTotal) return cudaErrorInvalidValue;  // tile_info holds 40-bit starts
  if ((e = cudaMemsetAsync(a.cnt, 0, sizeof(uint32_t) * kCntWords, st))) return e;
  if ((e = cudaMemsetAsync(a.seg_hist, 0, sizeof(uint32_t) * nslots * P * R, st))) return e;
  // status[0] serves pass 0 only with payloads (keys only, pass 0 takes cursors)
  if (HasVal<V>::value &&
      (e = cudaMemsetAsync(a.status[0], 0, sizeof(uint32_t) * R * a.max_tiles, st)))
    return e;
  if (a.nseg == 0) return cudaGetLastError();

  timer_begin(a.timer, "k_seg_classify", st);
  k_seg_classify<TILE><<<(unsigned)((a.nseg + 255) / 256), 256, 0, st>>>(
      a.offsets, a.nseg, a.total, 32 * WM, 64 * MM, a.btn_max, a.lists, a.cnt, a.slot_first,
      a.err);
  timer_end(a.timer, st);
  timer_begin(a.timer, "k_seg_fill", st);
  k_seg_fill<TILE><<<(unsigned)a.nseg, 256, 0, st>>>(a.offsets, a.nseg, a.total, a.lists, a.cnt,
                                                     a.slot_first, a.tile_slot);
  timer_end(a.timer, st);

  // short ranges: the three network classes, persistent grids
  K* keys = static_cast<K*>(a.keys);
  V* vals = static_cast<V*>(a.vals);
  {
    const bool oet = a.network == 1;
    using B0 = BtnShape<K, V, 32, WM, 256>;
    auto k0 = oet ? k_seg_btn<K, V, 32, WM, 256, true> : k_seg_btn<K, V, 32, WM, 256>;
    using B1 = BtnShape<K, V, 64, MM, 64>;
    auto k1 = oet ? k_seg_btn<K, V, 64, MM, 64, true> : k_seg_btn<K, V, 64, MM, 64>;
    using B2 = BtnShape<K, V, 256, CM, 256>;
    auto k2 = oet ? k_seg_btn<K, V, 256, CM, 256, true> : k_seg_btn<K, V, 256, CM, 256>;
    if ((e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B2::SMEM)))
      return e;
    timer_begin(a.timer, "k_seg_btn_warp", st);
    k0<<<a.num_sms * 4, 256, B0::SMEM, st>>>(keys, vals, a.offsets, a.nseg, a.total,
                                             a.lists + (size_t)kSegWarp * a.nseg, a.cnt, kSegWarp);
    timer_end(a.timer, st);
    timer_begin(a.timer, "k_seg_btn_mid", st);
    k1<<<a.num_sms * 8, 64, B1::SMEM, st>>>(keys, vals, a.offsets, a.nseg, a.total,
                                            a.lists + (size_t)kSegMid * a.nseg, a.cnt, kSegMid);
    timer_end(a.timer, st);
    timer_begin(a.timer, "k_seg_btn_cta", st);
    k2<<<a.num_sms * 2, 256, B2::SMEM, st>>>(keys, vals, a.offsets, a.nseg, a.total,
                                             a.lists + (size_t)kSegCta * a.nseg, a.cnt, kSegCta);
    timer_end(a.timer, st);
  }

  // long ranges: histograms, bases, then the rounds over all their tiles
  timer_begin(a.timer, "k_seg_hist", st);
  {
    constexpr int LANES = sizeof(K) == 4 ? 32 : 16;  // 128 KiB of counters either way
    constexpr size_t HSMEM = sizeof(uint32_t) * (size_t)P * R * (LANES + 1);
    auto hk = k_seg_hist<K, 8, TILE, LANES>;
    if ((e = cudaFuncSetAttribute(hk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HSMEM)))
      return e;
    hk<<<a.num_sms, 1024, HSMEM, st>>>(keys, a.offsets, a.nseg, a.total, a.lists, a.cnt,
                                       a.slot_first, a.tile_slot, a.seg_hist);
  }
  timer_end(a.timer, st);
  timer_begin(a.timer, "k_seg_scan", st);
  k_seg_scan<8, P, TILE><<<(unsigned)nslots, R, 0, st>>>(
      a.cnt, a.seg_hist, a.seg_base, a.seg_skip, HasVal<V>::value ? nullptr : a.seg_claim,
      a.offsets, a.nseg, a.total, a.lists, a.slot_first, a.tile_info);
  timer_end(a.timer, st);

  auto kern = k_seg_onesweep<K, V, 8, THREADS, KPT, MINB>;
  auto kern_agg = k_seg_onesweep<K, V, 8, THREADS, KPT, MINB, false, true>;
  constexpr size_t SEG_SMEM = OrderedShape<K, V, 8, THREADS, KPT>::SMEM;
  if (SEG_SMEM > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)SEG_SMEM)))
      return e;
    if (a.agg_top && (e = cudaFuncSetAttribute(kern_agg,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)SEG_SMEM)))
      return e;
  }
  using FC = FirstCfg<K, THREADS, KPT, MINB>;  // the order-free first round's CTA shape
  constexpr size_t FIRST_SMEM = FirstShape<K, 8, FC::T, FC::KP>::SMEM;
  if constexpr (!HasVal<V>::value && FIRST_SMEM > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(k_seg_onesweep<K, V, 8, FC::T, FC::KP, MINB, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FIRST_SMEM)))
      return e;
  }
  SegPassParams sp;
  sp.off = a.offsets;
  sp.nseg = a.nseg;
  sp.total = a.total;
  sp.list = a.lists;
  sp.cnt = a.cnt;
  sp.slot_first = a.slot_first;
  sp.tile_slot = a.tile_slot;
  sp.seg_base = a.seg_base;
  sp.seg_skip = a.seg_skip;
  sp.seg_claim = a.seg_claim;
  sp.tile_info = a.tile_info;
  sp.passes = P;
  PassParams& pp = sp.p;
  pp.keys[0] = a.keys;
  pp.keys[1] = a.alt_keys;
  pp.vals[0] = a.vals;
  pp.vals[1] = a.alt_vals;
  pp.n = a.total;
  pp.base = nullptr;
  pp.skip = nullptr;
  pp.err = a.err;
  pp.spin_limit = a.spin_limit;
  pp.stall_tile = -1;
  pp.claim = nullptr;
  pp.prefetch_tiles = (int64_t)a.num_sms * 4;  // one wave of tiles ahead
  pp.check_mode = a.check_mode;
  for (int q = 0; q < P; ++q) {
    pp.pass = q;
    pp.shift = q * 8;
    pp.mask = (1u << L::width(q)) - 1;
    pp.byte_sel = radix8_byte_sel(pp.shift);
    pp.low_shift = pp.shift;
    pp.status = a.status[q & 1];
    pp.status_next = (q + 1 < P) ? a.status[(q + 1) & 1] : nullptr;
    pp.counter = a.cnt + kCntPassTiles + q;
    if constexpr (!HasVal<V>::value) {
      if (q == 0) {  // keys only: the order-free first round
        timer_begin(a.timer, "k_seg_onesweep_first", st);
        k_seg_onesweep<K, V, 8, FC::T, FC::KP, MINB, true>
            <<<(unsigned)a.max_tiles, FC::T, FIRST_SMEM, st>>>(sp);
        timer_end(a.timer, st);
        continue;
      }
    }
    timer_begin(a.timer, "k_seg_onesweep", st);
    if (a.agg_top && q == P - 1)  // the top digit, nearly constant inside each range
      kern_agg<<<(unsigned)a.max_tiles, THREADS, SEG_SMEM, st>>>(sp);
    else
      kern<<<(unsigned)a.max_tiles, THREADS, SEG_SMEM, st>>>(sp);
    timer_end(a.timer, st);
  }
  timer_begin(a.timer, "k_seg_copy_back", st);
  k_seg_copy_back<K, V, TILE><<<a.num_sms * 8, 256, 0, st>>>(
      keys, static_cast<const K*>(a.alt_keys), vals, static_cast<const V*>(a.alt_vals),
      a.offsets, a.nseg, a.total, a.lists, a.cnt, a.slot_first, a.tile_slot, a.seg_skip, P);
  timer_end(a.timer, st);
  return cudaGetLastError();
}

template <typename K, typename V, int WM, int MM, int CM, int THREADS, int KPT, int MINB>
constexpr SegConfig seg_config() {
  return SegConfig{(int)(8 * sizeof(K)),
                   HasVal<V>::value ? (int)(8 * sizeof(V)) : 0,
                   WM,
                   MM,
                   CM,
                   (int64_t)THREADS * KPT,
                   DigitLayout<K, 8>::PASSES,
                   256,
                   &seg_launch<K, V, WM, MM, CM, THREADS, KPT, MINB>};
}

}  // namespace isort
