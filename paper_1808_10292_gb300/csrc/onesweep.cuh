// LSD radix sort passes with a single-pass decoupled look-back (radix 2^BITS).
//
// Paper mapping (Gerbessiotis, arXiv 1808.10292, Section "SR4, PR2, PR4, BTN
// and OET under MBSP"): one count-sort round counts the digits of its input,
// turns the counts into prefix sums and writes every key, in input order, to
// the next free slot of its digit. PR4 splits the keys over p workers, each
// counts its own share, the p x r count matrix is exchanged ("scatter and
// gather", the 2prg term of Eq. Tp) and each worker routes its keys to global
// positions (4Ng). Here a worker is a CTA-sized tile of keys, and the count
// exchange is a decoupled look-back: tile t publishes its digit counts, then
// adds up its predecessors' published counts, so that every pass reads its
// keys once and writes them once.
//
//   k_hist      counts the digits of ALL passes in one read of the keys (the
//               per-round "counting process" hoisted out of the rounds; the
//               counts are the same).
//   k_scan      exclusive prefix of each pass's digit counts -> global digit
//               bases; flags passes whose digit is constant (identity).
//   k_onesweep  one round ("ordered" form): load a tile, count and publish
//               the tile's digit counts, give each key its slot with one shared
//               atomic on its warp's counter of its digit (stable when the
//               hardware serves same-address lanes in lane order), look back
//               over earlier tiles, write the tile out in runs while checking
//               that every digit run is in order, and re-rank a tile that is
//               not (onesweep_tile_ordered).
//   k_onesweep_first  pass 0 of a keys-only sort: the same round without the
//               check (one CTA-wide counter per digit), since the first round's
//               input order carries no information.
//   k_copy_back copies the result home when an odd number of rounds ran.
#pragma once
#include <algorithm>

#include "common.cuh"
#include "isort_internal.h"

namespace isort {

template <typename K, int BITS>
struct DigitLayout {
  static constexpr int KB = 8 * sizeof(K);
  static constexpr int R = 1 << BITS;
  static constexpr int PASSES = (KB + BITS - 1) / BITS;
  __host__ __device__ static constexpr int width(int p) {
    return (KB - p * BITS) < BITS ? (KB - p * BITS) : BITS;
  }
};

template <typename K>
struct Vec16 {};
template <>
struct Vec16<uint32_t> {
  using T = uint4;
  static constexpr int N = 4;
  __device__ static uint32_t get(const uint4& v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
  }
};
template <>
struct Vec16<uint64_t> {
  using T = ulonglong2;
  static constexpr int N = 2;
  __device__ static uint64_t get(const ulonglong2& v, int i) { return i == 0 ? v.x : v.y; }
};

// ---------------------------------------------------------------------------
// k_hist: hist[p][d] += #{keys with digit p == d} for every pass p, one read.
// The CTA's shared counters are laid out [p][d][lane % LANES]: lane l of every
// warp counts into its own column, so the 32 atomics of one warp instruction
// fall in different banks (no bank conflicts); warps of the CTA share columns
// through the atomics.
template <typename K, int BITS, int THREADS, int LANES>
struct HistShape {
  using L = DigitLayout<K, BITS>;
  static constexpr size_t SMEM = sizeof(uint32_t) * (size_t)L::PASSES * L::R * LANES;
};

// Calls count(k) for every key of keys[0..n): thread `me` of `nth` takes the
// unaligned head and tail one key at a time and the 16-byte-aligned middle as
// 16-byte loads, U of them in flight.
template <typename K, typename F>
__device__ __forceinline__ void count_keys(const K* __restrict__ keys, int64_t n, int64_t me,
                                           int64_t nth, F&& count) {
  using V16 = Vec16<K>;
  const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
  int64_t head = (int64_t)(((16 - (addr & 15)) & 15) / sizeof(K));
  if (head > n) head = n;
  const int64_t nvec = (n - head) / V16::N;
  const typename V16::T* vec = reinterpret_cast<const typename V16::T*>(keys + head);
  if (me < head) count(keys[me]);
  constexpr int U = 4;
  int64_t i = me;
  for (; i + (U - 1) * nth < nvec; i += U * nth) {
    typename V16::T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = vec[i + u * nth];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int c = 0; c < V16::N; ++c) count(V16::get(v[u], c));
  }
  for (; i < nvec; i += nth) {
    typename V16::T v = vec[i];
#pragma unroll
    for (int c = 0; c < V16::N; ++c) count(V16::get(v, c));
  }
  const int64_t tail0 = head + nvec * V16::N;
  if (tail0 + me < n) count(keys[tail0 + me]);
}

template <typename K, int BITS, int THREADS, int LANES>
__global__ void __launch_bounds__(THREADS) k_hist(const K* __restrict__ keys, int64_t n,
                                                  uint32_t* __restrict__ hist) {
  using L = DigitLayout<K, BITS>;
  constexpr int R = L::R, P = L::PASSES;
  extern __shared__ __align__(16) uint32_t s_cnt[];  // [P][R][LANES]
  for (int i = threadIdx.x; i < P * R * LANES; i += THREADS) s_cnt[i] = 0;
  __syncthreads();
  uint32_t* my = s_cnt + (threadIdx.x & (LANES - 1));

  auto count = [&](K k) {
#pragma unroll
    for (int p = 0; p < P; ++p)
      atomicAdd(&my[(p * R + digit_of(k, p * BITS, (1u << L::width(p)) - 1)) * LANES], 1u);
  };

  count_keys(keys, n, blockIdx.x * (int64_t)THREADS + threadIdx.x, (int64_t)gridDim.x * THREADS,
             count);
  __syncthreads();
  for (int j = threadIdx.x; j < P * R; j += THREADS) {
    uint32_t s = 0;
#pragma unroll 8
    for (int b = 0; b < LANES; ++b) s += s_cnt[j * LANES + ((b + j) & (LANES - 1))];
    if (s) atomicAdd(&hist[j], s);
  }
}

// ---------------------------------------------------------------------------
// k_scan: block p turns hist[p][0..R) into exclusive prefix sums base[p][..]
// and sets skip[p] when one digit holds all n keys.
// Also zeroes `claim` (R words, or null): the output cursors of the order-free
// first round (onesweep_tile_first), which start from the bases.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_scan(const uint32_t* __restrict__ hist,
                                                  uint32_t* __restrict__ base,
                                                  uint32_t* __restrict__ skip, int R, int64_t n,
                                                  uint32_t* __restrict__ claim) {
  __shared__ uint32_t s_warp[THREADS / 32];
  __shared__ uint32_t s_trivial;
  const int p = blockIdx.x;
  const uint32_t* h = hist + (size_t)p * R;
  uint32_t* b = base + (size_t)p * R;
  const int per = (R + THREADS - 1) / THREADS;  // consecutive digits per thread
  const int d0 = threadIdx.x * per;
  if (threadIdx.x == 0) s_trivial = 0;
  uint32_t local = 0;
  bool trivial = false;
  for (int j = 0; j < per; ++j) {
    int d = d0 + j;
    if (d < R) {
      uint32_t c = h[d];
      local += c;
      trivial |= (int64_t)c == n;
    }
  }
  __syncthreads();
  if (trivial) s_trivial = 1;
  uint32_t total;
  uint32_t run = block_exclusive_scan<THREADS>(local, s_warp, total);
  for (int j = 0; j < per; ++j) {
    int d = d0 + j;
    if (d < R) {
      b[d] = run;
      run += h[d];
    }
  }
  if (threadIdx.x == 0) skip[p] = s_trivial;
  if (claim && p == 0)
    for (int d = threadIdx.x; d < R; d += THREADS) claim[d] = 0;
}

// ---------------------------------------------------------------------------
struct PassParams {
  void* keys[2];  // [0] caller's array, [1] alternate buffer
  void* vals[2];
  int64_t n;
  int pass;
  int shift;
  uint32_t mask;
  const uint32_t* base;   // [R] exclusive global base per digit (this pass)
  const uint32_t* skip;   // [passes]
  uint32_t* status;       // [tiles][R] this pass's look-back words, zeroed
  uint32_t* status_next;  // [tiles][R] zeroed here for the next pass, or null
  uint32_t* counter;      // this pass's tile-id counter, zeroed
  uint32_t* claim;        // [R] order-free first round: per-digit output cursors, zeroed
                          // (null: that round uses the look-back too)
  uint32_t* err;
  uint32_t spin_limit;
  int64_t stall_tile;
  int64_t prefetch_tiles;     // L2-prefetch the input of the tile this many ids ahead (0: off)
  uint32_t check_mode;        // test hook of the ordered rounds (kCheck*; 0 in normal use)
  uint32_t byte_sel;          // radix-256 rounds: radix8_byte_sel(shift)
  int low_shift;              // keys only: the input is sorted by bits [0, low_shift)
};

// Test hooks of the ordered keys-only rounds (onesweep_tile_ordered).
constexpr uint32_t kCheckNormal = 0;
constexpr uint32_t kCheckForceFallback = 1;  // every tile takes the stable re-rank
constexpr uint32_t kCheckPerturb = 2;        // odd lanes take their slots first (unstable)

// The digit of a key in one round: bits [shift, shift + width) of the key. The
// early-counts tile functions take the digit as a function object, so a round
// can also distribute keys by another rule (a splitter bucket, for instance).
// The tile code asks for digits through four calls, so a rule whose digits are
// costly can compute each once (prepare) and hand back the stored value:
//   prepare(key)  after the tile's keys are loaded into registers;
//   of(k, i)      the digit of this thread's key i (k = key[i]);
//   keep(pos, d)  the key with digit d was placed at tile slot pos;
//   staged(k, j)  the digit of the key at tile slot j (k = that key).
// RadixDigit refers to the round's parameters (shift and mask stay where the
// kernel received them instead of being copied into registers).
// Radix-256 rounds only (8-bit digits on byte boundaries): the digit is byte
// shift / 8 of the key, taken with one byte permute (selector p.byte_sel).
struct RadixDigit {
  const PassParams& p;
  template <typename K>
  __device__ __forceinline__ uint32_t operator()(K k) const {
    if constexpr (sizeof(K) == 4) {
      return __byte_perm((uint32_t)k, 0u, p.byte_sel);
    } else {
      const uint32_t w = p.shift >= 32 ? (uint32_t)(k >> 32) : (uint32_t)k;
      return __byte_perm(w, 0u, p.byte_sel);
    }
  }
  template <typename K, int KPT>
  __device__ __forceinline__ void prepare(const K (&)[KPT]) {}
  template <typename K>
  __device__ __forceinline__ uint32_t of(K k, int) const {
    return (*this)(k);
  }
  __device__ __forceinline__ void keep(uint32_t, uint32_t) const {}
  template <typename K>
  __device__ __forceinline__ uint32_t staged(K k, int) const {
    return (*this)(k);
  }
};

// Any digit of at most 8 bits: bits [p.shift, p.shift + width) of the key, with
// p.mask = 2^width - 1 (the steps of the wide-radix rounds, whose digit parts
// need not sit on byte boundaries).
struct ShiftMaskDigit {
  const PassParams& p;
  template <typename K>
  __device__ __forceinline__ uint32_t operator()(K k) const {
    return digit_of(k, p.shift, p.mask);
  }
  template <typename K, int KPT>
  __device__ __forceinline__ void prepare(const K (&)[KPT]) {}
  template <typename K>
  __device__ __forceinline__ uint32_t of(K k, int) const {
    return (*this)(k);
  }
  __device__ __forceinline__ void keep(uint32_t, uint32_t) const {}
  template <typename K>
  __device__ __forceinline__ uint32_t staged(K k, int) const {
    return (*this)(k);
  }
};

// Byte-permute selector that moves byte (shift / 8) % 4 of a word to byte 0
// and zeroes the others (bytes 4..7 of the permute's input are the zero word).
__host__ __device__ constexpr uint32_t radix8_byte_sel(int shift) {
  return 0x4440u | (uint32_t)((shift >> 3) & 3);
}

// Keep DRAM busy while tiles are ranking: one thread of the CTA asks the copy
// engine to bring the input of a tile about one wave ahead into L2, so that
// tile's loads hit L2. The bulk prefetch takes 16-byte aligned addresses and
// sizes, so a range that does not start or end on 16 bytes (a segment or a
// bucket inside the keys) is prefetched without its partial 16-byte ends,
// which stay inside the range.
template <typename T>
__device__ __forceinline__ void prefetch_tile(const T* base, int64_t first, int64_t count) {
  if (count <= 0) return;
  const uintptr_t a = reinterpret_cast<uintptr_t>(base + first);
  const uintptr_t lo = (a + 15) & ~uintptr_t(15);
  const uintptr_t hi = (a + (uintptr_t)count * sizeof(T)) & ~uintptr_t(15);
  if (hi > lo) prefetch_l2(reinterpret_cast<const void*>(lo), (uint32_t)(hi - lo));
}

template <typename K, typename V, int BITS, int THREADS, int KPT>
struct OnesweepShape {
  static constexpr int R = 1 << BITS;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int TILE = THREADS * KPT;
  static constexpr bool HV = HasVal<V>::value;
  // shared words before the staged tile: per-warp counters, output offsets, misc
  static constexpr int HEADER_WORDS = WARPS * R + R + 64;
  static constexpr int DPT = R >= THREADS ? R / THREADS : 1;  // digits per owning thread
  static constexpr int DTHREADS = R >= THREADS ? THREADS : R;  // threads that own digits
  static_assert(THREADS >= R || R % THREADS == 0,
                "every digit needs exactly one owner thread: THREADS >= R or THREADS divides R");
};

// Decoupled look-back for digit d of tile `tile` (> 0): the sum of the counts of
// digit d in all earlier tiles. Walks back from tile-1, adding AGG counts until
// it reaches an INC word (which already holds the sum of everything before it).
// LB predecessor words are read at once, so one L2 round trip covers LB tiles
// of the walk. A word that is not published yet is polled again after a short
// sleep; polls are bounded by spin_limit, after which the error word gets
// kErrTimeout and the partial sum is returned (the output is then garbage, but
// every write stays bounds-checked).
constexpr int kLookbackWindow = 8;

template <int R, int LB>
__device__ __forceinline__ uint32_t lookback_exclusive(const uint32_t* status, uint32_t tile,
                                                       int d, uint32_t spin_limit, uint32_t* err,
                                                       uint32_t& windows) {
  static_assert(LB <= 32, "window flags are kept in one word");
  uint32_t excl = 0, polls = 0;
  int64_t t = (int64_t)tile - 1;
  while (true) {
    ++windows;
    uint32_t s[LB];
#pragma unroll
    for (int k = 0; k < LB; ++k)  // below tile 0 reads as "inclusive, count 0"
      s[k] = (t - k >= 0) ? ld_relaxed(&status[(size_t)(t - k) * R + d]) : kFlagInc;
    // Branch-free scan of the window: stop at the first word that is not
    // published yet (poll it again) or that is inclusive (done after it).
    uint32_t unpublished = 0, inclusive = 0;
#pragma unroll
    for (int k = 0; k < LB; ++k) {
      unpublished |= (uint32_t)(s[k] < kFlagAgg) << k;
      inclusive |= (s[k] >> 31) << k;
    }
    const uint32_t stop = unpublished | inclusive;
    const int first = stop ? __ffs(stop) - 1 : LB;
    const bool done = (inclusive >> first) & 1u;  // LB <= 31: bit LB is 0 when no stop
    const int take = first + (done ? 1 : 0);
#pragma unroll
    for (int k = 0; k < LB; ++k) excl += (k < take) ? (s[k] & kCountMask) : 0u;
    if (done) break;
    t -= take;
    if (take < LB) {  // blocked on tile t: it has published nothing yet
      if (++polls >= spin_limit) {
        atomicOr(err, kErrTimeout);
        break;
      }
      __nanosleep(64);
    }
  }
  return excl;
}

// Zero `words` 32-bit words of shared memory (16-byte aligned, words % 4 == 0)
// with 16-byte stores.
template <int THREADS>
__device__ __forceinline__ void zero_words(uint32_t* p, int words) {
  uint4* q = reinterpret_cast<uint4*>(p);
  for (int i = threadIdx.x; i < words / 4; i += THREADS) q[i] = make_uint4(0, 0, 0, 0);
}

// ---- the phases of one tile (shared by the plain and segmented rounds and
// the sample sort's split round). FULL: the tile holds TILE keys, so no
// per-key bounds predicate.

// Load: warp w owns keys [w*32*KPT, (w+1)*32*KPT) of the tile, lane-striped,
// so each warp instruction reads 32 consecutive keys.
template <typename K, typename V, int KPT, bool FULL>
__device__ __forceinline__ void tile_load(const K* __restrict__ kin, const V* vin,
                                          int64_t tile_base, int tile_n, int wofs, K (&key)[KPT],
                                          V (&val)[HasVal<V>::value ? KPT : 1]) {
  const int64_t g0 = tile_base + wofs;
#pragma unroll
  for (int i = 0; i < KPT; ++i)
    key[i] = (FULL || wofs + i * 32 < tile_n) ? kin[g0 + i * 32] : K(0);
  if constexpr (HasVal<V>::value) {
#pragma unroll
    for (int i = 0; i < KPT; ++i)
      val[i] = (FULL || wofs + i * 32 < tile_n) ? vin[g0 + i * 32] : V(0);
  }
}

// Write out (keys only): consecutive threads take consecutive tile slots, so
// each digit's run lands on consecutive global addresses; every index is
// bounds-checked.
template <typename K, int THREADS, int KPT, bool FULL, typename DS>
__device__ __forceinline__ void tile_scatter(const K* s_keys, const uint32_t* s_adj,
                                             const DS& dig, int tile_n, K* kout, uint32_t bound,
                                             uint32_t* err) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int j = k * THREADS + tid;
    if (FULL || j < tile_n) {
      const K kk = s_keys[j];
      const uint32_t g = s_adj[dig.staged(kk, j)] + (uint32_t)j;
      if (g < bound)
        kout[g] = kk;
      else
        atomicOr(err, kErrBounds);
    }
  }
}

// Early counts: each warp counts the digits of its keys into its private row of
// s_wcnt (one shared atomic add per key, order irrelevant).
template <typename K, int R, int KPT, bool FULL, typename DS>
__device__ __forceinline__ void tile_count(const K (&key)[KPT], const DS& dig, int tile_n,
                                           int wofs, uint32_t* my) {
#pragma unroll
  for (int i = 0; i < KPT; ++i)
    if (FULL || wofs + i * 32 < tile_n) atomicAdd(&my[dig.of(key[i], i)], 1u);
}

// Shared memory of the ordered round: the per-warp counters, digit offsets and
// misc words, the staged keys (in tile order), and with payloads the staged
// payloads (in input order) and each staged key's input index (16 bits).
template <typename K, typename V, int BITS, int THREADS, int KPT>
struct OrderedShape {
  using S = OnesweepShape<K, V, BITS, THREADS, KPT>;
  static constexpr bool HV = HasVal<V>::value;
  static constexpr size_t KEYS = (size_t)S::HEADER_WORDS * 4;
  static constexpr size_t VALS = KEYS + (size_t)S::TILE * sizeof(K);
  static constexpr size_t SRC = VALS + (HV ? (size_t)S::TILE * sizeof(V) : 0);
  static constexpr size_t SMEM = SRC + (HV ? (size_t)S::TILE * 2 : 0);
  static_assert(S::TILE <= 65536, "input indices are kept in 16 bits");
};

// One tile of a count-sort round, "ordered" form (every round of k_onesweep;
// the rounds after the first of a keys-only segmented sort and all rounds of a
// segmented pair sort). A key's stable rank among the warp's keys of its digit
// is the value one shared-memory atomicAdd on the warp's counter of the digit
// returns, provided the lanes of one warp instruction that hit the same
// counter are served in lane order and successive instructions in program
// order -- which is what GB300 does (a probe of a million 32-lane rows found
// no exception), but nothing in CUDA promises it. So the tile checks its
// result instead of trusting the order, in the write-out, key by key against
// the next staged key of the same digit:
//  - keys only: the round's input is sorted by the key bits below its digit
//    (`low` = bits [0, p.low_shift); the invariant of LSD rounds on keys; a
//    round that sorts by part of a wider digit names the bits sorted so far),
//    so the tile is placed
//    acceptably iff every digit run is non-decreasing in those bits (keys that
//    agree on the digit and the low bits may take either order: later rounds
//    order them by their higher bits, or they are equal);
//  - with payloads: every digit run must hold its keys in input order (the
//    staged input indices increase), which is exact stability.
// A tile that fails is ranked again stably (peers found with __match_any_sync)
// and written out again to the same positions. Payloads are copied into shared
// memory in input order (one bulk copy per tile, or cp.async; no registers)
// and gathered by the staged input indices at the write-out. Per key the fast
// path makes three digit-indexed shared accesses (count add, slot add, key
// store; with payloads also the index store and the payload gather).
//
// A slot add that returns the old value is served one lane at a time for the
// lanes of a warp instruction that hit the same counter, so a row whose keys
// share one or two digits takes up to ~30 times longer than a row of random
// digits. With AGG, a tile with at most kAggDigits distinct digits (the top
// digit inside the buckets of a sample sort, for instance) ranks without slot
// adds: the owners list the tile's digit values, and each warp keeps one
// running count per value in registers, taking a row's ranks from a ballot per
// value (lane order within the row, rows in order: the same ranks the slot
// adds give, so the check is unchanged). The warp's counters are then set as
// the slot adds would have left them, for the fallback.
constexpr int kAggDigits = 3;

template <typename K, typename V, int BITS, int THREADS, int KPT, bool FULL,
          typename DS = RadixDigit, bool AGG = false>
__device__ __forceinline__ void onesweep_tile_ordered(const PassParams& p, uint32_t tile,
                                                      bool first, int64_t tile_base, int tile_n,
                                                      const K* __restrict__ kin,
                                                      K* __restrict__ kout, const V* vin, V* vout,
                                                      const uint32_t* base, uint32_t bound,
                                                      unsigned char* smem, DS& dig,
                                                      bool bulk = false) {
  // bulk: the kernel started one bulk copy of this (whole) tile into the
  // staging area, and of its payloads into the staged-payload area, completing
  // on the mbarrier at s_misc[56..57]; otherwise keys are loaded lane-striped
  // from global memory and payloads copied by cp.async.
  using S = OnesweepShape<K, V, BITS, THREADS, KPT>;
  using O = OrderedShape<K, V, BITS, THREADS, KPT>;
  constexpr int R = S::R, WARPS = S::WARPS, DPT = S::DPT;
  constexpr bool HV = O::HV;
  uint32_t* s_wcnt = reinterpret_cast<uint32_t*>(smem);  // [WARPS][R]
  uint32_t* s_adj = s_wcnt + WARPS * R;                   // [R]
  uint32_t* s_misc = s_adj + R;                           // [64]
  K* s_keys = reinterpret_cast<K*>(smem + O::KEYS);
  V* s_vals = reinterpret_cast<V*>(smem + O::VALS);          // payloads only
  uint16_t* s_src = reinterpret_cast<uint16_t*>(smem + O::SRC);  // payloads only
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wofs = warp * 32 * KPT + lane;
  const bool publish = (int64_t)tile != p.stall_tile;
  uint32_t* my = s_wcnt + warp * R;
  // the fallback re-reads the tile's input address from here (fewer live registers)
  if (tid == 0) *reinterpret_cast<const K**>(s_misc + 48) = kin + tile_base;
  if constexpr (AGG)
    if (tid == 0) s_misc[40] = 0;  // AGG: the number of listed digit values

  K key[KPT];
  NoVal nv[1];
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_misc + 56);
  if (FULL && bulk) {
    if (!mbar_wait_bounded(bar, 0, p.spin_limit)) {
      // the copy did not complete in time: flag it, and still wait (bounded)
      // for it to land before the staging area is read or reused
      atomicOr(p.err, kErrTimeout);
      mbar_wait_bounded(bar, 0, p.spin_limit);
    }
#pragma unroll
    for (int i = 0; i < KPT; ++i) key[i] = s_keys[wofs + i * 32];
  } else {
    tile_load<K, NoVal, KPT, FULL>(kin, nullptr, tile_base, tile_n, wofs, key, nv);
    if constexpr (HV) {
#pragma unroll
      for (int i = 0; i < KPT; ++i)
        if (FULL || wofs + i * 32 < tile_n)
          cp_async<sizeof(V)>(&s_vals[wofs + i * 32], vin + tile_base + wofs + i * 32);
    }
  }
  dig.prepare(key);
  tile_count<K, R, KPT, FULL>(key, dig, tile_n, wofs, my);
  __syncthreads();  // every thread holds its keys: the staging area is free
  if (FULL && bulk && tid == 0) mbar_inval(bar);  // used once; every thread has passed it

  // per digit: the tile's count (published now), warp starts, tile starts;
  // with up to 8 warps the warp-exclusive prefixes stay in registers across
  // the block scan (more would spill), else they go back to shared memory
  constexpr bool WREG = WARPS <= 8;
  uint32_t dcnt[DPT], wpre[DPT][WREG ? WARPS : 1];
  uint32_t tsum = 0;
  const bool owner = tid < S::DTHREADS;
  if (owner) {
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int d = tid * DPT + j;
      uint32_t sum = 0;
#pragma unroll
      for (int w = 0; w < WARPS; ++w) {
        const uint32_t c = s_wcnt[w * R + d];
        if constexpr (WREG)
          wpre[j][w] = sum;
        else
          s_wcnt[w * R + d] = sum;
        sum += c;
      }
      dcnt[j] = sum;
      tsum += sum;
      if (publish)
        st_relaxed(&p.status[(size_t)tile * R + d], (first ? kFlagInc : kFlagAgg) | sum);
    }
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan<THREADS>(tsum, s_misc + 1, total);
  uint32_t tstart[DPT];
  if (owner) {
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int d = tid * DPT + j;
      tstart[j] = run;
#pragma unroll
      for (int w = 0; w < WARPS; ++w) {
        if constexpr (WREG)
          s_wcnt[w * R + d] = run + wpre[j][w];
        else
          s_wcnt[w * R + d] += run;
      }
      run += dcnt[j];
    }
  }
  __syncthreads();

  // place: one slot add per key
  auto place = [&](int i, uint32_t pos, uint32_t d) {
    s_keys[pos] = key[i];
    dig.keep(pos, d);
    if constexpr (HV) s_src[pos] = (uint16_t)(wofs + i * 32);
  };
  bool few = false;  // AGG: at most kAggDigits distinct digits in the tile
  if constexpr (AGG && DPT == 1) {
    const bool used = owner && dcnt[0] > 0;
    if (used) {
      const uint32_t k = atomicAdd(&s_misc[40], 1u);
      if (k < (uint32_t)kAggDigits) s_misc[41 + k] = (uint32_t)tid;
    }
    few = __syncthreads_count(used) <= kAggDigits;
  }
  if (p.check_mode != kCheckPerturb && few) {
    const uint32_t lt = lanemask_lt();
    const uint32_t nv = s_misc[40];
    uint32_t v[kAggDigits], c[kAggDigits];
#pragma unroll
    for (int j = 0; j < kAggDigits; ++j) {
      v[j] = (uint32_t)j < nv ? s_misc[41 + j] : 0xffffffffu;  // no digit equals ~0
      c[j] = (uint32_t)j < nv ? my[v[j]] : 0u;  // this warp's first slot of the value
    }
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      const bool valid = FULL || wofs + i * 32 < tile_n;
      const uint32_t d = valid ? dig.of(key[i], i) : 0xffffffffu;
      uint32_t pos = 0;
#pragma unroll
      for (int j = 0; j < kAggDigits; ++j) {
        const uint32_t m = __ballot_sync(kFullMask, d == v[j]);
        if (d == v[j]) pos = c[j] + __popc(m & lt);
        c[j] += __popc(m);
      }
      if (valid) place(i, pos, d);
    }
    if (lane == 0)
#pragma unroll
      for (int j = 0; j < kAggDigits; ++j)
        if ((uint32_t)j < nv) my[v[j]] = c[j];
  } else if (p.check_mode != kCheckPerturb) {
#pragma unroll
    for (int i = 0; i < KPT; ++i)
      if (FULL || wofs + i * 32 < tile_n) {
        const uint32_t d = dig.of(key[i], i);
        place(i, atomicAdd(&my[d], 1u), d);
      }
  } else {  // test hook: odd lanes of each row first, an order the check must reject
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      const bool valid = FULL || wofs + i * 32 < tile_n;
      uint32_t pos = 0;
      if (valid && (lane & 1)) pos = atomicAdd(&my[dig.of(key[i], i)], 1u);
      __syncwarp();
      if (valid && !(lane & 1)) pos = atomicAdd(&my[dig.of(key[i], i)], 1u);
      __syncwarp();
      if (valid) place(i, pos, dig.of(key[i], i));
    }
  }

  // look back over earlier tiles, publish the inclusive counts, output offsets
  uint32_t windows = 0;
  if (owner) {
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int d = tid * DPT + j;
      uint32_t excl = 0;
      if (!first) {
        excl = lookback_exclusive<R, kLookbackWindow>(p.status, tile, d, p.spin_limit, p.err,
                                                      windows);
        if (publish) st_relaxed(&p.status[(size_t)tile * R + d], kFlagInc | (excl + dcnt[j]));
      }
      s_adj[d] = base[d] + excl - tstart[j];
    }
  }
  if constexpr (HV) cp_async_wait_all();  // this thread's payload copies have landed
  __syncthreads();

  // write out (payloads gathered by input index), checking every staged key
  // against the next one of its run
  const K low = p.low_shift ? (K(1) << p.low_shift) - K(1) : K(0);
  bool bad = p.check_mode == kCheckForceFallback;
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int j = k * THREADS + tid;
    if (FULL || j < tile_n) {
      const K kk = s_keys[j];
      const uint32_t d = dig.staged(kk, j);
      const uint32_t g = s_adj[d] + (uint32_t)j;
      uint32_t src = 0;
      if constexpr (HV) src = s_src[j];
      if (g < bound) {
        kout[g] = kk;
        if constexpr (HV) vout[g] = s_vals[src];
      } else {
        atomicOr(p.err, kErrBounds);
      }
      if (j + 1 < (FULL ? S::TILE : tile_n)) {
        const K nx = s_keys[j + 1];
        if constexpr (HV)
          bad |= dig.staged(nx, j + 1) == d && s_src[j + 1] < src;
        else
          bad |= dig.staged(nx, j + 1) == d && (nx & low) < (kk & low);
      }
    }
  }
  if (!__syncthreads_or(bad)) return;

  // Fallback: rank the tile again, stably, and write it out again. After the
  // slot adds, warp w's counter of digit d holds warp w+1's start, and the
  // last warp's holds the end of the digit's run, i.e. the start of digit d+1:
  // shift the rows back to the warp starts.
  uint32_t prev_end[DPT];
  if (owner)
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int d = tid * DPT + j;
      prev_end[j] = d ? s_wcnt[(WARPS - 1) * R + d - 1] : 0u;
    }
  __syncthreads();
  if (owner)
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int d = tid * DPT + j;
#pragma unroll
      for (int w = WARPS - 1; w > 0; --w) s_wcnt[w * R + d] = s_wcnt[(w - 1) * R + d];
      s_wcnt[d] = prev_end[j];
    }
  __syncthreads();
  // Row by row, keys re-read from the input: peers by __match_any_sync, the
  // highest peer advances the counter, ranks in lane order (slow, but this path
  // is for tiles whose check failed). Payloads stay where they are (input order).
  const uint32_t lt = lanemask_lt();
  const K* tile_in = *reinterpret_cast<const K* const*>(s_misc + 48);
  uint32_t* my_row = s_wcnt + (threadIdx.x >> 5) * R;
  const int wofs2 = (threadIdx.x >> 5) * 32 * KPT + (threadIdx.x & 31);
#pragma unroll 1
  for (int i = 0; i < KPT; ++i) {
    const bool valid = FULL || wofs2 + i * 32 < tile_n;
    const K k = valid ? tile_in[wofs2 + i * 32] : K(0);
    const uint32_t d = dig(k);
    const uint32_t peers = __match_any_sync(kFullMask, valid ? d : (0x80000000u | lane));
    uint32_t old = 0;
    if (valid && (peers >> lane) == 1u) old = atomicAdd(&my_row[d], __popc(peers));
    old = __shfl_sync(kFullMask, old, 31 - __clz(peers));
    if (valid) {
      const uint32_t pos = old + __popc(peers & lt);
      s_keys[pos] = k;
      dig.keep(pos, d);
      if constexpr (HV) s_src[pos] = (uint16_t)(wofs2 + i * 32);
    }
    __syncwarp();  // this row's counter updates precede the next row's
  }
  __syncthreads();
#pragma unroll 1
  for (int j = tid; j < tile_n; j += THREADS) {
    const K kk = s_keys[j];
    const uint32_t g = s_adj[dig.staged(kk, j)] + (uint32_t)j;
    if (g < bound) {
      kout[g] = kk;
      if constexpr (HV) vout[g] = s_vals[s_src[j]];
    } else {
      atomicOr(p.err, kErrBounds);
    }
  }
}

// One count-sort round over all n keys, one tile per CTA (tile ids in launch
// order), in the ordered form. DS: the digit rule (bytes for radix 256).
template <typename K, typename V, int BITS, int THREADS, int KPT, int MINB,
          typename DS = RadixDigit>
__global__ void __launch_bounds__(THREADS, MINB) k_onesweep(PassParams p) {
  using S = OnesweepShape<K, V, BITS, THREADS, KPT>;
  constexpr int R = S::R, WARPS = S::WARPS, TILE = S::TILE;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_wcnt = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_misc = s_wcnt + WARPS * R + R;
  const int tid = threadIdx.x;

  // Rows of the next pass's look-back array are cleared here, so one memset
  // before the first pass is the only one a sort needs.
  if (p.status_next)
    for (int d = tid; d < R; d += THREADS) p.status_next[(size_t)blockIdx.x * R + d] = 0;
  if (p.skip[p.pass]) return;  // the digit is constant: this round is the identity

  int src = 0;  // input buffer = parity of the rounds executed before this one
  for (int q = 0; q < p.pass; ++q) src ^= (p.skip[q] == 0);

  if (tid == 0) {
    const uint32_t t = atomicAdd(p.counter, 1u);  // tiles in launch order
    s_misc[0] = t;
    // A whole tile at 16-byte aligned addresses comes by one bulk copy (keys
    // into the staging area, payloads in input order into the staged-payload
    // area): no per-key load instructions or cp.async, and with payloads one
    // copy instead of a cp.async per payload.
    const int64_t tb = (int64_t)t * TILE;
    const K* k0 = static_cast<const K*>(src ? p.keys[1] : p.keys[0]) + tb;
    const V* v0 = static_cast<const V*>(src ? p.vals[1] : p.vals[0]) + tb;
    bool bulk = tb + TILE <= p.n && (reinterpret_cast<uintptr_t>(k0) & 15) == 0;
    if constexpr (HasVal<V>::value) bulk = bulk && (reinterpret_cast<uintptr_t>(v0) & 15) == 0;
    if (bulk) {
      using O = OrderedShape<K, V, BITS, THREADS, KPT>;
      uint64_t* bar = reinterpret_cast<uint64_t*>(s_misc + 56);
      mbar_init(bar, 1);
      fence_mbar_init();
      constexpr uint32_t kb = TILE * sizeof(K);
      constexpr uint32_t vb = HasVal<V>::value ? TILE * sizeof(V) : 0;
      mbar_arrive_expect_tx(bar, kb + vb);
      bulk_copy_g2s(smem + O::KEYS, k0, kb, bar);
      if constexpr (HasVal<V>::value) bulk_copy_g2s(smem + O::VALS, v0, vb, bar);
    }
    s_misc[60] = bulk;
  }
  zero_words<THREADS>(s_wcnt, WARPS * R);
  __syncthreads();
  const uint32_t tile = s_misc[0];
  const bool bulk = s_misc[60] != 0;
  const int tile_n = (int)min((int64_t)TILE, p.n - (int64_t)tile * TILE);
  if (p.prefetch_tiles && tid == 0) {
    const int64_t pf = ((int64_t)tile + p.prefetch_tiles) * TILE;
    const int64_t cnt = min((int64_t)TILE, p.n - pf);
    prefetch_tile(static_cast<const K*>(src ? p.keys[1] : p.keys[0]), pf, cnt);
    if constexpr (HasVal<V>::value)
      prefetch_tile(static_cast<const V*>(src ? p.vals[1] : p.vals[0]), pf, cnt);
  }
  // select with branches, not a dynamic index, so the parameters stay out of local memory
  const K* kin = static_cast<const K*>(src ? p.keys[1] : p.keys[0]);
  K* kout = static_cast<K*>(src ? p.keys[0] : p.keys[1]);
  const V* vin = static_cast<const V*>(src ? p.vals[1] : p.vals[0]);
  V* vout = static_cast<V*>(src ? p.vals[0] : p.vals[1]);
  const int64_t tile_base = (int64_t)tile * TILE;
  DS dig{p};
  if (tile_n == TILE)
    onesweep_tile_ordered<K, V, BITS, THREADS, KPT, true, DS>(
        p, tile, tile == 0, tile_base, tile_n, kin, kout, vin, vout, p.base, (uint32_t)p.n, smem,
        dig, bulk);
  else
    onesweep_tile_ordered<K, V, BITS, THREADS, KPT, false, DS>(
        p, tile, tile == 0, tile_base, tile_n, kin, kout, vin, vout, p.base, (uint32_t)p.n, smem,
        dig);
}

// ---------------------------------------------------------------------------
// First round of a keys-only sort. Radix sort needs every round to be stable
// so that a round keeps the order the earlier rounds made; the first round has
// no earlier round, and keys with equal digits in it may land in any order
// without changing the final (unique) sorted result. So this round drops the
// stable rank: a key's tile slot is the return value of one shared atomic add
// on its digit's tile-wide counter (which holds the tile start of the digit
// after the scan), and the tile's output ranges come from per-digit cursors
// instead of a look-back. Per key that is a count add, a slot add and the
// store into the staging area, and no check. Later rounds rank stably.
// The first round's CTA shape for an ordered round of THREADS x KPT at MINB
// CTAs per SM: the same tile (so the tile counts match), with twice the
// threads holding half the keys each where their registers fit (the keys'
// words plus about 26 more per thread, against 65536 / (threads x MINB)).
// The round keeps no per-warp counters or warp prefixes, so it needs fewer
// registers than the ordered round; more warps per SM hide more latency.
template <typename K, int THREADS, int KPT, int MINB>
struct FirstCfg {
  static constexpr bool WIDE = KPT % 2 == 0 && THREADS * 2 <= 1024 &&
                               (KPT / 2) * (int)(sizeof(K) / 4) + 26 <= 65536 / (2 * THREADS * MINB);
  static constexpr int T = WIDE ? THREADS * 2 : THREADS;
  static constexpr int KP = WIDE ? KPT / 2 : KPT;
  static_assert(T * KP == THREADS * KPT, "same tile as the stable round");
};

template <typename K, int BITS, int THREADS, int KPT>
struct FirstShape {
  using S = OnesweepShape<K, NoVal, BITS, THREADS, KPT>;
  static constexpr int HEADER_WORDS = 2 * S::R + 64;  // s_slot, s_adj, s_misc
  static constexpr size_t SMEM = (size_t)HEADER_WORDS * 4 + (size_t)S::TILE * sizeof(K);
};

// Arguments as for onesweep_tile_ordered (keys only). With `claim` (R words
// starting at zero before the round) a tile takes each digit's output range
// with one global atomic add of its count on the digit's cursor, instead of a
// look-back over earlier tiles: the round is order-free, so the tiles' runs of
// a digit may lie in any order, and no tile waits on another. Without it the
// tile publishes its counts and looks back like the ordered round.
template <typename K, int BITS, int THREADS, int KPT, bool FULL, typename DS = RadixDigit>
__device__ __forceinline__ void onesweep_tile_first(const PassParams& p, uint32_t tile, bool first,
                                                    int64_t tile_base, int tile_n,
                                                    const K* __restrict__ kin,
                                                    K* __restrict__ kout, const uint32_t* base,
                                                    uint32_t bound, unsigned char* smem,
                                                    DS& dig, uint32_t* claim = nullptr) {
  using S = OnesweepShape<K, NoVal, BITS, THREADS, KPT>;
  using F = FirstShape<K, BITS, THREADS, KPT>;
  constexpr int R = S::R, DPT = S::DPT;
  uint32_t* s_slot = reinterpret_cast<uint32_t*>(smem);  // [R] counts, then next free slot
  uint32_t* s_adj = s_slot + R;                           // [R]
  uint32_t* s_misc = s_adj + R;                           // [64]
  K* s_keys = reinterpret_cast<K*>(smem + F::HEADER_WORDS * 4);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wofs = warp * 32 * KPT + lane;
  const bool publish = (int64_t)tile != p.stall_tile;

  K key[KPT];
  NoVal val[1];
  tile_load<K, NoVal, KPT, FULL>(kin, nullptr, tile_base, tile_n, wofs, key, val);
  dig.prepare(key);
#pragma unroll
  for (int i = 0; i < KPT; ++i)
    if (FULL || wofs + i * 32 < tile_n) atomicAdd(&s_slot[dig.of(key[i], i)], 1u);
  __syncthreads();

  uint32_t dcnt[DPT], claimed[DPT];
  uint32_t tsum = 0;
  const bool owner = tid < S::DTHREADS;
  if (owner) {
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      dcnt[j] = s_slot[tid * DPT + j];
      tsum += dcnt[j];
      claimed[j] = 0;
      if (claim) {  // the add returns before it is needed (after the placement)
        if (dcnt[j]) claimed[j] = atomicAdd(&claim[tid * DPT + j], dcnt[j]);
      } else if (publish) {
        st_relaxed(&p.status[(size_t)tile * R + tid * DPT + j],
                   (first ? kFlagInc : kFlagAgg) | dcnt[j]);
      }
    }
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan<THREADS>(tsum, s_misc + 1, total);
  uint32_t tstart[DPT];
  if (owner) {
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      tstart[j] = run;
      s_slot[tid * DPT + j] = run;
      run += dcnt[j];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < KPT; ++i)
    if (FULL || wofs + i * 32 < tile_n) {
      const uint32_t d = dig.of(key[i], i);
      const uint32_t pos = atomicAdd(&s_slot[d], 1u);
      s_keys[pos] = key[i];
      dig.keep(pos, d);
    }

  uint32_t windows = 0;
  if (owner) {
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int d = tid * DPT + j;
      uint32_t excl = claimed[j];
      if (!claim && !first) {
        excl = lookback_exclusive<R, kLookbackWindow>(p.status, tile, d, p.spin_limit, p.err,
                                                      windows);
        if (publish) st_relaxed(&p.status[(size_t)tile * R + d], kFlagInc | (excl + dcnt[j]));
      }
      s_adj[d] = base[d] + excl - tstart[j];
    }
  }
  __syncthreads();
  tile_scatter<K, THREADS, KPT, FULL>(s_keys, s_adj, dig, tile_n, kout, bound, p.err);
}

// The first round (pass 0) of a keys-only sort; a skipped pass 0 leaves the
// first executed round to the ordered kernel.
// DS: the digit rule (bytes for radix 256; a digit part for the first routing
// step of a wide radix).
template <typename K, int BITS, int THREADS, int KPT, int MINB, typename DS = RadixDigit>
__global__ void __launch_bounds__(THREADS, MINB) k_onesweep_first(PassParams p) {
  using S = OnesweepShape<K, NoVal, BITS, THREADS, KPT>;
  constexpr int R = S::R, TILE = S::TILE;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_slot = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_misc = s_slot + 2 * R;
  const int tid = threadIdx.x;
  if (p.status_next)
    for (int d = tid; d < R; d += THREADS) p.status_next[(size_t)blockIdx.x * R + d] = 0;
  if (p.skip[0]) return;
  if (tid == 0) s_misc[0] = atomicAdd(p.counter, 1u);  // tiles in launch order
  zero_words<THREADS>(s_slot, R);
  __syncthreads();
  const uint32_t tile = s_misc[0];
  const int tile_n = (int)min((int64_t)TILE, p.n - (int64_t)tile * TILE);
  const K* kin = static_cast<const K*>(p.keys[0]);
  K* kout = static_cast<K*>(p.keys[1]);
  if (p.prefetch_tiles && tid == 0) {  // the tile one wave ahead into L2, as the ordered round
    const int64_t pf = ((int64_t)tile + p.prefetch_tiles) * TILE;
    prefetch_tile(kin, pf, min((int64_t)TILE, p.n - pf));
  }
  const int64_t tile_base = (int64_t)tile * TILE;
  DS dig{p};
  if (tile_n == TILE)
    onesweep_tile_first<K, BITS, THREADS, KPT, true, DS>(p, tile, tile == 0, tile_base, tile_n,
                                                         kin, kout, p.base, (uint32_t)p.n, smem,
                                                         dig, p.claim);
  else
    onesweep_tile_first<K, BITS, THREADS, KPT, false, DS>(p, tile, tile == 0, tile_base, tile_n,
                                                          kin, kout, p.base, (uint32_t)p.n, smem,
                                                          dig, p.claim);
}

// ---------------------------------------------------------------------------
// k_copy_back: after an odd number of executed rounds the sorted keys sit in
// the alternate buffer; copy them (and payloads) home. Otherwise a no-op.
template <typename K, typename V>
__global__ void k_copy_back(const uint32_t* __restrict__ skip, int passes, K* keys,
                            const K* alt, V* vals, const V* valt, int64_t n) {
  int parity = 0;
  for (int q = 0; q < passes; ++q) parity ^= (skip[q] == 0);
  if (!parity) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = alt[i];
    if constexpr (HasVal<V>::value) vals[i] = valt[i];
  }
}

// ---------------------------------------------------------------------------
// Host launcher for one whole sort with a given kernel shape: one tile per CTA
// with a per-tile look-back.
template <typename K, typename V, int BITS, int THREADS, int KPT, int MINB>
cudaError_t lsd_launch(const LsdArgs& a, cudaStream_t st) {
  static_assert(BITS == 8, "the rounds take digits as bytes (RadixDigit)");
  using L = DigitLayout<K, BITS>;
  using S = OnesweepShape<K, V, BITS, THREADS, KPT>;
  constexpr int R = L::R, P = L::PASSES;
  constexpr bool HV = HasVal<V>::value;
  const int64_t tiles = (a.n + S::TILE - 1) / S::TILE;
  cudaError_t e;
  // hist and counters are zeroed; status[0] too (later passes clear their own)
  if ((e = cudaMemsetAsync(a.hist, 0, sizeof(uint32_t) * P * R, st))) return e;
  if ((e = cudaMemsetAsync(a.counters, 0, sizeof(uint32_t) * P, st))) return e;
  // status[0] serves pass 0 only when that pass looks back (payloads: every
  // round is ordered); later passes clear their successor's rows themselves
  if (HV && (e = cudaMemsetAsync(a.status[0], 0, sizeof(uint32_t) * R * tiles, st))) return e;

  // 32 counter columns for 32-bit keys (4 passes: 128 KiB), 16 for 64-bit
  // keys (8 passes: 128 KiB); one 1024-thread CTA per SM.
  constexpr int HT = 1024;
  constexpr int LANES = sizeof(K) == 4 ? 32 : 16;
  using HS = HistShape<K, BITS, HT, LANES>;
  auto hk = k_hist<K, BITS, HT, LANES>;
  if ((e = cudaFuncSetAttribute(hk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HS::SMEM)))
    return e;
  int64_t want = (a.n / Vec16<K>::N + HT * 4 - 1) / (HT * 4);
  int hblocks = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)a.num_sms);
  timer_begin(a.timer, "k_hist", st);
  hk<<<hblocks, HT, HS::SMEM, st>>>(static_cast<const K*>(a.keys), a.n, a.hist);
  timer_end(a.timer, st);
  timer_begin(a.timer, "k_scan", st);
  k_scan<256><<<P, 256, 0, st>>>(a.hist, a.base, a.skip, R, a.n, HV ? nullptr : a.claim);
  timer_end(a.timer, st);

  PassParams pp;
  pp.keys[0] = a.keys;
  pp.keys[1] = a.alt_keys;
  pp.vals[0] = a.vals;
  pp.vals[1] = a.alt_vals;
  pp.n = a.n;
  pp.skip = a.skip;
  pp.err = a.err;
  pp.spin_limit = a.spin_limit;
  pp.prefetch_tiles = a.prefetch_tiles;
  pp.check_mode = a.check_mode;
  constexpr size_t smem = OrderedShape<K, V, BITS, THREADS, KPT>::SMEM;
  auto kern = k_onesweep<K, V, BITS, THREADS, KPT, MINB>;
  if (smem > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
      return e;
  }
  // keys only: pass 0 is the order-free round (k_onesweep_first)
  using FC = FirstCfg<K, THREADS, KPT, MINB>;
  constexpr size_t fsmem = FirstShape<K, BITS, FC::T, FC::KP>::SMEM;
  if constexpr (!HV && fsmem > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(k_onesweep_first<K, BITS, FC::T, FC::KP, MINB>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem)))
      return e;
  }
  for (int q = 0; q < P; ++q) {
    pp.pass = q;
    pp.shift = q * BITS;
    pp.mask = (1u << L::width(q)) - 1;
    pp.byte_sel = radix8_byte_sel(pp.shift);
    pp.low_shift = pp.shift;
    pp.base = a.base + (size_t)q * R;
    pp.status = a.status[q & 1];
    pp.status_next = (q + 1 < P) ? a.status[(q + 1) & 1] : nullptr;
    pp.counter = a.counters + q;
    pp.claim = (!HV && q == 0) ? a.claim : nullptr;
    // the stall hook applies to the first round with a look-back
    pp.stall_tile = (q == (HV ? 0 : 1)) ? a.stall_tile : -1;
    bool launched = false;
    if constexpr (!HV) {
      if (q == 0) {
        timer_begin(a.timer, "k_onesweep_first", st);
        k_onesweep_first<K, BITS, FC::T, FC::KP, MINB><<<(unsigned)tiles, FC::T, fsmem, st>>>(pp);
        launched = true;
      }
    }
    if (!launched) {
      timer_begin(a.timer, "k_onesweep", st);
      kern<<<(unsigned)tiles, THREADS, smem, st>>>(pp);
    }
    timer_end(a.timer, st);
  }
  int cblocks = (int)std::min<int64_t>((a.n + 255) / 256, (int64_t)a.num_sms * 8);
  timer_begin(a.timer, "k_copy_back", st);
  k_copy_back<K, V><<<cblocks, 256, 0, st>>>(a.skip, P, static_cast<K*>(a.keys),
                                             static_cast<const K*>(a.alt_keys),
                                             static_cast<V*>(a.vals),
                                             static_cast<const V*>(a.alt_vals), a.n);
  timer_end(a.timer, st);
  return cudaGetLastError();
}

// MINB = CTAs that must fit on one SM (caps registers at 65536 / (THREADS * MINB)).
template <typename K, typename V, int BITS, int THREADS, int KPT, int MINB>
constexpr LsdEntry lsd_entry() {
  using S = OnesweepShape<K, V, BITS, THREADS, KPT>;
  return LsdEntry{(int)(8 * sizeof(K)),
                  HasVal<V>::value ? (int)(8 * sizeof(V)) : 0,
                  BITS,
                  THREADS,
                  KPT,
                  (int64_t)S::TILE,  // one look-back row per tile
                  S::R,
                  DigitLayout<K, BITS>::PASSES,
                  (size_t)S::R,
                  2,
                  &lsd_launch<K, V, BITS, THREADS, KPT, MINB>};
}

}  // namespace isort
