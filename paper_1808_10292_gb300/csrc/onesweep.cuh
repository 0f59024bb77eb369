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
//   k_onesweep  one round: load a tile, rank each key among equal digits in
//               input order (warp match + per-warp counters), publish the tile's
//               digit counts, look back over earlier tiles, reorder the tile by
//               digit in shared memory and write it out in runs.
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

  using V16 = Vec16<K>;
  const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
  int64_t head = (int64_t)(((16 - (addr & 15)) & 15) / sizeof(K));
  if (head > n) head = n;
  const int64_t nvec = (n - head) / V16::N;
  const typename V16::T* vec = reinterpret_cast<const typename V16::T*>(keys + head);
  const int64_t gtid = blockIdx.x * (int64_t)THREADS + threadIdx.x;
  const int64_t gsize = (int64_t)gridDim.x * THREADS;

  if (gtid < head) count(keys[gtid]);
  constexpr int U = 4;  // independent 16-byte loads in flight per thread
  int64_t i = gtid;
  for (; i + (U - 1) * gsize < nvec; i += U * gsize) {
    typename V16::T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = vec[i + u * gsize];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int c = 0; c < V16::N; ++c) count(V16::get(v[u], c));
  }
  for (; i < nvec; i += gsize) {
    typename V16::T v = vec[i];
#pragma unroll
    for (int c = 0; c < V16::N; ++c) count(V16::get(v, c));
  }
  const int64_t tail0 = head + nvec * V16::N;
  if (tail0 + gtid < n) count(keys[tail0 + gtid]);
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
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_scan(const uint32_t* __restrict__ hist,
                                                  uint32_t* __restrict__ base,
                                                  uint32_t* __restrict__ skip, int R, int64_t n) {
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
  uint32_t* err;
  uint32_t spin_limit;
  int64_t stall_tile;
  unsigned long long* trace;  // measurement hook: per tile, phase timestamps (or null)
};

__device__ __forceinline__ uint32_t lanemask_ge() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_ge;" : "=r"(m));
  return m;
}

template <typename K, typename V, int BITS, int THREADS, int KPT>
struct OnesweepShape {
  static constexpr int R = 1 << BITS;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int TILE = THREADS * KPT;
  static constexpr bool HV = HasVal<V>::value;
  static constexpr int STAGE_ELEM = (HV && sizeof(V) > sizeof(K)) ? sizeof(V) : sizeof(K);
  static constexpr int MASK_BUFS = 3;  // peer-mask buffers per warp (see the rank loop)
  // shared words: per-warp counters, output offsets, misc; then the staging area
  static constexpr int HEADER_WORDS = WARPS * R + R + 64;
  static constexpr size_t STAGE_BYTES =
      (size_t)TILE * STAGE_ELEM > (size_t)WARPS * MASK_BUFS * R * 4
          ? (size_t)TILE * STAGE_ELEM
          : (size_t)WARPS * MASK_BUFS * R * 4;
  static constexpr size_t SMEM = HEADER_WORDS * 4 + STAGE_BYTES;
  static constexpr int DPT = R >= THREADS ? R / THREADS : 1;  // digits per owning thread
  static constexpr int DTHREADS = R >= THREADS ? THREADS : R;  // threads that own digits
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
  uint32_t excl = 0, polls = 0;
  int64_t t = (int64_t)tile - 1;
  while (true) {
    ++windows;
    uint32_t s[LB];
#pragma unroll
    for (int k = 0; k < LB; ++k)  // below tile 0 reads as "inclusive, count 0"
      s[k] = (t - k >= 0) ? ld_relaxed(&status[(size_t)(t - k) * R + d]) : kFlagInc;
    uint32_t add = 0;
    int consumed = 0;
    bool found_inc = false, blocked = false;
#pragma unroll
    for (int k = 0; k < LB; ++k) {
      if (!found_inc && !blocked) {
        const uint32_t f = s[k] & ~kCountMask;
        if (f == 0) {
          blocked = true;  // tile t-k has published nothing yet: poll it again
        } else {
          add += s[k] & kCountMask;
          ++consumed;
          found_inc = (f & kFlagInc) != 0;
        }
      }
    }
    excl += add;
    if (found_inc) break;
    t -= consumed;
    if (blocked) {
      if (++polls >= spin_limit) {
        atomicOr(err, kErrTimeout);
        break;
      }
      __nanosleep(32);
    }
  }
  return excl;
}

// One tile of one count-sort round. FULL: the tile holds TILE keys, so no
// per-key bounds predicate is needed.
//   tile       row of the look-back arrays (tile id in launch order)
//   first      the tile opens its range (segment), so it has no predecessor
//   tile_base  index of the tile's first key in kin / vin
//   kout/vout  the range's output (positions are relative to the range start)
//   base       [R] the range's exclusive digit bases for this pass
//   bound      keys in the range (every output index is checked against it)
template <typename K, typename V, int BITS, int THREADS, int KPT, bool FULL>
__device__ __forceinline__ void onesweep_tile(const PassParams& p, uint32_t tile, bool first,
                                              int64_t tile_base, int tile_n,
                                              const K* __restrict__ kin, K* __restrict__ kout,
                                              const V* vin, V* vout, const uint32_t* base,
                                              uint32_t bound, unsigned char* smem) {
  using S = OnesweepShape<K, V, BITS, THREADS, KPT>;
  constexpr int R = S::R, WARPS = S::WARPS, DPT = S::DPT;
  constexpr bool HV = S::HV;
  uint32_t* s_wcnt = reinterpret_cast<uint32_t*>(smem);  // [WARPS][R]
  uint32_t* s_adj = s_wcnt + WARPS * R;                   // [R]
  uint32_t* s_misc = s_adj + R;                           // [64]
  K* s_keys = reinterpret_cast<K*>(smem + S::HEADER_WORDS * 4);
  V* s_vals = reinterpret_cast<V*>(smem + S::HEADER_WORDS * 4);
  (void)s_vals;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool publish = (int64_t)tile != p.stall_tile;

  // ---- load: warp w owns keys [w*32*KPT, (w+1)*32*KPT) of the tile, lane-striped
  K key[KPT];
  V val[HV ? KPT : 1];
  const int wofs = warp * 32 * KPT + lane;
  const int64_t g0 = tile_base + wofs;
#pragma unroll
  for (int i = 0; i < KPT; ++i)
    key[i] = (FULL || wofs + i * 32 < tile_n) ? kin[g0 + i * 32] : K(0);
  if constexpr (HV) {
#pragma unroll
    for (int i = 0; i < KPT; ++i)
      val[i] = (FULL || wofs + i * 32 < tile_n) ? vin[g0 + i * 32] : V(0);
  }

  // ---- rank: position of each key among the warp's keys of the same digit,
  // in input order (i ascending, then lane ascending). Lanes find their peers
  // (same digit, same iteration) through a per-warp shared-memory mask per
  // digit: each lane ORs in its bit, and after a warp barrier reads the mask
  // back. The highest peer advances the warp's private counter of the digit
  // with one atomic add and hands the old value to its peers.
  // Ordering with one warp barrier per iteration: three mask buffers rotate,
  // and the slot used in iteration i-2 is cleared in iteration i -- after the
  // barrier of i-1 (so every read of it is done) and before the barrier of i
  // (which precedes the next OR into that buffer, in i+1). A counter update of
  // iteration i precedes the barrier of i+1, which precedes the next update.
  // The masks live in the staging area, which is free until the reorder.
  // Ranks (< TILE <= 65536) are kept as 16-bit halves to save registers.
  uint32_t rank2[(KPT + 1) / 2];
  {
    uint32_t* my = s_wcnt + warp * R;
    uint32_t* mm = reinterpret_cast<uint32_t*>(s_keys) + warp * S::MASK_BUFS * R;
    const uint32_t ge = lanemask_ge();
    const uint32_t bit = 1u << lane;
    uint32_t* slot1 = mm;  // slot of iteration i-1
    uint32_t* slot2 = mm;  // slot of iteration i-2
    bool lead1 = false, lead2 = false;
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      const bool valid = FULL || wofs + i * 32 < tile_n;
      const uint32_t d = digit_of(key[i], p.shift, p.mask);
      uint32_t* slot = mm + (i % S::MASK_BUFS) * R + d;
      if (lead2) *slot2 = 0u;
      if (valid) atomicOr(slot, bit);
      __syncwarp();
      const uint32_t peers = valid ? *slot : 0u;
      const bool leader = valid && (peers >> lane) == 1u;  // highest peer
      uint32_t after = 0;
      if (leader) after = atomicAdd(&my[d], __popc(peers)) + __popc(peers);
      after = __shfl_sync(kFullMask, after, (31 - __clz(peers)) & 31);
      const uint32_t r = after - __popc(peers & ge);  // = old count + peers below me
      rank2[i >> 1] = (i & 1) ? (rank2[i >> 1] | (r << 16)) : r;
      slot2 = slot1;
      lead2 = lead1;
      slot1 = slot;
      lead1 = leader;
    }
  }
  __syncthreads();
  if (p.trace && tid == 0) p.trace[(size_t)tile * 8 + 1] = globaltimer();

  // ---- per digit: warp-exclusive offsets and the tile's count, published at
  // once (AGG, or INC for tile 0) so that later tiles can use it
  uint32_t dcnt[DPT];
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

  // ---- look-back over earlier tiles, then publish the inclusive count
  uint32_t windows = 0;
  if (p.trace && tid == 0) p.trace[(size_t)tile * 8 + 2] = globaltimer();
  if (owner) {
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int d = tid * DPT + j;
      const uint32_t tstart = run;  // tile-local start of digit d
      run += dcnt[j];
      uint32_t excl = 0;
      if (!first) {
        excl = lookback_exclusive<R, kLookbackWindow>(p.status, tile, d, p.spin_limit, p.err,
                                                      windows);
        if (publish) st_relaxed(&p.status[(size_t)tile * R + d], kFlagInc | (excl + dcnt[j]));
      }
      s_adj[d] = base[d] + excl - tstart;
#pragma unroll
      for (int w = 0; w < WARPS; ++w) s_wcnt[w * R + d] += tstart;
    }
  }
  if (p.trace && tid == 0) p.trace[(size_t)tile * 8 + 6] = windows;
  __syncthreads();
  if (p.trace && tid == 0) p.trace[(size_t)tile * 8 + 3] = globaltimer();

  // ---- reorder the tile by digit in shared memory (stable by construction)
  const uint32_t* myofs = s_wcnt + warp * R;
#pragma unroll
  for (int i = 0; i < KPT; ++i) {
    if (FULL || wofs + i * 32 < tile_n) {
      const uint32_t r = (rank2[i >> 1] >> ((i & 1) * 16)) & 0xffffu;
      const uint32_t pos = myofs[digit_of(key[i], p.shift, p.mask)] + r;
      s_keys[pos] = key[i];
      if constexpr (HV) {  // keep the tile position for the payload pass
        rank2[i >> 1] = (i & 1) ? ((rank2[i >> 1] & 0xffffu) | (pos << 16))
                                : ((rank2[i >> 1] & 0xffff0000u) | pos);
      }
    }
  }
  __syncthreads();
  if (p.trace && tid == 0) p.trace[(size_t)tile * 8 + 4] = globaltimer();

  // ---- write out: consecutive threads take consecutive tile slots, so each
  // digit's run lands on consecutive global addresses
  uint32_t gpos[HV ? KPT : 1];
  const uint32_t n32 = bound;
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int j = k * THREADS + tid;
    if (FULL || j < tile_n) {
      const K kk = s_keys[j];
      const uint32_t g = s_adj[digit_of(kk, p.shift, p.mask)] + (uint32_t)j;
      if (g < n32)
        kout[g] = kk;
      else
        atomicOr(p.err, kErrBounds);
      if constexpr (HV) gpos[k] = g;
    }
  }
  if constexpr (HV) {
    __syncthreads();
#pragma unroll
    for (int i = 0; i < KPT; ++i)
      if (FULL || wofs + i * 32 < tile_n)
        s_vals[(rank2[i >> 1] >> ((i & 1) * 16)) & 0xffffu] = val[i];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int j = k * THREADS + tid;
      if ((FULL || j < tile_n) && gpos[k] < n32) vout[gpos[k]] = s_vals[j];
    }
  }
  if (p.trace && tid == 0) p.trace[(size_t)tile * 8 + 5] = globaltimer();
}

template <typename K, typename V, int BITS, int THREADS, int KPT, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_onesweep(PassParams p) {
  using S = OnesweepShape<K, V, BITS, THREADS, KPT>;
  constexpr int R = S::R, WARPS = S::WARPS, TILE = S::TILE;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_wcnt = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_misc = s_wcnt + WARPS * R + R;
  uint32_t* s_stage = reinterpret_cast<uint32_t*>(smem + S::HEADER_WORDS * 4);
  const int tid = threadIdx.x;

  // Rows of the next pass's look-back array are cleared here, so one memset
  // before the first pass is the only one a sort needs.
  if (p.status_next)
    for (int d = tid; d < R; d += THREADS) p.status_next[(size_t)blockIdx.x * R + d] = 0;
  if (p.skip[p.pass]) return;  // the digit is constant: this round is the identity

  int src = 0;  // input buffer = parity of the rounds executed before this one
  for (int q = 0; q < p.pass; ++q) src ^= (p.skip[q] == 0);

  if (tid == 0) s_misc[0] = atomicAdd(p.counter, 1u);  // tiles in launch order
  for (int i = tid; i < WARPS * R; i += THREADS) s_wcnt[i] = 0;
  for (int i = tid; i < WARPS * S::MASK_BUFS * R; i += THREADS) s_stage[i] = 0;
  __syncthreads();
  const uint32_t tile = s_misc[0];
  const int tile_n = (int)min((int64_t)TILE, p.n - (int64_t)tile * TILE);
  if (p.trace && tid == 0) {
    p.trace[(size_t)tile * 8 + 0] = globaltimer();
    p.trace[(size_t)tile * 8 + 7] = smid();
  }
  // select with branches, not a dynamic index, so the parameters stay out of local memory
  const K* kin = static_cast<const K*>(src ? p.keys[1] : p.keys[0]);
  K* kout = static_cast<K*>(src ? p.keys[0] : p.keys[1]);
  const V* vin = static_cast<const V*>(src ? p.vals[1] : p.vals[0]);
  V* vout = static_cast<V*>(src ? p.vals[0] : p.vals[1]);
  const int64_t tile_base = (int64_t)tile * TILE;
  if (tile_n == TILE)
    onesweep_tile<K, V, BITS, THREADS, KPT, true>(p, tile, tile == 0, tile_base, tile_n, kin, kout,
                                                  vin, vout, p.base, (uint32_t)p.n, smem);
  else
    onesweep_tile<K, V, BITS, THREADS, KPT, false>(p, tile, tile == 0, tile_base, tile_n, kin,
                                                   kout, vin, vout, p.base, (uint32_t)p.n, smem);
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
// Host launcher for one whole sort with a given kernel shape.
template <typename K, typename V, int BITS, int THREADS, int KPT, int MINB>
cudaError_t lsd_launch(const LsdArgs& a, cudaStream_t st) {
  using L = DigitLayout<K, BITS>;
  using S = OnesweepShape<K, V, BITS, THREADS, KPT>;
  constexpr int R = L::R, P = L::PASSES;
  const int64_t tiles = (a.n + S::TILE - 1) / S::TILE;
  cudaError_t e;
  // hist and counters are zeroed; status[0] too (later passes clear their own)
  if ((e = cudaMemsetAsync(a.hist, 0, sizeof(uint32_t) * P * R, st))) return e;
  if ((e = cudaMemsetAsync(a.counters, 0, sizeof(uint32_t) * P, st))) return e;
  if ((e = cudaMemsetAsync(a.status[0], 0, sizeof(uint32_t) * R * tiles, st))) return e;

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
  k_scan<256><<<P, 256, 0, st>>>(a.hist, a.base, a.skip, R, a.n);
  timer_end(a.timer, st);

  auto kern = k_onesweep<K, V, BITS, THREADS, KPT, MINB>;
  if (S::SMEM > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)S::SMEM)))
      return e;
  }
  PassParams pp;
  pp.keys[0] = a.keys;
  pp.keys[1] = a.alt_keys;
  pp.vals[0] = a.vals;
  pp.vals[1] = a.alt_vals;
  pp.n = a.n;
  pp.skip = a.skip;
  pp.err = a.err;
  pp.spin_limit = a.spin_limit;
  for (int q = 0; q < P; ++q) {
    pp.pass = q;
    pp.shift = q * BITS;
    pp.mask = (1u << L::width(q)) - 1;
    pp.base = a.base + (size_t)q * R;
    pp.status = a.status[q & 1];
    pp.status_next = (q + 1 < P) ? a.status[(q + 1) & 1] : nullptr;
    pp.counter = a.counters + q;
    pp.stall_tile = (q == 0) ? a.stall_tile : -1;
    pp.trace = (q == a.trace_pass) ? a.trace : nullptr;
    timer_begin(a.timer, "k_onesweep", st);
    kern<<<(unsigned)tiles, THREADS, S::SMEM, st>>>(pp);
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
                  S::TILE,
                  S::R,
                  DigitLayout<K, BITS>::PASSES,
                  (size_t)S::R,
                  2,
                  &lsd_launch<K, V, BITS, THREADS, KPT, MINB>};
}

}  // namespace isort
