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
// SUBS sub-histograms per CTA (warp w uses w % SUBS) spread shared atomics.
template <typename K, int BITS, int THREADS, int SUBS>
__global__ void __launch_bounds__(THREADS) k_hist(const K* __restrict__ keys, int64_t n,
                                                  uint32_t* __restrict__ hist) {
  using L = DigitLayout<K, BITS>;
  constexpr int R = L::R, P = L::PASSES;
  __shared__ uint32_t s_hist[SUBS][P * R];
  for (int i = threadIdx.x; i < SUBS * P * R; i += THREADS) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  uint32_t* my = s_hist[(threadIdx.x >> 5) % SUBS];

  auto count = [&](K k) {
#pragma unroll
    for (int p = 0; p < P; ++p)
      atomicAdd(&my[p * R + digit_of(k, p * BITS, (1u << L::width(p)) - 1)], 1u);
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
#pragma unroll
    for (int b = 0; b < SUBS; ++b) s += s_hist[b][j];
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
};

template <typename K, typename V, int BITS, int THREADS, int KPT>
struct OnesweepShape {
  static constexpr int R = 1 << BITS;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int TILE = THREADS * KPT;
  static constexpr bool HV = HasVal<V>::value;
  static constexpr int STAGE_ELEM = (HV && sizeof(V) > sizeof(K)) ? sizeof(V) : sizeof(K);
  static constexpr int HEADER_WORDS = WARPS * R + R + 64;
  static constexpr size_t SMEM = HEADER_WORDS * 4 + (size_t)TILE * STAGE_ELEM;
  static constexpr int DPT = R >= THREADS ? R / THREADS : 1;  // digits per owning thread
  static constexpr int DTHREADS = R >= THREADS ? THREADS : R;  // threads that own digits
};

template <typename K, typename V, int BITS, int THREADS, int KPT>
__global__ void __launch_bounds__(THREADS) k_onesweep(PassParams p) {
  using S = OnesweepShape<K, V, BITS, THREADS, KPT>;
  constexpr int R = S::R, WARPS = S::WARPS, TILE = S::TILE, DPT = S::DPT;
  constexpr bool HV = S::HV;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_wcnt = reinterpret_cast<uint32_t*>(smem);  // [WARPS][R]
  uint32_t* s_adj = s_wcnt + WARPS * R;                   // [R]
  uint32_t* s_misc = s_adj + R;                           // [64]
  K* s_keys = reinterpret_cast<K*>(smem + S::HEADER_WORDS * 4);
  V* s_vals = reinterpret_cast<V*>(smem + S::HEADER_WORDS * 4);
  (void)s_vals;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // Rows of the next pass's look-back array are cleared here, so one memset
  // before the first pass is the only one a sort needs.
  if (p.status_next)
    for (int d = tid; d < R; d += THREADS) p.status_next[(size_t)blockIdx.x * R + d] = 0;
  if (p.skip[p.pass]) return;  // the digit is constant: this round is the identity

  int src = 0;  // input buffer = parity of the rounds executed before this one
  for (int q = 0; q < p.pass; ++q) src ^= (p.skip[q] == 0);
  // select with branches, not a dynamic index, so the parameters stay out of local memory
  const K* __restrict__ kin = static_cast<const K*>(src ? p.keys[1] : p.keys[0]);
  K* __restrict__ kout = static_cast<K*>(src ? p.keys[0] : p.keys[1]);

  if (tid == 0) s_misc[0] = atomicAdd(p.counter, 1u);  // tiles in launch order
  for (int i = tid; i < WARPS * R; i += THREADS) s_wcnt[i] = 0;
  __syncthreads();
  const uint32_t tile = s_misc[0];
  const int64_t tile_base = (int64_t)tile * TILE;
  const int tile_n = (int)min((int64_t)TILE, p.n - tile_base);

  // ---- load: warp w owns keys [w*32*KPT, (w+1)*32*KPT) of the tile, lane-striped
  K key[KPT];
  V val[HV ? KPT : 1];
  const int wofs = warp * 32 * KPT + lane;
  const int64_t g0 = tile_base + wofs;
  if (tile_n == TILE) {
#pragma unroll
    for (int i = 0; i < KPT; ++i) key[i] = kin[g0 + i * 32];
    if constexpr (HV) {
      const V* vin = static_cast<const V*>(src ? p.vals[1] : p.vals[0]);
#pragma unroll
      for (int i = 0; i < KPT; ++i) val[i] = vin[g0 + i * 32];
    }
  } else {
#pragma unroll
    for (int i = 0; i < KPT; ++i) key[i] = (wofs + i * 32 < tile_n) ? kin[g0 + i * 32] : K(0);
    if constexpr (HV) {
      const V* vin = static_cast<const V*>(src ? p.vals[1] : p.vals[0]);
#pragma unroll
      for (int i = 0; i < KPT; ++i) val[i] = (wofs + i * 32 < tile_n) ? vin[g0 + i * 32] : V(0);
    }
  }

  // ---- rank: position of each key among the warp's keys of the same digit,
  // in input order (i ascending, then lane ascending). Invalid tail slots use
  // the sentinel digit R and are not counted.
  uint32_t rank[KPT];
  {
    uint32_t* my = s_wcnt + warp * R;
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      const uint32_t d = (wofs + i * 32 < tile_n) ? digit_of(key[i], p.shift, p.mask) : R;
      const uint32_t peers = __match_any_sync(kFullMask, d);
      const int leader = 31 - __clz(peers);
      uint32_t before = 0;
      if (lane == leader && d < R) {
        before = my[d];
        my[d] = before + __popc(peers);
      }
      before = __shfl_sync(kFullMask, before, leader);
      rank[i] = before + __popc(peers & lt);
      __syncwarp();
    }
  }
  __syncthreads();

  // ---- per digit: warp-exclusive offsets, the tile's count, early publication
  uint32_t dcnt[DPT];
  uint32_t tsum = 0;
  const bool owner = tid < S::DTHREADS;
  const bool publish = (int64_t)tile != p.stall_tile;
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
        st_relaxed(&p.status[(size_t)tile * R + d], (tile == 0 ? kFlagInc : kFlagAgg) | sum);
    }
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan<THREADS>(tsum, s_misc + 1, total);

  // ---- look-back over earlier tiles, then publish the inclusive count
  if (owner) {
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int d = tid * DPT + j;
      const uint32_t tstart = run;  // tile-local start of digit d
      run += dcnt[j];
      uint32_t excl = 0;
      if (tile > 0) {
        int64_t t = (int64_t)tile - 1;
        while (true) {
          const uint32_t* w = &p.status[(size_t)t * R + d];
          uint32_t s = ld_relaxed(w);
          uint32_t spins = 0;
          while ((s & ~kCountMask) == 0 && ++spins < p.spin_limit) s = ld_relaxed(w);
          if ((s & ~kCountMask) == 0) {
            atomicOr(p.err, kErrTimeout);
            break;
          }
          excl += s & kCountMask;
          if ((s & kFlagInc) || t == 0) break;
          --t;
        }
        if (publish) st_relaxed(&p.status[(size_t)tile * R + d], kFlagInc | (excl + dcnt[j]));
      }
      s_adj[d] = p.base[d] + excl - tstart;
#pragma unroll
      for (int w = 0; w < WARPS; ++w) s_wcnt[w * R + d] += tstart;
    }
  }
  __syncthreads();

  // ---- reorder the tile by digit in shared memory (stable by construction)
  const uint32_t* myofs = s_wcnt + warp * R;
#pragma unroll
  for (int i = 0; i < KPT; ++i) {
    if (wofs + i * 32 < tile_n) {
      const uint32_t pos = myofs[digit_of(key[i], p.shift, p.mask)] + rank[i];
      s_keys[pos] = key[i];
      rank[i] = pos;
    }
  }
  __syncthreads();

  // ---- write out: consecutive threads take consecutive tile slots, so each
  // digit's run lands on consecutive global addresses
  uint32_t gpos[HV ? KPT : 1];
  const uint32_t n32 = (uint32_t)p.n;
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int j = k * THREADS + tid;
    if (j < tile_n) {
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
    V* __restrict__ vout = static_cast<V*>(src ? p.vals[0] : p.vals[1]);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < KPT; ++i)
      if (wofs + i * 32 < tile_n) s_vals[rank[i]] = val[i];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int j = k * THREADS + tid;
      if (j < tile_n && gpos[k] < n32) vout[gpos[k]] = s_vals[j];
    }
  }
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
template <typename K, typename V, int BITS, int THREADS, int KPT>
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

  constexpr int HT = 512;
  int64_t want = (a.n / Vec16<K>::N + HT * 4 - 1) / (HT * 4);
  int hblocks = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)a.num_sms * 4);
  timer_begin(a.timer, "k_hist", st);
  k_hist<K, BITS, HT, 4><<<hblocks, HT, 0, st>>>(static_cast<const K*>(a.keys), a.n, a.hist);
  timer_end(a.timer, st);
  timer_begin(a.timer, "k_scan", st);
  k_scan<256><<<P, 256, 0, st>>>(a.hist, a.base, a.skip, R, a.n);
  timer_end(a.timer, st);

  auto kern = k_onesweep<K, V, BITS, THREADS, KPT>;
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

template <typename K, typename V, int BITS, int THREADS, int KPT>
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
                  &lsd_launch<K, V, BITS, THREADS, KPT>};
}

}  // namespace isort
