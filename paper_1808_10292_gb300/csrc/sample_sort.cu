// GVR on one GPU: the paper's random-oversampling sample sort (Algorithm 3,
// Section "Oversampling algorithms: GSD, GVR, GER") as a splitter partition
// pass in front of the segmented sort.
//
//   k_gvr_sample  one CTA draws the sample of s*p - 1 keys at counter-based
//                 random positions, sorts it with the BTN network and keeps
//                 the (i*s)-th smallest keys, 1 <= i <= p - 1, as splitters.
//   k_gvr_hist    per key, its bucket = the number of splitters smaller than
//                 it (a binary search in shared memory); bucket counts.
//   k_gvr_scan    bucket bases (the round's digit bases), the int64 bucket
//                 offsets for the segmented sort, the caller's bucket counts.
//   k_gvr_split   one count-sort round with digit = bucket: the radix-256
//                 round's tile machinery with the bucket as the digit. With
//                 payloads the ordered round (early counts, look-back,
//                 scatter; stable, so payloads keep input order inside a
//                 bucket); keys only the order-free round, whose tiles take
//                 their bucket ranges from per-bucket cursors.
// The buckets are then sorted independently by the segmented sort (the
// paper's step 4 sorts each with SR4); that part lives in api.cu.
#include "segmented.cuh"

namespace isort {
namespace {

// SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
// generators", 2014): the output mix, and the stream construction used for
// the sample: S = mix(seed * gamma ^ stream * C), draw i = mix(S + (i+1) * gamma).
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kStreamMul = 0xD1B54A32D192ED03ull;
constexpr uint64_t kSampleStream = 30;  // stream id of the sample positions

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Position of sample item m in [0, n): the high 32 bits of the draw scaled to n.
__device__ __forceinline__ int64_t sample_pos(uint64_t seed, uint64_t m, int64_t n) {
  const uint64_t S = sm64_mix(seed * kGamma ^ kSampleStream * kStreamMul);
  const uint64_t d = sm64_mix(S + (m + 1) * kGamma);
  return (int64_t)(((d >> 32) * (uint64_t)n) >> 32);
}

constexpr int kSampleThreads = 256;
constexpr int kSampleItems = 16;  // per thread: at most 4096 sample keys
constexpr int kMaxSplit = 255;    // p <= 256 buckets

// Bucket of key k: the number of splitters smaller than k. s holds the p - 1
// splitters ascending followed by copies of the largest key value, 255 in
// all; eight halving steps over those 255 entries.
template <typename K>
__device__ __forceinline__ uint32_t bucket_of(const K* s, K k) {
  uint32_t pos = 0;
#pragma unroll
  for (uint32_t step = 128; step; step >>= 1)
    if (s[pos + step - 1] < k) pos += step;
  return pos;
}

// A key's bucket lies between the buckets of the smallest and the largest key
// with the same top kCellBits bits: cell[c] = lo | hi << 8 for cell c. The
// search then runs over [lo, hi] only, often a single splitter or none.
constexpr int kCellBits = 10;
constexpr int kCells = 1 << kCellBits;

template <typename K>
__device__ __forceinline__ uint32_t cell_of(K k) {
  return (uint32_t)(k >> (8 * sizeof(K) - kCellBits));
}

template <typename K>
__device__ __forceinline__ uint32_t bucket_in_cell(const K* s, const uint16_t* cell, K k) {
  const uint32_t e = cell[cell_of(k)];
  uint32_t lo = e & 0xffu, hi = e >> 8;  // s[lo - 1] < k <= s[hi] (where they exist)
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (s[mid] < k)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

template <typename K>
struct SplitDigit {
  const K* s;
  const uint16_t* cell;
  __device__ __forceinline__ uint32_t operator()(K k) const { return bucket_in_cell(s, cell, k); }
};

// The split round's digit rule: each key's bucket is searched once, right
// after the tile is loaded, and kept as a byte (four per register); the
// ranking records the bucket of every slot of the reordered tile in s_slot,
// which the write-out reads back.
template <typename K, int KPT>
struct CachedSplitDigit {
  const K* s;
  const uint16_t* cell;
  uint8_t* s_slot;  // [tile] bucket of each slot of the reordered tile
  uint32_t packed[(KPT + 3) / 4];
  __device__ __forceinline__ void prepare(const K (&key)[KPT]) {
#pragma unroll
    for (int i = 0; i < (KPT + 3) / 4; ++i) packed[i] = 0;
#pragma unroll
    for (int i = 0; i < KPT; ++i)
      packed[i >> 2] |= bucket_in_cell(s, cell, key[i]) << ((i & 3) * 8);
  }
  __device__ __forceinline__ uint32_t operator()(K k) const { return bucket_in_cell(s, cell, k); }
  __device__ __forceinline__ uint32_t of(K, int i) const {
    return (packed[i >> 2] >> ((i & 3) * 8)) & 0xffu;
  }
  __device__ __forceinline__ void keep(uint32_t pos, uint32_t d) const {
    s_slot[pos] = (uint8_t)d;
  }
  __device__ __forceinline__ uint32_t staged(K, int j) const { return s_slot[j]; }
};

template <typename K>
__global__ void __launch_bounds__(kSampleThreads)
    k_gvr_sample(const K* __restrict__ keys, int64_t n, int buckets, int oversample, uint64_t seed,
                 K* __restrict__ split, uint16_t* __restrict__ cell) {
  constexpr int Q = kSampleThreads, M = kSampleItems;
  __shared__ K sk[M * Q];
  __shared__ K s_split[kMaxSplit];
  const int t = threadIdx.x;
  const int ns = buckets * oversample - 1;  // sample size s*p - 1 <= 4095
  BtnItem<K, false> x[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int m = i * Q + t;
    x[i].k = m < ns ? keys[sample_pos(seed, (uint64_t)m, n)] : ~K(0);  // padding sorts last
  }
  btn_local_sort<false>(x);
  btn_network<false, K, M, Q>(x, t, sk, nullptr);
  // thread t holds sorted ranks [t*M, t*M + M); splitter j (1-based) = rank j*s - 1
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int r = t * M + i;
    if ((r + 1) % oversample == 0) {
      const int j = (r + 1) / oversample;
      if (j >= 1 && j <= buckets - 1) s_split[j - 1] = x[i].k;
    }
  }
  if (t < kMaxSplit && t >= buckets - 1) s_split[t] = ~K(0);
  __syncthreads();
  if (t < kMaxSplit) split[t] = s_split[t];
  // cell c holds the keys c << low .. ((c + 1) << low) - 1
  constexpr int LOW = 8 * sizeof(K) - kCellBits;
  for (int c = t; c < kCells; c += Q) {
    const K first = (K)c << LOW;
    const K last = first | (((K)1 << LOW) - 1);
    cell[c] = (uint16_t)(bucket_of(s_split, first) | (bucket_of(s_split, last) << 8));
  }
}

// Bucket counts: lane-private counter columns [bucket][lane] in shared memory
// (no bank conflicts within a warp), 16-byte loads.
template <typename K>
__global__ void __launch_bounds__(1024) k_gvr_hist(const K* __restrict__ keys, int64_t n,
                                                   const K* __restrict__ split,
                                                   const uint16_t* __restrict__ cell,
                                                   uint32_t* __restrict__ hist) {
  __shared__ K s_split[kMaxSplit];
  __shared__ uint16_t s_cell[kCells];
  __shared__ uint32_t s_cnt[256 * 32];
  for (int i = threadIdx.x; i < kMaxSplit; i += 1024) s_split[i] = split[i];
  for (int i = threadIdx.x; i < kCells; i += 1024) s_cell[i] = cell[i];
  for (int i = threadIdx.x; i < 256 * 32; i += 1024) s_cnt[i] = 0;
  __syncthreads();
  const SplitDigit<K> dig{s_split, s_cell};
  uint32_t* my = s_cnt + (threadIdx.x & 31);
  count_keys(keys, n, blockIdx.x * (int64_t)1024 + threadIdx.x, (int64_t)gridDim.x * 1024,
             [&](K k) { atomicAdd(&my[dig(k) * 32], 1u); });
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += 1024) {
    uint32_t sum = 0;
#pragma unroll 8
    for (int l = 0; l < 32; ++l) sum += s_cnt[b * 32 + ((l + b) & 31)];
    if (sum) atomicAdd(&hist[b], sum);
  }
}

// One CTA of 256 threads: thread b owns bucket b.
__global__ void __launch_bounds__(256) k_gvr_scan(const uint32_t* __restrict__ hist, int buckets,
                                                  int64_t n, uint32_t* __restrict__ base,
                                                  int64_t* __restrict__ offsets,
                                                  uint32_t* __restrict__ counts_out,
                                                  uint32_t* __restrict__ skip,
                                                  uint32_t* __restrict__ claim) {
  __shared__ uint32_t s_warp[8];
  const int b = threadIdx.x;
  const uint32_t c = b < buckets ? hist[b] : 0u;
  uint32_t tot;
  const uint32_t start = block_exclusive_scan<256>(c, s_warp, tot);
  base[b] = start;
  if (claim) claim[b] = 0;  // the keys-only split round's cursors
  if (b < buckets) {
    offsets[b] = start;
    if (counts_out) counts_out[b] = c;
  }
  if (b == 0) {
    offsets[buckets] = n;
    skip[0] = 0;  // the split round always runs (its output buffer is the next input)
  }
}

template <typename K, typename V, int THREADS, int KPT, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_gvr_split(PassParams p,
                                                             const K* __restrict__ split,
                                                             const uint16_t* __restrict__ cell) {
  using S = OnesweepShape<K, V, 8, THREADS, KPT>;
  using O = OrderedShape<K, V, 8, THREADS, KPT>;
  // keys only: the split round is the first round over the input, so the
  // order of keys within a bucket is free (onesweep_tile_first); with payloads
  // the ordered round (stable, checked)
  constexpr bool FIRST = !HasVal<V>::value;
  constexpr int R = S::R, WARPS = S::WARPS, TILE = S::TILE;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ K s_split[kMaxSplit];
  __shared__ uint16_t s_cell[kCells];
  uint32_t* s_wcnt = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_misc = FIRST ? s_wcnt + 2 * R : s_wcnt + WARPS * R + R;
  const int tid = threadIdx.x;
  for (int i = tid; i < kMaxSplit; i += THREADS) s_split[i] = split[i];
  for (int i = tid; i < kCells; i += THREADS) s_cell[i] = cell[i];
  if (tid == 0) s_misc[0] = atomicAdd(p.counter, 1u);  // tiles in launch order
  zero_words<THREADS>(s_wcnt, FIRST ? R : WARPS * R);
  __syncthreads();
  const uint32_t tile = s_misc[0];
  const int tile_n = (int)min((int64_t)TILE, p.n - (int64_t)tile * TILE);
  const K* kin = static_cast<const K*>(p.keys[0]);
  K* kout = static_cast<K*>(p.keys[1]);
  const V* vin = static_cast<const V*>(p.vals[0]);
  V* vout = static_cast<V*>(p.vals[1]);
  if (p.prefetch_tiles && tid == 0) {
    const int64_t pf = ((int64_t)tile + p.prefetch_tiles) * TILE;
    const int64_t cnt = min((int64_t)TILE, p.n - pf);
    prefetch_tile(kin, pf, cnt);
    if constexpr (HasVal<V>::value) prefetch_tile(vin, pf, cnt);
  }
  CachedSplitDigit<K, KPT> dig;
  dig.s = s_split;
  dig.cell = s_cell;
  const int64_t tile_base = (int64_t)tile * TILE;
  if constexpr (FIRST) {
    dig.s_slot = smem + FirstShape<K, 8, THREADS, KPT>::SMEM;
    if (tile_n == TILE)
      onesweep_tile_first<K, 8, THREADS, KPT, true>(p, tile, tile == 0, tile_base, tile_n, kin,
                                                    kout, p.base, (uint32_t)p.n, smem, dig,
                                                    p.claim);
    else
      onesweep_tile_first<K, 8, THREADS, KPT, false>(p, tile, tile == 0, tile_base, tile_n, kin,
                                                     kout, p.base, (uint32_t)p.n, smem, dig,
                                                     p.claim);
    return;
  }
  dig.s_slot = smem + O::SMEM;
  using DS = CachedSplitDigit<K, KPT>;
  if (tile_n == TILE)
    onesweep_tile_ordered<K, V, 8, THREADS, KPT, true, DS>(p, tile, tile == 0, tile_base, tile_n,
                                                           kin, kout, vin, vout, p.base,
                                                           (uint32_t)p.n, smem, dig);
  else
    onesweep_tile_ordered<K, V, 8, THREADS, KPT, false, DS>(p, tile, tile == 0, tile_base,
                                                            tile_n, kin, kout, vin, vout, p.base,
                                                            (uint32_t)p.n, smem, dig);
}

template <typename K, typename V, int THREADS, int KPT, int MINB>
cudaError_t gvr_launch(const GvrArgs& a, cudaStream_t st) {
  using S = OnesweepShape<K, V, 8, THREADS, KPT>;
  constexpr int R = S::R;
  const int64_t tiles = (a.n + S::TILE - 1) / S::TILE;
  cudaError_t e;
  if ((e = cudaMemsetAsync(a.hist, 0, sizeof(uint32_t) * R, st))) return e;
  if ((e = cudaMemsetAsync(a.counter, 0, sizeof(uint32_t), st))) return e;
  // keys only, the split round takes its ranges from cursors and needs no look-back words
  if (HasVal<V>::value &&
      (e = cudaMemsetAsync(a.status, 0, sizeof(uint32_t) * R * tiles, st)))
    return e;
  const K* keys = static_cast<const K*>(a.keys);
  K* split = static_cast<K*>(a.split);

  timer_begin(a.timer, "k_gvr_sample", st);
  uint16_t* cell = static_cast<uint16_t*>(a.cell);
  k_gvr_sample<K><<<1, kSampleThreads, 0, st>>>(keys, a.n, a.buckets, a.oversample, a.seed,
                                                split, cell);
  timer_end(a.timer, st);
  timer_begin(a.timer, "k_gvr_hist", st);
  const int64_t want = (a.n / 4 + 4095) / 4096;
  const int hblocks = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)a.num_sms);
  k_gvr_hist<K><<<hblocks, 1024, 0, st>>>(keys, a.n, split, cell, a.hist);
  timer_end(a.timer, st);
  timer_begin(a.timer, "k_gvr_scan", st);
  k_gvr_scan<<<1, 256, 0, st>>>(a.hist, a.buckets, a.n, a.base, a.offsets, a.counts_out, a.skip,
                                HasVal<V>::value ? nullptr : a.claim);
  timer_end(a.timer, st);

  PassParams pp;
  pp.keys[0] = const_cast<void*>(a.keys);
  pp.keys[1] = a.out_keys;
  pp.vals[0] = const_cast<void*>(a.vals);
  pp.vals[1] = a.out_vals;
  pp.n = a.n;
  pp.pass = 0;
  pp.shift = 0;
  pp.mask = 0xffu;
  pp.byte_sel = radix8_byte_sel(0);
  pp.low_shift = 0;
  pp.base = a.base;
  pp.skip = a.skip;
  pp.status = a.status;
  pp.status_next = nullptr;
  pp.counter = a.counter;
  pp.err = a.err;
  pp.spin_limit = a.spin_limit;
  pp.stall_tile = -1;
  pp.claim = HasVal<V>::value ? nullptr : a.claim;
  pp.prefetch_tiles = (int64_t)a.num_sms * 4;
  pp.check_mode = kCheckNormal;
  // keys only: the order-free round, in its own CTA shape (same tile)
  using FC = FirstCfg<K, THREADS, KPT, MINB>;
  constexpr bool HV = HasVal<V>::value;
  constexpr int CT = HV ? THREADS : FC::T, CK = HV ? KPT : FC::KP;
  auto kern = k_gvr_split<K, V, CT, CK, MINB>;
  // the round's layout, then one bucket byte per tile slot
  const size_t smem =
      (HV ? OrderedShape<K, V, 8, CT, CK>::SMEM : FirstShape<K, 8, CT, CK>::SMEM) + S::TILE;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return e;
  timer_begin(a.timer, "k_gvr_split", st);
  kern<<<(unsigned)tiles, CT, smem, st>>>(pp, split, cell);
  timer_end(a.timer, st);
  return cudaGetLastError();
}

}  // namespace

// Split-round shapes: the radix-256 defaults of each (key, payload) width.
int64_t gvr_tile(int key_bits, int val_bits) {
  if (key_bits == 32) return val_bits == 0 ? 256 * 32 : val_bits == 32 ? 256 * 20 : 256 * 16;
  return val_bits == 0 ? 256 * 20 : val_bits == 32 ? 256 * 16 : 256 * 12;
}

cudaError_t gvr_split_launch(int key_bits, int val_bits, const GvrArgs& a, cudaStream_t st) {
  if (key_bits == 32) {
    if (val_bits == 0) return gvr_launch<uint32_t, NoVal, 256, 32, 3>(a, st);
    if (val_bits == 32) return gvr_launch<uint32_t, uint32_t, 256, 20, 3>(a, st);
    return gvr_launch<uint32_t, uint64_t, 256, 16, 2>(a, st);
  }
  if (val_bits == 0) return gvr_launch<uint64_t, NoVal, 256, 20, 3>(a, st);
  if (val_bits == 32) return gvr_launch<uint64_t, uint32_t, 256, 16, 2>(a, st);
  return gvr_launch<uint64_t, uint64_t, 256, 12, 2>(a, st);
}

}  // namespace isort
