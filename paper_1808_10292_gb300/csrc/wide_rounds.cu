// Wide radixes: 65536 (the paper's PR2: 16-bit digits, two rounds on 32-bit
// keys, four on 64-bit keys) and 2048 (11-bit digits: 11, 11, 10 bits on
// 32-bit keys; 5 x 11 + 9 on 64-bit keys). Section "SR4, PR2, PR4, BTN and OET
// under MBSP", Eqs. Tp, Tp2.
//
// Each round is one count-sort round by a W-bit digit: the 2^W-bin digit
// histogram, its exclusive prefix (every key's destination = the prefix of its
// digit plus its rank among the earlier keys of that digit), and the routing of
// every key to its destination. Routing 2^W ways at once leaves each digit's
// run of a GPU tile at a fraction of a 32-byte sector, and the partly written
// sectors of every tile in flight overflow the L2 (a direct 65536-way scatter
// measured 9.5x DRAM read and write amplification; the 2048-way one 2.4x
// write amplification and one L2 write request per key). So routing takes two
// steps, each writing long runs, the high W - 8 bits of the digit first:
//
//   histogram of    radix 2048: k_hist_small, the 2048-bin histogram of the
//   the digit       round's digit (eight copies of the bins per CTA), then
//                   k_scan_wide. Radix 65536: the buckets are the digit's high
//                   byte, whose counts come from one k_hist read of all keys
//                   before round 0 (every byte's 256 bins), scanned by
//                   k_scan_high into step A's bases; the 65536 digit counts are
//                   taken after step A, when each bucket's keys sit together
//                   (k_bucket_hist: 256 lane-private bins per bucket slice),
//                   then k_scan_buckets (one CTA per bucket: the bucket's
//                   start from step A plus the prefix of its 256 counts).
//   k_scan_wide     radix 2048: exclusive prefix of the 2^W counts (base); per
//                   high part h (a "bucket", 2^(W-8) of them): its start
//                   base[h*256], its tiles, and whether its low byte is
//                   constant.
//   A: k_onesweep   an ordered round by the HIGH part over all keys (stable),
//                   which moves every key into its bucket (bases base[h*256]);
//                   in round 0 of a keys-only sort, whose input order carries
//                   nothing, the order-free k_onesweep_first (output ranges
//                   from per-bucket cursors, no look-back).
//   B: k_bucket     an ordered round by the LOW byte inside every bucket
//                   (stable; tiles never straddle a bucket) with bases
//                   base[h*256 + l]: every key lands at its digit's place.
// Step B of a bucket whose low byte is constant copies the bucket. Stability of
// both steps makes the round the stable count-sort by the W-bit digit.
#include "onesweep.cuh"

namespace isort {
namespace {

constexpr int kHistThreads = 1024;
constexpr int kMaxBuckets = 256;

__device__ __forceinline__ int parity_of(const uint32_t* skip, int pass) {
  int src = 0;
  for (int q = 0; q < pass; ++q) src ^= (skip[q] == 0);
  return src;
}

// Counts one key whose digit is d into bins (via add(bin, count)), combining
// the lanes whose digit equals that of the first active lane into one add
// (keys whose digit is nearly constant would otherwise serialise on one bin).
template <typename Add>
__device__ __forceinline__ void count_digit(uint32_t d, Add&& add) {
  const uint32_t m = __activemask();
  const uint32_t first = __ffs(m) - 1;
  const uint32_t d0 = __shfl_sync(m, d, first);
  const uint32_t same = __ballot_sync(m, d == d0);
  if (d != d0)
    add(d, 1u);
  else if ((threadIdx.x & 31) == first)
    add(d0, (uint32_t)__popc(same));
}

// The BINS-bin histogram (BINS <= 4096) of the digit (k >> shift) & mask:
// every CTA takes a chunk of the keys, warp w counting into copy w % 8 of the
// bins, and adds the copies' sums into hist.
template <typename K, int BINS>
__global__ void __launch_bounds__(kHistThreads)
    k_hist_small(const K* buf0, const K* buf1, const uint32_t* skip, int pass, int64_t n,
                 int shift, uint32_t mask, uint32_t* hist) {
  constexpr int COPIES = 8;
  extern __shared__ __align__(16) uint32_t s_bins[];  // [COPIES][BINS]
  for (int i = threadIdx.x; i < COPIES * BINS; i += kHistThreads) s_bins[i] = 0;
  __syncthreads();
  const K* keys = parity_of(skip, pass) ? buf1 : buf0;
  const int64_t lo = n * blockIdx.x / gridDim.x, hi = n * (blockIdx.x + 1) / gridDim.x;
  uint32_t* my = s_bins + ((threadIdx.x >> 5) % COPIES) * BINS;
  count_keys(keys + lo, hi - lo, threadIdx.x, kHistThreads, [&](K k) {
    count_digit(digit_of(k, shift, mask), [&](uint32_t d, uint32_t c) { atomicAdd(&my[d], c); });
  });
  __syncthreads();
  for (int d = threadIdx.x; d < BINS; d += kHistThreads) {
    uint32_t sum = 0;
#pragma unroll
    for (int c = 0; c < COPIES; ++c) sum += s_bins[c * BINS + d];
    if (sum) atomicAdd(&hist[d], sum);
  }
}

// Radix 65536, per round before step A: the 256 buckets are the values of the
// digit's high byte, whose counts come from one read of all keys before round
// 0 (hist8: one 256-bin histogram per byte, k_hist). Exclusive prefix of the
// row -> baseA (step A's bases), the buckets' first tiles for step B, skip[passA]
// (the high byte is constant: step A is the identity), skip[passA + 1] = 1
// (step B is needed: cleared by k_scan_buckets once a bucket's low byte is
// seen to vary), and step A's cursors zeroed when it runs order-free (claimA,
// or null).
template <int TILE>
__global__ void __launch_bounds__(256) k_scan_high(const uint32_t* __restrict__ row, int64_t n,
                                                   uint32_t* __restrict__ baseA,
                                                   uint32_t* __restrict__ tile_first,
                                                   uint32_t* __restrict__ skip, int passA,
                                                   uint32_t* __restrict__ claimA) {
  __shared__ uint32_t s_warp[8];
  const int h = threadIdx.x;
  const uint32_t c = row[h];
  uint32_t total;
  baseA[h] = block_exclusive_scan<256>(c, s_warp, total);
  const int trivial = __syncthreads_or((int64_t)c == n);
  const uint32_t tiles = (c + TILE - 1) / TILE;
  __syncthreads();  // s_warp is reused
  const uint32_t first = block_exclusive_scan<256>(tiles, s_warp, total);
  tile_first[h] = first;
  if (h == 255) tile_first[256] = first + tiles;
  if (claimA) claimA[h] = 0;
  if (h == 0) {
    skip[passA] = trivial;
    skip[passA + 1] = 1;
  }
}

// Radix 65536, per round after step A: the keys of bucket h (high byte) sit
// together at [baseA[h], baseA[h + 1]); count the low byte of every key into
// hist[h*256 + l]. CTA c takes the slice [n*c/C, n*(c+1)/C) and counts each
// bucket's part of it in lane-private columns (lane l of every warp counts
// into column l: no bank conflicts), adding the 256 sums to hist when it
// leaves the bucket. One read of the keys with conflict-free shared atomics,
// in place of a 65536-bin histogram.
constexpr int kBucketHistThreads = 1024;
template <typename K>
__global__ void __launch_bounds__(kBucketHistThreads, 2)
    k_bucket_hist(const K* buf0, const K* buf1, const uint32_t* skip, int passB, int64_t n,
                  int shift, const uint32_t* __restrict__ baseA, uint32_t* __restrict__ hist) {
  __shared__ __align__(16) uint32_t s_cnt[256 * 32];  // [low byte][lane]
  __shared__ uint32_t s_start[257];
  const int t = threadIdx.x, lane = t & 31;
  const K* keys = parity_of(skip, passB) ? buf1 : buf0;
  for (int h = t; h < 256; h += kBucketHistThreads) s_start[h] = baseA[h];
  if (t == 0) s_start[256] = (uint32_t)n;
  const int64_t hi = n * (blockIdx.x + 1) / gridDim.x;
  int64_t lo = n * blockIdx.x / gridDim.x;
  __syncthreads();
  int b = 0;  // the bucket holding key lo: the last h with s_start[h] <= lo
  for (int step = 128; step; step >>= 1)
    if ((int64_t)s_start[b + step] <= lo) b += step;
  while (lo < hi) {
    while ((int64_t)s_start[b + 1] <= lo) ++b;  // skip empty buckets
    const int64_t end = min(hi, (int64_t)s_start[b + 1]);
    for (int i = t; i < 256 * 32 / 4; i += kBucketHistThreads)
      reinterpret_cast<uint4*>(s_cnt)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    count_keys(keys + lo, end - lo, t, kBucketHistThreads,
               [&](K k) { atomicAdd(&s_cnt[digit_of(k, shift, 0xffu) * 32 + lane], 1u); });
    __syncthreads();
    if (t < 256) {
      uint32_t sum = 0;
#pragma unroll 8
      for (int j = 0; j < 32; ++j) sum += s_cnt[t * 32 + ((j + t) & 31)];
      if (sum) atomicAdd(&hist[b * 256 + t], sum);
    }
    __syncthreads();
    lo = end;
  }
}

// Radix 65536, per round after k_bucket_hist: CTA h scans bucket h's 256
// low-byte counts, so that base[h*256 + l] = baseA[h] + (the bucket's keys
// with a smaller low byte); bucket_trivial[h] = one low byte holds all of the
// bucket's keys, and a bucket whose low byte varies clears skip[passB]
// (preset to 1 by k_scan_high). With claim (keys only, round 0), the bucket's
// 256 cursors of the order-free step B are zeroed. The buckets' bases are
// known from step A, so the 256 scans are independent: one CTA per bucket.
__global__ void __launch_bounds__(256) k_scan_buckets(const uint32_t* __restrict__ hist,
                                                      const uint32_t* __restrict__ baseA,
                                                      uint32_t* __restrict__ base,
                                                      uint32_t* __restrict__ bucket_trivial,
                                                      uint32_t* __restrict__ skip, int passB,
                                                      uint32_t* __restrict__ claim) {
  __shared__ uint32_t s_warp[8];
  const int h = blockIdx.x, l = threadIdx.x;
  const uint32_t c = hist[h * 256 + l];
  uint32_t len;
  const uint32_t excl = block_exclusive_scan<256>(c, s_warp, len);
  base[h * 256 + l] = baseA[h] + excl;
  if (claim) claim[h * 256 + l] = 0;
  const int one = __syncthreads_or(len > 0 && c == len);
  if (l == 0) {
    bucket_trivial[h] = one;
    if (len > 0 && !one) skip[passB] = 0;
  }
}

// Per round (BINS = 2^W bins, NB = BINS / 256 buckets): base = exclusive prefix
// of hist; per bucket h: baseA[h] = base[h*256] (the bases of step A), its
// first tile among step B's tiles (tile_first[0..NB], tiles of TILE keys) and
// bucket_trivial[h] (one low byte holds all of the bucket's keys); skip[passA]
// (one bucket holds all n keys) and skip[passA + 1] (every bucket is trivial).
// One CTA of 1024 threads.
template <int BINS, int TILE>
__global__ void __launch_bounds__(1024) k_scan_wide(const uint32_t* __restrict__ hist,
                                                    uint32_t* __restrict__ base,
                                                    uint32_t* __restrict__ baseA,
                                                    uint32_t* __restrict__ tile_first,
                                                    uint32_t* __restrict__ bucket_trivial,
                                                    uint32_t* __restrict__ skip, int passA,
                                                    int64_t n, uint32_t* __restrict__ claim) {
  constexpr int PER = BINS / 1024 > 0 ? BINS / 1024 : 1;  // digits per thread
  constexpr int NB = BINS / 256;
  static_assert(BINS >= 256 && BINS % 256 == 0 && NB <= kMaxBuckets, "buckets of 256 digits");
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_len[NB];
  __shared__ uint32_t s_flags[2];
  const int t = threadIdx.x;
  if (t < 2) s_flags[t] = 0;
  // keys only, round 0: the cursors of the order-free steps, claim[0, BINS)
  // for step B's digits and claim[BINS, BINS + 256) for step A's buckets
  if (claim)
    for (int j = t; j < BINS + 256; j += 1024) claim[j] = 0;
  // thread t owns digits [t*PER, t*PER + PER): their sum and largest count,
  // then their exclusive prefixes (16-byte loads and stores where PER allows)
  uint32_t local = 0, mx = 0;
  if (t * PER < BINS) {
    if constexpr (PER % 4 == 0) {
      const uint4* h4 = reinterpret_cast<const uint4*>(hist + t * PER);
#pragma unroll 4
      for (int j = 0; j < PER / 4; ++j) {
        const uint4 v = h4[j];
        local += v.x + v.y + v.z + v.w;
        mx = max(max(mx, max(v.x, v.y)), max(v.z, v.w));
      }
    } else {
      for (int j = 0; j < PER; ++j) {
        const uint32_t c = hist[t * PER + j];
        local += c;
        mx = max(mx, c);
      }
    }
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan<1024>(local, s_warp, total);
  const uint32_t my_start = run;  // base of this thread's first digit
  if (t * PER < BINS) {
    if constexpr (PER % 4 == 0) {
      const uint4* h4 = reinterpret_cast<const uint4*>(hist + t * PER);
      uint4* b4 = reinterpret_cast<uint4*>(base + t * PER);
#pragma unroll 4
      for (int j = 0; j < PER / 4; ++j) {
        const uint4 v = h4[j];
        uint4 o;
        o.x = run;
        o.y = o.x + v.x;
        o.z = o.y + v.y;
        o.w = o.z + v.z;
        run = o.w + v.w;
        b4[j] = o;
      }
    } else {
      for (int j = 0; j < PER; ++j) {
        base[t * PER + j] = run;
        run += hist[t * PER + j];
      }
    }
  }
  // per bucket (256 digits = TPB threads): start, length, largest digit count
  constexpr int TPB = 256 / PER;
  uint32_t blen = local, bmax = mx;
#pragma unroll
  for (int o = 1; o < TPB && o < 32; o <<= 1) {
    blen += __shfl_xor_sync(kFullMask, blen, o);
    bmax = max(bmax, __shfl_xor_sync(kFullMask, bmax, o));
  }
  if constexpr (TPB > 32) {  // buckets wider than a warp: combine the warps' results
    __shared__ uint32_t s_part[2][32];
    if ((t & 31) == 0) {
      s_part[0][t >> 5] = blen;
      s_part[1][t >> 5] = bmax;
    }
    __syncthreads();
    if (t % TPB == 0) {
      blen = 0, bmax = 0;
      for (int w = 0; w < TPB / 32; ++w) {
        blen += s_part[0][t / 32 + w];
        bmax = max(bmax, s_part[1][t / 32 + w]);
      }
    }
  }
  if (t % TPB == 0 && t * PER < BINS) {
    const int h = t / TPB;
    s_len[h] = blen;
    baseA[h] = my_start;  // the bucket's first digit is this thread's first
    bucket_trivial[h] = blen > 0 && bmax == blen;
    if ((int64_t)blen == n) s_flags[0] = 1;      // step A is the identity
    if (blen > 0 && bmax != blen) s_flags[1] = 1;  // some bucket needs step B
  }
  __syncthreads();
  if (t < 32) {  // tiles per bucket and their exclusive prefix
    constexpr int BPL = (NB + 31) / 32;  // buckets per lane
    uint32_t tiles[BPL], sum = 0;
#pragma unroll
    for (int j = 0; j < BPL; ++j) {
      const int h = t * BPL + j;
      tiles[j] = h < NB ? (s_len[h] + TILE - 1) / TILE : 0u;
      sum += tiles[j];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFullMask, incl, o);
      if (t >= o) incl += y;
    }
    uint32_t first = incl - sum;
#pragma unroll
    for (int j = 0; j < BPL; ++j) {
      const int h = t * BPL + j;
      if (h < NB) tile_first[h] = first;
      first += tiles[j];
    }
    if (t == 31) tile_first[NB] = first;
  }
  if (t == 0) {
    skip[passA] = s_flags[0];
    skip[passA + 1] = s_flags[1] ? 0u : 1u;
  }
}

// Step B: an ordered radix-256 round by the low byte (bits [p.shift, p.shift
// + 8)) inside every bucket. Tile ids come in launch order; tile t belongs to
// the bucket h with tile_first[h] <= t < tile_first[h + 1], and the look-back
// never leaves the bucket (its first tile publishes inclusive counts).
// Positions are absolute: the digit bases are base[h*256 + l].
template <typename K, typename V, int THREADS, int KPT, int MINB, int NB, typename DS>
__global__ void __launch_bounds__(THREADS, MINB)
    k_bucket(PassParams p, const uint32_t* __restrict__ base,
             const uint32_t* __restrict__ tile_first,
             const uint32_t* __restrict__ bucket_trivial) {
  using S = OnesweepShape<K, V, 8, THREADS, KPT>;
  constexpr int R = S::R, WARPS = S::WARPS, TILE = S::TILE;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_wcnt = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_misc = s_wcnt + WARPS * R + R;
  const int tid = threadIdx.x;
  if (p.skip[p.pass]) return;  // every bucket's low byte is constant: identity
  const int src = parity_of(p.skip, p.pass);
  if (tid == 0) s_misc[0] = atomicAdd(p.counter, 1u);
  zero_words<THREADS>(s_wcnt, WARPS * R);
  __syncthreads();
  const uint32_t tile = s_misc[0];
  if (tile >= tile_first[NB]) return;  // more CTAs than tiles
  int lo = 0, hi = NB - 1;  // the last bucket whose first tile is <= tile
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_first[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  const int h = lo;
  const int64_t start = base[h * 256];
  const int64_t end = h + 1 < NB ? (int64_t)base[(h + 1) * 256] : p.n;
  const int64_t lt = (int64_t)tile - tile_first[h];
  const int64_t tile_base = start + lt * TILE;
  const int tile_n = (int)min((int64_t)TILE, end - tile_base);
  const K* kin = static_cast<const K*>(src ? p.keys[1] : p.keys[0]);
  K* kout = static_cast<K*>(src ? p.keys[0] : p.keys[1]);
  const V* vin = static_cast<const V*>(src ? p.vals[1] : p.vals[0]);
  V* vout = static_cast<V*>(src ? p.vals[0] : p.vals[1]);
  if (bucket_trivial[h]) {  // the bucket's low byte is constant: it stays in order
    for (int j = tid; j < tile_n; j += THREADS) {
      kout[tile_base + j] = kin[tile_base + j];
      if constexpr (HasVal<V>::value) vout[tile_base + j] = vin[tile_base + j];
    }
    return;
  }
  DS dig{p};
  if (tile_n == TILE)
    onesweep_tile_ordered<K, V, 8, THREADS, KPT, true, DS>(p, tile, lt == 0, tile_base, tile_n,
                                                           kin, kout, vin, vout, base + h * 256,
                                                           (uint32_t)p.n, smem, dig);
  else
    onesweep_tile_ordered<K, V, 8, THREADS, KPT, false, DS>(p, tile, lt == 0, tile_base, tile_n,
                                                            kin, kout, vin, vout, base + h * 256,
                                                            (uint32_t)p.n, smem, dig);
}

// Step B of round 0 of a keys-only sort (order-free, as step A there): the
// tiles of bucket h take their digits' ranges from the cursors claim[h*256 +
// l] (zeroed by k_scan_buckets, or k_scan_wide at radix 2048) instead of
// looking back; CTA shape of the order-free round (THREADS x KPT, the same
// tile as the ordered step).
template <typename K, int THREADS, int KPT, int MINB, int NB, typename DS>
__global__ void __launch_bounds__(THREADS, MINB)
    k_bucket_first(PassParams p, const uint32_t* __restrict__ base,
                   const uint32_t* __restrict__ tile_first,
                   const uint32_t* __restrict__ bucket_trivial) {
  using S = OnesweepShape<K, NoVal, 8, THREADS, KPT>;
  constexpr int R = S::R, TILE = S::TILE;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_slot = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_misc = s_slot + 2 * R;
  const int tid = threadIdx.x;
  if (p.skip[p.pass]) return;
  const int src = parity_of(p.skip, p.pass);
  if (tid == 0) s_misc[0] = atomicAdd(p.counter, 1u);
  zero_words<THREADS>(s_slot, R);
  __syncthreads();
  const uint32_t tile = s_misc[0];
  if (tile >= tile_first[NB]) return;  // more CTAs than tiles
  int lo = 0, hi = NB - 1;  // the last bucket whose first tile is <= tile
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_first[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  const int h = lo;
  const int64_t start = base[h * 256];
  const int64_t end = h + 1 < NB ? (int64_t)base[(h + 1) * 256] : p.n;
  const int64_t lt = (int64_t)tile - tile_first[h];
  const int64_t tile_base = start + lt * TILE;
  const int tile_n = (int)min((int64_t)TILE, end - tile_base);
  const K* kin = static_cast<const K*>(src ? p.keys[1] : p.keys[0]);
  K* kout = static_cast<K*>(src ? p.keys[0] : p.keys[1]);
  if (bucket_trivial[h]) {  // the bucket's low byte is constant: copy it
    for (int j = tid; j < tile_n; j += THREADS) kout[tile_base + j] = kin[tile_base + j];
    return;
  }
  DS dig{p};
  uint32_t* claim = p.claim + h * 256;
  if (tile_n == TILE)
    onesweep_tile_first<K, 8, THREADS, KPT, true, DS>(p, tile, lt == 0, tile_base, tile_n, kin,
                                                      kout, base + h * 256, (uint32_t)p.n, smem,
                                                      dig, claim);
  else
    onesweep_tile_first<K, 8, THREADS, KPT, false, DS>(p, tile, lt == 0, tile_base, tile_n, kin,
                                                       kout, base + h * 256, (uint32_t)p.n, smem,
                                                       dig, claim);
}

// Scratch of the rounds inside the workspace: hist holds the 2^W counts, then
// baseA[256], tile_first[257] (padded to 512) and bucket_trivial[256]; base
// holds the prefix; status[0] the look-back rows of step A, status[1] those of
// step B.
struct WideScratch {
  uint32_t *hist, *baseA, *tile_first, *bucket_trivial, *base;
  uint32_t* hist8;  // radix 65536: the 256-bin histogram of every key byte (k_hist)
};

// One round with a W-bit digit at `shift` (kernel passes 2q and 2q + 1).
// Byte-aligned digit parts (W = 16) use the byte-permute digit rule.
template <typename K, typename V, int THREADS, int KPT, int MINB, int W>
cudaError_t wide_round(const LsdArgs& a, PassParams& pp, const WideScratch& w, int q, int shift,
                       int64_t tiles, cudaStream_t st) {
  constexpr int BINS = 1 << W, NB = BINS / 256, TILE = THREADS * KPT;
  constexpr bool BYTES = W == 16;
  using DS = typename std::conditional<BYTES, RadixDigit, ShiftMaskDigit>::type;
  cudaError_t e;
  // keys only, round 0: both steps are order-free and take their ranges from
  // cursors instead of looking back
  const bool free0 = !HasVal<V>::value && q == 0;
  if ((e = cudaMemsetAsync(w.hist, 0, sizeof(uint32_t) * BINS, st))) return e;
  if constexpr (W == 16) {
    // step A's bases and step B's bucket tiles from the high byte's histogram;
    // the 65536 digit counts are taken after step A (k_bucket_hist)
    timer_begin(a.timer, "k_scan_high", st);
    k_scan_high<TILE><<<1, 256, 0, st>>>(w.hist8 + (size_t)(2 * q + 1) * 256, a.n, w.baseA,
                                         w.tile_first, a.skip, 2 * q,
                                         free0 ? a.claim + BINS : nullptr);
    timer_end(a.timer, st);
  } else {
    constexpr size_t HSMEM = sizeof(uint32_t) * 8 * BINS;
    if ((e = cudaFuncSetAttribute(k_hist_small<K, BINS>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HSMEM)))
      return e;
    timer_begin(a.timer, "k_hist_wide", st);
    k_hist_small<K, BINS><<<a.num_sms * (HSMEM <= 64 * 1024 ? 2 : 1), kHistThreads, HSMEM, st>>>(
        static_cast<const K*>(a.keys), static_cast<const K*>(a.alt_keys), a.skip, 2 * q, a.n,
        shift, (uint32_t)(BINS - 1), w.hist);
    timer_end(a.timer, st);
    timer_begin(a.timer, "k_scan_wide", st);
    k_scan_wide<BINS, TILE><<<1, 1024, 0, st>>>(w.hist, w.base, w.baseA, w.tile_first,
                                                w.bucket_trivial, a.skip, 2 * q, a.n,
                                                free0 ? a.claim : nullptr);
    timer_end(a.timer, st);
  }
  if (!free0 && (e = cudaMemsetAsync(a.status[0], 0, sizeof(uint32_t) * 256 * tiles, st)))
    return e;
  if (!free0 && (e = cudaMemsetAsync(a.status[1], 0, sizeof(uint32_t) * 256 * (tiles + NB), st)))
    return e;
  constexpr size_t smem = OrderedShape<K, V, 8, THREADS, KPT>::SMEM;
  auto kA = k_onesweep<K, V, 8, THREADS, KPT, MINB, DS>;
  auto kB = k_bucket<K, V, THREADS, KPT, MINB, NB, DS>;
  if (smem > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(kA, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
      return e;
    if ((e = cudaFuncSetAttribute(kB, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
      return e;
  }
  // step A: the high W - 8 bits, over all keys (the input is sorted by bits [0, shift))
  pp.pass = 2 * q;
  pp.shift = shift + 8;
  pp.mask = (uint32_t)(NB - 1);
  pp.byte_sel = radix8_byte_sel(shift + 8);
  pp.low_shift = shift;
  pp.base = w.baseA;
  pp.status = a.status[0];
  pp.counter = a.counters + 2 * q;
  timer_begin(a.timer, "k_wide_high", st);
  bool launched = false;
  if constexpr (!HasVal<V>::value) {
    if (free0) {
      using FC = FirstCfg<K, THREADS, KPT, MINB>;  // the order-free round's CTA shape, same tile
      constexpr size_t fsmem = FirstShape<K, 8, FC::T, FC::KP>::SMEM;
      auto kF = k_onesweep_first<K, 8, FC::T, FC::KP, MINB, DS>;
      if (fsmem > 48 * 1024 && (e = cudaFuncSetAttribute(
                                    kF, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem)))
        return e;
      pp.claim = a.claim + BINS;
      kF<<<(unsigned)tiles, FC::T, fsmem, st>>>(pp);
      pp.claim = nullptr;
      launched = true;
    }
  }
  if (!launched) kA<<<(unsigned)tiles, THREADS, smem, st>>>(pp);
  timer_end(a.timer, st);
  if constexpr (W == 16) {
    // the low byte's counts per bucket, from step A's output, then the prefix
    timer_begin(a.timer, "k_bucket_hist", st);
    k_bucket_hist<K><<<a.num_sms * 2, kBucketHistThreads, 0, st>>>(
        static_cast<const K*>(a.keys), static_cast<const K*>(a.alt_keys), a.skip, 2 * q + 1, a.n,
        shift, w.baseA, w.hist);
    timer_end(a.timer, st);
    timer_begin(a.timer, "k_scan_buckets", st);
    k_scan_buckets<<<NB, 256, 0, st>>>(w.hist, w.baseA, w.base, w.bucket_trivial, a.skip,
                                       2 * q + 1, free0 ? a.claim : nullptr);
    timer_end(a.timer, st);
  }
  // step B: the low byte, inside every bucket
  pp.pass = 2 * q + 1;
  pp.shift = shift;
  pp.mask = 0xffu;
  pp.byte_sel = radix8_byte_sel(shift);
  pp.low_shift = shift;
  pp.base = nullptr;
  pp.status = a.status[1];
  pp.counter = a.counters + 2 * q + 1;
  timer_begin(a.timer, "k_wide_low", st);
  launched = false;
  if constexpr (!HasVal<V>::value) {
    if (free0) {  // round 0, keys only: order-free inside the buckets too
      using FC = FirstCfg<K, THREADS, KPT, MINB>;
      constexpr size_t fsmem = FirstShape<K, 8, FC::T, FC::KP>::SMEM;
      auto kFB = k_bucket_first<K, FC::T, FC::KP, MINB, NB, DS>;
      if (fsmem > 48 * 1024 && (e = cudaFuncSetAttribute(
                                    kFB, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem)))
        return e;
      pp.claim = a.claim;
      kFB<<<(unsigned)(tiles + NB), FC::T, fsmem, st>>>(pp, w.base, w.tile_first,
                                                       w.bucket_trivial);
      pp.claim = nullptr;
      launched = true;
    }
  }
  if (!launched)
    kB<<<(unsigned)(tiles + NB), THREADS, smem, st>>>(pp, w.base, w.tile_first, w.bucket_trivial);
  timer_end(a.timer, st);
  return cudaSuccess;
}

}  // namespace

// One whole sort at radix 2^BITS (BITS = 16 or 11): round q takes the digit of
// width W = min(BITS, key bits - BITS*q) at shift BITS*q; kernel passes 2q
// (step A) and 2q + 1 (step B) share the skip and tile-counter arrays, so the
// buffer parity follows the executed passes.
template <typename K, typename V, int BITS, int THREADS, int KPT, int MINB>
cudaError_t wide_launch(const LsdArgs& a, cudaStream_t st) {
  constexpr int KB = 8 * (int)sizeof(K), ROUNDS = (KB + BITS - 1) / BITS, P2 = 2 * ROUNDS;
  constexpr int TILE = THREADS * KPT;
  const int64_t tiles = (a.n + TILE - 1) / TILE;
  WideScratch w;
  w.hist = a.hist;
  w.baseA = a.hist + (1 << BITS);
  w.tile_first = w.baseA + 256;
  w.bucket_trivial = w.tile_first + 512;
  w.hist8 = w.bucket_trivial + 256;
  w.base = a.base;
  cudaError_t e;
  if ((e = cudaMemsetAsync(a.counters, 0, sizeof(uint32_t) * P2, st))) return e;
  if constexpr (BITS == 16) {
    // the 256-bin histogram of every key byte, one read of the input: the
    // buckets (high bytes of the digits) of every round
    constexpr int P8 = KB / 8;
    constexpr int LANES = sizeof(K) == 4 ? 32 : 16;
    using HS = HistShape<K, 8, kHistThreads, LANES>;
    if ((e = cudaMemsetAsync(w.hist8, 0, sizeof(uint32_t) * P8 * 256, st))) return e;
    auto hk = k_hist<K, 8, kHistThreads, LANES>;
    if ((e = cudaFuncSetAttribute(hk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)HS::SMEM)))
      return e;
    const int64_t want = (a.n / Vec16<K>::N + kHistThreads * 4 - 1) / (kHistThreads * 4);
    const int hblocks = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)a.num_sms);
    timer_begin(a.timer, "k_hist", st);
    hk<<<hblocks, kHistThreads, HS::SMEM, st>>>(static_cast<const K*>(a.keys), a.n, w.hist8);
    timer_end(a.timer, st);
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
  pp.stall_tile = -1;
  pp.claim = nullptr;
  pp.prefetch_tiles = a.prefetch_tiles;
  pp.check_mode = a.check_mode;
  pp.status_next = nullptr;
  for (int q = 0; q < ROUNDS; ++q) {
    const int shift = BITS * q;
    const int width = KB - shift < BITS ? KB - shift : BITS;
    switch (width) {
      case 16: e = wide_round<K, V, THREADS, KPT, MINB, 16>(a, pp, w, q, shift, tiles, st); break;
      case 11: e = wide_round<K, V, THREADS, KPT, MINB, 11>(a, pp, w, q, shift, tiles, st); break;
      case 10: e = wide_round<K, V, THREADS, KPT, MINB, 10>(a, pp, w, q, shift, tiles, st); break;
      case 9: e = wide_round<K, V, THREADS, KPT, MINB, 9>(a, pp, w, q, shift, tiles, st); break;
      default: return cudaErrorInvalidValue;
    }
    if (e) return e;
  }
  const int cblocks = (int)std::min<int64_t>((a.n + 255) / 256, (int64_t)a.num_sms * 8);
  timer_begin(a.timer, "k_copy_back", st);
  k_copy_back<K, V><<<cblocks, 256, 0, st>>>(a.skip, P2, static_cast<K*>(a.keys),
                                             static_cast<const K*>(a.alt_keys),
                                             static_cast<V*>(a.vals),
                                             static_cast<const V*>(a.alt_vals), a.n);
  timer_end(a.timer, st);
  return cudaGetLastError();
}

template <typename K, typename V, int BITS, int THREADS, int KPT, int MINB>
constexpr LsdEntry wide_entry() {
  constexpr int KB = 8 * (int)sizeof(K);
  LsdEntry e{KB,
             HasVal<V>::value ? (int)(8 * sizeof(V)) : 0,
             BITS,
             THREADS,
             KPT,
             (int64_t)THREADS * KPT,
             1 << BITS,                     // hist and base: 2^BITS words per kernel pass
             2 * ((KB + BITS - 1) / BITS),  // kernel passes: two steps per round
             256,                           // look-back words per tile
             2,
             &wide_launch<K, V, BITS, THREADS, KPT, MINB>};
  e.extra_status_rows = kMaxBuckets;  // step B: at most one partial tile per bucket
  return e;
}

// Shapes of the radix-256 defaults for each (key, payload) width.
#define ISORT_WIDE_TABLES(B)                                                              \
  static const LsdEntry kW##B##None32[] = {wide_entry<uint32_t, NoVal, B, 256, 32, 3>()};   \
  static const LsdEntry kW##B##V32_32[] = {wide_entry<uint32_t, uint32_t, B, 256, 20, 3>()}; \
  static const LsdEntry kW##B##V64_32[] = {wide_entry<uint32_t, uint64_t, B, 256, 16, 2>()}; \
  static const LsdEntry kW##B##None64[] = {wide_entry<uint64_t, NoVal, B, 256, 20, 3>()};   \
  static const LsdEntry kW##B##V32_64[] = {wide_entry<uint64_t, uint32_t, B, 256, 16, 2>()}; \
  static const LsdEntry kW##B##V64_64[] = {wide_entry<uint64_t, uint64_t, B, 256, 12, 2>()};
ISORT_WIDE_TABLES(16)
ISORT_WIDE_TABLES(11)
#undef ISORT_WIDE_TABLES

int wide_variants(int key_bits, int val_bits, int radix_bits, const LsdEntry** out) {
  if (key_bits != 32 && key_bits != 64) return 0;
  if (val_bits != 0 && val_bits != 32 && val_bits != 64) return 0;
  const int ki = key_bits == 32 ? 0 : 1, vi = val_bits == 0 ? 0 : val_bits == 32 ? 1 : 2;
  const LsdEntry* t16[2][3] = {{kW16None32, kW16V32_32, kW16V64_32},
                               {kW16None64, kW16V32_64, kW16V64_64}};
  const LsdEntry* t11[2][3] = {{kW11None32, kW11V32_32, kW11V64_32},
                               {kW11None64, kW11V32_64, kW11V64_64}};
  if (radix_bits == 16)
    *out = t16[ki][vi];
  else if (radix_bits == 11)
    *out = t11[ki][vi];
  else
    return 0;
  return 1;
}

}  // namespace isort
