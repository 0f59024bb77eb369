// Radix 65536: the paper's PR2 (16-bit digits; two rounds on 32-bit keys,
// four on 64-bit keys), Section "SR4, PR2, PR4, BTN and OET under MBSP",
// Eqs. Tp, Tp2.
//
// Each round is one count-sort round by a 16-bit digit: the 65536-bin digit
// histogram, its exclusive prefix (every key's destination = the prefix of its
// digit plus its rank among the earlier keys of that digit), and the routing of
// every key to its destination. Routing 65536 ways at once leaves each digit's
// run of a GPU tile at a fraction of a 32-byte sector, and the partly written
// sectors of every tile in flight (tiles x 65536 x 32 B) overflow the L2: a
// direct scatter measured 9.5x DRAM write amplification. So the routing is
// done in two steps that both write long runs, the high byte of the digit
// first (most significant first inside the digit):
//
//   k_hist16        the 65536-bin histogram of the round's digit, one read of
//                   the keys from DRAM (pairs of CTAs share a chunk, each
//                   counting half of the bins in shared memory).
//   k_scan16        exclusive prefix of the 65536 counts (base16), per high
//                   byte h: the bucket [base16[h*256], base16[h*256+256]), its
//                   tiles, and whether its low byte is constant.
//   A: k_onesweep   an ordered radix-256 round by the HIGH byte over all keys
//                   (stable), which moves every key into its bucket; the
//                   bucket's start is base16[h*256].
//   B: k_bucket16   an ordered radix-256 round by the LOW byte inside every
//                   bucket (stable; tiles never straddle a bucket), whose
//                   digit bases are base16[h*256 + l]: every key lands at its
//                   16-bit digit's destination.
// Step B of a bucket whose low byte is constant copies the bucket. Stability of
// both steps makes the round the stable count-sort by the 16-bit digit.
#include "onesweep.cuh"

namespace isort {
namespace {

constexpr int kR16 = 65536;
constexpr int kHalf16 = kR16 / 2;
constexpr int kHistThreads = 1024;

template <typename K>
__device__ __forceinline__ uint32_t digit16(K k, int shift) {
  return static_cast<uint32_t>(k >> shift) & 0xffffu;
}

__device__ __forceinline__ int parity_of(const uint32_t* skip, int pass) {
  int src = 0;
  for (int q = 0; q < pass; ++q) src ^= (skip[q] == 0);
  return src;
}

// The 65536-bin histogram of digit16(key, shift) of all n keys of the round's
// input buffer (the parity of the passes executed before `pass`), added into
// hist. CTAs 2c and 2c+1 read the same chunk c of the keys (the second read
// mostly hits L2); CTA 2c + r counts only the digits of bin half r, in its own
// shared memory (32768 counters, 128 KiB). Lanes whose digit equals that of
// the first active lane are counted with one add (keys whose digit is nearly
// constant would otherwise serialise on one counter).
template <typename K>
__global__ void __launch_bounds__(kHistThreads)
    k_hist16(const K* buf0, const K* buf1, const uint32_t* skip, int pass, int64_t n, int shift,
             uint32_t* hist) {
  extern __shared__ __align__(16) uint32_t s_bins[];  // kHalf16
  const uint32_t rank = blockIdx.x & 1u;
  for (int i = threadIdx.x; i < kHalf16; i += kHistThreads) s_bins[i] = 0;
  __syncthreads();
  const K* keys = parity_of(skip, pass) ? buf1 : buf0;
  const int64_t chunks = gridDim.x >> 1, chunk = blockIdx.x >> 1;
  const int64_t lo = n * chunk / chunks, hi = n * (chunk + 1) / chunks;
  const uint32_t lane = threadIdx.x & 31;
  count_keys(keys + lo, hi - lo, threadIdx.x, kHistThreads, [&](K k) {
    const uint32_t d = digit16(k, shift);
    const uint32_t m = __activemask();
    const uint32_t first = __ffs(m) - 1;
    const uint32_t d0 = __shfl_sync(m, d, first);
    const uint32_t same = __ballot_sync(m, d == d0);
    if (d != d0) {
      if ((d >> 15) == rank) atomicAdd(&s_bins[d & (kHalf16 - 1)], 1u);
    } else if (lane == first && (d0 >> 15) == rank) {
      atomicAdd(&s_bins[d0 & (kHalf16 - 1)], (uint32_t)__popc(same));
    }
  });
  __syncthreads();
  for (int i = threadIdx.x; i < kHalf16; i += kHistThreads) {
    const uint32_t c = s_bins[i];
    if (c) atomicAdd(&hist[rank * kHalf16 + i], c);
  }
}

// Per round: base16 = exclusive prefix of hist (65536 entries); per high byte
// h: baseA[h] = base16[h*256] (the bases of step A), the first tile of bucket
// h among step B's tiles (tile_first[0..256], tiles of `tile` keys) and
// bucket_trivial[h] (one low byte holds all of the bucket's keys); skip[passA]
// (one bucket holds all n keys) and skip[passB] (every bucket is trivial).
// One CTA of 1024 threads; thread t owns the 64 digits [64t, 64t + 64).
template <int TILE>
__global__ void __launch_bounds__(1024) k_scan16(const uint32_t* __restrict__ hist,
                                                 uint32_t* __restrict__ base16,
                                                 uint32_t* __restrict__ baseA,
                                                 uint32_t* __restrict__ tile_first,
                                                 uint32_t* __restrict__ bucket_trivial,
                                                 uint32_t* __restrict__ skip, int passA,
                                                 int64_t n) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_len[256];
  __shared__ uint32_t s_flags[2];
  constexpr int PER = kR16 / 1024;  // 64: a quarter of a bucket per thread
  const int t = threadIdx.x;
  if (t < 2) s_flags[t] = 0;
  uint32_t local = 0, mx = 0;
  for (int j = 0; j < PER; ++j) {
    const uint32_t c = hist[t * PER + j];
    local += c;
    mx = max(mx, c);
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan<1024>(local, s_warp, total);
  for (int j = 0; j < PER; ++j) {
    base16[t * PER + j] = run;
    run += hist[t * PER + j];
  }
  // per bucket (4 threads each): length and the largest low-byte count
  uint32_t blen = local, bmax = mx;
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    blen += __shfl_xor_sync(kFullMask, blen, o);
    bmax = max(bmax, __shfl_xor_sync(kFullMask, bmax, o));
  }
  const int h = t >> 2;
  if ((t & 3) == 0) {
    s_len[h] = blen;
    baseA[h] = base16[h * 256];
    bucket_trivial[h] = blen > 0 && bmax == blen;
    if ((int64_t)blen == n) s_flags[0] = 1;          // step A is the identity
    if (blen > 0 && bmax != blen) s_flags[1] = 1;    // some bucket needs step B
  }
  __syncthreads();
  if (t < 32) {  // tiles per bucket and their exclusive prefix: lane l takes buckets [8l, 8l+8)
    uint32_t tiles[8], sum = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      tiles[j] = (s_len[t * 8 + j] + TILE - 1) / TILE;
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
    for (int j = 0; j < 8; ++j) {
      tile_first[t * 8 + j] = first;
      first += tiles[j];
    }
    if (t == 31) tile_first[256] = first;
  }
  if (t == 0) {
    skip[passA] = s_flags[0];
    skip[passA + 1] = s_flags[1] ? 0u : 1u;
  }
}

// Step B: an ordered radix-256 round by the low byte inside every bucket. Tile
// ids come in launch order; tile t belongs to the bucket h with
// tile_first[h] <= t < tile_first[h + 1], and the look-back never leaves the
// bucket (its first tile publishes inclusive counts). Positions are absolute:
// the digit bases are base16[h*256 + l].
template <typename K, typename V, int THREADS, int KPT, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
    k_bucket16(PassParams p, const uint32_t* __restrict__ base16,
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
  if (tile >= tile_first[256]) return;  // more CTAs than tiles
  int lo = 0, hi = 255;  // the last bucket whose first tile is <= tile
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_first[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  const int h = lo;
  const int64_t start = base16[h * 256];
  const int64_t end = h < 255 ? (int64_t)base16[(h + 1) * 256] : p.n;
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
  if (tile_n == TILE)
    onesweep_tile_ordered<K, V, 8, THREADS, KPT, true>(p, tile, lt == 0, tile_base, tile_n, kin,
                                                       kout, vin, vout, base16 + h * 256,
                                                       (uint32_t)p.n, smem);
  else
    onesweep_tile_ordered<K, V, 8, THREADS, KPT, false>(p, tile, lt == 0, tile_base, tile_n,
                                                        kin, kout, vin, vout, base16 + h * 256,
                                                        (uint32_t)p.n, smem);
}

}  // namespace

// One whole radix-65536 sort: per round (16-bit digit at `shift`) the
// histogram, the scan, step A (high byte, all keys) and step B (low byte, per
// bucket); kernel passes 2q (A) and 2q+1 (B) of round q share the skip and
// tile-counter arrays, so the buffer parity follows the executed passes.
// Workspace: hist holds the 65536 counts, then baseA[256], tile_first[257]
// (padded to 512) and bucket_trivial[256]; base holds base16; status[0] the
// look-back rows of step A, status[1] those of step B.
template <typename K, typename V, int THREADS, int KPT, int MINB>
cudaError_t pr2_launch(const LsdArgs& a, cudaStream_t st) {
  using S = OnesweepShape<K, V, 8, THREADS, KPT>;
  constexpr int KB = 8 * (int)sizeof(K), ROUNDS = KB / 16, P2 = 2 * ROUNDS;
  constexpr bool HV = HasVal<V>::value;
  constexpr int TILE = S::TILE;
  const int64_t tiles = (a.n + TILE - 1) / TILE;
  uint32_t* hist16 = a.hist;
  uint32_t* baseA = hist16 + kR16;
  uint32_t* tile_first = baseA + 256;
  uint32_t* bucket_trivial = tile_first + 512;
  uint32_t* base16 = a.base;
  cudaError_t e;
  if ((e = cudaMemsetAsync(a.counters, 0, sizeof(uint32_t) * P2, st))) return e;
  constexpr size_t HSMEM = sizeof(uint32_t) * kHalf16;
  if ((e = cudaFuncSetAttribute(k_hist16<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)HSMEM)))
    return e;
  constexpr size_t smem = OrderedShape<K, V, 8, THREADS, KPT>::SMEM;
  auto kA = k_onesweep<K, V, 8, THREADS, KPT, MINB>;
  auto kB = k_bucket16<K, V, THREADS, KPT, MINB>;
  if (smem > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(kA, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
      return e;
    if ((e = cudaFuncSetAttribute(kB, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
      return e;
  }
  using FC = FirstCfg<K, THREADS, KPT, MINB>;
  constexpr size_t fsmem = FirstShape<K, 8, FC::T, FC::KP>::SMEM;
  if constexpr (!HV && fsmem > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(k_onesweep_first<K, 8, FC::T, FC::KP, MINB>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem)))
      return e;
  }
  const int hgrid = std::max(2, (a.num_sms / 2) * 2);  // pairs of CTAs, one CTA per SM
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
  pp.trace = nullptr;
  pp.prefetch_tiles = a.prefetch_tiles;
  pp.check_mode = a.check_mode;
  pp.mask = 0xffu;
  pp.status_next = nullptr;
  for (int q = 0; q < ROUNDS; ++q) {
    const int shift = 16 * q;
    if ((e = cudaMemsetAsync(hist16, 0, sizeof(uint32_t) * kR16, st))) return e;
    timer_begin(a.timer, "k_hist16", st);
    k_hist16<K><<<hgrid, kHistThreads, HSMEM, st>>>(static_cast<const K*>(a.keys),
                                                      static_cast<const K*>(a.alt_keys), a.skip,
                                                      2 * q, a.n, shift, hist16);
    timer_end(a.timer, st);
    timer_begin(a.timer, "k_scan16", st);
    k_scan16<TILE><<<1, 1024, 0, st>>>(hist16, base16, baseA, tile_first, bucket_trivial,
                                       a.skip, 2 * q, a.n);
    timer_end(a.timer, st);
    if ((e = cudaMemsetAsync(a.status[0], 0, sizeof(uint32_t) * 256 * tiles, st))) return e;
    if ((e = cudaMemsetAsync(a.status[1], 0, sizeof(uint32_t) * 256 * (tiles + 256), st)))
      return e;
    // step A: the high byte, over all keys (the input is sorted by bits [0, shift))
    pp.pass = 2 * q;
    pp.shift = shift + 8;
    pp.byte_sel = radix8_byte_sel(shift + 8);
    pp.low_shift = shift;
    pp.base = baseA;
    pp.status = a.status[0];
    pp.counter = a.counters + 2 * q;
    timer_begin(a.timer, "k_pr2_high", st);
    if (!HV && q == 0)  // keys only, first round: order-free
      k_onesweep_first<K, 8, FC::T, FC::KP, MINB><<<(unsigned)tiles, FC::T, fsmem, st>>>(pp);
    else
      kA<<<(unsigned)tiles, THREADS, smem, st>>>(pp);
    timer_end(a.timer, st);
    // step B: the low byte, inside every bucket
    pp.pass = 2 * q + 1;
    pp.shift = shift;
    pp.byte_sel = radix8_byte_sel(shift);
    pp.low_shift = shift;
    pp.base = nullptr;
    pp.status = a.status[1];
    pp.counter = a.counters + 2 * q + 1;
    timer_begin(a.timer, "k_pr2_low", st);
    kB<<<(unsigned)(tiles + 256), THREADS, smem, st>>>(pp, base16, tile_first, bucket_trivial);
    timer_end(a.timer, st);
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

template <typename K, typename V, int THREADS, int KPT, int MINB>
constexpr LsdEntry pr2_entry() {
  using S = OnesweepShape<K, V, 8, THREADS, KPT>;
  constexpr int KB = 8 * (int)sizeof(K);
  LsdEntry e{KB,
             HasVal<V>::value ? (int)(8 * sizeof(V)) : 0,
             16,
             THREADS,
             KPT,
             (int64_t)S::TILE,
             kR16,          // hist and base hold 65536 words per kernel pass
             2 * (KB / 16),  // kernel passes: two steps per 16-bit round
             256,           // look-back words per tile
             2,
             &pr2_launch<K, V, THREADS, KPT, MINB>};
  e.extra_status_rows = 256;  // step B: at most one partial tile per bucket
  return e;
}

static const LsdEntry kR16None32[] = {pr2_entry<uint32_t, NoVal, 256, 32, 3>()};
static const LsdEntry kR16V32_32[] = {pr2_entry<uint32_t, uint32_t, 256, 20, 3>()};
static const LsdEntry kR16V64_32[] = {pr2_entry<uint32_t, uint64_t, 256, 16, 2>()};
static const LsdEntry kR16None64[] = {pr2_entry<uint64_t, NoVal, 256, 20, 3>()};
static const LsdEntry kR16V32_64[] = {pr2_entry<uint64_t, uint32_t, 256, 16, 2>()};
static const LsdEntry kR16V64_64[] = {pr2_entry<uint64_t, uint64_t, 256, 12, 2>()};

int pr2_variants(int key_bits, int val_bits, const LsdEntry** out) {
  const LsdEntry* t[2][3] = {{kR16None32, kR16V32_32, kR16V64_32},
                             {kR16None64, kR16V32_64, kR16V64_64}};
  if (key_bits != 32 && key_bits != 64) return 0;
  if (val_bits != 0 && val_bits != 32 && val_bits != 64) return 0;
  *out = t[key_bits == 32 ? 0 : 1][val_bits == 0 ? 0 : val_bits == 32 ? 1 : 2];
  return 1;
}

}  // namespace isort
