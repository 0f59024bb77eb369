// Radix 2048 (11-bit digits: three rounds of 11, 11 and 10 bits on 32-bit
// keys, six on 64-bit keys); radix 65536 is radix16.cu.
//
// Paper mapping (Section "SR4, PR2, PR4, BTN and OET under MBSP", Eqs. Tp,
// Tp2): each worker counts the digits of its share of the keys, the p x r count
// matrix is exchanged (the 2prg term, which grows with r), and every worker
// routes its keys to their global positions. A per-tile decoupled look-back
// would need 8 KiB of status per tile at r = 2048 (a quarter of a tile's keys),
// so each round here is the paper's count-sort literally: the input is read
// twice (count, then place) and written once. A "block" is one row of the
// count matrix, 2^16 keys.
//
//   k_count_smem   per block, the histogram in one CTA's shared memory, eight
//                  copies of the bins to spread contention.
//   k_colscan      per digit, the exclusive prefix over blocks (the count
//                  matrix exchange), in place, and the digit totals.
//   k_digscan      exclusive prefix over the digit totals -> global bases;
//                  flags a pass whose digit is constant.
//   k_scatter_wide per block, in input order, sub-tiles of kSubKeys keys are
//                  sorted stably by the digit in shared memory (a stable
//                  partition by its low 8 bits, then by the rest), then each
//                  key goes to base[d] + (earlier blocks' d-keys) + (this
//                  block's d-keys so far) + (its rank in the sub-tile's run of
//                  d). The per-block running offsets live in shared memory.
#include <algorithm>

#include "common.cuh"
#include "isort_internal.h"

namespace isort {
namespace {


// Keys per count-matrix row (block) and kernel names, per digit width.
template <int BITS>
struct Wide;
template <>
struct Wide<11> {
  static constexpr int64_t BLOCK_KEYS = int64_t(1) << 16;
  static constexpr const char* COUNT = "k_count11";
  static constexpr const char* SCATTER = "k_scatter11";
};
constexpr int kCountThreads = 1024;
constexpr int kScatterThreads = 256;
constexpr int kScatterKpt = 16;
constexpr int kSubKeys = kScatterThreads * kScatterKpt;  // 4096 keys per sub-tile
constexpr int kWarps = kScatterThreads / 32;
constexpr int kMaskBufs = 3;
// The run phase reads the sorted sub-tile in a blocked arrangement (thread t
// takes positions [16t, 16t+16)); one pad word per 32 keeps those reads free of
// bank conflicts.
constexpr int kPadded = kSubKeys + kSubKeys / 32;
__device__ __forceinline__ int padj(int j) { return j + (j >> 5); }
constexpr uint32_t kNoDigit = 0x10000u;  // differs from every 16-bit digit


template <typename K>
__device__ __forceinline__ uint32_t digit_w(K k, int shift, uint32_t mask) {
  return static_cast<uint32_t>(k >> shift) & mask;
}

__device__ __forceinline__ int input_parity(const uint32_t* skip, int pass) {
  int src = 0;
  for (int q = 0; q < pass; ++q) src ^= (skip[q] == 0);
  return src;
}

// ---------------------------------------------------------------------------
// Per block of Wide<11>::BLOCK_KEYS keys, the R-bin digit histogram in shared
// memory (R <= 4096): warp w adds into copy w % 8 of the bins, so equal digits
// from different warps rarely meet on one counter; the copies are summed into
// the block's row of the count matrix.
template <typename K, int R>
__global__ void __launch_bounds__(kCountThreads)
    k_count_smem(const K* buf0, const K* buf1, const uint32_t* skip, int pass, int64_t n,
                 int shift, uint32_t mask, uint32_t* counts) {
  constexpr int COPIES = 8;
  extern __shared__ __align__(16) uint32_t s_bins[];  // [COPIES][R]
  for (int i = threadIdx.x; i < COPIES * R; i += kCountThreads) s_bins[i] = 0;
  __syncthreads();
  const K* keys = input_parity(skip, pass) ? buf1 : buf0;
  const int64_t lo = (int64_t)blockIdx.x * Wide<11>::BLOCK_KEYS;
  const int64_t hi = min(n, lo + Wide<11>::BLOCK_KEYS);
  uint32_t* my = s_bins + ((threadIdx.x >> 5) % COPIES) * R;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kCountThreads)
    atomicAdd(&my[digit_w(keys[i], shift, mask)], 1u);
  __syncthreads();
  uint32_t* row = counts + (size_t)blockIdx.x * R;
  for (int d = threadIdx.x; d < R; d += kCountThreads) {
    uint32_t sum = 0;
#pragma unroll
    for (int c = 0; c < COPIES; ++c) sum += s_bins[c * R + d];
    row[d] = sum;
  }
}

// Per digit: exclusive prefix over the blocks (in place) and the total. One
// CTA per 32 digits: lane = digit, warp w takes a contiguous slice of the
// blocks (coalesced 128-byte rows), the 32 slice sums are scanned in shared
// memory, and a second sweep writes the prefixes.
template <int R>
__global__ void __launch_bounds__(1024) k_colscan(uint32_t* counts, int64_t nblocks,
                                                  uint32_t* total) {
  __shared__ uint32_t s_sum[32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int d = blockIdx.x * 32 + lane;
  const int64_t per = (nblocks + 31) / 32;
  const int64_t b0 = min(nblocks, warp * per), b1 = min(nblocks, b0 + per);
  uint32_t sum = 0;
  int64_t b = b0;
  for (; b + 4 <= b1; b += 4) {
    uint32_t c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) c[u] = counts[(size_t)(b + u) * R + d];
    sum += c[0] + c[1] + c[2] + c[3];
  }
  for (; b < b1; ++b) sum += counts[(size_t)b * R + d];
  s_sum[warp][lane] = sum;
  __syncthreads();
  uint32_t run = 0;  // blocks before this warp's slice
  for (int w = 0; w < warp; ++w) run += s_sum[w][lane];
  if (warp == 31) total[d] = run + sum;
  for (b = b0; b + 4 <= b1; b += 4) {
    uint32_t c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) c[u] = counts[(size_t)(b + u) * R + d];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      counts[(size_t)(b + u) * R + d] = run;
      run += c[u];
    }
  }
  for (; b < b1; ++b) {
    const uint32_t c = counts[(size_t)b * R + d];
    counts[(size_t)b * R + d] = run;
    run += c;
  }
}

// One CTA: base[d] = sum of totals below d; skip[pass] = (one digit holds all n).
template <int R>
__global__ void __launch_bounds__(1024) k_digscan(const uint32_t* total, uint32_t* base,
                                                  uint32_t* skip, int pass, int64_t n) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_trivial;
  constexpr int PER = R / 1024;
  static_assert(PER >= 1 && R % 1024 == 0, "at least one digit per thread");
  const int d0 = threadIdx.x * PER;
  if (threadIdx.x == 0) s_trivial = 0;
  uint32_t local = 0;
  bool trivial = false;
  for (int j = 0; j < PER; ++j) {
    const uint32_t c = total[d0 + j];
    local += c;
    trivial |= (int64_t)c == n;
  }
  __syncthreads();
  if (trivial) s_trivial = 1;
  uint32_t tot;
  uint32_t run = block_exclusive_scan<1024>(local, s_warp, tot);
  for (int j = 0; j < PER; ++j) {
    base[d0 + j] = run;
    run += total[d0 + j];
  }
  if (threadIdx.x == 0) skip[pass] = s_trivial;
}

// ---------------------------------------------------------------------------
// Shared memory of k_scatter_wide.
template <typename K, typename V>
struct Scatter16Smem {
  static constexpr bool HV = HasVal<V>::value;
  uint32_t wcnt[kWarps][256];           // per-warp digit counters / offsets
  uint32_t warp_tot[32];
  K keys_a[kSubKeys];                   // after the low-byte partition
  K keys_b[kPadded];                    // after the high-byte partition (padded index)
  uint16_t idx_a[kSubKeys];             // sub-tile index of each key
  uint32_t idx_b[kPadded];              // (padded index)
  uint32_t masks[kWarps][kMaskBufs][256];  // warp peer masks
  typename std::conditional<HV, V, uint32_t>::type vals[HV ? kSubKeys : 1];
};

// Stable partition of the sub-tile's keys (registers, warp-striped in input
// order) by an 8-bit digit: pos[i] = the key's position in the partitioned
// sub-tile. Same warp ranking as the onesweep pass (peer masks in shared
// memory, one warp barrier per key row), then per-warp counts and a block scan.
template <bool FULL, typename DigitFn>
__device__ __forceinline__ void partition8(int n_sub, uint32_t* wcnt, uint32_t (*masks)[256],
                                           uint32_t* warp_tot, DigitFn digit,
                                           uint32_t pos[kScatterKpt]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wofs = warp * 32 * kScatterKpt + lane;
  for (int i = tid; i < kWarps * 256; i += kScatterThreads) wcnt[i] = 0;
  for (int i = tid; i < kWarps * kMaskBufs * 256; i += kScatterThreads) (&masks[0][0])[i] = 0;
  __syncthreads();
  uint32_t* my = wcnt + warp * 256;
  uint32_t(*mm)[256] = masks + warp * kMaskBufs;
  const uint32_t ge = []() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_ge;" : "=r"(m));
    return m;
  }();
  const uint32_t bit = 1u << lane;
  uint32_t* slot1 = &mm[0][0];
  uint32_t* slot2 = &mm[0][0];
  bool lead1 = false, lead2 = false;
#pragma unroll
  for (int i = 0; i < kScatterKpt; ++i) {
    const bool valid = FULL || wofs + i * 32 < n_sub;
    const uint32_t d = digit(i);
    uint32_t* slot = &mm[i % kMaskBufs][d];
    if (lead2) *slot2 = 0u;
    if (valid) atomicOr(slot, bit);
    __syncwarp();
    const uint32_t peers = valid ? *slot : 0u;
    const bool leader = valid && (peers >> lane) == 1u;
    uint32_t after = 0;
    if (leader) after = atomicAdd(&my[d], __popc(peers)) + __popc(peers);
    after = __shfl_sync(kFullMask, after, (31 - __clz(peers)) & 31);
    pos[i] = after - __popc(peers & ge);
    slot2 = slot1;
    lead2 = lead1;
    slot1 = slot;
    lead1 = leader;
  }
  __syncthreads();
  // per digit (thread tid owns digit tid): warp-exclusive offsets, then the
  // block-wide digit starts
  uint32_t sum = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const uint32_t c = wcnt[w * 256 + tid];
    wcnt[w * 256 + tid] = sum;
    sum += c;
  }
  uint32_t tot;
  const uint32_t start = block_exclusive_scan<kScatterThreads>(sum, warp_tot, tot);
#pragma unroll
  for (int w = 0; w < kWarps; ++w) wcnt[w * 256 + tid] += start;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScatterKpt; ++i) pos[i] += wcnt[warp * 256 + digit(i)];
}

// width = the pass's digit width (9..16 bits): the first partition takes its
// low 8 bits, the second the remaining width - 8. col[d] = the block's running
// offset of digit d; with COMBINED it already includes the global base[d]
// (and base is not read).
template <typename K, typename V, bool FULL, bool COMBINED>
__device__ __forceinline__ void scatter_subtile(Scatter16Smem<K, V>& sm, const K* kin, K* kout,
                                                const V* vin, V* vout, int64_t sub_base,
                                                int n_sub, int shift, int width, uint32_t* col,
                                                const uint32_t* base, int64_t n, uint32_t* err) {
  const uint32_t wmask = (1u << width) - 1u;
  const uint32_t hmask = (1u << (width - 8)) - 1u;
  constexpr bool HV = HasVal<V>::value;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wofs = warp * 32 * kScatterKpt + lane;
  K key[kScatterKpt];
  uint32_t pos[kScatterKpt];
#pragma unroll
  for (int i = 0; i < kScatterKpt; ++i)
    key[i] = (FULL || wofs + i * 32 < n_sub) ? kin[sub_base + wofs + i * 32] : K(0);
  if constexpr (HV) {
#pragma unroll
    for (int i = 0; i < kScatterKpt; ++i)
      if (FULL || wofs + i * 32 < n_sub) sm.vals[wofs + i * 32] = vin[sub_base + wofs + i * 32];
  }
  // partition by the low byte of the digit
  partition8<FULL>(n_sub, &sm.wcnt[0][0], sm.masks[0], sm.warp_tot,
                   [&](int i) { return static_cast<uint32_t>(key[i] >> shift) & 0xffu; }, pos);
#pragma unroll
  for (int i = 0; i < kScatterKpt; ++i)
    if (FULL || wofs + i * 32 < n_sub) {
      sm.keys_a[pos[i]] = key[i];
      sm.idx_a[pos[i]] = (uint16_t)(wofs + i * 32);
    }
  __syncthreads();
  // then stably by the high bits: the sub-tile ends up ordered by the digit
  uint32_t idx[kScatterKpt];
#pragma unroll
  for (int i = 0; i < kScatterKpt; ++i) {
    key[i] = (FULL || wofs + i * 32 < n_sub) ? sm.keys_a[wofs + i * 32] : K(0);
    idx[i] = (FULL || wofs + i * 32 < n_sub) ? sm.idx_a[wofs + i * 32] : 0u;
  }
  partition8<FULL>(n_sub, &sm.wcnt[0][0], sm.masks[0], sm.warp_tot,
                   [&](int i) { return static_cast<uint32_t>(key[i] >> (shift + 8)) & hmask; },
                   pos);
#pragma unroll
  for (int i = 0; i < kScatterKpt; ++i)
    if (FULL || wofs + i * 32 < n_sub) {
      sm.keys_b[padj(pos[i])] = key[i];
      sm.idx_b[padj(pos[i])] = idx[i];
    }
  __syncthreads();

  // Runs of equal digits in the sorted sub-tile: thread t takes the blocked
  // range [t*KPT, (t+1)*KPT) into registers; the start of the run holding
  // position j is the last run start at or before j (a block-wide max scan of
  // the threads' last run starts).
  const int j0 = tid * kScatterKpt;
  K kk[kScatterKpt];
  uint32_t ix[kScatterKpt], dg[kScatterKpt];
#pragma unroll
  for (int k = 0; k < kScatterKpt; ++k) {
    const int j = j0 + k;
    const bool valid = FULL || j < n_sub;
    kk[k] = valid ? sm.keys_b[padj(j)] : K(0);
    ix[k] = valid ? sm.idx_b[padj(j)] : 0u;
    dg[k] = valid ? digit_w(kk[k], shift, wmask) : kNoDigit;
  }
  const uint32_t prev = j0 > 0 && (FULL || j0 - 1 < n_sub)
                            ? digit_w(sm.keys_b[padj(j0 - 1)], shift, wmask)
                            : kNoDigit;
  const uint32_t next = (FULL ? j0 + kScatterKpt < kSubKeys : j0 + kScatterKpt < n_sub)
                            ? digit_w(sm.keys_b[padj(j0 + kScatterKpt)], shift, wmask)
                            : kNoDigit;
  uint32_t starts = 0, ends = 0;  // bit k: position j0+k starts / ends a run
#pragma unroll
  for (int k = 0; k < kScatterKpt; ++k) {
    const bool valid = FULL || j0 + k < n_sub;
    const uint32_t before = k == 0 ? prev : dg[k - 1];
    const uint32_t after = k == kScatterKpt - 1 ? next : dg[k + 1];
    if (valid && before != dg[k]) starts |= 1u << k;
    if (valid && after != dg[k]) ends |= 1u << k;
  }
  uint32_t carry_in = 0;  // last run start strictly before this thread's range
  {
    uint32_t v = starts ? (uint32_t)(j0 + 31 - __clz(starts)) : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFullMask, v, o);
      if (lane >= o) v = max(v, y);
    }
    if (lane == 31) sm.warp_tot[warp] = v;
    __syncthreads();
    uint32_t wmax = 0;
    for (int w = 0; w < warp; ++w) wmax = max(wmax, sm.warp_tot[w]);
    const uint32_t below = __shfl_up_sync(kFullMask, v, 1);
    carry_in = max(wmax, lane ? below : 0u);
  }
  // global positions: column running offset + global base + rank in the run
  uint32_t gpos[kScatterKpt];
  int cur = (int)carry_in;
#pragma unroll
  for (int k = 0; k < kScatterKpt; ++k) {
    if ((starts >> k) & 1u) cur = j0 + k;
    if (FULL || j0 + k < n_sub)
      gpos[k] = col[dg[k]] + (COMBINED ? 0u : base[dg[k]]) + (uint32_t)(j0 + k - cur);
  }
  __syncthreads();  // every read of col[] precedes the updates below
  const uint32_t n32 = (uint32_t)n;
  cur = (int)carry_in;
#pragma unroll
  for (int k = 0; k < kScatterKpt; ++k) {
    if ((starts >> k) & 1u) cur = j0 + k;
    if (FULL || j0 + k < n_sub) {
      if (gpos[k] < n32) {
        kout[gpos[k]] = kk[k];
        if constexpr (HV) vout[gpos[k]] = sm.vals[ix[k]];
      } else {
        atomicOr(err, kErrBounds);
      }
      // a run end advances the column by the run's length (one run per digit
      // per sub-tile, so a single writer)
      if ((ends >> k) & 1u) col[dg[k]] += (uint32_t)(j0 + k - cur + 1);
    }
  }
  __syncthreads();  // column updates visible to the next sub-tile; smem reusable
}

template <typename K, typename V, int BITS>
__global__ void __launch_bounds__(kScatterThreads, 2)
    k_scatter_wide(K* kbuf0, K* kbuf1, V* vbuf0, V* vbuf1, const uint32_t* skip, int pass,
                   int64_t n, int shift, int width, uint32_t* counts, const uint32_t* base,
                   uint32_t* err) {
  if (skip[pass]) return;  // the digit is constant: this round is the identity
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Scatter16Smem<K, V>& sm = *reinterpret_cast<Scatter16Smem<K, V>*>(smem_raw);
  const int src = input_parity(skip, pass);
  const K* kin = src ? kbuf1 : kbuf0;
  K* kout = src ? kbuf0 : kbuf1;
  const V* vin = src ? vbuf1 : vbuf0;
  V* vout = src ? vbuf0 : vbuf1;
  constexpr int R = 1 << BITS;
  const int64_t block = blockIdx.x;
  const int64_t lo = block * Wide<BITS>::BLOCK_KEYS;
  const int64_t hi = min(n, lo + Wide<BITS>::BLOCK_KEYS);
  uint32_t* col = counts + (size_t)block * R;
  if constexpr (R <= 4096) {
    // the block's running output positions (row offset + global base) fit in
    // shared memory: one read of the row, no global traffic per key or run
    uint32_t* s_pos = reinterpret_cast<uint32_t*>(smem_raw + sizeof(Scatter16Smem<K, V>));
    for (int d = threadIdx.x; d < R; d += kScatterThreads) s_pos[d] = col[d] + base[d];
    __syncthreads();
    for (int64_t sb = lo; sb < hi; sb += kSubKeys) {
      const int n_sub = (int)min((int64_t)kSubKeys, hi - sb);
      if (n_sub == kSubKeys)
        scatter_subtile<K, V, true, true>(sm, kin, kout, vin, vout, sb, n_sub, shift, width,
                                          s_pos, nullptr, n, err);
      else
        scatter_subtile<K, V, false, true>(sm, kin, kout, vin, vout, sb, n_sub, shift, width,
                                           s_pos, nullptr, n, err);
    }
  } else {
    for (int64_t sb = lo; sb < hi; sb += kSubKeys) {
      const int n_sub = (int)min((int64_t)kSubKeys, hi - sb);
      if (n_sub == kSubKeys)
        scatter_subtile<K, V, true, false>(sm, kin, kout, vin, vout, sb, n_sub, shift, width, col,
                                           base, n, err);
      else
        scatter_subtile<K, V, false, false>(sm, kin, kout, vin, vout, sb, n_sub, shift, width,
                                            col, base, n, err);
    }
  }
}

template <typename K, typename V>
__global__ void k_copy_back16(const uint32_t* __restrict__ skip, int passes, K* keys,
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

}  // namespace

template <typename K, typename V, int BITS>
cudaError_t wide_launch(const LsdArgs& a, cudaStream_t st) {
  constexpr int KB = 8 * (int)sizeof(K);
  constexpr int R = 1 << BITS;
  constexpr int P = (KB + BITS - 1) / BITS;
  constexpr int64_t BK = Wide<BITS>::BLOCK_KEYS;
  const int64_t nblocks = (a.n + BK - 1) / BK;
  uint32_t* counts = a.status[0];  // the count matrix lives in the status area
  uint32_t* total = a.hist;        // [R]
  uint32_t* base = a.base;         // [R] (one pass at a time)
  cudaError_t e;
  const size_t count_smem = sizeof(uint32_t) * 8 * R;
  if ((e = cudaFuncSetAttribute(k_count_smem<K, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)count_smem)))
    return e;
  const size_t sc_smem = sizeof(Scatter16Smem<K, V>) + (R <= 4096 ? sizeof(uint32_t) * R : 0);
  if ((e = cudaFuncSetAttribute(k_scatter_wide<K, V, BITS>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc_smem)))
    return e;
  for (int q = 0; q < P; ++q) {
    const int shift = BITS * q;
    const int width = KB - shift < BITS ? KB - shift : BITS;
    timer_begin(a.timer, Wide<BITS>::COUNT, st);
    k_count_smem<K, R><<<(unsigned)nblocks, kCountThreads, count_smem, st>>>(
        static_cast<const K*>(a.keys), static_cast<const K*>(a.alt_keys), a.skip, q, a.n, shift,
        (1u << width) - 1u, counts);
    timer_end(a.timer, st);
    timer_begin(a.timer, "k_colscan", st);
    k_colscan<R><<<R / 32, 1024, 0, st>>>(counts, nblocks, total);
    timer_end(a.timer, st);
    timer_begin(a.timer, "k_digscan", st);
    k_digscan<R><<<1, 1024, 0, st>>>(total, base, a.skip, q, a.n);
    timer_end(a.timer, st);
    timer_begin(a.timer, Wide<BITS>::SCATTER, st);
    k_scatter_wide<K, V, BITS><<<(unsigned)nblocks, kScatterThreads, sc_smem, st>>>(
        static_cast<K*>(a.keys), static_cast<K*>(a.alt_keys), static_cast<V*>(a.vals),
        static_cast<V*>(a.alt_vals), a.skip, q, a.n, shift, width, counts, base, a.err);
    timer_end(a.timer, st);
  }
  const int cblocks = (int)std::min<int64_t>((a.n + 255) / 256, (int64_t)a.num_sms * 8);
  timer_begin(a.timer, "k_copy_back", st);
  k_copy_back16<K, V><<<cblocks, 256, 0, st>>>(a.skip, P, static_cast<K*>(a.keys),
                                               static_cast<const K*>(a.alt_keys),
                                               static_cast<V*>(a.vals),
                                               static_cast<const V*>(a.alt_vals), a.n);
  timer_end(a.timer, st);
  return cudaGetLastError();
}

template <typename K, typename V, int BITS>
constexpr LsdEntry wide_entry() {
  constexpr int KB = 8 * (int)sizeof(K);
  return LsdEntry{KB,
                  HasVal<V>::value ? (int)(8 * sizeof(V)) : 0,
                  BITS,
                  kScatterThreads,
                  kScatterKpt,
                  Wide<BITS>::BLOCK_KEYS,  // "tile" = one count-matrix row
                  1 << BITS,
                  (KB + BITS - 1) / BITS,
                  (size_t)1 << BITS,       // the count matrix: one row per block
                  1,                       // in one buffer
                  &wide_launch<K, V, BITS>};
}

#define ISORT_WIDE_TABLES(B)                                                             \
  static const LsdEntry kW##B##None32[] = {wide_entry<uint32_t, NoVal, B>()};            \
  static const LsdEntry kW##B##V32_32[] = {wide_entry<uint32_t, uint32_t, B>()};         \
  static const LsdEntry kW##B##V64_32[] = {wide_entry<uint32_t, uint64_t, B>()};         \
  static const LsdEntry kW##B##None64[] = {wide_entry<uint64_t, NoVal, B>()};            \
  static const LsdEntry kW##B##V32_64[] = {wide_entry<uint64_t, uint32_t, B>()};         \
  static const LsdEntry kW##B##V64_64[] = {wide_entry<uint64_t, uint64_t, B>()};
ISORT_WIDE_TABLES(11)
#undef ISORT_WIDE_TABLES

int wide_variants(int key_bits, int val_bits, int radix_bits, const LsdEntry** out) {
  if (val_bits != 0 && val_bits != 32 && val_bits != 64) return 0;
  const int vi = val_bits == 0 ? 0 : val_bits == 32 ? 1 : 2;
  const LsdEntry* t11[2][3] = {{kW11None32, kW11V32_32, kW11V64_32},
                               {kW11None64, kW11V32_64, kW11V64_64}};
  if (key_bits != 32 && key_bits != 64) return 0;
  const int ki = key_bits == 32 ? 0 : 1;
  if (radix_bits == 11) *out = t11[ki][vi];
  else return 0;
  return 1;
}

}  // namespace isort
