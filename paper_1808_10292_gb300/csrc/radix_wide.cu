// Radix-65536 passes (the paper's PR2: 16-bit digits, two rounds on 32-bit keys).
//
// Paper mapping (Section "SR4, PR2, PR4, BTN and OET under MBSP", Eqs. Tp,
// Tp2): each worker counts the digits of its share of the keys, the p x r count
// matrix is exchanged (the 2prg term, which grows with r and is why the paper
// found PR2 slower than PR4), and every worker routes its keys to their global
// positions. With r = 65536 a per-tile decoupled look-back would need 256 KiB
// of status per tile, so each round here is the paper's count-sort literally:
// the input is read twice (count, then place) and written once.
//
//   k_count16    per block of kBlockKeys keys, the 65536-bin digit histogram.
//                A 2-CTA thread-block cluster holds it in distributed shared
//                memory: CTA r owns bins [r*32768, (r+1)*32768) as 32-bit
//                counters (128 KiB) and each CTA reads half of the block,
//                adding into the owner's shared memory (local or remote).
//   k_colscan16  per digit, the exclusive prefix over blocks (the count
//                matrix exchange) and the digit totals.
//   k_digscan16  exclusive prefix over the 65536 digit totals -> global bases;
//                flags a pass whose digit is constant.
//   k_scatter16  per block, in input order, sub-tiles of kSubKeys keys are
//                sorted stably by the 16-bit digit in shared memory (two
//                stable 8-bit partitions), then each key goes to
//                base[d] + (earlier blocks' d-keys) + (this block's d-keys so
//                far) + (its rank in the sub-tile's run of d). The per-block
//                running offsets live in the block's column of the matrix.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "isort_internal.h"

namespace cg = cooperative_groups;

namespace isort {
namespace {

constexpr int kR16 = 65536;
constexpr int kHalfBins = kR16 / 2;
constexpr int64_t kBlockKeys = int64_t(1) << 19;  // keys per count-matrix row
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
__device__ __forceinline__ uint32_t digit16(K k, int shift) {
  return static_cast<uint32_t>(k >> shift) & 0xffffu;
}

__device__ __forceinline__ int input_parity(const uint32_t* skip, int pass) {
  int src = 0;
  for (int q = 0; q < pass; ++q) src ^= (skip[q] == 0);
  return src;
}

// ---------------------------------------------------------------------------
template <typename K>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kCountThreads)
    k_count16(const K* buf0, const K* buf1, const uint32_t* skip, int pass, int64_t n, int shift,
              uint32_t* counts) {
  extern __shared__ __align__(16) uint32_t s_bins[];  // kHalfBins
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned rank = cluster.block_rank();
  for (int i = threadIdx.x; i < kHalfBins; i += kCountThreads) s_bins[i] = 0;
  cluster.sync();  // both halves zeroed before any remote add
  uint32_t* remote = cluster.map_shared_rank(s_bins, rank ^ 1);

  const K* keys = input_parity(skip, pass) ? buf1 : buf0;
  const int64_t block = blockIdx.x / 2;
  const int64_t lo = block * kBlockKeys;
  const int64_t hi = min(n, lo + kBlockKeys);
  const int64_t len = hi - lo;
  const int64_t half = (len + 1) / 2;
  const int64_t my_lo = lo + (rank ? half : 0);
  const int64_t my_hi = rank ? hi : lo + half;
  for (int64_t i = my_lo + threadIdx.x; i < my_hi; i += kCountThreads) {
    const uint32_t d = digit16(keys[i], shift);
    if ((d >> 15) == rank)
      atomicAdd(&s_bins[d & (kHalfBins - 1)], 1u);
    else
      atomicAdd(&remote[d & (kHalfBins - 1)], 1u);
  }
  cluster.sync();  // every add into my bins has landed; the partner may exit after this
  uint32_t* row = counts + (size_t)block * kR16 + (size_t)rank * kHalfBins;
  for (int i = threadIdx.x; i < kHalfBins; i += kCountThreads) row[i] = s_bins[i];
}

// Per digit: exclusive prefix over the blocks (in place) and the total.
__global__ void __launch_bounds__(256) k_colscan16(uint32_t* counts, int64_t nblocks,
                                                   uint32_t* total) {
  const int d = blockIdx.x * 256 + threadIdx.x;
  uint32_t sum = 0;
  int64_t b = 0;
  for (; b + 4 <= nblocks; b += 4) {
    uint32_t c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) c[u] = counts[(size_t)(b + u) * kR16 + d];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      counts[(size_t)(b + u) * kR16 + d] = sum;
      sum += c[u];
    }
  }
  for (; b < nblocks; ++b) {
    const uint32_t c = counts[(size_t)b * kR16 + d];
    counts[(size_t)b * kR16 + d] = sum;
    sum += c;
  }
  total[d] = sum;
}

// One CTA: base[d] = sum of totals below d; skip[pass] = (one digit holds all n).
__global__ void __launch_bounds__(1024) k_digscan16(const uint32_t* total, uint32_t* base,
                                                    uint32_t* skip, int pass, int64_t n) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_trivial;
  constexpr int PER = kR16 / 1024;
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
// Shared memory of k_scatter16.
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

template <typename K, typename V, bool FULL>
__device__ __forceinline__ void scatter16_subtile(Scatter16Smem<K, V>& sm, const K* kin, K* kout,
                                                  const V* vin, V* vout, int64_t sub_base,
                                                  int n_sub, int shift, uint32_t* col,
                                                  const uint32_t* base, int64_t n, uint32_t* err) {
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
  // then stably by the high byte: the sub-tile ends up ordered by the 16-bit digit
  uint32_t idx[kScatterKpt];
#pragma unroll
  for (int i = 0; i < kScatterKpt; ++i) {
    key[i] = (FULL || wofs + i * 32 < n_sub) ? sm.keys_a[wofs + i * 32] : K(0);
    idx[i] = (FULL || wofs + i * 32 < n_sub) ? sm.idx_a[wofs + i * 32] : 0u;
  }
  partition8<FULL>(n_sub, &sm.wcnt[0][0], sm.masks[0], sm.warp_tot,
                   [&](int i) { return static_cast<uint32_t>(key[i] >> (shift + 8)) & 0xffu; },
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
    dg[k] = valid ? digit16(kk[k], shift) : kNoDigit;
  }
  const uint32_t prev = j0 > 0 && (FULL || j0 - 1 < n_sub) ? digit16(sm.keys_b[padj(j0 - 1)], shift)
                                                           : kNoDigit;
  const uint32_t next = (FULL ? j0 + kScatterKpt < kSubKeys : j0 + kScatterKpt < n_sub)
                            ? digit16(sm.keys_b[padj(j0 + kScatterKpt)], shift)
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
    if (FULL || j0 + k < n_sub) gpos[k] = col[dg[k]] + base[dg[k]] + (uint32_t)(j0 + k - cur);
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

template <typename K, typename V>
__global__ void __launch_bounds__(kScatterThreads) k_scatter16(K* kbuf0, K* kbuf1, V* vbuf0,
                                                               V* vbuf1, const uint32_t* skip,
                                                               int pass, int64_t n, int shift,
                                                               uint32_t* counts,
                                                               const uint32_t* base,
                                                               uint32_t* err) {
  if (skip[pass]) return;  // the digit is constant: this round is the identity
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Scatter16Smem<K, V>& sm = *reinterpret_cast<Scatter16Smem<K, V>*>(smem_raw);
  const int src = input_parity(skip, pass);
  const K* kin = src ? kbuf1 : kbuf0;
  K* kout = src ? kbuf0 : kbuf1;
  const V* vin = src ? vbuf1 : vbuf0;
  V* vout = src ? vbuf0 : vbuf1;
  const int64_t block = blockIdx.x;
  const int64_t lo = block * kBlockKeys;
  const int64_t hi = min(n, lo + kBlockKeys);
  uint32_t* col = counts + (size_t)block * kR16;
  for (int64_t sb = lo; sb < hi; sb += kSubKeys) {
    const int n_sub = (int)min((int64_t)kSubKeys, hi - sb);
    if (n_sub == kSubKeys)
      scatter16_subtile<K, V, true>(sm, kin, kout, vin, vout, sb, n_sub, shift, col, base, n, err);
    else
      scatter16_subtile<K, V, false>(sm, kin, kout, vin, vout, sb, n_sub, shift, col, base, n,
                                     err);
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

template <typename K, typename V>
cudaError_t r16_launch(const LsdArgs& a, cudaStream_t st) {
  constexpr int P = (8 * sizeof(K)) / 16;
  const int64_t nblocks = (a.n + kBlockKeys - 1) / kBlockKeys;
  uint32_t* counts = a.status[0];  // the count matrix lives in the status area
  uint32_t* total = a.hist;        // [65536]
  uint32_t* base = a.base;         // [65536] (one pass at a time)
  cudaError_t e;
  const size_t count_smem = sizeof(uint32_t) * kHalfBins;
  if ((e = cudaFuncSetAttribute(k_count16<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)count_smem)))
    return e;
  const size_t sc_smem = sizeof(Scatter16Smem<K, V>);
  if ((e = cudaFuncSetAttribute(k_scatter16<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sc_smem)))
    return e;
  for (int q = 0; q < P; ++q) {
    const int shift = 16 * q;
    timer_begin(a.timer, "k_count16", st);
    k_count16<K><<<(unsigned)(2 * nblocks), kCountThreads, count_smem, st>>>(
        static_cast<const K*>(a.keys), static_cast<const K*>(a.alt_keys), a.skip, q, a.n, shift,
        counts);
    timer_end(a.timer, st);
    timer_begin(a.timer, "k_colscan16", st);
    k_colscan16<<<kR16 / 256, 256, 0, st>>>(counts, nblocks, total);
    timer_end(a.timer, st);
    timer_begin(a.timer, "k_digscan16", st);
    k_digscan16<<<1, 1024, 0, st>>>(total, base, a.skip, q, a.n);
    timer_end(a.timer, st);
    timer_begin(a.timer, "k_scatter16", st);
    k_scatter16<K, V><<<(unsigned)nblocks, kScatterThreads, sc_smem, st>>>(
        static_cast<K*>(a.keys), static_cast<K*>(a.alt_keys), static_cast<V*>(a.vals),
        static_cast<V*>(a.alt_vals), a.skip, q, a.n, shift, counts, base, a.err);
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

template <typename K, typename V>
constexpr LsdEntry r16_entry() {
  return LsdEntry{(int)(8 * sizeof(K)),
                  HasVal<V>::value ? (int)(8 * sizeof(V)) : 0,
                  16,
                  kScatterThreads,
                  kScatterKpt,
                  kBlockKeys,          // "tile" = one count-matrix row
                  kR16,
                  (int)(8 * sizeof(K)) / 16,
                  (size_t)kR16,        // the count matrix: one row per block
                  1,                   // in one buffer
                  &r16_launch<K, V>,
                  1};
}

static const LsdEntry kR16None32[] = {r16_entry<uint32_t, NoVal>()};
static const LsdEntry kR16V32_32[] = {r16_entry<uint32_t, uint32_t>()};
static const LsdEntry kR16V64_32[] = {r16_entry<uint32_t, uint64_t>()};
static const LsdEntry kR16None64[] = {r16_entry<uint64_t, NoVal>()};
static const LsdEntry kR16V32_64[] = {r16_entry<uint64_t, uint32_t>()};
static const LsdEntry kR16V64_64[] = {r16_entry<uint64_t, uint64_t>()};

int r16_variants(int key_bits, int val_bits, const LsdEntry** out) {
  const LsdEntry* t = nullptr;
  if (key_bits == 32) t = val_bits == 0 ? kR16None32 : val_bits == 32 ? kR16V32_32 : kR16V64_32;
  if (key_bits == 64) t = val_bits == 0 ? kR16None64 : val_bits == 32 ? kR16V32_64 : kR16V64_64;
  if (!t || (val_bits != 0 && val_bits != 32 && val_bits != 64)) return 0;
  *out = t;
  return 1;
}

}  // namespace isort
