// GSD on one GPU: the paper's deterministic regular-oversampling sort
// (Algorithm 1, Section "Oversampling algorithms: GSD, GVR, GER"; Theorem 1).
//
//   1. LocalSorting: the input is split into p sequences of about n/p keys,
//      each sorted (the segmented sort; api.cu launches it).
//   2. Sample Selection (k_gsd_sample): from each sorted sequence X_k the r*p
//      keys that end its r*p evenly sized segments (the last one is the
//      maximum); all r*p*p sampled keys sorted with the BTN network.
//   3. Splitter Selection: the (i*s)-th smallest sampled keys, s = r*p,
//      1 <= i <= p - 1.
//   4. Split (k_gsd_bounds, k_gsd_plan): X_k's part for bucket j holds its keys
//      above splitter j-1 and at most splitter j (binary searches in X_k).
//   5. Merging: the p parts of every bucket are merged in lg p rounds of
//      pairwise stable merges (k_gsd_round, k_gsd_merge: merge-path
//      partitioning, one output tile per CTA); the first round reads the parts
//      where the local sort left them, so it also gathers each bucket.
// p is a power of two; equal keys keep input order (sequence k before k+1 in
// every merge, each sequence sorted stably), so payloads sort stably.
#include <algorithm>

#include "btn.cuh"
#include "isort_internal.h"

namespace isort {
namespace {

constexpr int kSampleThreads = 256;
constexpr int kSampleItems = 16;  // r*p*p <= 4096 sampled keys
constexpr int kMergeThreads = 256;

// Output keys per merge CTA: ITEMS per thread, odd so that a warp's merge
// reads and writes (stride ITEMS) spread over all 32 banks. 4-byte keys alone
// take 31 (each thread's merge-path search shared by more outputs; 15, 23 and
// 47 measured slower); wider items 15 or 11, as many as the staged tile
// (keys and payloads) allows within 48 KB of static shared memory.
template <typename K, typename V>
struct MergeShape {
  static constexpr int BYTES = (int)sizeof(K) + (HasVal<V>::value ? (int)sizeof(V) : 0);
  static constexpr int ITEMS = BYTES <= 4 ? 31 : BYTES <= 12 ? 15 : 11;
  static constexpr int TILE = kMergeThreads * ITEMS;
  static_assert(ITEMS % 2 == 1, "odd items per thread");
  static_assert((size_t)TILE * BYTES <= 48 * 1024, "static shared memory");
  static_assert(TILE >= kGsdMinMergeTile, "the workspace sizes one cut per kGsdMinMergeTile keys");
};

__device__ __forceinline__ int64_t seq_start(int64_t n, int p, int k) { return n * k / p; }

// Sample item m = k * (r*p) + i (i = 0 .. r*p - 1) of sorted sequence X_k: the
// last key of segment i + 1 of the r*p evenly sized segments, i.e. position
// floor((i+1) * |X_k| / (r*p)) - 1 of X_k (clamped to its first key); an
// empty sequence contributes copies of the largest key value.
template <typename K>
__global__ void __launch_bounds__(kSampleThreads)
    k_gsd_sample(const K* __restrict__ keys, int64_t n, int p, int rp, K* __restrict__ split) {
  constexpr int Q = kSampleThreads, M = kSampleItems;
  __shared__ K sk[M * Q];
  const int t = threadIdx.x;
  const int ns = rp * p;  // sampled keys in all
  BtnItem<K, false> x[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int m = i * Q + t;
    K v = ~K(0);  // padding (and empty sequences) sort last
    if (m < ns) {
      const int k = m / rp, seg = m % rp;
      const int64_t a = seq_start(n, p, k), len = seq_start(n, p, k + 1) - a;
      if (len > 0) {
        int64_t pos = (int64_t)(seg + 1) * len / rp - 1;
        if (pos < 0) pos = 0;
        v = keys[a + pos];
      }
    }
    x[i].k = v;
  }
  btn_local_sort<false>(x);
  btn_network<false, K, M, Q>(x, t, sk, nullptr);
  // thread t holds sorted ranks [t*M, t*M + M); splitter j (1-based) = rank j*s - 1, s = rp
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int r = t * M + i;
    if ((r + 1) % rp == 0) {
      const int j = (r + 1) / rp;
      if (j >= 1 && j <= p - 1) split[j - 1] = x[i].k;
    }
  }
}

// bound[k][j], j = 0..p: the end (relative to X_k) of X_k's part for buckets
// < j: 0, then the number of keys of X_k at most splitter j, then |X_k|.
// One CTA per sequence; thread j - 1 searches for splitter j.
template <typename K>
__global__ void __launch_bounds__(256) k_gsd_bounds(const K* __restrict__ keys, int64_t n, int p,
                                                    const K* __restrict__ split,
                                                    int64_t* __restrict__ bound) {
  const int k = blockIdx.x;
  const int64_t a = seq_start(n, p, k), len = seq_start(n, p, k + 1) - a;
  int64_t* row = bound + (size_t)k * (p + 1);
  for (int j = threadIdx.x; j <= p; j += 256) {
    if (j == 0) {
      row[0] = 0;
    } else if (j == p) {
      row[p] = len;
    } else {
      const K s = split[j - 1];
      int64_t lo = 0, hi = len;  // first position whose key is above s
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[a + mid] <= s)
          lo = mid + 1;
        else
          hi = mid;
      }
      row[j] = lo;
    }
  }
}

// One CTA: part sizes c[k][j], bucket sizes and offsets, and pre[j][k] = the
// offset of part (k, j) inside bucket j (the sum of c[k'][j] for k' < k).
__global__ void __launch_bounds__(256) k_gsd_plan(const int64_t* __restrict__ bound, int p,
                                                  int64_t* __restrict__ pre,
                                                  int64_t* __restrict__ bucket_off,
                                                  uint32_t* __restrict__ counts_out) {
  __shared__ int64_t s_tot[256];
  const int j = threadIdx.x;
  if (j < p) {
    int64_t run = 0;
    for (int k = 0; k < p; ++k) {
      pre[(size_t)j * (p + 1) + k] = run;
      run += bound[(size_t)k * (p + 1) + j + 1] - bound[(size_t)k * (p + 1) + j];
    }
    pre[(size_t)j * (p + 1) + p] = run;
    s_tot[j] = run;
    if (counts_out) counts_out[j] = (uint32_t)run;
  }
  __syncthreads();
  if (j == 0) {
    int64_t o = 0;
    for (int b = 0; b < p; ++b) {
      bucket_off[b] = o;
      o += s_tot[b];
    }
    bucket_off[p] = o;
  }
}

// Merge round t (runs of 2^(t-1) parts -> runs of 2^t parts). Pair (j, q)
// merges runs 2q and 2q+1 of bucket j. Round 1 reads part (k, j) at
// seq_start(k) + bound[k][j] (the local-sort layout); later rounds read runs
// at bucket_off[j] + pre[j][k]. Writes pair_*: A start/len, B start/len,
// output start, and the exclusive prefix of the pairs' tile counts.
__global__ void __launch_bounds__(256) k_gsd_round(const int64_t* __restrict__ bound,
                                                   const int64_t* __restrict__ pre,
                                                   const int64_t* __restrict__ bucket_off,
                                                   int64_t n, int p, int t, int64_t tile_keys,
                                                   int64_t* __restrict__ pair_info,
                                                   int64_t* __restrict__ pair_tile) {
  const int per = 1 << t;                 // parts per output run
  const int runs = p / per;               // output runs per bucket
  const int pairs = p * runs;
  __shared__ int64_t s_tiles[4096];
  for (int id = threadIdx.x; id < pairs; id += 256) {
    const int j = id / runs, q = id % runs;
    const int ka = q * per, kb = ka + per / 2;  // first parts of the two input runs
    const int64_t* P = pre + (size_t)j * (p + 1);
    const int64_t la = P[kb] - P[ka], lb = P[ka + per] - P[kb];
    int64_t sa, sb;
    if (t == 1) {
      sa = seq_start(n, p, ka) + bound[(size_t)ka * (p + 1) + j];
      sb = seq_start(n, p, kb) + bound[(size_t)kb * (p + 1) + j];
    } else {
      sa = bucket_off[j] + P[ka];
      sb = bucket_off[j] + P[kb];
    }
    int64_t* info = pair_info + (size_t)id * 5;
    info[0] = sa;
    info[1] = la;
    info[2] = sb;
    info[3] = lb;
    info[4] = bucket_off[j] + P[ka];
    s_tiles[id] = (la + lb + tile_keys - 1) / tile_keys;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int id = 0; id < pairs; ++id) {
      pair_tile[id] = run;
      run += s_tiles[id];
    }
    pair_tile[pairs] = run;
  }
}

// Merge-path split of diagonal d of A (la keys) and B (lb keys): the number
// of A keys among the first d of the stable merge (A first on equal keys).
template <typename K, typename GA, typename GB>
__device__ __forceinline__ int64_t merge_split(GA a_at, GB b_at, int64_t la, int64_t lb,
                                               int64_t d) {
  int64_t lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a_at(mid) <= b_at(d - mid - 1))
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// The pair of output tile `tile`: the last id with pair_tile[id] <= tile.
__device__ __forceinline__ int pair_of(const int64_t* __restrict__ pair_tile, int pairs,
                                       int64_t tile) {
  int lo = 0, hi = pairs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pair_tile[mid] <= tile)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// cut[t] = the merge-path split (A keys before the tile) of output tile t's
// first diagonal; one thread per tile, so the searches run side by side
// instead of at the start of every merge CTA.
template <typename K>
__global__ void __launch_bounds__(256) k_gsd_cuts(const K* __restrict__ kin,
                                                  const int64_t* __restrict__ pair_info,
                                                  const int64_t* __restrict__ pair_tile,
                                                  int pairs, int64_t tile_keys,
                                                  int64_t* __restrict__ cut) {
  const int64_t tile = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tile >= pair_tile[pairs]) return;
  const int q = pair_of(pair_tile, pairs, tile);
  const int64_t* info = pair_info + (size_t)q * 5;
  const int64_t sa = info[0], la = info[1], sb = info[2], lb = info[3];
  const int64_t d0 = (tile - pair_tile[q]) * tile_keys;
  cut[tile] = merge_split<K>([&](int64_t i) { return kin[sa + i]; },
                             [&](int64_t i) { return kin[sb + i]; }, la, lb, d0);
}

template <typename K, typename V>
__global__ void __launch_bounds__(kMergeThreads)
    k_gsd_merge(const K* __restrict__ kin, K* __restrict__ kout, const V* __restrict__ vin,
                V* __restrict__ vout, const int64_t* __restrict__ pair_info,
                const int64_t* __restrict__ pair_tile, const int64_t* __restrict__ cut,
                int pairs, int64_t n, uint32_t* err) {
  constexpr bool HV = HasVal<V>::value;
  constexpr int kMergeItems = MergeShape<K, V>::ITEMS, kMergeTile = MergeShape<K, V>::TILE;
  using VS = typename std::conditional<HV, V, uint32_t>::type;
  __shared__ K s_k[kMergeTile];                // staged A then B, later the merged tile
  __shared__ VS s_v[HV ? kMergeTile : 1];
  const int64_t tile = blockIdx.x;
  if (tile >= pair_tile[pairs]) return;
  const int q = pair_of(pair_tile, pairs, tile);
  const int64_t* info = pair_info + (size_t)q * 5;
  const int64_t sa = info[0], la = info[1], sb = info[2], lb = info[3], so = info[4];
  const int64_t d0 = (tile - pair_tile[q]) * kMergeTile;
  const int64_t d1 = min(d0 + kMergeTile, la + lb);
  const bool last = tile + 1 == pair_tile[q + 1];  // the pair's last tile ends at la, lb
  const int64_t a0 = cut[tile], a1 = last ? la : cut[tile + 1];
  const int64_t b0 = d0 - a0, b1 = d1 - a1;
  const int na = (int)(a1 - a0), nb = (int)(b1 - b0), nt = na + nb;
  for (int i = threadIdx.x; i < nt; i += kMergeThreads) {  // stage A[a0:a1], then B[b0:b1]
    const int64_t src = i < na ? sa + a0 + i : sb + b0 + (i - na);
    s_k[i] = kin[src];
    if constexpr (HV) s_v[i] = vin[src];
  }
  __syncthreads();
  // each thread merges kMergeItems outputs starting at its own diagonal
  K ok[kMergeItems];
  VS ov[kMergeItems];
  const int dd = threadIdx.x * kMergeItems;
  if (dd < nt) {
    int ia = (int)merge_split<K>([&](int64_t i) { return s_k[i]; },
                                 [&](int64_t i) { return s_k[na + i]; }, na, nb, dd);
    int ib = dd - ia;
    if constexpr (kMergeItems >= 23) {
      // long per-thread merges: the two runs' heads stay in registers, one
      // shared load per output (the consumed run's next key)
      K ka = ia < na ? s_k[ia] : K(0), kb = ib < nb ? s_k[na + ib] : K(0);
#pragma unroll
      for (int o = 0; o < kMergeItems; ++o) {
        if (dd + o < nt) {
          const bool take_a = ib >= nb || (ia < na && ka <= kb);
          ok[o] = take_a ? ka : kb;
          if constexpr (HV) ov[o] = s_v[take_a ? ia : na + ib];
          if (take_a)
            ++ia;
          else
            ++ib;
          const bool more = take_a ? ia < na : ib < nb;
          const K next = more ? s_k[take_a ? ia : na + ib] : K(0);
          if (take_a)
            ka = next;
          else
            kb = next;
        }
      }
    } else {
      // short ones: both heads re-read each step (measured faster at 15 items)
#pragma unroll
      for (int o = 0; o < kMergeItems; ++o) {
        if (dd + o < nt) {
          const bool take_a = ib >= nb || (ia < na && s_k[ia] <= s_k[na + ib]);
          const int src = take_a ? ia++ : na + ib++;
          ok[o] = s_k[src];
          if constexpr (HV) ov[o] = s_v[src];
        }
      }
    }
  }
  __syncthreads();  // every thread has read the staged tile
#pragma unroll
  for (int o = 0; o < kMergeItems; ++o)
    if (dd + o < nt) {
      s_k[dd + o] = ok[o];
      if constexpr (HV) s_v[dd + o] = ov[o];
    }
  __syncthreads();
  for (int i = threadIdx.x; i < nt; i += kMergeThreads) {  // coalesced write-out
    const int64_t dst = so + d0 + i;
    if (dst < n) {
      kout[dst] = s_k[i];
      if constexpr (HV) vout[dst] = s_v[i];
    } else {
      atomicOr(err, kErrBounds);
    }
  }
}

template <typename K, typename V>
cudaError_t gsd_launch(const GsdArgs& a, cudaStream_t st) {
  const int p = a.buckets;
  K* keys = static_cast<K*>(a.keys);
  V* vals = static_cast<V*>(a.vals);
  K* split = static_cast<K*>(a.split);
  timer_begin(a.timer, "k_gsd_sample", st);
  k_gsd_sample<K><<<1, kSampleThreads, 0, st>>>(keys, a.n, p, a.oversample * p, split);
  timer_end(a.timer, st);
  timer_begin(a.timer, "k_gsd_bounds", st);
  k_gsd_bounds<K><<<p, 256, 0, st>>>(keys, a.n, p, split, a.bound);
  timer_end(a.timer, st);
  timer_begin(a.timer, "k_gsd_plan", st);
  k_gsd_plan<<<1, 256, 0, st>>>(a.bound, p, a.pre, a.bucket_off, a.counts_out);
  timer_end(a.timer, st);
  // lg p merge rounds, ping-pong between the caller's arrays and the workspace
  constexpr int64_t kTile = MergeShape<K, V>::TILE;
  const int64_t max_tiles = a.n / kTile + (int64_t)p * p + 1;
  K* kbuf[2] = {keys, static_cast<K*>(a.alt_keys)};
  V* vbuf[2] = {vals, static_cast<V*>(a.alt_vals)};
  int src = 0;
  for (int t = 1; (1 << t) <= p; ++t) {
    const int pairs = p * (p >> t);
    timer_begin(a.timer, "k_gsd_round", st);
    k_gsd_round<<<1, 256, 0, st>>>(a.bound, a.pre, a.bucket_off, a.n, p, t, kTile, a.pair_info,
                                   a.pair_tile);
    timer_end(a.timer, st);
    timer_begin(a.timer, "k_gsd_cuts", st);
    k_gsd_cuts<K><<<(unsigned)((max_tiles + 255) / 256), 256, 0, st>>>(
        kbuf[src], a.pair_info, a.pair_tile, pairs, kTile, a.cut);
    timer_end(a.timer, st);
    timer_begin(a.timer, "k_gsd_merge", st);
    k_gsd_merge<K, V><<<(unsigned)max_tiles, kMergeThreads, 0, st>>>(
        kbuf[src], kbuf[src ^ 1], vbuf[src], vbuf[src ^ 1], a.pair_info, a.pair_tile, a.cut,
        pairs, a.n, a.err);
    timer_end(a.timer, st);
    src ^= 1;
  }
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  if (src) {  // an odd number of rounds: the result is in the workspace
    if ((e = cudaMemcpyAsync(keys, kbuf[1], sizeof(K) * (size_t)a.n, cudaMemcpyDeviceToDevice,
                             st)))
      return e;
    if constexpr (HasVal<V>::value)
      if ((e = cudaMemcpyAsync(vals, vbuf[1], sizeof(V) * (size_t)a.n, cudaMemcpyDeviceToDevice,
                               st)))
        return e;
  }
  return cudaSuccess;
}

// off[k] = n*k/p, k = 0..p: the p sequences of the local sort.
__global__ void k_gsd_offsets(int64_t n, int p, int64_t* __restrict__ off) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k <= p) off[k] = seq_start(n, p, k);
}

}  // namespace

cudaError_t gsd_offsets_launch(int64_t n, int p, int64_t* off, cudaStream_t st) {
  k_gsd_offsets<<<(p + 256) / 256, 256, 0, st>>>(n, p, off);
  return cudaGetLastError();
}

cudaError_t gsd_merge_launch(int key_bits, int val_bits, const GsdArgs& a, cudaStream_t st) {
  if (key_bits == 32) {
    if (val_bits == 0) return gsd_launch<uint32_t, NoVal>(a, st);
    if (val_bits == 32) return gsd_launch<uint32_t, uint32_t>(a, st);
    return gsd_launch<uint32_t, uint64_t>(a, st);
  }
  if (val_bits == 0) return gsd_launch<uint64_t, NoVal>(a, st);
  if (val_bits == 32) return gsd_launch<uint64_t, uint32_t>(a, st);
  return gsd_launch<uint64_t, uint64_t>(a, st);
}

}  // namespace isort
