// BTN: the paper's p-processor bitonic merge-split sort ("Algorithm BTN",
// Section "Related work", cost Eq. Tb), with GPU threads as the processors.
//
// Each of q threads holds a run of M items that it sorts locally first (the
// paper sorts locally with SR4; here a register sorting network, the paper
// leaves the local method open). Then lg q (lg q + 1) / 2 stages of a
// q-"key" bitonic sorting network run over the runs, where a comparator
// between threads t < u is a merge-split: both merge their two sorted runs and
// the lower-indexed thread keeps the M smallest (ascending comparator) or the
// M largest (descending comparator), the other thread the rest. Afterwards the
// runs, concatenated in thread order, are the sorted sequence.
//
// Merge-split of two ascending runs A (mine) and B (partner's): the sequence
// min(A[i], B[M-1-i]) holds the M smallest items and is bitonic, the sequence
// max(A[i], B[M-1-i]) the M largest; a bitonic half-cleaner cascade sorts it.
//
// BTN by itself is not stable (the paper notes this). Items here compare as
// (key, index in the segment), which makes the result the unique stable order;
// for keys-only sorts equal keys are indistinguishable and the index is omitted.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace isort {

template <typename K, bool STABLE>
struct BtnItem {
  K k;
  uint32_t i;
};

template <bool STABLE, typename K>
__device__ __forceinline__ bool btn_less(const BtnItem<K, STABLE>& a, const BtnItem<K, STABLE>& b) {
  if constexpr (STABLE)
    return a.k < b.k || (a.k == b.k && a.i < b.i);
  else
    return a.k < b.k;
}

template <bool STABLE, typename K>
__device__ __forceinline__ void btn_cas(BtnItem<K, STABLE>& a, BtnItem<K, STABLE>& b) {
  // order the pair ascending
  if (btn_less<STABLE>(b, a)) {
    BtnItem<K, STABLE> t = a;
    a = b;
    b = t;
  }
}

// Sort M items in registers ascending (bitonic sorting network).
template <bool STABLE, typename K, int M>
__device__ __forceinline__ void btn_local_sort(BtnItem<K, STABLE> (&x)[M]) {
#pragma unroll
  for (int k = 2; k <= M; k <<= 1)
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
      for (int i = 0; i < M; ++i) {
        const int l = i ^ j;
        if (l > i) {
          if ((i & k) == 0)
            btn_cas<STABLE>(x[i], x[l]);
          else
            btn_cas<STABLE>(x[l], x[i]);
        }
      }
}

// Turn a bitonic sequence of M items into an ascending one (half-cleaners).
template <bool STABLE, typename K, int M>
__device__ __forceinline__ void btn_bitonic_clean(BtnItem<K, STABLE> (&x)[M]) {
#pragma unroll
  for (int j = M >> 1; j > 0; j >>= 1)
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const int l = i ^ j;
      if (l > i) btn_cas<STABLE>(x[i], x[l]);
    }
}

// Merge-split with the partner's run b (ascending): keep the low or high half.
template <bool STABLE, typename K, int M>
__device__ __forceinline__ void btn_merge_split(BtnItem<K, STABLE> (&x)[M],
                                                const BtnItem<K, STABLE> (&b)[M], bool keep_low) {
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const BtnItem<K, STABLE>& o = b[M - 1 - i];
    const bool take = keep_low ? btn_less<STABLE>(o, x[i]) : btn_less<STABLE>(x[i], o);
    if (take) x[i] = o;
  }
  btn_bitonic_clean<STABLE>(x);
}

// Exchange a run with lane (lane ^ j) of the same warp.
template <bool STABLE, typename K, int M>
__device__ __forceinline__ void btn_shfl_run(const BtnItem<K, STABLE> (&x)[M],
                                             BtnItem<K, STABLE> (&b)[M], int j) {
#pragma unroll
  for (int i = 0; i < M; ++i) {
    b[i].k = __shfl_xor_sync(kFullMask, x[i].k, j);
    if constexpr (STABLE) b[i].i = __shfl_xor_sync(kFullMask, x[i].i, j);
  }
}

// The merge-split network over q = Q threads (thread index t in [0, Q)).
// Partners within a warp exchange through shuffles; farther partners through
// the shared buffers sk/si ([M][Q] each, item i of thread t at i*Q + t).
// Contains __syncthreads when Q > 32 (all Q threads must call it).
template <bool STABLE, typename K, int M, int Q>
__device__ __forceinline__ void btn_network(BtnItem<K, STABLE> (&x)[M], int t, K* sk,
                                            uint32_t* si) {
  BtnItem<K, STABLE> b[M];
#pragma unroll 1
  for (int k = 2; k <= Q; k <<= 1) {
#pragma unroll 1
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int u = t ^ j;
      const bool asc = (t & k) == 0;
      const bool keep_low = asc == (t < u);
      if (j < 32) {
        btn_shfl_run<STABLE>(x, b, j);
      } else {
#pragma unroll
        for (int i = 0; i < M; ++i) {
          sk[i * Q + t] = x[i].k;
          if constexpr (STABLE) si[i * Q + t] = x[i].i;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < M; ++i) {
          b[i].k = sk[i * Q + u];
          if constexpr (STABLE) b[i].i = si[i * Q + u];
        }
        __syncthreads();
      }
      btn_merge_split<STABLE>(x, b, keep_low);
    }
  }
}

// OET: the paper's p-wide odd-even transposition sort ("Algorithm OET",
// Section "Related work", cost Eq. To) over the same runs. Q rounds; in an
// even round threads (2i, 2i+1) merge-split, in an odd round (2i+1, 2i+2); the
// lower-indexed thread of a pair keeps the M smallest items. After Q rounds
// the runs, concatenated in thread order, are sorted (odd-even transposition
// sorts Q "keys" in Q rounds, and a merge-split is a comparator on runs).
// Partners are neighbours: even rounds stay within a warp (shuffles); odd
// rounds cross warp boundaries when Q > 32 and then go through sk/si.
// Contains __syncthreads when Q > 32 (all Q threads must call it).
template <bool STABLE, typename K, int M, int Q>
__device__ __forceinline__ void oet_network(BtnItem<K, STABLE> (&x)[M], int t, K* sk,
                                            uint32_t* si) {
  BtnItem<K, STABLE> b[M];
  const int lane = t & 31;
#pragma unroll 1
  for (int r = 0; r < Q; ++r) {
    const bool odd = r & 1;
    // partner: t ^ 1 in even rounds; t + 1 (t odd) or t - 1 (t even) in odd rounds
    const int u = odd ? ((t & 1) ? t + 1 : t - 1) : (t ^ 1);
    const bool active = u >= 0 && u < Q;
    if (!odd || Q == 32) {
      // within the warp: lane u & 31 (idle lanes read something and ignore it)
      const int src = active ? (u & 31) : lane;
#pragma unroll
      for (int i = 0; i < M; ++i) {
        b[i].k = __shfl_sync(kFullMask, x[i].k, src);
        if constexpr (STABLE) b[i].i = __shfl_sync(kFullMask, x[i].i, src);
      }
    } else {
#pragma unroll
      for (int i = 0; i < M; ++i) {
        sk[i * Q + t] = x[i].k;
        if constexpr (STABLE) si[i * Q + t] = x[i].i;
      }
      __syncthreads();
      if (active) {
#pragma unroll
        for (int i = 0; i < M; ++i) {
          b[i].k = sk[i * Q + u];
          if constexpr (STABLE) b[i].i = si[i * Q + u];
        }
      }
      __syncthreads();
    }
    if (active) btn_merge_split<STABLE>(x, b, t < u);
  }
}

}  // namespace isort
