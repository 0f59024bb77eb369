/*
 * Oracle: a plain, slow, serial LSD radix sort of unsigned integer keys.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. The GPU sort library shares no code,
 * header, table or helper with it, and neither calls the other.
 *
 * What it computes (the plain definition): the ascending order of the input
 * keys; with payloads, the STABLE ascending order (equal keys keep their input
 * order and every payload moves with its key); for a segmented sort, the same
 * on each [offsets[i], offsets[i+1]) independently. Radix sort reaches exactly
 * this result, which is unique, so any correct sort agrees with it bit for bit.
 *
 * How: the paper's serial radix sort SR4 (Section "SR4, PR2, PR4, BTN and OET
 * under MBSP", Eq. Ts): rounds of count-sort, one per r-ary digit, least
 * significant digit first (the CLRS RADIX-SORT/COUNTING-SORT pair the paper
 * cites). Each round
 *   1. allocates and zeroes a count array of r counters,
 *   2. reads the input once, counting each key's digit,
 *   3. turns the counts into exclusive prefix sums (first output slot per digit),
 *   4. reads the input a second time, in ascending index order, writing each key
 *      (and its payload) to the next free slot of its digit -- one output write.
 * Reading the input twice and writing once is the paper's 3N main-memory words
 * per round. The rounds ping-pong between the array and a scratch copy; after an
 * odd number of rounds the result is copied back.
 *
 * Digit p of key k is (k >> (p*b)) & (2^b - 1); when b does not divide the key
 * width the last digit is narrower (e.g. 11, 11, 10 bits for b = 11 on 32-bit
 * keys). Readings where the paper is silent: LSD order, unsigned keys, forward
 * output loop with exclusive prefix (CLRS loops backwards with inclusive counts;
 * both are stable and give the same array).
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

static uint64_t get_key(const void *a, int64_t i, int key_bytes) {
  if (key_bytes == 4) return ((const uint32_t *)a)[i];
  return ((const uint64_t *)a)[i];
}

static void put_key(void *a, int64_t i, uint64_t k, int key_bytes) {
  if (key_bytes == 4)
    ((uint32_t *)a)[i] = (uint32_t)k;
  else
    ((uint64_t *)a)[i] = k;
}

static void copy_val(void *dst, int64_t j, const void *src, int64_t i, int val_bytes) {
  if (val_bytes == 4)
    ((uint32_t *)dst)[j] = ((const uint32_t *)src)[i];
  else if (val_bytes == 8)
    ((uint64_t *)dst)[j] = ((const uint64_t *)src)[i];
}

int oracle_count_sort_round(const void *keys_in, void *keys_out, const void *vals_in,
                            void *vals_out, int64_t n, int key_bits, int val_bits, int shift,
                            int digit_bits) {
  if (n < 0 || (key_bits != 32 && key_bits != 64) ||
      (val_bits != 0 && val_bits != 32 && val_bits != 64) || digit_bits < 1 ||
      digit_bits > 24 || shift < 0 || shift + digit_bits > key_bits)
    return 1;
  const int kb = key_bits / 8, vb = val_bits / 8;
  const int64_t r = (int64_t)1 << digit_bits;
  const uint64_t mask = (uint64_t)r - 1;

  /* 1. count array of r counters, zeroed */
  int64_t *count = (int64_t *)calloc((size_t)r, sizeof(int64_t));
  if (!count) return 2;

  /* 2. first read of the input: count digits */
  for (int64_t i = 0; i < n; ++i) count[(get_key(keys_in, i, kb) >> shift) & mask]++;

  /* 3. exclusive prefix sums: count[d] becomes the first output slot of digit d */
  int64_t sum = 0;
  for (int64_t d = 0; d < r; ++d) {
    int64_t c = count[d];
    count[d] = sum;
    sum += c;
  }

  /* 4. second read, ascending index order: stable placement, one output write */
  for (int64_t i = 0; i < n; ++i) {
    uint64_t k = get_key(keys_in, i, kb);
    int64_t pos = count[(k >> shift) & mask]++;
    put_key(keys_out, pos, k, kb);
    if (vb) copy_val(vals_out, pos, vals_in, i, vb);
  }
  free(count);
  return 0;
}

int oracle_num_passes(int key_bits, int radix_bits) {
  return (key_bits + radix_bits - 1) / radix_bits;
}

int oracle_radix_sort(void *keys, void *vals, int64_t n, int key_bits, int val_bits,
                      int radix_bits) {
  if (n < 0 || (key_bits != 32 && key_bits != 64) ||
      (val_bits != 0 && val_bits != 32 && val_bits != 64) || radix_bits < 1 || radix_bits > 24 ||
      (n > 0 && !keys) || (n > 0 && val_bits && !vals))
    return 1;
  if (n <= 1) return 0;
  const int kb = key_bits / 8, vb = val_bits / 8;
  void *kscratch = malloc((size_t)n * kb);
  void *vscratch = vb ? malloc((size_t)n * vb) : NULL;
  if (!kscratch || (vb && !vscratch)) {
    free(kscratch);
    free(vscratch);
    return 2;
  }
  void *kin = keys, *kout = kscratch, *vin = vals, *vout = vscratch;
  const int passes = oracle_num_passes(key_bits, radix_bits);
  int rc = 0;
  for (int p = 0; p < passes && rc == 0; ++p) {
    int shift = p * radix_bits;
    int bits = key_bits - shift < radix_bits ? key_bits - shift : radix_bits;
    rc = oracle_count_sort_round(kin, kout, vin, vout, n, key_bits, val_bits, shift, bits);
    void *t = kin; kin = kout; kout = t;   /* swap in/out */
    t = vin; vin = vout; vout = t;
  }
  if (rc == 0 && kin != keys) { /* odd number of rounds: copy the result back */
    memcpy(keys, kin, (size_t)n * kb);
    if (vb) memcpy(vals, vin, (size_t)n * vb);
  }
  free(kscratch);
  free(vscratch);
  return rc;
}

int oracle_segmented_sort(void *keys, void *vals, const int64_t *offsets, int64_t num_segments,
                          int key_bits, int val_bits, int radix_bits) {
  if (num_segments < 0 || (num_segments > 0 && !offsets)) return 1;
  if (key_bits != 32 && key_bits != 64) return 1;
  if (num_segments > 0 && offsets[0] != 0) return 1;
  for (int64_t s = 0; s < num_segments; ++s)
    if (offsets[s + 1] < offsets[s]) return 1;
  const int kb = key_bits / 8, vb = val_bits / 8;
  for (int64_t s = 0; s < num_segments; ++s) {
    int64_t lo = offsets[s], len = offsets[s + 1] - offsets[s];
    int rc = oracle_radix_sort((char *)keys + lo * kb, vb ? (char *)vals + lo * vb : NULL, len,
                               key_bits, val_bits, radix_bits);
    if (rc) return rc;
  }
  return 0;
}

/* ------------------------------------------------------------------------
 * GVR, the paper's random-oversampling sample sort (Algorithm 3, Section
 * "Oversampling algorithms: GSD, GVR, GER"), serially, in the algorithm's order:
 *   1. Sample Selection: s*p - 1 keys at random positions, sorted;
 *   2. Splitter Selection: the (i*s)-th smallest sampled keys, 1 <= i <= p-1;
 *   3. Split input keys: each key's destination j = the number of splitters
 *      smaller than it, then a count-sort by j (stable), so every key moves once;
 *   4. LocalSorting: each destination sequence sorted by SR4 (radix 256).
 * Random positions: SplitMix64 (Steele, Lea & Flood 2014), stream 30 of the
 * seed: S = mix(seed*G ^ 30*C), draw m = mix(S + (m+1)*G), position = high 32
 * bits of the draw times n, shifted right 32. Sorting the sample uses the C
 * library's qsort (the paper sorts it with BTN; the sorted sample is the same).
 */
static uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static int cmp_u64(const void *a, const void *b) {
  const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return (x > y) - (x < y);
}

int oracle_gvr_sort(void *keys, void *vals, int64_t n, int key_bits, int val_bits, int p, int s,
                    uint64_t seed, uint32_t *bucket_counts, uint64_t *splitters) {
  if (n < 0 || (key_bits != 32 && key_bits != 64) ||
      (val_bits != 0 && val_bits != 32 && val_bits != 64) || p < 1 || s < 1)
    return 1;
  const int kb = key_bits / 8, vb = val_bits / 8;
  const int64_t ns = (int64_t)s * p - 1;
  uint64_t *sample = malloc(sizeof(uint64_t) * (size_t)(ns > 0 ? ns : 1));
  uint64_t *split = malloc(sizeof(uint64_t) * (size_t)(p > 1 ? p - 1 : 1));
  int64_t *count = calloc((size_t)p + 1, sizeof(int64_t));
  uint32_t *dest = malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  void *kout = malloc((size_t)(n > 0 ? n : 1) * kb);
  void *vout = vb ? malloc((size_t)(n > 0 ? n : 1) * vb) : NULL;
  int rc = 0;
  if (!sample || !split || !count || !dest || !kout || (vb && !vout)) {
    rc = 2;
    goto done;
  }
  /* 1. Sample Selection */
  if (n > 0) {
    const uint64_t G = 0x9E3779B97F4A7C15ull, C = 0xD1B54A32D192ED03ull;
    const uint64_t S = sm64_mix(seed * G ^ 30ull * C);
    for (int64_t m = 0; m < ns; ++m) {
      const uint64_t d = sm64_mix(S + (uint64_t)(m + 1) * G);
      const int64_t pos = (int64_t)(((d >> 32) * (uint64_t)n) >> 32);
      sample[m] = get_key(keys, pos, kb);
    }
    qsort(sample, (size_t)ns, sizeof(uint64_t), cmp_u64);
  }
  /* 2. Splitter Selection: split[i-1] = the (i*s)-th smallest, 1 <= i <= p-1 */
  for (int i = 1; i <= p - 1; ++i) split[i - 1] = n > 0 ? sample[(int64_t)i * s - 1] : 0;
  /* 3. Split input keys: destinations, their counts, then the count-sort by destination */
  for (int64_t i = 0; i < n; ++i) {
    const uint64_t k = get_key(keys, i, kb);
    uint32_t j = 0;
    while ((int)j < p - 1 && split[j] < k) ++j;  /* splitters ascending: count those below k */
    dest[i] = j;
    ++count[j + 1];
  }
  for (int j = 0; j < p; ++j) count[j + 1] += count[j]; /* count[j] = first slot of j */
  {
    int64_t *next = malloc(sizeof(int64_t) * (size_t)p);
    if (!next) {
      rc = 2;
      goto done;
    }
    memcpy(next, count, sizeof(int64_t) * (size_t)p);
    for (int64_t i = 0; i < n; ++i) {
      const int64_t o = next[dest[i]]++;
      put_key(kout, o, get_key(keys, i, kb), kb);
      if (vb) copy_val(vout, o, vals, i, vb);
    }
    free(next);
  }
  /* 4. LocalSorting of each destination sequence (SR4), then the concatenation */
  rc = oracle_segmented_sort(kout, vout, count, p, key_bits, val_bits, 8);
  if (rc) goto done;
  memcpy(keys, kout, (size_t)n * kb);
  if (vb) memcpy(vals, vout, (size_t)n * vb);
  if (bucket_counts)
    for (int j = 0; j < p; ++j) bucket_counts[j] = (uint32_t)(count[j + 1] - count[j]);
  if (splitters)
    for (int i = 0; i < p - 1; ++i) splitters[i] = split[i];
done:
  free(sample);
  free(split);
  free(count);
  free(dest);
  free(kout);
  free(vout);
  return rc;
}

/* ------------------------------------------------------------------------
 * GSD, the paper's deterministic regular-oversampling sort (Algorithm 1), in
 * the algorithm's order:
 *   1. LocalSorting: sequences [n*k/p, n*(k+1)/p), each sorted by SR4;
 *   2. Sample Selection: from each sorted sequence X_k the r*p keys that end its
 *      r*p evenly sized segments (position floor(i*len/(r*p)) - 1, i = 1..r*p,
 *      the last one its maximum); all r*p*p samples sorted (qsort);
 *   3. Splitter Selection: the (i*r*p)-th smallest samples, 1 <= i <= p-1;
 *   4. Split: part (k, j) of X_k holds its keys above splitter j-1 and at most
 *      splitter j (binary search);
 *   5. Merging: bucket j = the p-way merge of parts (0, j) .. (p-1, j), taking
 *      the smallest head each time (the lowest k on equal keys); the buckets
 *      concatenated.
 * An empty sequence contributes samples equal to the largest key value.
 */
static int64_t count_le(const void *keys, int64_t lo, int64_t hi, uint64_t s, int kb) {
  /* number of keys in the sorted range [lo, hi) that are at most s */
  int64_t a = lo, b = hi;
  while (a < b) {
    const int64_t mid = a + (b - a) / 2;
    if (get_key(keys, mid, kb) <= s)
      a = mid + 1;
    else
      b = mid;
  }
  return a - lo;
}

int oracle_gsd_sort(void *keys, void *vals, int64_t n, int key_bits, int val_bits, int p, int r,
                    uint32_t *bucket_counts, uint64_t *splitters) {
  if (n < 0 || (key_bits != 32 && key_bits != 64) ||
      (val_bits != 0 && val_bits != 32 && val_bits != 64) || p < 1 || r < 1)
    return 1;
  const int kb = key_bits / 8, vb = val_bits / 8;
  const int rp = r * p;
  const uint64_t maxkey = key_bits == 32 ? 0xFFFFFFFFull : ~0ull;
  int64_t *start = malloc(sizeof(int64_t) * (size_t)(p + 1));
  uint64_t *sample = malloc(sizeof(uint64_t) * (size_t)rp * p);
  uint64_t *split = malloc(sizeof(uint64_t) * (size_t)(p > 1 ? p - 1 : 1));
  int64_t *part = malloc(sizeof(int64_t) * (size_t)p * (p + 1)); /* part[k][j]: start in X_k */
  int64_t *head = malloc(sizeof(int64_t) * (size_t)p);
  void *kout = malloc((size_t)(n > 0 ? n : 1) * kb);
  void *vout = vb ? malloc((size_t)(n > 0 ? n : 1) * vb) : NULL;
  int rc = 0;
  if (!start || !sample || !split || !part || !head || !kout || (vb && !vout)) {
    rc = 2;
    goto done;
  }
  /* 1. LocalSorting */
  for (int k = 0; k <= p; ++k) start[k] = n * k / p;
  rc = oracle_segmented_sort(keys, vals, start, p, key_bits, val_bits, 8);
  if (rc) goto done;
  /* 2. Sample Selection */
  for (int k = 0; k < p; ++k) {
    const int64_t len = start[k + 1] - start[k];
    for (int i = 1; i <= rp; ++i) {
      int64_t pos = (int64_t)i * len / rp - 1;
      if (pos < 0) pos = 0;
      sample[(int64_t)k * rp + (i - 1)] = len > 0 ? get_key(keys, start[k] + pos, kb) : maxkey;
    }
  }
  qsort(sample, (size_t)rp * p, sizeof(uint64_t), cmp_u64);
  /* 3. Splitter Selection */
  for (int i = 1; i <= p - 1; ++i) split[i - 1] = sample[(int64_t)i * rp - 1];
  /* 4. Split each sorted sequence */
  for (int k = 0; k < p; ++k) {
    int64_t *row = part + (size_t)k * (p + 1);
    row[0] = 0;
    for (int j = 1; j <= p - 1; ++j)
      row[j] = count_le(keys, start[k], start[k + 1], split[j - 1], kb);
    row[p] = start[k + 1] - start[k];
  }
  /* 5. Merging: p-way merge per bucket, smallest head first, lowest k on ties */
  {
    int64_t o = 0;
    for (int j = 0; j < p; ++j) {
      int64_t size = 0;
      for (int k = 0; k < p; ++k) {
        head[k] = part[(size_t)k * (p + 1) + j];
        size += part[(size_t)k * (p + 1) + j + 1] - head[k];
      }
      if (bucket_counts) bucket_counts[j] = (uint32_t)size;
      for (int64_t m = 0; m < size; ++m) {
        int best = -1;
        uint64_t bk = 0;
        for (int k = 0; k < p; ++k) {
          if (head[k] >= part[(size_t)k * (p + 1) + j + 1]) continue;
          const uint64_t x = get_key(keys, start[k] + head[k], kb);
          if (best < 0 || x < bk) {
            best = k;
            bk = x;
          }
        }
        put_key(kout, o, bk, kb);
        if (vb) copy_val(vout, o, vals, start[best] + head[best], vb);
        ++head[best];
        ++o;
      }
    }
  }
  memcpy(keys, kout, (size_t)n * kb);
  if (vb) memcpy(vals, vout, (size_t)n * vb);
  if (splitters)
    for (int i = 0; i < p - 1; ++i) splitters[i] = split[i];
done:
  free(start);
  free(sample);
  free(split);
  free(part);
  free(head);
  free(kout);
  free(vout);
  return rc;
}
