/*
 * Oracle for the LSD radix sort (serial C). TEST INFRASTRUCTURE ONLY: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * GPU library shares nothing with it.
 *
 * All calls return 0 on success, 1 on bad arguments, 2 when malloc fails.
 * Keys are unsigned, key_bits 32 or 64; payload width val_bits 0 (none), 32 or 64.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One count-sort round (SR4, "first the counting process ... then the output"):
 * stable distribution of keys_in[0..n) by digit (k >> shift) & (2^digit_bits - 1)
 * into keys_out; payloads follow. Input and output must not overlap. */
int oracle_count_sort_round(const void *keys_in, void *keys_out, const void *vals_in,
                            void *vals_out, int64_t n, int key_bits, int val_bits, int shift,
                            int digit_bits);

/* ceil(key_bits / radix_bits): the "32 / lg r" rounds of Eq. Ts. */
int oracle_num_passes(int key_bits, int radix_bits);

/* In-place LSD radix sort with radix 2^radix_bits (1..24), least significant
 * digit first; stable on equal keys when payloads are present. */
int oracle_radix_sort(void *keys, void *vals, int64_t n, int key_bits, int val_bits,
                      int radix_bits);

/* Each [offsets[s], offsets[s+1]) sorted independently (offsets: num_segments+1
 * entries, offsets[0] = 0, non-decreasing). */
int oracle_segmented_sort(void *keys, void *vals, const int64_t *offsets, int64_t num_segments,
                          int key_bits, int val_bits, int radix_bits);

/* GVR sample sort (Algorithm 3): sample s*p - 1 keys at SplitMix64 positions
 * (stream 30 of seed), splitters = the (i*s)-th smallest sampled keys, stable
 * count-sort by destination (number of splitters below the key), SR4 on each
 * destination sequence. Sorts in place; bucket_counts (p entries) and
 * splitters (p - 1 entries) receive the intermediates when not NULL. */
int oracle_gvr_sort(void *keys, void *vals, int64_t n, int key_bits, int val_bits, int p, int s,
                    uint64_t seed, uint32_t *bucket_counts, uint64_t *splitters);

/* GSD (Algorithm 1): p sequences [n*k/p, n*(k+1)/p) sorted by SR4, r*p regular
 * samples per sequence, splitters = the (i*r*p)-th smallest samples, split by
 * binary search (part j: keys above splitter j-1, at most splitter j), p-way
 * merge per bucket (lowest sequence first on equal keys). Sorts in place;
 * bucket_counts (p) and splitters (p - 1) receive the intermediates when not NULL. */
int oracle_gsd_sort(void *keys, void *vals, int64_t n, int key_bits, int val_bits, int p, int r,
                    uint32_t *bucket_counts, uint64_t *splitters);

#ifdef __cplusplus
}
#endif
#endif
