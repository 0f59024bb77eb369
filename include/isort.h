/*
 * isort -- LSD radix sort of unsigned integer keys on one GB300 GPU (sm_103a).
 *
 * The operation is the paper's radix sort (Gerbessiotis, "A study of integer
 * sorting on multicores", arXiv 1808.10292): rounds of stable count-sort, one
 * per r-ary digit, least significant digit first -- SR4 / PR4 with r = 2^8
 * (four rounds on 32-bit keys) and PR2 with r = 2^16 (two rounds), Section
 * "SR4, PR2, PR4, BTN and OET under MBSP", Eqs. Ts, Tp, Tp4, Tp2. Each round is
 * a digit histogram, an exclusive prefix over the digit counts (the paper's
 * p x r count exchange, done here as a single-pass decoupled look-back across
 * GPU tiles), and a stable scatter.
 *
 * The result is the unique stable ascending order of the input: equal keys keep
 * their input order and payloads move with their keys.
 *
 * Conventions for every call:
 *  - keys, vals, offsets are DEVICE pointers owned by the caller (except the
 *    *_host calls, whose buffers are in host memory); the library never frees
 *    caller memory. Sorts are in place (the *_host calls may also write to
 *    separate output buffers).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls are
 *    asynchronous: they validate arguments, enqueue kernels on `stream` and
 *    return. Argument errors are returned at once and enqueue nothing.
 *  - Scratch memory ("workspace") is per stream: either bound by the caller with
 *    isort_set_workspace, or allocated by the library on first use with
 *    stream-ordered cudaMallocAsync and grown as needed.
 *  - Device-side errors (a bounded wait that gave up, an index check that
 *    failed) are latched in the stream's workspace error word and reported by
 *    isort_stream_status.
 *  - Keys are unsigned 32- or 64-bit (key_bits 32|64); payloads 32- or 64-bit
 *    (val_bits 32|64). n <= 2^30 (the look-back status word packs a 30-bit
 *    count); larger n returns ISORT_EUNSUPPORTED.
 *  - radix_bits: 0 = automatic (the width and kernel variant that the autotuner
 *    chose for these key/payload widths and the size bucket floor(log2 n), see
 *    isort_tune_auto; radix 256 when nothing was tuned), 8 = radix 256
 *    (SR4/PR4), 16 = radix 65536 (PR2), 11 = radix 2048 (between the two; not
 *    one of the paper's configurations). Passes = ceil(key_bits / radix_bits);
 *    when radix_bits does not divide key_bits the last digit is narrower (11,
 *    11, 10 bits for 32-bit keys at radix_bits 11). A pass whose digit is the same for every key is
 *    skipped (it is the identity permutation).
 */
#ifndef ISORT_H
#define ISORT_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ISORT_OK = 0,
  ISORT_EINVAL = 1,         /* bad argument: null pointer, bad width, bad offsets size */
  ISORT_ENOMEM = 2,         /* workspace allocation failed or bound workspace too small */
  ISORT_ECUDA = 3,          /* a CUDA runtime call failed */
  ISORT_ETIMEOUT = 4,       /* a bounded device-side wait gave up (result is garbage) */
  ISORT_EUNSUPPORTED = 5    /* valid but unsupported combination (n > 2^30, radix) */
} isort_status;

/* Sort keys[0..n) ascending in place. Paper: the SR4/PR4/PR2 radix sort,
 * Section "SR4, PR2, PR4, BTN and OET under MBSP". n = 0 or 1 is a no-op. */
isort_status isort_keys(void *keys, int64_t n, int key_bits, int radix_bits, void *stream);

/* Stable key-value sort: keys ascending, equal keys keep input order, vals[i]
 * moves with keys[i]. Same algorithm; the payload rides along every round. */
isort_status isort_pairs(void *keys, void *vals, int64_t n, int key_bits, int val_bits,
                         int radix_bits, void *stream);

/* The same sorts for keys (and payloads) held in HOST memory: keys_out[0..n)
 * receives keys_in[0..n) in ascending order (vals_out the payloads, stably);
 * an output may be its input (in place). Nothing is read from or written to
 * the host buffers outside [0, n) elements.
 *
 * The call enqueues on `stream`: the copy of the input into the stream's
 * workspace, the sort of that device copy (as isort_keys / isort_pairs), and the
 * copy of the result to the output buffers; it returns once this is enqueued.
 * The output is complete when the stream has reached that point (e.g. after
 * cudaStreamSynchronize); the input must stay unchanged, and every buffer
 * allocated, until then. Device-side errors are latched as for isort_keys.
 *
 * Buffers move by cudaMemcpyAsync (the copy engines; for pageable memory the
 * call then returns only when the copies are done, for page-locked memory at
 * once). ISORT_DEBUG_HOST_COPY 2 moves page-locked, 16-byte aligned buffers
 * with copy kernels instead (every SM reads or writes the host buffer through
 * its device mapping): as fast alone, slower when several streams' sorts and
 * copies overlap.
 * Workspace: isort_workspace_size(n, key_bits, val_bits, radix_bits) plus the
 * device copies, each rounded up to 256 bytes: n * key_bits / 8 (and
 * n * val_bits / 8 for pairs).
 * Errors: ISORT_EINVAL for null buffers, bad widths or misaligned elements;
 * ISORT_ENOMEM when a bound workspace cannot hold the device copies;
 * otherwise as isort_keys. n = 0 does nothing; n = 1 copies the element. */
isort_status isort_keys_host(const void *keys_in, void *keys_out, int64_t n, int key_bits,
                             int radix_bits, void *stream);
isort_status isort_pairs_host(const void *keys_in, const void *vals_in, void *keys_out,
                              void *vals_out, int64_t n, int key_bits, int val_bits,
                              int radix_bits, void *stream);

/* Segmented sort: each range [offsets[s], offsets[s+1]) is sorted independently
 * (vals may be NULL, then val_bits is ignored). offsets: DEVICE int64 array of
 * num_segments + 1 entries, offsets[0] = 0, non-decreasing, offsets[num_segments]
 * = total_keys; each segment at most 2^30 keys. The paper's sample sorts split
 * the input into p ranges and sort each independently (Algorithms 1-3); here
 * the ranges are given. Short segments use the paper's BTN merge-split bitonic
 * network ("Algorithm BTN", Eq. Tb), long ones the radix-256 passes, all
 * segments of a class in the same launch.
 *  - total_keys: the key count (= offsets[num_segments]) given on the host, so
 *    that the call can size its workspace without reading the device-resident
 *    offsets (which keeps the call asynchronous and graph-capturable); below
 *    2^40 (ISORT_EINVAL otherwise: the radix tiles record their first key in
 *    40 bits).
 *  - radix_bits: 0 or 8 (the segmented rounds are radix-256 rounds only; 11
 *    and 16 return ISORT_EUNSUPPORTED).
 * Offsets are read on the device only: a segment that breaks these rules is
 * skipped (left as it is) and isort_stream_status reports ISORT_EINVAL. */
isort_status isort_segmented(void *keys, void *vals, const int64_t *offsets, int64_t num_segments,
                             int64_t total_keys, int key_bits, int val_bits, int radix_bits,
                             void *stream);

/* Sort without allocating: isort_keys for 32-bit keys, radix 256, whose scratch
 * memory is a fixed array inside the library (about 5 MiB of device memory per
 * GPU that loads the library, held until the process exits) instead of a
 * workspace. The paper has no counterpart; this exists for callers that must
 * not allocate device memory while running -- a framework that owns all device
 * memory through its own pool, a latency-critical loop where cudaMalloc could
 * synchronise the device, code that must not hit out-of-memory after start-up.
 *  - keys: DEVICE array of n uint32 keys on the current device, sorted
 *    ascending in place. It always runs the built-in default radix-256 kernel
 *    variant (the autotuner's choice does not apply), so its speed can differ
 *    from isort_keys at the same n; the result is the same.
 *  - n > ISORT_NOALLOC_MAX_KEYS returns ISORT_ENOMEM (the array is too small);
 *    n = 0 or 1 is a no-op.
 *  - err_out: required DEVICE word on the current device (NULL returns
 *    ISORT_EINVAL): device-side error bits (a bounded wait that gave up, a
 *    failed output bounds check) are OR-ed into it. The caller zeroes it and
 *    reads it after the stream has finished; nonzero means the keys are not
 *    sorted.
 *  - The first call on a device looks up the array's device address (with that
 *    device current); make that first call before any stream capture.
 *  - Every call shares the one array, which keeps the previous call's contents
 *    (the call clears what must start at zero). Calls that overlap on the GPU
 *    -- on different streams, or from different threads -- race on it and give
 *    wrong results: serialise them. */
#define ISORT_NOALLOC_MAX_KEYS (1 << 20)
isort_status isort_keys_noalloc(void *keys, int64_t n, uint32_t *err_out, void *stream);

/* Segmented sort tuning: ranges of at most btn_max_keys keys use the BTN
 * network, longer ones the radix passes (capped by the BTN capacity, 4096
 * keys for 32-bit keys, 2048 for 64-bit; < 0 restores the default). */
isort_status isort_tune_segmented(int key_bits, int val_bits, int64_t btn_max_keys);

/* Network for the short ranges of a segmented sort (the paper compares both,
 * Section "Related work", Eqs. Tb and To; Tables 1-4):
 *   ISORT_NET_BTN (default): bitonic merge-split over q runs, lg q (lg q + 1) / 2 stages;
 *   ISORT_NET_OET: odd-even transposition merge-split over q runs, q rounds.
 * Both give the same (stable) result. Other values return ISORT_EINVAL. */
#define ISORT_NET_BTN 0
#define ISORT_NET_OET 1
isort_status isort_tune_segmented_network(int key_bits, int val_bits, int network);

/* Sample sort: the paper's GVR (Algorithm 3, Section "Oversampling algorithms:
 * GSD, GVR, GER") with the buckets sorted on this GPU. Sorts keys[0..n)
 * ascending in place (stable with vals, which may be NULL):
 *   1. s*p - 1 keys are drawn at random positions (SplitMix64, stream 30 of
 *      `seed`; position = high 32 bits of the draw times n, shifted right 32)
 *      and sorted with the BTN network;
 *   2. the (i*s)-th smallest sampled keys, 1 <= i <= p-1, are the splitters;
 *   3. one stable count-sort round moves every key to bucket j = the number of
 *      splitters smaller than it;
 *   4. each bucket is sorted independently (the segmented sort).
 * buckets = p in 1..256, oversample = s >= 1 with p*s <= 4096 (else
 * ISORT_EINVAL); n <= 2^30. bucket_counts: DEVICE array of p uint32 that
 * receives the bucket sizes, or NULL. The result is the same as isort_keys /
 * isort_pairs; the bucket sizes depend on the sample. */
isort_status isort_sample_sort(void *keys, void *vals, int64_t n, int key_bits, int val_bits,
                               int buckets, int oversample, uint64_t seed,
                               uint32_t *bucket_counts, void *stream);

/* Deterministic regular-oversampling sort: the paper's GSD (Algorithm 1,
 * Theorem 1). Sorts keys[0..n) ascending in place (stable with vals, which may
 * be NULL):
 *   1. the p sequences [n*k/p, n*(k+1)/p) are sorted independently;
 *   2. from each sorted sequence the r*p keys that end its r*p evenly sized
 *      segments (position floor(i * len / (r*p)) - 1, i = 1..r*p; the last is
 *      its maximum) are sampled, and all r*p*p samples sorted with BTN;
 *   3. the (i*r*p)-th smallest samples, 1 <= i <= p-1, are the splitters;
 *   4. each sorted sequence is split by binary search: part j holds its keys
 *      above splitter j-1 and at most splitter j;
 *   5. the p parts of every bucket are merged (lg p rounds of pairwise stable
 *      merges) and the buckets concatenated.
 * buckets = p: a power of two, 1..64; oversample = r >= 1 with r*p*p <= 4096
 * (else ISORT_EINVAL); n <= 2^30. bucket_counts: DEVICE array of p uint32 that
 * receives the bucket sizes, or NULL. No randomness: the result and the bucket
 * sizes depend on the input only. */
isort_status isort_gsd_sort(void *keys, void *vals, int64_t n, int key_bits, int val_bits,
                            int buckets, int oversample, uint32_t *bucket_counts, void *stream);

/* Bytes of workspace one isort_gsd_sort call with these arguments needs. */
isort_status isort_gsd_sort_workspace_size(int64_t n, int key_bits, int val_bits, int buckets,
                                           int oversample, size_t *bytes);

/* Bytes of workspace one isort_sample_sort call with these arguments needs. */
isort_status isort_sample_sort_workspace_size(int64_t n, int key_bits, int val_bits, int buckets,
                                              int oversample, size_t *bytes);

/* Bytes of workspace one isort_segmented call with these arguments needs. */
isort_status isort_segmented_workspace_size(int64_t num_segments, int64_t total_keys, int key_bits,
                                            int val_bits, size_t *bytes);

/* Bytes of workspace one call with these arguments needs (bytes may be NULL-checked). */
isort_status isort_workspace_size(int64_t n, int key_bits, int val_bits, int radix_bits,
                                  size_t *bytes);

/* Bind caller-owned device memory [dev_ptr, dev_ptr + bytes) as the workspace of
 * `stream` (dev_ptr 256-byte aligned). Later calls on that stream use it and
 * return ISORT_ENOMEM when it is too small; dev_ptr = NULL unbinds (the library
 * then allocates its own again). The memory must stay valid until the last
 * call on the stream has completed. Clears the stream's error word. */
isort_status isort_set_workspace(void *dev_ptr, size_t bytes, void *stream);

/* Synchronise `stream`, then report and clear its device error word:
 * ISORT_ETIMEOUT if a bounded wait gave up, ISORT_EINVAL if isort_segmented
 * met offsets that are not a valid partition, ISORT_ECUDA on a CUDA error or
 * a failed output bounds check. */
isort_status isort_stream_status(void *stream);

/* Release the library-allocated workspaces (synchronises their streams). */
isort_status isort_release_workspaces(void);

/* Human-readable name of a status code (static string). */
const char *isort_strerror(isort_status s);

/* Tuning of one kernel family: variant index into the library's table of
 * (threads, keys per thread) for radix-256 passes of (key_bits, val_bits).
 * -1 restores the built-in default. Returns ISORT_EINVAL for an unknown variant. */
isort_status isort_tune_set(int key_bits, int val_bits, int radix_bits, int variant);
/* Number of variants and the (threads, keys-per-thread) of variant v. */
int isort_tune_num_variants(int key_bits, int val_bits, int radix_bits);
isort_status isort_tune_describe(int key_bits, int val_bits, int radix_bits, int variant,
                                 int *threads, int *keys_per_thread);

/* Automatic choice, per size bucket: sorts of these widths with radix_bits = 0
 * and floor(log2 n) nearest to size_log2 (the lower bucket on a tie) use radix
 * width radix_bits (8, 11 or 16) and kernel variant `variant` of that width's
 * table. radix_bits < 0 clears the entry of size_log2, or every entry of these
 * widths when size_log2 < 0. Entries set here take precedence over the
 * built-in ones (the autotuner's choices measured on a GB300); an explicit
 * radix_bits uses the variant fixed by isort_tune_set, else the automatic
 * choice's variant when that chose the same width, else variant 0.
 * ISORT_EINVAL for an unknown width, bucket (0..30) or variant. The Python
 * tuner (paper_1808_10292_gb300/tune.py) measures the choices and loads its
 * cache through this call. */
isort_status isort_tune_auto(int key_bits, int val_bits, int size_log2, int radix_bits,
                             int variant);

/* The radix width and variant a sort of n keys with these arguments would use
 * (radix_bits 0 = automatic). No device work. */
isort_status isort_tune_resolve(int64_t n, int key_bits, int val_bits, int radix_bits,
                                int *radix_out, int *variant_out);

/* Test hooks. isort_debug_set(ISORT_DEBUG_SPIN_LIMIT, k): bounded waits give up
 * after k polls (0 restores the default). isort_debug_set(ISORT_DEBUG_STALL_TILE,
 * t): in the first round with a look-back of the next radix-256 sort (pass 1
 * of a keys-only sort, whose order-free pass 0 needs none; pass 0 with
 * payloads), tile t never publishes its counts so its successors' waits run
 * out (-1 = off; the sort's output is then garbage and isort_stream_status
 * reports ISORT_ETIMEOUT). */
enum {
  ISORT_DEBUG_SPIN_LIMIT = 1,
  ISORT_DEBUG_STALL_TILE = 2,
  ISORT_DEBUG_KERNEL_TIMING = 3,
  /* value = L2 prefetch distance of the radix-256 rounds in tiles (0 = off,
   * -1 = default: one wave, SMs x 4). A tuning knob; results are unchanged. */
  ISORT_DEBUG_PREFETCH_TILES = 6,
  /* Keys-only rounds after the first rank keys by the order in which shared
   * atomics serve the lanes of a warp and then check every tile (a tile that
   * fails is ranked again stably). value 1: every tile takes that stable
   * re-rank; value 2: the fast ranks are deliberately made unstable (odd lanes
   * first), which the check must catch; 0 = normal. Test hooks; results are
   * unchanged. */
  ISORT_DEBUG_CHECK_MODE = 7,
  /* How isort_keys_host / isort_pairs_host move a buffer between host and
   * device memory: 0 = automatic (the copy engines), 1 = copy engines
   * (cudaMemcpyAsync), 2 = copy kernels for page-locked, 16-byte aligned
   * buffers that the device maps at their own address (copy engines for the
   * rest). A tuning knob; results are unchanged. */
  ISORT_DEBUG_HOST_COPY = 8
};
isort_status isort_debug_set(int what, int64_t value);

/* Measurement hook. With isort_debug_set(ISORT_DEBUG_KERNEL_TIMING, 1) every sort
 * records a CUDA event on its stream before and after each kernel it enqueues.
 * This call waits for those events of the most recent sort and writes up to
 * `max` kernel names (static strings) and durations in milliseconds; it returns
 * how many it wrote (-1.0 for a duration that could not be read). */
int isort_debug_kernel_times(const char **names, float *ms, int max);

/* Measurement hook: the number of kernels this library has enqueued since it
 * was loaded (all streams and entry points; CUDA-graph replays of a captured
 * call are not counted again). */
int64_t isort_debug_launch_count(void);

/* Measurement hook: bytes of device memory the library currently holds as
 * workspaces it allocated itself (caller-bound workspaces and the fixed array
 * of isort_keys_noalloc are not counted). */
int64_t isort_debug_workspace_bytes(void);

#ifdef __cplusplus
}
#endif
#endif /* ISORT_H */
