/*
 * kc.h - C ABI of a single-GPU k-mer counter for NVIDIA GB300 (sm_103a).
 *
 * The operation (Section II, problem statement; Algorithm 1, serial counter;
 * Algorithm 3, FA-BSP counter): given DNA reads, return the ordered array of
 * {k-mer, count} pairs of all length-k substrings of the reads.
 *
 *   - A read is a run of bytes; read i is reads[offsets[i] .. offsets[i+1]).
 *   - A window of k consecutive bytes inside one read counts iff every byte is
 *     one of A C G T a c g t (lowercase reads as uppercase).  A window with any
 *     other byte ('N', junk) is skipped whole; windows never span two reads.
 *   - The key of a window is the k-digit base-4 number with digits A=0 C=1 G=2
 *     T=3, first base most significant (Algorithm 1: kmer = (kmer << 2) OR
 *     Encode(base), keeping the low 2k bits).
 *   - Canonical mode: key = min(forward value, value of the reverse complement)
 *     as unsigned integers (the paper counts forward k-mers; canonical form is
 *     this library's reading for double-stranded reads).
 *   - Keys are 64-bit for k <= 32 and 128-bit for 33 <= k <= 64 (Section VII
 *     names 128-bit k-mers as the extension for long reads).
 *   - Result: distinct keys in strictly ascending unsigned order with their
 *     occurrence counts (Algorithm 1: Sort, then Accumulate).
 *
 * Every function returns a kc_status; no C++ exception crosses this ABI.  On
 * failure kc_last_error() describes the error (per calling thread).
 */
#ifndef KC_H
#define KC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KC_OK = 0,
  KC_EINVAL = 1,     /* bad argument; nothing was launched */
  KC_ENOMEM = 2,     /* the allocator returned NULL */
  KC_ECUDA = 3,      /* a CUDA runtime call failed */
  KC_EOVERFLOW = 4,  /* a count exceeded 2^32 - 1 */
  KC_ETIMEOUT = 5,   /* a bounded device-side wait gave up (result invalid) */
  KC_EBUSY = 6       /* the plan is in use by another call */
} kc_status;

typedef struct kc_plan_s *kc_plan_t;

/* Device memory hooks.  alloc returns a device pointer of at least `bytes`
 * bytes usable on `stream` (NULL on failure); free_ releases it. */
typedef void *(*kc_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*kc_free_fn)(void *ptr, void *stream, void *ctx);

typedef struct {
  int device;                 /* CUDA device ordinal the plan runs on */
  void *stream;               /* cudaStream_t for all work; NULL = legacy default stream */
  kc_alloc_fn alloc;          /* NULL: cudaMallocAsync on `stream` */
  kc_free_fn free_;           /* NULL: cudaFreeAsync on `stream` */
  void *alloc_ctx;            /* passed back to alloc / free_ */
  uint64_t max_device_bytes;  /* 0: no limit; else kc_count fails with KC_ENOMEM above it */
  uint32_t n_partitions_hint; /* coarse partitions (power of two, <= 4096); 0: chosen from input size */
  uint32_t block_size_hint;   /* reserved (0) */
  float table_load;           /* distinct keys aimed at per fine partition, as a fraction of the
                                 count table's slots (the fine split is sized by it); 0: 0.55 */
  uint32_t table_slots_max;   /* 0: largest table that fits shared memory; smaller values
                                 (>= 64) force the overflow path, for testing */
  uint32_t flags;             /* KC_PLAN_* bits */
} kc_plan_opts;

/* kc_plan_opts.flags: record a CUDA event on the plan's stream after every kernel
 * launch of kc_count, so kc_last_kernel_times can report each kernel's device time. */
#define KC_PLAN_PROFILE 1u
/* Testing: every fine partition writes its run to its own input region and the final
 * compaction pass moves it (the path taken when a partition's output offset is not yet
 * known when it is ready to write). */
#define KC_PLAN_DEFER_ALL 2u
/* Testing: kc_count_batch's scratch arena (counts that share batched launches) is limited
 * to 32 MiB, so that small batches form several groups and larger counts run alone. */
#define KC_PLAN_BATCH_ARENA_SMALL 4u
/* Aggregation variants (the GPU analogue of the paper's experiment that adds its L2 and L3
 * aggregation layers one at a time, Section VI); the result is unchanged, only the work
 * differs.  ABLATE_NO_SMEM_BUCKETS: pass B writes every key on its own through a global
 * atomic cursor per partition, instead of grouping each tile's keys by partition in shared
 * memory and writing runs (the L2 per-destination buffers).  WARP_MERGE: the count kernel
 * adds a warp's equal keys with one atomic (the L3 heavy-hitter merge); off by default,
 * because on GB300 the shared-memory atomics absorb equal keys faster than the merge's warp
 * vote costs, even when every key is the same.  kc_count only. */
#define KC_PLAN_ABLATE_NO_SMEM_BUCKETS 8u
#define KC_PLAN_WARP_MERGE 16u
/* Testing: the first fine partition never publishes its output offset and the device-side
 * wait for it is cut to a few iterations, so that the later partitions' bounded waits run
 * out: kc_count then returns KC_ETIMEOUT (no GPU fault, no hang). */
#define KC_PLAN_TEST_WITHHOLD_PREFIX 32u
/* Testing: counts above 2^16 - 1 are reported as overflowing (KC_EOVERFLOW), so that the
 * overflow report can be checked without an input of 2^32 windows of one k-mer. */
#define KC_PLAN_TEST_COUNT_LIMIT 64u
/* Testing: fine partition regions sized from a sample of the keys at any input size (by
 * default only counts of at least 2^26 bases do), and, with the second flag, without slack,
 * so that regions overflow and the exact fine split that follows is exercised. */
#define KC_PLAN_TEST_FINE_SAMPLED 128u
#define KC_PLAN_TEST_TIGHT_SLACK 256u

typedef struct {
  uint64_t n;               /* number of distinct keys */
  uint32_t key_words;       /* 1: keys are uint64[n]; 2: keys are uint64[2n], (lo, hi) per key */
  void *keys;               /* device pointer, ascending (for key_words 2: by hi, then lo) */
  uint32_t *counts;         /* device pointer, n counts, each >= 1 */
  uint64_t n_valid_windows; /* number of windows that counted = sum of counts */
  uint64_t capacity;        /* entries allocated behind keys / counts (>= n) */
  void *_owner;             /* library bookkeeping; do not touch */
} kc_result;

/* Create a plan (device properties, kernel attributes, memory hooks).  The plan
 * keeps its scratch memory between calls and grows it on demand.
 * Errors: KC_EINVAL (opts NULL or bad values), KC_ECUDA. */
kc_status kc_plan(const kc_plan_opts *opts, kc_plan_t *out);

/* Count the k-mers of n_reads reads.
 *   reads    bytes of all reads, back to back; host or device memory (detected
 *            with cudaPointerGetAttributes); borrowed until the call returns.
 *   offsets  n_reads + 1 uint64 offsets into `reads`, offsets[0] == 0,
 *            non-decreasing; host or device memory.
 *   k        1..64.   canonical  0: forward keys; nonzero: canonical keys.
 * On KC_OK, *out holds device buffers owned by the library until kc_free.
 * The call is synchronous with respect to the plan's stream (it returns after
 * the result is complete).  The order of the offsets is checked on the device (host
 * offsets too), so that a long offsets array costs no host-side pass.
 * Errors: KC_EINVAL (k out of range, NULL pointers, offsets[0] != 0, offsets not
 * non-decreasing), KC_ENOMEM, KC_ECUDA, KC_EOVERFLOW (a count above 2^32 - 1),
 * KC_ETIMEOUT (device wait limit hit).  On any error *out is zeroed. */
kc_status kc_count(kc_plan_t plan, const uint8_t *reads, const uint64_t *offsets, uint64_t n_reads, int k,
                   int canonical, kc_result *out);

/* Release the buffers of a result returned by kc_count (stream-ordered on the
 * plan's stream).  A zeroed result is accepted.  Errors: KC_EINVAL. */
kc_status kc_free(kc_plan_t plan, kc_result *res);

/* Copy a result to host memory: keys_host must hold n * key_words uint64,
 * counts_host n uint32.  Synchronous.  Errors: KC_EINVAL, KC_ECUDA. */
kc_status kc_result_copy_to_host(kc_plan_t plan, const kc_result *res, uint64_t *keys_host, uint32_t *counts_host);

/* Device memory a count of n_reads reads and n_bases bases with this k would take on this
 * plan: *scratch_bytes for its working buffers (a plan keeps one scratch block, grown to the
 * largest count it has run, and reuses it) and *result_bytes for the result buffers it
 * allocates (held until kc_free).  reads_on_device / offsets_on_device: whether the inputs
 * will be passed as device memory (16-byte aligned reads), so that no staging copy is
 * counted.  Host arithmetic only (the rules kc_count sizes a count by); nothing is
 * allocated.  Serves admission control: a server admits a request when free device memory
 * covers it.  Errors: KC_EINVAL (NULL arguments, k outside 1..64). */
kc_status kc_footprint(kc_plan_t plan, uint64_t n_reads, uint64_t n_bases, int k, int reads_on_device,
                       int offsets_on_device, uint64_t *scratch_bytes, uint64_t *result_bytes);

/* Destroy a plan and its scratch memory.  Results must be freed first. */
kc_status kc_plan_destroy(kc_plan_t plan);

/* Message for the last error on this thread ("" if none). */
const char *kc_last_error(void);

/* Launch statistics of the last kc_count on this plan: number of kernel
 * launches and the coarse/fine partition counts used.  Errors: KC_EINVAL. */
typedef struct {
  uint32_t kernel_launches;
  uint32_t n_partitions;       /* coarse partitions (phase 1) */
  uint64_t n_fine;             /* fine partitions (one shared-memory table each) */
  uint64_t n_overflow_fine;    /* fine partitions that needed the overflow path */
  uint64_t n_deferred_fine;    /* fine partitions whose run was moved to its place after the count
                                  (their output offset was not known in time) */
  uint64_t workspace_bytes;    /* scratch currently held by the plan */
  uint64_t phase_cycles[8];    /* KC_PLAN_PROFILE only: SM cycles of the count kernel's phases
                                  (clear, insert, sort, count, look-back, emit, overflow path,
                                  setup), summed over its thread blocks */
  uint64_t sub_cycles[8];      /* KC_PLAN_PROFILE only: cycles of the ordering sub-steps (key
                                  range, rank, scan, place, small sorts, large sorts) and the
                                  number of large buckets */
  uint32_t fine_sampled;       /* 1 if the fine partitions' regions were sized from a sample
                                  of the keys (large single counts) */
  uint32_t fine_resplit;       /* 1 if a sampled region overflowed and the exact fine split
                                  ran instead (the result is the same either way) */
} kc_stats;
kc_status kc_last_stats(kc_plan_t plan, kc_stats *out);

/* Device time of each kernel launched by the last kc_count on a plan created with
 * KC_PLAN_PROFILE, measured with CUDA events on the plan's stream.  Fills up to
 * `max` entries of names (static strings) and ms; *n_out = entries available.
 * Errors: KC_EINVAL (NULL plan / n_out, or the plan was not created with
 * KC_PLAN_PROFILE). */
kc_status kc_last_kernel_times(kc_plan_t plan, uint32_t max, const char **names, float *ms, uint32_t *n_out);

/* ---- Counting without allocation -------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that may not
 * allocate device memory while they count: for example an application that has given all
 * device memory to its own pool at start-up, or a latency-bound loop where an allocation,
 * and the synchronisation it can bring, is not acceptable.  It computes exactly what
 * kc_count computes, with the same kernels, but allocates nothing: every scratch buffer
 * lives in one fixed device array of KC_NOALLOC_SCRATCH_BYTES inside the library, which
 * every GPU that loads the library holds until the process exits.
 *
 *   reads, offsets  device memory (reads 16-byte aligned); offsets[n_reads] (the number
 *                   of bases) at most KC_NOALLOC_MAX_BASES.
 *   out_keys        device buffer of out_capacity * key_words uint64 (key_words = 1 for
 *                   k <= 32, else 2, (lo, hi) per key); out_counts: out_capacity uint32.
 *                   out_capacity must be at least offsets[n_reads].
 *   n_distinct, n_valid_windows   host pointers, written on success.
 *   stream          cudaStream_t (NULL = legacy default); the call returns after the
 *                   result is complete on it.
 * Alignment: offsets 8 bytes, out_counts 4 bytes, out_keys 8 bytes (16 bytes for k > 32);
 * a misaligned buffer is refused on the host before anything is launched.
 * The first call on a device (with that device current) looks up the scratch array's
 * device address and sets kernel attributes.  Every call reads the offsets and its status record back, so it synchronises
 * its stream.  All calls share the one array, and each call clears what it needs: calls
 * that overlap on the GPU (other streams, other host threads) race and must not be made.
 * Errors: KC_EINVAL (sizes beyond the maximum, host or misaligned buffers, small
 * out_capacity, bad k or offsets), KC_ECUDA, KC_EOVERFLOW, KC_ETIMEOUT; kc_last_error()
 * gives the message. */
#define KC_NOALLOC_MAX_BASES (1u << 20)
#define KC_NOALLOC_SCRATCH_BYTES (48u << 20)
kc_status kc_count_noalloc(const uint8_t *reads, const uint64_t *offsets, uint64_t n_reads, int k, int canonical,
                           uint64_t *out_keys, uint32_t *out_counts, uint64_t out_capacity, uint64_t *n_distinct,
                           uint64_t *n_valid_windows, void *stream);

/* Batched counting: the histograms of n_samples independent read sets in one call
 * (the same operation as kc_count, per sample; Section II, Algorithms 1 and 3).
 *
 *   reads[i], offsets[i], n_reads[i]   sample i, as for kc_count (reads host or device;
 *                   offsets host or device, offsets[i][0] = 0, non-decreasing).
 *   n_bases[i]      offsets[i][n_reads[i]], the sample's base count (host array), so
 *                   that nothing has to be read back before the samples are enqueued.
 *   out[i]          sample i's result, as kc_count returns it (free each with kc_free).
 *
 * Samples are grouped so that a group's scratch fits one arena (16 GiB; a quarter of
 * max_device_bytes when that is set), and every kernel of the path is launched once per
 * group, each thread block working for one sample of the group (a table maps blocks to
 * samples), so that many small samples fill the GPU together; a sample larger than the
 * arena is counted alone.  Everything is enqueued on the plan's stream with one host
 * synchronisation at the end.  The results of one group share two device allocations,
 * released when the last of their results is freed with kc_free.
 * On any error no result is returned (all out[i] zeroed) and kc_last_error() names the
 * sample.  Errors as for kc_count; KC_ENOMEM if the batch's results and scratch exceed
 * max_device_bytes. */
kc_status kc_count_batch(kc_plan_t plan, uint32_t n_samples, const uint8_t *const *reads,
                         const uint64_t *const *offsets, const uint64_t *n_reads, const uint64_t *n_bases, int k,
                         int canonical, kc_result *out);

/* Submitted counts: the same operation as kc_count, returned later, so that one host
 * thread can keep many counts queued (for a service that takes requests as they arrive)
 * and the GPU runs them back to back, without a host round trip between two counts.
 *
 * kc_submit checks the arguments, sizes the count and enqueues its kernels at once on the
 * plan's stream, behind the counts already queued there (the plan's scratch grows in
 * stream order when a count needs more), and returns without waiting for the GPU.  Counts
 * never run concurrently with each other on the device.  Inputs in host memory are copied
 * into a device buffer of the job's own on the plan's transfer stream (a second stream the
 * plan creates at its first submission), and the count's kernels wait for that copy: the
 * copy of the next count's inputs runs while the counts before it are still counting.
 *   reads, offsets, n_reads   as for kc_count (host or device memory).  They are read
 *                  after kc_submit returns: keep them valid and unchanged until the job
 *                  is collected.  Host buffers should be pinned (cudaMallocHost /
 *                  cudaHostRegister); copies from pageable memory may make the call wait.
 *   n_bases        offsets[n_reads] (known to the caller, so nothing is read back).
 *   *job           a nonzero job id, valid until the job is collected.
 * At most 4096 jobs are in flight per plan (KC_EBUSY beyond).
 * Errors: KC_EINVAL (as for kc_count; for host offsets offsets[0] = 0 and
 * offsets[n_reads] = n_bases are checked at once, the order of all offsets by the GPU and
 * reported when the job is collected), KC_ENOMEM, KC_ECUDA; no job is created then.
 *
 * kc_job_poll collects a job if it has finished: *done = 0 while it runs (KC_OK, *out
 * zeroed); once finished *done = 1 and *out holds the result exactly as kc_count returns
 * it (free with kc_free), or the job's error is returned (its buffers are released).
 * Either way the job id is then invalid.  kc_job_wait blocks until the job finishes and
 * collects it.  kc_plan_destroy waits for jobs not collected and releases them.
 * Errors: KC_EINVAL (NULL arguments, unknown job id), and the job's own errors. */
kc_status kc_submit(kc_plan_t plan, const uint8_t *reads, const uint64_t *offsets, uint64_t n_reads, uint64_t n_bases,
                    int k, int canonical, uint64_t *job);
kc_status kc_job_poll(kc_plan_t plan, uint64_t job, kc_result *out, int *done);

/* Submitted batch: the samples of kc_count_batch (same arguments) enqueued on the plan's
 * stream as kc_count_batch enqueues them (groups of samples sharing batched launches) and
 * returned at once, one job id per sample in job_ids[i] (collect each with kc_job_poll /
 * kc_job_wait; the results of a group share buffers released with the last kc_free).
 * Host arrays and buffers must stay valid until the jobs are collected.  Errors as for
 * kc_submit; on error no job is created. */
kc_status kc_submit_batch(kc_plan_t plan, uint32_t n_samples, const uint8_t *const *reads,
                          const uint64_t *const *offsets, const uint64_t *n_reads, const uint64_t *n_bases, int k,
                          int canonical, uint64_t *job_ids);
kc_status kc_job_wait(kc_plan_t plan, uint64_t job, kc_result *out);

/* Result of a submitted count copied to host memory as soon as the count ends, so that
 * the copy runs while the counts queued after it count (the pipelined form of kc_count +
 * kc_result_copy_to_host for a stream of inputs).  Call it after kc_submit /
 * kc_submit_batch and before the job is collected.  When the host sees the count end
 * (kc_job_poll / kc_job_wait), the result's keys and counts (out->n entries, laid out as
 * in kc_result) are copied on the plan's transfer stream to keys_host / counts_host, and
 * the job is reported done only once that copy has completed; the device result is still
 * returned and must still be freed with kc_free.
 *   keys_host      capacity * key_words uint64 words; counts_host: capacity uint32 (host
 *                  memory, pinned for the copy to overlap; device pointers also work).
 *                  Both must stay valid until the job is collected.
 *   capacity       entries the buffers hold; a result with more distinct keys fails the
 *                  job with KC_EINVAL when it is collected (its buffers are released).
 * Errors: KC_EINVAL (NULL arguments, unknown job, copy already under way), KC_EBUSY,
 * KC_ECUDA. */
kc_status kc_job_copy_to_host(kc_plan_t plan, uint64_t job, uint64_t *keys_host, uint32_t *counts_host,
                              uint64_t capacity);

#ifdef __cplusplus
}
#endif
#endif /* KC_H */
