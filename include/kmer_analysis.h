/*
 * k-mer analysis on one GB300 GPU (sm_103a) -- C ABI.
 *
 * The operation is the first stage of iterative contig generation
 * (Algorithm 1, K-merAnalysis(k, R)) as defined in Sec. II-B of
 * "Extreme Scale De Novo Metagenome Assembly" (MetaHipMer): split every read
 * into k-mers overlapping by k-1 bases, count each k-mer, tally the bases
 * seen just before and just after it in the reads (its left and right
 * extensions), drop k-mers seen fewer than min_count times, and classify each
 * side of every surviving k-mer as a unique extension, a fork or a dead end
 * (Sec. II-C: contigs follow unique high-quality extensions; the two-letter
 * code [ACGT][ACGT] names them).
 *
 * Definitions used throughout:
 *  - A base is one of the bytes 'A','C','G','T' (uppercase); any other byte
 *    is N.  A window (k consecutive bytes of one read) containing an N is
 *    skipped.  Windows never span two reads.
 *  - A k-mer and its reverse complement are one vertex: each window is
 *    counted under the lexicographically smaller of the two (A<C<G<T), its
 *    "canonical" key.  When the reverse complement is the key, the window's
 *    left and right neighbours swap sides and are complemented.
 *  - An extension base counts when it exists in the read, is a base (not N)
 *    and its Phred quality (byte - qual_offset) is >= qual_threshold.  Every
 *    window without N is counted regardless of quality.
 *  - Classes: 0..3 = unique extension A,C,G,T; 4 = FORK; 5 = DEAD_END.
 *    ext_mode 0 (depth adaptive, Sec. II-C): with m the most common
 *    extension base and alt the sum of the other three tallies, a side is
 *    UNIQUE(m) iff alt * err_den <= max(t_base * err_den, err_num * count),
 *    i.e. alt <= t_hq = max(t_base, e * d) with e = err_num / err_den, exact
 *    in integers; no extension at all is DEAD_END; a tie for most common is
 *    FORK.  ext_mode 1 (static, Sec. II-B): bases with tally >= t_ext are
 *    high-quality extensions; exactly one is UNIQUE, none DEAD_END, more FORK.
 *    The paper calls a base high quality when it is seen more than t_hq
 *    times; t_ext is that threshold written inclusively, t_ext = t_hq + 1.
 *
 * Keys are returned 2 bits per base (A=0, C=1, G=2, T=3), first base most
 * significant, in W = ceil(2k/64) 64-bit words; word 0 is the most
 * significant and holds the first 2k - 64(W-1) bits right-aligned.  Numeric
 * order of (word 0, word 1, ...) equals lexicographic order of the k-mer.
 *
 * Error handling: every call returns KMER_OK (0) or a negative KMER_ERR_*
 * code and never aborts.  Device-side failures (a table or buffer too small,
 * a bounded wait that gave up) are latched in a device status word and turn
 * into a retry with larger buffers or into an error code at the next
 * synchronising call (query).  kmer_last_error_message() describes the last
 * failure of the calling thread.
 *
 * Streams: every handle is bound to one CUDA stream (NULL = the legacy
 * default stream) and to the device current when it was created.  Calls
 * marked "asynchronous" only enqueue work on that stream.
 */
#ifndef KMER_ANALYSIS_H
#define KMER_ANALYSIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KMER_OK 0
#define KMER_ERR_INVALID_ARG (-1)       /* bad pointer, size, k or threshold */
#define KMER_ERR_OOM (-2)               /* device or host allocation failed */
#define KMER_ERR_TABLE_FULL (-3)        /* a hash table could not grow enough */
#define KMER_ERR_COUNTER_OVERFLOW (-4)  /* a count would exceed 2^32 - 1 */
#define KMER_ERR_TIMEOUT (-5)           /* a bounded device wait gave up */
#define KMER_ERR_CUDA (-6)              /* a CUDA runtime call failed */
#define KMER_ERR_BAD_STATE (-7)         /* call out of order (e.g. results before query) */
#define KMER_ERR_NO_DEVICE (-8)         /* no usable CUDA device */

#define KMER_MAX_K 127

/* Where a buffer lives.  KMER_HOST_STAGED is host memory that moves
 * through device buffers by the copy engines (cudaMemcpyAsync, in 64 MB
 * pieces) instead of being read or written in place by the kernels: the
 * kernels then touch only HBM, and the SMs are not held while the transfer
 * runs.  KMER_HOST reads and writes page-locked memory in place, which
 * overlaps the transfer with the kernels that make it; other host memory is
 * staged in both modes.  For one stream alone the in-place form is faster;
 * host threads that pipeline steps on their own streams do better staging
 * every transfer and running one step's counting at a time, so that each
 * step's transfers overlap another step's kernels. */
enum kmer_where { KMER_HOST = 0, KMER_DEVICE = 1, KMER_HOST_STAGED = 2 };
enum kmer_ext_mode { KMER_EXT_DEPTH_ADAPTIVE = 0, KMER_EXT_STATIC = 1 };
enum kmer_class { KMER_CLS_A = 0, KMER_CLS_C = 1, KMER_CLS_G = 2, KMER_CLS_T = 3,
                  KMER_CLS_FORK = 4, KMER_CLS_DEAD_END = 5 };
enum kmer_variant {
    KMER_VARIANT_PARTITIONED = 0, /* hash-partition windows in HBM, count each partition on chip (default) */
    KMER_VARIANT_HBM_TABLE = 1    /* one open-addressing table in HBM updated by atomics */
};

typedef struct kmer_readset kmer_readset_t;
typedef struct kmer_analysis kmer_analysis_t;

/* Parameters of one analysis (Sec. II-B / II-C).  Fill with
 * kmer_analysis_default_params() and override fields. */
typedef struct {
    uint32_t k;              /* odd, 1..127; even k is rejected (a k-mer could be its own reverse complement) */
    uint32_t min_count;      /* keep k-mers seen >= min_count times (the paper's epsilon + 1); >= 1 */
    uint32_t qual_offset;    /* byte value of Phred 0 (33 for FASTQ) */
    uint32_t qual_threshold; /* extension base counts iff Phred >= qual_threshold */
    uint32_t ext_mode;       /* enum kmer_ext_mode */
    uint32_t t_base;         /* mode 0: hard floor of t_hq */
    uint32_t err_num;        /* mode 0: e = err_num / err_den */
    uint32_t err_den;        /* mode 0: > 0 */
    uint32_t t_ext;          /* mode 1: tally at which a base is a high-quality extension */
    uint32_t variant;        /* enum kmer_variant */
    uint64_t distinct_hint;  /* expected distinct canonical k-mers; 0 = assume every window distinct */
    uint64_t memory_budget;  /* device bytes the analysis may hold while querying; 0 = 85% of free memory */
    uint32_t leaf_bits;      /* tuning override: log2 of the number of partitions (0 = automatic) */
    uint32_t flags;          /* KMER_FLAG_* */
    uint32_t l1_bits;        /* tuning override: log2 of the first-level fan-out when two levels are used (0 = automatic) */
    uint32_t reserved[3];    /* must be zero */
} kmer_analysis_params;

/* flags: record CUDA events around each stage on the analysis stream and
 * report the per-stage device times in kmer_analysis_stats. */
#define KMER_FLAG_PROFILE 1u
/* flags: Bloom-filter gate (Sec. II-B: Bloom filters keep erroneous k-mers,
 * mostly seen once, out of the hash tables).  A first pass over the reads
 * adds every window's canonical k-mer to a blocked Bloom filter F1 and
 * k-mers already in F1 to a second filter F2; the counting pass then keeps
 * only the windows of k-mers in F2.  Exact for min_count >= 2 (a k-mer seen
 * twice is always in F2; a k-mer seen once that slips through as a false
 * positive is counted, once, and dropped): keys, counts, tallies, classes
 * and `windows` are those of the ungated analysis, while `distinct` counts
 * only the k-mers that passed the gate.  Costs two filters of 8 bits per
 * expected distinct k-mer (about one byte per window on a first query) and
 * one more pass over the reads; pays where k-mers seen once are a large
 * share of the windows and memory is tight.  Requires min_count >= 2 and the
 * partitioned variant (INVALID_ARG otherwise); ignored by batches. */
#define KMER_FLAG_BLOOM_GATE 2u
/* flags: results in ascending key order.  The k-mer set has no order of its
 * own (Sec. II-A, use case 1: inserts commute); without this flag the
 * survivors come out grouped by partition.  With it, query, query_into and
 * merge_contigs leave them sorted by key (word 0 first, numerically; the
 * same as the lexicographic order of the k-mers) with count, ext and cls
 * moved along: a least-significant-digit radix sort on the device, 2k/8
 * passes over the keys, in place in the result arrays.  Its scratch (about
 * 8W + 74 bytes per survivor) reuses the query's record buffers when they are
 * large enough.  query_into with page-locked host arrays (KMER_HOST) then
 * stages through the analysis's device buffers as with KMER_HOST_STAGED.
 * At most 2^32 - 2 survivors (INVALID_ARG beyond).  Ignored by batches. */
#define KMER_FLAG_SORTED_OUTPUT 4u

/* Results of the last query.  Device pointers owned by the analysis; valid
 * until the next submit, query, reset or destroy of the same handle. */
typedef struct {
    uint64_t n;              /* surviving k-mers */
    uint32_t k;
    uint32_t words;          /* W = ceil(2k/64) */
    const uint64_t *keys;    /* n * W words, row-major (key i at keys[i*W]) */
    const uint32_t *count;   /* n occurrence counts */
    const uint32_t *ext;     /* n * 8 tallies: left A,C,G,T then right A,C,G,T */
    const uint8_t *cls;      /* n * 2 classes: left, right (enum kmer_class) */
    uint64_t windows;        /* windows counted (all valid windows, before the count filter) */
    uint64_t distinct;       /* distinct canonical k-mers before the count filter */
} kmer_result_view;

/* Counters of the last query, for tuning and tests. */
typedef struct {
    uint64_t windows, distinct, survivors;
    uint64_t records_emitted;   /* windows written to level-1 partitions, all passes */
    uint32_t passes;            /* passes over the reads (1 unless memory-bound) */
    uint32_t pass_bits, l1_bits, l2_bits;
    uint32_t retries;           /* re-runs after a buffer was too small */
    uint32_t fallback_leaves;   /* partitions recounted in an HBM table */
    uint32_t leaf_table_slots;  /* shared-memory table capacity per partition */
    uint32_t variant;
    uint64_t device_bytes;      /* device memory held by the analysis */
    float ms_total;             /* wall time of the query, host clock */
    uint32_t launches;          /* kernels launched by the query */
    /* with KMER_FLAG_PROFILE: device time (CUDA events on the analysis
     * stream) of each stage summed over passes and retries, and launches */
    float ms_scatter, ms_repart, ms_leaf, ms_fallback;
    uint32_t n_scatter, n_repart, n_leaf, n_fallback;
    uint64_t records_l2;        /* records moved by the level-2 repartition */
    uint64_t leaf_splits;       /* partitions whose keys did not fit one table and were counted in key ranges */
    uint64_t l2_waves;          /* level-2 waves (windows of level-1 buckets repartitioned and counted one after
                                   another, when their records do not fit the memory budget together); 0 = the
                                   level-2 stages took every bucket at once */
    uint64_t gate_first;        /* KMER_FLAG_BLOOM_GATE: windows whose k-mer the gate saw first (about the
                                   distinct k-mers) */
    uint64_t gate_twice;        /* KMER_FLAG_BLOOM_GATE: k-mers the gate saw at least twice (about the k-mers
                                   the counting pass kept) */
    float ms_gate;              /* with KMER_FLAG_PROFILE: device time of the gate's pass */
    uint32_t n_gate;
    float ms_sort;              /* with KMER_FLAG_PROFILE and KMER_FLAG_SORTED_OUTPUT: device time of the sort */
    uint32_t n_sort;
} kmer_analysis_stats;

/* Fills *p with defaults: min_count 2, qual_offset 33, qual_threshold 20,
 * depth-adaptive classes with t_base 2, e = 1/10, t_ext 2, partitioned variant. */
void kmer_analysis_default_params(kmer_analysis_params *p, uint32_t k);

/* Packs reads for the device (step a1).  Reads are given flat: read i is
 * bases[offsets[i] .. offsets[i+1]) with one quality byte per base in quals
 * (same indexing); offsets has n_reads + 1 non-decreasing entries, offsets[0]
 * is normally 0, and every read is shorter than 2^31 bases.  `where` says
 * whether bases, quals and offsets are host (KMER_HOST, any host memory:
 * page-locked memory is read in place by the pack kernel, other memory is
 * staged; KMER_HOST_STAGED: always staged by the copy engines) or device
 * (KMER_DEVICE) pointers.  The
 * quality test (Phred >= qual_threshold, Phred = byte - qual_offset) is
 * applied here, so every analysis that submits this readset must use the
 * same two values.  The caller keeps ownership of its buffers; they may be
 * released once this call returns (it synchronises the stream).  The readset
 * owns its packed copy (about 0.5 byte per base plus 16 bytes per read).
 * Errors: INVALID_ARG (null pointer with n_reads > 0, decreasing offsets,
 * a read of 2^31 bases or more), OOM, CUDA. */
int kmer_readset_create(const char *bases, const uint8_t *quals, const uint64_t *offsets, uint64_t n_reads,
                        uint32_t qual_offset, uint32_t qual_threshold, int where, void *cuda_stream,
                        kmer_readset_t **out);
/* Re-packs new reads into an existing readset (same arguments as
 * kmer_readset_create, its qual_offset / qual_threshold are kept); device
 * buffers are reused when large enough.  Synchronises the stream. */
int kmer_readset_pack(kmer_readset_t *rs, const char *bases, const uint8_t *quals, const uint64_t *offsets,
                      uint64_t n_reads, int where, void *cuda_stream);
/* Kernels launched by the last create/pack of this readset. */
int kmer_readset_launches(const kmer_readset_t *rs, uint32_t *launches);
/* Number of reads and bases of a readset. */
int kmer_readset_info(const kmer_readset_t *rs, uint64_t *n_reads, uint64_t *n_bases);
/* Frees a readset.  It must not be submitted to an analysis that has not
 * yet been queried or reset. */
int kmer_readset_destroy(kmer_readset_t *rs);

/* Creates an analysis bound to the current device and `cuda_stream`.
 * Errors: INVALID_ARG (k even, 0 or > 127; min_count 0; err_den 0 in mode 0;
 * unknown mode or variant; nonzero reserved fields), NO_DEVICE, OOM. */
int kmer_analysis_create(const kmer_analysis_params *p, void *cuda_stream, kmer_analysis_t **out);

/* Adds a readset to the analysis.  Submits are commutative and may be
 * repeated (the result counts every submitted read, Sec. II-A use case 1);
 * the readset must stay alive until the next query or reset.  Cheap: the
 * counting itself runs in query.  Errors: INVALID_ARG (null, or the readset
 * was packed with a different qual_offset / qual_threshold). */
int kmer_analysis_submit(kmer_analysis_t *h, const kmer_readset_t *rs);

/* Packs reads (as kmer_readset_create) into a readset owned by the analysis
 * and submits it; released at the next reset or destroy. */
int kmer_analysis_submit_raw(kmer_analysis_t *h, const char *bases, const uint8_t *quals, const uint64_t *offsets,
                             uint64_t n_reads, int where);

/* Counts, filters and classifies everything submitted since the last reset
 * (steps a2-a7) and fills *out with device pointers to the survivors, in no
 * particular order (ascending key order with KMER_FLAG_SORTED_OUTPUT).
 * Synchronises the stream.  Buffers grow as needed and are kept for the next
 * query.  Errors: OOM, TABLE_FULL, COUNTER_OVERFLOW, TIMEOUT, CUDA, and
 * INVALID_ARG for sorted output of more than 2^32 - 2 survivors; the
 * previous results are invalid after an error. */
int kmer_analysis_query(kmer_analysis_t *h, kmer_result_view *out);

/* As kmer_analysis_query, but the survivors are written straight into the
 * caller's arrays (layouts as in kmer_result_view) as the kernels find them,
 * instead of into the analysis's buffers: with page-locked host arrays
 * (where = KMER_HOST) the transfer to the host overlaps the counting.  With
 * where = KMER_HOST_STAGED (any host arrays) the survivors go to the
 * analysis's own device buffers first and are then copied to the arrays by
 * the copy engines.  The arrays hold `capacity` k-mers and must not
 * overlap; with KMER_DEVICE and KMER_HOST the kernels write them directly,
 * so keys must be 8-byte, count 4-byte, ext 16-byte and cls 2-byte aligned
 * (as any allocation is).  *out points at them.  The results stay valid (for
 * views, copies and lookups) until the next query, reset or destroy.
 * Errors: as kmer_analysis_query, plus INVALID_ARG for NULL or misaligned
 * arrays, host arrays that are not page-locked, or more survivors than
 * `capacity` (kmer_last_error_message gives the count). */
int kmer_analysis_query_into(kmer_analysis_t *h, uint64_t *keys, uint32_t *count, uint32_t *ext, uint8_t *cls,
                             uint64_t capacity, int where, kmer_result_view *out);

/* Copies the survivors of the last query to host memory: keys (n * W words),
 * count (n), ext (n * 8), cls (n * 2); any pointer may be NULL to skip that
 * array; `capacity` is the number of k-mers the buffers hold.  The copy
 * engines move them in 64 MB pieces; the call waits for them (synchronous).
 * Errors: BAD_STATE (no successful query), INVALID_ARG (capacity < n). */
int kmer_analysis_copy_results(kmer_analysis_t *h, uint64_t *keys, uint32_t *count, uint32_t *ext, uint8_t *cls,
                               uint64_t capacity);

/* One looked-up k-mer (kmer_analysis_lookup), 40 bytes. */
typedef struct {
    uint32_t count;    /* occurrences; 0 when the k-mer is not a survivor */
    uint32_t ext[8];   /* tallies of the canonical k-mer: left A,C,G,T then right A,C,G,T */
    uint8_t cls[2];    /* classes of the canonical k-mer's sides (enum kmer_class) */
    uint8_t found;     /* 1 if the k-mer is among the survivors */
    uint8_t flipped;   /* 1 if the given k-mer is the reverse complement of its canonical form */
} kmer_record;

/* Looks up n k-mers among the survivors of the last query (the table the
 * graph traversal of Sec. II-C consults: count and the class of each side of
 * a vertex).  keys: n * W words, row-major, word 0 most significant, bits
 * above 2k zero (a key with such bits is reported not found); either
 * orientation (a k-mer and its reverse complement are one vertex, Sec.
 * II-B).  One record per key is written to out.  keys and out are both host
 * memory (where = KMER_HOST or KMER_HOST_STAGED, both staged) or both
 * device memory (KMER_DEVICE).  The first
 * lookup after a query builds an index of the survivors in device memory
 * (4 bytes per slot, 2-4 slots per survivor); later lookups reuse it.
 * Synchronous.  Errors: BAD_STATE (no successful query), INVALID_ARG (NULL
 * with n > 0, bad where), OOM, CUDA. */
int kmer_analysis_lookup(kmer_analysis_t *h, const uint64_t *keys, uint64_t n, kmer_record *out, int where);

/* Merge of Algorithm 1 (Merge(k-mer_set, prev_k-mer_set), Sec. II-G): the
 * survivors of the last query are merged with ExtractKmers(C, k), the k-mers
 * of a contig set C, which the paper treats as error-free k-mers with unique
 * high-quality extensions.  A contig k-mer's extension on a side is the
 * contig's neighbouring base (none at a contig end), in the k-mer's canonical
 * orientation; over all its occurrences in C a side with one such base is
 * UNIQUE, with none DEAD_END, with several FORK.  A k-mer found among the
 * survivors keeps the survivor's record (the two occurrences collapse into
 * one); a k-mer found only in the contigs is appended after the survivors
 * with count 0 (no read supports it beyond the count filter), zero tallies
 * and those classes.  Contigs are given flat like reads (contig i is
 * contigs[offsets[i] .. offsets[i+1]), any byte other than A, C, G, T breaks
 * the windows), where = HOST / HOST_STAGED / DEVICE.  *added receives the
 * number of appended k-mers (may be NULL) and *out the merged view (valid as
 * a query's view).  Later lookups see the merged set.  Synchronous.  Errors:
 * INVALID_ARG, BAD_STATE (no successful query, or results written to caller
 * arrays by kmer_analysis_query_into), OOM, CUDA. */
int kmer_analysis_merge_contigs(kmer_analysis_t *h, const char *contigs, const uint64_t *offsets, uint64_t n_contigs,
                                int where, uint64_t *added, kmer_result_view *out);

/* Contigs of a de Bruijn graph traversal (kmer_analysis_traverse): device
 * pointers owned by the analysis, valid until the next query, merge, reset or
 * destroy.  Contig i is seq[offsets[i] .. offsets[i+1]) (ASCII A/C/G/T). */
typedef struct {
    uint64_t n_contigs;
    uint64_t bases;             /* offsets[n_contigs] */
    const char *seq;
    const uint64_t *offsets;    /* n_contigs + 1 entries */
} kmer_contigs_view;

/* De Bruijn graph traversal (Sec. II-C, DeBruijnGraphTraversal of Algorithm
 * 1) over the current k-mer set (the last query's survivors, merged with
 * contig k-mers if kmer_analysis_merge_contigs ran): contigs are the paths
 * formed by k-mers with unique extensions.  A vertex is a k-mer whose two
 * sides are both UNIQUE; a k-mer read in an orientation x and its right
 * neighbour y = x[1..k) + (x's right base) are joined when y's canonical form
 * is another vertex whose left base, in y's orientation, is x[0] (each names
 * the other; a k-mer followed by its own reverse complement is joined to
 * nothing there).  A contig is a maximal path (its first k-mer, then one base
 * per later k-mer); a ring is cut before its smallest canonical k-mer.  Each
 * contig is reported as the smaller of itself and its reverse complement;
 * the contigs come in no particular order.  Computed by list ranking on the
 * device.  Synchronous.  Errors: BAD_STATE (no successful query),
 * INVALID_ARG (more than 2^31 - 1 k-mers), OOM, CUDA. */
int kmer_analysis_traverse(kmer_analysis_t *h, kmer_contigs_view *out);

/* Copies the contigs of the last traversal to host (or device) memory:
 * seq (bases), offsets (n_contigs + 1); either may be NULL.  Errors:
 * BAD_STATE (no traversal since the last query), INVALID_ARG (too small). */
int kmer_analysis_copy_contigs(kmer_analysis_t *h, char *seq, uint64_t *offsets, uint64_t seq_capacity,
                               uint64_t contig_capacity);

/* Counters of the last query. */
int kmer_analysis_get_stats(const kmer_analysis_t *h, kmer_analysis_stats *out);

/* Forgets submitted readsets and results; keeps device buffers for reuse. */
int kmer_analysis_reset(kmer_analysis_t *h);

/* Releases the analysis and every buffer it owns.  NULL is accepted. */
int kmer_analysis_destroy(kmer_analysis_t *h);

/* ---------------------------------------------------------------- batches
 * Many independent analyses (samples of uneven size, mixed k) run together
 * (Algorithm 1 runs K-merAnalysis once per k; a sample collection runs it
 * once per sample).  Each job is one readset with its own parameters and
 * gives exactly the result of a separate create/submit/query.  The jobs are
 * grouped into waves whose scratch fits the memory budget; each wave is
 * captured once as a CUDA graph in which every stage is one launch over all
 * jobs of a key width, and kmer_batch_run replays the graphs.  A job whose
 * output or leaf layout turns out too small is repaired inside its wave (the
 * stages after the scatter re-run for that job); a job whose level-1 buckets
 * overflow, or that is too large for any wave, is re-run alone through the
 * regular path.  Results are always exact.  A run whose counts differ from
 * what a job was planned for (distinct keys more than 10% above or 25% below
 * the plan) teaches the batch: the next run re-plans with those counts and
 * re-captures the graphs. */
typedef struct kmer_batch kmer_batch_t;

typedef struct {
    const kmer_readset_t *readset;  /* must outlive the batch and keep its size */
    kmer_analysis_params params;    /* variant must be KMER_VARIANT_PARTITIONED; distinct_hint, leaf_bits and
                                       l1_bits size the job's partitions (an autotuner can set them) */
    uint64_t survivors_hint;        /* expected surviving k-mers, sizes the output (0 = a quarter of the windows) */
} kmer_batch_job;

typedef struct {
    uint32_t jobs, waves;
    uint32_t graph_launches;  /* by the last run: one per wave */
    uint32_t jobs_alone;      /* jobs of the last run that went through the regular path */
    uint32_t fallback_leaves; /* leaves of the last run recounted in an HBM table after their wave */
    float ms_total;           /* wall time of the last run, host clock */
    uint32_t jobs_repaired;   /* jobs of the last run whose output, fallback list or level-2 layout was grown
                                 inside their wave, the later stages re-run for that job only */
    uint32_t alone_level1;    /* jobs_alone because a level-1 bucket overflowed */
    uint32_t alone_other;     /* jobs_alone for another reason (too large for a wave, a failed wait) */
    uint32_t replans;         /* times the batch was re-planned from a run's counts (since creation) */
} kmer_batch_stats;

/* Plans the jobs, allocates every buffer (memory_budget bytes of device
 * memory at most; 0 = 60% of free memory) and captures the graphs.  The
 * stream is used for every run.  Errors: INVALID_ARG (NULL, bad parameters,
 * readset/quality mismatch), NO_DEVICE, OOM, CUDA. */
int kmer_batch_create(const kmer_batch_job *jobs, uint32_t n_jobs, uint64_t memory_budget, void *cuda_stream,
                      kmer_batch_t **out);
/* Runs every job (one graph launch per wave) and synchronises the stream.
 * The readsets may be re-packed between runs with reads of the same sizes. */
int kmer_batch_run(kmer_batch_t *b);
/* Device view of job `job`'s survivors after a run (as kmer_analysis_query);
 * valid until the next run or destroy.  Errors: INVALID_ARG, BAD_STATE. */
int kmer_batch_result(kmer_batch_t *b, uint32_t job, kmer_result_view *out);
/* Host copy of job `job`'s survivors (as kmer_analysis_copy_results). */
int kmer_batch_copy_results(kmer_batch_t *b, uint32_t job, uint64_t *keys, uint32_t *count, uint32_t *ext,
                            uint8_t *cls, uint64_t capacity);
int kmer_batch_get_stats(const kmer_batch_t *b, kmer_batch_stats *out);
int kmer_batch_destroy(kmer_batch_t *b);

/* ---------------------------------------------------------------- serving
 * A request loop: requests (a resident readset + parameters) arrive at any
 * time from any thread; each is admitted, in arrival order, as soon as its
 * estimated device footprint fits the memory budget, and runs on one of the
 * server's worker threads with its own CUDA stream, so admitted requests
 * overlap on the device.  A finished request holds its results until it is
 * released; released analyses are pooled per worker and reused by later
 * requests with the same parameters (evicted when memory is needed).  Every
 * request gives exactly the result of a separate create/submit/query. */
typedef struct kmer_server kmer_server_t;

typedef struct {
    uint64_t id;
    int32_t status;            /* KMER_OK or the request's error code */
    uint32_t reserved;
    double t_submit_ms, t_admit_ms, t_start_ms, t_done_ms;  /* since the server was created */
    uint64_t footprint_bytes;  /* device memory the request was admitted with */
} kmer_request_info;

typedef struct {
    uint64_t submitted, completed, failed;
    uint32_t workers, peak_running;   /* most requests running at the same time */
    uint32_t pending, running, pooled;
    uint32_t reserved;
    uint64_t bytes_in_use, budget;
} kmer_server_stats;

/* memory_budget: device bytes for all admitted requests (0 = 70% of free
 * memory); workers: requests that may run at once (1..64). */
int kmer_server_create(uint64_t memory_budget, uint32_t workers, kmer_server_t **out);
/* Queues a request (non-blocking).  The readset must stay alive until the
 * request is released.  p->memory_budget, if nonzero, caps the request's
 * footprint; a request larger than the budget runs in several passes. */
int kmer_server_submit(kmer_server_t *s, const kmer_readset_t *rs, const kmer_analysis_params *p, uint64_t *id);
int kmer_server_poll(kmer_server_t *s, uint64_t id, int *done);
/* Blocks until the request is done; *out is its device result view (valid
 * until release), *info its timestamps.  Returns the request's status. */
int kmer_server_wait(kmer_server_t *s, uint64_t id, kmer_result_view *out, kmer_request_info *info);
int kmer_server_copy_results(kmer_server_t *s, uint64_t id, uint64_t *keys, uint32_t *count, uint32_t *ext,
                             uint8_t *cls, uint64_t capacity);
/* Frees the request's results (its analysis goes back to the pool). */
int kmer_server_release(kmer_server_t *s, uint64_t id);
int kmer_server_get_stats(kmer_server_t *s, kmer_server_stats *out);
/* Waits for admitted requests, drops requests never admitted, frees everything. */
int kmer_server_destroy(kmer_server_t *s);

/* k-mer analysis without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code that runs inside an allocator or memory-pool hook and
 * must not re-enter it, plugins whose host application owns every device
 * allocation, and paths where an allocation (with the synchronisation it can
 * imply) is not allowed.  It computes the same result as kmer_analysis_query
 * (variant KMER_VARIANT_HBM_TABLE) for one batch of reads given as DEVICE
 * pointers (bases, quals, offsets as in kmer_readset_create), with only
 * k, min_count, qual_offset, qual_threshold and the classification fields of
 * *p used.  Its only device scratch is a 32 MiB array at file scope, reserved
 * on each device where the library is used and held until the process exits;
 * it bounds the input: the reads may span at most 393216 bases for k <= 63
 * and 196608 bases for k >= 65 (larger inputs return INVALID_ARG before any
 * work).  Offsets must not decrease: a read whose offsets decrease or leave
 * [offsets[0], offsets[n_reads]] is skipped without reading its bases, and
 * the call returns INVALID_ARG.  The caller passes the output arrays (device
 * pointers, `capacity` k-mers, layout of kmer_result_view); *n_out receives
 * the number of survivors, and if it exceeds `capacity` the call returns
 * INVALID_ARG with the surplus not written.  Synchronises `cuda_stream`
 * (it reads two offsets and its counters back to the host).  The first call
 * on each device, and in each CUDA context, also looks up the scratch
 * array's device address, so make that first call before any stream capture
 * begins.  Every call reuses the same array (each call clears it first):
 * calls that overlap on the GPU, from several streams or threads, race and
 * must be serialised by the caller.  Errors: INVALID_ARG, NO_DEVICE,
 * TABLE_FULL, COUNTER_OVERFLOW, TIMEOUT, CUDA. */
int kmer_analysis_run_noalloc(const char *bases, const uint8_t *quals, const uint64_t *offsets, uint64_t n_reads,
                              const kmer_analysis_params *p, uint64_t *keys, uint32_t *count, uint32_t *ext,
                              uint8_t *cls, uint64_t capacity, uint64_t *n_out, void *cuda_stream);

/* Static description of an error code. */
const char *kmer_strerror(int code);

/* Human-readable detail of the last failure on the calling thread. */
const char *kmer_last_error_message(void);

/* Library version, e.g. "1.0.0". */
const char *kmer_version(void);

#ifdef __cplusplus
}
#endif
#endif /* KMER_ANALYSIS_H */
