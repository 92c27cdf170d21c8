/*
 * minjoin.h — C ABI of the GB300 (sm_103a) MinJoin edit-similarity join.
 *
 * The library computes the join of Zhang & Zhang, "MinJoin: Efficient Edit
 * Similarity Joins via Local Hash Minima" (arXiv 1810.08833):
 *   given strings s_0..s_{n-1} and a threshold K (Sec. 1, problem statement),
 *   return the pairs (i, j), i < j, with ED(s_i, s_j) <= K that share a
 *   partition (Alg. 3), together with their edit distances.
 *
 * Conventions shared by every entry point:
 *  - Strings are a concatenated byte array `bytes` plus `offsets` (int64,
 *    n+1 entries, non-decreasing, offsets[0] = 0): string i is
 *    bytes[offsets[i] .. offsets[i+1]).  Positions are 0-based.
 *  - Pointers named d_* are device pointers on the context's device; h_* are
 *    host pointers.  Inputs stay owned by the caller and are only read.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is stream-ordered; calls that return a count synchronise
 *    the stream before returning.
 *  - Every function returns 0 (MJ_OK) or a negative MJ_ERR_* code; it never
 *    aborts the process.  mj_strerror() names a code.  After an error the
 *    context stays usable.
 *  - Results of the last call are held in memory the context owns, valid
 *    until the next call of the same family on that context; *_copy entry
 *    points copy them into caller buffers.
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef MINJOIN_H
#define MINJOIN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MJ_OK 0
#define MJ_ERR_ARG (-1)          /* invalid argument (null pointer, size, parameter) */
#define MJ_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define MJ_ERR_OOM (-3)          /* device allocation failed */
#define MJ_ERR_DEVICE (-4)       /* a device-side check failed (see mj_stats.device_flags) */
#define MJ_ERR_UNSUPPORTED (-5)  /* input outside the supported range (e.g. radius too large) */
#define MJ_ERR_TIMEOUT (-6)      /* a bounded device-side wait ran out */
#define MJ_ERR_STATE (-7)        /* call order (e.g. copy before compute, no trained band model) */

/* mj_params.flags */
#define MJ_FLAG_KEY_CHECK 1u     /* check byte equality of every group of equal partition keys */
#define MJ_FLAG_FEATURES 16u     /* mj_join keeps every candidate's band features (mj_features_copy) */
#define MJ_FLAG_FIRST_PASS 32u   /* learned mode: run the first passes however few pairs they hold (by default
                                    they run only with at least 384 pairs per SM, below which their latency
                                    exceeds what they save, and every pair goes to band K) */
/* Deduplication of the candidate pairs (last step of Alg. 3's join).  By
 * default the library picks per call: a bitmap with one bit per pair i < j
 * (n^2/16 bytes, cleared, set by every raw pair, then compacted row by row
 * into the sorted list) when sweeping it costs less than sorting the raw
 * pairs and it fits in device memory, else a radix sort of the raw pairs.
 * Learned mode and MJ_FLAG_FEATURES always sort (they need each candidate's
 * multiplicity).  Both give the same candidate set. */
#define MJ_FLAG_DEDUP_SORT 64u     /* always sort the raw pairs */
#define MJ_FLAG_DEDUP_BITMAP 128u  /* use the pair bitmap whenever multiplicities are not needed (an allocation
                                      failure is then MJ_ERR_OOM) */

/* verification modes (mj_params.verify_mode) */
#define MJ_VERIFY_PLAIN 0        /* one pass with band K */
#define MJ_VERIFY_LEARNED 1      /* learned first-pass band k' < K, fallback to K */

/* verification kernels (mj_verify_config.kernel) */
#define MJ_VERIFY_KERNEL_AUTO 0       /* diagonal for K <= 255, wavefront above */
#define MJ_VERIFY_KERNEL_DIAGONAL 1   /* one thread per pair, band as ceil((K+1)/32) words */
#define MJ_VERIFY_KERNEL_WAVEFRONT 2  /* G lanes per pair, 32-row blocks, skewed wavefront: within one warp up
                                         to 32 lanes, one CTA of several warps from 64 to 1,024 lanes */
#define MJ_VERIFY_KERNEL_TUNED 3      /* per length bucket, as chosen by mj_autotune_verify */

typedef struct mj_ctx mj_ctx;

/* Choice of verification kernel for a context (used by mj_verify and mj_join).
 * Pairs are verified longest first; with MJ_VERIFY_KERNEL_TUNED each length
 * bucket (floor(log2) of the shorter length) uses the kernel the autotuner
 * picked for it.
 *  kernel    MJ_VERIFY_KERNEL_*.
 *  lanes     wavefront only: lanes per pair, 2, 4, 8, 16 or 32 (one warp) or
 *            64, 128, 256, 512 or 1024 (one CTA per pair, its warps handing
 *            block boundaries over through shared memory); 0 = the fewest that
 *            hold the band: one warp holds bands up to K = 1,024, a CTA of G
 *            lanes bands with 34 G >= K + 32 (K up to 34,784 with 1,024).  Too
 *            few lanes for a band is MJ_ERR_UNSUPPORTED.
 *  batching  TUNED only: 0 = one persistent launch per run of consecutive
 *            buckets that share a kernel; 1 = one launch per length bucket.
 *  graph     1 = capture the plain verification stage (ordering, bucketing,
 *            launches) in a CUDA graph and replay it on later calls with the
 *            same inputs and sizes (the first call with new inputs runs
 *            uncaptured, the second captures).  Needs a stream other than the
 *            legacy or per-thread default stream; on those it runs uncaptured. */
typedef struct {
  uint32_t kernel;
  uint32_t lanes;
  uint32_t batching;
  uint32_t graph;
} mj_verify_config;

/* Result of mj_autotune_verify, per length bucket b (shorter length in
 * [2^b, 2^(b+1))): pairs seen, the kernel and lanes chosen, and the time of
 * every candidate tried on the bucket's sample (candidates: diagonal when
 * K <= 255, then the wavefront with 2^c times the fewest lanes). */
#define MJ_TUNE_CANDIDATES 6
typedef struct {
  uint32_t count[32];
  uint32_t kernel[32];
  uint32_t lanes[32];
  float ms[32][MJ_TUNE_CANDIDATES];   /* 0 = not tried */
  uint32_t cand_kernel[MJ_TUNE_CANDIDATES];
  uint32_t cand_lanes[MJ_TUNE_CANDIDATES];
  uint32_t n_candidates;
} mj_autotune_report;

/* Parameters of one join.
 *  K       edit-distance threshold (Sec. 1).
 *  T       targeted number of partitions per string (Alg. 2); 0 = K.
 *  q       q-gram length; 0 = the rule of Sec. 2.2, q = ceil(3 log_|Sigma|(N/T)),
 *          with Sigma the distinct byte values present and N the longest length;
 *          capped so that q * ceil(log2 |Sigma|) <= 64.
 *  r_min   lower bound applied to the neighbourhood radius of Alg. 2
 *          (default 1; the literal rule gives r <= 0 for short strings).
 *  seed    seed of the random q-gram function Pi and of the partition key.
 *  verify_mode  MJ_VERIFY_PLAIN or MJ_VERIFY_LEARNED.
 *  flags   MJ_FLAG_KEY_CHECK: check every group of equal partition keys for
 *          byte equality (mismatches counted in mj_stats.key_collisions);
 *          MJ_FLAG_FEATURES: keep the candidates' band features;
 *          MJ_FLAG_FIRST_PASS: run the learned first passes however few pairs they hold;
 *          MJ_FLAG_DEDUP_SORT / MJ_FLAG_DEDUP_BITMAP: how candidates are deduplicated.
 *  repeats parallel repetition (Sec. 2.2, Thm 1): R = 1..64 independent random
 *          functions Pi_0 .. Pi_{R-1}; every string is partitioned under each,
 *          and the join matches the union of the R partition sets.  Pi_k has
 *          the seed  seed + k * 0x9E3779B97F4A7C15  (mod 2^64); the partition
 *          key keeps the base seed, so equal substrings get equal keys under
 *          every Pi_k.  Partition records come repetition by repetition, each
 *          in position order.  1 (the default) is the plain method; an
 *          explicit Pi table allows only 1.  Other values: MJ_ERR_ARG. */
typedef struct {
  uint32_t K;
  uint32_t T;
  uint32_t q;
  int32_t r_min;
  uint64_t seed;
  uint32_t verify_mode;
  uint32_t flags;
  uint32_t repeats;
} mj_params;

/* Parameters as derived for an input (Sec. 2.2, Alg. 2). */
typedef struct {
  uint32_t sigma;        /* distinct byte values present */
  uint32_t bits;         /* bits per rank code, max(1, ceil(log2 sigma)) */
  uint32_t q, T, K;
  int32_t r_max;         /* radius of the longest string */
  uint64_t N;            /* longest string length (the fixed one after mj_set_alphabet) */
  uint8_t rank[256];     /* rank code of every byte value (ascending byte order) */
  uint64_t input_max_len; /* longest string length of this input */
  uint8_t present[256];  /* 1 for every byte value present in this input */
} mj_derived;

/* Counters and timings of the last call (see each field). */
typedef struct {
  uint64_t n_strings, n_bytes;
  uint64_t n_partitions;       /* records of Alg. 1 over all strings */
  uint64_t n_raw_pairs;        /* pairs passing both filters, before dedup */
  uint64_t n_candidates;       /* |C| after dedup (Alg. 3) */
  uint64_t n_output;           /* pairs with ED <= K */
  uint64_t key_collisions;     /* groups with equal keys but different bytes (flags bit 0) */
  uint64_t band_cells;         /* K-band cells of all candidates: sum over pairs of
                                  #{(i,j): 1<=i<=|a|, 1<=j<=|b|, |i-j| <= K} */
  uint64_t first_pass_settled; /* learned mode: pairs decided by the first pass */
  uint64_t fallback_pairs;     /* learned mode: pairs re-run with band K */
  uint32_t device_flags;       /* bit set by a failed device-side check */
  float ms_derive, ms_partition, ms_join_filter, ms_verify, ms_total;
  uint64_t n_launches;         /* kernels the library launched during the call */
  /* device time (CUDA events on the call's stream) of the sections of the
   * last mj_join, in this order: 0 anchor test (Alg. 2), 1 partition
   * records from the anchors (Alg. 1), 2 record grouping sort, 3 pair emission
   * (filters of Alg. 3), 4 pair dedup, 5 equality bit-planes, 6 verification
   * kernel(s), 7 output compaction, 8 the candidates' longest-first order for
   * verification (a counting sort) */
  float ms_section[9];
  uint64_t verify_word_columns; /* 32-bit band words x columns the verifier advanced */
} mj_stats;

void mj_params_default(mj_params* p, uint32_t K);
const char* mj_strerror(int status);

/* Create a context on CUDA device `device` (the calling thread's current
 * device is left unchanged after the call). */
int mj_create(mj_ctx** ctx, int device);
void mj_destroy(mj_ctx* ctx);
int mj_get_stats(const mj_ctx* ctx, mj_stats* out);
/* Sets the verification kernel of the context (default: MJ_VERIFY_KERNEL_AUTO). */
int mj_set_verify_config(mj_ctx* ctx, const mj_verify_config* cfg);

/* Autotuner of the verifier's band tiling: times every candidate kernel on up
 * to `sample` pairs of every length bucket of the given pairs (band K) and
 * stores the fastest per bucket in the context, for MJ_VERIFY_KERNEL_TUNED.
 * Synchronises.  rep (nullable) receives the measurements. */
int mj_autotune_verify(mj_ctx* ctx, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n,
                       const uint32_t* d_i, const uint32_t* d_j, uint64_t m, uint32_t K, uint32_t sample,
                       void* stream, mj_autotune_report* rep);

/* Step a1 (Sec. 2.2, Alg. 2): Sigma, rank codes, N, q, T, r_max. */
int mj_derive(mj_ctx* ctx, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n,
              const mj_params* p, void* stream, mj_derived* out);

/* Steps a2-a4 (Alg. 1-2): partitions of every string.  The anchor test holds
 * a 4,096-position tile and halos of r_max positions in shared memory, so
 * r_max is limited to about 7,400 (32-bit Pi values; about 2,600 when Pi is
 * 64-bit, q * bits > 32, or given as a table); beyond, this and mj_join
 * return MJ_ERR_UNSUPPORTED.  *count receives the
 * number of partitions; mj_partition_copy writes them in string order (with
 * p->repeats = R > 1: repetition by repetition, each in string order), each
 * (sid, pos, len, key) with key the 64-bit partition-substring hash
 * (Alg. 3's partition hash f).  `d_qgram_table` (nullable) replaces Pi by a table of
 * 2^(q*bits) 64-bit values indexed by the packed rank code of a q-gram (first
 * symbol most significant) — the form of Table 2's worked example. */
int mj_partition(mj_ctx* ctx, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n,
                 const mj_params* p, const uint64_t* d_qgram_table, void* stream, uint64_t* count);
int mj_partition_copy(mj_ctx* ctx, uint32_t* d_sid, uint32_t* d_pos, uint32_t* d_len,
                      uint64_t* d_key, void* stream);

/* Steps a2-a7 (Alg. 3's hash join): the deduplicated candidate set C.
 * *count receives |C|; mj_candidates_copy writes the pairs (i < j) sorted. */
int mj_candidates(mj_ctx* ctx, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n,
                  const mj_params* p, const uint64_t* d_qgram_table, void* stream, uint64_t* count);
int mj_candidates_copy(mj_ctx* ctx, uint32_t* d_i, uint32_t* d_j, void* stream);

/* ---- Sharded join over several GPUs (one process per GPU; the exchange
 * itself, by collective communication, is the caller's: see the package's
 * sharded module).  The strings are split by id range; every shard is
 * partitioned locally under the global alphabet and longest length; the
 * partition records go to the rank owning their (length, key) class, so that
 * Alg. 3's hash join (grouping by partition substring) runs with every group
 * whole on one rank; the candidate pairs go to the rank owning the pair for
 * the dedup of C; verification needs every string on every rank.
 *
 * mj_set_alphabet: later mj_derive / mj_partition / mj_join calls on this
 * context take Sigma = the byte values with h_present[b] != 0 (256 flags) and
 * N as the longest length instead of the input's own, so that all shards
 * derive the same rank codes, q and Pi; an input with a byte value outside
 * Sigma or a string longer than N is MJ_ERR_ARG.  h_present = NULL reverts to
 * the input's own values. */
int mj_set_alphabet(mj_ctx* ctx, const uint8_t* h_present, uint64_t N);
/* Steps a5-a7 on given partition records (Alg. 3's join and filters, dedup):
 * record r is partition (d_pos[r], d_len[r]) of string d_sid[r] (global id
 * < n_strings) of length d_slen[r], with partition key d_key[r] (as written
 * by mj_partition_copy).  Records of one (length, key) class must all be
 * here.  *count receives the candidates; mj_candidates_copy writes them (i <
 * j, sorted).  Key equality stands for byte equality (no bytes are given, so
 * MJ_FLAG_KEY_CHECK is MJ_ERR_ARG); ids >= n_strings are MJ_ERR_ARG.
 * Synchronises. */
int mj_candidates_records(mj_ctx* ctx, const uint32_t* d_sid, const uint32_t* d_pos, const uint32_t* d_len,
                          const uint64_t* d_key, const uint32_t* d_slen, uint64_t n_rec, uint32_t n_strings,
                          const mj_params* p, void* stream, uint64_t* count);
/* The distinct pairs among (d_i[t], d_j[t]), t < m, each as (min, max):
 * *count receives their number and mj_candidates_copy writes them sorted
 * (the dedup of C over candidates gathered from several shards).  Ids >=
 * n_strings are MJ_ERR_ARG.  Synchronises. */
int mj_pairs_unique(mj_ctx* ctx, const uint32_t* d_i, const uint32_t* d_j, uint64_t m, uint32_t n_strings,
                    void* stream, uint64_t* count);

/* Step a8 (Sec. 3, verification with Ukkonen's band): for every pair
 * (d_i[t], d_j[t]), t < m, writes d_ed[t] = ED if ED <= k_t, else k_t + 1,
 * where k_t = d_k[t] if d_k is non-null, else K.  Any pair of strings is
 * allowed (equal ids, empty strings).  Stream-ordered; does not synchronise.
 * Rank codes are derived from the n strings given.  Bands: the diagonal
 * kernel holds K <= 255, one warp's wavefront K <= 1,024 and a CTA's up to
 * K = 34,784 (lanes of mj_verify_config); a wider band (or K >= 65,536)
 * returns MJ_ERR_UNSUPPORTED and writes nothing.  A pair id >= n yields
 * k_t + 1 and sets bit 0 of the context's device flags: mj_device_flags
 * reads them once the stream has run the call. */
int mj_verify(mj_ctx* ctx, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n,
              const uint32_t* d_i, const uint32_t* d_j, const uint32_t* d_k, uint64_t m, uint32_t K,
              void* stream, uint32_t* d_ed);

/* Device-side check flags of the context's last call (bit 0: an index
 * outside its buffer, e.g. a pair id >= n, was skipped and its pair given
 * k + 1; bit 1: a bounded wait gave up; bit 2: an output buffer was too
 * small; bit 3: a string too long for 32-bit column indexing).  Synchronises
 * `stream`, copies the flags into *flags and into mj_stats.device_flags.
 * Calls that return a count check these flags themselves (MJ_ERR_DEVICE);
 * mj_verify does not synchronise, so its flags are read here. */
int mj_device_flags(mj_ctx* ctx, void* stream, uint32_t* flags);

/* Failure injection for tests of the error paths (no GPU fault involved):
 * the nth device allocation the library makes from now on, on the calling
 * host thread, fails as if the device were out of memory (nth = 1: the next
 * one); 0 switches the injection off.  The call that hits it returns
 * MJ_ERR_OOM, frees nothing that it does not own and leaves its context
 * usable; mj_destroy still releases every buffer. */
int mj_inject_alloc_failure(int64_t nth);

/* mj_verify for callers that cannot allocate device memory.  No counterpart
 * in the paper: it exists for code that may not call cudaMalloc, such as a
 * plug-in whose host application owns all device memory through its own
 * pool, a latency-critical path that must avoid the synchronisation an
 * allocation can imply, or a deployment with a device-memory budget fixed at
 * start-up.  It allocates nothing: its scratch (equality bit-planes of the
 * input and a work counter) is one file-scope __device__ array of
 * MJ_VERIFY_STATIC_SCRATCH_BYTES that every GPU loading the library keeps
 * until the process exits.  No context is needed.
 *  - Arguments as for mj_verify without d_k (one band K for all pairs); the
 *    caller passes the inputs and the output array d_ed.
 *  - Limits: the input may hold at most about MJ_VERIFY_STATIC_SCRATCH_BYTES
 *    bytes (one byte of scratch per input byte, plus guard words) and K at
 *    most MJ_VERIFY_STATIC_MAX_K; larger inputs or bands return
 *    MJ_ERR_UNSUPPORTED without running anything.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The call synchronises `stream` once to read
 *    the input size, then queues the work and returns.
 *  - All calls share the one array: calls that overlap on the GPU (other
 *    streams, other threads) race and give wrong results; serialise them.
 *    Every call clears what must start at zero.
 *  - A pair id >= n gives K + 1 (the pair is skipped) and sets bit 0 of the
 *    call's device flags, kept in the same array: mj_verify_static_flags
 *    synchronises `stream` and returns them (until the next call). */
#define MJ_VERIFY_STATIC_SCRATCH_BYTES (16u << 20)
#define MJ_VERIFY_STATIC_MAX_K 255u
int mj_verify_static(const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n, const uint32_t* d_i,
                     const uint32_t* d_j, uint64_t m, uint32_t K, void* stream, uint32_t* d_ed);
/* Device flags of the last mj_verify_static call on the current device (bits
 * as in mj_device_flags); allocates nothing and synchronises `stream`. */
int mj_verify_static_flags(void* stream, uint32_t* flags);

/* The whole path (Alg. 3): *count receives the number of output pairs;
 * mj_result_copy writes them sorted by (i, j) with their edit distances.
 * In MJ_VERIFY_LEARNED mode a band model must have been trained or loaded. */
int mj_join(mj_ctx* ctx, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n,
            const mj_params* p, void* stream, uint64_t* count);
int mj_result_copy(mj_ctx* ctx, uint32_t* d_i, uint32_t* d_j, uint32_t* d_ed, void* stream);

/* mj_join on HOST buffers: copies bytes and offsets to the device on
 * `stream`, runs mj_join, and leaves the result for mj_result_copy_host,
 * which copies it to host buffers of *count entries each (pinned memory
 * avoids a staging copy). */
int mj_join_host(mj_ctx* ctx, const uint8_t* h_bytes, const int64_t* h_offsets, uint32_t n,
                 const mj_params* p, void* stream, uint64_t* count);
int mj_result_copy_host(mj_ctx* ctx, uint32_t* h_i, uint32_t* h_j, uint32_t* h_ed, void* stream);

/* ---- Learned first-pass band (no counterpart in the paper).
 * A small FP32 MLP (MJ_BAND_FEATURES -> 64 -> 64 -> 1, ReLU) predicts, from
 * features of a candidate pair, its edit distance as a fraction of K.  In
 * MJ_VERIFY_LEARNED mode mj_join verifies each candidate first with the
 * widest band that fits in the fewest 32-bit words holding the prediction
 * (plus `margin`), but only when that is fewer words than band K needs and
 * the candidate came from at least `min_multiplicity` matched partition
 * pairs; every pair the first pass does not settle (result > its band) is
 * verified again with band K, so the output equals the plain mode's.
 * Features of candidate (i, j), with n the shorter length, d0 the length
 * difference, c the matched partition pairs behind the candidate and pa, pb
 * the partition counts of the two strings:
 *   log2(1+n)/16, d0/K, c/(T+1), pa/(T+1), pb/(T+1), c/min(pa,pb),
 *   log2(1+c)/8, K/(K+100).
 * Parameters are MJ_BAND_PARAMS floats: W1[64][8], b1[64], W2[64][64],
 * b2[64], W3[64], b3. */
#define MJ_BAND_FEATURES 8
#define MJ_BAND_PARAMS 4801

typedef struct {
  uint32_t steps;   /* Adam steps */
  uint32_t batch;   /* samples per step, drawn with replacement */
  float lr;         /* Adam step size */
  float tau;        /* pinball-loss quantile in (0,1); 0 = mean squared error */
  uint64_t seed;    /* sampling seed (non-zero) */
} mj_band_train_params;

/* Features and band-K results of every candidate of the last mj_join run
 * with MJ_FLAG_FEATURES: d_x gets m x MJ_BAND_FEATURES
 * floats (row-major), d_ed min(ED, K+1) per candidate (plain mode), d_i/d_j
 * the pairs (all nullable).  *count (nullable) receives m. */
int mj_features_copy(mj_ctx* ctx, float* d_x, uint32_t* d_ed, uint32_t* d_i, uint32_t* d_j, uint64_t* count,
                     void* stream);
/* Fresh model: He-normal weights from `seed`, zero biases; sets the band rule.
 * min_multiplicity = 0 lets mj_band_train set it to the 1st percentile of the
 * multiplicity of the training samples whose band-K result fits a narrower
 * first band (candidates below it always get band K). */
int mj_band_init(mj_ctx* ctx, uint64_t seed, uint32_t margin, uint32_t min_multiplicity);
/* Trains the model on m samples (features d_x, band-K results d_ed with
 * target min(ED, K+1)/K) with the project's forward, backward and Adam
 * kernels; *final_loss (nullable) gets the last step's batch loss. */
int mj_band_train(mj_ctx* ctx, const float* d_x, const uint32_t* d_ed, uint64_t m, uint32_t K,
                  const mj_band_train_params* tp, void* stream, float* final_loss);
/* Model output for m feature rows (no gate). */
int mj_band_forward(mj_ctx* ctx, const float* d_x, uint64_t m, void* stream, float* d_yhat);
/* Loss and its gradient with respect to all MJ_BAND_PARAMS parameters over
 * the m samples (targets d_y), tau as in mj_band_train; synchronises. */
int mj_band_grad(mj_ctx* ctx, const float* d_x, const float* d_y, uint64_t m, float tau, void* stream,
                 float* d_grad, float* loss);
int mj_band_get_weights(const mj_ctx* ctx, float* h_w, uint64_t count);
int mj_band_set_weights(mj_ctx* ctx, const float* h_w, uint64_t count);
/* Calibration of learned mode on a held-out instance of the workload: the
 * join of (d_bytes, d_offsets, n) under p runs in plain mode and in learned
 * mode (one warm-up and three timed runs each, host wall time of the whole
 * call, median), and learned mode stays on for this context only if it was
 * faster.  Otherwise later learned-mode joins run the plain path (same
 * output), unless p->flags has MJ_FLAG_FIRST_PASS.  The network cannot gain
 * where false candidates carry the verification work: no narrower band can
 * reject a pair whose distance exceeds K, so only pairs with ED <= K can be
 * settled sooner, while the network runs on every candidate and learned mode
 * must sort the raw pairs to count each candidate's matched partitions.
 * Training, initialising, loading or setting the weights clears the
 * calibration (learned mode then runs the network).  Synchronises. */
typedef struct {
  float plain_ms, learned_ms;          /* median join times */
  uint64_t plain_word_columns;         /* band words x columns the verifier advanced, plain */
  uint64_t learned_word_columns;       /* the same in learned mode (first passes included) */
  uint64_t first_pass_settled;         /* pairs the first passes decided */
  uint32_t enabled;                    /* 1: learned mode runs the network from now on */
} mj_band_calibration;
int mj_band_calibrate(mj_ctx* ctx, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n,
                      const mj_params* p, void* stream, mj_band_calibration* out);
/* Binary file: magic "MJBAND01", margin, min_multiplicity, the parameters. */
int mj_band_save(const mj_ctx* ctx, const char* path);
int mj_band_load(mj_ctx* ctx, const char* path);

#ifdef __cplusplus
}
#endif

#endif /* MINJOIN_H */
