// Internal declarations of the MinJoin CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "../../include/minjoin.h"

#define MJ_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) {                                \
      mj::set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return MJ_ERR_CUDA;                                   \
    }                                                       \
  } while (0)

// every kernel launch of the library is followed by MJ_KERNEL_DONE(): it
// counts the launch (mj_stats.n_launches) and checks the launch error
#define MJ_KERNEL_DONE()                  \
  do {                                    \
    mj::note_launch();                    \
    MJ_CUDA_TRY(cudaGetLastError());      \
  } while (0)

#define MJ_TRY(expr)          \
  do {                        \
    int _s = (expr);          \
    if (_s != MJ_OK) return _s; \
  } while (0)

namespace mj {

constexpr int kNumSMsHint = 152;

// device-side error flags (mj_stats.device_flags)
enum : uint32_t {
  FLAG_BOUNDS = 1u << 0,       // an index left its buffer (access skipped)
  FLAG_TIMEOUT = 1u << 1,      // a bounded wait gave up
  FLAG_CAPACITY = 1u << 2,     // an output buffer was too small (write skipped)
  FLAG_LENGTH = 1u << 3,       // a string too long for 32-bit column indexing (pair rejected)
};

void set_last_cuda_error(cudaError_t e, const char* expr, const char* file, int line);
void note_launch();
uint64_t launch_count();

// ---------------------------------------------------------------- workspace
// A growable device buffer owned by a context; reallocated (contents
// dropped) only when a larger size is requested.
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
  int reserve(size_t need, cudaStream_t s);
  // as reserve, but the first `keep` bytes survive a reallocation
  int grow_keep(size_t need, size_t keep, cudaStream_t s);
  template <class T>
  T* as() const { return static_cast<T*>(p); }
  void release();
};

// Derived parameters of one input (host copy).
struct Derived {
  uint32_t sigma = 0, bits = 1, q = 1, T = 1, K = 0;
  int32_t r_min = 1, r_max = 0;
  uint64_t N = 0, seed = 0;
  uint32_t repeats = 1;   // parallel repetition: independent Pi functions
  uint8_t rank[256] = {0};
};

// ---------------------------------------------------------------- kernels (launchers)
// All launchers are stream-ordered and return MJ_OK or MJ_ERR_CUDA.

// a1: 256-bin byte histogram (u64 counts) and the longest string length.
int launch_byte_histogram(const uint8_t* bytes, uint64_t nbytes, unsigned long long* hist,
                          cudaStream_t s);
int launch_max_length(const int64_t* offsets, uint32_t n, unsigned long long* out, cudaStream_t s);
// *out = max of v[0 .. n-1] (0 when n = 0)
int launch_max_u32(const uint32_t* v, uint64_t n, unsigned int* out, cudaStream_t s);

// A partition record, packed in two 16-byte words: Karp-Rabin key, group
// run (the hash bits of the grouping sort key; 0 until the records are put
// in group order), string length, partition length, string id, position.
struct alignas(16) PRec {
  uint64_t h61;
  uint32_t run, slen, len, sid, pos, pad;
};
static_assert(sizeof(PRec) == 32, "PRec is two 16-byte words");

__device__ __forceinline__ PRec load_rec(const PRec* __restrict__ r, uint64_t u) {
  const uint4* p = reinterpret_cast<const uint4*>(r + u);
  const uint4 a = __ldg(p), b = __ldg(p + 1);
  PRec x;
  x.h61 = (uint64_t)a.x | ((uint64_t)a.y << 32);
  x.run = a.z;
  x.slen = a.w;
  x.len = b.x;
  x.sid = b.y;
  x.pos = b.z;
  x.pad = b.w;
  return x;
}

__device__ __forceinline__ void store_rec(PRec* __restrict__ r, uint64_t u, const PRec& x) {
  uint4* p = reinterpret_cast<uint4*>(r + u);
  p[0] = make_uint4((uint32_t)x.h61, (uint32_t)(x.h61 >> 32), x.run, x.slen);
  p[1] = make_uint4(x.len, x.sid, x.pos, x.pad);
}

// a2-a3: anchor bitmap (1 bit per byte position) and per-tile anchor counts.
struct PartitionArgs {
  const uint8_t* bytes;
  const int64_t* offsets;
  uint32_t n;
  uint64_t nbytes;
  uint32_t q, bits, T;
  int32_t r_min, r_max;
  uint32_t seed32;
  uint64_t seed64;
  const uint64_t* table;  // nullable explicit Pi
  uint8_t rank[256];
  uint8_t* codes = nullptr;  // nullable: also the input's rank codes, one byte per input byte (with the planes)
  // set by the launcher: 2^19 and 2^16, so that x >> 13 and x >> 16 are the
  // high words of x * mul (the mixer's shifts on the multiply pipe)
  uint32_t mul_shr13, mul_shr16;
};
constexpr int kPartTile = 2048;  // byte positions per CTA tile
uint64_t partition_num_tiles(uint64_t nbytes);
// planes (nullable): also writes the rank-code bit-planes of the tile for the
// verifier (plane p word guard_words + g/32 holds positions g .. g+31), and
// with a.codes the rank codes themselves (a.codes[g] for position g; the
// buffer covers whole tiles).
int launch_anchor_flags(const PartitionArgs& a, uint32_t* bitmap, uint32_t* tile_count,
                        uint32_t* dev_flags, uint32_t* planes, uint64_t plane_words,
                        uint32_t guard_words, uint32_t* tile_first, cudaStream_t s);
// a4: one partition record per anchor, in position order (so string order),
// from the bitmap and the per-tile list offsets; key = (len, H61(substring)).
int launch_partition_records(const PartitionArgs& a, const uint32_t* bitmap, const uint32_t* tile_offset,
                             const uint32_t* tile_first, uint64_t key_base, PRec* recs, cudaStream_t s);
// The fields of n records as separate arrays (any may be null).
int launch_unpack_records(const PRec* recs, uint64_t n, uint32_t* sid, uint32_t* pos, uint32_t* len, uint64_t* key,
                          cudaStream_t s);

// scans (exclusive, in place allowed); temp from scan_temp_bytes
size_t scan_temp_bytes(uint64_t n);
int launch_exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, void* temp,
                              uint32_t* total_out, cudaStream_t s);
int launch_exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, void* temp,
                              uint64_t* total_out, cudaStream_t s);
int launch_exclusive_scan_u32_to_u64(const uint32_t* in, uint64_t* out, uint64_t n, void* temp,
                                     uint64_t* total_out, cudaStream_t s);

// LSD radix sort of 64-bit keys (optionally with 32-bit values) on bits
// [bit_lo, bit_hi).  Ping-pongs between (keys, keys_alt); *result_in_alt
// tells which buffer holds the sorted data.
size_t radix_temp_bytes(uint64_t n);
int radix_sort_u64(uint64_t* keys, uint64_t* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                   uint64_t n, int bit_lo, int bit_hi, void* temp, bool* result_in_alt,
                   cudaStream_t s);

// a5-a6: grouping keys and pair emission.  A group key is hash_bits (<= 32)
// bits of a hash of (len, Karp-Rabin key), then pb_bits bits of the
// position bucket pos / W (W >= K, so the partner of a record under the
// position filter lies in its bucket or the next), then slen_bits bits of
// string length.
struct GroupKeyShape {
  int hash_bits, pb_bits, slen_bits;
  uint32_t W;
};
int launch_make_group_keys(const PRec* recs, uint32_t n_rec, const GroupKeyShape& g, uint64_t* keys, uint32_t* idx,
                           cudaStream_t s);
// Records in group order: out[t] = recs[idx[t]] with run = the hash bits of
// keys[t] and pad = its position bucket.
int launch_gather_records(const uint32_t* idx, const uint64_t* keys, uint32_t n_rec, const GroupKeyShape& g,
                          const PRec* recs, PRec* out, cudaStream_t s);
int launch_count_pairs(const PRec* r, uint32_t n_rec, uint32_t K, const GroupKeyShape& g, uint32_t* count,
                       cudaStream_t s);
// pairs are packed as (i << nb) | j, i < j
int launch_fill_pairs(const PRec* r, uint32_t n_rec, uint32_t K, const GroupKeyShape& g, int nb,
                      const uint64_t* offs, uint64_t* pairs, cudaStream_t s);
// a7 by the pair bitmap: bit (a, b), a < b < n_str, in row a (ceil((n_str - 1
// - a) / 32) words, rows back to back); pair_bitmap_words(n_str) words in all.
// launch_mark_pairs clears the bitmap (unless `clear` is false: the caller
// knows it is zero), sets the bit of every pair the walk finds and counts
// them (raw pairs, duplicates included) into *raw_total; launch_bitmap_rows
// writes the candidates per row, launch_bitmap_write the candidates (i, j)
// sorted, at the row offsets `off` (exclusive scan of the row counts), and
// with `clear` clears the bitmap's words as it reads them.
uint64_t pair_bitmap_words(uint32_t n_str);
int launch_mark_pairs(const PRec* r, uint32_t n_rec, uint32_t K, const GroupKeyShape& g, uint32_t n_str, uint32_t* bm,
                      unsigned long long* raw_total, bool clear, cudaStream_t s);
int launch_bitmap_rows(const uint32_t* bm, uint32_t n_str, uint32_t* cnt, cudaStream_t s);
int launch_bitmap_write(uint32_t* bm, uint32_t n_str, const uint32_t* off, uint32_t* oi, uint32_t* oj, bool clear,
                        cudaStream_t s);
int launch_key_check(const PRec* r, const uint8_t* bytes, const int64_t* offsets, uint32_t n_rec,
                     unsigned long long* mismatches, cudaStream_t s);
// Sharded join: records from separate arrays, pairs packed for a dedup sort.
int launch_pack_records(const uint32_t* sid, const uint32_t* pos, const uint32_t* len, const uint64_t* key,
                        const uint32_t* slen, uint64_t n, PRec* out, cudaStream_t s);
int launch_pack_pairs(const uint32_t* pi, const uint32_t* pj, uint64_t m, int nb, uint64_t* out, cudaStream_t s);
// a7: unique of sorted u64 pairs -> flags; then compaction.
int launch_unique_flags(const uint64_t* sorted, uint64_t n, uint32_t* flags, cudaStream_t s);
// run_start (nullable): run_start[u] = index of candidate u's first raw pair
int launch_compact_pairs(const uint64_t* sorted, const uint32_t* flags, const uint32_t* offs, uint64_t n, int nb,
                         uint32_t* out_i, uint32_t* out_j, uint32_t* run_start, cudaStream_t s);

// a8: banded verification (diagonal bit-vector, one thread per pair).
struct RankTable {
  uint8_t r[256];
};
struct VerifyArgs {
  const uint32_t* planes = nullptr;    // bit-planes of rank codes: plane p at planes + p * plane_words
  uint32_t bits;
  const uint8_t* bytes = nullptr;
  const int64_t* offsets = nullptr;
  uint32_t n_strings;        // pair ids >= n_strings are rejected (flagged, ed = k + 1)
  const uint32_t* pi = nullptr;
  const uint32_t* pj = nullptr;
  const uint32_t* pk = nullptr;        // nullable per-pair band
  const uint32_t* order = nullptr;     // nullable: pair indices in the order to verify them
  const uint32_t* skip_kband = nullptr; // nullable: skip pair t when fed[t] <= skip_kband[t] < K (already settled)
  const uint32_t* first_ed = nullptr;  // nullable: first-pass results fed (else ed itself); a skipped pair copies fed[t] to ed[t]
  const uint32_t* range_lo = nullptr;  // nullable: with range_hi, process order positions [*range_lo, *range_hi) only
  const uint32_t* range_hi = nullptr;
  unsigned long long* skipped = nullptr; // nullable: number of pairs skipped that way
  uint32_t K;
  uint64_t m;
  uint32_t* ed = nullptr;
  unsigned long long* cells = nullptr; // nullable: K-band cells accumulated
  unsigned long long* work = nullptr;  // nullable: word-columns processed (columns x W) accumulated
  uint32_t* dev_flags = nullptr;
  const uint4* pair_geo = nullptr;     // nullable: at order position q, (oA, oB, m, n) of pair order[q], A the
                                       // longer string (n = kGeoBadIds: an id out of range); loaded with order[q]
  uint32_t* out_t = nullptr;           // nullable: indices of the pairs with result <= K, appended (order arbitrary)
  const uint8_t* rank_table = nullptr; // device copy of the 256 rank codes
  const uint8_t* codes = nullptr;      // the input's rank codes, one byte per input byte (digit-table kernels)
  uint64_t nbytes = 0;                 // bytes of the input
  unsigned long long* out_count = nullptr;
};
int verify_words_for(uint32_t kmax);
inline uint32_t plane_guard_words(uint32_t kmax) { return kmax / 64 + (uint32_t)verify_words_for(kmax) + 4; }
// codes (nullable, nbytes + 32 bytes): also the rank code of every byte.
int launch_build_planes(const uint8_t* bytes, uint64_t nbytes, const RankTable& rt, uint32_t bits,
                        uint32_t* planes, uint64_t plane_words, uint32_t guard_words, uint8_t* codes,
                        cudaStream_t s);
// `next` is a device counter the persistent kernel hands pairs out from.
// kernel: MJ_VERIFY_KERNEL_*; lanes: wavefront lanes per pair (0 = fewest that fit).
int launch_verify(const VerifyArgs& a, uint64_t plane_words, uint32_t guard_words, uint32_t kmax,
                  unsigned long long* next, cudaStream_t s, int kernel = MJ_VERIFY_KERNEL_AUTO, int lanes = 0);
int wave_lanes_for(uint32_t kmax);
// lanes of the CTA wavefront (several warps per pair) for bands up to kmax,
// and the fewest lanes of either wavefront form; at most kMaxCtaLanes
constexpr int kMaxCtaLanes = 1024;
int cta_lanes_for(uint32_t kmax);
int fewest_lanes_for(uint32_t kmax);

// Verification order: pair indices longest first (by the shorter length), a
// counting sort over 256 length classes; within a class the order is
// arbitrary.  counts[b] and ranges[2b], ranges[2b+1] = [start, end) of the
// pairs whose shorter length has floor(log2) = b (lengths 0 and 1: b = 0),
// the autotuner's length buckets, contiguous and longest first.  scratch:
// kOrderScratchWords words (256 class counts for each of up to 8 blocks per
// SM of the counting sort).
constexpr int kLenBuckets = 32;
constexpr int kOrderScratchWords = 256 * kNumSMsHint * 8;
// cells (nullable): set to the pairs' K-band cells (mj_stats.band_cells).
// geo (nullable): the pairs' geometry at their order positions (VerifyArgs::
// pair_geo).  Pair ids >= n_str count as empty strings here (the verifier
// flags them).
constexpr uint32_t kGeoBadIds = 0xffffffffu;
// sg: n_str entries of scratch for the strings' {offset, length} (inputs
// are under 4 GB).
int launch_length_order(const uint32_t* ci, const uint32_t* cj, const int64_t* offsets, uint32_t n_str, uint64_t m,
                        uint32_t K, uint32_t* scratch, uint2* sg, uint32_t* order, uint4* geo, uint32_t* counts,
                        uint32_t* ranges, unsigned long long* cells, cudaStream_t s);

// ---- learned first-pass band (MLP 8 -> 64 -> 64 -> 1)
// features of a candidate (i, j), n = min length, d0 = length difference,
// c = matched partition pairs behind the candidate (its multiplicity before
// dedup), pa/pb = partitions of the two strings:
//   log2(1+n)/16, d0/K, c/(T+1), pa/(T+1), pb/(T+1), c/min(pa,pb),
//   log2(1+c)/8, K/(K+100)
constexpr int kBandFeatures = 8;
constexpr int kBandHidden = 64;
constexpr int kBandParams = kBandHidden * kBandFeatures + kBandHidden + kBandHidden * kBandHidden + kBandHidden +
                            kBandHidden + 1;
static_assert(kBandParams == MJ_BAND_PARAMS && kBandFeatures == MJ_BAND_FEATURES, "ABI constants");
int launch_band_features(const uint32_t* ci, const uint32_t* cj, const uint32_t* mult, const uint32_t* parts,
                         const int64_t* offsets, uint64_t m, uint32_t K, uint32_t T, float* X, cudaStream_t s);
int launch_band_forward(const float* P, const float* X, uint64_t m, const uint32_t* gate, uint32_t min_gate,
                        float* out, cudaStream_t s);
size_t band_grad_smem();
int launch_band_grad(const float* P, const float* X, const float* Y, const uint32_t* ed, uint32_t K, uint64_t m,
                     uint64_t batch, uint64_t seed, float tau, float* grad, float* loss, cudaStream_t s);
int launch_band_adam(float* P, const float* G, float* M, float* V, float lr, float b1, float b2, float eps, int step,
                     cudaStream_t s);
int launch_band_fused(const float* P, const uint32_t* ci, const uint32_t* cj, const uint32_t* run_start, uint64_t raw,
                      const uint32_t* parts, const int64_t* offsets, uint64_t m, uint32_t K, uint32_t T, uint32_t margin,
                      uint32_t min_mult, uint32_t* kband, cudaStream_t s);
int launch_gate_hist(const float* X, const uint32_t* ed, uint64_t m, uint32_t K, unsigned int* hist, cudaStream_t s);
int launch_band_rule(const float* yhat, const uint32_t* ci, const uint32_t* cj, const int64_t* offsets, uint64_t m,
                     uint32_t K, uint32_t margin, uint32_t* kband, cudaStream_t s);

// multiplicity of every candidate from the run starts written by the pair
// compaction; partitions per string counted over the records
int launch_multiplicity(const uint32_t* run_start, uint64_t nc, uint64_t raw, uint32_t* mult, cudaStream_t s);
int launch_partition_counts(const PRec* recs, uint64_t n_rec, uint32_t n, uint32_t* parts, cudaStream_t s);
// Learned first passes: the pairs of every first-pass bucket b = 1 .. nb
// (band widths below band K's word count; bucket 0 = no first pass) listed
// contiguously in list, bucket b at [ranges[2b], ranges[2b+1]); cnt holds
// 2 * (kMaxBandBuckets + 2) words of scratch; *first_total = pairs listed.
constexpr uint32_t kMaxBandBuckets = 16;
int launch_band_buckets(const uint32_t* kband, uint64_t m, uint32_t K, uint32_t nb, uint32_t* cnt, uint32_t* ranges,
                        uint32_t* list, unsigned long long* first_total, cudaStream_t s);

// output of the join: the listed pair indices (sorted ascending, which is
// (i, j) order since the candidates are sorted) gathered into (i, j, ED);
// keys/keys_alt: 8 * n bytes each, temp: radix_temp_bytes(n)
int launch_gather_output(const uint32_t* out_t, uint64_t n, uint64_t m, const uint32_t* ci, const uint32_t* cj,
                         const uint32_t* ed, uint64_t* keys, uint64_t* keys_alt, void* temp, uint32_t* oi,
                         uint32_t* oj, uint32_t* oed, cudaStream_t s);

}  // namespace mj
