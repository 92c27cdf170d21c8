// Steps a1 and a5-a7: parameter statistics, grouping of equal partitions,
// pair emission under the length and position filters of Alg. 3,
// and deduplication of the candidate pairs (the last step of Alg. 3's join).
//
// The paper's sequential hash join visits strings in length order and evicts
// bucket entries whose length differs by more than K.  Its result is the set
// of pairs (i != j) holding byte-identical partitions that pass both filters.
// Here that set is produced by sorting the partition records by a group key:
// a hash of (len, substring key) in the high bits, then the partition's
// position bucket (position / W with W >= K), then the string length.  Equal
// partitions are adjacent; inside a run they are ordered by position bucket
// and, within a bucket, by string length.  The position filter implies
// |pos_x - pos_y| <= K, so a partner lies in the same bucket or the next one;
// every record walks forward through its own bucket while the length
// difference stays <= K, then through the length window [slen - K, slen + K]
// of the next bucket (found by a galloping search), testing the exact
// (len, key) equality, i != j and the position filter.  Frequent partitions
// (a common word in text) make runs of 10^5 records; the position buckets cut
// each walk to the records that can pass both filters.
//
// Deduplication: either the raw pairs are written (count -> scan -> fill),
// radix-sorted and made unique (which also gives every candidate's
// multiplicity), or every pair sets its bit in a triangular bitmap over all
// pairs i < j, whose rows are then counted and compacted into the sorted
// candidate list.
#include "mj_internal.cuh"

namespace mj {
namespace {

__global__ void byte_hist_kernel(const uint8_t* __restrict__ bytes, uint64_t nbytes,
                                 unsigned long long* __restrict__ hist) {
  __shared__ uint32_t s[256];
  s[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * 16;
  for (uint64_t base = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * 16; base < nbytes; base += stride) {
    if (base + 16 <= nbytes && (((uintptr_t)(bytes + base)) & 15) == 0) {
      uint4 v = __ldg(reinterpret_cast<const uint4*>(bytes + base));
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int b = 0; b < 4; ++b) atomicAdd(&s[(w[k] >> (8 * b)) & 255u], 1u);
      }
    } else {
      for (uint64_t g = base; g < base + 16 && g < nbytes; ++g) atomicAdd(&s[__ldg(bytes + g)], 1u);
    }
  }
  __syncthreads();
  if (s[threadIdx.x]) atomicAdd(&hist[threadIdx.x], (unsigned long long)s[threadIdx.x]);
}

__global__ void max_len_kernel(const int64_t* __restrict__ off, uint32_t n, unsigned long long* __restrict__ out) {
  unsigned long long m = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    int64_t L = off[i + 1] - off[i];
    if ((unsigned long long)L > m) m = (unsigned long long)L;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long y = __shfl_down_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

__global__ void max_u32_kernel(const uint32_t* __restrict__ v, uint64_t n, unsigned int* __restrict__ out) {
  uint32_t m = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    m = max(m, v[i]);
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

__device__ __forceinline__ uint64_t mix64(uint64_t k) {  // MurmurHash3 fmix64
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// Group key: hash bits of (len, key), then pb_bits bits of position bucket
// (pos / W), then slen_bits bits of string length.
__global__ void group_keys_kernel(const PRec* __restrict__ recs, uint32_t n, int slen_bits, int pb_bits, uint32_t W,
                                  int hash_bits, uint64_t* __restrict__ keys, uint32_t* __restrict__ idx) {
  const uint32_t pb_max = pb_bits ? (1u << pb_bits) - 1u : 0u;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
    const PRec r = load_rec(recs, t);
    uint64_t g = mix64(r.h61 ^ ((uint64_t)r.len * 0x9e3779b97f4a7c15ull));
    const uint32_t pb = min(r.pos / W, pb_max);
    keys[t] = (((g >> (64 - hash_bits)) << pb_bits | pb) << slen_bits) | (uint64_t)r.slen;
    idx[t] = (uint32_t)t;
  }
}

// Records in group order; run = the hash bits, pad = the position bucket.
__global__ void gather_kernel(const uint32_t* __restrict__ idx, const uint64_t* __restrict__ keys, uint32_t n,
                              int slen_bits, int pb_bits, const PRec* __restrict__ recs, PRec* __restrict__ o) {
  const uint64_t pb_mask = pb_bits ? (1ull << pb_bits) - 1ull : 0ull;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
    PRec r = load_rec(recs, idx[t]);
    const uint64_t k = keys[t];
    r.run = (uint32_t)(k >> (slen_bits + pb_bits));
    r.pad = (uint32_t)((k >> slen_bits) & pb_mask);
    store_rec(o, t, r);
  }
}

__global__ void unpack_records_kernel(const PRec* __restrict__ recs, uint64_t n, uint32_t* __restrict__ sid,
                                      uint32_t* __restrict__ pos, uint32_t* __restrict__ len,
                                      uint64_t* __restrict__ key) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
    const PRec r = load_rec(recs, t);
    if (sid) sid[t] = r.sid;
    if (pos) pos[t] = r.pos;
    if (len) len[t] = r.len;
    if (key) key[t] = r.h61;
  }
}

// Sort key of a record in group order (the key group_keys_kernel made).
__device__ __forceinline__ uint64_t rec_key(const PRec& o, int pb_shift, int run_shift) {
  return ((uint64_t)o.run << run_shift) | ((uint64_t)o.pad << pb_shift) | (uint64_t)o.slen;
}

// First index u >= lo (u < n) whose sort key is >= target, n if none:
// galloping steps from lo, then a binary search.
__device__ uint64_t key_lower_bound(const PRec* __restrict__ r, uint64_t lo, uint64_t n, uint64_t target, int pb_shift,
                                    int run_shift) {
  uint64_t a = lo, b = lo, step = 1;
  while (b < n && rec_key(load_rec(r, b), pb_shift, run_shift) < target) {
    a = b + 1;
    b = a + step;
    step <<= 1;
  }
  if (b > n) b = n;
  while (a < b) {   // every index < a is below target; b is n or at/above it
    const uint64_t mid = a + (b - a) / 2;
    if (rec_key(load_rec(r, mid), pb_shift, run_shift) < target) a = mid + 1;
    else b = mid;
  }
  return a;
}

enum : int { WALK_COUNT = 0, WALK_FILL = 1, WALK_MARK = 2 };

__device__ __forceinline__ uint64_t tri_words(uint64_t x) {   // sum over y = 1 .. x of ceil(y / 32)
  const uint64_t k = x >> 5, r = x & 31u;
  return 16u * k * (k + 1) + r * (k + 1);
}

// Word offset of row a of the pair bitmap over n strings: row a holds the
// pairs (a, b), a < b < n, as bits b - a - 1 in ceil((n - 1 - a) / 32) words.
__device__ __forceinline__ uint64_t bitmap_row(uint64_t a, uint64_t n) {
  return tri_words(n - 1) - tri_words(n - 1 - a);
}

// Walks the pairs of record t (see the file comment).  WALK_COUNT: count[t]
// = pairs found; WALK_FILL: writes them packed (i << nb | j, i < j) from
// offs[t]; WALK_MARK: sets their bits in the pair bitmap and adds their number
// to *raw_total.
template <int MODE>
__global__ void walk_kernel(const PRec* __restrict__ r, uint32_t n, uint32_t K, int pb_shift, int run_shift, int nb,
                            uint32_t* __restrict__ count, const uint64_t* __restrict__ offs,
                            uint64_t* __restrict__ pairs, uint32_t* __restrict__ bm, uint32_t n_str,
                            unsigned long long* __restrict__ raw_total) {
  unsigned long long raw = 0;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
    const PRec me = load_rec(r, t);
    const int32_t pos = (int32_t)me.pos, slen = (int32_t)me.slen;
    uint32_t c = 0;
    uint64_t out = MODE == WALK_FILL ? offs[t] : 0;
    auto visit = [&](const PRec& o) {
      if (o.len != me.len || o.h61 != me.h61) return;    // same partition substring
      if (o.sid == me.sid) return;                       // i != j
      const int32_t pos_u = (int32_t)o.pos;
      const int32_t dl = pos - pos_u, dr = (slen - pos) - ((int32_t)o.slen - pos_u);
      if (abs(dl) + abs(dr) > (int32_t)K) return;       // position filter
      ++c;
      const uint32_t a = me.sid < o.sid ? me.sid : o.sid, b = me.sid < o.sid ? o.sid : me.sid;
      if (MODE == WALK_FILL) {
        pairs[out++] = ((uint64_t)a << nb) | b;
      } else if (MODE == WALK_MARK) {
        const uint64_t bit = (uint64_t)(b - a - 1);
        atomicOr(bm + bitmap_row(a, n_str) + (bit >> 5), 1u << (bit & 31u));
      }
    };
    // this bucket: later records with string length up to slen + K (the
    // length filter; lengths ascend within a bucket)
    uint64_t u = t + 1;
    bool next = false;
    while (u < n) {
      const PRec o = load_rec(r, u);
      if (o.run != me.run) break;
      if (o.pad != me.pad) {
        next = o.pad == me.pad + 1;
        break;
      }
      if ((int32_t)o.slen - slen > (int32_t)K) {
        next = true;
        ++u;
        break;
      }
      visit(o);
      ++u;
    }
    // the next bucket: string lengths in [slen - K, slen + K]
    if (next) {
      const uint32_t lo_len = me.slen > K ? me.slen - K : 0u;
      const uint64_t target = ((uint64_t)me.run << run_shift) | ((uint64_t)(me.pad + 1) << pb_shift) | lo_len;
      u = key_lower_bound(r, u, n, target, pb_shift, run_shift);
      while (u < n) {
        const PRec o = load_rec(r, u);
        if (o.run != me.run || o.pad != me.pad + 1 || (int32_t)o.slen - slen > (int32_t)K) break;
        visit(o);
        ++u;
      }
    }
    if (MODE == WALK_COUNT) count[t] = c;
    raw += c;
  }
  if (MODE == WALK_MARK) {
    for (int o = 16; o > 0; o >>= 1) raw += __shfl_down_sync(0xffffffffu, raw, o);
    if ((threadIdx.x & 31) == 0 && raw) atomicAdd(raw_total, raw);
  }
}

// cnt[a] = candidates in row a of the pair bitmap (one warp per row, four
// independent word loads per lane in flight).
__global__ void bitmap_rows_kernel(const uint32_t* __restrict__ bm, uint32_t n, uint32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t a = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n; a += warps) {
    const uint64_t w0 = bitmap_row(a, n), w1 = a + 1 < n ? bitmap_row(a + 1, n) : w0;
    uint32_t c = 0;
    for (uint64_t w = w0 + 4 * (uint64_t)lane; w < w1; w += 128) {
      uint32_t v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = w + k < w1 ? __ldcs(bm + w + k) : 0u;
#pragma unroll
      for (int k = 0; k < 4; ++k) c += __popc(v[k]);
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) cnt[a] = c;
  }
}

// The candidates (a, b) of every row, in (a, b) order, from the row offsets:
// per warp step 128 words of the row, four per lane.
// With `clear`, words with bits are cleared after they are read, so the
// bitmap is zero again for the next marking.
__global__ void bitmap_write_kernel(uint32_t* __restrict__ bm, uint32_t n, const uint32_t* __restrict__ off,
                                    uint32_t* __restrict__ oi, uint32_t* __restrict__ oj, bool clear) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t a = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n; a += warps) {
    const uint64_t w0 = bitmap_row(a, n), w1 = a + 1 < n ? bitmap_row(a + 1, n) : w0;
    uint32_t base = off[a];
    for (uint64_t w = w0; w < w1; w += 128) {
      const uint64_t lw = w + 4 * (uint64_t)lane;
      uint32_t v[4];
      uint32_t p = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        v[k] = lw + k < w1 ? __ldcs(bm + lw + k) : 0u;
        p += __popc(v[k]);
      }
      if (clear) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (v[k]) __stcs(bm + lw + k, 0u);
      }
      uint32_t incl = p;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      uint32_t at = base + incl - p;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t b0 = (uint32_t)a + 1u + 32u * (uint32_t)(lw + k - w0);
        uint32_t x = v[k];
        while (x) {
          const uint32_t bit = __ffs(x) - 1;
          x &= x - 1;
          oi[at] = (uint32_t)a;
          oj[at] = b0 + bit;
          ++at;
        }
      }
      base += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

// flags bit 0 check: every record's bytes equal the first record of its
// (len, key) class inside the run.
__global__ void key_check_kernel(const PRec* __restrict__ r, const uint8_t* __restrict__ bytes,
                                 const int64_t* __restrict__ offsets, uint32_t n,
                                 unsigned long long* __restrict__ mismatches) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
    const PRec me = load_rec(r, t);
    // first record of the run with the same (len, key)
    uint64_t f = t;
    PRec first = me;
    for (uint64_t u = t; u-- > 0;) {
      const PRec o = load_rec(r, u);
      if (o.run != me.run) break;
      if (o.len == me.len && o.h61 == me.h61) {
        f = u;
        first = o;
      }
    }
    if (f == t) continue;
    const uint8_t* a = bytes + offsets[me.sid] + me.pos;
    const uint8_t* b = bytes + offsets[first.sid] + first.pos;
    for (uint32_t x = 0; x < me.len; ++x) {
      if (a[x] != b[x]) {
        atomicAdd(mismatches, 1ull);
        break;
      }
    }
  }
}

__global__ void unique_flags_kernel(const uint64_t* __restrict__ s, uint64_t n, uint32_t* __restrict__ flags) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x)
    flags[t] = (t == 0 || s[t] != s[t - 1]) ? 1u : 0u;
}

__global__ void compact_pairs_kernel(const uint64_t* __restrict__ s, const uint32_t* __restrict__ flags,
                                     const uint32_t* __restrict__ offs, uint64_t n, int nb, uint32_t* __restrict__ oi,
                                     uint32_t* __restrict__ oj, uint32_t* __restrict__ run_start) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
    if (flags[t]) {
      uint32_t o = offs[t];
      oi[o] = (uint32_t)(s[t] >> nb);
      oj[o] = (uint32_t)(s[t] & ((1ull << nb) - 1));
      if (run_start) run_start[o] = (uint32_t)t;
    }
  }
}

__global__ void out_keys_kernel(const uint32_t* __restrict__ out_t, uint64_t n, uint64_t* __restrict__ keys) {
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (uint64_t)gridDim.x * blockDim.x)
    keys[u] = out_t[u];
}

__global__ void gather_out_kernel(const uint64_t* __restrict__ keys, uint64_t n, const uint32_t* __restrict__ ci,
                                  const uint32_t* __restrict__ cj, const uint32_t* __restrict__ ed,
                                  uint32_t* __restrict__ oi, uint32_t* __restrict__ oj, uint32_t* __restrict__ oed) {
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t t = keys[u];
    oi[u] = ci[t];
    oj[u] = cj[t];
    oed[u] = ed[t];
  }
}

__global__ void multiplicity_kernel(const uint32_t* __restrict__ run_start, uint64_t nc, uint64_t raw,
                                    uint32_t* __restrict__ mult) {
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nc; u += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t e = u + 1 < nc ? run_start[u + 1] : raw;
    mult[u] = (uint32_t)(e - run_start[u]);
  }
}

// parts[s] = number of partitions of string s, counted over all records
// (with parallel repetition the records come repetition by repetition, so
// they are counted, not searched)
// Records of one string are mostly consecutive, so the lanes of a warp that
// hold the same string add their count in one atomic (from the lowest lane).
__global__ void partition_counts_kernel(const PRec* __restrict__ recs, uint64_t n_rec, uint32_t n,
                                        uint32_t* __restrict__ parts) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) - lane;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = warp0; base < n_rec; base += stride) {   // warp-uniform
    const uint64_t t = base + lane;
    const uint32_t sid = t < n_rec ? __ldg(&recs[t].sid) : 0xffffffffu;
    const uint32_t peers = __match_any_sync(0xffffffffu, sid);
    if (sid < n && lane == __ffs(peers) - 1) atomicAdd(parts + sid, (uint32_t)__popc(peers));
  }
}

// First-pass bucket of a learned band k (0: no first pass).  Band widths
// (words of k + 1 bits) below the band-K word count wK: one bucket per word
// count when wK <= 8, else power-of-two ranges [1,2), [2,4), ...
__device__ __forceinline__ uint32_t first_pass_bucket(uint32_t k, uint32_t K, uint32_t wK) {
  if (k >= K) return 0;
  const uint32_t kw = (k + 1 + 31) / 32;
  if (kw >= wK) return 0;
  return wK <= 8 ? kw : 32 - __clz(kw);
}

// cnt[b] += pairs t with first-pass bucket b >= 1 (warp-aggregated)
__global__ void band_bucket_count_kernel(const uint32_t* __restrict__ kband, uint64_t m, uint32_t K, uint32_t wK,
                                         uint32_t* __restrict__ cnt) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t b = first_pass_bucket(kband[t], K, wK);
    const uint32_t active = __activemask();
    const uint32_t peers = __match_any_sync(active, b);
    if (b && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(cnt + b, __popc(peers));
  }
}

// ranges[2b], ranges[2b+1] = [start, end) of bucket b (b = 1 .. nb) in the
// list, from the counts; cursor[b] = start; *first_total = all first-pass pairs
__global__ void band_bucket_ranges_kernel(const uint32_t* __restrict__ cnt, uint32_t nb, uint32_t* __restrict__ ranges,
                                          uint32_t* __restrict__ cursor, unsigned long long* __restrict__ first_total) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    uint32_t run = 0;
    ranges[0] = ranges[1] = 0;
    for (uint32_t b = 1; b <= nb; ++b) {
      ranges[2 * b] = run;
      cursor[b] = run;
      run += cnt[b];
      ranges[2 * b + 1] = run;
    }
    if (first_total) *first_total = run;
  }
}

// list[cursor[b]++] = t for every pair t with first-pass bucket b >= 1
__global__ void band_bucket_scatter_kernel(const uint32_t* __restrict__ kband, uint64_t m, uint32_t K, uint32_t wK,
                                           uint32_t* __restrict__ cursor, uint32_t* __restrict__ list) {
  const int lane = threadIdx.x & 31;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t b = first_pass_bucket(kband[t], K, wK);
    const uint32_t active = __activemask();
    const uint32_t peers = __match_any_sync(active, b);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (b && lane == leader) base = atomicAdd(cursor + b, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    if (b) list[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)t;
  }
}


// ---- verification order: longest pairs first, by a counting sort of the
// pairs' shorter lengths n over 256 length classes: n itself below 8, else
// floor(log2 n) and the next three bits.  Classes are monotone in n, and the
// pairs of one floor(log2 n) bucket (the autotuner's unit) are a run of
// consecutive classes.  Order within a class is arbitrary.
constexpr int kOrderClasses = 256;

__device__ __forceinline__ uint32_t length_class(uint64_t n) {
  if (n < 8) return (uint32_t)n;
  const uint32_t e = 63u - (uint32_t)__clzll(n);   // >= 3
  return (e - 2u) * 8u + (uint32_t)((n >> (e - 3u)) & 7u);
}

// Offsets and lengths of pair t's strings from the per-string table sg
// ({offset, length}, 32-bit: inputs are under 4 GB); ids >= n_str read
// nothing and count as empty strings.
struct PairLens {
  uint32_t ox, lx, oy, ly;
  bool bad;
};
__device__ __forceinline__ PairLens pair_lens(const uint32_t* __restrict__ ci, const uint32_t* __restrict__ cj,
                                              const uint2* __restrict__ sg, uint32_t n_str, uint64_t t) {
  const uint32_t x = ci[t], y = cj[t];
  PairLens r{0, 0, 0, 0, x >= n_str || y >= n_str};
  if (!r.bad) {
    const uint2 gx = __ldg(sg + x), gy = __ldg(sg + y);
    r.ox = gx.x;
    r.lx = gx.y;
    r.oy = gy.x;
    r.ly = gy.y;
  }
  return r;
}

// sg[i] = {offset, length} of string i.
__global__ void string_geo_kernel(const int64_t* __restrict__ offsets, uint32_t n, uint2* __restrict__ sg) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const int64_t o = offsets[i];
    sg[i] = make_uint2((uint32_t)o, (uint32_t)(offsets[i + 1] - o));
  }
}

__device__ __forceinline__ uint64_t band_cells_of(int64_t m, int64_t n, int64_t K) {   // m >= n
  if (n <= 0) return 0;
  if (m < ((int64_t)1 << 31) && K < ((int64_t)1 << 31)) {   // the same sums with 32-bit factors
    const uint32_t M = (uint32_t)m, N = (uint32_t)n, KK = (uint32_t)K;
    const uint32_t a = M > KK ? min(M - KK, N) : 0u;
    const uint64_t smin = (((uint64_t)a * (a + 1u)) >> 1) + (uint64_t)a * KK + (uint64_t)(N - a) * M;
    const uint32_t b = min(KK, N);
    const uint64_t smax = b + (N > KK ? (((uint64_t)(N - KK) * (N - KK + 1u)) >> 1) : 0ull);
    return smin - smax + N;
  }
  int64_t a = m - K;
  a = a < 0 ? 0 : (a > n ? n : a);
  const int64_t smin = a * (a + 1) / 2 + a * K + (n - a) * m;
  const int64_t b = K < n ? K : n;
  const int64_t smax = b + (n > K ? (n - K) * (n - K + 1) / 2 : 0);
  return (uint64_t)(smin - smax + n);
}

// The histogram and the scatter give block b of G the pairs [b R, (b + 1) R)
// (R a multiple of the scatter's chunk): the histogram writes each block's
// class counts, block-major (bh[b * 256 + c]); the scan turns them into each
// block's first position per class, so the scatter needs no global atomics.
constexpr int kOrderThreads = 256;
constexpr int kOrderItems = 8;
constexpr uint64_t kOrderChunk = (uint64_t)kOrderThreads * kOrderItems;
constexpr int kOrderBlocksMax = kNumSMsHint * 8;

// Class histogram of each block's pairs; with cells non-null also their
// K-band cells (mj_stats.band_cells), summed.
__global__ void __launch_bounds__(kOrderThreads) order_hist_kernel(const uint32_t* __restrict__ ci,
                                                                   const uint32_t* __restrict__ cj,
                                                                   const uint2* __restrict__ sg, uint32_t n_str,
                                                                   uint64_t m, uint64_t R, uint32_t K,
                                                                   uint32_t* __restrict__ bh,
                                                                   unsigned long long* __restrict__ cells) {
  __shared__ uint32_t h[kOrderClasses];
  for (int c = threadIdx.x; c < kOrderClasses; c += blockDim.x) h[c] = 0;
  __syncthreads();
  unsigned long long acc = 0;
  const uint64_t t0 = (uint64_t)blockIdx.x * R;
  const uint64_t t1 = t0 + R < m ? t0 + R : m;
  for (uint64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
    const PairLens L = pair_lens(ci, cj, sg, n_str, t);
    const uint32_t n = L.lx < L.ly ? L.lx : L.ly, mm = L.lx < L.ly ? L.ly : L.lx;
    atomicAdd(&h[length_class((uint64_t)n)], 1u);
    if (cells) acc += band_cells_of(mm, n, K);
  }
  if (cells) {
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(cells, acc);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < kOrderClasses; c += blockDim.x) bh[(uint64_t)blockIdx.x * kOrderClasses + c] = h[c];
}

// One block of kOrderClasses threads.  Class c's pairs start at cursor c
// (classes in descending order: longest first) and block b's pairs of
// class c at cursor c + the counts of the blocks before b, written over bh;
// counts[b] and ranges[2b], ranges[2b+1] = the pairs and [start, end) of
// floor(log2) bucket b (n <= 1 in bucket 0).
__global__ void order_scan_kernel(uint32_t* __restrict__ bh, uint32_t G, uint32_t* __restrict__ counts,
                                  uint32_t* __restrict__ ranges) {
  __shared__ uint32_t v[kOrderClasses], tot[kOrderClasses], cursor[kOrderClasses];
  const int c = threadIdx.x;
  uint32_t sum = 0;
#pragma unroll 8
  for (uint32_t b = 0; b < G; ++b) sum += bh[(uint64_t)b * kOrderClasses + c];
  tot[c] = sum;
  __syncthreads();
  // exclusive scan over classes in descending order
  v[c] = tot[kOrderClasses - 1 - c];
  __syncthreads();
  for (int o = 1; o < kOrderClasses; o <<= 1) {
    const uint32_t y = c >= o ? v[c - o] : 0u;
    __syncthreads();
    v[c] += y;
    __syncthreads();
  }
  const int cls = kOrderClasses - 1 - c;
  cursor[cls] = v[c] - tot[cls];
  __syncthreads();
  uint32_t run = cursor[c];
  for (uint32_t b = 0; b < G; ++b) {
    const uint64_t at = (uint64_t)b * kOrderClasses + c;
    const uint32_t x = bh[at];
    bh[at] = run;
    run += x;
  }
  if (c < kLenBuckets) {
    // classes of bucket b: n in [2^b, 2^(b+1)) (b = 0: n <= 1)
    const int b = c;
    int lo, hi;   // classes [lo, hi]
    if (b == 0) { lo = 0; hi = 1; }
    else if (b == 1) { lo = 2; hi = 3; }
    else if (b == 2) { lo = 4; hi = 7; }
    else { lo = (b - 2) * 8; hi = lo + 7; }
    // longest first: class hi comes first; the bucket spans [cursor[hi], cursor[lo] + tot[lo])
    uint32_t cnt = 0;
    for (int k = lo; k <= hi; ++k) cnt += tot[k];
    counts[b] = cnt;
    ranges[2 * b] = cursor[hi];
    ranges[2 * b + 1] = cursor[hi] + cnt;
  }
}

// Scatter of each block's pairs into the order, a chunk of kOrderChunk pairs
// at a time: ranks within the chunk from shared-memory counters, positions
// from the block's running base per class.
__global__ void __launch_bounds__(kOrderThreads) order_scatter_kernel(const uint32_t* __restrict__ ci,
                                                                     const uint32_t* __restrict__ cj,
                                                                     const uint2* __restrict__ sg,
                                                                     uint32_t n_str, uint64_t m, uint64_t R,
                                                                     const uint32_t* __restrict__ bbase,
                                                                     uint32_t* __restrict__ order,
                                                                     uint4* __restrict__ geo) {
  __shared__ uint32_t h[kOrderClasses];
  __shared__ uint32_t run[kOrderClasses];
  for (int c = threadIdx.x; c < kOrderClasses; c += kOrderThreads) {
    h[c] = 0;
    run[c] = bbase[(uint64_t)blockIdx.x * kOrderClasses + c];
  }
  __syncthreads();
  const uint64_t t0 = (uint64_t)blockIdx.x * R;
  const uint64_t t1 = t0 + R < m ? t0 + R : m;
  for (uint64_t base = t0; base < t1; base += kOrderChunk) {
    uint32_t cls[kOrderItems], rank[kOrderItems];
    uint4 g[kOrderItems];
#pragma unroll
    for (int k = 0; k < kOrderItems; ++k) {
      const uint64_t t = base + (uint64_t)k * kOrderThreads + threadIdx.x;
      cls[k] = 0xffffffffu;
      if (t < t1) {
        const PairLens L = pair_lens(ci, cj, sg, n_str, t);
        const bool xa = L.lx >= L.ly;
        g[k] = L.bad ? make_uint4(0u, 0u, 0u, kGeoBadIds)
                     : make_uint4(xa ? L.ox : L.oy, xa ? L.oy : L.ox, xa ? L.lx : L.ly, xa ? L.ly : L.lx);
        cls[k] = length_class((uint64_t)(L.lx < L.ly ? L.lx : L.ly));
        rank[k] = atomicAdd(&h[cls[k]], 1u);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kOrderItems; ++k) {
      const uint64_t t = base + (uint64_t)k * kOrderThreads + threadIdx.x;
      if (cls[k] != 0xffffffffu) {
        const uint32_t pos = run[cls[k]] + rank[k];
        order[pos] = (uint32_t)t;
        if (geo) geo[pos] = g[k];
      }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < kOrderClasses; c += kOrderThreads) {
      run[c] += h[c];
      h[c] = 0;
    }
    __syncthreads();
  }
}

// Records given as separate arrays (a sharded join's exchanged records).
__global__ void pack_records_kernel(const uint32_t* __restrict__ sid, const uint32_t* __restrict__ pos,
                                    const uint32_t* __restrict__ len, const uint64_t* __restrict__ key,
                                    const uint32_t* __restrict__ slen, uint64_t n, PRec* __restrict__ out) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
    PRec r;
    r.h61 = key[t];
    r.run = 0;
    r.slen = slen[t];
    r.len = len[t];
    r.sid = sid[t];
    r.pos = pos[t];
    r.pad = 0;
    store_rec(out, t, r);
  }
}

// Pairs as packed keys (min << nb | max) for the dedup sort.
__global__ void pack_pairs_kernel(const uint32_t* __restrict__ pi, const uint32_t* __restrict__ pj, uint64_t m, int nb,
                                  uint64_t* __restrict__ out) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t a = pi[t], b = pj[t];
    out[t] = ((uint64_t)(a < b ? a : b) << nb) | (a < b ? b : a);
  }
}

unsigned grid_for(uint64_t n, int threads = 256) {
  uint64_t g = (n + threads - 1) / threads;
  uint64_t cap = (uint64_t)kNumSMsHint * 32;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

int launch_byte_histogram(const uint8_t* bytes, uint64_t nbytes, unsigned long long* hist, cudaStream_t s) {
  MJ_CUDA_TRY(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned long long), s));
  if (!nbytes) return MJ_OK;
  byte_hist_kernel<<<grid_for((nbytes + 15) / 16), 256, 0, s>>>(bytes, nbytes, hist);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_max_u32(const uint32_t* v, uint64_t n, unsigned int* out, cudaStream_t s) {
  MJ_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(unsigned int), s));
  if (!n) return MJ_OK;
  max_u32_kernel<<<grid_for(n), 256, 0, s>>>(v, n, out);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_max_length(const int64_t* offsets, uint32_t n, unsigned long long* out, cudaStream_t s) {
  MJ_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(unsigned long long), s));
  if (!n) return MJ_OK;
  max_len_kernel<<<grid_for(n), 256, 0, s>>>(offsets, n, out);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_make_group_keys(const PRec* recs, uint32_t n, const GroupKeyShape& g, uint64_t* keys, uint32_t* idx,
                           cudaStream_t s) {
  if (!n) return MJ_OK;
  if (g.hash_bits < 1 || g.hash_bits > 32 || g.slen_bits < 1 || g.pb_bits < 0 || g.W < 1 ||
      g.slen_bits + g.pb_bits + g.hash_bits > 64)
    return MJ_ERR_ARG;
  group_keys_kernel<<<grid_for(n), 256, 0, s>>>(recs, n, g.slen_bits, g.pb_bits, g.W, g.hash_bits, keys, idx);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_gather_records(const uint32_t* idx, const uint64_t* keys, uint32_t n, const GroupKeyShape& g,
                          const PRec* recs, PRec* o, cudaStream_t s) {
  if (!n) return MJ_OK;
  gather_kernel<<<grid_for(n), 256, 0, s>>>(idx, keys, n, g.slen_bits, g.pb_bits, recs, o);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_unpack_records(const PRec* recs, uint64_t n, uint32_t* sid, uint32_t* pos, uint32_t* len, uint64_t* key,
                          cudaStream_t s) {
  if (!n) return MJ_OK;
  unpack_records_kernel<<<grid_for(n), 256, 0, s>>>(recs, n, sid, pos, len, key);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_count_pairs(const PRec* r, uint32_t n, uint32_t K, const GroupKeyShape& g, uint32_t* count,
                       cudaStream_t s) {
  if (!n) return MJ_OK;
  walk_kernel<WALK_COUNT><<<grid_for(n), 256, 0, s>>>(r, n, K, g.slen_bits, g.slen_bits + g.pb_bits, 0, count,
                                                      nullptr, nullptr, nullptr, 0, nullptr);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_fill_pairs(const PRec* r, uint32_t n, uint32_t K, const GroupKeyShape& g, int nb, const uint64_t* offs,
                      uint64_t* pairs, cudaStream_t s) {
  if (!n) return MJ_OK;
  walk_kernel<WALK_FILL><<<grid_for(n), 256, 0, s>>>(r, n, K, g.slen_bits, g.slen_bits + g.pb_bits, nb, nullptr,
                                                     offs, pairs, nullptr, 0, nullptr);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

uint64_t pair_bitmap_words(uint32_t n_str) {
  if (n_str < 2) return 0;
  const uint64_t x = n_str - 1, k = x >> 5, r = x & 31u;
  return 16u * k * (k + 1) + r * (k + 1);
}

int launch_mark_pairs(const PRec* r, uint32_t n, uint32_t K, const GroupKeyShape& g, uint32_t n_str, uint32_t* bm,
                      unsigned long long* raw_total, bool clear, cudaStream_t s) {
  MJ_CUDA_TRY(cudaMemsetAsync(raw_total, 0, sizeof(unsigned long long), s));
  const uint64_t words = pair_bitmap_words(n_str);
  if (words && clear) MJ_CUDA_TRY(cudaMemsetAsync(bm, 0, words * 4, s));
  if (!n || !words) return MJ_OK;
  walk_kernel<WALK_MARK><<<grid_for(n), 256, 0, s>>>(r, n, K, g.slen_bits, g.slen_bits + g.pb_bits, 0, nullptr,
                                                     nullptr, nullptr, bm, n_str, raw_total);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_bitmap_rows(const uint32_t* bm, uint32_t n_str, uint32_t* cnt, cudaStream_t s) {
  if (!n_str) return MJ_OK;
  bitmap_rows_kernel<<<grid_for((uint64_t)n_str * 32), 256, 0, s>>>(bm, n_str, cnt);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_bitmap_write(uint32_t* bm, uint32_t n_str, const uint32_t* off, uint32_t* oi, uint32_t* oj, bool clear,
                        cudaStream_t s) {
  if (!n_str) return MJ_OK;
  bitmap_write_kernel<<<grid_for((uint64_t)n_str * 32), 256, 0, s>>>(bm, n_str, off, oi, oj, clear);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_key_check(const PRec* r, const uint8_t* bytes, const int64_t* offsets, uint32_t n,
                     unsigned long long* mismatches, cudaStream_t s) {
  if (!n) return MJ_OK;
  key_check_kernel<<<grid_for(n), 256, 0, s>>>(r, bytes, offsets, n, mismatches);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_unique_flags(const uint64_t* sorted, uint64_t n, uint32_t* flags, cudaStream_t s) {
  if (!n) return MJ_OK;
  unique_flags_kernel<<<grid_for(n), 256, 0, s>>>(sorted, n, flags);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_compact_pairs(const uint64_t* sorted, const uint32_t* flags, const uint32_t* offs, uint64_t n, int nb,
                         uint32_t* out_i, uint32_t* out_j, uint32_t* run_start, cudaStream_t s) {
  if (!n) return MJ_OK;
  compact_pairs_kernel<<<grid_for(n), 256, 0, s>>>(sorted, flags, offs, n, nb, out_i, out_j, run_start);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_length_order(const uint32_t* ci, const uint32_t* cj, const int64_t* offsets, uint32_t n_str, uint64_t m,
                        uint32_t K, uint32_t* scratch, uint2* sg, uint32_t* order, uint4* geo, uint32_t* counts,
                        uint32_t* ranges, unsigned long long* cells, cudaStream_t s) {
  if (n_str) {
    string_geo_kernel<<<grid_for(n_str), 256, 0, s>>>(offsets, n_str, sg);
    MJ_KERNEL_DONE();
  }
  // G blocks of R pairs (R a whole number of chunks), at least one block
  const uint64_t chunks = (m + kOrderChunk - 1) / kOrderChunk;
  const uint32_t G = (uint32_t)(chunks < 1 ? 1 : (chunks < (uint64_t)kOrderBlocksMax ? chunks : kOrderBlocksMax));
  const uint64_t R = (chunks + G - 1) / G * kOrderChunk;
  if (cells) MJ_CUDA_TRY(cudaMemsetAsync(cells, 0, sizeof(unsigned long long), s));
  order_hist_kernel<<<G, kOrderThreads, 0, s>>>(ci, cj, sg, n_str, m, R, K, scratch, cells);
  MJ_KERNEL_DONE();
  order_scan_kernel<<<1, kOrderClasses, 0, s>>>(scratch, G, counts, ranges);
  MJ_KERNEL_DONE();
  if (m) {
    order_scatter_kernel<<<G, kOrderThreads, 0, s>>>(ci, cj, sg, n_str, m, R, scratch, order, geo);
    MJ_KERNEL_DONE();
  }
  return MJ_OK;
}

int launch_multiplicity(const uint32_t* run_start, uint64_t nc, uint64_t raw, uint32_t* mult, cudaStream_t s) {
  if (!nc) return MJ_OK;
  multiplicity_kernel<<<grid_for(nc), 256, 0, s>>>(run_start, nc, raw, mult);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_partition_counts(const PRec* recs, uint64_t n_rec, uint32_t n, uint32_t* parts, cudaStream_t s) {
  if (!n) return MJ_OK;
  MJ_CUDA_TRY(cudaMemsetAsync(parts, 0, (size_t)n * sizeof(uint32_t), s));
  if (!n_rec) return MJ_OK;
  partition_counts_kernel<<<grid_for(n_rec), 256, 0, s>>>(recs, n_rec, n, parts);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_band_buckets(const uint32_t* kband, uint64_t m, uint32_t K, uint32_t nb, uint32_t* cnt, uint32_t* ranges,
                        uint32_t* list, unsigned long long* first_total, cudaStream_t s) {
  const uint32_t wK = (K + 1 + 31) / 32;
  MJ_CUDA_TRY(cudaMemsetAsync(cnt, 0, 4 * (kMaxBandBuckets + 2), s));
  if (m) {
    band_bucket_count_kernel<<<grid_for(m), 256, 0, s>>>(kband, m, K, wK, cnt);
    MJ_KERNEL_DONE();
  }
  uint32_t* cursor = cnt + kMaxBandBuckets + 2;
  band_bucket_ranges_kernel<<<1, 32, 0, s>>>(cnt, nb, ranges, cursor, first_total);
  MJ_KERNEL_DONE();
  if (m) {
    band_bucket_scatter_kernel<<<grid_for(m), 256, 0, s>>>(kband, m, K, wK, cursor, list);
    MJ_KERNEL_DONE();
  }
  return MJ_OK;
}


int launch_gather_output(const uint32_t* out_t, uint64_t n, uint64_t m, const uint32_t* ci, const uint32_t* cj,
                         const uint32_t* ed, uint64_t* keys, uint64_t* keys_alt, void* temp, uint32_t* oi,
                         uint32_t* oj, uint32_t* oed, cudaStream_t s) {
  if (!n) return MJ_OK;
  out_keys_kernel<<<grid_for(n), 256, 0, s>>>(out_t, n, keys);
  MJ_KERNEL_DONE();
  int bits = 1;
  while (bits < 64 && ((m - 1) >> bits)) ++bits;
  bool alt = false;
  MJ_TRY(radix_sort_u64(keys, keys_alt, nullptr, nullptr, n, 0, bits, temp, &alt, s));
  gather_out_kernel<<<grid_for(n), 256, 0, s>>>(alt ? keys_alt : keys, n, ci, cj, ed, oi, oj, oed);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_pack_records(const uint32_t* sid, const uint32_t* pos, const uint32_t* len, const uint64_t* key,
                        const uint32_t* slen, uint64_t n, PRec* out, cudaStream_t s) {
  if (!n) return MJ_OK;
  pack_records_kernel<<<grid_for(n), 256, 0, s>>>(sid, pos, len, key, slen, n, out);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_pack_pairs(const uint32_t* pi, const uint32_t* pj, uint64_t m, int nb, uint64_t* out, cudaStream_t s) {
  if (!m) return MJ_OK;
  pack_pairs_kernel<<<grid_for(m), 256, 0, s>>>(pi, pj, m, nb, out);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

}  // namespace mj
