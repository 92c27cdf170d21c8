// Steps a1 and a5-a7: parameter statistics, grouping of equal partitions,
// pair emission under the length and position filters of Alg. 3,
// and deduplication of the candidate pairs (the last step of Alg. 3's join).
//
// The paper's sequential hash join visits strings in length order and evicts
// bucket entries whose length differs by more than K.  Its result is the set
// of pairs (i != j) holding byte-identical partitions that pass both filters.
// Here that set is produced by sorting the partition records by a group key
// (a hash of (len, substring key) in the high bits, the string length in the
// low bits), so equal partitions are adjacent and ordered by string length
// within the run; every record then walks forward through its run while the
// length difference stays <= K, testing the exact (len, key) equality, i != j,
// and the position filter.  Count -> scan -> fill.
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

// Group key: hash bits of (len, key) above slen_bits bits of string length.
__global__ void group_keys_kernel(const PRec* __restrict__ recs, uint32_t n, int slen_bits, int hash_bits,
                                  uint64_t* __restrict__ keys, uint32_t* __restrict__ idx) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
    const PRec r = load_rec(recs, t);
    uint64_t g = mix64(r.h61 ^ ((uint64_t)r.len * 0x9e3779b97f4a7c15ull));
    keys[t] = ((g >> (64 - hash_bits)) << slen_bits) | (uint64_t)r.slen;
    idx[t] = (uint32_t)t;
  }
}

__global__ void gather_kernel(const uint32_t* __restrict__ idx, const uint64_t* __restrict__ keys, uint32_t n,
                              int slen_bits, const PRec* __restrict__ recs, PRec* __restrict__ o) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
    PRec r = load_rec(recs, idx[t]);
    r.run = (uint32_t)(keys[t] >> slen_bits);
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

// Walks the run of record t; EMIT=false counts, EMIT=true writes pairs.
template <bool EMIT>
__global__ void pairs_kernel(const PRec* __restrict__ r, uint32_t n, uint32_t K, int nb, uint32_t* __restrict__ count,
                             const uint64_t* __restrict__ offs, uint64_t* __restrict__ pairs) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
    const PRec me = load_rec(r, t);
    const int32_t pos = (int32_t)me.pos, slen = (int32_t)me.slen;
    uint32_t c = 0;
    uint64_t out = EMIT ? offs[t] : 0;
    for (uint64_t u = t + 1; u < n; ++u) {
      const PRec o = load_rec(r, u);
      if (o.run != me.run) break;
      if ((int32_t)o.slen - slen > (int32_t)K) break;      // length filter (run sorted by length)
      if (o.len != me.len || o.h61 != me.h61) continue;    // same partition substring
      if (o.sid == me.sid) continue;                       // i != j
      const int32_t pos_u = (int32_t)o.pos;
      const int32_t dl = pos - pos_u, dr = (slen - pos) - ((int32_t)o.slen - pos_u);
      if (abs(dl) + abs(dr) > (int32_t)K) continue;       // position filter
      if (EMIT) {
        const uint32_t a = me.sid < o.sid ? me.sid : o.sid, b = me.sid < o.sid ? o.sid : me.sid;
        pairs[out++] = ((uint64_t)a << nb) | b;
      } else {
        ++c;
      }
    }
    if (!EMIT) count[t] = c;
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

__global__ void ed_flags_kernel(const uint32_t* __restrict__ ed, uint64_t m, uint32_t K, uint32_t* __restrict__ flags) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (uint64_t)gridDim.x * blockDim.x)
    flags[t] = ed[t] <= K ? 1u : 0u;
}

__global__ void compact_out_kernel(const uint32_t* __restrict__ ci, const uint32_t* __restrict__ cj,
                                   const uint32_t* __restrict__ ed, const uint32_t* __restrict__ flags,
                                   const uint32_t* __restrict__ offs, uint64_t m, uint32_t* __restrict__ oi,
                                   uint32_t* __restrict__ oj, uint32_t* __restrict__ oed) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (uint64_t)gridDim.x * blockDim.x) {
    if (flags[t]) {
      uint32_t o = offs[t];
      oi[o] = ci[t];
      oj[o] = cj[t];
      oed[o] = ed[t];
    }
  }
}

// Work-order key of a candidate: longest pairs first (key = N - min length).
__global__ void work_keys_kernel(const uint32_t* __restrict__ ci, const uint32_t* __restrict__ cj,
                                 const int64_t* __restrict__ offsets, uint64_t m, uint64_t N,
                                 uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = ci[t], y = cj[t];
    const int64_t lx = offsets[x + 1] - offsets[x], ly = offsets[y + 1] - offsets[y];
    const int64_t n = lx < ly ? lx : ly;
    keys[t] = N - (uint64_t)n;
    vals[t] = (uint32_t)t;
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

// K-band cells of every candidate, summed (mj_stats.band_cells).
__global__ void band_cells_kernel(const uint32_t* __restrict__ ci, const uint32_t* __restrict__ cj,
                                  const int64_t* __restrict__ offsets, uint64_t m, uint32_t K,
                                  unsigned long long* __restrict__ out) {
  unsigned long long acc = 0;
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < m; u += (uint64_t)gridDim.x * blockDim.x) {
    const int64_t lx = offsets[ci[u] + 1] - offsets[ci[u]], ly = offsets[cj[u] + 1] - offsets[cj[u]];
    const int64_t mm = lx > ly ? lx : ly, n = lx > ly ? ly : lx;
    if (n <= 0) continue;
    int64_t a = mm - (int64_t)K;
    a = a < 0 ? 0 : (a > n ? n : a);
    const int64_t smin = a * (a + 1) / 2 + a * (int64_t)K + (n - a) * mm;
    const int64_t b = (int64_t)K < n ? (int64_t)K : n;
    const int64_t smax = b + (n > (int64_t)K ? (n - (int64_t)K) * (n - (int64_t)K + 1) / 2 : 0);
    acc += (unsigned long long)(smin - smax + n);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

__device__ __forceinline__ uint32_t len_bucket(uint64_t n) { return n <= 1 ? 0u : 63u - (uint32_t)__clzll(n); }

__global__ void bucket_hist_kernel(const uint64_t* __restrict__ keys, uint64_t m, uint64_t N,
                                   uint32_t* __restrict__ counts) {
  __shared__ uint32_t h[kLenBuckets];
  if (threadIdx.x < kLenBuckets) h[threadIdx.x] = 0;
  __syncthreads();
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t b = len_bucket(N - keys[q]);
    atomicAdd(&h[b < kLenBuckets ? b : kLenBuckets - 1], 1u);
  }
  __syncthreads();
  if (threadIdx.x < kLenBuckets && h[threadIdx.x]) atomicAdd(&counts[threadIdx.x], h[threadIdx.x]);
}

// longest first: bucket b starts after all pairs of the buckets above it
__global__ void bucket_scan_kernel(const uint32_t* __restrict__ counts, uint32_t* __restrict__ ranges) {
  uint32_t run = 0;
  for (int b = kLenBuckets - 1; b >= 0; --b) {
    ranges[2 * b] = run;
    run += counts[b];
    ranges[2 * b + 1] = run;
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

int launch_make_group_keys(const PRec* recs, uint32_t n, int slen_bits, int hash_bits, uint64_t* keys,
                           uint32_t* idx, cudaStream_t s) {
  if (!n) return MJ_OK;
  if (hash_bits < 1 || hash_bits > 32 || slen_bits < 1 || slen_bits + hash_bits > 64) return MJ_ERR_ARG;
  group_keys_kernel<<<grid_for(n), 256, 0, s>>>(recs, n, slen_bits, hash_bits, keys, idx);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_gather_records(const uint32_t* idx, const uint64_t* keys, uint32_t n, int slen_bits, const PRec* recs,
                          PRec* o, cudaStream_t s) {
  if (!n) return MJ_OK;
  gather_kernel<<<grid_for(n), 256, 0, s>>>(idx, keys, n, slen_bits, recs, o);
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

int launch_count_pairs(const PRec* r, uint32_t n, uint32_t K, uint32_t* count, cudaStream_t s) {
  if (!n) return MJ_OK;
  pairs_kernel<false><<<grid_for(n), 256, 0, s>>>(r, n, K, 0, count, nullptr, nullptr);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_fill_pairs(const PRec* r, uint32_t n, uint32_t K, int nb, const uint64_t* offs, uint64_t* pairs,
                      cudaStream_t s) {
  if (!n) return MJ_OK;
  pairs_kernel<true><<<grid_for(n), 256, 0, s>>>(r, n, K, nb, nullptr, offs, pairs);
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

int launch_bucket_ranges(const uint64_t* sorted_keys, uint64_t m, uint64_t N, uint32_t* counts, uint32_t* ranges,
                         cudaStream_t s) {
  MJ_CUDA_TRY(cudaMemsetAsync(counts, 0, kLenBuckets * sizeof(uint32_t), s));
  if (m) {
    bucket_hist_kernel<<<grid_for(m), 256, 0, s>>>(sorted_keys, m, N, counts);
    MJ_KERNEL_DONE();
  }
  bucket_scan_kernel<<<1, 1, 0, s>>>(counts, ranges);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_work_keys(const uint32_t* ci, const uint32_t* cj, const int64_t* offsets, uint64_t m, uint64_t N,
                     uint64_t* keys, uint32_t* vals, cudaStream_t s) {
  if (!m) return MJ_OK;
  work_keys_kernel<<<grid_for(m), 256, 0, s>>>(ci, cj, offsets, m, N, keys, vals);
  MJ_KERNEL_DONE();
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

int launch_band_cells(const uint32_t* ci, const uint32_t* cj, const int64_t* offsets, uint64_t m, uint32_t K,
                      unsigned long long* out, cudaStream_t s) {
  MJ_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(unsigned long long), s));
  if (!m) return MJ_OK;
  band_cells_kernel<<<grid_for(m), 256, 0, s>>>(ci, cj, offsets, m, K, out);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_ed_flags(const uint32_t* ed, uint64_t m, uint32_t K, uint32_t* flags, cudaStream_t s) {
  if (!m) return MJ_OK;
  ed_flags_kernel<<<grid_for(m), 256, 0, s>>>(ed, m, K, flags);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_compact_output(const uint32_t* ci, const uint32_t* cj, const uint32_t* ed, const uint32_t* flags,
                          const uint32_t* offs, uint64_t m, uint32_t* oi, uint32_t* oj, uint32_t* oed,
                          cudaStream_t s) {
  if (!m) return MJ_OK;
  compact_out_kernel<<<grid_for(m), 256, 0, s>>>(ci, cj, ed, flags, offs, m, oi, oj, oed);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

}  // namespace mj
