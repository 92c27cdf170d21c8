// Steps a2-a4: q-gram hashing, anchors (strict local minima) and partition
// records — Alg. 1 (Partition-String) and Alg. 2 (Find-Anchor) of the MinJoin
// paper, computed for all strings at once over the concatenated bytes.
//
// Work decomposition: the concatenation is cut into tiles of kPartTile byte
// positions, one CTA per tile.  A tile stages its bytes (as rank codes) plus a
// halo of r_max positions on the left and r_max + q - 1 on the right in shared
// memory, computes Pi of every q-gram start in tile+halo there, then tests the
// tile's own positions.  A position's string is found by binary search over
// the offsets; the strict-minimum test of a position never looks outside its
// own string (positions i in [r, m-1-r] of a string have all their 2r
// neighbours inside the string's q-gram range), so halos that run into a
// neighbouring string are harmless.
#include "mj_internal.cuh"

namespace mj {
namespace {

// MurmurHash3 32-bit finaliser (A. Appleby, public domain): the random
// function Pi on q-grams whose packed code fits 32 bits.  A bijection, so
// equal values mean equal q-grams.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// MurmurHash3 64-bit finaliser, for packed codes wider than 32 bits.
__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// Largest s with offsets[s] <= g (g < offsets[n]): the string holding byte g.
__device__ __forceinline__ uint32_t string_of(const int64_t* __restrict__ off, uint32_t n, uint64_t g) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if ((uint64_t)__ldg(off + mid) <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// Alg. 2's neighbourhood radius with floor division and the r_min clamp.
__device__ __forceinline__ int32_t radius_of(int64_t slen, int32_t q, int32_t T, int32_t r_min) {
  int64_t num = slen - q + 1 - T, den = 2 * (int64_t)T + 2;
  int64_t r = num >= 0 ? num / den : -((-num + den - 1) / den);
  return r < r_min ? r_min : (int32_t)r;
}

constexpr int kThreads = 256;
constexpr int kPerThread = kPartTile / kThreads;  // positions per thread in the emit kernel
constexpr int kWarpPositions = kPartTile / (kThreads / 32);
constexpr int kMaxTileStrings = 1024;             // string offsets cached per tile

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline int floor_log2(int x) {
  int t = 0;
  while ((2 << t) <= x) ++t;
  return t;
}

// Shared memory of the anchor kernel: staged rank codes, then the range-minimum
// table of Pi values: level t holds min(h[x .. x + 2^t - 1]) for every x.
template <class HT>
__host__ __device__ inline size_t anchor_smem_bytes(int r_max, int q) {
  size_t span = kPartTile + 2 * (size_t)r_max;
  int levels = floor_log2(r_max < 1 ? 1 : r_max) + 1;
  return 256 + align16(span + q) + (size_t)levels * span * sizeof(HT);
}

// Pi of the q-gram whose packed code is `code` (see mjo_hash_qgrams for the
// definition shared with the paper's Table 2 form).
template <class HT, bool WIDE, bool TABLE>
__device__ __forceinline__ HT pi_value(uint64_t code, const PartitionArgs& a) {
  if (TABLE) return (HT)__ldg(a.table + code);
  if (WIDE) return (HT)fmix64(code ^ a.seed64);
  return (HT)fmix32((uint32_t)code ^ a.seed32);
}

// tile_first[t] = the string holding byte t * kPartTile: every non-empty
// string marks the tiles that start inside it.
__global__ void tile_first_kernel(const int64_t* __restrict__ offsets, uint32_t n, uint64_t tiles,
                                  uint32_t* __restrict__ tile_first) {
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (uint64_t)gridDim.x * blockDim.x) {
    const int64_t lo = offsets[s], hi = offsets[s + 1];
    if (hi <= lo) continue;
    uint64_t t = ((uint64_t)lo + kPartTile - 1) / kPartTile;
    for (; t < tiles && (int64_t)(t * kPartTile) < hi; ++t) tile_first[t] = (uint32_t)s;
  }
}

// Alg. 2 for one tile: a position i of string s (0-based, m = |s| - q + 1
// q-gram starts, radius r) is an anchor iff i = 0, or r <= i <= m - 1 - r and
// h[i] is strictly below both min(h[i-r .. i-1]) and min(h[i+1 .. i+r]).
// Both window minima come from a sparse table over the tile's Pi values: a
// window of length r is the union of two windows of length 2^t, t =
// floor(log2 r).  Every step is branch-free across a warp.
template <class HT, bool WIDE, bool TABLE>
__global__ void __launch_bounds__(kThreads) anchor_flags_kernel(PartitionArgs a, uint32_t* __restrict__ bitmap,
                                                                uint32_t* __restrict__ tile_count,
                                                                uint32_t* __restrict__ dev_flags,
                                                                uint32_t* __restrict__ planes, uint64_t plane_words,
                                                                uint32_t guard_words,
                                                                const uint32_t* __restrict__ tile_first) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int64_t s_off[kMaxTileStrings + 1];   // offsets[sid0 .. sid0 + cap]
  __shared__ uint32_t s_ns;
  __shared__ uint32_t s_warp[kThreads / 32];
  const int HL = a.r_max;
  const int span = kPartTile + 2 * HL;        // positions holding a Pi value
  const int nb = span + (int)a.q;              // staged symbols
  const int levels = floor_log2(HL < 1 ? 1 : HL) + 1;
  uint8_t* s_rank = smem;                      // 256-entry rank table
  uint8_t* s_code = smem + 256;                // staged rank codes
  HT* s_h = reinterpret_cast<HT*>(smem + 256 + align16(nb));   // level 0; level t at s_h + t * span

  const uint64_t g0 = (uint64_t)blockIdx.x * kPartTile;
  const int64_t base = (int64_t)g0 - HL;       // global position of s_code[0] and s_h[0]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

  s_rank[threadIdx.x] = a.rank[threadIdx.x];
  const uint32_t sid0 = __ldg(tile_first + blockIdx.x);
  const uint32_t cap = min((uint32_t)kMaxTileStrings, a.n - sid0);
  for (uint32_t t = threadIdx.x; t <= cap; t += kThreads) s_off[t] = __ldg(a.offsets + sid0 + t);
  __syncthreads();
  // rank codes of [base, base + nb), 16-byte loads where aligned and in range
  {
    const int64_t al = base & ~int64_t(15);
    for (int64_t c = al + 16 * (int64_t)threadIdx.x; c < base + nb; c += 16 * kThreads) {
      if (c >= 0 && (uint64_t)c + 16 <= a.nbytes) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(a.bytes + c));
        const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int b = 0; b < 16; ++b) {
          const int64_t idx = c + b - base;
          if (idx >= 0 && idx < nb) s_code[idx] = s_rank[(w4[b >> 2] >> (8 * (b & 3))) & 255u];
        }
      } else {
        for (int b = 0; b < 16; ++b) {
          const int64_t g = c + b, idx = g - base;
          if (idx >= 0 && idx < nb) s_code[idx] = (g >= 0 && (uint64_t)g < a.nbytes) ? s_rank[__ldg(a.bytes + g)] : 0;
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // strings that may hold tile positions: indices 0 .. ns-1 of s_off
    uint32_t lo = 0, hi = cap;
    const int64_t gend = (int64_t)g0 + kPartTile;
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) >> 1;
      if (s_off[mid] < gend) lo = mid; else hi = mid;
    }
    s_ns = lo + 1;
  }
  // bit-planes of the tile's rank codes for the verifier (one ballot per word)
  if (planes) {
    for (int w = wid; w < kPartTile / 32; w += kThreads / 32) {
      const uint32_t r = s_code[HL + 32 * w + lane];
      const uint64_t word = guard_words + (g0 >> 5) + w;
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        if (p < (int)a.bits) {
          const uint32_t bw = __ballot_sync(0xffffffffu, (r >> p) & 1u);
          if (lane == p) planes[(uint64_t)p * plane_words + word] = bw;
        }
      }
    }
  }

  // Pi of every q-gram start in [0, span): contiguous chunk per thread,
  // packed code rolled forward (first symbol most significant).
  {
    const int per = (span + kThreads - 1) / kThreads;
    const int p0 = threadIdx.x * per;
    const int p1 = min(p0 + per, span);
    const uint32_t qb = a.q * a.bits;
    const uint64_t mask = qb >= 64 ? ~0ull : ((1ull << qb) - 1);
    if (p0 < p1) {
      uint64_t code = 0;
      for (uint32_t t = 0; t + 1 < a.q; ++t) code = (code << a.bits) | s_code[p0 + t];
      for (int p = p0; p < p1; ++p) {
        code = ((code << a.bits) | s_code[p + a.q - 1]) & mask;
        s_h[p] = pi_value<HT, WIDE, TABLE>(code, a);
      }
    }
  }
  __syncthreads();
  // sparse table levels 1 .. levels-1
  for (int t = 1; t < levels; ++t) {
    const HT* src = s_h + (size_t)(t - 1) * span;
    HT* dst = s_h + (size_t)t * span;
    const int half = 1 << (t - 1);
    const int cnt = span - (1 << t) + 1;
    for (int x = threadIdx.x; x < cnt; x += kThreads) {
      const HT u = src[x], v = src[x + half];
      dst[x] = u < v ? u : v;
    }
    __syncthreads();
  }

  // the test: warp wid owns positions [g0 + kWarpPositions * wid, +kWarpPositions),
  // lane l takes positions 32k + l
  const uint64_t wbase = g0 + (uint64_t)wid * kWarpPositions;
  const uint32_t ns = s_ns;
  const bool cached = ns < cap || sid0 + cap == a.n;   // every string of the tile is in s_off
  uint32_t sid = 0;
  int64_t s_o = 0, s_e = -1, m = 0;
  int32_t r = 0;
  {
    const uint64_t g = wbase + lane;
    if (g < a.nbytes) {
      if (cached) {
        uint32_t lo = 0, hi = ns;   // s_off[lo] <= g < s_off[hi]
        while (hi - lo > 1) {
          uint32_t mid = (lo + hi) >> 1;
          if ((uint64_t)s_off[mid] <= g) lo = mid; else hi = mid;
        }
        sid = sid0 + lo;
      } else {
        sid = string_of(a.offsets, a.n, g);
      }
      s_o = (sid - sid0 < cap) ? s_off[sid - sid0] : __ldg(a.offsets + sid);
      s_e = (sid + 1 - sid0 <= cap) ? s_off[sid + 1 - sid0] : __ldg(a.offsets + sid + 1);
      m = s_e - s_o - a.q + 1;
      r = radius_of(s_e - s_o, a.q, a.T, a.r_min);
    }
  }
  uint32_t tot = 0;
#pragma unroll 1
  for (int k = 0; k < kWarpPositions / 32; ++k) {
    const uint64_t g = wbase + 32 * k + lane;
    bool anchor = false;
    if (g < a.nbytes) {
      while ((int64_t)g >= s_e) {   // next non-empty string holding g
        ++sid;
        s_o = s_e;
        s_e = (sid + 1 - sid0 <= cap) ? s_off[sid + 1 - sid0] : __ldg(a.offsets + sid + 1);
        m = s_e - s_o - a.q + 1;
        r = radius_of(s_e - s_o, a.q, a.T, a.r_min);
      }
      const int64_t i = (int64_t)g - s_o;
      const bool tested = i >= r && i <= m - 1 - r;
      if (r > HL && tested) atomicOr(dev_flags, FLAG_BOUNDS);    // cannot happen: r_max bounds every r
      const int p = (int)((int64_t)g - base);
      const int rr = r < 1 ? 1 : (r > HL ? HL : r);
      const int t = 31 - __clz(rr);
      const int w = 1 << t;
      const HT* lv = s_h + (size_t)t * span;
      // indices stay inside [0, span) for every position of the tile
      const HT lmin = min(lv[p - rr], lv[p - w]);
      const HT rmin = min(lv[p + 1], lv[p + rr - w + 1]);
      const HT v = s_h[p];
      anchor = (i == 0) || (tested && r <= HL && (r == 0 || (v < lmin && v < rmin)));
    }
    const uint32_t word = __ballot_sync(0xffffffffu, anchor);
    if (lane == 0) bitmap[(wbase >> 5) + k] = word;
    tot += __popc(word);
  }
  if (lane == 0) s_warp[wid] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kThreads / 32; ++w) t += s_warp[w];
    tile_count[blockIdx.x] = t;
  }
}

// Anchors of one tile in position order, at the tile's offset in the list.
// Thread t takes kPerThread consecutive positions (a slice of one bitmap word).
__global__ void __launch_bounds__(kThreads) anchor_emit_kernel(PartitionArgs a, const uint32_t* __restrict__ bitmap,
                                                               const uint32_t* __restrict__ tile_offset,
                                                               const uint32_t* __restrict__ tile_first,
                                                               uint32_t* __restrict__ anchor_pos,
                                                               uint32_t* __restrict__ anchor_sid) {
  constexpr int kPer = 32 / kPerThread;  // threads sharing one bitmap word
  const uint32_t word = __ldg(bitmap + (uint64_t)blockIdx.x * (kPartTile / 32) + threadIdx.x / kPer);
  const uint32_t flags = (word >> (kPerThread * (threadIdx.x % kPer))) & ((1u << kPerThread) - 1u);
  const uint32_t c = __popc(flags);
  // block exclusive scan of c
  uint32_t x = c;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __shared__ uint32_t s_warp[kThreads / 32];
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  uint32_t wsum = 0;
  for (int w = 0; w < wid; ++w) wsum += s_warp[w];
  uint32_t out = __ldg(tile_offset + blockIdx.x) + wsum + x - c;
  if (!flags) return;
  const uint64_t gfirst = (uint64_t)blockIdx.x * kPartTile + (uint64_t)threadIdx.x * kPerThread;
  uint32_t sid = __ldg(tile_first + blockIdx.x);
  int64_t s_end = __ldg(a.offsets + sid + 1);
  uint32_t f = flags;
  while (f) {
    int k = __ffs(f) - 1;
    f &= f - 1;
    uint64_t g = gfirst + k;
    while ((int64_t)g >= s_end) { ++sid; s_end = __ldg(a.offsets + sid + 1); }
    anchor_pos[out] = (uint32_t)g;
    anchor_sid[out] = sid;
    ++out;
  }
}

constexpr uint64_t kM61 = (1ull << 61) - 1;

__device__ __forceinline__ uint64_t mulmod61(uint64_t a, uint64_t b) {
  uint64_t lo = a * b, hi = __umul64hi(a, b);
  uint64_t r = (lo & kM61) + ((lo >> 61) | (hi << 3));
  return r >= kM61 ? r - kM61 : r;
}

// One partition per anchor: it runs to the next anchor of the same string,
// else to the string's end (Alg. 1).  The key is a Karp-Rabin polynomial of
// the substring modulo 2^61-1 with base `key_base`, over symbols byte+1.
__global__ void partition_records_kernel(const uint8_t* __restrict__ bytes, const int64_t* __restrict__ offsets,
                                         const uint32_t* __restrict__ anchor_pos,
                                         const uint32_t* __restrict__ anchor_sid, uint32_t n_anchor,
                                         uint64_t key_base, uint32_t* __restrict__ rec_sid,
                                         uint32_t* __restrict__ rec_pos, uint32_t* __restrict__ rec_len,
                                         uint32_t* __restrict__ rec_slen, uint64_t* __restrict__ rec_h61) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_anchor;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t g = anchor_pos[t], sid = anchor_sid[t];
    const int64_t s_off = __ldg(offsets + sid), s_end = __ldg(offsets + sid + 1);
    int64_t end = s_end;
    if (t + 1 < n_anchor && anchor_sid[t + 1] == sid) end = anchor_pos[t + 1];
    uint64_t h = 0;
    for (int64_t x = g; x < end; ++x) {
      h = mulmod61(h, key_base) + (uint64_t)__ldg(bytes + x) + 1;
      if (h >= kM61) h -= kM61;
    }
    rec_sid[t] = sid;
    rec_pos[t] = (uint32_t)((int64_t)g - s_off);
    rec_len[t] = (uint32_t)(end - (int64_t)g);
    rec_slen[t] = (uint32_t)(s_end - s_off);
    rec_h61[t] = h;
  }
}

}  // namespace

uint64_t partition_num_tiles(uint64_t nbytes) { return (nbytes + kPartTile - 1) / kPartTile; }

int launch_anchor_flags(const PartitionArgs& a, uint32_t* bitmap, uint32_t* tile_count, uint32_t* dev_flags,
                        uint32_t* planes, uint64_t plane_words, uint32_t guard_words, uint32_t* tile_first,
                        cudaStream_t s) {
  const uint64_t tiles = partition_num_tiles(a.nbytes);
  if (tiles == 0) return MJ_OK;
  {
    uint64_t blocks = (a.n + 255) / 256;
    if (blocks > (uint64_t)kNumSMsHint * 32) blocks = (uint64_t)kNumSMsHint * 32;
    tile_first_kernel<<<(unsigned)(blocks ? blocks : 1), 256, 0, s>>>(a.offsets, a.n, tiles, tile_first);
    MJ_KERNEL_DONE();
  }
  const bool wide = (uint64_t)a.q * a.bits > 32;
  const bool table = a.table != nullptr;
  const size_t smem = (table || wide) ? anchor_smem_bytes<uint64_t>(a.r_max, a.q)
                                      : anchor_smem_bytes<uint32_t>(a.r_max, a.q);
  int dev = 0, max_optin = 0;
  MJ_CUDA_TRY(cudaGetDevice(&dev));
  MJ_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem + sizeof(int64_t) * (kMaxTileStrings + 1) + 64 > (size_t)max_optin) return MJ_ERR_UNSUPPORTED;
  if (table) {
    auto k = anchor_flags_kernel<uint64_t, false, true>;
    MJ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<(unsigned)tiles, kThreads, smem, s>>>(a, bitmap, tile_count, dev_flags, planes, plane_words, guard_words,
                                              tile_first);
  } else if (wide) {
    auto k = anchor_flags_kernel<uint64_t, true, false>;
    MJ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<(unsigned)tiles, kThreads, smem, s>>>(a, bitmap, tile_count, dev_flags, planes, plane_words, guard_words,
                                              tile_first);
  } else {
    auto k = anchor_flags_kernel<uint32_t, false, false>;
    MJ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<(unsigned)tiles, kThreads, smem, s>>>(a, bitmap, tile_count, dev_flags, planes, plane_words, guard_words,
                                              tile_first);
  }
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_anchor_emit(const PartitionArgs& a, const uint32_t* bitmap, const uint32_t* tile_offset,
                       const uint32_t* tile_first, uint32_t* anchor_pos, uint32_t* anchor_sid, cudaStream_t s) {
  const uint64_t tiles = partition_num_tiles(a.nbytes);
  if (tiles == 0) return MJ_OK;
  anchor_emit_kernel<<<(unsigned)tiles, kThreads, 0, s>>>(a, bitmap, tile_offset, tile_first, anchor_pos,
                                                            anchor_sid);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_partition_records(const uint8_t* bytes, const int64_t* offsets, const uint32_t* anchor_pos,
                             const uint32_t* anchor_sid, uint32_t n_anchor, uint64_t key_base, uint32_t* rec_sid,
                             uint32_t* rec_pos, uint32_t* rec_len, uint32_t* rec_slen, uint64_t* rec_h61,
                             cudaStream_t s) {
  if (n_anchor == 0) return MJ_OK;
  unsigned grid = (unsigned)std::min<uint64_t>((n_anchor + 255) / 256, (uint64_t)kNumSMsHint * 16);
  partition_records_kernel<<<grid, 256, 0, s>>>(bytes, offsets, anchor_pos, anchor_sid, n_anchor, key_base,
                                                rec_sid, rec_pos, rec_len, rec_slen, rec_h61);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

}  // namespace mj
