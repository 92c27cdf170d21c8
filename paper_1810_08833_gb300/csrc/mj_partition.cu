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
#include <type_traits>

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

constexpr int kThreads = 256;
constexpr int kPerThread = kPartTile / kThreads;  // positions per thread in the emit kernel

// The anchor kernel: one CTA per kATile positions (two kPartTile tiles).
constexpr int kATile = 2 * kPartTile;
constexpr int kAPer = kATile / kThreads;           // 16 positions per thread
constexpr int kAWarpSpan = kATile / (kThreads / 32);   // 512 positions per warp
constexpr int kAMaxStrings = 256;                  // string offsets cached per CTA

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Halo of the anchor kernel: r_max positions rounded up to 16.
__host__ __device__ inline int anchor_halo(int r_max) { return (int)align16((size_t)(r_max < 1 ? 1 : r_max)); }

// Shared memory of the anchor kernel: rank table, staged rank codes of the
// tile, its halo and q-gram tail, then two range-minimum levels (ping-pong).
template <class HT>
__host__ __device__ inline size_t anchor_smem_bytes(int r_max) {
  const size_t span = kATile + 2 * (size_t)anchor_halo(r_max);
  return 256 + align16(span + 80) + 2 * align16((span + 8) * sizeof(HT));
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

// Alg. 2's neighbourhood radius in 32-bit arithmetic (every length < 2^32).
__device__ __forceinline__ int32_t radius32(uint32_t slen, uint32_t q, uint32_t T, int32_t r_min) {
  const int64_t num = (int64_t)slen - q + 1 - T;
  if (num < 0) return r_min;   // floor(num / den) < 0 <= r_min
  const uint32_t r = (uint32_t)num / (2 * T + 2);
  return r < (uint32_t)r_min ? r_min : (int32_t)r;
}

// Four consecutive table entries (16-byte aligned for 32-bit entries).
__device__ __forceinline__ void load4(const uint32_t* p, uint32_t (&v)[4]) {
  const uint4 u = *reinterpret_cast<const uint4*>(p);
  v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
}
__device__ __forceinline__ void load4(const uint64_t* p, uint64_t (&v)[4]) {
  const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(p);
  const ulonglong2 b = *reinterpret_cast<const ulonglong2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void store4(uint32_t* p, const uint32_t (&v)[4]) {
  *reinterpret_cast<uint4*>(p) = make_uint4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(uint64_t* p, const uint64_t (&v)[4]) {
  *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(v[0], v[1]);
  *reinterpret_cast<ulonglong2*>(p + 2) = make_ulonglong2(v[2], v[3]);
}

// Alg. 2 for kATile positions: position i of string s (0-based, m = |s| - q
// + 1 q-gram starts, radius r) is an anchor iff i = 0, or r <= i <= m - 1 - r
// and h[i] is strictly below both min(h[i-r .. i-1]) and min(h[i+1 .. i+r]).
// A window of length r is the union of two windows of length 2^t, t =
// floor(log2 r), so level t of a range-minimum table answers it with two
// reads.  The levels are built one at a time into two ping-pong buffers; a
// position is tested right after its string's level is built.
//   phase 1  rank codes of the tile and halos, staged with 16-byte loads;
//   phase 2  Pi of every q-gram start (16 consecutive starts per thread,
//            packed code rolled forward), and the verifier's bit-planes;
//   phase 3  level 0 (Pi itself), then levels 1 .. t_max, 4 entries per
//            thread and step; after level t the positions of strings with
//            floor(log2 r) = t are tested (lane-interleaved: warp w holds
//            positions 512 w + 32 j + lane);
//   phase 4  one ballot per 32 positions gives the bitmap word.
template <class HT, bool WIDE, bool TABLE>
__global__ void __launch_bounds__(kThreads, sizeof(HT) == 4 ? 4 : 1) anchor_flags_kernel(PartitionArgs a, uint32_t* __restrict__ bitmap,
                                                                uint32_t* __restrict__ tile_count,
                                                                uint32_t* __restrict__ dev_flags,
                                                                uint32_t* __restrict__ planes, uint64_t plane_words,
                                                                uint32_t guard_words,
                                                                const uint32_t* __restrict__ tile_first,
                                                                uint64_t tiles) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int64_t s_off[kAMaxStrings + 1];   // offsets[sid0 .. sid0 + cap]
  __shared__ uint32_t s_ns;
  __shared__ uint32_t s_warp[kThreads / 32];
  __shared__ uint32_t s_levels;
  const int Hs = anchor_halo(a.r_max);
  const int span = kATile + 2 * Hs;             // positions holding a Pi value
  const int nsym = span + 80;                   // staged symbols (q-gram tails)
  uint8_t* s_rank = smem;
  uint8_t* s_code = smem + 256;
  HT* lev0 = reinterpret_cast<HT*>(smem + 256 + align16(nsym));
  HT* lev1 = reinterpret_cast<HT*>(reinterpret_cast<uint8_t*>(lev0) + align16((span + 8) * sizeof(HT)));

  const uint32_t g0 = blockIdx.x * (uint32_t)kATile;
  const int64_t base = (int64_t)g0 - Hs;        // global position of s_code[0] and lev[0]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t nbytes = (uint32_t)a.nbytes;

  // ---- phase 0: rank table and the CTA's string offsets
  s_rank[threadIdx.x] = a.rank[threadIdx.x];
  if (threadIdx.x == 0) s_levels = 0;
  const uint32_t sid0 = __ldg(tile_first + 2 * (uint64_t)blockIdx.x);
  const uint32_t cap = min((uint32_t)kAMaxStrings, a.n - sid0);
  for (uint32_t t = threadIdx.x; t <= cap; t += kThreads) s_off[t] = __ldg(a.offsets + sid0 + t);
  __syncthreads();

  // ---- phase 1: rank codes of [base, base + nsym), 16 per thread and step
  {
    const bool vec = ((uintptr_t)a.bytes & 15) == 0;
    for (int c = 16 * threadIdx.x; c < nsym; c += 16 * kThreads) {
      const int64_t gb = base + c;
      uint32_t out[4];
      if (vec && gb >= 0 && gb + 16 <= (int64_t)nbytes) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(a.bytes + gb));
        const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          out[k] = (uint32_t)s_rank[w4[k] & 255u] | ((uint32_t)s_rank[(w4[k] >> 8) & 255u] << 8) |
                   ((uint32_t)s_rank[(w4[k] >> 16) & 255u] << 16) | ((uint32_t)s_rank[w4[k] >> 24] << 24);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          uint32_t x = 0;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int64_t g = gb + 4 * k + b;
            if (g >= 0 && g < (int64_t)nbytes) x |= (uint32_t)s_rank[__ldg(a.bytes + g)] << (8 * b);
          }
          out[k] = x;
        }
      }
      *reinterpret_cast<uint4*>(s_code + c) = make_uint4(out[0], out[1], out[2], out[3]);
    }
  }
  if (threadIdx.x == 0) {
    // strings that may hold CTA positions: indices 0 .. ns-1 of s_off
    uint32_t lo = 0, hi = cap;
    const int64_t gend = (int64_t)g0 + kATile;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_off[mid] < gend) lo = mid; else hi = mid;
    }
    s_ns = lo + 1;
  }
  __syncthreads();

  // ---- phase 2: Pi of every q-gram start in [0, span), and the bit-planes
  {
    // packed codes fit 32 bits unless WIDE (a table is indexed by codes < 2^32 too)
    using CT = typename std::conditional<WIDE, uint64_t, uint32_t>::type;
    const uint32_t qb = a.q * a.bits;
    const CT mask = qb >= 8 * sizeof(CT) ? ~CT(0) : ((CT(1) << qb) - 1);
    const uint32_t bsh = a.bits, qm1 = a.q - 1;
    for (int x0 = kAPer * threadIdx.x; x0 < span; x0 += kAPer * kThreads) {
      CT code = 0;
      for (uint32_t t = 0; t < qm1; ++t) code = (code << bsh) | s_code[x0 + t];
      const uint8_t* nxt = s_code + x0 + qm1;
      HT hv[kAPer];
#pragma unroll
      for (int j = 0; j < kAPer; ++j) {
        code = ((code << bsh) | nxt[j]) & mask;
        hv[j] = pi_value<HT, WIDE, TABLE>((uint64_t)code, a);
      }
      if (sizeof(HT) == 4) {
#pragma unroll
        for (int j = 0; j < kAPer; j += 4)
          *reinterpret_cast<uint4*>(lev0 + x0 + j) =
              make_uint4((uint32_t)hv[j], (uint32_t)hv[j + 1], (uint32_t)hv[j + 2], (uint32_t)hv[j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < kAPer; ++j) lev0[x0 + j] = hv[j];
      }
    }
  }
  if (planes) {
    // plane p, word (g0 + 512 w) / 32 + j: one ballot per word; lane j stores it
    const uint64_t word0 = guard_words + (uint64_t)(g0 >> 5) + (uint64_t)wid * (kAWarpSpan / 32);
    const uint64_t wlimit = guard_words + tiles * (kPartTile / 32);
    uint32_t sym[kAWarpSpan / 32];
#pragma unroll
    for (int j = 0; j < kAWarpSpan / 32; ++j) sym[j] = s_code[Hs + kAWarpSpan * wid + 32 * j + lane];
    for (int p = 0; p < (int)a.bits; ++p) {
      uint32_t mine = 0;
#pragma unroll
      for (int j = 0; j < kAWarpSpan / 32; ++j) {
        const uint32_t bw = __ballot_sync(0xffffffffu, (sym[j] >> p) & 1u);
        if (lane == j) mine = bw;
      }
      if (lane < kAWarpSpan / 32 && word0 + lane < wlimit) planes[(uint64_t)p * plane_words + word0 + lane] = mine;
    }
  }
  __syncthreads();

  // ---- phase 3: per position (lane-interleaved) string, radius and level
  const uint32_t wbase = g0 + (uint32_t)(kAWarpSpan * wid);
  const uint32_t ns = s_ns;
  const bool cached = ns < cap || sid0 + cap == a.n;   // every string of the CTA is in s_off
  uint32_t rq2[kAPer / 2];   // radius of position j in bits 16(j&1) .. of word j/2 (0: not queried)
  uint32_t flags = 0;   // anchor bit per position
  uint32_t level_mask = 0;
  {
    // the current string: [s_o, s_e), radius r, level t; positions i of it
    // with r <= i <= i_hi are tested (i_hi < r: none)
    uint32_t sid = 0, s_o = 0, s_e = 0;
    int32_t r = 0, i_hi = -1;
    uint32_t lvl = 0;
    auto set_string = [&]() {
      const uint32_t slen = s_e - s_o;
      r = radius32(slen, a.q, a.T, a.r_min);
      const int64_t hi = (int64_t)slen - a.q - r;   // m - 1 - r, m = |s| - q + 1
      i_hi = hi < 0 ? -1 : (hi > 0x7fffffff ? 0x7fffffff : (int32_t)hi);
      if (r > Hs && i_hi >= r) atomicOr(dev_flags, FLAG_BOUNDS);   // cannot happen: r_max bounds every r
      lvl = (r == 0 || r > Hs || i_hi < r) ? 0u : (uint32_t)r;   // radius of a range query, 0: none
    };
    const uint32_t gfirst = wbase + lane;
    if (gfirst < nbytes) {
      if (cached) {
        uint32_t lo = 0, hi = ns;   // s_off[lo] <= g < s_off[hi]
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if ((uint64_t)s_off[mid] <= gfirst) lo = mid; else hi = mid;
        }
        sid = sid0 + lo;
      } else {
        sid = string_of(a.offsets, a.n, gfirst);
      }
      s_o = (uint32_t)((sid - sid0 <= cap) ? s_off[sid - sid0] : __ldg(a.offsets + sid));
      s_e = (uint32_t)((sid + 1 - sid0 <= cap) ? s_off[sid + 1 - sid0] : __ldg(a.offsets + sid + 1));
      set_string();
    }
#pragma unroll
    for (int j = 0; j < kAPer / 2; ++j) rq2[j] = 0;
#pragma unroll
    for (int j = 0; j < kAPer; ++j) {
      const uint32_t g = wbase + 32 * j + lane;
      if (g < nbytes) {
        while (g >= s_e) {   // next non-empty string holding g
          ++sid;
          s_o = s_e;
          s_e = (uint32_t)((sid + 1 - sid0 <= cap) ? s_off[sid + 1 - sid0] : __ldg(a.offsets + sid + 1));
          set_string();
        }
        const int32_t i = (int32_t)(g - s_o);
        const bool tested = i >= r && i <= i_hi;
        if (i == 0 || (tested && r == 0)) flags |= 1u << j;
        if (tested && lvl) {
          rq2[j / 2] |= lvl << (16 * (j & 1));
          level_mask |= 1u << (31 - __clz(lvl));
        }
      }
    }
  }
  // levels this CTA needs: 0 .. the highest floor(log2 r) of its tested positions
  if (level_mask) atomicOr(&s_levels, level_mask);
  __syncthreads();
  const int t_top = s_levels ? 31 - __clz(s_levels) : 0;
  HT v[kAPer];          // Pi of the position
#pragma unroll
  for (int j = 0; j < kAPer; ++j) v[j] = lev0[Hs + kAWarpSpan * wid + 32 * j + lane];
  HT* cur = lev0;
  HT* oth = lev1;
#pragma unroll 1
  for (int t = 0; t <= t_top; ++t) {
    if (t > 0) {
      // level t from level t - 1: min of entries x and x + 2^(t-1)
      const int half = 1 << (t - 1);
      const int cnt = span - (1 << t) + 1;
      for (int x = 4 * threadIdx.x; x < cnt; x += 4 * kThreads) {
        HT lo4[4], nx4[4], hi4[4];
        load4(cur + x, lo4);
        if (half >= 4) {
          load4(cur + x + half, hi4);
        } else {
          load4(cur + x + 4, nx4);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int y = k + half;   // 1 .. 5
            hi4[k] = y < 4 ? lo4[y & 3] : nx4[y & 3];
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) lo4[k] = lo4[k] < hi4[k] ? lo4[k] : hi4[k];
        store4(oth + x, lo4);
      }
      __syncthreads();
      HT* tmp = cur;
      cur = oth;
      oth = tmp;
    }
    if ((level_mask >> t) & 1u) {
      const int w = 1 << t;
#pragma unroll
      for (int j = 0; j < kAPer; ++j) {
        const int r = (int)((rq2[j / 2] >> (16 * (j & 1))) & 0xffffu);
        if (r != 0 && 31 - __clz(r) == t) {
          const int x = Hs + kAWarpSpan * wid + 32 * j + lane;
          const HT lmin = min(cur[x - r], cur[x - w]);
          const HT rmin = min(cur[x + 1], cur[x + r - w + 1]);
          if (v[j] < lmin && v[j] < rmin) flags |= 1u << j;
        }
      }
    }
  }

  // ---- phase 4: bitmap words (lane j stores word j of the warp) and counts
  uint32_t mine = 0, tot = 0;
#pragma unroll
  for (int j = 0; j < kAPer; ++j) {
    const uint32_t word = __ballot_sync(0xffffffffu, (flags >> j) & 1u);
    if (lane == j) mine = word;
    tot += __popc(word);
  }
  const uint64_t wword = (uint64_t)(wbase >> 5) + lane;
  if (lane < kAPer && wword < tiles * (kPartTile / 32)) bitmap[wword] = mine;
  if (lane == 0) s_warp[wid] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    constexpr int kHalf = kThreads / 64;   // warps per kPartTile tile
    uint32_t c0 = 0, c1 = 0;
    for (int w = 0; w < kHalf; ++w) {
      c0 += s_warp[w];
      c1 += s_warp[kHalf + w];
    }
    tile_count[2 * (uint64_t)blockIdx.x] = c0;
    if (2 * (uint64_t)blockIdx.x + 1 < tiles) tile_count[2 * (uint64_t)blockIdx.x + 1] = c1;
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

__device__ __forceinline__ uint64_t addmod61(uint64_t a, uint64_t b) {
  uint64_t r = a + b;   // a, b < 2^61: no overflow
  return r >= kM61 ? r - kM61 : r;
}

// One partition per anchor: it runs to the next anchor of the same string,
// else to the string's end (Alg. 1).  The key is the Karp-Rabin polynomial
// sum of (byte + 1) * base^(len-1-x) modulo 2^61-1, evaluated by Horner's
// rule four bytes per modular multiply: with T_k[c] = (c+1) * base^k (k = 1..3,
// shared-memory tables built per block), a block of four bytes adds
// T3[b0] + T2[b1] + T1[b2] + (b3+1) to h * base^4.  The key equals the
// byte-at-a-time polynomial.
constexpr int kRecThreads = 256;

__global__ void __launch_bounds__(kRecThreads) partition_records_kernel(
    const uint8_t* __restrict__ bytes, const int64_t* __restrict__ offsets, const uint32_t* __restrict__ anchor_pos,
    const uint32_t* __restrict__ anchor_sid, uint32_t n_anchor, uint64_t key_base, uint32_t* __restrict__ rec_sid,
    uint32_t* __restrict__ rec_pos, uint32_t* __restrict__ rec_len, uint32_t* __restrict__ rec_slen,
    uint64_t* __restrict__ rec_h61) {
  __shared__ uint64_t s_t[3][256];
  const uint64_t b2 = mulmod61(key_base, key_base), b3 = mulmod61(b2, key_base), b4 = mulmod61(b3, key_base);
  {
    const uint64_t c1 = (uint64_t)threadIdx.x + 1;
    s_t[0][threadIdx.x] = mulmod61(c1, key_base);
    s_t[1][threadIdx.x] = mulmod61(c1, b2);
    s_t[2][threadIdx.x] = mulmod61(c1, b3);
  }
  __syncthreads();
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_anchor;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t g = anchor_pos[t], sid = anchor_sid[t];
    const int64_t s_off = __ldg(offsets + sid), s_end = __ldg(offsets + sid + 1);
    int64_t end = s_end;
    if (t + 1 < n_anchor && anchor_sid[t + 1] == sid) end = anchor_pos[t + 1];
    const uint8_t* p = bytes + g;
    const uint32_t len = (uint32_t)(end - (int64_t)g);
    const uint32_t head = len & 3u;
    uint64_t h = 0;
    for (uint32_t x = 0; x < head; ++x) h = addmod61(mulmod61(h, key_base), (uint64_t)__ldg(p + x) + 1);
    for (uint32_t x = head; x < len; x += 4) {
      const uint32_t c0 = __ldg(p + x), c1 = __ldg(p + x + 1), c2 = __ldg(p + x + 2), c3 = __ldg(p + x + 3);
      uint64_t u = s_t[2][c0] + s_t[1][c1];     // < 2^62
      u = (u & kM61) + (u >> 61);
      u += s_t[0][c2] + (uint64_t)c3 + 1;       // < 2^63
      u = (u & kM61) + (u >> 61);
      h = addmod61(mulmod61(h, b4), u >= kM61 ? u - kM61 : u);
    }
    rec_sid[t] = sid;
    rec_pos[t] = (uint32_t)((int64_t)g - s_off);
    rec_len[t] = len;
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
  const size_t smem = (table || wide) ? anchor_smem_bytes<uint64_t>(a.r_max) : anchor_smem_bytes<uint32_t>(a.r_max);
  int dev = 0, max_optin = 0;
  MJ_CUDA_TRY(cudaGetDevice(&dev));
  MJ_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem + sizeof(int64_t) * (kAMaxStrings + 1) + 64 > (size_t)max_optin) return MJ_ERR_UNSUPPORTED;
  const unsigned grid = (unsigned)((tiles + 1) / 2);
  if (table) {
    auto k = anchor_flags_kernel<uint64_t, false, true>;
    MJ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<grid, kThreads, smem, s>>>(a, bitmap, tile_count, dev_flags, planes, plane_words, guard_words, tile_first,
                                   tiles);
  } else if (wide) {
    auto k = anchor_flags_kernel<uint64_t, true, false>;
    MJ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<grid, kThreads, smem, s>>>(a, bitmap, tile_count, dev_flags, planes, plane_words, guard_words, tile_first,
                                   tiles);
  } else {
    auto k = anchor_flags_kernel<uint32_t, false, false>;
    MJ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<grid, kThreads, smem, s>>>(a, bitmap, tile_count, dev_flags, planes, plane_words, guard_words, tile_first,
                                   tiles);
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
  partition_records_kernel<<<grid, kRecThreads, 0, s>>>(bytes, offsets, anchor_pos, anchor_sid, n_anchor, key_base,
                                                rec_sid, rec_pos, rec_len, rec_slen, rec_h61);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

}  // namespace mj
