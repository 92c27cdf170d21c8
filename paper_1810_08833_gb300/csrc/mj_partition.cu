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

// Alg. 2 line 2 with floor division and the r_min clamp.
__device__ __forceinline__ int32_t radius_of(int64_t slen, int32_t q, int32_t T, int32_t r_min) {
  int64_t num = slen - q + 1 - T, den = 2 * (int64_t)T + 2;
  int64_t r = num >= 0 ? num / den : -((-num + den - 1) / den);
  return r < r_min ? r_min : (int32_t)r;
}

constexpr int kThreads = 256;
constexpr int kPerThread = kPartTile / kThreads;  // 16 positions per thread
static_assert(kPerThread == 16, "bitmap packing assumes 16 positions per thread");

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <class HT>
__host__ __device__ inline size_t anchor_smem_bytes(int r_max, int q) {
  size_t span = kPartTile + 2 * (size_t)r_max;
  return align16(span + q) + span * sizeof(HT) + 256;
}

// Pi of the q-gram whose packed code is `code` (see mjo_hash_qgrams for the
// definition shared with the paper's Table 2 form).
template <class HT, bool WIDE, bool TABLE>
__device__ __forceinline__ HT pi_value(uint64_t code, const PartitionArgs& a) {
  if (TABLE) return (HT)__ldg(a.table + code);
  if (WIDE) return (HT)fmix64(code ^ a.seed64);
  return (HT)fmix32((uint32_t)code ^ a.seed32);
}

template <class HT, bool WIDE, bool TABLE>
__global__ void __launch_bounds__(kThreads) anchor_flags_kernel(PartitionArgs a, uint32_t* __restrict__ bitmap,
                                                                uint32_t* __restrict__ tile_count,
                                                                uint32_t* __restrict__ dev_flags) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int HL = a.r_max;
  const int span = kPartTile + 2 * HL;        // positions holding a Pi value
  const int nb = span + (int)a.q;              // staged bytes
  uint8_t* s_rank = smem;                      // 256-entry rank table
  uint8_t* s_code = smem + 256;                // staged rank codes
  HT* s_h = reinterpret_cast<HT*>(smem + 256 + align16(nb));

  const uint64_t g0 = (uint64_t)blockIdx.x * kPartTile;
  const int64_t base = (int64_t)g0 - HL;       // global position of s_code[0] and s_h[0]

  s_rank[threadIdx.x] = a.rank[threadIdx.x];
  __syncthreads();
  for (int t = threadIdx.x; t < nb; t += kThreads) {
    int64_t g = base + t;
    s_code[t] = (g >= 0 && (uint64_t)g < a.nbytes) ? s_rank[__ldg(a.bytes + g)] : 0;
  }
  __syncthreads();

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

  // Alg. 2 for the tile's own positions, 16 consecutive per thread.
  uint32_t flags = 0;
  const uint64_t gfirst = g0 + (uint64_t)threadIdx.x * kPerThread;
  if (gfirst < a.nbytes) {
    uint32_t sid = string_of(a.offsets, a.n, gfirst);
    int64_t s_off = __ldg(a.offsets + sid), s_end = __ldg(a.offsets + sid + 1);
    int64_t slen = s_end - s_off, m = slen - a.q + 1;
    int32_t r = radius_of(slen, a.q, a.T, a.r_min);
#pragma unroll 1
    for (int k = 0; k < kPerThread; ++k) {
      uint64_t g = gfirst + k;
      if (g >= a.nbytes) break;
      while ((int64_t)g >= s_end) {  // next non-empty string holding g
        ++sid;
        s_off = __ldg(a.offsets + sid);
        s_end = __ldg(a.offsets + sid + 1);
        slen = s_end - s_off;
        m = slen - a.q + 1;
        r = radius_of(slen, a.q, a.T, a.r_min);
      }
      int64_t i = (int64_t)g - s_off;
      bool anchor = (i == 0);                    // A starts as {first position}
      if (!anchor && i >= r && i <= m - 1 - r) {
        if (r > HL) {                            // cannot happen: r_max bounds every r
          atomicOr(dev_flags, FLAG_BOUNDS);
        } else {
          const int p = (int)((int64_t)g - base);
          const HT v = s_h[p];
          bool ok = true;
#pragma unroll 1
          for (int d = 1; d <= r; ++d) {
            if (s_h[p - d] <= v || s_h[p + d] <= v) { ok = false; break; }
          }
          anchor = ok;
        }
      }
      flags |= (uint32_t)anchor << k;
    }
  }
  // two threads' 16-bit flag groups form one bitmap word
  uint32_t hi = __shfl_down_sync(0xffffffffu, flags, 1);
  if ((threadIdx.x & 1) == 0) bitmap[(uint64_t)blockIdx.x * (kPartTile / 32) + threadIdx.x / 2] = flags | (hi << 16);
  // tile anchor count
  uint32_t c = __popc(flags);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  __shared__ uint32_t s_warp[kThreads / 32];
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int w = 0; w < kThreads / 32; ++w) tot += s_warp[w];
    tile_count[blockIdx.x] = tot;
  }
}

// Anchors of one tile in position order, at the tile's offset in the list.
__global__ void __launch_bounds__(kThreads) anchor_emit_kernel(PartitionArgs a, const uint32_t* __restrict__ bitmap,
                                                               const uint32_t* __restrict__ tile_offset,
                                                               uint32_t* __restrict__ anchor_pos,
                                                               uint32_t* __restrict__ anchor_sid) {
  const uint32_t word = __ldg(bitmap + (uint64_t)blockIdx.x * (kPartTile / 32) + threadIdx.x / 2);
  const uint32_t flags = (threadIdx.x & 1) ? (word >> 16) : (word & 0xffffu);
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
  uint32_t wbase = 0;
  for (int w = 0; w < wid; ++w) wbase += s_warp[w];
  uint32_t out = __ldg(tile_offset + blockIdx.x) + wbase + x - c;
  if (!flags) return;
  const uint64_t gfirst = (uint64_t)blockIdx.x * kPartTile + (uint64_t)threadIdx.x * kPerThread;
  uint32_t sid = string_of(a.offsets, a.n, gfirst);
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
                        cudaStream_t s) {
  const uint64_t tiles = partition_num_tiles(a.nbytes);
  if (tiles == 0) return MJ_OK;
  const bool wide = (uint64_t)a.q * a.bits > 32;
  const bool table = a.table != nullptr;
  size_t smem;
  if (table || wide) {
    smem = anchor_smem_bytes<uint64_t>(a.r_max, a.q);
    if (table) {
      auto k = anchor_flags_kernel<uint64_t, false, true>;
      MJ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k<<<(unsigned)tiles, kThreads, smem, s>>>(a, bitmap, tile_count, dev_flags);
    } else {
      auto k = anchor_flags_kernel<uint64_t, true, false>;
      MJ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k<<<(unsigned)tiles, kThreads, smem, s>>>(a, bitmap, tile_count, dev_flags);
    }
  } else {
    smem = anchor_smem_bytes<uint32_t>(a.r_max, a.q);
    auto k = anchor_flags_kernel<uint32_t, false, false>;
    MJ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<(unsigned)tiles, kThreads, smem, s>>>(a, bitmap, tile_count, dev_flags);
  }
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_anchor_emit(const PartitionArgs& a, const uint32_t* bitmap, const uint32_t* tile_offset,
                       uint32_t* anchor_pos, uint32_t* anchor_sid, cudaStream_t s) {
  const uint64_t tiles = partition_num_tiles(a.nbytes);
  if (tiles == 0) return MJ_OK;
  anchor_emit_kernel<<<(unsigned)tiles, kThreads, 0, s>>>(a, bitmap, tile_offset, anchor_pos, anchor_sid);
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
