// Steps a2-a4: q-gram hashing, anchors (strict local minima) and partition
// records — Alg. 1 (Partition-String) and Alg. 2 (Find-Anchor) of the MinJoin
// paper, computed for all strings at once over the concatenated bytes.
//
// Work decomposition: the concatenation is cut into tiles of kPartTile byte
// positions, two per CTA of the anchor kernel.  A CTA stages its bytes (as
// rank codes) plus a halo of r_max positions (rounded up to 32) on each side
// and the q - 1 symbols after it in shared memory, computes Pi of every
// q-gram start of tiles and halos there, then tests the tiles' own positions.  A position's string is found by binary search over
// the offsets; the strict-minimum test of a position never looks outside its
// own string (positions i in [r, m-1-r] of a string have all their 2r
// neighbours inside the string's q-gram range), so halos that run into a
// neighbouring string are harmless.
#include <type_traits>

#include "mj_internal.cuh"

namespace mj {
namespace {

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

// The anchor kernel: one CTA per kATile positions (two kPartTile tiles).
// Each of the first 256 threads owns a run of 16 consecutive positions of the
// tile; a ninth warp takes the runs of the halos.
constexpr int kATile = 2 * kPartTile;
constexpr int kARun = 16;                          // positions per thread run
constexpr int kATileRuns = kATile / kARun;         // 256 runs per tile
constexpr int kAThreads = kATileRuns + 32;         // tile runs + one warp of halo runs
constexpr int kAMaxStrings = 256;                  // strings cached per CTA
constexpr int kABlockRadius = 15;                  // radius from which block tests use run minima

// Halo of the anchor kernel: r_max positions rounded up to 32, so that the
// span starts on a 32-position word of the bitmap and bit-planes.
__host__ __device__ inline int anchor_halo(int r_max) { return ((r_max < 1 ? 1 : r_max) + 31) & ~31; }

// Shared memory of the anchor kernel: Pi of every position of the span, and
// for radii of 15 and more also the prefix and suffix minima of every run.
template <class HT>
__host__ __device__ inline size_t anchor_smem_bytes(int r_max) {
  const size_t span = kATile + 2 * (size_t)anchor_halo(r_max);
  return span * sizeof(HT) * (r_max >= kABlockRadius ? 3 : 1);
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

// Bit j set iff h[j] equals the minimum of its aligned block of B positions.
template <int B, class HT>
__device__ __forceinline__ uint32_t block_min_mask(const HT (&h)[kARun]) {
  uint32_t e = 0;
#pragma unroll
  for (int b = 0; b < kARun; b += B) {
    HT m = h[b];
#pragma unroll
    for (int j = 1; j < B; ++j) m = h[b + j] < m ? h[b + j] : m;
#pragma unroll
    for (int j = 0; j < B; ++j) e |= (h[b + j] == m ? 1u : 0u) << (b + j);
  }
  return e;
}

// Minimum of the n entries p[0 .. n-1] and of m.
template <class HT>
__device__ __forceinline__ HT range_min(const HT* p, int n, HT m) {
  for (; n >= 4; n -= 4, p += 4) {
    const HT a = p[0] < p[1] ? p[0] : p[1], b = p[2] < p[3] ? p[2] : p[3];
    const HT c = a < b ? a : b;
    m = c < m ? c : m;
  }
  for (; n > 0; --n, ++p) m = *p < m ? *p : m;
  return m;
}

// The MurmurHash3 32-bit finaliser (A. Appleby, public domain) of code ^ seed:
// the random function Pi on q-grams whose packed code fits 32 bits.  A
// bijection, so equal values mean equal q-grams.  seed' = seed ^ (seed >> 16)
// folds the seed into the first step: (c ^ s) ^ ((c ^ s) >> 16) = c ^ (c >> 16)
// ^ s'.  The other two shifts are taken as high words of products (m13 =
// 2^19, m16 = 2^16), which run on the multiply pipe beside the logic ops.
__device__ __forceinline__ uint32_t pi32(uint32_t code, uint32_t seed_folded, uint32_t m13, uint32_t m16) {
  uint32_t h = code ^ (code >> 16) ^ seed_folded;
  h *= 0x85ebca6bu;
  h ^= __umulhi(h, m13);
  h *= 0xc2b2ae35u;
  h ^= __umulhi(h, m16);
  return h;
}

// Pi of the q-gram whose packed code is `code` (see mjo_hash_qgrams for the
// definition shared with the paper's Table 2 form).
template <class HT, bool WIDE, bool TABLE>
__device__ __forceinline__ HT pi_value(uint64_t code, const PartitionArgs& a, uint32_t seed_folded) {
  if (TABLE) return (HT)__ldg(a.table + code);
  if (WIDE) return (HT)fmix64(code ^ a.seed64);
  return (HT)pi32((uint32_t)code, seed_folded, a.mul_shr13, a.mul_shr16);
}

// hi32(a * b) + c in one multiply-add.
__device__ __forceinline__ uint32_t mad_hi(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// One backward step of the packed q-gram code: the symbol enters at the top
// field (bits top .. top + bits - 1) and the lowest field drops out, so the
// code holds the q symbols starting at the last one entered.  The fields are
// disjoint, so for 32-bit codes (code >> bits) | (sym << top) is the multiply
// -add hi32(code * 2^(32 - bits)) + sym * 2^top.
struct Roll {
  uint32_t bsh, top, rmul, tmul;
  __device__ __forceinline__ uint32_t operator()(uint32_t code, uint32_t sym) const {
    return mad_hi(code, rmul, sym * tmul);
  }
  __device__ __forceinline__ uint64_t operator()(uint64_t code, uint32_t sym) const {
    return (code >> bsh) | ((uint64_t)sym << top);
  }
};

// Rank code of byte g, 0 outside [0, nbytes).
__device__ __forceinline__ uint32_t rank_at(const PartitionArgs& a, const uint8_t* s_rank, int64_t g) {
  return (g >= 0 && g < (int64_t)a.nbytes) ? (uint32_t)s_rank[__ldg(a.bytes + g)] : 0u;
}

// The 16 bytes at global position g (a 16-byte aligned load; PARTIAL: chunks
// at the ends of the input, read byte by byte with 0 codes outside it).
template <bool PARTIAL>
__device__ __forceinline__ void load_chunk(const PartitionArgs& a, int64_t g, uint32_t (&w)[4]) {
  if (PARTIAL) {
    w[0] = w[1] = w[2] = w[3] = 0;
  } else {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(a.bytes + g));
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  }
}

// Rank code of symbol j (0..15) of the chunk at g.
template <bool PARTIAL>
__device__ __forceinline__ uint32_t chunk_sym(const uint32_t (&w)[4], int j, const PartitionArgs& a,
                                              const uint8_t* s_rank, int64_t g) {
  if (PARTIAL) return rank_at(a, s_rank, g + j);
  return (uint32_t)s_rank[(w[j >> 2] >> (8 * (j & 3))) & 255u];
}

// The code rolled backwards over the first N symbols of the chunk at g.
template <bool PARTIAL, int N, class CT>
__device__ __forceinline__ CT prime_chunk(CT code, const PartitionArgs& a, const uint8_t* s_rank, int64_t g,
                                          const Roll& roll) {
  uint32_t w[4];
  load_chunk<PARTIAL>(a, g, w);
#pragma unroll
  for (int j = N - 1; j >= 0; --j) code = roll(code, chunk_sym<PARTIAL>(w, j, a, s_rank, g));
  return code;
}

template <int N, class CT>
__device__ __forceinline__ CT prime(CT code, const PartitionArgs& a, const uint8_t* s_rank, int64_t g, bool vec,
                                    const Roll& roll) {
  return (vec && g >= 0 && g + 16 <= (int64_t)a.nbytes) ? prime_chunk<false, N, CT>(code, a, s_rank, g, roll)
                                                        : prime_chunk<true, N, CT>(code, a, s_rank, g, roll);
}

// Pi of the 16 q-grams starting at g (h[j] for start g + j), continuing the
// backward roll from `code` (which holds the q - 1 symbols after the run in
// its upper fields); with PACK, symw gets the run's rank codes, one per byte.
template <bool PARTIAL, bool PACK, class CT, class HT, bool WIDE, bool TABLE>
__device__ __forceinline__ void hash_run(CT code, const PartitionArgs& a, const uint8_t* s_rank, int64_t g,
                                         const Roll& roll, uint32_t seed_folded, HT (&h)[kARun],
                                         uint32_t (&symw)[4]) {
  uint32_t w[4];
  load_chunk<PARTIAL>(a, g, w);
#pragma unroll
  for (int j = kARun - 1; j >= 0; --j) {
    const uint32_t sym = chunk_sym<PARTIAL>(w, j, a, s_rank, g);
    if (PACK) symw[j >> 2] = __byte_perm(symw[j >> 2], sym, (0x3210u & ~(0xfu << (4 * (j & 3)))) | (4u << (4 * (j & 3))));
    code = roll(code, sym);
    h[j] = pi_value<HT, WIDE, TABLE>((uint64_t)code, a, seed_folded);
  }
}

template <bool PACK, class CT, class HT, bool WIDE, bool TABLE>
__device__ __forceinline__ void hash_run_at(CT code, const PartitionArgs& a, const uint8_t* s_rank, int64_t g,
                                            bool vec, const Roll& roll, uint32_t seed_folded, HT (&h)[kARun],
                                            uint32_t (&symw)[4]) {
  if (vec && g >= 0 && g + 16 <= (int64_t)a.nbytes)
    hash_run<false, PACK, CT, HT, WIDE, TABLE>(code, a, s_rank, g, roll, seed_folded, h, symw);
  else
    hash_run<true, PACK, CT, HT, WIDE, TABLE>(code, a, s_rank, g, roll, seed_folded, h, symw);
}

// Index of entry o of the prefix- and suffix-minimum arrays: the four 16-byte
// quarters of a run are rotated by (run / 2) mod 4, which puts the quarter
// stores of the 8 lanes of a store phase in 8 different bank groups.
__device__ __forceinline__ int swz(int o) { return o ^ (((o >> 5) & 3) << 2); }

// Alg. 2 for kATile positions: position i of string s (0-based, m = |s| - q
// + 1 q-gram starts, radius r) is an anchor iff i = 0, or r <= i <= m - 1 - r
// and h[i] < h[j] for every other j in [i - r, i + r].
// The test runs on candidates only.  Take B = 2^floor(log2(r + 1)), at most
// 16: the aligned block of B positions holding i lies inside i's window, so
// an anchor is a minimum of its block.  For r < 15 a candidate is compared
// with the 2r other positions of its window.  For r >= 15 the block is the
// whole run and the candidate must be its unique minimum; the window outside
// the run is then covered by a suffix minimum, the minima of whole runs and a
// prefix minimum.
//   phase 0  rank table, the CTA's string offsets and radii, and which of
//            the two tests its strings need;
//   phase 1  per run: Pi of the 16 q-grams starting in it, from the packed
//            code rolled backwards, primed with the q - 1 symbols after the
//            run; the run's Pi values (or its prefix and suffix minima) go to
//            shared memory; the runs of the tiles also give the verifier's
//            bit-planes;
//   phase 2  per tile run: its strings, tested positions, block minima and
//            candidate tests; one 16-bit bitmap store per run, and counts.
template <class HT, bool WIDE, bool TABLE>
__global__ void __launch_bounds__(kAThreads, sizeof(HT) == 4 ? 4 : 2) anchor_flags_kernel(
    PartitionArgs a, uint32_t* __restrict__ bitmap, uint32_t* __restrict__ tile_count,
    uint32_t* __restrict__ dev_flags, uint32_t* __restrict__ planes, uint64_t plane_words, uint32_t guard_words,
    const uint32_t* __restrict__ tile_first, uint64_t tiles) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint8_t s_rank[256];
  __shared__ uint32_t s_off[kAMaxStrings + 1];  // offsets[sid0 .. sid0 + cap]
  __shared__ int32_t s_rad[kAMaxStrings];       // radius of strings sid0 .. sid0 + cap - 1
  __shared__ uint32_t s_ns;
  __shared__ uint32_t s_warp[kATileRuns / 32];
  const int Hs = anchor_halo(a.r_max);
  const int span = kATile + 2 * Hs;             // positions holding a Pi value
  HT* s_h = reinterpret_cast<HT*>(smem);
  HT* s_P = s_h + span;                          // present if r_max >= kABlockRadius
  HT* s_S = s_P + span;

  const uint32_t g0 = blockIdx.x * (uint32_t)kATile;
  const uint32_t gend = g0 + (uint32_t)kATile;
  const int64_t base = (int64_t)g0 - Hs;        // global position of entry 0
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t nbytes = (uint32_t)a.nbytes;

  // ---- phase 0
  if (threadIdx.x < 256) s_rank[threadIdx.x] = a.rank[threadIdx.x];
  const uint32_t sid0 = __ldg(tile_first + 2 * (uint64_t)blockIdx.x);
  const uint32_t cap = min((uint32_t)kAMaxStrings, a.n - sid0);
  bool need_scan = false, need_minima = false;   // tests of this thread's strings
  for (uint32_t t = threadIdx.x; t <= cap; t += kAThreads) {
    const uint32_t so = (uint32_t)__ldg(a.offsets + sid0 + t);
    s_off[t] = so;
    if (t < cap) {
      const uint32_t se = (uint32_t)__ldg(a.offsets + sid0 + t + 1);
      const int32_t r = radius32(se - so, a.q, a.T, a.r_min);
      s_rad[t] = r;
      if (so < gend && se > g0 && se > so && r > 0) {
        need_scan |= r < kABlockRadius;
        need_minima |= r >= kABlockRadius;
      }
    } else if (sid0 + cap < a.n && so < gend) {
      need_scan = need_minima = true;   // strings beyond the cache: both
    }
  }
  need_minima = __syncthreads_or(need_minima) && a.r_max >= kABlockRadius;
  need_scan = __syncthreads_or(need_scan);
  if (threadIdx.x == 0) {
    // strings that may hold CTA positions: indices 0 .. ns-1 of s_off
    uint32_t lo = 0, hi = cap;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_off[mid] < gend) lo = mid; else hi = mid;
    }
    s_ns = lo + 1;
  }

  // ---- phase 1: Pi of the runs (tile runs: threads 0..255; halo runs: warp 8)
  HT h[kARun];
  {
    using CT = typename std::conditional<WIDE, uint64_t, uint32_t>::type;
    Roll roll;
    roll.bsh = a.bits;
    roll.top = a.bits * (a.q - 1);
    roll.rmul = 1u << (32 - a.bits);
    roll.tmul = roll.top < 32 ? 1u << roll.top : 0u;   // 32-bit codes only
    const int qm1 = (int)a.q - 1;
    const int prime_chunks = (qm1 + 15) / 16;                  // chunks after the run holding q - 1 symbols
    const int far_syms = qm1 - 16 * (prime_chunks - 1);         // needed symbols of the farthest one
    const uint32_t seed_folded = a.seed32 ^ (a.seed32 >> 16);
    const bool vec = ((uintptr_t)a.bytes & 15) == 0;
    const int halo_runs = 2 * Hs / kARun;
    const int nwork = threadIdx.x < kATileRuns ? 1 : (halo_runs + 31 - lane) / 32;
    for (int it = 0; it < nwork; ++it) {
      int u;   // run index in the span
      if (threadIdx.x < kATileRuns) {
        u = Hs / kARun + threadIdx.x;
      } else {
        const int k = lane + 32 * it;
        u = k < Hs / kARun ? k : k + kATileRuns;
      }
      const int o0 = kARun * u;
      const int64_t gx = base + o0;
      // prime with the q - 1 symbols after the run, farthest chunk first
      CT code = 0;
      if (prime_chunks > 0) {
        const int64_t gf = gx + 16 * prime_chunks;
        if (far_syms <= 4) code = prime<4, CT>(code, a, s_rank, gf, vec, roll);
        else if (far_syms <= 8) code = prime<8, CT>(code, a, s_rank, gf, vec, roll);
        else if (far_syms <= 12) code = prime<12, CT>(code, a, s_rank, gf, vec, roll);
        else code = prime<16, CT>(code, a, s_rank, gf, vec, roll);
        for (int c = prime_chunks - 1; c >= 1; --c) code = prime<16, CT>(code, a, s_rank, gx + 16 * c, vec, roll);
      }
      uint32_t symw[4] = {0, 0, 0, 0};   // rank codes of the run, one per byte
      const bool pack = planes && threadIdx.x < kATileRuns;
      if (pack)
        hash_run_at<true, CT, HT, WIDE, TABLE>(code, a, s_rank, gx, vec, roll, seed_folded, h, symw);
      else
        hash_run_at<false, CT, HT, WIDE, TABLE>(code, a, s_rank, gx, vec, roll, seed_folded, h, symw);
      if (need_scan) {
#pragma unroll
        for (int j = 0; j < kARun; j += 4) {
          if (sizeof(HT) == 4) {
            *reinterpret_cast<uint4*>(s_h + o0 + j) =
                make_uint4((uint32_t)h[j], (uint32_t)h[j + 1], (uint32_t)h[j + 2], (uint32_t)h[j + 3]);
          } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) s_h[o0 + j + e] = h[j + e];
          }
        }
      }
      if (need_minima) {
        HT P[kARun], S[kARun];
        P[0] = h[0];
#pragma unroll
        for (int j = 1; j < kARun; ++j) P[j] = h[j] < P[j - 1] ? h[j] : P[j - 1];
        S[kARun - 1] = h[kARun - 1];
#pragma unroll
        for (int j = kARun - 2; j >= 0; --j) S[j] = h[j] < S[j + 1] ? h[j] : S[j + 1];
#pragma unroll
        for (int j = 0; j < kARun; j += 4) {
          const int o = swz(o0 + j);
          if (sizeof(HT) == 4) {
            *reinterpret_cast<uint4*>(s_P + o) =
                make_uint4((uint32_t)P[j], (uint32_t)P[j + 1], (uint32_t)P[j + 2], (uint32_t)P[j + 3]);
            *reinterpret_cast<uint4*>(s_S + o) =
                make_uint4((uint32_t)S[j], (uint32_t)S[j + 1], (uint32_t)S[j + 2], (uint32_t)S[j + 3]);
          } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              s_P[o + e] = P[j + e];
              s_S[o + e] = S[j + e];
            }
          }
        }
      }
      if (pack) {
        // plane p, positions g .. g+15 of this run: one 16-bit half of word g / 32
        const uint64_t g = (uint64_t)gx;
        const uint64_t word = guard_words + (g >> 5);
        if (word < guard_words + tiles * (kPartTile / 32)) {
          for (int p = 0; p < (int)a.bits; ++p) {
            uint32_t half = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              // bit p of the four byte-codes of symw[k] into a nibble (k-th symbol at bit k)
              const uint32_t x = (symw[k] >> p) & 0x01010101u;
              half += ((x * 0x01020408u) >> 24) << (4 * k);
            }
            reinterpret_cast<uint16_t*>(planes + (uint64_t)p * plane_words + word)[(g >> 4) & 1] = (uint16_t)half;
          }
          if (a.codes) *reinterpret_cast<uint4*>(a.codes + g) = make_uint4(symw[0], symw[1], symw[2], symw[3]);
        }
      }
    }
  }
  __syncthreads();

  // ---- phase 2: the tested positions of each tile run
  uint32_t flags = 0;   // anchor bit per position of the run
  const int v = threadIdx.x;
  const uint32_t x0 = g0 + kARun * (uint32_t)v;   // first position of the run
  if (v < kATileRuns && x0 < nbytes) {
    const int o0 = Hs + kARun * v;
    const uint32_t ns = s_ns;
    const bool cached = ns < cap || sid0 + cap == a.n;   // every string of the CTA is in s_off
    uint32_t k;   // the string holding x0
    if (cached) {
      uint32_t lo = 0, hi = ns;   // s_off[lo] <= x0 < s_off[hi]
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_off[mid] <= x0) lo = mid; else hi = mid;
      }
      k = sid0 + lo;
    } else {
      k = string_of(a.offsets, a.n, x0);
    }
    const uint32_t xl = x0 + kARun - 1;   // last position of the run
    for (;;) {
      uint32_t s_o, s_e;
      int32_t r;
      if (k - sid0 < cap) {
        s_o = s_off[k - sid0];
        s_e = s_off[k - sid0 + 1];
        r = s_rad[k - sid0];
      } else {
        s_o = (uint32_t)__ldg(a.offsets + k);
        s_e = (uint32_t)__ldg(a.offsets + k + 1);
        r = radius32(s_e - s_o, a.q, a.T, a.r_min);
      }
      if (s_e > s_o) {
        if (s_o >= x0) flags |= 1u << (s_o - x0);   // i = 0
        const int64_t i_hi = (int64_t)(s_e - s_o) - (int64_t)a.q - r;   // m - 1 - r
        if (i_hi >= r) {
          const uint32_t lo = max(s_o + (uint32_t)r, x0), hi = min(s_o + (uint32_t)i_hi, xl);
          if (r > Hs) {
            atomicOr(dev_flags, FLAG_BOUNDS);   // cannot happen: r_max bounds every r
          } else if (lo <= hi) {
            const uint32_t tested = (0xffffu >> (xl - hi)) & (0xffffu << (lo - x0));
            if (r == 0) {
              flags |= tested;
            } else if (r >= kABlockRadius) {
              // the run lies in every tested window: a candidate is its unique minimum
              const uint32_t eq = block_min_mask<16>(h);
              if (__popc(eq) == 1 && (eq & tested)) {
                const int j = __ffs(eq) - 1;
                const int o = o0 + j;
                const HT hx = s_P[swz(o0 + kARun - 1)];
                // [o - r, o0): suffix minimum of the first run, then whole runs
                const int la = o - r;
                HT m = ~HT(0);
                if (la < o0) {
                  m = s_S[swz(la)];
                  for (int u = (la >> 4) + 1; u < (o0 >> 4); ++u) m = min(m, s_S[swz(16 * u)]);
                }
                // (o0 + 15, o + r]: whole runs, then a prefix minimum of the last run
                const int rb = o + r;
                for (int u = (o0 >> 4) + 1; u < (rb >> 4); ++u) m = min(m, s_S[swz(16 * u)]);
                if (rb >= o0 + kARun) m = min(m, s_P[swz(rb)]);
                if (hx < m) flags |= 1u << j;
              }
            } else {
              const int B = r >= 7 ? 8 : (r >= 3 ? 4 : 2);
              uint32_t cand = (B == 8 ? block_min_mask<8>(h) : (B == 4 ? block_min_mask<4>(h) : block_min_mask<2>(h))) &
                              tested;
              while (cand) {
                const int j = __ffs(cand) - 1;
                cand &= cand - 1;
                const int o = o0 + j;
                const HT hx = s_h[o];
                HT m = range_min<HT>(s_h + o - r, r, ~HT(0));
                m = range_min<HT>(s_h + o + 1, r, m);
                if (hx < m) flags |= 1u << j;
              }
            }
          }
        }
      }
      if (s_e > xl || k + 1 >= a.n) break;
      ++k;
    }
  }

  // ---- bitmap half-words (16 positions each) and the two tiles' counts
  if (v < kATileRuns) {
    const uint64_t hw = (uint64_t)x0 >> 4;
    if (hw < tiles * (kPartTile / 16)) reinterpret_cast<uint16_t*>(bitmap)[hw] = (uint16_t)flags;
    const uint32_t tot = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(flags));
    if (lane == 0) s_warp[wid] = tot;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    constexpr int kHalf = kATileRuns / 64;   // warps per kPartTile tile
    uint32_t c0 = 0, c1 = 0;
    for (int w = 0; w < kHalf; ++w) {
      c0 += s_warp[w];
      c1 += s_warp[kHalf + w];
    }
    tile_count[2 * (uint64_t)blockIdx.x] = c0;
    if (2 * (uint64_t)blockIdx.x + 1 < tiles) tile_count[2 * (uint64_t)blockIdx.x + 1] = c1;
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

// One partition per anchor (Alg. 1): it runs from the anchor to the next
// anchor of its string, else to the string's end.  Every non-empty string
// starts with an anchor, so that end is the next anchor of the bitmap (or the
// end of the input).  The key is the Karp-Rabin polynomial sum of
// (byte + 1) * base^(len-1-x) modulo 2^61-1, evaluated by Horner's rule eight
// bytes per modular multiply: with T_k[c] = (c+1) * base^k (k = 1..7,
// shared-memory tables built per block), a block of eight bytes adds
// T7[b0] + T6[b1] + ... + T1[b6] + (b7+1) to h * base^8 (the leading len mod 8
// bytes go first, one at a time or as one block of four).  The key equals the
// byte-at-a-time polynomial.
// A CTA takes chunks of kRecWords bitmap words (whole kPartTile tiles) in
// turn, and builds its tables once.  For a chunk it lists the anchors in
// shared memory (a block scan of the words' counts), then its threads take
// one anchor at a time; an anchor's record goes to its tile's list offset
// plus its rank within the tile.
constexpr int kRecThreads = 256;
constexpr int kRecWords = kRecThreads;                 // 8,192 positions: 4 tiles
constexpr int kRecTileWords = kPartTile / 32;          // 64 words per tile
constexpr int kRecStrings = 256;                       // string offsets cached per chunk

__global__ void __launch_bounds__(kRecThreads) partition_records_kernel(
    PartitionArgs a, const uint32_t* __restrict__ bitmap, uint64_t nwords, const uint32_t* __restrict__ tile_offset,
    const uint32_t* __restrict__ tile_first, uint64_t key_base, PRec* __restrict__ recs) {
  __shared__ uint64_t s_t[7][256];                 // s_t[k - 1][c] = (c + 1) * base^k
  __shared__ uint16_t s_anc[kRecWords * 32];       // anchor offsets in the chunk, in order
  __shared__ uint32_t s_off[kRecStrings + 1];     // offsets[sid0 .. sid0 + cap]
  __shared__ uint32_t s_warp[kRecThreads / 32];
  __shared__ uint32_t s_tile0[kRecWords / kRecTileWords];   // list index of each tile's first anchor
  __shared__ uint32_t s_total;
  uint64_t b4 = 0, b8 = key_base;   // base^4 and base^8
  {
    const uint64_t c1 = (uint64_t)threadIdx.x + 1;
    uint64_t bk = key_base;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      s_t[k][threadIdx.x] = mulmod61(c1, bk);
      if (k == 3) b4 = bk;
      bk = mulmod61(bk, key_base);
    }
    b8 = bk;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t nbytes = (uint32_t)a.nbytes;
  const uint64_t nchunks = (nwords + kRecWords - 1) / kRecWords;
  for (uint64_t chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const uint64_t w0 = chunk * kRecWords;
    const uint32_t g0 = (uint32_t)(w0 * 32);
    const uint64_t word = w0 + threadIdx.x;
    const uint32_t bits = word < nwords ? __ldg(bitmap + word) : 0u;
    const uint32_t sid0 = __ldg(tile_first + w0 / kRecTileWords);
    const uint32_t cap = min((uint32_t)kRecStrings, a.n - sid0);
    __syncthreads();   // the previous chunk's lists are no longer read
    for (uint32_t t = threadIdx.x; t <= cap; t += kRecThreads) s_off[t] = (uint32_t)__ldg(a.offsets + sid0 + t);
    // block exclusive scan of the anchor counts, then the chunk's anchor list
    const uint32_t c = __popc(bits);
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    uint32_t excl = x - c;
    for (int w = 0; w < wid; ++w) excl += s_warp[w];
    if (threadIdx.x % kRecTileWords == 0) s_tile0[threadIdx.x / kRecTileWords] = excl;
    if (threadIdx.x == kRecThreads - 1) s_total = excl + c;
    {
      uint32_t f = bits, at = excl;
      while (f) {
        s_anc[at++] = (uint16_t)(32 * threadIdx.x + (__ffs(f) - 1));
        f &= f - 1;
      }
    }
    __syncthreads();
    const uint32_t total = s_total;
    const bool all_cached = sid0 + cap == a.n;
    for (uint32_t t = threadIdx.x; t < total; t += kRecThreads) {
      const uint32_t g = g0 + s_anc[t];
      // the string holding g
      uint32_t k;
      if (all_cached || s_off[cap] > g) {
        uint32_t lo = 0, hi = cap;   // s_off[lo] <= g < s_off[hi]
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (s_off[mid] <= g) lo = mid; else hi = mid;
        }
        k = sid0 + lo;
      } else {
        k = string_of(a.offsets, a.n, g);
      }
      const uint32_t s_o = k - sid0 <= cap ? s_off[k - sid0] : (uint32_t)__ldg(a.offsets + k);
      const uint32_t s_e = k + 1 - sid0 <= cap ? s_off[k + 1 - sid0] : (uint32_t)__ldg(a.offsets + k + 1);
      // the next anchor: in the list, else in the words after the chunk's
      uint32_t end = s_e;
      if (t + 1 < total) {
        end = g0 + s_anc[t + 1];
      } else {
        for (uint64_t ww = w0 + kRecWords; ww < nwords && ww * 32 < s_e; ++ww) {
          const uint32_t y = __ldg(bitmap + ww);
          if (y) {
            end = (uint32_t)(ww * 32) + (uint32_t)(__ffs(y) - 1);
            break;
          }
        }
      }
      end = min(end, min(s_e, nbytes));
      const uint8_t* p = a.bytes + g;
      const uint32_t len = end - g;
      const uint32_t head = len & 3u;
      uint64_t h = 0;
      for (uint32_t x2 = 0; x2 < head; ++x2) h = addmod61(mulmod61(h, key_base), (uint64_t)__ldg(p + x2) + 1);
      uint32_t x2 = head;
      if (len & 4u) {
        const uint64_t u = s_t[2][__ldg(p + x2)] + s_t[1][__ldg(p + x2 + 1)] + s_t[0][__ldg(p + x2 + 2)] +
                           (uint64_t)__ldg(p + x2 + 3) + 1;   // < 2^63
        const uint64_t v = (u & kM61) + (u >> 61);
        h = addmod61(mulmod61(h, b4), v >= kM61 ? v - kM61 : v);
        x2 += 4;
      }
      if (x2 < len) {
        // blocks of eight, the next block's bytes loaded one step ahead
        uint32_t nb[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) nb[e] = __ldg(p + x2 + e);
        for (;;) {
          uint64_t u = (uint64_t)nb[7] + 1;   // seven terms < 2^61 and one < 2^9: < 2^64
#pragma unroll
          for (int e = 0; e < 7; ++e) u += s_t[6 - e][nb[e]];
          x2 += 8;
          const bool more = x2 < len;
          if (more) {
#pragma unroll
            for (int e = 0; e < 8; ++e) nb[e] = __ldg(p + x2 + e);
          }
          const uint64_t v = (u & kM61) + (u >> 61);
          h = addmod61(mulmod61(h, b8), v >= kM61 ? v - kM61 : v);
          if (!more) break;
        }
      }
      PRec r;
      r.h61 = h;
      r.run = 0;
      r.slen = s_e - s_o;
      r.len = len;
      r.sid = k;
      r.pos = g - s_o;
      r.pad = 0;
      const uint32_t tile = (uint32_t)(s_anc[t] / kPartTile);   // tile within the chunk
      store_rec(recs, (uint64_t)__ldg(tile_offset + w0 / kRecTileWords + tile) + t - s_tile0[tile], r);
    }
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
  PartitionArgs ka = a;
  ka.mul_shr13 = 1u << 19;
  ka.mul_shr16 = 1u << 16;
  const bool wide = (uint64_t)a.q * a.bits > 32;
  const bool table = a.table != nullptr;
  const size_t smem = (table || wide) ? anchor_smem_bytes<uint64_t>(a.r_max) : anchor_smem_bytes<uint32_t>(a.r_max);
  int dev = 0, max_optin = 0;
  MJ_CUDA_TRY(cudaGetDevice(&dev));
  MJ_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem + 256 + sizeof(int64_t) * (kAMaxStrings + 1) + sizeof(int32_t) * kAMaxStrings + 64 > (size_t)max_optin)
    return MJ_ERR_UNSUPPORTED;
  const unsigned grid = (unsigned)((tiles + 1) / 2);
  if (table) {
    auto k = anchor_flags_kernel<uint64_t, false, true>;
    MJ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<grid, kAThreads, smem, s>>>(ka, bitmap, tile_count, dev_flags, planes, plane_words, guard_words, tile_first,
                                   tiles);
  } else if (wide) {
    auto k = anchor_flags_kernel<uint64_t, true, false>;
    MJ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<grid, kAThreads, smem, s>>>(ka, bitmap, tile_count, dev_flags, planes, plane_words, guard_words, tile_first,
                                   tiles);
  } else {
    auto k = anchor_flags_kernel<uint32_t, false, false>;
    MJ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<grid, kAThreads, smem, s>>>(ka, bitmap, tile_count, dev_flags, planes, plane_words, guard_words, tile_first,
                                   tiles);
  }
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_partition_records(const PartitionArgs& a, const uint32_t* bitmap, const uint32_t* tile_offset,
                             const uint32_t* tile_first, uint64_t key_base, PRec* recs, cudaStream_t s) {
  const uint64_t tiles = partition_num_tiles(a.nbytes);
  if (tiles == 0) return MJ_OK;
  const uint64_t nwords = tiles * kRecTileWords;
  int dev = 0, sms = 0, per_sm = 0;
  MJ_CUDA_TRY(cudaGetDevice(&dev));
  MJ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  MJ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, partition_records_kernel, kRecThreads, 0));
  const uint64_t grid = std::min<uint64_t>((nwords + kRecWords - 1) / kRecWords,
                                           (uint64_t)std::max(1, sms) * std::max(1, per_sm));
  partition_records_kernel<<<(unsigned)grid, kRecThreads, 0, s>>>(a, bitmap, nwords, tile_offset, tile_first,
                                                                  key_base, recs);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

}  // namespace mj
