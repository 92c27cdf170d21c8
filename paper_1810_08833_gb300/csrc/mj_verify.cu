// Step a8: verification of candidate pairs (Sec. 3: Ukkonen's banded dynamic
// program) as a bit-parallel computation over a diagonal band.
//
// For a pair, A is the longer string (rows i = 1..m) and B the shorter
// (columns j = 1..n), d0 = m - n <= k.  A path of cost <= k from (0,0) to
// (m,n) never leaves the diagonals d = i - j in
//     [dlo, dhi] = [-floor((k-d0)/2), d0 + floor((k-d0)/2)],
// because reaching diagonal d costs |d| and returning costs |d0 - d|.  The
// kernel holds, for every column j, the vertical deltas D[i][j] - D[i-1][j]
// of the rows i = j + dlo + t (t = 0 .. 32W-1, W 32-bit words, 32W >= width)
// as two bit-vectors (+1 and -1 bits), and advances a column with the
// bit-vector recurrence of Myers (1999) in Hyyro's formulation:
//     Xv = Eq | Mv;  Xh = (((Eq & Pv) + Pv) ^ Pv) | Eq
//     Ph = Mv | ~(Xh | Pv);  Mh = Pv & Xh
//     Ph = (Ph << 1) | hin;  Mh = Mh << 1
//     Pv = Mh | ~(Xv | Ph);  Mv = Ph & Xv
// Between columns the band slides down one row, so the vectors shift right by
// one bit.  Cells outside the band take over-estimates that keep every delta
// in {-1, 0, +1}: the row entering at the bottom gets a vertical delta of +1,
// the row above the top a horizontal delta of +1 (hin).  Rows above row 0 are
// virtual, with D[i][j] = j - i, which reproduces D[0][j] = j exactly.  The
// computed values are then >= the true ones everywhere and exact along any
// path that stays in the band, so D[m][n] is exact whenever ED <= k and > k
// otherwise.
//
// Early exit: along a diagonal, D[i+1][j+1] >= D[i][j], so D[m][n] >=
// D[j+d0][j] for every j; once that cell exceeds k the pair is rejected
// (checked every 32 columns).  The kernel tracks the value of the band's top
// row (bit 0) and recovers the cell on diagonal d0 (bit t0) by summing the
// deltas of bits 1..t0.
//
// Equality bits: rank codes of all bytes are stored as bit-planes over the
// concatenated input (plane p holds bit p of every code).  For column j the
// 32(W+1) plane bits starting at A's row j + dlo are ANDed against the rank of
// B[j-1] (XNOR per plane) and funnel-shifted into band position.
#include <algorithm>

#include "mj_internal.cuh"

namespace mj {
namespace {

constexpr int kMaxBits = 8;

// One 32-symbol word per thread (two 16-byte loads where aligned).
__global__ void build_planes_kernel(const uint8_t* __restrict__ bytes, uint64_t nbytes, RankTable rt, uint32_t bits,
                                    uint32_t* __restrict__ planes, uint64_t plane_words, uint32_t guard_words,
                                    uint8_t* __restrict__ codes) {
  __shared__ uint8_t s_rank[256];
  s_rank[threadIdx.x] = rt.r[threadIdx.x];
  __syncthreads();
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < plane_words;
       w += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t acc[kMaxBits] = {0};
    const int64_t c0 = ((int64_t)w - (int64_t)guard_words) * 32;
    uint32_t sym[8];
    const bool full = c0 >= 0 && (uint64_t)c0 + 32 <= nbytes && ((uintptr_t)(bytes + c0) & 15) == 0;
    if (full) {
      const uint4 u = __ldg(reinterpret_cast<const uint4*>(bytes + c0));
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(bytes + c0 + 16));
      sym[0] = u.x; sym[1] = u.y; sym[2] = u.z; sym[3] = u.w;
      sym[4] = v.x; sym[5] = v.y; sym[6] = v.z; sym[7] = v.w;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        uint32_t x = 0;
        for (int b = 0; b < 4; ++b) {
          const int64_t c = c0 + 4 * q + b;
          if (c >= 0 && (uint64_t)c < nbytes) x |= (uint32_t)__ldg(bytes + c) << (8 * b);
        }
        sym[q] = x;
      }
    }
    uint32_t cw[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // the 32 rank codes, four per word
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const int64_t c = c0 + t;
      const uint32_t r = (c >= 0 && (uint64_t)c < nbytes) ? s_rank[(sym[t >> 2] >> (8 * (t & 3))) & 255u] : 0u;
      cw[t >> 2] |= r << (8 * (t & 3));
#pragma unroll
      for (int p = 0; p < kMaxBits; ++p) acc[p] |= ((r >> p) & 1u) << t;
    }
    if (codes && c0 >= 0 && (uint64_t)c0 < nbytes) {   // codes + c0 is 32-byte aligned, the buffer nbytes + 32 long
      *reinterpret_cast<uint4*>(codes + c0) = make_uint4(cw[0], cw[1], cw[2], cw[3]);
      *reinterpret_cast<uint4*>(codes + c0 + 16) = make_uint4(cw[4], cw[5], cw[6], cw[7]);
    }
#pragma unroll
    for (int p = 0; p < kMaxBits; ++p)
      if (p < (int)bits) planes[(uint64_t)p * plane_words + w] = acc[p];
  }
}

// Result of pair t: ed[t] = v; a pair within the join's threshold (v <= K)
// is also listed in out_t (when given), so the join's output needs no pass
// over all candidates.
__device__ __forceinline__ void put_result(const VerifyArgs& a, uint64_t t, uint32_t v) {
  a.ed[t] = v;
  if (a.out_t && v <= a.K) a.out_t[atomicAdd(a.out_count, 1ull)] = (uint32_t)t;
}

// Number of cells (i, j), 1 <= i <= m, 1 <= j <= n, with |i - j| <= K (m >= n).
__device__ __forceinline__ uint64_t band_cells(int64_t m, int64_t n, int64_t K) {
  if (n <= 0 || m <= 0) return 0;
  int64_t a = m - K;                                   // j <= a: min(m, j+K) = j + K
  a = a < 0 ? 0 : (a > n ? n : a);
  int64_t smin = a * (a + 1) / 2 + a * K + (n - a) * m;
  int64_t b = K < n ? K : n;                           // j <= K: max(1, j-K) = 1
  int64_t smax = b + (n > K ? (n - K) * (n - K + 1) / 2 : 0);
  return (uint64_t)(smin - smax + n);
}

// Per-lane state of one pair in flight.
template <int W, int P>
struct PairState {
  uint32_t Pv[W], Mv[W], M1[W];
  uint64_t abit;           // plane bit index of the band's top row at column 1
  uint64_t bpos;           // plane bit index of B's symbol of column j
  int32_t j, n;            // next column, number of columns
  int32_t score;           // D at the band's top row
  uint32_t k;              // band of this pair
  uint64_t t;              // pair index
};

// Sets up pair t; returns false if the pair is decided without the DP
// (result written to *res).
// Geometry of the pair at order position q (index t): offsets of A (the
// longer string) and B, their lengths; false for an id out of range.
__device__ __forceinline__ bool pair_geometry(const VerifyArgs& a, uint64_t q, uint64_t t, int64_t& oA, int64_t& oB,
                                              int64_t& m, int64_t& n) {
  if (a.pair_geo) {   // written with the order: one load, no chain through the ids
    const uint4 g = a.pair_geo[q];
    if (g.w == kGeoBadIds) return false;
    oA = g.x;
    oB = g.y;
    m = g.z;
    n = g.w;
    return true;
  }
  const uint32_t x = a.pi[t], y = a.pj[t];
  if (x >= a.n_strings || y >= a.n_strings) return false;
  const int64_t ox = __ldg(a.offsets + x), lx = __ldg(a.offsets + x + 1) - ox;
  const int64_t oy = __ldg(a.offsets + y), ly = __ldg(a.offsets + y + 1) - oy;
  const bool xa = lx >= ly;
  oA = xa ? ox : oy;
  m = xa ? lx : ly;
  oB = xa ? oy : ox;
  n = xa ? ly : lx;
  return true;
}

template <int W, int P>
__device__ __forceinline__ bool pair_init(PairState<W, P>& st, const VerifyArgs& a, uint32_t GW, uint64_t q, uint64_t t,
                                          uint32_t* res) {
  const uint32_t k = a.pk ? a.pk[t] : a.K;
  st.t = t;
  st.k = k;
  int64_t oA, oB, m, n;
  if (!pair_geometry(a, q, t, oA, oB, m, n)) {
    atomicOr(a.dev_flags, FLAG_BOUNDS);
    *res = k + 1;
    return false;
  }
  const int64_t d0 = m - n;
  if (d0 > (int64_t)k) {
    *res = k + 1;
    return false;
  }
  if (n == 0) {
    *res = (uint32_t)d0;
    return false;
  }
  if (m >= ((int64_t)1 << 30)) {         // column counters are 32-bit
    atomicOr(a.dev_flags, FLAG_LENGTH);
    *res = k + 1;
    return false;
  }
  const int32_t dlo = -(int32_t)(((int64_t)k - d0) >> 1);
  const int32_t t0 = (int32_t)d0 - dlo;  // bit of diagonal d0
  if (t0 >= 32 * W) {                    // cannot happen with a correct dispatch
    atomicOr(a.dev_flags, FLAG_BOUNDS);
    *res = k + 1;
    return false;
  }
  const int32_t nneg = 1 - dlo;          // band rows dlo..0 (virtual rows and row 0)
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const int lo = 32 * w;
    const uint32_t neg = nneg >= lo + 32 ? 0xffffffffu : (nneg <= lo ? 0u : ((1u << (nneg - lo)) - 1u));
    st.Mv[w] = neg;
    st.Pv[w] = ~neg;
    int32_t a0 = 1 - lo, a1 = t0 + 1 - lo;  // bits 1..t0 within this word: [a0, a1)
    a0 = a0 < 0 ? 0 : a0;
    a1 = a1 > 32 ? 32 : a1;
    const uint32_t hiMask = a1 >= 32 ? 0xffffffffu : (a1 <= 0 ? 0u : ((1u << a1) - 1u));
    const uint32_t loMask = a0 >= 32 ? 0xffffffffu : ((1u << a0) - 1u);
    st.M1[w] = a1 > a0 ? (hiMask & ~loMask) : 0u;
  }
  // the state is kept one row down, ready for the next column: the band's
  // vectors (and the diagonal mask) shifted right by one bit, Pv's new bottom
  // row +1
#pragma unroll
  for (int w = 0; w < W - 1; ++w) {
    st.Pv[w] = __funnelshift_r(st.Pv[w], st.Pv[w + 1], 1);
    st.Mv[w] = __funnelshift_r(st.Mv[w], st.Mv[w + 1], 1);
    st.M1[w] = __funnelshift_r(st.M1[w], st.M1[w + 1], 1);
  }
  st.Pv[W - 1] = (st.Pv[W - 1] >> 1) | 0x80000000u;
  st.Mv[W - 1] >>= 1;
  st.M1[W - 1] >>= 1;
  st.score = -dlo;                       // D[dlo][0] = -dlo
  st.abit = (uint64_t)(oA + dlo + 32 * (int64_t)GW);   // plane bit of row 1 + dlo (column 1)
  st.bpos = (uint64_t)(oB + 32 * (int64_t)GW);
  st.j = 1;
  st.n = (int32_t)n;
  return true;
}

// s = a + b over W 32-bit words (word 0 least significant): one carry chain
// (add.cc / addc) for bands up to 8 words, 64-bit partial sums beyond.
template <int W>
struct add_chain {
  static __device__ __forceinline__ void run(const uint32_t* a, const uint32_t* b, uint32_t* s) {
    uint32_t carry = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint64_t sum = (uint64_t)a[w] + b[w] + carry;
      carry = (uint32_t)(sum >> 32);
      s[w] = (uint32_t)sum;
    }
  }
};
template <>
struct add_chain<1> {
  static __device__ __forceinline__ void run(const uint32_t* a, const uint32_t* b, uint32_t* s) { s[0] = a[0] + b[0]; }
};
template <> struct add_chain<2> {
  static __device__ __forceinline__ void run(const uint32_t* a, const uint32_t* b, uint32_t* s) {
    asm("add.cc.u32 %0, %2, %4;\n\taddc.u32 %1, %3, %5;"
        : "=r"(s[0]), "=r"(s[1])
        : "r"(a[0]), "r"(a[1]), "r"(b[0]), "r"(b[1]));
  }
};
template <> struct add_chain<3> {
  static __device__ __forceinline__ void run(const uint32_t* a, const uint32_t* b, uint32_t* s) {
    asm("add.cc.u32 %0, %3, %6;\n\taddc.cc.u32 %1, %4, %7;\n\taddc.u32 %2, %5, %8;"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b[0]), "r"(b[1]), "r"(b[2]));
  }
};
template <> struct add_chain<4> {
  static __device__ __forceinline__ void run(const uint32_t* a, const uint32_t* b, uint32_t* s) {
    asm("add.cc.u32 %0, %4, %8;\n\taddc.cc.u32 %1, %5, %9;\n\taddc.cc.u32 %2, %6, %10;\n\taddc.u32 %3, %7, %11;"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]));
  }
};
template <> struct add_chain<5> {
  static __device__ __forceinline__ void run(const uint32_t* a, const uint32_t* b, uint32_t* s) {
    asm("add.cc.u32 %0, %5, %10;\n\taddc.cc.u32 %1, %6, %11;\n\taddc.cc.u32 %2, %7, %12;\n\taddc.cc.u32 %3, %8, %13;\n\taddc.u32 %4, %9, %14;"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]));
  }
};
template <> struct add_chain<6> {
  static __device__ __forceinline__ void run(const uint32_t* a, const uint32_t* b, uint32_t* s) {
    asm("add.cc.u32 %0, %6, %12;\n\taddc.cc.u32 %1, %7, %13;\n\taddc.cc.u32 %2, %8, %14;\n\taddc.cc.u32 %3, %9, %15;\n\taddc.cc.u32 %4, %10, %16;\n\taddc.u32 %5, %11, %17;"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]));
  }
};
template <> struct add_chain<7> {
  static __device__ __forceinline__ void run(const uint32_t* a, const uint32_t* b, uint32_t* s) {
    asm("add.cc.u32 %0, %7, %14;\n\taddc.cc.u32 %1, %8, %15;\n\taddc.cc.u32 %2, %9, %16;\n\taddc.cc.u32 %3, %10, %17;\n\taddc.cc.u32 %4, %11, %18;\n\taddc.cc.u32 %5, %12, %19;\n\taddc.u32 %6, %13, %20;"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]));
  }
};
template <> struct add_chain<8> {
  static __device__ __forceinline__ void run(const uint32_t* a, const uint32_t* b, uint32_t* s) {
    asm("add.cc.u32 %0, %8, %16;\n\taddc.cc.u32 %1, %9, %17;\n\taddc.cc.u32 %2, %10, %18;\n\taddc.cc.u32 %3, %11, %19;\n\taddc.cc.u32 %4, %12, %20;\n\taddc.cc.u32 %5, %13, %21;\n\taddc.cc.u32 %6, %14, %22;\n\taddc.u32 %7, %15, %23;"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
  }
};

// Columns between two early-exit checks: 32 (the most one load of B's bits
// covers).  With the XNOR path (8 planes), bands of one or two words take 16,
// since their pairs are often short and exit early (measured before the
// digit tables: 32 was 5% faster at 3-4 words and 8% slower at 2).  With
// digit tables every chunk rebuilds them, and 32 columns won at two words
// too (protein verify 24.9 -> 22.6 ms, with 25% more word-columns advanced).
template <int P>
constexpr bool kDigitTables = P == 2 || P == 5 || P == 7;
template <int W, int P>
constexpr int kChunkFor = (W <= 2 && !kDigitTables<P>) ? 16 : 32;

// Advances up to kChunkFor<W, P> columns; returns true when the pair is decided.
// The chunk's symbols are loaded at its start for every lane at once: A's
// plane words of the rows the band covers in these columns (pre-shifted so
// that column j0 + c needs a shift by c < 32), and B's symbols of the
// columns: with digit tables its rank codes, one byte per column; with the
// XNORs (8 planes) its plane bits, bit-reversed so that the next column's
// bit is the sign bit.
// Equality bits by digit tables (2, 5 and 7 bit-planes).  Per chunk, every
// thread writes to shared memory, for each of A's band words, the masks "rows
// whose rank code has digit value d" for each digit of the code: one digit of
// 2 bits for 2 planes (4 masks), 3 + 2 bits for 5 planes (8 + 4), 3 + 2 + 2
// bits for 7 planes (8 + 4 + 4); a column then takes its symbol's rank code
// from the input's code bytes and ANDs one mask of each digit's table (one load per word
// for 2 planes, one three-input logic op per word for 7), instead of an XNOR
// per plane and word.  Tables: word (d * (W + 1) + w) * 128 + thread, the
// digits' tables back to back.  (For 7 planes, two digits of 4 and 3 bits,
// 24 masks a word, take 50% more shared memory: 4 blocks per SM instead of
// 6.)  8 planes (byte alphabets) keep the XNORs.
template <int P>
constexpr int digit_masks() { return P == 2 ? 4 : (P == 5 ? 12 : 16); }
template <int W, int P>
constexpr size_t digit_smem_bytes() { return (size_t)digit_masks<P>() * (W + 1) * 128 * 4; }

// The masks of band word w (A's pre-shifted plane words pa) into the tables.
template <int W, int P>
__device__ __forceinline__ void build_digit_tables(const uint32_t (&pa)[P][W + 1], int w, uint32_t* __restrict__ tab,
                                                   int tid) {
  auto put = [&](int d, uint32_t v) { tab[(d * (W + 1) + w) * 128 + tid] = v; };
  auto two = [&](int p, int base) {   // a 2-bit digit from planes p, p + 1
    const uint32_t x = pa[p][w], y = pa[p + 1][w];
    put(base + 0, ~x & ~y);
    put(base + 1, x & ~y);
    put(base + 2, ~x & y);
    put(base + 3, x & y);
  };
  if constexpr (P == 2) {
    two(0, 0);
  } else {
    // a 3-bit digit from planes 0-2
    const uint32_t a0 = pa[0][w], a1 = pa[1][w], a2 = pa[2][w];
    const uint32_t t2[4] = {~a0 & ~a1, a0 & ~a1, ~a0 & a1, a0 & a1};
#pragma unroll
    for (int d = 0; d < 8; ++d) put(d, t2[d & 3] & ((d & 4) ? a2 : ~a2));
    two(3, 8);
    if constexpr (P == 7) two(5, 12);
  }
}

// The equality bits of a symbol with rank code `code` over the band's words.
template <int W, int P>
__device__ __forceinline__ void digit_lookup(const uint32_t* __restrict__ tab, uint32_t code, int tid,
                                             uint32_t (&EqF)[W + 1]) {
  constexpr int S = (W + 1) * 128;
  if constexpr (P == 2) {
    const uint32_t* t = tab + code * S + tid;
#pragma unroll
    for (int w = 0; w <= W; ++w) EqF[w] = t[w * 128];
  } else if constexpr (P == 5) {
    const uint32_t* ta = tab + (code & 7u) * S + tid;
    const uint32_t* tb = tab + (8u + (code >> 3)) * S + tid;
#pragma unroll
    for (int w = 0; w <= W; ++w) EqF[w] = ta[w * 128] & tb[w * 128];
  } else {
    const uint32_t* ta = tab + (code & 7u) * S + tid;
    const uint32_t* tb = tab + (8u + ((code >> 3) & 3u)) * S + tid;
    const uint32_t* tc = tab + (12u + (code >> 5)) * S + tid;
#pragma unroll
    for (int w = 0; w <= W; ++w) EqF[w] = ta[w * 128] & tb[w * 128] & tc[w * 128];
  }
}

template <int W, int P>
__device__ __forceinline__ bool pair_chunk(PairState<W, P>& st, const VerifyArgs& a, uint64_t PW, uint32_t* res,
                                           uint32_t* __restrict__ tab, uint32_t GW) {
  constexpr bool kDigits = kDigitTables<P>;
  const int32_t j0 = st.j;
  uint32_t pa[P][W + 1];
  uint32_t bw[P];
  uint32_t bsym[kDigits ? 8 : 1];   // B's rank codes of the chunk's columns, four per word
  {
    const uint64_t ab = st.abit + (uint64_t)(j0 - 1);
    const uint64_t aw = ab >> 5;
    const uint32_t ash = (uint32_t)(ab & 31);
    const uint64_t wb = st.bpos >> 5;
    const uint32_t sb = (uint32_t)(st.bpos & 31);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      if (p < (int)a.bits) {
        const uint32_t* plane = a.planes + (uint64_t)p * PW;
        uint32_t w0 = __ldg(plane + aw);
#pragma unroll
        for (int w = 0; w <= W; ++w) {
          const uint32_t w1 = __ldg(plane + aw + w + 1);
          pa[p][w] = __funnelshift_r(w0, w1, ash);
          w0 = w1;
        }
        if (!kDigits) bw[p] = __brev(__funnelshift_r(__ldg(plane + wb), __ldg(plane + wb + 1), sb));
      } else {
#pragma unroll
        for (int w = 0; w <= W; ++w) pa[p][w] = 0u;
        bw[p] = 0u;
      }
    }
    if (kDigits) {
      const int tid = threadIdx.x;
#pragma unroll
      for (int w = 0; w <= W; ++w) build_digit_tables<W, P>(pa, w, tab, tid);
      // B's rank codes of columns j0 .. j0 + 31, aligned so that column j0 + c
      // is byte c (words beyond the input read as zero)
      const uint64_t bi = st.bpos - 32 * (uint64_t)GW;   // byte index of column j0's symbol
      const uintptr_t at0 = (uintptr_t)(a.codes + bi);
      const uint32_t sh = 8u * (uint32_t)(at0 & 3);
      const uintptr_t wa = at0 & ~(uintptr_t)3;
      const uintptr_t lo_end = (uintptr_t)a.codes, hi_end = (uintptr_t)(a.codes + a.nbytes);
      uint32_t raw[9];
      if (wa >= lo_end && wa + 36 <= hi_end) {   // the common case: nine aligned words inside the input
#pragma unroll
        for (int k = 0; k < 9; ++k) raw[k] = __ldg(reinterpret_cast<const uint32_t*>(wa) + k);
      } else {   // near an end of the input: byte by byte, zero outside it
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          uint32_t x = 0;
          for (int b = 0; b < 4; ++b) {
            const uintptr_t q = wa + 4 * k + b;
            if (q >= lo_end && q < hi_end) x |= (uint32_t)__ldg(reinterpret_cast<const uint8_t*>(q)) << (8 * b);
          }
          raw[k] = x;
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) bsym[k] = __funnelshift_r(raw[k], raw[k + 1], sh);
    }
  }
  constexpr int kChunk = kChunkFor<W, P>;
  const int32_t cnt = min(kChunk, st.n - j0 + 1);
  // The top row's D moves along a diagonal, so it rises by 0 or 1 per
  // column: by 1 exactly when the vertical delta entering the row and the
  // horizontal delta leaving it are +1 and 0 or 0 and +1 (the pairs summing
  // to 2 or -2 cannot occur).  Bit 0 of (Pv | Ph) & ~(Mv | Mh) per column,
  // shifted into `rises` (one bit per column, at most 32), and counted at the
  // end of the chunk.
  uint32_t rises = 0;
#pragma unroll 8   // part of the chunk: a smaller body is fetched better (measured)
  for (int c = 0; c < kChunk; ++c) {
    if (c >= cnt) break;
    // equality bits of column j0 + c: A's plane bits XNOR B's, over the planes
    uint32_t EqF[W + 1];
    if constexpr (kDigits) {
      const uint32_t code = (bsym[c >> 2] >> (8 * (c & 3))) & 255u;
      digit_lookup<W, P>(tab, code, threadIdx.x, EqF);
    } else {
#pragma unroll
      for (int w = 0; w <= W; ++w) EqF[w] = 0xffffffffu;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        if (p < (int)a.bits) {
          const uint32_t xb = (uint32_t)__mulhi((int32_t)bw[p], 1);   // B's bit broadcast (sign)
          bw[p] *= 2u;
#pragma unroll
          for (int w = 0; w <= W; ++w) EqF[w] &= ~(pa[p][w] ^ xb);
        }
      }
    }
    uint32_t Eq[W];
#pragma unroll
    for (int w = 0; w < W; ++w) Eq[w] = __funnelshift_r(EqF[w], EqF[w + 1], (uint32_t)c);


    uint32_t Xv[W], Ph[W], Mh[W], EP[W], SUM[W];
#pragma unroll
    for (int w = 0; w < W; ++w) EP[w] = Eq[w] & st.Pv[w];
    add_chain<W>::run(EP, st.Pv, SUM);   // (Eq & Pv) + Pv across the band's words
#pragma unroll
    for (int w = 0; w < W; ++w) {
      Xv[w] = Eq[w] | st.Mv[w];
      const uint32_t Xh = (SUM[w] ^ st.Pv[w]) | Eq[w];
      Ph[w] = st.Mv[w] | ~(Xh | st.Pv[w]);
      Mh[w] = st.Pv[w] & Xh;
    }
    // the band has slid down one row already (the vectors are kept shifted):
    // bit 0 of Pv / Mv is the vertical delta entering the top row
    rises = __funnelshift_r(rises, (st.Pv[0] | Ph[0]) & ~(st.Mv[0] | Mh[0]), 1);
    // Myers' update Pv' = (Mh << 1) | ~(Xv | (Ph << 1) | 1), Mv' = ((Ph << 1) | 1)
    // & Xv, followed by the next column's slide (>> 1, Pv's new bottom row +1),
    // is Pv = Mh | ~((Xv >> 1) | Ph) | top, Mv = Ph & (Xv >> 1): one shift
    // instead of four per word.
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t xs = w + 1 < W ? __funnelshift_r(Xv[w], Xv[w + 1], 1) : Xv[w] >> 1;
      st.Pv[w] = Mh[w] | ~(xs | Ph[w]);
      st.Mv[w] = Ph[w] & xs;
    }
    st.Pv[W - 1] |= 0x80000000u;
  }
  const int32_t jend = j0 + cnt - 1;
  st.j = jend + 1;
  st.bpos += (uint64_t)cnt;
  st.score += __popc(rises);
  // D on diagonal d0 at column jend: a lower bound of D[m][n] (exact at n);
  // M1 (kept shifted like the vectors) selects the rows below the top row
  // down to diagonal d0
  int32_t diag = st.score;
#pragma unroll
  for (int w = 0; w < W; ++w) diag += (int32_t)__popc(st.Pv[w] & st.M1[w]) - (int32_t)__popc(st.Mv[w] & st.M1[w]);
  if (diag > (int32_t)st.k) {
    *res = st.k + 1;
    return true;
  }
  if (jend == st.n) {
    *res = (uint32_t)diag;
    return true;
  }
  return false;
}

// Persistent verifier: every lane keeps one pair in flight and fetches the
// next pair index (warp-aggregated atomic on *next) as soon as its pair is
// decided, so early exits do not leave lanes idle behind slow pairs.
template <int W, int P>
__global__ void __launch_bounds__(128, (P == 7 && W <= 3) ? 7 : ((P == 5 && W <= 2) ? 8 : 1)) verify_diag_kernel(VerifyArgs a, uint64_t PW, uint32_t GW,
                                                          unsigned long long* __restrict__ next) {
  extern __shared__ __align__(16) uint32_t vsm[];   // the digit tables
  uint32_t* tab = vsm;
  const int lane = threadIdx.x & 31;
  const uint64_t q_lo = a.range_lo ? *a.range_lo : 0;
  const uint64_t q_hi = a.range_hi ? *a.range_hi : a.m;
  PairState<W, P> st;
  bool active = false;
  bool more = true;
  uint64_t cells = 0, work = 0, nskip = 0;
  while (true) {
    // lanes without a pair fetch the next indices
    const bool need = !active && more;
    const uint32_t nmask = __ballot_sync(0xffffffffu, need);
    if (nmask) {
      unsigned long long base = 0;
      const int leader = __ffs(nmask) - 1;
      if (lane == leader) base = atomicAdd(next, (unsigned long long)__popc(nmask));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const uint64_t q = q_lo + base + __popc(nmask & ((1u << lane) - 1u));
        if (q >= q_hi) {
          more = false;
        } else {
          const uint64_t t = a.order ? a.order[q] : q;
          // a pair the first pass already decided needs nothing: the lane
          // stays idle and fetches again at the next iteration
          const uint32_t* fed = a.first_ed ? a.first_ed : a.ed;
          const bool settled = a.skip_kband && a.skip_kband[t] < a.K && fed[t] <= a.skip_kband[t];
          if (settled && a.first_ed) put_result(a, t, fed[t]);
          nskip += settled ? 1 : 0;
          if (!settled) {
            if (a.cells) {
              const uint32_t x = a.pi[t], y = a.pj[t];
              if (x < a.n_strings && y < a.n_strings) {
                const int64_t lx = __ldg(a.offsets + x + 1) - __ldg(a.offsets + x);
                const int64_t ly = __ldg(a.offsets + y + 1) - __ldg(a.offsets + y);
                cells += band_cells(lx > ly ? lx : ly, lx > ly ? ly : lx, a.K);
              }
            }
            uint32_t res;
            if (pair_init<W, P>(st, a, GW, q, t, &res)) {
              active = true;
            } else {
              put_result(a, t, res);
            }
          }
        }
      }
    }
    if (!__any_sync(0xffffffffu, active || more)) break;
    if (active) {
      uint32_t res;
      const int32_t j_before = st.j;
      const bool done = pair_chunk<W, P>(st, a, PW, &res, tab, GW);
      work += (uint64_t)(st.j - j_before) * W;
      if (done) {
        put_result(a, st.t, res);
        active = false;
      }
    }
  }
  if (a.cells) {
    for (int o = 16; o > 0; o >>= 1) cells += __shfl_down_sync(0xffffffffu, cells, o);
    if (lane == 0 && cells) atomicAdd(a.cells, (unsigned long long)cells);
  }
  if (a.work) {
    for (int o = 16; o > 0; o >>= 1) work += __shfl_down_sync(0xffffffffu, work, o);
    if (lane == 0 && work) atomicAdd(a.work, (unsigned long long)work);
  }
  if (a.skipped) {
    for (int o = 16; o > 0; o >>= 1) nskip += __shfl_down_sync(0xffffffffu, nskip, o);
    if (lane == 0 && nskip) atomicAdd(a.skipped, (unsigned long long)nskip);
  }
}

// ---------------------------------------------------------------- wide bands
// Row-fixed blocks with a skewed wavefront, G lanes per pair.
//
// Rows are cut into 32-row blocks (block b = rows 32b+1 .. 32b+32, one 32-bit
// word per vector); lane b mod G of the pair's group owns block b.  Block b
// advances column j at step s = j + b: it needs the horizontal delta of the
// row just above it in column j, which the lane owning block b-1 produced one
// step earlier and passes on by a shuffle.  A block works on the columns in
// which some of its rows lie in the band [j + dlo, j + dhi]; outside, a block
// entering the band starts from vertical deltas of +1 and the row above a
// retired block gets a horizontal delta of +1 (the same over-estimates as the
// diagonal kernel).  With an incoming horizontal delta hin in {-1, 0, +1}, a
// block step is the recurrence of the diagonal kernel with the top row's
// chain seeded by hin: Xh's carry chain starts set when hin = -1, and the
// shifted-in top bit of Ph (Mh) is set when hin = +1 (-1).  Each block keeps
// D of its bottom row; the bottom row of the block holding row m at column n
// gives D[m][n], and the block holding row j + d0 at column j gives the
// diagonal lower bound used for the early exit.
constexpr int kWaveSteps = 32;   // wavefront steps between refills and votes (<= 32: B's bits per reload)

// Each lane publishes one word per wavefront step for the lane holding the
// next block of rows:
//   bit 31      the block's bottom row gained +1 in this column (hout = +1)
//   bits 1..30  D at the block's bottom row in this column (the score)
//   bit 0       hout = -1
// The next lane reads it only in the columns that block b - 1 shares with
// block b; elsewhere the top row's delta is kIdle, +1 (the band's edge).
constexpr uint32_t kIdle = 0x80000000u;
constexpr int32_t kDeadU = -0x40000000;   // step offset of a lane without a block
constexpr uint32_t kMaxLen = 1u << 27;     // scores must fit bits 1..30

template <int P>
__device__ __forceinline__ void wave_load_bits(const VerifyArgs& a, uint64_t PW, uint64_t pos, uint32_t (&v)[P],
                                               bool reverse) {
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const uint32_t lo = p < (int)a.bits ? __ldg(a.planes + (uint64_t)p * PW + (pos >> 5)) : 0u;
    const uint32_t hi = p < (int)a.bits ? __ldg(a.planes + (uint64_t)p * PW + (pos >> 5) + 1) : 0u;
    const uint32_t x = __funnelshift_r(lo, hi, (uint32_t)(pos & 31));
    v[p] = reverse ? __brev(x) : x;
  }
}

// One column of a 32-row block (Myers' step in Hyyro's formulation).  wv
// carries the horizontal delta entering the top row (bit 31: +1, bit 0: -1,
// neither: 0); B's symbol is bit 31 of bw[] (consumed, shifted out); T's
// score bits (1..30) follow the bottom row; Ph keeps the bottom row's +1 in
// bit 31 and hn is its -1.  Bit extraction, shifts and disjoint ORs are
// written as integer multiply-adds, which the FMA pipe can take: the logic
// ops already fill the ALU pipe.
__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {   // a * b + c on the FMA pipe
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// pub: the word published to the next lane, ((Ph & 2^31) | T) + hn with the
// updated T (bit 31 and bit 0 of T are clear), formed by multiply-adds as
// T_old + hp (2^31 + 2) - hn.
template <int P>
__device__ __forceinline__ void wave_column(const uint32_t (&pa)[P], uint32_t (&bw)[P], uint32_t wv, uint32_t& Pv,
                                            uint32_t& Mv, uint32_t& T, uint32_t& Ph, uint32_t& hn, uint32_t& pub) {
  uint32_t Eq = 0xffffffffu;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const uint32_t xb = (uint32_t)__mulhi((int32_t)bw[p], 1);   // B's bit p broadcast (sign of bw)
    Eq &= ~(pa[p] ^ xb);
    bw[p] *= 2u;
  }
  const uint32_t hin_neg = wv & 1u;
  const uint32_t hin_pos = __umulhi(wv, 2u);
  const uint32_t Xv = Eq | Mv;
  const uint32_t Eh = Eq | hin_neg;
  const uint32_t Xh = (((Eh & Pv) + Pv) ^ Pv) | Eh;
  Ph = Mv | ~(Xh | Pv);
  const uint32_t Mh = Pv & Xh;
  hn = __umulhi(Mh, 2u);
  const uint32_t hp = __umulhi(Ph, 2u);
  pub = mad_lo(hn, 0xffffffffu, mad_lo(hp, 0x80000002u, T));
  T = mad_lo(hn, 0xfffffffeu, mad_lo(hp, 2u, T));
  const uint32_t Ph1 = Ph * 2u + hin_pos;   // (Ph << 1) | hin > 0
  const uint32_t Mh1 = Mh * 2u + hin_neg;   // (Mh << 1) | hin < 0
  Pv = Mh1 | ~(Xv | Ph1);
  Mv = Ph1 & Xv;
}

template <int G, int P>
__global__ void __launch_bounds__(128, P <= 2 ? 8 : 1) verify_wave_kernel(VerifyArgs a, uint64_t PW, uint32_t GW,
                                                          unsigned long long* __restrict__ next) {
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1);
  const int gbase = lane - gl;
  const uint32_t gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << gbase);
  const int prev_lane = gbase + ((gl + G - 1) & (G - 1));
  const uint64_t q_lo = a.range_lo ? *a.range_lo : 0;
  const uint64_t q_hi = a.range_hi ? *a.range_hi : a.m;
  // pair state (identical in the G lanes of a group)
  bool has = false, more = true;
  uint64_t t = 0;
  uint32_t k = 0;
  int64_t oA = 0, oB = 0;
  int32_t m = 0, n = 0, d0 = 0, dlo = 0, dhi = 0, bm = 0;
  int32_t sbase = 0;   // wavefront steps done on the pair
  // block state (this lane): block b runs at the steps where 0 <= u <= span
  // (u counts up by one per step); block b - 1 computed the same column one
  // step earlier while u <= u_valid; diagonal d0 crosses it where
  // 0 <= u + dg < 32
  int32_t b = 0, u = kDeadU, span = 0, u_valid = -1, dg = 0x40000000;
  uint32_t T = 0;   // score << 1
  uint32_t Pv = 0, Mv = 0;
  uint32_t pa[P], bw[P];
  uint32_t pub = kIdle;
  bool done = false, reject = false;
  int32_t result = 0;
  uint64_t work = 0, cells = 0, nskip = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) pa[p] = bw[p] = 0u;

  // Take block nb after step s.  Its columns are [jf, jl]; block nb computes
  // column j at step j + nb.  Blocks past row m never run.
  auto take_block = [&](int32_t nb, int32_t s) {
    b = nb;
    if (b <= bm) {
      const int32_t jf = max(1, 32 * b + 1 - dhi);
      const int32_t jl = min(n, 32 * b + 32 - dlo);
      u = s - (jf + b);
      span = jl - jf;
      u_valid = b == 0 ? -1 : min(n, 32 * b - dlo) - jf;   // last column of block b - 1
      dg = jf - 32 * b - 1 + d0;   // row j + d0 is row 32 b + 1 + (u + dg)
    } else {
      u = kDeadU;
      span = 0;
      u_valid = -1;
      dg = 0x40000000;
    }
  };

  while (true) {
    // ---- groups without a pair take pairs until they hold one that needs
    // the wavefront (one vote while all groups are busy)
    while (true) {
      const bool need = !has && more;
      const uint32_t leaders = __ballot_sync(0xffffffffu, need && gl == 0);
      if (!leaders) break;
      const int first = __ffs(leaders) - 1;
      unsigned long long base = 0;
      if (lane == first) base = atomicAdd(next, (unsigned long long)__popc(leaders));
      base = __shfl_sync(0xffffffffu, base, first);
      const uint64_t q = q_lo + base + __popc(leaders & ((1u << gbase) - 1u));
      if (need) {
        if (q >= q_hi) {
          more = false;
        } else {
          t = a.order ? a.order[q] : q;
          int64_t gm = 0, gn = 0;
          k = a.pk ? a.pk[t] : a.K;
          uint32_t res = 0xffffffffu;
          const uint32_t* fed = a.first_ed ? a.first_ed : a.ed;
          const bool skip = a.skip_kband && a.skip_kband[t] < a.K && fed[t] <= a.skip_kband[t];
          if (skip) {
            if (a.first_ed && gl == 0) put_result(a, t, fed[t]);
            res = 0xfffffffeu;   // settled by the first pass: nothing to do
          } else if (!pair_geometry(a, q, t, oA, oB, gm, gn)) {
            if (gl == 0) atomicOr(a.dev_flags, FLAG_BOUNDS);
            res = k + 1;
          } else {
            if (a.cells && gl == 0) cells += band_cells(gm, gn, a.K);
            const int64_t mm = gm, nn = gn;
            if (mm >= (int64_t)kMaxLen) {
              if (gl == 0) atomicOr(a.dev_flags, FLAG_LENGTH);
              res = k + 1;
            } else if (mm - nn > (int64_t)k) {
              res = k + 1;
            } else if (nn == 0) {
              res = (uint32_t)mm;
            } else {
              m = (int32_t)mm;
              n = (int32_t)nn;
              d0 = m - n;
              dlo = -(int32_t)((k - (uint32_t)d0) >> 1);
              dhi = d0 + (int32_t)((k - (uint32_t)d0) >> 1);
              if (dhi - dlo < 63) dlo = dhi - 63;   // at least 64 band rows (any wider band is exact)
              bm = (m - 1) >> 5;
              sbase = 0;
              take_block(gl, 0);
              pub = kIdle;
              done = reject = false;
            }
          }
          if (res == 0xfffffffeu) {
            if (gl == 0) ++nskip;
          } else if (res != 0xffffffffu) {
            if (gl == 0) put_result(a, t, res);
          } else {
            has = true;
          }
        }
      }
    }
    if (!__any_sync(0xffffffffu, has || more)) break;

    // ---- kWaveSteps wavefront steps.  Every lane runs the column step; a lane
    // outside its block's steps computes on stale state (rebuilt at the
    // block's first column) that no other lane reads.  First and last
    // columns and the diagonal test take one rarely divergent branch.
    // Steps in which no lane of the warp meets such an event (a block's first
    // or last column, its input word switching from the predecessor's to the
    // band edge's, the window's last step) run in a loop without the tests:
    // their number is the warp's minimum of the steps to each lane's next
    // event.
    int it = 0;
    while (it < kWaveSteps) {
      {
        const int64_t un = (int64_t)u + 1;   // u at the next step
        int64_t fr = kWaveSteps - 1 - it;
        if (un <= 0) fr = min(fr, -un);
        if (un <= span) fr = min(fr, (int64_t)span - un);
        if (un <= u_valid) fr = min(fr, (int64_t)u_valid - un + 1);
        const int free = __reduce_min_sync(0xffffffffu, (int)fr);
        const bool from_prev = un <= u_valid;
        const uint32_t keep_in = from_prev ? 1u : 0u, idle_in = from_prev ? 0u : kIdle;
#pragma unroll 4
        for (int f = 0; f < free; ++f) {
          const uint32_t w_in = __shfl_sync(0xffffffffu, pub, prev_lane);
          const uint32_t wv = mad_lo(w_in, keep_in, idle_in);   // w_in, or kIdle at the band's edge
          uint32_t Ph, hn;
          wave_column<P>(pa, bw, wv, Pv, Mv, T, Ph, hn, pub);
        }
        u += free;
        it += free;
      }
      const uint32_t w_in = __shfl_sync(0xffffffffu, pub, prev_lane);
      ++u;
      const uint32_t wv = u <= u_valid ? w_in : kIdle;
      uint32_t Ph, hn;
      wave_column<P>(pa, bw, wv, Pv, Mv, T, Ph, hn, pub);
      const bool diag_here = it == kWaveSteps - 1 && (uint32_t)(u + dg) < 32u;
      if (u == 0 || u == span || diag_here) {
        if (u == 0) {   // first column: load the block's symbols, rows start from +1 deltas
          const int32_t jf = sbase + it + 1 - b;
          wave_load_bits<P>(a, PW, (uint64_t)(oA + 32 * (int64_t)b + 32 * (int64_t)GW), pa, false);
          wave_load_bits<P>(a, PW, (uint64_t)(oB + jf - 1 + 32 * (int64_t)GW), bw, true);
          Pv = 0xffffffffu;
          Mv = 0u;
          wave_column<P>(pa, bw, wv, Pv, Mv, T, Ph, hn, pub);
          // D of the row above the block in this column, plus the block's deltas
          const int32_t above = b == 0 ? 1 : (int32_t)((w_in >> 1) & 0x3fffffffu);
          const int32_t score = above + (int32_t)__popc(Pv) - (int32_t)__popc(Mv);
          T = (uint32_t)score << 1;
          pub = ((Ph & 0x80000000u) | T) + hn;
        }
        // D at row r of this block = score minus the deltas of the rows below r
        if (diag_here && (uint32_t)u <= (uint32_t)span) {   // row j + d0 of diagonal d0
          const int tr = u + dg;
          const uint32_t below = tr == 31 ? 0u : (0xffffffffu << (tr + 1));
          const int32_t diag = (int32_t)(T >> 1) - (int32_t)__popc(Pv & below) + (int32_t)__popc(Mv & below);
          if (diag > (int32_t)k) reject = true;
        }
        if (u == span) {   // the block leaves the band
          if (b == bm) {
            const int tm = (m - 1) & 31;
            const uint32_t below = tm == 31 ? 0u : (0xffffffffu << (tm + 1));
            result = (int32_t)(T >> 1) - (int32_t)__popc(Pv & below) + (int32_t)__popc(Mv & below);
            done = true;
          }
          work += (uint64_t)(span + 1);
          take_block(b + G, sbase + it + 1);
        }
      }
      ++it;
    }
    sbase += kWaveSteps;
    if ((sbase & 31) == 0 && u >= 0 && u <= span) {   // B's symbols of the next 32 columns, all lanes at once
      wave_load_bits<P>(a, PW, (uint64_t)(oB + (sbase - b) + 32 * (int64_t)GW), bw, true);
    }
    // ---- a group whose pair finished (or was rejected) writes it and frees
    // its lanes; one vote in the common case where none did
    const bool overrun = has && sbase >= n + bm;   // cannot happen: the last block ends at step n + bm
    if (__ballot_sync(0xffffffffu, done || reject || overrun)) {
      const uint32_t dmask = __ballot_sync(0xffffffffu, done) & gmask;
      const uint32_t rmask = __ballot_sync(0xffffffffu, reject) & gmask;
      const int src = dmask ? __ffs(dmask) - 1 : lane;
      const int32_t fin = __shfl_sync(0xffffffffu, result, src);
      bool end = false;
      if (has && (dmask || rmask)) {
        if (gl == 0) put_result(a, t, rmask ? k + 1 : (fin > (int32_t)k ? k + 1 : (uint32_t)fin));
        end = true;
      } else if (overrun) {
        if (gl == 0) {
          atomicOr(a.dev_flags, FLAG_BOUNDS);
          put_result(a, t, k + 1);
        }
        end = true;
      }
      if (end) {
        if (u >= 0 && u <= span) work += (uint64_t)(u + 1);   // block cut short by the exit
        has = false;
        u = kDeadU;
        span = 0;
        u_valid = -1;
        dg = 0x40000000;
        pub = kIdle;
        done = reject = false;
      }
    }
  }
  if (a.work) {
    for (int o = 16; o > 0; o >>= 1) work += __shfl_down_sync(0xffffffffu, work, o);
    if (lane == 0 && work) atomicAdd(a.work, (unsigned long long)work);
  }
  if (a.cells) {
    for (int o = 16; o > 0; o >>= 1) cells += __shfl_down_sync(0xffffffffu, cells, o);
    if (lane == 0 && cells) atomicAdd(a.cells, (unsigned long long)cells);
  }
  if (a.skipped) {
    for (int o = 16; o > 0; o >>= 1) nskip += __shfl_down_sync(0xffffffffu, nskip, o);
    if (lane == 0 && nskip) atomicAdd(a.skipped, (unsigned long long)nskip);
  }
}

// ---------------------------------------------------------------- bands wider than one warp
// One CTA of V warps (G = 32 V lanes) per pair, for bands whose wavefront
// needs more than 32 lanes (K >= 1025).  Blocks, lanes and the column step
// are those of verify_wave_kernel (lane g owns blocks b = g mod G), with one
// change to the schedule: block b computes column j at step
//     j + b + 32 floor(b / 32),
// i.e. every group of 32 blocks runs one window of kWaveSteps (= 32) steps
// behind the group above it.  Inside a group the predecessor block b - 1 is
// the next lane down in the same warp and hands its word over by a shuffle,
// one step earlier as before.  The first block of a group (lane 0 of its
// warp) takes its predecessor's word from the last lane of the previous warp,
// written 33 steps earlier into a ring in shared memory: the CTA synchronises
// once per window (__syncthreads), after which the previous window's words
// are visible.  The extra skew also spaces a lane's consecutive blocks b and
// b + G by 2G steps instead of G, so G lanes hold any band with
//     34 G >= 32 + (dhi - dlo),  dhi - dlo <= K.
// Pair fetch, the early exit and the result are CTA-wide decisions taken at
// the window barrier; every loop bound is uniform over the CTA.
constexpr int kRing = 128;   // words per warp in the ring: steps s - 128 .. s - 1 (reads reach s - 33)

template <int V, int P>
__global__ void __launch_bounds__(32 * V) verify_cta_kernel(VerifyArgs a, uint64_t PW, uint32_t GW,
                                                            unsigned long long* __restrict__ next) {
  constexpr int G = 32 * V;
  constexpr int S = kWaveSteps;
  static_assert(S == 32 && kRing >= 2 * S + 2 && (kRing & (kRing - 1)) == 0, "window and ring sizes");
  __shared__ uint32_t ring[V][kRing];
  __shared__ unsigned long long s_t;   // pair of the CTA (~0: none left)
  __shared__ longlong2 s_geo;          // its offsets of A and B
  __shared__ int2 s_len;               // and lengths m >= n
  __shared__ int s_flag[3];            // per window (mod 3): 1 = finished, 2 = rejected
  __shared__ int32_t s_result[3];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int prev_warp = (warp + V - 1) % V;
  const uint64_t q_lo = a.range_lo ? *a.range_lo : 0;
  const uint64_t q_hi = a.range_hi ? *a.range_hi : a.m;
  if (tid < 3) s_flag[tid] = 0;
  uint32_t k = 0;
  int64_t oA = 0, oB = 0;
  int32_t m = 0, n = 0, d0 = 0, dlo = 0, dhi = 0, bm = 0;
  int32_t b = 0, u = kDeadU, span = 0, u_valid = -1, dg = 0x40000000, colbase = 0;
  uint32_t T = 0, Pv = 0, Mv = 0;
  uint32_t pa[P], bw[P];
  uint32_t pub = kIdle;
  bool done = false, reject = false;
  int32_t result = 0;
  uint32_t win = 0;   // windows run by the CTA (selects the flag slot)
  uint64_t work = 0, cells = 0, nskip = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) pa[p] = bw[p] = 0u;

  // Take block nb after s steps.  Its columns are [jf, jl]; it computes
  // column j at step j + colbase (colbase = nb + 32 floor(nb / 32)).
  auto take_block = [&](int32_t nb, int32_t s) {
    b = nb;
    if (b <= bm) {
      const int32_t jf = max(1, 32 * b + 1 - dhi);
      const int32_t jl = min(n, 32 * b + 32 - dlo);
      colbase = b + S * (b >> 5);
      u = s - (jf + colbase);
      span = jl - jf;
      u_valid = b == 0 ? -1 : min(n, 32 * b - dlo) - jf;   // last column of block b - 1
      dg = jf - 32 * b - 1 + d0;
    } else {
      u = kDeadU;
      span = 0;
      u_valid = -1;
      dg = 0x40000000;
      colbase = 0;
    }
  };

  while (true) {
    // ---- thread 0 takes pairs until one needs the wavefront
    if (tid == 0) {
      unsigned long long got = ~0ull;
      while (true) {
        const uint64_t q = q_lo + atomicAdd(next, 1ull);
        if (q >= q_hi) break;
        const uint64_t t = a.order ? a.order[q] : q;
        const uint32_t kt = a.pk ? a.pk[t] : a.K;
        const uint32_t* fed = a.first_ed ? a.first_ed : a.ed;
        if (a.skip_kband && a.skip_kband[t] < a.K && fed[t] <= a.skip_kband[t]) {
          if (a.first_ed) put_result(a, t, fed[t]);
          ++nskip;
          continue;
        }
        int64_t gA, gB, mm, nn;
        if (!pair_geometry(a, q, t, gA, gB, mm, nn)) {
          atomicOr(a.dev_flags, FLAG_BOUNDS);
          put_result(a, t, kt + 1);
          continue;
        }
        if (a.cells) cells += band_cells(mm, nn, a.K);
        if (mm >= (int64_t)kMaxLen) {
          atomicOr(a.dev_flags, FLAG_LENGTH);
          put_result(a, t, kt + 1);
          continue;
        }
        if (mm - nn > (int64_t)kt) {
          put_result(a, t, kt + 1);
          continue;
        }
        if (nn == 0) {
          put_result(a, t, (uint32_t)mm);
          continue;
        }
        got = t;
        s_geo = make_longlong2(gA, gB);
        s_len = make_int2((int32_t)mm, (int32_t)nn);
        break;
      }
      s_t = got;
    }
    __syncthreads();
    const unsigned long long t = s_t;
    if (t == ~0ull) break;
    {
      k = a.pk ? a.pk[t] : a.K;
      const longlong2 geo = s_geo;
      const int2 len = s_len;
      oA = geo.x;
      oB = geo.y;
      m = len.x;
      n = len.y;
      d0 = m - n;
      dlo = -(int32_t)((k - (uint32_t)d0) >> 1);
      dhi = d0 + (int32_t)((k - (uint32_t)d0) >> 1);
      if (dhi - dlo < 63) dlo = dhi - 63;
      bm = (m - 1) >> 5;
    }
    take_block(tid, 0);
    pub = kIdle;
    done = reject = false;
    const int32_t last_step = n + bm + S * (bm >> 5);   // block bm's last column
    int32_t sbase = 0;
    while (true) {
#pragma unroll 8
      for (int it = 0; it < S; ++it) {
        const int32_t s1 = sbase + it + 1;   // this step, counted from 1
        uint32_t w_in = __shfl_up_sync(0xffffffffu, pub, 1);
        if (lane == 0) w_in = ring[prev_warp][(uint32_t)(s1 - 1 - S) & (kRing - 1)];
        ++u;
        const uint32_t wv = u <= u_valid ? w_in : kIdle;
        uint32_t Ph, hn;
        wave_column<P>(pa, bw, wv, Pv, Mv, T, Ph, hn, pub);
        const bool diag_here = it == S - 1 && (uint32_t)(u + dg) < 32u;
        if (u == 0 || u == span || diag_here) {
          if (u == 0) {   // first column: load the block's symbols, rows start from +1 deltas
            const int32_t jf = s1 - colbase;
            wave_load_bits<P>(a, PW, (uint64_t)(oA + 32 * (int64_t)b + 32 * (int64_t)GW), pa, false);
            wave_load_bits<P>(a, PW, (uint64_t)(oB + jf - 1 + 32 * (int64_t)GW), bw, true);
            Pv = 0xffffffffu;
            Mv = 0u;
            wave_column<P>(pa, bw, wv, Pv, Mv, T, Ph, hn, pub);
            const int32_t above = b == 0 ? 1 : (int32_t)((w_in >> 1) & 0x3fffffffu);
            const int32_t score = above + (int32_t)__popc(Pv) - (int32_t)__popc(Mv);
            T = (uint32_t)score << 1;
            pub = ((Ph & 0x80000000u) | T) + hn;
          }
          if (diag_here && (uint32_t)u <= (uint32_t)span) {   // row j + d0 of diagonal d0
            const int tr = u + dg;
            const uint32_t below = tr == 31 ? 0u : (0xffffffffu << (tr + 1));
            const int32_t diag = (int32_t)(T >> 1) - (int32_t)__popc(Pv & below) + (int32_t)__popc(Mv & below);
            if (diag > (int32_t)k) reject = true;
          }
          if (u == span) {   // the block leaves the band
            if (b == bm) {
              const int tm = (m - 1) & 31;
              const uint32_t below = tm == 31 ? 0u : (0xffffffffu << (tm + 1));
              result = (int32_t)(T >> 1) - (int32_t)__popc(Pv & below) + (int32_t)__popc(Mv & below);
              done = true;
            }
            work += (uint64_t)(span + 1);
            take_block(b + G, s1);
          }
        }
        if (lane == 31) ring[warp][(uint32_t)s1 & (kRing - 1)] = pub;
      }
      sbase += S;
      if (u >= 0 && u <= span)   // B's symbols of the next 32 columns
        wave_load_bits<P>(a, PW, (uint64_t)(oB + (sbase - colbase) + 32 * (int64_t)GW), bw, true);
      const uint32_t slot = win % 3;
      if (done) {
        s_result[slot] = result;
        atomicOr(&s_flag[slot], 1);
      }
      if (reject) atomicOr(&s_flag[slot], 2);
      __syncthreads();
      const int f = s_flag[slot];
      const int32_t fin = s_result[slot];
      if (tid == 0) s_flag[(win + 2) % 3] = 0;
      ++win;
      const bool overrun = sbase >= last_step;   // finished at the latest in the window of step last_step
      if (f || overrun) {
        if (tid == 0) {
          if (f & 1) {
            put_result(a, t, fin > (int32_t)k ? k + 1 : (uint32_t)fin);
          } else if (f & 2) {
            put_result(a, t, k + 1);
          } else {
            atomicOr(a.dev_flags, FLAG_BOUNDS);
            put_result(a, t, k + 1);
          }
        }
        if (u >= 0 && u <= span) work += (uint64_t)(u + 1);   // block cut short by the exit
        break;
      }
    }
  }
  if (a.work) {
    for (int o = 16; o > 0; o >>= 1) work += __shfl_down_sync(0xffffffffu, work, o);
    if (lane == 0 && work) atomicAdd(a.work, (unsigned long long)work);
  }
  if (tid == 0 && a.cells && cells) atomicAdd(a.cells, (unsigned long long)cells);
  if (tid == 0 && a.skipped && nskip) atomicAdd(a.skipped, (unsigned long long)nskip);
}

template <int G, int P>
int launch_gp(const VerifyArgs& a, uint64_t PW, uint32_t GW, unsigned long long* next, cudaStream_t s) {
  int dev = 0, sms = kNumSMsHint, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, verify_wave_kernel<G, P>, 128, 0);
  if (per_sm < 1) per_sm = 1;
  uint64_t need = (a.m * G + 127) / 128;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (need < grid) grid = need;
  verify_wave_kernel<G, P><<<(unsigned)(grid ? grid : 1), 128, 0, s>>>(a, PW, GW, next);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

template <int G>
int launch_g(const VerifyArgs& a, uint64_t PW, uint32_t GW, unsigned long long* next, cudaStream_t s) {
  if (a.bits <= 2) return launch_gp<G, 2>(a, PW, GW, next, s);
  if (a.bits <= 5) return launch_gp<G, 5>(a, PW, GW, next, s);
  return launch_gp<G, 8>(a, PW, GW, next, s);
}

template <int V, int P>
int launch_vp(const VerifyArgs& a, uint64_t PW, uint32_t GW, unsigned long long* next, cudaStream_t s) {
  int dev = 0, sms = kNumSMsHint, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, verify_cta_kernel<V, P>, 32 * V, 0);
  if (per_sm < 1) per_sm = 1;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (a.m < grid) grid = a.m;
  verify_cta_kernel<V, P><<<(unsigned)(grid ? grid : 1), 32 * V, 0, s>>>(a, PW, GW, next);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

template <int V>
int launch_v(const VerifyArgs& a, uint64_t PW, uint32_t GW, unsigned long long* next, cudaStream_t s) {
  if (a.bits <= 2) return launch_vp<V, 2>(a, PW, GW, next, s);
  if (a.bits <= 5) return launch_vp<V, 5>(a, PW, GW, next, s);
  return launch_vp<V, 8>(a, PW, GW, next, s);
}

template <int W, int P>
int launch_wp(const VerifyArgs& a, uint64_t PW, uint32_t GW, unsigned long long* next, cudaStream_t s) {
  int dev = 0, sms = kNumSMsHint, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = kDigitTables<P> ? digit_smem_bytes<W, P>() : 0;
  if (kDigitTables<P>) {
    if (!a.codes) return MJ_ERR_ARG;
    MJ_CUDA_TRY(cudaFuncSetAttribute(verify_diag_kernel<W, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, verify_diag_kernel<W, P>, 128, smem);
  // at least ~3 pairs per lane, so that the shared queue evens out the early
  // exits (a warp lasts as long as its slowest lane), but at least 3 blocks
  // per SM to hide the recurrence's latency
  const uint64_t per_sm_pairs = (a.m + 3ull * 128 * sms - 1) / (3ull * 128 * sms);
  per_sm = (int)std::min<uint64_t>((uint64_t)per_sm, std::max<uint64_t>(3, per_sm_pairs));
  if (per_sm < 1) per_sm = 1;
  uint64_t need = (a.m + 127) / 128;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (need < grid) grid = need;
  verify_diag_kernel<W, P><<<(unsigned)(grid ? grid : 1), 128, smem, s>>>(a, PW, GW, next);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

template <int W>
int launch_w(const VerifyArgs& a, uint64_t PW, uint32_t GW, unsigned long long* next, cudaStream_t s) {
  // digit tables read B's rank codes; without them (raw byte planes) every
  // plane is XNORed
  if (!a.codes) return launch_wp<W, 8>(a, PW, GW, next, s);
  if (a.bits <= 2) return launch_wp<W, 2>(a, PW, GW, next, s);
  if (a.bits <= 5) return launch_wp<W, 5>(a, PW, GW, next, s);
  if (a.bits == 7) return launch_wp<W, 7>(a, PW, GW, next, s);   // text (65-128 symbols)
  return launch_wp<W, 8>(a, PW, GW, next, s);
}

}  // namespace

int launch_build_planes(const uint8_t* bytes, uint64_t nbytes, const RankTable& rt, uint32_t bits,
                        uint32_t* planes, uint64_t plane_words, uint32_t guard_words, uint8_t* codes,
                        cudaStream_t s) {
  if (bits > (uint32_t)kMaxBits) return MJ_ERR_UNSUPPORTED;
  uint64_t blocks = (plane_words + 255) / 256;
  uint64_t cap = (uint64_t)kNumSMsHint * 32;
  build_planes_kernel<<<(unsigned)(blocks > cap ? cap : blocks), 256, 0, s>>>(bytes, nbytes, rt, bits, planes,
                                                                              plane_words, guard_words, codes);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int verify_words_for(uint32_t kmax) {
  // widest band: d0 + 2 floor((k - d0) / 2) + 1 <= k + 1 bits
  return (int)((kmax + 1 + 31) / 32);
}

int wave_lanes_for(uint32_t kmax) {
  // blocks of one pair active at one step: floor((w + 30) / 33) + 1, w <= kmax + 1 (>= 64)
  uint32_t w = kmax + 1 < 64 ? 64 : kmax + 1;
  uint32_t cnt = (w + 30) / 33 + 1;
  uint32_t g = 2;
  while (g < cnt) g <<= 1;
  return (int)g;
}

int cta_lanes_for(uint32_t kmax) {
  // a lane's blocks b and b + G are 2G steps apart in the CTA schedule, so
  // G lanes hold bands with 34 G >= 32 + (dhi - dlo), dhi - dlo <= max(kmax, 63)
  const uint32_t w = kmax + 1 < 64 ? 64 : kmax + 1;
  const uint32_t need = (31 + w + 33) / 34;
  uint32_t g = 64;
  while (g < need) g <<= 1;
  return (int)g;
}

int fewest_lanes_for(uint32_t kmax) {
  const int g = wave_lanes_for(kmax);
  return g <= 32 ? g : cta_lanes_for(kmax);
}

int launch_verify(const VerifyArgs& a, uint64_t PW, uint32_t GW, uint32_t kmax, unsigned long long* next,
                  cudaStream_t s, int kernel, int lanes) {
  if (a.m == 0) return MJ_OK;
  const int W = verify_words_for(kmax);
  if (kernel == MJ_VERIFY_KERNEL_AUTO) kernel = W <= 8 ? MJ_VERIFY_KERNEL_DIAGONAL : MJ_VERIFY_KERNEL_WAVEFRONT;
  if (kernel == MJ_VERIFY_KERNEL_WAVEFRONT && (lanes > 32 || (lanes <= 0 && wave_lanes_for(kmax) > 32))) {
    // one CTA of several warps per pair
    const int G = lanes > 0 ? lanes : cta_lanes_for(kmax);
    if (G < cta_lanes_for(kmax) || G > kMaxCtaLanes || (G & (G - 1))) return MJ_ERR_UNSUPPORTED;
    MJ_CUDA_TRY(cudaMemsetAsync(next, 0, sizeof(unsigned long long), s));
    switch (G / 32) {
      case 2: return launch_v<2>(a, PW, GW, next, s);
      case 4: return launch_v<4>(a, PW, GW, next, s);
      case 8: return launch_v<8>(a, PW, GW, next, s);
      case 16: return launch_v<16>(a, PW, GW, next, s);
      case 32: return launch_v<32>(a, PW, GW, next, s);
      default: return MJ_ERR_UNSUPPORTED;
    }
  }
  MJ_CUDA_TRY(cudaMemsetAsync(next, 0, sizeof(unsigned long long), s));
  if (kernel == MJ_VERIFY_KERNEL_WAVEFRONT) {
    const int need = wave_lanes_for(kmax);
    int G = lanes > 0 ? lanes : need;
    if (G < need || G > 32 || (G & (G - 1))) return MJ_ERR_UNSUPPORTED;
    switch (G) {
      case 2: return launch_g<2>(a, PW, GW, next, s);
      case 4: return launch_g<4>(a, PW, GW, next, s);
      case 8: return launch_g<8>(a, PW, GW, next, s);
      case 16: return launch_g<16>(a, PW, GW, next, s);
      case 32: return launch_g<32>(a, PW, GW, next, s);
      default: return MJ_ERR_UNSUPPORTED;
    }
  }
  if (kernel != MJ_VERIFY_KERNEL_DIAGONAL) return MJ_ERR_ARG;
  switch (W) {
    case 1: return launch_w<1>(a, PW, GW, next, s);
    case 2: return launch_w<2>(a, PW, GW, next, s);
    case 3: return launch_w<3>(a, PW, GW, next, s);
    case 4: return launch_w<4>(a, PW, GW, next, s);
    case 5: return launch_w<5>(a, PW, GW, next, s);
    case 6: return launch_w<6>(a, PW, GW, next, s);
    case 7: return launch_w<7>(a, PW, GW, next, s);
    case 8: return launch_w<8>(a, PW, GW, next, s);
    default: break;
  }
  if (W <= 16) return launch_wp<16, 8>(a, PW, GW, next, s);
  if (W <= 32) return launch_wp<32, 8>(a, PW, GW, next, s);
  return MJ_ERR_UNSUPPORTED;
}

}  // namespace mj
