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
#include "mj_internal.cuh"

namespace mj {
namespace {

constexpr int kMaxBits = 8;

__global__ void build_planes_kernel(const uint8_t* __restrict__ bytes, uint64_t nbytes, RankTable rt, uint32_t bits,
                                    uint32_t* __restrict__ planes, uint64_t plane_words, uint32_t guard_words) {
  __shared__ uint8_t s_rank[256];
  s_rank[threadIdx.x] = rt.r[threadIdx.x];
  __syncthreads();
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < plane_words;
       w += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t acc[kMaxBits] = {0};
    int64_t c0 = ((int64_t)w - (int64_t)guard_words) * 32;
    for (int t = 0; t < 32; ++t) {
      int64_t c = c0 + t;
      if (c < 0 || (uint64_t)c >= nbytes) continue;
      uint32_t r = s_rank[__ldg(bytes + c)];
#pragma unroll
      for (int p = 0; p < kMaxBits; ++p) acc[p] |= ((r >> p) & 1u) << t;
    }
#pragma unroll
    for (int p = 0; p < kMaxBits; ++p)
      if (p < (int)bits) planes[(uint64_t)p * plane_words + w] = acc[p];
  }
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

template <int W>
__device__ uint32_t verify_pair(const VerifyArgs& a, const uint8_t* s_rank, uint64_t PW, uint32_t GW,
                                uint32_t x, uint32_t y, uint32_t k) {
  const int64_t ox = __ldg(a.offsets + x), lx = __ldg(a.offsets + x + 1) - ox;
  const int64_t oy = __ldg(a.offsets + y), ly = __ldg(a.offsets + y + 1) - oy;
  const bool xa = lx >= ly;
  const int64_t oA = xa ? ox : oy, m = xa ? lx : ly;
  const int64_t oB = xa ? oy : ox, n = xa ? ly : lx;
  const int64_t d0 = m - n;
  if (d0 > (int64_t)k) return k + 1;
  if (n == 0) return (uint32_t)d0;
  const int32_t dlo = -(int32_t)(((int64_t)k - d0) >> 1);
  const int32_t t0 = (int32_t)d0 - dlo;                // bit of diagonal d0, < 32W by dispatch
  if (t0 >= 32 * W) {                                  // cannot happen with a correct dispatch
    atomicOr(a.dev_flags, FLAG_BOUNDS);
    return k + 1;
  }

  uint32_t Pv[W], Mv[W], M1[W];
  const int32_t nneg = 1 - dlo;                        // band rows dlo..0 (virtual or row 0)
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const int lo = 32 * w;
    uint32_t neg = nneg >= lo + 32 ? 0xffffffffu : (nneg <= lo ? 0u : ((1u << (nneg - lo)) - 1u));
    Mv[w] = neg;
    Pv[w] = ~neg;
    // bits 1..t0
    int32_t a0 = 1 - lo, a1 = t0 + 1 - lo;             // [a0, a1) within this word
    a0 = a0 < 0 ? 0 : a0;
    a1 = a1 > 32 ? 32 : a1;
    uint32_t hiMask = a1 >= 32 ? 0xffffffffu : (a1 <= 0 ? 0u : ((1u << a1) - 1u));
    uint32_t loMask = a0 >= 32 ? 0xffffffffu : ((1u << a0) - 1u);
    M1[w] = a1 > a0 ? (hiMask & ~loMask) : 0u;
  }
  int64_t score = -dlo;                                // D[dlo][0] = -dlo

  // plane window: bit S = oA + j + dlo - 1 + 32*GW of every plane is row j + dlo
  uint64_t S = (uint64_t)(oA + dlo + 32 * (int64_t)GW);  // for j = 1
  uint64_t wbase = S >> 5;
  uint32_t sh = (uint32_t)(S & 31);
  const int bits = (int)a.bits;
  uint32_t pw[kMaxBits][W + 1];
#pragma unroll
  for (int p = 0; p < kMaxBits; ++p) {
#pragma unroll
    for (int w = 0; w <= W; ++w) pw[p][w] = p < bits ? __ldg(a.planes + (uint64_t)p * PW + wbase + w) : 0u;
  }
  const uint8_t* B = a.bytes + oB;
  uint32_t result = 0;
  bool rejected = false;
  for (int64_t j = 1; j <= n; ++j) {
    if (j > 1) {
      sh = (sh + 1) & 31;
      if (sh == 0) {
        ++wbase;
#pragma unroll
        for (int p = 0; p < kMaxBits; ++p) {
#pragma unroll
          for (int w = 0; w < W; ++w) pw[p][w] = pw[p][w + 1];
          pw[p][W] = p < bits ? __ldg(a.planes + (uint64_t)p * PW + wbase + W) : 0u;
        }
      }
    }
    // equality bits of column j
    const uint32_t c = s_rank[__ldg(B + j - 1)];
    uint32_t EqF[W + 1];
#pragma unroll
    for (int w = 0; w <= W; ++w) EqF[w] = 0xffffffffu;
#pragma unroll
    for (int p = 0; p < kMaxBits; ++p) {
      if (p < bits) {
        const uint32_t cm = ((c >> p) & 1u) ? 0u : 0xffffffffu;
#pragma unroll
        for (int w = 0; w <= W; ++w) EqF[w] &= pw[p][w] ^ cm;
      }
    }
    uint32_t Eq[W];
#pragma unroll
    for (int w = 0; w < W; ++w) Eq[w] = __funnelshift_r(EqF[w], EqF[w + 1], sh);

    // band slides down one row: new bottom row gets a +1 vertical delta
#pragma unroll
    for (int w = 0; w < W - 1; ++w) {
      Pv[w] = __funnelshift_r(Pv[w], Pv[w + 1], 1);
      Mv[w] = __funnelshift_r(Mv[w], Mv[w + 1], 1);
    }
    Pv[W - 1] = (Pv[W - 1] >> 1) | 0x80000000u;
    Mv[W - 1] = Mv[W - 1] >> 1;
    const int sv = (int)(Pv[0] & 1u) - (int)(Mv[0] & 1u);

    uint32_t Xv[W], Ph[W], Mh[W];
    uint32_t carry = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      Xv[w] = Eq[w] | Mv[w];
      const uint64_t sum = (uint64_t)(Eq[w] & Pv[w]) + Pv[w] + carry;
      carry = (uint32_t)(sum >> 32);
      const uint32_t Xh = ((uint32_t)sum ^ Pv[w]) | Eq[w];
      Ph[w] = Mv[w] | ~(Xh | Pv[w]);
      Mh[w] = Pv[w] & Xh;
    }
    score += sv + (int)(Ph[0] & 1u) - (int)(Mh[0] & 1u);
#pragma unroll
    for (int w = W - 1; w > 0; --w) {
      Ph[w] = __funnelshift_l(Ph[w - 1], Ph[w], 1);
      Mh[w] = __funnelshift_l(Mh[w - 1], Mh[w], 1);
    }
    Ph[0] = (Ph[0] << 1) | 1u;
    Mh[0] = Mh[0] << 1;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      Pv[w] = Mh[w] | ~(Xv[w] | Ph[w]);
      Mv[w] = Ph[w] & Xv[w];
    }
    if ((j & 31) == 0 || j == n) {
      int64_t diag = score;
#pragma unroll
      for (int w = 0; w < W; ++w) diag += (int)__popc(Pv[w] & M1[w]) - (int)__popc(Mv[w] & M1[w]);
      if (diag > (int64_t)k) {
        rejected = true;
        break;
      }
      if (j == n) result = (uint32_t)diag;
    }
  }
  return rejected ? k + 1 : result;
}

template <int W>
__global__ void __launch_bounds__(128) verify_diag_kernel(VerifyArgs a, RankTable rt, uint64_t PW, uint32_t GW) {
  __shared__ uint8_t s_rank[256];
  for (int t = threadIdx.x; t < 256; t += blockDim.x) s_rank[t] = rt.r[t];
  __syncthreads();
  uint64_t cells = 0;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.m; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = a.pi[t], y = a.pj[t];
    const uint32_t k = a.pk ? a.pk[t] : a.K;
    if (x >= a.n_strings || y >= a.n_strings) {
      atomicOr(a.dev_flags, FLAG_BOUNDS);
      a.ed[t] = k + 1;
      continue;
    }
    a.ed[t] = verify_pair<W>(a, s_rank, PW, GW, x, y, k);
    if (a.cells) {
      const int64_t lx = __ldg(a.offsets + x + 1) - __ldg(a.offsets + x);
      const int64_t ly = __ldg(a.offsets + y + 1) - __ldg(a.offsets + y);
      cells += band_cells(lx > ly ? lx : ly, lx > ly ? ly : lx, a.K);
    }
  }
  if (a.cells) {
    for (int o = 16; o > 0; o >>= 1) cells += __shfl_down_sync(0xffffffffu, cells, o);
    if ((threadIdx.x & 31) == 0 && cells) atomicAdd(a.cells, (unsigned long long)cells);
  }
}

template <int W>
int launch_w(const VerifyArgs& a, const RankTable& rt, uint64_t PW, uint32_t GW, cudaStream_t s) {
  uint64_t blocks = (a.m + 127) / 128;
  uint64_t cap = (uint64_t)kNumSMsHint * 16;
  unsigned grid = (unsigned)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
  verify_diag_kernel<W><<<grid, 128, 0, s>>>(a, rt, PW, GW);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

}  // namespace

int launch_build_planes(const uint8_t* bytes, uint64_t nbytes, const RankTable& rt, uint32_t bits,
                        uint32_t* planes, uint64_t plane_words, uint32_t guard_words, cudaStream_t s) {
  if (bits > (uint32_t)kMaxBits) return MJ_ERR_UNSUPPORTED;
  uint64_t blocks = (plane_words + 255) / 256;
  uint64_t cap = (uint64_t)kNumSMsHint * 32;
  build_planes_kernel<<<(unsigned)(blocks > cap ? cap : blocks), 256, 0, s>>>(bytes, nbytes, rt, bits, planes,
                                                                              plane_words, guard_words);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int verify_words_for(uint32_t kmax) {
  // widest band: d0 + 2 floor((k - d0) / 2) + 1 <= k + 1 bits
  return (int)((kmax + 1 + 31) / 32);
}

int launch_verify(const VerifyArgs& a, const RankTable& rt, uint64_t PW, uint32_t GW, uint32_t kmax, cudaStream_t s) {
  if (a.m == 0) return MJ_OK;
  int W = verify_words_for(kmax);
  switch (W) {
    case 1: return launch_w<1>(a, rt, PW, GW, s);
    case 2: return launch_w<2>(a, rt, PW, GW, s);
    case 3: return launch_w<3>(a, rt, PW, GW, s);
    case 4: return launch_w<4>(a, rt, PW, GW, s);
    case 5: return launch_w<5>(a, rt, PW, GW, s);
    case 6: return launch_w<6>(a, rt, PW, GW, s);
    case 7: return launch_w<7>(a, rt, PW, GW, s);
    case 8: return launch_w<8>(a, rt, PW, GW, s);
    default: break;
  }
  if (W <= 16) return launch_w<16>(a, rt, PW, GW, s);
  if (W <= 32) return launch_w<32>(a, rt, PW, GW, s);
  return MJ_ERR_UNSUPPORTED;
}

}  // namespace mj
