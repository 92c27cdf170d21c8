// Device-wide exclusive scans and an LSD radix sort of 64-bit keys with
// optional 32-bit values: the sorting primitives behind grouping the
// partition records (Alg. 3's hash join) and deduplicating candidate pairs
// (the last step of Alg. 3's join).
#include "mj_internal.cuh"

namespace mj {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;                          // per thread
constexpr int kScanTile = kScanThreads * kScanItems;   // 2048 per block

template <class T>
__device__ T block_exclusive_scan(T v, T* s_warp, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T x = v;
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = lane < kScanThreads / 32 ? s_warp[lane] : T(0);
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) s_warp[lane] = w;
  }
  __syncthreads();
  T wprefix = wid ? s_warp[wid - 1] : T(0);
  *total = s_warp[kScanThreads / 32 - 1];
  __syncthreads();
  return wprefix + x - v;
}

// Phase 1: per-block sums.
template <class TI, class TO>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const TI* __restrict__ in, uint64_t n,
                                                                  TO* __restrict__ block_sum) {
  __shared__ TO s_warp[kScanThreads / 32];
  uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  TO sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) sum += (TO)in[base + k];
  TO tot;
  block_exclusive_scan<TO>(sum, s_warp, &tot);
  if (threadIdx.x == 0) block_sum[blockIdx.x] = tot;
}

// Phase 3: block-local exclusive scan plus the block's scanned prefix.
template <class TI, class TO>
__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const TI* __restrict__ in, TO* __restrict__ out,
                                                                uint64_t n, const TO* __restrict__ block_prefix) {
  __shared__ TO s_warp[kScanThreads / 32];
  uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  TO v[kScanItems];
  TO sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? (TO)in[base + k] : TO(0);
    sum += v[k];
  }
  TO tot;
  TO run = block_exclusive_scan<TO>(sum, s_warp, &tot) + (block_prefix ? block_prefix[blockIdx.x] : TO(0));
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
}

uint64_t blocks_for(uint64_t n) { return (n + kScanTile - 1) / kScanTile; }

// temp elements needed by exclusive_scan: 2 per block at every level
size_t scan_temp_elems(uint64_t n) {
  size_t e = 0;
  while (n > kScanTile) {
    uint64_t b = blocks_for(n);
    e += 2 * b;
    n = b;
  }
  return e + 2;
}

// Exclusive scan of `in` (type TI) into `out` (type TO, may alias `in`); the
// total of all inputs goes to the device word total_out if non-null.
// Reduce-then-scan: block sums, a recursive scan of the sums, then a
// block-local scan offset by the scanned sums.
template <class TI, class TO>
int exclusive_scan(const TI* in, TO* out, uint64_t n, TO* temp, TO* total_out, cudaStream_t s) {
  if (n == 0) {
    if (total_out) MJ_CUDA_TRY(cudaMemsetAsync(total_out, 0, sizeof(TO), s));
    return MJ_OK;
  }
  uint64_t b = blocks_for(n);
  if (b == 1) {
    if (total_out) {
      scan_reduce_kernel<TI, TO><<<1, kScanThreads, 0, s>>>(in, n, total_out);
      MJ_KERNEL_DONE();
    }
    scan_down_kernel<TI, TO><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
    MJ_KERNEL_DONE();
    return MJ_OK;
  }
  TO* sums = temp;
  TO* sums_scanned = temp + b;
  scan_reduce_kernel<TI, TO><<<(unsigned)b, kScanThreads, 0, s>>>(in, n, sums);
  MJ_KERNEL_DONE();
  MJ_TRY((exclusive_scan<TO, TO>(sums, sums_scanned, b, temp + 2 * b, total_out, s)));
  scan_down_kernel<TI, TO><<<(unsigned)b, kScanThreads, 0, s>>>(in, out, n, sums_scanned);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

// ---------------------------------------------------------------- radix sort
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys per tile

__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint64_t* __restrict__ keys, uint64_t n,
                                                                  int shift, uint32_t num_tiles,
                                                                  uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_hist[256];
  s_hist[threadIdx.x] = 0;
  __syncthreads();
  uint64_t base = (uint64_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int k = 0; k < kSortItems; ++k) {
    uint64_t idx = base + (uint64_t)k * kSortThreads + threadIdx.x;
    if (idx < n) atomicAdd(&s_hist[(uint32_t)(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(uint64_t)threadIdx.x * num_tiles + blockIdx.x] = s_hist[threadIdx.x];
}

// Stable scatter of one tile.  Warp w owns items [w*512, w*512+512) of the
// tile, taken in 16 rounds of 32 consecutive items; ranks among equal digits
// come from __match_any_sync within a round plus running per-warp counters.
// The tile is first placed in digit order in shared memory, then written out
// item by item in that order: items of one digit go to consecutive global
// addresses, so a warp's stores form a few contiguous runs.
constexpr size_t kScatterSmem = (size_t)kSortTile * (sizeof(uint64_t) + sizeof(uint32_t));
constexpr int kScatThreads = 512;                       // threads of the scatter kernel
constexpr int kScatItems = kSortTile / kScatThreads;    // items per thread
constexpr int kScatWarps = kScatThreads / 32;

__global__ void __launch_bounds__(kScatThreads) radix_scatter_kernel(
    const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, uint64_t n, int shift,
    uint32_t num_tiles, const uint32_t* __restrict__ offs, uint64_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t* s_keys = reinterpret_cast<uint64_t*>(smem);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(smem + (size_t)kSortTile * sizeof(uint64_t));
  __shared__ uint32_t s_cnt[kScatWarps][256];
  __shared__ uint32_t s_start[256];   // first local position of each digit
  __shared__ uint32_t s_goff[256];    // global position of each digit's first item
  __shared__ uint32_t s_wsum[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kScatWarps * 256; d += kScatThreads) (&s_cnt[0][0])[d] = 0;
  if (threadIdx.x < 256) s_goff[threadIdx.x] = offs[(uint64_t)threadIdx.x * num_tiles + blockIdx.x];
  __syncthreads();
  const uint64_t tile0 = (uint64_t)blockIdx.x * kSortTile;
  const uint64_t base = tile0 + (uint64_t)wid * (kSortTile / kScatWarps);
  const uint32_t valid = (uint32_t)min((uint64_t)kSortTile, n - tile0);
  uint64_t k_[kScatItems];
  uint32_t rank_[kScatItems];
  const uint32_t lt = (1u << lane) - 1;
#pragma unroll
  for (int r = 0; r < kScatItems; ++r) {
    const uint64_t idx = base + (uint64_t)r * 32 + lane;
    k_[r] = idx < n ? keys[idx] : ~0ull;
  }
#pragma unroll
  for (int r = 0; r < kScatItems; ++r) {
    // invalid items sit at the end of the last tile: digit 255 after every
    // valid item, so they take the last local positions
    const uint32_t d = (uint32_t)(k_[r] >> shift) & 255u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = __popc(peers & lt);
    const uint32_t cnt = s_cnt[wid][d];
    rank_[r] = cnt + before;
    __syncwarp();
    if (before == 0) s_cnt[wid][d] = cnt + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over warps; the digit's tile total, then an
  // exclusive scan over digits (threads 0..255, warps 0..7) gives its first
  // local position
  uint32_t run = 0, x = 0;
  if (threadIdx.x < 256) {
    const uint32_t d = threadIdx.x;
    for (int w = 0; w < kScatWarps; ++w) {
      const uint32_t c = s_cnt[w][d];
      s_cnt[w][d] = run;
      run += c;
    }
    x = run;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[wid] = x;
  }
  __syncthreads();
  if (threadIdx.x < 256) {
    uint32_t pre = 0;
    for (int w = 0; w < wid; ++w) pre += s_wsum[w];
    s_start[threadIdx.x] = pre + x - run;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kScatItems; ++r) {
    const uint32_t d = (uint32_t)(k_[r] >> shift) & 255u;
    const uint32_t pos = s_start[d] + s_cnt[wid][d] + rank_[r];
    s_keys[pos] = k_[r];
    if (vals) {
      const uint64_t idx = base + (uint64_t)r * 32 + lane;
      s_vals[pos] = idx < n ? vals[idx] : 0u;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kScatItems; ++r) {
    const uint32_t i = (uint32_t)r * kScatThreads + threadIdx.x;
    if (i < valid) {
      const uint64_t key = s_keys[i];
      const uint32_t d = (uint32_t)(key >> shift) & 255u;
      const uint32_t dst = s_goff[d] + (i - s_start[d]);
      keys_out[dst] = key;
      if (vals) vals_out[dst] = s_vals[i];
    }
  }
}

}  // namespace

size_t scan_temp_bytes(uint64_t n) { return scan_temp_elems(n) * sizeof(uint64_t) + 64; }

int launch_exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, void* temp, uint32_t* total_out,
                              cudaStream_t s) {
  return exclusive_scan<uint32_t, uint32_t>(in, out, n, static_cast<uint32_t*>(temp), total_out, s);
}

int launch_exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, void* temp, uint64_t* total_out,
                              cudaStream_t s) {
  return exclusive_scan<uint64_t, uint64_t>(in, out, n, static_cast<uint64_t*>(temp), total_out, s);
}

int launch_exclusive_scan_u32_to_u64(const uint32_t* in, uint64_t* out, uint64_t n, void* temp,
                                     uint64_t* total_out, cudaStream_t s) {
  return exclusive_scan<uint32_t, uint64_t>(in, out, n, static_cast<uint64_t*>(temp), total_out, s);
}

size_t radix_temp_bytes(uint64_t n) {
  uint64_t tiles = (n + kSortTile - 1) / kSortTile;
  uint64_t h = tiles * 256;
  return 2 * h * sizeof(uint32_t) + scan_temp_bytes(h) + 256;
}

int radix_sort_u64(uint64_t* keys, uint64_t* keys_alt, uint32_t* vals, uint32_t* vals_alt, uint64_t n,
                   int bit_lo, int bit_hi, void* temp, bool* result_in_alt, cudaStream_t s) {
  *result_in_alt = false;
  if (n <= 1 || bit_hi <= bit_lo) return MJ_OK;
  if (n >= (1ull << 32)) return MJ_ERR_UNSUPPORTED;
  const uint32_t tiles = (uint32_t)((n + kSortTile - 1) / kSortTile);
  const uint64_t h = (uint64_t)tiles * 256;
  uint32_t* hist = static_cast<uint32_t*>(temp);
  uint32_t* offs = hist + h;
  void* scan_tmp = offs + h;
  uint64_t* src_k = keys;
  uint64_t* dst_k = keys_alt;
  uint32_t* src_v = vals;
  uint32_t* dst_v = vals_alt;
  bool alt = false;
  MJ_CUDA_TRY(cudaFuncSetAttribute(radix_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kScatterSmem));
  for (int shift = bit_lo; shift < bit_hi; shift += 8) {
    radix_hist_kernel<<<tiles, kSortThreads, 0, s>>>(src_k, n, shift, tiles, hist);
    MJ_KERNEL_DONE();
    MJ_TRY(launch_exclusive_scan_u32(hist, offs, h, scan_tmp, nullptr, s));
    radix_scatter_kernel<<<tiles, kScatThreads, kScatterSmem, s>>>(src_k, src_v, n, shift, tiles, offs, dst_k,
                                                                    dst_v);
    MJ_KERNEL_DONE();
    std::swap(src_k, dst_k);
    std::swap(src_v, dst_v);
    alt = !alt;
  }
  *result_in_alt = alt;
  return MJ_OK;
}

}  // namespace mj
