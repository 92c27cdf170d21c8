// C ABI of the MinJoin library: context, workspace and the host-side
// orchestration of steps a1-a8 (Alg. 1-3 of the MinJoin paper).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <chrono>

#include "mj_internal.cuh"

namespace mj {

static thread_local char g_cuda_err[512];
static unsigned long long g_launches = 0;  // host-side count of kernel launches

void note_launch() { __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED); }
uint64_t launch_count() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

void set_last_cuda_error(cudaError_t e, const char* expr, const char* file, int line) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s (%s:%d)", cudaGetErrorString(e), expr, file, line);
}

// Allocation-failure injection (mj_inject_alloc_failure): the countdown of
// device allocations left before one fails, per host thread; 0 = off.
static thread_local int64_t g_fail_alloc_in = 0;

static bool injected_failure() {
  return g_fail_alloc_in > 0 && --g_fail_alloc_in == 0;
}

int Buf::reserve(size_t need, cudaStream_t s) {
  if (need <= bytes && p) return MJ_OK;
  if (p) {
    // the old buffer may still be read by queued work on `s`
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_last_cuda_error(e, "cudaStreamSynchronize", __FILE__, __LINE__);
      return MJ_ERR_CUDA;
    }
    cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  size_t alloc = need < 256 ? 256 : need + need / 8;
  if (injected_failure()) return MJ_ERR_OOM;
  cudaError_t e = cudaMalloc(&p, alloc);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    return MJ_ERR_OOM;
  }
  bytes = alloc;
  return MJ_OK;
}

int Buf::grow_keep(size_t need, size_t keep, cudaStream_t s) {
  if (need <= bytes && p) return MJ_OK;
  void* old = p;
  const size_t old_bytes = bytes;
  const size_t alloc = need < 256 ? 256 : need + need / 8;
  void* q = nullptr;
  if (injected_failure()) return MJ_ERR_OOM;
  cudaError_t e = cudaMalloc(&q, alloc);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MJ_ERR_OOM;
  }
  if (old) {
    const size_t n = keep < old_bytes ? keep : old_bytes;
    if (n) MJ_CUDA_TRY(cudaMemcpyAsync(q, old, n, cudaMemcpyDeviceToDevice, s));
    // the old buffer may still be read by queued work on `s`
    MJ_CUDA_TRY(cudaStreamSynchronize(s));
    cudaFree(old);
  }
  p = q;
  bytes = alloc;
  return MJ_OK;
}

void Buf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

// ---------------------------------------------------------------- parameter rules
// Sec. 2.2: q = 3 log_|Sigma|(N/T), read as the smallest q >= 1 with
// |Sigma|^q >= (N/T)^3, decided in integers as |Sigma|^q T^3 >= N^3.
static uint32_t q_rule(uint64_t N, uint32_t T, uint32_t sigma) {
  if (sigma <= 1 || T == 0) return 1;
  const unsigned __int128 lhs_t = (unsigned __int128)T * T * T;
  const unsigned __int128 rhs = (unsigned __int128)N * N * N;
  unsigned __int128 pw = 1;
  uint32_t q = 0;
  while (pw * lhs_t < rhs && q < 64) {
    pw *= sigma;
    ++q;
  }
  return q ? q : 1;
}

// Alg. 2's neighbourhood radius, floor division, raised to r_min.
static int32_t radius_rule(int64_t slen, int64_t q, int64_t T, int32_t r_min) {
  int64_t num = slen - q + 1 - T, den = 2 * T + 2;
  int64_t r = num >= 0 ? num / den : -((-num + den - 1) / den);
  return r < r_min ? r_min : (int32_t)r;
}

static uint64_t splitmix(uint64_t x) {  // host-side seed expansion (Steele, Lea, Flood 2014)
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

static int bits_for(uint64_t v) {  // bits needed to hold 0..v
  int b = 1;
  while (b < 64 && (v >> b)) ++b;
  return b;
}

}  // namespace mj

using namespace mj;

constexpr int kCalibrationRuns = 3;   // timed joins per mode in mj_band_calibrate (median)

struct mj_ctx {
  int device = 0;
  int sms = 152;   // streaming multiprocessors of the device
  mj_stats stats{};
  Derived d;
  // pinned host staging for small readbacks
  unsigned long long* h_small = nullptr;
  // workspace
  Buf hist, dev_flags, small;
  Buf bitmap, tile_count, tile_off, scan_tmp, tile_first;
  Buf recs;   // partition records (PRec) in position order
  Buf keys, keys_alt, idx, idx_alt, sort_tmp;
  Buf srec;   // partition records in group order (PRec)
  Buf pair_count, pair_off, pairs, pairs_alt;
  Buf uflags, uoffs, cand_i, cand_j;
  Buf pairbm;  // pair bitmap of the candidate dedup (bit per pair i < j)
  // the bitmap's first pairbm_zero_words words are zero (its writer clears
  // what it reads), valid while the buffer is still at pairbm_zero_at
  uint64_t pairbm_zero_words = 0;
  const void* pairbm_zero_at = nullptr;
  Buf planes, ed;
  Buf out_i, out_j, out_ed;
  Buf out_t;          // indices of the candidates within K, listed by the band-K pass
  bool out_collect = false;
  Buf rank_dev;       // the derived rank codes on the device (256 bytes)
  Buf geo;            // pair geometry at the verification order's positions (uint4)
  Buf strgeo;         // per string {offset, length} for the ordering (uint2)
  bool geo_valid = false;
  // alphabet and longest length fixed by mj_set_alphabet (a sharded join's
  // global values), used by derive instead of the input's own
  bool fixed_alpha = false;
  uint8_t fixed_present[256] = {};
  uint64_t fixed_N = 0;
  Buf in_bytes, in_offsets;  // staging for mj_join_host
  uint64_t n_part = 0, n_cand = 0, n_out = 0;
  // bit-planes written by the partition kernel for the verifier
  mj_verify_config vcfg{MJ_VERIFY_KERNEL_AUTO, 0, 0, 0};
  // autotuned kernel per length bucket
  bool tuned = false;
  uint32_t tuned_kernel[kLenBuckets] = {};
  uint32_t tuned_lanes[kLenBuckets] = {};
  Buf branges;   // bucket counts [32] then ranges [64]
  // CUDA graph of the plain verification stage
  cudaGraphExec_t graph_exec = nullptr;
  uint64_t graph_sig[23] = {};
  uint64_t last_sig[23] = {};
  uint64_t graph_launches = 0;
  // learned first-pass band: parameters P, Adam moments M and V, gradient G, loss
  Buf band;
  bool band_ready = false;
  uint32_t band_margin = 0, band_min_mult = 2;
  bool band_gate_auto = false;   // set band_min_mult from the training data
  // learned mode's calibration (mj_band_calibrate): -1 not calibrated (the
  // network runs), 1 the network runs, 0 learned mode runs the plain path
  int band_enabled = -1;
  int band_step = 0;
  Buf feat_x, mult, run_start, parts, yhat, kband;
  // learned first passes: bucket-sorted order, per-bucket ranges and work
  // counters, and the streams the bucket launches run on concurrently
  Buf lvals, franges, fnext, fcnt, ed_first;
  static constexpr int kAuxStreams = 8;
  cudaStream_t aux[kAuxStreams] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kAuxStreams] = {};
  bool have_features = false;
  bool work_started = false;   // verification counters cleared in this call
  bool planes_ready = false;
  Buf codes;                  // the input's rank codes, one byte per input byte (digit-table verifiers)
  bool codes_ready = false;   // written in this call (with the planes)
  uint64_t planes_pw = 0;
  uint32_t planes_gw = 0;
  bool have_part = false, have_cand = false, have_out = false;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // section timers of mj_join (mj_stats.ms_section)
  static constexpr int kSections = 9;
  cudaEvent_t sec_ev[2 * kSections] = {};
  bool sec_used[kSections] = {};
  bool timing = false;
  // while the verification stage is captured, section events become event
  // nodes of the graph (recorded at every replay); graph_sections: the
  // sections the captured graph records
  bool capturing = false;
  uint32_t graph_sections = 0;
  uint64_t launches_at_start = 0;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

int readback(mj_ctx* c, const void* d_src, size_t bytes, cudaStream_t s) {
  MJ_CUDA_TRY(cudaMemcpyAsync(c->h_small, d_src, bytes, cudaMemcpyDeviceToHost, s));
  MJ_CUDA_TRY(cudaStreamSynchronize(s));
  return MJ_OK;
}

// A section's interval runs from its first start to its last stop in a call.
void record_event(mj_ctx* c, cudaEvent_t e, cudaStream_t s) {
  if (c->capturing) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
}
void tstart(mj_ctx* c, int i, cudaStream_t s) {
  if (c->timing && !c->sec_used[i]) {
    record_event(c, c->sec_ev[2 * i], s);
    c->sec_used[i] = true;
    if (c->capturing) c->graph_sections |= 1u << i;
  }
}
void tstop(mj_ctx* c, int i, cudaStream_t s) {
  if (c->timing) record_event(c, c->sec_ev[2 * i + 1], s);
}
// after a replay of the verification graph: its event nodes timed these
void mark_graph_sections(mj_ctx* c) {
  if (!c->timing) return;
  for (int i = 0; i < mj_ctx::kSections; ++i)
    if (c->graph_sections & (1u << i)) c->sec_used[i] = true;
}

void begin_call(mj_ctx* c, bool timing) {
  c->stats = mj_stats{};
  c->geo_valid = false;
  c->planes_ready = false;
  c->codes_ready = false;
  c->work_started = false;
  c->timing = timing;
  for (bool& u : c->sec_used) u = false;
  c->launches_at_start = launch_count();
}

int check_inputs(const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n, const mj_params* p) {
  if (!d_offsets || !p) return MJ_ERR_ARG;
  if (n > 0 && !d_bytes) {
    // an all-empty input may pass a null byte pointer; it is checked later
  }
  if (p->K > (1u << 20) || p->r_min < 0) return MJ_ERR_ARG;
  if (p->repeats < 1 || p->repeats > 64) return MJ_ERR_ARG;
  return MJ_OK;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    return 0.f;
  }
  return ms;
}

// a1: alphabet, longest length, q, T, radius bound.
int derive(mj_ctx* c, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n, const mj_params* p,
           cudaStream_t s) {
  MJ_TRY(c->hist.reserve(256 * sizeof(unsigned long long) + 64, s));
  unsigned long long* hist = c->hist.as<unsigned long long>();
  unsigned long long* maxlen = hist + 256;
  MJ_TRY(readback(c, d_offsets + n, sizeof(int64_t), s));
  const uint64_t nbytes = c->h_small[0];
  if (nbytes >= (1ull << 32)) return MJ_ERR_UNSUPPORTED;
  if (nbytes > 0 && !d_bytes) return MJ_ERR_ARG;
  MJ_TRY(launch_byte_histogram(d_bytes, nbytes, hist, s));
  MJ_TRY(launch_max_length(d_offsets, n, maxlen, s));
  MJ_TRY(readback(c, hist, 257 * sizeof(unsigned long long), s));
  Derived& d = c->d;
  d = Derived();
  uint32_t sigma = 0;
  if (c->fixed_alpha) {   // a global alphabet and length: every local byte and length must lie within them
    for (int b = 0; b < 256; ++b)
      if (c->h_small[b] && !c->fixed_present[b]) return MJ_ERR_ARG;
    if (c->h_small[256] > c->fixed_N) return MJ_ERR_ARG;
    for (int b = 0; b < 256; ++b)
      if (c->fixed_present[b]) d.rank[b] = (uint8_t)sigma++;
  } else {
    for (int b = 0; b < 256; ++b) {
      if (c->h_small[b]) d.rank[b] = (uint8_t)sigma++;
    }
  }
  d.sigma = sigma;
  d.bits = 1;
  while ((1u << d.bits) < sigma) ++d.bits;
  d.N = c->fixed_alpha ? c->fixed_N : c->h_small[256];
  d.K = p->K;
  d.T = p->T ? p->T : p->K;
  if (d.T == 0) d.T = 1;
  d.q = p->q ? p->q : q_rule(d.N, d.T, sigma);
  d.q = std::max<uint32_t>(1, std::min<uint32_t>(d.q, 64 / d.bits));
  d.r_min = p->r_min;
  d.r_max = radius_rule((int64_t)d.N, d.q, d.T, d.r_min);
  d.seed = p->seed;
  d.repeats = p->repeats;
  c->stats.n_strings = n;
  c->stats.n_bytes = nbytes;
  // the rank codes on the device (the text verifier reads B's bytes through
  // them), staged through pinned memory
  MJ_TRY(c->rank_dev.reserve(256, s));
  uint8_t* stage = reinterpret_cast<uint8_t*>(c->h_small) + 3072;
  MJ_CUDA_TRY(cudaStreamSynchronize(s));   // an earlier copy may still read the staging area
  memcpy(stage, d.rank, 256);
  MJ_CUDA_TRY(cudaMemcpyAsync(c->rank_dev.p, stage, 256, cudaMemcpyHostToDevice, s));
  return MJ_OK;
}

uint64_t key_base_for(uint64_t seed) {
  const uint64_t M61 = (1ull << 61) - 1;
  return 257 + splitmix(seed ^ 0x6b6579626173650aull) % (M61 - 1024);
}

// a2-a4 (after derive): partition records in c->recs (n_part of them).
// plane_kmax > 0: also write the verifier's bit-planes (guard sized for bands
// up to plane_kmax).
int partition(mj_ctx* c, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n, const uint64_t* d_table,
              uint32_t plane_kmax, cudaStream_t s) {
  const Derived& d = c->d;
  const uint64_t nbytes = c->stats.n_bytes;
  if (d.r_max > 8192) return MJ_ERR_UNSUPPORTED;
  PartitionArgs a;
  a.bytes = d_bytes;
  a.offsets = d_offsets;
  a.n = n;
  a.nbytes = nbytes;
  a.q = d.q;
  a.bits = d.bits;
  a.T = d.T;
  a.r_min = d.r_min;
  a.r_max = d.r_max < 1 ? 1 : d.r_max;   // halo of at least one position
  a.seed32 = (uint32_t)d.seed ^ (uint32_t)(d.seed >> 32);
  a.seed64 = d.seed;
  a.table = d_table;
  memcpy(a.rank, d.rank, 256);
  const uint64_t tiles = partition_num_tiles(nbytes);
  c->n_part = 0;
  if (tiles == 0) return MJ_OK;
  MJ_TRY(c->dev_flags.reserve(64, s));
  MJ_CUDA_TRY(cudaMemsetAsync(c->dev_flags.p, 0, 64, s));
  MJ_TRY(c->bitmap.reserve(tiles * (kPartTile / 32) * sizeof(uint32_t), s));
  MJ_TRY(c->tile_count.reserve(tiles * sizeof(uint32_t), s));
  MJ_TRY(c->tile_first.reserve(tiles * sizeof(uint32_t), s));
  MJ_TRY(c->tile_off.reserve(tiles * sizeof(uint32_t) + 16, s));
  MJ_TRY(c->scan_tmp.reserve(scan_temp_bytes(tiles), s));
  c->planes_ready = false;
  c->codes_ready = false;
  uint32_t* planes = nullptr;
  uint64_t PW = 0;
  uint32_t GW = 0;
  if (plane_kmax > 0) {
    GW = plane_guard_words(plane_kmax);
    PW = tiles * (kPartTile / 32) + 2 * (uint64_t)GW;
    MJ_TRY(c->planes.reserve(PW * d.bits * 4, s));
    planes = c->planes.as<uint32_t>();
    MJ_TRY(c->codes.reserve(tiles * kPartTile + 64, s));   // written by the first repetition's tiles
    // guard words before and after every plane's data are zero
    MJ_CUDA_TRY(cudaMemsetAsync(planes, 0, (size_t)GW * 4, s));
    for (uint32_t p = 0; p < d.bits; ++p) {
      const uint64_t from = (uint64_t)p * PW + GW + tiles * (kPartTile / 32);
      const uint64_t words = (p + 1 < d.bits) ? 2 * (uint64_t)GW : (uint64_t)GW;
      MJ_CUDA_TRY(cudaMemsetAsync(planes + from, 0, words * 4, s));
    }
  }
  // parallel repetition (Sec. 2.2): Pi_k has the seed d.seed + k * 0x9E3779B97F4A7C15;
  // the records of repetition k follow those of repetitions 0 .. k-1
  const uint32_t R = d.repeats;
  if (d_table && R > 1) return MJ_ERR_ARG;
  uint64_t n_total = 0;
  for (uint32_t k = 0; k < R; ++k) {
    const uint64_t seed_k = d.seed + (uint64_t)k * 0x9E3779B97F4A7C15ull;
    a.seed32 = (uint32_t)seed_k ^ (uint32_t)(seed_k >> 32);
    a.seed64 = seed_k;
    tstart(c, 0, s);
    a.codes = (planes && k == 0) ? c->codes.as<uint8_t>() : nullptr;
    MJ_TRY(launch_anchor_flags(a, c->bitmap.as<uint32_t>(), c->tile_count.as<uint32_t>(),
                               c->dev_flags.as<uint32_t>(), k == 0 ? planes : nullptr, PW, GW,
                               c->tile_first.as<uint32_t>(), s));
    tstop(c, 0, s);
    if (planes && k == 0) {
      c->planes_ready = true;
      c->codes_ready = true;
      c->planes_pw = PW;
      c->planes_gw = GW;
    }
    uint32_t* total = c->tile_off.as<uint32_t>() + tiles;
    MJ_TRY(launch_exclusive_scan_u32(c->tile_count.as<uint32_t>(), c->tile_off.as<uint32_t>(), tiles,
                                     c->scan_tmp.p, total, s));
    MJ_CUDA_TRY(cudaMemcpyAsync(c->h_small, total, 4, cudaMemcpyDeviceToHost, s));
    MJ_CUDA_TRY(cudaMemcpyAsync((char*)c->h_small + 8, c->dev_flags.p, 4, cudaMemcpyDeviceToHost, s));
    MJ_CUDA_TRY(cudaStreamSynchronize(s));
    const uint32_t n_anchor = *(uint32_t*)c->h_small;
    c->stats.device_flags |= *(uint32_t*)((char*)c->h_small + 8);
    if (c->stats.device_flags) return MJ_ERR_DEVICE;
    if (n_total + n_anchor >= (1ull << 32)) return MJ_ERR_UNSUPPORTED;   // record indexes are 32-bit
    MJ_TRY(c->recs.grow_keep((n_total + n_anchor + 1) * sizeof(PRec), n_total * sizeof(PRec), s));
    tstart(c, 1, s);
    MJ_TRY(launch_partition_records(a, c->bitmap.as<uint32_t>(), c->tile_off.as<uint32_t>(),
                                    c->tile_first.as<uint32_t>(), key_base_for(d.seed),
                                    c->recs.as<PRec>() + n_total, s));
    tstop(c, 1, s);
    n_total += n_anchor;
  }
  c->n_part = n_total;
  c->stats.n_partitions = n_total;
  return MJ_OK;
}

// a5-a7 (after partition): candidates in c->cand_i/j (sorted, distinct).
int candidates(mj_ctx* c, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n, uint32_t flags,
               cudaStream_t s, bool want_run_start = false) {
  const Derived& d = c->d;
  const uint32_t nr = (uint32_t)c->n_part;
  c->n_cand = 0;
  c->stats.n_raw_pairs = 0;
  c->stats.key_collisions = 0;
  if (nr == 0) return MJ_OK;
  // Group key shape: the hash bits fill whole 8-bit radix passes above the
  // position bucket and the string length, at least 24 and at most 32 (runs
  // only need to separate most (len, key) classes: the pair walk compares
  // len and key itself).  The bucket width W is K, or wider when the
  // position and length bits would leave fewer than 24 hash bits.
  GroupKeyShape g;
  g.slen_bits = bits_for(d.N);
  const int pb_room = std::max(0, 40 - g.slen_bits);
  g.W = std::max<uint32_t>(d.K, 1u);
  if (pb_room == 0) {
    g.pb_bits = 0;
  } else {
    if (bits_for(d.N / g.W) > pb_room) g.W = (uint32_t)std::min<uint64_t>((d.N >> pb_room) + 1, 0xffffffffull);
    g.pb_bits = bits_for(d.N / g.W);
  }
  const int low_bits = g.pb_bits + g.slen_bits;
  const int sort_passes = (24 + low_bits + 7) / 8;
  g.hash_bits = std::min(32, 8 * sort_passes - low_bits);
  MJ_TRY(c->keys.reserve((size_t)nr * 8, s));
  MJ_TRY(c->keys_alt.reserve((size_t)nr * 8, s));
  c->geo_valid = false;   // c->idx is reused by the record sort
  MJ_TRY(c->idx.reserve((size_t)nr * 4, s));
  MJ_TRY(c->idx_alt.reserve((size_t)nr * 4, s));
  MJ_TRY(c->sort_tmp.reserve(radix_temp_bytes(nr), s));
  tstart(c, 2, s);
  MJ_TRY(launch_make_group_keys(c->recs.as<PRec>(), nr, g, c->keys.as<uint64_t>(), c->idx.as<uint32_t>(), s));
  bool alt = false;
  MJ_TRY(radix_sort_u64(c->keys.as<uint64_t>(), c->keys_alt.as<uint64_t>(), c->idx.as<uint32_t>(),
                        c->idx_alt.as<uint32_t>(), nr, 0, g.hash_bits + low_bits, c->sort_tmp.p, &alt, s));
  const uint64_t* skeys = alt ? c->keys_alt.as<uint64_t>() : c->keys.as<uint64_t>();
  const uint32_t* sidx = alt ? c->idx_alt.as<uint32_t>() : c->idx.as<uint32_t>();
  MJ_TRY(c->srec.reserve((size_t)nr * sizeof(PRec), s));
  const PRec* r = c->srec.as<PRec>();
  MJ_TRY(launch_gather_records(sidx, skeys, nr, g, c->recs.as<PRec>(), c->srec.as<PRec>(), s));
  tstop(c, 2, s);
  if (flags & MJ_FLAG_KEY_CHECK) {
    MJ_TRY(c->small.reserve(128, s));
    MJ_CUDA_TRY(cudaMemsetAsync(c->small.p, 0, 8, s));
    MJ_TRY(launch_key_check(r, d_bytes, d_offsets, nr, c->small.as<unsigned long long>(), s));
    MJ_TRY(readback(c, c->small.p, 8, s));
    c->stats.key_collisions = c->h_small[0];
  }
  // Dedup by the pair bitmap when its sweep (clear, count, write: three
  // passes over n^2/16 bytes) costs less than sorting the raw pairs (about
  // 80 bytes of traffic per pair over the radix passes), unless the
  // candidates' multiplicities are wanted (only the sort gives them) or a
  // flag forces one way.  When the bitmap is at most 640 bytes per partition
  // record, the bitmap is taken without counting the raw pairs first (the
  // marking walk counts them itself): had the sort been the better choice,
  // the bitmap's three sweeps (3 x 640 bytes per record at about 6.5 TB/s,
  // 0.3 ns per record) cost no more than the counting walk they replace
  // (0.26-0.35 ns per record measured on protein and text).  Otherwise a
  // counting walk decides.
  const uint64_t bm_bytes = pair_bitmap_words(n) * 4;
  const bool bitmap_ok = !want_run_start && bm_bytes > 0 && !(flags & MJ_FLAG_DEDUP_SORT) &&
                         bm_bytes <= (48ull << 30);
  bool counted = false, use_bitmap = false;
  uint64_t raw = 0;
  if (bitmap_ok && ((flags & MJ_FLAG_DEDUP_BITMAP) || bm_bytes <= (uint64_t)nr * 640)) {
    const int st = c->pairbm.reserve(bm_bytes, s);
    if (st == MJ_OK) use_bitmap = true;
    else if (st != MJ_ERR_OOM || (flags & MJ_FLAG_DEDUP_BITMAP)) return st;   // OOM without the flag: count and decide
  }
  if (!use_bitmap) {
    MJ_TRY(c->pair_count.reserve((size_t)nr * 4, s));
    MJ_TRY(c->pair_off.reserve((size_t)nr * 8 + 16, s));
    MJ_TRY(c->scan_tmp.reserve(scan_temp_bytes(nr), s));
    tstart(c, 3, s);
    MJ_TRY(launch_count_pairs(r, nr, d.K, g, c->pair_count.as<uint32_t>(), s));
    uint64_t* total = c->pair_off.as<uint64_t>() + nr;
    MJ_TRY(launch_exclusive_scan_u32_to_u64(c->pair_count.as<uint32_t>(), c->pair_off.as<uint64_t>(), nr,
                                            c->scan_tmp.p, total, s));
    MJ_TRY(readback(c, total, 8, s));
    tstop(c, 3, s);
    raw = c->h_small[0];
    counted = true;
    c->stats.n_raw_pairs = raw;
    if (raw == 0) return MJ_OK;
    if (raw >= (1ull << 32)) return MJ_ERR_UNSUPPORTED;
    use_bitmap = bitmap_ok && ((flags & MJ_FLAG_DEDUP_BITMAP) || bm_bytes <= raw * 80);
    if (use_bitmap) {
      const int st = c->pairbm.reserve(bm_bytes, s);
      if (st == MJ_ERR_OOM && !(flags & MJ_FLAG_DEDUP_BITMAP)) {
        use_bitmap = false;   // not enough device memory: sort instead
      } else if (st != MJ_OK) {
        return st;
      }
    }
  }
  if (use_bitmap) {
    tstart(c, 4, s);
    MJ_TRY(c->small.reserve(128, s));
    const uint64_t words = pair_bitmap_words(n);
    const bool zero = c->pairbm.p == c->pairbm_zero_at && words <= c->pairbm_zero_words;
    const uint64_t zero_after = zero ? c->pairbm_zero_words : words;
    c->pairbm_zero_words = 0;   // bits are set from here until the writer clears them
    MJ_TRY(launch_mark_pairs(r, nr, d.K, g, n, c->pairbm.as<uint32_t>(), c->small.as<unsigned long long>() + 7, !zero,
                             s));
    MJ_TRY(c->uflags.reserve((size_t)n * 4, s));
    MJ_TRY(c->uoffs.reserve((size_t)n * 4 + 16, s));
    MJ_TRY(c->scan_tmp.reserve(scan_temp_bytes(n), s));
    MJ_TRY(launch_bitmap_rows(c->pairbm.as<uint32_t>(), n, c->uflags.as<uint32_t>(), s));
    uint32_t* ctotal = c->uoffs.as<uint32_t>() + n;
    MJ_TRY(launch_exclusive_scan_u32(c->uflags.as<uint32_t>(), c->uoffs.as<uint32_t>(), n, c->scan_tmp.p, ctotal, s));
    MJ_CUDA_TRY(cudaMemcpyAsync(c->h_small + 1, c->small.as<unsigned long long>() + 7, 8, cudaMemcpyDeviceToHost, s));
    MJ_TRY(readback(c, ctotal, 4, s));
    const uint32_t nc = *(uint32_t*)c->h_small;
    if (counted && c->h_small[1] != raw) return MJ_ERR_DEVICE;   // both walks must see the same pairs
    raw = c->h_small[1];
    c->stats.n_raw_pairs = raw;
    // the row counts' scan is 32-bit: the raw pairs bound the candidates
    if (raw >= (1ull << 32)) return MJ_ERR_UNSUPPORTED;
    // the writer clears the words it reads when few of them hold bits (at
    // most one candidate per eight words): cheaper than clearing all the
    // words before the next marking; denser bitmaps are cleared then
    const bool writer_clears = nc <= words / 8;
    if (nc) {
      MJ_TRY(c->cand_i.reserve((size_t)nc * 4 + 16, s));
      MJ_TRY(c->cand_j.reserve((size_t)nc * 4 + 16, s));
      MJ_TRY(launch_bitmap_write(c->pairbm.as<uint32_t>(), n, c->uoffs.as<uint32_t>(), c->cand_i.as<uint32_t>(),
                                 c->cand_j.as<uint32_t>(), writer_clears, s));
    }
    if (writer_clears) {   // every word read is zero again (none was set when nc = 0)
      c->pairbm_zero_words = zero_after;
      c->pairbm_zero_at = c->pairbm.p;
    }
    tstop(c, 4, s);
    c->n_cand = nc;
    c->stats.n_candidates = nc;
    return MJ_OK;
  }
  MJ_TRY(c->pairs.reserve(raw * 8, s));
  MJ_TRY(c->pairs_alt.reserve(raw * 8, s));
  tstart(c, 4, s);
  const int nb = bits_for(n ? n - 1 : 0);   // pair (i, j) packed as i << nb | j
  MJ_TRY(launch_fill_pairs(r, nr, d.K, g, nb, c->pair_off.as<uint64_t>(), c->pairs.as<uint64_t>(), s));
  MJ_TRY(c->sort_tmp.reserve(radix_temp_bytes(raw), s));
  MJ_TRY(radix_sort_u64(c->pairs.as<uint64_t>(), c->pairs_alt.as<uint64_t>(), nullptr, nullptr, raw, 0, 2 * nb,
                        c->sort_tmp.p, &alt, s));
  const uint64_t* sp = alt ? c->pairs_alt.as<uint64_t>() : c->pairs.as<uint64_t>();
  MJ_TRY(c->uflags.reserve(raw * 4, s));
  MJ_TRY(c->uoffs.reserve(raw * 4 + 16, s));
  MJ_TRY(c->scan_tmp.reserve(scan_temp_bytes(raw), s));
  MJ_TRY(launch_unique_flags(sp, raw, c->uflags.as<uint32_t>(), s));
  uint32_t* utotal = c->uoffs.as<uint32_t>() + raw;
  MJ_TRY(launch_exclusive_scan_u32(c->uflags.as<uint32_t>(), c->uoffs.as<uint32_t>(), raw, c->scan_tmp.p, utotal, s));
  MJ_TRY(readback(c, utotal, 4, s));
  const uint32_t nc = *(uint32_t*)c->h_small;
  MJ_TRY(c->cand_i.reserve((size_t)nc * 4 + 16, s));
  MJ_TRY(c->cand_j.reserve((size_t)nc * 4 + 16, s));
  if (want_run_start) MJ_TRY(c->run_start.reserve((size_t)nc * 4 + 16, s));
  MJ_TRY(launch_compact_pairs(sp, c->uflags.as<uint32_t>(), c->uoffs.as<uint32_t>(), raw, nb,
                              c->cand_i.as<uint32_t>(), c->cand_j.as<uint32_t>(),
                              want_run_start ? c->run_start.as<uint32_t>() : nullptr, s));
  tstop(c, 4, s);
  c->n_cand = nc;
  c->stats.n_candidates = nc;
  return MJ_OK;
}

// a8 on arbitrary pairs (rank codes from c->d).
// Device flags and verification counters cleared for this call (once), on s.
int verify_prep(mj_ctx* c, cudaStream_t s) {
  MJ_TRY(c->dev_flags.reserve(64, s));
  MJ_CUDA_TRY(cudaMemsetAsync(c->dev_flags.p, 0, 64, s));
  MJ_TRY(c->small.reserve(128, s));
  if (!c->work_started) {
    // counters 0-5 and the output count (8) start at zero once per call;
    // 6 and 7 hold values read back before verification starts
    MJ_CUDA_TRY(cudaMemsetAsync(c->small.p, 0, 72, s));
    c->work_started = true;
  }
  return MJ_OK;
}

int verify(mj_ctx* c, const uint8_t* d_bytes, const int64_t* d_offsets, const uint32_t* d_i, const uint32_t* d_j,
           const uint32_t* d_k, uint64_t m, uint32_t K, uint32_t kmax, uint32_t* d_ed, bool count_cells,
           cudaStream_t s, const uint32_t* order = nullptr, const uint32_t* skip_kband = nullptr,
           const uint32_t* range_lo = nullptr, const uint32_t* range_hi = nullptr, int kernel = -1, int lanes = -1,
           unsigned long long* next = nullptr, bool prep = true, const uint32_t* first_ed = nullptr) {
  const Derived& d = c->d;
  if (m == 0) return MJ_OK;
  if (kmax >= (1u << 16)) return MJ_ERR_UNSUPPORTED;
  const uint64_t nbytes = c->stats.n_bytes;
  uint32_t GW = plane_guard_words(kmax);
  uint64_t PW = (nbytes + 31) / 32 + 2 * (uint64_t)GW;
  if (c->planes_ready && c->planes_gw >= GW) {
    GW = c->planes_gw;   // written by the partition kernel of this call
    PW = c->planes_pw;
  } else {
    MJ_TRY(c->planes.reserve(PW * d.bits * 4, s));
    RankTable rt;
    memcpy(rt.r, d.rank, 256);
    MJ_TRY(c->codes.reserve(nbytes + 64, s));
    tstart(c, 5, s);
    MJ_TRY(launch_build_planes(d_bytes, nbytes, rt, d.bits, c->planes.as<uint32_t>(), PW, GW,
                               c->codes.as<uint8_t>(), s));
    tstop(c, 5, s);
    c->codes_ready = true;
  }
  if (prep) MJ_TRY(verify_prep(c, s));
  VerifyArgs a;
  a.planes = c->planes.as<uint32_t>();
  a.bits = d.bits;
  a.bytes = d_bytes;
  a.offsets = d_offsets;
  a.n_strings = (uint32_t)c->stats.n_strings;
  a.pi = d_i;
  a.pj = d_j;
  a.pk = d_k;
  a.order = order;
  a.skip_kband = skip_kband;
  a.first_ed = first_ed;
  a.range_lo = range_lo;
  a.range_hi = range_hi;
  a.skipped = skip_kband ? c->small.as<unsigned long long>() + 4 : nullptr;
  a.K = K;
  a.m = m;
  a.ed = d_ed;
  a.cells = count_cells ? c->small.as<unsigned long long>() : nullptr;
  a.work = c->small.as<unsigned long long>() + 2;
  a.dev_flags = c->dev_flags.as<uint32_t>();
  if (order && order == c->idx.as<uint32_t>() && c->geo_valid) a.pair_geo = c->geo.as<uint4>();
  a.rank_table = c->rank_dev.as<uint8_t>();
  a.codes = c->codes_ready ? c->codes.as<uint8_t>() : nullptr;
  a.nbytes = nbytes;
  if (c->out_collect) {   // the join's band-K pass lists the pairs within K
    a.out_t = c->out_t.as<uint32_t>();
    a.out_count = c->small.as<unsigned long long>() + 8;
  }
  tstart(c, 6, s);
  int kk = kernel >= 0 ? kernel : (int)c->vcfg.kernel;
  int ll = lanes >= 0 ? lanes : (int)c->vcfg.lanes;
  if (kk == MJ_VERIFY_KERNEL_TUNED) {
    kk = MJ_VERIFY_KERNEL_AUTO;
    ll = 0;
  }
  MJ_TRY(launch_verify(a, PW, GW, kmax, next ? next : c->small.as<unsigned long long>() + 1, s, kk, ll));
  tstop(c, 6, s);
  return MJ_OK;
}

// Longest-first order of pairs (d_i, d_j) (a counting sort of the shorter
// lengths into c->idx), with the pairs' floor(log2) length buckets: counts in
// branges words [0, 32), [start, end) ranges in words [32, 96).
constexpr size_t kOrderScratchAt = 128;   // words of branges before the ordering scratch

// The pairs' K-band cells are summed into small word 9 on the way.
int pair_order(mj_ctx* c, const uint32_t* ci, const uint32_t* cj, const int64_t* d_offsets, uint64_t m,
               const uint32_t** order, cudaStream_t s) {
  if (!c->small.p || !c->branges.p || !c->idx.p || !c->geo.p || !c->strgeo.p) return MJ_ERR_STATE;   // order_buffers first
  uint32_t* counts = c->branges.as<uint32_t>();
  tstart(c, 8, s);
  MJ_TRY(launch_length_order(ci, cj, d_offsets, (uint32_t)c->stats.n_strings, m, c->d.K, counts + kOrderScratchAt,
                             c->strgeo.as<uint2>(), c->idx.as<uint32_t>(), c->geo.as<uint4>(), counts,
                             counts + kLenBuckets, c->small.as<unsigned long long>() + 9, s));
  tstop(c, 8, s);
  *order = c->idx.as<uint32_t>();
  c->geo_valid = true;   // c->geo matches the order in c->idx
  return MJ_OK;
}

int order_buffers(mj_ctx* c, uint64_t m, cudaStream_t s) {
  MJ_TRY(c->small.reserve(128, s));   // word 9: the band cells summed by the ordering
  MJ_TRY(c->idx.reserve(m * 4, s));
  MJ_TRY(c->geo.reserve(m * 16, s));
  MJ_TRY(c->strgeo.reserve((size_t)c->stats.n_strings * 8 + 16, s));
  MJ_TRY(c->branges.reserve(4 * (kOrderScratchAt + kOrderScratchWords) + 64, s));
  return MJ_OK;
}

// Band-K verification of pairs (ci, cj) in longest-first order, as the
// context's kernel choice says (TUNED: per length bucket, batched).
int verify_ordered(mj_ctx* c, const uint8_t* d_bytes, const int64_t* d_offsets, const uint32_t* ci,
                   const uint32_t* cj, uint64_t m, uint32_t K, uint32_t* ed, cudaStream_t s) {
  const uint32_t* order;
  MJ_TRY(pair_order(c, ci, cj, d_offsets, m, &order, s));
  if (c->vcfg.kernel != MJ_VERIFY_KERNEL_TUNED || !c->tuned)
    return verify(c, d_bytes, d_offsets, ci, cj, nullptr, m, K, K, ed, false, s, order);
  uint32_t* counts = c->branges.as<uint32_t>();
  uint32_t* ranges = counts + kLenBuckets;
  if (c->vcfg.batching == 1) {
    for (int b = kLenBuckets - 1; b >= 0; --b)
      MJ_TRY(verify(c, d_bytes, d_offsets, ci, cj, nullptr, m, K, K, ed, false, s, order, nullptr, ranges + 2 * b,
                    ranges + 2 * b + 1, (int)c->tuned_kernel[b], (int)c->tuned_lanes[b]));
    return MJ_OK;
  }
  // one launch per run of consecutive buckets (longest first) sharing a kernel
  int b = kLenBuckets - 1;
  while (b >= 0) {
    int e = b;
    while (e - 1 >= 0 && c->tuned_kernel[e - 1] == c->tuned_kernel[b] && c->tuned_lanes[e - 1] == c->tuned_lanes[b]) --e;
    MJ_TRY(verify(c, d_bytes, d_offsets, ci, cj, nullptr, m, K, K, ed, false, s, order, nullptr, ranges + 2 * b,
                  ranges + 2 * e + 1, (int)c->tuned_kernel[b], (int)c->tuned_lanes[b]));
    b = e - 1;
  }
  return MJ_OK;
}

// verify_ordered, captured into a CUDA graph when the context asks for it and
// replayed while its inputs (pointers, sizes, kernel plan) stay the same.  The
// first call with new inputs runs uncaptured (it sizes every buffer), the
// second captures, later ones replay.
int verify_ordered_graph(mj_ctx* c, const uint8_t* d_bytes, const int64_t* d_offsets, const uint32_t* ci,
                         const uint32_t* cj, uint64_t m, uint32_t K, uint32_t* ed, cudaStream_t s) {
  MJ_TRY(order_buffers(c, m, s));
  // capture needs a stream of its own: the legacy and per-thread default
  // streams run the stage uncaptured
  const bool capturable = s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
  if (!c->vcfg.graph || !capturable) return verify_ordered(c, d_bytes, d_offsets, ci, cj, m, K, ed, s);
  uint64_t plan = (c->vcfg.kernel * 131u + c->vcfg.lanes * 7u + c->vcfg.batching) * 2u + (c->timing ? 1u : 0u);
  if (c->tuned) {
    for (int b = 0; b < kLenBuckets; ++b) plan = plan * 1000003u + c->tuned_kernel[b] * 64u + c->tuned_lanes[b];
  }
  // everything the captured launches read as a parameter: buffers, sizes, plan
  const uint64_t sig[23] = {(uint64_t)d_bytes, (uint64_t)d_offsets, (uint64_t)ci, (uint64_t)cj, m, K,
                            (uint64_t)ed, (uint64_t)c->planes.p, c->planes_pw, c->d.bits, plan,
                            (uint64_t)c->small.p, (uint64_t)c->idx.p, (uint64_t)c->branges.p,
                            (uint64_t)c->dev_flags.p, c->out_collect ? (uint64_t)c->out_t.p : 0, (uint64_t)c->geo.p,
                            c->stats.n_bytes, c->stats.n_strings, c->planes_gw,
                            (uint64_t)c->codes.p, (uint64_t)c->strgeo.p,
                            (uint64_t)c->rank_dev.p};
  if (c->graph_exec && memcmp(sig, c->graph_sig, sizeof(sig)) == 0) {
    MJ_CUDA_TRY(cudaGraphLaunch(c->graph_exec, s));
    mark_graph_sections(c);
    c->launches_at_start -= c->graph_launches;   // kernels replayed by the graph
    return MJ_OK;
  }
  if (memcmp(sig, c->last_sig, sizeof(sig)) != 0) {
    memcpy(c->last_sig, sig, sizeof(sig));
    return verify_ordered(c, d_bytes, d_offsets, ci, cj, m, K, ed, s);
  }
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  // the sections inside the stage are timed by event nodes of the graph
  bool used[mj_ctx::kSections];
  memcpy(used, c->sec_used, sizeof(used));
  for (bool& u : c->sec_used) u = false;
  c->graph_sections = 0;
  const uint64_t before = launch_count();
  MJ_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  c->capturing = true;
  const int st = verify_ordered(c, d_bytes, d_offsets, ci, cj, m, K, ed, s);
  c->capturing = false;
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(s, &graph);
  memcpy(c->sec_used, used, sizeof(used));
  if (st != MJ_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  MJ_CUDA_TRY(ce);
  const cudaError_t ie = cudaGraphInstantiate(&c->graph_exec, graph, 0);
  cudaGraphDestroy(graph);
  MJ_CUDA_TRY(ie);
  c->graph_launches = launch_count() - before;
  memcpy(c->graph_sig, sig, sizeof(sig));
  MJ_CUDA_TRY(cudaGraphLaunch(c->graph_exec, s));
  mark_graph_sections(c);
  return MJ_OK;
}

// Verification of all candidates of the last mj_join (a8, and a9 in learned
// mode), then the K-band cell count.  Plain: one pass with band K.  Learned:
// features -> MLP -> first-pass band per pair; first passes grouped by band
// words (narrower than band K's), then band K for every pair not settled.
int verify_stage(mj_ctx* c, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n, const mj_params* p,
                 cudaStream_t s) {
  const uint64_t m = c->n_cand;
  const uint32_t K = p->K;
  const bool learned = p->verify_mode == MJ_VERIFY_LEARNED;
  const bool want_feat = learned || (p->flags & MJ_FLAG_FEATURES);
  const uint32_t* ci = c->cand_i.as<uint32_t>();
  const uint32_t* cj = c->cand_j.as<uint32_t>();
  MJ_TRY(c->ed.reserve(m * 4, s));
  MJ_TRY(c->small.reserve(128, s));
  const bool want_x = (p->flags & MJ_FLAG_FEATURES) != 0;
  if (want_feat) {
    MJ_TRY(c->parts.reserve((size_t)n * 4 + 16, s));
    MJ_TRY(launch_partition_counts(c->recs.as<PRec>(), c->n_part, n, c->parts.as<uint32_t>(), s));
  }
  if (want_x) {
    MJ_TRY(c->mult.reserve(m * 4, s));
    MJ_TRY(c->feat_x.reserve(m * 4 * kBandFeatures, s));
    MJ_TRY(launch_multiplicity(c->run_start.as<uint32_t>(), m, c->stats.n_raw_pairs, c->mult.as<uint32_t>(), s));
    MJ_TRY(launch_band_features(ci, cj, c->mult.as<uint32_t>(), c->parts.as<uint32_t>(), d_offsets, m, K, c->d.T,
                                c->feat_x.as<float>(), s));
  }
  uint32_t* ed = c->ed.as<uint32_t>();
  MJ_TRY(c->out_t.reserve(m * 4, s));
  if (!learned) {
    // longest pairs first, so that the persistent verifier does not end on a
    // tail of long pairs
    c->out_collect = true;
    const int st = verify_ordered_graph(c, d_bytes, d_offsets, ci, cj, m, K, ed, s);
    c->out_collect = false;
    MJ_TRY(st);
  } else {
    if (!c->band_ready) return MJ_ERR_STATE;
    MJ_TRY(order_buffers(c, m, s));
    const uint32_t* order;
    MJ_TRY(pair_order(c, ci, cj, d_offsets, m, &order, s));
    MJ_TRY(c->kband.reserve(m * 4, s));
    MJ_TRY(c->lvals.reserve(m * 4 + 16, s));
    MJ_TRY(c->franges.reserve(8 * (kMaxBandBuckets + 2), s));
    MJ_TRY(c->fnext.reserve(8 * (kMaxBandBuckets + 2), s));
    MJ_TRY(c->fcnt.reserve(8 * (kMaxBandBuckets + 2), s));
    MJ_TRY(launch_band_fused(c->band.as<float>(), ci, cj, c->run_start.as<uint32_t>(), c->stats.n_raw_pairs,
                             c->parts.as<uint32_t>(), d_offsets, m, K, c->d.T, c->band_margin, c->band_min_mult,
                             c->kband.as<uint32_t>(), s));
    // the pairs of each first-pass bucket, listed contiguously
    const uint32_t wK = (K + 1 + 31) / 32;
    const uint32_t nb = wK <= 1 ? 0 : (wK <= 8 ? wK - 1 : 32 - __builtin_clz(wK - 1));
    uint32_t* ranges = c->franges.as<uint32_t>();
    unsigned long long* first_total = c->small.as<unsigned long long>() + 5;
    MJ_TRY(verify_prep(c, s));
    const uint32_t* forder = c->lvals.as<uint32_t>();
    // the first passes run only when they hold enough pairs to keep the
    // verifier's lanes busy (3 blocks of 128 per SM); fewer pairs are
    // latency-bound there (each on one lane) and cost more than they save,
    // so they go straight to band K
    bool first = false;
    if (nb > 0) {
      MJ_TRY(launch_band_buckets(c->kband.as<uint32_t>(), m, K, nb, c->fcnt.as<uint32_t>(), ranges,
                                 c->lvals.as<uint32_t>(), first_total, s));
      MJ_CUDA_TRY(cudaMemsetAsync(c->fnext.p, 0, 8 * (kMaxBandBuckets + 2), s));
      MJ_TRY(readback(c, first_total, 8, s));
      first = (p->flags & MJ_FLAG_FIRST_PASS) || c->h_small[0] >= (uint64_t)c->sms * 384;
    } else {
      MJ_CUDA_TRY(cudaMemsetAsync(first_total, 0, 8, s));
    }
    // first passes: one persistent launch per bucket (band widths up to the
    // bucket's word count), all buckets at once on the context's streams,
    // each reading its range from device memory and writing its own results;
    // then band K on s for every pair they did not settle (a settled pair
    // takes its first-pass result)
    if (first) {
      MJ_TRY(c->ed_first.reserve(m * 4, s));
      MJ_CUDA_TRY(cudaMemsetAsync(c->ed_first.p, 0xff, m * 4, s));
    }
    tstart(c, 6, s);
    if (first) {
      MJ_CUDA_TRY(cudaEventRecord(c->ev_fork, s));
      for (uint32_t b = 1; b <= nb; ++b) {
        const uint32_t whi = wK <= 8 ? b + 1 : std::min(wK, 1u << b);
        cudaStream_t sb = c->aux[(b - 1) % mj_ctx::kAuxStreams];
        if (b <= (uint32_t)mj_ctx::kAuxStreams) MJ_CUDA_TRY(cudaStreamWaitEvent(sb, c->ev_fork, 0));
        MJ_TRY(verify(c, d_bytes, d_offsets, ci, cj, c->kband.as<uint32_t>(), m, K, 32 * (whi - 1) - 1,
                      c->ed_first.as<uint32_t>(), false, sb, forder, nullptr, ranges + 2 * b, ranges + 2 * b + 1,
                      -1, -1, c->fnext.as<unsigned long long>() + b, false));
      }
      for (uint32_t b = 1; first && b <= std::min(nb, (uint32_t)mj_ctx::kAuxStreams); ++b) {
        MJ_CUDA_TRY(cudaEventRecord(c->ev_join[b - 1], c->aux[b - 1]));
        MJ_CUDA_TRY(cudaStreamWaitEvent(s, c->ev_join[b - 1], 0));
      }
    }
    c->out_collect = true;
    const int st = verify(c, d_bytes, d_offsets, ci, cj, nullptr, m, K, K, ed, false, s, order,
                          first ? c->kband.as<uint32_t>() : nullptr, nullptr, nullptr, -1, -1, nullptr, false,
                          first ? c->ed_first.as<uint32_t>() : nullptr);
    c->out_collect = false;
    MJ_TRY(st);
    MJ_TRY(readback(c, c->small.as<unsigned long long>() + 4, 16, s));
    const uint64_t settled = c->h_small[0];
    c->stats.first_pass_settled = settled;
    c->stats.fallback_pairs = first ? c->h_small[1] - settled : 0;
  }
  c->have_features = want_x;
  return MJ_OK;
}

// He-normal initial weights from a seeded host generator (splitmix64 +
// Box-Muller); biases zero.
void band_initial_weights(uint64_t seed, float* w) {
  uint64_t state = seed;
  auto uni = [&]() {
    state += 0x9e3779b97f4a7c15ull;
    uint64_t z = splitmix(state);
    return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  auto normal = [&]() {
    double u1 = uni(), u2 = uni();
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  };
  const int F = kBandFeatures, H = kBandHidden;
  int o = 0;
  for (int i = 0; i < H * F; ++i) w[o++] = (float)(normal() * sqrt(2.0 / F));
  for (int i = 0; i < H; ++i) w[o++] = 0.f;
  for (int i = 0; i < H * H; ++i) w[o++] = (float)(normal() * sqrt(2.0 / H));
  for (int i = 0; i < H; ++i) w[o++] = 0.f;
  for (int i = 0; i < H; ++i) w[o++] = (float)(normal() * sqrt(1.0 / H));
  w[o++] = 0.5f;
}

}  // namespace

extern "C" {

void mj_params_default(mj_params* p, uint32_t K) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->K = K;
  p->T = 0;
  p->q = 0;
  p->r_min = 1;
  p->seed = 0x5EED;
  p->verify_mode = MJ_VERIFY_PLAIN;
  p->flags = 0;
  p->repeats = 1;
}

const char* mj_strerror(int status) {
  switch (status) {
    case MJ_OK: return "ok";
    case MJ_ERR_ARG: return "invalid argument";
    case MJ_ERR_CUDA: return g_cuda_err[0] ? g_cuda_err : "CUDA runtime error";
    case MJ_ERR_OOM: return "device allocation failed";
    case MJ_ERR_DEVICE: return "device-side check failed";
    case MJ_ERR_UNSUPPORTED: return "input outside the supported range";
    case MJ_ERR_TIMEOUT: return "bounded device wait timed out";
    case MJ_ERR_STATE: return "invalid call order";
    default: return "unknown status";
  }
}

int mj_create(mj_ctx** ctx, int device) {
  if (!ctx) return MJ_ERR_ARG;
  *ctx = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MJ_ERR_CUDA;
  }
  DeviceGuard g(device);
  mj_ctx* c = new mj_ctx();
  c->device = device;
  if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || c->sms < 1) {
    cudaGetLastError();
    c->sms = 152;
  }
  if (cudaMallocHost(&c->h_small, 4096) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return MJ_ERR_OOM;
  }
  for (auto& e : c->sec_ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      mj_destroy(c);
      return MJ_ERR_CUDA;
    }
  }
  for (auto& e : c->ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      mj_destroy(c);
      return MJ_ERR_CUDA;
    }
  }
  bool ok = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < mj_ctx::kAuxStreams; ++i) {
    ok = cudaStreamCreateWithFlags(&c->aux[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    mj_destroy(c);
    return MJ_ERR_CUDA;
  }
  *ctx = c;
  return MJ_OK;
}

void mj_destroy(mj_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  Buf* bufs[] = {&c->hist, &c->dev_flags, &c->small, &c->bitmap, &c->tile_count, &c->tile_off, &c->scan_tmp,
                 &c->tile_first,
                 &c->recs, &c->keys, &c->keys_alt, &c->idx, &c->idx_alt, &c->sort_tmp, &c->srec, &c->pair_count, &c->pair_off, &c->pairs, &c->pairs_alt,
                 &c->uflags, &c->uoffs, &c->cand_i, &c->cand_j, &c->pairbm, &c->planes, &c->ed, &c->out_t, &c->geo, &c->strgeo, &c->codes, &c->rank_dev,
                 &c->out_i, &c->out_j, &c->out_ed, &c->in_bytes, &c->in_offsets, &c->branges,
                 &c->band, &c->feat_x, &c->mult, &c->run_start, &c->parts, &c->yhat, &c->kband, &c->lvals,
                 &c->franges, &c->fnext, &c->fcnt, &c->ed_first};
  for (Buf* b : bufs) b->release();
  for (int i = 0; i < mj_ctx::kAuxStreams; ++i) {
    if (c->aux[i]) cudaStreamDestroy(c->aux[i]);
    if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->sec_ev)
    if (e) cudaEventDestroy(e);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->h_small) cudaFreeHost(c->h_small);
  delete c;
}

int mj_set_verify_config(mj_ctx* c, const mj_verify_config* cfg) {
  if (!c || !cfg) return MJ_ERR_ARG;
  if (cfg->kernel > MJ_VERIFY_KERNEL_TUNED || cfg->batching > 1 || cfg->graph > 1) return MJ_ERR_ARG;
  if (cfg->lanes && (cfg->lanes > (uint32_t)kMaxCtaLanes || (cfg->lanes & (cfg->lanes - 1)) || cfg->lanes < 2))
    return MJ_ERR_ARG;
  c->vcfg = *cfg;
  return MJ_OK;
}

int mj_get_stats(const mj_ctx* c, mj_stats* out) {
  if (!c || !out) return MJ_ERR_ARG;
  *out = c->stats;
  return MJ_OK;
}

int mj_derive(mj_ctx* c, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n, const mj_params* p,
              void* stream, mj_derived* out) {
  if (!c || !out) return MJ_ERR_ARG;
  MJ_TRY(check_inputs(d_bytes, d_offsets, n, p));
  DeviceGuard g(c->device);
  begin_call(c, false);
  MJ_TRY(derive(c, d_bytes, d_offsets, n, p, S(stream)));
  const Derived& d = c->d;
  out->sigma = d.sigma;
  out->bits = d.bits;
  out->q = d.q;
  out->T = d.T;
  out->K = d.K;
  out->r_max = d.r_max;
  out->N = d.N;
  memcpy(out->rank, d.rank, 256);
  out->input_max_len = c->h_small[256];   // derive leaves the histogram and longest length here
  for (int b = 0; b < 256; ++b) out->present[b] = c->h_small[b] ? 1 : 0;
  return MJ_OK;
}

int mj_partition(mj_ctx* c, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n, const mj_params* p,
                 const uint64_t* d_table, void* stream, uint64_t* count) {
  if (!c || !count) return MJ_ERR_ARG;
  MJ_TRY(check_inputs(d_bytes, d_offsets, n, p));
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  begin_call(c, false);
  c->have_part = false;
  MJ_TRY(derive(c, d_bytes, d_offsets, n, p, s));
  MJ_TRY(partition(c, d_bytes, d_offsets, n, d_table, 0, s));
  MJ_CUDA_TRY(cudaStreamSynchronize(s));
  c->have_part = true;
  c->stats.n_launches = launch_count() - c->launches_at_start;
  *count = c->n_part;
  return MJ_OK;
}

int mj_partition_copy(mj_ctx* c, uint32_t* d_sid, uint32_t* d_pos, uint32_t* d_len, uint64_t* d_key,
                      void* stream) {
  if (!c) return MJ_ERR_ARG;
  if (!c->have_part) return MJ_ERR_STATE;
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  const size_t n = c->n_part;
  if (!n) return MJ_OK;
  return launch_unpack_records(c->recs.as<PRec>(), n, d_sid, d_pos, d_len, d_key, s);
}

int mj_candidates(mj_ctx* c, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n, const mj_params* p,
                  const uint64_t* d_table, void* stream, uint64_t* count) {
  if (!c || !count) return MJ_ERR_ARG;
  MJ_TRY(check_inputs(d_bytes, d_offsets, n, p));
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  begin_call(c, false);
  c->have_part = c->have_cand = false;
  MJ_TRY(derive(c, d_bytes, d_offsets, n, p, s));
  MJ_TRY(partition(c, d_bytes, d_offsets, n, d_table, 0, s));
  c->have_part = true;
  MJ_TRY(candidates(c, d_bytes, d_offsets, n, p->flags, s));
  MJ_CUDA_TRY(cudaStreamSynchronize(s));
  c->have_cand = true;
  c->stats.n_launches = launch_count() - c->launches_at_start;
  *count = c->n_cand;
  return MJ_OK;
}

int mj_candidates_copy(mj_ctx* c, uint32_t* d_i, uint32_t* d_j, void* stream) {
  if (!c) return MJ_ERR_ARG;
  if (!c->have_cand) return MJ_ERR_STATE;
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  const size_t n = c->n_cand;
  if (!n) return MJ_OK;
  if (d_i) MJ_CUDA_TRY(cudaMemcpyAsync(d_i, c->cand_i.p, n * 4, cudaMemcpyDeviceToDevice, s));
  if (d_j) MJ_CUDA_TRY(cudaMemcpyAsync(d_j, c->cand_j.p, n * 4, cudaMemcpyDeviceToDevice, s));
  return MJ_OK;
}

int mj_set_alphabet(mj_ctx* c, const uint8_t* h_present, uint64_t N) {
  if (!c) return MJ_ERR_ARG;
  if (!h_present) {
    c->fixed_alpha = false;
    return MJ_OK;
  }
  for (int b = 0; b < 256; ++b) c->fixed_present[b] = h_present[b] ? 1 : 0;
  c->fixed_N = N;
  c->fixed_alpha = true;
  return MJ_OK;
}

int mj_candidates_records(mj_ctx* c, const uint32_t* d_sid, const uint32_t* d_pos, const uint32_t* d_len,
                          const uint64_t* d_key, const uint32_t* d_slen, uint64_t n_rec, uint32_t n_strings,
                          const mj_params* p, void* stream, uint64_t* count) {
  if (!c || !p || !count) return MJ_ERR_ARG;
  if (n_rec && (!d_sid || !d_pos || !d_len || !d_key || !d_slen)) return MJ_ERR_ARG;
  if (p->flags & MJ_FLAG_KEY_CHECK) return MJ_ERR_ARG;   // no bytes to check against
  if (p->K > (1u << 20) || n_rec >= (1ull << 32)) return MJ_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  begin_call(c, false);
  c->have_part = c->have_cand = false;
  Derived& d = c->d;
  d = Derived();
  d.K = p->K;
  d.T = p->T ? p->T : p->K;
  d.seed = p->seed;
  c->stats.n_strings = n_strings;
  c->n_part = n_rec;
  c->n_cand = 0;
  if (n_rec) {
    // ids and lengths bound the grouping key and the pair bitmap: check them
    MJ_TRY(c->small.reserve(128, s));
    unsigned int* mx = reinterpret_cast<unsigned int*>(c->small.as<unsigned long long>() + 10);
    MJ_TRY(launch_max_u32(d_sid, n_rec, mx, s));
    MJ_TRY(launch_max_u32(d_slen, n_rec, mx + 2, s));
    MJ_TRY(readback(c, mx, 16, s));
    const uint32_t max_sid = ((uint32_t*)c->h_small)[0], max_slen = ((uint32_t*)c->h_small)[2];
    if (max_sid >= n_strings) return MJ_ERR_ARG;
    d.N = max_slen;
    MJ_TRY(c->recs.reserve(n_rec * sizeof(PRec), s));
    MJ_TRY(launch_pack_records(d_sid, d_pos, d_len, d_key, d_slen, n_rec, c->recs.as<PRec>(), s));
    MJ_TRY(candidates(c, nullptr, nullptr, n_strings, p->flags, s));
  }
  MJ_CUDA_TRY(cudaStreamSynchronize(s));
  c->have_cand = true;
  c->stats.n_launches = launch_count() - c->launches_at_start;
  *count = c->n_cand;
  return MJ_OK;
}

int mj_pairs_unique(mj_ctx* c, const uint32_t* d_i, const uint32_t* d_j, uint64_t m, uint32_t n_strings,
                    void* stream, uint64_t* count) {
  if (!c || !count) return MJ_ERR_ARG;
  if (m && (!d_i || !d_j)) return MJ_ERR_ARG;
  if (m >= (1ull << 32)) return MJ_ERR_UNSUPPORTED;
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  begin_call(c, false);
  c->have_part = c->have_cand = false;
  c->n_cand = 0;
  if (m) {
    MJ_TRY(c->small.reserve(128, s));
    unsigned int* mx = reinterpret_cast<unsigned int*>(c->small.as<unsigned long long>() + 10);
    MJ_TRY(launch_max_u32(d_i, m, mx, s));
    MJ_TRY(launch_max_u32(d_j, m, mx + 2, s));
    MJ_TRY(readback(c, mx, 16, s));
    if (((uint32_t*)c->h_small)[0] >= n_strings || ((uint32_t*)c->h_small)[2] >= n_strings) return MJ_ERR_ARG;
    const int nb = bits_for(n_strings ? n_strings - 1 : 0);
    MJ_TRY(c->pairs.reserve(m * 8, s));
    MJ_TRY(c->pairs_alt.reserve(m * 8, s));
    MJ_TRY(c->sort_tmp.reserve(radix_temp_bytes(m), s));
    MJ_TRY(c->uflags.reserve(m * 4, s));
    MJ_TRY(c->uoffs.reserve(m * 4 + 16, s));
    MJ_TRY(c->scan_tmp.reserve(scan_temp_bytes(m), s));
    MJ_TRY(launch_pack_pairs(d_i, d_j, m, nb, c->pairs.as<uint64_t>(), s));
    bool alt = false;
    MJ_TRY(radix_sort_u64(c->pairs.as<uint64_t>(), c->pairs_alt.as<uint64_t>(), nullptr, nullptr, m, 0, 2 * nb,
                          c->sort_tmp.p, &alt, s));
    const uint64_t* sp = alt ? c->pairs_alt.as<uint64_t>() : c->pairs.as<uint64_t>();
    MJ_TRY(launch_unique_flags(sp, m, c->uflags.as<uint32_t>(), s));
    uint32_t* utotal = c->uoffs.as<uint32_t>() + m;
    MJ_TRY(launch_exclusive_scan_u32(c->uflags.as<uint32_t>(), c->uoffs.as<uint32_t>(), m, c->scan_tmp.p, utotal, s));
    MJ_TRY(readback(c, utotal, 4, s));
    const uint32_t nc = *(uint32_t*)c->h_small;
    MJ_TRY(c->cand_i.reserve((size_t)nc * 4 + 16, s));
    MJ_TRY(c->cand_j.reserve((size_t)nc * 4 + 16, s));
    MJ_TRY(launch_compact_pairs(sp, c->uflags.as<uint32_t>(), c->uoffs.as<uint32_t>(), m, nb,
                                c->cand_i.as<uint32_t>(), c->cand_j.as<uint32_t>(), nullptr, s));
    c->n_cand = nc;
  }
  MJ_CUDA_TRY(cudaStreamSynchronize(s));
  c->stats.n_candidates = c->n_cand;
  c->have_cand = true;
  c->stats.n_launches = launch_count() - c->launches_at_start;
  *count = c->n_cand;
  return MJ_OK;
}

int mj_inject_alloc_failure(int64_t nth) {
  if (nth < 0) return MJ_ERR_ARG;
  g_fail_alloc_in = nth;
  return MJ_OK;
}

int mj_device_flags(mj_ctx* c, void* stream, uint32_t* flags) {
  if (!c || !flags) return MJ_ERR_ARG;
  DeviceGuard g(c->device);
  *flags = 0;
  if (!c->dev_flags.p) return MJ_OK;   // no device work yet
  MJ_TRY(readback(c, c->dev_flags.p, 4, S(stream)));
  *flags = *(uint32_t*)c->h_small;
  c->stats.device_flags |= *flags;
  return MJ_OK;
}

int mj_verify(mj_ctx* c, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n, const uint32_t* d_i,
              const uint32_t* d_j, const uint32_t* d_k, uint64_t m, uint32_t K, void* stream, uint32_t* d_ed) {
  if (!c || !d_offsets) return MJ_ERR_ARG;
  if (m && (!d_i || !d_j || !d_ed)) return MJ_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  mj_params p;
  mj_params_default(&p, K);
  begin_call(c, false);
  MJ_TRY(derive(c, d_bytes, d_offsets, n, &p, s));
  if (!d_k) {
    // one band for every pair: longest first, with the context's kernel plan
    if (m) MJ_TRY(verify_ordered_graph(c, d_bytes, d_offsets, d_i, d_j, m, K, d_ed, s));
  } else {
    // the widest per-pair band sizes the kernel (a device reduction, 4 bytes read back)
    MJ_TRY(c->small.reserve(128, s));
    unsigned int* dmax = reinterpret_cast<unsigned int*>(c->small.as<unsigned long long>() + 6);
    MJ_TRY(launch_max_u32(d_k, m, dmax, s));
    MJ_TRY(readback(c, dmax, 4, s));
    const uint32_t kmax = *(uint32_t*)c->h_small;
    MJ_TRY(verify(c, d_bytes, d_offsets, d_i, d_j, d_k, m, K, kmax, d_ed, true, s));
  }
  c->stats.n_launches = launch_count() - c->launches_at_start;
  return MJ_OK;
}

int mj_autotune_verify(mj_ctx* c, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n, const uint32_t* d_i,
                       const uint32_t* d_j, uint64_t m, uint32_t K, uint32_t sample, void* stream,
                       mj_autotune_report* rep) {
  if (!c || !d_offsets || (m && (!d_i || !d_j))) return MJ_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  mj_params p;
  mj_params_default(&p, K);
  begin_call(c, false);
  MJ_TRY(derive(c, d_bytes, d_offsets, n, &p, s));
  if (rep) memset(rep, 0, sizeof(*rep));
  // candidates: the diagonal kernel when its band fits 8 words, then the
  // wavefront with 1x, 2x, 4x ... the fewest lanes (one warp up to 32 lanes,
  // a CTA of several warps above)
  uint32_t ck[MJ_TUNE_CANDIDATES], cl[MJ_TUNE_CANDIDATES], nc = 0;
  if (verify_words_for(K) <= 8) {
    ck[nc] = MJ_VERIFY_KERNEL_DIAGONAL;
    cl[nc++] = 0;
  }
  if (fewest_lanes_for(K) > kMaxCtaLanes) return MJ_ERR_UNSUPPORTED;
  for (int lanes = fewest_lanes_for(K); lanes <= kMaxCtaLanes && nc < MJ_TUNE_CANDIDATES; lanes *= 2) {
    ck[nc] = MJ_VERIFY_KERNEL_WAVEFRONT;
    cl[nc++] = (uint32_t)lanes;
  }
  if (rep) {
    rep->n_candidates = nc;
    for (uint32_t k = 0; k < nc; ++k) {
      rep->cand_kernel[k] = ck[k];
      rep->cand_lanes[k] = cl[k];
    }
  }
  for (int b = 0; b < kLenBuckets; ++b) {
    c->tuned_kernel[b] = MJ_VERIFY_KERNEL_AUTO;
    c->tuned_lanes[b] = 0;
  }
  c->tuned = true;
  if (!m) return MJ_OK;
  MJ_TRY(order_buffers(c, m, s));
  MJ_TRY(c->ed.reserve(m * 4, s));
  const uint32_t* order;
  MJ_TRY(pair_order(c, d_i, d_j, d_offsets, m, &order, s));
  uint32_t* counts = c->branges.as<uint32_t>();
  uint32_t* ranges = counts + kLenBuckets;
  uint32_t* trial = ranges + 2 * kLenBuckets;   // [lo, hi) of the sample being timed
  uint32_t h[3 * kLenBuckets];
  MJ_CUDA_TRY(cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, s));
  MJ_CUDA_TRY(cudaStreamSynchronize(s));
  const uint32_t smp = sample ? sample : 4096;
  for (int b = 0; b < kLenBuckets; ++b) {
    const uint32_t cnt = h[b];
    if (rep) rep->count[b] = cnt;
    if (!cnt) continue;
    const uint32_t lo = h[kLenBuckets + 2 * b];
    const uint32_t hi = std::min(h[kLenBuckets + 2 * b + 1], lo + smp);
    const uint32_t r[2] = {lo, hi};
    MJ_CUDA_TRY(cudaMemcpyAsync(trial, r, sizeof(r), cudaMemcpyHostToDevice, s));
    float best = 0.f;
    for (uint32_t k = 0; k < nc; ++k) {
      for (int rep_i = 0; rep_i < 2; ++rep_i) {   // the first run warms the caches
        MJ_CUDA_TRY(cudaEventRecord(c->ev[0], s));
        MJ_TRY(verify(c, d_bytes, d_offsets, d_i, d_j, nullptr, m, K, K, c->ed.as<uint32_t>(), false, s, order,
                      nullptr, trial, trial + 1, (int)ck[k], (int)cl[k]));
        MJ_CUDA_TRY(cudaEventRecord(c->ev[1], s));
      }
      MJ_CUDA_TRY(cudaEventSynchronize(c->ev[1]));
      const float ms = elapsed(c->ev[0], c->ev[1]);
      if (rep) rep->ms[b][k] = ms;
      if (k == 0 || ms < best) {
        best = ms;
        c->tuned_kernel[b] = ck[k];
        c->tuned_lanes[b] = cl[k];
      }
    }
    if (rep) {
      rep->kernel[b] = c->tuned_kernel[b];
      rep->lanes[b] = c->tuned_lanes[b];
    }
  }
  c->stats.n_launches = launch_count() - c->launches_at_start;
  return MJ_OK;
}

int mj_join(mj_ctx* c, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n, const mj_params* p,
            void* stream, uint64_t* count) {
  if (!c || !count) return MJ_ERR_ARG;
  MJ_TRY(check_inputs(d_bytes, d_offsets, n, p));
  if (p->verify_mode > MJ_VERIFY_LEARNED) return MJ_ERR_ARG;
  if (p->verify_mode == MJ_VERIFY_LEARNED && !c->band_ready) return MJ_ERR_STATE;
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  // learned mode calibrated as not paying off on this workload runs the plain
  // path (the same output), unless the first passes are forced
  mj_params eff = *p;
  if (eff.verify_mode == MJ_VERIFY_LEARNED && c->band_enabled == 0 && !(eff.flags & MJ_FLAG_FIRST_PASS))
    eff.verify_mode = MJ_VERIFY_PLAIN;
  p = &eff;
  begin_call(c, true);
  c->have_part = c->have_cand = c->have_out = c->have_features = false;
  MJ_CUDA_TRY(cudaEventRecord(c->ev[0], s));
  MJ_TRY(derive(c, d_bytes, d_offsets, n, p, s));
  MJ_CUDA_TRY(cudaEventRecord(c->ev[1], s));
  MJ_TRY(partition(c, d_bytes, d_offsets, n, nullptr, p->K, s));
  c->have_part = true;
  MJ_CUDA_TRY(cudaEventRecord(c->ev[2], s));
  MJ_TRY(candidates(c, d_bytes, d_offsets, n, p->flags, s,
                    p->verify_mode == MJ_VERIFY_LEARNED || (p->flags & MJ_FLAG_FEATURES)));
  c->have_cand = true;
  MJ_CUDA_TRY(cudaEventRecord(c->ev[3], s));
  const uint64_t m = c->n_cand;
  c->n_out = 0;
  if (m) {
    MJ_TRY(verify_stage(c, d_bytes, d_offsets, n, p, s));
    tstart(c, 7, s);
    MJ_CUDA_TRY(cudaMemcpyAsync(c->h_small, c->small.as<unsigned long long>() + 8, 8, cudaMemcpyDeviceToHost, s));
    MJ_CUDA_TRY(cudaMemcpyAsync(c->h_small + 1, c->small.as<unsigned long long>() + 9, 8, cudaMemcpyDeviceToHost, s));
    MJ_CUDA_TRY(cudaMemcpyAsync(c->h_small + 2, c->dev_flags.p, 4, cudaMemcpyDeviceToHost, s));
    MJ_CUDA_TRY(cudaMemcpyAsync(c->h_small + 3, c->small.as<unsigned long long>() + 2, 8, cudaMemcpyDeviceToHost, s));
    MJ_CUDA_TRY(cudaStreamSynchronize(s));
    const uint64_t no = c->h_small[0];
    c->stats.band_cells = c->h_small[1];
    c->stats.device_flags |= *(uint32_t*)(c->h_small + 2);
    c->stats.verify_word_columns = c->h_small[3];
    if (no > m) return MJ_ERR_DEVICE;
    MJ_TRY(c->out_i.reserve((size_t)no * 4 + 16, s));
    MJ_TRY(c->out_j.reserve((size_t)no * 4 + 16, s));
    MJ_TRY(c->out_ed.reserve((size_t)no * 4 + 16, s));
    MJ_TRY(c->keys.reserve((size_t)no * 8 + 16, s));
    MJ_TRY(c->keys_alt.reserve((size_t)no * 8 + 16, s));
    MJ_TRY(c->sort_tmp.reserve(radix_temp_bytes(no), s));
    // sorted candidate indices are (i, j) order
    MJ_TRY(launch_gather_output(c->out_t.as<uint32_t>(), no, m, c->cand_i.as<uint32_t>(), c->cand_j.as<uint32_t>(),
                                c->ed.as<uint32_t>(), c->keys.as<uint64_t>(), c->keys_alt.as<uint64_t>(),
                                c->sort_tmp.p, c->out_i.as<uint32_t>(), c->out_j.as<uint32_t>(),
                                c->out_ed.as<uint32_t>(), s));
    tstop(c, 7, s);
    c->n_out = no;
  }
  MJ_CUDA_TRY(cudaEventRecord(c->ev[4], s));
  MJ_CUDA_TRY(cudaEventSynchronize(c->ev[4]));
  c->stats.n_output = c->n_out;
  c->stats.ms_derive = elapsed(c->ev[0], c->ev[1]);
  c->stats.ms_partition = elapsed(c->ev[1], c->ev[2]);
  c->stats.ms_join_filter = elapsed(c->ev[2], c->ev[3]);
  c->stats.ms_verify = elapsed(c->ev[3], c->ev[4]);
  c->stats.ms_total = elapsed(c->ev[0], c->ev[4]);
  for (int i = 0; i < mj_ctx::kSections; ++i)
    c->stats.ms_section[i] = c->sec_used[i] ? elapsed(c->sec_ev[2 * i], c->sec_ev[2 * i + 1]) : 0.f;
  c->stats.n_launches = launch_count() - c->launches_at_start;
  if (c->stats.device_flags) return MJ_ERR_DEVICE;
  c->have_out = true;
  *count = c->n_out;
  return MJ_OK;
}

int mj_features_copy(mj_ctx* c, float* d_x, uint32_t* d_ed, uint32_t* d_i, uint32_t* d_j, uint64_t* count,
                     void* stream) {
  if (!c) return MJ_ERR_ARG;
  if (!c->have_features) return MJ_ERR_STATE;
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  const size_t m = c->n_cand;
  if (count) *count = m;
  if (!m) return MJ_OK;
  if (d_x) MJ_CUDA_TRY(cudaMemcpyAsync(d_x, c->feat_x.p, m * 4 * kBandFeatures, cudaMemcpyDeviceToDevice, s));
  if (d_ed) MJ_CUDA_TRY(cudaMemcpyAsync(d_ed, c->ed.p, m * 4, cudaMemcpyDeviceToDevice, s));
  if (d_i) MJ_CUDA_TRY(cudaMemcpyAsync(d_i, c->cand_i.p, m * 4, cudaMemcpyDeviceToDevice, s));
  if (d_j) MJ_CUDA_TRY(cudaMemcpyAsync(d_j, c->cand_j.p, m * 4, cudaMemcpyDeviceToDevice, s));
  return MJ_OK;
}

static int band_buffers(mj_ctx* c, cudaStream_t s) {
  return c->band.reserve(sizeof(float) * (4 * (size_t)kBandParams + 8), s);
}

int mj_band_init(mj_ctx* c, uint64_t seed, uint32_t margin, uint32_t min_multiplicity) {
  if (!c) return MJ_ERR_ARG;
  c->band_enabled = -1;   // a new model is not calibrated
  DeviceGuard g(c->device);
  MJ_TRY(band_buffers(c, nullptr));
  std::vector<float> w(kBandParams);
  band_initial_weights(seed, w.data());
  MJ_CUDA_TRY(cudaMemcpy(c->band.p, w.data(), sizeof(float) * kBandParams, cudaMemcpyHostToDevice));
  MJ_CUDA_TRY(cudaMemset(c->band.as<float>() + kBandParams, 0, sizeof(float) * 2 * kBandParams));
  c->band_margin = margin;
  c->band_min_mult = min_multiplicity ? min_multiplicity : 1;
  c->band_gate_auto = min_multiplicity == 0;
  c->band_step = 0;
  c->band_ready = true;
  return MJ_OK;
}

int mj_band_train(mj_ctx* c, const float* d_x, const uint32_t* d_ed, uint64_t m, uint32_t K,
                  const mj_band_train_params* tp, void* stream, float* final_loss) {
  if (!c || !tp || (m && (!d_x || !d_ed))) return MJ_ERR_ARG;
  if (!c->band_ready) return MJ_ERR_STATE;
  if (!m || !tp->steps || !tp->batch) return MJ_ERR_ARG;
  c->band_enabled = -1;   // the model changes: its calibration is stale
  if (tp->tau < 0.f || tp->tau >= 1.f || tp->seed == 0) return MJ_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  begin_call(c, false);
  float* P = c->band.as<float>();
  float* M = P + kBandParams;
  float* V = M + kBandParams;
  float* G = V + kBandParams;
  float* L = G + kBandParams;
  for (uint32_t step = 0; step < tp->steps; ++step) {
    MJ_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(float) * (kBandParams + 1), s));
    MJ_TRY(launch_band_grad(P, d_x, nullptr, d_ed, K, m, tp->batch, tp->seed + (uint64_t)step * tp->batch, tp->tau,
                            G, L, s));
    MJ_TRY(launch_band_adam(P, G, M, V, tp->lr, 0.9f, 0.999f, 1e-8f, ++c->band_step, s));
  }
  float loss = 0.f;
  MJ_CUDA_TRY(cudaMemcpyAsync(&loss, L, sizeof(float), cudaMemcpyDeviceToHost, s));
  MJ_CUDA_TRY(cudaStreamSynchronize(s));
  if (final_loss) *final_loss = loss;
  if (c->band_gate_auto) {
    // gate = 1st percentile of the multiplicity of the samples a narrower
    // first band could settle
    unsigned int* hist = reinterpret_cast<unsigned int*>(G);   // gradient scratch, free after training
    MJ_TRY(launch_gate_hist(d_x, d_ed, m, K, hist, s));
    unsigned int h[256];
    MJ_CUDA_TRY(cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, s));
    MJ_CUDA_TRY(cudaStreamSynchronize(s));
    uint64_t tot = 0;
    for (unsigned int v : h) tot += v;
    uint32_t gate = 1;
    if (tot) {
      uint64_t acc = 0;
      for (int b = 0; b < 256; ++b) {
        acc += h[b];
        if (acc * 100 >= tot) {
          gate = b < 1 ? 1 : (uint32_t)b;
          break;
        }
      }
    }
    c->band_min_mult = gate;
  }
  c->stats.n_launches = launch_count() - c->launches_at_start;
  return MJ_OK;
}

int mj_band_forward(mj_ctx* c, const float* d_x, uint64_t m, void* stream, float* d_yhat) {
  if (!c || (m && (!d_x || !d_yhat))) return MJ_ERR_ARG;
  if (!c->band_ready) return MJ_ERR_STATE;
  DeviceGuard g(c->device);
  return launch_band_forward(c->band.as<float>(), d_x, m, nullptr, 0, d_yhat, S(stream));
}

int mj_band_grad(mj_ctx* c, const float* d_x, const float* d_y, uint64_t m, float tau, void* stream, float* d_grad,
                 float* loss) {
  if (!c || !d_grad || (m && (!d_x || !d_y))) return MJ_ERR_ARG;
  if (!c->band_ready) return MJ_ERR_STATE;
  if (tau < 0.f || tau >= 1.f || !m) return MJ_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  float* L = c->band.as<float>() + 4 * kBandParams;
  MJ_CUDA_TRY(cudaMemsetAsync(d_grad, 0, sizeof(float) * kBandParams, s));
  MJ_CUDA_TRY(cudaMemsetAsync(L, 0, sizeof(float), s));
  MJ_TRY(launch_band_grad(c->band.as<float>(), d_x, d_y, nullptr, 0, m, m, 0, tau, d_grad, L, s));
  float l = 0.f;
  MJ_CUDA_TRY(cudaMemcpyAsync(&l, L, sizeof(float), cudaMemcpyDeviceToHost, s));
  MJ_CUDA_TRY(cudaStreamSynchronize(s));
  if (loss) *loss = l;
  return MJ_OK;
}

int mj_band_get_weights(const mj_ctx* c, float* h_w, uint64_t count) {
  if (!c || !h_w || count != (uint64_t)kBandParams) return MJ_ERR_ARG;
  if (!c->band_ready) return MJ_ERR_STATE;
  DeviceGuard g(c->device);
  MJ_CUDA_TRY(cudaMemcpy(h_w, c->band.p, sizeof(float) * kBandParams, cudaMemcpyDeviceToHost));
  return MJ_OK;
}

int mj_band_set_weights(mj_ctx* c, const float* h_w, uint64_t count) {
  if (!c || !h_w || count != (uint64_t)kBandParams) return MJ_ERR_ARG;
  DeviceGuard g(c->device);
  MJ_TRY(band_buffers(c, nullptr));
  c->band_enabled = -1;
  MJ_CUDA_TRY(cudaMemcpy(c->band.p, h_w, sizeof(float) * kBandParams, cudaMemcpyHostToDevice));
  if (!c->band_ready) {
    MJ_CUDA_TRY(cudaMemset(c->band.as<float>() + kBandParams, 0, sizeof(float) * 2 * kBandParams));
    c->band_step = 0;
  }
  c->band_ready = true;
  return MJ_OK;
}

int mj_band_save(const mj_ctx* c, const char* path) {
  if (!c || !path) return MJ_ERR_ARG;
  if (!c->band_ready) return MJ_ERR_STATE;
  std::vector<float> w(kBandParams);
  MJ_TRY(mj_band_get_weights(c, w.data(), kBandParams));
  FILE* f = fopen(path, "wb");
  if (!f) return MJ_ERR_ARG;
  const uint32_t hdr[4] = {1u, (uint32_t)kBandParams, c->band_margin, c->band_min_mult};
  bool ok = fwrite("MJBAND01", 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
            fwrite(w.data(), sizeof(float), w.size(), f) == w.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? MJ_OK : MJ_ERR_ARG;
}

int mj_band_load(mj_ctx* c, const char* path) {
  if (!c || !path) return MJ_ERR_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return MJ_ERR_ARG;
  c->band_enabled = -1;
  char magic[8];
  uint32_t hdr[4];
  std::vector<float> w(kBandParams);
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "MJBAND01", 8) == 0 && fread(hdr, sizeof(hdr), 1, f) == 1 &&
            hdr[0] == 1u && hdr[1] == (uint32_t)kBandParams && fread(w.data(), sizeof(float), w.size(), f) == w.size();
  fclose(f);
  if (!ok) return MJ_ERR_ARG;
  MJ_TRY(mj_band_set_weights(c, w.data(), kBandParams));
  c->band_margin = hdr[2];
  c->band_min_mult = hdr[3];
  return MJ_OK;
}

int mj_band_calibrate(mj_ctx* c, const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n, const mj_params* p,
                      void* stream, mj_band_calibration* out) {
  if (!c || !p) return MJ_ERR_ARG;
  if (!c->band_ready) return MJ_ERR_STATE;
  mj_band_calibration r{};
  mj_params plain = *p, learned = *p;
  plain.verify_mode = MJ_VERIFY_PLAIN;
  learned.verify_mode = MJ_VERIFY_LEARNED;
  plain.flags &= ~(uint32_t)(MJ_FLAG_FEATURES | MJ_FLAG_KEY_CHECK);
  learned.flags &= ~(uint32_t)(MJ_FLAG_FEATURES | MJ_FLAG_KEY_CHECK);
  c->band_enabled = 1;   // the learned runs below use the network
  float t[2][kCalibrationRuns];
  uint64_t count = 0;
  for (int mode = 0; mode < 2; ++mode) {
    const mj_params* q = mode == 0 ? &plain : &learned;
    MJ_TRY(mj_join(c, d_bytes, d_offsets, n, q, stream, &count));   // warm-up: sizes the buffers
    for (int k = 0; k < kCalibrationRuns; ++k) {
      const auto t0 = std::chrono::steady_clock::now();
      MJ_TRY(mj_join(c, d_bytes, d_offsets, n, q, stream, &count));   // returns after its stream is done
      t[mode][k] = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (mode == 0) {
      r.plain_word_columns = c->stats.verify_word_columns;
    } else {
      r.learned_word_columns = c->stats.verify_word_columns;
      r.first_pass_settled = c->stats.first_pass_settled;
    }
  }
  std::sort(t[0], t[0] + kCalibrationRuns);
  std::sort(t[1], t[1] + kCalibrationRuns);
  r.plain_ms = t[0][kCalibrationRuns / 2];
  r.learned_ms = t[1][kCalibrationRuns / 2];
  r.enabled = r.learned_ms < r.plain_ms ? 1u : 0u;
  c->band_enabled = (int)r.enabled;
  if (out) *out = r;
  return MJ_OK;
}

int mj_result_copy(mj_ctx* c, uint32_t* d_i, uint32_t* d_j, uint32_t* d_ed, void* stream) {
  if (!c) return MJ_ERR_ARG;
  if (!c->have_out) return MJ_ERR_STATE;
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  const size_t n = c->n_out;
  if (!n) return MJ_OK;
  if (d_i) MJ_CUDA_TRY(cudaMemcpyAsync(d_i, c->out_i.p, n * 4, cudaMemcpyDeviceToDevice, s));
  if (d_j) MJ_CUDA_TRY(cudaMemcpyAsync(d_j, c->out_j.p, n * 4, cudaMemcpyDeviceToDevice, s));
  if (d_ed) MJ_CUDA_TRY(cudaMemcpyAsync(d_ed, c->out_ed.p, n * 4, cudaMemcpyDeviceToDevice, s));
  return MJ_OK;
}

int mj_join_host(mj_ctx* c, const uint8_t* h_bytes, const int64_t* h_offsets, uint32_t n, const mj_params* p,
                 void* stream, uint64_t* count) {
  if (!c || !h_offsets || !p || !count) return MJ_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  const uint64_t nbytes = (uint64_t)h_offsets[n];
  if (nbytes && !h_bytes) return MJ_ERR_ARG;
  MJ_TRY(c->in_bytes.reserve(nbytes + 16, s));
  MJ_TRY(c->in_offsets.reserve(((size_t)n + 1) * 8, s));
  if (nbytes) MJ_CUDA_TRY(cudaMemcpyAsync(c->in_bytes.p, h_bytes, nbytes, cudaMemcpyHostToDevice, s));
  MJ_CUDA_TRY(cudaMemcpyAsync(c->in_offsets.p, h_offsets, ((size_t)n + 1) * 8, cudaMemcpyHostToDevice, s));
  return mj_join(c, c->in_bytes.as<uint8_t>(), c->in_offsets.as<int64_t>(), n, p, stream, count);
}

int mj_result_copy_host(mj_ctx* c, uint32_t* h_i, uint32_t* h_j, uint32_t* h_ed, void* stream) {
  if (!c) return MJ_ERR_ARG;
  if (!c->have_out) return MJ_ERR_STATE;
  DeviceGuard g(c->device);
  cudaStream_t s = S(stream);
  const size_t n = c->n_out;
  if (n) {
    if (h_i) MJ_CUDA_TRY(cudaMemcpyAsync(h_i, c->out_i.p, n * 4, cudaMemcpyDeviceToHost, s));
    if (h_j) MJ_CUDA_TRY(cudaMemcpyAsync(h_j, c->out_j.p, n * 4, cudaMemcpyDeviceToHost, s));
    if (h_ed) MJ_CUDA_TRY(cudaMemcpyAsync(h_ed, c->out_ed.p, n * 4, cudaMemcpyDeviceToHost, s));
  }
  MJ_CUDA_TRY(cudaStreamSynchronize(s));
  return MJ_OK;
}

}  // extern "C"
