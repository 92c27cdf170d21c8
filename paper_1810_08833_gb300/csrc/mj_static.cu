// mj_verify_static: the verification entry point for callers that may not
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a host
// application whose device memory is all handed out by that application's own
// pool, real-time paths that must not take the device-wide synchronisation a
// cudaMalloc/cudaFree can imply, or deployments with a fixed device-memory
// budget decided at start-up.  This entry point does the work of mj_verify
// with no allocation at all: its scratch (the equality bit-planes and the
// persistent kernel's work counter) lives in one file-scope __device__ array of
// kStaticScratchBytes, which every GPU that loads the library holds until the
// process exits.
//
// The array's name is only a host-side stand-in in host code, so its device
// address is looked up with cudaGetSymbolAddress once per device (with that
// device current) on the first call there, and passed to the kernels.
#include <mutex>

#include "mj_internal.cuh"

namespace mj {
namespace {

constexpr size_t kStaticScratchBytes = (size_t)MJ_VERIFY_STATIC_SCRATCH_BYTES;
constexpr size_t kHeaderBytes = 256;   // work counter and device flags
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (set up once).
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return MJ_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      set_last_cuda_error(e, "cudaGetSymbolAddress(g_static_scratch)", __FILE__, __LINE__);
      return MJ_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return MJ_OK;
}

}  // namespace
}  // namespace mj

extern "C" int mj_verify_static(const uint8_t* d_bytes, const int64_t* d_offsets, uint32_t n,
                                const uint32_t* d_i, const uint32_t* d_j, uint64_t m, uint32_t K,
                                void* stream, uint32_t* d_ed) {
  using namespace mj;
  if (!d_offsets) return MJ_ERR_ARG;
  if (m && (!d_i || !d_j || !d_ed)) return MJ_ERR_ARG;
  if (K > MJ_VERIFY_STATIC_MAX_K) return MJ_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  MJ_CUDA_TRY(cudaGetDevice(&dev));
  void* scratch = nullptr;
  MJ_TRY(scratch_address(dev, &scratch));
  // total input size, read into host stack memory
  int64_t nbytes = 0;
  MJ_CUDA_TRY(cudaMemcpyAsync(&nbytes, d_offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  MJ_CUDA_TRY(cudaStreamSynchronize(s));
  if (nbytes < 0) return MJ_ERR_ARG;
  if (nbytes > 0 && !d_bytes) return MJ_ERR_ARG;
  if (m == 0) return MJ_OK;
  // eight bit-planes of the raw bytes (identity symbol codes)
  const uint32_t bits = 8;
  const uint32_t GW = plane_guard_words(K);
  const uint64_t PW = ((uint64_t)nbytes + 31) / 32 + 2 * (uint64_t)GW;
  if (kHeaderBytes + (size_t)PW * bits * 4 > kStaticScratchBytes) return MJ_ERR_UNSUPPORTED;
  unsigned long long* next = static_cast<unsigned long long*>(scratch);
  uint32_t* flags = reinterpret_cast<uint32_t*>(static_cast<char*>(scratch) + 64);
  uint32_t* planes = reinterpret_cast<uint32_t*>(static_cast<char*>(scratch) + kHeaderBytes);
  MJ_CUDA_TRY(cudaMemsetAsync(scratch, 0, kHeaderBytes, s));   // counter and flags start at zero
  RankTable rt;
  for (int b = 0; b < 256; ++b) rt.r[b] = (uint8_t)b;
  MJ_TRY(launch_build_planes(d_bytes, (uint64_t)nbytes, rt, bits, planes, PW, GW, nullptr, s));
  VerifyArgs a;
  a.planes = planes;
  a.bits = bits;
  a.bytes = d_bytes;
  a.offsets = d_offsets;
  a.n_strings = n;
  a.pi = d_i;
  a.pj = d_j;
  a.pk = nullptr;
  a.order = nullptr;
  a.skip_kband = nullptr;
  a.first_ed = nullptr;
  a.range_lo = nullptr;
  a.range_hi = nullptr;
  a.skipped = nullptr;
  a.K = K;
  a.m = m;
  a.ed = d_ed;
  a.cells = nullptr;
  a.work = nullptr;
  a.dev_flags = flags;
  return launch_verify(a, PW, GW, K, next, s);
}

extern "C" int mj_verify_static_flags(void* stream, uint32_t* flags) {
  using namespace mj;
  if (!flags) return MJ_ERR_ARG;
  *flags = 0;
  int dev = 0;
  MJ_CUDA_TRY(cudaGetDevice(&dev));
  void* scratch = nullptr;
  MJ_TRY(scratch_address(dev, &scratch));
  uint32_t f = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MJ_CUDA_TRY(cudaMemcpyAsync(&f, static_cast<char*>(scratch) + 64, sizeof(f), cudaMemcpyDeviceToHost, s));
  MJ_CUDA_TRY(cudaStreamSynchronize(s));
  *flags = f;
  return MJ_OK;
}
