// Learned first-pass band: candidate features and an FP32 MLP (8 -> 64 -> 64
// -> 1, ReLU) with hand-written forward, backward and Adam kernels.  Nothing
// here is in the MinJoin paper; the band it proposes only narrows a first
// verification pass, and every pair that pass does not settle is verified
// again with band K, so the join's output does not depend on the model.
#include "mj_internal.cuh"

namespace mj {
namespace {

constexpr int F = kBandFeatures;
constexpr int H = kBandHidden;
constexpr int OFF_W1 = 0;               // [H][F]
constexpr int OFF_B1 = OFF_W1 + H * F;  // [H]
constexpr int OFF_W2 = OFF_B1 + H;      // [H][H]
constexpr int OFF_B2 = OFF_W2 + H * H;  // [H]
constexpr int OFF_W3 = OFF_B2 + H;      // [H]
constexpr int OFF_B3 = OFF_W3 + H;      // [1]
static_assert(OFF_B3 + 1 == kBandParams, "parameter layout");

__device__ __forceinline__ float relu(float v) { return v > 0.f ? v : 0.f; }

// Features of candidate u (see kBandFeatures in mj_internal.cuh).
__global__ void features_kernel(const uint32_t* __restrict__ ci, const uint32_t* __restrict__ cj,
                                const uint32_t* __restrict__ mult, const uint32_t* __restrict__ parts,
                                const int64_t* __restrict__ offsets, uint64_t m, uint32_t K, uint32_t T,
                                float* __restrict__ X) {
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < m; u += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = ci[u], y = cj[u];
    const int64_t lx = offsets[x + 1] - offsets[x], ly = offsets[y + 1] - offsets[y];
    const float n = (float)(lx < ly ? lx : ly), d0 = (float)(lx < ly ? ly - lx : lx - ly);
    const float c = (float)mult[u];
    const float pa = (float)parts[x], pb = (float)parts[y];
    const float pmin = fminf(pa, pb) > 1.f ? fminf(pa, pb) : 1.f;
    const float t1 = (float)T + 1.f;
    float* o = X + u * F;
    o[0] = log2f(1.f + n) / 16.f;
    o[1] = d0 / (float)(K ? K : 1);
    o[2] = c / t1;
    o[3] = pa / t1;
    o[4] = pb / t1;
    o[5] = c / pmin;
    o[6] = log2f(1.f + c) / 8.f;
    o[7] = (float)K / (float)(K + 100);
  }
}

// ŷ of every sample (gate: samples with gate[u] < min_gate get +inf).
__global__ void __launch_bounds__(128) forward_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                      uint64_t m, const uint32_t* __restrict__ gate,
                                                      uint32_t min_gate, float* __restrict__ out) {
  __shared__ float s[kBandParams];
  for (int i = threadIdx.x; i < kBandParams; i += blockDim.x) s[i] = P[i];
  __syncthreads();
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < m; u += (uint64_t)gridDim.x * blockDim.x) {
    if (gate && gate[u] < min_gate) {
      out[u] = __int_as_float(0x7f800000);
      continue;
    }
    float x[F];
#pragma unroll
    for (int f = 0; f < F; ++f) x[f] = X[u * F + f];
    float h1[H];
#pragma unroll
    for (int a = 0; a < H; ++a) {
      float z = s[OFF_B1 + a];
#pragma unroll
      for (int f = 0; f < F; ++f) z = fmaf(s[OFF_W1 + a * F + f], x[f], z);
      h1[a] = relu(z);
    }
    float y = s[OFF_B3];
#pragma unroll 4
    for (int c = 0; c < H; ++c) {
      float z = s[OFF_B2 + c];
#pragma unroll
      for (int a = 0; a < H; ++a) z = fmaf(s[OFF_W2 + c * H + a], h1[a], z);
      y = fmaf(s[OFF_W3 + c], relu(z), y);
    }
    out[u] = y;
  }
}

__device__ __forceinline__ uint64_t mix(uint64_t z) {  // splitmix64 finaliser (Steele, Lea, Flood 2014)
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

constexpr int kSB = 64;   // samples per block chunk of the gradient kernel
constexpr int kLd = H + 1;

// Loss and parameter gradient of a batch, accumulated (atomically, one add
// per parameter and block chunk) into grad[] and *loss.
//  samples: batch indices idx[b] if idx is given, else b (b < batch); with
//           seed != 0 a sample is drawn as mix(seed + b) % m.
//  target:  y from Y, or from ed as min(ed, K+1) / K.
//  loss:    tau == 0: mean squared error; else pinball loss at quantile tau.
__global__ void __launch_bounds__(kSB) grad_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                   const float* __restrict__ Y, const uint32_t* __restrict__ ed,
                                                   uint32_t K, uint64_t m, uint64_t batch, uint64_t seed, float tau,
                                                   float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ float sm[];
  float* w = sm;                          // kBandParams
  float* h1s = w + kBandParams;           // [kSB][kLd]
  float* h2s = h1s + kSB * kLd;           // [kSB][kLd]
  float* d2s = h2s + kSB * kLd;           // [kSB][kLd]
  float* d1s = d2s + kSB * kLd;           // [kSB][kLd]
  float* xs = d1s + kSB * kLd;            // [kSB][F]
  float* dys = xs + kSB * F;              // [kSB]
  for (int i = threadIdx.x; i < kBandParams; i += blockDim.x) w[i] = P[i];
  const float inv = 1.f / (float)batch;
  for (uint64_t base = (uint64_t)blockIdx.x * kSB; base < batch; base += (uint64_t)gridDim.x * kSB) {
    __syncthreads();
    const uint64_t bidx = base + threadIdx.x;
    const int s = threadIdx.x;
    float dy = 0.f;
    if (bidx < batch) {
      const uint64_t u = seed ? mix(seed + bidx) % m : bidx;
      float x[F];
#pragma unroll
      for (int f = 0; f < F; ++f) {
        x[f] = X[u * F + f];
        xs[s * F + f] = x[f];
      }
      float h1[H];
#pragma unroll
      for (int a = 0; a < H; ++a) {
        float z = w[OFF_B1 + a];
#pragma unroll
        for (int f = 0; f < F; ++f) z = fmaf(w[OFF_W1 + a * F + f], x[f], z);
        h1[a] = relu(z);
        h1s[s * kLd + a] = h1[a];
      }
      float yhat = w[OFF_B3];
      for (int c = 0; c < H; ++c) {
        float z = w[OFF_B2 + c];
#pragma unroll
        for (int a = 0; a < H; ++a) z = fmaf(w[OFF_W2 + c * H + a], h1[a], z);
        const float h2 = relu(z);
        h2s[s * kLd + c] = h2;
        yhat = fmaf(w[OFF_W3 + c], h2, yhat);
      }
      const float y = Y ? Y[u] : (float)(ed[u] < K + 1 ? ed[u] : K + 1) / (float)(K ? K : 1);
      const float r = y - yhat;
      float l;
      if (tau == 0.f) {
        l = r * r;
        dy = -2.f * r;
      } else {
        l = r > 0.f ? tau * r : (tau - 1.f) * r;
        dy = r > 0.f ? -tau : (1.f - tau);
      }
      dy *= inv;
      atomicAdd(loss, l * inv);
      // back through layer 3 and the second ReLU
      float dh1[H];
#pragma unroll
      for (int a = 0; a < H; ++a) dh1[a] = 0.f;
      for (int c = 0; c < H; ++c) {
        const float d2 = h2s[s * kLd + c] > 0.f ? dy * w[OFF_W3 + c] : 0.f;
        d2s[s * kLd + c] = d2;
#pragma unroll
        for (int a = 0; a < H; ++a) dh1[a] = fmaf(w[OFF_W2 + c * H + a], d2, dh1[a]);
      }
#pragma unroll
      for (int a = 0; a < H; ++a) d1s[s * kLd + a] = h1[a] > 0.f ? dh1[a] : 0.f;
    } else {
      for (int a = 0; a < H; ++a) {
        h1s[s * kLd + a] = 0.f;
        h2s[s * kLd + a] = 0.f;
        d2s[s * kLd + a] = 0.f;
        d1s[s * kLd + a] = 0.f;
      }
      for (int f = 0; f < F; ++f) xs[s * F + f] = 0.f;
    }
    dys[s] = dy;
    __syncthreads();
    // parameter gradients of the chunk: sums over its samples
    for (int p = threadIdx.x; p < kBandParams; p += blockDim.x) {
      float g = 0.f;
      if (p < OFF_B1) {
        const int a = p / F, f = p % F;
        for (int q = 0; q < kSB; ++q) g = fmaf(d1s[q * kLd + a], xs[q * F + f], g);
      } else if (p < OFF_W2) {
        const int a = p - OFF_B1;
        for (int q = 0; q < kSB; ++q) g += d1s[q * kLd + a];
      } else if (p < OFF_B2) {
        const int c = (p - OFF_W2) / H, a = (p - OFF_W2) % H;
        for (int q = 0; q < kSB; ++q) g = fmaf(d2s[q * kLd + c], h1s[q * kLd + a], g);
      } else if (p < OFF_W3) {
        const int c = p - OFF_B2;
        for (int q = 0; q < kSB; ++q) g += d2s[q * kLd + c];
      } else if (p < OFF_B3) {
        const int c = p - OFF_W3;
        for (int q = 0; q < kSB; ++q) g = fmaf(dys[q], h2s[q * kLd + c], g);
      } else {
        for (int q = 0; q < kSB; ++q) g += dys[q];
      }
      if (g != 0.f) atomicAdd(grad + p, g);
    }
  }
}

// Adam (Kingma & Ba 2015) with bias correction.
__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                            float* __restrict__ V, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kBandParams) return;
  const float g = G[i];
  const float mm = b1 * M[i] + (1.f - b1) * g;
  const float vv = b2 * V[i] + (1.f - b2) * g * g;
  M[i] = mm;
  V[i] = vv;
  P[i] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// First-pass band of candidate u from ŷ: the widest band that still fits in
// the fewest 32-bit words holding ceil(ŷ K) + margin (and at least the
// length difference); pairs that would need as many words as band K get K.
__global__ void band_rule_kernel(const float* __restrict__ yhat, const uint32_t* __restrict__ ci,
                                 const uint32_t* __restrict__ cj, const int64_t* __restrict__ offsets, uint64_t m,
                                 uint32_t K, uint32_t margin, uint32_t* __restrict__ kband) {
  const uint32_t wK = (K + 1 + 31) / 32;
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < m; u += (uint64_t)gridDim.x * blockDim.x) {
    const float y = yhat[u];
    uint32_t kb = K;
    if (y == y && y < 1.f) {   // not NaN, predicted within K
      const uint32_t x = ci[u], z = cj[u];
      const int64_t lx = offsets[x + 1] - offsets[x], lz = offsets[z + 1] - offsets[z];
      const uint32_t d0 = (uint32_t)(lx > lz ? lx - lz : lz - lx);
      float want = ceilf(fmaxf(y, 0.f) * (float)K) + (float)margin;
      uint32_t kw = want > (float)K ? K : (uint32_t)want;
      if (kw < d0) kw = d0;
      const uint32_t w = (kw + 1 + 31) / 32;
      kb = w < wK ? 32 * w - 1 : K;
    }
    kband[u] = kb;
  }
}

// Network output for one feature row (weights in shared memory).
__device__ __forceinline__ float mlp_eval(const float* s, const float* xf) {
  float h1[H];
#pragma unroll
  for (int a = 0; a < H; ++a) {
    float zz = s[OFF_B1 + a];
#pragma unroll
    for (int f = 0; f < F; ++f) zz = fmaf(s[OFF_W1 + a * F + f], xf[f], zz);
    h1[a] = relu(zz);
  }
  float y = s[OFF_B3];
#pragma unroll 4
  for (int cc = 0; cc < H; ++cc) {
    float zz = s[OFF_B2 + cc];
#pragma unroll
    for (int a = 0; a < H; ++a) zz = fmaf(s[OFF_W2 + cc * H + a], h1[a], zz);
    y = fmaf(s[OFF_W3 + cc], relu(zz), y);
  }
  return y;
}

constexpr int kQueue = 128;   // threads per block of the fused band kernel

// Features, network and band rule in one pass over the candidates (learned
// joins).  Candidates from fewer than min_mult matched partition pairs keep
// band K without running the network; the others are gathered in a block
// queue and evaluated 128 at a time, so a sparse gate does not leave lanes
// idle during the network.
__global__ void __launch_bounds__(kQueue) band_fused_kernel(const float* __restrict__ P, const uint32_t* __restrict__ ci,
                                                            const uint32_t* __restrict__ cj,
                                                            const uint32_t* __restrict__ run_start, uint64_t raw,
                                                            const uint32_t* __restrict__ parts,
                                                            const int64_t* __restrict__ offsets, uint64_t m, uint32_t K,
                                                            uint32_t T, uint32_t margin, uint32_t min_mult,
                                                            uint32_t* __restrict__ kband) {
  __shared__ float s[kBandParams];
  __shared__ uint32_t q_u[2 * kQueue];
  __shared__ uint32_t q_c[2 * kQueue];
  __shared__ uint32_t qn;
  for (int i = threadIdx.x; i < kBandParams; i += blockDim.x) s[i] = P[i];
  if (threadIdx.x == 0) qn = 0;
  __syncthreads();
  const uint32_t wK = (K + 1 + 31) / 32;
  auto evaluate = [&](uint64_t u, uint32_t c) {
    const uint32_t x = ci[u], z = cj[u];
    const int64_t lx = offsets[x + 1] - offsets[x], lz = offsets[z + 1] - offsets[z];
    const uint32_t d0 = (uint32_t)(lx > lz ? lx - lz : lz - lx);
    const float n = (float)(lx < lz ? lx : lz);
    const float pa = (float)parts[x], pb = (float)parts[z];
    const float pmin = fminf(pa, pb) > 1.f ? fminf(pa, pb) : 1.f;
    const float t1 = (float)T + 1.f;
    const float xf[F] = {log2f(1.f + n) / 16.f, (float)d0 / (float)(K ? K : 1), (float)c / t1, pa / t1, pb / t1,
                         (float)c / pmin, log2f(1.f + (float)c) / 8.f, (float)K / (float)(K + 100)};
    const float y = mlp_eval(s, xf);
    uint32_t kb = K;
    if (y == y && y < 1.f) {
      const float want = ceilf(fmaxf(y, 0.f) * (float)K) + (float)margin;
      uint32_t kw = want > (float)K ? K : (uint32_t)want;
      if (kw < d0) kw = d0;
      const uint32_t w = (kw + 1 + 31) / 32;
      if (w < wK) kb = 32 * w - 1;
    }
    kband[u] = kb;
  };
  const uint64_t stride = (uint64_t)gridDim.x * kQueue;
  for (uint64_t base = (uint64_t)blockIdx.x * kQueue; base < m; base += stride) {
    const uint64_t u = base + threadIdx.x;
    if (u < m) {
      const uint64_t e = u + 1 < m ? run_start[u + 1] : raw;
      const uint32_t c = (uint32_t)(e - run_start[u]);
      kband[u] = K;
      if (c >= min_mult) {
        const uint32_t slot = atomicAdd(&qn, 1u);
        q_u[slot] = (uint32_t)u;
        q_c[slot] = c;
      }
    }
    __syncthreads();
    const uint32_t n_q = qn;
    const bool last = base + stride >= m;
    if (n_q >= kQueue || (last && n_q > 0)) {
      // evaluate the first min(n_q, kQueue) entries, keep the rest queued
      const uint32_t take = n_q < kQueue ? n_q : kQueue;
      if (threadIdx.x < take) evaluate(q_u[threadIdx.x], q_c[threadIdx.x]);
      __syncthreads();
      const uint32_t left = n_q - take;
      const bool mv = threadIdx.x < left;
      uint32_t qa = 0, qb = 0;
      if (mv) {
        qa = q_u[take + threadIdx.x];
        qb = q_c[take + threadIdx.x];
      }
      __syncthreads();
      if (mv) {
        q_u[threadIdx.x] = qa;
        q_c[threadIdx.x] = qb;
      }
      if (threadIdx.x == 0) qn = left;
      __syncthreads();
      if (last && left > 0) {
        if (threadIdx.x < left) evaluate(q_u[threadIdx.x], q_c[threadIdx.x]);
        __syncthreads();
        if (threadIdx.x == 0) qn = 0;
        __syncthreads();
      }
    }
  }
}

// Gate for the learned band from training samples: the 1st percentile of the
// multiplicity c (recovered from feature 6 = log2(1+c)/8) among samples whose
// band-K result fits a band narrower than K's word count, written to *out.
__global__ void gate_hist_kernel(const float* __restrict__ X, const uint32_t* __restrict__ ed, uint64_t m, uint32_t K,
                                 unsigned int* __restrict__ hist) {
  const uint32_t wK = (K + 1 + 31) / 32;
  const uint32_t kmax1 = wK > 1 ? 32 * (wK - 1) - 1 : 0;
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < m; u += (uint64_t)gridDim.x * blockDim.x) {
    if (wK <= 1 || ed[u] > kmax1) continue;
    const float c = exp2f(8.f * X[u * F + 6]) - 1.f;
    uint32_t ci = (uint32_t)(c + 0.5f);
    if (ci > 255) ci = 255;
    atomicAdd(hist + ci, 1u);
  }
}

unsigned grid1(uint64_t n, int threads) {
  uint64_t g = (n + threads - 1) / threads;
  uint64_t cap = (uint64_t)kNumSMsHint * 16;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

int launch_band_features(const uint32_t* ci, const uint32_t* cj, const uint32_t* mult, const uint32_t* parts,
                         const int64_t* offsets, uint64_t m, uint32_t K, uint32_t T, float* X, cudaStream_t s) {
  if (!m) return MJ_OK;
  features_kernel<<<grid1(m, 256), 256, 0, s>>>(ci, cj, mult, parts, offsets, m, K, T, X);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_band_forward(const float* P, const float* X, uint64_t m, const uint32_t* gate, uint32_t min_gate,
                        float* out, cudaStream_t s) {
  if (!m) return MJ_OK;
  forward_kernel<<<grid1(m, 128), 128, 0, s>>>(P, X, m, gate, min_gate, out);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

size_t band_grad_smem() { return sizeof(float) * (kBandParams + 4 * kSB * kLd + kSB * F + kSB); }

int launch_band_grad(const float* P, const float* X, const float* Y, const uint32_t* ed, uint32_t K, uint64_t m,
                     uint64_t batch, uint64_t seed, float tau, float* grad, float* loss, cudaStream_t s) {
  if (!batch) return MJ_OK;
  const size_t smem = band_grad_smem();
  MJ_CUDA_TRY(cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  uint64_t blocks = (batch + kSB - 1) / kSB;
  if (blocks > (uint64_t)kNumSMsHint * 2) blocks = (uint64_t)kNumSMsHint * 2;
  grad_kernel<<<(unsigned)blocks, kSB, smem, s>>>(P, X, Y, ed, K, m, batch, seed, tau, grad, loss);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_band_adam(float* P, const float* G, float* M, float* V, float lr, float b1, float b2, float eps, int step,
                     cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<(kBandParams + 255) / 256, 256, 0, s>>>(P, G, M, V, lr, b1, b2, eps, c1, c2);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_band_fused(const float* P, const uint32_t* ci, const uint32_t* cj, const uint32_t* run_start, uint64_t raw,
                      const uint32_t* parts, const int64_t* offsets, uint64_t m, uint32_t K, uint32_t T, uint32_t margin,
                      uint32_t min_mult, uint32_t* kband, cudaStream_t s) {
  if (!m) return MJ_OK;
  band_fused_kernel<<<grid1(m, kQueue), kQueue, 0, s>>>(P, ci, cj, run_start, raw, parts, offsets, m, K, T, margin,
                                                       min_mult, kband);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_gate_hist(const float* X, const uint32_t* ed, uint64_t m, uint32_t K, unsigned int* hist, cudaStream_t s) {
  MJ_CUDA_TRY(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned int), s));
  if (!m) return MJ_OK;
  gate_hist_kernel<<<grid1(m, 256), 256, 0, s>>>(X, ed, m, K, hist);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

int launch_band_rule(const float* yhat, const uint32_t* ci, const uint32_t* cj, const int64_t* offsets, uint64_t m,
                     uint32_t K, uint32_t margin, uint32_t* kband, cudaStream_t s) {
  if (!m) return MJ_OK;
  band_rule_kernel<<<grid1(m, 256), 256, 0, s>>>(yhat, ci, cj, offsets, m, K, margin, kband);
  MJ_KERNEL_DONE();
  return MJ_OK;
}

}  // namespace mj
