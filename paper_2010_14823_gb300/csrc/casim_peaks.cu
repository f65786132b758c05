// Instruction-throughput probes (see include/casim_peaks.h): each thread runs
// 8 independent chains of one operation, so that every scheduler always has
// independent work for the unit under test.
#include <cstdint>
#include <cuda_runtime.h>

#include "casim_peaks.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__device__ __forceinline__ float ex2a(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2a(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcpa(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float tanha(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// packed pair: x -> tanh(x) + 0.5 on both halves (bf16x2 add)
__device__ __forceinline__ uint32_t tanh2(uint32_t x) {
  uint32_t y;
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(x));
  asm("add.rn.bf16x2 %0, %1, %2;" : "=r"(y) : "r"(y), "r"(0x3f003f00u));
  return y;
}

template <int K>
__global__ void __launch_bounds__(kThreads) k_peak(long long iters, double *out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (K == CASIM_PEAK_TANH2) {
    uint32_t x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 0x3f203f30u + (uint32_t)i;   // pairs near 0.62
    for (long long n = 0; n < iters; ++n) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = tanh2(x[i]);
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s ^= x[i];
    out[t] = (double)s;
  } else if constexpr (K == CASIM_PEAK_DFMA) {
    double x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 0.5 + 0.01 * i + 1e-7 * (t & 63);
    const double a = 0.999, b = 0.0005;
    for (long long n = 0; n < iters; ++n) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    out[t] = s;
  } else {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.25f + 0.01f * i + 1e-6f * (t & 63);
    for (long long n = 0; n < iters; ++n) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        if constexpr (K == CASIM_PEAK_FFMA) x[i] = fmaf(x[i], 0.999f, 0.0005f);
        if constexpr (K == CASIM_PEAK_EX2) x[i] = ex2a(-x[i]);
        if constexpr (K == CASIM_PEAK_LG2) x[i] = lg2a(x[i]) + 2.f;
        if constexpr (K == CASIM_PEAK_RCP) x[i] = rcpa(x[i]) + 1.f;
        if constexpr (K == CASIM_PEAK_TANH) x[i] = tanha(x[i]) + 0.5f;
      }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    out[t] = s;
  }
}

template <int K>
cudaError_t launch(int blocks, long long iters, double *out, cudaStream_t st) {
  k_peak<K><<<blocks, kThreads, 0, st>>>(iters, out);
  return cudaGetLastError();
}

cudaError_t launch_kind(int kind, int blocks, long long iters, double *out, cudaStream_t st) {
  switch (kind) {
    case CASIM_PEAK_FFMA: return launch<CASIM_PEAK_FFMA>(blocks, iters, out, st);
    case CASIM_PEAK_DFMA: return launch<CASIM_PEAK_DFMA>(blocks, iters, out, st);
    case CASIM_PEAK_EX2: return launch<CASIM_PEAK_EX2>(blocks, iters, out, st);
    case CASIM_PEAK_LG2: return launch<CASIM_PEAK_LG2>(blocks, iters, out, st);
    case CASIM_PEAK_RCP: return launch<CASIM_PEAK_RCP>(blocks, iters, out, st);
    case CASIM_PEAK_TANH2: return launch<CASIM_PEAK_TANH2>(blocks, iters, out, st);
    default: return launch<CASIM_PEAK_TANH>(blocks, iters, out, st);
  }
}

}  // namespace

extern "C" int casim_peak_rate(int kind, long long iters, void *stream, double *rate) {
  if (kind < 0 || kind >= CASIM_PEAK_NKINDS || iters < 1 || !rate) return CASIM_PEAK_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CASIM_PEAK_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CASIM_PEAK_ERR_CUDA;
  const int blocks = nsm * kBlocksPerSm;
  double *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  cudaError_t e = cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch_kind(kind, blocks, iters, out, st);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_kind(kind, blocks, iters, out, st);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess || !(ms > 0.f)) return CASIM_PEAK_ERR_CUDA;
  const double per = kind == CASIM_PEAK_TANH2 ? 2.0 : 1.0;   // operations per instruction
  *rate = 3.0 * per * (double)blocks * kThreads * kChains * (double)iters / (ms * 1e-3);
  return 0;
}
