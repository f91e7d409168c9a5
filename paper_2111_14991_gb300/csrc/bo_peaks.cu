// Issue-rate probes of the arithmetic units the prediction kernels run on:
// the FP64 pipe (the FP64 pass's DFMA contraction and Matern), the FP32 pipe
// in scalar and packed f32x2 form (the tensor-core pass's K* producers) and
// the multi-function unit (their exp2 and reciprocal square root).  Each probe
// is a register-resident loop of independent chains, launched on every SM,
// timed with CUDA events; the rates are the denominators of the kernels'
// arithmetic rooflines.  Nothing here changes a clock or any other setting.
#include <cuda_runtime.h>

#include "bo_internal.h"

namespace bo {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void probe_dfma(double* sink, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.0) sink[0] = s;     // keeps the chains live; never true for these inputs
}

__global__ void probe_ffma(float* sink, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.0f) sink[0] = s;
}

__global__ void probe_ffma2(float* sink, int iters, float a, float b) {
  uint64_t x[kChains], av, bv;
  asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
  asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    const float v = threadIdx.x * 1e-3f + c;
    asm("mov.b64 %0, {%1, %1};" : "=l"(x[c]) : "f"(v));
  }
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
    s += lo + hi;
  }
  if (s == 12345.0f) sink[0] = s;
}

// ex2 of a bounded argument (x in (-1, 0]), alternating with rsqrt of a
// positive one: the two MUFU operations of the Matern evaluation.
__global__ void probe_mufu(float* sink, int iters) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 0.5f + 1e-4f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      float y;
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x[c]));
      asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(x[c]) : "f"(y + 1.0f));
    }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.0f) sink[0] = s;
}

}  // namespace
}  // namespace bo

using namespace bo;

extern "C" int bo_measure_alu_peaks(bo_alu_peaks* out) {
  if (!out) return report_error(BO_ERR_ARG, "null argument");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    return report_error(BO_ERR_CUDA, "no CUDA device");
  void* sink = nullptr;
  if (cudaMalloc(&sink, 256) != cudaSuccess) return report_error(BO_ERR_CUDA, "cudaMalloc failed");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int grid = sms * 8;                      // 64 warps per SM
  const double threads = (double)grid * kProbeThreads;
  // best of 5 timed launches after one warm-up; returns seconds
  auto best = [&](auto launch) {
    launch();
    float bestms = 1e30f;
    for (int r = 0; r < 5; ++r) {
      cudaEventRecord(e0);
      launch();
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms > 0.0f && ms < bestms) bestms = ms;
    }
    return bestms * 1e-3;
  };
  const int it64 = 2048, it32 = 16384, itm = 4096;
  const double t64 = best([&] { probe_dfma<<<grid, kProbeThreads>>>((double*)sink, it64, 0.999999, 1e-7); });
  const double t32 = best([&] { probe_ffma<<<grid, kProbeThreads>>>((float*)sink, it32, 0.9999f, 1e-5f); });
  const double t2 = best([&] { probe_ffma2<<<grid, kProbeThreads>>>((float*)sink, it32, 0.9999f, 1e-5f); });
  const double tm = best([&] { probe_mufu<<<grid, kProbeThreads>>>((float*)sink, itm); });
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) return report_error(BO_ERR_CUDA, "probe launch failed");
  out->fp64_fma_tflops = threads * it64 * kChains * 2.0 / t64 / 1e12;
  out->fp32_fma_tflops = threads * it32 * kChains * 2.0 / t32 / 1e12;
  out->fp32x2_fma_tflops = threads * it32 * kChains * 4.0 / t2 / 1e12;
  out->mufu_gops = threads * itm * kChains * 2.0 / tm / 1e9;
  out->sms = sms;
  return BO_OK;
}
