// Arithmetic peaks of this GPU, measured: the denominators of the ALU roofline.
// The library's kernels are bound by the FP32 pipe (packed FFMA2 / FMUL2 /
// FADD2 and scalar FFMA) and by the MUFU pipe (ex2, lg2, rcp, rsqrt, sqrt); no
// file the driver writes gives either rate, so they are taken here with chains
// of independent operations on every SM:
//   TBR_PEAK_FFMA2: packed fused multiply-adds, 8 independent float2 chains per
//                   thread, 2 FLOPs per lane per operation (4 per FFMA2);
//   TBR_PEAK_FFMA:  scalar fused multiply-adds, 8 chains, 2 FLOPs each;
//   TBR_PEAK_EX2 / TBR_PEAK_RCP: MUFU ex2.approx / rcp.approx, 8 chains, one
//                   result each (the rcp chain adds 1 before each reciprocal,
//                   on the FP32 pipe).
// A grid of 4 CTAs of 256 threads per SM keeps 32 warps per SM issuing.  The
// chains stay finite and the results are stored, so nothing is optimised away.
#include "tbr_host.h"

namespace tbr {
namespace {

constexpr int kPeakThreads = 256, kPeakCtasPerSm = 4, kChains = 8;

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma2(float* out, int iters, float a, float b) {
  float2 x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = make_float2(threadIdx.x * 1e-6f + k, k * 0.5f);
  const float2 A = make_float2(a, a), B = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], A, B);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k].x + x[k].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-6f + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// x <- 2^(-x) stays in (0.5, 1] for x in [0, 1]; x <- 1 / (x + 1) stays in (0.5, 1).
// (A bare x <- 1 / x was folded away by the compiler: its period is two.)
template <bool EX2>
__global__ void __launch_bounds__(kPeakThreads) k_peak_mufu(float* out, int iters) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 0.5f + (threadIdx.x & 31) * 1e-3f + k * 1e-2f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = EX2 ? ex2_a(-x[k]) : rcp_a(x[k] + 1.0f);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace tbr

using namespace tbr;

extern "C" {

tbr_status tbr_measure_peak(int32_t kind, int32_t iters, double* rate, double* elapsed_ms, void* stream) {
  if (!rate || iters <= 0 || kind < TBR_PEAK_FFMA2 || kind > TBR_PEAK_RCP)
    return fail(TBR_ERR_INVALID_ARG, "tbr_measure_peak: bad kind, iteration count or output");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "tbr_measure_peak");
  const int grid = sms * kPeakCtasPerSm;
  float* out = nullptr;
  e = dalloc(&out, static_cast<size_t>(grid) * kPeakThreads, st);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  auto launch = [&]() {
    switch (kind) {
      case TBR_PEAK_FFMA2: k_peak_ffma2<<<grid, kPeakThreads, 0, st>>>(out, iters, 0.9999f, 1e-4f); break;
      case TBR_PEAK_FFMA: k_peak_ffma<<<grid, kPeakThreads, 0, st>>>(out, iters, 0.9999f, 1e-4f); break;
      case TBR_PEAK_EX2: k_peak_mufu<true><<<grid, kPeakThreads, 0, st>>>(out, iters); break;
      default: k_peak_mufu<false><<<grid, kPeakThreads, 0, st>>>(out, iters); break;
    }
    return cudaGetLastError();
  };
  float ms = 0.0f;
  if (e == cudaSuccess) e = launch();  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(t0, st);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(t1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(t1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  dfree(out, st);
  if (e != cudaSuccess) return cuda_fail(e, "tbr_measure_peak");
  const double threads = static_cast<double>(grid) * kPeakThreads;
  // per thread and iteration: FFMA2 8 x 2 lanes x 2 FLOPs, FFMA 8 x 2 FLOPs, MUFU 8 results
  const double per = kind == TBR_PEAK_FFMA2 ? 4.0 * kChains : kind == TBR_PEAK_FFMA ? 2.0 * kChains : kChains;
  *rate = threads * iters * per / (static_cast<double>(ms) * 1e-3);
  if (elapsed_ms) *elapsed_ms = ms;
  return TBR_OK;
}

}  // extern "C"
