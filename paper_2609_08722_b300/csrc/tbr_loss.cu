// Pixel mean-squared error on sRGB values (Sec. 5.1 "Objective and metrics")
// and its adjoint seed lambda^C_0 = dL/dR (Sec. 5.2): a grid-stride pass writes
// dL/dR and one FP64 partial sum per block; a single block adds the partials in
// block order (reproducible).
#include "tbr_internal.cuh"

namespace tbr {

namespace {

constexpr int kLossThreads = 256;

__global__ void k_loss_partial(const float* __restrict__ rgb, const float* __restrict__ target, int64_t nval,
                               double* __restrict__ partial, float* __restrict__ dLdR) {
  const float scale = 2.0f / static_cast<float>(nval);
  double acc = 0.0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nval;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float d = rgb[i] - target[i];
    acc += static_cast<double>(d) * static_cast<double>(d);
    if (dLdR) dLdR[i] = scale * d;
  }
  __shared__ double sh[kLossThreads];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kLossThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_loss_final(const double* __restrict__ partial, int nblocks, int64_t nval,
                             float* __restrict__ loss_out) {
  __shared__ double sh[kLossThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) acc += partial[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kLossThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_out[0] = static_cast<float>(sh[0] / static_cast<double>(nval));
}

}  // namespace

int loss_blocks(int64_t npix) {
  const int64_t nval = 3 * npix;
  int64_t b = (nval + kLossThreads * 8 - 1) / (kLossThreads * 8);
  if (b < 1) b = 1;
  if (b > 1184) b = 1184;
  return static_cast<int>(b);
}

cudaError_t launch_loss(const float* rgb, const float* target, int64_t npix, double* partial, int nblocks,
                        float* loss_out, float* dLdR, cudaStream_t st) {
  const int64_t nval = 3 * npix;
  KernelTimer kt(TBR_K_LOSS, st);
  k_loss_partial<<<nblocks, kLossThreads, 0, st>>>(rgb, target, nval, partial, dLdR);
  k_loss_final<<<1, kLossThreads, 0, st>>>(partial, nblocks, nval, loss_out);
  return cudaGetLastError();
}

cudaError_t launch_loss_final(const double* partial, int nparts, int64_t nval, float* loss_out, cudaStream_t st) {
  KernelTimer kt(TBR_K_LOSS, st);
  k_loss_final<<<1, kLossThreads, 0, st>>>(partial, nparts, nval, loss_out);
  return cudaGetLastError();
}

}  // namespace tbr
