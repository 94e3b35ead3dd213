// Host-side internals shared by the C ABI translation units: error reporting,
// argument checks, stream-ordered allocation and the replay context.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "tbr.h"
#include "tbr_internal.cuh"

// Replay context (opaque in tbr.h): what one soft forward leaves for the
// replay adjoint of Sec. 5.2, plus the backward's reduction scratch.
struct tbr_ctx {
  int n = 0, k = 0, W = 0, H = 0, ck = 32, cap = 64, inert = 0, grid = 0;
  int coupled = 0;                    // 1: the program carries a coupling profile (Eq. coupling)
  float bg[3] = {0, 0, 0};
  float inv_tc = 1.0f;
  float* packed = nullptr;            // [n][kRec]
  float* probs = nullptr;             // [n][k] softmax probabilities
  float* palette = nullptr;           // [k][3] copy
  float4* s0 = nullptr;               // [P] x_0 as (x_hi, y_hi, x_lo, y_lo)
  float2* s0b = nullptr;              // [P] (log2 T_0, record count)
  float4* ckpt = nullptr;             // [(n-1)/ck][P] x_i checkpoints (hi/lo)
  float* ck_lt = nullptr;             // [(n-1)/ck][P] log2 T_i at the checkpoints
  float4* rec = nullptr;              // [cap][P] side table positions (hi/lo)
  int* rec_i = nullptr;               // [cap][P] side table stroke indices
  unsigned long long* status = nullptr;  // [ST_COUNT]
  float* partial = nullptr;           // [grid][n][8] per-CTA gradient partials
  float* grad8 = nullptr;             // [n][8]
  float drift_tol = 1e-5f;            // checkpoint drift that triggers the FP64 repair
  int repair_cap = 0;                 // repair list capacity (0: no repair)
  int2* repair_list = nullptr;        // [repair_cap] (pixel, segment start)
  int* repair_count = nullptr;        // [1]
  float* corr = nullptr;              // [repair_cap][n][8] gradient corrections
  unsigned char* repair_first = nullptr;  // [P] per-pixel "queued" flags
  cudaStream_t last_stream = nullptr;
  size_t bytes = 0;
};

namespace tbr {

tbr_status fail(tbr_status code, const char* fmt, ...);
const char* last_error_text();
tbr_status cuda_fail(cudaError_t e, const char* what);
tbr_status check_program(const tbr_program* p, int n_used);
tbr_status check_size(int32_t W, int32_t H);

// Keeps memory freed by cudaFreeAsync in the current device's default pool
// (release threshold = unlimited, set once per device in this process), so the
// allocating entry points reuse it across calls instead of returning it to the
// driver at every synchronisation.
void retain_pool_memory();

template <class T>
cudaError_t dalloc(T** p, size_t count, cudaStream_t st) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  retain_pool_memory();
  return cudaMallocAsync(reinterpret_cast<void**>(p), count * sizeof(T), st);
}
template <class T>
void dfree(T*& p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
  p = nullptr;
}

// Allocates every buffer of a context for n strokes, palette k, W x H pixels.
// repair_cap pixels can have a drifting segment regenerated in FP64 (0: none).
// coupled: the coupling variant's record and adjoint (no FP64 repair).
cudaError_t ctx_allocate(tbr_ctx* c, int n, int k, int W, int H, int ck, int cap, int inert, float drift_tol,
                         int repair_cap, cudaStream_t st, int coupled = 0);
constexpr int kDefaultRepairCap = 256;
void ctx_release(tbr_ctx* c);
// Soft forward into an allocated context (resets its status words).
cudaError_t ctx_forward(tbr_ctx* c, const tbr_program* prog, float tau, float tau_min,
                        float* out_rgb, cudaStream_t st);
// Replay adjoint of the context's last forward.
cudaError_t ctx_backward(tbr_ctx* c, const float* dLdR, float* g_cx, float* g_cy, float* g_th,
                         float* g_len, float* g_r, float* g_logits, float* g_pal, cudaStream_t st);
// Reads the status words (synchronising) and maps them to a tbr_status.
tbr_status ctx_read_status(tbr_ctx* c, unsigned long long host[ST_COUNT]);

// Buffers of the loss-fused forward + adjoint (tbr_fused.cu): a replay context
// plus the colour, the MSE seed and the loss partials.
struct FusedWork {
  tbr_ctx ctx;
  float* rgb = nullptr;                  // [P][3] when the caller keeps no colour
  float* dLdR = nullptr;                 // [P][3] MSE seed
  double* loss_part = nullptr;           // [nblk] FP64 loss partials
  float* loss_tmp = nullptr;             // [1] loss when the caller keeps none
  unsigned long long* status = nullptr;  // the context's status words
  int nblk = 0, cap = 0;
  size_t bytes = 0;
  // coupled: the program carries a coupling profile (its record and adjoint)
  cudaError_t allocate(int n, int k, int W, int H, int ck, int cap, cudaStream_t st, float drift_tol = 1e-5f,
                       int repair_cap = kDefaultRepairCap, int coupled = 0);
  void release(cudaStream_t st);
  // pack + soft forward + MSE and seed + replay adjoint + gradient epilogue;
  // status words reset first.
  cudaError_t run(const tbr_program* prog, float tau, float tau_min, const float* target, float* out_rgb,
                  float* loss_out, float* g_cx, float* g_cy, float* g_th, float* g_len, float* g_r,
                  float* g_logits, float* g_pal, cudaStream_t st);
};

}  // namespace tbr

#define TBR_CUDA(call, what)                                 \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return ::tbr::cuda_fail(e_, what); \
  } while (0)
