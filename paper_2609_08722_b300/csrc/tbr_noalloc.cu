// Allocation-free hard render: the same packing and hard-render kernels as
// tbr_render_hard, but their scratch (the packed stroke records and the status
// words) lives in one file-scope device array instead of memory allocated per
// call.  It serves callers that may not allocate device memory at all: a
// plugin hosted by another runtime that owns the whole device-memory budget,
// a real-time loop that must never block in an allocator, or code that runs
// when the memory pool is exhausted.  Such callers still pass their own input
// and output buffers.
#include <mutex>

#include "tbr_host.h"

namespace tbr {
namespace {

constexpr int kNoAllocMaxStrokes = 8192;  // 1 MiB of packed records
constexpr int kNoAllocFloats = kNoAllocMaxStrokes * kRec + 2 * ST_COUNT;  // + status words (8-byte each)

// Every GPU that loads the library holds this array until the process exits.
// In host code its name is only a host-side stand-in for the symbol: the device
// address comes from cudaGetSymbolAddress below, never from `g_noalloc_scratch`.
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {nullptr};

// Once per device, with that device current: look up the array's device address.
tbr_status scratch_for_current_device(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "tbr_render_hard_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(TBR_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "tbr_render_hard_noalloc: cudaGetSymbolAddress");
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return TBR_OK;
}

}  // namespace
}  // namespace tbr

using namespace tbr;

extern "C" {

tbr_status tbr_render_hard_noalloc(const tbr_program* prog, int32_t W, int32_t H, int32_t n_prefix, int32_t snap,
                                   float* out_rgb, int32_t* out_idx, void* stream) {
  if (!prog) return fail(TBR_ERR_INVALID_ARG, "program is NULL");
  const int n = (n_prefix < 0 || n_prefix > prog->n) ? prog->n : n_prefix;
  tbr_status s = check_program(prog, n);
  if (s != TBR_OK) return s;
  if ((s = check_size(W, H)) != TBR_OK) return s;
  if (!out_rgb) return fail(TBR_ERR_INVALID_ARG, "out_rgb is NULL");
  if (n > kNoAllocMaxStrokes)
    return fail(TBR_ERR_INVALID_ARG,
                "tbr_render_hard_noalloc replays at most %d strokes (got %d); use tbr_render_hard", kNoAllocMaxStrokes,
                n);
  float* scratch = nullptr;
  if ((s = scratch_for_current_device(&scratch)) != TBR_OK) return s;
  float* packed = scratch;
  unsigned long long* status = reinterpret_cast<unsigned long long*>(scratch + kNoAllocMaxStrokes * kRec);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: the status words must start at zero
  cudaError_t e = cudaMemsetAsync(status, 0, ST_COUNT * sizeof(unsigned long long), st);
  PackArgs pa{prog, n, 0.0f, 1.0f, snap ? 1 : 0, packed, nullptr, status};
  if (e == cudaSuccess) e = launch_pack(pa, st);
  if (e == cudaSuccess)
    e = launch_hard(packed, n, W, H, prog->background, out_rgb, out_idx, status, 0, st,
                    prog->coupling ? kTransportCoupled : kTransportCapsule);
  if (e != cudaSuccess) return cuda_fail(e, "tbr_render_hard_noalloc");
  return TBR_OK;
}

}  // extern "C"
