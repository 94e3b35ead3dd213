// Loss-fused soft forward + replay adjoint (Sec. 5.1 objective, Sec. 5.2
// adjoint) for the case where the image loss is the pixel MSE against a target:
// one call runs the pack, the soft forward with its replay record, the MSE and
// its seed lambda^C_0 = 2 (R - I*) / (3P), the replay adjoint and the gradient
// epilogue on the caller's stream, from buffers it allocates once (a fit keeps
// them across steps).  It uses the kernels of the split path, so its colours
// and gradients are those of tbr_render_soft + tbr_loss_mse +
// tbr_render_backward.  (A single kernel running forward, seed and adjoint per
// tile from a per-CTA record measured slower on B300: the adjoint's register
// budget caps the forward's occupancy.  The serving kernel keeps that form,
// where a bounded per-CTA record matters more.)
#include <cmath>

#include "tbr_host.h"

namespace tbr {

// ---------------------------------------------------------------------------
// Work buffers of the fused path (also held by a fit across steps).
// ---------------------------------------------------------------------------
cudaError_t FusedWork::allocate(int n, int k, int W, int H, int ck_, int cap_, cudaStream_t st, float drift_tol,
                                int repair_cap, int coupled) {
  cudaError_t e = ctx_allocate(&ctx, n, k, W, H, ck_, cap_, 0, drift_tol, repair_cap, st, coupled);
  const int64_t P = static_cast<int64_t>(W) * H;
  nblk = loss_blocks(P);
  if (e == cudaSuccess) e = dalloc(&rgb, static_cast<size_t>(P) * 3, st);
  if (e == cudaSuccess) e = dalloc(&dLdR, static_cast<size_t>(P) * 3, st);
  if (e == cudaSuccess) e = dalloc(&loss_part, static_cast<size_t>(nblk), st);
  if (e == cudaSuccess) e = dalloc(&loss_tmp, 1, st);
  status = ctx.status;
  cap = ctx.cap;
  bytes = ctx.bytes + static_cast<size_t>(P) * 24 + static_cast<size_t>(nblk) * 8 + 4;
  return e;
}

void FusedWork::release(cudaStream_t st) {
  ctx.last_stream = st;
  ctx_release(&ctx);
  dfree(rgb, st); dfree(dLdR, st); dfree(loss_part, st); dfree(loss_tmp, st);
  status = nullptr;
}

cudaError_t FusedWork::run(const tbr_program* prog, float tau, float tau_min, const float* target, float* out_rgb,
                           float* loss_out, float* g_cx, float* g_cy, float* g_th, float* g_len, float* g_r,
                           float* g_logits, float* g_pal, cudaStream_t st) {
  float* R = out_rgb ? out_rgb : rgb;
  const int64_t P = static_cast<int64_t>(ctx.W) * ctx.H;
  cudaError_t e = ctx_forward(&ctx, prog, tau, tau_min, R, st);
  if (e == cudaSuccess) e = launch_loss(R, target, P, loss_part, nblk, loss_out ? loss_out : loss_tmp, dLdR, st);
  if (e == cudaSuccess) e = ctx_backward(&ctx, dLdR, g_cx, g_cy, g_th, g_len, g_r, g_logits, g_pal, st);
  return e;
}

}  // namespace tbr

using namespace tbr;

extern "C" {

tbr_status tbr_render_soft_adjoint_mse(const tbr_program* prog, int32_t W, int32_t H, const tbr_soft_opts* opts,
                                       const float* target, float* out_rgb, float* loss_out, float* g_cx,
                                       float* g_cy, float* g_theta, float* g_length, float* g_half_width,
                                       float* g_logits, float* g_palette, tbr_ctx_stats* stats, void* stream) {
  tbr_status s = check_program(prog, prog ? prog->n : 0);
  if (s != TBR_OK) return s;
  if ((s = check_size(W, H)) != TBR_OK) return s;
  if (!opts || !target) return fail(TBR_ERR_INVALID_ARG, "opts or target is NULL");
  if (!(opts->tau >= 0.0f) || !(opts->tau_min > 0.0f)) return fail(TBR_ERR_INVALID_ARG, "need tau >= 0, tau_min > 0");
  if (opts->inert) return fail(TBR_ERR_INVALID_ARG, "the loss-fused path renders the transport model only");
  if (opts->transport != TBR_TRANSPORT_CAPSULE)
    return fail(TBR_ERR_INVALID_ARG, "the replay adjoint is built for the capsule transport");
  if (opts->checkpoint_every < 0 || opts->record_capacity < 0)
    return fail(TBR_ERR_INVALID_ARG, "negative checkpoint interval or record capacity");
  if (opts->repair_capacity < 0 || opts->repair_capacity > kRepairMax || !std::isfinite(opts->drift_tolerance))
    return fail(TBR_ERR_INVALID_ARG, "repair capacity outside [0, %d] or non-finite drift tolerance", kRepairMax);
  if (prog->n > 0 && (!g_cx || !g_cy || !g_theta || !g_length || !g_half_width || !g_logits))
    return fail(TBR_ERR_INVALID_ARG, "NULL gradient output");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FusedWork w;
  cudaError_t e = w.allocate(prog->n, prog->k, W, H, opts->checkpoint_every > 0 ? opts->checkpoint_every : 64,
                             opts->record_capacity > 0 ? opts->record_capacity : 64, st,
                             opts->drift_tolerance > 0.0f ? opts->drift_tolerance : kDriftTol,
                             opts->repair_capacity > 0 ? opts->repair_capacity : kDefaultRepairCap,
                             prog->coupling ? 1 : 0);
  if (e == cudaSuccess)
    e = w.run(prog, opts->tau, opts->tau_min, target, out_rgb, loss_out, g_cx, g_cy, g_theta, g_length,
              g_half_width, g_logits, g_palette, st);
  unsigned long long host[ST_COUNT] = {0};
  if (e == cudaSuccess && stats) {
    e = cudaMemcpyAsync(host, w.status, sizeof(host), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  w.release(st);
  if (e != cudaSuccess) return cuda_fail(e, "tbr_render_soft_adjoint_mse");
  if (stats) {
    stats->records = static_cast<int64_t>(host[ST_RECORDS]);
    stats->max_records = static_cast<int64_t>(host[ST_MAXREC]);
    stats->overflow_pixels = static_cast<int64_t>(host[ST_OVERFLOW]);
    stats->drift_resets = static_cast<int64_t>(host[ST_DRIFT]);
    stats->timeouts = static_cast<int64_t>(host[ST_TIMEOUT]);
    stats->invalid_params = static_cast<int64_t>(host[ST_INVALID]);
    stats->repaired_pixels = static_cast<int64_t>(host[ST_REPAIRED]);
    stats->repair_overflow = static_cast<int64_t>(host[ST_REPAIR_OVF]);
    if (host[ST_INVALID]) return fail(TBR_ERR_INVALID_ARG, "%llu strokes failed the value checks", host[ST_INVALID]);
    if (host[ST_OVERFLOW]) return fail(TBR_ERR_OVERFLOW, "%llu pixels exceeded the side-table capacity", host[ST_OVERFLOW]);
    if (host[ST_TIMEOUT]) return fail(TBR_ERR_TIMEOUT, "a bounded device wait gave up");
  }
  return TBR_OK;
}

}  // extern "C"
