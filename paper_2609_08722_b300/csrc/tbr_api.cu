// C ABI of the TBR library (include/tbr.h): argument checks, stream-ordered
// device memory for scratch and replay contexts, and kernel launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include <atomic>

#include "tbr_host.h"
#include "tbr_tile.cuh"

namespace tbr {

namespace {
thread_local std::string g_last_error = "no error";
}  // namespace

tbr_status fail(tbr_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

const char* last_error_text() { return g_last_error.c_str(); }

tbr_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(TBR_ERR_OOM, "%s: out of device memory", what);
  return fail(TBR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

tbr_status check_program(const tbr_program* p, int n_used) {
  if (!p) return fail(TBR_ERR_INVALID_ARG, "program is NULL");
  if (p->n < 0) return fail(TBR_ERR_INVALID_ARG, "n = %d < 0", p->n);
  if (p->k < 1) return fail(TBR_ERR_INVALID_ARG, "palette size k = %d < 1", p->k);
  if (!(p->color_temp > 0.0f) || !std::isfinite(p->color_temp))
    return fail(TBR_ERR_INVALID_ARG, "color_temp must be finite and > 0");
  for (int c = 0; c < 3; ++c)
    if (!std::isfinite(p->background[c])) return fail(TBR_ERR_INVALID_ARG, "background not finite");
  if (n_used > 0 && (!p->cx || !p->cy || !p->theta || !p->length || !p->half_width || !p->logits))
    return fail(TBR_ERR_INVALID_ARG, "NULL stroke array");
  if (!p->palette) return fail(TBR_ERR_INVALID_ARG, "palette is NULL");
  return TBR_OK;
}

void retain_pool_memory() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  const unsigned long long bit = 1ull << dev;
  if (done.load(std::memory_order_acquire) & bit) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    unsigned long long threshold = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
  }
  done.fetch_or(bit, std::memory_order_acq_rel);
}

tbr_status check_size(int32_t W, int32_t H) {
  if (W <= 0 || H <= 0) return fail(TBR_ERR_INVALID_ARG, "image size %dx%d must be positive", W, H);
  if (static_cast<int64_t>(W) * H > (int64_t(1) << 30))
    return fail(TBR_ERR_INVALID_ARG, "image of %dx%d pixels is too large", W, H);
  return TBR_OK;
}

cudaError_t ctx_allocate(tbr_ctx* c, int n, int k, int W, int H, int ck, int cap, int inert, float drift_tol,
                         int repair_cap, cudaStream_t st, int coupled) {
  const size_t P = static_cast<size_t>(W) * H;
  c->n = n; c->k = k; c->W = W; c->H = H;
  c->ck = ck; c->cap = cap; c->inert = inert; c->coupled = coupled;
  c->drift_tol = drift_tol;
  c->repair_cap = (inert || coupled) ? 0 : repair_cap;
  c->grid = coupled ? backward_grid_coupled(W, H) : backward_grid(W, H, inert);
  c->last_stream = st;
  const size_t nck = n > 1 ? static_cast<size_t>((n - 1) / ck) : 0;
  cudaError_t e = dalloc(&c->packed, static_cast<size_t>(n) * kRec, st);
  if (e == cudaSuccess) e = dalloc(&c->status, ST_COUNT, st);
  if (e == cudaSuccess) e = dalloc(&c->probs, static_cast<size_t>(n) * k, st);
  if (e == cudaSuccess) e = dalloc(&c->palette, static_cast<size_t>(k) * 3, st);
  if (e == cudaSuccess) e = dalloc(&c->s0, P, st);
  if (e == cudaSuccess) e = dalloc(&c->s0b, P, st);
  if (e == cudaSuccess) e = dalloc(&c->ckpt, nck * P, st);
  if (e == cudaSuccess) e = dalloc(&c->ck_lt, nck * P, st);
  if (e == cudaSuccess && !inert) e = dalloc(&c->rec, static_cast<size_t>(cap) * P, st);
  if (e == cudaSuccess && !inert) e = dalloc(&c->rec_i, static_cast<size_t>(cap) * P, st);
  if (e == cudaSuccess) e = dalloc(&c->partial, static_cast<size_t>(c->grid) * n * 8, st);
  if (e == cudaSuccess) e = dalloc(&c->grad8, static_cast<size_t>(n) * 8, st);
  if (e == cudaSuccess && c->repair_cap > 0) e = dalloc(&c->repair_list, static_cast<size_t>(c->repair_cap), st);
  if (e == cudaSuccess && c->repair_cap > 0) e = dalloc(&c->repair_count, 1, st);
  if (e == cudaSuccess && c->repair_cap > 0)
    e = dalloc(&c->corr, static_cast<size_t>(c->repair_cap) * n * 8, st);
  if (e == cudaSuccess && c->repair_cap > 0) e = dalloc(&c->repair_first, P + pair_tile_count(W, H), st);
  c->bytes = static_cast<size_t>(n) * kRec * 4 + ST_COUNT * 8 + static_cast<size_t>(n) * k * 4 +
             static_cast<size_t>(k) * 12 + P * 24 + nck * P * 20 +
             (inert ? 0 : static_cast<size_t>(cap) * P * 20) + static_cast<size_t>(c->grid) * n * 32 +
             static_cast<size_t>(n) * 32 +
             static_cast<size_t>(c->repair_cap) * (8 + static_cast<size_t>(n) * 32) + 4 +
             (c->repair_cap > 0 ? P : 0);
  return e;
}

void ctx_release(tbr_ctx* c) {
  cudaStream_t st = c->last_stream;
  dfree(c->packed, st); dfree(c->probs, st); dfree(c->palette, st);
  dfree(c->s0, st); dfree(c->s0b, st); dfree(c->ckpt, st); dfree(c->ck_lt, st);
  dfree(c->rec, st); dfree(c->rec_i, st);
  dfree(c->status, st); dfree(c->partial, st); dfree(c->grad8, st);
  dfree(c->repair_list, st); dfree(c->repair_count, st); dfree(c->corr, st); dfree(c->repair_first, st);
}

cudaError_t ctx_forward(tbr_ctx* c, const tbr_program* prog, float tau, float tau_min, float* out_rgb,
                        cudaStream_t st) {
  c->last_stream = st;
  for (int i = 0; i < 3; ++i) c->bg[i] = prog->background[i];
  c->inv_tc = 1.0f / prog->color_temp;
  cudaError_t e = cudaMemsetAsync(c->status, 0, ST_COUNT * sizeof(unsigned long long), st);
  if (e == cudaSuccess && c->k > 0)
    e = cudaMemcpyAsync(c->palette, prog->palette, static_cast<size_t>(c->k) * 12, cudaMemcpyDeviceToDevice, st);
  PackArgs pa{prog, c->n, tau, tau_min, 0, c->packed, c->probs, c->status};
  if (e == cudaSuccess) e = launch_pack(pa, st);
  SoftArgs sa;
  sa.packed = c->packed; sa.n = c->n; sa.W = c->W; sa.H = c->H;
  for (int i = 0; i < 3; ++i) sa.bg[i] = c->bg[i];
  sa.inert = c->inert; sa.ck_every = c->ck; sa.cap = c->cap;
  sa.transport = c->coupled ? kTransportCoupled : kTransportCapsule;
  sa.out_rgb = out_rgb; sa.s0 = c->s0; sa.s0b = c->s0b; sa.ckpt = c->ckpt; sa.ck_lt = c->ck_lt;
  sa.rec = c->rec; sa.rec_i = c->rec_i; sa.status = c->status;
  if (e == cudaSuccess) e = launch_soft(sa, st);
  return e;
}

cudaError_t ctx_backward(tbr_ctx* c, const float* dLdR, float* g_cx, float* g_cy, float* g_th,
                         float* g_len, float* g_r, float* g_logits, float* g_pal, cudaStream_t st) {
  c->last_stream = st;
  if (c->n == 0) {
    if (g_pal) return cudaMemsetAsync(g_pal, 0, static_cast<size_t>(c->k) * 12, st);
    return cudaSuccess;
  }
  BwdArgs ba;
  ba.packed = c->packed; ba.n = c->n; ba.W = c->W; ba.H = c->H;
  for (int i = 0; i < 3; ++i) ba.bg[i] = c->bg[i];
  ba.inert = c->inert; ba.ck_every = c->ck; ba.cap = c->cap;
  ba.s0 = c->s0; ba.s0b = c->s0b; ba.ckpt = c->ckpt; ba.ck_lt = c->ck_lt;
  ba.rec = c->rec; ba.rec_i = c->rec_i; ba.dLdR = dLdR;
  ba.partial = c->partial; ba.grid = c->grid; ba.status = c->status;
  ba.drift_tol = c->drift_tol;
  ba.repair_list = c->repair_list; ba.repair_count = c->repair_count; ba.repair_cap = c->repair_cap;
  ba.corr = c->corr; ba.repair_first = c->repair_first;
  ba.tile_drift = c->repair_first ? c->repair_first + static_cast<size_t>(c->W) * c->H : nullptr;
  ba.coupled = c->coupled;
  cudaError_t e = launch_backward(ba, st);
  if (e != cudaSuccess) return e;
  EpilogueArgs ea;
  ea.partial = c->partial; ea.grid = c->grid; ea.n = c->n; ea.k = c->k;
  ea.packed = c->packed; ea.probs = c->probs; ea.palette = c->palette; ea.inv_color_temp = c->inv_tc;
  ea.grad8 = c->grad8;
  ea.g_cx = g_cx; ea.g_cy = g_cy; ea.g_th = g_th; ea.g_len = g_len; ea.g_r = g_r;
  ea.g_logits = g_logits; ea.g_pal = g_pal; ea.status = c->status;
  if (c->repair_cap > 0) {
    ea.corr = c->corr; ea.repair_count = c->repair_count; ea.repair_cap = c->repair_cap;
  }
  return launch_backward_epilogue(ea, st);
}

tbr_status ctx_read_status(tbr_ctx* c, unsigned long long host[ST_COUNT]) {
  TBR_CUDA(cudaMemcpyAsync(host, c->status, ST_COUNT * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           c->last_stream),
           "reading context status");
  TBR_CUDA(cudaStreamSynchronize(c->last_stream), "synchronising context stream");
  if (host[ST_INVALID]) return fail(TBR_ERR_INVALID_ARG, "%llu strokes failed the value checks", host[ST_INVALID]);
  if (host[ST_OVERFLOW])
    return fail(TBR_ERR_OVERFLOW, "%llu pixels exceeded the side-table capacity %d", host[ST_OVERFLOW], c->cap);
  if (host[ST_TIMEOUT]) return fail(TBR_ERR_TIMEOUT, "a bounded device wait gave up");
  return TBR_OK;
}

}  // namespace tbr

using namespace tbr;

extern "C" {

const char* tbr_last_error(void) { return last_error_text(); }

const char* tbr_version(void) { return "tbr-b300 0.1 (sm_103a)"; }

tbr_status tbr_render_hard(const tbr_program* prog, int32_t W, int32_t H, int32_t n_prefix,
                           int32_t snap, float* out_rgb, int32_t* out_idx, tbr_hard_stats* stats,
                           void* stream) {
  return tbr_render_hard_transport(prog, W, H, n_prefix, snap, TBR_TRANSPORT_CAPSULE, out_rgb, out_idx, stats,
                                   stream);
}

tbr_status tbr_render_hard_transport(const tbr_program* prog, int32_t W, int32_t H, int32_t n_prefix,
                                     int32_t snap, int32_t transport, float* out_rgb, int32_t* out_idx,
                                     tbr_hard_stats* stats, void* stream) {
  if (!prog) return fail(TBR_ERR_INVALID_ARG, "program is NULL");
  if (transport != TBR_TRANSPORT_CAPSULE && transport != TBR_TRANSPORT_DROPS16)
    return fail(TBR_ERR_INVALID_ARG, "unknown transport %d", transport);
  if (prog->coupling && transport != TBR_TRANSPORT_CAPSULE)
    return fail(TBR_ERR_INVALID_ARG, "the coupling variant applies to the capsule transport only");
  const int n = (n_prefix < 0 || n_prefix > prog->n) ? prog->n : n_prefix;
  tbr_status s = check_program(prog, n);
  if (s != TBR_OK) return s;
  if ((s = check_size(W, H)) != TBR_OK) return s;
  if (!out_rgb) return fail(TBR_ERR_INVALID_ARG, "out_rgb is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* packed = nullptr;
  unsigned long long* status = nullptr;
  TBR_CUDA(dalloc(&packed, static_cast<size_t>(n) * kRec, st), "allocating packed strokes");
  cudaError_t e = dalloc(&status, ST_COUNT, st);
  if (e != cudaSuccess) {
    dfree(packed, st);
    return cuda_fail(e, "allocating status");
  }
  e = cudaMemsetAsync(status, 0, ST_COUNT * sizeof(unsigned long long), st);
  PackArgs pa{prog, n, 0.0f, 1.0f, snap ? 1 : 0, packed, nullptr, status};
  if (e == cudaSuccess) e = launch_pack(pa, st);
  if (e == cudaSuccess)
    e = launch_hard(packed, n, W, H, prog->background, out_rgb, out_idx, status, stats != nullptr, st,
                    prog->coupling ? kTransportCoupled : transport);
  unsigned long long host[ST_COUNT] = {0};
  if (e == cudaSuccess && stats) {
    e = cudaMemcpyAsync(host, status, sizeof(host), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  dfree(packed, st);
  dfree(status, st);
  if (e != cudaSuccess) return cuda_fail(e, "tbr_render_hard");
  if (stats) {
    stats->band_steps = static_cast<int64_t>(host[ST_BAND]);
    stats->background_pixels = static_cast<int64_t>(host[ST_BG]);
    stats->visited_steps = static_cast<int64_t>(host[ST_VISITED]);
    if (host[ST_INVALID])
      return fail(TBR_ERR_INVALID_ARG, "%llu strokes failed the value checks", host[ST_INVALID]);
    if (host[ST_TIMEOUT]) return fail(TBR_ERR_TIMEOUT, "a bounded device wait gave up");
  }
  return TBR_OK;
}

tbr_status tbr_render_soft(const tbr_program* prog, int32_t W, int32_t H, const tbr_soft_opts* opts,
                           float* out_rgb, tbr_ctx** ctx, void* stream) {
  tbr_status s = check_program(prog, prog ? prog->n : 0);
  if (s != TBR_OK) return s;
  if ((s = check_size(W, H)) != TBR_OK) return s;
  if (!opts) return fail(TBR_ERR_INVALID_ARG, "opts is NULL");
  if (!out_rgb) return fail(TBR_ERR_INVALID_ARG, "out_rgb is NULL");
  if (!(opts->tau >= 0.0f) || !(opts->tau_min > 0.0f) || !std::isfinite(opts->tau) ||
      !std::isfinite(opts->tau_min))
    return fail(TBR_ERR_INVALID_ARG, "need tau >= 0 and tau_min > 0");
  if (opts->checkpoint_every < 0 || opts->record_capacity < 0)
    return fail(TBR_ERR_INVALID_ARG, "negative checkpoint interval or record capacity");
  if (opts->repair_capacity < 0 || opts->repair_capacity > kRepairMax || !std::isfinite(opts->drift_tolerance))
    return fail(TBR_ERR_INVALID_ARG, "repair capacity outside [0, %d] or non-finite drift tolerance", kRepairMax);
  if (opts->transport != TBR_TRANSPORT_CAPSULE && opts->transport != TBR_TRANSPORT_DROPS16)
    return fail(TBR_ERR_INVALID_ARG, "unknown transport %d", opts->transport);
  if (opts->transport == TBR_TRANSPORT_DROPS16 && (ctx || opts->inert))
    return fail(TBR_ERR_INVALID_ARG, "the sixteen-drop transport renders forward only (no context, not inert)");
  if (!(opts->early_exit >= 0.0f && opts->early_exit < 1.0f))
    return fail(TBR_ERR_INVALID_ARG, "early_exit must be in [0, 1)");
  if (opts->early_exit > 0.0f && ctx)
    return fail(TBR_ERR_INVALID_ARG, "early exit applies to forward-only renders (the adjoint needs every stroke)");
  if (prog->coupling && (opts->inert || opts->transport != TBR_TRANSPORT_CAPSULE))
    return fail(TBR_ERR_INVALID_ARG, "the coupling variant uses the capsule transport (not inert)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int ck = opts->checkpoint_every > 0 ? opts->checkpoint_every : 32;
  const int cap = opts->record_capacity > 0 ? opts->record_capacity : 64;
  const float drift_tol = opts->drift_tolerance > 0.0f ? opts->drift_tolerance : kDriftTol;
  const int repair_cap = opts->repair_capacity > 0 ? opts->repair_capacity : kDefaultRepairCap;
  if (!ctx) {
    // forward only: the packed strokes and the status words are the only scratch
    float* packed = nullptr;
    unsigned long long* status = nullptr;
    TBR_CUDA(dalloc(&packed, static_cast<size_t>(prog->n) * kRec, st), "allocating packed strokes");
    cudaError_t e = dalloc(&status, ST_COUNT, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, ST_COUNT * sizeof(unsigned long long), st);
    PackArgs pa{prog, prog->n, opts->tau, opts->tau_min, 0, packed, nullptr, status};
    if (e == cudaSuccess) e = launch_pack(pa, st);
    SoftArgs sa;
    sa.packed = packed; sa.n = prog->n; sa.W = W; sa.H = H;
    for (int i = 0; i < 3; ++i) sa.bg[i] = prog->background[i];
    sa.inert = opts->inert ? 1 : 0; sa.ck_every = ck; sa.cap = cap;
    sa.transport = prog->coupling ? kTransportCoupled : opts->transport;
    if (opts->early_exit > 0.0f) sa.exit_lt = log2f(opts->early_exit);
    sa.out_rgb = out_rgb; sa.s0 = nullptr; sa.s0b = nullptr; sa.ckpt = nullptr; sa.ck_lt = nullptr;
    sa.rec = nullptr; sa.rec_i = nullptr; sa.status = status;
    if (e == cudaSuccess) e = launch_soft(sa, st);
    dfree(packed, st);
    dfree(status, st);
    if (e != cudaSuccess) return cuda_fail(e, "tbr_render_soft");
    return TBR_OK;
  }
  const int inert = opts->inert ? 1 : 0;
  const int coupled = prog->coupling ? 1 : 0;
  tbr_ctx* c = *ctx;
  if (c) {
    // reuse an existing context of the same shape: no allocation
    if (c->n != prog->n || c->k != prog->k || c->W != W || c->H != H || c->ck != ck || c->cap != cap ||
        c->inert != inert || c->coupled != coupled || c->repair_cap != ((inert || coupled) ? 0 : repair_cap))
      return fail(TBR_ERR_INVALID_ARG,
                  "context shape differs from this call (n, k, W, H, k_ckpt, capacity, inert, coupling, "
                  "repair capacity)");
    c->drift_tol = drift_tol;
    TBR_CUDA(ctx_forward(c, prog, opts->tau, opts->tau_min, out_rgb, st), "tbr_render_soft");
    return TBR_OK;
  }
  c = new tbr_ctx();
  cudaError_t e = ctx_allocate(c, prog->n, prog->k, W, H, ck, cap, inert, drift_tol, repair_cap, st, coupled);
  if (e == cudaSuccess) e = ctx_forward(c, prog, opts->tau, opts->tau_min, out_rgb, st);
  if (e != cudaSuccess) {
    ctx_release(c);
    delete c;
    return cuda_fail(e, "tbr_render_soft");
  }
  *ctx = c;
  return TBR_OK;
}

tbr_status tbr_render_backward(tbr_ctx* c, const float* dL_drgb, float* g_cx, float* g_cy, float* g_theta,
                               float* g_length, float* g_half_width, float* g_logits, float* g_palette,
                               void* stream) {
  if (!c) return fail(TBR_ERR_INVALID_ARG, "ctx is NULL");
  if (!dL_drgb) return fail(TBR_ERR_INVALID_ARG, "dL_drgb is NULL");
  if (c->n > 0 && (!g_cx || !g_cy || !g_theta || !g_length || !g_half_width || !g_logits))
    return fail(TBR_ERR_INVALID_ARG, "NULL gradient output");
  TBR_CUDA(ctx_backward(c, dL_drgb, g_cx, g_cy, g_theta, g_length, g_half_width, g_logits, g_palette,
                        static_cast<cudaStream_t>(stream)),
           "tbr_render_backward");
  return TBR_OK;
}

tbr_status tbr_ctx_status(tbr_ctx* c, tbr_ctx_stats* stats) {
  if (!c) return fail(TBR_ERR_INVALID_ARG, "ctx is NULL");
  unsigned long long host[ST_COUNT] = {0};
  const tbr_status s = ctx_read_status(c, host);
  if (stats) {
    stats->records = static_cast<int64_t>(host[ST_RECORDS]);
    stats->max_records = static_cast<int64_t>(host[ST_MAXREC]);
    stats->overflow_pixels = static_cast<int64_t>(host[ST_OVERFLOW]);
    stats->drift_resets = static_cast<int64_t>(host[ST_DRIFT]);
    stats->timeouts = static_cast<int64_t>(host[ST_TIMEOUT]);
    stats->invalid_params = static_cast<int64_t>(host[ST_INVALID]);
    stats->repaired_pixels = static_cast<int64_t>(host[ST_REPAIRED]);
    stats->repair_overflow = static_cast<int64_t>(host[ST_REPAIR_OVF]);
  }
  return s;
}

size_t tbr_ctx_bytes(const tbr_ctx* c) { return c ? c->bytes : 0; }

void tbr_ctx_destroy(tbr_ctx* c) {
  if (!c) return;
  ctx_release(c);
  delete c;
}

tbr_status tbr_loss_mse(const float* rgb, const float* target, int64_t n_pixels, float* loss_out,
                        float* dL_drgb, void* stream) {
  if (!rgb || !target || !loss_out) return fail(TBR_ERR_INVALID_ARG, "NULL argument");
  if (n_pixels <= 0) return fail(TBR_ERR_INVALID_ARG, "n_pixels must be positive");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nb = loss_blocks(n_pixels);
  double* partial = nullptr;
  TBR_CUDA(dalloc(&partial, static_cast<size_t>(nb), st), "allocating loss partials");
  cudaError_t e = launch_loss(rgb, target, n_pixels, partial, nb, loss_out, dL_drgb, st);
  dfree(partial, st);
  if (e != cudaSuccess) return cuda_fail(e, "tbr_loss_mse");
  return TBR_OK;
}

}  // extern "C"
