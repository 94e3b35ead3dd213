// C ABI of the TBR library (include/tbr.h): argument checks, stream-ordered
// device memory for scratch and replay contexts, and kernel launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "tbr_internal.cuh"

using namespace tbr;

namespace {

thread_local std::string g_last_error = "no error";

tbr_status fail(tbr_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

tbr_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(TBR_ERR_OOM, "%s: out of device memory", what);
  return fail(TBR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define TBR_CUDA(call, what)                       \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count, cudaStream_t st) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  return cudaMallocAsync(reinterpret_cast<void**>(p), count * sizeof(T), st);
}
template <class T>
void dfree(T*& p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
  p = nullptr;
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

tbr_status check_size(int32_t W, int32_t H) {
  if (W <= 0 || H <= 0) return fail(TBR_ERR_INVALID_ARG, "image size %dx%d must be positive", W, H);
  if (static_cast<int64_t>(W) * H > (int64_t(1) << 30))
    return fail(TBR_ERR_INVALID_ARG, "image of %dx%d pixels is too large", W, H);
  return TBR_OK;
}

}  // namespace

struct tbr_ctx {
  int n = 0, k = 0, W = 0, H = 0, ck = 32, cap = 64, inert = 0, grid = 0;
  float bg[3] = {0, 0, 0};
  float inv_tc = 1.0f;
  float* packed = nullptr;
  float* probs = nullptr;
  float* palette = nullptr;
  float4* s0 = nullptr;
  float4* ckpt = nullptr;
  float4* rec = nullptr;
  unsigned long long* status = nullptr;
  float* partial = nullptr;
  float* grad8 = nullptr;
  cudaStream_t create_stream = nullptr;
  cudaStream_t last_stream = nullptr;
  size_t bytes = 0;
};

namespace {

void ctx_free(tbr_ctx* c) {
  cudaStream_t st = c->last_stream;
  dfree(c->packed, st); dfree(c->probs, st); dfree(c->palette, st);
  dfree(c->s0, st); dfree(c->ckpt, st); dfree(c->rec, st);
  dfree(c->status, st); dfree(c->partial, st); dfree(c->grad8, st);
}

}  // namespace

extern "C" {

const char* tbr_last_error(void) { return g_last_error.c_str(); }

const char* tbr_version(void) { return "tbr-b300 0.1 (sm_103a)"; }

tbr_status tbr_render_hard(const tbr_program* prog, int32_t W, int32_t H, int32_t n_prefix,
                           int32_t snap, float* out_rgb, int32_t* out_idx, tbr_hard_stats* stats,
                           void* stream) {
  if (!prog) return fail(TBR_ERR_INVALID_ARG, "program is NULL");
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
  if (e != cudaSuccess) { dfree(packed, st); return cuda_fail(e, "allocating status"); }
  e = cudaMemsetAsync(status, 0, ST_COUNT * sizeof(unsigned long long), st);
  PackArgs pa{prog, n, 0.0f, 1.0f, snap ? 1 : 0, packed, nullptr, status};
  if (e == cudaSuccess) e = launch_pack(pa, st);
  if (e == cudaSuccess) e = launch_hard(packed, n, W, H, prog->background, out_rgb, out_idx, status,
                                        stats != nullptr, st);
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
    if (host[ST_INVALID]) return fail(TBR_ERR_INVALID_ARG, "%llu strokes failed the value checks", host[ST_INVALID]);
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
  if (ctx) *ctx = nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = prog->n, k = prog->k;
  const size_t P = static_cast<size_t>(W) * H;
  tbr_ctx* c = new tbr_ctx();
  c->n = n; c->k = k; c->W = W; c->H = H;
  c->ck = opts->checkpoint_every > 0 ? opts->checkpoint_every : 32;
  c->cap = opts->record_capacity > 0 ? opts->record_capacity : 64;
  c->inert = opts->inert ? 1 : 0;
  for (int i = 0; i < 3; ++i) c->bg[i] = prog->background[i];
  c->inv_tc = 1.0f / prog->color_temp;
  c->create_stream = st;
  c->last_stream = st;
  const bool record = ctx != nullptr;
  const size_t nck = (record && n > 1) ? static_cast<size_t>((n - 1) / c->ck) : 0;
  cudaError_t e = dalloc(&c->packed, static_cast<size_t>(n) * kRec, st);
  if (e == cudaSuccess) e = dalloc(&c->status, ST_COUNT, st);
  if (record) {
    c->grid = backward_grid(W, H);
    if (e == cudaSuccess) e = dalloc(&c->probs, static_cast<size_t>(n) * k, st);
    if (e == cudaSuccess) e = dalloc(&c->palette, static_cast<size_t>(k) * 3, st);
    if (e == cudaSuccess) e = dalloc(&c->s0, P, st);
    if (e == cudaSuccess) e = dalloc(&c->ckpt, nck * P, st);
    if (e == cudaSuccess && !c->inert) e = dalloc(&c->rec, static_cast<size_t>(c->cap) * P, st);
    if (e == cudaSuccess) e = dalloc(&c->partial, static_cast<size_t>(c->grid) * n * 8, st);
    if (e == cudaSuccess) e = dalloc(&c->grad8, static_cast<size_t>(n) * 8, st);
  }
  c->bytes = static_cast<size_t>(n) * kRec * 4 + ST_COUNT * 8;
  if (record)
    c->bytes += static_cast<size_t>(n) * k * 4 + k * 12 + P * 16 + nck * P * 16 +
                (c->inert ? 0 : static_cast<size_t>(c->cap) * P * 16) +
                static_cast<size_t>(c->grid) * n * 32 + static_cast<size_t>(n) * 32;
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, ST_COUNT * sizeof(unsigned long long), st);
  if (e == cudaSuccess && record)
    e = cudaMemcpyAsync(c->palette, prog->palette, static_cast<size_t>(k) * 12, cudaMemcpyDeviceToDevice, st);
  PackArgs pa{prog, n, opts->tau, opts->tau_min, 0, c->packed, c->probs, c->status};
  if (e == cudaSuccess) e = launch_pack(pa, st);
  SoftArgs sa;
  sa.packed = c->packed; sa.n = n; sa.W = W; sa.H = H;
  for (int i = 0; i < 3; ++i) sa.bg[i] = prog->background[i];
  sa.inert = c->inert; sa.ck_every = c->ck; sa.cap = c->cap;
  sa.out_rgb = out_rgb; sa.s0 = c->s0; sa.ckpt = c->ckpt; sa.rec = c->rec; sa.status = c->status;
  if (e == cudaSuccess) e = launch_soft(sa, st);
  if (e != cudaSuccess || !record) {
    ctx_free(c);
    delete c;
    if (e != cudaSuccess) return cuda_fail(e, "tbr_render_soft");
    return TBR_OK;
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
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  c->last_stream = st;
  if (c->n == 0) {
    if (g_palette) TBR_CUDA(cudaMemsetAsync(g_palette, 0, static_cast<size_t>(c->k) * 12, st), "memset");
    return TBR_OK;
  }
  BwdArgs ba;
  ba.packed = c->packed; ba.n = c->n; ba.W = c->W; ba.H = c->H;
  for (int i = 0; i < 3; ++i) ba.bg[i] = c->bg[i];
  ba.inert = c->inert; ba.ck_every = c->ck; ba.cap = c->cap;
  ba.s0 = c->s0; ba.ckpt = c->ckpt; ba.rec = c->rec; ba.dLdR = dL_drgb;
  ba.partial = c->partial; ba.grid = c->grid; ba.status = c->status;
  TBR_CUDA(launch_backward(ba, st), "launching the replay adjoint");
  EpilogueArgs ea;
  ea.partial = c->partial; ea.grid = c->grid; ea.n = c->n; ea.k = c->k;
  ea.packed = c->packed; ea.probs = c->probs; ea.palette = c->palette; ea.inv_color_temp = c->inv_tc;
  ea.grad8 = c->grad8;
  ea.g_cx = g_cx; ea.g_cy = g_cy; ea.g_th = g_theta; ea.g_len = g_length; ea.g_r = g_half_width;
  ea.g_logits = g_logits; ea.g_pal = g_palette; ea.status = c->status;
  TBR_CUDA(launch_backward_epilogue(ea, st), "launching the gradient epilogue");
  return TBR_OK;
}

tbr_status tbr_ctx_status(tbr_ctx* c, tbr_ctx_stats* stats) {
  if (!c) return fail(TBR_ERR_INVALID_ARG, "ctx is NULL");
  unsigned long long host[ST_COUNT] = {0};
  TBR_CUDA(cudaMemcpyAsync(host, c->status, sizeof(host), cudaMemcpyDeviceToHost, c->last_stream),
           "reading context status");
  TBR_CUDA(cudaStreamSynchronize(c->last_stream), "synchronising context stream");
  if (stats) {
    stats->records = static_cast<int64_t>(host[ST_RECORDS]);
    stats->max_records = static_cast<int64_t>(host[ST_MAXREC]);
    stats->overflow_pixels = static_cast<int64_t>(host[ST_OVERFLOW]);
    stats->drift_resets = static_cast<int64_t>(host[ST_DRIFT]);
    stats->timeouts = static_cast<int64_t>(host[ST_TIMEOUT]);
    stats->invalid_params = static_cast<int64_t>(host[ST_INVALID]);
  }
  if (host[ST_INVALID]) return fail(TBR_ERR_INVALID_ARG, "%llu strokes failed the value checks", host[ST_INVALID]);
  if (host[ST_OVERFLOW])
    return fail(TBR_ERR_OVERFLOW, "%llu pixels exceeded the side-table capacity %d", host[ST_OVERFLOW], c->cap);
  if (host[ST_TIMEOUT]) return fail(TBR_ERR_TIMEOUT, "a bounded device wait gave up");
  return TBR_OK;
}

size_t tbr_ctx_bytes(const tbr_ctx* c) { return c ? c->bytes : 0; }

void tbr_ctx_destroy(tbr_ctx* c) {
  if (!c) return;
  ctx_free(c);
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
