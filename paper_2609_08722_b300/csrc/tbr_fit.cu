// Fit step (Sec. 5.1 inverse rendering; Table "hyper"): one Adam iteration on
// the stroke parameters of a program against a target image.  A step runs the
// soft forward with the replay record at the annealed relaxation tau_t and
// colour temperature tau_c,t (Eq. relax; geometric schedules), the pixel MSE
// and its adjoint seed, the replay adjoint (Sec. 5.2), the length regulariser
// lambda sum_i L_i of Eq. inverse, and an Adam update with cosine step decay
// and projection onto the feasible set (0 <= L <= L_max, r in a per-stroke
// window [lo r0, hi r0], centres on the canvas, palette in [0,1]).
#include <cmath>
#include <cstring>

#include "tbr_host.h"

struct tbr_fit {
  tbr_fit_config cfg;
  int n = 0, k = 0, W = 0, H = 0, iter = 0;
  float bg[3] = {1, 1, 1};
  float tau_min = 0.0f;
  size_t nparam = 0;
  float* params = nullptr;   // [5n | n k | 3k]: cx cy theta L r, logits, palette
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* rlo = nullptr;      // [n]
  float* rhi = nullptr;      // [n]
  float* target = nullptr;   // [P][3]
  float* scal = nullptr;     // [2]: MSE, sum of lengths
  float* host = nullptr;     // pinned [2]
  float* coupling = nullptr; // [n][3] the coupling variant's fixed profile, or NULL (capsule map)
  tbr::FusedWork work;       // loss-fused forward + replay adjoint buffers
  cudaStream_t last_stream = nullptr;
};

namespace tbr {
namespace {

constexpr int kAdamThreads = 256;

struct AdamStep {
  float lr[7];       // cx, cy, theta, L, r, logits, palette (cosine-scaled)
  float b1, b2, eps, bc1, bc2;
  float lambda_len, len_max;
  int n, k, train_palette;
};

__global__ void k_adam(float* __restrict__ params, const float* __restrict__ grads, float* __restrict__ m,
                       float* __restrict__ v, const float* __restrict__ rlo, const float* __restrict__ rhi,
                       AdamStep s, const unsigned long long* __restrict__ status) {
  if (status[ST_INVALID] | status[ST_OVERFLOW] | status[ST_TIMEOUT]) return;  // keep the step
  const size_t n = s.n, nk = static_cast<size_t>(s.n) * s.k;
  const size_t total = 5 * n + nk + (s.train_palette ? 3 * static_cast<size_t>(s.k) : 0);
  const size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= total) return;
  int grp;
  size_t idx = e;
  if (e < 5 * n) { grp = static_cast<int>(e / n); idx = e % n; }
  else if (e < 5 * n + nk) grp = 5;
  else grp = 6;
  float g = grads[e];
  if (grp == 3) g += s.lambda_len;  // d(lambda sum L)/dL
  const float mm = fmaf(s.b1, m[e], (1.0f - s.b1) * g);
  const float vv = fmaf(s.b2, v[e], (1.0f - s.b2) * g * g);
  m[e] = mm;
  v[e] = vv;
  float p = params[e] - s.lr[grp] * (mm / s.bc1) / (sqrtf(vv / s.bc2) + s.eps);
  if (grp == 0 || grp == 1) p = fminf(fmaxf(p, 0.0f), 1.0f);
  else if (grp == 3) p = fminf(fmaxf(p, 0.0f), s.len_max);
  else if (grp == 4) p = fminf(fmaxf(p, rlo[idx]), rhi[idx]);
  else if (grp == 6) p = fminf(fmaxf(p, 0.0f), 1.0f);
  params[e] = p;
}

__global__ void k_length_sum(const float* __restrict__ L, int n, float* __restrict__ out) {
  __shared__ float sh[256];
  float acc = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += L[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

__global__ void k_width_window(const float* __restrict__ r0, int n, float lo, float hi, float* __restrict__ rlo,
                               float* __restrict__ rhi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { rlo[i] = lo * r0[i]; rhi[i] = hi * r0[i]; }
}

tbr_program view_of(const tbr_fit* f, float color_temp) {
  tbr_program p{};
  const size_t n = f->n;
  p.n = f->n; p.k = f->k;
  p.cx = f->params; p.cy = f->params + n; p.theta = f->params + 2 * n;
  p.length = f->params + 3 * n; p.half_width = f->params + 4 * n;
  p.logits = f->params + 5 * n;
  p.palette = f->params + 5 * n + n * f->k;
  for (int c = 0; c < 3; ++c) p.background[c] = f->bg[c];
  p.color_temp = color_temp;
  p.coupling = f->coupling;
  return p;
}

float geometric(float a, float b, int t, int T) {
  if (T <= 1) return b;
  return a * std::pow(b / a, static_cast<float>(t) / static_cast<float>(T - 1));
}

void fit_free(tbr_fit* f, cudaStream_t st) {
  f->work.release(st);
  dfree(f->params, st); dfree(f->grads, st); dfree(f->m, st); dfree(f->v, st);
  dfree(f->rlo, st); dfree(f->rhi, st); dfree(f->target, st); dfree(f->scal, st); dfree(f->coupling, st);
  if (f->host) cudaFreeHost(f->host);
  f->host = nullptr;
}

}  // namespace
}  // namespace tbr

using namespace tbr;

extern "C" {

void tbr_fit_default_config(tbr_fit_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->iterations = 240;
  c->tau_start = 0.35f; c->tau_end = 0.02f; c->tau_min = 0.0f;
  c->color_temp_start = 1.0f; c->color_temp_end = 0.05f;
  c->lr_center = 2e-3f; c->lr_angle = 1e-2f; c->lr_length = 2e-3f; c->lr_width = 5e-4f;
  c->lr_logits = 3e-2f; c->lr_palette = 1e-2f;
  c->beta1 = 0.9f; c->beta2 = 0.999f; c->adam_eps = 1e-8f;
  c->length_max = 0.30f;
  c->width_lo = 0.6f; c->width_hi = 1.7f;
  c->length_weight = 3e-4f;
  c->train_palette = 0;
  c->checkpoint_every = 64;
  c->record_capacity = 64;
}

tbr_status tbr_fit_create(const tbr_program* init, const float* target, int32_t W, int32_t H,
                          const tbr_fit_config* cfg, tbr_fit** out, void* stream) {
  if (!out) return fail(TBR_ERR_INVALID_ARG, "fit handle pointer is NULL");
  *out = nullptr;
  tbr_status s = check_program(init, init ? init->n : 0);
  if (s != TBR_OK) return s;
  if ((s = check_size(W, H)) != TBR_OK) return s;
  if (!target) return fail(TBR_ERR_INVALID_ARG, "target is NULL");
  tbr_fit_config c;
  if (cfg) c = *cfg; else tbr_fit_default_config(&c);
  if (c.iterations < 1 || !(c.tau_start > 0) || !(c.tau_end > 0) || !(c.color_temp_start > 0) ||
      !(c.color_temp_end > 0) || !(c.length_max > 0) || !(c.width_lo > 0) || !(c.width_hi >= c.width_lo) ||
      c.checkpoint_every < 0 || c.record_capacity < 0)
    return fail(TBR_ERR_INVALID_ARG, "invalid fit configuration");
  if (c.checkpoint_every == 0) c.checkpoint_every = 64;
  if (c.record_capacity == 0) c.record_capacity = 64;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tbr_fit* f = new tbr_fit();
  f->cfg = c;
  f->n = init->n; f->k = init->k; f->W = W; f->H = H;
  for (int i = 0; i < 3; ++i) f->bg[i] = init->background[i];
  f->tau_min = c.tau_min > 0 ? c.tau_min : 0.7f / static_cast<float>(W > H ? W : H);
  const size_t n = f->n, k = f->k, P = static_cast<size_t>(W) * H;
  f->nparam = 5 * n + n * k + 3 * k;
  f->last_stream = st;
  cudaError_t e = dalloc(&f->params, f->nparam, st);
  if (e == cudaSuccess) e = dalloc(&f->grads, f->nparam, st);
  if (e == cudaSuccess) e = dalloc(&f->m, f->nparam, st);
  if (e == cudaSuccess) e = dalloc(&f->v, f->nparam, st);
  if (e == cudaSuccess) e = dalloc(&f->rlo, n, st);
  if (e == cudaSuccess) e = dalloc(&f->rhi, n, st);
  if (e == cudaSuccess) e = dalloc(&f->target, 3 * P, st);
  if (e == cudaSuccess) e = dalloc(&f->scal, 2, st);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&f->host), 2 * sizeof(float));
  if (e == cudaSuccess && init->coupling && n > 0) {
    // the profile is an input of the program, kept fixed while the fit trains the rest
    e = dalloc(&f->coupling, 3 * n, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->coupling, init->coupling, 3 * n * 4, cudaMemcpyDeviceToDevice, st);
  }
  if (e == cudaSuccess)
    e = f->work.allocate(f->n, f->k, W, H, c.checkpoint_every, c.record_capacity, st, kDriftTol, kDefaultRepairCap,
                         f->coupling ? 1 : 0);
  const float* src[5] = {init->cx, init->cy, init->theta, init->length, init->half_width};
  for (int g = 0; g < 5 && e == cudaSuccess && n > 0; ++g)
    e = cudaMemcpyAsync(f->params + g * n, src[g], n * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && n > 0)
    e = cudaMemcpyAsync(f->params + 5 * n, init->logits, n * k * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(f->params + 5 * n + n * k, init->palette, k * 12, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->target, target, 12 * P, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->m, 0, f->nparam * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->v, 0, f->nparam * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->grads, 0, f->nparam * 4, st);
  if (e == cudaSuccess && n > 0) {
    k_width_window<<<(f->n + 255) / 256, 256, 0, st>>>(init->half_width, f->n, c.width_lo, c.width_hi,
                                                         f->rlo, f->rhi);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    fit_free(f, st);
    delete f;
    return cuda_fail(e, "tbr_fit_create");
  }
  *out = f;
  return TBR_OK;
}

tbr_status tbr_fit_step(tbr_fit* f, float* loss_out, void* stream) {
  if (!f) return fail(TBR_ERR_INVALID_ARG, "fit is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const tbr_fit_config& c = f->cfg;
  const int T = c.iterations, t = f->iter < T ? f->iter : T - 1;
  const float tau = geometric(c.tau_start, c.tau_end, t, T);
  const float tc = geometric(c.color_temp_start, c.color_temp_end, t, T);
  const float cosine = 0.5f * (1.0f + std::cos(3.14159265358979f * static_cast<float>(t) / static_cast<float>(T)));
  const size_t n = f->n, k = f->k;
  f->last_stream = st;
  for (int attempt = 0; attempt < 4; ++attempt) {
    const tbr_program view = view_of(f, tc);
    float* g = f->grads;
    TBR_CUDA(f->work.run(&view, tau, f->tau_min, f->target, nullptr, f->scal, g, g + n, g + 2 * n, g + 3 * n,
                         g + 4 * n, g + 5 * n, c.train_palette ? g + 5 * n + n * k : nullptr, st),
             "fit: loss-fused forward + replay adjoint");
    if (n > 0) k_length_sum<<<1, 256, 0, st>>>(f->params + 3 * n, f->n, f->scal + 1);
    AdamStep as;
    const float lr[7] = {c.lr_center, c.lr_center, c.lr_angle, c.lr_length, c.lr_width, c.lr_logits,
                         c.lr_palette};
    for (int i = 0; i < 7; ++i) as.lr[i] = lr[i] * cosine;
    as.b1 = c.beta1; as.b2 = c.beta2; as.eps = c.adam_eps;
    as.bc1 = 1.0f - std::pow(c.beta1, static_cast<float>(f->iter + 1));
    as.bc2 = 1.0f - std::pow(c.beta2, static_cast<float>(f->iter + 1));
    as.lambda_len = c.length_weight; as.len_max = c.length_max;
    as.n = f->n; as.k = f->k; as.train_palette = c.train_palette;
    const size_t total = 5 * n + n * k + (c.train_palette ? 3 * k : 0);
    {
      KernelTimer kt(TBR_K_UPDATE, st);
      if (total > 0)
        k_adam<<<static_cast<unsigned>((total + kAdamThreads - 1) / kAdamThreads), kAdamThreads, 0, st>>>(
            f->params, f->grads, f->m, f->v, f->rlo, f->rhi, as, f->work.status);
    }
    TBR_CUDA(cudaGetLastError(), "fit: update");
    unsigned long long host[ST_COUNT];
    TBR_CUDA(cudaMemcpyAsync(f->host, f->scal, 2 * sizeof(float), cudaMemcpyDeviceToHost, st), "fit: loss copy");
    TBR_CUDA(cudaMemcpyAsync(host, f->work.status, sizeof(host), cudaMemcpyDeviceToHost, st), "fit: status copy");
    TBR_CUDA(cudaStreamSynchronize(st), "fit: synchronise");
    if (host[ST_OVERFLOW]) {
      // the update was skipped on the device; grow the side table and redo the step
      const int cap = f->work.cap * 2;
      f->work.release(st);
      TBR_CUDA(f->work.allocate(f->n, f->k, f->W, f->H, c.checkpoint_every, cap, st, kDriftTol, kDefaultRepairCap,
                                f->coupling ? 1 : 0),
               "fit: growing the side table");
      continue;
    }
    if (host[ST_INVALID]) return fail(TBR_ERR_INVALID_ARG, "%llu strokes failed the value checks", host[ST_INVALID]);
    if (host[ST_TIMEOUT]) return fail(TBR_ERR_TIMEOUT, "a bounded device wait gave up");
    if (loss_out) *loss_out = f->host[0] + c.length_weight * (n > 0 ? f->host[1] : 0.0f);
    ++f->iter;
    return TBR_OK;
  }
  return fail(TBR_ERR_OVERFLOW, "side table kept overflowing");
}

tbr_status tbr_fit_get_program(const tbr_fit* f, tbr_program* view) {
  if (!f || !view) return fail(TBR_ERR_INVALID_ARG, "NULL argument");
  const tbr_fit_config& c = f->cfg;
  const int T = c.iterations, t = f->iter < T ? f->iter : T - 1;
  *view = view_of(f, geometric(c.color_temp_start, c.color_temp_end, t, T));
  return TBR_OK;
}

int32_t tbr_fit_iteration(const tbr_fit* f) { return f ? f->iter : -1; }

void tbr_fit_destroy(tbr_fit* f) {
  if (!f) return;
  fit_free(f, f->last_stream);
  delete f;
}

}  // extern "C"
