// Loss-fused soft forward + replay adjoint (Sec. 5.1 objective, Sec. 5.2
// adjoint) for the case where the image loss is the pixel MSE against a target:
// the adjoint seed lambda^C_0 = 2 (R - I*) / (3P) is pixel-local, so each tile
// runs its soft forward (writing the replay record into the CTA's own scratch,
// which stays in L2), seeds, and immediately runs the replay adjoint.  Grid and
// reductions are those of the plain adjoint: persistent CTAs, one gradient
// slice per CTA, fixed-order sums; the loss is summed per CTA in FP64.
#include "tbr_host.h"
#include "tbr_tile.cuh"

namespace tbr {

namespace {

constexpr int kFusedCH = 32;

template <int CH>
__global__ void __launch_bounds__(kTileThreads, 4) k_fused_mse(FusedArgs a) {
  __shared__ __align__(128) float sbuf[2 * CH * kRec];
  __shared__ __align__(8) uint64_t sbar[2];
  __shared__ float red[2][kTileThreads / 32][CH * 8];
  __shared__ double lsum[kTileThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int W = a.W, H = a.H, n = a.n;
  const int ntiles = ((W + kTileW - 1) / kTileW) * ((H + kTileH - 1) / kTileH);
  unsigned long long* status = a.status;
  const bool skip = status[ST_INVALID] != 0ull;
  ChunkRing<CH> ring;
  ring.init(sbuf, sbar);
  const size_t nck = n > 1 ? static_cast<size_t>((n - 1) / a.ck) : 0;
  const size_t cta = blockIdx.x;
  RecordView rv{a.rec + cta * a.cap * kTileThreads, a.rec_i + cta * a.cap * kTileThreads,
                a.ckpt + cta * nck * kTileThreads, a.ck_lt + cta * nck * kTileThreads,
                static_cast<size_t>(kTileThreads), static_cast<size_t>(threadIdx.x), a.cap, a.ck};
  float* slice = a.partial + cta * n * 8;
  double lacc = 0.0;
  unsigned drift = 0, recs = 0, maxrec = 0, ovf = 0;
  bool first = true;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int px, py;
    tile_pixel(tile, W, px, py);
    const bool valid = px < W && py < H && !skip;
    const size_t p = valid ? static_cast<size_t>(py) * W + px : 0;
    PixelState st;
    if (!soft_forward_tile<CH, true, false>(ring, a.packed, n, valid,
                                            (static_cast<float>(px) + 0.5f) / static_cast<float>(W),
                                            (static_cast<float>(py) + 0.5f) / static_cast<float>(H), rv, st,
                                            status))
      break;
    float lC0 = 0.0f, lC1 = 0.0f, lC2 = 0.0f;
    if (valid) {
      const float T0 = ex2_a(st.lt);
      const float R0 = fmaf(T0, a.bg[0], st.C0), R1 = fmaf(T0, a.bg[1], st.C1), R2 = fmaf(T0, a.bg[2], st.C2);
      if (a.out_rgb) {
        a.out_rgb[3 * p + 0] = R0;
        a.out_rgb[3 * p + 1] = R1;
        a.out_rgb[3 * p + 2] = R2;
      }
      const float d0 = R0 - a.target[3 * p + 0], d1 = R1 - a.target[3 * p + 1], d2 = R2 - a.target[3 * p + 2];
      lacc += static_cast<double>(d0) * d0 + static_cast<double>(d1) * d1 + static_cast<double>(d2) * d2;
      lC0 = a.seed_scale * d0; lC1 = a.seed_scale * d1; lC2 = a.seed_scale * d2;
      recs += static_cast<unsigned>(st.cnt);
      maxrec = max(maxrec, static_cast<unsigned>(st.cnt));
      if (st.cnt > a.cap) ++ovf;
    }
    if (!backward_tile<CH, false>(ring, a.packed, n, valid, st, lC0, lC1, lC2, a.bg, rv, red, slice, first,
                                  drift, status))
      break;
    first = false;
  }
  // loss partial of this CTA (fixed order: lanes, then warps)
  for (int o = 16; o > 0; o >>= 1) lacc += __shfl_xor_sync(0xffffffffu, lacc, o);
  if (lane == 0) lsum[warp] = lacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kTileThreads / 32; ++w) s += lsum[w];
    a.loss_part[blockIdx.x] = s;
  }
  const unsigned rsum = __reduce_add_sync(0xffffffffu, recs);
  const unsigned rmax = __reduce_max_sync(0xffffffffu, maxrec);
  const unsigned osum = __reduce_add_sync(0xffffffffu, ovf);
  const unsigned dsum = __reduce_add_sync(0xffffffffu, drift);
  if (lane == 0) {
    if (rsum) atomicAdd(status + ST_RECORDS, static_cast<unsigned long long>(rsum));
    if (rmax) atomicMax(status + ST_MAXREC, static_cast<unsigned long long>(rmax));
    if (osum) atomicAdd(status + ST_OVERFLOW, static_cast<unsigned long long>(osum));
    if (dsum) atomicAdd(status + ST_DRIFT, static_cast<unsigned long long>(dsum));
  }
}

}  // namespace

int fused_grid(int W, int H) {
  static int per_sm = -1, sms = 0;
  if (per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_mse<kFusedCH>, kTileThreads, 0) !=
            cudaSuccess || per_sm < 1)
      per_sm = 1;
  }
  const int tiles = ((W + kTileW - 1) / kTileW) * ((H + kTileH - 1) / kTileH);
  const int g0 = per_sm * sms;
  const int waves = (tiles + g0 - 1) / g0;
  return (tiles + waves - 1) / waves;
}

cudaError_t launch_fused(const FusedArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  KernelTimer kt(TBR_K_FUSED, st);
  k_fused_mse<kFusedCH><<<a.grid, kTileThreads, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Work buffers of the fused path (also held by a fit across steps).
// ---------------------------------------------------------------------------
cudaError_t FusedWork::allocate(int n_, int k_, int W_, int H_, int ck_, int cap_, cudaStream_t st) {
  n = n_; k = k_; W = W_; H = H_; ck = ck_; cap = cap_;
  grid = fused_grid(W, H);
  const size_t nck = n > 1 ? static_cast<size_t>((n - 1) / ck) : 0;
  const size_t per = static_cast<size_t>(grid) * kTileThreads;
  cudaError_t e = dalloc(&packed, static_cast<size_t>(n) * kRec, st);
  if (e == cudaSuccess) e = dalloc(&probs, static_cast<size_t>(n) * k, st);
  if (e == cudaSuccess) e = dalloc(&palette, static_cast<size_t>(k) * 3, st);
  if (e == cudaSuccess) e = dalloc(&status, ST_COUNT, st);
  if (e == cudaSuccess) e = dalloc(&rec, static_cast<size_t>(cap) * per, st);
  if (e == cudaSuccess) e = dalloc(&rec_i, static_cast<size_t>(cap) * per, st);
  if (e == cudaSuccess) e = dalloc(&ckpt, nck * per, st);
  if (e == cudaSuccess) e = dalloc(&ck_lt, nck * per, st);
  if (e == cudaSuccess) e = dalloc(&partial, static_cast<size_t>(grid) * n * 8, st);
  if (e == cudaSuccess) e = dalloc(&grad8, static_cast<size_t>(n) * 8, st);
  if (e == cudaSuccess) e = dalloc(&loss_part, static_cast<size_t>(grid), st);
  bytes = static_cast<size_t>(n) * kRec * 4 + static_cast<size_t>(n) * k * 4 + k * 12 + ST_COUNT * 8 +
          static_cast<size_t>(cap) * per * 20 + nck * per * 20 + static_cast<size_t>(grid) * n * 32 +
          static_cast<size_t>(n) * 32 + static_cast<size_t>(grid) * 8;
  return e;
}

void FusedWork::release(cudaStream_t st) {
  dfree(packed, st); dfree(probs, st); dfree(palette, st); dfree(status, st);
  dfree(rec, st); dfree(rec_i, st); dfree(ckpt, st); dfree(ck_lt, st);
  dfree(partial, st); dfree(grad8, st); dfree(loss_part, st);
}

cudaError_t FusedWork::run(const tbr_program* prog, float tau, float tau_min, const float* target, float* out_rgb,
                           float* loss_out, float* g_cx, float* g_cy, float* g_th, float* g_len, float* g_r,
                           float* g_logits, float* g_pal, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(status, 0, ST_COUNT * sizeof(unsigned long long), st);
  if (e == cudaSuccess && k > 0)
    e = cudaMemcpyAsync(palette, prog->palette, static_cast<size_t>(k) * 12, cudaMemcpyDeviceToDevice, st);
  PackArgs pa{prog, n, tau, tau_min, 0, packed, probs, status};
  if (e == cudaSuccess) e = launch_pack(pa, st);
  const int64_t P = static_cast<int64_t>(W) * H;
  FusedArgs fa;
  fa.packed = packed; fa.n = n; fa.W = W; fa.H = H;
  for (int i = 0; i < 3; ++i) fa.bg[i] = prog->background[i];
  fa.ck = ck; fa.cap = cap; fa.target = target; fa.out_rgb = out_rgb;
  fa.rec = rec; fa.rec_i = rec_i; fa.ckpt = ckpt; fa.ck_lt = ck_lt;
  fa.partial = partial; fa.loss_part = loss_part; fa.grid = grid;
  fa.seed_scale = 2.0f / static_cast<float>(3 * P);
  fa.status = status;
  if (e == cudaSuccess) e = launch_fused(fa, st);
  if (e == cudaSuccess && n > 0) {
    EpilogueArgs ea;
    ea.partial = partial; ea.grid = grid; ea.n = n; ea.k = k;
    ea.packed = packed; ea.probs = probs; ea.palette = palette; ea.inv_color_temp = 1.0f / prog->color_temp;
    ea.grad8 = grad8;
    ea.g_cx = g_cx; ea.g_cy = g_cy; ea.g_th = g_th; ea.g_len = g_len; ea.g_r = g_r;
    ea.g_logits = g_logits; ea.g_pal = g_pal; ea.status = status;
    e = launch_backward_epilogue(ea, st);
  } else if (e == cudaSuccess && g_pal) {
    e = cudaMemsetAsync(g_pal, 0, static_cast<size_t>(k) * 12, st);
  }
  if (e == cudaSuccess && loss_out) e = launch_loss_final(loss_part, n > 0 ? grid : 0, 3 * P, loss_out, st);
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
  if (opts->checkpoint_every < 0 || opts->record_capacity < 0)
    return fail(TBR_ERR_INVALID_ARG, "negative checkpoint interval or record capacity");
  if (prog->n > 0 && (!g_cx || !g_cy || !g_theta || !g_length || !g_half_width || !g_logits))
    return fail(TBR_ERR_INVALID_ARG, "NULL gradient output");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FusedWork w;
  cudaError_t e = w.allocate(prog->n, prog->k, W, H, opts->checkpoint_every > 0 ? opts->checkpoint_every : 64,
                             opts->record_capacity > 0 ? opts->record_capacity : 64, st);
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
    if (host[ST_INVALID]) return fail(TBR_ERR_INVALID_ARG, "%llu strokes failed the value checks", host[ST_INVALID]);
    if (host[ST_OVERFLOW]) return fail(TBR_ERR_OVERFLOW, "%llu pixels exceeded the side-table capacity", host[ST_OVERFLOW]);
    if (host[ST_TIMEOUT]) return fail(TBR_ERR_TIMEOUT, "a bounded device wait gave up");
  }
  return TBR_OK;
}

}  // extern "C"
