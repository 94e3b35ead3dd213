// Hard render (Sec. 3, Eq. chain and Eq. render with alpha = indicator of the
// closed footprint K_i).  One thread per pixel, a CTA per 32x8 pixel tile; the
// packed strokes stream through shared memory in chunks of CH records by 1-D
// bulk TMA (cp.async.bulk + mbarrier), last chunk first, and every thread reads
// the current stroke as a shared-memory broadcast.  A pixel stops at the first
// footprint that contains it; the CTA stops when all its pixels have.
#include <math.h>

#include "tbr_internal.cuh"

namespace tbr {

namespace {

constexpr int kHardCH = 64;
constexpr int kTileW = 32, kTileH = 8;

// Membership test and psi (Eq. back) recomputed in FP64 from the hi/lo
// position, used where |sigma' - r| < kBand.  Returns true if the point is inside.
__device__ __noinline__ bool hard_step_f64(float& xh, float& yh, float& xl, float& yl,
                                           const float* __restrict__ S) {
  const double* D = reinterpret_cast<const double*>(S + F_D64);
  const double mx = D[0], my = D[1], ex = D[2], ey = D[3], hl = D[4], r = D[5];
  const double L = 2.0 * hl;
  const double x = static_cast<double>(xh) + static_cast<double>(xl);
  const double y = static_cast<double>(yh) + static_cast<double>(yl);
  const double dx = x - mx, dy = y - my;
  const double s = dx * ex + dy * ey, h = dy * ex - dx * ey;
  const double as = fabs(s), ah = fabs(h), d = as - hl;
  const bool cap = d > 0.0;
  const double sp = cap ? sqrt(d * d + ah * ah) : ah;
  if (sp <= r) return true;
  const double C = (sp - r) * (2.0 * L + kPiD * (sp + r));
  const double sig = C / (L + sqrt(L * L + kPiD * C));
  const double Qp = L + kPiD * sp, Q = L + kPiD * sig;
  const double t = cap ? hl + sp * atan2(d, ah) : as;
  const double tn = t * (Q / Qp);
  double sn, hn;
  if (tn <= hl) {
    sn = tn; hn = sig;
  } else {
    double sb, cb;
    sincos((tn - hl) / sig, &sb, &cb);
    sn = hl + sig * sb; hn = sig * cb;
  }
  sn = copysign(sn, s); hn = copysign(hn, h);
  const double xo = mx + sn * ex - hn * ey, yo = my + sn * ey + hn * ex;
  xh = static_cast<float>(xo); xl = static_cast<float>(xo - static_cast<double>(xh));
  yh = static_cast<float>(yo); yl = static_cast<float>(yo - static_cast<double>(yh));
  return false;
}

// One stroke of the hard chain in FP32.  Returns true if x lies in K_i;
// otherwise moves x to psi_i(x) (displacement form, hi/lo position).
__device__ __forceinline__ bool hard_step(float& xh, float& yh, float& xl, float& yl,
                                          const float* __restrict__ S, unsigned& band) {
  const StrokeF g = load_stroke(S);
  float s, h;
  to_frame(xh, yh, xl, yl, g, s, h);
  const float as = fabsf(s), ah = fabsf(h);
  const float d = as - g.hl;
  const float sp = d > 0.0f ? sqrt_a(fmaf(d, d, ah * ah)) : ah;
  const float diff = sp - g.r;
  if (fabsf(diff) < kBand) {
    ++band;
    return hard_step_f64(xh, yh, xl, yl, S);
  }
  if (diff <= 0.0f) return true;
  Geo q;
  float ds, dh;
  psi_local<false>(s, h, g, q, ds, dh);
  add_frame_disp(xh, yh, xl, yl, g, ds, dh);
  return false;
}

template <int CH>
__global__ void __launch_bounds__(256) k_hard(const float* __restrict__ packed, int n, int W, int H,
                                              float bg0, float bg1, float bg2,
                                              float* __restrict__ out_rgb, int* __restrict__ out_idx,
                                              unsigned long long* __restrict__ status, int want_stats) {
  __shared__ __align__(128) float sbuf[2 * CH * kRec];
  __shared__ __align__(8) uint64_t sbar[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_x = (W + kTileW - 1) / kTileW;
  const int px = (blockIdx.x % tiles_x) * kTileW + lane;
  const int py = (blockIdx.x / tiles_x) * kTileH + warp;
  const bool valid = px < W && py < H;
  const bool invalid_prog = status[ST_INVALID] != 0ull;
  bool alive = valid && !invalid_prog;
  float xh = (static_cast<float>(px) + 0.5f) / static_cast<float>(W);
  float yh = (static_cast<float>(py) + 0.5f) / static_cast<float>(H);
  float xl = 0.0f, yl = 0.0f;
  int hit = -1;
  unsigned band = 0, visited = 0;

  ChunkRing<CH> ring;
  ring.init(sbuf, sbar);
  const int nch = (n + CH - 1) / CH;
  // iteration q consumes chunk nch-1-q (strokes are visited last to first)
  auto chunk_src = [&](int q) { return packed + static_cast<size_t>(nch - 1 - q) * CH * kRec; };
  auto chunk_cnt = [&](int q) { const int base = (nch - 1 - q) * CH; return min(CH, n - base); };
  if (threadIdx.x == 0) {
    if (nch > 0) ring.issue(0, chunk_src(0), chunk_cnt(0));
    if (nch > 1) ring.issue(1, chunk_src(1), chunk_cnt(1));
  }
  bool aborted = false;
  for (int q = 0; q < nch; ++q) {
    const int b = q & 1;
    if (!ring.wait(b, status)) aborted = true;
    if (__syncthreads_or(aborted)) {
      if (q + 1 < nch) ring.wait(b ^ 1, status);
      alive = false;
      break;
    }
    const int base = (nch - 1 - q) * CH;
    const int cnt = chunk_cnt(q);
    const float* S0 = ring.data(b);
    if (alive) {
      for (int j = cnt - 1; j >= 0; --j) {
        ++visited;
        if (hard_step(xh, yh, xl, yl, S0 + j * kRec, band)) {
          hit = base + j;
          alive = false;
          break;
        }
      }
    }
    const bool any = __syncthreads_or(alive);
    if (!any) {
      if (q + 1 < nch) ring.wait(b ^ 1, status);  // drain the prefetched chunk
      break;
    }
    if (threadIdx.x == 0 && q + 2 < nch) ring.issue(b, chunk_src(q + 2), chunk_cnt(q + 2));
  }

  if (valid) {
    const size_t p = static_cast<size_t>(py) * W + px;
    float c0 = bg0, c1 = bg1, c2 = bg2;
    if (invalid_prog || aborted) {
      c0 = c1 = c2 = __int_as_float(0x7fc00000);
    } else if (hit >= 0) {
      const float* R = packed + static_cast<size_t>(hit) * kRec;
      c0 = R[F_CR]; c1 = R[F_CG]; c2 = R[F_CB];
    }
    out_rgb[3 * p + 0] = c0;
    out_rgb[3 * p + 1] = c1;
    out_rgb[3 * p + 2] = c2;
    if (out_idx) out_idx[p] = hit;
  }
  if (want_stats) {
    const unsigned bsum = __reduce_add_sync(0xffffffffu, band);
    const unsigned vsum = __reduce_add_sync(0xffffffffu, visited);
    const unsigned bgs = __reduce_add_sync(0xffffffffu, (valid && hit < 0) ? 1u : 0u);
    if (lane == 0) {
      if (bsum) atomicAdd(status + ST_BAND, static_cast<unsigned long long>(bsum));
      if (vsum) atomicAdd(status + ST_VISITED, static_cast<unsigned long long>(vsum));
      if (bgs) atomicAdd(status + ST_BG, static_cast<unsigned long long>(bgs));
    }
  }
}

}  // namespace

cudaError_t launch_hard(const float* packed, int n, int W, int H, const float bg[3], float* out_rgb,
                        int* out_idx, unsigned long long* status, int want_stats, cudaStream_t st) {
  const int tiles = ((W + kTileW - 1) / kTileW) * ((H + kTileH - 1) / kTileH);
  KernelTimer kt(TBR_K_HARD, st);
  k_hard<kHardCH><<<tiles, 256, 0, st>>>(packed, n, W, H, bg[0], bg[1], bg[2], out_rgb, out_idx,
                                         status, want_stats);
  return cudaGetLastError();
}

}  // namespace tbr
