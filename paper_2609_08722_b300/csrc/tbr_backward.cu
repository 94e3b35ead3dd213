// Replay adjoint of the soft render (Sec. 5.2).  Per pixel, for i = 1..N:
//   x_i = Phi_i(x_{i-1})                   (Eq. rpos; Eq. fwd)
//         or the side-table record (i, x_i) where the forward's floor bound
//         (Lemma "Support of the replay record"),
//         or the position checkpoint every k strokes;
//   log T_i = log T_{i-1} - log(1 - alpha_i) (Eq. rT), or the checkpoint;
//   the adjoint step and the parameter gradients (Eq. adjstep, Eq. adjparam).
// The pixel-level work is one thread per pixel on a persistent grid; each CTA
// walks its tiles one after another, streaming the packed strokes first-to-last
// through a two-deep shared-memory ring (1-D bulk TMA).  The 8 per-stroke
// gradient values (cx, cy, theta, L, r, and the colour gradient) are reduced
// over the warp by a reduce-scatter of shuffles, over the CTA through shared
// memory, and written to the CTA's own slice of a partial buffer (no atomics);
// an epilogue sums the slices in a fixed order, so the result is reproducible.
#include <math.h>

#include "tbr_internal.cuh"

namespace tbr {

namespace {

constexpr int kBwdCH = 32;  // kBwdCH * 8 == blockDim.x: one partial per thread per chunk
constexpr int kTileW = 32, kTileH = 8;
constexpr int kBwdThreads = 256;

// d alpha path only (psi = id, inert-mark model): cotangent of sigma' pushed
// back to (x, theta, L, r).
__device__ __forceinline__ void inert_vjp(float s, float h, const StrokeF& g, float& sp_out, float& lamx,
                                          float& lamy, float mua, float z, bool want, float& gcx, float& gcy,
                                          float& gth, float& gL, float& gr) {
  const float as = fabsf(s), ah = fabsf(h);
  const float d = as - g.hl;
  const bool cap = d > 0.0f;
  const float sp = cap ? sqrt_a(fmaf(d, d, ah * ah)) : ah;
  sp_out = sp;
  if (!want) return;
  const float g_sp = -mua * g.iw;
  gr = mua * fmaf(-z, g.dlw, g.iw);
  float g_as = 0.0f, g_ah = g_sp, g_hl = 0.0f;
  if (cap && sp > 0.0f) {
    const float inv = rcp_a(sp);
    g_as = g_sp * d * inv;
    g_ah = g_sp * ah * inv;
    g_hl = -g_as;
  }
  gL = 0.5f * g_hl;
  const float GS = copysignf(1.0f, s) * g_as, GH = copysignf(1.0f, h) * g_ah;
  const float nx = fmaf(GS, g.ex, -GH * g.ey);
  const float ny = fmaf(GS, g.ey, GH * g.ex);
  gcx = -nx;
  gcy = -ny;
  gth = fmaf(GS, h, -GH * s);
  lamx += nx;
  lamy += ny;
}

template <int CH, bool INERT>
__global__ void __launch_bounds__(kBwdThreads, 4) k_backward(BwdArgs a) {
  static_assert(CH * 8 == kBwdThreads, "one partial per thread per chunk");
  __shared__ __align__(128) float sbuf[2 * CH * kRec];
  __shared__ __align__(8) uint64_t sbar[2];
  __shared__ float red[2][kBwdThreads / 32][CH * 8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int W = a.W, H = a.H, n = a.n, ck = a.ck_every;
  const int tiles_x = (W + kTileW - 1) / kTileW;
  const int ntiles = tiles_x * ((H + kTileH - 1) / kTileH);
  const int G = gridDim.x;
  const size_t P = static_cast<size_t>(W) * H;
  unsigned long long* status = a.status;
  const bool skip = status[ST_INVALID] != 0ull || status[ST_OVERFLOW] != 0ull;
  const int nch = (n + CH - 1) / CH;
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / G + 1 : 0;
  const int total = my_tiles * nch;

  ChunkRing<CH> ring;
  ring.init(sbuf, sbar);
  auto chunk_of = [&](int q) { return q % nch; };
  auto chunk_cnt = [&](int q) { return min(CH, n - chunk_of(q) * CH); };
  auto chunk_src = [&](int q) { return a.packed + static_cast<size_t>(chunk_of(q)) * CH * kRec; };
  if (threadIdx.x == 0) {
    if (total > 0) ring.issue(0, chunk_src(0), chunk_cnt(0));
    if (total > 1) ring.issue(1, chunk_src(1), chunk_cnt(1));
  }

  // per-pixel state (positions are hi/lo pairs)
  bool valid = false;
  size_t p = 0;
  float xh = 0.0f, yh = 0.0f, xl = 0.0f, yl = 0.0f, lt = 0.0f;
  float lC0 = 0.0f, lC1 = 0.0f, lC2 = 0.0f, lT = 0.0f, lx = 0.0f, ly = 0.0f;
  int rc = 0, nri = -1, next_ck = 0;
  float4 rpos = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  unsigned drift = 0;

  bool aborted = false;
  for (int q = 0; q < total; ++q) {
    const int b = q & 1;
    const int chunk = chunk_of(q);
    if (chunk == 0) {
      const int tile = blockIdx.x + (q / nch) * G;
      const int px = (tile % tiles_x) * kTileW + lane;
      const int py = (tile / tiles_x) * kTileH + warp;
      valid = px < W && py < H && !skip;
      p = valid ? static_cast<size_t>(py) * W + px : 0;
      if (valid) {
        const float4 s0 = a.s0[p];
        const float2 s0b = a.s0b[p];
        xh = s0.x; yh = s0.y; xl = s0.z; yl = s0.w; lt = s0b.x;
        rc = min(__float_as_int(s0b.y), a.cap);
        lC0 = a.dLdR[3 * p + 0]; lC1 = a.dLdR[3 * p + 1]; lC2 = a.dLdR[3 * p + 2];
        lT = fmaf(lC0, a.bg[0], fmaf(lC1, a.bg[1], lC2 * a.bg[2]));
        lx = 0.0f; ly = 0.0f;
        nri = -1;
        if (rc > 0) {
          const size_t o = static_cast<size_t>(rc - 1) * P + p;
          rpos = a.rec[o];
          nri = a.rec_i[o];
        }
        next_ck = (ck < n) ? ck : 0;
      }
    }
    if (!ring.wait(b, status)) aborted = true;
    if (__syncthreads_or(aborted)) {
      if (q + 1 < total) ring.wait(b ^ 1, status);
      break;
    }
    const int cntc = chunk_cnt(q);
    const float* S0 = ring.data(b);
    float (*rb)[CH * 8] = red[b];
    for (int j = 0; j < cntc; ++j) {
      const int i1 = chunk * CH + j + 1;
      float v[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      if (valid) {
        const float* S = S0 + j * kRec;
        const StrokeF g = load_stroke(S);
        const float cR = S[F_CR], cG = S[F_CG], cB = S[F_CB];
        const bool at_ck = (i1 == next_ck);
        size_t cko = 0;
        if (at_ck) {
          next_ck = (next_ck + ck < n) ? next_ck + ck : 0;
          cko = static_cast<size_t>(i1 / ck - 1) * P + p;
        }
        const float lCc = fmaf(lC0, cR, fmaf(lC1, cG, lC2 * cB));
        if (INERT) {
          float s, h, sp;
          to_frame(xh, yh, xl, yl, g, s, h);
          float d0, d1, d2, d3, d4;
          inert_vjp(s, h, g, sp, lx, ly, 0.0f, 0.0f, false, d0, d1, d2, d3, d4);
          const Cover cv = coverage(sp, g);
          if (at_ck) lt = a.ck_lt[cko]; else lt += cv.sp2;
          const float T = ex2_a(lt);
          const float mu = T * (lCc - lT);
          const float Ta = T * cv.alpha;
          v[5] = lC0 * Ta; v[6] = lC1 * Ta; v[7] = lC2 * Ta;
          inert_vjp(s, h, g, sp, lx, ly, mu * cv.dadz, cv.z, true, v[0], v[1], v[2], v[3], v[4]);
          lT = fmaf(cv.oma, lT, cv.alpha * lCc);
        } else {
          Geo gq;
          float s, h, ds, dh;
          if (i1 == nri) {
            // x_i was inside the floor's reach: read it back (Lemma "Support of the replay record")
            xh = rpos.x; yh = rpos.y; xl = rpos.z; yl = rpos.w;
            to_frame(xh, yh, xl, yl, g, s, h);
            psi_local<true>(s, h, g, gq, ds, dh);
            --rc;
            nri = -1;
            if (rc > 0) {
              const size_t o = static_cast<size_t>(rc - 1) * P + p;
              rpos = a.rec[o];
              nri = a.rec_i[o];
            }
          } else if (at_ck) {
            // regenerate, measure the drift against the stored position, then reset to it
            to_frame(xh, yh, xl, yl, g, s, h);
            phi_local(s, h, g, gq, ds, dh);
            add_frame_disp(xh, yh, xl, yl, g, ds, dh);
            const float4 c = a.ckpt[cko];
            if (fabsf((xh - c.x) + (xl - c.z)) > kDriftTol || fabsf((yh - c.y) + (yl - c.w)) > kDriftTol) ++drift;
            xh = c.x; yh = c.y; xl = c.z; yl = c.w;
            to_frame(xh, yh, xl, yl, g, s, h);
            psi_local<true>(s, h, g, gq, ds, dh);
          } else {
            // x_i = Phi_i(x_{i-1}) (Eq. rpos)
            to_frame(xh, yh, xl, yl, g, s, h);
            phi_local(s, h, g, gq, ds, dh);
            add_frame_disp(xh, yh, xl, yl, g, ds, dh);
          }
          const Cover cv = coverage(gq.sp, g);
          if (at_ck) lt = a.ck_lt[cko]; else lt += cv.sp2;
          const float T = ex2_a(lt);
          const float mu = T * (lCc - lT);
          const float Ta = T * cv.alpha;
          v[5] = lC0 * Ta; v[6] = lC1 * Ta; v[7] = lC2 * Ta;
          step_vjp(gq, g, lx, ly, mu * cv.dadz, cv.z, v[0], v[1], v[2], v[3], v[4]);
          lT = fmaf(cv.oma, lT, cv.alpha * lCc);
        }
      }
      const float r = warp_reduce8(v);
      if ((lane & 3) == 0) rb[warp][j * 8 + ((lane >> 2) & 7)] = r;
    }
    __syncthreads();
    if (threadIdx.x == 0 && q + 2 < total) ring.issue(b, chunk_src(q + 2), chunk_cnt(q + 2));
    const int t = threadIdx.x;
    if (t < cntc * 8) {
      float s = 0.0f;
#pragma unroll
      for (int w = 0; w < kBwdThreads / 32; ++w) s += rb[w][t];
      float* dst = a.partial + (static_cast<size_t>(blockIdx.x) * n + static_cast<size_t>(chunk) * CH) * 8 + t;
      *dst = (q < nch) ? s : *dst + s;
    }
  }
  const unsigned dsum = __reduce_add_sync(0xffffffffu, drift);
  if (lane == 0 && dsum) atomicAdd(status + ST_DRIFT, static_cast<unsigned long long>(dsum));
}

// grad8[t] = sum over CTAs g (in order) of partial[g][t], carried in FP64.
__global__ void k_grad_sum(const float* __restrict__ partial, int G, int n8, float* __restrict__ grad8) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n8) return;
  double s = 0.0;
  for (int g = 0; g < G; ++g) s += static_cast<double>(partial[static_cast<size_t>(g) * n8 + t]);
  grad8[t] = static_cast<float>(s);
}

// Per stroke: geometry gradients, and the colour chain rule
// dc_i/dz_iq = p_iq (Pal_q - c_i) / tau_c for the logits.
__global__ void k_grad_out(EpilogueArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const bool bad = a.status[ST_INVALID] != 0ull || a.status[ST_OVERFLOW] != 0ull ||
                   a.status[ST_TIMEOUT] != 0ull;
  const float nan = __int_as_float(0x7fc00000);
  const float* g8 = a.grad8 + static_cast<size_t>(i) * 8;
  a.g_cx[i] = bad ? nan : g8[0];
  a.g_cy[i] = bad ? nan : g8[1];
  a.g_th[i] = bad ? nan : g8[2];
  a.g_len[i] = bad ? nan : g8[3];
  a.g_r[i] = bad ? nan : g8[4];
  const float* R = a.packed + static_cast<size_t>(i) * kRec;
  const float c0 = R[F_CR], c1 = R[F_CG], c2 = R[F_CB];
  for (int q = 0; q < a.k; ++q) {
    const float* pal = a.palette + 3 * q;
    const float d = fmaf(pal[0] - c0, g8[5], fmaf(pal[1] - c1, g8[6], (pal[2] - c2) * g8[7]));
    a.g_logits[static_cast<size_t>(i) * a.k + q] =
        bad ? nan : a.probs[static_cast<size_t>(i) * a.k + q] * d * a.inv_color_temp;
  }
}

// dL/dPal_q[c] = sum_i p_iq dL/dc_i[c]; one block per (q, c), FP64 block sum.
__global__ void k_grad_palette(EpilogueArgs a) {
  const int qc = blockIdx.x;
  const int q = qc / 3, c = qc % 3;
  double s = 0.0;
  for (int i = threadIdx.x; i < a.n; i += blockDim.x)
    s += static_cast<double>(a.probs[static_cast<size_t>(i) * a.k + q]) *
         static_cast<double>(a.grad8[static_cast<size_t>(i) * 8 + 5 + c]);
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const bool bad = a.status[ST_INVALID] != 0ull || a.status[ST_OVERFLOW] != 0ull ||
                     a.status[ST_TIMEOUT] != 0ull;
    a.g_pal[qc] = bad ? __int_as_float(0x7fc00000) : static_cast<float>(sh[0]);
  }
}

}  // namespace

int backward_grid(int W, int H) {
  static int per_sm = -1, sms = 0;
  if (per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward<kBwdCH, false>, kBwdThreads, 0) !=
            cudaSuccess || per_sm < 1)
      per_sm = 1;
  }
  const int tiles = ((W + kTileW - 1) / kTileW) * ((H + kTileH - 1) / kTileH);
  const int g0 = per_sm * sms;
  const int waves = (tiles + g0 - 1) / g0;
  return (tiles + waves - 1) / waves;
}

cudaError_t launch_backward(const BwdArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  KernelTimer kt(TBR_K_BACKWARD, st);
  if (a.inert) k_backward<kBwdCH, true><<<a.grid, kBwdThreads, 0, st>>>(a);
  else k_backward<kBwdCH, false><<<a.grid, kBwdThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_backward_epilogue(const EpilogueArgs& a, cudaStream_t st) {
  if (a.n <= 0) {
    return cudaSuccess;
  }
  const int n8 = a.n * 8;
  KernelTimer kt(TBR_K_EPILOGUE, st);
  k_grad_sum<<<(n8 + 255) / 256, 256, 0, st>>>(a.partial, a.grid, n8, a.grad8);
  k_grad_out<<<(a.n + 127) / 128, 128, 0, st>>>(a);
  if (a.g_pal) k_grad_palette<<<a.k * 3, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace tbr
