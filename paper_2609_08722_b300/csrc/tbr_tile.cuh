// Per-tile device routines shared by the soft forward, the replay adjoint, the
// loss-fused forward+adjoint kernel and the serving kernel.  A tile is 32x8
// pixels, one pixel per thread (a warp = 32 consecutive pixels of one row);
// strokes stream through the CTA's two-deep shared-memory ring (ChunkRing).
#pragma once

#include "tbr_internal.cuh"

namespace tbr {

constexpr int kTileW = 32, kTileH = 8, kTileThreads = 256;
// Tiles of the soft kernels that carry two pixels per thread (32 x 16).
constexpr int kPairTileW = 32, kPairTileH = 16;
__host__ __device__ inline int tile_count(int W, int H) {
  return ((W + kTileW - 1) / kTileW) * ((H + kTileH - 1) / kTileH);
}
__host__ __device__ inline int pair_tile_count(int W, int H) {
  return ((W + kPairTileW - 1) / kPairTileW) * ((H + kPairTileH - 1) / kPairTileH);
}

// Where one pixel's replay record lives: element (slot, pixel) of each array is
// at slot * stride + off.  The plain kernels use [slot][P] with off = pixel;
// the fused kernels use a per-CTA scratch [slot][256] with off = threadIdx.x.
struct RecordView {
  float4* rec;     // side table positions (hi/lo), `cap` slots
  int* rec_i;      // side table stroke indices (1-based)
  float4* ckpt;    // checkpoints at i = ck, 2ck, ... (< n)
  float* ck_lt;    // log2 T at the checkpoints
  size_t stride;
  size_t off;
  int cap, ck;
  float drift_tol = kDriftTol;  // checkpoint drift that marks a segment for the FP64 repair
  int2* repair_list = nullptr;  // [repair_cap] (pixel, segment start) of drifting pixels, or NULL
  int* repair_count = nullptr;  // entries appended (may exceed repair_cap)
  int repair_cap = 0;
  unsigned char* repair_first = nullptr;  // [P] 1 once the pixel is queued (zeroed per adjoint)
};

// State of one pixel after the soft forward (s_0 of Eq. state plus the colour).
struct PixelState {
  float xh, yh, xl, yl;  // x_0 as a hi/lo pair
  float lt;              // log2 T_0
  int cnt;               // side-table records written (may exceed cap)
  float C0, C1, C2;      // accumulated colour C_0
};

__device__ __forceinline__ void tile_pixel(int tile, int W, int& px, int& py) {
  const int tiles_x = (W + kTileW - 1) / kTileW;
  px = (tile % tiles_x) * kTileW + (threadIdx.x & 31);
  py = (tile / tiles_x) * kTileH + (threadIdx.x >> 5);
}

// Soft forward (Eq. relax, Eq. state, floored psi) of one pixel per thread over
// strokes n-1 .. 0.  With RECORD, pushes (x_i, i) for floored samples and
// stores (x_i, log2 T_i) every ck strokes.  With EXIT (forward only), a pixel
// stops once log2 T < exit_lt after compositing a stroke (the early exit of the
// forward render) and the CTA once all its pixels have.  All threads of the CTA
// must call it.  Returns false if a bounded wait gave up (the status word is set).
template <int CH, bool RECORD, bool INERT, bool DROPS = false, bool COUPLED = false, bool EXIT = false>
__device__ bool soft_forward_tile(ChunkRing<CH>& ring, const float* __restrict__ packed, int n, bool valid,
                                  float x0, float y0, const RecordView& rv, PixelState& st,
                                  unsigned long long* status, float exit_lt = -3.0e38f) {
  static_assert(!(DROPS && (RECORD || INERT)), "the sixteen-drop transport renders forward only");
  static_assert(!(COUPLED && (INERT || DROPS)), "the coupling variant uses the capsule transport");
  static_assert(!(EXIT && RECORD), "the early exit applies to forward-only renders");
  st.xh = x0; st.yh = y0; st.xl = 0.0f; st.yl = 0.0f;
  st.lt = 0.0f; st.cnt = 0;
  st.C0 = st.C1 = st.C2 = 0.0f;
  const int ck = rv.ck;
  int next_ck = (RECORD && n > 1) ? ((n - 1) / ck) * ck : 0;  // largest checkpoint index < n
  const int nch = (n + CH - 1) / CH;
  auto chunk_src = [&](int q) { return packed + static_cast<size_t>(nch - 1 - q) * CH * kRec; };
  auto chunk_cnt = [&](int q) { return min(CH, n - (nch - 1 - q) * CH); };
  if (threadIdx.x == 0) {
    if (nch > 0) ring.issue(0, chunk_src(0), chunk_cnt(0));
    if (nch > 1) ring.issue(1, chunk_src(1), chunk_cnt(1));
  }
  bool ok = true;
  bool live = valid;  // false once the pixel has taken its early exit (EXIT)
  for (int q = 0; q < nch; ++q) {
    const int b = q & 1;
    const bool got = ring.wait(b, status);
    if (__syncthreads_or(!got)) {
      if (q + 1 < nch) ring.wait(b ^ 1, status);
      ok = false;
      break;
    }
    const int base = (nch - 1 - q) * CH;
    const int cntc = chunk_cnt(q);
    const float* S0 = ring.data(b);
    if (live) {
      // one stroke (j: index in the chunk); true once the pixel took its early exit
      auto stroke = [&](int j) -> bool {
        const int i1 = base + j + 1;  // the paper's 1-based stroke index
        const float* S = S0 + j * kRec;
        const StrokeF g = load_stroke(S);
        float sp, rb = g.r, ds = 0.0f, dh = 0.0f, ddx = 0.0f, ddy = 0.0f;
        bool floored = false;
        const bool drop = g.L == 0.0f;  // warp-uniform
        if (DROPS) {
          // capsule coverage; the transport (sixteen drops) is applied after compositing
          float s, h;
          to_frame(st.xh, st.yh, st.xl, st.yl, g, s, h);
          const float as = fabsf(s), ah = fabsf(h);
          const float d = as - g.hl;
          sp = d > 0.0f ? sqrt_a(fmaf(d, d, ah * ah)) : ah;
        } else if (drop && !COUPLED) {
          const float dx = (st.xh - g.mx) + st.xl, dy = (st.yh - g.my) + st.yl;
          if (INERT) sp = sqrt_a(fmaf(dx, dx, dy * dy));
          else sp = drop_step<true>(dx, dy, g, ddx, ddy, floored);
        } else {
          float s, h;
          to_frame(st.xh, st.yh, st.xl, st.yl, g, s, h);
          if (INERT) {
            const float as = fabsf(s), ah = fabsf(h);
            const float d = as - g.hl;
            sp = d > 0.0f ? sqrt_a(fmaf(d, d, ah * ah)) : ah;
          } else {
            Geo q;
            if (COUPLED) {
              psi_local<true, true>(s, h, g, q, ds, dh, *reinterpret_cast<const float4*>(S + F_G0));
              rb = q.rb;
            } else {
              psi_local<true>(s, h, g, q, ds, dh);
            }
            sp = q.sp;
            floored = q.floored;
            ddx = fmaf(ds, g.ex, -dh * g.ey);
            ddy = fmaf(ds, g.ey, dh * g.ex);
          }
        }
        const Cover cv = coverage(sp, rb, g);
        const float w = ex2_a(st.lt) * cv.alpha;
        st.C0 = fmaf(w, S[F_CR], st.C0);
        st.C1 = fmaf(w, S[F_CG], st.C1);
        st.C2 = fmaf(w, S[F_CB], st.C2);
        st.lt -= cv.sp2;
        if (EXIT && st.lt < exit_lt) {
          live = false;
          return true;
        }
        if (DROPS) {
          st.cnt += drops_step(st.xh, st.yh, st.xl, st.yl, g);
        } else if (!INERT) {
          if (RECORD && floored) {
            if (st.cnt < rv.cap) {
              const size_t o = static_cast<size_t>(st.cnt) * rv.stride + rv.off;
              rv.rec[o] = make_float4(st.xh, st.yh, st.xl, st.yl);
              rv.rec_i[o] = i1;
            }
            ++st.cnt;
          }
          st.xl += ddx;
          st.yl += ddy;
        }
        return false;
      };
      auto checkpoint = [&](int i1) {
        const size_t o = static_cast<size_t>(i1 / ck - 1) * rv.stride + rv.off;
        rv.ckpt[o] = make_float4(st.xh, st.yh, st.xl, st.yl);
        rv.ck_lt[o] = st.lt;
        next_ck -= ck;
      };
      // Blocks of kRenorm strokes aligned to the stroke index (base is a multiple
      // of kRenorm): the position is renormalised after each block's last stroke
      // (index = 1 mod kRenorm), and with a checkpoint interval that is a multiple
      // of kRenorm a checkpoint can only fall before a block's first stroke, so
      // neither test runs per stroke.
      const bool ck_aligned = (ck & (kRenorm - 1)) == 0;
      for (int hi = cntc - 1; hi >= 0;) {
        const int lo = hi & ~(kRenorm - 1);
        bool stop = false;
        if (!RECORD || ck_aligned) {
          if (RECORD && base + hi + 1 == next_ck) checkpoint(base + hi + 1);
#pragma unroll 4
          for (int j = hi; j >= lo; --j)
            if (stroke(j)) {
              stop = true;
              break;
            }
        } else {
          for (int j = hi; j >= lo; --j) {
            if (base + j + 1 == next_ck) checkpoint(base + j + 1);
            if (stroke(j)) {
              stop = true;
              break;
            }
          }
        }
        if (stop) break;
        if (!DROPS && !INERT) {
          pos_renorm(st.xh, st.xl);
          pos_renorm(st.yh, st.yl);
        }
        hi = lo - 1;
      }
    }
    if (!EXIT) {
      __syncthreads();
    } else if (!__syncthreads_or(live)) {
      if (q + 1 < nch) ring.wait(b ^ 1, status);  // drain the prefetched chunk
      break;
    }
    if (threadIdx.x == 0 && q + 2 < nch) ring.issue(b, chunk_src(q + 2), chunk_cnt(q + 2));
  }
  return ok;
}

// The record's stroke frame in FP64: m, L/2 and r are exact as floats, e is
// held as doubles (cos and sin of theta in FP64).
struct FrameF64 {
  double mx, my, ex, ey, hl, r;
};
__device__ __forceinline__ FrameF64 frame_f64(const float* __restrict__ S) {
  const double* D = reinterpret_cast<const double*>(S + F_D64);
  return FrameF64{static_cast<double>(S[F_MX]), static_cast<double>(S[F_MY]), D[0], D[1],
                  static_cast<double>(S[F_HL]), static_cast<double>(S[F_R])};
}

// Membership test and psi (Eq. back) recomputed in FP64 from the hi/lo
// position, used where |sigma' - r| < kBand (|sigma' - sigma_b(v)| for the
// coupling variant, whose membership is A_L(sigma') <= A_L(r) g(v), i.e. C <= 0).
// Returns true if the point is inside.  Inlined: as a called function, the
// register saves around the call ran on every step of the hard render's loop.
template <bool COUPLED = false>
static __device__ __forceinline__ bool hard_step_f64(float& xh, float& yh, float& xl, float& yl,
                                           const float* __restrict__ S) {
  const FrameF64 f = frame_f64(S);
  const double mx = f.mx, my = f.my, ex = f.ex, ey = f.ey, hl = f.hl, r = f.r;
  const double L = 2.0 * hl;
  const double x = static_cast<double>(xh) + static_cast<double>(xl);
  const double y = static_cast<double>(yh) + static_cast<double>(yl);
  const double dx = x - mx, dy = y - my;
  const double s = dx * ex + dy * ey, h = dy * ex - dx * ey;
  const double as = fabs(s), ah = fabs(h), d = as - hl;
  const bool cap = d > 0.0;
  const double sp = cap ? sqrt(d * d + ah * ah) : ah;
  if (!COUPLED && sp <= r) return true;
  double C = (sp - r) * (2.0 * L + kPiD * (sp + r));
  const double Qp = L + kPiD * sp;
  const double t = cap ? hl + sp * atan2(d, ah) : as;
  if (COUPLED) {  // Eq. coupling, w = cos 4 pi v = cos(2 pi t / Q')
    const double w = Qp > 0.0 ? cos(2.0 * kPiD * t / Qp) : 1.0;
    const double c1 = S[F_C1], c2 = S[F_C1 + 1], c3 = S[F_C1 + 2];
    const double gm1 = c1 * w + c2 * (2.0 * w * w - 1.0) + c3 * (4.0 * w * w * w - 3.0 * w);
    C -= (2.0 * L * r + kPiD * r * r) * gm1;
    if (C <= 0.0) return true;
  }
  const double sig = C / (L + sqrt(L * L + kPiD * C));
  const double Q = L + kPiD * sig;
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

// x_i = Phi_i(x_{i-1}) in FP64 (Eq. fwd, with the tangential map of Eq. phi)
// from the record's FP64 copy of (m, e, L/2, r): sigma' = B / (L + sqrt(L^2 +
// pi B)), B = 2L(sigma + r) + pi(sigma^2 + r^2); the arclength t from the flank
// midpoint scales by (L + pi sigma') / (L + pi sigma).  Used by the repair of a
// drifting checkpoint segment.
static __device__ __noinline__ void phi_f64(double& x, double& y, const float* __restrict__ S) {
  const FrameF64 f = frame_f64(S);
  const double mx = f.mx, my = f.my, ex = f.ex, ey = f.ey, hl = f.hl, r = f.r;
  const double L = 2.0 * hl;
  const double dx = x - mx, dy = y - my;
  const double s = dx * ex + dy * ey, h = dy * ex - dx * ey;
  const double as = fabs(s), ah = fabs(h), d = as - hl;
  const bool cap = d > 0.0;
  const double sig = cap ? sqrt(d * d + ah * ah) : ah;
  const double B = 2.0 * L * (sig + r) + kPiD * (sig * sig + r * r);
  const double sp = B / (L + sqrt(L * L + kPiD * B));
  const double tn = cap ? hl + sig * atan2(d, ah) : as;
  const double q = L + kPiD * sig;
  const double t = q > 0.0 ? tn * ((L + kPiD * sp) / q) : 0.0;
  double sn, hn;
  if (t <= hl) {
    sn = t; hn = sp;
  } else {
    double sb, cb;
    sincos((t - hl) / sp, &sb, &cb);
    sn = hl + sp * sb; hn = sp * cb;
  }
  sn = copysign(sn, s); hn = copysign(hn, h);
  x = mx + sn * ex - hn * ey;
  y = my + sn * ey + hn * ex;
}

// FP64 membership test of the hard render's band (|sigma' - r| < kBand) for
// the transfer renderer, whose transport is applied in FP32 afterwards.
static __device__ __noinline__ bool hard_member_f64(float xh, float yh, float xl, float yl,
                                                   const float* __restrict__ S) {
  const FrameF64 f = frame_f64(S);
  const double mx = f.mx, my = f.my, ex = f.ex, ey = f.ey, hl = f.hl, r = f.r;
  const double x = static_cast<double>(xh) + static_cast<double>(xl);
  const double y = static_cast<double>(yh) + static_cast<double>(yl);
  const double dx = x - mx, dy = y - my;
  const double as = fabs(dx * ex + dy * ey), ah = fabs(dy * ex - dx * ey), d = as - hl;
  const double sp = d > 0.0 ? sqrt(d * d + ah * ah) : ah;
  return sp <= r;
}

// One stroke of the hard chain in FP32.  Returns true if x lies in K_i;
// otherwise moves x to psi_i(x) (displacement form, hi/lo position).  COUPLED:
// the coupling variant's deposit and map (every stroke through the frame).
template <bool DROPS = false, bool COUPLED = false>
__device__ __forceinline__ bool hard_step(float& xh, float& yh, float& xl, float& yl,
                                          const float* __restrict__ S, unsigned& band) {
  const StrokeF g = load_stroke(S);
  if (COUPLED) {
    float s, h;
    to_frame(xh, yh, xl, yl, g, s, h);
    Geo q;
    float ds, dh;
    psi_local<false, true>(s, h, g, q, ds, dh, *reinterpret_cast<const float4*>(S + F_G0));
    const float diff = q.sp - q.rb;
    if (fabsf(diff) < kBand) {
      ++band;
      return hard_step_f64<true>(xh, yh, xl, yl, S);
    }
    if (diff <= 0.0f) return true;  // (the displacement computed inside K_i is not used)
    add_frame_disp(xh, yh, xl, yl, g, ds, dh);
    return false;
  }
  if (DROPS) {  // capsule membership, then the sixteen-drop pull-back
    float s, h;
    to_frame(xh, yh, xl, yl, g, s, h);
    const float as = fabsf(s), ah = fabsf(h);
    const float d = as - g.hl;
    const float diff = (d > 0.0f ? sqrt_a(fmaf(d, d, ah * ah)) : ah) - g.r;
    bool inside = diff <= 0.0f;
    if (fabsf(diff) < kBand) {
      ++band;
      inside = hard_member_f64(xh, yh, xl, yl, S);
    }
    if (inside) return true;
    drops_step(xh, yh, xl, yl, g);
    return false;
  }
  if (g.L == 0.0f) {  // drop (warp-uniform): radial step in world coordinates
    const float dx = (xh - g.mx) + xl, dy = (yh - g.my) + yl;
    const float rho = sqrt_a(fmaf(dx, dx, dy * dy));
    const float diff = rho - g.r;
    if (fabsf(diff) < kBand) {
      ++band;
      return hard_step_f64(xh, yh, xl, yl, S);
    }
    if (diff <= 0.0f) return true;
    float ddx, ddy;
    bool floored;
    drop_step<false>(dx, dy, g, ddx, ddy, floored);
    pos_add(xh, xl, ddx);
    pos_add(yh, yl, ddy);
    return false;
  }
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

// Hard render of one tile (Eq. chain + Eq. render with the indicator of K_i):
// strokes last to first, each pixel stops at the first footprint containing it,
// the CTA stops when all its pixels have.  Writes colour and index.
// All threads of the CTA must call it.  Returns false if a bounded wait gave up.
template <int CH, bool DROPS = false, bool COUPLED = false>
__device__ bool hard_tile(ChunkRing<CH>& ring, const float* __restrict__ packed, int n, int tile, int W, int H,
                          const float bg[3], bool poison, float* __restrict__ out_rgb, int* __restrict__ out_idx,
                          unsigned& band, unsigned& visited, bool& background, unsigned long long* status) {
  int px, py;
  tile_pixel(tile, W, px, py);
  const bool valid = px < W && py < H;
  bool alive = valid && !poison;
  float xh = (static_cast<float>(px) + 0.5f) / static_cast<float>(W);
  float yh = (static_cast<float>(py) + 0.5f) / static_cast<float>(H);
  float xl = 0.0f, yl = 0.0f;
  int hit = -1;
  const int nch = (n + CH - 1) / CH;
  auto chunk_src = [&](int q) { return packed + static_cast<size_t>(nch - 1 - q) * CH * kRec; };
  auto chunk_cnt = [&](int q) { return min(CH, n - (nch - 1 - q) * CH); };
  if (threadIdx.x == 0) {
    if (nch > 0) ring.issue(0, chunk_src(0), chunk_cnt(0));
    if (nch > 1) ring.issue(1, chunk_src(1), chunk_cnt(1));
  }
  bool ok = true;
  for (int q = 0; q < nch; ++q) {
    const int b = q & 1;
    const bool got = ring.wait(b, status);
    if (__syncthreads_or(!got)) {
      if (q + 1 < nch) ring.wait(b ^ 1, status);
      ok = false;
      break;
    }
    const int base = (nch - 1 - q) * CH;
    const int cnt = chunk_cnt(q);
    const float* S0 = ring.data(b);
    if (alive) {
      for (int j = cnt - 1; j >= 0; --j) {
        ++visited;
        if (hard_step<DROPS, COUPLED>(xh, yh, xl, yl, S0 + j * kRec, band)) {
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
  background = valid && hit < 0;
  if (valid) {
    const size_t p = static_cast<size_t>(py) * W + px;
    float c0 = bg[0], c1 = bg[1], c2 = bg[2];
    if (poison || !ok) {
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
  return ok;
}

// Live-pixel state moved between threads by hard_tile_compact.
struct HardLive {
  float xh[kTileThreads], yh[kTileThreads], xl[kTileThreads], yl[kTileThreads];
  int pix[kTileThreads];
  int warp_base[kTileThreads / 32 + 1];
};

// hard_tile with CTA-wide compaction of the live pixels.  The chain of Eq.
// chain stops at a different stroke for every pixel (a few hundred of 2000 on
// average, all of them for background pixels), so a warp whose pixels mostly
// finished would keep issuing for the few still alive.  After every chunk the
// live pixels (position hi/lo and pixel index) are packed, in pixel order, into
// the first threads of the CTA through shared memory; warps past the live count
// then skip the chunk's strokes.  A pixel's colour and index are written when
// it stops (or, for the background, after the last chunk).  Same arguments and
// results as hard_tile; st is shared scratch.
template <int CH, bool DROPS = false, bool COUPLED = false>
__device__ bool hard_tile_compact(ChunkRing<CH>& ring, const float* __restrict__ packed, int n, int tile, int W,
                                  int H, const float bg[3], bool poison, float* __restrict__ out_rgb,
                                  int* __restrict__ out_idx, HardLive& st, unsigned& band, unsigned& visited,
                                  unsigned& background, unsigned long long* status) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int px, py;
  tile_pixel(tile, W, px, py);
  const bool valid = px < W && py < H;
  int pix = valid ? py * W + px : -1;
  bool alive = valid && !poison;
  float xh = (static_cast<float>(px) + 0.5f) / static_cast<float>(W);
  float yh = (static_cast<float>(py) + 0.5f) / static_cast<float>(H);
  float xl = 0.0f, yl = 0.0f;
  auto write = [&](int p, int hit) {
    float c0 = bg[0], c1 = bg[1], c2 = bg[2];
    if (hit >= 0) {
      const float* R = packed + static_cast<size_t>(hit) * kRec;
      c0 = R[F_CR]; c1 = R[F_CG]; c2 = R[F_CB];
    }
    out_rgb[3 * static_cast<size_t>(p) + 0] = c0;
    out_rgb[3 * static_cast<size_t>(p) + 1] = c1;
    out_rgb[3 * static_cast<size_t>(p) + 2] = c2;
    if (out_idx) out_idx[p] = hit;
  };
  const int nch = (n + CH - 1) / CH;
  auto chunk_src = [&](int q) { return packed + static_cast<size_t>(nch - 1 - q) * CH * kRec; };
  auto chunk_cnt = [&](int q) { return min(CH, n - (nch - 1 - q) * CH); };
  if (threadIdx.x == 0) {
    if (nch > 0) ring.issue(0, chunk_src(0), chunk_cnt(0));
    if (nch > 1) ring.issue(1, chunk_src(1), chunk_cnt(1));
  }
  bool ok = true;
  int live = kTileThreads;  // threads [0, live) may hold a live pixel
  for (int q = 0; q < nch; ++q) {
    const int b = q & 1;
    const bool got = ring.wait(b, status);
    if (__syncthreads_or(!got)) {
      if (q + 1 < nch) ring.wait(b ^ 1, status);
      ok = false;
      break;
    }
    const int base = (nch - 1 - q) * CH;
    const int cnt = chunk_cnt(q);
    const float* S0 = ring.data(b);
    if (alive) {
#pragma unroll 4
      for (int j = cnt - 1; j >= 0; --j) {
        ++visited;
        if (hard_step<DROPS, COUPLED>(xh, yh, xl, yl, S0 + j * kRec, band)) {
          write(pix, base + j);
          alive = false;
          break;
        }
      }
    }
    // pack the live pixels into threads [0, live)
    const unsigned m = __ballot_sync(0xffffffffu, alive);
    if (lane == 0) st.warp_base[warp] = __popc(m);
    __syncthreads();  // every thread is done with the chunk's records here
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int w = 0; w < kTileThreads / 32; ++w) {
        const int c = st.warp_base[w];
        st.warp_base[w] = acc;
        acc += c;
      }
      st.warp_base[kTileThreads / 32] = acc;
      if (acc > 0 && q + 2 < nch) ring.issue(b, chunk_src(q + 2), chunk_cnt(q + 2));
    }
    __syncthreads();
    live = st.warp_base[kTileThreads / 32];
    if (live == 0) {
      if (q + 1 < nch) ring.wait(b ^ 1, status);  // drain the prefetched chunk
      break;
    }
    if (alive) {
      const int d = st.warp_base[warp] + __popc(m & ((1u << lane) - 1u));
      st.xh[d] = xh; st.yh[d] = yh; st.xl[d] = xl; st.yl[d] = yl; st.pix[d] = pix;
    }
    __syncthreads();
    alive = static_cast<int>(threadIdx.x) < live;
    if (alive) {
      const int t = threadIdx.x;
      xh = st.xh[t]; yh = st.yh[t]; xl = st.xl[t]; yl = st.yl[t]; pix = st.pix[t];
    }
    __syncthreads();  // the state area is rewritten after the next chunk
  }
  if (alive && ok) {  // background: no footprint reached
    write(pix, -1);
    ++background;
  }
  if (poison || !ok) {  // values failed the checks, or a wait gave up: every pixel of the tile is NaN
    __syncthreads();
    if (valid) {
      const size_t p = static_cast<size_t>(py) * W + px;
      const float nan = __int_as_float(0x7fc00000);
      out_rgb[3 * p + 0] = nan; out_rgb[3 * p + 1] = nan; out_rgb[3 * p + 2] = nan;
      if (out_idx) out_idx[p] = -1;
    }
  }
  return ok;
}

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

// Replay adjoint (Sec. 5.2) of one pixel per thread over strokes 1 .. n,
// starting from the forward's final state st and the cotangent lambda^C_0 =
// (lC0, lC1, lC2).  Per stroke the 8 gradient values are reduced over the warp
// (reduce-scatter) and the CTA (shared memory, fixed order) and stored to
// slice[i][8] (first == true) or added to it.  red is shared [2][8][CH * 8].
// All threads of the CTA must call it.  Returns false if a bounded wait gave up.
template <int CH, bool INERT>
__device__ bool backward_tile(ChunkRing<CH>& ring, const float* __restrict__ packed, int n, bool valid,
                              const PixelState& st, float lC0, float lC1, float lC2, const float bg[3],
                              const RecordView& rv, float (*red)[kTileThreads / 32][CH * 8],
                              float* __restrict__ slice, bool first, unsigned& drift,
                              unsigned long long* status) {
  static_assert(CH * 8 == kTileThreads, "one partial per thread per chunk");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ck = rv.ck;
  float xh = st.xh, yh = st.yh, xl = st.xl, yl = st.yl, lt = st.lt;
  // lambda^C . c_i - lambda^T_i, carried as a difference (pair_stroke, tbr_pair.cuh):
  // E_i = lD + lambda^C . (c_i - c_{i-1}), mu = T_i E_i, lD <- (1 - alpha_i) E_i
  float lD = 0.0f;
  float pcR = bg[0], pcG = bg[1], pcB = bg[2];  // c_{i-1} (c_0: the background)
  float lx = 0.0f, ly = 0.0f;
  int rc = min(st.cnt, rv.cap), nri = -1;
  float4 rpos = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (valid && rc > 0) {
    const size_t o = static_cast<size_t>(rc - 1) * rv.stride + rv.off;
    rpos = rv.rec[o];
    nri = rv.rec_i[o];
  }
  int next_ck = (ck < n) ? ck : 0;
  const int nch = (n + CH - 1) / CH;
  auto chunk_src = [&](int q) { return packed + static_cast<size_t>(q) * CH * kRec; };
  auto chunk_cnt = [&](int q) { return min(CH, n - q * CH); };
  if (threadIdx.x == 0) {
    if (nch > 0) ring.issue(0, chunk_src(0), chunk_cnt(0));
    if (nch > 1) ring.issue(1, chunk_src(1), chunk_cnt(1));
  }
  bool ok = true;
  for (int q = 0; q < nch; ++q) {
    const int b = q & 1;
    const bool got = ring.wait(b, status);
    if (__syncthreads_or(!got)) {
      if (q + 1 < nch) ring.wait(b ^ 1, status);
      ok = false;
      break;
    }
    const int cntc = chunk_cnt(q);
    const float* S0 = ring.data(b);
    float (*rb)[CH * 8] = red[b];
    for (int j = 0; j < cntc; ++j) {
      const int i1 = q * CH + j + 1;
      float v0 = 0.0f, v1 = 0.0f, v2 = 0.0f, v3 = 0.0f, v4 = 0.0f, v5 = 0.0f, v6 = 0.0f, v7 = 0.0f;
      const float cR = S0[j * kRec + F_CR], cG = S0[j * kRec + F_CG], cB = S0[j * kRec + F_CB];
      const float dR = cR - pcR, dG = cG - pcG, dB = cB - pcB;
      pcR = cR; pcG = cG; pcB = cB;
      if (valid) {
        const float* S = S0 + j * kRec;
        const StrokeF g = load_stroke(S);
        const bool at_ck = (i1 == next_ck);
        size_t cko = 0;
        if (at_ck) {
          next_ck = (next_ck + ck < n) ? next_ck + ck : 0;
          cko = static_cast<size_t>(i1 / ck - 1) * rv.stride + rv.off;
        }
        const float E = lD + fmaf(lC0, dR, fmaf(lC1, dG, lC2 * dB));
        if (INERT) {
          float s, h, sp;
          to_frame(xh, yh, xl, yl, g, s, h);
          float d0, d1, d2, d3, d4;
          inert_vjp(s, h, g, sp, lx, ly, 0.0f, 0.0f, false, d0, d1, d2, d3, d4);
          const Cover cv = coverage(sp, g);
          if (at_ck) lt = rv.ck_lt[cko]; else lt += cv.sp2;
          const float T = ex2_a(lt);
          const float mu = T * E;
          const float Ta = T * cv.alpha;
          v5 = lC0 * Ta; v6 = lC1 * Ta; v7 = lC2 * Ta;
          inert_vjp(s, h, g, sp, lx, ly, mu * cv.dadz, cv.z, true, v0, v1, v2, v3, v4);
          lD = cv.oma * E;
        } else {
          Geo gq;
          float s, h, ds, dh;
          if (i1 == nri) {
            // x_i was within the floor's reach: read it back (Lemma "Support of the replay record")
            xh = rpos.x; yh = rpos.y; xl = rpos.z; yl = rpos.w;
            to_frame(xh, yh, xl, yl, g, s, h);
            psi_local<true>(s, h, g, gq, ds, dh);
            --rc;
            nri = -1;
            if (rc > 0) {
              const size_t o = static_cast<size_t>(rc - 1) * rv.stride + rv.off;
              rpos = rv.rec[o];
              nri = rv.rec_i[o];
            }
          } else if (at_ck) {
            // regenerate, measure the drift against the stored position, then reset to it
            to_frame(xh, yh, xl, yl, g, s, h);
            phi_local(s, h, g, gq, ds, dh);
            add_frame_disp(xh, yh, xl, yl, g, ds, dh);
            const float4 c = rv.ckpt[cko];
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
          if (at_ck) lt = rv.ck_lt[cko]; else lt += cv.sp2;  // log T_i = log T_{i-1} - log(1 - alpha_i)
          const float T = ex2_a(lt);
          const float mu = T * E;
          const float Ta = T * cv.alpha;
          v5 = lC0 * Ta; v6 = lC1 * Ta; v7 = lC2 * Ta;
          step_vjp(gq, g, lx, ly, mu * cv.dadz, cv.z, v0, v1, v2, v3, v4);
          lD = cv.oma * E;
        }
      }
      const float vv[8] = {v0, v1, v2, v3, v4, v5, v6, v7};
      const float r = warp_reduce8(vv);
      if ((lane & 3) == 0) rb[warp][j * 8 + ((lane >> 2) & 7)] = r;
    }
    __syncthreads();
    if (threadIdx.x == 0 && q + 2 < nch) ring.issue(b, chunk_src(q + 2), chunk_cnt(q + 2));
    const int t = threadIdx.x;
    if (t < cntc * 8) {
      float sum = 0.0f;
#pragma unroll
      for (int w = 0; w < kTileThreads / 32; ++w) sum += rb[w][t];
      float* dst = slice + static_cast<size_t>(q) * CH * 8 + t;
      *dst = first ? sum : *dst + sum;
    }
  }
  return ok;
}

}  // namespace tbr
