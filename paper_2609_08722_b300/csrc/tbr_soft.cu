// Soft forward render (Eq. relax, Eq. state) with the replay record of Sec. 5.2.
// One thread per pixel, a CTA per 32x8 tile, strokes streamed last-to-first
// through a two-deep shared-memory ring filled by 1-D bulk TMA.  Per stroke:
// distance sigma', coverage alpha = sigmoid(z) in logit form, compositing
// C += T alpha c, log2 T += log2(1 - alpha), then psi with the epsilon-floor.
// When recording: a sample the floor touched pushes (x_i, i) onto the pixel's
// side table (Lemma "Support of the replay record"), every k-th stroke stores
// (x_i, log2 T_i), and s_0 = (x_0, log2 T_0, record count) closes the pixel.
#include <math.h>

#include "tbr_internal.cuh"

namespace tbr {

namespace {

constexpr int kSoftCH = 64;
constexpr int kTileW = 32, kTileH = 8;

template <int CH, bool RECORD, bool INERT>
__global__ void __launch_bounds__(256) k_soft(SoftArgs a) {
  __shared__ __align__(128) float sbuf[2 * CH * kRec];
  __shared__ __align__(8) uint64_t sbar[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int W = a.W, H = a.H, n = a.n;
  const int tiles_x = (W + kTileW - 1) / kTileW;
  const int px = (blockIdx.x % tiles_x) * kTileW + lane;
  const int py = (blockIdx.x / tiles_x) * kTileH + warp;
  const bool valid = px < W && py < H;
  const size_t P = static_cast<size_t>(W) * H;
  const size_t p = valid ? static_cast<size_t>(py) * W + px : 0;
  unsigned long long* status = a.status;
  const bool invalid_prog = status[ST_INVALID] != 0ull;
  float xh = (static_cast<float>(px) + 0.5f) / static_cast<float>(W);
  float yh = (static_cast<float>(py) + 0.5f) / static_cast<float>(H);
  float xl = 0.0f, yl = 0.0f;  // positions are hi/lo pairs
  float lt = 0.0f;  // log2 T
  float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
  int cnt = 0;
  const int ck = a.ck_every;
  int next_ck = n > 1 ? ((n - 1) / ck) * ck : 0;  // largest checkpoint index < n (0 = none)

  ChunkRing<CH> ring;
  ring.init(sbuf, sbar);
  const int nch = (n + CH - 1) / CH;
  auto chunk_src = [&](int q) { return a.packed + static_cast<size_t>(nch - 1 - q) * CH * kRec; };
  auto chunk_cnt = [&](int q) { return min(CH, n - (nch - 1 - q) * CH); };
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
      break;
    }
    const int base = (nch - 1 - q) * CH;
    const int cntc = chunk_cnt(q);
    const float* S0 = ring.data(b);
    if (valid) {
      for (int j = cntc - 1; j >= 0; --j) {
        const int i1 = base + j + 1;  // the paper's 1-based stroke index
        if (RECORD && i1 == next_ck) {
          const size_t o = static_cast<size_t>(i1 / ck - 1) * P + p;
          a.ckpt[o] = make_float4(xh, yh, xl, yl);
          a.ck_lt[o] = lt;
          next_ck -= ck;
        }
        const float* S = S0 + j * kRec;
        const StrokeF g = load_stroke(S);
        float s, h;
        to_frame(xh, yh, xl, yl, g, s, h);
        if (INERT) {
          const float as = fabsf(s), ah = fabsf(h);
          const float d = as - g.hl;
          const float sp = d > 0.0f ? sqrt_a(fmaf(d, d, ah * ah)) : ah;
          const Cover cv = coverage(sp, g);
          const float w = ex2_a(lt) * cv.alpha;
          C0 = fmaf(w, S[F_CR], C0);
          C1 = fmaf(w, S[F_CG], C1);
          C2 = fmaf(w, S[F_CB], C2);
          lt -= cv.sp2;
        } else {
          Geo q;
          float ds, dh;
          psi_local<true>(s, h, g, q, ds, dh);
          const Cover cv = coverage(q.sp, g);
          const float w = ex2_a(lt) * cv.alpha;
          C0 = fmaf(w, S[F_CR], C0);
          C1 = fmaf(w, S[F_CG], C1);
          C2 = fmaf(w, S[F_CB], C2);
          lt -= cv.sp2;
          if (RECORD && q.floored) {
            if (cnt < a.cap) {
              const size_t o = static_cast<size_t>(cnt) * P + p;
              a.rec[o] = make_float4(xh, yh, xl, yl);
              a.rec_i[o] = i1;
            }
            ++cnt;
          }
          add_frame_disp(xh, yh, xl, yl, g, ds, dh);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && q + 2 < nch) ring.issue(b, chunk_src(q + 2), chunk_cnt(q + 2));
  }

  if (valid) {
    const float T0 = ex2_a(lt);
    float o0 = fmaf(T0, a.bg[0], C0), o1 = fmaf(T0, a.bg[1], C1), o2 = fmaf(T0, a.bg[2], C2);
    if (invalid_prog || aborted) o0 = o1 = o2 = __int_as_float(0x7fc00000);
    a.out_rgb[3 * p + 0] = o0;
    a.out_rgb[3 * p + 1] = o1;
    a.out_rgb[3 * p + 2] = o2;
    if (RECORD) {
      a.s0[p] = make_float4(xh, yh, xl, yl);
      a.s0b[p] = make_float2(lt, __int_as_float(cnt));
    }
  }
  if (RECORD) {
    const unsigned c = valid ? static_cast<unsigned>(cnt) : 0u;
    const unsigned tot = __reduce_add_sync(0xffffffffu, c);
    const unsigned mx = __reduce_max_sync(0xffffffffu, c);
    const unsigned ovf = __reduce_add_sync(0xffffffffu, (c > static_cast<unsigned>(a.cap)) ? 1u : 0u);
    if (lane == 0) {
      if (tot) atomicAdd(status + ST_RECORDS, static_cast<unsigned long long>(tot));
      if (mx) atomicMax(status + ST_MAXREC, static_cast<unsigned long long>(mx));
      if (ovf) atomicAdd(status + ST_OVERFLOW, static_cast<unsigned long long>(ovf));
    }
  }
}

}  // namespace

cudaError_t launch_soft(const SoftArgs& a, cudaStream_t st) {
  const int tiles = ((a.W + kTileW - 1) / kTileW) * ((a.H + kTileH - 1) / kTileH);
  const bool rec = a.s0 != nullptr;
  KernelTimer kt(TBR_K_SOFT, st);
  if (rec && a.inert) k_soft<kSoftCH, true, true><<<tiles, 256, 0, st>>>(a);
  else if (rec) k_soft<kSoftCH, true, false><<<tiles, 256, 0, st>>>(a);
  else if (a.inert) k_soft<kSoftCH, false, true><<<tiles, 256, 0, st>>>(a);
  else k_soft<kSoftCH, false, false><<<tiles, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace tbr
