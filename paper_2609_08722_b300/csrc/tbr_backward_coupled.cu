// Replay adjoint of the coupling variant Phi_g (Sec. "A variant closer to
// line-source potential flow", Eq. coupling; the replay of Sec. 5.2 with
// Eq. rpos, Eq. rT, Eq. adjstep, Eq. adjparam).  Per pixel, for i = 1..N:
//   x_i = Phi_g,i(x_{i-1}) in FP32 displacement form, or the side-table record
//   where the forward's floor bound, or the position checkpoint;
//   log T_i from the coverage of the deposit {u <= A_L(r) g(v)};
//   the adjoint step as the hand-derived reverse product of psi_g's
//   displacement and of the coverage (tbr_coupled_vjp.cuh).
// One pixel per thread on the persistent grid of 32x8 tiles, strokes streamed
// first to last through the shared-memory ring; the 8 per-stroke gradient
// values go through the same warp reduce-scatter and CTA slice as the other
// adjoints, so the epilogue's fixed-order sum applies unchanged.
#include <math.h>

#include "tbr_coupled_vjp.cuh"
#include "tbr_tile.cuh"

namespace tbr {

namespace {

constexpr int kBwdCCH = 32;  // kBwdCCH * 8 == kTileThreads: one partial per thread per chunk

template <int CH>
__device__ bool backward_tile_coupled(ChunkRing<CH>& ring, const float* __restrict__ packed, int n, bool valid,
                                      const PixelState& st, float lC0, float lC1, float lC2, const float bg[3],
                                      const RecordView& rv, float (*red)[kTileThreads / 32][CH * 8],
                                      float* __restrict__ slice, bool first, unsigned& drift,
                                      unsigned long long* status) {
  static_assert(CH * 8 == kTileThreads, "one partial per thread per chunk");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ck = rv.ck;
  float xh = st.xh, yh = st.yh, xl = st.xl, yl = st.yl, lt = st.lt;
  float lT = fmaf(lC0, bg[0], fmaf(lC1, bg[1], lC2 * bg[2]));
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
      if (valid) {
        const float* S = S0 + j * kRec;
        const StrokeF g = load_stroke(S);
        const float4 gp = *reinterpret_cast<const float4*>(S + F_G0);
        const float lCc = fmaf(lC0, S[F_CR], fmaf(lC1, S[F_CG], lC2 * S[F_CB]));
        const bool at_ck = (i1 == next_ck);
        size_t cko = 0;
        if (at_ck) {
          next_ck = (next_ck + ck < n) ? next_ck + ck : 0;
          cko = static_cast<size_t>(i1 / ck - 1) * rv.stride + rv.off;
        }
        if (i1 == nri) {
          // x_i was within the floor's reach: read it back (Lemma "Support of the replay record")
          xh = rpos.x; yh = rpos.y; xl = rpos.z; yl = rpos.w;
          --rc;
          nri = -1;
          if (rc > 0) {
            const size_t o = static_cast<size_t>(rc - 1) * rv.stride + rv.off;
            rpos = rv.rec[o];
            nri = rv.rec_i[o];
          }
        } else {
          // x_i = Phi_g,i(x_{i-1}) (Eq. rpos with Eq. coupling)
          Geo gq;
          float s, h, ds, dh;
          to_frame(xh, yh, xl, yl, g, s, h);
          phi_local<true>(s, h, g, gq, ds, dh, gp);
          add_frame_disp(xh, yh, xl, yl, g, ds, dh);
          if (at_ck) {  // measure the drift against the stored position, then reset to it
            const float4 c = rv.ckpt[cko];
            if (fabsf((xh - c.x) + (xl - c.z)) > rv.drift_tol || fabsf((yh - c.y) + (yl - c.w)) > rv.drift_tol)
              ++drift;
            xh = c.x; yh = c.y; xl = c.z; yl = c.w;
          }
        }
        // Eq. adjstep / Eq. adjparam: G = d/d(x, theta, L, r) of lambda^x . disp + mu alpha,
        // mu = T_i (lC . c - lambda^T); log T_i = log T_{i-1} - log(1 - alpha_i)
        float G[5], alpha, oma, T = 0.0f;
        coupled_vjp(xh, yh, xl, yl, S,
                    [&](float, float, float sp2, float& sx, float& sy, float& smu) {
                      if (at_ck) lt = rv.ck_lt[cko]; else lt += sp2;
                      T = ex2_a(lt);
                      sx = lx;
                      sy = ly;
                      smu = T * (lCc - lT);
                    },
                    G, alpha, oma);
        const float Ta = T * alpha;
        v5 = lC0 * Ta; v6 = lC1 * Ta; v7 = lC2 * Ta;
        // psi_g and alpha depend on x_i - m, so d/dm = -d/dx
        v0 = -G[0]; v1 = -G[1]; v2 = G[2]; v3 = G[3]; v4 = G[4];
        lx += G[0];
        ly += G[1];
        lT = fmaf(oma, lT, alpha * lCc);
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

template <int CH>
__global__ void __launch_bounds__(kTileThreads) k_backward_c(BwdArgs a) {
  __shared__ __align__(128) float sbuf[2 * CH * kRec];
  __shared__ __align__(8) uint64_t sbar[2];
  __shared__ float red[2][kTileThreads / 32][CH * 8];
  const int lane = threadIdx.x & 31;
  const int W = a.W, H = a.H, n = a.n;
  const int ntiles = tile_count(W, H);
  const size_t P = static_cast<size_t>(W) * H;
  unsigned long long* status = a.status;
  const bool skip = status[ST_INVALID] != 0ull || status[ST_OVERFLOW] != 0ull;
  ChunkRing<CH> ring;
  ring.init(sbuf, sbar);
  float* slice = a.partial + static_cast<size_t>(blockIdx.x) * n * 8;
  unsigned drift = 0;
  bool first = true;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int px, py;
    tile_pixel(tile, W, px, py);
    const bool valid = px < W && py < H && !skip;
    const size_t p = valid ? static_cast<size_t>(py) * W + px : 0;
    PixelState st{};
    float lC0 = 0.0f, lC1 = 0.0f, lC2 = 0.0f;
    if (valid) {
      const float4 s0 = a.s0[p];
      const float2 s0b = a.s0b[p];
      st.xh = s0.x; st.yh = s0.y; st.xl = s0.z; st.yl = s0.w;
      st.lt = s0b.x;
      st.cnt = __float_as_int(s0b.y);
      lC0 = a.dLdR[3 * p + 0]; lC1 = a.dLdR[3 * p + 1]; lC2 = a.dLdR[3 * p + 2];
    }
    RecordView rv{const_cast<float4*>(a.rec), const_cast<int*>(a.rec_i), const_cast<float4*>(a.ckpt),
                  const_cast<float*>(a.ck_lt), P, p, a.cap, a.ck_every};
    rv.drift_tol = a.drift_tol;
    if (!backward_tile_coupled<CH>(ring, a.packed, n, valid, st, lC0, lC1, lC2, a.bg, rv, red, slice, first,
                                   drift, status))
      break;
    first = false;
  }
  const unsigned dsum = __reduce_add_sync(0xffffffffu, drift);
  if (lane == 0 && dsum) atomicAdd(status + ST_DRIFT, static_cast<unsigned long long>(dsum));
}

}  // namespace

int backward_grid_coupled(int W, int H) {
  static PerDeviceInt cache;
  const int per_sm = cache.get([](int) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward_c<kBwdCCH>, kTileThreads, 0) != cudaSuccess ||
        b < 1)
      b = 1;
    return b;
  });
  const int tiles = tile_count(W, H);
  const int g0 = per_sm * device_sm_count();
  const int waves = (tiles + g0 - 1) / g0;
  return (tiles + waves - 1) / waves;
}

cudaError_t launch_backward_coupled(const BwdArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  KernelTimer kt(TBR_K_BACKWARD, st);
  k_backward_c<kBwdCCH><<<a.grid, kTileThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace tbr
