// One-pass closed-form compensation baseline (Sec. "Closed-form compensation
// baseline"): from the last stroke to the first, each stroke is moved so that
// the transport of every later, already compensated stroke carries it back to
// the position the given (inert-mark) program selects.  Its segment start
// (anchor variant; the offset vector is kept) or both ends (endpoint variant)
// are pre-imaged through psi_j (Eq. back) of the strokes j after it, the last
// one first.  A point inside K_j has no pre-image (Lemma "obstruction"): the
// step is clamped onto the segment by the ideal extension of psi_j, or skipped,
// and the stroke is counted as blocked.
//
// The N (N - 1) / 2 point transforms run as a wavefront on one CTA: step
// j = N-1 .. 0 first finalises stroke j (its points have passed every later
// stroke), then every thread applies psi_j to the points of its strokes i < j.
// One barrier per step; positions are hi/lo float pairs.  Up to 4096 strokes
// the points stay in registers (k_compensate_reg); longer programs keep them,
// and the compensated geometry, in global memory (k_compensate).
#include <math.h>

#include "tbr_host.h"

namespace tbr {

namespace {

constexpr int kCompThreads = 1024;

struct CompArgs {
  const float* packed;  // [n][kRec] the given program
  int n, endpoint, skip;
  float4* pts;          // [n][2] hi/lo points being pre-imaged (scratch)
  float* geo;           // [n][6] compensated m, e, L/2, r (scratch)
  float *cx, *cy, *th, *len;
  int* blocked;         // [n]
  unsigned long long* status;
};

// The compensated geometry of one stroke as the steps read it (m, e, L/2, r and
// the constants derived from them, formed once per stroke).
__device__ __forceinline__ StrokeF comp_geometry(const float* __restrict__ G) {
  StrokeF g;
  g.mx = G[0]; g.my = G[1]; g.ex = G[2]; g.ey = G[3]; g.hl = G[4]; g.r = G[5];
  g.L = 2.0f * g.hl; g.twoL = 2.0f * g.L; g.L2 = g.L * g.L;
  g.kA = fmaf(kPiF, g.r, g.twoL);
  g.Ar = g.kA * g.r;
  g.fl2 = 0.0f; g.iw = 0.0f; g.dlw = 0.0f;
  return g;
}

// psi_j with the ideal interior extension at a hi/lo point (hard-render map):
// returns true if the point lies in K_j (then clamped onto the segment, or left
// in place when skip), else moves it by the exterior map.
__device__ __forceinline__ bool comp_step(float4& p, const StrokeF& g, bool skip) {
  float s, h;
  to_frame(p.x, p.y, p.z, p.w, g, s, h);
  const float as = fabsf(s), ah = fabsf(h), d = as - g.hl;
  const float sp = d > 0.0f ? sqrt_a(fmaf(d, d, ah * ah)) : ah;
  if (sp <= g.r) {
    if (skip) return true;
    // C = 0: sigma = 0, the arclength t shrinks by L / (L + pi sigma'); a drop's disc goes to its centre
    float sn = 0.0f;
    if (g.L > 0.0f) {
      const float t = d > 0.0f ? fmaf(sp, atan2_pos(d, ah), g.hl) : as;
      sn = fminf(t * g.L * rcp_a(fmaf(kPiF, sp, g.L)), g.hl);
    }
    const float xs = sgn1(s) * sn;
    const float x = fmaf(xs, g.ex, g.mx), y = fmaf(xs, g.ey, g.my);
    p = make_float4(x, y, 0.0f, 0.0f);
    return true;
  }
  Geo q;
  float ds, dh;
  psi_local<false>(s, h, g, q, ds, dh);
  add_frame_disp(p.x, p.y, p.z, p.w, g, ds, dh);
  return false;
}

// Start of stroke i's segment (c = 0) or its end (c = 1) from the packed record,
// with explicitly rounded operations (no contraction), so that the value formed
// when the points are set up and the one formed when the displacement is taken
// are the same bits.
__device__ __forceinline__ float2 seg_end(const float* __restrict__ R, int c) {
  const float hx = __fmul_rn(R[F_HL], R[F_EX]), hy = __fmul_rn(R[F_HL], R[F_EY]);
  return c ? make_float2(__fadd_rn(R[F_MX], hx), __fadd_rn(R[F_MY], hy))
           : make_float2(__fsub_rn(R[F_MX], hx), __fsub_rn(R[F_MY], hy));
}

// Stroke j has passed every later stroke: its compensated geometry is the given
// one moved by the displacement of its start (and end), p[c] its pre-imaged
// points.  A stroke no step moved keeps its parameters bit for bit.  Writes the
// outputs and the geometry G = (m, e, L/2, r) the steps read.
__device__ __forceinline__ void comp_finalize(const CompArgs& a, int j, const float4 (&p)[2], float* G) {
  const float* R = a.packed + static_cast<size_t>(j) * kRec;
  const int npt = a.endpoint ? 2 : 1;
  float2 dsp[2];
  for (int c = 0; c < npt; ++c) {
    const float2 q = seg_end(R, c);
    dsp[c] = make_float2((p[c].x - q.x) + p[c].z, (p[c].y - q.y) + p[c].w);
  }
  float mx, my, ex = R[F_EX], ey = R[F_EY], hl = R[F_HL], th = R[F_TH];
  if (a.endpoint) {
    mx = R[F_MX] + 0.5f * (dsp[0].x + dsp[1].x);
    my = R[F_MY] + 0.5f * (dsp[0].y + dsp[1].y);
    const float gx = dsp[1].x - dsp[0].x, gy = dsp[1].y - dsp[0].y;
    if (gx != 0.0f || gy != 0.0f) {
      const float dx = fmaf(2.0f * hl, ex, gx), dy = fmaf(2.0f * hl, ey, gy);
      const float Ln = sqrtf(fmaf(dx, dx, dy * dy));
      if (Ln > 0.0f) {
        ex = dx / Ln; ey = dy / Ln;
        th = atan2f(dy, dx);
      }
      hl = 0.5f * Ln;
    }
  } else {
    mx = R[F_MX] + dsp[0].x;
    my = R[F_MY] + dsp[0].y;
  }
  G[0] = mx; G[1] = my; G[2] = ex; G[3] = ey; G[4] = hl; G[5] = R[F_R];
  a.cx[j] = mx; a.cy[j] = my; a.th[j] = th; a.len[j] = a.endpoint ? 2.0f * hl : R[F_L];
}

__global__ void __launch_bounds__(kCompThreads) k_compensate(CompArgs a) {
  const int n = a.n, npt = a.endpoint ? 2 : 1;
  // the points start at the given segment's start (and end)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float* R = a.packed + static_cast<size_t>(i) * kRec;
    for (int c = 0; c < 2; ++c) {
      const float2 q = seg_end(R, c);
      a.pts[2 * i + c] = make_float4(q.x, q.y, 0.0f, 0.0f);
    }
    a.blocked[i] = 0;
  }
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    if ((j % kCompThreads) == static_cast<int>(threadIdx.x)) {
      float4 p[2] = {a.pts[2 * j], a.pts[2 * j + 1]};
      comp_finalize(a, j, p, a.geo + static_cast<size_t>(j) * 6);
    }
    __syncthreads();
    if (j == 0) break;
    const StrokeF g = comp_geometry(a.geo + static_cast<size_t>(j) * 6);
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
      bool blk = false;
      for (int c = 0; c < npt; ++c) {
        float4 p = a.pts[2 * i + c];
        blk |= comp_step(p, g, a.skip != 0);
        a.pts[2 * i + c] = p;
      }
      if (blk) a.blocked[i] = 1;
    }
  }
  // blocked count (fixed order: per thread, then one atomic per warp)
  __syncthreads();
  unsigned cnt = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) cnt += a.blocked[i] ? 1u : 0u;
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(a.status + ST_RECORDS, static_cast<unsigned long long>(cnt));
}

// The same wavefront with every point in registers: thread t owns strokes
// t + m kCompThreads (m < K), so for n <= K kCompThreads no point leaves its
// thread.  Stroke j's owner applies psi_{j+1} to point j and finalises stroke j
// at once, without waiting for the other points; the geometry goes through a
// double-buffered shared slot, so one barrier per step orders it before every
// thread applies psi_j.  The arithmetic is k_compensate's, operation for
// operation.
template <int K>
__global__ void __launch_bounds__(kCompThreads) k_compensate_reg(CompArgs a) {
  __shared__ float sgeo[2][6];
  const int n = a.n, npt = a.endpoint ? 2 : 1, t = threadIdx.x;
  const bool skip = a.skip != 0;
  float4 P[K][2];
  unsigned blk = 0;
#pragma unroll
  for (int m = 0; m < K; ++m) {
    const int i = t + m * kCompThreads;
    const float* R = a.packed + static_cast<size_t>(i < n ? i : 0) * kRec;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float2 q = seg_end(R, c);
      P[m][c] = make_float4(q.x, q.y, 0.0f, 0.0f);
    }
  }
  for (int j = n - 1; j >= 0; --j) {
    const int b = j & 1;
    if ((j % kCompThreads) == t) {
      const int mj = j / kCompThreads;
#pragma unroll
      for (int m = 0; m < K; ++m)
        if (m == mj) comp_finalize(a, j, P[m], sgeo[b]);
    }
    __syncthreads();
    if (j == 0) break;
    const StrokeF g = comp_geometry(sgeo[b]);
    // points nearest the front first: the owner of stroke j - 1 finalises it next
#pragma unroll
    for (int m = K - 1; m >= 0; --m) {
      const int i = t + m * kCompThreads;
      if (i < j) {
#pragma unroll
        for (int c = 0; c < 2; ++c)
          if (c < npt && comp_step(P[m][c], g, skip)) blk |= 1u << m;
      }
    }
  }
  unsigned cnt = 0;
#pragma unroll
  for (int m = 0; m < K; ++m) {
    const int i = t + m * kCompThreads;
    if (i < n) {
      const unsigned f = (blk >> m) & 1u;
      a.blocked[i] = static_cast<int>(f);
      cnt += f;
    }
  }
  // blocked count (fixed order: per thread, then one atomic per warp)
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(a.status + ST_RECORDS, static_cast<unsigned long long>(cnt));
}

constexpr int kCompRegPts = 4;  // strokes per thread held in registers

}  // namespace

}  // namespace tbr

using namespace tbr;

extern "C" {

tbr_status tbr_compensate(const tbr_program* prog, int32_t endpoint, int32_t skip_blocked, float* out_cx,
                          float* out_cy, float* out_theta, float* out_length, int32_t* out_blocked,
                          int64_t* n_blocked, void* stream) {
  tbr_status s = check_program(prog, prog ? prog->n : 0);
  if (s != TBR_OK) return s;
  if (prog->coupling) return fail(TBR_ERR_INVALID_ARG, "compensation runs on the capsule map (coupling must be NULL)");
  if (prog->n > 0 && (!out_cx || !out_cy || !out_theta || !out_length || !out_blocked))
    return fail(TBR_ERR_INVALID_ARG, "NULL output");
  if (prog->n == 0) {
    if (n_blocked) *n_blocked = 0;
    return TBR_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = prog->n;
  float* packed = nullptr;
  float4* pts = nullptr;
  float* geo = nullptr;
  unsigned long long* status = nullptr;
  cudaError_t e = dalloc(&packed, static_cast<size_t>(n) * kRec, st);
  if (e == cudaSuccess) e = dalloc(&pts, static_cast<size_t>(n) * 2, st);
  if (e == cudaSuccess) e = dalloc(&geo, static_cast<size_t>(n) * 6, st);
  if (e == cudaSuccess) e = dalloc(&status, ST_COUNT, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, ST_COUNT * sizeof(unsigned long long), st);
  PackArgs pa{prog, n, 0.0f, 1.0f, 0, packed, nullptr, status};
  if (e == cudaSuccess) e = launch_pack(pa, st);
  if (e == cudaSuccess) {
    CompArgs a{packed, n, endpoint ? 1 : 0, skip_blocked ? 1 : 0, pts, geo, out_cx, out_cy, out_theta,
               out_length, out_blocked, status};
    KernelTimer kt(TBR_K_COMPENSATE, st);
    if (n <= kCompRegPts * kCompThreads) k_compensate_reg<kCompRegPts><<<1, kCompThreads, 0, st>>>(a);
    else k_compensate<<<1, kCompThreads, 0, st>>>(a);
    e = cudaGetLastError();
  }
  unsigned long long host[ST_COUNT] = {0};
  if (e == cudaSuccess && n_blocked) {
    e = cudaMemcpyAsync(host, status, sizeof(host), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  dfree(packed, st); dfree(pts, st); dfree(geo, st); dfree(status, st);
  if (e != cudaSuccess) return cuda_fail(e, "tbr_compensate");
  if (n_blocked) {
    if (host[ST_INVALID]) return fail(TBR_ERR_INVALID_ARG, "%llu strokes failed the value checks", host[ST_INVALID]);
    *n_blocked = static_cast<int64_t>(host[ST_RECORDS]);
  }
  return TBR_OK;
}

}  // extern "C"
