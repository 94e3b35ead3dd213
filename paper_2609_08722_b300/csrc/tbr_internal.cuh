// Internal header of the TBR CUDA library (sm_103a): packed stroke layout,
// PTX wrappers for 1-D bulk TMA staging with mbarriers, and the per-step device
// math of the capsule transport (Sec. 4) and the replay adjoint (Sec. 5.2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "tbr.h"
#include "tbr_poly.h"

namespace tbr {

// ---------------------------------------------------------------------------
// Packed stroke record: 32 floats (128 B) per stroke, built once per call by
// k_pack (tbr_pack.cu) and staged into shared memory chunk by chunk.  The first
// 16 floats are the constants the paired adjoint loop reads (tbr_pair.cuh
// duplicates them into float2 pairs in this order), the next two the forward's
// floor constants.
// ---------------------------------------------------------------------------
constexpr int kRec = 32;
enum : int {
  F_MX = 0, F_MY = 1, F_EX = 2, F_EY = 3,    // centre m, direction e
  F_HL = 4, F_L = 5, F_2L = 6, F_L2 = 7,     // L/2, L, 2L, L^2
  F_AR = 8, F_R = 9, F_IW = 10, F_DLW = 11,  // A_L(r) = 2Lr + pi r^2, r, 1 / max(tau r, tau_min), (dw/dr)/w
  F_NPR = 12,                                // -(pi r + L) = dC/dr
  F_CR = 13, F_CG = 14, F_CB = 15,           // colour c_i
  F_KA = 16, F_FL2 = 17,                     // 2L + pi r, (eps r)^2
  F_TH = 18, F_BAD = 19,                     // theta, invalid flag
  F_D64 = 20,                                // 2 doubles: e in FP64 (FP64 band and repair)
  F_G0 = 24,                                 // g - 1 = G0 + G1 w + G2 w^2 + G3 w^3, w = cos 4 pi v
  F_C1 = 28                                  // c_1, c_2, c_3 of the profile (FP64 band), 1 spare
};

constexpr float kPiF = 3.14159265358979323846f;
constexpr double kPiD = 3.14159265358979323846;
constexpr float kEpsFloor = 1e-3f;           // epsilon of the floor (Sec. 5.2)
constexpr float kZMax = 16.11809565095832f;  // ln(1e7 - 1): alpha <= 1 - 1e-7
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kBand = 1e-4f;               // FP64 band half-width on |sigma' - r|
constexpr float kDriftTol = 1e-5f;           // checkpoint drift threshold

// Device status words (unsigned long long[ST_COUNT]).
enum : int {
  ST_TIMEOUT = 0, ST_OVERFLOW = 1, ST_DRIFT = 2, ST_BAND = 3, ST_INVALID = 4,
  ST_RECORDS = 5, ST_MAXREC = 6, ST_BG = 7, ST_VISITED = 8, ST_REPAIRED = 9, ST_REPAIR_OVF = 10,
  ST_COUNT = 16
};

// ---------------------------------------------------------------------------
// PTX wrappers: mbarrier + cp.async.bulk (1-D bulk TMA, global -> shared).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on an mbarrier phase: gives up after ~2 s of device time, sets
// the timeout status word and returns false.  Never traps.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && global_timer_ns() - t0 > 2000000000ull) break;
  }
  atomicAdd(status + ST_TIMEOUT, 1ull);
  return false;
}

// Two-deep ring of stroke chunks in shared memory.  Iteration q of a kernel's
// chunk loop consumes buffer q & 1; thread 0 refills it with the chunk of
// iteration q + 2 once every thread has passed the end-of-chunk barrier.
template <int CH>
struct ChunkRing {
  float* buf;         // [2][CH * kRec]
  uint64_t* bar;      // [2]
  uint32_t phase;     // bit b = expected parity of buffer b
  uint32_t pending;   // bit b = a copy into buffer b is in flight

  __device__ __forceinline__ void init(float* b, uint64_t* br) {
    buf = b; bar = br; phase = 0; pending = 0;
    if (threadIdx.x == 0) {
      mbar_init(&bar[0], 1);
      mbar_init(&bar[1], 1);
      fence_mbar_init();
    }
    __syncthreads();
  }
  // Thread 0 only: copy `count` packed strokes starting at `src` into buffer b.
  __device__ __forceinline__ void issue(int b, const float* src, int count) {
    const uint32_t bytes = static_cast<uint32_t>(count) * kRec * 4u;
    mbar_expect_tx(&bar[b], bytes);
    bulk_copy_g2s(buf + b * CH * kRec, src, bytes, &bar[b]);
  }
  // All threads: wait for buffer b; false on timeout.
  __device__ __forceinline__ bool wait(int b, unsigned long long* status) {
    const bool ok = mbar_wait_bounded(&bar[b], (phase >> b) & 1u, status);
    phase ^= (1u << b);
    return ok;
  }
  __device__ __forceinline__ const float* data(int b) const { return buf + b * CH * kRec; }
};

// ---------------------------------------------------------------------------
// Fast arithmetic: single-instruction PTX approximations (reciprocal, square
// root and reciprocal square root within 1-2 ulp, base-2 exponential /
// logarithm within ~2^-22) and
// polynomial atan / sin / 1-cos on the folded ranges the maps need
// (tbr_poly.h, generated by gen_poly.py), so that the hot loops avoid the
// multi-instruction IEEE division, square-root and range-reduction sequences.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_a(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_a(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_a(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_a(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lg2_a(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float div_a(float a, float b) { return a * rcp_a(b); }

template <int N>
__device__ __forceinline__ float horner(const float (&c)[N], float u) {
  float acc = c[N - 1];
#pragma unroll
  for (int k = N - 2; k >= 0; --k) acc = fmaf(acc, u, c[k]);
  return acc;
}
// atan2(y, x) for y, x >= 0 (result in [0, pi/2]).
__device__ __forceinline__ float atan2_pos(float y, float x) {
  const float mx = fmaxf(y, x), mn = fminf(y, x);
  const float z = mx > 0.0f ? mn * rcp_a(mx) : 0.0f;
  const float a = z * horner(kAtan, z * z);
  return y > x ? 0.5f * kPiF - a : a;
}
// sin(d) and 1 - cos(d) for |d| <= pi/2, both with full relative precision at small d.
__device__ __forceinline__ float sin_pi2(float d) { return d * horner(kSin, d * d); }
__device__ __forceinline__ float omc_pi2(float d) {
  const float u = d * d;
  return u * horner(kOmc, u);
}

// ---------------------------------------------------------------------------
// Stroke fields read from shared memory as broadcasts.
// ---------------------------------------------------------------------------
struct StrokeF {
  float mx, my, ex, ey, hl, L, r, L2, kA, Ar, fl2, iw, dlw, twoL;
};
__device__ __forceinline__ StrokeF load_stroke(const float* __restrict__ S) {
  const float4 a = *reinterpret_cast<const float4*>(S + F_MX);
  const float4 b = *reinterpret_cast<const float4*>(S + F_HL);
  const float4 c = *reinterpret_cast<const float4*>(S + F_AR);
  const float2 e = *reinterpret_cast<const float2*>(S + F_KA);
  StrokeF g;
  g.mx = a.x; g.my = a.y; g.ex = a.z; g.ey = a.w;
  g.hl = b.x; g.L = b.y; g.twoL = b.z; g.L2 = b.w;
  g.Ar = c.x; g.r = c.y; g.iw = c.z; g.dlw = c.w;
  g.kA = e.x; g.fl2 = e.y;
  return g;
}

// ---------------------------------------------------------------------------
// Positions are carried as unevaluated float pairs x = hi + lo: the local
// frame coordinate is formed as (hi - m) + lo.  The soft loops add each
// stroke's displacement to lo alone (one add on the loop-carried chain) and
// fold lo into hi with a TwoSum every kRenorm strokes, so |lo| stays within a
// few displacements and its rounding is far below ulp(hi).  pos_add is the
// per-step two-sum used by the hard render and the rare scalar steps.
// ---------------------------------------------------------------------------
constexpr int kRenorm = 16;
__device__ __forceinline__ void pos_add(float& hi, float& lo, float d) {
  const float s = hi + d;
  lo += d - (s - hi);  // exact error of hi + d when |hi| >= |d|
  hi = s;
}
// hi + lo -> (hi, lo) with |lo| <= ulp(hi) / 2 (TwoSum, exact for any magnitudes).
__device__ __forceinline__ void pos_renorm(float& hi, float& lo) {
  const float s = hi + lo;
  const float bp = s - hi;
  lo = (hi - (s - bp)) + (lo - bp);
  hi = s;
}

// ---------------------------------------------------------------------------
// Per-step quantities of one application of psi_i at x_i (to x_{i-1}) in the
// stroke frame, with the quadrant fold: s along e, h along e_perp, folded to
// |s|, |h|; t is the arclength from the flank midpoint along the parallel curve
// (the centred coordinate v of Eq. phi times the quarter perimeter fraction).
// On a cap the point is at angle phi from the flank normal, so t = L/2 + sigma phi.
// ---------------------------------------------------------------------------
struct Geo {
  float sgs, sgh;     // fold signs (psi keeps the quadrant)
  float si, hi;       // signed frame coordinates of x_i
  float so, ho;       // signed frame coordinates of x_{i-1}
  float sp, sig;      // sigma' = dist(x_i), sigma = dist(x_{i-1})
  float dsp;          // sigma' - sigma, in displacement form (exterior steps)
  float t, tn;        // folded arclength coordinates of x_i and x_{i-1}
  float ud, uh;       // at x_i: cap ? (sin phi, cos phi) : (0, 1)
  float phi;          // at x_i on a cap: angle from the flank normal
  float sb, cb, beta; // at x_{i-1} on a cap: angle and its sine / cosine
  float rb;           // coupling variant: distance of the deposit boundary at v
  bool cap_i, cap_o, floored;
};

__device__ __forceinline__ float sgn1(float v) { return copysignf(1.0f, v); }

// g(v) - 1 of the coupling variant (Eq. profile) at the angle 4 pi v in
// [0, pi] (folded v, both mirror symmetries): w = cos(4 pi v) = -sin(4 pi v -
// pi/2), then the cubic in w the record holds (the Chebyshev form of the modes).
__device__ __forceinline__ float profile_gm1(float ang, const float4& gp) {
  const float w = -sin_pi2(fminf(fmaxf(ang, 0.0f), kPiF) - 0.5f * kPiF);
  return fmaf(w, fmaf(w, fmaf(w, gp.w, gp.z), gp.y), gp.x);
}

// psi_i in displacement form at the frame point (s, h) of x_i (Eq. back with the
// centred arclength of Eq. phi).  The normal step uses
//   sigma - sigma' = -A_L(r) / (2L + pi (sigma' + sigma))  (exterior),
// the cap-to-cap tangential step rotates by
//   Delta = beta - phi = (sigma' - sigma) L (phi - pi/2) / (Q' sigma),
// both free of cancellation, so (ds, dh) keeps full relative precision even
// when the stroke is far.  FLOOR selects the epsilon-floor of Sec. 5.2 (soft
// render); without it the caller guarantees sigma' > r (hard render).
// COUPLED selects the coupling variant (Eq. coupling): the area removed is
// A_L(r) g(v) with g - 1 the cubic gp (F_G0..F_G3) in w = cos 4 pi v, v the
// folded centred arclength t / (2 Q'), so C and the normal step change and the
// tangential map, which keeps v, does not; q.rb receives the deposit boundary
// sigma_b(v), the root of 2 L sigma + pi sigma^2 = A_L(r) g(v).
template <bool FLOOR, bool COUPLED = false>
__device__ __forceinline__ void psi_local(float s, float h, const StrokeF& g, Geo& q, float& ds, float& dh,
                                          const float4 gp = make_float4(0.0f, 0.0f, 0.0f, 0.0f)) {
  if (g.L == 0.0f) {  // drop: radial map, delta = 0 (warp-uniform branch)
    q.sgs = sgn1(s); q.sgh = sgn1(h); q.si = s; q.hi = h;
    const float as = fabsf(s), ah = fabsf(h);
    q.cap_i = as > 0.0f;
    q.sp = sqrt_a(fmaf(as, as, ah * ah));
    if (q.cap_i) {
      const float inv = rcp_a(q.sp);
      q.ud = as * inv; q.uh = ah * inv;
      q.phi = atan2_pos(as, ah);
    } else {
      q.ud = 0.0f; q.uh = 1.0f; q.phi = 0.0f;
    }
    q.t = q.sp * q.phi;
    float C = (q.sp - g.r) * fmaf(kPiF, q.sp, g.kA);
    float Ag = g.Ar;
    if (COUPLED) {  // v = phi / (2 pi) on a drop's leaf
      const float gm1 = profile_gm1(2.0f * q.phi, gp);
      C = fmaf(-g.Ar, gm1, C);
      Ag = fmaf(g.Ar, gm1, g.Ar);
      q.rb = sqrt_a(Ag * (1.0f / kPiF));
    }
    q.floored = FLOOR && C < g.fl2;
    if (q.floored) C = g.fl2;
    q.sig = div_a(C, sqrt_a(kPiF * C));
    q.tn = q.sig * q.phi;
    q.cap_o = q.cap_i && q.tn > 0.0f;
    q.beta = q.cap_o ? q.phi : 0.0f;
    q.sb = q.cap_o ? q.ud : 0.0f;
    q.cb = q.cap_o ? q.uh : 1.0f;
    float dS, dH;
    if (q.floored) {                   // direct form, same ray
      q.dsp = q.sp - q.sig;
      dS = q.sig * q.sb - as;
      dH = q.sig * q.cb - ah;
    } else {
      const float dsig = -div_a(Ag, kPiF * (q.sp + q.sig));
      q.dsp = -dsig;
      dS = dsig * q.ud;
      dH = dsig * q.uh;
    }
    ds = q.sgs * dS;
    dh = q.sgh * dH;
    q.so = s + ds;
    q.ho = h + dh;
    return;
  }
  q.sgs = sgn1(s); q.sgh = sgn1(h); q.si = s; q.hi = h;
  const float as = fabsf(s), ah = fabsf(h);
  const float d = as - g.hl;
  q.cap_i = d > 0.0f;
  if (q.cap_i) {
    q.sp = sqrt_a(fmaf(d, d, ah * ah));
    const float inv = rcp_a(q.sp);
    q.ud = d * inv; q.uh = ah * inv;
    q.phi = atan2_pos(d, ah);
    q.t = fmaf(q.sp, q.phi, g.hl);
  } else {
    q.sp = ah; q.ud = 0.0f; q.uh = 1.0f; q.phi = 0.0f; q.t = as;
  }
  float C = (q.sp - g.r) * fmaf(kPiF, q.sp, g.kA);
  const float Qp = fmaf(kPiF, q.sp, g.L);
  const float iQp = Qp > 0.0f ? rcp_a(Qp) : 0.0f;
  float Ag = g.Ar;
  if (COUPLED) {  // 4 pi v = 2 pi t / Q'
    const float gm1 = profile_gm1(2.0f * kPiF * q.t * iQp, gp);
    C = fmaf(-g.Ar, gm1, C);
    Ag = fmaf(g.Ar, gm1, g.Ar);
    q.rb = div_a(Ag, g.L + sqrt_a(fmaf(kPiF, Ag, g.L2)));
  }
  q.floored = FLOOR && C < g.fl2;
  if (q.floored) C = g.fl2;
  q.sig = div_a(C, g.L + sqrt_a(fmaf(kPiF, C, g.L2)));
  const float Q = fmaf(kPiF, q.sig, g.L);
  const float dsig = q.floored ? q.sig - q.sp : -div_a(Ag, fmaf(kPiF, q.sp + q.sig, g.twoL));
  q.dsp = -dsig;
  q.tn = q.t * (Q * iQp);
  q.cap_o = q.tn > g.hl;
  float dS, dH;
  if (!q.floored && q.cap_i && q.cap_o) {
    float delta = -dsig * g.L * (q.phi - 0.5f * kPiF) * iQp * rcp_a(q.sig);
    delta = fminf(fmaxf(delta, -q.phi), 0.0f);
    const float sD = sin_pi2(delta), omc = omc_pi2(delta);
    dS = fmaf(dsig, q.ud, q.sig * fmaf(q.uh, sD, -q.ud * omc));
    dH = fmaf(dsig, q.uh, -q.sig * fmaf(q.ud, sD, q.uh * omc));
    const float cD = 1.0f - omc;
    q.beta = q.phi + delta;
    q.sb = fmaf(q.ud, cD, q.uh * sD);
    q.cb = fmaf(q.uh, cD, -q.ud * sD);
  } else if (!q.floored && !q.cap_i) {  // flank to flank (tn <= t <= L/2)
    dS = as * kPiF * dsig * iQp;
    dH = dsig;
    q.beta = 0.0f; q.sb = 0.0f; q.cb = 1.0f;
  } else {                             // floored, or cap to flank: direct form
    float sn, hn;
    if (q.cap_o) {
      q.beta = fminf((q.tn - g.hl) * rcp_a(q.sig), 0.5f * kPiF);
      q.sb = sin_pi2(q.beta);
      q.cb = 1.0f - omc_pi2(q.beta);
      sn = fmaf(q.sig, q.sb, g.hl); hn = q.sig * q.cb;
    } else {
      q.beta = 0.0f; q.sb = 0.0f; q.cb = 1.0f;
      sn = q.tn; hn = q.sig;
    }
    dS = sn - as; dH = hn - ah;
  }
  ds = q.sgs * dS;
  dh = q.sgh * dH;
  q.so = s + ds;
  q.ho = h + dh;
}

// Phi_i (Eq. fwd, Eq. rpos) in displacement form at the frame point (s, h) of
// x_{i-1}, recording the same intermediates as psi_local (the two maps share
// them exactly on the exterior):
//   sigma' - sigma = A_L(r) / (2L + pi (sigma + sigma')),
//   cap to cap: phi - beta = (sigma' - sigma) L (pi/2 - beta) / (Q sigma').
// COUPLED: the coupling variant's forward map (Eq. coupling), which adds
// A_L(r) g(v) with v taken at x_{i-1} (v is kept, so it is the same at x_i).
template <bool COUPLED = false>
__device__ __forceinline__ void phi_local(float s, float h, const StrokeF& g, Geo& q, float& ds, float& dh,
                                          const float4 gp = make_float4(0.0f, 0.0f, 0.0f, 0.0f)) {
  if (g.L == 0.0f) {  // drop: radial map, delta = 0 (warp-uniform branch)
    q.sgs = sgn1(s); q.sgh = sgn1(h); q.so = s; q.ho = h;
    const float as = fabsf(s), ah = fabsf(h);
    q.cap_o = as > 0.0f;
    q.sig = sqrt_a(fmaf(as, as, ah * ah));
    if (q.cap_o) {
      const float inv = rcp_a(q.sig);
      q.sb = as * inv; q.cb = ah * inv;
      q.beta = atan2_pos(as, ah);
    } else {
      q.sb = 0.0f; q.cb = 1.0f; q.beta = 0.0f;
    }
    q.tn = q.sig * q.beta;
    float Ag = g.Ar;
    if (COUPLED) Ag = fmaf(g.Ar, profile_gm1(2.0f * q.beta, gp), g.Ar);
    const float B = fmaf(q.sig, kPiF * q.sig, Ag);
    q.sp = div_a(B, sqrt_a(kPiF * B));
    const float dsp = div_a(Ag, kPiF * (q.sig + q.sp));
    q.dsp = dsp;
    q.t = q.sp * q.beta;
    q.cap_i = q.cap_o;
    q.phi = q.beta; q.ud = q.sb; q.uh = q.cb;
    q.floored = false;
    ds = q.sgs * (dsp * q.sb);
    dh = q.sgh * (dsp * q.cb);
    q.si = s + ds;
    q.hi = h + dh;
    return;
  }
  q.sgs = sgn1(s); q.sgh = sgn1(h); q.so = s; q.ho = h;
  const float as = fabsf(s), ah = fabsf(h);
  const float d = as - g.hl;
  q.cap_o = d > 0.0f;
  if (q.cap_o) {
    q.sig = sqrt_a(fmaf(d, d, ah * ah));
    const float inv = rcp_a(q.sig);
    q.sb = d * inv; q.cb = ah * inv;
    q.beta = atan2_pos(d, ah);
    q.tn = fmaf(q.sig, q.beta, g.hl);
  } else {
    q.sig = ah; q.sb = 0.0f; q.cb = 1.0f; q.beta = 0.0f; q.tn = as;
  }
  const float Q = fmaf(kPiF, q.sig, g.L);
  const float iQ = Q > 0.0f ? rcp_a(Q) : 0.0f;
  float Ag = g.Ar;
  if (COUPLED) Ag = fmaf(g.Ar, profile_gm1(2.0f * kPiF * q.tn * iQ, gp), g.Ar);  // 4 pi v = 2 pi t / Q
  const float B = fmaf(q.sig, fmaf(kPiF, q.sig, g.twoL), Ag);
  q.sp = div_a(B, g.L + sqrt_a(fmaf(kPiF, B, g.L2)));
  const float dsp = div_a(Ag, fmaf(kPiF, q.sig + q.sp, g.twoL));
  q.dsp = dsp;
  const float Qp = fmaf(kPiF, q.sp, g.L);
  q.t = q.tn * (Qp * iQ);
  q.cap_i = q.t > g.hl;
  float dS, dH;
  if (q.cap_o) {                       // cap to cap (t >= tn > L/2)
    float delta = dsp * g.L * (0.5f * kPiF - q.beta) * iQ * rcp_a(q.sp);
    delta = fminf(fmaxf(delta, 0.0f), 0.5f * kPiF - q.beta);
    const float sD = sin_pi2(delta), omc = omc_pi2(delta);
    dS = fmaf(dsp, q.sb, q.sp * fmaf(q.cb, sD, -q.sb * omc));
    dH = fmaf(dsp, q.cb, -q.sp * fmaf(q.sb, sD, q.cb * omc));
    const float cD = 1.0f - omc;
    q.phi = q.beta + delta;
    q.ud = fmaf(q.sb, cD, q.cb * sD);
    q.uh = fmaf(q.cb, cD, -q.sb * sD);
    q.cap_i = true;
  } else if (!q.cap_i) {               // flank to flank
    dS = q.tn * kPiF * dsp * iQ;
    dH = dsp;
    q.phi = 0.0f; q.ud = 0.0f; q.uh = 1.0f;
  } else {                             // flank to cap: direct form
    q.phi = fminf((q.t - g.hl) * rcp_a(q.sp), 0.5f * kPiF);
    q.ud = sin_pi2(q.phi);
    q.uh = 1.0f - omc_pi2(q.phi);
    dS = fmaf(q.sp, q.ud, g.hl) - as;
    dH = fmaf(q.sp, q.uh, -ah);
  }
  q.floored = false;
  ds = q.sgs * dS;
  dh = q.sgh * dH;
  q.si = s + ds;
  q.hi = h + dh;
}

// Drop (L = 0) forward step in world coordinates: the map is radial,
// x_{i-1} = m + (x_i - m) sigma / rho with sigma = sqrt(rho^2 - r^2) (Eq. back at
// L = 0), so the displacement is (x_i - m) (sigma - rho) / rho with the
// cancellation-free sigma - rho = -A_0(r) / (pi (rho + sigma)).  Returns rho
// (the distance sigma' used by the coverage) and the world displacement.
// FLOOR applies the epsilon-floor (then the point lands at distance
// sqrt((eps r)^2 / pi) on the same ray; at rho = 0 on the e_perp ray).
template <bool FLOOR>
__device__ __forceinline__ float drop_step(float dx, float dy, const StrokeF& g, float& ddx, float& ddy,
                                           bool& floored) {
  const float rho = sqrt_a(fmaf(dx, dx, dy * dy));
  float C = (rho - g.r) * fmaf(kPiF, rho, g.kA);
  floored = FLOOR && C < g.fl2;
  if (floored) C = g.fl2;
  const float sig = div_a(C, sqrt_a(kPiF * C));
  const float dsig = floored ? sig - rho : -div_a(g.Ar, kPiF * (rho + sig));
  if (rho > 0.0f) {
    const float k = dsig * rcp_a(rho);
    ddx = k * dx;
    ddy = k * dy;
  } else {  // the centre itself: the fold convention sends it along +e_perp
    ddx = -dsig * g.ey;
    ddy = dsig * g.ex;
  }
  return rho;
}

// Pull-back through the sixteen drops of the transfer renderer R_D (Sec.
// "Transfer across transport constructions"): stroke i's displacement is the
// composition of K = 16 classical drop maps of radius s, s^2 = A_L(r) / (16 pi)
// (so the inserted area is the stroke's own), centred at m + e L ((k + 1/2)/16 -
// 1/2) and inserted in one sweep k = 0..15; the pull-back undoes them in reverse
// order.  In displacement form a drop moves a point at distance rho from its
// centre by -(x - c) s^2 / (rho (rho + sigma)), sigma = sqrt(rho^2 - s^2), with
// rho (rho + sigma) formed as rho^2 + sqrt(rho^2 sigma^2);
// inside its disc (rho^2 - s^2 < (eps s)^2) the point is floored on the same ray
// at eps s (rho = 0: along e_perp).  The displacements go to the lo parts of the
// hi/lo position, which is renormalised at the end.  Returns the floor binds.
constexpr int kDrops = 16;
__device__ __forceinline__ int drops_step(float& xh, float& yh, float& xl, float& yl, const StrokeF& g) {
  const float s2 = g.Ar * (1.0f / (kDrops * kPiF));
  const float fl = (kEpsFloor * kEpsFloor) * s2;
  int binds = 0;
#pragma unroll 4
  for (int k = kDrops - 1; k >= 0; --k) {
    const float t = g.L * ((static_cast<float>(k) + 0.5f) * (1.0f / kDrops) - 0.5f);
    const float dx = (xh - fmaf(t, g.ex, g.mx)) + xl, dy = (yh - fmaf(t, g.ey, g.my)) + yl;
    const float rho2 = fmaf(dx, dx, dy * dy);
    const float sig2 = rho2 - s2;
    if (sig2 >= fl) {
      // rho (rho + sigma) = rho^2 + sqrt(rho^2 sigma^2): one square root and one reciprocal
      const float kf = -s2 * rcp_a(rho2 + sqrt_a(rho2 * sig2));
      xl = fmaf(kf, dx, xl);
      yl = fmaf(kf, dy, yl);
    } else {
      ++binds;
      const float sig = sqrt_a(fl);
      if (rho2 > 0.0f) {
        const float kf = fmaf(sig, rsqrt_a(rho2), -1.0f);
        xl = fmaf(kf, dx, xl);
        yl = fmaf(kf, dy, yl);
      } else {
        xl += -g.ey * sig - dx;
        yl += g.ex * sig - dy;
      }
    }
  }
  pos_renorm(xh, xl);
  pos_renorm(yh, yl);
  return binds;
}

// Frame coordinates of a hi/lo position.
__device__ __forceinline__ void to_frame(float xh, float yh, float xl, float yl, const StrokeF& g, float& s,
                                         float& h) {
  const float dx = (xh - g.mx) + xl, dy = (yh - g.my) + yl;
  s = fmaf(dx, g.ex, dy * g.ey);
  h = fmaf(dy, g.ex, -dx * g.ey);
}

// Adds a frame displacement (ds, dh) to a hi/lo position.
__device__ __forceinline__ void add_frame_disp(float& xh, float& yh, float& xl, float& yl, const StrokeF& g,
                                               float ds, float dh) {
  pos_add(xh, xl, fmaf(ds, g.ex, -dh * g.ey));
  pos_add(yh, yl, fmaf(ds, g.ey, dh * g.ex));
}

// The angle cotangent of one exterior step without the cancellation of its two
// rotation halves.  In the folded frame, rotating the stroke by theta about m is
// a rotation about the cap centre (L/2, 0) plus a shift of the cap centre by
// L/2 along the normal.  On a cap the pull-back keeps the centred arclength, so
// the first part only sees the stretch 1 - d beta/d phi = L (sigma - sigma') /
// (Q' sigma) of the angle; the second part is (L/2) (ghn - g_ah) with g_ah the
// full folded cotangent of |h| (coverage included, whose own angle term
// -(L/2) cos phi cancels against it), i.e. -(L/2) w_h with w the displacement
// cotangent of step_vjp_ext.  spm = sign(s) sign(h).
__device__ __forceinline__ float theta_vjp_cap(float spm, float L, float hl, float dsp, float iQp, float gsn,
                                               float ghn, float sb, float cb, float wh) {
  const float k = -L * dsp * iQp;  // sigma (1 - d beta / d phi)
  return spm * fmaf(k, fmaf(ghn, sb, -gsn * cb), -hl * wh);
}
// On a flank the map is (|s|, sigma') -> (|s| Q/Q', sigma) with d sigma/d sigma'
// = Q'/Q; the rotation's share is |s|-weighted and proportional to sigma' -
// sigma throughout: b1 = (sigma' - sigma) (L/Q' - pi^2 |s|^2 (Q + Q') / (Q Q'^2)),
// b2 = -pi |s| (sigma' - sigma) (Q + Q') / (Q Q'); the coverage adds -|s| g_cov
// (g_cov = its cotangent of sigma').
__device__ __forceinline__ float theta_vjp_flank(float spm, float L, float as, float dsp, float Q, float Qp,
                                                 float gsn, float ghn, float g_cov) {
  const float iQ = rcp_a(Q), iQp = rcp_a(Qp);
  const float QQ = (Q + Qp) * iQ * iQp;
  const float b1 = dsp * fmaf(-kPiF * kPiF * as * as, QQ * iQp, L * iQp);
  const float b2 = -kPiF * as * dsp * QQ;
  return spm * (fmaf(gsn, b1, ghn * b2) - as * g_cov);
}

// VJP of an exterior step that stays on a cap or on a flank, in displacement
// form.  psi moves the folded point p = (|s|, |h|) to p + D(p), D small far
// from the stroke; the step's cotangents are written through D alone:
// lambda_{i-1} = lambda_i + R S w and d/dm = -R S w with w = (dD/dp)^T g + the
// coverage's share (S the fold signs, R the frame), so none of them is the
// difference of two quantities of size |lambda|.
//   cap: p = c + sigma' u(phi), p + D = c + sigma u(beta), c = (L/2, 0),
//        u(a) = (sin a, cos a), beta = phi + delta with
//        delta = (sigma' - sigma) L (phi - pi/2) / (Q' sigma);
//        dD/dsigma' = (pi (sigma'-sigma)/Q) u(beta) + (u(beta) - u(phi)) + sigma delta_sigma' u'(beta),
//        dD/dphi    = -(sigma'-sigma) u'(beta) + sigma' (u'(beta) - u'(phi)) + sigma delta_phi u'(beta),
//        delta_phi = (sigma'-sigma) L / (Q' sigma),
//        delta_sigma' = -delta (pi/Q + pi/Q' + Q'/(Q sigma)),
//        and dsigma'/dp = u(phi), dphi/dp = u'(phi) / sigma';
//   flank: D = (-|s| pi (sigma'-sigma) / Q', -(sigma'-sigma)).
// L and r enter through sigma (dsigma/dL = (sigma'-sigma-r)/Q, dsigma/dr =
// -(L + pi r)/Q at fixed sigma'), through delta, and (L) through the cap
// centre, whose shift moves p relative to c.  The angle uses theta_vjp_*.
// Returns the 8 cotangents like step_vjp.  gsn, ghn: the folded cotangent of
// the output point; gcv: the coverage's cotangent of sigma'.
__device__ __forceinline__ void step_vjp_ext(const Geo& q, const StrokeF& g, float gsn, float ghn, float gcv,
                                             float mua, float z, float& lamx, float& lamy, float& gcx,
                                             float& gcy, float& gth, float& gL, float& gr) {
  const float Q = fmaf(kPiF, q.sig, g.L), Qp = fmaf(kPiF, q.sp, g.L);
  const float iQ = rcp_a(Q), iQp = rcp_a(Qp);
  const float sgL = (q.dsp - g.r) * iQ;           // d sigma / dL
  const float sgr = -fmaf(kPiF, g.r, g.L) * iQ;   // d sigma / dr
  float ws, wh, gLl, grl;
  if (q.cap_i) {
    const float isg = rcp_a(q.sig), isp = rcp_a(q.sp);
    const float room = q.phi - 0.5f * kPiF;        // phi - pi/2 <= 0
    const float sdphi = q.dsp * g.L * iQp;         // sigma delta_phi
    const float sdel = sdphi * room;               // sigma delta
    const float sdsp = -sdel * fmaf(kPiF, iQ + iQp, Qp * iQ * isg);  // sigma delta_sigma'
    const float pdQ = kPiF * q.dsp * iQ;
    // dD/dsigma' and dD/dphi (u'(a) = (cos a, -sin a))
    const float As0 = fmaf(pdQ, q.sb, fmaf(sdsp, q.cb, q.sb - q.ud));
    const float As1 = fmaf(pdQ, q.cb, fmaf(-sdsp, q.sb, q.cb - q.uh));
    const float Ap0 = fmaf(sdphi - q.dsp, q.cb, q.sp * (q.cb - q.uh));
    const float Ap1 = fmaf(q.dsp - sdphi, q.sb, q.sp * (q.ud - q.sb));
    const float g_sp = fmaf(gsn, As0, fmaf(ghn, As1, gcv));
    const float g_ph = fmaf(gsn, Ap0, ghn * Ap1) * isp;
    ws = fmaf(q.ud, g_sp, q.uh * g_ph);
    wh = fmaf(q.uh, g_sp, -q.ud * g_ph);
    // explicit L and r: D = sigma u(beta) - sigma' u(phi) through sigma and delta
    const float sdL = room * iQp * (fmaf(-g.L, sgL, q.dsp) - q.dsp * g.L * fmaf(sgL, isg, iQp));
    const float sdr = -room * g.L * sgr * q.sp * iQp * isg;
    gLl = fmaf(gsn, fmaf(sgL, q.sb, sdL * q.cb), ghn * fmaf(sgL, q.cb, -sdL * q.sb)) - 0.5f * ws;
    grl = fmaf(gsn, fmaf(sgr, q.sb, sdr * q.cb), ghn * fmaf(sgr, q.cb, -sdr * q.sb));
    gth = theta_vjp_cap(q.sgs * q.sgh, g.L, g.hl, q.dsp, iQp, gsn, ghn, q.sb, q.cb, wh);
  } else {
    const float as = fabsf(q.si);
    const float pdQp = kPiF * q.dsp * iQp;
    ws = -gsn * pdQp;
    wh = fmaf(gsn, as * kPiF * pdQp * (Q + Qp) * iQ * iQp, fmaf(ghn, kPiF * q.dsp * iQ, gcv));
    gLl = fmaf(gsn, as * kPiF * fmaf(q.dsp, iQp, sgL) * iQp, ghn * sgL);
    grl = fmaf(gsn, as * kPiF * sgr * iQp, ghn * sgr);
    gth = theta_vjp_flank(q.sgs * q.sgh, g.L, as, q.dsp, Q, Qp, gsn, ghn, gcv);
  }
  const float GS = q.sgs * ws, GH = q.sgh * wh;
  const float dlx = fmaf(GS, g.ex, -GH * g.ey);
  const float dly = fmaf(GS, g.ey, GH * g.ex);
  gcx = -dlx;
  gcy = -dly;
  gL = gLl;
  gr = fmaf(mua, fmaf(-z, g.dlw, g.iw), grl);
  lamx += dlx;
  lamy += dly;
}

// Vector-Jacobian product of one step (Eq. adjstep, Eq. adjparam), written out
// by reverse-mode differentiation of psi_local in the stroke frame.
//   lam     lambda^x_{i-1} (world), replaced by lambda^x_i
//   mua     mu_i * d alpha / d z (0 where the clamp binds)
//   z       the (clamped) coverage logit (r - sigma') / w
// Outputs: gradient of lambda^x_{i-1} . psi_i + mu_i alpha_i with respect to
// (cx, cy, theta, L, r).
__device__ __forceinline__ void step_vjp(const Geo& q, const StrokeF& g, float& lamx, float& lamy,
                                         float mua, float z, float& gcx, float& gcy, float& gth,
                                         float& gL, float& gr) {
  const float ls = fmaf(lamx, g.ex, lamy * g.ey);   // lambda . e
  const float lh = fmaf(lamy, g.ex, -lamx * g.ey);  // lambda . e_perp
  const float gsn = q.sgs * ls, ghn = q.sgh * lh;
  if (!q.floored && q.cap_i == q.cap_o) {  // exterior step on a cap or on a flank
    step_vjp_ext(q, g, gsn, ghn, -mua * g.iw, mua, z, lamx, lamy, gcx, gcy, gth, gL, gr);
    return;
  }
  float g_tn, g_sig, g_hl = 0.0f, g_L = 0.0f, g_r = 0.0f, g_sp = 0.0f;
  if (!q.cap_o) {
    g_tn = gsn; g_sig = ghn;
  } else {
    g_sig = fmaf(gsn, q.sb, ghn * q.cb);
    const float g_beta = q.sig * fmaf(gsn, q.cb, -ghn * q.sb);
    g_hl = gsn;
    g_tn = g_beta * rcp_a(q.sig);
    g_hl -= g_tn;
    g_sig -= g_tn * q.beta;
  }
  // tn = t * Q / Qp
  const float Q = fmaf(kPiF, q.sig, g.L), Qp = fmaf(kPiF, q.sp, g.L);
  float g_t = 0.0f;
  if (Qp > 0.0f) {
    const float iQp = rcp_a(Qp);
    g_t = g_tn * Q * iQp;
    const float g_Q = g_tn * q.t * iQp;
    const float g_Qp = -g_tn * q.tn * iQp;
    g_L += g_Q + g_Qp;
    g_sig = fmaf(kPiF, g_Q, g_sig);
    g_sp = fmaf(kPiF, g_Qp, g_sp);
  }
  // sigma solves A_L(sigma) = C: d sigma/dC = 1/(2Q), d sigma/dL = -sigma/Q
  float g_C = 0.0f;
  if (Q > 0.0f) {
    const float iQ = rcp_a(Q);
    g_C = 0.5f * g_sig * iQ;
    g_L -= g_sig * q.sig * iQ;
  }
  if (q.floored) {
    g_r = fmaf(g_C * 2.0f * kEpsFloor * kEpsFloor, g.r, g_r);
  } else {
    g_sp = fmaf(2.0f * g_C, Qp, g_sp);                 // dC/dsigma' = P_L(sigma')
    g_r -= 2.0f * g_C * fmaf(kPiF, g.r, g.L);          // dC/dr = -P_L(r)
    g_L = fmaf(2.0f * g_C, q.sp - g.r, g_L);           // dC/dL = 2(sigma' - r)
  }
  // coverage alpha(z), z = (r - sigma') / w(r)
  g_sp = fmaf(-mua, g.iw, g_sp);
  g_r = fmaf(mua, fmaf(-z, g.dlw, g.iw), g_r);
  // t and sigma' from (|s|, |h|): cap: t = L/2 + sigma' phi, sigma' = |(d, |h|)|
  float g_as, g_ah;
  if (q.cap_i) {
    g_hl += g_t;
    g_sp = fmaf(g_t, q.phi, g_sp);
    const float g_d = fmaf(g_sp, q.ud, g_t * q.uh);
    g_ah = fmaf(g_sp, q.uh, -g_t * q.ud);
    g_as = g_d;
    g_hl -= g_d;
  } else {
    g_as = g_t;
    g_ah = g_sp;
  }
  g_L = fmaf(0.5f, g_hl, g_L);
  const float GS = q.sgs * g_as, GH = q.sgh * g_ah;
  const float nlx = fmaf(GS, g.ex, -GH * g.ey);
  const float nly = fmaf(GS, g.ey, GH * g.ex);
  gcx = lamx - nlx;
  gcy = lamy - nly;
  // theta turns the frame about m: the cotangent is lambda . J (x_{i-1} - m) -
  // (D psi^T lambda) . J (x_i - m) plus the coverage's share.
  // floored steps and steps between a cap and a flank (near the stroke, no
  // cancellation to avoid): the rotation about m as the difference of its halves
  gth = fmaf(q.so, lh, -q.ho * ls) + fmaf(GS, q.hi, -GH * q.si);
  gL = g_L;
  gr = g_r;
  lamx = nlx;
  lamy = nly;
}

// Relaxed coverage (Eq. relax) in the logit form used by both soft kernels.
// With the logit clamped at z <= ln(1e7 - 1), e^z <= 1e7 stays finite, so
// alpha = e^z / (1 + e^z) and 1 - alpha = 1 / (1 + e^z) are both free of
// cancellation without a case split on the sign of z.
struct Cover {
  float z;      // clamped logit
  float alpha;  // sigmoid(z)
  float oma;    // 1 - alpha (computed without cancellation)
  float dadz;   // alpha (1 - alpha), 0 where the clamp binds
  float sp2;    // -log2(1 - alpha) = softplus(z) / ln 2
};
// Coverage of a point at distance sp from the segment whose deposit boundary
// lies at distance rb on its ray (rb = r for the capsule).
__device__ __forceinline__ Cover coverage(float sp, float rb, const StrokeF& g) {
  Cover c;
  const float zr = (rb - sp) * g.iw;
  const bool clamped = zr > kZMax;
  c.z = fminf(zr, kZMax);
  const float ez = ex2_a(c.z * kLog2e);
  const float opl = 1.0f + ez;
  c.oma = rcp_a(opl);
  c.alpha = ez * c.oma;
  c.dadz = clamped ? 0.0f : c.alpha * c.oma;
  c.sp2 = lg2_a(opl);
  return c;
}
__device__ __forceinline__ Cover coverage(float sp, const StrokeF& g) { return coverage(sp, g.r, g); }

// Warp reduce-scatter of 8 values: afterwards every lane holds the warp total
// of value (lane >> 2) & 7.
__device__ __forceinline__ float warp_reduce8(const float (&v)[8]) {
  const unsigned lane = threadIdx.x & 31u;
  const bool b4 = lane & 16u, b3 = lane & 8u, b2 = lane & 4u;
  float w[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float send = b4 ? v[j] : v[j + 4];
    const float keep = b4 ? v[j + 4] : v[j];
    w[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float u[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float send = b3 ? w[j] : w[j + 2];
    const float keep = b3 ? w[j + 2] : w[j];
    u[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const float send = b2 ? u[0] : u[1];
  float r = (b2 ? u[1] : u[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
  r += __shfl_xor_sync(0xffffffffu, r, 2);
  r += __shfl_xor_sync(0xffffffffu, r, 1);
  return r;
}

// ---------------------------------------------------------------------------
// Host launchers (defined in the .cu files of this directory).
// ---------------------------------------------------------------------------
// RAII: records CUDA events around one kernel launch when profiling is on
// (tbr_profile_enable); tbr_profile.cu.
class KernelTimer {
 public:
  KernelTimer(int kernel, cudaStream_t st);
  ~KernelTimer();
  KernelTimer(const KernelTimer&) = delete;
  KernelTimer& operator=(const KernelTimer&) = delete;

 private:
  int kernel_;
  cudaStream_t st_;
  cudaEvent_t start_ = nullptr, stop_ = nullptr;
  bool active_ = false;
};

struct PackArgs {
  const tbr_program* prog;   // host struct with device pointers
  int n;                     // strokes to pack (prefix)
  float tau, tau_min;
  int snap;
  float* packed;             // [n][kRec]
  float* probs;              // [n][k] softmax probabilities or NULL
  unsigned long long* status;
};
cudaError_t launch_pack(const PackArgs& a, cudaStream_t st);

// Internal transport codes: the capsule map, the sixteen drops of the transfer
// renderer, and the capsule map of the coupling variant (the program carries a
// profile; the packed record holds it).
enum : int { kTransportCapsule = 0, kTransportDrops = 1, kTransportCoupled = 2 };
cudaError_t launch_hard(const float* packed, int n, int W, int H, const float bg[3], float* out_rgb,
                        int* out_idx, unsigned long long* status, int want_stats, cudaStream_t st,
                        int transport = 0);

struct SoftArgs {
  const float* packed;
  int n, W, H;
  float bg[3];
  int inert;
  int transport = 0;         // kTransport*: drops and coupled render forward only, no record
  float exit_lt = -3.0e38f;  // forward only: a pixel stops once log2 T < exit_lt (this value: off)
  int ck_every;              // checkpoint interval k (>= 1)
  int cap;                   // side-table capacity per pixel
  float* out_rgb;
  // replay record (all NULL for a forward-only render); positions are hi/lo pairs
  float4* s0;                // [P] (x_hi, y_hi, x_lo, y_lo) of x_0
  float2* s0b;               // [P] (log2 T_0, record count as int bits)
  float4* ckpt;              // [(n-1)/k][P] x_i at i = k, 2k, ...
  float* ck_lt;              // [(n-1)/k][P] log2 T_i
  float4* rec;               // [cap][P] x_i of floored samples (LIFO per pixel)
  int* rec_i;                // [cap][P] their 1-based stroke index i
  unsigned long long* status;
};
cudaError_t launch_soft(const SoftArgs& a, cudaStream_t st);

struct BwdArgs {
  const float* packed;
  int n, W, H;
  float bg[3];
  int inert;
  int ck_every;
  int cap;                   // side-table capacity per pixel
  const float4* s0;
  const float2* s0b;
  const float4* ckpt;
  const float* ck_lt;
  const float4* rec;
  const int* rec_i;
  const float* dLdR;
  float* partial;            // [grid][n][8]
  int grid;
  unsigned long long* status;
  // FP64 repair of drifting checkpoint segments (all NULL / 0: off)
  float drift_tol = kDriftTol;
  int2* repair_list = nullptr;  // [repair_cap] (pixel, segment start)
  int* repair_count = nullptr;  // [1], zeroed by launch_backward
  int repair_cap = 0;           // <= kRepairMax
  float* corr = nullptr;        // [repair_cap][n][8] gradient corrections
  unsigned char* repair_first = nullptr;  // [P] per-pixel "queued" flags, zeroed by launch_backward
  unsigned char* tile_drift = nullptr;    // [pair tiles] drift seen in the tile (repair_first + P), zeroed too
  int coupled = 0;              // 1: the coupling variant (one pixel per thread, no repair)
};
constexpr int kRepairMax = 1024;  // largest repair list (sorted by one CTA)

// A launch-shape value (SM count, resident CTAs per SM) cached per device
// ordinal under a lock: several host threads may launch at once (the serving
// worker beside a caller), and one process may drive devices that differ in
// SM count.  compute(dev) runs once per device, with that device current.
struct PerDeviceInt {
  static constexpr int kMaxDevices = 64;
  std::mutex mu;
  int val[kMaxDevices] = {};
  bool have[kMaxDevices] = {};
  template <class F>
  int get(F&& compute) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return compute(dev < 0 ? 0 : dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!have[dev]) {
      val[dev] = compute(dev);
      have[dev] = true;
    }
    return val[dev];
  }
};
// Streaming multiprocessors of the current device (>= 1).
int device_sm_count();

int backward_grid(int W, int H, int inert);  // CTAs of the persistent backward grid
int backward_grid_coupled(int W, int H);     // the same for the coupling variant's adjoint
cudaError_t launch_backward_coupled(const BwdArgs& a, cudaStream_t st);
// Replay adjoint, then (with a repair list) the FP64 repair of the pixels whose
// checkpoint drift exceeded drift_tol.
cudaError_t launch_backward(const BwdArgs& a, cudaStream_t st);

struct EpilogueArgs {
  const float* partial;
  int grid, n, k;
  const float* corr = nullptr;          // [repair_cap][n][8] or NULL
  const int* repair_count = nullptr;    // entries in corr (used only if <= repair_cap)
  int repair_cap = 0;
  const float* packed;
  const float* probs;
  const float* palette;
  float inv_color_temp;
  float* grad8;              // [n][8] scratch
  float *g_cx, *g_cy, *g_th, *g_len, *g_r, *g_logits, *g_pal;
  const unsigned long long* status;
};
cudaError_t launch_backward_epilogue(const EpilogueArgs& a, cudaStream_t st);

cudaError_t launch_loss(const float* rgb, const float* target, int64_t npix, double* partial,
                        int nblocks, float* loss_out, float* dLdR, cudaStream_t st);
// loss_out[0] = (sum of the nparts FP64 partials, in order) / nval.
cudaError_t launch_loss_final(const double* partial, int nparts, int64_t nval, float* loss_out, cudaStream_t st);

int loss_blocks(int64_t npix);

}  // namespace tbr
