// Paired replay adjoint: each thread carries two vertically adjacent pixels
// through the replay adjoint (Sec. 5.2) with Blackwell's packed FP32 pairs
// (FFMA2 / FADD2 / FMUL2), so one instruction advances both pixels.  The common
// step -- regeneration by Phi (Eq. fwd, Eq. rpos), coverage (Eq. relax), the
// adjoint step and the parameter VJP (Eq. adjstep, Eq. adjparam) -- is written
// branch-free: on a capsule flank the cap formulas reduce to the flank ones once
// (sin beta, cos beta, beta) = (0, 1, 0) and (sin phi, cos phi, phi) = (0, 1, 0),
// so one instruction stream serves both.  Side-table pops, checkpoint resets and
// the rare flank-to-cap regeneration take the scalar routines per pixel.
#pragma once

#include "tbr_coupled_vjp.cuh"
#include "tbr_tile.cuh"

namespace tbr {

using f2 = float2;

__device__ __forceinline__ f2 F2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
// a - b as one FADD2 with the second operand negated (the same rounding as a - b)
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
// a * b - c as one FFMA2 with the addend negated (a single rounding)
__device__ __forceinline__ f2 fms2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, make_float2(-c.x, -c.y)); }
// c - a * b as one FFMA2 with a negated factor
__device__ __forceinline__ f2 fnma2(f2 a, f2 b, f2 c) { return __ffma2_rn(make_float2(-a.x, -a.y), b, c); }
__device__ __forceinline__ f2 abs2(f2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ f2 sgn2(f2 a) { return make_float2(sgn1(a.x), sgn1(a.y)); }
__device__ __forceinline__ f2 max2(f2 a, f2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ f2 min2(f2 a, f2 b) { return make_float2(fminf(a.x, b.x), fminf(a.y, b.y)); }
__device__ __forceinline__ f2 sqrt2(f2 a) { return make_float2(sqrt_a(a.x), sqrt_a(a.y)); }
__device__ __forceinline__ f2 rcp2(f2 a) { return make_float2(rcp_a(a.x), rcp_a(a.y)); }
// 1/a where a > 0, else 0
__device__ __forceinline__ f2 rcp2_pos(f2 a) {
  return make_float2(a.x > 0.0f ? rcp_a(a.x) : 0.0f, a.y > 0.0f ? rcp_a(a.y) : 0.0f);
}
// Smallest argument of the guarded reciprocals below: x * rsqrt(max(x, kTiny))
// is sqrt(x) for x >= kTiny and 0 at x = 0; mn * rcp(max(mx, kTiny)) is 0 when
// 0 <= mn <= mx < kTiny.
constexpr float kTiny = 1e-36f;
__device__ __forceinline__ f2 rsqrt2(f2 a) { return make_float2(rsqrt_a(a.x), rsqrt_a(a.y)); }
__device__ __forceinline__ f2 ex22(f2 a) { return make_float2(ex2_a(a.x), ex2_a(a.y)); }
__device__ __forceinline__ f2 lg22(f2 a) { return make_float2(lg2_a(a.x), lg2_a(a.y)); }
__device__ __forceinline__ f2 sel2(bool cx, bool cy, f2 a, f2 b) {
  return make_float2(cx ? a.x : b.x, cy ? a.y : b.y);
}
__device__ __forceinline__ float comp(const f2& v, int c) { return c == 0 ? v.x : v.y; }
__device__ __forceinline__ void put(f2& v, int c, float x) {
  if (c == 0) v.x = x;
  else v.y = x;
}

template <int N>
__device__ __forceinline__ f2 horner2(const float (&c)[N], f2 u) {
  f2 acc = F2(c[N - 1]);
#pragma unroll
  for (int k = N - 2; k >= 0; --k) acc = fma2(acc, u, F2(c[k]));
  return acc;
}
// atan2(y, x) for y, x >= 0, per component (as atan2_pos).
__device__ __forceinline__ f2 atan2_pos2(f2 y, f2 x) {
  const f2 mx = max2(y, x), mn = min2(y, x);
  const f2 z = mul2(mn, rcp2(max2(mx, F2(kTiny))));
  const f2 a = mul2(z, horner2(kAtan, mul2(z, z)));
  const f2 b = sub2(F2(0.5f * kPiF), a);
  return sel2(y.x > x.x, y.y > x.y, b, a);
}
__device__ __forceinline__ f2 sin_pi2_2(f2 d) { return mul2(d, horner2(kSin, mul2(d, d))); }
__device__ __forceinline__ f2 omc_pi2_2(f2 d) {
  const f2 u = mul2(d, d);
  return mul2(u, horner2(kOmc, u));
}

// ---------------------------------------------------------------------------
// Pair record: the per-stroke constants the paired loops read, each duplicated
// into both halves of a float2 so that it enters FFMA2 directly.  They are the
// first 16 floats of the packed record, in its order (128 bytes of pairs per
// stroke); the forward also reads the floor constants (KA, FL2) from a
// separate 2-entry array.  Built in shared memory once per staged chunk by a
// plain strided copy.  (A 144-byte record, and a fill that branched per field,
// each measured about 5% slower in the adjoint loop.)
// ---------------------------------------------------------------------------
enum : int {
  P_MX = F_MX, P_MY = F_MY, P_EX = F_EX, P_EY = F_EY, P_HL = F_HL, P_L = F_L, P_2L = F_2L, P_L2 = F_L2,
  P_AR = F_AR, P_R = F_R, P_IW = F_IW, P_DLW = F_DLW, P_NPR = F_NPR, P_CR = F_CR, P_CG = F_CG, P_CB = F_CB,
  kPairRec = 16,
  X_KA = F_KA - kPairRec, X_FL2 = F_FL2 - kPairRec,
  kPairExt = 2
};
static_assert(P_CB == kPairRec - 1 && X_FL2 == kPairExt - 1, "pair record = packed floats 0..17");

// All threads: fill the pair records of the cnt strokes staged at S0 (and, with
// EXT, the forward's extension).  With DCOL (the adjoint) the colour fields
// hold the colour step c_i - c_{i-1} instead of c_i, (pc0, pc1, pc2) being the
// colour of the stroke before the chunk's first (the background c_0 before
// stroke 1).  The caller synchronises before use.
template <bool EXT, bool DCOL = false>
__device__ __forceinline__ void pair_records_fill(const float* __restrict__ S0, int cnt, f2* __restrict__ pbuf,
                                                  f2* __restrict__ pext, float pc0 = 0.0f, float pc1 = 0.0f,
                                                  float pc2 = 0.0f) {
  for (int e = threadIdx.x; e < cnt * kPairRec; e += kTileThreads) {
    const int j = e / kPairRec, f = e % kPairRec;
    float v = S0[j * kRec + f];
    if (DCOL && f >= P_CR) v -= j > 0 ? S0[(j - 1) * kRec + f] : (f == P_CR ? pc0 : (f == P_CG ? pc1 : pc2));
    pbuf[e] = F2(v);
  }
  if (EXT) {
    for (int e = threadIdx.x; e < cnt * kPairExt; e += kTileThreads)
      pext[e] = F2(S0[(e / kPairExt) * kRec + kPairRec + (e % kPairExt)]);
  }
}

// Per-step quantities of one regeneration step for two pixels: the fields of
// Geo with the flank conventions above, plus Q = L + pi sigma, Q' = L + pi
// sigma' and their reciprocals (0 where the value is 0).
struct Geo2 {
  f2 sgs, sgh, si, hi, so, ho, sp, sig, tn, ud, uh, phi, sb, cb, beta;
  f2 Q, Qp, iQ, iQp;
  f2 dsp;       // sigma' - sigma (displacement form)
  f2 isg, isp;  // 1 / sigma, 1 / sigma'
};

// x_i = Phi_i(x_{i-1}) for two pixels at frame points (s, h) of x_{i-1}, in the
// displacement form of phi_local.  Returns a bit mask of the pixels whose step
// goes from the flank onto a cap (bit c for component c); their outputs are
// not valid and the caller recomputes them with phi_local.
__device__ __forceinline__ int phi_pair(f2 s, f2 h, const f2* __restrict__ P, Geo2& q, f2& ds, f2& dh) {
  const f2 L = P[P_L], Ar = P[P_AR];
  q.sgs = sgn2(s); q.sgh = sgn2(h); q.so = s; q.ho = h;
  const f2 as = abs2(s), ah = abs2(h);
  if (L.x == 0.0f) {  // drop: radial (warp-uniform branch)
    const f2 x2 = fma2(as, as, mul2(ah, ah));
    const f2 is = rsqrt2(max2(x2, F2(kTiny)));  // 1 / sigma
    q.sig = mul2(x2, is);
    q.sb = mul2(as, is);
    q.cb = sel2(x2.x > 0.0f, x2.y > 0.0f, mul2(ah, is), F2(1.0f));
    q.beta = atan2_pos2(as, ah);
    q.tn = mul2(q.sig, q.beta);
    const f2 B = fma2(q.sig, mul2(F2(kPiF), q.sig), Ar);
    q.sp = sqrt2(mul2(B, F2(1.0f / kPiF)));
    const f2 dsp = mul2(Ar, rcp2(mul2(F2(kPiF), add2(q.sig, q.sp))));
    q.dsp = dsp;
    q.phi = q.beta; q.ud = q.sb; q.uh = q.cb;
    q.Q = mul2(F2(kPiF), q.sig);
    q.Qp = mul2(F2(kPiF), q.sp);
    q.iQ = rcp2_pos(q.Q);
    q.iQp = rcp2(q.Qp);
    q.isg = is;
    q.isp = mul2(F2(kPiF), q.iQp);
    ds = mul2(q.sgs, mul2(dsp, q.sb));
    dh = mul2(q.sgh, mul2(dsp, q.cb));
    q.si = add2(s, ds);
    q.hi = add2(h, dh);
    return 0;
  }
  const f2 hl = P[P_HL];
  const f2 d = sub2(as, hl);
  const bool capo_x = d.x > 0.0f, capo_y = d.y > 0.0f;
  const f2 dp = max2(d, F2(0.0f));
  const f2 x2 = fma2(dp, dp, mul2(ah, ah));
  const f2 is = rsqrt2(max2(x2, F2(kTiny)));  // 1 / sigma
  q.sig = mul2(x2, is);
  q.sb = mul2(dp, is);
  q.cb = sel2(capo_x, capo_y, mul2(ah, is), F2(1.0f));
  q.beta = atan2_pos2(dp, ah);
  q.tn = fma2(q.sig, q.beta, min2(as, hl));
  const f2 B = fma2(q.sig, fma2(F2(kPiF), q.sig, P[P_2L]), Ar);
  q.sp = mul2(B, rcp2(add2(L, sqrt2(fma2(F2(kPiF), B, P[P_L2])))));
  const f2 dsp = mul2(Ar, rcp2(fma2(F2(kPiF), add2(q.sig, q.sp), P[P_2L])));
  q.dsp = dsp;
  q.Q = fma2(F2(kPiF), q.sig, L);
  q.Qp = fma2(F2(kPiF), q.sp, L);
  q.iQ = rcp2(q.Q);
  q.iQp = rcp2(q.Qp);
  const f2 t = mul2(q.tn, mul2(q.Qp, q.iQ));
  const bool capi_x = t.x > hl.x, capi_y = t.y > hl.y;
  // cap to cap: rotation by delta, clamped to the cap.  On the flank delta = 0,
  // and with (sb, cb, beta) = (0, 1, 0) the cap formulas give dH = dsigma',
  // (ud, uh, phi) = (0, 1, 0); only dS needs the flank's own form.
  const f2 room = sub2(F2(0.5f * kPiF), q.beta);
  q.isg = is;
  q.isp = rcp2(q.sp);
  f2 delta = mul2(mul2(mul2(dsp, L), room), mul2(q.iQ, q.isp));
  delta = sel2(capo_x, capo_y, min2(max2(delta, F2(0.0f)), room), F2(0.0f));
  const f2 sD = sin_pi2_2(delta), omc = omc_pi2_2(delta);
  const f2 cD = sub2(F2(1.0f), omc);
  const f2 dSc = fma2(dsp, q.sb, mul2(q.sp, fms2(q.cb, sD, mul2(q.sb, omc))));
  const f2 dH = fms2(dsp, q.cb, mul2(q.sp, fma2(q.sb, sD, mul2(q.cb, omc))));
  // flank to flank: translation along the flank
  const f2 dSf = mul2(mul2(q.tn, F2(kPiF)), mul2(dsp, q.iQ));
  const f2 dS = sel2(capo_x, capo_y, dSc, dSf);
  q.ud = fma2(q.sb, cD, mul2(q.cb, sD));
  q.uh = fms2(q.cb, cD, mul2(q.sb, sD));
  q.phi = add2(q.beta, delta);
  ds = mul2(q.sgs, dS);
  dh = mul2(q.sgh, dH);
  q.si = add2(s, ds);
  q.hi = add2(h, dh);
  return ((!capo_x && capi_x) ? 1 : 0) | ((!capo_y && capi_y) ? 2 : 0);
}

// x_{i-1} = psi_i(x_i) for two pixels at frame points (s, h) of x_i (L > 0),
// in the displacement form of psi_local<true>.  Outputs sigma' (the distance of
// x_i) and the frame displacement.  Returns a bit mask of the pixels that the
// floor touches or whose step leaves a cap for the flank; their outputs are not
// valid and the caller recomputes them with psi_local<true>.
__device__ __forceinline__ int psi_pair(f2 s, f2 h, const f2* __restrict__ P, const f2* __restrict__ X, f2& sp,
                                        f2& ds, f2& dh) {
  const f2 L = P[P_L], hl = P[P_HL];
  const f2 as = abs2(s), ah = abs2(h);
  const f2 d = sub2(as, hl);
  const bool ci_x = d.x > 0.0f, ci_y = d.y > 0.0f;
  const f2 dp = max2(d, F2(0.0f));
  const f2 x2 = fma2(dp, dp, mul2(ah, ah));
  const f2 is = rsqrt2(max2(x2, F2(kTiny)));  // 1 / sigma'
  sp = mul2(x2, is);
  const f2 ud = mul2(dp, is);
  const f2 uh = sel2(ci_x, ci_y, mul2(ah, is), F2(1.0f));
  const f2 phi = atan2_pos2(dp, ah);
  const f2 t = fma2(sp, phi, min2(as, hl));
  const f2 C = mul2(sub2(sp, P[P_R]), fma2(F2(kPiF), sp, X[X_KA]));
  const bool fl_x = C.x < X[X_FL2].x, fl_y = C.y < X[X_FL2].y;
  const f2 sig = mul2(C, rcp2(add2(L, sqrt2(fma2(F2(kPiF), C, P[P_L2])))));
  const f2 Q = fma2(F2(kPiF), sig, L), iQp = rcp2(fma2(F2(kPiF), sp, L));
  // sigma' - sigma = A_L(r) / (2L + pi (sigma' + sigma))
  const f2 nds = mul2(P[P_AR], rcp2(fma2(F2(kPiF), add2(sp, sig), P[P_2L])));
  const f2 tn = mul2(t, mul2(Q, iQp));
  const bool co_x = tn.x > hl.x, co_y = tn.y > hl.y;
  // cap to cap: rotation by delta = (sigma' - sigma) L (phi - pi/2) / (Q' sigma) in [-phi, 0];
  // on the flank delta = 0 and (ud, uh) = (0, 1), so dH is the flank's -(sigma' - sigma)
  f2 delta = mul2(mul2(mul2(nds, L), sub2(phi, F2(0.5f * kPiF))), mul2(iQp, rcp2(sig)));
  delta = sel2(ci_x, ci_y, min2(max2(delta, mul2(phi, F2(-1.0f))), F2(0.0f)), F2(0.0f));
  const f2 sD = sin_pi2_2(delta), omc = omc_pi2_2(delta);
  const f2 dSc = fms2(sig, fms2(uh, sD, mul2(ud, omc)), mul2(nds, ud));
  const f2 dH = mul2(F2(-1.0f), fma2(sig, fma2(ud, sD, mul2(uh, omc)), mul2(nds, uh)));
  // flank to flank: tangential step |s| pi (sigma - sigma') / Q'
  const f2 dSf = mul2(mul2(as, F2(-kPiF)), mul2(nds, iQp));
  const f2 dS = sel2(ci_x, ci_y, dSc, dSf);
  ds = mul2(sgn2(s), dS);
  dh = mul2(sgn2(h), dH);
  return ((fl_x || (ci_x && !co_x)) ? 1 : 0) | ((fl_y || (ci_y && !co_y)) ? 2 : 0);
}

// Drop (L = 0) pull-back for two pixels at world offsets (dx, dy) from the
// centre, as drop_step<true>.  Outputs rho = sigma' and the world
// displacement; returns the mask of pixels the floor touches (recomputed by the
// caller with drop_step<true>).
__device__ __forceinline__ int drop_pair(f2 dx, f2 dy, const f2* __restrict__ P, const f2* __restrict__ X, f2& rho,
                                         f2& ddx, f2& ddy) {
  const f2 x2 = fma2(dx, dx, mul2(dy, dy));
  const f2 is = rsqrt2(max2(x2, F2(kTiny)));
  rho = mul2(x2, is);
  const f2 C = mul2(sub2(rho, P[P_R]), fma2(F2(kPiF), rho, X[X_KA]));
  const bool fl_x = C.x < X[X_FL2].x, fl_y = C.y < X[X_FL2].y;
  const f2 sig = sqrt2(mul2(C, F2(1.0f / kPiF)));
  // (sigma - rho) / rho with sigma - rho = -A_0(r) / (pi (rho + sigma))
  const f2 k = mul2(mul2(P[P_AR], F2(-1.0f / kPiF)), mul2(rcp2(add2(rho, sig)), is));
  ddx = mul2(k, dx);
  ddy = mul2(k, dy);
  return (fl_x ? 1 : 0) | (fl_y ? 2 : 0);
}

// Relaxed coverage (Eq. relax, logit form) for two pixels, as coverage().
struct Cover2 {
  f2 z, alpha, oma, dadz, sp2;
};
__device__ __forceinline__ Cover2 coverage2(f2 sp, const f2* __restrict__ P) {
  Cover2 c;
  const f2 zr = mul2(sub2(P[P_R], sp), P[P_IW]);
  const bool clx = zr.x > kZMax, cly = zr.y > kZMax;
  c.z = min2(zr, F2(kZMax));
  const f2 ez = ex22(mul2(c.z, F2(kLog2e)));
  const f2 opl = add2(F2(1.0f), ez);
  c.oma = rcp2(opl);
  c.alpha = mul2(ez, c.oma);
  c.dadz = sel2(clx, cly, F2(0.0f), mul2(c.alpha, c.oma));
  c.sp2 = lg22(opl);
  return c;
}

// Frame coordinates of two hi/lo positions.
__device__ __forceinline__ void to_frame2(f2 xh, f2 yh, f2 xl, f2 yl, const f2* __restrict__ P, f2& s, f2& h) {
  const f2 dx = add2(sub2(xh, P[P_MX]), xl), dy = add2(sub2(yh, P[P_MY]), yl);
  s = fma2(dx, P[P_EX], mul2(dy, P[P_EY]));
  h = sub2(mul2(dy, P[P_EX]), mul2(dx, P[P_EY]));
}
// pos_renorm for two positions.
__device__ __forceinline__ void pos_renorm2(f2& hi, f2& lo) {
  const f2 s = add2(hi, lo);
  const f2 bp = sub2(s, hi);
  lo = add2(sub2(hi, sub2(s, bp)), sub2(lo, bp));
  hi = s;
}
// Adds a frame displacement to the lo parts of two hi/lo positions.
__device__ __forceinline__ void add_frame_disp2(f2& xl, f2& yl, const f2* __restrict__ P, f2 ds, f2 dh) {
  xl = fma2(ds, P[P_EX], fnma2(dh, P[P_EY], xl));
  yl = fma2(ds, P[P_EY], fma2(dh, P[P_EX], yl));
}

// VJP of one regeneration step for two pixels, in the displacement form of
// step_vjp_ext (tbr_internal.cuh): cap-to-cap components use its cap branch,
// flank-to-flank components its flank branch (evaluated only when a converged
// lane has one; a flank step has sin beta = 0).  Regenerated samples are never
// floored, and flank-to-cap steps take the scalar routines.
__device__ __forceinline__ f2 neg2(f2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void step_vjp2(const Geo2& q, const f2* __restrict__ P, f2& lamx, f2& lamy, f2 mua, f2 z,
                                          f2& gcx, f2& gcy, f2& gth, f2& gL, f2& gr) {
  const f2 ex = P[P_EX], ey = P[P_EY], L = P[P_L];
  const f2 ls = fma2(lamx, ex, mul2(lamy, ey));
  const f2 lh = fms2(lamy, ex, mul2(lamx, ey));
  const f2 gsn = mul2(q.sgs, ls), ghn = mul2(q.sgh, lh);
  const f2 gcvn = mul2(mua, P[P_IW]);               // minus the coverage's cotangent of sigma'
  // g . u(beta), g . u'(beta), g . u(phi), g . u'(phi)  (u(a) = (sin a, cos a), u' = (cos a, -sin a))
  const f2 gu = fma2(gsn, q.sb, mul2(ghn, q.cb));
  const f2 gup = fms2(gsn, q.cb, mul2(ghn, q.sb));
  const f2 guf = fma2(gsn, q.ud, mul2(ghn, q.uh));
  const f2 gufp = fms2(gsn, q.uh, mul2(ghn, q.ud));
  const f2 sgL = mul2(sub2(q.dsp, P[P_R]), q.iQ);   // d sigma / dL
  const f2 sgr = mul2(P[P_NPR], q.iQ);              // d sigma / dr
  const f2 dspL = mul2(q.dsp, L);
  const f2 sdphi = mul2(dspL, q.iQp);               // sigma delta_phi
  const f2 room = sub2(q.phi, F2(0.5f * kPiF));
  const f2 K = mul2(room, q.iQp);
  // cap to cap: g . dD/dsigma' and g . dD/dphi
  const f2 nsdsp = mul2(mul2(sdphi, room),
                        fma2(F2(kPiF), add2(q.iQ, q.iQp), mul2(mul2(q.Qp, q.iQ), q.isg)));  // -sigma delta_sigma'
  const f2 pdQ = mul2(mul2(F2(kPiF), q.dsp), q.iQ);
  const f2 g_sp = sub2(fma2(pdQ, gu, sub2(gu, guf)), fma2(nsdsp, gup, gcvn));
  const f2 g_ph = mul2(fma2(sub2(sdphi, q.dsp), gup, mul2(q.sp, sub2(gup, gufp))), q.isp);
  f2 ws = fma2(q.ud, g_sp, mul2(q.uh, g_ph));
  f2 wh = fms2(q.uh, g_sp, mul2(q.ud, g_ph));
  // explicit L and r through sigma and delta
  const f2 sdL = mul2(K, fnma2(dspL, fma2(sgL, q.isg, q.iQp), fma2(neg2(L), sgL, q.dsp)));
  const f2 nsdr = mul2(mul2(K, mul2(L, sgr)), mul2(q.sp, q.isg));  // -sigma delta_r
  f2 gLm = fma2(F2(-0.5f), ws, fma2(sgL, gu, mul2(sdL, gup)));
  f2 grm = fms2(sgr, gu, mul2(nsdr, gup));
  f2 th = fms2(sdphi, gup, mul2(P[P_HL], wh));
  const bool fx = q.sb.x == 0.0f, fy = q.sb.y == 0.0f;
  if (__any_sync(__activemask(), fx || fy)) {  // flank to flank
    const f2 as = abs2(q.si);
    const f2 pdQp = mul2(mul2(F2(kPiF), q.dsp), q.iQp);
    const f2 QQ = mul2(add2(q.Q, q.Qp), mul2(q.iQ, q.iQp));
    const f2 pas = mul2(F2(kPiF), as);
    const f2 wsf = mul2(neg2(gsn), pdQp);
    const f2 whf = sub2(fma2(gsn, mul2(mul2(pas, pdQp), QQ), mul2(ghn, pdQ)), gcvn);
    const f2 gLf = fma2(gsn, mul2(mul2(pas, fma2(q.dsp, q.iQp, sgL)), q.iQp), mul2(ghn, sgL));
    const f2 grf = fma2(gsn, mul2(mul2(pas, sgr), q.iQp), mul2(ghn, sgr));
    const f2 b1 = mul2(q.dsp, fma2(mul2(neg2(pas), pas), mul2(QQ, q.iQp), mul2(L, q.iQp)));
    const f2 b2 = mul2(neg2(pas), mul2(q.dsp, QQ));
    const f2 thf = fma2(as, gcvn, fma2(gsn, b1, mul2(ghn, b2)));
    ws = sel2(fx, fy, wsf, ws);
    wh = sel2(fx, fy, whf, wh);
    gLm = sel2(fx, fy, gLf, gLm);
    grm = sel2(fx, fy, grf, grm);
    th = sel2(fx, fy, thf, th);
  }
  gth = mul2(mul2(q.sgs, q.sgh), th);
  gL = gLm;
  gr = fma2(mua, fnma2(z, P[P_DLW], P[P_IW]), grm);
  const f2 GS = mul2(q.sgs, ws), GH = mul2(q.sgh, wh);
  // the centre's cotangent -dlambda, formed directly (the negations fold into the FFMA2 / FMUL2 operands)
  gcx = fms2(GH, ey, mul2(GS, ex));
  gcy = fnma2(GS, ey, mul2(neg2(GH), ex));
  lamx = sub2(lamx, gcx);
  lamy = sub2(lamy, gcy);
}

// Thread -> pixel pair of a 32 x 16 tile: column lane, rows 2 warp and 2 warp + 1.
__device__ __forceinline__ void pair_tile_pixel(int tile, int W, int& px, int& py0) {
  const int tiles_x = (W + kPairTileW - 1) / kPairTileW;
  px = (tile % tiles_x) * kPairTileW + (threadIdx.x & 31);
  py0 = (tile / tiles_x) * kPairTileH + 2 * (threadIdx.x >> 5);
}

// Soft forward (Eq. relax, Eq. state, floored psi) of a 32 x 16 tile, two
// pixels per thread, over strokes n-1 .. 0; otherwise as soft_forward_tile
// (exterior-transport model).  x0/y0[c], valid[c] and off[c] describe pixel c
// of the pair; an invalid pixel still carries a finite position.  pbuf and pext
// are shared [CH][kPairRec] and [CH][kPairExt] float2.  All threads of the CTA
// must call it.
template <int CH, bool RECORD>
__device__ bool soft_forward_tile2(ChunkRing<CH>& ring, const float* __restrict__ packed, int n,
                                   const bool (&valid)[2], const float (&x0)[2], const float (&y0)[2],
                                   const RecordView& rv, const size_t (&off)[2], f2* __restrict__ pbuf,
                                   f2* __restrict__ pext, PixelState (&st)[2], unsigned long long* status) {
  const bool any = valid[0] || valid[1];
  f2 Xh = make_float2(x0[0], x0[1]), Yh = make_float2(y0[0], y0[1]);
  f2 Xl = F2(0.0f), Yl = F2(0.0f), LT = F2(0.0f);
  f2 C0 = F2(0.0f), C1 = F2(0.0f), C2 = F2(0.0f);
  int cnt[2] = {0, 0};
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
    pair_records_fill<true>(S0, cntc, pbuf, pext);
    __syncthreads();
    if (any) {
      // one stroke (j: index in the chunk)
      auto stroke = [&](int j) {
        const int i1 = base + j + 1;  // the paper's 1-based stroke index
        const f2* P = pbuf + j * kPairRec;
        const f2* X = pext + j * kPairExt;
        const f2 dx = add2(sub2(Xh, P[P_MX]), Xl), dy = add2(sub2(Yh, P[P_MY]), Yl);
        const bool drop = P[P_L].x == 0.0f;  // warp-uniform
        f2 sp, ddx, ddy;
        int fix;
        if (drop) {
          fix = drop_pair(dx, dy, P, X, sp, ddx, ddy);
        } else {
          const f2 s = fma2(dx, P[P_EX], mul2(dy, P[P_EY]));
          const f2 h = fms2(dy, P[P_EX], mul2(dx, P[P_EY]));
          f2 ds, dh;
          fix = psi_pair(s, h, P, X, sp, ds, dh);
          ddx = fms2(ds, P[P_EX], mul2(dh, P[P_EY]));
          ddy = fma2(ds, P[P_EY], mul2(dh, P[P_EX]));
        }
        if (fix) {  // floored or cap to flank: scalar step per pixel
          const StrokeF g = load_stroke(S0 + j * kRec);
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            if (fix & (1 << c)) {
              const float dxc = comp(dx, c), dyc = comp(dy, c);
              float spc, ddxc, ddyc;
              bool floored;
              if (drop) {
                spc = drop_step<true>(dxc, dyc, g, ddxc, ddyc, floored);
              } else {
                const float s = fmaf(dxc, g.ex, dyc * g.ey), h = fmaf(dyc, g.ex, -dxc * g.ey);
                Geo gq;
                float ds, dh;
                psi_local<true>(s, h, g, gq, ds, dh);
                spc = gq.sp;
                floored = gq.floored;
                ddxc = fmaf(ds, g.ex, -dh * g.ey);
                ddyc = fmaf(ds, g.ey, dh * g.ex);
              }
              put(sp, c, spc); put(ddx, c, ddxc); put(ddy, c, ddyc);
              if (RECORD && floored && valid[c]) {
                if (cnt[c] < rv.cap) {
                  const size_t o = static_cast<size_t>(cnt[c]) * rv.stride + off[c];
                  rv.rec[o] = make_float4(comp(Xh, c), comp(Yh, c), comp(Xl, c), comp(Yl, c));
                  rv.rec_i[o] = i1;
                }
                ++cnt[c];
              }
            }
          }
        }
        const Cover2 cv = coverage2(sp, P);
        const f2 w = mul2(ex22(LT), cv.alpha);
        C0 = fma2(w, P[P_CR], C0);
        C1 = fma2(w, P[P_CG], C1);
        C2 = fma2(w, P[P_CB], C2);
        LT = sub2(LT, cv.sp2);  // log2 T_{i-1} = log2 T_i + log2(1 - alpha_i)
        Xl = add2(Xl, ddx);
        Yl = add2(Yl, ddy);
      };
      auto checkpoint = [&](int i1) {
        const size_t o = static_cast<size_t>(i1 / ck - 1) * rv.stride;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (valid[c]) {
            rv.ckpt[o + off[c]] = make_float4(comp(Xh, c), comp(Yh, c), comp(Xl, c), comp(Yl, c));
            rv.ck_lt[o + off[c]] = comp(LT, c);
          }
        }
        next_ck -= ck;
      };
      // blocks of kRenorm strokes aligned to the stroke index, as soft_forward_tile
      const bool ck_aligned = (ck & (kRenorm - 1)) == 0;
      for (int hi = cntc - 1; hi >= 0;) {
        const int lo = hi & ~(kRenorm - 1);
        if (!RECORD || ck_aligned) {
          if (RECORD && base + hi + 1 == next_ck) checkpoint(base + hi + 1);
          for (int j = hi; j >= lo; --j) stroke(j);
        } else {
          for (int j = hi; j >= lo; --j) {
            if (base + j + 1 == next_ck) checkpoint(base + j + 1);
            stroke(j);
          }
        }
        pos_renorm2(Xh, Xl);
        pos_renorm2(Yh, Yl);
        hi = lo - 1;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && q + 2 < nch) ring.issue(b, chunk_src(q + 2), chunk_cnt(q + 2));
  }
#pragma unroll
  for (int c = 0; c < 2; ++c)
    st[c] = PixelState{comp(Xh, c), comp(Yh, c), comp(Xl, c), comp(Yl, c), comp(LT, c), cnt[c],
                       comp(C0, c), comp(C1, c), comp(C2, c)};
  return ok;
}

// Adjoint state of one pixel in the scalar fallback.
struct PixAdj {
  float xh, yh, xl, yl;  // x_{i-1} (hi/lo), replaced by x_i
  float lt;              // log2 T_{i-1}, replaced by log2 T_i
  float lD;              // lambda^C . c_{i-1} - lambda^T_{i-1} (0 before stroke 1), replaced by its value at i
  float lx, ly;          // lambda^x
};

// One stroke of the replay adjoint for one pixel in scalar arithmetic, as in
// backward_tile: x_i from the side table (pop), from Phi_i followed by a reset
// to the checkpoint (at_ck), or from Phi_i; log2 T_i from the checkpoint or
// Eq. rT; then the adjoint step and the VJP, whose 8 gradient values are
// written to v.  P is the stroke's pair record (its colour fields hold the
// colour step c_i - c_{i-1}, pair_records_fill).  Returns true if, at a
// checkpoint of a valid pixel, the regenerated position differed from the
// stored one by more than drift_tol.
__device__ __forceinline__ bool scalar_stroke(PixAdj& a, const StrokeF& g, const f2* __restrict__ P, float lC0,
                                              float lC1, float lC2, bool pop, bool at_ck, bool valid, float4 rp,
                                              float4 ckp, float ck_lt, float drift_tol, float (&v)[8]) {
  Geo gq;
  float s, h, ds, dh;
  bool drifted = false;
  if (pop) {
    // x_i was within the floor's reach: read it back (Lemma "Support of the replay record")
    a.xh = rp.x; a.yh = rp.y; a.xl = rp.z; a.yl = rp.w;
    to_frame(a.xh, a.yh, a.xl, a.yl, g, s, h);
    psi_local<true>(s, h, g, gq, ds, dh);
  } else if (at_ck) {
    // regenerate, measure the drift against the stored position, then reset to it
    to_frame(a.xh, a.yh, a.xl, a.yl, g, s, h);
    phi_local(s, h, g, gq, ds, dh);
    add_frame_disp(a.xh, a.yh, a.xl, a.yl, g, ds, dh);
    if (valid) {
      drifted = fabsf((a.xh - ckp.x) + (a.xl - ckp.z)) > drift_tol ||
                fabsf((a.yh - ckp.y) + (a.yl - ckp.w)) > drift_tol;
      a.xh = ckp.x; a.yh = ckp.y; a.xl = ckp.z; a.yl = ckp.w;
    }
    to_frame(a.xh, a.yh, a.xl, a.yl, g, s, h);
    psi_local<true>(s, h, g, gq, ds, dh);
  } else {
    to_frame(a.xh, a.yh, a.xl, a.yl, g, s, h);
    phi_local(s, h, g, gq, ds, dh);
    add_frame_disp(a.xh, a.yh, a.xl, a.yl, g, ds, dh);
  }
  const Cover cv = coverage(gq.sp, g);
  if (at_ck) a.lt = ck_lt; else a.lt += cv.sp2;
  const float T = ex2_a(a.lt);
  // lambda^C . c_i - lambda^T_{i-1}, carried as a difference (see pair_stroke)
  const float E = a.lD + fmaf(lC0, P[P_CR].x, fmaf(lC1, P[P_CG].x, lC2 * P[P_CB].x));
  const float mu = T * E;
  const float Ta = T * cv.alpha;
  v[5] = lC0 * Ta; v[6] = lC1 * Ta; v[7] = lC2 * Ta;
  step_vjp(gq, g, a.lx, a.ly, mu * cv.dadz, cv.z, v[0], v[1], v[2], v[3], v[4]);
  a.lD = cv.oma * E;
  return drifted;
}

// Adjoint state of a pixel pair (component c = pixel c).
struct PairState {
  f2 Xh, Yh, Xl, Yl;  // x_{i-1}, hi/lo
  f2 LT;              // log2 T_{i-1}
  f2 LD, LX, LY;      // lambda^C . c_{i-1} - lambda^T_{i-1} (see pair_stroke), lambda^x
  f2 LC0, LC1, LC2;   // lambda^C_0 (constant)
  int rc[2], nri[2];  // side-table records left; stroke index of the top one (-1: none)
};

// Initial pair state from the forward's s_0 and the cotangent (Eq. adjstep
// initial values: lambda^T_0 = lambda^C_0 . c_0, so LD = 0; lambda^x_0 = 0).
__device__ __forceinline__ void pair_state_init(PairState& ps, const bool (&valid)[2], const PixelState (&st)[2],
                                                const float (&lC)[2][3], const RecordView& rv,
                                                const size_t (&off)[2]) {
  ps.Xh = make_float2(st[0].xh, st[1].xh); ps.Yh = make_float2(st[0].yh, st[1].yh);
  ps.Xl = make_float2(st[0].xl, st[1].xl); ps.Yl = make_float2(st[0].yl, st[1].yl);
  ps.LT = make_float2(st[0].lt, st[1].lt);
  ps.LC0 = make_float2(lC[0][0], lC[1][0]); ps.LC1 = make_float2(lC[0][1], lC[1][1]);
  ps.LC2 = make_float2(lC[0][2], lC[1][2]);
  ps.LD = F2(0.0f);
  ps.LX = F2(0.0f); ps.LY = F2(0.0f);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    ps.rc[c] = valid[c] ? min(st[c].cnt, rv.cap) : 0;
    ps.nri[c] = ps.rc[c] > 0 ? rv.rec_i[static_cast<size_t>(ps.rc[c] - 1) * rv.stride + off[c]] : -1;
  }
}

// The pixel pair (px, py0), (px, py0 + 1) as k_backward2 starts it: validity,
// record offsets, the forward's s_0 and the cotangent.  An invalid pixel keeps
// a finite position and a zero cotangent.
__device__ __forceinline__ void load_pair(const BwdArgs& a, int px, int py0, bool skip, bool (&valid)[2],
                                          size_t (&off)[2], PixelState (&st)[2], float (&lC)[2][3]) {
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int py = py0 + c;
    valid[c] = px < a.W && py < a.H && !skip;
    off[c] = valid[c] ? static_cast<size_t>(py) * a.W + px : 0;
    st[c] = PixelState{(static_cast<float>(px) + 0.5f) / static_cast<float>(a.W),
                       (static_cast<float>(py) + 0.5f) / static_cast<float>(a.H), 0.0f, 0.0f, 0.0f, 0,
                       0.0f, 0.0f, 0.0f};
    lC[c][0] = lC[c][1] = lC[c][2] = 0.0f;
    if (valid[c]) {
      const float4 s0 = a.s0[off[c]];
      const float2 s0b = a.s0b[off[c]];
      st[c].xh = s0.x; st[c].yh = s0.y; st[c].xl = s0.z; st[c].yl = s0.w;
      st[c].lt = s0b.x;
      st[c].cnt = __float_as_int(s0b.y);
      lC[c][0] = a.dLdR[3 * off[c] + 0];
      lC[c][1] = a.dLdR[3 * off[c] + 1];
      lC[c][2] = a.dLdR[3 * off[c] + 2];
    }
  }
}

// Stroke i1 of the paired replay adjoint (S: packed record, P: pair record;
// at_ck / cko: checkpoint stroke and its record offset; renorm: i1 is a
// multiple of kRenorm, after which a regenerated position is renormalised).
// Writes each pixel's 8 gradient values to g[c][.].  At a checkpoint, counts
// in drift the pixels whose regenerated position drifted past rv.drift_tol
// and, with QUEUE, queues a pixel's first drifting segment on rv.repair_list.
template <bool QUEUE>
__device__ __forceinline__ void pair_stroke(PairState& ps, const float* __restrict__ S, const f2* __restrict__ P,
                                            int i1, bool at_ck, size_t cko, bool renorm, const RecordView& rv,
                                            const bool (&valid)[2], const size_t (&off)[2], float (&g)[2][8],
                                            unsigned& drift) {
  const bool pop0 = i1 == ps.nri[0], pop1 = i1 == ps.nri[1];
  bool scalar = at_ck || pop0 || pop1;
  Geo2 gq;
  f2 ds, dh;
  if (!scalar) {
    // x_i = Phi_i(x_{i-1}) (Eq. rpos), both pixels at once
    f2 s, h;
    to_frame2(ps.Xh, ps.Yh, ps.Xl, ps.Yl, P, s, h);
    scalar = phi_pair(s, h, P, gq, ds, dh) != 0;  // flank to cap: redo this stroke per pixel
  }
  if (scalar) {
    const StrokeF sg = load_stroke(S);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const bool pop = c == 0 ? pop0 : pop1;
      float4 rp = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (pop) {
        rp = rv.rec[static_cast<size_t>(ps.rc[c] - 1) * rv.stride + off[c]];
        --ps.rc[c];
        ps.nri[c] = ps.rc[c] > 0 ? rv.rec_i[static_cast<size_t>(ps.rc[c] - 1) * rv.stride + off[c]] : -1;
      }
      float4 ckp = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      float ckl = 0.0f;
      if (at_ck && valid[c]) {
        ckp = rv.ckpt[cko + off[c]];
        ckl = rv.ck_lt[cko + off[c]];
      }
      PixAdj a{comp(ps.Xh, c), comp(ps.Yh, c), comp(ps.Xl, c), comp(ps.Yl, c), comp(ps.LT, c), comp(ps.LD, c),
               comp(ps.LX, c), comp(ps.LY, c)};
      if (scalar_stroke(a, sg, P, comp(ps.LC0, c), comp(ps.LC1, c), comp(ps.LC2, c), pop, at_ck, valid[c], rp,
                        ckp, ckl, rv.drift_tol, g[c])) {
        ++drift;
        // first drift of this pixel: queue the segment (i1 - ck, i1] for the FP64 repair
        if (QUEUE && rv.repair_first[off[c]] == 0) {
          rv.repair_first[off[c]] = 1;
          const int idx = atomicAdd(rv.repair_count, 1);
          if (idx < rv.repair_cap) rv.repair_list[idx] = make_int2(static_cast<int>(off[c]), i1 - rv.ck);
        }
      }
      put(ps.Xh, c, a.xh); put(ps.Yh, c, a.yh); put(ps.Xl, c, a.xl); put(ps.Yl, c, a.yl);
      put(ps.LT, c, a.lt); put(ps.LD, c, a.lD); put(ps.LX, c, a.lx); put(ps.LY, c, a.ly);
    }
  } else {
    add_frame_disp2(ps.Xl, ps.Yl, P, ds, dh);
    if (renorm) {
      pos_renorm2(ps.Xh, ps.Xl);
      pos_renorm2(ps.Yh, ps.Yl);
    }
    const Cover2 cv = coverage2(gq.sp, P);
    ps.LT = add2(ps.LT, cv.sp2);  // log T_i = log T_{i-1} - log(1 - alpha_i)
    const f2 T = ex22(ps.LT);
    // mu = T_i (lambda^C . c_i - lambda^T_{i-1}).  lambda^T tracks the colour
    // composited behind stroke i, which for strokes coloured like those behind
    // them differs from c_i only by (c_i - c_0) times the transmittance behind;
    // as a difference of two such numbers it would keep only eps / (that
    // transmittance) of its relative precision.  So the difference itself is
    // carried: LD_i = lambda^C . c_i - lambda^T_i = (1 - alpha_i) E_i, with
    // E_i = LD_{i-1} + lambda^C . (c_i - c_{i-1}) and LD_0 = 0 (lambda^T_0 =
    // lambda^C . c_0); the pair record holds the colour step.
    const f2 E = add2(ps.LD, fma2(ps.LC0, P[P_CR], fma2(ps.LC1, P[P_CG], mul2(ps.LC2, P[P_CB]))));
    const f2 mu = mul2(T, E);
    const f2 Ta = mul2(T, cv.alpha);
    const f2 c5 = mul2(ps.LC0, Ta), c6 = mul2(ps.LC1, Ta), c7 = mul2(ps.LC2, Ta);
    f2 gcx, gcy, gth, gL, gr;
    step_vjp2(gq, P, ps.LX, ps.LY, mul2(mu, cv.dadz), cv.z, gcx, gcy, gth, gL, gr);
    ps.LD = mul2(cv.oma, E);
    g[0][0] = gcx.x; g[0][1] = gcy.x; g[0][2] = gth.x; g[0][3] = gL.x; g[0][4] = gr.x;
    g[0][5] = c5.x; g[0][6] = c6.x; g[0][7] = c7.x;
    g[1][0] = gcx.y; g[1][1] = gcy.y; g[1][2] = gth.y; g[1][3] = gL.y; g[1][4] = gr.y;
    g[1][5] = c5.y; g[1][6] = c6.y; g[1][7] = c7.y;
  }
}

// ---------------------------------------------------------------------------
// The paired replay adjoint of the coupling variant Phi_g (Eq. coupling, Eq.
// profile).  Its pair extension record holds the floor constants and the
// profile cubic of each staged stroke.
// ---------------------------------------------------------------------------
enum : int { XG_KA = 0, XG_FL2 = 1, XG_G0 = 2, XG_G1 = 3, XG_G2 = 4, XG_G3 = 5, kPairExtG = 6 };

// All threads: fill the coupling extension of the cnt strokes staged at S0.
__device__ __forceinline__ void pair_ext_g_fill(const float* __restrict__ S0, int cnt, f2* __restrict__ gext) {
  for (int e = threadIdx.x; e < cnt * kPairExtG; e += kTileThreads) {
    const int j = e / kPairExtG, k = e - j * kPairExtG;
    gext[e] = F2(S0[j * kRec + (k < 2 ? F_KA + k : F_G0 + k - 2)]);
  }
}

// g - 1 at the angle 4 pi v, for two pixels (as profile_gm1).
__device__ __forceinline__ f2 profile_gm1_2(f2 ang, const f2* __restrict__ X) {
  const f2 a = sub2(min2(max2(ang, F2(0.0f)), F2(kPiF)), F2(0.5f * kPiF));
  const f2 w = neg2(sin_pi2_2(a));
  return fma2(w, fma2(w, fma2(w, X[XG_G3], X[XG_G2]), X[XG_G1]), X[XG_G0]);
}

// x_i = Phi_g,i(x_{i-1}) for two pixels at frame points (s, h) of x_{i-1}, in
// the displacement form of phi_local<true>: the normal step adds A_L(r) g(v),
// v the centred arclength of the point's own leaf (on a drop, beta / (2 pi)).
// Returns the mask of the pixels whose step goes from the flank onto a cap;
// their outputs are not valid and the caller recomputes them with phi_local.
__device__ __forceinline__ int phi_pair_g(f2 s, f2 h, const f2* __restrict__ P, const f2* __restrict__ X, f2& ds,
                                          f2& dh) {
  const f2 L = P[P_L], Ar = P[P_AR];
  const f2 sgs = sgn2(s), sgh = sgn2(h);
  const f2 as = abs2(s), ah = abs2(h);
  if (L.x == 0.0f) {  // drop: radial (warp-uniform branch)
    const f2 x2 = fma2(as, as, mul2(ah, ah));
    const f2 is = rsqrt2(max2(x2, F2(kTiny)));  // 1 / sigma
    const f2 sig = mul2(x2, is);
    const f2 sb = mul2(as, is);
    const f2 cb = sel2(x2.x > 0.0f, x2.y > 0.0f, mul2(ah, is), F2(1.0f));
    const f2 beta = atan2_pos2(as, ah);
    const f2 Ag = fma2(Ar, profile_gm1_2(add2(beta, beta), X), Ar);
    const f2 sp = sqrt2(mul2(fma2(sig, mul2(F2(kPiF), sig), Ag), F2(1.0f / kPiF)));
    const f2 dsp = mul2(Ag, rcp2(mul2(F2(kPiF), add2(sig, sp))));
    ds = mul2(sgs, mul2(dsp, sb));
    dh = mul2(sgh, mul2(dsp, cb));
    return 0;
  }
  const f2 hl = P[P_HL];
  const f2 d = sub2(as, hl);
  const bool co_x = d.x > 0.0f, co_y = d.y > 0.0f;
  const f2 dp = max2(d, F2(0.0f));
  const f2 x2 = fma2(dp, dp, mul2(ah, ah));
  const f2 is = rsqrt2(max2(x2, F2(kTiny)));  // 1 / sigma
  const f2 sig = mul2(x2, is);
  const f2 sb = mul2(dp, is);
  const f2 cb = sel2(co_x, co_y, mul2(ah, is), F2(1.0f));
  const f2 beta = atan2_pos2(dp, ah);
  const f2 tn = fma2(sig, beta, min2(as, hl));
  const f2 iQ = rcp2(fma2(F2(kPiF), sig, L));
  const f2 Ag = fma2(Ar, profile_gm1_2(mul2(F2(2.0f * kPiF), mul2(tn, iQ)), X), Ar);  // 4 pi v = 2 pi t / Q
  const f2 B = fma2(sig, fma2(F2(kPiF), sig, P[P_2L]), Ag);
  const f2 sp = mul2(B, rcp2(add2(L, sqrt2(fma2(F2(kPiF), B, P[P_L2])))));
  const f2 dsp = mul2(Ag, rcp2(fma2(F2(kPiF), add2(sig, sp), P[P_2L])));
  const f2 t = mul2(tn, mul2(fma2(F2(kPiF), sp, L), iQ));
  const bool ci_x = t.x > hl.x, ci_y = t.y > hl.y;
  // cap to cap: rotation by delta, clamped to the cap; on the flank delta = 0
  // and (sb, cb) = (0, 1), so the cap's dH is the flank's dsigma'
  const f2 room = sub2(F2(0.5f * kPiF), beta);
  f2 delta = mul2(mul2(mul2(dsp, L), room), mul2(iQ, rcp2(sp)));
  delta = sel2(co_x, co_y, min2(max2(delta, F2(0.0f)), room), F2(0.0f));
  const f2 sD = sin_pi2_2(delta), omc = omc_pi2_2(delta);
  const f2 dSc = fma2(dsp, sb, mul2(sp, sub2(mul2(cb, sD), mul2(sb, omc))));
  const f2 dH = sub2(mul2(dsp, cb), mul2(sp, fma2(sb, sD, mul2(cb, omc))));
  const f2 dSf = mul2(mul2(tn, F2(kPiF)), mul2(dsp, iQ));  // flank to flank
  ds = mul2(sgs, sel2(co_x, co_y, dSc, dSf));
  dh = mul2(sgh, dH);
  return ((!co_x && ci_x) ? 1 : 0) | ((!co_y && ci_y) ? 2 : 0);
}

// Pair form of coupled_vjp (tbr_coupled_vjp.cuh) at the hi/lo positions x_i of
// two pixels: the same primal and reverse pass, written branch-free for the
// cap-to-cap rotation and the flank (on the flank (ud, uh, phi) = (0, 1, 0)
// clamps delta to 0, so the rotation's formulas give dH, and the flank's own dS
// terms are added under a warp vote).  Returns the mask of pixels in the direct
// form (floored, or cap to flank); their G, alpha and oma are not valid and the
// caller recomputes them with coupled_vjp.  seed(alpha, oma, sp2, lx, ly, mu)
// as in coupled_vjp, for both pixels.
template <class Seed>
__device__ __forceinline__ int coupled_vjp2(f2 Xh, f2 Yh, f2 Xl, f2 Yl, const f2* __restrict__ P,
                                            const f2* __restrict__ X, Seed&& seed, f2 (&G)[5], f2& alpha, f2& oma) {
  const f2 ex = P[P_EX], ey = P[P_EY], L = P[P_L], r = P[P_R], hl = P[P_HL], Ar = P[P_AR], kA = X[XG_KA];
  const f2 dxw = add2(sub2(Xh, P[P_MX]), Xl), dyw = add2(sub2(Yh, P[P_MY]), Yl);
  const f2 s = fma2(dxw, ex, mul2(dyw, ey)), h = sub2(mul2(dyw, ex), mul2(dxw, ey));
  const f2 sgs = sgn2(s), sgh = sgn2(h);
  const f2 as = abs2(s), ah = abs2(h);
  // ---- primal
  const f2 d = sub2(as, hl);
  const bool ci_x = d.x > 0.0f, ci_y = d.y > 0.0f;
  const f2 dp = max2(d, F2(0.0f));
  const f2 x2 = fma2(dp, dp, mul2(ah, ah));
  const f2 inv = rsqrt2(max2(x2, F2(kTiny)));  // 1 / sigma'
  const f2 sp = mul2(x2, inv);
  const f2 ud = mul2(dp, inv);
  const f2 uh = sel2(ci_x, ci_y, mul2(ah, inv), F2(1.0f));
  const f2 phi = atan2_pos2(dp, ah);
  const f2 t = fma2(sp, phi, min2(as, hl));
  const f2 iQp = rcp2(fma2(F2(kPiF), sp, L));
  const f2 am = fma2(F2(2.0f * kPiF), mul2(t, iQp), F2(-0.5f * kPiF));  // 4 pi v - pi/2
  const f2 w = neg2(sin_pi2_2(am));
  const f2 gm1 = fma2(w, fma2(w, fma2(w, X[XG_G3], X[XG_G2]), X[XG_G1]), X[XG_G0]);
  const f2 Ag = fma2(Ar, gm1, Ar);
  const f2 kAs = fma2(F2(kPiF), sp, kA);
  const f2 spr = sub2(sp, r);
  const f2 C = fma2(spr, kAs, neg2(mul2(Ar, gm1)));
  const bool fl_x = C.x < X[XG_FL2].x, fl_y = C.y < X[XG_FL2].y;
  const f2 rin = fma2(F2(kPiF), C, P[P_L2]);
  const f2 iroot = rsqrt2(max2(rin, F2(kTiny)));
  const f2 iden1 = rcp2(fma2(rin, iroot, L));
  const f2 sig = mul2(C, iden1);
  const f2 Q = fma2(F2(kPiF), sig, L);
  const f2 tn = mul2(t, mul2(Q, iQp));
  const bool co_x = tn.x > hl.x, co_y = tn.y > hl.y;
  const int mask = ((fl_x || (ci_x && !co_x)) ? 1 : 0) | ((fl_y || (ci_y && !co_y)) ? 2 : 0);
  const f2 iden2 = rcp2(fma2(F2(kPiF), add2(sp, sig), P[P_2L]));
  const f2 dsig = neg2(mul2(Ag, iden2));
  const f2 isig = rcp2(sig);
  const f2 Pm = sub2(phi, F2(0.5f * kPiF));
  const f2 k0 = mul2(Pm, mul2(iQp, isig));
  const f2 delta0 = neg2(mul2(mul2(dsig, L), k0));
  const bool c1x = delta0.x < -phi.x, c1y = delta0.y < -phi.y;
  f2 delta = sel2(c1x, c1y, neg2(phi), delta0);
  const bool c2x = delta.x > 0.0f, c2y = delta.y > 0.0f;
  delta = sel2(c2x, c2y, F2(0.0f), delta);
  const f2 sD = sin_pi2_2(delta), omc = omc_pi2_2(delta);
  const f2 cD = sub2(F2(1.0f), omc);
  const f2 sigsD = mul2(sig, sD), sigomc = mul2(sig, omc);
  const f2 pQ = mul2(F2(kPiF), iQp);
  const f2 dS = sel2(ci_x, ci_y, fma2(dsig, ud, sub2(mul2(uh, sigsD), mul2(ud, sigomc))), mul2(mul2(as, pQ), dsig));
  const f2 dH = sub2(mul2(dsig, uh), fma2(ud, sigsD, mul2(uh, sigomc)));
  // coverage from the deposit boundary sigma_b(v)
  const f2 cin = fma2(F2(kPiF), Ag, P[P_L2]);
  const f2 iR2 = rsqrt2(max2(cin, F2(kTiny)));
  const f2 iD2 = rcp2(fma2(cin, iR2, L));
  const f2 rb = mul2(Ag, iD2);
  const f2 iw = P[P_IW];
  const f2 z = mul2(sub2(rb, sp), iw);
  const bool clx = z.x > kZMax, cly = z.y > kZMax;
  const f2 ez = ex22(mul2(min2(z, F2(kZMax)), F2(kLog2e)));
  const f2 opl = add2(F2(1.0f), ez);
  oma = rcp2(opl);
  alpha = mul2(ez, oma);
  f2 lx, ly, mu;
  seed(alpha, oma, lg22(opl), lx, ly, mu);

  // ---- reverse
  const f2 ls = fma2(lx, ex, mul2(ly, ey)), lh = sub2(mul2(ly, ex), mul2(lx, ey));
  const f2 b_dS = mul2(sgs, ls), b_dH = mul2(sgh, lh);
  const f2 b_z = sel2(clx, cly, F2(0.0f), mul2(mu, mul2(alpha, oma)));
  const f2 b_rb = mul2(b_z, iw);
  f2 b_sp = neg2(b_rb);
  f2 b_r = neg2(mul2(mul2(b_z, z), P[P_DLW]));
  const f2 b_D2 = neg2(mul2(mul2(b_rb, rb), iD2));
  const f2 b_cin = mul2(mul2(b_D2, F2(0.5f)), iR2);
  f2 b_Ag = fma2(F2(kPiF), b_cin, mul2(b_rb, iD2));
  f2 b_L = fma2(P[P_2L], b_cin, b_D2);
  // cap-to-cap rotation (the flank's terms follow)
  f2 b_dsig = fma2(b_dS, ud, mul2(b_dH, uh));
  f2 b_sig = sub2(mul2(b_dS, sub2(mul2(uh, sD), mul2(ud, omc))), mul2(b_dH, fma2(ud, sD, mul2(uh, omc))));
  const f2 dso = sub2(dsig, sigomc);
  const f2 b_ud = sub2(mul2(b_dS, dso), mul2(b_dH, sigsD));
  const f2 b_uh = fma2(b_dS, sigsD, mul2(b_dH, dso));
  const f2 b_sD = mul2(sig, sub2(mul2(b_dS, uh), mul2(b_dH, ud)));
  const f2 b_omc = neg2(mul2(sig, fma2(b_dS, ud, mul2(b_dH, uh))));
  const f2 b_delta = fma2(b_sD, cD, mul2(b_omc, sD));
  // delta free, clamped at -phi, or clamped at 0
  const f2 bdf = sel2(!c1x && !c2x, !c1y && !c2y, b_delta, F2(0.0f));
  f2 b_phi = sel2(c1x && !c2x, c1y && !c2y, neg2(b_delta), F2(0.0f));
  const f2 kd = neg2(mul2(bdf, mul2(dsig, L)));
  b_dsig = fma2(neg2(mul2(bdf, L)), k0, b_dsig);
  b_L = fma2(neg2(mul2(bdf, dsig)), k0, b_L);
  b_phi = fma2(kd, mul2(iQp, isig), b_phi);
  f2 b_iQp = mul2(kd, mul2(Pm, isig));
  b_sig = fma2(neg2(mul2(bdf, delta)), isig, b_sig);
  f2 b_as = F2(0.0f);
  if (__any_sync(__activemask(), !ci_x || !ci_y)) {
    // flank to flank: dS = pi |s| dsig / Q' (dH = dsig is the rotation's on the flank)
    const f2 fq = sel2(ci_x, ci_y, F2(0.0f), mul2(b_dS, pQ));
    b_dsig = fma2(fq, as, b_dsig);
    b_as = mul2(fq, dsig);
    b_iQp = fma2(sel2(ci_x, ci_y, F2(0.0f), mul2(b_dS, F2(kPiF))), mul2(as, dsig), b_iQp);
  }
  // dsig = -Ag / (pi (sp + sig) + 2L)
  const f2 b_den2 = neg2(mul2(mul2(b_dsig, dsig), iden2));
  b_Ag = fma2(neg2(b_dsig), iden2, b_Ag);
  b_sp = fma2(F2(kPiF), b_den2, b_sp);
  b_sig = fma2(F2(kPiF), b_den2, b_sig);
  b_L = fma2(F2(2.0f), b_den2, b_L);
  // sig = C / (L + sqrt(pi C + L^2))
  const f2 b_den1 = neg2(mul2(mul2(b_sig, sig), iden1));
  const f2 b_rin = mul2(mul2(b_den1, F2(0.5f)), iroot);
  const f2 b_C = fma2(F2(kPiF), b_rin, mul2(b_sig, iden1));
  b_L = fma2(P[P_2L], b_rin, add2(b_L, b_den1));
  // C = (sp - r)(2L + pi (r + sp)) - A_L(r) (g - 1); Ag = A_L(r) (1 + (g - 1))
  b_sp = fma2(b_C, fma2(F2(kPiF), spr, kAs), b_sp);
  b_r = fma2(neg2(b_C), kAs, b_r);
  f2 b_kA = mul2(b_C, spr);
  const f2 bAC = sub2(b_Ag, b_C);
  const f2 b_Ar = fma2(gm1, bAC, b_Ag);
  const f2 b_gm1 = mul2(Ar, bAC);
  // the cubic in w = cos 4 pi v = -sin(am)
  const f2 b_w = mul2(b_gm1, fma2(w, fma2(mul2(F2(3.0f), X[XG_G3]), w, mul2(F2(2.0f), X[XG_G2])), X[XG_G1]));
  const f2 b_ang = neg2(mul2(mul2(b_w, F2(2.0f * kPiF)), sub2(F2(1.0f), omc_pi2_2(am))));
  const f2 b_t = mul2(b_ang, iQp);
  b_iQp = fma2(b_ang, t, b_iQp);
  const f2 b_Qp = neg2(mul2(mul2(b_iQp, iQp), iQp));
  b_L = add2(b_L, b_Qp);
  b_sp = fma2(F2(kPiF), b_Qp, b_sp);
  // t = sp phi + min(|s|, L/2); on a cap u = (d, |h|) / sp, phi = atan2(d, |h|)
  b_sp = fma2(b_t, phi, b_sp);
  b_phi = fma2(b_t, sp, b_phi);
  const f2 ub = fma2(ud, b_ud, mul2(uh, b_uh));
  const f2 bdd = sel2(ci_x, ci_y, fma2(fma2(b_phi, uh, fma2(neg2(ud), ub, b_ud)), inv, mul2(b_sp, ud)), F2(0.0f));
  const f2 b_ah = fma2(fma2(neg2(b_phi), ud, fma2(neg2(uh), ub, b_uh)), inv, mul2(b_sp, uh));
  b_as = add2(b_as, add2(bdd, sel2(ci_x, ci_y, F2(0.0f), b_t)));
  b_L = fma2(F2(0.5f), sel2(ci_x, ci_y, sub2(b_t, bdd), F2(0.0f)), b_L);
  // A_L(r) = (2L + pi r) r
  b_kA = fma2(b_Ar, r, b_kA);
  b_r = fma2(b_Ar, kA, b_r);
  b_L = fma2(F2(2.0f), b_kA, b_L);
  b_r = fma2(F2(kPiF), b_kA, b_r);
  // frame, and the rotation of the displacement back to world
  const f2 g_s = mul2(sgs, b_as), g_h = mul2(sgh, b_ah);
  const f2 dsw = mul2(sgs, dS), dhw = mul2(sgh, dH);
  const f2 ddx = sub2(mul2(dsw, ex), mul2(dhw, ey)), ddy = fma2(dsw, ey, mul2(dhw, ex));
  G[0] = sub2(mul2(g_s, ex), mul2(g_h, ey));
  G[1] = fma2(g_s, ey, mul2(g_h, ex));
  G[2] = add2(sub2(mul2(g_s, h), mul2(g_h, s)), sub2(mul2(ly, ddx), mul2(lx, ddy)));
  G[3] = b_L;
  G[4] = b_r;
  return mask;
}

// One stroke of the Phi_g replay adjoint for one pixel in scalar arithmetic:
// x_i from the side table (pop), from Phi_g,i followed by a reset to the
// checkpoint (at_ck), or from Phi_g,i; log2 T_i from the checkpoint or Eq. rT;
// then the step VJP (coupled_vjp), whose 8 gradient values are written to v.
// Returns true if, at a checkpoint of a valid pixel, the regenerated position
// differed from the stored one by more than drift_tol.
__device__ __forceinline__ bool coupled_stroke(PixAdj& a, const StrokeF& g, const float* __restrict__ S,
                                               const f2* __restrict__ P, float lC0, float lC1, float lC2, bool pop,
                                               bool at_ck, bool valid, float4 rp, float4 ckp, float ck_lt,
                                               float drift_tol, float (&v)[8]) {
  bool drifted = false;
  if (pop) {
    // x_i was within the floor's reach: read it back (Lemma "Support of the replay record")
    a.xh = rp.x; a.yh = rp.y; a.xl = rp.z; a.yl = rp.w;
  } else {
    Geo gq;
    float s, h, ds, dh;
    to_frame(a.xh, a.yh, a.xl, a.yl, g, s, h);
    phi_local<true>(s, h, g, gq, ds, dh, *reinterpret_cast<const float4*>(S + F_G0));
    add_frame_disp(a.xh, a.yh, a.xl, a.yl, g, ds, dh);
    if (at_ck && valid) {  // measure the drift against the stored position, then reset to it
      drifted = fabsf((a.xh - ckp.x) + (a.xl - ckp.z)) > drift_tol ||
                fabsf((a.yh - ckp.y) + (a.yl - ckp.w)) > drift_tol;
      a.xh = ckp.x; a.yh = ckp.y; a.xl = ckp.z; a.yl = ckp.w;
    }
  }
  const float E = a.lD + fmaf(lC0, P[P_CR].x, fmaf(lC1, P[P_CG].x, lC2 * P[P_CB].x));  // as scalar_stroke
  float G[5], alpha, oma, T = 0.0f;
  coupled_vjp(a.xh, a.yh, a.xl, a.yl, S,
              [&](float, float, float sp2, float& sx, float& sy, float& smu) {
                if (at_ck) a.lt = ck_lt; else a.lt += sp2;
                T = ex2_a(a.lt);
                sx = a.lx;
                sy = a.ly;
                smu = T * E;
              },
              G, alpha, oma);
  const float Ta = T * alpha;
  v[5] = lC0 * Ta; v[6] = lC1 * Ta; v[7] = lC2 * Ta;
  // psi_g and alpha depend on x_i - m, so d/dm = -d/dx
  v[0] = -G[0]; v[1] = -G[1]; v[2] = G[2]; v[3] = G[3]; v[4] = G[4];
  a.lx += G[0];
  a.ly += G[1];
  a.lD = oma * E;
  return drifted;
}

// Stroke i1 of the paired replay adjoint under Phi_g (X: the coupling
// extension record), as pair_stroke: pops, checkpoints and flank-to-cap
// regeneration take coupled_stroke per pixel, and a pixel whose step VJP is in
// the direct form takes coupled_vjp from the same x_i.
__device__ __forceinline__ void pair_stroke_g(PairState& ps, const float* __restrict__ S, const f2* __restrict__ P,
                                              const f2* __restrict__ X, int i1, bool at_ck, size_t cko,
                                              const RecordView& rv, const bool (&valid)[2], const size_t (&off)[2],
                                              float (&g)[2][8], unsigned& drift) {
  const bool pop0 = i1 == ps.nri[0], pop1 = i1 == ps.nri[1];
  bool scalar = at_ck || pop0 || pop1;
  if (!scalar) {
    // x_i = Phi_g,i(x_{i-1}) (Eq. rpos), both pixels at once
    f2 s, h, ds, dh;
    to_frame2(ps.Xh, ps.Yh, ps.Xl, ps.Yl, P, s, h);
    scalar = phi_pair_g(s, h, P, X, ds, dh) != 0;  // flank to cap: redo this stroke per pixel
    if (!scalar) {  // hi/lo two-sum every step, as pos_add: no rounding of lo builds up between renormalisations
      const f2 ddx = sub2(mul2(ds, P[P_EX]), mul2(dh, P[P_EY]));
      const f2 ddy = fma2(ds, P[P_EY], mul2(dh, P[P_EX]));
      const f2 sx = add2(ps.Xh, ddx), sy = add2(ps.Yh, ddy);
      ps.Xl = add2(ps.Xl, sub2(ddx, sub2(sx, ps.Xh)));
      ps.Yl = add2(ps.Yl, sub2(ddy, sub2(sy, ps.Yh)));
      ps.Xh = sx;
      ps.Yh = sy;
    }
  }
  if (scalar) {
    const StrokeF sg = load_stroke(S);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const bool pop = c == 0 ? pop0 : pop1;
      float4 rp = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (pop) {
        rp = rv.rec[static_cast<size_t>(ps.rc[c] - 1) * rv.stride + off[c]];
        --ps.rc[c];
        ps.nri[c] = ps.rc[c] > 0 ? rv.rec_i[static_cast<size_t>(ps.rc[c] - 1) * rv.stride + off[c]] : -1;
      }
      float4 ckp = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      float ckl = 0.0f;
      if (at_ck && valid[c]) {
        ckp = rv.ckpt[cko + off[c]];
        ckl = rv.ck_lt[cko + off[c]];
      }
      PixAdj a{comp(ps.Xh, c), comp(ps.Yh, c), comp(ps.Xl, c), comp(ps.Yl, c), comp(ps.LT, c), comp(ps.LD, c),
               comp(ps.LX, c), comp(ps.LY, c)};
      if (coupled_stroke(a, sg, S, P, comp(ps.LC0, c), comp(ps.LC1, c), comp(ps.LC2, c), pop, at_ck, valid[c], rp,
                         ckp, ckl, rv.drift_tol, g[c]))
        ++drift;
      put(ps.Xh, c, a.xh); put(ps.Yh, c, a.yh); put(ps.Xl, c, a.xl); put(ps.Yl, c, a.yl);
      put(ps.LT, c, a.lt); put(ps.LD, c, a.lD); put(ps.LX, c, a.lx); put(ps.LY, c, a.ly);
    }
    return;
  }
  const f2 E = add2(ps.LD, fma2(ps.LC0, P[P_CR], fma2(ps.LC1, P[P_CG], mul2(ps.LC2, P[P_CB]))));  // as pair_stroke
  f2 nLT, T, G[5], alpha, oma;
  const int vm = coupled_vjp2(ps.Xh, ps.Yh, ps.Xl, ps.Yl, P, X,
                              [&](f2, f2, f2 sp2, f2& sx, f2& sy, f2& smu) {
                                nLT = add2(ps.LT, sp2);  // log T_i = log T_{i-1} - log(1 - alpha_i)
                                T = ex22(nLT);
                                sx = ps.LX;
                                sy = ps.LY;
                                smu = mul2(T, E);
                              },
                              G, alpha, oma);
  const f2 Ta = mul2(T, alpha);
  f2 nLD = mul2(oma, E);
  f2 nLX = add2(ps.LX, G[0]), nLY = add2(ps.LY, G[1]);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    g[c][0] = -comp(G[0], c); g[c][1] = -comp(G[1], c); g[c][2] = comp(G[2], c); g[c][3] = comp(G[3], c);
    g[c][4] = comp(G[4], c);
    g[c][5] = comp(ps.LC0, c) * comp(Ta, c); g[c][6] = comp(ps.LC1, c) * comp(Ta, c);
    g[c][7] = comp(ps.LC2, c) * comp(Ta, c);
  }
  if (vm) {  // the direct form (floored, or cap to flank) in scalar arithmetic from the same x_i
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (!(vm & (1 << c))) continue;
      float lt = comp(ps.LT, c), Tc = 0.0f, Gs[5], al, om;
      const float Ec = comp(E, c), lxo = comp(ps.LX, c), lyo = comp(ps.LY, c);
      coupled_vjp(comp(ps.Xh, c), comp(ps.Yh, c), comp(ps.Xl, c), comp(ps.Yl, c), S,
                  [&](float, float, float sp2, float& sx, float& sy, float& smu) {
                    lt += sp2;
                    Tc = ex2_a(lt);
                    sx = lxo;
                    sy = lyo;
                    smu = Tc * Ec;
                  },
                  Gs, al, om);
      put(nLT, c, lt);
      put(nLD, c, om * Ec);
      put(nLX, c, lxo + Gs[0]);
      put(nLY, c, lyo + Gs[1]);
      const float Tac = Tc * al;
      g[c][0] = -Gs[0]; g[c][1] = -Gs[1]; g[c][2] = Gs[2]; g[c][3] = Gs[3]; g[c][4] = Gs[4];
      g[c][5] = comp(ps.LC0, c) * Tac; g[c][6] = comp(ps.LC1, c) * Tac; g[c][7] = comp(ps.LC2, c) * Tac;
    }
  }
  ps.LT = nLT;
  ps.LD = nLD;
  ps.LX = nLX;
  ps.LY = nLY;
}

// Replay adjoint (Sec. 5.2) of a 32 x 16 tile, two pixels per thread, over
// strokes 1 .. n; otherwise as backward_tile.  st[c], lC[c][.], valid[c] and
// off[c] (the pixel's element offset in the replay record) describe pixel c of
// the pair; an invalid pixel must carry a finite position and a zero
// cotangent.  pbuf is shared [CH][kPairRec] float2.  With QUEUE, a pixel whose
// checkpoint drift first exceeds rv.drift_tol is appended, with the start of
// that segment, to rv.repair_list (off[c] is then the pixel index) for the
// FP64 repair pass.  With COUPLED, the strokes follow the coupling variant
// Phi_g (pair_stroke_g; gext is shared [CH][kPairExtG] float2).  With BLOCKED
// and a checkpoint interval that is a multiple of kRenorm, the strokes run in
// aligned blocks whose inner strokes skip the checkpoint and renormalisation
// tests (a second copy of the loop; it costs registers, but measured faster in
// every adjoint that uses this tile).  All threads of the CTA must call it.
// Returns false if a bounded wait gave up.
template <int CH, bool QUEUE, int UNROLL = 1, bool COUPLED = false, bool BLOCKED = false>
__device__ bool backward_tile2(ChunkRing<CH>& ring, const float* __restrict__ packed, int n, const bool (&valid)[2],
                               const PixelState (&st)[2], const float (&lC)[2][3], const float bg[3],
                               const RecordView& rv, const size_t (&off)[2], f2* __restrict__ pbuf,
                               float (*red)[kTileThreads / 32][CH * 8], float* __restrict__ slice, bool first,
                               unsigned& drift, unsigned long long* status, f2* __restrict__ gext = nullptr) {
  static_assert(!(COUPLED && QUEUE), "the coupling variant's adjoint has no FP64 repair");
  static_assert(CH * 8 == kTileThreads, "one partial per thread per chunk");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ck = rv.ck;
  const bool any = valid[0] || valid[1];
  PairState ps;
  pair_state_init(ps, valid, st, lC, rv, off);
  int next_ck = (ck < n) ? ck : 0;
  const bool ck_aligned = BLOCKED && (ck & (kRenorm - 1)) == 0 && (CH & (kRenorm - 1)) == 0;
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
    {  // colour of the stroke before the chunk (the background before stroke 1)
      const float* pc = q > 0 ? packed + (static_cast<size_t>(q) * CH - 1) * kRec + F_CR : nullptr;
      pair_records_fill<false, true>(S0, cntc, pbuf, nullptr, pc ? pc[0] : bg[0], pc ? pc[1] : bg[1],
                                     pc ? pc[2] : bg[2]);
    }
    if (COUPLED) pair_ext_g_fill(S0, cntc, gext);
    __syncthreads();
    float (*rb)[CH * 8] = red[b];
    // one stroke: regeneration, adjoint step, VJP, and the warp reduce-scatter of its 8 values
    auto stroke = [&](int j, bool at_ck, bool renorm) {
      const int i1 = q * CH + j + 1;
      float vv[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      size_t cko = 0;
      if (at_ck) {
        next_ck = (next_ck + ck < n) ? next_ck + ck : 0;
        cko = static_cast<size_t>(i1 / ck - 1) * rv.stride;
      }
      if (any) {
        float g[2][8];
        if constexpr (COUPLED)
          pair_stroke_g(ps, S0 + j * kRec, pbuf + j * kPairRec, gext + j * kPairExtG, i1, at_ck, cko, rv, valid,
                        off, g, drift);
        else
          pair_stroke<QUEUE>(ps, S0 + j * kRec, pbuf + j * kPairRec, i1, at_ck, cko, renorm, rv, valid, off, g,
                             drift);
#pragma unroll
        for (int k = 0; k < 8; ++k) vv[k] = g[0][k] + g[1][k];
      }
      const float r = warp_reduce8(vv);
      if ((lane & 3) == 0) rb[warp][j * 8 + ((lane >> 2) & 7)] = r;
    };
    if (BLOCKED && ck_aligned) {
      // blocks of kRenorm strokes aligned to the stroke index (q CH is a multiple
      // of kRenorm): only a block's last stroke can be a checkpoint or a
      // renormalisation point, so the others run without either test
      for (int j0 = 0; j0 < cntc; j0 += kRenorm) {
        const int jl = min(j0 + kRenorm, cntc) - 1;
#pragma unroll UNROLL
        for (int j = j0; j < jl; ++j) stroke(j, false, false);
        const int il = q * CH + jl + 1;
        stroke(jl, il == next_ck, (il & (kRenorm - 1)) == 0);  // (next_ck is CTA-uniform)
      }
    } else {
#pragma unroll UNROLL
      for (int j = 0; j < cntc; ++j) {
        const int i1 = q * CH + j + 1;
        stroke(j, i1 == next_ck, (i1 & (kRenorm - 1)) == 0);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && q + 2 < nch) ring.issue(b, chunk_src(q + 2), chunk_cnt(q + 2));
    const int t = threadIdx.x;
    if (!QUEUE && t < cntc * 8) {  // the queueing pass only finds drifting pixels
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
