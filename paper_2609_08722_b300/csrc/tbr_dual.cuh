// Local Jacobians of one step of the coupling variant (Eq. coupling) for its
// replay adjoint, by forward-mode dual numbers in FP32.
//
// At x_i the step needs, for Eq. adjstep / Eq. adjparam: the displacement of
// psi_g (x_{i-1} = x_i + disp) and its derivatives with respect to x_i and to
// the stroke's (cx, cy, theta, L, r), and the coverage alpha with the same
// derivatives.  psi_g depends on x_i - m only, so d/dcx = -d/dx and
// d/dcy = -d/dy, and five tangents suffice: (x, y, theta, L, r).  The
// displacement is evaluated in the displacement form of psi_local (normal step
// -A_L(r) g(v) / (2L + pi (sigma' + sigma)), the cap rotation by delta, the
// epsilon-floor's direct form), so D psi_g = I + D disp keeps full relative
// precision.  A drop (L = 0) goes through the same cap formulas, which gives
// the one-sided derivative in L of the capsule family at L = 0.
#pragma once

#include "tbr_internal.cuh"

namespace tbr {

constexpr int kNT = 5;  // tangents: x, y, theta, L, r

struct DF {
  float v;
  float d[kNT];
};

__device__ __forceinline__ DF dconst(float v) {
  DF a;
  a.v = v;
#pragma unroll
  for (int k = 0; k < kNT; ++k) a.d[k] = 0.0f;
  return a;
}
__device__ __forceinline__ DF dvar(float v, int k) {
  DF a = dconst(v);
  a.d[k] = 1.0f;
  return a;
}
__device__ __forceinline__ DF operator+(const DF& a, const DF& b) {
  DF c;
  c.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < kNT; ++k) c.d[k] = a.d[k] + b.d[k];
  return c;
}
__device__ __forceinline__ DF operator-(const DF& a, const DF& b) {
  DF c;
  c.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < kNT; ++k) c.d[k] = a.d[k] - b.d[k];
  return c;
}
__device__ __forceinline__ DF operator-(const DF& a) {
  DF c;
  c.v = -a.v;
#pragma unroll
  for (int k = 0; k < kNT; ++k) c.d[k] = -a.d[k];
  return c;
}
__device__ __forceinline__ DF operator*(const DF& a, const DF& b) {
  DF c;
  c.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < kNT; ++k) c.d[k] = fmaf(a.d[k], b.v, a.v * b.d[k]);
  return c;
}
__device__ __forceinline__ DF operator*(float s, const DF& a) {
  DF c;
  c.v = s * a.v;
#pragma unroll
  for (int k = 0; k < kNT; ++k) c.d[k] = s * a.d[k];
  return c;
}
__device__ __forceinline__ DF operator+(const DF& a, float s) {
  DF c = a;
  c.v += s;
  return c;
}
// f(a) with f(a.v) = fv and f'(a.v) = dfv
__device__ __forceinline__ DF dchain(const DF& a, float fv, float dfv) {
  DF c;
  c.v = fv;
#pragma unroll
  for (int k = 0; k < kNT; ++k) c.d[k] = dfv * a.d[k];
  return c;
}
__device__ __forceinline__ DF drcp(const DF& a) {
  const float r = rcp_a(a.v);
  return dchain(a, r, -r * r);
}
__device__ __forceinline__ DF ddiv(const DF& a, const DF& b) { return a * drcp(b); }
__device__ __forceinline__ DF dsqrt(const DF& a) {
  const float s = sqrt_a(a.v);
  return dchain(a, s, s > 0.0f ? 0.5f * rcp_a(s) : 0.0f);
}
__device__ __forceinline__ DF dabs(const DF& a) { return a.v < 0.0f ? -a : a; }
// atan2(y, x) for y, x >= 0
__device__ __forceinline__ DF datan2_pos(const DF& y, const DF& x) {
  DF c;
  c.v = atan2_pos(y.v, x.v);
  const float den = fmaf(x.v, x.v, y.v * y.v);
  const float inv = den > 0.0f ? rcp_a(den) : 0.0f;
#pragma unroll
  for (int k = 0; k < kNT; ++k) c.d[k] = fmaf(x.v, y.d[k], -y.v * x.d[k]) * inv;
  return c;
}
// sin and 1 - cos on |d| <= pi/2 (the polynomials of the primal path)
__device__ __forceinline__ DF dsin_pi2(const DF& a) { return dchain(a, sin_pi2(a.v), 1.0f - omc_pi2(a.v)); }
__device__ __forceinline__ DF domc_pi2(const DF& a) { return dchain(a, omc_pi2(a.v), sin_pi2(a.v)); }

// Output of one coupled step's local linearisation at x_i.
struct CoupledJac {
  float dd[2][kNT];  // d disp / d (x, y, theta, L, r), disp = x_{i-1} - x_i (world)
  float da[kNT];     // d alpha / d (x, y, theta, L, r); 0 where the clamp binds
  float alpha, oma, sp2;
};

// psi_g's displacement and the coupled coverage at the hi/lo point x_i for the
// packed stroke S (the soft render's epsilon-floor applies).
__device__ __forceinline__ void coupled_jac(float xh, float yh, float xl, float yl, const float* __restrict__ S,
                                            CoupledJac& o) {
  const float mx = S[F_MX], my = S[F_MY], exv = S[F_EX], eyv = S[F_EY];
  const float Xv = (xh - mx) + xl, Yv = (yh - my) + yl;
  const float sv = fmaf(Xv, exv, Yv * eyv), hv = fmaf(Yv, exv, -Xv * eyv);
  // frame coordinates: d/dx, d/dy of (s, h) are e and e_perp; d/dtheta: (h, -s)
  DF s = dconst(sv), h = dconst(hv);
  s.d[0] = exv; s.d[1] = eyv; s.d[2] = hv;
  h.d[0] = -eyv; h.d[1] = exv; h.d[2] = -sv;
  DF ex = dconst(exv), ey = dconst(eyv);
  ex.d[2] = -eyv; ey.d[2] = exv;
  const DF L = dvar(S[F_L], 3), r = dvar(S[F_R], 4);
  const DF hl = 0.5f * L, twoL = 2.0f * L;
  const DF kA = twoL + kPiF * r;                 // 2L + pi r
  const DF Ar = kA * r;                          // A_L(r)
  const float4 gp = *reinterpret_cast<const float4*>(S + F_G0);
  const float sgs = sgn1(sv), sgh = sgn1(hv);
  const DF as = dabs(s), ah = dabs(h);
  const DF d = as - hl;
  const bool cap_i = d.v > 0.0f;
  DF sp, ud, uh, phi, t;
  if (cap_i) {
    sp = dsqrt(d * d + ah * ah);
    const DF inv = drcp(sp);
    ud = d * inv; uh = ah * inv;
    phi = datan2_pos(d, ah);
    t = hl + sp * phi;
  } else {
    sp = ah; ud = dconst(0.0f); uh = dconst(1.0f); phi = dconst(0.0f); t = as;
  }
  const DF Qp = L + kPiF * sp;
  const DF iQp = drcp(Qp);
  // profile at the point's v: 4 pi v = 2 pi t / Q', w = cos(4 pi v) = -sin(4 pi v - pi/2)
  const DF ang = (2.0f * kPiF) * (t * iQp);
  const DF w = -dsin_pi2(ang + (-0.5f * kPiF));
  const DF gm1 = w * (w * (w * dconst(gp.w) + gp.z) + gp.y) + gp.x;
  const DF Ag = Ar + Ar * gm1;
  DF C = (sp - r) * (kA + kPiF * sp) - Ar * gm1;
  const bool floored = C.v < S[F_FL2];
  if (floored) C = (kEpsFloor * kEpsFloor) * (r * r);  // (eps r)^2
  const DF sig = ddiv(C, L + dsqrt(kPiF * C + L * L));
  const DF Q = L + kPiF * sig;
  const DF tn = t * (Q * iQp);
  const bool cap_o = tn.v > hl.v;
  DF dS, dH;
  if (!floored && cap_i && cap_o) {
    const DF dsig = -ddiv(Ag, kPiF * (sp + sig) + twoL);
    DF delta = -((dsig * L) * ((phi + (-0.5f * kPiF)) * (iQp * drcp(sig))));
    if (delta.v < -phi.v) delta = -phi;
    if (delta.v > 0.0f) delta = dconst(0.0f);
    const DF sD = dsin_pi2(delta), omc = domc_pi2(delta);
    dS = dsig * ud + sig * (uh * sD - ud * omc);
    dH = dsig * uh - sig * (ud * sD + uh * omc);
  } else if (!floored && !cap_i) {
    const DF dsig = -ddiv(Ag, kPiF * (sp + sig) + twoL);
    dS = kPiF * (as * (dsig * iQp));
    dH = dsig;
  } else {  // floored, or cap to flank: direct form
    DF sn, hn;
    if (cap_o) {
      DF beta = (tn - hl) * drcp(sig);
      if (beta.v > 0.5f * kPiF) beta = dconst(0.5f * kPiF);
      const DF sb = dsin_pi2(beta), cb = dconst(1.0f) - domc_pi2(beta);
      sn = sig * sb + hl;
      hn = sig * cb;
    } else {
      sn = tn;
      hn = sig;
    }
    dS = sn - as;
    dH = hn - ah;
  }
  const DF ds = sgs * dS, dh = sgh * dH;
  const DF ddx = ds * ex - dh * ey, ddy = ds * ey + dh * ex;
  // coverage from the deposit boundary sigma_b(v): root of 2 L sigma + pi sigma^2 = A g
  const DF rb = ddiv(Ag, L + dsqrt(kPiF * Ag + L * L));
  DF iw = dconst(S[F_IW]);
  iw.d[4] = -S[F_DLW] * S[F_IW];                 // d(1/w)/dr = -(dw/dr)/w^2
  const DF z = (rb - sp) * iw;
  const bool clamped = z.v > kZMax;
  const float zc = fminf(z.v, kZMax);
  const float ez = ex2_a(zc * kLog2e);
  const float opl = 1.0f + ez;
  o.oma = rcp_a(opl);
  o.alpha = ez * o.oma;
  o.sp2 = lg2_a(opl);
  const float dadz = clamped ? 0.0f : o.alpha * o.oma;
#pragma unroll
  for (int k = 0; k < kNT; ++k) {
    o.dd[0][k] = ddx.d[k];
    o.dd[1][k] = ddy.d[k];
    o.da[k] = dadz * z.d[k];
  }
}

}  // namespace tbr
