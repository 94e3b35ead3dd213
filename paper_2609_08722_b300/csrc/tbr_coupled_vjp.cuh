// Hand-derived vector-Jacobian product of one step of the coupling variant
// (Eq. coupling, Eq. profile) for its replay adjoint (Eq. adjstep, Eq.
// adjparam).
//
// At x_i the adjoint needs lambda^T D disp + mu D alpha with respect to x_i and
// to the stroke's (cx, cy, theta, L, r), where disp = x_{i-1} - x_i is psi_g's
// displacement and alpha the coverage of the deposit {u <= A_L(r) g(v)}.  Both
// depend on x_i - m only, so d/dcx = -d/dx and d/dcy = -d/dy and the five
// gradients (x, y, theta, L, r) are the whole product.
//
// The primal runs once in FP32 in the displacement form (normal step
// -A_L(r) g(v) / (2L + pi (sigma' + sigma)), the cap rotation by delta, the
// epsilon-floor's direct form), so D psi_g = I + D disp keeps full relative
// precision.  The product is then taken in reverse through the frame-local map
// (|s|, |h|, L, r) -> (dS, dH, z), and the frame rotation is applied to the
// result: the seeds are rotated into the stroke frame, the local gradients of
// |s| and |h| rotated back, and the rotation's own theta term added.  A drop
// (L = 0) goes through the same cap formulas, which gives the one-sided
// derivative in L of the capsule family at L = 0.
#pragma once

#include "tbr_internal.cuh"

namespace tbr {

// G[0..4] = d/d(x, y, theta, L, r) of lx disp_x + ly disp_y + mu alpha at x_i.
// seed(alpha, oma, sp2, lx, ly, mu) is called once the coverage is known: it
// receives alpha, 1 - alpha and log2(1 + e^z) (the step's -log2(1 - alpha))
// and sets the adjoint seeds.
template <class Seed>
__device__ __forceinline__ void coupled_vjp(float xh, float yh, float xl, float yl, const float* __restrict__ S,
                                            Seed&& seed, float G[5], float& alpha, float& oma) {
  // ---- primal: frame, centred arclength, profile (Eq. profile)
  const float mx = S[F_MX], my = S[F_MY], ex = S[F_EX], ey = S[F_EY];
  const float X = (xh - mx) + xl, Y = (yh - my) + yl;
  const float s = fmaf(X, ex, Y * ey), h = fmaf(Y, ex, -X * ey);
  const float L = S[F_L], r = S[F_R];
  const float4 gp = *reinterpret_cast<const float4*>(S + F_G0);
  const float sgs = sgn1(s), sgh = sgn1(h);
  const float as = fabsf(s), ah = fabsf(h);
  const float hl = 0.5f * L;
  const float kA = fmaf(kPiF, r, 2.0f * L);  // 2L + pi r
  const float Ar = kA * r;                   // A_L(r)
  const float d = as - hl;
  const bool cap_i = d > 0.0f;
  float sp, inv = 0.0f, ud = 0.0f, uh = 1.0f, phi = 0.0f, t;
  if (cap_i) {
    sp = sqrt_a(fmaf(d, d, ah * ah));
    inv = rcp_a(sp);
    ud = d * inv;
    uh = ah * inv;
    phi = atan2_pos(d, ah);
    t = fmaf(sp, phi, hl);
  } else {
    sp = ah;
    t = as;
  }
  const float Qp = fmaf(kPiF, sp, L);
  const float iQp = rcp_a(Qp);
  const float ang = (2.0f * kPiF) * (t * iQp);  // 4 pi v
  const float am = ang - 0.5f * kPiF;
  const float w = -sin_pi2(am);                // cos 4 pi v
  const float gm1 = fmaf(w, fmaf(w, fmaf(w, gp.w, gp.z), gp.y), gp.x);
  const float Ag = fmaf(Ar, gm1, Ar);
  const float kAs = fmaf(kPiF, sp, kA);        // 2L + pi (r + sigma')
  float C = fmaf(sp - r, kAs, -Ar * gm1);
  const bool floored = C < S[F_FL2];
  if (floored) C = (kEpsFloor * kEpsFloor) * (r * r);
  const float root = sqrt_a(fmaf(kPiF, C, L * L));
  const float den1 = L + root;
  const float iden1 = rcp_a(den1);
  const float sig = C * iden1;
  const float Q = fmaf(kPiF, sig, L);
  const float tn = t * (Q * iQp);
  const bool cap_o = tn > hl;
  // branch: 0 cap to cap (rotation), 1 flank to flank, 2 direct form
  const int br = (!floored && cap_i && cap_o) ? 0 : ((!floored && !cap_i) ? 1 : 2);
  float dS, dH;
  float den2 = 0.0f, dsig = 0.0f, P = 0.0f, isig = 0.0f, delta = 0.0f, sD = 0.0f, cD = 1.0f, omc = 0.0f;
  int dclamp = 0;
  float beta = 0.0f, sb = 0.0f, cb = 1.0f;
  bool bclamp = false;
  if (br != 2) {
    den2 = fmaf(kPiF, sp + sig, 2.0f * L);
    dsig = -Ag * rcp_a(den2);
  }
  if (br == 0) {
    isig = rcp_a(sig);
    P = phi - 0.5f * kPiF;
    delta = -((dsig * L) * (P * (iQp * isig)));
    if (delta < -phi) {
      delta = -phi;
      dclamp = 1;
    }
    if (delta > 0.0f) {
      delta = 0.0f;
      dclamp = 2;
    }
    sD = sin_pi2(delta);
    omc = omc_pi2(delta);
    cD = 1.0f - omc;
    dS = fmaf(dsig, ud, sig * fmaf(uh, sD, -ud * omc));
    dH = fmaf(dsig, uh, -sig * fmaf(ud, sD, uh * omc));
  } else if (br == 1) {
    dS = kPiF * (as * (dsig * iQp));
    dH = dsig;
  } else {
    float sn, hn;
    if (cap_o) {
      isig = rcp_a(sig);
      beta = (tn - hl) * isig;
      if (beta > 0.5f * kPiF) {
        beta = 0.5f * kPiF;
        bclamp = true;
      }
      sb = sin_pi2(beta);
      cb = 1.0f - omc_pi2(beta);
      sn = fmaf(sig, sb, hl);
      hn = sig * cb;
    } else {
      sn = tn;
      hn = sig;
    }
    dS = sn - as;
    dH = hn - ah;
  }
  const float dsw = sgs * dS, dhw = sgh * dH;
  const float ddx = fmaf(dsw, ex, -dhw * ey), ddy = fmaf(dsw, ey, dhw * ex);
  // coverage from the deposit boundary sigma_b(v): root of 2 L sigma + pi sigma^2 = A g
  const float R2 = sqrt_a(fmaf(kPiF, Ag, L * L));
  const float iD2 = rcp_a(L + R2);
  const float rb = Ag * iD2;
  const float iw = S[F_IW];
  const float z = (rb - sp) * iw;
  const bool clamped = z > kZMax;
  const float zc = fminf(z, kZMax);
  const float ez = ex2_a(zc * kLog2e);
  const float opl = 1.0f + ez;
  oma = rcp_a(opl);
  alpha = ez * oma;
  float lx, ly, mu;
  seed(alpha, oma, lg2_a(opl), lx, ly, mu);

  // ---- reverse: seeds of the frame-local outputs
  const float ls = fmaf(lx, ex, ly * ey), lh = fmaf(ly, ex, -lx * ey);  // lambda in the frame
  const float b_dS = sgs * ls, b_dH = sgh * lh;
  const float b_z = clamped ? 0.0f : mu * (alpha * oma);
  float b_as = 0.0f, b_ah = 0.0f, b_L = 0.0f, b_r = 0.0f, b_sp = 0.0f, b_sig = 0.0f, b_Ag = 0.0f;
  float b_t = 0.0f, b_phi = 0.0f, b_iQp = 0.0f, b_ud = 0.0f, b_uh = 0.0f;
  // z = (rb - sp) / w(r), rb = Ag / (L + sqrt(pi Ag + L^2))
  {
    const float b_rb = b_z * iw;
    b_sp = -b_rb;
    b_r = -b_z * z * S[F_DLW];
    b_Ag = b_rb * iD2;
    const float b_D2 = -b_rb * rb * iD2;
    const float b_in = b_D2 * 0.5f * rcp_a(R2);  // d/d(pi Ag + L^2)
    b_Ag = fmaf(kPiF, b_in, b_Ag);
    b_L = fmaf(2.0f * L, b_in, b_D2);
  }
  if (br == 0) {
    const float b_dsig0 = fmaf(b_dS, ud, b_dH * uh);
    b_sig = fmaf(b_dS, fmaf(uh, sD, -ud * omc), -b_dH * fmaf(ud, sD, uh * omc));
    b_ud = fmaf(b_dS, dsig - sig * omc, -b_dH * sig * sD);
    b_uh = fmaf(b_dS, sig * sD, b_dH * (dsig - sig * omc));
    const float b_sD = sig * fmaf(b_dS, uh, -b_dH * ud);
    const float b_omc = -sig * fmaf(b_dS, ud, b_dH * uh);
    const float b_delta = fmaf(b_sD, cD, b_omc * sD);
    float b_dsig = b_dsig0;
    if (dclamp == 1) {
      b_phi = -b_delta;
    } else if (dclamp == 0) {
      // delta = -dsig L P iQp / sig
      const float k0 = P * (iQp * isig);
      b_dsig = fmaf(-b_delta * L, k0, b_dsig);
      b_L = fmaf(-b_delta * dsig, k0, b_L);
      const float kd = -b_delta * (dsig * L);
      b_phi = kd * (iQp * isig);
      b_iQp = kd * (P * isig);
      b_sig = fmaf(-b_delta * delta, isig, b_sig);
    }
    // dsig = -Ag / den2, den2 = pi (sp + sig) + 2L
    const float b_den2 = -b_dsig * dsig * rcp_a(den2);
    b_Ag = fmaf(-b_dsig, rcp_a(den2), b_Ag);
    b_sp = fmaf(kPiF, b_den2, b_sp);
    b_sig = fmaf(kPiF, b_den2, b_sig);
    b_L = fmaf(2.0f, b_den2, b_L);
  } else if (br == 1) {
    const float b_dsig = fmaf(b_dS * kPiF, as * iQp, b_dH);
    b_as = b_dS * kPiF * (dsig * iQp);
    b_iQp = b_dS * kPiF * (as * dsig);
    const float b_den2 = -b_dsig * dsig * rcp_a(den2);
    b_Ag = fmaf(-b_dsig, rcp_a(den2), b_Ag);
    b_sp = fmaf(kPiF, b_den2, b_sp);
    b_sig = fmaf(kPiF, b_den2, b_sig);
    b_L = fmaf(2.0f, b_den2, b_L);
  } else {
    // dS = sn - |s|, dH = hn - |h|
    b_as = -b_dS;
    b_ah = -b_dH;
    float b_tn;
    if (cap_o) {
      b_sig = fmaf(b_dS, sb, b_dH * cb);
      b_L = fmaf(0.5f, b_dS, b_L);
      b_tn = 0.0f;
      if (!bclamp) {
        // beta = (tn - hl) / sig
        const float b_beta = sig * fmaf(b_dS, cb, -b_dH * sb);
        b_tn = b_beta * isig;
        b_L = fmaf(-0.5f, b_tn, b_L);
        b_sig = fmaf(-b_beta * beta, isig, b_sig);
      }
    } else {
      b_tn = b_dS;
      b_sig = b_dH;
    }
    // tn = t Q / Q', Q = L + pi sig
    const float b_Q = b_tn * (t * iQp);
    b_t = b_tn * (Q * iQp);
    b_iQp = b_tn * (t * Q);
    b_L += b_Q;
    b_sig = fmaf(kPiF, b_Q, b_sig);
  }
  // sig = C / (L + sqrt(pi C + L^2))
  float b_C = b_sig * iden1;
  {
    const float b_den1 = -b_sig * sig * iden1;
    const float b_in = b_den1 * 0.5f * rcp_a(root);
    b_C = fmaf(kPiF, b_in, b_C);
    b_L = fmaf(2.0f * L, b_in, b_L + b_den1);
  }
  float b_Ar = 0.0f, b_gm1 = 0.0f, b_kA = 0.0f;
  if (floored) {
    b_r = fmaf(b_C * (2.0f * kEpsFloor * kEpsFloor), r, b_r);
  } else {
    // C = (sp - r)(2L + pi (r + sp)) - A_L(r) (g - 1)
    b_sp = fmaf(b_C, fmaf(kPiF, sp - r, kAs), b_sp);
    b_r = fmaf(-b_C, kAs, b_r);
    b_kA = b_C * (sp - r);
    b_Ar = -b_C * gm1;
    b_gm1 = -b_C * Ar;
  }
  // Ag = A_L(r) (1 + (g - 1))
  b_Ar = fmaf(b_Ag, 1.0f + gm1, b_Ar);
  b_gm1 = fmaf(b_Ag, Ar, b_gm1);
  // g - 1 = cubic in w; w = cos(4 pi v) = -sin(am), dw/dang = -cos(am)
  const float b_w = b_gm1 * fmaf(w, fmaf(3.0f * gp.w, w, 2.0f * gp.z), gp.y);
  const float b_ang = -b_w * (1.0f - omc_pi2(am));
  // ang = 2 pi t / Q', Q' = L + pi sp
  b_t = fmaf(b_ang * (2.0f * kPiF), iQp, b_t);
  b_iQp = fmaf(b_ang * (2.0f * kPiF), t, b_iQp);
  const float b_Qp = -b_iQp * iQp * iQp;
  b_L += b_Qp;
  b_sp = fmaf(kPiF, b_Qp, b_sp);
  if (cap_i) {
    // t = hl + sp phi, phi = atan2(d, |h|), u = (d, |h|) / sp, sp = |(d, |h|)|
    b_L = fmaf(0.5f, b_t, b_L);
    b_sp = fmaf(b_t, phi, b_sp);
    b_phi = fmaf(b_t, sp, b_phi);
    // du/d(d, |h|) = (I - u u^T) / sp; dphi/d(d, |h|) = (uh, -ud) / sp
    const float ub = fmaf(ud, b_ud, uh * b_uh);
    const float bdd = fmaf(fmaf(b_phi, uh, b_ud - ud * ub), inv, b_sp * ud);
    const float bdh = fmaf(fmaf(-b_phi, ud, b_uh - uh * ub), inv, b_sp * uh);
    b_as += bdd;
    b_L = fmaf(-0.5f, bdd, b_L);
    b_ah += bdh;
  } else {
    b_ah += b_sp;
    b_as += b_t;
  }
  // A_L(r) = (2L + pi r) r
  b_kA = fmaf(b_Ar, r, b_kA);
  b_r = fmaf(b_Ar, kA, b_r);
  b_L = fmaf(2.0f, b_kA, b_L);
  b_r = fmaf(kPiF, b_kA, b_r);
  // frame: (s, h) = R(theta)^T (x - m); the rotation of disp back to world adds
  // theta's own term -lx ddy + ly ddx
  const float g_s = sgs * b_as, g_h = sgh * b_ah;
  G[0] = fmaf(g_s, ex, -g_h * ey);
  G[1] = fmaf(g_s, ey, g_h * ex);
  G[2] = fmaf(g_s, h, -g_h * s) + fmaf(ly, ddx, -lx * ddy);
  G[3] = b_L;
  G[4] = b_r;
}

}  // namespace tbr
