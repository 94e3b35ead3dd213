// Stroke packing (device prologue): turns the program's parameter arrays into
// one 128-byte record per stroke holding everything the per-pixel loops read:
// the frame (m, e), the Steiner constants of Eq. steiner (2L + pi r, A_L(r)),
// the floor (eps r)^2 of Sec. 5.2, the relaxation 1/max(tau r, tau_min) of
// Eq. relax and the colour softmax(logits / tau_c) . palette of Sec. 5.1, and
// for the coupling variant (Eq. coupling) its profile g - 1 as a cubic in
// w = cos 4 pi v, after checking g > 0 exactly (Eq. profile).
#include <math.h>

#include "tbr_internal.cuh"

namespace tbr {

namespace {

// min over w in [-1, 1] of g = 1 + c1 w + c2 (2 w^2 - 1) + c3 (4 w^3 - 3 w)
// (the modes cos 4 pi k v are Chebyshev polynomials of w): the smaller of the
// end values and the values at the roots of g'(w) = 12 c3 w^2 + 4 c2 w + c1 - 3 c3.
__device__ double profile_min_f64(double c1, double c2, double c3) {
  auto g = [&](double w) { return 1.0 + w * (c1 - 3.0 * c3 + w * (2.0 * c2 + w * 4.0 * c3)) - c2; };
  double m = fmin(g(-1.0), g(1.0));
  const double qa = 12.0 * c3, qb = 4.0 * c2, qc = c1 - 3.0 * c3;
  if (qa != 0.0) {
    const double disc = qb * qb - 4.0 * qa * qc;
    if (disc >= 0.0) {
      const double sq = sqrt(disc);
      const double w1 = (-qb - sq) / (2.0 * qa), w2 = (-qb + sq) / (2.0 * qa);
      if (w1 > -1.0 && w1 < 1.0) m = fmin(m, g(w1));
      if (w2 > -1.0 && w2 < 1.0) m = fmin(m, g(w2));
    }
  } else if (qb != 0.0) {
    const double w = -qc / qb;
    if (w > -1.0 && w < 1.0) m = fmin(m, g(w));
  }
  return m;
}

__global__ void k_pack(const float* __restrict__ cx, const float* __restrict__ cy,
                       const float* __restrict__ theta, const float* __restrict__ length,
                       const float* __restrict__ half_width, const float* __restrict__ logits,
                       const float* __restrict__ palette, const float* __restrict__ coupling, int n, int k,
                       float inv_tc, float tau, float tau_min, int snap, float* __restrict__ packed,
                       float* __restrict__ probs, unsigned long long* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float fx = cx[i], fy = cy[i], fth = theta[i], fL = length[i], fr = half_width[i];
  bool bad = !(isfinite(fx) && isfinite(fy) && isfinite(fth) && isfinite(fL) && isfinite(fr)) ||
             fL < 0.0f || !(fr > 0.0f);
  // colour: softmax over the k logits at temperature tau_c, or argmax (snap)
  const float* z = logits + static_cast<size_t>(i) * k;
  float zmax = z[0];
  int am = 0;
  for (int q = 1; q < k; ++q) {
    const float v = z[q];
    if (v > zmax) { zmax = v; am = q; }
  }
  bad = bad || !isfinite(zmax);
  float den = 0.0f;
  for (int q = 0; q < k; ++q) den += expf((z[q] - zmax) * inv_tc);
  const float iden = 1.0f / den;
  float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
  for (int q = 0; q < k; ++q) {
    const float p = expf((z[q] - zmax) * inv_tc) * iden;
    if (probs) probs[static_cast<size_t>(i) * k + q] = p;
    c0 = fmaf(p, palette[3 * q + 0], c0);
    c1 = fmaf(p, palette[3 * q + 1], c1);
    c2 = fmaf(p, palette[3 * q + 2], c2);
  }
  if (snap) { c0 = palette[3 * am]; c1 = palette[3 * am + 1]; c2 = palette[3 * am + 2]; }

  const double th = static_cast<double>(fth);
  const double dex = cos(th), dey = sin(th);
  const float w = fmaxf(tau * fr, tau_min);
  float* R = packed + static_cast<size_t>(i) * kRec;
  R[F_MX] = fx; R[F_MY] = fy;
  R[F_EX] = static_cast<float>(dex); R[F_EY] = static_cast<float>(dey);
  R[F_HL] = 0.5f * fL; R[F_L] = fL; R[F_2L] = 2.0f * fL; R[F_L2] = fL * fL;
  R[F_AR] = static_cast<float>((2.0 * fL + kPiD * fr) * fr);
  R[F_R] = fr;
  R[F_IW] = 1.0f / w;
  R[F_DLW] = (tau * fr > tau_min) ? tau / w : 0.0f;
  R[F_NPR] = static_cast<float>(-(kPiD * fr + fL));
  R[F_CR] = c0; R[F_CG] = c1; R[F_CB] = c2;
  R[F_KA] = static_cast<float>(2.0 * fL + kPiD * fr);
  R[F_FL2] = (kEpsFloor * fr) * (kEpsFloor * fr);
  R[F_TH] = fth;
  double* D = reinterpret_cast<double*>(R + F_D64);
  D[0] = dex; D[1] = dey;
  float q1 = 0.0f, q2 = 0.0f, q3 = 0.0f;  // profile coefficients c_1..c_3
  if (coupling) {
    q1 = coupling[3 * i]; q2 = coupling[3 * i + 1]; q3 = coupling[3 * i + 2];
    bad = bad || !(isfinite(q1) && isfinite(q2) && isfinite(q3)) || !(profile_min_f64(q1, q2, q3) > 0.0);
  }
  // g - 1 = -c2 + (c1 - 3 c3) w + 2 c2 w^2 + 4 c3 w^3
  R[F_G0] = -q2; R[F_G0 + 1] = q1 - 3.0f * q3; R[F_G0 + 2] = 2.0f * q2; R[F_G0 + 3] = 4.0f * q3;
  R[F_C1] = q1; R[F_C1 + 1] = q2; R[F_C1 + 2] = q3; R[F_C1 + 3] = 0.0f;
  R[F_BAD] = bad ? 1.0f : 0.0f;
  if (bad) atomicAdd(status + ST_INVALID, 1ull);
}

}  // namespace

cudaError_t launch_pack(const PackArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  const tbr_program* p = a.prog;
  const int threads = 128;
  const int blocks = (a.n + threads - 1) / threads;
  KernelTimer kt(TBR_K_PACK, st);
  k_pack<<<blocks, threads, 0, st>>>(p->cx, p->cy, p->theta, p->length, p->half_width, p->logits,
                                     p->palette, p->coupling, a.n, p->k, 1.0f / p->color_temp, a.tau, a.tau_min,
                                     a.snap, a.packed, a.probs, a.status);
  return cudaGetLastError();
}

}  // namespace tbr
