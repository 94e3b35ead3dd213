// TBR oracle: a plain, slow FP64 CPU implementation of transport-based rendering
// with capsule deposition strokes.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load
// this file: only the test suite, the smoke check and the benchmark's CPU-baseline
// leg use it.  It shares no code, header, table or constant generator with the
// CUDA path; both sides only receive the same seeded input arrays.
//
// What it computes, each function citing the passage it follows:
//   * the capsule insertion map in its two directions: backward psi (Eq. back)
//     and forward Phi (Eq. fwd), with the tangential coordinate kept as the
//     centred arclength v (Eq. phi, Prop. 2 "Centred arclength"), written on
//     the full stadium (no quadrant folding) from the definitions in Sec. 4;
//   * the interior extension by clamping C (Sec. 4 "The chain") and the
//     implemented epsilon-floor of Sec. 5.2;
//   * the hard and soft renderers (Eq. chain, Eq. render, Eq. relax, Eq. state),
//     the soft one with the optional early exit of the forward render (a pixel
//     stops once its transmittance falls below a threshold);
//   * the one-pass closed-form compensation baseline (Sec. "Closed-form
//     compensation baseline"): anchor or endpoint pre-images through every
//     later stroke's inverse map, with blocked steps clamped or skipped;
//   * the sixteen-drop operator psi_D of the transfer renderer R_D (Sec.
//     "Transfer across transport constructions"): K = 16 classical drop maps of
//     the stroke's total area laid along its segment, with capsule coverage;
//   * the coupling variant Phi_g (Sec. "A variant closer to line-source
//     potential flow", Eq. coupling, Eq. profile): the area coordinate shifted
//     by A_L(r) g(v) with v kept, the deposit {u <= A_L(r) g(v)}, and the exact
//     positivity check of g;
//   * a stored-state adjoint (Eq. adjstep, Eq. adjparam) whose local Jacobians
//     come from forward-mode dual numbers, and a forward-mode directional
//     derivative of the whole soft render used to pin that adjoint.
//
// Parity status: every function here is pinned by a "not gpu" test (round trip,
// drop limit, area, symmetry, commutation, compositing identity, brute force,
// finite differences).  None is "parity unpinned".
//
// Conventions (the readings of the paper used throughout):
//   * A stroke is (cx, cy, th, L, r): segment centre, direction angle, full
//     segment length and half-width.  The segment is [m - L e/2, m + L e/2],
//     e = (cos th, sin th).
//   * Program index j = 0..N-1 is the paper's stroke i = j+1; rendering visits
//     j = N-1 down to 0.
//   * Pixel (row, col) is sampled once at ((col+0.5)/W, (row+0.5)/H).
//   * Colour c_j = softmax(logits_j / tau_c) . palette, or the palette entry of
//     the largest logit when snapping.
//   * Soft coverage alpha = min(sigmoid((r - sigma')/max(tau r, tau_min)), 1 - 1e-7).
//   * epsilon-floor: C <- (eps r)^2 whenever C < (eps r)^2, eps = 1e-3; each such
//     sample counts as one side-table record.
//   * Phi_g: v is the centred arclength of the point's own leaf; the soft
//     coverage is sigmoid((sigma_b(v) - sigma') / w), sigma_b(v) the root of
//     A_L(sigma) = A_L(r) g(v) (= r when g = 1); the coupling applies to the
//     capsule transport only.
//   * R_D: drop k = 0..15 (inserted k-th, one sweep from the segment's start
//     m - L e/2 to its end) is centred at m + e L ((k + 1/2)/16 - 1/2) with
//     radius s = sqrt(A_L(r) / (16 pi)); inside a drop's disc the pull-back
//     uses the same epsilon-floor, sigma^2 <- (eps s)^2, on the same ray.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

static const double kPi = 3.14159265358979323846;
static const double kEps = 1e-3;            // epsilon of the floor, Sec. 5.2
static const double kAlphaMax = 1.0 - 1e-7;  // coverage clamp, Sec. 5.2 "Conditioning"

// ---------------------------------------------------------------------------
// Forward-mode dual numbers (value plus D directional derivatives).
// ---------------------------------------------------------------------------
template <int D>
struct Dual {
  double v;
  double d[D];
  Dual() : v(0.0) { for (int k = 0; k < D; ++k) d[k] = 0.0; }
  Dual(double x) : v(x) { for (int k = 0; k < D; ++k) d[k] = 0.0; }  // NOLINT
};

inline double value(double x) { return x; }
template <int D> inline double value(const Dual<D>& x) { return x.v; }

template <int D> inline Dual<D> operator+(const Dual<D>& a, const Dual<D>& b) {
  Dual<D> r; r.v = a.v + b.v; for (int k = 0; k < D; ++k) r.d[k] = a.d[k] + b.d[k]; return r;
}
template <int D> inline Dual<D> operator-(const Dual<D>& a, const Dual<D>& b) {
  Dual<D> r; r.v = a.v - b.v; for (int k = 0; k < D; ++k) r.d[k] = a.d[k] - b.d[k]; return r;
}
template <int D> inline Dual<D> operator-(const Dual<D>& a) {
  Dual<D> r; r.v = -a.v; for (int k = 0; k < D; ++k) r.d[k] = -a.d[k]; return r;
}
template <int D> inline Dual<D> operator*(const Dual<D>& a, const Dual<D>& b) {
  Dual<D> r; r.v = a.v * b.v;
  for (int k = 0; k < D; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <int D> inline Dual<D> operator/(const Dual<D>& a, const Dual<D>& b) {
  Dual<D> r; r.v = a.v / b.v;
  for (int k = 0; k < D; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
  return r;
}
template <int D> inline Dual<D> operator+(const Dual<D>& a, double b) { return a + Dual<D>(b); }
template <int D> inline Dual<D> operator+(double a, const Dual<D>& b) { return Dual<D>(a) + b; }
template <int D> inline Dual<D> operator-(const Dual<D>& a, double b) { return a - Dual<D>(b); }
template <int D> inline Dual<D> operator-(double a, const Dual<D>& b) { return Dual<D>(a) - b; }
template <int D> inline Dual<D> operator*(const Dual<D>& a, double b) { return a * Dual<D>(b); }
template <int D> inline Dual<D> operator*(double a, const Dual<D>& b) { return Dual<D>(a) * b; }
template <int D> inline Dual<D> operator/(const Dual<D>& a, double b) { return a / Dual<D>(b); }
template <int D> inline Dual<D> operator/(double a, const Dual<D>& b) { return Dual<D>(a) / b; }

// Chain rule helper: f(a) with f'(a) = df.
template <int D> inline Dual<D> chain(const Dual<D>& a, double f, double df) {
  Dual<D> r; r.v = f; for (int k = 0; k < D; ++k) r.d[k] = df * a.d[k]; return r;
}
template <int D> inline Dual<D> sqrt(const Dual<D>& a) {
  double s = std::sqrt(a.v); return chain(a, s, 0.5 / s);
}
template <int D> inline Dual<D> sin(const Dual<D>& a) { return chain(a, std::sin(a.v), std::cos(a.v)); }
template <int D> inline Dual<D> cos(const Dual<D>& a) { return chain(a, std::cos(a.v), -std::sin(a.v)); }
template <int D> inline Dual<D> exp(const Dual<D>& a) { double e = std::exp(a.v); return chain(a, e, e); }
template <int D> inline Dual<D> log1p(const Dual<D>& a) { return chain(a, std::log1p(a.v), 1.0 / (1.0 + a.v)); }
template <int D> inline Dual<D> fabs(const Dual<D>& a) { return a.v < 0.0 ? -a : a; }
template <int D> inline Dual<D> atan2(const Dual<D>& y, const Dual<D>& x) {
  Dual<D> r; r.v = std::atan2(y.v, x.v);
  double n = x.v * x.v + y.v * y.v;
  for (int k = 0; k < D; ++k) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) / n;
  return r;
}

// ---------------------------------------------------------------------------
// Operation counting (measurement only: no render calls it).  Ops carries a
// value and two flags: px, the value depends on the pixel's state, and act, it
// depends on the pixel's state or on a stroke parameter.  Only an operation
// whose result depends on the pixel is per pixel-stroke work; one on stroke
// parameters and constants alone can be hoisted out of the pixel loop and is
// not tallied.  Tallies are FP32-pipe operations (an add, subtract or multiply
// is one; this file writes no fused multiply-add, so a*b + c is two, the FLOP
// count) and special-function (XU) operations, as they run when the same
// formula is evaluated for one pixel-stroke:
//   forward:  +, -, *: 1.  a / b: 1 when b is per-stroke (a multiply by its
//             hoisted reciprocal), else a reciprocal (1 XU) and a multiply (1;
//             none when a is the constant 1).  sqrt, sin, cos, atan2: 1 XU.
//             exp and log1p: 1 XU + 1 (base-2 form).  Negation, fabs and
//             comparisons: 0.
//   reverse:  what a reverse sweep over the same operation costs, tallied as
//             the forward runs: the local partial times the result's adjoint
//             for each active operand -- a * b: 1 multiply per active operand;
//             a / b: 1 (adjoint times the reciprocal) + 1 when b is active;
//             sqrt: 1 XU + 2; sin, cos: 1 XU + 1; exp: 1; log1p: 1 XU + 1;
//             atan2: 1 XU + 4 + 1 per active operand; +, -, negation, fabs:
//             0 -- plus the additions that sum an adjoint's contributions:
//             (uses - 1) for a pixel-dependent value, and one per use for a
//             per-stroke active value (its adjoint is summed over pixels
//             before it is chained to the stroke's parameters).
// The per-thread node table below records each active value's uses.
// ---------------------------------------------------------------------------
struct OpTally {
  double f = 0.0, x = 0.0;     // forward FP32, XU
  double rf = 0.0, rx = 0.0;   // reverse contributions FP32, XU
  std::vector<unsigned char> px;
  std::vector<int> uses;
  void reset() { f = x = rf = rx = 0.0; px.clear(); uses.clear(); }
  int add_node(bool p) { px.push_back(p ? 1 : 0); uses.push_back(0); return (int)px.size() - 1; }
  // additions that sum the adjoint contributions of every recorded value
  double accumulation_adds() const {
    double a = 0.0;
    for (size_t i = 0; i < px.size(); ++i) a += px[i] ? std::max(0, uses[i] - 1) : uses[i];
    return a;
  }
};
static thread_local OpTally g_tally;

struct Ops {
  double v = 0.0;
  bool px = false, act = false;
  int id = -1;
  Ops() {}
  Ops(double x) : v(x) {}  // NOLINT: a constant
  static Ops leaf(double x, bool pixel) {
    Ops r(x);
    r.px = pixel; r.act = true; r.id = g_tally.add_node(pixel);
    return r;
  }
};
inline double value(const Ops& a) { return a.v; }

inline Ops ops_result(double v, const Ops& a, const Ops& b) {
  Ops r(v);
  r.px = a.px || b.px;
  r.act = a.act || b.act;
  if (r.act) r.id = g_tally.add_node(r.px);
  return r;
}
inline void ops_use(const Ops& a) { if (a.act && a.id >= 0) g_tally.uses[a.id] += 1; }

inline Ops operator+(const Ops& a, const Ops& b) {
  Ops r = ops_result(a.v + b.v, a, b);
  if (r.px) { g_tally.f += 1; ops_use(a); ops_use(b); }
  return r;
}
inline Ops operator-(const Ops& a, const Ops& b) {
  Ops r = ops_result(a.v - b.v, a, b);
  if (r.px) { g_tally.f += 1; ops_use(a); ops_use(b); }
  return r;
}
inline Ops operator-(const Ops& a) {
  Ops r = ops_result(-a.v, a, Ops());
  if (r.px) ops_use(a);
  return r;
}
inline Ops operator*(const Ops& a, const Ops& b) {
  Ops r = ops_result(a.v * b.v, a, b);
  if (r.px) {
    g_tally.f += 1;
    if (a.act) { g_tally.rf += 1; ops_use(a); }
    if (b.act) { g_tally.rf += 1; ops_use(b); }
  }
  return r;
}
inline Ops operator/(const Ops& a, const Ops& b) {
  Ops r = ops_result(a.v / b.v, a, b);
  if (r.px) {
    if (!b.px) g_tally.f += 1;
    else { g_tally.x += 1; if (a.act || std::fabs(a.v) != 1.0) g_tally.f += 1; }
    g_tally.rf += 1 + (b.act ? 1 : 0);
    ops_use(a); ops_use(b);
  }
  return r;
}
inline Ops ops_unary(double v, const Ops& a, double ff, double fx, double rf, double rx) {
  Ops r = ops_result(v, a, Ops());
  if (r.px) { g_tally.f += ff; g_tally.x += fx; g_tally.rf += rf; g_tally.rx += rx; ops_use(a); }
  return r;
}
inline Ops sqrt(const Ops& a) { return ops_unary(std::sqrt(a.v), a, 0, 1, 2, 1); }
inline Ops sin(const Ops& a) { return ops_unary(std::sin(a.v), a, 0, 1, 1, 1); }
inline Ops cos(const Ops& a) { return ops_unary(std::cos(a.v), a, 0, 1, 1, 1); }
inline Ops exp(const Ops& a) { return ops_unary(std::exp(a.v), a, 1, 1, 1, 0); }
inline Ops log1p(const Ops& a) { return ops_unary(std::log1p(a.v), a, 1, 1, 1, 1); }
inline Ops fabs(const Ops& a) { return ops_unary(std::fabs(a.v), a, 0, 0, 0, 0); }
inline Ops atan2(const Ops& y, const Ops& x) {
  Ops r = ops_result(std::atan2(y.v, x.v), y, x);
  if (r.px) {
    g_tally.x += 1;
    g_tally.rx += 1;
    g_tally.rf += 4 + (y.act ? 1 : 0) + (x.act ? 1 : 0);
    ops_use(y); ops_use(x);
  }
  return r;
}

using std::sqrt; using std::sin; using std::cos; using std::exp; using std::log1p;
using std::fabs; using std::atan2;

// c1..c3: the profile of the coupling variant Phi_g (Eq. coupling, Eq.
// profile); all zero for the capsule map (g = 1).
template <class T> struct Stroke {
  T cx, cy, th, L, r;
  double c1 = 0.0, c2 = 0.0, c3 = 0.0;
};

// ---------------------------------------------------------------------------
// Stroke frame.  Sec. 3: the footprint is the capsule about [a, a+d]; with the
// centre m = a + d/2 and e = d/|d| the segment is {m + t e : |t| <= L/2}.
// s is the coordinate along e, h the coordinate along e_perp = (-e_y, e_x).
// ---------------------------------------------------------------------------
template <class T>
void to_frame(const T& x, const T& y, const Stroke<T>& g, T& s, T& h) {
  T ex = cos(g.th), ey = sin(g.th);
  T dx = x - g.cx, dy = y - g.cy;
  s = dx * ex + dy * ey;
  h = dy * ex - dx * ey;
}
template <class T>
void from_frame(const T& s, const T& h, const Stroke<T>& g, T& x, T& y) {
  T ex = cos(g.th), ey = sin(g.th);
  x = g.cx + s * ex - h * ey;
  y = g.cy + s * ey + h * ex;
}

// sigma(x) = dist(x, segment) (Sec. 3, footprint definition): distance to the
// nearest point of the segment, which is the clamped projection onto it.
template <class T>
T segment_distance(const T& s, const T& h, const T& L) {
  T hl = 0.5 * L;
  T t = s;
  if (value(s) > value(hl)) t = hl;
  else if (value(s) < -value(hl)) t = -hl;
  T ds = s - t;
  if (value(ds) == 0.0) return fabs(h);
  return sqrt(ds * ds + h * h);
}

// Arclength along the parallel curve {sigma = const} (a stadium), measured
// counter-clockwise from the flank corner (-L/2, -sigma): lower flank (length L),
// right cap (pi sigma), upper flank (L), left cap (pi sigma).  Its perimeter is
// P_L(sigma) = 2L + 2 pi sigma (Eq. steiner).  q of Sec. 4 is this divided by P.
template <class T>
T stadium_arclength(const T& s, const T& h, const T& sig, const T& L) {
  T hl = 0.5 * L;
  if (value(s) > value(hl)) {               // right cap, angle from -pi/2 to pi/2
    T ang = atan2(h, s - hl);
    return L + sig * (ang + 0.5 * kPi);
  }
  if (value(s) < -value(hl)) {              // left cap, angle from 0 to pi
    T ang = atan2(-(s + hl), h);
    return 2.0 * L + kPi * sig + sig * ang;
  }
  if (value(h) < 0.0) return s + hl;        // lower flank, travelled towards +s
  return L + kPi * sig + (hl - s);          // upper flank, travelled towards -s
}

// Inverse of stadium_arclength on the stadium at distance sig.
template <class T>
void stadium_point(T a, const T& sig, const T& L, T& s, T& h) {
  T hl = 0.5 * L;
  T per = 2.0 * L + 2.0 * kPi * sig;
  if (value(per) <= 0.0) { s = T(0.0); h = T(0.0); return; }
  if (value(a) < 0.0) a = a + per;
  if (value(a) >= value(per)) a = a - per;
  double av = value(a), Lv = value(L), capv = kPi * value(sig);
  if (av < Lv) { s = a - hl; h = -sig; return; }
  if (av < Lv + capv) {
    T ang = (a - L) / sig - 0.5 * kPi;
    s = hl + sig * cos(ang); h = sig * sin(ang); return;
  }
  if (av < 2.0 * Lv + capv) { s = hl - (a - L - kPi * sig); h = sig; return; }
  T ang = (a - 2.0 * L - kPi * sig) / sig;
  s = -hl - sig * sin(ang); h = sig * cos(ang);
}

// ---------------------------------------------------------------------------
// Coupling variant Phi_g (Sec. "A variant closer to line-source potential
// flow", Eq. coupling): in the area chart (u, v) with u = A_L(sigma) the map
// shifts u by A_L(r) g(v) and keeps v, g(v) = 1 + sum_k c_k cos(4 pi k v)
// (Eq. profile).  The deposit is {u <= A_L(r) g(v)}.
// ---------------------------------------------------------------------------
template <class T>
bool coupled(const Stroke<T>& g) { return g.c1 != 0.0 || g.c2 != 0.0 || g.c3 != 0.0; }

// Centred arclength coordinate v = q - L / (2 P_L(sigma)) (Eq. phi) of a point
// on the leaf at distance sig: its arclength from the lower flank's midpoint
// over the leaf's perimeter.
template <class T>
T centred_v(const T& s, const T& h, const T& sig, const T& L) {
  T per = 2.0 * L + 2.0 * kPi * sig;
  if (value(per) <= 0.0) return T(0.0);
  return (stadium_arclength(s, h, sig, L) - 0.5 * L) / per;
}

// g(v) - 1 (Eq. profile).
template <class T>
T profile_m1(const Stroke<T>& g, const T& v) {
  return g.c1 * cos(4.0 * kPi * v) + g.c2 * cos(8.0 * kPi * v) + g.c3 * cos(12.0 * kPi * v);
}

// Distance of the deposit boundary u = A_L(r) g(v) at coordinate v: the root
// sigma_b of 2 L sigma + pi sigma^2 = A_L(r) g(v).
template <class T>
T deposit_sigma(const Stroke<T>& g, const T& v) {
  T Ag = (2.0 * g.L * g.r + kPi * g.r * g.r) * (1.0 + profile_m1(g, v));
  return Ag / (g.L + sqrt(g.L * g.L + kPi * Ag));
}

// Signed distance from the deposit boundary along sigma at the point's own v:
// sigma' - r for the capsule, sigma' - sigma_b(v') under Eq. coupling.  The
// point is in the deposit iff it is <= 0 (the tie counts as inside).
template <class T>
T deposit_margin(const T& s, const T& h, const T& sp, const Stroke<T>& g) {
  if (!coupled(g)) return sp - g.r;
  return sp - deposit_sigma(g, centred_v(s, h, sp, g.L));
}

enum Mode { kClamp = 0, kFloor = 1, kRawQ = 2, kFloorRawQ = 3 };

// Move a point from the parallel curve at distance sig_from to the one at
// distance sig_to, keeping the centred arclength fraction
// v = q - L/(2 P_L(sigma)) (Eq. phi; Prop. 2), or raw q for the negative control
// of Table "detj" (last row).
template <class T>
void keep_tangential(const T& s, const T& h, const T& sig_from, const T& sig_to,
                     const T& L, bool raw_q, T& s_out, T& h_out) {
  T a_from = stadium_arclength(s, h, sig_from, L);
  T p_from = 2.0 * L + 2.0 * kPi * sig_from;
  T p_to = 2.0 * L + 2.0 * kPi * sig_to;
  T a_to;
  if (value(p_from) <= 0.0) {
    a_to = T(0.0);
  } else if (raw_q) {
    a_to = (a_from / p_from) * p_to;
  } else {
    T q = a_from / p_from;
    T v = q - L / (2.0 * p_from);
    a_to = (v + L / (2.0 * p_to)) * p_to;
  }
  stadium_point(a_to, sig_to, L, s_out, h_out);
}

// Backward material map psi (Eq. back): subtract the inserted area A_L(r) in the
// area coordinate u = A_L(sigma) = 2 L sigma + pi sigma^2, i.e.
// C = A_L(sigma') - A_L(r) = (sigma' - r)(2L + pi(sigma' + r)), and take the
// cancellation-free root sigma = C / (L + sqrt(L^2 + pi C)).
// Inside the footprint C <= 0: clamped to 0 (ideal extension, Sec. 4 "The
// chain") or floored at (eps r)^2 (the implemented map, Sec. 5.2).
// Returns 1 if the floor bound (a side-table record), else 0.
template <class T>
int psi_from_frame(const T& s, const T& h, const T& sp, const Stroke<T>& g, int mode, T& x_out, T& y_out);

template <class T>
int psi(const T& x, const T& y, const Stroke<T>& g, int mode, T& x_out, T& y_out) {
  T s, h;
  to_frame(x, y, g, s, h);
  T sp = segment_distance(s, h, g.L);
  return psi_from_frame(s, h, sp, g, mode, x_out, y_out);
}

// The part of psi after the frame coordinates (s, h) and the distance sp of
// the point have been computed (shared with the coverage of the same point).
template <class T>
int psi_from_frame(const T& s, const T& h, const T& sp, const Stroke<T>& g, int mode, T& x_out, T& y_out) {
  T C = (sp - g.r) * (2.0 * g.L + kPi * (sp + g.r));
  if (coupled(g))  // Eq. coupling: subtract A_L(r) g(v) instead of A_L(r)
    C = C - (2.0 * g.L * g.r + kPi * g.r * g.r) * profile_m1(g, centred_v(s, h, sp, g.L));
  int floored = 0;
  if (mode == kFloor || mode == kFloorRawQ) {
    T fl = (kEps * g.r) * (kEps * g.r);
    if (value(C) < value(fl)) { C = fl; floored = 1; }
  } else if (value(C) < 0.0) {
    C = T(0.0);
    if (value(g.L) == 0.0) {  // the ideal extension maps a drop's disc onto its centre
      x_out = g.cx; y_out = g.cy;
      return 0;
    }
  }
  T sig = C / (g.L + sqrt(g.L * g.L + kPi * C));
  T sn, hn;
  keep_tangential(s, h, sp, sig, g.L, mode == kRawQ || mode == kFloorRawQ, sn, hn);
  from_frame(sn, hn, g, x_out, y_out);
  return floored;
}

// Forward (regeneration) map Phi (Eq. fwd): add the inserted area,
// B = A_L(sigma) + A_L(r) = 2L(sigma + r) + pi(sigma^2 + r^2),
// sigma' = B / (L + sqrt(L^2 + pi B)); same centred arclength.
template <class T>
void phi(const T& x, const T& y, const Stroke<T>& g, bool raw_q, T& x_out, T& y_out) {
  T s, h;
  to_frame(x, y, g, s, h);
  T sg = segment_distance(s, h, g.L);
  T B = 2.0 * g.L * (sg + g.r) + kPi * (sg * sg + g.r * g.r);
  if (coupled(g))  // Eq. coupling: add A_L(r) g(v) instead of A_L(r)
    B = B + (2.0 * g.L * g.r + kPi * g.r * g.r) * profile_m1(g, centred_v(s, h, sg, g.L));
  T sp = B / (g.L + sqrt(g.L * g.L + kPi * B));
  T sn, hn;
  keep_tangential(s, h, sg, sp, g.L, raw_q, sn, hn);
  from_frame(sn, hn, g, x_out, y_out);
}

// Sixteen-drop operator of the transfer renderer R_D (Sec. "Transfer across
// transport constructions"): stroke i's displacement is a composition of
// K = 16 classical drop maps (the radial disc insertion sigma' = sqrt(sigma^2 +
// s^2), i.e. Eq. back at L = 0) of radius s = sqrt(A_L(r) / (K pi)), so that the
// inserted area equals the stroke's own, laid in one sweep along the segment.
static const int kDrops = 16;
template <class T>
void drop_centre(const Stroke<T>& g, int k, T& cx, T& cy) {
  T t = g.L * ((k + 0.5) / kDrops - 0.5);
  cx = g.cx + t * cos(g.th);
  cy = g.cy + t * sin(g.th);
}
template <class T>
T drop_radius2(const Stroke<T>& g) {
  return (2.0 * g.L * g.r + kPi * g.r * g.r) / (kDrops * kPi);
}

// Pull-back psi_D: the inverse drops in reverse insertion order, each moving
// the point along the ray from its centre to distance sigma = sqrt(rho^2 -
// s^2).  Inside a disc (rho^2 - s^2 < (eps s)^2) the point is floored on the
// same ray at eps s (as the capsule's epsilon-floor); rho = 0 takes the
// direction e_perp.  Returns the number of floor binds.
template <class T>
int psi_drops(const T& x, const T& y, const Stroke<T>& g, T& x_out, T& y_out) {
  T px = x, py = y;
  int binds = 0;
  const T s2 = drop_radius2(g);
  const T fl = (kEps * kEps) * s2;
  for (int k = kDrops - 1; k >= 0; --k) {
    T cx, cy;
    drop_centre(g, k, cx, cy);
    T dx = px - cx, dy = py - cy;
    T rho2 = dx * dx + dy * dy;
    T sig2 = rho2 - s2;
    if (value(sig2) < value(fl)) { sig2 = fl; ++binds; }
    T sig = sqrt(sig2);
    if (value(rho2) > 0.0) {
      T f = sig / sqrt(rho2);
      px = cx + dx * f;
      py = cy + dy * f;
    } else {
      px = cx - sig * sin(g.th);
      py = cy + sig * cos(g.th);
    }
  }
  x_out = px; y_out = py;
  return binds;
}

// Forward Phi_D: the drops in insertion order, sigma' = sqrt(rho^2 + s^2).
template <class T>
void phi_drops(const T& x, const T& y, const Stroke<T>& g, T& x_out, T& y_out) {
  T px = x, py = y;
  const T s2 = drop_radius2(g);
  for (int k = 0; k < kDrops; ++k) {
    T cx, cy;
    drop_centre(g, k, cx, cy);
    T dx = px - cx, dy = py - cy;
    T rho2 = dx * dx + dy * dy;
    T sp = sqrt(rho2 + s2);
    if (value(rho2) > 0.0) {
      T f = sp / sqrt(rho2);
      px = cx + dx * f;
      py = cy + dy * f;
    } else {
      px = cx - sp * sin(g.th);
      py = cy + sp * cos(g.th);
    }
  }
  x_out = px; y_out = py;
}

// Transport of the renderers: the capsule map (R_A), none (the inert-mark
// renderer R_U, Definition 1), or the sixteen-drop operator (R_D).
enum Transport { kCapsule = 0, kInert = 1, kDrops16 = 2 };

// Relaxed coverage (Eq. relax), clamped at 1 - 1e-7 (Sec. 5.2 "Conditioning").
// margin: deposit_margin (sigma' - r for the capsule).
template <class T>
T soft_coverage(const T& margin, const T& r, double tau, double tau_min) {
  T w = tau * r;
  if (value(w) < tau_min) w = T(tau_min);
  T z = -margin / w;
  // sigmoid(z); far outside a deposit (z < -700) e^-z would overflow and its
  // derivative turn into inf / inf, so there the same value is written as
  // e^z / (1 + e^z)
  T a = value(z) < -700.0 ? exp(z) / (1.0 + exp(z)) : 1.0 / (1.0 + exp(-z));
  if (value(a) > kAlphaMax) a = T(kAlphaMax);
  return a;
}

}  // namespace orc

using namespace orc;

extern "C" {

// Program layout shared with the Python wrapper (ctypes).  All arrays are
// FP64, program order (index 0 = the paper's g_1).
typedef struct {
  int32_t n, k;
  const double* cx; const double* cy; const double* th; const double* L; const double* r;
  const double* logits;   // [n][k]
  const double* palette;  // [k][3]
  double background[3];   // c_0
  double color_temp;      // tau_c
  const double* coupling; // [n][3] c_1..c_3 of Eq. profile, or NULL (g = 1)
} orc_prog;

}  // extern "C"

namespace {

template <class T>
Stroke<T> stroke_of(const orc_prog* p, int j) {
  Stroke<T> g;
  g.cx = T(p->cx[j]); g.cy = T(p->cy[j]); g.th = T(p->th[j]); g.L = T(p->L[j]); g.r = T(p->r[j]);
  if (p->coupling) {
    g.c1 = p->coupling[3 * j]; g.c2 = p->coupling[3 * j + 1]; g.c3 = p->coupling[3 * j + 2];
  }
  return g;
}

// c_j = softmax(logits_j / tau_c) . palette (Sec. 5.1 "Parameterisation");
// with snap, the palette entry of the largest logit (export snapping).
void stroke_colours(const orc_prog* p, int snap, std::vector<double>& col, std::vector<double>& prob) {
  int n = p->n, k = p->k;
  col.assign((size_t)n * 3, 0.0);
  prob.assign((size_t)n * k, 0.0);
  for (int j = 0; j < n; ++j) {
    const double* z = p->logits + (size_t)j * k;
    int am = 0;
    double zmax = z[0];
    for (int q = 1; q < k; ++q) if (z[q] > zmax) { zmax = z[q]; am = q; }
    double den = 0.0;
    for (int q = 0; q < k; ++q) den += std::exp((z[q] - zmax) / p->color_temp);
    for (int q = 0; q < k; ++q) prob[(size_t)j * k + q] = std::exp((z[q] - zmax) / p->color_temp) / den;
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      if (snap) acc = p->palette[am * 3 + c];
      else for (int q = 0; q < k; ++q) acc += prob[(size_t)j * k + q] * p->palette[q * 3 + c];
      col[(size_t)j * 3 + c] = acc;
    }
  }
}

inline void pixel_centre(int64_t pidx, int W, int H, double& x, double& y) {
  int64_t row = pidx / W, colm = pidx % W;
  x = ((double)colm + 0.5) / (double)W;
  y = ((double)row + 0.5) / (double)H;
}

// Spectral norm of a 2x2 matrix [a b; c d].
double spectral_norm(double a, double b, double c, double d) {
  double p = a * a + b * b + c * c + d * d;
  double q = a * d - b * c;
  double disc = std::sqrt(std::max(0.0, p * p - 4.0 * q * q));
  return std::sqrt(0.5 * (p + disc));
}

}  // namespace

extern "C" {

// Single-map evaluation on a batch of points (for the operator pins).
// mode: 0 ideal clamp, 1 epsilon floor, 2 raw-q control, 3 floor + raw q.
// direction: 0 = psi (Eq. back), 1 = Phi (Eq. fwd; mode 2/3 select raw q).
// floored (nullable): per point 1 if the floor bound.
int orc_map(const double* pts, int64_t n, double cx, double cy, double th, double L, double r,
            int direction, int mode, double* out, int32_t* floored) {
  Stroke<double> g{cx, cy, th, L, r};
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double xo, yo;
    int f = 0;
    if (direction == 0) f = psi(pts[2 * i], pts[2 * i + 1], g, mode, xo, yo);
    else phi(pts[2 * i], pts[2 * i + 1], g, mode == kRawQ || mode == kFloorRawQ, xo, yo);
    out[2 * i] = xo; out[2 * i + 1] = yo;
    if (floored) floored[i] = f;
  }
  return 0;
}

// Jacobian of one map by dual numbers: jac[i] is the 2x7 matrix
// d(x_out, y_out)/d(x, y, cx, cy, th, L, r), row-major.
int orc_map_jacobian(const double* pts, int64_t n, double cx, double cy, double th, double L,
                     double r, int direction, int mode, double* jac) {
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    typedef Dual<7> D7;
    D7 x(pts[2 * i]), y(pts[2 * i + 1]);
    Stroke<D7> g{D7(cx), D7(cy), D7(th), D7(L), D7(r)};
    x.d[0] = 1; y.d[1] = 1; g.cx.d[2] = 1; g.cy.d[3] = 1; g.th.d[4] = 1; g.L.d[5] = 1; g.r.d[6] = 1;
    D7 xo, yo;
    if (direction == 0) psi(x, y, g, mode, xo, yo);
    else phi(x, y, g, mode == kRawQ || mode == kFloorRawQ, xo, yo);
    for (int k = 0; k < 7; ++k) { jac[i * 14 + k] = xo.d[k]; jac[i * 14 + 7 + k] = yo.d[k]; }
  }
  return 0;
}

// The sixteen-drop operator on a batch of points: direction 0 = psi_D (with
// the floor; binds per point in `binds`, nullable), 1 = Phi_D.  If jac is
// non-null it receives d(x_out, y_out)/d(x, y) per point (2x2, row-major).
int orc_map_drops(const double* pts, int64_t n, double cx, double cy, double th, double L, double r,
                  int direction, double* out, int32_t* binds, double* jac) {
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    typedef Dual<2> D2;
    D2 x(pts[2 * i]), y(pts[2 * i + 1]), xo, yo;
    x.d[0] = 1; y.d[1] = 1;
    Stroke<D2> g{D2(cx), D2(cy), D2(th), D2(L), D2(r)};
    int b = 0;
    if (direction == 0) b = psi_drops(x, y, g, xo, yo);
    else phi_drops(x, y, g, xo, yo);
    out[2 * i] = xo.v; out[2 * i + 1] = yo.v;
    if (binds) binds[i] = b;
    if (jac) { jac[4 * i] = xo.d[0]; jac[4 * i + 1] = xo.d[1]; jac[4 * i + 2] = yo.d[0]; jac[4 * i + 3] = yo.d[1]; }
  }
  return 0;
}

// Hard render (Eq. chain, Eq. render with alpha = indicator of K_i).
// Pixels: if pix is non-null, only the npix listed flat indices (row*W + col)
// are rendered and outputs are compact [npix]; otherwise npix must be W*H.
// For each pixel: rgb[3], idx (terminating program index or -1), margin =
// min |sigma'_j - r_j| over the visited strokes (terminating one included) and,
// if kappa is non-null, the product of the spectral norms of Dpsi_j over the
// strokes passed through (the chain's condition estimate).
// n_prefix < 0 renders all strokes; otherwise only the first n_prefix.
// transport: 0 = the capsule map (R_A), 1 = psi = id (the inert-mark renderer,
// Definition 1), 2 = the sixteen-drop operator (R_D).
int orc_render_hard(const orc_prog* p, int W, int H, int n_prefix, int snap, int transport,
                    const int64_t* pix, int64_t npix, double* rgb, int32_t* idx,
                    double* margin, double* kappa) {
  std::vector<double> col, prob;
  stroke_colours(p, snap, col, prob);
  int n = (n_prefix < 0 || n_prefix > p->n) ? p->n : n_prefix;
  #pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < npix; ++q) {
    int64_t pidx = pix ? pix[q] : q;
    double x, y;
    pixel_centre(pidx, W, H, x, y);
    int hit = -1;
    double mg = INFINITY, kap = 1.0;
    for (int j = n - 1; j >= 0; --j) {
      Stroke<double> g = stroke_of<double>(p, j);
      double s, h;
      to_frame(x, y, g, s, h);
      double sp = segment_distance(s, h, g.L);
      const double dm = deposit_margin(s, h, sp, g);
      mg = std::min(mg, std::fabs(dm));
      if (dm <= 0.0) { hit = j; break; }       // closed footprint: the tie is inside
      if (transport == kInert) continue;
      if (kappa) {
        typedef Dual<2> D2;
        D2 xd(x), yd(y), xo, yo;
        xd.d[0] = 1; yd.d[1] = 1;
        Stroke<D2> gd{D2(g.cx), D2(g.cy), D2(g.th), D2(g.L), D2(g.r), g.c1, g.c2, g.c3};
        if (transport == kDrops16) psi_drops(xd, yd, gd, xo, yo);
        else psi(xd, yd, gd, kClamp, xo, yo);
        kap *= spectral_norm(xo.d[0], xo.d[1], yo.d[0], yo.d[1]);
        x = xo.v; y = yo.v;
      } else {
        double xo, yo;
        if (transport == kDrops16) psi_drops(x, y, g, xo, yo);
        else psi(x, y, g, kClamp, xo, yo);
        x = xo; y = yo;
      }
    }
    for (int c = 0; c < 3; ++c) rgb[q * 3 + c] = hit >= 0 ? col[(size_t)hit * 3 + c] : p->background[c];
    if (idx) idx[q] = hit;
    if (margin) margin[q] = mg;
    if (kappa) kappa[q] = kap;
  }
  return 0;
}

}  // extern "C"

namespace {

// One pixel of the soft render (Eq. state): s_N = (x, 0, 1);
// C_{i-1} = C_i + T_i alpha_i c_i, T_{i-1} = T_i (1 - alpha_i), x_{i-1} = psi_i(x_i),
// R = C_0 + T_0 c_0.  Templated so that the same steps run in FP64 and in
// forward-mode dual numbers (the directional-derivative pin).  exit_T > 0 is the
// optional early exit of the forward render: the pixel stops once T falls below
// exit_T after compositing a stroke, and R = C + T c_0 with that T (the strokes
// below would add at most T).
template <class T>
void soft_pixel(const std::vector<Stroke<T>>& g, const std::vector<T>& col, const T bg[3],
                double tau, double tau_min, int transport, double px, double py,
                T out[3], double* T0, int* nrec, double exit_T = 0.0) {
  T x(px), y(py);
  T C[3] = {T(0.0), T(0.0), T(0.0)};
  T Tr(1.0);
  int rec = 0;
  for (int j = (int)g.size() - 1; j >= 0; --j) {
    T s, h;
    to_frame(x, y, g[j], s, h);
    T sp = segment_distance(s, h, g[j].L);
    T a = soft_coverage(deposit_margin(s, h, sp, g[j]), g[j].r, tau, tau_min);
    for (int c = 0; c < 3; ++c) C[c] = C[c] + Tr * a * col[(size_t)j * 3 + c];
    Tr = Tr * (1.0 - a);
    if (exit_T > 0.0 && value(Tr) < exit_T) break;
    if (transport == kCapsule) {
      T xo, yo;
      rec += psi(x, y, g[j], kFloor, xo, yo);
      x = xo; y = yo;
    } else if (transport == kDrops16) {
      T xo, yo;
      rec += psi_drops(x, y, g[j], xo, yo);
      x = xo; y = yo;
    }
  }
  for (int c = 0; c < 3; ++c) out[c] = C[c] + Tr * bg[c];
  if (T0) *T0 = value(Tr);
  if (nrec) *nrec = rec;
}

}  // namespace

extern "C" {

// Soft render (Eq. relax coverage, Eq. state compositing, epsilon-floored psi).
// Outputs per rendered pixel: rgb[3]; T0 (final transmittance, nullable);
// nrec (side-table records, i.e. floor binds, nullable).
// transport as orc_render_hard.  exit_T > 0: early exit once T < exit_T.
int orc_render_soft(const orc_prog* p, int W, int H, double tau, double tau_min, int transport,
                    const int64_t* pix, int64_t npix, double* rgb, double* T0, int32_t* nrec, double exit_T) {
  std::vector<double> col, prob;
  stroke_colours(p, 0, col, prob);
  std::vector<Stroke<double>> g(p->n);
  for (int j = 0; j < p->n; ++j) g[j] = stroke_of<double>(p, j);
  #pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < npix; ++q) {
    int64_t pidx = pix ? pix[q] : q;
    double x, y;
    pixel_centre(pidx, W, H, x, y);
    double out[3], t0;
    int nr;
    soft_pixel<double>(g, col, p->background, tau, tau_min, transport, x, y, out, &t0, &nr, exit_T);
    for (int c = 0; c < 3; ++c) rgb[q * 3 + c] = out[c];
    if (T0) T0[q] = t0;
    if (nrec) nrec[q] = nr;
  }
  return 0;
}

// Directional derivative of the soft render by forward-mode dual numbers.
// param in [0,5): geometry (cx, cy, th, L, r) of stroke `stroke`;
// param in [5, 5+k): logit (param-5) of stroke `stroke`;
// param in [5+k, 5+k+3k): palette entry (param-5-k)/3, channel (param-5-k)%3.
int orc_soft_jvp(const orc_prog* p, int W, int H, double tau, double tau_min, int inert,
                 const int64_t* pix, int64_t npix, int stroke, int param, double* drgb) {
  typedef Dual<1> D1;
  int n = p->n, k = p->k;
  std::vector<Stroke<D1>> g(n);
  for (int j = 0; j < n; ++j) g[j] = stroke_of<D1>(p, j);
  if (param < 5) {
    D1* f[5] = {&g[stroke].cx, &g[stroke].cy, &g[stroke].th, &g[stroke].L, &g[stroke].r};
    f[param]->d[0] = 1.0;
  }
  // colours as duals: softmax(z/tau_c) . palette
  std::vector<D1> col((size_t)n * 3);
  for (int j = 0; j < n; ++j) {
    std::vector<D1> z(k);
    for (int q = 0; q < k; ++q) {
      z[q] = D1(p->logits[(size_t)j * k + q]);
      if (param >= 5 && param < 5 + k && j == stroke && q == param - 5) z[q].d[0] = 1.0;
    }
    double zmax = z[0].v;
    for (int q = 1; q < k; ++q) zmax = std::max(zmax, z[q].v);
    std::vector<D1> e(k);
    D1 den(0.0);
    for (int q = 0; q < k; ++q) { e[q] = exp((z[q] - zmax) / p->color_temp); den = den + e[q]; }
    for (int c = 0; c < 3; ++c) {
      D1 acc(0.0);
      for (int q = 0; q < k; ++q) {
        D1 pal(p->palette[q * 3 + c]);
        if (param >= 5 + k && (param - 5 - k) == q * 3 + c) pal.d[0] = 1.0;
        acc = acc + (e[q] / den) * pal;
      }
      col[(size_t)j * 3 + c] = acc;
    }
  }
  D1 bg[3] = {D1(p->background[0]), D1(p->background[1]), D1(p->background[2])};
  #pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < npix; ++q) {
    int64_t pidx = pix ? pix[q] : q;
    double x, y;
    pixel_centre(pidx, W, H, x, y);
    D1 out[3];
    soft_pixel<D1>(g, col, bg, tau, tau_min, inert, x, y, out, nullptr, nullptr);
    for (int c = 0; c < 3; ++c) drgb[q * 3 + c] = out[c].d[0];
  }
  return 0;
}

// Stored-state adjoint of the soft render for the linear functional
// J = sum_pixels cot_p . R(p): runs Eq. state forward keeping every state
// s_i = (x_i, T_i) of the pixel, then applies Eq. adjstep / Eq. adjparam from
// i = 1 to N with lambda^C_0 = cot_p, lambda^T_0 = cot_p . c_0, lambda^x_0 = 0.
// The local derivatives d alpha/d(x, theta), D psi and d psi/d theta come from
// dual numbers over psi and the coverage; nothing is regenerated.
// Outputs (summed over the listed pixels): g_geo[n][5] (cx, cy, th, L, r),
// g_col[n][3] (dJ/dc_i), g_logits[n][k], g_pal[k][3] (nullable each except g_geo).
int orc_soft_vjp(const orc_prog* p, int W, int H, double tau, double tau_min, int inert,
                 const int64_t* pix, int64_t npix, const double* cot, double* g_geo,
                 double* g_col, double* g_logits, double* g_pal) {
  int n = p->n, k = p->k;
  std::vector<double> col, prob;
  stroke_colours(p, 0, col, prob);
  int nthreads = 1;
#ifdef _OPENMP
  nthreads = omp_get_max_threads();
#endif
  std::vector<std::vector<double>> acc(nthreads, std::vector<double>((size_t)n * 8, 0.0));
  #pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    std::vector<double>& my = acc[tid];
    std::vector<double> xs(n), ys(n), Ts(n);
    #pragma omp for schedule(dynamic, 16)
    for (int64_t q = 0; q < npix; ++q) {
      int64_t pidx = pix ? pix[q] : q;
      double x, y;
      pixel_centre(pidx, W, H, x, y);
      // forward, storing s_i (position at which stroke i is evaluated, and T_i)
      double Tr = 1.0;
      for (int j = n - 1; j >= 0; --j) {
        Stroke<double> g = stroke_of<double>(p, j);
        xs[j] = x; ys[j] = y; Ts[j] = Tr;
        double s, h;
        to_frame(x, y, g, s, h);
        double a = soft_coverage(deposit_margin(s, h, segment_distance(s, h, g.L), g), g.r, tau, tau_min);
        Tr = Tr * (1.0 - a);
        if (!inert) { double xo, yo; psi(x, y, g, kFloor, xo, yo); x = xo; y = yo; }
      }
      // backward, i = 1..N (program index j = 0..n-1)
      double lC[3] = {cot[q * 3], cot[q * 3 + 1], cot[q * 3 + 2]};
      double lT = lC[0] * p->background[0] + lC[1] * p->background[1] + lC[2] * p->background[2];
      double lx[2] = {0.0, 0.0};
      for (int j = 0; j < n; ++j) {
        typedef Dual<7> D7;
        D7 xd(xs[j]), yd(ys[j]);
        xd.d[0] = 1; yd.d[1] = 1;
        Stroke<D7> gd = stroke_of<D7>(p, j);
        gd.cx.d[2] = 1; gd.cy.d[3] = 1; gd.th.d[4] = 1; gd.L.d[5] = 1; gd.r.d[6] = 1;
        D7 s, h;
        to_frame(xd, yd, gd, s, h);
        D7 a = soft_coverage(deposit_margin(s, h, segment_distance(s, h, gd.L), gd), gd.r, tau, tau_min);
        double J[2][7];
        if (inert) {
          for (int r = 0; r < 2; ++r) for (int c = 0; c < 7; ++c) J[r][c] = (r == c) ? 1.0 : 0.0;
        } else {
          D7 xo, yo;
          psi(xd, yd, gd, kFloor, xo, yo);
          for (int c = 0; c < 7; ++c) { J[0][c] = xo.d[c]; J[1][c] = yo.d[c]; }
        }
        const double* cj = &col[(size_t)j * 3];
        double lCc = lC[0] * cj[0] + lC[1] * cj[1] + lC[2] * cj[2];
        double Ti = Ts[j];
        double mu = Ti * (lCc - lT);
        double* gj = &my[(size_t)j * 8];
        for (int t = 0; t < 5; ++t) gj[t] += mu * a.d[2 + t] + lx[0] * J[0][2 + t] + lx[1] * J[1][2 + t];
        for (int c = 0; c < 3; ++c) gj[5 + c] += lC[c] * Ti * a.v;
        double lT_new = (1.0 - a.v) * lT + a.v * lCc;
        double lx0 = J[0][0] * lx[0] + J[1][0] * lx[1] + mu * a.d[0];
        double lx1 = J[0][1] * lx[0] + J[1][1] * lx[1] + mu * a.d[1];
        lT = lT_new; lx[0] = lx0; lx[1] = lx1;
      }
    }
  }
  std::vector<double> tot((size_t)n * 8, 0.0);
  for (int t = 0; t < nthreads; ++t)
    for (size_t i = 0; i < tot.size(); ++i) tot[i] += acc[t][i];
  for (int j = 0; j < n; ++j) {
    for (int t = 0; t < 5; ++t) g_geo[(size_t)j * 5 + t] = tot[(size_t)j * 8 + t];
    if (g_col) for (int c = 0; c < 3; ++c) g_col[(size_t)j * 3 + c] = tot[(size_t)j * 8 + 5 + c];
  }
  // colour chain rule: c_j = sum_q p_jq Pal_q, p = softmax(z / tau_c):
  // dc_j/dz_jq = p_jq (Pal_q - c_j) / tau_c.
  if (g_logits) {
    for (int j = 0; j < n; ++j)
      for (int q = 0; q < k; ++q) {
        double d = 0.0;
        for (int c = 0; c < 3; ++c)
          d += (p->palette[q * 3 + c] - col[(size_t)j * 3 + c]) * tot[(size_t)j * 8 + 5 + c];
        g_logits[(size_t)j * k + q] = prob[(size_t)j * k + q] * d / p->color_temp;
      }
  }
  if (g_pal) {
    for (int q = 0; q < k; ++q)
      for (int c = 0; c < 3; ++c) {
        double d = 0.0;
        for (int j = 0; j < n; ++j) d += prob[(size_t)j * k + q] * tot[(size_t)j * 8 + 5 + c];
        g_pal[q * 3 + c] = d;
      }
  }
  return 0;
}

// One-pass closed-form compensation (Sec. "Closed-form compensation
// baseline"): from the last stroke to the first, each stroke of the given
// (inert-mark) program is moved so that the transport of every later, already
// compensated stroke carries it back to where the program puts it.  Its segment
// start (anchor variant: the offset vector is kept) or both ends (endpoint
// variant) are pre-imaged through psi_j (Eq. back) of the strokes j after it,
// the last one first.  A point inside K_j has no pre-image (Lemma
// "obstruction"); that step is clamped onto the segment by the ideal extension
// of psi_j (skip = 0) or skipped (skip = 1), and the stroke counts as blocked.
// Outputs the compensated cx, cy, th, L (r and colours are unchanged) and the
// blocked flags; returns the number of blocked strokes.
int orc_compensate(const orc_prog* p, int endpoint, int skip, double* cx, double* cy, double* th, double* L,
                   int32_t* blocked) {
  const int n = p->n;
  std::vector<Stroke<double>> c(n);
  int nblocked = 0;
  for (int i = n - 1; i >= 0; --i) {
    const Stroke<double> g = stroke_of<double>(p, i);
    const double ex = std::cos(g.th), ey = std::sin(g.th);
    double pt[2][2] = {{g.cx - 0.5 * g.L * ex, g.cy - 0.5 * g.L * ey},
                       {g.cx + 0.5 * g.L * ex, g.cy + 0.5 * g.L * ey}};
    int blk = 0;
    for (int q = 0; q < (endpoint ? 2 : 1); ++q) {
      double x = pt[q][0], y = pt[q][1];
      for (int j = n - 1; j > i; --j) {
        double s, h;
        to_frame(x, y, c[j], s, h);
        if (deposit_margin(s, h, segment_distance(s, h, c[j].L), c[j]) <= 0.0) {
          blk = 1;
          if (skip) continue;
        }
        double xo, yo;
        psi(x, y, c[j], kClamp, xo, yo);
        x = xo; y = yo;
      }
      pt[q][0] = x; pt[q][1] = y;
    }
    Stroke<double> o = g;
    if (endpoint) {
      const double dx = pt[1][0] - pt[0][0], dy = pt[1][1] - pt[0][1];
      o.L = std::hypot(dx, dy);
      if (o.L > 0.0) o.th = std::atan2(dy, dx);
      o.cx = 0.5 * (pt[0][0] + pt[1][0]);
      o.cy = 0.5 * (pt[0][1] + pt[1][1]);
    } else {
      o.cx = pt[0][0] + 0.5 * g.L * ex;
      o.cy = pt[0][1] + 0.5 * g.L * ey;
    }
    c[i] = o;
    cx[i] = o.cx; cy[i] = o.cy; th[i] = o.th; L[i] = o.L;
    blocked[i] = blk;
    nblocked += blk;
  }
  return nblocked;
}

// The coupling variant on a batch of points (Eq. coupling with the profile
// c1..c3 of Eq. profile): direction 0 = psi_g (mode as orc_map: 0 clamp,
// 1 floor), 1 = Phi_g.  If jac is non-null it receives d(x_out, y_out)/d(x, y)
// per point (2x2, row-major).  If v is non-null it receives the centred
// coordinate v of each input point, and sig_b (nullable) the deposit boundary
// sigma_b(v) there.
int orc_map_coupled(const double* pts, int64_t n, double cx, double cy, double th, double L, double r,
                    double c1, double c2, double c3, int direction, int mode, double* out, double* jac,
                    double* v, double* sig_b) {
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    typedef Dual<2> D2;
    D2 x(pts[2 * i]), y(pts[2 * i + 1]), xo, yo;
    x.d[0] = 1; y.d[1] = 1;
    Stroke<D2> g{D2(cx), D2(cy), D2(th), D2(L), D2(r), c1, c2, c3};
    if (direction == 0) psi(x, y, g, mode, xo, yo);
    else phi(x, y, g, false, xo, yo);
    out[2 * i] = xo.v; out[2 * i + 1] = yo.v;
    if (jac) { jac[4 * i] = xo.d[0]; jac[4 * i + 1] = xo.d[1]; jac[4 * i + 2] = yo.d[0]; jac[4 * i + 3] = yo.d[1]; }
    if (v || sig_b) {
      Stroke<double> gv{cx, cy, th, L, r, c1, c2, c3};
      double s, h;
      to_frame(pts[2 * i], pts[2 * i + 1], gv, s, h);
      const double vv = centred_v(s, h, segment_distance(s, h, L), L);
      if (v) v[i] = vv;
      if (sig_b) sig_b[i] = deposit_sigma(gv, vv);
    }
  }
  return 0;
}

// Smallest value of g over a leaf (Eq. profile).  In w = cos(4 pi v) the
// modes are Chebyshev polynomials, so g is the cubic
// 1 + c1 w + c2 (2 w^2 - 1) + c3 (4 w^3 - 3 w) on [-1, 1]; its minimum is at
// w = +-1 or at a root of its derivative 12 c3 w^2 + 4 c2 w + (c1 - 3 c3).
double orc_profile_min(double c1, double c2, double c3) {
  auto gw = [&](double w) { return 1.0 + c1 * w + c2 * (2.0 * w * w - 1.0) + c3 * (4.0 * w * w * w - 3.0 * w); };
  double m = std::min(gw(-1.0), gw(1.0));
  const double a = 12.0 * c3, b = 4.0 * c2, c = c1 - 3.0 * c3;
  if (a == 0.0) {
    if (b != 0.0) {
      const double w = -c / b;
      if (w > -1.0 && w < 1.0) m = std::min(m, gw(w));
    }
  } else {
    const double disc = b * b - 4.0 * a * c;
    if (disc >= 0.0) {
      const double sq = std::sqrt(disc);
      for (double w : {(-b - sq) / (2.0 * a), (-b + sq) / (2.0 * a)})
        if (w > -1.0 && w < 1.0) m = std::min(m, gw(w));
    }
  }
  return m;
}

// Operation counts per pixel-stroke (the tallies of the Ops scalar above;
// measurement only).  transport: 0 the capsule map (with the coupling profile
// when the program carries one), 2 the sixteen-drop operator of R_D (hard and
// soft render only: the paper uses R_D forward only).  For each listed pixel:
//   hard:     every visited step of Eq. chain (frame, distance, membership,
//             and psi with the ideal clamp when the point passes on);
//   soft:     every step of the soft render (frame, distance, Eq. relax
//             coverage, Eq. state compositing as written in soft_pixel, psi
//             with the floor);
//   adjoint:  every step of the replay adjoint of Sec. 5.2 in program order:
//             regeneration x_i = Phi_i(x_{i-1}) (Eq. rpos), the frame, distance
//             and coverage of x_i, the reverse sweep through psi_i and alpha_i
//             (psi's own forward is not tallied: its intermediates are Phi's),
//             and the scalar lines of Eq. rT / Eq. adjstep as the stored-state
//             adjoint writes them (T_i = T_{i-1} / (1 - alpha_i); lambda_C . c_i;
//             mu; the colour gradient; lambda_T).
// out[0..2]  hard: visited steps, FP32, XU (totals)
// out[3..5]  soft: pixel-strokes, FP32, XU
// out[6..7]  adjoint regeneration FP32, XU
// out[8..9]  adjoint coverage FP32, XU
// out[10..11] adjoint reverse sweep FP32 (contributions + accumulation adds), XU
// out[12..13] adjoint scalar step FP32, XU
int orc_count_ops(const orc_prog* p, int W, int H, double tau, double tau_min, int transport, const int64_t* pix,
                  int64_t npix, double* out) {
  if (transport != kCapsule && transport != kDrops16) return -1;
  if (transport == kDrops16 && p->coupling) return -1;
  const int n = p->n;
  std::vector<double> col, prob;
  stroke_colours(p, 0, col, prob);
  double tot[14] = {0};
  #pragma omp parallel
  {
    double my[14] = {0};
    std::vector<double> xs(n), ys(n);
    #pragma omp for schedule(dynamic, 16)
    for (int64_t q = 0; q < npix; ++q) {
      int64_t pidx = pix ? pix[q] : q;
      double px0, py0;
      pixel_centre(pidx, W, H, px0, py0);
      auto stroke_ops = [&](int j) {
        Stroke<Ops> g;
        g.cx = Ops::leaf(p->cx[j], false); g.cy = Ops::leaf(p->cy[j], false);
        g.th = Ops::leaf(p->th[j], false); g.L = Ops::leaf(p->L[j], false); g.r = Ops::leaf(p->r[j], false);
        if (p->coupling) {
          g.c1 = p->coupling[3 * j]; g.c2 = p->coupling[3 * j + 1]; g.c3 = p->coupling[3 * j + 2];
        }
        return g;
      };
      // the pull-back of one step from the frame quantities already computed
      auto pull_back = [&](const Ops& X, const Ops& Y, const Ops& s, const Ops& h, const Ops& sp,
                           const Stroke<Ops>& g, int mode, Ops& xo, Ops& yo) {
        if (transport == kDrops16) psi_drops(X, Y, g, xo, yo);
        else psi_from_frame(s, h, sp, g, mode, xo, yo);
      };
      // hard render
      double x = px0, y = py0;
      for (int j = n - 1; j >= 0; --j) {
        g_tally.reset();
        Stroke<Ops> g = stroke_ops(j);
        Ops X = Ops::leaf(x, true), Y = Ops::leaf(y, true), s, h, xo, yo;
        to_frame(X, Y, g, s, h);
        Ops sp = segment_distance(s, h, g.L);
        Ops m = deposit_margin(s, h, sp, g);
        my[0] += 1;
        if (value(m) <= 0.0) { my[1] += g_tally.f; my[2] += g_tally.x; break; }
        pull_back(X, Y, s, h, sp, g, kClamp, xo, yo);
        my[1] += g_tally.f; my[2] += g_tally.x;
        x = value(xo); y = value(yo);
      }
      // soft render, storing the position at which each stroke is evaluated
      x = px0; y = py0;
      double Tv = 1.0;
      for (int j = n - 1; j >= 0; --j) {
        xs[j] = x; ys[j] = y;
        g_tally.reset();
        Stroke<Ops> g = stroke_ops(j);
        Ops X = Ops::leaf(x, true), Y = Ops::leaf(y, true), s, h, xo, yo;
        Ops Tr = Ops::leaf(Tv, true);
        Ops C[3] = {Ops::leaf(0.1, true), Ops::leaf(0.2, true), Ops::leaf(0.3, true)};
        to_frame(X, Y, g, s, h);
        Ops sp = segment_distance(s, h, g.L);
        Ops a = soft_coverage(deposit_margin(s, h, sp, g), g.r, tau, tau_min);
        for (int c = 0; c < 3; ++c) C[c] = C[c] + Tr * a * Ops::leaf(col[(size_t)j * 3 + c], false);
        Tr = Tr * (1.0 - a);
        pull_back(X, Y, s, h, sp, g, kFloor, xo, yo);
        my[3] += 1; my[4] += g_tally.f; my[5] += g_tally.x;
        x = value(xo); y = value(yo); Tv = value(Tr);
      }
      // replay adjoint, program order; x is now the pulled-back point x_0
      for (int j = 0; j < n && transport == kCapsule; ++j) {
        // regeneration of x_j from the point below it
        g_tally.reset();
        {
          Stroke<Ops> g = stroke_ops(j);
          Ops X = Ops::leaf(x, true), Y = Ops::leaf(y, true), xo, yo;
          phi(X, Y, g, false, xo, yo);
        }
        my[6] += g_tally.f; my[7] += g_tally.x;
        // coverage of x_j, then the reverse sweep through psi_j and alpha_j
        g_tally.reset();
        Stroke<Ops> g = stroke_ops(j);
        Ops X = Ops::leaf(xs[j], true), Y = Ops::leaf(ys[j], true), s, h, xo, yo;
        to_frame(X, Y, g, s, h);
        Ops sp = segment_distance(s, h, g.L);
        Ops a = soft_coverage(deposit_margin(s, h, sp, g), g.r, tau, tau_min);
        my[8] += g_tally.f; my[9] += g_tally.x;
        psi_from_frame(s, h, sp, g, kFloor, xo, yo);
        ops_use(xo); ops_use(yo); ops_use(a);  // the seeds lambda_x and mu
        my[10] += g_tally.rf + g_tally.accumulation_adds(); my[11] += g_tally.rx;
        // T_i = T_{i-1} / (1 - alpha_i): 1 + a reciprocal + 1; lambda_C . c_i: 5;
        // mu = T_i (lambda_C . c_i - lambda_T): 2; colour gradient
        // g_c += lambda_C T_i alpha_i: 3 x 3; lambda_T = (1 - alpha) lambda_T +
        // alpha (lambda_C . c_i): 4
        my[12] += 2 + 5 + 2 + 9 + 4; my[13] += 1;
        x = xs[j]; y = ys[j];  // the next stroke's regeneration starts from x_j
      }
    }
    #pragma omp critical
    for (int i = 0; i < 14; ++i) tot[i] += my[i];
  }
  for (int i = 0; i < 14; ++i) out[i] = tot[i];
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
