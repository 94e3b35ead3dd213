"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/), closed forms (the drop map), exact invariants
(round trip, area, symmetry, commutation, compositing), brute force on tiny
inputs and finite differences.  A plausible slip in the oracle (a dropped term,
a wrong sign or index, a transposed operand) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2609_08722_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DETJ = json.load(open(os.path.join(GOLDEN, "table_detj.json")))
SIDE = json.load(open(os.path.join(GOLDEN, "side_table.json")))


def seg_distance(pts, stroke):
    """Distance to the segment by projection onto [a, b] (independent of the oracle's fold)."""
    cx, cy, th, L, r = stroke
    e = np.array([math.cos(th), math.sin(th)])
    a = np.array([cx, cy]) - 0.5 * L * e
    if L == 0:
        return np.hypot(pts[:, 0] - cx, pts[:, 1] - cy)
    t = np.clip((pts - a) @ e / L, 0.0, 1.0)
    foot = a[None, :] + (t * L)[:, None] * e[None, :]
    return np.hypot(*(pts - foot).T)


def exterior_sample(stroke, n=200_000, box=0.5, seed=7):
    cx, cy = stroke[0], stroke[1]
    u = inputs.uniform(seed, 4 * n).reshape(-1, 2)
    pts = np.array([cx, cy]) + (2 * u - 1) * box
    return pts[seg_distance(pts, stroke) > stroke[4]][:n]


CAPSULE = (0.0, 0.0, 0.0, DETJ["capsule"]["L"], DETJ["capsule"]["r"])
ROTATED = (0.31, 0.62, 1.1, 0.13, 0.045)


def reflect_bisector(p, stroke):
    """Mirror across the segment's perpendicular bisector."""
    cx, cy, th = stroke[:3]
    e = np.array([math.cos(th), math.sin(th)])
    d = p - np.array([cx, cy])
    return p - 2.0 * (d @ e)[:, None] * e[None, :]


def reflect_line(p, stroke):
    """Mirror across the segment's supporting line."""
    cx, cy, th = stroke[:3]
    n = np.array([-math.sin(th), math.cos(th)])
    d = p - np.array([cx, cy])
    return p - 2.0 * (d @ n)[:, None] * n[None, :]


def steiner_area(L, s):
    return 2 * L * s + math.pi * s * s


# --------------------------------------------------------------------------- operator

@pytest.mark.parametrize("stroke", [(0.3, 0.6, 0.7, 0.0, 0.04), (0.5, 0.5, 2.0, 0.0, 0.01)])
def test_drop_limit_is_the_drop_map(stroke):
    """At L = 0, Eq. back is the radial drop map sigma = sqrt(sigma'^2 - r^2) and
    its inverse is x' = c + (x - c) sqrt(1 + r^2/|x - c|^2) (Sec. 4, drop limit)."""
    cx, cy, _, _, r = stroke
    pts = exterior_sample(stroke, 20_000)
    c = np.array([cx, cy])
    d = pts - c
    rho = np.hypot(*d.T)
    back = c + d * (np.sqrt(rho ** 2 - r ** 2) / rho)[:, None]
    fwd = c + d * np.sqrt(1.0 + r ** 2 / rho ** 2)[:, None]
    assert np.abs(oracle.psi_map(pts, stroke, oracle.MODE_CLAMP) - back).max() < 1e-14
    assert np.abs(oracle.phi_map(pts, stroke) - fwd).max() < 1e-14


def test_short_capsule_converges_to_drop():
    """Table detj, row 'drop limit, L = 1e-6' prints 2.9e-6 (FP64) for an
    unspecified point sample; on the uniform sample the deviation is of that
    order and shrinks in proportion to L."""
    r = CAPSULE[4]
    pts = exterior_sample(CAPSULE)
    rho = np.hypot(*pts.T)
    drop = pts * (np.sqrt(rho ** 2 - r ** 2) / rho)[:, None]
    err = {}
    for L in (1e-6, 1e-7):
        got = oracle.psi_map(pts, (0.0, 0.0, 0.0, L, r), oracle.MODE_CLAMP)
        far = rho > r + 1e-3
        err[L] = np.abs(got - drop)[far].max()
    printed = DETJ["float64"]["drop_limit_L_1e-6"]
    assert printed / 30 < err[1e-6] < printed * 3
    assert 5.0 < err[1e-6] / err[1e-7] < 20.0


@pytest.mark.parametrize("stroke", [CAPSULE, ROTATED])
def test_round_trip(stroke):
    """Phi o psi = id on the exterior and psi o Phi = id off the segment
    (Prop. 1; Table detj prints 5.7e-15 in FP64)."""
    pts = exterior_sample(stroke)
    rt = oracle.phi_map(oracle.psi_map(pts, stroke, oracle.MODE_CLAMP), stroke)
    assert np.abs(rt - pts).max() < 20 * DETJ["float64"]["round_trip"]
    u = inputs.uniform(3, 2 * 50_000).reshape(-1, 2) - 0.5 + np.array(stroke[:2])
    rt2 = oracle.psi_map(oracle.phi_map(u, stroke), stroke, oracle.MODE_CLAMP)
    assert np.abs(rt2 - u).max() < 20 * DETJ["float64"]["round_trip"]


@pytest.mark.parametrize("direction", [0, 1])
def test_area_jacobian(direction):
    """det D psi = det D Phi = 1 on the exterior (Prop. 1; Table detj prints
    1.6e-15 for |det J - 1| in FP64)."""
    pts = exterior_sample(ROTATED, 50_000)
    J = oracle.map_jacobian(pts, ROTATED, direction=direction, mode=oracle.MODE_CLAMP)
    det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    assert np.abs(det - 1.0).max() < 1e-12


def _richardson_area(curve_fn, n):
    """Shoelace area of a closed curve sampled at n and 2n points, Richardson-extrapolated."""
    def shoelace(p):
        x, y = p[:, 0] - p[:, 0].mean(), p[:, 1] - p[:, 1].mean()
        return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))
    a1, a2 = shoelace(curve_fn(n)), shoelace(curve_fn(2 * n))
    return (4 * a2 - a1) / 3


def _square(x0, y0, side, n):
    t = np.arange(n) / n * 4
    k = np.floor(t).astype(int)
    f = t - k
    corners = np.array([[x0, y0], [x0 + side, y0], [x0 + side, y0 + side], [x0, y0 + side], [x0, y0]])
    return corners[k] + (corners[k + 1] - corners[k]) * f[:, None]


def test_polygon_area_preserved():
    """A fine polygon outside the footprint keeps its area under psi to 1e-9
    (Prop. 1, measure preservation)."""
    stroke = ROTATED
    side, x0, y0 = 0.05, 0.45, 0.78
    corners = _square(x0, y0, side, 64)
    assert seg_distance(corners, stroke).min() > stroke[4]
    area = _richardson_area(lambda n: oracle.psi_map(_square(x0, y0, side, n), stroke, oracle.MODE_CLAMP), 1 << 16)
    assert abs(area - side * side) / (side * side) < 1e-9


def test_deposit_adds_capsule_area():
    """Phi sends the parallel curve {sigma = s0} to the one enclosing
    A_L(s0) + A_L(r): the deposit adds 2 L r + pi r^2 (Eq. steiner, Eq. phi)."""
    cx, cy, th, L, r = ROTATED
    s0 = 0.02

    def stadium(n):
        t = np.arange(n) / n * (2 * L + 2 * math.pi * s0)
        pts = np.empty((n, 2))
        for i, a in enumerate(t):
            if a < L:
                p = (-L / 2 + a, -s0)
            elif a < L + math.pi * s0:
                ang = (a - L) / s0 - math.pi / 2
                p = (L / 2 + s0 * math.cos(ang), s0 * math.sin(ang))
            elif a < 2 * L + math.pi * s0:
                p = (L / 2 - (a - L - math.pi * s0), s0)
            else:
                ang = (a - 2 * L - math.pi * s0) / s0
                p = (-L / 2 - s0 * math.sin(ang), s0 * math.cos(ang))
            pts[i] = p
        e = np.array([math.cos(th), math.sin(th)])
        en = np.array([-math.sin(th), math.cos(th)])
        return np.array([cx, cy]) + pts[:, :1] * e + pts[:, 1:] * en

    area = _richardson_area(lambda n: oracle.phi_map(stadium(n), ROTATED), 1 << 13)
    want = steiner_area(L, s0) + steiner_area(L, r)
    assert abs(area - want) / want < 1e-9


@pytest.mark.parametrize("stroke", [CAPSULE, ROTATED])
def test_reflection_symmetry(stroke):
    """Centred v commutes with both mirror symmetries of the capsule (Prop. 2;
    Table detj: 5.9e-15); keeping raw q breaks the midplane mirror at ~4.6e-2."""
    pts = exterior_sample(stroke)
    for refl in (reflect_bisector, reflect_line):
        a = oracle.psi_map(refl(pts, stroke), stroke, oracle.MODE_CLAMP)
        b = refl(oracle.psi_map(pts, stroke, oracle.MODE_CLAMP), stroke)
        assert np.abs(a - b).max() < 1e-13
    if stroke is CAPSULE:
        a = oracle.psi_map(reflect_bisector(pts, stroke), stroke, oracle.MODE_RAWQ)
        b = reflect_bisector(oracle.psi_map(pts, stroke, oracle.MODE_RAWQ), stroke)
        printed = DETJ["float64"]["midplane_reflection_raw_q"]
        assert printed / 1.5 < np.abs(a - b).max() < printed * 1.5


def test_same_segment_insertions_commute():
    """Insertions at the same segment commute and compose to one insertion of
    the summed area (Sec. 3; Phi is a translation in u)."""
    cx, cy, th, L, _ = ROTATED
    r1, r2 = 0.02, 0.035
    area = steiner_area(L, r1) + steiner_area(L, r2)
    r3 = (-2 * L + math.sqrt(4 * L * L + 4 * math.pi * area)) / (2 * math.pi)
    s1, s2, s3 = (cx, cy, th, L, r1), (cx, cy, th, L, r2), (cx, cy, th, L, r3)
    pts = exterior_sample(s3, 50_000)
    a = oracle.psi_map(oracle.psi_map(pts, s2, oracle.MODE_CLAMP), s1, oracle.MODE_CLAMP)
    b = oracle.psi_map(oracle.psi_map(pts, s1, oracle.MODE_CLAMP), s2, oracle.MODE_CLAMP)
    c = oracle.psi_map(pts, s3, oracle.MODE_CLAMP)
    assert np.abs(a - b).max() < 1e-13
    assert np.abs(a - c).max() < 1e-13


def test_interior_extension_and_floor():
    """Inside the footprint the clamped map sends a flank point at signed
    arclength t and distance sigma' to l t/(l + pi sigma') on the segment (Sec. 4,
    'The chain'); the epsilon-floor lands within eps r / sqrt(pi) of the segment
    on the same side and flags the sample (Sec. 5.2)."""
    cx, cy, th, L, r = ROTATED
    u = inputs.uniform(11, 2 * 5000).reshape(-1, 2)
    s = (u[:, 0] - 0.5) * L
    h = (u[:, 1] - 0.5) * 2 * r * 0.999
    e = np.array([math.cos(th), math.sin(th)])
    en = np.array([-math.sin(th), math.cos(th)])
    pts = np.array([cx, cy]) + s[:, None] * e + h[:, None] * en
    out = oracle.psi_map(pts, ROTATED, oracle.MODE_CLAMP)
    d = out - np.array([cx, cy])
    s_new, h_new = d @ e, d @ en
    want = s * L / (L + math.pi * np.abs(h))
    assert np.abs(s_new - want).max() < 1e-14
    assert np.abs(h_new).max() < 1e-15
    outf, fl = oracle.psi_map(pts, ROTATED, oracle.MODE_FLOOR, return_floored=True)
    df = outf - np.array([cx, cy])
    hf = df @ en
    assert fl.all()
    assert (np.abs(hf) <= 1e-3 * r / math.sqrt(math.pi) * (1 + 1e-12)).all()
    assert (np.sign(hf) == np.sign(h)).all()


# --------------------------------------------------------------------------- renderers

def _tiny_program(n, seed, k=4, r_lo=0.05, r_hi=0.2, len_max=0.4):
    return inputs.make_program(n, seed=seed, palette_seed=seed + 1, k=k, r_lo=r_lo, r_hi=r_hi,
                               len_max=len_max)


def test_compositing_identity():
    """sum_i T_i alpha_i + T_0 = 1 per pixel (Sec. 6 visible-area identity):
    white strokes on a white background render exactly white, and white strokes
    on black render 1 - T_0."""
    p = _tiny_program(12, 5)
    p.palette[:] = 1.0
    got = oracle.render_soft(p, 24, 24, 0.1, 0.01)
    assert np.abs(got["rgb"] - 1.0).max() < 1e-12
    p.background[:] = 0.0
    got = oracle.render_soft(p, 24, 24, 0.1, 0.01)
    assert np.abs(got["rgb"] - (1.0 - got["T0"])[:, None]).max() < 1e-12


def test_inert_soft_render_is_over_compositing():
    """With psi = id (inert-mark model, Definition 1) Eq. render is ordinary
    back-to-front 'over' compositing of the coverage of each capsule."""
    p = _tiny_program(9, 17)
    W = H = 20
    tau, tau_min = 0.2, 0.01
    got = oracle.render_soft(p, W, H, tau, tau_min, inert=True)["rgb"]
    jj, ii = np.meshgrid(np.arange(W), np.arange(H))
    pts = np.stack([(jj.ravel() + 0.5) / W, (ii.ravel() + 0.5) / H], 1)
    z = p.logits.astype(np.float64) / p.color_temp
    prob = np.exp(z - z.max(1, keepdims=True))
    prob /= prob.sum(1, keepdims=True)
    col = prob @ p.palette.astype(np.float64)
    img = np.tile(p.background.astype(np.float64), (W * H, 1))
    for j in range(p.n):           # paint in program order, each stroke over the last
        st = tuple(float(v) for v in (p.cx[j], p.cy[j], p.theta[j], p.length[j], p.half_width[j]))
        w = max(tau * st[4], tau_min)
        a = np.minimum(1 / (1 + np.exp(-(st[4] - seg_distance(pts, st)) / w)), 1 - 1e-7)
        img = a[:, None] * col[j] + (1 - a[:, None]) * img
    assert np.abs(got - img).max() < 1e-12


def test_single_stroke_hard_render_is_the_capsule():
    st = (0.45, 0.55, 0.6, 0.3, 0.12)
    p = inputs.Program(cx=np.array([st[0]]), cy=np.array([st[1]]), theta=np.array([st[2]]),
                       length=np.array([st[3]]), half_width=np.array([st[4]]),
                       logits=np.zeros((1, 1)), palette=np.array([[0.2, 0.4, 0.6]]),
                       background=np.ones(3), color_temp=1.0)
    W = H = 64
    got = oracle.render_hard(p, W, H)
    jj, ii = np.meshgrid(np.arange(W), np.arange(H))
    pts = np.stack([(jj.ravel() + 0.5) / W, (ii.ravel() + 0.5) / H], 1)
    inside = seg_distance(pts, st) <= st[4]
    assert np.array_equal(got["idx"] == 0, inside)
    assert np.allclose(got["rgb"][inside], [0.2, 0.4, 0.6])


def test_hard_chain_against_forward_replay():
    """Brute force on a tiny program: trace each pixel back stroke by stroke
    (Eq. chain) with the single-map routine and the projection distance, compare
    the terminating stroke, then carry the in-deposit point forward through the
    later strokes with Phi and land back on the pixel (Eq. rpos)."""
    p = _tiny_program(8, 23, r_lo=0.03, r_hi=0.12)
    W = H = 16
    got = oracle.render_hard(p, W, H, with_kappa=True)
    checked = 0
    for q in range(W * H):
        x0 = np.array([[(q % W + 0.5) / W, (q // W + 0.5) / H]])
        x = x0.copy()
        hit = -1
        path = []
        for j in range(p.n - 1, -1, -1):
            st = tuple(float(v) for v in (p.cx[j], p.cy[j], p.theta[j], p.length[j], p.half_width[j]))
            if seg_distance(x, st)[0] <= st[4]:
                hit = j
                break
            path.append(st)
            x = oracle.psi_map(x, st, oracle.MODE_CLAMP)
        if got["margin"][q] < 1e-9:
            continue
        assert hit == got["idx"][q]
        y = x.copy()
        for st in reversed(path):
            y = oracle.phi_map(y, st)
        assert np.abs(y - x0).max() < 1e-12 * max(1.0, got["kappa"][q])
        checked += 1
    assert checked > 0.95 * W * H


def _drops_program(strokes):
    a = np.asarray(strokes, dtype=np.float64)
    n = a.shape[0]
    return inputs.Program(cx=a[:, 0], cy=a[:, 1], theta=a[:, 2], length=a[:, 3], half_width=a[:, 4],
                          logits=np.zeros((n, 1)), palette=np.array([[0.2, 0.4, 0.6]]),
                          background=np.ones(3), color_temp=1.0)


def _pixel_points(W, H):
    jj, ii = np.meshgrid(np.arange(W), np.arange(H))
    return np.stack([(jj.ravel() + 0.5) / W, (ii.ravel() + 0.5) / H], 1)


def test_chain_condition_of_concentric_drops_is_the_radial_stretch():
    """kappa (the product over the passed strokes of ||D psi_j||_2) in closed
    form.  A drop's pull-back sends radius rho to sqrt(rho^2 - r^2): it
    stretches radially by rho / sqrt(rho^2 - r^2) (> 1) and shrinks
    tangentially by the inverse, so ||D psi||_2 is the radial factor.  Two
    concentric drops telescope: rho / rho_1 for a pixel stopped by the first
    (program index 0), rho / rho_0 for one that passes both, 1 for a pixel
    inside the last.  A Frobenius norm, a smaller singular value or a missing
    factor fails it."""
    c = (0.5, 0.5)
    r0, r1 = 0.09, 0.07
    p = _drops_program([(c[0], c[1], 0.3, 0.0, r0), (c[0], c[1], 1.2, 0.0, r1)])
    W = H = 64
    got = oracle.render_hard(p, W, H, with_kappa=True)
    rho = np.hypot(*(_pixel_points(W, H) - np.array(c)).T)
    rho1 = np.sqrt(np.maximum(rho ** 2 - r1 ** 2, 0.0))
    rho0 = np.sqrt(np.maximum(rho1 ** 2 - r0 ** 2, 0.0))
    want = np.where(rho <= r1, 1.0, np.where(rho1 <= r0, rho / np.maximum(rho1, 1e-300),
                                             rho / np.maximum(rho0, 1e-300)))
    ok = got["margin"] > 1e-9
    assert np.array_equal(got["idx"][ok], np.where(rho <= r1, 1, np.where(rho1 <= r0, 0, -1))[ok])
    assert np.abs(got["kappa"][ok] / want[ok] - 1.0).max() < 1e-12
    assert (want[ok & (rho1 > r0)] > 1.0).all()


def test_chain_condition_against_svd_of_difference_jacobians():
    """kappa on a small capsule program against a brute-force chain: trace
    each pixel with the single-map routine, take each passed stroke's 2x2
    Jacobian by central differences and its largest singular value by numpy's
    SVD, and multiply.  Independent of the oracle's dual numbers and of its
    closed-form 2x2 spectral norm."""
    p = _tiny_program(6, 29, r_lo=0.04, r_hi=0.12)
    W = H = 12
    got = oracle.render_hard(p, W, H, with_kappa=True)
    h = 1e-6
    checked = 0
    for q, x0 in enumerate(_pixel_points(W, H)):
        if got["margin"][q] < 1e-6:
            continue
        x = x0[None, :].copy()
        kap = 1.0
        for j in range(p.n - 1, -1, -1):
            st = tuple(float(v) for v in (p.cx[j], p.cy[j], p.theta[j], p.length[j], p.half_width[j]))
            if seg_distance(x, st)[0] <= st[4]:
                break
            pts = x + np.array([[h, 0.0], [-h, 0.0], [0.0, h], [0.0, -h]])
            y = oracle.psi_map(pts, st, oracle.MODE_CLAMP)
            J = np.stack([(y[0] - y[1]) / (2 * h), (y[2] - y[3]) / (2 * h)], 1)
            kap *= np.linalg.svd(J, compute_uv=False)[0]
            x = oracle.psi_map(x, st, oracle.MODE_CLAMP)
        assert abs(got["kappa"][q] / kap - 1.0) < 1e-6, q
        checked += 1
    assert checked > 0.9 * W * H
    assert got["kappa"].max() > 1.5


def test_chain_condition_of_the_inert_render_is_one():
    p = _tiny_program(6, 31, r_lo=0.04, r_hi=0.12)
    got = oracle.render_hard(p, 16, 16, with_kappa=True, inert=True)
    assert np.array_equal(got["kappa"], np.ones(256))


def test_soft_render_tends_to_hard():
    """As the relaxation width goes to zero, Eq. relax tends to the indicator
    and the soft render to the hard render away from deposit boundaries."""
    p = _tiny_program(10, 31, r_lo=0.03, r_hi=0.1)
    W = H = 24
    hard = oracle.render_hard(p, W, H)
    errs = []
    for tmin in (1e-3, 1e-4, 1e-5):
        soft = oracle.render_soft(p, W, H, 0.0, tmin)["rgb"]
        far = hard["margin"] > 2e-2
        errs.append(np.abs(soft - hard["rgb"])[far].max())
    assert errs[-1] < 1e-6
    assert errs[0] >= errs[1] >= errs[2]


# --------------------------------------------------------------------------- adjoint

def _vec(g, p):
    return np.concatenate([g["cx"], g["cy"], g["theta"], g["length"], g["half_width"], g["logits"].ravel()])


@pytest.mark.parametrize("inert", [False, True])
def test_stored_state_adjoint_matches_finite_differences(inert):
    """Eq. adjstep / Eq. adjparam (stored-state form) against FP64 central
    differences of J = sum cot . R (the paper prints 2.5e-9 for its analytic
    VJP against central differences)."""
    p = _tiny_program(5, 41, r_lo=0.08, r_hi=0.2)
    W = H = 10
    tau, tau_min = 0.3, 0.02
    cot = inputs.make_cotangent(9, W * H).astype(np.float64)
    g = oracle.soft_vjp(p, W, H, tau, tau_min, cot, inert=inert)
    params = [(j, q) for j in range(p.n) for q in list(range(5)) + [5 + t for t in range(p.k)]]
    fd = oracle.fd_gradient(p, W, H, tau, tau_min, cot, params, h_geo=1e-6, h_logit=1e-6, inert=inert)
    got = np.array([g[oracle._FIELD[q]][j] if q < 5 else g["logits"][j, q - 5] for (j, q) in params])
    scale = np.abs(fd).max()
    assert np.abs(got - fd).max() < 1e-6 * scale


def test_far_stroke_keeps_the_adjoint_finite():
    """A stroke far off the canvas at the sharp relaxation (w = 1/200): its
    logit is about -720, where e^-z overflows FP64.  Its coverage is 0 to the
    precision of the arithmetic, and the adjoint (Eq. relax in its
    overflow-free form) must stay finite and match central differences: the
    far stroke still transports every pixel."""
    p = _tiny_program(5, 41, r_lo=0.08, r_hi=0.2)
    p.cx[2] = 3.0
    p.cy[2] = -2.0
    W = H = 10
    cot = inputs.make_cotangent(9, W * H).astype(np.float64)
    g = oracle.soft_vjp(p, W, H, 0.0, 1 / 200, cot)
    for k in ("cx", "cy", "theta", "length", "half_width", "logits"):
        assert np.isfinite(np.asarray(g[k])).all(), k
    params = [(j, q) for j in range(p.n) for q in range(5)]
    fd = oracle.fd_gradient(p, W, H, 0.0, 1 / 200, cot, params, h_geo=1e-6)
    got = np.array([g[oracle._FIELD[q]][j] for (j, q) in params])
    assert np.abs(got - fd).max() < 1e-5 * np.abs(fd).max()


def test_stored_state_adjoint_matches_forward_mode():
    """The reverse recurrence against exact forward-mode differentiation of the
    whole soft render (the paper prints 5.4e-15 against autograd)."""
    p = _tiny_program(6, 43, r_lo=0.06, r_hi=0.15)
    W = H = 8
    tau, tau_min = 0.25, 0.02
    cot = inputs.make_cotangent(13, W * H).astype(np.float64)
    g = oracle.soft_vjp(p, W, H, tau, tau_min, cot)
    for j in range(p.n):
        for q in range(5 + p.k):
            d = oracle.soft_jvp(p, W, H, tau, tau_min, j, q)
            want = float(np.sum(d * cot))
            got = g[oracle._FIELD[q]][j] if q < 5 else g["logits"][j, q - 5]
            assert abs(got - want) <= 1e-12 * (1 + abs(want))
    for q in range(p.k):
        for c in range(3):
            d = oracle.soft_jvp(p, W, H, tau, tau_min, 0, 5 + p.k + 3 * q + c)
            assert abs(g["palette"][q, c] - float(np.sum(d * cot))) < 1e-12


def test_zero_length_angle_gradient_vanishes():
    """A drop has no direction: d/d theta is zero at L = 0 (reading of the L = 0 kink)."""
    p = _tiny_program(6, 47)
    p.length[:] = 0.0
    cot = inputs.make_cotangent(5, 100).astype(np.float64)
    g = oracle.soft_vjp(p, 10, 10, 0.3, 0.02, cot)
    assert np.abs(g["theta"]).max() < 1e-13


def test_side_table_size_is_plausible():
    """Record count per pixel at 2000 strokes, sampled at 1024^2, against the
    paper's measured 9.9-14 records per pixel (a sanity band, not a bound)."""
    p = inputs.operating_program()
    pix = inputs.sample_pixels(3, 1024 * 1024, 1500)
    got = oracle.render_soft(p, 1024, 1024, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN, pix=pix)
    mean = got["nrec"].mean()
    lo, hi = SIDE["records_per_pixel_range"]
    assert lo / 4 < mean < hi * 4


# --------------------------------------------------------------------------- transfer renderer R_D

DSTROKE = (0.42, 0.57, 0.8, 0.15, 0.03)


def drop_sample(stroke, n=50_000, box=0.3, seed=11):
    """Points whose pull-back through the sixteen drops never enters a disc."""
    cx, cy = stroke[0], stroke[1]
    u = inputs.uniform(seed, 2 * n).reshape(-1, 2)
    pts = np.array([cx, cy]) + (2 * u - 1) * box
    out, binds = oracle.drops_map(pts, stroke, 0, return_binds=True)
    return pts[binds == 0], out[binds == 0]


@pytest.mark.parametrize("stroke", [(0.3, 0.6, 0.7, 0.0, 0.04), (0.5, 0.5, 2.0, 0.0, 0.01)])
def test_sixteen_drops_at_zero_length_are_one_drop(stroke):
    """At L = 0 the sixteen coincident drops of radius r/4 compose to the single
    drop of radius r, sigma = sqrt(rho^2 - r^2) along the ray (the classical drop
    map), which is also the capsule map at L = 0."""
    pts, out = drop_sample(stroke)
    c = np.array(stroke[:2])
    d = pts - c
    rho = np.hypot(*d.T)
    want = c + d * (np.sqrt(rho ** 2 - stroke[4] ** 2) / rho)[:, None]
    assert np.abs(out - want).max() < 1e-13
    assert np.abs(oracle.drops_map(pts, stroke, 1) - oracle.phi_map(pts, stroke)).max() < 1e-13


def test_sixteen_drops_round_trip_and_area():
    """Each drop map preserves area on its exterior: Phi_D inverts psi_D and
    det D psi_D = 1 wherever no disc is entered (Sec. "Transfer": each drop map
    preserves area on its exterior)."""
    pts, out = drop_sample(DSTROKE)
    assert np.abs(oracle.drops_map(out, DSTROKE, 1) - pts).max() < 1e-13
    _, _, J = oracle.drops_map(pts, DSTROKE, 0, return_binds=True, return_jacobian=True)
    # the determinant's rounding grows with the stretch near a disc boundary
    scale = 1.0 + (J ** 2).sum(axis=(1, 2))
    assert (np.abs(np.linalg.det(J) - 1.0) / scale).max() < 1e-13


def test_sixteen_drops_insert_the_stroke_area():
    """The drops have radius s = sqrt(A_L(r) / (16 pi)): Phi_D sends a circle of
    radius R around the stroke to a curve enclosing pi R^2 + A_L(r)."""
    cx, cy, th, L, r = DSTROKE
    R = 0.2

    def circle(n):
        t = np.arange(n) / n * 2 * math.pi
        return np.stack([cx + R * np.cos(t), cy + R * np.sin(t)], 1)

    area = _richardson_area(lambda n: oracle.drops_map(circle(n), DSTROKE, 1), 1 << 14)
    want = math.pi * R * R + steiner_area(L, r)
    assert abs(area - want) / want < 1e-9


def test_sixteen_drops_are_placed_symmetrically_and_swept_in_order():
    """The centres sit symmetrically about m along the segment, so reversing the
    sweep (theta + pi) is the mirror image across the perpendicular bisector;
    for L > 0 the order matters (the ordered drops do not commute), at L = 0 it
    does not; far from the stroke the sixteen drops act as one drop of the same
    area at m (the capsule's far field)."""
    rev = (DSTROKE[0], DSTROKE[1], DSTROKE[2] + math.pi, DSTROKE[3], DSTROKE[4])
    pts, out = drop_sample(DSTROKE)
    mirrored = reflect_bisector(oracle.drops_map(reflect_bisector(pts, DSTROKE), rev, 0), DSTROKE)
    assert np.abs(mirrored - out).max() < 1e-13
    assert np.abs(oracle.drops_map(pts, rev, 0) - out).max() > 1e-3
    z = (DSTROKE[0], DSTROKE[1], DSTROKE[2], 0.0, DSTROKE[4])
    zr = (z[0], z[1], z[2] + math.pi, 0.0, z[4])
    pz, oz = drop_sample(z)
    assert np.abs(oracle.drops_map(pz, zr, 0) - oz).max() < 1e-15
    far = np.array([[DSTROKE[0] + 30.0, DSTROKE[1] + 40.0], [DSTROKE[0] - 50.0, DSTROKE[1]]])
    one = (DSTROKE[0], DSTROKE[1], 0.0, 0.0, math.sqrt(steiner_area(DSTROKE[3], DSTROKE[4]) / math.pi))
    assert np.abs(oracle.drops_map(far, DSTROKE, 0) - oracle.psi_map(far, one, oracle.MODE_CLAMP)).max() < 1e-8


def test_drop_transport_renders_equal_the_capsule_renders_for_drops():
    """A program of drops only renders identically under R_D and R_A wherever
    no floor binds (the exterior transport is the same map at L = 0 and the
    coverage is the capsule's in both; inside a deposit the sixteen-drop
    operator floors once per drop, the capsule once per stroke)."""
    p = _tiny_program(14, 23)
    p.length[:] = 0.0
    W = H = 24
    a = oracle.render_soft(p, W, H, 0.1, 0.01)
    d = oracle.render_soft(p, W, H, 0.1, 0.01, transport="drops")
    clear = (a["nrec"] == 0) & (d["nrec"] == 0)
    assert clear.sum() > W * H // 4
    assert np.abs(a["rgb"] - d["rgb"])[clear].max() < 1e-12
    ha = oracle.render_hard(p, W, H)
    hd = oracle.render_hard(p, W, H, transport="drops")
    assert np.array_equal(ha["idx"], hd["idx"])
    q = _tiny_program(14, 23)
    assert np.abs(oracle.render_soft(q, W, H, 0.1, 0.01, transport="drops")["rgb"] - oracle.render_soft(q, W, H, 0.1, 0.01)["rgb"]).max() > 1e-3


# --------------------------------------------------------------------------- one-pass compensation

def _carry_forward(points, owner, comp, n):
    """Insert strokes 0..n-1 of the compensated program in order: a point that
    belongs to stroke i is moved by Phi_j (Eq. fwd) of every later stroke j."""
    pts = points.copy()
    for j in range(n):
        later = owner < j
        if later.any():
            st = (comp["cx"][j], comp["cy"][j], comp["theta"][j], comp["length"][j], comp["r"][j])
            pts[later] = oracle.phi_map(pts[later], st)
    return pts


def _ends(cx, cy, th, L):
    e = np.stack([np.cos(th), np.sin(th)], 1)
    m = np.stack([cx, cy], 1)
    return m - 0.5 * L[:, None] * e, m + 0.5 * L[:, None] * e


@pytest.mark.parametrize("endpoint", [False, True])
def test_compensation_round_trip(endpoint):
    """Sec. "Closed-form compensation baseline": where no step is blocked, the
    later strokes' forward maps carry each compensated stroke back to the given
    program's anchor (and end); the anchor variant keeps length and angle, and
    the last stroke is unchanged."""
    p = inputs.make_program(40, seed=5, palette_seed=6, k=4, r_lo=0.01, r_hi=0.05)
    o = oracle.compensate(p, endpoint=endpoint)
    o["r"] = p.half_width.astype(np.float64)
    n = p.n
    ok = o["blocked"] == 0
    assert ok.sum() > n // 2 and (~ok).sum() > 0
    a0, b0 = _ends(p.cx.astype(np.float64), p.cy.astype(np.float64), p.theta.astype(np.float64),
                   p.length.astype(np.float64))
    a1, b1 = _ends(o["cx"], o["cy"], o["theta"], o["length"])
    idx = np.arange(n)
    assert np.abs(_carry_forward(a1, idx, o, n)[ok] - a0[ok]).max() < 1e-11
    if endpoint:
        assert np.abs(_carry_forward(b1, idx, o, n)[ok] - b0[ok]).max() < 1e-11
    else:
        assert np.array_equal(o["length"], p.length.astype(np.float64))
        assert np.array_equal(o["theta"], p.theta.astype(np.float64))
    assert o["cx"][-1] == p.cx[-1] and o["cy"][-1] == p.cy[-1]


def test_compensation_blocked_step():
    """A point inside a later footprint has no pre-image (Lemma "obstruction"):
    the step is clamped onto the later segment (a drop's disc onto its centre)
    or skipped, and the stroke is counted as blocked."""
    def prog(cx, cy, th, L, r):
        n = len(cx)
        return inputs.Program(cx=np.array(cx), cy=np.array(cy), theta=np.array(th), length=np.array(L),
                              half_width=np.array(r), logits=np.zeros((n, 1)), palette=np.zeros((1, 3)),
                              background=np.ones(3), color_temp=1.0)
    p = prog([0.55, 0.5], [0.5, 0.5], [0.0, 0.0], [0.0, 0.0], [0.01, 0.2])
    c = oracle.compensate(p)
    assert list(c["blocked"]) == [1, 0]
    assert (c["cx"][0], c["cy"][0]) == (0.5, 0.5)
    s = oracle.compensate(p, skip_blocked=True)
    assert list(s["blocked"]) == [1, 0] and (s["cx"][0], s["cy"][0]) == (0.55, 0.5)
    q = prog([0.53, 0.5], [0.54, 0.5], [0.0, 0.4], [0.0, 0.3], [0.01, 0.08])
    c = oracle.compensate(q)
    assert c["blocked"][0] == 1
    seg = (0.5, 0.5, 0.4, 0.3, 0.08)
    assert seg_distance(np.array([[c["cx"][0], c["cy"][0]]]), seg)[0] < 1e-12


# --------------------------------------------------------------------------- coupling variant Phi_g

CPL_STROKE = (0.31, 0.62, 1.1, 0.13, 0.045)
CPL = (0.35, -0.1, 0.05)


def _leaf_points(stroke, sig, v):
    """Points of the leaf {sigma = sig} (sig may vary per point) at centred
    coordinate v: arclength v P + L/2 from the corner (-L/2, -sig), counter-
    clockwise (lower flank, right cap, upper flank, left cap)."""
    cx, cy, th, L, r = stroke
    sig = np.broadcast_to(np.asarray(sig, dtype=np.float64), np.shape(v))
    per = 2 * L + 2 * math.pi * sig
    a = np.mod(np.asarray(v) * per + 0.5 * L, per)
    s = np.empty_like(a)
    h = np.empty_like(a)
    for i in range(a.size):
        ai, si = a.flat[i], sig.flat[i]
        if ai < L:
            s.flat[i], h.flat[i] = -L / 2 + ai, -si
        elif ai < L + math.pi * si:
            ang = (ai - L) / si - math.pi / 2
            s.flat[i], h.flat[i] = L / 2 + si * math.cos(ang), si * math.sin(ang)
        elif ai < 2 * L + math.pi * si:
            s.flat[i], h.flat[i] = L / 2 - (ai - L - math.pi * si), si
        else:
            ang = (ai - 2 * L - math.pi * si) / si
            s.flat[i], h.flat[i] = -L / 2 - si * math.sin(ang), si * math.cos(ang)
    e = np.array([math.cos(th), math.sin(th)])
    en = np.array([-math.sin(th), math.cos(th)])
    return np.array([cx, cy]) + s.reshape(-1, 1) * e + h.reshape(-1, 1) * en


def _coupled_exterior(stroke, c, n=50_000):
    pts = exterior_sample(stroke, 4 * n)
    _, _, sb = oracle.coupled_map(pts, stroke, c, return_v=True)
    return pts[seg_distance(pts, stroke) > sb + 1e-9][:n]


@pytest.mark.parametrize("c", [(0.5, 0.0, 0.0), (0.0, 0.0, 0.3), (0.35, -0.1, 0.05), (0.2, 0.45, -0.3),
                               (-0.6, 0.3, 0.25)])
def test_coupling_profile_minimum_is_exact(c):
    """Positivity of g is decided exactly (Eq. profile: g is a cubic in
    w = cos 4 pi v): the closed-form minimum against dense sampling of
    1 + sum c_k cos(4 pi k v) over a quarter leaf, refined by golden section."""
    v = np.linspace(0.0, 0.25, 200_001)
    g = 1 + sum(ck * np.cos(4 * math.pi * (k + 1) * v) for k, ck in enumerate(c))
    i = int(np.argmin(g))
    lo, hi = v[max(i - 1, 0)], v[min(i + 1, v.size - 1)]
    f = lambda t: 1 + sum(ck * math.cos(4 * math.pi * (k + 1) * t) for k, ck in enumerate(c))
    for _ in range(200):
        m1, m2 = lo + (hi - lo) * 0.382, lo + (hi - lo) * 0.618
        if f(m1) < f(m2):
            hi = m2
        else:
            lo = m1
    sampled = min(g.min(), f(0.5 * (lo + hi)))
    assert abs(oracle.profile_min(c) - sampled) < 1e-12


@pytest.mark.parametrize("stroke", [CPL_STROKE, (0.5, 0.5, 0.4, 0.0, 0.03)])
def test_coupling_round_trip_and_unit_jacobian(stroke):
    """Phi_g o psi_g = id outside the deposit and psi_g o Phi_g = id off the
    segment; the Jacobian is unit triangular in the area chart, so det D psi_g
    = det D Phi_g = 1 (Eq. coupling)."""
    pts = _coupled_exterior(stroke, CPL)
    back = oracle.coupled_map(pts, stroke, CPL, direction=0)
    assert np.abs(oracle.coupled_map(back, stroke, CPL, direction=1) - pts).max() < 1e-13
    u = inputs.uniform(3, 2 * 20_000).reshape(-1, 2) - 0.5 + np.array(stroke[:2])
    fw = oracle.coupled_map(u, stroke, CPL, direction=1)
    assert np.abs(oracle.coupled_map(fw, stroke, CPL, direction=0) - u).max() < 1e-13
    for d, p in ((0, pts), (1, u)):
        _, J = oracle.coupled_map(p, stroke, CPL, direction=d, return_jacobian=True)
        det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
        assert np.abs(det - 1.0).max() < 1e-11
    # a profile that is not constant moves points differently from the capsule
    assert np.abs(back - oracle.psi_map(pts, stroke, oracle.MODE_CLAMP)).max() > 1e-4


def test_coupling_inserts_the_stroke_area():
    """g has unit mean over a leaf, so Phi_g sends the leaf {sigma = s0} to a
    curve enclosing A_L(s0) + A_L(r), as the capsule map does."""
    cx, cy, th, L, r = CPL_STROKE
    s0 = 0.02
    curve = lambda n: oracle.coupled_map(_leaf_points(CPL_STROKE, s0, np.arange(n) / n), CPL_STROKE, CPL,
                                         direction=1)
    area = _richardson_area(curve, 1 << 13)
    want = steiner_area(L, s0) + steiner_area(L, r)
    assert abs(area - want) / want < 1e-9


def test_coupling_reflection_symmetry():
    """The modes cos(4 pi k v) respect both mirror symmetries of the capsule
    (Eq. profile), so psi_g commutes with them."""
    pts = _coupled_exterior(CPL_STROKE, CPL)
    for refl in (reflect_bisector, reflect_line):
        a = oracle.coupled_map(refl(pts, CPL_STROKE), CPL_STROKE, CPL)
        b = refl(oracle.coupled_map(pts, CPL_STROKE, CPL), CPL_STROKE)
        assert np.abs(a - b).max() < 1e-13


def test_coupling_deposit_boundary():
    """The deposit is {u <= A_L(r) g(v)} with an explicit boundary: the leaf
    point at distance sigma_b(v), 2 L sigma_b + pi sigma_b^2 = A_L(r) g(v), has
    centred coordinate v and is carried by psi_g onto the segment; a positive
    first mode widens the flank (v = 0) and shortens the tips (v = 1/4)."""
    cx, cy, th, L, r = CPL_STROKE
    A = 2 * L * r + math.pi * r * r
    v = np.linspace(-0.5, 0.5, 801)[:-1]
    g = 1 + sum(ck * np.cos(4 * math.pi * (k + 1) * v) for k, ck in enumerate(CPL))
    sb = (-L + np.sqrt(L * L + math.pi * A * g)) / math.pi
    pts = _leaf_points(CPL_STROKE, sb, v)
    out, vo, sbo = oracle.coupled_map(pts, CPL_STROKE, CPL, direction=0, return_v=True)
    assert np.abs(np.mod(vo - v + 0.5, 1.0) - 0.5).max() < 1e-12
    assert np.abs(sbo - sb).max() < 1e-12
    assert seg_distance(out, CPL_STROKE).max() < 1e-9
    c1 = (0.3, 0.0, 0.0)
    _, _, s_flank = oracle.coupled_map(_leaf_points(CPL_STROKE, r, np.array([0.0])), CPL_STROKE, c1, return_v=True)
    _, _, s_tip = oracle.coupled_map(_leaf_points(CPL_STROKE, r, np.array([0.25])), CPL_STROKE, c1, return_v=True)
    assert s_flank[0] > r * 1.01 and s_tip[0] < r * 0.99
    for got, gval in ((s_flank[0], 1.3), (s_tip[0], 0.7)):
        assert abs(2 * L * got + math.pi * got * got - A * gval) < 1e-14


def test_zero_profile_is_the_capsule():
    """c = 0 is the capsule map: renders with an all-zero coupling array equal
    those without one bit for bit."""
    p = _tiny_program(12, 61, r_lo=0.03, r_hi=0.1)
    q = p.copy()
    q.coupling = np.zeros((p.n, 3))
    for fn in (lambda x: oracle.render_hard(x, 20, 20)["rgb"], lambda x: oracle.render_soft(x, 20, 20, 0.2, 0.01)["rgb"]):
        assert np.array_equal(fn(p), fn(q))


def test_coupled_single_stroke_hard_render_is_the_deposit():
    """One stroke under Eq. coupling: a pixel is coloured iff its distance to
    the segment is at most sigma_b(v) at its own v."""
    st = (0.45, 0.55, 0.6, 0.3, 0.12)
    c = (0.3, -0.1, 0.08)
    p = inputs.Program(cx=np.array([st[0]]), cy=np.array([st[1]]), theta=np.array([st[2]]),
                       length=np.array([st[3]]), half_width=np.array([st[4]]),
                       logits=np.zeros((1, 1)), palette=np.array([[0.2, 0.4, 0.6]]),
                       background=np.ones(3), color_temp=1.0, coupling=np.array([c]))
    W = H = 64
    got = oracle.render_hard(p, W, H)
    jj, ii = np.meshgrid(np.arange(W), np.arange(H))
    pts = np.stack([(jj.ravel() + 0.5) / W, (ii.ravel() + 0.5) / H], 1)
    _, _, sb = oracle.coupled_map(pts, st, c, return_v=True)
    inside = seg_distance(pts, st) <= sb
    assert np.array_equal(got["idx"] == 0, inside)
    assert inside.sum() != (seg_distance(pts, st) <= st[4]).sum()


def test_coupled_soft_render_tends_to_hard():
    """As the relaxation width goes to zero the coupled soft render tends to
    the coupled hard render away from deposit boundaries."""
    p = _tiny_program(10, 31, r_lo=0.03, r_hi=0.1)
    p.coupling = inputs.make_coupling(33, p.n)
    W = H = 24
    hard = oracle.render_hard(p, W, H)
    soft = oracle.render_soft(p, W, H, 0.0, 1e-5)["rgb"]
    far = hard["margin"] > 2e-2
    assert far.sum() > 0.5 * W * H
    assert np.abs(soft - hard["rgb"])[far].max() < 1e-6
    plain = p.copy()
    plain.coupling = None
    assert not np.array_equal(oracle.render_hard(plain, W, H)["idx"], hard["idx"])


def test_coupled_adjoint_matches_finite_differences():
    """The stored-state adjoint through psi_g and the coupled coverage against
    FP64 central differences."""
    p = _tiny_program(5, 41, r_lo=0.08, r_hi=0.2)
    p.coupling = inputs.make_coupling(43, p.n)
    W = H = 10
    tau, tau_min = 0.3, 0.02
    cot = inputs.make_cotangent(9, W * H).astype(np.float64)
    g = oracle.soft_vjp(p, W, H, tau, tau_min, cot)
    params = [(j, q) for j in range(p.n) for q in list(range(5)) + [5 + t for t in range(p.k)]]
    fd = oracle.fd_gradient(p, W, H, tau, tau_min, cot, params, h_geo=1e-6, h_logit=1e-6)
    got = np.array([g[oracle._FIELD[q]][j] if q < 5 else g["logits"][j, q - 5] for (j, q) in params])
    assert np.abs(got - fd).max() < 1e-6 * np.abs(fd).max()


def test_early_exit_changes_the_render_by_at_most_the_exit_transmittance():
    """Early exit of the forward render (stop once T < eps_T): the strokes it
    skips could add at most T < eps_T to each channel (colours and background
    in [0, 1]); pixels that never exit are unchanged."""
    p = inputs.make_program(400, seed=71, palette_seed=72, k=6, r_lo=0.03, r_hi=0.1)
    W = H = 40
    full = oracle.render_soft(p, W, H, 0.0, 1 / 200)
    for eps in (1e-3, 1e-6, 1e-12):
        ex = oracle.render_soft(p, W, H, 0.0, 1 / 200, early_exit=eps)
        d = np.abs(ex["rgb"] - full["rgb"]).max(1)
        exited = ex["T0"] < eps
        assert exited.sum() > 0.5 * W * H
        assert (d <= ex["T0"] + 1e-15).all()
        assert np.array_equal(ex["rgb"][~exited], full["rgb"][~exited])


# --------------------------------------------------------------------------- operation counts (measurement)

def test_operation_counts_by_hand():
    """The counting scalar against counts taken by hand from the definitions
    (FP32 add / subtract / multiply = 1, a division by a pixel value = 1 XU + 1,
    sqrt / atan2 / sin / cos = 1 XU, exp = 1 XU + 1).  One pixel at
    (0.4375, 0.4375) of an 8 x 8 canvas:
      * inside a capsule beside its flank: frame 8 (two differences, two dot
        products), distance 1 (the zero offset along the segment), margin 1;
      * inside a drop, on its cap: frame 8, distance 4 + 1 XU, margin 1;
      * outside a drop (right cap, passes on): the front 13 + 1 XU, then Eq.
        back 41 + 9 XU: C 5, the root 4 + 2 XU, the arclength 4 + 1 XU, the two
        perimeters 4, q 1 + 1 XU, v 3 + 1 XU, the new arclength 4 + 1 XU, the
        point on the stadium 8 + 3 XU, back to the canvas 8;
      * its soft step adds the coverage 3 + 2 XU and the compositing 11."""
    def one(strokes):
        a = np.asarray(strokes, float)
        n = a.shape[0]
        return inputs.Program(cx=a[:, 0], cy=a[:, 1], theta=a[:, 2], length=a[:, 3], half_width=a[:, 4],
                              logits=np.zeros((n, 1)), palette=np.array([[0.2, 0.4, 0.6]]),
                              background=np.ones(3), color_temp=1.0)
    pix = np.array([27])
    c = oracle.count_ops(one([(0.4375, 0.4375, 0.3, 0.2, 0.1)]), 8, 8, 0.0, 0.005, pix=pix)["hard"]
    assert (c["fp32"], c["xu"], c["visited_steps"]) == (10, 0, 1)
    c = oracle.count_ops(one([(0.30, 0.4375, 0.0, 0.0, 0.2)]), 8, 8, 0.0, 0.005, pix=pix)["hard"]
    assert (c["fp32"], c["xu"]) == (13, 1)
    c = oracle.count_ops(one([(0.20, 0.4375, 0.0, 0.0, 0.1)]), 8, 8, 0.0, 0.005, pix=pix)
    assert (c["hard"]["fp32"], c["hard"]["xu"]) == (54, 10)
    assert (c["soft"]["fp32"], c["soft"]["xu"]) == (68, 12)
    # the adjoint's regeneration is Eq. fwd on the pulled-back point, its coverage the front + Eq. relax
    parts = c["adjoint"]["parts"]
    assert (parts["coverage"]["fp32"], parts["coverage"]["xu"]) == (16, 3)
    # a reverse sweep costs a small multiple of the forward work it reverses
    fwd = 13 + 3 + 41
    assert 1.0 <= parts["reverse_sweep"]["fp32"] / fwd <= 4.0


@pytest.mark.slow
def test_frozen_operation_counts_are_reproducible():
    """The counts the benchmark divides by are what oracle/count_ops.py gives
    (integer tallies, so the sums are exact)."""
    path = os.path.join(os.path.dirname(GOLDEN), "..", "profiles", "opcount_1024_2000.json")
    frozen = json.load(open(path))
    pix = inputs.sample_pixels(4711, 1024 * 1024, frozen["pixels"])
    got = oracle.count_ops(inputs.operating_program(), 1024, 1024, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN, pix=pix)
    for part in ("soft", "adjoint"):
        key = "soft_forward" if part == "soft" else "adjoint"
        assert got[part]["fp32"] == frozen["capsule"][key]["fp32"]
        assert got[part]["xu"] == frozen["capsule"][key]["xu"]
    hard = oracle.count_ops(inputs.resolution_program(), 1024, 1024, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN,
                            pix=pix)["hard"]
    assert hard["fp32"] == frozen["capsule"]["hard_per_visited_step"]["fp32"]
