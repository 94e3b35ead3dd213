"""The replay adjoint at the operating point against FP64 finite differences.

Workload: the 2000-stroke program at 1024^2 (sharp relaxation w = 1/200), the
L2 data term of Sec. 5.1 against the hard render of a second seeded
2000-stroke program.  Twenty parameters are drawn (seed 401) uniformly over
{cx, cy, theta, L, r, 16 logits} x N, and twenty more over the strokes still
visible in the image.  The loss is restricted to a pixel
sample the oracle can afford (a uniform sample plus a strided patch over each
drawn stroke's footprint as it appears in the image), so the cotangent is
2 (R - I*) / (3 m) on those m pixels and zero elsewhere; both sides receive the
same float32 cotangent.  The GPU computes the whole image's replay adjoint with
that cotangent; the oracle differentiates its FP64 soft render of the sampled
pixels by central differences (Sec. 5.2's check of the analytic adjoint
against differences of rendered values).

Bound, per drawn parameter: |g_gpu - g_fd| <= 1e-3 * max(|g_fd|, 1e-3 * the
group's largest |g| from the oracle's stored-state adjoint on the same pixels),
or, for at most two of the twenty, within 4 x how far that gradient entry of the
oracle moves when every stroke parameter is perturbed by one FP32 rounding
(dense patches over visible strokes hold many pixels just outside a deposit,
whose pull-back stretch is unbounded, so a few entries are fixed by their FP32
inputs less tightly than 1e-3).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paritycheck import GRAD_TOL, SENS_FACTOR, oracle_sensitivity
from paper_2609_08722_b300 import inputs, tbr

pytestmark = pytest.mark.gpu

NAMES = ["cx", "cy", "theta", "length", "half_width"]


def drawn_parameters(seed, strokes, k, count=20):
    """(stroke, param) pairs uniform over {cx, cy, theta, L, r, k logits} x
    ``strokes``; param 0..4 is geometry, 5 + q is logit q."""
    u = inputs.uniform(seed, 2 * count).reshape(count, 2)
    n = len(strokes)
    return [(int(strokes[min(int(a * n), n - 1)]), min(int(b * (5 + k)), 4 + k)) for a, b in u]


def image_positions(p):
    """Where each stroke's centre appears in the image: the centre carried
    forward by every later stroke's map (Eq. fwd), [n, 2]."""
    x = np.stack([p.cx, p.cy], 1).astype(np.float64)
    for i in range(1, p.n):
        x[:i] = oracle.phi_map(x[:i], (float(p.cx[i]), float(p.cy[i]), float(p.theta[i]), float(p.length[i]),
                                       float(p.half_width[i])))
    return x


def footprint_pixels(p, j, centre, W, H, target=1600):
    """A strided patch over stroke j's footprint around its image position
    ``centre`` (about ``target`` pixels, stride <= 3 so the 1/200 coverage
    edge is sampled); empty when the stroke has left the canvas."""
    cx, cy = centre
    rad = float(p.half_width[j]) + 0.5 * float(p.length[j]) + 0.01
    half = int(math.ceil(rad * W))
    stride = max(1, min(3, int(math.ceil(2 * half / math.sqrt(target)))))
    c0, r0 = int(math.floor(cx * W)), int(math.floor(cy * H))
    cols = np.arange(max(0, c0 - half), min(W, c0 + half + 1), stride)
    rows = np.arange(max(0, r0 - half), min(H, r0 + half + 1), stride)
    rr, cc = np.meshgrid(rows, cols, indexing="ij")
    return (rr * W + cc).ravel()


@pytest.mark.parametrize("draw", ["all strokes", "on-canvas strokes"])
def test_operating_point_gradients_against_finite_differences(draw):
    """``all strokes``: the twenty parameters of seed 401 over the whole
    program.  Transport pushes most early strokes off the canvas (329 of the
    2000 centres stay on it), so most of those gradients are tiny and meet the
    floor.  ``on-canvas strokes``: twenty more (seed 403) over the strokes
    whose centre stays on the canvas, whose gradients are large."""
    p = inputs.operating_program()
    tgt = inputs.operating_target_program()
    W = H = 1024
    tau, tau_min = inputs.SHARP_TAU, inputs.SHARP_TAU_MIN
    pos = image_positions(p)
    if draw == "all strokes":
        params = drawn_parameters(401, np.arange(p.n), p.k)
    else:
        on = np.flatnonzero(((pos >= 0) & (pos < 1)).all(1))
        assert on.size > 100
        params = drawn_parameters(403, on, p.k)
    pix = [inputs.sample_pixels(402, W * H, 4096)]
    for j in sorted({j for j, _ in params}):
        pix.append(footprint_pixels(p, j, pos[j], W, H))
    pix = np.unique(np.concatenate(pix)).astype(np.int64)
    m = pix.size

    target = oracle.render_hard(tgt, W, H, pix=pix)["rgb"]
    R = oracle.render_soft(p, W, H, tau, tau_min, pix=pix)["rgb"]
    cot = (2.0 * (R - target) / (3.0 * m)).astype(np.float32)

    dp = tbr.DeviceProgram.from_host(p)
    _, ctx = tbr.render_soft(dp, W, H, tau, tau_min, record=True)
    full = torch.zeros((H * W, 3), device="cuda")
    full[torch.from_numpy(pix).cuda()] = torch.from_numpy(cot).cuda()
    g = ctx.backward(full.view(H, W, 3))
    assert ctx.status()["overflow_pixels"] == 0

    cot64 = cot.astype(np.float64)
    og = oracle.soft_vjp(p, W, H, tau, tau_min, cot64, pix=pix)
    sens = oracle_sensitivity(p, W, H, tau, tau_min, cot64, og, pix=pix)
    fd = oracle.fd_gradient(p, W, H, tau, tau_min, cot64, params, pix=pix)

    worst, by_sens = 0.0, 0
    for (j, q), want in zip(params, fd):
        grp = NAMES[q] if q < 5 else "logits"
        col = 0 if q < 5 else q - 5
        got = float(g[grp].cpu().numpy().reshape(p.n, -1)[j, col])
        adj = float(og[grp].reshape(p.n, -1)[j, col])
        s_j = float(sens["elem"][grp].reshape(p.n, -1)[j, col])
        floor = 1e-3 * float(np.abs(og[grp]).max())
        e = abs(got - want) / max(abs(want), floor)
        ok_sens = e > GRAD_TOL and abs(got - want) <= SENS_FACTOR * s_j
        print(f"stroke {j:4d} {grp:10s}{'' if q < 5 else f'[{col:2d}]'}: gpu {got:+.6e}  fd {want:+.6e}  "
              f"stored-state {adj:+.6e}  ratio {e:.2e}  (oracle sensitivity {s_j:.1e})"
              + ("  conditioning-limited" if ok_sens else ""))
        if ok_sens:
            by_sens += 1
        else:
            worst = max(worst, e)
            assert e <= GRAD_TOL, (j, q, got, want)
    print(f"{draw}: {m} pixels; worst GPU-vs-FD ratio {worst:.2e} over the parameters held to 1e-3; "
          f"{by_sens} of 20 within {SENS_FACTOR:g} x their sensitivity to one FP32 rounding of the inputs; "
          f"oracle norm sensitivity " + ", ".join(f"{k} {v:.1e}" for k, v in sens["norm"].items()))
    assert by_sens <= 2
