"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances:
  * hard render: terminating stroke index bit-exact except pixels whose oracle
    margin min_j |sigma'_j - r_j| < 1e-5 (counted); a mismatch outside that band
    is accepted only where the oracle's chain condition kappa makes an FP32
    trajectory uncertain beyond 1e-5 (kappa * 6e-8 > 1e-5), and is reported;
  * soft render: |R_gpu - R_oracle| <= 1e-4 per channel;
  * gradients: per parameter group ||g_gpu - g_oracle|| / ||g_oracle|| <= 1e-3,
    and per element |g - g_oracle| / max(|g_oracle|, 1e-3 max|g_oracle|) <= 1e-3,
    or within 4 x the element's own sensitivity to one FP32 rounding of the
    inputs (``paritycheck.compare``).
"""
import numpy as np
import pytest
import torch

import oracle
from paritycheck import check_hard, compare, oracle_sensitivity
from paper_2609_08722_b300 import inputs, tbr

pytestmark = pytest.mark.gpu

SOFT_TOL = 1e-4
GRAD_TOL = 1e-3
BAND = 1e-5
GROUPS = ["cx", "cy", "theta", "length", "half_width", "logits", "palette"]


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def small():
    p = inputs.small_program()
    return p, tbr.DeviceProgram.from_host(p)


def test_hard_small_program(small):
    p, dp = small
    W = H = 128
    rgb, idx, st = tbr.render_hard(dp, W, H, stats=True)
    o = oracle.render_hard(p, W, H, with_kappa=True)
    check_hard(p, idx.cpu().numpy(), o, W, H, f"hard 128^2, stats {st}")
    ok = idx.cpu().numpy().ravel() == o["idx"]
    assert np.abs(rgb.cpu().numpy().reshape(-1, 3)[ok] - o["rgb"][ok]).max() < 1e-6


@pytest.mark.parametrize("W,H,n", [(77, 45, 50), (33, 9, 1), (40, 40, 0), (1, 1, 50)])
def test_hard_ragged_sizes(small, W, H, n):
    p, _ = small
    q = p.prefix(n)
    if n == 0:
        q = p.prefix(0)
    dq = tbr.DeviceProgram.from_host(q)
    rgb, idx, _ = tbr.render_hard(dq, W, H)
    o = oracle.render_hard(q, W, H, with_kappa=True)
    check_hard(q, idx.cpu().numpy(), o, W, H, f"hard {W}x{H} n={n}")
    if n == 0:
        assert (idx.cpu().numpy() == -1).all()
        assert np.allclose(rgb.cpu().numpy(), 1.0)


def test_hard_prefix_and_snap(small):
    p, dp = small
    W = H = 64
    for m in (0, 1, 17, 50):
        _, idx, _ = tbr.render_hard(dp, W, H, n_prefix=m)
        o = oracle.render_hard(p, W, H, n_prefix=m, with_kappa=True)
        check_hard(p, idx.cpu().numpy(), o, W, H, f"prefix {m}", n_prefix=m)
        assert idx.max().item() < max(m, 0) or m == 0
    rgb, idx, _ = tbr.render_hard(dp, W, H, snap=True)
    o = oracle.render_hard(p, W, H, snap=True)
    ok = idx.cpu().numpy().ravel() == o["idx"]
    assert np.array_equal(rgb.cpu().numpy().reshape(-1, 3)[ok], o["rgb"][ok].astype(np.float32))


def test_recolour_edit_keeps_the_index_map(small):
    """Transport ignores pigment, so a recolour edit changes no terminating index (Sec. 7 edits)."""
    p, dp = small
    _, idx0, _ = tbr.render_hard(dp, 96, 96)
    q = p.copy()
    q.logits = np.ascontiguousarray(q.logits[:, ::-1])
    _, idx1, _ = tbr.render_hard(tbr.DeviceProgram.from_host(q), 96, 96)
    assert torch.equal(idx0, idx1)


@pytest.mark.parametrize("res", [512, 1024, 2048, 4096])
def test_hard_resolution_replay(res):
    """One 2000-stroke program replayed at 512^2 .. 4096^2; sampled pixels vs the oracle."""
    p = inputs.resolution_program()
    dp = tbr.DeviceProgram.from_host(p)
    rgb, idx, st = tbr.render_hard(dp, res, res, stats=True)
    pix = inputs.sample_pixels(res, res * res, 4000)
    o = oracle.render_hard(p, res, res, pix=pix, with_kappa=True)
    c = check_hard(p, idx.cpu().numpy().ravel()[pix], o, res, res, f"{res}^2 (fp64 steps {st['band_steps']})",
                   pix=pix)
    assert c["mismatch"] < 0.01 * pix.size


@pytest.mark.parametrize("tau,tau_min", [(0.0, 1 / 200), (0.3, 0.01)])
def test_soft_small_program(small, tau, tau_min):
    p, dp = small
    W = H = 128
    rgb, _ = tbr.render_soft(dp, W, H, tau, tau_min)
    o = oracle.render_soft(p, W, H, tau, tau_min)
    err = np.abs(rgb.cpu().numpy().reshape(-1, 3) - o["rgb"])
    print(f"soft max {err.max():.3e} mean {err.mean():.3e}")
    assert err.max() <= SOFT_TOL


@pytest.mark.parametrize("W,H", [(77, 45), (1, 1), (33, 9)])
def test_soft_ragged(small, W, H):
    p, dp = small
    rgb, ctx = tbr.render_soft(dp, W, H, 0.0, 1 / 200, record=True)
    o = oracle.render_soft(p, W, H, 0.0, 1 / 200)
    assert np.abs(rgb.cpu().numpy().reshape(-1, 3) - o["rgb"]).max() <= SOFT_TOL
    cot = inputs.make_cotangent(21, W * H)
    g = ctx.backward(torch.from_numpy(cot).reshape(H, W, 3).cuda())
    og = oracle.soft_vjp(p, W, H, 0.0, 1 / 200, cot.astype(np.float64))
    sens = oracle_sensitivity(p, W, H, 0.0, 1 / 200, cot.astype(np.float64), og)
    compare(g, og, sens=sens, label=f"ragged {W}x{H}")


@pytest.mark.parametrize("n", [0, 1])
def test_soft_and_adjoint_of_empty_and_single_stroke_programs(small, n):
    """No strokes: the soft render is the background, the stroke gradients are
    empty and the palette's is zero, through the recording render with its
    adjoint and through the loss-fused call.  One stroke: both against the
    oracle (a single chunk holding one stroke, no checkpoint)."""
    p, _ = small
    q = p.prefix(n)
    dq = tbr.DeviceProgram.from_host(q)
    W, H = 37, 21
    rgb, ctx = tbr.render_soft(dq, W, H, 0.0, 1 / 200, record=True)
    o = oracle.render_soft(q, W, H, 0.0, 1 / 200)
    assert np.abs(rgb.cpu().numpy().reshape(-1, 3) - o["rgb"]).max() <= (1e-7 if n == 0 else SOFT_TOL)
    cot = inputs.make_cotangent(22, W * H)
    g = ctx.backward(torch.from_numpy(cot).reshape(H, W, 3).cuda())
    og = oracle.soft_vjp(q, W, H, 0.0, 1 / 200, cot.astype(np.float64))
    target = torch.from_numpy(inputs.make_cotangent(23, W * H)).reshape(H, W, 3).cuda()
    loss, gf, _, _ = tbr.soft_adjoint_mse(dq, target, 0.0, 1 / 200)
    if n == 0:
        for k in GROUPS[:-1]:
            assert g[k].numel() == 0 and gf[k].numel() == 0
        assert torch.count_nonzero(g["palette"]).item() == 0 and torch.count_nonzero(gf["palette"]).item() == 0
        bg = torch.tensor(np.asarray(q.background, dtype=np.float32), device="cuda")
        want = float(((bg.double() - target.double()) ** 2).mean())
        assert abs(float(loss.item()) - want) <= 1e-6 * max(1.0, want)
    else:
        sens = oracle_sensitivity(q, W, H, 0.0, 1 / 200, cot.astype(np.float64), og)
        compare(g, og, sens=sens, label="one stroke")
        for k in GROUPS:
            assert torch.isfinite(gf[k]).all()


@pytest.mark.parametrize("W,H,ck,trials", [(58, 46, 32, 3), (58, 46, 48, 3), (29, 23, 64, 20)])
def test_soft_and_adjoint_of_a_long_program(W, H, ck, trials):
    """10000 strokes (five times the operating program) on ragged canvases:
    313 chunks through the stroke ring, up to 312 checkpoints (48 is not a
    multiple of the renormalisation block, so the stroke loops take their
    per-stroke checkpoint test), up to 27 side-table records per pixel.
    On the 29x23 canvas most strokes are smaller than a pixel, so one edge
    sample sets each of their entries; entries near the floor of the relative
    bound then move by up to 3e-3 of themselves under one FP32 rounding of the
    inputs, and three perturbation trials underestimate that move by about
    half, so that case samples twenty."""
    p = inputs.make_program(10000, seed=131, palette_seed=231, k=16, r_lo=0.003, r_hi=0.03)
    dp = tbr.DeviceProgram.from_host(p)
    rgb, ctx = tbr.render_soft(dp, W, H, 0.0, 1 / 200, record=True, checkpoint_every=ck)
    o = oracle.render_soft(p, W, H, 0.0, 1 / 200)
    err = np.abs(rgb.cpu().numpy().reshape(-1, 3) - o["rgb"])
    print(f"long program soft max {err.max():.3e}")
    assert err.max() <= SOFT_TOL
    st = ctx.status()
    recs = o["nrec"].mean()
    print(f"records/px gpu {st['records'] / (W * H):.2f} oracle {recs:.2f}, max {st['max_records']} / {o['nrec'].max()}")
    assert abs(st["records"] / (W * H) - recs) < 0.05 * recs + 0.5
    cot = inputs.make_cotangent(24, W * H)
    g = ctx.backward(torch.from_numpy(cot).reshape(H, W, 3).cuda())
    og = oracle.soft_vjp(p, W, H, 0.0, 1 / 200, cot.astype(np.float64))
    sens = oracle_sensitivity(p, W, H, 0.0, 1 / 200, cot.astype(np.float64), og, trials=trials)
    compare(g, og, sens=sens, label=f"10000 strokes, {W}x{H}, k = {ck}")


@pytest.mark.parametrize("R,n", [(4096, 500), (8192, 100)])
def test_soft_and_adjoint_at_the_largest_sizes(R, n):
    """16.7M and 67.1M pixels: the side table, checkpoints and slices hold up to
    1.1e9 elements (24 GB at 8192^2), so every pixel-indexed offset must be
    formed in 64 bits.  Soft colours and the adjoint (cotangent on 2048
    sampled pixels) against the oracle on those pixels."""
    p = inputs.make_program(n, seed=141, palette_seed=241, k=16, r_lo=0.003, r_hi=0.05)
    dp = tbr.DeviceProgram.from_host(p)
    rgb, ctx = tbr.render_soft(dp, R, R, 0.0, 1 / 200, record=True, record_capacity=16)
    pix = inputs.sample_pixels(43, R * R, 2048)
    o = oracle.render_soft(p, R, R, 0.0, 1 / 200, pix=pix)
    err = np.abs(rgb.view(-1, 3)[torch.from_numpy(pix).cuda()].cpu().numpy() - o["rgb"])
    print(f"{R}^2 soft max {err.max():.3e}")
    assert err.max() <= SOFT_TOL
    del rgb
    cot = inputs.make_cotangent(44, pix.size)
    full = torch.zeros((R * R, 3), device="cuda")
    full[torch.from_numpy(pix).cuda()] = torch.from_numpy(cot).cuda()
    g = ctx.backward(full.view(R, R, 3))
    assert ctx.status()["overflow_pixels"] == 0
    og = oracle.soft_vjp(p, R, R, 0.0, 1 / 200, cot.astype(np.float64), pix=pix)
    sens = oracle_sensitivity(p, R, R, 0.0, 1 / 200, cot.astype(np.float64), og, pix=pix)
    compare(g, og, sens=sens, label=f"{R}^2, {n} strokes (2048 sampled pixels)")
    ctx.destroy()


@pytest.mark.parametrize("k", [64, 256])
def test_large_palettes(k):
    """Palettes of 64 and 256 colours: the softmax colour of the pack, the
    logits chain rule of the epilogue (sum over the palette per stroke) and the
    palette gradient, against the oracle."""
    p = inputs.make_program(80, seed=151, palette_seed=251, k=k, r_lo=0.01, r_hi=0.08)
    dp = tbr.DeviceProgram.from_host(p)
    W, H = 70, 45
    rgb, ctx = tbr.render_soft(dp, W, H, 0.0, 1 / 200, record=True)
    o = oracle.render_soft(p, W, H, 0.0, 1 / 200)
    assert np.abs(rgb.cpu().numpy().reshape(-1, 3) - o["rgb"]).max() <= SOFT_TOL
    cot = inputs.make_cotangent(45, W * H)
    g = ctx.backward(torch.from_numpy(cot).reshape(H, W, 3).cuda())
    og = oracle.soft_vjp(p, W, H, 0.0, 1 / 200, cot.astype(np.float64))
    sens = oracle_sensitivity(p, W, H, 0.0, 1 / 200, cot.astype(np.float64), og)
    compare(g, og, sens=sens, label=f"palette of {k}")


def extreme_program():
    """60 strokes, with: one swallowing a third of the canvas (r = 0.3, L =
    0.4), one thinner than a pixel (r = 1e-4), one centred far off the canvas
    at (3, -2) (logits near -720 at the sharp relaxation), one longer than the
    canvas (L = 2), angles of +-37 rad, and one centred on a corner."""
    p = inputs.make_program(60, seed=161, palette_seed=261, k=8, r_lo=0.01, r_hi=0.06)
    p.half_width[5] = 0.3
    p.length[5] = 0.4
    p.half_width[12] = 1e-4
    p.length[12] = 0.05
    p.cx[20] = 3.0
    p.cy[20] = -2.0
    p.length[25] = 2.0
    p.half_width[25] = 0.02
    p.theta[30] = 37.0
    p.theta[31] = -37.0
    p.cx[50] = 0.0
    p.cy[50] = 0.0
    return p


@pytest.mark.parametrize("tau,tau_min", [(0.0, 1 / 200), (0.3, 1 / 50)])
def test_extreme_geometry(tau, tau_min):
    p = extreme_program()
    dp = tbr.DeviceProgram.from_host(p)
    W, H = 96, 80
    _, idx, _ = tbr.render_hard(dp, W, H)
    check_hard(p, idx.cpu().numpy(), oracle.render_hard(p, W, H, with_kappa=True), W, H, "extreme hard")
    rgb, ctx = tbr.render_soft(dp, W, H, tau, tau_min, record=True)
    o = oracle.render_soft(p, W, H, tau, tau_min)
    assert np.abs(rgb.cpu().numpy().reshape(-1, 3) - o["rgb"]).max() <= SOFT_TOL
    cot = inputs.make_cotangent(46, W * H)
    g = ctx.backward(torch.from_numpy(cot).reshape(H, W, 3).cuda())
    og = oracle.soft_vjp(p, W, H, tau, tau_min, cot.astype(np.float64))
    sens = oracle_sensitivity(p, W, H, tau, tau_min, cot.astype(np.float64), og)
    compare(g, og, sens=sens, label=f"extreme geometry tau={tau}")


@pytest.mark.parametrize("tau,tau_min", [(0.0, 1 / 200), (0.3, 1 / 50)])
def test_extreme_geometry_transfer_and_coupling(tau, tau_min):
    """The same extreme program through the transfer renderer R_D (hard and
    soft) and under the coupling variant Phi_g (hard, soft and adjoint; its
    entries keep the coupled tests' 20% share by the sensitivity allowance)."""
    W, H = 96, 80
    p = extreme_program()
    dp = tbr.DeviceProgram.from_host(p)
    _, idx, _ = tbr.render_hard(dp, W, H, transport="drops")
    check_hard(p, idx.cpu().numpy(), oracle.render_hard(p, W, H, with_kappa=True, transport="drops"), W, H,
               "extreme R_D hard", transport="drops")
    rgb, _ = tbr.render_soft(dp, W, H, tau, tau_min, transport="drops")
    o = oracle.render_soft(p, W, H, tau, tau_min, transport="drops")
    assert np.abs(rgb.cpu().numpy().reshape(-1, 3) - o["rgb"]).max() <= SOFT_TOL
    q = extreme_program()
    q.coupling = inputs.make_coupling(403, q.n)
    dq = tbr.DeviceProgram.from_host(q)
    _, idx, _ = tbr.render_hard(dq, W, H)
    check_hard(q, idx.cpu().numpy(), oracle.render_hard(q, W, H, with_kappa=True), W, H, "extreme Phi_g hard")
    rgb, ctx = tbr.render_soft(dq, W, H, tau, tau_min, record=True)
    o = oracle.render_soft(q, W, H, tau, tau_min)
    assert np.abs(rgb.cpu().numpy().reshape(-1, 3) - o["rgb"]).max() <= SOFT_TOL
    cot = inputs.make_cotangent(48, W * H)
    g = ctx.backward(torch.from_numpy(cot).reshape(H, W, 3).cuda())
    og = oracle.soft_vjp(q, W, H, tau, tau_min, cot.astype(np.float64))
    sens = oracle_sensitivity(q, W, H, tau, tau_min, cot.astype(np.float64), og)
    compare(g, og, sens=sens, label=f"extreme Phi_g tau={tau}", max_cond_frac=0.2)


@pytest.mark.parametrize("color_temp,background,palette_shift", [
    (0.05, (0.0, 0.0, 0.0), 0.0),     # the end of the fit's schedule: nearly one-hot colours, black ground
    (20.0, (0.2, 0.5, 0.9), 0.0),     # nearly uniform mixtures on a coloured ground
    (1.0, (1.0, 1.0, 1.0), 0.7),      # palette values above 1 and below 0 (no clamp in the method)
])
def test_colour_extremes(color_temp, background, palette_shift):
    """The colour chain of Eq. state and the softmax colours under extreme
    temperatures, backgrounds and palettes: the soft render, the adjoint's
    colour and transmittance terms, and the logits and palette gradients."""
    p = inputs.make_program(60, seed=171, palette_seed=271, k=8, r_lo=0.01, r_hi=0.08)
    p.color_temp = color_temp
    p.background = np.asarray(background, dtype=np.float32)
    if palette_shift:
        p.palette = (p.palette * 2.0 - palette_shift).astype(np.float32)
    dp = tbr.DeviceProgram.from_host(p)
    W, H = 80, 60
    rgb, ctx = tbr.render_soft(dp, W, H, 0.0, 1 / 200, record=True)
    o = oracle.render_soft(p, W, H, 0.0, 1 / 200)
    assert np.abs(rgb.cpu().numpy().reshape(-1, 3) - o["rgb"]).max() <= SOFT_TOL
    cot = inputs.make_cotangent(47, W * H)
    g = ctx.backward(torch.from_numpy(cot).reshape(H, W, 3).cuda())
    og = oracle.soft_vjp(p, W, H, 0.0, 1 / 200, cot.astype(np.float64))
    sens = oracle_sensitivity(p, W, H, 0.0, 1 / 200, cot.astype(np.float64), og)
    compare(g, og, sens=sens, label=f"colours tau_c={color_temp} bg={background} shift={palette_shift}")


@pytest.mark.parametrize("W,H", [(75, 61), (64, 33)])
def test_backward_long_strokes(W, H):
    """No drops and strokes up to 0.8 long: most samples sit beside a flank,
    and many steps cross from a flank onto a cap (the paired kernel's
    per-pixel fallback)."""
    p = inputs.make_program(120, seed=311, palette_seed=312, k=8, r_lo=0.004, r_hi=0.04, len_max=0.8, p_drop=0.0)
    dp = tbr.DeviceProgram.from_host(p)
    rgb, ctx = tbr.render_soft(dp, W, H, 0.0, 1 / 200, record=True)
    o = oracle.render_soft(p, W, H, 0.0, 1 / 200)
    assert np.abs(rgb.cpu().numpy().reshape(-1, 3) - o["rgb"]).max() <= SOFT_TOL
    cot = inputs.make_cotangent(313, W * H)
    g = ctx.backward(torch.from_numpy(cot).reshape(H, W, 3).cuda())
    og = oracle.soft_vjp(p, W, H, 0.0, 1 / 200, cot.astype(np.float64))
    sens = oracle_sensitivity(p, W, H, 0.0, 1 / 200, cot.astype(np.float64), og)
    compare(g, og, sens=sens, label=f"long strokes {W}x{H}")


@pytest.mark.parametrize("tau,tau_min,inert", [(0.0, 1 / 200, False), (0.3, 0.01, False),
                                               (0.3, 0.01, True)])
def test_backward_small_program(small, tau, tau_min, inert):
    p, dp = small
    W = H = 128
    rgb, ctx = tbr.render_soft(dp, W, H, tau, tau_min, record=True, inert=inert)
    cot = inputs.make_cotangent(5, W * H)
    g = ctx.backward(torch.from_numpy(cot).reshape(H, W, 3).cuda())
    st = ctx.status()
    og = oracle.soft_vjp(p, W, H, tau, tau_min, cot.astype(np.float64), inert=inert)
    sens = oracle_sensitivity(p, W, H, tau, tau_min, cot.astype(np.float64), og, inert=inert)
    compare(g, og, sens=sens, label=f"small tau={tau} inert={inert}")
    assert st["overflow_pixels"] == 0


def test_backward_is_reproducible(small):
    p, dp = small
    _, ctx = tbr.render_soft(dp, 96, 96, 0.0, 1 / 200, record=True)
    cot = torch.from_numpy(inputs.make_cotangent(7, 96 * 96)).reshape(96, 96, 3).cuda()
    a = ctx.backward(cot)
    b = ctx.backward(cot)
    for k in GROUPS:
        assert torch.equal(a[k], b[k])


@pytest.mark.parametrize("k", [8, 32, 1000])
def test_checkpoint_interval_does_not_change_gradients(small, k):
    p, dp = small
    W = H = 64
    cot = inputs.make_cotangent(8, W * H)
    _, ctx = tbr.render_soft(dp, W, H, 0.0, 1 / 200, record=True, checkpoint_every=k)
    g = ctx.backward(torch.from_numpy(cot).reshape(H, W, 3).cuda())
    og = oracle.soft_vjp(p, W, H, 0.0, 1 / 200, cot.astype(np.float64))
    sens = oracle_sensitivity(p, W, H, 0.0, 1 / 200, cot.astype(np.float64), og)
    compare(g, og, sens=sens, label=f"checkpoint every {k}")


def test_fp64_repair_of_drifting_segments(small):
    """A drift tolerance of 1e-12 marks (nearly) every pixel at its first
    checkpoint: the adjoint regenerates those segments in FP64 and replaces the
    pixels' contributions.  The result stays within the oracle tolerance, is
    reproducible, and differs from the unrepaired gradients only by rounding
    (which also checks that the repair's replay of each pixel pair reproduces
    the main adjoint exactly before it substitutes the FP64 trajectory)."""
    p, dp = small
    W, H = 40, 24
    cot = torch.from_numpy(inputs.make_cotangent(17, W * H)).reshape(H, W, 3).cuda()
    _, ctx0 = tbr.render_soft(dp, W, H, 0.0, 1 / 200, record=True, checkpoint_every=8)
    g0 = ctx0.backward(cot)
    s0 = ctx0.status()
    assert s0["repaired_pixels"] == 0 and s0["drift_resets"] == 0
    _, ctx = tbr.render_soft(dp, W, H, 0.0, 1 / 200, record=True, checkpoint_every=8, drift_tolerance=1e-12,
                             repair_capacity=1024)
    g1 = ctx.backward(cot)
    st = ctx.status()
    g2 = ctx.backward(cot)
    print(f"repair stats {st}")
    assert st["repaired_pixels"] > W * H // 2 and st["repair_overflow"] == 0
    cot64 = cot.double().cpu().numpy().reshape(-1, 3)
    og = oracle.soft_vjp(p, W, H, 0.0, 1 / 200, cot64)
    compare(g1, og, sens=oracle_sensitivity(p, W, H, 0.0, 1 / 200, cot64, og), label="FP64-repaired")
    for k in GROUPS:
        assert torch.equal(g1[k], g2[k]), k
        e_mix = rel(g1[k].cpu().numpy().ravel(), g0[k].cpu().numpy().ravel())
        print(f"{k}: vs unrepaired {e_mix:.2e}")
        assert e_mix <= 1e-4, k


def test_fp64_repair_overflow_is_reported_and_skipped(small):
    """More drifting pixels than the repair capacity: none is repaired (so the
    result stays deterministic), the count is reported, and the gradients are
    those of the unrepaired adjoint."""
    p, dp = small
    W, H = 40, 24
    cot = torch.from_numpy(inputs.make_cotangent(18, W * H)).reshape(H, W, 3).cuda()
    _, ctx0 = tbr.render_soft(dp, W, H, 0.0, 1 / 200, record=True, checkpoint_every=8, repair_capacity=1)
    g0 = ctx0.backward(cot)
    _, ctx = tbr.render_soft(dp, W, H, 0.0, 1 / 200, record=True, checkpoint_every=8, drift_tolerance=1e-12,
                             repair_capacity=1)
    g1 = ctx.backward(cot)
    st = ctx.status()
    assert st["repair_overflow"] > 1 and st["repaired_pixels"] == 0
    for k in GROUPS:
        assert torch.equal(g0[k], g1[k]), k


@pytest.fixture(scope="module")
def operating():
    p = inputs.operating_program()
    return p, tbr.DeviceProgram.from_host(p)


def test_soft_operating_point_sampled(operating):
    """2000 strokes at 1024^2 in the launch configuration the benchmark times."""
    p, dp = operating
    W = H = 1024
    rgb, ctx = tbr.render_soft(dp, W, H, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN, record=True)
    pix = inputs.sample_pixels(31, W * H, 3000)
    o = oracle.render_soft(p, W, H, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN, pix=pix)
    err = np.abs(rgb.cpu().numpy().reshape(-1, 3)[pix] - o["rgb"])
    print(f"soft op max {err.max():.3e} mean {err.mean():.3e}")
    assert err.max() <= SOFT_TOL
    st = ctx.status()
    recs = o["nrec"].mean()
    print(f"records/px gpu {st['records'] / (W * H):.2f} oracle(sampled) {recs:.2f}, max {st['max_records']}")
    assert abs(st["records"] / (W * H) - recs) < 0.25 * recs + 0.5


def test_backward_operating_point_sampled(operating):
    """Full-size replay adjoint with the cotangent supported on sampled pixels,
    against the oracle's stored-state adjoint on those pixels."""
    p, dp = operating
    W = H = 1024
    _, ctx = tbr.render_soft(dp, W, H, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN, record=True)
    pix = inputs.sample_pixels(41, W * H, 2048)
    cot = inputs.make_cotangent(42, pix.size)
    full = torch.zeros((H * W, 3), device="cuda")
    full[torch.from_numpy(pix).cuda()] = torch.from_numpy(cot).cuda()
    g = ctx.backward(full.view(H, W, 3))
    og = oracle.soft_vjp(p, W, H, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN, cot.astype(np.float64), pix=pix)
    sens = oracle_sensitivity(p, W, H, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN, cot.astype(np.float64), og, pix=pix)
    compare(g, og, sens=sens, label="operating point (2048 sampled pixels)")


def test_loss_mse_matches_numpy():
    rng = np.random.default_rng(0)
    a = rng.random((37, 53, 3), dtype=np.float32)
    b = rng.random((37, 53, 3), dtype=np.float32)
    loss, d = tbr.loss_mse(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
    want = np.mean((a.astype(np.float64) - b) ** 2)
    assert abs(loss.item() - want) < 1e-6 * want
    assert np.allclose(d.cpu().numpy(), 2 * (a - b) / a.size, rtol=1e-6, atol=1e-12)


def test_invalid_stroke_values_are_reported(small):
    p, _ = small
    q = p.copy()
    q.half_width[3] = -0.01
    dq = tbr.DeviceProgram.from_host(q)
    with pytest.raises(tbr.TbrError) as ei:
        tbr.render_hard(dq, 32, 32, stats=True)
    assert ei.value.status == tbr.TBR_ERR_INVALID_ARG
    rgb, ctx = tbr.render_soft(dq, 32, 32, 0.0, 1 / 200, record=True)
    assert torch.isnan(rgb).all()
    with pytest.raises(tbr.TbrError):
        ctx.status()


def test_side_table_overflow_is_reported(operating):
    p, dp = operating
    _, ctx = tbr.render_soft(dp, 256, 256, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN, record=True,
                             record_capacity=2)
    g = ctx.backward(torch.ones((256, 256, 3), device="cuda"))
    st = ctx.status(raise_on_error=False)
    assert st["status"] == tbr.TBR_ERR_OVERFLOW and st["overflow_pixels"] > 0
    assert torch.isnan(g["cx"]).all()


@pytest.mark.parametrize("W,H", [(128, 128), (77, 45)])
def test_fused_mse_adjoint_matches_split_path_and_oracle(small, W, H):
    """The loss-fused forward + adjoint equals render_soft + loss_mse +
    render_backward, and the oracle's stored-state adjoint of the same seed."""
    p, dp = small
    tgt_h = inputs.make_program(50, seed=7001, palette_seed=201, k=8, r_lo=0.01, r_hi=0.08)
    target, _, _ = tbr.render_hard(tbr.DeviceProgram.from_host(tgt_h), W, H)
    loss_f, g_f, rgb_f, st = tbr.soft_adjoint_mse(dp, target, 0.0, 1 / 200, want_rgb=True, stats=True)
    rgb, ctx = tbr.render_soft(dp, W, H, 0.0, 1 / 200, record=True)
    loss_s, dL = tbr.loss_mse(rgb, target)
    g_s = ctx.backward(dL)
    assert torch.equal(rgb_f, rgb)
    assert abs(loss_f.item() - loss_s.item()) <= 1e-6 * abs(loss_s.item())
    for k in GROUPS:
        assert rel(g_f[k].cpu().numpy().ravel(), g_s[k].cpu().numpy().ravel()) <= 1e-4, k
    cot = dL.cpu().numpy().reshape(-1, 3).astype(np.float64)
    og = oracle.soft_vjp(p, W, H, 0.0, 1 / 200, cot)
    compare(g_f, og, sens=oracle_sensitivity(p, W, H, 0.0, 1 / 200, cot, og), label=f"loss-fused {W}x{H}")
    assert st["overflow_pixels"] == 0


def test_fused_mse_adjoint_operating_point(operating):
    """Full-size loss-fused path against the split path (same seed, same record)."""
    p, dp = operating
    W = H = 1024
    tgt = tbr.DeviceProgram.from_host(inputs.operating_target_program())
    target, _, _ = tbr.render_hard(tgt, W, H)
    loss_f, g_f, _, st = tbr.soft_adjoint_mse(dp, target, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN, stats=True)
    rgb, ctx = tbr.render_soft(dp, W, H, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN, record=True)
    loss_s, dL = tbr.loss_mse(rgb, target)
    g_s = ctx.backward(dL)
    assert abs(loss_f.item() - loss_s.item()) <= 1e-6 * abs(loss_s.item())
    for k in GROUPS:
        assert rel(g_f[k].cpu().numpy().ravel(), g_s[k].cpu().numpy().ravel()) <= 1e-4, k


# --------------------------------------------------------------------------- transfer renderer R_D

def _long_program():
    return inputs.make_program(120, seed=311, palette_seed=312, k=8, r_lo=0.004, r_hi=0.04, len_max=0.8,
                               p_drop=0.0)


@pytest.mark.parametrize("which", ["small", "long"])
def test_hard_sixteen_drops(small, which):
    """R_D hard render (capsule membership, sixteen-drop pull-back) against the
    oracle's, with the same band rule as the capsule renderer."""
    p = small[0] if which == "small" else _long_program()
    dp = tbr.DeviceProgram.from_host(p)
    W, H = 128, 96
    rgb, idx, st = tbr.render_hard(dp, W, H, stats=True, transport="drops")
    o = oracle.render_hard(p, W, H, with_kappa=True, transport="drops")
    c = check_hard(p, idx.cpu().numpy(), o, W, H, f"R_D {which}, stats {st}", transport="drops")
    assert c["mismatch"] < 0.01 * W * H
    ok = idx.cpu().numpy().ravel() == o["idx"]
    assert np.abs(rgb.cpu().numpy().reshape(-1, 3)[ok] - o["rgb"][ok]).max() < 1e-6


@pytest.mark.parametrize("which,W,H", [("small", 128, 128), ("long", 75, 61)])
def test_soft_sixteen_drops(small, which, W, H):
    p = small[0] if which == "small" else _long_program()
    dp = tbr.DeviceProgram.from_host(p)
    rgb, _ = tbr.render_soft(dp, W, H, 0.0, 1 / 200, transport="drops")
    o = oracle.render_soft(p, W, H, 0.0, 1 / 200, transport="drops")
    err = np.abs(rgb.cpu().numpy().reshape(-1, 3) - o["rgb"])
    print(f"R_D soft {which}: max {err.max():.3e} mean {err.mean():.3e}")
    assert err.max() <= SOFT_TOL


def test_soft_sixteen_drops_operating_point_sampled(operating):
    p, dp = operating
    W = H = 1024
    rgb, _ = tbr.render_soft(dp, W, H, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN, transport="drops")
    pix = inputs.sample_pixels(33, W * H, 2000)
    o = oracle.render_soft(p, W, H, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN, pix=pix, transport="drops")
    err = np.abs(rgb.cpu().numpy().reshape(-1, 3)[pix] - o["rgb"])
    print(f"R_D soft op max {err.max():.3e} mean {err.mean():.3e}")
    assert err.max() <= SOFT_TOL


def test_sixteen_drops_render_forward_only(small):
    _, dp = small
    with pytest.raises(tbr.TbrError) as ei:
        tbr.render_soft(dp, 32, 32, 0.0, 1 / 200, record=True, transport="drops")
    assert ei.value.status == tbr.TBR_ERR_INVALID_ARG


# --------------------------------------------------------------------------- early exit of the forward render

def _dense_program():
    return inputs.make_program(400, seed=71, palette_seed=72, k=6, r_lo=0.03, r_hi=0.1)


@pytest.mark.parametrize("eps", [1e-3, 1e-12])
def test_soft_early_exit_against_oracle(eps):
    """A pixel stops once T < eps (forward only): against the oracle's render
    with the same exit, and within eps of the GPU's full render."""
    p = _dense_program()
    dp = tbr.DeviceProgram.from_host(p)
    W, H = 97, 61
    ex, _ = tbr.render_soft(dp, W, H, 0.0, 1 / 200, early_exit=eps)
    full, _ = tbr.render_soft(dp, W, H, 0.0, 1 / 200)
    o = oracle.render_soft(p, W, H, 0.0, 1 / 200, early_exit=eps)
    err = np.abs(ex.cpu().numpy().reshape(-1, 3) - o["rgb"])
    gap = (ex - full).abs().max().item()
    print(f"early exit {eps:g}: vs oracle max {err.max():.3e}; vs full render {gap:.3e}; "
          f"oracle exited {(o['T0'] < eps).mean():.3f}")
    assert err.max() <= SOFT_TOL
    assert gap <= eps + 1e-6


def test_soft_early_exit_operating_point(operating):
    p, dp = operating
    W = H = 1024
    ex, _ = tbr.render_soft(dp, W, H, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN, early_exit=1e-12)
    pix = inputs.sample_pixels(37, W * H, 2000)
    o = oracle.render_soft(p, W, H, inputs.SHARP_TAU, inputs.SHARP_TAU_MIN, pix=pix, early_exit=1e-12)
    err = np.abs(ex.cpu().numpy().reshape(-1, 3)[pix] - o["rgb"])
    print(f"early exit op: max {err.max():.3e}, oracle exited {(o['T0'] < 1e-12).mean():.3f}")
    assert err.max() <= SOFT_TOL


@pytest.mark.parametrize("variant", ["drops", "coupled"])
def test_early_exit_with_other_transports(variant):
    p = _dense_program()
    if variant == "coupled":
        p.coupling = inputs.make_coupling(404, p.n)
    dp = tbr.DeviceProgram.from_host(p)
    tr = "drops" if variant == "drops" else "capsule"
    ex, _ = tbr.render_soft(dp, 64, 64, 0.0, 1 / 200, transport=tr, early_exit=1e-9)
    full, _ = tbr.render_soft(dp, 64, 64, 0.0, 1 / 200, transport=tr)
    assert (ex - full).abs().max().item() <= 1e-6


def test_early_exit_arguments(small):
    _, dp = small
    for kw in ({"early_exit": 1e-9, "record": True}, {"early_exit": 1.0}, {"early_exit": -1e-3}):
        with pytest.raises(tbr.TbrError) as ei:
            tbr.render_soft(dp, 16, 16, 0.0, 1 / 200, **kw)
        assert ei.value.status == tbr.TBR_ERR_INVALID_ARG
