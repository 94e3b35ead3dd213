"""Fit (Sec. 5.1 with Table "hyper") and the torch autograd wrapper, on the GPU.

- The first fit step is exactly one Adam update (bias-corrected, cosine-scaled
  rates, length regulariser, projections) of the gradient the loss-fused call
  returns for the same program, relaxation and colour temperature.
- A short fit lowers the loss, keeps every parameter in its feasible set, is
  bitwise reproducible, and its final loss agrees with the FP64 oracle's loss
  of the same program.
- SoftRender (torch.autograd.Function) gives the gradients of the plain
  forward + loss + replay adjoint calls.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2609_08722_b300 import inputs, tbr

pytestmark = pytest.mark.gpu

W = H = 96
GROUPS5 = ["cx", "cy", "theta", "length", "half_width"]


@pytest.fixture(scope="module")
def problem():
    init = inputs.make_program(60, seed=901, palette_seed=903, k=8, r_lo=0.01, r_hi=0.06)
    targ = inputs.make_program(60, seed=902, palette_seed=903, k=8, r_lo=0.01, r_hi=0.06)
    target, _, _ = tbr.render_hard(tbr.DeviceProgram.from_host(targ), W, H)
    return init, target


def schedule(c, t):
    T = c.iterations
    geo = lambda a, b: a * (b / a) ** (t / (T - 1))
    return geo(c.tau_start, c.tau_end), geo(c.color_temp_start, c.color_temp_end), \
        0.5 * (1.0 + math.cos(math.pi * t / T))


def to_program(dp, color_temp):
    """Host copy of a device program (the float32 values the GPU holds)."""
    a = lambda t: t.detach().cpu().numpy().astype(np.float32).copy()
    return inputs.Program(cx=a(dp.cx), cy=a(dp.cy), theta=a(dp.theta), length=a(dp.length),
                          half_width=a(dp.half_width), logits=a(dp.logits), palette=a(dp.palette),
                          background=np.asarray(dp.background, dtype=np.float32), color_temp=color_temp)


def params_of(dp):
    return {k: getattr(dp, k).detach().double().cpu().numpy().ravel().copy()
            for k in GROUPS5 + ["logits", "palette"]}


def test_first_step_is_one_adam_update(problem):
    init, target = problem
    cfg = tbr.default_fit_config(iterations=50)
    dp = tbr.DeviceProgram.from_host(init)
    fit = tbr.Fit(dp, target, cfg)
    tau, tc, cosine = schedule(cfg, 0)
    tau_min = 0.7 / max(W, H)
    view = fit.program()
    assert abs(view.color_temp - tc) < 1e-6
    loss_g, g, _, _ = tbr.soft_adjoint_mse(view, target, tau, tau_min, want_palette=False)
    p0 = params_of(view)
    loss = fit.step()
    p1 = params_of(fit.program())
    fit.destroy()
    torch.cuda.synchronize()
    lam = cfg.length_weight
    assert abs(loss - (loss_g.item() + lam * p0["length"].sum())) <= 1e-5 * abs(loss)
    lr = {"cx": cfg.lr_center, "cy": cfg.lr_center, "theta": cfg.lr_angle, "length": cfg.lr_length,
          "half_width": cfg.lr_width, "logits": cfg.lr_logits}
    r0 = init.half_width.astype(np.float64)
    for name in GROUPS5 + ["logits"]:
        gr = g[name].double().cpu().numpy().ravel()
        if name == "length":
            gr = gr + lam
        m = (1 - cfg.beta1) * gr
        v = (1 - cfg.beta2) * gr * gr
        step = lr[name] * cosine * (m / (1 - cfg.beta1)) / (np.sqrt(v / (1 - cfg.beta2)) + cfg.adam_eps)
        want = p0[name] - step
        if name in ("cx", "cy"):
            want = np.clip(want, 0.0, 1.0)
        elif name == "length":
            want = np.clip(want, 0.0, cfg.length_max)
        elif name == "half_width":
            want = np.clip(want, cfg.width_lo * r0, cfg.width_hi * r0)
        err = np.abs(p1[name] - want).max()
        assert err <= 2e-6 * max(1.0, np.abs(want).max()), (name, err)
    assert np.array_equal(p1["palette"], p0["palette"])  # palette not trained by default


def run_fit(init, target, steps, cfg):
    fit = tbr.Fit(tbr.DeviceProgram.from_host(init), target, cfg)
    losses = [fit.step() for _ in range(steps)]
    prog = fit.program()
    fit.destroy()
    return losses, prog


def test_fit_lowers_the_loss_and_stays_feasible(problem):
    init, target = problem
    cfg = tbr.default_fit_config(iterations=40)
    losses, prog = run_fit(init, target, 40, cfg)
    print(f"loss {losses[0]:.5f} -> {losses[-1]:.5f}")
    assert losses[-1] < 0.9 * losses[0]
    p = params_of(prog)
    r0 = init.half_width.astype(np.float64)
    assert (p["cx"] >= 0).all() and (p["cx"] <= 1).all() and (p["cy"] >= 0).all() and (p["cy"] <= 1).all()
    assert (p["length"] >= 0).all() and (p["length"] <= cfg.length_max + 1e-7).all()
    assert (p["half_width"] >= cfg.width_lo * r0 * (1 - 1e-6)).all()
    assert (p["half_width"] <= cfg.width_hi * r0 * (1 + 1e-6)).all()
    # FP32 loss of the final program against the FP64 oracle's (final schedule values)
    tau, tc, _ = schedule(cfg, cfg.iterations - 1)
    tau_min = 0.7 / max(W, H)
    final = to_program(prog, tc)
    rgb, _ = tbr.render_soft(tbr.DeviceProgram.from_host(final), W, H, tau, tau_min)
    loss_gpu, _ = tbr.loss_mse(rgb, target, want_grad=False)
    o = oracle.render_soft(final, W, H, tau, tau_min)
    loss_o = float(np.mean((o["rgb"] - target.double().cpu().numpy().reshape(-1, 3)) ** 2))
    print(f"final loss gpu {loss_gpu.item():.8f} oracle {loss_o:.8f}")
    assert abs(loss_gpu.item() - loss_o) <= 1e-4 * loss_o


def test_fit_is_reproducible(problem):
    init, target = problem
    cfg = tbr.default_fit_config(iterations=10)
    la, pa = run_fit(init, target, 5, cfg)
    lb, pb = run_fit(init, target, 5, cfg)
    assert la == lb
    for k in GROUPS5 + ["logits"]:
        assert torch.equal(getattr(pa, k), getattr(pb, k))


def test_soft_render_autograd_matches_the_adjoint_calls(problem):
    init, target = problem
    dp = tbr.DeviceProgram.from_host(init)
    leaves = {k: getattr(dp, k).clone().requires_grad_(True) for k in GROUPS5 + ["logits", "palette"]}
    rgb = tbr.soft_render(leaves["cx"], leaves["cy"], leaves["theta"], leaves["length"], leaves["half_width"],
                          leaves["logits"], leaves["palette"], W, H, 0.0, 1 / 200, background=dp.background,
                          color_temp=dp.color_temp)
    loss = ((rgb - target) ** 2).mean()
    loss.backward()
    rgb2, ctx = tbr.render_soft(dp, W, H, 0.0, 1 / 200, record=True)
    assert torch.equal(rgb.detach(), rgb2)
    _, dL = tbr.loss_mse(rgb2, target)
    g = ctx.backward(dL)
    for k in GROUPS5 + ["logits", "palette"]:
        a, b = leaves[k].grad, g[k]
        rel = (a - b).norm().item() / max(b.norm().item(), 1e-30)
        assert rel <= 1e-5, (k, rel)


def test_full_fit_workload_fp32_vs_fp64_loss():
    """The 200-step fit at 1024^2 x 2000 strokes (seeds 104/105): the final
    program's FP32 soft loss against the FP64 oracle's on 16384 sampled pixels."""
    from paper_2609_08722_b300 import fit_bench
    rep, final_h, target = fit_bench.run(200)
    W = H = fit_bench.RES
    soft, _ = tbr.render_soft(tbr.DeviceProgram.from_host(final_h), W, H, rep["tau_end"], rep["tau_min"])
    pix = inputs.sample_pixels(77, W * H, 16384)
    tgt = target.reshape(-1, 3).double().cpu().numpy()[pix]
    gpu = soft.reshape(-1, 3).double().cpu().numpy()[pix]
    o = oracle.render_soft(final_h, W, H, rep["tau_end"], rep["tau_min"], pix=pix)
    loss_gpu = float(np.mean((gpu - tgt) ** 2))
    loss_fp64 = float(np.mean((o["rgb"] - tgt) ** 2))
    gap = abs(loss_gpu - loss_fp64) / loss_fp64
    print(f"fit report {rep}")
    print(f"final soft loss on the sample: fp32 {loss_gpu:.8f} fp64 {loss_fp64:.8f} gap {gap:.2e}")
    assert rep["loss_last"] < rep["loss_first"]
    assert gap <= 1e-3
