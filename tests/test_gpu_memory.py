"""Memory side of the replay adjoint (Sec. 5.2, Table "adjoint" and the
checkpoint sweep): the replay context at checkpoint intervals k = 32 .. 256 on
the 2000-stroke operating program at 1024^2, and the checkpointed-AD baseline
the benchmark times beside it.

  * every k gives the oracle's gradients within the bounds of
    ``paritycheck.compare`` (the interval only moves where positions are reset,
    not what is computed), and the context shrinks as k grows;
  * the checkpointed-AD baseline (plain PyTorch autograd, a checkpoint every 20
    strokes) renders and differentiates the same soft render as the oracle, so
    its peak memory is that of the same computation.  It is plain FP32 without
    the displacement form, so it is held to 1e-4 on colour and 3e-3 on the
    gradient group norms.
"""
import numpy as np
import pytest
import torch

import oracle
from paritycheck import compare, norm_ratio, oracle_sensitivity
from paper_2609_08722_b300 import ad_baseline, inputs, tbr

pytestmark = pytest.mark.gpu

NAMES = ["cx", "cy", "theta", "length", "half_width", "logits"]


def test_checkpoint_interval_sweep_operating_point():
    p = inputs.operating_program()
    dp = tbr.DeviceProgram.from_host(p)
    W = H = 1024
    tau, tau_min = inputs.SHARP_TAU, inputs.SHARP_TAU_MIN
    pix = inputs.sample_pixels(45, W * H, 2048)
    cot = inputs.make_cotangent(46, pix.size)
    full = torch.zeros((H * W, 3), device="cuda")
    full[torch.from_numpy(pix).cuda()] = torch.from_numpy(cot).cuda()
    og = oracle.soft_vjp(p, W, H, tau, tau_min, cot.astype(np.float64), pix=pix)
    sens = oracle_sensitivity(p, W, H, tau, tau_min, cot.astype(np.float64), og, pix=pix)
    ref, sizes = None, {}
    for k in (32, 64, 128, 256):
        _, ctx = tbr.render_soft(dp, W, H, tau, tau_min, record=True, checkpoint_every=k)
        g = ctx.backward(full.view(H, W, 3))
        st = ctx.status()
        sizes[k] = ctx.nbytes()
        compare(g, og, sens=sens, label=f"k = {k} (context {sizes[k] / 2**30:.2f} GiB, drift resets "
                                        f"{st['drift_resets']})")
        if ref is None:
            ref = g
        else:
            for name in NAMES:
                assert norm_ratio(g[name], ref[name]) <= 1e-5, (k, name)
        ctx.destroy()
    assert sizes[32] > sizes[64] > sizes[128] > sizes[256]


def _device_program(p):
    class P:
        pass
    d = P()
    for name in ("cx", "cy", "theta", "length", "half_width", "logits", "palette", "background"):
        setattr(d, name, torch.tensor(np.asarray(getattr(p, name), np.float32), device="cuda"))
    d.color_temp = float(p.color_temp)
    return d


@pytest.mark.parametrize("segment", [20, 0])
def test_checkpointed_ad_baseline_is_the_same_computation(segment):
    p = inputs.small_program()
    W, H = 64, 48
    d = _device_program(p)
    R = ad_baseline.soft_render(d.cx, d.cy, d.theta, d.length, d.half_width, d.logits, d.palette, d.background,
                                d.color_temp, W, H, 0.0, 1 / 200, segment=segment)
    o = oracle.render_soft(p, W, H, 0.0, 1 / 200)
    err = np.abs(R.detach().cpu().numpy().reshape(-1, 3) - o["rgb"]).max()
    assert err <= 1e-4, err
    # a target for which dL/dR is the seeded cotangent: 2 (R - target) / (3P) = cot
    cot = inputs.make_cotangent(47, W * H)
    target = R.detach() - torch.from_numpy(cot).cuda().reshape(H, W, 3) * (1.5 * W * H)
    _, g = ad_baseline.mse_step(d, target, W, H, 0.0, 1 / 200, segment=segment)
    og = oracle.soft_vjp(p, W, H, 0.0, 1 / 200, cot.astype(np.float64))
    errs = {k: norm_ratio(g[k], og[k]) for k in NAMES}
    print(f"checkpointed AD (segment {segment}): colour {err:.2e}, gradients "
          + ", ".join(f"{k} {e:.2e}" for k, e in errs.items()))
    for k, e in errs.items():
        assert e <= 3e-3, k
