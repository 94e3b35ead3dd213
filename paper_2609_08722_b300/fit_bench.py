"""Full-fit workload (Sec. 5.1 inverse rendering with Table "hyper"): a
2000-stroke program (seed 104) fitted for 200 Adam steps at 1024^2 to the hard
render of a second program (seed 105).  Reports seconds per step (mean of
steps 2..200, CUDA events), the loss trace, the final hard-render L2 against
the target, the final soft loss (at the last relaxation and colour
temperature) and the device memory the fit holds.  The final program is
returned too, for the FP64 loss comparison in the GPU tests.

    python -m paper_2609_08722_b300.fit_bench [steps]
"""
from __future__ import annotations

import json
import sys

import numpy as np
import torch

from . import inputs, tbr

RES = 1024


def _schedule(c, t):
    T = c.iterations
    geo = lambda a, b: a * (b / a) ** (t / (T - 1)) if T > 1 else b
    return geo(c.tau_start, c.tau_end), geo(c.color_temp_start, c.color_temp_end)


def _host_program(dp, color_temp):
    a = lambda t: t.detach().cpu().numpy().astype(np.float32).copy()
    return inputs.Program(cx=a(dp.cx), cy=a(dp.cy), theta=a(dp.theta), length=a(dp.length),
                          half_width=a(dp.half_width), logits=a(dp.logits), palette=a(dp.palette),
                          background=np.asarray(dp.background, dtype=np.float32), color_temp=color_temp)


def run(steps: int = 200) -> tuple[dict, inputs.Program, torch.Tensor]:
    """Returns (report, final program on the host, target image)."""
    init_h, targ_h = inputs.fit_programs()
    W = H = RES
    target, _, _ = tbr.render_hard(tbr.DeviceProgram.from_host(targ_h), W, H, with_idx=False)
    cfg = tbr.default_fit_config(iterations=steps, checkpoint_every=64)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    fit = tbr.Fit(tbr.DeviceProgram.from_host(init_h), target, cfg)
    losses, times = [], []
    peak = 0
    for t in range(steps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        losses.append(fit.step())
        e.record()
        e.synchronize()
        times.append(s.elapsed_time(e))
        peak = max(peak, free0 - torch.cuda.mem_get_info()[0])
    final = fit.program()
    fit.destroy()
    tau, tc = _schedule(cfg, steps - 1)
    tau_min = 0.7 / max(W, H)
    final_h = _host_program(final, tc)
    # final hard render against the target
    dp_final = tbr.DeviceProgram.from_host(final_h)
    hard, _, _ = tbr.render_hard(dp_final, W, H, with_idx=False)
    hard_l2 = float(((hard - target) ** 2).mean().item())
    soft, _ = tbr.render_soft(dp_final, W, H, tau, tau_min)
    soft_loss, _ = tbr.loss_mse(soft, target, want_grad=False)
    ms = float(np.mean(times[1:])) if steps > 1 else float(times[0])
    report = {
        "workload": f"fit of a 2000-stroke program (seed 104) to the hard render of seed 105 at {W}x{H}",
        "steps": steps, "s_per_step": ms * 1e-3, "first_step_s": times[0] * 1e-3,
        "loss_first": losses[0], "loss_last": losses[-1],
        "loss_trace": [losses[i] for i in range(0, steps, max(1, steps // 20))] + [losses[-1]],
        "final_hard_l2": hard_l2, "final_soft_loss": float(soft_loss.item()),
        "device_memory_held_gb": peak / 1e9,
        "tau_end": tau, "tau_min": tau_min, "color_temp_end": tc,
    }
    return report, final_h, target


if __name__ == "__main__":
    steps = int(sys.argv[1]) if len(sys.argv) > 1 else 200
    print(json.dumps(run(steps)[0]))
