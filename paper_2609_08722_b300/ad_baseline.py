"""Checkpointed automatic differentiation of the soft render: the baseline the
replay adjoint is weighed against in memory and time (Sec. 5.2, Table
"adjoint": autograd with a checkpoint every 20 strokes).

Plain PyTorch tensor operations on the GPU, in FP32: for each stroke, the
frame coordinates, the distance to the segment, the relaxed coverage (Eq.
relax, clamped at 1 - 1e-7), the compositing update (Eq. state) and the
epsilon-floored pull-back (Eq. back with the centred arclength of Eq. phi),
over all pixels at once.  Autograd differentiates it; torch.utils.checkpoint
wraps every run of ``segment`` strokes, so the forward keeps only the states at
segment boundaries and the backward recomputes one segment at a time.

This is a measurement baseline, not the product path: the library's renders
and adjoint are the CUDA kernels behind the C ABI.  It makes no claim of speed;
it measures what checkpointed AD holds in device memory for the same loss and
gradients.
"""
from __future__ import annotations

import math

import torch
from torch.utils.checkpoint import checkpoint

EPS_FLOOR = 1e-3                      # the epsilon of the floor, Sec. 5.2
Z_MAX = math.log(1e7 - 1.0)           # coverage clamp alpha <= 1 - 1e-7
PI = math.pi


def _stroke(x, y, C, T, cx, cy, th, L, r, col, w):
    """One stroke of the soft render at pixel positions (x, y): returns the
    pulled-back positions and the composited colour and transmittance."""
    ex, ey = torch.cos(th), torch.sin(th)
    dx, dy = x - cx, y - cy
    s = dx * ex + dy * ey
    h = dy * ex - dx * ey
    a_s, a_h = s.abs(), h.abs()
    hl = 0.5 * L
    u = (a_s - hl).clamp_min(0.0)
    sp = torch.sqrt(u * u + a_h * a_h + 1e-30)          # sigma'
    z = ((r - sp) / w).clamp(max=Z_MAX)
    alpha = torch.sigmoid(z)
    C = C + (T * alpha).unsqueeze(-1) * col
    T = T * (1.0 - alpha)
    # Eq. back: C_a = A_L(sigma') - A_L(r), floored at (eps r)^2, and the root
    area = torch.maximum((sp - r) * (2.0 * L + PI * (sp + r)), (EPS_FLOOR * r) ** 2)
    sig = area / (L + torch.sqrt(L * L + PI * area))
    # centred arclength kept: folded arclength t from the flank midpoint
    cap_in = a_s > hl
    phi = torch.atan2(u, a_h)
    t = torch.where(cap_in, hl + sp * phi, a_s)
    tn = t * (L + PI * sig) / (L + PI * sp)
    cap_out = tn > hl
    beta = ((tn - hl) / sig).clamp(max=0.5 * PI)
    sn = torch.where(cap_out, hl + sig * torch.sin(beta), tn)
    hn = torch.where(cap_out, sig * torch.cos(beta), sig)
    so = torch.where(s >= 0, sn, -sn)
    ho = torch.where(h >= 0, hn, -hn)
    return cx + so * ex - ho * ey, cy + so * ey + ho * ex, C, T


def _segment(x, y, C, T, cx, cy, th, L, r, col, w):
    """Strokes of one segment, last first (the tensors hold that order)."""
    for j in range(cx.shape[0]):
        x, y, C, T = _stroke(x, y, C, T, cx[j], cy[j], th[j], L[j], r[j], col[j], w[j])
    return x, y, C, T


def soft_render(cx, cy, theta, length, half_width, logits, palette, background, color_temp, W, H, tau, tau_min,
                segment=20, rows=None):
    """Soft render R [len(rows) or H, W, 3] (FP32) with autograd, checkpointed
    every ``segment`` strokes (0: no checkpoints).  rows: optional 1-D tensor of
    pixel rows to render (a band of the image)."""
    dev = cx.device
    ys = torch.arange(H, device=dev, dtype=torch.float32) if rows is None else rows.to(dev, torch.float32)
    xs = torch.arange(W, device=dev, dtype=torch.float32)
    y = ((ys + 0.5) / H)[:, None].expand(-1, W).contiguous()
    x = ((xs + 0.5) / W)[None, :].expand(ys.shape[0], -1).contiguous()
    col = torch.softmax(logits / color_temp, dim=1) @ palette       # [n, 3]
    w = torch.clamp_min(tau * half_width, tau_min)
    C = torch.zeros(x.shape + (3,), device=dev)
    T = torch.ones_like(x)
    n = cx.shape[0]
    seg = n if segment <= 0 else segment
    for hi in range(n, 0, -seg):
        lo = max(0, hi - seg)
        idx = torch.arange(hi - 1, lo - 1, -1, device=dev)   # strokes hi-1 .. lo
        args = (cx[idx], cy[idx], theta[idx], length[idx], half_width[idx], col[idx], w[idx])
        if segment > 0:
            x, y, C, T = checkpoint(_segment, x, y, C, T, *args, use_reentrant=False)
        else:
            x, y, C, T = _segment(x, y, C, T, *args)
    return C + T.unsqueeze(-1) * background


def mse_step(prog, target, W, H, tau, tau_min, segment=20, rows=None):
    """One loss + gradient evaluation: the mean squared error of the soft
    render against ``target`` ([len(rows) or H, W, 3]), differentiated by
    autograd.  prog holds device tensors cx, cy, theta, length, half_width,
    logits, palette, background and the float color_temp.  Returns (loss,
    {name: gradient}) for the stroke parameters and the logits."""
    names = ("cx", "cy", "theta", "length", "half_width", "logits")
    leaves = {k: getattr(prog, k).detach().clone().requires_grad_(True) for k in names}
    R = soft_render(leaves["cx"], leaves["cy"], leaves["theta"], leaves["length"], leaves["half_width"],
                    leaves["logits"], prog.palette, prog.background, prog.color_temp, W, H, tau, tau_min,
                    segment=segment, rows=rows)
    loss = torch.mean((R - target) ** 2)
    loss.backward()
    return loss.detach(), {k: v.grad for k, v in leaves.items()}
