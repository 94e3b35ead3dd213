"""Comparisons shared by the GPU parity tests: gradients and hard-render indices.

Gradients.  Two measures of a GPU gradient group g against the oracle's g_ref:

  * the group norm ratio  ||g - g_ref||_2 / ||g_ref||_2 <= 1e-3;
  * per element: |g_j - g_ref_j| <= 1e-3 * max(|g_ref_j|, 1e-3 * max_j |g_ref_j|),
    i.e. each entry held to the relative bound on its own, except entries
    smaller than a thousandth of the group's largest, which are held to the
    bound times that floor.

Some entries are fixed by their inputs less tightly than that: moving every
stroke parameter by one FP32 rounding (relative 6e-8) moves the oracle's own
FP64 gradient entry by more than 1e-3 of it (a pixel just outside a deposit is
pulled back with an unbounded stretch, Eq. back).  No FP32 evaluation can do
better there, so an entry also passes when its error is within 4 x that
measured move (``oracle_sensitivity``); those entries are counted, printed and
limited to a small share of the group.  The worst element is printed with its
index so that a failure names the stroke.

A group that is zero by construction (d/d theta when every stroke is a drop:
a drop has no direction) has no relative error: the oracle returns FP64
rounding around zero there.  A group whose oracle norm is below ZERO_GROUP of
the largest group norm is therefore held to an absolute bound instead, its
GPU norm below ZERO_TOL of that largest norm.
"""
import numpy as np

import oracle

GRAD_TOL = 1e-3
GROUPS = ["cx", "cy", "theta", "length", "half_width", "logits", "palette"]
SENS_FACTOR = 4.0
MAX_COND_FRAC = 0.05   # share of a group's entries that may pass by the sensitivity allowance
KAPPA_EPS = 6e-8       # one FP32 rounding, relative
ZERO_GROUP = 1e-12     # a group this small against the largest is zero by construction
ZERO_TOL = 1e-9        # ... and its GPU values must stay this small against the largest


def as_np(t):
    if hasattr(t, "detach"):
        t = t.detach().cpu().numpy()
    return np.asarray(t, dtype=np.float64).ravel()


def norm_ratio(a, b):
    a, b = as_np(a), as_np(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def elem_ratio(a, b, floor_frac=1e-3):
    """(worst per-element ratio, its flat index)."""
    a, b = as_np(a), as_np(b)
    if b.size == 0:
        return 0.0, -1
    floor = max(floor_frac * float(np.abs(b).max()), 1e-300)
    r = np.abs(a - b) / np.maximum(np.abs(b), floor)
    j = int(np.argmax(r))
    return float(r[j]), j


def perturbed_programs(p, trials, seed=2026):
    """Copies of p with every geometric stroke parameter moved by at most one
    FP32 rounding (relative 6e-8), in FP64."""
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        q = p.copy()
        for k in ("cx", "cy", "theta", "length", "half_width"):
            v = np.asarray(getattr(q, k), np.float64)
            setattr(q, k, v * (1.0 + rng.uniform(-KAPPA_EPS, KAPPA_EPS, v.shape)))
        yield q


def oracle_sensitivity(p, W, H, tau, tau_min, cot, og, pix=None, inert=False, trials=3):
    """Per group: the largest elementwise move |g'_j - g_j| of the oracle's
    stored-state gradient over ``trials`` perturbations of the inputs by one
    FP32 rounding, and the largest group norm ratio of that move."""
    elem = {k: np.zeros(as_np(og[k]).size) for k in GROUPS}
    norm = {k: 0.0 for k in GROUPS}
    for q in perturbed_programs(p, trials):
        oq = oracle.soft_vjp(q, W, H, tau, tau_min, cot, inert=inert, pix=pix)
        for k in GROUPS:
            elem[k] = np.maximum(elem[k], np.abs(as_np(oq[k]) - as_np(og[k])))
            norm[k] = max(norm[k], norm_ratio(oq[k], og[k]))
    return {"elem": elem, "norm": norm}


def compare(g, og, groups=GROUPS, tol=GRAD_TOL, elem_tol=None, sens=None, label="", max_cond_frac=MAX_COND_FRAC,
            norm_sens=False):
    """Assert the norm and per-element bounds above (elem_tol defaults to tol);
    with ``sens`` (``oracle_sensitivity``) an entry may instead be within
    SENS_FACTOR x its measured sensitivity.  With ``norm_sens`` a group's norm
    ratio may exceed tol only where the oracle's own group norm moves by more
    than tol under one FP32 rounding of the inputs, and is then held to that
    measured move (no factor).  Returns {group: (norm ratio, worst element
    ratio over the entries held to the relative bound, its index, entries that
    passed by the allowance)}."""
    elem_tol = tol if elem_tol is None else elem_tol
    out = {}
    scale = max([float(np.linalg.norm(as_np(og[k]))) for k in groups if as_np(og[k]).size] + [0.0])
    for k in groups:
        a, b = as_np(g[k]), as_np(og[k])
        n = norm_ratio(a, b)
        if b.size == 0:
            out[k] = (n, 0.0, -1, 0)
            continue
        if float(np.linalg.norm(b)) <= ZERO_GROUP * scale:  # zero by construction
            za = float(np.linalg.norm(a))
            assert za <= ZERO_TOL * scale, f"{label} {k}: zero group, GPU norm {za:.3e} against {scale:.3e}"
            out[k] = (0.0, 0.0, -1, 0)
            continue
        floor = max(1e-3 * float(np.abs(b).max()), 1e-300)
        err = np.abs(a - b)
        r = err / np.maximum(np.abs(b), floor)
        cond = np.zeros(b.size, bool)
        if sens is not None:
            cond = (r > elem_tol) & (err <= SENS_FACTOR * sens["elem"][k])
        rr = np.where(cond, 0.0, r)
        j = int(np.argmax(rr))
        out[k] = (n, float(rr[j]), j, int(cond.sum()))
    print(f"{label} gradients: " + ", ".join(
        f"{k} norm {n:.2e} elem {e:.2e}@{j}" + (f" ({c} by sensitivity)" if c else "")
        for k, (n, e, j, c) in out.items()))
    for k, (n, e, j, c) in out.items():
        bound = max(tol, sens["norm"][k]) if (norm_sens and sens is not None) else tol
        if n > tol:
            print(f"{label} {k}: norm ratio {n:.3e} against the oracle's own move {bound:.3e}")
        assert n <= bound, f"{label} {k}: norm ratio {n:.3e} > {bound:.3e}"
        assert e <= elem_tol, f"{label} {k}: element {j} ratio {e:.3e} > {elem_tol}"
        size = as_np(og[k]).size
        assert c <= max(1, max_cond_frac * size), f"{label} {k}: {c} of {size} entries pass only by sensitivity"
    return out


# --------------------------------------------------------------------------- hard render

BAND = 1e-5            # oracle margin min_j |sigma'_j - r_j| below which a pixel is a boundary pixel
MAX_EXCUSED_FRAC = 2e-3


def check_hard(p, idx_gpu, o, W, H, label, pix=None, trials=8, max_excused_frac=MAX_EXCUSED_FRAC, **render_kw):
    """Terminating-index agreement of a GPU hard render with the oracle's.

    o is the oracle's render (with kappa) of the pixels ``pix`` (all when None);
    idx_gpu the GPU's indices of the same pixels.  Rules:
      * pixels whose oracle margin is below BAND are boundary pixels: counted,
        not compared;
      * a mismatch outside the band is excused only where the oracle's chain
        condition kappa makes the FP32 trajectory uncertain beyond BAND
        (kappa * 6e-8 > BAND); any other mismatch fails;
      * excused pixels are at most ``max_excused_frac`` of the pixels, and each
        is re-rendered by the oracle under ``trials`` perturbations of the
        inputs by one FP32 rounding: the number whose GPU index one of those
        runs reproduces is reported.
    Returns the counts."""
    idx_gpu = np.asarray(idx_gpu).ravel()
    mism = idx_gpu != o["idx"]
    band = o["margin"] < BAND
    outside = mism & ~band
    cond = o["kappa"] * KAPPA_EPS > BAND
    excused = outside & cond
    n = idx_gpu.size
    reproduced = 0
    if excused.any():
        where = np.flatnonzero(excused)
        opix = where if pix is None else np.asarray(pix)[where]
        hit = np.zeros(where.size, bool)
        for q in perturbed_programs(p, trials):
            oq = oracle.render_hard(q, W, H, pix=opix, **render_kw)
            hit |= oq["idx"] == idx_gpu[where]
        reproduced = int(hit.sum())
    print(f"{label}: {n} px, band {int(band.sum())}, mismatches {int(mism.sum())}, outside band "
          f"{int(outside.sum())}, excused by kappa {int(excused.sum())} (reproduced by a perturbed oracle "
          f"{reproduced})")
    bad = np.flatnonzero(outside & ~cond)
    assert bad.size == 0, f"{label}: {bad.size} unexplained index mismatches, first at {bad[:5]}"
    assert excused.sum() <= max(2, max_excused_frac * n), f"{label}: {int(excused.sum())} kappa-excused pixels"
    return {"band": int(band.sum()), "mismatch": int(mism.sum()), "excused": int(excused.sum()),
            "reproduced": reproduced}
