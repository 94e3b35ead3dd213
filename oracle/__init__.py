"""FP64 CPU oracle for transport-based rendering (TEST INFRASTRUCTURE ONLY).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (``paper_2609_08722_b300``) never
does, and the two share no code: the oracle receives the same seeded input arrays
and recomputes everything from the paper's definitions in ``tbr_oracle.cpp``.

Functions (all FP64, citing the paper's passages in the C++ source):
  * ``psi_map`` / ``phi_map``     -- Eq. back / Eq. fwd on a batch of points;
  * ``map_jacobian``             -- their 2x7 Jacobians by dual numbers;
  * ``coupled_map``              -- the coupling variant Phi_g / psi_g (Eq. coupling);
  * ``profile_min``              -- exact minimum of its profile g (Eq. profile);
  * ``drops_map``                -- the sixteen-drop operator of R_D;
  * ``compensate``               -- the one-pass closed-form compensation baseline;
  * ``render_hard``              -- Eq. chain + Eq. render with indicator coverage;
  * ``render_soft``              -- Eq. relax + Eq. state;
  * ``soft_jvp``                 -- forward-mode derivative of the soft render;
  * ``soft_vjp``                 -- stored-state adjoint (Eq. adjstep, Eq. adjparam);
  * ``fd_gradient``              -- central finite differences of a linear
                                    functional of the soft render;
  * ``count_ops``                -- operation counts per pixel-stroke of the
                                    hard render, the soft render and the
                                    replay adjoint (measurement only).

A program is any object with attributes ``cx, cy, theta, length, half_width``
([n]), ``logits`` ([n, k]), ``palette`` ([k, 3]), ``background`` ([3]) and
``color_temp`` (float), and optionally ``coupling`` ([n, 3] c_1..c_3 of Eq.
profile, or None for the capsule map).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tbr_oracle.cpp")
_LIB = os.path.join(_HERE, "libtbr_oracle.so")
_lock = threading.Lock()
_lib = None

MODE_CLAMP, MODE_FLOOR, MODE_RAWQ, MODE_FLOOR_RAWQ = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libtbr_oracle.so`` (g++ -O2 -fopenmp)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared",
               "-ffp-contract=off", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Prog(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("k", ctypes.c_int32),
        ("cx", ctypes.c_void_p), ("cy", ctypes.c_void_p), ("th", ctypes.c_void_p),
        ("L", ctypes.c_void_p), ("r", ctypes.c_void_p),
        ("logits", ctypes.c_void_p), ("palette", ctypes.c_void_p),
        ("background", ctypes.c_double * 3), ("color_temp", ctypes.c_double),
        ("coupling", ctypes.c_void_p),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            lib.orc_map.argtypes = [P, i64, dbl, dbl, dbl, dbl, dbl, ctypes.c_int, ctypes.c_int, P, P]
            lib.orc_map_jacobian.argtypes = [P, i64, dbl, dbl, dbl, dbl, dbl, ctypes.c_int, ctypes.c_int, P]
            lib.orc_render_hard.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, P, i64, P, P, P, P]
            lib.orc_render_soft.argtypes = [P, ctypes.c_int, ctypes.c_int, dbl, dbl, ctypes.c_int,
                                            P, i64, P, P, P, dbl]
            lib.orc_soft_jvp.argtypes = [P, ctypes.c_int, ctypes.c_int, dbl, dbl, ctypes.c_int,
                                         P, i64, ctypes.c_int, ctypes.c_int, P]
            lib.orc_soft_vjp.argtypes = [P, ctypes.c_int, ctypes.c_int, dbl, dbl, ctypes.c_int,
                                         P, i64, P, P, P, P, P]
            lib.orc_map_drops.argtypes = [P, i64, dbl, dbl, dbl, dbl, dbl, ctypes.c_int, P, P, P]
            lib.orc_map_drops.restype = ctypes.c_int
            lib.orc_compensate.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P, P, P]
            lib.orc_compensate.restype = ctypes.c_int
            lib.orc_map_coupled.argtypes = [P, i64, dbl, dbl, dbl, dbl, dbl, dbl, dbl, dbl, ctypes.c_int,
                                            ctypes.c_int, P, P, P, P]
            lib.orc_map_coupled.restype = ctypes.c_int
            lib.orc_profile_min.argtypes = [dbl, dbl, dbl]
            lib.orc_profile_min.restype = dbl
            lib.orc_count_ops.argtypes = [P, ctypes.c_int, ctypes.c_int, dbl, dbl, ctypes.c_int, P, i64, P]
            lib.orc_count_ops.restype = ctypes.c_int
            lib.orc_num_threads.restype = ctypes.c_int
            for f in ("orc_map", "orc_map_jacobian", "orc_render_hard", "orc_render_soft",
                      "orc_soft_jvp", "orc_soft_vjp"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def num_threads() -> int:
    return _load().orc_num_threads()


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class _Packed:
    """Holds FP64 copies of a program's arrays and the ctypes struct pointing at them."""

    def __init__(self, prog):
        f64 = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        self.cx, self.cy = f64(prog.cx), f64(prog.cy)
        self.th, self.L, self.r = f64(prog.theta), f64(prog.length), f64(prog.half_width)
        self.logits, self.palette = f64(prog.logits), f64(prog.palette)
        n = self.cx.shape[0]
        k = self.palette.shape[0]
        if self.logits.shape != (n, k):
            raise ValueError("logits must be [n, k]")
        s = _Prog()
        s.n, s.k = n, k
        s.cx, s.cy, s.th = _ptr(self.cx), _ptr(self.cy), _ptr(self.th)
        s.L, s.r = _ptr(self.L), _ptr(self.r)
        s.logits, s.palette = _ptr(self.logits), _ptr(self.palette)
        bg = np.asarray(prog.background, dtype=np.float64)
        s.background = (ctypes.c_double * 3)(*bg.tolist())
        s.color_temp = float(prog.color_temp)
        cpl = getattr(prog, "coupling", None)
        self.coupling = None
        if cpl is not None:
            self.coupling = f64(cpl)
            if self.coupling.shape != (n, 3):
                raise ValueError("coupling must be [n, 3]")
            s.coupling = _ptr(self.coupling)
        self.struct = s
        self.n, self.k = n, k

    @property
    def ref(self):
        return ctypes.byref(self.struct)


def _pixels(W, H, pix):
    if pix is None:
        return None, W * H
    pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int64))
    if pix.size and (pix.min() < 0 or pix.max() >= W * H):
        raise ValueError("pixel index out of range")
    return pix, pix.shape[0]


def psi_map(pts, stroke, mode=MODE_FLOOR, return_floored=False):
    """Backward map psi (Eq. back) of one stroke (cx, cy, th, L, r) on points [n,2]."""
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 2))
    out = np.empty_like(pts)
    fl = np.empty(pts.shape[0], dtype=np.int32)
    _load().orc_map(_ptr(pts), pts.shape[0], *map(float, stroke), 0, int(mode), _ptr(out), _ptr(fl))
    return (out, fl) if return_floored else out


def phi_map(pts, stroke, raw_q=False):
    """Forward map Phi (Eq. fwd) of one stroke on points [n,2]."""
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 2))
    out = np.empty_like(pts)
    _load().orc_map(_ptr(pts), pts.shape[0], *map(float, stroke), 1,
                    MODE_RAWQ if raw_q else MODE_CLAMP, _ptr(out), None)
    return out


def map_jacobian(pts, stroke, direction=0, mode=MODE_FLOOR):
    """[n, 2, 7] Jacobian d(out)/d(x, y, cx, cy, th, L, r) by dual numbers."""
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 2))
    jac = np.empty((pts.shape[0], 2, 7), dtype=np.float64)
    _load().orc_map_jacobian(_ptr(pts), pts.shape[0], *map(float, stroke), int(direction),
                             int(mode), _ptr(jac))
    return jac


TRANSPORTS = {"capsule": 0, "inert": 1, "drops": 2}


def _transport(inert, transport, prog=None):
    t = (1 if inert else 0) if transport is None else TRANSPORTS[transport]
    if t == TRANSPORTS["drops"] and getattr(prog, "coupling", None) is not None:
        raise ValueError("the coupling variant applies to the capsule transport only")
    return t


def drops_map(pts, stroke, direction=0, return_binds=False, return_jacobian=False):
    """The sixteen-drop operator of the transfer renderer R_D on points [n,2]:
    direction 0 = the pull-back psi_D (epsilon-floored), 1 = the forward Phi_D.
    Optionally the per-point floor binds and the 2x2 Jacobians d(out)/d(x, y)."""
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 2))
    out = np.empty_like(pts)
    binds = np.empty(pts.shape[0], dtype=np.int32)
    jac = np.empty((pts.shape[0], 2, 2)) if return_jacobian else None
    _load().orc_map_drops(_ptr(pts), pts.shape[0], *map(float, stroke), int(direction), _ptr(out),
                          _ptr(binds), _ptr(jac))
    res = [out]
    if return_binds:
        res.append(binds)
    if return_jacobian:
        res.append(jac)
    return res[0] if len(res) == 1 else tuple(res)


def coupled_map(pts, stroke, coeffs, direction=0, mode=MODE_CLAMP, return_jacobian=False, return_v=False):
    """The coupling variant (Eq. coupling) of stroke (cx, cy, th, L, r) with the
    profile coeffs (c1, c2, c3) of Eq. profile on points [n,2]: direction 0 =
    psi_g (mode MODE_CLAMP or MODE_FLOOR), 1 = Phi_g.  Optionally the 2x2
    Jacobians d(out)/d(x, y), and the centred coordinate v of each input point
    with the deposit boundary sigma_b(v) there."""
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 2))
    m = pts.shape[0]
    out = np.empty_like(pts)
    jac = np.empty((m, 2, 2)) if return_jacobian else None
    v = np.empty(m) if return_v else None
    sb = np.empty(m) if return_v else None
    _load().orc_map_coupled(_ptr(pts), m, *map(float, stroke), *map(float, coeffs), int(direction), int(mode),
                            _ptr(out), _ptr(jac), _ptr(v), _ptr(sb))
    res = [out]
    if return_jacobian:
        res.append(jac)
    if return_v:
        res += [v, sb]
    return res[0] if len(res) == 1 else tuple(res)


def profile_min(coeffs):
    """min over v of g(v) = 1 + sum_k c_k cos(4 pi k v) (Eq. profile), exact."""
    return float(_load().orc_profile_min(*map(float, coeffs)))


def compensate(prog, endpoint=False, skip_blocked=False):
    """One-pass closed-form compensation of a program (anchor or endpoint
    variant); returns dict cx, cy, theta, length [n] (FP64), blocked [n]."""
    pk = _Packed(prog)
    n = pk.n
    out = {k: np.empty(n) for k in ("cx", "cy", "theta", "length")}
    blocked = np.empty(n, dtype=np.int32)
    _load().orc_compensate(pk.ref, int(bool(endpoint)), int(bool(skip_blocked)), _ptr(out["cx"]), _ptr(out["cy"]),
                           _ptr(out["theta"]), _ptr(out["length"]), _ptr(blocked))
    out["blocked"] = blocked
    return out


def render_hard(prog, W, H, n_prefix=-1, snap=False, inert=False, pix=None, with_kappa=False, transport=None):
    """Hard render; returns dict rgb [m,3], idx [m], margin [m] (+ kappa [m]).
    transport: "capsule" (R_A, default), "inert" (R_U) or "drops" (R_D)."""
    pk = _Packed(prog)
    pix, m = _pixels(W, H, pix)
    rgb = np.empty((m, 3))
    idx = np.empty(m, dtype=np.int32)
    margin = np.empty(m)
    kappa = np.empty(m) if with_kappa else None
    _load().orc_render_hard(pk.ref, W, H, int(n_prefix), int(bool(snap)), _transport(inert, transport, prog),
                            _ptr(pix), m, _ptr(rgb), _ptr(idx), _ptr(margin), _ptr(kappa))
    out = {"rgb": rgb, "idx": idx, "margin": margin}
    if with_kappa:
        out["kappa"] = kappa
    return out


def render_soft(prog, W, H, tau, tau_min, inert=False, pix=None, transport=None, early_exit=0.0):
    """Soft render; returns dict rgb [m,3], T0 [m], nrec [m] (floor binds).
    transport as render_hard.  early_exit > 0 stops a pixel once its
    transmittance falls below that value (T0 is then the T at the exit)."""
    pk = _Packed(prog)
    pix, m = _pixels(W, H, pix)
    rgb = np.empty((m, 3))
    T0 = np.empty(m)
    nrec = np.empty(m, dtype=np.int32)
    _load().orc_render_soft(pk.ref, W, H, float(tau), float(tau_min), _transport(inert, transport, prog),
                            _ptr(pix), m, _ptr(rgb), _ptr(T0), _ptr(nrec), float(early_exit))
    return {"rgb": rgb, "T0": T0, "nrec": nrec}


def soft_jvp(prog, W, H, tau, tau_min, stroke, param, inert=False, pix=None):
    """d rgb / d param of the soft render by forward-mode duals ([m,3])."""
    pk = _Packed(prog)
    pix, m = _pixels(W, H, pix)
    d = np.empty((m, 3))
    _load().orc_soft_jvp(pk.ref, W, H, float(tau), float(tau_min), int(bool(inert)),
                         _ptr(pix), m, int(stroke), int(param), _ptr(d))
    return d


def soft_vjp(prog, W, H, tau, tau_min, cot, inert=False, pix=None):
    """Stored-state adjoint of J = sum cot . R; returns dict of gradients."""
    pk = _Packed(prog)
    pix, m = _pixels(W, H, pix)
    cot = np.ascontiguousarray(np.asarray(cot, dtype=np.float64).reshape(m, 3))
    g_geo = np.empty((pk.n, 5))
    g_col = np.empty((pk.n, 3))
    g_logits = np.empty((pk.n, pk.k))
    g_pal = np.empty((pk.k, 3))
    _load().orc_soft_vjp(pk.ref, W, H, float(tau), float(tau_min), int(bool(inert)), _ptr(pix), m,
                         _ptr(cot), _ptr(g_geo), _ptr(g_col), _ptr(g_logits), _ptr(g_pal))
    return {"cx": g_geo[:, 0], "cy": g_geo[:, 1], "theta": g_geo[:, 2], "length": g_geo[:, 3],
            "half_width": g_geo[:, 4], "color": g_col, "logits": g_logits, "palette": g_pal}


_FIELD = {0: "cx", 1: "cy", 2: "theta", 3: "length", 4: "half_width"}


def fd_gradient(prog, W, H, tau, tau_min, cot, params, h_geo=1e-6, h_logit=1e-5,
                inert=False, pix=None):
    """Central differences of J = sum cot . R_soft with respect to the listed
    parameters, each given as (stroke, param) with param as in ``soft_jvp``
    (palette entries excluded).  A length at 0 uses the second-order one-sided
    difference (-3 J(0) + 4 J(h) - J(2h)) / 2h: the map is even in L, so only
    the one-sided derivative exists there."""
    import copy
    cot = np.asarray(cot, dtype=np.float64).reshape(-1, 3)

    def J(pr):
        return float(np.sum(render_soft(pr, W, H, tau, tau_min, inert, pix)["rgb"] * cot))

    def perturbed(j, q, delta):
        pr = copy.copy(prog)
        if q < 5:
            name = _FIELD[q]
            arr = np.array(getattr(prog, name), dtype=np.float64)
            arr[j] += delta
            setattr(pr, name, arr)
        else:
            arr = np.array(prog.logits, dtype=np.float64)
            arr[j, q - 5] += delta
            pr.logits = arr
        return pr

    out = []
    for (j, q) in params:
        h = h_geo if q < 5 else h_logit
        if q == 3 and float(np.asarray(prog.length)[j]) == 0.0:
            out.append((-3 * J(prog) + 4 * J(perturbed(j, q, h)) - J(perturbed(j, q, 2 * h))) / (2 * h))
        else:
            out.append((J(perturbed(j, q, h)) - J(perturbed(j, q, -h))) / (2 * h))
    return np.array(out)


def count_ops(prog, W, H, tau, tau_min, pix=None, transport="capsule"):
    """Tallied operations per unit (see ``orc_count_ops``): a dict with
    ``hard`` per visited step of the hard render, ``soft`` per pixel-stroke of
    the soft render and, for the capsule map (with or without a coupling
    profile), ``adjoint`` per pixel-stroke of the replay adjoint with its
    parts; each as FP32-pipe and XU operation counts, plus the unit totals.
    transport: "capsule" or "drops" (R_D, forward only)."""
    pk = _Packed(prog)
    pix, m = _pixels(W, H, pix)
    out = np.zeros(14)
    t = TRANSPORTS[transport]
    if _load().orc_count_ops(pk.ref, W, H, float(tau), float(tau_min), t, _ptr(pix), m, _ptr(out)) != 0:
        raise ValueError("operation counts cover the capsule map (optionally coupled) and R_D")
    steps, ps = out[0], out[3]
    res = {
        "hard": {"fp32": out[1] / steps, "xu": out[2] / steps, "visited_steps": steps, "pixels": m},
        "soft": {"fp32": out[4] / ps, "xu": out[5] / ps, "pixel_strokes": ps},
    }
    if transport == "capsule":
        parts = {"regeneration": (out[6], out[7]), "coverage": (out[8], out[9]),
                 "reverse_sweep": (out[10], out[11]), "scalar_step": (out[12], out[13])}
        adj = {k: {"fp32": f / ps, "xu": x / ps} for k, (f, x) in parts.items()}
        res["adjoint"] = {"fp32": sum(v["fp32"] for v in adj.values()), "xu": sum(v["xu"] for v in adj.values()),
                          "parts": adj, "pixel_strokes": ps}
    return res
