#!/usr/bin/env python3
"""Generates tbr_poly.h: polynomial approximations used by the kernels on the
folded argument ranges they need, so no range reduction is required.

  atan(z)       z in [0, 1]        z * A(z^2)          (relative error)
  sin(d)        |d| <= pi/2        d * S(d^2)          (relative error)
  1 - cos(d)    |d| <= pi/2        d^2 * K(d^2)        (relative error)

Method: a discrete minimax fit (Lawson's iteratively reweighted least squares,
C. L. Lawson, "Contributions to the theory of linear least maximum
approximation", 1961) of the relative error on dense Chebyshev-distributed
samples, solved in float64 with numpy, then evaluated (float64 and a float32
Horner emulation) to report the achieved maximum relative error.  The header
records those bounds next to the coefficients.

  python gen_poly.py > tbr_poly.h
"""
import math

import numpy as np


def lawson_fit(u, target, weight, degree, iters=200):
    """Minimise max_i weight_i * |sum_k c_k u_i^k - target_i| over c."""
    V = np.vander(u, degree + 1, increasing=True)
    w = np.full(u.shape, 1.0 / u.size)
    c = None
    for _ in range(iters):
        sw = np.sqrt(w) * weight
        c, *_ = np.linalg.lstsq(V * sw[:, None], target * sw, rcond=None)
        err = np.abs(V @ c - target) * weight
        w = w * err
        s = w.sum()
        if s == 0:
            break
        w /= s
    return c


def cheb_nodes(a, b, m):
    k = np.arange(m)
    x = np.cos((2 * k + 1) * np.pi / (2 * m))
    return np.sort(0.5 * (a + b) + 0.5 * (b - a) * x)


def horner32(c, u):
    u = u.astype(np.float32)
    acc = np.full(u.shape, np.float32(c[-1]))
    for ck in c[-2::-1]:
        acc = (acc * u + np.float32(ck)).astype(np.float32)
    return acc


def fit_atan(deg):
    z = cheb_nodes(0.0, 1.0, 4000)
    u = z * z
    target = np.where(z > 0, np.arctan(z) / np.where(z > 0, z, 1), 1.0)
    c = lawson_fit(u, target, np.ones_like(u), deg)
    zz = np.linspace(1e-6, 1.0, 200001)
    approx = zz * np.polyval(c[::-1], zz * zz)
    rel = np.max(np.abs(approx - np.arctan(zz)) / np.arctan(zz))
    a32 = zz.astype(np.float32) * horner32(c, (zz * zz).astype(np.float32))
    rel32 = np.max(np.abs(a32 - np.arctan(zz)) / np.arctan(zz))
    return c, rel, rel32


def fit_sin(deg):
    d = cheb_nodes(0.0, math.pi / 2, 4000)
    u = d * d
    target = np.sin(d) / d
    c = lawson_fit(u, target, np.ones_like(u), deg)
    dd = np.linspace(1e-6, math.pi / 2, 200001)
    approx = dd * np.polyval(c[::-1], dd * dd)
    rel = np.max(np.abs(approx - np.sin(dd)) / np.sin(dd))
    a32 = dd.astype(np.float32) * horner32(c, (dd * dd).astype(np.float32))
    rel32 = np.max(np.abs(a32 - np.sin(dd)) / np.sin(dd))
    return c, rel, rel32


def fit_omc(deg):
    d = cheb_nodes(0.0, math.pi / 2, 4000)
    u = d * d
    ref = 2.0 * np.sin(0.5 * d) ** 2
    target = ref / u
    c = lawson_fit(u, target, np.ones_like(u), deg)
    dd = np.linspace(1e-6, math.pi / 2, 200001)
    ref2 = 2.0 * np.sin(0.5 * dd) ** 2
    approx = dd * dd * np.polyval(c[::-1], dd * dd)
    rel = np.max(np.abs(approx - ref2) / ref2)
    u32 = (dd * dd).astype(np.float32)
    a32 = u32 * horner32(c, u32)
    rel32 = np.max(np.abs(a32 - ref2) / ref2)
    return c, rel, rel32


def emit(name, c, rel, rel32, what):
    lines = [f"// {what}: max relative error {rel:.2e} (float64 evaluation), "
             f"{rel32:.2e} (float32 Horner)"]
    lines.append(f"constexpr int k{name}Deg = {len(c) - 1};")
    coeffs = ", ".join(f"{float(v):.9e}f" for v in c)
    lines.append(f"__device__ constexpr float k{name}[{len(c)}] = {{{coeffs}}};")
    return "\n".join(lines)


def main():
    ca, ra, ra32 = fit_atan(7)
    cs, rs, rs32 = fit_sin(4)
    co, ro, ro32 = fit_omc(4)
    print("// Generated by gen_poly.py -- do not edit by hand.")
    print("// Discrete minimax (Lawson) fits of the relative error on the folded ranges")
    print("// the kernels need; coefficients in increasing powers of u = x^2.")
    print("#pragma once")
    print()
    print("namespace tbr {")
    print()
    print(emit("Atan", ca, ra, ra32, "atan(z) ~ z * A(z^2), z in [0, 1]"))
    print()
    print(emit("Sin", cs, rs, rs32, "sin(d) ~ d * S(d^2), |d| <= pi/2"))
    print()
    print(emit("Omc", co, ro, ro32, "1 - cos(d) ~ d^2 * K(d^2), |d| <= pi/2"))
    print()
    print("}  // namespace tbr")


if __name__ == "__main__":
    main()
