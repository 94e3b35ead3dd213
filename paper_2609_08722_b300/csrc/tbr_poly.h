// Generated by gen_poly.py -- do not edit by hand.
// Discrete minimax (Lawson) fits of the relative error on the folded ranges
// the kernels need; coefficients in increasing powers of u = x^2.
#pragma once

namespace tbr {

// atan(z) ~ z * A(z^2), z in [0, 1]: max relative error 1.13e-07 (float64 evaluation), 2.63e-07 (float32 Horner)
constexpr int kAtanDeg = 7;
__device__ constexpr float kAtan[8] = {9.999999115e-01f, -3.333209391e-01f, 1.997137959e-01f, -1.402944137e-01f, 9.942812869e-02f, -5.990542961e-02f, 2.455760621e-02f, -4.780585124e-03f};

// sin(d) ~ d * S(d^2), |d| <= pi/2: max relative error 6.70e-09 (float64 evaluation), 1.75e-07 (float32 Horner)
constexpr int kSinDeg = 4;
__device__ constexpr float kSin[5] = {9.999999957e-01f, -1.666665799e-01f, 8.333051102e-03f, -1.980907740e-04f, 2.605228711e-06f};

// 1 - cos(d) ~ d^2 * K(d^2), |d| <= pi/2: max relative error 8.84e-10 (float64 evaluation), 1.42e-07 (float32 Horner)
constexpr int kOmcDeg = 4;
__device__ constexpr float kOmc[5] = {4.999999996e-01f, -4.166665939e-02f, 1.388865232e-03f, -2.477462307e-05f, 2.629839132e-07f};

}  // namespace tbr
