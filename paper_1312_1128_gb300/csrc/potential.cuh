// potential.cuh -- the lensing potential psi of each component (Eq. alpha:
// alpha = grad psi; Eq. timedelay: delta t = |alpha|^2 / 2 - psi), in the
// working precision, for the potential walk (psi.cu).
//
// For an axisymmetric component psi(r) = psi(r_e) - int_r^{r_e} Mt(r')/r' dr'
// with Mt the enclosed m-unit mass; outside its support a finite component
// is a point mass, psi = m ln r, which fixes the additive constant:
//   point (softened within r0):  m ln r;  inside r0: m (ln r0 + (r^2/r0^2 - 1)/2)
//   truncated Gaussian (u = c r^2, U = q^2/2, N = 1 - e^-U):
//       inside  m ln(q sigma) - m/(2N) (Ein(U) - Ein(u)),
//       Ein(u) = int_0^u (1 - e^-t)/t dt
//   projected NFW (x = r/r_s, X = R_max/r_s, A = m/g(X)):
//       inside  m ln R_max - A (H(X) - H(x)),  H = ln^2(x/2)/2 - (1 - x^2) F^2/2
//   SIS: r_E r;  uniform disk: as the softened point with r0 = R.
// A far cell (monopole + quadrupole about its centre of mass, w = z - z_cm):
//   psi = M ln|w| - Re(Q2 / (2 w^2)).
#pragma once

#include "profiles.cuh"

namespace lens {

constexpr double kEulerGamma = 0.57721566490153286061;

// coefficient of u^(k+1) in Ein(u): (-1)^k / ((k+1) (k+1)!)
LENS_HD constexpr double ein_coef(int k)
{
    double f = 1.0;
    for (int j = 2; j <= k + 1; ++j) f *= j;
    return ((k & 1) ? -1.0 : 1.0) / ((k + 1) * f);
}

// Horner over the coefficients k = K-1 .. 0, each a compile-time constant
template <typename T, int K, int k> LENS_HD T ein_horner(T u, T s)
{
    if constexpr (k < 0) {
        return s;
    } else {
        constexpr T c = T(ein_coef(k));
        return ein_horner<T, K, k - 1>(u, fma(s, u, c));
    }
}

// Ein(u) = sum_k>=1 (-1)^(k+1) u^k / (k k!): the series by Horner on its
// coefficients for u < 5 (20 terms in FP32, 34 in FP64: below 6 ulp on
// [0, 5]; a truncated Gaussian with q <= 3.16 never leaves this branch), else
// E1(u) + ln u + gamma with E1 from its continued fraction (modified Lentz;
// 8 steps in FP32, 20 in FP64 suffice from u = 5 on).
template <typename T> LENS_HD T ein(T u)
{
    if (u < T(5)) {
        constexpr int K = sizeof(T) == 4 ? 20 : 34;
        constexpr T top = T(ein_coef(K - 1));
        return ein_horner<T, K, K - 2>(u, top) * u;
    }
    const int N = sizeof(T) == 4 ? 8 : 20;
    T b = u + T(1), cc = T(1e30), d = T(1) / b, h = d;
    for (int i = 1; i < N; ++i) {
        const T an = -T(i) * T(i);
        b += T(2);
        d = T(1) / (an * d + b);
        cc = b + an / cc;
        h *= cc * d;
    }
    return h * exp(-u) + log(u) + T(kEulerGamma);
}

// Ein on [0, 4.5] (truncated Gaussians with q <= 3): Ein(u) = u p(u - 9/4),
// p of degree 9 interpolating Ein(u)/u at the Chebyshev nodes of [0, 4.5]
// (coefficients by gen_ein_poly.py from 40-digit quadrature of the
// definition); within 2.1e-7 of Ein there in FP32, as the series.
LENS_HD constexpr double ein_cheb_coef(int k)
{
    switch (k) {
        case 0: return 6.3240353766460487812e-1;
        case 1: return -1.0435697376997954498e-1;
        case 2: return 1.7521483101271278799e-2;
        case 3: return -2.7063436946789297185e-3;
        case 4: return 3.7667792743572055091e-4;
        case 5: return -4.7141933700249675007e-5;
        case 6: return 5.3065068463045642612e-6;
        case 7: return -5.4535985953828259233e-7;
        case 8: return 5.5981593702543123488e-8;
        default: return -4.7716717058873290062e-9;
    }
}
constexpr double kEinChebMax = 4.5;

// NFW potential shape H(x) (H(0) = 0) from F(x) and g(x) = ln(x/2) + F(x) of
// nfw_Ffg; the cancellation-free form below 1/2, H = -e (2L + e)/2 with
// L = ln(2/x), e = log1p(-x^2 / (2 (1 + sqrt(1 - x^2)))).
template <typename T> LENS_DEV T nfw_H_Fg(T x, T F, T g)
{
    if (x <= T(0)) return T(0);
    if (x < T(0.5)) {
        const T t = sqrt(T(1) - x * x), L = log(T(2) / x);
        const T e = log1p(-x * x / (T(2) * (T(1) + t)));
        return T(-0.5) * e * (T(2) * L + e);
    }
    const T lx = g - F;
    return T(0.5) * lx * lx - T(0.5) * (T(1) - x * x) * F * F;
}

template <typename T> LENS_DEV T nfw_H(T x)
{
    if (x <= T(0)) return T(0);
    T F = T(0), f, g = T(0);
    if (x >= T(0.5)) nfw_Ffg(x, F, f, g);
    return nfw_H_Fg(x, F, g);
}

// Point mass softened within r0 (r0sq = 0: none): psi and kb = Mt / r^2.
template <typename T> LENS_DEV void psi_point(T m, T r2, T r0sq, T& psi, T& kb)
{
    if (r2 >= r0sq) {
        psi = r2 > T(0) ? T(0.5) * m * log(r2) : T(0);
        kb = r2 > T(0) ? m * rcp(r2) : T(0);
    } else {
        const T i0 = rcp(r0sq);
        psi = m * (T(0.5) * log(r0sq) + T(0.5) * fma(r2, i0, T(-1)));
        kb = m * i0;
    }
}

// Truncated Gaussian (c = 1/(2 sigma^2); EinU = Ein(Uq)).
template <typename T> LENS_DEV void psi_gauss(T m, T c, T r2, T Uq, T invNq, T EinU, T& psi, T& kb)
{
    const T u = r2 * c;
    if (u < Uq) {
        psi = T(0.5) * m * log(Uq / c) - T(0.5) * m * invNq * (EinU - ein(u));
        T kap, Dp;
        gauss_terms(m, c, r2, Uq, invNq, kb, kap, Dp);
    } else {
        psi = T(0.5) * m * log(r2);
        kb = m * rcp(r2);
    }
}

// Projected NFW truncated at R_max (R2 = R_max^2, A = m/g(X), B = 1/r_s,
// HX = H(X)).
template <typename T> LENS_DEV void psi_nfw(T m, T R2, T A, T B, T HX, T r2, T& psi, T& kb)
{
    if (r2 < R2 && r2 > T(0)) {
        const T x = sqrt(r2) * B;
        T F, f, g;
        nfw_Ffg(x, F, f, g);
        psi = T(0.5) * m * log(R2) - A * (HX - nfw_H_Fg(x, F, g));
        kb = A * g * rcp(r2);
    } else if (r2 > T(0)) {
        psi = T(0.5) * m * log(r2);
        kb = m * rcp(r2);
    } else {
        psi = T(0.5) * m * log(R2) - A * HX;
        kb = T(0);
    }
}

// Far cell: psi and alpha of the monopole + quadrupole at w = (wx, wy).
template <typename T> LENS_DEV void psi_cell(T wx, T wy, T M, T qr, T qi, T& psi, T& a1, T& a2)
{
    const T r2 = fma(wx, wx, wy * wy), inv = rcp(r2);
    const T c2 = fma(wx, wx, -wy * wy), s2 = (wx + wx) * wy;
    psi = T(0.5) * M * log(r2) - T(0.5) * (qr * c2 + qi * s2) * inv * inv;
    // conj(alpha) = M/w + Q2/w^3, with u = 1/w
    const T ux = wx * inv, uy = -wy * inv;
    const T u2x = fma(ux, ux, -uy * uy), u2y = (ux + ux) * uy;
    const T u3x = fma(u2x, ux, -u2y * uy), u3y = fma(u2x, uy, u2y * ux);
    a1 = fma(M, ux, fma(qr, u3x, -qi * u3y));
    a2 = -fma(M, uy, fma(qr, u3y, qi * u3x));
}

}  // namespace lens
