// profiles.cuh -- per-interaction lensing kernels on the device.
//
// Every particle kind is axisymmetric about its centre, so its contribution
// at offset w = ray - centre (r^2 = |w|^2) is written as
//     alpha += kb * w,   kappa += kap,   gamma -= Dp * (wx^2 - wy^2, 2 wx wy)
// with kb = Mt(<r)/r^2 the mean convergence inside r, kap the convergence at r
// and Dp = (kb - kap)/r^2 (Sec. 3.2, Eqs. alpha-gamma_2 for a circular lens:
// gamma = -(kb - kappa) e^{2 i phi}).  Masses are in m-units (pi Sigma_crit = 1,
// so a point mass has kb = m / r^2, Sec. 3.5).
//
// Far cells use the complex multipole form (Sec. 3.2 monopole + quadrupole):
// conj(alpha) = M/w + Q2/w^3, conj(gamma) = -M/w^2 - 3 Q2/w^4, kappa = 0.
#pragma once

#include "common.cuh"

namespace lens {

template <typename T> LENS_DEV T rcp(T x);
template <> LENS_DEV float rcp<float>(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <> LENS_DEV double rcp<double>(double x) { return 1.0 / x; }

LENS_DEV float expneg(float u) { return __expf(-u); }
LENS_DEV double expneg(double u) { return exp(-u); }

// Five accumulators per ray.
template <typename T> struct Acc5 {
    T a1, a2, k, g1, g2;
    LENS_DEV void zero() { a1 = a2 = k = g1 = g2 = T(0); }
    template <bool AO> LENS_DEV void radial(T wx, T wy, T kb, T kap, T Dp)
    {
        a1 = fma(kb, wx, a1);
        a2 = fma(kb, wy, a2);
        if (!AO) {
            k += kap;
            T c2 = fma(wx, wx, -wy * wy);
            T s2 = (wx + wx) * wy;
            g1 = fma(-Dp, c2, g1);
            g2 = fma(-Dp, s2, g2);
        }
    }
};

// Neumaier-compensated total of a sequence of partial sums.
template <typename T> struct Comp5 {
    T s[5], c[5];
    LENS_DEV void zero()
    {
#pragma unroll
        for (int q = 0; q < 5; ++q) s[q] = c[q] = T(0);
    }
    LENS_DEV static void add1(T& s, T& c, T v)
    {
        T t = s + v;
        if (fabs(s) >= fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    LENS_DEV void add(const Acc5<T>& p)
    {
        add1(s[0], c[0], p.a1);
        add1(s[1], c[1], p.a2);
        add1(s[2], c[2], p.k);
        add1(s[3], c[3], p.g1);
        add1(s[4], c[4], p.g2);
    }
    LENS_DEV T get(int q) const { return s[q] + c[q]; }
};

// ----------------------------------------------------------- point mass
// Sec. 3.5 star deflection; kappa = 0 off the mass; a ray exactly on the mass
// gets nothing from it.  r2s >= r2 is the softened square radius used for a
// listed particle inside a leaf (equal to r2 wherever it matters, see walk).
template <typename T> LENS_DEV void point_terms(T m, T r2s, T& kb, T& Dp)
{
    T inv = r2s > T(0) ? rcp(r2s) : T(0);
    kb = m * inv;
    Dp = kb * inv;
}

// --------------------------------------------- truncated 2D Gaussian
// Sec. 3.1 Eq. smoothing and Sec. 3.2 smoothed-particle deflection (exponent
// r^2 / (2 r_sm^2)).  With u = r^2 c, c = 1/(2 r_sm^2), inside the support:
//   kb = m c h1(u)/N_q,  kap = m c e^-u / N_q,  kb - kap = m c g(u)/N_q,
//   h1 = (1 - e^-u)/u,   g = h1 - e^-u = [1 - e^-u (1 + u)]/u.
// Both are cancellation-prone for small u; their Taylor series are used there:
//   h1 = sum_k (-u)^k/(k+1)!,   g = sum_{n>=1} (-1)^(n+1) n u^n/(n+1)!.
LENS_DEV void gauss_h1_g(float u, float e, float& h1, float& g)
{
    if (u < 0.5f) {
        h1 = fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u,
             -1.0f / 3628800, 1.0f / 362880), -1.0f / 40320), 1.0f / 5040), -1.0f / 720),
             1.0f / 120), -1.0f / 24), 1.0f / 6), -0.5f), 1.0f);
        g = u * fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u,
            1.0f / 403200, -1.0f / 45360), 1.0f / 5760), -1.0f / 840), 1.0f / 144),
            -1.0f / 30), 1.0f / 8), -1.0f / 3), 0.5f);
    } else {
        h1 = (1.0f - e) * rcp(u);
        g = h1 - e;
    }
}
LENS_DEV void gauss_h1_g(double u, double e, double& h1, double& g)
{
    if (u < 0.05) {
        h1 = fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u,
             -1.0 / 3628800, 1.0 / 362880), -1.0 / 40320), 1.0 / 5040), -1.0 / 720),
             1.0 / 120), -1.0 / 24), 1.0 / 6), -0.5), 1.0);
        g = u * fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u,
            1.0 / 403200, -1.0 / 45360), 1.0 / 5760), -1.0 / 840), 1.0 / 144),
            -1.0 / 30), 1.0 / 8), -1.0 / 3), 0.5);
    } else {
        h1 = -expm1(-u) / u;
        g = h1 - e;
    }
}

// Exact Gaussian terms for a particle with c > 0 (c = 1/(2 r_sm^2)); outside
// the support q r_sm (u >= q^2/2) it is a point mass.
template <typename T>
LENS_DEV void gauss_terms(T m, T c, T r2, T Uq, T invNq, T& kb, T& kap, T& Dp)
{
    T u = r2 * c;
    T inv = r2 > T(0) ? rcp(r2) : T(0);
    if (u < Uq) {
        T e = expneg(u), h1, g;
        gauss_h1_g(u, e, h1, g);
        T mcn = m * c * invNq;
        kb = mcn * h1;
        kap = mcn * e;
        Dp = (mcn * g) * inv;
    } else {
        kb = m * inv;
        kap = T(0);
        Dp = kb * inv;
    }
}

// ------------------------------------------------------- projected NFW
// Sec. 3.2 analytic halo; projected NFW truncated in 2D at R_max, a point mass
// outside.  With x = r/r_s, A = m / g(X) (X = R_max/r_s), B = 1/r_s:
//   Mt = A g(x),  kap = A B^2 f(x)/2,  F = arccosh(1/x)/sqrt(1-x^2) (x<1),
//   arccos(1/x)/sqrt(x^2-1) (x>1),  f = (1 - F)/(x^2 - 1),  g = ln(x/2) + F.
// With u = 1 - x^2 both F and f are power series in u:
//   F = sum_k u^k/(2k+1),  f = sum_k u^k/(2k+3)  (|u| < 1),
// used near x = 1.  For x < 1 the closed form is rewritten with t = sqrt(u):
//   F = ln((1+t)/x)/t,  g = [log1p(-x^2/(2(1+t))) + x^2 ln(2/x)/(1+t)]/t,
// which keeps full precision as x -> 0; for x > 1, t = sqrt(-u), F = atan(t)/t.
template <typename T> LENS_DEV void nfw_Ffg(T x, T& F, T& f, T& g);

LENS_DEV void nfw_Ffg(float x, float& F, float& f, float& g)
{
    float x2 = x * x, u = 1.0f - x2;
    if (fabsf(u) < 0.2f) {
        float sF = 0.0f, sf = 0.0f;
#pragma unroll
        for (int k = 10; k >= 0; --k) {
            sF = fmaf(sF, u, 1.0f / (2 * k + 1));
            sf = fmaf(sf, u, 1.0f / (2 * k + 3));
        }
        F = sF;
        f = sf;
        g = logf(0.5f * x) + F;
    } else if (u > 0.0f) {
        float t = sqrtf(u), op = 1.0f + t;
        F = logf(op / x) / t;
        g = (log1pf(-x2 / (2.0f * op)) + x2 * logf(2.0f / x) / op) / t;
        f = (F - 1.0f) / u;
    } else {
        float t = sqrtf(-u);
        F = atanf(t) / t;
        g = logf(0.5f * x) + F;
        f = (F - 1.0f) / u;
    }
}
LENS_DEV void nfw_Ffg(double x, double& F, double& f, double& g)
{
    double x2 = x * x, u = 1.0 - x2;
    if (fabs(u) < 0.02) {
        double sF = 0.0, sf = 0.0;
#pragma unroll
        for (int k = 12; k >= 0; --k) {
            sF = fma(sF, u, 1.0 / (2 * k + 1));
            sf = fma(sf, u, 1.0 / (2 * k + 3));
        }
        F = sF;
        f = sf;
        g = log(0.5 * x) + F;
    } else if (u > 0.0) {
        double t = sqrt(u), op = 1.0 + t;
        F = log(op / x) / t;
        g = (log1p(-x2 / (2.0 * op)) + x2 * log(2.0 / x) / op) / t;
        f = (F - 1.0) / u;
    } else {
        double t = sqrt(-u);
        F = atan(t) / t;
        g = log(0.5 * x) + F;
        f = (F - 1.0) / u;
    }
}

template <typename T>
LENS_DEV void nfw_terms(T m, T R2, T A, T B, T r2, T& kb, T& kap, T& Dp)
{
    T inv = r2 > T(0) ? rcp(r2) : T(0);
    if (r2 < R2 && r2 > T(0)) {
        T x = sqrt(r2) * B, F, f, g;
        nfw_Ffg(x, F, f, g);
        kb = A * g * inv;
        kap = T(0.5) * A * f * B * B;
        Dp = (kb - kap) * inv;
    } else {
        kb = m * inv;
        kap = T(0);
        Dp = kb * inv;
    }
}

// ---------------------------------------------------------- far cells
template <typename T, bool AO>
LENS_DEV void cell_terms(Acc5<T>& acc, T wx, T wy, T M, T qr, T qi)
{
    T r2 = fma(wx, wx, wy * wy);
    T inv = rcp(r2);
    T ux = wx * inv, uy = -wy * inv;                 // u = 1/w
    T u2x = fma(ux, ux, -uy * uy), u2y = (ux + ux) * uy;
    T u3x = fma(u2x, ux, -u2y * uy), u3y = fma(u2x, uy, u2y * ux);
    // conj(alpha) = M u + Q2 u^3
    acc.a1 = fma(M, ux, fma(qr, u3x, fma(-qi, u3y, acc.a1)));
    acc.a2 = fma(-M, uy, fma(-qr, u3y, fma(-qi, u3x, acc.a2)));
    if (!AO) {
        T u4x = fma(u2x, u2x, -u2y * u2y), u4y = (u2x + u2x) * u2y;
        T q3r = T(3) * qr, q3i = T(3) * qi;
        // conj(gamma) = -M u^2 - 3 Q2 u^4
        acc.g1 = fma(-M, u2x, fma(-q3r, u4x, fma(q3i, u4y, acc.g1)));
        acc.g2 = fma(M, u2y, fma(q3r, u4y, fma(q3i, u4x, acc.g2)));
    }
}

}  // namespace lens
