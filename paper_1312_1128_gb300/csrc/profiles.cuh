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
    if (u < 0.25f) {
        h1 = fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u,
             -1.0f / 40320, 1.0f / 5040), -1.0f / 720), 1.0f / 120), -1.0f / 24), 1.0f / 6), -0.5f), 1.0f);
        g = u * fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u,
            -1.0f / 45360, 1.0f / 5760), -1.0f / 840), 1.0f / 144), -1.0f / 30), 1.0f / 8), -1.0f / 3), 0.5f);
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

// Same h1, g with 1/u supplied (inv_u = 1/(r^2 c)), so the direct branch
// needs no reciprocal of its own.
LENS_DEV void gauss_h1_g_inv(float u, float e, float inv_u, float& h1, float& g)
{
    if (u < 0.25f) {
        h1 = fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u,
             -1.0f / 40320, 1.0f / 5040), -1.0f / 720), 1.0f / 120), -1.0f / 24), 1.0f / 6), -0.5f), 1.0f);
        g = u * fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u,
            -1.0f / 45360, 1.0f / 5760), -1.0f / 840), 1.0f / 144), -1.0f / 30), 1.0f / 8), -1.0f / 3), 0.5f);
    } else {
        h1 = (1.0f - e) * inv_u;
        g = h1 - e;
    }
}
LENS_DEV void gauss_h1_g_inv(double u, double e, double inv_u, double& h1, double& g)
{
    (void)inv_u;
    gauss_h1_g(u, e, h1, g);
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

// Gaussian big-list correction in base-2 form, FP32: with t = r^2 c log2(e)
// (c' = c log2 e stored per particle) e^-u = 2^-t costs one ex2, and the
// small-u series above are rewritten in t (u = t ln 2):
//   h1 = sum_k (-ln2)^k t^k/(k+1)!,   g = t sum_j b_j ln2^(j+1) t^j,
// b = {1/2, -1/3, 1/8, -1/30, 1/144, -1/840, 1/5760, -1/45360}; u < 1/4
// becomes t < 1/(4 ln 2).
namespace gser {
constexpr double L = 0.69314718055994530942;
constexpr float kTSeries = (float)(0.25 / L);
constexpr float h(int k, double fact, int sgn)
{
    double p = 1.0;
    for (int i = 0; i < k; ++i) p *= L;
    return (float)(sgn * p / fact);
}
constexpr float gco(int j, double b)
{
    double p = 1.0;
    for (int i = 0; i <= j; ++i) p *= L;
    return (float)(b * p);
}
constexpr float H0 = 1.0f, H1 = h(1, 2.0, -1), H2 = h(2, 6.0, 1), H3 = h(3, 24.0, -1), H4 = h(4, 120.0, 1),
                H5 = h(5, 720.0, -1), H6 = h(6, 5040.0, 1), H7 = h(7, 40320.0, -1);
constexpr float G0 = gco(0, 1.0 / 2), G1 = gco(1, -1.0 / 3), G2 = gco(2, 1.0 / 8), G3 = gco(3, -1.0 / 30),
                G4 = gco(4, 1.0 / 144), G5 = gco(5, -1.0 / 840), G6 = gco(6, 1.0 / 5760),
                G7 = gco(7, -1.0 / 45360);
}  // namespace gser

LENS_DEV float exp2neg(float t)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-t));
    return r;
}
LENS_DEV double exp2neg(double t) { return exp2(-t); }

// Correction (full truncated Gaussian - softened point) at offset w, for an
// entry that some ray of the group approaches within its softening radius.
// q = {., ., s^2, 1/r0^2}, q1 = {m/N_q, c log2 e, m c / N_q, 1/c};
// Uq2 = q^2/2 log2 e.
// Outside the support both terms are the same point mass: the result is 0.
template <bool AO>
LENS_DEV void gauss_correction(Acc5<float>& acc, float wx, float wy, const float4& q, const float4& q1,
                               float Uq2, float Nq)
{
    using namespace gser;
    float r2 = fmaf(wx, wx, wy * wy);
    float inv = r2 > 0.0f ? rcp(r2) : 0.0f;
    float inv_s = fminf(inv, q.w);
    float kbp = (q1.x * Nq) * inv_s;
    float t = r2 * q1.y;
    float e = exp2neg(t);
    float h1, g;
    if (t < kTSeries) {
        h1 = fmaf(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, H7, H6), H5), H4), H3), H2), H1), H0);
        g = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, G7, G6), G5), G4), G3), G2), G1), G0);
    } else {
        h1 = (1.0f - e) * (inv * q1.w);
        g = h1 - e;
    }
    bool in = t < Uq2;
    float dkb = in ? fmaf(q1.z, h1, -kbp) : 0.0f;
    float kap = in ? q1.z * e : 0.0f;
    float dDp = in ? fmaf(q1.z * g, inv, -kbp * inv_s) : 0.0f;
    acc.template radial<AO>(wx, wy, dkb, kap, dDp);
}

// The same correction when no ray of the group is inside the softening
// radius (decided per entry when it is queued), written without cancellation:
// with Mt(<r) = m (1 - e^-min(u, q^2/2)) / N_q (a point mass m outside),
//   kb_exact - kb_point = (m/N_q)(1/r^2)(e^-q^2/2 - e^-min(u, q^2/2)),
// exactly 0 outside the support and well conditioned as u -> 0 (no series,
// no branch); kappa = m c e^-u / N_q inside, 0 outside; for the shear
// D = kb - kappa, so D_exact - D_point = (kb_exact - kb_point) - kappa.
// q1 = {m/N_q, c log2 e, m c / N_q, 1/c}; Uq2 = q^2/2 log2 e; eU = e^-q^2/2.
template <bool AO>
LENS_DEV void gauss_correction_fast(Acc5<float>& acc, float wx, float wy, const float4& q1, float Uq2,
                                    float eU)
{
    float r2 = fmaf(wx, wx, wy * wy);
    float inv = rcp(r2);
    float t = r2 * q1.y;
    float e = exp2neg(fminf(t, Uq2));
    float dkb = (q1.x * inv) * (eU - e);
    float kap = t < Uq2 ? q1.z * e : 0.0f;
    acc.template radial<AO>(wx, wy, dkb, kap, (dkb - kap) * inv);
}
// The same when, in addition, the support contains every ray of the group:
// no select for the support edge, and kappa accumulates with one FMA.
template <bool AO>
LENS_DEV void gauss_correction_inside(Acc5<float>& acc, float wx, float wy, const float4& q1, float eU)
{
    float wy2 = wy * wy;
    float r2 = fmaf(wx, wx, wy2);
    float inv = rcp(r2);
    float e = exp2neg(r2 * q1.y);
    float dkb = (q1.x * inv) * (eU - e);
    acc.a1 = fmaf(dkb, wx, acc.a1);
    acc.a2 = fmaf(dkb, wy, acc.a2);
    if (!AO) {
        acc.k = fmaf(q1.z, e, acc.k);
        float Dp = fmaf(-q1.z, e, dkb) * inv;
        float c2 = fmaf(wx, wx, -wy2), s2 = (wx + wx) * wy;
        acc.g1 = fmaf(-Dp, c2, acc.g1);
        acc.g2 = fmaf(-Dp, s2, acc.g2);
    }
}
template <bool AO>
LENS_DEV void gauss_correction_fast(Acc5<double>& acc, double wx, double wy, const dbl4& q1, double Uq2,
                                    double eU)
{
    const double L = 0.69314718055994530942;
    double r2 = fma(wx, wx, wy * wy);
    double inv = 1.0 / r2;
    double t = r2 * q1.y;
    double e = exp(-fmin(t, Uq2) * L);
    double dkb = (q1.x * inv) * (eU - e);
    double kap = t < Uq2 ? q1.z * e : 0.0;
    acc.template radial<AO>(wx, wy, dkb, kap, (dkb - kap) * inv);
}

template <bool AO>
LENS_DEV void gauss_correction_inside(Acc5<double>& acc, double wx, double wy, const dbl4& q1, double eU)
{
    gauss_correction_fast<AO>(acc, wx, wy, q1, INFINITY, eU);
}

// Two big-list entries of the same ray at once, in packed FP32x2 arithmetic
// (one instruction issues both halves).  The closed form above, for entries
// that no ray of the group reaches inside the softening radius; EDGE selects
// the form with the support edge (clamped exponent, kappa 0 outside), else
// every ray lies inside both supports.  Operands are pairs over the two
// entries: nx, ny = minus the entry positions, cl = -c log2 e, kz = m c/N_q,
// mN = m/N_q, nmE = -(m/N_q) e^-q^2/2; lx, ly = the ray's position in both
// halves; nUq2 = -q^2/2 log2 e.  With P = kappa - dkb (= -dD r^2):
//   -dkb = ((m/N_q) e - (m/N_q) eU)/r^2,   -dD = P/r^2,
//   -alpha += -dkb w,  gamma1 = sum P - 2 sum (-dD) wy^2 (= sum -dD (wx^2 - wy^2)),
//   gamma2/2 = sum -dD wx wy,
// so every update is one FMA or add; the halves are summed when the buffer
// is folded.  Accumulators: na1, na2 = -alpha; k = kappa; g1p = sum P;
// g1y = sum -dD wy^2; hg2 = gamma2/2.
struct Acc5x2 {
    float2 na1, na2, k, g1p, g1y, hg2;
    LENS_DEV void zero()
    {
        na1 = na2 = k = g1p = g1y = hg2 = make_float2(0.0f, 0.0f);
    }
};

LENS_DEV float exp2_approx(float t)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
    return r;
}

template <bool AO, bool EDGE>
LENS_DEV void gauss_correction_x2(Acc5x2& acc, float2 lx, float2 ly, float2 nx, float2 ny, float2 cl, float2 mN,
                                  float2 nmE, float2 kz, float nUq2)
{
    float2 wx = __fadd2_rn(lx, nx);
    float2 wy = __fadd2_rn(ly, ny);
    float2 wyy = __fmul2_rn(wy, wy);
    float2 r2 = __ffma2_rn(wx, wx, wyy);
    float2 t = __fmul2_rn(r2, cl);
    float2 tc = t;
    if (EDGE) {
        tc.x = fmaxf(t.x, nUq2);
        tc.y = fmaxf(t.y, nUq2);
    }
    float2 e = make_float2(exp2_approx(tc.x), exp2_approx(tc.y));
    float2 inv = make_float2(rcp(r2.x), rcp(r2.y));
    float2 ndkb = __fmul2_rn(__ffma2_rn(mN, e, nmE), inv);
    acc.na1 = __ffma2_rn(ndkb, wx, acc.na1);
    acc.na2 = __ffma2_rn(ndkb, wy, acc.na2);
    if (!AO) {
        float2 ek = e;
        if (EDGE) {
            ek.x = t.x > nUq2 ? e.x : 0.0f;
            ek.y = t.y > nUq2 ? e.y : 0.0f;
        }
        acc.k = __ffma2_rn(kz, ek, acc.k);
        float2 P = __ffma2_rn(kz, ek, ndkb);
        acc.g1p = __fadd2_rn(acc.g1p, P);
        float2 ndD = __fmul2_rn(P, inv);
        acc.g1y = __ffma2_rn(ndD, wyy, acc.g1y);
        acc.hg2 = __ffma2_rn(ndD, __fmul2_rn(wx, wy), acc.hg2);
    }
}

// Two big-list entries of the same ray at once when some ray of the group may
// be inside the softening radius of one of them: gauss_correction (full -
// softened point; the series below t = kTSeries; zero outside the support)
// in packed FP32x2, each half choosing by select instead of a branch; a half
// whose entry was queued for the closed form (no ray inside its softening
// radius: ws = +inf) takes gauss_correction_fast's values instead, so that
// an entry gets the same form whatever entry it is paired with.  Operands
// are pairs over the two entries: nx, ny as above; t_c = c log2 e; kz =
// m c/N_q; mN = m/N_q; nmass = -m (mass); ws = 1/r0^2; ic = 1/c; Uq2 =
// q^2/2 log2 e; eU = e^-q^2/2.
template <bool AO>
LENS_DEV void gauss_correction_soft_x2(Acc5x2& acc, float2 lx, float2 ly, float2 nx, float2 ny, float2 t_c,
                                       float2 kz, float2 mN, float2 nmass, float2 ws, float2 ic, float Uq2,
                                       float eU)
{
    using namespace gser;
    const float2 wx = __fadd2_rn(lx, nx);
    const float2 wy = __fadd2_rn(ly, ny);
    const float2 wyy = __fmul2_rn(wy, wy);
    const float2 r2 = __ffma2_rn(wx, wx, wyy);
    float2 inv, inv_s;
    inv.x = r2.x > 0.0f ? rcp(r2.x) : 0.0f;
    inv.y = r2.y > 0.0f ? rcp(r2.y) : 0.0f;
    inv_s.x = fminf(inv.x, ws.x);
    inv_s.y = fminf(inv.y, ws.y);
    const float2 nkbp = __fmul2_rn(nmass, inv_s);  // minus the softened point's kb
    const float2 t = __fmul2_rn(r2, t_c);
    const float2 e = make_float2(exp2neg(t.x), exp2neg(t.y));
    // h1 and g: the series (small t) and the closed form, chosen per half
    const float2 hs = __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t,
                      __ffma2_rn(t, make_float2(H7, H7), make_float2(H6, H6)), make_float2(H5, H5)),
                      make_float2(H4, H4)), make_float2(H3, H3)), make_float2(H2, H2)), make_float2(H1, H1)),
                      make_float2(H0, H0));
    const float2 gs = __fmul2_rn(t, __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t,
                      __ffma2_rn(t, __ffma2_rn(t, make_float2(G7, G7), make_float2(G6, G6)), make_float2(G5, G5)),
                      make_float2(G4, G4)), make_float2(G3, G3)), make_float2(G2, G2)), make_float2(G1, G1)),
                      make_float2(G0, G0)));
    const float2 hc = __fmul2_rn(__ffma2_rn(e, make_float2(-1.0f, -1.0f), make_float2(1.0f, 1.0f)),
                                 __fmul2_rn(inv, ic));
    const float2 gc = __fadd2_rn(hc, __fmul2_rn(e, make_float2(-1.0f, -1.0f)));
    const bool sx = t.x < kTSeries, sy = t.y < kTSeries;
    const float2 h1 = make_float2(sx ? hs.x : hc.x, sy ? hs.y : hc.y);
    const float2 g = make_float2(sx ? gs.x : gc.x, sy ? gs.y : gc.y);
    const bool inx = t.x < Uq2, iny = t.y < Uq2;
    const bool fx = ws.x == INFINITY, fy = ws.y == INFINITY;
    // the closed form (full - point) of gauss_correction_fast
    const float2 ef = make_float2(inx ? e.x : eU, iny ? e.y : eU);
    const float2 dkbf = __fmul2_rn(__fmul2_rn(mN, inv), __fadd2_rn(make_float2(eU, eU), __fmul2_rn(ef, make_float2(-1.0f, -1.0f))));
    const float2 dkbg = __ffma2_rn(kz, h1, nkbp);
    const float2 ndkb = make_float2(fx ? -dkbf.x : (inx ? -dkbg.x : 0.0f), fy ? -dkbf.y : (iny ? -dkbg.y : 0.0f));
    acc.na1 = __ffma2_rn(ndkb, wx, acc.na1);
    acc.na2 = __ffma2_rn(ndkb, wy, acc.na2);
    if (!AO) {
        const float2 ke = __fmul2_rn(kz, e);
        const float2 kap = make_float2(inx ? ke.x : 0.0f, iny ? ke.y : 0.0f);
        acc.k = __fadd2_rn(acc.k, kap);
        const float2 dDf = __fmul2_rn(__fadd2_rn(dkbf, __fmul2_rn(kap, make_float2(-1.0f, -1.0f))), inv);
        const float2 dD = __ffma2_rn(__fmul2_rn(kz, g), inv, __fmul2_rn(nkbp, inv_s));
        const float2 ndD = make_float2(fx ? -dDf.x : (inx ? -dD.x : 0.0f), fy ? -dDf.y : (iny ? -dD.y : 0.0f));
        acc.g1p = __ffma2_rn(ndD, r2, acc.g1p);
        acc.g1y = __ffma2_rn(ndD, wyy, acc.g1y);
        acc.hg2 = __ffma2_rn(ndD, __fmul2_rn(wx, wy), acc.hg2);
    }
}

// FP64 form of the same correction (q1.y holds c log2 e as well).
template <bool AO>
LENS_DEV void gauss_correction(Acc5<double>& acc, double wx, double wy, const dbl4& q, const dbl4& q1,
                               double Uq2, double Nq)
{
    const double L = 0.69314718055994530942;
    double r2 = fma(wx, wx, wy * wy);
    double inv = r2 > 0.0 ? 1.0 / r2 : 0.0;
    double inv_s = fmin(inv, q.w);
    double kbp = (q1.x * Nq) * inv_s;
    double u = r2 * q1.y * L;
    if (!(r2 * q1.y < Uq2)) return;
    double e = exp(-u), h1, g;
    gauss_h1_g(u, e, h1, g);
    acc.template radial<AO>(wx, wy, fma(q1.z, h1, -kbp), q1.z * e, fma(q1.z * g, inv, -kbp * inv_s));
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
