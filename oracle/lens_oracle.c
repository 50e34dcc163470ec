/*
 * lens_oracle.c -- FP64 CPU oracle for the ray-shooting path of
 * Metcalf & Petkova, "GLAMER Part I" (arXiv:1312.1128).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header or constant table with
 * the CUDA path.
 *
 * What it computes (every function cites the passage it follows):
 *   - per-component lensing quantities (alpha1, alpha2, kappa, gamma1, gamma2)
 *     for point masses (Sec. 3.5, star deflection equation), truncated 2D
 *     Gaussian particles (Sec. 3.1 Eq. "smoothing" and the smoothed-particle
 *     deflection of Sec. 3.2), projected NFW halos truncated at R_max
 *     (Sec. 3.2: analytic halos, point mass outside the outer radius), the
 *     singular isothermal sphere (App. B) and a uniform disk (Sec. 3.5, the
 *     subtracted mass sheet);
 *   - the direct sum over all components for every ray (the theta_force = 0
 *     limit of Sec. 5.1), Neumaier-compensated, plus sum |term| per output;
 *   - the paper's tree algorithm (Sec. 3.2): equal-area quadtree, leaf when a
 *     box holds fewer than leaf_max particles, monopole + quadrupole moments,
 *     r_cut = r_cm / theta_force (Eq. r_cut), the 2D MAC, big-particle lists;
 *     evaluated ray by ray with per-ray interaction counts;
 *   - the vector-Jacobian product of the direct sum (gradient of a loss with
 *     respect to particle masses, positions and shape parameters) for the
 *     differentiable fit.
 *
 * Units: masses are in "m-units", m = M / (pi Sigma_crit), so a point mass has
 * alpha = m x / |x|^2 (Sec. 3.5) and kappa = pi * (m-unit surface density).
 * Shear follows Eq. gamma_1, gamma_2: gamma1 = (d1 a1 - d2 a2)/2, gamma2 = d1 a2.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_POINT = 0, OR_GAUSS = 1, OR_NFW = 2, OR_SIS = 3, OR_DISK = 4 };

/* One lens component.  GAUSS: p0 = r_sm (sigma), p1 = q.  NFW: p0 = r_s,
 * p1 = R_max.  SIS: p0 = Einstein radius r_E.  DISK: p0 = radius R (m may be
 * negative for a subtracted sheet).  POINT: p0, p1 unused. */
typedef struct {
    double x, y, m, p0, p1;
    int32_t type, pad;
} or_comp;

/* ------------------------------------------------------------------------ */
/* Radial profiles: enclosed m-unit mass Mt(<r) and kappa(r).                */
/* For an axisymmetric lens, alpha = Mt(<r) r_hat / r, mean kappa inside r is */
/* kb = Mt / r^2 and gamma1 + i gamma2 = -(kb - kappa) exp(2 i phi); these    */
/* follow from Eqs. alpha-gamma_2 with the Poisson equation (Sec. 3.2).       */
/* ------------------------------------------------------------------------ */

/* Projected NFW helper F(x) (SEF92-style closed form, Sec. 3.2 "analytic
 * models"): arccosh(1/x)/sqrt(1-x^2) for x<1, arccos(1/x)/sqrt(x^2-1) for x>1,
 * F(1) = 1.  Near x = 1 both forms are 0/0 and arccosh(1/x) is
 * ill-conditioned; for |u| < 0.1, u = 1 - x^2, the series
 * F = sum_k u^k/(2k+1) is used instead (40 terms: below 1e-40 there). */
static double nfw_F(double x)
{
    double u = 1.0 - x * x;
    if (fabs(u) < 0.1) {
        double s = 0.0, p = 1.0;
        for (int k = 0; k < 40; ++k) { s += p / (2 * k + 1); p *= u; }
        return s;
    }
    if (x < 1.0) return acosh(1.0 / x) / sqrt(u);
    return acos(1.0 / x) / sqrt(-u);
}

/* Projected NFW surface-density shape f(x) = (1 - F)/(x^2 - 1), f(1) = 1/3;
 * for |u| < 0.1 its series f = sum_k u^k/(2k+3) (the quotient cancels). */
static double nfw_f(double x)
{
    double u = 1.0 - x * x;
    if (fabs(u) < 0.1) {
        double s = 0.0, p = 1.0;
        for (int k = 0; k < 40; ++k) { s += p / (2 * k + 3); p *= u; }
        return s;
    }
    return (1.0 - nfw_F(x)) / (x * x - 1.0);
}

/* Projected NFW enclosed-mass shape g(x) = ln(x/2) + F(x), g' = x f.  For
 * x < 0.01 the closed form cancels; the small-x expansion with L = ln(2/x)
 * is g = x^2(L/2 - 1/4) + x^4(3L/8 - 7/32) + x^6(5L/16 - 37/192)
 *      + x^8(35L/128 - 533/3072) + O(x^10 L). */
static double nfw_g(double x)
{
    if (x <= 0.0) return 0.0;
    if (x < 1e-2) {
        double L = log(2.0 / x), x2 = x * x;
        return x2 * ((L / 2 - 0.25) +
               x2 * ((3 * L / 8 - 7.0 / 32) +
               x2 * ((5 * L / 16 - 37.0 / 192) +
               x2 * (35 * L / 128 - 533.0 / 3072))));
    }
    return log(x / 2.0) + nfw_F(x);
}

/* Enclosed mass and kappa at radius r > 0 for one component. */
static void or_profile(const or_comp* c, double r, double* Mt, double* kap)
{
    switch (c->type) {
    case OR_POINT:  /* Sec. 3.5: alpha = m r_hat / r; no surface density off the mass */
        *Mt = c->m; *kap = 0.0; return;
    case OR_GAUSS: { /* Sec. 3.1 Eq. smoothing; Sec. 3.2 smoothed deflection */
        double sig = c->p0, q = c->p1;
        double Nq = -expm1(-0.5 * q * q);
        if (r < q * sig) {
            double u = r * r / (2.0 * sig * sig);
            *Mt = c->m * (-expm1(-u)) / Nq;
            *kap = c->m * exp(-u) / (2.0 * sig * sig * Nq);
        } else { *Mt = c->m; *kap = 0.0; }
        return;
    }
    case OR_NFW: {   /* projected NFW truncated in 2D at R_max; point mass outside */
        double rs = c->p0, Rmax = c->p1;
        if (r < Rmax) {
            double gX = nfw_g(Rmax / rs), x = r / rs;
            *Mt = c->m * nfw_g(x) / gX;
            *kap = c->m * nfw_f(x) / (2.0 * rs * rs * gX);
        } else { *Mt = c->m; *kap = 0.0; }
        return;
    }
    case OR_SIS:     /* App. B: alpha = r_E x/|x|, kappa = r_E/(2r) */
        *Mt = c->p0 * r; *kap = c->p0 / (2.0 * r); return;
    case OR_DISK: {  /* uniform disk: kappa = m/R^2 inside, point mass outside */
        double R = c->p0;
        if (r < R) { *Mt = c->m * r * r / (R * R); *kap = c->m / (R * R); }
        else { *Mt = c->m; *kap = 0.0; }
        return;
    }
    }
    *Mt = 0.0; *kap = 0.0;
}

/* kappa at the centre (r = 0) of a component with a finite central density;
 * singular profiles (point, NFW, SIS) contribute nothing at r = 0 exactly. */
static double or_central_kappa(const or_comp* c)
{
    if (c->type == OR_GAUSS) {
        double sig = c->p0, q = c->p1;
        return c->m / (2.0 * sig * sig * (-expm1(-0.5 * q * q)));
    }
    if (c->type == OR_DISK) return c->m / (c->p0 * c->p0);
    return 0.0;
}

/* The five lensing quantities of one component at ray (x, y). */
void or_eval_component(const or_comp* c, double x, double y, double out[5])
{
    double dx = x - c->x, dy = y - c->y;
    double r2 = dx * dx + dy * dy;
    if (r2 == 0.0) {
        out[0] = out[1] = out[3] = out[4] = 0.0;
        out[2] = or_central_kappa(c);
        return;
    }
    double r = sqrt(r2), Mt, kap;
    or_profile(c, r, &Mt, &kap);
    double kb = Mt / r2;
    out[0] = Mt * dx / r2;
    out[1] = Mt * dy / r2;
    out[2] = kap;
    double c2 = (dx * dx - dy * dy) / r2, s2 = 2.0 * dx * dy / r2;
    out[3] = -(kb - kap) * c2;
    out[4] = -(kb - kap) * s2;
}

/* ------------------------------------------------------------------------ */
/* Lensing potential (Eq. alpha: alpha = grad psi; Eq. timedelay uses psi).  */
/* For an axisymmetric component psi(r) = psi(r_e) - int_r^{r_e} Mt(r')/r' dr'*/
/* with Mt the enclosed m-unit mass above; outside its support every finite  */
/* component is a point mass, psi = m ln r.  The additive constant is fixed   */
/* by that choice (SIS: psi = r_E r).                                         */
/* ------------------------------------------------------------------------ */

/* Ein(u) = int_0^u (1 - e^-t)/t dt: its alternating series for u < 8, and
 * Ein = E1(u) + ln u + gamma_E with the continued fraction of E1 beyond. */
static double or_ein(double u)
{
    if (u < 8.0) {
        double s = 0.0, term = 1.0;  /* term = u^k / k! */
        for (int k = 1; k < 200; ++k) {
            term *= u / k;
            double add = ((k & 1) ? term : -term) / k;
            s += add;
            if (fabs(add) < 1e-18 * fabs(s)) break;
        }
        return s;
    }
    /* E1(u) = e^-u / (u + 1 - 1/(u + 3 - 4/(u + 5 - 9/(u + 7 - ...)))) (modified Lentz) */
    double b = u + 1.0, cc = 1e300, d = 1.0 / b, h = d;
    for (int i = 1; i < 300; ++i) {
        double an = -(double)i * i;
        b += 2.0;
        d = 1.0 / (an * d + b);
        cc = b + an / cc;
        double del = cc * d;
        h *= del;
        if (fabs(del - 1.0) < 1e-16) break;
    }
    return h * exp(-u) + log(u) + 0.57721566490153286061;
}

/* NFW potential shape H(x) = int g(x)/x dx = ln^2(x/2)/2 - (1 - x^2) F(x)^2/2
 * (H(0) = 0).  For x < 1/2 the two squares nearly cancel; there
 * arccosh(1/x) = L + e with L = ln(2/x), e = log1p(-x^2 / (2 (1 + t))),
 * t = sqrt(1 - x^2), and H = -e (2L + e)/2. */
static double nfw_H(double x)
{
    if (x <= 0.0) return 0.0;
    if (x < 0.5) {
        double t = sqrt(1.0 - x * x), L = log(2.0 / x);
        double e = log1p(-x * x / (2.0 * (1.0 + t)));
        return -0.5 * e * (2.0 * L + e);
    }
    double lx = log(0.5 * x), F = nfw_F(x);
    return 0.5 * lx * lx - 0.5 * (1.0 - x * x) * F * F;
}

/* psi(r) of one component (r >= 0; a point mass and an SIS give 0 at r = 0). */
static double or_potential_profile(const or_comp* c, double r)
{
    switch (c->type) {
    case OR_POINT:
        return r > 0.0 ? c->m * log(r) : 0.0;
    case OR_GAUSS: {
        double sig = c->p0, q = c->p1, re = q * sig;
        if (r >= re) return c->m * log(r);
        double Nq = -expm1(-0.5 * q * q), u = r * r / (2.0 * sig * sig);
        return c->m * log(re) - c->m / (2.0 * Nq) * (or_ein(0.5 * q * q) - or_ein(u));
    }
    case OR_NFW: {
        double rs = c->p0, Rmax = c->p1;
        if (r >= Rmax) return c->m * log(r);
        double X = Rmax / rs;
        return c->m * log(Rmax) - c->m / nfw_g(X) * (nfw_H(X) - nfw_H(r / rs));
    }
    case OR_SIS:
        return c->p0 * r;
    case OR_DISK: {
        double R = c->p0;
        if (r >= R) return c->m * log(r);
        return c->m * (log(R) + 0.5 * (r * r / (R * R) - 1.0));
    }
    }
    return 0.0;
}

double or_potential_component(const or_comp* c, double x, double y)
{
    double dx = x - c->x, dy = y - c->y;
    return or_potential_profile(c, sqrt(dx * dx + dy * dy));
}

/* Neumaier compensated accumulator. */
typedef struct { double s, c; } nsum;
static inline void nadd(nsum* a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}

/* Direct sum over all components for every ray (Sec. 5.1: theta_force = 0 adds
 * the contributions one by one; superposition, Sec. 3.2).  out: nr x 5,
 * absum (optional): nr x 5 of sum |term|.  Returns 0. */
int or_direct_sum(const or_comp* comps, int64_t nc, const double* rx, const double* ry,
                  int64_t nr, double* out, double* absum, int nthreads)
{
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int64_t i = 0; i < nr; ++i) {
        nsum acc[5] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
        double ab[5] = {0, 0, 0, 0, 0};
        double t[5];
        for (int64_t j = 0; j < nc; ++j) {
            or_eval_component(&comps[j], rx[i], ry[i], t);
            for (int q = 0; q < 5; ++q) { nadd(&acc[q], t[q]); ab[q] += fabs(t[q]); }
        }
        for (int q = 0; q < 5; ++q) {
            out[5 * i + q] = acc[q].s + acc[q].c;
            if (absum) absum[5 * i + q] = ab[q];
        }
    }
    return 0;
}

/* Direct sum of the potential (Neumaier), with sum |term| (optional). */
int or_direct_potential(const or_comp* comps, int64_t nc, const double* rx, const double* ry,
                        int64_t nr, double* psi, double* absum, int nthreads)
{
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int64_t i = 0; i < nr; ++i) {
        nsum acc = {0, 0};
        double ab = 0.0;
        for (int64_t j = 0; j < nc; ++j) {
            double t = or_potential_component(&comps[j], rx[i], ry[i]);
            nadd(&acc, t);
            ab += fabs(t);
        }
        psi[i] = acc.s + acc.c;
        if (absum) absum[i] = ab;
    }
    return 0;
}

/* Derivatives of the enclosed mass Mt(<r) with respect to the component's
 * shape parameters p0 and p1 at radius r > 0 (the profiles of or_profile
 * above, differentiated at fixed r and m).  alpha = Mt w / r^2, so
 * d alpha / d p = (d Mt / d p) w / r^2.
 *   GAUSS (p0 = r_sm, p1 = q), inside r < q r_sm, u = r^2 / (2 r_sm^2):
 *     Mt = m (1 - e^-u) / N_q,  du/dr_sm = -2u / r_sm,
 *     dN_q/dq = q e^{-q^2/2}; the support edge moves with both but Mt is
 *     continuous there (= m), so nothing is added at the edge.
 *   NFW (p0 = r_s, p1 = R_max), inside r < R_max, x = r/r_s, X = R_max/r_s:
 *     Mt = m g(x) / g(X) with g' = x f (Sec. 3.2 projected NFW).
 *   SIS (p0 = r_E): Mt = r_E r.
 *   DISK (p0 = R), inside r < R: Mt = m r^2 / R^2.
 *   Outside a truncated profile Mt = m does not depend on p0, p1. */
static void or_profile_dparams(const or_comp* c, double r, double* d0, double* d1)
{
    *d0 = 0.0;
    *d1 = 0.0;
    switch (c->type) {
    case OR_GAUSS: {
        double sig = c->p0, q = c->p1;
        if (r < q * sig) {
            double Nq = -expm1(-0.5 * q * q), u = r * r / (2.0 * sig * sig);
            double Mt = c->m * (-expm1(-u)) / Nq;
            *d0 = c->m * exp(-u) * (-2.0 * u / sig) / Nq;
            *d1 = -Mt * q * exp(-0.5 * q * q) / Nq;
        }
        return;
    }
    case OR_NFW: {
        double rs = c->p0, Rmax = c->p1;
        if (r < Rmax) {
            double x = r / rs, X = Rmax / rs, gx = nfw_g(x), gX = nfw_g(X);
            double dgx = x * nfw_f(x), dgX = X * nfw_f(X);   /* g'(x), g'(X) */
            /* dx/dr_s = -x/r_s, dX/dr_s = -X/r_s, dX/dR_max = 1/r_s */
            *d0 = c->m * (dgx * (-x / rs) * gX - gx * dgX * (-X / rs)) / (gX * gX);
            *d1 = -c->m * gx * dgX / (rs * gX * gX);
        }
        return;
    }
    case OR_SIS:
        *d0 = r;
        return;
    case OR_DISK: {
        double R = c->p0;
        if (r < R) *d0 = -2.0 * c->m * r * r / (R * R * R);
        return;
    }
    default:
        return;
    }
}

/* Vector-Jacobian product of the direct sum: given upstream gradients
 * G (nr x 5, for alpha1, alpha2, kappa, gamma1, gamma2 at each ray), returns
 * grad (nc x 3, or nc x 5 with with_params) = dL/d(m, x, y[, p0, p1]) of every
 * component.  Only the alpha part of G may be non-zero (the loss of the
 * differentiable fit is a function of alpha); a non-zero kappa/gamma gradient
 * returns -1.
 *   d alpha / d m = alpha / m (every profile is linear in m at fixed shape);
 *   d alpha / d x_p = -(Jacobian of alpha at the ray), with the Jacobian
 *   [[kappa+gamma1, gamma2], [gamma2, kappa-gamma1]] from Eqs. kappa-gamma_2;
 *   d alpha / d p0, p1 = (d Mt / d p) w / r^2 (or_profile_dparams). */
int or_direct_vjp(const or_comp* comps, int64_t nc, const double* rx, const double* ry,
                  int64_t nr, const double* G, double* grad, int with_params, int nthreads)
{
    for (int64_t i = 0; i < nr; ++i)
        if (G[5 * i + 2] != 0.0 || G[5 * i + 3] != 0.0 || G[5 * i + 4] != 0.0) return -1;
    const int st = with_params ? 5 : 3;
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t j = 0; j < nc; ++j) {
        nsum gm = {0, 0}, gx = {0, 0}, gy = {0, 0}, g0 = {0, 0}, g1s = {0, 0};
        double t[5];
        for (int64_t i = 0; i < nr; ++i) {
            double g1 = G[5 * i], g2 = G[5 * i + 1];
            if (g1 == 0.0 && g2 == 0.0) continue;
            or_eval_component(&comps[j], rx[i], ry[i], t);
            if (comps[j].m != 0.0) nadd(&gm, (g1 * t[0] + g2 * t[1]) / comps[j].m);
            /* dalpha_k/dx_p = -d alpha_k / d x_ray */
            double a11 = t[2] + t[3], a22 = t[2] - t[3], a12 = t[4];
            nadd(&gx, -(g1 * a11 + g2 * a12));
            nadd(&gy, -(g1 * a12 + g2 * a22));
            if (with_params) {
                double dx = rx[i] - comps[j].x, dy = ry[i] - comps[j].y, r2 = dx * dx + dy * dy;
                if (r2 > 0.0) {
                    double d0, d1;
                    or_profile_dparams(&comps[j], sqrt(r2), &d0, &d1);
                    double gw = (g1 * dx + g2 * dy) / r2;
                    nadd(&g0, d0 * gw);
                    nadd(&g1s, d1 * gw);
                }
            }
        }
        grad[st * j] = gm.s + gm.c;
        grad[st * j + 1] = gx.s + gx.c;
        grad[st * j + 2] = gy.s + gy.c;
        if (with_params) {
            grad[st * j + 3] = g0.s + g0.c;
            grad[st * j + 4] = g1s.s + g1s.c;
        }
    }
    return 0;
}

/* ======================================================================== */
/* The paper's tree (Sec. 3.2), scalar and recursive, one ray at a time.     */
/* ======================================================================== */

typedef struct {
    double cx, cy, half;        /* box centre and half side */
    int32_t child[4];           /* -1 when absent; all -1 for a leaf */
    int32_t leaf;               /* 1 if not subdivided */
    int64_t first, count;       /* particle range in the tree's index array */
    double M, xcm, ycm;         /* monopole and centre of mass */
    double complex Q2;          /* quadrupole: sum m (z - z_cm)^2 */
    double rcut;                /* r_cm / theta (Eq. r_cut); +inf when theta = 0 */
    int64_t big_first, big_count; /* big-particle list (indices into bigidx) */
} or_box;

typedef struct {
    const or_comp* p;           /* caller's components (not owned) */
    int64_t n;
    int64_t* idx;               /* particle order: boxes own contiguous ranges */
    or_box* box;
    int64_t nbox, cap;
    int64_t* bigidx;            /* concatenated big lists */
    int64_t nbig;
    unsigned char* listed;      /* 1 if the particle sits in some box's big list */
    int leaf_max;
    double theta, lambda;
} or_tree;

/* Support radius of a component: beyond it the component acts as a point. */
static double or_size(const or_comp* c)
{
    switch (c->type) {
    case OR_GAUSS: return c->p0 * c->p1;
    case OR_NFW: return c->p1;
    case OR_DISK: return c->p0;
    case OR_SIS: return INFINITY;
    default: return 0.0;
    }
}

static int64_t or_newbox(or_tree* t)
{
    if (t->nbox == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 1024;
        t->box = (or_box*)realloc(t->box, (size_t)t->cap * sizeof(or_box));
    }
    return t->nbox++;
}

/* Subdivide recursively: four equal-area children; a box with fewer than
 * leaf_max particles is a leaf (Sec. 3.2).  The moments, r_cut and big list of
 * each box are computed as the box is made. */
static void or_build_box(or_tree* t, int64_t b, int depth,
                         int64_t* tmp)
{
    or_box* B = &t->box[b];
    const or_comp* P = t->p;
    int64_t f = B->first, n = B->count;
    /* monopole and centre of mass (2D projected distances) */
    double M = 0, sx = 0, sy = 0;
    for (int64_t k = f; k < f + n; ++k) {
        const or_comp* c = &P[t->idx[k]];
        M += c->m; sx += c->m * c->x; sy += c->m * c->y;
    }
    double xcm = (M != 0.0) ? sx / M : B->cx, ycm = (M != 0.0) ? sy / M : B->cy;
    double complex Q2 = 0;
    for (int64_t k = f; k < f + n; ++k) {
        const or_comp* c = &P[t->idx[k]];
        double complex d = (c->x - xcm) + I * (c->y - ycm);
        Q2 += c->m * d * d;
    }
    /* r_cm: distance from the centre of mass to the farthest box corner */
    double ddx = fabs(xcm - B->cx) + B->half, ddy = fabs(ycm - B->cy) + B->half;
    double rcm = sqrt(ddx * ddx + ddy * ddy);
    B->M = M; B->xcm = xcm; B->ycm = ycm; B->Q2 = Q2;
    B->rcut = (t->theta > 0.0) ? rcm / t->theta : INFINITY;
    /* big list: particles of this box larger than lambda * side not listed higher */
    B->big_first = t->nbig; B->big_count = 0;
    double side = 2.0 * B->half;
    for (int64_t k = f; k < f + n; ++k) {
        int64_t pi = t->idx[k];
        if (t->listed[pi]) continue;
        if (or_size(&P[pi]) > t->lambda * side) {
            t->listed[pi] = 1;
            t->bigidx[t->nbig++] = pi;
            B->big_count++;
        }
    }
    for (int q = 0; q < 4; ++q) B->child[q] = -1;
    B->leaf = (n < t->leaf_max || depth >= 60) ? 1 : 0;
    if (B->leaf) return;
    /* partition into quadrants: q = (x >= cx) + 2 (y >= cy) */
    double cx = B->cx, cy = B->cy, h = B->half;
    int64_t cnt[4] = {0, 0, 0, 0};
    for (int64_t k = f; k < f + n; ++k) {
        const or_comp* c = &P[t->idx[k]];
        int q = (c->x >= cx) + 2 * (c->y >= cy);
        cnt[q]++;
    }
    int64_t off[4] = {0, cnt[0], cnt[0] + cnt[1], cnt[0] + cnt[1] + cnt[2]};
    for (int64_t k = f; k < f + n; ++k) {
        const or_comp* c = &P[t->idx[k]];
        int q = (c->x >= cx) + 2 * (c->y >= cy);
        tmp[off[q]++] = t->idx[k];
    }
    memcpy(t->idx + f, tmp, (size_t)n * sizeof(int64_t));
    int64_t start = f;
    for (int q = 0; q < 4; ++q) {
        if (cnt[q] == 0) continue;
        int64_t c = or_newbox(t);
        B = &t->box[b];  /* realloc may move */
        or_box* C = &t->box[c];
        C->half = 0.5 * h;
        C->cx = cx + ((q & 1) ? 0.5 * h : -0.5 * h);
        C->cy = cy + ((q & 2) ? 0.5 * h : -0.5 * h);
        C->first = start; C->count = cnt[q];
        start += cnt[q];
        B->child[q] = (int32_t)c;
        or_build_box(t, c, depth + 1, tmp);
        B = &t->box[b];
    }
}

/* Build the paper's tree over n components (SIS components are not allowed:
 * they have no outer radius).  The big-list threshold is lambda * side with
 * lambda = min(1/2, (1/theta - 1)/sqrt(2)): the paper's "half the box size"
 * whenever theta <= 1/(1 + 1/sqrt 2), tightened above that so that every
 * particle whose support covers a ray is listed in a box the ray visits. */
or_tree* or_tree_build(const or_comp* p, int64_t n, int leaf_max, double theta)
{
    if (n <= 0 || leaf_max < 1) return NULL;
    for (int64_t i = 0; i < n; ++i) if (p[i].type == OR_SIS) return NULL;
    or_tree* t = (or_tree*)calloc(1, sizeof(or_tree));
    t->p = p; t->n = n; t->leaf_max = leaf_max; t->theta = theta;
    t->lambda = 0.5;
    if (theta > 0.0) {
        double lam = (1.0 / theta - 1.0) / sqrt(2.0);
        if (lam < t->lambda) t->lambda = lam > 0.0 ? lam : 0.0;
    }
    t->idx = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    t->bigidx = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    t->listed = (unsigned char*)calloc((size_t)n, 1);
    int64_t* tmp = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        t->idx[i] = i;
        if (p[i].x < x0) x0 = p[i].x;
        if (p[i].x > x1) x1 = p[i].x;
        if (p[i].y < y0) y0 = p[i].y;
        if (p[i].y > y1) y1 = p[i].y;
    }
    double half = 0.5 * fmax(x1 - x0, y1 - y0);
    half = half > 0 ? half * (1.0 + 1e-9) : 1e-9;
    int64_t r = or_newbox(t);
    t->box[r].cx = 0.5 * (x0 + x1); t->box[r].cy = 0.5 * (y0 + y1);
    t->box[r].half = half; t->box[r].first = 0; t->box[r].count = n;
    or_build_box(t, r, 0, tmp);
    free(tmp);
    return t;
}

void or_tree_free(or_tree* t)
{
    if (!t) return;
    free(t->idx); free(t->box); free(t->bigidx); free(t->listed); free(t);
}

int64_t or_tree_nboxes(const or_tree* t) { return t ? t->nbox : 0; }

/* Counts per ray: [0] far cells accepted, [1] near particles evaluated as a
 * point mass, [2] near particles evaluated with their full profile, [3] big-
 * list corrections applied (ray inside the support), [4] boxes visited. */
typedef struct { int64_t far, near_pt, near_ex, big, visited; } or_counts;

static void or_add(nsum* acc, const double t[5], double sign)
{
    for (int q = 0; q < 5; ++q) nadd(&acc[q], sign * t[q]);
}

static void or_walk(const or_tree* t, int64_t b, double x, double y, nsum* acc, or_counts* cn)
{
    const or_box* B = &t->box[b];
    const or_comp* P = t->p;
    double tt[5], tp[5];
    cn->visited++;
    /* big list of a visited box: add (full profile - point) when the ray is
     * inside the particle's support (Sec. 3.2, the big particle problem) */
    for (int64_t k = 0; k < B->big_count; ++k) {
        const or_comp* c = &P[t->bigidx[B->big_first + k]];
        double dx = x - c->x, dy = y - c->y;
        if (dx * dx + dy * dy < or_size(c) * or_size(c)) {
            or_comp pt = *c; pt.type = OR_POINT;
            or_eval_component(c, x, y, tt);
            or_eval_component(&pt, x, y, tp);
            or_add(acc, tt, 1.0); or_add(acc, tp, -1.0);
            cn->big++;
        }
    }
    /* MAC, 2D: |x - x_cm| > r_cut accepts the box's multipoles */
    double wx = x - B->xcm, wy = y - B->ycm;
    if (sqrt(wx * wx + wy * wy) > B->rcut) {
        /* conj(alpha) = M/w + Q2/w^3 ; conj(gamma) = -M/w^2 - 3 Q2/w^4 */
        double complex w = wx + I * wy, u = 1.0 / w;
        double complex ca = B->M * u + B->Q2 * u * u * u;
        double complex cg = -B->M * u * u - 3.0 * B->Q2 * u * u * u * u;
        tt[0] = creal(ca); tt[1] = -cimag(ca); tt[2] = 0.0;
        tt[3] = creal(cg); tt[4] = -cimag(cg);
        or_add(acc, tt, 1.0);
        cn->far++;
        return;
    }
    if (B->leaf) {
        for (int64_t k = B->first; k < B->first + B->count; ++k) {
            int64_t pi = t->idx[k];
            const or_comp* c = &P[pi];
            if (t->listed[pi]) {           /* listed particles count as points here */
                or_comp pt = *c; pt.type = OR_POINT;
                or_eval_component(&pt, x, y, tt);
                cn->near_pt++;
            } else {
                or_eval_component(c, x, y, tt);
                double dx = x - c->x, dy = y - c->y;
                if (dx * dx + dy * dy < or_size(c) * or_size(c)) cn->near_ex++;
                else cn->near_pt++;
            }
            or_add(acc, tt, 1.0);
        }
        return;
    }
    for (int q = 0; q < 4; ++q)
        if (B->child[q] >= 0) or_walk(t, B->child[q], x, y, acc, cn);
}

/* Evaluate the tree for nr rays.  counts (optional): nr x 5 int64. */
int or_tree_eval(const or_tree* t, const double* rx, const double* ry, int64_t nr,
                 double* out, int64_t* counts, int nthreads)
{
    if (!t) return -1;
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int64_t i = 0; i < nr; ++i) {
        nsum acc[5] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
        or_counts cn = {0, 0, 0, 0, 0};
        or_walk(t, 0, rx[i], ry[i], acc, &cn);
        for (int q = 0; q < 5; ++q) out[5 * i + q] = acc[q].s + acc[q].c;
        if (counts) {
            counts[5 * i] = cn.far; counts[5 * i + 1] = cn.near_pt;
            counts[5 * i + 2] = cn.near_ex; counts[5 * i + 3] = cn.big;
            counts[5 * i + 4] = cn.visited;
        }
    }
    return 0;
}

/* Threads the OpenMP runtime will use (for reporting the CPU baseline). */
int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
