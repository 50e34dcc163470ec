// halo_rays.cu -- shooting through a lens of analytic components only (Sec.
// 3.2 host analytic terms, no particles): one thread per ray sums the halos'
// (alpha, kappa, gamma) directly, without the ray grouping and tree walk the
// particle species need.  The terms are those of the walk's halo pass (the
// same profile functions, the same accumulation order over the halos); the
// separation from a halo is taken in FP64 from the FP64 ray position and
// then rounded to the working precision.
#include "common.cuh"
#include "profiles.cuh"
#include "tree.cuh"

namespace lens {
namespace {

template <typename T, typename TR, bool AO>
__global__ void k_halo_rays(const TR* dx, const TR* dy, int64_t n, double ox, double oy, const HaloDev* halos,
                            int n_halos, T* o0, T* o1, T* o2, T* o3, T* o4, int accumulate)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = ox + (double)dx[i], y = oy + (double)dy[i];
    Acc5<T> acc;
    acc.zero();
    for (int h = 0; h < n_halos; ++h) {
        const HaloDev& hd = halos[h];
        const T wx = (T)(x - hd.x), wy = (T)(y - hd.y);
        const T r2 = fma(wx, wx, wy * wy);
        const T m = (T)hd.m;
        T kb = T(0), kap = T(0), Dp = T(0);
        if (hd.kind == LENS_POINT) {
            point_terms(m, r2, kb, Dp);
        } else if (hd.kind == LENS_GAUSS) {
            gauss_terms(m, (T)hd.c0, r2, (T)hd.c1, (T)hd.c2, kb, kap, Dp);
        } else if (hd.kind == LENS_NFW) {
            nfw_terms(m, (T)hd.c2, (T)hd.c0, (T)hd.c1, r2, kb, kap, Dp);
        } else if (hd.kind == LENS_SIS) {
            if (r2 > T(0)) {
                const T rr = sqrt(r2), re = (T)hd.p0;
                kb = re / rr;
                kap = T(0.5) * kb;
                Dp = kap / r2;
            }
        } else {  // uniform disk
            const T R2 = (T)hd.c2;
            if (r2 < R2) {
                kb = m / R2;
                kap = kb;
                Dp = T(0);
            } else {
                point_terms(m, r2, kb, Dp);
            }
        }
        acc.template radial<AO>(wx, wy, kb, kap, Dp);
    }
    const T v[5] = {acc.a1, acc.a2, acc.k, acc.g1, acc.g2};
    T* out[5] = {o0, o1, o2, o3, o4};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        if (AO && q >= 2) break;
        out[q][i] = accumulate ? out[q][i] + v[q] : v[q];
    }
}

template <typename T, typename TR>
void launch(const void* dx, const void* dy, int64_t n, double ox, double oy, const lens_tree* t, void* const out[5],
            bool ao, int acc, cudaStream_t s)
{
    const unsigned nb = (unsigned)((n + 255) / 256);
    T* o[5];
    for (int q = 0; q < 5; ++q) o[q] = (T*)out[q];
    if (ao)
        k_halo_rays<T, TR, true><<<nb, 256, 0, s>>>((const TR*)dx, (const TR*)dy, n, ox, oy, t->halos,
                                                    (int)t->n_halos, o[0], o[1], o[2], o[3], o[4], acc);
    else
        k_halo_rays<T, TR, false><<<nb, 256, 0, s>>>((const TR*)dx, (const TR*)dy, n, ox, oy, t->halos,
                                                     (int)t->n_halos, o[0], o[1], o[2], o[3], o[4], acc);
    note_launch();
}

}  // namespace

bool halos_only(const lens_tree* t)
{
    for (const SpeciesTree& st : t->sp)
        if (st.n > 0) return false;
    return t->n_halos > 0;
}

lens_status shoot_halos_only(lens_tree* t, double ox, double oy, const void* dx, const void* dy, int dtype,
                             int64_t n, void* const out[5], int flags, cudaStream_t s)
{
    const bool ao = (flags & LENS_ALPHA_ONLY) != 0;
    const int acc = (flags & LENS_ACCUMULATE) ? 1 : 0;
    const bool f64 = t->precision == LENS_PREC_FP64;
    if (f64) {
        if (dtype == LENS_F64) launch<double, double>(dx, dy, n, ox, oy, t, out, ao, acc, s);
        else launch<double, float>(dx, dy, n, ox, oy, t, out, ao, acc, s);
    } else {
        if (dtype == LENS_F64) launch<float, double>(dx, dy, n, ox, oy, t, out, ao, acc, s);
        else launch<float, float>(dx, dy, n, ox, oy, t, out, ao, acc, s);
    }
    LENS_CUDA(cudaGetLastError());
    return LENS_OK;
}

}  // namespace lens
