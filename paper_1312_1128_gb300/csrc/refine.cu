// refine.cu -- cell refinement by the linear lens equation (Sec. 3.4
// interpolation; magnification matrix from deflections, App. A).
//
// Rays sit on a uniform grid, ray (i, j) at (x0 + i h, y0 + j h), flat index
// i + nx j; each ray is the centre of a cell of side h whose neighbours are
// the edge-adjacent rays E, N, W, S.  Per cell (k_refine_cells, one thread per
// cell) the uniformity test and the magnification matrix A:
//   kappa/gamma mode: every neighbour's kappa, gamma1, gamma2 within tol of the
//     centre's; A = [[1 - kappa - gamma1, -gamma2], [-gamma2, 1 - kappa + gamma1]]
//     (Eq. magmatrix) at the centre;
//   deflection mode: for each neighbour pair not colinear with the centre
//     (E-N, N-W, W-S, S-E), A from the three points by the App. A solve of
//     dy = A dx with y = x - alpha; uniform if no element of A differs by more
//     than tol between the pairs; A = their average.
// Then, per sub-cell centre (k_refine_sub, one thread per sub-cell, so the
// dominant output is written coalesced), y = y_c + A (x - x_c) (Eq.
// linear_lens_equation) for uniform cells and NaN otherwise.
#include <cmath>

#include "common.cuh"

namespace lens {

constexpr int kRefineMaxK = 15;

template <typename C>
LENS_DEV void app_a(C dx1a, C dx1b, C dy1a, C dy1b, C dx2a, C dx2b, C dy2a, C dy2b, C (&A)[4])
{
    // two displacement pairs dy = A dx, A = [[a11, a21], [a12, a22]]
    const C det = dx1a * dx2b - dx1b * dx2a;
    A[0] = (dx2b * dy1a - dx1b * dy2a) / det;  // a11
    A[1] = (dx1a * dy2a - dx2a * dy1a) / det;  // a21
    A[2] = (dx2b * dy1b - dx1b * dy2b) / det;  // a12
    A[3] = (dx1a * dy2b - dx2a * dy1b) / det;  // a22
}

template <typename TA>
__global__ void k_refine_cells(int64_t n_cells, const int64_t* cells, int64_t nx, int64_t ny, double h,
                               const TA* a1, const TA* a2, const float* ka, const float* g1, const float* g2,
                               double tol, int mode, uint8_t* uniform, float* amat,
                               unsigned long long* n_nonuniform)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const int64_t id = cells[c];
    const int64_t i = id >= 0 ? id % nx : -1, j = id >= 0 ? id / nx : -1;
    if (id < 0 || i < 1 || i > nx - 2 || j < 1 || j > ny - 2) {
        uniform[c] = 2;  // not an interior cell of the grid
        for (int q = 0; q < 4; ++q) amat[4 * c + q] = NAN;
        return;
    }
    const int64_t nb[4] = {id + 1, id + nx, id - 1, id - nx};  // E, N, W, S
    float A[4];
    bool uni;
    if (mode == LENS_REFINE_KAPPA_GAMMA) {
        const float kc = ka[id], g1c = g1[id], g2c = g2[id];
        float stat = 0.0f;
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            stat = fmaxf(stat, fabsf(ka[nb[n]] - kc));
            stat = fmaxf(stat, fabsf(g1[nb[n]] - g1c));
            stat = fmaxf(stat, fabsf(g2[nb[n]] - g2c));
        }
        uni = stat <= (float)tol;
        A[0] = 1.0f - kc - g1c;
        A[1] = -g2c;
        A[2] = -g2c;
        A[3] = 1.0f - kc + g1c;
    } else {
        // in the precision of the deflections (FP64 deflections keep the
        // differences between neighbours, the reason App. A exists)
        using C = TA;
        const C hh = (C)h;
        const C dxa[4] = {hh, C(0), -hh, C(0)}, dxb[4] = {C(0), hh, C(0), -hh};
        const C ac1 = a1[id], ac2 = a2[id];
        C dya[4], dyb[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            dya[n] = dxa[n] - (a1[nb[n]] - ac1);
            dyb[n] = dxb[n] - (a2[nb[n]] - ac2);
        }
        C lo[4], hi[4], sum[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int u = p, v = (p + 1) & 3;  // E-N, N-W, W-S, S-E
            C Ap[4];
            app_a<C>(dxa[u], dxb[u], dya[u], dyb[u], dxa[v], dxb[v], dya[v], dyb[v], Ap);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                lo[q] = p == 0 ? Ap[q] : fmin(lo[q], Ap[q]);
                hi[q] = p == 0 ? Ap[q] : fmax(hi[q], Ap[q]);
                sum[q] = p == 0 ? Ap[q] : sum[q] + Ap[q];
            }
        }
        C stat = C(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            stat = fmax(stat, hi[q] - lo[q]);
            A[q] = (float)(sum[q] * C(0.25));
        }
        uni = stat <= (C)tol;
    }
    uniform[c] = uni ? 1 : 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) amat[4 * c + q] = A[q];
    if (!uni && n_nonuniform) atomicAdd(n_nonuniform, 1ull);
}

template <typename TA>
__global__ void k_refine_sub(int64_t n_cells, int k, const int64_t* cells, int64_t nx, double x0, double y0,
                             double h, const TA* a1, const TA* a2, const uint8_t* uniform, const float* amat,
                             double2* y_sub)
{
    const int kk = k * k;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_cells * kk) return;
    const int64_t c = t / kk;
    const int s = (int)(t - c * kk), a = s % k, b = s / k;
    if (uniform[c] != 1) {
        y_sub[t] = make_double2(NAN, NAN);
        return;
    }
    const int64_t id = cells[c];
    const int64_t i = id % nx, j = id / nx;
    const double xc = x0 + (double)i * h, yc = y0 + (double)j * h;
    const double ycx = xc - (double)a1[id], ycy = yc - (double)a2[id];
    const double half = 0.5 * (k - 1);
    const double da = ((double)a - half) * h / k, db = ((double)b - half) * h / k;
    const float* A = amat + 4 * c;
    y_sub[t] = make_double2(ycx + (double)A[0] * da + (double)A[1] * db, ycy + (double)A[2] * da + (double)A[3] * db);
}

}  // namespace lens

using namespace lens;

extern "C" lens_status lens_refine_cells(double x0, double y0, double h, int64_t nx, int64_t ny,
                                         const void* alpha1, const void* alpha2, int32_t alpha_dtype,
                                         const float* kappa, const float* gamma1, const float* gamma2,
                                         const int64_t* cells, int64_t n_cells, int32_t k, double tol,
                                         int32_t mode, uint8_t* uniform, float* amat, double* y_sub,
                                         unsigned long long* n_nonuniform, void* stream)
{
    if (n_cells < 0) return lens_set_error(LENS_ERR_INVALID_ARG, "n_cells < 0");
    if (nx < 3 || ny < 3) return lens_set_error(LENS_ERR_INVALID_ARG, "the grid needs at least 3 x 3 rays");
    if (!(h > 0.0) || !std::isfinite(h) || !std::isfinite(x0) || !std::isfinite(y0))
        return lens_set_error(LENS_ERR_INVALID_ARG, "bad grid origin or spacing");
    if (k < 1 || k > kRefineMaxK || (k & 1) == 0)
        return lens_set_error(LENS_ERR_INVALID_ARG, "k must be odd, 1..%d", kRefineMaxK);
    if (!(tol >= 0.0)) return lens_set_error(LENS_ERR_INVALID_ARG, "tol must be >= 0");
    if (mode != LENS_REFINE_KAPPA_GAMMA && mode != LENS_REFINE_DEFLECTION)
        return lens_set_error(LENS_ERR_INVALID_ARG, "unknown refine mode");
    if (alpha_dtype != LENS_F32 && alpha_dtype != LENS_F64)
        return lens_set_error(LENS_ERR_INVALID_ARG, "alpha_dtype must be LENS_F32 or LENS_F64");
    if (n_cells == 0) return LENS_OK;
    if (!alpha1 || !alpha2 || !cells || !uniform || !amat || !y_sub)
        return lens_set_error(LENS_ERR_INVALID_ARG, "NULL array");
    if (mode == LENS_REFINE_KAPPA_GAMMA && (!kappa || !gamma1 || !gamma2))
        return lens_set_error(LENS_ERR_INVALID_ARG, "kappa/gamma mode needs kappa, gamma1 and gamma2");
    cudaStream_t s = (cudaStream_t)stream;
    const int TB = 256;
    const int64_t g1 = (n_cells + TB - 1) / TB, g2 = (n_cells * k * k + TB - 1) / TB;
    if (alpha_dtype == LENS_F32) {
        k_refine_cells<float><<<(unsigned)g1, TB, 0, s>>>(n_cells, cells, nx, ny, h, (const float*)alpha1,
                                                            (const float*)alpha2, kappa, gamma1, gamma2,
                                                            tol, mode, uniform, amat, n_nonuniform);
        note_launch();
        k_refine_sub<float><<<(unsigned)g2, TB, 0, s>>>(n_cells, k, cells, nx, x0, y0, h, (const float*)alpha1,
                                                          (const float*)alpha2, uniform, amat, (double2*)y_sub);
        note_launch();
    } else {
        k_refine_cells<double><<<(unsigned)g1, TB, 0, s>>>(n_cells, cells, nx, ny, h, (const double*)alpha1,
                                                             (const double*)alpha2, kappa, gamma1, gamma2,
                                                             tol, mode, uniform, amat, n_nonuniform);
        note_launch();
        k_refine_sub<double><<<(unsigned)g2, TB, 0, s>>>(n_cells, k, cells, nx, x0, y0, h,
                                                           (const double*)alpha1, (const double*)alpha2, uniform,
                                                           amat, (double2*)y_sub);
        note_launch();
    }
    LENS_CUDA(cudaGetLastError());
    return LENS_OK;
}
