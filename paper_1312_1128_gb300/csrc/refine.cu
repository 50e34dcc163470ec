// refine.cu -- cell refinement by the linear lens equation (Sec. 3.4
// interpolation; magnification matrix from deflections, App. A).
//
// Rays sit on a uniform grid, ray (i, j) at (x0 + i h, y0 + j h), flat index
// i + nx j; each ray is the centre of a cell of side h whose neighbours are
// the edge-adjacent rays E, N, W, S.  Per cell the uniformity test and the
// magnification matrix A:
//   kappa/gamma mode: every neighbour's kappa, gamma1, gamma2 within tol of the
//     centre's; A = [[1 - kappa - gamma1, -gamma2], [-gamma2, 1 - kappa + gamma1]]
//     (Eq. magmatrix) at the centre;
//   deflection mode: for each neighbour pair not colinear with the centre
//     (E-N, N-W, W-S, S-E), A from the three points by the App. A solve of
//     dy = A dx with y = x - alpha; uniform if no element of A differs by more
//     than tol between the pairs; A = their average.
// Then, per sub-cell centre, y = y_c + A (x - x_c) (Eq. linear_lens_equation)
// for uniform cells and NaN otherwise.  One kernel does both: a block first
// evaluates its cells (one thread per cell) into shared memory, then writes
// the block's contiguous run of sub-cell positions with all its threads, so
// every 32-byte sector of the dominant output is written whole, once.
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

constexpr int kRefineBlock = 256;  // cells (and threads) per block

// Sub-cell offsets (a - (k-1)/2) h / k, rounded once on the host.
struct SubOffsets {
    float d[kRefineMaxK];
};

// K > 0: k fixed at compile time (divisions by constants); K = 0: any odd k.
template <typename TA, typename I, int K>
__global__ void __launch_bounds__(kRefineBlock, 4)
k_refine(int64_t n_cells, const int64_t* cells, I nx, I ny, double x0, double y0, double h, int k_rt,
         SubOffsets off, const TA* a1, const TA* a2, const float* ka, const float* g1, const float* g2, double tol,
         int mode, uint8_t* uniform, float* amat, double2* y_sub, unsigned long long* n_nonuniform)
{
    __shared__ float sA[kRefineBlock][4];
    __shared__ double2 sY[kRefineBlock];
    __shared__ uint8_t sU[kRefineBlock];
    const int64_t c0 = (int64_t)blockIdx.x * kRefineBlock;
    const int64_t c = c0 + threadIdx.x;
    if (c < n_cells) {
        // cells == NULL: every interior cell, row by row
        const int64_t id64 = cells ? cells[c] : (c % (nx - 2) + 1) + (int64_t)nx * (c / (nx - 2) + 1);
        const bool in_range = id64 >= nx + 1 && id64 < (int64_t)nx * (ny - 1) - 1;
        const I id = in_range ? (I)id64 : I(0);
        const I i = id % nx, j = id / nx;
        float A[4] = {NAN, NAN, NAN, NAN};
        uint8_t u = 2;  // not an interior cell of the grid
        double2 yc = make_double2(NAN, NAN);
        if (in_range && i >= 1 && i <= nx - 2) {
            const I nb[4] = {id + 1, id + nx, id - 1, id - nx};  // E, N, W, S
            const TA ac1 = a1[id], ac2 = a2[id];
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
                // in the precision of the deflections (FP64 deflections keep
                // the differences between neighbours, the reason App. A exists)
                using C = TA;
                const C hh = (C)h;
                const C dxa[4] = {hh, C(0), -hh, C(0)}, dxb[4] = {C(0), hh, C(0), -hh};
                C dya[4], dyb[4];
#pragma unroll
                for (int n = 0; n < 4; ++n) {
                    dya[n] = dxa[n] - (a1[nb[n]] - ac1);
                    dyb[n] = dxb[n] - (a2[nb[n]] - ac2);
                }
                C lo[4], hi[4], sum[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const int pu = p, pv = (p + 1) & 3;  // E-N, N-W, W-S, S-E
                    C Ap[4];
                    app_a<C>(dxa[pu], dxb[pu], dya[pu], dyb[pu], dxa[pv], dxb[pv], dya[pv], dyb[pv], Ap);
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
            u = uni ? 1 : 0;
            if (uni) yc = make_double2((x0 + (double)i * h) - (double)ac1, (y0 + (double)j * h) - (double)ac2);
            else if (n_nonuniform)
                atomicAdd(n_nonuniform, 1ull);
        }
        uniform[c] = u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            amat[4 * c + q] = A[q];
            sA[threadIdx.x][q] = A[q];
        }
        sU[threadIdx.x] = u;
        sY[threadIdx.x] = yc;
    }
    __syncthreads();
    // the block's sub-cells, in output order
    const int k = K > 0 ? K : k_rt;
    const int kk = k * k;
    const int nc = (int)(n_cells - c0 < kRefineBlock ? n_cells - c0 : kRefineBlock);
    double2* out = y_sub + c0 * kk;
    for (int e = threadIdx.x; e < nc * kk; e += kRefineBlock) {
        const int cl = e / kk, s = e - cl * kk;
        double2 y = make_double2(NAN, NAN);
        if (sU[cl] == 1) {
            const float da = off.d[s % k], db = off.d[s / k];
            const float* A = sA[cl];
            y = make_double2(sY[cl].x + (double)fmaf(A[0], da, A[1] * db),
                             sY[cl].y + (double)fmaf(A[2], da, A[3] * db));
        }
        out[e] = y;
    }
}

template <typename TA, typename I, int K>
static void launch_refine(int64_t grid, cudaStream_t s, int64_t n_cells, const int64_t* cells, int64_t nx,
                          int64_t ny, double x0, double y0, double h, int k, const SubOffsets& off,
                          const void* a1, const void* a2, const float* ka, const float* g1, const float* g2,
                          double tol, int mode, uint8_t* uniform, float* amat, double* y_sub,
                          unsigned long long* n_nonuniform)
{
    k_refine<TA, I, K><<<(unsigned)grid, kRefineBlock, 0, s>>>(n_cells, cells, (I)nx, (I)ny, x0, y0, h, k, off,
                                                               (const TA*)a1, (const TA*)a2, ka, g1, g2, tol, mode,
                                                               uniform, amat, (double2*)y_sub, n_nonuniform);
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
    if (!alpha1 || !alpha2 || !uniform || !amat || !y_sub) return lens_set_error(LENS_ERR_INVALID_ARG, "NULL array");
    if (!cells && n_cells != (nx - 2) * (ny - 2))
        return lens_set_error(LENS_ERR_INVALID_ARG, "cells == NULL needs n_cells = (nx - 2)(ny - 2)");
    if (mode == LENS_REFINE_KAPPA_GAMMA && (!kappa || !gamma1 || !gamma2))
        return lens_set_error(LENS_ERR_INVALID_ARG, "kappa/gamma mode needs kappa, gamma1 and gamma2");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t grid = (n_cells + kRefineBlock - 1) / kRefineBlock;
    SubOffsets off{};
    for (int a = 0; a < k; ++a) off.d[a] = (float)(((double)a - 0.5 * (k - 1)) * h / k);
    // 32-bit index arithmetic whenever the grid's indices fit; k = 3 (the
    // paper's one-third refinement) specialised
    const bool small = nx * ny < ((int64_t)1 << 31);
    if (alpha_dtype == LENS_F32) {
        if (small && k == 3)
            launch_refine<float, int32_t, 3>(grid, s, n_cells, cells, nx, ny, x0, y0, h, k, off, alpha1, alpha2,
                                             kappa, gamma1, gamma2, tol, mode, uniform, amat, y_sub, n_nonuniform);
        else if (small)
            launch_refine<float, int32_t, 0>(grid, s, n_cells, cells, nx, ny, x0, y0, h, k, off, alpha1, alpha2,
                                             kappa, gamma1, gamma2, tol, mode, uniform, amat, y_sub, n_nonuniform);
        else
            launch_refine<float, int64_t, 0>(grid, s, n_cells, cells, nx, ny, x0, y0, h, k, off, alpha1, alpha2,
                                             kappa, gamma1, gamma2, tol, mode, uniform, amat, y_sub, n_nonuniform);
    } else {
        if (small && k == 3)
            launch_refine<double, int32_t, 3>(grid, s, n_cells, cells, nx, ny, x0, y0, h, k, off, alpha1, alpha2,
                                              kappa, gamma1, gamma2, tol, mode, uniform, amat, y_sub, n_nonuniform);
        else if (small)
            launch_refine<double, int32_t, 0>(grid, s, n_cells, cells, nx, ny, x0, y0, h, k, off, alpha1, alpha2,
                                              kappa, gamma1, gamma2, tol, mode, uniform, amat, y_sub, n_nonuniform);
        else
            launch_refine<double, int64_t, 0>(grid, s, n_cells, cells, nx, ny, x0, y0, h, k, off, alpha1, alpha2,
                                              kappa, gamma1, gamma2, tol, mode, uniform, amat, y_sub, n_nonuniform);
    }
    note_launch();
    LENS_CUDA(cudaGetLastError());
    return LENS_OK;
}
