// psi.cu -- the lensing potential psi with the deflection (Eq. alpha, Eq.
// timedelay: delta t = |alpha|^2 / 2 - psi), by the same tree walk as the
// other lensing quantities: far cells add the monopole + quadrupole potential
// (the multipole ln terms), leaves their particles' potentials, visited big
// lists (full - softened point) for the rays inside the support, and every
// ray the analytic halos.  One warp per group of rays; the traversal, the
// buffers and their appends are those of the walk (walk_dev.cuh), only the
// evaluation differs.  psi is Neumaier-compensated like the other outputs.
#include <algorithm>
#include <cmath>

#include "potential.cuh"
#include "walk_dev.cuh"

namespace lens {

template <typename T> struct PsiConsts {
    T EinU;  // Ein(q^2/2) of the species (Gaussian)
    T HX;    // H(R_max / r_s) of the species (NFW)
    T A0;    // N_q ln U_q - Ein(U_q) (Gaussian)
    int series;  // 2: U_q <= 4.5, Ein by the degree-9 polynomial; 1: U_q <= 5, by the 20-term series
};

LENS_DEV float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int k> LENS_DEV float2 ein_horner2(float2 u, float2 s)
{
    if constexpr (k < 0) {
        return s;
    } else {
        constexpr float c = float(ein_coef(k));
        return ein_horner2<k - 1>(u, __ffma2_rn(s, u, make_float2(c, c)));
    }
}

// Ein(u) for u < 5 on a pair, the 20-term series of ein<float>
LENS_DEV float2 ein_series2(float2 u)
{
    constexpr float top = float(ein_coef(19));
    return __fmul2_rn(ein_horner2<18>(u, make_float2(top, top)), u);
}

template <int k> LENS_DEV float2 ein_cheb2(float2 t, float2 s)
{
    if constexpr (k < 0) {
        return s;
    } else {
        constexpr float c = float(ein_cheb_coef(k));
        return ein_cheb2<k - 1>(t, __ffma2_rn(s, t, make_float2(c, c)));
    }
}

// Ein(u) for u <= 4.5 on a pair: u p(u - 9/4)
LENS_DEV float2 ein_poly2(float2 u)
{
    constexpr float top = float(ein_cheb_coef(9)), mid = float(0.5 * kEinChebMax);
    const float2 t = __fadd2_rn(u, make_float2(-mid, -mid));
    return __fmul2_rn(ein_cheb2<8>(t, make_float2(top, top)), u);
}

template <int KIND, typename T, int R> struct PsiCtx {
    using value_type = T;
    using Buf = WalkBuf<KIND, T>;
    static constexpr int kKind = KIND;
    static constexpr int kNear = Buf::kNear, kBig = Buf::kBig;
    const WalkParams<T>& P;
    const PsiConsts<T> K;
    WalkBuf<KIND, T>* B;
    WalkRanges* Rg;
    v2_t<T> H;
    vec4_t<T> box;
    int nf = 0, nn = 0, nb = 0;
    uint32_t* rec = nullptr;  // (the potential keeps no interaction lists)
    int rec_n = 0, rec_cap = 0;
    T lx[R], ly[R];
    T part[R][3];              // psi, alpha1, alpha2 of the current flush
    T tot_s[R][3], tot_c[R][3];  // compensated totals

    LENS_DEV PsiCtx(const WalkParams<T>& p, const PsiConsts<T>& k, WalkShared<KIND, T>& s)
        : P(p), K(k), B(&s.buf), Rg(&s.rng) {}

    LENS_DEV void zero()
    {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q) part[r][q] = tot_s[r][q] = tot_c[r][q] = T(0);
    }
    LENS_DEV void add(int r, T wx, T wy, T psi, T kb)
    {
        part[r][0] += psi;
        part[r][1] = fma(kb, wx, part[r][1]);
        part[r][2] = fma(kb, wy, part[r][2]);
    }
    LENS_DEV void fold()
    {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                Comp5<T>::add1(tot_s[r][q], tot_c[r][q], part[r][q]);
                part[r][q] = T(0);
            }
    }

    LENS_DEV void flush_far()
    {
        for (int c = 0; c < nf; ++c) {
            const T dx = B->fdx[c], dy = B->fdy[c], M = B->fM[c], qr = B->fqr[c], qi = B->fqi[c];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                T psi, a1, a2;
                psi_cell(lx[r] - dx, ly[r] - dy, M, qr, qi, psi, a1, a2);
                part[r][0] += psi;
                part[r][1] += a1;
                part[r][2] += a2;
            }
        }
        fold();
        nf = 0;
    }

    // full profile, or a listed particle as a point softened within r0
    LENS_DEV void particle(int r, const vec4_t<T>& q, const vec4_t<T>& q1)
    {
        const T wx = lx[r] - q.x, wy = ly[r] - q.y, r2 = fma(wx, wx, wy * wy);
        T psi, kb;
        if (KIND == LENS_POINT || q.w <= T(0)) {
            psi_point(q.z, r2, KIND == LENS_POINT ? T(0) : -q.w, psi, kb);
        } else if (KIND == LENS_GAUSS) {
            psi_gauss(q.z, q.w, r2, P.Uq, P.invNq, K.EinU, psi, kb);
        } else {
            psi_nfw(q.z, q.w, q1.x, q1.y, K.HX, r2, psi, kb);
        }
        add(r, wx, wy, psi, kb);
    }

    LENS_DEV void flush_near()
    {
        for (int i = 0; i < nn; ++i) {
            const vec4_t<T> q = B->n0[i];
            vec4_t<T> q1{};
            if constexpr (KIND == LENS_NFW) q1 = B->n1[i];
#pragma unroll
            for (int r = 0; r < R; ++r) particle(r, q, q1);
        }
        fold();
        nn = 0;
    }

    // (full profile - softened point) of one big entry at (x, y); w < 0 marks
    // an entry no ray of the group reaches inside its softening radius
    LENS_DEV void big_one(T x, T y, T m, T w, T c, T R2, T A, T Bs)
    {
        const T r0sq = w > T(0) ? T(1) / w : T(0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const T wx = lx[r] - x, wy = ly[r] - y, r2 = fma(wx, wx, wy * wy);
            T pf, kf, pp, kp;
            if (KIND == LENS_GAUSS) psi_gauss(m, c, r2, P.Uq, P.invNq, K.EinU, pf, kf);
            else psi_nfw(m, R2, A, Bs, K.HX, r2, pf, kf);
            psi_point(m, r2, r0sq, pp, kp);
            add(r, wx, wy, pf - pp, kf - kp);
        }
    }

    // One packed FP32 Gaussian entry (m' = m/N_q, c, w) for every ray, in the
    // closed form of (full - point) inside the support, u = c r^2 < U_q:
    //   psi: m'/2 (A0 + Ein(u) - N_q ln u),  kb: m' (e^-U_q - e^-u) / r^2;
    // a ray inside the softening radius (s = r^2 w < 1) adds the difference
    // of the softened point from the plain one: m'N_q/2 (ln s - s + 1) to psi
    // and m'N_q (1/r^2 - w) to kb.  Zero outside the support.
    LENS_DEV void big_packed(int i, float Nq)
    {
        const float nx = B->bnx[i], ny = B->bny[i], cl = B->bcl[i], mp = B->bm[i], nme = B->bme[i];
        const float w = B->bw[i];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float wx = lx[r] + nx, wy = ly[r] + ny, r2 = fmaf(wx, wx, wy * wy);
            const float t = r2 * cl;  // -u log2 e
            if (!(t > -P.Uq2)) continue;
            const float e = exp2_approx(t), u = t * -0.69314718055994530942f;
            const float E = ein(u);
            const float inv = r2 > 0.0f ? rcp(r2) : 0.0f;
            float kb = -fmaf(mp, e, nme) * inv;
            float psi = 0.5f * mp * fmaf(-Nq, __logf(u), K.A0 + E);
            const float sw = r2 * w;
            if (w > 0.0f && sw < 1.0f) {
                const float mq = mp * Nq;
                psi = 0.5f * mp * (K.A0 + E + Nq * (logf(w * B->bic[i]) - sw + 1.0f));
                kb = fmaf(mp, (1.0f - e) * inv, -mq * w);
            }
            part[r][0] += psi;
            part[r][1] = fmaf(kb, wx, part[r][1]);
            part[r][2] = fmaf(kb, wy, part[r][2]);
        }
    }

    // The same closed form on two entries (i, i+1) at once in FP32x2, every
    // ray beyond both softening radii (needs U_q <= 5).  P2 accumulates psi,
    // -alpha1, -alpha2 per entry slot.  EDGE: a ray may be outside a support,
    // where its terms are set to 0.
    template <bool EDGE, bool POLY>
    LENS_DEV void big_pair(int i, float2 (&P2)[R][3], const float2 (&LX)[R], const float2 (&LY)[R])
    {
        const float2 nx = *reinterpret_cast<const float2*>(&B->bnx[i]);
        const float2 ny = *reinterpret_cast<const float2*>(&B->bny[i]);
        const float2 cl = *reinterpret_cast<const float2*>(&B->bcl[i]);
        const float2 mp = *reinterpret_cast<const float2*>(&B->bm[i]);
        const float2 nme = *reinterpret_cast<const float2*>(&B->bme[i]);
        const float2 hmp = __fmul2_rn(mp, make_float2(0.5f, 0.5f));
        const float nUq2 = -P.Uq2, nNqL = -P.Nq * 0.69314718055994530942f;
        const float2 A0 = make_float2(K.A0, K.A0);
        constexpr float nL = -0.69314718055994530942f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 wx = __fadd2_rn(LX[r], nx), wy = __fadd2_rn(LY[r], ny);
            const float2 r2 = __ffma2_rn(wx, wx, __fmul2_rn(wy, wy));
            const float2 t = __fmul2_rn(r2, cl);
            float2 tc = t;
            if (EDGE) {
                tc.x = fmaxf(t.x, nUq2);
                tc.y = fmaxf(t.y, nUq2);
            }
            const float2 e = make_float2(exp2_approx(tc.x), exp2_approx(tc.y));
            const float2 u = __fmul2_rn(tc, make_float2(nL, nL));
            const float2 E = POLY ? ein_poly2(u) : ein_series2(u);
            const float2 inv = make_float2(rcp(r2.x), rcp(r2.y));
            float2 nkb = __fmul2_rn(__ffma2_rn(mp, e, nme), inv);
            const float2 lg = make_float2(lg2_approx(u.x), lg2_approx(u.y));
            float2 psi = __fmul2_rn(hmp, __ffma2_rn(make_float2(nNqL, nNqL), lg, __fadd2_rn(A0, E)));
            if (EDGE) {
                const bool ix = t.x > nUq2, iy = t.y > nUq2;
                psi = make_float2(ix ? psi.x : 0.0f, iy ? psi.y : 0.0f);
                nkb = make_float2(ix ? nkb.x : 0.0f, iy ? nkb.y : 0.0f);
            }
            P2[r][0] = __fadd2_rn(P2[r][0], psi);
            P2[r][1] = __ffma2_rn(nkb, wx, P2[r][1]);
            P2[r][2] = __ffma2_rn(nkb, wy, P2[r][2]);
        }
    }

    // Packed FP32 Gaussian buffer: the whole-group-inside region pair by pair
    // without tests, then the edge region pair by pair where both entries
    // have every ray beyond their softening radii, else entry by entry.
    template <bool POLY> LENS_DEV void flush_big_pairs(int nbuf, float Nq)
    {
        const int n_in = nbuf & 0xffff, n_out = nbuf >> 16;
        float2 P2[R][3], LX[R], LY[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            LX[r] = make_float2(lx[r], lx[r]);
            LY[r] = make_float2(ly[r], ly[r]);
#pragma unroll
            for (int q = 0; q < 3; ++q) P2[r][q] = make_float2(0.0f, 0.0f);
        }
        int i = 0;
        for (; i + 1 < n_in; i += 2) big_pair<false, POLY>(i, P2, LX, LY);
        if (i < n_in) big_packed(i, Nq);
        i = kBigCap - n_out;
        if ((i & 1) && i < kBigCap) big_packed(i++, Nq);
        for (; i + 1 < kBigCap; i += 2) {
            const float2 w = *reinterpret_cast<const float2*>(&B->bw[i]);
            if (w.x < 0.0f && w.y < 0.0f) {
                big_pair<true, POLY>(i, P2, LX, LY);
            } else {
                big_packed(i, Nq);
                big_packed(i + 1, Nq);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            part[r][0] += P2[r][0].x + P2[r][0].y;
            part[r][1] -= P2[r][1].x + P2[r][1].y;
            part[r][2] -= P2[r][2].x + P2[r][2].y;
        }
    }

    LENS_DEV void flush_big()
    {
        if constexpr (KIND != LENS_POINT) {
            const T Nq = P.invNq > T(0) ? T(1) / P.invNq : T(0);
            if constexpr (WalkBuf<KIND, T>::kPackedBig) {
                if (K.series == 2) {
                    flush_big_pairs<true>(nb, Nq);
                } else if (K.series == 1) {
                    flush_big_pairs<false>(nb, Nq);
                } else {
                    const int n_in = nb & 0xffff, n_out = nb >> 16;
                    for (int i = 0; i < n_in; ++i) big_packed(i, Nq);
                    for (int i = kBigCap - n_out; i < kBigCap; ++i) big_packed(i, Nq);
                }
            } else {
                for (int i = 0; i < nb; ++i) {
                    const vec4_t<T> q = B->b0[i], q1 = B->b1[i];
                    if (KIND == LENS_GAUSS) big_one(q.x, q.y, q1.x * Nq, q.w, T(1) / q1.w, T(0), T(0), T(0));
                    else big_one(q.x, q.y, q1.x, q.w, T(0), q.z, q1.y, q1.z);
                }
            }
        }
        fold();
        nb = 0;
    }

    LENS_DEV void halos()
    {
        for (int h = 0; h < P.n_halos; ++h) {
            const HaloDev& hd = P.halos[h];
            const T hx = (T)((double)H.x - hd.x), hy = (T)((double)H.y - hd.y), m = (T)hd.m;
            T EinU = T(0), HX = T(0);
            if (hd.kind == LENS_GAUSS) EinU = ein((T)hd.c1);
            if (hd.kind == LENS_NFW) HX = nfw_H((T)(hd.p1 / hd.p0));
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const T wx = lx[r] + hx, wy = ly[r] + hy, r2 = fma(wx, wx, wy * wy);
                T psi = T(0), kb = T(0);
                if (hd.kind == LENS_POINT) {
                    psi_point(m, r2, T(0), psi, kb);
                } else if (hd.kind == LENS_GAUSS) {
                    psi_gauss(m, (T)hd.c0, r2, (T)hd.c1, (T)hd.c2, EinU, psi, kb);
                } else if (hd.kind == LENS_NFW) {
                    psi_nfw(m, (T)hd.c2, (T)hd.c0, (T)hd.c1, HX, r2, psi, kb);
                } else if (hd.kind == LENS_SIS) {
                    const T rr = sqrt(r2), re = (T)hd.p0;
                    psi = re * rr;
                    kb = rr > T(0) ? re / rr : T(0);
                } else {  // uniform disk: a point softened within R
                    psi_point(m, r2, (T)hd.c2, psi, kb);
                }
                add(r, wx, wy, psi, kb);
            }
        }
        fold();
    }
};

template <int KIND, typename T, int R, bool DIRECT>
__global__ void __launch_bounds__(kWalkWarps * 32) psi_kernel(WalkParams<T> P, PsiConsts<T> K)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned full = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WalkShared<KIND, T>& S = reinterpret_cast<WalkShared<KIND, T>*>(smem_raw)[warp];
    int* stack = P.stack + ((int64_t)blockIdx.x * kWalkWarps + warp) * kStackCap;
    PsiCtx<KIND, T, R> C(P, K, S);
    uint32_t ridx[R];
    bool rv[R];
    for (;;) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(P.counter, 1u);
        g = __shfl_sync(full, g, 0);
        if ((int64_t)g >= P.n_groups) break;
        C.H = P.gH[g];
        C.box = P.gbox[g];
        const uint2 rg = P.grange[g];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = r * 32 + lane;
            rv[r] = k < (int)rg.y;
            if (rv[r]) {
                const v2_t<T> l = P.ray_l[rg.x + k];
                C.lx[r] = l.x;
                C.ly[r] = l.y;
                ridx[r] = P.ray_idx[rg.x + k];
            } else {
                C.lx[r] = C.box.x;
                C.ly[r] = C.box.y;
                ridx[r] = 0;
            }
        }
        C.zero();
        C.nf = C.nn = C.nb = 0;
        int c_vis = 0, c_acc = 0, c_near = 0, c_bigs = 0, c_bigk = 0, c_dummy = 0;
        if (P.n_part > 0) {
            if (DIRECT) {
                for (int64_t base = 0; base < P.n_part; base += 0x40000000) {
                    const int64_t rem = P.n_part - base;
                    const int c = (int)(rem < 0x40000000 ? rem : 0x40000000);
                    append_ranges(C, lane == 0 ? c : 0, (int)base, P.leaf0, P.leaf1, c_near, c_dummy);
                }
                C.flush_near();
            } else {
                traverse(C, stack, c_vis, c_acc, c_near, c_bigs, c_bigk);
                C.flush_far();
                C.flush_near();
                C.flush_big();
            }
        }
        if (P.n_halos > 0) C.halos();
        if (P.stats && lane == 0) {
            const unsigned long long nr = rg.y;
            atomicAdd(&P.stats[0], 1ull);
            atomicAdd(&P.stats[1], (unsigned long long)c_vis);
            atomicAdd(&P.stats[2], (unsigned long long)c_acc);
            atomicAdd(&P.stats[3], (unsigned long long)c_near);
            atomicAdd(&P.stats[4], (unsigned long long)c_bigs);
            atomicAdd(&P.stats[5], (unsigned long long)c_bigk);
            atomicAdd(&P.stats[6], nr * (unsigned long long)(c_acc + c_near + c_bigk));
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!rv[r]) continue;
            const uint32_t i = ridx[r];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (!P.out[q]) continue;
                T val = C.tot_s[r][q] + C.tot_c[r][q];
                if (P.accumulate) val += P.out[q][i];
                P.out[q][i] = val;
            }
        }
        __syncwarp();
    }
}

template <int KIND, typename T, int R, bool DIRECT>
static void psi_launch_one(const WalkParams<T>& P, const PsiConsts<T>& K, int num_sms, cudaStream_t s)
{
    const size_t smem = kWalkWarps * sizeof(WalkShared<KIND, T>);
    static int bps = -1;
    if (bps < 0) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(psi_kernel<KIND, T, R, DIRECT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, psi_kernel<KIND, T, R, DIRECT>, kWalkWarps * 32, smem);
        bps = std::min(std::max(nb, 1), 16);  // stacks are allocated for 16 blocks per SM
    }
    { psi_kernel<KIND, T, R, DIRECT><<<num_sms * bps, kWalkWarps * 32, smem, s>>>(P, K); note_launch(); }
}

template <typename T, int R, bool DIRECT>
static void psi_launch_kind(int kind, const WalkParams<T>& P, const PsiConsts<T>& K, int num_sms, cudaStream_t s)
{
    if (kind == LENS_POINT) psi_launch_one<LENS_POINT, T, R, DIRECT>(P, K, num_sms, s);
    else if (kind == LENS_GAUSS) psi_launch_one<LENS_GAUSS, T, R, DIRECT>(P, K, num_sms, s);
    else psi_launch_one<LENS_NFW, T, R, DIRECT>(P, K, num_sms, s);
}

// Host values of the per-species constants (FP64).
static double host_nfw_H(double x)
{
    if (x <= 0.0) return 0.0;
    const double u = 1.0 - x * x;
    if (x < 0.5) {
        const double t = std::sqrt(u), L = std::log(2.0 / x), e = std::log1p(-x * x / (2.0 * (1.0 + t)));
        return -0.5 * e * (2.0 * L + e);
    }
    double F;
    if (std::fabs(u) < 1e-4) {
        double p = 1.0;
        F = 0.0;
        for (int k = 0; k < 10; ++k) {
            F += p / (2 * k + 1);
            p *= u;
        }
    } else if (x < 1.0) {
        F = std::acosh(1.0 / x) / std::sqrt(u);
    } else {
        F = std::acos(1.0 / x) / std::sqrt(-u);
    }
    const double lx = std::log(0.5 * x);
    return 0.5 * lx * lx - 0.5 * u * F * F;
}

template <typename T>
static lens_status psi_typed(lens_tree* t, const ShootPlan& plan, const void* dx, const void* dy, int dtype,
                             void* const out[3], int flags, cudaStream_t s)
{
    using T4 = vec4_t<T>;
    using T2 = v2_t<T>;
    Layout L = make_layout(t->ray_cap, t->batch_cap, max_slots(t));
    char* base = (char*)t->ray_scratch.ptr;
    const bool timing = (flags & LENS_TIMING) != 0;
    if (timing) {
        for (int i = 0; i < 4; ++i)
            if (!t->ev[i]) LENS_CUDA(cudaEventCreate(&t->ev[i]));
        LENS_CUDA(cudaEventRecord(t->ev[0], s));
    }
    if (plan.n > 0) LENS_TRY(enqueue_groups<T>(t, plan, dx, dy, dtype, s));
    if (timing) LENS_CUDA(cudaEventRecord(t->ev[1], s));
    LENS_TRY(wait_built(t, s));  // the grouping reads only the rays
    if (timing) LENS_CUDA(cudaEventRecord(t->ev[2], s));
    WalkParams<T> P{};
    P.gH = (T2*)(base + L.gH);
    P.gbox = (T4*)(base + L.gbox);
    P.grange = (uint2*)(base + L.grange);
    P.ray_l = (T2*)(base + L.rl);
    P.ray_idx = (uint32_t*)(base + L.ridx);
    P.n_groups = (int64_t)plan.ng;
    P.stack = (int*)(base + L.stack);
    P.err = t->d_err;
    P.stats = (flags & LENS_COUNT) ? t->d_stats : nullptr;
    for (int q = 0; q < 3; ++q) P.out[q] = (T*)out[q];
    P.out[3] = P.out[4] = nullptr;
    uint32_t* counter = (uint32_t*)(base + L.counter);
    const bool direct = (flags & LENS_DIRECT) != 0;
    bool first = true;
    int launches = 0;
    auto launch = [&](int kind, const PsiConsts<T>& K) {
        P.counter = counter + 2 * launches;
        cudaMemsetAsync(P.counter, 0, sizeof(uint32_t), s);
        if (plan.n == 0) return;
        if (plan.R == 1) {
            if (direct) psi_launch_kind<T, 1, true>(kind, P, K, t->num_sms, s);
            else psi_launch_kind<T, 1, false>(kind, P, K, t->num_sms, s);
        } else {
            if (direct) psi_launch_kind<T, 2, true>(kind, P, K, t->num_sms, s);
            else psi_launch_kind<T, 2, false>(kind, P, K, t->num_sms, s);
        }
    };
    for (const SpeciesTree& st : t->sp) {
        if (st.n == 0) continue;
        P.nodeA = (const T4*)st.nodeA;
        P.nodeB = (const T2*)st.nodeB;
        P.link = st.link;
        P.leaf0 = (const T4*)((direct || st.kind == LENS_POINT) ? st.exact0 : st.leaf0);
        P.leaf1 = (const T4*)st.exact1;
        P.big0 = (const T4*)st.big0;
        P.big1 = (const T4*)st.big1;
        P.big_chunk = (const T4*)st.big_chunk;
        P.node_bigbox = (const T4*)st.node_bigbox;
        P.n_part = st.n;
        P.Uq = (T)st.Uq;
        P.invNq = (T)st.invNq;
        P.Uq2 = (T)(st.Uq * 1.4426950408889634074);
        P.Nq = (T)(st.invNq > 0 ? 1.0 / st.invNq : 0.0);
        P.eU = (T)std::exp(-st.Uq);
        P.halos = t->halos;
        P.n_halos = first ? (int)t->n_halos : 0;
        P.accumulate = first ? ((flags & LENS_ACCUMULATE) ? 1 : 0) : 1;
        PsiConsts<T> K{};
        if (st.kind == LENS_GAUSS) {
            K.EinU = (T)ein<double>(st.Uq);
            K.A0 = (T)((1.0 - std::exp(-st.Uq)) * std::log(st.Uq) - ein<double>(st.Uq));
            K.series = st.Uq <= kEinChebMax ? 2 : (st.Uq <= 5.0 ? 1 : 0);
        }
        if (st.kind == LENS_NFW) K.HX = (T)host_nfw_H(st.shape);
        launch(st.kind, K);
        first = false;
        ++launches;
    }
    if (first) {  // analytic components only
        P.n_part = 0;
        P.halos = t->halos;
        P.n_halos = (int)t->n_halos;
        P.accumulate = (flags & LENS_ACCUMULATE) ? 1 : 0;
        launch(LENS_POINT, PsiConsts<T>{});
    }
    if (timing) {
        LENS_CUDA(cudaEventRecord(t->ev[3], s));
        t->timed = true;
    }
    LENS_CUDA(cudaGetLastError());
    return LENS_OK;
}

}  // namespace lens

using namespace lens;

extern "C" lens_status lens_shoot_potential(lens_tree* tree, double origin_x, double origin_y, const void* ray_dx,
                                            const void* ray_dy, int32_t ray_dtype, int64_t n, void* psi,
                                            void* alpha1, void* alpha2, int32_t flags, void* stream)
{
    if (!tree) return lens_set_error(LENS_ERR_INVALID_ARG, "tree is NULL");
    if (n < 0) return lens_set_error(LENS_ERR_INVALID_ARG, "n < 0");
    if (ray_dtype != LENS_F32 && ray_dtype != LENS_F64) return lens_set_error(LENS_ERR_INVALID_ARG, "bad ray dtype");
    if (flags & ~(LENS_DIRECT | LENS_ACCUMULATE | LENS_TIMING | LENS_COUNT))
        return lens_set_error(LENS_ERR_INVALID_ARG, "lens_shoot_potential takes LENS_DIRECT, LENS_ACCUMULATE, "
                                                    "LENS_TIMING and LENS_COUNT only");
    if (n == 0) return LENS_OK;
    if (!ray_dx || !ray_dy || !psi) return lens_set_error(LENS_ERR_INVALID_ARG, "NULL ray or psi array");
    if (!std::isfinite(origin_x) || !std::isfinite(origin_y))
        return lens_set_error(LENS_ERR_INVALID_ARG, "non-finite origin");
    cudaStream_t s = (cudaStream_t)stream;
    ShootPlan plan;
    const int64_t off[2] = {0, n};
    const double orig[2] = {origin_x, origin_y};
    LENS_TRY(upload_batches(tree, 1, off, orig, s, &plan));
    void* out[3] = {psi, alpha1, alpha2};
    if (tree->precision == LENS_PREC_FP64) return psi_typed<double>(tree, plan, ray_dx, ray_dy, ray_dtype, out, flags, s);
    return psi_typed<float>(tree, plan, ray_dx, ray_dy, ray_dtype, out, flags, s);
}
