// backward.cu -- adjoint of the tree walk: gradient of a loss of the
// deflection with respect to particle masses and positions and halo
// parameters (no counterpart in the paper; it differentiates the tree
// approximation of Sec. 3.2 that the forward walk computes).
//
// The rays are grouped exactly as in the forward call and every group walks
// the tree with the same acceptance tests, so it meets the same accepted
// cells, opened leaves and big-list entries.  The buffers are evaluated
// transposed: each lane owns one buffered entry (cell or particle) and loops
// over the group's rays, whose offsets and upstream gradients G = dL/dalpha
// sit in shared memory; a lane ends with its entry's gradient and adds it
// with one atomic per quantity.
//
//   particle terms (leaf particles, big-list corrections, halos): alpha is
//   linear in the mass, so dalpha/dm = alpha/m, and dalpha/dx_p = -J with J
//   the term's own Jacobian [[kappa+g1, g2], [g2, kappa-g1]] (Eqs. kappa,
//   gamma_1, gamma_2);
//   sizes: a profile of size s and fixed shape encloses Mt = m F(r/s), and
//   dMt/dr = 2 r kappa (m-units), so dMt/ds = -2 r^2 kappa / s and
//   dalpha/ds = -(2 kappa / s) w: a particle's size gradient is
//   -(2/s) sum kappa (G.w) over the rays inside its support (kappa = 0
//   outside).  Every such ray meets the particle's full profile in the walk
//   (a leaf, or the big list of a visited box), so the tree's size gradient
//   is the direct sum's.  Analytic halos add the derivatives of their other
//   shape parameters (q, R_max) through the enclosed mass the same way;
//   far cells, conj(alpha) = M/w + Q2/w^3 with w = x - x_cm: per cell the
//   adjoints a = dL/dM, C = dL/dQ2 and B = dL/dz_cm (dL = Re(G dA) with
//   A = conj(alpha)).  Since dM = dm_i, dz_cm = (dm_i d_i + m_i dz_i)/M and
//   dQ2 = dm_i d_i^2 + 2 m_i d_i dz_i (d_i = z_i - z_cm), a particle inside
//   the cell receives dL/dm_i = Re P(d_i) and dL/dz_i = m_i P'(d_i) with the
//   quadratic P(d) = a + (B/M) d + C d^2.  The polynomials of all accepted
//   ancestors are re-centred and summed from the root down, then evaluated at
//   every particle of every leaf.
#include <algorithm>
#include <cmath>

#include "profiles.cuh"
#include "walk_shared.cuh"

namespace lens {

template <typename T> struct BackParams {
    const vec4_t<T>* nodeA;
    const v2_t<T>* nodeB;
    const int4* link;
    const vec4_t<T>* leaf0;
    const vec4_t<T>* leaf1;
    const vec4_t<T>* big0;
    const vec4_t<T>* big1;
    const vec4_t<T>* big_chunk;
    const vec4_t<T>* node_bigbox;
    const uint32_t* big_pid;
    int64_t n_part;
    T Uq, invNq, Uq2, Nq, eU;
    const v2_t<T>* gH;
    const vec4_t<T>* gbox;
    const uint2* grange;
    const v2_t<T>* ray_l;
    const uint32_t* ray_idx;
    int64_t n_groups;
    const T* ga1;   // dL/dalpha1 per caller ray
    const T* ga2;
    const HaloDev* halos;
    int n_halos;
    double* ghalo;  // n_halos x 5 {dL/dm (dL/dr_E for the SIS), dL/dx, dL/dy, dL/dp0, dL/dp1}, or null
    double* adj;    // n_nodes x 5: dL/dM, dL/dQ2 (re, im), dL/dz_cm (re, im)
    double* gpart;  // n x 4 in tree order: dL/dm, dL/dx, dL/dy, sum kappa (G.w)
    // (FP64 accumulators: these sums run over up to millions of rays with
    // strong cancellation)
    uint32_t* counter;
    int* stack;
    uint32_t* err;
    const uint32_t* order;  // heaviest-first order of the groups, or null
    // split heavy groups (heavy_first_order): hdr {Kc, Hn} and Hn slice
    // entries, or null.  Every slice walks the group's tree and takes every
    // ns-th accepted cell, leaf particle and kept big-list entry: the
    // gradients are sums of atomics, so a slice needs no partial buffer.
    const uint32_t* heavy_hdr;
    const uint32_t* heavy;
    // the forward's kept interaction lists (LENS_KEEP_LISTS), or null: group
    // g replays list_ids[g * list_K ...] (list_n[g] entries) instead of
    // walking the tree, unless list_n[g] is kListOverflow
    const uint32_t* list_ids;
    const uint32_t* list_n;
    int list_K;
};

constexpr int kMaxGroup = 64;
// The adjoint's leaf and big-list buffers (entries per warp).  Halving them
// raises the occupancy from five to seven blocks per SM but did not speed
// the lens-fit adjoint up (4.0 against 3.9 ms): it is not occupancy-bound.
constexpr int kBackNear = kNearCap, kBackBig = kBigCap;

template <int KIND, typename T> struct BackShared {
    T rx[kMaxGroup], ry[kMaxGroup], rg1[kMaxGroup], rg2[kMaxGroup];
    // FP32: the rays in pairs for the packed (f32x2) far-cell adjoint:
    // pk_a[p] = (x_2p, x_2p+1, y_2p, y_2p+1), pk_b[p] = (g1, g1', g2, g2')
    // (an odd group's last pair repeats its first ray with zero gradient)
    float4 pk_a[sizeof(T) == 4 ? kMaxGroup / 2 : 1];
    float4 pk_b[sizeof(T) == 4 ? kMaxGroup / 2 : 1];
    T fdx[kFarCap], fdy[kFarCap], fM[kFarCap], fqr[kFarCap], fqi[kFarCap];
    int fnode[kFarCap];
    vec4_t<T> n0[kBackNear];
    vec4_t<T> n1[KIND == LENS_NFW ? kBackNear : 1];
    int npid[kBackNear];
    vec4_t<T> b0[KIND == LENS_POINT ? 1 : kBackBig];
    vec4_t<T> b1[KIND == LENS_POINT ? 1 : kBackBig];
    int bpid[KIND == LENS_POINT ? 1 : kBackBig];
    int rs_off[33];
    int rs_first[32];
    int rs_end[32];
};

// Gradient of the loss through one particle term (kb, kap, Dp) at offset w
// for upstream gradient (g1, g2): adds G.alpha_t (to be divided by m),
// -J^T G and kappa (G.w) (the size gradient's sum).
template <typename T>
LENS_DEV void term_grad(T wx, T wy, T kb, T kap, T Dp, T g1, T g2, T& gm, T& gx, T& gy, T& gk)
{
    T gw = fma(g1, wx, g2 * wy);
    T c2 = fma(wx, wx, -wy * wy), s2 = (wx + wx) * wy;
    T gg1 = -Dp * c2, gg2 = -Dp * s2;
    gm = fma(kb, gw, gm);
    gk = fma(kap, gw, gk);
    gx -= fma(g1, kap + gg1, g2 * gg2);
    gy -= fma(g1, gg2, g2 * (kap - gg1));
}

// Term values of the forward's leaf records and big-list corrections.
template <int KIND, typename T>
LENS_DEV void leaf_term(const BackParams<T>& P, const vec4_t<T>& q, const vec4_t<T>& q1, T r2, T& kb, T& kap,
                        T& Dp)
{
    kap = T(0);
    if constexpr (KIND == LENS_POINT) {
        point_terms(q.z, r2, kb, Dp);
    } else if constexpr (KIND == LENS_GAUSS) {
        if (q.w > T(0)) gauss_terms(q.z, q.w, r2, P.Uq, P.invNq, kb, kap, Dp);
        else point_terms(q.z, fmax(r2, -q.w), kb, Dp);
    } else {
        if (q.w > T(0)) nfw_terms(q.z, q.w, q1.x, q1.y, r2, kb, kap, Dp);
        else point_terms(q.z, fmax(r2, -q.w), kb, Dp);
    }
}

template <int KIND, typename T>
LENS_DEV void big_term(const BackParams<T>& P, const vec4_t<T>& q, const vec4_t<T>& q1, T r2, T& kb, T& kap,
                       T& Dp)
{
    if constexpr (KIND == LENS_GAUSS) {
        const T L = T(0.69314718055994530942);
        if (q.w < T(0)) {
            // no ray inside the softening radius: closed form of (full - point)
            T inv = rcp(r2);
            T t = r2 * q1.y;
            T e = exp2neg(fmin(t, P.Uq2));
            kb = (q1.x * inv) * (P.eU - e);
            kap = t < P.Uq2 ? q1.z * e : T(0);
            Dp = (kb - kap) * inv;
        } else {
            T inv = r2 > T(0) ? rcp(r2) : T(0);
            T inv_s = fmin(inv, q.w);
            T kbp = (q1.x * P.Nq) * inv_s;
            T t = r2 * q1.y;
            if (t < P.Uq2) {
                T u = t * L;
                T e = expneg(u), h1, g;
                gauss_h1_g(u, e, h1, g);
                kb = q1.z * h1 - kbp;
                kap = q1.z * e;
                Dp = (q1.z * g) * inv - kbp * inv_s;
            } else {
                kb = T(0);
                kap = T(0);
                Dp = T(0);
            }
        }
    } else {
        T inv = r2 > T(0) ? rcp(r2) : T(0);
        T inv_s = fmin(inv, q.w);
        T kbp = q1.x * inv_s;
        T kbe, kape, Dpe;
        nfw_terms(q1.x, q.z, q1.y, q1.z, r2, kbe, kape, Dpe);
        kb = kbe - kbp;
        kap = kape;
        Dp = Dpe - kbp * inv_s;
    }
}

template <int KIND, typename T> struct BackCtx {
    const BackParams<T>& P;
    BackShared<KIND, T>& S;
    int nr;  // rays in the group
    v2_t<T> H;
    vec4_t<T> box;
    int sl = 0, ns = 1;               // this item's slice of the group's work
    int seq_f = 0, seq_n = 0, seq_b = 0;  // cells, leaf particles, kept big entries met so far

    LENS_DEV BackCtx(const BackParams<T>& p, BackShared<KIND, T>& s) : P(p), S(s) {}

    // lane c owns far cells c, c + 32, ...: dL/dM, dL/dQ2, dL/dz_cm over the
    // group's rays (the buffer holds up to kFarCap cells when it is flushed)
    LENS_DEV void flush_far(int nf)
    {
        int lane = threadIdx.x & 31;
        __syncwarp();
        if constexpr (sizeof(T) == 4) {
            flush_far_packed(nf);
            return;
        }
        for (int cell = lane; cell < nf; cell += 32) {
            T dx = S.fdx[cell], dy = S.fdy[cell], M = S.fM[cell], qr = S.fqr[cell], qi = S.fqi[cell];
            T aM = T(0), cr = T(0), ci = T(0), br = T(0), bi = T(0);
            for (int j = 0; j < nr; ++j) {
                T wx = S.rx[j] - dx, wy = S.ry[j] - dy;
                T g1 = S.rg1[j], g2 = S.rg2[j];
                T inv = rcp(fma(wx, wx, wy * wy));
                T ux = wx * inv, uy = -wy * inv;
                T u2x = fma(ux, ux, -uy * uy), u2y = (ux + ux) * uy;
                T u3x = fma(u2x, ux, -u2y * uy), u3y = fma(u2x, uy, u2y * ux);
                T u4x = fma(u2x, u2x, -u2y * u2y), u4y = (u2x + u2x) * u2y;
                // G = g1 + i g2 multiplies dA (A = conj(alpha)); dL = Re(G dA)
                aM += g1 * ux - g2 * uy;
                cr += g1 * u3x - g2 * u3y;
                ci += g1 * u3y + g2 * u3x;
                T tx = M * u2x + T(3) * (qr * u4x - qi * u4y), ty = M * u2y + T(3) * (qr * u4y + qi * u4x);
                br += g1 * tx - g2 * ty;
                bi += g1 * ty + g2 * tx;
            }
            double* a = P.adj + 5 * (int64_t)S.fnode[cell];
            atomicAdd(a + 0, (double)aM);
            atomicAdd(a + 1, (double)cr);
            atomicAdd(a + 2, (double)ci);
            atomicAdd(a + 3, (double)br);
            atomicAdd(a + 4, (double)bi);
        }
        __syncwarp();
    }

    // The same sums in FP32 two rays at a time (f32x2 multiply-adds): per ray
    // pair 19 packed FMA-pipe operations and two reciprocals.
    LENS_DEV void flush_far_packed(int nf)
    {
        const int lane = threadIdx.x & 31;
        const int np = (nr + 1) >> 1;
        const float2 M1 = make_float2(-1.f, -1.f);
        for (int cell = lane; cell < nf; cell += 32) {
            const float dx = (float)S.fdx[cell], dy = (float)S.fdy[cell], M = (float)S.fM[cell];
            const float qr = (float)S.fqr[cell], qi = (float)S.fqi[cell];
            const float2 NDX = make_float2(-dx, -dx), DY = make_float2(dy, dy), MM = make_float2(M, M);
            const float2 QR3 = make_float2(3.f * qr, 3.f * qr), QI3 = make_float2(3.f * qi, 3.f * qi);
            const float2 NQI3 = make_float2(-3.f * qi, -3.f * qi);
            float2 aM = make_float2(0.f, 0.f), cr = aM, ci = aM, br = aM, bi = aM;
            for (int p = 0; p < np; ++p) {
                const float4 A = S.pk_a[p], B = S.pk_b[p];
                const float2 G1 = make_float2(B.x, B.y), G2 = make_float2(B.z, B.w);
                const float2 NG2 = __fmul2_rn(G2, M1);
                const float2 wx = __fadd2_rn(make_float2(A.x, A.y), NDX);
                const float2 nwy = __ffma2_rn(make_float2(A.z, A.w), M1, DY);  // -(y - y_cell)
                const float2 r2 = __ffma2_rn(wx, wx, __fmul2_rn(nwy, nwy));
                const float2 inv = make_float2(rcp(r2.x), rcp(r2.y));
                // u = 1 / w and its powers
                const float2 ux = __fmul2_rn(wx, inv), uy = __fmul2_rn(nwy, inv);
                const float2 nuy = __fmul2_rn(uy, M1);
                const float2 u2x = __ffma2_rn(ux, ux, __fmul2_rn(uy, nuy));
                const float2 u2y = __fmul2_rn(__fadd2_rn(ux, ux), uy);
                const float2 u3x = __ffma2_rn(u2x, ux, __fmul2_rn(u2y, nuy));
                const float2 u3y = __ffma2_rn(u2x, uy, __fmul2_rn(u2y, ux));
                const float2 nu2y = __fmul2_rn(u2y, M1);
                const float2 u4x = __ffma2_rn(u2x, u2x, __fmul2_rn(u2y, nu2y));
                const float2 u4y = __fmul2_rn(__fadd2_rn(u2x, u2x), u2y);
                aM = __ffma2_rn(G1, ux, __ffma2_rn(NG2, uy, aM));
                cr = __ffma2_rn(G1, u3x, __ffma2_rn(NG2, u3y, cr));
                ci = __ffma2_rn(G1, u3y, __ffma2_rn(G2, u3x, ci));
                const float2 tx = __ffma2_rn(MM, u2x, __ffma2_rn(QR3, u4x, __fmul2_rn(NQI3, u4y)));
                const float2 ty = __ffma2_rn(MM, u2y, __ffma2_rn(QR3, u4y, __fmul2_rn(QI3, u4x)));
                br = __ffma2_rn(G1, tx, __ffma2_rn(NG2, ty, br));
                bi = __ffma2_rn(G1, ty, __ffma2_rn(G2, tx, bi));
            }
            double* a = P.adj + 5 * (int64_t)S.fnode[cell];
            atomicAdd(a + 0, (double)(aM.x + aM.y));
            atomicAdd(a + 1, (double)(cr.x + cr.y));
            atomicAdd(a + 2, (double)(ci.x + ci.y));
            atomicAdd(a + 3, (double)(br.x + br.y));
            atomicAdd(a + 4, (double)(bi.x + bi.y));
        }
        __syncwarp();
    }

    LENS_DEV void add_particle(int pid, T m, T gm, T gx, T gy, T gk)
    {
        double* g = P.gpart + 4 * (int64_t)pid;
        // dL/dm = gm / m in the working precision (an FP64 division is slow on
        // this GPU's FP64 pipe); accumulated in FP64
        if (m != T(0)) atomicAdd(g + 0, (double)(gm / m));
        atomicAdd(g + 1, (double)gx);
        atomicAdd(g + 2, (double)gy);
        if (gk != T(0)) atomicAdd(g + 3, (double)gk);
    }

    LENS_DEV void flush_near(int nn)
    {
        int lane = threadIdx.x & 31;
        __syncwarp();
        for (int i = lane; i < nn; i += 32) {
            vec4_t<T> q = S.n0[i], q1;
            if constexpr (KIND == LENS_NFW) q1 = S.n1[i];
            T gm = T(0), gx = T(0), gy = T(0), gk = T(0);
            for (int j = 0; j < nr; ++j) {
                T wx = S.rx[j] - q.x, wy = S.ry[j] - q.y;
                T r2 = fma(wx, wx, wy * wy), kb, kap, Dp;
                leaf_term<KIND, T>(P, q, q1, r2, kb, kap, Dp);
                term_grad(wx, wy, kb, kap, Dp, S.rg1[j], S.rg2[j], gm, gx, gy, gk);
            }
            add_particle(S.npid[i], q.z, gm, gx, gy, gk);
        }
        __syncwarp();
    }

    LENS_DEV void flush_big(int nb)
    {
        int lane = threadIdx.x & 31;
        __syncwarp();
        for (int i = lane; i < nb; i += 32) {
            vec4_t<T> q = S.b0[i], q1 = S.b1[i];
            T gm = T(0), gx = T(0), gy = T(0), gk = T(0);
            for (int j = 0; j < nr; ++j) {
                T wx = S.rx[j] - q.x, wy = S.ry[j] - q.y;
                T r2 = fma(wx, wx, wy * wy), kb, kap, Dp;
                big_term<KIND, T>(P, q, q1, r2, kb, kap, Dp);
                term_grad(wx, wy, kb, kap, Dp, S.rg1[j], S.rg2[j], gm, gx, gy, gk);
            }
            T m = KIND == LENS_GAUSS ? q1.x * P.Nq : q1.x;
            add_particle(S.bpid[i], m, gm, gx, gy, gk);
        }
        __syncwarp();
    }
};

// Same selection as the forward's leaf append, recording tree positions.
template <int KIND, typename T>
LENS_DEV void back_append_near(BackCtx<KIND, T>& C, int cnt, int first, int& nbuf, const vec4_t<T>* src0,
                               const vec4_t<T>* src1)
{
    int lane = threadIdx.x & 31;
    int tot;
    int off = warp_exclusive_scan(cnt, &tot);
    if (tot == 0) return;
    BackShared<KIND, T>& S = C.S;
    S.rs_off[lane] = off;
    S.rs_first[lane] = first;
    if (lane == 31) S.rs_off[32] = tot;
    __syncwarp();
    // a slice takes particles i = i0, i0 + ns, ... (its share of the group's sequence)
    int i0 = 0, cnt_s = tot;
    if (C.ns > 1) {
        i0 = (C.sl - C.seq_n % C.ns + C.ns) % C.ns;
        cnt_s = tot > i0 ? (tot - i0 + C.ns - 1) / C.ns : 0;
        C.seq_n += tot;
    }
    for (int base = 0; base < cnt_s; base += 32) {
        if (nbuf + 32 > kBackNear) {
            C.flush_near(nbuf);
            nbuf = 0;
        }
        int j = base + lane;
        if (j < cnt_s) {
            int i = i0 + j * C.ns;
            int lo = 0, hi = 32;
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (S.rs_off[mid] <= i) lo = mid;
                else hi = mid;
            }
            int p = S.rs_first[lo] + (i - S.rs_off[lo]);
            vec4_t<T> q0 = src0[p];
            q0.x -= C.H.x;
            q0.y -= C.H.y;
            S.n0[nbuf + lane] = q0;
            if constexpr (KIND == LENS_NFW) S.n1[nbuf + lane] = src1[p];
            S.npid[nbuf + lane] = p;
        }
        nbuf += cnt_s - base < 32 ? cnt_s - base : 32;
        __syncwarp();
    }
}

// Same selection as the forward's big-list append (two-level support boxes,
// per-entry support test, fast-path flag), recording tree positions.
template <int KIND, typename T>
LENS_DEV void back_append_big(BackCtx<KIND, T>& C, bool has, int v, int z, int w, int& nbuf)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const BackParams<T>& P = C.P;
    BackShared<KIND, T>& S = C.S;
    int cnt = 0;
    if (has) {
        vec4_t<T> nb4 = P.node_bigbox[v];
        if (box_reaches_group<T>(nb4, C.H, C.box)) cnt = ((z + w - 1) >> 5) - (z >> 5) + 1;
    }
    int tot;
    int off = warp_exclusive_scan(cnt, &tot);
    if (tot == 0) return;
    S.rs_off[lane] = off;
    S.rs_first[lane] = z;
    S.rs_end[lane] = z + w;
    if (lane == 31) S.rs_off[32] = tot;
    __syncwarp();
    for (int base = 0; base < tot; base += 32) {
        int i = base + lane;
        int cid = -1, own = 0;
        bool pass = false;
        if (i < tot) {
            int lo = 0, hi = 32;
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (S.rs_off[mid] <= i) lo = mid;
                else hi = mid;
            }
            own = lo;
            cid = (S.rs_first[lo] >> 5) + (i - S.rs_off[lo]);
            pass = box_reaches_group<T>(P.big_chunk[cid], C.H, C.box);
        }
        unsigned ball = __ballot_sync(full, pass);
        while (ball) {
            int src = __ffs(ball) - 1;
            ball &= ball - 1;
            int c = __shfl_sync(full, cid, src);
            int o = __shfl_sync(full, own, src);
            if (nbuf + 32 > kBackBig) {
                C.flush_big(nbuf);
                nbuf = 0;
            }
            int e = 32 * c + lane;
            bool keep = false;
            vec4_t<T> q0;
            if (e >= S.rs_first[o] && e < S.rs_end[o]) {
                q0 = P.big0[e];
                q0.x -= C.H.x;
                q0.y -= C.H.y;
                T ex = fmax(fabs(q0.x - C.box.x) - C.box.z, T(0));
                T ey = fmax(fabs(q0.y - C.box.y) - C.box.w, T(0));
                T near2 = fma(ex, ex, ey * ey);
                keep = near2 < q0.z;
                if constexpr (KIND == LENS_GAUSS) {
                    if (keep && near2 > T(0) && near2 * q0.w >= T(1.000001)) q0.w = T(-1);
                }
            }
            unsigned kb = __ballot_sync(full, keep);
            if (C.ns > 1) {
                const int q = C.seq_b + __popc(kb & ((1u << lane) - 1u));
                C.seq_b += __popc(kb);
                keep = keep && q % C.ns == C.sl;
                kb = __ballot_sync(full, keep);
            }
            if (keep) {
                int slot = nbuf + __popc(kb & ((1u << lane) - 1u));
                S.b0[slot] = q0;
                S.b1[slot] = P.big1[e];
                S.bpid[slot] = (int)P.big_pid[e];
            }
            nbuf += __popc(kb);
            __syncwarp();
        }
    }
}

// One step of boxes (one per lane): an accepted cell goes to the far buffer
// (this item's share of them), an opened leaf's particles and a big list that
// reaches the group to theirs.  The tree walk and the replay of kept lists
// both feed it.
template <int KIND, typename T>
LENS_DEV void back_step(BackCtx<KIND, T>& C, int v, bool acc, bool leaf, bool big_has, const vec4_t<T>& A,
                        const int4& Lk, T dxv, T dyv, int& nf, int& nn, int& nb)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const BackParams<T>& P = C.P;
    BackShared<KIND, T>& S = C.S;
    unsigned ball = __ballot_sync(full, acc);
    bool take = acc;  // this slice's share of the accepted cells
    if (C.ns > 1) {
        const int q = C.seq_f + __popc(ball & ((1u << lane) - 1u));
        C.seq_f += __popc(ball);
        take = acc && q % C.ns == C.sl;
        ball = __ballot_sync(full, take);
    }
    if (take) {
        int pos = nf + __popc(ball & ((1u << lane) - 1u));
        v2_t<T> Q = P.nodeB[v];
        S.fdx[pos] = dxv;
        S.fdy[pos] = dyv;
        S.fM[pos] = A.z;
        S.fqr[pos] = Q.x;
        S.fqi[pos] = Q.y;
        S.fnode[pos] = v;
    }
    nf += __popc(ball);
    back_append_near<KIND, T>(C, leaf ? (Lk.y & kCountMask) : 0, Lk.x, nn, P.leaf0, P.leaf1);
    if constexpr (KIND != LENS_POINT) back_append_big<KIND, T>(C, big_has, v, Lk.z, Lk.w, nb);
    __syncwarp();
    if (nf >= 32) {
        C.flush_far(nf);
        nf = 0;
    }
}

template <int KIND, typename T, bool DIRECT>
__global__ void __launch_bounds__(kWalkWarps * 32)
back_kernel(BackParams<T> P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned full = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    BackShared<KIND, T>& S = reinterpret_cast<BackShared<KIND, T>*>(smem_raw)[warp];
    int* stack = P.stack + ((int64_t)blockIdx.x * kWalkWarps + warp) * kStackCap;
    BackCtx<KIND, T> C(P, S);

    uint32_t Kc = 0, Hn = 0;
    if (P.heavy_hdr) {
        Kc = P.heavy_hdr[0];
        Hn = P.heavy_hdr[1];
    }
    const int64_t n_items = P.n_groups - (int64_t)Kc + (int64_t)Hn;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(P.counter, 1u);
        item = __shfl_sync(full, item, 0);
        if ((int64_t)item >= n_items) break;
        uint32_t g;
        C.sl = 0;
        C.ns = 1;
        if (item < Hn) {
            const uint32_t e = P.heavy[item];
            g = P.order[e >> 10];
            C.sl = (int)((e >> 5) & 31u);
            C.ns = (int)(e & 31u) + 1;
        } else {
            const uint32_t j = item - Hn + Kc;
            g = P.order ? P.order[j] : j;
        }
        C.seq_f = C.seq_n = C.seq_b = 0;
        C.H = P.gH[g];
        C.box = P.gbox[g];
        uint2 rg = P.grange[g];
        C.nr = (int)rg.y;
        for (int k = lane; k < (int)rg.y; k += 32) {
            v2_t<T> l = P.ray_l[rg.x + k];
            uint32_t i = P.ray_idx[rg.x + k];
            S.rx[k] = l.x;
            S.ry[k] = l.y;
            S.rg1[k] = P.ga1[i];
            S.rg2[k] = P.ga2[i];
        }
        __syncwarp();
        if constexpr (sizeof(T) == 4) {
            for (int p = lane; 2 * p < C.nr; p += 32) {
                const bool two = 2 * p + 1 < C.nr;
                const int j0 = 2 * p, j1 = two ? 2 * p + 1 : 2 * p;
                S.pk_a[p] = make_float4(S.rx[j0], S.rx[j1], S.ry[j0], S.ry[j1]);
                S.pk_b[p] = make_float4(S.rg1[j0], two ? S.rg1[j1] : 0.f, S.rg2[j0], two ? S.rg2[j1] : 0.f);
            }
            __syncwarp();
        }

        if (P.n_part > 0) {
            int nn = 0, nb = 0;
            if (DIRECT) {
                for (int64_t base = 0; base < P.n_part; base += 0x40000000) {
                    int64_t rem = P.n_part - base;
                    int c = (int)(rem < 0x40000000 ? rem : 0x40000000);
                    back_append_near<KIND, T>(C, lane == 0 ? c : 0, (int)base, nn, P.leaf0, P.leaf1);
                }
                C.flush_near(nn);
            } else {
                // boxes 32 at a time, either replayed from the forward's kept
                // lists of this group or found by walking the tree; one copy of
                // the step's code serves both (the kernel's code stays small)
                const uint32_t ln = P.list_n ? P.list_n[g] : kListOverflow;
                const bool replay = ln != kListOverflow;
                const uint32_t* ids = P.list_ids + (int64_t)g * P.list_K;
                int nf = 0, sp = 1;
                uint32_t base = 0;
                // replay: entries read two steps ahead, their boxes one step
                // ahead (the lists come from DRAM, not from L1 like a stack)
                uint32_t e0 = 0u, e1 = 0u;
                int4 Lk1 = make_int4(0, 0, 0, 0);
                vec4_t<T> A1{};
                if (replay) {
                    e0 = lane < ln ? __ldcs(ids + lane) : 0u;
                    e1 = 32 + lane < ln ? __ldcs(ids + 32 + lane) : 0u;
                    if (e0) Lk1 = P.link[e0 & kListIdMask];
                    if (e0 & kListFar) A1 = P.nodeA[e0 & kListIdMask];
                } else {
                    if (lane == 0) stack[0] = 0;
                    __syncwarp();
                }
                while (replay ? base < ln : sp > 0) {
                    int v = -1;
                    bool acc = false, leaf = false, big = false;
                    vec4_t<T> A{};
                    int4 Lk = make_int4(0, 0, 0, 0);
                    T dxv = T(0), dyv = T(0);
                    if (replay) {
                        const uint32_t e = e0;
                        Lk = Lk1;
                        A = A1;
                        const uint32_t e2 = base + 64 + lane < ln ? __ldcs(ids + base + 64 + lane) : 0u;
                        Lk1 = e1 ? P.link[e1 & kListIdMask] : make_int4(0, 0, 0, 0);
                        if (e1 & kListFar) A1 = P.nodeA[e1 & kListIdMask];
                        e0 = e1;
                        e1 = e2;
                        base += 32;
                        v = (int)(e & kListIdMask);
                        acc = (e & kListFar) != 0u;
                        leaf = (e & kListLeaf) != 0u;
                        big = (e & kListBig) != 0u;
                        if (acc) {
                            dxv = A.x - C.H.x;
                            dyv = A.y - C.H.y;
                        }
                    } else {
                        int k = sp < 32 ? sp : 32;
                        sp -= k;
                        v = lane < k ? stack[sp + lane] : -1;
                        __syncwarp();
                        const bool valid = v >= 0;
                        bool open = false;
                        if (valid) {
                            A = P.nodeA[v];
                            Lk = P.link[v];
                            dxv = A.x - C.H.x;
                            dyv = A.y - C.H.y;
                            T ex = fmax(fabs(dxv - C.box.x) - C.box.z, T(0));
                            T ey = fmax(fabs(dyv - C.box.y) - C.box.w, T(0));
                            acc = fma(ex, ex, ey * ey) > A.w;
                            leaf = !acc && (Lk.y & kLeafBit);
                            open = !acc && !leaf;
                        }
                        big = valid && Lk.w > 0;
                        int nc = open ? Lk.y : 0;
                        int totc;
                        int offc = warp_exclusive_scan(nc, &totc);
                        if (sp + totc > kStackCap) {
                            if (lane == 0) atomicOr(P.err, DERR_STACK_OVERFLOW);
                            break;
                        }
                        for (int c = 0; c < nc; ++c) stack[sp + offc + c] = Lk.x + c;
                        sp += totc;
                    }
                    back_step<KIND, T>(C, v, acc, leaf, big, A, Lk, dxv, dyv, nf, nn, nb);
                }
                C.flush_far(nf);
                C.flush_near(nn);
                if constexpr (KIND != LENS_POINT) C.flush_big(nb);
            }
        }

        // analytic halos: lanes own rays; reduce each halo's gradient over the warp
        if (P.n_halos > 0 && P.ghalo && C.sl == 0) {
            for (int h = 0; h < P.n_halos; ++h) {
                const HaloDev& hd = P.halos[h];
                T hx = (T)((double)C.H.x - hd.x), hy = (T)((double)C.H.y - hd.y);
                T m = (T)hd.m;
                // gk = sum kappa (G.w); gin = sum kb (G.w) over the rays inside
                // the support (the enclosed mass depends on q, R_max only there)
                T gm = T(0), gx = T(0), gy = T(0), gk = T(0), gin = T(0);
                for (int k = lane; k < C.nr; k += 32) {
                    T wx = S.rx[k] + hx, wy = S.ry[k] + hy;
                    T r2 = fma(wx, wx, wy * wy);
                    T kb = T(0), kap = T(0), Dp = T(0);
                    bool inside = false;
                    if (hd.kind == LENS_POINT) {
                        point_terms(m, r2, kb, Dp);
                    } else if (hd.kind == LENS_GAUSS) {
                        gauss_terms(m, (T)hd.c0, r2, (T)hd.c1, (T)hd.c2, kb, kap, Dp);
                        inside = r2 * (T)hd.c0 < (T)hd.c1;
                    } else if (hd.kind == LENS_NFW) {
                        nfw_terms(m, (T)hd.c2, (T)hd.c0, (T)hd.c1, r2, kb, kap, Dp);
                        inside = r2 < (T)hd.c2 && r2 > T(0);
                    } else if (hd.kind == LENS_SIS) {
                        if (r2 > T(0)) {
                            T rr = sqrt(r2), re = (T)hd.p0;
                            kb = re / rr;
                            kap = T(0.5) * kb;
                            Dp = kap / r2;
                        }
                    } else {
                        T R2 = (T)hd.c2;
                        if (r2 < R2) {
                            kb = m / R2;
                            kap = kb;
                        } else {
                            point_terms(m, r2, kb, Dp);
                        }
                    }
                    T gm0 = gm;
                    term_grad(wx, wy, kb, kap, Dp, S.rg1[k], S.rg2[k], gm, gx, gy, gk);
                    if (inside) gin += gm - gm0;
                }
                for (int o = 16; o; o >>= 1) {
                    gm += __shfl_xor_sync(full, gm, o);
                    gx += __shfl_xor_sync(full, gx, o);
                    gy += __shfl_xor_sync(full, gy, o);
                    gk += __shfl_xor_sync(full, gk, o);
                    gin += __shfl_xor_sync(full, gin, o);
                }
                if (lane == 0) {
                    // the strength parameter: m, or r_E for the SIS
                    double strength = hd.kind == LENS_SIS ? hd.p0 : hd.m;
                    double gs = strength != 0.0 ? (double)gm / strength : 0.0;
                    // shape parameters p0, p1 (d alpha / d p = (d kb / d p) w)
                    double g0 = 0.0, g1 = 0.0;
                    if (hd.kind == LENS_GAUSS) {
                        // p0 = r_sm: dkb = -2 kappa / r_sm; p1 = q: dkb = -kb N_q'(q) / N_q
                        g0 = -2.0 * (double)gk / hd.p0;
                        g1 = -hd.p1 * exp(-hd.c1) * hd.c2 * (double)gin;
                    } else if (hd.kind == LENS_NFW) {
                        // p0 = r_s: dkb = (-2 kappa + X c3 kb) / r_s; p1 = R_max:
                        // dkb = -c3 kb / r_s (X = R_max / r_s, c3 = X f(X) / g(X))
                        double X = hd.p1 / hd.p0;
                        g0 = (-2.0 * (double)gk + X * hd.c3 * (double)gin) * hd.c1;
                        g1 = -hd.c3 * (double)gin * hd.c1;
                    } else if (hd.kind == LENS_DISK) {
                        g0 = -2.0 * (double)gk / hd.p0;  // p0 = R
                    } else if (hd.kind == LENS_SIS) {
                        g0 = gs;                          // p0 = r_E
                    }
                    double* out = P.ghalo + 5 * h;
                    if (gs != 0.0) atomicAdd(out, gs);
                    atomicAdd(out + 1, (double)gx);
                    atomicAdd(out + 2, (double)gy);
                    if (g0 != 0.0) atomicAdd(out + 3, g0);
                    if (g1 != 0.0) atomicAdd(out + 4, g1);
                }
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------- polynomial push-down

// P_v(z) = a + b (z - z_v) + c (z - z_v)^2 (a real, b and c complex) for node v:
// its own cell adjoint plus its parent's polynomial re-centred at v's centre
// of mass.  One launch per level, root first.
template <typename T>
__global__ void k_push(uint32_t b0, uint32_t b1, const int* parent, const vec4_t<T>* nodeA, const double* adj,
                       dbl4* polyA, double2* polyC)
{
    uint32_t v = b0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= b1) return;
    vec4_t<T> A = nodeA[v];
    const double* a = adj + 5 * (int64_t)v;
    double M = (double)A.z;
    double pa = a[0], pbr = 0, pbi = 0, pcr = a[1], pci = a[2];
    if (M != 0.0) {
        pbr = a[3] / M;
        pbi = a[4] / M;
    }
    int p = parent[v];
    if (p >= 0) {
        dbl4 PA = polyA[p];        // {a, b_re, b_im, unused}
        double2 PC = polyC[p];     // c
        vec4_t<T> Ap = nodeA[p];
        double dx = (double)A.x - (double)Ap.x, dy = (double)A.y - (double)Ap.y;  // delta = z_v - z_p
        // a + b delta + c delta^2 (real part), b + 2 c delta, c
        double d2x = dx * dx - dy * dy, d2y = 2.0 * dx * dy;
        pa += PA.x + (PA.y * dx - PA.z * dy) + (PC.x * d2x - PC.y * d2y);
        pbr += PA.y + 2.0 * (PC.x * dx - PC.y * dy);
        pbi += PA.z + 2.0 * (PC.x * dy + PC.y * dx);
        pcr += PC.x;
        pci += PC.y;
    }
    polyA[v] = make_dbl4(pa, pbr, pbi, 0.0);
    polyC[v] = make_double2(pcr, pci);
}

// Every particle of every leaf: dL/dm += Re P(d), dL/dz += m P'(d), then
// scatter (with the direct terms) to the caller's input order; the size
// gradient is -(2/s) sum kappa (G.w) with s the particle's size (r_sm from
// c = 1/(2 r_sm^2) of a Gaussian record, r_s = 1/B of an NFW record).
template <typename T>
__global__ void k_leafgrad(uint32_t n_nodes, const int4* link, const vec4_t<T>* nodeA, const vec4_t<T>* exact0,
                           const vec4_t<T>* exact1, int kind, const dbl4* polyA, const double2* polyC,
                           const double* gpart, const uint32_t* perm, T* out)
{
    uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_nodes) return;
    int4 L = link[v];
    if (!(L.y & kLeafBit)) return;
    vec4_t<T> A = nodeA[v];
    dbl4 PA = polyA[v];
    double2 PC = polyC[v];
    int cnt = L.y & kCountMask;
    for (int k = 0; k < cnt; ++k) {
        int j = L.x + k;
        vec4_t<T> q = exact0[j];
        double dx = (double)q.x - (double)A.x, dy = (double)q.y - (double)A.y;
        double d2x = dx * dx - dy * dy, d2y = 2.0 * dx * dy;
        double gm = PA.x + (PA.y * dx - PA.z * dy) + (PC.x * d2x - PC.y * d2y);
        double kr = PA.y + 2.0 * (PC.x * dx - PC.y * dy), ki = PA.z + 2.0 * (PC.x * dy + PC.y * dx);
        double m = (double)q.z;
        const double* gp = gpart + 4 * (int64_t)j;
        // dL = Re(m P'(d) dz): dL/dx = m Re P', dL/dy = -m Im P'
        gm += gp[0];
        double gx = m * kr + gp[1];
        double gy = -m * ki + gp[2];
        double inv_s = 0.0;  // 1/s
        if (kind == LENS_GAUSS) inv_s = sqrt(2.0 * (double)q.w);
        else if (kind == LENS_NFW) inv_s = (double)exact1[j].y;
        double gs = -2.0 * inv_s * gp[3];
        uint32_t i = perm[j];
        out[4 * (int64_t)i] += (T)gm;
        out[4 * (int64_t)i + 1] += (T)gx;
        out[4 * (int64_t)i + 2] += (T)gy;
        out[4 * (int64_t)i + 3] += (T)gs;
    }
}

// ------------------------------------------------------------- host

template <int KIND, typename T, bool DIRECT>
static void back_launch(const BackParams<T>& P, int num_sms, cudaStream_t s)
{
    size_t smem = kWalkWarps * sizeof(BackShared<KIND, T>);
    static int bps = -1;
    if (bps < 0) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(back_kernel<KIND, T, DIRECT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, back_kernel<KIND, T, DIRECT>, kWalkWarps * 32, smem);
        if (bps < 1) bps = 1;
        if (bps > 16) bps = 16;  // stack slots are allocated for 16 blocks per SM
    }
    { back_kernel<KIND, T, DIRECT><<<num_sms * bps, kWalkWarps * 32, smem, s>>>(P); note_launch(); }
}

template <typename T, bool DIRECT>
static void back_dispatch(int kind, const BackParams<T>& P, int num_sms, cudaStream_t s)
{
    if (kind == LENS_POINT) back_launch<LENS_POINT, T, DIRECT>(P, num_sms, s);
    else if (kind == LENS_GAUSS) back_launch<LENS_GAUSS, T, DIRECT>(P, num_sms, s);
    else back_launch<LENS_NFW, T, DIRECT>(P, num_sms, s);
}

template <typename T>
static lens_status backward_typed(lens_tree* t, double ox, double oy, const void* dx, const void* dy, int dtype,
                                  int64_t n, const void* const g[5], void* const* g_species, void* g_halos,
                                  int flags, cudaStream_t s)
{
    using T4 = vec4_t<T>;
    using T2 = v2_t<T>;
    int64_t off[2] = {0, n};
    double orig[2] = {ox, oy};
    ShootPlan plan;
    LENS_TRY(upload_batches(t, 1, off, orig, s, &plan));
    if (32 * plan.R > kMaxGroup) return lens_set_error(LENS_ERR_INTERNAL, "group larger than the adjoint buffer");
    RayKey key;
    key.dx = dx; key.dy = dy; key.n = n; key.dtype = dtype; key.R = plan.R; key.ox = ox; key.oy = oy;
    // with LENS_KEEP_LISTS the caller vouches that these are the forward's
    // rays, unchanged: the forward's groups, still in the scratch, serve
    const bool keep = (flags & LENS_KEEP_LISTS) && !(flags & LENS_DIRECT) && kept_lists(t, key);
    if (!(keep && groups_hold(t, key))) LENS_TRY(enqueue_groups<T>(t, plan, dx, dy, dtype, s));
    // the forward call on these rays recorded its groups' work: heaviest first
    // (a quarter of one warp's share for a launch of about 16 warps per SM)
    const HeavyPlan hp = (flags & LENS_DIRECT) ? HeavyPlan{}
                                               : heavy_first_order<T>(t, plan, key, (int64_t)t->num_sms * 16, s);
    Layout Lay = make_layout(t->ray_cap, t->batch_cap, max_slots(t));
    char* base = (char*)t->ray_scratch.ptr;
    BackParams<T> P{};
    P.gH = (const T2*)(base + Lay.gH);
    P.gbox = (const T4*)(base + Lay.gbox);
    P.grange = (const uint2*)(base + Lay.grange);
    P.ray_l = (const T2*)(base + Lay.rl);
    P.ray_idx = (const uint32_t*)(base + Lay.ridx);
    P.n_groups = (int64_t)plan.ng;
    P.stack = (int*)(base + Lay.stack);
    P.err = t->d_err;
    P.order = hp.order;
    P.heavy_hdr = hp.hdr;
    P.heavy = hp.table;
    const uint32_t* lists = keep ? kept_lists(t, key) : nullptr;
    P.list_ids = lists;
    P.list_n = lists ? t->list_n : nullptr;
    P.list_K = lists ? t->list_K : 0;
    if (hp.hdr) LENS_CUDA(cudaMemcpyAsync(t->d_stats + 8, hp.hdr, 2 * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    else LENS_CUDA(cudaMemsetAsync(t->d_stats + 8, 0, 2 * sizeof(uint32_t), s));
    P.ga1 = (const T*)g[0];
    P.ga2 = (const T*)g[1];
    uint32_t* counter = (uint32_t*)(base + Lay.counter);
    const bool direct = (flags & LENS_DIRECT) != 0;
    bool first = true;
    int launches = 0;
    for (size_t si = 0; si < t->sp.size(); ++si) {
        const SpeciesTree& st = t->sp[si];
        bool want = st.n > 0 && g_species && g_species[si];
        bool halos_here = first && t->n_halos > 0 && g_halos;
        if (!want && !halos_here) continue;
        double* adj = nullptr;
        double* gpart = nullptr;
        dbl4* polyA = nullptr;
        double2* polyC = nullptr;
        StreamTemps tmps(s);  // this species' accumulators, released on every return path
        if (st.n > 0) {
            LENS_CUDA(tmps.get(&adj, st.n_nodes * 5 * sizeof(double)));
            LENS_CUDA(tmps.get(&gpart, st.n * 4 * sizeof(double)));
            LENS_CUDA(tmps.get(&polyA, st.n_nodes * sizeof(dbl4)));
            LENS_CUDA(tmps.get(&polyC, st.n_nodes * sizeof(double2)));
            LENS_CUDA(cudaMemsetAsync(adj, 0, st.n_nodes * 5 * sizeof(double), s));
            LENS_CUDA(cudaMemsetAsync(gpart, 0, st.n * 4 * sizeof(double), s));
        }
        P.nodeA = (const T4*)st.nodeA;
        P.nodeB = (const T2*)st.nodeB;
        P.link = st.link;
        P.leaf0 = (const T4*)((direct || st.kind == LENS_POINT) ? st.exact0 : st.leaf0);
        P.leaf1 = (const T4*)st.exact1;
        P.big0 = (const T4*)st.big0;
        P.big1 = (const T4*)st.big1;
        P.big_chunk = (const T4*)st.big_chunk;
        P.node_bigbox = (const T4*)st.node_bigbox;
        P.big_pid = st.big_pid;
        P.n_part = want ? st.n : 0;
        P.Uq = (T)st.Uq;
        P.invNq = (T)st.invNq;
        P.Uq2 = (T)(st.Uq * 1.4426950408889634074);
        P.Nq = (T)(st.invNq > 0 ? 1.0 / st.invNq : 0.0);
        P.eU = (T)std::exp(-st.Uq);
        P.halos = t->halos;
        P.n_halos = halos_here ? (int)t->n_halos : 0;
        P.ghalo = (double*)g_halos;
        P.adj = adj;
        P.gpart = gpart;
        P.counter = counter + 2 * launches;
        LENS_CUDA(cudaMemsetAsync(P.counter, 0, sizeof(uint32_t), s));
        int kind = st.n > 0 ? st.kind : LENS_POINT;
        if (direct) back_dispatch<T, true>(kind, P, t->num_sms, s);
        else back_dispatch<T, false>(kind, P, t->num_sms, s);
        if (want) {
            const int TB = 256;
            if (!direct) {
                LENS_TRY(finish_species(const_cast<SpeciesTree&>(st)));  // the level table
                for (int l = 0; l <= st.depth; ++l) {
                    uint32_t b0 = (uint32_t)st.level_start[l], b1 = (uint32_t)st.level_start[l + 1];
                    if (b1 > b0)
                        { k_push<T><<<grid_for(b1 - b0, TB), TB, 0, s>>>(b0, b1, st.parent, (const T4*)st.nodeA, adj,
                                                                      polyA, polyC); note_launch(); }
                }
            } else {
                LENS_CUDA(cudaMemsetAsync(polyA, 0, st.n_nodes * sizeof(dbl4), s));
                LENS_CUDA(cudaMemsetAsync(polyC, 0, st.n_nodes * sizeof(double2), s));
            }
            { k_leafgrad<T><<<grid_for(st.n_nodes, TB), TB, 0, s>>>((uint32_t)st.n_nodes, st.link, (const T4*)st.nodeA,
                                                                    (const T4*)st.exact0, (const T4*)st.exact1, st.kind,
                                                                    polyA, polyC, gpart, st.perm,
                                                                    (T*)g_species[si]); note_launch(); }
        }
        first = false;
        ++launches;
    }
    if (first && t->n_halos > 0 && g_halos) {
        // no species: halos only
        P.n_part = 0;
        P.halos = t->halos;
        P.n_halos = (int)t->n_halos;
        P.ghalo = (double*)g_halos;
        P.counter = counter;
        LENS_CUDA(cudaMemsetAsync(P.counter, 0, sizeof(uint32_t), s));
        back_dispatch<T, true>(LENS_POINT, P, t->num_sms, s);
    }
    LENS_CUDA(cudaGetLastError());
    return LENS_OK;
}

lens_status shoot_backward(lens_tree* t, double ox, double oy, const void* dx, const void* dy, int dtype,
                           int64_t n, const void* const g[5], void* const* g_species, void* g_halos,
                           int flags, cudaStream_t s)
{
    LENS_TRY(wait_built(t, s));
    if (t->precision == LENS_PREC_FP64)
        return backward_typed<double>(t, ox, oy, dx, dy, dtype, n, g, g_species, g_halos, flags, s);
    return backward_typed<float>(t, ox, oy, dx, dy, dtype, n, g, g_species, g_halos, flags, s);
}

}  // namespace lens
