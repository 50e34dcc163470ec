// walk_dev.cuh -- device code of the tree walk shared by the walk kernel
// (walk.cu) and its warp-specialised form (walk_ws.cu): parameters, shared
// buffers, the evaluation of far cells, leaf particles, big-list corrections
// and analytic halos for a lane's rays (Sec. 3.2), and the traversal with its
// buffer appends, written against a context whose flush either evaluates a
// full buffer or hands it to another warp.
#pragma once

#include "profiles.cuh"
#include "walk_shared.cuh"

namespace lens {

template <typename T> struct WalkParams {
    const vec4_t<T>* nodeA;
    const v2_t<T>* nodeB;
    const int4* link;
    const vec4_t<T>* leaf0;   // near records (listed particles marked)
    const vec4_t<T>* leaf1;   // NFW second record
    const vec4_t<T>* big0;       // {x, y, s^2, r0^2}
    const vec4_t<T>* big1;       // {m, c | A, B, 0}
    const vec4_t<T>* big_chunk;  // support bounding box per 32 entries
    const vec4_t<T>* node_bigbox;
    int64_t n_part;
    T Uq, invNq, Uq2, Nq, eU;
    const v2_t<T>* gH;
    const vec4_t<T>* gbox;
    const uint2* grange;
    const v2_t<T>* ray_l;
    const uint32_t* ray_idx;
    int64_t n_groups;
    const HaloDev* halos;
    int n_halos;
    T* out[5];
    int accumulate;
    uint32_t* counter;
    int* stack;
    uint32_t* err;
    unsigned long long* stats;  // optional walk counters
    long long wait_cycles;      // bound of every wait between cooperating warps (SM clock cycles)
    // direct sum split over particle slices (n_slices > 1): work item
    // g * n_slices + k sums slice k of the particles for group g's rays into
    // split[(k * 5 + q) * split_n + ray]; k_split_sum adds the slices
    int n_slices;
    int64_t split_n;
    T* split;
    // group order and work record (walk_shared.cuh): item g walks group
    // order[g] (identity if null); the walk adds each group's work to gcost[g]
    const uint32_t* order;
    uint32_t* gcost;
    // interaction lists kept for the adjoint (LENS_KEEP_LISTS): group g's
    // tagged box indices at list_ids + g * list_K, their count in list_n[g]
    uint32_t* list_ids;
    uint32_t* list_n;
    int list_K;
};

// Record one traversal step's boxes that matter to the adjoint (one entry
// per box, lane order) into the context's list, if it keeps one.
template <class Ctx>
LENS_DEV void record_step(Ctx& C, int v, bool acc, bool leaf, bool big)
{
    if (!C.rec) return;
    const int lane = threadIdx.x & 31;
    const uint32_t tag = (acc ? kListFar : 0u) | (leaf ? kListLeaf : 0u) | (big ? kListBig : 0u);
    const unsigned m = __ballot_sync(0xffffffffu, tag != 0u);
    const int pos = C.rec_n + __popc(m & ((1u << lane) - 1u));
    if (tag != 0u && pos < C.rec_cap) C.rec[pos] = (uint32_t)v | tag;
    C.rec_n += __popc(m);
}

// The shared-memory tiles of the near field: TILE 0 holds kNearCap leaf
// particles and kBigCap big-list entries per warp, TILE 1 twice as many
// (fewer flushes and folds, more shared memory per warp); the autotuner
// times both.
template <int KIND, typename T, int TILE = 0> struct WalkBuf {
    static constexpr int kNear = TILE ? 2 * kNearCap : kNearCap;
    static constexpr int kBig = TILE ? 2 * kBigCap : kBigCap;
    // FP32 Gaussian big entries are stored one array per field, so that two
    // consecutive entries load as one float2 operand of the packed form
    static constexpr bool kPackedBig = KIND == LENS_GAUSS && sizeof(T) == 4;
    static constexpr int kB = kPackedBig ? kBig : 1;
    T fdx[kFarCap], fdy[kFarCap], fM[kFarCap], fqr[kFarCap], fqi[kFarCap];
    vec4_t<T> n0[kNear];
    vec4_t<T> n1[KIND == LENS_NFW ? kNear : 1];
    vec4_t<T> b0[KIND == LENS_POINT || kPackedBig ? 1 : kBig];
    vec4_t<T> b1[KIND == LENS_POINT || kPackedBig ? 1 : kBig];
    // -x, -y (from the group anchor), -c log2 e, m/N_q, -(m/N_q) e^-q^2/2,
    // m c/N_q, the flag or 1/r0^2 (b0.w of the generic layout) and 1/c.
    // Entries whose support contains every ray of the group fill slots
    // [0, n_in) from the bottom; the others fill [kBig - n_out, kBig)
    // from the top (the buffer count packs n_in | n_out << 16).
    float bnx[kB], bny[kB], bcl[kB], bm[kB], bme[kB], bk[kB], bw[kB], bic[kB];
};

// The list ranges of one traversal step (one per lane) and the Neumaier-
// compensated totals of each lane's rays ([component][ray][lane]; touched once
// per buffer flush, so they live here rather than in registers).
struct WalkRanges {
    int rs_off[33];
    int rs_first[32];
    int rs_end[32];
};

// NR: rays per lane the totals have room for (2, or 4 for 128-ray groups).
template <typename T, int NR = 2> struct WalkTot {
    T tot_s[5][NR][32], tot_c[5][NR][32];
};

// Shared memory of one warp of the walk kernel.
template <int KIND, typename T, int TILE = 0, int NR = 2> struct WalkShared {
    WalkBuf<KIND, T, TILE> buf;
    WalkRanges rng;
    WalkTot<T, NR> tot;
};

// Room in the totals for R rays per lane.
template <int R> constexpr int tot_rays() { return R > 2 ? R : 2; }

template <int KIND, typename T, int R, bool AO, int TILE = 0> struct WalkEval {
    static_assert(R <= kMaxRaysPerLane, "rays per lane");
    static constexpr int kQ = AO ? 2 : 5;  // components accumulated
    static constexpr int kNR = tot_rays<R>();
    using Buf = WalkBuf<KIND, T, TILE>;
    const WalkParams<T>& P;
    Buf* B;                // the buffers being evaluated
    WalkTot<T, kNR>* Tt;   // compensated totals of the lane's rays
    T lx[R], ly[R];
    Acc5<T> part[R];
    v2_t<T> H;
    vec4_t<T> box;

    LENS_DEV WalkEval(const WalkParams<T>& p, Buf* b, WalkTot<T, kNR>* t) : P(p), B(b), Tt(t) {}

    LENS_DEV void tot_zero()
    {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int q = 0; q < kQ; ++q) Tt->tot_s[q][r][lane] = Tt->tot_c[q][r][lane] = T(0);
    }

    LENS_DEV T tot_get(int r, int q) const
    {
        const int lane = threadIdx.x & 31;
        return Tt->tot_s[q][r][lane] + Tt->tot_c[q][r][lane];
    }

    // Add the partial sums of the last flush to the compensated totals.
    LENS_DEV void fold()
    {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const T v[5] = {part[r].a1, part[r].a2, part[r].k, part[r].g1, part[r].g2};
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                T ts = Tt->tot_s[q][r][lane], tc = Tt->tot_c[q][r][lane];
                Comp5<T>::add1(ts, tc, v[q]);
                Tt->tot_s[q][r][lane] = ts;
                Tt->tot_c[q][r][lane] = tc;
            }
            part[r].zero();
        }
    }

    LENS_DEV void eval_far(int nf)
    {
        for (int c = 0; c < nf; ++c) {
            T dx = B->fdx[c], dy = B->fdy[c], M = B->fM[c], qr = B->fqr[c], qi = B->fqi[c];
#pragma unroll
            for (int r = 0; r < R; ++r) cell_terms<T, AO>(part[r], lx[r] - dx, ly[r] - dy, M, qr, qi);
        }
        fold();
    }

    // Leaf particles: full profile unless marked as a listed (softened) point.
    LENS_DEV void eval_near(int nn)
    {
        for (int i = 0; i < nn; ++i) {
            vec4_t<T> q = B->n0[i];
            vec4_t<T> q1;
            if constexpr (KIND == LENS_NFW) q1 = B->n1[i];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                T wx = lx[r] - q.x, wy = ly[r] - q.y;
                T r2 = fma(wx, wx, wy * wy);
                T kb, kap = T(0), Dp;
                if (KIND == LENS_POINT) {
                    point_terms(q.z, r2, kb, Dp);
                } else if (KIND == LENS_GAUSS) {
                    if (q.w > T(0)) gauss_terms(q.z, q.w, r2, P.Uq, P.invNq, kb, kap, Dp);
                    else point_terms(q.z, fmax(r2, -q.w), kb, Dp);
                } else {
                    if (q.w > T(0)) nfw_terms(q.z, q.w, q1.x, q1.y, r2, kb, kap, Dp);
                    else point_terms(q.z, fmax(r2, -q.w), kb, Dp);
                }
                part[r].template radial<AO>(wx, wy, kb, kap, Dp);
            }
        }
        fold();
    }

    // One packed-layout entry for every ray, in scalar arithmetic (entries
    // with a ray inside the softening radius, and unpaired entries).
    LENS_DEV void big_entry_scalar(int i, Acc5x2 (&pa)[R])
    {
        const float nx = B->bnx[i], ny = B->bny[i], w = B->bw[i];
        const float4 q = make_float4(0.0f, 0.0f, 0.0f, w);
        const float4 q1 = make_float4(B->bm[i], -B->bcl[i], B->bk[i], B->bic[i]);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            Acc5<float> a;
            a.zero();
            if (w < 0.0f) gauss_correction_fast<AO>(a, lx[r] + nx, ly[r] + ny, q1, P.Uq2, P.eU);
            else gauss_correction<AO>(a, lx[r] + nx, ly[r] + ny, q, q1, P.Uq2, P.Nq);
            pa[r].na1.x -= a.a1;
            pa[r].na2.x -= a.a2;
            if (!AO) {
                pa[r].k.x += a.k;
                pa[r].g1p.x += a.g1;
                pa[r].hg2.x = fmaf(0.5f, a.g2, pa[r].hg2.x);
            }
        }
    }

    // Two entries of the other region of which some ray may come inside a
    // softening radius: the packed general form.
    LENS_DEV void big_pair_soft(int i, Acc5x2 (&pa)[R], const float2 (&LX)[R], const float2 (&LY)[R])
    {
        const float2 nx = *reinterpret_cast<const float2*>(&B->bnx[i]);
        const float2 ny = *reinterpret_cast<const float2*>(&B->bny[i]);
        const float2 cl = *reinterpret_cast<const float2*>(&B->bcl[i]);
        const float2 mN = *reinterpret_cast<const float2*>(&B->bm[i]);
        const float2 kz = *reinterpret_cast<const float2*>(&B->bk[i]);
        const float2 w = *reinterpret_cast<const float2*>(&B->bw[i]);
        const float2 ic = *reinterpret_cast<const float2*>(&B->bic[i]);
        const float2 t_c = make_float2(-cl.x, -cl.y);
        const float2 nmass = make_float2(-(mN.x * P.Nq), -(mN.y * P.Nq));
        const float2 ws = make_float2(w.x < 0.0f ? INFINITY : w.x, w.y < 0.0f ? INFINITY : w.y);
#pragma unroll
        for (int r = 0; r < R; ++r)
            gauss_correction_soft_x2<AO>(pa[r], LX[r], LY[r], nx, ny, t_c, kz, mN, nmass, ws, ic, P.Uq2, P.eU);
    }

    template <bool EDGE>
    LENS_DEV void big_pair_packed(int i, Acc5x2 (&pa)[R], const float2 (&LX)[R], const float2 (&LY)[R])
    {
        const float2 nx = *reinterpret_cast<const float2*>(&B->bnx[i]);
        const float2 ny = *reinterpret_cast<const float2*>(&B->bny[i]);
        const float2 cl = *reinterpret_cast<const float2*>(&B->bcl[i]);
        const float2 mN = *reinterpret_cast<const float2*>(&B->bm[i]);
        const float2 nmE = *reinterpret_cast<const float2*>(&B->bme[i]);
        const float2 kz = *reinterpret_cast<const float2*>(&B->bk[i]);
#pragma unroll
        for (int r = 0; r < R; ++r)
            gauss_correction_x2<AO, EDGE>(pa[r], LX[r], LY[r], nx, ny, cl, mN, nmE, kz, -P.Uq2);
    }

    // FP32 Gaussian big buffer in packed arithmetic: the whole-group-inside
    // region four entries at a time without tests, then the other region
    // pair by pair (packed closed form with the support edge; where a ray may
    // be inside a softening radius, the packed general form for alpha only,
    // else entry by entry).
    LENS_DEV void eval_big_packed(int nbuf)
    {
        const int n_in = nbuf & 0xffff, n_out = nbuf >> 16;
        Acc5x2 pa[R];
        float2 LX[R], LY[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            pa[r].zero();
            LX[r] = make_float2(lx[r], lx[r]);
            LY[r] = make_float2(ly[r], ly[r]);
        }
        int i = 0;
        for (; i + 3 < n_in; i += 4) {
            big_pair_packed<false>(i, pa, LX, LY);
            big_pair_packed<false>(i + 2, pa, LX, LY);
        }
        if (i + 1 < n_in) {
            big_pair_packed<false>(i, pa, LX, LY);
            i += 2;
        }
        if (i < n_in) big_entry_scalar(i, pa);
        i = Buf::kBig - n_out;
        if ((i & 1) && i < Buf::kBig) big_entry_scalar(i++, pa);
        for (; i + 1 < Buf::kBig; i += 2) {
            const float2 w = *reinterpret_cast<const float2*>(&B->bw[i]);
            if (w.x < 0.0f && w.y < 0.0f) {
                big_pair_packed<true>(i, pa, LX, LY);
            } else if constexpr (AO) {
                // (alpha only: the registers allow the packed general form;
                // with kappa and gamma it would push the walk's hot loop
                // into spills)
                big_pair_soft(i, pa, LX, LY);
            } else {
                big_entry_scalar(i, pa);
                big_entry_scalar(i + 1, pa);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            part[r].a1 -= pa[r].na1.x + pa[r].na1.y;
            part[r].a2 -= pa[r].na2.x + pa[r].na2.y;
            if (!AO) {
                part[r].k += pa[r].k.x + pa[r].k.y;
                part[r].g1 += (pa[r].g1p.x + pa[r].g1p.y) - 2.0f * (pa[r].g1y.x + pa[r].g1y.y);
                part[r].g2 += 2.0f * (pa[r].hg2.x + pa[r].hg2.y);
            }
        }
        fold();
    }

    // Big-list corrections: (full profile - softened point); zero outside the
    // support, where both are the same point mass.
    // b0 = {x - H.x, y - H.y, s^2, 1/r0^2}; b1 = {m/N_q, c log2 e, m c / N_q,
    // 1/c} (GAUSS) or {m, A, B, 0} (NFW).  1/max(r^2, r0^2) = min(1/r^2, 1/r0^2).
    // The generic layout takes two entries per iteration for instruction-level
    // parallelism.
    LENS_DEV void eval_big(int nb)
    {
        if constexpr (Buf::kPackedBig) {
            eval_big_packed(nb);
            return;
        }
        int i = 0;
        if constexpr (KIND == LENS_GAUSS) {
            // b0.w < 0 marks an entry whose softening radius no ray of the
            // group reaches (the common case); b0.w = -2 also that its
            // support contains every ray of the group
            for (; i + 1 < nb; i += 2) {
                vec4_t<T> q = B->b0[i], q1 = B->b1[i], p = B->b0[i + 1], p1 = B->b1[i + 1];
                if (q.w < T(-1.5) && p.w < T(-1.5)) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        gauss_correction_inside<AO>(part[r], lx[r] - q.x, ly[r] - q.y, q1, P.eU);
                        gauss_correction_inside<AO>(part[r], lx[r] - p.x, ly[r] - p.y, p1, P.eU);
                    }
                } else if (q.w < T(0) && p.w < T(0)) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        gauss_correction_fast<AO>(part[r], lx[r] - q.x, ly[r] - q.y, q1, P.Uq2, P.eU);
                        gauss_correction_fast<AO>(part[r], lx[r] - p.x, ly[r] - p.y, p1, P.Uq2, P.eU);
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (q.w < T(0)) gauss_correction_fast<AO>(part[r], lx[r] - q.x, ly[r] - q.y, q1, P.Uq2, P.eU);
                        else gauss_correction<AO>(part[r], lx[r] - q.x, ly[r] - q.y, q, q1, P.Uq2, P.Nq);
                        if (p.w < T(0)) gauss_correction_fast<AO>(part[r], lx[r] - p.x, ly[r] - p.y, p1, P.Uq2, P.eU);
                        else gauss_correction<AO>(part[r], lx[r] - p.x, ly[r] - p.y, p, p1, P.Uq2, P.Nq);
                    }
                }
            }
        }
        for (; i < nb; ++i) {
            vec4_t<T> q = B->b0[i], q1 = B->b1[i];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                T wx = lx[r] - q.x, wy = ly[r] - q.y;
                if constexpr (KIND == LENS_GAUSS) {
                    if (q.w < T(0)) gauss_correction_fast<AO>(part[r], wx, wy, q1, P.Uq2, P.eU);
                    else gauss_correction<AO>(part[r], wx, wy, q, q1, P.Uq2, P.Nq);
                } else {
                    T r2 = fma(wx, wx, wy * wy);
                    T inv = r2 > T(0) ? rcp(r2) : T(0);
                    T inv_s = fmin(inv, q.w);
                    T kbp = q1.x * inv_s;
                    T kb, kap, Dp;
                    nfw_terms(q1.x, q.z, q1.y, q1.z, r2, kb, kap, Dp);
                    part[r].template radial<AO>(wx, wy, kb - kbp, kap, Dp - kbp * inv_s);
                }
            }
        }
        fold();
    }

    // Analytic components for every ray (Sec. 3.2 analytic models, App. B).
    LENS_DEV void halos()
    {
        for (int h = 0; h < P.n_halos; ++h) {
            const HaloDev& hd = P.halos[h];
            T hx = (T)((double)H.x - hd.x), hy = (T)((double)H.y - hd.y);
            int kind = hd.kind;
            T m = (T)hd.m;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                T wx = lx[r] + hx, wy = ly[r] + hy;
                T r2 = fma(wx, wx, wy * wy);
                T kb = T(0), kap = T(0), Dp = T(0);
                if (kind == LENS_POINT) {
                    point_terms(m, r2, kb, Dp);
                } else if (kind == LENS_GAUSS) {
                    gauss_terms(m, (T)hd.c0, r2, (T)hd.c1, (T)hd.c2, kb, kap, Dp);
                } else if (kind == LENS_NFW) {
                    nfw_terms(m, (T)hd.c2, (T)hd.c0, (T)hd.c1, r2, kb, kap, Dp);
                } else if (kind == LENS_SIS) {
                    if (r2 > T(0)) {
                        T rr = sqrt(r2), re = (T)hd.p0;
                        kb = re / rr;
                        kap = T(0.5) * kb;
                        Dp = kap / r2;
                    }
                } else {  // uniform disk
                    T R2 = (T)hd.c2;
                    if (r2 < R2) {
                        kb = m / R2;
                        kap = kb;
                        Dp = T(0);
                    } else {
                        point_terms(m, r2, kb, Dp);
                    }
                }
                part[r].template radial<AO>(wx, wy, kb, kap, Dp);
            }
        }
        fold();
    }
};

// The walk kernel's context: evaluation plus the buffer counts, where a full
// buffer is evaluated on the spot.
template <int KIND, typename T, int R, bool AO, int TILE = 0> struct WalkCtx : WalkEval<KIND, T, R, AO, TILE> {
    using value_type = T;
    using Buf = WalkBuf<KIND, T, TILE>;
    static constexpr int kKind = KIND;
    static constexpr int kNear = Buf::kNear, kBig = Buf::kBig;
    WalkRanges* Rg;
    int nf = 0, nn = 0, nb = 0;  // entries in the far, near and big buffers
    uint32_t* rec = nullptr;     // the group's kept interaction list, or null
    int rec_n = 0, rec_cap = 0;

    LENS_DEV WalkCtx(const WalkParams<T>& p, WalkShared<KIND, T, TILE, tot_rays<R>()>& s)
        : WalkEval<KIND, T, R, AO, TILE>(p, &s.buf, &s.tot), Rg(&s.rng) {}
    LENS_DEV void flush_far()
    {
        this->eval_far(nf);
        nf = 0;
    }
    LENS_DEV void flush_near()
    {
        this->eval_near(nn);
        nn = 0;
    }
    LENS_DEV void flush_big()
    {
        this->eval_big(nb);
        nb = 0;
    }
};

// Append, in order, the leaf particles of up to 32 index ranges (one per
// lane) to the near buffer, flushing it whenever fewer than 32 slots remain.
template <class Ctx, typename T = typename Ctx::value_type>
LENS_DEV void append_ranges(Ctx& C, int cnt, int first, const vec4_t<T>* src0, const vec4_t<T>* src1,
                            int& n_seen, int& n_kept)
{
    constexpr int KIND = Ctx::kKind;
    const unsigned full = 0xffffffffu;
    int lane = threadIdx.x & 31;
    int tot;
    int off = warp_exclusive_scan(cnt, &tot);
    if (tot == 0) return;
    n_seen += tot;
    C.Rg->rs_off[lane] = off;
    C.Rg->rs_first[lane] = first;
    if (lane == 31) C.Rg->rs_off[32] = tot;
    __syncwarp();
    for (int base = 0; base < tot; base += 32) {
        if (C.nn + 32 > Ctx::kNear) {
            C.flush_near();
            __syncwarp();
        }
        int i = base + lane;
        bool have = i < tot;
        vec4_t<T> q0, q1;
        bool keep = false;
        if (have) {
            int lo = 0, hi = 32;  // last lane o with rs_off[o] <= i
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (C.Rg->rs_off[mid] <= i) lo = mid;
                else hi = mid;
            }
            int p = C.Rg->rs_first[lo] + (i - C.Rg->rs_off[lo]);
            q0 = src0[p];
            if constexpr (KIND == LENS_NFW) q1 = src1[p];
            q0.x -= C.H.x;
            q0.y -= C.H.y;
            keep = true;
        }
        unsigned ball = __ballot_sync(full, keep);
        if (keep) {
            int slot = C.nn + __popc(ball & ((1u << lane) - 1u));
            C.B->n0[slot] = q0;
            if constexpr (KIND == LENS_NFW) C.B->n1[slot] = q1;
        }
        C.nn += __popc(ball);
        n_kept += __popc(ball);
        __syncwarp();
    }
}

// Slots in use in the big buffer (the packed layout counts both regions).
template <int KIND, typename T> LENS_DEV int big_used(int nbuf)
{
    if constexpr (WalkBuf<KIND, T>::kPackedBig) return (nbuf & 0xffff) + (nbuf >> 16);
    else return nbuf;
}

// Big lists of the visited boxes (one list per lane: entries [z, z + w) of
// the big arrays).  A list whose support box misses the group is skipped;
// otherwise its 32-entry chunks are tested by their support boxes and the
// entries of the chunks that pass are tested one by one; entries whose
// support reaches the group's box are appended to the big buffer.
template <class Ctx, typename T = typename Ctx::value_type>
LENS_DEV bool append_big(Ctx& C, bool has, int v, int z, int w, int& n_seen, int& n_kept)
{
    constexpr int KIND = Ctx::kKind;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const WalkParams<T>& P = C.P;
    int cnt = 0;
    if (has) {
        vec4_t<T> nb4 = P.node_bigbox[v];
        if (box_reaches_group<T>(nb4, C.H, C.box)) cnt = ((z + w - 1) >> 5) - (z >> 5) + 1;
    }
    int tot;
    int off = warp_exclusive_scan(cnt, &tot);
    if (tot == 0) return false;
    C.Rg->rs_off[lane] = off;
    C.Rg->rs_first[lane] = z;
    C.Rg->rs_end[lane] = z + w;
    if (lane == 31) C.Rg->rs_off[32] = tot;
    __syncwarp();
    for (int base = 0; base < tot; base += 32) {
        int i = base + lane;
        int cid = -1, own = 0;
        bool pass = false;
        if (i < tot) {
            int lo = 0, hi = 32;
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (C.Rg->rs_off[mid] <= i) lo = mid;
                else hi = mid;
            }
            own = lo;
            cid = (C.Rg->rs_first[lo] >> 5) + (i - C.Rg->rs_off[lo]);
            pass = box_reaches_group<T>(P.big_chunk[cid], C.H, C.box);
        }
        unsigned ball = __ballot_sync(full, pass);
        while (ball) {
            int src = __ffs(ball) - 1;
            ball &= ball - 1;
            int c = __shfl_sync(full, cid, src);
            int o = __shfl_sync(full, own, src);
            if (big_used<KIND, T>(C.nb) + 32 > Ctx::kBig) {
                C.flush_big();
                __syncwarp();
            }
            int e = 32 * c + lane;
            bool keep = false;
            vec4_t<T> q0, q1;
            bool inr = e >= C.Rg->rs_first[o] && e < C.Rg->rs_end[o];
            n_seen += __popc(__ballot_sync(full, inr));
            if (inr) {
                q0 = P.big0[e];
                q0.x -= C.H.x;
                q0.y -= C.H.y;
                T ex = fmax(fabs(q0.x - C.box.x) - C.box.z, T(0));
                T ey = fmax(fabs(q0.y - C.box.y) - C.box.w, T(0));
                T near2 = fma(ex, ex, ey * ey);
                keep = near2 < q0.z;
                if constexpr (KIND == LENS_GAUSS) {
                    // every ray of the group beyond the softening radius?  and
                    // all inside the support?
                    if (keep && near2 > T(0) && near2 * q0.w >= T(1.000001)) {
                        T fx = fabs(q0.x - C.box.x) + C.box.z, fy = fabs(q0.y - C.box.y) + C.box.w;
                        T far2 = fma(fx, fx, fy * fy) * T(1.000001);
                        q0.w = far2 < q0.z ? T(-2) : T(-1);
                    }
                }
            }
            unsigned kb = __ballot_sync(full, keep);
            if constexpr (Ctx::Buf::kPackedBig) {
                const bool in = keep && q0.w < T(-1.5);
                const unsigned bi = __ballot_sync(full, in), lt = (1u << lane) - 1u;
                if (keep) {
                    q1 = P.big1[e];
                    int slot = in ? (C.nb & 0xffff) + __popc(bi & lt)
                                  : Ctx::kBig - 1 - ((C.nb >> 16) + __popc(kb & ~bi & lt));
                    C.B->bnx[slot] = -q0.x;
                    C.B->bny[slot] = -q0.y;
                    C.B->bcl[slot] = -q1.y;
                    C.B->bm[slot] = q1.x;
                    C.B->bme[slot] = -q1.x * P.eU;
                    C.B->bk[slot] = q1.z;
                    C.B->bw[slot] = q0.w;
                    C.B->bic[slot] = q1.w;
                }
                C.nb += __popc(bi) + (__popc(kb & ~bi) << 16);
            } else {
                if (keep) {
                    q1 = P.big1[e];
                    int slot = C.nb + __popc(kb & ((1u << lane) - 1u));
                    C.B->b0[slot] = q0;
                    C.B->b1[slot] = q1;
                }
                C.nb += __popc(kb);
            }
            n_kept += __popc(kb);
            __syncwarp();
        }
    }
    return cnt > 0;
}


// Walk the tree for the context's group (Sec. 3.2): up to 32 candidate boxes
// per step, one per lane, tested against the group's bounding box; accepted
// boxes go to the far buffer, opened leaves to the near buffer, opened
// internal boxes push their children, and every visited box's big list is
// scanned.  Full buffers are flushed through the context (evaluated on the
// spot, or handed to an evaluating warp); the caller flushes what remains.
// Returns false if the warp's stack overflowed (the error word is set).
template <class Ctx, typename T = typename Ctx::value_type>
LENS_DEV bool traverse(Ctx& C, int* stack, int& c_vis, int& c_acc, int& c_near, int& c_bigs, int& c_bigk)
{
    constexpr int KIND = Ctx::kKind;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const WalkParams<T>& P = C.P;
    int sp = 1, c_dummy = 0;
    if (lane == 0) stack[0] = 0;
    __syncwarp();
    while (sp > 0) {
        int k = sp < 32 ? sp : 32;
        sp -= k;
        int v = lane < k ? stack[sp + lane] : -1;
        __syncwarp();
        bool valid = v >= 0, acc = false, leaf = false, open = false;
        vec4_t<T> A;
        int4 Lk = make_int4(0, 0, 0, 0);
        T dxv = T(0), dyv = T(0);
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
        unsigned ball = __ballot_sync(full, acc);
        if (acc) {
            int pos = C.nf + __popc(ball & ((1u << lane) - 1u));
            v2_t<T> Q = P.nodeB[v];
            C.B->fdx[pos] = dxv;
            C.B->fdy[pos] = dyv;
            C.B->fM[pos] = A.z;
            C.B->fqr[pos] = Q.x;
            C.B->fqi[pos] = Q.y;
        }
        C.nf += __popc(ball);
        c_vis += k;
        c_acc += __popc(ball);
        int nc = open ? Lk.y : 0;
        int totc;
        int offc = warp_exclusive_scan(nc, &totc);
        if (sp + totc > kStackCap) {
            if (lane == 0) atomicOr(P.err, DERR_STACK_OVERFLOW);
            return false;
        }
        for (int c = 0; c < nc; ++c) stack[sp + offc + c] = Lk.x + c;
        sp += totc;
        append_ranges(C, leaf ? (Lk.y & kCountMask) : 0, Lk.x, P.leaf0, P.leaf1, c_near, c_dummy);
        bool big = false;
        if constexpr (KIND != LENS_POINT) big = append_big(C, valid && Lk.w > 0, v, Lk.z, Lk.w, c_bigs, c_bigk);
        record_step(C, v, acc, leaf, big);
        __syncwarp();
        if (C.nf >= 32) {
            C.flush_far();
            __syncwarp();
        }
    }
    return true;
}

// Launch the producer/consumer form of the walk (walk_ws.cu); false if it
// cannot run here (the caller then launches the one-warp walk).
template <typename T, int R>
bool launch_ws(int kind, bool ao, const WalkParams<T>& P, int num_sms, cudaStream_t s, int consumers);

}  // namespace lens
