// build.cu -- quadtree construction on the GPU (Sec. 3.2).
//
// The paper inserts particles into an equal-area quadtree and, while the tree
// is built, computes each box's monopole and quadrupole moments, r_cut
// (Eq. r_cut) and its big-particle list.  Here the same tree is produced in
// bulk-parallel form:
//   1. stage + bounding box  -> square root box
//   2. 48-bit Morton keys (24 levels) -> radix sort: every box is a run of
//      equal key prefixes in the sorted order;
//   3. topology without a level loop: particle j's leaf level is one past the
//      deepest level at which a window of leaf_max consecutive keys containing
//      j shares its prefix; j "owns" the boxes it starts (levels from
//      lcp(K[j-1], K[j]) + 1 down to its leaf level), so a scan of the owned
//      counts numbers every box in depth-first preorder;
//   4. a stable sort by level gives breadth-first order (children contiguous);
//   5. moments bottom-up in one launch (the last child of a box to finish
//      computes the box), in FP64 at the top levels (FP32 below them in an
//      FP32 tree), stored in FP32 (or FP64) with r_cut^2 rounded up;
//   6. big lists: a particle whose support radius s exceeds lambda times the
//      side of a box on its path is listed at the shallowest such box; lists
//      are grouped per box by a stable sort (deterministic order).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "profiles.cuh"
#include "sort.cuh"
#include "tree.cuh"

namespace lens {

struct RootBox {
    double cx, cy, half, x0, y0;
    double inv;  // 2^24 / (2 half): Morton quantisation scale
};

template <typename T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };

__device__ __forceinline__ int lcp_digits(uint64_t a, uint64_t b)
{
    uint64_t x = a ^ b;
    if (x == 0) return kMaxDepth;
    return (__clzll((long long)x) - (64 - kKeyBits)) >> 1;
}

__device__ __forceinline__ uint64_t spread24(uint32_t v)
{
    uint64_t x = v & 0xffffffu;
    x = (x | (x << 16)) & 0x0000ffff0000ffffull;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

__device__ __forceinline__ uint32_t compact24(uint64_t x)
{
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x >> 4)) & 0x00ff00ff00ff00ffull;
    x = (x | (x >> 8)) & 0x0000ffff0000ffffull;
    x = (x | (x >> 16)) & 0x00000000ffffffffull;
    return (uint32_t)x & 0xffffffu;
}

// ------------------------------------------------------------- 1. stage

// Staging: the input rows as the tree's records {x, y, m, p}, checked
// (finite, m >= 0, p > 0 for profiles); the bounding box of the stored
// positions.  FP32 input into an FP32 tree stays in FP32 (the FP64 pipe of
// this GPU has 1/64 of the FP32 rate); the box is reduced in the stored
// precision and only the block's result goes through FP64.
template <typename T>
__global__ void k_stage(const void* data, int dtype, int64_t n, int kind, vec4_t<T>* staged,
                        unsigned long long* bbox, uint32_t* err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = i < n;
    T x = 0, y = 0;
    if (valid) {
        vec4_t<T> r;
        bool ok;
        if (dtype == LENS_F32) {
            const float* d = (const float*)data + 4 * i;  // the caller's rows need only 4-byte alignment
            const float4 v = make_float4(d[0], d[1], d[2], d[3]);
            ok = isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && v.z >= 0.0f;
            if (kind != LENS_POINT) ok = ok && isfinite(v.w) && v.w > 0.0f;
            r.x = (T)v.x; r.y = (T)v.y; r.z = (T)v.z; r.w = (T)v.w;
        } else {
            const double* d = (const double*)data + 4 * i;
            const double dx = d[0], dy = d[1], dm = d[2], dp = d[3];
            ok = isfinite(dx) && isfinite(dy) && isfinite(dm) && dm >= 0.0;
            if (kind != LENS_POINT) ok = ok && isfinite(dp) && dp > 0.0;
            r.x = (T)dx; r.y = (T)dy; r.z = (T)dm; r.w = (T)dp;
        }
        if (!ok) {
            atomicOr(err, DERR_BAD_INPUT);
            r.x = r.y = r.z = T(0);
            r.w = T(1);
        }
        staged[i] = r;
        x = r.x;
        y = r.y;
    }
    // bounding box of the stored (rounded) positions: warp, then block, then
    // four atomics per block
    __shared__ T red[4][32];
    T xmin = valid ? x : T(INFINITY), xmax = valid ? x : T(-INFINITY);
    T ymin = valid ? y : T(INFINITY), ymax = valid ? y : T(-INFINITY);
    for (int o = 16; o; o >>= 1) {
        xmin = fmin(xmin, __shfl_xor_sync(0xffffffffu, xmin, o));
        xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
        ymin = fmin(ymin, __shfl_xor_sync(0xffffffffu, ymin, o));
        ymax = fmax(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
    }
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = xmin; red[1][w] = xmax; red[2][w] = ymin; red[3][w] = ymax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nw; ++k) {
            xmin = fmin(xmin, red[0][k]); xmax = fmax(xmax, red[1][k]);
            ymin = fmin(ymin, red[2][k]); ymax = fmax(ymax, red[3][k]);
        }
        if (xmin <= xmax) {
            atomicMin(&bbox[0], dbl_to_ordered((double)xmin));
            atomicMax(&bbox[1], dbl_to_ordered((double)xmax));
            atomicMin(&bbox[2], dbl_to_ordered((double)ymin));
            atomicMax(&bbox[3], dbl_to_ordered((double)ymax));
        }
    }
}

__global__ void k_root(const unsigned long long* bbox, RootBox* rb)
{
    double x0 = ordered_to_dbl(bbox[0]), x1 = ordered_to_dbl(bbox[1]);
    double y0 = ordered_to_dbl(bbox[2]), y1 = ordered_to_dbl(bbox[3]);
    double cx = 0.5 * (x0 + x1), cy = 0.5 * (y0 + y1);
    double half = 0.5 * fmax(x1 - x0, y1 - y0);
    double scale = fmax(1.0, fmax(fabs(cx), fabs(cy)));
    if (!(half > 1e-12 * scale)) half = 1e-12 * scale;
    half *= 1.0 + 1.0 / 65536.0;  // every particle strictly inside
    rb->cx = cx;
    rb->cy = cy;
    rb->half = half;
    rb->x0 = cx - half;
    rb->y0 = cy - half;
    rb->inv = 16777216.0 / (2.0 * half);
}

// ----------------------------------------------------------- 2. Morton

template <typename T>
__global__ void k_morton(const vec4_t<T>* staged, int64_t n, const RootBox* rb, uint64_t* keys,
                         uint32_t* vals)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    vec4_t<T> r = staged[i];
    const double inv = rb->inv;
    // FP64 differences and scaling (exact cell of the stored position), the
    // floor and the clamp in integer arithmetic
    long long ix = __double2ll_rd(((double)r.x - rb->x0) * inv), iy = __double2ll_rd(((double)r.y - rb->y0) * inv);
    uint32_t qx = (uint32_t)min(max(ix, 0ll), 16777215ll);
    uint32_t qy = (uint32_t)min(max(iy, 0ll), 16777215ll);
    keys[i] = spread24(qx) | (spread24(qy) << 1);
    vals[i] = (uint32_t)i;
}

// Full-profile records of particle r (see walk.cu for their use).
template <typename T>
__device__ __forceinline__ void exact_records(const vec4_t<T>& r, int64_t j, int kind, double shape, double gX,
                                              vec4_t<T>* e0, vec4_t<T>* e1, vec4_t<T>* leaf0)
{
    vec4_t<T> a;
    a.x = r.x; a.y = r.y; a.z = r.z;
    double p = (double)r.w;
    if (kind == LENS_POINT) {
        a.w = (T)0;
    } else if (kind == LENS_GAUSS) {
        a.w = (T)(1.0 / (2.0 * p * p));
    } else {
        double Rm = shape * p;
        a.w = (T)(Rm * Rm);
        vec4_t<T> b;
        b.x = (T)((double)r.z / gX);
        b.y = (T)(1.0 / p);
        b.z = (T)0;
        b.w = (T)0;
        e1[j] = b;
    }
    e0[j] = a;
    if (leaf0) leaf0[j] = a;
}

// The particles in key order, the order kept for the caller (out_perm) and
// their full-profile records.
template <typename T>
__global__ void k_gather(const vec4_t<T>* staged, const uint32_t* perm, int64_t n, vec4_t<T>* sorted,
                         uint32_t* out_perm, int kind, double shape, double gX, vec4_t<T>* e0, vec4_t<T>* e1,
                         vec4_t<T>* leaf0)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t pj = perm[j];
    const vec4_t<T> r = staged[pj];
    sorted[j] = r;
    out_perm[j] = pj;
    exact_records<T>(r, j, kind, shape, gX, e0, e1, leaf0);
}

// --------------------------------------------------------- 3. topology

// Leaf level L_j and the number of boxes particle j starts.
__global__ void k_levels(const uint64_t* K, int64_t n, int N, uint8_t* Lp, uint32_t* cnt)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int D = -1;
    int64_t a0 = j - N + 1 > 0 ? j - N + 1 : 0;
    int64_t a1 = j < n - N ? j : n - N;
    for (int64_t a = a0; a <= a1; ++a) {
        int w = lcp_digits(K[a], K[a + N - 1]);
        D = w > D ? w : D;
    }
    int L = D + 1 < kMaxDepth ? D + 1 : kMaxDepth;
    int s = j == 0 ? 0 : lcp_digits(K[j - 1], K[j]) + 1;
    Lp[j] = (uint8_t)L;
    cnt[j] = L >= s ? (uint32_t)(L - s + 1) : 0u;
}

// First index e > j whose key leaves j's box at level l (n if none): a
// galloping search (steps 1, 2, 4, ... from j, then bisection of the last
// step), so a box of c particles costs about 2 log2 c probes.
__device__ __forceinline__ int64_t run_end(const uint64_t* K, int64_t n, int64_t j, int l)
{
    if (l == 0) return n;
    uint64_t kj = K[j];
    int64_t lo = j, step = 1;  // lcp(kj, K[lo]) >= l
    int64_t hi = n;            // the first failing candidate, or n
    for (;;) {
        const int64_t probe = j + step;
        if (probe >= n) break;
        if (lcp_digits(kj, K[probe]) >= l) {
            lo = probe;
            step <<= 1;
        } else {
            hi = probe;
            break;
        }
    }
    while (hi - lo > 1) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (lcp_digits(kj, K[mid]) >= l) lo = mid;
        else hi = mid;
    }
    return hi;
}

__device__ __forceinline__ int first_level(const uint64_t* K, int64_t j)
{
    return j == 0 ? 0 : lcp_digits(K[j - 1], K[j]) + 1;
}

// The boxes in preorder, one thread per box (balanced: a particle may start
// up to 25 boxes, most start none): k_owner writes, for every box, the
// particle that starts it; k_nodes_by_box then finds the box's level and
// run.
__global__ void k_owner(int64_t n, const uint32_t* off, uint32_t* owner)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t a = off[j], b = off[j + 1];
    for (uint32_t v = a; v < b; ++v) owner[v] = (uint32_t)j;
}

__global__ void k_nodes_by_box(const uint64_t* K, int64_t n, const uint8_t* Lp, const uint32_t* off,
                               const uint32_t* owner, uint32_t n_nodes, uint32_t* lvl, uint32_t* first,
                               uint32_t* count, uint32_t* skip, uint8_t* isleaf)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_nodes) return;
    const int64_t j = owner[v];
    const int l = first_level(K, j) + (int)(v - off[j]);
    const int64_t e = run_end(K, n, j, l);
    lvl[v] = (uint32_t)l;
    first[v] = (uint32_t)j;
    count[v] = (uint32_t)(e - j);
    isleaf[v] = l == Lp[j] ? 1 : 0;
    skip[v] = e < n ? off[e] : n_nodes;
}

__global__ void k_nchild(uint32_t n_nodes, const uint8_t* isleaf, const uint32_t* skip,
                         uint8_t* nchild, uint32_t* err)
{
    uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_nodes) return;
    if (isleaf[v]) { nchild[v] = 0; return; }
    uint32_t c = v + 1, end = skip[v];
    int k = 0;
    while (c < end && k < 5) { ++k; c = skip[c]; }
    if (k < 1 || k > 4) atomicOr(err, DERR_INDEX);
    nchild[v] = (uint8_t)(k > 4 ? 4 : k);
}

__global__ void k_invert(const uint32_t* bfs2pre, uint32_t n_nodes, uint32_t* pre2bfs)
{
    uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n_nodes) pre2bfs[bfs2pre[b]] = b;
}

__global__ void k_level_bounds(const uint32_t* lvl_sorted, uint32_t n_nodes, uint32_t* level_start)
{
    uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_nodes) return;
    uint32_t l = lvl_sorted[b];
    if (b == 0 || lvl_sorted[b - 1] != l) level_start[l] = b;
    if (b == n_nodes - 1) level_start[kMaxDepth + 1] = l;  // deepest level
}

__global__ void k_links(uint32_t n_nodes, const uint32_t* bfs2pre, const uint32_t* pre2bfs,
                        const uint32_t* lvl, const uint32_t* first, const uint32_t* count,
                        const uint8_t* isleaf, const uint8_t* nchild, int4* link, uint8_t* node_level,
                        uint32_t* n_leaves, int* parent, uint32_t* first_bfs, uint32_t* leaf_of)
{
    uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_nodes) return;
    uint32_t v = bfs2pre[b];
    first_bfs[b] = first[v];
    int4 L;
    if (isleaf[v]) {
        L.x = (int)first[v];
        L.y = (int)count[v] | kLeafBit;
        atomicAdd(n_leaves, 1u);
        for (uint32_t k = 0; k < count[v]; ++k) leaf_of[first[v] + k] = b;
    } else {
        L.x = (int)pre2bfs[v + 1];
        L.y = (int)nchild[v];
        for (int c = 0; c < L.y; ++c) parent[L.x + c] = (int)b;
    }
    if (b == 0) parent[0] = -1;
    L.z = 0;
    L.w = 0;
    link[b] = L;
    node_level[b] = (uint8_t)lvl[v];
}

// ---------------------------------------------------------- 5. moments

__device__ __forceinline__ float f32_up(double x) { return __double2float_ru(x); }

template <typename T> __device__ __forceinline__ T round_up(double x);
template <> __device__ __forceinline__ float round_up<float>(double x) { return __double2float_ru(x); }
template <> __device__ __forceinline__ double round_up<double>(double x) { return x * (1.0 + 4e-16); }

// Monopole, centre of mass, quadrupole, r_cm and r_cut^2 of box b (BFS
// index) from its particles (a leaf) or its children (children in order),
// about the box centre, in the arithmetic type A: FP64 for the FP64 tree and
// for the top kFp64Levels levels of the FP32 tree, FP32 below (a box there
// holds few particles, and its moments are stored in FP32 anyway; GB300's
// FP64 pipe has 1/64 of the FP32 rate).  r_cm and r_cut^2 are formed in FP64
// from the stored centre of mass in every case (r_cm rounded down, r_cut^2
// up).  Level and first particle come in BFS order.  Children are read
// through L2 (__ldcg): other threads of the launch wrote them, and a line
// cached in L1 before one of them was written would be stale.  A box's
// (M, centre of mass, Q2) for its parent are kept in the type they were
// computed in (mom/q2 in FP64, momf/q2f in FP32), so that a parent in FP32
// reads its children without conversions on the FP64 pipe.
// inv_theta2 = 1/theta^2 (infinite r_cut when theta = 0).
constexpr int kFp64Levels = 8;

struct MomentsOut {
    dbl4* mom;      // FP64 boxes: {M, x_cm, y_cm, side}
    double2* q2;
    float4* momf;   // FP32 boxes: {M, x_cm, y_cm, 0}
    float2* q2f;
};

// GEO: also r_cm and r_cut^2 here (the FP64 tree); the FP32 tree's boxes get
// them from k_rcut, one thread per box, so that the FP64 arithmetic they
// need runs in full warps rather than in the climb's divergent ones, and an
// FP32 box's reference point is formed in FP32 (side0f = 2 half, x0f, y0f:
// the root box in FP32).
template <typename T, typename A, bool GEO>
__device__ __forceinline__ void node_moments(uint32_t b, int l, uint32_t ix, uint32_t iy, const int4 L,
                                             const vec4_t<T>* sorted, const RootBox* rb, double inv_theta2,
                                             const MomentsOut& O, vec4_t<T>* nodeA,
                                             typename V2<T>::type* nodeB, float* rcm_out, float side0f,
                                             float x0f, float y0f)
{
    // box (ix, iy) of level l; the moments are taken about its centre (any
    // point of the box would do: in FP32 boxes the centre rounded in FP32)
    // 2^-l built from its exponent: exact, and no FP64 division (slow here)
    double side = 0.0, cxd = 0.0, cyd = 0.0;
    A cx, cy;
    if (GEO || sizeof(A) == 8) {
        side = (2.0 * rb->half) * __longlong_as_double((long long)(1023 - l) << 52);
        cxd = rb->x0 + (ix + 0.5) * side;
        cyd = rb->y0 + (iy + 0.5) * side;
        cx = (A)cxd;
        cy = (A)cyd;
    } else {
        const float sf = side0f * __int_as_float((127 - l) << 23);
        cx = (A)fmaf((float)ix + 0.5f, sf, x0f);
        cy = (A)fmaf((float)iy + 0.5f, sf, y0f);
    }
    A M = 0, sx = 0, sy = 0, qr = 0, qi = 0;
    if (L.y & kLeafBit) {
        const int cnt = L.y & kCountMask;
        for (int k = 0; k < cnt; ++k) {
            vec4_t<T> r = sorted[L.x + k];
            A m = (A)r.z;
            M += m;
            sx += m * ((A)r.x - cx);
            sy += m * ((A)r.y - cy);
        }
        const A inv = M > A(0) ? A(1) / M : A(0);
        const A dx = sx * inv, dy = sy * inv;
        for (int k = 0; k < cnt; ++k) {
            vec4_t<T> r = sorted[L.x + k];
            A m = (A)r.z;
            A ax = (A)r.x - cx - dx, ay = (A)r.y - cy - dy;
            qr += m * (ax * ax - ay * ay);
            qi += m * A(2) * ax * ay;
        }
        sx = dx;
        sy = dy;
    } else {
        A cm[4], cxk[4], cyk[4], cqr[4], cqi[4];
        if (sizeof(T) == 4 && l + 1 >= kFp64Levels) {
            // children stored in FP32
            for (int k = 0; k < L.y; ++k) {
                const float4 m4 = __ldcg(O.momf + L.x + k);
                const float2 cq = __ldcg(O.q2f + L.x + k);
                cm[k] = (A)m4.x;
                cxk[k] = (A)m4.y - cx;
                cyk[k] = (A)m4.z - cy;
                cqr[k] = (A)cq.x;
                cqi[k] = (A)cq.y;
            }
        } else {
            for (int k = 0; k < L.y; ++k) {
                const double* pm = reinterpret_cast<const double*>(O.mom + L.x + k);
                const double2 cq = __ldcg(O.q2 + L.x + k);
                cm[k] = (A)__ldcg(pm);
                cxk[k] = (A)__ldcg(pm + 1) - cx;
                cyk[k] = (A)__ldcg(pm + 2) - cy;
                cqr[k] = (A)cq.x;
                cqi[k] = (A)cq.y;
            }
        }
        for (int k = 0; k < L.y; ++k) {
            M += cm[k];
            sx += cm[k] * cxk[k];
            sy += cm[k] * cyk[k];
        }
        const A inv = M > A(0) ? A(1) / M : A(0);
        const A dx = sx * inv, dy = sy * inv;
        for (int k = 0; k < L.y; ++k) {
            A ax = cxk[k] - dx, ay = cyk[k] - dy;
            qr += cqr[k] + cm[k] * (ax * ax - ay * ay);
            qi += cqi[k] + cm[k] * A(2) * ax * ay;
        }
        sx = dx;
        sy = dy;
    }
    const A cmx = cx + sx, cmy = cy + sy;
    if (sizeof(T) == 4 && l >= kFp64Levels) {
        O.momf[b] = make_float4((float)M, (float)cmx, (float)cmy, 0.f);
        O.q2f[b] = make_float2((float)qr, (float)qi);
    } else {
        O.mom[b] = make_dbl4((double)M, (double)cmx, (double)cmy, side);
        O.q2[b] = make_double2((double)qr, (double)qi);
    }
    vec4_t<T> Av;
    Av.x = (T)cmx; Av.y = (T)cmy; Av.z = (T)M; Av.w = (T)0;
    if constexpr (GEO) {
        // r_cm: distance from the centre of mass to the farthest corner of the box
        const double ex = fabs((double)cmx - cxd) + 0.5 * side, ey = fabs((double)cmy - cyd) + 0.5 * side;
        const double rcm2 = ex * ex + ey * ey;
        Av.w = round_up<T>(rcm2 * inv_theta2);
        rcm_out[b] = __fsqrt_rd(__double2float_rd(rcm2));
    }
    nodeA[b] = Av;
    typename V2<T>::type B;
    B.x = (T)qr; B.y = (T)qi;
    nodeB[b] = B;
}

// r_cm and r_cut^2 of every box of the FP32 tree from its stored centre of
// mass (the one the walk uses), in FP64 about the exact box centre: r_cm
// rounded down, r_cut^2 = r_cm^2 / theta^2 rounded up.
__global__ void k_rcut(uint32_t n_nodes, const uint8_t* node_level, const uint32_t* first_bfs, const uint64_t* K,
                       const RootBox* rb, double inv_theta2, float4* nodeA, float* rcm_out)
{
    uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_nodes) return;
    const int l = node_level[b];
    const uint64_t key = K[first_bfs[b]];
    const uint32_t ix = compact24(key) >> (kMaxDepth - l), iy = compact24(key >> 1) >> (kMaxDepth - l);
    const double side = (2.0 * rb->half) * __longlong_as_double((long long)(1023 - l) << 52);
    const double cxd = rb->x0 + (ix + 0.5) * side, cyd = rb->y0 + (iy + 0.5) * side;
    float4 A = nodeA[b];
    const double ex = fabs((double)A.x - cxd) + 0.5 * side, ey = fabs((double)A.y - cyd) + 0.5 * side;
    const double rcm2 = ex * ex + ey * ey;
    A.w = __double2float_ru(rcm2 * inv_theta2);
    nodeA[b] = A;
    rcm_out[b] = __fsqrt_rd(__double2float_rd(rcm2));
}

// The moments of every box in one launch, bottom-up.  One thread per box;
// a leaf's thread computes the leaf, then counts it at its parent (one
// atomic per box), and the child that completes the count computes the
// parent from its children and climbs on.  Every box is computed once, by
// whichever child finishes last; no thread ever waits for another.
template <typename T>
__global__ void k_moments_up(uint32_t n_nodes, const uint8_t* node_level, const uint32_t* first_bfs,
                             const int4* link, const int* parent, const vec4_t<T>* sorted, const uint64_t* K,
                             const RootBox* rb, double inv_theta2, MomentsOut O, vec4_t<T>* nodeA,
                             typename V2<T>::type* nodeB, float* rcm_out, uint32_t* ready)
{
    uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_nodes) return;
    int4 L = link[b];
    if (!(L.y & kLeafBit)) return;
    int l = node_level[b];
    constexpr bool GEO = sizeof(T) == 8;
    const float side0f = GEO ? 0.f : (float)(2.0 * rb->half);
    const float x0f = GEO ? 0.f : (float)rb->x0, y0f = GEO ? 0.f : (float)rb->y0;
    const uint64_t key = K[first_bfs[b]];
    // the climb derives each parent's cell from its child's: no further
    // loads of keys or levels on the way up
    uint32_t ix = compact24(key) >> (kMaxDepth - l), iy = compact24(key >> 1) >> (kMaxDepth - l);
    int p = parent[b];
    for (;;) {
        if (sizeof(T) == 4 && l >= kFp64Levels)
            node_moments<T, float, GEO>(b, l, ix, iy, L, sorted, rb, inv_theta2, O, nodeA, nodeB, rcm_out, side0f,
                                        x0f, y0f);
        else
            node_moments<T, double, GEO>(b, l, ix, iy, L, sorted, rb, inv_theta2, O, nodeA, nodeB, rcm_out, side0f,
                                         x0f, y0f);
        if (p < 0) return;
        // the parent's links (written by earlier launches) are read beside
        // the count.  The count is an acquire-release atomic: it publishes this
        // box's moments, and the completing count sees every sibling's.
        const int4 Lp = link[p];
        const int pp = parent[p];
        uint32_t done;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(done) : "l"(ready + p) : "memory");
        if (done + 1u < (uint32_t)Lp.y) return;   // a box's y is its child count
        b = (uint32_t)p;
        L = Lp;
        p = pp;
        --l;
        ix >>= 1;
        iy >>= 1;
    }
}

// ------------------------------------------- 6. records and big lists

__device__ __forceinline__ double support_radius(int kind, double shape, double p)
{
    return kind == LENS_POINT ? 0.0 : shape * p;
}

// Listing box of every particle: the shallowest box on its path whose side
// times lambda its support radius s exceeds (found by climbing the parent
// links from its leaf), and the softening radius r0 of a listed particle.
// Sort keys: the listing level (kUnlisted if none).  Boxes are numbered
// level by level, in Morton order within a level, and the particles are in
// Morton order, so the particles listed at one level are already in the
// order of their listing boxes: a stable sort by level is the stable sort by
// box (one 8-bit radix pass instead of a pass per 8 bits of box index).
constexpr uint32_t kUnlisted = 31;
template <typename T>
__global__ void k_biglevel(const vec4_t<T>* sorted, int64_t n, const uint8_t* node_level, const uint32_t* leaf_of,
                           const int* parent, const float* rcm, const RootBox* rb, int kind, double shape,
                           double theta, double lambda, uint32_t n_nodes, uint32_t* bkey, uint32_t* bval,
                           uint32_t* bnode, double* r0sq, uint32_t* n_big)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool listed = false;
    if (j < n) {
        double s = support_radius(kind, shape, (double)sorted[j].w);
        const uint32_t leaf = leaf_of[j];
        const int L = node_level[leaf];
        // the smallest l with s > c 2^-l, c = lambda * side0 (2^-l scales
        // exactly): with c = mc 2^ec and s = ms 2^es (mantissas in [0.5, 1)),
        // l = ec - es if ms > mc, else ec - es + 1 (at least 0)
        const double c = lambda * (2.0 * rb->half);
        int lp = -1;
        if (s > 0.0) {
            if (c == 0.0) {
                lp = 0;
            } else {
                int ec, es;
                const double mc = frexp(c, &ec), ms = frexp(s, &es);
                const int l0 = ec - es + (ms > mc ? 0 : 1);
                lp = l0 < 0 ? 0 : l0;
                if (lp > L) lp = -1;
            }
        }
        bval[j] = (uint32_t)j;
        if (lp < 0) {
            bkey[j] = kUnlisted;
            bnode[j] = n_nodes;
            r0sq[j] = 0.0;
        } else {
            uint32_t v = leaf;
            for (int l = L; l > lp; --l) v = (uint32_t)parent[v];
            bkey[j] = (uint32_t)lp;
            bnode[j] = v;
            // softening radius of the listed particle inside its leaf: any cell
            // whose multipole contains the particle and is accepted lies farther
            // than r_cm(leaf) (1/theta - 1) from the ray (r_cm grows towards the root)
            double r0;
            if (theta <= 0.0) r0 = s;
            else if (theta >= 1.0) r0 = 0.0;
            else r0 = fmin(s, (double)rcm[leaf] * (1.0 / theta - 1.0));
            r0 *= 0.999;
            r0sq[j] = r0 * r0;
            listed = true;
        }
    }
    const unsigned ball = __ballot_sync(0xffffffffu, listed);
    if ((threadIdx.x & 31) == 0 && ball) atomicAdd(n_big, (uint32_t)__popc(ball));
}

// The listing box of each entry in sorted order.
__global__ void k_bigkeys(const uint32_t* sval, const uint32_t* bnode, int64_t n, uint32_t* skey)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) skey[i] = bnode[sval[i]];
}

__global__ void k_bigcsr(const uint32_t* skey, int64_t n, uint32_t n_nodes, int4* link, uint32_t* end)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k = skey[i];
    if (k >= n_nodes) return;
    if (i == 0 || skey[i - 1] != k) link[k].z = (int)i;
    if (i == n - 1 || skey[i + 1] != k) end[k] = (uint32_t)(i + 1);
}

__global__ void k_bigcount(uint32_t n_nodes, int4* link, const uint32_t* end)
{
    uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_nodes) return;
    uint32_t e = end[b];
    if (e) link[b].w = (int)(e - (uint32_t)link[b].z);
}

template <typename T>
__global__ void k_bigrecords(const uint32_t* sval, const uint32_t* d_nbig, const vec4_t<T>* e0,
                             const vec4_t<T>* e1, const vec4_t<T>* sorted, const double* r0sq,
                             int kind, double shape, double invNq, vec4_t<T>* big0, vec4_t<T>* big1,
                             uint32_t* big_pid, vec4_t<T>* leaf0, uint8_t* listed)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)*d_nbig) return;
    uint32_t j = sval[i];
    vec4_t<T> q = e0[j];
    double s = support_radius(kind, shape, (double)sorted[j].w);
    vec4_t<T> a, b;
    a.x = q.x;
    a.y = q.y;
    a.z = (T)(s * s);
    a.w = r0sq[j] > 0.0 ? (T)(1.0 / r0sq[j]) : (T)INFINITY;  // 1/r0^2
    b.x = kind == LENS_GAUSS ? (T)((double)q.z * invNq) : q.z;  // m/N_q (GAUSS) or m
    if (kind == LENS_NFW) {
        vec4_t<T> q1 = e1[j];
        b.y = q1.x;  // A = m / g(X)
        b.z = q1.y;  // B = 1 / r_s
        b.w = (T)0;
    } else {
        double c = (double)q.w, sig = (double)sorted[j].w;
        b.y = (T)(c * 1.4426950408889634074);                 // c log2(e), c = 1/(2 r_sm^2)
        b.z = (T)((double)q.z * c * invNq);                   // m c / N_q
        b.w = (T)(2.0 * sig * sig);                           // 1 / c
    }
    big0[i] = a;
    big1[i] = b;
    big_pid[i] = j;
    leaf0[j].w = -(T)r0sq[j];  // listed: a softened point inside leaves
    listed[j] = 1;
}

// Support extent of one big entry {x, y, s^2, .}, rounded outwards.
__device__ __forceinline__ void entry_extent(const float4& q, float& x0, float& y0, float& x1, float& y1)
{
    const float r = __fsqrt_ru(q.z);
    x0 = fminf(x0, __fsub_rd(q.x, r));
    y0 = fminf(y0, __fsub_rd(q.y, r));
    x1 = fmaxf(x1, __fadd_ru(q.x, r));
    y1 = fmaxf(y1, __fadd_ru(q.y, r));
}
__device__ __forceinline__ void entry_extent(const dbl4& q, double& x0, double& y0, double& x1, double& y1)
{
    const double r = sqrt(q.z);
    x0 = fmin(x0, q.x - r);
    y0 = fmin(y0, q.y - r);
    x1 = fmax(x1, q.x + r);
    y1 = fmax(y1, q.y + r);
}

// Bounding box of the support squares [x - s, x + s] x [y - s, y + s] of big
// entries [b, e): per 32-entry chunk and per node list (conservative bounds
// for skipping a list or a chunk whose supports cannot reach a ray group).
template <typename T>
__device__ __forceinline__ vec4_t<T> support_box(const vec4_t<T>* big0, int64_t b, int64_t e)
{
    T x0 = T(INFINITY), y0 = T(INFINITY), x1 = T(-INFINITY), y1 = T(-INFINITY);
    for (int64_t i = b; i < e; ++i) entry_extent(big0[i], x0, y0, x1, y1);
    vec4_t<T> r;
    r.x = x0; r.y = y0; r.z = x1; r.w = y1;
    return r;
}

template <typename T>
__global__ void k_chunkbox(const vec4_t<T>* big0, const uint32_t* d_nbig, int64_t max_chunks, vec4_t<T>* out)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nbig = *d_nbig;
    if (c >= max_chunks || 32 * c >= nbig) return;
    int64_t b = 32 * c, e = b + 32 < nbig ? b + 32 : nbig;
    out[c] = support_box<T>(big0, b, e);
}

// Boxes of 1,024-entry superchunks (32 chunks): one warp each.
template <typename T>
__global__ void k_superbox(const vec4_t<T>* chunk, const uint32_t* d_nbig, int64_t n_super, vec4_t<T>* out)
{
    const int64_t sc = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (sc >= n_super) return;
    const int64_t nbig = *d_nbig, c = 32 * sc + lane;
    T x0 = T(INFINITY), y0 = T(INFINITY), x1 = T(-INFINITY), y1 = T(-INFINITY);
    if (32 * c < nbig) {
        vec4_t<T> b = chunk[c];
        x0 = b.x; y0 = b.y; x1 = b.z; y1 = b.w;
    }
    for (int o = 16; o; o >>= 1) {
        x0 = fmin(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        x1 = fmax(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        y0 = fmin(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        y1 = fmax(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    }
    if (lane == 0) {
        vec4_t<T> r;
        r.x = x0; r.y = y0; r.z = x1; r.w = y1;
        out[sc] = r;
    }
}

// Entries [z, e) of a list by this lane: whole 32-entry chunks by their
// boxes, the partial chunks at the two ends entry by entry.
template <typename T>
__device__ __forceinline__ void range_extent(int64_t z, int64_t e, int lane, const vec4_t<T>* big0,
                                             const vec4_t<T>* chunk, T& x0, T& y0, T& x1, T& y1)
{
    int64_t c0 = (z + 31) >> 5, c1 = e >> 5;  // whole chunks [c0, c1)
    for (int64_t c = c0 + lane; c < c1; c += 32) {
        vec4_t<T> b = chunk[c];
        x0 = fmin(x0, b.x); y0 = fmin(y0, b.y);
        x1 = fmax(x1, b.z); y1 = fmax(y1, b.w);
    }
    int64_t head_end = c0 < c1 ? 32 * c0 : e, tail_begin = c0 < c1 ? 32 * c1 : e;
    for (int64_t i = z + lane; i < head_end; i += 32) entry_extent(big0[i], x0, y0, x1, y1);
    for (int64_t i = tail_begin + lane; i < e; i += 32) entry_extent(big0[i], x0, y0, x1, y1);
}

// Big-list box of every node, in two launches.  k_nodebox: one thread per
// node; a node without a list gets the empty box (+inf, +inf, -inf, -inf),
// which no reader looks at; a list of at most kShortList entries is reduced
// by its own thread; a longer list is queued.  k_nodebox_long: each warp
// takes queued lists one at a time, all 32 lanes on one list [z, z + w):
// covered by the boxes of its whole 1,024-entry superchunks, of the whole
// 32-entry chunks at its two ends and by the single entries of the partial
// chunks, reduced in the tree's precision (chunk boxes are already rounded
// outwards; min and max do not round).  The long lists are those of the top
// levels: spread over warps rather than met one after another by the warp
// that holds the first boxes.
constexpr int kShortList = 32;

template <typename T>
__global__ void k_nodebox(const int4* link, uint32_t n_nodes, const vec4_t<T>* big0, vec4_t<T>* out,
                          uint32_t* queue, uint32_t* n_queued)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = v < n_nodes;
    const int4 L = valid ? link[v] : make_int4(0, 0, 0, 0);
    const bool longl = valid && L.w > kShortList;
    const unsigned q = __ballot_sync(0xffffffffu, longl);
    uint32_t at = 0;
    if (lane == 0 && q) at = atomicAdd(n_queued, (uint32_t)__popc(q));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (longl) queue[at + __popc(q & ((1u << lane) - 1u))] = (uint32_t)v;
    if (!valid || longl) return;
    T x0 = T(INFINITY), y0 = T(INFINITY), x1 = T(-INFINITY), y1 = T(-INFINITY);
#pragma unroll 4
    for (int k = 0; k < L.w; ++k) entry_extent(big0[(int64_t)L.z + k], x0, y0, x1, y1);
    vec4_t<T> r;
    r.x = x0; r.y = y0; r.z = x1; r.w = y1;
    out[v] = r;
}

template <typename T>
__global__ void k_nodebox_long(const int4* link, const vec4_t<T>* big0, const vec4_t<T>* chunk,
                               const vec4_t<T>* super, const uint32_t* queue, const uint32_t* n_queued,
                               vec4_t<T>* out)
{
    const int lane = threadIdx.x & 31;
    const uint32_t nq = *n_queued;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t k = ((uint32_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nq; k += nw) {
        const uint32_t v = queue[k];
        const int4 L = link[v];
        const int64_t z = L.z, e = z + L.w;
        T x0 = T(INFINITY), y0 = T(INFINITY), x1 = T(-INFINITY), y1 = T(-INFINITY);
        // whole superchunks [s0, s1) by their boxes, the ends by range_extent
        const int64_t s0 = (z + 1023) >> 10, s1 = e >> 10;
        if (s0 < s1) {
            for (int64_t sc = s0 + lane; sc < s1; sc += 32) {
                vec4_t<T> b = super[sc];
                x0 = fmin(x0, b.x); y0 = fmin(y0, b.y);
                x1 = fmax(x1, b.z); y1 = fmax(y1, b.w);
            }
            range_extent<T>(z, 1024 * s0, lane, big0, chunk, x0, y0, x1, y1);
            range_extent<T>(1024 * s1, e, lane, big0, chunk, x0, y0, x1, y1);
        } else {
            range_extent<T>(z, e, lane, big0, chunk, x0, y0, x1, y1);
        }
        for (int o = 16; o; o >>= 1) {
            x0 = fmin(x0, __shfl_xor_sync(0xffffffffu, x0, o));
            x1 = fmax(x1, __shfl_xor_sync(0xffffffffu, x1, o));
            y0 = fmin(y0, __shfl_xor_sync(0xffffffffu, y0, o));
            y1 = fmax(y1, __shfl_xor_sync(0xffffffffu, y1, o));
        }
        if (lane == 0) {
            vec4_t<T> r;
            r.x = x0; r.y = y0; r.z = x1; r.w = y1;
            out[v] = r;
        }
    }
}

__global__ void k_iota_u32(uint32_t* a, uint32_t n)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = i;
}

// ================================================================ host

// What the host learns of a build only when it asks (lens_tree_get_info,
// lens_tree_export, the adjoint): written on the device at the end of the
// build, so the build itself synchronises once (to size the node arrays).
struct BuildMeta {
    uint32_t level_start[kMaxDepth + 2];  // BFS start of each level; [kMaxDepth + 1] = deepest level
    uint32_t nbig, nleaves, pad[2];
    RootBox rb;
};

lens_status wait_built(const lens_tree* t, cudaStream_t s)
{
    if (!t->built) return LENS_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    LENS_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return LENS_OK;
    LENS_CUDA(cudaStreamWaitEvent(s, t->built, 0));
    return LENS_OK;
}

// A non-blocking stream of the current device for the host's reads of a
// finished build's counts: a copy on the legacy default stream would also
// wait for whatever was queued after the build there (a walk, an adjoint).
static lens_status meta_stream(cudaStream_t* out)
{
    static std::mutex mu;
    static std::vector<cudaStream_t> streams;
    int dev = 0;
    LENS_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if ((int)streams.size() <= dev) streams.resize(dev + 1, nullptr);
    if (!streams[dev]) LENS_CUDA(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking));
    *out = streams[dev];
    return LENS_OK;
}

lens_status finish_species(SpeciesTree& st)
{
    if (st.meta_ready || st.n == 0) return LENS_OK;
    LENS_CUDA(cudaEventSynchronize(st.ev[4]));  // the build (and its count copies) are done
    BuildMeta m;
    cudaStream_t ms;
    LENS_TRY(meta_stream(&ms));
    LENS_CUDA(cudaMemcpyAsync(&m, st.d_meta, sizeof(m), cudaMemcpyDeviceToHost, ms));
    LENS_CUDA(cudaStreamSynchronize(ms));
    int depth = (int)m.level_start[kMaxDepth + 1];
    if (depth < 0 || depth > kMaxDepth) return lens_set_error(LENS_ERR_INTERNAL, "tree build: bad depth %d", depth);
    st.depth = depth;
    st.level_start.assign(depth + 2, 0);
    for (int l = 0; l <= depth; ++l) st.level_start[l] = m.level_start[l];
    st.level_start[depth + 1] = st.n_nodes;
    st.n_big = m.nbig;
    st.n_chunks = ((int64_t)m.nbig + 31) / 32;
    st.n_leaves = m.nleaves;
    st.root_cx = m.rb.cx;
    st.root_cy = m.rb.cy;
    st.root_half = m.rb.half;
    for (int k = 0; k < 4; ++k) {
        float ms = 0;
        LENS_CUDA(cudaEventElapsedTime(&ms, st.ev[k], st.ev[k + 1]));
        st.phase_ms[k] = ms;
    }
    st.meta_ready = true;
    return LENS_OK;
}

template <typename T>
static lens_status build_typed(lens_tree* t, SpeciesTree& st, const lens_species& in, cudaStream_t s)
{
    using T4 = vec4_t<T>;
    using T2 = typename V2<T>::type;
    // device time of the phases: events 0..4 around sort, layout, moments +
    // big lists, finish
    for (int k = 0; k < 5; ++k) LENS_CUDA(cudaEventCreate(&st.ev[k]));
    LENS_CUDA(cudaEventRecord(st.ev[0], s));
    const int64_t n = in.n;
    const int TB = 256;
    const unsigned G = grid_for(n, TB);
    StreamTemps tmps(s);  // temporaries (stream ordered), released on every return path
    T4* staged = nullptr;
    T4* sorted = nullptr;
    unsigned long long* bbox = nullptr;
    RootBox* rb = nullptr;
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = std::max(radix_sort_temp_bytes<uint64_t>(n), scan_temp_bytes(n + 1));
    LENS_CUDA(tmps.get(&staged, n * sizeof(T4)));
    LENS_CUDA(tmps.get(&sorted, n * sizeof(T4)));
    LENS_CUDA(tmps.get(&bbox, 4 * sizeof(unsigned long long)));
    LENS_CUDA(tmps.get(&rb, sizeof(RootBox)));
    LENS_CUDA(tmps.get(&k0, n * sizeof(uint64_t)));
    LENS_CUDA(tmps.get(&k1, n * sizeof(uint64_t)));
    LENS_CUDA(tmps.get(&v0, (n + 1) * sizeof(uint32_t)));
    LENS_CUDA(tmps.get(&v1, (n + 1) * sizeof(uint32_t)));
    LENS_CUDA(tmps.get(&tmp, tmp_bytes));

    unsigned long long init[4] = {~0ull, 0ull, ~0ull, 0ull};
    LENS_CUDA(cudaMemcpyAsync(bbox, init, sizeof(init), cudaMemcpyHostToDevice, s));
    { k_stage<T><<<G, TB, 0, s>>>(in.data, in.dtype, n, in.kind, staged, bbox, t->d_err); note_launch(); }
    { k_root<<<1, 1, 0, s>>>(bbox, rb); note_launch(); }
    { k_morton<T><<<G, TB, 0, s>>>(staged, n, rb, k0, v0); note_launch(); }
    uint64_t* K;
    uint32_t* P;
    radix_sort_pairs<uint64_t>(k0, v0, k1, v1, n, 0, kKeyBits, tmp, s, &K, &P, t->d_err);
    // the per-particle arrays the tree keeps (sized by n alone)
    LENS_CUDA(lens_malloc_async((void**)&st.perm, n * sizeof(uint32_t), s));
    LENS_CUDA(lens_malloc_async((void**)&st.exact0, n * sizeof(T4), s));
    if (in.kind == LENS_NFW) LENS_CUDA(lens_malloc_async((void**)&st.exact1, n * sizeof(T4), s));
    if (in.kind != LENS_POINT) {
        LENS_CUDA(lens_malloc_async((void**)&st.leaf0, n * sizeof(T4), s));
        LENS_CUDA(lens_malloc_async((void**)&st.listed, n, s));
        LENS_CUDA(cudaMemsetAsync(st.listed, 0, n, s));
    }
    double gX = 1.0;
    if (in.kind == LENS_NFW) {
        // host evaluation of g(X) = ln(X/2) + F(X), X = R_max / r_s
        double X = in.shape, F;
        if (std::fabs(1.0 - X * X) < 1e-4) {
            double u = 1.0 - X * X, sF = 0.0;
            for (int k = 12; k >= 0; --k) sF = sF * u + 1.0 / (2 * k + 1);
            F = sF;
        } else if (X < 1.0) {
            F = std::acosh(1.0 / X) / std::sqrt(1.0 - X * X);
        } else {
            F = std::acos(1.0 / X) / std::sqrt(X * X - 1.0);
        }
        gX = std::log(0.5 * X) + F;
    }
    { k_gather<T><<<G, TB, 0, s>>>(staged, P, n, sorted, st.perm, in.kind, in.shape, gX, (T4*)st.exact0,
                                 (T4*)st.exact1, (T4*)st.leaf0); note_launch(); }
    LENS_CUDA(cudaEventRecord(st.ev[1], s));

    // topology
    uint8_t* Lp = nullptr;
    uint32_t* off = nullptr;   // n + 1: owned-box offsets, last = n_nodes
    LENS_CUDA(tmps.get(&Lp, n));
    LENS_CUDA(tmps.get(&off, (n + 1) * sizeof(uint32_t)));
    { k_levels<<<G, TB, 0, s>>>(K, n, t->leaf_max, Lp, off); note_launch(); }
    scan_exclusive_u32(off, off, n, off + n, tmp, s);
    // the one synchronisation of the build: the node count sizes the node
    // arrays; the staging kernel's input check is read with it
    uint32_t n_nodes = 0, herr = 0;
    LENS_CUDA(cudaMemcpyAsync(&n_nodes, off + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    LENS_CUDA(cudaMemcpyAsync(&herr, t->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    LENS_CUDA(cudaStreamSynchronize(s));
    if (herr & DERR_BAD_INPUT)
        return lens_set_error(LENS_ERR_INVALID_ARG, "negative or non-finite particle mass or size");
    if (n_nodes == 0 || n_nodes > (uint32_t)kCountMask)
        return lens_set_error(LENS_ERR_INTERNAL, "tree build: bad node count %u", n_nodes);
    st.n_nodes = n_nodes;
    const unsigned GN = grid_for(n_nodes, TB);
    {
        // the level sort and scans below run over n_nodes elements
        size_t need = std::max(radix_sort_temp_bytes<uint32_t>(n_nodes), scan_temp_bytes((int64_t)n_nodes + 1));
        if (need > tmp_bytes) {
            tmps.release(tmp);
            tmp_bytes = need;
            LENS_CUDA(tmps.get(&tmp, tmp_bytes));
        }
    }

    uint32_t *lvl = nullptr, *first = nullptr, *count = nullptr, *skip = nullptr;
    uint32_t *lk1 = nullptr, *lv0 = nullptr, *lv1 = nullptr, *pre2bfs = nullptr;
    uint32_t *level_start = nullptr, *counters = nullptr;
    uint8_t *isleaf = nullptr, *nchild = nullptr;
    LENS_CUDA(tmps.get(&lvl, n_nodes * sizeof(uint32_t)));
    LENS_CUDA(tmps.get(&first, n_nodes * sizeof(uint32_t)));
    LENS_CUDA(tmps.get(&count, n_nodes * sizeof(uint32_t)));
    LENS_CUDA(tmps.get(&skip, n_nodes * sizeof(uint32_t)));
    LENS_CUDA(tmps.get(&lk1, n_nodes * sizeof(uint32_t)));
    LENS_CUDA(tmps.get(&lv0, n_nodes * sizeof(uint32_t)));
    LENS_CUDA(tmps.get(&lv1, n_nodes * sizeof(uint32_t)));
    LENS_CUDA(tmps.get(&pre2bfs, n_nodes * sizeof(uint32_t)));
    LENS_CUDA(tmps.get(&level_start, (kMaxDepth + 2) * sizeof(uint32_t)));
    LENS_CUDA(tmps.get(&counters, 4 * sizeof(uint32_t)));
    LENS_CUDA(tmps.get(&isleaf, n_nodes));
    LENS_CUDA(tmps.get(&nchild, n_nodes));
    LENS_CUDA(cudaMemsetAsync(counters, 0, 4 * sizeof(uint32_t), s));
    LENS_CUDA(cudaMemsetAsync(level_start, 0xff, (kMaxDepth + 2) * sizeof(uint32_t), s));
    {
        uint32_t* owner = lv1;  // free until the level sort
        { k_owner<<<G, TB, 0, s>>>(n, off, owner); note_launch(); }
        { k_nodes_by_box<<<GN, TB, 0, s>>>(K, n, Lp, off, owner, n_nodes, lvl, first, count, skip, isleaf);
          note_launch(); }
    }
    { k_nchild<<<GN, TB, 0, s>>>(n_nodes, isleaf, skip, nchild, t->d_err); note_launch(); }
    // breadth-first order: stable sort of preorder ids by level
    LENS_CUDA(cudaMemcpyAsync(lv0, lvl, n_nodes * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    uint32_t* ids = nullptr;  // values of the level sort: preorder ids
    LENS_CUDA(tmps.get(&ids, n_nodes * sizeof(uint32_t)));
    { k_iota_u32<<<GN, TB, 0, s>>>(ids, n_nodes); note_launch(); }
    uint32_t *lvl_sorted, *bfs2pre;
    radix_sort_pairs<uint32_t>(lv0, ids, lv1, lk1, n_nodes, 0, 8, tmp, s, &lvl_sorted, &bfs2pre, t->d_err);
    { k_invert<<<GN, TB, 0, s>>>(bfs2pre, n_nodes, pre2bfs); note_launch(); }
    { k_level_bounds<<<GN, TB, 0, s>>>(lvl_sorted, n_nodes, level_start); note_launch(); }
    LENS_CUDA(lens_malloc_async(&st.d_meta, sizeof(BuildMeta), s));
    LENS_CUDA(cudaMemcpyAsync(((BuildMeta*)st.d_meta)->level_start, level_start, (kMaxDepth + 2) * sizeof(uint32_t),
                              cudaMemcpyDeviceToDevice, s));

    // persistent node arrays
    LENS_CUDA(lens_malloc_async((void**)&st.nodeA, n_nodes * sizeof(T4), s));
    LENS_CUDA(lens_malloc_async((void**)&st.nodeB, n_nodes * sizeof(T2), s));
    LENS_CUDA(lens_malloc_async((void**)&st.link, n_nodes * sizeof(int4), s));
    LENS_CUDA(lens_malloc_async((void**)&st.node_rcm, n_nodes * sizeof(float), s));
    LENS_CUDA(lens_malloc_async((void**)&st.node_level, n_nodes, s));
    LENS_CUDA(lens_malloc_async((void**)&st.parent, n_nodes * sizeof(int), s));

    uint32_t* first_bfs = nullptr;  // first particle of every node, BFS order
    uint32_t* leaf_of = nullptr;    // leaf (BFS) of every particle
    LENS_CUDA(tmps.get(&first_bfs, n_nodes * sizeof(uint32_t)));
    LENS_CUDA(tmps.get(&leaf_of, n * sizeof(uint32_t)));
    { k_links<<<GN, TB, 0, s>>>(n_nodes, bfs2pre, pre2bfs, lvl, first, count, isleaf, nchild, st.link,
                              st.node_level, counters, st.parent, first_bfs, leaf_of); note_launch(); }
    LENS_CUDA(cudaEventRecord(st.ev[2], s));

    dbl4* mom = nullptr;
    double2* q2 = nullptr;
    uint32_t* ready = nullptr;
    LENS_CUDA(tmps.get(&mom, n_nodes * sizeof(dbl4)));
    LENS_CUDA(tmps.get(&q2, n_nodes * sizeof(double2)));
    MomentsOut mo{mom, q2, nullptr, nullptr};
    if (sizeof(T) == 4) {
        LENS_CUDA(tmps.get(&mo.momf, n_nodes * sizeof(float4)));
        LENS_CUDA(tmps.get(&mo.q2f, n_nodes * sizeof(float2)));
    }
    LENS_CUDA(tmps.get(&ready, n_nodes * sizeof(uint32_t)));
    LENS_CUDA(cudaMemsetAsync(ready, 0, n_nodes * sizeof(uint32_t), s));
    const double inv_theta2 = t->theta > 0.0 ? 1.0 / (t->theta * t->theta) : INFINITY;
    { k_moments_up<T><<<GN, TB, 0, s>>>(n_nodes, st.node_level, first_bfs, st.link, st.parent, sorted, K, rb,
                                      inv_theta2, mo, (T4*)st.nodeA, (T2*)st.nodeB, st.node_rcm, ready);
      note_launch(); }
    if (sizeof(T) == 4)
        { k_rcut<<<GN, TB, 0, s>>>(n_nodes, st.node_level, first_bfs, K, rb, inv_theta2, (float4*)st.nodeA,
                                   st.node_rcm); note_launch(); }

    if (in.kind != LENS_POINT) {
        double lambda = 0.5;
        if (t->theta > 0.0) lambda = std::min(0.5, std::max(0.0, (1.0 / t->theta - 1.0) / std::sqrt(2.0)));
        double* r0sq = nullptr;
        uint32_t *bk0 = nullptr, *bk1 = nullptr, *bv0 = nullptr, *bv1 = nullptr, *end = nullptr, *bnode = nullptr;
        LENS_CUDA(tmps.get(&r0sq, n * sizeof(double)));
        LENS_CUDA(tmps.get(&bnode, n * sizeof(uint32_t)));
        LENS_CUDA(tmps.get(&bk0, n * sizeof(uint32_t)));
        LENS_CUDA(tmps.get(&bk1, n * sizeof(uint32_t)));
        LENS_CUDA(tmps.get(&bv0, n * sizeof(uint32_t)));
        LENS_CUDA(tmps.get(&bv1, n * sizeof(uint32_t)));
        LENS_CUDA(tmps.get(&end, n_nodes * sizeof(uint32_t)));
        LENS_CUDA(cudaMemsetAsync(end, 0, n_nodes * sizeof(uint32_t), s));
        { k_biglevel<T><<<G, TB, 0, s>>>(sorted, n, st.node_level, leaf_of, st.parent, st.node_rcm, rb, in.kind, in.shape,
                                       t->theta, lambda, n_nodes, bk0, bv0, bnode, r0sq, counters + 1);
          note_launch(); }
        uint32_t *skey, *sval;
        radix_sort_pairs<uint32_t>(bk0, bv0, bk1, bv1, n, 0, 8, tmp, s, &skey, &sval, t->d_err);
        uint32_t* nkey = skey == bk0 ? bk1 : bk0;
        { k_bigkeys<<<G, TB, 0, s>>>(sval, bnode, n, nkey); note_launch(); }
        { k_bigcsr<<<G, TB, 0, s>>>(nkey, n, n_nodes, st.link, end); note_launch(); }
        { k_bigcount<<<GN, TB, 0, s>>>(n_nodes, st.link, end); note_launch(); }
        // the big arrays hold up to one entry per particle (the count is read
        // on the device), so the build does not wait for it
        const uint32_t* d_nbig = counters + 1;
        const int64_t max_chunks = (n + 31) / 32;
        LENS_CUDA(lens_malloc_async((void**)&st.big0, n * sizeof(T4), s));
        LENS_CUDA(lens_malloc_async((void**)&st.big1, n * sizeof(T4), s));
        LENS_CUDA(lens_malloc_async((void**)&st.big_pid, n * sizeof(uint32_t), s));
        { k_bigrecords<T><<<G, TB, 0, s>>>(
            sval, d_nbig, (T4*)st.exact0, (T4*)st.exact1, sorted, r0sq, in.kind, in.shape, st.invNq, (T4*)st.big0,
            (T4*)st.big1, st.big_pid, (T4*)st.leaf0, st.listed); note_launch(); }
        LENS_CUDA(lens_malloc_async((void**)&st.big_chunk, max_chunks * sizeof(T4), s));
        LENS_CUDA(lens_malloc_async((void**)&st.node_bigbox, (size_t)n_nodes * sizeof(T4), s));
        { k_chunkbox<T><<<grid_for(max_chunks, TB), TB, 0, s>>>((T4*)st.big0, d_nbig, max_chunks,
                                                              (T4*)st.big_chunk); note_launch(); }
        const int64_t n_super = (max_chunks + 31) / 32;
        T4* super = nullptr;
        LENS_CUDA(tmps.get(&super, n_super * sizeof(T4)));
        { k_superbox<T><<<grid_for(n_super * 32, TB), TB, 0, s>>>((T4*)st.big_chunk, d_nbig, n_super, super);
          note_launch(); }
        uint32_t* queue = nullptr;
        LENS_CUDA(tmps.get(&queue, (n_nodes + 1) * sizeof(uint32_t)));
        uint32_t* n_queued = queue + n_nodes;
        LENS_CUDA(cudaMemsetAsync(n_queued, 0, sizeof(uint32_t), s));
        { k_nodebox<T><<<grid_for((int64_t)n_nodes, TB), TB, 0, s>>>(st.link, n_nodes, (T4*)st.big0,
                                                                      (T4*)st.node_bigbox, queue, n_queued);
          note_launch(); }
        { k_nodebox_long<T><<<t->num_sms * 8, TB, 0, s>>>(st.link, (T4*)st.big0, (T4*)st.big_chunk, super, queue,
                                                          n_queued, (T4*)st.node_bigbox); note_launch(); }
    }
    LENS_CUDA(cudaEventRecord(st.ev[3], s));

    BuildMeta* dm = (BuildMeta*)st.d_meta;
    LENS_CUDA(cudaMemcpyAsync(&dm->nleaves, counters, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    LENS_CUDA(cudaMemcpyAsync(&dm->nbig, counters + 1, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    LENS_CUDA(cudaMemcpyAsync(&dm->rb, rb, sizeof(RootBox), cudaMemcpyDeviceToDevice, s));
    tmps.release_all();
    LENS_CUDA(cudaEventRecord(st.ev[4], s));
    LENS_CUDA(cudaGetLastError());
    return LENS_OK;
}

lens_status build_species(lens_tree* t, SpeciesTree& st, const lens_species& in, cudaStream_t s)
{
    st.kind = in.kind;
    st.prec = t->precision;
    st.n = in.n;
    st.shape = in.shape;
    if (in.kind == LENS_GAUSS) {
        st.Uq = 0.5 * in.shape * in.shape;
        st.invNq = 1.0 / (-std::expm1(-st.Uq));
    }
    if (in.n == 0) return LENS_OK;
    if (t->precision == LENS_PREC_FP64) return build_typed<double>(t, st, in, s);
    return build_typed<float>(t, st, in, s);
}

void free_species(SpeciesTree& st)
{
    void* ptrs[] = {st.nodeA, st.nodeB, st.link, st.node_rcm, st.node_level, st.exact0, st.exact1,
                    st.leaf0, st.big0, st.big1, st.perm, st.big_pid, st.listed, st.big_chunk,
                    st.node_bigbox, st.parent, st.d_meta};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, 0);
    for (cudaEvent_t& e : st.ev)
        if (e) cudaEventDestroy(e);
    st = SpeciesTree();
}

}  // namespace lens
