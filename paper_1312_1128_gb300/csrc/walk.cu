// walk.cu -- ray grouping and the warp-cooperative tree walk (Sec. 3.2 tree
// walk, Sec. 3.3 ray-parallel evaluation), plus the direct sum (Sec. 5.1,
// theta_force = 0) and the analytic components evaluated for every ray.
//
// One warp owns a group of up to 32*R spatially sorted rays and walks the tree
// once for the whole group:
//   - up to 32 candidate boxes are taken from the warp's stack at a time, one
//     per lane, and the MAC |x - x_cm| > r_cut is applied to the group's
//     bounding box (accepting a box only if every ray of the group would);
//   - accepted boxes go to a far buffer (monopole + quadrupole), opened leaves
//     to a near buffer of particle records, opened internal boxes push their
//     children; the big list of every visited box is scanned and the
//     particles whose support reaches the group's box go to a big buffer;
//   - full buffers are evaluated by all lanes, each lane for its own rays,
//     with the records broadcast from shared memory; partial sums are folded
//     into Neumaier-compensated totals after every buffer.
// Big-particle semantics (Sec. 3.2): every box's moments include all its
// particles as point masses.  A listed particle counts inside leaves as a
// point mass softened within r0 = min(s, r_cm(leaf)(1/theta - 1)), which is
// exactly the point mass wherever a cell containing it can be accepted, and
// its box's list adds (full profile - softened point) for rays inside its
// support s.  The softening removes the cancellation of a huge point term
// against its correction when a ray passes close to a listed particle.
#include <algorithm>
#include <cmath>

#include "profiles.cuh"
#include "sort.cuh"
#include "walk_shared.cuh"
#include "walk_dev.cuh"

namespace lens {

// ------------------------------------------------------------ grouping

__global__ void k_ray_bbox(const int64_t* boff, int nb, const double* borig, const void* dx,
                           const void* dy, int dtype, int64_t n, unsigned long long* bbox)
{
    __shared__ unsigned long long red[4][8];
    __shared__ int bsame;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = i < n;
    int b = valid ? batch_of(boff, nb, i) : -1;
    double px = 0, py = 0;
    if (valid) {
        px = borig[2 * b] + ray_offset(dx, dtype, i);
        py = borig[2 * b + 1] + ray_offset(dy, dtype, i);
    }
    // whole block in one batch (the common case): reduce in the block, then
    // four atomics per block
    int64_t first = (int64_t)blockIdx.x * blockDim.x;
    int64_t last = first + blockDim.x - 1 < n - 1 ? first + blockDim.x - 1 : n - 1;
    if (threadIdx.x == 0) bsame = batch_of(boff, nb, first) == batch_of(boff, nb, last);
    __syncthreads();
    const unsigned full = 0xffffffffu;
    unsigned long long x0 = valid ? dbl_to_ordered(px) : ~0ull, x1 = valid ? dbl_to_ordered(px) : 0ull;
    unsigned long long y0 = valid ? dbl_to_ordered(py) : ~0ull, y1 = valid ? dbl_to_ordered(py) : 0ull;
    if (bsame) {
        for (int o = 16; o; o >>= 1) {
            x0 = min(x0, __shfl_xor_sync(full, x0, o));
            x1 = max(x1, __shfl_xor_sync(full, x1, o));
            y0 = min(y0, __shfl_xor_sync(full, y0, o));
            y1 = max(y1, __shfl_xor_sync(full, y1, o));
        }
        int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) {
            red[0][w] = x0; red[1][w] = x1; red[2][w] = y0; red[3][w] = y1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int bb = batch_of(boff, nb, first);
            for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
                red[0][0] = min(red[0][0], red[0][k]);
                red[1][0] = max(red[1][0], red[1][k]);
                red[2][0] = min(red[2][0], red[2][k]);
                red[3][0] = max(red[3][0], red[3][k]);
            }
            atomicMin(&bbox[4 * bb + 0], red[0][0]);
            atomicMax(&bbox[4 * bb + 1], red[1][0]);
            atomicMin(&bbox[4 * bb + 2], red[2][0]);
            atomicMax(&bbox[4 * bb + 3], red[3][0]);
        }
        return;
    }
    if (!valid) return;
    atomicMin(&bbox[4 * b + 0], x0);
    atomicMax(&bbox[4 * b + 1], x1);
    atomicMin(&bbox[4 * b + 2], y0);
    atomicMax(&bbox[4 * b + 3], y1);
}

__global__ void k_bbox_init(unsigned long long* bbox, int64_t nb)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    bbox[4 * b] = ~0ull;
    bbox[4 * b + 1] = 0ull;
    bbox[4 * b + 2] = ~0ull;
    bbox[4 * b + 3] = 0ull;
}

__device__ __forceinline__ uint32_t spread16(uint32_t x)
{
    x &= 0xffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

__global__ void k_ray_keys(const int64_t* boff, int nb, const double* borig, const void* dx,
                           const void* dy, int dtype, int64_t n, const unsigned long long* bbox,
                           uint64_t* keys, uint32_t* vals)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int b = batch_of(boff, nb, i);
    double px = borig[2 * b] + ray_offset(dx, dtype, i);
    double py = borig[2 * b + 1] + ray_offset(dy, dtype, i);
    double x0 = ordered_to_dbl(bbox[4 * b]), x1 = ordered_to_dbl(bbox[4 * b + 1]);
    double y0 = ordered_to_dbl(bbox[4 * b + 2]), y1 = ordered_to_dbl(bbox[4 * b + 3]);
    double ext = fmax(x1 - x0, y1 - y0);
    double inv = ext > 0 ? 65535.99 / ext : 0.0;
    uint32_t qx = (uint32_t)fmin(fmax((px - x0) * inv, 0.0), 65535.0);
    uint32_t qy = (uint32_t)fmin(fmax((py - y0) * inv, 0.0), 65535.0);
    keys[i] = ((uint64_t)b << 32) | (uint64_t)(spread16(qx) | (spread16(qy) << 1));
    vals[i] = (uint32_t)i;
}

template <typename T, int R>
__global__ void k_groups(int64_t n_groups, const int64_t* boff, const uint32_t* gfirst, int nb,
                         const double* borig, const void* dx, const void* dy, int dtype,
                         const uint32_t* svals, v2_t<T>* gH, vec4_t<T>* gbox, uint2* grange,
                         v2_t<T>* ray_l, uint32_t* ray_idx)
{
    const unsigned full = 0xffffffffu;
    int lane = threadIdx.x & 31;
    int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= n_groups) return;
    int lo = 0, hi = nb;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if ((int64_t)gfirst[mid] <= g) lo = mid;
        else hi = mid;
    }
    const int b = lo;
    const int GR = 32 * R;
    int64_t first = boff[b] + (g - (int64_t)gfirst[b]) * GR;
    int64_t cnt64 = boff[b + 1] - first;
    int count = (int)(cnt64 < GR ? cnt64 : GR);
    double px[R], py[R];
    uint32_t idx[R];
    bool v[R];
    double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int k = r * 32 + lane;
        v[r] = k < count;
        idx[r] = 0;
        px[r] = py[r] = 0.0;
        if (v[r]) {
            idx[r] = svals[first + k];
            px[r] = borig[2 * b] + ray_offset(dx, dtype, idx[r]);
            py[r] = borig[2 * b + 1] + ray_offset(dy, dtype, idx[r]);
            xmin = fmin(xmin, px[r]); xmax = fmax(xmax, px[r]);
            ymin = fmin(ymin, py[r]); ymax = fmax(ymax, py[r]);
        }
    }
    for (int o = 16; o; o >>= 1) {
        xmin = fmin(xmin, __shfl_xor_sync(full, xmin, o));
        xmax = fmax(xmax, __shfl_xor_sync(full, xmax, o));
        ymin = fmin(ymin, __shfl_xor_sync(full, ymin, o));
        ymax = fmax(ymax, __shfl_xor_sync(full, ymax, o));
    }
    // Anchor: if every ray of the group is exactly representable in T (for
    // example FP32 rays with origin 0), H = 0 keeps each separation a single
    // rounding of (ray - particle); otherwise H is the T value nearest the
    // group centre, so that far from the coordinate zero the small offsets
    // l = ray - H keep their resolution.
    bool exact = true;
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (v[r]) exact = exact && (double)(T)px[r] == px[r] && (double)(T)py[r] == py[r];
    exact = __all_sync(full, exact);
    T Hx = exact ? T(0) : (T)(0.5 * (xmin + xmax)), Hy = exact ? T(0) : (T)(0.5 * (ymin + ymax));
    T lxmin = (T)INFINITY, lxmax = (T)-INFINITY, lymin = (T)INFINITY, lymax = (T)-INFINITY;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (!v[r]) continue;
        T lx = (T)(px[r] - (double)Hx), ly = (T)(py[r] - (double)Hy);
        lxmin = fmin(lxmin, lx); lxmax = fmax(lxmax, lx);
        lymin = fmin(lymin, ly); lymax = fmax(lymax, ly);
        v2_t<T> l;
        l.x = lx;
        l.y = ly;
        ray_l[first + r * 32 + lane] = l;
        ray_idx[first + r * 32 + lane] = idx[r];
    }
    for (int o = 16; o; o >>= 1) {
        lxmin = fmin(lxmin, __shfl_xor_sync(full, lxmin, o));
        lxmax = fmax(lxmax, __shfl_xor_sync(full, lxmax, o));
        lymin = fmin(lymin, __shfl_xor_sync(full, lymin, o));
        lymax = fmax(lymax, __shfl_xor_sync(full, lymax, o));
    }
    if (lane == 0) {
        T cx = T(0.5) * (lxmin + lxmax), cy = T(0.5) * (lymin + lymax);
        T hx = fmax(lxmax - cx, cx - lxmin), hy = fmax(lymax - cy, cy - lymin);
        // inflate so that every ray is inside after rounding
        hx = hx * T(1.0 + 1e-5) + T(1e-30);
        hy = hy * T(1.0 + 1e-5) + T(1e-30);
        v2_t<T> H;
        H.x = Hx;
        H.y = Hy;
        gH[g] = H;
        vec4_t<T> bx;
        bx.x = cx; bx.y = cy; bx.z = hx; bx.w = hy;
        gbox[g] = bx;
        grange[g] = make_uint2((uint32_t)first, (uint32_t)count);
    }
}

// One batch of FP32 offsets (the common case) needs no FP64 on the grouping
// path (FP64 runs at 1/64 of the FP32 rate here): the offsets' bounding box
// from order-preserving uint32 images of the floats, 32-bit Morton keys of
// the offsets (relative positions do not depend on the origin), and, when
// the origin is zero, groups anchored at H = 0 with l = the offsets
// themselves -- what the FP64 path computes in that case.
__device__ __forceinline__ uint32_t flt_to_ordered(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_flt(uint32_t u)
{
    u = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    return __uint_as_float(u);
}

// bb = {min x, min y, max x, max y} as ordered images; the caller sets the
// minima to 0xffffffff and the maxima to 0 first.
__global__ void __launch_bounds__(256) k_ray_bbox32(const float* dx, const float* dy, int64_t n, uint32_t* bb)
{
    __shared__ uint32_t red[4][8];
    const unsigned full = 0xffffffffu;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t v[4] = {~0u, ~0u, 0u, 0u};
    if (i < n) {
        v[0] = v[2] = flt_to_ordered(dx[i]);
        v[1] = v[3] = flt_to_ordered(dy[i]);
    }
    for (int o = 16; o; o >>= 1) {
        v[0] = min(v[0], __shfl_xor_sync(full, v[0], o));
        v[1] = min(v[1], __shfl_xor_sync(full, v[1], o));
        v[2] = max(v[2], __shfl_xor_sync(full, v[2], o));
        v[3] = max(v[3], __shfl_xor_sync(full, v[3], o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 4; ++q) red[q][w] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            v[0] = min(v[0], red[0][k]);
            v[1] = min(v[1], red[1][k]);
            v[2] = max(v[2], red[2][k]);
            v[3] = max(v[3], red[3][k]);
        }
        atomicMin(&bb[0], v[0]);
        atomicMin(&bb[1], v[1]);
        atomicMax(&bb[2], v[2]);
        atomicMax(&bb[3], v[3]);
    }
}

__global__ void k_ray_keys32(const float* dx, const float* dy, int64_t n, const uint32_t* bb, uint32_t* keys,
                             uint32_t* vals)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x0 = ordered_to_flt(bb[0]), y0 = ordered_to_flt(bb[1]);
    const float ext = fmaxf(ordered_to_flt(bb[2]) - x0, ordered_to_flt(bb[3]) - y0);
    const float inv = ext > 0.f ? 65535.99f / ext : 0.f;
    const uint32_t qx = (uint32_t)fminf(fmaxf((dx[i] - x0) * inv, 0.f), 65535.f);
    const uint32_t qy = (uint32_t)fminf(fmaxf((dy[i] - y0) * inv, 0.f), 65535.f);
    keys[i] = spread16(qx) | (spread16(qy) << 1);
    vals[i] = (uint32_t)i;
}

// Groups of one batch of FP32 offsets at origin zero: every ray is exact in
// T, so H = 0 and l = the offset (as k_groups then has it).
template <typename T, int R>
__global__ void k_groups32(int64_t n_groups, int64_t n, const float* dx, const float* dy, const uint32_t* svals,
                           v2_t<T>* gH, vec4_t<T>* gbox, uint2* grange, v2_t<T>* ray_l, uint32_t* ray_idx)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= n_groups) return;
    const int64_t first = g * (32 * R);
    const int count = (int)(n - first < 32 * R ? n - first : 32 * R);
    T lxmin = (T)INFINITY, lxmax = (T)-INFINITY, lymin = (T)INFINITY, lymax = (T)-INFINITY;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int k = r * 32 + lane;
        if (k >= count) continue;
        const uint32_t idx = svals[first + k];
        v2_t<T> l;
        l.x = (T)dx[idx];
        l.y = (T)dy[idx];
        lxmin = fmin(lxmin, l.x); lxmax = fmax(lxmax, l.x);
        lymin = fmin(lymin, l.y); lymax = fmax(lymax, l.y);
        ray_l[first + k] = l;
        ray_idx[first + k] = idx;
    }
    for (int o = 16; o; o >>= 1) {
        lxmin = fmin(lxmin, __shfl_xor_sync(full, lxmin, o));
        lxmax = fmax(lxmax, __shfl_xor_sync(full, lxmax, o));
        lymin = fmin(lymin, __shfl_xor_sync(full, lymin, o));
        lymax = fmax(lymax, __shfl_xor_sync(full, lymax, o));
    }
    if (lane == 0) {
        T cx = T(0.5) * (lxmin + lxmax), cy = T(0.5) * (lymin + lymax);
        T hx = fmax(lxmax - cx, cx - lxmin), hy = fmax(lymax - cy, cy - lymin);
        hx = hx * T(1.0 + 1e-5) + T(1e-30);
        hy = hy * T(1.0 + 1e-5) + T(1e-30);
        v2_t<T> H;
        H.x = T(0);
        H.y = T(0);
        gH[g] = H;
        vec4_t<T> bx;
        bx.x = cx; bx.y = cy; bx.z = hx; bx.w = hy;
        gbox[g] = bx;
        grange[g] = make_uint2((uint32_t)first, (uint32_t)count);
    }
}

// ---------------------------------------------------------------- walk

template <int KIND, typename T, int R, bool AO, bool DIRECT, int TILE>
__global__ void __launch_bounds__(kWalkWarps * 32, sizeof(T) == 4 ? (R == 4 ? 4 : (R == 2 ? 5 : 6)) : 2)
walk_kernel(WalkParams<T> P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned full = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    using WS = WalkShared<KIND, T, TILE, tot_rays<R>()>;
    WS& S = reinterpret_cast<WS*>(smem_raw)[warp];
    int* stack = P.stack + ((int64_t)blockIdx.x * kWalkWarps + warp) * kStackCap;
    WalkCtx<KIND, T, R, AO, TILE> C(P, S);
    uint32_t ridx[R];
    bool rv[R];

    const int NS = DIRECT && P.n_slices > 1 ? P.n_slices : 1;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(P.counter, 1u);
        item = __shfl_sync(full, item, 0);
        if ((int64_t)item >= P.n_groups * NS) break;
        const uint32_t slice = item % (uint32_t)NS;
        const uint32_t g = P.order ? P.order[item / (uint32_t)NS] : item / (uint32_t)NS;
        C.H = P.gH[g];
        C.box = P.gbox[g];
        uint2 rg = P.grange[g];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int k = r * 32 + lane;
            rv[r] = k < (int)rg.y;
            if (rv[r]) {
                v2_t<T> l = P.ray_l[rg.x + k];
                C.lx[r] = l.x;
                C.ly[r] = l.y;
                ridx[r] = P.ray_idx[rg.x + k];
            } else {
                C.lx[r] = C.box.x;
                C.ly[r] = C.box.y;
                ridx[r] = 0;
            }
            C.part[r].zero();
        }
        C.tot_zero();

        int c_vis = 0, c_acc = 0, c_near = 0, c_bigs = 0, c_bigk = 0, c_dummy = 0;
        C.nf = C.nn = C.nb = 0;
        if (KIND >= 0 && P.n_part > 0) {
            if (DIRECT) {
                // every particle of this item's slice with its full profile
                const int64_t p0 = P.n_part * slice / NS, p1 = P.n_part * (slice + 1) / NS;
                for (int64_t base = p0; base < p1; base += 0x40000000) {
                    int64_t rem = p1 - base;
                    int c = (int)(rem < 0x40000000 ? rem : 0x40000000);
                    append_ranges(C, lane == 0 ? c : 0, (int)base, P.leaf0, P.leaf1, c_near, c_dummy);
                }
                C.flush_near();
            } else {
                C.rec = P.list_ids ? P.list_ids + (int64_t)g * P.list_K : nullptr;
                C.rec_n = 0;
                C.rec_cap = P.list_K;
                const bool whole = traverse(C, stack, c_vis, c_acc, c_near, c_bigs, c_bigk);
                if (C.rec && lane == 0)
                    P.list_n[g] = whole && C.rec_n <= C.rec_cap ? (uint32_t)C.rec_n : kListOverflow;
                C.flush_far();
                C.flush_near();
                if constexpr (KIND != LENS_POINT) C.flush_big();
            }
        }
        if (P.n_halos > 0 && slice == 0) C.halos();
        if (P.gcost && lane == 0) P.gcost[g] += (uint32_t)(c_vis + c_acc + c_near + c_bigk);
        if (P.stats && lane == 0) {
            unsigned long long nr = rg.y;
            if (slice == 0) atomicAdd(&P.stats[0], 1ull);
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
            uint32_t i = ridx[r];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                if (AO && q >= 2) break;
                T val = C.tot_get(r, q);
                if (NS > 1) {
                    P.split[((int64_t)slice * 5 + q) * P.split_n + i] = val;
                    continue;
                }
                if (P.accumulate) val += P.out[q][i];
                P.out[q][i] = val;
            }
        }
        __syncwarp();
    }
}

// The slices of a split direct sum, added per ray in slice order with
// Neumaier compensation (deterministic), into the outputs.
template <typename T>
__global__ void k_split_sum(int64_t n, int S, int nq, const T* split, T* o0, T* o1, T* o2, T* o3, T* o4,
                            int accumulate)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T* out[5] = {o0, o1, o2, o3, o4};
    for (int q = 0; q < nq; ++q) {
        T s = T(0), c = T(0);
        for (int k = 0; k < S; ++k) Comp5<T>::add1(s, c, split[((int64_t)k * 5 + q) * n + i]);
        T v = s + c;
        if (accumulate) v += out[q][i];
        out[q][i] = v;
    }
}

// Particle slices for a direct sum of ng ray groups over n_part particles:
// enough work items (group x slice) for about 16 warps per SM when the rays
// alone give fewer, each slice at least 128 particles, the partial sums
// within the scratch of the split region.
static int split_slices(const lens_tree* t, int64_t ng, int64_t n_rays, int64_t n_part)
{
    const int64_t target = (int64_t)t->num_sms * 16;
    if (ng <= 0 || ng >= target) return 1;
    int64_t S = (target + ng - 1) / ng;
    S = std::min<int64_t>(S, std::max<int64_t>(1, n_part / 128));
    S = std::min<int64_t>(S, 64);
    S = std::min<int64_t>(S, (int64_t)split_values(max_slots(const_cast<lens_tree*>(t))) / std::max<int64_t>(1, n_rays));
    return S < 2 ? 1 : (int)S;
}

// ------------------------------------------------------------- host side

template <int KIND, typename T, int R, bool AO, bool DIRECT, int TILE>
static int walk_blocks_per_sm()
{
    static int cached = -1;
    if (cached < 0) {
        size_t smem = kWalkWarps * sizeof(WalkShared<KIND, T, TILE, tot_rays<R>()>);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(walk_kernel<KIND, T, R, AO, DIRECT, TILE>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        // the walk keeps its working set in shared memory and registers:
        // prefer the largest shared-memory carveout
        cudaFuncSetAttribute(walk_kernel<KIND, T, R, AO, DIRECT, TILE>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, walk_kernel<KIND, T, R, AO, DIRECT, TILE>,
                                                      kWalkWarps * 32, smem);
        cached = nb > 0 ? nb : 1;
    }
    return cached;
}

void free_graphs(lens_tree* t);

lens_status reserve_rays(lens_tree* t, int64_t n, int64_t nb, cudaStream_t s)
{
    if (n <= t->ray_cap && nb <= t->batch_cap && t->ray_scratch.ptr) return LENS_OK;
    int64_t nn = std::max(n, t->ray_cap), bb = std::max(nb, t->batch_cap);
    Layout L = make_layout(nn, bb, max_slots(t));
    free_graphs(t);  // captured graphs point into the old scratch
    t->cost_n = -1;  // so does the work record
    t->grp_n = -1;   // and the groups
    if (t->ray_scratch.ptr) cudaFreeAsync(t->ray_scratch.ptr, s);
    t->ray_scratch.ptr = nullptr;
    t->ray_cap = t->batch_cap = 0;
    cudaError_t e = lens_malloc_async(&t->ray_scratch.ptr, L.total, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return lens_set_error(LENS_ERR_OOM, "cannot allocate %zu bytes of ray scratch", L.total);
    }
    t->ray_scratch.bytes = L.total;
    t->ray_cap = nn;
    t->batch_cap = bb;
    return LENS_OK;
}

template <int KIND, typename T, int R, bool AO, bool DIRECT, int TILE>
static void launch_one(const WalkParams<T>& P, int num_sms, cudaStream_t s)
{
    size_t smem = kWalkWarps * sizeof(WalkShared<KIND, T, TILE, tot_rays<R>()>);
    int bps = walk_blocks_per_sm<KIND, T, R, AO, DIRECT, TILE>();
    if (bps > 16) bps = 16;  // stack slots are allocated for 16 blocks per SM
    int grid = num_sms * bps;
    { walk_kernel<KIND, T, R, AO, DIRECT, TILE><<<grid, kWalkWarps * 32, smem, s>>>(P); note_launch(); }
}

template <typename T, int R, bool AO, bool DIRECT, int TILE>
static void launch_kind(int kind, const WalkParams<T>& P, int num_sms, cudaStream_t s)
{
    if (kind == LENS_POINT) launch_one<LENS_POINT, T, R, AO, DIRECT, TILE>(P, num_sms, s);
    else if (kind == LENS_GAUSS) launch_one<LENS_GAUSS, T, R, AO, DIRECT, TILE>(P, num_sms, s);
    else launch_one<LENS_NFW, T, R, AO, DIRECT, TILE>(P, num_sms, s);
}

// tile: the near-field tile size of the tree walk (WalkBuf); the larger tile
// is built for FP32 tree walks only (the direct sum and the FP64 tree keep
// the standard one).
template <typename T, int R>
static void launch_dispatch(int kind, bool ao, bool direct, const WalkParams<T>& P, int num_sms,
                            cudaStream_t s, int tile = 0)
{
    if (direct) {
        if (ao) launch_kind<T, R, true, true, 0>(kind, P, num_sms, s);
        else launch_kind<T, R, false, true, 0>(kind, P, num_sms, s);
    } else {
        if constexpr (sizeof(T) == 4) {
            if (tile == 1) {
                if (ao) launch_kind<T, R, true, false, 1>(kind, P, num_sms, s);
                else launch_kind<T, R, false, false, 1>(kind, P, num_sms, s);
                return;
            }
        }
        if (ao) launch_kind<T, R, true, false, 0>(kind, P, num_sms, s);
        else launch_kind<T, R, false, false, 0>(kind, P, num_sms, s);
    }
}

// 128-ray groups (four rays per lane): the one-warp tree walk of an FP32 tree.
template <typename T>
static void launch_tree4(int kind, bool ao, const WalkParams<T>& P, int num_sms, cudaStream_t s, int tile)
{
    if constexpr (sizeof(T) == 4) {
        if (tile == 1) {
            if (ao) launch_kind<T, 4, true, false, 1>(kind, P, num_sms, s);
            else launch_kind<T, 4, false, false, 1>(kind, P, num_sms, s);
        } else {
            if (ao) launch_kind<T, 4, true, false, 0>(kind, P, num_sms, s);
            else launch_kind<T, 4, false, false, 0>(kind, P, num_sms, s);
        }
    }
}

static int rays_per_lane(const lens_tree* t, int max_r)
{
    const int r = (t->precision == LENS_PREC_FP64 || t->group_rays <= 32) ? 1 : t->group_rays >= 128 ? 4 : 2;
    return r < max_r ? r : max_r;
}

// 128-ray groups only for the one-warp tree walk of an FP32 tree.
int shoot_max_r(const lens_tree* t, int flags)
{
    const bool ws = t->walk_mode == LENS_WALK_PAIRS || t->walk_mode == LENS_WALK_TRIOS;
    return (flags & LENS_DIRECT) || ws || t->precision != LENS_PREC_FP32 ? 2 : 4;
}

// Copy the batch table to the device (stream ordered) and size the groups.
lens_status upload_batches(lens_tree* t, int64_t nb, const int64_t* h_off, const double* h_orig,
                           cudaStream_t s, ShootPlan* plan, int max_r)
{
    const int64_t n = h_off[nb];
    const int R = rays_per_lane(t, max_r);
    const int GR = 32 * R;
    LENS_TRY(reserve_rays(t, n, nb, s));
    Layout L = make_layout(t->ray_cap, t->batch_cap, max_slots(t));
    char* base = (char*)t->ray_scratch.ptr;
    // pageable host copies: the CUDA driver stages them before returning
    std::vector<uint32_t> gf(nb + 1);
    uint64_t ng = 0;
    for (int64_t b = 0; b < nb; ++b) {
        gf[b] = (uint32_t)ng;
        ng += (uint64_t)((h_off[b + 1] - h_off[b] + GR - 1) / GR);
    }
    gf[nb] = (uint32_t)ng;
    LENS_CUDA(cudaMemcpyAsync(base + L.boff, h_off, (nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    LENS_CUDA(cudaMemcpyAsync(base + L.borig, h_orig, nb * 2 * sizeof(double), cudaMemcpyHostToDevice, s));
    LENS_CUDA(cudaMemcpyAsync(base + L.gfirst, gf.data(), (nb + 1) * sizeof(uint32_t),
                              cudaMemcpyHostToDevice, s));
    plan->n = n;
    plan->nb = nb;
    plan->ng = ng;
    plan->R = R;
    plan->ox = nb == 1 ? h_orig[0] : 0.0;
    plan->oy = nb == 1 ? h_orig[1] : 0.0;
    return LENS_OK;
}

template <typename T>
lens_status enqueue_groups(lens_tree* t, const ShootPlan& plan, const void* dx, const void* dy, int dtype,
                           cudaStream_t s)
{
    t->grp_n = -1;  // (set again below once these rays are grouped)
    using T4 = vec4_t<T>;
    using T2 = v2_t<T>;
    const int64_t n = plan.n, nb = plan.nb;
    const uint64_t ng = plan.ng;
    const int R = plan.R;
    Layout L = make_layout(t->ray_cap, t->batch_cap, max_slots(t));
    char* base = (char*)t->ray_scratch.ptr;
    int64_t* d_boff = (int64_t*)(base + L.boff);
    double* d_borig = (double*)(base + L.borig);
    uint32_t* d_gfirst = (uint32_t*)(base + L.gfirst);
    unsigned long long* d_bbox = (unsigned long long*)(base + L.bbox);
    T2* ray_l = (T2*)(base + L.rl);
    uint32_t* ray_idx = (uint32_t*)(base + L.ridx);
    T2* gH = (T2*)(base + L.gH);
    T4* gbox = (T4*)(base + L.gbox);
    uint2* grange = (uint2*)(base + L.grange);
    if (nb == 1 && dtype == LENS_F32) {
        const int TB = 256;
        const float* fx = (const float*)dx;
        const float* fy = (const float*)dy;
        uint32_t* bb = (uint32_t*)d_bbox;
        uint32_t* k0 = (uint32_t*)(base + L.k0);
        uint32_t* k1 = (uint32_t*)(base + L.k1);
        uint32_t* v0 = (uint32_t*)(base + L.v0);
        uint32_t* v1 = (uint32_t*)(base + L.v1);
        LENS_CUDA(cudaMemsetAsync(bb, 0xff, 2 * sizeof(uint32_t), s));
        LENS_CUDA(cudaMemsetAsync(bb + 2, 0, 2 * sizeof(uint32_t), s));
        { k_ray_bbox32<<<grid_for(n, TB), TB, 0, s>>>(fx, fy, n, bb); note_launch(); }
        { k_ray_keys32<<<grid_for(n, TB), TB, 0, s>>>(fx, fy, n, bb, k0, v0); note_launch(); }
        uint32_t *sk, *sv;
        radix_sort_pairs<uint32_t>(k0, v0, k1, v1, n, 0, 32, base + L.tmp, s, &sk, &sv, t->d_err);
        unsigned gg = grid_for((int64_t)ng * 32, TB);
        if (plan.ox == 0.0 && plan.oy == 0.0) {
            if (R == 1)
                { k_groups32<T, 1><<<gg, TB, 0, s>>>((int64_t)ng, n, fx, fy, sv, gH, gbox, grange, ray_l, ray_idx);
                  note_launch(); }
            else if (R == 2)
                { k_groups32<T, 2><<<gg, TB, 0, s>>>((int64_t)ng, n, fx, fy, sv, gH, gbox, grange, ray_l, ray_idx);
                  note_launch(); }
            else
                { k_groups32<T, 4><<<gg, TB, 0, s>>>((int64_t)ng, n, fx, fy, sv, gH, gbox, grange, ray_l, ray_idx);
                  note_launch(); }
        } else if (R == 1) {
            { k_groups<T, 1><<<gg, TB, 0, s>>>((int64_t)ng, d_boff, d_gfirst, (int)nb, d_borig, dx, dy, dtype,
                                             sv, gH, gbox, grange, ray_l, ray_idx); note_launch(); }
        } else if (R == 2) {
            { k_groups<T, 2><<<gg, TB, 0, s>>>((int64_t)ng, d_boff, d_gfirst, (int)nb, d_borig, dx, dy, dtype,
                                             sv, gH, gbox, grange, ray_l, ray_idx); note_launch(); }
        } else {
            { k_groups<T, 4><<<gg, TB, 0, s>>>((int64_t)ng, d_boff, d_gfirst, (int)nb, d_borig, dx, dy, dtype,
                                             sv, gH, gbox, grange, ray_l, ray_idx); note_launch(); }
        }
    } else {
        const int TB = 256;
        { k_bbox_init<<<grid_for(nb, 128), 128, 0, s>>>(d_bbox, nb); note_launch(); }
        { k_ray_bbox<<<grid_for(n, TB), TB, 0, s>>>(d_boff, (int)nb, d_borig, dx, dy, dtype, n, d_bbox); note_launch(); }
        uint64_t* k0 = (uint64_t*)(base + L.k0);
        uint64_t* k1 = (uint64_t*)(base + L.k1);
        uint32_t* v0 = (uint32_t*)(base + L.v0);
        uint32_t* v1 = (uint32_t*)(base + L.v1);
        { k_ray_keys<<<grid_for(n, TB), TB, 0, s>>>(d_boff, (int)nb, d_borig, dx, dy, dtype, n, d_bbox, k0, v0); note_launch(); }
        int bbits = 0;
        while ((1ll << bbits) < nb) ++bbits;
        int end_bit = (32 + bbits + 7) & ~7;
        uint64_t* sk;
        uint32_t* sv;
        radix_sort_pairs<uint64_t>(k0, v0, k1, v1, n, 0, end_bit, base + L.tmp, s, &sk, &sv, t->d_err);
        unsigned gg = grid_for((int64_t)ng * 32, TB);
        if (R == 1)
            { k_groups<T, 1><<<gg, TB, 0, s>>>((int64_t)ng, d_boff, d_gfirst, (int)nb, d_borig, dx, dy, dtype,
                                             sv, gH, gbox, grange, ray_l, ray_idx); note_launch(); }
        else if (R == 2)
            { k_groups<T, 2><<<gg, TB, 0, s>>>((int64_t)ng, d_boff, d_gfirst, (int)nb, d_borig, dx, dy, dtype,
                                             sv, gH, gbox, grange, ray_l, ray_idx); note_launch(); }
        else
            { k_groups<T, 4><<<gg, TB, 0, s>>>((int64_t)ng, d_boff, d_gfirst, (int)nb, d_borig, dx, dy, dtype,
                                             sv, gH, gbox, grange, ray_l, ray_idx); note_launch(); }
    }

    if (nb == 1) {
        t->grp_dx = dx;
        t->grp_dy = dy;
        t->grp_n = n;
        t->grp_dtype = dtype;
        t->grp_R = R;
        t->grp_ox = plan.ox;
        t->grp_oy = plan.oy;
    }
    return LENS_OK;
}
template lens_status enqueue_groups<float>(lens_tree*, const ShootPlan&, const void*, const void*, int, cudaStream_t);
template lens_status enqueue_groups<double>(lens_tree*, const ShootPlan&, const void*, const void*, int, cudaStream_t);

void set_cost_key(lens_tree* t, const RayKey& k);

// Enqueue the kernels of one shoot call (no allocation, no host sync: safe
// to capture into a CUDA graph).
template <typename T>
static lens_status enqueue_typed(lens_tree* t, const ShootPlan& plan, const void* dx, const void* dy,
                                 int dtype, void* const out[5], int flags, cudaStream_t s)
{
    using T4 = vec4_t<T>;
    using T2 = v2_t<T>;
    const int64_t n = plan.n, nb = plan.nb;
    const uint64_t ng = plan.ng;
    const int R = plan.R;
    Layout L = make_layout(t->ray_cap, t->batch_cap, max_slots(t));
    char* base = (char*)t->ray_scratch.ptr;
    int64_t* d_boff = (int64_t*)(base + L.boff);
    double* d_borig = (double*)(base + L.borig);
    uint32_t* d_gfirst = (uint32_t*)(base + L.gfirst);
    unsigned long long* d_bbox = (unsigned long long*)(base + L.bbox);
    T2* ray_l = (T2*)(base + L.rl);
    uint32_t* ray_idx = (uint32_t*)(base + L.ridx);
    T2* gH = (T2*)(base + L.gH);
    T4* gbox = (T4*)(base + L.gbox);
    uint2* grange = (uint2*)(base + L.grange);
    uint32_t* counter = (uint32_t*)(base + L.counter);
    int* stack = (int*)(base + L.stack);
    const bool timing = (flags & LENS_TIMING) != 0;
    if (timing) {
        for (int i = 0; i < 4; ++i)
            if (!t->ev[i]) LENS_CUDA(cudaEventCreate(&t->ev[i]));
        LENS_CUDA(cudaEventRecord(t->ev[0], s));
    }
    if (n > 0) LENS_TRY(enqueue_groups<T>(t, plan, dx, dy, dtype, s));
    // a tree walk of one batch records its groups' work, and takes them
    // heaviest first when these rays were walked before on this tree
    RayKey key;
    key.dx = dx; key.dy = dy; key.n = n; key.dtype = dtype; key.R = R; key.ox = plan.ox; key.oy = plan.oy;
    const bool record = n > 0 && nb == 1 && !(flags & LENS_DIRECT);
    const uint32_t* order = record ? heavy_first_order<T>(t, plan, key, 0, s).order : nullptr;
    uint32_t* gcost = record ? (uint32_t*)(base + L.gcost) : nullptr;
    if (gcost) LENS_CUDA(cudaMemsetAsync(gcost, 0, ng * sizeof(uint32_t), s));
    // interaction lists for the adjoint (room made by the caller, shoot())
    const bool keep = record && (flags & LENS_KEEP_LISTS) && t->list_ids && t->list_groups >= (int64_t)ng;
    if (keep) LENS_CUDA(cudaMemsetAsync(t->list_n, 0xff, ng * sizeof(uint32_t), s));  // kListOverflow

    if (timing) LENS_CUDA(cudaEventRecord(t->ev[1], s));
    // the grouping above reads only the rays: it may overlap the end of a
    // build on another stream; the walk reads the tree
    LENS_TRY(wait_built(t, s));
    if (timing) LENS_CUDA(cudaEventRecord(t->ev[2], s));
    WalkParams<T> P{};
    P.stats = (flags & LENS_COUNT) ? t->d_stats : nullptr;
    P.gH = gH; P.gbox = gbox; P.grange = grange; P.ray_l = ray_l; P.ray_idx = ray_idx;
    P.n_groups = (int64_t)ng;
    P.stack = stack;
    P.err = t->d_err;
    P.wait_cycles = t->wait_cycles;
    P.order = order;
    P.gcost = gcost;
    P.list_ids = keep ? t->list_ids : nullptr;
    P.list_n = keep ? t->list_n : nullptr;
    P.list_K = keep ? t->list_K : 0;
    for (int q = 0; q < 5; ++q) P.out[q] = (T*)out[q];
    const bool ao = (flags & LENS_ALPHA_ONLY) != 0;
    const bool direct = (flags & LENS_DIRECT) != 0;
    bool first_launch = true;
    int launches = 0;
    for (size_t si = 0; si < t->sp.size(); ++si) {
        const SpeciesTree& st = t->sp[si];
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
        P.n_halos = first_launch ? (int)t->n_halos : 0;
        P.accumulate = first_launch ? ((flags & LENS_ACCUMULATE) ? 1 : 0) : 1;
        P.counter = counter + 2 * launches;
        LENS_CUDA(cudaMemsetAsync(P.counter, 0, sizeof(uint32_t), s));
        // few ray groups in a direct sum: split the particles over slices too
        P.n_slices = direct ? split_slices(t, (int64_t)ng, n, st.n) : 1;
        P.split_n = n;
        P.split = (T*)(base + L.split);
        if (n > 0) {
            bool done = false;
            if (!direct && (t->walk_mode == LENS_WALK_PAIRS || t->walk_mode == LENS_WALK_TRIOS)) {
                const int consumers = t->walk_mode == LENS_WALK_TRIOS ? 2 : 1;
                if (R <= 2)
                    done = R == 1 ? launch_ws<T, 1>(st.kind, ao, P, t->num_sms, s, consumers)
                                  : launch_ws<T, 2>(st.kind, ao, P, t->num_sms, s, consumers);
            }
            if (!done) {
                if (R == 1) launch_dispatch<T, 1>(st.kind, ao, direct, P, t->num_sms, s, t->tile);
                else if (R == 2) launch_dispatch<T, 2>(st.kind, ao, direct, P, t->num_sms, s, t->tile);
                else if (!direct) launch_tree4<T>(st.kind, ao, P, t->num_sms, s, t->tile);
                else return lens_set_error(LENS_ERR_INTERNAL, "128-ray groups in a direct sum");
            }
            if (P.n_slices > 1) {
                k_split_sum<T><<<grid_for(n, 256), 256, 0, s>>>(n, P.n_slices, ao ? 2 : 5, P.split, P.out[0], P.out[1],
                                                              P.out[2], P.out[3], P.out[4], P.accumulate);
                note_launch();
            }
        }
        first_launch = false;
        ++launches;
    }
    if (first_launch && n > 0) {
        // no particles at all: analytic components only
        P.n_part = 0;
        P.halos = t->halos;
        P.n_halos = (int)t->n_halos;
        P.accumulate = (flags & LENS_ACCUMULATE) ? 1 : 0;
        P.counter = counter;
        LENS_CUDA(cudaMemsetAsync(P.counter, 0, sizeof(uint32_t), s));
        if (R == 1) launch_dispatch<T, 1>(LENS_POINT, ao, true, P, t->num_sms, s);
        else if (R == 2) launch_dispatch<T, 2>(LENS_POINT, ao, true, P, t->num_sms, s);
        else return lens_set_error(LENS_ERR_INTERNAL, "128-ray groups without particles");
    }
    if (timing) {
        LENS_CUDA(cudaEventRecord(t->ev[3], s));
        t->timed = true;
    }
    if (record) set_cost_key(t, key);
    if (keep) {
        t->list_dx = key.dx;
        t->list_dy = key.dy;
        t->list_rays = key.n;
        t->list_dtype = key.dtype;
        t->list_R = key.R;
        t->list_ox = key.ox;
        t->list_oy = key.oy;
    }
    LENS_CUDA(cudaGetLastError());
    return LENS_OK;
}

lens_status enqueue_shoot(lens_tree* t, const ShootPlan& plan, const void* dx, const void* dy, int dtype,
                          void* const out[5], int flags, cudaStream_t s)
{
    if (t->precision == LENS_PREC_FP64) return enqueue_typed<double>(t, plan, dx, dy, dtype, out, flags, s);
    return enqueue_typed<float>(t, plan, dx, dy, dtype, out, flags, s);
}

// Room for the interaction lists of ng groups of R * 32 rays (512 entries
// per 32 rays).  The old lists are dropped.
static lens_status reserve_lists(lens_tree* t, int64_t ng, int R, cudaStream_t s)
{
    const int K = 512 * R;
    t->list_rays = -1;  // whatever is kept belongs to no rays until the walk records
    if (t->list_ids && t->list_groups >= ng && t->list_K == K) return LENS_OK;
    if (t->list_ids || t->list_n) {
        LENS_CUDA(cudaStreamSynchronize(s));  // the old lists may still be read
        if (t->list_ids) cudaFreeAsync(t->list_ids, s);
        if (t->list_n) cudaFreeAsync(t->list_n, s);
    }
    t->list_ids = t->list_n = nullptr;
    t->list_groups = 0;
    // from the stream-ordered pool: a new tree's first kept lists cost no
    // device allocation call
    LENS_CUDA(lens_malloc_async((void**)&t->list_ids, (size_t)ng * K * sizeof(uint32_t), s));
    cudaError_t e = lens_malloc_async((void**)&t->list_n, (size_t)ng * sizeof(uint32_t), s);
    if (e != cudaSuccess) {
        cudaFreeAsync(t->list_ids, s);
        t->list_ids = nullptr;
        return lens_cuda_check(e, "cudaMallocAsync(lists)");
    }
    t->list_groups = ng;
    t->list_K = K;
    return LENS_OK;
}

lens_status shoot(lens_tree* t, int64_t nb, const int64_t* h_off, const double* h_orig, const void* dx,
                  const void* dy, int dtype, void* const out[5], int flags, cudaStream_t s)
{
    ShootPlan plan;
    LENS_TRY(upload_batches(t, nb, h_off, h_orig, s, &plan, shoot_max_r(t, flags)));
    // kept lists hold box indices in 29 bits
    bool small_tree = true;
    for (const auto& st : t->sp) small_tree = small_tree && st.n_nodes < (int64_t)kListIdMask;
    // (the adjoint groups at most 64 rays: lists of 128-ray groups would not be its)
    if ((flags & LENS_KEEP_LISTS) && !(flags & LENS_DIRECT) && nb == 1 && plan.n > 0 && small_tree && plan.R <= 2)
        LENS_TRY(reserve_lists(t, (int64_t)plan.ng, plan.R, s));
    else
        flags &= ~LENS_KEEP_LISTS;
    return enqueue_shoot(t, plan, dx, dy, dtype, out, flags, s);
}

bool groups_hold(const lens_tree* t, const RayKey& k)
{
    return t->grp_n >= 0 && t->grp_dx == k.dx && t->grp_dy == k.dy && t->grp_n == k.n &&
           t->grp_dtype == k.dtype && t->grp_R == k.R && t->grp_ox == k.ox && t->grp_oy == k.oy;
}

// The kept interaction lists if they belong to these rays, else null.
const uint32_t* kept_lists(const lens_tree* t, const RayKey& k)
{
    if (!t->list_ids || t->list_rays < 0) return nullptr;
    const bool same = t->list_dx == k.dx && t->list_dy == k.dy && t->list_rays == k.n && t->list_dtype == k.dtype &&
                      t->list_R == k.R && t->list_ox == k.ox && t->list_oy == k.oy;
    return same ? t->list_ids : nullptr;
}

// Scratch views shared with the backward walk.
void* scratch_base(lens_tree* t) { return t->ray_scratch.ptr; }

__global__ void k_cost_keys(uint32_t ng, const uint32_t* gcost, uint32_t* keys, uint32_t* vals,
                            unsigned long long* total)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t c = g < ng ? gcost[g] : 0u;
    if (g < ng) {
        keys[g] = ~c;  // ascending sort of the complement: heaviest first, ties in group order
        vals[g] = g;
    }
    unsigned long long w = c;
    for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(total, w);
}

// Slices of the heaviest groups (one block of kHeavyGroups threads; thread
// i owns the group at position i of the order).  The slice counts are
// non-increasing along the order, so the split groups are its first Kc.
__global__ void __launch_bounds__(kHeavyGroups) k_heavy_plan(uint32_t ng, const uint32_t* sorted_keys,
                                                             unsigned long long n_warps, uint32_t* hdr,
                                                             uint32_t* table)
{
    __shared__ uint32_t wsum[kHeavyGroups / 32];
    const uint32_t i = threadIdx.x, lane = i & 31, warp = i >> 5;
    const unsigned long long total = *(const unsigned long long*)(hdr + 8);
    unsigned long long cap = total / (4ull * n_warps);  // a quarter of one warp's share
    if (cap < 1) cap = 1;
    uint32_t v = 0;  // slices of a split group, 0 for a whole one
    if (i < ng) {
        unsigned long long q = ((unsigned long long)(~sorted_keys[i]) + cap - 1) / cap;
        if (q > 1) v = q > 32 ? 32u : (uint32_t)q;
    }
    uint32_t x = v;  // inclusive scan over the block
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    const int kc = __syncthreads_count(v > 0);
    if (warp == 0) {
        uint32_t w = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= (uint32_t)o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    const uint32_t first = x - v + (warp ? wsum[warp - 1] : 0u);
    for (uint32_t k = 0; k < v; ++k) table[first + k] = (i << 10) | (k << 5) | (v - 1);
    if (i == 0) {
        hdr[0] = (uint32_t)kc;
        hdr[1] = wsum[kHeavyGroups / 32 - 1];
    }
}

static bool cost_key_matches(const lens_tree* t, const RayKey& k)
{
    return t->cost_dx == k.dx && t->cost_dy == k.dy && t->cost_n == k.n && t->cost_dtype == k.dtype &&
           t->cost_R == k.R && t->cost_ox == k.ox && t->cost_oy == k.oy;
}

void set_cost_key(lens_tree* t, const RayKey& k)
{
    t->cost_dx = k.dx;
    t->cost_dy = k.dy;
    t->cost_n = k.n;
    t->cost_dtype = k.dtype;
    t->cost_R = k.R;
    t->cost_ox = k.ox;
    t->cost_oy = k.oy;
}

template <typename T>
HeavyPlan heavy_first_order(lens_tree* t, const ShootPlan& plan, const RayKey& key, int64_t n_warps,
                            cudaStream_t s)
{
    HeavyPlan hp;
    if (plan.nb != 1 || plan.ng < 2 || !cost_key_matches(t, key)) return hp;
    Layout L = make_layout(t->ray_cap, t->batch_cap, max_slots(t));
    char* base = (char*)t->ray_scratch.ptr;
    uint32_t* k0 = (uint32_t*)(base + L.k0);
    uint32_t* k1 = (uint32_t*)(base + L.k1);
    uint32_t* v0 = (uint32_t*)(base + L.v0);
    uint32_t* v1 = (uint32_t*)(base + L.v1);
    uint32_t* hdr = (uint32_t*)(base + L.heavy);
    uint32_t* table = hdr + 16;
    const uint32_t ng = (uint32_t)plan.ng;
    if (cudaMemsetAsync(hdr, 0, 64, s) != cudaSuccess) return hp;
    {
        k_cost_keys<<<grid_for(ng, 256), 256, 0, s>>>(ng, (const uint32_t*)(base + L.gcost), k0, v0,
                                                       (unsigned long long*)(hdr + 8));
        note_launch();
    }
    uint32_t *sk, *sv;
    radix_sort_pairs<uint32_t>(k0, v0, k1, v1, ng, 0, 32, base + L.tmp, s, &sk, &sv, t->d_err);
    hp.order = sv;
    if (n_warps > 0) {
        { k_heavy_plan<<<1, kHeavyGroups, 0, s>>>(ng, sk, (unsigned long long)n_warps, hdr, table); note_launch(); }
        hp.hdr = hdr;
        hp.table = table;
    }
    return hp;
}
template HeavyPlan heavy_first_order<float>(lens_tree*, const ShootPlan&, const RayKey&, int64_t, cudaStream_t);
template HeavyPlan heavy_first_order<double>(lens_tree*, const ShootPlan&, const RayKey&, int64_t, cudaStream_t);

}  // namespace lens

// ===================================================== allocation-free shoot
//
// lens_shoot_rays_direct_noalloc: the direct sum over every particle of a
// built tree, for callers that must not allocate device memory while they
// shoot rays.  Its ray-group scratch (work counters, per-group anchors and
// boxes, per-ray offsets and indices) lives in one file-scope device array of
// fixed size instead of the tree's on-demand buffers; rays are grouped in
// their input order, 32 per group, so no sort buffers are needed.

namespace lens {

constexpr int64_t kNoAllocMaxRays = 262144;
constexpr size_t kNoAllocGroups = (size_t)(kNoAllocMaxRays / 32 + 1);
constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
// byte offsets of the pieces (every piece 256-byte aligned; sizes for FP64)
constexpr size_t kNaCounters = 0;  // one work counter per launch (64 launches)
constexpr size_t kNaRayL = kNaCounters + 256;
constexpr size_t kNaRayIdx = kNaRayL + al256((size_t)kNoAllocMaxRays * 2 * sizeof(double));
constexpr size_t kNaGH = kNaRayIdx + al256((size_t)kNoAllocMaxRays * sizeof(uint32_t));
constexpr size_t kNaGBox = kNaGH + al256(kNoAllocGroups * 2 * sizeof(double));
constexpr size_t kNaGRange = kNaGBox + al256(kNoAllocGroups * 4 * sizeof(double));
constexpr size_t kNoAllocBytes = kNaGRange + al256(kNoAllocGroups * sizeof(uint2));

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

template <typename T>
__global__ void k_groups_inorder(int64_t n, double ox, double oy, const void* dx, const void* dy, int dtype,
                                 int64_t n_groups, v2_t<T>* gH, vec4_t<T>* gbox, uint2* grange,
                                 v2_t<T>* ray_l, uint32_t* ray_idx)
{
    const unsigned full = 0xffffffffu;
    int lane = threadIdx.x & 31;
    int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= n_groups) return;
    int64_t i = 32 * g + lane;
    bool v = i < n;
    double px = v ? ox + ray_offset(dx, dtype, i) : 0.0, py = v ? oy + ray_offset(dy, dtype, i) : 0.0;
    double xmin = v ? px : INFINITY, xmax = v ? px : -INFINITY, ymin = v ? py : INFINITY, ymax = v ? py : -INFINITY;
    for (int o = 16; o; o >>= 1) {
        xmin = fmin(xmin, __shfl_xor_sync(full, xmin, o));
        xmax = fmax(xmax, __shfl_xor_sync(full, xmax, o));
        ymin = fmin(ymin, __shfl_xor_sync(full, ymin, o));
        ymax = fmax(ymax, __shfl_xor_sync(full, ymax, o));
    }
    bool exact = !v || ((double)(T)px == px && (double)(T)py == py);
    exact = __all_sync(full, exact);
    T Hx = exact ? T(0) : (T)(0.5 * (xmin + xmax)), Hy = exact ? T(0) : (T)(0.5 * (ymin + ymax));
    T lx = v ? (T)(px - (double)Hx) : T(0), ly = v ? (T)(py - (double)Hy) : T(0);
    T lxmin = v ? lx : (T)INFINITY, lxmax = v ? lx : (T)-INFINITY, lymin = v ? ly : (T)INFINITY,
      lymax = v ? ly : (T)-INFINITY;
    for (int o = 16; o; o >>= 1) {
        lxmin = fmin(lxmin, __shfl_xor_sync(full, lxmin, o));
        lxmax = fmax(lxmax, __shfl_xor_sync(full, lxmax, o));
        lymin = fmin(lymin, __shfl_xor_sync(full, lymin, o));
        lymax = fmax(lymax, __shfl_xor_sync(full, lymax, o));
    }
    if (v) {
        v2_t<T> l;
        l.x = lx;
        l.y = ly;
        ray_l[i] = l;
        ray_idx[i] = (uint32_t)i;
    }
    if (lane == 0) {
        T cx = T(0.5) * (lxmin + lxmax), cy = T(0.5) * (lymin + lymax);
        T hx = fmax(lxmax - cx, cx - lxmin) * T(1.0 + 1e-5) + T(1e-30);
        T hy = fmax(lymax - cy, cy - lymin) * T(1.0 + 1e-5) + T(1e-30);
        v2_t<T> H;
        H.x = Hx;
        H.y = Hy;
        gH[g] = H;
        vec4_t<T> bx;
        bx.x = cx; bx.y = cy; bx.z = hx; bx.w = hy;
        gbox[g] = bx;
        int64_t cnt = n - 32 * g;
        grange[g] = make_uint2((uint32_t)(32 * g), (uint32_t)(cnt < 32 ? cnt : 32));
    }
}

// Device address of the scratch array on the current device (the host-side
// name of a __device__ array is only a handle, not a device address).
// lens_build_tree looks it up with the tree's device current and keeps it in
// the tree, so the allocation-free call itself makes no runtime lookup, and a
// tree built after a device reset holds the new address.
lens_status noalloc_scratch_address(void** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        *out = nullptr;
        return lens_cuda_check(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress(no-alloc scratch)");
    }
    *out = p;
    return LENS_OK;
}

template <typename T>
static lens_status noalloc_typed(lens_tree* t, double ox, double oy, const void* dx, const void* dy,
                                 int dtype, int64_t n, void* const out[5], int flags, cudaStream_t s)
{
    using T4 = vec4_t<T>;
    using T2 = v2_t<T>;
    unsigned char* base = (unsigned char*)t->noalloc_scratch;
    if (!base) return lens_set_error(LENS_ERR_INTERNAL, "tree holds no address of the no-alloc scratch");
    uint32_t* counters = (uint32_t*)(base + kNaCounters);
    T2* ray_l = (T2*)(base + kNaRayL);
    uint32_t* ray_idx = (uint32_t*)(base + kNaRayIdx);
    T2* gH = (T2*)(base + kNaGH);
    T4* gbox = (T4*)(base + kNaGBox);
    uint2* grange = (uint2*)(base + kNaGRange);
    const int64_t ng = (n + 31) / 32;
    // the work counters must start at zero: the array keeps the last call's values
    LENS_CUDA(cudaMemsetAsync(counters, 0, 256, s));
    { k_groups_inorder<T><<<grid_for(ng * 32, 256), 256, 0, s>>>(n, ox, oy, dx, dy, dtype, ng, gH, gbox, grange,
                                                                 ray_l, ray_idx); note_launch(); }
    WalkParams<T> P{};
    P.gH = gH; P.gbox = gbox; P.grange = grange; P.ray_l = ray_l; P.ray_idx = ray_idx;
    P.n_groups = ng;
    P.stack = (int*)base;  // the direct sum never touches a stack
    P.err = t->d_err;
    for (int q = 0; q < 5; ++q) P.out[q] = (T*)out[q];
    const bool ao = (flags & LENS_ALPHA_ONLY) != 0;
    int launches = 0;
    bool first_launch = true;
    for (size_t si = 0; si < t->sp.size(); ++si) {
        const SpeciesTree& sp = t->sp[si];
        if (sp.n == 0) continue;
        P.leaf0 = (const T4*)sp.exact0;
        P.leaf1 = (const T4*)sp.exact1;
        P.n_part = sp.n;
        P.Uq = (T)sp.Uq;
        P.invNq = (T)sp.invNq;
        P.halos = t->halos;
        P.n_halos = first_launch ? (int)t->n_halos : 0;
        P.accumulate = first_launch ? ((flags & LENS_ACCUMULATE) ? 1 : 0) : 1;
        P.counter = counters + launches;
        launch_dispatch<T, 1>(sp.kind, ao, true, P, t->num_sms, s);
        first_launch = false;
        ++launches;
    }
    if (first_launch) {
        P.n_part = 0;
        P.halos = t->halos;
        P.n_halos = (int)t->n_halos;
        P.accumulate = (flags & LENS_ACCUMULATE) ? 1 : 0;
        P.counter = counters;
        launch_dispatch<T, 1>(LENS_POINT, ao, true, P, t->num_sms, s);
    }
    LENS_CUDA(cudaGetLastError());
    return LENS_OK;
}

}  // namespace lens

extern "C" lens_status lens_shoot_rays_direct_noalloc(lens_tree* tree, double origin_x, double origin_y,
                                                      const void* ray_dx, const void* ray_dy,
                                                      int32_t ray_dtype, int64_t n, void* alpha1,
                                                      void* alpha2, void* kappa, void* gamma1, void* gamma2,
                                                      int32_t flags, void* stream)
{
    using namespace lens;
    if (!tree) return lens_set_error(LENS_ERR_INVALID_ARG, "tree is NULL");
    if (flags & ~(LENS_ALPHA_ONLY | LENS_ACCUMULATE))
        return lens_set_error(LENS_ERR_INVALID_ARG, "only LENS_ALPHA_ONLY and LENS_ACCUMULATE apply here");
    if (n < 0) return lens_set_error(LENS_ERR_INVALID_ARG, "n must be >= 0");
    if (n > kNoAllocMaxRays)
        return lens_set_error(LENS_ERR_INVALID_ARG,
                              "lens_shoot_rays_direct_noalloc takes at most %lld rays per call (got %lld)",
                              (long long)kNoAllocMaxRays, (long long)n);
    if (ray_dtype != LENS_F32 && ray_dtype != LENS_F64) return lens_set_error(LENS_ERR_INVALID_ARG, "bad ray dtype");
    if (!std::isfinite(origin_x) || !std::isfinite(origin_y))
        return lens_set_error(LENS_ERR_INVALID_ARG, "origin must be finite");
    if (n == 0) return LENS_OK;
    if (!ray_dx || !ray_dy || !alpha1 || !alpha2) return lens_set_error(LENS_ERR_INVALID_ARG, "NULL array");
    if (!(flags & LENS_ALPHA_ONLY) && (!kappa || !gamma1 || !gamma2))
        return lens_set_error(LENS_ERR_INVALID_ARG, "kappa/gamma outputs are NULL without LENS_ALPHA_ONLY");
    int dev = -1;
    LENS_CUDA(cudaGetDevice(&dev));
    if (dev != tree->device) return lens_set_error(LENS_ERR_INVALID_ARG, "tree was built on another device");
    void* out[5] = {alpha1, alpha2, kappa, gamma1, gamma2};
    cudaStream_t s = (cudaStream_t)stream;
    LENS_TRY(wait_built(tree, s));
    if (tree->precision == LENS_PREC_FP64)
        return noalloc_typed<double>(tree, origin_x, origin_y, ray_dx, ray_dy, ray_dtype, n, out, flags, s);
    return noalloc_typed<float>(tree, origin_x, origin_y, ray_dx, ray_dy, ray_dtype, n, out, flags, s);
}
