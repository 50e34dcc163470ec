// walk_shared.cuh -- definitions shared by the forward walk (walk.cu), the
// adjoint walk (backward.cu) and graph replay (batch.cu).
#pragma once

#include "sort.cuh"
#include "tree.cuh"

namespace lens {

template <typename T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };
template <typename T> using v2_t = typename V2<T>::type;

__device__ __forceinline__ int batch_of(const int64_t* boff, int nb, int64_t i)
{
    int lo = 0, hi = nb;  // boff[lo] <= i < boff[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (boff[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ double ray_offset(const void* p, int dtype, int64_t i)
{
    return dtype == LENS_F32 ? (double)((const float*)p)[i] : ((const double*)p)[i];
}

// Does the box {x0, y0, x1, y1} (frame coordinates) reach the group's ray
// box?  The subtraction of H is rounded; a relative margin keeps the test
// conservative.
template <typename T>
LENS_DEV bool box_reaches_group(const vec4_t<T>& b, const v2_t<T>& H, const vec4_t<T>& g)
{
    const T eps = sizeof(T) == 4 ? T(4.8e-7) : T(8.9e-16);
    T x0 = b.x - H.x, x1 = b.z - H.x, y0 = b.y - H.y, y1 = b.w - H.y;
    T tx = eps * (fabs(b.x) + fabs(b.z) + T(2) * fabs(H.x)), ty = eps * (fabs(b.y) + fabs(b.w) + T(2) * fabs(H.y));
    return x0 - tx <= g.x + g.z && x1 + tx >= g.x - g.z && y0 - ty <= g.y + g.w && y1 + ty >= g.y - g.w;
}

// ------------------------------------------------------- shoot scratch

struct Layout {
    size_t boff, borig, gfirst, bbox, k0, k1, v0, v1, tmp, rl, ridx, gH, gbox, grange, counter,
        stack, split, gcost, heavy, total;
};

// Tags of a kept interaction-list entry (LENS_KEEP_LISTS): the box's index
// in the low 29 bits; a box may be accepted (far cell) or an opened leaf, and
// its big list may reach the group as well.
constexpr uint32_t kListFar = 1u << 31, kListLeaf = 1u << 30, kListBig = 1u << 29, kListIdMask = kListBig - 1u;
constexpr uint32_t kListOverflow = 0xffffffffu;  // list_n value of a group whose lists did not fit

// Split heavy groups (heavy_first_order): at most kHeavyGroups groups, each
// in at most 32 slices; the plan's table holds one entry per slice.
constexpr int kHeavyGroups = 1024, kHeavyItems = kHeavyGroups * 32;

// Partial sums of a direct sum split over particle slices: room for 32 rays
// per warp slot of the device, five outputs, FP64 (see split_slices).
inline size_t split_values(int64_t slots) { return (size_t)slots * 32; }

inline Layout make_layout(int64_t n, int64_t nb, int64_t slots)
{
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    Layout L{};
    int64_t ng = n / 32 + nb + 1;
    size_t o = 0;
    L.boff = o; o += al((nb + 1) * sizeof(int64_t));
    L.borig = o; o += al(nb * 2 * sizeof(double));
    L.gfirst = o; o += al((nb + 1) * sizeof(uint32_t));
    L.bbox = o; o += al(nb * 4 * sizeof(unsigned long long));
    L.k0 = o; o += al(n * sizeof(uint64_t));
    L.k1 = o; o += al(n * sizeof(uint64_t));
    L.v0 = o; o += al(n * sizeof(uint32_t));
    L.v1 = o; o += al(n * sizeof(uint32_t));
    L.tmp = o; o += al(radix_sort_temp_bytes<uint64_t>(n));
    L.rl = o; o += al(n * 2 * sizeof(double));
    L.ridx = o; o += al(n * sizeof(uint32_t));
    L.gH = o; o += al(ng * 2 * sizeof(double));
    L.gbox = o; o += al(ng * 4 * sizeof(double));
    L.grange = o; o += al(ng * sizeof(uint2));
    L.counter = o; o += al(64 * sizeof(uint32_t));
    L.stack = o; o += al((size_t)slots * kStackCap * sizeof(int));
    L.split = o; o += al(split_values(slots) * 5 * sizeof(double));
    L.gcost = o; o += al(ng * sizeof(uint32_t));
    L.heavy = o; o += al(64 + (size_t)kHeavyItems * sizeof(uint32_t));
    L.total = o;
    return L;
}

inline int max_slots(lens_tree* t) { return t->num_sms * 16 * kWalkWarps; }


// Host-side plan of one shoot call: sizes fixed by the batch table.
struct ShootPlan {
    int64_t n = 0, nb = 0;
    uint64_t ng = 0;
    int R = 1;
    double ox = 0, oy = 0;  // the origin of a single batch
};

// Work order of the ray groups: a tree walk records every group's work
// (boxes visited + cells + leaf particles + kept big-list entries) in the
// scratch; a later walk over the same rays (the adjoint of a forward call, a
// repeated shot) takes the groups heaviest first, so that a heavy group (rays
// in the densest region) does not run alone at the end of the launch.
struct RayKey {
    const void* dx = nullptr;
    const void* dy = nullptr;
    int64_t n = -1;
    int dtype = -1, R = 0;
    double ox = 0, oy = 0;
    bool operator==(const RayKey& o) const
    {
        return dx == o.dx && dy == o.dy && n == o.n && dtype == o.dtype && R == o.R && ox == o.ox && oy == o.oy;
    }
};
// The heaviest-first order of the plan's groups if the tree's recorded costs
// belong to these rays (order null otherwise); uses the ray sort's buffers.
// With n_warps > 0 it also splits the heaviest groups for a launch of that
// many warps: a group whose work exceeds a quarter of one warp's share gets
// ns = ceil(work / quarter share) slices (at most 32).  hdr[0] = Kc (groups
// split; they lead the order), hdr[1] = Hn (their slices); table[k] for
// k < Hn = (i << 10) | (slice << 5) | (ns - 1), i the group's position in
// the order.  Work item k < Hn is that slice; item k >= Hn walks the whole
// group order[k - Hn + Kc].
struct HeavyPlan {
    const uint32_t* order = nullptr;
    const uint32_t* hdr = nullptr;
    const uint32_t* table = nullptr;
};
template <typename T>
HeavyPlan heavy_first_order(lens_tree* t, const ShootPlan& plan, const RayKey& key, int64_t n_warps,
                            cudaStream_t s);

// The interaction lists kept by the last LENS_KEEP_LISTS walk if they belong
// to these rays (walk.cu), else null.
const uint32_t* kept_lists(const lens_tree* t, const RayKey& k);
// Does the shoot scratch hold the groups of these rays (walk.cu)?
bool groups_hold(const lens_tree* t, const RayKey& k);

lens_status reserve_rays(lens_tree* t, int64_t n, int64_t nb, cudaStream_t s);
// max_r caps the rays per lane (4: 128-ray groups for the one-warp tree walk;
// 2 for the other kernels, which hold at most 64 rays per group).
lens_status upload_batches(lens_tree* t, int64_t nb, const int64_t* h_off, const double* h_orig,
                           cudaStream_t s, ShootPlan* plan, int max_r = 2);
// The cap of upload_batches for a shoot call with these flags on this tree.
int shoot_max_r(const lens_tree* t, int flags);
// Ray grouping of one shoot call (sort + groups) into the tree's scratch.
template <typename T>
lens_status enqueue_groups(lens_tree* t, const ShootPlan& plan, const void* dx, const void* dy, int dtype,
                           cudaStream_t s);

}  // namespace lens
