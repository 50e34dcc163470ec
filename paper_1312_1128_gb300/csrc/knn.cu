// knn.cu -- smoothing lengths on the GPU (Sec. 3.1): for every particle the
// distance to its k-th nearest other particle in 3D, the size the smoothed
// particles of the lens are given (the paper prefers the 3D neighbour
// distance).
//
// Particles are sorted by 63-bit 3D Morton keys of a cube around them, which
// makes every octree cell one run of the sorted keys.  A query first takes
// the k nearest among its 2k neighbours in key order (an upper bound on the
// k-th distance), then descends the implicit octree from the root: a cell's
// run splits into its children's runs by binary search within it, children
// whose box lies farther than the current k-th distance are skipped, the
// nearest child is visited first, and cells of at most kKnnLeaf particles
// are scanned.  32 consecutive particles share one warp and one descent
// (the union of what their queries need); each lane keeps its own k
// smallest squared distances; the search is exact.
#include <cmath>

#include "common.cuh"
#include "sort.cuh"

namespace lens {

constexpr int kKnnMax = 64;    // largest k
constexpr int kKnnBits = 21;   // key bits per axis
constexpr int kKnnLeaf = 16;   // a cell with at most this many particles is scanned
constexpr int kKnnStack = 8 * kKnnBits + 8;  // depth-first: at most 7 siblings pending per level

// Spread the 21 bits of v to every third bit.
LENS_DEV uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffull;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

LENS_DEV uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) { return spread3(x) | spread3(y) << 1 | spread3(z) << 2; }

// Inverse of spread3: every third bit back to 21 contiguous bits.
LENS_DEV uint32_t compact3(uint64_t x)
{
    x &= 0x1249249249249249ull;
    x = (x | x >> 2) & 0x10c30c30c30c30c3ull;
    x = (x | x >> 4) & 0x100f00f00f00f00full;
    x = (x | x >> 8) & 0x1f0000ff0000ffull;
    x = (x | x >> 16) & 0x1f00000000ffffull;
    x = (x | x >> 32) & 0x1fffffull;
    return (uint32_t)x;
}

struct KnnCube {
    float ox, oy, oz;  // lower corner
    float inv_q;       // quanta per unit length (2^21 / side)
    float side;
};

LENS_DEV uint32_t quantise(float v, float o, float inv_q)
{
    float t = (v - o) * inv_q;
    t = fminf(fmaxf(t, 0.0f), (float)((1u << kKnnBits) - 1));
    return (uint32_t)t;
}

__global__ void k_knn_bbox(const float* xyz, int64_t n, unsigned long long* bb)
{
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            const float v = xyz[3 * i + a];
            lo[a] = fminf(lo[a], v);
            hi[a] = fmaxf(hi[a], v);
        }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            atomicMin(&bb[a], dbl_to_ordered((double)lo[a]));
            atomicMax(&bb[3 + a], dbl_to_ordered((double)hi[a]));
        }
}

__global__ void k_knn_bbox_init(unsigned long long* bb)
{
    if (threadIdx.x < 3) {
        bb[threadIdx.x] = dbl_to_ordered(INFINITY);
        bb[3 + threadIdx.x] = dbl_to_ordered(-INFINITY);
    }
}

__global__ void k_knn_keys(const float* xyz, int64_t n, KnnCube c, uint64_t* keys, uint32_t* idx, uint32_t* err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) atomicOr(err, 1u);
    keys[i] = morton3(quantise(x, c.ox, c.inv_q), quantise(y, c.oy, c.inv_q), quantise(z, c.oz, c.inv_q));
    idx[i] = (uint32_t)i;
}

__global__ void k_knn_gather(const float* xyz, int64_t n, const uint32_t* idx, float4* sp)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = idx[i];
    sp[i] = make_float4(xyz[3 * (int64_t)j], xyz[3 * (int64_t)j + 1], xyz[3 * (int64_t)j + 2], __uint_as_float(j));
}

// The k smallest values seen (k <= K), unordered, in shared memory: slot q
// of a lane at v[32 q] (the lanes' slots interleaved: no bank conflicts), in
// groups of 8 slots whose largest value and its slot stay in registers, so
// that a replacement writes one slot and rescans one group (8 loads).  (K
// register slots cannot be indexed at run time: every replacement would
// select through all of them twice, which held the query's ALU pipe.)
template <int K> struct KSmallestSh {
    static constexpr int kS = 8, kG = K / kS;
    static_assert(K % kS == 0, "groups of 8 slots");
    float* v;
    float gmax[kG];
    int gidx[kG];
    int k, cnt, iw;
    float worst;
    LENS_DEV void reset(float* base, int kk, float bound)
    {
        v = base;
        k = kk;
        cnt = 0;
        iw = 0;
        worst = bound;  // values above the bound are not kept
#pragma unroll
        for (int q = 0; q < K; ++q) v[32 * q] = -INFINITY;
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            gmax[g] = -INFINITY;
            gidx[g] = g * kS;
        }
    }
    // rescan group g, then take the largest of the groups' largest values
    LENS_DEV void group(int g)
    {
        float m = -INFINITY;
        int mi = g * kS;
#pragma unroll
        for (int t = 0; t < kS; ++t) {
            const int q = g * kS + t;
            const float x = v[32 * q];
            if (x > m) {
                m = x;
                mi = q;
            }
        }
#pragma unroll
        for (int h = 0; h < kG; ++h)
            if (h == g) {
                gmax[h] = m;
                gidx[h] = mi;
            }
        worst = gmax[0];
        iw = gidx[0];
#pragma unroll
        for (int h = 1; h < kG; ++h)
            if (gmax[h] > worst) {
                worst = gmax[h];
                iw = gidx[h];
            }
    }
    LENS_DEV void offer(float d2)
    {
        if (cnt < k) {
            if (d2 > worst) return;
            v[32 * cnt] = d2;
            if (++cnt == k)
                for (int g = 0; g < kG; ++g) group(g);  // slots at or beyond k hold -inf
        } else if (d2 < worst) {
            v[32 * iw] = d2;
            group(iw / kS);
        }
    }
};

LENS_DEV uint32_t lower_bound_u64(const uint64_t* a, uint32_t lo, uint32_t hi, uint64_t key)
{
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// A pending octree cell: key prefix (3 level bits), level, run [a, b).
struct KnnNode {
    uint64_t prefix;
    uint32_t a, b;
    int level;
};

constexpr int kKnnWarps = 4;   // warps per block of the query (k <= 32)
// warps per block of the query with capacity K: the k smallest distances of
// 64 slots take twice the shared memory, so two warps a block keep a block's
// static shared memory under 48 KB
template <int K> constexpr int knn_warps() { return K <= 32 ? kKnnWarps : 2; }

// One warp per 32 consecutive particles of the key order (spatially close
// queries, one per lane), sharing one descent of the octree: a child cell is
// visited if any lane's query may have a neighbour in it (its box within
// that lane's current k-th distance), the 8 children's runs are found by 8
// lanes' binary searches at once, children are pushed nearest-first by the
// smallest of the lanes' distances, and a scanned cell's particles are
// broadcast to every lane, each keeping its own k smallest.  The stack is
// the warp's, in shared memory.  Exact: a lane never prunes a cell that
// could hold one of its k nearest.
template <int K>
__global__ void __launch_bounds__(knn_warps<K>() * 32)
k_knn_query(const float4* sp4, const uint64_t* keys, int64_t n, int k, KnnCube c, float* r_out, uint32_t* err)
{
    constexpr int KW = knn_warps<K>();
    __shared__ KnnNode stacks[KW][kKnnStack];
    __shared__ float kvals[KW][K][32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    KnnNode* stack = stacks[warp];
    float* kbase = &kvals[warp][0][lane];
    const int64_t i0 = ((int64_t)blockIdx.x * KW + warp) * 32;
    if (i0 >= n) return;
    const int64_t i = i0 + lane;
    const bool valid = i < n;
    const float4 p = valid ? sp4[i] : sp4[i0];
    KSmallestSh<K> S;
    // upper bound: the k nearest among the 2k neighbours in key order
    S.reset(kbase, k, INFINITY);
    if (valid) {
        const int64_t w0 = i - k > 0 ? i - k : 0, w1 = i + k + 1 < n ? i + k + 1 : n;
        for (int64_t j = w0; j < w1; ++j) {
            if (j == i) continue;
            const float4 q = sp4[j];
            const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
            S.offer(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        }
    }
    // descend with the bound as the initial search radius (inflated for the
    // rounding of the squared distances); an invalid lane needs nothing
    const float R2 = valid ? S.worst * 1.000002f : -1.0f;
    S.reset(kbase, k, R2);
    const float qlen = 1.0f / c.inv_q;  // length of one quantum
    int sp = 0;
    if (lane == 0) stack[0] = KnnNode{0ull, 0u, (uint32_t)n, 0};
    sp = 1;
    __syncwarp();
    while (sp > 0) {
        const KnnNode nd = stack[--sp];
        __syncwarp();
        if (nd.b - nd.a <= (uint32_t)kKnnLeaf || nd.level == kKnnBits) {
            for (uint32_t j = nd.a; j < nd.b; ++j) {
                const float4 q = sp4[j];   // the same record for every lane
                if (valid && (int64_t)j != i) {
                    const float ddx = q.x - p.x, ddy = q.y - p.y, ddz = q.z - p.z;
                    S.offer(fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz)));
                }
            }
            continue;
        }
        const int cl = nd.level + 1, shift = kKnnBits - cl;
        const float side = qlen * (float)(1u << shift);
        // lane ch < 8 finds where child ch's run starts
        uint32_t start = nd.a;
        if (lane > 0 && lane < 8) start = lower_bound_u64(keys, nd.a, nd.b, (nd.prefix * 8 + lane) << (3 * shift));
        // children in order, each with the smallest of the lanes' distances to
        // its box (a quantum of margin on every side); kept if any lane needs it
        float cd[8];
        uint32_t ca[8], cb[8];
        int order[8], m = 0;
        for (int ch = 0; ch < 8; ++ch) {
            const uint32_t lo = __shfl_sync(full, start, ch);
            const uint32_t hi = ch == 7 ? nd.b : __shfl_sync(full, start, ch + 1);
            if (hi <= lo) continue;
            const uint64_t pre = nd.prefix * 8 + ch;
            const float bx = c.ox + qlen * (float)(compact3(pre) << shift) - qlen;
            const float by = c.oy + qlen * (float)(compact3(pre >> 1) << shift) - qlen;
            const float bz = c.oz + qlen * (float)(compact3(pre >> 2) << shift) - qlen;
            const float ex = fmaxf(fmaxf(bx - p.x, p.x - (bx + side + 2.0f * qlen)), 0.0f);
            const float ey = fmaxf(fmaxf(by - p.y, p.y - (by + side + 2.0f * qlen)), 0.0f);
            const float ez = fmaxf(fmaxf(bz - p.z, p.z - (bz + side + 2.0f * qlen)), 0.0f);
            const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            const bool need = valid && d2 <= S.worst;
            if (!__any_sync(full, need)) continue;
            float dmin = need ? d2 : INFINITY;
            for (int o = 16; o; o >>= 1) dmin = fminf(dmin, __shfl_xor_sync(full, dmin, o));
            cd[m] = dmin;
            ca[m] = lo;
            cb[m] = hi;
            order[m] = ch;
            ++m;
        }
        // insertion sort by decreasing distance, then push (nearest on top)
        for (int u = 1; u < m; ++u)
            for (int v = u; v > 0 && cd[v] > cd[v - 1]; --v) {
                float td = cd[v]; cd[v] = cd[v - 1]; cd[v - 1] = td;
                uint32_t ta = ca[v]; ca[v] = ca[v - 1]; ca[v - 1] = ta;
                uint32_t tb = cb[v]; cb[v] = cb[v - 1]; cb[v - 1] = tb;
                int to = order[v]; order[v] = order[v - 1]; order[v - 1] = to;
            }
        if (sp + m > kKnnStack) {
            if (lane == 0) atomicOr(err, 4u);  // cannot happen: at most 7 pending siblings per level
            break;
        }
        if (lane == 0)
            for (int u = 0; u < m; ++u) stack[sp + u] = KnnNode{nd.prefix * 8 + order[u], ca[u], cb[u], cl};
        sp += m;
        __syncwarp();
    }
    if (!valid) return;
    if (S.cnt < k) {
        atomicOr(err, 2u);  // cannot happen: the bound's k particles are within the radius
        r_out[__float_as_uint(p.w)] = NAN;
        return;
    }
    r_out[__float_as_uint(p.w)] = sqrtf(S.worst);
}

}  // namespace lens

using namespace lens;

extern "C" lens_status lens_smoothing_lengths(const float* xyz, int64_t n, int32_t k, float* r_sm, void* stream)
{
    if (k < 1 || k > kKnnMax) return lens_set_error(LENS_ERR_INVALID_ARG, "k must be 1..%d", kKnnMax);
    if (n < 0 || n > 0xffffffffll) return lens_set_error(LENS_ERR_INVALID_ARG, "bad particle count");
    if (n == 0) return LENS_OK;
    if (n <= k) return lens_set_error(LENS_ERR_INVALID_ARG, "need more than k particles");
    if (!xyz || !r_sm) return lens_set_error(LENS_ERR_INVALID_ARG, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    const int TB = 256;
    const int64_t G = (n + TB - 1) / TB;
    // scratch: bbox + error word, keys x 2, indices x 2, sorted points, sort temp
    const size_t tmp_bytes = radix_sort_temp_bytes<uint64_t>(n);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_bb = 0, o_err = o_bb + al(6 * 8), o_k0 = o_err + al(8), o_k1 = o_k0 + al(n * 8),
                 o_v0 = o_k1 + al(n * 8), o_v1 = o_v0 + al(n * 4), o_sp = o_v1 + al(n * 4),
                 o_tmp = o_sp + al(n * 16), total = o_tmp + al(tmp_bytes);
    char* base = nullptr;
    LENS_CUDA(lens_malloc_async((void**)&base, total, s));
    unsigned long long* bb = (unsigned long long*)(base + o_bb);
    uint32_t* err = (uint32_t*)(base + o_err);
    uint64_t *k0 = (uint64_t*)(base + o_k0), *k1 = (uint64_t*)(base + o_k1);
    uint32_t *v0 = (uint32_t*)(base + o_v0), *v1 = (uint32_t*)(base + o_v1);
    float4* sp = (float4*)(base + o_sp);
    lens_status st = LENS_OK;
    unsigned long long hbb[6];
    uint32_t herr = 0;
    do {
        cudaError_t e = cudaMemsetAsync(err, 0, 4, s);
        if (e != cudaSuccess) { st = lens_cuda_check(e, "memset"); break; }
        k_knn_bbox_init<<<1, 32, 0, s>>>(bb);
        note_launch();
        k_knn_bbox<<<(unsigned)(G < 1024 ? G : 1024), TB, 0, s>>>(xyz, n, bb);
        note_launch();
        e = cudaMemcpyAsync(hbb, bb, sizeof(hbb), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { st = lens_cuda_check(e, "bbox"); break; }
        double lo[3], hi[3], side = 0.0;
        for (int a = 0; a < 3; ++a) {
            lo[a] = ordered_to_dbl(hbb[a]);
            hi[a] = ordered_to_dbl(hbb[3 + a]);
            side = std::max(side, hi[a] - lo[a]);
        }
        if (!std::isfinite(side)) { st = lens_set_error(LENS_ERR_INVALID_ARG, "non-finite particle position"); break; }
        side = side > 0.0 ? side * (1.0 + 1e-5) : 1.0;
        KnnCube c;
        c.ox = (float)lo[0];
        c.oy = (float)lo[1];
        c.oz = (float)lo[2];
        c.side = (float)side;
        c.inv_q = (float)((double)(1u << kKnnBits) / side);
        k_knn_keys<<<(unsigned)G, TB, 0, s>>>(xyz, n, c, k0, v0, err);
        note_launch();
        uint64_t* sk;
        uint32_t* sv;
        radix_sort_pairs<uint64_t>(k0, v0, k1, v1, n, 0, 3 * kKnnBits, base + o_tmp, s, &sk, &sv, err);
        k_knn_gather<<<(unsigned)G, TB, 0, s>>>(xyz, n, sv, sp);
        note_launch();
        if (k <= 32) {
            constexpr int W = knn_warps<32>();
            const unsigned qb = (unsigned)((n + 32 * W - 1) / (32 * W));
            k_knn_query<32><<<qb, W * 32, 0, s>>>(sp, sk, n, k, c, r_sm, err);
        } else {
            constexpr int W = knn_warps<kKnnMax>();
            const unsigned qb = (unsigned)((n + 32 * W - 1) / (32 * W));
            k_knn_query<kKnnMax><<<qb, W * 32, 0, s>>>(sp, sk, n, k, c, r_sm, err);
        }
        note_launch();
        e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { st = lens_cuda_check(e, "smoothing lengths"); break; }
        if (herr & 1u) st = lens_set_error(LENS_ERR_INVALID_ARG, "non-finite particle position");
        else if (herr) st = lens_set_error(LENS_ERR_INTERNAL, "neighbour search check failed (code %u)", herr);
    } while (false);
    cudaFreeAsync(base, s);
    return st;
}
