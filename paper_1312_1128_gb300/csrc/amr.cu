// amr.cu -- image finding for uniform circular sources by adaptive grid
// refinement (Sec. 4), many sources at once.
//
// Each source has its own grid: N x N cells over [x0, x0+S]^2 refined by
// thirds (a cell (L, i, j) has side h_L = S / (N 3^L) and 9 children
// (L+1, 3i+a, 3j+b)); a leaf cell carries the source-plane point y = x -
// alpha(x) of its centre.  Leaves of all sources live in one array ordered
// by a key: the source, the level-0 cell i N + j, then one base-9 digit
// 3a + b per level, padded to level L_max -- a leaf covers the keys
// [key, key + 9^(L_max - L)).  Refining a leaf writes its 9 children in
// digit order where it stood, so the array stays ordered with one scan and
// no sort; the middle child keeps the parent's point (same centre).
//
// Neighbours (cells sharing an edge, Sec. 4 "neighbors of neighbors"): the
// leaf containing cell (L, i +- 1, j) or (L, i, j +- 1) is found by binary
// search of its key; a leaf accepts only neighbours at its own level or
// coarser, so each pair is found by its finer (or both equal) member.
// Images are connected sets of cells whose point lies in the source, found
// by a lock-free union-find over those pairs (roots hooked to the smaller
// index, so an image's root is its smallest key).  Inner border: image cells
// with a non-image neighbour; outer border: non-image cells with an image
// neighbour.
//
// Per source, the steps of Sec. 4 run as a small state machine, and one
// round refines the marked cells of every source together:
//   telescoping: source radius r_0 = h_0 / sqrt(mu_min), divided by 3 down
//     to R; at each radius r cells with a point inside r and h_L > r
//     sqrt(mu_min) / 3 are refined until none remain;
//   uniform: while an image has fewer than n_min cells, its cells and its
//     outer border are refined;
//   border: until its largest border cell has area < f_area x its area and
//     its outer border is as fine as its inner border, an image's border
//     cells of the largest size are refined;
// cells at level L_max are never refined.  A source's images are final in
// the border round that marks none of its cells: they are recorded then, and
// its cells leave the working array in the same refinement pass (a count of
// 0 in the scan), so later rounds touch only unfinished sources.  Every
// decision compares FP64
// values formed by the same operations on the host (exact per-level cell
// counts for the areas) and on the device (explicit round-to-nearest
// operations, no contraction), so that the cell sets follow the method's
// definition exactly.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "sort.cuh"
#include "tree.cuh"

namespace lens {
namespace {

constexpr int kAmrThreads = 256;
constexpr int kAmrMaxLevel = 20;
enum : int { MODE_TELE = 0, MODE_UNIFORM = 1, MODE_BORDER = 2, MODE_DONE = 3 };
enum : int { ACT_NONE = -1, ACT_UNIFORM = -2 };

struct AmrConst {
    double x0, y0;
    double h[kAmrMaxLevel + 1];                // S / (N 3^L)
    unsigned long long pow9[kAmrMaxLevel + 1];
    unsigned int pow3[kAmrMaxLevel + 1];
    unsigned long long src_span;               // N^2 9^L_max keys per source
    int n, l_max;
};

struct Leaves {
    uint64_t* key;
    uint8_t* lv;
    uint32_t* i;
    uint32_t* j;
    int32_t* src;
    double* yx;
    double* yy;
};

inline unsigned blocks(int64_t n) { return (unsigned)((n + kAmrThreads - 1) / kAmrThreads); }

__device__ __forceinline__ uint64_t make_key(const AmrConst& C, int s, int lv, uint32_t i, uint32_t j)
{
    // base-9 digits from the finest level up (constant divisions by 3), then
    // the level-0 cell
    uint64_t c = 0, m = 1;
    for (int l = 0; l < lv; ++l) {
        c += (uint64_t)(3u * (i % 3u) + (j % 3u)) * m;
        i /= 3u;
        j /= 3u;
        m *= 9ull;
    }
    c += ((uint64_t)i * (uint64_t)C.n + j) * m;
    return (uint64_t)s * C.src_span + c * C.pow9[C.l_max - lv];
}

// cell centre coordinate x0 + (i + 1/2) h_L, one rounding per operation
__device__ __forceinline__ double centre(double x0, uint32_t i, double h)
{
    return __dadd_rn(x0, __dmul_rn((double)i + 0.5, h));
}

__global__ void k_init(Leaves L, AmrConst C, int64_t n, double* rx, double* ry, uint32_t* rslot)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t nn = (int64_t)C.n * C.n;
    const int s = (int)(k / nn);
    const uint32_t c0 = (uint32_t)(k % nn), i = c0 / C.n, j = c0 % C.n;
    L.key[k] = (uint64_t)k * C.pow9[C.l_max];
    L.lv[k] = 0;
    L.i[k] = i;
    L.j[k] = j;
    L.src[k] = s;
    rx[k] = centre(C.x0, i, C.h[0]);
    ry[k] = centre(C.y0, j, C.h[0]);
    rslot[k] = (uint32_t)k;
}

template <typename T>
__global__ void k_sety(Leaves L, const double* rx, const double* ry, const T* a1, const T* a2, const uint32_t* rslot,
                       int64_t nr)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    const uint32_t s = rslot[r];
    L.yx[s] = __dsub_rn(rx[r], (double)a1[r]);
    L.yy[s] = __dsub_rn(ry[r], (double)a2[r]);
}

// in[k]: the leaf's point lies inside its source's current circle
__global__ void k_inside(Leaves L, int64_t n, const double* scx, const double* scy, const double* sr2, uint8_t* in)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int s = L.src[k];
    const double dx = __dsub_rn(L.yx[k], scx[s]), dy = __dsub_rn(L.yy[k], scy[s]);
    in[k] = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) < sr2[s] ? 1 : 0;
}

__global__ void k_mark_tele(Leaves L, int64_t n, AmrConst C, const uint8_t* in, const int* mode, const double* thr,
                            uint8_t* mark)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int s = L.src[k], lv = L.lv[k];
    mark[k] = (mode[s] == MODE_TELE && in[k] && C.h[lv] > thr[s] && lv < C.l_max) ? 1 : 0;
}

// nb[4k + d]: the leaf at k's level or coarser sharing k's edge d, or -1
__global__ void k_neighbours(Leaves L, int64_t n, AmrConst C, const uint8_t* want, int32_t* nb)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int s = L.src[k], lv = L.lv[k];
    const uint32_t i = L.i[k], j = L.j[k], lim = (uint32_t)C.n * C.pow3[lv];
    const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        int32_t res = -1;
        const int64_t ni = (int64_t)i + di[d], nj = (int64_t)j + dj[d];
        if (want[s] && ni >= 0 && nj >= 0 && ni < lim && nj < lim) {
            const uint64_t q = make_key(C, s, lv, (uint32_t)ni, (uint32_t)nj);
            // the last leaf with key <= q, galloping out from k (a +x / +y
            // neighbour has a larger key, a -x / -y one a smaller) to
            // key[lo] <= q < key[hi], then bisecting
            int64_t lo, hi, step = 1;
            if (L.key[k] <= q) {
                lo = k;
                hi = k + 1;
                while (hi < n && L.key[hi] <= q) {
                    lo = hi;
                    step *= 2;
                    hi = k + step;
                }
                if (hi > n) hi = n;
            } else {
                hi = k;
                lo = k - 1;
                while (lo >= 0 && L.key[lo] > q) {
                    hi = lo;
                    step *= 2;
                    lo = k - step;
                }
                if (lo < 0) lo = -1;
            }
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (L.key[mid] <= q) lo = mid;
                else hi = mid;
            }
            const int64_t c = lo;
            if (c >= 0) {
                const int lc = L.lv[c];
                if (lc <= lv && q < L.key[c] + C.pow9[C.l_max - lc]) res = (int32_t)c;
            }
        }
        nb[4 * k + d] = res;
    }
}

// ------------------------------------------------------------ union-find
__device__ __forceinline__ int32_t uf_find(int32_t* parent, int32_t u)
{
    volatile int32_t* p = parent;
    for (;;) {
        const int32_t q = p[u];
        if (q == u) return u;
        const int32_t r = p[q];
        if (r != q) p[u] = r;  // path halving on a non-root node
        u = q;
    }
}

// Union-find, first inside each block of kAmrThreads consecutive leaves (in
// shared memory: the pairs whose both cells lie in the block), then across
// blocks.  Every hook points to a smaller index, so a root is its
// component's smallest index.  Equal-level pairs are taken once (from the
// +x / +y side); a cell of another source or outside an image is -1.
__device__ __forceinline__ int32_t uf_find_shared(volatile int32_t* p, int32_t u)
{
    for (;;) {
        const int32_t q = p[u];
        if (q == u) return u;
        u = q;
    }
}

__global__ void __launch_bounds__(kAmrThreads) k_uf_local(Leaves L, int64_t n, const uint8_t* in, const uint8_t* want,
                                                        const int32_t* nb, int32_t* parent)
{
    __shared__ int32_t sp[kAmrThreads];
    const int t = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * kAmrThreads, k = base + t;
    const bool mine = k < n && in[k] && want[L.src[k]];
    sp[t] = mine ? t : -1;
    __syncthreads();
    if (mine) {
        for (int d = 0; d < 4; ++d) {
            const int32_t c = nb[4 * k + d];
            if (c < base || c >= base + kAmrThreads || sp[c - base] < 0) continue;
            if ((d & 1) && L.lv[c] == L.lv[k]) continue;
            int32_t a = t, b = (int32_t)(c - base);
            for (;;) {
                a = uf_find_shared(sp, a);
                b = uf_find_shared(sp, b);
                if (a == b) break;
                const int32_t hi = a > b ? a : b, lo = a > b ? b : a;
                if (atomicCAS(&sp[hi], hi, lo) == hi) break;
            }
        }
    }
    __syncthreads();
    if (k < n) parent[k] = mine ? (int32_t)(base + uf_find_shared(sp, t)) : -1;
}

__global__ void k_uf_unite(Leaves L, int64_t n, const int32_t* nb, int32_t* parent)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || parent[k] < 0) return;
    const int64_t base = (int64_t)blockIdx.x * kAmrThreads;
    for (int d = 0; d < 4; ++d) {
        const int32_t c = nb[4 * k + d];
        if (c < 0 || parent[c] < 0) continue;
        if (c >= base && c < base + kAmrThreads) continue;  // united inside the block
        if ((d & 1) && L.lv[c] == L.lv[k]) continue;  // an equal-level pair is also found from c's +x / +y side
        int32_t a = (int32_t)k, b = c;
        for (;;) {
            a = uf_find(parent, a);
            b = uf_find(parent, b);
            if (a == b) break;
            const int32_t hi = a > b ? a : b, lo = a > b ? b : a;
            if (atomicCAS(&parent[hi], hi, lo) == hi) break;
        }
    }
}

__global__ void k_uf_roots(int64_t n, int32_t* parent, uint32_t* is_root)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int32_t p = parent[k];
    if (p >= 0) {
        p = uf_find(parent, (int32_t)k);
        parent[k] = p;
    }
    is_root[k] = (p == (int32_t)k) ? 1u : 0u;
}

__global__ void k_label(Leaves L, int64_t n, AmrConst C, const int32_t* parent, const uint32_t* rank, int32_t* img,
                        uint32_t* cnt, int32_t* isrc, unsigned long long* ifirst, int32_t cap)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t slot = 0xffffffffu;
    if (k < n) {
        const int32_t p = parent[k];
        int32_t id = -1;
        if (p >= 0) {
            id = (int32_t)rank[p];
            if (id < cap) {
                slot = (uint32_t)id * (uint32_t)(C.l_max + 1) + L.lv[k];
                if (p == (int32_t)k) {
                    isrc[id] = L.src[k];
                    ifirst[id] = L.key[k];
                }
            } else {
                id = -1;
            }
        }
        img[k] = id;
    }
    // neighbouring leaves mostly share an image and a level: one atomic per
    // distinct (image, level) in the warp
    const unsigned peers = __match_any_sync(0xffffffffu, slot);
    if (slot != 0xffffffffu && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1))
        atomicAdd(&cnt[slot], (uint32_t)__popc(peers));
}

// per pair (a in an image, b not): a is inner border, b outer border of a's image
__global__ void k_borders(Leaves L, int64_t n, const int32_t* nb, const int32_t* img, int32_t* lin, int32_t* lout)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    for (int d = 0; d < 4; ++d) {
        const int32_t c = nb[4 * k + d];
        if (c < 0) continue;
        const int32_t ik = img[k], ic = img[c];
        if ((ik >= 0) == (ic >= 0)) continue;
        const int64_t a = ik >= 0 ? k : c, b = ik >= 0 ? c : k;
        const int32_t id = ik >= 0 ? ik : ic;
        atomicMin(&lin[id], (int32_t)L.lv[a]);
        atomicMin(&lout[id], (int32_t)L.lv[b]);
    }
}

__global__ void k_mark_images(Leaves L, int64_t n, AmrConst C, const int32_t* nb, const int32_t* img,
                              const int32_t* act, uint8_t* mark)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t ik = img[k];
    if (ik >= 0 && act[ik] == ACT_UNIFORM && L.lv[k] < C.l_max) mark[k] = 1;
    for (int d = 0; d < 4; ++d) {
        const int32_t c = nb[4 * k + d];
        if (c < 0) continue;
        const int32_t ic = img[c];
        if ((ik >= 0) == (ic >= 0)) continue;
        const int64_t a = ik >= 0 ? k : c, b = ik >= 0 ? c : k;
        const int32_t A = act[ik >= 0 ? ik : ic];
        const int la = L.lv[a], lb = L.lv[b];
        if (A == ACT_UNIFORM) {
            if (lb < C.l_max) mark[b] = 1;
        } else if (A >= 0) {
            if (la == A && la < C.l_max) mark[a] = 1;
            if (lb == A && lb < C.l_max) mark[b] = 1;
        }
    }
}

__global__ void k_count_marks(Leaves L, int64_t n, const uint8_t* mark, uint32_t* cnt9, uint32_t* rmark,
                              uint32_t* nmark)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const bool m = mark[k] != 0;
    cnt9[k] = m ? 9u : 1u;
    rmark[k] = m ? 1u : 0u;
    if (m) atomicAdd(&nmark[L.src[k]], 1u);
}

// the leaves of sources that have just finished leave the working array
// (their images are recorded): output count 0
__global__ void k_drop(Leaves L, int64_t n, const uint8_t* drop, uint32_t* cnt9)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (drop[L.src[k]]) cnt9[k] = 0u;
}

// children of marked leaves in digit order where the parent stood
__global__ void k_refine(Leaves A, int64_t n, AmrConst C, const uint8_t* mark, const uint8_t* drop,
                         const uint32_t* pos, const uint32_t* rpos, Leaves B, double* rx, double* ry,
                         uint32_t* rslot)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || drop[A.src[k]]) return;
    const int64_t p = pos[k];
    const uint64_t key = A.key[k];
    const int lv = A.lv[k];
    const uint32_t i = A.i[k], j = A.j[k];
    const int32_t s = A.src[k];
    if (!mark[k]) {
        B.key[p] = key;
        B.lv[p] = (uint8_t)lv;
        B.i[p] = i;
        B.j[p] = j;
        B.src[p] = s;
        B.yx[p] = A.yx[k];
        B.yy[p] = A.yy[k];
        return;
    }
    const uint64_t step = C.pow9[C.l_max - lv - 1];
    const double h = C.h[lv + 1];
    const int64_t rbase = 8 * (int64_t)rpos[k];  // 8 rays per marked leaf before k
    for (int t = 0; t < 9; ++t) {
        const uint32_t ci = 3u * i + (uint32_t)(t / 3), cj = 3u * j + (uint32_t)(t % 3);
        const int64_t o = p + t;
        B.key[o] = key + (uint64_t)t * step;
        B.lv[o] = (uint8_t)(lv + 1);
        B.i[o] = ci;
        B.j[o] = cj;
        B.src[o] = s;
        if (t == 4) {
            B.yx[o] = A.yx[k];
            B.yy[o] = A.yy[k];
        } else {
            const int64_t r = rbase + (t < 4 ? t : t - 1);
            rx[r] = centre(C.x0, ci, h);
            ry[r] = centre(C.y0, cj, h);
            rslot[r] = (uint32_t)o;
        }
    }
}

template <typename T> struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    ~DevBuf() { release(); }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    cudaError_t alloc(size_t want)
    {
        want = std::max<size_t>(want, 1);
        if (want <= n) return cudaSuccess;
        release();
        cudaError_t e = lens_malloc((void**)&p, want * sizeof(T));
        if (e == cudaSuccess) n = want;
        else p = nullptr;
        return e;
    }
};

struct LeafBufs {
    DevBuf<uint64_t> key;
    DevBuf<uint8_t> lv;
    DevBuf<uint32_t> i, j;
    DevBuf<int32_t> src;
    DevBuf<double> yx, yy;
    cudaError_t alloc(size_t c)
    {
        cudaError_t e;
        if ((e = key.alloc(c)) || (e = lv.alloc(c)) || (e = i.alloc(c)) || (e = j.alloc(c)) || (e = src.alloc(c)) ||
            (e = yx.alloc(c)) || (e = yy.alloc(c)))
            return e;
        return cudaSuccess;
    }
    Leaves view() { return Leaves{key.p, lv.p, i.p, j.p, src.p, yx.p, yy.p}; }
};

// Device memory of one call, kept with the tree and grown when a call needs more.
struct AmrWorkspace {
    LeafBufs A, B;
    DevBuf<uint8_t> in, mark, want, drop;
    DevBuf<int32_t> nb, parent, img, mode, lin, lout, isrc, act;
    DevBuf<uint32_t> is_root, cnt9, rmark, rslot, icnt, nmark, total;
    DevBuf<unsigned long long> ifirst;
    DevBuf<double> rx, ry, a1, a2, scx, scy, sr2, thr;
    DevBuf<char> tmp;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    ~AmrWorkspace()
    {
        for (cudaEvent_t& e : ev)
            if (e) cudaEventDestroy(e);
    }
    cudaError_t alloc(size_t cap, size_t ns, size_t M, int LM)
    {
        cudaError_t e;
        if ((e = A.alloc(cap)) || (e = B.alloc(cap)) || (e = in.alloc(cap)) || (e = mark.alloc(cap)) ||
            (e = want.alloc(ns)) || (e = drop.alloc(ns)) || (e = nb.alloc(4 * cap)) || (e = parent.alloc(cap)) || (e = img.alloc(cap)) ||
            (e = mode.alloc(ns)) || (e = lin.alloc(M)) || (e = lout.alloc(M)) || (e = isrc.alloc(M)) ||
            (e = act.alloc(M)) || (e = is_root.alloc(cap)) || (e = cnt9.alloc(cap)) || (e = rmark.alloc(cap)) || (e = rslot.alloc(cap)) ||
            (e = icnt.alloc(M * (LM + 1))) || (e = nmark.alloc(ns)) || (e = total.alloc(1)) ||
            (e = ifirst.alloc(M)) || (e = rx.alloc(cap)) || (e = ry.alloc(cap)) || (e = a1.alloc(cap)) ||
            (e = a2.alloc(cap)) || (e = scx.alloc(ns)) || (e = scy.alloc(ns)) || (e = sr2.alloc(ns)) ||
            (e = thr.alloc(ns)) || (e = tmp.alloc(scan_temp_bytes((int64_t)cap))))
            return e;
        for (cudaEvent_t& v : ev)
            if (!v && (e = cudaEventCreate(&v))) return e;
        return cudaSuccess;
    }
};

void free_workspace(void* w) { delete static_cast<AmrWorkspace*>(w); }

}  // namespace
}  // namespace lens

using namespace lens;

extern "C" lens_status lens_find_images(lens_tree* tree, const lens_amr_params* prm, int32_t n_sources,
                                        const double* sources, int32_t max_images, lens_image* images,
                                        int32_t* n_images, int64_t* stats, void* stream)
{
    if (!tree || !prm || !n_images) return lens_set_error(LENS_ERR_INVALID_ARG, "NULL tree, params or n_images");
    *n_images = 0;
    if (n_sources < 0 || max_images < 0) return lens_set_error(LENS_ERR_INVALID_ARG, "negative count");
    if (n_sources == 0) return LENS_OK;
    if (!sources || (max_images > 0 && !images))
        return lens_set_error(LENS_ERR_INVALID_ARG, "NULL sources or images array");
    const int N = prm->n, LM = prm->l_max;
    if (N < 1 || N > 4096) return lens_set_error(LENS_ERR_INVALID_ARG, "n must be in [1, 4096]");
    if (LM < 0 || LM > kAmrMaxLevel - 1) return lens_set_error(LENS_ERR_INVALID_ARG, "l_max must be in [0, 19]");
    if (!(prm->side > 0.0) || !std::isfinite(prm->side) || !std::isfinite(prm->x0) || !std::isfinite(prm->y0))
        return lens_set_error(LENS_ERR_INVALID_ARG, "bad grid");
    if (!(prm->mu_min > 0.0 && prm->mu_min <= 1.0) || !(prm->f_area > 0.0) || prm->n_min < 0)
        return lens_set_error(LENS_ERR_INVALID_ARG, "bad mu_min, f_area or n_min");
    // keys: n_sources N^2 9^L_max < 2^63; N 3^L_max < 2^32
    {
        unsigned __int128 span = (unsigned __int128)N * N;
        for (int l = 0; l < LM; ++l) span *= 9;
        if (span * (unsigned)n_sources >= ((unsigned __int128)1 << 63))
            return lens_set_error(LENS_ERR_INVALID_ARG, "n_sources * n^2 * 9^l_max must be below 2^63");
        unsigned long long side_cells = (unsigned long long)N;
        for (int l = 0; l < LM; ++l) side_cells *= 3;
        if (side_cells >= (1ull << 32)) return lens_set_error(LENS_ERR_INVALID_ARG, "n * 3^l_max must be below 2^32");
    }
    for (int s = 0; s < n_sources; ++s)
        if (!(sources[3 * s + 2] > 0.0) || !std::isfinite(sources[3 * s]) || !std::isfinite(sources[3 * s + 1]))
            return lens_set_error(LENS_ERR_INVALID_ARG, "source %d: bad centre or radius", s);
    const int64_t cap = prm->max_cells > 0 ? prm->max_cells : (int64_t)1 << 23;
    const int64_t n0 = (int64_t)n_sources * N * N;
    if (cap > 0xffffffffll || n0 > cap) return lens_set_error(LENS_ERR_INVALID_ARG, "max_cells below the initial grid");
    const int max_rounds = prm->max_rounds > 0 ? prm->max_rounds : 10000;
    const int M = std::max(max_images, 1);
    cudaStream_t st = (cudaStream_t)stream;

    AmrConst C{};
    C.x0 = prm->x0;
    C.y0 = prm->y0;
    C.n = N;
    C.l_max = LM;
    {
        unsigned long long p9 = 1;
        unsigned int p3 = 1;
        for (int l = 0; l <= kAmrMaxLevel; ++l) {
            C.pow9[l] = p9;
            C.pow3[l] = p3;
            double n3 = (double)N;
            for (int q = 0; q < l; ++q) n3 *= 3.0;
            C.h[l] = prm->side / n3;
            if (l < 20) p9 *= 9;
            if (l < 19) p3 *= 3;
        }
        C.src_span = (unsigned long long)N * N * C.pow9[LM];
    }

    if (!tree->amr_ws) {
        tree->amr_ws = new AmrWorkspace();
        tree->amr_free = free_workspace;
    }
    AmrWorkspace& W = *static_cast<AmrWorkspace*>(tree->amr_ws);
    if (cudaError_t e = W.alloc((size_t)cap, (size_t)n_sources, (size_t)M, LM)) {
        cudaGetLastError();
        return lens_set_error(LENS_ERR_OOM, "image finding: device allocation for %lld cells failed (%s)",
                              (long long)cap, cudaGetErrorString(e));
    }
    LeafBufs* cur = &W.A;
    LeafBufs* nxt = &W.B;
    const bool f64 = tree->precision == LENS_PREC_FP64;
    int64_t rays_total = 0, rounds = 0, find_cells = 0;
    double find_ms = 0.0, shoot_ms = 0.0;

    auto shoot = [&](int64_t nr) -> lens_status {
        if (nr == 0) return LENS_OK;
        LENS_CUDA(cudaEventRecord(W.ev[2], st));
        LENS_TRY(lens_shoot_rays(tree, 0.0, 0.0, W.rx.p, W.ry.p, LENS_F64, nr, W.a1.p, W.a2.p, nullptr, nullptr,
                                 nullptr, LENS_ALPHA_ONLY, stream));
        if (f64) {
            k_sety<double><<<blocks(nr), kAmrThreads, 0, st>>>(cur->view(), W.rx.p, W.ry.p, W.a1.p, W.a2.p,
                                                               W.rslot.p, nr);
        } else {
            k_sety<float><<<blocks(nr), kAmrThreads, 0, st>>>(cur->view(), W.rx.p, W.ry.p, (const float*)W.a1.p,
                                                              (const float*)W.a2.p, W.rslot.p, nr);
        }
        note_launch();
        LENS_CUDA(cudaEventRecord(W.ev[3], st));
        rays_total += nr;
        return LENS_OK;
    };
    auto shoot_time = [&]() -> lens_status {
        float ms = 0.0f;
        LENS_CUDA(cudaEventElapsedTime(&ms, W.ev[2], W.ev[3]));
        shoot_ms += ms;
        return LENS_OK;
    };

    // the initial grids
    int64_t n = n0;
    k_init<<<blocks(n), kAmrThreads, 0, st>>>(cur->view(), C, n, W.rx.p, W.ry.p, W.rslot.p);
    note_launch();
    LENS_TRY(shoot(n));
    LENS_CUDA(cudaStreamSynchronize(st));
    LENS_TRY(shoot_time());

    const double smu = std::sqrt(prm->mu_min);
    std::vector<int> mode(n_sources, MODE_TELE);
    std::vector<double> rcur(n_sources), rad(n_sources), h_cx(n_sources), h_cy(n_sources), h_r2(n_sources),
        h_thr(n_sources);
    std::vector<uint8_t> h_want(n_sources), h_drop(n_sources, 0);
    std::vector<std::vector<lens_image>> done_images(n_sources);
    int64_t final_cells = 0;
    for (int s = 0; s < n_sources; ++s) {
        h_cx[s] = sources[3 * s];
        h_cy[s] = sources[3 * s + 1];
        rad[s] = sources[3 * s + 2];
        double r = C.h[0] / smu;
        if (r < rad[s]) r = rad[s];
        rcur[s] = r;
    }
    LENS_CUDA(cudaMemsetAsync(W.drop.p, 0, n_sources, st));
    LENS_CUDA(cudaMemcpyAsync(W.scx.p, h_cx.data(), n_sources * sizeof(double), cudaMemcpyHostToDevice, st));
    LENS_CUDA(cudaMemcpyAsync(W.scy.p, h_cy.data(), n_sources * sizeof(double), cudaMemcpyHostToDevice, st));
    const std::vector<int32_t> sentinel(M, LM + 1);

    std::vector<uint32_t> h_nmark(n_sources), h_icnt;
    std::vector<int32_t> h_lin, h_lout, h_isrc, h_act;
    std::vector<unsigned long long> h_ifirst;
    int32_t n_img = 0;

    // Images of the sources with want[s] (in[] already holds the in-image
    // test): neighbours, union-find, labels, per-image counts and borders,
    // enqueued back to back (timed by events), then read back.
    auto find = [&]() -> lens_status {
        LENS_CUDA(cudaMemsetAsync(W.icnt.p, 0, (size_t)M * (LM + 1) * sizeof(uint32_t), st));
        LENS_CUDA(cudaMemcpyAsync(W.lin.p, sentinel.data(), M * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        LENS_CUDA(cudaMemcpyAsync(W.lout.p, sentinel.data(), M * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        LENS_CUDA(cudaEventRecord(W.ev[0], st));
        k_neighbours<<<blocks(n), kAmrThreads, 0, st>>>(cur->view(), n, C, W.want.p, W.nb.p);
        note_launch();
        k_uf_local<<<blocks(n), kAmrThreads, 0, st>>>(cur->view(), n, W.in.p, W.want.p, W.nb.p, W.parent.p);
        note_launch();
        k_uf_unite<<<blocks(n), kAmrThreads, 0, st>>>(cur->view(), n, W.nb.p, W.parent.p);
        note_launch();
        k_uf_roots<<<blocks(n), kAmrThreads, 0, st>>>(n, W.parent.p, W.is_root.p);
        note_launch();
        scan_exclusive_u32(W.is_root.p, W.is_root.p, n, W.total.p, W.tmp.p, st);
        k_label<<<blocks(n), kAmrThreads, 0, st>>>(cur->view(), n, C, W.parent.p, W.is_root.p, W.img.p, W.icnt.p,
                                                   W.isrc.p, W.ifirst.p, M);
        note_launch();
        k_borders<<<blocks(n), kAmrThreads, 0, st>>>(cur->view(), n, W.nb.p, W.img.p, W.lin.p, W.lout.p);
        note_launch();
        LENS_CUDA(cudaEventRecord(W.ev[1], st));
        uint32_t total = 0;
        LENS_CUDA(cudaMemcpyAsync(&total, W.total.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        const size_t ni = (size_t)M;
        h_icnt.assign(ni * (LM + 1), 0);
        h_lin.assign(ni, 0);
        h_lout.assign(ni, 0);
        h_isrc.assign(ni, 0);
        h_ifirst.assign(ni, 0);
        LENS_CUDA(cudaStreamSynchronize(st));
        if ((int64_t)total > M)
            return lens_set_error(LENS_ERR_INVALID_ARG, "image finding: %u images exceed max_images = %d", total, M);
        n_img = (int32_t)total;
        if (n_img > 0) {
            LENS_CUDA(cudaMemcpyAsync(h_icnt.data(), W.icnt.p, (size_t)n_img * (LM + 1) * sizeof(uint32_t),
                                      cudaMemcpyDeviceToHost, st));
            LENS_CUDA(cudaMemcpyAsync(h_lin.data(), W.lin.p, n_img * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            LENS_CUDA(cudaMemcpyAsync(h_lout.data(), W.lout.p, n_img * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            LENS_CUDA(cudaMemcpyAsync(h_isrc.data(), W.isrc.p, n_img * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            LENS_CUDA(cudaMemcpyAsync(h_ifirst.data(), W.ifirst.p, n_img * sizeof(unsigned long long),
                                      cudaMemcpyDeviceToHost, st));
            LENS_CUDA(cudaStreamSynchronize(st));
        }
        float ms = 0.0f;
        LENS_CUDA(cudaEventElapsedTime(&ms, W.ev[0], W.ev[1]));
        find_ms += ms;
        find_cells += n;
        return LENS_OK;
    };
    auto area_of = [&](int id) {
        double a = 0.0;
        for (int l = 0; l <= LM; ++l) {
            const double h = C.h[l];
            a += (double)h_icnt[(size_t)id * (LM + 1) + l] * (h * h);
        }
        return a;
    };

    for (;;) {
        bool all_done = true, any_img = false;
        for (int s = 0; s < n_sources; ++s) {
            all_done = all_done && mode[s] == MODE_DONE;
            const bool im = mode[s] == MODE_UNIFORM || mode[s] == MODE_BORDER;
            any_img = any_img || im;
            h_want[s] = im ? 1 : 0;
            const double r = mode[s] == MODE_TELE ? rcur[s] : rad[s];
            h_r2[s] = r * r;
            h_thr[s] = rcur[s] * smu / 3.0;
        }
        if (all_done) break;
        if (++rounds > max_rounds)
            return lens_set_error(LENS_ERR_INTERNAL, "image finding did not finish within %d rounds", max_rounds);
        LENS_CUDA(cudaMemcpyAsync(W.sr2.p, h_r2.data(), n_sources * sizeof(double), cudaMemcpyHostToDevice, st));
        LENS_CUDA(cudaMemcpyAsync(W.thr.p, h_thr.data(), n_sources * sizeof(double), cudaMemcpyHostToDevice, st));
        LENS_CUDA(cudaMemcpyAsync(W.mode.p, mode.data(), n_sources * sizeof(int), cudaMemcpyHostToDevice, st));
        LENS_CUDA(cudaMemcpyAsync(W.want.p, h_want.data(), n_sources, cudaMemcpyHostToDevice, st));
        k_inside<<<blocks(n), kAmrThreads, 0, st>>>(cur->view(), n, W.scx.p, W.scy.p, W.sr2.p, W.in.p);
        note_launch();
        k_mark_tele<<<blocks(n), kAmrThreads, 0, st>>>(cur->view(), n, C, W.in.p, W.mode.p, W.thr.p, W.mark.p);
        note_launch();
        if (any_img) {
            LENS_TRY(find());
            h_act.assign(std::max(n_img, 1), ACT_NONE);
            for (int id = 0; id < n_img; ++id) {
                const int s = h_isrc[id];
                uint32_t cells = 0;
                for (int l = 0; l <= LM; ++l) cells += h_icnt[(size_t)id * (LM + 1) + l];
                if (mode[s] == MODE_UNIFORM) {
                    if ((int64_t)cells < prm->n_min) h_act[id] = ACT_UNIFORM;
                } else if (mode[s] == MODE_BORDER) {
                    const int li = h_lin[id] > LM ? LM : h_lin[id], lo = h_lout[id] > LM ? LM : h_lout[id];
                    const int lb = std::min(li, lo);
                    const double hb = C.h[lb];
                    const bool done = (hb * hb < prm->f_area * area_of(id) && lo >= li) || lb >= LM;
                    if (!done) h_act[id] = lb;
                }
            }
            if (n_img > 0) {
                LENS_CUDA(cudaMemcpyAsync(W.act.p, h_act.data(), n_img * sizeof(int32_t), cudaMemcpyHostToDevice,
                                          st));
                k_mark_images<<<blocks(n), kAmrThreads, 0, st>>>(cur->view(), n, C, W.nb.p, W.img.p, W.act.p,
                                                                 W.mark.p);
                note_launch();
            }
        }
        LENS_CUDA(cudaMemsetAsync(W.nmark.p, 0, n_sources * sizeof(uint32_t), st));
        k_count_marks<<<blocks(n), kAmrThreads, 0, st>>>(cur->view(), n, W.mark.p, W.cnt9.p, W.rmark.p,
                                                         W.nmark.p);
        note_launch();
        LENS_CUDA(cudaMemcpyAsync(h_nmark.data(), W.nmark.p, n_sources * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                  st));
        LENS_CUDA(cudaStreamSynchronize(st));
        int64_t marks = 0;
        bool any_drop = false;
        std::fill(h_drop.begin(), h_drop.end(), (uint8_t)0);
        for (int s = 0; s < n_sources; ++s) {
            marks += h_nmark[s];
            if (h_nmark[s] != 0) continue;
            if (mode[s] == MODE_TELE) {
                if (rcur[s] <= rad[s]) {
                    mode[s] = MODE_UNIFORM;
                } else {
                    double r = rcur[s] / 3.0;
                    if (r < rad[s]) r = rad[s];
                    rcur[s] = r;
                }
            } else if (mode[s] == MODE_UNIFORM) {
                mode[s] = MODE_BORDER;
            } else if (mode[s] == MODE_BORDER) {
                // this round's images are final (its cells no longer change)
                mode[s] = MODE_DONE;
                h_drop[s] = 1;
                any_drop = true;
            }
        }
        if (any_drop) {
            for (int id = 0; id < n_img; ++id) {
                const int s = h_isrc[id];
                if (!h_drop[s]) continue;
                lens_image o{};
                o.source = s;
                uint32_t cells = 0;
                for (int l = 0; l <= LM; ++l) cells += h_icnt[(size_t)id * (LM + 1) + l];
                o.n_cells = (int32_t)cells;
                o.area = area_of(id);
                o.mu = o.area / (M_PI * rad[s] * rad[s]);
                o.first = (int64_t)(h_ifirst[id] - (unsigned long long)s * C.src_span);
                done_images[s].push_back(o);
            }
            LENS_CUDA(cudaMemcpyAsync(W.drop.p, h_drop.data(), n_sources, cudaMemcpyHostToDevice, st));
            k_drop<<<blocks(n), kAmrThreads, 0, st>>>(cur->view(), n, W.drop.p, W.cnt9.p);
            note_launch();
        }
        if (marks == 0 && !any_drop) continue;
        if (n + 8 * marks > cap)
            return lens_set_error(LENS_ERR_INVALID_ARG, "image finding needs more than max_cells = %lld cells",
                                  (long long)cap);
        scan_exclusive_u32(W.cnt9.p, W.cnt9.p, n, W.total.p, W.tmp.p, st);
        scan_exclusive_u32(W.rmark.p, W.rmark.p, n, nullptr, W.tmp.p, st);
        k_refine<<<blocks(n), kAmrThreads, 0, st>>>(cur->view(), n, C, W.mark.p, W.drop.p, W.cnt9.p, W.rmark.p,
                                                    nxt->view(), W.rx.p, W.ry.p, W.rslot.p);
        note_launch();
        uint32_t n2 = 0;
        LENS_CUDA(cudaMemcpyAsync(&n2, W.total.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        if (any_drop) {
            std::fill(h_drop.begin(), h_drop.end(), (uint8_t)0);
            LENS_CUDA(cudaMemcpyAsync(W.drop.p, h_drop.data(), n_sources, cudaMemcpyHostToDevice, st));
        }
        std::swap(cur, nxt);
        LENS_TRY(shoot(8 * marks));
        LENS_CUDA(cudaStreamSynchronize(st));
        LENS_TRY(shoot_time());
        final_cells += n + 8 * marks - (int64_t)n2;  // the dropped leaves
        n = n2;
    }

    // every source's images, recorded as it finished, by source and key
    int32_t total_img = 0;
    for (int s = 0; s < n_sources; ++s) total_img += (int32_t)done_images[s].size();
    if (total_img > max_images)
        return lens_set_error(LENS_ERR_INVALID_ARG, "%d images exceed max_images = %d", total_img, max_images);
    int32_t o = 0;
    for (int s = 0; s < n_sources; ++s)
        for (const lens_image& im : done_images[s]) images[o++] = im;
    *n_images = total_img;
    if (stats) {
        stats[0] = rays_total;
        stats[1] = final_cells;
        stats[2] = rounds;
        stats[3] = find_cells;
        stats[4] = (int64_t)std::llround(find_ms * 1e6);
        stats[5] = (int64_t)std::llround(shoot_ms * 1e6);
    }
    LENS_CUDA(cudaGetLastError());
    return LENS_OK;
}
