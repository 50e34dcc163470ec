// sort.cu -- device-wide exclusive scan and stable LSD radix sort of
// (key, value) pairs, used by the tree build (Morton order, level order,
// big-list grouping) and by ray grouping.  Hand-written; no CUB/Thrust.
#include "common.cuh"
#include "sort.cuh"

namespace lens {

// ------------------------------------------------------------------ scan

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan across the block; *total (shared) receives the block sum.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total)
{
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
        uint32_t s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = s - t;
        if (lane == kScanThreads / 32 - 1) *total = s;
    }
    __syncthreads();
    uint32_t r = warp_tot[wid] + x - v;
    __syncthreads();
    return r;
}

__global__ void scan_reduce_kernel(const uint32_t* in, int64_t n, uint32_t* block_sums)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    __shared__ uint32_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// Each thread owns kScanItems consecutive elements.
__global__ void scan_apply_kernel(const uint32_t* in, uint32_t* out, int64_t n,
                                  const uint32_t* block_offsets, uint32_t* total_out, int64_t nblocks)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0u;
        s += v[i];
    }
    __shared__ uint32_t tot;
    uint32_t run = block_exclusive_scan(s, &tot) + (block_offsets ? block_offsets[blockIdx.x] : 0u);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (total_out && blockIdx.x == nblocks - 1 && threadIdx.x == 0)
        *total_out = (block_offsets ? block_offsets[blockIdx.x] : 0u) + tot;
}

size_t scan_temp_bytes(int64_t n)
{
    size_t bytes = 0;
    while (n > kScanTile) {
        int64_t nb = (n + kScanTile - 1) / kScanTile;
        bytes += ((size_t)nb * sizeof(uint32_t) + 255) & ~(size_t)255;
        n = nb;
    }
    return bytes + 256;
}

// Exclusive scan of n uint32 (in-place allowed).  total (device, optional)
// receives the sum.  tmp must hold scan_temp_bytes(n).
void scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total,
                        void* tmp, cudaStream_t s)
{
    if (n <= 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
        return;
    }
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        { scan_apply_kernel<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, total, 1); note_launch(); }
        return;
    }
    uint32_t* sums = (uint32_t*)tmp;
    void* rest = (char*)tmp + (((size_t)nb * sizeof(uint32_t) + 255) & ~(size_t)255);
    { scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums); note_launch(); }
    scan_exclusive_u32(sums, sums, nb, nullptr, rest, s);
    { scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums, total, nb); note_launch(); }
}

// ------------------------------------------------------------ radix sort

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadix = 256;

template <typename K>
__global__ void radix_hist_kernel(const K* keys, int64_t n, int shift, uint32_t* hist, int64_t nblocks)
{
    __shared__ uint32_t cnt[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) cnt[d] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        int64_t idx = base + (int64_t)r * kSortThreads + threadIdx.x;
        if (idx < n) atomicAdd(&cnt[(uint32_t)(keys[idx] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads)
        hist[(int64_t)d * nblocks + blockIdx.x] = cnt[d];
}

// Exclusive scan of one digit's counts over the tiles (block d scans
// hist[d * nblocks ...]), in place; the digit's total goes to digit_tot[d].
__global__ void __launch_bounds__(kScanThreads) radix_colscan_kernel(uint32_t* hist, int64_t nblocks,
                                                                       uint32_t* digit_tot)
{
    uint32_t* col = hist + (int64_t)blockIdx.x * nblocks;
    __shared__ uint32_t tot;
    uint32_t run = 0;
    for (int64_t base = 0; base < nblocks; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = i < nblocks ? col[i] : 0u;
        const uint32_t ex = block_exclusive_scan(v, &tot);
        if (i < nblocks) col[i] = run + ex;
        run += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) digit_tot[blockIdx.x] = run;
}

// Stable scatter.  Warp w of the block holds elements [w, w + 1) * 32 *
// kSortItems of the tile, round r its 32 elements from r * 32, so (warp,
// round, lane) is the elements' index order.  Each warp ranks its elements
// among its own equal digits (match_any per round, running counts in a
// warp-private shared histogram); one scan over (digit, warp) then gives each
// element its place in the tile ordered by digit, equal digits in index
// order.  The ordered tile is written out so that a digit's run of the tile
// goes to consecutive output positions and the stores coalesce.
template <typename K>
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const K* kin, const uint32_t* vin, K* kout,
                                                                     uint32_t* vout, int64_t n, int shift,
                                                                     const uint32_t* offs, const uint32_t* digit_tot,
                                                                     int64_t nblocks, uint32_t* err)
{
    constexpr int kWarps = kSortThreads / 32;
    static_assert(kSortThreads == kRadix && kSortThreads == kScanThreads, "one thread per digit");
    __shared__ K sk[kSortTile];
    __shared__ uint32_t sv[kSortTile];
    __shared__ uint32_t wcnt[kWarps][kRadix];  // a warp's digit counts, then its start within the digit's run
    __shared__ uint32_t tstart[kRadix];        // the digit's start in the ordered tile
    __shared__ uint32_t base_off[kRadix];      // the digit's first output position for this tile
    __shared__ uint32_t scan_tot;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const int tile_n = (int)(n - base < kSortTile ? n - base : kSortTile);
    const int d_own = threadIdx.x;  // the digit this thread scans
    for (int w = 0; w < kWarps; ++w) wcnt[w][d_own] = 0;
    // the digits' global starts plus this tile's place among the tiles of each digit
    const uint32_t gstart = block_exclusive_scan(digit_tot[d_own], &scan_tot);
    base_off[d_own] = gstart + offs[(int64_t)d_own * nblocks + blockIdx.x];
    __syncthreads();
    K key[kSortItems];
    uint32_t val[kSortItems], lrank[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int e = wid * 32 * kSortItems + r * 32 + lane;
        const bool valid = e < tile_n;
        key[r] = valid ? kin[base + e] : K(0);
        val[r] = valid ? vin[base + e] : 0u;
        const uint32_t d = valid ? ((uint32_t)(key[r] >> shift) & 0xffu) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t prev = valid ? wcnt[wid][d] : 0u;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[wid][d] = prev + __popc(peers);
        __syncwarp();
        lrank[r] = prev + __popc(peers & ((1u << lane) - 1u));
    }
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = wcnt[w][d_own];
        wcnt[w][d_own] = tot;
        tot += c;
    }
    tstart[d_own] = block_exclusive_scan(tot, &scan_tot);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int e = wid * 32 * kSortItems + r * 32 + lane;
        if (e < tile_n) {
            const uint32_t d = (uint32_t)(key[r] >> shift) & 0xffu;
            const uint32_t tp = tstart[d] + wcnt[wid][d] + lrank[r];
            if (tp >= (uint32_t)tile_n) {  // cannot happen: the ranks are a permutation of the tile
                if (err) atomicOr(err, DERR_INDEX);
                continue;
            }
            sk[tp] = key[r];
            sv[tp] = val[r];
        }
    }
    __syncthreads();
    // out in digit order: element e of the ordered tile has digit d and goes to
    // base_off[d] + (e - tstart[d])
    for (int e = threadIdx.x; e < tile_n; e += kSortThreads) {
        const K k = sk[e];
        const uint32_t d = (uint32_t)(k >> shift) & 0xffu;
        const uint32_t pos = base_off[d] + (uint32_t)e - tstart[d];
        if ((int64_t)pos >= n) {  // cannot happen: the offsets are a scan of the histogram
            if (err) atomicOr(err, DERR_INDEX);
            continue;
        }
        kout[pos] = k;
        vout[pos] = sv[e];
    }
}

template <typename K>
size_t radix_sort_temp_bytes(int64_t n)
{
    int64_t nb = (n + kSortTile - 1) / kSortTile;
    size_t hist = ((size_t)nb * kRadix * sizeof(uint32_t) + 255) & ~(size_t)255;
    return hist + kRadix * sizeof(uint32_t) + 256;
}

#ifdef LENS_SORT_DEBUG
__global__ void k_perm_mark(const uint32_t* v, int64_t n, uint32_t* bits, uint32_t* err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t x = v[i];
    if ((int64_t)x >= n) { atomicOr(err, DERR_BUFFER); return; }
    const uint32_t old = atomicOr(bits + (x >> 5), 1u << (x & 31));
    if (old & (1u << (x & 31))) atomicOr(err, DERR_BUFFER);
}
#endif

// Sort (keys, vals) by bits [begin_bit, end_bit) of the key.  Uses the
// alternate buffers; on return *kres / *vres point at the sorted data (one of
// the two buffers).  n must be < 2^32.
template <typename K>
void radix_sort_pairs(K* k0, uint32_t* v0, K* k1, uint32_t* v1, int64_t n, int begin_bit,
                      int end_bit, void* tmp, cudaStream_t s, K** kres, uint32_t** vres, uint32_t* err)
{
    K* ki = k0; uint32_t* vi = v0;
    K* ko = k1; uint32_t* vo = v1;
    if (n > 1) {
        int64_t nb = (n + kSortTile - 1) / kSortTile;
        uint32_t* hist = (uint32_t*)tmp;
        uint32_t* dtot = (uint32_t*)((char*)tmp + (((size_t)nb * kRadix * sizeof(uint32_t) + 255) & ~(size_t)255));
        for (int b = begin_bit; b < end_bit; b += 8) {
            { radix_hist_kernel<K><<<(unsigned)nb, kSortThreads, 0, s>>>(ki, n, b, hist, nb); note_launch(); }
            { radix_colscan_kernel<<<kRadix, kScanThreads, 0, s>>>(hist, nb, dtot); note_launch(); }
            { radix_scatter_kernel<K><<<(unsigned)nb, kSortThreads, 0, s>>>(ki, vi, ko, vo, n, b, hist, dtot, nb,
                                                                                err);
              note_launch(); }
            K* tk = ki; ki = ko; ko = tk;
            uint32_t* tv = vi; vi = vo; vo = tv;
        }
    }
#ifdef LENS_SORT_DEBUG
    if (n > 1 && err) {
        // every caller sorts an index array 0..n-1: check that a permutation comes out
        uint32_t* bits = nullptr;
        cudaMallocAsync((void**)&bits, ((n + 31) / 32) * 4, s);
        cudaMemsetAsync(bits, 0, ((n + 31) / 32) * 4, s);
        k_perm_mark<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(vi, n, bits, err);
        cudaFreeAsync(bits, s);
    }
#endif
    *kres = ki;
    *vres = vi;
}

template size_t radix_sort_temp_bytes<uint64_t>(int64_t);
template size_t radix_sort_temp_bytes<uint32_t>(int64_t);
template void radix_sort_pairs<uint64_t>(uint64_t*, uint32_t*, uint64_t*, uint32_t*, int64_t, int, int,
                                         void*, cudaStream_t, uint64_t**, uint32_t**, uint32_t*);
template void radix_sort_pairs<uint32_t>(uint32_t*, uint32_t*, uint32_t*, uint32_t*, int64_t, int, int,
                                         void*, cudaStream_t, uint32_t**, uint32_t**, uint32_t*);

}  // namespace lens
