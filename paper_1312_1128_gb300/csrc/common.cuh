// common.cuh -- shared definitions of liblens's CUDA sources (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "lens.h"

#define LENS_DEV __device__ __forceinline__
#define LENS_HD __host__ __device__ __forceinline__

// Device error word bits, latched with atomicOr and read by lens_sync_status.
enum : uint32_t {
    DERR_STACK_OVERFLOW = 1u,   // walk stack capacity exceeded (cannot happen by construction)
    DERR_BAD_INPUT = 2u,        // negative / non-finite mass or size in the input
    DERR_INDEX = 4u,            // an index check in a kernel failed
    DERR_BUFFER = 8u,           // an interaction buffer check failed
    DERR_WAIT_TIMEOUT = 16u     // a bounded wait between cooperating warps gave up
};

// Morton keys: 24 levels of 2 bits below the root.
constexpr int kMaxDepth = 24;
constexpr int kKeyBits = 2 * kMaxDepth;

// Walk geometry.
constexpr int kWalkWarps = 4;          // warps per block in the walk kernels
constexpr int kStackCap = 4096;        // node entries per warp stack (bound: 128 per level + 128)
constexpr int kFarCap = 64;            // far-cell buffer entries per warp
constexpr int kNearCap = 128;          // near-particle buffer entries per warp
constexpr int kBigCap = 128;           // big-list buffer entries per warp
constexpr int kMaxRaysPerLane = 4;     // rays per lane in the walk (32-, 64- or 128-ray groups)

// 32-byte aligned four-double record (CUDA 13 deprecates the plain double4).
struct alignas(32) dbl4 {
    double x, y, z, w;
};
LENS_HD dbl4 make_dbl4(double x, double y, double z, double w) { return dbl4{x, y, z, w}; }

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = dbl4; };
template <typename T> using vec4_t = typename Vec4<T>::type;

LENS_DEV uint32_t lane_id() { return threadIdx.x & 31u; }
LENS_DEV uint32_t lanemask_lt() { return (1u << lane_id()) - 1u; }

// Exclusive warp prefix sum of v; total returned through *tot.
LENS_DEV int warp_exclusive_scan(int v, int* tot)
{
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane_id() >= o) x += y;
    }
    *tot = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// Order-preserving map of a double to uint64 (for atomic min/max).
LENS_HD unsigned long long dbl_to_ordered(double d)
{
    unsigned long long u = *reinterpret_cast<unsigned long long*>(&d);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
LENS_HD double ordered_to_dbl(unsigned long long u)
{
    u = (u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u;
    return *reinterpret_cast<double*>(&u);
}

// Host-side helpers (defined in api.cu).
// Every device allocation of the library goes through these two, so that the
// failure-injection hook (lens_fail_allocations) can fail the n-th one.
cudaError_t lens_malloc(void** p, size_t bytes);
cudaError_t lens_malloc_async(void** p, size_t bytes, cudaStream_t s);
void note_launch();  // counts every kernel launch made by the library
void note_launches(int64_t n);  // adds n launches (a graph replay), or takes back -n
lens_status lens_set_error(lens_status s, const char* fmt, ...);
lens_status lens_cuda_check(cudaError_t e, const char* what);

#define LENS_CUDA(call)                                                        \
    do {                                                                       \
        cudaError_t _e = (call);                                               \
        if (_e != cudaSuccess) return lens_cuda_check(_e, #call);              \
    } while (0)

#define LENS_TRY(call)                                                         \
    do {                                                                       \
        lens_status _s = (call);                                               \
        if (_s != LENS_OK) return _s;                                          \
    } while (0)

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

// Stream-ordered temporaries of one call, released on every return path
// (an allocation that fails part-way through leaves nothing behind).
struct StreamTemps {
    cudaStream_t s;
    std::vector<void*> p;
    explicit StreamTemps(cudaStream_t st) : s(st) {}
    StreamTemps(const StreamTemps&) = delete;
    StreamTemps& operator=(const StreamTemps&) = delete;
    ~StreamTemps() { release_all(); }
    template <typename P> cudaError_t get(P** out, size_t bytes)
    {
        void* q = nullptr;
        cudaError_t e = lens_malloc_async(&q, bytes, s);
        if (e == cudaSuccess) p.push_back(q);
        *out = (P*)q;
        return e;
    }
    void release(void* q)
    {
        for (auto& x : p)
            if (x == q && x) {
                cudaFreeAsync(x, s);
                x = nullptr;
            }
    }
    void release_all()
    {
        for (auto& x : p)
            if (x) cudaFreeAsync(x, s);
        p.clear();
    }
};

