// api.cu -- the C ABI of liblens (include/lens.h): argument checking, tree
// ownership, error reporting and the FP32 / FP64 peak microbenchmarks.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <string>

#include "tree.cuh"

namespace lens {
lens_status shoot(lens_tree* t, int64_t nb, const int64_t* h_off, const double* h_orig, const void* dx,
                  const void* dy, int dtype, void* const out[5], int flags, cudaStream_t s);
lens_status reserve_rays(lens_tree* t, int64_t n, int64_t nb, cudaStream_t s);
lens_status shoot_backward(lens_tree* t, double ox, double oy, const void* dx, const void* dy,
                           int dtype, int64_t n, const void* const g[5], void* const* g_species,
                           void* g_halos, int flags, cudaStream_t s);
lens_status graph_shoot_batches(lens_tree* t, int64_t nb, const int64_t* off, const double* orig,
                                const void* dx, const void* dy, int dtype, void* const out[5],
                                int flags, cudaStream_t s);
void free_graphs(lens_tree* t);
bool halos_only(const lens_tree* t);
lens_status shoot_halos_only(lens_tree* t, double ox, double oy, const void* dx, const void* dy, int dtype,
                             int64_t n, void* const out[5], int flags, cudaStream_t s);
lens_status noalloc_scratch_address(void** out);
}  // namespace lens

static thread_local char g_msg[512] = "";
static std::atomic<long long> g_launches{0};

static std::atomic<long long> g_fail_after{-1};

// The failure-injection hook: true if this allocation is the one to fail.
static bool alloc_should_fail()
{
    long long c = g_fail_after.load();
    while (c >= 0) {
        if (g_fail_after.compare_exchange_weak(c, c - 1)) return c == 0;
    }
    return false;
}

cudaError_t lens_malloc(void** p, size_t bytes)
{
    if (alloc_should_fail()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t lens_malloc_async(void** p, size_t bytes, cudaStream_t s)
{
    if (alloc_should_fail()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, s);
}

extern "C" void lens_fail_allocations(int64_t after) { g_fail_after.store(after < 0 ? -1 : (long long)after); }

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

lens_status lens_set_error(lens_status s, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return s;
}

lens_status lens_cuda_check(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return lens_set_error(LENS_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return lens_set_error(LENS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

using namespace lens;

// Projected NFW shape functions at X = R_max / r_s (Sec. 3.2): F, the
// surface-density shape f = (1 - F)/(X^2 - 1) and the enclosed-mass shape
// g = ln(X/2) + F; near X = 1 both F and f are power series in u = 1 - X^2.
static void nfw_host(double X, double* Fo, double* fo, double* go)
{
    double u = 1.0 - X * X, F, f;
    if (std::fabs(u) < 1e-2) {
        double s = 0.0, t = 0.0;
        for (int k = 16; k >= 0; --k) {
            s = s * u + 1.0 / (2 * k + 1);
            t = t * u + 1.0 / (2 * k + 3);
        }
        F = s;
        f = t;
    } else {
        F = X < 1.0 ? std::acosh(1.0 / X) / std::sqrt(u) : std::acos(1.0 / X) / std::sqrt(-u);
        f = (1.0 - F) / (X * X - 1.0);
    }
    *Fo = F;
    *fo = f;
    *go = std::log(0.5 * X) + F;
}

static lens_status check_halo(const lens_halo& h, HaloDev& d)
{
    d = HaloDev{};
    d.kind = h.kind;
    d.x = h.x; d.y = h.y; d.m = h.m; d.p0 = h.p0; d.p1 = h.p1;
    bool fin = std::isfinite(h.x) && std::isfinite(h.y) && std::isfinite(h.m) && std::isfinite(h.p0) &&
               std::isfinite(h.p1);
    if (!fin) return lens_set_error(LENS_ERR_INVALID_ARG, "halo with non-finite field");
    switch (h.kind) {
    case LENS_POINT:
        return LENS_OK;
    case LENS_GAUSS:
        if (!(h.p0 > 0 && h.p1 > 0)) return lens_set_error(LENS_ERR_INVALID_ARG, "Gaussian halo needs r_sm > 0, q > 0");
        d.c0 = 1.0 / (2.0 * h.p0 * h.p0);
        d.c1 = 0.5 * h.p1 * h.p1;
        d.c2 = 1.0 / (-std::expm1(-d.c1));
        return LENS_OK;
    case LENS_NFW:
        if (!(h.p0 > 0 && h.p1 > 0)) return lens_set_error(LENS_ERR_INVALID_ARG, "NFW halo needs r_s > 0, R_max > 0");
    {
        double X = h.p1 / h.p0, F, f, g;
        nfw_host(X, &F, &f, &g);
        d.c0 = h.m / g;
        d.c1 = 1.0 / h.p0;
        d.c2 = h.p1 * h.p1;
        d.c3 = X * f / g;
        return LENS_OK;
    }
    case LENS_SIS:
        if (!(h.p0 >= 0)) return lens_set_error(LENS_ERR_INVALID_ARG, "SIS halo needs r_E >= 0");
        return LENS_OK;
    case LENS_DISK:
        if (!(h.p0 > 0)) return lens_set_error(LENS_ERR_INVALID_ARG, "disk halo needs R > 0");
        d.c2 = h.p0 * h.p0;
        return LENS_OK;
    }
    return lens_set_error(LENS_ERR_INVALID_ARG, "unknown halo kind %d", h.kind);
}

extern "C" {

int32_t lens_api_version(void) { return LENS_API_VERSION; }

int64_t lens_kernel_launches(void) { return (int64_t)g_launches.load(); }

const char* lens_last_error(void) { return g_msg; }

const char* lens_status_string(lens_status s)
{
    switch (s) {
    case LENS_OK: return "ok";
    case LENS_ERR_INVALID_ARG: return "invalid argument";
    case LENS_ERR_CUDA: return "CUDA error";
    case LENS_ERR_OOM: return "out of device memory";
    case LENS_ERR_TIMEOUT: return "bounded device wait expired";
    case LENS_ERR_INTERNAL: return "internal consistency check failed";
    case LENS_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

void lens_free_tree(lens_tree* t)
{
    if (!t) return;
    cudaDeviceSynchronize();  // no kernel of this tree may still be running
    free_graphs(t);
    for (auto& st : t->sp) free_species(st);
    if (t->halos) cudaFree(t->halos);
    if (t->d_err) cudaFree(t->d_err);
    if (t->ray_scratch.ptr) cudaFreeAsync(t->ray_scratch.ptr, 0);
    if (t->d_stats) cudaFree(t->d_stats);
    if (t->list_ids) cudaFreeAsync(t->list_ids, 0);
    if (t->list_n) cudaFreeAsync(t->list_n, 0);
    if (t->amr_ws && t->amr_free) t->amr_free(t->amr_ws);
    for (int i = 0; i < 4; ++i)
        if (t->ev[i]) cudaEventDestroy(t->ev[i]);
    if (t->built) cudaEventDestroy(t->built);
    delete t;
}

lens_status lens_build_tree(const lens_species* species, int32_t n_species, const lens_halo* halos,
                            int64_t n_halos, const lens_params* params, void* stream, lens_tree** out)
{
    if (!out) return lens_set_error(LENS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!params) return lens_set_error(LENS_ERR_INVALID_ARG, "params is NULL");
    if (n_species < 0 || n_species > 8) return lens_set_error(LENS_ERR_INVALID_ARG, "n_species must be 0..8");
    if (n_species > 0 && !species) return lens_set_error(LENS_ERR_INVALID_ARG, "species is NULL");
    if (n_halos < 0 || (n_halos > 0 && !halos)) return lens_set_error(LENS_ERR_INVALID_ARG, "bad halos");
    if (!(params->theta >= 0.0) || !std::isfinite(params->theta))
        return lens_set_error(LENS_ERR_INVALID_ARG, "theta must be finite and >= 0");
    if (params->leaf_max < 1 || params->leaf_max > 64)
        return lens_set_error(LENS_ERR_INVALID_ARG, "leaf_max must be in 1..64");
    if (params->precision != LENS_PREC_FP32 && params->precision != LENS_PREC_FP64)
        return lens_set_error(LENS_ERR_INVALID_ARG, "unknown precision %d", params->precision);
    if (params->group_rays != 0 && params->group_rays != 32 && params->group_rays != 64 && params->group_rays != 128)
        return lens_set_error(LENS_ERR_INVALID_ARG, "group_rays must be 0, 32, 64 or 128");
    if (params->walk < LENS_WALK_DEFAULT || params->walk > LENS_WALK_TRIOS)
        return lens_set_error(LENS_ERR_INVALID_ARG, "walk must be LENS_WALK_DEFAULT, _WARP, _PAIRS or _TRIOS");
    if (params->tile < LENS_TILE_DEFAULT || params->tile > LENS_TILE_LARGE)
        return lens_set_error(LENS_ERR_INVALID_ARG, "tile must be LENS_TILE_DEFAULT, _STANDARD or _LARGE");
    for (int i = 0; i < n_species; ++i) {
        const lens_species& s = species[i];
        if (s.kind != LENS_POINT && s.kind != LENS_GAUSS && s.kind != LENS_NFW)
            return lens_set_error(LENS_ERR_INVALID_ARG, "species %d: kind must be POINT, GAUSS or NFW", i);
        if (s.dtype != LENS_F32 && s.dtype != LENS_F64)
            return lens_set_error(LENS_ERR_INVALID_ARG, "species %d: bad dtype", i);
        if (s.n < 0 || s.n >= (1ll << 30))
            return lens_set_error(LENS_ERR_INVALID_ARG, "species %d: n must be in [0, 2^30)", i);
        if (s.n > 0 && !s.data) return lens_set_error(LENS_ERR_INVALID_ARG, "species %d: data is NULL", i);
        if (s.kind != LENS_POINT && !(s.shape > 0.0 && std::isfinite(s.shape)))
            return lens_set_error(LENS_ERR_INVALID_ARG, "species %d: shape must be > 0", i);
    }
    std::vector<HaloDev> hd((size_t)n_halos);
    for (int64_t i = 0; i < n_halos; ++i) LENS_TRY(check_halo(halos[i], hd[i]));

    lens_tree* t = new lens_tree();
    t->precision = params->precision;
    t->theta = params->theta;
    t->leaf_max = params->leaf_max;
    t->group_rays = params->group_rays == 0 ? 32 : params->group_rays;
    t->walk_mode = params->walk == LENS_WALK_DEFAULT ? LENS_WALK_WARP : params->walk;
    t->walk_fixed = params->walk != LENS_WALK_DEFAULT;
    t->tile = params->tile == LENS_TILE_LARGE && params->precision == LENS_PREC_FP32 ? 1 : 0;
    t->tile_fixed = params->tile != LENS_TILE_DEFAULT;
    cudaStream_t s = (cudaStream_t)stream;
    auto fail = [&](lens_status st) {
        lens_free_tree(t);
        return st;
    };
    cudaError_t e = cudaGetDevice(&t->device);
    if (e != cudaSuccess) return fail(lens_cuda_check(e, "cudaGetDevice"));
    {
        // Tree arrays and ray scratch come from the device's stream-ordered
        // pool; keep freed blocks in the pool so rebuilding a lens allocates
        // at pool speed instead of cudaMalloc speed.
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, t->device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    e = cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, t->device);
    if (e != cudaSuccess) return fail(lens_cuda_check(e, "cudaDeviceGetAttribute"));
    e = lens_malloc((void**)&t->d_err, sizeof(uint32_t));
    if (e != cudaSuccess) return fail(lens_cuda_check(e, "cudaMalloc(err)"));
    e = cudaMemsetAsync(t->d_err, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return fail(lens_cuda_check(e, "cudaMemsetAsync"));
    e = lens_malloc((void**)&t->d_stats, 9 * sizeof(unsigned long long));
    if (e != cudaSuccess) return fail(lens_cuda_check(e, "cudaMalloc(stats)"));
    e = cudaMemsetAsync(t->d_stats, 0, 9 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return fail(lens_cuda_check(e, "cudaMemsetAsync"));
    t->halos_host.assign(halos, halos + n_halos);
    t->n_halos = n_halos;
    if (n_halos > 0) {
        e = lens_malloc((void**)&t->halos, n_halos * sizeof(HaloDev));
        if (e != cudaSuccess) return fail(lens_cuda_check(e, "cudaMalloc(halos)"));
        e = cudaMemcpy(t->halos, hd.data(), n_halos * sizeof(HaloDev), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(lens_cuda_check(e, "cudaMemcpy(halos)"));
    }
    t->sp.resize(n_species);
    for (int i = 0; i < n_species; ++i) {
        lens_status st = build_species(t, t->sp[i], species[i], s);
        if (st != LENS_OK) return fail(st);
    }
    // no synchronisation here: each species' build waited once for its node
    // count (and its input check); the rest runs on in stream order, and a
    // device-side check that fails later is reported by lens_sync_status
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(lens_cuda_check(e, "tree build"));
    e = cudaEventCreateWithFlags(&t->built, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(t->built, s);
    if (e != cudaSuccess) return fail(lens_cuda_check(e, "cudaEventRecord(built)"));
    // the allocation-free shoot's scratch: its address on this device, taken
    // here (the first lookup on a device loads the array) so that the shoot
    // call itself makes no runtime lookup
    {
        lens_status st = noalloc_scratch_address(&t->noalloc_scratch);
        if (st != LENS_OK) return fail(st);
    }
    *out = t;
    return LENS_OK;
}

static lens_status check_outputs(const lens_tree* t, void* a1, void* a2, void* k, void* g1, void* g2,
                                 int32_t flags, int64_t n)
{
    if (!t) return lens_set_error(LENS_ERR_INVALID_ARG, "tree is NULL");
    if (flags & ~(LENS_ALPHA_ONLY | LENS_DIRECT | LENS_ACCUMULATE | LENS_USE_GRAPH | LENS_COUNT | LENS_TIMING |
                  LENS_KEEP_LISTS))
        return lens_set_error(LENS_ERR_INVALID_ARG, "unknown flag bits");
    if (n < 0 || n >= (1ll << 31)) return lens_set_error(LENS_ERR_INVALID_ARG, "n must be in [0, 2^31)");
    if (n == 0) return LENS_OK;
    if (!a1 || !a2) return lens_set_error(LENS_ERR_INVALID_ARG, "alpha outputs are NULL");
    if (!(flags & LENS_ALPHA_ONLY) && (!k || !g1 || !g2))
        return lens_set_error(LENS_ERR_INVALID_ARG, "kappa/gamma outputs are NULL without LENS_ALPHA_ONLY");
    return LENS_OK;
}

lens_status lens_shoot_rays(lens_tree* tree, double origin_x, double origin_y, const void* ray_dx,
                            const void* ray_dy, int32_t ray_dtype, int64_t n, void* alpha1, void* alpha2,
                            void* kappa, void* gamma1, void* gamma2, int32_t flags, void* stream)
{
    LENS_TRY(check_outputs(tree, alpha1, alpha2, kappa, gamma1, gamma2, flags, n));
    if (flags & LENS_USE_GRAPH) return lens_set_error(LENS_ERR_INVALID_ARG, "LENS_USE_GRAPH is for lens_shoot_batches");
    if (ray_dtype != LENS_F32 && ray_dtype != LENS_F64) return lens_set_error(LENS_ERR_INVALID_ARG, "bad ray dtype");
    if (!std::isfinite(origin_x) || !std::isfinite(origin_y))
        return lens_set_error(LENS_ERR_INVALID_ARG, "origin must be finite");
    if (n == 0) return LENS_OK;
    if (!ray_dx || !ray_dy) return lens_set_error(LENS_ERR_INVALID_ARG, "ray arrays are NULL");
    int64_t off[2] = {0, n};
    double orig[2] = {origin_x, origin_y};
    void* out[5] = {alpha1, alpha2, kappa, gamma1, gamma2};
    // analytic components only: one thread per ray, no grouping or walk
    if (!(flags & (LENS_TIMING | LENS_COUNT)) && halos_only(tree))
        return shoot_halos_only(tree, origin_x, origin_y, ray_dx, ray_dy, ray_dtype, n, out, flags,
                                (cudaStream_t)stream);
    return shoot(tree, 1, off, orig, ray_dx, ray_dy, ray_dtype, out, flags, (cudaStream_t)stream);
}

static lens_status check_batches(int64_t n_batches, const int64_t* offsets, const double* origins)
{
    if (n_batches < 0 || n_batches > (1 << 24)) return lens_set_error(LENS_ERR_INVALID_ARG, "bad n_batches");
    if (!offsets) return lens_set_error(LENS_ERR_INVALID_ARG, "offsets is NULL");
    if (n_batches > 0 && !origins) return lens_set_error(LENS_ERR_INVALID_ARG, "origins is NULL");
    if (offsets[0] != 0) return lens_set_error(LENS_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (int64_t b = 0; b < n_batches; ++b) {
        if (offsets[b + 1] < offsets[b]) return lens_set_error(LENS_ERR_INVALID_ARG, "offsets must be non-decreasing");
        if (!std::isfinite(origins[2 * b]) || !std::isfinite(origins[2 * b + 1]))
            return lens_set_error(LENS_ERR_INVALID_ARG, "origins must be finite");
    }
    return LENS_OK;
}

lens_status lens_shoot_batches(lens_tree* tree, int64_t n_batches, const int64_t* offsets,
                               const double* origins, const void* ray_dx, const void* ray_dy,
                               int32_t ray_dtype, void* alpha1, void* alpha2, void* kappa, void* gamma1,
                               void* gamma2, int32_t flags, void* stream)
{
    LENS_TRY(check_batches(n_batches, offsets, origins));
    int64_t n = offsets[n_batches];
    LENS_TRY(check_outputs(tree, alpha1, alpha2, kappa, gamma1, gamma2, flags, n));
    if (flags & LENS_KEEP_LISTS) return lens_set_error(LENS_ERR_INVALID_ARG, "LENS_KEEP_LISTS is for lens_shoot_rays");
    if (ray_dtype != LENS_F32 && ray_dtype != LENS_F64) return lens_set_error(LENS_ERR_INVALID_ARG, "bad ray dtype");
    if (n == 0) return LENS_OK;
    if (!ray_dx || !ray_dy) return lens_set_error(LENS_ERR_INVALID_ARG, "ray arrays are NULL");
    void* out[5] = {alpha1, alpha2, kappa, gamma1, gamma2};
    if ((flags & LENS_USE_GRAPH) && (flags & LENS_TIMING))
        return lens_set_error(LENS_ERR_INVALID_ARG, "LENS_TIMING cannot be combined with LENS_USE_GRAPH; "
                                                    "time a replay with events on the caller's stream");
    if (flags & LENS_USE_GRAPH)
        return graph_shoot_batches(tree, n_batches, offsets, origins, ray_dx, ray_dy, ray_dtype, out,
                                   flags & ~LENS_USE_GRAPH, (cudaStream_t)stream);
    return shoot(tree, n_batches, offsets, origins, ray_dx, ray_dy, ray_dtype, out, flags, (cudaStream_t)stream);
}

lens_status lens_shoot_rays_backward(lens_tree* tree, double origin_x, double origin_y, const void* ray_dx,
                                     const void* ray_dy, int32_t ray_dtype, int64_t n, const void* g_alpha1,
                                     const void* g_alpha2, const void* g_kappa, const void* g_gamma1,
                                     const void* g_gamma2, void* const* g_species, void* g_halos,
                                     int32_t flags, void* stream)
{
    if (!tree) return lens_set_error(LENS_ERR_INVALID_ARG, "tree is NULL");
    if (flags & ~(LENS_DIRECT | LENS_KEEP_LISTS))
        return lens_set_error(LENS_ERR_INVALID_ARG, "backward accepts LENS_DIRECT and LENS_KEEP_LISTS only");
    if (n < 0 || n >= (1ll << 31)) return lens_set_error(LENS_ERR_INVALID_ARG, "n must be in [0, 2^31)");
    if (g_kappa || g_gamma1 || g_gamma2)
        return lens_set_error(LENS_ERR_UNSUPPORTED, "gradients of kappa and gamma are not implemented");
    if (ray_dtype != LENS_F32 && ray_dtype != LENS_F64) return lens_set_error(LENS_ERR_INVALID_ARG, "bad ray dtype");
    if (n == 0) return LENS_OK;
    if (!ray_dx || !ray_dy || !g_alpha1 || !g_alpha2) return lens_set_error(LENS_ERR_INVALID_ARG, "NULL array");
    if (tree->sp.size() > 0 && !g_species) return lens_set_error(LENS_ERR_INVALID_ARG, "g_species is NULL");
    const void* g[5] = {g_alpha1, g_alpha2, nullptr, nullptr, nullptr};
    return shoot_backward(tree, origin_x, origin_y, ray_dx, ray_dy, ray_dtype, n, g, g_species, g_halos,
                          flags, (cudaStream_t)stream);
}

lens_status lens_autotune(lens_tree* tree, double origin_x, double origin_y, const void* ray_dx,
                          const void* ray_dy, int32_t ray_dtype, int64_t n, void* stream,
                          int32_t* group_rays)
{
    if (!tree || !group_rays) return lens_set_error(LENS_ERR_INVALID_ARG, "NULL argument");
    if (ray_dtype != LENS_F32 && ray_dtype != LENS_F64) return lens_set_error(LENS_ERR_INVALID_ARG, "bad ray dtype");
    if (n <= 0 || !ray_dx || !ray_dy) return lens_set_error(LENS_ERR_INVALID_ARG, "no rays to tune on");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t m = n < (1 << 23) ? n : (1 << 23);
    size_t es = tree->precision == LENS_PREC_FP64 ? 8 : 4;
    void* buf = nullptr;
    LENS_CUDA(lens_malloc_async(&buf, 5 * m * es, s));
    void* out[5];
    for (int q = 0; q < 5; ++q) out[q] = (char*)buf + q * m * es;
    int64_t off[2] = {0, m};
    double orig[2] = {origin_x, origin_y};
    // candidates: group size x walk form x near-field tile (the walk form and
    // the tile only if the caller left them open; the large tile serves the
    // one-warp FP32 walk)
    // (128-ray groups: the one-warp walk only)
    const int cand_g[8] = {32, 64, 32, 64, 64, 32, 64, 128};
    const int cand_w[8] = {LENS_WALK_WARP, LENS_WALK_WARP, LENS_WALK_PAIRS, LENS_WALK_PAIRS, LENS_WALK_TRIOS,
                           LENS_WALK_WARP, LENS_WALK_WARP, LENS_WALK_WARP};
    const int cand_t[8] = {0, 0, 0, 0, 0, 1, 1, 0};
    double best = 1e300;
    int best_g = tree->group_rays, best_w = tree->walk_mode, best_t = tree->tile;
    const int user_w = tree->walk_mode, user_t = tree->tile;
    lens_status st = LENS_OK;
    for (int c = 0; c < 8 && st == LENS_OK; ++c) {
        if (tree->precision == LENS_PREC_FP64 && (cand_g[c] != 32 || cand_t[c] != 0)) continue;
        if (tree->walk_fixed && cand_w[c] != user_w) continue;
        if (tree->tile_fixed && cand_t[c] != user_t) continue;
        tree->group_rays = cand_g[c];
        tree->walk_mode = cand_w[c];
        tree->tile = cand_t[c];
        double ms = 0;
        for (int rep = 0; rep < 2 && st == LENS_OK; ++rep) {  // first run warms up
            st = shoot(tree, 1, off, orig, ray_dx, ray_dy, ray_dtype, out, LENS_TIMING, s);
            if (st != LENS_OK) break;
            double g = 0, w = 0;
            st = lens_last_timing(tree, &g, &w);
            ms = g + w;
        }
        if (st == LENS_OK && ms < best) {
            best = ms;
            best_g = cand_g[c];
            best_w = cand_w[c];
            best_t = cand_t[c];
        }
    }
    cudaFreeAsync(buf, s);
    tree->group_rays = best_g;
    tree->walk_mode = best_w;
    tree->tile = best_t;
    *group_rays = best_g;
    return st;
}

lens_status lens_reserve(lens_tree* tree, int64_t max_rays, int64_t max_batches)
{
    if (!tree) return lens_set_error(LENS_ERR_INVALID_ARG, "tree is NULL");
    if (max_rays < 0 || max_batches < 1) return lens_set_error(LENS_ERR_INVALID_ARG, "bad reserve sizes");
    LENS_TRY(reserve_rays(tree, max_rays, max_batches, 0));
    LENS_CUDA(cudaStreamSynchronize(0));
    return LENS_OK;
}

lens_status lens_sync_status(lens_tree* tree, void* stream)
{
    if (!tree) return lens_set_error(LENS_ERR_INVALID_ARG, "tree is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    LENS_CUDA(cudaStreamSynchronize(s));
    uint32_t herr = 0;
    LENS_CUDA(cudaMemcpy(&herr, tree->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (herr) {
        LENS_CUDA(cudaMemset(tree->d_err, 0, sizeof(uint32_t)));
        if (herr & DERR_BAD_INPUT) return lens_set_error(LENS_ERR_INVALID_ARG, "bad input found on the device");
        if (herr & DERR_WAIT_TIMEOUT)
            return lens_set_error(LENS_ERR_TIMEOUT, "a hand-over wait between walk warps timed out (code %u)", herr);
        return lens_set_error(LENS_ERR_INTERNAL, "device check failed (code %u)", herr);
    }
    return LENS_OK;
}

lens_status lens_set_wait_limit(lens_tree* tree, int64_t cycles)
{
    if (!tree) return lens_set_error(LENS_ERR_INVALID_ARG, "tree is NULL");
    if (cycles < 0) return lens_set_error(LENS_ERR_INVALID_ARG, "cycles must be >= 0");
    tree->wait_cycles = cycles == 0 ? 4000000000ll : cycles;
    return LENS_OK;
}

lens_status lens_tree_counters(lens_tree* t, int64_t* out, int32_t reset)
{
    if (!t || !out) return lens_set_error(LENS_ERR_INVALID_ARG, "NULL argument");
    unsigned long long h[8];
    LENS_CUDA(cudaDeviceSynchronize());
    LENS_CUDA(cudaMemcpy(h, t->d_stats, sizeof(h), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 8; ++i) out[i] = (int64_t)h[i];
    if (reset) LENS_CUDA(cudaMemset(t->d_stats, 0, sizeof(h)));
    return LENS_OK;
}

lens_status lens_last_timing(lens_tree* t, double* group_ms, double* walk_ms)
{
    if (!t || !group_ms || !walk_ms) return lens_set_error(LENS_ERR_INVALID_ARG, "NULL argument");
    *group_ms = *walk_ms = 0.0;
    if (!t->timed) return LENS_OK;
    LENS_CUDA(cudaEventSynchronize(t->ev[3]));
    float a = 0, b = 0;
    LENS_CUDA(cudaEventElapsedTime(&a, t->ev[0], t->ev[1]));
    LENS_CUDA(cudaEventElapsedTime(&b, t->ev[2], t->ev[3]));  // from the end of any wait for the build
    *group_ms = a;
    *walk_ms = b;
    return LENS_OK;
}

lens_status lens_tree_get_info(const lens_tree* t, lens_tree_info* info)
{
    if (!t || !info) return lens_set_error(LENS_ERR_INVALID_ARG, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    for (auto& st : const_cast<lens_tree*>(t)->sp) LENS_TRY(finish_species(st));
    info->n_species = (int32_t)t->sp.size();
    info->precision = t->precision;
    info->n_halos = t->n_halos;
    for (size_t i = 0; i < t->sp.size() && i < 8; ++i) {
        const SpeciesTree& s = t->sp[i];
        info->n_particles[i] = s.n;
        info->n_nodes[i] = s.n_nodes;
        info->n_leaves[i] = s.n_leaves;
        info->n_big[i] = s.n_big;
        info->depth[i] = s.depth;
        info->root[i][0] = s.root_cx;
        info->root[i][1] = s.root_cy;
        info->root[i][2] = s.root_half;
        for (int k = 0; k < 4; ++k) info->build_ms[i][k] = s.phase_ms[k];
    }
    info->group_rays = t->group_rays;
    info->walk = t->walk_mode;
    info->tile = t->tile ? LENS_TILE_LARGE : LENS_TILE_STANDARD;
    uint32_t split[2] = {0, 0};
    LENS_CUDA(cudaDeviceSynchronize());
    LENS_CUDA(cudaMemcpy(split, t->d_stats + 8, sizeof(split), cudaMemcpyDeviceToHost));
    info->split_groups = (int32_t)split[0];
    return LENS_OK;
}

lens_status lens_tree_export(const lens_tree* t, int32_t si, void* nodes, int32_t* links, int32_t* perm,
                             int32_t* listed)
{
    if (!t) return lens_set_error(LENS_ERR_INVALID_ARG, "tree is NULL");
    if (si < 0 || si >= (int32_t)t->sp.size()) return lens_set_error(LENS_ERR_INVALID_ARG, "bad species index");
    LENS_TRY(finish_species(const_cast<lens_tree*>(t)->sp[si]));
    const SpeciesTree& s = t->sp[si];
    int64_t nn = s.n_nodes, n = s.n;
    LENS_CUDA(cudaDeviceSynchronize());
    if (nodes && nn > 0) {
        bool dbl = s.prec == LENS_PREC_FP64;
        size_t es = dbl ? 8 : 4;
        std::vector<char> A(nn * 4 * es), B(nn * 2 * es);
        std::vector<float> rcm(nn);
        std::vector<uint8_t> lev(nn);
        LENS_CUDA(cudaMemcpy(A.data(), s.nodeA, A.size(), cudaMemcpyDeviceToHost));
        LENS_CUDA(cudaMemcpy(B.data(), s.nodeB, B.size(), cudaMemcpyDeviceToHost));
        LENS_CUDA(cudaMemcpy(lev.data(), s.node_level, nn, cudaMemcpyDeviceToHost));
        for (int64_t b = 0; b < nn; ++b) {
            double v[8];
            for (int k = 0; k < 4; ++k)
                v[k] = dbl ? ((double*)A.data())[4 * b + k] : ((float*)A.data())[4 * b + k];
            for (int k = 0; k < 2; ++k)
                v[4 + k] = dbl ? ((double*)B.data())[2 * b + k] : ((float*)B.data())[2 * b + k];
            v[6] = 2.0 * s.root_half / (double)(1u << lev[b]);
            v[7] = lev[b];
            for (int k = 0; k < 8; ++k) {
                if (dbl) ((double*)nodes)[8 * b + k] = v[k];
                else ((float*)nodes)[8 * b + k] = (float)v[k];
            }
        }
    }
    if (links && nn > 0) {
        std::vector<int4> L(nn);
        LENS_CUDA(cudaMemcpy(L.data(), s.link, nn * sizeof(int4), cudaMemcpyDeviceToHost));
        for (int64_t b = 0; b < nn; ++b) {
            links[4 * b] = L[b].x;
            links[4 * b + 1] = L[b].y & kCountMask;
            links[4 * b + 2] = (L[b].y & kLeafBit) ? 1 : 0;
            links[4 * b + 3] = L[b].w;
        }
    }
    if (perm && n > 0) LENS_CUDA(cudaMemcpy(perm, s.perm, n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (listed && n > 0) {
        std::vector<uint32_t> P(n);
        std::vector<uint8_t> Ls(n, 0);
        LENS_CUDA(cudaMemcpy(P.data(), s.perm, n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
        if (s.listed) LENS_CUDA(cudaMemcpy(Ls.data(), s.listed, n, cudaMemcpyDeviceToHost));
        for (int64_t j = 0; j < n; ++j) listed[P[j]] = Ls[j];
    }
    return LENS_OK;
}

}  // extern "C"

// ------------------------------------------- FP32 / FP64 peak microbenchmarks

// Eight independent dependent-FMA chains per thread (enough ILP to keep the
// FMA pipes busy), written to memory at the end so nothing is eliminated.
template <typename T>
__global__ void k_fma_peak(T* sink, int64_t iters, T a, T b)
{
    T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    T r = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (r == T(1234.5)) sink[0] = r;
}

template <typename T>
static lens_status fma_peak(int64_t iters, double* flops, cudaStream_t s)
{
    int dev = 0, sms = 0;
    LENS_CUDA(cudaGetDevice(&dev));
    LENS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    T* sink = nullptr;
    LENS_CUDA(lens_malloc((void**)&sink, sizeof(T)));
    const int threads = 256, blocks = sms * 8;
    cudaEvent_t e0, e1;
    LENS_CUDA(cudaEventCreate(&e0));
    LENS_CUDA(cudaEventCreate(&e1));
    { k_fma_peak<T><<<blocks, threads, 0, s>>>(sink, iters / 8 + 1, T(0.999), T(0.001)); note_launch(); }  // warm up
    LENS_CUDA(cudaEventRecord(e0, s));
    { k_fma_peak<T><<<blocks, threads, 0, s>>>(sink, iters, T(0.999), T(0.001)); note_launch(); }
    LENS_CUDA(cudaEventRecord(e1, s));
    LENS_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    LENS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    double total = 2.0 * 8.0 * 16.0 * (double)iters * (double)threads * (double)blocks;
    *flops = total / (ms * 1e-3);
    return LENS_OK;
}

extern "C" lens_status lens_fp32_peak(int64_t iters, double* flops, void* stream)
{
    if (!flops || iters < 1) return lens_set_error(LENS_ERR_INVALID_ARG, "bad arguments");
    return fma_peak<float>(iters, flops, (cudaStream_t)stream);
}

extern "C" lens_status lens_fp64_peak(int64_t iters, double* flops, void* stream)
{
    if (!flops || iters < 1) return lens_set_error(LENS_ERR_INVALID_ARG, "bad arguments");
    return fma_peak<double>(iters, flops, (cudaStream_t)stream);
}
