// tree.cuh -- device data of a built lens and the internal entry points that
// the C ABI (api.cu) drives.
#pragma once

#include <vector>

#include "common.cuh"

namespace lens {

// Link word y: particle/child count with the leaf flag in bit 30.
constexpr int kLeafBit = 1 << 30;
constexpr int kCountMask = kLeafBit - 1;

// One species' quadtree.  Node arrays are in breadth-first order (children of
// a node are contiguous); particle arrays in Morton order.
struct SpeciesTree {
    int kind = LENS_POINT;
    int prec = LENS_PREC_FP32;
    int64_t n = 0;
    int64_t n_nodes = 0, n_leaves = 0, n_big = 0;
    int depth = 0;
    double root_cx = 0, root_cy = 0, root_half = 0;
    double shape = 0;          // q (GAUSS) or R_max / r_s (NFW)
    double Uq = 0, invNq = 0;  // GAUSS: q^2/2 and 1/(1 - e^{-q^2/2})
    std::vector<int64_t> level_start;  // BFS offset of each level, depth + 2 entries
    double phase_ms[4] = {0, 0, 0, 0};   // device time of the build phases (CUDA events)
    // depth, level_start, n_big, n_chunks, n_leaves, root_* and phase_ms are
    // filled from the device by finish_species when first needed
    bool meta_ready = false;
    void* d_meta = nullptr;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};

    // node data (BFS order); element type T = float or double by prec
    void* nodeA = nullptr;     // T4 {x_cm, y_cm, M, r_cut^2}
    void* nodeB = nullptr;     // T2 {Re Q2, Im Q2}
    int4* link = nullptr;      // {first child | first particle, count | leaf bit, big start, big count}
    float* node_rcm = nullptr; // r_cm (distance from the centre of mass to the farthest corner)
    int* parent = nullptr;     // parent node (-1 at the root), for the adjoint push-down
    uint8_t* node_level = nullptr;
    // particles (Morton order)
    void* exact0 = nullptr;    // T4 full-profile records (see walk)
    void* exact1 = nullptr;    // T4 second record (NFW only)
    void* leaf0 = nullptr;     // T4 leaf records: listed particles marked as softened points
    void* big0 = nullptr;      // T4 big-list test records {x, y, s^2, r0^2}
    void* big1 = nullptr;      // T4 {m, c, 0, 0} (GAUSS) or {m, A, B, 0} (NFW)
    void* big_chunk = nullptr; // T4 per 32 big entries: bounding box of their support squares
    void* node_bigbox = nullptr;  // T4 per node: bounding box of its list's support squares
    int64_t n_chunks = 0;
    uint32_t* perm = nullptr;  // Morton position -> input index
    uint32_t* big_pid = nullptr;  // big entry -> Morton position
    uint8_t* listed = nullptr;    // per Morton position: 1 if in a big list
};

struct HaloDev {
    int32_t kind, pad;
    double x, y, m, p0, p1;
    double c0, c1, c2;  // derived constants (GAUSS: c, Uq, invNq; NFW: A, B, R^2)
    double c3;          // NFW: X f(X) / g(X), X = R_max / r_s (the adjoint's d/dR_max)
};

struct DevScratch {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct GraphEntry;

}  // namespace lens

struct lens_tree {
    int precision = LENS_PREC_FP32;
    double theta = 0.1;
    int leaf_max = 5;
    int group_rays = 32;
    int walk_mode = LENS_WALK_WARP;
    int tile = 0;             // near-field tile of the one-warp FP32 tree walk: 0 standard, 1 doubled
    bool tile_fixed = false;  // chosen by the caller at build time (not autotuned)
    bool walk_fixed = false;  // chosen by the caller at build time (not autotuned)
    std::vector<lens::SpeciesTree> sp;
    std::vector<lens_halo> halos_host;
    lens::HaloDev* halos = nullptr;  // device copy
    int64_t n_halos = 0;
    uint32_t* d_err = nullptr;       // device error word
    // shoot scratch (grown on demand)
    lens::DevScratch ray_scratch;
    int64_t ray_cap = 0, batch_cap = 0;
    int num_sms = 0;
    int device = 0;
    long long wait_cycles = 4000000000ll;   // bound of a wait between cooperating warps (~2 s at 2 GHz)
    std::vector<lens::GraphEntry*> graphs;
    unsigned long long* d_stats = nullptr;  // 8 walk counters (LENS_COUNT), then the last adjoint's split {Kc, Hn}
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // LENS_TIMING: start, grouped, tree ready, walked
    // recorded on the build's stream when the build is complete: a call that
    // reads the tree on another stream waits for it on the device first
    cudaEvent_t built = nullptr;
    // the rays whose per-group work the scratch holds (walk_shared.cuh), as
    // an opaque copy of their identity: pointers, size, dtype, origin, R
    const void* cost_dx = nullptr;
    const void* cost_dy = nullptr;
    int64_t cost_n = -1;
    int cost_dtype = -1, cost_R = 0;
    double cost_ox = 0, cost_oy = 0;
    // the rays whose groups the scratch holds (set by the grouping, n = -1 if
    // none): the adjoint of a LENS_KEEP_LISTS call reuses them
    const void* grp_dx = nullptr;
    const void* grp_dy = nullptr;
    int64_t grp_n = -1;
    int grp_dtype = -1, grp_R = 0;
    double grp_ox = 0, grp_oy = 0;
    // interaction lists kept by the last lens_shoot_rays with LENS_KEEP_LISTS
    // (walk_dev.cuh tags), for the rays identified as for the work record
    uint32_t* list_ids = nullptr;  // list_groups x list_K tagged box indices
    uint32_t* list_n = nullptr;    // per group: entries, or kListOverflow
    int64_t list_groups = 0;
    int list_K = 0;
    const void* list_dx = nullptr;
    const void* list_dy = nullptr;
    int64_t list_rays = -1;
    int list_dtype = -1, list_R = 0;
    double list_ox = 0, list_oy = 0;
    bool timed = false;
    void* noalloc_scratch = nullptr;        // device address of the no-alloc scratch array (walk.cu)
    void* amr_ws = nullptr;                 // image-finding workspace (amr.cu), kept between calls
    void (*amr_free)(void*) = nullptr;
};

namespace lens {

lens_status build_species(lens_tree* t, SpeciesTree& st, const lens_species& in, cudaStream_t s);
lens_status finish_species(SpeciesTree& st);  // host copies of the build's counts (synchronises once)
void free_species(SpeciesTree& st);
// Make stream s wait on the device for the end of the tree's build (no-op
// while s is being captured into a graph: the graph's launch waits instead).
lens_status wait_built(const lens_tree* t, cudaStream_t s);

}  // namespace lens
