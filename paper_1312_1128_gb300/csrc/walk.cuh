// walk.cuh -- ray groups and the launch interface of the walk / direct kernels.
#pragma once

#include "tree.cuh"

namespace lens {

// Rays of one shoot call, grouped: groups of up to 32*R spatially sorted rays
// share one interaction list.  Ray positions are split as H (per group, the
// FP32/FP64 value nearest the group centre) + l (per ray), both in type T,
// formed from the FP64 absolute position; the walk forms every separation as
// (l - (p - H)), so rays far from the coordinate zero keep full resolution.
template <typename T> struct RayGroups {
    int64_t n_rays = 0, n_groups = 0;
    int rays_per_group = 32;
    const void* gH = nullptr;       // T2 per group: H
    const void* gbox = nullptr;     // T4 per group: {l centre x, y, l half-extent x, y}
    const uint2* grange = nullptr;  // per group: {first sorted position, count}
    const void* ray_l = nullptr;    // T2 per sorted position
    const uint32_t* ray_idx = nullptr;  // per sorted position: caller's ray index
};

struct WalkLaunch {
    const SpeciesTree* st;          // may be null when only halos are evaluated
    const HaloDev* halos;
    int n_halos;                    // halos evaluated in this launch (0 or all)
    void* out[5];                   // alpha1, alpha2, kappa, gamma1, gamma2 (T)
    int accumulate;
    int alpha_only;
    int direct;                     // 1: direct sum over all particles
    uint32_t* counter;              // work counter (zeroed by the launcher)
    int* stack;                     // per-warp stacks
    int64_t stack_slots;
    uint32_t* err;
    int grid;                       // persistent grid size
};

// Grouping: fills the device arrays in `scratch` and returns the group view.
struct ShootScratch;
lens_status group_rays(lens_tree* t, int64_t n_batches, const int64_t* h_offsets,
                       const double* h_origins, const void* dx, const void* dy, int ray_dtype,
                       int64_t n, cudaStream_t s, void** view_out);

lens_status launch_walk(lens_tree* t, const void* view, const WalkLaunch& L, cudaStream_t s);

}  // namespace lens
