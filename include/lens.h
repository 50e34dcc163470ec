/*
 * lens.h -- C ABI of liblens, a GB300 (sm_103a) implementation of the ray-
 * shooting deflection solver of Metcalf & Petkova, "GLAMER Part I: A Code for
 * Gravitational Lensing Simulations with Adaptive Mesh Refinement"
 * (arXiv:1312.1128).
 *
 * For every ray position x on the lens plane the library returns the
 * deflection alpha (2 components), the convergence kappa and the shear
 * gamma1, gamma2 (Sec. 3.2, Eqs. alpha, kappa, gamma_1, gamma_2) produced by
 * point masses (Sec. 3.5), truncated-Gaussian smoothed particles (Sec. 3.1,
 * Eq. smoothing) and analytic halos (Sec. 3.2), using the paper's tree
 * algorithm (Sec. 3.2: equal-area quadtree, monopole + quadrupole cells,
 * r_cut = r_cm / theta_force (Eq. r_cut), the 2D multipole acceptability
 * criterion, big-particle lists) or, with LENS_DIRECT, the direct sum that
 * the tree converges to at theta_force = 0 (Sec. 5.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Units: masses are given in "m-units", m = M / (pi Sigma_crit) (Sec. 2,
 *   Sec. 3.5), so that a point mass deflects by alpha = m x / |x|^2.  The lens
 *   equation is y = x - alpha(x) (Sec. 2, Eq. lens_eq).
 * - Shear follows Eqs. gamma_1, gamma_2: gamma1 = (d1 alpha1 - d2 alpha2)/2,
 *   gamma2 = d1 alpha2; the magnification matrix is
 *   [[1-kappa-gamma1, -gamma2], [-gamma2, 1-kappa+gamma1]] (App. A).
 * - Pointers named "device" are CUDA device (or managed) memory owned by the
 *   caller; "host" pointers are ordinary host memory.  The library never
 *   frees caller memory.  A lens_tree owns its internal device buffers until
 *   lens_free_tree.
 * - Every call is asynchronous on the CUDA stream it is given (NULL = the
 *   legacy default stream), except where a call says it synchronises.  The
 *   returned status reports argument, allocation and launch errors at once;
 *   errors detected inside kernels are latched in the tree and reported by
 *   lens_sync_status (and by the next lens_* call on that tree that
 *   synchronises).  Kernels never trap, assert or spin without a bound.
 * - n == 0 rays is a valid no-op.  NaN inputs propagate to the outputs.
 * - One lens_tree must not be used by two calls concurrently (its scratch
 *   buffers are shared); distinct trees are independent.
 * - On failure, lens_last_error() returns a message for the calling thread.
 */
#ifndef LENS_H
#define LENS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LENS_API_VERSION 2

typedef enum lens_status {
    LENS_OK = 0,
    LENS_ERR_INVALID_ARG = 1,   /* bad pointer, size, kind, dtype or parameter */
    LENS_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    LENS_ERR_OOM = 3,           /* device allocation failed */
    LENS_ERR_TIMEOUT = 4,       /* a bounded device wait ran out */
    LENS_ERR_INTERNAL = 5,      /* a device-side consistency check failed */
    LENS_ERR_UNSUPPORTED = 6    /* valid request this build does not implement */
} lens_status;

/* Lens component kinds. */
enum {
    LENS_POINT = 0,  /* point mass: alpha = m r_hat / r (Sec. 3.5)                        */
    LENS_GAUSS = 1,  /* truncated 2D Gaussian of width r_sm, cut at q r_sm (Sec. 3.1)      */
    LENS_NFW = 2,    /* projected NFW, scale radius r_s, truncated in 2D at R_max; a point  *
                      * mass outside R_max (Sec. 3.2 "analytic models")                    */
    LENS_SIS = 3,    /* singular isothermal sphere, Einstein radius r_E (App. B)           */
    LENS_DISK = 4    /* uniform disk of radius R; m < 0 subtracts a mass sheet (Sec. 3.5)   */
};

/* Element types of caller arrays. */
enum { LENS_F32 = 0, LENS_F64 = 1 };

/* Arithmetic precision of a tree (fixed at build time). */
enum {
    LENS_PREC_FP32 = 0,  /* FP32 interactions, compensated accumulation; FP32 outputs */
    LENS_PREC_FP64 = 1   /* FP64 throughout; FP64 outputs                             */
};

/* Flags for the shooting calls. */
enum {
    LENS_ALPHA_ONLY = 1,  /* compute alpha only; kappa/gamma pointers may be NULL (Sec. 3.2) */
    LENS_DIRECT = 2,      /* direct sum over every particle instead of the tree walk        */
    LENS_ACCUMULATE = 4,  /* add to the output arrays instead of overwriting them           */
    LENS_USE_GRAPH = 8,   /* lens_shoot_batches: replay a cached CUDA graph of the launch    */
    LENS_COUNT = 16,      /* accumulate walk interaction counters (lens_tree_counters)     */
    LENS_TIMING = 32,     /* time the grouping and walk kernels (lens_last_timing); not with *
                           * LENS_USE_GRAPH (time a replay with events on the caller's stream) */
    LENS_KEEP_LISTS = 64  /* lens_shoot_rays: keep the walk's interaction lists for the     *
                           * adjoint; lens_shoot_rays_backward: replay them (see there)     */
};

/* One particle species: a homogeneous set of particles of one kind (Sec. 3.1
 * treats each species separately).  data is DEVICE memory, n x 4 elements of
 * type dtype, row-major {x, y, m, p}:
 *   LENS_POINT: p unused;                        shape unused
 *   LENS_GAUSS: p = r_sm (> 0);                  shape = q (> 0), support q r_sm
 *   LENS_NFW:   p = r_s (> 0);                   shape = R_max / r_s (> 0)
 * Masses must be finite and >= 0 (the tree's centre-of-mass bounds rely on it). */
typedef struct lens_species {
    int32_t kind;
    int32_t dtype;
    int64_t n;
    const void* data;
    double shape;
} lens_species;

/* An analytic component evaluated directly for every ray (host memory).
 *   LENS_POINT: m;  LENS_GAUSS: m, p0 = r_sm, p1 = q;  LENS_NFW: m, p0 = r_s,
 *   p1 = R_max;  LENS_SIS: p0 = r_E (m unused);  LENS_DISK: m, p0 = R. */
typedef struct lens_halo {
    int32_t kind;
    int32_t reserved;
    double x, y, m, p0, p1;
} lens_halo;

typedef struct lens_params {
    double theta;        /* opening angle theta_force of Eq. r_cut (>= 0; 0 = never accept a cell) */
    int32_t leaf_max;    /* a box holding fewer than leaf_max particles is a leaf (>= 1; paper: 5)  */
    int32_t precision;   /* LENS_PREC_FP32 or LENS_PREC_FP64                                          */
    int32_t group_rays;  /* rays sharing one interaction list: 0 = default (32), else 32, 64 or 128;  *
                          * 128 serves the one-warp FP32 tree walk (other calls use 64)         */
    int32_t walk;        /* LENS_WALK_*: how warps share a group's walk (0 = default, autotuned)      */
    int32_t tile;        /* LENS_TILE_*: near-field tile of the walk (0 = default, autotuned)         */
    int32_t reserved;    /* 0                                                                         */
} lens_params;

/* lens_params.tile: the shared-memory tiles in which a warp stages leaf
 * particles and big-list entries before evaluating them for its rays
 * (Sec. 3.2 near field).  LENS_TILE_STANDARD: 128 of each per warp;
 * LENS_TILE_LARGE: 256 (fewer flushes, twice the shared memory; FP32 trees,
 * one-warp walk).  LENS_TILE_DEFAULT = STANDARD until lens_autotune picks
 * one.  Same results up to the order of summation. */
enum { LENS_TILE_DEFAULT = 0, LENS_TILE_STANDARD = 1, LENS_TILE_LARGE = 2 };

/* lens_params.walk.  LENS_WALK_WARP: one warp walks the tree for its group
 * and evaluates every full buffer itself.  LENS_WALK_PAIRS: a producer warp
 * walks and fills shared-memory buffers that a consumer warp, holding the
 * group's rays, evaluates (the latency-bound walk overlaps the arithmetic).
 * LENS_WALK_TRIOS: a producer warp feeds two consumer warps that split the
 * 64 rays of its group (32 each), so that two warps of three do arithmetic;
 * with 32-ray groups it is the pairs form.  Same results up to the order of
 * summation.  LENS_WALK_DEFAULT = WARP until lens_autotune picks one. */
enum { LENS_WALK_DEFAULT = 0, LENS_WALK_WARP = 1, LENS_WALK_PAIRS = 2, LENS_WALK_TRIOS = 3 };

typedef struct lens_tree lens_tree;  /* opaque, library-owned */

/* Summary of a built tree, for inspection and tests. */
typedef struct lens_tree_info {
    int32_t n_species;
    int32_t precision;
    int64_t n_halos;
    int64_t n_particles[8];   /* per species (first 8 species) */
    int64_t n_nodes[8];
    int64_t n_leaves[8];
    int64_t n_big[8];         /* big-list entries (Sec. 3.2) */
    int32_t depth[8];         /* deepest level (root = 0) */
    double root[8][3];        /* root box centre x, y and half side */
    double build_ms[8][4];    /* device time (CUDA events) of the build phases: stage +
                                 Morton sort, topology + node layout, moments + big
                                 lists, finish */
    int32_t group_rays;       /* current ray-group size (32, 64 or 128) */
    int32_t walk;             /* current walk form: LENS_WALK_WARP, _PAIRS or _TRIOS */
    int32_t tile;             /* current near-field tile: LENS_TILE_STANDARD or LENS_TILE_LARGE */
    int32_t split_groups;     /* ray groups the last lens_shoot_rays_backward split into
                                 slices (the heaviest groups of a recorded walk), 0 if none;
                                 reading it synchronises the device */
} lens_tree_info;

/*
 * lens_build_tree -- build the quadtree of every species (Sec. 3.2: equal-
 * area quadtree; per box the monopole and quadrupole moments, r_cut of
 * Eq. r_cut and the list of particles whose size exceeds half the box side
 * and that no ancestor lists).
 *   species, n_species: host array of n_species (0..8) descriptors; each
 *       data pointer is device memory, read during the call only.
 *   halos, n_halos: host array of analytic components evaluated for every
 *       ray (may be NULL when n_halos == 0); copied.
 *   params: host pointer; theta >= 0, leaf_max >= 1.
 *   stream: cudaStream_t to build on (NULL = default stream).
 *   out: receives the new tree on LENS_OK, NULL otherwise.
 * The call synchronises on `stream` once per species, to size the node
 * arrays (and read the input check); the rest of the build is enqueued on
 * `stream` and finishes in stream order.  The tree may then be used on any
 * stream: the build records an event when it is complete, and every call
 * that reads the tree makes its stream wait for that event on the device
 * before its first kernel that reads the tree (a shoot or potential call
 * groups its rays first, so on a second stream the grouping overlaps the
 * end of the build).  A call captured into a CUDA graph does not wait:
 * launch the graph after the build has completed or in stream order after
 * it.  Counts the host reports (lens_tree_get_info) are read from the device
 * when first asked for.
 * Errors: LENS_ERR_INVALID_ARG for NULL pointers, negative sizes, unknown
 * kinds or dtypes, theta < 0, leaf_max < 1 or a negative / non-finite mass or
 * size found on the device; LENS_ERR_OOM (nothing is kept); LENS_ERR_CUDA; a
 * consistency check that fails on the device after the call returned is
 * reported by lens_sync_status.
 */
lens_status lens_build_tree(const lens_species* species, int32_t n_species,
                            const lens_halo* halos, int64_t n_halos,
                            const lens_params* params, void* stream, lens_tree** out);

/*
 * lens_shoot_rays -- evaluate alpha, kappa, gamma at n rays (Sec. 3.2 tree
 * walk; Sec. 3.3 ray-parallel evaluation).
 *   origin_x, origin_y: FP64 origin added to every ray offset.
 *   ray_dx, ray_dy: DEVICE arrays of n offsets of type ray_dtype; ray i sits
 *       at (origin_x + ray_dx[i], origin_y + ray_dy[i]), formed in FP64, so a
 *       microlensing patch keeps its resolution far from the coordinate zero.
 *   alpha1 .. gamma2: output arrays of n elements, float for an FP32
 *       tree, double for an FP64 tree, in device memory or in page-locked
 *       host memory (cudaHostAlloc / cudaMallocHost: unified addressing maps
 *       it for every device); the kernels write each element once, so
 *       host outputs receive the results with no separate copy (read them
 *       after the stream has synchronised; a second species or
 *       LENS_ACCUMULATE also reads them back).  kappa, gamma1, gamma2 may be
 *       NULL only with LENS_ALPHA_ONLY.
 *   flags: LENS_ALPHA_ONLY, LENS_DIRECT, LENS_ACCUMULATE, LENS_COUNT,
 *       LENS_TIMING, LENS_KEEP_LISTS.  LENS_KEEP_LISTS (tree walk) also
 *       stores, per ray group, the walk's interaction lists -- the cells it
 *       accepted, the leaves it opened and the boxes whose big lists reach
 *       the group, as tagged box indices, up to 512 per 32 rays -- for a
 *       following lens_shoot_rays_backward on the same rays; they replace
 *       the lists of the previous such call and are kept with the tree
 *       (4 B per entry: 2 KB per 32 rays, from cudaMalloc when they grow).
 *       A group whose lists exceed the room is marked and walked again by
 *       the adjoint.
 * A tree without particles (analytic components only) is shot one thread
 * per ray with no ray grouping, except with LENS_COUNT or LENS_TIMING, whose
 * counters and times refer to the grouped walk (the same terms either way).
 * Scratch buffers grow on demand (cudaMalloc, outside any graph capture).
 */
lens_status lens_shoot_rays(lens_tree* tree, double origin_x, double origin_y,
                            const void* ray_dx, const void* ray_dy, int32_t ray_dtype, int64_t n,
                            void* alpha1, void* alpha2, void* kappa, void* gamma1, void* gamma2,
                            int32_t flags, void* stream);

/*
 * lens_shoot_batches -- evaluate many ray batches of uneven size in one
 * persistent launch (the refinement batches of Sec. 4 / Sec. 3.3, "bigger
 * chunks are more efficient").
 *   n_batches: number of batches (>= 0).
 *   offsets: HOST array of n_batches + 1 non-decreasing int64 with
 *       offsets[0] = 0; batch b owns rays [offsets[b], offsets[b+1]).
 *   origins: HOST array n_batches x 2 of FP64 batch origins.
 *   ray_dx, ray_dy, outputs, flags: as lens_shoot_rays, over all
 *       offsets[n_batches] rays.  LENS_USE_GRAPH captures the launch sequence
 *       into a CUDA graph on first use for this (sizes, pointers, flags) key
 *       and replays it afterwards; call lens_reserve first when the stream is
 *       being captured by the caller.
 */
lens_status lens_shoot_batches(lens_tree* tree, int64_t n_batches, const int64_t* offsets,
                               const double* origins, const void* ray_dx, const void* ray_dy,
                               int32_t ray_dtype, void* alpha1, void* alpha2, void* kappa,
                               void* gamma1, void* gamma2, int32_t flags, void* stream);

/*
 * lens_shoot_rays_backward -- vector-Jacobian product of lens_shoot_rays:
 * given dL/d(outputs) at n rays, accumulates dL/d(particle mass, position,
 * size) and dL/d(halo parameters).  No counterpart in the paper: it
 * differentiates the tree approximation the forward computes (cells'
 * monopole and quadrupole moments as functions of their particles; each
 * profile's enclosed mass as a function of its size and shape, Sec. 3.1 and
 * Sec. 3.2), for lens-model fitting.
 *   ray arguments: exactly those of the forward call.
 *   g_alpha1, g_alpha2: DEVICE arrays of n gradients (output dtype); g_kappa,
 *       g_gamma1, g_gamma2 must be NULL in this version (LENS_ERR_UNSUPPORTED
 *       otherwise).
 *   g_species: HOST array of n_species DEVICE pointers (NULL entries skip a
 *       species); each receives n x 4 {dL/dm, dL/dx, dL/dy, dL/dp} in the
 *       tree's precision, ADDED to its contents, in the species' input order;
 *       p is the species' fourth column (GAUSS r_sm, NFW r_s at the fixed
 *       ratio R_max / r_s; 0 for POINT).
 *   g_halos: DEVICE array n_halos x 5 doubles, added to, or NULL:
 *       {dL/dm (dL/dr_E for the SIS), dL/dx, dL/dy, dL/dp0, dL/dp1} with p0, p1
 *       the lens_halo fields (GAUSS r_sm, q; NFW r_s, R_max; SIS r_E again,
 *       0; DISK R, 0; POINT 0, 0).
 *   flags: LENS_DIRECT differentiates the direct sum instead of the tree.
 *       LENS_KEEP_LISTS: if the last lens_shoot_rays with LENS_KEEP_LISTS on
 *       this tree had these very rays (same arrays, unchanged since, same
 *       count, dtype and origin), the adjoint replays that call's
 *       interaction lists instead of walking the tree again (the forward's
 *       near field is recomputed, not stored), and reuses its ray groups
 *       if no other call has grouped rays on this tree since; otherwise the
 *       flag has no effect.  Changing the ray values in between is the caller's error:
 *       the replayed lists then belong to the old rays.
 * Tree gradients with respect to masses and positions follow the tree's
 * moments (so they carry the tree's own approximation error); size and halo
 * parameter gradients equal the direct sum's, since every ray inside a
 * particle's support meets its full profile.  Scratch: about 32 B per
 * particle and 88 B per tree node, from the stream-ordered pool.
 */
lens_status lens_shoot_rays_backward(lens_tree* tree, double origin_x, double origin_y,
                                     const void* ray_dx, const void* ray_dy, int32_t ray_dtype,
                                     int64_t n, const void* g_alpha1, const void* g_alpha2,
                                     const void* g_kappa, const void* g_gamma1,
                                     const void* g_gamma2, void* const* g_species,
                                     void* g_halos, int32_t flags, void* stream);

/*
 * lens_autotune -- pick the ray-group size (rays sharing one interaction
 * list: 32, 64, or 128 with the one-warp walk of an FP32 tree) and, unless the tree was built with them fixed in
 * lens_params, the walk form (LENS_WALK_WARP, _PAIRS or _TRIOS) and the
 * near-field tile (LENS_TILE_STANDARD or LENS_TILE_LARGE) for this tree by
 * timing the walk on the given rays (at most the first 8,388,608; same
 * arguments as lens_shoot_rays) with CUDA events, and keep the fastest for
 * later calls.  *group_rays receives the group size; lens_tree_get_info
 * reports all three.  Synchronous; allocates temporary outputs on the
 * device.
 */
lens_status lens_autotune(lens_tree* tree, double origin_x, double origin_y, const void* ray_dx,
                          const void* ray_dy, int32_t ray_dtype, int64_t n, void* stream,
                          int32_t* group_rays);

/*
 * lens_shoot_rays_direct_noalloc -- the direct sum of lens_shoot_rays with
 * LENS_DIRECT, for callers that cannot allocate device memory during the
 * call: code that runs while another component owns the device allocator,
 * latency-bound loops that cannot absorb the device-wide synchronisation a
 * cudaMalloc may cause, or deployments that reserve a fixed device budget up
 * front.  The paper has no counterpart; it is a deployment variant only.
 *   Arguments, output layout and results are those of lens_shoot_rays with
 *   LENS_DIRECT, except that rays are grouped 32 at a time in their input
 *   order instead of being sorted: give them in a spatially coherent order
 *   (rows of a grid, Morton order).  An FP32 tree forms each ray's offset
 *   from its group's anchor in FP32 (exactly when the positions are FP32
 *   values), so a group that spans a large extent rounds its rays' positions
 *   more coarsely than the sorting call does.
 *   flags: LENS_ALPHA_ONLY and LENS_ACCUMULATE only.
 *   n: at most 262,144 rays per call; larger n returns LENS_ERR_INVALID_ARG
 *   and launches nothing.
 * Scratch: a fixed 5.4 MiB device array defined in the library.  Each GPU
 * holds its copy from the first lens_build_tree on it until the process
 * exits; lens_build_tree looks up the array's device address (with the
 * tree's device current) and keeps it in the tree, so this call makes no
 * cudaMalloc, cudaFree, other allocating call or symbol lookup.  A tree built
 * before a cudaDeviceReset of its device is invalid afterwards (like all its
 * device buffers); build a new one.  All calls share the one array, which
 * keeps the last call's contents (the call clears what must start at zero):
 * calls that overlap on the GPU, on any streams and through any trees, race,
 * so order them (one stream, or events).  The tree must have been built on
 * the current device.
 */
lens_status lens_shoot_rays_direct_noalloc(lens_tree* tree, double origin_x, double origin_y,
                                           const void* ray_dx, const void* ray_dy, int32_t ray_dtype,
                                           int64_t n, void* alpha1, void* alpha2, void* kappa,
                                           void* gamma1, void* gamma2, int32_t flags, void* stream);

/*
 * lens_shoot_potential -- the lensing potential psi (Eq. alpha: alpha =
 * grad psi), with the deflection, for the time delay of Eq. timedelay
 * (delta t = |alpha|^2 / 2 - psi on a single plane), by the tree walk of
 * lens_shoot_rays: far cells add the monopole + quadrupole potential
 * M ln|w| - Re(Q2 / (2 w^2)) about their centre of mass; particles and halos
 * their own potentials; big lists (full - softened point).  Each component's
 * additive constant is fixed by psi = m ln r outside its support (SIS:
 * r_E r).  LENS_DIRECT sums every particle's potential instead of walking.
 *   Same ray arguments as lens_shoot_rays; psi (required), alpha1, alpha2
 *   (may be NULL): arrays of n values in the tree's precision, in device or
 *   page-locked host memory as lens_shoot_rays' outputs.
 *   flags: LENS_DIRECT, LENS_ACCUMULATE, LENS_TIMING (lens_last_timing then
 *   reports this call's grouping and potential-walk times) and LENS_COUNT
 *   (the walk counters of lens_tree_counters) only.
 * Asynchronous; errors as lens_shoot_rays.
 */
lens_status lens_shoot_potential(lens_tree* tree, double origin_x, double origin_y, const void* ray_dx,
                                 const void* ray_dy, int32_t ray_dtype, int64_t n, void* psi, void* alpha1,
                                 void* alpha2, int32_t flags, void* stream);

/* lens_refine_cells modes (see below). */
enum { LENS_REFINE_KAPPA_GAMMA = 0, LENS_REFINE_DEFLECTION = 1 };

/*
 * lens_refine_cells -- refine cells of a uniform grid of already-shot rays by
 * the linear lens equation y = y_c + A (x - x_c) (Sec. 3.4 interpolation,
 * Eq. linear_lens_equation), where the magnification matrix A is uniform over
 * the cell.  Needs no tree: it reads the outputs of an earlier shot.
 *   x0, y0, h, nx, ny: ray (i, j) sits at (x0 + i h, y0 + j h), flat index
 *       i + nx j (nx, ny >= 3, h > 0).  Each ray is the centre of a cell of
 *       side h; its neighbours are the rays E (i+1, j), N (i, j+1),
 *       W (i-1, j), S (i, j-1).
 *   alpha1, alpha2: device, nx*ny deflections, alpha_dtype LENS_F32 or
 *       LENS_F64 (the deflection mode differences neighbouring deflections:
 *       with FP32 deflections the rounding of alpha over h limits A to about
 *       ulp(alpha)/h, so FP64 deflections are what it is for; Sec. 3.4).
 *   kappa, gamma1, gamma2: device, nx*ny float; required by
 *       LENS_REFINE_KAPPA_GAMMA, ignored (may be NULL) by LENS_REFINE_DEFLECTION.
 *   cells, n_cells: device int64, flat indices of the cells' centre rays;
 *       cells == NULL means every interior cell in row-major order
 *       (i = 1..nx-2 fastest, then j = 1..ny-2; n_cells must be
 *       (nx - 2)(ny - 2)).
 *   k: sub-cells per side, odd, 1..15; sub-cell (a, b) is centred at
 *       x_c + ((a - (k-1)/2) h/k, (b - (k-1)/2) h/k).
 *   tol: uniformity tolerance (the paper uses 1e-4).
 *   mode: LENS_REFINE_KAPPA_GAMMA -- uniform if kappa, gamma1, gamma2 of every
 *       neighbour are within tol of the centre's (compared in FP32); A is
 *       Eq. magmatrix at the centre.  LENS_REFINE_DEFLECTION -- A from the
 *       three points centre + each neighbour pair not colinear with it
 *       (E-N, N-W, W-S, S-E) by the App. A solve with y = x - alpha; uniform if
 *       no element differs by more than tol between the pairs (compared in
 *       the precision of alpha); A = the pairs' average.
 *   Outputs (device, caller-owned): uniform[n_cells] uint8 (1 uniform, 0 not,
 *       2 = the index is not an interior cell of the grid); amat[4 n_cells]
 *       float (a11, a21, a12, a22 with dy1 = a11 dx1 + a21 dx2,
 *       dy2 = a12 dx1 + a22 dx2; NaN for index 2); y_sub[2 k k n_cells]
 *       double, [cell][b][a][x, y] source positions of the sub-cell centres,
 *       NaN unless uniform (the caller shoots those rays instead);
 *       n_nonuniform: optional device counter, incremented once per cell with
 *       uniform == 0.
 * Asynchronous on `stream`; allocates nothing; n_cells == 0 is a no-op.
 * Errors: LENS_ERR_INVALID_ARG for bad sizes, k, tol, mode, dtype or NULL
 * arrays; launch failures as LENS_ERR_CUDA.
 */
lens_status lens_refine_cells(double x0, double y0, double h, int64_t nx, int64_t ny, const void* alpha1,
                              const void* alpha2, int32_t alpha_dtype, const float* kappa,
                              const float* gamma1, const float* gamma2, const int64_t* cells,
                              int64_t n_cells, int32_t k, double tol, int32_t mode, uint8_t* uniform,
                              float* amat, double* y_sub, unsigned long long* n_nonuniform, void* stream);

/*
 * lens_smoothing_lengths -- the smoothing length of every particle (Sec.
 * 3.1): the distance in 3D to its k-th nearest other particle (the paper
 * prefers the 3D neighbour distance; its workloads use k = 32).  Exact
 * k-nearest search: particles are sorted by 3D Morton keys, the k nearest of
 * each particle's 2k key-order neighbours bound the distance, and the 3x3x3
 * octree cells at least that large around the particle are scanned.
 * Distances are computed in FP32.
 *   xyz: device float32, n x 3 row-major {x, y, z}; r_sm: device float32,
 *       n outputs (caller-owned; may not alias xyz).
 *   k: 1..64; n = 0 is a no-op, otherwise n > k and n < 2^32.
 * Synchronous on `stream` (reads the particles' bounding box); allocates its
 * scratch (about 40 B per particle) from the stream-ordered pool.
 * Errors: LENS_ERR_INVALID_ARG for bad k or n, NULL arrays or non-finite
 * positions; LENS_ERR_CUDA / LENS_ERR_OOM from the device.
 */
lens_status lens_smoothing_lengths(const float* xyz, int64_t n, int32_t k, float* r_sm, void* stream);

/* lens_reserve -- grow the tree's scratch for up to max_rays rays in up to
 * max_batches batches, so that later calls of that size allocate nothing. */
lens_status lens_reserve(lens_tree* tree, int64_t max_rays, int64_t max_batches);

/* lens_sync_status -- synchronise `stream` and report (then clear) any error
 * latched by a kernel of this tree: LENS_ERR_TIMEOUT when a bounded wait
 * between cooperating warps ran out (see lens_set_wait_limit),
 * LENS_ERR_INVALID_ARG for bad values found on the device, LENS_ERR_INTERNAL
 * for a failed consistency check. */
lens_status lens_sync_status(lens_tree* tree, void* stream);

/* lens_set_wait_limit -- the bound, in SM clock cycles, of every wait
 * between the cooperating warps of the LENS_WALK_PAIRS walk (a consumer
 * waiting for a filled buffer, a producer for an empty one); 0 restores the
 * default of 4e9 cycles (about 2 s at the maximum SM clock).  A wait that
 * runs out latches an error, both warps of the pair return, and the next
 * lens_sync_status reports LENS_ERR_TIMEOUT; the outputs of that call are
 * then incomplete, and the tree and the CUDA context stay usable.  Applies
 * to calls made after it (a CUDA graph that lens_shoot_batches cached
 * earlier keeps the limit it was captured with).  Host-only, cheap. */
lens_status lens_set_wait_limit(lens_tree* tree, int64_t cycles);

/* lens_tree_get_info -- fill *info (host).  Synchronous (waits for the
 * build), cheap. */
lens_status lens_tree_get_info(const lens_tree* tree, lens_tree_info* info);

/*
 * lens_tree_export -- copy species s's tree to HOST arrays for inspection
 * (any pointer may be NULL to skip it).  Node order is breadth first.
 *   nodes: n_nodes x 8 floats (FP32 tree) or doubles (FP64 tree):
 *          {x_cm, y_cm, M, r_cut^2, Re Q2, Im Q2, side, level}
 *   links: n_nodes x 4 int32 {first child or first particle, count,
 *          is_leaf, big-list count}
 *   perm:  n particle indices in tree order (sorted index -> input index)
 *   listed: n int32, 1 where the particle (input order) sits in a big list
 * Synchronous.
 */
lens_status lens_tree_export(const lens_tree* tree, int32_t s, void* nodes, int32_t* links,
                             int32_t* perm, int32_t* listed);

/*
 * lens_tree_counters -- copy (and, if reset != 0, clear) the walk counters
 * accumulated by shooting calls made with LENS_COUNT.  Synchronous.
 *   out: HOST array of 8 int64:
 *     [0] ray groups walked        [1] boxes visited (MAC evaluated)
 *     [2] cells accepted           [3] leaf particles evaluated
 *     [4] big-list entries scanned [5] big-list entries kept for a group
 *     [6] ray-interactions evaluated: sum over groups of rays x (cells +
 *         leaf particles + kept big entries)   [7] reserved (0)
 * Counts are per species launch and summed over species.
 */
lens_status lens_tree_counters(lens_tree* tree, int64_t* out, int32_t reset);

/*
 * lens_last_timing -- device time of the last shooting call made with
 * LENS_TIMING, measured with CUDA events on its stream: grouping (ray sort
 * and group set-up) and walk (all species' walk or direct-sum kernels, from
 * the end of the stream's wait for the tree's build).
 * Synchronises on those events.  Both are 0 if no timed call was made.
 */
lens_status lens_last_timing(lens_tree* tree, double* group_ms, double* walk_ms);

/* lens_fp32_peak -- time a dependent-FFMA microbenchmark on every SM of the
 * current device for about `iters` FMAs per thread and return the achieved
 * FP32 rate in FLOP/s (FFMA = 2 flops) in *flops.  Synchronous. */
lens_status lens_fp32_peak(int64_t iters, double* flops, void* stream);

/* lens_fp64_peak -- the same microbenchmark with dependent FP64 DFMAs: the
 * achieved FP64 rate in FLOP/s (DFMA = 2 flops) in *flops.  Synchronous. */
lens_status lens_fp64_peak(int64_t iters, double* flops, void* stream);

/* lens_fail_allocations -- failure-injection hook for tests of the error
 * paths: the library's next `after` device allocations succeed and the one
 * after them fails as if the device were out of memory (the call that makes
 * it returns LENS_ERR_OOM and releases what it had allocated); after < 0
 * (the default) turns the hook off.  The hook then turns itself off.  It
 * affects every tree and thread of the process; it changes no setting of the
 * GPU. */
void lens_fail_allocations(int64_t after);

/* lens_kernel_launches -- number of CUDA kernels this library has launched
 * in the process so far (all trees, all threads); a CUDA-graph replay adds
 * the number of kernels the graph contains. */
int64_t lens_kernel_launches(void);

void lens_free_tree(lens_tree* tree);
const char* lens_status_string(lens_status s);
const char* lens_last_error(void);
int32_t lens_api_version(void);


/*
 * Image finding by adaptive grid refinement (Sec. 4) for uniform circular
 * sources, many at once.  Each source gets its own grid of n x n cells over
 * [x0, x0 + side] x [y0, y0 + side]; a cell (L, i, j) has side
 * h_L = side / (n 3^L) and is refined into its 9 thirds.  Per source:
 *   telescoping -- source radius r = h_0 / sqrt(mu_min), divided by 3 down
 *     to the source's R; at each r, cells whose source point
 *     y = x - alpha(x) lies within r of the source centre and whose side
 *     exceeds r sqrt(mu_min) / 3 are refined until none remain;
 *   images -- connected sets (cells sharing an edge) of cells whose point lies
 *     inside the source; inner border: image cells with a non-image
 *     neighbour, outer border: non-image cells with an image neighbour;
 *   uniform step -- while an image has fewer than n_min cells, its cells and
 *     its outer border are refined;
 *   border step -- until an image's largest border cell has area below
 *     f_area times the image's area and its outer border is as fine as its
 *     inner border, its border cells of the largest size are refined;
 * cells at level l_max are never refined (the minimum grid size).
 */
typedef struct lens_amr_params {
    double x0, y0, side;  /* the initial grid                                  */
    int32_t n;            /* initial cells per side, 1..4096                    */
    int32_t l_max;        /* level cap, 0..19                                   */
    double mu_min;        /* smallest |magnification| to find, (0, 1]          */
    double f_area;        /* stopping fraction of the border step (paper 5e-4)  */
    int32_t n_min;        /* cells per image after the uniform step (paper 50)  */
    int32_t max_rounds;   /* refinement rounds before giving up, 0: 10000       */
    int64_t max_cells;    /* leaf-cell capacity of the call, 0: 2^23            */
} lens_amr_params;

/* One image found by lens_find_images. */
typedef struct lens_image {
    int32_t source;   /* index of its source                                   */
    int32_t n_cells;  /* cells of the image                                    */
    double area;      /* sum of its cells' areas (per-level counts x h_L^2)    */
    double mu;        /* area / (pi R^2): its magnification                    */
    int64_t first;    /* smallest cell key of the image within its source:     */
                      /* (i0 n + j0) 9^l_max + the base-9 digits 3a + b of the  */
                      /* cell's refinements, padded to level l_max              */
} lens_image;

/*
 * lens_find_images -- the images and magnifications of n_sources uniform
 * circular sources through the tree's lens (deflections by lens_shoot_rays
 * in the tree's precision, ray positions in FP64).
 *   sources: host, 3 doubles per source {y_c1, y_c2, R}, R > 0.
 *   images: host, max_images records (caller-owned), ordered by source and
 *     then by first; *n_images receives the count.
 *   stats: host, 6 int64 or NULL: rays shot, final leaf cells, rounds, cells
 *     visited by the image-labelling passes (neighbours, union-find, labels,
 *     borders), their device time in ns, the shooting's device time in ns.
 * Limits: n_sources n^2 9^l_max < 2^63, n 3^l_max < 2^32.  Device memory:
 * about 150 bytes per cell of max_cells, kept with the tree for later calls
 * (grown when a call needs more) and freed by lens_free_tree.
 * Synchronous on stream (the refinement reads small counts back each round).
 * Errors: LENS_ERR_INVALID_ARG for bad parameters, more images than
 * max_images or more cells than max_cells; LENS_ERR_INTERNAL when max_rounds
 * runs out; LENS_ERR_OOM; shooting errors as lens_shoot_rays.
 */
lens_status lens_find_images(lens_tree* tree, const lens_amr_params* params, int32_t n_sources,
                             const double* sources, int32_t max_images, lens_image* images, int32_t* n_images,
                             int64_t* stats, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LENS_H */
