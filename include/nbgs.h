/*
 * nbgs.h -- C ABI of the GB300 (sm_103a) hard-contact granular time step.
 *
 * One call of nbgs_step() advances a scene of spheres and half-space walls by
 * one time step of the method of Preclik & Ruede, "Ultrascale Simulations of
 * Non-smooth Granular Dynamics" (arXiv:1501.05810):
 *
 *   contact detection  (Sect. 4, eq. expansionradius, eq. contactpos)
 *   -> contact colouring (replaces the subdomain numbers s_c(j) of Alg. 1:
 *      contacts of one colour share no body of finite mass)
 *   -> nonlinear block Gauss-Seidel sweeps (Sect. 5, Alg. 1 with one
 *      subdomain and relaxation omega; one-contact problem of Sect. 3,
 *      eq. nonpenetration and eq. coulomb; in-place velocity accumulators
 *      of Sect. 6.3)
 *   -> semi-implicit Euler integration (Sect. 3, eq. integrationscheme)
 *
 * in the order of Alg. 2 (Sect. 6.6), all on the GPU.
 *
 * Conventions
 *   - Every function returns nbgs_status.  Nothing throws across the ABI.
 *   - Work is enqueued on the scene's CUDA stream and is asynchronous unless
 *     the function documents that it synchronises (it then returns host
 *     values or writes host memory).
 *   - Array arguments are double precision; 3-vectors are n x 3 row-major,
 *     quaternions n x 4 in (w, x, y, z) order.  Input and output pointers may
 *     be host or device memory (copied with cudaMemcpyDefault).
 *   - The scene owns every device buffer, allocated through the caller's
 *     allocator (or cudaMallocAsync on the scene stream when none is given).
 *     Inputs are copied; outputs are copies.
 *   - The first error sticks: later calls return it until the scene is
 *     destroyed; nbgs_last_error() returns its text.
 *   - A scene is not thread-safe.  Different scenes are independent.
 *   - Device-side failures (capacity overflow, NaN, a timed-out wait) are
 *     written to a device status word and reported by the next call that
 *     synchronises.
 */
#ifndef NBGS_H
#define NBGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum nbgs_status {
    NBGS_OK = 0,
    NBGS_EINVAL = 1,     /* bad argument or scene state                          */
    NBGS_ENOMEM = 2,     /* the allocator returned NULL                          */
    NBGS_ECUDA = 3,      /* a CUDA runtime call failed                           */
    NBGS_ECAPACITY = 4,  /* more contacts / colours than the buffers hold        */
    NBGS_ENOTCONV = 5,   /* tolerance not reached in max_sweeps; results valid   */
    NBGS_ENAN = 6,       /* a NaN or Inf appeared in the state                   */
    NBGS_ETIMEOUT = 7    /* a device-side wait gave up (grid barrier)            */
} nbgs_status;

enum { NBGS_FP64 = 0, NBGS_FP32 = 1 };           /* arithmetic of the sweeps      */
enum {                                           /* initial impulses of a solve */
    NBGS_WARM_NONE = 0,  /* zero (Alg. 1)                                                  */
    NBGS_WARM_PREV = 1,  /* the previous step's impulse of the same contact (Sect. 5)     */
    NBGS_WARM_MLP = 2    /* previous-step impulse; the network of nbgs_mlp_load for new contacts */
};
enum {                                           /* scheduling of the colour sweeps */
    NBGS_SOLVER_PERSISTENT = 0,  /* one cooperative launch per solve, grid barrier between colours */
    NBGS_SOLVER_PER_COLOUR = 1   /* one launch per colour and sweep                              */
};

enum {                                           /* nbgs_params.sweep_flags bits (persistent solver) */
    NBGS_SWEEP_GLOBAL_SYNC = 1,  /* grid barrier after every colour instead of waiting only for the
                                    blocks whose contacts share bodies with this block's contacts      */
    NBGS_SWEEP_TMA_STAGE = 2,    /* stage each block's chunk of the next colour (records, impulses)
                                    in shared memory with bulk copies while it waits                   */
    NBGS_SWEEP_WARP_SYNC = 4,    /* every warp has its own chunk, window and progress word, so the
                                    warps of a block do not wait for one another (no TMA staging)      */
    NBGS_SWEEP_GATHER2 = 8       /* a thread loads records, impulses and body states of two of its
                                    contacts of a colour before relaxing either (block scheduling, no
                                    TMA staging; three resident blocks per SM instead of four)         */
};

enum {                                           /* nbgs_params.subdomain_mode: s_c(j) of Alg. 1 */
    NBGS_SUB_NONE = 0,    /* one subdomain: classic NBGS in colour order                             */
    NBGS_SUB_GRID = 1,    /* a regular subdomains[0] x [1] x [2] grid over the box; a contact belongs
                             to the cell holding the centre of its body j1 (Sect. 6.2 lets any rule
                             that partitions the contacts decide, favouring the particles' parents):
                             k_a = floor((x_a - lo_a) g_a / (hi_a - lo_a)) clamped to [0, g_a - 1],
                             id = (k_2 g_1 + k_1) g_0 + k_0                                          */
    NBGS_SUB_JACOBI = 2   /* every contact its own subdomain: non-linear block Jacobi; the contacts
                             are not coloured (one colour)                                           */
};

typedef struct nbgs_allocator {
    void* ctx;
    void* (*alloc)(void* ctx, size_t bytes, void* stream); /* returns NULL on failure */
    void (*free)(void* ctx, void* ptr, void* stream);
} nbgs_allocator;

typedef struct nbgs_params {
    double dt;            /* time step                                              */
    double gravity[3];    /* external acceleration                                  */
    double mu;            /* Coulomb coefficient of every contact                   */
    double omega;         /* relaxation of Alg. 1, in (0, 2); 1 = classic NBGS      */
    double tau;           /* hull safety margin of eq. expansionradius, > 0         */
    double beta;          /* scale of the xi/dt term when xi < 0 (Sect. 3)          */
    double box_lo[3];     /* domain box: the cell grid spans it; periodic axes wrap */
    double box_hi[3];
    int32_t periodic[3];  /* 1 = periodic along this axis (needs >= 3 grid cells)   */
    int32_t precision;    /* NBGS_FP64 or NBGS_FP32 (positions are always FP64)     */
    int32_t warm_start;   /* NBGS_WARM_*                                            */
    int32_t solver;       /* NBGS_SOLVER_*                                          */
    uint64_t colour_seed; /* priorities of the colouring: splitmix64(key ^ seed)    */
    int32_t contacts_per_body; /* contact buffer capacity per body, 0 = default 8   */
    int32_t sweep_flags;  /* NBGS_SWEEP_*: scheduling details of the persistent solver */
    int32_t subdomain_mode;  /* NBGS_SUB_*.  With subdomains a contact sees, within a sweep,
                                the new reactions of the earlier contacts of its own subdomain
                                only and the previous sweep's of all others (Alg. 1; the
                                velocity accumulators and corrections of Sect. 6.3).  Single
                                scenes only (not nbgs_create_batch).                            */
    int32_t subdomains[3];   /* grid of NBGS_SUB_GRID, each >= 1, product < 2^31                 */
} nbgs_params;

typedef struct nbgs_step_stats {
    int64_t n_contacts;
    int32_t n_colours;
    int32_t sweeps_done;
    double residual;      /* R_k = max_j |velocity change at j| / v_ref, last sweep */
    double v_ref;         /* max(max_i |v_i| at step start, |g| dt, 1e-12)          */
} nbgs_step_stats;

typedef struct nbgs_residuals {  /* maxima over contacts, dimensionless (/ v_ref)  */
    double non_penetration;      /* max(0, -(xi'/dt + u_n))                         */
    double cone;                 /* max(0, |p_to| - mu p_n) w_t                     */
    double complementarity;      /* |min(w_n p_n, xi'/dt + u_n)|                    */
    double dissipation;          /* | |u_to| p_to + mu p_n u_to | w_t / v_ref^2     */
} nbgs_residuals;

typedef struct nbgs_scene nbgs_scene;

/* Create a scene of n spheres (Sect. 2: m = density 4/3 pi r^3,
 * I = 2/5 m r^2, quaternion (1,0,0,0)).  pos, vel, angvel: n x 3; radius,
 * density: n.  allocator may be NULL.  stream: a cudaStream_t or NULL for the
 * legacy default stream.  Synchronises.  n = 0 is allowed. */
nbgs_status nbgs_create_scene(const nbgs_params* params, int64_t n,
                              const double* pos, const double* vel, const double* angvel,
                              const double* radius, const double* density,
                              const nbgs_allocator* allocator, void* stream,
                              nbgs_scene** out);
void nbgs_destroy_scene(nbgs_scene* scene);
const char* nbgs_last_error(const nbgs_scene* scene);

/* Add a wall: the half-space solid {y : n . y <= c}, n a unit vector
 * pointing out of the solid (Sect. 6.4 "global bodies" of infinite mass).
 * Wall k gets body index n_bodies + k.  At most 16 walls. */
nbgs_status nbgs_add_plane(nbgs_scene* scene, const double n[3], double c);

/* Add a conical hopper wall (configuration 5 of the experiments built on
 * Sect. 7): the frustum of the cone with apex `apex`, axis `axis` (any
 * length; normalised here; the cone opens along it) and half-angle
 * half_angle (radians, 0 < half_angle < pi/2), between the orifice circle of
 * radius r_orifice and the top circle of radius r_top > r_orifice.  The
 * solid lies outside the cone.  A sphere inside touches its face; below the
 * face it touches the orifice rim; above the top circle it touches nothing.
 * The contact is a wall contact (infinite mass, Sect. 6.4) at the point of
 * the solid nearest the sphere's centre, whose normal is the direction from
 * that point to the centre (the cone's axis for a centre on the axis).
 * Cone k gets body index n_bodies + n_planes + k.  At most 4 cones; plain
 * scenes only (a batched scene returns NBGS_EINVAL). */
nbgs_status nbgs_add_cone(nbgs_scene* scene, const double apex[3], const double axis[3], double half_angle,
                          double r_orifice, double r_top);

/* Replace 1/m and/or 1/I of every sphere (n doubles each, NULL = keep).
 * 0 makes the quantity infinite (e.g. invI = 0 locks the rotation). */
nbgs_status nbgs_set_mass_properties(nbgs_scene* scene, const double* invm, const double* invI);

/* Overwrite / read the body state; NULL arrays are skipped.
 * nbgs_set_bodies starts a new history: the next solve has no previous-step
 * impulses to warm start from.  nbgs_get_bodies synchronises. */
nbgs_status nbgs_set_bodies(nbgs_scene* scene, const double* pos, const double* quat,
                            const double* vel, const double* angvel);
nbgs_status nbgs_get_bodies(nbgs_scene* scene, double* pos, double* quat,
                            double* vel, double* angvel);
/* Overwrite the body state as nbgs_set_bodies does, but continue the
 * history: the next solve warm starts from the impulses of the last one,
 * matched by contact key as after an ordinary step (Sect. 5).  For a caller
 * that reads the state back, changes it on the host (external forces, a
 * coupled code) and writes it again between steps; writing back unchanged
 * what nbgs_get_bodies returned leaves the next step exactly as without the
 * round trip.  NULL arrays are skipped; errors as for nbgs_set_bodies. */
nbgs_status nbgs_update_bodies(nbgs_scene* scene, const double* pos, const double* quat,
                               const double* vel, const double* angvel);

/* Sect. 4: hull radii h_i = dt(|v_i| + |w_i| r_i) + tau from the current
 * velocities, uniform cell grid sorted by radix sort, narrow phase
 * (sphere-sphere, sphere-wall, sphere-cone).  A pair is kept iff
 * (d - r_a) - r_b <= h_a + h_b (walls: h = tau).  Contacts are stored in
 * canonical order of (j1 << 32) | j2, j1 < j2.  With a warm start, the
 * contacts and impulses of the last solved step become the previous-step
 * contacts here (detecting again without a solve keeps them).  Synchronises
 * once to read the contact count (grows the buffers and retries on
 * overflow). */
nbgs_status nbgs_detect_contacts(nbgs_scene* scene, int64_t* n_contacts /* nullable */);

/* Jones-Plassmann colouring of the conflict graph (contacts sharing a body
 * of finite mass) with priorities splitmix64(key ^ colour_seed); equal to
 * sequential first-fit in decreasing priority.  With NBGS_SUB_JACOBI every
 * contact takes colour 0.  With subdomains it also assigns s_c(j) and the
 * velocity instances of the sweep.  Asynchronous unless n_colours is
 * non-NULL. */
nbgs_status nbgs_colour_contacts(nbgs_scene* scene, int32_t* n_colours /* nullable */);

/* One NBGS solve (Alg. 1): v += dt g, apply the initial impulses, then up to
 * max_sweeps sweeps over the colours; stop early once R_k <= tol (tol = 0:
 * exactly max_sweeps).  With subdomains each sweep ends by adding every
 * subdomain's velocity corrections to the bodies (Sect. 6.3).  Colours the
 * contacts first if needed.  Asynchronous unless sweeps_done or residual is
 * non-NULL.  Call once per step. */
nbgs_status nbgs_solve_nbgs(nbgs_scene* scene, int32_t max_sweeps, double tol,
                            int32_t* sweeps_done /* nullable */, double* residual /* nullable */);

/* eq. integrationscheme: x += dt v, q += dt Q(q) w, renormalise q, wrap
 * periodic axes into [lo, hi).  Asynchronous. */
nbgs_status nbgs_integrate(nbgs_scene* scene);

/* detect -> colour -> solve -> integrate (Alg. 2).  stats may be NULL
 * (then only the detection synchronises). */
nbgs_status nbgs_step(nbgs_scene* scene, int32_t max_sweeps, double tol, nbgs_step_stats* stats);

/* ------------------------------------------------------------------------
 * Batched scenes: S independent walled-box scenes stepped together in the
 * same kernels (one persistent sweep launch for all of them).  Bodies of
 * scene s are [body_offset[s], body_offset[s+1]) of the arrays given to
 * nbgs_create_batch; positions are in one common frame and the scene boxes
 * should not overlap (contacts never cross scenes either way; overlapping
 * boxes only cost detection time).  Each scene has six walls on the faces of
 * its box (after any nbgs_add_plane walls, which apply to every scene), its
 * own friction coefficient, its own v_ref and its own convergence test:
 * with tol > 0 the contacts of a scene are no longer relaxed once that
 * scene's R_k <= tol, so every scene ends exactly where a separate solve of
 * that scene alone would (colouring priorities use scene-local keys).
 * params.box_lo/box_hi must enclose every scene box; periodic axes are not
 * allowed.  The returned scene works with every other entry point.
 * ------------------------------------------------------------------------ */
typedef struct nbgs_batch_desc {
    int64_t n_scenes;
    const int64_t* body_offset;  /* n_scenes + 1, increasing, body_offset[0] = 0 */
    const double* box_lo;        /* n_scenes x 3 (host) */
    const double* box_hi;        /* n_scenes x 3 (host) */
    const double* mu;            /* n_scenes (host) */
} nbgs_batch_desc;

nbgs_status nbgs_create_batch(const nbgs_params* params, const nbgs_batch_desc* batch, int64_t n_bodies,
                              const double* pos, const double* vel, const double* angvel,
                              const double* radius, const double* density,
                              const nbgs_allocator* allocator, void* stream, nbgs_scene** out);

/* nbgs_step() plus per-scene results of its solve: sweeps_done[s] = sweeps
 * scene s took to reach tol (max_sweeps if it did not), residual[s] = its
 * R_k at that sweep.  Either output may be NULL (then nothing synchronises
 * beyond nbgs_step itself).  For a plain scene, S = 1. */
nbgs_status nbgs_batch_step(nbgs_scene* scene, int32_t max_sweeps, double tol, int32_t* sweeps_done,
                            double* residual);

/* n_steps time steps captured as CUDA graphs and replayed on the scene
 * stream, with no host synchronisation inside or between the steps (the
 * batched extension: thousands of scenes in one persistent sweep launch
 * under a captured graph).  Every step does what nbgs_step(max_sweeps, tol)
 * does, with device-sized launches: the contact count stays on the device,
 * the colouring rounds run in one cooperative launch, and the buffers keep
 * the capacities they had at capture (contacts: the capacity the last
 * nbgs_step left, at least contacts_per_body per body).  A step that needs
 * more sets an error
 * bit and the next synchronising call returns NBGS_ECAPACITY (take ordinary
 * nbgs_step calls then, which grow the buffers).  The first call, and any
 * call with other max_sweeps or tol or after the buffers grew, captures the
 * step first (two graphs, one for each parity of the warm-start buffers).
 * Needs one ordinary nbgs_step before (it sizes the buffers and starts the
 * warm-start history); sphere scenes or batches, the persistent solver, no
 * subdomains, no network warm start, timing off (else NBGS_EINVAL).  Results
 * equal those of nbgs_step.  Asynchronous: statistics, contacts and bodies
 * are read afterwards with the usual calls (nbgs_get_scene_stats,
 * nbgs_sync, ...), which synchronise and report device-side errors. */
nbgs_status nbgs_graph_step(nbgs_scene* scene, int32_t max_sweeps, double tol, int32_t n_steps);

/* Per-scene results of the last solve (see nbgs_batch_step).  Synchronises. */
nbgs_status nbgs_get_scene_stats(nbgs_scene* scene, int32_t* sweeps_done, double* residual);

/* Autotuner: times the solve of the current contacts (state saved and
 * restored) under every sweep schedule (point-to-point or grid-barrier
 * synchronisation, with or without shared-memory staging, warp-level units,
 * two contacts gathered per thread) and 1 to the maximum resident blocks
 * per SM, keeps the fastest, and returns its
 * sweep_flags and blocks per SM.  Call after nbgs_detect_contacts and
 * nbgs_colour_contacts.  Synchronises. */
nbgs_status nbgs_autotune(nbgs_scene* scene, int32_t max_sweeps, double tol, int32_t* sweep_flags,
                          int32_t* blocks_per_sm);

/* ------------------------------------------------------------------------
 * Learned warm start.  A 12 -> 64 -> 64 -> 64 -> 3 multilayer perceptron
 * with SiLU activations predicts each contact's converged impulse from
 * local features; the sweeps then start from it (Sect. 5: "any other
 * initialization can be used") and the NBGS residual judges it.  The paper
 * has no network; this is an extension of its warm start.
 *
 * Parameters: 9,347 FP32 values, for each layer W (out x in, row-major)
 * then b (out).  Features (12, dimensionless) in the frame n, e2, e3 with
 * e2 = -u_t / |u_t| along the free tangential relative velocity (the
 * contact frame's t when that is ~0), e3 = n x e2:
 *   u_n/v_ref, |u_t|/v_ref, (xi/dt)/v_ref, previous impulse in (n, e2, e3)
 *   times w_n/v_ref (3), log(w_n), w_t/w_n, r_a, r_b, mu,
 *   (contacts at j1 + contacts at j2)/12,
 * with u the relative velocity after the gravity kick and before any
 * impulse.  Output: the impulse in (n, e2, e3) times w_n/v_ref, formed as
 * inputs 3..5 (the previous impulse) plus the layers' correction (a skip
 * connection, added in FP32); it is projected onto the friction cone.  The
 * prediction is used for contacts that had no previous-step impulse (new
 * contacts); contacts with one keep it, as does a non-finite output.
 * ------------------------------------------------------------------------ */

/* Change the warm start of later solves (NBGS_WARM_*).  The previous-step
 * impulses are kept whenever the mode is not NBGS_WARM_NONE. */
nbgs_status nbgs_set_warm_start(nbgs_scene* scene, int32_t warm_start);

/* Copy the network into the scene (host or device pointer).  Required
 * before a solve with warm_start = NBGS_WARM_MLP. */
nbgs_status nbgs_mlp_load(nbgs_scene* scene, const float* theta, int64_t count /* 9347 */);

/* Features of the current contacts (after nbgs_colour_contacts, before the
 * solve): 16 floats per contact in canonical order -- the 12 inputs, then
 * cos and sin of the angle of e2 in the contact frame (t, o), w_n and v_ref,
 * to express a solved impulse in the network's frame and scale.  *n_out =
 * contact count; nothing is written when out is NULL or cap < count.
 * Synchronises. */
nbgs_status nbgs_mlp_features(nbgs_scene* scene, float* out, int64_t cap, int64_t* n_out);

/* Network on n rows of X (n x 12, device, 16-byte aligned, else
 * NBGS_EINVAL) -> Y (n x 3, device): evaluation
 * on the 5th-generation tensor cores (tcgen05, 128 rows per CTA, TMEM
 * accumulators), BF16 operands and FP32 accumulation.  theta: device
 * pointer.  Asynchronous on stream; rows of a tile whose tensor-core wait
 * gave up (never expected) are NaN. */
nbgs_status nbgs_mlp_infer(const float* theta, const float* X, float* Y, int64_t n, void* stream);

/* Training: loss L = sum((Y - T)^2) / (2 n) over n rows and its gradient
 * (FP32, device pointers; grad: 9347 floats, loss: one double, both
 * overwritten).  Asynchronous on stream. */
nbgs_status nbgs_mlp_grad(const float* theta, const float* X, const float* T, int64_t n, float* grad,
                          double* loss, void* stream);

/* One Adam step (Kingma & Ba) with bias correction for step >= 1; theta,
 * grad, m, v: count floats on the device.  Asynchronous on stream. */
nbgs_status nbgs_mlp_adam(float* theta, const float* grad, float* m, float* v, int64_t count, float lr,
                          float beta1, float beta2, float eps, int32_t step, void* stream);

/* Copy the contacts in canonical order.  Any output may be NULL; at most cap
 * contacts are written; *n_out receives the count.  impulse = (p_n, p_t, p_o)
 * of the last solve in the contact frame (n, t, o), t and o from the
 * orthonormal-basis construction of Duff et al. (JCGT 2017).  Synchronises. */
nbgs_status nbgs_get_contacts(nbgs_scene* scene, int64_t cap,
                              uint32_t* j1, uint32_t* j2, int32_t* colour,
                              double* normal, double* xi, double* impulse, int64_t* n_out);

/* Change the subdomains of later solves (NBGS_SUB_*; grid: three counts for
 * NBGS_SUB_GRID, may be NULL otherwise).  The contacts are coloured again
 * before the next solve.  NBGS_EINVAL for a bad mode or grid, or for any
 * subdomains on a batch. */
nbgs_status nbgs_set_subdomains(nbgs_scene* scene, int32_t mode, const int32_t* grid);

/* Composite particles (Sect. 2: non-convex objects as composites of convex
 * particles): n_bodies rigid bodies made of n_members member spheres.
 * pos, vel, angvel: n_bodies x 3 (pos is each body's reference point);
 * density: n_bodies, > 0; member_body: n_members, non-decreasing, every body with
 * 1..4 members; member_offset: n_members x 3, from the reference point along
 * the observational axes; member_radius: n_members.  All host pointers;
 * copied in.  The members' masses and inertias add up (an overlap counts for
 * every member it belongs to), m = sum density 4/3 pi r^3; the body's
 * position becomes its centre of mass X = sum m_m d_m / m and its body-frame
 * inertia about X is sum [2/5 m_m r_m^2 1 + m_m (|d'|^2 1 - d' d'^T)],
 * d' = d - X; the bounding radius max |d'| + r enters the hull of
 * eq. expansionradius; orientation starts at the identity.  Contacts join
 * members of different bodies (j1 < j2 member indices) or a member and a
 * wall (j2 = n_members + k); their levers are full vectors, so the
 * one-contact problem has a full 3x3 Delassus block: separation, sticking,
 * else the sliding root of the friction direction equation (a trigonometric
 * polynomial of degree 2, bracketed by 64 samples and refined by Newton
 * steps kept inside the bracket; the valid root of least 1/2 p.W p + b.p).
 * The velocity step adds the gyroscopic term -w x I w of
 * eq. integrationscheme.  nbgs_get_bodies and
 * nbgs_set_bodies take bodies (n_bodies rows, centres of mass); colours,
 * contacts and residual histories work as for spheres.  Not available for
 * composites: cones, nbgs_set_mass_properties, subdomains, the network warm
 * start, nbgs_final_residuals, checkpoints, nbgs_autotune, batches.
 * NBGS_EINVAL on bad arguments; synchronises. */
nbgs_status nbgs_create_composite_scene(const nbgs_params* params, int64_t n_bodies, const double* pos,
                                        const double* vel, const double* angvel, const double* density,
                                        int64_t n_members, const int32_t* member_body, const double* member_offset,
                                        const double* member_radius, const nbgs_allocator* allocator, void* stream,
                                        nbgs_scene** out);

/* Subdomain s_c(j) of every contact of the last colouring, canonical order
 * (NBGS_SUB_GRID: the grid cell id; NBGS_SUB_JACOBI: the contact's index;
 * NBGS_SUB_NONE: 0).  out may be NULL; at most cap values are written;
 * *n_out receives the contact count.  Synchronises. */
nbgs_status nbgs_get_subdomains(nbgs_scene* scene, int64_t cap, uint32_t* out, int64_t* n_out);

/* Checkpoint and resume.  The paper runs long simulations but says nothing
 * about saving them; these calls cover what a time step reads (Alg. 2):
 * the body state as the device holds it (FP64 positions and radii,
 * quaternions, velocities with 1/m and 1/I in the sweep precision,
 * finite-mass flags), the parameters, the shared walls, and the previous
 * step's contacts with their world-frame impulses, which the warm start of
 * Sect. 5 matches by key; plus the warm-start network if one is loaded.
 *
 * nbgs_save_state writes them to the file at path (a binary file in host
 * byte order, overwritten).  Synchronises.  Plain scenes only: a batched
 * scene returns NBGS_EINVAL.  A file error returns NBGS_EINVAL.
 *
 * nbgs_load_state restores such a file into a scene created with the same
 * body count, box, periodic axes and sweep precision (else NBGS_EINVAL,
 * before anything is copied); the steps that follow are bit-identical to
 * those of the scene that saved it.  A damaged file is refused the same way:
 * plane or cone counts beyond their arrays, parameters a scene could not be
 * created with, a non-finite largest radius or a radius beyond it, and
 * previous-step rows that do not rise from 0 to the stored contact count.  The parameters stored in the file
 * replace the scene's.  Synchronises.  Every error sticks in the scene, as
 * for the other calls. */
nbgs_status nbgs_save_state(nbgs_scene* scene, const char* path);
nbgs_status nbgs_load_state(nbgs_scene* scene, const char* path);

/* The one-contact problem of Sect. 3 (eq. nonpenetration and eq. coulomb
 * for one contact, the others' reactions frozen) with a full symmetric
 * Delassus block, solved on the GPU for n independent contacts by the same
 * solver the composite sweep relaxes every contact with: separation, then
 * sticking p = -W^-1 b if inside the friction cone, else sliding on the
 * cone with the friction direction against the tangential velocity, the
 * least-energy slide where several qualify.  Device pointers: W6 n x 6
 * (W_nn, W_tt, W_oo, W_nt, W_no, W_to in the contact frame), mu n, b n x 3
 * (the contact's velocity without its own reaction, plus the gap term), p
 * n x 3 out (impulse in the contact frame).  Enqueued on `stream`.
 * NBGS_EINVAL on bad arguments, NBGS_ECUDA if the launch fails. */
nbgs_status nbgs_one_contact(int64_t n, const double* W6, const double* mu, const double* b, double* p,
                             void* stream);

/* Sphere contact geometry of Sect. 2 eq. (contactpos) as the detection
 * computes it, for n centre differences x_i - x_j: the distance
 * d = |x_i - x_j| (the square root of the squares summed in x, y, z order)
 * and the unit normal n = (x_i - x_j) / d, every operation rounded to
 * nearest (the quotients through one correctly rounded reciprocal of d and
 * a fused correction step, which gives the correctly rounded quotient);
 * coincident centres give n = (0, 0, 1).  Device pointers: dvec n x 3 in,
 * out n x 4 (n_x, n_y, n_z, d).  Enqueued on `stream`.  NBGS_EINVAL on bad
 * arguments, NBGS_ECUDA if the launch fails. */
nbgs_status nbgs_pair_normals(int64_t n, const double* dvec, double* out, void* stream);

/* R_k of every sweep of the last solve.  Synchronises. */
nbgs_status nbgs_residual_history(nbgs_scene* scene, double* out, int32_t cap, int32_t* n_out);

/* FP64 residuals of eq. nonpenetration and eq. coulomb at the current
 * velocities and impulses.  Synchronises. */
nbgs_status nbgs_final_residuals(nbgs_scene* scene, nbgs_residuals* out);

/* Replace the impulses of the current contacts (Sect. 5: Alg. 1 may start
 * from any reactions; Sect. 3: p = dt lambda).  impulse: n_contacts x 3
 * doubles, host or device memory, in the canonical contact order of
 * nbgs_get_contacts() and in the contact frame (n, t, o); n_contacts is the
 * count of the last nbgs_detect_contacts().  The values are copied: they
 * become what nbgs_get_contacts() and nbgs_final_residuals() read and the
 * previous-step impulses the next step's warm start matches.  Sphere scenes
 * (and batches) after a solve of the current contacts, else NBGS_EINVAL;
 * NBGS_ENOMEM if the staging buffer cannot be allocated.  Synchronises. */
nbgs_status nbgs_set_impulses(nbgs_scene* scene, const double* impulse);

/* Allocation-free variant of nbgs_final_residuals() for callers that cannot
 * allocate device memory (fixed arenas, plugins handed only buffers,
 * processes whose allocator belongs to someone else).  The paper has no
 * counterpart: this entry point only repackages the residual evaluation.
 *
 * Inputs are device pointers in the layout nbgs_get_contacts() and
 * nbgs_get_bodies() produce: j1, j2 (n_contacts; j2 >= n_bodies marks a
 * wall), normal (n_contacts x 3), xi (n_contacts), impulse (n_contacts x 3,
 * contact frame), vel and angvel (n_bodies x 3), radius, invm, invI
 * (n_bodies).  dt, beta, mu and v_ref as in the scene and its step stats:
 * one mu and one v_ref for all contacts, so the contacts of one sphere scene
 * (not of a batch, whose scenes have their own mu and v_ref; composites are
 * refused by nbgs_final_residuals as well).  Maxima above 1e300 and NaN are
 * reported as +inf, as nbgs_final_residuals() does.
 * out: device pointer to 4 doubles, written in nbgs_residuals order.
 * Enqueued on `stream` (a cudaStream_t, NULL = legacy default stream).
 *
 * Scratch is a file-scope device array of 32 KiB held by every GPU that
 * loads the library until the process exits; no memory is allocated.
 * n_contacts may not exceed 2,097,152 (NBGS_ECAPACITY otherwise).  The
 * first call on a device looks up the array's address (cudaGetSymbolAddress)
 * with that device current: make that first call before any stream capture.
 * Every later call on a stream that is not capturing looks it up again (so a
 * device reset that reloads the library's module is followed).
 * All calls share the array, so calls that overlap on the GPU (different
 * streams, or different host threads on one device) race and may return
 * wrong maxima; serialise them.  Returns NBGS_EINVAL on bad arguments and
 * NBGS_ECUDA if a launch fails. */
nbgs_status nbgs_final_residuals_noalloc(int64_t n_bodies, int64_t n_contacts, const uint32_t* j1,
                                         const uint32_t* j2, const double* normal, const double* xi,
                                         const double* impulse, const double* vel, const double* angvel,
                                         const double* radius, const double* invm, const double* invI,
                                         double dt, double beta, double mu, double v_ref, double* out,
                                         void* stream);

/* Contact updates since the scene was created or this call last read
 * them: every contact relaxed once per sweep its scene ran (a scene of a
 * batch stops at its own tolerance), counted on the device, so that graph
 * steps need no host read per step.  Reads and resets.  Synchronises. */
nbgs_status nbgs_get_updates(nbgs_scene* scene, int64_t* updates);

/* Wait for the scene's stream and report device-side errors. */
nbgs_status nbgs_sync(nbgs_scene* scene);

/* Device time of the phases of the calls since the last reset, measured
 * with CUDA events on the scene stream when timing is enabled:
 * ms[0] detect, ms[1] colour, ms[2] solve (everything nbgs_solve_nbgs
 * enqueues), ms[3] integrate, ms[4] the sweep kernels alone (the
 * persistent launch, or the per-colour launches); launches[k] counts the
 * kernel launches of each.  nbgs_get_timings synchronises and resets. */
nbgs_status nbgs_enable_timing(nbgs_scene* scene, int32_t on);
nbgs_status nbgs_get_timings(nbgs_scene* scene, double ms[5], int64_t launches[5]);

#ifdef __cplusplus
}
#endif
#endif
