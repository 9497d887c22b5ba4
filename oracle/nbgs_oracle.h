/*
 * nbgs_oracle.h -- FP64 sequential CPU reference ("oracle") for one time step
 * of the hard-contact granular method of Preclik & Ruede, "Ultrascale
 * Simulations of Non-smooth Granular Dynamics" (arXiv:1501.05810).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path: only
 * the test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, header, table or helper with the
 * CUDA library; the two only see the same seeded input arrays.
 *
 * Everything is double precision, single-threaded and written for
 * readability: O(N^2) brute-force contact detection, a sequential greedy
 * colouring, and the nonlinear block Gauss-Seidel (NBGS) of Alg. 1, run
 * contact by contact in colour order: with a single subdomain (classic
 * NBGS), with subdomains on a grid, or with one subdomain per contact
 * (non-linear block Jacobi).
 *
 * Passages followed (section / equation / algorithm of the paper):
 *   Sect. 2, eq. (wrench) and the Q(phi) block  - wrench and quaternion rate
 *   Sect. 2, eq. (contactpos)                   - contact point, normal, gap
 *   Sect. 3, eq. (integrationscheme)            - semi-implicit Euler step
 *   Sect. 3, eq. (nonpenetration), eq. (coulomb)- one-contact constraints
 *   Sect. 4, eq. (expansionradius)              - intersection hulls
 *   Sect. 5, Alg. 1                             - subdomain NBGS, relaxation
 *   Sect. 6.2 (contact treatment rule)          - subdomain of a contact
 *   Sect. 6.3 (velocity accumulators and        - in-place velocity updates;
 *              corrections)                       per-subdomain corrections
 *   Sect. 6.6, Alg. 2                           - order of one time step
 *
 * Return codes: 0 = ok, 1 = invalid argument, 2 = out of memory.
 * All pointers are host pointers.  Arrays of 3-vectors are n x 3 row-major;
 * quaternions are n x 4 in (w, x, y, z) order.
 */
#ifndef NBGS_ORACLE_H
#define NBGS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_MAX_PLANES 16
#define ORACLE_MAX_CONES 4
#define ORACLE_MAX_MEMBERS 4   /* member spheres of a composite particle */

enum { ORACLE_WARM_NONE = 0, ORACLE_WARM_PREV = 1 };
/* Subdomains s_c(j) of Alg. 1: none (one subdomain: classic NBGS), a regular
 * grid over the box (a contact belongs to the subdomain holding the centre
 * of its body j1), or one subdomain per contact (non-linear block Jacobi). */
enum { ORACLE_SUB_NONE = 0, ORACLE_SUB_GRID = 1, ORACLE_SUB_JACOBI = 2 };

typedef struct oracle_params {
    double dt;          /* time step */
    double gravity[3];  /* external acceleration (force / mass) */
    double mu;          /* Coulomb friction coefficient, every contact */
    double omega;       /* relaxation parameter of Alg. 1 (1 = classic NBGS) */
    double tau;         /* hull safety margin of eq. (expansionradius) */
    double beta;        /* scale of the penetration-correction term, xi < 0 */
    double box_lo[3];   /* domain box; used for periodic wrapping only */
    double box_hi[3];
    int32_t periodic[3];
    int32_t warm_start; /* ORACLE_WARM_NONE or ORACLE_WARM_PREV */
    uint64_t colour_seed;
    int32_t subdomain_mode; /* ORACLE_SUB_* */
    int32_t subdomains[3];  /* grid of ORACLE_SUB_GRID, each >= 1 */
} oracle_params;

typedef struct oracle_step_stats {
    int64_t n_contacts;
    int32_t n_colours;
    int32_t sweeps_done;
    double residual;    /* R_k of the last sweep */
    double v_ref;
} oracle_step_stats;

typedef struct oracle_residuals {
    double non_penetration;   /* max_j max(0, -(xi'/dt + u_n)) / v_ref        */
    double cone;              /* max_j max(0, |p_to| - mu p_n) w_t / v_ref     */
    double complementarity;   /* max_j |min(w_n p_n, xi'/dt + u_n)| / v_ref    */
    double dissipation;       /* max_j | |u_to| p_to + mu p_n u_to | w_t/v_ref^2 */
} oracle_residuals;

typedef struct oracle_scene oracle_scene;

int  oracle_create_scene(const oracle_params* prm, int64_t n,
                         const double* pos, const double* vel, const double* angvel,
                         const double* radius, const double* density,
                         oracle_scene** out);
void oracle_destroy_scene(oracle_scene* s);
/* Half-space wall {y : n . y <= c}; n must be a unit vector pointing out of
 * the wall solid.  Walls are bodies of infinite mass with index n_bodies + k. */
int  oracle_add_plane(oracle_scene* s, const double n[3], double c);
/* Conical hopper wall: the frustum of the cone with apex `apex`, axis
 * `axis` (normalised here; the cone opens along it) and half-angle
 * half_angle (radians, in (0, pi/2)) between the orifice circle of radius
 * r_orifice and the top circle of radius r_top.  The solid lies outside the
 * cone; spheres inside touch its face or, below the face, the orifice rim.
 * sin and cos of the half-angle are taken with the C library.  Cones are
 * walls with index n_bodies + n_planes + k (planes are added first). */
int  oracle_add_cone(oracle_scene* s, const double apex[3], const double axis[3], double half_angle,
                     double r_orifice, double r_top);
/* Signed distance of x from cone k and the unit normal pointing from the
 * surface to x; returns 0 when x lies above the frustum (no contact), 1 on
 * the face, 2 at the rim.  Exported for the known-answer tests. */
int  oracle_cone_distance(const oracle_scene* s, int32_t k, const double x[3], double* sd, double n[3]);
/* Override inverse mass / inverse inertia (e.g. 0 = locked rotation). */
int  oracle_set_mass_properties(oracle_scene* s, const double* invm, const double* invI);
int  oracle_set_bodies(oracle_scene* s, const double* pos, const double* quat,
                       const double* vel, const double* angvel);
int  oracle_get_bodies(const oracle_scene* s, double* pos, double* quat,
                       double* vel, double* angvel);

int  oracle_detect_contacts(oracle_scene* s, int64_t* n_contacts);
int  oracle_colour_contacts(oracle_scene* s, int32_t* n_colours);
int  oracle_solve_nbgs(oracle_scene* s, int32_t max_sweeps, double tol,
                       int32_t* sweeps_done, double* residual);
int  oracle_integrate(oracle_scene* s);
int  oracle_step(oracle_scene* s, int32_t max_sweeps, double tol, oracle_step_stats* st);

/* Composite particles (Sect. 2, composites of convex particles): n rigid
 * bodies made of nm member spheres.  member_body (nm, non-decreasing, every
 * body 1..ORACLE_MAX_MEMBERS members), member_offset (nm x 3, from the
 * body's reference point pos, observational axes), member_radius (nm);
 * density > 0 (walls are the bodies of infinite mass).  Mass, centre of mass and inertia follow from the members (see the
 * definition); the body's position becomes its centre of mass and its
 * orientation the identity.  Contacts join members of different bodies
 * (j1 < j2 member indices) or a member and a wall (j2 = nm + k).  No cones,
 * subdomains, mass overrides or final residuals. */
int  oracle_create_composite_scene(const oracle_params* prm, int64_t n, const double* pos, const double* vel,
                                   const double* angvel, const double* density, int64_t nm,
                                   const int32_t* member_body, const double* member_offset,
                                   const double* member_radius, oracle_scene** out);
/* 1/m and the body-frame inertia about the centre of mass (n x 9) of every
 * composite body. */
int  oracle_body_mass_properties(const oracle_scene* s, double* invm, double* I0);
/* World positions of the members (nm x 3). */
int  oracle_member_positions(const oracle_scene* s, double* out);

/* Subdomain s_c(j) of every contact (canonical order) under the scene's
 * subdomain mode, from the current positions; 0 for every contact when
 * there are no subdomains. */
int  oracle_contact_subdomains(const oracle_scene* s, int64_t* out);

/* Contacts in canonical order (ascending (j1 << 32) | j2).  Any output
 * pointer may be NULL.  impulse = (p_n, p_t, p_o) in the contact frame. */
int  oracle_get_contacts(const oracle_scene* s, int64_t cap,
                         uint32_t* j1, uint32_t* j2, int32_t* colour,
                         double* normal, double* xi, double* impulse,
                         int64_t* n_out);
/* Overwrite the contact-frame impulses (canonical order, 3 per contact). */
int  oracle_set_impulses(oracle_scene* s, const double* impulse);
int  oracle_residual_history(const oracle_scene* s, double* out, int32_t cap,
                             int32_t* n_out);
int  oracle_final_residuals(const oracle_scene* s, oracle_residuals* out);

/* Unit-level pieces, exported for the known-answer tests. */
void     oracle_contact_frame(const double n[3], double t[3], double o[3]);
void     oracle_one_contact(double w_n, double w_t, double mu, const double b[3],
                            double p[3]);
uint64_t oracle_splitmix64(uint64_t x);
/* One-contact problem with a full symmetric Delassus block in the contact
 * frame, W = (Wnn, Wtt, Woo, Wnt, Wno, Wto): separation, sticking or
 * sliding (see the definition in nbgs_oracle.c).  Returns 0, or -1 when it
 * fell back to the diagonal solution. */
int      oracle_one_contact_general(const double W[6], double mu, const double b[3], double p[3]);

#ifdef __cplusplus
}
#endif
#endif
