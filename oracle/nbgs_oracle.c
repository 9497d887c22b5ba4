/*
 * nbgs_oracle.c -- FP64 sequential CPU reference of one NBGS time step.
 *
 * TEST INFRASTRUCTURE ONLY (see nbgs_oracle.h).  Plain, slow and written to
 * be read next to the paper.  Compile with -ffp-contract=off: the hull
 * predicate that decides which contacts exist must round exactly as written.
 */
#include "nbgs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct oracle_scene {
    oracle_params prm;
    int64_t n;                     /* spheres */
    double *x, *q, *v, *w;         /* position, quaternion (w,x,y,z), velocity, angular velocity */
    double *r, *invm, *invI;       /* radius, 1/m, 1/I (sphere: I = 2/5 m r^2) */
    double *h;                     /* hull expansion radius of this step */
    int32_t nplanes;
    double plane_n[ORACLE_MAX_PLANES][3];
    double plane_c[ORACLE_MAX_PLANES];
    int32_t ncones;
    struct {
        double apex[3], axis[3];
        double sa, ca;           /* sin, cos of the half-angle */
        double s_o, s_t;         /* orifice and top along a generatrix, from the apex */
    } cone[ORACLE_MAX_CONES];

    /* contacts of the current step, canonical order */
    int64_t nc, cap;
    uint32_t *j1, *j2;
    double *cn;                    /* normal, 3 per contact */
    double *xi;                    /* signed distance */
    double *la, *lb;               /* lever lengths: l_a = -la n, l_b = lb n */
    int32_t *colour;
    double *p;                     /* contact-frame impulse (p_n, p_t, p_o) = dt * lambda */
    int32_t ncolours;
    int coloured;

    /* previous step's contacts for the warm start (canonical keys, world impulse) */
    int64_t nprev;
    uint64_t *prev_key;
    double *prev_P;

    int64_t* sub;                  /* s_c(j) the last solve used (NULL: none since the detection) */

    /* composite particles (Sect. 2: composites of convex particles): bodies
     * are rigid unions of member spheres; contacts join members of different
     * bodies, j1/j2 are member indices and walls follow the members */
    int composite;
    int64_t nm;                    /* member spheres */
    int32_t* mbody;                /* body of each member, non-decreasing */
    double *moff, *mr;             /* body-frame offset from the centre of mass (3 per member), radius */
    double *I0, *I0inv;            /* body-frame inertia about the centre of mass, and its inverse (9 per body) */

    double vmax_start;             /* max_i |v_i| at the start of the step */
    double v_ref;
    double *hist;                  /* R_k per sweep */
    int32_t nhist, cap_hist;
};

/* ------------------------------------------------------------------ */
/* small vector helpers                                                 */
/* ------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Body that contact end j acts on (a sphere, or the body of a member of a
 * composite), -1 for a wall. */
static int64_t end_body(const oracle_scene* s, uint32_t j)
{
    if (s->composite) return (int64_t)j < s->nm ? (int64_t)s->mbody[j] : -1;
    return (int64_t)j < s->n ? (int64_t)j : -1;
}

static int is_finite_body(const oracle_scene* s, uint32_t j)
{
    int64_t i = end_body(s, j);
    return i >= 0 && (s->invm[i] > 0.0 || s->invI[i] > 0.0);
}

/* splitmix64 (Steele, Lea & Flood, OOPSLA 2014; Vigna's reference
 * formulation): one step of the Weyl sequence followed by the mix. */
uint64_t oracle_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Orthonormal tangent basis (t, o) of a unit normal n: the branchless
 * construction of Duff et al., "Building an Orthonormal Basis, Revisited"
 * (JCGT 6(1), 2017).  Sect. 2 only requires that t and o span the
 * tangential plane; this fixes which pair is used. */
void oracle_contact_frame(const double n[3], double t[3], double o[3])
{
    double sign = copysign(1.0, n[2]);
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    t[0] = 1.0 + sign * n[0] * n[0] * a;
    t[1] = sign * b;
    t[2] = -sign * n[0];
    o[0] = b;
    o[1] = sign + n[1] * n[1] * a;
    o[2] = -n[1];
}

/* One-contact problem F_j^{-1}(0, lambda_jbar) of Sect. 3 for a contact
 * whose Delassus block in the contact frame is diag(w_n, w_t, w_t).
 * b = post-velocity of the contact without its own reaction, normal
 * component including the gap term xi'/dt.  Output p satisfies
 *   b_n + w_n p_n >= 0  _|_  p_n >= 0                 (eq. nonpenetration)
 *   |p_to| <= mu p_n,  |u_to| p_to = -mu p_n u_to     (eq. coulomb)
 * with u = b + W p.  The normal part decouples because W is diagonal; the
 * tangential part is the stick impulse, or its radial projection onto the
 * friction disk when the stick impulse lies outside it. */
void oracle_one_contact(double w_n, double w_t, double mu, const double b[3], double p[3])
{
    double pn = -b[0] / w_n;
    if (!(pn > 0.0)) pn = 0.0;
    double pt = -b[1] / w_t;
    double po = -b[2] / w_t;
    double lim = mu * pn;
    double len = sqrt(pt * pt + po * po);
    if (len > lim) {
        if (len > 0.0) {
            pt = pt * (lim / len);
            po = po * (lim / len);
        } else {
            pt = 0.0;
            po = 0.0;
        }
    }
    p[0] = pn;
    p[1] = pt;
    p[2] = po;
}

/* One-contact problem with a full symmetric Delassus block W (contact frame
 * (n, t, o); W[0..5] = Wnn, Wtt, Woo, Wnt, Wno, Wto), as composite particles
 * give it (levers not parallel to n).  Find p with u = W p + b satisfying
 * eq. (nonpenetration) and eq. (coulomb):
 *   1. separation: p = 0 is a solution whenever b_n >= 0, and is taken then;
 *   2. sticking: u = 0, p = -W^-1 b, if p_n > 0 and |p_to| <= mu p_n;
 *   3. sliding: p = p_n (1, mu cos th, mu sin th) with u_n = 0, so
 *      p_n = -b_n / D(th), D = Wnn + mu (Wnt cos th + Wno sin th) > 0, and
 *      u_to antiparallel to (cos th, sin th).  Parallel: the cross product of
 *      (cos th, sin th) with D u_to vanishes, a trigonometric polynomial of
 *      degree 2 in th (a quartic in tan(th/2), the route of Bonnefon et al.
 *      cited in Sect. 3).  Its roots are bracketed by 64 equal samples of
 *      [0, 2 pi) and refined by 60 bisections; a root is a solution if D > 0
 *      and u_to points against (cos th, sin th).  Where several are, the one
 *      of least 1/2 p.W p + b.p is taken (first in th on ties).
 * For diagonal W with Wtt = Woo this is exactly oracle_one_contact.  Should
 * no sliding root qualify (a double root the samples cannot bracket), the
 * diagonal solution with w_n = Wnn, w_t = (Wtt + Woo)/2 is returned and the
 * result is -1 (0 otherwise). */
static void w_full(const double W[6], double M[3][3])
{
    M[0][0] = W[0]; M[1][1] = W[1]; M[2][2] = W[2];
    M[0][1] = M[1][0] = W[3];
    M[0][2] = M[2][0] = W[4];
    M[1][2] = M[2][1] = W[5];
}

/* D(th) u_to(th) for p = p_n (1, mu c, mu s), p_n = -b_n / D */
static void slide_dut(double M[3][3], double mu, const double b[3], double c, double s, double* D, double* vt,
                      double* vo)
{
    *D = M[0][0] + mu * (M[0][1] * c + M[0][2] * s);
    *vt = -b[0] * (M[1][0] + mu * (M[1][1] * c + M[1][2] * s)) + *D * b[1];
    *vo = -b[0] * (M[2][0] + mu * (M[2][1] * c + M[2][2] * s)) + *D * b[2];
}

static double slide_g(double M[3][3], double mu, const double b[3], double th)
{
    double D, vt, vo, c = cos(th), s = sin(th);
    slide_dut(M, mu, b, c, s, &D, &vt, &vo);
    return -s * vt + c * vo;
}

static double energy(double M[3][3], const double b[3], const double p[3])
{
    double e = 0.0;
    for (int i = 0; i < 3; ++i) {
        double wp = (M[i][0] * p[0] + M[i][1] * p[1]) + M[i][2] * p[2];
        e += p[i] * (0.5 * wp + b[i]);
    }
    return e;
}

int oracle_one_contact_general(const double W[6], double mu, const double b[3], double p[3])
{
    double M[3][3];
    w_full(W, M);
    p[0] = p[1] = p[2] = 0.0;
    if (b[0] >= 0.0) return 0;
    /* sticking: W p = -b by Cramer's rule (W is symmetric positive definite) */
    double c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1];
    double c01 = M[1][2] * M[2][0] - M[1][0] * M[2][2];
    double c02 = M[1][0] * M[2][1] - M[1][1] * M[2][0];
    double det = (M[0][0] * c00 + M[0][1] * c01) + M[0][2] * c02;
    double inv[3][3] = {
        { c00, M[0][2] * M[2][1] - M[0][1] * M[2][2], M[0][1] * M[1][2] - M[0][2] * M[1][1] },
        { c01, M[0][0] * M[2][2] - M[0][2] * M[2][0], M[0][2] * M[1][0] - M[0][0] * M[1][2] },
        { c02, M[0][1] * M[2][0] - M[0][0] * M[2][1], M[0][0] * M[1][1] - M[0][1] * M[1][0] },
    };
    double ps[3];
    for (int i = 0; i < 3; ++i) ps[i] = -((inv[i][0] * b[0] + inv[i][1] * b[1]) + inv[i][2] * b[2]) / det;
    if (ps[0] > 0.0 && sqrt(ps[1] * ps[1] + ps[2] * ps[2]) <= mu * ps[0]) {
        p[0] = ps[0]; p[1] = ps[1]; p[2] = ps[2];
        return 0;
    }
    /* sliding */
    const int K = 64;
    const double two_pi = 6.283185307179586;
    double best = 0.0;
    int found = 0;
    double g0 = slide_g(M, mu, b, 0.0);
    for (int k = 0; k < K; ++k) {
        double lo = two_pi * k / K, hi = two_pi * (k + 1) / K;
        double glo = k == 0 ? g0 : slide_g(M, mu, b, lo);
        double ghi = k + 1 == K ? g0 : slide_g(M, mu, b, hi);
        double th;
        if (glo == 0.0) th = lo;
        else if ((glo < 0.0) != (ghi < 0.0) && ghi != 0.0) {
            for (int it = 0; it < 60; ++it) {
                double mid = 0.5 * (lo + hi);
                double gm = slide_g(M, mu, b, mid);
                if ((gm < 0.0) == (glo < 0.0)) { lo = mid; glo = gm; }
                else hi = mid;
            }
            th = 0.5 * (lo + hi);
        } else continue;
        double c = cos(th), s = sin(th), D, vt, vo;
        slide_dut(M, mu, b, c, s, &D, &vt, &vo);
        if (!(D > 0.0) || c * vt + s * vo > 0.0) continue;
        double pn = -b[0] / D;
        double q[3] = { pn, mu * pn * c, mu * pn * s };
        double e = energy(M, b, q);
        if (!found || e < best) {
            best = e;
            p[0] = q[0]; p[1] = q[1]; p[2] = q[2];
            found = 1;
        }
    }
    if (found) return 0;
    oracle_one_contact(W[0], 0.5 * (W[1] + W[2]), mu, b, p);
    return -1;
}

/* ------------------------------------------------------------------ */
/* scene lifecycle                                                      */
/* ------------------------------------------------------------------ */
void oracle_destroy_scene(oracle_scene* s)
{
    if (!s) return;
    free(s->x); free(s->q); free(s->v); free(s->w);
    free(s->r); free(s->invm); free(s->invI); free(s->h);
    free(s->j1); free(s->j2); free(s->cn); free(s->xi); free(s->la); free(s->lb);
    free(s->colour); free(s->p);
    free(s->prev_key); free(s->prev_P);
    free(s->hist);
    free(s->sub);
    free(s->mbody); free(s->moff); free(s->mr); free(s->I0); free(s->I0inv);
    free(s);
}

int oracle_create_scene(const oracle_params* prm, int64_t n,
                        const double* pos, const double* vel, const double* angvel,
                        const double* radius, const double* density,
                        oracle_scene** out)
{
    if (!prm || !out || n < 0 || (n > 0 && (!pos || !vel || !angvel || !radius || !density))) return 1;
    if (!(prm->dt > 0.0)) return 1;
    if (prm->subdomain_mode < ORACLE_SUB_NONE || prm->subdomain_mode > ORACLE_SUB_JACOBI) return 1;
    if (prm->subdomain_mode == ORACLE_SUB_GRID)
        for (int a = 0; a < 3; ++a)
            if (prm->subdomains[a] < 1 || !(prm->box_hi[a] > prm->box_lo[a])) return 1;
    oracle_scene* s = (oracle_scene*)calloc(1, sizeof(oracle_scene));
    if (!s) return 2;
    s->prm = *prm;
    s->n = n;
    size_t m = (size_t)(n > 0 ? n : 1);
    s->x = (double*)malloc(3 * m * sizeof(double));
    s->q = (double*)malloc(4 * m * sizeof(double));
    s->v = (double*)malloc(3 * m * sizeof(double));
    s->w = (double*)malloc(3 * m * sizeof(double));
    s->r = (double*)malloc(m * sizeof(double));
    s->invm = (double*)malloc(m * sizeof(double));
    s->invI = (double*)malloc(m * sizeof(double));
    s->h = (double*)malloc(m * sizeof(double));
    s->cap_hist = 64;
    s->hist = (double*)malloc((size_t)s->cap_hist * sizeof(double));
    if (!s->x || !s->q || !s->v || !s->w || !s->r || !s->invm || !s->invI || !s->h || !s->hist) {
        oracle_destroy_scene(s);
        return 2;
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) {
            s->x[3 * i + k] = pos[3 * i + k];
            s->v[3 * i + k] = vel[3 * i + k];
            s->w[3 * i + k] = angvel[3 * i + k];
        }
        s->q[4 * i + 0] = 1.0;
        s->q[4 * i + 1] = 0.0;
        s->q[4 * i + 2] = 0.0;
        s->q[4 * i + 3] = 0.0;
        s->r[i] = radius[i];
        /* Sect. 2: block-diagonal mass matrix; a homogeneous sphere has
         * m = rho 4/3 pi r^3 and the isotropic inertia I = 2/5 m r^2. */
        double mass = density[i] * (4.0 / 3.0) * M_PI * radius[i] * radius[i] * radius[i];
        double inertia = 0.4 * mass * radius[i] * radius[i];
        s->invm[i] = mass > 0.0 ? 1.0 / mass : 0.0;
        s->invI[i] = inertia > 0.0 ? 1.0 / inertia : 0.0;
    }
    *out = s;
    return 0;
}

int oracle_add_cone(oracle_scene* s, const double apex[3], const double axis[3], double half_angle,
                    double r_orifice, double r_top)
{
    if (!s || !apex || !axis || s->ncones >= ORACLE_MAX_CONES || s->composite) return 1;
    if (!(half_angle > 0.0 && half_angle < 1.5707963267948966) || !(r_orifice >= 0.0) || !(r_top > r_orifice))
        return 1;
    double len = sqrt((axis[0] * axis[0] + axis[1] * axis[1]) + axis[2] * axis[2]);
    if (!(len > 0.0)) return 1;
    int k = s->ncones++;
    for (int d = 0; d < 3; ++d) {
        s->cone[k].apex[d] = apex[d];
        s->cone[k].axis[d] = axis[d] / len;
    }
    s->cone[k].sa = sin(half_angle);
    s->cone[k].ca = cos(half_angle);
    s->cone[k].s_o = r_orifice / s->cone[k].sa;
    s->cone[k].s_t = r_top / s->cone[k].sa;
    return 0;
}

/* Distance from x to the frustum, worked in the half-plane through the axis
 * and x: zeta = height of x above the apex along the axis, rho = distance
 * from the axis, e = unit radial direction.  A generatrix runs along
 * g = (sin a, cos a) in (rho, zeta); the face is the segment s in [s_o, s_t]
 * of it, the solid lies on the outer side, and the inward unit normal of the
 * face is (-cos a, sin a).  Position along the generatrix of the foot of x:
 * s = rho sin a + zeta cos a.  Face (s_o <= s <= s_t): signed distance
 * zeta sin a - rho cos a, normal -cos a e + sin a axis.  Below the face
 * (s < s_o) the nearest point of the solid is on the orifice rim, the circle
 * (rho_o, zeta_o) = s_o (sin a, cos a): distance |(rho - rho_o, zeta - zeta_o)|,
 * normal along that difference.  On the axis (rho = 0) e is undefined: the
 * face distance is kept and the normal is the axis. */
int oracle_cone_distance(const oracle_scene* s, int32_t k, const double x[3], double* sd, double n[3])
{
    const double* A = s->cone[k].apex;
    const double* ax = s->cone[k].axis;
    const double sa = s->cone[k].sa, ca = s->cone[k].ca;
    double d[3], e[3];
    for (int i = 0; i < 3; ++i) d[i] = x[i] - A[i];
    double zeta = (d[0] * ax[0] + d[1] * ax[1]) + d[2] * ax[2];
    for (int i = 0; i < 3; ++i) e[i] = d[i] - zeta * ax[i];
    double rho = sqrt((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]);
    double s_gen = rho * sa + zeta * ca;
    if (s_gen > s->cone[k].s_t) return 0;
    if (rho > 0.0)
        for (int i = 0; i < 3; ++i) e[i] = e[i] / rho;
    if (s_gen >= s->cone[k].s_o) {
        *sd = zeta * sa - rho * ca;
        for (int i = 0; i < 3; ++i) n[i] = rho > 0.0 ? sa * ax[i] - ca * e[i] : ax[i];
        return 1;
    }
    double drho = rho - s->cone[k].s_o * sa, dzeta = zeta - s->cone[k].s_o * ca;
    double dist = sqrt(drho * drho + dzeta * dzeta);
    *sd = dist;
    for (int i = 0; i < 3; ++i) {
        if (dist > 0.0 && rho > 0.0) n[i] = (drho * e[i] + dzeta * ax[i]) / dist;
        else n[i] = ax[i];
    }
    return 2;
}

int oracle_add_plane(oracle_scene* s, const double n[3], double c)
{
    if (!s || !n || s->nplanes >= ORACLE_MAX_PLANES) return 1;
    int k = s->nplanes++;
    s->plane_n[k][0] = n[0];
    s->plane_n[k][1] = n[1];
    s->plane_n[k][2] = n[2];
    s->plane_c[k] = c;
    return 0;
}

int oracle_set_mass_properties(oracle_scene* s, const double* invm, const double* invI)
{
    if (!s || s->composite) return 1;
    for (int64_t i = 0; i < s->n; ++i) {
        if (invm) s->invm[i] = invm[i];
        if (invI) s->invI[i] = invI[i];
    }
    return 0;
}

int oracle_set_bodies(oracle_scene* s, const double* pos, const double* quat,
                      const double* vel, const double* angvel)
{
    if (!s) return 1;
    if (pos) memcpy(s->x, pos, 3 * (size_t)s->n * sizeof(double));
    if (quat) memcpy(s->q, quat, 4 * (size_t)s->n * sizeof(double));
    if (vel) memcpy(s->v, vel, 3 * (size_t)s->n * sizeof(double));
    if (angvel) memcpy(s->w, angvel, 3 * (size_t)s->n * sizeof(double));
    return 0;
}

int oracle_get_bodies(const oracle_scene* s, double* pos, double* quat, double* vel, double* angvel)
{
    if (!s) return 1;
    if (pos) memcpy(pos, s->x, 3 * (size_t)s->n * sizeof(double));
    if (quat) memcpy(quat, s->q, 4 * (size_t)s->n * sizeof(double));
    if (vel) memcpy(vel, s->v, 3 * (size_t)s->n * sizeof(double));
    if (angvel) memcpy(angvel, s->w, 3 * (size_t)s->n * sizeof(double));
    return 0;
}

/* ------------------------------------------------------------------ */
/* contact detection (Sect. 4), brute force over all pairs              */
/* ------------------------------------------------------------------ */
static int push_contact(oracle_scene* s, uint32_t a, uint32_t b, const double nrm[3],
                        double xi, double la, double lb)
{
    if (s->nc == s->cap) {
        int64_t nc = s->cap ? 2 * s->cap : 1024;
        uint32_t* j1 = (uint32_t*)realloc(s->j1, (size_t)nc * sizeof(uint32_t));
        if (j1) s->j1 = j1;
        uint32_t* j2 = (uint32_t*)realloc(s->j2, (size_t)nc * sizeof(uint32_t));
        if (j2) s->j2 = j2;
        double* cn = (double*)realloc(s->cn, 3 * (size_t)nc * sizeof(double));
        if (cn) s->cn = cn;
        double* xv = (double*)realloc(s->xi, (size_t)nc * sizeof(double));
        if (xv) s->xi = xv;
        double* lav = (double*)realloc(s->la, (size_t)nc * sizeof(double));
        if (lav) s->la = lav;
        double* lbv = (double*)realloc(s->lb, (size_t)nc * sizeof(double));
        if (lbv) s->lb = lbv;
        int32_t* col = (int32_t*)realloc(s->colour, (size_t)nc * sizeof(int32_t));
        if (col) s->colour = col;
        double* pv = (double*)realloc(s->p, 3 * (size_t)nc * sizeof(double));
        if (pv) s->p = pv;
        if (!j1 || !j2 || !cn || !xv || !lav || !lbv || !col || !pv) return 2;
        s->cap = nc;
    }
    int64_t k = s->nc++;
    s->j1[k] = a;
    s->j2[k] = b;
    s->cn[3 * k + 0] = nrm[0];
    s->cn[3 * k + 1] = nrm[1];
    s->cn[3 * k + 2] = nrm[2];
    s->xi[k] = xi;
    s->la[k] = la;
    s->lb[k] = lb;
    s->colour[k] = -1;
    s->p[3 * k + 0] = 0.0;
    s->p[3 * k + 1] = 0.0;
    s->p[3 * k + 2] = 0.0;
    return 0;
}

static int detect_composite(oracle_scene* s);

int oracle_detect_contacts(oracle_scene* s, int64_t* n_contacts)
{
    if (!s) return 1;
    const oracle_params* P = &s->prm;
    const double dt = P->dt;
    free(s->sub);   /* new contacts: no subdomains assigned yet */
    s->sub = NULL;
    if (s->composite) {
        int rc = detect_composite(s);
        if (rc == 0 && n_contacts) *n_contacts = s->nc;
        return rc;
    }

    /* eq. (expansionradius): h_i = dt (|v_i| + |omega_i| r_i) + tau, with the
     * velocities at the start of the step; a sphere's bounding radius is r. */
    s->vmax_start = 0.0;
    for (int64_t i = 0; i < s->n; ++i) {
        double nv = norm3(&s->v[3 * i]);
        double nw = norm3(&s->w[3 * i]);
        s->h[i] = dt * (nv + nw * s->r[i]) + P->tau;
        if (nv > s->vmax_start) s->vmax_start = nv;
    }
    double L[3];
    for (int k = 0; k < 3; ++k) L[k] = P->box_hi[k] - P->box_lo[k];

    s->nc = 0;
    s->coloured = 0;
    for (int64_t a = 0; a < s->n; ++a) {
        /* Sphere-sphere pairs (a, b), a < b: j1 = a, j2 = b.  Eq. (contactpos)
         * for two spheres: the point of S_b closest to x_a is
         * x_hat = x_b + r_b n with n = (x_a - x_b)/|x_a - x_b| the outward
         * normal of S_b, and xi = f_a(x_hat) = d - r_a - r_b. */
        for (int64_t b = a + 1; b < s->n; ++b) {
            double d3[3];
            for (int k = 0; k < 3; ++k) {
                double dk = s->x[3 * a + k] - s->x[3 * b + k];
                if (P->periodic[k]) { /* minimum image */
                    if (dk > 0.5 * L[k]) dk -= L[k];
                    else if (dk < -0.5 * L[k]) dk += L[k];
                }
                d3[k] = dk;
            }
            double d = sqrt((d3[0] * d3[0] + d3[1] * d3[1]) + d3[2] * d3[2]);
            /* Sect. 4: keep the pair iff the hulls intersect. */
            if (((d - s->r[a]) - s->r[b]) <= (s->h[a] + s->h[b])) {
                double nrm[3];
                if (d > 0.0) {
                    nrm[0] = d3[0] / d;
                    nrm[1] = d3[1] / d;
                    nrm[2] = d3[2] / d;
                } else { /* coincident centres: the argmin is degenerate */
                    nrm[0] = 0.0; nrm[1] = 0.0; nrm[2] = 1.0;
                }
                double xi = (d - s->r[a]) - s->r[b];
                /* l_a = x_hat - x_a = -(d - r_b) n ;  l_b = x_hat - x_b = r_b n */
                if (push_contact(s, (uint32_t)a, (uint32_t)b, nrm, xi, d - s->r[b], s->r[b])) return 2;
            }
        }
        /* Sphere-wall pairs (a, wall k): j2 = n + k.  The wall solid is
         * {y : n_k . y <= c_k}, its outward normal is n_k, the point of the
         * solid closest to x_a is x_a - (n_k . x_a - c_k) n_k, and the walls
         * have no velocity, so their hull radius is tau alone. */
        for (int32_t k = 0; k < s->nplanes; ++k) {
            const double* nk = s->plane_n[k];
            double sd = ((nk[0] * s->x[3 * a + 0] + nk[1] * s->x[3 * a + 1]) + nk[2] * s->x[3 * a + 2]) - s->plane_c[k];
            double xi = sd - s->r[a];
            if (xi <= (s->h[a] + P->tau)) {
                if (push_contact(s, (uint32_t)a, (uint32_t)(s->n + k), nk, xi, sd, 0.0)) return 2;
            }
        }
        /* Sphere-cone pairs (a, cone k): j2 = n + nplanes + k.  The point of
         * the solid closest to x_a is x_a - sd n (oracle_cone_distance), so
         * the contact has the form of a wall contact: xi = sd - r_a,
         * l_a = -sd n, and the cone's hull radius is tau. */
        for (int32_t k = 0; k < s->ncones; ++k) {
            double sd, nk[3];
            if (!oracle_cone_distance(s, k, &s->x[3 * a], &sd, nk)) continue;
            double xi = sd - s->r[a];
            if (xi <= (s->h[a] + P->tau)) {
                if (push_contact(s, (uint32_t)a, (uint32_t)(s->n + s->nplanes + k), nk, xi, sd, 0.0)) return 2;
            }
        }
    }
    /* The loops above emit keys (j1 << 32) | j2 in ascending order, which is
     * the canonical order every other part of the oracle relies on. */
    if (n_contacts) *n_contacts = s->nc;
    return 0;
}

/* ------------------------------------------------------------------ */
/* colouring: sequential greedy in descending priority                  */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t prio; uint64_t key; int64_t idx; } prio_item;

static int cmp_prio_desc(const void* pa, const void* pb)
{
    const prio_item* a = (const prio_item*)pa;
    const prio_item* b = (const prio_item*)pb;
    if (a->prio != b->prio) return a->prio > b->prio ? -1 : 1;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return 0;
}

/* Two contacts conflict iff they share a body of finite mass (walls and
 * infinite-mass bodies are never written by the sweep).  Contacts are taken
 * in order of decreasing priority splitmix64(key ^ seed), ties to the lower
 * key; each takes the smallest colour unused by its already-coloured
 * conflicting contacts.  Contacts of one colour then touch disjoint finite
 * bodies, so relaxing them in any order gives bit-identical results. */
int oracle_colour_contacts(oracle_scene* s, int32_t* n_colours)
{
    if (!s) return 1;
    const int64_t nc = s->nc, n = s->n;
    if (s->prm.subdomain_mode == ORACLE_SUB_JACOBI) {
        /* Non-linear block Jacobi: every contact is a subdomain of its own,
         * so within a sweep each one sees only the previous sweep's
         * reactions and the order cannot matter: a single colour. */
        for (int64_t c = 0; c < nc; ++c) s->colour[c] = 0;
        s->ncolours = nc > 0 ? 1 : 0;
        s->coloured = 1;
        if (n_colours) *n_colours = s->ncolours;
        return 0;
    }
    int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    prio_item* items = (prio_item*)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(prio_item));
    if (!deg || !items) { free(deg); free(items); return 2; }
    for (int64_t c = 0; c < nc; ++c) {
        if (is_finite_body(s, s->j1[c])) deg[end_body(s, s->j1[c]) + 1]++;
        if (is_finite_body(s, s->j2[c])) deg[end_body(s, s->j2[c]) + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) deg[i + 1] += deg[i];
    int64_t* adj = (int64_t*)malloc((size_t)(deg[n] > 0 ? deg[n] : 1) * sizeof(int64_t));
    int64_t* fill = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!adj || !fill) { free(deg); free(items); free(adj); free(fill); return 2; }
    for (int64_t c = 0; c < nc; ++c) {
        uint32_t b[2] = { s->j1[c], s->j2[c] };
        for (int e = 0; e < 2; ++e)
            if (is_finite_body(s, b[e])) {
                int64_t i = end_body(s, b[e]);
                adj[deg[i] + fill[i]++] = c;
            }
    }
    for (int64_t c = 0; c < nc; ++c) {
        uint64_t key = ((uint64_t)s->j1[c] << 32) | s->j2[c];
        items[c].key = key;
        items[c].prio = oracle_splitmix64(key ^ s->prm.colour_seed);
        items[c].idx = c;
        s->colour[c] = -1;
    }
    qsort(items, (size_t)nc, sizeof(prio_item), cmp_prio_desc);

    int64_t maxdeg = 0;
    for (int64_t i = 0; i < n; ++i)
        if (deg[i + 1] - deg[i] > maxdeg) maxdeg = deg[i + 1] - deg[i];
    int64_t ncol_max = 2 * maxdeg + 2;
    int64_t* mark = (int64_t*)malloc((size_t)ncol_max * sizeof(int64_t));
    if (!mark) { free(deg); free(items); free(adj); free(fill); return 2; }
    for (int64_t k = 0; k < ncol_max; ++k) mark[k] = -1;

    int32_t ncolours = 0;
    for (int64_t it = 0; it < nc; ++it) {
        int64_t c = items[it].idx;
        uint32_t b[2] = { s->j1[c], s->j2[c] };
        for (int e = 0; e < 2; ++e) {
            if (!is_finite_body(s, b[e])) continue;
            int64_t i = end_body(s, b[e]);
            for (int64_t k = deg[i]; k < deg[i + 1]; ++k) {
                int64_t d = adj[k];
                if (d != c && s->colour[d] >= 0) mark[s->colour[d]] = c;
            }
        }
        int32_t col = 0;
        while (mark[col] == c) ++col;
        s->colour[c] = col;
        if (col + 1 > ncolours) ncolours = col + 1;
    }
    free(deg); free(items); free(adj); free(fill); free(mark);
    s->ncolours = ncolours;
    s->coloured = 1;
    if (n_colours) *n_colours = ncolours;
    return 0;
}

/* ------------------------------------------------------------------ */
/* NBGS solve (Sect. 5, Alg. 1 with one subdomain)                      */
/* ------------------------------------------------------------------ */

/* Per-contact constants of one step. */
typedef struct {
    uint32_t a, b;
    int fa, fb;                 /* finite (mutable) bodies */
    double n[3], t[3], o[3];
    double la, lb;              /* l_a = -la n, l_b = lb n */
    double bias;                /* xi'/dt */
    double w_n, w_t;            /* contact-frame Delassus block diag(w_n, w_t, w_t) */
} contact_k;

static void build_contact(const oracle_scene* s, int64_t c, contact_k* k)
{
    k->a = s->j1[c];
    k->b = s->j2[c];
    k->fa = (int64_t)k->a < s->n;
    k->fb = (int64_t)k->b < s->n;
    for (int e = 0; e < 3; ++e) k->n[e] = s->cn[3 * c + e];
    oracle_contact_frame(k->n, k->t, k->o);
    k->la = s->la[c];
    k->lb = s->lb[c];
    /* eq. (nonpenetration): the gap term xi/dt; a penetration (xi < 0) is
     * corrected with the scaled term beta xi/dt (Sect. 3). */
    double xi = s->xi[c];
    double xs = xi >= 0.0 ? xi : s->prm.beta * xi;
    k->bias = xs / s->prm.dt;
    /* W = J M^-1 J^T for the two bodies.  With levers parallel to n,
     * (l x P) x l = |l|^2 (P - n (n.P)), so W = w_n 1 + (w_t - w_n)(1 - n n^T). */
    double ima = k->fa ? s->invm[k->a] : 0.0, iIa = k->fa ? s->invI[k->a] : 0.0;
    double imb = k->fb ? s->invm[k->b] : 0.0, iIb = k->fb ? s->invI[k->b] : 0.0;
    k->w_n = ima + imb;
    k->w_t = k->w_n + iIa * k->la * k->la + iIb * k->lb * k->lb;
}

/* Relative contact velocity u = v_a + w_a x l_a - v_b - w_b x l_b
 * (Sect. 2), in world coordinates. */
static void rel_velocity(const oracle_scene* s, const contact_k* k, double u[3])
{
    double la3[3] = { -k->la * k->n[0], -k->la * k->n[1], -k->la * k->n[2] };
    double lb3[3] = { k->lb * k->n[0], k->lb * k->n[1], k->lb * k->n[2] };
    double wa[3] = { 0, 0, 0 }, wb[3] = { 0, 0, 0 };
    for (int e = 0; e < 3; ++e) u[e] = 0.0;
    if (k->fa) {
        cross3(&s->w[3 * k->a], la3, wa);
        for (int e = 0; e < 3; ++e) u[e] += s->v[3 * k->a + e] + wa[e];
    }
    if (k->fb) {
        cross3(&s->w[3 * k->b], lb3, wb);
        for (int e = 0; e < 3; ++e) u[e] -= s->v[3 * k->b + e] + wb[e];
    }
}

/* Apply a world-frame impulse P acting +P on j1 and -P on j2 at x_hat:
 * the contact terms of eq. (wrench) times dt, divided by the mass matrix,
 * added to the velocity accumulators in place (Sect. 6.3). */
static void apply_impulse(oracle_scene* s, const contact_k* k, const double P[3])
{
    if (k->fa && (s->invm[k->a] > 0.0 || s->invI[k->a] > 0.0)) {
        double la3[3] = { -k->la * k->n[0], -k->la * k->n[1], -k->la * k->n[2] };
        double tq[3];
        cross3(la3, P, tq);
        for (int e = 0; e < 3; ++e) {
            s->v[3 * k->a + e] += s->invm[k->a] * P[e];
            s->w[3 * k->a + e] += s->invI[k->a] * tq[e];
        }
    }
    if (k->fb && (s->invm[k->b] > 0.0 || s->invI[k->b] > 0.0)) {
        double lb3[3] = { k->lb * k->n[0], k->lb * k->n[1], k->lb * k->n[2] };
        double tq[3];
        cross3(lb3, P, tq);
        for (int e = 0; e < 3; ++e) {
            s->v[3 * k->b + e] -= s->invm[k->b] * P[e];
            s->w[3 * k->b + e] -= s->invI[k->b] * tq[e];
        }
    }
}

typedef struct { int32_t colour; int64_t idx; } order_item;
static int cmp_order(const void* pa, const void* pb)
{
    const order_item* a = (const order_item*)pa;
    const order_item* b = (const order_item*)pb;
    if (a->colour != b->colour) return a->colour < b->colour ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

static int64_t find_prev(const oracle_scene* s, uint64_t key)
{
    int64_t lo = 0, hi = s->nprev;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (s->prev_key[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < s->nprev && s->prev_key[lo] == key) ? lo : -1;
}

/* Subdomain s_c(j) of contact c (Alg. 1).  Sect. 6.2 lets any rule that
 * partitions the contact set decide which process treats a contact and
 * recommends favouring the particles' parent processes: with a regular grid
 * of g0 x g1 x g2 subdomains over the box, contact c belongs to the
 * subdomain holding the centre of its body j1 (cell k_a = floor((x_a - lo_a)
 * g_a / L_a), clamped to [0, g_a - 1]; id = (k_2 g_1 + k_1) g_0 + k_0).
 * Non-linear block Jacobi: every contact its own subdomain. */
static int64_t contact_subdomain(const oracle_scene* s, int64_t c)
{
    if (s->prm.subdomain_mode == ORACLE_SUB_JACOBI) return c;
    if (s->prm.subdomain_mode != ORACLE_SUB_GRID) return 0;
    const double* x = &s->x[3 * (int64_t)s->j1[c]];
    int64_t id = 0;
    for (int a = 2; a >= 0; --a) {
        const int32_t g = s->prm.subdomains[a];
        const double L = s->prm.box_hi[a] - s->prm.box_lo[a];
        double k = floor(((x[a] - s->prm.box_lo[a]) * (double)g) / L);
        if (!(k >= 0.0)) k = 0.0;
        if (k > (double)(g - 1)) k = (double)(g - 1);
        id = id * g + (int64_t)k;
    }
    return id;
}

int oracle_contact_subdomains(const oracle_scene* s, int64_t* out)
{
    if (!s || (s->nc > 0 && !out)) return 1;
    /* after a solve: the subdomains it used (positions at the start of the
     * step); before: from the current positions */
    for (int64_t c = 0; c < s->nc; ++c) out[c] = s->sub ? s->sub[c] : contact_subdomain(s, c);
    return 0;
}

/* Correction variables of Sect. 6.3 in the velocity form: one slot per pair
 * (finite body i, subdomain p) that some contact of p touches, holding
 * (delta v_i^[p], delta w_i^[p]).  Slots of one body are consecutive, in
 * increasing subdomain order. */
typedef struct { int64_t body, sub, end; } slot_item;

static int cmp_slot(const void* pa, const void* pb)
{
    const slot_item* a = (const slot_item*)pa;
    const slot_item* b = (const slot_item*)pb;
    if (a->body != b->body) return a->body < b->body ? -1 : 1;
    if (a->sub != b->sub) return a->sub < b->sub ? -1 : 1;
    return a->end < b->end ? -1 : (a->end > b->end ? 1 : 0);
}

/* slot_of[2 c + e] = correction slot of end e (0: j1, 1: j2) of contact c,
 * -1 for an end without a finite body; slot_body[k] = body of slot k. */
static int build_slots(const oracle_scene* s, const contact_k* K, int64_t* slot_of, int64_t** slot_body,
                       int64_t* nslot)
{
    const int64_t nc = s->nc;
    slot_item* it = (slot_item*)malloc((size_t)(2 * nc > 0 ? 2 * nc : 1) * sizeof(slot_item));
    int64_t* sb = (int64_t*)malloc((size_t)(2 * nc > 0 ? 2 * nc : 1) * sizeof(int64_t));
    if (!it || !sb) { free(it); free(sb); return 2; }
    int64_t m = 0;
    for (int64_t c = 0; c < nc; ++c) {
        const int64_t sub = contact_subdomain(s, c);
        slot_of[2 * c] = slot_of[2 * c + 1] = -1;
        if (K[c].fa) { it[m].body = K[c].a; it[m].sub = sub; it[m].end = 2 * c; ++m; }
        if (K[c].fb) { it[m].body = K[c].b; it[m].sub = sub; it[m].end = 2 * c + 1; ++m; }
    }
    qsort(it, (size_t)m, sizeof(slot_item), cmp_slot);
    int64_t k = -1;
    for (int64_t i = 0; i < m; ++i) {
        if (i == 0 || it[i].body != it[i - 1].body || it[i].sub != it[i - 1].sub) sb[++k] = it[i].body;
        slot_of[it[i].end] = k;
    }
    free(it);
    *slot_body = sb;
    *nslot = k + 1;
    return 0;
}

static int solve_composite(oracle_scene* s, int32_t max_sweeps, double tol, int32_t* sweeps_done,
                           double* residual);

int oracle_solve_nbgs(oracle_scene* s, int32_t max_sweeps, double tol,
                      int32_t* sweeps_done, double* residual)
{
    if (!s || max_sweeps < 0) return 1;
    if (!s->coloured) {
        int rc = oracle_colour_contacts(s, NULL);
        if (rc) return rc;
    }
    if (s->composite) return solve_composite(s, max_sweeps, tol, sweeps_done, residual);
    const oracle_params* P = &s->prm;
    const int64_t nc = s->nc;
    contact_k* K = (contact_k*)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(contact_k));
    order_item* ord = (order_item*)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(order_item));
    if (!K || !ord) { free(K); free(ord); return 2; }
    for (int64_t c = 0; c < nc; ++c) {
        build_contact(s, c, &K[c]);
        ord[c].colour = s->colour[c];
        ord[c].idx = c;
    }
    /* Contact order of the sweep: colours ascending, canonical inside. */
    qsort(ord, (size_t)nc, sizeof(order_item), cmp_order);

    double gdt = norm3(P->gravity) * P->dt;
    s->v_ref = s->vmax_start;
    if (gdt > s->v_ref) s->v_ref = gdt;
    if (1e-12 > s->v_ref) s->v_ref = 1e-12;

    /* eq. (integrationscheme), velocity part without contact reactions:
     * v += dt M^-1 f_ext with f_ext = m g; the gyroscopic term w x I w
     * vanishes for the isotropic inertia of a sphere. */
    for (int64_t i = 0; i < s->n; ++i)
        if (s->invm[i] > 0.0)
            for (int e = 0; e < 3; ++e) s->v[3 * i + e] += P->dt * P->gravity[e];

    /* Alg. 1 starts from lambda = 0 "or any other initialization", in
     * particular the previous step's reactions (Sect. 5). */
    for (int64_t c = 0; c < nc; ++c) {
        double* p = &s->p[3 * c];
        p[0] = p[1] = p[2] = 0.0;
        if (P->warm_start == ORACLE_WARM_PREV && s->nprev > 0) {
            uint64_t key = ((uint64_t)s->j1[c] << 32) | s->j2[c];
            int64_t k = find_prev(s, key);
            if (k >= 0) {
                const double* Pw = &s->prev_P[3 * k];
                const contact_k* kc = &K[c];
                double pn = dot3(kc->n, Pw);
                if (!(pn > 0.0)) pn = 0.0;
                double pt = dot3(kc->t, Pw), po = dot3(kc->o, Pw);
                double lim = P->mu * pn, len = sqrt(pt * pt + po * po);
                if (len > lim) {
                    if (len > 0.0) { pt = pt * (lim / len); po = po * (lim / len); }
                    else { pt = 0.0; po = 0.0; }
                }
                p[0] = pn; p[1] = pt; p[2] = po;
            }
        }
    }
    for (int64_t it = 0; it < nc; ++it) {
        int64_t c = ord[it].idx;
        const contact_k* k = &K[c];
        const double* p = &s->p[3 * c];
        if (p[0] == 0.0 && p[1] == 0.0 && p[2] == 0.0) continue;
        double Pw[3];
        for (int e = 0; e < 3; ++e) Pw[e] = p[0] * k->n[e] + p[1] * k->t[e] + p[2] * k->o[e];
        apply_impulse(s, k, Pw);
    }

    /* Subdomains (Alg. 1 in general): the velocity of body i seen by a
     * contact of subdomain p is the accumulator v_i (all reactions of the
     * previous sweep) plus the correction delta v_i^[p] of the contacts of p
     * already relaxed in this sweep (Sect. 6.3).  After the sweep every
     * accumulator takes the sum of its corrections. */
    const int sub = P->subdomain_mode != ORACLE_SUB_NONE;
    int64_t* slot_of = NULL;
    int64_t* slot_body = NULL;
    int64_t nslot = 0;
    double *dv = NULL, *dw = NULL;
    if (sub) {
        slot_of = (int64_t*)malloc((size_t)(2 * nc > 0 ? 2 * nc : 1) * sizeof(int64_t));
        free(s->sub);
        s->sub = (int64_t*)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int64_t));
        if (s->sub)
            for (int64_t c = 0; c < nc; ++c) s->sub[c] = contact_subdomain(s, c);
        int rc = (slot_of && s->sub) ? build_slots(s, K, slot_of, &slot_body, &nslot) : 2;
        if (rc == 0) {
            dv = (double*)calloc(3 * (size_t)(nslot > 0 ? nslot : 1), sizeof(double));
            dw = (double*)calloc(3 * (size_t)(nslot > 0 ? nslot : 1), sizeof(double));
        }
        if (rc != 0 || !dv || !dw) {
            free(slot_of); free(slot_body); free(dv); free(dw); free(K); free(ord);
            return 2;
        }
    }

    s->nhist = 0;
    int32_t k_done = 0;
    double Rk = 0.0;
    for (int32_t sweep = 0; sweep < max_sweeps && sub; ++sweep) {
        double rmax = 0.0;
        for (int64_t i = 0; i < 3 * nslot; ++i) dv[i] = dw[i] = 0.0;
        for (int64_t it = 0; it < nc; ++it) {
            int64_t c = ord[it].idx;
            const contact_k* k = &K[c];
            if (!(k->w_n > 0.0)) continue;
            double* p = &s->p[3 * c];
            const int64_t sa = slot_of[2 * c], sb = slot_of[2 * c + 1];
            /* velocities seen by this contact: accumulator + its subdomain's correction */
            double va[3] = { 0, 0, 0 }, wa[3] = { 0, 0, 0 }, vb[3] = { 0, 0, 0 }, wb[3] = { 0, 0, 0 };
            for (int e = 0; e < 3; ++e) {
                if (sa >= 0) {
                    va[e] = s->v[3 * k->a + e] + dv[3 * sa + e];
                    wa[e] = s->w[3 * k->a + e] + dw[3 * sa + e];
                }
                if (sb >= 0) {
                    vb[e] = s->v[3 * k->b + e] + dv[3 * sb + e];
                    wb[e] = s->w[3 * k->b + e] + dw[3 * sb + e];
                }
            }
            double la3[3] = { -k->la * k->n[0], -k->la * k->n[1], -k->la * k->n[2] };
            double lb3[3] = { k->lb * k->n[0], k->lb * k->n[1], k->lb * k->n[2] };
            double ca[3], cb[3], u[3];
            cross3(wa, la3, ca);
            cross3(wb, lb3, cb);
            for (int e = 0; e < 3; ++e) u[e] = (va[e] + ca[e]) - (vb[e] + cb[e]);
            double b[3];
            b[0] = (dot3(k->n, u) - k->w_n * p[0]) + k->bias;
            b[1] = dot3(k->t, u) - k->w_t * p[1];
            b[2] = dot3(k->o, u) - k->w_t * p[2];
            double y[3];
            oracle_one_contact(k->w_n, k->w_t, P->mu, b, y);
            double pnew[3], dp[3];
            for (int e = 0; e < 3; ++e) {
                pnew[e] = P->omega * y[e] + (1.0 - P->omega) * p[e];
                dp[e] = pnew[e] - p[e];
            }
            double Pw[3];
            for (int e = 0; e < 3; ++e) Pw[e] = dp[0] * k->n[e] + dp[1] * k->t[e] + dp[2] * k->o[e];
            /* Sect. 6.3: the corrections of subdomain s_c(j) take the change
             * of reaction j (+ on j1, - on j2) */
            double ta[3], tb[3];
            cross3(la3, Pw, ta);
            cross3(lb3, Pw, tb);
            for (int e = 0; e < 3; ++e) {
                if (sa >= 0) {
                    dv[3 * sa + e] += s->invm[k->a] * Pw[e];
                    dw[3 * sa + e] += s->invI[k->a] * ta[e];
                }
                if (sb >= 0) {
                    dv[3 * sb + e] -= s->invm[k->b] * Pw[e];
                    dw[3 * sb + e] -= s->invI[k->b] * tb[e];
                }
            }
            for (int e = 0; e < 3; ++e) p[e] = pnew[e];
            double r1 = k->w_n * dp[0], r2 = k->w_t * dp[1], r3 = k->w_t * dp[2];
            double rj = sqrt((r1 * r1 + r2 * r2) + r3 * r3);
            if (rj > rmax) rmax = rj;
        }
        /* end of the sweep: accumulators += corrections, in increasing
         * subdomain order per body; the corrections restart from zero */
        for (int64_t q = 0; q < nslot; ++q)
            for (int e = 0; e < 3; ++e) {
                s->v[3 * slot_body[q] + e] += dv[3 * q + e];
                s->w[3 * slot_body[q] + e] += dw[3 * q + e];
            }
        Rk = rmax / s->v_ref;
        if (s->nhist == s->cap_hist) {
            double* hh = (double*)realloc(s->hist, 2 * (size_t)s->cap_hist * sizeof(double));
            if (!hh) { free(slot_of); free(slot_body); free(dv); free(dw); free(K); free(ord); return 2; }
            s->hist = hh;
            s->cap_hist *= 2;
        }
        s->hist[s->nhist++] = Rk;
        k_done = sweep + 1;
        if (tol > 0.0 && Rk <= tol) break;
    }
    free(slot_of); free(slot_body); free(dv); free(dw);
    for (int32_t sweep = 0; sweep < max_sweeps && !sub; ++sweep) {
        double rmax = 0.0;
        for (int64_t it = 0; it < nc; ++it) {
            int64_t c = ord[it].idx;
            const contact_k* k = &K[c];
            if (!(k->w_n > 0.0)) continue; /* two infinite masses: nothing moves */
            double* p = &s->p[3 * c];
            double u[3];
            rel_velocity(s, k, u);
            /* Remove the contact's own reaction to get the velocity given the
             * other contacts' reactions lambda_jbar (Alg. 1, Alg. 2), and add
             * the gap term of eq. (nonpenetration). */
            double b[3];
            b[0] = (dot3(k->n, u) - k->w_n * p[0]) + k->bias;
            b[1] = dot3(k->t, u) - k->w_t * p[1];
            b[2] = dot3(k->o, u) - k->w_t * p[2];
            double y[3];
            oracle_one_contact(k->w_n, k->w_t, P->mu, b, y);
            /* Alg. 1: lambda_j <- omega y + (1 - omega) lambda_j */
            double pnew[3], dp[3];
            for (int e = 0; e < 3; ++e) {
                pnew[e] = P->omega * y[e] + (1.0 - P->omega) * p[e];
                dp[e] = pnew[e] - p[e];
            }
            double Pw[3];
            for (int e = 0; e < 3; ++e) Pw[e] = dp[0] * k->n[e] + dp[1] * k->t[e] + dp[2] * k->o[e];
            apply_impulse(s, k, Pw);
            for (int e = 0; e < 3; ++e) p[e] = pnew[e];
            /* velocity change at the contact caused by this relaxation */
            double r1 = k->w_n * dp[0], r2 = k->w_t * dp[1], r3 = k->w_t * dp[2];
            double rj = sqrt((r1 * r1 + r2 * r2) + r3 * r3);
            if (rj > rmax) rmax = rj;
        }
        Rk = rmax / s->v_ref;
        if (s->nhist == s->cap_hist) {
            double* hh = (double*)realloc(s->hist, 2 * (size_t)s->cap_hist * sizeof(double));
            if (!hh) { free(K); free(ord); return 2; }
            s->hist = hh;
            s->cap_hist *= 2;
        }
        s->hist[s->nhist++] = Rk;
        k_done = sweep + 1;
        if (tol > 0.0 && Rk <= tol) break;
    }

    /* Keep this step's reactions (world frame) for the next warm start. */
    free(s->prev_key);
    free(s->prev_P);
    s->prev_key = (uint64_t*)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(uint64_t));
    s->prev_P = (double*)malloc(3 * (size_t)(nc > 0 ? nc : 1) * sizeof(double));
    if (!s->prev_key || !s->prev_P) { free(K); free(ord); s->nprev = 0; return 2; }
    for (int64_t c = 0; c < nc; ++c) {
        s->prev_key[c] = ((uint64_t)s->j1[c] << 32) | s->j2[c];
        const double* p = &s->p[3 * c];
        for (int e = 0; e < 3; ++e)
            s->prev_P[3 * c + e] = p[0] * K[c].n[e] + p[1] * K[c].t[e] + p[2] * K[c].o[e];
    }
    s->nprev = nc;
    free(K);
    free(ord);
    if (sweeps_done) *sweeps_done = k_done;
    if (residual) *residual = Rk;
    return 0;
}

/* ------------------------------------------------------------------ */
/* composite particles                                                  */
/* ------------------------------------------------------------------ */
/* Rotation matrix of the unit quaternion (w, x, y, z). */
static void quat_matrix(const double q[4], double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z); R[0][1] = 2.0 * (x * y - w * z); R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z); R[1][1] = 1.0 - 2.0 * (x * x + z * z); R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y); R[2][1] = 2.0 * (y * z + w * x); R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

static void mat_vec(double A[3][3], const double v[3], double out[3])
{
    for (int k = 0; k < 3; ++k) out[k] = (A[k][0] * v[0] + A[k][1] * v[1]) + A[k][2] * v[2];
}

/* R T0 R^T for a body-frame tensor T0 (9, row-major) */
static void to_world(double R[3][3], const double* T0, double T[3][3])
{
    double RT[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            RT[a][b] = (R[a][0] * T0[0 * 3 + b] + R[a][1] * T0[1 * 3 + b]) + R[a][2] * T0[2 * 3 + b];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) T[a][b] = (RT[a][0] * R[b][0] + RT[a][1] * R[b][1]) + RT[a][2] * R[b][2];
}

static int inverse3(const double* A, double* Ai)
{
    double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    double det = (A[0] * c00 + A[1] * c01) + A[2] * c02;
    if (!(det > 0.0)) return 1;
    Ai[0] = c00 / det; Ai[1] = (A[2] * A[7] - A[1] * A[8]) / det; Ai[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    Ai[3] = c01 / det; Ai[4] = (A[0] * A[8] - A[2] * A[6]) / det; Ai[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    Ai[6] = c02 / det; Ai[7] = (A[1] * A[6] - A[0] * A[7]) / det; Ai[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    return 0;
}

/* Sect. 2: a body of k member spheres (radius r_m, density rho, offset d_m
 * from the given reference point, body frame = observational frame at the
 * start).  Reading: the members' masses and inertias add up (overlapping
 * volume counted once per member), m = sum rho 4/3 pi r_m^3; the body's
 * position is its centre of mass X = sum m_m d_m / m (added to the
 * reference point); the body-frame inertia about X is
 * sum [2/5 m_m r_m^2 1 + m_m (|d'|^2 1 - d' d'^T)], d' = d_m - X; the
 * bounding radius of eq. (expansionradius) is max |d'| + r_m. */
int oracle_create_composite_scene(const oracle_params* prm, int64_t n, const double* pos, const double* vel,
                                  const double* angvel, const double* density, int64_t nm,
                                  const int32_t* member_body, const double* member_offset,
                                  const double* member_radius, oracle_scene** out)
{
    if (!prm || !out || n < 1 || nm < n || !pos || !vel || !angvel || !density || !member_body || !member_offset ||
        !member_radius || prm->subdomain_mode != ORACLE_SUB_NONE)
        return 1;
    for (int64_t m = 0; m < nm; ++m) {
        if (member_body[m] < 0 || member_body[m] >= n || !(member_radius[m] > 0.0)) return 1;
        if (m > 0 && member_body[m] < member_body[m - 1]) return 1;
        if (m > 0 && member_body[m] > member_body[m - 1] + 1) return 1;   /* every body has members */
    }
    if (member_body[0] != 0 || member_body[nm - 1] != n - 1) return 1;
    for (int64_t i = 0; i < n; ++i)
        if (!(density[i] > 0.0)) return 1;   /* the centre of mass needs a mass */
    double* ones = (double*)malloc((size_t)n * sizeof(double));
    if (!ones) return 2;
    for (int64_t i = 0; i < n; ++i) ones[i] = 1.0;
    oracle_scene* s = NULL;
    int rc = oracle_create_scene(prm, n, pos, vel, angvel, ones, density, &s);
    free(ones);
    if (rc) return rc;
    s->composite = 1;
    s->nm = nm;
    s->mbody = (int32_t*)malloc((size_t)nm * sizeof(int32_t));
    s->moff = (double*)malloc(3 * (size_t)nm * sizeof(double));
    s->mr = (double*)malloc((size_t)nm * sizeof(double));
    s->I0 = (double*)malloc(9 * (size_t)n * sizeof(double));
    s->I0inv = (double*)malloc(9 * (size_t)n * sizeof(double));
    if (!s->mbody || !s->moff || !s->mr || !s->I0 || !s->I0inv) { oracle_destroy_scene(s); return 2; }
    int64_t m0 = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t m1 = m0;
        while (m1 < nm && member_body[m1] == i) ++m1;
        if (m1 - m0 > ORACLE_MAX_MEMBERS) { oracle_destroy_scene(s); return 1; }
        double M = 0.0, X[3] = { 0.0, 0.0, 0.0 };
        for (int64_t m = m0; m < m1; ++m) {
            double r = member_radius[m];
            double mm = density[i] * (4.0 / 3.0) * M_PI * r * r * r;
            M += mm;
            for (int e = 0; e < 3; ++e) X[e] += mm * member_offset[3 * m + e];
        }
        for (int e = 0; e < 3; ++e) X[e] = X[e] / M;
        double* I = &s->I0[9 * i];
        for (int k = 0; k < 9; ++k) I[k] = 0.0;
        double rbar = 0.0;
        for (int64_t m = m0; m < m1; ++m) {
            double r = member_radius[m];
            double mm = density[i] * (4.0 / 3.0) * M_PI * r * r * r;
            double d[3];
            for (int e = 0; e < 3; ++e) d[e] = member_offset[3 * m + e] - X[e];
            double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    I[3 * a + b] += (a == b ? 0.4 * mm * r * r + mm * d2 : 0.0) - mm * d[a] * d[b];
            s->mbody[m] = (int32_t)i;
            for (int e = 0; e < 3; ++e) s->moff[3 * m + e] = d[e];
            s->mr[m] = r;
            double reach = sqrt(d2) + r;
            if (reach > rbar) rbar = reach;
        }
        for (int e = 0; e < 3; ++e) s->x[3 * i + e] = pos[3 * i + e] + X[e];
        s->r[i] = rbar;
        s->invm[i] = M > 0.0 ? 1.0 / M : 0.0;
        if (M > 0.0) {
            if (inverse3(I, &s->I0inv[9 * i])) { oracle_destroy_scene(s); return 1; }
            s->invI[i] = 1.0;   /* finite: takes impulses; the tensor is I0inv */
        } else {
            for (int k = 0; k < 9; ++k) s->I0inv[9 * i + k] = 0.0;
            s->invI[i] = 0.0;
        }
        m0 = m1;
    }
    *out = s;
    return 0;
}

/* World position of member m: X_b + R(q_b) d'_m. */
static void member_position(const oracle_scene* s, int64_t m, double p[3])
{
    const int64_t b = s->mbody[m];
    double R[3][3], rd[3];
    quat_matrix(&s->q[4 * b], R);
    mat_vec(R, &s->moff[3 * m], rd);
    for (int e = 0; e < 3; ++e) p[e] = s->x[3 * b + e] + rd[e];
}

int oracle_body_mass_properties(const oracle_scene* s, double* invm, double* I0)
{
    if (!s || !s->composite) return 1;
    for (int64_t i = 0; i < s->n; ++i) {
        if (invm) invm[i] = s->invm[i];
        if (I0)
            for (int k = 0; k < 9; ++k) I0[9 * i + k] = s->I0[9 * i + k];
    }
    return 0;
}

int oracle_member_positions(const oracle_scene* s, double* out)
{
    if (!s || !s->composite || !out) return 1;
    for (int64_t m = 0; m < s->nm; ++m) member_position(s, m, &out[3 * m]);
    return 0;
}

/* Contacts between members of different bodies and between members and the
 * walls, tested like spheres (eq. contactpos for two spheres) against the
 * hulls of their bodies (eq. expansionradius with the bounding radius). */
static int detect_composite(oracle_scene* s)
{
    const oracle_params* P = &s->prm;
    const double dt = P->dt;
    s->vmax_start = 0.0;
    for (int64_t i = 0; i < s->n; ++i) {
        double nv = norm3(&s->v[3 * i]);
        double nw = norm3(&s->w[3 * i]);
        s->h[i] = dt * (nv + nw * s->r[i]) + P->tau;
        if (nv > s->vmax_start) s->vmax_start = nv;
    }
    double L[3];
    for (int k = 0; k < 3; ++k) L[k] = P->box_hi[k] - P->box_lo[k];
    double* pm = (double*)malloc(3 * (size_t)s->nm * sizeof(double));
    if (!pm) return 2;
    for (int64_t m = 0; m < s->nm; ++m) member_position(s, m, &pm[3 * m]);
    s->nc = 0;
    s->coloured = 0;
    for (int64_t a = 0; a < s->nm; ++a) {
        const int64_t A = s->mbody[a];
        for (int64_t b = a + 1; b < s->nm; ++b) {
            const int64_t B = s->mbody[b];
            if (A == B) continue;
            double d3[3];
            for (int k = 0; k < 3; ++k) {
                double dk = pm[3 * a + k] - pm[3 * b + k];
                if (P->periodic[k]) {
                    if (dk > 0.5 * L[k]) dk -= L[k];
                    else if (dk < -0.5 * L[k]) dk += L[k];
                }
                d3[k] = dk;
            }
            double d = sqrt((d3[0] * d3[0] + d3[1] * d3[1]) + d3[2] * d3[2]);
            if (((d - s->mr[a]) - s->mr[b]) <= (s->h[A] + s->h[B])) {
                double nrm[3];
                if (d > 0.0) { nrm[0] = d3[0] / d; nrm[1] = d3[1] / d; nrm[2] = d3[2] / d; }
                else { nrm[0] = 0.0; nrm[1] = 0.0; nrm[2] = 1.0; }
                double xi = (d - s->mr[a]) - s->mr[b];
                if (push_contact(s, (uint32_t)a, (uint32_t)b, nrm, xi, d - s->mr[b], s->mr[b])) { free(pm); return 2; }
            }
        }
        for (int32_t k = 0; k < s->nplanes; ++k) {
            const double* nk = s->plane_n[k];
            double sd = ((nk[0] * pm[3 * a + 0] + nk[1] * pm[3 * a + 1]) + nk[2] * pm[3 * a + 2]) - s->plane_c[k];
            double xi = sd - s->mr[a];
            if (xi <= (s->h[A] + P->tau))
                if (push_contact(s, (uint32_t)a, (uint32_t)(s->nm + k), nk, xi, sd, 0.0)) { free(pm); return 2; }
        }
    }
    free(pm);
    return 0;
}

/* Per-contact constants of a composite contact: bodies, contact frame,
 * levers l = x_hat - X of both bodies (eq. wrench), and the Delassus block
 * W = sum over the bodies of 1/m 1 - [l]x I^-1 [l]x in the contact frame. */
typedef struct {
    int64_t A, B;              /* bodies; B = -1 for a wall */
    double n[3], t[3], o[3];
    double lA[3], lB[3];
    double W[6];               /* Wnn, Wtt, Woo, Wnt, Wno, Wto */
    double bias;
} ccontact;

static void add_response(double W[3][3], double invm, double Iinv[3][3], const double l[3])
{
    /* - [l]x I^-1 [l]x e_b for every column b */
    for (int b = 0; b < 3; ++b) {
        double e[3] = { 0.0, 0.0, 0.0 }, lxe[3], Il[3], col[3];
        e[b] = 1.0;
        cross3(l, e, lxe);
        mat_vec(Iinv, lxe, Il);
        cross3(Il, l, col);   /* (I^-1 (l x e)) x l = -l x (I^-1 (l x e)) */
        for (int a = 0; a < 3; ++a) W[a][b] += (a == b ? invm : 0.0) + col[a];
    }
}

static void comp_apply(oracle_scene* s, const ccontact* k, double (*Iwinv)[3][3], const double P[3])
{
    double tq[3], dw[3];
    if (k->A >= 0 && s->invm[k->A] > 0.0) {
        cross3(k->lA, P, tq);
        mat_vec(Iwinv[k->A], tq, dw);
        for (int e = 0; e < 3; ++e) {
            s->v[3 * k->A + e] += s->invm[k->A] * P[e];
            s->w[3 * k->A + e] += dw[e];
        }
    }
    if (k->B >= 0 && s->invm[k->B] > 0.0) {
        cross3(k->lB, P, tq);
        mat_vec(Iwinv[k->B], tq, dw);
        for (int e = 0; e < 3; ++e) {
            s->v[3 * k->B + e] -= s->invm[k->B] * P[e];
            s->w[3 * k->B + e] -= dw[e];
        }
    }
}

static int solve_composite(oracle_scene* s, int32_t max_sweeps, double tol, int32_t* sweeps_done, double* residual)
{
    const oracle_params* P = &s->prm;
    const int64_t nc = s->nc, n = s->n;
    ccontact* K = (ccontact*)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(ccontact));
    order_item* ord = (order_item*)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(order_item));
    double (*Iwinv)[3][3] = malloc((size_t)n * sizeof(*Iwinv));
    double (*Iw)[3][3] = malloc((size_t)n * sizeof(*Iw));
    if (!K || !ord || !Iwinv || !Iw) { free(K); free(ord); free(Iwinv); free(Iw); return 2; }
    for (int64_t i = 0; i < n; ++i) {
        double R[3][3];
        quat_matrix(&s->q[4 * i], R);
        to_world(R, &s->I0inv[9 * i], Iwinv[i]);
        to_world(R, &s->I0[9 * i], Iw[i]);
    }
    for (int64_t c = 0; c < nc; ++c) {
        ccontact* k = &K[c];
        const uint32_t a = s->j1[c], b = s->j2[c];
        k->A = s->mbody[a];
        k->B = (int64_t)b < s->nm ? (int64_t)s->mbody[b] : -1;
        for (int e = 0; e < 3; ++e) k->n[e] = s->cn[3 * c + e];
        oracle_contact_frame(k->n, k->t, k->o);
        double R[3][3], rd[3];
        quat_matrix(&s->q[4 * k->A], R);
        mat_vec(R, &s->moff[3 * a], rd);
        for (int e = 0; e < 3; ++e) k->lA[e] = rd[e] - s->la[c] * k->n[e];
        for (int e = 0; e < 3; ++e) k->lB[e] = 0.0;
        double Wd[3][3] = { { 0, 0, 0 }, { 0, 0, 0 }, { 0, 0, 0 } };
        if (s->invm[k->A] > 0.0) add_response(Wd, s->invm[k->A], Iwinv[k->A], k->lA);
        if (k->B >= 0) {
            quat_matrix(&s->q[4 * k->B], R);
            mat_vec(R, &s->moff[3 * b], rd);
            for (int e = 0; e < 3; ++e) k->lB[e] = rd[e] + s->lb[c] * k->n[e];
            if (s->invm[k->B] > 0.0) add_response(Wd, s->invm[k->B], Iwinv[k->B], k->lB);
        }
        const double* F[3] = { k->n, k->t, k->o };
        double Wc[3][3];
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) {
                double wf[3];
                mat_vec(Wd, F[y], wf);
                Wc[x][y] = dot3(F[x], wf);
            }
        k->W[0] = Wc[0][0]; k->W[1] = Wc[1][1]; k->W[2] = Wc[2][2];
        k->W[3] = Wc[0][1]; k->W[4] = Wc[0][2]; k->W[5] = Wc[1][2];
        double xi = s->xi[c];
        double xs = xi >= 0.0 ? xi : P->beta * xi;
        k->bias = xs / P->dt;
        ord[c].colour = s->colour[c];
        ord[c].idx = c;
    }
    qsort(ord, (size_t)nc, sizeof(order_item), cmp_order);

    double gdt = norm3(P->gravity) * P->dt;
    s->v_ref = s->vmax_start;
    if (gdt > s->v_ref) s->v_ref = gdt;
    if (1e-12 > s->v_ref) s->v_ref = 1e-12;

    /* eq. (integrationscheme) without contact reactions: v += dt g and
     * w += dt I^-1 (-w x I w) with the inertia of the orientation at t */
    for (int64_t i = 0; i < n; ++i) {
        if (!(s->invm[i] > 0.0)) continue;
        double* w = &s->w[3 * i];
        double Lw[3], g[3], dw[3];
        mat_vec(Iw[i], w, Lw);
        cross3(w, Lw, g);
        for (int e = 0; e < 3; ++e) g[e] = -g[e];
        mat_vec(Iwinv[i], g, dw);
        for (int e = 0; e < 3; ++e) {
            w[e] += P->dt * dw[e];
            s->v[3 * i + e] += P->dt * P->gravity[e];
        }
    }
    for (int64_t c = 0; c < nc; ++c) {
        double* p = &s->p[3 * c];
        p[0] = p[1] = p[2] = 0.0;
        if (P->warm_start == ORACLE_WARM_PREV && s->nprev > 0) {
            uint64_t key = ((uint64_t)s->j1[c] << 32) | s->j2[c];
            int64_t kk = find_prev(s, key);
            if (kk >= 0) {
                const double* Pw = &s->prev_P[3 * kk];
                const ccontact* kc = &K[c];
                double pn = dot3(kc->n, Pw);
                if (!(pn > 0.0)) pn = 0.0;
                double pt = dot3(kc->t, Pw), po = dot3(kc->o, Pw);
                double lim = P->mu * pn, len = sqrt(pt * pt + po * po);
                if (len > lim) {
                    if (len > 0.0) { pt = pt * (lim / len); po = po * (lim / len); }
                    else { pt = 0.0; po = 0.0; }
                }
                p[0] = pn; p[1] = pt; p[2] = po;
            }
        }
    }
    for (int64_t it = 0; it < nc; ++it) {
        int64_t c = ord[it].idx;
        const ccontact* k = &K[c];
        const double* p = &s->p[3 * c];
        if (p[0] == 0.0 && p[1] == 0.0 && p[2] == 0.0) continue;
        double Pw[3];
        for (int e = 0; e < 3; ++e) Pw[e] = p[0] * k->n[e] + p[1] * k->t[e] + p[2] * k->o[e];
        comp_apply(s, k, Iwinv, Pw);
    }
    s->nhist = 0;
    int32_t k_done = 0;
    double Rk = 0.0;
    for (int32_t sweep = 0; sweep < max_sweeps; ++sweep) {
        double rmax = 0.0;
        for (int64_t it = 0; it < nc; ++it) {
            int64_t c = ord[it].idx;
            const ccontact* k = &K[c];
            if (!(k->W[0] > 0.0)) continue;
            double* p = &s->p[3 * c];
            double u[3] = { 0.0, 0.0, 0.0 }, cr[3];
            if (k->A >= 0) {
                cross3(&s->w[3 * k->A], k->lA, cr);
                for (int e = 0; e < 3; ++e) u[e] += s->v[3 * k->A + e] + cr[e];
            }
            if (k->B >= 0) {
                cross3(&s->w[3 * k->B], k->lB, cr);
                for (int e = 0; e < 3; ++e) u[e] -= s->v[3 * k->B + e] + cr[e];
            }
            double Wm[3][3];
            w_full(k->W, Wm);
            double uc[3] = { dot3(k->n, u), dot3(k->t, u), dot3(k->o, u) }, wp[3], b[3];
            mat_vec(Wm, p, wp);
            for (int e = 0; e < 3; ++e) b[e] = uc[e] - wp[e];
            b[0] += k->bias;
            double y[3];
            oracle_one_contact_general(k->W, P->mu, b, y);
            double pnew[3], dp[3];
            for (int e = 0; e < 3; ++e) {
                pnew[e] = P->omega * y[e] + (1.0 - P->omega) * p[e];
                dp[e] = pnew[e] - p[e];
            }
            double Pw[3];
            for (int e = 0; e < 3; ++e) Pw[e] = dp[0] * k->n[e] + dp[1] * k->t[e] + dp[2] * k->o[e];
            comp_apply(s, k, Iwinv, Pw);
            for (int e = 0; e < 3; ++e) p[e] = pnew[e];
            double wd[3];
            mat_vec(Wm, dp, wd);
            double rj = sqrt((wd[0] * wd[0] + wd[1] * wd[1]) + wd[2] * wd[2]);
            if (rj > rmax) rmax = rj;
        }
        Rk = rmax / s->v_ref;
        if (s->nhist == s->cap_hist) {
            double* hh = (double*)realloc(s->hist, 2 * (size_t)s->cap_hist * sizeof(double));
            if (!hh) { free(K); free(ord); free(Iwinv); free(Iw); return 2; }
            s->hist = hh;
            s->cap_hist *= 2;
        }
        s->hist[s->nhist++] = Rk;
        k_done = sweep + 1;
        if (tol > 0.0 && Rk <= tol) break;
    }
    free(s->prev_key);
    free(s->prev_P);
    s->prev_key = (uint64_t*)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(uint64_t));
    s->prev_P = (double*)malloc(3 * (size_t)(nc > 0 ? nc : 1) * sizeof(double));
    if (!s->prev_key || !s->prev_P) { free(K); free(ord); free(Iwinv); free(Iw); s->nprev = 0; return 2; }
    for (int64_t c = 0; c < nc; ++c) {
        s->prev_key[c] = ((uint64_t)s->j1[c] << 32) | s->j2[c];
        const double* p = &s->p[3 * c];
        for (int e = 0; e < 3; ++e)
            s->prev_P[3 * c + e] = p[0] * K[c].n[e] + p[1] * K[c].t[e] + p[2] * K[c].o[e];
    }
    s->nprev = nc;
    free(K); free(ord); free(Iwinv); free(Iw);
    if (sweeps_done) *sweeps_done = k_done;
    if (residual) *residual = Rk;
    return 0;
}

/* ------------------------------------------------------------------ */
/* time integration (Sect. 3, eq. integrationscheme)                    */
/* ------------------------------------------------------------------ */
int oracle_integrate(oracle_scene* s)
{
    if (!s) return 1;
    const oracle_params* P = &s->prm;
    const double dt = P->dt;
    for (int64_t i = 0; i < s->n; ++i) {
        double* x = &s->x[3 * i];
        double* q = &s->q[4 * i];
        const double* v = &s->v[3 * i];
        const double* w = &s->w[3 * i];
        for (int e = 0; e < 3; ++e) x[e] = x[e] + dt * v[e];
        /* phi' = phi + dt Q(phi) omega' with the 4x3 block of Sect. 2
         * (rows w, x, y, z; factor 1/2), then renormalisation (Sect. 3). */
        double qw = q[0], qx = q[1], qy = q[2], qz = q[3];
        double dw = 0.5 * (-qx * w[0] - qy * w[1] - qz * w[2]);
        double dx = 0.5 * (qw * w[0] + qz * w[1] - qy * w[2]);
        double dy = 0.5 * (-qz * w[0] + qw * w[1] + qx * w[2]);
        double dz = 0.5 * (qy * w[0] - qx * w[1] + qw * w[2]);
        qw += dt * dw; qx += dt * dx; qy += dt * dy; qz += dt * dz;
        double qn = sqrt(((qw * qw + qx * qx) + qy * qy) + qz * qz);
        q[0] = qw / qn; q[1] = qx / qn; q[2] = qy / qn; q[3] = qz / qn;
        /* periodic axes: a centre that left [lo, hi) re-enters at the
         * opposite face; one inside stays exactly where it is */
        for (int e = 0; e < 3; ++e) {
            if (!P->periodic[e]) continue;
            double L = P->box_hi[e] - P->box_lo[e];
            if (x[e] >= P->box_lo[e] && x[e] < P->box_lo[e] + L) continue;
            double sft = fmod(x[e] - P->box_lo[e], L);
            if (sft < 0.0) sft += L;
            x[e] = P->box_lo[e] + sft;
        }
    }
    return 0;
}

int oracle_step(oracle_scene* s, int32_t max_sweeps, double tol, oracle_step_stats* st)
{
    /* Alg. 2: detection -> (filter: one process, nothing to filter) ->
     * initialisation -> NBGS sweeps -> integration. */
    int64_t nc = 0;
    int32_t ncol = 0, done = 0;
    double R = 0.0;
    int rc = oracle_detect_contacts(s, &nc);
    if (!rc) rc = oracle_colour_contacts(s, &ncol);
    if (!rc) rc = oracle_solve_nbgs(s, max_sweeps, tol, &done, &R);
    if (!rc) rc = oracle_integrate(s);
    if (!rc && st) {
        st->n_contacts = nc;
        st->n_colours = ncol;
        st->sweeps_done = done;
        st->residual = R;
        st->v_ref = s->v_ref;
    }
    return rc;
}

/* ------------------------------------------------------------------ */
/* read-out                                                             */
/* ------------------------------------------------------------------ */
int oracle_get_contacts(const oracle_scene* s, int64_t cap,
                        uint32_t* j1, uint32_t* j2, int32_t* colour,
                        double* normal, double* xi, double* impulse, int64_t* n_out)
{
    if (!s) return 1;
    if (n_out) *n_out = s->nc;
    int64_t m = s->nc < cap ? s->nc : cap;
    for (int64_t c = 0; c < m; ++c) {
        if (j1) j1[c] = s->j1[c];
        if (j2) j2[c] = s->j2[c];
        if (colour) colour[c] = s->colour[c];
        if (xi) xi[c] = s->xi[c];
        for (int e = 0; e < 3; ++e) {
            if (normal) normal[3 * c + e] = s->cn[3 * c + e];
            if (impulse) impulse[3 * c + e] = s->p[3 * c + e];
        }
    }
    return 0;
}

int oracle_set_impulses(oracle_scene* s, const double* impulse)
{
    if (!s || !impulse) return 1;
    memcpy(s->p, impulse, 3 * (size_t)s->nc * sizeof(double));
    return 0;
}

int oracle_residual_history(const oracle_scene* s, double* out, int32_t cap, int32_t* n_out)
{
    if (!s) return 1;
    if (n_out) *n_out = s->nhist;
    for (int32_t k = 0; k < s->nhist && k < cap; ++k) out[k] = s->hist[k];
    return 0;
}

/* Residuals of the discrete constraints eq. (nonpenetration) and
 * eq. (coulomb) at the current velocities and impulses, scaled to
 * velocity units by v_ref. */
int oracle_final_residuals(const oracle_scene* s, oracle_residuals* out)
{
    if (!s || !out || s->composite) return 1;
    memset(out, 0, sizeof(*out));
    double vr = s->v_ref > 0.0 ? s->v_ref : 1e-12;
    for (int64_t c = 0; c < s->nc; ++c) {
        contact_k k;
        build_contact(s, c, &k);
        if (!(k.w_n > 0.0)) continue;
        const double* p = &s->p[3 * c];
        double u[3];
        rel_velocity(s, &k, u);
        double un = dot3(k.n, u), ut = dot3(k.t, u), uo = dot3(k.o, u);
        double gn = k.bias + un;
        double r_np = (gn < 0.0 ? -gn : 0.0) / vr;
        double ptl = sqrt(p[1] * p[1] + p[2] * p[2]);
        double cone = ptl - s->prm.mu * p[0];
        double r_cone = (cone > 0.0 ? cone : 0.0) * k.w_t / vr;
        double m = k.w_n * p[0] < gn ? k.w_n * p[0] : gn;
        double r_comp = fabs(m) / vr;
        double utl = sqrt(ut * ut + uo * uo);
        double e1 = utl * p[1] + s->prm.mu * p[0] * ut;
        double e2 = utl * p[2] + s->prm.mu * p[0] * uo;
        double r_diss = sqrt(e1 * e1 + e2 * e2) * k.w_t / (vr * vr);
        if (r_np > out->non_penetration) out->non_penetration = r_np;
        if (r_cone > out->cone) out->cone = r_cone;
        if (r_comp > out->complementarity) out->complementarity = r_comp;
        if (r_diss > out->dissipation) out->dissipation = r_diss;
    }
    return 0;
}
