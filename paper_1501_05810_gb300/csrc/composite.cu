// composite.cu -- composite particles: rigid bodies made of member spheres
// (Sect. 2: non-convex objects as composites of convex particles).
//
// The detection runs on the members (detect.cu: member positions X + R(q) d,
// the bodies' hulls; pairs inside one body are skipped), so a contact joins
// two members or a member and a wall and keeps its member key.  The
// colouring's conflict graph is over the bodies.  The sweeps act on bodies:
// levers l = x_hat - X are full vectors, so the contact-frame Delassus block
// W = sum over the bodies of 1/m 1 - [l]x I^-1 [l]x is a full symmetric 3x3
// and the one-contact problem takes the general solution below.  The
// velocity step includes the gyroscopic term of eq. (integrationscheme),
// w += dt I^-1 (-w x I w), with the inertia of the orientation at the start
// of the step; orientations are integrated in FP64 (they feed back into the
// dynamics through the members and the inertia).
//
// Layouts: bvel R4[4 nb] = (v, 1/m), (w, 0), (Ixx, Iyy, Izz, Ixy),
// (Ixz, Iyz, 0, 0) of the world inverse inertia; sweep record CompRec<R>
// (colour order) = (ids, bias), (n, Wnn), (l_a, Wtt), (l_b, Woo),
// (Wnt, Wno, Wto, -).
#include <cmath>

#include "nbgs_internal.cuh"

namespace nbgs {

namespace {

template <class R> struct CompRec {
    R4<R> a, b, c, d, e;
};

template <class R> struct Sym3 {
    R nn, tt, oo, nt, no, to;
};

__device__ __forceinline__ void quat_rows(const double4_32a& q, double Rm[3][3])
{
    const double w = q.x, x = q.y, y = q.z, z = q.w;
    Rm[0][0] = 1.0 - 2.0 * (y * y + z * z);
    Rm[0][1] = 2.0 * (x * y - w * z);
    Rm[0][2] = 2.0 * (x * z + w * y);
    Rm[1][0] = 2.0 * (x * y + w * z);
    Rm[1][1] = 1.0 - 2.0 * (x * x + z * z);
    Rm[1][2] = 2.0 * (y * z - w * x);
    Rm[2][0] = 2.0 * (x * z - w * y);
    Rm[2][1] = 2.0 * (y * z + w * x);
    Rm[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

// R T0 R^T of a body-frame tensor T0 (9, row-major)
__device__ __forceinline__ void to_world(const double Rm[3][3], const double* T0, double T[3][3])
{
    double RT[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) RT[a][b] = Rm[a][0] * T0[b] + Rm[a][1] * T0[3 + b] + Rm[a][2] * T0[6 + b];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) T[a][b] = RT[a][0] * Rm[b][0] + RT[a][1] * Rm[b][1] + RT[a][2] * Rm[b][2];
}

template <class T>
__device__ __forceinline__ void cross(const T a[3], const T b[3], T c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// I^-1 (xx, yy, zz, xy, xz, yz) times v
template <class T>
__device__ __forceinline__ void sym_mul(const T I[6], const T v[3], T out[3])
{
    out[0] = I[0] * v[0] + I[3] * v[1] + I[4] * v[2];
    out[1] = I[3] * v[0] + I[1] * v[1] + I[5] * v[2];
    out[2] = I[4] * v[0] + I[5] * v[1] + I[2] * v[2];
}

// --- the one-contact problem with a full Delassus block --------------------
// 1. separation (p = 0) whenever b_n >= 0;  2. sticking p = -W^-1 b inside
// the cone;  3. sliding p = p_n (1, mu cos th, mu sin th): u_n = 0 gives
// p_n = -b_n / D(th), D = Wnn + mu (Wnt cos th + Wno sin th) > 0, and u_to
// must point against (cos th, sin th): the cross product of the two
// vanishes, a trigonometric polynomial of degree 2 in th (a quartic in
// tan(th/2), the route of Bonnefon et al. cited in Sect. 3).  Its roots
// are bracketed by 64 equal samples of [0, 2 pi) and refined inside the
// bracket (safeguarded Newton on the polynomial expanded in cos, sin);
// a root qualifies if D > 0 and u_to . (cos th, sin th) <= 0; the one of
// least 1/2 p.W p + b.p is taken (the first in th on ties).  Without a
// qualifying root (a double root the samples miss), the diagonal solution
// with w_n = Wnn, w_t = (Wtt + Woo)/2.
template <class R>
__device__ __forceinline__ void slide_dut(const Sym3<R>& W, R mu, const R b[3], R c, R s, R& D, R& vt, R& vo)
{
    D = W.nn + mu * (W.nt * c + W.no * s);
    vt = -b[0] * (W.nt + mu * (W.tt * c + W.to * s)) + D * b[1];
    vo = -b[0] * (W.no + mu * (W.to * c + W.oo * s)) + D * b[2];
}

template <class R>
__device__ __forceinline__ R energy(const Sym3<R>& W, const R b[3], const R p[3])
{
    const R w0 = W.nn * p[0] + W.nt * p[1] + W.no * p[2];
    const R w1 = W.nt * p[0] + W.tt * p[1] + W.to * p[2];
    const R w2 = W.no * p[0] + W.to * p[1] + W.oo * p[2];
    return p[0] * (R(0.5) * w0 + b[0]) + p[1] * (R(0.5) * w1 + b[1]) + p[2] * (R(0.5) * w2 + b[2]);
}

// cos and sin of the 64 sample angles 2 pi k / 64 (set from the host's libm)
__constant__ double c_cos64[64], c_sin64[64];
__constant__ float c_cos32[64], c_sin32[64];

template <class R> __device__ __forceinline__ R tab_cos(int k);
template <class R> __device__ __forceinline__ R tab_sin(int k);
template <> __device__ __forceinline__ float tab_cos<float>(int k) { return c_cos32[k]; }
template <> __device__ __forceinline__ float tab_sin<float>(int k) { return c_sin32[k]; }
template <> __device__ __forceinline__ double tab_cos<double>(int k) { return c_cos64[k]; }
template <> __device__ __forceinline__ double tab_sin<double>(int k) { return c_sin64[k]; }

// cos and sin of an angle th in [0, 2 pi]: in FP32 the hardware
// approximations on th moved into [-pi, pi] (their absolute error there is
// below 2^-21, far inside what an FP32 sweep resolves; the root found is
// the root of g to that accuracy), in FP64 the library's sincos.
template <class R>
__device__ __forceinline__ void slide_sincos(R th, R& sn, R& cs)
{
    if constexpr (sizeof(R) == 4) {
        const float t = th > 3.14159265f ? th - 6.28318531f : th;
        __sincosf(t, &sn, &cs);
    } else {
        sincos(th, &sn, &cs);
    }
}

// g(th) of the sliding condition, expanded in c = cos th, s = sin th.
template <class R>
__device__ __forceinline__ R slide_g(const R co[5], R c, R s)
{
    return co[0] * s + co[1] * c + co[2] * s * c + co[3] * s * s + co[4] * c * c;
}

// The root of g in the bracket [k dth, (k + 1) dth] (g(lo) = glo, g(hi) =
// ghi of opposite signs, or glo = 0: the sample itself): Newton steps from
// the secant point, kept inside the bracket (bisection where a step would
// leave it).
template <class R>
__device__ __forceinline__ R slide_root(const R co[5], int k, R glo, R ghi, R dth)
{
    constexpr int kIter = sizeof(R) == 4 ? 12 : 24;
    if (glo == R(0)) return dth * (R)k;
    R lo = dth * (R)k, hi = dth * (R)(k + 1);
    R gl = glo;
    R th = lo + (hi - lo) * (glo / (glo - ghi));
    for (int it = 0; it < kIter; ++it) {
        R sn, cs;
        slide_sincos(th, sn, cs);
        const R g = slide_g(co, cs, sn);
        if (g == R(0)) break;
        if ((g < R(0)) == (gl < R(0))) {
            lo = th;
            gl = g;
        } else {
            hi = th;
        }
        const R dg = co[0] * cs - co[1] * sn + co[2] * (cs * cs - sn * sn) + R(2) * (co[3] - co[4]) * sn * cs;
        const R step = g / dg;
        // a step below the resolution of th: converged (checked before the
        // bracket, which has shrunk onto th)
        if (fabs(step) <= (R)(sizeof(R) == 4 ? 1e-7 : 1e-15) * (R(1) + fabs(th))) break;
        R nt = th - step;
        if (!(nt > lo && nt < hi)) nt = R(0.5) * (lo + hi);
        th = nt;
    }
    return th;
}

// The sliding state at th, if it qualifies (D > 0, u_to against the
// friction direction), replaces the best one so far when its energy is
// lower (the first in th on ties).
template <class R>
__device__ __forceinline__ void slide_candidate(const Sym3<R>& W, R mu, const R b[3], R th, bool& found, R& best,
                                                R p[3])
{
    R sn, cs, D, vt, vo;
    slide_sincos(th, sn, cs);
    slide_dut(W, mu, b, cs, sn, D, vt, vo);
    if (!(D > R(0)) || cs * vt + sn * vo > R(0)) return;
    const R pn = -b[0] / D;
    const R q[3] = {pn, mu * pn * cs, mu * pn * sn};
    const R e = energy(W, b, q);
    if (!found || e < best) {
        best = e;
        p[0] = q[0];
        p[1] = q[1];
        p[2] = q[2];
        found = true;
    }
}

template <class R>
__device__ void one_contact_general(const Sym3<R>& W, R mu, const R b[3], R p[3])
{
    p[0] = p[1] = p[2] = R(0);
    if (b[0] >= R(0)) return;
    // sticking: Cramer's rule
    const R c00 = W.tt * W.oo - W.to * W.to;
    const R c01 = W.to * W.no - W.nt * W.oo;
    const R c02 = W.nt * W.to - W.tt * W.no;
    const R det = W.nn * c00 + W.nt * c01 + W.no * c02;
    const R i01 = W.no * W.to - W.nt * W.oo, i02 = W.nt * W.to - W.no * W.tt;
    const R i11 = W.nn * W.oo - W.no * W.no, i12 = W.no * W.nt - W.nn * W.to;
    const R i22 = W.nn * W.tt - W.nt * W.nt;
    const R ps0 = -(c00 * b[0] + i01 * b[1] + i02 * b[2]) / det;
    const R ps1 = -(c01 * b[0] + i11 * b[1] + i12 * b[2]) / det;
    const R ps2 = -(c02 * b[0] + i12 * b[1] + i22 * b[2]) / det;
    if (ps0 > R(0) && sqrt(ps1 * ps1 + ps2 * ps2) <= mu * ps0) {
        p[0] = ps0;
        p[1] = ps1;
        p[2] = ps2;
        return;
    }
    // sliding: the condition (cos th, sin th) x D u_to = 0 expanded in
    // c = cos th, s = sin th: g = P1 s + Q1 c + Rsc s c + S2 s^2 + C2 c^2
    const R co[5] = {b[0] * W.nt - b[1] * W.nn, b[2] * W.nn - b[0] * W.no,
                     mu * (b[0] * (W.tt - W.oo) - b[1] * W.nt + b[2] * W.no), mu * (b[0] * W.to - b[1] * W.no),
                     mu * (b[2] * W.nt - b[0] * W.to)};
    constexpr int K = 64;
    const R two_pi = (R)6.283185307179586;
    const R dth = two_pi / (R)K;
    bool found = false;
    R best = R(0);
    // Pass 1 finds the brackets (at most four sign changes: g has degree 2
    // in cos and sin), pass 2 refines them in order.  Refining inside the
    // sampling loop would run one lane's refinement at a time (lanes meet
    // their roots at different samples); in pass 2 the lanes of a warp
    // refine their r-th roots together.  More than four (rounding near a
    // double root): the sampling loop refines as it goes.
    int nbr = 0, k0 = 0, k1 = 0, k2 = 0, k3 = 0;
    R l0 = R(0), l1 = R(0), l2 = R(0), l3 = R(0), h0 = R(0), h1 = R(0), h2 = R(0), h3 = R(0);
    R gprev = slide_g(co, tab_cos<R>(0), tab_sin<R>(0));
    for (int k = 0; k < K; ++k) {
        const int kn = k + 1 == K ? 0 : k + 1;
        const R glo = gprev;
        const R ghi = slide_g(co, tab_cos<R>(kn), tab_sin<R>(kn));
        gprev = ghi;
        if (!(glo == R(0) || ((glo < R(0)) != (ghi < R(0)) && ghi != R(0)))) continue;
        if (nbr == 0) {
            k0 = k;
            l0 = glo;
            h0 = ghi;
        } else if (nbr == 1) {
            k1 = k;
            l1 = glo;
            h1 = ghi;
        } else if (nbr == 2) {
            k2 = k;
            l2 = glo;
            h2 = ghi;
        } else if (nbr == 3) {
            k3 = k;
            l3 = glo;
            h3 = ghi;
        }
        ++nbr;
    }
    if (nbr <= 4) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (r >= nbr) break;
            const int k = r == 0 ? k0 : (r == 1 ? k1 : (r == 2 ? k2 : k3));
            const R glo = r == 0 ? l0 : (r == 1 ? l1 : (r == 2 ? l2 : l3));
            const R ghi = r == 0 ? h0 : (r == 1 ? h1 : (r == 2 ? h2 : h3));
            slide_candidate(W, mu, b, slide_root(co, k, glo, ghi, dth), found, best, p);
        }
    } else {
        gprev = slide_g(co, tab_cos<R>(0), tab_sin<R>(0));
        for (int k = 0; k < K; ++k) {
            const int kn = k + 1 == K ? 0 : k + 1;
            const R glo = gprev;
            const R ghi = slide_g(co, tab_cos<R>(kn), tab_sin<R>(kn));
            gprev = ghi;
            if (!(glo == R(0) || ((glo < R(0)) != (ghi < R(0)) && ghi != R(0)))) continue;
            slide_candidate(W, mu, b, slide_root(co, k, glo, ghi, dth), found, best, p);
        }
    }
    if (found) return;
    // diagonal fallback (the closed form of spheres)
    const R wt = R(0.5) * (W.tt + W.oo);
    R pn = -b[0] / W.nn;
    pn = pn > R(0) ? pn : R(0);
    R pt = -b[1] / wt, po = -b[2] / wt;
    const R lim = mu * pn, len = sqrt(pt * pt + po * po);
    if (len > lim) {
        if (len > R(0)) {
            pt *= lim / len;
            po *= lim / len;
        } else {
            pt = po = R(0);
        }
    }
    p[0] = pn;
    p[1] = pt;
    p[2] = po;
}

// --- per-step kernels -----------------------------------------------------
__global__ void k_comp_ends(int64_t C, int64_t nm, int64_t nb, const uint32_t* __restrict__ cj1,
                            const uint32_t* __restrict__ cj2, const uint32_t* __restrict__ mbody,
                            uint32_t* __restrict__ cb1, uint32_t* __restrict__ cb2)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        cb1[c] = mbody[cj1[c]];
        const uint32_t b = cj2[c];
        cb2[c] = b < (uint64_t)nm ? mbody[b] : (uint32_t)nb;
    }
}

// World inverse inertia of every body for the step (FP64, and its copy in
// the sweep record of the body).
template <class R>
__global__ void k_comp_iinv(int64_t nb, const double4_32a* __restrict__ bquat, const double* __restrict__ bI0inv,
                            double* __restrict__ bIinv, R4<R>* __restrict__ bvel)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
        double Rm[3][3], T[3][3];
        quat_rows(bquat[i], Rm);
        to_world(Rm, bI0inv + 9 * i, T);
        const double I6[6] = {T[0][0], T[1][1], T[2][2], T[0][1], T[0][2], T[1][2]};
        for (int k = 0; k < 6; ++k) bIinv[6 * i + k] = I6[k];
        R4<R> a, b;
        a.x = (R)I6[0];
        a.y = (R)I6[1];
        a.z = (R)I6[2];
        a.w = (R)I6[3];
        b.x = (R)I6[4];
        b.y = (R)I6[5];
        b.z = R(0);
        b.w = R(0);
        bvel[4 * i + 2] = a;
        bvel[4 * i + 3] = b;
    }
}

// A canonical contact position per body for the dependency windows: the
// first contact of its first member (any fixed position serves).
__global__ void k_comp_anchor(int64_t nb, const uint32_t* __restrict__ bfirst, const uint32_t* __restrict__ row_off,
                              uint32_t* __restrict__ anchor)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x)
        anchor[b] = row_off[bfirst[b]];
}

// Sweep record of slot s (contact perm[s]) and its initial impulse.
// Component k of the normal of a contact's geometry record.
__device__ __forceinline__ double g_comp(const double4_32a& g, int k) { return k == 0 ? g.x : (k == 1 ? g.y : g.z); }

template <class R>
__global__ void k_comp_records(int64_t C, int64_t nm, const uint32_t* __restrict__ perm,
                               const uint32_t* __restrict__ cj1, const uint32_t* __restrict__ cj2,
                               const uint32_t* __restrict__ mbody, const double4_32a* __restrict__ moff,
                               const double4_32a* __restrict__ bquat, const double* __restrict__ bIinv,
                               const double* __restrict__ binvm, const double4_32a* __restrict__ cgeo,
                               const double2* __restrict__ clev, double dt, double beta, double mu, int warm,
                               const uint32_t* __restrict__ prev_row_off, const uint32_t* __restrict__ prev_j2,
                               const double4_32a* __restrict__ prev_P, CompRec<R>* __restrict__ rec,
                               R4<R>* __restrict__ p)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < C; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = perm[s];
        const uint32_t ma = cj1[c], mbm = cj2[c];
        const uint32_t A = mbody[ma];
        const bool hasB = mbm < (uint64_t)nm;
        const uint32_t B = hasB ? mbody[mbm] : 0xFFFFFFFFu;
        const double4_32a g = cgeo[c];
        const double2 l = clev[c];
        // the block and the levers in the sweep's precision R (FP64 arithmetic
        // is scarce on this GPU; an FP32 sweep reads them in FP32 anyway), in
        // the frame the sweep builds from the normal as stored
        const R n[3] = {(R)g.x, (R)g.y, (R)g.z};
        R t[3], o[3];
        tangent_basis<R>(n[0], n[1], n[2], t[0], t[1], t[2], o[0], o[1], o[2]);
        // levers from the centres of mass to x_hat: R_A d_a - l_a n, R_B d_b + l_b n
        double Rm[3][3];
        quat_rows(bquat[A], Rm);
        const double4_32a da = moff[ma];
        R lA[3], lB[3] = {R(0), R(0), R(0)};
        for (int k = 0; k < 3; ++k)
            lA[k] = (R)((Rm[k][0] * da.x + Rm[k][1] * da.y + Rm[k][2] * da.z) - l.x * g_comp(g, k));
        if (hasB) {
            quat_rows(bquat[B], Rm);
            const double4_32a db = moff[mbm];
            for (int k = 0; k < 3; ++k)
                lB[k] = (R)((Rm[k][0] * db.x + Rm[k][1] * db.y + Rm[k][2] * db.z) + l.y * g_comp(g, k));
        }
        // W = sum 1/m 1 - [l]x I^-1 [l]x, then W_c = F^T W F, F = [n t o]
        R Wd[3][3] = {{R(0), R(0), R(0)}, {R(0), R(0), R(0)}, {R(0), R(0), R(0)}};
        for (int body = 0; body < (hasB ? 2 : 1); ++body) {
            const uint32_t id = body == 0 ? A : B;
            const R im = (R)binvm[id];
            if (!(im > R(0))) continue;
            const double* I6d = bIinv + 6 * id;
            const R I6[6] = {(R)I6d[0], (R)I6d[1], (R)I6d[2], (R)I6d[3], (R)I6d[4], (R)I6d[5]};
            const R* lv = body == 0 ? lA : lB;
            for (int col = 0; col < 3; ++col) {
                R e[3] = {R(0), R(0), R(0)}, lxe[3], Il[3], cc[3];
                e[col] = R(1);
                cross(lv, e, lxe);
                sym_mul(I6, lxe, Il);
                cross(Il, lv, cc);
                for (int r = 0; r < 3; ++r) Wd[r][col] += (r == col ? im : R(0)) + cc[r];
            }
        }
        const R* F[3] = {n, t, o};
        R Wc[3][3];
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) {
                R acc = R(0);
                for (int r = 0; r < 3; ++r) acc += F[x][r] * (Wd[r][0] * F[y][0] + Wd[r][1] * F[y][1] + Wd[r][2] * F[y][2]);
                Wc[x][y] = acc;
            }
        const double xs = g.w >= 0.0 ? g.w : beta * g.w;
        const double bias = xs / dt;
        CompRec<R> rr;
        if constexpr (sizeof(R) == 4) {
            rr.a = make_float4(__uint_as_float(A), __uint_as_float(B), (float)bias, 0.f);
        } else {
            rr.a = make_double4_32a(__longlong_as_double((long long)(((uint64_t)B << 32) | A)), bias, 0.0, 0.0);
        }
        rr.b.x = (R)n[0];
        rr.b.y = (R)n[1];
        rr.b.z = (R)n[2];
        rr.b.w = (R)Wc[0][0];
        rr.c.x = (R)lA[0];
        rr.c.y = (R)lA[1];
        rr.c.z = (R)lA[2];
        rr.c.w = (R)Wc[1][1];
        rr.d.x = (R)lB[0];
        rr.d.y = (R)lB[1];
        rr.d.z = (R)lB[2];
        rr.d.w = (R)Wc[2][2];
        rr.e.x = (R)Wc[0][1];
        rr.e.y = (R)Wc[0][2];
        rr.e.z = (R)Wc[1][2];
        rr.e.w = R(0);
        rec[s] = rr;
        // warm start: the previous world impulse in the new frame, in the cone
        R pn = R(0), pt = R(0), po = R(0), found = R(0);
        if (warm) {
            const uint32_t e = prev_row_off[ma + 1];
            for (uint32_t k = prev_row_off[ma]; k < e; ++k) {
                if (prev_j2[k] != mbm) continue;
                const double4_32a P = prev_P[k];
                found = R(1);
                pn = (R)(n[0] * P.x + n[1] * P.y + n[2] * P.z);
                if (!(pn > R(0))) pn = R(0);
                pt = (R)(t[0] * P.x + t[1] * P.y + t[2] * P.z);
                po = (R)(o[0] * P.x + o[1] * P.y + o[2] * P.z);
                const R lim = (R)mu * pn, len = sqrt(pt * pt + po * po);
                if (len > lim) {
                    if (len > R(0)) {
                        pt *= lim / len;
                        po *= lim / len;
                    } else {
                        pt = po = R(0);
                    }
                }
                break;
            }
        }
        R4<R> q;
        q.x = pn;
        q.y = pt;
        q.z = po;
        q.w = found;
        p[s] = q;
    }
}

// eq. (integrationscheme) without contact reactions: v += dt g,
// w += dt I^-1 (-w x I w), I = R I0 R^T at the start of the step.
template <class R>
__global__ void k_comp_velinit(int64_t nb, const double4_32a* __restrict__ bquat, const double* __restrict__ bI0,
                               const double* __restrict__ bIinv, const double* __restrict__ binvm, double3 gdt,
                               double dt, R4<R>* __restrict__ bvel)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
        if (!(binvm[i] > 0.0)) continue;
        R4<R> v = bvel[4 * i], w = bvel[4 * i + 1];
        double Rm[3][3], I[3][3];
        quat_rows(bquat[i], Rm);
        to_world(Rm, bI0 + 9 * i, I);
        const double wv[3] = {(double)w.x, (double)w.y, (double)w.z};
        double L[3], g[3], dw[3];
        for (int k = 0; k < 3; ++k) L[k] = I[k][0] * wv[0] + I[k][1] * wv[1] + I[k][2] * wv[2];
        cross(wv, L, g);
        for (int k = 0; k < 3; ++k) g[k] = -g[k];
        sym_mul(bIinv + 6 * i, g, dw);
        w.x = (R)(wv[0] + dt * dw[0]);
        w.y = (R)(wv[1] + dt * dw[1]);
        w.z = (R)(wv[2] + dt * dw[2]);
        v.x = (R)((double)v.x + gdt.x);
        v.y = (R)((double)v.y + gdt.y);
        v.z = (R)((double)v.z + gdt.z);
        bvel[4 * i] = v;
        bvel[4 * i + 1] = w;
    }
}

template <class R> struct CompArgs {
    int local;                 // dependency windows (else a grid barrier after every colour)
    int* prog;                 // per block: last sweep phase completed
    const int2* dep;           // per (colour, block): ring window of blocks sharing bodies with the chunk
    const uint32_t* cstart;    // per colour, B + 1 chunk boundaries
    int64_t C, nb;
    const CompRec<R>* rec;
    R4<R>* p;
    R4<R>* bv;
    const uint32_t* col_off;
    DevInfo* info;
    R mu, omega;
    double gdt_norm;
    int max_sweeps;
    double tol;
    int warm;
};

// Relax one composite contact (apply_only: add the stored impulse), its
// record and impulse already loaded.
template <class R, bool apply_only>
__device__ __forceinline__ R relax_comp_loaded(const CompArgs<R>& A, int64_t s, const CompRec<R>& rr, const R4<R>& pp)
{
    uint32_t ia, ib;
    R bias;
    if constexpr (sizeof(R) == 4) {
        ia = __float_as_uint(rr.a.x);
        ib = __float_as_uint(rr.a.y);
        bias = rr.a.z;
    } else {
        const uint64_t ids = (uint64_t)__double_as_longlong(rr.a.x);
        ia = (uint32_t)(ids & 0xFFFFFFFFu);
        ib = (uint32_t)(ids >> 32);
        bias = rr.a.y;
    }
    const bool hasB = ib < (uint64_t)A.nb;
    const Sym3<R> W = {rr.b.w, rr.c.w, rr.d.w, rr.e.x, rr.e.y, rr.e.z};
    if (!(W.nn > R(0))) return R(0);
    const R n[3] = {rr.b.x, rr.b.y, rr.b.z};
    const R lA[3] = {rr.c.x, rr.c.y, rr.c.z}, lB[3] = {rr.d.x, rr.d.y, rr.d.z};
    R t[3], o[3];
    tangent_basis<R>(n[0], n[1], n[2], t[0], t[1], t[2], o[0], o[1], o[2]);
    // a body's state is 4 vectors: v, w and the 6 entries of its world inverse
    // inertia, read as two 256-bit accesses
    R4<R> va, wa, ia1, ia2;
    ld_body(A.bv + 4 * (int64_t)ia, va, wa);
    ld_body(A.bv + 4 * (int64_t)ia + 2, ia1, ia2);
    R4<R> vb, wb, ib1, ib2;
    vb.x = vb.y = vb.z = vb.w = R(0);
    wb = ib1 = ib2 = vb;
    if (hasB) {
        ld_body(A.bv + 4 * (int64_t)ib, vb, wb);
        ld_body(A.bv + 4 * (int64_t)ib + 2, ib1, ib2);
    }
    R d[3];
    if (apply_only) {
        d[0] = pp.x;
        d[1] = pp.y;
        d[2] = pp.z;
    } else {
        const R wav[3] = {wa.x, wa.y, wa.z}, wbv[3] = {wb.x, wb.y, wb.z};
        R ca[3], cb[3];
        cross(wav, lA, ca);
        cross(wbv, lB, cb);
        const R u[3] = {(va.x + ca[0]) - (vb.x + cb[0]), (va.y + ca[1]) - (vb.y + cb[1]),
                        (va.z + ca[2]) - (vb.z + cb[2])};
        const R un = n[0] * u[0] + n[1] * u[1] + n[2] * u[2];
        const R ut = t[0] * u[0] + t[1] * u[1] + t[2] * u[2];
        const R uo = o[0] * u[0] + o[1] * u[1] + o[2] * u[2];
        R b[3];
        b[0] = (un - (W.nn * pp.x + W.nt * pp.y + W.no * pp.z)) + bias;
        b[1] = ut - (W.nt * pp.x + W.tt * pp.y + W.to * pp.z);
        b[2] = uo - (W.no * pp.x + W.to * pp.y + W.oo * pp.z);
        R y[3];
        one_contact_general<R>(W, A.mu, b, y);
        const R om = A.omega, om1 = R(1) - A.omega;
        R4<R> q;
        q.x = om * y[0] + om1 * pp.x;
        q.y = om * y[1] + om1 * pp.y;
        q.z = om * y[2] + om1 * pp.z;
        q.w = R(0);
        d[0] = q.x - pp.x;
        d[1] = q.y - pp.y;
        d[2] = q.z - pp.z;
        A.p[s] = q;
    }
    const R P[3] = {d[0] * n[0] + d[1] * t[0] + d[2] * o[0], d[0] * n[1] + d[1] * t[1] + d[2] * o[1],
                    d[0] * n[2] + d[1] * t[2] + d[2] * o[2]};
    if (va.w > R(0)) {
        const R I6[6] = {ia1.x, ia1.y, ia1.z, ia1.w, ia2.x, ia2.y};
        R tq[3], dw[3];
        cross(lA, P, tq);
        sym_mul(I6, tq, dw);
        va.x += va.w * P[0];
        va.y += va.w * P[1];
        va.z += va.w * P[2];
        wa.x += dw[0];
        wa.y += dw[1];
        wa.z += dw[2];
        st_body(A.bv + 4 * (int64_t)ia, va, wa);
    }
    if (hasB && vb.w > R(0)) {
        const R I6[6] = {ib1.x, ib1.y, ib1.z, ib1.w, ib2.x, ib2.y};
        R tq[3], dw[3];
        cross(lB, P, tq);
        sym_mul(I6, tq, dw);
        vb.x -= vb.w * P[0];
        vb.y -= vb.w * P[1];
        vb.z -= vb.w * P[2];
        wb.x -= dw[0];
        wb.y -= dw[1];
        wb.z -= dw[2];
        st_body(A.bv + 4 * (int64_t)ib, vb, wb);
    }
    const R r0 = W.nn * d[0] + W.nt * d[1] + W.no * d[2];
    const R r1 = W.nt * d[0] + W.tt * d[1] + W.to * d[2];
    const R r2 = W.no * d[0] + W.to * d[1] + W.oo * d[2];
    return sqrt(r0 * r0 + r1 * r1 + r2 * r2);
}

template <class R, bool apply_only>
__device__ __forceinline__ R relax_comp(const CompArgs<R>& A, int64_t s)
{
    const CompRec<R> rr = A.rec[s];
    const R4<R> pp = A.p[s];
    return relax_comp_loaded<R, apply_only>(A, s, rr, pp);
}

__device__ __forceinline__ void block_max_atomic(double x, unsigned long long* dst)
{
    __shared__ double sm[32];
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) x = fmax(x, sm[k]);
        if (!(x <= 1e300)) x = __longlong_as_double(0x7FF0000000000000LL);
        atomicMax(dst, (unsigned long long)__double_as_longlong(x));
    }
    __syncthreads();
}

constexpr int kCompThreads = 256;

// The whole composite solve in one cooperative launch: the initial impulses
// colour by colour, then the sweeps, a grid barrier after every colour (each
// colour's contacts touch disjoint finite bodies) and R_k after every sweep.
template <class R>
__global__ void __launch_bounds__(kCompThreads) k_solve_comp(CompArgs<R> A)
{
    const unsigned nb = gridDim.x;
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    const int ncol = (int)A.info->n_colours;
    double vref = __longlong_as_double((long long)A.info->vmax_bits);
    vref = fmax(fmax(vref, A.gdt_norm), 1e-12);
    if (A.warm) {
        for (int c = 0; c < ncol; ++c) {
            for (int64_t s = A.col_off[c] + gtid; s < A.col_off[c + 1]; s += gstride) relax_comp<R, true>(A, s);
            if (!grid_barrier(A.info, nb)) return;
        }
    }
    __shared__ int s_ok;
    int k = 0;
    double Rk = 0.0;
    bool synced = true;
    for (; k < A.max_sweeps; ++k) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && k + 1 >= kHistKept) A.info->rk_bits[rk_slot(k + 1)] = 0ull;
        R rmax = R(0);
        for (int c = 0; c < ncol; ++c) {
            if (A.local) {
                // this block's chunk of the colour, after the blocks sharing
                // its bodies have finished the phase before
                const int g = k * ncol + c;
                int64_t b0, b1;
                colour_chunk(A.cstart, c, b0, b1);
                // the first record and impulse of this thread do not depend on
                // the neighbours: loaded before the wait
                const int64_t s0 = b0 + threadIdx.x;
                CompRec<R> rr;
                R4<R> pp;
                if (s0 < b1) {
                    rr = A.rec[s0];
                    pp = A.p[s0];
                }
                if (b1 > b0 && !wait_deps(A.prog, A.dep[c * (int)nb + blockIdx.x], g, A.info, &s_ok)) return;
                for (int64_t s = s0; s < b1; s += blockDim.x) {
                    if (s != s0) {
                        rr = A.rec[s];
                        pp = A.p[s];
                    }
                    const R r = relax_comp_loaded<R, false>(A, s, rr, pp);
                    rmax = r > rmax ? r : rmax;
                }
                if (c == ncol - 1) block_max_atomic((double)rmax, &A.info->rk_bits[rk_slot(k)]);
                publish(A.prog, g);
            } else {
                for (int64_t s = A.col_off[c] + gtid; s < A.col_off[c + 1]; s += gstride) {
                    const R r = relax_comp<R, false>(A, s);
                    rmax = r > rmax ? r : rmax;
                }
                if (c == ncol - 1) block_max_atomic((double)rmax, &A.info->rk_bits[rk_slot(k)]);
                if (!grid_barrier(A.info, nb)) return;
            }
        }
        synced = !A.local;
        // R_k needs every block: a grid barrier per sweep when the tolerance
        // is tested (and near the rotating residual slots)
        if (A.local && ncol > 0 && (A.tol > 0.0 || k + 2 >= kHistKept)) {
            if (!grid_barrier(A.info, nb)) return;
            synced = true;
        }
        if (synced) {
            Rk = __longlong_as_double((long long)((volatile unsigned long long*)A.info->rk_bits)[rk_slot(k)]) / vref;
            if (A.tol > 0.0 && ncol > 0 && Rk <= A.tol) {
                ++k;
                break;
            }
        }
    }
    if (!synced && k > 0) {
        if (!grid_barrier(A.info, nb)) return;
        Rk = __longlong_as_double((long long)((volatile unsigned long long*)A.info->rk_bits)[rk_slot(k - 1)]) / vref;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.info->sweeps_done = (uint32_t)k;
        A.info->residual = Rk;
        A.info->v_ref = vref;
    }
}

// x += dt v, q += dt Q(q) w renormalised (FP64), periodic wrap.
template <class R>
__global__ void k_comp_integrate(int64_t nb, double4_32a* __restrict__ bpos, double4_32a* __restrict__ bquat,
                                 const R4<R>* __restrict__ bvel, double dt, double3 lo, double3 L, int3 periodic)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
        const R4<R> v = bvel[4 * i], w = bvel[4 * i + 1];
        double4_32a x = bpos[i];
        x.x = xadd(x.x, xmul(dt, (double)v.x));
        x.y = xadd(x.y, xmul(dt, (double)v.y));
        x.z = xadd(x.z, xmul(dt, (double)v.z));
        const double4_32a q = bquat[i];
        const double qw = q.x, qx = q.y, qy = q.z, qz = q.w;
        const double wx = w.x, wy = w.y, wz = w.z;
        const double dw = 0.5 * (-qx * wx - qy * wy - qz * wz);
        const double dx = 0.5 * (qw * wx + qz * wy - qy * wz);
        const double dy = 0.5 * (-qz * wx + qw * wy + qx * wz);
        const double dz = 0.5 * (qy * wx - qx * wy + qw * wz);
        const double nw = qw + dt * dw, nx = qx + dt * dx, ny = qy + dt * dy, nz = qz + dt * dz;
        const double qn = sqrt(((nw * nw + nx * nx) + ny * ny) + nz * nz);
        bquat[i] = make_double4_32a(nw / qn, nx / qn, ny / qn, nz / qn);
        double* xs[3] = {&x.x, &x.y, &x.z};
        const double los[3] = {lo.x, lo.y, lo.z}, Ls[3] = {L.x, L.y, L.z};
        const int per[3] = {periodic.x, periodic.y, periodic.z};
        for (int a = 0; a < 3; ++a) {
            if (!per[a] || (*xs[a] >= los[a] && *xs[a] < los[a] + Ls[a])) continue;
            double sft = fmod(*xs[a] - los[a], Ls[a]);
            if (sft < 0.0) sft += Ls[a];
            *xs[a] = los[a] + sft;
        }
        bpos[i] = x;
    }
}

// staging: pos (3 nb) | quat (4 nb) | vel (3 nb) | angvel (3 nb)
template <class R>
__global__ void k_comp_pack(int64_t nb, double* __restrict__ stg, const double4_32a* __restrict__ bpos,
                            const double4_32a* __restrict__ bquat, const R4<R>* __restrict__ bvel)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
        const double4_32a x = bpos[i], q = bquat[i];
        const R4<R> v = bvel[4 * i], w = bvel[4 * i + 1];
        stg[3 * i] = x.x;
        stg[3 * i + 1] = x.y;
        stg[3 * i + 2] = x.z;
        stg[3 * nb + 4 * i] = q.x;
        stg[3 * nb + 4 * i + 1] = q.y;
        stg[3 * nb + 4 * i + 2] = q.z;
        stg[3 * nb + 4 * i + 3] = q.w;
        stg[7 * nb + 3 * i] = v.x;
        stg[7 * nb + 3 * i + 1] = v.y;
        stg[7 * nb + 3 * i + 2] = v.z;
        stg[10 * nb + 3 * i] = w.x;
        stg[10 * nb + 3 * i + 1] = w.y;
        stg[10 * nb + 3 * i + 2] = w.z;
    }
}

template <class R>
__global__ void k_comp_unpack(int64_t nb, const double* __restrict__ stg, int has_pos, int has_quat, int has_vel,
                              int has_ang, double4_32a* __restrict__ bpos, double4_32a* __restrict__ bquat,
                              R4<R>* __restrict__ bvel)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
        if (has_pos) {
            double4_32a x = bpos[i];
            x.x = stg[3 * i];
            x.y = stg[3 * i + 1];
            x.z = stg[3 * i + 2];
            bpos[i] = x;
        }
        if (has_quat)
            bquat[i] = make_double4_32a(stg[3 * nb + 4 * i], stg[3 * nb + 4 * i + 1], stg[3 * nb + 4 * i + 2],
                                        stg[3 * nb + 4 * i + 3]);
        if (has_vel) {
            R4<R> v = bvel[4 * i];
            v.x = (R)stg[7 * nb + 3 * i];
            v.y = (R)stg[7 * nb + 3 * i + 1];
            v.z = (R)stg[7 * nb + 3 * i + 2];
            bvel[4 * i] = v;
        }
        if (has_ang) {
            R4<R> w = bvel[4 * i + 1];
            w.x = (R)stg[10 * nb + 3 * i];
            w.y = (R)stg[10 * nb + 3 * i + 1];
            w.z = (R)stg[10 * nb + 3 * i + 2];
            bvel[4 * i + 1] = w;
        }
    }
}

size_t comp_rec_bytes(const nbgs_scene* s) { return s->fp32 ? sizeof(CompRec<float>) : sizeof(CompRec<double>); }

template <class R>
int comp_blocks(nbgs_scene* s)
{
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve_comp<R>, kCompThreads, 0);
    cudaGetLastError();
    return occ * s->num_sms;
}

template <class R>
nbgs_status solve_comp_impl(nbgs_scene* s, int max_sweeps, double tol)
{
    cudaStream_t st = s->stream;
    const int T = 256;
    const int nk = max_sweeps < kHistKept ? max_sweeps : kHistKept + 3;
    cudaMemsetAsync(s->info->rk_bits, 0, (size_t)(nk > 0 ? nk : 1) * sizeof(unsigned long long), st);
    cudaMemsetAsync(&s->info->barrier_count, 0, 2 * sizeof(uint32_t), st);
    const double* g = s->prm.gravity;
    const double3 gdt = make_double3(s->prm.dt * g[0], s->prm.dt * g[1], s->prm.dt * g[2]);
    if (s->timing) cudaEventRecord(s->ev[8], st);
    k_comp_velinit<R><<<grid_for(s->nb, T, 8, s->num_sms), T, 0, st>>>(s->nb, s->bquat, s->bI0, s->bIinv, s->binvm, gdt,
                                                                       s->prm.dt, (R4<R>*)s->bvel);
    CompArgs<R> A;
    A.C = s->n_contacts;
    A.nb = s->nb;
    A.rec = (const CompRec<R>*)s->crec;
    A.p = (R4<R>*)s->sp;
    A.bv = (R4<R>*)s->bvel;
    A.col_off = s->col_off;
    A.info = s->info;
    A.mu = (R)s->prm.mu;
    A.omega = (R)s->prm.omega;
    A.gdt_norm = sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]) * s->prm.dt;
    A.max_sweeps = max_sweeps;
    A.tol = tol;
    A.warm = (s->prm.warm_start == NBGS_WARM_PREV && s->have_prev) ? 1 : 0;
    const int blocks = std::min(comp_blocks<R>(s), s->max_coop_blocks);
    if (blocks < 1) return fail(s, NBGS_EINVAL, "composite solve: the device cannot launch it cooperatively");
    // local synchronisation unless a grid barrier per colour is asked for
    A.local = (A.C > 0 && !(s->prm.sweep_flags & NBGS_SWEEP_GLOBAL_SYNC)) ? 1 : 0;
    A.prog = s->prog;
    A.dep = s->dep;
    A.cstart = s->cstart;
    if (A.local) {
        k_comp_anchor<<<grid_for(s->nb, T, 8, s->num_sms), T, 0, st>>>(s->nb, s->bfirst, s->row_off, s->banchor);
        nbgs_status rc = build_windows(s, blocks, s->nb, s->cb1, s->cb2, s->banchor, s->bfinite);
        if (rc != NBGS_OK) return rc;
    }
    void* args[] = {&A};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_solve_comp<R>, dim3(blocks), dim3(kCompThreads), args, 0,
                                                st);
    if (s->timing) {
        cudaEventRecord(s->ev[9], st);
        s->phase_launches[2] += 2;
        s->sweep_launches += 1;
    }
    return cuda_check(s, e, "composite solve: cooperative launch");
}

}  // namespace

void free_composite_buffers(nbgs_scene* s)
{
    void* ps[] = {s->bpos, s->bquat, s->bvel, s->bI0, s->bI0inv, s->bIinv, s->binvm, s->bfinite, s->mbody,
                  s->moff, s->cb1, s->cb2, s->crec, s->bfirst, s->banchor};
    for (void* p : ps) dev_free(s, p);
}

// Contact-sized composite arrays for the current capacity.
nbgs_status ensure_composite_buffers(nbgs_scene* s)
{
    if (!s->composite) return NBGS_OK;
    if (s->comp_ccap == 0) {   // the sample angles of the one-contact solve
        double c64[64], s64[64];
        float c32[64], s32[64];
        for (int k = 0; k < 64; ++k) {
            const double th = 6.283185307179586 * k / 64;
            c64[k] = std::cos(th);
            s64[k] = std::sin(th);
            c32[k] = (float)c64[k];
            s32[k] = (float)s64[k];
        }
        cudaMemcpyToSymbolAsync(c_cos64, c64, sizeof(c64), 0, cudaMemcpyHostToDevice, s->stream);
        cudaMemcpyToSymbolAsync(c_sin64, s64, sizeof(s64), 0, cudaMemcpyHostToDevice, s->stream);
        cudaMemcpyToSymbolAsync(c_cos32, c32, sizeof(c32), 0, cudaMemcpyHostToDevice, s->stream);
        cudaMemcpyToSymbolAsync(c_sin32, s32, sizeof(s32), 0, cudaMemcpyHostToDevice, s->stream);
        nbgs_status rc = cuda_check(s, cudaStreamSynchronize(s->stream), "composite: sample table");
        if (rc != NBGS_OK) return rc;
    }
    if (s->comp_ccap >= s->ccap) return NBGS_OK;
    dev_free(s, s->cb1);
    dev_free(s, s->cb2);
    dev_free(s, s->crec);
    s->cb1 = (uint32_t*)dev_alloc(s, (size_t)s->ccap * sizeof(uint32_t));
    s->cb2 = (uint32_t*)dev_alloc(s, (size_t)s->ccap * sizeof(uint32_t));
    s->crec = dev_alloc(s, (size_t)s->ccap * comp_rec_bytes(s));
    if (!s->cb1 || !s->cb2 || !s->crec) return fail(s, NBGS_ENOMEM, "composite: allocation failed");
    s->comp_ccap = s->ccap;
    return NBGS_OK;
}

nbgs_status run_comp_ends(nbgs_scene* s)
{
    nbgs_status rc = ensure_composite_buffers(s);
    if (rc != NBGS_OK) return rc;
    const int64_t C = s->n_contacts;
    const int T = 256;
    k_comp_ends<<<grid_for(C, T, 8, s->num_sms), T, 0, s->stream>>>(C, s->n, s->nb, s->cj1, s->cj2, s->mbody, s->cb1,
                                                                     s->cb2);
    if (s->timing) s->phase_launches[1] += 1;
    return cuda_check(s, cudaGetLastError(), "composite: contact bodies");
}

nbgs_status run_comp_records(nbgs_scene* s, int warm)
{
    nbgs_status rc = ensure_composite_buffers(s);
    if (rc != NBGS_OK) return rc;
    cudaStream_t st = s->stream;
    const int64_t C = s->n_contacts;
    const int T = 256;
    if (s->fp32) {
        k_comp_iinv<float><<<grid_for(s->nb, T, 8, s->num_sms), T, 0, st>>>(s->nb, s->bquat, s->bI0inv, s->bIinv,
                                                                             (float4*)s->bvel);
        k_comp_records<float><<<grid_for(C, T, 8, s->num_sms), T, 0, st>>>(
            C, s->n, s->perm, s->cj1, s->cj2, s->mbody, s->moff, s->bquat, s->bIinv, s->binvm, s->cgeo, s->clev,
            s->prm.dt, s->prm.beta, s->prm.mu, warm, s->prev_row_off, s->prev_j2, s->prev_P,
            (CompRec<float>*)s->crec, (float4*)s->sp);
    } else {
        k_comp_iinv<double><<<grid_for(s->nb, T, 8, s->num_sms), T, 0, st>>>(s->nb, s->bquat, s->bI0inv, s->bIinv,
                                                                              (double4_32a*)s->bvel);
        k_comp_records<double><<<grid_for(C, T, 8, s->num_sms), T, 0, st>>>(
            C, s->n, s->perm, s->cj1, s->cj2, s->mbody, s->moff, s->bquat, s->bIinv, s->binvm, s->cgeo, s->clev,
            s->prm.dt, s->prm.beta, s->prm.mu, warm, s->prev_row_off, s->prev_j2, s->prev_P,
            (CompRec<double>*)s->crec, (double4_32a*)s->sp);
    }
    if (s->timing) s->phase_launches[1] += 2;
    return cuda_check(s, cudaGetLastError(), "composite: sweep records");
}

nbgs_status run_solve_comp(nbgs_scene* s, int max_sweeps, double tol)
{
    if (s->nb == 0) return NBGS_OK;
    if (s->n_contacts == 0) {   // the velocity step still runs (gravity, gyroscopic term)
        nbgs_status rc = ensure_composite_buffers(s);
        if (rc != NBGS_OK) return rc;
        const int T = 256;
        if (s->fp32)
            k_comp_iinv<float><<<grid_for(s->nb, T, 8, s->num_sms), T, 0, s->stream>>>(s->nb, s->bquat, s->bI0inv,
                                                                                        s->bIinv, (float4*)s->bvel);
        else
            k_comp_iinv<double><<<grid_for(s->nb, T, 8, s->num_sms), T, 0, s->stream>>>(
                s->nb, s->bquat, s->bI0inv, s->bIinv, (double4_32a*)s->bvel);
    }
    return s->fp32 ? solve_comp_impl<float>(s, max_sweeps, tol) : solve_comp_impl<double>(s, max_sweeps, tol);
}

nbgs_status run_integrate_comp(nbgs_scene* s)
{
    if (s->nb == 0) return NBGS_OK;
    cudaStream_t st = s->stream;
    if (s->timing) cudaEventRecord(s->ev[6], st);
    const double3 lo = make_double3(s->prm.box_lo[0], s->prm.box_lo[1], s->prm.box_lo[2]);
    const double3 L = make_double3(s->prm.box_hi[0] - s->prm.box_lo[0], s->prm.box_hi[1] - s->prm.box_lo[1],
                                   s->prm.box_hi[2] - s->prm.box_lo[2]);
    const int3 per = make_int3(s->prm.periodic[0], s->prm.periodic[1], s->prm.periodic[2]);
    const int T = 256, gb = grid_for(s->nb, T, 8, s->num_sms);
    if (s->fp32)
        k_comp_integrate<float><<<gb, T, 0, st>>>(s->nb, s->bpos, s->bquat, (const float4*)s->bvel, s->prm.dt, lo, L,
                                                  per);
    else
        k_comp_integrate<double><<<gb, T, 0, st>>>(s->nb, s->bpos, s->bquat, (const double4_32a*)s->bvel, s->prm.dt,
                                                   lo, L, per);
    if (s->timing) {
        s->phase_launches[3] += 1;
        cudaEventRecord(s->ev[7], st);
    }
    s->detected = s->coloured = false;
    return cuda_check(s, cudaGetLastError(), "composite: integrate");
}

nbgs_status run_comp_get_bodies(nbgs_scene* s, double* pos, double* quat, double* vel, double* angvel)
{
    const int64_t nb = s->nb;
    if (nb == 0) return NBGS_OK;
    cudaStream_t st = s->stream;
    const int T = 256;
    if (s->fp32)
        k_comp_pack<float><<<grid_for(nb, T, 8, s->num_sms), T, 0, st>>>(nb, s->stage, s->bpos, s->bquat,
                                                                         (const float4*)s->bvel);
    else
        k_comp_pack<double><<<grid_for(nb, T, 8, s->num_sms), T, 0, st>>>(nb, s->stage, s->bpos, s->bquat,
                                                                          (const double4_32a*)s->bvel);
    nbgs_status rc = cuda_check(s, cudaGetLastError(), "get_bodies");
    if (rc == NBGS_OK && pos)
        rc = cuda_check(s, cudaMemcpyAsync(pos, s->stage, 3 * nb * sizeof(double), cudaMemcpyDefault, st), "get pos");
    if (rc == NBGS_OK && quat)
        rc = cuda_check(s, cudaMemcpyAsync(quat, s->stage + 3 * nb, 4 * nb * sizeof(double), cudaMemcpyDefault, st),
                        "get quat");
    if (rc == NBGS_OK && vel)
        rc = cuda_check(s, cudaMemcpyAsync(vel, s->stage + 7 * nb, 3 * nb * sizeof(double), cudaMemcpyDefault, st),
                        "get vel");
    if (rc == NBGS_OK && angvel)
        rc = cuda_check(s, cudaMemcpyAsync(angvel, s->stage + 10 * nb, 3 * nb * sizeof(double), cudaMemcpyDefault, st),
                        "get angvel");
    if (rc == NBGS_OK) rc = cuda_check(s, cudaStreamSynchronize(st), "get_bodies");
    return rc;
}

nbgs_status run_comp_set_bodies(nbgs_scene* s, const double* pos, const double* quat, const double* vel,
                                const double* angvel)
{
    const int64_t nb = s->nb;
    if (nb == 0) return NBGS_OK;
    cudaStream_t st = s->stream;
    nbgs_status rc = NBGS_OK;
    if (pos) rc = cuda_check(s, cudaMemcpyAsync(s->stage, pos, 3 * nb * sizeof(double), cudaMemcpyDefault, st), "pos");
    if (rc == NBGS_OK && quat)
        rc = cuda_check(s, cudaMemcpyAsync(s->stage + 3 * nb, quat, 4 * nb * sizeof(double), cudaMemcpyDefault, st),
                        "quat");
    if (rc == NBGS_OK && vel)
        rc = cuda_check(s, cudaMemcpyAsync(s->stage + 7 * nb, vel, 3 * nb * sizeof(double), cudaMemcpyDefault, st),
                        "vel");
    if (rc == NBGS_OK && angvel)
        rc = cuda_check(s, cudaMemcpyAsync(s->stage + 10 * nb, angvel, 3 * nb * sizeof(double), cudaMemcpyDefault, st),
                        "angvel");
    if (rc != NBGS_OK) return rc;
    const int T = 256;
    if (s->fp32)
        k_comp_unpack<float><<<grid_for(nb, T, 8, s->num_sms), T, 0, st>>>(nb, s->stage, pos != nullptr,
                                                                           quat != nullptr, vel != nullptr,
                                                                           angvel != nullptr, s->bpos, s->bquat,
                                                                           (float4*)s->bvel);
    else
        k_comp_unpack<double><<<grid_for(nb, T, 8, s->num_sms), T, 0, st>>>(nb, s->stage, pos != nullptr,
                                                                            quat != nullptr, vel != nullptr,
                                                                            angvel != nullptr, s->bpos, s->bquat,
                                                                            (double4_32a*)s->bvel);
    rc = cuda_check(s, cudaGetLastError(), "set_bodies");
    if (rc == NBGS_OK) rc = cuda_check(s, cudaStreamSynchronize(st), "set_bodies");
    return rc;
}

}  // namespace nbgs

namespace nbgs {

// Independent one-contact problems with the solver of the composite sweep.
__global__ void k_one_contact(int64_t n, const double* __restrict__ W6, const double* __restrict__ mu,
                              const double* __restrict__ b, double* __restrict__ p)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double* w = W6 + 6 * i;
        const Sym3<double> W{w[0], w[1], w[2], w[3], w[4], w[5]};
        const double bb[3] = {b[3 * i], b[3 * i + 1], b[3 * i + 2]};
        double y[3];
        one_contact_general<double>(W, mu[i], bb, y);
        p[3 * i] = y[0];
        p[3 * i + 1] = y[1];
        p[3 * i + 2] = y[2];
    }
}

}  // namespace nbgs

extern "C" nbgs_status nbgs_one_contact(int64_t n, const double* W6, const double* mu, const double* b, double* p,
                                        void* stream)
{
    using namespace nbgs;
    if (n < 0 || (n > 0 && (!W6 || !mu || !b || !p))) return NBGS_EINVAL;
    if (n == 0) return NBGS_OK;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_one_contact<<<grid_for(n, 128, 8, sms), 128, 0, (cudaStream_t)stream>>>(n, W6, mu, b, p);
    return cudaGetLastError() == cudaSuccess ? NBGS_OK : NBGS_ECUDA;
}
