// solve.cu -- NBGS sweeps (Sect. 5, Alg. 1) and FP64 residuals.
//
// One relaxation of contact j (sweep record s):
//   u   = v_a + w_a x l_a - v_b - w_b x l_b              relative velocity (Sect. 2)
//   W   = diag(w_n, w_t, w_t) in the contact frame, w_n = 1/m_a + 1/m_b,
//         w_t = w_n + la^2/I_a + lb^2/I_b (levers parallel to n for spheres)
//   b   = (n.u - w_n p_n + xi'/dt, t.u - w_t p_t, o.u - w_t p_o)
//         (velocity without the contact's own reaction, plus the gap term of
//         eq. nonpenetration)
//   y   = F_j^{-1}(0, lambda_jbar): p_n = max(0, -b_n/w_n); stick impulse
//         -b_to/w_t projected radially onto the disk |p_to| <= mu p_n
//         (eq. coulomb; exact because W is diagonal)
//   p  <- omega y + (1 - omega) p                        (Alg. 1, relaxation)
//   v, w of both bodies += the impulse change             (Sect. 6.3, in place)
//   r_j = |W (p_new - p_old)|                             (convergence measure)
//
// Contacts of one colour touch disjoint finite bodies, so a colour is one
// data-parallel pass with plain loads and stores.
#include <cstring>

#include "nbgs_internal.cuh"

namespace nbgs {

template <class R> struct SolveArgs {
    int64_t n;
    int64_t C;
    R4<R>* vel;
    const SweepRec<R>* rec;
    R4<R>* p;
    const uint32_t* col_off;
    DevInfo* info;
    R mu, omega;
    R gdt[3];            // dt * gravity
    double gdt_norm;     // |g| dt
    int max_sweeps;
    double tol;
    int warm;
};

template <class R>
__device__ __forceinline__ void decode(const SweepRec<R>& r, uint32_t& a, uint32_t& b, R& la, R& lb, R& nx, R& ny, R& nz,
                                       R& bias);

template <>
__device__ __forceinline__ void decode<float>(const SweepRec<float>& r, uint32_t& a, uint32_t& b, float& la, float& lb,
                                              float& nx, float& ny, float& nz, float& bias)
{
    a = __float_as_uint(r.a.x);
    b = __float_as_uint(r.a.y);
    la = r.a.z;
    lb = r.a.w;
    nx = r.b.x;
    ny = r.b.y;
    nz = r.b.z;
    bias = r.b.w;
}

template <>
__device__ __forceinline__ void decode<double>(const SweepRec<double>& r, uint32_t& a, uint32_t& b, double& la,
                                               double& lb, double& nx, double& ny, double& nz, double& bias)
{
    const uint64_t ids = (uint64_t)__double_as_longlong(r.ids_bias.x);
    a = (uint32_t)(ids & 0xFFFFFFFFu);
    b = (uint32_t)(ids >> 32);
    bias = r.ids_bias.y;
    la = r.lev.x;
    lb = r.lev.y;
    nx = r.nxy.x;
    ny = r.nxy.y;
    nz = r.nz_.x;
}

template <class R>
__device__ __forceinline__ void load_rec(const SweepRec<R>* rec, int64_t s, SweepRec<R>& r)
{
    r = rec[s];
}

// Relax one contact; returns r_j.  apply_only: add the stored impulse p to
// the bodies (initial impulses of a warm start) instead of relaxing.
template <class R, bool apply_only>
__device__ __forceinline__ R relax(const SolveArgs<R>& A, int64_t s)
{
    SweepRec<R> rr;
    load_rec(A.rec, s, rr);
    uint32_t ia, ib;
    R la, lb, nx, ny, nz, bias;
    decode<R>(rr, ia, ib, la, lb, nx, ny, nz, bias);
    const R4<R> pp = A.p[s];
    R4<R> va = A.vel[2 * (int64_t)ia], wa = A.vel[2 * (int64_t)ia + 1];
    const bool dyn_b = ib < (uint32_t)A.n;
    R4<R> vb, wb;
    if (dyn_b) {
        vb = A.vel[2 * (int64_t)ib];
        wb = A.vel[2 * (int64_t)ib + 1];
    } else {
        vb.x = vb.y = vb.z = vb.w = R(0);
        wb = vb;
    }
    const R ima = va.w, iIa = wa.w, imb = vb.w, iIb = wb.w;
    R tx, ty, tz, ox, oy, oz;
    tangent_basis<R>(nx, ny, nz, tx, ty, tz, ox, oy, oz);
    const R wn = ima + imb;
    if (!(wn > R(0))) return R(0);  // both masses infinite: nothing can move
    const R wt = wn + iIa * la * la + iIb * lb * lb;
    R dn, dt_, do_;
    if (apply_only) {
        dn = pp.x;
        dt_ = pp.y;
        do_ = pp.z;
    } else {
        // u = v_a - la (w_a x n) - v_b - lb (w_b x n)
        const R cax = wa.y * nz - wa.z * ny, cay = wa.z * nx - wa.x * nz, caz = wa.x * ny - wa.y * nx;
        const R cbx = wb.y * nz - wb.z * ny, cby = wb.z * nx - wb.x * nz, cbz = wb.x * ny - wb.y * nx;
        const R ux = (va.x - la * cax) - (vb.x + lb * cbx);
        const R uy = (va.y - la * cay) - (vb.y + lb * cby);
        const R uz = (va.z - la * caz) - (vb.z + lb * cbz);
        const R un = nx * ux + ny * uy + nz * uz;
        const R ut = tx * ux + ty * uy + tz * uz;
        const R uo = ox * ux + oy * uy + oz * uz;
        const R bn = un - wn * pp.x + bias;
        const R bt = ut - wt * pp.y;
        const R bo = uo - wt * pp.z;
        R yn = -bn / wn;
        yn = yn > R(0) ? yn : R(0);
        R yt = -bt / wt, yo = -bo / wt;
        const R lim = A.mu * yn;
        const R len2 = yt * yt + yo * yo;
        if (len2 > lim * lim) {
            if (len2 > R(0)) {
                const R sc = lim / sqrt(len2);
                yt *= sc;
                yo *= sc;
            } else {
                yt = yo = R(0);
            }
        }
        const R om = A.omega, om1 = R(1) - A.omega;
        const R pn = om * yn + om1 * pp.x, pt = om * yt + om1 * pp.y, po = om * yo + om1 * pp.z;
        dn = pn - pp.x;
        dt_ = pt - pp.y;
        do_ = po - pp.z;
        R4<R> q;
        q.x = pn;
        q.y = pt;
        q.z = po;
        q.w = R(0);
        A.p[s] = q;
    }
    // world impulse change P = dn n + dt t + do o; torque arm n x P
    const R Px = dn * nx + dt_ * tx + do_ * ox;
    const R Py = dn * ny + dt_ * ty + do_ * oy;
    const R Pz = dn * nz + dt_ * tz + do_ * oz;
    const R qx = ny * Pz - nz * Py, qy = nz * Px - nx * Pz, qz = nx * Py - ny * Px;
    if (ima > R(0) || iIa > R(0)) {
        va.x += ima * Px;
        va.y += ima * Py;
        va.z += ima * Pz;
        const R ka = la * iIa;
        wa.x -= ka * qx;
        wa.y -= ka * qy;
        wa.z -= ka * qz;
        A.vel[2 * (int64_t)ia] = va;
        A.vel[2 * (int64_t)ia + 1] = wa;
    }
    if (dyn_b && (imb > R(0) || iIb > R(0))) {
        vb.x -= imb * Px;
        vb.y -= imb * Py;
        vb.z -= imb * Pz;
        const R kb = lb * iIb;
        wb.x -= kb * qx;
        wb.y -= kb * qy;
        wb.z -= kb * qz;
        A.vel[2 * (int64_t)ib] = vb;
        A.vel[2 * (int64_t)ib + 1] = wb;
    }
    const R r1 = wn * dn, r2 = wt * dt_, r3 = wt * do_;
    return sqrt(r1 * r1 + r2 * r2 + r3 * r3);
}

template <class R>
__device__ __forceinline__ void gravity_pass(const SolveArgs<R>& A, int64_t gtid, int64_t gstride)
{
    for (int64_t i = gtid; i < A.n; i += gstride) {
        R4<R> v = A.vel[2 * i];
        if (v.w > R(0)) {
            v.x += A.gdt[0];
            v.y += A.gdt[1];
            v.z += A.gdt[2];
            A.vel[2 * i] = v;
        }
    }
}

template <class R>
__device__ __forceinline__ double block_max_to(R v, unsigned long long* dst)
{
    __shared__ double sm[32];
    double x = (double)v;
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) x = fmax(x, sm[k]);
        if (!(x <= 1e300)) x = __longlong_as_double(0x7FF0000000000000LL);  // NaN/Inf -> +Inf
        atomicMax(dst, (unsigned long long)__double_as_longlong(x));
    }
    __syncthreads();
    return x;
}

__device__ __forceinline__ double v_ref_of(const DevInfo* info, double gdt_norm)
{
    double v = __longlong_as_double((long long)info->vmax_bits);
    v = fmax(v, gdt_norm);
    return fmax(v, 1e-12);
}

// Whole solve in one cooperative launch: gravity, warm-start impulses and
// the sweeps, with a bounded grid barrier after every colour.
template <class R>
__global__ void __launch_bounds__(256) k_solve_persistent(SolveArgs<R> A)
{
    const unsigned nb = gridDim.x;
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    const int ncol = (int)A.info->n_colours;
    const double vref = v_ref_of(A.info, A.gdt_norm);
    gravity_pass<R>(A, gtid, gstride);
    if (!grid_barrier(A.info, nb)) return;
    if (A.warm) {
        for (int c = 0; c < ncol; ++c) {
            const int64_t e = A.col_off[c + 1];
            for (int64_t s = A.col_off[c] + gtid; s < e; s += gstride) relax<R, true>(A, s);
            if (!grid_barrier(A.info, nb)) return;
        }
    }
    int k = 0;
    double Rk = 0.0;
    for (; k < A.max_sweeps; ++k) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && k + 1 >= kHistKept) A.info->rk_bits[rk_slot(k + 1)] = 0ull;
        R rmax = R(0);
        for (int c = 0; c < ncol; ++c) {
            const int64_t e = A.col_off[c + 1];
            for (int64_t s = A.col_off[c] + gtid; s < e; s += gstride) {
                const R r = relax<R, false>(A, s);
                rmax = r > rmax ? r : rmax;
            }
            if (c == ncol - 1) block_max_to<R>(rmax, &A.info->rk_bits[rk_slot(k)]);
            if (!grid_barrier(A.info, nb)) return;
        }
        Rk = __longlong_as_double((long long)((volatile unsigned long long*)A.info->rk_bits)[rk_slot(k)]) / vref;
        if (A.tol > 0.0 && Rk <= A.tol) {
            ++k;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.info->sweeps_done = (uint32_t)k;
        A.info->residual = Rk;
        A.info->v_ref = vref;
    }
}

// --- one launch per colour ------------------------------------------------
template <class R>
__global__ void k_gravity(SolveArgs<R> A)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.info->v_ref = v_ref_of(A.info, A.gdt_norm);
        A.info->residual = 0.0;
    }
    gravity_pass<R>(A, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

template <class R, bool apply_only>
__global__ void __launch_bounds__(256) k_relax_colour(SolveArgs<R> A, int colour, int sweep)
{
    if (!apply_only && A.info->sweeps_done != 0xFFFFFFFFu) return;  // converged earlier
    const int64_t b = A.col_off[colour], e = A.col_off[colour + 1];
    R rmax = R(0);
    for (int64_t s = b + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < e; s += (int64_t)gridDim.x * blockDim.x) {
        const R r = relax<R, apply_only>(A, s);
        rmax = r > rmax ? r : rmax;
    }
    if (!apply_only) block_max_to<R>(rmax, &A.info->rk_bits[rk_slot(sweep)]);
}

template <class R>
__global__ void k_sweep_done(SolveArgs<R> A, int sweep)
{
    if (threadIdx.x != 0 || A.info->sweeps_done != 0xFFFFFFFFu) return;
    const double vref = v_ref_of(A.info, A.gdt_norm);
    const double Rk = __longlong_as_double((long long)A.info->rk_bits[rk_slot(sweep)]) / vref;
    if (sweep + 1 >= kHistKept) A.info->rk_bits[rk_slot(sweep + 1)] = 0ull;
    A.info->residual = Rk;
    A.info->v_ref = vref;
    if ((A.tol > 0.0 && Rk <= A.tol) || sweep + 1 == A.max_sweeps) A.info->sweeps_done = (uint32_t)(sweep + 1);
}

// Canonical impulses (contact frame) and world-frame impulses for the next
// warm start.
template <class R>
__global__ void k_finish(int64_t C, const uint32_t* __restrict__ perm, const R4<R>* __restrict__ p,
                         const double4_32a* __restrict__ cgeo, double4_32a* __restrict__ cimp, double4_32a* __restrict__ cworld)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < C; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = perm[s];
        const R4<R> q = p[s];
        const double4_32a g = cgeo[c];
        double tx, ty, tz, ox, oy, oz;
        tangent_basis<double>(g.x, g.y, g.z, tx, ty, tz, ox, oy, oz);
        const double pn = q.x, pt = q.y, po = q.z;
        cimp[c] = make_double4_32a(pn, pt, po, 0.0);
        cworld[c] = make_double4_32a(pn * g.x + pt * tx + po * ox, pn * g.y + pt * ty + po * oy,
                                 pn * g.z + pt * tz + po * oz, 0.0);
    }
}

template <class R>
static SolveArgs<R> make_args(nbgs_scene* s, int max_sweeps, double tol)
{
    SolveArgs<R> A;
    A.n = s->n;
    A.C = s->n_contacts;
    A.vel = (R4<R>*)s->vel;
    A.rec = (const SweepRec<R>*)s->srec;
    A.p = (R4<R>*)s->sp;
    A.col_off = s->col_off;
    A.info = s->info;
    A.mu = (R)s->prm.mu;
    A.omega = (R)s->prm.omega;
    for (int k = 0; k < 3; ++k) A.gdt[k] = (R)(s->prm.dt * s->prm.gravity[k]);
    const double* g = s->prm.gravity;
    A.gdt_norm = sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]) * s->prm.dt;
    A.max_sweeps = max_sweeps;
    A.tol = tol;
    A.warm = (s->prm.warm_start == NBGS_WARM_PREV && s->have_prev) ? 1 : 0;
    return A;
}

template <class R>
static nbgs_status solve_impl(nbgs_scene* s, int max_sweeps, double tol)
{
    cudaStream_t st = s->stream;
    SolveArgs<R> A = make_args<R>(s, max_sweeps, tol);
    const int nk = max_sweeps < kHistKept ? max_sweeps : kHistKept + 3;
    cudaMemsetAsync(A.info->rk_bits, 0, (size_t)(nk > 0 ? nk : 1) * sizeof(unsigned long long), st);
    cudaMemsetAsync(&A.info->barrier_count, 0, 2 * sizeof(uint32_t), st);
    const uint32_t not_done = 0xFFFFFFFFu;
    if (s->prm.solver == NBGS_SOLVER_PERSISTENT) {
        void* args[] = {&A};
        cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_solve_persistent<R>, dim3(s->coop_blocks),
                                                    dim3(s->coop_threads), args, 0, st);
        if (s->timing) s->phase_launches[2] += 1;
        return cuda_check(s, e, "solve: cooperative launch");
    }
    // per-colour launches: needs the colour count on the host
    cudaMemcpyAsync(&A.info->sweeps_done, &not_done, sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    uint32_t ncol = 0;
    nbgs_status rc = cuda_check(s, cudaMemcpyAsync(&ncol, &A.info->n_colours, sizeof(uint32_t),
                                                   cudaMemcpyDeviceToHost, st), "solve: colours");
    if (rc == NBGS_OK) rc = cuda_check(s, cudaStreamSynchronize(st), "solve");
    if (rc != NBGS_OK) return rc;
    const int T = 256;
    k_gravity<R><<<grid_for(s->n, T, 8, s->num_sms), T, 0, st>>>(A);
    if (A.warm)
        for (uint32_t c = 0; c < ncol; ++c)
            k_relax_colour<R, true><<<grid_for(A.C, T, 8, s->num_sms), T, 0, st>>>(A, (int)c, 0);
    for (int k = 0; k < max_sweeps; ++k) {
        for (uint32_t c = 0; c < ncol; ++c)
            k_relax_colour<R, false><<<grid_for(A.C, T, 8, s->num_sms), T, 0, st>>>(A, (int)c, k);
        k_sweep_done<R><<<1, 32, 0, st>>>(A, k);
    }
    if (s->timing) s->phase_launches[2] += 1 + (A.warm ? ncol : 0) + (int64_t)max_sweeps * (ncol + 1);
    return cuda_check(s, cudaGetLastError(), "solve");
}

nbgs_status run_solve(nbgs_scene* s, int max_sweeps, double tol)
{
    if (!s->coloured) {
        nbgs_status rc = run_colour(s);
        if (rc != NBGS_OK) return rc;
    }
    if (max_sweeps < 0) return fail(s, NBGS_EINVAL, "solve: max_sweeps < 0");
    cudaStream_t st = s->stream;
    if (s->timing) cudaEventRecord(s->ev[4], st);
    nbgs_status rc = s->fp32 ? solve_impl<float>(s, max_sweeps, tol) : solve_impl<double>(s, max_sweeps, tol);
    if (rc != NBGS_OK) return rc;
    if (s->timing) cudaEventRecord(s->ev[5], st);
    const int64_t C = s->n_contacts;
    if (C > 0) {
        const int T = 256;
        if (s->fp32)
            k_finish<float><<<grid_for(C, T, 8, s->num_sms), T, 0, st>>>(C, s->perm, (const float4*)s->sp, s->cgeo,
                                                                         s->cimp, s->cworld);
        else
            k_finish<double><<<grid_for(C, T, 8, s->num_sms), T, 0, st>>>(C, s->perm, (const double4_32a*)s->sp, s->cgeo,
                                                                          s->cimp, s->cworld);
    }
    s->solved = true;
    s->last_sweeps = max_sweeps;
    return cuda_check(s, cudaGetLastError(), "solve");
}

// ---------------------------------------------------------------------------
// FP64 residuals of eq. (nonpenetration) and eq. (coulomb)
// ---------------------------------------------------------------------------
template <class R>
__global__ void k_final_residuals(int64_t C, int64_t n, const uint32_t* __restrict__ cj1, const uint32_t* __restrict__ cj2,
                                  const double4_32a* __restrict__ cgeo, const double2* __restrict__ clev,
                                  const double4_32a* __restrict__ cimp, const R4<R>* __restrict__ vel, double dt,
                                  double beta, double mu, const DevInfo* info, unsigned long long* out)
{
    double m[4] = {0, 0, 0, 0};
    const double vr = info->v_ref > 0.0 ? info->v_ref : 1e-12;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = cj1[c], b = cj2[c];
        const double4_32a g = cgeo[c];
        const double2 l = clev[c];
        const double4_32a p = cimp[c];
        const R4<R> va = vel[2 * (int64_t)a], wa = vel[2 * (int64_t)a + 1];
        double vb[4] = {0, 0, 0, 0}, wb[4] = {0, 0, 0, 0};
        if (b < n) {
            const R4<R> x = vel[2 * (int64_t)b], y = vel[2 * (int64_t)b + 1];
            vb[0] = x.x; vb[1] = x.y; vb[2] = x.z; vb[3] = x.w;
            wb[0] = y.x; wb[1] = y.y; wb[2] = y.z; wb[3] = y.w;
        }
        const double wn = (double)va.w + vb[3];
        const double wt = wn + (double)wa.w * l.x * l.x + wb[3] * l.y * l.y;
        if (!(wn > 0.0)) continue;
        double tx, ty, tz, ox, oy, oz;
        tangent_basis<double>(g.x, g.y, g.z, tx, ty, tz, ox, oy, oz);
        const double cax = (double)wa.y * g.z - (double)wa.z * g.y, cay = (double)wa.z * g.x - (double)wa.x * g.z,
                     caz = (double)wa.x * g.y - (double)wa.y * g.x;
        const double cbx = wb[1] * g.z - wb[2] * g.y, cby = wb[2] * g.x - wb[0] * g.z, cbz = wb[0] * g.y - wb[1] * g.x;
        const double ux = ((double)va.x - l.x * cax) - (vb[0] + l.y * cbx);
        const double uy = ((double)va.y - l.x * cay) - (vb[1] + l.y * cby);
        const double uz = ((double)va.z - l.x * caz) - (vb[2] + l.y * cbz);
        const double un = g.x * ux + g.y * uy + g.z * uz;
        const double ut = tx * ux + ty * uy + tz * uz, uo = ox * ux + oy * uy + oz * uz;
        const double xs = g.w >= 0.0 ? g.w : beta * g.w;
        const double gn = xs / dt + un;
        const double r_np = (gn < 0.0 ? -gn : 0.0) / vr;
        const double cone = sqrt(p.y * p.y + p.z * p.z) - mu * p.x;
        const double r_cone = (cone > 0.0 ? cone : 0.0) * wt / vr;
        const double r_comp = fabs(fmin(wn * p.x, gn)) / vr;
        const double utl = sqrt(ut * ut + uo * uo);
        const double e1 = utl * p.y + mu * p.x * ut, e2 = utl * p.z + mu * p.x * uo;
        const double r_diss = sqrt(e1 * e1 + e2 * e2) * wt / (vr * vr);
        m[0] = fmax(m[0], r_np);
        m[1] = fmax(m[1], r_cone);
        m[2] = fmax(m[2], r_comp);
        m[3] = fmax(m[3], r_diss);
    }
    for (int k = 0; k < 4; ++k) {
        double x = m[k];
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
        if ((threadIdx.x & 31) == 0) {
            if (!(x <= 1e300)) x = __longlong_as_double(0x7FF0000000000000LL);
            atomicMax(&out[k], (unsigned long long)__double_as_longlong(x));
        }
    }
}

nbgs_status run_final_residuals(nbgs_scene* s, nbgs_residuals* out)
{
    if (!s->solved) return fail(s, NBGS_EINVAL, "final_residuals: no solve yet");
    cudaStream_t st = s->stream;
    const int64_t C = s->n_contacts;
    // reuse the tail of the residual history as the 4 output slots
    unsigned long long* slots = &s->info->rk_bits[kMaxSweepsHist - 4];
    cudaMemsetAsync(slots, 0, 4 * sizeof(unsigned long long), st);
    if (C > 0) {
        const int T = 256;
        if (s->fp32)
            k_final_residuals<float><<<grid_for(C, T, 8, s->num_sms), T, 0, st>>>(
                C, s->n, s->cj1, s->cj2, s->cgeo, s->clev, s->cimp, (const float4*)s->vel, s->prm.dt, s->prm.beta,
                s->prm.mu, s->info, slots);
        else
            k_final_residuals<double><<<grid_for(C, T, 8, s->num_sms), T, 0, st>>>(
                C, s->n, s->cj1, s->cj2, s->cgeo, s->clev, s->cimp, (const double4_32a*)s->vel, s->prm.dt, s->prm.beta,
                s->prm.mu, s->info, slots);
    }
    unsigned long long h[4];
    nbgs_status rc = cuda_check(s, cudaMemcpyAsync(h, slots, sizeof(h), cudaMemcpyDeviceToHost, st), "residuals");
    if (rc == NBGS_OK) rc = cuda_check(s, cudaStreamSynchronize(st), "residuals");
    if (rc != NBGS_OK) return rc;
    double d[4];
    for (int k = 0; k < 4; ++k) {
        long long bits = (long long)h[k];
        memcpy(&d[k], &bits, sizeof(double));
    }
    out->non_penetration = d[0];
    out->cone = d[1];
    out->complementarity = d[2];
    out->dissipation = d[3];
    return NBGS_OK;
}

}  // namespace nbgs

namespace nbgs {

// Resident blocks of the persistent solve kernel (cooperative launches need
// every block resident).  0 and a switch to per-colour launches when the
// device cannot launch cooperatively.
int persistent_blocks(nbgs_scene* s)
{
    int coop = 0, occ = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device);
    if (s->fp32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve_persistent<float>, s->coop_threads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve_persistent<double>, s->coop_threads, 0);
    cudaGetLastError();
    if (!coop || occ < 1) {
        s->prm.solver = NBGS_SOLVER_PER_COLOUR;
        return 0;
    }
    return occ * s->num_sms;
}

}  // namespace nbgs
