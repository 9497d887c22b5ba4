// integrate.cu -- time integration (Sect. 3, eq. integrationscheme) and the
// conversions between the caller's double arrays and the body layout.
#include <cstring>

#include "nbgs_internal.cuh"

namespace nbgs {

// x' = x + dt v';  phi' = phi + dt Q(phi) w' with the 4x3 block of Sect. 2,
// renormalised (Sect. 3); periodic axes wrapped into [lo, hi).
template <class R>
__global__ void k_integrate(int64_t n, double4_32a* __restrict__ pos_r, double4_32a* __restrict__ quat,
                            const R4<R>* __restrict__ vel, double dt, double3 lo, double3 L, int3 periodic,
                            DevInfo* info)
{
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        R4<R> v, w;
        ld_body(vel + 2 * i, v, w);
        double4_32a x = ld_d4(pos_r + i);
        x.x += dt * (double)v.x;
        x.y += dt * (double)v.y;
        x.z += dt * (double)v.z;
        double4_32a q = ld_d4(quat + i);
        {
            // quaternion update in the sweep precision (FP64 is scarce on this
            // GPU; orientations of spheres never feed back into the dynamics)
            using Q = R;
            Q qw = (Q)q.x, qx = (Q)q.y, qy = (Q)q.z, qz = (Q)q.w;
            const Q wx = w.x, wy = w.y, wz = w.z, hdt = (Q)(0.5 * dt);
            const Q dw = -qx * wx - qy * wy - qz * wz;
            const Q dx = qw * wx + qz * wy - qy * wz;
            const Q dy = -qz * wx + qw * wy + qx * wz;
            const Q dz = qy * wx - qx * wy + qw * wz;
            qw += hdt * dw;
            qx += hdt * dx;
            qy += hdt * dy;
            qz += hdt * dz;
            const Q inv = Q(1) / sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
            q = make_double4_32a(qw * inv, qx * inv, qy * inv, qz * inv);
        }
        // periodic wrap into [lo, hi); only bodies that left the box pay for fmod
        if (periodic.x && !(x.x >= lo.x && x.x < lo.x + L.x)) {
            double s = fmod(x.x - lo.x, L.x);
            if (s < 0.0) s += L.x;
            x.x = lo.x + s;
        }
        if (periodic.y && !(x.y >= lo.y && x.y < lo.y + L.y)) {
            double s = fmod(x.y - lo.y, L.y);
            if (s < 0.0) s += L.y;
            x.y = lo.y + s;
        }
        if (periodic.z && !(x.z >= lo.z && x.z < lo.z + L.z)) {
            double s = fmod(x.z - lo.z, L.z);
            if (s < 0.0) s += L.z;
            x.z = lo.z + s;
        }
        if (!(fabs(x.x) + fabs(x.y) + fabs(x.z) <= 1e300)) bad = true;
        st_d4(pos_r + i, x);
        st_d4(quat + i, q);
    }
    if (bad) atomicOr(&info->err, kErrNaN);
}

nbgs_status run_integrate(nbgs_scene* s)
{
    if (s->composite) return run_integrate_comp(s);
    if (s->n == 0) return NBGS_OK;
    cudaStream_t st = s->stream;
    if (s->timing) cudaEventRecord(s->ev[6], st);
    const double3 lo = make_double3(s->prm.box_lo[0], s->prm.box_lo[1], s->prm.box_lo[2]);
    const double3 L = make_double3(s->prm.box_hi[0] - s->prm.box_lo[0], s->prm.box_hi[1] - s->prm.box_lo[1],
                                   s->prm.box_hi[2] - s->prm.box_lo[2]);
    const int3 per = make_int3(s->prm.periodic[0], s->prm.periodic[1], s->prm.periodic[2]);
    const int T = 256, gb = grid_for(s->n, T, 8, s->num_sms);
    if (s->fp32)
        k_integrate<float><<<gb, T, 0, st>>>(s->n, s->pos_r, s->quat, (const float4*)s->vel, s->prm.dt, lo, L, per,
                                             s->info);
    else
        k_integrate<double><<<gb, T, 0, st>>>(s->n, s->pos_r, s->quat, (const double4_32a*)s->vel, s->prm.dt, lo, L, per,
                                              s->info);
    if (s->timing) {
        s->phase_launches[3] += 1;
        cudaEventRecord(s->ev[7], st);
    }
    s->detected = s->coloured = false;
    return cuda_check(s, cudaGetLastError(), "integrate");
}

// ---------------------------------------------------------------------------
// state transfer: staging holds pos (3n) | quat (4n) | vel (3n) | angvel (3n)
// ---------------------------------------------------------------------------
template <class R>
__global__ void k_unpack_state(int64_t n, const double* __restrict__ stg, int has_pos, int has_quat, int has_vel,
                               int has_ang, double4_32a* __restrict__ pos_r, double4_32a* __restrict__ quat,
                               R4<R>* __restrict__ vel)
{
    const double* P = stg;
    const double* Q = stg + 3 * n;
    const double* V = stg + 7 * n;
    const double* W = stg + 10 * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (has_pos) {
            double4_32a x = pos_r[i];
            x.x = P[3 * i];
            x.y = P[3 * i + 1];
            x.z = P[3 * i + 2];
            pos_r[i] = x;
        }
        if (has_quat) quat[i] = make_double4_32a(Q[4 * i], Q[4 * i + 1], Q[4 * i + 2], Q[4 * i + 3]);
        if (has_vel) {
            R4<R> v = vel[2 * i];
            v.x = (R)V[3 * i];
            v.y = (R)V[3 * i + 1];
            v.z = (R)V[3 * i + 2];
            vel[2 * i] = v;
        }
        if (has_ang) {
            R4<R> w = vel[2 * i + 1];
            w.x = (R)W[3 * i];
            w.y = (R)W[3 * i + 1];
            w.z = (R)W[3 * i + 2];
            vel[2 * i + 1] = w;
        }
    }
}

template <class R>
__global__ void k_pack_state(int64_t n, double* __restrict__ stg, const double4_32a* __restrict__ pos_r,
                             const double4_32a* __restrict__ quat, const R4<R>* __restrict__ vel)
{
    double* P = stg;
    double* Q = stg + 3 * n;
    double* V = stg + 7 * n;
    double* W = stg + 10 * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double4_32a x = pos_r[i];
        P[3 * i] = x.x;
        P[3 * i + 1] = x.y;
        P[3 * i + 2] = x.z;
        const double4_32a q = quat[i];
        Q[4 * i] = q.x;
        Q[4 * i + 1] = q.y;
        Q[4 * i + 2] = q.z;
        Q[4 * i + 3] = q.w;
        const R4<R> v = vel[2 * i], w = vel[2 * i + 1];
        V[3 * i] = v.x;
        V[3 * i + 1] = v.y;
        V[3 * i + 2] = v.z;
        W[3 * i] = w.x;
        W[3 * i + 1] = w.y;
        W[3 * i + 2] = w.z;
    }
}

// Sect. 2: m = rho 4/3 pi r^3, I = 2/5 m r^2 (init), or explicit 1/m, 1/I.
template <class R>
__global__ void k_set_mass(int64_t n, const double* __restrict__ a, const double* __restrict__ b, int mode,
                           int has_a, int has_b, double4_32a* __restrict__ pos_r, R4<R>* __restrict__ vel,
                           uint8_t* __restrict__ finite, double* __restrict__ rmax_out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        R4<R> v = vel[2 * i], w = vel[2 * i + 1];
        double im = v.w, iI = w.w;
        if (mode == 0) {  // a = radius, b = density
            const double r = a[i], rho = b[i];
            const double mass = rho * (4.0 / 3.0) * 3.14159265358979323846 * r * r * r;
            const double inertia = 0.4 * mass * r * r;
            im = mass > 0.0 ? 1.0 / mass : 0.0;
            iI = inertia > 0.0 ? 1.0 / inertia : 0.0;
            double4_32a x = pos_r[i];
            x.w = r;
            pos_r[i] = x;
        } else {
            if (has_a) im = a[i];
            if (has_b) iI = b[i];
        }
        v.w = (R)im;
        w.w = (R)iI;
        vel[2 * i] = v;
        vel[2 * i + 1] = w;
        finite[i] = (im > 0.0 || iI > 0.0) ? 1 : 0;
    }
}

template <class R>
static nbgs_status set_bodies_impl(nbgs_scene* s, const double* pos, const double* quat, const double* vel,
                                   const double* angvel)
{
    const int64_t n = s->n;
    cudaStream_t st = s->stream;
    nbgs_status rc = NBGS_OK;
    if (pos) rc = cuda_check(s, cudaMemcpyAsync(s->stage, pos, 3 * n * sizeof(double), cudaMemcpyDefault, st), "set pos");
    if (rc == NBGS_OK && quat)
        rc = cuda_check(s, cudaMemcpyAsync(s->stage + 3 * n, quat, 4 * n * sizeof(double), cudaMemcpyDefault, st),
                        "set quat");
    if (rc == NBGS_OK && vel)
        rc = cuda_check(s, cudaMemcpyAsync(s->stage + 7 * n, vel, 3 * n * sizeof(double), cudaMemcpyDefault, st),
                        "set vel");
    if (rc == NBGS_OK && angvel)
        rc = cuda_check(s, cudaMemcpyAsync(s->stage + 10 * n, angvel, 3 * n * sizeof(double), cudaMemcpyDefault, st),
                        "set angvel");
    if (rc != NBGS_OK) return rc;
    const int T = 256;
    k_unpack_state<R><<<grid_for(n, T, 8, s->num_sms), T, 0, st>>>(n, s->stage, pos != nullptr, quat != nullptr,
                                                                   vel != nullptr, angvel != nullptr, s->pos_r,
                                                                   s->quat, (R4<R>*)s->vel);
    s->detected = s->coloured = false;
    return cuda_check(s, cudaGetLastError(), "set_bodies");
}

nbgs_status run_set_bodies(nbgs_scene* s, const double* pos, const double* quat, const double* vel,
                           const double* angvel)
{
    if (s->composite) return run_comp_set_bodies(s, pos, quat, vel, angvel);
    if (s->n == 0) return NBGS_OK;
    return s->fp32 ? set_bodies_impl<float>(s, pos, quat, vel, angvel) : set_bodies_impl<double>(s, pos, quat, vel, angvel);
}

nbgs_status run_get_bodies(nbgs_scene* s, double* pos, double* quat, double* vel, double* angvel)
{
    if (s->composite) return run_comp_get_bodies(s, pos, quat, vel, angvel);
    const int64_t n = s->n;
    if (n == 0) return NBGS_OK;
    cudaStream_t st = s->stream;
    const int T = 256;
    if (s->fp32)
        k_pack_state<float><<<grid_for(n, T, 8, s->num_sms), T, 0, st>>>(n, s->stage, s->pos_r, s->quat,
                                                                         (const float4*)s->vel);
    else
        k_pack_state<double><<<grid_for(n, T, 8, s->num_sms), T, 0, st>>>(n, s->stage, s->pos_r, s->quat,
                                                                          (const double4_32a*)s->vel);
    nbgs_status rc = cuda_check(s, cudaGetLastError(), "get_bodies");
    if (rc == NBGS_OK && pos)
        rc = cuda_check(s, cudaMemcpyAsync(pos, s->stage, 3 * n * sizeof(double), cudaMemcpyDefault, st), "get pos");
    if (rc == NBGS_OK && quat)
        rc = cuda_check(s, cudaMemcpyAsync(quat, s->stage + 3 * n, 4 * n * sizeof(double), cudaMemcpyDefault, st),
                        "get quat");
    if (rc == NBGS_OK && vel)
        rc = cuda_check(s, cudaMemcpyAsync(vel, s->stage + 7 * n, 3 * n * sizeof(double), cudaMemcpyDefault, st),
                        "get vel");
    if (rc == NBGS_OK && angvel)
        rc = cuda_check(s, cudaMemcpyAsync(angvel, s->stage + 10 * n, 3 * n * sizeof(double), cudaMemcpyDefault, st),
                        "get angvel");
    if (rc == NBGS_OK) rc = cuda_check(s, cudaStreamSynchronize(st), "get_bodies");
    return rc;
}

nbgs_status run_set_mass(nbgs_scene* s, const double* a, const double* b, bool init, const double* radius,
                         const double* density)
{
    const int64_t n = s->n;
    if (n == 0) return NBGS_OK;
    cudaStream_t st = s->stream;
    double* A = s->stage;
    double* B = s->stage + n;
    const double* srcA = init ? radius : a;
    const double* srcB = init ? density : b;
    nbgs_status rc = NBGS_OK;
    if (srcA) rc = cuda_check(s, cudaMemcpyAsync(A, srcA, n * sizeof(double), cudaMemcpyDefault, st), "mass a");
    if (rc == NBGS_OK && srcB)
        rc = cuda_check(s, cudaMemcpyAsync(B, srcB, n * sizeof(double), cudaMemcpyDefault, st), "mass b");
    if (rc != NBGS_OK) return rc;
    const int T = 256;
    if (s->fp32)
        k_set_mass<float><<<grid_for(n, T, 8, s->num_sms), T, 0, st>>>(n, A, B, init ? 0 : 1, srcA != nullptr,
                                                                       srcB != nullptr, s->pos_r, (float4*)s->vel,
                                                                       s->finite, nullptr);
    else
        k_set_mass<double><<<grid_for(n, T, 8, s->num_sms), T, 0, st>>>(n, A, B, init ? 0 : 1, srcA != nullptr,
                                                                        srcB != nullptr, s->pos_r, (double4_32a*)s->vel,
                                                                        s->finite, nullptr);
    s->detected = s->coloured = false;
    return cuda_check(s, cudaGetLastError(), "set_mass_properties");
}

// ---------------------------------------------------------------------------
// contacts out: staging of 10 doubles per contact
// ---------------------------------------------------------------------------
__global__ void k_pack_contacts(int64_t m, const uint32_t* __restrict__ cstate, const double4_32a* __restrict__ cgeo,
                                const double4_32a* __restrict__ cimp, int solved, int32_t* __restrict__ col,
                                double* __restrict__ nrm, double* __restrict__ xi, double* __restrict__ imp)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < m; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t sc = cstate[c];
        col[c] = sc == kUncoloured ? -1 : (int32_t)(sc & 0xFFu);
        const double4_32a g = cgeo[c];
        nrm[3 * c] = g.x;
        nrm[3 * c + 1] = g.y;
        nrm[3 * c + 2] = g.z;
        xi[c] = g.w;
        const double4_32a p = solved ? cimp[c] : make_double4_32a(0, 0, 0, 0);
        imp[3 * c] = p.x;
        imp[3 * c + 1] = p.y;
        imp[3 * c + 2] = p.z;
    }
}

nbgs_status run_get_contacts(nbgs_scene* s, int64_t cap, uint32_t* j1, uint32_t* j2, int32_t* colour, double* normal,
                             double* xi, double* impulse)
{
    const int64_t m = s->n_contacts < cap ? s->n_contacts : cap;
    if (m <= 0) return NBGS_OK;
    cudaStream_t st = s->stream;
    // 8 doubles per contact: colour (as int32 in a double slot), normal 3, xi, impulse 3
    double* buf = (double*)dev_alloc(s, (size_t)m * 8 * sizeof(double));
    if (!buf) return fail(s, NBGS_ENOMEM, "get_contacts: staging allocation failed");
    int32_t* col = (int32_t*)buf;
    double* nrm = buf + m;
    double* xiv = buf + 4 * m;
    double* imp = buf + 5 * m;
    if (!s->coloured && !s->solved) cudaMemsetAsync(s->cstate, 0xFF, m * sizeof(uint32_t), st);
    const int T = 256;
    k_pack_contacts<<<grid_for(m, T, 8, s->num_sms), T, 0, st>>>(m, s->cstate, s->cgeo, s->cimp, s->solved ? 1 : 0, col,
                                                                 nrm, xiv, imp);
    nbgs_status rc = cuda_check(s, cudaGetLastError(), "get_contacts");
    if (rc == NBGS_OK && j1) rc = cuda_check(s, cudaMemcpyAsync(j1, s->cj1, m * 4, cudaMemcpyDefault, st), "j1");
    if (rc == NBGS_OK && j2) rc = cuda_check(s, cudaMemcpyAsync(j2, s->cj2, m * 4, cudaMemcpyDefault, st), "j2");
    if (rc == NBGS_OK && colour) rc = cuda_check(s, cudaMemcpyAsync(colour, col, m * 4, cudaMemcpyDefault, st), "col");
    if (rc == NBGS_OK && normal)
        rc = cuda_check(s, cudaMemcpyAsync(normal, nrm, m * 24, cudaMemcpyDefault, st), "normal");
    if (rc == NBGS_OK && xi) rc = cuda_check(s, cudaMemcpyAsync(xi, xiv, m * 8, cudaMemcpyDefault, st), "xi");
    if (rc == NBGS_OK && impulse)
        rc = cuda_check(s, cudaMemcpyAsync(impulse, imp, m * 24, cudaMemcpyDefault, st), "impulse");
    if (rc == NBGS_OK) rc = cuda_check(s, cudaStreamSynchronize(st), "get_contacts");
    dev_free(s, buf);
    return rc;
}

}  // namespace nbgs
