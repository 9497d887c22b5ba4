// api.cu -- the extern "C" entry points declared in include/nbgs.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "nbgs_internal.cuh"

namespace nbgs {

nbgs_status fail(nbgs_scene* s, nbgs_status st, const std::string& msg)
{
    if (s && s->status == NBGS_OK) {
        s->status = st;
        s->err = msg;
    }
    return st;
}

nbgs_status cuda_check(nbgs_scene* s, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return NBGS_OK;
    return fail(s, NBGS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void* dev_alloc(nbgs_scene* s, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (s->has_alloc) {
        p = s->alloc.alloc(s->alloc.ctx, bytes, (void*)s->stream);
    } else if (cudaMallocAsync(&p, bytes, s->stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dev_free(nbgs_scene* s, void* p)
{
    if (!p) return;
    if (s->has_alloc) s->alloc.free(s->alloc.ctx, p, (void*)s->stream);
    else cudaFreeAsync(p, s->stream);
}

template <class T>
static bool take(nbgs_scene* s, T*& p, size_t count)
{
    p = (T*)dev_alloc(s, count * sizeof(T));
    return p != nullptr;
}

int persistent_blocks(nbgs_scene* s);  // solve.cu

static size_t rec_bytes(const nbgs_scene* s) { return s->fp32 ? 32 : 64; }
static size_t vec4_bytes(const nbgs_scene* s) { return s->fp32 ? 16 : 32; }

static bool alloc_contact_arrays(nbgs_scene* s, int64_t cap)
{
    const size_t c = (size_t)cap;
    bool ok = take(s, s->cj1, c) && take(s, s->cj2, c) && take(s, s->cgeo, c) && take(s, s->clev, c) &&
              take(s, s->cimp, c) && take(s, s->cworld, c) && take(s, s->prev_j2, c) && take(s, s->prev_P, c) &&
              take(s, s->adj, 2 * c) && take(s, s->cstate, c) && take(s, s->cprio, c) && take(s, s->wl[0], 2 * c) &&
              take(s, s->wl[1], 2 * c) && take(s, s->colour_key, c) && take(s, s->colour_key2, c) &&
              take(s, s->cpack, c) &&
              take(s, s->perm, c) && take(s, s->perm_in, c);
    if (!ok) return false;
    s->srec = dev_alloc(s, c * rec_bytes(s));
    s->sp = dev_alloc(s, c * vec4_bytes(s));
    return s->srec && s->sp;
}

static void free_contact_arrays(nbgs_scene* s)
{
    void* ps[] = {s->cj1, s->cj2, s->cgeo, s->clev, s->cimp, s->cworld, s->prev_j2, s->prev_P, s->adj, s->cstate,
                  s->cprio, s->wl[0], s->wl[1], s->colour_key, s->colour_key2, s->perm, s->perm_in, s->srec, s->sp,
                  s->cpack};
    for (void* p : ps) dev_free(s, p);
}

static bool alloc_sort_temps(nbgs_scene* s)
{
    const int64_t big = std::max<int64_t>(std::max<int64_t>(s->n, s->ccap), 1);
    const int64_t nb = (big + 4095) / 4096;
    s->radix_hist_len = 256 * nb;
    const int64_t scan_len =
        std::max<int64_t>(std::max<int64_t>(s->radix_hist_len, s->n + 1), std::max<int64_t>(s->ccap, s->max_cells) + 1);
    s->scan_tmp_len = (scan_len + 4095) / 4096 + 1;
    return take(s, s->radix_hist, (size_t)s->radix_hist_len + 1) && take(s, s->scan_tmp, (size_t)s->scan_tmp_len);
}

// Grow every contact-sized buffer to hold `need` contacts; the previous
// step's contacts (warm start) are carried over.
nbgs_status grow_contacts(nbgs_scene* s, int64_t need)
{
    int64_t cap = need + need / 4 + 1024;
    if (cap > 0xFFFFFFF0LL) return fail(s, NBGS_ECAPACITY, "contact count exceeds 32-bit indexing");
    uint32_t* old_j2 = s->prev_j2;
    double4_32a* old_P = s->prev_P;
    s->prev_j2 = nullptr;
    s->prev_P = nullptr;
    free_contact_arrays(s);
    dev_free(s, s->radix_hist);
    dev_free(s, s->scan_tmp);
    s->ccap = cap;
    if (!alloc_contact_arrays(s, cap) || !alloc_sort_temps(s)) {
        dev_free(s, old_j2);
        dev_free(s, old_P);
        return fail(s, NBGS_ENOMEM, "grow_contacts: allocation failed");
    }
    if (s->have_prev && s->prev_count > 0) {
        cudaMemcpyAsync(s->prev_j2, old_j2, s->prev_count * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s->stream);
        cudaMemcpyAsync(s->prev_P, old_P, s->prev_count * sizeof(double4_32a), cudaMemcpyDeviceToDevice, s->stream);
    }
    dev_free(s, old_j2);
    dev_free(s, old_P);
    return cuda_check(s, cudaGetLastError(), "grow_contacts");
}

static void timing_collect(nbgs_scene* s)
{
    if (!s->timing) return;
    for (int k = 0; k < 5; ++k) {
        float ms = 0.f;
        if (cudaEventQuery(s->ev[2 * k + 1]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, s->ev[2 * k], s->ev[2 * k + 1]) == cudaSuccess)
            s->phase_ms[k] += ms;
        cudaGetLastError();
    }
}

// Events of a phase are re-recorded each call: fold the finished pair into
// the running sums before it is overwritten.
static void timing_fold(nbgs_scene* s, int k)
{
    if (!s->timing) return;
    float ms = 0.f;
    cudaEventSynchronize(s->ev[2 * k + 1]);
    if (cudaEventElapsedTime(&ms, s->ev[2 * k], s->ev[2 * k + 1]) == cudaSuccess) s->phase_ms[k] += ms;
    cudaGetLastError();
}

static nbgs_status check_device_errors(nbgs_scene* s)
{
    nbgs_status rc = cuda_check(s, cudaMemcpyAsync(s->hinfo, s->info, offsetof(DevInfo, rk_bits),
                                                   cudaMemcpyDeviceToHost, s->stream), "sync: info");
    if (rc == NBGS_OK) rc = cuda_check(s, cudaStreamSynchronize(s->stream), "sync");
    if (rc != NBGS_OK) return rc;
    const uint32_t e = s->hinfo->err;
    if (e & kErrTimeout) return fail(s, NBGS_ETIMEOUT, "a grid barrier wait timed out");
    if (e & kErrNaN) return fail(s, NBGS_ENAN, "NaN or Inf in the body state");
    if (e & kErrContacts) return fail(s, NBGS_ECAPACITY, "a graph step found more contacts than its buffers hold");
    if (e & kErrColours) return fail(s, NBGS_ECAPACITY, "more than 256 colours needed");
    return NBGS_OK;
}

// After graph steps the host does not know the contact counts: read them
// (and the device's error bits) before anything else uses them.
static nbgs_status refresh_after_graphs(nbgs_scene* s)
{
    if (!s->counts_stale) return NBGS_OK;
    s->counts_stale = false;
    nbgs_status rc = check_device_errors(s);
    if (rc != NBGS_OK) return rc;
    s->n_contacts = s->hinfo->n_contacts;
    s->prev_count = s->hinfo->prev_contacts;
    s->have_prev = s->prm.warm_start != NBGS_WARM_NONE;
    s->solved = true;
    s->detected = s->coloured = false;
    s->n_colours = -1;
    return NBGS_OK;
}

// Subdomain mode and grid (NBGS_SUB_GRID: every count >= 1, ids below 2^31).
bool subdomains_valid(int32_t mode, const int32_t g[3])
{
    if (mode < NBGS_SUB_NONE || mode > NBGS_SUB_JACOBI) return false;
    if (mode != NBGS_SUB_GRID) return true;
    int64_t cells = 1;
    for (int a = 0; a < 3; ++a) {
        if (g[a] < 1) return false;
        cells *= g[a];
        if (cells >= ((int64_t)1 << 31)) return false;
    }
    return true;
}

// The parameters every scene needs, checked where a scene is created and
// where a checkpoint replaces them.
bool params_valid(const nbgs_params* p)
{
    if (!(p->dt > 0.0) || !(p->tau > 0.0) || !(p->omega > 0.0) || !(p->mu >= 0.0)) return false;
    if (p->precision != NBGS_FP64 && p->precision != NBGS_FP32) return false;
    if (p->warm_start < NBGS_WARM_NONE || p->warm_start > NBGS_WARM_MLP) return false;
    for (int a = 0; a < 3; ++a)
        if (!(p->box_hi[a] > p->box_lo[a])) return false;
    return subdomains_valid(p->subdomain_mode, p->subdomains);
}

}  // namespace nbgs

using namespace nbgs;

#define NBGS_GUARD(s)                                         \
    do {                                                      \
        if (!(s)) return NBGS_EINVAL;                         \
        if ((s)->status != NBGS_OK) return (s)->status;       \
        if ((s)->counts_stale) {                              \
            const nbgs_status guard_rc_ = refresh_after_graphs(s); \
            if (guard_rc_ != NBGS_OK) return guard_rc_;       \
        }                                                     \
    } while (0)

extern "C" {

static nbgs_status create_common(const nbgs_params* params, const nbgs_batch_desc* batch, int64_t n,
                                 const double* pos, const double* vel, const double* angvel, const double* radius,
                                 const double* density, const nbgs_allocator* allocator, void* stream,
                                 nbgs_scene** out);

nbgs_status nbgs_create_scene(const nbgs_params* params, int64_t n, const double* pos, const double* vel,
                              const double* angvel, const double* radius, const double* density,
                              const nbgs_allocator* allocator, void* stream, nbgs_scene** out)
{
    return create_common(params, nullptr, n, pos, vel, angvel, radius, density, allocator, stream, out);
}

nbgs_status nbgs_create_batch(const nbgs_params* params, const nbgs_batch_desc* batch, int64_t n_bodies,
                              const double* pos, const double* vel, const double* angvel, const double* radius,
                              const double* density, const nbgs_allocator* allocator, void* stream, nbgs_scene** out)
{
    if (!batch || batch->n_scenes < 1 || !batch->body_offset || !batch->box_lo || !batch->box_hi || !batch->mu)
        return NBGS_EINVAL;
    if (batch->n_scenes > 0x7FFFFFF0LL / 6) return NBGS_EINVAL;
    if (batch->body_offset[0] != 0 || batch->body_offset[batch->n_scenes] != n_bodies) return NBGS_EINVAL;
    for (int64_t k = 0; k < batch->n_scenes; ++k) {
        if (batch->body_offset[k + 1] < batch->body_offset[k] || !(batch->mu[k] >= 0.0)) return NBGS_EINVAL;
        for (int a = 0; a < 3; ++a)
            if (!(batch->box_hi[3 * k + a] > batch->box_lo[3 * k + a])) return NBGS_EINVAL;
    }
    if (!params || params->periodic[0] || params->periodic[1] || params->periodic[2]) return NBGS_EINVAL;
    return create_common(params, batch, n_bodies, pos, vel, angvel, radius, density, allocator, stream, out);
}

nbgs_status nbgs_create_composite_scene(const nbgs_params* params, int64_t n_bodies, const double* pos,
                                        const double* vel, const double* angvel, const double* density,
                                        int64_t n_members, const int32_t* member_body, const double* member_offset,
                                        const double* member_radius, const nbgs_allocator* allocator, void* stream,
                                        nbgs_scene** out)
{
    if (!params || !out || n_bodies < 1 || n_members < n_bodies || n_members > 0x7FFFFFF0LL || !pos || !vel ||
        !angvel || !density || !member_body || !member_offset || !member_radius)
        return NBGS_EINVAL;
    if (params->subdomain_mode != NBGS_SUB_NONE || params->warm_start == NBGS_WARM_MLP) return NBGS_EINVAL;
    const int64_t nb = n_bodies, nm = n_members;
    if (member_body[0] != 0 || member_body[nm - 1] != nb - 1) return NBGS_EINVAL;
    for (int64_t i = 0; i < nb; ++i)
        if (!(density[i] > 0.0)) return NBGS_EINVAL;   // the centre of mass needs a mass
    for (int64_t m = 0; m < nm; ++m) {
        if (!(member_radius[m] > 0.0)) return NBGS_EINVAL;
        if (m > 0 && (member_body[m] < member_body[m - 1] || member_body[m] > member_body[m - 1] + 1))
            return NBGS_EINVAL;
    }
    // mass properties on the host, rounded as the oracle writes them: the
    // members' masses and inertias add up; the body's position is its centre
    // of mass; the bounding radius max |d'| + r enters the hull
    std::vector<double> bpos(4 * nb), I0(9 * nb), I0inv(9 * nb), invm(nb), moff(4 * nm), mzero(3 * nm, 0.0),
        ones(nm, 1.0);
    std::vector<uint32_t> mbody(nm), bfirst(nb);
    std::vector<uint8_t> bfin(nb);
    int64_t m0 = 0;
    for (int64_t i = 0; i < nb; ++i) {
        int64_t m1 = m0;
        while (m1 < nm && member_body[m1] == i) ++m1;
        if (m1 - m0 > kMaxMembers) return NBGS_EINVAL;
        bfirst[i] = (uint32_t)m0;
        double M = 0.0, X[3] = {0.0, 0.0, 0.0};
        for (int64_t m = m0; m < m1; ++m) {
            const double r = member_radius[m];
            const double mm = density[i] * (4.0 / 3.0) * 3.14159265358979323846 * r * r * r;
            M += mm;
            for (int e = 0; e < 3; ++e) X[e] += mm * member_offset[3 * m + e];
        }
        for (int e = 0; e < 3; ++e) X[e] = X[e] / M;
        double* I = &I0[9 * i];
        double rbar = 0.0;
        for (int64_t m = m0; m < m1; ++m) {
            const double r = member_radius[m];
            const double mm = density[i] * (4.0 / 3.0) * 3.14159265358979323846 * r * r * r;
            double d[3];
            for (int e = 0; e < 3; ++e) d[e] = member_offset[3 * m + e] - X[e];
            const double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) I[3 * a + b] += (a == b ? 0.4 * mm * r * r + mm * d2 : 0.0) - mm * d[a] * d[b];
            mbody[m] = (uint32_t)i;
            for (int e = 0; e < 3; ++e) moff[4 * m + e] = d[e];
            moff[4 * m + 3] = r;
            const double reach = std::sqrt(d2) + r;
            if (reach > rbar) rbar = reach;
        }
        for (int e = 0; e < 3; ++e) bpos[4 * i + e] = pos[3 * i + e] + X[e];
        bpos[4 * i + 3] = rbar;
        invm[i] = M > 0.0 ? 1.0 / M : 0.0;
        bfin[i] = M > 0.0 ? 1 : 0;
        // inverse by cofactors (positive definite)
        const double* A = I;
        double* Ai = &I0inv[9 * i];
        const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
        const double det = (A[0] * c00 + A[1] * c01) + A[2] * c02;
        if (M > 0.0 && !(det > 0.0)) return NBGS_EINVAL;
        if (M > 0.0) {
            Ai[0] = c00 / det; Ai[1] = (A[2] * A[7] - A[1] * A[8]) / det; Ai[2] = (A[1] * A[5] - A[2] * A[4]) / det;
            Ai[3] = c01 / det; Ai[4] = (A[0] * A[8] - A[2] * A[6]) / det; Ai[5] = (A[2] * A[3] - A[0] * A[5]) / det;
            Ai[6] = c02 / det; Ai[7] = (A[1] * A[6] - A[0] * A[7]) / det; Ai[8] = (A[0] * A[4] - A[1] * A[3]) / det;
        }
        m0 = m1;
    }
    // the detection machinery sized for the members (as spheres at the origin)
    nbgs_scene* s = nullptr;
    nbgs_status rc = create_common(params, nullptr, nm, mzero.data(), mzero.data(), mzero.data(), member_radius,
                                   ones.data(), allocator, stream, &s);
    if (rc != NBGS_OK) return rc;
    s->composite = true;
    s->nb = nb;
    const size_t v4 = s->fp32 ? 16 : 32;
    bool ok = take(s, s->bpos, (size_t)nb) && take(s, s->bquat, (size_t)nb) && take(s, s->bI0, 9 * (size_t)nb) &&
              take(s, s->bI0inv, 9 * (size_t)nb) && take(s, s->bIinv, 6 * (size_t)nb) && take(s, s->binvm, (size_t)nb) &&
              take(s, s->bfinite, (size_t)nb) && take(s, s->mbody, (size_t)nm) && take(s, s->moff, (size_t)nm) &&
              take(s, s->bfirst, (size_t)nb) && take(s, s->banchor, (size_t)nb);
    if (ok) {
        s->bvel = dev_alloc(s, 4 * (size_t)nb * v4);
        ok = s->bvel != nullptr;
    }
    if (!ok) {
        nbgs_destroy_scene(s);
        return NBGS_ENOMEM;
    }
    std::vector<double> q(4 * nb, 0.0);
    for (int64_t i = 0; i < nb; ++i) q[4 * i] = 1.0;
    // body records: (v, 1/m), (w, 0); the inverse inertia rows are set each step
    std::vector<unsigned char> bv(4 * (size_t)nb * v4, 0);
    for (int64_t i = 0; i < nb; ++i) {
        const double vals[8] = {vel[3 * i], vel[3 * i + 1], vel[3 * i + 2], invm[i],
                                angvel[3 * i], angvel[3 * i + 1], angvel[3 * i + 2], 0.0};
        for (int k = 0; k < 8; ++k) {
            if (s->fp32) {
                const float f = (float)vals[k];
                std::memcpy(&bv[4 * i * v4 + 4 * k], &f, 4);
            } else {
                std::memcpy(&bv[4 * i * v4 + 8 * k], &vals[k], 8);
            }
        }
    }
    cudaStream_t st = s->stream;
    cudaMemcpyAsync(s->bpos, bpos.data(), bpos.size() * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s->bquat, q.data(), q.size() * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s->bI0, I0.data(), I0.size() * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s->bI0inv, I0inv.data(), I0inv.size() * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s->binvm, invm.data(), invm.size() * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s->bfinite, bfin.data(), bfin.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s->mbody, mbody.data(), mbody.size() * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s->bfirst, bfirst.data(), bfirst.size() * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s->moff, moff.data(), moff.size() * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s->bvel, bv.data(), bv.size(), cudaMemcpyHostToDevice, st);
    rc = ensure_composite_buffers(s);
    if (rc == NBGS_OK) rc = cuda_check(s, cudaStreamSynchronize(st), "create_composite_scene");
    if (rc != NBGS_OK) {
        nbgs_destroy_scene(s);
        return rc;
    }
    *out = s;
    return NBGS_OK;
}

static nbgs_status create_common(const nbgs_params* params, const nbgs_batch_desc* batch, int64_t n,
                                 const double* pos, const double* vel, const double* angvel, const double* radius,
                                 const double* density, const nbgs_allocator* allocator, void* stream,
                                 nbgs_scene** out)
{
    if (!params || !out || n < 0 || n > 0x7FFFFFF0LL) return NBGS_EINVAL;
    if (n > 0 && (!pos || !vel || !angvel || !radius || !density)) return NBGS_EINVAL;
    if (!params_valid(params) || (batch && params->subdomain_mode != NBGS_SUB_NONE)) return NBGS_EINVAL;
    *out = nullptr;
    nbgs_scene* s = new (std::nothrow) nbgs_scene();
    if (!s) return NBGS_ENOMEM;
    s->prm = *params;
    s->n = n;
    s->fp32 = params->precision == NBGS_FP32;
    if (batch) {
        s->batch = true;
        s->n_scenes = batch->n_scenes;
        s->prm.solver = NBGS_SOLVER_PERSISTENT;
    }
    s->stream = (cudaStream_t)stream;
    if (allocator && allocator->alloc && allocator->free) {
        s->alloc = *allocator;
        s->has_alloc = true;
    }
    nbgs_status rc = cuda_check(s, cudaGetDevice(&s->device), "cudaGetDevice");
    if (rc == NBGS_OK)
        rc = cuda_check(s, cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device), "SM count");
    if (rc != NBGS_OK) {
        delete s;
        return rc;
    }
    // largest radius: cell size lower bound
    double rmax = 0.0;
    if (n > 0) {
        cudaPointerAttributes at{};
        bool dev_ptr = cudaPointerGetAttributes(&at, radius) == cudaSuccess && at.type == cudaMemoryTypeDevice;
        cudaGetLastError();
        if (dev_ptr) {
            double* h = (double*)malloc(n * sizeof(double));
            if (!h || cudaMemcpy(h, radius, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
                free(h);
                delete s;
                return NBGS_ECUDA;
            }
            for (int64_t i = 0; i < n; ++i) rmax = std::max(rmax, h[i]);
            free(h);
        } else {
            for (int64_t i = 0; i < n; ++i) rmax = std::max(rmax, radius[i]);
        }
    }
    s->r_max = rmax;
    const double cs_min = 2.0 * (rmax + params->tau);
    s->max_cells = 1;
    for (int a = 0; a < 3; ++a) {
        const double L = params->box_hi[a] - params->box_lo[a];
        double d = std::floor(L / cs_min);
        if (d < 1.0) d = 1.0;
        if (d > 2048.0) d = 2048.0;
        s->dims_max[a] = (int)d;
        s->max_cells *= (int64_t)d;
    }
    if (s->max_cells > (int64_t)1 << 31) {
        delete s;
        return NBGS_EINVAL;
    }
    s->key_bits = 1;
    while (((int64_t)1 << s->key_bits) < s->max_cells) ++s->key_bits;
    const int cpb = params->contacts_per_body > 0 ? params->contacts_per_body : 8;
    s->ccap = std::max<int64_t>(1024, (int64_t)cpb * n);
    const size_t nn = (size_t)std::max<int64_t>(n, 1);

    bool ok = take(s, s->pos_r, nn) && take(s, s->quat, nn) && take(s, s->hull, nn) && take(s, s->hvw, nn) &&
              take(s, s->p32, nn) &&
              take(s, s->p32s, nn) && take(s, s->finite, nn) &&
              take(s, s->stage, 13 * nn) && take(s, s->cell_start, (size_t)s->max_cells + 1) &&
              take(s, s->cell_end, (size_t)s->max_cells) && take(s, s->keys[0], nn) && take(s, s->keys[1], nn) &&
              take(s, s->vals[0], nn) && take(s, s->vals[1], nn) && take(s, s->cand, nn * kCandCap) &&
              take(s, s->sph_cnt, nn) && take(s, s->row_cnt, nn) && take(s, s->row_off, nn + 1) &&
              take(s, s->prev_row_off, nn + 1) && take(s, s->deg, nn + 1) && take(s, s->adj_off, nn + 1) &&
              take(s, s->cmask, 8 * (nn + 1)) &&
              take(s, s->col_count, kMaxColours + 1) && take(s, s->col_off, kMaxColours + 1) &&
              take(s, s->info, 1);
    if (ok) {
        s->vel = dev_alloc(s, 2 * nn * vec4_bytes(s));
        ok = s->vel && alloc_contact_arrays(s, s->ccap) && alloc_sort_temps(s);
    }
    if (ok) ok = cudaMallocHost((void**)&s->hinfo, sizeof(DevInfo)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        nbgs_destroy_scene(s);
        return NBGS_ENOMEM;
    }
    cudaMemsetAsync(s->info, 0, sizeof(DevInfo), s->stream);
    cudaMemsetAsync(s->vel, 0, 2 * nn * vec4_bytes(s), s->stream);
    cudaMemsetAsync(s->pos_r, 0, nn * sizeof(double4_32a), s->stream);
    cudaMemsetAsync(s->cstate, 0xFF, s->ccap * sizeof(uint32_t), s->stream);
    cudaMemsetAsync(s->row_off, 0, (nn + 1) * sizeof(uint32_t), s->stream);
    cudaMemsetAsync(s->prev_row_off, 0, (nn + 1) * sizeof(uint32_t), s->stream);
    for (int k = 0; k < 10; ++k) cudaEventCreate(&s->ev[k]);
    s->coop_blocks = persistent_blocks(s);
    s->max_coop_blocks = s->coop_blocks;
    if (s->batch && s->coop_blocks == 0) {
        nbgs_destroy_scene(s);
        return NBGS_EINVAL;   // batches need the cooperative persistent solver
    }
    if (s->batch) {
        cudaStreamSynchronize(s->stream);   // stream-ordered allocations before the blocking copies
        const size_t S = (size_t)s->n_scenes;
        bool okb = take(s, s->scene_of, nn) && take(s, s->scene_off, S + 1) && take(s, s->scene_box, 6 * S) &&
                   take(s, s->scene_box32, 6 * S) &&
                   take(s, s->scene_mu, S) && take(s, s->scene_vmax, S) && take(s, s->scene_vref, S) &&
                   take(s, s->scene_rk, 3 * S) && take(s, s->scene_done, S) && take(s, s->scene_res, S);
        uint32_t* h_of = okb ? (uint32_t*)malloc(nn * sizeof(uint32_t)) : nullptr;
        uint32_t* h_off = okb ? (uint32_t*)malloc((S + 1) * sizeof(uint32_t)) : nullptr;
        double* h_box = okb ? (double*)malloc(6 * S * sizeof(double)) : nullptr;
        float* h_box32 = okb ? (float*)malloc(6 * S * sizeof(float)) : nullptr;
        if (!h_of || !h_off || !h_box || !h_box32) {
            free(h_of);
            free(h_off);
            free(h_box);
            free(h_box32);
            nbgs_destroy_scene(s);
            return NBGS_ENOMEM;
        }
        for (size_t k = 0; k < S; ++k) {
            h_off[k] = (uint32_t)batch->body_offset[k];
            for (int64_t i = batch->body_offset[k]; i < batch->body_offset[k + 1]; ++i) h_of[i] = (uint32_t)k;
            for (int a = 0; a < 3; ++a) {
                h_box[6 * k + a] = batch->box_lo[3 * k + a];
                h_box[6 * k + 3 + a] = batch->box_hi[3 * k + a];
                h_box32[6 * k + a] = (float)(batch->box_lo[3 * k + a] - params->box_lo[a]);
                h_box32[6 * k + 3 + a] = (float)(batch->box_hi[3 * k + a] - params->box_lo[a]);
            }
        }
        h_off[S] = (uint32_t)n;
        rc = cuda_check(s, cudaMemcpy(s->scene_of, h_of, (size_t)n * sizeof(uint32_t), cudaMemcpyHostToDevice),
                        "batch: scene ids");
        if (rc == NBGS_OK)
            rc = cuda_check(s, cudaMemcpy(s->scene_off, h_off, (S + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice),
                            "batch: offsets");
        if (rc == NBGS_OK)
            rc = cuda_check(s, cudaMemcpy(s->scene_box, h_box, 6 * S * sizeof(double), cudaMemcpyHostToDevice),
                            "batch: boxes");
        if (rc == NBGS_OK)
            rc = cuda_check(s, cudaMemcpy(s->scene_box32, h_box32, 6 * S * sizeof(float), cudaMemcpyHostToDevice),
                            "batch: boxes");
        if (rc == NBGS_OK)
            rc = cuda_check(s, cudaMemcpy(s->scene_mu, batch->mu, S * sizeof(double), cudaMemcpyHostToDevice),
                            "batch: mu");
        free(h_of);
        free(h_off);
        free(h_box);
        free(h_box32);
        if (rc != NBGS_OK) {
            nbgs_destroy_scene(s);
            return rc;
        }
    }
    if (s->coop_blocks > 0) {
        // scheduling units: up to one per warp (NBGS_SWEEP_WARP_SYNC)
        const size_t units = (size_t)s->coop_blocks * (size_t)(s->coop_threads / 32);
        if (!take(s, s->dep, (size_t)kMaxColours * units) || !take(s, s->prog, units) ||
            !take(s, s->cstart, (size_t)kMaxColours * (units + 1))) {
            nbgs_destroy_scene(s);
            return NBGS_ENOMEM;
        }
    }
    if (n > 0) {
        // identity quaternions: staged by the unpack kernel
        double* q = (double*)malloc(4 * n * sizeof(double));
        if (!q) {
            nbgs_destroy_scene(s);
            return NBGS_ENOMEM;
        }
        for (int64_t i = 0; i < n; ++i) {
            q[4 * i] = 1.0;
            q[4 * i + 1] = q[4 * i + 2] = q[4 * i + 3] = 0.0;
        }
        rc = run_set_mass(s, nullptr, nullptr, true, radius, density);
        if (rc == NBGS_OK) rc = run_set_bodies(s, pos, q, vel, angvel);
        if (rc == NBGS_OK) rc = cuda_check(s, cudaStreamSynchronize(s->stream), "create_scene");
        free(q);
        if (rc != NBGS_OK) {
            nbgs_destroy_scene(s);
            return rc;
        }
    } else {
        rc = cuda_check(s, cudaStreamSynchronize(s->stream), "create_scene");
        if (rc != NBGS_OK) {
            nbgs_destroy_scene(s);
            return rc;
        }
    }
    *out = s;
    return NBGS_OK;
}

static void drop_graphs(nbgs_scene* s);

void nbgs_destroy_scene(nbgs_scene* s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    drop_graphs(s);
    void* ps[] = {s->pos_r, s->quat, s->vel, s->hull, s->hvw, s->p32, s->p32s, s->finite, s->stage, s->cell_start,
                  s->cell_end, s->keys[0], s->keys[1], s->vals[0], s->vals[1], s->radix_hist, s->scan_tmp,
                  s->cand, s->sph_cnt, s->row_cnt, s->row_off, s->prev_row_off, s->deg, s->adj_off,
                  s->col_count, s->col_off, s->info, s->dep, s->prog, s->cstart, s->scene_of, s->scene_off,
                  s->scene_box, s->scene_box32, s->scene_mu, s->scene_vmax, s->scene_vref, s->scene_rk,
                  s->scene_done, s->scene_res, s->mlp_theta, s->cmask};
    for (void* p : ps) dev_free(s, p);
    free_contact_arrays(s);
    free_subdomain_buffers(s);
    free_composite_buffers(s);
    cudaStreamSynchronize(s->stream);
    if (s->hinfo) cudaFreeHost(s->hinfo);
    for (int k = 0; k < 10; ++k)
        if (s->ev[k]) cudaEventDestroy(s->ev[k]);
    cudaGetLastError();
    delete s;
}

const char* nbgs_last_error(const nbgs_scene* s)
{
    if (!s) return "null scene";
    return s->err.c_str();
}

nbgs_status nbgs_add_plane(nbgs_scene* s, const double n[3], double c)
{
    NBGS_GUARD(s);
    if (!n || s->planes.count >= kMaxPlanes) return fail(s, NBGS_EINVAL, "add_plane: bad normal or too many walls");
    const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(std::fabs(len - 1.0) < 1e-9)) return fail(s, NBGS_EINVAL, "add_plane: normal must be a unit vector");
    const int k = s->planes.count++;
    for (int e = 0; e < 3; ++e) s->planes.n[k][e] = n[e];
    s->planes.c[k] = c;
    s->detected = s->coloured = false;
    return NBGS_OK;
}

nbgs_status nbgs_add_cone(nbgs_scene* s, const double apex[3], const double axis[3], double half_angle,
                          double r_orifice, double r_top)
{
    NBGS_GUARD(s);
    if (s->batch || s->composite) return fail(s, NBGS_EINVAL, "add_cone: batches and composite scenes take no cones");
    if (!apex || !axis || s->planes.ncones >= kMaxCones) return fail(s, NBGS_EINVAL, "add_cone: bad cone or too many");
    if (!(half_angle > 0.0 && half_angle < 1.5707963267948966) || !(r_orifice >= 0.0) || !(r_top > r_orifice))
        return fail(s, NBGS_EINVAL, "add_cone: need 0 < half_angle < pi/2 and 0 <= r_orifice < r_top");
    // the same operations as the oracle's (host code is built without FMA
    // contraction), so that both sides hold the same cone
    const double len = std::sqrt((axis[0] * axis[0] + axis[1] * axis[1]) + axis[2] * axis[2]);
    if (!(len > 0.0)) return fail(s, NBGS_EINVAL, "add_cone: zero axis");
    Cone& C = s->planes.cone[s->planes.ncones++];
    for (int e = 0; e < 3; ++e) {
        C.apex[e] = apex[e];
        C.axis[e] = axis[e] / len;
    }
    C.sa = std::sin(half_angle);
    C.ca = std::cos(half_angle);
    C.s_o = r_orifice / C.sa;
    C.s_t = r_top / C.sa;
    s->detected = s->coloured = false;
    return NBGS_OK;
}

nbgs_status nbgs_set_mass_properties(nbgs_scene* s, const double* invm, const double* invI)
{
    NBGS_GUARD(s);
    if (s->composite) return fail(s, NBGS_EINVAL, "set_mass_properties: composites take theirs from the members");
    return run_set_mass(s, invm, invI, false, nullptr, nullptr);
}

nbgs_status nbgs_set_bodies(nbgs_scene* s, const double* pos, const double* quat, const double* vel,
                            const double* angvel)
{
    NBGS_GUARD(s);
    s->have_prev = false;
    s->solved = false;
    return run_set_bodies(s, pos, quat, vel, angvel);
}

nbgs_status nbgs_update_bodies(nbgs_scene* s, const double* pos, const double* quat, const double* vel,
                               const double* angvel)
{
    NBGS_GUARD(s);
    return run_set_bodies(s, pos, quat, vel, angvel);
}

nbgs_status nbgs_get_bodies(nbgs_scene* s, double* pos, double* quat, double* vel, double* angvel)
{
    NBGS_GUARD(s);
    return run_get_bodies(s, pos, quat, vel, angvel);
}

nbgs_status nbgs_detect_contacts(nbgs_scene* s, int64_t* n_contacts)
{
    NBGS_GUARD(s);
    if (s->timing) timing_fold(s, 0);
    nbgs_status rc = run_detect(s);
    if (rc == NBGS_OK && n_contacts) *n_contacts = s->n_contacts;
    return rc;
}

nbgs_status nbgs_colour_contacts(nbgs_scene* s, int32_t* n_colours)
{
    NBGS_GUARD(s);
    if (s->timing && s->coloured) timing_fold(s, 1);
    nbgs_status rc = run_colour(s);
    if (rc == NBGS_OK && n_colours) {
        uint32_t nc = 0;
        rc = cuda_check(s, cudaMemcpyAsync(&nc, &s->info->n_colours, 4, cudaMemcpyDeviceToHost, s->stream), "colours");
        if (rc == NBGS_OK) rc = check_device_errors(s);
        if (rc == NBGS_OK) *n_colours = (int32_t)nc;
    }
    return rc;
}

nbgs_status nbgs_solve_nbgs(nbgs_scene* s, int32_t max_sweeps, double tol, int32_t* sweeps_done, double* residual)
{
    NBGS_GUARD(s);
    if (!s->detected) return fail(s, NBGS_EINVAL, "solve_nbgs: call detect_contacts first");
    if (max_sweeps < 0) return fail(s, NBGS_EINVAL, "solve_nbgs: max_sweeps < 0");
    nbgs_status rc = run_solve(s, max_sweeps, tol);
    if (rc != NBGS_OK) return rc;
    if (sweeps_done || residual) {
        rc = check_device_errors(s);
        if (rc != NBGS_OK) return rc;
        uint32_t k = s->hinfo->sweeps_done;
        if (max_sweeps == 0) k = 0;
        if (sweeps_done) *sweeps_done = (int32_t)k;
        if (residual) *residual = s->hinfo->residual;
    }
    return NBGS_OK;
}

nbgs_status nbgs_integrate(nbgs_scene* s)
{
    NBGS_GUARD(s);
    return run_integrate(s);
}

nbgs_status nbgs_step(nbgs_scene* s, int32_t max_sweeps, double tol, nbgs_step_stats* st)
{
    NBGS_GUARD(s);
    if (s->timing) {
        timing_fold(s, 1);
        timing_fold(s, 2);
        timing_fold(s, 3);
        timing_fold(s, 4);
    }
    nbgs_status rc = nbgs_detect_contacts(s, nullptr);
    if (rc == NBGS_OK) rc = run_colour(s);
    if (rc == NBGS_OK) rc = run_solve(s, max_sweeps, tol);
    if (rc == NBGS_OK) rc = run_integrate(s);
    if (rc != NBGS_OK) return rc;
    if (st) {
        rc = cuda_check(s, cudaMemcpyAsync(s->hinfo, s->info, offsetof(DevInfo, rk_bits), cudaMemcpyDeviceToHost,
                                           s->stream), "step stats");
        if (rc == NBGS_OK) rc = check_device_errors(s);
        if (rc != NBGS_OK) return rc;
        st->n_contacts = s->n_contacts;
        st->n_colours = (int32_t)s->hinfo->n_colours;
        st->sweeps_done = max_sweeps == 0 ? 0 : (int32_t)s->hinfo->sweeps_done;
        st->residual = s->hinfo->residual;
        st->v_ref = s->hinfo->v_ref;
    }
    return NBGS_OK;
}

nbgs_status nbgs_set_warm_start(nbgs_scene* s, int32_t warm_start)
{
    NBGS_GUARD(s);
    if (warm_start < NBGS_WARM_NONE || warm_start > NBGS_WARM_MLP) return fail(s, NBGS_EINVAL, "set_warm_start: mode");
    if (s->composite && warm_start == NBGS_WARM_MLP)
        return fail(s, NBGS_EINVAL, "set_warm_start: the network takes sphere contacts only");
    s->prm.warm_start = warm_start;
    return NBGS_OK;
}

nbgs_status nbgs_set_subdomains(nbgs_scene* s, int32_t mode, const int32_t grid[3])
{
    NBGS_GUARD(s);
    const int32_t one[3] = {1, 1, 1};
    const int32_t* g = grid ? grid : one;
    if (!subdomains_valid(mode, g) || (mode == NBGS_SUB_GRID && !grid))
        return fail(s, NBGS_EINVAL, "set_subdomains: bad mode or grid");
    if ((s->batch || s->composite) && mode != NBGS_SUB_NONE)
        return fail(s, NBGS_EINVAL, "set_subdomains: batches and composite scenes have none");
    s->prm.subdomain_mode = mode;
    for (int a = 0; a < 3; ++a) s->prm.subdomains[a] = g[a];
    s->coloured = false;   // s_c(j), the colours and the sweep records follow the mode
    return NBGS_OK;
}

nbgs_status nbgs_get_scene_stats(nbgs_scene* s, int32_t* sweeps_done, double* residual)
{
    NBGS_GUARD(s);
    nbgs_status rc = check_device_errors(s);
    if (rc != NBGS_OK) return rc;
    if (!s->batch) {
        if (sweeps_done) *sweeps_done = s->last_sweeps == 0 ? 0 : (int32_t)s->hinfo->sweeps_done;
        if (residual) *residual = s->hinfo->residual;
        return NBGS_OK;
    }
    if (sweeps_done) {
        static_assert(sizeof(int32_t) == sizeof(uint32_t), "sweep counts");
        rc = cuda_check(s, cudaMemcpy(sweeps_done, s->scene_done, s->n_scenes * sizeof(uint32_t), cudaMemcpyDefault),
                        "scene stats");
        if (rc == NBGS_OK && s->last_sweeps == 0)
            for (int64_t k = 0; k < s->n_scenes; ++k) sweeps_done[k] = 0;
    }
    if (rc == NBGS_OK && residual)
        rc = cuda_check(s, cudaMemcpy(residual, s->scene_res, s->n_scenes * sizeof(double), cudaMemcpyDefault),
                        "scene stats");
    return rc;
}

nbgs_status nbgs_batch_step(nbgs_scene* s, int32_t max_sweeps, double tol, int32_t* sweeps_done, double* residual)
{
    NBGS_GUARD(s);
    nbgs_status rc = nbgs_step(s, max_sweeps, tol, nullptr);
    if (rc == NBGS_OK && (sweeps_done || residual)) rc = nbgs_get_scene_stats(s, sweeps_done, residual);
    return rc;
}

// The host-side half of the warm-start swap run_detect performs (the
// device-side arrays a graph step reads and writes follow these pointers).
static void swap_warm_buffers(nbgs_scene* s)
{
    std::swap(s->row_off, s->prev_row_off);
    std::swap(s->cj2, s->prev_j2);
    std::swap(s->cworld, s->prev_P);
}

static void drop_graphs(nbgs_scene* s)
{
    for (int k = 0; k < 2; ++k) {
        if (s->gexec[k]) cudaGraphExecDestroy(s->gexec[k]);
        s->gexec[k] = nullptr;
    }
    s->g_sweeps = -1;
}

// One step (detect, colour, solve, integrate) recorded without any host
// synchronisation.  The recording runs on a private stream (the scene's
// stream may be the legacy default stream, which cannot be captured); the
// graph is later launched on the scene's stream, which orders it.
static nbgs_status capture_step(nbgs_scene* s, int32_t max_sweeps, double tol, cudaGraphExec_t* out)
{
    cudaStream_t cap = nullptr;
    nbgs_status rc = cuda_check(s, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "graph_step: stream");
    if (rc != NBGS_OK) return rc;
    cudaStream_t scene_stream = s->stream;
    s->stream = cap;
    rc = cuda_check(s, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "graph_step: begin capture");
    if (rc == NBGS_OK) {
        rc = run_detect(s);
        if (rc == NBGS_OK) rc = run_colour(s);
        if (rc == NBGS_OK) rc = run_solve(s, max_sweeps, tol);
        if (rc == NBGS_OK) rc = run_integrate(s);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cap, &g);
        if (rc == NBGS_OK) rc = cuda_check(s, e, "graph_step: end capture");
        if (rc == NBGS_OK) rc = cuda_check(s, cudaGraphInstantiate(out, g, 0), "graph_step: instantiate");
        if (g) cudaGraphDestroy(g);
    }
    s->stream = scene_stream;
    cudaStreamDestroy(cap);
    return rc;
}

nbgs_status nbgs_graph_step(nbgs_scene* s, int32_t max_sweeps, double tol, int32_t n_steps)
{
    if (!s) return NBGS_EINVAL;
    if (s->status != NBGS_OK) return s->status;
    if (n_steps < 0 || max_sweeps < 0 || !(tol >= 0.0)) return fail(s, NBGS_EINVAL, "graph_step: bad arguments");
    if (s->composite || s->prm.subdomain_mode != NBGS_SUB_NONE || s->prm.warm_start == NBGS_WARM_MLP ||
        s->prm.solver != NBGS_SOLVER_PERSISTENT || s->coop_blocks == 0)
        return fail(s, NBGS_EINVAL, "graph_step: sphere scenes or batches with the persistent solver, no subdomains, "
                                    "no network warm start");
    if (s->timing) return fail(s, NBGS_EINVAL, "graph_step: disable timing first");
    if (n_steps == 0) return NBGS_OK;
    const bool fresh = s->gexec[0] && max_sweeps == s->g_sweeps && tol == s->g_tol && s->ccap == s->g_ccap;
    if (!fresh) {
        nbgs_status rc = refresh_after_graphs(s);
        if (rc != NBGS_OK) return rc;
        if (!s->solved || s->n == 0)
            return fail(s, NBGS_EINVAL, "graph_step: take one nbgs_step first (it sizes the buffers)");
        drop_graphs(s);
        s->device_sized = true;
        rc = capture_step(s, max_sweeps, tol, &s->gexec[0]);
        if (rc == NBGS_OK) rc = capture_step(s, max_sweeps, tol, &s->gexec[1]);
        s->device_sized = false;
        if (rc != NBGS_OK) {
            drop_graphs(s);
            return rc;
        }
        // each capture swapped the warm-start pointers once: back where they were
        s->g_sweeps = max_sweeps;
        s->g_tol = tol;
        s->g_ccap = s->ccap;
        s->g_next = 0;
        s->last_sweeps = max_sweeps;
    }
    for (int32_t k = 0; k < n_steps; ++k) {
        nbgs_status rc = cuda_check(s, cudaGraphLaunch(s->gexec[s->g_next], s->stream), "graph_step: launch");
        if (rc != NBGS_OK) return rc;
        swap_warm_buffers(s);
        s->g_next ^= 1;
    }
    s->counts_stale = true;
    return NBGS_OK;
}

nbgs_status nbgs_autotune(nbgs_scene* s, int32_t max_sweeps, double tol, int32_t* sweep_flags, int32_t* blocks_per_sm)
{
    NBGS_GUARD(s);
    if (s->composite) return fail(s, NBGS_EINVAL, "autotune: composite scenes have one schedule");
    if (!s->detected) return fail(s, NBGS_EINVAL, "autotune: call detect_contacts first");
    if (s->prm.solver != NBGS_SOLVER_PERSISTENT || s->max_coop_blocks == 0)
        return fail(s, NBGS_EINVAL, "autotune: needs the persistent solver");
    nbgs_status rc = NBGS_OK;
    if (!s->coloured) rc = run_colour(s);
    if (rc != NBGS_OK) return rc;
    cudaStream_t st = s->stream;
    const size_t vb = 2 * (size_t)std::max<int64_t>(s->n, 1) * vec4_bytes(s);
    const size_t pb = (size_t)std::max<int64_t>(s->n_contacts, 1) * vec4_bytes(s);
    void* vsave = dev_alloc(s, vb);
    void* psave = dev_alloc(s, pb);
    if (!vsave || !psave) {
        dev_free(s, vsave);
        dev_free(s, psave);
        return fail(s, NBGS_ENOMEM, "autotune: save buffers");
    }
    cudaMemcpyAsync(vsave, s->vel, vb, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(psave, s->sp, pb, cudaMemcpyDeviceToDevice, st);
    const bool had_timing = s->timing;
    s->timing = false;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int max_bps = std::max(1, s->max_coop_blocks / std::max(1, s->num_sms));
    const int flags_list[6] = {0, NBGS_SWEEP_GLOBAL_SYNC, NBGS_SWEEP_TMA_STAGE,
                               NBGS_SWEEP_GLOBAL_SYNC | NBGS_SWEEP_TMA_STAGE, NBGS_SWEEP_WARP_SYNC,
                               NBGS_SWEEP_GATHER2};
    float best = 3.4e38f;
    int best_flags = s->prm.sweep_flags, best_bps = max_bps;
    for (int fi = 0; fi < 6 && rc == NBGS_OK; ++fi) {
        for (int bps = 1; bps <= max_bps && rc == NBGS_OK; ++bps) {
            s->prm.sweep_flags = flags_list[fi];
            s->coop_blocks = bps * s->num_sms;
            float t_min = 3.4e38f;
            for (int rep = 0; rep < 2 && rc == NBGS_OK; ++rep) {
                cudaMemcpyAsync(s->vel, vsave, vb, cudaMemcpyDeviceToDevice, st);
                cudaMemcpyAsync(s->sp, psave, pb, cudaMemcpyDeviceToDevice, st);
                s->coloured = true;
                cudaEventRecord(e0, st);
                rc = run_solve(s, max_sweeps, tol);
                cudaEventRecord(e1, st);
                if (rc == NBGS_OK) rc = check_device_errors(s);
                float ms = 0.f;
                if (rc == NBGS_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) t_min = std::min(t_min, ms);
            }
            if (t_min < best) {
                best = t_min;
                best_flags = flags_list[fi];
                best_bps = bps;
            }
        }
    }
    s->prm.sweep_flags = best_flags;
    s->coop_blocks = best_bps * s->num_sms;
    cudaMemcpyAsync(s->vel, vsave, vb, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(s->sp, psave, pb, cudaMemcpyDeviceToDevice, st);
    cudaStreamSynchronize(st);
    dev_free(s, vsave);
    dev_free(s, psave);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->timing = had_timing;
    s->coloured = true;
    s->solved = false;
    if (rc != NBGS_OK) return rc;
    if (sweep_flags) *sweep_flags = best_flags;
    if (blocks_per_sm) *blocks_per_sm = best_bps;
    return NBGS_OK;
}

nbgs_status nbgs_get_contacts(nbgs_scene* s, int64_t cap, uint32_t* j1, uint32_t* j2, int32_t* colour,
                              double* normal, double* xi, double* impulse, int64_t* n_out)
{
    NBGS_GUARD(s);
    if (cap < 0) return fail(s, NBGS_EINVAL, "get_contacts: cap < 0");
    if (n_out) *n_out = s->n_contacts;
    nbgs_status rc = run_get_contacts(s, cap, j1, j2, colour, normal, xi, impulse);
    if (rc == NBGS_OK) rc = check_device_errors(s);
    return rc;
}

nbgs_status nbgs_residual_history(nbgs_scene* s, double* out, int32_t cap, int32_t* n_out)
{
    NBGS_GUARD(s);
    nbgs_status rc = check_device_errors(s);
    if (rc != NBGS_OK) return rc;
    int32_t k = s->solved ? (int32_t)s->hinfo->sweeps_done : 0;
    if (s->solved && s->last_sweeps == 0) k = 0;
    if (k > kHistKept) k = kHistKept;
    if (n_out) *n_out = k;
    const int32_t m = std::min(k, cap);
    if (m > 0 && out) {
        unsigned long long* tmp = (unsigned long long*)malloc(m * sizeof(unsigned long long));
        if (!tmp) return fail(s, NBGS_ENOMEM, "residual_history: host allocation");
        rc = cuda_check(s, cudaMemcpy(tmp, s->info->rk_bits, m * sizeof(unsigned long long), cudaMemcpyDeviceToHost),
                        "residual_history");
        const double vr = s->hinfo->v_ref > 0 ? s->hinfo->v_ref : 1e-12;
        for (int32_t i = 0; i < m && rc == NBGS_OK; ++i) {
            double d;
            std::memcpy(&d, &tmp[i], sizeof(double));
            out[i] = d / vr;
        }
        free(tmp);
    }
    return rc;
}

nbgs_status nbgs_set_impulses(nbgs_scene* s, const double* impulse)
{
    NBGS_GUARD(s);
    if (!impulse) return fail(s, NBGS_EINVAL, "set_impulses: null impulses");
    if (s->composite) return fail(s, NBGS_EINVAL, "set_impulses: sphere scenes only");
    if (!s->solved) return fail(s, NBGS_EINVAL, "set_impulses: solve the current contacts first");
    nbgs_status rc = run_set_impulses(s, impulse);
    if (rc == NBGS_OK) rc = check_device_errors(s);
    return rc;
}

nbgs_status nbgs_final_residuals(nbgs_scene* s, nbgs_residuals* out)
{
    NBGS_GUARD(s);
    if (!out) return fail(s, NBGS_EINVAL, "final_residuals: null output");
    if (s->composite) return fail(s, NBGS_EINVAL, "final_residuals: sphere scenes only");
    nbgs_status rc = run_final_residuals(s, out);
    if (rc == NBGS_OK) rc = check_device_errors(s);
    return rc;
}

nbgs_status nbgs_get_updates(nbgs_scene* s, int64_t* updates)
{
    NBGS_GUARD(s);
    if (!updates) return fail(s, NBGS_EINVAL, "get_updates: null output");
    unsigned long long u = 0;
    nbgs_status rc = cuda_check(s, cudaMemcpyAsync(&u, &s->info->updates, sizeof(u), cudaMemcpyDeviceToHost, s->stream),
                                "get_updates");
    if (rc == NBGS_OK) rc = cuda_check(s, cudaMemsetAsync(&s->info->updates, 0, sizeof(u), s->stream), "get_updates");
    if (rc == NBGS_OK) rc = check_device_errors(s);
    if (rc == NBGS_OK) *updates = (int64_t)u;
    return rc;
}

nbgs_status nbgs_sync(nbgs_scene* s)
{
    NBGS_GUARD(s);
    return check_device_errors(s);
}

nbgs_status nbgs_enable_timing(nbgs_scene* s, int32_t on)
{
    NBGS_GUARD(s);
    nbgs_status rc = cuda_check(s, cudaStreamSynchronize(s->stream), "enable_timing");
    s->timing = on != 0;
    for (int k = 0; k < 5; ++k) s->phase_ms[k] = 0.0;
    for (int k = 0; k < 4; ++k) s->phase_launches[k] = 0;
    s->sweep_launches = 0;
    // mark every event pair as empty: record start and end back to back
    for (int k = 0; k < 10; ++k) cudaEventRecord(s->ev[k], s->stream);
    cudaStreamSynchronize(s->stream);
    return rc;
}

nbgs_status nbgs_get_timings(nbgs_scene* s, double ms[5], int64_t launches[5])
{
    NBGS_GUARD(s);
    nbgs_status rc = cuda_check(s, cudaStreamSynchronize(s->stream), "get_timings");
    if (rc != NBGS_OK) return rc;
    timing_collect(s);
    for (int k = 0; k < 5; ++k) {
        if (ms) ms[k] = s->phase_ms[k];
        if (launches) launches[k] = k < 4 ? s->phase_launches[k] : s->sweep_launches;
        s->phase_ms[k] = 0.0;
    }
    // collected pairs must not be folded again
    for (int k = 0; k < 10; ++k) cudaEventRecord(s->ev[k], s->stream);
    cudaStreamSynchronize(s->stream);
    return NBGS_OK;
}

}  // extern "C"
