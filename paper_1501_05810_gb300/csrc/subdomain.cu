// subdomain.cu -- the subdomain NBGS of Alg. 1 and its non-linear block
// Jacobi limit on one GPU: the subdomain of each contact and the velocity
// instances the sweep reads and writes.
//
// Alg. 1 relaxes contact j with the reactions of the current sweep for the
// earlier contacts of its own subdomain s_c(j) and with those of the
// previous sweep for every other contact.  Sect. 6.3 realises this with
// accumulated velocities (all reactions of the previous sweep) plus one set
// of velocity corrections per subdomain.  Here every pair (finite body i,
// subdomain p) that a contact of p touches gets a velocity record of its own
// (an instance) holding v_i + delta v_i^[p] in the sweep's body layout: the
// body's own record serves its lowest subdomain, the others take extra
// records after the n bodies.  The sweep records name instances instead of
// bodies, so the sweep kernels run unchanged -- contacts of one colour share
// no body, hence no instance.  After each sweep the solver adds up the
// instances of every body that has extras (solve.cu, inst_reduce_pass):
// v <- v_acc + sum_p (instance_p - v_acc) in increasing p, and every
// instance restarts from v -- the two message exchanges of Sect. 6.3.
//
// Subdomain rule.  Sect. 6.2 lets any rule that partitions the contact set
// decide which process treats a contact and favours the particles' parent
// processes; a contact belongs to the cell of a regular g0 x g1 x g2 grid over
// the box that holds the centre of its body j1: k_a = floor((x_a - lo_a) g_a
// / L_a), clamped to [0, g_a - 1], id = (k_2 g_1 + k_1) g_0 + k_0, in FP64
// with every operation rounded as written.  Non-linear block Jacobi:
// s_c(j) = j.
#include "nbgs_internal.cuh"

namespace nbgs {

namespace {

struct SubGrid {
    int mode;
    int g[3];
    double lo[3], L[3];
};

// Grid cell of every body centre (the subdomain of the contacts it is j1 of).
__global__ void k_body_sub(int64_t n, const double4_32a* __restrict__ pos_r, SubGrid G, uint32_t* __restrict__ bsub)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double4_32a x = pos_r[i];
        uint32_t id = 0;
        for (int ax = 2; ax >= 0; --ax) {
            const double xa = ax == 0 ? x.x : (ax == 1 ? x.y : x.z);
            double k = floor(xdiv(xmul(xsub(xa, G.lo[ax]), (double)G.g[ax]), G.L[ax]));
            if (!(k >= 0.0)) k = 0.0;
            if (k > (double)(G.g[ax] - 1)) k = (double)(G.g[ax] - 1);
            id = id * (uint32_t)G.g[ax] + (uint32_t)k;
        }
        bsub[i] = id;
    }
}

// Subdomain of every contact; every contact end names its own body until
// k_inst_assign gives the finite ones their instances (walls: 0xFFFFFFFF,
// beyond every velocity record).
__global__ void k_sub_assign(int64_t C, int64_t n, const uint32_t* __restrict__ cj1, const uint32_t* __restrict__ cj2,
                             const uint32_t* __restrict__ bsub, int jacobi, uint32_t* __restrict__ csub,
                             uint32_t* __restrict__ inst)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = cj1[c], b = cj2[c];
        csub[c] = jacobi ? (uint32_t)c : bsub[a];
        inst[2 * c] = a;
        inst[2 * c + 1] = b < (uint64_t)n ? b : 0xFFFFFFFFu;
    }
}

// Number of distinct subdomains among the incidence entries [e0, e1) of a
// body that are below p (the rank of subdomain p at that body).
__device__ __forceinline__ uint32_t sub_rank(const uint32_t* __restrict__ adj, const uint32_t* __restrict__ csub,
                                             uint32_t e0, uint32_t e1, uint32_t p)
{
    uint32_t r = 0;
    for (uint32_t e = e0; e < e1; ++e) {
        const uint32_t q = csub[adj[e]];
        if (q >= p) continue;
        bool first = true;   // count each subdomain at its first entry only
        for (uint32_t f = e0; f < e && first; ++f) first = csub[adj[f]] != q;
        r += first ? 1u : 0u;
    }
    return r;
}

// Extra instances per body (distinct subdomains - 1) into ext[i]; bodies
// with extras join the shared list.
__global__ void k_inst_count(int64_t n, const uint32_t* __restrict__ adj_off, const uint32_t* __restrict__ adj,
                             const uint32_t* __restrict__ csub, int jacobi, uint32_t* __restrict__ ext,
                             uint32_t* __restrict__ shared, DevInfo* info)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e0 = adj_off[i], e1 = adj_off[i + 1];
        uint32_t distinct = 0;
        uint32_t lo = 0xFFFFFFFFu, hi = 0;
        if (!jacobi)
            for (uint32_t e = e0; e < e1; ++e) {
                const uint32_t q = csub[adj[e]];
                lo = q < lo ? q : lo;
                hi = q > hi ? q : hi;
            }
        if (jacobi) {
            distinct = e1 - e0;   // one subdomain per contact
        } else if (lo == hi) {
            distinct = e1 > e0 ? 1u : 0u;   // inside one subdomain: the common case
        } else {
            for (uint32_t e = e0; e < e1; ++e) {
                const uint32_t q = csub[adj[e]];
                bool first = true;
                for (uint32_t f = e0; f < e && first; ++f) first = csub[adj[f]] != q;
                distinct += first ? 1u : 0u;
            }
        }
        const uint32_t x = distinct > 1 ? distinct - 1 : 0u;
        ext[i] = x;
        if (x > 0) shared[atomicAdd(&info->n_shared, 1u)] = (uint32_t)i;
    }
}

// The instance of every finite contact end: rank 0 -> the body's own
// record, rank r > 0 -> record n + ext_off[i] + r - 1.
__global__ void k_inst_assign(int64_t n, const uint32_t* __restrict__ adj_off, const uint32_t* __restrict__ adj,
                              const uint32_t* __restrict__ csub, const uint32_t* __restrict__ cj1,
                              const uint32_t* __restrict__ ext_off, int jacobi, uint32_t* __restrict__ inst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e0 = adj_off[i], e1 = adj_off[i + 1];
        if (ext_off[i + 1] == ext_off[i]) continue;   // one instance: the body's own record (already set)
        // grid: the body's distinct subdomains in increasing order (few: the
        // cells around one point), or the quadratic rank beyond kFew of them
        constexpr int kFew = 16;
        uint32_t few[kFew];
        int nfew = 0;
        bool listed = !jacobi;
        for (uint32_t e = e0; e < e1 && listed; ++e) {
            const uint32_t q = csub[adj[e]];
            int pos = 0;
            while (pos < nfew && few[pos] < q) ++pos;
            if (pos < nfew && few[pos] == q) continue;
            if (nfew == kFew) {
                listed = false;
                break;
            }
            for (int t = nfew; t > pos; --t) few[t] = few[t - 1];
            few[pos] = q;
            ++nfew;
        }
        for (uint32_t e = e0; e < e1; ++e) {
            const uint32_t c = adj[e];
            uint32_t r = 0;
            if (jacobi) {   // s_c(j) = j: all distinct, the rank counts the lower contacts
                for (uint32_t f = e0; f < e1; ++f) r += adj[f] < c ? 1u : 0u;
            } else if (listed) {
                const uint32_t q = csub[c];
                while (few[r] != q) ++r;
            } else {
                r = sub_rank(adj, csub, e0, e1, csub[c]);
            }
            const uint32_t slot = r == 0 ? (uint32_t)i : (uint32_t)n + ext_off[i] + r - 1u;
            inst[2 * (int64_t)c + (cj1[c] == (uint32_t)i ? 0 : 1)] = slot;
        }
    }
}

}  // namespace

void free_subdomain_buffers(nbgs_scene* s)
{
    void* ps[] = {s->csub, s->inst, s->ext_off, s->shared, s->vacc, s->rlist, s->rstart, s->rcount, s->dep_r};
    for (void* p : ps) dev_free(s, p);
    s->csub = s->inst = s->ext_off = s->shared = s->rlist = s->rstart = s->rcount = nullptr;
    s->vacc = nullptr;
    s->dep_r = nullptr;
    s->sub_ccap = 0;
}

// Subdomain arrays for the current contact capacity, and room for up to
// 2 ccap extra instances after the bodies in vel (every contact end at most
// one): the body records are carried over.
nbgs_status ensure_subdomain_buffers(nbgs_scene* s)
{
    if (s->prm.subdomain_mode == NBGS_SUB_NONE) return NBGS_OK;
    const size_t v4 = s->fp32 ? 16 : 32;
    const int64_t n = s->n;
    const int64_t need = 2 * s->ccap;
    if ((uint64_t)n + (uint64_t)need > 0xFFFFFFF0ull)
        return fail(s, NBGS_ECAPACITY, "subdomains: velocity instances exceed 32-bit indexing");
    if (s->icap < need) {
        void* nv = dev_alloc(s, 2 * (size_t)(n + need) * v4);
        if (!nv) return fail(s, NBGS_ENOMEM, "subdomains: velocity instances: allocation failed");
        if (n > 0) cudaMemcpyAsync(nv, s->vel, 2 * (size_t)n * v4, cudaMemcpyDeviceToDevice, s->stream);
        dev_free(s, s->vel);
        s->vel = nv;
        s->icap = need;
    }
    if (s->sub_ccap < s->ccap) {
        dev_free(s, s->csub);
        dev_free(s, s->inst);
        s->csub = (uint32_t*)dev_alloc(s, (size_t)s->ccap * sizeof(uint32_t));
        s->inst = (uint32_t*)dev_alloc(s, 2 * (size_t)s->ccap * sizeof(uint32_t));
        if (!s->csub || !s->inst) return fail(s, NBGS_ENOMEM, "subdomains: allocation failed");
        s->sub_ccap = s->ccap;
    }
    if (!s->ext_off) {
        const size_t nn = (size_t)(n > 0 ? n : 1);
        const size_t units = (size_t)std::max(s->max_coop_blocks, 1) * (size_t)(s->coop_threads / 32);
        s->ext_off = (uint32_t*)dev_alloc(s, (nn + 1) * sizeof(uint32_t));
        s->shared = (uint32_t*)dev_alloc(s, nn * sizeof(uint32_t));
        s->vacc = dev_alloc(s, 2 * nn * v4);
        s->rlist = (uint32_t*)dev_alloc(s, nn * sizeof(uint32_t));
        s->rstart = (uint32_t*)dev_alloc(s, (units + 1) * sizeof(uint32_t));
        s->rcount = (uint32_t*)dev_alloc(s, (units + 1) * sizeof(uint32_t));
        s->dep_r = (int2*)dev_alloc(s, units * sizeof(int2));
        if (!s->ext_off || !s->shared || !s->vacc || !s->rlist || !s->rstart || !s->rcount || !s->dep_r)
            return fail(s, NBGS_ENOMEM, "subdomains: allocation failed");
    }
    return cuda_check(s, cudaGetLastError(), "subdomains: buffers");
}

// s_c(j), instance counts and slots, and the shared-body list.  Needs the
// body -> contact incidence lists of the colouring (adj_off, adj); uses deg
// as scratch.
nbgs_status run_subdomains(nbgs_scene* s)
{
    nbgs_status rc = ensure_subdomain_buffers(s);
    if (rc != NBGS_OK) return rc;
    cudaStream_t st = s->stream;
    const int64_t C = s->n_contacts, n = s->n;
    SubGrid G;
    G.mode = s->prm.subdomain_mode;
    for (int a = 0; a < 3; ++a) {
        G.g[a] = s->prm.subdomains[a] > 0 ? s->prm.subdomains[a] : 1;
        G.lo[a] = s->prm.box_lo[a];
        G.L[a] = s->prm.box_hi[a] - s->prm.box_lo[a];
    }
    const int T = 256;
    cudaMemsetAsync(&s->info->n_shared, 0, 2 * sizeof(uint32_t), st);   // n_shared, n_extra
    const int jacobi = G.mode == NBGS_SUB_JACOBI ? 1 : 0;
    if (!jacobi && n > 0)   // body cells in ext_off (free until the scan below)
        k_body_sub<<<grid_for(n, T, 8, s->num_sms), T, 0, st>>>(n, s->pos_r, G, s->ext_off);
    k_sub_assign<<<grid_for(C, T, 8, s->num_sms), T, 0, st>>>(C, n, s->cj1, s->cj2, s->ext_off, jacobi, s->csub,
                                                              s->inst);
    if (n > 0) {
        // per-body counts in deg (free once the incidence lists are filled)
        k_inst_count<<<grid_for(n, T, 8, s->num_sms), T, 0, st>>>(n, s->adj_off, s->adj, s->csub,
                                                                   jacobi, s->deg, s->shared, s->info);
        rc = exclusive_scan_u32(s, s->deg, s->ext_off, n, &s->info->n_extra);
        if (rc != NBGS_OK) return rc;
        k_inst_assign<<<grid_for(n, T, 8, s->num_sms), T, 0, st>>>(n, s->adj_off, s->adj, s->csub, s->cj1,
                                                                    s->ext_off, jacobi, s->inst);
    }
    if (s->timing) s->phase_launches[1] += n > 0 ? (jacobi ? 6 : 7) : 1;
    return cuda_check(s, cudaGetLastError(), "subdomains");
}

nbgs_status run_get_subdomains(nbgs_scene* s, int64_t cap, uint32_t* out)
{
    const int64_t m = std::min<int64_t>(cap, s->n_contacts);
    if (!out || m <= 0) return NBGS_OK;
    if (!s->csub || s->sub_count != s->n_contacts) {   // no subdomains in the last colouring
        for (int64_t c = 0; c < m; ++c) out[c] = 0;
        return NBGS_OK;
    }
    nbgs_status rc = cuda_check(s, cudaMemcpyAsync(out, s->csub, (size_t)m * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                                   s->stream), "get_subdomains");
    if (rc == NBGS_OK) rc = cuda_check(s, cudaStreamSynchronize(s->stream), "get_subdomains");
    return rc;
}

}  // namespace nbgs

extern "C" nbgs_status nbgs_get_subdomains(nbgs_scene* s, int64_t cap, uint32_t* out, int64_t* n_out)
{
    if (!s) return NBGS_EINVAL;
    if (s->status != NBGS_OK) return s->status;
    if (cap < 0 || (cap > 0 && !out)) return nbgs::fail(s, NBGS_EINVAL, "get_subdomains: bad arguments");
    if (n_out) *n_out = s->n_contacts;
    return nbgs::run_get_subdomains(s, cap, out);
}
