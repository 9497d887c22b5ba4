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
#include <algorithm>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "mlp_tc.cuh"

namespace nbgs {

template <class R> struct SolveArgs {
    int64_t n;
    int64_t nslot;       // velocity records: n, or n + extra instances with subdomains (walls beyond)
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
    int flags;           // NBGS_SWEEP_* bits
    int* prog;           // per block: last sweep phase completed (local synchronisation)
    const int2* dep;     // per (colour, block): window [lo, hi] of blocks sharing bodies with the chunk
    const uint32_t* cstart;  // per colour, B + 1 chunk boundaries (sweep slots)
    SceneView V;             // batched scenes (V.batch == 0: one scene)
    int64_t nscene;
    unsigned long long* scene_rk;   // 3 x S rotating slots of max r_j / v_ref_s
    uint32_t* scene_done;
    double* scene_res;
    int sub;                   // subdomains: instances reduced after every sweep
    const uint32_t* shared;    // bodies with extra instances (info->n_shared)
    const uint32_t* ext_off;   // n + 1: their extra instances, records n + ext_off[i] ...
    R4<R>* vacc;               // 2 n: accumulated velocity at the start of the sweep
    const uint32_t* rlist;     // shared bodies grouped by the block that reduces them (local scheduling)
    const uint32_t* rstart;    // B + 1: each block's range of rlist
    const int2* dep_r;         // B: window of each block's reduction phase
    int mlp;                   // the network's warm start of new contacts runs in the kernel's prologue
    WarmArgs<R> W;             // its arguments
};

// Rotating per-scene residual slot of sweep k (three, so that clearing the
// slot of sweep k + 1 while sweep k runs touches nothing still read).
__host__ __device__ __forceinline__ int scene_slot(int k) { return k % 3; }

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

// State of the two bodies of a contact, gathered before anything is stored.
template <class R> struct Bodies {
    R4<R> va, wa, vb, wb;
};

// Sweep records do not change during a solve.
__device__ __forceinline__ SweepRec<float> ld_rec(const SweepRec<float>* p)
{
    SweepRec<float> r;
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(r.a.x), "=f"(r.a.y), "=f"(r.a.z), "=f"(r.a.w), "=f"(r.b.x), "=f"(r.b.y), "=f"(r.b.z), "=f"(r.b.w)
        : "l"(p));
    return r;
}
__device__ __forceinline__ SweepRec<double> ld_rec(const SweepRec<double>* p)
{
    SweepRec<double> r;
    asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
        : "=d"(r.ids_bias.x), "=d"(r.ids_bias.y), "=d"(r.lev.x), "=d"(r.lev.y)
        : "l"(p));
    asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
        : "=d"(r.nxy.x), "=d"(r.nxy.y), "=d"(r.nz_.x), "=d"(r.nz_.y)
        : "l"(reinterpret_cast<const char*>(p) + 32));
    return r;
}

template <class R>
__device__ __forceinline__ void gather(const SolveArgs<R>& A, const SweepRec<R>& rr, Bodies<R>& B)
{
    uint32_t ia, ib;
    R la, lb, nx, ny, nz, bias;
    decode<R>(rr, ia, ib, la, lb, nx, ny, nz, bias);
    ld_body(A.vel + 2 * (int64_t)ia, B.va, B.wa);
    if (ib < (uint64_t)A.nslot) {
        ld_body(A.vel + 2 * (int64_t)ib, B.vb, B.wb);
    } else {
        B.vb.x = B.vb.y = B.vb.z = B.vb.w = R(0);
        B.wb = B.vb;
    }
}

// Relax one contact whose record, impulse and bodies are already loaded;
// returns r_j.  apply_only: add the stored impulse p to the bodies (initial
// impulses of a warm start) instead of relaxing.
template <class R, bool apply_only, bool Batch = false>
__device__ __forceinline__ R relax_gathered(const SolveArgs<R>& A, int64_t s, const SweepRec<R>& rr, const R4<R>& pp,
                                            Bodies<R> B, int sweep)
{
    uint32_t ia, ib;
    R la, lb, nx, ny, nz, bias;
    decode<R>(rr, ia, ib, la, lb, nx, ny, nz, bias);
    R mu = A.mu;
    double vref_s = 1.0;
    uint32_t scene = 0;
    if (Batch) {
        scene = A.V.scene_of[ia];
        if (!apply_only && sweep > 0) {
            // this scene met its tolerance in an earlier sweep: it is done
            const double prev = __longlong_as_double(
                (long long)A.scene_rk[scene_slot(sweep - 1) * A.nscene + scene]);
            if (prev <= A.tol) return R(0);
        }
        mu = (R)A.V.mu[scene];
        vref_s = A.V.vref[scene];
    }
    R4<R> va = B.va, wa = B.wa, vb = B.vb, wb = B.wb;
    const bool dyn_b = ib < (uint64_t)A.nslot;
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
        const R lim = mu * yn;
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
        st_body(A.vel + 2 * (int64_t)ia, va, wa);
    }
    if (dyn_b && (imb > R(0) || iIb > R(0))) {
        vb.x -= imb * Px;
        vb.y -= imb * Py;
        vb.z -= imb * Pz;
        const R kb = lb * iIb;
        wb.x -= kb * qx;
        wb.y -= kb * qy;
        wb.z -= kb * qz;
        st_body(A.vel + 2 * (int64_t)ib, vb, wb);
    }
    const R r1 = wn * dn, r2 = wt * dt_, r3 = wt * do_;
    const R r = sqrt(r1 * r1 + r2 * r2 + r3 * r3);
    if (Batch && !apply_only) {
        // per-scene R_k; the read filter only saves atomics
        const double rn = (double)r / vref_s;
        unsigned long long* dst = A.scene_rk + scene_slot(sweep) * A.nscene + scene;
        const unsigned long long bits = (unsigned long long)__double_as_longlong(rn);
        if (bits > *(volatile unsigned long long*)dst) atomicMax(dst, bits);
        return (R)rn;
    }
    return r;
}

template <class R, bool apply_only, bool Batch = false>
__device__ __forceinline__ R relax(const SolveArgs<R>& A, int64_t s, int sweep)
{
    const SweepRec<R> rr = ld_rec(A.rec + s);
    const R4<R> pp = A.p[s];
    Bodies<R> B;
    gather<R>(A, rr, B);
    return relax_gathered<R, apply_only, Batch>(A, s, rr, pp, B, sweep);
}

// Two contacts of one colour: both gathers are issued before either store
// (they touch disjoint finite bodies, so the order does not matter).
template <class R, bool apply_only>
__device__ __forceinline__ R relax_pair(const SolveArgs<R>& A, int64_t s0, int64_t s1, int sweep)
{
    const SweepRec<R> r0 = A.rec[s0];
    const R4<R> p0 = A.p[s0];
    SweepRec<R> r1;
    R4<R> p1;
    if (s1 >= 0) {
        r1 = A.rec[s1];
        p1 = A.p[s1];
    }
    Bodies<R> B0, B1;
    gather<R>(A, r0, B0);
    if (s1 >= 0) gather<R>(A, r1, B1);
    R r = relax_gathered<R, apply_only>(A, s0, r0, p0, B0, sweep);
    if (s1 >= 0) {
        const R q = relax_gathered<R, apply_only>(A, s1, r1, p1, B1, sweep);
        r = q > r ? q : r;
    }
    return r;
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

// Subdomains (Sect. 6.3): every instance of a shared body starts a sweep
// from the accumulated velocity.
template <class R>
__device__ __forceinline__ void inst_init_pass(const SolveArgs<R>& A, int64_t gtid, int64_t gstride)
{
    const uint32_t ns = A.info->n_shared;
    for (int64_t t = gtid; t < ns; t += gstride) {
        const int64_t i = A.shared[t];
        R4<R> v, w;
        ld_body(A.vel + 2 * i, v, w);
        st_body(A.vacc + 2 * i, v, w);
        for (uint32_t e = A.ext_off[i]; e < A.ext_off[i + 1]; ++e) st_body(A.vel + 2 * (A.n + e), v, w);
    }
}

// End of a sweep with subdomains: v <- v_acc + sum_p (instance_p - v_acc)
// over the instances in increasing subdomain (the body's own record first),
// then every instance and the accumulator restart from v.
template <class R>
__device__ __forceinline__ void inst_reduce_body(const SolveArgs<R>& A, int64_t i)
{
    R4<R> v0, w0, v, w;
    ld_body(A.vacc + 2 * i, v0, w0);
    ld_body(A.vel + 2 * i, v, w);
    R4<R> av = v0, aw = w0;
    av.x += v.x - v0.x;
    av.y += v.y - v0.y;
    av.z += v.z - v0.z;
    aw.x += w.x - w0.x;
    aw.y += w.y - w0.y;
    aw.z += w.z - w0.z;
    const uint32_t e0 = A.ext_off[i], e1 = A.ext_off[i + 1];
    for (uint32_t e = e0; e < e1; ++e) {
        ld_body(A.vel + 2 * (A.n + e), v, w);
        av.x += v.x - v0.x;
        av.y += v.y - v0.y;
        av.z += v.z - v0.z;
        aw.x += w.x - w0.x;
        aw.y += w.y - w0.y;
        aw.z += w.z - w0.z;
    }
    av.w = v0.w;   // 1/m and 1/I ride along unchanged
    aw.w = w0.w;
    st_body(A.vel + 2 * i, av, aw);
    st_body(A.vacc + 2 * i, av, aw);
    for (uint32_t e = e0; e < e1; ++e) st_body(A.vel + 2 * (A.n + e), av, aw);
}

template <class R>
__device__ __forceinline__ void inst_reduce_pass(const SolveArgs<R>& A, int64_t gtid, int64_t gstride)
{
    const uint32_t ns = A.info->n_shared;
    for (int64_t t = gtid; t < ns; t += gstride) inst_reduce_body<R>(A, A.shared[t]);
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

// ---------------------------------------------------------------------------
// Whole solve in one cooperative launch: gravity, warm-start impulses and the
// sweeps.  Block b owns the same contiguous chunk of every colour in every
// sweep.  The next colour's records and impulses do not depend on the colour
// being relaxed (records are read-only; a thread's impulses are written only
// by that thread), so they are loaded before waiting at the grid barrier and
// only the body gathers remain behind it.
// ---------------------------------------------------------------------------
constexpr int kPersistThreads = 256;

// Shared-memory stage of one colour chunk: CAP records and impulses, 48 KiB.
template <class R> struct Stage {
    static constexpr int CAP = sizeof(R) == 4 ? 256 : 128;
    static constexpr int BYTES = CAP * (int)(sizeof(SweepRec<R>) + sizeof(R4<R>));
};

// Block b owns, in every colour, the contacts whose canonical index lies in
// [ceil(b C / B), ceil((b + 1) C / B)): a contiguous range of the colour
// (the colour sort is stable), balanced by contact count and local in body
// index, so that a chunk's bodies are touched only by nearby blocks.
// --- TMA bulk copies (global -> shared) completed on an mbarrier -----------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait for the stage of the given parity; false (timeout bit set)
// after ~2^31 SM clocks.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, DevInfo* info)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1LL << 31)) {
            atomicOr(&info->err, kErrTimeout);
            return false;
        }
    }
    return true;
}

// Thread 0 starts the copy of this block's chunk of colour c (its first CAP
// contacts) into the stage; returns the number of staged contacts.
template <class R>
__device__ __forceinline__ int stage_issue(const SolveArgs<R>& A, int c, SweepRec<R>* srec, R4<R>* sp, uint64_t* bar)
{
    int64_t b0, b1;
    colour_chunk(A.cstart, c, b0, b1);
    const int m = (int)(b1 - b0 < Stage<R>::CAP ? b1 - b0 : Stage<R>::CAP);
    if (threadIdx.x == 0 && m > 0) {
        // the impulses were written through the generic proxy
        asm volatile("fence.proxy.async.global;" ::: "memory");
        const uint32_t br = (uint32_t)(m * sizeof(SweepRec<R>)), bp = (uint32_t)(m * sizeof(R4<R>));
        mbar_expect_tx(bar, br + bp);
        bulk_g2s(srec, A.rec + b0, br, bar);
        bulk_g2s(sp, A.p + b0, bp, bar);
    }
    return m;
}

template <class R, bool apply_only, bool Batch>
__device__ __forceinline__ R process_colour(const SolveArgs<R>& A, int c, int m, const SweepRec<R>* srec,
                                            const R4<R>* sp, int sweep)
{
    R rmax = R(0);
    int64_t b0, b1;
    colour_chunk(A.cstart, c, b0, b1);
    const int T = blockDim.x;
    // staged part: records and impulses from shared memory
    for (int slot = threadIdx.x; slot < m; slot += T) {
        const SweepRec<R> r0 = srec[slot];
        const R4<R> p0 = sp[slot];
        Bodies<R> B0;
        gather<R>(A, r0, B0);
        const R r = relax_gathered<R, apply_only, Batch>(A, b0 + slot, r0, p0, B0, sweep);
        rmax = r > rmax ? r : rmax;
    }
    // the rest of the chunk straight from global memory
    for (int64_t s = b0 + m + threadIdx.x; s < b1; s += T) {
        const R r = relax<R, apply_only, Batch>(A, s, sweep);
        rmax = r > rmax ? r : rmax;
    }
    return rmax;
}

// L2 prefetch of the records and impulses of this block's chunk of colour c:
// a hint issued one colour ahead, so that the lines stream in from HBM while
// the current colour is relaxed (the bodies stay in L2 anyway).
template <class R>
__device__ __forceinline__ void prefetch_chunk(const SolveArgs<R>& A, int c)
{
    int64_t b0, b1;
    colour_chunk(A.cstart, c, b0, b1);
    if (b1 <= b0) return;
    const char* r0 = reinterpret_cast<const char*>(A.rec + b0);
    const char* r1 = reinterpret_cast<const char*>(A.rec + b1);
    const char* p0 = reinterpret_cast<const char*>(A.p + b0);
    const char* p1 = reinterpret_cast<const char*>(A.p + b1);
    const int64_t nr = (r1 - r0 + 127) / 128, np = (p1 - p0 + 127) / 128;
    for (int64_t i = threadIdx.x; i < nr + np; i += blockDim.x) {
        const char* a = i < nr ? r0 + 128 * i : p0 + 128 * (i - nr);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
}

// Split grid barrier: arrive (after this block's stores), do independent
// work, then wait.  The wait gives up after ~2^31 SM clocks (about a
// second), sets the timeout bit and returns false.
__device__ __forceinline__ void barrier_arrive(DevInfo* info, unsigned nblocks, uint32_t* s_gen)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t* vgen = &info->barrier_gen;
        const uint32_t gen = *vgen;
        __threadfence();
        const uint32_t arrived = atomicAdd(&info->barrier_count, 1u);
        if (arrived == nblocks - 1) {
            info->barrier_count = 0;
            __threadfence();
            atomicAdd(&info->barrier_gen, 1u);
        }
        *s_gen = gen;
    }
}

__device__ __forceinline__ bool barrier_wait(DevInfo* info, const uint32_t* s_gen, int* s_ok)
{
    if (threadIdx.x == 0) {
        volatile uint32_t* vgen = &info->barrier_gen;
        volatile uint32_t* verr = &info->err;
        const uint32_t gen = *s_gen;
        int ok = 1;
        const long long t0 = clock64();
        while (*vgen == gen) {
            if (*verr & kErrTimeout) {
                ok = 0;
                break;
            }
            if (clock64() - t0 > (1LL << 31)) {
                atomicOr(&info->err, kErrTimeout);
                ok = 0;
                break;
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

template <class R, bool Batch, int K = 1> struct PersistMinBlocks {
    // FP64 and the per-scene bookkeeping of batches need more registers per
    // thread, and so does a second contact whose state a thread holds
    static constexpr int value = sizeof(R) == 4 ? (K == 1 ? (Batch ? 3 : 4) : (Batch ? 2 : 3)) : (K == 1 ? 2 : 1);
};

// --- warp-level scheduling (NBGS_SWEEP_WARP_SYNC) ---------------------------
// Every warp is a scheduling unit of its own ("virtual block" vb = 8 b + w of
// V = 8 B): its own chunk of each colour, its own window and progress word,
// so that warps of a block never wait for one another inside a sweep.
__device__ __forceinline__ void warp_chunk(const uint32_t* cstart, int c, int nv, int vb, int64_t& b0, int64_t& b1)
{
    const uint32_t* row = cstart + (int64_t)c * (nv + 1);
    b0 = row[vb];
    b1 = row[vb + 1];
}

// The lanes of the warp poll the progress words of its window (bounded like
// every other wait); returns the same value on every lane.
__device__ __forceinline__ bool wait_deps_warp(const int* prog, int2 win, int g, DevInfo* info, int nv, int self)
{
    const int lane = threadIdx.x & 31;
    int ok = 1;
    for (int off = win.x + lane; off <= win.y && ok; off += 32) {
        if (off == 0) continue;
        const int b = ((self + off) % nv + nv) % nv;
        const long long t0 = clock64();
        while (ld_acquire(prog + b) < g - 1) {
            if (((volatile uint32_t*)&info->err)[0] & kErrTimeout) {
                ok = 0;
                break;
            }
            if (clock64() - t0 > (1LL << 31)) {
                atomicOr(&info->err, kErrTimeout);
                ok = 0;
                break;
            }
        }
    }
    return __all_sync(0xffffffffu, ok) != 0;
}

// Publish that this warp finished phase g (after all its lanes' stores).
__device__ __forceinline__ void publish_warp(int* prog, int vb, int g)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        __threadfence();
        atomicExch(prog + vb, g);
    }
}

template <class R, bool apply_only, bool Batch>
__device__ __forceinline__ R process_chunk_warp(const SolveArgs<R>& A, int64_t b0, int64_t b1, int sweep)
{
    R rmax = R(0);
    for (int64_t s = b0 + (threadIdx.x & 31); s < b1; s += 32) {
        const R r = relax<R, apply_only, Batch>(A, s, sweep);
        rmax = r > rmax ? r : rmax;
    }
    return rmax;
}

template <class R>
__device__ __forceinline__ void prefetch_range(const SolveArgs<R>& A, int64_t b0, int64_t b1, int lane, int width)
{
    if (b1 <= b0) return;
    const char* r0 = reinterpret_cast<const char*>(A.rec + b0);
    const char* r1 = reinterpret_cast<const char*>(A.rec + b1);
    const char* p0 = reinterpret_cast<const char*>(A.p + b0);
    const char* p1 = reinterpret_cast<const char*>(A.p + b1);
    const int64_t nr = (r1 - r0 + 127) / 128, np = (p1 - p0 + 127) / 128;
    for (int64_t i = lane; i < nr + np; i += width) {
        const char* a = i < nr ? r0 + 128 * i : p0 + 128 * (i - nr);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
}

// Gathered processing of a chunk: a thread loads the records and impulses
// of up to K of its contacts, then the state of all their bodies, and only
// then relaxes them one after the other.  Contacts of one colour share no
// finite body, so the loads of contact k + 1 may precede the stores of
// contact k; the K dependent chains (record -> bodies -> stores) overlap
// instead of running back to back.  The first K records and impulses of a
// colour are loaded before the wait for the neighbouring blocks (they do not
// depend on it: records are read-only and a slot's impulse is written by
// the same thread only).
template <class R, int K>
__device__ __forceinline__ void preload(const SolveArgs<R>& A, int64_t base, int64_t b1, SweepRec<R> (&pr)[K],
                                        R4<R> (&pq)[K])
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t s = base + (int64_t)k * blockDim.x;
        if (s < b1) {
            pr[k] = ld_rec(A.rec + s);
            pq[k] = A.p[s];
        }
    }
}

template <class R, bool Batch, int K>
__device__ __forceinline__ R process_gathered(const SolveArgs<R>& A, int64_t b0, int64_t b1, SweepRec<R> (&pr)[K],
                                              R4<R> (&pq)[K], int sweep)
{
    R rmax = R(0);
    const int64_t T = blockDim.x;
    for (int64_t base = b0 + threadIdx.x; base < b1; base += K * T) {
        if (base != b0 + threadIdx.x) preload<R, K>(A, base, b1, pr, pq);
        Bodies<R> B[K];
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (base + k * T < b1) gather<R>(A, pr[k], B[k]);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (base + k * T < b1) {
                const R r = relax_gathered<R, false, Batch>(A, base + k * T, pr[k], pq[k], B[k], sweep);
                rmax = r > rmax ? r : rmax;
            }
        }
    }
    return rmax;
}

// The tolerance test of sweep k without a grid barrier.  R_k <= tol holds
// exactly when every block's own maximum (divided by the same v_ref) is at
// or below tol, so a block above it announces that and goes on at once; a
// block at or below it counts itself and waits until either some block has
// announced (the sweeps go on) or every block has counted itself (the solve
// stops after sweep k).  Every block reaches the end of sweep k, so the
// wait ends; bounded like every other.  Returns 1 to go on, 0 to stop, -1
// when the wait ran out.
__device__ __forceinline__ int tol_vote(DevInfo* info, int k, double rb, double vnorm, double tol, unsigned nb,
                                        int* s_vote)
{
    if (threadIdx.x == 0) {
        uint32_t* flag = info->votes + 2 * k;
        int v = 1;
        if (!(rb / vnorm <= tol)) {
            atomicExch(flag, 1u);
        } else {
            atomicAdd(flag + 1, 1u);
            const long long t0 = clock64();
            for (;;) {
                if (((volatile uint32_t*)flag)[0] != 0u) break;
                if (((volatile uint32_t*)flag)[1] == nb) {
                    v = 0;
                    break;
                }
                if ((((volatile uint32_t*)&info->err)[0] & kErrTimeout) || clock64() - t0 > (1LL << 31)) {
                    atomicOr(&info->err, kErrTimeout);
                    v = -1;
                    break;
                }
            }
        }
        *s_vote = v;
    }
    __syncthreads();
    return *s_vote;
}

template <class R, bool Batch, bool Warp, bool Sub, int K = 1, bool Mlp = false>
__global__ void __launch_bounds__(kPersistThreads, (PersistMinBlocks<R, Batch, K>::value)) k_solve_persistent(SolveArgs<R> A)
{
    extern __shared__ __align__(128) unsigned char stage_mem[];
    SweepRec<R>* srec = reinterpret_cast<SweepRec<R>*>(stage_mem);
    R4<R>* sp = reinterpret_cast<R4<R>*>(stage_mem + Stage<R>::CAP * sizeof(SweepRec<R>));
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_gen;
    __shared__ int s_ok;
    __shared__ int s_vote;
    const unsigned nb = gridDim.x;
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    const int ncol = (int)A.info->n_colours;
    const double vref = v_ref_of(A.info, A.gdt_norm);
    const double vnorm = Batch ? 1.0 : vref;   // batched residuals arrive already divided by v_ref_s
    const bool stage = K == 1 && !Warp && (A.flags & NBGS_SWEEP_TMA_STAGE) != 0;
    const bool local = (A.flags & NBGS_SWEEP_GLOBAL_SYNC) == 0;
    if (threadIdx.x == 0) mbar_init(&bar);
    if constexpr (Mlp) {
        // the network's warm start (tensor cores, 128 contacts per tile, the
        // dynamic shared memory as its operand space), every impulse written
        // before any block applies them
        warm_tiles<R>(A.W, reinterpret_cast<TcMlpSmem*>(stage_mem));
        if (!grid_barrier(A.info, nb)) return;
    }
    gravity_pass<R>(A, gtid, gstride);
    if (!grid_barrier(A.info, nb)) return;
    if (Sub) {
        inst_init_pass<R>(A, gtid, gstride);
        if (!grid_barrier(A.info, nb)) return;
    }
    const int nv = (int)nb * (kPersistThreads / 32), vb = (int)blockIdx.x * (kPersistThreads / 32) + (threadIdx.x >> 5);
    if (A.warm) {
        for (int c = 0; c < ncol; ++c) {
            if (Warp) {
                int64_t w0, w1;
                warp_chunk(A.cstart, c, nv, vb, w0, w1);
                process_chunk_warp<R, true, Batch>(A, w0, w1, 0);
            } else {
                process_colour<R, true, Batch>(A, c, 0, srec, sp, 0);
            }
            if (!grid_barrier(A.info, nb)) return;
        }
        if (Sub) {   // the initial impulses land in the accumulators
            inst_reduce_pass<R>(A, gtid, gstride);
            if (!grid_barrier(A.info, nb)) return;
        }
    }
    // subdomains under local scheduling: the reduction is one more phase of
    // every sweep, each block summing the shared bodies assigned to it after
    // the blocks that touch them have finished the sweep
    const bool wred = Sub && local && !Warp;
    const int P = wred ? ncol + 1 : ncol;   // phases per sweep
    uint32_t parity = 0;
    int m = (stage && ncol > 0) ? stage_issue<R>(A, 0, srec, sp, &bar) : 0;   // a copy is in flight iff m > 0
    int k = 0;
    double Rk = 0.0;
    bool ok = true, synced = true;
    for (; k < A.max_sweeps && ok; ++k) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && k + 1 >= kHistKept) A.info->rk_bits[rk_slot(k + 1)] = 0ull;
        if (Batch)   // the slot of sweep k + 1 is neither read nor written during sweep k
            for (int64_t sc = gtid; sc < A.nscene; sc += gstride) A.scene_rk[scene_slot(k + 1) * A.nscene + sc] = 0ull;
        R rmax = R(0);
        double rb = 0.0;   // this block's max_j r_j of the sweep (thread 0)
        if (Warp) {
            // each warp on its own; a warp whose wait gave up skips the rest
            // of the sweep (the timeout bit makes every other wait return)
            bool wok = true;
            for (int c = 0; c < ncol; ++c) {
                const int g = k * ncol + c;
                int64_t w0, w1;
                warp_chunk(A.cstart, c, nv, vb, w0, w1);
                if (wok && w1 > w0 && !wait_deps_warp(A.prog, A.dep[(int64_t)c * nv + vb], g, A.info, nv, vb))
                    wok = false;
                if (wok) {
                    int64_t n0, n1;
                    warp_chunk(A.cstart, c + 1 < ncol ? c + 1 : 0, nv, vb, n0, n1);
                    prefetch_range<R>(A, n0, n1, threadIdx.x & 31, 32);
                    const R r = process_chunk_warp<R, false, Batch>(A, w0, w1, k);
                    rmax = r > rmax ? r : rmax;
                    publish_warp(A.prog, vb, g);
                }
            }
            block_max_to<R>(rmax, &A.info->rk_bits[rk_slot(k)]);
            if (!__syncthreads_and(wok)) {
                ok = false;
                break;
            }
        }
        for (int c = 0; c < (Warp ? 0 : ncol); ++c) {
            const int g = k * P + c;
            int64_t cb0, cb1;
            colour_chunk(A.cstart, c, cb0, cb1);
            SweepRec<R> pr[K];
            R4<R> pq[K];
            if (!stage) preload<R, K>(A, cb0 + threadIdx.x, cb1, pr, pq);
            // an empty chunk touches no body: nothing to wait for (this block's
            // own earlier phases are complete, which is all a neighbour needs)
            if (local && cb1 > cb0 && !wait_deps(A.prog, A.dep[c * (int)nb + blockIdx.x], g, A.info, &s_ok)) {
                ok = false;
                break;
            }
            if (m > 0) {
                if (!mbar_wait(&bar, parity, A.info)) {
                    ok = false;
                    break;
                }
                parity ^= 1u;
            }
            const int cn = c + 1 < ncol ? c + 1 : 0;
            prefetch_chunk<R>(A, c + 1 < ncol ? c + 1 : 0);
            const R r = !stage ? process_gathered<R, Batch, K>(A, cb0, cb1, pr, pq, k)
                               : process_colour<R, false, Batch>(A, c, m, srec, sp, k);
            rmax = r > rmax ? r : rmax;
            if (c == ncol - 1) rb = block_max_to<R>(rmax, &A.info->rk_bits[rk_slot(k)]);
            if (local) {
                publish(A.prog, g);   // its __syncthreads also ends every read of the stage
                m = stage ? stage_issue<R>(A, cn, srec, sp, &bar) : 0;
            } else {
                barrier_arrive(A.info, nb, &s_gen);
                m = stage ? stage_issue<R>(A, cn, srec, sp, &bar) : 0;
                if (!barrier_wait(A.info, &s_gen, &s_ok)) {
                    ok = false;
                    break;
                }
            }
        }
        if (!ok) break;
        synced = !local;
        if (wred && ncol > 0) {
            const int g = k * P + ncol;
            const uint32_t r0 = A.rstart[blockIdx.x], r1 = A.rstart[blockIdx.x + 1];
            if (r1 > r0 && !wait_deps(A.prog, A.dep_r[blockIdx.x], g, A.info, &s_ok)) {
                ok = false;
                break;
            }
            for (uint32_t t = r0 + threadIdx.x; t < r1; t += blockDim.x) inst_reduce_body<R>(A, A.rlist[t]);
            publish(A.prog, g);
        } else if (Sub && ncol > 0) {
            // subdomains: every contact of the sweep is done before the
            // corrections are summed, and the sum before the next sweep
            if (!grid_barrier(A.info, nb)) {
                ok = false;
                break;
            }
            inst_reduce_pass<R>(A, gtid, gstride);
            if (!grid_barrier(A.info, nb)) {
                ok = false;
                break;
            }
            synced = true;
        }
        // a single scene's tolerance test: a vote instead of a grid barrier
        if (!synced && local && !Warp && !Batch && !Sub && ncol > 0 && A.tol > 0.0 && k + 2 < kHistKept) {
            const int v = tol_vote(A.info, k, rb, vnorm, A.tol, nb, &s_vote);
            if (v < 0) {
                ok = false;
                break;
            }
            if (v == 0) {
                ++k;
                break;
            }
            continue;
        }
        // R_k needs every block's contribution: a grid barrier per sweep when
        // the tolerance is tested (and near the rotating residual slots)
        if (!synced && local && ncol > 0 && (A.tol > 0.0 || Batch || k + 2 >= kHistKept)) {
            if (!grid_barrier(A.info, nb)) {
                ok = false;
                break;
            }
            synced = true;
        }
        if (synced && Batch && A.tol > 0.0) {   // scenes that met their tolerance in this sweep
            for (int64_t sc = gtid; sc < A.nscene; sc += gstride) {
                const double rs = __longlong_as_double(
                    (long long)((volatile unsigned long long*)A.scene_rk)[scene_slot(k) * A.nscene + sc]);
                if (A.scene_done[sc] == 0 && rs <= A.tol) {
                    A.scene_done[sc] = (uint32_t)(k + 1);
                    A.scene_res[sc] = rs;
                }
            }
        }
        if (synced) {
            Rk = __longlong_as_double((long long)((volatile unsigned long long*)A.info->rk_bits)[rk_slot(k)]) / vnorm;
            if (A.tol > 0.0 && Rk <= A.tol) {
                ++k;
                break;
            }
        }
    }
    // never leave with a copy into this block's shared memory in flight
    if (m > 0) mbar_wait(&bar, parity, A.info);
    if (!ok) return;
    if (!synced && k > 0) {
        if (!grid_barrier(A.info, nb)) return;
        Rk = __longlong_as_double((long long)((volatile unsigned long long*)A.info->rk_bits)[rk_slot(k - 1)]) / vnorm;
    }
    if (Batch) {   // scenes still short of their tolerance ran every sweep
        for (int64_t sc = gtid; sc < A.nscene; sc += gstride) {
            if (A.scene_done[sc] == 0) {
                A.scene_done[sc] = (uint32_t)k;
                A.scene_res[sc] = k > 0 ? __longlong_as_double((long long)((volatile unsigned long long*)
                                                                               A.scene_rk)[scene_slot(k - 1) * A.nscene + sc])
                                        : 0.0;
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.info->sweeps_done = (uint32_t)k;
        A.info->residual = Rk;
        A.info->v_ref = vref;
    }
}

// --- block windows of the chunks (local synchronisation) -------------------
// Blocks form a ring.  Body x is mapped to its home block ref(x) = x B / n;
// the blocks whose chunks (any colour) hold a contact of x are recorded as
// circular offsets from ref(x) in [-B/2, B/2), so the contacts that close a
// periodic box (first and last bodies) stay neighbours on the ring.
__device__ __forceinline__ int ring_off(int64_t d, int nblk)
{
    const int64_t h = nblk / 2;
    return (int)((((d + h) % nblk) + nblk) % nblk - h);
}

// Block owning canonical contact k: floor(k B / C); home block of body x:
// the block of its first canonical contact (row_off[x]).
__device__ __forceinline__ int block_of(int64_t k, int64_t C, int nblk)
{
    const int64_t b = (k * nblk) / C;
    return (int)(b < nblk ? b : nblk - 1);
}

// Subdomains under local scheduling: shared body i is reduced by the first
// block on the ring whose chunks hold a contact of it (home block + dmin);
// every block touching i lies within dmax - dmin blocks after it, so that
// block's reduction window is [0, largest span of its bodies], and every
// chunk touching i has the reducing block in its own window.
__global__ void k_reduce_count(int64_t C, int nblk, const uint32_t* __restrict__ shared,
                               const DevInfo* __restrict__ info, const uint32_t* __restrict__ row_off,
                               const int* __restrict__ dmin, const int* __restrict__ dmax,
                               uint32_t* __restrict__ rcount, int2* __restrict__ dep_r)
{
    const uint32_t ns = info->n_shared;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ns; t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = shared[t];
        const int r = ((block_of(row_off[i], C, nblk) + dmin[i]) % nblk + nblk) % nblk;
        atomicAdd(&rcount[r], 1u);
        atomicMax(&dep_r[r].y, dmax[i] - dmin[i]);
    }
}

__global__ void k_reduce_fill(int64_t C, int nblk, const uint32_t* __restrict__ shared,
                              const DevInfo* __restrict__ info, const uint32_t* __restrict__ row_off,
                              const int* __restrict__ dmin, const uint32_t* __restrict__ rstart,
                              uint32_t* __restrict__ rfill, uint32_t* __restrict__ rlist)
{
    const uint32_t ns = info->n_shared;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ns; t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = shared[t];
        const int r = ((block_of(row_off[i], C, nblk) + dmin[i]) % nblk + nblk) % nblk;
        rlist[rstart[r] + atomicAdd(&rfill[r], 1u)] = i;
    }
}

// Chunk boundaries: cstart[c][b] = first slot of colour c whose canonical
// index is >= ceil(b C / B) (binary search; perm is increasing in a colour).
__global__ void k_chunk_starts(DCount Cc, int nblk, const uint32_t* __restrict__ col_off,
                               const uint32_t* __restrict__ perm, const DevInfo* __restrict__ info,
                               uint32_t* __restrict__ cstart)
{
    const int64_t C = Cc.get();
    const int ncol = (int)info->n_colours;
    const int64_t total = (int64_t)ncol * (nblk + 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / (nblk + 1)), b = (int)(t % (nblk + 1));
        const int64_t target = ((int64_t)b * C + nblk - 1) / nblk;
        int64_t lo = col_off[c], hi = col_off[c + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)perm[mid] < target) lo = mid + 1;
            else hi = mid;
        }
        cstart[t] = (uint32_t)lo;
    }
}

// Pass 1: per finite body, min and max ring offset (from its home block) of
// the blocks whose chunks hold a contact of the body.
__global__ void k_body_blocks(DCount Cc, int64_t n, int nblk, const uint32_t* __restrict__ perm,
                              const uint32_t* __restrict__ cj1, const uint32_t* __restrict__ cj2,
                              const uint32_t* __restrict__ row_off, const uint8_t* __restrict__ finite,
                              int* __restrict__ dmin, int* __restrict__ dmax)
{
    const int64_t C = Cc.get();
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < C; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = perm[s];
        const int b = block_of(k, C, nblk);
        const uint32_t x = cj1[k], y = cj2[k];
        if (finite[x]) {
            const int d = ring_off(b - block_of(row_off[x], C, nblk), nblk);
            atomicMin(&dmin[x], d);
            atomicMax(&dmax[x], d);
        }
        if (y < n && finite[y]) {
            const int d = ring_off(b - block_of(row_off[y], C, nblk), nblk);
            atomicMin(&dmin[y], d);
            atomicMax(&dmax[y], d);
        }
    }
}

// Pass 2: block b computes, for its chunk of every colour, the ring window
// [lo, hi] (offsets from b) covering every block that touches one of the
// chunk's bodies.
__global__ void k_chunk_windows(DCount Cc, int64_t n, const uint32_t* __restrict__ cstart,
                                const uint32_t* __restrict__ perm, const uint32_t* __restrict__ cj1,
                                const uint32_t* __restrict__ cj2, const uint32_t* __restrict__ row_off,
                                const uint8_t* __restrict__ finite, const int* __restrict__ dmin,
                                const int* __restrict__ dmax, const DevInfo* __restrict__ info,
                                int2* __restrict__ dep)
{
    const int64_t C = Cc.get();
    __shared__ int slo[32], shi[32];
    const int ncol = (int)info->n_colours;
    const int nblk = gridDim.x;
    const int self = blockIdx.x;
    for (int c = 0; c < ncol; ++c) {
        int64_t b0, b1;
        colour_chunk(cstart, c, b0, b1);
        int lo = 0, hi = 0;
        for (int64_t s = b0 + threadIdx.x; s < b1; s += blockDim.x) {
            const uint32_t k = perm[s];
            const uint32_t xs[2] = {cj1[k], cj2[k]};
            for (int e = 0; e < 2; ++e) {
                const uint32_t x = xs[e];
                if (x >= n || !finite[x]) continue;
                const int l = ring_off((int64_t)block_of(row_off[x], C, nblk) + dmin[x] - self, nblk);
                lo = min(lo, l);
                hi = max(hi, l + (dmax[x] - dmin[x]));
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_down_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_down_sync(0xffffffffu, hi, o));
        }
        if ((threadIdx.x & 31) == 0) {
            slo[threadIdx.x >> 5] = lo;
            shi[threadIdx.x >> 5] = hi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                lo = min(lo, slo[w]);
                hi = max(hi, shi[w]);
            }
            if (hi - lo >= nblk) {   // the window covers the ring: every block
                lo = -self;
                hi = nblk - 1 - self;
            }
            dep[c * nblk + self] = make_int2(lo, hi);
        }
        __syncthreads();
    }
}

// Chunk starts and dependency windows of a cooperative sweep over B blocks,
// for contacts whose ends act on the bodies ib1, ib2 (>= ninc: a wall) of
// finiteness finc, body x anchored at the canonical contact position
// anchor[x] (any fixed position: the windows are offsets from it); the
// progress words start at -1.  The body degree arrays of the colouring serve
// as scratch.
nbgs_status build_windows(nbgs_scene* s, int B, int64_t ninc, const uint32_t* ib1, const uint32_t* ib2,
                          const uint32_t* anchor, const uint8_t* finc)
{
    const int T = 256;
    const int64_t C = s->n_contacts;
    cudaStream_t st = s->stream;
    k_chunk_starts<<<grid_for((int64_t)kMaxColours * (B + 1), T, 8, s->num_sms), T, 0, st>>>(DCount{C, nullptr}, B, s->col_off,
                                                                                          s->perm, s->info, s->cstart);
    int* dmin = (int*)s->deg;
    int* dmax = (int*)s->adj_off;
    cudaMemsetAsync(dmin, 0x7F, (size_t)std::max<int64_t>(ninc, 1) * sizeof(int), st);
    cudaMemsetAsync(dmax, 0x80, (size_t)std::max<int64_t>(ninc, 1) * sizeof(int), st);
    k_body_blocks<<<grid_for(C, T, 8, s->num_sms), T, 0, st>>>(DCount{C, nullptr}, ninc, B, s->perm, ib1, ib2, anchor, finc, dmin,
                                                                dmax);
    k_chunk_windows<<<B, T, 0, st>>>(DCount{C, nullptr}, ninc, s->cstart, s->perm, ib1, ib2, anchor, finc, dmin, dmax, s->info,
                                      s->dep);
    cudaMemsetAsync(s->prog, 0xFF, (size_t)B * sizeof(int), st);
    if (s->timing) s->phase_launches[2] += 3;
    return cuda_check(s, cudaGetLastError(), "solve: dependency windows");
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
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = b + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < e; s += 2 * T) {
        const R r = relax_pair<R, apply_only>(A, s, s + T < e ? s + T : -1, sweep);
        rmax = r > rmax ? r : rmax;
    }
    if (!apply_only) block_max_to<R>(rmax, &A.info->rk_bits[rk_slot(sweep)]);
}

template <class R>
__global__ void k_inst_init(SolveArgs<R> A)
{
    inst_init_pass<R>(A, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// after_sweep: skip once an earlier sweep met the tolerance (nothing moved)
template <class R>
__global__ void k_inst_reduce(SolveArgs<R> A, int after_sweep)
{
    if (after_sweep && A.info->sweeps_done != 0xFFFFFFFFu) return;
    inst_reduce_pass<R>(A, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
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

__global__ void k_scene_vref(int64_t S, const unsigned long long* __restrict__ vmax, double gdt_norm,
                             double* __restrict__ vref)
{
    for (int64_t sc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sc < S; sc += (int64_t)gridDim.x * blockDim.x)
        vref[sc] = fmax(fmax(xsqrt(__longlong_as_double((long long)vmax[sc])), gdt_norm), 1e-12);   // max |v|^2 kept
}

// Canonical impulses (contact frame) and world-frame impulses for the next
// warm start.
template <class R>
__global__ void k_finish(DCount Cc, const uint32_t* __restrict__ inv, const R4<R>* __restrict__ p,
                         const double4_32a* __restrict__ cgeo, double4_32a* __restrict__ cimp, double4_32a* __restrict__ cworld)
{
    const int64_t C = Cc.get();
    // a thread per canonical contact: only the impulse is read scattered
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const R4<R> q = p[inv[c]];
        const double4_32a g = cgeo[c];
        double tx, ty, tz, ox, oy, oz;
        tangent_basis<double>(g.x, g.y, g.z, tx, ty, tz, ox, oy, oz);
        const double pn = q.x, pt = q.y, po = q.z;
        cimp[c] = make_double4_32a(pn, pt, po, 0.0);
        cworld[c] = make_double4_32a(pn * g.x + pt * tx + po * ox, pn * g.y + pt * ty + po * oy,
                                 pn * g.z + pt * tz + po * oz, 0.0);
    }
}

// Contact updates of the solve just finished: every contact relaxed once
// per sweep its scene ran (a scene of a batch stops at its own tolerance).
__global__ void k_count_updates(DCount Cc, int max_sweeps, const uint32_t* __restrict__ perm,
                                const uint32_t* __restrict__ cj1, SceneView V, const uint32_t* __restrict__ scene_done,
                                DevInfo* info)
{
    const int64_t C = Cc.get();
    if (max_sweeps == 0) return;
    if (!V.batch) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&info->updates, (unsigned long long)C * info->sweeps_done);
        return;
    }
    unsigned long long u = 0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < C; s += (int64_t)gridDim.x * blockDim.x)
        u += scene_done[V.scene_of[cj1[perm[s]]]];
    for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
    if ((threadIdx.x & 31) == 0 && u) atomicAdd(&info->updates, u);
}

// Impulses given in canonical order and in the contact frame (n, t, o)
// become the contacts' current impulses: the ones the residuals evaluate
// and the next step's warm start reads (as world vectors, like k_finish).
__global__ void k_set_impulses(int64_t C, const double* __restrict__ p3, const double4_32a* __restrict__ cgeo,
                               double4_32a* __restrict__ cimp, double4_32a* __restrict__ cworld)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const double pn = p3[3 * c], pt = p3[3 * c + 1], po = p3[3 * c + 2];
        const double4_32a g = cgeo[c];
        double tx, ty, tz, ox, oy, oz;
        tangent_basis<double>(g.x, g.y, g.z, tx, ty, tz, ox, oy, oz);
        cimp[c] = make_double4_32a(pn, pt, po, 0.0);
        cworld[c] = make_double4_32a(pn * g.x + pt * tx + po * ox, pn * g.y + pt * ty + po * oy,
                                     pn * g.z + pt * tz + po * oz, 0.0);
    }
}

nbgs_status run_set_impulses(nbgs_scene* s, const double* impulse)
{
    const int64_t C = s->n_contacts;
    if (C == 0) return NBGS_OK;
    cudaStream_t st = s->stream;
    double* tmp = (double*)dev_alloc(s, (size_t)C * 3 * sizeof(double));
    if (!tmp) return fail(s, NBGS_ENOMEM, "set_impulses: staging buffer");
    nbgs_status rc = cuda_check(s, cudaMemcpyAsync(tmp, impulse, (size_t)C * 3 * sizeof(double), cudaMemcpyDefault, st),
                                "set_impulses: copy");
    if (rc == NBGS_OK) {
        k_set_impulses<<<grid_for(C, 256, 8, s->num_sms), 256, 0, st>>>(C, tmp, s->cgeo, s->cimp, s->cworld);
        rc = cuda_check(s, cudaGetLastError(), "set_impulses");
    }
    if (rc == NBGS_OK) rc = cuda_check(s, cudaStreamSynchronize(st), "set_impulses");
    dev_free(s, tmp);
    return rc;
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
    A.warm = ((s->prm.warm_start == NBGS_WARM_PREV && s->have_prev) || s->prm.warm_start == NBGS_WARM_MLP) ? 1 : 0;
    A.flags = s->prm.sweep_flags;
    A.prog = s->prog;
    A.dep = s->dep;
    A.cstart = s->cstart;
    A.V = scene_view(s);
    A.nscene = s->n_scenes;
    A.scene_rk = s->scene_rk;
    A.scene_done = s->scene_done;
    A.scene_res = s->scene_res;
    A.sub = (s->prm.subdomain_mode != NBGS_SUB_NONE && !s->batch) ? 1 : 0;
    A.nslot = A.sub ? s->n + s->icap : s->n;
    A.shared = s->shared;
    A.ext_off = s->ext_off;
    A.vacc = (R4<R>*)s->vacc;
    A.rlist = s->rlist;
    A.rstart = s->rstart;
    A.dep_r = s->dep_r;
    A.mlp = 0;
    return A;
}

// Contacts a thread gathers at once in the persistent sweep (sweep flags).
static int gather_k(int flags) { return (flags & NBGS_SWEEP_GATHER2) ? 2 : 1; }

// Resident blocks per SM of one persistent sweep variant (with the shared
// memory of the TMA stage reserved), looked up once per variant.
template <class R>
static int persist_occ(const void* fn)
{
    static std::mutex mu;
    static std::vector<std::pair<const void*, int>> known;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto& kv : known)
        if (kv.first == fn) return kv.second;
    int o = 0;
    const int dyn = (int)std::max<size_t>(Stage<R>::BYTES, sizeof(TcMlpSmem));   // TMA stage or network operands
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, kPersistThreads, dyn);
    cudaGetLastError();
    known.emplace_back(fn, o);
    return o;
}

template <class R>
static nbgs_status solve_impl(nbgs_scene* s, int max_sweeps, double tol)
{
    cudaStream_t st = s->stream;
    SolveArgs<R> A = make_args<R>(s, max_sweeps, tol);
    const int nk = max_sweeps < kHistKept ? max_sweeps : kHistKept + 3;
    cudaMemsetAsync(A.info->rk_bits, 0, (size_t)(nk > 0 ? nk : 1) * sizeof(unsigned long long), st);
    cudaMemsetAsync(A.info->votes, 0, (size_t)(nk > 0 ? 2 * nk : 2) * sizeof(uint32_t), st);
    cudaMemsetAsync(&A.info->barrier_count, 0, 2 * sizeof(uint32_t), st);
    const uint32_t not_done = 0xFFFFFFFFu;
    if (s->batch) {
        k_scene_vref<<<grid_for(s->n_scenes, 256, 8, s->num_sms), 256, 0, st>>>(s->n_scenes, s->scene_vmax, A.gdt_norm,
                                                                               s->scene_vref);
        cudaMemsetAsync(s->scene_rk, 0, 3 * s->n_scenes * sizeof(unsigned long long), st);
        cudaMemsetAsync(s->scene_done, 0, s->n_scenes * sizeof(uint32_t), st);
        cudaMemsetAsync(s->scene_res, 0, s->n_scenes * sizeof(double), st);
        if (s->timing) s->phase_launches[2] += 1;
    }
    if (s->prm.warm_start == NBGS_WARM_MLP) {
        const bool warp_sched = (s->prm.sweep_flags & NBGS_SWEEP_WARP_SYNC) && !(s->prm.sweep_flags & NBGS_SWEEP_GLOBAL_SYNC);
        if (s->prm.solver == NBGS_SOLVER_PERSISTENT && !s->composite && s->n_contacts > 0 && !A.sub && !warp_sched) {
            // fused into the persistent kernel's prologue
            if (!s->mlp_theta) return fail(s, NBGS_EINVAL, "MLP warm start: no network loaded (nbgs_mlp_load)");
            A.mlp = 1;
            A.W = warm_args<R>(s, 1, nullptr);
            A.W.C = s->n_contacts;
        } else {
            nbgs_status rc = run_mlp_prologue(s, 1, nullptr);
            if (rc != NBGS_OK) return rc;
        }
    }
    if (s->prm.solver == NBGS_SOLVER_PERSISTENT) {
        // scheduling units: blocks, or warps with NBGS_SWEEP_WARP_SYNC
        const bool warp = (s->prm.sweep_flags & NBGS_SWEEP_WARP_SYNC) && !(s->prm.sweep_flags & NBGS_SWEEP_GLOBAL_SYNC);
        const int gk = gather_k(s->prm.sweep_flags);
        const void* fn = A.mlp ? (s->batch ? (const void*)k_solve_persistent<R, true, false, false, 1, true>
                                           : (const void*)k_solve_persistent<R, false, false, false, 1, true>)
                         : s->batch ? (warp      ? (const void*)k_solve_persistent<R, true, true, false>
                                     : gk == 2 ? (const void*)k_solve_persistent<R, true, false, false, 2>
                                               : (const void*)k_solve_persistent<R, true, false, false>)
                         : A.sub  ? (warp ? (const void*)k_solve_persistent<R, false, true, true>
                                          : (const void*)k_solve_persistent<R, false, false, true>)
                                  : (warp      ? (const void*)k_solve_persistent<R, false, true, false>
                                     : gk == 2 ? (const void*)k_solve_persistent<R, false, false, false, 2>
                                               : (const void*)k_solve_persistent<R, false, false, false>);
        // every block of a cooperative launch must be resident: variants that
        // hold more contacts per thread fit fewer blocks per SM
        const int nblocks = std::min(s->coop_blocks, persist_occ<R>(fn) * s->num_sms);
        if (nblocks < 1) return fail(s, NBGS_ECUDA, "solve: persistent kernel does not fit");
        const DCount Cn = contact_count(s);
        if (A.C > 0) {
            const int T = 256, B = nblocks * (warp ? kPersistThreads / 32 : 1);
            k_chunk_starts<<<grid_for((int64_t)kMaxColours * (B + 1), T, 8, s->num_sms), T, 0, st>>>(
                Cn, B, s->col_off, s->perm, s->info, s->cstart);
            if (s->timing) s->phase_launches[2] += 1;
            if (!(s->prm.sweep_flags & NBGS_SWEEP_GLOBAL_SYNC)) {
                // scratch free during the solve: the colouring's body degrees and the
                // detection's per-body counts (the body offsets adj_off stay: the
                // network's features read them in the kernel's prologue)
                int* dmin = (int*)s->deg;
                int* dmax = (int*)s->row_cnt;
                cudaMemsetAsync(dmin, 0x7F, s->n * sizeof(int), st);   // large positive
                cudaMemsetAsync(dmax, 0x80, s->n * sizeof(int), st);   // large negative
                k_body_blocks<<<grid_for(A.C, T, 8, s->num_sms), T, 0, st>>>(Cn, s->n, B, s->perm, s->cj1, s->cj2,
                                                                              s->row_off, s->finite, dmin, dmax);
                k_chunk_windows<<<B, T, 0, st>>>(Cn, s->n, s->cstart, s->perm, s->cj1, s->cj2, s->row_off,
                                                  s->finite, dmin, dmax, s->info, s->dep);
                cudaMemsetAsync(s->prog, 0xFF, B * sizeof(int), st);
                if (s->timing) s->phase_launches[2] += 2;
                if (A.sub && !warp) {
                    const int gs = grid_for(std::max<int64_t>(s->n, 1), T, 8, s->num_sms);
                    cudaMemsetAsync(s->rcount, 0, (B + 1) * sizeof(uint32_t), st);
                    cudaMemsetAsync(s->dep_r, 0, B * sizeof(int2), st);
                    k_reduce_count<<<gs, T, 0, st>>>(A.C, B, s->shared, s->info, s->row_off, dmin, dmax, s->rcount,
                                                     s->dep_r);
                    nbgs_status rc = exclusive_scan_u32(s, s->rcount, s->rstart, B, nullptr);
                    if (rc != NBGS_OK) return rc;
                    cudaMemsetAsync(s->rcount, 0, (B + 1) * sizeof(uint32_t), st);
                    k_reduce_fill<<<gs, T, 0, st>>>(A.C, B, s->shared, s->info, s->row_off, dmin, s->rstart,
                                                    s->rcount, s->rlist);
                    if (s->timing) s->phase_launches[2] += 5;
                }
            }
        }
        void* args[] = {&A};
        if (s->timing) cudaEventRecord(s->ev[8], st);
        size_t dyn = (s->prm.sweep_flags & NBGS_SWEEP_TMA_STAGE) ? Stage<R>::BYTES : 0;
        if (A.mlp) dyn = std::max(dyn, sizeof(TcMlpSmem));
        cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(s->coop_threads), args, dyn, st);
        if (s->timing) {
            cudaEventRecord(s->ev[9], st);
            s->phase_launches[2] += 1;
            s->sweep_launches += 1;
        }
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
    if (s->timing) cudaEventRecord(s->ev[8], st);
    const int gi = grid_for(std::max<int64_t>(s->n, 1), T, 8, s->num_sms);   // shared bodies <= n
    k_gravity<R><<<grid_for(s->n, T, 8, s->num_sms), T, 0, st>>>(A);
    if (A.sub) k_inst_init<R><<<gi, T, 0, st>>>(A);
    if (A.warm) {
        for (uint32_t c = 0; c < ncol; ++c)
            k_relax_colour<R, true><<<grid_for(A.C, T, 8, s->num_sms), T, 0, st>>>(A, (int)c, 0);
        if (A.sub) k_inst_reduce<R><<<gi, T, 0, st>>>(A, 0);
    }
    for (int k = 0; k < max_sweeps; ++k) {
        for (uint32_t c = 0; c < ncol; ++c)
            k_relax_colour<R, false><<<grid_for(A.C, T, 8, s->num_sms), T, 0, st>>>(A, (int)c, k);
        if (A.sub) k_inst_reduce<R><<<gi, T, 0, st>>>(A, 1);
        k_sweep_done<R><<<1, 32, 0, st>>>(A, k);
    }
    if (s->timing) {
        cudaEventRecord(s->ev[9], st);
        const int64_t l = 1 + (A.warm ? ncol : 0) + (int64_t)max_sweeps * (ncol + 1) +
                          (A.sub ? 1 + (A.warm ? 1 : 0) + max_sweeps : 0);
        s->phase_launches[2] += l;
        s->sweep_launches += l;
    }
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
    nbgs_status rc = s->composite ? run_solve_comp(s, max_sweeps, tol)
                     : s->fp32    ? solve_impl<float>(s, max_sweeps, tol)
                                  : solve_impl<double>(s, max_sweeps, tol);
    if (rc != NBGS_OK) return rc;
    if (s->timing) cudaEventRecord(s->ev[5], st);
    const int64_t C = s->n_contacts;
    if (C > 0) {
        const int T = 256;
        if (s->fp32)
            k_finish<float><<<grid_for(C, T, 8, s->num_sms), T, 0, st>>>(contact_count(s), s->perm_in, (const float4*)s->sp, s->cgeo,
                                                                         s->cimp, s->cworld);
        else
            k_finish<double><<<grid_for(C, T, 8, s->num_sms), T, 0, st>>>(contact_count(s), s->perm_in, (const double4_32a*)s->sp, s->cgeo,
                                                                          s->cimp, s->cworld);
    }
    if (C > 0 && !s->composite)
        k_count_updates<<<s->batch ? grid_for(C, 256, 8, s->num_sms) : 1, 256, 0, st>>>(
            contact_count(s), max_sweeps, s->perm, s->cj1, scene_view(s), s->scene_done, s->info);
    else if (C > 0)
        k_count_updates<<<1, 32, 0, st>>>(contact_count(s), max_sweeps, s->perm, s->cj1, scene_view(s), nullptr,
                                          s->info);
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
                                  double beta, double mu_all, SceneView V, const DevInfo* info, unsigned long long* out)
{
    double m[4] = {0, 0, 0, 0};
    const double vr_all = info->v_ref > 0.0 ? info->v_ref : 1e-12;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = cj1[c], b = cj2[c];
        const double vr = V.batch ? V.vref[V.scene_of[a]] : vr_all;
        const double mu = V.batch ? V.mu[V.scene_of[a]] : mu_all;
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
                s->prm.mu, scene_view(s), s->info, slots);
        else
            k_final_residuals<double><<<grid_for(C, T, 8, s->num_sms), T, 0, st>>>(
                C, s->n, s->cj1, s->cj2, s->cgeo, s->clev, s->cimp, (const double4_32a*)s->vel, s->prm.dt, s->prm.beta,
                s->prm.mu, scene_view(s), s->info, slots);
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
// Smallest occupancy over the variants a scene may launch (the single-scene
// ones: block or warp scheduling, with or without subdomains; the batched
// ones), with the shared-memory stage allowed.
template <class R>
static void persist_occupancy(int threads, int& occ, int& occ_b)
{
    const void* single[] = {(const void*)k_solve_persistent<R, false, false, false>,
                            (const void*)k_solve_persistent<R, false, true, false>,
                            (const void*)k_solve_persistent<R, false, false, true>,
                            (const void*)k_solve_persistent<R, false, true, true>};
    const void* batched[] = {(const void*)k_solve_persistent<R, true, false, false>,
                             (const void*)k_solve_persistent<R, true, true, false>};
    occ = occ_b = 1 << 30;
    const int dyn = (int)std::max<size_t>(Stage<R>::BYTES, sizeof(TcMlpSmem));   // TMA stage or network operands
    for (const void* f : single) {
        int o = 0;
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, f, threads, dyn);
        occ = std::min(occ, o);
    }
    for (const void* f : batched) {
        int o = 0;
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, f, threads, dyn);
        occ_b = std::min(occ_b, o);
    }
}

int persistent_blocks(nbgs_scene* s)
{
    int coop = 0, occ = 0, occ_b = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device);
    if (s->fp32) persist_occupancy<float>(s->coop_threads, occ, occ_b);
    else persist_occupancy<double>(s->coop_threads, occ, occ_b);
    if (s->batch) occ = occ_b;
    cudaGetLastError();
    if (!coop || occ < 1) {
        s->prm.solver = NBGS_SOLVER_PER_COLOUR;
        return 0;
    }
    return occ * s->num_sms;
}

}  // namespace nbgs
