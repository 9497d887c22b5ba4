// mlp_tc.cuh -- the warm-start network on the 5th-generation tensor cores
// (tcgen05), shared by its own kernels (mlp.cu) and by the prologue of the
// persistent sweep kernel (solve.cu): operand layouts, descriptors, the
// forward pass of a 128-row tile, and the 12 features of a contact.
#pragma once
#include <cuda_bf16.h>

#include "nbgs_internal.cuh"

namespace nbgs {

constexpr int kIn = 12, kHid = 64, kOutN = 3;
constexpr int kOffW1 = 0, kOffB1 = 768, kOffW2 = 832, kOffB2 = 4928, kOffW3 = 4992, kOffB3 = 9088, kOffW4 = 9152,
              kOffB4 = 9344, kNParams = 9347;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (low half) = lo
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + __expf(-z)); }
// the inference epilogue's SiLU (its result is rounded to BF16 anyway)
__device__ __forceinline__ float silu_fast(float z) { return __fdividef(z, 1.f + __expf(-z)); }

// --- the network on the 5th-generation tensor cores (tcgen05) ---------------
// A CTA of 128 threads evaluates 128 rows at a time, thread r owning row r.
// Operands live in shared memory in the K-major layout without swizzle:
// core matrices of 8 rows x 16 bytes (8 BF16), K-adjacent core matrices 128
// bytes apart (LBO), 8-row groups K/8 * 128 bytes apart (SBO).  One thread
// issues tcgen05.mma (M = 128, N = 64 or 16, K = 16 per instruction) into a
// 64-column TMEM accumulator and commits it to an mbarrier; each warp reads
// its 32 TMEM lanes (rows) back with tcgen05.ld, adds the bias, applies SiLU
// and writes the next layer's operand.  Every wait is bounded; TMEM is freed
// on every exit path.
constexpr int kTcRows = 128;
constexpr int kTcCols = 64;      // TMEM columns allocated per CTA

__device__ __forceinline__ uint32_t kmaj_off(int r, int k, int K)
{
    return (uint32_t)((r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

struct TcMlpSmem {
    alignas(128) __nv_bfloat16 x[kTcRows * 16];    // layer-1 operand (12 inputs + 4 zeros)
    alignas(128) __nv_bfloat16 h[kTcRows * kHid];  // hidden operand
    alignas(128) __nv_bfloat16 w1[kHid * 16];
    alignas(128) __nv_bfloat16 w2[kHid * kHid];
    alignas(128) __nv_bfloat16 w3[kHid * kHid];
    alignas(128) __nv_bfloat16 w4[16 * kHid];      // 3 outputs padded to N = 16
    float b1[kHid], b2[kHid], b3[kHid], b4[16];
    alignas(8) uint64_t bar;
    uint32_t tmem;
    int ok;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start >> 4, LBO >> 4, SBO >> 4, the fixed
// version bits (46..48 = 0b001), no base offset, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: F32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, int accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// Waits for the mbarrier phase with the given parity; false after ~2^31
// SM clocks (about a second).
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done = 0;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1LL << 31)) return false;
    }
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per thread).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// Weights into the operand layouts, biases, mbarrier, TMEM (warp 0).  All
// 128 threads; returns with the TMEM base in S.tmem.
static __device__ void tc_setup(const float* __restrict__ th, TcMlpSmem& S)
{
    for (int e = threadIdx.x; e < kHid * 16; e += blockDim.x) {
        const int n = e / 16, k = e % 16;
        S.w1[kmaj_off(n, k, 16) / 2] = __float2bfloat16_rn(k < kIn ? th[kOffW1 + n * kIn + k] : 0.f);
    }
    for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
        const int n = e / kHid, k = e % kHid;
        S.w2[kmaj_off(n, k, kHid) / 2] = __float2bfloat16_rn(th[kOffW2 + n * kHid + k]);
        S.w3[kmaj_off(n, k, kHid) / 2] = __float2bfloat16_rn(th[kOffW3 + n * kHid + k]);
    }
    for (int e = threadIdx.x; e < 16 * kHid; e += blockDim.x) {
        const int n = e / kHid, k = e % kHid;
        S.w4[kmaj_off(n, k, kHid) / 2] = __float2bfloat16_rn(n < kOutN ? th[kOffW4 + n * kHid + k] : 0.f);
    }
    for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
        S.b1[k] = th[kOffB1 + k];
        S.b2[k] = th[kOffB2 + k];
        S.b3[k] = th[kOffB3 + k];
    }
    if (threadIdx.x < 16) S.b4[threadIdx.x] = threadIdx.x < kOutN ? th[kOffB4 + threadIdx.x] : 0.f;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.bar)) : "memory");
        S.ok = 1;
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&S.tmem)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // weights: generic stores -> MMA reads
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

static __device__ void tc_teardown(TcMlpSmem& S)
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem), "r"(kTcCols) : "memory");
    }
}

// One layer: MMAs over K (kk slices of 16) from operand a (K columns) and
// weights b (N rows), committed and waited for.  All threads; thread 0 issues.
__device__ __forceinline__ bool tc_layer(TcMlpSmem& S, const __nv_bfloat16* a, const __nv_bfloat16* b, int K, int N,
                                         uint32_t& phase)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // operand rows written by every thread
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sa = smem_addr(a), sb = smem_addr(b);
        const uint32_t idesc = tc_idesc(kTcRows, N);
        for (int kk = 0; kk < K / 16; ++kk)
            tc_mma(S.tmem, tc_desc(sa + 256u * kk, 128u, (uint32_t)(K / 8) * 128u),
                   tc_desc(sb + 256u * kk, 128u, (uint32_t)(K / 8) * 128u), idesc, kk > 0);
        tc_commit(&S.bar);
    }
    const bool ok = tc_wait(&S.bar, phase & 1u);
    phase += 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return __syncthreads_and(ok) != 0;   // the same answer on every thread
}

// Epilogue of a hidden layer: row r's 64 accumulators + bias, SiLU, BF16
// into the hidden operand.  Threads 0..127 (warps 0..3, whose TMEM lanes
// hold rows 0..127); further threads of a larger block have no row.
__device__ __forceinline__ void tc_hidden_out(TcMlpSmem& S, const float* bias)
{
    if (threadIdx.x >= kTcRows) return;
    const int r = threadIdx.x, w = threadIdx.x >> 5;
    const uint32_t lane_base = S.tmem + ((uint32_t)(32 * w) << 16);
    for (int c0 = 0; c0 < kHid; c0 += 16) {
        float v[16];
        tc_ld16(lane_base + (uint32_t)c0, v);
        uint32_t pk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            pk[j] = pack_bf16(silu_fast(v[2 * j] + bias[c0 + 2 * j]), silu_fast(v[2 * j + 1] + bias[c0 + 2 * j + 1]));
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(S.h) + kmaj_off(r, c0, kHid)) =
            make_uint4(pk[0], pk[1], pk[2], pk[3]);
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(S.h) + kmaj_off(r, c0 + 8, kHid)) =
            make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
}

// The network on this CTA's 128 rows: in = the thread's 12 inputs (zeros
// for an empty row), out = the 3 outputs before the skip connection; thread
// r < 128 owns row r, further threads of a larger block only take part in
// the barriers.  Returns false if a wait gave up (outputs undefined).
static __device__ bool tc_forward(TcMlpSmem& S, const float (&in)[kIn], float (&out)[kOutN], uint32_t& phase)
{
    const int r = threadIdx.x;
    if (r < kTcRows) {
        uint32_t pk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float lo = 2 * j < kIn ? in[2 * j] : 0.f, hi = 2 * j + 1 < kIn ? in[2 * j + 1] : 0.f;
            pk[j] = pack_bf16(lo, hi);
        }
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(S.x) + kmaj_off(r, 0, 16)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(S.x) + kmaj_off(r, 8, 16)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
    bool ok = tc_layer(S, S.x, S.w1, 16, kHid, phase);
    if (ok) tc_hidden_out(S, S.b1);
    // the next MMA reads S.h and overwrites the accumulator: every thread has
    // finished its tcgen05.ld (waited) and its stores before the barrier in tc_layer
    ok = ok && tc_layer(S, S.h, S.w2, kHid, kHid, phase);
    if (ok) tc_hidden_out(S, S.b2);
    ok = ok && tc_layer(S, S.h, S.w3, kHid, kHid, phase);
    if (ok) tc_hidden_out(S, S.b3);
    ok = ok && tc_layer(S, S.h, S.w4, kHid, 16, phase);
    if (ok && r < kTcRows) {
        float v[16];
        tc_ld16(S.tmem + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16), v);
#pragma unroll
        for (int k = 0; k < kOutN; ++k) out[k] = v[k] + S.b4[k];
    }
    return ok;
}

// --- the warm-start prologue of a solve ---------------------------------------
template <class R> struct WarmArgs {
    int64_t C, n;
    const SweepRec<R>* rec;
    R4<R>* p;                    // in: previous-step warm start (n, t, o); out: network's impulse
    const R4<R>* vel;
    const double4_32a* pos_r;
    const uint32_t* adj_off;     // contacts per finite body = adj_off[i + 1] - adj_off[i]
    const uint8_t* finite;
    const float* theta;
    const uint32_t* perm;
    const uint32_t *cj1, *cj2;   // canonical bodies (j2 >= n: a wall)
    const double4_32a* cgeo;     // canonical (n, xi)
    float* feat_out;             // optional: canonical order, 16 per contact (12 features, cos, sin, w_n, v_ref)
    int apply;                   // 0: features only
    double gdt[3];
    double gdt_norm;
    double dt;
    double mu;
    SceneView V;
    DevInfo* info;
};

// Features of sweep slot s (see the top of this file) and what applying the
// network's output needs: the frame angle (cth, sth), w_n, v_ref, mu and the
// previous-step impulse (p0.w != 0: the contact existed in the last step).
template <class R> struct ContactFeatures {
    float f[kIn];
    double cth, sth, wn, vr, mu;
    R4<R> p0;
};

template <class R>
static __device__ void contact_features(const WarmArgs<R>& A, int64_t s, double vr_all, ContactFeatures<R>& F)
{
    double nx, ny, nz, tx, ty, tz, ox, oy, oz;
    const SweepRec<R> rr = A.rec[s];
    // the bodies themselves (the record may name subdomain instances, which
    // all hold the body's velocity before the sweeps)
    const uint32_t c = A.perm[s];
    const uint32_t ia = A.cj1[c], ib = A.cj2[c];
    double la, lb;
    if constexpr (sizeof(R) == 4) {
        la = rr.a.z;
        lb = rr.a.w;
        nx = rr.b.x;
        ny = rr.b.y;
        nz = rr.b.z;
    } else {
        la = rr.lev.x;
        lb = rr.lev.y;
        nx = rr.nxy.x;
        ny = rr.nxy.y;
        nz = rr.nz_.x;
    }
    F.p0 = A.p[s];
    const bool dyn_b = ib < (uint64_t)A.n;
    const R4<R> va = A.vel[2 * (int64_t)ia], wa = A.vel[2 * (int64_t)ia + 1];
    R4<R> vb, wb;
    vb.x = vb.y = vb.z = vb.w = R(0);
    wb = vb;
    if (dyn_b) {
        vb = A.vel[2 * (int64_t)ib];
        wb = A.vel[2 * (int64_t)ib + 1];
    }
    F.mu = A.mu;
    if (A.V.batch) {
        const uint32_t sc = A.V.scene_of[ia];
        F.vr = A.V.vref[sc];
        F.mu = A.V.mu[sc];
    } else {
        F.vr = vr_all;
    }
    const double vr = F.vr;
    const double ka = va.w > R(0) ? 1.0 : 0.0, kb = vb.w > R(0) ? 1.0 : 0.0;   // gravity kick of finite masses
    const double vax = va.x + ka * A.gdt[0], vay = va.y + ka * A.gdt[1], vaz = va.z + ka * A.gdt[2];
    const double vbx = vb.x + kb * A.gdt[0], vby = vb.y + kb * A.gdt[1], vbz = vb.z + kb * A.gdt[2];
    const double cax = wa.y * nz - wa.z * ny, cay = wa.z * nx - wa.x * nz, caz = wa.x * ny - wa.y * nx;
    const double cbx = wb.y * nz - wb.z * ny, cby = wb.z * nx - wb.x * nz, cbz = wb.x * ny - wb.y * nx;
    const double ux = (vax - la * cax) - (vbx + lb * cbx);
    const double uy = (vay - la * cay) - (vby + lb * cby);
    const double uz = (vaz - la * caz) - (vbz + lb * cbz);
    tangent_basis<double>(nx, ny, nz, tx, ty, tz, ox, oy, oz);
    const double un = nx * ux + ny * uy + nz * uz;
    const double ut = tx * ux + ty * uy + tz * uz, uo = ox * ux + oy * uy + oz * uz;
    const double utl = sqrt(ut * ut + uo * uo);
    F.cth = 1.0;
    F.sth = 0.0;
    if (utl > 1e-12 * vr) {   // e2 = -u_t / |u_t| = cos t + sin o
        F.cth = -ut / utl;
        F.sth = -uo / utl;
    }
    const double wn = (double)va.w + (double)vb.w;
    F.wn = wn;
    const double wt = wn + (double)wa.w * la * la + (double)wb.w * lb * lb;
    // previous impulse in (n, e2, e3): e3 = -sin t + cos o
    const double q2 = F.p0.y * F.cth + F.p0.z * F.sth, q3 = -F.p0.y * F.sth + F.p0.z * F.cth;
    const double sc = wn / vr;
    const double ra = A.pos_r[ia].w, rb = dyn_b ? A.pos_r[ib].w : 0.0;
    const uint32_t da = A.finite[ia] ? A.adj_off[ia + 1] - A.adj_off[ia] : 0;
    const uint32_t db = (dyn_b && A.finite[ib]) ? A.adj_off[ib + 1] - A.adj_off[ib] : 0;
    const uint32_t cidx = A.perm[s];
    const double xi_dt = A.cgeo[cidx].w / A.dt;   // the geometric gap, not the beta-scaled term
    const double f[kIn] = {un / vr,   utl / vr,      xi_dt / vr,      F.p0.x * sc, q2 * sc, q3 * sc,
                           log(fmax(wn, 1e-300)),    wt / wn, ra,     rb,          F.mu,    (double)(da + db) / 12.0};
#pragma unroll
    for (int k = 0; k < kIn; ++k) F.f[k] = (float)f[k];
    if (A.feat_out) {
        float* o = A.feat_out + (int64_t)cidx * 16;
        for (int k = 0; k < kIn; ++k) o[k] = F.f[k];
        o[12] = (float)F.cth;
        o[13] = (float)F.sth;
        o[14] = (float)wn;
        o[15] = (float)vr;
    }
}


// The warm start of the current contacts, 128 sweep slots per tile, thread
// r < 128 the slot of row r (a larger block's further threads only join
// the barriers).  With S, the network runs on the tensor cores and a contact
// without a previous-step impulse takes its prediction (previous impulse +
// network correction, in the frame and scale of the features, projected
// onto the friction cone); the others keep theirs, as does a non-finite
// output.  Without S only the features are computed (and written out when
// A.feat_out is set).  A tensor-core wait that gives up sets the timeout
// bit and leaves the remaining impulses as they are.
template <class R>
static __device__ __noinline__ void warm_tiles(const WarmArgs<R>& A, TcMlpSmem* S)
{
    if (S) tc_setup(A.theta, *S);
    const double vr_all = fmax(fmax(__longlong_as_double((long long)A.info->vmax_bits), A.gdt_norm), 1e-12);
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t base = (int64_t)blockIdx.x * kTcRows; base < A.C; base += (int64_t)gridDim.x * kTcRows) {
        const int64_t s = base + threadIdx.x;
        const bool live = threadIdx.x < kTcRows && s < A.C;
        ContactFeatures<R> F;
        if (live) {
            contact_features<R>(A, s, vr_all, F);
        } else {
#pragma unroll
            for (int k = 0; k < kIn; ++k) F.f[k] = 0.f;
            F.p0.w = R(1);
        }
        if (!S || !ok) continue;   // both uniform over the CTA
        float out[kOutN];
        if (!tc_forward(*S, F.f, out, phase)) {
            ok = false;
            if (threadIdx.x == 0) atomicOr(&A.info->err, kErrTimeout);
            continue;
        }
        if (live && F.p0.w == R(0)) {
            const double k = F.vr / F.wn;   // skip connection: previous impulse + network correction
            const double y1 = ((double)out[0] + F.f[3]) * k;
            const double y2 = ((double)out[1] + F.f[4]) * k;
            const double y3 = ((double)out[2] + F.f[5]) * k;
            double pn = y1, pt = y2 * F.cth - y3 * F.sth, po = y2 * F.sth + y3 * F.cth;
            if (isfinite(pn) && isfinite(pt) && isfinite(po)) {   // otherwise keep the previous-step impulse
                pn = pn > 0.0 ? pn : 0.0;
                const double lim = F.mu * pn, len = sqrt(pt * pt + po * po);
                if (len > lim) {
                    const double f = len > 0.0 ? lim / len : 0.0;
                    pt *= f;
                    po *= f;
                }
                R4<R> q;
                q.x = (R)pn;
                q.y = (R)pt;
                q.z = (R)po;
                q.w = R(0);
                A.p[s] = q;
            }
        }
    }
    if (S) tc_teardown(*S);
}

template <class R>
inline WarmArgs<R> warm_args(nbgs_scene* s, int apply, float* feat_out)
{
    WarmArgs<R> A;
    A.C = s->n_contacts;
    A.n = s->n;
    A.rec = (const SweepRec<R>*)s->srec;
    A.p = (R4<R>*)s->sp;
    A.vel = (const R4<R>*)s->vel;
    A.pos_r = s->pos_r;
    A.adj_off = s->adj_off;
    A.finite = s->finite;
    A.theta = s->mlp_theta;
    A.perm = s->perm;
    A.cj1 = s->cj1;
    A.cj2 = s->cj2;
    A.cgeo = s->cgeo;
    A.feat_out = feat_out;
    A.apply = apply;
    for (int k = 0; k < 3; ++k) A.gdt[k] = s->prm.dt * s->prm.gravity[k];
    const double* g = s->prm.gravity;
    A.gdt_norm = sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]) * s->prm.dt;
    A.dt = s->prm.dt;
    A.mu = s->prm.mu;
    A.V = scene_view(s);
    A.info = s->info;
    return A;
}

}  // namespace nbgs
