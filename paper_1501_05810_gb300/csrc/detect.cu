// detect.cu -- contact detection (Sect. 4) on a uniform cell grid.
//
// Per step:
//   k_hull          h_i = dt(|v_i| + |w_i| r_i) + tau       eq. (expansionradius)
//                   + max h, max |v| (for the cell size and v_ref)
//   k_grid_setup    cell width >= 2 (r_max + h_max), dims per axis
//   k_cell_keys     linear cell index of every body
//   radix sort      (cell, body) pairs, LSD, 8-bit digits, stable
//   scan            first sorted slot of every cell, from the cell counts
//   k_gather_sorted FP32 positions in cell order
//   k_narrow        per body i: bodies j > i in the 27 neighbour cells whose
//                   hulls intersect, sorted by j; wall hull tests
//   scan            contacts per body -> CSR offsets by j1
//   k_write         canonical contact records (n, xi, lever lengths)
//                   for sphere-sphere and sphere-wall pairs, eq. (contactpos)
#include <algorithm>
#include <cmath>
#include <utility>

#include "nbgs_internal.cuh"

namespace nbgs {

int grid_for(int64_t work, int threads, int max_blocks_per_sm, int num_sms)
{
    int64_t b = (work + threads - 1) / threads;
    int64_t cap = (int64_t)max_blocks_per_sm * (num_sms > 0 ? num_sms : 1);
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// ---------------------------------------------------------------------------
// exclusive scan of u32 (reduce -> scan block sums -> downsweep)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Exclusive block scan of one value per thread; returns the block total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t& excl)
{
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t block_tot;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane < nw ? warp_tot[lane] : 0;
        uint32_t ti = warp_incl_scan(t);
        if (lane < nw) warp_tot[lane] = ti - t;
        if (lane == nw - 1) block_tot = ti;
    }
    __syncthreads();
    excl = warp_tot[wid] + inc - v;
    uint32_t total = block_tot;
    __syncthreads();
    return total;
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, DCount nc, uint32_t* __restrict__ sums)
{
    const int64_t n = nc.get();
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) acc += in[i];
    }
    uint32_t excl;
    uint32_t tot = block_excl_scan(acc, excl);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_top(uint32_t* sums, int64_t nb)
{
    // single block: exclusive scan of the block sums in chunks
    uint32_t carry = 0;
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        uint32_t v = i < nb ? sums[i] : 0;
        uint32_t excl;
        uint32_t tot = block_excl_scan(v, excl);
        if (i < nb) sums[i] = carry + excl;
        carry += tot;
    }
}

__global__ void k_scan_down(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, DCount nc,
                            const uint32_t* __restrict__ sums, uint32_t* __restrict__ total_dst)
{
    __shared__ uint32_t tile[kScanTile];
    const int64_t n = nc.get();   // tiles past n hold zeros: the last block's total is the total
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        tile[k * kScanThreads + threadIdx.x] = i < n ? in[i] : 0;
    }
    __syncthreads();
    uint32_t loc[kScanItems];
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = acc;
        acc += tile[threadIdx.x * kScanItems + k];
    }
    uint32_t excl;
    uint32_t tot = block_excl_scan(acc, excl);
    const uint32_t off = sums[blockIdx.x] + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) tile[threadIdx.x * kScanItems + k] = loc[k] + off;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) out[i] = tile[k * kScanThreads + threadIdx.x];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        uint32_t total = sums[blockIdx.x] + tot;
        out[n] = total;
        if (total_dst) *total_dst = total;
    }
}

// out must hold n + 1 entries; out[n] receives the total (also *total_dst).
// A device-read count: the launch covers n.v entries (the capacity).
nbgs_status exclusive_scan_u32(nbgs_scene* s, const uint32_t* in, uint32_t* out, DCount n, uint32_t* total_dst)
{
    int64_t nb = (n.v + kScanTile - 1) / kScanTile;
    if (nb < 1) nb = 1;
    if (nb > s->scan_tmp_len) return fail(s, NBGS_EINVAL, "scan: block-sum buffer too small");
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s->stream>>>(in, n, s->scan_tmp);
    k_scan_top<<<1, 1024, 0, s->stream>>>(s->scan_tmp, nb);
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, s->stream>>>(in, out, n, s->scan_tmp, total_dst);
    return cuda_check(s, cudaGetLastError(), "scan");
}

nbgs_status exclusive_scan_u32(nbgs_scene* s, const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dst)
{
    return exclusive_scan_u32(s, in, out, DCount{n, nullptr}, total_dst);
}

// ---------------------------------------------------------------------------
// LSD radix sort of (key, value) u32 pairs: 8-bit digits, one pass =
// per-tile digit histogram -> scan (digit-major) -> stable scatter with
// warp-level ranking (__match_any_sync), so equal keys keep input order.
// ---------------------------------------------------------------------------
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 16;
constexpr int kRadixTile = kRadixThreads * kRadixItems;   // 4096
constexpr int kWarps = kRadixThreads / 32;

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, DCount nc, int shift, uint32_t* __restrict__ hist,
                             int64_t nblocks)
{
    __shared__ uint32_t h[256];
    const int64_t n = nc.get();
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
#pragma unroll 4
    for (int k = 0; k < kRadixItems; ++k) {
        int64_t i = base + (int64_t)k * kRadixThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kRadixThreads)
k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
                uint32_t* __restrict__ vout, DCount nc, int shift, const uint32_t* __restrict__ hist_scan,
                int64_t nblocks)
{
    const int64_t n = nc.get();
    __shared__ uint32_t cnt[kWarps][256];
    __shared__ uint32_t goff[256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < 256; d += kRadixThreads) {
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) cnt[ww][d] = 0;
        goff[d] = hist_scan[(int64_t)d * nblocks + blockIdx.x];
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kRadixTile + (int64_t)w * (kRadixItems * 32);
    uint32_t key[kRadixItems], val[kRadixItems], rank[kRadixItems];
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool valid = i < n;
        key[r] = valid ? kin[i] : 0u;
        val[r] = valid ? vin[i] : 0u;
        const uint32_t d = (key[r] >> shift) & 255u;
        const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 0x100u);
        const uint32_t before = cnt[w][d & 255u];
        __syncwarp();
        if (valid && (peers & lt) == 0) cnt[w][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    // exclusive prefix of each digit over the warps (warp order = input order)
    for (int d = threadIdx.x; d < 256; d += kRadixThreads) {
        uint32_t sum = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            uint32_t t = cnt[ww][d];
            cnt[ww][d] = sum;
            sum += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const int64_t i = base + r * 32 + lane;
        if (i < n) {
            const uint32_t d = (key[r] >> shift) & 255u;
            const uint32_t pos = goff[d] + cnt[w][d] + rank[r];
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

nbgs_status radix_sort_pairs(nbgs_scene* s, uint32_t*& keys, uint32_t*& vals, uint32_t*& keys_alt,
                             uint32_t*& vals_alt, DCount n, int bits)
{
    if (!n.dev && n.v <= 1) return NBGS_OK;
    const int64_t nb = std::max<int64_t>((n.v + kRadixTile - 1) / kRadixTile, 1);
    if (256 * nb > s->radix_hist_len) return fail(s, NBGS_EINVAL, "radix sort: histogram buffer too small");
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<(unsigned)nb, kRadixThreads, 0, s->stream>>>(keys, n, shift, s->radix_hist, nb);
        nbgs_status st = exclusive_scan_u32(s, s->radix_hist, s->radix_hist, 256 * nb, nullptr);
        if (st != NBGS_OK) return st;
        k_radix_scatter<<<(unsigned)nb, kRadixThreads, 0, s->stream>>>(keys, vals, keys_alt, vals_alt, n, shift,
                                                                       s->radix_hist, nb);
        uint32_t* t = keys;
        keys = keys_alt;
        keys_alt = t;
        t = vals;
        vals = vals_alt;
        vals_alt = t;
        if (s->timing) s->phase_launches[0] += 4;
    }
    return cuda_check(s, cudaGetLastError(), "radix sort");
}

nbgs_status radix_sort_pairs(nbgs_scene* s, uint32_t*& keys, uint32_t*& vals, uint32_t*& keys_alt,
                             uint32_t*& vals_alt, int64_t n, int bits)
{
    return radix_sort_pairs(s, keys, vals, keys_alt, vals_alt, DCount{n, nullptr}, bits);
}

// ---------------------------------------------------------------------------
// detection kernels
// ---------------------------------------------------------------------------
struct GridArgs {
    double lo[3], hi[3];
    int periodic[3];
    int dims_max[3];
    double r_max, dt, tau;
    float Lf[3];         // box extents in FP32
    float margin;        // FP32 pre-filter margin: 1e-4 + 1e-6 max(L)
    double pos_err;      // bound on the error of an FP32 relative position (2^-22 max(L))
    // FP32 wall pre-filter: plane k as n . (x - lo) + pc[k] (= n . x - c),
    // margin 1e-4 + 4e-6 (max(L) + max |pc|)
    float pn[kMaxPlanes][3];
    float pc[kMaxPlanes];
    float tauf, wmargin;
    // FP32 cone pre-filter: apex relative to lo, axis, sin, cos, s_o, s_t;
    // margin 1e-4 + 1e-5 (max(L) + max |apex - lo|)
    float ca_apex[kMaxCones][3], ca_axis[kMaxCones][3], ca_sc[kMaxCones][4];
    float cmargin;
};

__device__ __forceinline__ double norm_exact(double x, double y, double z)
{
    return xsqrt(xadd(xadd(xmul(x, x), xmul(y, y)), xmul(z, z)));
}

// a / b rounded to nearest, given y = 1/b rounded to nearest: the quotient
// q = RN(a y) is within one ulp of a / b, the remainder a - b q is exact in
// one fused multiply-add, and RN(q + (a - b q) y) is the correctly rounded
// quotient (Markstein's theorem, IBM J. Res. Dev. 34(1), 1990; Muller et
// al., Handbook of Floating-Point Arithmetic, the chapter on division with
// an FMA).  The theorem excludes underflow: zeros and tiny numerators take
// the division itself, as does the caller for a tiny or huge b.
__device__ __forceinline__ double div_by(double a, double b, double y)
{
    if (fabs(a) < 0x1p-900) return xdiv(a, b);
    const double q = __dmul_rn(a, y);
    const double r = __fma_rn(-q, b, a);
    return __fma_rn(r, y, q);
}

// Sphere pair geometry of eq. (contactpos) from the centre difference
// (dx, dy, dz) = x_i - x_j: d = |x_i - x_j| and the unit normal
// n = (x_i - x_j) / d, every operation rounded to nearest as written (the
// three quotients share one correctly rounded reciprocal of d); coincident
// centres take n = (0, 0, 1).
__device__ __forceinline__ double pair_normal(double dx, double dy, double dz, double n[3])
{
    const double d = norm_exact(dx, dy, dz);
    if (d > 0x1p-1000 && d < 0x1p1000) {
        const double y = __drcp_rn(d);
        n[0] = div_by(dx, d, y);
        n[1] = div_by(dy, d, y);
        n[2] = div_by(dz, d, y);
    } else if (d > 0.0) {
        n[0] = xdiv(dx, d);
        n[1] = xdiv(dy, d);
        n[2] = xdiv(dz, d);
    } else {
        n[0] = 0.0;
        n[1] = 0.0;
        n[2] = 1.0;
    }
    return d;
}

// Composite particles: the members' world positions X + R(q) d (FP64, each
// operation rounded as written: the contact geometry depends on them bit for
// bit), their bodies' hulls h = dt (|v| + |w| r_bound) + tau (eq.
// expansionradius with the bounding radius) and the FP32 copies for the cell
// grid, wrapped into the box on periodic axes (the FP64 positions stay
// unwrapped; the exact tests take minimum images of differences).
template <class R>
__global__ void k_member_update(int64_t n, const uint32_t* __restrict__ mbody, const double4_32a* __restrict__ moff,
                                const double4_32a* __restrict__ bpos, const double4_32a* __restrict__ bquat,
                                const R4<R>* __restrict__ bvel, double dt, double tau,
                                double4_32a* __restrict__ pos_r, double* __restrict__ hull, float4* __restrict__ p32,
                                GridArgs g, DevInfo* info)
{
    double hmax = 0.0, vmax = 0.0;
    bool bad = false;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = mbody[m];
        const double4_32a X = ld_d4(bpos + b), q = ld_d4(bquat + b), d = ld_d4(moff + m);
        const R4<R> v = bvel[4 * (int64_t)b], w = bvel[4 * (int64_t)b + 1];
        // R(q) rows, as 1 - 2 (y^2 + z^2), 2 (xy - wz), ... (unit quaternion)
        const double qw = q.x, qx = q.y, qy = q.z, qz = q.w;
        const double r00 = xsub(1.0, xmul(2.0, xadd(xmul(qy, qy), xmul(qz, qz))));
        const double r01 = xmul(2.0, xsub(xmul(qx, qy), xmul(qw, qz)));
        const double r02 = xmul(2.0, xadd(xmul(qx, qz), xmul(qw, qy)));
        const double r10 = xmul(2.0, xadd(xmul(qx, qy), xmul(qw, qz)));
        const double r11 = xsub(1.0, xmul(2.0, xadd(xmul(qx, qx), xmul(qz, qz))));
        const double r12 = xmul(2.0, xsub(xmul(qy, qz), xmul(qw, qx)));
        const double r20 = xmul(2.0, xsub(xmul(qx, qz), xmul(qw, qy)));
        const double r21 = xmul(2.0, xadd(xmul(qy, qz), xmul(qw, qx)));
        const double r22 = xsub(1.0, xmul(2.0, xadd(xmul(qx, qx), xmul(qy, qy))));
        double4_32a p;
        p.x = xadd(X.x, xadd(xadd(xmul(r00, d.x), xmul(r01, d.y)), xmul(r02, d.z)));
        p.y = xadd(X.y, xadd(xadd(xmul(r10, d.x), xmul(r11, d.y)), xmul(r12, d.z)));
        p.z = xadd(X.z, xadd(xadd(xmul(r20, d.x), xmul(r21, d.y)), xmul(r22, d.z)));
        p.w = d.w;
        st_d4(pos_r + m, p);
        const double nv = norm_exact((double)v.x, (double)v.y, (double)v.z);
        const double nw = norm_exact((double)w.x, (double)w.y, (double)w.z);
        const double h = xadd(xmul(dt, xadd(nv, xmul(nw, X.w))), tau);
        hull[m] = h;
        double rel[3] = {p.x - g.lo[0], p.y - g.lo[1], p.z - g.lo[2]};
        for (int a = 0; a < 3; ++a) {
            const double L = g.hi[a] - g.lo[a];
            if (g.periodic[a] && !(rel[a] >= 0.0 && rel[a] < L)) {
                double sft = fmod(rel[a], L);
                if (sft < 0.0) sft += L;
                rel[a] = sft;
            }
        }
        p32[m] = make_float4((float)rel[0], (float)rel[1], (float)rel[2], (float)(p.w + h));
        if (!(h <= 1e300)) bad = true;
        hmax = fmax(hmax, h);
        vmax = fmax(vmax, nv);
    }
    __shared__ double sh[2][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        hmax = fmax(hmax, __shfl_down_sync(0xffffffffu, hmax, o));
        vmax = fmax(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
    }
    if (lane == 0) {
        sh[0][wid] = hmax;
        sh[1][wid] = vmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            hmax = fmax(hmax, sh[0][k]);
            vmax = fmax(vmax, sh[1][k]);
        }
        atomicMax(&info->hmax_bits, (unsigned long long)__double_as_longlong(hmax));
        atomicMax(&info->vmax_bits, (unsigned long long)__double_as_longlong(vmax));
    }
    if (bad) atomicOr(&info->err, kErrNaN);
}

// Hull radius of eq. (expansionradius), h = dt (|v| + |w| r) + tau, rounded
// as the FP64 step computes it: for a sphere from the squares of |v| and |w|
// stored by k_hull (so that only the contacts that need the exact value pay
// for its two square roots), for a composite member from the member hulls.
struct HullView {
    const double* hull;   // member hulls (composites), else null
    const double2* vw;    // |v|^2, |w|^2 per sphere
    double dt, tau;
};
__device__ __forceinline__ double hull_of(const HullView& H, uint32_t x, double r)
{
    if (H.hull) return H.hull[x];
    const double2 q = H.vw[x];
    return xadd(xmul(H.dt, xadd(xsqrt(q.x), xmul(xsqrt(q.y), r))), H.tau);
}

// Per sphere: |v|^2 and |w|^2 in FP64 (the exact hull's inputs), the FP32
// position relative to the box corner and the reach r + h with h in FP32
// (cell keys and the narrow phase's screens run on these; the FP32 hull is
// within 5e-7 of h relative, inside the screens' margins), an upper bound
// of the largest hull for the grid, and max |v| (v_ref) exactly: the
// square root of the largest |v|^2, square roots being monotone.
template <class R>
__global__ void k_hull(int64_t n, const R4<R>* __restrict__ vel, const double4_32a* __restrict__ pos_r, double dt,
                       double tau, double2* __restrict__ vw, float4* __restrict__ p32, GridArgs g, DevInfo* info,
                       const uint32_t* __restrict__ scene_of, unsigned long long* __restrict__ scene_vmax)
{
    double hmax = 0.0, v2max = 0.0;
    bool bad = false;
    const float dtf = (float)dt, tauf = (float)tau;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        R4<R> v, w;
        ld_body(vel + 2 * i, v, w);
        const double4_32a x = ld_d4(pos_r + i);
        const double r = x.w;
        const double vx = v.x, vy = v.y, vz = v.z, wx = w.x, wy = w.y, wz = w.z;
        const double v2 = xadd(xadd(xmul(vx, vx), xmul(vy, vy)), xmul(vz, vz));
        const double w2 = xadd(xadd(xmul(wx, wx), xmul(wy, wy)), xmul(wz, wz));
        vw[i] = make_double2(v2, w2);
        const float h32 = dtf * (sqrtf((float)v2) + sqrtf((float)w2) * (float)r) + tauf;
        p32[i] = make_float4((float)(x.x - g.lo[0]), (float)(x.y - g.lo[1]), (float)(x.z - g.lo[2]),
                             (float)(r + (double)h32));
        if (!(v2 <= 1e300) || !(w2 <= 1e300)) bad = true;
        if (scene_of) {   // per-scene max |v|^2 (v_ref); the filter only saves atomics
            unsigned long long* dst = scene_vmax + scene_of[i];
            const unsigned long long bits = (unsigned long long)__double_as_longlong(v2);
            if (bits > *(volatile unsigned long long*)dst) atomicMax(dst, bits);
        }
        hmax = fmax(hmax, (double)h32);
        v2max = fmax(v2max, v2);
    }
    // block max, then one atomic per block (non-negative doubles order like their bits)
    __shared__ double sh[2][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        hmax = fmax(hmax, __shfl_down_sync(0xffffffffu, hmax, o));
        v2max = fmax(v2max, __shfl_down_sync(0xffffffffu, v2max, o));
    }
    if (lane == 0) {
        sh[0][wid] = hmax;
        sh[1][wid] = v2max;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            hmax = fmax(hmax, sh[0][k]);
            v2max = fmax(v2max, sh[1][k]);
        }
        // the FP32 hulls are within 5e-7 of h relative: 1e-5 makes an upper bound
        atomicMax(&info->hmax_bits, (unsigned long long)__double_as_longlong(hmax * (1.0 + 1e-5)));
        atomicMax(&info->vmax_bits, (unsigned long long)__double_as_longlong(xsqrt(v2max)));
    }
    if (bad) atomicOr(&info->err, kErrNaN);
}

__global__ void k_grid_setup(GridArgs g, DevInfo* info)
{
    const double hmax = __longlong_as_double((long long)info->hmax_bits);
    // any kept pair has d <= r_a + r_b + h_a + h_b <= 2 (r_max + h_max); the
    // cell keys come from FP32 positions with error <= pos_err, so a cell at
    // least need + 4 pos_err wide keeps every such pair in adjacent cells
    const double need = 2.0 * (g.r_max + hmax) * (1.0 + 1e-9) + 4.0 * g.pos_err + 1e-300;
    uint32_t ncells = 1;
    for (int a = 0; a < 3; ++a) {
        const double L = g.hi[a] - g.lo[a];
        double dd = floor(L / need);
        int d = dd < 1.0 ? 1 : (dd > (double)g.dims_max[a] ? g.dims_max[a] : (int)dd);
        if (g.periodic[a] && d < 3) atomicOr(&info->err, kErrGrid);
        info->dims[a] = d;
        info->cell_w[a] = L / d;
        info->inv_wf[a] = (float)(d / L);
        ncells *= (uint32_t)d;
    }
    info->ncells = ncells;
}

__device__ __forceinline__ int cell_coord(float x, float inv_w, int d)
{
    const float f = floorf(x * inv_w);
    return f < 0.f ? 0 : (f > (float)(d - 1) ? d - 1 : (int)f);
}

// Cell key of every body, and the body count of every cell.
__global__ void k_cell_keys(int64_t n, const float4* __restrict__ p32, const DevInfo* __restrict__ info,
                            uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, uint32_t* __restrict__ cnt)
{
    const int d0 = info->dims[0], d1 = info->dims[1], d2 = info->dims[2];
    const float i0 = info->inv_wf[0], i1 = info->inv_wf[1], i2 = info->inv_wf[2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = p32[i];
        const int cx = cell_coord(p.x, i0, d0), cy = cell_coord(p.y, i1, d1), cz = cell_coord(p.z, i2, d2);
        const uint32_t k = ((uint32_t)cz * (uint32_t)d1 + (uint32_t)cy) * (uint32_t)d0 + (uint32_t)cx;
        keys[i] = k;
        vals[i] = (uint32_t)i;
        atomicAdd(&cnt[k], 1u);
    }
}

// The FP32 positions gathered into cell order, so that the narrow phase
// reads each cell's candidates contiguously.
__global__ void k_gather_sorted(int64_t n, const uint32_t* __restrict__ vals, const float4* __restrict__ p32,
                                float4* __restrict__ p32s)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        p32s[s] = p32[vals[s]];
}

// Minimum-image difference a - b along one axis (periodic: |d| <= L/2).
__device__ __forceinline__ double min_image(double d, int periodic, double L)
{
    if (periodic) {
        const double half = xmul(0.5, L);
        if (d > half) d = xsub(d, L);
        else if (d < -half) d = xadd(d, L);
    }
    return d;
}

// Distance from x to cone C, worked in the half-plane through the axis and
// x: zeta = height above the apex along the axis, rho = distance from the
// axis, e = unit radial direction.  A generatrix runs along (sin a, cos a)
// in (rho, zeta); the face is its segment s in [s_o, s_t], the solid lies
// outside, and the face's inward unit normal is (-cos a, sin a).  The foot
// of x on the generatrix is at s = rho sin a + zeta cos a.  Face:
// sd = zeta sin a - rho cos a, n = sin a axis - cos a e.  Below the face
// (s < s_o) the orifice rim (rho_o, zeta_o) = s_o (sin a, cos a) is
// nearest: sd = |(rho - rho_o, zeta - zeta_o)|, n along that difference.
// On the axis (rho = 0) the normal is the axis.  Returns 0 above the
// frustum (no contact), 1 on the face, 2 at the rim.  Every operation is
// rounded to nearest, in this order, so that the contact sets are exact.
__device__ __forceinline__ int cone_distance(const Cone& C, const double4_32a& x, double& sd, double n[3])
{
    const double d0 = xsub(x.x, C.apex[0]), d1 = xsub(x.y, C.apex[1]), d2 = xsub(x.z, C.apex[2]);
    const double zeta = xadd(xadd(xmul(d0, C.axis[0]), xmul(d1, C.axis[1])), xmul(d2, C.axis[2]));
    double e0 = xsub(d0, xmul(zeta, C.axis[0])), e1 = xsub(d1, xmul(zeta, C.axis[1])),
           e2 = xsub(d2, xmul(zeta, C.axis[2]));
    const double rho = xsqrt(xadd(xadd(xmul(e0, e0), xmul(e1, e1)), xmul(e2, e2)));
    const double sg = xadd(xmul(rho, C.sa), xmul(zeta, C.ca));
    if (sg > C.s_t) return 0;
    if (rho > 0.0) {
        e0 = xdiv(e0, rho);
        e1 = xdiv(e1, rho);
        e2 = xdiv(e2, rho);
    }
    if (sg >= C.s_o) {
        sd = xsub(xmul(zeta, C.sa), xmul(rho, C.ca));
        if (rho > 0.0) {
            n[0] = xsub(xmul(C.sa, C.axis[0]), xmul(C.ca, e0));
            n[1] = xsub(xmul(C.sa, C.axis[1]), xmul(C.ca, e1));
            n[2] = xsub(xmul(C.sa, C.axis[2]), xmul(C.ca, e2));
        } else {
            n[0] = C.axis[0];
            n[1] = C.axis[1];
            n[2] = C.axis[2];
        }
        return 1;
    }
    const double drho = xsub(rho, xmul(C.s_o, C.sa)), dzeta = xsub(zeta, xmul(C.s_o, C.ca));
    const double dist = xsqrt(xadd(xmul(drho, drho), xmul(dzeta, dzeta)));
    sd = dist;
    if (dist > 0.0 && rho > 0.0) {
        n[0] = xdiv(xadd(xmul(drho, e0), xmul(dzeta, C.axis[0])), dist);
        n[1] = xdiv(xadd(xmul(drho, e1), xmul(dzeta, C.axis[1])), dist);
        n[2] = xdiv(xadd(xmul(drho, e2), xmul(dzeta, C.axis[2])), dist);
    } else {
        n[0] = C.axis[0];
        n[1] = C.axis[1];
        n[2] = C.axis[2];
    }
    return 2;
}

// The same distance in FP32 from the relative position q (the pre-filter;
// the distance is continuous across the face/rim boundary, so a case taken
// differently under rounding changes it little).  Returns a huge value
// above the frustum.
__device__ __forceinline__ float cone_distance_f(const GridArgs& g, int k, const float4& q)
{
    const float d0 = q.x - g.ca_apex[k][0], d1 = q.y - g.ca_apex[k][1], d2 = q.z - g.ca_apex[k][2];
    const float* ax = g.ca_axis[k];
    const float sa = g.ca_sc[k][0], ca = g.ca_sc[k][1], so = g.ca_sc[k][2], st = g.ca_sc[k][3];
    const float zeta = d0 * ax[0] + d1 * ax[1] + d2 * ax[2];
    const float e0 = d0 - zeta * ax[0], e1 = d1 - zeta * ax[1], e2 = d2 - zeta * ax[2];
    const float rho = sqrtf(e0 * e0 + e1 * e1 + e2 * e2);
    const float sg = rho * sa + zeta * ca;
    if (sg > st + g.cmargin) return 3.0e38f;
    if (sg >= so) return zeta * sa - rho * ca;
    const float dr = rho - so * sa, dz = zeta - so * ca;
    return sqrtf(dr * dr + dz * dz);
}

__device__ __forceinline__ bool wall_kept(const double nrm[3], double c, double4_32a p, double h, double tau, double& sd,
                                          double& xi)
{
    sd = xsub(xadd(xadd(xmul(nrm[0], p.x), xmul(nrm[1], p.y)), xmul(nrm[2], p.z)), c);
    xi = xsub(sd, p.w);
    return xi <= xadd(h, tau);
}

// Per body i (visited in cell order for locality): hull-intersecting
// partners j > i from the 27 neighbour cells, sorted ascending; wall count.
// cs[c] is the first sorted slot of cell c for every cell (cs[ncells] = n),
// so the three cells x - 1 .. x + 1 of a (y, z) row are one contiguous
// range; a periodic image adds one constant shift to a whole range.
struct NarrowPair {
    uint32_t list[kCandCap];
    int cnt;
};

__device__ __forceinline__ void narrow_range(uint32_t t0, uint32_t t1, float sx, float sy, float sz, uint32_t i,
                                             uint32_t si, const float4& qi, const double4_32a& pi, double& hi_,
                                             const uint32_t* __restrict__ svals, const float4* __restrict__ p32s,
                                             const double4_32a* __restrict__ pos_r, const HullView& H,
                                             const GridArgs& g, const SceneView& V, double L0, double L1, double L2,
                                             NarrowPair& P)
{
    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t j = svals[t];
        const float4 qj = p32s[t];   // loaded with j: one dependent load fewer
        if (j <= i) continue;
        if (V.batch && V.scene_of[j] != si) continue;   // scenes never touch
        if (V.body_of && V.body_of[j] == V.body_of[i]) continue;   // members of one body never touch
        // Conservative FP32 screens (FP64 throughput is scarce on this GPU).
        // R = r_a + h_a + r_b + h_b bounds d for every kept pair.  The FP32
        // relative positions are off by at most pos_err per coordinate, the
        // periodic shift adds an ulp of L, so the FP32 distance is within
        // 1e-6 max(L) of d; the FP32 square and reach add relative errors
        // below 4e-7 and 1.2e-7, covered by the extra 1e-4 while R < ~100 (the FP32 hull's own error
        // included).
        // So (fl(R) + margin)^2 >= fl(d^2) for every kept pair, and
        // fl(d^2) < (fl(R) - margin)^2 only for pairs with d below R by more
        // than the FP64 keep rule's rounding: those are kept without it.
        // Only the pairs in the band between take the exact FP64 test.
        const float fx = (qi.x - qj.x) + sx, fy = (qi.y - qj.y) + sy, fz = (qi.z - qj.z) + sz;
        const float rs = qi.w + qj.w;
        const float rr = rs + g.margin, rl = rs - g.margin;
        const float d2f = fx * fx + fy * fy + fz * fz;
        if (rs < 100.f && d2f > rr * rr) continue;
        bool keep = rl > 0.f && rs < 100.f && d2f < rl * rl;
        if (!keep) {
            const double4_32a pj = pos_r[j];
            const double dx3 = min_image(xsub(pi.x, pj.x), g.periodic[0], L0);
            const double dy3 = min_image(xsub(pi.y, pj.y), g.periodic[1], L1);
            const double dz3 = min_image(xsub(pi.z, pj.z), g.periodic[2], L2);
            const double d = norm_exact(dx3, dy3, dz3);
            // Sect. 4: keep the pair iff the hulls intersect (the exact hulls,
            // body i's computed once)
            if (!(hi_ >= 0.0)) hi_ = hull_of(H, i, pi.w);
            keep = xsub(xsub(d, pi.w), pj.w) <= xadd(hi_, hull_of(H, j, pj.w));
        }
        if (keep) {
            if (P.cnt < kCandCap) {
                // insertion keeps the list sorted by j
                int k = P.cnt;
                while (k > 0 && P.list[k - 1] > j) {
                    P.list[k] = P.list[k - 1];
                    --k;
                }
                P.list[k] = j;
            }
            ++P.cnt;
        }
    }
}

// Neighbour index along one axis: the cell and the shift of the periodic
// image (the image of cell d - 1 left of cell 0 sits at -L); false when the
// cell lies outside a bounded axis.
__device__ __forceinline__ bool axis_cell(int c, int d, int periodic, float Lf, int& out, float& shift)
{
    shift = 0.f;
    if (c >= 0 && c < d) {
        out = c;
        return true;
    }
    if (!periodic || d < 3) return false;
    out = c < 0 ? c + d : c - d;
    shift = c < 0 ? Lf : -Lf;
    return true;
}

__global__ void __launch_bounds__(128)
k_narrow(int64_t n, const uint32_t* __restrict__ skeys, const uint32_t* __restrict__ svals,
         const double4_32a* __restrict__ pos_r, HullView H, const float4* __restrict__ p32s,
         const uint32_t* __restrict__ cs, GridArgs g, Planes planes, SceneView V, DevInfo* info,
         uint32_t* __restrict__ cand, uint32_t* __restrict__ sph_cnt, uint32_t* __restrict__ row_cnt)
{
    const int d0 = info->dims[0], d1 = info->dims[1], d2 = info->dims[2];
    const double L0 = g.hi[0] - g.lo[0], L1 = g.hi[1] - g.lo[1], L2 = g.hi[2] - g.lo[2];
    const bool wrap_x = g.periodic[0] && d0 >= 3;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = svals[s];
        const uint32_t key = skeys[s];
        const int cx = (int)(key % (uint32_t)d0);
        const int cy = (int)((key / (uint32_t)d0) % (uint32_t)d1);
        const int cz = (int)(key / ((uint32_t)d0 * (uint32_t)d1));
        const double4_32a pi = pos_r[i];
        double hi_ = -1.0;   // the exact hull of i, computed when a test needs it
        const float4 qi = p32s[s];
        const uint32_t si = V.batch ? V.scene_of[i] : 0u;
        NarrowPair P;
        P.cnt = 0;
        const int xlo = cx > 0 ? cx - 1 : 0, xhi = cx + 1 < d0 ? cx + 1 : d0 - 1;
        for (int dz = -1; dz <= 1; ++dz) {
            int z;
            float sz;
            if (!axis_cell(cz + dz, d2, g.periodic[2], g.Lf[2], z, sz)) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                int y;
                float sy;
                if (!axis_cell(cy + dy, d1, g.periodic[1], g.Lf[1], y, sy)) continue;
                const uint32_t row = ((uint32_t)z * (uint32_t)d1 + (uint32_t)y) * (uint32_t)d0;
                narrow_range(cs[row + xlo], cs[row + xhi + 1], 0.f, sy, sz, i, si, qi, pi, hi_, svals, p32s, pos_r,
                             H, g, V, L0, L1, L2, P);
                if (wrap_x && cx == 0)
                    narrow_range(cs[row + d0 - 1], cs[row + d0], g.Lf[0], sy, sz, i, si, qi, pi, hi_, svals, p32s,
                                 pos_r, H, g, V, L0, L1, L2, P);
                if (wrap_x && cx == d0 - 1)
                    narrow_range(cs[row], cs[row + 1], -g.Lf[0], sy, sz, i, si, qi, pi, hi_, svals, p32s, pos_r,
                                 H, g, V, L0, L1, L2, P);
            }
        }
        int cnt = P.cnt;
        uint32_t* list = P.list;
        if (cnt > kCandCap) {
            atomicOr(&info->err, kErrCand);
            atomicMax(&info->cand_need, (uint32_t)cnt);
            cnt = kCandCap;
        }
        uint32_t* out = cand + (int64_t)i * kCandCap;
        for (int k = 0; k < cnt; ++k) out[k] = list[k];
        // walls: a conservative FP32 test of the signed distance (errors as
        // for the pairs, within wmargin), the exact FP64 test for the rest
        uint32_t wmask = 0;
        const int nwall = planes.count + planes.ncones + (V.batch ? 6 : 0);
        const float reach = qi.w + g.tauf + g.wmargin;
        for (int k = 0; k < nwall; ++k) {
            const int kc = k - planes.count;
            if (kc >= 0 && kc < planes.ncones) {   // cone (plain scenes only)
                if (cone_distance_f(g, kc, qi) > qi.w + g.tauf + g.cmargin) continue;
                double nrm[3], sd;
                if (!(hi_ >= 0.0)) hi_ = hull_of(H, i, pi.w);
                if (cone_distance(planes.cone[kc], pi, sd, nrm) && xsub(sd, pi.w) <= xadd(hi_, g.tau))
                    wmask |= 1u << k;
                continue;
            }
            float sdf;
            if (k < planes.count) {
                sdf = g.pn[k][0] * qi.x + g.pn[k][1] * qi.y + g.pn[k][2] * qi.z + g.pc[k];
            } else {
                const int f = k - planes.count, axis = f >> 1;
                const float q = axis == 0 ? qi.x : (axis == 1 ? qi.y : qi.z);
                const float* b = V.box32 + 6 * (int64_t)si;
                sdf = (f & 1) == 0 ? q - b[axis] : b[3 + axis] - q;
            }
            if (sdf > reach) continue;
            double nrm[3], c, sd, xi;
            uint32_t widx;
            wall_plane(planes, V, si, k, nrm, c, widx);
            if (!(hi_ >= 0.0)) hi_ = hull_of(H, i, pi.w);
            if (wall_kept(nrm, c, pi, hi_, g.tau, sd, xi)) wmask |= 1u << k;
        }
        sph_cnt[i] = (uint32_t)cnt | (wmask << 8);
        row_cnt[i] = (uint32_t)(cnt + __popc(wmask));
    }
}

// Canonical contact records: row i of the CSR holds (i, j) for the sorted
// partners j, then the walls in the order they were added.  A warp takes 32
// bodies (in cell order) and spreads their sphere pairs over its lanes, one
// pair per lane and pass, so that the FP64 chains of a row run side by side;
// the walls of a body stay with its own lane.
__global__ void k_write_contacts(int64_t n, int64_t ccap, const uint32_t* __restrict__ svals,
                                 const double4_32a* __restrict__ pos_r,
                                 const uint32_t* __restrict__ cand, const uint32_t* __restrict__ sph_cnt,
                                 const uint32_t* __restrict__ row_off, GridArgs g, Planes planes, SceneView V,
                                 uint32_t* __restrict__ cj1, uint32_t* __restrict__ cj2, double4_32a* __restrict__ cgeo,
                                 double2* __restrict__ clev)
{
    const double L0 = g.hi[0] - g.lo[0], L1 = g.hi[1] - g.lo[1], L2 = g.hi[2] - g.lo[2];
    const int lane = threadIdx.x & 31;
    const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform trip count: every lane takes part in the shuffles
    for (int64_t s0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u); s0 < n; s0 += wstride) {
        const int64_t s = s0 + lane;
        uint32_t i = 0, packed = 0, ro = 0;
        double4_32a pi = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        if (s < n) {
            i = svals[s];
            packed = sph_cnt[i];
            if (packed != 0) {
                pi = pos_r[i];
                ro = row_off[i];
            }
        }
        const uint32_t ns = packed & 0xFFu;
        uint32_t pre = ns;   // inclusive prefix of the pair counts over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += v;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, pre, 31);
        for (uint32_t base = 0; base < total; base += 32) {
            const uint32_t t = base + lane;
            // owner: the number of lanes whose pairs end at or before t
            int own = 0;
#pragma unroll
            for (int b = 16; b >= 1; b >>= 1) {
                const uint32_t v = __shfl_sync(0xffffffffu, pre, own + b - 1);
                if (v <= t) own += b;
            }
            own = own < 31 ? own : 31;
            const uint32_t i_o = __shfl_sync(0xffffffffu, i, own);
            const uint32_t ro_o = __shfl_sync(0xffffffffu, ro, own);
            const uint32_t end_o = __shfl_sync(0xffffffffu, pre, own);
            const uint32_t ns_o = __shfl_sync(0xffffffffu, ns, own);
            double4_32a po;
            po.x = __shfl_sync(0xffffffffu, pi.x, own);
            po.y = __shfl_sync(0xffffffffu, pi.y, own);
            po.z = __shfl_sync(0xffffffffu, pi.z, own);
            po.w = __shfl_sync(0xffffffffu, pi.w, own);
            if (t >= total) continue;
            const uint32_t k = t - (end_o - ns_o);
            const int64_t idx = (int64_t)ro_o + k;
            if (idx >= ccap) continue;
            const uint32_t j = cand[(int64_t)i_o * kCandCap + k];
            const double4_32a pj = pos_r[j];
            const double dx3 = min_image(xsub(po.x, pj.x), g.periodic[0], L0);
            const double dy3 = min_image(xsub(po.y, pj.y), g.periodic[1], L1);
            const double dz3 = min_image(xsub(po.z, pj.z), g.periodic[2], L2);
            // eq. (contactpos) for spheres: n = (x_i - x_j)/d, the outward
            // normal of S_j at its point closest to x_i; xi = d - r_i - r_j
            double nrm[3];
            const double d = pair_normal(dx3, dy3, dz3, nrm);
            double4_32a geo;
            geo.x = nrm[0];
            geo.y = nrm[1];
            geo.z = nrm[2];
            geo.w = xsub(xsub(d, po.w), pj.w);
            cj1[idx] = i_o;
            cj2[idx] = j;
            cgeo[idx] = geo;
            clev[idx] = make_double2(xsub(d, pj.w), pj.w);
        }
        const uint32_t wm = packed >> 8;
        if (wm == 0) continue;
        const uint32_t si = V.batch ? V.scene_of[i] : 0u;
        int64_t idx = (int64_t)ro + ns;
        for (uint32_t m = wm; m; m &= m - 1) {   // the walls k_narrow kept, in wall order
            const int k = __ffs(m) - 1;
            double nrm[3], c, sd, xi;
            uint32_t widx;
            const int kc = k - planes.count;
            if (kc >= 0 && kc < planes.ncones) {
                // the point of the cone's solid nearest to x_i is x_i - sd n:
                // a wall contact with xi = sd - r_i and l_i = -sd n
                cone_distance(planes.cone[kc], pi, sd, nrm);
                xi = xsub(sd, pi.w);
                widx = (uint32_t)(V.n + k);
            } else {
                wall_plane(planes, V, si, k, nrm, c, widx);
                wall_kept(nrm, c, pi, 0.0, g.tau, sd, xi);   // kept already: only sd and xi are used
            }
            if (idx < ccap) {
                cj1[idx] = i;
                cj2[idx] = widx;
                cgeo[idx] = make_double4_32a(nrm[0], nrm[1], nrm[2], xi);
                clev[idx] = make_double2(sd, 0.0);
            }
            ++idx;
        }
    }
}

SceneView scene_view(const nbgs_scene* s)
{
    SceneView v;
    v.batch = s->batch ? 1 : 0;
    v.nplanes = s->planes.count;
    v.n = s->n;
    v.scene_of = s->scene_of;
    v.scene_off = s->scene_off;
    v.box = s->scene_box;
    v.box32 = s->scene_box32;
    v.mu = s->scene_mu;
    v.vref = s->scene_vref;
    v.body_of = s->composite ? s->mbody : nullptr;
    return v;
}

static GridArgs grid_args(const nbgs_scene* s)
{
    GridArgs g;
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = s->prm.box_lo[a];
        g.hi[a] = s->prm.box_hi[a];
        g.periodic[a] = s->prm.periodic[a];
        g.dims_max[a] = s->dims_max[a];
    }
    g.r_max = s->r_max;
    g.dt = s->prm.dt;
    g.tau = s->prm.tau;
    double lmax = 0.0;
    for (int a = 0; a < 3; ++a) {
        g.Lf[a] = (float)(g.hi[a] - g.lo[a]);
        lmax = std::max(lmax, g.hi[a] - g.lo[a]);
    }
    g.margin = (float)(1e-4 + 1e-6 * lmax);
    g.pos_err = std::ldexp(lmax, -22);
    double cmax = 0.0;
    for (int k = 0; k < s->planes.count; ++k) {
        double off = -s->planes.c[k];
        for (int a = 0; a < 3; ++a) {
            g.pn[k][a] = (float)s->planes.n[k][a];
            off += s->planes.n[k][a] * g.lo[a];
        }
        g.pc[k] = (float)off;
        cmax = std::max(cmax, std::fabs(off));
    }
    g.tauf = (float)g.tau;
    g.wmargin = (float)(1e-4 + 4e-6 * (lmax + cmax));
    double amax = 0.0;
    for (int k = 0; k < s->planes.ncones; ++k) {
        const Cone& C = s->planes.cone[k];
        for (int a = 0; a < 3; ++a) {
            g.ca_apex[k][a] = (float)(C.apex[a] - g.lo[a]);
            g.ca_axis[k][a] = (float)C.axis[a];
            amax = std::max(amax, std::fabs(C.apex[a] - g.lo[a]));
        }
        g.ca_sc[k][0] = (float)C.sa;
        g.ca_sc[k][1] = (float)C.ca;
        g.ca_sc[k][2] = (float)C.s_o;
        g.ca_sc[k][3] = (float)C.s_t;
    }
    g.cmargin = (float)(1e-4 + 1e-5 * (lmax + amax));
    return g;
}

nbgs_status grow_contacts(nbgs_scene* s, int64_t need);  // api.cu

// Device-sized steps: the previous step's contact count, kept before the
// detection clears it; a count beyond the buffers sets the contact error bit.
__global__ void k_keep_count(DevInfo* info) { info->prev_contacts = info->n_contacts; }

__global__ void k_check_contacts(DevInfo* info, int64_t ccap)
{
    if ((int64_t)info->n_contacts > ccap) atomicOr(&info->err, kErrContacts);
}

nbgs_status run_detect(nbgs_scene* s)
{
    const int64_t n = s->n;
    cudaStream_t st = s->stream;
    if (s->timing) cudaEventRecord(s->ev[0], st);
    // keep the previous step's contacts for the warm start
    if (s->prm.warm_start != NBGS_WARM_NONE && s->solved) {
        std::swap(s->row_off, s->prev_row_off);
        std::swap(s->cj2, s->prev_j2);
        std::swap(s->cworld, s->prev_P);
        s->prev_count = s->n_contacts;
        s->have_prev = true;
    }
    // otherwise the previous-step arrays keep what they hold: the contacts of
    // the last solved step, or of a restored checkpoint (nbgs_set_bodies
    // starts a new history)
    s->detected = s->coloured = s->solved = false;
    s->n_contacts = 0;
    s->sub_count = -1;
    if (s->device_sized) k_keep_count<<<1, 1, 0, st>>>(s->info);
    cudaMemsetAsync(s->info, 0, offsetof(DevInfo, cell_w), st);   // hmax, vmax
    cudaMemsetAsync(&s->info->n_contacts, 0, sizeof(uint32_t), st);
    if (n == 0) {
        cudaMemsetAsync(s->row_off, 0, sizeof(uint32_t), st);
        s->detected = true;
        return cuda_check(s, cudaGetLastError(), "detect");
    }
    const GridArgs g = grid_args(s);
    const int T = 256;
    const int gb = grid_for(n, T, 8, s->num_sms);
    if (s->batch) cudaMemsetAsync(s->scene_vmax, 0, s->n_scenes * sizeof(unsigned long long), st);
    if (s->composite) {
        if (s->fp32)
            k_member_update<float><<<gb, T, 0, st>>>(n, s->mbody, s->moff, s->bpos, s->bquat, (const float4*)s->bvel,
                                                     s->prm.dt, s->prm.tau, s->pos_r, s->hull, s->p32, g, s->info);
        else
            k_member_update<double><<<gb, T, 0, st>>>(n, s->mbody, s->moff, s->bpos, s->bquat,
                                                      (const double4_32a*)s->bvel, s->prm.dt, s->prm.tau, s->pos_r,
                                                      s->hull, s->p32, g, s->info);
    } else if (s->fp32)
        k_hull<float><<<gb, T, 0, st>>>(n, (const float4*)s->vel, s->pos_r, s->prm.dt, s->prm.tau, s->hvw, s->p32,
                                        g, s->info, s->scene_of, s->scene_vmax);
    else
        k_hull<double><<<gb, T, 0, st>>>(n, (const double4_32a*)s->vel, s->pos_r, s->prm.dt, s->prm.tau, s->hvw,
                                         s->p32, g, s->info, s->scene_of, s->scene_vmax);
    k_grid_setup<<<1, 1, 0, st>>>(g, s->info);
    cudaMemsetAsync(s->cell_end, 0, (size_t)s->max_cells * sizeof(uint32_t), st);   // cell counts
    k_cell_keys<<<gb, T, 0, st>>>(n, s->p32, s->info, s->keys[0], s->vals[0], s->cell_end);
    if (s->timing) s->phase_launches[0] += 4;
    nbgs_status rc = radix_sort_pairs(s, s->keys[0], s->vals[0], s->keys[1], s->vals[1], n, s->key_bits);
    if (rc != NBGS_OK) return rc;
    // first sorted slot of every cell (empty ones included); cell_start[max_cells] = n
    rc = exclusive_scan_u32(s, s->cell_end, s->cell_start, s->max_cells, nullptr);
    if (rc != NBGS_OK) return rc;
    k_gather_sorted<<<gb, T, 0, st>>>(n, s->vals[0], s->p32, s->p32s);
    const HullView H{s->composite ? s->hull : nullptr, s->hvw, s->prm.dt, s->prm.tau};
    k_narrow<<<grid_for(n, 128, 16, s->num_sms), 128, 0, st>>>(n, s->keys[0], s->vals[0], s->pos_r, H,
                                                                 s->p32s, s->cell_start, g, s->planes,
                                                                 scene_view(s), s->info, s->cand, s->sph_cnt,
                                                                 s->row_cnt);
    rc = exclusive_scan_u32(s, s->row_cnt, s->row_off, n, &s->info->n_contacts);
    if (rc != NBGS_OK) return rc;
    if (s->timing) s->phase_launches[0] += 5;
    if (s->device_sized) {
        // no synchronisation: the buffers keep their capacity, an overflow
        // sets an error bit (the writes past it are skipped), and every
        // later kernel reads the count on the device
        k_check_contacts<<<1, 1, 0, st>>>(s->info, s->ccap);
        k_write_contacts<<<grid_for(n, T, 8, s->num_sms), T, 0, st>>>(n, s->ccap, s->vals[0], s->pos_r,
                                                                      s->cand, s->sph_cnt, s->row_off, g, s->planes,
                                                                      scene_view(s), s->cj1, s->cj2, s->cgeo, s->clev);
        if (s->timing) {
            s->phase_launches[0] += 3;
            cudaEventRecord(s->ev[1], st);
        }
        s->n_contacts = s->ccap;   // an upper bound; the count itself stays on the device
        s->detected = true;
        return cuda_check(s, cudaGetLastError(), "detect");
    }
    // one synchronisation per step: the contact count sizes everything after
    rc = cuda_check(s, cudaMemcpyAsync(s->hinfo, s->info, offsetof(DevInfo, rk_bits), cudaMemcpyDeviceToHost, st),
                    "detect: read info");
    if (rc != NBGS_OK) return rc;
    rc = cuda_check(s, cudaStreamSynchronize(st), "detect");
    if (rc != NBGS_OK) return rc;
    const DevInfo& hi = *s->hinfo;
    if (hi.err & kErrNaN) return fail(s, NBGS_ENAN, "detect: NaN or Inf in the velocities");
    if (hi.err & kErrGrid) return fail(s, NBGS_EINVAL, "detect: a periodic axis holds fewer than 3 grid cells");
    if (hi.err & kErrCand)
        return fail(s, NBGS_ECAPACITY, "detect: a body has " + std::to_string(hi.cand_need) +
                                           " hull neighbours above it (limit " + std::to_string(kCandCap) + ")");
    const int64_t nc = hi.n_contacts;
    if (nc > s->ccap) {
        rc = grow_contacts(s, nc);
        if (rc != NBGS_OK) return rc;
    }
    k_write_contacts<<<grid_for(n, T, 8, s->num_sms), T, 0, st>>>(n, s->ccap, s->vals[0], s->pos_r, s->cand,
                                                                  s->sph_cnt, s->row_off, g, s->planes, scene_view(s),
                                                                  s->cj1, s->cj2, s->cgeo, s->clev);
    if (s->timing) {
        s->phase_launches[0] += 1;
        cudaEventRecord(s->ev[1], st);
    }
    s->n_contacts = nc;
    s->detected = true;
    return cuda_check(s, cudaGetLastError(), "detect");
}

}  // namespace nbgs

namespace nbgs {
__global__ void k_pair_normals(int64_t n, const double* __restrict__ dvec, double* __restrict__ out)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double nrm[3];
        const double d = pair_normal(dvec[3 * k], dvec[3 * k + 1], dvec[3 * k + 2], nrm);
        out[4 * k] = nrm[0];
        out[4 * k + 1] = nrm[1];
        out[4 * k + 2] = nrm[2];
        out[4 * k + 3] = d;
    }
}
}  // namespace nbgs

extern "C" nbgs_status nbgs_pair_normals(int64_t n, const double* dvec, double* out, void* stream)
{
    using namespace nbgs;
    if (n < 0 || (n > 0 && (!dvec || !out))) return NBGS_EINVAL;
    if (n == 0) return NBGS_OK;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_pair_normals<<<grid_for(n, 256, 8, sms), 256, 0, (cudaStream_t)stream>>>(n, dvec, out);
    return cudaGetLastError() == cudaSuccess ? NBGS_OK : NBGS_ECUDA;
}
