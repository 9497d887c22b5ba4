// nbgs_internal.cuh -- shared declarations of the sm_103a NBGS library.
//
// Layout in HBM (one scene):
//   bodies  pos_r  double4_32a[n]  (x, y, z, radius)          -- FP64 always
//           quat   double4_32a[n]  (w, x, y, z)
//           vel    R4[2n]      (v, 1/m), (omega, 1/I) adjacent per body:
//                              32 B per body in FP32 (one sector), 64 B in FP64
//           hull   double[n]   h_i of this step
//   grid    cell_start/end u32[max_cells], keys/vals u32[n] x2 (radix sort)
//   contacts (canonical, CSR by j1): cj1, cj2 u32; cgeo double4_32a (n, xi);
//           clev double2 (la, lb) with lever arms l_a = -la n, l_b = lb n
//   sweep   srec SweepRec<R>[C] in colour order; sp R4[C] impulses (p_n, p_t, p_o)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/nbgs.h"

namespace nbgs {

constexpr int kMaxPlanes = 16;
constexpr int kMaxColours = 256;       // a colour is 8 bits of the colouring state
constexpr int kCandCap = 32;           // sphere candidates per body with j > i
constexpr uint32_t kUncoloured = 0xFFFFFFFFu;
constexpr int kMaxSweepsHist = 4096;   // residual slots: history, 3 rotating, 4 final
constexpr int kHistKept = kMaxSweepsHist - 8;   // sweeps whose R_k is kept

// Slot of max_j r_j for sweep k: its own slot for the first kHistKept
// sweeps, then three slots used in rotation (the slot of sweep k + 1 is
// cleared while sweep k runs; every reader of sweep k - 2 is done by then).
__host__ __device__ __forceinline__ int rk_slot(int k) { return k < kHistKept ? k : kHistKept + k % 3; }

// device error bits (DevInfo::err)
enum : uint32_t {
    kErrCand = 1u,        // more than kCandCap neighbours above i
    kErrContacts = 2u,    // contact buffer too small
    kErrColours = 4u,     // more than kMaxColours colours
    kErrTimeout = 8u,     // a grid barrier wait gave up
    kErrNaN = 16u,        // NaN / Inf in velocities or positions
    kErrGrid = 32u        // periodic axis with fewer than 3 cells
};

// A count that the host either knows (dev == nullptr: v is the count) or
// leaves to the device (v is the capacity the launch is sized for, *dev the
// count, read by the kernel): device-sized steps read every contact count
// on the device, so that no step waits for the host.  A device count beyond
// the capacity (an overflow, reported by an error bit) is clamped to it, so
// that no kernel reads or writes past the buffers.
struct DCount {
    int64_t v;
    const uint32_t* dev;
    __device__ __forceinline__ int64_t get() const
    {
        if (!dev) return v;
        const int64_t c = (int64_t)*dev;
        return c < v ? c : v;
    }
};

constexpr int kMaxCones = 4;
constexpr int kMaxMembers = 4;          // member spheres of a composite particle

// Conical hopper wall (frustum between the orifice and the top circle);
// sin and cos of the half-angle come from the host's C library.
struct Cone {
    double apex[3], axis[3];   // axis unit, the cone opens along it
    double sa, ca;             // sin, cos of the half-angle
    double s_o, s_t;           // orifice and top along a generatrix, from the apex
};

// Shared walls: half-spaces, then cones (wall index n + k, k < count, then
// n + count + k for cone k).
struct Planes {
    int count;
    double n[kMaxPlanes][3];
    double c[kMaxPlanes];
    int ncones;
    Cone cone[kMaxCones];
};

// Batched scenes as the kernels see them (batch == 0: one plain scene).
struct SceneView {
    int batch;
    int nplanes;                  // walls shared by every scene (nbgs_add_plane)
    int64_t n;                    // bodies in total
    const uint32_t* scene_of;     // n
    const uint32_t* scene_off;    // S + 1
    const double* box;            // S x 6
    const float* box32;           // S x 6: box - global box lo, FP32 (the wall pre-filter)
    const double* mu;             // S
    const double* vref;           // S
    const uint32_t* body_of;      // composite scenes: body of each member sphere (null otherwise)
};

// Wall k of body i's scene: k < nplanes are the shared planes, then the six
// faces of the scene box (+x at lo, -x at hi, +y, -y, +z, -z).  Body index
// of the wall: n + k for shared planes, n + nplanes + 6 s + face.
__device__ __forceinline__ void wall_plane(const Planes& P, const SceneView& V, uint32_t s, int k, double nrm[3],
                                           double& c, uint32_t& index)
{
    if (k < P.count) {
        nrm[0] = P.n[k][0];
        nrm[1] = P.n[k][1];
        nrm[2] = P.n[k][2];
        c = P.c[k];
        index = (uint32_t)(V.n + k);
        return;
    }
    const int f = k - P.count, axis = f >> 1;
    nrm[0] = nrm[1] = nrm[2] = 0.0;
    if ((f & 1) == 0) {
        nrm[axis] = 1.0;
        c = V.box[6 * (int64_t)s + axis];
    } else {
        nrm[axis] = -1.0;
        c = -V.box[6 * (int64_t)s + 3 + axis];
    }
    index = (uint32_t)(V.n + P.count + 6 * (int64_t)s + f);
}

// Everything a step's kernels communicate through device memory.
struct DevInfo {
    unsigned long long hmax_bits;   // max hull radius (bits of a non-negative double)
    unsigned long long vmax_bits;   // max |v_i| at the start of the step
    double cell_w[3];
    float inv_wf[3];                 // 1 / cell width, FP32 (cell keys from the FP32 positions)
    int dims[3];
    uint32_t ncells;
    uint32_t n_contacts;
    uint32_t n_colours;
    uint32_t err;
    uint32_t cand_need;              // largest candidate count seen
    uint32_t sweeps_done;
    uint32_t wl_count[6];            // colouring list sizes (|L|, |X|), three rotating pairs
    uint32_t barrier_count;          // grid barrier arrival counter
    uint32_t barrier_gen;            // grid barrier generation
    uint32_t rounds;                 // colouring rounds used
    uint32_t n_shared;               // subdomains: bodies with more than one velocity instance
    uint32_t n_extra;                // subdomains: velocity instances after the n bodies
    uint32_t prev_contacts;          // contacts of the previous step (device-sized steps)
    unsigned long long updates;      // contact updates (contacts x sweeps relaxed) since the last read
    double residual;                 // R of the last sweep
    double v_ref;
    unsigned long long rk_bits[kMaxSweepsHist];  // max_j r_j of sweep k (bits)
    uint32_t votes[2 * kMaxSweepsHist];          // tolerance test of sweep k: (a block above tol, blocks at or below)
};

// ---------------------------------------------------------------------------
// FP64 arithmetic with explicit round-to-nearest and no contraction: used
// wherever a floating-point result decides an integer outcome (which pairs
// become contacts), so that it rounds exactly as the expression is written.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double xadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double xsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double xdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double xsqrt(double a) { return __dsqrt_rn(a); }

// splitmix64 (Steele, Lea & Flood 2014): Weyl increment, then the mixer.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class R> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = double4_32a; };
template <class R> using R4 = typename Vec4<R>::T;

// Tangent basis (t, o) of a unit normal n: Duff et al., "Building an
// Orthonormal Basis, Revisited", JCGT 6(1) 2017 (branchless form).
template <class R>
__device__ __forceinline__ void tangent_basis(R nx, R ny, R nz, R& tx, R& ty, R& tz, R& ox, R& oy, R& oz)
{
    const R sign = copysign(R(1), nz);
    const R a = R(-1) / (sign + nz);
    const R b = nx * ny * a;
    tx = R(1) + sign * nx * nx * a;
    ty = sign * b;
    tz = -sign * nx;
    ox = b;
    oy = sign + ny * ny * a;
    oz = -ny;
}

// Sweep record of one contact in colour order: ids, lever lengths, normal and
// gap term xi'/dt.  32 B in FP32, 64 B in FP64.
template <class R> struct SweepRec;
template <> struct __align__(16) SweepRec<float> {
    float4 a;  // (j1 bits, j2 bits, la, lb)
    float4 b;  // (nx, ny, nz, bias)
};
template <> struct __align__(16) SweepRec<double> {
    double2 ids_bias;  // (j1 | j2 << 32 bits, bias)
    double2 lev;       // (la, lb)
    double2 nxy;       // (nx, ny)
    double2 nz_;       // (nz, unused)
};

// 256-bit global accesses: a body's (v, 1/m) and (w, 1/I) pair and an FP32
// sweep record each move as one request instead of two (FP64: two instead
// of four).  The body accesses keep their order with every other memory
// access of the thread.
__device__ __forceinline__ void ld_body(const float4* p, float4& v, float4& w)
{
    asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w), "=f"(w.x), "=f"(w.y), "=f"(w.z), "=f"(w.w)
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ void ld_body(const double4_32a* p, double4_32a& v, double4_32a& w)
{
    asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(v.x), "=d"(v.y), "=d"(v.z), "=d"(v.w)
                 : "l"(p)
                 : "memory");
    asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(w.x), "=d"(w.y), "=d"(w.z), "=d"(w.w)
                 : "l"(p + 1)
                 : "memory");
}
__device__ __forceinline__ void st_body(float4* p, const float4& v, const float4& w)
{
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w), "f"(w.x), "f"(w.y), "f"(w.z), "f"(w.w)
                 : "memory");
}
__device__ __forceinline__ void st_body(double4_32a* p, const double4_32a& v, const double4_32a& w)
{
    asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v.x), "d"(v.y), "d"(v.z), "d"(v.w)
                 : "memory");
    asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p + 1), "d"(w.x), "d"(w.y), "d"(w.z), "d"(w.w)
                 : "memory");
}
// A 32-byte FP64 4-vector as one 256-bit access.
__device__ __forceinline__ double4_32a ld_d4(const double4_32a* p)
{
    double4_32a v;
    asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(v.x), "=d"(v.y), "=d"(v.z), "=d"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}
__device__ __forceinline__ void st_d4(double4_32a* p, const double4_32a& v)
{
    asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v.x), "d"(v.y), "d"(v.z), "d"(v.w) : "memory");
}

// Bounded grid-wide barrier for a cooperative launch (all blocks resident).
// Returns false when the wait ran out (the error bit is set and every block
// leaves at its next check).  Never spins without a limit.
__device__ __forceinline__ bool grid_barrier(DevInfo* info, unsigned nblocks)
{
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        volatile uint32_t* vgen = &info->barrier_gen;
        volatile uint32_t* verr = &info->err;
        const uint32_t gen = *vgen;
        __threadfence();
        const uint32_t arrived = atomicAdd(&info->barrier_count, 1u);
        int good = 1;
        if (arrived == nblocks - 1) {
            info->barrier_count = 0;
            __threadfence();
            atomicAdd(&info->barrier_gen, 1u);
        } else {
            long long spins = 0;
            while (*vgen == gen) {
                if ((*verr & kErrTimeout) || ++spins > 20000000LL) {  // ~1 s with the sleep below
                    atomicOr(&info->err, kErrTimeout);
                    good = 0;
                    break;
                }
                __nanosleep(40);
            }
        }
        __threadfence();
        ok = good && !(*verr & kErrTimeout);
    }
    __syncthreads();
    return ok != 0;
}

// ---------------------------------------------------------------------------
// Local synchronisation of the colour sweeps (dependency windows): block b
// of a cooperative launch owns the slots [cstart[c][b], cstart[c][b + 1]) of
// colour c, chunks balanced by contact count and local in body index.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void colour_chunk(const uint32_t* cstart, int c, int64_t& b0, int64_t& b1)
{
    const uint32_t* row = cstart + (int64_t)c * (gridDim.x + 1);
    b0 = row[blockIdx.x];
    b1 = row[blockIdx.x + 1];
}


// Acquire load of a progress word: the reads that follow it in this thread
// (and, through a block barrier, in the block) see every store the writer
// released before the value read.
__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until every block in this chunk's window has completed sweep phase
// g - 1 (it and all earlier phases): then every contact of another colour
// that shares a body with this chunk is settled.  Warp 0 polls the progress
// words with acquire loads (no fence after the wait: on the settled 1M pour
// the sweeps run 9 % faster than with relaxed polls and a fence); bounded
// like every other wait.
__device__ __forceinline__ bool wait_deps(const int* prog, int2 win, int g, DevInfo* info, int* s_ok)
{
    if (threadIdx.x < 32) {
        int ok = 1;
        const int nblk = (int)gridDim.x, self = (int)blockIdx.x;
        for (int off = win.x + (int)threadIdx.x; off <= win.y && ok; off += 32) {
            if (off == 0) continue;
            const int b = ((self + off) % nblk + nblk) % nblk;
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
        ok = __all_sync(0xffffffffu, ok);
        if (threadIdx.x == 0) *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Publish that this block finished sweep phase g (after all its stores).
// Phases are numbered 0, 1, 2, ... and a block publishes every one of them
// in order, its word starting at -1, so advancing the word by one sets it to
// g.  The increment is a release reduction: it orders the block's stores
// (before the barrier) ahead of the new value without waiting for a reply.
__device__ __forceinline__ void publish(int* prog, int g)
{
    (void)g;
    __syncthreads();
    if (threadIdx.x == 0)
        asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(prog + blockIdx.x) : "memory");
}



}  // namespace nbgs

// ---------------------------------------------------------------------------
// Host-side scene
// ---------------------------------------------------------------------------
struct nbgs_scene {
    nbgs_params prm;
    int64_t n = 0;
    nbgs::Planes planes{};
    cudaStream_t stream = nullptr;
    nbgs_allocator alloc{};
    bool has_alloc = false;
    nbgs_status status = NBGS_OK;
    std::string err;
    int device = 0;
    int num_sms = 0;
    double r_max = 0.0;
    bool fp32 = false;

    // batched scenes (n_scenes == 1 and no arrays for a plain scene)
    int64_t n_scenes = 1;
    bool batch = false;
    uint32_t* scene_of = nullptr;       // n: scene of each body
    uint32_t* scene_off = nullptr;      // S + 1: first body of each scene
    double* scene_box = nullptr;        // S x 6: lo xyz, hi xyz
    float* scene_box32 = nullptr;       // S x 6: the same minus the global box lo, FP32
    double* scene_mu = nullptr;         // S
    unsigned long long* scene_vmax = nullptr;  // S: max |v| at step start (bits)
    double* scene_vref = nullptr;       // S
    unsigned long long* scene_rk = nullptr;    // 3 x S rotating slots: max r_j / v_ref per sweep (bits)
    uint32_t* scene_done = nullptr;     // S: sweeps to tolerance
    double* scene_res = nullptr;        // S: R_k at that sweep
    int max_coop_blocks = 0;            // occupancy limit of the persistent kernel

    // bodies
    double4_32a* pos_r = nullptr;
    double4_32a* quat = nullptr;
    void* vel = nullptr;          // R4[2 (n + icap)]: (v, 1/m), (w, 1/I) per body, then extra instances
    double* hull = nullptr;
    double2* hvw = nullptr;        // |v|^2, |w|^2 per sphere (the exact hulls' inputs)
    float4* p32 = nullptr;        // (x - lo, y - lo, z - lo, r + h) in FP32: cell keys and the narrow-phase pre-filter
    float4* p32s = nullptr;       // p32 in cell order (the narrow phase's candidate reads)
    uint8_t* finite = nullptr;    // body takes impulses (1/m > 0 or 1/I > 0)
    double* stage = nullptr;      // 13 n doubles for state transfer
    // grid
    int dims_max[3] = {1, 1, 1};
    int64_t max_cells = 1;
    int key_bits = 1;
    uint32_t* cell_start = nullptr;   // max_cells + 1: first sorted slot of every cell
    uint32_t* cell_end = nullptr;     // max_cells: bodies per cell
    uint32_t* keys[2] = {nullptr, nullptr};
    uint32_t* vals[2] = {nullptr, nullptr};
    uint32_t* radix_hist = nullptr;
    int64_t radix_hist_len = 0;
    uint32_t* scan_tmp = nullptr;  // block sums of the scans
    int64_t scan_tmp_len = 0;
    // candidates
    uint32_t* cand = nullptr;      // n * kCandCap
    uint32_t* sph_cnt = nullptr;   // sphere contacts per body (bits 0-7), kept-wall mask (bits 8-31)
    uint32_t* row_cnt = nullptr;   // contacts per body (sphere + wall)
    uint32_t* row_off = nullptr;   // n + 1
    // contacts (canonical)
    int64_t ccap = 0;
    uint32_t* cj1 = nullptr;
    uint32_t* cj2 = nullptr;
    double4_32a* cgeo = nullptr;
    double2* clev = nullptr;
    double4_32a* cimp = nullptr;       // canonical (p_n, p_t, p_o, -) after the solve
    double4_32a* cworld = nullptr;     // canonical world-frame impulse after the solve
    // warm start: previous step (CSR by j1)
    uint32_t* prev_row_off = nullptr;
    uint32_t* prev_j2 = nullptr;
    double4_32a* prev_P = nullptr;     // world-frame impulse
    int64_t prev_count = 0;
    bool have_prev = false;
    // colouring
    uint32_t* deg = nullptr;       // n + 1
    uint32_t* adj_off = nullptr;   // n + 1
    uint32_t* adj = nullptr;       // 2 ccap
    uint32_t* cstate = nullptr;    // (round << 8) | colour, kUncoloured before
    uint64_t* cprio = nullptr;
    uint4* cpack = nullptr;        // colouring: per contact (body 1, body 2 or none, its positions in their lists)
    uint32_t* cmask = nullptr;     // colouring: 8 x 32 colour bits per body (its coloured prefix)
    int colour_rounds = 0;         // rounds the last colouring took (the host checks after as many)
    uint32_t* wl[2] = {nullptr, nullptr};
    uint32_t* colour_key = nullptr;   // colour per contact (sort key)
    uint32_t* colour_key2 = nullptr;
    uint32_t* perm = nullptr;      // sweep slot -> canonical index
    uint32_t* perm_in = nullptr;   // the sort's input, then canonical index -> sweep slot (perm inverted)
    uint32_t* col_count = nullptr; // kMaxColours + 1
    uint32_t* col_off = nullptr;   // kMaxColours + 1
    uint32_t* colour_sorted = nullptr;  // colour of each sweep slot (points into colour_key / colour_key2)
    int2* dep = nullptr;           // kMaxColours x coop_blocks block windows [lo, hi] of each chunk
    int* prog = nullptr;           // coop_blocks: last sweep phase each block completed
    uint32_t* cstart = nullptr;    // kMaxColours x (coop_blocks + 1) chunk boundaries
    // subdomains (Alg. 1 with s_c(j)): one velocity instance per (finite body,
    // subdomain) pair; the body's own record serves its lowest subdomain, the
    // others sit after the n bodies in vel
    uint32_t* csub = nullptr;      // sub_ccap: subdomain of each contact (canonical order)
    uint32_t* inst = nullptr;      // 2 sub_ccap: velocity record of end j1 / j2 of each contact
    uint32_t* ext_off = nullptr;   // n + 1: extra instances per body, then their exclusive scan
    uint32_t* shared = nullptr;    // n: bodies with extra instances (n_shared of them)
    void* vacc = nullptr;          // R4[2n]: accumulated velocity at the start of the sweep (shared bodies)
    uint32_t* rlist = nullptr;     // n: shared bodies grouped by the block that reduces them
    uint32_t* rstart = nullptr;    // units + 1: each block's range of rlist
    uint32_t* rcount = nullptr;    // units + 1: scratch counts
    int2* dep_r = nullptr;         // units: window of each block's reduction phase
    int64_t sub_ccap = 0;          // contacts the subdomain arrays hold
    int64_t sub_count = -1;        // contacts csub describes (-1: none since the last detection)
    int64_t icap = 0;              // extra instance records allocated after the n bodies in vel
    // composite particles: the detection spheres (n of them) are the members
    // of nb rigid bodies; contacts join members, the sweeps act on bodies
    bool composite = false;
    int64_t nb = 0;
    double4_32a* bpos = nullptr;   // nb: centre of mass, bounding radius
    double4_32a* bquat = nullptr;  // nb: orientation (w, x, y, z)
    void* bvel = nullptr;          // R4[4 nb]: (v, 1/m), (w, 0), (Ixx, Iyy, Izz, Ixy), (Ixz, Iyz, 0, 0) of I^-1 (world)
    double* bI0 = nullptr;         // 9 nb: body-frame inertia about the centre of mass
    double* bI0inv = nullptr;      // 9 nb: its inverse
    double* bIinv = nullptr;       // 6 nb: world inverse inertia of the current orientation (FP64)
    double* binvm = nullptr;       // nb: 1/m (FP64)
    uint8_t* bfinite = nullptr;    // nb
    uint32_t* mbody = nullptr;     // n: body of each member
    uint32_t* bfirst = nullptr;    // nb: first member of each body
    uint32_t* banchor = nullptr;   // nb: a canonical contact position per body (dependency windows)
    double4_32a* moff = nullptr;   // n: body-frame offset from the centre of mass, radius
    uint32_t* cb1 = nullptr;       // comp_ccap: body of contact end j1
    uint32_t* cb2 = nullptr;       // comp_ccap: body of contact end j2 (nb: a wall)
    void* crec = nullptr;          // comp_ccap composite sweep records (colour order)
    int64_t comp_ccap = 0;
    // learned warm start
    float* mlp_theta = nullptr;    // 9,347 FP32 parameters
    // sweep
    void* srec = nullptr;
    void* sp = nullptr;
    // device info
    nbgs::DevInfo* info = nullptr;
    nbgs::DevInfo* hinfo = nullptr;   // pinned host copy
    // state
    int64_t n_contacts = 0;
    int32_t n_colours = 0;
    bool detected = false;
    bool coloured = false;
    bool solved = false;
    int32_t last_sweeps = 0;
    // device-sized steps (nbgs_graph_step): no host synchronisation inside a
    // step; contact counts are read on the device, buffers keep their
    // capacities and overflows set error bits; the step is captured as two
    // CUDA graphs (the two parities of the warm-start buffer swap)
    bool device_sized = false;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int32_t g_sweeps = -1;
    double g_tol = -1.0;
    int g_next = 0;                // graph of the next replay
    int64_t g_ccap = -1;   // contact capacity the graphs were captured with
    bool counts_stale = false;     // graphs ran since the host last read the counts
    // timing
    bool timing = false;
    cudaEvent_t ev[10] = {};            // start/end of detect, colour, solve, integrate, sweep kernels
    double phase_ms[5] = {0, 0, 0, 0, 0};
    int64_t phase_launches[4] = {0, 0, 0, 0};
    int64_t sweep_launches = 0;
    int coop_blocks = 0;           // resident blocks of the persistent sweep kernel
    int coop_threads = 256;
};

namespace nbgs {

// host helpers (api.cu)
nbgs_status fail(nbgs_scene* s, nbgs_status st, const std::string& msg);
nbgs_status cuda_check(nbgs_scene* s, cudaError_t e, const char* what);
void* dev_alloc(nbgs_scene* s, size_t bytes);
void dev_free(nbgs_scene* s, void* p);

// phases (detect.cu / colour.cu / solve.cu / integrate.cu)
nbgs_status run_detect(nbgs_scene* s);
nbgs_status run_colour(nbgs_scene* s);
nbgs_status run_solve(nbgs_scene* s, int max_sweeps, double tol);
nbgs_status run_integrate(nbgs_scene* s);
nbgs_status run_final_residuals(nbgs_scene* s, nbgs_residuals* out);
nbgs_status run_set_impulses(nbgs_scene* s, const double* impulse);
nbgs_status run_mlp_prologue(nbgs_scene* s, int apply, float* feat_out);
nbgs_status run_subdomains(nbgs_scene* s);            // subdomain.cu: s_c(j), instances (after the adjacency)
nbgs_status ensure_subdomain_buffers(nbgs_scene* s);  // subdomain.cu
void free_subdomain_buffers(nbgs_scene* s);          // subdomain.cu
nbgs_status run_get_subdomains(nbgs_scene* s, int64_t cap, uint32_t* out);
bool subdomains_valid(int32_t mode, const int32_t g[3]);   // api.cu
// composite particles (composite.cu)
nbgs_status ensure_composite_buffers(nbgs_scene* s);
nbgs_status run_comp_ends(nbgs_scene* s);               // bodies of the contact ends (colouring)
nbgs_status build_windows(nbgs_scene* s, int B, int64_t ninc, const uint32_t* ib1, const uint32_t* ib2,
                          const uint32_t* anchor, const uint8_t* finc);   // solve.cu
nbgs_status run_comp_records(nbgs_scene* s, int warm);   // after colouring: inverse inertias, sweep records
nbgs_status run_solve_comp(nbgs_scene* s, int max_sweeps, double tol);
nbgs_status run_integrate_comp(nbgs_scene* s);
nbgs_status run_comp_get_bodies(nbgs_scene* s, double* pos, double* quat, double* vel, double* angvel);
nbgs_status run_comp_set_bodies(nbgs_scene* s, const double* pos, const double* quat, const double* vel,
                                const double* angvel);
void free_composite_buffers(nbgs_scene* s);
nbgs_status run_set_bodies(nbgs_scene* s, const double* pos, const double* quat, const double* vel,
                           const double* angvel);
nbgs_status run_get_bodies(nbgs_scene* s, double* pos, double* quat, double* vel, double* angvel);
nbgs_status run_set_mass(nbgs_scene* s, const double* invm, const double* invI, bool init,
                         const double* radius, const double* density);
nbgs_status run_get_contacts(nbgs_scene* s, int64_t cap, uint32_t* j1, uint32_t* j2, int32_t* colour,
                             double* normal, double* xi, double* impulse);

// primitives (detect.cu)
nbgs_status exclusive_scan_u32(nbgs_scene* s, const uint32_t* in, uint32_t* out, int64_t n,
                               uint32_t* total_dst);
nbgs_status radix_sort_pairs(nbgs_scene* s, uint32_t*& keys, uint32_t*& vals, uint32_t*& keys_alt,
                             uint32_t*& vals_alt, int64_t n, int bits);
nbgs_status exclusive_scan_u32(nbgs_scene* s, const uint32_t* in, uint32_t* out, DCount n, uint32_t* total_dst);
nbgs_status radix_sort_pairs(nbgs_scene* s, uint32_t*& keys, uint32_t*& vals, uint32_t*& keys_alt,
                             uint32_t*& vals_alt, DCount n, int bits);
int grid_for(int64_t work, int threads, int max_blocks_per_sm, int num_sms);
// The contact count of the current step for kernels: host-known, or read on
// the device (device-sized steps; launches sized for the capacity).
inline DCount contact_count(const nbgs_scene* s)
{
    return s->device_sized ? DCount{s->ccap, &s->info->n_contacts} : DCount{s->n_contacts, nullptr};
}
SceneView scene_view(const nbgs_scene* s);

}  // namespace nbgs
