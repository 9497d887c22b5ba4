// noalloc.cu -- residual evaluation that allocates no memory.
//
// For callers that cannot allocate device memory at all: code running where
// cudaMalloc is forbidden or unavailable (inside a fixed memory arena of a
// host application, a plugin that only receives buffers, a process whose
// allocator is owned by someone else).  They hold the contacts and bodies in
// their own device buffers and need the FP64 constraint residuals that
// nbgs_final_residuals() computes for a scene.
//
// The per-block partial maxima live in the file-scope array below instead of
// caller- or scene-allocated scratch.  Every GPU that loads the library holds
// this array (32 KiB) until the process exits.
#include <mutex>

#include "nbgs_internal.cuh"

namespace nbgs {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaPerThread = 8;
constexpr int kNaTile = kNaThreads * kNaPerThread;   // contacts per block
constexpr int kNaMaxBlocks = 1024;
constexpr int64_t kNaMaxContacts = (int64_t)kNaTile * kNaMaxBlocks;   // 2,097,152

// Shared by every call on a device; the last call's partial maxima stay here.
static __device__ __align__(256) double g_na_partial[4 * kNaMaxBlocks];

// Device address of g_na_partial per device, taken with that device current
// (the host-side name is only a stand-in for the device symbol).
constexpr int kNaMaxDevices = 64;
static double* g_na_addr[kNaMaxDevices] = {};
static std::mutex g_na_mutex;

__global__ void __launch_bounds__(kNaThreads)
k_na_partial(int64_t C, int64_t n, const uint32_t* __restrict__ j1, const uint32_t* __restrict__ j2,
             const double* __restrict__ normal, const double* __restrict__ xi, const double* __restrict__ imp,
             const double* __restrict__ vel, const double* __restrict__ ang, const double* __restrict__ radius,
             const double* __restrict__ invm, const double* __restrict__ invI, double dt, double beta, double mu,
             double vr, double* __restrict__ partial)
{
    double m[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t base = (int64_t)blockIdx.x * kNaTile;
    for (int k = 0; k < kNaPerThread; ++k) {
        const int64_t c = base + (int64_t)k * kNaThreads + threadIdx.x;
        if (c >= C) break;
        const uint32_t a = j1[c], b = j2[c];
        const bool dyn_b = b < (uint64_t)n;
        const double nx = normal[3 * c], ny = normal[3 * c + 1], nz = normal[3 * c + 2];
        // lever lengths of a sphere pair / sphere-wall pair: l_a = -(xi + r_a) n, l_b = r_b n
        const double la = xi[c] + radius[a];
        const double lb = dyn_b ? radius[b] : 0.0;
        const double ima = invm[a], iIa = invI[a];
        const double imb = dyn_b ? invm[b] : 0.0, iIb = dyn_b ? invI[b] : 0.0;
        const double wn = ima + imb;
        if (!(wn > 0.0)) continue;
        const double wt = wn + iIa * la * la + iIb * lb * lb;
        double tx, ty, tz, ox, oy, oz;
        tangent_basis<double>(nx, ny, nz, tx, ty, tz, ox, oy, oz);
        const double* va = vel + 3 * (int64_t)a;
        const double* wa = ang + 3 * (int64_t)a;
        double vb[3] = {0.0, 0.0, 0.0}, wb[3] = {0.0, 0.0, 0.0};
        if (dyn_b) {
            for (int e = 0; e < 3; ++e) {
                vb[e] = vel[3 * (int64_t)b + e];
                wb[e] = ang[3 * (int64_t)b + e];
            }
        }
        // u = v_a - la (w_a x n) - v_b - lb (w_b x n)
        const double cax = wa[1] * nz - wa[2] * ny, cay = wa[2] * nx - wa[0] * nz, caz = wa[0] * ny - wa[1] * nx;
        const double cbx = wb[1] * nz - wb[2] * ny, cby = wb[2] * nx - wb[0] * nz, cbz = wb[0] * ny - wb[1] * nx;
        const double ux = (va[0] - la * cax) - (vb[0] + lb * cbx);
        const double uy = (va[1] - la * cay) - (vb[1] + lb * cby);
        const double uz = (va[2] - la * caz) - (vb[2] + lb * cbz);
        const double un = nx * ux + ny * uy + nz * uz;
        const double ut = tx * ux + ty * uy + tz * uz, uo = ox * ux + oy * uy + oz * uz;
        const double pn = imp[3 * c], pt = imp[3 * c + 1], po = imp[3 * c + 2];
        const double xs = xi[c] >= 0.0 ? xi[c] : beta * xi[c];
        const double gn = xs / dt + un;
        const double cone = sqrt(pt * pt + po * po) - mu * pn;
        const double utl = sqrt(ut * ut + uo * uo);
        const double e1 = utl * pt + mu * pn * ut, e2 = utl * po + mu * pn * uo;
        m[0] = fmax(m[0], (gn < 0.0 ? -gn : 0.0) / vr);
        m[1] = fmax(m[1], (cone > 0.0 ? cone : 0.0) * wt / vr);
        m[2] = fmax(m[2], fabs(fmin(wn * pn, gn)) / vr);
        m[3] = fmax(m[3], sqrt(e1 * e1 + e2 * e2) * wt / (vr * vr));
    }
    __shared__ double sm[4][kNaThreads / 32];
    for (int k = 0; k < 4; ++k) {
        double x = m[k];
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
        if ((threadIdx.x & 31) == 0) sm[k][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double x = 0.0;
        for (int w = 0; w < kNaThreads / 32; ++w) x = fmax(x, sm[threadIdx.x][w]);
        partial[4 * blockIdx.x + threadIdx.x] = x;   // every slot this call reads is written first
    }
}

__global__ void k_na_final(int nblocks, const double* __restrict__ partial, double* __restrict__ out)
{
    if (threadIdx.x < 4) {
        double x = 0.0;
        for (int b = 0; b < nblocks; ++b) x = fmax(x, partial[4 * b + threadIdx.x]);
        // as the scene entry point reports them: NaN and anything above 1e300 as +inf
        out[threadIdx.x] = x <= 1e300 ? x : __longlong_as_double(0x7FF0000000000000LL);
    }
}

// Address of the static scratch on the current device, looked up with
// cudaGetSymbolAddress with that device current.  It is looked up again on
// every call whose stream is not being captured (a device reset can reload
// the module elsewhere); a capturing call uses the address cached by an
// earlier call on the device.
nbgs_status na_scratch(cudaStream_t st, double** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
        cudaGetLastError();
        return NBGS_ECUDA;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return NBGS_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev] || cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_na_partial);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return NBGS_ECUDA;
        }
        g_na_addr[dev] = (double*)p;
    }
    *out = g_na_addr[dev];
    return NBGS_OK;
}

}  // namespace
}  // namespace nbgs

extern "C" nbgs_status nbgs_final_residuals_noalloc(int64_t n_bodies, int64_t n_contacts, const uint32_t* j1,
                                                    const uint32_t* j2, const double* normal, const double* xi,
                                                    const double* impulse, const double* vel, const double* angvel,
                                                    const double* radius, const double* invm, const double* invI,
                                                    double dt, double beta, double mu, double v_ref, double* out,
                                                    void* stream)
{
    using namespace nbgs;
    if (n_bodies < 0 || n_contacts < 0 || !out || !(dt > 0.0)) return NBGS_EINVAL;
    if (n_contacts > kNaMaxContacts) return NBGS_ECAPACITY;
    if (n_contacts > 0 && (!j1 || !j2 || !normal || !xi || !impulse || !vel || !angvel || !radius || !invm || !invI))
        return NBGS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    double* partial = nullptr;
    nbgs_status rc = na_scratch(st, &partial);
    if (rc != NBGS_OK) return rc;
    const int nblocks = n_contacts > 0 ? (int)((n_contacts + kNaTile - 1) / kNaTile) : 1;
    const double vr = v_ref > 0.0 ? v_ref : 1e-12;
    k_na_partial<<<nblocks, kNaThreads, 0, st>>>(n_contacts, n_bodies, j1, j2, normal, xi, impulse, vel, angvel,
                                                 radius, invm, invI, dt, beta, mu, vr, partial);
    k_na_final<<<1, 32, 0, st>>>(nblocks, partial, out);
    return cudaGetLastError() == cudaSuccess ? NBGS_OK : NBGS_ECUDA;
}
