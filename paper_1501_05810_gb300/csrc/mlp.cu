// mlp.cu -- learned warm start: a 12 -> 64 -> 64 -> 64 -> 3 MLP (SiLU) that
// predicts a contact's converged impulse from local features, evaluated on
// tensor cores (BF16 operands, FP32 accumulation) before the sweeps, and its
// training kernels (FP32 forward/backward, Adam).
//
// Parameter layout (shared with every user of the network): for each layer
// the weight matrix W (out x in, row-major) then the bias b (out); 9,347
// FP32 values.
//
// Features of a contact (frame n, e2, e3 with e2 = -u_t/|u_t| along the
// free tangential relative velocity, or the contact frame's t when it is
// ~0; e3 = n x e2), all dimensionless:
//   0 u_n / v_ref            1 |u_t| / v_ref         2 (xi/dt) / v_ref
//   3..5 previous-step impulse (n, e2, e3) * w_n / v_ref
//   6 log(w_n)               7 w_t / w_n
//   8 r_a                    9 r_b (0 for a wall)
//   10 mu                    11 (contacts at j1 + contacts at j2) / 12
// u is the relative velocity of the free motion (velocities after the
// gravity kick, no contact impulses).  Output: the impulse in (n, e2, e3)
// times w_n / v_ref, computed as inputs 3..5 (the previous impulse) plus the
// network's correction; it is projected onto the friction cone.  It is used
// for contacts without a previous-step impulse; the others keep theirs (a
// converged previous impulse is far more accurate than any BF16 prediction
// where the contact network persists), as does a non-finite output.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "nbgs_internal.cuh"

namespace nbgs {

constexpr int kIn = 12, kHid = 64, kOutN = 3;
constexpr int kOffW1 = 0, kOffB1 = 768, kOffW2 = 832, kOffB2 = 4928, kOffW3 = 4992, kOffB3 = 9088, kOffW4 = 9152,
              kOffB4 = 9344, kNParams = 9347;

// Shared-memory image of the network for the tensor-core forward: BF16
// weights with padded rows (conflict-free fragment loads), FP32 biases.
constexpr int kS1 = 24;   // layer 1 row stride (12 inputs padded to 16, + 8)
constexpr int kS2 = 72;   // 64-wide rows + 8
struct MlpSmem {
    __nv_bfloat16 w1[kHid * kS1];
    __nv_bfloat16 w2[kHid * kS2];
    __nv_bfloat16 w3[kHid * kS2];
    __nv_bfloat16 w4[8 * kS2];      // 3 outputs padded to 8
    float b1[kHid], b2[kHid], b3[kHid], b4[8];
};

__device__ void load_mlp_smem(const float* __restrict__ th, MlpSmem& S)
{
    for (int k = threadIdx.x; k < kHid * kS1; k += blockDim.x) {
        const int o = k / kS1, i = k % kS1;
        S.w1[k] = __float2bfloat16_rn(i < kIn ? th[kOffW1 + o * kIn + i] : 0.f);
    }
    for (int k = threadIdx.x; k < kHid * kS2; k += blockDim.x) {
        const int o = k / kS2, i = k % kS2;
        S.w2[k] = __float2bfloat16_rn(i < kHid ? th[kOffW2 + o * kHid + i] : 0.f);
        S.w3[k] = __float2bfloat16_rn(i < kHid ? th[kOffW3 + o * kHid + i] : 0.f);
    }
    for (int k = threadIdx.x; k < 8 * kS2; k += blockDim.x) {
        const int o = k / kS2, i = k % kS2;
        S.w4[k] = __float2bfloat16_rn(o < kOutN && i < kHid ? th[kOffW4 + o * kHid + i] : 0.f);
    }
    for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
        S.b1[k] = th[kOffB1 + k];
        S.b2[k] = th[kOffB2 + k];
        S.b3[k] = th[kOffB3 + k];
    }
    if (threadIdx.x < 8) S.b4[threadIdx.x] = threadIdx.x < kOutN ? th[kOffB4 + threadIdx.x] : 0.f;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (low half) = lo
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t ld_u32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + __expf(-z)); }

// One warp evaluates the network on 16 rows.  feat: 16 x 16 FP32 (inputs in
// columns 0..11, zeros after); out: 16 x 8 FP32 (outputs in columns 0..2).
// Fragment layouts of mma.m16n8k16 (g = lane / 4, t = lane % 4):
//   A: {row g, cols 2t,2t+1}, {row g+8, 2t,2t+1}, {row g, 2t+8,2t+9}, {row g+8, 2t+8,2t+9}
//   B: {k 2t,2t+1; col g}, {k 2t+8,2t+9; col g}
//   C: {row g, col 2t}, {row g, 2t+1}, {row g+8, 2t}, {row g+8, 2t+1}
// The accumulators of column tiles 2k and 2k+1 are exactly the A fragment of
// k-block k of the next layer, so activations stay in registers.
__device__ void mlp_warp(const MlpSmem& S, const float (*feat)[16], float (*out)[8])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t A[4][4];
    {
        const uint32_t a0 = pack_bf16(feat[g][2 * t], feat[g][2 * t + 1]);
        const uint32_t a1 = pack_bf16(feat[g + 8][2 * t], feat[g + 8][2 * t + 1]);
        const uint32_t a2 = pack_bf16(feat[g][2 * t + 8], feat[g][2 * t + 9]);
        const uint32_t a3 = pack_bf16(feat[g + 8][2 * t + 8], feat[g + 8][2 * t + 9]);
        float acc[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            acc[j][0] = acc[j][2] = S.b1[8 * j + 2 * t];
            acc[j][1] = acc[j][3] = S.b1[8 * j + 2 * t + 1];
            const __nv_bfloat16* w = S.w1 + (8 * j + g) * kS1 + 2 * t;
            mma_bf16(acc[j], a0, a1, a2, a3, ld_u32(w), ld_u32(w + 8));
        }
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
            A[kb][0] = pack_bf16(silu_f(acc[2 * kb][0]), silu_f(acc[2 * kb][1]));
            A[kb][1] = pack_bf16(silu_f(acc[2 * kb][2]), silu_f(acc[2 * kb][3]));
            A[kb][2] = pack_bf16(silu_f(acc[2 * kb + 1][0]), silu_f(acc[2 * kb + 1][1]));
            A[kb][3] = pack_bf16(silu_f(acc[2 * kb + 1][2]), silu_f(acc[2 * kb + 1][3]));
        }
    }
#pragma unroll
    for (int layer = 0; layer < 2; ++layer) {
        const __nv_bfloat16* W = layer == 0 ? S.w2 : S.w3;
        const float* b = layer == 0 ? S.b2 : S.b3;
        float acc[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            acc[j][0] = acc[j][2] = b[8 * j + 2 * t];
            acc[j][1] = acc[j][3] = b[8 * j + 2 * t + 1];
        }
#pragma unroll
        for (int kb = 0; kb < 4; ++kb)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const __nv_bfloat16* w = W + (8 * j + g) * kS2 + 16 * kb + 2 * t;
                mma_bf16(acc[j], A[kb][0], A[kb][1], A[kb][2], A[kb][3], ld_u32(w), ld_u32(w + 8));
            }
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
            A[kb][0] = pack_bf16(silu_f(acc[2 * kb][0]), silu_f(acc[2 * kb][1]));
            A[kb][1] = pack_bf16(silu_f(acc[2 * kb][2]), silu_f(acc[2 * kb][3]));
            A[kb][2] = pack_bf16(silu_f(acc[2 * kb + 1][0]), silu_f(acc[2 * kb + 1][1]));
            A[kb][3] = pack_bf16(silu_f(acc[2 * kb + 1][2]), silu_f(acc[2 * kb + 1][3]));
        }
    }
    float acc[4];
    acc[0] = acc[2] = S.b4[2 * t];
    acc[1] = acc[3] = S.b4[2 * t + 1];
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
        const __nv_bfloat16* w = S.w4 + g * kS2 + 16 * kb + 2 * t;
        mma_bf16(acc, A[kb][0], A[kb][1], A[kb][2], A[kb][3], ld_u32(w), ld_u32(w + 8));
    }
    out[g][2 * t] = acc[0];
    out[g][2 * t + 1] = acc[1];
    out[g + 8][2 * t] = acc[2];
    out[g + 8][2 * t + 1] = acc[3];
}

// --- plain inference on given rows (tests, evaluation) ------------------------
constexpr int kMlpWarps = 8;

__global__ void __launch_bounds__(32 * kMlpWarps) k_mlp_infer(const float* __restrict__ theta, const float* __restrict__ X,
                                                              float* __restrict__ Y, int64_t n)
{
    __shared__ MlpSmem S;
    __shared__ float feat[kMlpWarps][16][16];
    __shared__ float out[kMlpWarps][16][8];
    load_mlp_smem(theta, S);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t base = ((int64_t)blockIdx.x * kMlpWarps + w) * 16; base < n; base += (int64_t)gridDim.x * kMlpWarps * 16) {
        if (lane < 16) {
            const int64_t r = base + lane;
            for (int k = 0; k < 16; ++k) feat[w][lane][k] = (r < n && k < kIn) ? X[r * kIn + k] : 0.f;
        }
        __syncwarp();
        mlp_warp(S, feat[w], out[w]);
        __syncwarp();
        if (lane < 16 && base + lane < n)   // skip connection: + previous impulse (inputs 3..5), in FP32
            for (int k = 0; k < kOutN; ++k) Y[(base + lane) * kOutN + k] = out[w][lane][k] + feat[w][lane][3 + k];
        __syncwarp();
    }
}

// --- training: FP32 forward + backward on CUDA cores --------------------------
constexpr int kTile = 32;        // samples per tile
constexpr int kTrainThreads = 256;

struct TrainSmem {
    float th[kNParams];
    float gr[kNParams];
    float x[kTile][kIn];
    float z[3][kTile][kHid];     // pre-activations of the hidden layers
    float d[2][kTile][kHid];     // back-propagated deltas
    float y[kTile][4];           // output, then dL/dY
};

__device__ __forceinline__ float act(const TrainSmem& S, int layer, int s, int i)
{
    // input of layer `layer` (0 = network input)
    return layer == 0 ? S.x[s][i] : silu_f(S.z[layer - 1][s][i]);
}

__device__ __forceinline__ float silu_grad_f(float z)
{
    const float sg = 1.f / (1.f + __expf(-z));
    return sg * (1.f + z * (1.f - sg));
}

__global__ void __launch_bounds__(kTrainThreads) k_mlp_grad(const float* __restrict__ theta, const float* __restrict__ X,
                                                            const float* __restrict__ T, int64_t n,
                                                            float* __restrict__ grad, double* __restrict__ loss)
{
    extern __shared__ __align__(16) unsigned char train_smem[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(train_smem);
    for (int k = threadIdx.x; k < kNParams; k += blockDim.x) {
        S.th[k] = theta[k];
        S.gr[k] = 0.f;
    }
    const int offW[4] = {kOffW1, kOffW2, kOffW3, kOffW4}, offB[4] = {kOffB1, kOffB2, kOffB3, kOffB4};
    const int nin[4] = {kIn, kHid, kHid, kHid}, nout[4] = {kHid, kHid, kHid, kOutN};
    const float inv_n = 1.f / (float)n;
    double lsum = 0.0;
    __syncthreads();
    for (int64_t base = (int64_t)blockIdx.x * kTile; base < n; base += (int64_t)gridDim.x * kTile) {
        const int m = (int)(n - base < kTile ? n - base : kTile);
        for (int k = threadIdx.x; k < kTile * kIn; k += blockDim.x) {
            const int s = k / kIn, i = k % kIn;
            S.x[s][i] = s < m ? X[(base + s) * kIn + i] : 0.f;
        }
        __syncthreads();
        // forward: z_L = W_L a_{L-1} + b_L
        for (int L = 0; L < 4; ++L) {
            for (int k = threadIdx.x; k < kTile * nout[L]; k += blockDim.x) {
                const int s = k / nout[L], o = k % nout[L];
                float z = S.th[offB[L] + o];
                const float* w = S.th + offW[L] + o * nin[L];
                for (int i = 0; i < nin[L]; ++i) z += w[i] * act(S, L, s, i);
                if (L < 3) S.z[L][s][o] = z;
                else S.y[s][o] = z + S.x[s][3 + o];   // skip connection: + previous impulse
            }
            __syncthreads();
        }
        // loss and dL/dY = (Y - T) / n (rows beyond m contribute nothing)
        for (int k = threadIdx.x; k < kTile * kOutN; k += blockDim.x) {
            const int s = k / kOutN, o = k % kOutN;
            float dy = 0.f;
            if (s < m) {
                const float e = S.y[s][o] - T[(base + s) * kOutN + o];
                lsum += 0.5 * (double)e * (double)e;
                dy = e * inv_n;
            }
            S.y[s][o] = dy;
        }
        __syncthreads();
        // backward, layer 4 .. 1; delta of layer L lives in y (L = 3) or d[L % 2]
        for (int L = 3; L >= 0; --L) {
            const int no = nout[L], ni = nin[L];
            auto delta = [&](int s, int o) -> float { return L == 3 ? S.y[s][o] : S.d[L & 1][s][o]; };
            // weight and bias gradients: each thread owns whole entries
            for (int k = threadIdx.x; k < no * ni + no; k += blockDim.x) {
                float acc = 0.f;
                if (k < no * ni) {
                    const int o = k / ni, i = k % ni;
                    for (int s = 0; s < m; ++s) acc += delta(s, o) * act(S, L, s, i);
                    S.gr[offW[L] + k] += acc;
                } else {
                    const int o = k - no * ni;
                    for (int s = 0; s < m; ++s) acc += delta(s, o);
                    S.gr[offB[L] + o] += acc;
                }
            }
            if (L > 0) {   // delta of layer L - 1: (W_L^T delta_L) * silu'(z_{L-1})
                for (int k = threadIdx.x; k < kTile * ni; k += blockDim.x) {
                    const int s = k / ni, i = k % ni;
                    float acc = 0.f;
                    for (int o = 0; o < no; ++o) acc += S.th[offW[L] + o * ni + i] * delta(s, o);
                    S.d[(L - 1) & 1][s][i] = acc * silu_grad_f(S.z[L - 1][s][i]);
                }
            }
            __syncthreads();
        }
    }
    for (int k = threadIdx.x; k < kNParams; k += blockDim.x) atomicAdd(&grad[k], S.gr[k]);
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, lsum / (double)n);
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t count, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        th[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
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
    const double4_32a* cgeo;     // canonical (n, xi)
    float* feat_out;             // optional: canonical order, 16 per contact (12 features, cos, sin, w_n, v_ref)
    int apply;                   // 0: features only
    double gdt[3];
    double gdt_norm;
    double dt;
    double mu;
    SceneView V;
    const DevInfo* info;
};

template <class R>
__global__ void __launch_bounds__(32 * kMlpWarps) k_mlp_warmstart(WarmArgs<R> A)
{
    __shared__ MlpSmem S;
    __shared__ float feat[kMlpWarps][16][16];
    __shared__ float out[kMlpWarps][16][8];
    if (A.apply) load_mlp_smem(A.theta, S);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double vr_all = fmax(fmax(__longlong_as_double((long long)A.info->vmax_bits), A.gdt_norm), 1e-12);
    for (int64_t base = ((int64_t)blockIdx.x * kMlpWarps + w) * 16; base < A.C;
         base += (int64_t)gridDim.x * kMlpWarps * 16) {
        const int64_t s = base + lane;
        const bool live = lane < 16 && s < A.C;
        double nx = 0, ny = 0, nz = 0, tx = 0, ty = 0, tz = 0, ox = 0, oy = 0, oz = 0, cth = 1, sth = 0, wn = 1, vr = 1,
               mu = A.mu;
        R4<R> p0;
        p0.x = p0.y = p0.z = p0.w = R(0);
        if (live) {
            const SweepRec<R> rr = A.rec[s];
            uint32_t ia, ib;
            double la, lb, bias;
            if constexpr (sizeof(R) == 4) {
                ia = __float_as_uint(rr.a.x);
                ib = __float_as_uint(rr.a.y);
                la = rr.a.z;
                lb = rr.a.w;
                nx = rr.b.x;
                ny = rr.b.y;
                nz = rr.b.z;
            } else {
                const uint64_t ids = (uint64_t)__double_as_longlong(rr.ids_bias.x);
                ia = (uint32_t)(ids & 0xFFFFFFFFu);
                ib = (uint32_t)(ids >> 32);
                la = rr.lev.x;
                lb = rr.lev.y;
                nx = rr.nxy.x;
                ny = rr.nxy.y;
                nz = rr.nz_.x;
            }
            (void)bias;
            p0 = A.p[s];
            const bool dyn_b = ib < (uint64_t)A.n;
            const R4<R> va = A.vel[2 * (int64_t)ia], wa = A.vel[2 * (int64_t)ia + 1];
            R4<R> vb, wb;
            vb.x = vb.y = vb.z = vb.w = R(0);
            wb = vb;
            if (dyn_b) {
                vb = A.vel[2 * (int64_t)ib];
                wb = A.vel[2 * (int64_t)ib + 1];
            }
            if (A.V.batch) {
                const uint32_t sc = A.V.scene_of[ia];
                vr = A.V.vref[sc];
                mu = A.V.mu[sc];
            } else {
                vr = vr_all;
            }
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
            if (utl > 1e-12 * vr) {   // e2 = -u_t / |u_t| = cos t + sin o
                cth = -ut / utl;
                sth = -uo / utl;
            }
            wn = (double)va.w + (double)vb.w;
            const double wt = wn + (double)wa.w * la * la + (double)wb.w * lb * lb;
            // previous impulse in (n, e2, e3): e3 = -sin t + cos o
            const double q2 = p0.y * cth + p0.z * sth, q3 = -p0.y * sth + p0.z * cth;
            const double sc = wn / vr;
            const double ra = A.pos_r[ia].w, rb = dyn_b ? A.pos_r[ib].w : 0.0;
            const uint32_t da = A.finite[ia] ? A.adj_off[ia + 1] - A.adj_off[ia] : 0;
            const uint32_t db = (dyn_b && A.finite[ib]) ? A.adj_off[ib + 1] - A.adj_off[ib] : 0;
            const uint32_t cidx = A.perm[s];
            const double xi_dt = A.cgeo[cidx].w / A.dt;   // the geometric gap, not the beta-scaled term
            const double f[14] = {un / vr,       utl / vr,      xi_dt / vr,     p0.x * sc,  q2 * sc,
                                  q3 * sc,       log(fmax(wn, 1e-300)), wt / wn, ra,       rb,
                                  mu,            (double)(da + db) / 12.0, cth, sth};
            for (int k = 0; k < 16; ++k) feat[w][lane][k] = k < kIn ? (float)f[k] : 0.f;
            if (A.feat_out) {
                float* o = A.feat_out + (int64_t)cidx * 16;
                for (int k = 0; k < 14; ++k) o[k] = (float)f[k];
                o[14] = (float)wn;
                o[15] = (float)vr;
            }
        } else if (lane < 16) {
            for (int k = 0; k < 16; ++k) feat[w][lane][k] = 0.f;
        }
        if (!A.apply) continue;
        __syncwarp();
        mlp_warp(S, feat[w], out[w]);
        __syncwarp();
        // a contact with a previous-step impulse keeps it; the network
        // predicts the impulses of contacts that had none
        if (live && p0.w == R(0)) {
            const double k = vr / wn;   // skip connection: previous impulse + network correction
            const double y1 = ((double)out[w][lane][0] + feat[w][lane][3]) * k;
            const double y2 = ((double)out[w][lane][1] + feat[w][lane][4]) * k;
            const double y3 = ((double)out[w][lane][2] + feat[w][lane][5]) * k;
            double pn = y1, pt = y2 * cth - y3 * sth, po = y2 * sth + y3 * cth;
            if (isfinite(pn) && isfinite(pt) && isfinite(po)) {   // otherwise keep the previous-step impulse
                pn = pn > 0.0 ? pn : 0.0;
                const double lim = mu * pn, len = sqrt(pt * pt + po * po);
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
        __syncwarp();
    }
}

template <class R>
static WarmArgs<R> warm_args(nbgs_scene* s, int apply, float* feat_out)
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

// Features (and, with apply, the network's warm start) for the current
// contacts; runs before the sweeps (after colouring, before the gravity kick).
nbgs_status run_mlp_prologue(nbgs_scene* s, int apply, float* feat_out)
{
    const int64_t C = s->n_contacts;
    if (C <= 0) return NBGS_OK;
    if (apply && !s->mlp_theta) return fail(s, NBGS_EINVAL, "MLP warm start: no network loaded (nbgs_mlp_load)");
    const int T = 32 * kMlpWarps;
    const int64_t groups = (C + 15) / 16;
    const int gb = grid_for(groups * 32, T, 4, s->num_sms);
    if (s->fp32) k_mlp_warmstart<float><<<gb, T, 0, s->stream>>>(warm_args<float>(s, apply, feat_out));
    else k_mlp_warmstart<double><<<gb, T, 0, s->stream>>>(warm_args<double>(s, apply, feat_out));
    if (s->timing) s->phase_launches[2] += 1;
    return cuda_check(s, cudaGetLastError(), "MLP prologue");
}

}  // namespace nbgs

using namespace nbgs;

extern "C" {

nbgs_status nbgs_mlp_infer(const float* theta, const float* X, float* Y, int64_t n, void* stream)
{
    if (!theta || n < 0 || (n > 0 && (!X || !Y))) return NBGS_EINVAL;
    if (n == 0) return NBGS_OK;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t groups = (n + 15) / 16;
    k_mlp_infer<<<grid_for(groups * 32, 32 * kMlpWarps, 4, sms), 32 * kMlpWarps, 0, (cudaStream_t)stream>>>(theta, X, Y,
                                                                                                         n);
    return cudaGetLastError() == cudaSuccess ? NBGS_OK : NBGS_ECUDA;
}

nbgs_status nbgs_mlp_grad(const float* theta, const float* X, const float* T, int64_t n, float* grad, double* loss,
                          void* stream)
{
    if (!theta || !grad || !loss || n <= 0 || !X || !T) return NBGS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    static_assert(sizeof(TrainSmem) < 227 * 1024, "training tile too large");
    if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem)) !=
        cudaSuccess)
        return NBGS_ECUDA;
    cudaMemsetAsync(grad, 0, kNParams * sizeof(float), st);
    cudaMemsetAsync(loss, 0, sizeof(double), st);
    const int64_t tiles = (n + kTile - 1) / kTile;
    const int blocks = (int)std::min<int64_t>(tiles, (int64_t)sms);
    k_mlp_grad<<<blocks, kTrainThreads, sizeof(TrainSmem), st>>>(theta, X, T, n, grad, loss);
    return cudaGetLastError() == cudaSuccess ? NBGS_OK : NBGS_ECUDA;
}

nbgs_status nbgs_mlp_adam(float* theta, const float* grad, float* m, float* v, int64_t count, float lr, float beta1,
                          float beta2, float eps, int32_t step, void* stream)
{
    if (!theta || !grad || !m || !v || count <= 0 || step < 1) return NBGS_EINVAL;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_adam<<<(int)((count + 255) / 256), 256, 0, (cudaStream_t)stream>>>(theta, grad, m, v, count, lr, beta1, beta2, eps,
                                                                        c1, c2);
    return cudaGetLastError() == cudaSuccess ? NBGS_OK : NBGS_ECUDA;
}

nbgs_status nbgs_mlp_load(nbgs_scene* s, const float* theta, int64_t count)
{
    if (!s) return NBGS_EINVAL;
    if (s->status != NBGS_OK) return s->status;
    if (!theta || count != kNParams) return fail(s, NBGS_EINVAL, "mlp_load: expected 9347 parameters");
    if (!s->mlp_theta) {
        s->mlp_theta = (float*)dev_alloc(s, kNParams * sizeof(float));
        if (!s->mlp_theta) return fail(s, NBGS_ENOMEM, "mlp_load: allocation");
    }
    return cuda_check(s, cudaMemcpyAsync(s->mlp_theta, theta, kNParams * sizeof(float), cudaMemcpyDefault, s->stream),
                      "mlp_load");
}

nbgs_status nbgs_mlp_features(nbgs_scene* s, float* out, int64_t cap, int64_t* n_out)
{
    if (!s) return NBGS_EINVAL;
    if (s->status != NBGS_OK) return s->status;
    if (!s->coloured) return fail(s, NBGS_EINVAL, "mlp_features: detect and colour the contacts first");
    if (n_out) *n_out = s->n_contacts;
    if (!out || cap < s->n_contacts || s->n_contacts == 0) return NBGS_OK;
    float* buf = (float*)dev_alloc(s, (size_t)s->n_contacts * 16 * sizeof(float));
    if (!buf) return fail(s, NBGS_ENOMEM, "mlp_features: staging");
    nbgs_status rc = run_mlp_prologue(s, 0, buf);
    if (rc == NBGS_OK)
        rc = cuda_check(s, cudaMemcpyAsync(out, buf, (size_t)s->n_contacts * 16 * sizeof(float), cudaMemcpyDefault,
                                           s->stream), "mlp_features");
    if (rc == NBGS_OK) rc = cuda_check(s, cudaStreamSynchronize(s->stream), "mlp_features");
    dev_free(s, buf);
    return rc;
}

}  // extern "C"
