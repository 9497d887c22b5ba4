// mlp.cu -- learned warm start: a 12 -> 64 -> 64 -> 64 -> 3 MLP (SiLU) that
// predicts a contact's converged impulse from local features, evaluated on
// the 5th-generation tensor cores (tcgen05: BF16 operands in shared memory,
// FP32 accumulators in TMEM) before the sweeps, and its training kernels
// (forward and backward on the tensor cores, Adam).
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
#include <algorithm>
#include <cmath>

#include "mlp_tc.cuh"

namespace nbgs {

__device__ unsigned g_mlp_status;   // nbgs_mlp_infer: a tensor-core wait gave up

// --- plain inference on given rows (tests, evaluation) ------------------------
__global__ void __launch_bounds__(kTcRows) k_mlp_infer_tc(const float* __restrict__ theta, const float* __restrict__ X,
                                                          float* __restrict__ Y, int64_t n)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    TcMlpSmem& S = *reinterpret_cast<TcMlpSmem*>(tc_smem);
    tc_setup(theta, S);
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t base = (int64_t)blockIdx.x * kTcRows; base < n; base += (int64_t)gridDim.x * kTcRows) {
        const int64_t row = base + threadIdx.x;
        float in[kIn], out[kOutN];
        if (row < n) {   // a row is 48 bytes: three 16-byte loads (X is 16-byte aligned)
            const float4* xr = reinterpret_cast<const float4*>(X + row * kIn);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float4 v = xr[q];
                in[4 * q] = v.x;
                in[4 * q + 1] = v.y;
                in[4 * q + 2] = v.z;
                in[4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kIn; ++k) in[k] = 0.f;
        }
        if (ok && !tc_forward(S, in, out, phase)) {   // a wait gave up (uniform): NaN from here on
            ok = false;
            if (threadIdx.x == 0) atomicOr(&g_mlp_status, 1u);
        }
        if (row < n)   // skip connection: + previous impulse (inputs 3..5), in FP32
            for (int k = 0; k < kOutN; ++k) Y[row * kOutN + k] = ok ? out[k] + in[3 + k] : __int_as_float(0x7FC00000);
    }
    tc_teardown(S);
}

// --- training: forward and backward on the tensor cores (tcgen05) -----------
// One CTA per SM, 128 threads, 128 samples per tile, thread r sample r.  All
// products are tcgen05.mma with BF16 operands in shared memory (K-major, no
// swizzle) and FP32 accumulators in TMEM:
//   forward   Z_L   = A_{L-1} W_L^T        (M 128 samples, N out, K in)
//   backward  B_L   = D_L W_L              (M 128 samples, N in, K out)
//             dW_L += D_L^T A_{L-1}        (M out, padded to 128, N in, K 128 samples)
// with D_4 = (Y - T) / n, D_{L-1} = B_L * silu'(Z_{L-1} + b_{L-1}).  The
// pre-activations stay in TMEM for the backward pass; every A_L and D_L is
// written twice, sample-major for the products that run over features and
// feature-major for the weight gradients, which run over samples; the weight
// gradients accumulate in TMEM over all tiles of the CTA and are added to
// the global gradient once.  Bias gradients and the loss: FP32 sums of the
// unrounded deltas on the CUDA cores.
constexpr int kTrRows = 128;
constexpr int kTrCols = 512;                       // TMEM columns (one CTA per SM)
constexpr uint32_t kZ1 = 0, kZ2 = 64, kZ3 = 128, kZ4 = 192, kBk = 208;   // TMEM column offsets
constexpr uint32_t kDW1 = 272, kDW2 = 288, kDW3 = 352, kDW4 = 416;

struct TrainTcSmem {
    alignas(128) __nv_bfloat16 a0[kTrRows * 16];           // inputs, sample-major (K 16)
    alignas(128) __nv_bfloat16 a[3][kTrRows * kHid];       // hidden activations, sample-major
    alignas(128) __nv_bfloat16 a0t[16 * kTrRows];          // inputs, feature-major (K 128 samples)
    alignas(128) __nv_bfloat16 at[3][kHid * kTrRows];      // hidden activations, feature-major
    alignas(128) __nv_bfloat16 d[kTrRows * kHid];          // deltas, sample-major (K = layer outputs)
    alignas(128) __nv_bfloat16 dt[kTrRows * kTrRows];      // deltas, output-major, rows >= outputs unused
    alignas(128) __nv_bfloat16 w1[kHid * 16];              // W_L (rows = outputs, K = inputs)
    alignas(128) __nv_bfloat16 w2[kHid * kHid];
    alignas(128) __nv_bfloat16 w3[kHid * kHid];
    alignas(128) __nv_bfloat16 w4[16 * kHid];
    alignas(128) __nv_bfloat16 w2t[kHid * kHid];           // W_L^T (rows = inputs, K = outputs)
    alignas(128) __nv_bfloat16 w3t[kHid * kHid];
    alignas(128) __nv_bfloat16 w4t[kHid * 16];
    float b1[kHid], b2[kHid], b3[kHid], b4[16];
    float gb[kHid * 3 + 16];                                // bias gradients b1, b2, b3, b4
    alignas(8) uint64_t bar;
    uint32_t tmem;
};

__device__ __forceinline__ void st_bf16(__nv_bfloat16* base, uint32_t byte_off, float v)
{
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(base) + byte_off) = __float2bfloat16_rn(v);
}

// Row r (< 128) of a sample-major operand with K columns from 2K FP32 values
// (K a multiple of 8), eight columns per 16-byte store.
__device__ __forceinline__ void st_row(__nv_bfloat16* base, int r, int K, const float* v)
{
    for (int c0 = 0; c0 < K; c0 += 8) {
        const uint4 q = make_uint4(pack_bf16(v[c0], v[c0 + 1]), pack_bf16(v[c0 + 2], v[c0 + 3]),
                                   pack_bf16(v[c0 + 4], v[c0 + 5]), pack_bf16(v[c0 + 6], v[c0 + 7]));
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(base) + kmaj_off(r, c0, K)) = q;
    }
}

// Column r of a feature-major operand (rows = features, K = 128 samples).
__device__ __forceinline__ void st_col(__nv_bfloat16* base, int r, int nfeat, const float* v)
{
    for (int f = 0; f < nfeat; ++f) st_bf16(base, kmaj_off(f, r, kTrRows), v[f]);
}

// 64 FP32 columns of this thread's TMEM lane (row) starting at column col.
__device__ __forceinline__ void tm_row64(uint32_t tmem, uint32_t col, float (&v)[64])
{
    const uint32_t lane = (uint32_t)(32 * (threadIdx.x >> 5)) << 16;
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
        float t[16];
        tc_ld16(tmem + lane + col + (uint32_t)c0, t);
#pragma unroll
        for (int k = 0; k < 16; ++k) v[c0 + k] = t[k];
    }
}

// K/16 MMAs D(+)= A B^T of an M = 128 product; acc: accumulate into D from the first slice on.
__device__ __forceinline__ void tr_mma(uint32_t d, const void* a, const void* b, int K, int N, bool acc)
{
    const uint32_t sa = smem_addr(a), sb = smem_addr(b);
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    for (int kk = 0; kk < K / 16; ++kk)
        tc_mma(d, tc_desc(sa + 256u * kk, 128u, sbo), tc_desc(sb + 256u * kk, 128u, sbo), tc_idesc(kTrRows, N),
               (acc || kk > 0) ? 1 : 0);
}

// Operands written by every thread -> barrier -> thread 0 issues (issue())
// and commits -> all wait.  False when the wait gave up (same on all threads).
template <class F>
__device__ __forceinline__ bool tr_step(TrainTcSmem& S, uint32_t& phase, F issue)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        issue();
        tc_commit(&S.bar);
    }
    const bool ok = tc_wait(&S.bar, phase & 1u);
    phase += 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return __syncthreads_and(ok) != 0;
}

__device__ __forceinline__ float silu_grad_f(float z)
{
    const float sg = 1.f / (1.f + __expf(-z));
    return sg * (1.f + z * (1.f - sg));
}

// Sum over the CTA's 128 rows of v[0..m) into gb[0..m) (shared memory).
__device__ __forceinline__ void bias_grad(float* gb, const float* v, int m)
{
    for (int o = 0; o < m; ++o) {
        float x = v[o];
        for (int k = 16; k > 0; k >>= 1) x += __shfl_xor_sync(0xffffffffu, x, k);
        if ((threadIdx.x & 31) == 0) atomicAdd(&gb[o], x);
    }
}

__global__ void __launch_bounds__(kTrRows, 1) k_mlp_grad_tc(const float* __restrict__ th, const float* __restrict__ X,
                                                            const float* __restrict__ T, int64_t n,
                                                            float* __restrict__ grad, double* __restrict__ loss,
                                                            unsigned* status)
{
    extern __shared__ __align__(1024) unsigned char tr_smem[];
    TrainTcSmem& S = *reinterpret_cast<TrainTcSmem*>(tr_smem);
    const int r = threadIdx.x;
    // weights in both layouts, biases, bias gradients, the unused delta rows
    for (int e = r; e < kHid * 16; e += kTrRows) {
        const int o = e / 16, i = e % 16;
        st_bf16(S.w1, kmaj_off(o, i, 16), i < kIn ? th[kOffW1 + o * kIn + i] : 0.f);
    }
    for (int e = r; e < kHid * kHid; e += kTrRows) {
        const int o = e / kHid, i = e % kHid;
        const float w2 = th[kOffW2 + o * kHid + i], w3 = th[kOffW3 + o * kHid + i];
        st_bf16(S.w2, kmaj_off(o, i, kHid), w2);
        st_bf16(S.w3, kmaj_off(o, i, kHid), w3);
        st_bf16(S.w2t, kmaj_off(i, o, kHid), w2);
        st_bf16(S.w3t, kmaj_off(i, o, kHid), w3);
    }
    for (int e = r; e < 16 * kHid; e += kTrRows) {
        const int o = e / kHid, i = e % kHid;
        const float w = o < kOutN ? th[kOffW4 + o * kHid + i] : 0.f;
        st_bf16(S.w4, kmaj_off(o, i, kHid), w);
        st_bf16(S.w4t, kmaj_off(i, o, 16), w);
    }
    for (int k = r; k < kHid; k += kTrRows) {
        S.b1[k] = th[kOffB1 + k];
        S.b2[k] = th[kOffB2 + k];
        S.b3[k] = th[kOffB3 + k];
    }
    if (r < 16) S.b4[r] = r < kOutN ? th[kOffB4 + r] : 0.f;
    for (int k = r; k < kHid * 3 + 16; k += kTrRows) S.gb[k] = 0.f;
    for (int e = r; e < kTrRows * kTrRows; e += kTrRows) S.dt[e] = __float2bfloat16_rn(0.f);
    if (r == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.bar)) : "memory");
    if (r < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&S.tmem)),
                     "r"(kTrCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tm = S.tmem;
    const float inv_n = 1.f / (float)n;
    double lsum = 0.0;
    uint32_t phase = 0;
    bool ok = true, first = true;
    __nv_bfloat16* const A[4] = {S.a0, S.a[0], S.a[1], S.a[2]};
    for (int64_t base = (int64_t)blockIdx.x * kTrRows; base < n && ok; base += (int64_t)gridDim.x * kTrRows) {
        const int64_t row = base + r;
        const bool valid = row < n;
        float x[16], t[kOutN];
#pragma unroll
        for (int k = 0; k < 16; ++k) x[k] = (valid && k < kIn) ? X[row * kIn + k] : 0.f;
#pragma unroll
        for (int k = 0; k < kOutN; ++k) t[k] = valid ? T[row * kOutN + k] : 0.f;
        st_row(S.a0, r, 16, x);
        st_col(S.a0t, r, 16, x);
        // forward
        const uint32_t zc[4] = {kZ1, kZ2, kZ3, kZ4};
        const __nv_bfloat16* W[4] = {S.w1, S.w2, S.w3, S.w4};
        const float* bias[3] = {S.b1, S.b2, S.b3};
        for (int L = 0; L < 4 && ok; ++L) {
            const int K = L == 0 ? 16 : kHid, N = L == 3 ? 16 : kHid;
            ok = tr_step(S, phase, [&] { tr_mma(tm + zc[L], A[L], W[L], K, N, false); });
            if (!ok) break;
            if (L < 3) {
                float z[64];
                tm_row64(tm, zc[L], z);
#pragma unroll
                for (int k = 0; k < 64; ++k) z[k] = silu_fast(z[k] + bias[L][k]);
                st_row(A[L + 1], r, kHid, z);
                st_col(S.at[L], r, kHid, z);
            }
        }
        if (!ok) break;
        // output, loss, D_4
        {
            float y[16];
            tc_ld16(tm + ((uint32_t)(32 * (r >> 5)) << 16) + kZ4, y);
            float d4[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) d4[k] = 0.f;
#pragma unroll
            for (int k = 0; k < kOutN; ++k) {
                const float e = valid ? (y[k] + S.b4[k] + x[3 + k]) - t[k] : 0.f;
                lsum += 0.5 * (double)e * (double)e;
                d4[k] = e * inv_n;
            }
            st_row(S.d, r, 16, d4);
            st_col(S.dt, r, 16, d4);
            bias_grad(S.gb + 3 * kHid, d4, kOutN);
        }
        // backward: layer 4 .. 1
        const uint32_t dwc[4] = {kDW1, kDW2, kDW3, kDW4};
        const __nv_bfloat16* WT[4] = {nullptr, S.w2t, S.w3t, S.w4t};
        const __nv_bfloat16* AT[4] = {S.a0t, S.at[0], S.at[1], S.at[2]};
        for (int L = 3; L >= 0 && ok; --L) {
            const int Kout = L == 3 ? 16 : kHid, Nin = L == 0 ? 16 : kHid;
            const bool acc = !first;
            ok = tr_step(S, phase, [&] {
                tr_mma(tm + dwc[L], S.dt, AT[L], kTrRows, Nin, acc);      // dW_L (+)= D_L^T A_{L-1}
                if (L > 0) tr_mma(tm + kBk, S.d, WT[L], Kout, kHid, false);   // B_L = D_L W_L
            });
            if (!ok || L == 0) break;
            float bk[64], z[64];
            tm_row64(tm, kBk, bk);
            tm_row64(tm, zc[L - 1], z);
#pragma unroll
            for (int k = 0; k < 64; ++k) bk[k] *= silu_grad_f(z[k] + bias[L - 1][k]);
            st_row(S.d, r, kHid, bk);
            st_col(S.dt, r, kHid, bk);
            bias_grad(S.gb + (L - 1) * kHid, bk, kHid);
        }
        first = false;
    }
    if (!ok && r == 0) atomicOr(status, 1u);
    // weight gradients: rows (outputs) of the TMEM accumulators, lanes 0..63
    // (warps 0 and 1; the rows of warps 2 and 3 are padding)
    if (ok && !first && r < kHid) {
        float v[64];
        tm_row64(tm, kDW2, v);
        for (int i = 0; i < kHid; ++i) atomicAdd(&grad[kOffW2 + r * kHid + i], v[i]);
        tm_row64(tm, kDW3, v);
        for (int i = 0; i < kHid; ++i) atomicAdd(&grad[kOffW3 + r * kHid + i], v[i]);
        tm_row64(tm, kDW4, v);
        if (r < kOutN)
            for (int i = 0; i < kHid; ++i) atomicAdd(&grad[kOffW4 + r * kHid + i], v[i]);
        float w[16];
        tc_ld16(tm + ((uint32_t)(32 * (r >> 5)) << 16) + kDW1, w);
        for (int i = 0; i < kIn; ++i) atomicAdd(&grad[kOffW1 + r * kIn + i], w[i]);
    }
    __syncthreads();
    if (ok && !first) {
        const int boff[4] = {kOffB1, kOffB2, kOffB3, kOffB4};
        for (int k = r; k < kHid * 3 + kOutN; k += kTrRows) atomicAdd(&grad[boff[k / kHid] + k % kHid], S.gb[k]);
    }
    for (int k = 16; k > 0; k >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, k);
    if ((r & 31) == 0 && lsum != 0.0) atomicAdd(loss, lsum / (double)n);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (r < 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kTrCols) : "memory");
    }
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

// One CTA: 128 contacts per tile (warm_tiles).
template <class R>
__global__ void __launch_bounds__(kTcRows) k_mlp_warmstart(WarmArgs<R> A)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    warm_tiles<R>(A, A.apply ? reinterpret_cast<TcMlpSmem*>(tc_smem) : nullptr);
}

// Features (and, with apply, the network's warm start) for the current
// contacts; runs before the sweeps (after colouring, before the gravity kick).
nbgs_status run_mlp_prologue(nbgs_scene* s, int apply, float* feat_out)
{
    if (s->composite) return fail(s, NBGS_EINVAL, "MLP: the network takes sphere contacts only");
    const int64_t C = s->n_contacts;
    if (C <= 0) return NBGS_OK;
    if (apply && !s->mlp_theta) return fail(s, NBGS_EINVAL, "MLP warm start: no network loaded (nbgs_mlp_load)");
    const int gb = grid_for(C, kTcRows, 4, s->num_sms);
    const size_t smem = apply ? sizeof(TcMlpSmem) : 0;
    if (s->fp32) k_mlp_warmstart<float><<<gb, kTcRows, smem, s->stream>>>(warm_args<float>(s, apply, feat_out));
    else k_mlp_warmstart<double><<<gb, kTcRows, smem, s->stream>>>(warm_args<double>(s, apply, feat_out));
    if (s->timing) s->phase_launches[2] += 1;
    return cuda_check(s, cudaGetLastError(), "MLP prologue");
}

}  // namespace nbgs

using namespace nbgs;

extern "C" {

nbgs_status nbgs_mlp_infer(const float* theta, const float* X, float* Y, int64_t n, void* stream)
{
    if (!theta || n < 0 || (n > 0 && (!X || !Y)) || ((uintptr_t)X & 15u)) return NBGS_EINVAL;
    if (n == 0) return NBGS_OK;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (n + kTcRows - 1) / kTcRows;
    k_mlp_infer_tc<<<grid_for(tiles * kTcRows, kTcRows, 4, sms), kTcRows, sizeof(TcMlpSmem), (cudaStream_t)stream>>>(
        theta, X, Y, n);
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
    static_assert(sizeof(TrainTcSmem) < 227 * 1024, "training tile too large");
    const int smem = (int)sizeof(TrainTcSmem);
    if (cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return NBGS_ECUDA;
    unsigned* status = nullptr;
    if (cudaGetSymbolAddress((void**)&status, g_mlp_status) != cudaSuccess) return NBGS_ECUDA;
    cudaMemsetAsync(grad, 0, kNParams * sizeof(float), st);
    cudaMemsetAsync(loss, 0, sizeof(double), st);
    const int64_t tiles = (n + kTrRows - 1) / kTrRows;
    const int blocks = (int)std::min<int64_t>(tiles, (int64_t)sms);   // one CTA per SM (all of its TMEM)
    k_mlp_grad_tc<<<blocks, kTrRows, smem, st>>>(theta, X, T, n, grad, loss, status);
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
