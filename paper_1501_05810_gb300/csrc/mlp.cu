// mlp.cu -- learned warm start: a 12 -> 64 -> 64 -> 64 -> 3 MLP (SiLU) that
// predicts a contact's converged impulse from local features, evaluated on
// the 5th-generation tensor cores (tcgen05: BF16 operands in shared memory,
// FP32 accumulators in TMEM) before the sweeps, and its training kernels
// (FP32 forward/backward, Adam).
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
