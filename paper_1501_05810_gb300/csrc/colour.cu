// colour.cu -- contact colouring and the colour-ordered sweep records.
//
// The subdomain numbers s_c(j) of Alg. 1 become colours: two contacts that
// share a body of finite mass never get the same colour, so all contacts of
// one colour can be relaxed at once with in-place velocity updates and no
// atomics, and the result equals the sequential NBGS in colour order.
//
//   k_colour_init   priority splitmix64(key ^ seed), body degrees
//   scan + k_adj_fill  body -> contact incidence lists (finite bodies only)
//   k_pred_masks    per contact: which incident contacts beat it
//   k_jp_round      Jones-Plassmann round: an uncoloured contact whose
//                   priority beats every uncoloured neighbour takes the
//                   smallest colour unused by its coloured neighbours; this
//                   equals first-fit greedy in decreasing priority
//   k_colour_keys   colour histogram
//   radix pass      stable counting sort by colour -> permutation
//   k_build_sweep   sweep records in colour order, initial impulses
#include <utility>

#include "nbgs_internal.cuh"

namespace nbgs {

// Key of a contact in its own scene's numbering (bodies from 0, walls
// after the scene's bodies: shared planes, then the six box faces), so that
// batched scenes are coloured exactly as each would be alone.
__device__ __forceinline__ uint64_t local_key(uint32_t a, uint32_t b, const SceneView& V)
{
    if (!V.batch) return ((uint64_t)a << 32) | b;
    const uint32_t s = V.scene_of[a];
    const uint32_t off = V.scene_off[s], ns = V.scene_off[s + 1] - off;
    uint64_t lb;
    if (b < (uint64_t)V.n) {
        lb = b - off;
    } else {
        const uint64_t w = b - (uint64_t)V.n;
        lb = ns + (w < (uint64_t)V.nplanes ? w : V.nplanes + (w - V.nplanes - 6ull * s));
    }
    return ((uint64_t)(a - off) << 32) | lb;
}

__global__ void k_colour_init(int64_t C, int64_t n, const uint32_t* __restrict__ cj1, const uint32_t* __restrict__ cj2,
                              const uint8_t* __restrict__ finite, uint64_t seed, SceneView V, uint32_t* __restrict__ deg,
                              uint64_t* __restrict__ prio, uint32_t* __restrict__ cstate, uint32_t* __restrict__ wl)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = cj1[c], b = cj2[c];
        prio[c] = splitmix64(local_key(a, b, V) ^ seed);
        cstate[c] = kUncoloured;
        wl[c] = (uint32_t)c;
        if (finite[a]) atomicAdd(&deg[a], 1u);
        if (b < n && finite[b]) atomicAdd(&deg[b], 1u);
    }
}

__global__ void k_adj_fill(int64_t C, int64_t n, const uint32_t* __restrict__ cj1, const uint32_t* __restrict__ cj2,
                           const uint8_t* __restrict__ finite, const uint32_t* __restrict__ adj_off,
                           uint32_t* __restrict__ fill, uint32_t* __restrict__ adj)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = cj1[c], b = cj2[c];
        if (finite[a]) adj[adj_off[a] + atomicAdd(&fill[a], 1u)] = (uint32_t)c;
        if (b < n && finite[b]) adj[adj_off[b] + atomicAdd(&fill[b], 1u)] = (uint32_t)c;
    }
}

// (prio, key) of d beats that of c: higher priority, ties to the lower key.
__device__ __forceinline__ bool beats(uint64_t pd, uint32_t d, uint64_t pc, uint32_t c, const uint32_t* cj1,
                                      const uint32_t* cj2)
{
    if (pd != pc) return pd > pc;
    const uint64_t kd = ((uint64_t)cj1[d] << 32) | cj2[d];
    const uint64_t kc = ((uint64_t)cj1[c] << 32) | cj2[c];
    return kd < kc;
}

// Predecessor masks: bit j of pmask[c] is set when entry j of the
// concatenated incidence lists of c's bodies (first body, then second) holds
// a contact that beats c.  blocker[c] = the weakest such contact (kUncoloured:
// none), cinfo[c] = (start, length) of the two lists.  pmask = ~0 marks a
// contact with more than 64 entries, which compares priorities whenever it
// is examined.
__global__ void k_pred_masks(int64_t C, int64_t n, const uint32_t* __restrict__ cj1, const uint32_t* __restrict__ cj2,
                             const uint8_t* __restrict__ finite, const uint32_t* __restrict__ adj_off,
                             const uint32_t* __restrict__ adj, const uint64_t* __restrict__ prio,
                             uint64_t* __restrict__ pmask, uint32_t* __restrict__ blocker, uint4* __restrict__ cinfo)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = cj1[c], b = cj2[c];
        const bool fa = finite[a], fb = b < n && finite[b];
        const uint32_t a0 = fa ? adj_off[a] : 0, na = fa ? adj_off[a + 1] - a0 : 0;
        const uint32_t b0 = fb ? adj_off[b] : 0, nb = fb ? adj_off[b + 1] - b0 : 0;
        uint64_t m = 0;
        uint32_t first = kUncoloured;
        if (na + nb > 64) {
            m = ~0ull;
        } else {
            const uint64_t pc = prio[c];
            uint64_t pfirst = 0;
            for (uint32_t j = 0; j < na + nb; ++j) {
                const uint32_t d = j < na ? adj[a0 + j] : adj[b0 + j - na];
                const uint64_t pd = prio[d];
                if (d != (uint32_t)c && beats(pd, d, pc, (uint32_t)c, cj1, cj2)) {
                    if (!m || beats(pfirst, first, pd, d, cj1, cj2)) {
                        first = d;
                        pfirst = pd;
                    }
                    m |= 1ull << j;
                }
            }
        }
        pmask[c] = m;
        blocker[c] = first;
        cinfo[c] = make_uint4(a0, na, b0, nb);
    }
}

// cstate[d] = (round << 8) | colour, or kUncoloured.  Within round r a
// contact coloured in round r still counts as uncoloured, so every decision
// of the round sees the state at its start.
__device__ __forceinline__ bool uncoloured_now(uint32_t sd, uint32_t round)
{
    return sd == kUncoloured || (sd >> 8) >= round;
}

// One warp examines contact c: its lanes cover the incidence entries.  If a
// predecessor is still uncoloured, c waits (its blocker becomes the
// uncoloured predecessor of lowest priority); otherwise c is a local maximum and takes the smallest
// colour none of its predecessors has (every coloured neighbour is a
// predecessor: the others wait for c).  Returns whether c waits.
__device__ bool jp_examine(uint32_t c, uint32_t round, int lane, const uint32_t* __restrict__ cj1,
                           const uint32_t* __restrict__ cj2, const uint32_t* __restrict__ adj,
                           const uint64_t* __restrict__ prio, const uint64_t* __restrict__ pmask,
                           uint32_t* __restrict__ blocker, const uint4* __restrict__ cinfo, uint32_t* cstate,
                           DevInfo* info)
{
    const uint4 ci = cinfo[c];
    const uint32_t len = ci.y + ci.w;
    const uint64_t pm = pmask[c];
    const bool slow = pm == ~0ull;
    const uint64_t pc = slow ? prio[c] : 0;
    uint32_t used[4] = {0u, 0u, 0u, 0u};
    for (uint32_t j0 = 0; j0 < len; j0 += 32) {
        const uint32_t j = j0 + lane;
        bool pred = false, unc = false;
        uint32_t d = 0, sd = kUncoloured;
        if (j < len) {
            d = j < ci.y ? adj[ci.x + j] : adj[ci.z + j - ci.y];
            pred = slow ? (d != c && beats(prio[d], d, pc, c, cj1, cj2)) : ((pm >> j) & 1ull) != 0;
            if (pred) {
                sd = cstate[d];
                unc = uncoloured_now(sd, round);
            }
        }
        const uint32_t wait = __ballot_sync(0xffffffffu, pred && unc);
        if (wait) {
            if (!slow) {
                // wait for the weakest uncoloured predecessor: it tends to be
                // coloured last, so c is examined again fewer times
                const uint64_t pd = (pred && unc) ? prio[d] : ~0ull;
                uint64_t pmin = pd;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const uint64_t y = __shfl_xor_sync(0xffffffffu, pmin, o);
                    pmin = y < pmin ? y : pmin;
                }
                const uint32_t at = __ballot_sync(0xffffffffu, (pred && unc) && pd == pmin);
                if (lane == __ffs(at) - 1) blocker[c] = d;
            }
            return true;
        }
        if (pred) {
            const uint32_t col = sd & 0xFFu;
#pragma unroll
            for (int w = 0; w < 4; ++w)
                if ((col >> 5) == (uint32_t)w) used[w] |= 1u << (col & 31u);
        }
    }
    uint32_t col = kMaxColours;
#pragma unroll
    for (int w = 3; w >= 0; --w) {
        const uint32_t u = __reduce_or_sync(0xffffffffu, used[w]);
        if (~u) col = 32u * w + (__ffs(~u) - 1);
    }
    if (lane == 0) {
        if (col >= kMaxColours) {
            atomicOr(&info->err, kErrColours);
            col = kMaxColours - 1;
        }
        cstate[c] = (round << 8) | col;
    }
    return false;
}

// Appends val to list for every lane with pred set (one shared-memory
// counter update per warp).
__device__ __forceinline__ void warp_push(bool pred, uint32_t val, uint32_t* list, uint32_t* count, int lane)
{
    const uint32_t mask = __ballot_sync(0xffffffffu, pred);
    uint32_t b = 0;
    if (lane == 0 && mask) b = atomicAdd(count, (uint32_t)__popc(mask));
    b = __shfl_sync(0xffffffffu, b, 0);
    if (pred) list[b + __popc(mask & ((1u << lane) - 1u))] = val;
}

// One Jones-Plassmann round over the worklist, a tile of kJpItems per thread
// at a time.  Phase 1, a thread per contact: a contact whose remembered
// blocker is still uncoloured waits (two loads).  Phase 2, a warp per
// remaining contact (jp_examine).  The waiting contacts of the tile go to
// wl_out with one global counter update.
constexpr int kJpThreads = 256;
constexpr int kJpItems = 4;

__global__ void __launch_bounds__(kJpThreads) k_jp_round(uint32_t round, const uint32_t* __restrict__ wl_in,
                                  const uint32_t* __restrict__ cnt_in, uint32_t* __restrict__ wl_out,
                                  uint32_t* __restrict__ cnt_out, const uint32_t* __restrict__ cj1,
                                  const uint32_t* __restrict__ cj2, const uint32_t* __restrict__ adj,
                                  const uint64_t* __restrict__ prio, const uint64_t* __restrict__ pmask,
                                  uint32_t* __restrict__ blocker, const uint4* __restrict__ cinfo,
                                  uint32_t* cstate, DevInfo* info)
{
    __shared__ uint32_t s_exam[kJpThreads * kJpItems];
    __shared__ uint32_t s_keep[kJpThreads * kJpItems];
    __shared__ uint32_t s_nexam, s_nkeep, s_base;
    const uint32_t m = *cnt_in;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr uint32_t nwarps = kJpThreads / 32, tile = kJpThreads * kJpItems;
    for (uint32_t base = blockIdx.x * tile; base < m; base += gridDim.x * tile) {
        if (threadIdx.x == 0) {
            s_nexam = 0;
            s_nkeep = 0;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kJpItems; ++i) {
            const uint32_t k = base + i * kJpThreads + threadIdx.x;
            uint32_t c = 0;
            bool waits = false;
            if (k < m) {
                c = wl_in[k];
                const uint32_t bl = blocker[c];
                waits = bl != kUncoloured && uncoloured_now(cstate[bl], round);
            }
            warp_push(waits, c, s_keep, &s_nkeep, lane);
            warp_push(k < m && !waits, c, s_exam, &s_nexam, lane);
        }
        __syncthreads();
        const uint32_t ne = s_nexam;
        for (uint32_t e = warp; e < ne; e += nwarps) {
            const uint32_t c = s_exam[e];
            if (jp_examine(c, round, lane, cj1, cj2, adj, prio, pmask, blocker, cinfo, cstate, info) && lane == 0)
                s_keep[atomicAdd(&s_nkeep, 1u)] = c;
        }
        __syncthreads();
        const uint32_t nk = s_nkeep;
        if (threadIdx.x == 0) s_base = nk ? atomicAdd(cnt_out, nk) : 0u;
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < nk; t += kJpThreads) wl_out[s_base + t] = s_keep[t];
        __syncthreads();   // the shared lists are refilled by the next tile
    }
}

__global__ void k_colour_keys(int64_t C, const uint32_t* __restrict__ cstate, uint32_t* __restrict__ ckey,
                              uint32_t* __restrict__ cval, uint32_t* __restrict__ col_count, DevInfo* info)
{
    __shared__ uint32_t h[kMaxColours];
    for (int t = threadIdx.x; t < kMaxColours; t += blockDim.x) h[t] = 0;
    __syncthreads();
    uint32_t cmax = 0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        uint32_t col = cstate[c] & 0xFFu;
        if (col >= (uint32_t)kMaxColours) {   // uncoloured or out of range: report, keep indices in bounds
            atomicOr(&info->err, kErrColours);
            col = kMaxColours - 1;
        }
        ckey[c] = col;
        cval[c] = (uint32_t)c;
        atomicAdd(&h[col], 1u);
        cmax = max(cmax, col + 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kMaxColours; t += blockDim.x)
        if (h[t]) atomicAdd(&col_count[t], h[t]);
    for (int o = 16; o > 0; o >>= 1) cmax = max(cmax, __shfl_down_sync(0xffffffffu, cmax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&info->n_colours, cmax);
}

__global__ void k_colour_offsets(const uint32_t* __restrict__ col_count, uint32_t* __restrict__ col_off)
{
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int c = 0; c < kMaxColours; ++c) {
            col_off[c] = acc;
            acc += col_count[c];
        }
        col_off[kMaxColours] = acc;
    }
}

// Sweep record s <- canonical contact perm[s]; initial impulse from the
// previous step (world frame, re-projected onto the new frame and the cone)
// or zero.
template <class R>
__global__ void k_build_sweep(int64_t C, int64_t n, const uint32_t* __restrict__ perm, const uint32_t* __restrict__ cj1,
                              const uint32_t* __restrict__ cj2, const double4_32a* __restrict__ cgeo,
                              const double2* __restrict__ clev, double dt, double beta, double mu_all, SceneView V,
                              int warm,
                              const uint32_t* __restrict__ prev_row_off, const uint32_t* __restrict__ prev_j2,
                              const double4_32a* __restrict__ prev_P, SweepRec<R>* __restrict__ rec,
                              R4<R>* __restrict__ p)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < C; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = perm[s];
        const uint32_t a = cj1[c], b = cj2[c];
        const double4_32a g = cgeo[c];
        const double2 l = clev[c];
        // eq. (nonpenetration): gap term xi/dt, scaled by beta when xi < 0
        const double xs = g.w >= 0.0 ? g.w : beta * g.w;
        const double bias = xs / dt;
        SweepRec<R> r;
        if constexpr (sizeof(R) == 4) {
            r.a = make_float4(__uint_as_float(a), __uint_as_float(b), (float)l.x, (float)l.y);
            r.b = make_float4((float)g.x, (float)g.y, (float)g.z, (float)bias);
        } else {
            r.ids_bias = make_double2(__longlong_as_double((long long)(((uint64_t)b << 32) | a)), bias);
            r.lev = make_double2(l.x, l.y);
            r.nxy = make_double2(g.x, g.y);
            r.nz_ = make_double2(g.z, 0.0);
        }
        rec[s] = r;
        double pn = 0.0, pt = 0.0, po = 0.0, found = 0.0;
        if (warm) {
            const uint32_t e = prev_row_off[a + 1];
            for (uint32_t t = prev_row_off[a]; t < e; ++t) {
                if (prev_j2[t] != b) continue;
                const double4_32a P = prev_P[t];
                const double mu = V.batch ? V.mu[V.scene_of[a]] : mu_all;
                found = 1.0;
                double tx, ty, tz, ox, oy, oz;
                tangent_basis<double>(g.x, g.y, g.z, tx, ty, tz, ox, oy, oz);
                pn = g.x * P.x + g.y * P.y + g.z * P.z;
                if (!(pn > 0.0)) pn = 0.0;
                pt = tx * P.x + ty * P.y + tz * P.z;
                po = ox * P.x + oy * P.y + oz * P.z;
                const double lim = mu * pn, len = sqrt(pt * pt + po * po);
                if (len > lim) {
                    if (len > 0.0) {
                        pt *= lim / len;
                        po *= lim / len;
                    } else {
                        pt = po = 0.0;
                    }
                }
                break;
            }
        }
        R4<R> q;
        q.x = (R)pn;
        q.y = (R)pt;
        q.z = (R)po;
        q.w = (R)found;   // 1: the contact existed in the previous step (read by the network warm start)
        p[s] = q;
    }
}

nbgs_status run_colour(nbgs_scene* s)
{
    if (!s->detected) return fail(s, NBGS_EINVAL, "colour_contacts: call detect_contacts first");
    cudaStream_t st = s->stream;
    const int64_t C = s->n_contacts, n = s->n;
    if (s->timing) cudaEventRecord(s->ev[2], st);
    cudaMemsetAsync(s->col_count, 0, (kMaxColours + 1) * sizeof(uint32_t), st);
    cudaMemsetAsync(&s->info->n_colours, 0, sizeof(uint32_t), st);
    if (C > 0) {
        const int T = 256;
        const int gb = grid_for(C, T, 8, s->num_sms);
        cudaMemsetAsync(s->deg, 0, (n + 1) * sizeof(uint32_t), st);
        k_colour_init<<<gb, T, 0, st>>>(C, n, s->cj1, s->cj2, s->finite, s->prm.colour_seed, scene_view(s), s->deg,
                                        s->cprio, s->cstate, s->wl[0]);
        nbgs_status rc = exclusive_scan_u32(s, s->deg, s->adj_off, n, nullptr);
        if (rc != NBGS_OK) return rc;
        cudaMemsetAsync(s->deg, 0, (n + 1) * sizeof(uint32_t), st);
        k_adj_fill<<<gb, T, 0, st>>>(C, n, s->cj1, s->cj2, s->finite, s->adj_off, s->deg, s->adj);
        k_pred_masks<<<gb, T, 0, st>>>(C, n, s->cj1, s->cj2, s->finite, s->adj_off, s->adj, s->cprio, s->pmask,
                                       s->blocker, s->cinfo);
        if (s->timing) s->phase_launches[1] += 5;
        // Jones-Plassmann rounds; the host checks the worklist every few rounds
        const uint32_t c32 = (uint32_t)C;
        const int gbr = grid_for((C + kJpItems - 1) / kJpItems, kJpThreads, 8, s->num_sms);
        cudaMemcpyAsync(&s->info->wl_count[0], &c32, sizeof(uint32_t), cudaMemcpyHostToDevice, st);
        uint32_t round = 0;
        int cur = 0;
        for (int batch = 0; batch < 64; ++batch) {
            for (int r = 0; r < 6; ++r) {
                ++round;
                cudaMemsetAsync(&s->info->wl_count[1 - cur], 0, sizeof(uint32_t), st);
                k_jp_round<<<gbr, kJpThreads, 0, st>>>(round, s->wl[cur], &s->info->wl_count[cur], s->wl[1 - cur],
                                                       &s->info->wl_count[1 - cur], s->cj1, s->cj2, s->adj, s->cprio,
                                                       s->pmask, s->blocker, s->cinfo, s->cstate, s->info);
                cur = 1 - cur;
            }
            if (s->timing) s->phase_launches[1] += 6;
            uint32_t left = 0;
            rc = cuda_check(s, cudaMemcpyAsync(&left, &s->info->wl_count[cur], sizeof(uint32_t),
                                               cudaMemcpyDeviceToHost, st), "colour: worklist");
            if (rc != NBGS_OK) return rc;
            rc = cuda_check(s, cudaStreamSynchronize(st), "colour");
            if (rc != NBGS_OK) return rc;
            if (left == 0) break;
            if (batch == 63) return fail(s, NBGS_ETIMEOUT, "colour: Jones-Plassmann did not finish in 384 rounds");
        }
        k_colour_keys<<<gb, T, 0, st>>>(C, s->cstate, s->colour_key, s->perm_in, s->col_count, s->info);
        k_colour_offsets<<<1, 32, 0, st>>>(s->col_count, s->col_off);
        // stable counting sort by colour (one 8-bit radix pass): contacts of a
        // colour stay in canonical order
        uint32_t *k0 = s->colour_key, *k1 = s->colour_key2, *v0 = s->perm_in, *v1 = s->perm;
        rc = radix_sort_pairs(s, k0, v0, k1, v1, C, 8);
        if (rc != NBGS_OK) return rc;
        // radix_sort_pairs swapped the pointers: v0 / k0 now hold the sorted values / keys
        if (v0 != s->perm) std::swap(s->perm, s->perm_in);
        if (v0 != s->perm) return fail(s, NBGS_EINVAL, "colour: permutation buffer mix-up");
        s->colour_sorted = k0;
        const int warm = (s->prm.warm_start != NBGS_WARM_NONE && s->have_prev) ? 1 : 0;
        if (s->fp32)
            k_build_sweep<float><<<gb, T, 0, st>>>(C, n, s->perm, s->cj1, s->cj2, s->cgeo, s->clev, s->prm.dt,
                                                   s->prm.beta, s->prm.mu, scene_view(s), warm, s->prev_row_off,
                                                   s->prev_j2,
                                                   s->prev_P, (SweepRec<float>*)s->srec, (float4*)s->sp);
        else
            k_build_sweep<double><<<gb, T, 0, st>>>(C, n, s->perm, s->cj1, s->cj2, s->cgeo, s->clev, s->prm.dt,
                                                    s->prm.beta, s->prm.mu, scene_view(s), warm, s->prev_row_off,
                                                    s->prev_j2,
                                                    s->prev_P, (SweepRec<double>*)s->srec, (double4_32a*)s->sp);
        if (s->timing) s->phase_launches[1] += 3;
        s->n_colours = -1;  // known on the device; read lazily
    } else {
        s->n_colours = 0;
    }
    if (s->timing) cudaEventRecord(s->ev[3], st);
    s->coloured = true;
    return cuda_check(s, cudaGetLastError(), "colour");
}

}  // namespace nbgs
