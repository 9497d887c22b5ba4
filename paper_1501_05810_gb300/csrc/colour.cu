// colour.cu -- contact colouring and the colour-ordered sweep records.
//
// The subdomain numbers s_c(j) of Alg. 1 become colours: two contacts that
// share a body of finite mass never get the same colour, so all contacts of
// one colour can be relaxed at once with in-place velocity updates and no
// atomics, and the result equals the sequential NBGS in colour order.
//
//   k_colour_init   priority splitmix64(key ^ seed), body degrees
//   scan + k_adj_fill  body -> contact incidence lists (finite bodies only)
//   k_pred_count, scan, k_pred_lists
//                   per contact: the incident contacts that beat it (its
//                   predecessors); it waits on the weakest
//   k_jp_round      a contact whose predecessors are all coloured takes the
//                   smallest colour none of them has: first-fit greedy in
//                   decreasing priority, as Jones-Plassmann rounds give it,
//                   driven by waiting lists (k_jp_persistent: every round
//                   in one cooperative launch, for device-sized steps)
//   k_colour_keys   colour histogram
//   radix pass      stable counting sort by colour -> permutation
//   k_build_sweep   sweep records in colour order, initial impulses
#include <algorithm>
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

// Priorities from the contacts' keys; body degrees from the incidence ends
// ib1, ib2 (the contact's bodies: the contact ends themselves for spheres,
// the members' bodies for composites; >= n marks a wall).
__global__ void k_colour_init(DCount Cc, int64_t n, const uint32_t* __restrict__ cj1, const uint32_t* __restrict__ cj2,
                              const uint32_t* __restrict__ ib1, const uint32_t* __restrict__ ib2,
                              const uint8_t* __restrict__ finite, uint64_t seed, SceneView V, uint32_t* __restrict__ deg,
                              uint64_t* __restrict__ prio, uint32_t* __restrict__ cstate)
{
    const int64_t C = Cc.get();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        prio[c] = splitmix64(local_key(cj1[c], cj2[c], V) ^ seed);
        cstate[c] = kUncoloured;
        const uint32_t a = ib1[c], b = ib2[c];
        if (finite[a]) atomicAdd(&deg[a], 1u);
        if (b < n && finite[b]) atomicAdd(&deg[b], 1u);
    }
}

__global__ void k_adj_fill(DCount Cc, int64_t n, const uint32_t* __restrict__ cj1, const uint32_t* __restrict__ cj2,
                           const uint8_t* __restrict__ finite, const uint32_t* __restrict__ adj_off,
                           uint32_t* __restrict__ fill, uint32_t* __restrict__ adj)
{
    const int64_t C = Cc.get();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = cj1[c], b = cj2[c];
        if (finite[a]) adj[adj_off[a] + atomicAdd(&fill[a], 1u)] = (uint32_t)c;
        if (b < n && finite[b]) adj[adj_off[b] + atomicAdd(&fill[b], 1u)] = (uint32_t)c;
    }
}

// (prio, key) of d beats that of c: higher priority, ties to the lower key.
// Contacts are stored in canonical order, so the lower index is the lower key.
__device__ __forceinline__ bool beats(uint64_t pd, uint32_t d, uint64_t pc, uint32_t c)
{
    if (pd != pc) return pd > pc;
    return d < c;
}

// Colouring by waiting lists.  First-fit greedy colouring in decreasing
// priority gives each contact the smallest colour none of its predecessors
// (neighbours that beat it) has; the colour depends only on the
// predecessors' colours, not on when it is computed.  So a contact is
// examined only when it may be ready: at the start if it has no
// predecessor, later when the predecessor it waits for (its blocker) has
// been coloured.  A contact that finds a predecessor still uncoloured puts
// itself on that predecessor's waiting list (whead / wnext, a lock-free
// stack); the round after a contact is coloured walks its list.  A waiter
// always registers in a round no later than the one that colours its
// blocker (it saw the blocker uncoloured), so the walk, one launch later,
// sees it.  Every round needs only the contacts coloured in the previous
// round and their waiters, not a pass over all uncoloured contacts.
//
// Worklists: a buffer of C entries holds the contacts coloured in a round
// (L, from the front) and the contacts to examine directly in the next
// round (X, from the back: contacts with more than 64 incidence entries,
// which keep no blocker, and examinations that did not fit a block's shared
// buffer).  The counters (|L|, |X|) rotate through three pairs: a round
// reads one, writes the next and clears the third.

// Appends val to list (from the front, or from the back of a buffer of cap
// entries) for every lane with pred set; one counter update per warp.
__device__ __forceinline__ void warp_push(bool pred, uint32_t val, uint32_t* list, uint32_t* count, int lane,
                                          bool from_back = false, uint32_t cap = 0)
{
    const uint32_t mask = __ballot_sync(0xffffffffu, pred);
    uint32_t b = 0;
    if (lane == 0 && mask) b = atomicAdd(count, (uint32_t)__popc(mask));
    b = __shfl_sync(0xffffffffu, b, 0);
    if (pred) {
        const uint32_t i = b + __popc(mask & ((1u << lane) - 1u));
        list[from_back ? cap - 1u - i : i] = val;
    }
}

// Incidence entry j of contact c: the lists of its first body, then of its
// second (finite bodies only).
__device__ __forceinline__ uint32_t incident(const uint32_t* __restrict__ adj, uint32_t a0, uint32_t na, uint32_t b0,
                                             uint32_t j)
{
    return j < na ? adj[a0 + j] : adj[b0 + j - na];
}

__device__ __forceinline__ void incidence(uint32_t c, int64_t n, const uint32_t* __restrict__ cj1,
                                          const uint32_t* __restrict__ cj2, const uint8_t* __restrict__ finite,
                                          const uint32_t* __restrict__ adj_off, uint32_t& a0, uint32_t& na,
                                          uint32_t& b0, uint32_t& nb)
{
    const uint32_t a = cj1[c], b = cj2[c];
    const bool fa = finite[a], fb = b < n && finite[b];
    a0 = fa ? adj_off[a] : 0;
    na = fa ? adj_off[a + 1] - a0 : 0;
    b0 = fb ? adj_off[b] : 0;
    nb = fb ? adj_off[b + 1] - b0 : 0;
}

// Predecessors of contact c: the incident contacts that beat it.  Pass 1
// counts them (npred) and keeps them as a bit mask over the incidence
// entries (pmask; ~0 for more than 64 entries, where pass 2 compares
// priorities again).
__global__ void k_pred_count(DCount Cc, int64_t n, const uint32_t* __restrict__ cj1, const uint32_t* __restrict__ cj2,
                             const uint8_t* __restrict__ finite, const uint32_t* __restrict__ adj_off,
                             const uint32_t* __restrict__ adj, const uint64_t* __restrict__ prio,
                             uint64_t* __restrict__ pmask, uint32_t* __restrict__ npred)
{
    const int64_t C = Cc.get();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        uint32_t a0, na, b0, nb;
        incidence((uint32_t)c, n, cj1, cj2, finite, adj_off, a0, na, b0, nb);
        const uint64_t pc = prio[c];
        uint64_t m = 0;
        uint32_t k = 0;
        for (uint32_t j = 0; j < na + nb; ++j) {
            const uint32_t d = incident(adj, a0, na, b0, j);
            if (d != (uint32_t)c && beats(prio[d], d, pc, (uint32_t)c)) {
                ++k;
                if (j < 64) m |= 1ull << j;
            }
        }
        pmask[c] = na + nb > 64 ? ~0ull : m;
        npred[c] = k;
    }
}

// Pass 2: the predecessor list of c at preds[poff[c] ..], each entry the
// predecessor and the high half of its priority.  A contact with
// predecessors waits on the weakest (it tends to be coloured last, so the
// contact is examined again fewer times); the others form the first round's
// direct list.
__device__ __forceinline__ uint32_t prio_hi(uint64_t p) { return (uint32_t)(p >> 32); }

__global__ void k_pred_lists(DCount Cc, int64_t n, const uint32_t* __restrict__ cj1, const uint32_t* __restrict__ cj2,
                             const uint8_t* __restrict__ finite, const uint32_t* __restrict__ adj_off,
                             const uint32_t* __restrict__ adj, const uint64_t* __restrict__ prio,
                             const uint64_t* __restrict__ pmask, const uint32_t* __restrict__ poff,
                             uint2* __restrict__ preds, int64_t pcap, uint32_t* whead, uint32_t* __restrict__ wnext,
                             uint32_t* __restrict__ wl, uint32_t* count)
{
    const int64_t C = Cc.get();
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform trip count: every lane takes part in warp_push
    for (int64_t c0 = blockIdx.x * (int64_t)blockDim.x; c0 < C; c0 += stride) {
        const int64_t c = c0 + threadIdx.x;
        bool direct = false;
        if (c < C) {
            uint32_t a0, na, b0, nb;
            incidence((uint32_t)c, n, cj1, cj2, finite, adj_off, a0, na, b0, nb);
            const uint32_t p0 = poff[c], np = poff[c + 1] - p0;
            const uint64_t m = pmask[c];
            const uint64_t pc = prio[c];
            uint32_t k = 0, weakest = kUncoloured;
            uint64_t pweak = ~0ull;
            for (uint32_t j = 0; j < na + nb && k < np; ++j) {
                if (m != ~0ull && !((m >> j) & 1ull)) continue;
                const uint32_t d = incident(adj, a0, na, b0, j);
                const uint64_t pd = prio[d];
                if (m == ~0ull && (d == (uint32_t)c || !beats(pd, d, pc, (uint32_t)c))) continue;
                if (p0 + k < pcap) preds[p0 + k] = make_uint2(d, prio_hi(pd));   // beyond: the error bit is set
                if (pd < pweak) {
                    pweak = pd;
                    weakest = d;
                }
                ++k;
            }
            if (np == 0) direct = true;
            else wnext[c] = atomicExch(&whead[weakest], (uint32_t)c);
        }
        warp_push(direct, (uint32_t)c, wl, count, lane, true, (uint32_t)C);
    }
}

// Examination of contact c by a group of 4 lanes (lanes 4g..4g+3 of a
// warp; every lane of the warp calls this, valid = false for a group with no
// contact).  The lanes cover the predecessor list, 16 entries per pass, all
// loads of a pass in flight together.  If a predecessor is still
// uncoloured, c waits on the weakest such one.  Otherwise c takes the
// smallest colour none of its predecessors has.  Returns whether c was
// coloured.
__device__ bool jp_examine(bool valid, uint32_t c, uint32_t round, int lane, const uint32_t* __restrict__ poff,
                           const uint2* __restrict__ preds, uint32_t* cstate, uint32_t* whead,
                           uint32_t* __restrict__ wnext, DevInfo* info)
{
    const int gl = lane & 3;
    uint32_t p0 = 0, np = 0;
    if (valid) {
        p0 = poff[c];
        np = poff[c + 1] - p0;
    }
    const uint32_t maxnp = __reduce_max_sync(0xffffffffu, np);
    uint32_t used[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};   // colours taken by predecessors (kMaxColours bits)
    uint32_t wph = ~0u, wd = kUncoloured;   // weakest uncoloured predecessor seen by this lane
    for (uint32_t w0 = 0; w0 < maxnp; w0 += 16) {
        uint2 e[4];
        uint32_t sd[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t j = w0 + 4 * k + gl;
            e[k] = j < np ? preds[p0 + j] : make_uint2(kUncoloured, 0u);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) sd[k] = e[k].x != kUncoloured ? cstate[e[k].x] : 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (e[k].x == kUncoloured) continue;
            if (sd[k] == kUncoloured) {
                if (wd == kUncoloured || e[k].y < wph) {
                    wph = e[k].y;
                    wd = e[k].x;
                }
            } else {
                const uint32_t col = sd[k] & 0xFFu;
#pragma unroll
                for (int w = 0; w < 8; ++w)
                    if ((col >> 5) == (uint32_t)w) used[w] |= 1u << (col & 31u);
            }
        }
    }
    // group reductions (xor 1, 2 stays inside the group)
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        const uint32_t wp2 = __shfl_xor_sync(0xffffffffu, wph, o);
        const uint32_t wd2 = __shfl_xor_sync(0xffffffffu, wd, o);
        if (wd2 != kUncoloured && (wd == kUncoloured || wp2 < wph)) {
            wph = wp2;
            wd = wd2;
        }
#pragma unroll
        for (int w = 0; w < 8; ++w) used[w] |= __shfl_xor_sync(0xffffffffu, used[w], o);
    }
    if (!valid) return false;
    if (wd != kUncoloured) {
        if (gl == 0) wnext[c] = atomicExch(&whead[wd], c);
        return false;
    }
    if (gl == 0) {
        uint32_t col = kMaxColours;
#pragma unroll
        for (int w = 7; w >= 0; --w)
            if (~used[w]) col = 32u * w + (__ffs(~used[w]) - 1);
        if (col >= kMaxColours) {
            atomicOr(&info->err, kErrColours);
            col = kMaxColours - 1;
        }
        cstate[c] = (round << 8) | col;   // the round is informational
    }
    return true;
}

// One round, a tile of kJpThreads input entries at a time.  Phase 1, a
// thread per entry: an entry of L has its waiting list walked, an entry of
// X is taken as it is; both fill the block's examination buffer (overflow
// goes to the next round's X).  Phase 2, 4 lanes per buffered contact
// (jp_examine); the contacts coloured go to the next L.
constexpr int kJpThreads = 256;
constexpr int kJpCap = 2048;

// Round `round` over the input lists (tiles of kJpThreads entries, grid-
// stride).  What other blocks wrote in earlier rounds (lists, counters,
// states, waiting lists) is visible after the grid barrier between rounds
// (its acquire fence); the counters are read through L2.
__device__ __forceinline__ void jp_round(uint32_t round, uint32_t C, const uint32_t* __restrict__ wl_in,
                                         const uint32_t* cnt_in, uint32_t* __restrict__ wl_out, uint32_t* cnt_out,
                                         uint32_t* cnt_clear, const uint32_t* __restrict__ poff,
                                         const uint2* __restrict__ preds, uint32_t* cstate, uint32_t* whead,
                                         uint32_t* __restrict__ wnext, DevInfo* info)
{
    __shared__ uint32_t s_exam[kJpCap];
    __shared__ uint32_t s_done[kJpCap];
    __shared__ uint32_t s_nexam, s_ndone, s_base;
    const uint32_t nl = __ldcg(cnt_in), nx = __ldcg(cnt_in + 1), m = nl + nx;
    if (blockIdx.x == 0 && threadIdx.x < 2) cnt_clear[threadIdx.x] = 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr uint32_t nwarps = kJpThreads / 32;
    for (uint32_t base = blockIdx.x * kJpThreads; base < m; base += gridDim.x * kJpThreads) {
        if (threadIdx.x == 0) {
            s_nexam = 0;
            s_ndone = 0;
        }
        __syncthreads();
        const uint32_t k = base + threadIdx.x;
        if (k < nl) {
            const uint32_t c = wl_in[k];
            uint32_t h = whead[c];
            whead[c] = kUncoloured;
            while (h != kUncoloured) {
                const uint32_t i = atomicAdd(&s_nexam, 1u);
                if (i < kJpCap) {
                    s_exam[i] = h;
                } else {
                    const uint32_t g = atomicAdd(&cnt_out[1], 1u);
                    wl_out[C - 1u - g] = h;
                }
                h = wnext[h];
            }
        } else if (k < m) {
            const uint32_t c = wl_in[C - 1u - (k - nl)];
            const uint32_t i = atomicAdd(&s_nexam, 1u);
            if (i < kJpCap) {
                s_exam[i] = c;
            } else {
                const uint32_t g = atomicAdd(&cnt_out[1], 1u);
                wl_out[C - 1u - g] = c;
            }
        }
        __syncthreads();
        const uint32_t ne = s_nexam < kJpCap ? s_nexam : kJpCap;
        for (uint32_t e0 = 8 * warp; e0 < ne; e0 += 8 * nwarps) {
            const uint32_t e = e0 + (lane >> 2);
            const bool valid = e < ne;
            const uint32_t c = valid ? s_exam[e] : 0u;
            if (jp_examine(valid, c, round, lane, poff, preds, cstate, whead, wnext, info) && (lane & 3) == 0)
                s_done[atomicAdd(&s_ndone, 1u)] = c;
        }
        __syncthreads();
        const uint32_t nd = s_ndone;
        if (threadIdx.x == 0) s_base = nd ? atomicAdd(&cnt_out[0], nd) : 0u;
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < nd; t += kJpThreads) wl_out[s_base + t] = s_done[t];
        __syncthreads();   // the shared lists are refilled by the next tile
    }
}

// One round per launch (the host checks the lists every few rounds).
__global__ void __launch_bounds__(kJpThreads) k_jp_round(uint32_t round, uint32_t C, const uint32_t* __restrict__ wl_in,
                                  const uint32_t* __restrict__ cnt_in, uint32_t* __restrict__ wl_out,
                                  uint32_t* __restrict__ cnt_out, uint32_t* __restrict__ cnt_clear,
                                  const uint32_t* __restrict__ poff, const uint2* __restrict__ preds,
                                  uint32_t* cstate, uint32_t* whead, uint32_t* __restrict__ wnext, DevInfo* info)
{
    __shared__ uint32_t s_exam[kJpCap];
    __shared__ uint32_t s_done[kJpCap];
    __shared__ uint32_t s_nexam, s_ndone, s_base;
    const uint32_t nl = cnt_in[0], nx = cnt_in[1], m = nl + nx;
    if (blockIdx.x == 0 && threadIdx.x < 2) cnt_clear[threadIdx.x] = 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr uint32_t nwarps = kJpThreads / 32;
    for (uint32_t base = blockIdx.x * kJpThreads; base < m; base += gridDim.x * kJpThreads) {
        if (threadIdx.x == 0) {
            s_nexam = 0;
            s_ndone = 0;
        }
        __syncthreads();
        const uint32_t k = base + threadIdx.x;
        if (k < nl) {
            const uint32_t c = wl_in[k];
            uint32_t h = whead[c];
            whead[c] = kUncoloured;
            while (h != kUncoloured) {
                const uint32_t i = atomicAdd(&s_nexam, 1u);
                if (i < kJpCap) {
                    s_exam[i] = h;
                } else {
                    const uint32_t g = atomicAdd(&cnt_out[1], 1u);
                    wl_out[C - 1u - g] = h;
                }
                h = wnext[h];
            }
        } else if (k < m) {
            const uint32_t c = wl_in[C - 1u - (k - nl)];
            const uint32_t i = atomicAdd(&s_nexam, 1u);
            if (i < kJpCap) {
                s_exam[i] = c;
            } else {
                const uint32_t g = atomicAdd(&cnt_out[1], 1u);
                wl_out[C - 1u - g] = c;
            }
        }
        __syncthreads();
        const uint32_t ne = s_nexam < kJpCap ? s_nexam : kJpCap;
        for (uint32_t e0 = 8 * warp; e0 < ne; e0 += 8 * nwarps) {
            const uint32_t e = e0 + (lane >> 2);
            const bool valid = e < ne;
            const uint32_t c = valid ? s_exam[e] : 0u;
            if (jp_examine(valid, c, round, lane, poff, preds, cstate, whead, wnext, info) && (lane & 3) == 0)
                s_done[atomicAdd(&s_ndone, 1u)] = c;
        }
        __syncthreads();
        const uint32_t nd = s_ndone;
        if (threadIdx.x == 0) s_base = nd ? atomicAdd(&cnt_out[0], nd) : 0u;
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < nd; t += kJpThreads) wl_out[s_base + t] = s_done[t];
        __syncthreads();   // the shared lists are refilled by the next tile
    }
}

// All rounds in one cooperative launch (no host in the loop, so a step can
// be captured in a CUDA graph): a grid barrier ends each round (it
// plays the part of a launch boundary: every waiter registered and every
// colour written before the next round walks the lists), and the round's
// output counters, read by every block after the barrier, tell whether
// anything is left.  A contact count of zero leaves at once; more than
// kJpMaxRounds rounds set the colour error bit.
constexpr int kJpMaxRounds = 1024;

// Grid barrier of the colouring rounds: the arrival count and generation
// words of the grid barrier, polled without sleeping (rounds are short);
// bounded like every wait (~1 s of SM clocks), then the timeout bit.
__device__ __forceinline__ bool jp_barrier(DevInfo* info)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t* vgen = &info->barrier_gen;
        const uint32_t gen = *vgen;
        __threadfence();
        int good = 1;
        if (atomicAdd(&info->barrier_count, 1u) == gridDim.x - 1) {
            info->barrier_count = 0;
            __threadfence();
            atomicAdd(&info->barrier_gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == gen) {
                if (clock64() - t0 > (1LL << 31)) {
                    atomicOr(&info->err, kErrTimeout);
                    good = 0;
                    break;
                }
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

__global__ void __launch_bounds__(kJpThreads) k_jp_persistent(DCount Cc, uint32_t* wl0,
                                                              uint32_t* wl1, uint32_t* cnt,
                                                              const uint32_t* __restrict__ poff,
                                                              const uint2* __restrict__ preds, uint32_t* cstate,
                                                              uint32_t* whead, uint32_t* __restrict__ wnext,
                                                              DevInfo* info)
{
    const uint32_t C = (uint32_t)Cc.get();
    if (C == 0 || (info->err & kErrPreds)) return;   // overflowed lists: the colours stay unset (error bit)
    for (uint32_t round = 1; round <= (uint32_t)kJpMaxRounds; ++round) {
        const int ci = (round - 1) % 3, co = round % 3, cc = (round + 1) % 3;
        const bool odd = (round & 1u) != 0u;   // round 1 reads wl0 and writes wl1, round 2 the reverse, ...
        jp_round(round, C, odd ? wl0 : wl1, cnt + 2 * ci, odd ? wl1 : wl0, cnt + 2 * co, cnt + 2 * cc, poff, preds,
                 cstate, whead, wnext, info);
        if (!jp_barrier(info)) return;
        if (__ldcg(cnt + 2 * co) + __ldcg(cnt + 2 * co + 1) == 0u) return;   // nothing coloured or left to examine
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&info->err, kErrColours);
}

__global__ void k_colour_keys(DCount Cc, const uint32_t* __restrict__ cstate, uint32_t* __restrict__ ckey,
                              uint32_t* __restrict__ cval, uint32_t* __restrict__ col_count, DevInfo* info)
{
    const int64_t C = Cc.get();
    __shared__ uint32_t h[kMaxColours];
    for (int t = threadIdx.x; t < kMaxColours; t += blockDim.x) h[t] = 0;
    __syncthreads();
    uint32_t cmax = 0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t st = cstate[c];
        uint32_t col = st & 0xFFu;
        if (st == kUncoloured || col >= (uint32_t)kMaxColours) {   // uncoloured or out of range: report, keep indices in bounds
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
__global__ void k_build_sweep(DCount Cc, int64_t n, const uint32_t* __restrict__ perm, const uint32_t* __restrict__ cj1,
                              const uint32_t* __restrict__ cj2, const uint32_t* __restrict__ inst,
                              const double4_32a* __restrict__ cgeo,
                              const double2* __restrict__ clev, double dt, double beta, double mu_all, SceneView V,
                              int warm,
                              const uint32_t* __restrict__ prev_row_off, const uint32_t* __restrict__ prev_j2,
                              const double4_32a* __restrict__ prev_P, int64_t prev_cap, SweepRec<R>* __restrict__ rec,
                              R4<R>* __restrict__ p)
{
    const int64_t C = Cc.get();
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < C; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = perm[s];
        const uint32_t a = cj1[c], b = cj2[c];
        // the velocity records the sweep reads: the bodies, or with subdomains
        // their instances for the contact's subdomain
        const uint32_t ra = inst ? inst[2 * (int64_t)c] : a, rb = inst ? inst[2 * (int64_t)c + 1] : b;
        const double4_32a g = cgeo[c];
        const double2 l = clev[c];
        // eq. (nonpenetration): gap term xi/dt, scaled by beta when xi < 0
        const double xs = g.w >= 0.0 ? g.w : beta * g.w;
        const double bias = xs / dt;
        SweepRec<R> r;
        if constexpr (sizeof(R) == 4) {
            r.a = make_float4(__uint_as_float(ra), __uint_as_float(rb), (float)l.x, (float)l.y);
            r.b = make_float4((float)g.x, (float)g.y, (float)g.z, (float)bias);
        } else {
            r.ids_bias = make_double2(__longlong_as_double((long long)(((uint64_t)rb << 32) | ra)), bias);
            r.lev = make_double2(l.x, l.y);
            r.nxy = make_double2(g.x, g.y);
            r.nz_ = make_double2(g.z, 0.0);
        }
        rec[s] = r;
        // the previous world impulse in the new contact frame, projected onto
        // the friction cone; in the sweep precision (FP64 arithmetic is scarce
        // on this GPU, and an FP32 sweep starts from an FP32 impulse anyway)
        R pn = R(0), pt = R(0), po = R(0), found = R(0);
        if (warm) {
            const uint32_t e = prev_row_off[a + 1];
            for (uint32_t t = prev_row_off[a]; t < e && t < prev_cap; ++t) {
                if (prev_j2[t] != b) continue;
                const double4_32a P = prev_P[t];
                const R mu = (R)(V.batch ? V.mu[V.scene_of[a]] : mu_all);
                const R nx = (R)g.x, ny = (R)g.y, nz = (R)g.z, Px = (R)P.x, Py = (R)P.y, Pz = (R)P.z;
                found = R(1);
                R tx, ty, tz, ox, oy, oz;
                tangent_basis<R>(nx, ny, nz, tx, ty, tz, ox, oy, oz);
                pn = nx * Px + ny * Py + nz * Pz;
                if (!(pn > R(0))) pn = R(0);
                pt = tx * Px + ty * Py + tz * Pz;
                po = ox * Px + oy * Py + oz * Pz;
                const R lim = mu * pn, len = sqrt(pt * pt + po * po);
                if (len > lim) {
                    if (len > R(0)) {
                        pt *= lim / len;
                        po *= lim / len;
                    } else {
                        pt = po = R(0);
                    }
                }
                break;
            }
        }
        R4<R> q;
        q.x = pn;
        q.y = pt;
        q.z = po;
        q.w = found;   // 1: the contact existed in the previous step (read by the network warm start)
        p[s] = q;
    }
}

// Device-sized steps: predecessor entries beyond the buffer set an error bit.
__global__ void k_check_preds(DevInfo* info, int64_t pcap)
{
    if ((int64_t)info->pred_total > pcap) atomicOr(&info->err, kErrPreds);
}

// Resident blocks of the cooperative colouring launch (every block must be
// resident for its grid barriers), looked up once.
static int jp_blocks(const nbgs_scene* s)
{
    static int occ = -1;
    if (occ < 0) {
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, (const void*)k_jp_persistent, kJpThreads, 0);
        cudaGetLastError();
        occ = o > 0 ? o : 1;
    }
    return occ * s->num_sms;
}

nbgs_status run_colour(nbgs_scene* s)
{
    if (!s->detected) return fail(s, NBGS_EINVAL, "colour_contacts: call detect_contacts first");
    cudaStream_t st = s->stream;
    // C: the count, or in device-sized steps the capacity the launches are
    // sized for (the kernels read the count, Cn, on the device)
    const int64_t C = s->n_contacts, n = s->n;
    const DCount Cn = contact_count(s);
    if (s->timing) cudaEventRecord(s->ev[2], st);
    cudaMemsetAsync(s->col_count, 0, (kMaxColours + 1) * sizeof(uint32_t), st);
    cudaMemsetAsync(&s->info->n_colours, 0, sizeof(uint32_t), st);
    cudaMemsetAsync(&s->info->n_shared, 0, 2 * sizeof(uint32_t), st);   // no shared bodies until assigned
    const bool sub = s->prm.subdomain_mode != NBGS_SUB_NONE;
    const bool jacobi = s->prm.subdomain_mode == NBGS_SUB_JACOBI;
    if (C > 0) {
        const int T = 256;
        const int gb = grid_for(C, T, 8, s->num_sms);
        // the conflict graph: contacts sharing a body of finite mass (for
        // composites the body of a member, not the member)
        if (s->composite) {
            nbgs_status rc = run_comp_ends(s);
            if (rc != NBGS_OK) return rc;
        }
        const uint32_t* ib1 = s->composite ? s->cb1 : s->cj1;
        const uint32_t* ib2 = s->composite ? s->cb2 : s->cj2;
        const uint8_t* finc = s->composite ? s->bfinite : s->finite;
        const int64_t ninc = s->composite ? s->nb : n;
        cudaMemsetAsync(s->deg, 0, (ninc + 1) * sizeof(uint32_t), st);
        k_colour_init<<<gb, T, 0, st>>>(Cn, ninc, s->cj1, s->cj2, ib1, ib2, finc, s->prm.colour_seed, scene_view(s),
                                        s->deg, s->cprio, s->cstate);
        nbgs_status rc = exclusive_scan_u32(s, s->deg, s->adj_off, ninc, nullptr);
        if (rc != NBGS_OK) return rc;
        cudaMemsetAsync(s->deg, 0, (ninc + 1) * sizeof(uint32_t), st);
        k_adj_fill<<<gb, T, 0, st>>>(Cn, ninc, ib1, ib2, finc, s->adj_off, s->deg, s->adj);
        if (sub) {
            rc = run_subdomains(s);
            if (rc != NBGS_OK) return rc;
        }
        s->sub_count = sub ? C : -1;
        if (jacobi) {
            // non-linear block Jacobi: no contact sees another's reaction of
            // the same sweep, so a single colour
            cudaMemsetAsync(s->cstate, 0, C * sizeof(uint32_t), st);
        } else {
            // predecessor lists (counts, offsets, lists weakest first)
            k_pred_count<<<gb, T, 0, st>>>(Cn, ninc, ib1, ib2, finc, s->adj_off, s->adj, s->cprio, s->pmask,
                                           s->colour_key);
            rc = exclusive_scan_u32(s, s->colour_key, s->poff, Cn, s->device_sized ? &s->info->pred_total : nullptr);
            if (rc != NBGS_OK) return rc;
            if (s->device_sized) {
                // the lists keep their capacity; an overflow sets an error bit
                k_check_preds<<<1, 1, 0, st>>>(s->info, s->preds_cap);
            } else {
                uint32_t total = 0;
                rc = cuda_check(s, cudaMemcpyAsync(&total, s->poff + C, sizeof(uint32_t), cudaMemcpyDeviceToHost, st),
                                "colour: predecessor count");
                if (rc == NBGS_OK) rc = cuda_check(s, cudaStreamSynchronize(st), "colour");
                if (rc != NBGS_OK) return rc;
                rc = grow_preds(s, total);
                if (rc != NBGS_OK) return rc;
            }
            // waiting lists empty; round-1 counters (|L| = 0, |X| filled below)
            cudaMemsetAsync(s->whead, 0xFF, C * sizeof(uint32_t), st);
            cudaMemsetAsync(s->info->wl_count, 0, sizeof(s->info->wl_count), st);
            k_pred_lists<<<gb, T, 0, st>>>(Cn, ninc, ib1, ib2, finc, s->adj_off, s->adj, s->cprio, s->pmask,
                                           s->poff, s->preds, s->preds_cap, s->whead, s->wnext, s->wl[0],
                                           &s->info->wl_count[1]);
            if (s->timing) s->phase_launches[1] += 9;
            if (s->device_sized) {
                // all rounds in one cooperative launch (grid barrier between rounds)
                cudaMemsetAsync(&s->info->barrier_count, 0, 2 * sizeof(uint32_t), st);
                const int gbr = std::min(jp_blocks(s), grid_for(C, kJpThreads, 8, s->num_sms));
                DCount Cd = Cn;
                uint32_t *wl0 = s->wl[0], *wl1 = s->wl[1], *cnt = s->info->wl_count;
                void* args[] = {(void*)&Cd, (void*)&wl0, (void*)&wl1, (void*)&cnt, (void*)&s->poff, (void*)&s->preds,
                                (void*)&s->cstate, (void*)&s->whead, (void*)&s->wnext, (void*)&s->info};
                rc = cuda_check(s, cudaLaunchCooperativeKernel((const void*)k_jp_persistent, dim3(gbr),
                                                               dim3(kJpThreads), args, 0, st),
                                "colour: rounds");
                if (rc != NBGS_OK) return rc;
                if (s->timing) s->phase_launches[1] += 2;
            } else {
                // one launch per round; the host checks the lists every few rounds
                const int gbr = grid_for(C, kJpThreads, 8, s->num_sms);
                uint32_t round = 0;
                int cur = 0;
                for (int batch = 0; batch < 64; ++batch) {
                    for (int r = 0; r < 6; ++r) {
                        ++round;
                        const int ci = (round - 1) % 3, co = round % 3, cc = (round + 1) % 3;
                        k_jp_round<<<gbr, kJpThreads, 0, st>>>(round, (uint32_t)C, s->wl[cur],
                                                               &s->info->wl_count[2 * ci], s->wl[1 - cur],
                                                               &s->info->wl_count[2 * co], &s->info->wl_count[2 * cc],
                                                               s->poff, s->preds, s->cstate, s->whead, s->wnext,
                                                               s->info);
                        cur = 1 - cur;
                    }
                    if (s->timing) s->phase_launches[1] += 6;
                    uint32_t left[2] = {0, 0};
                    rc = cuda_check(s, cudaMemcpyAsync(left, &s->info->wl_count[2 * (round % 3)], 2 * sizeof(uint32_t),
                                                       cudaMemcpyDeviceToHost, st), "colour: worklist");
                    if (rc != NBGS_OK) return rc;
                    rc = cuda_check(s, cudaStreamSynchronize(st), "colour");
                    if (rc != NBGS_OK) return rc;
                    if (left[0] + left[1] == 0) break;
                    if (batch == 63) return fail(s, NBGS_ETIMEOUT, "colour: did not finish in 384 rounds");
                }
            }
        }
        k_colour_keys<<<gb, T, 0, st>>>(Cn, s->cstate, s->colour_key, s->perm_in, s->col_count, s->info);
        k_colour_offsets<<<1, 32, 0, st>>>(s->col_count, s->col_off);
        // stable counting sort by colour (one 8-bit radix pass): contacts of a
        // colour stay in canonical order
        uint32_t *k0 = s->colour_key, *k1 = s->colour_key2, *v0 = s->perm_in, *v1 = s->perm;
        rc = radix_sort_pairs(s, k0, v0, k1, v1, Cn, 8);
        if (rc != NBGS_OK) return rc;
        // radix_sort_pairs swapped the pointers: v0 / k0 now hold the sorted values / keys
        if (v0 != s->perm) std::swap(s->perm, s->perm_in);
        if (v0 != s->perm) return fail(s, NBGS_EINVAL, "colour: permutation buffer mix-up");
        s->colour_sorted = k0;
        const int warm = (s->prm.warm_start != NBGS_WARM_NONE && s->have_prev) ? 1 : 0;
        if (s->composite) {
            rc = run_comp_records(s, warm);
            if (rc != NBGS_OK) return rc;
        } else if (s->fp32)
            k_build_sweep<float><<<gb, T, 0, st>>>(Cn, n, s->perm, s->cj1, s->cj2, sub ? s->inst : nullptr, s->cgeo,
                                                   s->clev, s->prm.dt,
                                                   s->prm.beta, s->prm.mu, scene_view(s), warm, s->prev_row_off,
                                                   s->prev_j2,
                                                   s->prev_P, s->ccap, (SweepRec<float>*)s->srec, (float4*)s->sp);
        else
            k_build_sweep<double><<<gb, T, 0, st>>>(Cn, n, s->perm, s->cj1, s->cj2, sub ? s->inst : nullptr, s->cgeo,
                                                    s->clev, s->prm.dt,
                                                    s->prm.beta, s->prm.mu, scene_view(s), warm, s->prev_row_off,
                                                    s->prev_j2,
                                                    s->prev_P, s->ccap, (SweepRec<double>*)s->srec,
                                                    (double4_32a*)s->sp);
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
