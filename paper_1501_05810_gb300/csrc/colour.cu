// colour.cu -- contact colouring and the colour-ordered sweep records.
//
// The subdomain numbers s_c(j) of Alg. 1 become colours: two contacts that
// share a body of finite mass never get the same colour, so all contacts of
// one colour can be relaxed at once with in-place velocity updates and no
// atomics, and the result equals the sequential NBGS in colour order.
//
//   k_colour_init   priority splitmix64(key ^ seed), body degrees
//   scan + k_adj_fill  body -> contact incidence lists (finite bodies only)
//   k_adj_sort_*    every incidence list in decreasing priority; each
//                   contact's position in the lists of its bodies
//   k_fr_round      rounds of first-fit greedy colouring in decreasing
//                   priority, as Jones-Plassmann rounds give it: a contact
//                   at the front of the remaining lists of all its bodies
//                   takes the smallest colour absent from their coloured
//                   prefixes (k_fr_persistent: every round in one
//                   cooperative launch, for device-sized steps)
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

constexpr uint32_t kNoList = 0xFFFFFFFFu;   // a contact end without an incidence list (wall, infinite mass)

// Priorities from the contacts' keys; body degrees from the incidence ends
// ib1, ib2 (the contact's bodies: the contact ends themselves for spheres,
// the members' bodies for composites; >= n marks a wall).
__global__ void k_colour_init(DCount Cc, int64_t n, const uint32_t* __restrict__ cj1, const uint32_t* __restrict__ cj2,
                              const uint32_t* __restrict__ ib1, const uint32_t* __restrict__ ib2,
                              const uint8_t* __restrict__ finite, uint64_t seed, SceneView V, uint32_t* __restrict__ deg,
                              uint64_t* __restrict__ prio, uint32_t* __restrict__ cstate, uint4* __restrict__ cpack)
{
    const int64_t C = Cc.get();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        prio[c] = splitmix64(local_key(cj1[c], cj2[c], V) ^ seed);
        cstate[c] = kUncoloured;
        const uint32_t a = ib1[c], b = ib2[c];
        const bool fa = finite[a] != 0, fb = b < n && finite[b];
        if (fa) atomicAdd(&deg[a], 1u);
        if (fb) atomicAdd(&deg[b], 1u);
        // the bodies whose incidence lists hold c (none: no list), positions later
        cpack[c] = make_uint4(fa ? a : kNoList, fb ? b : kNoList, 0u, 0u);
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

// Colouring by priority-ordered incidence lists.  First-fit greedy
// colouring in decreasing priority gives each contact the smallest colour
// none of its predecessors (incident contacts that beat it) has.  With the
// incidence list of every body sorted by priority, the predecessors of c
// are the entries before c in the lists of its bodies.  A body's front is
// the length of the coloured prefix of its list, and its mask the set of
// colours in that prefix; c can be coloured once it is at the front of the
// lists of all its (finite) bodies, and its colour is the smallest one in
// none of their masks.  Colouring c adds its colour to those masks,
// advances the fronts by one and exposes the next entry of each list, which
// the next round colours if it is at the front of its other body's list
// too (else that body's front exposes it later).  Each round colours
// exactly the contacts whose predecessors were all coloured before it: the
// rounds of Jones-Plassmann, with O(1) work per contact and round.
//
// A body's front is advanced at most once per round (only its front entry
// can be coloured), and it is tagged with the round that advanced it: a
// contact checked in the same round sees the value the front had when the
// round began.  So each round reads only what earlier rounds wrote (a launch
// boundary or a grid barrier apart), and a body's mask is written only by
// the one contact at its front.
constexpr uint32_t kFrontBits = 20;   // position bits of a front word; the round above them
constexpr int kJpThreads = 256;       // threads of a colouring round's blocks
constexpr uint32_t kClaimed = 0xFFFFFFFEu;

__device__ __forceinline__ uint32_t front_at(uint32_t f, uint32_t round)
{
    const uint32_t v = f & ((1u << kFrontBits) - 1u);
    return (f >> kFrontBits) == round ? v - 1u : v;
}

// Incidence lists in decreasing priority ("beats" order), and each
// contact's position in the lists of its bodies (cpack z for its first
// body, w for its second).  Short lists (up to 16 contacts, every sphere
// scene) take a bitonic network in a thread's registers; longer ones a
// warp, lane l holding entries l, l + 32, ..., an entry's position being the
// number of entries that beat it, counted over the others broadcast by
// shuffles (one lane sorts lists beyond the warp's slots in place).
constexpr uint32_t kShortList = 16;
constexpr int kSortSlots = 8;   // entries per lane of the warp sort: lists of up to 256 contacts

__device__ __forceinline__ void set_position(uint4* cpack, uint32_t c, uint32_t x, uint32_t k)
{
    uint32_t* q = reinterpret_cast<uint32_t*>(cpack + c);
    q[q[0] == x ? 2 : 3] = k;
}

// Also empties the front and colour mask of every body with a list (the
// rounds read no other body's) and collects the bodies with long lists.
__global__ void k_adj_sort_short(int64_t n, const uint8_t* __restrict__ finite, const uint32_t* __restrict__ adj_off,
                                 uint32_t* __restrict__ adj, const uint64_t* __restrict__ prio,
                                 uint4* __restrict__ cpack, uint32_t* __restrict__ front, uint32_t* __restrict__ mask,
                                 uint32_t* __restrict__ longs, uint32_t* n_long)
{
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        if (!finite[x]) continue;
        const uint32_t a0 = adj_off[x], m = adj_off[x + 1] - a0;
        if (m == 0) continue;
        front[x] = 0u;
        uint4* mk = reinterpret_cast<uint4*>(mask + 8 * x);
        mk[0] = make_uint4(0u, 0u, 0u, 0u);
        mk[1] = make_uint4(0u, 0u, 0u, 0u);
        if (m > kShortList) {
            longs[atomicAdd(n_long, 1u)] = (uint32_t)x;
            continue;
        }
        uint32_t id[kShortList];
        uint64_t pr[kShortList];
#pragma unroll
        for (uint32_t i = 0; i < kShortList; ++i) id[i] = i < m ? adj[a0 + i] : 0xFFFFFFFFu;
#pragma unroll
        for (uint32_t i = 0; i < kShortList; ++i) pr[i] = i < m ? prio[id[i]] : 0ull;   // padding sorts last
        // bitonic network: after it, entry i beats entry i + 1
#pragma unroll
        for (uint32_t k = 2; k <= kShortList; k <<= 1) {
#pragma unroll
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
                for (uint32_t i = 0; i < kShortList; ++i) {
                    const uint32_t l = i ^ j;
                    if (l <= i) continue;
                    const bool first = (i & k) == 0;   // this half ends with i beating l
                    const bool swap = first ? beats(pr[l], id[l], pr[i], id[i]) : beats(pr[i], id[i], pr[l], id[l]);
                    if (swap) {
                        const uint32_t ti = id[i];
                        const uint64_t tp = pr[i];
                        id[i] = id[l];
                        pr[i] = pr[l];
                        id[l] = ti;
                        pr[l] = tp;
                    }
                }
            }
        }
#pragma unroll
        for (uint32_t i = 0; i < kShortList; ++i) {
            if (i < m) {
                adj[a0 + i] = id[i];
                set_position(cpack, id[i], (uint32_t)x, i);
            }
        }
    }
}

// One list of m entries (m <= 32 K) by the warp: lane l holds entries l,
// l + 32, ...; an entry's position is the number of entries that beat it.
template <int K>
__device__ __forceinline__ void warp_sort_list(uint32_t x, uint32_t a0, uint32_t m, uint32_t lane,
                                               uint32_t* __restrict__ adj, const uint64_t* __restrict__ prio,
                                               uint4* __restrict__ cpack)
{
    uint32_t id[K], rk[K];
    uint64_t pr[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const uint32_t i = lane + 32u * k;
        id[k] = i < m ? adj[a0 + i] : 0u;
        rk[k] = 0u;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) pr[k] = lane + 32u * k < m ? prio[id[k]] : 0ull;
#pragma unroll
    for (int kc = 0; kc < K; ++kc) {
        if (32u * kc >= m) break;
        const uint32_t cnt = min(32u, m - 32u * kc);
        for (uint32_t l = 0; l < cnt; ++l) {
            const uint32_t idj = __shfl_sync(0xffffffffu, id[kc], l);
            const uint64_t prj = __shfl_sync(0xffffffffu, pr[kc], l);
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (lane + 32u * k < m && beats(prj, idj, pr[k], id[k])) ++rk[k];
        }
    }
    __syncwarp();   // every entry read before any is overwritten
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (lane + 32u * k >= m) continue;
        adj[a0 + rk[k]] = id[k];
        set_position(cpack, id[k], x, rk[k]);
    }
}

__global__ void k_adj_sort_long(const uint32_t* __restrict__ longs, const uint32_t* __restrict__ n_long,
                                const uint32_t* __restrict__ adj_off, uint32_t* __restrict__ adj,
                                const uint64_t* __restrict__ prio, uint4* __restrict__ cpack)
{
    const uint32_t lane = threadIdx.x & 31u;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5, nl = *n_long;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nl; k += nw) {
        const uint32_t x = longs[k];   // the same for every lane of the warp
        const uint32_t a0 = adj_off[x], m = adj_off[x + 1] - a0;
        if (m <= 32u) warp_sort_list<1>(x, a0, m, lane, adj, prio, cpack);
        else if (m <= 64u) warp_sort_list<2>(x, a0, m, lane, adj, prio, cpack);
        else if (m <= 128u) warp_sort_list<4>(x, a0, m, lane, adj, prio, cpack);
        else if (m <= 32u * kSortSlots) warp_sort_list<kSortSlots>(x, a0, m, lane, adj, prio, cpack);
        else if (lane == 0) {   // beyond the slots: insertion sort by one lane
            for (uint32_t i = 1; i < m; ++i) {
                const uint32_t c = adj[a0 + i];
                const uint64_t pc = prio[c];
                uint32_t j = i;
                while (j > 0) {
                    const uint32_t d = adj[a0 + j - 1];
                    if (!beats(pc, c, prio[d], d)) break;
                    adj[a0 + j] = d;
                    --j;
                }
                adj[a0 + j] = c;
            }
            for (uint32_t q = 0; q < m; ++q) set_position(cpack, adj[a0 + q], x, q);
        }
    }
}

// Block-wide append of up to two values per thread to list (cap entries):
// one counter update per block (a counter every block of a round appends
// to is contended).  Entries beyond cap set the colour error bit.
__device__ __forceinline__ void block_push2(uint32_t e0, uint32_t e1, uint32_t* list, uint32_t* count, int64_t cap,
                                            DevInfo* info)
{
    __shared__ uint32_t s_buf[2 * kJpThreads];
    __shared__ uint32_t s_n, s_base;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    if (e0 != kUncoloured) s_buf[atomicAdd(&s_n, 1u)] = e0;
    if (e1 != kUncoloured) s_buf[atomicAdd(&s_n, 1u)] = e1;
    __syncthreads();
    const uint32_t k = s_n;
    if (threadIdx.x == 0) s_base = k ? atomicAdd(count, k) : 0u;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) {
        const int64_t idx = (int64_t)s_base + i;
        if (idx < cap) list[idx] = s_buf[i];
        else atomicOr(&info->err, kErrColours);
    }
    __syncthreads();   // the buffer is refilled by the next call
}

// The contacts at the front of all their lists from the start (no
// predecessor) form the first round's list.
__global__ void k_fr_seed(DCount Cc, const uint4* __restrict__ cpack, uint32_t* __restrict__ wl, uint32_t* count,
                          DevInfo* info)
{
    const int64_t C = Cc.get();
    // block-uniform trip count: every thread takes part in block_push2
    for (int64_t c0 = blockIdx.x * (int64_t)blockDim.x; c0 < C; c0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = c0 + threadIdx.x;
        bool ready = false;
        if (c < C) {
            const uint4 q = cpack[c];
            ready = (q.x == kNoList || q.z == 0u) && (q.y == kNoList || q.w == 0u);
        }
        block_push2(ready ? (uint32_t)c : kUncoloured, kUncoloured, wl, count, C, info);
    }
}

// One round over the list `in` (cnt_in entries); the contacts exposed go to
// `out`.  cnt_clear (the counter two rounds ahead) is zeroed for reuse.
__device__ __forceinline__ void fr_round(uint32_t round, const uint4* __restrict__ cpack,
                                         const uint32_t* __restrict__ adj_off, const uint32_t* __restrict__ adj,
                                         uint32_t* front, uint32_t* mask, const uint32_t* in, uint32_t m, uint32_t* out,
                                         uint32_t* cnt_out, int64_t cap, uint32_t* cstate, DevInfo* info)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // block-uniform trip count: every thread takes part in block_push2
    for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x; t0 < m; t0 += stride) {
        const int64_t t = t0 + threadIdx.x;
        uint32_t e0 = kUncoloured, e1 = kUncoloured;
        if (t < m) {
            const uint32_t c = in[t];
            const uint4 q = cpack[c];
            const uint32_t a = q.x, b = q.y, pa = q.z, pb = q.w;
            const bool fa = a != kNoList, fb = b != kNoList;
            const bool ready = (!fa || front_at(__ldcg(front + a), round) == pa) &&
                               (!fb || front_at(__ldcg(front + b), round) == pb);
            // an entry exposed twice, or already coloured: the claim fails
            if (ready && atomicCAS(cstate + c, kUncoloured, kClaimed) == kUncoloured) {
                const uint4 z = make_uint4(0u, 0u, 0u, 0u);
                const uint4* ma = reinterpret_cast<const uint4*>(mask + 8 * (int64_t)a);
                const uint4* mb = reinterpret_cast<const uint4*>(mask + 8 * (int64_t)b);
                const uint4 a_lo = fa ? __ldcg(ma) : z, a_hi = fa ? __ldcg(ma + 1) : z;
                const uint4 b_lo = fb ? __ldcg(mb) : z, b_hi = fb ? __ldcg(mb + 1) : z;
                const uint32_t used[8] = {a_lo.x | b_lo.x, a_lo.y | b_lo.y, a_lo.z | b_lo.z, a_lo.w | b_lo.w,
                                          a_hi.x | b_hi.x, a_hi.y | b_hi.y, a_hi.z | b_hi.z, a_hi.w | b_hi.w};
                uint32_t col = kMaxColours;
#pragma unroll
                for (int k = 7; k >= 0; --k)
                    if (~used[k]) col = 32u * k + (__ffs(~used[k]) - 1);
                if (col >= (uint32_t)kMaxColours) {
                    atomicOr(&info->err, kErrColours);
                    col = kMaxColours - 1;
                }
                cstate[c] = col;
                const uint32_t bit = 1u << (col & 31u), wd = col >> 5;
                // only c, the front of a and of b, writes their masks and fronts
                if (fa) {
                    __stcg(mask + 8 * (int64_t)a + wd, __ldcg(mask + 8 * (int64_t)a + wd) | bit);
                    __stcg(front + a, (round << kFrontBits) | (pa + 1));
                    const uint32_t a0 = adj_off[a];
                    if (pa + 1 < adj_off[a + 1] - a0) e0 = adj[a0 + pa + 1];
                }
                if (fb) {
                    __stcg(mask + 8 * (int64_t)b + wd, __ldcg(mask + 8 * (int64_t)b + wd) | bit);
                    __stcg(front + b, (round << kFrontBits) | (pb + 1));
                    const uint32_t b0 = adj_off[b];
                    if (pb + 1 < adj_off[b + 1] - b0) e1 = adj[b0 + pb + 1];
                }
            }
        }
        block_push2(e0, e1, out, cnt_out, cap, info);
    }
}

// One round per launch (the host checks the list counts every few rounds).
// The counters rotate through three slots: a round reads one, writes the
// next and clears the third.
__global__ void __launch_bounds__(kJpThreads) k_fr_round(uint32_t round, const uint4* __restrict__ cpack,
                                                         const uint32_t* __restrict__ adj_off,
                                                         const uint32_t* __restrict__ adj, uint32_t* front,
                                                         uint32_t* mask, const uint32_t* in, const uint32_t* cnt_in,
                                                         uint32_t* out, uint32_t* cnt_out, uint32_t* cnt_clear,
                                                         int64_t cap, uint32_t* cstate, DevInfo* info)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *cnt_clear = 0u;
        if (*cnt_in > 0u) info->rounds = round;   // the last round with work
    }
    fr_round(round, cpack, adj_off, adj, front, mask, in, *cnt_in, out, cnt_out, cap, cstate, info);
}

// All rounds in one cooperative launch (no host in the loop, so a step can
// be captured in a CUDA graph): a grid barrier ends each round (it plays
// the part of a launch boundary), and the round's output count, read by
// every block after the barrier, tells whether anything is left.  More than
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

__global__ void __launch_bounds__(kJpThreads) k_fr_persistent(DCount Cc, const uint4* __restrict__ cpack,
                                                              const uint32_t* __restrict__ adj_off,
                                                              const uint32_t* __restrict__ adj, uint32_t* front,
                                                              uint32_t* mask, uint32_t* wl0, uint32_t* wl1,
                                                              uint32_t* cnt, uint32_t* cstate, DevInfo* info)
{
    const int64_t C = Cc.get();
    if (C == 0) return;
    for (uint32_t round = 1; round <= (uint32_t)kJpMaxRounds; ++round) {
        const int ci = (round - 1) % 3, co = round % 3, cc = (round + 1) % 3;
        const bool odd = (round & 1u) != 0u;   // round 1 reads wl0 and writes wl1, round 2 the reverse, ...
        if (blockIdx.x == 0 && threadIdx.x == 0) cnt[cc] = 0u;
        fr_round(round, cpack, adj_off, adj, front, mask, odd ? wl0 : wl1, __ldcg(cnt + ci), odd ? wl1 : wl0,
                 cnt + co, 2 * C, cstate, info);
        if (!jp_barrier(info)) return;
        if (__ldcg(cnt + co) == 0u) return;   // nothing exposed: every contact is coloured
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

// Slot of every canonical contact in colour order: the inverse of perm.
__global__ void k_invert(DCount Cc, const uint32_t* __restrict__ perm, uint32_t* __restrict__ inv)
{
    const int64_t C = Cc.get();
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < C; s += (int64_t)gridDim.x * blockDim.x)
        inv[perm[s]] = (uint32_t)s;
}

// Sweep record inv[c] <- canonical contact c; initial impulse from the
// previous step (world frame, re-projected onto the new frame and the cone)
// or zero.  A thread per canonical contact: the contact arrays and the
// previous step's rows are read in order, the records written scattered.
template <class R>
__global__ void k_build_sweep(DCount Cc, int64_t n, const uint32_t* __restrict__ inv, const uint32_t* __restrict__ cj1,
                              const uint32_t* __restrict__ cj2, const uint32_t* __restrict__ inst,
                              const double4_32a* __restrict__ cgeo,
                              const double2* __restrict__ clev, double dt, double beta, double mu_all, SceneView V,
                              int warm,
                              const uint32_t* __restrict__ prev_row_off, const uint32_t* __restrict__ prev_j2,
                              const double4_32a* __restrict__ prev_P, int64_t prev_cap, SweepRec<R>* __restrict__ rec,
                              R4<R>* __restrict__ p)
{
    const int64_t C = Cc.get();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = inv[c];
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

// Resident blocks of the cooperative colouring launch (every block must be
// resident for its grid barriers), looked up once.
static int fr_blocks(const nbgs_scene* s)
{
    static int occ = -1;
    if (occ < 0) {
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, (const void*)k_fr_persistent, kJpThreads, 0);
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
                                        s->deg, s->cprio, s->cstate, s->cpack);
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
            // incidence lists in priority order, fronts and masks empty, the
            // contacts without predecessors as the first round's list
            uint32_t* front = s->deg;   // scratch again (the degrees are adj_off's differences); emptied per body below
            // (the bodies with long lists go to wl[1], counted in wl_count[3])
            cudaMemsetAsync(s->info->wl_count, 0, 4 * sizeof(uint32_t), st);
            k_adj_sort_short<<<grid_for(ninc, T, 8, s->num_sms), T, 0, st>>>(ninc, finc, s->adj_off, s->adj,
                                                                              s->cprio, s->cpack, front, s->cmask,
                                                                              s->wl[1], &s->info->wl_count[3]);
            k_adj_sort_long<<<8 * s->num_sms, T, 0, st>>>(s->wl[1], &s->info->wl_count[3], s->adj_off, s->adj,
                                                           s->cprio, s->cpack);
            k_fr_seed<<<gb, T, 0, st>>>(Cn, s->cpack, s->wl[0], &s->info->wl_count[0], s->info);
            if (s->timing) s->phase_launches[1] += 5;
            if (s->device_sized) {
                // all rounds in one cooperative launch (grid barrier between rounds)
                cudaMemsetAsync(&s->info->barrier_count, 0, 2 * sizeof(uint32_t), st);
                const int gbr = std::min(fr_blocks(s), grid_for(C, kJpThreads, 8, s->num_sms));
                DCount Cd = Cn;
                uint32_t *wl0 = s->wl[0], *wl1 = s->wl[1], *cnt = s->info->wl_count, *msk = s->cmask;
                const uint4* cp = s->cpack;
                void* args[] = {(void*)&Cd, (void*)&cp, (void*)&s->adj_off, (void*)&s->adj, (void*)&front,
                                (void*)&msk, (void*)&wl0, (void*)&wl1, (void*)&cnt, (void*)&s->cstate, (void*)&s->info};
                rc = cuda_check(s, cudaLaunchCooperativeKernel((const void*)k_fr_persistent, dim3(gbr),
                                                               dim3(kJpThreads), args, 0, st),
                                "colour: rounds");
                if (rc != NBGS_OK) return rc;
                if (s->timing) s->phase_launches[1] += 2;
            } else {
                // one launch per round; the host checks the list counts after as
                // many rounds as the last colouring took, then every four
                const int gbr = grid_for(C, kJpThreads, 8, s->num_sms);
                uint32_t round = 0;
                int cur = 0;
                int batch = std::max(4, s->colour_rounds);
                for (;;) {
                    for (int r = 0; r < batch; ++r) {
                        ++round;
                        const int ci = (round - 1) % 3, co = round % 3, cc = (round + 1) % 3;
                        k_fr_round<<<gbr, kJpThreads, 0, st>>>(round, s->cpack, s->adj_off, s->adj, front, s->cmask,
                                                               s->wl[cur], &s->info->wl_count[ci], s->wl[1 - cur],
                                                               &s->info->wl_count[co], &s->info->wl_count[cc], 2 * C,
                                                               s->cstate, s->info);
                        cur = 1 - cur;
                    }
                    if (s->timing) s->phase_launches[1] += batch;
                    uint32_t left = 0, used = 0;
                    rc = cuda_check(s, cudaMemcpyAsync(&left, &s->info->wl_count[round % 3], sizeof(uint32_t),
                                                       cudaMemcpyDeviceToHost, st), "colour: list count");
                    if (rc == NBGS_OK)
                        rc = cuda_check(s, cudaMemcpyAsync(&used, &s->info->rounds, sizeof(uint32_t),
                                                           cudaMemcpyDeviceToHost, st), "colour: rounds");
                    if (rc != NBGS_OK) return rc;
                    rc = cuda_check(s, cudaStreamSynchronize(st), "colour");
                    if (rc != NBGS_OK) return rc;
                    if (left == 0) {
                        s->colour_rounds = (int)used + 1;
                        break;
                    }
                    if (round >= (uint32_t)kJpMaxRounds) return fail(s, NBGS_ETIMEOUT, "colour: did not finish in 1024 rounds");
                    batch = 4;
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
        // the slots of the canonical contacts (perm_in is free after the sort;
        // the records and the solve's finish read it)
        k_invert<<<gb, T, 0, st>>>(Cn, s->perm, s->perm_in);
        if (s->timing) s->phase_launches[1] += 1;
        if (s->composite) {
            rc = run_comp_records(s, warm);
            if (rc != NBGS_OK) return rc;
        } else if (s->fp32)
            k_build_sweep<float><<<gb, T, 0, st>>>(Cn, n, s->perm_in, s->cj1, s->cj2, sub ? s->inst : nullptr, s->cgeo,
                                                   s->clev, s->prm.dt,
                                                   s->prm.beta, s->prm.mu, scene_view(s), warm, s->prev_row_off,
                                                   s->prev_j2,
                                                   s->prev_P, s->ccap, (SweepRec<float>*)s->srec, (float4*)s->sp);
        else
            k_build_sweep<double><<<gb, T, 0, st>>>(Cn, n, s->perm_in, s->cj1, s->cj2, sub ? s->inst : nullptr, s->cgeo,
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
