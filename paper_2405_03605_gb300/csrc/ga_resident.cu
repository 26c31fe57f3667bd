// ga_resident.cu -- resident stepping: a run whose islands all fit on the GPU at once stays
// in registers for a whole chunk of generations, in one cooperative launch, and its islands
// trade migrants through mailboxes in global memory (L2) instead of through launch
// boundaries.  The paper's processors keep their populations in place and exchange only
// migrants with their neighbours (Sec. 2); this is that arrangement on the GPU, for runs
// small enough that a launch per generation would be bound by launch latency.
//
// Scope: synchronous runs whose counters all equal the generation, 16-byte records (trait or
// float fitness, counter, 64-bit surface).  Results are bit-identical to the streamed
// kernels: the same draws, landing slots, tournaments, mutations and deposits.
//
// Islands of 32 and 64 agents take resident_warp_kernel: one island per warp, which pushes,
// polls and lands its own migrants with no block barrier (described at the kernel).
// Islands of 8 and 16 agents share warps and take resident_kernel.  Its block: WARPS island
// warps (the mapping of step_block) plus BK bookkeeping warps, one lane per (island,
// direction).  On each migration generation g:
//   A. block barrier: the bookkeeping lanes have prepared g's sends (below) and the island
//      warps hold the state before g;
//   B. island warps push: for each direction d the member that the neighbour R = nb(I, d)
//      draws (bits 8..15 of word 3 of R's slot-(d^1) birth draw) is written, with one 128-bit
//      atomic exchange, into R's mailbox for direction d^1 and generation parity (g/k) & 1;
//      bookkeeping lanes poll their island's mailbox for direction d (128-bit atomic reads)
//      until it holds a record whose counter is g -- the record is its own ready flag, as
//      every counter equals the generation -- and place it at the landing slot (the partial
//      Fisher-Yates draw of the synchronous mode);
//      meanwhile the island warps compute g's birth draws, which need nothing exchanged;
//   C. block barrier; island warps land the immigrants and reproduce g and the generations up
//      to the next migration, while the bookkeeping lanes prepare the next migration
//      generation's sends (two Philox calls per lane: the neighbour's draw for the emigrant
//      and the island's own for the landing slot).
// Every island pushes before it polls, and a cooperative launch keeps every block resident,
// so each poll is answered once the neighbour reaches the same generation.  Mailboxes are
// double-buffered by generation parity: a sender can only overwrite a parity slot after it
// has received the receiver's next push, which the receiver makes after reading that slot.
//
// Waits are bounded: a poll gives up after the run's wait limit (wall clock, %globaltimer),
// records GA_ETIMEOUT in the status word and sets the launch's abort word; every poll also
// watches the abort word, so once one block gives up every block leaves at its next
// migration generation.  The population is then undefined; the status is returned by the
// next ga_sync.
#include "ga_device.cuh"
#include "ga_internal.h"
#include "ga_island.cuh"

namespace ga {

RunParams run_params(const ga_run *run, const void *src, void *dst, uint32_t g0, uint32_t n_gens,
                     bool migrate);

namespace {

struct ResidentArgs {
    RunParams r;
    RoundKeys rk;
    uint4 *mail;             // [2][n_islands * 4] mailboxes (all ones when empty)
    uint32_t *abort_word;    // 0; set to 1 by a block that gave up waiting
    unsigned long long wait_ns;
    uint32_t every_k, per_neighbor;
    uint32_t drop_island;    // fault injection: this island's pushes are dropped (~0u: none)
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// 128-bit atomic read: a compare-and-swap of all ones with all ones never changes memory
// (a record is all ones only when its mailbox is empty) and returns the 16 bytes at once.
__device__ __forceinline__ uint4 read128(uint4 *p)
{
    unsigned long long lo, hi;
    const unsigned long long ones = ~0ull;
    asm volatile("{\n\t.reg .b128 cv, ov;\n\t"
                 "mov.b128 cv, {%2, %3};\n\t"
                 "atom.relaxed.gpu.global.cas.b128 ov, [%4], cv, cv;\n\t"
                 "mov.b128 {%0, %1}, ov;\n\t}"
                 : "=l"(lo), "=l"(hi) : "l"(ones), "l"(ones), "l"(p) : "memory");
    return make_uint4(static_cast<uint32_t>(lo), static_cast<uint32_t>(lo >> 32),
                      static_cast<uint32_t>(hi), static_cast<uint32_t>(hi >> 32));
}

// 128-bit atomic write (exchange; the old contents are not needed).
__device__ __forceinline__ void write128(uint4 *p, uint4 v)
{
    [[maybe_unused]] unsigned long long lo, hi;
    const unsigned long long vlo = static_cast<unsigned long long>(v.x) |
                                   (static_cast<unsigned long long>(v.y) << 32);
    const unsigned long long vhi = static_cast<unsigned long long>(v.z) |
                                   (static_cast<unsigned long long>(v.w) << 32);
    asm volatile("{\n\t.reg .b128 nv, ov;\n\t"
                 "mov.b128 nv, {%2, %3};\n\t"
                 "atom.relaxed.gpu.global.exch.b128 ov, [%4], nv;\n\t"
                 "mov.b128 {%0, %1}, ov;\n\t}"
                 : "=l"(lo), "=l"(hi) : "l"(vlo), "l"(vhi), "l"(p) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int N, int WARPS>
struct ResidentShape {
    static constexpr int BI = WARPS * Shape<N>::P;  // islands per block
    static constexpr int ML = 4 * BI;               // bookkeeping lanes
    static constexpr int BK = (ML + 31) / 32;       // bookkeeping warps
    static constexpr int THREADS = (WARPS + BK) * 32;
};

// Next migration generation at or after g (~0u: none before `end`).
__device__ __forceinline__ uint32_t next_migration(uint32_t g, uint32_t end, uint32_t k, uint32_t on)
{
    if (!on) return ~0u;
    const uint32_t r = g % k;
    const uint64_t m = static_cast<uint64_t>(g) + (r ? k - r : 0u);
    return m < end ? static_cast<uint32_t>(m) : ~0u;
}

template <int N, int TS, int MODEL, int WARPS>
__global__ void __launch_bounds__(ResidentShape<N, WARPS>::THREADS)
resident_kernel(const ResidentArgs a)
{
    using RS = ResidentShape<N, WARPS>;
    constexpr int A = Shape<N>::A, P = Shape<N>::P, SEG = Shape<N>::SEG;
    constexpr int BI = RS::BI, ML = RS::ML, LW = 4;
    static_assert(N <= 16, "islands of 32 and 64 agents take resident_warp_kernel");
    __shared__ uint32_t s_send_e[ML];    // member of the island that neighbour R draws
    __shared__ uint32_t s_send_box[ML];  // R's mailbox index: R * 4 + (d ^ 1)
    __shared__ uint4 s_in[BI * N];       // arrivals by (island, slot)
    __shared__ uint32_t s_hit[BI];       // slots that received one, by island
    __shared__ int s_abort;
    const RunParams &p = a.r;

    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const bool island_warp = warp < static_cast<uint32_t>(WARPS);
    const uint32_t island0 = blockIdx.x * BI;
    const uint32_t end = p.g0 + p.n_gens;

    // island lanes
    const uint32_t seg_lane = lane % SEG;
    const uint32_t local = warp * P + lane / SEG;
    const uint32_t island = island0 + local;
    const bool valid = island_warp && island < p.n_islands;
    const unsigned mask = __ballot_sync(0xffffffffu, valid);

    // bookkeeping lanes: (island t / 4, direction t % 4)
    const uint32_t t = threadIdx.x - WARPS * 32u;
    const bool bk = !island_warp && t < static_cast<uint32_t>(ML);
    const unsigned bk_mask = __ballot_sync(0xffffffffu, bk);
    const uint32_t md = t & 3u;
    const uint32_t bk_isl = island0 + (t >> 2);
    const bool bk_ok = bk && bk_isl < p.n_islands;
    uint32_t bk_slot = 0;  // landing slot of this lane's direction at the prepared generation

    // the bookkeeping lanes' share of migration generation gm: the emigrant the neighbour
    // draws, where it goes, and this island's own landing slot for direction md
    auto prepare = [&](uint32_t gm) {
        uint32_t r = md;
        if (bk_ok) {
            const uint32_t y = div_cols(bk_isl, p.cols_m, p.cols_l), x = bk_isl - y * p.cols;
            const uint32_t yn = md == 0u ? (y == 0u ? p.rows - 1u : y - 1u)
                              : md == 1u ? (y + 1u == p.rows ? 0u : y + 1u) : y;
            const uint32_t xn = md == 2u ? (x + 1u == p.cols ? 0u : x + 1u)
                              : md == 3u ? (x == 0u ? p.cols - 1u : x - 1u) : x;
            const uint32_t nb = yn * p.cols + xn;
            const uint32_t un = philox_rk(gm, nb, (md ^ 1u) | (kBirth << 16), p.run_id, a.rk).w;
            s_send_e[t] = (((un >> 8) & 0xFFu) * N) >> 8;
            s_send_box[t] = nb * 4u + (md ^ 1u);
            const uint32_t uo = philox_rk(gm, bk_isl, md | (kBirth << 16), p.run_id, a.rk).w;
            r = md + (((uo >> 16) * static_cast<uint32_t>(N - md)) >> 16);
        }
        if (bk) {
            uint32_t rr[4];
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) rr[dd] = __shfl_sync(bk_mask, r, dd, 4);
            uint32_t v[4];
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) {
                uint32_t vd = dd, vr = rr[dd];
#pragma unroll
                for (int e = 0; e < dd; ++e) {
                    if (rr[e] == static_cast<uint32_t>(dd)) vd = v[e];
                    if (rr[e] == rr[dd]) vr = v[e];
                }
                if (static_cast<uint32_t>(dd) == md) bk_slot = vr;
                v[dd] = vd;
            }
        }
    };

    uint32_t rec[A][LW];
    if (valid) {
#pragma unroll
        for (int ag = 0; ag < A; ++ag) {
            const uint4 v = __ldg(&p.src[static_cast<size_t>(island) * N + seg_lane + 32u * ag]);
            rec[ag][0] = v.x;
            rec[ag][1] = v.y;
            rec[ag][2] = v.z;
            rec[ag][3] = v.w;
        }
    }
    if (threadIdx.x == 0) s_abort = 0;
    uint32_t gm = next_migration(p.g0, end, a.every_k, a.per_neighbor);
    if (gm != ~0u) prepare(gm);

    bool aborted = false;
    for (uint32_t it = 0; it < p.n_gens; ++it) {
        const uint32_t g = p.g0 + it;
        uint4 w[A];
        bool drawn = false;
        if (g == gm) {  // the same generation for every thread of the block
            __syncthreads();  // A
            uint4 *box = a.mail + static_cast<size_t>((g / a.every_k) & 1u) * p.n_islands * 4u;
            if (valid && island != a.drop_island) {
#pragma unroll
                for (int dd = 0; dd < 4; ++dd) {
                    const uint32_t e = s_send_e[4u * local + dd];
#pragma unroll
                    for (int ag = 0; ag < A; ++ag) {
                        if (seg_lane + 32u * ag == e) {
                            const uint32_t dst = s_send_box[4u * local + dd];
                            if (in_bounds(dst < p.n_islands * 4u, p.status))
                                write128(box + dst, make_uint4(rec[ag][0], rec[ag][1], rec[ag][2], rec[ag][3]));
                        }
                    }
                }
            }
            // the generation's birth draws need nothing from the neighbours: the island warps
            // compute them while the bookkeeping lanes wait for the mailboxes
            if (valid) {
                birth_draws<N>(w, p, a.rk, g, island, seg_lane);
                drawn = true;
            }
            uint4 imm = make_uint4(0u, 0u, 0u, 0u);
            if (bk_ok) {
                uint4 *mine = box + static_cast<size_t>(bk_isl) * 4u + md;
                const unsigned long long t0 = global_ns();
                for (uint32_t polls = 0;; ++polls) {
                    // the abort word is read beside the mailbox, not after it: a poll that
                    // finds nothing costs one round trip to L2, not two
                    imm = read128(mine);
                    const uint32_t ab = ld_relaxed_u32(a.abort_word);
                    if (imm.y == g) break;
                    if (ab != 0u) {
                        s_abort = 1;
                        break;
                    }
                    if (global_ns() - t0 > a.wait_ns) {
                        atomicCAS(p.status, 0, GA_ETIMEOUT);
                        atomicExch(a.abort_word, 1u);
                        s_abort = 1;
                        break;
                    }
                    if (polls >= 8u) __nanosleep(64);
                }
            }
            if (bk) {
                const uint32_t li = t >> 2;
                uint32_t bit = 1u << bk_slot;
                bit |= __shfl_xor_sync(bk_mask, bit, 1, 4);
                bit |= __shfl_xor_sync(bk_mask, bit, 2, 4);
                if (bk_ok && in_bounds(li * N + bk_slot < static_cast<uint32_t>(BI * N), p.status))
                    s_in[li * N + bk_slot] = imm;
                if (md == 0u) s_hit[li] = bit;
            }
            __syncthreads();  // C
            if (s_abort) {
                aborted = true;
                break;
            }
            if (valid) {
                const bool hit = ((s_hit[local] >> seg_lane) & 1u) != 0u;
                const uint4 xq = s_in[local * N + seg_lane];
                if (hit) {
                    rec[0][0] = xq.x;
                    rec[0][1] = xq.y;
                    rec[0][2] = xq.z;
                    rec[0][3] = xq.w;
                }
            }
            gm = next_migration(g + 1u, end, a.every_k, a.per_neighbor);
            if (gm != ~0u) prepare(gm);
        }
        if (valid) {
            if (!drawn) birth_draws<N>(w, p, a.rk, g, island, seg_lane);
            reproduce<N, 2, TS, MODEL, 0, 1>(rec, w, p, a.rk, island, seg_lane, mask, g, 0,
                                             gen_mask_at(p, it));
        }
    }
    if (valid && !aborted) {
#pragma unroll
        for (int ag = 0; ag < A; ++ag)
            p.dst[static_cast<size_t>(island) * N + seg_lane + 32u * ag] =
                make_uint4(rec[ag][0], rec[ag][1], rec[ag][2], rec[ag][3]);
    }
}

// One island per warp (32 and 64 agents), no block barrier: on a migration generation g the
// warp's lanes 0..3 compute, for direction d, the neighbour R = nb(I, d)'s own slot-(d^1)
// birth draw (the member e_d it takes from I), and the lane holding member e_d pushes it into
// R's mailbox for direction d^1 (one 128-bit atomic exchange); while those writes reach L2
// the warp computes g's birth draws, the landing slots (the partial Fisher-Yates draw of the
// synchronous mode, from the island's own slot-0..3 draws) and the next migration
// generation's emigrant draws, none of which needs an arrival; lanes 0..3 read the island's
// four mailboxes once right after the pushes (that read travels while the warp draws, so an
// island whose neighbours got to g first has their records without a further round trip),
// then poll until each holds the record of generation g, and every lane takes the arrival
// meant for its slot by shuffles.  Warps never wait for one another inside a
// block; each poll is bounded as in resident_kernel, and a warp that sees the abort word
// leaves.
template <int N, int TS, int MODEL, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 8)
resident_warp_kernel(const ResidentArgs a)
{
    constexpr int A = Shape<N>::A, LW = 4;
    static_assert(N >= 32, "one island per warp");
    const RunParams &p = a.r;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t island = blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (island >= p.n_islands) return;  // whole warps
    const uint32_t end = p.g0 + p.n_gens;
    const uint32_t d = lane & 3u;
    const bool dir_lane = lane < 4u;

    // torus neighbour of this island in direction d (lanes 0..3)
    uint32_t nb = island;
    if (dir_lane) {
        const uint32_t y = div_cols(island, p.cols_m, p.cols_l), x = island - y * p.cols;
        const uint32_t yn = d == 0u ? (y == 0u ? p.rows - 1u : y - 1u)
                          : d == 1u ? (y + 1u == p.rows ? 0u : y + 1u) : y;
        const uint32_t xn = d == 2u ? (x + 1u == p.cols ? 0u : x + 1u)
                          : d == 3u ? (x == 0u ? p.cols - 1u : x - 1u) : x;
        nb = yn * p.cols + xn;
    }

    uint32_t rec[A][LW];
#pragma unroll
    for (int ag = 0; ag < A; ++ag) {
        const uint4 v = __ldg(&p.src[static_cast<size_t>(island) * N + lane + 32u * ag]);
        rec[ag][0] = v.x;
        rec[ag][1] = v.y;
        rec[ag][2] = v.z;
        rec[ag][3] = v.w;
    }
    // the member the neighbour in direction d draws from this island at migration generation
    // gm (lanes 0..3; every lane computes it, so the draw is not a divergent branch and can
    // overlap other work): it depends on no state, so it is drawn a migration ahead
    auto emigrant = [&](uint32_t gm) {
        const uint32_t un = philox_rk(gm, nb, (d ^ 1u) | (kBirth << 16), p.run_id, a.rk).w;
        return (((un >> 8) & 0xFFu) * N) >> 8;
    };
    uint32_t nd[4];
#pragma unroll
    for (int dd = 0; dd < 4; ++dd) nd[dd] = __shfl_sync(0xffffffffu, nb, dd);
    uint32_t gm = next_migration(p.g0, end, a.every_k, a.per_neighbor);
    uint32_t e = emigrant(gm);
    bool aborted = false;
    for (uint32_t it = 0; it < p.n_gens; ++it) {
        const uint32_t g = p.g0 + it;
        const uint2 dm = gen_mask_at(p, it);  // the generation's deposit masks, read up front
        uint4 w[A];
        if (g == gm) {
            uint4 *box = a.mail + static_cast<size_t>((g / a.every_k) & 1u) * p.n_islands * 4u;
            // sends: lane holding the member e_d pushes it to the neighbour in direction d
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) {
                const uint32_t ed = __shfl_sync(0xffffffffu, e, dd);
#pragma unroll
                for (int ag = 0; ag < A; ++ag) {
                    if (lane + 32u * ag == ed && island != a.drop_island &&
                        in_bounds(nd[dd] < p.n_islands, p.status))
                        write128(box + static_cast<size_t>(nd[dd]) * 4u + (static_cast<uint32_t>(dd) ^ 1u),
                                 make_uint4(rec[ag][0], rec[ag][1], rec[ag][2], rec[ag][3]));
                }
            }
            // an early read of the island's own mailboxes: an island that reaches g after its
            // neighbours (the one that sets the pace) usually finds their records already there,
            // and this read returns while the warp draws instead of after
            uint4 *mine = box + static_cast<size_t>(island) * 4u + d;
            uint4 early = make_uint4(0u, 0u, 0u, 0u);
            if (dir_lane) early = read128(mine);
            // while the neighbours' writes travel: the next migration's emigrant draws, this
            // generation's birth draws and the landing slots, none of which needs an arrival
            const uint32_t gm_next = next_migration(g + 1u, end, a.every_k, a.per_neighbor);
            const uint32_t e_next = emigrant(gm_next);
            birth_draws<N>(w, p, a.rk, g, island, lane);
            // landing slots: partial Fisher-Yates over [0, N) in direction order from slot d's
            // own draw (word 3 of lane d's first birth draw), the same on every lane
            const uint32_t u = __shfl_sync(0xffffffffu, w[0].w, static_cast<int>(d));
            const uint32_t r_own = d + (((u >> 16) * static_cast<uint32_t>(N - d)) >> 16);
            uint32_t rr[4];
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) rr[dd] = __shfl_sync(0xffffffffu, r_own, dd);
            uint32_t v[4], slot[4];
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) {
                uint32_t vd = dd, vr = rr[dd];
#pragma unroll
                for (int e2 = 0; e2 < dd; ++e2) {
                    if (rr[e2] == static_cast<uint32_t>(dd)) vd = v[e2];
                    if (rr[e2] == rr[dd]) vr = v[e2];
                }
                slot[dd] = vr;
                v[dd] = vd;
            }
            int from[A];
#pragma unroll
            for (int ag = 0; ag < A; ++ag) {
                const uint32_t mine = lane + 32u * ag;
                from[ag] = -1;
#pragma unroll
                for (int dd = 0; dd < 4; ++dd)
                    if (slot[dd] == mine) from[ag] = dd;
            }
            // receives: lanes 0..3 wait for the records of generation g
            uint4 imm = early;
            bool gave_up = false;
            if (dir_lane && imm.y != g) {
                const unsigned long long t0 = global_ns();
                for (uint32_t polls = 0;; ++polls) {
                    imm = read128(mine);  // the abort word beside it, as in resident_kernel
                    const uint32_t ab = ld_relaxed_u32(a.abort_word);
                    if (imm.y == g) break;
                    if (ab != 0u) {
                        gave_up = true;
                        break;
                    }
                    if (global_ns() - t0 > a.wait_ns) {
                        atomicCAS(p.status, 0, GA_ETIMEOUT);
                        atomicExch(a.abort_word, 1u);
                        gave_up = true;
                        break;
                    }
                    if (polls >= 8u) __nanosleep(64);
                }
            }
            if (__any_sync(0xffffffffu, gave_up)) {
                aborted = true;
                break;
            }
            const uint32_t im[4] = {imm.x, imm.y, imm.z, imm.w};
#pragma unroll
            for (int ag = 0; ag < A; ++ag) {
#pragma unroll
                for (int k = 0; k < LW; ++k) {
                    const uint32_t val = __shfl_sync(0xffffffffu, im[k], from[ag] < 0 ? 0 : from[ag]);
                    if (from[ag] >= 0) rec[ag][k] = val;
                }
            }
            gm = gm_next;
            e = e_next;
        } else {
            birth_draws<N>(w, p, a.rk, g, island, lane);
        }
        reproduce<N, 2, TS, MODEL, 0, 1>(rec, w, p, a.rk, island, lane, 0xffffffffu, g, 0, dm);
    }
    if (!aborted) {
#pragma unroll
        for (int ag = 0; ag < A; ++ag)
            p.dst[static_cast<size_t>(island) * N + lane + 32u * ag] =
                make_uint4(rec[ag][0], rec[ag][1], rec[ag][2], rec[ag][3]);
    }
}

using ResidentKernel = void (*)(ResidentArgs);

template <int N, int WARPS>
ResidentKernel pick_model(uint32_t model, uint32_t tsize)
{
    if (model == GA_MODEL_FITNESS) {  // the float-fitness model: islands of 16 to 64 agents
        if constexpr (N >= 16)
            return tsize == 5u ? resident_kernel<N, 5, 1, WARPS> : resident_kernel<N, 0, 1, WARPS>;
        return nullptr;
    }
    return tsize == 5u ? resident_kernel<N, 5, 0, WARPS> : resident_kernel<N, 0, 0, WARPS>;
}

// Island warps per block: 4 (small grids spread over more SMs).
constexpr int kResidentWarps = 4;

// Islands of 32 and 64 agents: one island per warp, no bookkeeping warp and no block barrier
// (2.10 against 2.49 us per generation for the block kernel on the 32x32 torus of 32-agent
// islands); smaller islands share a warp and keep the block kernel.
template <int N>
ResidentKernel pick_warp_model(uint32_t model, uint32_t tsize)
{
    if (model == GA_MODEL_FITNESS)
        return tsize == 5u ? resident_warp_kernel<N, 5, 1, kResidentWarps>
                           : resident_warp_kernel<N, 0, 1, kResidentWarps>;
    return tsize == 5u ? resident_warp_kernel<N, 5, 0, kResidentWarps>
                       : resident_warp_kernel<N, 0, 0, kResidentWarps>;
}

ResidentKernel pick_resident(uint32_t island_size, uint32_t model, uint32_t tsize, uint32_t &threads,
                             uint32_t &islands_per_block)
{
    switch (island_size) {
    case 8:
        threads = ResidentShape<8, kResidentWarps>::THREADS;
        islands_per_block = ResidentShape<8, kResidentWarps>::BI;
        return pick_model<8, kResidentWarps>(model, tsize);
    case 16:
        threads = ResidentShape<16, kResidentWarps>::THREADS;
        islands_per_block = ResidentShape<16, kResidentWarps>::BI;
        return pick_model<16, kResidentWarps>(model, tsize);
    case 32:
        threads = kResidentWarps * 32;
        islands_per_block = kResidentWarps;
        return pick_warp_model<32>(model, tsize);
    case 64:
        threads = kResidentWarps * 32;
        islands_per_block = kResidentWarps;
        return pick_warp_model<64>(model, tsize);
    default:
        return nullptr;
    }
}

}  // namespace

size_t resident_state_bytes(uint32_t n_islands, uint32_t record_bytes)
{
    if (record_bytes != 16u || n_islands > kResidentMaxIslands) return 0;
    // abort word (256 bytes), then two parities of four 16-byte mailboxes per island
    return 256u + static_cast<size_t>(n_islands) * 4u * 2u * 16u;
}

bool resident_possible(const ga_run *run, uint32_t *blocks_out)
{
    if (!run->resident_state || run->cfg.mode != GA_SYNC || !run->counters_uniform) return false;
    uint32_t threads = 0, per_block = 0;
    const ResidentKernel k =
        pick_resident(run->cfg.island_size, run->cfg.model, run->cfg.tournament_size, threads, per_block);
    if (!k) return false;
    const uint32_t blocks = (run->n_islands + per_block - 1) / per_block;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, static_cast<int>(threads), 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (blocks > static_cast<uint32_t>(sms) * static_cast<uint32_t>(per_sm)) return false;
    if (blocks_out) *blocks_out = blocks;
    return true;
}

cudaError_t launch_resident(ga_run *run, const void *src, void *dst, uint32_t g0, uint32_t n_gens,
                            cudaStream_t stream)
{
    uint32_t threads = 0, per_block = 0;
    const ResidentKernel k =
        pick_resident(run->cfg.island_size, run->cfg.model, run->cfg.tournament_size, threads, per_block);
    if (!k) return cudaErrorInvalidValue;
    const uint32_t blocks = (run->n_islands + per_block - 1) / per_block;
    // empty mailboxes (all ones) and a clear abort word for this launch
    uint8_t *state = static_cast<uint8_t *>(run->resident_state);
    cudaError_t e = cudaMemsetAsync(state, 0, 256, stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(state + 256, 0xFF, static_cast<size_t>(run->n_islands) * 4u * 2u * 16u, stream);
    if (e != cudaSuccess) return e;
    ResidentArgs a;
    a.r = run_params(run, src, dst, g0, n_gens, false);
    a.rk = round_keys(Key{static_cast<uint32_t>(run->cfg.seed), static_cast<uint32_t>(run->cfg.seed >> 32)});
    a.mail = reinterpret_cast<uint4 *>(state + 256);
    a.abort_word = reinterpret_cast<uint32_t *>(state);
    a.wait_ns = static_cast<unsigned long long>(run->resident_wait_us) * 1000ull;
    a.every_k = run->every_k;
    a.per_neighbor = run->per_neighbor;
    a.drop_island = run->drop_island;
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k), dim3(blocks), dim3(threads),
                                    args, 0, stream);
    run->launches += 1;
    return e;
}

}  // namespace ga
