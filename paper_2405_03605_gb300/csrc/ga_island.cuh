// ga_island.cuh -- the fused island step shared by the single-run and batched kernels.
//
// One generation (Sec. 2 of the paper, in its order): migration (when due), evaluation
// (fitness = trait), tournament selection of every next-generation slot, copy and mutation
// of the child, and the hstrat deposit for the elapsed generation.
//
// Mapping: one island per warp for N >= 32 (N/32 agents per lane), 32/N islands per warp
// for N < 32 (one agent per lane, shuffles of width N).  A block owns WARPS warps of
// consecutive islands.  Each lane keeps its agents' records in registers; tournaments read
// candidate traits and copy the winner's record with __shfl_sync, so an island never leaves
// the register file between the launch's first load and last store.  A launch runs
// generations [g0, g0 + n) with migration only at g0: the population is read once from `src`
// and written once to `dst` per launch, and immigrants are read straight from the
// neighbours' records in `src` (the whole previous population doubles as the migration
// halo, so no separate halo buffer or grid barrier is needed and the result does not depend
// on launch order).
//
// Migration bookkeeping is lane-parallel across the block: one thread per (island,
// direction) pair recomputes that island's birth draw for slot d (the draw that carries the
// migration bits), derives the immigrant index and landing draw, finds the torus neighbour,
// loads the immigrant record and resolves the partial Fisher-Yates landing slot with its
// three sibling lanes; records and slots go through shared memory, so an island's warp only
// compares four slot numbers and reads at most one record per agent.
#pragma once

#include "ga_device.cuh"

namespace ga {

// Everything one launch needs to know about one run.
struct RunParams {
    const uint4 *__restrict__ src;          // records before generation g0
    uint4 *__restrict__ dst;                // records after generation g0 + n_gens - 1
    uint32_t rows, cols, n_islands;
    uint32_t cols_m, cols_l;                // island / cols as a multiply-shift (div_cols)
    uint32_t tsize;
    uint32_t theta_ben, theta_del;
    uint32_t policy, log2_sites, sites, bits;
    uint32_t run_id;
    uint32_t g0, n_gens, migrate;           // migration (if set) happens at g0 only
    const int32_t *__restrict__ gen_sites;  // curation site of generation g0 + i
    float effect_scale;                     // fitness model: mutation amount scale
    uint32_t gen_sites_left;                // entries of gen_sites from g0 on
    int *status;                            // the run's device status word
    // deposit masks of generation g0 + i (records with a 64-bit surface, S b <= 64): the bits of
    // surface words 0 and 1 that the generation's deposit overwrites, (0, 0) for none; the
    // differentia (low b bits of the draw) is spread over every b-bit field by one multiply
    const uint2 *__restrict__ gen_masks;
    uint32_t dif_mask, dif_rep;             // 2^b - 1 and the b-bit repetition pattern
};

// Curation site of generation g0 + it from the launch's site table (-1, no deposit, if a
// device-check build finds `it` past the table).
__device__ __forceinline__ int gen_site_at(const RunParams &p, uint32_t it)
{
    return in_bounds(it < p.gen_sites_left, p.status) ? __ldg(&p.gen_sites[it]) : -1;
}

// Deposit masks of generation g0 + it ((0, 0), no deposit, if a device-check build finds `it`
// past the table).
__device__ __forceinline__ uint2 gen_mask_at(const RunParams &p, uint32_t it)
{
    return in_bounds(it < p.gen_sites_left, p.status) ? __ldg(&p.gen_masks[it]) : make_uint2(0u, 0u);
}

// Candidate trait of slot `sel` of this lane's island.  For N <= 32 `sel` may carry extra
// high bits: a shuffle of width N reads lane sel mod N, which is exactly the drawn slot.
template <int N, int A, int SEG>
__device__ __forceinline__ int candidate_trait(unsigned mask, const int (&trait)[A], uint32_t sel)
{
    if constexpr (N <= 32) {
        return __shfl_sync(mask, trait[0], static_cast<int>(sel), SEG);
    } else {
        int t = 0;
#pragma unroll
        for (int q = 0; q < A; ++q) {
            const int x = __shfl_sync(mask, trait[q], static_cast<int>(sel & 31u));
            if ((sel >> 5) == static_cast<uint32_t>(q)) t = x;
        }
        return t;
    }
}

template <int N>
struct Shape {
    static constexpr int A = N >= 32 ? N / 32 : 1;   // agents per lane
    static constexpr int P = N >= 32 ? 1 : 32 / N;   // islands per warp
    static constexpr int SEG = N >= 32 ? 32 : N;     // lanes per island
    static constexpr int LOGN = N >= 128 ? 7 : N >= 64 ? 6 : N >= 32 ? 5 : N >= 16 ? 4 : N >= 8 ? 3 : 2;
};

// Birth draws of this lane's child slots in generation g: (B0, B1) tournament bytes, B2
// mutation, B3 differentia (low bits) and, for slots 0..3, the migration bits.
template <int N>
__device__ __forceinline__ void birth_draws(uint4 (&w)[Shape<N>::A], const RunParams &p,
                                            const RoundKeys &rk, uint32_t g, uint32_t island,
                                            uint32_t seg_lane)
{
#pragma unroll
    for (int ag = 0; ag < Shape<N>::A; ++ag)
        w[ag] = philox_rk(g, island, (seg_lane + 32u * ag) | (kBirth << 16), p.run_id, rk);
}

// Evaluation, tournament, copy, mutation and hstrat deposit of one generation, in place.
// Closed-form curation site, called only for agents whose counter differs from the
// generation (never in synchronous runs); kept out of line so the common path stays a load.
static __device__ __noinline__ int curation_site_of(uint32_t policy, uint32_t log2_sites, uint32_t sites,
                                            uint32_t T)
{
    return curation_site(policy, log2_sites, sites, T);
}

// g: the generation; gen_site: its curation site, valid for agents whose counter is g -- any
// other counter takes the closed form.  CF = 0 compiles the closed form out: only for
// launches in which every counter equals the generation (synchronous runs whose counters
// were never loaded mixed), where it would never be taken.
// MODEL 0: int32 trait, +1 / -1; MODEL 1: float fitness, -/+ effect_scale * |normal|.
// DM = 1 (64-bit surfaces, every counter equal to g): the deposit takes the generation's
// precomputed masks `dmask` instead of the site: the differentia spread over every b-bit
// field, kept where the mask is set -- the same bits as writing it at site * b.
template <int N, int SW, int TS, int MODEL, int CF = 1, int DM = 0>
__device__ __forceinline__ void reproduce(uint32_t (&rec)[Shape<N>::A][2 + SW],
                                          const uint4 (&w)[Shape<N>::A], const RunParams &p,
                                          const RoundKeys &rk, uint32_t island, uint32_t seg_lane,
                                          unsigned mask, uint32_t g, int gen_site,
                                          uint2 dmask = make_uint2(0u, 0u))
{
    constexpr int A = Shape<N>::A, SEG = Shape<N>::SEG, LOGN = Shape<N>::LOGN;
    constexpr int LW = 2 + SW;
    // tournament: best of n draws with replacement, earliest wins ties; draw i's slot is byte
    // (i mod 4) of B0 / B1 scaled to N, i.e. that byte's top log2 N bits
    int trait[A];
#pragma unroll
    for (int ag = 0; ag < A; ++ag) trait[ag] = static_cast<int>(rec[ag][0]);
    uint32_t win[A];
#pragma unroll
    for (int ag = 0; ag < A; ++ag) {
        uint32_t best = 0;
        int best_trait = 0;
        if constexpr (TS > 0) {
#pragma unroll
            for (int i = 0; i < TS; ++i) {
                const uint32_t word = i < 4 ? w[ag].x : w[ag].y;
                uint32_t sel = word >> (8 * (i & 3) + 8 - LOGN);
                if constexpr (N > 32) sel &= N - 1u;
                const int t = candidate_trait<N, A, SEG>(mask, trait, sel);
                bool better;
                if constexpr (MODEL == 1) better = __int_as_float(t) > __int_as_float(best_trait);
                else better = t > best_trait;
                if (i == 0 || better) {
                    best = sel;
                    best_trait = t;
                }
            }
        } else {
            // size n from the run (1..8): draws n-1 down to 0, each replacing the best when at
            // least as good, from a start below every trait (INT_MIN; -inf for the float model,
            // whose fitness is never NaN) -- the earliest maximal draw is kept, as above, and the
            // switch enters the unrolled draws once instead of testing n at every draw
            best_trait = MODEL == 1 ? static_cast<int>(0xFF800000u) : static_cast<int>(0x80000000u);
            auto draw = [&](const int i) {
                const uint32_t word = i < 4 ? w[ag].x : w[ag].y;
                uint32_t sel = word >> (8 * (i & 3) + 8 - LOGN);
                if constexpr (N > 32) sel &= N - 1u;
                const int t = candidate_trait<N, A, SEG>(mask, trait, sel);
                bool better;
                if constexpr (MODEL == 1) better = __int_as_float(t) >= __int_as_float(best_trait);
                else better = t >= best_trait;
                if (better) {
                    best = sel;
                    best_trait = t;
                }
            };
            switch (p.tsize) {
            case 8: draw(7); [[fallthrough]];
            case 7: draw(6); [[fallthrough]];
            case 6: draw(5); [[fallthrough]];
            case 5: draw(4); [[fallthrough]];
            case 4: draw(3); [[fallthrough]];
            case 3: draw(2); [[fallthrough]];
            case 2: draw(1); [[fallthrough]];
            default: draw(0);
            }
        }
        win[ag] = best;
    }

    // copy the winner's record
    uint32_t child[A][LW];
#pragma unroll
    for (int ag = 0; ag < A; ++ag) {
#pragma unroll
        for (int k = 0; k < LW; ++k) {
            if constexpr (N <= 32) {
                child[ag][k] = __shfl_sync(mask, rec[0][k], static_cast<int>(win[ag]), SEG);
            } else {
                uint32_t val = 0;
#pragma unroll
                for (int q = 0; q < A; ++q) {
                    const uint32_t xv = __shfl_sync(mask, rec[q][k], static_cast<int>(win[ag] & 31u));
                    if ((win[ag] >> 5) == static_cast<uint32_t>(q)) val = xv;
                }
                child[ag][k] = val;
            }
        }
    }

    // mutation and hstrat deposit
#pragma unroll
    for (int ag = 0; ag < A; ++ag) {
        const uint32_t xm = w[ag].z;
        if constexpr (MODEL == 1) {
            const bool del = xm < p.theta_del;
            const bool ben = !del && xm - p.theta_del < p.theta_ben;
            if (del || ben) {
                const uint4 mw = philox_rk(g, island, (seg_lane + 32u * ag) | (kMutate << 16),
                                           p.run_id, rk);
                const float amount = __fmul_rn(p.effect_scale, fabsf(normal_rn(mw.x, mw.y)));
                const float f = __uint_as_float(child[ag][0]);
                child[ag][0] = __float_as_uint(del ? __fsub_rn(f, amount) : __fadd_rn(f, amount));
            }
        } else {
            uint32_t t = child[ag][0];
            if (xm < p.theta_del) t -= 1u;
            else if (xm - p.theta_del < p.theta_ben) t += 1u;
            child[ag][0] = t;
        }

        const uint32_t c = child[ag][1];
        int site = gen_site;
        if constexpr (CF != 0) {
            if (c != g) site = curation_site_of(p.policy, p.log2_sites, p.sites, c);
        }
        if constexpr (DM != 0) {
            static_assert(SW == 2 && CF == 0, "mask deposits: 64-bit surfaces, uniform counters");
            const uint32_t rep = (w[ag].w & p.dif_mask) * p.dif_rep;
            child[ag][2] = (child[ag][2] & ~dmask.x) | (rep & dmask.x);
            child[ag][3] = (child[ag][3] & ~dmask.y) | (rep & dmask.y);
        } else if (site >= 0 && in_bounds(static_cast<uint32_t>(site) < p.sites &&
                                              site * p.bits < 32u * SW,
                                          p.status)) {
            const uint32_t pos = static_cast<uint32_t>(site) * p.bits;
            const uint32_t wi = pos >> 5, sh = pos & 31u;
            const uint32_t m = ((1u << p.bits) - 1u) << sh;
            const uint32_t val = (w[ag].w << sh) & m;
#pragma unroll
            for (int k = 0; k < SW; ++k)
                if (static_cast<uint32_t>(k) == wi) child[ag][2 + k] = (child[ag][2 + k] & ~m) | val;
        }
        child[ag][1] = c + 1u;
#pragma unroll
        for (int k = 0; k < LW; ++k) rec[ag][k] = child[ag][k];
    }
}

// One block's work: `unit` is the block's index within the run (islands
// [unit * BI, unit * BI + BI)).  N: island size; SW: surface words carried per record (the
// record is RW words); TS: the tournament size when fixed at compile time (0: read from the
// run); WARPS: warps per block; MODEL: genome model (0 trait, 1 float fitness); CF: closed-form
// curation available (see reproduce).
template <int N, int SW, int TS, int WARPS, int MODEL = 0, int CF = 1>
__device__ __forceinline__ void step_block(const RunParams &p, const RoundKeys &rk, uint32_t unit)
{
    constexpr int A = Shape<N>::A, P = Shape<N>::P, SEG = Shape<N>::SEG;
    constexpr int LW = 2 + SW;                   // live words: trait, counter, surface
    constexpr int RW = (LW + 3) / 4 * 4;         // record words
    constexpr int Q = RW / 4;                    // 128-bit words per record
    constexpr int BI = WARPS * P;           // islands per block
    constexpr int ML = BI * 4;                   // migration lanes: (island, direction)

    // Islands of at most 32 agents: each immigrant is written straight to its landing slot
    // (s_in, indexed by island and slot) and a per-island mask marks the four slots that
    // receive one, so an island lane tests one bit.  Larger islands: records and landing slots
    // by (island, direction), each lane comparing its slot with the four.
    constexpr bool kSlotTable = N <= 32;
    __shared__ uint4 s_imm[kSlotTable ? 1 : ML][Q];                // by (island, direction)
    __shared__ __align__(16) uint32_t s_slot[kSlotTable ? 1 : ML]; // landing slot of each
    __shared__ uint4 s_in[kSlotTable ? BI * N : 1][Q];             // by (island, slot)
    __shared__ uint32_t s_hit[kSlotTable ? BI : 1];                // bit s: slot s receives

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t seg_lane = lane % SEG;
    const uint32_t local = (threadIdx.x >> 5) * P + lane / SEG;
    const uint32_t island0 = unit * BI;
    const uint32_t island = island0 + local;
    const bool valid = island < p.n_islands;
    const unsigned mask = __ballot_sync(0xffffffffu, valid);

    // Migration bookkeeping, part 1 (threads < ML): the immigrant loads are issued first, so
    // their latency overlaps everything up to the block barrier.  ML is a multiple of 4 but
    // not always of 32 (4-warp blocks of N >= 32 islands use 16 lanes), so the shuffles among
    // an island's four bookkeeping lanes use the ballot of exactly those lanes.
    const bool mig_lane = p.migrate && threadIdx.x < ML;
    const unsigned mig_mask = __ballot_sync(0xffffffffu, mig_lane);
    const uint32_t md = threadIdx.x & 3u;  // direction of this bookkeeping lane
    uint32_t r = md;                       // its landing draw
    uint4 imm[Q];
    if (mig_lane) {
        const uint32_t isl = island0 + (threadIdx.x >> 2);
        if (isl < p.n_islands) {
            // birth draw of slot d: bits 8..15 pick the immigrant, bits 16..31 its landing
            const uint32_t u = philox_rk(p.g0, isl, md | (kBirth << 16), p.run_id, rk).w;
            r = md + (((u >> 16) * static_cast<uint32_t>(N - md)) >> 16);
            const uint32_t e = (((u >> 8) & 0xFFu) * N) >> 8;
            const uint32_t y = div_cols(isl, p.cols_m, p.cols_l), x = isl - y * p.cols;
            const uint32_t yn = md == 0u ? (y == 0u ? p.rows - 1u : y - 1u)
                              : md == 1u ? (y + 1u == p.rows ? 0u : y + 1u) : y;
            const uint32_t xn = md == 2u ? (x + 1u == p.cols ? 0u : x + 1u)
                              : md == 3u ? (x == 0u ? p.cols - 1u : x - 1u) : x;
            const uint32_t nb = yn * p.cols + xn;
            const uint4 *srec = p.src + (static_cast<size_t>(nb) * N + e) * Q;
            if (in_bounds(nb < p.n_islands && e < static_cast<uint32_t>(N), p.status)) {
#pragma unroll
                for (int q = 0; q < Q; ++q) imm[q] = __ldg(&srec[q]);
            } else {
#pragma unroll
                for (int q = 0; q < Q; ++q) imm[q] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
    }

    // this lane's records and its birth draws of generation g0
    uint32_t rec[A][LW];
    uint4 w[A];
    if (valid) {
#pragma unroll
        for (int ag = 0; ag < A; ++ag) {
            const size_t agent = static_cast<size_t>(island) * N + seg_lane + 32u * ag;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const uint4 v = __ldg(&p.src[agent * Q + q]);
                const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (4 * q + e < LW) rec[ag][4 * q + e] = w4[e];
            }
        }
        birth_draws<N>(w, p, rk, p.g0, island, seg_lane);
    }

    // Migration bookkeeping, part 2: the partial Fisher-Yates landing slots (over [0, N) in
    // direction order, among the island's four lanes: entry e records "position r[e] now
    // holds value v[e]", later entries winning), then records and slots to shared memory.
    if (p.migrate) {
        if (mig_lane) {
            uint32_t rr[4];
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) rr[dd] = __shfl_sync(mig_mask, r, dd, 4);
            uint32_t v[4], slot = 0;
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) {
                uint32_t vd = dd, vr = rr[dd];
#pragma unroll
                for (int e = 0; e < dd; ++e) {
                    if (rr[e] == static_cast<uint32_t>(dd)) vd = v[e];
                    if (rr[e] == rr[dd]) vr = v[e];
                }
                if (static_cast<uint32_t>(dd) == md) slot = vr;
                v[dd] = vd;
            }
            if constexpr (kSlotTable) {
                const uint32_t li = threadIdx.x >> 2;  // the block's island of this lane
                uint32_t bit = 1u << slot;
                bit |= __shfl_xor_sync(mig_mask, bit, 1, 4);
                bit |= __shfl_xor_sync(mig_mask, bit, 2, 4);
                if (island0 + li < p.n_islands &&
                    in_bounds(li * N + slot < static_cast<uint32_t>(BI * N), p.status)) {
#pragma unroll
                    for (int q = 0; q < Q; ++q) s_in[li * N + slot][q] = imm[q];
                }
                if (md == 0u) s_hit[li] = bit;
            } else {
                s_slot[threadIdx.x] = slot;
                if (island0 + (threadIdx.x >> 2) < p.n_islands) {
#pragma unroll
                    for (int q = 0; q < Q; ++q) s_imm[threadIdx.x][q] = imm[q];
                }
            }
        }
        __syncthreads();
    }
    if (!valid) return;

    if (p.migrate && kSlotTable) {
        // the four immigrants land in their slots: every lane reads its slot's entry, the four
        // receivers keep it
        const bool hit = ((s_hit[local] >> seg_lane) & 1u) != 0u;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const uint4 xq = s_in[local * N + seg_lane][q];
            const uint32_t w4[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (4 * q + k < LW) rec[0][4 * q + k] = hit ? w4[k] : rec[0][4 * q + k];
        }
    } else if (p.migrate) {
        // the four immigrants land in their slots
        const uint4 sl = *reinterpret_cast<const uint4 *>(&s_slot[4 * local]);
#pragma unroll
        for (int ag = 0; ag < A; ++ag) {
            const uint32_t mine = seg_lane + 32u * ag;
            const int from = sl.x == mine ? 0 : sl.y == mine ? 1 : sl.z == mine ? 2
                           : sl.w == mine ? 3 : -1;
            {  // branch-free: every lane reads a slot, the four receivers keep it
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const uint4 xq = s_imm[4 * local + (from < 0 ? 0 : from)][q];
                    const uint32_t w4[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (4 * q + k < LW) rec[ag][4 * q + k] = from >= 0 ? w4[k] : rec[ag][4 * q + k];
                }
            }
        }
    }
    reproduce<N, SW, TS, MODEL, CF>(rec, w, p, rk, island, seg_lane, mask, p.g0, gen_site_at(p, 0u));

    // generations g0 + 1 .. g0 + n - 1: no migration, the island stays in registers
    for (uint32_t it = 1; it < p.n_gens; ++it) {
        birth_draws<N>(w, p, rk, p.g0 + it, island, seg_lane);
        reproduce<N, SW, TS, MODEL, CF>(rec, w, p, rk, island, seg_lane, mask, p.g0 + it,
                                        gen_site_at(p, it));
    }

#pragma unroll
    for (int ag = 0; ag < A; ++ag) {
        const size_t agent = static_cast<size_t>(island) * N + seg_lane + 32u * ag;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            uint32_t w4[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) w4[e] = (4 * q + e < LW) ? rec[ag][4 * q + e] : 0u;
            p.dst[agent * Q + q] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Multi-unit blocks for islands of 16, 32 or 64 agents with 16-byte records whose counters
// all equal the generation (every synchronous run unless a population with other counters
// was loaded).  A block of 8 warps runs U units of 8 * P islands in turn (P = 32 / N islands
// per warp below 32 agents, one island per warp otherwise); warp w runs its share of every
// unit.  Each warp's records come into shared memory by asynchronous copies (cp.async): the
// next unit's while the current one is computed, so a warp never waits for a record load
// except the block's first.  The migration bookkeeping of all U units is done once, at the
// start, spread over the block's threads (unit u: threads [u * 4BI, (u + 1) * 4BI), one per
// (island, direction), as in step_block), and its immigrant copies go straight into shared
// memory.  An island's lanes then find their landing direction in a per-island table of N
// bytes (0xFF: no immigrant) and take the immigrant record from shared memory.  Deposits use
// the generation's precomputed masks.  The only block barrier is the one after the
// bookkeeping.
// ---------------------------------------------------------------------------------------

// 16-byte asynchronous global -> shared copy (bypassing L1), and its group operations.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" :: "r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" :: "n"(PENDING) : "memory"); }

// Units per block: as many as the block's 256 threads can do the bookkeeping for, at most 8.
template <int N>
constexpr int units_per_block()
{
    return (256 / (4 * 8 * Shape<N>::P)) < 8 ? (256 / (4 * 8 * Shape<N>::P)) : 8;
}

template <int N, int TS, int U, int MODEL = 0, bool UNROLL = true>
__device__ __forceinline__ void step_units(const RunParams &p, const RoundKeys &rk, uint32_t blk)
{
    constexpr int SW = 2, LW = 4, WARPS = 8;
    constexpr int A = Shape<N>::A, P = Shape<N>::P, SEG = Shape<N>::SEG;
    constexpr int BI = WARPS * P;  // islands per unit
    constexpr int ML = 4 * BI;     // bookkeeping lanes per unit (a multiple of 32)
    constexpr int RPW = 32 * A;    // records per warp and unit
    static_assert(N >= 16 && N <= 64, "islands of 16 to 64 agents");
    static_assert(U >= 1 && U * ML <= WARPS * 32, "the block's threads cover every unit's bookkeeping");
    __shared__ uint4 s_rec[WARPS][2][RPW];                   // per warp: current and next unit's records
    __shared__ uint4 s_imm[U][ML];                           // immigrants by (unit, island, direction)
    __shared__ __align__(16) uint8_t s_dir[U][BI][N];        // landing direction of each slot

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t seg_lane = lane % SEG;
    const uint32_t local = warp * P + lane / SEG;  // this lane's island within a unit
    const uint32_t island0 = blk * (U * BI);       // first island of the block's first unit

    // the first unit's records: the warp's P islands are 32 A consecutive records
    {
        const uint32_t island = island0 + local;
        if (island < p.n_islands) {
            const uint4 *src = p.src + static_cast<size_t>(island0 + warp * P) * N + lane;
#pragma unroll
            for (int ag = 0; ag < A; ++ag) cp_async16(&s_rec[warp][0][lane + 32u * ag], src + 32u * ag);
        }
        cp_async_commit();
    }

    // migration bookkeeping of unit t / ML: lane (island i, direction d); the birth draw of
    // slot d carries the immigrant index (bits 8..15) and the landing draw (bits 16..31)
    if (p.migrate && threadIdx.x < static_cast<uint32_t>(U * ML)) {
        const uint32_t u = threadIdx.x / ML, idx = threadIdx.x % ML;
        const uint32_t li = idx >> 2, md = idx & 3u;
        // the island's own four lanes clear its table (N bytes)
        uint32_t *dirw = reinterpret_cast<uint32_t *>(&s_dir[u][li][0]);
#pragma unroll
        for (uint32_t k = md; k < static_cast<uint32_t>(N / 4); k += 4u) dirw[k] = 0xFFFFFFFFu;
        const uint32_t isl = island0 + u * BI + li;
        const bool ok = isl < p.n_islands;
        uint32_t r = md;
        if (ok) {
            const uint32_t w3 = philox_rk(p.g0, isl, md | (kBirth << 16), p.run_id, rk).w;
            r = md + (((w3 >> 16) * static_cast<uint32_t>(N - md)) >> 16);
            const uint32_t e = (((w3 >> 8) & 0xFFu) * N) >> 8;
            const uint32_t y = div_cols(isl, p.cols_m, p.cols_l), x = isl - y * p.cols;
            const uint32_t yn = md == 0u ? (y == 0u ? p.rows - 1u : y - 1u)
                              : md == 1u ? (y + 1u == p.rows ? 0u : y + 1u) : y;
            const uint32_t xn = md == 2u ? (x + 1u == p.cols ? 0u : x + 1u)
                              : md == 3u ? (x == 0u ? p.cols - 1u : x - 1u) : x;
            const uint32_t nb = yn * p.cols + xn;
            if (in_bounds(nb < p.n_islands, p.status))
                cp_async16(&s_imm[u][idx], &p.src[static_cast<size_t>(nb) * N + e]);
        }
        cp_async_commit();
        // partial Fisher-Yates over [0, N) in direction order among the island's four lanes
        uint32_t rr[4];
#pragma unroll
        for (int dd = 0; dd < 4; ++dd) rr[dd] = __shfl_sync(0xffffffffu, r, dd, 4);
        uint32_t v[4], slot = 0;
#pragma unroll
        for (int dd = 0; dd < 4; ++dd) {
            uint32_t vd = dd, vr = rr[dd];
#pragma unroll
            for (int e = 0; e < dd; ++e) {
                if (rr[e] == static_cast<uint32_t>(dd)) vd = v[e];
                if (rr[e] == rr[dd]) vr = v[e];
            }
            if (static_cast<uint32_t>(dd) == md) slot = vr;
            v[dd] = vd;
        }
        __syncwarp();  // the table is cleared before any entry is set (same warp)
        if (ok && in_bounds(slot < static_cast<uint32_t>(N), p.status))
            s_dir[u][li][slot] = static_cast<uint8_t>(md);
        cp_async_wait<0>();
    }
    __syncthreads();

    const uint2 dmask = gen_mask_at(p, 0u);
    // UNROLL: fully unrolled over the block's units, so the double-buffer index, the
    // shared-memory offsets of each unit and the loop control become constants (94.2 against
    // 101.7 us per generation of 16.8M agents with the loop kept rolled; 3-10% on the other
    // island and tournament sizes, results identical)
#pragma unroll (UNROLL ? U : 1)
    for (uint32_t un = 0; un < static_cast<uint32_t>(U); ++un) {
        const uint32_t first = island0 + un * BI + warp * P;  // the warp's first island
        if (first >= p.n_islands) break;  // uniform in the warp; later units lie further on
        const uint32_t island = first + lane / SEG;
        bool valid = true;  // one island per warp: the whole warp, checked above
        unsigned mask = 0xffffffffu;
        if constexpr (P > 1) {
            valid = island < p.n_islands;
            mask = __ballot_sync(0xffffffffu, valid);
        }
        if (un + 1u < static_cast<uint32_t>(U) && island + BI < p.n_islands) {
            const uint4 *src = p.src + static_cast<size_t>(first + BI) * N + lane;
#pragma unroll
            for (int ag = 0; ag < A; ++ag)
                cp_async16(&s_rec[warp][(un + 1u) & 1u][lane + 32u * ag], src + 32u * ag);
        }
        cp_async_commit();
        if constexpr (P > 1) {
            if (!valid) break;  // only lanes of a missing last island; later units are past too
        }
        uint4 w[A];
        birth_draws<N>(w, p, rk, p.g0, island, seg_lane);
        cp_async_wait<1>();  // this unit's records have landed
        uint32_t rec[A][LW];
#pragma unroll
        for (int ag = 0; ag < A; ++ag) {
            uint4 v = s_rec[warp][un & 1u][lane + 32u * ag];
            if (p.migrate) {
                const uint32_t dd = s_dir[un][local][seg_lane + 32u * ag];
                const uint4 x = s_imm[un][local * 4u + (dd & 3u)];
                if (dd < 4u) v = x;
            }
            rec[ag][0] = v.x;
            rec[ag][1] = v.y;
            rec[ag][2] = v.z;
            rec[ag][3] = v.w;
        }
        reproduce<N, SW, TS, MODEL, 0, 1>(rec, w, p, rk, island, seg_lane, mask, p.g0, 0, dmask);
        for (uint32_t it = 1; it < p.n_gens; ++it) {
            birth_draws<N>(w, p, rk, p.g0 + it, island, seg_lane);
            reproduce<N, SW, TS, MODEL, 0, 1>(rec, w, p, rk, island, seg_lane, mask, p.g0 + it, 0,
                                              gen_mask_at(p, it));
        }
        uint4 *dst = p.dst + static_cast<size_t>(first) * N + lane;
#pragma unroll
        for (int ag = 0; ag < A; ++ag)
            dst[32u * ag] = make_uint4(rec[ag][0], rec[ag][1], rec[ag][2], rec[ag][3]);
    }
}

}  // namespace ga
