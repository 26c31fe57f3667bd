// ga_async.cu -- the asynchronous island step: migration through one-genome send buffers.
//
// This follows the wafer-scale loop of the paper (Sec. 2): each island owns one send buffer
// per cardinal direction; on each migration generation it copies in the genomes whose
// receive completed (each replacing a random member), then refills the send buffers whose
// send completed -- those whose genome the neighbour has taken -- with copies of randomly
// sampled members; then it evaluates, selects, mutates and deposits as usual.  Nothing ever
// waits: a buffer that is not ready is simply skipped, so islands exchange migrants at
// whatever pace the hardware runs them, and a migrant keeps the counter of its lineage
// (deposits then follow each agent's own counter, as in the synchronous kernels'
// closed-form branch).  The loop tests every flag before anything moves (Sec. 2), so a buffer
// that an island empties itself -- only possible where it is its own neighbour, on one-row
// or one-column tori -- tested full and is refilled a pass later.
//
// Counter 2^32 - 1 is reserved: the 16-byte buffers mark "empty" with an all-ones record.
// ga_load refuses such counters in the asynchronous modes, and a birth that would produce
// one records GA_ESTATE in the run's status word (the run is then invalid; such a genome is
// never put into a buffer).
//
// Two handoff protocols, both single producer / single consumer and wait-free:
//
//  * 16-byte records (the paper's 128-bit genome): the buffer is the record itself, all
//    ones when empty.  The neighbour takes with one 128-bit atomic exchange (leaving all
//    ones) and the owner refills with one 128-bit compare-and-swap against all ones, so a
//    record moves in a single atomic access and is never seen half-written.  The take for a
//    generation is issued right after the previous generation's buffer step and its result
//    is used a generation later, so its latency hides behind reproduction; the refill's
//    result is never needed, so nothing waits on it.
//
//  * 32- and 48-byte records: a flag word (0 empty, 1 full) beside the record, in the PTX
//    memory model at GPU scope.  The owner writes a genome only into an empty buffer, with
//    relaxed stores, and publishes it by a release store of 1 at the start of its next
//    generation (or the end of the launch), when the record stores have long completed; the
//    neighbour takes a genome only from a full buffer, with relaxed loads, and hands the
//    buffer back by a release store of 0.  Flag tests are relaxed loads issued right after
//    the previous generation's buffer step and followed, before the record is touched, by
//    an acq_rel fence that makes them acquires; a buffer whose publication is still due
//    counts as full.
//
// On tori with one row or one column an island is its own neighbour, so its own lanes sit
// on both sides of a buffer: there the takes are made at the start of the generation and the
// refills after them, between warp barriers, publication is immediate, and a buffer the
// island has just taken a genome out of is left empty for this pass.  On the sequential
// schedule (one island per launch) every variant gives the same result as the oracle's
// model: test, take and land, then refill what tested empty.
//
// Draws: the birth draws of the synchronous mode, keyed by the generation the island is
// running.  For direction d, word 3 of slot d's draw supplies bits 16..31 for the landing
// slot of the arrival from d (the partial Fisher-Yates draw of the synchronous mode, the
// swap made whether or not anything arrives) and bits 8..15 for the member sent towards d.
//
// Mapping (island_async_kernel): one island per warp for N >= 32, 32/N islands per warp
// below; island lanes 0..3 take from the neighbours (lane d: direction d), lanes 4..7 own the
// island's send buffers (lane 4 + d: towards d).  Every lane runs the window's generations
// back to back with its agents in registers, as in the synchronous kernels.  Launches of a
// single generation with 16-byte records use island_async_gen_kernel instead, whose block
// shares the takes and landing draws of its islands like the synchronous kernel's migration
// bookkeeping (described there).
#include "ga_device.cuh"
#include "ga_internal.h"
#include "ga_island.cuh"

namespace ga {

// Defined with the synchronous launchers.
RunParams run_params(const ga_run *run, const void *src, void *dst, uint32_t g0, uint32_t n_gens,
                     bool migrate);

namespace {

constexpr uint32_t kNeverSent = 0xFFFFFFFFu;  // counter value of the empty-buffer record

// A birth gave a counter of 2^32 - 1, the value reserved for empty buffers: the run is
// invalid from here on (GA_ESTATE, returned by the next ga_sync / ga_snapshot).
template <int A, int LW>
__device__ __forceinline__ void check_counters(const uint32_t (&rec)[A][LW], int *status)
{
#pragma unroll
    for (int ag = 0; ag < A; ++ag)
        if (rec[ag][1] == kNeverSent) atomicCAS(status, 0, -5);
}

// GPU-scope memory-model accesses to the send buffers (global memory, 16-byte aligned).
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ uint4 ld_relaxed_v4(const uint4 *p)
{
    uint4 v;
    asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_v4(uint4 *p, uint4 v)
{
    asm volatile("st.relaxed.gpu.global.v4.u32 [%0], {%1, %2, %3, %4};"
                 :: "l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long pack64(uint32_t lo, uint32_t hi)
{
    return static_cast<unsigned long long>(lo) | (static_cast<unsigned long long>(hi) << 32);
}

// 128-bit atomic exchange: the record at p is replaced by all ones and returned.
__device__ __forceinline__ uint4 take128(uint4 *p)
{
    unsigned long long lo, hi;
    const unsigned long long ones = ~0ull;
    asm volatile("{\n\t.reg .b128 nv, ov;\n\t"
                 "mov.b128 nv, {%2, %3};\n\t"
                 "atom.relaxed.gpu.global.exch.b128 ov, [%4], nv;\n\t"
                 "mov.b128 {%0, %1}, ov;\n\t}"
                 : "=l"(lo), "=l"(hi) : "l"(ones), "l"(ones), "l"(p) : "memory");
    return make_uint4(static_cast<uint32_t>(lo), static_cast<uint32_t>(lo >> 32),
                      static_cast<uint32_t>(hi), static_cast<uint32_t>(hi >> 32));
}

// 128-bit compare-and-swap: the record v is stored at p if p holds all ones (empty).  The
// outcome is not needed, so the caller never waits for it.
__device__ __forceinline__ void refill128(uint4 *p, const uint32_t (&v)[4])
{
    [[maybe_unused]] unsigned long long lo, hi;
    const unsigned long long ones = ~0ull;
    asm volatile("{\n\t.reg .b128 cv, nv, ov;\n\t"
                 "mov.b128 cv, {%2, %3};\n\t"
                 "mov.b128 nv, {%4, %5};\n\t"
                 "atom.relaxed.gpu.global.cas.b128 ov, [%6], cv, nv;\n\t"
                 "mov.b128 {%0, %1}, ov;\n\t}"
                 : "=l"(lo), "=l"(hi)
                 : "l"(ones), "l"(ones), "l"(pack64(v[0], v[1])), "l"(pack64(v[2], v[3])), "l"(p)
                 : "memory");
}

constexpr int kAsyncThreads = 256;
constexpr int kAsyncWarps = kAsyncThreads / 32;

struct AsyncArgs {
    RunParams r;
    RoundKeys rk;
    uint4 *mail;           // [island][4] send buffers (16-byte records: the record itself;
                           // otherwise 1 + Q uint4: flag word, record)
    uint32_t every_k;      // migration on generations g with g mod every_k == 0
    uint32_t phase0;       // g0 mod every_k
    uint32_t first, last;  // islands [first, last) run in this launch
};


// Send-buffer size in uint4 for a record of Q uint4.
__host__ __device__ constexpr int box_words(int Q) { return Q == 1 ? 1 : 1 + Q; }

// Resident blocks per SM asked of the compiler: the buffer steps are latency-bound, so
// occupancy pays; six blocks (40 registers) fit the 16-byte-record kernels of N <= 32
// without spilling, the others keep their registers.
template <int N, int SW>
constexpr int async_min_blocks() { return SW <= 2 && N <= 32 ? 6 : 1; }

// TS: the tournament size when fixed at compile time (0: read from the run).
template <int N, int SW, int TS, int MODEL>
__global__ void __launch_bounds__(kAsyncThreads, (async_min_blocks<N, SW>()))
island_async_kernel(const AsyncArgs a)
{
    constexpr int A = Shape<N>::A, P = Shape<N>::P, SEG = Shape<N>::SEG;
    constexpr int LW = 2 + SW;
    constexpr int RW = (LW + 3) / 4 * 4;
    constexpr int Q = RW / 4;
    constexpr bool kAtomic = Q == 1;  // the whole record in one 128-bit atomic
    constexpr int MB = box_words(Q);
    const RunParams &p = a.r;

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t seg_lane = lane % SEG;
    const uint32_t island =
        a.first + (blockIdx.x * blockDim.x + threadIdx.x) / 32u * P + lane / SEG;
    const bool valid = island < a.last;
    const unsigned mask = __ballot_sync(0xffffffffu, valid);
    if (!valid) return;

    uint32_t rec[A][LW];
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

    // lanes 0..3 take from the neighbour in direction d (0 north, 1 south, 2 east, 3 west),
    // out of its buffer towards this island (its direction d ^ 1); lanes 4..7 own this
    // island's buffer towards d = lane - 4
    const uint32_t d = seg_lane & 3u;
    const bool taker = seg_lane < 4u;
    const bool sender = seg_lane >= 4u && seg_lane < 8u;
    uint4 *box = nullptr;
    bool self_nb = false;  // taker lane: the neighbour in direction d is this island
    if (taker) {
        const uint32_t y = div_cols(island, p.cols_m, p.cols_l), x = island - y * p.cols;
        const uint32_t yn = d == 0u ? (y == 0u ? p.rows - 1u : y - 1u)
                          : d == 1u ? (y + 1u == p.rows ? 0u : y + 1u) : y;
        const uint32_t xn = d == 2u ? (x + 1u == p.cols ? 0u : x + 1u)
                          : d == 3u ? (x == 0u ? p.cols - 1u : x - 1u) : x;
        const uint32_t nb = yn * p.cols + xn;
        self_nb = nb == island;
        box = a.mail + (static_cast<size_t>(in_bounds(nb < p.n_islands, p.status) ? nb : island) * 4u +
                        (d ^ 1u)) * MB;
    } else if (sender) {
        box = a.mail + (static_cast<size_t>(island) * 4u + d) * MB;
    }
    uint32_t *const flag = reinterpret_cast<uint32_t *>(box);  // flag protocol only
    const bool early = p.rows > 1u && p.cols > 1u;  // no island is its own neighbour
    uint4 got = make_uint4(~0u, ~0u, ~0u, ~0u);     // atomic protocol: the taken record
    uint32_t f = 0;                                 // flag protocol: the tested flag
    bool pending = false;                           // flag protocol: publication due

    // Take (atomic protocol) or test (flag protocol) ahead of a migration generation's
    // buffer step.
    auto prepare = [&]() {
        if constexpr (kAtomic) {
            if (taker) got = take128(box);
        } else {
            if (taker || sender) f = pending ? 1u : ld_relaxed(flag);
        }
    };
    // generations since the last migration generation (g mod every_k), kept incrementally
    uint32_t phase = a.phase0;
    if (early && p.migrate && phase == 0u) prepare();

    for (uint32_t it = 0; it < p.n_gens; ++it) {
        const uint32_t g = p.g0 + it;
        uint4 w[A];
        birth_draws<N>(w, p, a.rk, g, island, seg_lane);
        const bool mig = p.migrate && phase == 0u;
        phase = phase + 1u == a.every_k ? 0u : phase + 1u;  // now (g + 1) mod every_k
        if (mig && !early) {
            __syncwarp(mask);  // after the previous generation's refills by this warp
            prepare();
        }
        if constexpr (!kAtomic) {
            if (mig) fence_acq_rel();  // the flag tests act as acquire loads
            if (pending) {             // sends started in the previous generation complete
                st_release(flag, 1u);
                pending = false;
            }
        }

        if (mig) {
            // 1. collect
            uint32_t imm[LW];
#pragma unroll
            for (int k = 0; k < LW; ++k) imm[k] = 0u;
            bool arrived;
            if constexpr (kAtomic) {
                arrived = taker && got.y != kNeverSent;
                if (arrived) {
                    const uint32_t g4[4] = {got.x, got.y, got.z, got.w};
#pragma unroll
                    for (int k = 0; k < LW; ++k) imm[k] = g4[k];
                }
            } else {
                arrived = taker && f != 0u;
                if (arrived) {
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        const uint4 xq = ld_relaxed_v4(box + 1 + q);
                        const uint32_t w4[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (4 * q + k < LW) imm[4 * q + k] = w4[k];
                    }
                    st_release(flag, 0u);  // the buffer goes back to its owner
                }
            }
            // landing slots: partial Fisher-Yates over [0, N) in direction order (entry e:
            // "position r[e] now holds value v[e]", later entries winning)
            const uint32_t u = __shfl_sync(mask, w[0].w, static_cast<int>(d), SEG);  // slot d's draw
            const uint32_t r_own = d + (((u >> 16) * static_cast<uint32_t>(N - d)) >> 16);
            uint32_t r[4];
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) r[dd] = __shfl_sync(mask, r_own, dd, SEG);
            const uint32_t came = __ballot_sync(mask, arrived);
            const uint32_t came_seg = (came >> (lane - seg_lane)) & 0xFu;
            uint32_t v[4], slot[4];
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) {
                uint32_t vd = dd, vr = r[dd];
#pragma unroll
                for (int e = 0; e < dd; ++e) {
                    if (r[e] == static_cast<uint32_t>(dd)) vd = v[e];
                    if (r[e] == r[dd]) vr = v[e];
                }
                slot[dd] = vr;
                v[dd] = vd;
            }
            if (came != 0u) {  // uniform across the warp: every valid lane joins the shuffles
#pragma unroll
                for (int ag = 0; ag < A; ++ag) {
                    const uint32_t mine = seg_lane + 32u * ag;
                    int src_lane = -1;
#pragma unroll
                    for (int dd = 0; dd < 4; ++dd)
                        if (slot[dd] == mine && ((came_seg >> dd) & 1u)) src_lane = dd;
#pragma unroll
                    for (int k = 0; k < LW; ++k) {
                        const uint32_t val = __shfl_sync(mask, imm[k], src_lane < 0 ? 0 : src_lane, SEG);
                        if (src_lane >= 0) rec[ag][k] = val;
                    }
                }
            }
            // 2. refill: sender lane 4 + d copies member e_d of the island as it now stands
            // into its buffer if that is empty
            const uint32_t e = (((u >> 8) & 0xFFu) * N) >> 8;
            uint32_t out[LW];
#pragma unroll
            for (int k = 0; k < LW; ++k) {
                if constexpr (N <= 32) {
                    out[k] = __shfl_sync(mask, rec[0][k], static_cast<int>(e), SEG);
                } else {
                    uint32_t val = 0;
#pragma unroll
                    for (int q = 0; q < A; ++q) {
                        const uint32_t xv = __shfl_sync(mask, rec[q][k], static_cast<int>(e & 31u));
                        if ((e >> 5) == static_cast<uint32_t>(q)) val = xv;
                    }
                    out[k] = val;
                }
            }
            // a buffer this island took a genome out of itself in this pass (its own
            // buffer towards d ^ 1, taken by its lane d) tested full: no refill now
            const uint32_t self_took =
                early ? 0u : (__ballot_sync(mask, arrived && self_nb) >> (lane - seg_lane)) & 0xFu;
            const bool sendable =
                sender && out[1] != kNeverSent && ((self_took >> (d ^ 1u)) & 1u) == 0u;
            if (!early) __syncwarp(mask);  // after this generation's takes by this warp
            if constexpr (kAtomic) {
                if (sendable) refill128(box, out);
            } else {
                bool fill;
                if (early) {
                    fill = sendable && f == 0u;
                } else {
                    const uint32_t now = sender ? ld_relaxed(flag) : 1u;
                    fence_acq_rel();
                    fill = sendable && now == 0u;
                }
                if (fill) {
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        uint32_t w4[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) w4[k] = (4 * q + k < LW) ? out[4 * q + k] : 0u;
                        st_relaxed_v4(box + 1 + q, make_uint4(w4[0], w4[1], w4[2], w4[3]));
                    }
                    if (early) pending = true;
                    else st_release(flag, 1u);
                }
            }
        }
        // the next generation's take / test, in flight during this generation's reproduction
        if (early && p.migrate && it + 1u < p.n_gens && phase == 0u) prepare();
        // 3. evaluation, selection, mutation, deposit
        reproduce<N, SW, TS, MODEL>(rec, w, p, a.rk, island, seg_lane, mask, g,
                                    gen_site_at(p, it));
        check_counters(rec, p.status);
    }
    if constexpr (!kAtomic) {
        if (pending) st_release(flag, 1u);
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

// One generation of 16-byte-record islands (a window of 1), migration bookkeeping shared by
// the block as in the synchronous kernel: thread t < 4 * islands-per-block serves island
// t / 4 and direction d = t % 4 -- it recomputes that island's slot-d birth draw (bits
// 16..31: the landing draw), takes the genome out of the neighbour's buffer facing the island
// with one 128-bit exchange, and resolves the landing slot with its three sibling lanes; the
// genomes and slots reach the island warps through shared memory.  The island warps then
// land the arrivals, refill their own buffers (lanes 4..7, compare-and-swap) from the island
// as it now stands, and reproduce.  Every take of the launch precedes every refill (block
// barrier), so an island that is its own neighbour takes what it sent in the previous
// generation and leaves that buffer empty for this pass, as in the one-warp kernel.
template <int N, int TS, int MODEL>
__global__ void __launch_bounds__(kAsyncThreads) island_async_gen_kernel(const AsyncArgs a)
{
    constexpr int A = Shape<N>::A, P = Shape<N>::P, SEG = Shape<N>::SEG;
    constexpr int LW = 4;                    // 16-byte records
    constexpr int BI = kAsyncWarps * P;      // islands per block
    constexpr int ML = BI * 4;               // bookkeeping lanes: (island, direction)
    constexpr uint32_t kNone = 0xFFFFFFFFu;  // no arrival from that direction
    __shared__ uint4 s_got[ML];
    __shared__ __align__(16) uint32_t s_slot[ML];
    __shared__ uint8_t s_self[ML];  // by (island, direction): own buffer emptied by itself
    const RunParams &p = a.r;
    const uint32_t g = p.g0;

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t seg_lane = lane % SEG;
    const uint32_t local = (threadIdx.x >> 5) * P + lane / SEG;
    const uint32_t island0 = a.first + blockIdx.x * BI;
    const uint32_t island = island0 + local;
    const bool valid = island < a.last;
    const unsigned mask = __ballot_sync(0xffffffffu, valid);
    const bool mig = p.migrate && a.phase0 == 0u;

    // Bookkeeping, part 1: the takes are issued first, so their latency overlaps the island
    // warps' record loads and birth draws.
    const bool bk = mig && threadIdx.x < ML;
    const unsigned bk_mask = __ballot_sync(0xffffffffu, bk);
    const uint32_t md = threadIdx.x & 3u;
    uint32_t r = md;
    uint4 got = make_uint4(~0u, ~0u, ~0u, ~0u);
    bool self_nb = false;
    if (bk) {
        const uint32_t isl = island0 + (threadIdx.x >> 2);
        if (isl < a.last) {
            const uint32_t u = philox_rk(g, isl, md | (kBirth << 16), p.run_id, a.rk).w;
            r = md + (((u >> 16) * static_cast<uint32_t>(N - md)) >> 16);
            const uint32_t y = div_cols(isl, p.cols_m, p.cols_l), x = isl - y * p.cols;
            const uint32_t yn = md == 0u ? (y == 0u ? p.rows - 1u : y - 1u)
                              : md == 1u ? (y + 1u == p.rows ? 0u : y + 1u) : y;
            const uint32_t xn = md == 2u ? (x + 1u == p.cols ? 0u : x + 1u)
                              : md == 3u ? (x == 0u ? p.cols - 1u : x - 1u) : x;
            const uint32_t nb = yn * p.cols + xn;
            self_nb = nb == isl;
            if (in_bounds(nb < p.n_islands, p.status))
                got = take128(a.mail + (static_cast<size_t>(nb) * 4u + (md ^ 1u)));
        }
    }

    uint32_t rec[A][LW];
    uint4 w[A];
    if (valid) {
#pragma unroll
        for (int ag = 0; ag < A; ++ag) {
            const uint4 v = __ldg(&p.src[static_cast<size_t>(island) * N + seg_lane + 32u * ag]);
            rec[ag][0] = v.x;
            rec[ag][1] = v.y;
            rec[ag][2] = v.z;
            rec[ag][3] = v.w;
        }
        birth_draws<N>(w, p, a.rk, g, island, seg_lane);
    }

    // Bookkeeping, part 2: the partial Fisher-Yates landing slots among the island's four
    // lanes (entry e: "position r[e] now holds value v[e]", later entries winning); a
    // direction with nothing to deliver keeps its swap but lands nothing.
    if (mig) {
        if (bk) {
            uint32_t rr[4];
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) rr[dd] = __shfl_sync(bk_mask, r, dd, 4);
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
            s_got[threadIdx.x] = got;
            s_slot[threadIdx.x] = got.y != kNeverSent ? slot : kNone;
            // this lane took from the island's own buffer towards md ^ 1 (entry t ^ 1)
            s_self[threadIdx.x ^ 1u] = self_nb && got.y != kNeverSent;
        }
        __syncthreads();
    }
    if (!valid) return;

    if (mig) {
        // land (branch-free: every lane reads a slot, the receivers keep it)
        const uint4 sl = *reinterpret_cast<const uint4 *>(&s_slot[4 * local]);
#pragma unroll
        for (int ag = 0; ag < A; ++ag) {
            const uint32_t mine = seg_lane + 32u * ag;
            const int from = sl.x == mine ? 0 : sl.y == mine ? 1 : sl.z == mine ? 2
                           : sl.w == mine ? 3 : -1;
            const uint4 xq = s_got[4 * local + (from < 0 ? 0 : from)];
            rec[ag][0] = from >= 0 ? xq.x : rec[ag][0];
            rec[ag][1] = from >= 0 ? xq.y : rec[ag][1];
            rec[ag][2] = from >= 0 ? xq.z : rec[ag][2];
            rec[ag][3] = from >= 0 ? xq.w : rec[ag][3];
        }
        // refill: lane 4 + d copies member e_d of the island as it now stands into its
        // buffer towards d if that is empty
        const uint32_t d = seg_lane & 3u;
        const uint32_t u = __shfl_sync(mask, w[0].w, static_cast<int>(d), SEG);
        const uint32_t e = (((u >> 8) & 0xFFu) * N) >> 8;
        uint32_t out[LW];
#pragma unroll
        for (int k = 0; k < LW; ++k) {
            if constexpr (N <= 32) {
                out[k] = __shfl_sync(mask, rec[0][k], static_cast<int>(e), SEG);
            } else {
                uint32_t val = 0;
#pragma unroll
                for (int q = 0; q < A; ++q) {
                    const uint32_t xv = __shfl_sync(mask, rec[q][k], static_cast<int>(e & 31u));
                    if ((e >> 5) == static_cast<uint32_t>(q)) val = xv;
                }
                out[k] = val;
            }
        }
        if (seg_lane >= 4u && seg_lane < 8u && out[1] != kNeverSent && !s_self[4 * local + d])
            refill128(a.mail + (static_cast<size_t>(island) * 4u + d), out);
    }
    reproduce<N, 2, TS, MODEL>(rec, w, p, a.rk, island, seg_lane, mask, g, gen_site_at(p, 0u));
    check_counters(rec, p.status);
#pragma unroll
    for (int ag = 0; ag < A; ++ag)
        p.dst[static_cast<size_t>(island) * N + seg_lane + 32u * ag] =
            make_uint4(rec[ag][0], rec[ag][1], rec[ag][2], rec[ag][3]);
}

using AsyncKernel = void (*)(AsyncArgs);

template <int N, int TS>
AsyncKernel pick_async_n(uint32_t surface_words, uint32_t model)
{
    if (model == GA_MODEL_FITNESS) {  // the float-fitness model: islands of 16 to 64 agents
        if constexpr (N >= 16 && N <= 64)
            return surface_words <= 2 ? island_async_kernel<N, 2, TS, 1> : nullptr;
        return nullptr;
    }
    if (surface_words <= 2) return island_async_kernel<N, 2, TS, 0>;
    if (surface_words <= 6) return island_async_kernel<N, 6, TS, 0>;
    if (surface_words <= 8) return island_async_kernel<N, 8, TS, 0>;
    return nullptr;
}

// Tournament size 5 (the paper's) is compiled in; other sizes are read from the run.
template <int N>
AsyncKernel pick_async_ts(uint32_t surface_words, uint32_t tsize, uint32_t model)
{
    return tsize == 5u ? pick_async_n<N, 5>(surface_words, model)
                       : pick_async_n<N, 0>(surface_words, model);
}

AsyncKernel pick_async(uint32_t island_size, uint32_t surface_words, uint32_t tsize, uint32_t model)
{
    switch (island_size) {  // N >= 8: an island needs lanes 0..3 to take and 4..7 to send
    case 8: return pick_async_ts<8>(surface_words, tsize, model);
    case 16: return pick_async_ts<16>(surface_words, tsize, model);
    case 32: return pick_async_ts<32>(surface_words, tsize, model);
    case 64: return pick_async_ts<64>(surface_words, tsize, model);
    case 128: return pick_async_ts<128>(surface_words, tsize, model);
    default: return nullptr;
    }
}

// One-generation launches of 16-byte records.
template <int N>
AsyncKernel pick_async_gen_n(uint32_t tsize, uint32_t model)
{
    if (model == GA_MODEL_FITNESS) {
        if constexpr (N >= 16 && N <= 64)
            return tsize == 5u ? island_async_gen_kernel<N, 5, 1> : island_async_gen_kernel<N, 0, 1>;
        return nullptr;
    }
    return tsize == 5u ? island_async_gen_kernel<N, 5, 0> : island_async_gen_kernel<N, 0, 0>;
}

AsyncKernel pick_async_gen(uint32_t island_size, uint32_t tsize, uint32_t model)
{
    switch (island_size) {
    case 8: return pick_async_gen_n<8>(tsize, model);
    case 16: return pick_async_gen_n<16>(tsize, model);
    case 32: return pick_async_gen_n<32>(tsize, model);
    case 64: return pick_async_gen_n<64>(tsize, model);
    case 128: return pick_async_gen_n<128>(tsize, model);
    default: return nullptr;
    }
}

// 16-byte records travel through 16-byte buffers (all ones when empty); larger records
// through a 16-byte flag word plus the record (flag 0 when empty).
bool atomic_buffers(uint32_t record_bytes) { return record_bytes == 16u; }

size_t buffer_bytes(uint32_t record_bytes)
{
    return atomic_buffers(record_bytes) ? 16u : 16u + record_bytes;
}

}  // namespace

bool async_supported(uint32_t island_size, uint32_t surface_words, uint32_t model)
{
    return pick_async(island_size, surface_words, 1u, model) != nullptr;
}

// Send buffers: [island][4] buffers.
size_t async_state_bytes(uint32_t n_islands, uint32_t record_bytes)
{
    const size_t bytes = static_cast<size_t>(n_islands) * 4u * buffer_bytes(record_bytes);
    return (bytes + 255u) / 256u * 256u;
}

// Empty every send buffer.
cudaError_t async_clear(ga_run *run, cudaStream_t stream)
{
    return cudaMemsetAsync(run->mail, atomic_buffers(run->record_bytes) ? 0xFF : 0x00,
                           async_state_bytes(run->n_islands, run->record_bytes), stream);
}

cudaError_t launch_island_async(ga_run *run, const void *src, void *dst, uint32_t g0,
                                uint32_t n_gens, uint32_t first, uint32_t last,
                                cudaStream_t stream)
{
    // a single generation of 16-byte records: the block-cooperative kernel
    const AsyncKernel k =
        n_gens == 1u && atomic_buffers(run->record_bytes)
            ? pick_async_gen(run->cfg.island_size, run->cfg.tournament_size, run->cfg.model)
            : pick_async(run->cfg.island_size, run->surface_words, run->cfg.tournament_size,
                         run->cfg.model);
    if (!k || first >= last || last > run->n_islands) return cudaErrorInvalidValue;
    AsyncArgs a;
    a.r = run_params(run, src, dst, g0, n_gens, run->per_neighbor != 0);
    a.rk = round_keys(Key{static_cast<uint32_t>(run->cfg.seed),
                          static_cast<uint32_t>(run->cfg.seed >> 32)});
    a.mail = reinterpret_cast<uint4 *>(run->mail);
    a.every_k = run->every_k;
    a.phase0 = g0 % run->every_k;
    a.first = first;
    a.last = last;
    const uint32_t N = run->cfg.island_size;
    const uint32_t per_block = kAsyncWarps * (N >= 32 ? 1u : 32u / N);
    const uint32_t blocks = (last - first + per_block - 1) / per_block;
    k<<<blocks, kAsyncThreads, 0, stream>>>(a);
    run->launches += 1;
    return cudaGetLastError();
}

// ga_step in the asynchronous modes: windows of async_window generations (cut also at the
// site-table chunks); GA_ASYNC runs every island in one launch per window,
// GA_ASYNC_SEQUENTIAL one launch per island in index order.  The population is
// double-buffered per window: every island reads its records from the current buffer and
// writes them to the other, while the send buffers persist in the workspace.
int async_step(ga_run *run, uint32_t n_gens, cudaStream_t stream)
{
    if (run->generation + n_gens > 0xFFFFFFFFull) return GA_EINVAL;
    const bool sequential = run->cfg.mode == GA_ASYNC_SEQUENTIAL;
    while (n_gens > 0) {
        const uint32_t chunk = n_gens < kSiteTableCap ? n_gens : kSiteTableCap;
        if (launch_site_table(run, static_cast<uint32_t>(run->generation), chunk, stream) !=
            cudaSuccess)
            return GA_ECUDA;
        run->sites_base = run->generation;
        uint32_t left = chunk;
        while (left > 0) {
            const uint32_t len = left < run->async_window ? left : run->async_window;
            const uint32_t g0 = static_cast<uint32_t>(run->generation);
            const void *src = run->pop[run->cur];
            void *dst = run->pop[run->cur ^ 1];
            if (sequential) {
                for (uint32_t i = 0; i < run->n_islands; ++i)
                    if (launch_island_async(run, src, dst, g0, len, i, i + 1u, stream) != cudaSuccess)
                        return GA_ECUDA;
            } else if (launch_island_async(run, src, dst, g0, len, 0u, run->n_islands, stream) !=
                       cudaSuccess) {
                return GA_ECUDA;
            }
            run->cur ^= 1;
            run->generation += len;
            left -= len;
        }
        n_gens -= chunk;
    }
    return GA_OK;
}

}  // namespace ga
