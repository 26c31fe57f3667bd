// ga_async.cu -- the asynchronous island step: migration through per-island mailboxes.
//
// This follows the wafer-scale loop of the paper (Sec. 2) more literally than the
// synchronous mode: each island owns one outgoing mailbox per cardinal direction; on each
// migration generation it first takes whatever its neighbours posted since it last looked,
// landing each arrival in a random slot, then refills its own mailboxes with copies of
// randomly sampled members, then evaluates, selects, mutates and deposits as usual.  Nothing
// ever waits: an unchanged or half-written mailbox is skipped, so islands exchange migrants
// at whatever pace the hardware runs them, and a migrant keeps the counter of its lineage
// (deposit sites then follow each agent's own counter, as in the synchronous kernels'
// closed-form branch).
//
// Mailbox protocol (a sequence lock without waiting): the owner stores seq + 1 (odd: being
// written), fences, stores the record, fences, stores seq + 2.  A reader loads seq and skips
// the mailbox when seq is zero (never posted), odd (being written) or equal to the last
// sequence it took; otherwise it loads the record, fences, re-loads seq and keeps the record
// only if seq did not move.  Mailbox words are accessed with volatile loads and stores (no
// stale L1 copies) and __threadfence orders them device-wide.  Sequence words grow by 2 per
// post and wrap after 2^31 posts of one mailbox.
//
// Draws: the birth draws of the synchronous mode, keyed by the generation the island is
// running.  For direction d, word 3 of slot d's draw supplies bits 8..15 to choose the
// member posted towards d (the sender samples) and bits 16..31 for the landing slot of the
// arrival from d (the partial Fisher-Yates draw of the synchronous mode; an arrival that did
// not come leaves its slot as it was).
//
// Mapping: one island per warp for N >= 32, 32/N islands per warp below; lane d < 4 of an
// island polls direction d and owns the island's mailbox towards d.  Every lane runs the
// window's generations back to back with its agents in registers, as in the synchronous
// kernels.
#include "ga_device.cuh"
#include "ga_internal.h"
#include "ga_island.cuh"

namespace ga {

// Defined with the synchronous launchers.
RunParams run_params(const ga_run *run, const void *src, void *dst, uint32_t g0, uint32_t n_gens,
                     bool migrate);

namespace {

constexpr int kAsyncThreads = 256;
constexpr int kAsyncWarps = kAsyncThreads / 32;

struct AsyncArgs {
    RunParams r;
    RoundKeys rk;
    uint4 *mail;       // [island][4] mailboxes of 1 + Q uint4: sequence word, record
    uint32_t *seen;    // [island][4] last sequence taken from each direction
    uint32_t every_k;  // migration on generations g with g mod every_k == 0
    uint32_t first, last;  // islands [first, last) run in this launch
};

template <int N, int SW, int MODEL>
__global__ void __launch_bounds__(kAsyncThreads) island_async_kernel(const AsyncArgs a)
{
    constexpr int A = Shape<N>::A, P = Shape<N>::P, SEG = Shape<N>::SEG;
    constexpr int LW = 2 + SW;
    constexpr int RW = (LW + 3) / 4 * 4;
    constexpr int Q = RW / 4;
    constexpr int MB = 1 + Q;  // mailbox size in uint4
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

    // lane d < 4: polls the neighbour in direction d (0 north, 1 south, 2 east, 3 west),
    // whose mailbox facing this island is the opposite direction d ^ 1, and owns this
    // island's mailbox towards d
    const uint32_t d = seg_lane;
    const bool io_lane = d < 4u;
    volatile uint32_t *in_seq = nullptr;
    volatile uint32_t *out_seq = nullptr;
    uint32_t seen = 0, my_seq = 0;
    if (io_lane) {
        const uint32_t y = island / p.cols, x = island - y * p.cols;
        const uint32_t yn = d == 0u ? (y == 0u ? p.rows - 1u : y - 1u)
                          : d == 1u ? (y + 1u == p.rows ? 0u : y + 1u) : y;
        const uint32_t xn = d == 2u ? (x + 1u == p.cols ? 0u : x + 1u)
                          : d == 3u ? (x == 0u ? p.cols - 1u : x - 1u) : x;
        const uint32_t from = yn * p.cols + xn;
        in_seq = reinterpret_cast<volatile uint32_t *>(
            a.mail + (static_cast<size_t>(from) * 4u + (d ^ 1u)) * MB);
        out_seq = reinterpret_cast<volatile uint32_t *>(
            a.mail + (static_cast<size_t>(island) * 4u + d) * MB);
        seen = a.seen[static_cast<size_t>(island) * 4u + d];
        my_seq = *out_seq;
    }

    for (uint32_t it = 0; it < p.n_gens; ++it) {
        const uint32_t g = p.g0 + it;
        uint4 w[A];
        birth_draws<N>(w, p, a.rk, g, island, seg_lane);

        if (p.migrate && g % a.every_k == 0u) {
            // 1. collect: lane d takes its neighbour's latest post, if new and not torn
            uint32_t imm[LW];
#pragma unroll
            for (int k = 0; k < LW; ++k) imm[k] = 0u;
            bool arrived = false;
            if (io_lane) {
                const uint32_t s1 = *in_seq;
                if (s1 != 0u && (s1 & 1u) == 0u && s1 != seen) {
                    __threadfence();
                    const volatile uint32_t *body = in_seq + 4;
#pragma unroll
                    for (int k = 0; k < LW; ++k) imm[k] = body[k];
                    __threadfence();
                    if (*in_seq == s1) {
                        arrived = true;
                        seen = s1;
                    }
                }
            }
            // landing slots: partial Fisher-Yates over [0, N) in direction order (entry e:
            // "position r[e] now holds value v[e]", later entries winning)
            const uint32_t u = w[0].w;  // word 3 of this lane's slot-seg_lane draw
            const uint32_t r_own = (d & 3u) + (((u >> 16) * static_cast<uint32_t>(N - (d & 3u))) >> 16);
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
            // 2. post: lane d copies member e_d of the island (after the arrivals landed)
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
            if (io_lane) {
                *out_seq = my_seq + 1u;
                __threadfence();
                volatile uint32_t *body = out_seq + 4;
#pragma unroll
                for (int k = 0; k < LW; ++k) body[k] = out[k];
                __threadfence();
                my_seq += 2u;
                *out_seq = my_seq;
            }
        }
        // 3. evaluation, selection, mutation, deposit
        reproduce<N, SW, 0, MODEL>(rec, w, p, a.rk, island, seg_lane, mask, g,
                                   __ldg(&p.gen_sites[it]));
    }

    if (io_lane) a.seen[static_cast<size_t>(island) * 4u + d] = seen;
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

using AsyncKernel = void (*)(AsyncArgs);

template <int N>
AsyncKernel pick_async_n(uint32_t surface_words, uint32_t model)
{
    if (model == GA_MODEL_FITNESS) return surface_words <= 2 ? island_async_kernel<N, 2, 1> : nullptr;
    if (surface_words <= 2) return island_async_kernel<N, 2, 0>;
    if (surface_words <= 6) return island_async_kernel<N, 6, 0>;
    if (surface_words <= 8) return island_async_kernel<N, 8, 0>;
    return nullptr;
}

AsyncKernel pick_async(uint32_t island_size, uint32_t surface_words, uint32_t model)
{
    switch (island_size) {
    case 16: return pick_async_n<16>(surface_words, model);
    case 32: return pick_async_n<32>(surface_words, model);
    case 64: return pick_async_n<64>(surface_words, model);
    default: return nullptr;
    }
}

size_t align256(size_t x) { return (x + 255u) / 256u * 256u; }

}  // namespace

bool async_supported(uint32_t island_size, uint32_t surface_words, uint32_t model)
{
    return pick_async(island_size, surface_words, model) != nullptr;
}

// Mailboxes ([island][4] of 16 + record_bytes bytes), then sequence marks ([island][4] uint32).
size_t async_state_bytes(uint32_t n_islands, uint32_t record_bytes)
{
    return align256(static_cast<size_t>(n_islands) * 4u * (16u + record_bytes)) +
           align256(static_cast<size_t>(n_islands) * 16u);
}

cudaError_t launch_island_async(ga_run *run, const void *src, void *dst, uint32_t g0,
                                uint32_t n_gens, uint32_t first, uint32_t last,
                                cudaStream_t stream)
{
    const AsyncKernel k = pick_async(run->cfg.island_size, run->surface_words, run->cfg.model);
    if (!k || first >= last || last > run->n_islands) return cudaErrorInvalidValue;
    AsyncArgs a;
    a.r = run_params(run, src, dst, g0, n_gens, run->per_neighbor != 0);
    a.rk = round_keys(Key{static_cast<uint32_t>(run->cfg.seed),
                          static_cast<uint32_t>(run->cfg.seed >> 32)});
    a.mail = reinterpret_cast<uint4 *>(run->mail);
    a.seen = run->seen;
    a.every_k = run->every_k;
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
// writes them to the other, while mailboxes and sequence marks persist in the workspace.
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
