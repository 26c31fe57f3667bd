// ga_async.cu -- the asynchronous island step: migration through one-genome send buffers.
//
// This follows the wafer-scale loop of the paper (Sec. 2): each island owns one send buffer
// per cardinal direction; on each migration generation it first tests every completion
// flag, then copies in the genomes that arrived (each replacing a random member), then
// refills the send buffers whose previous genome was taken, with copies of randomly sampled
// members; then it evaluates, selects, mutates and deposits as usual.  Nothing ever waits: a
// buffer that is not ready is simply skipped, so islands exchange migrants at whatever pace
// the hardware runs them, and a migrant keeps the counter of its lineage (deposits then
// follow each agent's own counter, as in the synchronous kernels' closed-form branch).
//
// Buffer protocol (single producer, single consumer, PTX memory model at GPU scope): the
// flag word is 0 (empty) or 1 (full).  The owner writes a genome only into an empty buffer
// (seen with an acquire load), with relaxed stores, and publishes it by a release store of
// 1; the neighbour takes a genome only from a full buffer (acquire load), with relaxed
// loads, and hands the buffer back by a release store of 0.  Each side touches the record
// only while the flag says the buffer is its own, and the release/acquire pairs order the
// other side's record accesses before its own, so a record is never read half-written.
// The owner's release of a new genome is issued at the start of its next generation (or at
// the end of the launch), by which time the record stores have long completed, so the
// release costs no wait.
//
// Draws: the birth draws of the synchronous mode, keyed by the generation the island is
// running.  For direction d, word 3 of slot d's draw supplies bits 16..31 for the landing
// slot of the arrival from d (the partial Fisher-Yates draw of the synchronous mode, the
// swap made whether or not anything arrives) and bits 8..15 for the member sent towards d.
//
// Mapping: one island per warp for N >= 32, 32/N islands per warp below; island lanes 0..3
// take from the neighbours (lane d: direction d), lanes 4..7 own the island's send buffers
// (lane 4 + d: towards d), so the eight flag tests of a generation are issued together.
// Every lane runs the window's generations back to back with its agents in registers, as in
// the synchronous kernels.
#include "ga_device.cuh"
#include "ga_internal.h"
#include "ga_island.cuh"

namespace ga {

// Defined with the synchronous launchers.
RunParams run_params(const ga_run *run, const void *src, void *dst, uint32_t g0, uint32_t n_gens,
                     bool migrate);

namespace {

// GPU-scope memory-model accesses to the send buffers (global memory, 16-byte aligned).
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
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

constexpr int kAsyncThreads = 256;
constexpr int kAsyncWarps = kAsyncThreads / 32;

struct AsyncArgs {
    RunParams r;
    RoundKeys rk;
    uint4 *mail;           // [island][4] send buffers of 1 + Q uint4: flag word, record
    uint32_t every_k;      // migration on generations g with g mod every_k == 0
    uint32_t first, last;  // islands [first, last) run in this launch
};

template <int N, int SW, int MODEL>
__global__ void __launch_bounds__(kAsyncThreads) island_async_kernel(const AsyncArgs a)
{
    constexpr int A = Shape<N>::A, P = Shape<N>::P, SEG = Shape<N>::SEG;
    constexpr int LW = 2 + SW;
    constexpr int RW = (LW + 3) / 4 * 4;
    constexpr int Q = RW / 4;
    constexpr int MB = 1 + Q;  // send buffer size in uint4
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
    if (taker) {
        const uint32_t y = island / p.cols, x = island - y * p.cols;
        const uint32_t yn = d == 0u ? (y == 0u ? p.rows - 1u : y - 1u)
                          : d == 1u ? (y + 1u == p.rows ? 0u : y + 1u) : y;
        const uint32_t xn = d == 2u ? (x + 1u == p.cols ? 0u : x + 1u)
                          : d == 3u ? (x == 0u ? p.cols - 1u : x - 1u) : x;
        box = a.mail + (static_cast<size_t>(yn * p.cols + xn) * 4u + (d ^ 1u)) * MB;
    } else if (sender) {
        box = a.mail + (static_cast<size_t>(island) * 4u + d) * MB;
    }
    uint32_t *const flag = reinterpret_cast<uint32_t *>(box);
    bool pending = false;  // sender: a genome written, its release not yet issued

    for (uint32_t it = 0; it < p.n_gens; ++it) {
        const uint32_t g = p.g0 + it;
        uint4 w[A];
        birth_draws<N>(w, p, a.rk, g, island, seg_lane);
        if (pending) {
            st_release(flag, 1u);
            pending = false;
        }

        if (p.migrate && g % a.every_k == 0u) {
            // 1. test all eight flags (after this warp's earlier buffer accesses: an island
            // can be its own neighbour)
            __syncwarp(mask);
            const uint32_t f = (taker || sender) ? ld_acquire(flag) : 0u;
            __syncwarp(mask);  // every test precedes every take (an island can feed itself)
            // 2. collect
            uint32_t imm[LW];
#pragma unroll
            for (int k = 0; k < LW; ++k) imm[k] = 0u;
            const bool arrived = taker && f != 0u;
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
            // 3. refill: sender lane 4 + d copies member e_d of the island as it now stands
            // into an empty buffer; the release follows at the next generation
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
            if (sender && f == 0u) {
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    uint32_t w4[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) w4[k] = (4 * q + k < LW) ? out[4 * q + k] : 0u;
                    st_relaxed_v4(box + 1 + q, make_uint4(w4[0], w4[1], w4[2], w4[3]));
                }
                pending = true;
            }
        }
        // 4. evaluation, selection, mutation, deposit
        reproduce<N, SW, 0, MODEL>(rec, w, p, a.rk, island, seg_lane, mask, g,
                                   __ldg(&p.gen_sites[it]));
    }
    if (pending) st_release(flag, 1u);

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

}  // namespace

bool async_supported(uint32_t island_size, uint32_t surface_words, uint32_t model)
{
    return pick_async(island_size, surface_words, model) != nullptr;
}

// Send buffers: [island][4] of 16 + record_bytes bytes (flag word padded to 16 bytes, record).
size_t async_state_bytes(uint32_t n_islands, uint32_t record_bytes)
{
    const size_t bytes = static_cast<size_t>(n_islands) * 4u * (16u + record_bytes);
    return (bytes + 255u) / 256u * 256u;
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
