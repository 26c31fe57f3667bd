// ga_step.cu -- founder initialisation and the fused island-step kernel.
//
// One generation (Sec. 2 of the paper, in its order): migration (when due), evaluation
// (fitness = trait), tournament selection of every next-generation slot, copy and mutation
// of the child, and the hstrat deposit for the elapsed generation.
//
// Mapping: one island per warp for N >= 32 (N/32 agents per lane), 32/N islands per warp
// for N < 32 (one agent per lane, shuffles of width N).  A block owns 8 warps of consecutive
// islands.  Each lane keeps its agents' records in registers; tournaments read candidate
// traits and copy the winner's record with __shfl_sync, so an island never leaves the
// register file between the launch's first load and last store.  A launch runs generations
// [g0, g0 + n) with migration only at g0: the population is read once from `src` and
// written once to `dst` per launch, and immigrants are read straight from the neighbours'
// records in `src` (the whole previous population doubles as the migration halo, so no
// separate halo buffer or grid barrier is needed and the result does not depend on launch
// order).
//
// Migration bookkeeping is lane-parallel across the block: one thread per (island,
// direction) pair recomputes that island's birth draw for slot d (the draw that carries the
// migration bits), derives the immigrant index and landing draw, finds the torus neighbour,
// loads the immigrant record and resolves the partial Fisher-Yates landing slot with its
// three sibling lanes; records and slots go through shared memory, so an island's warp only
// compares four slot numbers and reads at most one record per agent.
#include "ga_device.cuh"
#include "ga_internal.h"

namespace ga {

constexpr int kStepThreads = 256;
constexpr int kStepWarps = kStepThreads / 32;

struct StepArgs {
    const uint4 *__restrict__ src;
    uint4 *__restrict__ dst;
    uint32_t rows, cols, n_islands;
    uint32_t tsize;
    uint32_t theta_ben, theta_del;
    uint32_t policy, log2_sites, sites, bits;
    RoundKeys rk;
    uint32_t run_id;
    uint32_t g0, n_gens, migrate;
    const int32_t *__restrict__ gen_sites;  // curation site of generation g0 + i
};

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
__device__ __forceinline__ void birth_draws(uint4 (&w)[Shape<N>::A], const StepArgs &p, uint32_t g,
                                            uint32_t island, uint32_t seg_lane)
{
#pragma unroll
    for (int ag = 0; ag < Shape<N>::A; ++ag)
        w[ag] = philox_rk(g, island, (seg_lane + 32u * ag) | (kBirth << 16), p.run_id, p.rk);
}

// Evaluation, tournament, copy, mutation and hstrat deposit of one generation, in place.
// Closed-form curation site, called only for agents whose counter differs from the
// generation (never in synchronous runs); kept out of line so the common path stays a load.
__device__ __noinline__ int curation_site_of(uint32_t policy, uint32_t log2_sites, uint32_t sites,
                                            uint32_t T)
{
    return curation_site(policy, log2_sites, sites, T);
}

// g: the generation; gen_site: its curation site, valid for agents whose counter is g (all
// agents in synchronous runs) -- any other counter takes the closed form.
template <int N, int SW, int TS>
__device__ __forceinline__ void reproduce(uint32_t (&rec)[Shape<N>::A][2 + SW],
                                          const uint4 (&w)[Shape<N>::A], const StepArgs &p,
                                          unsigned mask, uint32_t g, int gen_site)
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
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if constexpr (TS > 0) {
                if (i >= TS) break;
            } else {
                if (static_cast<uint32_t>(i) >= p.tsize) break;
            }
            const uint32_t word = i < 4 ? w[ag].x : w[ag].y;
            uint32_t sel = word >> (8 * (i & 3) + 8 - LOGN);
            if constexpr (N > 32) sel &= N - 1u;
            const int t = candidate_trait<N, A, SEG>(mask, trait, sel);
            if (i == 0 || t > best_trait) {
                best = sel;
                best_trait = t;
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
        uint32_t t = child[ag][0];
        if (xm < p.theta_del) t -= 1u;
        else if (xm - p.theta_del < p.theta_ben) t += 1u;
        child[ag][0] = t;

        const uint32_t c = child[ag][1];
        int site = gen_site;
        if (c != g) site = curation_site_of(p.policy, p.log2_sites, p.sites, c);
        if (site >= 0) {
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

// N: island size; SW: surface words carried per record (the record is RW words); TS: the
// tournament size when fixed at compile time (0: read from the arguments).
template <int N, int SW, int TS>
__global__ void __launch_bounds__(kStepThreads) island_step_kernel(const StepArgs p)
{
    constexpr int A = Shape<N>::A, P = Shape<N>::P, SEG = Shape<N>::SEG;
    constexpr int LW = 2 + SW;                   // live words: trait, counter, surface
    constexpr int RW = (LW + 3) / 4 * 4;         // record words
    constexpr int Q = RW / 4;                    // 128-bit words per record
    constexpr int BI = kStepWarps * P;           // islands per block
    constexpr int ML = BI * 4;                   // migration lanes: (island, direction)

    __shared__ uint4 s_imm[ML][Q];                // immigrant records
    __shared__ __align__(16) uint32_t s_slot[ML]; // landing slot of each immigrant

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t seg_lane = lane % SEG;
    const uint32_t local = (threadIdx.x >> 5) * P + lane / SEG;
    const uint32_t island0 = blockIdx.x * BI;
    const uint32_t island = island0 + local;
    const bool valid = island < p.n_islands;
    const unsigned mask = __ballot_sync(0xffffffffu, valid);

    // Migration bookkeeping, part 1 (threads < ML, whole warps): the immigrant loads are
    // issued first, so their latency overlaps everything up to the block barrier.
    const bool mig_lane = p.migrate && threadIdx.x < ML;
    const uint32_t md = threadIdx.x & 3u;  // direction of this bookkeeping lane
    uint32_t r = md;                       // its landing draw
    uint4 imm[Q];
    if (mig_lane) {
        const uint32_t isl = island0 + (threadIdx.x >> 2);
        if (isl < p.n_islands) {
            // birth draw of slot d: bits 8..15 pick the immigrant, bits 16..31 its landing
            const uint32_t u = philox_rk(p.g0, isl, md | (kBirth << 16), p.run_id, p.rk).w;
            r = md + (((u >> 16) * static_cast<uint32_t>(N - md)) >> 16);
            const uint32_t e = (((u >> 8) & 0xFFu) * N) >> 8;
            const uint32_t y = isl / p.cols, x = isl - y * p.cols;
            const uint32_t yn = md == 0u ? (y == 0u ? p.rows - 1u : y - 1u)
                              : md == 1u ? (y + 1u == p.rows ? 0u : y + 1u) : y;
            const uint32_t xn = md == 2u ? (x + 1u == p.cols ? 0u : x + 1u)
                              : md == 3u ? (x == 0u ? p.cols - 1u : x - 1u) : x;
            const uint4 *srec = p.src + (static_cast<size_t>(yn * p.cols + xn) * N + e) * Q;
#pragma unroll
            for (int q = 0; q < Q; ++q) imm[q] = __ldg(&srec[q]);
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
        birth_draws<N>(w, p, p.g0, island, seg_lane);
    }

    // Migration bookkeeping, part 2: the partial Fisher-Yates landing slots (over [0, N) in
    // direction order, among the island's four lanes: entry e records "position r[e] now
    // holds value v[e]", later entries winning), then records and slots to shared memory.
    if (p.migrate) {
        if (mig_lane) {
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
            s_slot[threadIdx.x] = slot;
            if (island0 + (threadIdx.x >> 2) < p.n_islands) {
#pragma unroll
                for (int q = 0; q < Q; ++q) s_imm[threadIdx.x][q] = imm[q];
            }
        }
        __syncthreads();
    }
    if (!valid) return;

    if (p.migrate) {
        // the four immigrants land in their slots
        const uint4 sl = *reinterpret_cast<const uint4 *>(&s_slot[4 * local]);
#pragma unroll
        for (int ag = 0; ag < A; ++ag) {
            const uint32_t mine = seg_lane + 32u * ag;
            const int from = sl.x == mine ? 0 : sl.y == mine ? 1 : sl.z == mine ? 2
                           : sl.w == mine ? 3 : -1;
            if (from >= 0) {
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const uint4 xq = s_imm[4 * local + from][q];
                    const uint32_t w4[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (4 * q + k < LW) rec[ag][4 * q + k] = w4[k];
                }
            }
        }
    }
    reproduce<N, SW, TS>(rec, w, p, mask, p.g0, __ldg(&p.gen_sites[0]));

    // generations g0 + 1 .. g0 + n - 1: no migration, the island stays in registers
    for (uint32_t it = 1; it < p.n_gens; ++it) {
        birth_draws<N>(w, p, p.g0 + it, island, seg_lane);
        reproduce<N, SW, TS>(rec, w, p, mask, p.g0 + it, __ldg(&p.gen_sites[it]));
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

// Every record becomes the founder: trait 0, counter 0, surface word w = word 0 of
// Philox((0, 0, w | FOUNDER << 16, run_id)); surface bits past S*b are zero.
__global__ void founder_kernel(uint4 *__restrict__ dst, uint32_t n_agents, uint32_t q_per_rec,
                               uint32_t surface_words, uint32_t top_bits, Key key,
                               uint32_t run_id)
{
    __shared__ uint32_t words[12];
    if (threadIdx.x < 12) {
        uint32_t val = 0u;
        const uint32_t k = threadIdx.x;
        if (k >= 2 && k - 2 < surface_words) {
            val = philox(0u, 0u, (k - 2) | (kFounder << 16), run_id, key).x;
            if (k - 2 == surface_words - 1 && top_bits) val &= (1u << top_bits) - 1u;
        }
        words[k] = val;
    }
    __syncthreads();
    const size_t total = static_cast<size_t>(n_agents) * q_per_rec;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const uint32_t q = static_cast<uint32_t>(i % q_per_rec);
        dst[i] = make_uint4(words[4 * q], words[4 * q + 1], words[4 * q + 2], words[4 * q + 3]);
    }
}

__global__ void curation_sites_kernel(uint32_t policy, uint32_t log2_sites, uint32_t sites,
                                      uint32_t t0, uint32_t count, int32_t *__restrict__ out)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += gridDim.x * blockDim.x)
        out[i] = curation_site(policy, log2_sites, sites, t0 + i);
}

namespace {

using StepKernel = void (*)(StepArgs);

// The template's surface-word count fills the record: 16-byte records carry 2 surface words,
// 32-byte records 6 and 48-byte records 8 (words past the run's own S*b bits are zero).
// Tournament size 5 (the paper's, Sec. 3) has its own instantiation; other sizes use the
// kernel that reads the size from its arguments.
template <int N, int SW>
StepKernel pick_ts(uint32_t tsize)
{
    return tsize == 5 ? island_step_kernel<N, SW, 5> : island_step_kernel<N, SW, 0>;
}

template <int N>
StepKernel pick_sw(uint32_t surface_words, uint32_t tsize)
{
    if (surface_words <= 2) return pick_ts<N, 2>(tsize);
    if (surface_words <= 6) return pick_ts<N, 6>(tsize);
    if (surface_words <= 8) return pick_ts<N, 8>(tsize);
    return nullptr;
}

StepKernel pick_kernel(uint32_t island_size, uint32_t surface_words, uint32_t tsize)
{
    switch (island_size) {
    case 4: return pick_sw<4>(surface_words, tsize);
    case 8: return pick_sw<8>(surface_words, tsize);
    case 16: return pick_sw<16>(surface_words, tsize);
    case 32: return pick_sw<32>(surface_words, tsize);
    case 64: return pick_sw<64>(surface_words, tsize);
    case 128: return pick_sw<128>(surface_words, tsize);
    default: return nullptr;
    }
}

uint32_t sm_count()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return static_cast<uint32_t>(sms);
}

}  // namespace

bool step_supported(uint32_t island_size, uint32_t surface_words)
{
    return pick_kernel(island_size, surface_words, 1) != nullptr;
}

cudaError_t launch_founder(ga_run *run, void *dst)
{
    const uint32_t q = run->record_bytes / 16;
    const uint32_t top = (run->cfg.surface_sites * run->cfg.differentia_bits) % 32u;
    const Key key{static_cast<uint32_t>(run->cfg.seed), static_cast<uint32_t>(run->cfg.seed >> 32)};
    const size_t total = static_cast<size_t>(run->n_agents) * q;
    size_t blocks = (total + 255) / 256;
    const size_t cap = static_cast<size_t>(sm_count()) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    founder_kernel<<<static_cast<unsigned>(blocks), 256, 0, run->stream>>>(
        static_cast<uint4 *>(dst), run->n_agents, q, run->surface_words, top, key, run->cfg.run_id);
    run->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_island_step(ga_run *run, const void *src, void *dst, uint32_t g0,
                               uint32_t n_gens, bool migrate)
{
    const StepKernel k =
        pick_kernel(run->cfg.island_size, run->surface_words, run->cfg.tournament_size);
    if (!k) return cudaErrorInvalidValue;
    StepArgs a;
    a.src = static_cast<const uint4 *>(src);
    a.dst = static_cast<uint4 *>(dst);
    a.rows = run->cfg.rows;
    a.cols = run->cfg.cols;
    a.n_islands = run->n_islands;
    a.tsize = run->cfg.tournament_size;
    a.theta_ben = run->theta_ben;
    a.theta_del = run->theta_del;
    a.policy = run->cfg.curation;
    a.log2_sites = run->log2_sites;
    a.sites = run->cfg.surface_sites;
    a.bits = run->cfg.differentia_bits;
    a.rk = round_keys(Key{static_cast<uint32_t>(run->cfg.seed),
                          static_cast<uint32_t>(run->cfg.seed >> 32)});
    a.run_id = run->cfg.run_id;
    a.g0 = g0;
    a.n_gens = n_gens;
    a.migrate = migrate ? 1u : 0u;
    a.gen_sites = run->d_sites + (g0 - run->sites_base);
    const uint32_t N = run->cfg.island_size;
    const uint32_t islands_per_block = kStepWarps * (N >= 32 ? 1u : 32u / N);
    const uint32_t blocks = (run->n_islands + islands_per_block - 1) / islands_per_block;
    k<<<blocks, kStepThreads, 0, run->stream>>>(a);
    run->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_site_table(ga_run *run, uint32_t g0, uint32_t count)
{
    const cudaError_t e = launch_curation_sites(run->cfg.curation, run->cfg.surface_sites, g0,
                                                count, run->d_sites, run->stream);
    run->launches += 1;
    return e;
}

cudaError_t launch_curation_sites(uint32_t policy, uint32_t sites, uint32_t t0, uint32_t count,
                                  int32_t *d_sites, cudaStream_t stream)
{
    if (count == 0) return cudaSuccess;
    uint32_t s = 0;
    while ((1u << s) < sites) ++s;
    uint32_t blocks = (count + 255u) / 256u;
    if (blocks > 8192u) blocks = 8192u;
    curation_sites_kernel<<<blocks, 256, 0, stream>>>(policy, s, sites, t0, count, d_sites);
    return cudaGetLastError();
}

}  // namespace ga
