// ga_step.cu -- founder initialisation, the single-run island-step kernel (the block body
// lives in ga_island.cuh) and the curation-site kernels.
#include "ga_device.cuh"
#include "ga_internal.h"
#include "ga_island.cuh"

namespace ga {

constexpr int kStepThreads = 256;
constexpr int kStepWarps = kStepThreads / 32;

// Single run: per-run values and round keys are kernel parameters (constant bank).
struct StepArgs {
    RunParams r;
    RoundKeys rk;
};

template <int N, int SW, int TS, int MODEL = 0, int CF = 1>
__global__ void __launch_bounds__(kStepThreads) island_step_kernel(const StepArgs a)
{
    step_block<N, SW, TS, kStepWarps, MODEL, CF>(a.r, a.rk, blockIdx.x);
}

// Multi-unit kernel (step_units in ga_island.cuh) for 16-byte records whose counters all
// equal the generation, islands of 16, 32 or 64 agents, any tournament size, both genome
// models; TS = 0 reads the tournament size from the run.
// Resident blocks per SM asked of the compiler: 8 (32 registers) below 64 agents; the two
// agents per lane of 64-agent islands need 40 registers (6 blocks).
template <int N>
constexpr int units_min_blocks() { return N >= 64 ? 6 : 8; }

template <int N, int TS, int MODEL>
__global__ void __launch_bounds__(kStepThreads, units_min_blocks<N>()) island_units_kernel(const StepArgs a)
{
    step_units<N, TS, units_per_block<N>(), MODEL>(a.r, a.rk, blockIdx.x);
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

__global__ void counter_check_kernel(const uint32_t *__restrict__ pop, uint32_t record_words,
                                     uint32_t n_agents, uint32_t generation, int *__restrict__ flag)
{
    for (size_t a = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; a < n_agents;
         a += static_cast<size_t>(gridDim.x) * blockDim.x)
        if (pop[a * record_words + 1u] != generation) *flag = 1;  // every writer stores 1
}

__global__ void curation_sites_kernel(uint32_t policy, uint32_t log2_sites, uint32_t sites,
                                      uint32_t t0, uint32_t count, int32_t *__restrict__ out,
                                      uint32_t bits, uint2 *__restrict__ masks)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += gridDim.x * blockDim.x) {
        const int site = curation_site(policy, log2_sites, sites, t0 + i);
        out[i] = site;
        if (masks) {  // sites * bits <= 64: the deposit's bits within surface words 0 and 1
            const uint32_t pos = site >= 0 ? static_cast<uint32_t>(site) * bits : 0u;
            const uint32_t m = site >= 0 ? ((1u << bits) - 1u) << (pos & 31u) : 0u;
            masks[i] = make_uint2(pos < 32u ? m : 0u, pos < 32u ? 0u : m);
        }
    }
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

// The float-fitness model (16-byte records: fitness, counter, 64-bit surface -- the paper's
// 128-bit genome of Sec. 3) has kernels for islands of 16, 32 and 64.
template <int N>
StepKernel pick_fitness(uint32_t surface_words, uint32_t tsize)
{
    if (surface_words > 2) return nullptr;
    return tsize == 5 ? island_step_kernel<N, 2, 5, 1> : island_step_kernel<N, 2, 0, 1>;
}

// Kernels without the closed-form curation path, for launches whose counters all equal the
// generation, tournament size 5 (the paper's, Sec. 3): 16-byte trait records for every island
// size, 32- and 48-byte trait records and the float-fitness model for islands of 16, 32 and 64.
template <int N>
StepKernel pick_uniform_wide(uint32_t surface_words)
{
    if (surface_words <= 6) return island_step_kernel<N, 6, 5, 0, 0>;
    if (surface_words <= 8) return island_step_kernel<N, 8, 5, 0, 0>;
    return nullptr;
}

StepKernel pick_uniform(uint32_t island_size, uint32_t surface_words, uint32_t model)
{
    if (surface_words > 2) {
        if (model != GA_MODEL_TRAIT) return nullptr;
        switch (island_size) {
        case 16: return pick_uniform_wide<16>(surface_words);
        case 32: return pick_uniform_wide<32>(surface_words);
        case 64: return pick_uniform_wide<64>(surface_words);
        default: return nullptr;
        }
    }
    if (model == GA_MODEL_FITNESS) {
        switch (island_size) {
        case 16: return island_step_kernel<16, 2, 5, 1, 0>;
        case 32: return island_step_kernel<32, 2, 5, 1, 0>;
        case 64: return island_step_kernel<64, 2, 5, 1, 0>;
        default: return nullptr;
        }
    }
    switch (island_size) {
    case 4: return island_step_kernel<4, 2, 5, 0, 0>;
    case 8: return island_step_kernel<8, 2, 5, 0, 0>;
    case 16: return island_step_kernel<16, 2, 5, 0, 0>;
    case 32: return island_step_kernel<32, 2, 5, 0, 0>;
    case 64: return island_step_kernel<64, 2, 5, 0, 0>;
    case 128: return island_step_kernel<128, 2, 5, 0, 0>;
    default: return nullptr;
    }
}

StepKernel pick_kernel(uint32_t island_size, uint32_t surface_words, uint32_t tsize,
                       uint32_t model)
{
    if (model == GA_MODEL_FITNESS) {
        switch (island_size) {
        case 16: return pick_fitness<16>(surface_words, tsize);
        case 32: return pick_fitness<32>(surface_words, tsize);
        case 64: return pick_fitness<64>(surface_words, tsize);
        default: return nullptr;
        }
    }
    if (model != GA_MODEL_TRAIT) return nullptr;
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

// SM count of the current device, read once (a function-local static: initialised once even
// when handles are used from several threads).
uint32_t sm_count()
{
    static const uint32_t sms = [] {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n > 0 ? static_cast<uint32_t>(n) : 1u;
    }();
    return sms;
}

}  // namespace

RunParams run_params(const ga_run *run, const void *src, void *dst, uint32_t g0, uint32_t n_gens,
                     bool migrate)
{
    RunParams r;
    r.src = static_cast<const uint4 *>(src);
    r.dst = static_cast<uint4 *>(dst);
    r.rows = run->cfg.rows;
    r.cols = run->cfg.cols;
    r.n_islands = run->n_islands;
    division_magic(run->cfg.cols, r.cols_m, r.cols_l);
    r.tsize = run->cfg.tournament_size;
    r.theta_ben = run->theta_ben;
    r.theta_del = run->theta_del;
    r.policy = run->cfg.curation;
    r.log2_sites = run->log2_sites;
    r.sites = run->cfg.surface_sites;
    r.bits = run->cfg.differentia_bits;
    r.run_id = run->cfg.run_id;
    r.g0 = g0;
    r.n_gens = n_gens;
    r.migrate = migrate ? 1u : 0u;
    r.gen_sites = run->d_sites + (g0 - run->sites_base);
    r.effect_scale = static_cast<float>(run->cfg.effect_scale);
    r.gen_sites_left = kSiteTableCap - static_cast<uint32_t>(g0 - run->sites_base);
    r.status = run->d_status;
    r.gen_masks = run->d_masks + (g0 - run->sites_base);
    const uint32_t b = run->cfg.differentia_bits;
    r.dif_mask = (1u << b) - 1u;
    r.dif_rep = b == 1u ? 0xFFFFFFFFu : b == 2u ? 0x55555555u : b == 4u ? 0x11111111u : 0x01010101u;
    return r;
}

bool step_supported(uint32_t island_size, uint32_t surface_words, uint32_t model)
{
    return pick_kernel(island_size, surface_words, 1, model) != nullptr;
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

cudaError_t launch_counter_check(ga_run *run, uint32_t generation, int *d_flag)
{
    size_t blocks = (static_cast<size_t>(run->n_agents) + 255) / 256;
    const size_t cap = static_cast<size_t>(sm_count()) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    counter_check_kernel<<<static_cast<unsigned>(blocks), 256, 0, run->stream>>>(
        static_cast<const uint32_t *>(static_cast<const void *>(run->pop[run->cur])),
        run->record_bytes / 4u, run->n_agents, generation, d_flag);
    run->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_island_step(ga_run *run, const void *src, void *dst, uint32_t g0,
                               uint32_t n_gens, bool migrate, cudaStream_t stream)
{
    const bool uniform = run->cfg.mode == GA_SYNC && run->counters_uniform &&
                         run->cfg.tournament_size == 5;
    if (run->cfg.mode == GA_SYNC && run->counters_uniform && run->surface_words <= 2) {
        const uint32_t N = run->cfg.island_size, ts = run->cfg.tournament_size;
        const bool fit = run->cfg.model == GA_MODEL_FITNESS;
        StepKernel ku = nullptr;
        uint32_t islands_per_block = 0;
        switch (N) {
        case 16:
            ku = fit ? (ts == 5 ? island_units_kernel<16, 5, 1> : island_units_kernel<16, 0, 1>)
                     : (ts == 5 ? island_units_kernel<16, 5, 0> : island_units_kernel<16, 0, 0>);
            islands_per_block = units_per_block<16>() * 16;
            break;
        case 32:
            ku = fit ? (ts == 5 ? island_units_kernel<32, 5, 1> : island_units_kernel<32, 0, 1>)
                     : (ts == 5 ? island_units_kernel<32, 5, 0> : island_units_kernel<32, 0, 0>);
            islands_per_block = units_per_block<32>() * 8;
            break;
        case 64:
            ku = fit ? (ts == 5 ? island_units_kernel<64, 5, 1> : island_units_kernel<64, 0, 1>)
                     : (ts == 5 ? island_units_kernel<64, 5, 0> : island_units_kernel<64, 0, 0>);
            islands_per_block = units_per_block<64>() * 8;
            break;
        default: break;
        }
        if (ku) {
            StepArgs a;
            a.r = run_params(run, src, dst, g0, n_gens, migrate);
            a.rk = round_keys(Key{static_cast<uint32_t>(run->cfg.seed),
                                  static_cast<uint32_t>(run->cfg.seed >> 32)});
            const uint32_t blocks = (run->n_islands + islands_per_block - 1) / islands_per_block;
            ku<<<blocks, kStepThreads, 0, stream>>>(a);
            run->launches += 1;
            return cudaGetLastError();
        }
    }
    StepKernel k =
        uniform ? pick_uniform(run->cfg.island_size, run->surface_words, run->cfg.model) : nullptr;
    if (!k)
        k = pick_kernel(run->cfg.island_size, run->surface_words, run->cfg.tournament_size,
                        run->cfg.model);
    if (!k) return cudaErrorInvalidValue;
    StepArgs a;
    a.r = run_params(run, src, dst, g0, n_gens, migrate);
    a.rk = round_keys(Key{static_cast<uint32_t>(run->cfg.seed),
                          static_cast<uint32_t>(run->cfg.seed >> 32)});
    const uint32_t N = run->cfg.island_size;
    const uint32_t islands_per_block = kStepWarps * (N >= 32 ? 1u : 32u / N);
    const uint32_t blocks = (run->n_islands + islands_per_block - 1) / islands_per_block;
    k<<<blocks, kStepThreads, 0, stream>>>(a);
    run->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_site_table(ga_run *run, uint32_t g0, uint32_t count, cudaStream_t stream)
{
    const bool masks = run->surface_words <= 2u;
    const cudaError_t e = launch_curation_sites(
        run->cfg.curation, run->cfg.surface_sites, g0, count, run->d_sites, stream,
        run->cfg.differentia_bits, masks ? run->d_masks : nullptr);
    run->launches += 1;
    return e;
}

cudaError_t launch_curation_sites(uint32_t policy, uint32_t sites, uint32_t t0, uint32_t count,
                                  int32_t *d_sites, cudaStream_t stream, uint32_t bits,
                                  uint2 *d_masks)
{
    if (count == 0) return cudaSuccess;
    uint32_t s = 0;
    while ((1u << s) < sites) ++s;
    uint32_t blocks = (count + 255u) / 256u;
    if (blocks > 8192u) blocks = 8192u;
    curation_sites_kernel<<<blocks, 256, 0, stream>>>(policy, s, sites, t0, count, d_sites, bits,
                                                      d_masks);
    return cudaGetLastError();
}

}  // namespace ga
