// ga_batch.cu -- many independent runs advanced together.
//
// Runs of one batch share each generation's launches: one launch per class (island size,
// record size, tournament size 5 or other, seed) and generation covers every member run of that class, each block
// looking up its run and its unit within the run.  Results are bit-identical to stepping each
// run alone: every draw is keyed by (seed; generation, island, slot, purpose, run_id), and
// the block body is the same as the single-run kernel's.
//
// A chunk of generations is a fixed launch sequence -- the curation-site table of the chunk,
// one launch per class and generation, then a tiny kernel that advances every run's
// generation and buffer parity on the device -- so it is captured once into a CUDA graph and
// replayed; the per-launch generation offset is a kernel parameter, the per-run state lives
// in device descriptors.
//
// Members with 65,536 islands or more (and float-fitness runs) fill the GPU on their own; they
// step with the single-run kernels on the batch's stream instead of joining a class launch.
//
// The autotuner times, on the real member runs (their state is saved and restored around
// the trials), warps per block for each class and the graph's chunk length, and keeps the
// fastest; the choice changes no result.
#include <algorithm>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "ga_device.cuh"
#include "ga_internal.h"
#include "ga_island.cuh"

namespace ga {
namespace {

// Per-run state on the device.  g and cur are the generation and current buffer at the start
// of the chunk being executed; the advance kernel moves them at the end of each chunk.
struct RunDesc {
    const uint4 *pop[2];
    uint32_t rows, cols, n_islands, tsize;
    uint32_t cols_m, cols_l;  // island / cols as a multiply-shift
    uint32_t theta_ben, theta_del, policy, log2_sites;
    uint32_t sites, bits, run_id, per_neighbor;
    uint32_t every_k, g, cur, pad;
    int *status;  // the run's device status word
};

struct BatchArgs {
    const RunDesc *__restrict__ runs;
    const uint32_t *__restrict__ unit_run;    // block -> run index
    const uint32_t *__restrict__ unit_local;  // block -> unit (or chunk of units) within the run
    const int32_t *__restrict__ sites;        // [run][chunk] curation sites of the chunk
    const uint2 *__restrict__ masks;          // [run][chunk] deposit masks (64-bit surfaces)
    uint32_t chunk, dg;                       // chunk length, generation within the chunk
    uint32_t n_runs;
    int *status;                              // the batch's device status word
    RoundKeys rk;
};

// The block's run parameters, staged once in shared memory by thread 0: the block body reads
// them from there (uniform, broadcast) instead of holding them in registers.
__device__ __forceinline__ void stage_params(const BatchArgs &a, RunParams &s_r, uint32_t &s_unit)
{
    if (threadIdx.x == 0) {
        uint32_t run = __ldg(&a.unit_run[blockIdx.x]);
        if (!in_bounds(run < a.n_runs, a.status)) run = 0;
        const RunDesc &d = a.runs[run];
        const uint32_t cur = d.cur ^ (a.dg & 1u);
        s_r.src = d.pop[cur];
        s_r.dst = const_cast<uint4 *>(d.pop[cur ^ 1u]);
        s_r.rows = d.rows;
        s_r.cols = d.cols;
        s_r.n_islands = d.n_islands;
        s_r.cols_m = d.cols_m;
        s_r.cols_l = d.cols_l;
        s_r.tsize = d.tsize;
        s_r.theta_ben = d.theta_ben;
        s_r.theta_del = d.theta_del;
        s_r.policy = d.policy;
        s_r.log2_sites = d.log2_sites;
        s_r.sites = d.sites;
        s_r.bits = d.bits;
        s_r.run_id = d.run_id;
        s_r.g0 = d.g + a.dg;
        s_r.n_gens = 1;
        s_r.migrate = d.per_neighbor && (d.every_k == 1u || s_r.g0 % d.every_k == 0u);
        s_r.gen_sites = a.sites + static_cast<size_t>(run) * a.chunk + a.dg;
        s_r.effect_scale = 1.0f;
        s_r.gen_sites_left = a.chunk - a.dg;
        s_r.status = d.status;
        s_r.gen_masks = a.masks + static_cast<size_t>(run) * a.chunk + a.dg;
        s_r.dif_mask = (1u << d.bits) - 1u;
        s_r.dif_rep = d.bits == 1u ? 0xFFFFFFFFu : d.bits == 2u ? 0x55555555u
                    : d.bits == 4u ? 0x11111111u : 0x01010101u;
        s_unit = __ldg(&a.unit_local[blockIdx.x]);
    }
    __syncthreads();
}

template <int N, int SW, int TS, int W, int CF = 1>
__global__ void __launch_bounds__(W * 32) batch_step_kernel(const BatchArgs a)
{
    __shared__ RunParams s_r;
    __shared__ uint32_t s_unit;
    stage_params(a, s_r, s_unit);
    step_block<N, SW, TS, W, 0, CF>(s_r, a.rk, s_unit);
}

// Classes of 16-byte records whose counters all equal their generation, islands of 16, 32 or
// 64 agents: the multi-unit block body of the single-run kernel (step_units); a block runs a
// chunk of units_per_block<N>() units of one member.
template <int N, int TS>
__global__ void __launch_bounds__(256, (N >= 64 ? 6 : 8)) batch_units_kernel(const BatchArgs a)
{
    __shared__ RunParams s_r;
    __shared__ uint32_t s_unit;
    stage_params(a, s_r, s_unit);
    // the unit loop unrolled for the compiled-in tournament size only: with the run's
    // parameters read from shared memory the unrolled run-time-size body spills (146.6 against
    // 152.2e9 agent-gens/s on the 256-run mix)
    step_units<N, TS, units_per_block<N>(), 0, TS == 5>(s_r, a.rk, s_unit);
}

__global__ void batch_sites_kernel(const RunDesc *__restrict__ runs, uint32_t n_runs,
                                   uint32_t chunk, int32_t *__restrict__ sites,
                                   uint2 *__restrict__ masks)
{
    const uint32_t total = n_runs * chunk;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += gridDim.x * blockDim.x) {
        const RunDesc &d = runs[i / chunk];
        const int site = curation_site(d.policy, d.log2_sites, d.sites, d.g + i % chunk);
        sites[i] = site;
        // deposit masks within surface words 0 and 1 (used by members with 64-bit surfaces)
        const uint32_t pos = site >= 0 ? static_cast<uint32_t>(site) * d.bits : 0u;
        const uint32_t m = (site >= 0 && pos < 64u) ? ((1u << d.bits) - 1u) << (pos & 31u) : 0u;
        masks[i] = make_uint2(pos < 32u ? m : 0u, pos < 32u ? 0u : m);
    }
}

__global__ void batch_advance_kernel(RunDesc *__restrict__ runs, uint32_t n_runs, uint32_t gens)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_runs) {
        runs[i].g += gens;
        runs[i].cur ^= gens & 1u;
    }
}

using BatchKernel = void (*)(BatchArgs);

// Tournament size 5 (the paper's, Sec. 3) has its own instantiations; other sizes use the
// kernels that read the size from the run.  CF = 0: classes whose members' counters all equal
// their generations, compiled without the closed-form curation path (16-byte records only).
template <int N, int SW, int TS, int CF>
BatchKernel pick_w(uint32_t warps)
{
    switch (warps) {
    case 4: return batch_step_kernel<N, SW, TS, 4, CF>;
    case 8: return batch_step_kernel<N, SW, TS, 8, CF>;
    case 16: return batch_step_kernel<N, SW, TS, 16, CF>;
    default: return nullptr;
    }
}

template <int N, int SW, int CF>
BatchKernel pick_ts(uint32_t ts, uint32_t warps)
{
    return ts == 5 ? pick_w<N, SW, 5, CF>(warps) : pick_w<N, SW, 0, CF>(warps);
}

template <int N>
BatchKernel pick_sw(uint32_t sw, uint32_t ts, uint32_t warps, bool uniform)
{
    if constexpr (N >= 16 && N <= 64) {
        if (sw <= 2 && uniform)
            return ts == 5 ? batch_units_kernel<N, 5> : batch_units_kernel<N, 0>;
    }
    if (sw <= 2) return uniform ? pick_ts<N, 2, 0>(ts, warps) : pick_ts<N, 2, 1>(ts, warps);
    if (sw <= 6) return pick_ts<N, 6, 1>(ts, warps);
    if (sw <= 8) return pick_ts<N, 8, 1>(ts, warps);
    return nullptr;
}

BatchKernel pick(uint32_t n, uint32_t sw, uint32_t ts, uint32_t warps, bool uniform = false)
{
    switch (n) {
    case 8: return pick_sw<8>(sw, ts, warps, uniform);
    case 16: return pick_sw<16>(sw, ts, warps, uniform);
    case 32: return pick_sw<32>(sw, ts, warps, uniform);
    case 64: return pick_sw<64>(sw, ts, warps, uniform);
    default: return nullptr;
    }
}

constexpr uint32_t kWarpChoices[] = {4, 8, 16};
constexpr uint32_t kChunkChoices[] = {16, 64, 256};

struct Class {
    uint32_t island_size, sw_class, ts_class;
    uint64_t seed;
    bool uniform = false;  // every member's counters equal its generation (no closed form)
    uint32_t warps = 8;
    // islands one block covers: warps x islands per warp, or for the multi-unit kernel of
    // uniform 16-byte classes (8 warps, fixed) its units per block x islands per unit
    uint32_t per_block() const
    {
        const uint32_t per_warp = island_size >= 32 ? 1u : 32u / island_size;
        if (uniform && sw_class == 2u && island_size >= 16u && island_size <= 64u) {
            const uint32_t units = island_size == 16u ? static_cast<uint32_t>(units_per_block<16>())
                                 : island_size == 32u ? static_cast<uint32_t>(units_per_block<32>())
                                                      : static_cast<uint32_t>(units_per_block<64>());
            return units * 8u * per_warp;
        }
        return warps * per_warp;
    }
    // threads per block of the class's kernel
    uint32_t threads() const
    {
        return (uniform && sw_class == 2u && island_size >= 16u && island_size <= 64u) ? 256u
                                                                                       : warps * 32u;
    }
    std::vector<uint32_t> members;  // indices into the batch's run list
    uint32_t *d_unit_run = nullptr, *d_unit_local = nullptr;
    uint32_t units = 0;
};

uint32_t sw_class(uint32_t surface_words) { return surface_words <= 2 ? 2 : surface_words <= 6 ? 6 : 8; }
uint32_t ts_class(uint32_t tsize) { return tsize == 5 ? 5 : 0; }

// Members this large fill the GPU on their own: they step with the single-run kernels (their
// round keys and parameters in the constant bank) instead of joining a class launch; so do
// asynchronous members and members of a model or island size the batched kernels do not
// cover.
constexpr uint32_t kSoloIslands = 1u << 16;

// Side streams a batch uses at most (classes and solo members beyond this share them).
constexpr size_t kMaxSideStreams = 16;

bool solo(const ga_run *r)
{
    return r->n_islands >= kSoloIslands || r->cfg.model != GA_MODEL_TRAIT ||
           r->cfg.mode != GA_SYNC ||
           !pick(r->cfg.island_size, sw_class(r->surface_words), 0, 8);
}

}  // namespace
}  // namespace ga

struct ga_batch {
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    std::vector<ga_run *> runs;
    // members' (generation, cur, counters uniform) as the device tables hold them
    std::vector<std::tuple<uint64_t, int, bool>> expect;
    std::vector<ga::Class> classes;
    ga::RunDesc *d_runs = nullptr;
    int32_t *d_sites = nullptr;
    uint2 *d_masks = nullptr;  // deposit masks, laid out as d_sites
    uint32_t sites_cap = 0;  // chunk length the site table holds
    uint32_t chunk = 64;
    bool dirty = true;
    cudaGraphExec_t graph = nullptr;
    uint32_t graph_chunk = 0;
    // graphs replaced while a launch of them may still be queued: destroyed at the next
    // host synchronisation of the batch stream
    std::vector<cudaGraphExec_t> retired;
    // side streams: class launches and solo members run on these between a fork from and a
    // join into the batch stream, so independent classes overlap on the GPU
    std::vector<cudaStream_t> side;
    uint64_t launches = 0;
    int *d_status = nullptr;  // device-check builds: failed index checks of the batch tables
};

namespace {

int rc_of(cudaError_t e) { return e == cudaSuccess ? GA_OK : GA_ECUDA; }

// Device tables are allocated and freed in the batch stream's order (the library's memory
// pool, stream-ordered), so a rebuild never waits for the launches already queued: they finish with
// the tables they were given before those are freed.
void free_device(ga_batch *b)
{
    for (auto &c : b->classes) {
        if (c.d_unit_run) ga::pool_free(c.d_unit_run, b->stream);
        if (c.d_unit_local) ga::pool_free(c.d_unit_local, b->stream);
        c.d_unit_run = c.d_unit_local = nullptr;
    }
    if (b->d_runs) ga::pool_free(b->d_runs, b->stream);
    if (b->d_sites) ga::pool_free(b->d_sites, b->stream);
    if (b->d_masks) ga::pool_free(b->d_masks, b->stream);
    b->d_runs = nullptr;
    b->d_sites = nullptr;
    b->d_masks = nullptr;
    b->sites_cap = 0;
    if (b->graph) b->retired.push_back(b->graph);
    b->graph = nullptr;
    b->graph_chunk = 0;
}

// At least `n` side streams (created once, kept until the batch is destroyed).
int ensure_side(ga_batch *b, size_t n)
{
    n = std::min<size_t>(n, ga::kMaxSideStreams);
    while (b->side.size() < n) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return GA_ECUDA;
        b->side.push_back(st);
    }
    return GA_OK;
}

// The first `n` side streams wait for the batch stream's work so far (fork), or the batch
// stream waits for theirs (join); captured as graph dependencies when the batch stream is
// being captured.
cudaError_t fork_join(ga_batch *b, size_t n, bool fork)
{
    n = std::min(n, b->side.size());
    for (size_t i = 0; i < n; ++i) {
        cudaEvent_t ev = nullptr;
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        cudaStream_t from = fork ? b->stream : b->side[i], to = fork ? b->side[i] : b->stream;
        e = cudaEventRecord(ev, from);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(to, ev, 0);
        cudaEventDestroy(ev);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Destroy replaced graphs (the caller has synchronised the batch stream).
void drop_retired(ga_batch *b)
{
    for (cudaGraphExec_t g : b->retired) cudaGraphExecDestroy(g);
    b->retired.clear();
}

// Make `waiter` wait, on the device, for the work queued on `from` so far (no host wait).
cudaError_t order_after(cudaStream_t waiter, cudaStream_t from)
{
    if (waiter == from) return cudaSuccess;
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev, from);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(waiter, ev, 0);
    cudaEventDestroy(ev);
    return e;
}

// (Re)build classes, descriptors and block tables after membership or tuning changes.
int rebuild(ga_batch *b)
{
    using Key = std::tuple<uint32_t, uint32_t, uint32_t, uint64_t, bool>;
    std::map<Key, uint32_t> warps_of;
    for (const auto &c : b->classes)
        warps_of[{c.island_size, c.sw_class, c.ts_class, c.seed, c.uniform}] = c.warps;
    free_device(b);
    b->classes.clear();
    std::map<Key, size_t> index;
    for (uint32_t i = 0; i < b->runs.size(); ++i) {
        const ga_run *r = b->runs[i];
        if (ga::solo(r)) continue;
        const uint32_t swc = ga::sw_class(r->surface_words);
        const Key key = std::make_tuple(r->cfg.island_size, swc,
                                        ga::ts_class(r->cfg.tournament_size), r->cfg.seed,
                                        swc == 2u && r->counters_uniform);
        auto it = index.find(key);
        if (it == index.end()) {
            ga::Class c;
            c.island_size = std::get<0>(key);
            c.sw_class = std::get<1>(key);
            c.ts_class = std::get<2>(key);
            c.seed = std::get<3>(key);
            c.uniform = std::get<4>(key);
            auto w = warps_of.find(key);
            if (w != warps_of.end()) c.warps = w->second;
            index[key] = b->classes.size();
            b->classes.push_back(c);
            it = index.find(key);
        }
        b->classes[it->second].members.push_back(i);
    }
    const size_t n = b->runs.size();
    if (n == 0) {
        b->dirty = false;
        return GA_OK;
    }
    std::vector<ga::RunDesc> desc(n);
    for (size_t i = 0; i < n; ++i) {
        const ga_run *r = b->runs[i];
        ga::RunDesc &d = desc[i];
        d.pop[0] = reinterpret_cast<const uint4 *>(r->pop[0]);
        d.pop[1] = reinterpret_cast<const uint4 *>(r->pop[1]);
        d.rows = r->cfg.rows;
        d.cols = r->cfg.cols;
        d.n_islands = r->n_islands;
        ga::division_magic(r->cfg.cols, d.cols_m, d.cols_l);
        d.tsize = r->cfg.tournament_size;
        d.theta_ben = r->theta_ben;
        d.theta_del = r->theta_del;
        d.policy = r->cfg.curation;
        d.log2_sites = r->log2_sites;
        d.sites = r->cfg.surface_sites;
        d.bits = r->cfg.differentia_bits;
        d.run_id = r->cfg.run_id;
        d.per_neighbor = r->per_neighbor;
        d.every_k = r->every_k;
        d.g = static_cast<uint32_t>(r->generation);
        d.cur = static_cast<uint32_t>(r->cur);
        d.pad = 0;
        d.status = r->d_status;
    }
    // pageable host sources: each copy is staged before the call returns, so the host vectors
    // may go out of scope without a wait
    if (ga::pool_alloc(reinterpret_cast<void **>(&b->d_runs), n * sizeof(ga::RunDesc), b->stream) !=
        cudaSuccess)
        return GA_ENOMEM;
    int rc = rc_of(cudaMemcpyAsync(b->d_runs, desc.data(), n * sizeof(ga::RunDesc),
                                   cudaMemcpyHostToDevice, b->stream));
    if (rc != GA_OK) return rc;
    for (auto &c : b->classes) {
        const uint32_t per_block = c.per_block();
        std::vector<uint32_t> ur, ul;
        for (uint32_t m : c.members) {
            const uint32_t units = (b->runs[m]->n_islands + per_block - 1) / per_block;
            for (uint32_t u = 0; u < units; ++u) {
                ur.push_back(m);
                ul.push_back(u);
            }
        }
        c.units = static_cast<uint32_t>(ur.size());
        if (ga::pool_alloc(reinterpret_cast<void **>(&c.d_unit_run), ur.size() * 4, b->stream) !=
                cudaSuccess ||
            ga::pool_alloc(reinterpret_cast<void **>(&c.d_unit_local), ul.size() * 4, b->stream) !=
                cudaSuccess)
            return GA_ENOMEM;
        rc = rc_of(cudaMemcpyAsync(c.d_unit_run, ur.data(), ur.size() * 4, cudaMemcpyHostToDevice,
                                   b->stream));
        if (rc == GA_OK)
            rc = rc_of(cudaMemcpyAsync(c.d_unit_local, ul.data(), ul.size() * 4,
                                       cudaMemcpyHostToDevice, b->stream));
        if (rc != GA_OK) return rc;
    }
    b->expect.clear();
    for (const ga_run *r : b->runs) b->expect.emplace_back(r->generation, r->cur, r->counters_uniform);
    b->dirty = false;
    return GA_OK;
}

// A member stepped, reset or loaded outside the batch no longer matches the descriptors.
bool members_moved(const ga_batch *b)
{
    if (b->expect.size() != b->runs.size()) return true;
    for (size_t i = 0; i < b->runs.size(); ++i)
        if (b->expect[i] != std::make_tuple(b->runs[i]->generation, b->runs[i]->cur,
                                            b->runs[i]->counters_uniform))
            return true;
    return false;
}

int ensure_sites(ga_batch *b, uint32_t chunk)
{
    if (b->sites_cap >= chunk) return GA_OK;
    if (b->d_sites) ga::pool_free(b->d_sites, b->stream);
    if (b->d_masks) ga::pool_free(b->d_masks, b->stream);
    b->d_sites = nullptr;
    b->d_masks = nullptr;
    const size_t entries = b->runs.size() * static_cast<size_t>(chunk);
    if (ga::pool_alloc(reinterpret_cast<void **>(&b->d_sites), entries * sizeof(int32_t), b->stream) !=
            cudaSuccess ||
        ga::pool_alloc(reinterpret_cast<void **>(&b->d_masks), entries * sizeof(uint2), b->stream) !=
            cudaSuccess)
        return GA_ENOMEM;
    b->sites_cap = chunk;
    return GA_OK;
}

// Enqueue one chunk of `gens` generations for every member run (no host synchronisation).
// Classes share no run, so each class's launches go to its own side stream between a fork
// after the site table and a join before the generation advance: the classes' launches of a
// generation overlap on the GPU.
int enqueue_chunk(ga_batch *b, uint32_t gens)
{
    const uint32_t n = static_cast<uint32_t>(b->runs.size());
    ga::batch_sites_kernel<<<std::min<uint32_t>((n * gens + 255) / 256, 4096), 256, 0, b->stream>>>(
        b->d_runs, n, gens, b->d_sites, b->d_masks);
    b->launches += 1;
    if (ensure_side(b, b->classes.size()) != GA_OK) return GA_ECUDA;
    if (fork_join(b, b->classes.size(), true) != cudaSuccess) return GA_ECUDA;
    for (uint32_t dg = 0; dg < gens; ++dg) {
        for (size_t ci = 0; ci < b->classes.size(); ++ci) {
            const auto &c = b->classes[ci];
            cudaStream_t st = b->side[ci % b->side.size()];
            const ga::BatchKernel k =
                ga::pick(c.island_size, c.sw_class, c.ts_class, c.warps, c.uniform);
            if (!k) return GA_EUNSUPPORTED;
            ga::BatchArgs a;
            a.runs = b->d_runs;
            a.unit_run = c.d_unit_run;
            a.unit_local = c.d_unit_local;
            a.sites = b->d_sites;
            a.masks = b->d_masks;
            a.chunk = gens;
            a.dg = dg;
            a.n_runs = n;
            a.status = b->d_status;
            a.rk = ga::round_keys(ga::Key{static_cast<uint32_t>(c.seed), static_cast<uint32_t>(c.seed >> 32)});
            k<<<c.units, c.threads(), 0, st>>>(a);
            b->launches += 1;
        }
    }
    if (fork_join(b, b->classes.size(), false) != cudaSuccess) return GA_ECUDA;
    ga::batch_advance_kernel<<<(n + 255) / 256, 256, 0, b->stream>>>(b->d_runs, n, gens);
    b->launches += 1;
    return rc_of(cudaGetLastError());
}

int capture_graph(ga_batch *b, uint32_t chunk)
{
    if (b->graph && b->graph_chunk == chunk) return GA_OK;
    if (b->graph) b->retired.push_back(b->graph);
    b->graph = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return GA_ECUDA;
    const uint64_t before = b->launches;
    const int rc = enqueue_chunk(b, chunk);
    const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    b->launches = before;  // captured, not launched
    if (rc != GA_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc != GA_OK ? rc : GA_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        b->graph = nullptr;
        return GA_ECUDA;
    }
    b->graph_chunk = chunk;
    return GA_OK;
}

uint64_t chunk_launches(const ga_batch *b, uint32_t chunk)
{
    return 2 + static_cast<uint64_t>(chunk) * b->classes.size();
}

int step_device(ga_batch *b, uint32_t n_gens)
{
    if (b->classes.empty()) return GA_OK;
    int rc = GA_OK;
    uint32_t left = n_gens;
    if (left >= b->chunk) {
        rc = ensure_sites(b, b->chunk);
        if (rc == GA_OK) rc = capture_graph(b, b->chunk);
        while (rc == GA_OK && left >= b->chunk) {
            rc = rc_of(cudaGraphLaunch(b->graph, b->stream));
            b->launches += chunk_launches(b, b->chunk);
            left -= b->chunk;
        }
    }
    if (rc == GA_OK && left > 0) {
        rc = ensure_sites(b, left);
        if (rc == GA_OK) rc = enqueue_chunk(b, left);
    }
    return rc;
}

void advance_host(ga_batch *b, uint32_t n_gens)
{
    for (size_t i = 0; i < b->runs.size(); ++i) {
        ga_run *r = b->runs[i];
        if (!ga::solo(r)) {  // solo members were advanced by their own steps
            r->generation += n_gens;
            r->cur ^= static_cast<int>(n_gens & 1u);
            r->launches += n_gens;  // one island-step launch per generation covers each run
        }
        b->expect[i] = std::make_tuple(r->generation, r->cur, r->counters_uniform);
    }
}

}  // namespace

extern "C" {

int ga_batch_create(void *stream, ga_batch **out)
{
    if (!out) return GA_EINVAL;
    *out = nullptr;
    ga_batch *b = new (std::nothrow) ga_batch();
    if (!b) return GA_ENOMEM;
    if (stream) {
        b->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return GA_ECUDA;
        }
        b->owns_stream = true;
    }
    if (cudaMalloc(&b->d_status, sizeof(int)) != cudaSuccess ||
        cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream) != cudaSuccess) {
        cudaGetLastError();
        if (b->d_status) cudaFree(b->d_status);
        if (b->owns_stream) cudaStreamDestroy(b->stream);
        delete b;
        return GA_ENOMEM;
    }
    *out = b;
    return GA_OK;
}

int ga_batch_add(ga_batch *b, ga_run *run)
{
    if (!b || !run) return GA_EINVAL;
    if (run->batch) return GA_EINVAL;  // already a member of this or another batch

    if (run->generation + 1 > 0xFFFFFFFFull) return GA_EINVAL;
    // the run's own queued work comes before anything the batch stream does to its buffers
    if (order_after(b->stream, run->stream) != cudaSuccess) return GA_ECUDA;
    b->runs.push_back(run);
    run->batch = b;
    b->dirty = true;
    return GA_OK;
}

int ga_batch_remove(ga_batch *b, ga_run *run)
{
    if (!b || !run) return GA_EINVAL;
    auto it = std::find(b->runs.begin(), b->runs.end(), run);
    if (it == b->runs.end()) return GA_EINVAL;
    // work queued on the run's own stream from now on (and ga_destroy's wait) comes after the
    // batch's launches that still step it; the run leaves the batch even if that fails
    const int rc = rc_of(order_after(run->stream, b->stream));
    b->runs.erase(it);
    run->batch = nullptr;
    b->dirty = true;
    return rc;
}

int ga_batch_size(const ga_batch *b, uint32_t *n_runs)
{
    if (!b || !n_runs) return GA_EINVAL;
    *n_runs = static_cast<uint32_t>(b->runs.size());
    return GA_OK;
}

int ga_batch_step(ga_batch *b, uint32_t n_gens)
{
    if (!b) return GA_EINVAL;
    if (b->runs.empty() || n_gens == 0) return GA_OK;
    for (const ga_run *r : b->runs)
        if (r->generation + n_gens > 0xFFFFFFFFull) return GA_EINVAL;
    if (b->dirty || members_moved(b)) {
        // members' own streams may still hold work queued outside the batch
        for (const ga_run *r : b->runs)
            if (order_after(b->stream, r->stream) != cudaSuccess) return GA_ECUDA;
        const int rc = rebuild(b);
        if (rc != GA_OK) return rc;
    }
    // solo members on side streams of their own (forked from and joined into the batch
    // stream), overlapping one another and the class launches
    // (class launches use side streams 0..C-1, solo members the ones after them)
    size_t n_solo = 0;
    for (const ga_run *r : b->runs) n_solo += ga::solo(r) ? 1u : 0u;
    const size_t n_side = b->classes.size() + n_solo;
    if (n_solo > 0) {
        if (ensure_side(b, n_side) != GA_OK) return GA_ECUDA;
        if (fork_join(b, n_side, true) != cudaSuccess) return GA_ECUDA;
        size_t k = b->classes.size();
        for (ga_run *r : b->runs) {
            if (!ga::solo(r)) continue;
            const int rs = ga::step_run(r, n_gens, b->side[k++ % b->side.size()]);
            if (rs != GA_OK) return rs;
        }
    }
    const int rc = step_device(b, n_gens);
    if (n_solo > 0 && fork_join(b, n_side, false) != cudaSuccess) return GA_ECUDA;
    if (rc != GA_OK) return rc;
    advance_host(b, n_gens);
    return GA_OK;
}

int ga_batch_sync(ga_batch *b)
{
    if (!b) return GA_EINVAL;
    int rc = rc_of(cudaStreamSynchronize(b->stream));
    if (rc == GA_OK) drop_retired(b);
#if GA_DEVICE_CHECKS
    // only device-check builds write the batch's status word
    int st = GA_OK;
    if (rc == GA_OK && cudaMemcpy(&st, b->d_status, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = GA_ECUDA;
    if (rc == GA_OK && st != GA_OK) {
        cudaMemset(b->d_status, 0, sizeof(int));
        rc = st;
    }
#endif
    return rc;
}

int ga_batch_launch_count(const ga_batch *b, uint64_t *launches)
{
    if (!b || !launches) return GA_EINVAL;
    *launches = b->launches;
    return GA_OK;
}

int ga_batch_autotune(ga_batch *b, uint32_t trial_gens, uint32_t *chosen_chunk)
{
    if (!b || trial_gens == 0) return GA_EINVAL;
    if (b->runs.empty()) return GA_OK;
    if (b->dirty) {
        const int rc = rebuild(b);
        if (rc != GA_OK) return rc;
    }
    // save every run's current buffer so the trials leave no trace
    std::vector<void *> saved(b->runs.size(), nullptr);
    int rc = GA_OK;
    for (size_t i = 0; i < b->runs.size() && rc == GA_OK; ++i) {
        ga_run *r = b->runs[i];
        const size_t bytes = static_cast<size_t>(r->n_agents) * r->record_bytes;
        if (cudaMalloc(&saved[i], bytes) != cudaSuccess) rc = GA_ENOMEM;
        else rc = rc_of(cudaMemcpyAsync(saved[i], r->pop[r->cur], bytes, cudaMemcpyDeviceToDevice, b->stream));
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == GA_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = GA_ECUDA;
    auto restore = [&]() {
        for (size_t i = 0; i < b->runs.size(); ++i) {
            ga_run *r = b->runs[i];
            if (saved[i])
                cudaMemcpyAsync(r->pop[r->cur], saved[i], static_cast<size_t>(r->n_agents) * r->record_bytes,
                                cudaMemcpyDeviceToDevice, b->stream);
        }
        b->dirty = true;  // descriptors back to the runs' (unchanged) host state
    };
    auto timed = [&](uint32_t gens, float *ms) -> int {
        int r2 = rebuild(b);
        if (r2 != GA_OK) return r2;
        r2 = step_device(b, gens);  // warm (graph capture, caches)
        if (r2 != GA_OK) return r2;
        if (cudaEventRecord(e0, b->stream) != cudaSuccess) return GA_ECUDA;
        r2 = step_device(b, gens);
        if (r2 != GA_OK) return r2;
        if (cudaEventRecord(e1, b->stream) != cudaSuccess) return GA_ECUDA;
        if (cudaEventSynchronize(e1) != cudaSuccess) return GA_ECUDA;
        return rc_of(cudaEventElapsedTime(ms, e0, e1));
    };
    const uint32_t saved_chunk = b->chunk;
    // warps per block, class by class (the others held at their current choice)
    b->chunk = trial_gens;
    for (size_t ci = 0; ci < b->classes.size() && rc == GA_OK; ++ci) {
        float best = 3.4e38f;
        uint32_t best_w = b->classes[ci].warps;
        for (uint32_t w : ga::kWarpChoices) {
            b->classes[ci].warps = w;
            float ms = 0.f;
            rc = timed(trial_gens, &ms);
            restore();
            if (rc != GA_OK) break;
            if (ms < best) {
                best = ms;
                best_w = w;
            }
        }
        b->classes[ci].warps = best_w;
    }
    // graph chunk length
    uint32_t best_chunk = saved_chunk;
    if (rc == GA_OK) {
        float best = 3.4e38f;
        for (uint32_t c : ga::kChunkChoices) {
            b->chunk = c;
            float ms = 0.f;
            rc = timed(c, &ms);
            restore();
            if (rc != GA_OK) break;
            if (ms / c < best) {
                best = ms / c;
                best_chunk = c;
            }
        }
    }
    b->chunk = best_chunk;
    if (chosen_chunk) *chosen_chunk = best_chunk;
    cudaStreamSynchronize(b->stream);
    drop_retired(b);
    for (void *p : saved) cudaFree(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    b->dirty = true;
    return rc;
}

int ga_batch_class_warps(const ga_batch *b, uint32_t index, uint32_t *island_size,
                         uint32_t *warps)
{
    if (!b || !island_size || !warps || index >= b->classes.size()) return GA_EINVAL;
    *island_size = b->classes[index].island_size;
    *warps = b->classes[index].warps;
    return GA_OK;
}

int ga_batch_destroy(ga_batch *b)
{
    if (!b) return GA_EINVAL;
    int rc = rc_of(cudaStreamSynchronize(b->stream));
    for (ga_run *r : b->runs) r->batch = nullptr;
    free_device(b);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) rc = GA_ECUDA;
    drop_retired(b);
    for (cudaStream_t st : b->side) cudaStreamDestroy(st);
    cudaFree(b->d_status);
    if (b->owns_stream) cudaStreamDestroy(b->stream);
    delete b;
    return rc;
}

}  // extern "C"
