// ga_api.cu -- the C ABI declared in include/ga.h: configuration checks, workspace layout,
// generation scheduling (which launches cover which generations), snapshots and the MRCA
// entry points.  All arithmetic of the method runs in the kernels of ga_step.cu/ga_mrca.cu.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "ga_internal.h"

namespace {

bool is_pow2(uint32_t v) { return v != 0u && (v & (v - 1u)) == 0u; }

uint32_t log2_exact(uint32_t v)
{
    uint32_t s = 0;
    while ((1u << s) < v) ++s;
    return s;
}

// Mutation probability -> 32-bit threshold, once on the host: min(2^32 - 1, floor(p 2^32)).
uint32_t threshold(double p)
{
    double x = std::floor(p * 4294967296.0);
    if (x < 0.0) x = 0.0;
    if (x > 4294967295.0) x = 4294967295.0;
    return static_cast<uint32_t>(x);
}

uint32_t surface_words_of(const ga_config *c)
{
    return (c->surface_sites * c->differentia_bits + 31u) / 32u;
}

uint32_t record_bytes_of(const ga_config *c)
{
    return (8u + 4u * surface_words_of(c) + 15u) / 16u * 16u;
}

int check_config(const ga_config *c)
{
    if (!c) return GA_EINVAL;
    if (c->rows == 0 || c->cols == 0) return GA_EINVAL;
    if (!is_pow2(c->island_size) || c->island_size < 4 || c->island_size > 256) return GA_EINVAL;
    if (c->tournament_size < 1 || c->tournament_size > 8) return GA_EINVAL;
    if (!(c->p_ben >= 0.0) || !(c->p_del >= 0.0) || c->p_ben + c->p_del > 1.0) return GA_EINVAL;
    const uint32_t b = c->differentia_bits;
    if (!(b == 1 || b == 2 || b == 4 || b == 8)) return GA_EINVAL;
    if (!is_pow2(c->surface_sites)) return GA_EINVAL;
    if (c->curation > GA_HYBRID) return GA_EINVAL;
    if (c->surface_sites < (c->curation == GA_HYBRID ? 8u : 4u)) return GA_EINVAL;
    if (static_cast<uint64_t>(c->surface_sites) * b > 256u) return GA_EINVAL;
    if (c->mode > GA_ASYNC_SEQUENTIAL || c->model > GA_MODEL_FITNESS) return GA_EINVAL;
    if (c->model == GA_MODEL_FITNESS && !(c->effect_scale > 0.0 && c->effect_scale < 1e30))
        return GA_EINVAL;
    const uint64_t agents = static_cast<uint64_t>(c->rows) * c->cols * c->island_size;
    if (agents > 0xFFFFFFFFull) return GA_EINVAL;
    if (!ga::step_supported(c->island_size, surface_words_of(c), c->model)) return GA_EUNSUPPORTED;
    if (c->mode != GA_SYNC && !ga::async_supported(c->island_size, surface_words_of(c), c->model))
        return GA_EUNSUPPORTED;
    return GA_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

size_t population_bytes(const ga_config *c)
{
    return static_cast<size_t>(c->rows) * c->cols * c->island_size * record_bytes_of(c);
}

size_t buffer_stride(const ga_config *c) { return align_up(population_bytes(c), 256); }

// Workspace: header, two population buffers, then the send buffers (asynchronous modes) or
// the resident mailboxes (synchronous runs small enough to step resident).
size_t workspace_need(const ga_config *c)
{
    size_t need = ga::kHeaderBytes + 2 * buffer_stride(c);
    if (c->mode != GA_SYNC) need += ga::async_state_bytes(c->rows * c->cols, record_bytes_of(c));
    else need += ga::resident_state_bytes(c->rows * c->cols, record_bytes_of(c));
    return need;
}

// Empty every send buffer (asynchronous modes).
int clear_async_state(ga_run *run)
{
    if (!run->mail) return GA_OK;
    return ga::async_clear(run, run->stream) == cudaSuccess ? GA_OK : GA_ECUDA;
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? GA_OK : GA_ECUDA; }

// Read and clear the device error word (the caller has synchronised the stream).
int take_status(ga_run *run)
{
    int st = GA_OK;
    if (cudaMemcpy(&st, run->d_status, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess)
        return GA_ECUDA;
    if (st != GA_OK) {
        const int zero = GA_OK;
        if (cudaMemcpy(run->d_status, &zero, sizeof zero, cudaMemcpyHostToDevice) != cudaSuccess)
            return GA_ECUDA;
    }
    return st;
}

}  // namespace

namespace ga {

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t stream)
{
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaMallocAsync(p, bytes, stream);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t created;
            e = cudaMemPoolCreate(&created, &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = kPoolKeepBytes;
            e = cudaMemPoolSetAttribute(created, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) {
                cudaMemPoolDestroy(created);
                return e;
            }
            pools[dev] = created;
        }
        pool = pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, stream);
}

int step_run(ga_run *run, uint32_t n_gens, cudaStream_t stream)
{
    if (run->cfg.mode != GA_SYNC) return async_step(run, n_gens, stream);
    if (run->generation + n_gens > 0xFFFFFFFFull) return GA_EINVAL;
    // resident launches: one cooperative launch per chunk of the site table
    bool resident = false;
    if (n_gens > 0 && run->resident_mode != GA_RESIDENT_OFF) {
        const bool wanted = run->resident_mode == GA_RESIDENT_ON || run->n_islands <= kResidentAutoIslands;
        resident = wanted && resident_possible(run, nullptr);
        if (run->resident_mode == GA_RESIDENT_ON && !resident) return GA_EUNSUPPORTED;
    }
    while (n_gens > 0) {
        // curation sites of the next chunk of generations, computed on the device once
        const uint32_t chunk = n_gens < kSiteTableCap ? n_gens : kSiteTableCap;
        int rc = cuda_rc(launch_site_table(run, static_cast<uint32_t>(run->generation), chunk, stream));
        if (rc != GA_OK) return rc;
        run->sites_base = run->generation;
        if (resident) {
            rc = cuda_rc(launch_resident(run, run->pop[run->cur], run->pop[run->cur ^ 1],
                                         static_cast<uint32_t>(run->generation), chunk, stream));
            if (rc != GA_OK) return rc;
            run->cur ^= 1;
            run->generation += chunk;
            n_gens -= chunk;
            continue;
        }
        uint32_t left = chunk;
        while (left > 0) {
            const uint64_t g = run->generation;
            uint64_t len = left;
            bool migrate = false;
            if (run->per_neighbor) {
                migrate = (g % run->every_k) == 0;
                const uint64_t next = (g / run->every_k + 1) * run->every_k;
                if (next - g < len) len = next - g;
            }
            if (len > kMaxGensPerLaunch) len = kMaxGensPerLaunch;
            rc = cuda_rc(launch_island_step(run, run->pop[run->cur], run->pop[run->cur ^ 1],
                                            static_cast<uint32_t>(g), static_cast<uint32_t>(len),
                                            migrate, stream));
            if (rc != GA_OK) return rc;
            run->cur ^= 1;
            run->generation += len;
            left -= static_cast<uint32_t>(len);
        }
        n_gens -= chunk;
    }
    return GA_OK;
}

}  // namespace ga

extern "C" {

int ga_config_default(ga_config *cfg)
{
    if (!cfg) return GA_EINVAL;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->rows = 32;
    cfg->cols = 32;
    cfg->island_size = 32;
    cfg->tournament_size = 5;
    cfg->p_ben = 0.01;
    cfg->p_del = 0.01;
    cfg->surface_sites = 64;
    cfg->differentia_bits = 1;
    cfg->curation = GA_STEADY;
    cfg->mode = GA_SYNC;
    cfg->seed = 42;
    cfg->run_id = 0;
    cfg->model = GA_MODEL_TRAIT;
    cfg->stream = nullptr;
    cfg->effect_scale = 1.0;
    return GA_OK;
}

int ga_config_check(const ga_config *cfg) { return check_config(cfg); }

int ga_record_bytes(const ga_config *cfg, uint32_t *bytes)
{
    if (!cfg || !bytes) return GA_EINVAL;
    const int rc = check_config(cfg);
    if (rc == GA_EINVAL) return rc;
    *bytes = record_bytes_of(cfg);
    return GA_OK;
}

int ga_workspace_bytes(const ga_config *cfg, size_t *bytes)
{
    if (!cfg || !bytes) return GA_EINVAL;
    const int rc = check_config(cfg);
    if (rc != GA_OK) return rc;
    *bytes = workspace_need(cfg);
    return GA_OK;
}

int ga_create(const ga_config *cfg, void *workspace, size_t workspace_bytes, ga_run **out)
{
    if (!out) return GA_EINVAL;
    *out = nullptr;
    int rc = check_config(cfg);
    if (rc != GA_OK) return rc;
    const size_t need = workspace_need(cfg);
    if (workspace) {
        if (workspace_bytes < need) return GA_ENOMEM;
        if (reinterpret_cast<uintptr_t>(workspace) % 256u != 0u) return GA_EINVAL;
    }
    ga_run *run = new (std::nothrow) ga_run();
    if (!run) return GA_ENOMEM;
    run->cfg = *cfg;
    run->stream = static_cast<cudaStream_t>(cfg->stream);
    run->n_islands = cfg->rows * cfg->cols;
    run->n_agents = run->n_islands * cfg->island_size;
    run->record_bytes = record_bytes_of(cfg);
    run->surface_words = surface_words_of(cfg);
    run->log2_sites = log2_exact(cfg->surface_sites);
    run->theta_ben = threshold(cfg->p_ben);
    run->theta_del = threshold(cfg->p_del);
    run->per_neighbor = 1;
    run->every_k = 1;
    run->generation = 0;
    run->launches = 0;
    if (workspace) {
        run->workspace = workspace;
        run->owns_workspace = false;
        run->workspace_bytes = workspace_bytes;
    } else {
        if (cudaMalloc(&run->workspace, need) != cudaSuccess) {
            cudaGetLastError();
            delete run;
            return GA_ENOMEM;
        }
        run->owns_workspace = true;
        run->workspace_bytes = need;
    }
    uint8_t *base = static_cast<uint8_t *>(run->workspace);
    run->d_status = reinterpret_cast<int *>(base);
    run->d_flag = reinterpret_cast<int *>(base + ga::kStatusBytes / 2);
    run->d_sites = reinterpret_cast<int32_t *>(base + ga::kStatusBytes);
    run->d_masks = reinterpret_cast<uint2 *>(base + ga::kMaskOffset);
    run->resident_state = nullptr;
    if (cfg->mode == GA_SYNC &&
        ga::resident_state_bytes(run->n_islands, run->record_bytes) != 0)
        run->resident_state = base + ga::kHeaderBytes + 2 * buffer_stride(cfg);
    run->resident_mode = GA_RESIDENT_AUTO;
    run->resident_wait_us = 1000000u;
    run->drop_island = 0xFFFFFFFFu;
    run->sites_base = 0;
    run->pop[0] = base + ga::kHeaderBytes;
    run->pop[1] = base + ga::kHeaderBytes + buffer_stride(cfg);
    run->cur = 0;
    run->mail = nullptr;
    run->async_window = 1;
    run->batch = nullptr;
    run->counters_uniform = true;
    if (cfg->mode != GA_SYNC) run->mail = base + ga::kHeaderBytes + 2 * buffer_stride(cfg);
    rc = cuda_rc(cudaMemsetAsync(base, 0, ga::kHeaderBytes, run->stream));
    if (rc == GA_OK) rc = clear_async_state(run);
    if (rc == GA_OK) rc = cuda_rc(ga::launch_founder(run, run->pop[0]));
    if (rc != GA_OK) {
        if (run->owns_workspace) cudaFree(run->workspace);
        delete run;
        return rc;
    }
    *out = run;
    return GA_OK;
}

int ga_reset(ga_run *run)
{
    if (!run) return GA_EINVAL;
    run->cur = 0;
    run->generation = 0;
    run->counters_uniform = true;
    const int rc = clear_async_state(run);
    if (rc != GA_OK) return rc;
    return cuda_rc(ga::launch_founder(run, run->pop[0]));
}

int ga_migrate_policy(ga_run *run, uint32_t per_neighbor, uint32_t every_k)
{
    if (!run || per_neighbor > 1u || every_k == 0u) return GA_EINVAL;
    run->per_neighbor = per_neighbor;
    run->every_k = every_k;
    return GA_OK;
}

int ga_async_window(ga_run *run, uint32_t window)
{
    if (!run || window == 0u || window > GA_ASYNC_MAX_WINDOW) return GA_EINVAL;
    if (run->cfg.mode == GA_SYNC) return GA_ESTATE;
    run->async_window = window;
    return GA_OK;
}

int ga_resident_policy(ga_run *run, uint32_t mode, uint32_t wait_limit_us)
{
    if (!run || mode > GA_RESIDENT_ON || wait_limit_us == 0u) return GA_EINVAL;
    run->resident_mode = mode;
    run->resident_wait_us = wait_limit_us;
    return GA_OK;
}

int ga_inject_lost_migrants(ga_run *run, uint32_t island)
{
    if (!run || (island != 0xFFFFFFFFu && island >= run->n_islands)) return GA_EINVAL;
    run->drop_island = island;
    return GA_OK;
}

int ga_step(ga_run *run, uint32_t n_gens)
{
    if (!run) return GA_EINVAL;
    return ga::step_run(run, n_gens, run->stream);
}

int ga_sync(ga_run *run)
{
    if (!run) return GA_EINVAL;
    if (cudaStreamSynchronize(run->stream) != cudaSuccess) return GA_ECUDA;
    return take_status(run);
}

int ga_generation(const ga_run *run, uint64_t *generation)
{
    if (!run || !generation) return GA_EINVAL;
    *generation = run->generation;
    return GA_OK;
}

int ga_launch_count(const ga_run *run, uint64_t *launches)
{
    if (!run || !launches) return GA_EINVAL;
    *launches = run->launches;
    return GA_OK;
}

int ga_population(ga_run *run, void **device_ptr, size_t *bytes)
{
    if (!run || !device_ptr || !bytes) return GA_EINVAL;
    *device_ptr = run->pop[run->cur];
    *bytes = population_bytes(&run->cfg);
    return GA_OK;
}

int ga_snapshot(ga_run *run, void *host_dst, size_t cap, size_t *written)
{
    if (!run || !host_dst) return GA_EINVAL;
    const size_t need = population_bytes(&run->cfg);
    if (written) *written = need;
    if (cap < need) return GA_ERANGE;
    if (cudaMemcpyAsync(host_dst, run->pop[run->cur], need, cudaMemcpyDeviceToHost,
                        run->stream) != cudaSuccess)
        return GA_ECUDA;
    if (cudaStreamSynchronize(run->stream) != cudaSuccess) return GA_ECUDA;
    return take_status(run);
}

int ga_snapshot_device(ga_run *run, void *device_dst, size_t cap, size_t *written)
{
    if (!run || !device_dst) return GA_EINVAL;
    const size_t need = population_bytes(&run->cfg);
    if (written) *written = need;
    if (cap < need) return GA_ERANGE;
    return cuda_rc(cudaMemcpyAsync(device_dst, run->pop[run->cur], need,
                                   cudaMemcpyDeviceToDevice, run->stream));
}

int ga_load(ga_run *run, const void *host_src, size_t bytes, uint64_t generation)
{
    if (!run || !host_src) return GA_EINVAL;
    if (bytes != population_bytes(&run->cfg) || generation > 0xFFFFFFFFull) return GA_EINVAL;
    if (run->cfg.mode != GA_SYNC) {
        // counter 2^32 - 1 is reserved in the asynchronous modes (it marks an empty buffer)
        const uint8_t *rec = static_cast<const uint8_t *>(host_src);
        for (uint32_t a = 0; a < run->n_agents; ++a) {
            uint32_t c;
            std::memcpy(&c, rec + static_cast<size_t>(a) * run->record_bytes + 4, sizeof c);
            if (c == 0xFFFFFFFFu) return GA_EINVAL;
        }
    }
    if (cudaMemcpyAsync(run->pop[run->cur], host_src, bytes, cudaMemcpyHostToDevice,
                        run->stream) != cudaSuccess)
        return GA_ECUDA;
    if (clear_async_state(run) != GA_OK) return GA_ECUDA;
    // do all loaded counters equal the generation?  (synchronous steps then skip the
    // closed-form curation path)
    int mixed = 1;
    if (run->cfg.mode == GA_SYNC) {
        if (cudaMemsetAsync(run->d_flag, 0, sizeof(int), run->stream) != cudaSuccess ||
            ga::launch_counter_check(run, static_cast<uint32_t>(generation), run->d_flag) !=
                cudaSuccess ||
            cudaMemcpyAsync(&mixed, run->d_flag, sizeof(int), cudaMemcpyDeviceToHost,
                            run->stream) != cudaSuccess)
            return GA_ECUDA;
    }
    if (cudaStreamSynchronize(run->stream) != cudaSuccess) return GA_ECUDA;
    run->generation = generation;
    run->counters_uniform = mixed == 0;
    return GA_OK;
}

int ga_mrca_bounds_device(ga_run *run, const uint32_t *d_agent_ids, uint32_t n, uint32_t *d_lo,
                          uint32_t *d_hi)
{
    if (!run || !d_agent_ids || !d_lo || !d_hi || n < 2 || n > 65536u) return GA_EINVAL;
    void *scratch = nullptr;
    const size_t bytes = ga::mrca_scratch_bytes(run, n);
    if (ga::pool_alloc(&scratch, bytes, run->stream) != cudaSuccess) {
        cudaGetLastError();
        return GA_ENOMEM;
    }
    int rc = cuda_rc(ga::launch_mrca(run, d_agent_ids, n, d_lo, d_hi, scratch));
    const int rc2 = cuda_rc(ga::pool_free(scratch, run->stream));
    return rc != GA_OK ? rc : rc2;
}

int ga_mrca_bounds(ga_run *run, const uint32_t *agent_ids, uint32_t n, uint32_t *lo,
                   uint32_t *hi)
{
    if (!run || !agent_ids || !lo || !hi || n < 2 || n > 65536u) return GA_EINVAL;
    for (uint32_t i = 0; i < n; ++i)
        if (agent_ids[i] >= run->n_agents) return GA_EINVAL;
    const size_t pairs = static_cast<size_t>(n) * (n - 1) / 2;
    const size_t ids_bytes = align_up(n * sizeof(uint32_t), 256);
    const size_t out_bytes = align_up(pairs * sizeof(uint32_t), 256);
    uint8_t *buf = nullptr;
    if (ga::pool_alloc(reinterpret_cast<void **>(&buf), ids_bytes + 2 * out_bytes, run->stream) !=
        cudaSuccess) {
        cudaGetLastError();
        return GA_ENOMEM;
    }
    uint32_t *d_ids = reinterpret_cast<uint32_t *>(buf);
    uint32_t *d_lo = reinterpret_cast<uint32_t *>(buf + ids_bytes);
    uint32_t *d_hi = reinterpret_cast<uint32_t *>(buf + ids_bytes + out_bytes);
    int rc = cuda_rc(cudaMemcpyAsync(d_ids, agent_ids, n * sizeof(uint32_t),
                                     cudaMemcpyHostToDevice, run->stream));
    if (rc == GA_OK) rc = ga_mrca_bounds_device(run, d_ids, n, d_lo, d_hi);
    if (rc == GA_OK)
        rc = cuda_rc(cudaMemcpyAsync(lo, d_lo, pairs * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                     run->stream));
    if (rc == GA_OK)
        rc = cuda_rc(cudaMemcpyAsync(hi, d_hi, pairs * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                     run->stream));
    ga::pool_free(buf, run->stream);
    if (cudaStreamSynchronize(run->stream) != cudaSuccess) return GA_ECUDA;
    if (rc != GA_OK) return rc;
    return take_status(run);
}

int ga_curation_sites(uint32_t policy, uint32_t surface_sites, uint32_t t0, uint32_t count,
                      int32_t *d_sites, void *stream)
{
    if (!d_sites || policy > GA_HYBRID || !is_pow2(surface_sites) || surface_sites > 256u ||
        surface_sites < (policy == GA_HYBRID ? 8u : 4u))
        return GA_EINVAL;
    if (static_cast<uint64_t>(t0) + count > 0x100000000ull) return GA_EINVAL;
    return cuda_rc(ga::launch_curation_sites(policy, surface_sites, t0, count, d_sites,
                                             static_cast<cudaStream_t>(stream)));
}

int ga_destroy(ga_run *run)
{
    if (!run) return GA_EINVAL;
    int rc = GA_OK;
    if (run->batch) rc = ga_batch_remove(run->batch, run);
    if (cudaStreamSynchronize(run->stream) != cudaSuccess) rc = GA_ECUDA;
    if (run->owns_workspace && cudaFree(run->workspace) != cudaSuccess) rc = GA_ECUDA;
    delete run;
    return rc;
}

const char *ga_strerror(int code)
{
    switch (code) {
    case GA_OK: return "ok";
    case GA_EINVAL: return "invalid argument or configuration";
    case GA_ENOMEM: return "out of device memory or workspace too small";
    case GA_ECUDA: return "CUDA runtime error";
    case GA_ETIMEOUT: return "bounded device wait expired";
    case GA_ESTATE: return "device state does not allow the request";
    case GA_EUNSUPPORTED: return "configuration has no compiled kernel";
    case GA_ERANGE: return "caller buffer too small";
    case GA_EBOUNDS: return "device index check failed";
    default: return "unknown error";
    }
}

}  // extern "C"
