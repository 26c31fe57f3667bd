// ga_internal.h -- host-side state of a run and the launchers shared by the library's
// translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "ga.h"

struct ga_run {
    ga_config cfg;
    cudaStream_t stream;
    uint32_t n_islands;
    uint32_t n_agents;
    uint32_t record_bytes;   // 16, 32 or 48
    uint32_t surface_words;  // ceil(S*b/32)
    uint32_t log2_sites;
    uint32_t theta_ben, theta_del;
    uint32_t per_neighbor, every_k;
    uint64_t generation;
    uint64_t launches;
    void *workspace;
    size_t workspace_bytes;
    bool owns_workspace;
    int *d_status;       // device error word (GA_OK or a GA_E* code), in the workspace header
    int32_t *d_sites;    // curation site of generation sites_base + i (workspace header)
    uint64_t sites_base;
    uint8_t *pop[2];     // double-buffered population
    int cur;             // index of the current population buffer
    // asynchronous modes only (null otherwise)
    uint8_t *mail;       // [island][direction] send buffers
    uint32_t async_window;
    ga_batch *batch;     // the batch this run belongs to, if any
    bool counters_uniform;  // every agent's counter equals `generation` (founder, sync steps)
    int *d_flag;         // device scratch word for ga_load's counter check (workspace header)
    uint2 *d_masks;      // deposit masks of generation sites_base + i (workspace header)
    // resident stepping (ga_resident.cu): abort word and mailboxes (null when the run is too
    // large or not synchronous), policy, wait limit and the fault-injection island
    void *resident_state;
    uint32_t resident_mode;
    uint32_t resident_wait_us;
    uint32_t drop_island;
};

namespace ga {

// Stream-ordered device memory of the library (per-call scratch, batch tables): a memory pool
// of the library's own on each device, created on first use, which keeps up to
// kPoolKeepBytes reserved across synchronisations.  The device's default pool returns freed
// memory at every synchronisation, so a caller that synchronises between calls would pay for
// mapping the memory again on each call.
constexpr uint64_t kPoolKeepBytes = 512ull << 20;
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t stream);
inline cudaError_t pool_free(void *p, cudaStream_t stream) { return cudaFreeAsync(p, stream); }

// Launch `kernel` as a programmatic dependent of the previous kernel on `stream` (see
// wait_previous_grid in ga_device.cuh).
template <typename... P, typename... A>
cudaError_t launch_dependent(void (*kernel)(P...), dim3 grid, dim3 block, cudaStream_t stream,
                             A... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

// Workspace header: the device status word (first 256 bytes), then the curation-site table
// of the generations a ga_step call is about to run (one int32 per generation), then their
// deposit masks (two uint32 per generation; filled for surfaces of at most 64 bits).
constexpr size_t kStatusBytes = 256;
constexpr uint32_t kSiteTableCap = 4096;
constexpr size_t kMaskOffset = kStatusBytes + kSiteTableCap * sizeof(int32_t);
constexpr size_t kHeaderBytes = kMaskOffset + kSiteTableCap * 2 * sizeof(uint32_t);

// Largest number of generations one island-step launch runs without migration.
constexpr uint32_t kMaxGensPerLaunch = 256;

// island_step launch: generations [g0, g0 + n_gens) read from src, write dst; migration (if
// `migrate`) happens only at g0.
bool step_supported(uint32_t island_size, uint32_t surface_words, uint32_t model);
cudaError_t launch_founder(ga_run *run, void *dst);
// Set *d_flag to 1 if some agent of the current population has a counter other than
// `generation` (the caller clears it first).
cudaError_t launch_counter_check(ga_run *run, uint32_t generation, int *d_flag);
cudaError_t launch_island_step(ga_run *run, const void *src, void *dst, uint32_t g0,
                               uint32_t n_gens, bool migrate, cudaStream_t stream);
// Fill the site table with the curation sites of generations [g0, g0 + count).
cudaError_t launch_site_table(ga_run *run, uint32_t g0, uint32_t count, cudaStream_t stream);
// Advance one run by n_gens generations with the single-run kernels on `stream` (the body of
// ga_step; the batch uses it for members that fill the GPU on their own).
int step_run(ga_run *run, uint32_t n_gens, cudaStream_t stream);
cudaError_t launch_mrca(ga_run *run, const uint32_t *d_ids, uint32_t n, uint32_t *d_lo,
                        uint32_t *d_hi, void *scratch);
size_t mrca_scratch_bytes(const ga_run *run, uint32_t n);
// Asynchronous mode (ga_async.cu).
bool async_supported(uint32_t island_size, uint32_t surface_words, uint32_t model);
size_t async_state_bytes(uint32_t n_islands, uint32_t record_bytes);
// Empty every send buffer of an asynchronous run.
cudaError_t async_clear(ga_run *run, cudaStream_t stream);
// Generations [g0, g0 + n_gens) of islands [first, last), reading src and writing dst.
cudaError_t launch_island_async(ga_run *run, const void *src, void *dst, uint32_t g0,
                                uint32_t n_gens, uint32_t first, uint32_t last,
                                cudaStream_t stream);
int async_step(ga_run *run, uint32_t n_gens, cudaStream_t stream);

// Resident stepping (ga_resident.cu).  Runs of at most kResidentMaxIslands islands with
// 16-byte records get the mailbox state in their workspace; GA_RESIDENT_AUTO uses resident
// launches up to kResidentAutoIslands islands.
constexpr uint32_t kResidentMaxIslands = 8192;
constexpr uint32_t kResidentAutoIslands = 8192;
size_t resident_state_bytes(uint32_t n_islands, uint32_t record_bytes);
// The run can step resident now: state present, synchronous, counters equal to the generation,
// a kernel for its island size, and its grid co-resident on the device.
bool resident_possible(const ga_run *run, uint32_t *blocks);
// Generations [g0, g0 + n_gens) of the whole run in one cooperative launch (src -> dst).
cudaError_t launch_resident(ga_run *run, const void *src, void *dst, uint32_t g0, uint32_t n_gens,
                            cudaStream_t stream);

// Curation sites of ranks [t0, t0 + count); with d_masks (S * bits <= 64) also the deposit
// masks of those ranks.
cudaError_t launch_curation_sites(uint32_t policy, uint32_t sites, uint32_t t0, uint32_t count,
                                  int32_t *d_sites, cudaStream_t stream, uint32_t bits = 0,
                                  uint2 *d_masks = nullptr);

}  // namespace ga
