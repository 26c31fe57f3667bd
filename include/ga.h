/*
 * ga.h -- C ABI of libga, the GB300 (sm_103a) trackable island-model genetic algorithm.
 *
 * The library runs the per-generation island step of Moreno et al., "Trackable Island-model
 * Genetic Algorithms at Wafer Scale" (GECCO'24 Companion), Sec. 2, on one GPU: a torus of
 * islands, each a population of N agents; every generation handles migration first (one
 * migrant from each of the four cardinal neighbours, replacing randomly chosen members),
 * then evaluation (fitness = trait), tournament selection (n random picks, ties broken
 * randomly), mutation of the trait (+1 with p_ben, -1 with p_del; the paper's adaptive vs
 * purifying-only treatments of Sec. 3 are p_ben > 0 vs p_ben = 0) and the hereditary
 * stratigraphy (hstrat) update for the elapsed generation; the run halts after the
 * requested number of generations.  Post hoc, ga_mrca_bounds estimates pairwise relatedness
 * from the hstrat surfaces (Fig. 1 caption).
 *
 * Conventions
 *   - Every call returns GA_OK (0) or a negative GA_E* code; nothing throws or exits.
 *   - Host buffers passed in are owned by the caller and only read/written during the call.
 *   - Device memory: the run's state lives in one device workspace, either supplied by the
 *     caller (ga_create with a non-NULL workspace; the caller frees it after ga_destroy) or
 *     allocated by the library (workspace NULL; freed by ga_destroy).
 *   - All GPU work of a run is enqueued on the stream given in its config (NULL = the
 *     legacy default stream).  Calls that end in "_device" or ga_step are asynchronous with
 *     respect to the host; the others synchronise that stream before returning.
 *   - A ga_run handle is not thread-safe; distinct handles may be used from distinct threads.
 *   - Agent id = island * island_size + slot; island id = y * cols + x on a rows x cols
 *     torus.
 *
 * Canonical agent record (the device layout and the snapshot layout are the same):
 *   int32 trait; uint32 counter; uint32 surface[W]; zero padding to record_bytes,
 *   W = ceil(S*b/32), record_bytes = round_up(8 + 4W, 16).  Differentia of site k occupies
 *   bits [k*b, k*b + b) of the surface, least-significant bit first, little-endian words.
 *   Records are 16-byte aligned so each agent moves as whole 128-bit words.
 */
#ifndef GA_H
#define GA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GA_OK 0
#define GA_EINVAL (-1)       /* invalid argument or configuration                        */
#define GA_ENOMEM (-2)       /* device allocation failed, or caller workspace too small  */
#define GA_ECUDA (-3)        /* a CUDA runtime call or kernel launch failed              */
#define GA_ETIMEOUT (-4)     /* a bounded device-side wait expired (resident stepping)   */
#define GA_ESTATE (-5)       /* device state does not allow the request (e.g. counters of
                                sampled agents differ, so no common rank table exists)   */
#define GA_EUNSUPPORTED (-6) /* valid configuration with no compiled kernel for it       */
#define GA_ERANGE (-7)       /* caller buffer too small                                  */
#define GA_EBOUNDS (-8)      /* a device index check failed; only builds with device checks
                                (libga_debug.so) test indices, skipping the access      */

/* Curation policy: which surface site the deposit of generation T overwrites. */
#define GA_STEADY 0u /* evenly spaced retained ranks (gap <= 2T/S), any T                */
#define GA_TILTED 1u /* recency-weighted: two ranks per hanoi level, S/2 levels           */
#define GA_HYBRID 2u /* first S/2 sites steady on even ranks, last S/2 tilted on odd ranks */

#define GA_SYNC 0u  /* synchronous generations: deterministic, bit-exact                 */
#define GA_ASYNC 1u /* asynchronous migration through per-island send buffers (Sec. 2 loop):
                       islands advance without waiting for one another, so results depend on
                       scheduling and agents' counters drift apart                         */
#define GA_ASYNC_SEQUENTIAL 2u /* the GA_ASYNC step on a reproducible schedule: within each
                       window of generations, islands run one at a time in index order
                       (one launch per island; slow; for debugging and checking)            */

/* Largest asynchronous window (generations one island runs per launch). */
#define GA_ASYNC_MAX_WINDOW 256u

/* Genome model: what the first record word means and how it mutates. */
#define GA_MODEL_TRAIT 0u   /* int32 trait; +1 with p_ben, -1 with p_del                     */
#define GA_MODEL_FITNESS 1u /* IEEE float fitness (Sec. 3 treatments): -/+ effect_scale * |z|
                               with p_del / p_ben, z a standard normal deviate (Box-Muller in
                               single precision, correctly rounded operations only, from
                               Philox words 0 and 1 of counter (g, island, slot | 3 << 16,
                               run_id)); tournaments compare fitness as floats              */

typedef struct ga_run ga_run;

typedef struct ga_config {
    uint32_t rows, cols;        /* torus of islands, each >= 1                                 */
    uint32_t island_size;       /* N: power of two; GPU kernels exist for 4..128              */
    uint32_t tournament_size;   /* n in [1, 8], draws with replacement (Sec. 2; Sec. 3 uses 5) */
    double p_ben, p_del;        /* per-birth probabilities, p >= 0, p_ben + p_del <= 1        */
    uint32_t surface_sites;     /* S: power of two, >= 4 (>= 8 for GA_HYBRID)                 */
    uint32_t differentia_bits;  /* b in {1, 2, 4, 8}; S * b <= 256                            */
    uint32_t curation;          /* GA_STEADY / GA_TILTED / GA_HYBRID                          */
    uint32_t mode;              /* GA_SYNC / GA_ASYNC / GA_ASYNC_SEQUENTIAL                   */
    uint64_t seed;              /* Philox key = (low 32 bits, high 32 bits)                   */
    uint32_t run_id;            /* fourth Philox counter word: distinct runs draw disjointly  */
    uint32_t model;             /* GA_MODEL_TRAIT / GA_MODEL_FITNESS                          */
    void *stream;               /* cudaStream_t for all of this run's GPU work (NULL: default) */
    double effect_scale;        /* GA_MODEL_FITNESS: scale of the normal mutation amount > 0  */
} ga_config;

/* Fill *cfg with the 32x32-torus defaults: N = 32, n = 5, p_ben = p_del = 0.01, S = 64,
   b = 1, steady, sync, trait model, seed 42, run_id 0, default stream, effect_scale 1. */
int ga_config_default(ga_config *cfg);

/* Check a configuration without touching the GPU.  GA_EINVAL: invalid;
   GA_EUNSUPPORTED: valid but no kernel is compiled for its island/record size. */
int ga_config_check(const ga_config *cfg);

/* Bytes of one canonical agent record for cfg (16, 32 or 48). */
int ga_record_bytes(const ga_config *cfg, uint32_t *bytes);

/* Bytes of device workspace a run of cfg needs (two population buffers plus a header; in the
   asynchronous modes also four send buffers per island: 16 bytes each for 16-byte records,
   16 + record_bytes otherwise; for synchronous runs of at most 8,192 islands with 16-byte
   records also the resident-stepping mailboxes, 128 bytes per island plus 256). */
int ga_workspace_bytes(const ga_config *cfg, size_t *bytes);

/*
 * Create a run and enqueue its founder initialisation (Sec. 2 "initialize"): every agent is
 * a clone of one founder with trait 0, counter 0 and surface word w equal to word 0 of
 * Philox4x32-10(counter (0, 0, w | 2 << 16, run_id), key seed).
 * workspace: device pointer of at least ga_workspace_bytes() bytes, 256-byte aligned, owned
 * by the caller; or NULL to let the library allocate (and later free) it.
 * Errors: GA_EINVAL (config, alignment), GA_EUNSUPPORTED, GA_ENOMEM, GA_ECUDA.
 */
int ga_create(const ga_config *cfg, void *workspace, size_t workspace_bytes, ga_run **out);

/* Re-enqueue founder initialisation and set the generation counter to 0 (same effect as a
   fresh ga_create with the same config).  Asynchronous. */
int ga_reset(ga_run *run);

/*
 * Migration policy (Sec. 2): per_neighbor migrants arrive from each of the four neighbours
 * on every generation g with g mod every_k == 0.  per_neighbor in {0, 1} (0 disables
 * migration); every_k >= 1.  The default after ga_create is (1, 1).
 */
int ga_migrate_policy(ga_run *run, uint32_t per_neighbor, uint32_t every_k);

/*
 * Asynchronous modes (Sec. 2: the wafer-scale loop tests completion flags of asynchronous
 * sends and receives and never waits for them).  Each island owns one send buffer per
 * direction, holding at most one genome; a send completes when the neighbour takes the
 * genome out.  On each of its migration generations g (g mod every_k == 0) an island, in
 * this order: (0) tests every buffer facing it and each of its own buffers; (1) for
 * directions N, S, E, W takes the genome out of each buffer facing it that tested full (the
 * buffer becomes empty) and lands it in the slot chosen by the partial Fisher-Yates draw of
 * GA_SYNC (missing arrivals leave their slot alone); (2) fills each of its own buffers that
 * tested empty with a copy of member e_d = (bits 8..15 of word 3 of its slot-d birth draw)
 * * N >> 8; then (3) reproduces as in GA_SYNC.  Nothing ever waits.  Only where an island
 * is its own neighbour (one-row or one-column tori) can a buffer change between (0) and (2):
 * one it empties itself in (1) is refilled a pass later.  A migrant keeps its counter, so
 * counters drift apart and each deposit uses the site of the agent's own counter.  Counter
 * 2^32 - 1 is reserved (it marks an empty buffer): a birth that produces it makes the run
 * invalid, reported as GA_ESTATE by the next ga_sync or ga_snapshot.
 *
 * A launch runs `window` generations of every island (all islands start it at the same
 * generation).  With window 1 no island gets more than a generation ahead of another, as
 * when processors run side by side.  Larger windows keep each island in registers for
 * longer (faster), but a launch whose blocks run in many waves lets islands of late blocks
 * start a window after early ones have finished it; a lineage that keeps migrating towards
 * later blocks is then born in each of them and its counter runs ahead of the generation
 * -- under beneficial mutation such lineages are fitter and take over.  GA_ASYNC_SEQUENTIAL
 * runs each window island by island in index order: a reproducible schedule the CPU model
 * follows exactly.  window in [1, GA_ASYNC_MAX_WINDOW]; the default after ga_create is 1.
 * Send buffers are emptied by ga_create, ga_reset and ga_load.  Asynchronous kernels exist
 * for island sizes 8 to 128 (4-agent islands: GA_EUNSUPPORTED from ga_create).
 * Errors: GA_EINVAL (window out of range), GA_ESTATE (run not in an asynchronous mode).
 */
int ga_async_window(ga_run *run, uint32_t window);

/*
 * Resident stepping (Sec. 2: each processor keeps its population in place and exchanges only
 * migrants with its neighbours).  A synchronous run whose islands all fit on the GPU at once
 * can step a whole chunk of up to 4,096 generations in one cooperative launch: every island
 * stays in registers, and on each migration generation an island pushes the member each
 * neighbour draws into that neighbour's mailbox (one 16-byte atomic write) and reads its own
 * four mailboxes, waiting until each holds the record of the current generation.  Results are
 * bit-identical to the streamed launches.  Eligible: GA_SYNC, 16-byte records, island sizes
 * 8 to 64, counters equal to the generation, at most 8,192 islands, and a grid that the
 * device can hold resident; the mailboxes (128 bytes per island) are part of the workspace of
 * such runs.
 *   GA_RESIDENT_AUTO  (default) resident launches whenever eligible;
 *   GA_RESIDENT_OFF   one launch per migration interval, the population streamed;
 *   GA_RESIDENT_ON    resident launches; ga_step returns GA_EUNSUPPORTED if not eligible.
 * wait_limit_us bounds every wait for a mailbox (wall clock, default 1,000,000 = 1 s): when
 * it runs out the launch records GA_ETIMEOUT, every block leaves at its next migration
 * generation, the population is undefined, and the next ga_sync returns GA_ETIMEOUT (the
 * run can then be reset or loaded and stepped again).  Errors: GA_EINVAL (mode, limit 0).
 */
#define GA_RESIDENT_AUTO 0u
#define GA_RESIDENT_OFF 1u
#define GA_RESIDENT_ON 2u
int ga_resident_policy(ga_run *run, uint32_t mode, uint32_t wait_limit_us);

/*
 * Fault injection for testing the bounded waits above (the paper has no counterpart): in
 * resident launches, island `island` never pushes its emigrants, so its four neighbours wait
 * for mailboxes that nothing fills until their limit runs out.  0xFFFFFFFF (the default)
 * turns it off.  Errors: GA_EINVAL (island out of range).
 */
int ga_inject_lost_migrants(ga_run *run, uint32_t island);

/*
 * Enqueue n_gens generations on the run's stream (Sec. 2 generational cycle, halting after
 * n_gens).  Asynchronous; launch failures are returned here, nothing is read back.
 * Generation g of a run always draws the same random numbers, so splitting n_gens over
 * several calls gives bit-identical results.  Errors: GA_EINVAL (null run), GA_ECUDA.
 */
int ga_step(ga_run *run, uint32_t n_gens);

/* Wait for the run's stream and report any error the device recorded. */
int ga_sync(ga_run *run);

/* Generations completed (enqueued) so far. */
int ga_generation(const ga_run *run, uint64_t *generation);

/* Kernels this run has launched so far (all of them the library's own). */
int ga_launch_count(const ga_run *run, uint64_t *launches);

/* Device pointer and size of the current population buffer (valid until the next
   ga_step / ga_load / ga_destroy).  Read it only on the run's stream, or after ga_sync. */
int ga_population(ga_run *run, void **device_ptr, size_t *bytes);

/* Copy the whole population (canonical records, agent-id order) to host_dst.  Synchronous.
   GA_ERANGE when cap is smaller than n_agents * record_bytes (*written gets the need). */
int ga_snapshot(ga_run *run, void *host_dst, size_t cap, size_t *written);

/* As ga_snapshot but into device memory, asynchronously on the run's stream. */
int ga_snapshot_device(ga_run *run, void *device_dst, size_t cap, size_t *written);

/* Replace the population with canonical records from host_src and set the generation
   counter (checkpoint resume; bit-exact because draws are keyed by generation).  bytes
   must equal n_agents * record_bytes.  Agents may carry any counters, except 2^32 - 1 in the
   asynchronous modes (reserved: it marks an empty send buffer; GA_EINVAL); in GA_SYNC mode a
   device pass checks whether every counter equals `generation` (the usual case, a snapshot of
   a synchronous run), and later steps use kernels without the closed-form curation path only
   then.  Synchronous. */
int ga_load(ga_run *run, const void *host_src, size_t bytes, uint64_t generation);

/*
 * Pairwise MRCA bounds (Fig. 1: post hoc relatedness from hstrat markers).
 * agent_ids: n distinct agent ids (host); lo, hi: n(n-1)/2 uint32 each (host), pairs (i, j),
 * i < j, in row-major upper-triangle order: pair index i*(2n-i-1)/2 + (j-i-1).
 * In GA_SYNC mode all sampled agents must hold the same counter T.  With the
 * sites' retained ranks r_1 < ... < r_m (ranks < T) and i* the first index at which the
 * two differentiae differ, the divergence rank D (first rank the two lineages drew in
 * separate births) satisfies D in [lo, hi]:
 *   hi = r_{i*} (certain), lo = r_{i*-K} + 1 or 0 if i* <= K; with no mismatch hi = T and
 *   lo = r_{m-K+1} + 1 (0 if m < K); K = smallest integer with 2^(-bK) < 0.05, so lo holds
 *   with confidence 0.95.
 * In the asynchronous modes agents i and j may hold different counters Ti and Tj: the
 * ranks compared are those retained by both (a rank sits at the same site in both tables,
 * so these are the sites whose rank tables at Ti and Tj agree), in ascending order, and the
 * same rule applies to that list with hi = min(Ti, Tj) when nothing mismatches.  The
 * retained ranks at a counter come from the curation rule in closed form, without replaying
 * earlier ranks: O(S) work per distinct table, O(n^2) (GA_SYNC) or O(n^2 S) (mixed
 * counters) for the pairs.
 * Synchronous.  Scratch memory is taken from and returned to the library's own memory pool
 * in the run's stream order (one pool per device, which keeps up to 512 MiB mapped across
 * synchronisations, so repeated calls do not map memory again).
 * Errors: GA_EINVAL (n < 2, n > 65536, id out of range, null pointers), GA_ESTATE
 * (GA_SYNC mode and counters differ), GA_ENOMEM, GA_ECUDA.
 */
int ga_mrca_bounds(ga_run *run, const uint32_t *agent_ids, uint32_t n, uint32_t *lo,
                   uint32_t *hi);

/* As ga_mrca_bounds with device buffers for ids, lo and hi; asynchronous on the run's
   stream.  Ids are not range-checked on the host (the kernel skips out-of-range ids and
   records GA_EINVAL, reported by ga_sync), counter mismatches (GA_SYNC mode) are reported
   by ga_sync. */
int ga_mrca_bounds_device(ga_run *run, const uint32_t *d_agent_ids, uint32_t n,
                          uint32_t *d_lo, uint32_t *d_hi);

/*
 * Batches: many independent runs advanced by shared launches.  The paper runs each
 * population on its own processor (Sec. 2) and its trials one at a time (Sec. 3); a batch
 * instead packs the islands of all member runs into one launch per class (island size,
 * record size, seed) and generation, so small runs fill the GPU together.  Each member's
 * results are bit-identical to stepping it alone (draws are keyed by seed, run_id,
 * generation, island and slot).  A fixed-length chunk of generations is captured once as a
 * CUDA graph and replayed.
 *
 * A run belongs to at most one batch at a time.  Call ga_batch_sync before any per-run call
 * on a member (ga_snapshot, ga_mrca_bounds, ga_step, ga_reset, ga_load, ...); a member whose
 * generation or buffer changed through such calls is picked up by the next ga_batch_step.  Member runs may have different shapes, mutation rates, tournament
 * sizes, curation policies, seeds and migration policies.  Members with 65,536 islands or
 * more, float-fitness runs, asynchronous runs and island sizes without a batched kernel
 * (4, 128) step with the single-run kernels on the batch's stream instead of sharing class
 * launches.
 */
typedef struct ga_batch ga_batch;

/* Create an empty batch whose launches go to `stream` (NULL: a stream the batch creates
   and owns).  Errors: GA_EINVAL, GA_ENOMEM, GA_ECUDA. */
int ga_batch_create(void *stream, ga_batch **out);

/* Add a run.  The batch's stream is ordered after the work already queued on the run's
   stream (a device-side wait; the host does not block).  GA_EINVAL if it is already a member
   of this or another batch. */
int ga_batch_add(ga_batch *batch, ga_run *run);

/* Remove a member run (the run keeps its state).  Work queued on the run's own stream
   afterwards, ga_destroy's wait included, is ordered after the batch launches already queued
   (a device-side wait; the host does not block). */
int ga_batch_remove(ga_batch *batch, ga_run *run);

/* Number of member runs. */
int ga_batch_size(const ga_batch *batch, uint32_t *n_runs);

/* Advance every member run by n_gens generations (Sec. 2 generational cycle), on the
   batch's stream, asynchronously.  Errors: GA_EINVAL, GA_ENOMEM, GA_ECUDA. */
int ga_batch_step(ga_batch *batch, uint32_t n_gens);

/* Wait for the batch's stream. */
int ga_batch_sync(ga_batch *batch);

/* Kernels the batch has launched (a graph replay counts its kernel nodes). */
int ga_batch_launch_count(const ga_batch *batch, uint64_t *launches);

/*
 * Autotune the launch shape: for each class, warps per block in {4, 8, 16}; then the graph
 * chunk length in {16, 64, 256} generations -- each candidate timed with CUDA events over
 * trial_gens generations of the real member runs, whose state is saved before and restored
 * after the trials (results are unchanged by any choice).  *chosen_chunk (optional) gets the
 * chunk length.  Synchronous.  Errors: GA_EINVAL, GA_ENOMEM, GA_ECUDA.
 */
int ga_batch_autotune(ga_batch *batch, uint32_t trial_gens, uint32_t *chosen_chunk);

/* Island size and warps per block of class `index` (classes ordered by first member). */
int ga_batch_class_warps(const ga_batch *batch, uint32_t index, uint32_t *island_size,
                         uint32_t *warps);

/* Destroy the batch (synchronises its stream; member runs are left intact and belong to no
   batch afterwards). */
int ga_batch_destroy(ga_batch *batch);

/*
 * Curation table: d_sites[i] = site that the deposit of rank t0 + i overwrites under the
 * given policy over S sites, or -1 when that rank is not stored (hstrat update of Sec. 2;
 * the policies are those of GA_STEADY / GA_TILTED / GA_HYBRID).  Computed by a kernel on
 * `stream` (NULL: default stream), asynchronously.  Errors: GA_EINVAL (policy, S, or a
 * range past 2^32 - 1), GA_ECUDA.
 */
int ga_curation_sites(uint32_t policy, uint32_t surface_sites, uint32_t t0, uint32_t count,
                      int32_t *d_sites, void *stream);

/*
 * ga_mrca_bounds without any device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- for instance a process
 * whose framework has already reserved the GPU's memory for its own caching allocator (so
 * cudaMalloc fails), a plugin or callback that its host forbids from allocating, or a
 * latency-critical path that cannot afford cudaMalloc/cudaFree, which may synchronise the
 * device.  It computes exactly what ga_mrca_bounds_device computes, from caller-owned
 * device buffers and without a ga_run:
 *   d_records      canonical records of n_agents agents (16-byte aligned device memory),
 *                  record_bytes = round_up(8 + 4 ceil(S b / 32), 16);
 *   curation, surface_sites, differentia_bits: the run's GA_STEADY/TILTED/HYBRID, S, b;
 *   generation     T, the counter every sampled agent must hold;
 *   d_agent_ids    n device uint32 ids, 2 <= n <= 4096 (larger n: GA_EINVAL);
 *   d_lo, d_hi     n(n-1)/2 device uint32 each, pairs in row-major upper-triangle order.
 * Its scratch (133,632 bytes) is a fixed array inside the library's device image, which
 * every GPU that loads the library holds until the process exits.  Each call looks up that
 * array's device address (cudaGetSymbolAddress, with the caller's device current), so it
 * stays valid after a device reset.  All calls on a device share the one array and each call
 * overwrites it, so calls that overlap on the GPU (from several host threads or streams at
 * once) race and must be serialised by the caller.
 * Synchronous: enqueues on `stream` (NULL: default stream) and waits for it, so it must not
 * be called while that stream is being captured into a CUDA graph.  Returns GA_ESTATE when
 * an agent's counter differs from T, GA_EINVAL for an id >= n_agents, GA_EINVAL for invalid
 * arguments, GA_ECUDA for runtime failures (an error left pending by earlier work on the
 * calling thread is cleared first and not reported).  It calls no cudaMalloc, cudaFree or
 * other allocating routine.
 */
int ga_mrca_bounds_noalloc(const void *d_records, uint32_t record_bytes, uint32_t n_agents,
                           uint32_t curation, uint32_t surface_sites, uint32_t differentia_bits,
                           uint32_t generation, const uint32_t *d_agent_ids, uint32_t n,
                           uint32_t *d_lo, uint32_t *d_hi, void *stream);

/*
 * Integer-pipe throughput probe.  The paper has no counterpart: a measurement aid that gives
 * a measured ceiling for the island step's integer work, next to the nominal issue limit.
 * Runs, on the current device, 8 resident blocks of 256 threads per SM, each thread
 * independent chains of one operation `kind` (eight chains of 32 steps per iteration; for
 * GA_PEAK_MIX two Philox states of 16 rounds), `iters` iterations, after a short warm-up;
 * times the launch with CUDA events on `stream` (NULL: default stream).
 *   GA_PEAK_LOP3  three-input logic (lop3.b32)
 *   GA_PEAK_IMAD  32 x 32 -> 64-bit multiply-add (mad.wide.u32)
 *   GA_PEAK_MIX   Philox4x32 rounds: two 32 x 32 -> 64-bit multiplies and two three-input
 *                 XORs each (the island step's random-number arithmetic)
 * *ops_per_s gets operations (one per PTX instruction above) per second; *seconds (optional)
 * the timed launch's duration.  Synchronous.  Errors: GA_EINVAL, GA_ENOMEM, GA_ECUDA.
 */
#define GA_PEAK_LOP3 0u
#define GA_PEAK_IMAD 1u
#define GA_PEAK_MIX 2u
int ga_int_peak(uint32_t kind, uint32_t iters, void *stream, double *ops_per_s, double *seconds);

/* Destroy the run (synchronises its stream; frees library-owned memory).  A member of a
   batch is first removed from it, as by ga_batch_remove. */
int ga_destroy(ga_run *run);

/* Static description of an error code. */
const char *ga_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* GA_H */
