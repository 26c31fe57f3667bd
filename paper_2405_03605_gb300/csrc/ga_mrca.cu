// ga_mrca.cu -- pairwise MRCA bounds over sampled end-state agents (post hoc relatedness
// estimation from hstrat markers, Fig. 1 caption of the paper).
//
// Pipeline (all on the run's stream):
//   1. rank_table_kernel: the ranks the surface retains at counter T, in closed form (no
//                      replay of ranks 0..T-1): one thread per retained rank (steady) or per
//                      site (tilted), each rank placed at its site; then the occupied sites
//                      sorted by rank in the same block (S <= 256): r_1 < ... < r_m.
//   2. pack_kernel   : gather each sampled agent's differentiae in rank order into a bit
//                      string (differentia i at bits [i*b, i*b + b)), 8 words per agent; one
//                      warp per agent, one warp OR-reduction per packed word.
//   3. pair_kernel   : one thread per pair (i, j), j > i, in output order; the first set bit of
//                      packed[i] ^ packed[j] gives the first mismatching rank index i*,
//                      from which hi = r_{i*} and lo = r_{i*-K} + 1 (0 if i* <= K); with no
//                      mismatch hi = T, lo = r_{m-K+1} + 1 (0 if m < K).
// The pair kernel is bound by its output: 8 bytes (lo, hi) per pair, written once with
// streaming stores.
#include "ga_device.cuh"
#include "ga_internal.h"

namespace ga {

namespace {

constexpr uint32_t kPackWords = 8;  // 256-bit rank-ordered strings
constexpr int kPairThreads = 256;
constexpr unsigned long long kPairGrid = 152ull * 8ull;  // 8 resident blocks on each of 152 SMs


struct MrcaLayout {
    uint32_t *order;   // [S]  sites sorted by rank
    uint32_t *ranks;   // [S]  sorted ranks
    uint32_t *meta;    // [4]  m
    uint32_t *packed;  // [n][kPackWords]
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Scratch bytes of one synchronous MRCA call: order, ranks, meta, packed strings.
size_t sync_scratch_bytes(uint32_t S, uint32_t n)
{
    return 2 * align_up(S * 4u, 256) + 256 + static_cast<size_t>(n) * kPackWords * 4u;
}

MrcaLayout carve(void *scratch, uint32_t S)
{
    uint8_t *p = static_cast<uint8_t *>(scratch);
    MrcaLayout l;
    size_t off = 0;
    l.order = reinterpret_cast<uint32_t *>(p + off);
    off = align_up(off + S * 4u, 256);
    l.ranks = reinterpret_cast<uint32_t *>(p + off);
    off = align_up(off + S * 4u, 256);
    l.meta = reinterpret_cast<uint32_t *>(p + off);
    off = align_up(off + 16u, 256);
    l.packed = reinterpret_cast<uint32_t *>(p + off);
    return l;
}

// ---------------------------------------------------------------------------------------
// Ranks retained at count T (ranks 0..T-1 deposited), without replaying them.
//
// Steady, S = 2^s sites: while T <= S every rank below T is held.  Otherwise let t >= 1 be
// the epoch of rank T - 1 (bit length minus s) and P = 2^(s+t-1) its first rank.  At P the
// surface holds exactly the ranks below P whose hanoi value is at least t - 1: the S/2 with
// hanoi >= t (rank + 1 = 2^t q, q = 1..S/2) and the S/2 with hanoi exactly t - 1 (rank + 1 =
// 2^(t-1) (2m + 1), m = 0..S/2-1).  Each of the c = T / 2^t - S/2 ranks of epoch t stored so
// far (hanoi >= t: rank + 1 = 2^t (S/2 + 1), 2^t (S/2 + 2), ...) replaced the oldest remaining
// rank of hanoi t - 1, so those m < c are gone.  Retained rank q (0 <= q < S), as rank + 1:
// q < S/2: 2^t (q + 1); S/2 <= q < S - c: 2^(t-1) (2 (c + q - S/2) + 1); else 2^t (S/2 + 1 +
// q - (S - c)).  A rank never moves, so its site is the closed-form site of the rank itself.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t steady_retained(uint32_t s, uint32_t T, uint32_t q)
{
    const uint32_t S = 1u << s;
    if (T <= S) return q < T ? q + 1u : 0u;
    const uint32_t t = 32u - __clz(T - 1u) - s;
    const uint32_t half = S >> 1;
    const uint32_t c = (T >> t) - half;
    uint64_t r1;
    if (q < half) r1 = static_cast<uint64_t>(q + 1u) << t;
    else if (q < S - c) r1 = static_cast<uint64_t>(2u * (c + q - half) + 1u) << (t - 1u);
    else r1 = static_cast<uint64_t>(half + 1u + q - (S - c)) << t;
    return static_cast<uint32_t>(r1);
}

// Tilted, S sites in L = S/2 levels: site k = 2h + p.  Below the top level (h < L - 1) the
// site holds the newest rank < T whose hanoi value is exactly h -- rank + 1 = 2^h (2m + 1) --
// with m of parity p; the top level the newest whose hanoi value is at least L - 1 -- rank + 1
// = 2^(L-1) m', m' >= 1 -- with m' - 1 of parity p.  Returns rank + 1, or 0 for an empty site.
__device__ __forceinline__ uint32_t tilted_holder(uint32_t S, uint32_t T, uint32_t k)
{
    const uint32_t L = S >> 1, h = k >> 1, p = k & 1u;
    if (h + 1u < L) {
        if (h >= 32u || static_cast<uint64_t>(T) < (1ull << h)) return 0u;
        const uint64_t mmax = (static_cast<uint64_t>(T) - (1ull << h)) >> (h + 1u);
        const int64_t m = (mmax & 1u) == p ? static_cast<int64_t>(mmax) : static_cast<int64_t>(mmax) - 1;
        if (m < 0) return 0u;
        return static_cast<uint32_t>(static_cast<uint64_t>(2 * m + 1) << h);
    }
    const uint32_t e = L - 1u;
    if (e >= 32u) return 0u;
    const int64_t mpmax = static_cast<int64_t>(static_cast<uint64_t>(T) >> e);
    const int64_t mp = ((mpmax - 1) & 1) == static_cast<int64_t>(p) ? mpmax : mpmax - 1;
    if (mp < 1) return 0u;
    return static_cast<uint32_t>(static_cast<uint64_t>(mp) << e);
}

// Retained entry q of the surface at count T (q < S): its site and rank + 1 (0: none).
// Hybrid: q < S/2 are the steady half's retained ranks over the even ranks (local count
// ceil(T/2), global rank 2 x local), q >= S/2 the tilted half's sites over the odd ranks
// (local count floor(T/2), global rank 2 x local + 1).
__device__ __forceinline__ uint32_t retained_entry(uint32_t policy, uint32_t s, uint32_t S,
                                                   uint32_t T, uint32_t q, uint32_t &site)
{
    if (policy == kSteady) {
        const uint32_t r1 = steady_retained(s, T, q);
        site = r1 ? static_cast<uint32_t>(steady_site(s, r1 - 1u)) : 0u;
        return r1;
    }
    if (policy == kTilted) {
        site = q;
        return tilted_holder(S, T, q);
    }
    const uint32_t half = S >> 1;
    if (q < half) {
        const uint32_t Te = static_cast<uint32_t>((static_cast<uint64_t>(T) + 1u) >> 1);
        const uint32_t r1 = steady_retained(s - 1u, Te, q);
        site = r1 ? static_cast<uint32_t>(steady_site(s - 1u, r1 - 1u)) : 0u;
        return r1 ? 2u * (r1 - 1u) + 1u : 0u;
    }
    site = q;
    const uint32_t r1 = tilted_holder(half, T >> 1, q - half);
    return r1 ? 2u * r1 : 0u;
}

// One block of 256 threads: the retained ranks at T placed at their sites (shared memory),
// then the occupied sites sorted by rank: order[i] = site of the i-th smallest retained rank,
// ranks[i] = that rank, meta[0] = m.
__global__ void __launch_bounds__(256)
rank_table_kernel(uint32_t *__restrict__ order, uint32_t *__restrict__ ranks,
                  uint32_t *__restrict__ meta, uint32_t policy, uint32_t log2_sites,
                  uint32_t sites, uint32_t T)
{
    __shared__ uint32_t h[256];
    release_next_grid();  // the pack kernel may start loading its agents' records
    const uint32_t k = threadIdx.x;
    h[k] = 0u;
    __syncthreads();
    if (k < sites) {
        uint32_t site = 0;
        const uint32_t r1 = retained_entry(policy, log2_sites, sites, T, k, site);
        if (r1 != 0u) h[site] = r1;
    }
    __syncthreads();
    const uint32_t mine = h[k];
    const int m = __syncthreads_count(mine != 0u);
    if (mine != 0u) {
        uint32_t pos = 0;
        for (uint32_t q = 0; q < sites; ++q) pos += (h[q] != 0u && h[q] < mine) ? 1u : 0u;
        order[pos] = k;
        ranks[pos] = mine - 1u;
    }
    if (k == 0) meta[0] = static_cast<uint32_t>(m);
}

// Retained ranks at counter T, sorted (order, ranks, meta[0] = m): one launch for any T.
cudaError_t launch_rank_table(uint32_t *order, uint32_t *ranks, uint32_t *meta, uint32_t policy,
                              uint32_t log2_sites, uint32_t sites, uint32_t T, cudaStream_t stream)
{
    rank_table_kernel<<<1, 256, 0, stream>>>(order, ranks, meta, policy, log2_sites, sites, T);
    return cudaGetLastError();
}

// One warp per sampled agent: lanes 0..7 hold the agent's surface words; for packed word w,
// lane l gathers differentia index w * (32/b) + l (site order[i], fetched from the lane that
// holds its surface word) and one warp OR-reduction assembles the word.
// reverse64 (strings of at most 64 bits): the 64-bit string (word 1 : word 0) is stored
// bit-reversed, so the first rank index sits at bit 63 and a pair's first mismatch is the
// count of leading zeros of the XOR.
__global__ void pack_kernel(const uint32_t *__restrict__ pop, uint32_t record_words,
                            uint32_t n_agents, const uint32_t *__restrict__ ids, uint32_t n,
                            const uint32_t *__restrict__ order, const uint32_t *__restrict__ meta,
                            uint32_t bits, uint32_t T, uint32_t *__restrict__ packed,
                            int *__restrict__ status, uint32_t reverse64)
{
    __shared__ uint32_t ord[256];
    release_next_grid();  // the pair kernel may start its index set-up
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // the agent's record does not depend on the rank order: load it before waiting for it
    const uint32_t id = a < n ? ids[a] : 0u;
    const bool ok = a < n && id < n_agents;
    const uint32_t *rec = pop + static_cast<size_t>(ok ? id : 0u) * record_words;
    const uint32_t counter = ok ? rec[1] : T;
    const uint32_t surf = (ok && lane < kPackWords && 2u + lane < record_words) ? rec[2 + lane] : 0u;
    wait_previous_grid();
    const uint32_t m = meta[0];
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) ord[i] = order[i];
    __syncthreads();
    if (a >= n) return;  // whole warps
    uint32_t word_out = 0;
    if (!ok) {
        if (lane == 0) atomicCAS(status, GA_OK, GA_EINVAL);
    } else {
        if (lane == 0 && counter != T) atomicCAS(status, GA_OK, GA_ESTATE);
        const uint32_t per = 32u / bits, mask = (1u << bits) - 1u;
        const uint32_t pw = (m * bits + 31u) >> 5;
        for (uint32_t w = 0; w < pw; ++w) {
            const uint32_t i = w * per + lane;
            const uint32_t pos = (lane < per && i < m) ? ord[i] * bits : 0u;
            const uint32_t sw = __shfl_sync(0xffffffffu, surf, static_cast<int>(pos >> 5));
            const uint32_t v = (lane < per && i < m) ? ((sw >> (pos & 31u)) & mask) << (lane * bits) : 0u;
            const uint32_t full = __reduce_or_sync(0xffffffffu, v);
            if (lane == w) word_out = full;
        }
    }
    if (reverse64) {  // lanes 0 and 1 swap words and reverse their bits
        const uint32_t other = __shfl_xor_sync(0xffffffffu, word_out, 1);
        if (lane < 2u) word_out = __brev(other);
    }
    if (lane < kPackWords) packed[static_cast<size_t>(a) * kPackWords + lane] = word_out;
}

// Pairs in output order, each warp a contiguous stretch of them: lane t takes pairs
// base + t, base + t + 32, ..., so a warp's (lo, hi) writes are contiguous.  A lane finds
// the row of its first pair once -- row i holds pairs off(i) <= p < off(i + 1) with
// off(i) = i (2n - i - 1) / 2; a single-precision root of i^2 - (2n - 1) i + 2p = 0 from the
// exact 64-bit discriminant is within one row, and integer comparisons correct it -- then
// steps 32 pairs at a time, carrying into the next rows when j passes n - 1, and reloads row
// i's string only when i changes.  Pair indices fit 32 bits (n <= 65536: fewer than 2^31
// pairs).  The first set bit of packed[i] ^ packed[j] gives the first mismatching rank index
// i*.  With 0-based sorted ranks r_0 < ... < r_{m-1}, a mismatch at index i* gives
// hi = r_{i*}, lo = r_{i*-K} + 1 (0 if i* < K), and no mismatch hi = T, lo = r_{m-K} + 1.
// 64-bit strings (S*b <= 64) are stored bit-reversed (pack_kernel): a pair's first mismatching
// bit is the count c of leading zeros of the XOR, 64 when none (the bits past m*b are zero in
// every string), and one shared table holds both bounds for every c in [0, 64]:
// i* = min(c / b, m), tab[c] = (i* >= K ? r_{i*-K} + 1 : 0, i* < m ? r_{i*} : T).  WIDE
// strings (more than 64 bits) take the first nonzero word of the XOR and the two rules
// separately (measured faster for them than a table).
template <bool WIDE>
__global__ void __launch_bounds__(kPairThreads)
pair_kernel(const uint32_t *__restrict__ packed, uint32_t n, const uint32_t *__restrict__ ranks_g,
            const uint32_t *__restrict__ meta, uint32_t log2_bits, uint32_t K, uint32_t T,
            uint32_t per_warp, uint32_t *__restrict__ lo, uint32_t *__restrict__ hi,
            int *__restrict__ status)
{
    __shared__ uint2 tab[WIDE ? 1 : 65];
    __shared__ uint32_t ranks[WIDE ? 256 : 1];
    // pairs [warp * per_warp, (warp + 1) * per_warp) of n (n - 1) / 2 (per_warp: a multiple of
    // 32 chosen on the host so that the grid covers every pair)
    const uint32_t n_pairs = n * (n - 1u) / 2u;
    const uint32_t warp = (blockIdx.x * kPairThreads + threadIdx.x) >> 5;
    const unsigned long long w_end = static_cast<unsigned long long>(warp + 1u) * per_warp;
    const uint32_t p_end = w_end < n_pairs ? static_cast<uint32_t>(w_end) : n_pairs;
    const unsigned long long p0 = static_cast<unsigned long long>(warp) * per_warp + (threadIdx.x & 31u);
    const bool active = p0 < p_end;
    const uint32_t p = active ? static_cast<uint32_t>(p0) : 0u;

    const unsigned long long b = 2ull * n - 1ull;  // off(r) = r (b - r) / 2
    const float est = (static_cast<float>(b) - sqrtf(static_cast<float>(b * b - 8ull * p))) * 0.5f;
    uint32_t i = est > 0.0f ? static_cast<uint32_t>(est) : 0u;
    if (i > n - 2u) i = n - 2u;
    while (i > 0u && static_cast<unsigned long long>(i) * (b - i) / 2ull > p) --i;
    while (i + 2u < n && static_cast<unsigned long long>(i + 1u) * (b - i - 1u) / 2ull <= p) ++i;
    uint32_t j = i + 1u + static_cast<uint32_t>(p - static_cast<unsigned long long>(i) * (b - i) / 2ull);
    uint32_t q = p;
    const uint32_t q_end = p_end;
    uint32_t *lo_q = lo + q;
    uint32_t *hi_q = hi + q;

    // the rank table and the packed strings come from the kernels before this one
    wait_previous_grid();
    const uint32_t m = meta[0];
    if constexpr (!WIDE) {
        for (uint32_t c = threadIdx.x; c <= 64u; c += blockDim.x) {
            uint32_t r = c >> log2_bits;
            r = r < m ? r : m;
            tab[c] = make_uint2(r >= K ? ranks_g[r - K] + 1u : 0u, r < m ? ranks_g[r] : T);
        }
    } else {
        for (uint32_t r = threadIdx.x; r < m; r += blockDim.x) ranks[r] = ranks_g[r];
    }
    __syncthreads();
    if (!active) return;

    uint32_t row = 0xFFFFFFFFu;  // row whose string a0n (or a0, a1) holds
    unsigned long long a0n = 0ull;
    uint4 a0 = make_uint4(0u, 0u, 0u, 0u), a1 = a0;
    for (;;) {
        if (!in_bounds(i < j && j < n, status)) break;
        if (i != row) {
            if constexpr (!WIDE) {
                a0n = __ldg(reinterpret_cast<const unsigned long long *>(packed) + i * (kPackWords / 2u));
            } else {
                a0 = __ldg(reinterpret_cast<const uint4 *>(packed) + i * (kPackWords / 4u));
                a1 = __ldg(reinterpret_cast<const uint4 *>(packed) + i * (kPackWords / 4u) + 1u);
            }
            row = i;
        }
        if constexpr (!WIDE) {
            const unsigned long long x =
                __ldg(reinterpret_cast<const unsigned long long *>(packed) + j * (kPackWords / 2u)) ^ a0n;
            const uint2 bound = tab[__clzll(static_cast<long long>(x))];  // first differing bit, 64: none
            __stcs(lo_q, bound.x);
            __stcs(hi_q, bound.y);
        } else {
            const uint4 b0 = __ldg(reinterpret_cast<const uint4 *>(packed) + j * (kPackWords / 4u));
            const uint4 b1 = __ldg(reinterpret_cast<const uint4 *>(packed) + j * (kPackWords / 4u) + 1u);
            const uint32_t x[kPackWords] = {b0.x ^ a0.x, b0.y ^ a0.y, b0.z ^ a0.z, b0.w ^ a0.w,
                                            b1.x ^ a1.x, b1.y ^ a1.y, b1.z ^ a1.z, b1.w ^ a1.w};
            uint32_t first_bit = 0xFFFFFFFFu;
#pragma unroll
            for (int w = kPackWords - 1; w >= 0; --w)
                if (x[w] != 0u) first_bit = 32u * w + (__ffs(x[w]) - 1u);
            uint32_t l, h;
            if (first_bit == 0xFFFFFFFFu) {
                h = T;
                l = m >= K ? ranks[m - K] + 1u : 0u;
            } else {
                uint32_t istar = first_bit >> log2_bits;  // first mismatch, 0-based
                if (!in_bounds(istar < m, status)) istar = 0u;
                h = ranks[istar];
                l = istar >= K ? ranks[istar - K] + 1u : 0u;
            }
            __stcs(lo_q, l);
            __stcs(hi_q, h);
        }
        q += 32u;
        if (q >= q_end) break;
        lo_q += 32;
        hi_q += 32;
        j += 32u;
        while (j >= n) {  // past the end of row i: pair (i + 1, i + 2) follows (i, n - 1)
            j = j - n + i + 2u;
            ++i;
        }
    }
}

// pack + pair launches shared by the allocating and the fixed-scratch entry points; both are
// programmatically dependent launches (each starts its independent set-up while the kernel
// before it finishes)
cudaError_t launch_pack_and_pairs(const uint32_t *pop, uint32_t record_words, uint32_t n_agents,
                           const uint32_t *d_ids, uint32_t n, const uint32_t *order,
                           const uint32_t *ranks, const uint32_t *meta, uint32_t sites,
                           uint32_t bits, uint32_t K, uint32_t T, uint32_t *packed,
                           uint32_t *d_lo, uint32_t *d_hi, int *status, cudaStream_t stream)
{
    // sites * bits <= 64: every rank-ordered string fits in its first 64 bits (bit-reversed)
    const bool narrow = sites * bits <= 64u;
    const cudaError_t e = launch_dependent(pack_kernel, (n + 7u) / 8u, 256, stream, pop,
                                           record_words, n_agents, d_ids, n, order, meta, bits, T,
                                           packed, status, narrow ? 1u : 0u);
    if (e != cudaSuccess) return e;
    // enough resident blocks for the whole GPU, each thread then sweeping several pairs
    const unsigned long long pairs = static_cast<unsigned long long>(n) * (n - 1u) / 2ull;
    const unsigned long long want = (pairs + kPairThreads - 1) / kPairThreads;
    const uint32_t grid = static_cast<uint32_t>(want < kPairGrid ? want : kPairGrid);
    const unsigned long long n_warps = static_cast<unsigned long long>(grid) * (kPairThreads / 32);
    const uint32_t per_warp =
        static_cast<uint32_t>(((pairs + n_warps - 1ull) / n_warps + 31ull) / 32ull * 32ull);
    const uint32_t log2_bits = bits == 1u ? 0u : bits == 2u ? 1u : bits == 4u ? 2u : 3u;
    return launch_dependent(narrow ? pair_kernel<false> : pair_kernel<true>, grid,
                            kPairThreads, stream, packed, n, ranks, meta, log2_bits, K, T, per_warp,
                            d_lo, d_hi, status);
}

uint32_t margin(uint32_t bits)
{
    // smallest K with 2^(-bits*K) < 0.05, i.e. bits*K > log2(20) = 4.32
    uint32_t K = 1;
    while (bits * K <= 4u) ++K;
    return K;
}

// ---------------------------------------------------------------------------------------
// Mixed counters (asynchronous runs): agents i and j may hold different counters Ti, Tj.  A
// rank, once deposited, stays at its own site until overwritten, so the ranks retained at
// both counters are exactly the sites whose holder tables at Ti and Tj agree.
//   1. counter_kernel: each sampled agent's counter.
//   2. table_kernel  : one block per sampled agent: the holder table at its counter, in
//                      closed form as for the synchronous table; table row i (rank + 1 per
//                      site, 0: empty).
//   3. mixed_pair_kernel: 16 x 16 pairs per block with the 32 agents' tables and surfaces in
//                      shared memory; one thread per pair makes two passes over the sites:
//                      (a) the smallest common rank whose differentiae differ (hi), (b) the
//                      K largest common ranks below it (lo = the K-th + 1).
// ---------------------------------------------------------------------------------------
constexpr int kMixTile = 16;

struct MixedLayout {
    uint32_t *cnt;     // [n] counters of the sampled agents
    uint32_t *tables;  // [n][S] rank + 1 held by each site at the agent's counter
};

size_t mixed_scratch_bytes(uint32_t S, uint32_t n)
{
    return align_up(static_cast<size_t>(n) * 4u, 256) + align_up(static_cast<size_t>(n) * S * 4u, 256);
}

MixedLayout carve_mixed(void *scratch, uint32_t n)
{
    uint8_t *p = static_cast<uint8_t *>(scratch);
    MixedLayout l;
    l.cnt = reinterpret_cast<uint32_t *>(p);
    l.tables = reinterpret_cast<uint32_t *>(p + align_up(static_cast<size_t>(n) * 4u, 256));
    return l;
}

__global__ void counter_kernel(const uint32_t *__restrict__ pop, uint32_t record_words,
                               uint32_t n_agents, const uint32_t *__restrict__ ids, uint32_t n,
                               uint32_t *__restrict__ cnt, int *__restrict__ status)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t id = ids[i];
    uint32_t c = 0;
    if (id >= n_agents) atomicCAS(status, GA_OK, GA_EINVAL);
    else c = pop[static_cast<size_t>(id) * record_words + 1];
    cnt[i] = c;
}

__global__ void __launch_bounds__(256)
table_kernel(const uint32_t *__restrict__ cnt, uint32_t *__restrict__ tables, uint32_t policy,
             uint32_t log2_sites, uint32_t sites)
{
    __shared__ uint32_t h[256];
    const uint32_t i = blockIdx.x, k = threadIdx.x;
    h[k] = 0u;
    __syncthreads();
    if (k < sites) {
        uint32_t site = 0;
        const uint32_t r1 = retained_entry(policy, log2_sites, sites, cnt[i], k, site);
        if (r1 != 0u) h[site] = r1;
    }
    __syncthreads();
    if (k < sites) tables[static_cast<size_t>(i) * sites + k] = h[k];
}

// Block (x, y): rows i in tile y, columns j in tile x (tiles below the diagonal exit).
__global__ void __launch_bounds__(kMixTile * kMixTile)
mixed_pair_kernel(const uint32_t *__restrict__ pop, uint32_t record_words, uint32_t n_agents,
                  const uint32_t *__restrict__ ids, uint32_t n, const uint32_t *__restrict__ cnt,
                  const uint32_t *__restrict__ tables, uint32_t sites, uint32_t bits, uint32_t K,
                  uint32_t *__restrict__ lo, uint32_t *__restrict__ hi)
{
    constexpr int kSurfPad = kPackWords + 1;
    __shared__ uint32_t tab[2 * kMixTile][256 + 1];
    __shared__ uint32_t surf[2 * kMixTile][kSurfPad];
    __shared__ uint32_t count[2 * kMixTile];
    if (blockIdx.x < blockIdx.y) return;  // uniform across the block
    const uint32_t i0 = blockIdx.y * kMixTile, j0 = blockIdx.x * kMixTile;
    // rows 0..15: agents i0 + r; rows 16..31: agents j0 + r
    for (uint32_t idx = threadIdx.x; idx < 2u * kMixTile * sites; idx += blockDim.x) {
        const uint32_t row = idx / sites, k = idx - row * sites;
        const uint32_t a = row < kMixTile ? i0 + row : j0 + row - kMixTile;
        tab[row][k] = a < n ? tables[static_cast<size_t>(a) * sites + k] : 0u;
    }
    for (uint32_t idx = threadIdx.x; idx < 2u * kMixTile * kPackWords; idx += blockDim.x) {
        const uint32_t row = idx / kPackWords, w = idx - row * kPackWords;
        const uint32_t a = row < kMixTile ? i0 + row : j0 + row - kMixTile;
        uint32_t v = 0;
        if (a < n && w + 2u < record_words) {
            const uint32_t id = ids[a];
            if (id < n_agents) v = pop[static_cast<size_t>(id) * record_words + 2u + w];
        }
        surf[row][w] = v;
    }
    if (threadIdx.x < 2u * kMixTile) {
        const uint32_t row = threadIdx.x;
        const uint32_t a = row < kMixTile ? i0 + row : j0 + row - kMixTile;
        count[row] = a < n ? cnt[a] : 0u;
    }
    __syncthreads();

    const uint32_t ty = threadIdx.x / kMixTile, tx = threadIdx.x % kMixTile;
    const uint32_t i = i0 + ty, j = j0 + tx;
    if (!(i < j && j < n)) return;
    const uint32_t *ta = tab[ty], *tb = tab[kMixTile + tx];
    const uint32_t *sa = surf[ty], *sb = surf[kMixTile + tx];
    const uint32_t dmask = (1u << bits) - 1u;

    // (a) smallest common rank (+1) whose differentiae differ
    bool mismatch = false;
    uint32_t hmin = 0xFFFFFFFFu;
    for (uint32_t k = 0; k < sites; ++k) {
        const uint32_t va = ta[k];
        if (va == 0u || va != tb[k]) continue;
        const uint32_t pos = k * bits;
        const uint32_t da = (sa[pos >> 5] >> (pos & 31u)) & dmask;
        const uint32_t db = (sb[pos >> 5] >> (pos & 31u)) & dmask;
        if (da != db && (!mismatch || va < hmin)) {
            hmin = va;
            mismatch = true;
        }
    }
    // (b) the K largest common ranks (+1) below it, descending
    uint32_t top[5] = {0u, 0u, 0u, 0u, 0u};
    for (uint32_t k = 0; k < sites; ++k) {
        uint32_t v = ta[k];
        if (v == 0u || v != tb[k] || (mismatch && v >= hmin)) continue;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const uint32_t t = top[q];
            const bool up = v > t;
            top[q] = up ? v : t;
            v = up ? t : v;
        }
    }
    const uint32_t Ta = count[ty], Tb = count[kMixTile + tx];
    const uint32_t h = mismatch ? hmin - 1u : (Ta < Tb ? Ta : Tb);
    const uint32_t l = top[K - 1u];  // rank + 1 of the K-th largest, 0 if fewer than K
    const size_t p = static_cast<size_t>(i) * (2ull * n - i - 1ull) / 2ull + (j - i - 1u);
    __stcs(&lo[p], l);
    __stcs(&hi[p], h);
}

}  // namespace

size_t mrca_scratch_bytes(const ga_run *run, uint32_t n)
{
    const uint32_t S = run->cfg.surface_sites;
    if (run->cfg.mode != GA_SYNC) return mixed_scratch_bytes(S, n);
    return sync_scratch_bytes(S, n);
}

namespace {

cudaError_t launch_mrca_mixed(ga_run *run, const uint32_t *d_ids, uint32_t n, uint32_t *d_lo,
                              uint32_t *d_hi, void *scratch)
{
    const uint32_t S = run->cfg.surface_sites, b = run->cfg.differentia_bits;
    MixedLayout l = carve_mixed(scratch, n);
    const uint32_t *pop = reinterpret_cast<const uint32_t *>(run->pop[run->cur]);
    const uint32_t rw = run->record_bytes / 4u;
    counter_kernel<<<(n + 255u) / 256u, 256, 0, run->stream>>>(pop, rw, run->n_agents, d_ids, n,
                                                               l.cnt, run->d_status);
    table_kernel<<<n, 256, 0, run->stream>>>(l.cnt, l.tables, run->cfg.curation, run->log2_sites, S);
    const uint32_t tiles = (n + kMixTile - 1) / kMixTile;
    mixed_pair_kernel<<<dim3(tiles, tiles), kMixTile * kMixTile, 0, run->stream>>>(
        pop, rw, run->n_agents, d_ids, n, l.cnt, l.tables, S, b, margin(b), d_lo, d_hi);
    run->launches += 3;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mrca(ga_run *run, const uint32_t *d_ids, uint32_t n, uint32_t *d_lo,
                        uint32_t *d_hi, void *scratch)
{
    if (run->cfg.mode != GA_SYNC) return launch_mrca_mixed(run, d_ids, n, d_lo, d_hi, scratch);
    const uint32_t S = run->cfg.surface_sites, b = run->cfg.differentia_bits;
    const uint32_t T = static_cast<uint32_t>(run->generation);
    MrcaLayout l = carve(scratch, S);
    cudaError_t e0 = launch_rank_table(l.order, l.ranks, l.meta, run->cfg.curation,
                                       run->log2_sites, S, T, run->stream);
    if (e0 != cudaSuccess) return e0;
    run->launches += 1;
    const cudaError_t e = launch_pack_and_pairs(
        reinterpret_cast<const uint32_t *>(run->pop[run->cur]), run->record_bytes / 4u,
        run->n_agents, d_ids, n, l.order, l.ranks, l.meta, S, b, margin(b), T, l.packed, d_lo,
        d_hi, run->d_status, run->stream);
    if (e != cudaSuccess) return e;
    run->launches += 2;
    return cudaGetLastError();
}

}  // namespace ga

// ---------------------------------------------------------------------------------------
// ga_mrca_bounds_noalloc: the same MRCA kernels with their scratch held in a fixed
// device array instead of memory allocated per call, for callers that cannot allocate
// device memory (see include/ga.h).
//
// The array is a file-scope __device__ variable, so every GPU that loads this library holds
// its own copy until the process exits.  In host code the name g_mrca_fixed_scratch is only
// a host-side stand-in for the symbol, never a device address; each call looks the address
// up with cudaGetSymbolAddress, with the caller's device current, and passes it to the
// kernels (a lookup per call stays right after a device reset reloads the module, which a
// cached address would not).  Every call on a device reuses the same array: the status word
// is cleared at the start of each call, the rank table and strings are fully rewritten
// before they are read.
// ---------------------------------------------------------------------------------------
namespace ga {
namespace {

constexpr uint32_t kFixedMaxSample = 4096;    // largest n accepted
constexpr uint32_t kFixedMaxSites = 256;      // S * b <= 256 bits
constexpr size_t kFixedStatusBytes = 256;     // device status word, padded
// status, then the layout carve() gives the per-call scratch, sized for S = 256, n = 4096:
// 256 + 2 x 1,024 + 256 + 4,096 x 32 = 133,632 bytes
constexpr size_t kFixedScratchBytes = kFixedStatusBytes + 2 * 1024 + 256 +
                                      static_cast<size_t>(kFixedMaxSample) * kPackWords * 4;

static __device__ __align__(256) unsigned char g_mrca_fixed_scratch[kFixedScratchBytes];

}  // namespace
}  // namespace ga

extern "C" int ga_mrca_bounds_noalloc(const void *d_records, uint32_t record_bytes,
                                      uint32_t n_agents, uint32_t curation,
                                      uint32_t surface_sites, uint32_t differentia_bits,
                                      uint32_t generation, const uint32_t *d_agent_ids,
                                      uint32_t n, uint32_t *d_lo, uint32_t *d_hi, void *stream)
{
    using namespace ga;
    const uint32_t S = surface_sites, b = differentia_bits;
    if (!d_records || !d_agent_ids || !d_lo || !d_hi) return GA_EINVAL;
    if (n < 2 || n > kFixedMaxSample) return GA_EINVAL;
    if (curation > GA_HYBRID) return GA_EINVAL;
    if (S == 0u || (S & (S - 1u)) != 0u || S < (curation == GA_HYBRID ? 8u : 4u)) return GA_EINVAL;
    if (!(b == 1u || b == 2u || b == 4u || b == 8u) || S * b > kFixedMaxSites) return GA_EINVAL;
    const uint32_t words = (S * b + 31u) / 32u;
    if (record_bytes != (8u + 4u * words + 15u) / 16u * 16u || n_agents == 0u) return GA_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_records) % 16u != 0u) return GA_EINVAL;
    static_assert(kFixedStatusBytes + 2 * 1024 + 256 + kFixedMaxSample * kPackWords * 4 <=
                      kFixedScratchBytes, "fixed scratch too small for its largest call");

    // an error left pending by earlier, unrelated work on this thread is not this call's
    cudaGetLastError();
    void *base = nullptr;
    if (cudaGetSymbolAddress(&base, g_mrca_fixed_scratch) != cudaSuccess || base == nullptr) {
        cudaGetLastError();
        return GA_ECUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *status = static_cast<int *>(base);
    MrcaLayout l = carve(static_cast<uint8_t *>(base) + kFixedStatusBytes, S);
    uint32_t log2_sites = 0;
    while ((1u << log2_sites) < S) ++log2_sites;

    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return GA_ECUDA;
    if (launch_rank_table(l.order, l.ranks, l.meta, curation, log2_sites, S, generation, st) !=
        cudaSuccess)
        return GA_ECUDA;
    if (launch_pack_and_pairs(static_cast<const uint32_t *>(d_records), record_bytes / 4u,
                              n_agents, d_agent_ids, n, l.order, l.ranks, l.meta, S, b, margin(b),
                              generation, l.packed, d_lo, d_hi, status, st) != cudaSuccess)
        return GA_ECUDA;
    int device_status = GA_OK;
    if (cudaMemcpyAsync(&device_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GA_ECUDA;
    return device_status;
}
