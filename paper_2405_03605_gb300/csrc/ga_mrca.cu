// ga_mrca.cu -- pairwise MRCA bounds over sampled end-state agents (post hoc relatedness
// estimation from hstrat markers, Fig. 1 caption of the paper).
//
// Pipeline (all on the run's stream).  Strings of at most 64 bits (S b <= 64), two launches:
//   1. pack64_kernel : one thread per sampled agent; each block first finds the ranks the
//                      surface retains at counter T in closed form (no replay of ranks
//                      0..T-1: one thread per retained rank or site) and sorts the occupied
//                      sites by rank, r_0 < ... < r_{m-1} (block 0 also writes them out for
//                      the pair kernel); each thread then gathers its agent's differentiae in
//                      rank order into one 64-bit string, stored bit-reversed (the first rank
//                      index at bit 63), 8 bytes per agent.
//   2. pair64_kernel : one thread per pair (i, j), j > i, in output order; the count of
//                      leading zeros of packed[i] ^ packed[j] gives the first mismatching
//                      rank index i*, from which hi = r_{i*} and lo = r_{i*-K} + 1 (0 if
//                      i* < K); with no mismatch hi = T, lo = r_{m-K} + 1 (0 if m < K).
// Wider strings (up to 256 bits), three launches: rank_table_kernel (the same closed form,
// once), pack_kernel (one warp per agent, 8 words), pair_kernel (the first nonzero word of the
// XOR, then the same rules).
// The pair kernels are bound by their output: 8 bytes (lo, hi) per pair, written once with
// streaming stores.
#include "ga_device.cuh"
#include "ga_internal.h"

namespace ga {

namespace {

constexpr uint32_t kPackWords = 8;  // 256-bit rank-ordered strings
constexpr int kPairThreads = 256;
constexpr unsigned long long kPairGrid = 152ull * 8ull;  // 8 resident blocks on each of 152 SMs
constexpr uint32_t kPack64Threads = 128;  // >= 64 sites; small blocks spread a sample over SMs


struct MrcaLayout {
    uint32_t *order;   // [S]  sites sorted by rank
    uint32_t *ranks;   // [S]  sorted ranks
    uint32_t *meta;    // [4]  m
    uint32_t *packed;  // [n][kPackWords] (strings of at most 64 bits: [n] 64-bit words)
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
__global__ void pack_kernel(const uint32_t *__restrict__ pop, uint32_t record_words,
                            uint32_t n_agents, const uint32_t *__restrict__ ids, uint32_t n,
                            const uint32_t *__restrict__ order, const uint32_t *__restrict__ meta,
                            uint32_t bits, uint32_t T, uint32_t *__restrict__ packed,
                            int *__restrict__ status)
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
    if (lane < kPackWords) packed[static_cast<size_t>(a) * kPackWords + lane] = word_out;
}

// Row and column of pair p in output order: row i holds pairs off(i) <= p < off(i + 1) with
// off(i) = i (2n - i - 1) / 2.  A single-precision root of i^2 - (2n - 1) i + 2p = 0 from the
// exact 64-bit discriminant is within one row; integer comparisons correct it.
__device__ __forceinline__ void first_pair(uint32_t n, uint32_t p, uint32_t &i, uint32_t &j)
{
    const unsigned long long b = 2ull * n - 1ull;  // off(r) = r (b - r) / 2
    const float est = (static_cast<float>(b) - sqrtf(static_cast<float>(b * b - 8ull * p))) * 0.5f;
    i = est > 0.0f ? static_cast<uint32_t>(est) : 0u;
    if (i > n - 2u) i = n - 2u;
    while (i > 0u && static_cast<unsigned long long>(i) * (b - i) / 2ull > p) --i;
    while (i + 2u < n && static_cast<unsigned long long>(i + 1u) * (b - i - 1u) / 2ull <= p) ++i;
    j = i + 1u + static_cast<uint32_t>(p - static_cast<unsigned long long>(i) * (b - i) / 2ull);
}

// Strings of at most 64 bits: one thread per sampled agent.  Each block first builds the
// rank order itself (threads k < S: retained entry k in closed form, placed at its site; the
// occupied sites then sorted by rank), so no launch precedes this one; block 0 also writes the
// sorted ranks and m for the pair kernel.  Thread a then reads agent ids[a]'s 64-bit surface
// (differentia at site k in bits [k b, k b + b)) and assembles the string with differentia
// index i at bits [i b, i b + b), stored bit-reversed: the first rank index at bit 63, so a
// pair's first mismatch is the count of leading zeros of the XOR.  Bits past m b stay zero.
__global__ void __launch_bounds__(kPack64Threads)
pack64_kernel(const uint32_t *__restrict__ pop, uint32_t record_words, uint32_t n_agents,
              const uint32_t *__restrict__ ids, uint32_t n, uint32_t policy, uint32_t log2_sites,
              uint32_t sites, uint32_t bits, uint32_t T, uint32_t *__restrict__ ranks,
              uint32_t *__restrict__ meta, unsigned long long *__restrict__ packed,
              int *__restrict__ status)
{
    __shared__ __align__(16) uint32_t h[64];
    __shared__ uint32_t shift[64];  // surface bit offset of differentia index i
    release_next_grid();  // the pair kernel may start its index set-up
    const uint32_t k = threadIdx.x;
    const uint32_t a = blockIdx.x * blockDim.x + k;
    const uint32_t id = a < n ? ids[a] : 0u;
    const bool ok = a < n && id < n_agents;
    const uint32_t *rec = pop + static_cast<size_t>(ok ? id : 0u) * record_words;
    const uint32_t counter = ok ? rec[1] : T;
    const uint32_t w0 = ok ? rec[2] : 0u;
    const uint32_t w1 = (ok && record_words > 3u) ? rec[3] : 0u;
    if (k < 64u) h[k] = 0u;
    __syncthreads();
    if (k < sites) {
        uint32_t site = 0;
        const uint32_t r1 = retained_entry(policy, log2_sites, sites, T, k, site);
        if (r1 != 0u && in_bounds(site < sites, status)) h[site] = r1;
    }
    __syncthreads();
    const uint32_t mine = k < sites ? h[k] : 0u;
    const uint32_t m = static_cast<uint32_t>(__syncthreads_count(mine != 0u));
    if (mine != 0u) {  // position among the occupied sites, all 64 entries read at once
        uint32_t pos = 0;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const uint4 v = reinterpret_cast<const uint4 *>(h)[q];
            pos += (v.x != 0u && v.x < mine) + (v.y != 0u && v.y < mine) +
                   (v.z != 0u && v.z < mine) + (v.w != 0u && v.w < mine);
        }
        shift[pos] = k * bits;
        if (blockIdx.x == 0) ranks[pos] = mine - 1u;
    }
    if (blockIdx.x == 0 && k == 0) meta[0] = m;
    __syncthreads();
    if (a >= n) return;
    if (!ok) {
        atomicCAS(status, GA_OK, GA_EINVAL);
        packed[a] = 0ull;
        return;
    }
    if (counter != T) atomicCAS(status, GA_OK, GA_ESTATE);
    // differentia index i goes to bits [i b, i b + b) of (o1 : o0); a differentia never
    // straddles a surface word (b divides 32)
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t o0 = 0u, o1 = 0u;
#pragma unroll 8
    for (uint32_t i = 0; i < m; ++i) {
        const uint32_t sh = shift[i];
        const uint32_t v = (((sh & 32u) ? w1 : w0) >> (sh & 31u)) & mask;
        const uint32_t ob = i * bits;
        if (ob & 32u) o1 |= v << (ob & 31u);
        else o0 |= v << (ob & 31u);
    }
    // bit-reversed 64-bit string: reverse(o1 : o0) = reverse(o0) : reverse(o1)
    packed[a] = (static_cast<unsigned long long>(__brev(o0)) << 32) | __brev(o1);
}

// Pairs of 64-bit strings, in output order, each warp a contiguous stretch of them: lane t
// takes pairs base + t, base + t + 32, ... (the row of its first pair found as in pair_kernel
// below), steps 32 pairs at a time and reloads row i's string only when a step carries it into
// the next rows.  tab[c] holds both bounds for a leading-zero count c in [0, 64]:
// i* = min(c / b, m), tab[c] = (i* >= K ? r_{i*-K} + 1 : 0, i* < m ? r_{i*} : T).
__global__ void __launch_bounds__(kPairThreads)
pair64_kernel(const unsigned long long *__restrict__ packed, uint32_t n,
              const uint32_t *__restrict__ ranks_g, const uint32_t *__restrict__ meta,
              uint32_t log2_bits, uint32_t K, uint32_t T, uint32_t per_warp,
              uint32_t *__restrict__ lo, uint32_t *__restrict__ hi, int *__restrict__ status)
{
    __shared__ uint2 tab[65];
    const uint32_t n_pairs = n * (n - 1u) / 2u;
    const uint32_t warp = (blockIdx.x * kPairThreads + threadIdx.x) >> 5;
    const unsigned long long w_end = static_cast<unsigned long long>(warp + 1u) * per_warp;
    const uint32_t p_end = w_end < n_pairs ? static_cast<uint32_t>(w_end) : n_pairs;
    const unsigned long long p0 = static_cast<unsigned long long>(warp) * per_warp + (threadIdx.x & 31u);
    const bool active = p0 < p_end;
    const uint32_t p = active ? static_cast<uint32_t>(p0) : 0u;
    uint32_t i = 0, j = 1;
    first_pair(n, p, i, j);

    wait_previous_grid();  // ranks, m and the strings come from pack64_kernel
    const uint32_t m = meta[0];
    for (uint32_t c = threadIdx.x; c <= 64u; c += blockDim.x) {
        uint32_t r = c >> log2_bits;
        r = r < m ? r : m;
        tab[c] = make_uint2(r >= K ? ranks_g[r - K] + 1u : 0u, r < m ? ranks_g[r] : T);
    }
    __syncthreads();
    if (!active || !in_bounds(i < j && j < n, status)) return;

    unsigned long long row = __ldg(packed + i);
    for (uint32_t q = p;;) {
        const unsigned long long x = __ldg(packed + j) ^ row;
        const uint2 bound = tab[__clzll(static_cast<long long>(x))];  // first differing bit, 64: none
        __stcs(lo + q, bound.x);
        __stcs(hi + q, bound.y);
        q += 32u;
        if (q >= p_end) break;
        j += 32u;
        if (j >= n) {  // past the end of row i: pair (i + 1, i + 2) follows (i, n - 1)
            do {
                j = j - n + i + 2u;
                ++i;
            } while (j >= n);
            if (!in_bounds(i < j, status)) break;
            row = __ldg(packed + i);
        }
    }
}

// Pairs of strings wider than 64 bits, in output order, each warp a contiguous stretch of
// them: lane t takes pairs base + t, base + t + 32, ..., so a warp's (lo, hi) writes are
// contiguous.  A lane finds the row of its first pair once (first_pair), then steps 32 pairs
// at a time, carrying into the next rows when j passes n - 1, and reloads row i's string only
// when i changes.  Pair indices fit 32 bits (n <= 65536: fewer than 2^31 pairs).  The first
// set bit of packed[i] ^ packed[j] (the first nonzero word, then its lowest set bit) gives the
// first mismatching rank index i*.  With 0-based sorted ranks r_0 < ... < r_{m-1}, a mismatch
// at index i* gives hi = r_{i*}, lo = r_{i*-K} + 1 (0 if i* < K), and no mismatch hi = T,
// lo = r_{m-K} + 1.
__global__ void __launch_bounds__(kPairThreads)
pair_kernel(const uint32_t *__restrict__ packed, uint32_t n, const uint32_t *__restrict__ ranks_g,
            const uint32_t *__restrict__ meta, uint32_t log2_bits, uint32_t K, uint32_t T,
            uint32_t per_warp, uint32_t *__restrict__ lo, uint32_t *__restrict__ hi,
            int *__restrict__ status)
{
    __shared__ uint32_t ranks[256];
    // pairs [warp * per_warp, (warp + 1) * per_warp) of n (n - 1) / 2 (per_warp: a multiple of
    // 32 chosen on the host so that the grid covers every pair)
    const uint32_t n_pairs = n * (n - 1u) / 2u;
    const uint32_t warp = (blockIdx.x * kPairThreads + threadIdx.x) >> 5;
    const unsigned long long w_end = static_cast<unsigned long long>(warp + 1u) * per_warp;
    const uint32_t p_end = w_end < n_pairs ? static_cast<uint32_t>(w_end) : n_pairs;
    const unsigned long long p0 = static_cast<unsigned long long>(warp) * per_warp + (threadIdx.x & 31u);
    const bool active = p0 < p_end;
    const uint32_t p = active ? static_cast<uint32_t>(p0) : 0u;
    uint32_t i = 0, j = 1;
    first_pair(n, p, i, j);
    uint32_t q = p;
    uint32_t *lo_q = lo + q;
    uint32_t *hi_q = hi + q;

    // the rank table and the packed strings come from the kernels before this one
    wait_previous_grid();
    const uint32_t m = meta[0];
    for (uint32_t r = threadIdx.x; r < m; r += blockDim.x) ranks[r] = ranks_g[r];
    __syncthreads();
    if (!active) return;

    uint32_t row = 0xFFFFFFFFu;  // row whose string a0, a1 hold
    uint4 a0 = make_uint4(0u, 0u, 0u, 0u), a1 = a0;
    for (;;) {
        if (!in_bounds(i < j && j < n, status)) break;
        if (i != row) {
            a0 = __ldg(reinterpret_cast<const uint4 *>(packed) + i * (kPackWords / 4u));
            a1 = __ldg(reinterpret_cast<const uint4 *>(packed) + i * (kPackWords / 4u) + 1u);
            row = i;
        }
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
        q += 32u;
        if (q >= p_end) break;
        lo_q += 32;
        hi_q += 32;
        j += 32u;
        while (j >= n) {  // past the end of row i: pair (i + 1, i + 2) follows (i, n - 1)
            j = j - n + i + 2u;
            ++i;
        }
    }
}

// Grid and stretch length of a pair kernel: enough resident blocks for the whole GPU, each
// warp then sweeping a contiguous stretch of pairs (a multiple of 32).
void pair_grid(uint32_t n, uint32_t &grid, uint32_t &per_warp)
{
    const unsigned long long pairs = static_cast<unsigned long long>(n) * (n - 1u) / 2ull;
    const unsigned long long want = (pairs + kPairThreads - 1) / kPairThreads;
    grid = static_cast<uint32_t>(want < kPairGrid ? want : kPairGrid);
    const unsigned long long n_warps = static_cast<unsigned long long>(grid) * (kPairThreads / 32);
    per_warp = static_cast<uint32_t>(((pairs + n_warps - 1ull) / n_warps + 31ull) / 32ull * 32ull);
}

uint32_t margin(uint32_t bits);

// Every launch of one synchronous MRCA call (shared by the allocating and the fixed-scratch
// entry points): two for strings of at most 64 bits (pack64, then pair64 as a programmatically
// dependent launch), three otherwise (rank table, then pack and pair as dependent launches).
cudaError_t launch_sync_mrca(const uint32_t *pop, uint32_t record_words, uint32_t n_agents,
                             const uint32_t *d_ids, uint32_t n, const MrcaLayout &l,
                             uint32_t policy, uint32_t log2_sites, uint32_t sites, uint32_t bits,
                             uint32_t T, uint32_t *d_lo, uint32_t *d_hi, int *status,
                             cudaStream_t stream, uint32_t &launches)
{
    const uint32_t K = margin(bits);
    const uint32_t log2_bits = bits == 1u ? 0u : bits == 2u ? 1u : bits == 4u ? 2u : 3u;
    uint32_t grid = 0, per_warp = 0;
    pair_grid(n, grid, per_warp);
    unsigned long long *packed64 = reinterpret_cast<unsigned long long *>(l.packed);
    if (sites * bits <= 64u) {
        pack64_kernel<<<(n + kPack64Threads - 1u) / kPack64Threads, kPack64Threads, 0, stream>>>(
            pop, record_words, n_agents, d_ids, n, policy, log2_sites, sites, bits, T, l.ranks,
            l.meta, packed64, status);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        launches += 1;
        e = launch_dependent(pair64_kernel, grid, kPairThreads, stream,
                             static_cast<const unsigned long long *>(packed64), n,
                             static_cast<const uint32_t *>(l.ranks),
                             static_cast<const uint32_t *>(l.meta), log2_bits, K, T, per_warp,
                             d_lo, d_hi, status);
        if (e == cudaSuccess) launches += 1;
        return e;
    }
    cudaError_t e = launch_rank_table(l.order, l.ranks, l.meta, policy, log2_sites, sites, T, stream);
    if (e != cudaSuccess) return e;
    launches += 1;
    e = launch_dependent(pack_kernel, (n + 7u) / 8u, 256, stream, pop, record_words, n_agents,
                         d_ids, n, static_cast<const uint32_t *>(l.order),
                         static_cast<const uint32_t *>(l.meta), bits, T, l.packed, status);
    if (e != cudaSuccess) return e;
    launches += 1;
    e = launch_dependent(pair_kernel, grid, kPairThreads, stream,
                         static_cast<const uint32_t *>(l.packed), n,
                         static_cast<const uint32_t *>(l.ranks),
                         static_cast<const uint32_t *>(l.meta), log2_bits, K, T, per_warp, d_lo,
                         d_hi, status);
    if (e == cudaSuccess) launches += 1;
    return e;
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
    uint32_t launches = 0;
    const cudaError_t e = launch_sync_mrca(
        reinterpret_cast<const uint32_t *>(run->pop[run->cur]), run->record_bytes / 4u,
        run->n_agents, d_ids, n, l, run->cfg.curation, run->log2_sites, S, b, T, d_lo, d_hi,
        run->d_status, run->stream, launches);
    run->launches += launches;
    if (e != cudaSuccess) return e;
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
    uint32_t launches = 0;
    if (launch_sync_mrca(static_cast<const uint32_t *>(d_records), record_bytes / 4u, n_agents,
                         d_agent_ids, n, l, curation, log2_sites, S, b, generation, d_lo, d_hi,
                         status, st, launches) != cudaSuccess)
        return GA_ECUDA;
    int device_status = GA_OK;
    if (cudaMemcpyAsync(&device_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GA_ECUDA;
    return device_status;
}
