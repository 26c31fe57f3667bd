// ga_device.cuh -- device building blocks of the island step: counter-based random draws,
// closed-form curation sites and the agent-record layout.
#pragma once

#include <cstdint>

namespace ga {

// Draw purposes, carried in the high half of the third Philox counter word.
constexpr uint32_t kBirth = 1u;
constexpr uint32_t kFounder = 2u;

constexpr uint32_t kSteady = 0u, kTilted = 1u, kHybrid = 2u;

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11).  Each round multiplies counter words 0 and 2 by the
// two Philox multipliers (one 32x32->64 product each), swaps the halves into place, XORs in
// the other counter words and the round key; the key advances by the two Weyl increments.
// The round keys depend only on the seed, so they stay uniform across a warp.
// ---------------------------------------------------------------------------------------
struct Key {
    uint32_t k0, k1;
};

// The ten round keys (key + r * Weyl increment, mod 2^32) depend only on the seed; the
// island step receives them precomputed as kernel parameters, so each round XORs its key
// straight from the constant bank instead of keeping a schedule in registers.
struct RoundKeys {
    uint32_t k0[10], k1[10];
};

inline RoundKeys round_keys(Key key)
{
    RoundKeys rk;
    uint32_t k0 = key.k0, k1 = key.k1;
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = k0;
        rk.k1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return rk;
}

__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        Key key)
{
    uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t a = static_cast<uint64_t>(c0) * 0xD2511F53ull;
        const uint64_t b = static_cast<uint64_t>(c2) * 0xCD9E8D57ull;
        const uint32_t n0 = static_cast<uint32_t>(b >> 32) ^ c1 ^ k0;
        const uint32_t n2 = static_cast<uint32_t>(a >> 32) ^ c3 ^ k1;
        c1 = static_cast<uint32_t>(b);
        c3 = static_cast<uint32_t>(a);
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           const RoundKeys &rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t a = static_cast<uint64_t>(c0) * 0xD2511F53ull;
        const uint64_t b = static_cast<uint64_t>(c2) * 0xCD9E8D57ull;
        const uint32_t n0 = static_cast<uint32_t>(b >> 32) ^ c1 ^ rk.k0[r];
        const uint32_t n2 = static_cast<uint32_t>(a >> 32) ^ c3 ^ rk.k1[r];
        c1 = static_cast<uint32_t>(b);
        c3 = static_cast<uint32_t>(a);
        c0 = n0;
        c2 = n2;
    }
    return make_uint4(c0, c1, c2, c3);
}

// ---------------------------------------------------------------------------------------
// Curation sites in closed form.  -1: the deposit of rank T is not kept.
//
// Steady (S = 2^s sites): ranks below S fill sites in order; in epoch t = bitlen(T) - s a
// rank is kept iff its hanoi value (trailing ones of T) is >= t, and it replaces the oldest
// retained rank of hanoi value t-1.  Following the victim chain back to a rank below S
// clears, at each step, the top set bit p of T together with bit p - s; processing T in
// s-bit chunks from the most significant, the chunk that survives at each level is the
// chunk AND NOT the surviving chunk above it, and the site is the survivor of chunk 0.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int steady_site(uint32_t s, uint32_t T)
{
    const uint32_t S = 1u << s;
    if (T < S) return static_cast<int>(T);
    const uint32_t len = 32u - __clz(T);
    const uint32_t epoch = len - s;
    const uint32_t hanoi = __clz(__brev(~T));  // trailing ones of T
    if (hanoi < epoch) return -1;
    const uint32_t mask = S - 1u;
    uint32_t top = (len - 1u) / s * s;
    uint32_t keep = 0u;
    for (int sh = static_cast<int>(top); sh >= 0; sh -= static_cast<int>(s))
        keep = (T >> sh) & mask & ~keep;
    return static_cast<int>(keep);
}

// Tilted (S sites, L = S/2 levels of two sites): a rank of hanoi value h goes to level
// min(h, L-1); within the level the two sites alternate with the class's occurrence count.
__device__ __forceinline__ int tilted_site(uint32_t S, uint32_t T)
{
    const uint32_t L = S >> 1;
    const uint32_t h = __clz(__brev(~T));
    if (h < L - 1u) return static_cast<int>(2u * h + ((T >> (h + 1u)) & 1u));
    // class hanoi >= L-1: earlier occurrences = (T + 1) / 2^(L-1) - 1 = T >> (L-1), because
    // the low L-1 bits of T are all ones
    return static_cast<int>(2u * (L - 1u) + ((T >> (L - 1u)) & 1u));
}

__device__ __forceinline__ int curation_site(uint32_t policy, uint32_t s, uint32_t S,
                                             uint32_t T)
{
    if (policy == kSteady) return steady_site(s, T);
    if (policy == kTilted) return tilted_site(S, T);
    // hybrid: even ranks -> steady over S/2 at T/2, odd ranks -> S/2 + tilted over S/2
    if ((T & 1u) == 0u) return steady_site(s - 1u, T >> 1);
    return static_cast<int>(S >> 1) + tilted_site(S >> 1, T >> 1);
}

// ---------------------------------------------------------------------------------------
// Torus neighbour of island (y, x) in direction d: 0 north, 1 south, 2 east, 3 west.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t torus_neighbour(uint32_t island, uint32_t d, uint32_t rows,
                                                    uint32_t cols)
{
    uint32_t y = island / cols, x = island - y * cols;
    if (d == 0u) y = (y == 0u) ? rows - 1u : y - 1u;
    else if (d == 1u) y = (y + 1u == rows) ? 0u : y + 1u;
    else if (d == 2u) x = (x + 1u == cols) ? 0u : x + 1u;
    else x = (x == 0u) ? cols - 1u : x - 1u;
    return y * cols + x;
}

}  // namespace ga
