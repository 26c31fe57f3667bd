// ga_device.cuh -- device building blocks of the island step: counter-based random draws,
// closed-form curation sites and the agent-record layout.
#pragma once

#include <cstdint>

// Builds with device checks (libga_debug.so, -DGA_DEVICE_CHECKS=1) test the global-memory
// indices of every kernel before use; a failed test records GA_EBOUNDS (-8) in the status
// word it is given and the access is skipped.  In the normal build the tests compile away.
#ifndef GA_DEVICE_CHECKS
#define GA_DEVICE_CHECKS 0
#endif

namespace ga {

// true when `ok`; otherwise (device-check builds only) records GA_EBOUNDS and returns false
__device__ __forceinline__ bool in_bounds(bool ok, int *status)
{
#if GA_DEVICE_CHECKS
    if (!ok) {
        atomicCAS(status, 0, -8);
        return false;
    }
    return true;
#else
    (void)ok;
    (void)status;
    return true;
#endif
}

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may
// start while the kernel before it on the stream is still running; it does the part of its
// work that needs nothing from that kernel, then waits here (a hardware wait for the previous
// grid's completion and memory flush; a no-op for a kernel launched without the attribute).
__device__ __forceinline__ void wait_previous_grid() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
// Lets the next programmatically dependent kernel on the stream be scheduled now.
__device__ __forceinline__ void release_next_grid() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Draw purposes, carried in the high half of the third Philox counter word.
constexpr uint32_t kBirth = 1u;
constexpr uint32_t kFounder = 2u;

constexpr uint32_t kSteady = 0u, kTilted = 1u, kHybrid = 2u;

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11).  Each round multiplies counter words 0 and 2 by the
// two Philox multipliers (one 32x32->64 product each), swaps the halves into place, XORs in
// the other counter words and the round key; the key advances by the two Weyl increments.
// The round keys depend only on the seed, so they stay uniform across a warp.  Each product
// is written as its low half (a 32-bit multiply) and its high half (__umulhi) rather than as
// one 64-bit product: the same bits, and on sm_103a the island step runs 2% faster in this
// form (101.8 against 104.0 us per generation of 16.8M agents).
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
        const uint32_t alo = c0 * 0xD2511F53u, ahi = __umulhi(c0, 0xD2511F53u);
        const uint32_t blo = c2 * 0xCD9E8D57u, bhi = __umulhi(c2, 0xCD9E8D57u);
        const uint32_t n0 = bhi ^ c1 ^ k0;
        const uint32_t n2 = ahi ^ c3 ^ k1;
        c1 = blo;
        c3 = alo;
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
        const uint32_t alo = c0 * 0xD2511F53u, ahi = __umulhi(c0, 0xD2511F53u);
        const uint32_t blo = c2 * 0xCD9E8D57u, bhi = __umulhi(c2, 0xCD9E8D57u);
        const uint32_t n0 = bhi ^ c1 ^ rk.k0[r];
        const uint32_t n2 = ahi ^ c3 ^ rk.k1[r];
        c1 = blo;
        c3 = alo;
        c0 = n0;
        c2 = n2;
    }
    return make_uint4(c0, c1, c2, c3);
}

// ---------------------------------------------------------------------------------------
// Standard normal deviate from two Philox words (float-fitness model, Sec. 3 "normally
// distributed amount"): Box-Muller z = sqrt(-2 ln u1) cos(2 pi u2) in IEEE single precision,
// every operation an explicitly rounded intrinsic (never fused), so the result is a fixed
// function of the two words:
//   u1 = (top 24 bits of a, + 1) 2^-24 in (0, 1];
//   ln u1: u1 = m 2^e, m in [0.5, 1); ln m = 2 atanh(s), s = (m - 1)/(m + 1), series to s^13;
//   cos(2 pi k 2^-24), k = top 24 bits of b: quadrant k >> 22, angle (k mod 2^22) 2^-22 pi/2,
//   Taylor series of cos (to a^14) and sin (to a^15).
// ---------------------------------------------------------------------------------------
constexpr uint32_t kMutate = 3u;

__device__ __forceinline__ float unit_log_rn(float x)
{
    const uint32_t bits = __float_as_uint(x);
    const int e = static_cast<int>((bits >> 23) & 0xFFu) - 126;
    const float m = __uint_as_float((bits & 0x007FFFFFu) | 0x3F000000u);
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float t = __fmul_rn(s, s);
    float p = static_cast<float>(1.0 / 13.0);
    p = __fadd_rn(__fmul_rn(p, t), static_cast<float>(1.0 / 11.0));
    p = __fadd_rn(__fmul_rn(p, t), static_cast<float>(1.0 / 9.0));
    p = __fadd_rn(__fmul_rn(p, t), static_cast<float>(1.0 / 7.0));
    p = __fadd_rn(__fmul_rn(p, t), static_cast<float>(1.0 / 5.0));
    p = __fadd_rn(__fmul_rn(p, t), static_cast<float>(1.0 / 3.0));
    p = __fadd_rn(__fmul_rn(p, t), 1.0f);
    const float ln_m = __fmul_rn(__fmul_rn(2.0f, s), p);
    return __fadd_rn(__fmul_rn(static_cast<float>(e), static_cast<float>(0.69314718055994530942)),
                     ln_m);
}

__device__ __forceinline__ float turn_cos_rn(uint32_t k)
{
    const uint32_t q = (k >> 22) & 3u;
    const float a = __fmul_rn(__fmul_rn(static_cast<float>(k & 0x3FFFFFu),
                                        static_cast<float>(1.0 / 4194304.0)),
                              static_cast<float>(3.14159265358979323846 / 2.0));
    const float a2 = __fmul_rn(a, a);
    float c = -static_cast<float>(1.0 / 87178291200.0);
    c = __fadd_rn(__fmul_rn(c, a2), static_cast<float>(1.0 / 479001600.0));
    c = __fsub_rn(__fmul_rn(c, a2), static_cast<float>(1.0 / 3628800.0));
    c = __fadd_rn(__fmul_rn(c, a2), static_cast<float>(1.0 / 40320.0));
    c = __fsub_rn(__fmul_rn(c, a2), static_cast<float>(1.0 / 720.0));
    c = __fadd_rn(__fmul_rn(c, a2), static_cast<float>(1.0 / 24.0));
    c = __fsub_rn(__fmul_rn(c, a2), 0.5f);
    c = __fadd_rn(__fmul_rn(c, a2), 1.0f);
    float sn = -static_cast<float>(1.0 / 1307674368000.0);
    sn = __fadd_rn(__fmul_rn(sn, a2), static_cast<float>(1.0 / 6227020800.0));
    sn = __fsub_rn(__fmul_rn(sn, a2), static_cast<float>(1.0 / 39916800.0));
    sn = __fadd_rn(__fmul_rn(sn, a2), static_cast<float>(1.0 / 362880.0));
    sn = __fsub_rn(__fmul_rn(sn, a2), static_cast<float>(1.0 / 5040.0));
    sn = __fadd_rn(__fmul_rn(sn, a2), static_cast<float>(1.0 / 120.0));
    sn = __fsub_rn(__fmul_rn(sn, a2), static_cast<float>(1.0 / 6.0));
    sn = __fadd_rn(__fmul_rn(sn, a2), 1.0f);
    sn = __fmul_rn(sn, a);
    return q == 0u ? c : q == 1u ? -sn : q == 2u ? -c : sn;
}

__device__ __forceinline__ float normal_rn(uint32_t a, uint32_t b)
{
    const float u1 = __fmul_rn(static_cast<float>((a >> 8) + 1u), static_cast<float>(1.0 / 16777216.0));
    const float r = __fsqrt_rn(__fmul_rn(-2.0f, unit_log_rn(u1)));
    return __fmul_rn(r, turn_cos_rn(b >> 8));
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

// Unsigned division by the torus width as a multiply and shifts, with the magic number of
// Granlund and Montgomery ("Division by invariant integers using multiplication", PLDI
// 1994, the round-up method for a 32-bit divisor d >= 2): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((n - t) >> 1)) >> (l - 1) with t = umulhi(m, n).
inline void division_magic(uint32_t d, uint32_t &m, uint32_t &l)
{
    if (d <= 1u) {
        m = 0;
        l = 0;
        return;
    }
    l = 0;
    while ((1ull << l) < d) ++l;
    m = static_cast<uint32_t>((((1ull << 32) * ((1ull << l) - d)) / d) + 1ull);
}

__device__ __forceinline__ uint32_t div_cols(uint32_t n, uint32_t m, uint32_t l)
{
    if (l == 0u) return n;  // cols == 1
    const uint32_t t = __umulhi(m, n);
    return (t + ((n - t) >> 1)) >> (l - 1u);
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
