// ga_peak.cu -- integer-pipe throughput probe.  The paper has no counterpart: this is a
// measurement aid that puts a measured ceiling next to the nominal issue limit when the
// island step's integer work is reported as a fraction of a roofline.
//
// Each thread runs independent chains (eight; two Philox states for the mix -- no chain waits
// on another, so latency is hidden within the thread as well as across the 64 resident warps
// of an SM) of one operation kind,
// written in inline PTX so that each step is one instruction:
//   GA_PEAK_LOP3  c = a ^ b ^ c            lop3.b32 (three-input logic)
//   GA_PEAK_IMAD  p = a * M + p            mad.wide.u32 (32 x 32 -> 64-bit multiply-add)
//   GA_PEAK_MIX   Philox4x32 rounds:       2 x mul.wide.u32 + 2 x lop3.b32 each (the island
//                                          step's random-number arithmetic), two states
// Each iteration is unrolled (256 or 128 operations per thread), so loop overhead stays
// near 1% of the instructions.
#include "ga_internal.h"

namespace ga {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakUnroll = 32;

__device__ __forceinline__ uint32_t lop3_xor(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint64_t mad_wide(uint32_t a, uint32_t m, uint64_t acc)
{
    uint64_t d;
    asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(m), "l"(acc));
    return d;
}

__device__ __forceinline__ uint64_t mul_wide(uint32_t a, uint32_t m)
{
    uint64_t d;
    asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(d) : "r"(a), "r"(m));
    return d;
}

template <int KIND>
__global__ void __launch_bounds__(kPeakThreads, 8) int_peak_kernel(uint32_t iters, uint32_t seed,
                                                                    uint32_t *sink)
{
    const uint32_t t = blockIdx.x * kPeakThreads + threadIdx.x;
    uint32_t x[8], y[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        x[c] = t * (2u * c + 1u) ^ seed;
        y[c] = seed + 0x9E3779B9u * (c + 1u);
    }
    uint32_t acc = 0u;
    if constexpr (KIND == GA_PEAK_LOP3) {
        for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
                for (int c = 0; c < 8; ++c) x[c] = lop3_xor(x[c], y[c], seed + c);
            }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) acc ^= x[c];
    } else if constexpr (KIND == GA_PEAK_IMAD) {
        uint64_t p[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) p[c] = t + 0x9E3779B9u * (c + 1u);
        for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
                for (int c = 0; c < 8; ++c) p[c] = mad_wide(static_cast<uint32_t>(p[c]), 0xD2511F53u + c, p[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) acc ^= static_cast<uint32_t>(p[c] >> 32) ^ static_cast<uint32_t>(p[c]);
    } else {
        // two Philox states per thread (with 64 resident warps per SM, enough independent
        // work to keep the pipes busy), kPeakUnroll / 2 rounds each per iteration
        uint32_t c0[2], c1[2], c2[2], c3[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            c0[s] = x[2 * s];
            c1[s] = y[2 * s];
            c2[s] = x[2 * s + 1];
            c3[s] = y[2 * s + 1];
        }
        for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kPeakUnroll / 2; ++u) {
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const uint64_t a = mul_wide(c0[s], 0xD2511F53u);
                    const uint64_t b = mul_wide(c2[s], 0xCD9E8D57u);
                    const uint32_t n0 = lop3_xor(static_cast<uint32_t>(b >> 32), c1[s], seed);
                    const uint32_t n2 = lop3_xor(static_cast<uint32_t>(a >> 32), c3[s], seed + 1u);
                    c1[s] = static_cast<uint32_t>(b);
                    c3[s] = static_cast<uint32_t>(a);
                    c0[s] = n0;
                    c2[s] = n2;
                }
            }
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) acc ^= c0[s] ^ c1[s] ^ c2[s] ^ c3[s];
    }
    if (acc == 0x12345678u) sink[t & 255u] = acc;  // keeps the chains live
}

}  // namespace
}  // namespace ga

extern "C" int ga_int_peak(uint32_t kind, uint32_t iters, void *stream, double *ops_per_s,
                           double *seconds)
{
    using namespace ga;
    if (kind > GA_PEAK_MIX || iters == 0 || !ops_per_s) return GA_EINVAL;
    cudaGetLastError();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return GA_ECUDA;
    const uint32_t blocks = static_cast<uint32_t>(sms) * 8u;  // 64 resident warps per SM
    uint32_t *sink = nullptr;
    if (pool_alloc(reinterpret_cast<void **>(&sink), 256 * sizeof(uint32_t), st) != cudaSuccess) {
        cudaGetLastError();
        return GA_ENOMEM;
    }
    auto launch = [&](uint32_t n) {
        switch (kind) {
        case GA_PEAK_LOP3: int_peak_kernel<GA_PEAK_LOP3><<<blocks, kPeakThreads, 0, st>>>(n, 7u, sink); break;
        case GA_PEAK_IMAD: int_peak_kernel<GA_PEAK_IMAD><<<blocks, kPeakThreads, 0, st>>>(n, 7u, sink); break;
        default: int_peak_kernel<GA_PEAK_MIX><<<blocks, kPeakThreads, 0, st>>>(n, 7u, sink); break;
        }
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GA_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = GA_ECUDA;
    if (rc == GA_OK) {
        launch(iters / 8u + 1u);  // warm-up
        cudaEventRecord(e0, st);
        launch(iters);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = GA_ECUDA;
    }
    float ms = 0.0f;
    if (rc == GA_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = GA_ECUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    pool_free(sink, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = GA_ECUDA;
    if (rc != GA_OK) return rc;
    // operations of the timed launch per iteration and thread: 8 chains x 32 steps (LOP3,
    // IMAD); 2 Philox states x 16 rounds x 4 instructions (MIX)
    const double per_iter = kind == GA_PEAK_MIX ? 2.0 * (kPeakUnroll / 2) * 4.0 : 8.0 * kPeakUnroll;
    const double ops = static_cast<double>(blocks) * kPeakThreads * iters * per_iter;
    *ops_per_s = ops / (ms * 1e-3);
    if (seconds) *seconds = ms * 1e-3;
    return GA_OK;
}
