// Prints cuRAND's Philox4x32-10 block function for a fixed set of counters and keys, so the
// tests can compare the CPU oracle's Philox with an independent implementation, run on the
// GPU.  Counter i: (i, 7 i, 13 i, 17 i) with key (i, i ^ 0xdeadbeef), i = 0 .. 1023.
#include <cstdio>
#include <curand_kernel.h>

__global__ void eval(uint4 *out)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 1024) return;
    const uint4 c = make_uint4(i, 7u * i, 13u * i, 17u * i);
    const uint2 k = make_uint2(i, i ^ 0xdeadbeefu);
    out[i] = curand_Philox4x32_10(c, k);
}

int main()
{
    uint4 *d = nullptr;
    uint4 h[1024];
    if (cudaMalloc(&d, sizeof h) != cudaSuccess) return 2;
    eval<<<4, 256>>>(d);
    if (cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
    cudaFree(d);
    for (int i = 0; i < 1024; ++i) printf("%08x %08x %08x %08x\n", h[i].x, h[i].y, h[i].z, h[i].w);
    return 0;
}
