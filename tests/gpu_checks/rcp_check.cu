// Error of the Newton-Raphson double reciprocal of the FP64 sweep
// (drcp_newton in w5ct_physics.cuh) against the IEEE division 1.0 / y, in
// units in the last place, over y = m * 2^e for uniformly random mantissas
// m in [1, 2) and exponents e in [-1000, 1000] (both signs).  Prints the
// largest error in ulps and the number of values checked.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../paper_1812_04278_gb300/csrc/w5ct_physics.cuh"

__device__ __forceinline__ uint64_t mix(uint64_t x) {      // splitmix64 finaliser
    x += 0x9e3779b97f4a7c15ULL;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
    return x ^ (x >> 31);
}

__global__ void check(long long n, unsigned long long *worst) {
    unsigned long long w = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint64_t r = mix((uint64_t)i);
        const uint64_t mant = r & 0xfffffffffffffULL;
        const int e = (int)((r >> 52) % 2001) - 1000;
        const uint64_t bits = ((uint64_t)(e + 1023) << 52) | mant | ((r & 1ULL) << 63);
        const double y = __longlong_as_double((long long)bits);
        const double a = w5ct::drcp_newton(y);
        const double b = 1.0 / y;
        const long long da = __double_as_longlong(a), db = __double_as_longlong(b);
        const unsigned long long d = (unsigned long long)(da > db ? da - db : db - da);
        if (d > w) w = d;
    }
    atomicMax(worst, w);
}

int main() {
    unsigned long long *w = nullptr, h = 0;
    const long long n = 1LL << 24;
    if (cudaMalloc(&w, sizeof(h)) != cudaSuccess) return 2;
    cudaMemset(w, 0, sizeof(h));
    check<<<1024, 256>>>(n, w);
    if (cudaMemcpy(&h, w, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
    cudaFree(w);
    printf("max_ulp %llu checked %lld\n", h, n);
    return 0;
}
