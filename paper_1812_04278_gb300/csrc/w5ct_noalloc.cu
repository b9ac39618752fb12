// w5ct_noalloc.cu -- w5ct_conserved_totals_noalloc: the conserved-totals
// reduction of w5ct_conserved_totals, for callers that cannot allocate
// device memory (frameworks that reserve all device memory up front and
// forbid later cudaMalloc, and real-time host loops that cannot afford the
// implicit synchronisation of an allocation).  It takes the caller's device
// arrays directly, needs no context, and keeps its scratch -- one partial
// record per block and the final record -- in a fixed array in this file.
// It ends by copying the totals to the host and synchronising the stream,
// so it is not meant for a stream under capture.
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "w5ct.h"
#include "w5ct_internal.h"

constexpr int kNaThreads = 256;
constexpr long long kNaCellsPerBlock = 16384;
constexpr int kNaMaxBlocks = (int)(W5CT_NOALLOC_MAX_CELLS / kNaCellsPerBlock);
constexpr int kNaRecord = 8;   // rho, m_x, m_y, m_z, E, b_x, b_y, b_z
static_assert(W5CT_NOALLOC_MAX_CELLS % kNaCellsPerBlock == 0, "cell limit must be a whole number of blocks");

// Scratch of this entry point: kNaMaxBlocks partial records followed by the
// final record (8 doubles each), 512 KB + 64 B.  Every GPU that loads the
// library holds it until the process exits.  Each call overwrites every
// record it later reads, so nothing has to be cleared between calls.  Host
// code must not pass this name to a kernel: on the host it is only a
// stand-in, and the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_totals_scratch[(kNaMaxBlocks + 1) * kNaRecord];

namespace {

// device address of g_totals_scratch per device, looked up once per device
// (void after a cudaDeviceReset of that device, which the library never does)
std::mutex g_mu;
double *g_scratch_ptr[256] = {nullptr};

__device__ __forceinline__ void na_block_sum(double (&v)[kNaRecord], double *red /* kNaRecord * 32 */) {
#pragma unroll
    for (int q = 0; q < kNaRecord; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < kNaRecord; ++q) red[q * 32 + warp] = v[q];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int q = 0; q < kNaRecord; ++q) {
            double x = lane < nw ? red[q * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            v[q] = x;
        }
    }
}

// block b sums cells [b * kNaCellsPerBlock, (b + 1) * kNaCellsPerBlock) of the
// five conserved planes and the three face planes into record b
__global__ void __launch_bounds__(kNaThreads) na_partial_kernel(long long n, const double *__restrict__ cons,
                                                                const double *__restrict__ bface, double *scratch) {
    __shared__ double red[kNaRecord * 32];
    double v[kNaRecord] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long begin = (long long)blockIdx.x * kNaCellsPerBlock;
    long long end = begin + kNaCellsPerBlock;
    if (end > n) end = n;
    for (long long p = begin + threadIdx.x; p < end; p += kNaThreads) {
#pragma unroll
        for (int f = 0; f < 5; ++f) v[f] += cons[(size_t)f * (size_t)n + (size_t)p];
#pragma unroll
        for (int f = 0; f < 3; ++f) v[5 + f] += bface[(size_t)f * (size_t)n + (size_t)p];
    }
    na_block_sum(v, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < kNaRecord; ++q) scratch[(size_t)blockIdx.x * kNaRecord + q] = v[q];
}

// one block: records 0 .. nblk-1 in a fixed order into the final record
__global__ void __launch_bounds__(kNaThreads) na_final_kernel(int nblk, double *scratch) {
    __shared__ double red[kNaRecord * 32];
    double v[kNaRecord] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += kNaThreads)
#pragma unroll
        for (int q = 0; q < kNaRecord; ++q) v[q] += scratch[(size_t)b * kNaRecord + q];
    na_block_sum(v, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < kNaRecord; ++q) scratch[(size_t)kNaMaxBlocks * kNaRecord + q] = v[q];
}

int na_fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    w5ct::set_global_error(buf);
    return code;
}

}  // namespace

extern "C" int w5ct_conserved_totals_noalloc(const double *cons, const double *bface, int nx, int ny, int nz,
                                             double dx, double dy, double dz, double out[8], void *stream) {
    if (!cons || !bface || !out) return na_fail(W5CT_ERR_ARG, "w5ct_conserved_totals_noalloc: null pointer");
    if (nx < 1 || ny < 1 || nz < 1) return na_fail(W5CT_ERR_ARG, "w5ct_conserved_totals_noalloc: sizes must be >= 1");
    if (!(dx > 0) || !(dy > 0) || !(dz > 0))
        return na_fail(W5CT_ERR_ARG, "w5ct_conserved_totals_noalloc: spacings must be > 0");
    const long long n = (long long)nx * ny * nz;
    if (n > (long long)W5CT_NOALLOC_MAX_CELLS)
        return na_fail(W5CT_ERR_ARG,
                       "w5ct_conserved_totals_noalloc: %lld cells exceed the fixed scratch limit of %lld cells",
                       n, (long long)W5CT_NOALLOC_MAX_CELLS);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(W5CT_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return na_fail(W5CT_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    double *scratch = nullptr;
    {
        // first call on this device: look up the device address of the scratch
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_totals_scratch);
            if (e != cudaSuccess) return na_fail(W5CT_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_scratch_ptr[dev] = (double *)p;
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nblk = (int)((n + kNaCellsPerBlock - 1) / kNaCellsPerBlock);
    na_partial_kernel<<<nblk, kNaThreads, 0, s>>>(n, cons, bface, scratch);
    na_final_kernel<<<1, kNaThreads, 0, s>>>(nblk, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(W5CT_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    double tot[kNaRecord];
    e = cudaMemcpyAsync(tot, scratch + (size_t)kNaMaxBlocks * kNaRecord, sizeof(tot), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return na_fail(W5CT_ERR_CUDA, "copy of the totals: %s", cudaGetErrorString(e));
    const double dv = dx * dy * dz;
    for (int q = 0; q < kNaRecord; ++q) out[q] = tot[q] * dv;
    return W5CT_OK;
}
