// peaks.cu -- measured ceilings for the rooflines the bench reports next to
// the kernels of the local-energy path: on-chip (L2) read bandwidth at the
// working-set sizes of the integral table, the rate of independent random
// 8-byte gathers from such a table (the access pattern of the Slater-Condon
// integral reads), and the FP64 / FP32 fused multiply-add rates of the CUDA
// cores (the plain FP64 form's arithmetic).
//
// C ABI (separate library, libnqs_peaks.so; not part of the local-energy
// interface): every call launches on `stream`, times `reps` launches with CUDA
// events after one untimed launch, writes the mean milliseconds per launch to
// *ms and returns 0, or a cudaError_t code. Buffers are the caller's device
// memory.
//
//   int peaks_read(const void* buf, size_t bytes, int passes, int blocks, void* sink,
//                  int reps, void* stream, float* ms)
//       streams `passes` times over buf (16-byte loads, grid-stride); bytes a
//       multiple of 16; sink receives one float per block (keeps loads live).
//   int peaks_gather8(const void* buf, size_t n_words, int loads_per_thread, int blocks,
//                     void* sink, int reps, void* stream, float* ms)
//       blocks x 256 threads, each `loads_per_thread` (a multiple of 8) 8-byte
//       loads at pseudo-random word indices (a 32-bit hash of the thread and
//       load number, masked to n_words, a power of two), 8 independent
//       streams per thread.
//   int peaks_fma64(int iters, int blocks, void* sink, int reps, void* stream, float* ms)
//   int peaks_fma32(int iters, int blocks, void* sink, int reps, void* stream, float* ms)
//       blocks x 256 threads, 8 independent FMA chains of `iters` steps each.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__global__ void __launch_bounds__(256) k_read(const float4* __restrict__ buf, size_t n4, int passes,
                                              float* sink)
{
    float acc = 0.f;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p) {
        size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
        // four loads in flight per thread before they are consumed
        for (; i + 3 * stride < n4; i += 4 * stride) {
            const float4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
            const float4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
            acc += (a.x + b.y) + (c.z + d.w);
        }
        for (; i < n4; i += stride) {
            const float4 a = __ldcg(buf + i);
            acc += a.x;
        }
    }
    if (acc == 1.2345f) sink[blockIdx.x] = acc;   // never true for the zeroed buffers used
}

__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16; x *= 0x7feb352du;
    x ^= x >> 15; x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__global__ void __launch_bounds__(256) k_gather8(const double* __restrict__ buf, uint32_t mask, int loads,
                                                 double* sink)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int l = 0; l < loads; l += 8) {
        #pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t idx = mix32(t * 0x9E3779B9u + (uint32_t)(l + u) * 0x85EBCA6Bu) & mask;
            acc[u] += __ldg(buf + idx);
        }
    }
    double s = 0.0;
    #pragma unroll
    for (int u = 0; u < 8; ++u) s += acc[u];
    if (s == 1.2345) sink[blockIdx.x] = s;
}

template <typename T>
__global__ void __launch_bounds__(256) k_fma(int iters, T* sink)
{
    T x[8];
    #pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = (T)(threadIdx.x + u) * (T)1e-3;
    const T a = (T)0.999999, b = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
        #pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = fma(x[u], a, b);
    }
    T s = 0;
    #pragma unroll
    for (int u = 0; u < 8; ++u) s += x[u];
    if (s == (T)1.2345) sink[blockIdx.x] = s;
}

template <class L>
int timed(L launch, int reps, cudaStream_t st, float* ms)
{
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return (int)e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) { cudaEventDestroy(a); return (int)e; }
    launch();
    cudaEventRecord(a, st);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = reps > 0 ? t / reps : 0.f;
    return (int)e;
}

}  // namespace

extern "C" int peaks_read(const void* buf, size_t bytes, int passes, int blocks, void* sink, int reps,
                          void* stream, float* ms)
{
    if (!buf || !sink || !ms || bytes % 16 || blocks <= 0 || passes <= 0) return (int)cudaErrorInvalidValue;
    cudaStream_t st = (cudaStream_t)stream;
    return timed([&] { k_read<<<blocks, 256, 0, st>>>((const float4*)buf, bytes / 16, passes, (float*)sink); },
                 reps, st, ms);
}

extern "C" int peaks_gather8(const void* buf, size_t n_words, int loads, int blocks, void* sink, int reps,
                             void* stream, float* ms)
{
    if (!buf || !sink || !ms || n_words == 0 || n_words > 0x80000000ull || (n_words & (n_words - 1)) ||
        loads <= 0 || loads % 8 || blocks <= 0)
        return (int)cudaErrorInvalidValue;
    cudaStream_t st = (cudaStream_t)stream;
    return timed([&] { k_gather8<<<blocks, 256, 0, st>>>((const double*)buf, (uint32_t)(n_words - 1), loads,
                                                         (double*)sink); },
                 reps, st, ms);
}

extern "C" int peaks_fma64(int iters, int blocks, void* sink, int reps, void* stream, float* ms)
{
    if (!sink || !ms || iters <= 0 || blocks <= 0) return (int)cudaErrorInvalidValue;
    cudaStream_t st = (cudaStream_t)stream;
    return timed([&] { k_fma<double><<<blocks, 256, 0, st>>>(iters, (double*)sink); }, reps, st, ms);
}

extern "C" int peaks_fma32(int iters, int blocks, void* sink, int reps, void* stream, float* ms)
{
    if (!sink || !ms || iters <= 0 || blocks <= 0) return (int)cudaErrorInvalidValue;
    cudaStream_t st = (cudaStream_t)stream;
    return timed([&] { k_fma<float><<<blocks, 256, 0, st>>>(iters, (float*)sink); }, reps, st, ms);
}
