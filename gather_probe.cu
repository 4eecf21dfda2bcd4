// Measurement aid for the benchmark (not part of the minimizer): the rate at which this GPU
// serves independent random 4-byte loads from a table held in L2, the access pattern of the
// signature rounds' block-id gathers.  Every element reads one int4 of indices (streamed) and
// gathers the four table entries they name.  Indices come from a counter-based hash on the
// device.  Reports the best of `reps` launches (CUDA events).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ uint32_t mix(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return (uint32_t)(x ^ (x >> 31));
}

__global__ void fill_idx(int4* idx, int64_t n, uint32_t table)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        idx[i] = make_int4((int)(mix(4 * i) % table), (int)(mix(4 * i + 1) % table),
                           (int)(mix(4 * i + 2) % table), (int)(mix(4 * i + 3) % table));
}

__global__ void gather4(const int4* __restrict__ idx, const int* __restrict__ tab, int64_t n,
                        int* sink)
{
    int acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int4 r = __ldcs(idx + i);
        acc += __ldcg(tab + r.x) + __ldcg(tab + r.y) + __ldcg(tab + r.z) + __ldcg(tab + r.w);
    }
    if (acc == 0x7fffffff) sink[0] = acc;
}

}  // namespace

// Returns 0 and *best_ms on success, a CUDA error code otherwise.  n elements (4 gathers each)
// over a table of `table` ints; device memory: 16n + 4*table bytes, freed before returning.
extern "C" __attribute__((visibility("default"))) int gather_probe(int64_t n, uint32_t table,
                                                                   int reps, float* best_ms)
{
    if (n < 1 || table < 1 || reps < 1 || !best_ms) return (int)cudaErrorInvalidValue;
    int4* idx = nullptr;
    int* tab = nullptr;
    int* sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    int sms = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMalloc(&idx, sizeof(int4) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&tab, sizeof(int) * (size_t)table);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(tab, 0, sizeof(int) * (size_t)table);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) {
        fill_idx<<<sms * 8, 256>>>(idx, n, table);
        e = cudaGetLastError();
    }
    float best = 1e30f;
    for (int r = 0; r < reps + 1 && e == cudaSuccess; ++r) {
        cudaEventRecord(a);
        gather4<<<sms * 8, 256>>>(idx, tab, n, sink);
        cudaEventRecord(b);
        e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && r > 0 && ms < best) best = ms;   // launch 0 warms up
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(idx);
    cudaFree(tab);
    cudaFree(sink);
    if (e != cudaSuccess) return (int)e;
    *best_ms = best;
    return 0;
}
