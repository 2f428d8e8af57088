// Device measurement for the roofline of the row kernel: the rate of random
// 8- or 16-byte gathers from an L2-resident table (kura_measure_gather_rate
// in kura.h).  Not part of the method; the row kernel's sparse-block entries
// are exactly such gathers.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "kura.h"

namespace {

constexpr int PROBE_THREADS = 256;

// Counter-based indices (splitmix64 finaliser of the position), uniform in [0, range).
__global__ void k_probe_fill(int32_t* idx, int64_t n, int64_t range)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        unsigned long long z = (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        idx[i] = int32_t(z % (unsigned long long)range);
    }
}

// Grid-stride: one int4 of indices per thread and step, four independent gathers.
template <class E>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_gather(const int4* __restrict__ idx, int64_t n4,
                                                                const E* __restrict__ table, float* sink)
{
    float acc = 0.0f;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const int4 v = __ldcs(idx + i);
        const E a = __ldg(table + v.x), b = __ldg(table + v.y), c = __ldg(table + v.z), d = __ldg(table + v.w);
        acc += float(a.x) + float(b.x) + float(c.x) + float(d.x);
    }
    if (acc == 1234.5f) sink[0] = acc;     // keeps the loads; the table is zero
}

}  // namespace

extern "C" kura_status kura_measure_gather_rate(int64_t table_entries, int64_t gathers, int32_t entry_bytes,
                                                void* stream, double* gathers_per_s)
{
    if (!gathers_per_s || table_entries < 1 || table_entries > (int64_t(1) << 30) || gathers < 4096 ||
        gathers > (int64_t(1) << 31) || (entry_bytes != 8 && entry_bytes != 16))
        return KURA_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gathers = gathers / 4 * 4;
    void* table = nullptr;
    int32_t* idx = nullptr;
    float* sink = nullptr;
    kura_status st = KURA_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    do {
        if (cudaMalloc(&table, size_t(table_entries) * size_t(entry_bytes)) != cudaSuccess ||
            cudaMalloc(&idx, size_t(gathers) * 4) != cudaSuccess || cudaMalloc(&sink, 16) != cudaSuccess) {
            st = KURA_ENOMEM;
            break;
        }
        if (cudaMemsetAsync(table, 0, size_t(table_entries) * size_t(entry_bytes), s) != cudaSuccess ||
            cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            st = KURA_ECUDA;
            break;
        }
        k_probe_fill<<<unsigned(nsm * 8), PROBE_THREADS, 0, s>>>(idx, gathers, table_entries);
        const unsigned grid = unsigned(nsm * 8);      // full occupancy: 8 CTAs of 256 threads per SM
        std::vector<float> ms;
        for (int r = 0; r < 4; r++) {
            cudaEventRecord(e0, s);
            if (entry_bytes == 8)
                k_probe_gather<float2><<<grid, PROBE_THREADS, 0, s>>>(reinterpret_cast<const int4*>(idx), gathers / 4,
                                                                      static_cast<const float2*>(table), sink);
            else
                k_probe_gather<double2><<<grid, PROBE_THREADS, 0, s>>>(reinterpret_cast<const int4*>(idx), gathers / 4,
                                                                       static_cast<const double2*>(table), sink);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = KURA_ECUDA;
                break;
            }
            float v = 0.0f;
            cudaEventElapsedTime(&v, e0, e1);
            if (r > 0) ms.push_back(v);                // the first run warms L2 with the table
        }
        if (st) break;
        std::sort(ms.begin(), ms.end());
        *gathers_per_s = double(gathers) / (double(ms[ms.size() / 2]) * 1e-3);
    } while (false);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(table);
    cudaFree(idx);
    cudaFree(sink);
    if (st == KURA_OK && cudaGetLastError() != cudaSuccess) st = KURA_ECUDA;
    return st;
}

namespace {

// Grid-stride int4 reads of a buffer, `passes` times over (the buffer stays in
// L2 when it is smaller than L2).
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_stream(const int4* __restrict__ buf, int64_t n16, int passes,
                                                                int* sink)
{
    int acc = 0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int p = 0; p < passes; p++)
        for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n16; i += stride) {
            const int4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x12345678) sink[0] = acc;     // keeps the loads; the buffer is zero
}

__global__ void k_probe_empty() {}

}  // namespace

extern "C" kura_status kura_measure_l2_bandwidth(int64_t bytes, void* stream, double* gb_per_s)
{
    if (!gb_per_s || bytes < (int64_t(1) << 20) || bytes > (int64_t(1) << 30)) return KURA_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bytes = bytes / 16 * 16;
    void* buf = nullptr;
    int* sink = nullptr;
    kura_status st = KURA_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int passes = 16;
    do {
        if (cudaMalloc(&buf, size_t(bytes)) != cudaSuccess || cudaMalloc(&sink, 16) != cudaSuccess) {
            st = KURA_ENOMEM;
            break;
        }
        if (cudaMemsetAsync(buf, 0, size_t(bytes), s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
            cudaEventCreate(&e1) != cudaSuccess) {
            st = KURA_ECUDA;
            break;
        }
        const unsigned grid = unsigned(nsm * 8);
        std::vector<float> ms;
        for (int r = 0; r < 4; r++) {
            cudaEventRecord(e0, s);
            k_probe_stream<<<grid, PROBE_THREADS, 0, s>>>(static_cast<const int4*>(buf), bytes / 16, passes, sink);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = KURA_ECUDA;
                break;
            }
            float v = 0.0f;
            cudaEventElapsedTime(&v, e0, e1);
            if (r > 0) ms.push_back(v);
        }
        if (st) break;
        std::sort(ms.begin(), ms.end());
        *gb_per_s = double(bytes) * passes / (double(ms[ms.size() / 2]) * 1e-3) / 1e9;
    } while (false);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(sink);
    if (st == KURA_OK && cudaGetLastError() != cudaSuccess) st = KURA_ECUDA;
    return st;
}

extern "C" kura_status kura_measure_graph_launch_floor(int32_t kernels, int32_t replays, void* stream,
                                                       double* us_per_kernel)
{
    if (!us_per_kernel || kernels < 1 || kernels > 4096 || replays < 1 || replays > 100000) return KURA_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    kura_status st = KURA_OK;
    do {
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            st = KURA_ECUDA;
            break;
        }
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            st = KURA_ECUDA;
            break;
        }
        for (int k = 0; k < kernels; k++) k_probe_empty<<<1, 32, 0, cap>>>();
        if (cudaStreamEndCapture(cap, &graph) != cudaSuccess ||
            cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
            st = KURA_ECUDA;
            break;
        }
        for (int r = 0; r < 3; r++) cudaGraphLaunch(exec, s);
        cudaEventRecord(e0, s);
        for (int r = 0; r < replays; r++) cudaGraphLaunch(exec, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = KURA_ECUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        *us_per_kernel = double(ms) * 1e3 / (double(replays) * kernels);
    } while (false);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (cap) cudaStreamDestroy(cap);
    if (st == KURA_OK && cudaGetLastError() != cudaSuccess) st = KURA_ECUDA;
    return st;
}
