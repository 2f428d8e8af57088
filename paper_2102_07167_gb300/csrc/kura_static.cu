// Order parameters without any allocation by the library: the scratch lives
// in a file-scope __device__ array (see kura_order_params_static in kura.h).
#include <cuda.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cmath>
#include <mutex>

#include "kura.h"

namespace {

constexpr int STATIC_THREADS = 256;
constexpr int64_t STATIC_SCRATCH_WORDS = 3 * int64_t(KURA_STATIC_MAX_COMM) + 4;

// Layout for a call with n_comm communities: [3 J, 3 J + 3) = fixed-point
// sin sum, cos sum and member count of community J; word 3 n_comm holds the
// last-block ticket, word 3 n_comm + 1 the number of labels outside
// [0, n_comm).  All of it is zero before every call (the call clears it) and
// is zeroed again by the call's last block.
__device__ __align__(256) unsigned long long g_static_scratch[STATIC_SCRATCH_WORDS];

int ceil_log2(int64_t v)
{
    int k = 0;
    while ((int64_t(1) << k) < v) k++;
    return k;
}

// One node per thread: FP64 sin/cos rounded to fixed point and summed per
// community with 64-bit integer atomics (associative, so the sums do not
// depend on the order of the atomics); the last CTA turns the sums into
// r, psi (global, then per community) and zeroes the scratch.  A label
// outside [0, n_comm) is device data the host cannot check: such a node is
// skipped (no atomic touches memory outside the caller's n_comm rows) and
// counted, and a call that counted any writes NaN to every output.
__global__ void __launch_bounds__(STATIC_THREADS)
k_order_params_static(int64_t n, const double* __restrict__ theta, const int32_t* __restrict__ label,
                      int32_t n_comm, double scale_q, double inv_scale_q, unsigned long long* scratch,
                      double* out)
{
    unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + 3 * int64_t(n_comm));
    unsigned long long* bad = scratch + 3 * int64_t(n_comm) + 1;
    const int64_t i = int64_t(blockIdx.x) * STATIC_THREADS + threadIdx.x;
    if (i < n) {
        const int J = label ? label[i] : 0;
        if (J >= 0 && J < n_comm) {
            double s, c;
            sincos(theta[i], &s, &c);
            const long long sf = __double2ll_rn(s * scale_q), cf = __double2ll_rn(c * scale_q);
            atomicAdd(&scratch[3 * J], static_cast<unsigned long long>(sf));
            atomicAdd(&scratch[3 * J + 1], static_cast<unsigned long long>(cf));
            atomicAdd(&scratch[3 * J + 2], 1ull);
        } else {
            atomicAdd(bad, 1ull);
        }
    }
    __threadfence();
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    const bool invalid = __ldcg(bad) != 0ull;
    if (threadIdx.x == 0) {
        long long S = 0, C = 0;
        for (int J = 0; J < n_comm; J++) {
            S += static_cast<long long>(__ldcg(&scratch[3 * J]));
            C += static_cast<long long>(__ldcg(&scratch[3 * J + 1]));
        }
        const double sm = static_cast<double>(S) * inv_scale_q / static_cast<double>(n);
        const double cm = static_cast<double>(C) * inv_scale_q / static_cast<double>(n);
        const double r = sqrt(sm * sm + cm * cm);
        out[0] = invalid ? CUDART_NAN : r;
        out[1] = invalid ? CUDART_NAN : ((r == 0.0) ? 0.0 : atan2(sm, cm));
    }
    for (int J = threadIdx.x; J < n_comm; J += STATIC_THREADS) {
        const double m = static_cast<double>(__ldcg(&scratch[3 * J + 2]));
        double r = 0.0, psi = 0.0;
        if (m > 0) {
            const double s = static_cast<double>(static_cast<long long>(__ldcg(&scratch[3 * J]))) * inv_scale_q / m;
            const double c = static_cast<double>(static_cast<long long>(__ldcg(&scratch[3 * J + 1]))) * inv_scale_q / m;
            r = sqrt(s * s + c * c);
            psi = (r == 0.0) ? 0.0 : atan2(s, c);
        }
        out[2 + 2 * J] = invalid ? CUDART_NAN : r;
        out[3 + 2 * J] = invalid ? CUDART_NAN : psi;
    }
    __syncthreads();
    for (int64_t w = threadIdx.x; w < 3 * int64_t(n_comm) + 2; w += STATIC_THREADS) scratch[w] = 0ull;
}

// Device address of the scratch array.  In host code the array's name only
// stands in for it, so the address is looked up (cudaGetSymbolAddress) with
// the device current and passed to the kernel.  The lookup is made once per
// CUDA context and cached with that context's unique id: after
// cudaDeviceReset the device gets a new primary context, whose id differs,
// and the next call looks the address up again instead of reusing a stale one.
typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);

struct ScratchSlot {
    unsigned long long ctx_id = 0;
    unsigned long long* addr = nullptr;
};

std::mutex g_setup_mutex;
constexpr int MAX_DEVICES = 64;
ScratchSlot g_slot[MAX_DEVICES];
ctx_get_current_fn g_ctx_get_current = nullptr;
ctx_get_id_fn g_ctx_get_id = nullptr;

cudaError_t driver_entry_points()
{
    if (g_ctx_get_current && g_ctx_get_id) return cudaSuccess;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound;
    cudaDriverEntryPointQueryResult q2 = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e != cudaSuccess) return e;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
        return cudaErrorSymbolNotFound;
    g_ctx_get_current = reinterpret_cast<ctx_get_current_fn>(f1);
    g_ctx_get_id = reinterpret_cast<ctx_get_id_fn>(f2);
    return cudaSuccess;
}

cudaError_t scratch_address(int dev, unsigned long long** out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    cudaError_t e = driver_entry_points();
    if (e != cudaSuccess) return e;
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    if (!ctx) {
        // no context current on this thread yet: make the device's primary
        // context current (cudaSetDevice initialises it)
        if ((e = cudaSetDevice(dev)) != cudaSuccess) return e;
        if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
    }
    unsigned long long id = 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    ScratchSlot& slot = g_slot[dev];
    if (!slot.addr || slot.ctx_id != id) {
        void* p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, g_static_scratch)) != cudaSuccess) return e;
        slot.addr = static_cast<unsigned long long*>(p);
        slot.ctx_id = id;
    }
    *out = slot.addr;
    return cudaSuccess;
}

}  // namespace

extern "C" kura_status kura_order_params_static(int64_t n, const double* theta, const int32_t* label,
                                                int32_t n_comm, double* out, void* stream)
{
    if (n <= 0 || !theta || !out) return KURA_EINVAL;
    if (n_comm < 1 || n_comm > KURA_STATIC_MAX_COMM) return KURA_EINVAL;
    if (!label && n_comm != 1) return KURA_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return KURA_ECUDA;
    }
    unsigned long long* scratch = nullptr;
    if (scratch_address(dev, &scratch) != cudaSuccess) {
        cudaGetLastError();
        return KURA_ECUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // zero what this call uses (the previous call's last block already did,
    // unless that call never ran to completion)
    if (cudaMemsetAsync(scratch, 0, size_t(3 * int64_t(n_comm) + 2) * sizeof(unsigned long long), s) !=
        cudaSuccess) {
        cudaGetLastError();
        return KURA_ECUDA;
    }
    const int q = 61 - ceil_log2(n > 2 ? n : 2);
    const unsigned blocks = unsigned((n + STATIC_THREADS - 1) / STATIC_THREADS);
    k_order_params_static<<<blocks, STATIC_THREADS, 0, s>>>(n, theta, label, n_comm, std::ldexp(1.0, q),
                                                            std::ldexp(1.0, -q), scratch, out);
    if (cudaGetLastError() != cudaSuccess) return KURA_ECUDA;
    return KURA_OK;
}
