// Small graphs: every RK4 step in one launch of one thread-block cluster.
//
// For a graph of at most SMALL_MAX_N nodes the step loop is launch-bound:
// eight kernels per step that each occupy one or two SMs.  Here one cluster
// of SMALL_CLUSTER CTAs runs all steps.  CTA r owns the permuted nodes
// [r P, r P + P): per stage it computes their (sin, cos) table slice in its
// own shared memory and their fixed-point community sums, then the cluster
// barrier publishes both; every CTA adds up the community sums of all CTAs
// (distributed shared memory, a fixed order) into T_I, and its rows gather
// their listed corrections from whichever CTA owns the column (ld from the
// owner's shared memory through the cluster window).  Thread t of CTA r owns
// node r P + t for the whole launch: its state, stage input and RK4 sum stay
// in registers (the state is written back once, at the end), and it runs the
// node's FP64 epilogue and RK4 update.  A second cluster barrier ends each
// stage before any table slice is overwritten.  Method: eq:KuramotoGraph by
// eq:KuramotoGraphApproach (Sec. 3), classical RK4.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kura_kernels.cuh"

namespace kura {

constexpr int SMALL_CLUSTER = 8;          // CTAs in the cluster (portable size)
constexpr int SMALL_THREADS = 512;
constexpr int SMALL_MAX_N = 4096;         // nodes: at most 512 per CTA
constexpr int SMALL_MAX_P = SMALL_MAX_N / SMALL_CLUSTER;
constexpr int SMALL_MAX_COMM = 256;

struct SmallArgs {
    int n, n_comm, P;                 // nodes, communities, nodes per CTA (a multiple of 32)
    const int32_t* node_comm;         // [n] community of each permuted node
    const int32_t* dptr;              // [n_comm + 1] dense column blocks of each row block
    const int32_t* dcol;
    const int32_t* row_off;           // [n + 1] per-row listed entries: [missing | present]
    const int32_t* row_nm;            // [n] missing entries at the start of the row's list
    const int32_t* ent;               // permuted column of each listed entry
    const double* omega;              // [n] permuted
    const double* rscale;             // [n] K / deg (degree scaling) or null
    double scale;                     // K / n (uniform scaling)
    double scale_q, inv_scale_q;      // fixed point 2^q, 2^-q
    double* y;                        // [n] state, in place (read at the start, written at the end)
    int* err;
};

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// every thread of every CTA of the cluster: shared-memory writes before it are visible to all CTAs after it
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// address of the same shared-memory object in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(const void* local, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 ld_cluster(const float2* local, uint32_t rank)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(cluster_addr(local, rank)));
    return v;
}
__device__ __forceinline__ longlong2 ld_cluster(const longlong2* local, uint32_t rank)
{
    longlong2 v;
    asm volatile("ld.shared::cluster.v2.s64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "r"(cluster_addr(local, rank)));
    return v;
}
__device__ __forceinline__ unsigned long long ld_cluster(const unsigned long long* local, uint32_t rank)
{
    unsigned long long v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(cluster_addr(local, rank)));
    return v;
}

template <int MODE>
__global__ void __launch_bounds__(SMALL_THREADS, 1) k_small_rk4(SmallArgs a, double h, int64_t n_steps)
{
    static_assert(SMALL_MAX_P <= SMALL_THREADS, "one own node per thread");
    using E = typename EntryT<MODE>::T;
    using A = typename EntryT<MODE>::A;
    __shared__ E tab[SMALL_MAX_P];                           // this CTA's slice of the (sin, cos) table
    __shared__ E stash[SMALL_MAX_P];                         // listed-entry sums of the own rows
    __shared__ unsigned long long S[2 * SMALL_MAX_COMM];     // this CTA's fixed-point community sums
    __shared__ long long Tq[2 * SMALL_MAX_COMM];             // T_I in fixed point (exact cluster totals)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = SMALL_THREADS / 32;
    const uint32_t rank = cluster_rank();
    const int base = int(rank) * a.P;
    const int cnt = max(0, min(a.P, a.n - base));
    const int nc = a.n_comm;
    // thread tid owns node base + tid for the whole launch: its frequency, scaling and community stay in
    // registers, and its state is read and written by this thread only
    const bool own = tid < cnt;
    const int row = base + tid;
    const double om = own ? a.omega[row] : 0.0;
    const double sc = own ? (a.rscale ? a.rscale[row] : a.scale) : 0.0;
    const int Jown = own ? a.node_comm[row] : 0;
    double yv = own ? a.y[row] : 0.0, kv = 0.0, Yv = yv;
    for (int q = tid; q < 2 * nc; q += SMALL_THREADS) S[q] = 0ull;
    __syncthreads();
    for (int64_t step = 0; step < n_steps; step++) {
        for (int st = 1; st <= 4; st++) {
            // ---- table entry and fixed-point community sums of the own node
            if (own) {
                const double th = st == 1 ? yv : Yv;
                if (!isfinite(th)) atomicOr(a.err, ERR_NONFINITE);
                long long sf, cf;
                if constexpr (MODE == MODE_FP64) {
                    double s, c;
                    sincos(th, &s, &c);
                    sf = __double2ll_rn(s * a.scale_q);
                    cf = __double2ll_rn(c * a.scale_q);
                    reinterpret_cast<longlong2*>(tab)[tid] = make_longlong2(sf, cf);
                } else {
                    const double k = rint(th * KURA_INV_TWO_PI);
                    double r = fma(-k, KURA_TWO_PI_HI, th);
                    r = fma(-k, KURA_TWO_PI_LO, r);
                    float s, c;
                    sincosf(static_cast<float>(r), &s, &c);
                    reinterpret_cast<float2*>(tab)[tid] = make_float2(s, c);
                    sf = __float2ll_rn(s * static_cast<float>(a.scale_q));
                    cf = __float2ll_rn(c * static_cast<float>(a.scale_q));
                }
                atomicAdd(&S[2 * Jown], static_cast<unsigned long long>(sf));
                atomicAdd(&S[2 * Jown + 1], static_cast<unsigned long long>(cf));
            }
            cluster_barrier();
            // ---- T_I from the exact totals over the cluster (integer sums: order free)
            for (int I = tid; I < nc; I += SMALL_THREADS) {
                long long ts = 0, tc = 0;
                for (int k = a.dptr[I]; k < a.dptr[I + 1]; k++) {
                    const int J = a.dcol[k];
                    for (uint32_t r = 0; r < SMALL_CLUSTER; r++) {
                        ts += static_cast<long long>(ld_cluster(&S[2 * J], r));
                        tc += static_cast<long long>(ld_cluster(&S[2 * J + 1], r));
                    }
                }
                Tq[2 * I] = ts;
                Tq[2 * I + 1] = tc;
            }
            // ---- rows: a warp per own row with listed entries, gathered from the owning CTA's slice
            for (int i = warp; i < cnt; i += NW) {
                const int rr = base + i;
                const int beg = a.row_off[rr], end = a.row_off[rr + 1], nm = a.row_nm[rr];
                A as = 0, ac = 0;
                if (end > beg) {                                       // warp-uniform
                    for (int k = beg + lane; k < end; k += 32) {
                        const int c = a.ent[k];
                        const E v = ld_cluster(&tab[c % a.P], uint32_t(c / a.P));
                        if (k - beg < nm) { as -= v.x; ac -= v.y; }
                        else              { as += v.x; ac += v.y; }
                    }
#pragma unroll
                    for (int o = 16; o; o >>= 1) {
                        as += __shfl_xor_sync(0xffffffffu, as, o);
                        ac += __shfl_xor_sync(0xffffffffu, ac, o);
                    }
                }
                if (lane == 0) {
                    E v;
                    v.x = as;
                    v.y = ac;
                    stash[i] = v;
                }
            }
            __syncthreads();
            // ---- FP64 epilogue and RK4 stage update of the own node
            if (own) {
                const E sum = stash[tid];
                const E me = tab[tid];
                double acc_s, acc_c, s_i, c_i;
                if constexpr (MODE == MODE_FP64) {
                    // exact integer sums, rounded once
                    acc_s = static_cast<double>(Tq[2 * Jown] + static_cast<long long>(sum.x)) * a.inv_scale_q;
                    acc_c = static_cast<double>(Tq[2 * Jown + 1] + static_cast<long long>(sum.y)) * a.inv_scale_q;
                    s_i = static_cast<double>(me.x) * a.inv_scale_q;
                    c_i = static_cast<double>(me.y) * a.inv_scale_q;
                } else {
                    acc_s = static_cast<double>(Tq[2 * Jown]) * a.inv_scale_q + static_cast<double>(sum.x);
                    acc_c = static_cast<double>(Tq[2 * Jown + 1]) * a.inv_scale_q + static_cast<double>(sum.y);
                    s_i = static_cast<double>(me.x);
                    c_i = static_cast<double>(me.y);
                }
                const double f = om + sc * (c_i * acc_s - s_i * acc_c);
                if (st == 1) {
                    kv = f;
                    Yv = yv + (0.5 * h) * f;
                } else if (st == 2) {
                    kv += 2.0 * f;
                    Yv = yv + (0.5 * h) * f;
                } else if (st == 3) {
                    kv += 2.0 * f;
                    Yv = yv + h * f;
                } else {
                    yv = yv + (h / 6.0) * (kv + f);
                }
            }
            // every CTA is done reading the other slices and sums before they are overwritten
            cluster_barrier();
            for (int q = tid; q < 2 * nc; q += SMALL_THREADS) S[q] = 0ull;
            __syncthreads();
        }
    }
    if (own) a.y[row] = yv;
}

}  // namespace kura
