// Batched ensembles: many independent trajectories (own graph, omega, K) in
// one persistent launch.  Each CTA takes whole trajectories from a queue
// ordered by decreasing cost (longest processing time first) and integrates
// all RK4 steps of a trajectory inside the CTA, so no grid-wide barrier is
// needed.  Per stage: the trajectory's (sin, cos) table lives in shared
// memory, block sums are exact fixed-point sums (shared 64-bit atomics,
// order independent), rows gather their local corrections from the shared
// table, and an FP64 thread-per-row epilogue does the RK4 stage update.
// Method: eq:KuramotoGraphApproach (Sec. 3) in the mixed precision mode.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace kura {

constexpr int BATCH_THREADS = 1024;
constexpr int BATCH_MAX_N = 16384;       // nodes per trajectory: FP32 (sin, cos) table of 128 KB
constexpr int BATCH_MAX_COMM = 1024;

struct BatchTraj {
    int64_t node_off;     // first node (permuted order) in the concatenated vectors
    int64_t entry_off;    // first correction entry
    int32_t n, n_comm;
    int32_t comm_base;    // first word of its community offsets (n_comm + 1 entries)
    int32_t dense_base;   // first word of its dense-block pointers (n_comm + 1 entries, into dcol)
    double scale;         // K / n
    int32_t q_bits, pad;
};

struct BatchDev {
    const BatchTraj* traj;
    const int32_t* order;         // trajectory ids by decreasing cost
    int32_t n_traj;
    const int32_t* comm_off;      // concatenated local community offsets
    const int32_t* dptr;          // concatenated dense-block pointers (local into dcol slice)
    const int32_t* dcol;          // dense column blocks (local community ids)
    const uint16_t* node_comm;    // community of each node (local)
    const int32_t* row_off;       // per node: first entry (relative to entry_off), n + 1 per trajectory
    const int32_t* row_nm;        // per node: missing entries at the start of its segment
    const uint16_t* entries;      // local permuted column indices
    const double* omega;          // permuted
    double* y;
    double* Y;
    double* krk;
    float2* stash;                // per node row sums
    unsigned int* queue;
    int* err;
};

__global__ void __launch_bounds__(BATCH_THREADS, 1) k_batch_rk4(BatchDev b, double h, int64_t n_steps)
{
    extern __shared__ __align__(128) unsigned char batch_smem[];
    float2* tab = reinterpret_cast<float2*>(batch_smem);                                   // BATCH_MAX_N
    unsigned long long* S = reinterpret_cast<unsigned long long*>(tab + BATCH_MAX_N);    // 2 x BATCH_MAX_COMM
    double2* T = reinterpret_cast<double2*>(S + 2 * BATCH_MAX_COMM);                      // BATCH_MAX_COMM
    __shared__ int cur;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = BATCH_THREADS / 32;
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const unsigned q = atomicAdd(b.queue, 1u);
            cur = (q < unsigned(b.n_traj)) ? b.order[q] : -1;
        }
        __syncthreads();
        if (cur < 0) return;
        const BatchTraj tr = b.traj[cur];
        const int n = tr.n, nc = tr.n_comm;
        const int64_t o = tr.node_off;
        const int32_t* coff = b.comm_off + tr.comm_base;
        const int32_t* dp = b.dptr + tr.dense_base;
        const double sq = ldexp(1.0, tr.q_bits), isq = ldexp(1.0, -tr.q_bits);
        for (int i = tid; i < 2 * nc; i += BATCH_THREADS) S[i] = 0ull;
        __syncthreads();
        for (int64_t step = 0; step < n_steps; step++) {
            for (int st = 1; st <= 4; st++) {
                // ---- (sin, cos) table and fixed-point block sums: lane 0 of each warp keeps a running
                // sum of its community run (communities are contiguous) and flushes it with one atomic
                const double* th_in = (st == 1) ? b.y + o : b.Y + o;
                const float fq = static_cast<float>(sq);
                long long run_s = 0, run_c = 0;
                int run_J = -1;
                for (int base = warp * 32; base < n; base += BATCH_THREADS) {
                    const int i = base + lane;
                    long long sf = 0, cf = 0;
                    int J = -1;
                    if (i < n) {
                        const double th = th_in[i];
                        if (!isfinite(th)) atomicOr(b.err, 1);
                        const double kk = rint(th * 0.15915494309189533577);
                        double r = fma(-kk, 6.283185307179586232, th);
                        r = fma(-kk, 2.4492935982947064e-16, r);
                        float s, c;
                        sincosf(static_cast<float>(r), &s, &c);
                        tab[i] = make_float2(s, c);
                        J = b.node_comm[o + i];
                        sf = __float2ll_rn(s * fq);
                        cf = __float2ll_rn(c * fq);
                    }
                    const int J0 = __shfl_sync(0xffffffffu, J, 0);
                    if (__all_sync(0xffffffffu, J == J0 || J < 0)) {
#pragma unroll
                        for (int off = 16; off; off >>= 1) {
                            sf += __shfl_xor_sync(0xffffffffu, sf, off);
                            cf += __shfl_xor_sync(0xffffffffu, cf, off);
                        }
                        if (lane == 0) {
                            if (J0 != run_J && run_J >= 0) {
                                atomicAdd(&S[2 * run_J], static_cast<unsigned long long>(run_s));
                                atomicAdd(&S[2 * run_J + 1], static_cast<unsigned long long>(run_c));
                                run_s = run_c = 0;
                            }
                            run_J = J0;
                            run_s += sf;
                            run_c += cf;
                        }
                    } else if (J >= 0) {
                        atomicAdd(&S[2 * J], static_cast<unsigned long long>(sf));
                        atomicAdd(&S[2 * J + 1], static_cast<unsigned long long>(cf));
                    }
                }
                if (lane == 0 && run_J >= 0) {
                    atomicAdd(&S[2 * run_J], static_cast<unsigned long long>(run_s));
                    atomicAdd(&S[2 * run_J + 1], static_cast<unsigned long long>(run_c));
                }
                __syncthreads();
                for (int I = tid; I < nc; I += BATCH_THREADS) {
                    long long ts = 0, tc = 0;
                    for (int k = dp[I]; k < dp[I + 1]; k++) {
                        const int Jd = b.dcol[k];
                        ts += static_cast<long long>(S[2 * Jd]);
                        tc += static_cast<long long>(S[2 * Jd + 1]);
                    }
                    T[I] = make_double2(static_cast<double>(ts) * isq, static_cast<double>(tc) * isq);
                }
                __syncthreads();
                for (int i = tid; i < 2 * nc; i += BATCH_THREADS) S[i] = 0ull;
                // ---- rows: a warp per row gathers its corrections from the shared table
                const int32_t* roff = b.row_off + o + cur;            // n + 1 offsets per trajectory
                for (int r = warp; r < n; r += NW) {
                    const int beg = __ldg(roff + r), end = __ldg(roff + r + 1), nm = __ldg(b.row_nm + o + r);
                    float as = 0.f, ac = 0.f;
                    const uint16_t* e = b.entries + tr.entry_off;
                    for (int k0 = beg; k0 < end; k0 += 128) {      // up to 128 index loads in flight per row
                        int idx[4];
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            const int k = k0 + 32 * q + lane;
                            idx[q] = (k < end) ? int(__ldg(e + k)) : -1;
                        }
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            if (idx[q] >= 0) {
                                const float2 v = tab[idx[q]];
                                if (k0 + 32 * q + lane - beg < nm) { as -= v.x; ac -= v.y; }
                                else                               { as += v.x; ac += v.y; }
                            }
                        }
                    }
#pragma unroll
                    for (int off = 16; off; off >>= 1) {
                        as += __shfl_xor_sync(0xffffffffu, as, off);
                        ac += __shfl_xor_sync(0xffffffffu, ac, off);
                    }
                    if (lane == 0) b.stash[o + r] = make_float2(as, ac);
                }
                __syncthreads();
                // ---- FP64 epilogue and RK4 stage update, a thread per row
                for (int i = tid; i < n; i += BATCH_THREADS) {
                    const int J = b.node_comm[o + i];
                    const float2 a = b.stash[o + i];
                    const float2 own = tab[i];
                    const double acc_s = T[J].x + static_cast<double>(a.x);
                    const double acc_c = T[J].y + static_cast<double>(a.y);
                    const double f = b.omega[o + i] + tr.scale * (static_cast<double>(own.y) * acc_s -
                                                                  static_cast<double>(own.x) * acc_c);
                    const int64_t g = o + i;
                    if (st == 1) {
                        b.krk[g] = f;
                        b.Y[g] = b.y[g] + (0.5 * h) * f;
                    } else if (st == 2) {
                        b.krk[g] = b.krk[g] + 2.0 * f;
                        b.Y[g] = b.y[g] + (0.5 * h) * f;
                    } else if (st == 3) {
                        b.krk[g] = b.krk[g] + 2.0 * f;
                        b.Y[g] = b.y[g] + h * f;
                    } else {
                        b.y[g] = b.y[g] + (h / 6.0) * (b.krk[g] + f);
                    }
                }
                __syncthreads();
            }
        }
    }
}

}  // namespace kura
