// Batched ensembles: many independent trajectories (own graph, omega, K) in
// one persistent launch.  Each CTA takes whole trajectories from a queue
// ordered by decreasing cost (longest processing time first) and integrates
// all RK4 steps of a trajectory inside the CTA, so no grid-wide barrier is
// needed.  Per stage: the trajectory's (sin, cos) table lives in shared
// memory, block sums are exact fixed-point sums (shared 64-bit atomics,
// order independent), rows gather their local corrections from the shared
// table, and an FP64 thread-per-row epilogue does the RK4 stage update.
// Method: eq:KuramotoGraphApproach (Sec. 3).
//
// Precision modes:
//   MODE_MIXED  FP32 sin/cos of the phase reduced mod 2 pi in FP64, FP32
//               per-row correction sums, exact fixed-point block sums, FP64
//               epilogue and state (n <= 16384: a 128 KB FP32 table);
//   MODE_FP64   FP64 sin/cos rounded once to 64-bit fixed point; block sums,
//               corrections and T_I are exact integer sums (n <= 8192: a
//               128 KB fixed-point table); FP64 epilogue and state.
//
// Tensor-core form of the dense blocks (MODE_MIXED, TC = true): for the
// communities the plan puts on the tensor cores, the sum over a dense block
// row's zeros is the product of the 0/1 zero mask with the columns'
// (sin, cos).  Per tile of at most 128 rows and per 64 mask columns the CTA
// expands the mask bits into a BF16 operand tile (exact 0/1) and writes the
// columns' split BF16 values (hi = bf16(v), lo = bf16(v - hi)) as the other
// operand; one thread issues tcgen05.mma.kind::f16 (M = 128, N = 16: rows
// s_hi, s_lo, c_hi, c_lo and 12 zero rows; K = 16 per instruction) with the
// FP32 accumulator in tensor memory.  With one graph per trajectory this is
// a matrix-vector product padded to N = 16: the tensor cores do 4 useful
// columns of 16.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kura_kernels.cuh"

namespace kura {

constexpr int BATCH_THREADS = 1024;
constexpr int BATCH_MAX_N = 16384;       // mixed: FP32 (sin, cos) table of 128 KB
constexpr int BATCH_MAX_N_FP64 = 8192;   // FP64: fixed-point (sin, cos) table of 128 KB
constexpr int BATCH_MAX_COMM = 1024;
constexpr int BATCH_TAB_BYTES = BATCH_MAX_N * 8;
constexpr int BATCH_SMEM_BASE = BATCH_TAB_BYTES + 2 * BATCH_MAX_COMM * 8 + BATCH_MAX_COMM * 16;
// tensor-core operand tiles: A = 128 mask rows x 64 columns of BF16 (128 B per
// row, 128-byte swizzle), B = 16 rows x 64 columns of BF16; two stages each
constexpr int BATCH_TC_KSUB = 64;
constexpr int BATCH_TC_N = 16;
constexpr int BATCH_TC_ABYTES = TC_MBLOCK * BATCH_TC_KSUB * 2;      // 16 KB
constexpr int BATCH_TC_BBYTES = BATCH_TC_N * BATCH_TC_KSUB * 2;     // 2 KB
constexpr int BATCH_TC_SMEM = 1024 + 2 * BATCH_TC_ABYTES + 2 * BATCH_TC_BBYTES;
constexpr int BATCH_TMEM_COLS = 32;                                  // smallest allocation; 16 used
// tcgen05.mma.kind::f16: D F32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
// both K-major, N = 16 (bits 17-22 = N/8), M = 128 (bits 24-28 = M/16)
constexpr uint32_t BATCH_TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BATCH_TC_N / 8) << 17) |
                                    (uint32_t(TC_MBLOCK / 16) << 24);

struct BatchTraj {
    int64_t node_off;     // first node (permuted order) in the concatenated vectors
    int64_t entry_off;    // first correction entry
    int32_t n, n_comm;
    int32_t comm_base;    // first word of its community offsets (n_comm + 1 entries)
    int32_t dense_base;   // first word of its dense-block pointers (n_comm + 1 entries, into dcol)
    double scale;         // K / n
    int32_t q_bits;
    int32_t tc0, tc1;     // its tensor-core tiles [tc0, tc1) in BatchDev::tc_tiles
    int32_t row_lanes;    // lanes that gather one row's listed entries (32, 16 or 8; 32 / row_lanes rows per warp)
};

// A tile of at most 128 rows of one community whose dense-block zeros are a
// mask: bits[(kb * 128 + r) * 4 + w] bit j <=> column wbeg + 128 kb + 32 w + j
// of local row r0 + r is a zero of a dense block (the diagonal excluded).
struct BatchTcTile {
    int32_t r0, nrows;    // local rows (permuted order)
    int32_t wbeg, nkb;    // first column (a multiple of 128), 128-column blocks
    int64_t bits_off;     // first word in BatchDev::tc_bits
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
    const BatchTcTile* tc_tiles;
    const uint32_t* tc_bits;
    const double* omega;          // permuted
    double* y;
    double* Y;
    double* krk;                  // k1 + 2 k2 + 2 k3 (right-hand side only: f)
    void* stash;                  // per node row sums: float2 (mixed) or longlong2 (FP64)
    unsigned int* queue;
    int* err;
};

template <int MODE> struct BatchT;
template <> struct BatchT<MODE_MIXED> { using E = float2; using A = float; using TT = double2; };
template <> struct BatchT<MODE_FP64> { using E = longlong2; using A = long long; using TT = longlong2; };

// the 8 mask bits of columns 8 c .. 8 c + 7 as eight BF16 values 1.0 / 0 (16 bytes)
__device__ __forceinline__ uint4 batch_bf16_mask8(uint32_t byte)
{
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint32_t two = (byte >> (2 * k)) & 3u;
        v[k] = (two & 1u) * 0x3F80u + (two >> 1) * 0x3F800000u;
    }
    return make_uint4(v[0], v[1], v[2], v[3]);
}
// byte offset of (row d, column c) in a BF16 operand tile of 64 columns, 128-byte swizzle
__device__ __forceinline__ int batch_tc_offset(int d, int c)
{
    return d * 128 + ((((c >> 3) ^ (d & 7)) << 4) | ((c & 7) << 1));
}

constexpr uint64_t BATCH_LIMIT_NS = 1000000000ull;   // bound of every wait on the tensor cores

template <int MODE, bool TC>
__global__ void __launch_bounds__(BATCH_THREADS, 1)
    k_batch_rk4(BatchDev b, double h, int64_t n_steps, int rhs_only)
{
    static_assert(!TC || MODE == MODE_MIXED, "the tensor-core form runs in the mixed mode");
    using E = typename BatchT<MODE>::E;
    using A = typename BatchT<MODE>::A;
    using TT = typename BatchT<MODE>::TT;
    extern __shared__ __align__(128) unsigned char batch_smem[];
    E* tab = reinterpret_cast<E*>(batch_smem);                                                   // 128 KB
    unsigned long long* S = reinterpret_cast<unsigned long long*>(batch_smem + BATCH_TAB_BYTES);   // 2 x MAX_COMM
    TT* T = reinterpret_cast<TT*>(S + 2 * BATCH_MAX_COMM);                                         // MAX_COMM
    E* stash = reinterpret_cast<E*>(b.stash);
    __shared__ int cur;
    __shared__ __align__(8) uint64_t mma_bar[2], d_bar;   // d_bar: the final drain after a wait gave up
    __shared__ uint32_t tmem_base;
    __shared__ int tc_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = BATCH_THREADS / 32;
    uint32_t sa = 0, sb = 0;
    unsigned char* A_ = nullptr;
    unsigned char* B_ = nullptr;
    uint32_t ph0 = 0, ph1 = 0;              // thread 0: parity of the next completion of mma_bar[0], mma_bar[1]
    if constexpr (TC) {
        const uint32_t sbase = smem_u32(batch_smem);
        sa = (sbase + uint32_t(BATCH_SMEM_BASE) + 1023u) & ~1023u;
        sb = sa + 2u * BATCH_TC_ABYTES;
        A_ = batch_smem + (sa - sbase);
        B_ = batch_smem + (sb - sbase);
        // rows 4-15 of both B stages stay zero for the whole launch
        for (int q = tid; q < 2 * BATCH_TC_BBYTES / 16; q += BATCH_THREADS)
            reinterpret_cast<uint4*>(B_)[q] = make_uint4(0u, 0u, 0u, 0u);
        if (tid == 0) {
            mbar_init(&mma_bar[0], 1);
            mbar_init(&mma_bar[1], 1);
            mbar_init(&d_bar, 1);
            tc_fail = 0;
        }
        if (warp == 0) tc_alloc(&tmem_base, BATCH_TMEM_COLS);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const unsigned q = atomicAdd(b.queue, 1u);
            cur = (q < unsigned(b.n_traj)) ? b.order[q] : -1;
        }
        __syncthreads();
        if (cur < 0) break;
        const BatchTraj tr = b.traj[cur];
        const int n = tr.n, nc = tr.n_comm;
        const int64_t o = tr.node_off;
        const int32_t* dp = b.dptr + tr.dense_base;
        const double sq = ldexp(1.0, tr.q_bits), isq = ldexp(1.0, -tr.q_bits);
        for (int i = tid; i < 2 * nc; i += BATCH_THREADS) S[i] = 0ull;
        __syncthreads();
        const int64_t steps = rhs_only ? 1 : n_steps;
        for (int64_t step = 0; step < steps; step++) {
            for (int st = 1; st <= (rhs_only ? 1 : 4); st++) {
                // ---- (sin, cos) table and fixed-point block sums: lane 0 of each warp keeps a running
                // sum of its community run (communities are contiguous) and flushes it with one atomic
                const double* th_in = (st == 1) ? b.y + o : b.Y + o;
                long long run_s = 0, run_c = 0;
                int run_J = -1;
                for (int base = warp * 32; base < n; base += BATCH_THREADS) {
                    const int i = base + lane;
                    long long sf = 0, cf = 0;
                    int J = -1;
                    if (i < n) {
                        const double th = th_in[i];
                        if (!isfinite(th)) atomicOr(b.err, ERR_NONFINITE);
                        if constexpr (MODE == MODE_FP64) {
                            double s, c;
                            sincos(th, &s, &c);
                            sf = __double2ll_rn(s * sq);
                            cf = __double2ll_rn(c * sq);
                            reinterpret_cast<longlong2*>(tab)[i] = make_longlong2(sf, cf);
                        } else {
                            const double kk = rint(th * KURA_INV_TWO_PI);
                            double r = fma(-kk, KURA_TWO_PI_HI, th);
                            r = fma(-kk, KURA_TWO_PI_LO, r);
                            float s, c;
                            sincosf(static_cast<float>(r), &s, &c);
                            reinterpret_cast<float2*>(tab)[i] = make_float2(s, c);
                            const float fq = static_cast<float>(sq);
                            sf = __float2ll_rn(s * fq);
                            cf = __float2ll_rn(c * fq);
                        }
                        J = b.node_comm[o + i];
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
                // ---- T_I = sum over the dense column blocks J of row block I of (S_J, C_J)
                for (int I = tid; I < nc; I += BATCH_THREADS) {
                    long long ts = 0, tc = 0;
                    for (int k = dp[I]; k < dp[I + 1]; k++) {
                        const int Jd = b.dcol[k];
                        ts += static_cast<long long>(S[2 * Jd]);
                        tc += static_cast<long long>(S[2 * Jd + 1]);
                    }
                    if constexpr (MODE == MODE_FP64)
                        reinterpret_cast<longlong2*>(T)[I] = make_longlong2(ts, tc);
                    else
                        reinterpret_cast<double2*>(T)[I] =
                            make_double2(static_cast<double>(ts) * isq, static_cast<double>(tc) * isq);
                }
                __syncthreads();
                for (int i = tid; i < 2 * nc; i += BATCH_THREADS) S[i] = 0ull;
                // ---- rows: a group of L lanes per row (L = 32, 16 or 8, the trajectory's row tile:
                // 32 / L rows per warp) gathers the row's listed corrections from the shared table
                const int32_t* roff = b.row_off + o + cur;            // n + 1 offsets per trajectory
                const uint16_t* e = b.entries + tr.entry_off;
                const int L = tr.row_lanes, rpw = 32 / L, sub = lane / L, sl = lane - sub * L;
                for (int r0 = warp * rpw; r0 < n; r0 += NW * rpw) {
                    const int r = r0 + sub;
                    int beg = 0, end = 0, nm = 0;
                    if (r < n) { beg = __ldg(roff + r); end = __ldg(roff + r + 1); nm = __ldg(b.row_nm + o + r); }
                    A as = 0, ac = 0;
                    for (int k0 = beg; k0 < end; k0 += 4 * L) {    // up to 4 index loads in flight per lane
                        int idx[4];
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            const int k = k0 + L * q + sl;
                            idx[q] = (k < end) ? int(__ldg(e + k)) : -1;
                        }
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            if (idx[q] >= 0) {
                                const E v = tab[idx[q]];
                                if (k0 + L * q + sl - beg < nm) { as -= v.x; ac -= v.y; }
                                else                            { as += v.x; ac += v.y; }
                            }
                        }
                    }
                    for (int off = L >> 1; off; off >>= 1) {       // within the lane group
                        as += __shfl_xor_sync(0xffffffffu, as, off);
                        ac += __shfl_xor_sync(0xffffffffu, ac, off);
                    }
                    if (sl == 0 && r < n) {
                        E v;
                        v.x = as;
                        v.y = ac;
                        stash[o + r] = v;
                    }
                }
                __syncthreads();
                // ---- tensor-core tiles: rows' zero sums of their dense blocks as mask x (sin, cos)
                if constexpr (TC) if (tr.tc1 > tr.tc0) {
                    const float2* tabf = reinterpret_cast<const float2*>(tab);
                    for (int tt_i = tr.tc0; tt_i < tr.tc1; tt_i++) {
                        const BatchTcTile tt = b.tc_tiles[tt_i];
                        const uint32_t* bits = b.tc_bits + tt.bits_off;
                        const int nT = 2 * tt.nkb;                 // 64-column operand blocks
                        // the 4 mask words of this thread's row for one 128-column block cover two operand
                        // blocks; the next block's words are loaded one block ahead
                        const int ar = tid >> 3, ac = tid & 7;
                        const uint4* rowbits = reinterpret_cast<const uint4*>(bits) + ar;
                        uint4 wcur = __ldg(rowbits), wnext = make_uint4(0u, 0u, 0u, 0u);
                        // One waiter (thread 0) and one block barrier per operand block q: the CTA writes
                        // stage q & 1 while thread 0 waits for the MMAs of block q - 1 (the last readers of
                        // stage (q + 1) & 1, which block q + 1 overwrites); after the barrier thread 0 issues
                        // the MMAs of block q.  The stage of block q was last read by block q - 2, whose
                        // completion thread 0 waited for before the previous barrier.
                        for (int q = 0; q < nT; q++) {
                            if ((q & 1) == 0) {
                                if (q > 0) wcur = wnext;
                                if (q + 2 < nT) wnext = __ldg(rowbits + size_t((q >> 1) + 1) * TC_MBLOCK);
                            }
                            const int sst = q & 1;
                            {   // A: thread -> (row ar, 8-column chunk ac) of the 128 x 64 mask tile
                                const int wi = (q & 1) * 2 + (ac >> 2);
                                const uint32_t w = wi == 0 ? wcur.x : wi == 1 ? wcur.y : wi == 2 ? wcur.z : wcur.w;
                                *reinterpret_cast<uint4*>(A_ + sst * BATCH_TC_ABYTES + ar * 128 +
                                                          ((ac ^ (ar & 7)) << 4)) =
                                    batch_bf16_mask8((w >> ((ac & 3) * 8)) & 0xFFu);
                            }
                            if (tid < BATCH_TC_KSUB) {   // B rows 0-3: split BF16 (sin, cos) of the 64 columns
                                const int col = tt.wbeg + q * BATCH_TC_KSUB + tid;
                                const float2 v = col < n ? tabf[col] : make_float2(0.0f, 0.0f);
                                const __nv_bfloat16 sh = __float2bfloat16_rn(v.x), ch = __float2bfloat16_rn(v.y);
                                const __nv_bfloat16 sl = __float2bfloat16_rn(v.x - __bfloat162float(sh));
                                const __nv_bfloat16 cl = __float2bfloat16_rn(v.y - __bfloat162float(ch));
                                unsigned char* Bs = B_ + sst * BATCH_TC_BBYTES;
                                *reinterpret_cast<__nv_bfloat16*>(Bs + batch_tc_offset(0, tid)) = sh;
                                *reinterpret_cast<__nv_bfloat16*>(Bs + batch_tc_offset(1, tid)) = sl;
                                *reinterpret_cast<__nv_bfloat16*>(Bs + batch_tc_offset(2, tid)) = ch;
                                *reinterpret_cast<__nv_bfloat16*>(Bs + batch_tc_offset(3, tid)) = cl;
                            }
                            fence_proxy_async();           // the operand writes, visible to the tensor cores
                            if (tid == 0 && q >= 1) {
                                const int ps = (q - 1) & 1;    // stage of block q - 1
                                if (!tc_fail && !mbar_wait_bounded(&mma_bar[ps], ps ? ph1 : ph0, BATCH_LIMIT_NS))
                                    tc_fail = 1;
                                if (ps) ph1 ^= 1u; else ph0 ^= 1u;
                            }
                            __syncthreads();
                            if (tid == 0 && !tc_fail) {
                                tc_fence_after();
                                const uint64_t da = tc_sdesc(sa + uint32_t(sst * BATCH_TC_ABYTES));
                                const uint64_t db = tc_sdesc(sb + uint32_t(sst * BATCH_TC_BBYTES));
#pragma unroll
                                for (int k = 0; k < BATCH_TC_KSUB / 16; k++)   // K = 16 BF16: 32 bytes along a row
                                    tc_mma_f16(tmem_base, da + uint64_t(2 * k), db + uint64_t(2 * k), BATCH_TC_IDESC,
                                               (q | k) != 0 ? 1u : 0u);
                                tc_commit(&mma_bar[sst]);
                            }
                        }
                        if (tid == 0) {
                            // the last block's commit: all MMAs of the tile are complete when it arrives
                            const int ps = (nT - 1) & 1;
                            if (!tc_fail && !mbar_wait_bounded(&mma_bar[ps], ps ? ph1 : ph0, BATCH_LIMIT_NS))
                                tc_fail = 1;
                            if (ps) ph1 ^= 1u; else ph0 ^= 1u;
                        }
                        __syncthreads();
                        tc_fence_after();
                        if (!tc_fail && warp < 4) {
                            // warp w reads tensor-memory lanes 32 w .. 32 w + 31: rows of the tile
                            uint32_t d[16];
                            tc_ld16(tmem_base + (uint32_t(32 * warp) << 16), d);
                            const int r = 32 * warp + lane;
                            if (r < tt.nrows) {
                                float2* sp = reinterpret_cast<float2*>(b.stash) + o + tt.r0 + r;
                                float2 v = *sp;
                                v.x -= __uint_as_float(d[0]) + __uint_as_float(d[1]);
                                v.y -= __uint_as_float(d[2]) + __uint_as_float(d[3]);
                                *sp = v;
                            }
                        }
                        tc_fence_before();
                        __syncthreads();     // accumulator read before the next tile's first MMA overwrites it
                    }
                    if (tid == 0 && tc_fail) atomicOr(b.err, ERR_TIMEOUT);
                }
                // ---- FP64 epilogue and RK4 stage update, a thread per row
                for (int i = tid; i < n; i += BATCH_THREADS) {
                    const int J = b.node_comm[o + i];
                    const E a = stash[o + i];
                    const E own = tab[i];
                    double acc_s, acc_c, s_i, c_i;
                    if constexpr (MODE == MODE_FP64) {
                        const longlong2 t2 = reinterpret_cast<const longlong2*>(T)[J];
                        acc_s = static_cast<double>(t2.x + static_cast<long long>(a.x)) * isq;
                        acc_c = static_cast<double>(t2.y + static_cast<long long>(a.y)) * isq;
                        s_i = static_cast<double>(own.x) * isq;
                        c_i = static_cast<double>(own.y) * isq;
                    } else {
                        const double2 t2 = reinterpret_cast<const double2*>(T)[J];
                        acc_s = t2.x + static_cast<double>(a.x);
                        acc_c = t2.y + static_cast<double>(a.y);
                        s_i = static_cast<double>(own.x);
                        c_i = static_cast<double>(own.y);
                    }
                    const double f = b.omega[o + i] + tr.scale * (c_i * acc_s - s_i * acc_c);
                    const int64_t g = o + i;
                    if (rhs_only) {
                        b.krk[g] = f;
                    } else if (st == 1) {
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
    if constexpr (TC) {
        // after a wait that gave up, let the MMAs still in flight land before tensor memory is freed
        if (tid == 0 && tc_fail) {
            tc_commit(&d_bar);
            mbar_wait_bounded(&d_bar, 0u, BATCH_LIMIT_NS);
        }
        tc_fence_before();
        __syncthreads();
        if (warp == 0) tc_dealloc(tmem_base, BATCH_TMEM_COLS);
    }
}

}  // namespace kura
