// Ensembles of trajectories that share one graph (kura_ensemble_create): the
// right-hand side of eq:KuramotoGraphApproach for ENS_B trajectories at once.
// With a shared graph the dense-block product A_IJ [sin theta, cos theta]
// over all trajectories is a real matrix product: per tile of 128 rows the
// 0/1 mask of the dense blocks' missing entries (BF16, exact) times the
// split BF16 hi + lo (sin, cos) of every trajectory (N = 4 ENS_B columns)
// runs on tcgen05 with FP32 accumulation in tensor memory.  Listed entries
// (present entries of sparse blocks; missing entries of communities without
// a mask) are gathered for all trajectories at once from a node-major table.
//
// Per stage of one group of ENS_B trajectories (blockIdx.y = group; k_ens_row
// runs the groups of a tile next to each other in a one-dimensional grid):
//   k_ens_trig   FP32 (sin, cos) of the FP64-reduced phases -> node-major table
//                and the split BF16 image of the mask product's B operand
//   k_ens_bsum   S_J, C_J per community and trajectory (compensated FP32 per
//                thread, FP64 across threads, fixed order)
//   k_ens_T      T_I = sum_{J in D(I)} (S_J, C_J)
//   k_ens_row    mask product + listed gathers + FP64 epilogue and RK4 update
#pragma once
#include <cuda_bf16.h>

#include "kura_kernels.cuh"

namespace kura {

constexpr int ENS_B = 16;                         // trajectories per group
constexpr int ENS_N = 4 * ENS_B;                  // GEMM columns: (s_hi, s_lo, c_hi, c_lo) per trajectory
constexpr int ENS_THREADS = 512;                  // 16 warps
constexpr int ENS_MMA_WARP = 4;                   // one lane issues the operand copies and the MMAs
constexpr int ENS_LIST_WARPS = ENS_THREADS / 32 - 1;   // every other warp gathers the listed entries
constexpr int ENS_KSUB = 64;                      // mask columns per operand tile (128 bytes of BF16)
constexpr int ENS_ABYTES = TC_MBLOCK * ENS_KSUB * 2;   // 16 KB
constexpr int ENS_BBYTES = ENS_N * ENS_KSUB * 2;       // 8 KB: one 64-node block of the image
constexpr int ENS_SMEM = 1024 + 2 * ENS_ABYTES + 2 * ENS_BBYTES;
constexpr int ENS_TMEM_COLS = ENS_N;              // 64 columns: one 128 x 64 FP32 accumulator
// tcgen05.mma.kind::f16: D F32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
// both K-major, N = ENS_N (bits 17-22 = N/8), M = 128 (bits 24-28 = M/16)
constexpr uint32_t ENS_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(ENS_N / 8) << 17) |
                               (uint32_t(TC_MBLOCK / 16) << 24);
// byte of image row d (0 .. ENS_N-1), column c (0 .. 63) in an 8 KB block
__host__ __device__ constexpr int ens_image_offset(int d, int c)
{
    return d * 128 + ((((c >> 3) ^ (d & 7)) << 4) | ((c & 7) << 1));
}

struct EnsArgs {
    int64_t n;
    int32_t n_comm, groups;
    const int32_t* node_comm;                 // [n]
    const int64_t* comm_off;                  // [n_comm+1]
    const int64_t* dptr;                      // [n_comm+1]
    const int32_t* dcol;
    const Tile* tiles;
    const int64_t* lptr;                      // [n+1] listed entries of each row in lidx
    const int32_t* lidx;                      // column (present: added) or ~column (missing: subtracted)
    const uint32_t* bitmap;                   // mask blocks of TILE_TC tiles
    const uint8_t* aimage;                    // the same masks as BF16 operand tiles (128 x 64, swizzled, 16 KB)
    float2* table;                            // [groups][n + 2][ENS_B]
    __nv_bfloat16* image;                     // [groups][nblk64][ENS_N][64] (swizzled blocks)
    int64_t nblk64;                           // 2 ceil(n / 128): covers every 128-column mask block
    double2* bsum;                            // [groups][n_comm][ENS_B]
    double2* T;                               // [groups][n_comm][ENS_B]
    const double* omega;                      // [groups][n][ENS_B] permuted
    const double* scale;                      // [groups][ENS_B]  K_b / N
    int* err;
};

// One node per thread, all ENS_B trajectories of the group: the (sin, cos)
// table (128 B per node) and the split image (hi = bf16(v), lo = bf16(v - hi)).
__global__ void __launch_bounds__(256) k_ens_trig(EnsArgs a, const double* __restrict__ theta)
{
    const int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x;
    const int grp = blockIdx.y;
    if (i >= a.n) return;
    const double* th = theta + (size_t(grp) * a.n + i) * ENS_B;
    float2* tab = a.table + (size_t(grp) * (a.n + 2) + i) * ENS_B;
    unsigned char* blk = reinterpret_cast<unsigned char*>(a.image) + (size_t(grp) * a.nblk64 + (i >> 6)) * ENS_BBYTES;
    const int c = int(i & 63);
    bool bad = false;
#pragma unroll 4
    for (int b = 0; b < ENS_B; b++) {
        const double t = th[b];
        bad |= !isfinite(t);
        const double k = rint(t * KURA_INV_TWO_PI);
        double r = fma(-k, KURA_TWO_PI_HI, t);
        r = fma(-k, KURA_TWO_PI_LO, r);
        float s, co;
        sincosf(static_cast<float>(r), &s, &co);
        tab[b] = make_float2(s, co);
        const __nv_bfloat16 sh = __float2bfloat16_rn(s), ch = __float2bfloat16_rn(co);
        const __nv_bfloat16 sl = __float2bfloat16_rn(s - __bfloat162float(sh));
        const __nv_bfloat16 cl = __float2bfloat16_rn(co - __bfloat162float(ch));
        *reinterpret_cast<__nv_bfloat16*>(blk + ens_image_offset(4 * b + 0, c)) = sh;
        *reinterpret_cast<__nv_bfloat16*>(blk + ens_image_offset(4 * b + 1, c)) = sl;
        *reinterpret_cast<__nv_bfloat16*>(blk + ens_image_offset(4 * b + 2, c)) = ch;
        *reinterpret_cast<__nv_bfloat16*>(blk + ens_image_offset(4 * b + 3, c)) = cl;
    }
    if (bad) atomicOr(a.err, ERR_NONFINITE);
}

// One CTA per (community, group): sums of the table over the community's
// nodes in a fixed order, per trajectory.
__global__ void __launch_bounds__(256) k_ens_bsum(EnsArgs a)
{
    const int J = blockIdx.x, grp = blockIdx.y;
    const int b = threadIdx.x % ENS_B, part = threadIdx.x / ENS_B;     // 16 node lanes per trajectory
    const int64_t lo = a.comm_off[J], hi = a.comm_off[J + 1];
    const float2* tab = a.table + size_t(grp) * (a.n + 2) * ENS_B;
    // per thread: compensated (Kahan-Neumaier) FP32 sums, full-rate arithmetic;
    // across threads: FP64 in a fixed order
    float s = 0.0f, es = 0.0f, c = 0.0f, ec = 0.0f;
    for (int64_t i = lo + part; i < hi; i += 256 / ENS_B) {
        const float2 v = tab[i * ENS_B + b];
        float t1 = s + v.x;
        es += fabsf(s) >= fabsf(v.x) ? (s - t1) + v.x : (v.x - t1) + s;
        s = t1;
        t1 = c + v.y;
        ec += fabsf(c) >= fabsf(v.y) ? (c - t1) + v.y : (v.y - t1) + c;
        c = t1;
    }
    __shared__ double rs[256], rc[256];
    rs[threadIdx.x] = double(s) + double(es);
    rc[threadIdx.x] = double(c) + double(ec);
    __syncthreads();
    if (threadIdx.x < ENS_B) {
        double ts = 0.0, tc = 0.0;
        for (int q = 0; q < 256 / ENS_B; q++) {
            ts += rs[q * ENS_B + threadIdx.x];
            tc += rc[q * ENS_B + threadIdx.x];
        }
        a.bsum[(size_t(grp) * a.n_comm + J) * ENS_B + threadIdx.x] = make_double2(ts, tc);
    }
}

// T_I per trajectory: one thread per (community, trajectory), fixed order over D(I).
__global__ void k_ens_T(EnsArgs a)
{
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int grp = blockIdx.y;
    if (q >= int64_t(a.n_comm) * ENS_B) return;
    const int I = int(q / ENS_B), b = int(q % ENS_B);
    const double2* bs = a.bsum + size_t(grp) * a.n_comm * ENS_B;
    double s = 0.0, c = 0.0;
    for (int64_t k = a.dptr[I]; k < a.dptr[I + 1]; k++) {
        const double2 v = bs[size_t(a.dcol[k]) * ENS_B + b];
        s += v.x;
        c += v.y;
    }
    a.T[(size_t(grp) * a.n_comm + I) * ENS_B + b] = make_double2(s, c);
}

// Mask operand images, once per plan: one thread per (128 x 128 mask block, 64-column
// half, row) writes the row's 64 mask bits as BF16 1.0 / 0 (128 bytes, 16-byte
// chunk c at c xor (row mod 8): the 128-byte swizzle of the operand tile).
__global__ void k_ens_expand_masks(const uint32_t* __restrict__ bits, int64_t n_blocks, uint8_t* __restrict__ out)
{
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= n_blocks * 2 * TC_MBLOCK) return;
    const int r = int(q % TC_MBLOCK);
    const int64_t qt = q / TC_MBLOCK;                // operand tile: 2 block + half
    const uint2 w = reinterpret_cast<const uint2*>(bits)[(qt >> 1) * TC_MBLOCK * 2 + int64_t(r) * 2 + (qt & 1)];
    unsigned char* row = out + size_t(qt) * ENS_ABYTES + size_t(r) * 128;
#pragma unroll
    for (int c = 0; c < 8; c++) {                    // 8 columns -> 16 bytes
        const uint32_t byte = ((c < 4 ? w.x : w.y) >> ((c & 3) * 8)) & 0xFFu;
        uint32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const uint32_t two = (byte >> (2 * k)) & 3u;
            v[k] = (two & 1u) * 0x3F80u + (two >> 1) * 0x3F800000u;
        }
        *reinterpret_cast<uint4*>(row + ((c ^ (r & 7)) << 4)) = make_uint4(v[0], v[1], v[2], v[3]);
    }
}

// One CTA per (tile of at most 128 rows, group), the groups of a tile adjacent
// in the launch order so that they share the tile's mask images in L2.
template <int STAGE>
__global__ void __launch_bounds__(ENS_THREADS, 2) k_ens_row(EnsArgs a, RkArgs rk)
{
    constexpr uint64_t LIMIT_NS = 1000000000ull;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t a_full[2], a_empty[2], b_full[2], b_empty[2], d_full;
    __shared__ float stash[TC_MBLOCK][2 * ENS_B];     // listed-entry sums per row: (s, c) per trajectory
    __shared__ uint32_t tmem_base;
    __shared__ int fail_flag, a_issued[2], b_issued[2], next_row;
    const Tile t = a.tiles[blockIdx.x / a.groups];
    const int grp = int(blockIdx.x % a.groups);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nrows = t.r1 - t.r0;
    const bool tc = (t.flags & TILE_TC) != 0;
    const int nT = tc ? 2 * t.nsw : 0;               // 64-column operand tiles
    const uint32_t sbase = smem_u32(smem_raw);
    const uint32_t sa = (sbase + 1023u) & ~1023u, sb = sa + 2 * ENS_ABYTES;
    unsigned char* A_ = smem_raw + (sa - sbase);
    unsigned char* B_ = smem_raw + (sb - sbase);
    const float2* tab = a.table + size_t(grp) * (a.n + 2) * ENS_B;
    const size_t gofs = size_t(grp) * a.n * ENS_B;    // offset of the group's node-major vectors

    if (tid == 0) {
        for (int q = 0; q < 2; q++) {
            mbar_init(&a_full[q], 1);
            mbar_init(&a_empty[q], 1);
            mbar_init(&b_full[q], 1);
            mbar_init(&b_empty[q], 1);
        }
        mbar_init(&d_full, 1);
        fail_flag = 0;
        a_issued[0] = a_issued[1] = b_issued[0] = b_issued[1] = 0;
        next_row = ENS_LIST_WARPS;                   // rows 0 .. LW - 1 go to the list warps in order
    }
    if (tc && warp == ENS_MMA_WARP) tc_alloc(&tmem_base, ENS_TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tc ? tmem_base : 0u;

    if (warp == ENS_MMA_WARP) {
        // ---- operand copies (mask images and trajectory images) and MMAs
        if (tc && lane == 0) {
            const unsigned char* img = reinterpret_cast<const unsigned char*>(a.image) +
                                       (size_t(grp) * a.nblk64 + size_t(t.wbeg / ENS_KSUB)) * ENS_BBYTES;
            const unsigned char* aimg = a.aimage + size_t(t.bm_off / (TC_MBLOCK * 4)) * 2 * ENS_ABYTES;
            bool fail = false;
            for (int q = 0; q < 2 && q < nT; q++) {
                mbar_arrive_expect_tx(&a_full[q], ENS_ABYTES);
                bulk_g2s(A_ + q * ENS_ABYTES, aimg + size_t(q) * ENS_ABYTES, ENS_ABYTES, &a_full[q]);
                a_issued[q] = 1;
                mbar_arrive_expect_tx(&b_full[q], ENS_BBYTES);
                bulk_g2s(B_ + q * ENS_BBYTES, img + size_t(q) * ENS_BBYTES, ENS_BBYTES, &b_full[q]);
                b_issued[q] = 1;
            }
            for (int q = 0; q < nT; q++) {
                const int st = q & 1;
                const uint32_t ph = uint32_t(q >> 1) & 1u;
                if (!mbar_wait_bounded(&b_full[st], ph, LIMIT_NS) || !mbar_wait_bounded(&a_full[st], ph, LIMIT_NS)) {
                    fail = true;
                    break;
                }
                tc_fence_after();
                const uint64_t da = tc_sdesc(sa + uint32_t(st * ENS_ABYTES)), db = tc_sdesc(sb + uint32_t(st * ENS_BBYTES));
#pragma unroll
                for (int k = 0; k < ENS_KSUB / 16; k++)      // K = 16 BF16 per MMA: 32 bytes along the row
                    tc_mma_f16(tmem, da + uint64_t(2 * k), db + uint64_t(2 * k), ENS_IDESC, (q | k) != 0 ? 1u : 0u);
                tc_commit(&a_empty[st]);
                tc_commit(&b_empty[st]);
                if (q + 2 < nT) {
                    if (!mbar_wait_bounded(&a_empty[st], ph, LIMIT_NS) || !mbar_wait_bounded(&b_empty[st], ph, LIMIT_NS)) {
                        fail = true;
                        break;
                    }
                    mbar_arrive_expect_tx(&a_full[st], ENS_ABYTES);
                    bulk_g2s(A_ + st * ENS_ABYTES, aimg + size_t(q + 2) * ENS_ABYTES, ENS_ABYTES, &a_full[st]);
                    a_issued[st] = ((q + 2) >> 1) + 1;
                    mbar_arrive_expect_tx(&b_full[st], ENS_BBYTES);
                    bulk_g2s(B_ + st * ENS_BBYTES, img + size_t(q + 2) * ENS_BBYTES, ENS_BBYTES, &b_full[st]);
                    b_issued[st] = ((q + 2) >> 1) + 1;
                }
            }
            tc_commit(&d_full);
            if (fail) {
                atomicOr(a.err, ERR_TIMEOUT);
                fail_flag = 1;
            }
        }
    } else {
        // ---- listed entries: a warp per row, rows claimed from a shared counter one row
        // ahead (rows differ in length); lane l holds trajectory l / 2, component l mod 2.
        // The next row's range and each segment's next 32 indices are loaded ahead; all 32 row
        // loads of a round are in flight before any is summed; lanes past the end read the
        // table's zero entry n.
        const float* tabf = reinterpret_cast<const float*>(tab);
        int r = warp < ENS_MMA_WARP ? warp : warp - 1;
        int64_t beg = 0, end = 0;
        if (r < nrows) { beg = a.lptr[t.r0 + r]; end = a.lptr[t.r0 + r + 1]; }
        const int zero = int(a.n);
        while (r < nrows) {
            int rn = 0;
            if (lane == 0) rn = atomicAdd(&next_row, 1);
            rn = __shfl_sync(0xffffffffu, rn, 0);
            int64_t nbeg = 0, nend = 0;
            if (rn < nrows) { nbeg = a.lptr[t.r0 + rn]; nend = a.lptr[t.r0 + rn + 1]; }
            const int cnt = int(end - beg);
            float acc = 0.0f;
            int nidx = lane < cnt ? a.lidx[beg + lane] : zero;
            for (int k0 = 0; k0 < cnt; k0 += 32) {
                const int idx = nidx;
                if (k0 + 32 < cnt) nidx = k0 + 32 + lane < cnt ? a.lidx[beg + k0 + 32 + lane] : zero;
                float v[32];
#pragma unroll
                for (int u = 0; u < 32; u++) {
                    const int j = __shfl_sync(0xffffffffu, idx, u);
                    const float e = __ldg(tabf + size_t(j >= 0 ? j : ~j) * (2 * ENS_B) + lane);
                    v[u] = j >= 0 ? e : -e;
                }
#pragma unroll
                for (int u = 0; u < 32; u++) acc += v[u];
            }
            stash[r][lane] = acc;
            r = rn;
            beg = nbeg;
            end = nend;
        }
    }
    __syncthreads();

    // ---- epilogue: warp w takes rows 32 (w mod 4) + l (its tensor-memory lane quarter)
    // and trajectories 4 (w / 4) .. + 3 (accumulator columns 16 (w / 4) ..)
    const int r = 32 * (warp & 3) + lane, b0 = 4 * (warp >> 2);
    uint32_t d[16];
#pragma unroll
    for (int q = 0; q < 16; q++) d[q] = 0u;
    const bool ok = !fail_flag;
    if (tc && ok && 32 * (warp & 3) < nrows) {
        if (!mbar_wait_bounded(&d_full, 0u, LIMIT_NS)) atomicOr(a.err, ERR_TIMEOUT);
        tc_fence_after();
        tc_ld16(tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(4 * b0), d);
    }
    if (ok && r < nrows) {
        const int64_t row = int64_t(t.r0) + r;
        const size_t base = gofs + size_t(row) * ENS_B;
#pragma unroll
        for (int bb = 0; bb < 4; bb++) {
            const int b = b0 + bb;
            // corrections (FP32 sums of FP32 terms: missing from the mask product, hi + lo;
            // listed from the gathers) in FP32, added to the FP64 block sums in FP64
            const float cs = (__uint_as_float(d[4 * bb]) + __uint_as_float(d[4 * bb + 1])) - stash[r][2 * b];
            const float cc = (__uint_as_float(d[4 * bb + 2]) + __uint_as_float(d[4 * bb + 3])) - stash[r][2 * b + 1];
            const double2 T = a.T[(size_t(grp) * a.n_comm + t.comm) * ENS_B + b];
            const double acc_s = T.x - double(cs);
            const double acc_c = T.y - double(cc);
            const float2 own = tab[size_t(row) * ENS_B + b];
            const double f = a.omega[base + b] + a.scale[grp * ENS_B + b] *
                                                     (double(own.y) * acc_s - double(own.x) * acc_c);
            if (!isfinite(f)) atomicOr(a.err, ERR_NONFINITE);
            const size_t q = base + b;
            if (STAGE == ST_RHS) {
                rk.out[q] = f;
            } else if (STAGE == ST_1) {
                rk.krk[q] = f;
                rk.Y[q] = rk.y[q] + (0.5 * rk.h) * f;
            } else if (STAGE == ST_2) {
                rk.krk[q] = rk.krk[q] + 2.0 * f;
                rk.Y[q] = rk.y[q] + (0.5 * rk.h) * f;
            } else if (STAGE == ST_3) {
                rk.krk[q] = rk.krk[q] + 2.0 * f;
                rk.Y[q] = rk.y[q] + rk.h * f;
            } else {
                rk.y_out[q] = rk.y[q] + (rk.h / 6.0) * (rk.krk[q] + f);
            }
        }
    }
    if (tc) {
        if (!ok && tid == 0) {
            // let every copy and MMA in flight land before the CTA leaves
            for (int q = 0; q < 2; q++) {
                if (a_issued[q] > 0) mbar_wait_bounded(&a_full[q], uint32_t(a_issued[q] - 1) & 1u, LIMIT_NS);
                if (b_issued[q] > 0) mbar_wait_bounded(&b_full[q], uint32_t(b_issued[q] - 1) & 1u, LIMIT_NS);
            }
            mbar_wait_bounded(&d_full, 0u, LIMIT_NS);
        }
        tc_fence_before();
        __syncthreads();
        if (warp == ENS_MMA_WARP) tc_dealloc(tmem, ENS_TMEM_COLS);
    }
}

// theta [groups][ENS_B][n] user order <-> y [groups][n][ENS_B] permuted
__global__ void k_ens_gather(int64_t n, int groups, const int32_t* __restrict__ perm, const double* __restrict__ src,
                             double* __restrict__ dst)
{
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= n * ENS_B * groups) return;
    const int64_t grp = q / (n * ENS_B), rem = q % (n * ENS_B), i = rem / ENS_B, b = rem % ENS_B;
    dst[q] = src[(grp * ENS_B + b) * n + perm[i]];
}
__global__ void k_ens_scatter(int64_t n, int groups, const int32_t* __restrict__ perm, const double* __restrict__ src,
                              double* __restrict__ dst)
{
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= n * ENS_B * groups) return;
    const int64_t grp = q / (n * ENS_B), rem = q % (n * ENS_B), i = rem / ENS_B, b = rem % ENS_B;
    dst[(grp * ENS_B + b) * n + perm[i]] = src[q];
}

}  // namespace kura
