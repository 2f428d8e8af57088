// C ABI of libkura (declared in include/kura.h): handle, device buffers,
// CUDA-graph step loop and the host-only plan inspection entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <queue>
#include <string>
#include <vector>

#include "kura.h"
#include "kura_batch.cuh"
#include "kura_ensemble.cuh"
#include "kura_kernels.cuh"
#include "kura_small.cuh"
#include "plan.hpp"

using namespace kura;

namespace {

thread_local std::string g_create_error;

// SM count of the current device (the planner sizes tiles by it); 152, the
// GB300 count, if the query fails.
int current_sm_count()
{
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) {
        cudaGetLastError();
        return 152;
    }
    return nsm;
}

// ---------------------------------------------------------------- device memory
struct DevMem {
    void* p = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem&) = delete;
    DevMem& operator=(const DevMem&) = delete;
    ~DevMem() { release(); }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t alloc(size_t b)
    {
        release();
        if (b == 0) b = 16;
        cudaError_t e = cudaMalloc(&p, b);
        if (e == cudaSuccess) bytes = b;
        else p = nullptr;
        return e;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> events;   // begin/end pairs around every row-kernel launch
    ~GraphEntry()
    {
        if (exec) cudaGraphExecDestroy(exec);
        for (auto e : events) cudaEventDestroy(e);
    }
};

int ceil_log2(int64_t v)
{
    int k = 0;
    while ((int64_t(1) << k) < v) k++;
    return k;
}

}  // namespace

// Plan choices of one batch trajectory (set by kura_batch_create, moved by kura_autotune).
struct BatchChoice {
    double tau = 0.5;      // dense iff zero fraction < tau
    int32_t tc = 0;        // tensor-core masks: as kura_opts.tensor_cores
    int32_t lanes = 32;    // lanes that gather one row's listed entries: 32, 16 or 8
};

// Host copy of one batch trajectory's graph.
struct HostGraph {
    kura_graph_desc desc{};
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col, label;
    std::vector<double> omega;
    void rebind()
    {
        desc.omega = omega.data();
        desc.row_ptr = row_ptr.empty() ? nullptr : row_ptr.data();
        desc.col = row_ptr.empty() ? nullptr : col.data();
        desc.label = row_ptr.empty() ? nullptr : label.data();
    }
};

// Device data of a batch handle (kura_batch_create).
struct BatchData {
    int32_t n_traj = 0;
    int64_t n_total = 0, entries = 0, missing = 0, present = 0;
    int64_t tc_tiles = 0, tc_mask_bits = 0;   // tensor-core tiles and their mask bits (0: CUDA cores only)
    int32_t tc_traj = 0;                       // trajectories with tensor-core tiles
    DevMem traj, order, comm_off, dptr, dcol, node_comm, row_off, row_nm, entries_d, queue, stash, tc_tiles_d,
        tc_bits_d;
    std::vector<BatchChoice> choice;     // plan choices of every trajectory
    std::vector<HostGraph> host;         // host copies of the graphs (keep_host_csr), for kura_autotune
};

// Device data of an ensemble handle (kura_ensemble_create): trajectories in
// groups of ENS_B sharing one graph, node-major per group.
struct EnsData {
    int32_t groups = 0;
    int64_t nblk64 = 0;
    DevMem comm_off, dptr, dcol, tiles, lptr, lidx, bitmap, aimage, node_comm;
    DevMem table, image, bsum, T, omega, scale, y, Y, krk, f, user;
};

struct kura_ctx {
    std::string err;
    std::unique_ptr<BatchData> batch;    // non-null for a batch handle
    std::unique_ptr<EnsData> ens;        // non-null for an ensemble handle
    std::unique_ptr<kura_ctx> tr;        // plan of A^T for the adjoint of a directed A (built on first use)
    int device = 0;
    kura_opts opts{};
    int64_t n = 0;
    int32_t n_comm = 0;
    double K = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;        // capture stream (graphs are replayed on `stream`)
    cudaStream_t ad_stream = nullptr;  // adjoint: the recompute of the next segment runs here
    cudaEvent_t ad_ev[5] = {};         // adjoint: start, recompute done (per set), adjoint done (per set)
    // host copies
    std::vector<int64_t> h_row_ptr;
    std::vector<int32_t> h_col, h_label, h_val;   // h_val: values of a finite-valued matrix (else empty)
    std::vector<double> h_omega;        // user order
    Plan plan;                          // host plan (streams released after upload)
    int64_t miss_total = 0, pres_total = 0, nnz = 0, stream_bytes = 0, bitmap_rows = 0;
    int64_t tc_tiles = 0, tc_rows = 0, tc_mask_bits = 0;
    bool has_tc = false;                // some tile runs on the tensor cores (digit image kept up to date)
    int64_t tile_work = 0;              // planner work target per tile (0: automatic); set by kura_autotune
    int32_t bm_stash_off = 0;
    // device buffers
    DevMem perm, node_comm, gstream, groups, tiles, row_sub0, bitmap, dptr, dcol, comm_off, dig, dval, tcmask;
    bool valued = false;
    DevMem omega, rscale, rinvdeg, table, bsum, bsum_out, tot, T, Tq, counter, err_flags;
    DevMem table2, dig2, bsum4;               // fused trig: second table and digit image, 4 sum accumulators
    // adjoint (allocated on first use)
    DevMem ad_ck, ad_Y, ad_F, ad_lam, ad_asum, ad_a0, ad_a1, ad_w, ad_nu, ad_sc, ad_gom, ad_bs, ad_gk, ad_part,
        ad_tgt, ad_scratch, ad_absmax, ad_chunks, ad_chunk_ptr, ad_cpart,
        ad_Y2, ad_F2,                          // the second set of stage inputs and row sums
        ad_table, ad_dig;                      // the nu-weighted table and its digits (the adjoint's own)
    int32_t ad_nchunks = 0;
    int64_t ad_M = 0, ad_nck = 0;
    int sym = -1;   // host CSR symmetric? (-1 unknown)
    DevMem y, Y, krk, fbuf, user, red, order_out;
    // small graphs: per-row lists of the persistent cluster step loop (kura_small.cuh)
    bool small = false;
    int32_t small_P = 0;
    DevMem sm_row_off, sm_row_nm, sm_ent, sm_node_comm, sm_dptr, sm_dcol;
    DevMem deg, sums, diag;                   // diagnostics: degrees, row sums, partials (lazily)
    DevMem d_row_ptr, d_col, d_omega_user;   // direct baseline (user order), lazily uploaded
    int q_bits = 0;
    int32_t n_tiles = 0, max_wlen = 0;
    size_t row_smem = 0;
    // graphs
    std::map<std::pair<double, int64_t>, std::unique_ptr<GraphEntry>> graphs;
    GraphEntry* last_graph = nullptr;
    bool timing = false;

    kura_status fail(kura_status s, const char* fmt, ...)
    {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        err = buf;
        return s;
    }
    kura_status cuda_fail(cudaError_t e, const char* what)
    {
        return fail(e == cudaErrorMemoryAllocation ? KURA_ENOMEM : KURA_ECUDA, "%s: %s", what,
                    cudaGetErrorString(e));
    }
    ~kura_ctx()
    {
        if (device >= 0) cudaSetDevice(device);
        graphs.clear();
        if (cap) cudaStreamDestroy(cap);
        if (ad_stream) cudaStreamDestroy(ad_stream);
        for (cudaEvent_t e : ad_ev)
            if (e) cudaEventDestroy(e);
    }
};

#define KCHECK(h, call, what)                                  \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return (h)->cuda_fail(e_, what); \
    } while (0)

namespace {

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t upload(DevMem& d, const std::vector<T>& v, cudaStream_t s)
{
    cudaError_t e = d.alloc(sizeof(T) * std::max<size_t>(v.size(), 1));
    if (e != cudaSuccess) return e;
    if (v.empty()) return cudaMemsetAsync(d.p, 0, d.bytes, s);
    return cudaMemcpyAsync(d.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s);
}

DevGraph dev_graph(kura_ctx* h)
{
    DevGraph g{};
    g.n = h->n;
    g.n_comm = h->n_comm;
    g.q_bits = h->q_bits;
    g.scale_q = std::ldexp(1.0, h->q_bits);
    g.inv_scale_q = std::ldexp(1.0, -h->q_bits);
    g.scale = h->K / double(h->n);
    g.rscale = h->opts.scaling == KURA_SCALING_DEGREE ? h->rscale.as<double>() : nullptr;
    g.rinvdeg = h->opts.scaling == KURA_SCALING_DEGREE ? h->rinvdeg.as<double>() : nullptr;
    g.inv_n = 1.0 / double(h->n);
    g.node_comm = h->node_comm.as<int32_t>();
    g.gstream = h->gstream.as<int32_t>();
    g.groups = h->groups.as<Group>();
    g.tiles = h->tiles.as<Tile>();
    g.row_sub0 = h->row_sub0.as<int32_t>();
    g.bitmap = h->bitmap.as<uint32_t>();
    g.dig = h->has_tc ? h->dig.as<uint8_t>() : nullptr;
    g.tcmask = h->has_tc ? h->tcmask.as<uint8_t>() : nullptr;
    g.dval = h->valued ? h->dval.as<int32_t>() : nullptr;
    g.bm_stash_off = h->bm_stash_off;
    g.dptr = h->dptr.as<int64_t>();
    g.dcol = h->dcol.as<int32_t>();
    g.comm_off = h->comm_off.as<int64_t>();
    g.omega = h->omega.as<double>();
    g.table = h->table.p;
    g.bsum = h->bsum.as<unsigned long long>();
    g.bsum_out = h->bsum_out.as<long long>();
    g.tot = h->tot.as<long long>();
    g.T = h->T.p;
    g.Tq = h->Tq.as<long long>();
    g.counter = h->counter.as<unsigned int>();
    g.err = h->err_flags.as<int>();
    return g;
}

inline unsigned blocks_for(int64_t n, int threads) { return unsigned((n + threads - 1) / threads); }

// ---- launches of one right-hand-side evaluation on stream s
template <int MODE>
void launch_trig(kura_ctx* h, const DevGraph& g, const double* theta_perm, int what, cudaStream_t s)
{
    const unsigned nb = blocks_for(h->n, TRIG_THREADS);
    if (what == (TB_TABLE | TB_T)) k_trig_blocksum<MODE, TB_TABLE | TB_T><<<nb, TRIG_THREADS, 0, s>>>(g, theta_perm);
    else if (what == (TB_TABLE | TB_KEEP))
        k_trig_blocksum<MODE, TB_TABLE | TB_KEEP><<<nb, TRIG_THREADS, 0, s>>>(g, theta_perm);
    else k_trig_blocksum<MODE, 0><<<nb, TRIG_THREADS, 0, s>>>(g, theta_perm);
}

template <int MODE, int STAGE>
void launch_row(kura_ctx* h, const DevGraph& g, const RkArgs& rk, cudaStream_t s, const AdjArgs& adj = AdjArgs{})
{
    k_row_stage<MODE, STAGE><<<unsigned(h->n_tiles), ROW_THREADS, h->row_smem, s>>>(g, rk, adj);
}

template <int MODE>
void launch_row_stage(kura_ctx* h, const DevGraph& g, const RkArgs& rk, int stage, cudaStream_t s)
{
    switch (stage) {
    case ST_RHS: launch_row<MODE, ST_RHS>(h, g, rk, s); break;
    case ST_1: launch_row<MODE, ST_1>(h, g, rk, s); break;
    case ST_2: launch_row<MODE, ST_2>(h, g, rk, s); break;
    case ST_3: launch_row<MODE, ST_3>(h, g, rk, s); break;
    default: launch_row<MODE, ST_4>(h, g, rk, s); break;
    }
}

template <int MODE>
cudaError_t set_row_attrs(size_t smem)
{
    // The limit is a property of the kernel function on the device, shared by every handle: it only ever
    // grows, so that a handle built later with a smaller plan cannot shrink it below what another live
    // handle launches with.
    static std::mutex mu;
    static size_t granted[2][64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = granted[MODE == MODE_MIXED ? 1 : 0][dev >= 0 && dev < 64 ? dev : 0];
    if (smem <= cur) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const void* fns[] = {(const void*)k_row_stage<MODE, ST_RHS>, (const void*)k_row_stage<MODE, ST_1>,
                         (const void*)k_row_stage<MODE, ST_2>, (const void*)k_row_stage<MODE, ST_3>,
                         (const void*)k_row_stage<MODE, ST_4>, (const void*)k_row_stage<MODE, ST_ADJ>};
    for (const void* f : fns) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
    }
    cur = smem;
    return e;
}

RkArgs rk_args(kura_ctx* h, double step)
{
    RkArgs rk{};
    rk.y = h->y.as<double>();
    rk.y_out = h->y.as<double>();
    rk.Y = h->Y.as<double>();
    rk.krk = h->krk.as<double>();
    rk.out = h->fbuf.as<double>();
    rk.h = step;
    return rk;
}

// One RK4 step (4 stages) enqueued on s; events (if any) bracket the row kernels.
void enqueue_rk4_step(kura_ctx* h, double step, cudaStream_t s, cudaEvent_t* ev)
{
    const DevGraph g = dev_graph(h);
    const RkArgs rk = rk_args(h, step);
    for (int st = ST_1; st <= ST_4; st++) {
        const double* in = (st == ST_1) ? h->y.as<double>() : h->Y.as<double>();
        if (h->opts.precision == KURA_PREC_MIXED) launch_trig<MODE_MIXED>(h, g, in, TB_TABLE | TB_T, s);
        else launch_trig<MODE_FP64>(h, g, in, TB_TABLE | TB_T, s);
        if (ev) cudaEventRecordWithFlags(ev[2 * (st - 1)], s, cudaEventRecordExternal);
        if (h->opts.precision == KURA_PREC_MIXED) launch_row_stage<MODE_MIXED>(h, g, rk, st, s);
        else launch_row_stage<MODE_FP64>(h, g, rk, st, s);
        if (ev) cudaEventRecordWithFlags(ev[2 * (st - 1) + 1], s, cudaEventRecordExternal);
    }
}

// The fused trig (opts.fused_trig).  A run of RK4 stages starts with one
// trig/block-sum launch on the first stage's input: it makes the table in
// buffer 0 and leaves its block sums in accumulator 0.  Stage st = 1..4 of
// every step then reads table buffer (st - 1) mod 2 and accumulator st - 1;
// its row kernel writes the next stage's table into buffer st mod 2 and its
// sums into accumulator st mod 4, and clears accumulator (st + 1) mod 4, which
// no kernel of the stage touches.  Every step has four stages, so the same
// buffers serve every step.
void enqueue_fused_start(kura_ctx* h, const double* y_first, cudaStream_t s)
{
    unsigned long long* acc = h->bsum4.as<unsigned long long>();
    cudaMemsetAsync(acc, 0, 2 * 2 * size_t(h->n_comm) * sizeof(unsigned long long), s);   // accumulators 0, 1
    DevGraph g0 = dev_graph(h);
    g0.bsum = acc;
    if (h->opts.precision == KURA_PREC_MIXED) launch_trig<MODE_MIXED>(h, g0, y_first, TB_TABLE | TB_KEEP, s);
    else launch_trig<MODE_FP64>(h, g0, y_first, TB_TABLE | TB_KEEP, s);
}

// The tables, digit images and accumulators of fused stage st (see enqueue_fused_start).
void fused_stage_args(kura_ctx* h, int st, DevGraph& g, RkArgs& rk)
{
    void* tables[2] = {h->table.p, h->table2.p};
    uint8_t* digs[2] = {h->has_tc ? h->dig.as<uint8_t>() : nullptr, h->has_tc ? h->dig2.as<uint8_t>() : nullptr};
    unsigned long long* acc = h->bsum4.as<unsigned long long>();
    const size_t nc2 = 2 * size_t(h->n_comm);
    g.table = tables[(st - 1) % 2];
    g.dig = digs[(st - 1) % 2];
    rk.next_table = tables[st % 2];
    rk.next_dig = digs[st % 2];
    rk.bsum_cur = acc + nc2 * size_t(st - 1);
    rk.bsum_next = acc + nc2 * size_t(st % 4);
    rk.bsum_zero = acc + nc2 * size_t((st + 1) % 4);
}

// c RK4 steps enqueued on s; events (if any, 8 per step) bracket the row kernels.
void enqueue_rk4_steps(kura_ctx* h, double step, int64_t c, cudaStream_t s, cudaEvent_t* ev)
{
    if (!h->opts.fused_trig) {
        for (int64_t k = 0; k < c; k++) enqueue_rk4_step(h, step, s, ev ? ev + 8 * k : nullptr);
        return;
    }
    const bool mixed = h->opts.precision == KURA_PREC_MIXED;
    enqueue_fused_start(h, h->y.as<double>(), s);
    const RkArgs rk0 = rk_args(h, step);
    for (int64_t k = 0; k < c; k++) {
        for (int st = ST_1; st <= ST_4; st++) {
            DevGraph g = dev_graph(h);
            RkArgs rk = rk0;
            fused_stage_args(h, st, g, rk);
            if (ev) cudaEventRecordWithFlags(ev[8 * k + 2 * (st - 1)], s, cudaEventRecordExternal);
            if (mixed) launch_row_stage<MODE_MIXED>(h, g, rk, st, s);
            else launch_row_stage<MODE_FP64>(h, g, rk, st, s);
            if (ev) cudaEventRecordWithFlags(ev[8 * k + 2 * (st - 1) + 1], s, cudaEventRecordExternal);
        }
    }
}

// f(X) -> fbuf for a permuted state X (trig + row kernel, right-hand-side stage)
void enqueue_rhs_of(kura_ctx* h, const DevGraph& g, const double* X, cudaStream_t s)
{
    RkArgs rk = rk_args(h, 0.0);
    if (h->opts.precision == KURA_PREC_MIXED) {
        launch_trig<MODE_MIXED>(h, g, X, TB_TABLE | TB_T, s);
        launch_row_stage<MODE_MIXED>(h, g, rk, ST_RHS, s);
    } else {
        launch_trig<MODE_FP64>(h, g, X, TB_TABLE | TB_T, s);
        launch_row_stage<MODE_FP64>(h, g, rk, ST_RHS, s);
    }
}

// One step of explicit (method 1) or implicit (method 2, `iters` sweeps) midpoint on y; stage in Y.
void enqueue_rk2_step(kura_ctx* h, double step, int method, int iters, cudaStream_t s)
{
    const DevGraph g = dev_graph(h);
    const unsigned nb = blocks_for(h->n, 256);
    double* y = h->y.as<double>();
    double* Z = h->Y.as<double>();
    double* f = h->fbuf.as<double>();
    enqueue_rhs_of(h, g, y, s);
    k_axpy<<<nb, 256, 0, s>>>(h->n, Z, y, 0.5 * step, f);
    if (method == KURA_INT_RK2) {
        enqueue_rhs_of(h, g, Z, s);
        k_axpy<<<nb, 256, 0, s>>>(h->n, y, y, step, f);
        return;
    }
    for (int it = 0; it < iters; it++) {
        enqueue_rhs_of(h, g, Z, s);
        k_axpy<<<nb, 256, 0, s>>>(h->n, Z, y, 0.5 * step, f);
    }
    k_midpoint_final<<<nb, 256, 0, s>>>(h->n, y, Z);
}

EnsArgs ens_args(kura_ctx* h)
{
    EnsData& e = *h->ens;
    EnsArgs a{};
    a.n = h->n;
    a.n_comm = h->n_comm;
    a.groups = e.groups;
    a.node_comm = e.node_comm.as<int32_t>();
    a.comm_off = e.comm_off.as<int64_t>();
    a.dptr = e.dptr.as<int64_t>();
    a.dcol = e.dcol.as<int32_t>();
    a.tiles = e.tiles.as<Tile>();
    a.lptr = e.lptr.as<int64_t>();
    a.lidx = e.lidx.as<int32_t>();
    a.bitmap = e.bitmap.as<uint32_t>();
    a.aimage = e.aimage.as<uint8_t>();
    a.table = e.table.as<float2>();
    a.image = e.image.as<__nv_bfloat16>();
    a.nblk64 = e.nblk64;
    a.bsum = e.bsum.as<double2>();
    a.T = e.T.as<double2>();
    a.omega = e.omega.as<double>();
    a.scale = e.scale.as<double>();
    a.err = h->err_flags.as<int>();
    return a;
}

// One right-hand-side evaluation of every trajectory (stage `stage`), on stream s.
void enqueue_ens_stage(kura_ctx* h, const EnsArgs& a, const double* in, const RkArgs& rk, int stage, cudaStream_t s)
{
    const unsigned G = unsigned(a.groups);
    k_ens_trig<<<dim3(blocks_for(h->n, 256), G), 256, 0, s>>>(a, in);
    k_ens_bsum<<<dim3(unsigned(h->n_comm), G), 256, 0, s>>>(a);
    k_ens_T<<<dim3(blocks_for(int64_t(h->n_comm) * ENS_B, 256), G), 256, 0, s>>>(a);
    const unsigned grid = unsigned(h->n_tiles) * G;      // group fastest: a tile's groups share its mask images
    switch (stage) {
    case ST_RHS: k_ens_row<ST_RHS><<<grid, ENS_THREADS, ENS_SMEM, s>>>(a, rk); break;
    case ST_1: k_ens_row<ST_1><<<grid, ENS_THREADS, ENS_SMEM, s>>>(a, rk); break;
    case ST_2: k_ens_row<ST_2><<<grid, ENS_THREADS, ENS_SMEM, s>>>(a, rk); break;
    case ST_3: k_ens_row<ST_3><<<grid, ENS_THREADS, ENS_SMEM, s>>>(a, rk); break;
    default: k_ens_row<ST_4><<<grid, ENS_THREADS, ENS_SMEM, s>>>(a, rk); break;
    }
}

RkArgs ens_rk_args(kura_ctx* h, double step)
{
    EnsData& e = *h->ens;
    RkArgs rk{};
    rk.y = e.y.as<double>();
    rk.y_out = e.y.as<double>();
    rk.Y = e.Y.as<double>();
    rk.krk = e.krk.as<double>();
    rk.out = e.f.as<double>();
    rk.h = step;
    return rk;
}

void enqueue_ens_step(kura_ctx* h, double step, cudaStream_t s)
{
    const EnsArgs a = ens_args(h);
    const RkArgs rk = ens_rk_args(h, step);
    for (int st = ST_1; st <= ST_4; st++)
        enqueue_ens_stage(h, a, st == ST_1 ? rk.y : rk.Y, rk, st, s);
}

// Bytes of the correction data one right-hand side reads: the listed indices
// (4 B each), the sub-row headers (16 B each), the row bitmaps, and for
// tensor-core tiles their mask bits and the digit blocks of their K-blocks.
int64_t plan_stream_bytes(const Plan& p)
{
    int64_t listed = 0;
    for (const Group& G : p.groups) listed += G.len - 4 * int64_t(G.nsub);   // includes segment padding
    int64_t bm = 0;
    for (const Tile& t : p.tiles) {
        if (t.flags & TILE_BITMAP) bm += int64_t(t.r1 - t.r0) * t.nsw * 128;
        if (t.flags & TILE_TC)     // FP8 mask images (16 KB per 128 x 128 block) and digit blocks
            bm += int64_t((t.r1 - t.r0 + TC_MBLOCK - 1) / TC_MBLOCK) * t.nsw * TC_ABYTES +
                  int64_t(t.nsw) * TC_BBYTES;
    }
    return 4 * listed + 16 * int64_t(p.row_sub0.empty() ? 0 : p.row_sub0.back()) + bm;
}

// Per-row lists for the persistent cluster step loop of small graphs, from the host CSR and the plan's
// permutation and dense blocks: [zeros of the row's dense blocks (the diagonal excluded) | non-zeros of its
// sparse blocks], permuted columns.  Only graphs with n <= SMALL_MAX_N, n_comm <= SMALL_MAX_COMM, a 0/1
// matrix, the host CSR kept and at most 16 listed entries per row on average take this path.
kura_status build_small(kura_ctx* h)
{
    h->small = false;
    const Plan& p = h->plan;
    const int64_t n = h->n;
    if (!h->opts.persistent_small || p.valued || n > SMALL_MAX_N || h->n_comm > SMALL_MAX_COMM ||
        (h->h_col.empty() && h->nnz > 0))
        return KURA_OK;
    const int nc = h->n_comm;
    std::vector<int32_t> inv(static_cast<size_t>(n));
    for (int64_t r = 0; r < n; r++) inv[size_t(p.perm[size_t(r)])] = int32_t(r);
    std::vector<uint8_t> dense(size_t(nc) * size_t(nc), 0);
    for (int I = 0; I < nc; I++)
        for (int64_t k = p.dptr[size_t(I)]; k < p.dptr[size_t(I) + 1]; k++) dense[size_t(I) * nc + size_t(p.dcol[size_t(k)])] = 1;
    std::vector<int32_t> row_off(size_t(n) + 1, 0), row_nm(size_t(n), 0), ent;
    std::vector<uint8_t> mark(static_cast<size_t>(n), 0);
    for (int64_t r = 0; r < n; r++) {
        const int64_t v = p.perm[size_t(r)];
        const int I = p.node_comm[size_t(r)];
        const int64_t b = h->h_row_ptr[size_t(v)], e = h->h_row_ptr[size_t(v) + 1];
        for (int64_t q = b; q < e; q++) mark[size_t(inv[size_t(h->h_col[size_t(q)])])] = 1;
        int32_t nm = 0;
        for (int64_t k = p.dptr[size_t(I)]; k < p.dptr[size_t(I) + 1]; k++) {
            const int J = p.dcol[size_t(k)];
            for (int64_t c = p.comm_off[size_t(J)]; c < p.comm_off[size_t(J) + 1]; c++)
                if (!mark[size_t(c)] && c != r) { ent.push_back(int32_t(c)); nm++; }
        }
        for (int64_t q = b; q < e; q++) {
            const int32_t c = inv[size_t(h->h_col[size_t(q)])];
            if (c != r && !dense[size_t(I) * nc + size_t(p.node_comm[size_t(c)])]) ent.push_back(c);
        }
        for (int64_t q = b; q < e; q++) mark[size_t(inv[size_t(h->h_col[size_t(q)])])] = 0;
        row_nm[size_t(r)] = nm;
        row_off[size_t(r) + 1] = int32_t(ent.size());
        if (int64_t(ent.size()) > 16 * n) return KURA_OK;        // too many listed entries: keep the graph loop
    }
    std::vector<int32_t> nci(p.node_comm.begin(), p.node_comm.end());
    std::vector<int32_t> dp(p.dptr.begin(), p.dptr.end()), dc(p.dcol.begin(), p.dcol.end());
    cudaStream_t s = h->stream;
    KCHECK(h, upload(h->sm_row_off, row_off, s), "upload small-graph rows");
    KCHECK(h, upload(h->sm_row_nm, row_nm, s), "upload small-graph rows");
    KCHECK(h, upload(h->sm_ent, ent, s), "upload small-graph entries");
    KCHECK(h, upload(h->sm_node_comm, nci, s), "upload small-graph communities");
    KCHECK(h, upload(h->sm_dptr, dp, s), "upload small-graph dense blocks");
    KCHECK(h, upload(h->sm_dcol, dc, s), "upload small-graph dense blocks");
    h->small_P = int32_t(((n + SMALL_CLUSTER - 1) / SMALL_CLUSTER + 31) / 32 * 32);
    h->small = true;
    return KURA_OK;
}

// All n_steps RK4 steps of a small graph in one launch of one cluster of SMALL_CLUSTER CTAs (the permuted
// state in h->y).
kura_status launch_small(kura_ctx* h, double step, int64_t n_steps, cudaStream_t s)
{
    SmallArgs a{};
    a.n = int(h->n);
    a.n_comm = h->n_comm;
    a.P = h->small_P;
    a.node_comm = h->sm_node_comm.as<int32_t>();
    a.dptr = h->sm_dptr.as<int32_t>();
    a.dcol = h->sm_dcol.as<int32_t>();
    a.row_off = h->sm_row_off.as<int32_t>();
    a.row_nm = h->sm_row_nm.as<int32_t>();
    a.ent = h->sm_ent.as<int32_t>();
    a.omega = h->omega.as<double>();
    a.rscale = h->opts.scaling == KURA_SCALING_DEGREE ? h->rscale.as<double>() : nullptr;
    a.scale = h->K / double(h->n);
    a.scale_q = std::ldexp(1.0, h->q_bits);
    a.inv_scale_q = std::ldexp(1.0, -h->q_bits);
    a.y = h->y.as<double>();
    a.err = h->err_flags.as<int>();
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(SMALL_CLUSTER);
    cfg.blockDim = dim3(SMALL_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = SMALL_CLUSTER;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = h->opts.precision == KURA_PREC_MIXED
                        ? cudaLaunchKernelEx(&cfg, k_small_rk4<MODE_MIXED>, a, step, n_steps)
                        : cudaLaunchKernelEx(&cfg, k_small_rk4<MODE_FP64>, a, step, n_steps);
    KCHECK(h, e, "launching the small-graph step loop");
    return KURA_OK;
}

kura_status build_device(kura_ctx* h, Plan&& plan)
{
    cudaStream_t s = h->stream;
    h->plan = std::move(plan);
    Plan& p = h->plan;
    h->n_tiles = int32_t(p.tiles.size());
    h->max_wlen = p.max_wlen;
    h->miss_total = p.miss_total;
    h->pres_total = p.pres_total;
    h->bitmap_rows = p.bitmap_rows;
    h->tc_tiles = p.tc_tiles;
    h->tc_rows = p.tc_rows;
    h->tc_mask_bits = p.tc_mask_bits;
    h->has_tc = p.tc_tiles > 0;
    h->stream_bytes = plan_stream_bytes(p);
    h->valued = p.valued;
    // fixed point: n values of at most 2^q each, times the largest weight, stay below 2^61
    h->q_bits = 61 - ceil_log2(std::max<int64_t>(h->n, 2)) - (p.valued ? ceil_log2(int64_t(p.max_weight) + 1) : 0);
    const int mode = h->opts.precision == KURA_PREC_MIXED ? MODE_MIXED : MODE_FP64;
    const size_t esize = h->opts.precision == KURA_PREC_MIXED ? sizeof(float2) : sizeof(longlong2);
    // dynamic shared memory: the ring, then either [16 B | window | bitmap-pass
    // stash] or the tensor-core operand stages
    const size_t win_end = size_t(ring_bytes_for(mode)) + 16 + ((size_t(std::max(p.max_wlen, 2)) * esize + 15) & ~size_t(15));
    h->bm_stash_off = int32_t(win_end);
    size_t need = p.bitmap_rows > 0 ? win_end + size_t(TILE_MAX_ROWS) * 2 * (esize / 2) : win_end;
    if (h->has_tc) need = std::max(need, size_t(ring_bytes_for(mode)) + size_t(TC_SMEM));
    h->row_smem = need;
    KCHECK(h, (h->opts.precision == KURA_PREC_MIXED ? set_row_attrs<MODE_MIXED>(h->row_smem)
                                                    : set_row_attrs<MODE_FP64>(h->row_smem)),
           "setting the row kernel's shared-memory size");

    KCHECK(h, upload(h->perm, p.perm, s), "upload perm");
    KCHECK(h, upload(h->node_comm, p.node_comm, s), "upload node_comm");
    KCHECK(h, upload(h->gstream, p.gstream, s), "upload the correction stream");
    KCHECK(h, upload(h->groups, p.groups, s), "upload row groups");
    KCHECK(h, upload(h->tiles, p.tiles, s), "upload tiles");
    KCHECK(h, upload(h->row_sub0, p.row_sub0, s), "upload row_sub0");
    KCHECK(h, upload(h->bitmap, p.bitmap, s), "upload row bitmaps");
    KCHECK(h, upload(h->dptr, p.dptr, s), "upload dptr");
    KCHECK(h, upload(h->dcol, p.dcol, s), "upload dcol");
    if (p.valued) KCHECK(h, upload(h->dval, p.dval, s), "upload block values");
    KCHECK(h, upload(h->comm_off, p.comm_off, s), "upload comm_off");
    {
        std::vector<double> om(size_t(h->n));
        for (int64_t v = 0; v < h->n; v++) om[size_t(v)] = h->h_omega[size_t(p.perm[size_t(v)])];
        KCHECK(h, upload(h->omega, om, s), "upload omega");
        std::vector<double> rs;
        if (h->opts.scaling == KURA_SCALING_DEGREE) {
            rs.resize(size_t(h->n));
            for (int64_t v = 0; v < h->n; v++) rs[size_t(v)] = p.deg[size_t(v)] > 0 ? h->K / p.deg[size_t(v)] : 0.0;
        }
        KCHECK(h, upload(h->rscale, rs, s), "upload rscale");
        std::vector<double> ri;
        if (h->opts.scaling == KURA_SCALING_DEGREE) {
            ri.resize(size_t(h->n));
            for (int64_t v = 0; v < h->n; v++) ri[size_t(v)] = p.deg[size_t(v)] > 0 ? 1.0 / p.deg[size_t(v)] : 0.0;
        }
        KCHECK(h, upload(h->rinvdeg, ri, s), "upload rinvdeg");
    }
    const size_t n = size_t(h->n), nc = size_t(h->n_comm);
    // two tables and digit images: with the fused trig a stage reads one and writes the other
    for (DevMem* d : {&h->table, &h->table2}) {
        KCHECK(h, d->alloc(esize * (n + 2)), "alloc table");
        KCHECK(h, cudaMemsetAsync(d->p, 0, d->bytes, s), "memset table");
    }
    KCHECK(h, h->bsum4.alloc(4 * 16 * nc), "alloc the fused block-sum accumulators");
    KCHECK(h, cudaMemsetAsync(h->bsum4.p, 0, h->bsum4.bytes, s), "memset the fused block-sum accumulators");
    if (h->has_tc) {
        // digit images: one 4 KB block per 128 nodes; columns past n stay zero
        for (DevMem* d : {&h->dig, &h->dig2}) {
            KCHECK(h, d->alloc(size_t((h->n + TC_KBLOCK - 1) / TC_KBLOCK) * TC_BBYTES), "alloc digit image");
            KCHECK(h, cudaMemsetAsync(d->p, 0, d->bytes, s), "memset digit image");
        }
        // mask images: every 128 x 128 block of mask bits (512 words) as 16 KB of FP8 operand
        const int64_t n_blocks = int64_t(p.bitmap.size()) / (TC_MBLOCK * 4);
        KCHECK(h, h->tcmask.alloc(size_t(n_blocks) * TC_ABYTES), "alloc mask images");
        k_tc_expand_masks<<<blocks_for(n_blocks * TC_MBLOCK, 256), 256, 0, s>>>(h->bitmap.as<uint32_t>(), n_blocks,
                                                                             h->tcmask.as<uint8_t>());
        KCHECK(h, cudaGetLastError(), "expanding the masks");
    } else {
        h->dig.release();
        h->dig2.release();
        h->tcmask.release();
    }
    KCHECK(h, h->bsum.alloc(16 * nc), "alloc bsum");
    KCHECK(h, cudaMemsetAsync(h->bsum.p, 0, h->bsum.bytes, s), "memset bsum");
    KCHECK(h, h->bsum_out.alloc(16 * nc), "alloc bsum_out");
    KCHECK(h, h->tot.alloc(16), "alloc tot");
    KCHECK(h, h->T.alloc(16 * nc), "alloc T");
    KCHECK(h, h->Tq.alloc(16 * nc), "alloc fixed-point T");
    KCHECK(h, h->counter.alloc(16), "alloc counter");
    KCHECK(h, cudaMemsetAsync(h->counter.p, 0, 16, s), "memset counter");
    if (!h->err_flags.p) {
        KCHECK(h, h->err_flags.alloc(16), "alloc error flags");
        KCHECK(h, cudaMemsetAsync(h->err_flags.p, 0, 16, s), "memset error flags");
    }
    for (DevMem* d : {&h->y, &h->Y, &h->krk, &h->fbuf, &h->user}) KCHECK(h, d->alloc(8 * n), "alloc state");
    KCHECK(h, h->order_out.alloc(8 * (2 + 2 * nc)), "alloc order_out");
    if (kura_status st = build_small(h)) return st;
    KCHECK(h, cudaStreamSynchronize(s), "upload");
    // the correction stream now lives on the device
    std::vector<int32_t>().swap(p.gstream);
    std::vector<uint32_t>().swap(p.bitmap);
    h->deg.release();
    h->graphs.clear();
    h->last_graph = nullptr;
    return KURA_OK;
}

kura_status check_handle(kura_t h)
{
    if (!h) return KURA_EINVAL;
    cudaSetDevice(h->device);
    return KURA_OK;
}

// Calls that need a single-graph handle.
kura_status check_single(kura_t h)
{
    if (!h) return KURA_EINVAL;
    if (h->batch) return h->fail(KURA_ESTATE, "not available on a batch handle");
    if (h->ens) return h->fail(KURA_ESTATE, "not available on an ensemble handle");
    cudaSetDevice(h->device);
    return KURA_OK;
}

// Latched device conditions -> status (clears them).
kura_status read_flags(kura_t h)
{
    int flags = 0;
    KCHECK(h, cudaMemcpyAsync(&flags, h->err_flags.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "read flags");
    KCHECK(h, cudaStreamSynchronize(h->stream), "synchronise");
    if (flags) {
        KCHECK(h, cudaMemsetAsync(h->err_flags.p, 0, sizeof(int), h->stream), "clear flags");
        if (flags & ERR_TIMEOUT) return h->fail(KURA_ETIMEOUT, "a bounded device-side wait gave up");
        if (flags & ERR_NONFINITE) return h->fail(KURA_ENUMERIC, "non-finite phase or right-hand side");
    }
    return KURA_OK;
}

// Resolves a user vector: device pointer used as is, host pointer staged
// through the handle's `user` buffer.
kura_status stage_in(kura_t h, const double* src, const double** dev, bool* host)
{
    *host = !is_device_ptr(src);
    if (*host) {
        KCHECK(h, cudaMemcpyAsync(h->user.p, src, size_t(h->n) * 8, cudaMemcpyHostToDevice, h->stream), "copy in");
        *dev = h->user.as<double>();
    } else {
        *dev = src;
    }
    return KURA_OK;
}

}  // namespace

// =========================================================================
extern "C" {

void kura_default_opts(kura_opts* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = KURA_PREC_FP64;
    o->scaling = KURA_SCALING_UNIFORM;
    o->tau = 0.5;
    o->keep_host_csr = 1;
    o->tensor_cores = 1;
    o->bitmap_zmin = -1.0;
    o->persistent_small = 1;
    o->fused_trig = 1;
}

int32_t kura_version(void) { return 100; }

const char* kura_status_string(kura_status s)
{
    switch (s) {
    case KURA_OK: return "ok";
    case KURA_EINVAL: return "invalid argument";
    case KURA_ENOMEM: return "out of memory";
    case KURA_ECUDA: return "CUDA error";
    case KURA_ESTATE: return "invalid state";
    case KURA_ETIMEOUT: return "device wait timed out";
    case KURA_ENUMERIC: return "non-finite value";
    }
    return "unknown status";
}

const char* kura_last_error(kura_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

static kura_status create_impl(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* val,
                               const int32_t* label, int32_t n_comm, const double* omega, double K,
                               const kura_opts* opts, void* stream, kura_t* out);

kura_status kura_create(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* label,
                        int32_t n_comm, const double* omega, double K, const kura_opts* opts, void* stream,
                        kura_t* out)
{
    return create_impl(n, row_ptr, col, nullptr, label, n_comm, omega, K, opts, stream, out);
}

kura_status kura_create_valued(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* val,
                               const int32_t* label, int32_t n_comm, const double* omega, double K,
                               const kura_opts* opts, void* stream, kura_t* out)
{
    g_create_error.clear();
    if (!val) {
        g_create_error = "val is NULL";
        if (out) *out = nullptr;
        return KURA_EINVAL;
    }
    return create_impl(n, row_ptr, col, val, label, n_comm, omega, K, opts, stream, out);
}

static kura_status create_impl(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* val,
                               const int32_t* label, int32_t n_comm, const double* omega, double K,
                               const kura_opts* opts, void* stream, kura_t* out)
{
    g_create_error.clear();
    if (!out) { g_create_error = "out is NULL"; return KURA_EINVAL; }
    *out = nullptr;
    kura_opts o;
    kura_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != KURA_PREC_FP64 && o.precision != KURA_PREC_MIXED) { g_create_error = "bad precision"; return KURA_EINVAL; }
    if (o.scaling != KURA_SCALING_UNIFORM && o.scaling != KURA_SCALING_DEGREE) { g_create_error = "bad scaling"; return KURA_EINVAL; }
    if (!omega || !std::isfinite(K)) { g_create_error = "omega is NULL or K is not finite"; return KURA_EINVAL; }
    if (n > 0) {
        for (int64_t i = 0; i < n; i++)
            if (!std::isfinite(omega[i])) { g_create_error = "omega has a non-finite entry"; return KURA_EINVAL; }
    }
    if (val && o.scaling != KURA_SCALING_UNIFORM) {
        g_create_error = "finite-valued matrices use uniform scaling";
        return KURA_EINVAL;
    }
    PlanInput in;
    in.n_sms = current_sm_count();
    in.n = n; in.row_ptr = row_ptr; in.col = col; in.label = label; in.n_comm = n_comm; in.tau = o.tau;
    in.val = val;
    in.tile_max_rows = TILE_MAX_ROWS;
    in.tile_max_sub = tile_max_sub_for(o.precision == KURA_PREC_MIXED ? MODE_MIXED : MODE_FP64);
    in.slot_ints = slot_ints_for(o.precision == KURA_PREC_MIXED ? MODE_MIXED : MODE_FP64);
    in.entry_bytes = o.precision == KURA_PREC_MIXED ? 8 : 16;
    in.bitmap_zmin = o.bitmap_zmin;
    in.tensor_cores = o.tensor_cores;
    Plan plan;
    std::string err;
    int rc = build_plan(in, plan, err);
    if (rc) { g_create_error = err; return rc == 2 ? KURA_ENOMEM : KURA_EINVAL; }

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        g_create_error = std::string("no usable CUDA device: ") + cudaGetErrorString(e);
        return KURA_ECUDA;
    }
    std::unique_ptr<kura_ctx> h(new (std::nothrow) kura_ctx());
    if (!h) { g_create_error = "out of host memory"; return KURA_ENOMEM; }
    cudaGetDevice(&h->device);
    h->opts = o;
    h->n = n;
    h->n_comm = n_comm;
    h->K = K;
    h->stream = static_cast<cudaStream_t>(stream);
    h->nnz = row_ptr[n];
    if ((e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking)) != cudaSuccess) {
        g_create_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
        return KURA_ECUDA;
    }
    h->h_omega.assign(omega, omega + n);
    if (o.keep_host_csr) {
        h->h_row_ptr.assign(row_ptr, row_ptr + n + 1);
        h->h_col.assign(col, col + row_ptr[n]);
        h->h_label.assign(label, label + n);
        if (val) h->h_val.assign(val, val + row_ptr[n]);
    }
    kura_status st = build_device(h.get(), std::move(plan));
    if (st != KURA_OK) { g_create_error = h->err; return st; }
    *out = h.release();
    return KURA_OK;
}

kura_status kura_get_stats(kura_t h, kura_block_stats* s)
{
    if (check_handle(h) || !s) return KURA_EINVAL;
    std::memset(s, 0, sizeof *s);
    const Plan& p = h->plan;
    s->n = h->n;
    s->nnz = h->nnz;
    s->self_loops = p.self_loops;
    s->n_comm = h->n_comm;
    s->q_bits = h->q_bits;
    s->tau = p.tau;
    s->dense_blocks = p.dense_blocks;
    s->sparse_blocks = p.sparse_blocks;
    s->nonempty_blocks = p.nonempty_blocks;
    s->missing_entries = h->miss_total;
    s->sparse_entries = h->pres_total;
    s->max_row_entries = p.max_row_entries;
    s->tiles = h->n_tiles;
    s->max_window = h->max_wlen;
    const int64_t esize = h->opts.precision == KURA_PREC_MIXED ? 8 : 16;
    // algorithmic bytes: 4 B per listed index, a 16 B header per sub-row, the row bitmaps, the
    // tensor-core operands; with the fused trig also the next stage's digit image (32 B per node)
    s->stream_bytes = h->stream_bytes + (h->opts.fused_trig && h->has_tc ? 32 * h->n : 0);
    // row kernel per node: omega, y, krk (read+write), Y (write) or y (write), own entry, and with
    // the fused trig the next stage's table entry
    s->node_bytes_row = (8 + 8 + 16 + 8 + esize + (h->opts.fused_trig ? esize : 0)) * h->n;
    // trig kernel per node: theta read, table write, community id
    s->node_bytes_trig = (8 + esize + 4) * h->n;
    s->direct_edges = h->nnz - p.self_loops;
    s->tc_tiles = h->tc_tiles;
    s->tc_rows = h->tc_rows;
    s->tc_mask_bits = h->tc_mask_bits;
    return KURA_OK;
}

kura_status kura_classify_blocks(kura_t h, double tau, kura_block_stats* stats)
{
    if (kura_status st0 = check_single(h)) return st0;
    if (tau >= 0) {
        if (tau > 1.0) return h->fail(KURA_EINVAL, "tau must be in [0, 1]");
        if (h->h_col.empty() && h->nnz > 0)
            return h->fail(KURA_ESTATE, "re-classification needs the host CSR copy (keep_host_csr = 1)");
        PlanInput in;
        in.n_sms = current_sm_count();
        in.n = h->n; in.row_ptr = h->h_row_ptr.data(); in.col = h->h_col.data(); in.label = h->h_label.data();
        in.n_comm = h->n_comm; in.tau = tau;
        in.val = h->h_val.empty() ? nullptr : h->h_val.data();
        in.tile_max_rows = TILE_MAX_ROWS;
        in.tile_max_sub = tile_max_sub_for(h->opts.precision == KURA_PREC_MIXED ? MODE_MIXED : MODE_FP64);
        in.slot_ints = slot_ints_for(h->opts.precision == KURA_PREC_MIXED ? MODE_MIXED : MODE_FP64);
        in.entry_bytes = h->opts.precision == KURA_PREC_MIXED ? 8 : 16;
        in.bitmap_zmin = h->opts.bitmap_zmin;
        in.tensor_cores = h->opts.tensor_cores;
        in.tile_work = h->tile_work;
        Plan plan;
        std::string err;
        int rc = build_plan(in, plan, err);
        if (rc) return h->fail(rc == 2 ? KURA_ENOMEM : KURA_EINVAL, "%s", err.c_str());
        KCHECK(h, cudaStreamSynchronize(h->stream), "synchronise before re-classification");
        kura_status st = build_device(h, std::move(plan));
        if (st) return st;
    }
    return stats ? kura_get_stats(h, stats) : KURA_OK;
}

namespace {

// Plan of the handle's host CSR with the given parameters, uploaded.
kura_status rebuild_plan(kura_t h, double tau, int32_t tensor_cores, int64_t tile_work)
{
    PlanInput in;
    in.n_sms = current_sm_count();
    in.n = h->n; in.row_ptr = h->h_row_ptr.data(); in.col = h->h_col.data(); in.label = h->h_label.data();
    in.n_comm = h->n_comm; in.tau = tau;
    in.val = h->h_val.empty() ? nullptr : h->h_val.data();
    const int mode = h->opts.precision == KURA_PREC_MIXED ? MODE_MIXED : MODE_FP64;
    in.tile_max_rows = TILE_MAX_ROWS;
    in.tile_max_sub = tile_max_sub_for(mode);
    in.slot_ints = slot_ints_for(mode);
    in.entry_bytes = mode == MODE_MIXED ? 8 : 16;
    in.bitmap_zmin = h->opts.bitmap_zmin;
    in.tensor_cores = tensor_cores;
    in.tile_work = tile_work;
    Plan plan;
    std::string err;
    int rc = build_plan(in, plan, err);
    if (rc) return h->fail(rc == 2 ? KURA_ENOMEM : KURA_EINVAL, "%s", err.c_str());
    KCHECK(h, cudaStreamSynchronize(h->stream), "synchronise before re-planning");
    kura_status st = build_device(h, std::move(plan));
    if (st) return st;
    h->opts.tau = tau;
    h->opts.tensor_cores = tensor_cores;
    h->tile_work = tile_work;
    return KURA_OK;
}

// Median of `reps` timed right-hand sides (after two untimed ones).
kura_status time_rhs(kura_t h, const double* theta, double* out, int reps, double* ms)
{
    cudaEvent_t e0, e1;
    KCHECK(h, cudaEventCreate(&e0), "event");
    KCHECK(h, cudaEventCreate(&e1), "event");
    std::vector<float> t;
    kura_status st = KURA_OK;
    for (int r = 0; r < reps + 2 && st == KURA_OK; r++) {
        cudaEventRecord(e0, h->stream);
        st = kura_rhs(h, theta, out);
        cudaEventRecord(e1, h->stream);
        if (st == KURA_OK && cudaEventSynchronize(e1) != cudaSuccess) st = h->fail(KURA_ECUDA, "timing the right-hand side");
        float v = 0.0f;
        cudaEventElapsedTime(&v, e0, e1);
        if (r >= 2) t.push_back(v);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == KURA_OK) st = read_flags(h);
    if (st) return st;
    std::sort(t.begin(), t.end());
    *ms = double(t[t.size() / 2]);
    return KURA_OK;
}

}  // namespace

static kura_status batch_autotune(kura_t h, const double* theta, double budget_s, kura_tune_result* out);

kura_status kura_autotune(kura_t h, const double* theta, double budget_s, kura_tune_result* out)
{
    if (h && h->batch) {
        cudaSetDevice(h->device);
        if (!theta || !out) return h->fail(KURA_EINVAL, "theta or out is NULL");
        return batch_autotune(h, theta, budget_s, out);
    }
    if (kura_status st0 = check_single(h)) return st0;
    if (!theta || !out) return h->fail(KURA_EINVAL, "theta or out is NULL");
    if (h->h_col.empty() && h->nnz > 0)
        return h->fail(KURA_ESTATE, "the autotuner rebuilds plans from the host CSR copy (keep_host_csr = 1)");
    const auto t_start = std::chrono::steady_clock::now();
    auto elapsed = [&]() {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    };
    std::memset(out, 0, sizeof *out);
    DevMem scratch;
    KCHECK(h, scratch.alloc(size_t(h->n) * 8), "alloc tuning output");
    double* f = scratch.as<double>();
    const int reps = 5;
    double best_ms = 0.0;
    if (kura_status st = time_rhs(h, theta, f, reps, &best_ms)) return st;
    out->initial_rhs_ms = best_ms;
    int32_t cand = 1;
    double best_tau = h->opts.tau;
    int32_t best_tc = h->opts.tensor_cores;
    // the automatic work target, as the planner computes it
    int64_t total = 0;
    for (int64_t v = 0; v < h->n; v++) total += h->plan.miss_cnt[size_t(v)] + h->plan.pres_cnt[size_t(v)] + 8;
    const int64_t auto_work = std::max<int64_t>(2048, total / (int64_t(current_sm_count()) * 12));
    int64_t best_work = h->tile_work > 0 ? h->tile_work : auto_work;
    auto try_plan = [&](double tau, int32_t tc, int64_t work) -> kura_status {
        if (elapsed() > budget_s) return KURA_OK;
        if (kura_status st = rebuild_plan(h, tau, tc, work)) return st;
        double ms = 0.0;
        if (kura_status st = time_rhs(h, theta, f, reps, &ms)) return st;
        cand++;
        if (ms < best_ms) {
            best_ms = ms;
            best_tau = tau;
            best_tc = tc;
            best_work = work;
        }
        return KURA_OK;
    };
    // one parameter at a time, each from the best so far
    for (int32_t tc : {1, 0})
        if (tc != best_tc)
            if (kura_status st = try_plan(best_tau, tc, best_work)) return st;
    for (double sc : {0.6, 1.6}) {
        const int64_t w = std::max<int64_t>(1024, int64_t(double(best_work) * sc));
        if (kura_status st = try_plan(best_tau, best_tc, w)) return st;
    }
    for (double tau : {0.35, 0.65})
        if (tau != best_tau)
            if (kura_status st = try_plan(tau, best_tc, best_work)) return st;
    // keep the winner on the handle
    if (h->opts.tau != best_tau || h->opts.tensor_cores != best_tc || h->tile_work != best_work)
        if (kura_status st = rebuild_plan(h, best_tau, best_tc, best_work)) return st;
    out->tau = best_tau;
    out->tensor_cores = best_tc;
    out->tile_work = best_work;
    out->rhs_ms = best_ms;
    out->candidates = cand;
    out->seconds = elapsed();
    return KURA_OK;
}

kura_status kura_set_stream(kura_t h, void* stream)
{
    if (check_handle(h)) return KURA_EINVAL;
    h->stream = static_cast<cudaStream_t>(stream);
    return KURA_OK;
}

kura_status kura_sync(kura_t h)
{
    if (check_handle(h)) return KURA_EINVAL;
    return read_flags(h);
}

static kura_status ens_rhs(kura_t h, const double* theta, double* dtheta);
static kura_status ens_rk4_steps(kura_t h, double* theta, double step, int64_t n_steps);

static kura_status batch_launch(kura_t h, const double* theta, double* out, double step, int64_t n_steps,
                                bool rhs_only);

kura_status kura_rhs(kura_t h, const double* theta, double* dtheta)
{
    if (h && h->ens) {
        cudaSetDevice(h->device);
        return ens_rhs(h, theta, dtheta);
    }
    if (h && h->batch) {
        cudaSetDevice(h->device);
        if (!theta || !dtheta || theta == dtheta) return h->fail(KURA_EINVAL, "theta/dtheta NULL or aliased");
        return batch_launch(h, theta, dtheta, 0.0, 1, true);
    }
    if (kura_status st0 = check_single(h)) return st0;
    if (!theta || !dtheta || theta == dtheta) return h->fail(KURA_EINVAL, "theta/dtheta NULL or aliased");
    const double* th_dev;
    bool host_in;
    if (kura_status st = stage_in(h, theta, &th_dev, &host_in)) return st;
    const bool host_out = !is_device_ptr(dtheta);
    cudaStream_t s = h->stream;
    const DevGraph g = dev_graph(h);
    RkArgs rk = rk_args(h, 0.0);
    const unsigned nb = blocks_for(h->n, 256);
    k_gather_perm<<<nb, 256, 0, s>>>(h->n, h->perm.as<int32_t>(), th_dev, h->Y.as<double>());
    if (h->opts.precision == KURA_PREC_MIXED) {
        launch_trig<MODE_MIXED>(h, g, h->Y.as<double>(), TB_TABLE | TB_T, s);
        launch_row_stage<MODE_MIXED>(h, g, rk, ST_RHS, s);
    } else {
        launch_trig<MODE_FP64>(h, g, h->Y.as<double>(), TB_TABLE | TB_T, s);
        launch_row_stage<MODE_FP64>(h, g, rk, ST_RHS, s);
    }
    double* out_dev = host_out ? h->user.as<double>() : dtheta;
    k_scatter_perm<<<nb, 256, 0, s>>>(h->n, h->perm.as<int32_t>(), h->fbuf.as<double>(), out_dev);
    KCHECK(h, cudaGetLastError(), "launching the right-hand side");
    if (host_out) {
        KCHECK(h, cudaMemcpyAsync(dtheta, out_dev, size_t(h->n) * 8, cudaMemcpyDeviceToHost, s), "copy out");
        return read_flags(h);
    }
    return KURA_OK;
}

static kura_status batch_rk4_steps(kura_t h, double* theta, double step, int64_t n_steps);

kura_status kura_rk4_steps(kura_t h, double* theta, double step, int64_t n_steps)
{
    if (check_handle(h)) return KURA_EINVAL;
    if (!theta) return h->fail(KURA_EINVAL, "theta is NULL");
    if (!(step > 0) || !std::isfinite(step)) return h->fail(KURA_EINVAL, "step must be positive and finite");
    if (n_steps < 0) return h->fail(KURA_EINVAL, "n_steps must be >= 0");
    if (h->batch) return batch_rk4_steps(h, theta, step, n_steps);
    if (h->ens) return ens_rk4_steps(h, theta, step, n_steps);
    const double* th_dev;
    bool host;
    if (kura_status st = stage_in(h, theta, &th_dev, &host)) return st;
    double* io = host ? h->user.as<double>() : theta;
    cudaStream_t s = h->stream;
    const unsigned nb = blocks_for(h->n, 256);
    k_gather_perm<<<nb, 256, 0, s>>>(h->n, h->perm.as<int32_t>(), io, h->y.as<double>());
    KCHECK(h, cudaGetLastError(), "launching the permutation");
    const int64_t chunk_max = 8;
    int64_t left = n_steps;
    if (h->small && !h->timing && n_steps > 0) {
        // small graph: every step in one launch of one thread-block cluster
        if (kura_status st = launch_small(h, step, n_steps, s)) return st;
        left = 0;
    }
    while (left > 0) {
        const int64_t c = std::min(left, chunk_max);
        auto key = std::make_pair(step, c * (h->timing ? -1 : 1));
        auto it = h->graphs.find(key);
        if (it == h->graphs.end()) {
            std::unique_ptr<GraphEntry> ge(new GraphEntry());
            if (h->timing) {
                ge->events.resize(size_t(8 * c));
                for (auto& e : ge->events) KCHECK(h, cudaEventCreate(&e), "cudaEventCreate");
            }
            cudaGraph_t graph = nullptr;
            KCHECK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
            if (h->ens) {
                for (int64_t k = 0; k < c; k++) enqueue_ens_step(h, step, h->cap);
            } else {
                enqueue_rk4_steps(h, step, c, h->cap, h->timing ? ge->events.data() : nullptr);
            }
            cudaError_t ec = cudaStreamEndCapture(h->cap, &graph);
            if (ec != cudaSuccess) return h->cuda_fail(ec, "end capture");
            ec = cudaGraphInstantiate(&ge->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ec != cudaSuccess) return h->cuda_fail(ec, "instantiate graph");
            it = h->graphs.emplace(key, std::move(ge)).first;
        }
        KCHECK(h, cudaGraphLaunch(it->second->exec, s), "graph launch");
        h->last_graph = it->second.get();
        left -= c;
    }
    k_scatter_perm<<<nb, 256, 0, s>>>(h->n, h->perm.as<int32_t>(), h->y.as<double>(), io);
    KCHECK(h, cudaGetLastError(), "launching the permutation");
    if (host) {
        KCHECK(h, cudaMemcpyAsync(theta, io, size_t(h->n) * 8, cudaMemcpyDeviceToHost, s), "copy out");
        return read_flags(h);
    }
    return KURA_OK;
}

kura_status kura_potential(kura_t h, const double* theta, double* V)
{
    if (kura_status st0 = check_single(h)) return st0;
    if (h->valued) return h->fail(KURA_ESTATE, "the potential is defined here for 0/1 matrices");
    if (!theta || !V) return h->fail(KURA_EINVAL, "NULL argument");
    const int64_t n = h->n;
    const int64_t nb = (n + DIAG_THREADS - 1) / DIAG_THREADS;
    if (!h->deg.p) {
        // degree plus 1 where the row's own diagonal block is dense: its block sums then include the
        // don't-care self term, which adds cos 0 = 1 to the row's cosine sum (and sin 0 = 0 elsewhere)
        const Plan& p = h->plan;
        std::vector<int32_t> degx(static_cast<size_t>(n));
        for (int64_t v = 0; v < n; v++) {
            const int32_t I = p.node_comm[size_t(v)];
            const bool self = std::binary_search(p.dcol.begin() + p.dptr[size_t(I)], p.dcol.begin() + p.dptr[size_t(I) + 1], I);
            degx[size_t(v)] = p.deg[size_t(v)] + (self ? 1 : 0);
        }
        KCHECK(h, upload(h->deg, degx, h->stream), "upload degrees");
        KCHECK(h, cudaStreamSynchronize(h->stream), "upload degrees");
    }
    if (!h->sums.p) KCHECK(h, h->sums.alloc(size_t(n) * 16), "alloc row sums");
    if (h->diag.bytes < size_t(nb + 1) * 8) KCHECK(h, h->diag.alloc(size_t(nb + 1) * 8), "alloc partials");
    const double* th_dev;
    bool host;
    if (kura_status st = stage_in(h, theta, &th_dev, &host)) return st;
    cudaStream_t s = h->stream;
    const DevGraph g = dev_graph(h);
    RkArgs rk = rk_args(h, 0.0);
    rk.sums_out = h->sums.as<double2>();
    k_gather_perm<<<blocks_for(n, 256), 256, 0, s>>>(n, h->perm.as<int32_t>(), th_dev, h->Y.as<double>());
    if (h->opts.precision == KURA_PREC_MIXED) {
        launch_trig<MODE_MIXED>(h, g, h->Y.as<double>(), TB_TABLE | TB_T, s);
        launch_row_stage<MODE_MIXED>(h, g, rk, ST_RHS, s);
    } else {
        launch_trig<MODE_FP64>(h, g, h->Y.as<double>(), TB_TABLE | TB_T, s);
        launch_row_stage<MODE_FP64>(h, g, rk, ST_RHS, s);
    }
    double* part = h->diag.as<double>();
    k_potential_terms<<<unsigned(nb), DIAG_THREADS, 0, s>>>(g, h->Y.as<double>(), h->sums.as<double2>(),
                                                             h->deg.as<int32_t>(), h->K, part);
    k_sum_partials<<<1, DIAG_THREADS, 0, s>>>(part, nb, part + nb);
    KCHECK(h, cudaGetLastError(), "launching the potential");
    KCHECK(h, cudaMemcpyAsync(V, part + nb, 8, cudaMemcpyDeviceToHost, s), "copy V");
    return read_flags(h);
}

kura_status kura_mean_deviation(kura_t h, const double* theta_t, const double* theta_0, double t, double* out)
{
    if (kura_status st0 = check_single(h)) return st0;
    if (!theta_t || !theta_0 || !out || !std::isfinite(t)) return h->fail(KURA_EINVAL, "NULL argument or non-finite t");
    const int64_t n = h->n;
    const int64_t nb = (n + DIAG_THREADS - 1) / DIAG_THREADS;
    if (h->diag.bytes < size_t(nb + 1) * 8) KCHECK(h, h->diag.alloc(size_t(nb + 1) * 8), "alloc partials");
    cudaStream_t s = h->stream;
    const DevGraph g = dev_graph(h);
    const double* dev;
    bool host;
    // theta_t -> Y, theta_0 -> krk (permuted); both staged through the user buffer when on the host
    if (kura_status st = stage_in(h, theta_t, &dev, &host)) return st;
    k_gather_perm<<<blocks_for(n, 256), 256, 0, s>>>(n, h->perm.as<int32_t>(), dev, h->Y.as<double>());
    if (kura_status st = stage_in(h, theta_0, &dev, &host)) return st;
    k_gather_perm<<<blocks_for(n, 256), 256, 0, s>>>(n, h->perm.as<int32_t>(), dev, h->krk.as<double>());
    double* part = h->diag.as<double>();
    k_meandev_terms<<<unsigned(nb), DIAG_THREADS, 0, s>>>(g, h->Y.as<double>(), h->krk.as<double>(), t, part);
    k_sum_partials<<<1, DIAG_THREADS, 0, s>>>(part, nb, part + nb);
    KCHECK(h, cudaGetLastError(), "launching the mean deviation");
    double v = 0.0;
    KCHECK(h, cudaMemcpyAsync(&v, part + nb, 8, cudaMemcpyDeviceToHost, s), "copy result");
    if (kura_status st = read_flags(h)) return st;
    *out = v / double(n);
    return KURA_OK;
}

kura_status kura_order_params(kura_t h, const double* theta, double* r, double* psi, double* r_comm,
                              double* psi_comm)
{
    if (kura_status st0 = check_single(h)) return st0;
    if (!theta || !r || !psi) return h->fail(KURA_EINVAL, "NULL argument");
    const double* th_dev;
    bool host;
    if (kura_status st = stage_in(h, theta, &th_dev, &host)) return st;
    cudaStream_t s = h->stream;
    const unsigned nb = blocks_for(h->n, 256);
    k_gather_perm<<<nb, 256, 0, s>>>(h->n, h->perm.as<int32_t>(), th_dev, h->Y.as<double>());
    const DevGraph g = dev_graph(h);
    // order parameters always in FP64 (FP64 sin/cos, exact fixed-point sums)
    launch_trig<MODE_FP64>(h, g, h->Y.as<double>(), 0, s);
    k_order_finalize<<<blocks_for(std::max(h->n_comm, 1), 256), 256, 0, s>>>(
        h->n_comm, h->n, h->bsum_out.as<long long>(), h->tot.as<long long>(), h->comm_off.as<int64_t>(),
        std::ldexp(1.0, -h->q_bits), h->order_out.as<double>());
    KCHECK(h, cudaGetLastError(), "launching the order parameters");
    std::vector<double> res(size_t(2 + 2 * h->n_comm));
    KCHECK(h, cudaMemcpyAsync(res.data(), h->order_out.p, res.size() * 8, cudaMemcpyDeviceToHost, s), "copy out");
    kura_status st = read_flags(h);
    if (st) return st;
    *r = res[0];
    *psi = res[1];
    for (int32_t I = 0; I < h->n_comm; I++) {
        if (r_comm) r_comm[I] = res[size_t(2 + 2 * I)];
        if (psi_comm) psi_comm[I] = res[size_t(3 + 2 * I)];
    }
    return KURA_OK;
}

kura_status kura_set_param(kura_t h, const double* omega, const double* K)
{
    if (kura_status st0 = check_single(h)) return st0;
    if (K) {
        if (!std::isfinite(*K)) return h->fail(KURA_EINVAL, "K is not finite");
        h->K = *K;
        if (h->opts.scaling == KURA_SCALING_DEGREE) {
            std::vector<double> rs(size_t(h->n));
            for (int64_t v = 0; v < h->n; v++)
                rs[size_t(v)] = h->plan.deg[size_t(v)] > 0 ? h->K / h->plan.deg[size_t(v)] : 0.0;
            KCHECK(h, cudaMemcpyAsync(h->rscale.p, rs.data(), rs.size() * 8, cudaMemcpyHostToDevice, h->stream),
                   "upload rscale");
            KCHECK(h, cudaStreamSynchronize(h->stream), "synchronise");
        }
        h->graphs.clear();   // K / N is a kernel argument baked into the graphs
        h->last_graph = nullptr;
    }
    if (omega) {
        const double* om_dev;
        bool host;
        if (kura_status st = stage_in(h, omega, &om_dev, &host)) return st;
        if (host) {
            for (int64_t i = 0; i < h->n; i++)
                if (!std::isfinite(omega[i])) return h->fail(KURA_EINVAL, "omega has a non-finite entry");
            h->h_omega.assign(omega, omega + h->n);
        }
        k_gather_perm<<<blocks_for(h->n, 256), 256, 0, h->stream>>>(h->n, h->perm.as<int32_t>(), om_dev,
                                                                       h->omega.as<double>());
        KCHECK(h, cudaGetLastError(), "launching the permutation");
        if (h->d_omega_user.p)
            KCHECK(h, cudaMemcpyAsync(h->d_omega_user.p, om_dev, size_t(h->n) * 8, cudaMemcpyDeviceToDevice,
                                      h->stream), "update omega");
        if (host) KCHECK(h, cudaStreamSynchronize(h->stream), "synchronise");
    }
    return KURA_OK;
}

static kura_status ensure_direct(kura_t h)
{
    if (h->d_col.p) return KURA_OK;
    if (h->h_col.empty() && h->nnz > 0)
        return h->fail(KURA_ESTATE, "the direct baseline needs the host CSR copy (keep_host_csr = 1)");
    KCHECK(h, upload(h->d_row_ptr, h->h_row_ptr, h->stream), "upload row_ptr");
    KCHECK(h, upload(h->d_col, h->h_col, h->stream), "upload col");
    KCHECK(h, upload(h->d_omega_user, h->h_omega, h->stream), "upload omega");
    KCHECK(h, h->red.alloc(4 * size_t(h->n)), "alloc reduced phases");
    KCHECK(h, cudaStreamSynchronize(h->stream), "synchronise");
    return KURA_OK;
}

static void launch_direct(kura_t h, const double* th_user, double* out_user, int32_t precision, cudaStream_t s)
{
    const int deg = h->opts.scaling == KURA_SCALING_DEGREE;
    const unsigned nbw = unsigned((h->n * 32 + 255) / 256);
    if (precision == KURA_PREC_MIXED) {
        k_reduce_phase<<<blocks_for(h->n, 256), 256, 0, s>>>(h->n, th_user, h->red.as<float>());
        k_direct_fp32<<<nbw, 256, 0, s>>>(h->n, h->d_row_ptr.as<int64_t>(), h->d_col.as<int32_t>(),
                                           h->d_omega_user.as<double>(), h->red.as<float>(), h->K, deg, out_user);
    } else {
        k_direct_fp64<<<nbw, 256, 0, s>>>(h->n, h->d_row_ptr.as<int64_t>(), h->d_col.as<int32_t>(),
                                           h->d_omega_user.as<double>(), th_user, h->K, deg, out_user);
    }
}

kura_status kura_direct_rhs(kura_t h, const double* theta, double* dtheta, int32_t precision)
{
    if (kura_status st0 = check_single(h)) return st0;
    if (h->valued) return h->fail(KURA_ESTATE, "the direct baseline sums 0/1 matrices");
    if (!theta || !dtheta || theta == dtheta) return h->fail(KURA_EINVAL, "theta/dtheta NULL or aliased");
    if (precision != KURA_PREC_FP64 && precision != KURA_PREC_MIXED) return h->fail(KURA_EINVAL, "bad precision");
    if (kura_status st = ensure_direct(h)) return st;
    const double* th_dev;
    bool host;
    if (kura_status st = stage_in(h, theta, &th_dev, &host)) return st;
    const bool host_out = !is_device_ptr(dtheta);
    double* out = host_out ? h->fbuf.as<double>() : dtheta;
    launch_direct(h, th_dev, out, precision, h->stream);
    KCHECK(h, cudaGetLastError(), "launching the direct baseline");
    if (host_out) {
        KCHECK(h, cudaMemcpyAsync(dtheta, out, size_t(h->n) * 8, cudaMemcpyDeviceToHost, h->stream), "copy out");
        KCHECK(h, cudaStreamSynchronize(h->stream), "synchronise");
    }
    return KURA_OK;
}

kura_status kura_direct_rk4_steps(kura_t h, double* theta, double step, int64_t n_steps, int32_t precision)
{
    if (kura_status st0 = check_single(h)) return st0;
    if (h->valued) return h->fail(KURA_ESTATE, "the direct baseline sums 0/1 matrices");
    if (!theta) return h->fail(KURA_EINVAL, "theta is NULL");
    if (!(step > 0) || !std::isfinite(step) || n_steps < 0) return h->fail(KURA_EINVAL, "bad step or n_steps");
    if (precision != KURA_PREC_FP64 && precision != KURA_PREC_MIXED) return h->fail(KURA_EINVAL, "bad precision");
    if (kura_status st = ensure_direct(h)) return st;
    const double* th_dev;
    bool host;
    if (kura_status st = stage_in(h, theta, &th_dev, &host)) return st;
    double* io = host ? h->user.as<double>() : theta;
    cudaStream_t s = h->stream;
    const unsigned nb = blocks_for(h->n, 256);
    // the direct path works in user order: y = io
    RkArgs rk{};
    rk.y = io;
    rk.y_out = io;
    rk.Y = h->Y.as<double>();
    rk.krk = h->krk.as<double>();
    rk.h = step;
    double* f = h->fbuf.as<double>();
    for (int64_t k = 0; k < n_steps; k++) {
        launch_direct(h, io, f, precision, s);
        k_rk4_update<ST_1><<<nb, 256, 0, s>>>(h->n, f, rk);
        launch_direct(h, h->Y.as<double>(), f, precision, s);
        k_rk4_update<ST_2><<<nb, 256, 0, s>>>(h->n, f, rk);
        launch_direct(h, h->Y.as<double>(), f, precision, s);
        k_rk4_update<ST_3><<<nb, 256, 0, s>>>(h->n, f, rk);
        launch_direct(h, h->Y.as<double>(), f, precision, s);
        k_rk4_update<ST_4><<<nb, 256, 0, s>>>(h->n, f, rk);
    }
    KCHECK(h, cudaGetLastError(), "launching the direct baseline");
    if (host) {
        KCHECK(h, cudaMemcpyAsync(theta, io, size_t(h->n) * 8, cudaMemcpyDeviceToHost, s), "copy out");
        KCHECK(h, cudaStreamSynchronize(s), "synchronise");
    }
    return KURA_OK;
}

// ---------------------------------------------------------------- adjoint
static bool csr_symmetric(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& col)
{
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 1024) reduction(|:bad)
    for (int64_t i = 0; i < n; i++) {
        for (int64_t e = rp[size_t(i)]; e < rp[size_t(i) + 1] && !bad; e++) {
            const int64_t j = col[size_t(e)];
            if (j == i) continue;
            if (!std::binary_search(col.begin() + rp[size_t(j)], col.begin() + rp[size_t(j) + 1], int32_t(i))) bad = 1;
        }
    }
    return !bad;
}

// RK4 steps on the permuted state y through the cached graphs (no boundary permutation).
static kura_status run_steps_perm(kura_t h, double step, int64_t n_steps)
{
    const int64_t chunk_max = 8;
    int64_t left = n_steps;
    while (left > 0) {
        const int64_t c = std::min(left, chunk_max);
        auto key = std::make_pair(step, c * (h->timing ? -1 : 1));
        auto it = h->graphs.find(key);
        if (it == h->graphs.end()) {
            std::unique_ptr<GraphEntry> ge(new GraphEntry());
            if (h->timing) {
                ge->events.resize(size_t(8 * c));
                for (auto& e : ge->events) KCHECK(h, cudaEventCreate(&e), "cudaEventCreate");
            }
            cudaGraph_t graph = nullptr;
            KCHECK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
            if (h->ens) {
                for (int64_t k = 0; k < c; k++) enqueue_ens_step(h, step, h->cap);
            } else {
                enqueue_rk4_steps(h, step, c, h->cap, h->timing ? ge->events.data() : nullptr);
            }
            cudaError_t ec = cudaStreamEndCapture(h->cap, &graph);
            if (ec != cudaSuccess) return h->cuda_fail(ec, "end capture");
            ec = cudaGraphInstantiate(&ge->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ec != cudaSuccess) return h->cuda_fail(ec, "instantiate graph");
            it = h->graphs.emplace(key, std::move(ge)).first;
        }
        KCHECK(h, cudaGraphLaunch(it->second->exec, h->stream), "graph launch");
        h->last_graph = it->second.get();
        left -= c;
    }
    return KURA_OK;
}

kura_status kura_integrate(kura_t h, double* theta, double step, int64_t n_steps, int32_t method, int32_t iters)
{
    if (method == KURA_INT_RK4) return kura_rk4_steps(h, theta, step, n_steps);
    if (kura_status st0 = check_single(h)) return st0;
    if (!theta) return h->fail(KURA_EINVAL, "theta is NULL");
    if (!(step > 0) || !std::isfinite(step)) return h->fail(KURA_EINVAL, "step must be positive and finite");
    if (n_steps < 0) return h->fail(KURA_EINVAL, "n_steps must be >= 0");
    if (method != KURA_INT_RK2 && method != KURA_INT_IMPLICIT_MIDPOINT) return h->fail(KURA_EINVAL, "unknown method");
    if (method == KURA_INT_IMPLICIT_MIDPOINT && (iters < 1 || iters > 64)) return h->fail(KURA_EINVAL, "iters in 1..64");
    if (method == KURA_INT_RK2) iters = 0;
    const double* th_dev;
    bool host;
    if (kura_status st = stage_in(h, theta, &th_dev, &host)) return st;
    double* io = host ? h->user.as<double>() : theta;
    cudaStream_t s = h->stream;
    const unsigned nb = blocks_for(h->n, 256);
    k_gather_perm<<<nb, 256, 0, s>>>(h->n, h->perm.as<int32_t>(), io, h->y.as<double>());
    KCHECK(h, cudaGetLastError(), "launching the permutation");
    const int64_t chunk_max = 8;
    int64_t left = n_steps;
    while (left > 0) {
        const int64_t c = std::min(left, chunk_max);
        // cache key: step size and (method, iters, chunk) in one integer, disjoint from the RK4 keys
        auto key = std::make_pair(step, int64_t(1) << 40 | int64_t(method) << 32 | int64_t(iters) << 16 | c);
        auto it = h->graphs.find(key);
        if (it == h->graphs.end()) {
            std::unique_ptr<GraphEntry> ge(new GraphEntry());
            cudaGraph_t graph = nullptr;
            KCHECK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
            for (int64_t k = 0; k < c; k++) enqueue_rk2_step(h, step, method, iters, h->cap);
            cudaError_t ec = cudaStreamEndCapture(h->cap, &graph);
            if (ec != cudaSuccess) return h->cuda_fail(ec, "end capture");
            ec = cudaGraphInstantiate(&ge->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ec != cudaSuccess) return h->cuda_fail(ec, "instantiate graph");
            it = h->graphs.emplace(key, std::move(ge)).first;
        }
        KCHECK(h, cudaGraphLaunch(it->second->exec, s), "graph launch");
        left -= c;
    }
    k_scatter_perm<<<nb, 256, 0, s>>>(h->n, h->perm.as<int32_t>(), h->y.as<double>(), io);
    KCHECK(h, cudaGetLastError(), "launching the permutation");
    if (host) {
        KCHECK(h, cudaMemcpyAsync(theta, io, size_t(h->n) * 8, cudaMemcpyDeviceToHost, s), "copy out");
        return read_flags(h);
    }
    return KURA_OK;
}

// ---------------------------------------------------------------- ensembles sharing one graph
// theta: n_traj x n (trajectory-major, user order), host or device
static kura_status ens_stage_in(kura_t h, const double* src, const double** dev, bool* host)
{
    EnsData& e = *h->ens;
    const size_t bytes = size_t(e.groups) * ENS_B * size_t(h->n) * 8;
    *host = !is_device_ptr(src);
    if (*host) {
        KCHECK(h, cudaMemcpyAsync(e.user.p, src, bytes, cudaMemcpyHostToDevice, h->stream), "copy in");
        *dev = e.user.as<double>();
    } else {
        *dev = src;
    }
    return KURA_OK;
}

static kura_status ens_rhs(kura_t h, const double* theta, double* dtheta)
{
    if (!theta || !dtheta || theta == dtheta) return h->fail(KURA_EINVAL, "theta/dtheta NULL or aliased");
    EnsData& e = *h->ens;
    const double* th;
    bool host_in;
    if (kura_status st = ens_stage_in(h, theta, &th, &host_in)) return st;
    const bool host_out = !is_device_ptr(dtheta);
    cudaStream_t s = h->stream;
    const int64_t tot = int64_t(e.groups) * ENS_B * h->n;
    const unsigned nb = blocks_for(tot, 256);
    k_ens_gather<<<nb, 256, 0, s>>>(h->n, e.groups, h->perm.as<int32_t>(), th, e.Y.as<double>());
    const EnsArgs a = ens_args(h);
    const RkArgs rk = ens_rk_args(h, 0.0);
    enqueue_ens_stage(h, a, rk.Y, rk, ST_RHS, s);
    double* out = host_out ? e.user.as<double>() : dtheta;
    k_ens_scatter<<<nb, 256, 0, s>>>(h->n, e.groups, h->perm.as<int32_t>(), e.f.as<double>(), out);
    KCHECK(h, cudaGetLastError(), "launching the ensemble right-hand side");
    if (host_out) {
        KCHECK(h, cudaMemcpyAsync(dtheta, out, size_t(tot) * 8, cudaMemcpyDeviceToHost, s), "copy out");
        return read_flags(h);
    }
    return KURA_OK;
}

static kura_status run_steps_perm(kura_t h, double step, int64_t n_steps);

static kura_status ens_rk4_steps(kura_t h, double* theta, double step, int64_t n_steps)
{
    EnsData& e = *h->ens;
    const double* th;
    bool host;
    if (kura_status st = ens_stage_in(h, theta, &th, &host)) return st;
    double* io = host ? e.user.as<double>() : theta;
    cudaStream_t s = h->stream;
    const int64_t tot = int64_t(e.groups) * ENS_B * h->n;
    const unsigned nb = blocks_for(tot, 256);
    k_ens_gather<<<nb, 256, 0, s>>>(h->n, e.groups, h->perm.as<int32_t>(), io, e.y.as<double>());
    KCHECK(h, cudaGetLastError(), "launching the permutation");
    if (kura_status st = run_steps_perm(h, step, n_steps)) return st;
    k_ens_scatter<<<nb, 256, 0, s>>>(h->n, e.groups, h->perm.as<int32_t>(), e.y.as<double>(), io);
    KCHECK(h, cudaGetLastError(), "launching the permutation");
    if (host) {
        KCHECK(h, cudaMemcpyAsync(theta, io, size_t(tot) * 8, cudaMemcpyDeviceToHost, s), "copy out");
        return read_flags(h);
    }
    return KURA_OK;
}

kura_status kura_ensemble_create(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* label,
                                 int32_t n_comm, int32_t n_traj, const double* omega, const double* K,
                                 const kura_opts* opts, void* stream, kura_t* out)
{
    g_create_error.clear();
    if (!out) { g_create_error = "out is NULL"; return KURA_EINVAL; }
    *out = nullptr;
    kura_opts o;
    kura_default_opts(&o);
    if (opts) o = *opts;
    if (n_traj <= 0 || n_traj % ENS_B) { g_create_error = "n_traj must be a positive multiple of 16"; return KURA_EINVAL; }
    if (o.scaling != KURA_SCALING_UNIFORM) { g_create_error = "ensembles use uniform scaling"; return KURA_EINVAL; }
    if (!omega || !K) { g_create_error = "omega or K is NULL"; return KURA_EINVAL; }
    for (int64_t q = 0; q < int64_t(n_traj) * n; q++)
        if (!std::isfinite(omega[q])) { g_create_error = "omega has a non-finite entry"; return KURA_EINVAL; }
    for (int32_t b = 0; b < n_traj; b++)
        if (!std::isfinite(K[b])) { g_create_error = "K has a non-finite entry"; return KURA_EINVAL; }
    PlanInput in;
    in.n_sms = current_sm_count();
    in.n = n; in.row_ptr = row_ptr; in.col = col; in.label = label; in.n_comm = n_comm; in.tau = o.tau;
    in.tile_max_rows = TC_MBLOCK;                  // one M-block per CTA
    in.tile_max_sub = tile_max_sub_for(MODE_MIXED);
    in.slot_ints = slot_ints_for(MODE_MIXED);
    in.tensor_cores = o.tensor_cores > 0 ? 2 : 0;  // the mask product serves every trajectory of a group
    Plan plan;
    std::string err;
    int rc = build_plan(in, plan, err);
    if (rc) { g_create_error = err; return rc == 2 ? KURA_ENOMEM : KURA_EINVAL; }
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        g_create_error = std::string("no usable CUDA device: ") + cudaGetErrorString(ce);
        return KURA_ECUDA;
    }
    std::unique_ptr<kura_ctx> h(new (std::nothrow) kura_ctx());
    if (!h) { g_create_error = "out of host memory"; return KURA_ENOMEM; }
    cudaGetDevice(&h->device);
    o.precision = KURA_PREC_MIXED;
    h->opts = o;
    h->n = n;
    h->n_comm = n_comm;
    h->stream = static_cast<cudaStream_t>(stream);
    h->nnz = row_ptr[n];
    h->ens.reset(new EnsData());
    EnsData& e = *h->ens;
    e.groups = n_traj / ENS_B;
    auto fail = [&](cudaError_t c, const char* what) {
        g_create_error = std::string(what) + ": " + cudaGetErrorString(c);
        return c == cudaErrorMemoryAllocation ? KURA_ENOMEM : KURA_ECUDA;
    };
#define ECHECK(call, what) do { cudaError_t c_ = (call); if (c_ != cudaSuccess) return fail(c_, what); } while (0)
    ECHECK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaStream_t s = h->stream;
    const Plan& p = plan;
    ECHECK(upload(h->perm, p.perm, s), "upload perm");
    ECHECK(upload(e.node_comm, p.node_comm, s), "upload node_comm");
    ECHECK(upload(e.comm_off, p.comm_off, s), "upload comm_off");
    ECHECK(upload(e.dptr, p.dptr, s), "upload dptr");
    ECHECK(upload(e.dcol, p.dcol, s), "upload dcol");
    ECHECK(upload(e.tiles, p.tiles, s), "upload tiles");
    {
        // per row, its listed entries in one run: present as the column, missing as ~column
        std::vector<int64_t> lptr(size_t(n) + 1, 0);
        std::vector<int32_t> lidx;
        lidx.reserve(size_t(p.miss_total + p.pres_total));
        for (int64_t v = 0; v < n; v++) {
            for (int32_t sg = p.row_sub0[size_t(v)]; sg < p.row_sub0[size_t(v) + 1]; sg++) {
                const int32_t* hdr = p.gstream.data() + p.sub_hdr[size_t(sg)];
                for (int32_t k = 0; k < hdr[1]; k++) lidx.push_back(~p.gstream[size_t(p.sub_mpos[size_t(sg)] + k)]);
                for (int32_t k = 0; k < hdr[3]; k++) lidx.push_back(p.gstream[size_t(p.sub_ppos[size_t(sg)] + k)]);
            }
            lptr[size_t(v) + 1] = int64_t(lidx.size());
        }
        ECHECK(upload(e.lptr, lptr, s), "upload listed-entry offsets");
        ECHECK(upload(e.lidx, lidx, s), "upload listed entries");
    }
    ECHECK(upload(e.bitmap, p.bitmap, s), "upload masks");
    {
        // the masks as BF16 operand tiles (128 rows x 64 columns, swizzled), expanded once
        const int64_t n_blocks = int64_t(p.bitmap.size()) / (TC_MBLOCK * 4);
        ECHECK(e.aimage.alloc(std::max<size_t>(size_t(n_blocks) * 2 * ENS_ABYTES, 16)), "alloc mask images");
        if (n_blocks > 0)
            k_ens_expand_masks<<<blocks_for(n_blocks * 2 * TC_MBLOCK, 256), 256, 0, s>>>(e.bitmap.as<uint32_t>(), n_blocks,
                                                                                      e.aimage.as<uint8_t>());
        ECHECK(cudaGetLastError(), "expanding the masks");
    }
    const size_t G = size_t(e.groups), N = size_t(n), B = ENS_B;
    {
        std::vector<double> om(G * N * B), sc(G * B);
        for (size_t g = 0; g < G; g++)
            for (size_t i = 0; i < N; i++)
                for (size_t b = 0; b < B; b++)
                    om[(g * N + i) * B + b] = omega[(g * B + b) * N + size_t(p.perm[i])];
        for (size_t q = 0; q < G * B; q++) sc[q] = K[q] / double(n);
        ECHECK(upload(e.omega, om, s), "upload omega");
        ECHECK(upload(e.scale, sc, s), "upload K");
    }
    e.nblk64 = 2 * ((int64_t(n) + TC_KBLOCK - 1) / TC_KBLOCK);
    ECHECK(e.table.alloc(G * (N + 2) * B * sizeof(float2)), "alloc table");
    ECHECK(cudaMemsetAsync(e.table.p, 0, e.table.bytes, s), "memset table");
    ECHECK(e.image.alloc(G * size_t(e.nblk64) * ENS_BBYTES), "alloc image");
    ECHECK(cudaMemsetAsync(e.image.p, 0, e.image.bytes, s), "memset image");
    ECHECK(e.bsum.alloc(G * size_t(n_comm) * B * 16), "alloc block sums");
    ECHECK(e.T.alloc(G * size_t(n_comm) * B * 16), "alloc T");
    for (DevMem* d : {&e.y, &e.Y, &e.krk, &e.f, &e.user}) ECHECK(d->alloc(G * N * B * 8), "alloc state");
    ECHECK(h->err_flags.alloc(16), "alloc error flags");
    ECHECK(cudaMemsetAsync(h->err_flags.p, 0, 16, s), "memset error flags");
    const void* fns[] = {(const void*)k_ens_row<ST_RHS>, (const void*)k_ens_row<ST_1>, (const void*)k_ens_row<ST_2>,
                         (const void*)k_ens_row<ST_3>, (const void*)k_ens_row<ST_4>};
    for (const void* fn : fns) ECHECK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ENS_SMEM),
                                      "setting the ensemble kernel's shared-memory size");
    ECHECK(cudaStreamSynchronize(s), "upload");
#undef ECHECK
    h->n_tiles = int32_t(p.tiles.size());
    h->miss_total = p.miss_total;
    h->pres_total = p.pres_total;
    h->tc_tiles = p.tc_tiles;
    h->tc_rows = p.tc_rows;
    h->tc_mask_bits = p.tc_mask_bits;
    h->has_tc = p.tc_tiles > 0;
    h->stream_bytes = plan_stream_bytes(p);
    h->q_bits = 61 - ceil_log2(std::max<int64_t>(n, 2));
    h->plan = std::move(plan);
    std::vector<int32_t>().swap(h->plan.gstream);
    std::vector<uint32_t>().swap(h->plan.bitmap);
    *out = h.release();
    return KURA_OK;
}

kura_status kura_adjoint(kura_t h, const double* theta0, double step, int64_t n_steps, int32_t ckpt_every,
                         int32_t loss_kind, const double* target, double* loss, double* g_omega, double* g_K,
                         double* g_theta0)
{
    if (kura_status st0 = check_single(h)) return st0;
    if (!theta0 || !loss || !g_omega || !g_K || !g_theta0) return h->fail(KURA_EINVAL, "NULL argument");
    if (!(step > 0) || !std::isfinite(step) || n_steps < 1 || ckpt_every < 1)
        return h->fail(KURA_EINVAL, "step > 0, n_steps >= 1 and ckpt_every >= 1 are required");
    if (loss_kind != 0 && loss_kind != 1) return h->fail(KURA_EINVAL, "loss_kind must be 0 or 1");
    if (loss_kind == 1 && !target) return h->fail(KURA_EINVAL, "loss_kind 1 needs a target");
    if (h->opts.precision != KURA_PREC_MIXED)
        return h->fail(KURA_ESTATE, "the adjoint runs on handles created with KURA_PREC_MIXED");
    if (h->valued) return h->fail(KURA_ESTATE, "the adjoint runs on 0/1 matrices");
    if (h->sym < 0) {
        if (h->h_col.empty() && h->nnz > 0)
            return h->fail(KURA_ESTATE, "the adjoint needs the host CSR copy to check symmetry");
        h->sym = csr_symmetric(h->n, h->h_row_ptr, h->h_col) ? 1 : 0;
    }
    if (!h->sym && !h->tr) {
        // directed A: the nu-weighted sums of J^T w run over A^T, planned from the transposed host CSR with
        // the same labels (hence the same permutation and communities) and the handle's options
        if (h->h_col.empty() && h->nnz > 0)
            return h->fail(KURA_ESTATE, "the adjoint of a directed A needs the host CSR copy");
        const int64_t nn = h->n;
        std::vector<int64_t> rpT(size_t(nn) + 1, 0);
        for (int64_t v = 0; v < nn; v++)
            for (int64_t e = h->h_row_ptr[size_t(v)]; e < h->h_row_ptr[size_t(v) + 1]; e++) rpT[size_t(h->h_col[size_t(e)]) + 1]++;
        for (int64_t v = 0; v < nn; v++) rpT[size_t(v) + 1] += rpT[size_t(v)];
        std::vector<int32_t> colT(static_cast<size_t>(rpT[size_t(nn)]));
        std::vector<int64_t> fill(rpT.begin(), rpT.end() - 1);
        for (int64_t v = 0; v < nn; v++)            // rows of A^T come out sorted: v increases
            for (int64_t e = h->h_row_ptr[size_t(v)]; e < h->h_row_ptr[size_t(v) + 1]; e++)
                colT[size_t(fill[size_t(h->h_col[size_t(e)])]++)] = int32_t(v);
        kura_opts o = h->opts;
        o.keep_host_csr = 0;
        kura_t t = nullptr;
        const kura_status st = kura_create(nn, rpT.data(), colT.empty() ? nullptr : colT.data(), h->h_label.data(),
                                           h->n_comm, h->h_omega.data(), h->K, &o, h->stream, &t);
        if (st) return h->fail(st, "plan of the transposed matrix: %s", kura_last_error(nullptr));
        h->tr.reset(t);
        cudaSetDevice(h->device);
    }
    kura_ctx* ah = h->tr ? h->tr.get() : h;           // the plan the nu-weighted pass runs on
    cudaStream_t s = h->stream;
    if (h->ad_stream && h->ad_ev[0]) {
        // a previous call that failed midway may have left recompute work on the second stream: this
        // call's work on the handle's stream comes after it
        KCHECK(h, cudaEventRecord(h->ad_ev[0], h->ad_stream), "order after the recompute stream");
        KCHECK(h, cudaStreamWaitEvent(s, h->ad_ev[0], 0), "order after the recompute stream");
    }
    const size_t n = size_t(h->n), N8 = 8 * n;
    const int64_t M = ckpt_every;
    const int64_t nck = (n_steps + M - 1) / M;
    // buffers
    if (h->ad_M != M || h->ad_nck < nck || !h->ad_lam.p) {
        KCHECK(h, h->ad_ck.alloc(N8 * size_t(nck)), "alloc checkpoints");
        for (DevMem* d : {&h->ad_Y, &h->ad_Y2}) KCHECK(h, d->alloc(N8 * size_t(4 * M + 1)), "alloc stage inputs");
        for (DevMem* d : {&h->ad_F, &h->ad_F2}) KCHECK(h, d->alloc(16 * n * size_t(4 * M)), "alloc stage sums");
        KCHECK(h, h->ad_table.alloc(8 * (n + 2)), "alloc the nu-weighted table");
        KCHECK(h, cudaMemsetAsync(h->ad_table.p, 0, h->ad_table.bytes, s), "zero the nu-weighted table");
        for (DevMem* d : {&h->ad_lam, &h->ad_asum, &h->ad_a0, &h->ad_a1, &h->ad_w, &h->ad_nu, &h->ad_gom, &h->ad_tgt,
                          &h->ad_scratch})
            KCHECK(h, d->alloc(N8), "alloc adjoint vectors");
        KCHECK(h, h->ad_sc.alloc(8 * n), "alloc sc");
        KCHECK(h, h->ad_bs.alloc(16 * size_t(h->n_comm)), "alloc block sums");
        KCHECK(h, h->ad_part.alloc(8 * ((n + 255) / 256)), "alloc loss partials");
        KCHECK(h, h->ad_absmax.alloc(16), "alloc table maximum");        // [0] max |entry|, [2] ticket
        KCHECK(h, cudaMemsetAsync(h->ad_absmax.p, 0, 16, s), "zero the table maximum and the ticket");
        // chunks of at most 256 nodes of one community each, communities in order (the stage kernel's CTAs)
        {
            std::vector<int4> chunks;
            std::vector<int32_t> cptr(size_t(h->n_comm) + 1, 0);
            for (int32_t J = 0; J < h->n_comm; J++) {
                cptr[size_t(J)] = int32_t(chunks.size());
                for (int64_t b = h->plan.comm_off[size_t(J)]; b < h->plan.comm_off[size_t(J) + 1]; b += 256)
                    chunks.push_back(make_int4(J, int(b), int(std::min<int64_t>(b + 256, h->plan.comm_off[size_t(J) + 1])), 0));
            }
            cptr[size_t(h->n_comm)] = int32_t(chunks.size());
            if (chunks.empty()) chunks.push_back(make_int4(0, 0, 0, 0));         // n = 0 cannot happen; keep a CTA
            h->ad_nchunks = int32_t(chunks.size());
            KCHECK(h, upload(h->ad_chunks, chunks, s), "upload adjoint chunks");
            KCHECK(h, upload(h->ad_chunk_ptr, cptr, s), "upload adjoint chunk pointers");
            KCHECK(h, h->ad_cpart.alloc(16 * chunks.size()), "alloc chunk sums");
        }
        h->ad_M = M;
        h->ad_nck = nck;
        h->graphs.clear();                 // captured segments point at the old buffers
        h->last_graph = nullptr;
    }
    // the dK accumulators follow the tiles of the nu-weighted pass's plan, which kura_autotune or
    // kura_classify_blocks may have rebuilt since the last call; so does the need for digits of the
    // nu-weighted table (tensor-core tiles of A's own plan; A^T's plan has a digit image of its own)
    if (h->ad_gk.bytes < 8 * size_t(std::max(ah->n_tiles, 1))) {
        KCHECK(h, h->ad_gk.alloc(8 * size_t(std::max(ah->n_tiles, 1))), "alloc dK accumulators");
        h->graphs.clear();
        h->last_graph = nullptr;
    }
    if (!h->tr && h->has_tc && h->ad_dig.bytes < h->dig.bytes) {
        KCHECK(h, h->ad_dig.alloc(h->dig.bytes), "alloc the nu-weighted digit image");
        KCHECK(h, cudaMemsetAsync(h->ad_dig.p, 0, h->ad_dig.bytes, s), "zero the nu-weighted digit image");
        h->graphs.clear();
        h->last_graph = nullptr;
    }
    double* ck = h->ad_ck.as<double>();
    // two sets of stage inputs (slot 4 t + (s - 1), plus one spare) and forward row sums per (t, s)
    double* Ysets[2] = {h->ad_Y.as<double>(), h->ad_Y2.as<double>()};
    double2* Fsets[2] = {h->ad_F.as<double2>(), h->ad_F2.as<double2>()};
    const unsigned nb = blocks_for(h->n, 256);
    const DevGraph g = dev_graph(h);

    // ---- forward with checkpoints (permuted state y)
    const double* th_dev;
    bool host;
    if (kura_status st = stage_in(h, theta0, &th_dev, &host)) return st;
    k_gather_perm<<<nb, 256, 0, s>>>(h->n, h->perm.as<int32_t>(), th_dev, h->y.as<double>());
    if (loss_kind == 1) {
        const double* tg_dev;
        bool th;
        if (kura_status st = stage_in(h, target, &tg_dev, &th)) return st;
        k_gather_perm<<<nb, 256, 0, s>>>(h->n, h->perm.as<int32_t>(), tg_dev, h->ad_tgt.as<double>());
    }
    KCHECK(h, cudaGetLastError(), "launching the permutation");
    auto seg_len = [&](int64_t c) { return std::min(M, n_steps - c * M); };
    // with the fused trig the backward runs two streams (below), and the forward keeps the stage inputs
    // and row sums of its last segment, which then needs no recompute
    const bool pipe = h->opts.fused_trig != 0;
    // one segment of L steps from the state in Ysets[set] slot 0: integrate it, keeping every stage input
    // and the forward row sums; the last step's new state goes to y_last
    auto enqueue_recompute = [&](int64_t L, int set, double* y_last, cudaStream_t q) {
        double* Ybuf = Ysets[set];
        double2* Fbuf = Fsets[set];
        const bool fused = h->opts.fused_trig != 0;
        if (fused) enqueue_fused_start(h, Ybuf, q);
        for (int64_t t = 0; t < L; t++) {
            for (int st = ST_1; st <= ST_4; st++) {
                RkArgs rk{};
                rk.y = Ybuf + size_t(4 * t) * n;
                rk.Y = Ybuf + size_t(4 * t + st) * n;                         // next stage input
                rk.y_out = (t + 1 < L) ? Ybuf + size_t(4 * (t + 1)) * n : y_last;
                rk.krk = h->krk.as<double>();
                rk.sums_out = Fbuf + size_t(4 * t + st - 1) * n;
                rk.h = step;
                DevGraph gs = g;
                if (fused) fused_stage_args(h, st, gs, rk);
                else launch_trig<MODE_MIXED>(h, g, Ybuf + size_t(4 * t + st - 1) * n, TB_TABLE | TB_T, q);
                launch_row_stage<MODE_MIXED>(h, gs, rk, st, q);
            }
        }
    };
    // half 0: recompute a segment (its new state is not needed); 1: its adjoint steps; 2: the forward's
    // last segment, kept for the backward (its new state is theta(T)).  Full segments are captured once
    // per (half, set) as CUDA graphs, keyed apart from the forward step graphs.
    std::function<void(int64_t, int, cudaStream_t)> enqueue_adjoint;
    auto enqueue_half = [&](int half, int64_t L, int set, cudaStream_t q) {
        if (half == 1) enqueue_adjoint(L, set, q);
        else enqueue_recompute(L, set, half == 2 ? h->y.as<double>() : h->ad_scratch.as<double>(), q);
    };
    auto run_half = [&](int half, int64_t L, int set, cudaStream_t q) -> kura_status {
        if (!(L == M && nck > 2)) {
            enqueue_half(half, L, set, q);
            return KURA_OK;
        }
        const std::pair<double, int64_t> key{step, -(int64_t(1) << 41) - 8 * M - 3 * set - half};
        auto it = h->graphs.find(key);
        if (it == h->graphs.end()) {
            std::unique_ptr<GraphEntry> ge(new GraphEntry());
            cudaGraph_t graph = nullptr;
            KCHECK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
            enqueue_half(half, L, set, h->cap);
            cudaError_t ec = cudaStreamEndCapture(h->cap, &graph);
            if (ec != cudaSuccess) return h->cuda_fail(ec, "end capture of an adjoint segment");
            ec = cudaGraphInstantiate(&ge->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ec != cudaSuccess) return h->cuda_fail(ec, "instantiate an adjoint segment");
            it = h->graphs.emplace(key, std::move(ge)).first;
        }
        KCHECK(h, cudaGraphLaunch(it->second->exec, q), "adjoint segment launch");
        return KURA_OK;
    };
    for (int64_t c = 0; c < nck; c++) {
        if (pipe && c == nck - 1) {
            const int set = int(c % 2);
            KCHECK(h, cudaMemcpyAsync(Ysets[set], h->y.p, N8, cudaMemcpyDeviceToDevice, s), "last segment's start");
            if (kura_status st = run_half(2, seg_len(c), set, s)) return st;
            KCHECK(h, cudaGetLastError(), "launching the last forward segment");
            break;
        }
        KCHECK(h, cudaMemcpyAsync(ck + size_t(c) * n, h->y.p, N8, cudaMemcpyDeviceToDevice, s), "checkpoint");
        if (kura_status st = run_steps_perm(h, step, seg_len(c))) return st;
    }
    // ---- terminal loss and lambda
    double* lam = h->ad_lam.as<double>();
    double* yT = h->y.as<double>();
    if (loss_kind == 0) {
        launch_trig<MODE_FP64>(h, g, yT, 0, s);   // exact block sums of FP64 sin/cos of theta(T)
        k_order_finalize<<<blocks_for(std::max(h->n_comm, 1), 256), 256, 0, s>>>(
            h->n_comm, h->n, h->bsum_out.as<long long>(), h->tot.as<long long>(), h->comm_off.as<int64_t>(),
            std::ldexp(1.0, -h->q_bits), h->order_out.as<double>());
        k_adj_terminal_r<<<nb, 256, 0, s>>>(h->n, yT, h->order_out.as<double>(), lam);
    } else {
        k_adj_terminal_misfit<<<nb, 256, 0, s>>>(h->n, yT, h->ad_tgt.as<double>(), lam, h->ad_part.as<double>());
    }
    KCHECK(h, cudaMemsetAsync(h->ad_gom.p, 0, N8, s), "zero g_omega");
    KCHECK(h, cudaMemsetAsync(h->ad_gk.p, 0, h->ad_gk.bytes, s), "zero dK accumulators");
    KCHECK(h, cudaGetLastError(), "launching the terminal adjoint");

    // ---- backward, segment by segment
    const double cl[5] = {0, step / 6.0, step / 3.0, step / 3.0, step / 6.0};
    const double ca[5] = {0, 0.5 * step, 0.5 * step, step, 0.0};
    unsigned int* absmax = ah->has_tc ? h->ad_absmax.as<unsigned int>() : nullptr;
    unsigned int* ticket = h->ad_absmax.as<unsigned int>() + 2;
    // graph of the nu-weighted pass: A's own, or A^T's plan reading A's T, scalings and error word; the
    // nu-weighted table (and A's digits of it) are the adjoint's own buffers, so that the recompute of
    // another segment, which uses the handle's tables, may run at the same time
    DevGraph ga = g;
    if (h->tr) {
        ga = dev_graph(h->tr.get());
        ga.T = g.T;
        ga.scale = g.scale;
        ga.rscale = g.rscale;
        ga.rinvdeg = g.rinvdeg;
        ga.inv_n = g.inv_n;
        ga.err = g.err;
    } else if (absmax) {
        ga.dig = h->ad_dig.as<uint8_t>();
    }
    ga.table = h->ad_table.p;
    // a segment's adjoint steps, last to first
    enqueue_adjoint = [&](int64_t L, int set, cudaStream_t q) {
        double* Ybuf = Ysets[set];
        double2* Fbuf = Fsets[set];
        for (int64_t t = L - 1; t >= 0; t--) {
            for (int st = 4; st >= 1; st--) {
                double* a_next = (st < 4) ? ((st % 2 == 1) ? h->ad_a0.as<double>() : h->ad_a1.as<double>()) : nullptr;
                double* a_out = (st % 2 == 0) ? h->ad_a0.as<double>() : h->ad_a1.as<double>();
                if (absmax) cudaMemsetAsync(absmax, 0, sizeof(unsigned int), q);
                k_adj_prep_bsum<<<unsigned(h->ad_nchunks), 256, 0, q>>>(
                    ga, h->ad_chunks.as<int4>(), h->ad_chunk_ptr.as<int32_t>(), Ybuf + size_t(4 * t + st - 1) * n, lam,
                    a_next, cl[st], ca[st], h->ad_w.as<double>(), h->ad_nu.as<double>(), h->ad_sc.as<float2>(),
                    h->ad_gom.as<double>(), absmax, h->ad_cpart.as<double2>(), h->ad_bs.as<double2>(), ticket);
                if (absmax) k_adj_digits<<<nb, 256, 0, q>>>(ga, absmax);
                AdjArgs adj{};
                adj.fsums = Fbuf + size_t(4 * t + st - 1) * n;
                adj.sc = h->ad_sc.as<float2>();
                adj.nu = h->ad_nu.as<double>();
                adj.w = h->ad_w.as<double>();
                adj.a_out = a_out;
                adj.asum = h->ad_asum.as<double>();
                adj.lam = lam;
                adj.gk_acc = h->ad_gk.as<double>();
                adj.absmax = absmax;
                adj.stage = st;
                RkArgs rk{};
                launch_row<MODE_MIXED, ST_ADJ>(ah, ga, rk, q, adj);
            }
        }
    };
    if (!pipe) {
        // a trig launch per recompute stage writes the handle's T and block-sum counter, which the adjoint
        // stages use too: one segment after the other on the handle's stream
        for (int64_t c = nck - 1; c >= 0; c--) {
            KCHECK(h, cudaMemcpyAsync(Ysets[0], ck + size_t(c) * n, N8, cudaMemcpyDeviceToDevice, s), "restore checkpoint");
            if (kura_status st = run_half(0, seg_len(c), 0, s)) return st;
            if (kura_status st = run_half(1, seg_len(c), 0, s)) return st;
            KCHECK(h, cudaGetLastError(), "launching the adjoint");
        }
    } else {
        // segment c's adjoint stages run on the handle's stream while segment c - 1 is recomputed on a
        // second stream into the other set of stage buffers: the two share no buffer but read-only ones.
        // Events: recomputing into a set waits for the end of the adjoint that last read it; an adjoint
        // waits for its segment's recompute.
        if (!h->ad_stream) KCHECK(h, cudaStreamCreateWithFlags(&h->ad_stream, cudaStreamNonBlocking), "adjoint stream");
        for (cudaEvent_t& e : h->ad_ev)
            if (!e) KCHECK(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "adjoint events");
        cudaStream_t r = h->ad_stream;
        cudaEvent_t ev_start = h->ad_ev[0], *rec_done = h->ad_ev + 1, *adj_done = h->ad_ev + 3;
        KCHECK(h, cudaEventRecord(ev_start, s), "record the backward start");
        KCHECK(h, cudaStreamWaitEvent(r, ev_start, 0), "order the recompute stream");
        auto recompute = [&](int64_t c) -> kura_status {
            const int set = int(c % 2);
            KCHECK(h, cudaMemcpyAsync(Ysets[set], ck + size_t(c) * n, N8, cudaMemcpyDeviceToDevice, r),
                   "restore checkpoint");
            if (kura_status st = run_half(0, seg_len(c), set, r)) return st;
            KCHECK(h, cudaEventRecord(rec_done[set], r), "record a recompute");
            return KURA_OK;
        };
        // the last segment's stage buffers come from the forward pass, on this stream
        for (int64_t c = nck - 1; c >= 0; c--) {
            const int set = int(c % 2);
            if (c >= 1) {
                // set (c - 1) mod 2 was last read by the adjoint of segment c + 1
                if (c + 1 <= nck - 1) KCHECK(h, cudaStreamWaitEvent(r, adj_done[(c - 1) % 2], 0), "order a recompute");
                if (kura_status st = recompute(c - 1)) return st;
            }
            if (c < nck - 1) KCHECK(h, cudaStreamWaitEvent(s, rec_done[set], 0), "order an adjoint segment");
            if (kura_status st = run_half(1, seg_len(c), set, s)) return st;
            KCHECK(h, cudaEventRecord(adj_done[set], s), "record an adjoint segment");
            KCHECK(h, cudaGetLastError(), "launching the adjoint");
        }
    }
    // ---- outputs
    double* gth_dev = host ? h->user.as<double>() : g_theta0;
    k_scatter_perm<<<nb, 256, 0, s>>>(h->n, h->perm.as<int32_t>(), lam, gth_dev);
    const bool gom_host = !is_device_ptr(g_omega);
    double* gom_dev = gom_host ? h->fbuf.as<double>() : g_omega;
    k_scatter_perm<<<nb, 256, 0, s>>>(h->n, h->perm.as<int32_t>(), h->ad_gom.as<double>(), gom_dev);
    KCHECK(h, cudaGetLastError(), "launching the permutation");
    std::vector<double> gk(size_t(std::max(ah->n_tiles, 1)));
    KCHECK(h, cudaMemcpyAsync(gk.data(), h->ad_gk.p, gk.size() * 8, cudaMemcpyDeviceToHost, s), "copy dK");
    double Lval = 0.0;
    std::vector<double> part;
    if (loss_kind == 0) {
        KCHECK(h, cudaMemcpyAsync(&Lval, h->order_out.p, 8, cudaMemcpyDeviceToHost, s), "copy r");
    } else {
        part.resize((n + 255) / 256);
        KCHECK(h, cudaMemcpyAsync(part.data(), h->ad_part.p, part.size() * 8, cudaMemcpyDeviceToHost, s), "copy loss");
    }
    if (host && g_theta0 != gth_dev)
        KCHECK(h, cudaMemcpyAsync(g_theta0, gth_dev, N8, cudaMemcpyDeviceToHost, s), "copy g_theta0");
    if (gom_host) KCHECK(h, cudaMemcpyAsync(g_omega, gom_dev, N8, cudaMemcpyDeviceToHost, s), "copy g_omega");
    kura_status st = read_flags(h);
    if (st) return st;
    double gks = 0.0;
    for (double v : gk) gks += v;
    *g_K = gks;
    if (loss_kind == 0) {
        *loss = 1.0 - Lval;
    } else {
        double lsum = 0.0;
        for (double v : part) lsum += v;
        *loss = lsum;
    }
    return KURA_OK;
}

// ---------------------------------------------------------------- batched ensembles
static size_t batch_smem_bytes(bool tc) { return size_t(BATCH_SMEM_BASE) + (tc ? size_t(BATCH_TC_SMEM) : 0); }

// One persistent launch over every trajectory: n_steps RK4 steps on theta in
// place, or (rhs_only) one right-hand side of theta written to out.
static kura_status batch_launch(kura_t h, const double* theta, double* out, double step, int64_t n_steps,
                                bool rhs_only)
{
    BatchData& B = *h->batch;
    const double* th_dev;
    bool host;
    if (kura_status st = stage_in(h, theta, &th_dev, &host)) return st;
    const bool host_out = rhs_only ? !is_device_ptr(out) : host;
    double* io = host_out ? h->user.as<double>() : out;
    cudaStream_t s = h->stream;
    const unsigned nb = blocks_for(h->n, 256);
    k_gather_perm<<<nb, 256, 0, s>>>(h->n, h->perm.as<int32_t>(), th_dev, h->y.as<double>());
    KCHECK(h, cudaMemsetAsync(B.queue.p, 0, 16, s), "reset the trajectory queue");
    BatchDev bd{};
    bd.traj = B.traj.as<BatchTraj>();
    bd.order = B.order.as<int32_t>();
    bd.n_traj = B.n_traj;
    bd.comm_off = B.comm_off.as<int32_t>();
    bd.dptr = B.dptr.as<int32_t>();
    bd.dcol = B.dcol.as<int32_t>();
    bd.node_comm = B.node_comm.as<uint16_t>();
    bd.row_off = B.row_off.as<int32_t>();
    bd.row_nm = B.row_nm.as<int32_t>();
    bd.entries = B.entries_d.as<uint16_t>();
    bd.tc_tiles = B.tc_tiles_d.as<BatchTcTile>();
    bd.tc_bits = B.tc_bits_d.as<uint32_t>();
    bd.omega = h->omega.as<double>();
    bd.y = h->y.as<double>();
    bd.Y = h->Y.as<double>();
    bd.krk = h->krk.as<double>();
    bd.stash = B.stash.p;
    bd.queue = B.queue.as<unsigned int>();
    bd.err = h->err_flags.as<int>();
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
    const bool tc = B.tc_tiles > 0;
    const size_t smem = batch_smem_bytes(tc);
    if (n_steps > 0) {
        if (h->timing) {
            if (!h->last_graph || h->last_graph->events.size() != 2) {
                h->graphs.clear();
                std::unique_ptr<GraphEntry> ge(new GraphEntry());
                ge->events.resize(2);
                for (auto& e : ge->events) KCHECK(h, cudaEventCreate(&e), "cudaEventCreate");
                h->last_graph = ge.get();
                h->graphs.emplace(std::make_pair(0.0, int64_t(0)), std::move(ge));
            }
            cudaEventRecord(h->last_graph->events[0], s);
        }
        const unsigned grid = unsigned(std::min(std::max(nsm, 1), B.n_traj));
        const int ro = rhs_only ? 1 : 0;
        if (h->opts.precision == KURA_PREC_FP64)
            k_batch_rk4<MODE_FP64, false><<<grid, BATCH_THREADS, smem, s>>>(bd, step, n_steps, ro);
        else if (tc)
            k_batch_rk4<MODE_MIXED, true><<<grid, BATCH_THREADS, smem, s>>>(bd, step, n_steps, ro);
        else
            k_batch_rk4<MODE_MIXED, false><<<grid, BATCH_THREADS, smem, s>>>(bd, step, n_steps, ro);
        if (h->timing) cudaEventRecord(h->last_graph->events[1], s);
    }
    k_scatter_perm<<<nb, 256, 0, s>>>(h->n, h->perm.as<int32_t>(), rhs_only ? h->krk.as<double>() : h->y.as<double>(),
                                      io);
    KCHECK(h, cudaGetLastError(), "launching the batched integrator");
    if (host_out) {
        KCHECK(h, cudaMemcpyAsync(out, io, size_t(h->n) * 8, cudaMemcpyDeviceToHost, s), "copy out");
        return read_flags(h);
    }
    return KURA_OK;
}

static kura_status batch_rk4_steps(kura_t h, double* theta, double step, int64_t n_steps)
{
    return batch_launch(h, theta, theta, step, n_steps, false);
}

// Checks trajectory t of a batch and plans it with choice c: a complete graph
// (NULL row_ptr) is one dense community with nothing stored, anything else
// goes through the planner with tiles of one 128-row M-block.
static kura_status plan_batch_traj(const kura_graph_desc& gd, int32_t t, const BatchChoice& c, bool fp64, Plan& p,
                                   std::string& err)
{
    const int64_t max_n = fp64 ? BATCH_MAX_N_FP64 : BATCH_MAX_N;
    if (gd.n < 1 || gd.n > max_n || gd.n_comm < 1 || gd.n_comm > BATCH_MAX_COMM || !gd.omega || !std::isfinite(gd.K)) {
        err = "trajectory " + std::to_string(t) + ": need 1 <= n <= " + std::to_string(max_n) +
              ", 1 <= n_comm <= " + std::to_string(BATCH_MAX_COMM) + ", omega and finite K";
        return KURA_EINVAL;
    }
    if (gd.row_ptr == nullptr) {
        if (gd.n_comm != 1) { err = "a complete-graph trajectory has n_comm = 1"; return KURA_EINVAL; }
        p.n = gd.n;
        p.n_comm = 1;
        p.perm.resize(size_t(gd.n));
        for (int64_t v = 0; v < gd.n; v++) p.perm[size_t(v)] = int32_t(v);
        p.comm_off = {0, gd.n};
        p.node_comm.assign(size_t(gd.n), 0);
        p.dptr = {0, 1};
        p.dcol = {0};
        p.row_sub0.assign(size_t(gd.n) + 1, 0);      // no sub-rows: no stored corrections
        return KURA_OK;
    }
    PlanInput in;
    in.n_sms = current_sm_count();
    in.n = gd.n; in.row_ptr = gd.row_ptr; in.col = gd.col; in.label = gd.label; in.n_comm = gd.n_comm;
    in.tau = c.tau;
    in.tile_max_rows = TC_MBLOCK;     // a tensor-core tile is one 128-row M-block
    in.tile_max_sub = tile_max_sub_for(MODE_MIXED);
    in.slot_ints = slot_ints_for(MODE_MIXED);
    in.tensor_cores = fp64 ? 0 : c.tc;
    std::string perr;
    const int rc = build_plan(in, p, perr);
    if (rc) { err = "trajectory " + std::to_string(t) + ": " + perr; return rc == 2 ? KURA_ENOMEM : KURA_EINVAL; }
    return KURA_OK;
}

// The work-queue cost of a planned batch trajectory: per-node work, its listed
// entries, and about 600 entries' worth per 64-column operand block of the
// tensor-core tiles (expansion, barriers and MMA issue).
static double batch_traj_cost(const Plan& p)
{
    int64_t listed = 0;
    for (size_t sg = 0; sg < p.sub_hdr.size(); sg++) {
        const int32_t* hdr = p.gstream.data() + p.sub_hdr[sg];
        listed += hdr[1] + hdr[3];
    }
    double tc_cost = 0.0;
    for (const Tile& tl : p.tiles)
        if (tl.flags & TILE_TC) tc_cost += 1200.0 * double(tl.nsw);
    return double(p.n) * 24.0 + double(listed) + tc_cost;
}

// (Re)builds the device data of batch handle h for the trajectories gds with
// the per-trajectory plan choices ch (h->device, h->stream and h->opts set).
static kura_status batch_build(kura_ctx* h, const std::vector<kura_graph_desc>& gds,
                               const std::vector<BatchChoice>& ch, std::string& err)
{
    const int32_t n_traj = int32_t(gds.size());
    const bool fp64 = h->opts.precision == KURA_PREC_FP64;
    h->batch.reset(new BatchData());
    BatchData& B = *h->batch;
    B.n_traj = n_traj;
    B.choice = ch;
    std::vector<BatchTraj> traj(static_cast<size_t>(n_traj));
    std::vector<int32_t> comm_off, dptr, dcol, row_off, row_nm, perm_g;
    std::vector<uint16_t> node_comm, entries;
    std::vector<BatchTcTile> tc_tiles;
    std::vector<uint32_t> tc_bits;
    std::vector<double> om;
    std::vector<double> cost(static_cast<size_t>(n_traj));
    const kura_graph_desc* graphs = gds.data();
    int64_t node_off = 0;
    for (int32_t t = 0; t < n_traj; t++) {
        const kura_graph_desc& gd = graphs[size_t(t)];
        Plan p;
        if (kura_status st = plan_batch_traj(gd, t, ch[size_t(t)], fp64, p, err)) return st;
        BatchTraj& tr = traj[size_t(t)];
        tr.tc0 = int32_t(tc_tiles.size());
        for (const Tile& tl : p.tiles) {
            if (!(tl.flags & TILE_TC)) continue;
            BatchTcTile bt{};
            bt.r0 = tl.r0;
            bt.nrows = tl.r1 - tl.r0;
            bt.wbeg = tl.wbeg;
            bt.nkb = tl.nsw;
            bt.bits_off = int64_t(tc_bits.size());
            const int64_t words = int64_t(tl.nsw) * TC_MBLOCK * 4;     // one M-block per tile
            tc_bits.insert(tc_bits.end(), p.bitmap.begin() + tl.bm_off, p.bitmap.begin() + tl.bm_off + words);
            tc_tiles.push_back(bt);
            B.tc_mask_bits += int64_t(tl.nsw) * TC_MBLOCK * TC_KBLOCK;
        }
        tr.tc1 = int32_t(tc_tiles.size());
        if (tr.tc1 > tr.tc0) B.tc_traj++;
        tr.node_off = node_off;
        tr.entry_off = int64_t(entries.size());
        tr.n = int32_t(gd.n);
        tr.n_comm = gd.n_comm;
        tr.comm_base = int32_t(comm_off.size());
        tr.dense_base = int32_t(dptr.size());
        tr.scale = gd.K / double(gd.n);
        int k = 0;
        while ((int64_t(1) << k) < std::max<int64_t>(gd.n, 2)) k++;
        tr.q_bits = 61 - k;
        tr.row_lanes = ch[size_t(t)].lanes;
        for (int64_t v : p.comm_off) comm_off.push_back(int32_t(v));
        const int32_t dbase = int32_t(dcol.size());
        for (int64_t v : p.dptr) dptr.push_back(int32_t(v) + dbase);
        for (int32_t v : p.dcol) dcol.push_back(v);
        for (int64_t v = 0; v < gd.n; v++) {
            node_comm.push_back(uint16_t(p.node_comm[size_t(v)]));
            perm_g.push_back(int32_t(node_off + p.perm[size_t(v)]));
            om.push_back(gd.omega[p.perm[size_t(v)]]);
        }
        // per row: [missing | present] local indices
        int32_t pos = 0;
        for (int64_t v = 0; v < gd.n; v++) {
            row_off.push_back(pos);
            int32_t nm = 0;
            std::vector<int32_t> pres;
            for (int32_t sg = p.row_sub0[size_t(v)]; sg < p.row_sub0[size_t(v) + 1]; sg++) {
                const int32_t* hdr = p.gstream.data() + p.sub_hdr[size_t(sg)];
                for (int32_t q = 0; q < hdr[1]; q++) { entries.push_back(uint16_t(p.gstream[size_t(p.sub_mpos[size_t(sg)] + q)])); nm++; }
                for (int32_t q = 0; q < hdr[3]; q++) pres.push_back(p.gstream[size_t(p.sub_ppos[size_t(sg)] + q)]);
            }
            for (int32_t c : pres) entries.push_back(uint16_t(c));
            row_nm.push_back(nm);
            pos += nm + int32_t(pres.size());
            B.missing += nm;
            B.present += int64_t(pres.size());
        }
        row_off.push_back(pos);
        cost[size_t(t)] = batch_traj_cost(p);          // the LPT order of the work queue
        node_off += gd.n;
    }
    B.n_total = node_off;
    B.entries = int64_t(entries.size());
    std::vector<int32_t> order(static_cast<size_t>(n_traj));
    for (int32_t t = 0; t < n_traj; t++) order[size_t(t)] = t;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost[size_t(a)] > cost[size_t(b)]; });

    h->n = node_off;
    h->n_comm = 0;
    B.tc_tiles = int64_t(tc_tiles.size());
    const bool use_tc = B.tc_tiles > 0;
    const size_t smem = batch_smem_bytes(use_tc);
    cudaStream_t s = h->stream;
    kura_ctx* hc = h;
#define BCHECK(call, what)                                                              \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            err = std::string(what) + ": " + cudaGetErrorString(e_);                    \
            return e_ == cudaErrorMemoryAllocation ? KURA_ENOMEM : KURA_ECUDA;          \
        }                                                                               \
    } while (0)
    if (fp64)
        BCHECK(cudaFuncSetAttribute((const void*)k_batch_rk4<MODE_FP64, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)), "shared memory size");
    else if (use_tc)
        BCHECK(cudaFuncSetAttribute((const void*)k_batch_rk4<MODE_MIXED, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)), "shared memory size");
    else
        BCHECK(cudaFuncSetAttribute((const void*)k_batch_rk4<MODE_MIXED, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)), "shared memory size");
    BCHECK(upload(B.tc_tiles_d, tc_tiles, s), "upload tensor-core tiles");
    BCHECK(upload(B.tc_bits_d, tc_bits, s), "upload tensor-core masks");
    BCHECK(upload(B.traj, traj, s), "upload trajectories");
    BCHECK(upload(B.order, order, s), "upload order");
    BCHECK(upload(B.comm_off, comm_off, s), "upload community offsets");
    BCHECK(upload(B.dptr, dptr, s), "upload dense pointers");
    BCHECK(upload(B.dcol, dcol, s), "upload dense blocks");
    BCHECK(upload(B.node_comm, node_comm, s), "upload node communities");
    BCHECK(upload(B.row_off, row_off, s), "upload row offsets");
    BCHECK(upload(B.row_nm, row_nm, s), "upload row missing counts");
    BCHECK(upload(B.entries_d, entries, s), "upload corrections");
    BCHECK(upload(hc->omega, om, s), "upload omega");
    BCHECK(upload(hc->perm, perm_g, s), "upload permutation");
    BCHECK(B.queue.alloc(16), "alloc queue");
    BCHECK(B.stash.alloc((fp64 ? 16 : 8) * size_t(node_off)), "alloc stash");
    for (DevMem* d : {&hc->y, &hc->Y, &hc->krk, &hc->user}) BCHECK(d->alloc(8 * size_t(node_off)), "alloc state");
    if (!hc->err_flags.p) {
        BCHECK(hc->err_flags.alloc(16), "alloc error flags");
        BCHECK(cudaMemsetAsync(hc->err_flags.p, 0, 16, s), "memset error flags");
    }
    if (!hc->cap) BCHECK(cudaStreamCreateWithFlags(&hc->cap, cudaStreamNonBlocking), "stream");
    BCHECK(cudaStreamSynchronize(s), "upload");
#undef BCHECK
    return KURA_OK;
}


kura_status kura_batch_create(int32_t n_traj, const kura_graph_desc* graphs, const kura_opts* opts, void* stream,
                              kura_t* out)
{
    g_create_error.clear();
    if (!out) { g_create_error = "out is NULL"; return KURA_EINVAL; }
    *out = nullptr;
    if (n_traj <= 0 || !graphs) { g_create_error = "n_traj must be positive and graphs non-NULL"; return KURA_EINVAL; }
    kura_opts o;
    kura_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != KURA_PREC_MIXED && o.precision != KURA_PREC_FP64) {
        g_create_error = "unknown precision";
        return KURA_EINVAL;
    }
    if (o.scaling != KURA_SCALING_UNIFORM) { g_create_error = "batches use uniform scaling"; return KURA_EINVAL; }
    if (!(o.tau >= 0.0 && o.tau <= 1.0)) { g_create_error = "tau must be in [0, 1]"; return KURA_EINVAL; }
    if (o.row_lanes != 0 && o.row_lanes != 32 && o.row_lanes != 16 && o.row_lanes != 8) {
        g_create_error = "row_lanes must be 0, 32, 16 or 8";
        return KURA_EINVAL;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        g_create_error = std::string("no usable CUDA device: ") + cudaGetErrorString(e);
        return KURA_ECUDA;
    }
    std::unique_ptr<kura_ctx> h(new (std::nothrow) kura_ctx());
    if (!h) return KURA_ENOMEM;
    cudaGetDevice(&h->device);
    h->opts = o;
    h->stream = static_cast<cudaStream_t>(stream);
    std::vector<kura_graph_desc> gds(graphs, graphs + n_traj);
    BatchChoice c0;
    c0.tau = o.tau;
    // the mask product touches every entry of a dense block (the lists only its zeros): measured 15-17x
    // slower on the batch workload, so only tensor_cores = 2 asks for it; the autotuner may still pick it
    c0.tc = (o.precision == KURA_PREC_FP64 || o.tensor_cores != 2) ? 0 : 2;
    c0.lanes = o.row_lanes ? o.row_lanes : 32;
    std::vector<BatchChoice> ch(size_t(n_traj), c0);
    std::string err;
    kura_status st = batch_build(h.get(), gds, ch, err);
    if (st) { g_create_error = err; return st; }
    if (o.keep_host_csr) {
        // host copies for kura_autotune, which rebuilds the batch with other plan choices
        BatchData& B = *h->batch;
        B.host.resize(size_t(n_traj));
        for (int32_t t = 0; t < n_traj; t++) {
            const kura_graph_desc& gd = graphs[t];
            HostGraph& hg = B.host[size_t(t)];
            hg.desc = gd;
            hg.omega.assign(gd.omega, gd.omega + gd.n);
            if (gd.row_ptr) {
                hg.row_ptr.assign(gd.row_ptr, gd.row_ptr + gd.n + 1);
                hg.col.assign(gd.col, gd.col + gd.row_ptr[gd.n]);
                hg.label.assign(gd.label, gd.label + gd.n);
            }
            hg.rebind();
        }
    }
    *out = h.release();
    return KURA_OK;
}

// Milliseconds per RK4 step of batch handle h started from the device phases th0 (user order): one warm-up
// step, then the median of three timed runs of `steps` steps, each from a fresh copy of th0.
static kura_status batch_step_ms(kura_t h, const double* th0, int64_t steps, double* ms)
{
    DevMem th;
    KCHECK(h, th.alloc(size_t(h->n) * 8), "alloc tuning phases");
    cudaStream_t s = h->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    KCHECK(h, cudaEventCreate(&e0), "cudaEventCreate");
    KCHECK(h, cudaEventCreate(&e1), "cudaEventCreate");
    std::vector<float> t;
    kura_status st = KURA_OK;
    for (int r = 0; r < 4 && !st; r++) {
        if (cudaMemcpyAsync(th.p, th0, size_t(h->n) * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            st = h->fail(KURA_ECUDA, "copy tuning phases");
            break;
        }
        cudaEventRecord(e0, s);
        st = batch_launch(h, th.as<double>(), th.as<double>(), 0.01, r == 0 ? 1 : steps, false);
        cudaEventRecord(e1, s);
        if (!st && cudaEventSynchronize(e1) != cudaSuccess) st = h->fail(KURA_ECUDA, "tuning run");
        float v = 0.0f;
        cudaEventElapsedTime(&v, e0, e1);
        if (r > 0) t.push_back(v);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    std::sort(t.begin(), t.end());
    *ms = double(t[1]) / double(steps);
    return read_flags(h);
}

// The batch autotuner: trajectories with a stored graph are grouped by size class (ceil(log2 n)); per class,
// starting from the handle's choices, one parameter at a time is moved -- the encoding of the dense-block
// zeros (tensor-core mask or index lists; mixed precision), the row tile (lanes per row 32, 16, 8) and tau
// (0.35, 0.5, 0.65) -- each candidate timed on a sub-batch of that class (at most one trajectory per SM, one
// launch); the fastest choice is kept for the whole class and the handle is rebuilt with the choices.
static kura_status batch_autotune(kura_t h, const double* theta, double budget_s, kura_tune_result* out)
{
    BatchData& B = *h->batch;
    if (B.host.empty()) return h->fail(KURA_ESTATE, "the autotuner rebuilds batches from host copies (keep_host_csr = 1)");
    const auto t_start = std::chrono::steady_clock::now();
    auto elapsed = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count(); };
    std::memset(out, 0, sizeof *out);
    const int32_t n_traj = B.n_traj;
    // user-order phases of every trajectory on the host
    std::vector<double> th(size_t(h->n));
    if (is_device_ptr(theta)) {
        KCHECK(h, cudaMemcpyAsync(th.data(), theta, size_t(h->n) * 8, cudaMemcpyDeviceToHost, h->stream), "copy phases");
        KCHECK(h, cudaStreamSynchronize(h->stream), "copy phases");
    } else {
        std::memcpy(th.data(), theta, size_t(h->n) * 8);
    }
    std::vector<int64_t> off(size_t(n_traj) + 1, 0);
    for (int32_t t = 0; t < n_traj; t++) off[size_t(t) + 1] = off[size_t(t)] + B.host[size_t(t)].desc.n;
    DevMem th_all;
    KCHECK(h, th_all.alloc(size_t(h->n) * 8), "alloc phases");
    KCHECK(h, cudaMemcpyAsync(th_all.p, th.data(), size_t(h->n) * 8, cudaMemcpyHostToDevice, h->stream), "phases");
    double ms0 = 0.0;
    if (kura_status st = batch_step_ms(h, th_all.as<double>(), 3, &ms0)) return st;
    out->initial_rhs_ms = ms0;
    int32_t cand = 1;
    // size classes of the trajectories with a stored graph (complete graphs store nothing)
    std::map<int, std::vector<int32_t>> classes;
    for (int32_t t = 0; t < n_traj; t++) {
        const kura_graph_desc& gd = B.host[size_t(t)].desc;
        if (!gd.row_ptr) continue;
        int k = 0;
        while ((int64_t(1) << k) < gd.n) k++;
        classes[k].push_back(t);
    }
    std::vector<BatchChoice> ch = B.choice;
    const bool fp64 = h->opts.precision == KURA_PREC_FP64;
    const int nsm = current_sm_count();
    // heaviest classes first: sum of n^2 over the class
    std::vector<std::pair<double, int>> order;
    for (auto& kv : classes) {
        double w = 0.0;
        for (int32_t t : kv.second) w += double(B.host[size_t(t)].desc.n) * double(B.host[size_t(t)].desc.n);
        order.push_back({-w, kv.first});
    }
    std::sort(order.begin(), order.end());
    BatchChoice heaviest = ch.empty() ? BatchChoice() : ch[0];
    bool first_class = true;
    for (auto& ow : order) {
        if (elapsed() > budget_s) break;
        const std::vector<int32_t>& members = classes[ow.second];
        // the sub-batch: up to one trajectory per SM, evenly spaced over the class
        std::vector<int32_t> sub;
        const size_t m = members.size(), take = std::min<size_t>(m, size_t(std::max(nsm, 1)));
        for (size_t q = 0; q < take; q++) sub.push_back(members[q * m / take]);
        std::vector<kura_graph_desc> gds;
        std::vector<double> th_sub;
        for (int32_t t : sub) {
            gds.push_back(B.host[size_t(t)].desc);
            th_sub.insert(th_sub.end(), th.begin() + off[size_t(t)], th.begin() + off[size_t(t) + 1]);
        }
        auto time_choice = [&](const BatchChoice& c, double* ms) -> kura_status {
            std::unique_ptr<kura_ctx> tmp(new (std::nothrow) kura_ctx());
            if (!tmp) return h->fail(KURA_ENOMEM, "tuning handle");
            tmp->device = h->device;
            tmp->opts = h->opts;
            tmp->stream = h->stream;
            std::string err;
            std::vector<BatchChoice> cs(gds.size(), c);
            if (kura_status st = batch_build(tmp.get(), gds, cs, err)) return h->fail(st, "tuning build: %s", err.c_str());
            DevMem d;
            KCHECK(h, d.alloc(th_sub.size() * 8), "alloc tuning phases");
            KCHECK(h, cudaMemcpyAsync(d.p, th_sub.data(), th_sub.size() * 8, cudaMemcpyHostToDevice, h->stream), "phases");
            kura_status st = batch_step_ms(tmp.get(), d.as<double>(), 3, ms);
            if (st) return h->fail(st, "tuning run: %s", tmp->err.c_str());
            cand++;
            return KURA_OK;
        };
        BatchChoice best = ch[size_t(members[0])];
        double best_ms = 0.0;
        if (kura_status st = time_choice(best, &best_ms)) return st;
        auto try_c = [&](const BatchChoice& c) -> kura_status {
            if (elapsed() > budget_s) return KURA_OK;
            double ms = 0.0;
            if (kura_status st = time_choice(c, &ms)) return st;
            if (ms < best_ms) { best_ms = ms; best = c; }
            return KURA_OK;
        };
        if (!fp64) {
            const BatchChoice base = best;
            for (int32_t tc : {0, 2}) {
                if (tc == base.tc) continue;
                BatchChoice c = base;
                c.tc = tc;
                if (kura_status st = try_c(c)) return st;
            }
        }
        {
            const BatchChoice base = best;
            for (int32_t lanes : {32, 16, 8}) {
                if (lanes == base.lanes) continue;
                BatchChoice c = base;
                c.lanes = lanes;
                if (kura_status st = try_c(c)) return st;
            }
        }
        {
            const BatchChoice base = best;
            for (double tau : {0.35, 0.5, 0.65}) {
                if (tau == base.tau) continue;
                BatchChoice c = base;
                c.tau = tau;
                if (kura_status st = try_c(c)) return st;
            }
        }
        for (int32_t t : members) ch[size_t(t)] = best;
        if (first_class) heaviest = best;
        first_class = false;
    }
    // rebuild the handle with the chosen plans (keeping the host copies)
    std::vector<HostGraph> host = std::move(B.host);
    std::vector<kura_graph_desc> gds;
    for (auto& hg : host) gds.push_back(hg.desc);
    KCHECK(h, cudaStreamSynchronize(h->stream), "synchronise before re-planning");
    h->graphs.clear();
    h->last_graph = nullptr;
    std::string err;
    if (kura_status st = batch_build(h, gds, ch, err)) return h->fail(st, "%s", err.c_str());
    h->batch->host = std::move(host);
    double ms1 = 0.0;
    if (kura_status st = batch_step_ms(h, th_all.as<double>(), 3, &ms1)) return st;
    out->rhs_ms = ms1;
    out->tau = heaviest.tau;
    out->tensor_cores = heaviest.tc;
    out->tile_work = heaviest.lanes;
    out->candidates = cand;
    out->seconds = elapsed();
    return KURA_OK;
}

kura_status kura_batch_traj_params(kura_t h, int32_t t, double* tau, int32_t* tensor_cores, int32_t* row_lanes)
{
    if (check_handle(h)) return KURA_EINVAL;
    if (!h->batch) return h->fail(KURA_ESTATE, "not a batch handle");
    if (t < 0 || t >= h->batch->n_traj) return h->fail(KURA_EINVAL, "trajectory index out of range");
    const BatchChoice& c = h->batch->choice[size_t(t)];
    if (tau) *tau = c.tau;
    if (tensor_cores) *tensor_cores = c.tc;
    if (row_lanes) *row_lanes = c.lanes;
    return KURA_OK;
}

kura_status kura_batch_info(kura_t h, kura_batch_info_t* out)
{
    if (check_handle(h) || !out) return KURA_EINVAL;
    if (!h->batch) return h->fail(KURA_ESTATE, "not a batch handle");
    const BatchData& B = *h->batch;
    std::memset(out, 0, sizeof *out);
    out->n_traj = B.n_traj;
    out->precision = h->opts.precision;
    out->n_total = B.n_total;
    out->missing_listed = B.missing;
    out->present = B.present;
    out->tc_traj = B.tc_traj;
    out->tc_tiles = B.tc_tiles;
    out->tc_mask_bits = B.tc_mask_bits;
    return KURA_OK;
}

kura_status kura_batch_costs(int32_t n_traj, const kura_graph_desc* graphs, const kura_opts* opts, double* cost)
{
    g_create_error.clear();
    if (n_traj < 0 || (n_traj > 0 && (!graphs || !cost))) {
        g_create_error = "n_traj must be non-negative, graphs and cost non-NULL";
        return KURA_EINVAL;
    }
    kura_opts o;
    kura_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != KURA_PREC_MIXED && o.precision != KURA_PREC_FP64) {
        g_create_error = "unknown precision";
        return KURA_EINVAL;
    }
    if (!(o.tau >= 0.0 && o.tau <= 1.0)) { g_create_error = "tau must be in [0, 1]"; return KURA_EINVAL; }
    const bool fp64 = o.precision == KURA_PREC_FP64;
    BatchChoice c;                               // the choice kura_batch_create starts from
    c.tau = o.tau;
    c.tc = (fp64 || o.tensor_cores != 2) ? 0 : 2;
    for (int32_t t = 0; t < n_traj; t++) {
        Plan p;
        std::string err;
        if (kura_status st = plan_batch_traj(graphs[t], t, c, fp64, p, err)) { g_create_error = err; return st; }
        cost[t] = batch_traj_cost(p);
    }
    return KURA_OK;
}

kura_status kura_partition_lpt(const double* cost, int32_t n, int32_t n_parts, int32_t* part, double* load)
{
    g_create_error.clear();
    if (n < 0 || n_parts < 1 || (n > 0 && (!cost || !part))) {
        g_create_error = "need n >= 0, n_parts >= 1, cost and part non-NULL";
        return KURA_EINVAL;
    }
    for (int32_t i = 0; i < n; i++)
        if (!(cost[i] >= 0.0) || !std::isfinite(cost[i])) {
            g_create_error = "cost " + std::to_string(i) + " is negative or not finite";
            return KURA_EINVAL;
        }
    std::vector<int32_t> order(static_cast<size_t>(n));
    for (int32_t i = 0; i < n; i++) order[size_t(i)] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
    // least-loaded part first, lower part on equal loads
    using Slot = std::pair<double, int32_t>;
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
    for (int32_t q = 0; q < n_parts; q++) heap.push(Slot(0.0, q));
    std::vector<double> acc(static_cast<size_t>(n_parts), 0.0);
    for (int32_t i : order) {
        const Slot s = heap.top();
        heap.pop();
        part[i] = s.second;
        acc[size_t(s.second)] = s.first + cost[i];
        heap.push(Slot(acc[size_t(s.second)], s.second));
    }
    if (load)
        for (int32_t q = 0; q < n_parts; q++) load[q] = acc[size_t(q)];
    return KURA_OK;
}

kura_status kura_batch_stats(kura_t h, int64_t* n_total, int64_t* missing, int64_t* present)
{
    if (check_handle(h)) return KURA_EINVAL;
    if (!h->batch) return h->fail(KURA_ESTATE, "not a batch handle");
    if (n_total) *n_total = h->batch->n_total;
    if (missing) *missing = h->batch->missing;
    if (present) *present = h->batch->present;
    return KURA_OK;
}

kura_status kura_set_timing(kura_t h, int32_t on)
{
    if (check_handle(h)) return KURA_EINVAL;
    h->timing = on != 0;
    return KURA_OK;
}

kura_status kura_kernel_times(kura_t h, float* ms, int32_t cap, int32_t* count)
{
    if (check_handle(h) || !count) return KURA_EINVAL;
    *count = 0;
    if (!h->last_graph || h->last_graph->events.empty()) return KURA_OK;
    KCHECK(h, cudaStreamSynchronize(h->stream), "synchronise");
    const auto& ev = h->last_graph->events;
    const int32_t avail = int32_t(ev.size() / 2);
    for (int32_t k = 0; k < avail && k < cap && ms; k++)
        KCHECK(h, cudaEventElapsedTime(&ms[k], ev[size_t(2 * k)], ev[size_t(2 * k + 1)]), "event time");
    *count = avail;
    return KURA_OK;
}

void kura_destroy(kura_t h) { delete h; }

// ---------------------------------------------------------------- host-only plan
struct kura_plan_s {
    Plan p;
};

static kura_status plan_build_impl(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* val,
                                   const int32_t* label, int32_t n_comm, const kura_opts* opts, kura_plan_t* out);

kura_status kura_plan_build(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* label,
                            int32_t n_comm, const kura_opts* opts, kura_plan_t* out)
{
    return plan_build_impl(n, row_ptr, col, nullptr, label, n_comm, opts, out);
}

kura_status kura_plan_build_valued(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* val,
                                   const int32_t* label, int32_t n_comm, const kura_opts* opts, kura_plan_t* out)
{
    if (!val) return KURA_EINVAL;
    return plan_build_impl(n, row_ptr, col, val, label, n_comm, opts, out);
}

kura_status kura_plan_dense_values(kura_plan_t pl, int32_t I, int32_t* v, int32_t cap, int32_t* count)
{
    if (!pl || !count || I < 0 || I >= pl->p.n_comm) return KURA_EINVAL;
    const Plan& p = pl->p;
    *count = int32_t(p.dptr[size_t(I) + 1] - p.dptr[size_t(I)]);
    for (int32_t k = 0; k < *count && k < cap && v; k++) v[k] = p.dval[size_t(p.dptr[size_t(I)] + k)];
    return KURA_OK;
}

static kura_status plan_build_impl(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* val,
                                   const int32_t* label, int32_t n_comm, const kura_opts* opts, kura_plan_t* out)
{
    g_create_error.clear();
    if (!out) return KURA_EINVAL;
    *out = nullptr;
    kura_opts o;
    kura_default_opts(&o);
    if (opts) o = *opts;
    std::unique_ptr<kura_plan_s> p(new (std::nothrow) kura_plan_s());
    if (!p) return KURA_ENOMEM;
    const int mode = o.precision == KURA_PREC_MIXED ? MODE_MIXED : MODE_FP64;
    PlanInput in;                      // host only: tile sizing for GB300's 152 SMs
    in.n = n; in.row_ptr = row_ptr; in.col = col; in.label = label; in.n_comm = n_comm; in.tau = o.tau;
    in.tile_max_rows = TILE_MAX_ROWS;
    in.tile_max_sub = tile_max_sub_for(mode);
    in.slot_ints = slot_ints_for(mode);
    in.entry_bytes = mode == MODE_MIXED ? 8 : 16;
    in.bitmap_zmin = o.bitmap_zmin;
    in.val = val;
    in.tensor_cores = o.tensor_cores;
    std::string err;
    int rc = build_plan(in, p->p, err);
    if (rc) { g_create_error = err; return rc == 2 ? KURA_ENOMEM : KURA_EINVAL; }
    *out = p.release();
    return KURA_OK;
}

kura_status kura_plan_stats(kura_plan_t pl, kura_block_stats* s)
{
    if (!pl || !s) return KURA_EINVAL;
    const Plan& p = pl->p;
    std::memset(s, 0, sizeof *s);
    s->n = p.n;
    s->nnz = p.nnz_in;
    s->self_loops = p.self_loops;
    s->n_comm = p.n_comm;
    s->q_bits = 61 - ceil_log2(std::max<int64_t>(p.n, 2));
    s->tau = p.tau;
    s->dense_blocks = p.dense_blocks;
    s->sparse_blocks = p.sparse_blocks;
    s->nonempty_blocks = p.nonempty_blocks;
    s->missing_entries = p.miss_total;
    s->sparse_entries = p.pres_total;
    s->max_row_entries = p.max_row_entries;
    s->tiles = int64_t(p.tiles.size());
    s->max_window = p.max_wlen;
    s->stream_bytes = plan_stream_bytes(p);
    s->node_bytes_row = (8 + 8 + 16 + 8 + 16) * p.n;
    s->node_bytes_trig = (8 + 16 + 4) * p.n;
    s->direct_edges = p.nnz_in - p.self_loops;
    s->tc_tiles = p.tc_tiles;
    s->tc_rows = p.tc_rows;
    s->tc_mask_bits = p.tc_mask_bits;
    return KURA_OK;
}

kura_status kura_plan_perm(kura_plan_t pl, int32_t* perm, int64_t* comm_off)
{
    if (!pl) return KURA_EINVAL;
    if (perm) std::copy(pl->p.perm.begin(), pl->p.perm.end(), perm);
    if (comm_off) std::copy(pl->p.comm_off.begin(), pl->p.comm_off.end(), comm_off);
    return KURA_OK;
}

kura_status kura_plan_row(kura_plan_t pl, int64_t row, int32_t* missing, int64_t* n_missing, int32_t* present,
                          int64_t* n_present, int64_t cap)
{
    if (!pl || !n_missing || !n_present) return KURA_EINVAL;
    const Plan& p = pl->p;
    if (row < 0 || row >= p.n) return KURA_EINVAL;
    *n_missing = p.miss_cnt[size_t(row)];
    *n_present = p.pres_cnt[size_t(row)];
    int64_t km = 0, kp = 0;
    const Tile& T = p.tiles[size_t(p.row_tile[size_t(row)])];
    if (T.flags & TILE_BITMAP) {
        const uint32_t* bm = p.bitmap.data() + T.bm_off + (row - T.r0) * int64_t(T.nsw) * 32;
        for (int64_t k = 0; k < T.wlen; k++)
            if ((bm[(k >> 10) * 32 + (k & 31)] >> ((k >> 5) & 31)) & 1u) {
                if (missing && km < cap) missing[km] = int32_t(T.wbeg + k);
                km++;
            }
    }
    if (T.flags & TILE_TC) {
        const int64_t lr = row - T.r0, nM = (T.r1 - T.r0 + TC_MBLOCK - 1) / TC_MBLOCK;
        for (int64_t kb = 0; kb < T.nsw; kb++) {
            const uint32_t* w = p.bitmap.data() + T.bm_off + ((kb * nM + lr / TC_MBLOCK) * TC_MBLOCK + lr % TC_MBLOCK) * 4;
            for (int64_t c = 0; c < TC_KBLOCK; c++)
                if ((w[c >> 5] >> (c & 31)) & 1u) {
                    if (missing && km < cap) missing[km] = int32_t(T.wbeg + kb * TC_KBLOCK + c);
                    km++;
                }
        }
    }
    for (int32_t sg = p.row_sub0[size_t(row)]; sg < p.row_sub0[size_t(row) + 1]; sg++) {
        const int32_t* hdr = p.gstream.data() + p.sub_hdr[size_t(sg)];
        for (int32_t q = 0; q < hdr[1]; q++, km++)
            if (missing && km < cap) missing[km] = p.gstream[size_t(p.sub_mpos[size_t(sg)] + q)];
        for (int32_t q = 0; q < hdr[3]; q++, kp++)
            if (present && kp < cap) present[kp] = p.gstream[size_t(p.sub_ppos[size_t(sg)] + q)];
    }
    if (km != *n_missing || kp != *n_present) return KURA_ESTATE;
    if (missing) std::sort(missing, missing + std::min(km, cap));      // stored in bank-balanced order
    return KURA_OK;
}

kura_status kura_plan_dense_blocks(kura_plan_t pl, int32_t I, int32_t* J, int32_t cap, int32_t* count)
{
    if (!pl || !count || I < 0 || I >= pl->p.n_comm) return KURA_EINVAL;
    const Plan& p = pl->p;
    *count = int32_t(p.dptr[size_t(I) + 1] - p.dptr[size_t(I)]);
    for (int32_t k = 0; k < *count && k < cap && J; k++) J[k] = p.dcol[size_t(p.dptr[size_t(I)] + k)];
    return KURA_OK;
}

kura_status kura_plan_export(kura_plan_t pl, const int32_t** gstream, int64_t* gstream_len, const void** groups,
                             int64_t* n_groups, const void** tiles, int64_t* n_tiles, const int32_t** row_sub0,
                             const uint32_t** bitmap, int64_t* bitmap_len)
{
    if (!pl) return KURA_EINVAL;
    const Plan& p = pl->p;
    if (gstream) *gstream = p.gstream.data();
    if (gstream_len) *gstream_len = int64_t(p.gstream.size());
    if (groups) *groups = p.groups.data();
    if (n_groups) *n_groups = int64_t(p.groups.size());
    if (tiles) *tiles = p.tiles.data();
    if (n_tiles) *n_tiles = int64_t(p.tiles.size());
    if (row_sub0) *row_sub0 = p.row_sub0.data();
    if (bitmap) *bitmap = p.bitmap.data();
    if (bitmap_len) *bitmap_len = int64_t(p.bitmap.size());
    return KURA_OK;
}

void kura_plan_destroy(kura_plan_t p) { delete p; }

}  // extern "C"
