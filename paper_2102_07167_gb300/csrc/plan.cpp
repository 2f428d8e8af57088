// Host-side block plan: permutation, dense/sparse block classification and the
// per-row correction streams of eq:KuramotoGraphApproach (Sec. 3 of
// arXiv 2102.07167).  See plan.hpp for the layout.
#include "plan.hpp"

#include <algorithm>
#include <cstring>
#include <new>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace kura {

namespace {

inline int64_t round_up4(int64_t x) { return (x + 3) & ~int64_t(3); }

// Writes the n missing entries of one sub-row to out[0, n) in an order that
// spreads the shared-memory banks of each warp-wide gather: the row kernel's
// lane l gathers, in step t of iteration i, the entry at position
// 128 i + 4 l + t, so the 32 positions {128 i + 4 l + t : l} are read by one
// instruction.  Entries are bucketed by bank group ((column - wbeg) mod K,
// K = 128 bytes / entry size) and dealt to each instruction one per bucket
// per round, fullest buckets first, so every instruction touches every bank
// group about equally often.  Any order gives
// the same sum up to rounding; this one is deterministic.
void balance_banks(const int32_t* in, int64_t n, int32_t wbeg, int K, int32_t* out)
{
    int32_t cnt[16] = {0}, start[17] = {0}, fill[16] = {0};
    std::vector<int32_t> sorted(size_t(n > 0 ? n : 1));
    for (int64_t k = 0; k < n; k++) cnt[((in[k] - wbeg) % K + K) % K]++;
    for (int b = 0; b < K; b++) start[b + 1] = start[b] + cnt[b];
    for (int64_t k = 0; k < n; k++) {
        const int b = ((in[k] - wbeg) % K + K) % K;
        sorted[size_t(start[b] + fill[b]++)] = in[k];
    }
    std::fill(fill, fill + 16, 0);
    // per instruction: deal one entry per bucket per round, fullest buckets
    // first, so the buckets drain evenly and the tail stays spread too
    int order[16];
    int64_t pos_list[32];
    for (int64_t i = 0; 128 * i < n; i++)
        for (int t = 0; t < 4; t++) {
            int np_ = 0;
            for (int l = 0; l < 32; l++)
                if (128 * i + 4 * l + t < n) pos_list[np_++] = 128 * i + 4 * l + t;
            int taken = 0;
            while (taken < np_) {
                for (int b = 0; b < K; b++) order[b] = b;
                std::sort(order, order + K, [&](int a, int b) {
                    const int ra = cnt[a] - fill[a], rb = cnt[b] - fill[b];
                    return ra != rb ? ra > rb : a < b;
                });
                for (int k = 0; k < K && taken < np_; k++) {
                    const int b = order[k];
                    if (fill[b] == cnt[b]) break;
                    out[pos_list[taken++]] = sorted[size_t(start[b] + fill[b]++)];
                }
            }
        }
}

// Dense-block membership of column block J for row block I (sorted list).
inline bool is_dense(const Plan& p, int32_t I, int32_t J)
{
    const int32_t* b = p.dcol.data() + p.dptr[I];
    const int32_t* e = p.dcol.data() + p.dptr[I + 1];
    if (e - b <= 8) {
        for (const int32_t* q = b; q < e; ++q) if (*q == J) return true;
        return false;
    }
    return std::binary_search(b, e, J);
}

// Value of dense block (I, J), 0 when the block is sparse.
inline int32_t dense_value(const Plan& p, int32_t I, int32_t J)
{
    const int32_t* b = p.dcol.data() + p.dptr[I];
    const int32_t* e = p.dcol.data() + p.dptr[I + 1];
    const int32_t* q = std::lower_bound(b, e, J);
    return (q != e && *q == J) ? p.dval[size_t(p.dptr[I] + (q - b))] : 0;
}

int validate(const PlanInput& in, std::string& err)
{
    if (in.n <= 0 || in.n >= (int64_t(1) << 31) - 8) { err = "n must be in [1, 2^31 - 8)"; return 1; }
    if (in.n_comm <= 0) { err = "n_comm must be positive"; return 1; }
    if (!in.row_ptr || !in.label) { err = "null graph array"; return 1; }
    if (!(in.tau >= 0.0 && in.tau <= 1.0)) { err = "tau must be in [0, 1]"; return 1; }
    if (in.row_ptr[0] != 0) { err = "row_ptr[0] must be 0"; return 1; }
    if (!in.col && in.row_ptr[in.n] != 0) { err = "null column array with edges"; return 1; }
    const int64_t n = in.n;
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 4096) reduction(|:bad)
    for (int64_t i = 0; i < n; i++) {
        int64_t b = in.row_ptr[i], e = in.row_ptr[i + 1];
        if (e < b) { bad |= 1; continue; }
        int64_t prev = -1;
        for (int64_t k = b; k < e; k++) {
            int64_t c = in.col[k];
            if (c < 0 || c >= n) { bad |= 2; break; }
            if (c <= prev) { bad |= 4; break; }
            prev = c;
        }
        if (in.label[i] < 0 || in.label[i] >= in.n_comm) bad |= 8;
    }
    if (bad & 1) { err = "row_ptr is not non-decreasing"; return 1; }
    if (bad & 2) { err = "column index out of range"; return 1; }
    if (bad & 4) { err = "columns not strictly increasing within a row (unsorted or duplicate)"; return 1; }
    if (bad & 8) { err = "label out of range [0, n_comm)"; return 1; }
    if (in.val) {
        if (n > VALUED_MAX_N) { err = "a finite-valued matrix needs n <= 2^24 - 2"; return 1; }
        const int64_t nnz = in.row_ptr[n];
        for (int64_t k = 0; k < nnz; k++)
            if (in.val[k] < 1 || in.val[k] > VALUED_MAX) { err = "values must be in [1, 127]"; return 1; }
    }
    return 0;
}

}  // namespace

int build_plan(const PlanInput& in, Plan& p, std::string& err)
{
    int rc = validate(in, err);
    if (rc) return rc;
    try {
        const int64_t n = in.n;
        const int32_t nc = in.n_comm;
        p = Plan();
        p.n = n;
        p.n_comm = nc;
        p.tau = in.tau;
        p.nnz_in = in.row_ptr[n];

        // ---- permutation: stable counting sort by label (P of Sec. 3)
        p.comm_off.assign(size_t(nc) + 1, 0);
        for (int64_t i = 0; i < n; i++) p.comm_off[size_t(in.label[i]) + 1]++;
        for (int32_t I = 0; I < nc; I++) p.comm_off[I + 1] += p.comm_off[I];
        p.perm.resize(size_t(n));
        p.inv_perm.resize(size_t(n));
        {
            std::vector<int64_t> pos(p.comm_off.begin(), p.comm_off.end() - 1);
            for (int64_t i = 0; i < n; i++) p.perm[size_t(pos[size_t(in.label[i])]++)] = int32_t(i);
        }
        p.node_comm.resize(size_t(n));
        #pragma omp parallel for schedule(static)
        for (int64_t v = 0; v < n; v++) {
            p.inv_perm[size_t(p.perm[size_t(v)])] = int32_t(v);
            p.node_comm[size_t(v)] = in.label[p.perm[size_t(v)]];
        }
        auto csize = [&](int32_t I) { return p.comm_off[size_t(I) + 1] - p.comm_off[size_t(I)]; };

        // ---- degrees and self-loops
        p.deg.resize(size_t(n));
        int64_t loops = 0;
        #pragma omp parallel for schedule(static) reduction(+:loops)
        for (int64_t v = 0; v < n; v++) {
            int64_t o = p.perm[size_t(v)], d = 0;
            for (int64_t k = in.row_ptr[o]; k < in.row_ptr[o + 1]; k++) {
                if (in.col[k] == o) loops++; else d++;
            }
            p.deg[size_t(v)] = int32_t(d);
        }
        p.self_loops = loops;

        // ---- block classification: non-zeros per block (I, J), zero fraction
        // over n_I n_J entries (n_I (n_I - 1) off-diagonal entries on the
        // diagonal block, whose diagonal is don't-care); dense iff below tau.
        std::vector<std::vector<int32_t>> dense_of(static_cast<size_t>(nc));
        std::vector<std::vector<int32_t>> dval_of(static_cast<size_t>(nc));
        int64_t nonempty = 0, ndense = 0;
        p.valued = in.val != nullptr;
        if (p.valued)
            for (int64_t k = 0; k < in.row_ptr[n]; k++) p.max_weight = std::max(p.max_weight, in.val[k]);
        if (p.valued) {
            // finite values: per block the nonzero value of largest count (ties:
            // the smaller); dense with that value iff the fraction of entries
            // different from it is below tau
            #pragma omp parallel reduction(+:nonempty, ndense)
            {
                std::vector<int64_t> keys;
                #pragma omp for schedule(dynamic, 1)
                for (int32_t I = 0; I < nc; I++) {
                    keys.clear();
                    for (int64_t v = p.comm_off[I]; v < p.comm_off[I + 1]; v++) {
                        int64_t o = p.perm[size_t(v)];
                        for (int64_t k = in.row_ptr[o]; k < in.row_ptr[o + 1]; k++) {
                            if (in.col[k] == o) continue;
                            keys.push_back(int64_t(in.label[in.col[k]]) * 128 + in.val[k]);
                        }
                    }
                    std::sort(keys.begin(), keys.end());
                    for (size_t a = 0; a < keys.size();) {
                        const int32_t J = int32_t(keys[a] / 128);
                        int32_t best = 0;
                        int64_t bestc = 0;
                        size_t b = a;
                        while (b < keys.size() && keys[b] / 128 == J) {
                            size_t c = b;
                            while (c < keys.size() && keys[c] == keys[b]) c++;
                            if (int64_t(c - b) > bestc) { bestc = int64_t(c - b); best = int32_t(keys[b] % 128); }
                            b = c;
                        }
                        const double entries = (J == I) ? double(csize(I)) * double(csize(I) - 1)
                                                        : double(csize(I)) * double(csize(J));
                        nonempty++;
                        if (1.0 - double(bestc) / entries < in.tau) {
                            dense_of[size_t(I)].push_back(J);
                            dval_of[size_t(I)].push_back(best);
                            ndense++;
                        }
                        a = b;
                    }
                }
            }
        } else
        #pragma omp parallel reduction(+:nonempty, ndense)
        {
            std::vector<int64_t> cnt(size_t(nc), 0);
            std::vector<int32_t> touched;
            #pragma omp for schedule(dynamic, 1)
            for (int32_t I = 0; I < nc; I++) {
                touched.clear();
                for (int64_t v = p.comm_off[I]; v < p.comm_off[I + 1]; v++) {
                    int64_t o = p.perm[size_t(v)];
                    for (int64_t k = in.row_ptr[o]; k < in.row_ptr[o + 1]; k++) {
                        int32_t c = in.col[k];
                        if (c == o) continue;
                        int32_t J = in.label[c];
                        if (cnt[size_t(J)]++ == 0) touched.push_back(J);
                    }
                }
                std::sort(touched.begin(), touched.end());
                for (int32_t J : touched) {
                    double entries = (J == I) ? double(csize(I)) * double(csize(I) - 1)
                                              : double(csize(I)) * double(csize(J));
                    double zero_frac = 1.0 - double(cnt[size_t(J)]) / entries;
                    nonempty++;
                    if (zero_frac < in.tau) { dense_of[size_t(I)].push_back(J); dval_of[size_t(I)].push_back(1); ndense++; }
                    cnt[size_t(J)] = 0;
                }
            }
        }
        p.nonempty_blocks = nonempty;
        p.dense_blocks = ndense;
        p.sparse_blocks = nonempty - ndense;
        p.dptr.assign(size_t(nc) + 1, 0);
        for (int32_t I = 0; I < nc; I++) p.dptr[I + 1] = p.dptr[I] + int64_t(dense_of[size_t(I)].size());
        p.dcol.resize(size_t(p.dptr[nc]));
        p.dval.resize(size_t(p.dptr[nc]));
        for (int32_t I = 0; I < nc; I++) {
            std::copy(dense_of[size_t(I)].begin(), dense_of[size_t(I)].end(), p.dcol.begin() + p.dptr[I]);
            std::copy(dval_of[size_t(I)].begin(), dval_of[size_t(I)].end(), p.dval.begin() + p.dptr[I]);
        }
        std::vector<int64_t> dense_span(size_t(nc), 0);   // sum of n_J over D(I)
        std::vector<uint8_t> self_dense(size_t(nc), 0);
        for (int32_t I = 0; I < nc; I++)
            for (int64_t k = p.dptr[I]; k < p.dptr[I + 1]; k++) {
                dense_span[size_t(I)] += csize(p.dcol[size_t(k)]);
                if (p.dcol[size_t(k)] == I) self_dense[size_t(I)] = 1;
            }

        // ---- per-row counts
        p.miss_cnt.resize(size_t(n));
        p.pres_cnt.resize(size_t(n));
        #pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t v = 0; v < n; v++) {
            int32_t I = p.node_comm[size_t(v)];
            int64_t o = p.perm[size_t(v)], in_dense = 0, np_ = 0;
            for (int64_t k = in.row_ptr[o]; k < in.row_ptr[o + 1]; k++) {
                int32_t c = in.col[k];
                if (c == o) continue;
                if (p.valued) {
                    // in_dense counts the dense-block entries equal to their block's value
                    const int32_t bv = dense_value(p, I, in.label[c]);
                    if (bv == 0) np_++;
                    else if (in.val[k] == bv) in_dense++;
                } else if (is_dense(p, I, in.label[c])) {
                    in_dense++;
                } else {
                    np_++;
                }
            }
            p.miss_cnt[size_t(v)] = int32_t(dense_span[size_t(I)] - self_dense[size_t(I)] - in_dense);
            p.pres_cnt[size_t(v)] = int32_t(np_);
        }
        int64_t mx = 0;
        for (int64_t v = 0; v < n; v++) {
            p.miss_total += p.miss_cnt[size_t(v)];
            p.pres_total += p.pres_cnt[size_t(v)];
            mx = std::max<int64_t>(mx, int64_t(p.miss_cnt[size_t(v)]) + p.pres_cnt[size_t(v)]);
        }
        p.max_row_entries = mx;

        // ---- staged window of every community: its own columns joined with
        // its dense column blocks when that span fits the cap, else its own
        // columns (aligned to an even start and length for 16-byte copies).
        // When every dense column is inside the window, the missing entries
        // become a tensor-core mask (TILE_TC) if that is smaller than their
        // index lists (tensor_cores = 1) or always (2), else row bitmaps if
        // the zero fraction over the dense columns exceeds bitmap_zmin.
        std::vector<int32_t> c_wbeg(size_t(nc), 0), c_wlen(size_t(nc), 0), c_nsw(size_t(nc), 0);
        std::vector<int32_t> c_kb0(size_t(nc), 0), c_nkb(size_t(nc), 0);
        std::vector<uint8_t> c_bitmap(size_t(nc), 0), c_inwin(size_t(nc), 0), c_tc(size_t(nc), 0);
        std::vector<int32_t> c_mpad(static_cast<size_t>(nc), static_cast<int32_t>(n));
        for (int32_t I = 0; I < nc; I++) {
            int64_t rb = p.comm_off[I], re = p.comm_off[I + 1];
            if (rb == re) continue;
            int64_t lo = rb, hi = re;
            for (int64_t k = p.dptr[I]; k < p.dptr[I + 1]; k++) {
                lo = std::min(lo, p.comm_off[size_t(p.dcol[size_t(k)])]);
                hi = std::max(hi, p.comm_off[size_t(p.dcol[size_t(k)]) + 1]);
            }
            bool covers = true;
            if (hi - lo > in.window_cap) { lo = rb; hi = re; covers = false; }
            int64_t wb = lo & ~int64_t(1), we = (hi + 1) & ~int64_t(1);
            int32_t wbeg = int32_t(wb), wlen = int32_t(we - wb);
            if (wlen > in.window_cap + 2) { wbeg = 0; wlen = 0; covers = false; }
            c_wbeg[size_t(I)] = wbeg;
            c_wlen[size_t(I)] = wlen;
            if (covers && wlen > 0) {
                c_inwin[size_t(I)] = 1;
                c_mpad[size_t(I)] = wbeg - 1;
            }
            p.max_wlen = std::max(p.max_wlen, wlen);
            if (covers && in.tensor_cores > 0 && !p.valued && p.dptr[I + 1] > p.dptr[I]) {
                // tensor-core mask over the K-blocks spanning the dense columns [lo, hi)
                const int64_t kb0 = lo / TC_KBLOCK, kb1 = (hi + TC_KBLOCK - 1) / TC_KBLOCK;
                int64_t zeros = 0;
                for (int64_t v = rb; v < re; v++) zeros += p.miss_cnt[size_t(v)];
                const int64_t bits_bytes = (re - rb + TC_MBLOCK - 1) / TC_MBLOCK * TC_MBLOCK * (kb1 - kb0) * 16;
                if (zeros > 0 && (in.tensor_cores >= 2 || bits_bytes < 4 * zeros)) {
                    c_tc[size_t(I)] = 1;
                    c_kb0[size_t(I)] = int32_t(kb0);
                    c_nkb[size_t(I)] = int32_t(kb1 - kb0);
                    continue;
                }
            }
            if (covers && wlen > 0 && in.bitmap_zmin >= 0 && !p.valued && p.dptr[I + 1] > p.dptr[I]) {
                double zeros = 0, entries = 0;
                for (int64_t v = rb; v < re; v++) zeros += p.miss_cnt[size_t(v)];
                entries = double(re - rb) * double(dense_span[size_t(I)]);
                const int32_t nsw = int32_t((wlen + 1023) / 1024);
                if (entries > 0 && zeros / entries > in.bitmap_zmin && nsw <= BITMAP_MAX_SW) {
                    c_bitmap[size_t(I)] = 1;
                    c_nsw[size_t(I)] = nsw;
                    p.bitmap_rows += re - rb;
                }
            }
        }
        // missing entries given as index lists (not in a bitmap)
        auto listed_miss = [&](int64_t v) -> int64_t {
            const size_t I = size_t(p.node_comm[size_t(v)]);
            return (c_bitmap[I] || c_tc[I]) ? 0 : p.miss_cnt[size_t(v)];
        };

        // ---- sub-rows: each row is cut into ceil((nm + np) / SUBROW_MAX)
        // pieces (at least one) of consecutive entries of [missing | present]
        // (nm = listed missing entries).
        p.row_sub0.assign(size_t(n) + 1, 0);
        for (int64_t v = 0; v < n; v++) {
            const int64_t e = listed_miss(v) + p.pres_cnt[size_t(v)];
            p.row_sub0[size_t(v) + 1] = p.row_sub0[size_t(v)] + int32_t(std::max<int64_t>(1, (e + SUBROW_MAX - 1) / SUBROW_MAX));
        }
        const int64_t n_sub = p.row_sub0[size_t(n)];
        for (int64_t v = 0; v < n; v++)
            if (p.row_sub0[size_t(v) + 1] - p.row_sub0[size_t(v)] > in.tile_max_sub) {
                err = "a row stores more corrections than the row kernel supports (" +
                      std::to_string(int64_t(in.tile_max_sub) * SUBROW_MAX) + "); raise tau or split the community";
                return 1;
            }
        // missing / present parts of sub-row (row v, piece k)
        auto sub_parts = [&](int64_t v, int64_t k, int64_t& mb, int64_t& mn, int64_t& pb, int64_t& pn) {
            const int64_t nm = listed_miss(v), np_ = p.pres_cnt[size_t(v)];
            const int64_t b = k * SUBROW_MAX, e = std::min<int64_t>(b + SUBROW_MAX, nm + np_);
            mb = std::min(b, nm);
            mn = std::min(e, nm) - mb;
            pb = std::max<int64_t>(b, nm) - nm;
            pn = std::max<int64_t>(e, nm) - nm - pb;
            if (pn < 0) pn = 0;
        };
        auto sub_ints = [&](int64_t v, int64_t k) {
            int64_t mb, mn, pb, pn;
            sub_parts(v, k, mb, mn, pb, pn);
            return 4 + round_up4(mn) + round_up4(pn);
        };

        // ---- tiles (rows of one community, bounded work, rows and sub-rows;
        // staged window = the community's own columns joined with its dense
        // column blocks when that span fits the cap, else the community's
        // columns) and row groups (consecutive sub-rows of a tile, at most
        // GROUP_MAX_SUB, whose packed stream fits one slot of the row kernel).
        int64_t total_work = 0;
        for (int64_t v = 0; v < n; v++) total_work += p.miss_cnt[size_t(v)] + p.pres_cnt[size_t(v)] + 8;
        const int64_t target = in.tile_work > 0 ? in.tile_work : std::max<int64_t>(2048, total_work / (int64_t(std::max(in.n_sms, 1)) * 12));
        p.sub_hdr.resize(size_t(n_sub));
        std::vector<int64_t>& sub_mpos = p.sub_mpos;
        std::vector<int64_t>& sub_ppos = p.sub_ppos;
        sub_mpos.resize(size_t(n_sub));
        sub_ppos.resize(size_t(n_sub));
        int64_t goff = 0;
        int64_t bm_words = 0;
        std::vector<int64_t> tile_work;       // work estimate of each tile (entries + per-row overhead)
        p.row_tile.resize(size_t(n));
        for (int32_t I = 0; I < nc; I++) {
            int64_t rb = p.comm_off[I], re = p.comm_off[I + 1];
            if (rb == re) continue;
            const int32_t wbeg = c_wbeg[size_t(I)], wlen = c_wlen[size_t(I)];
            int64_t r = rb;
            while (r < re) {
                int64_t w = 0, s = r;
                while (r < re && (r == s || (w < target && r - s < in.tile_max_rows &&
                                             p.row_sub0[size_t(r) + 1] - p.row_sub0[size_t(s)] <= in.tile_max_sub))) {
                    w += (c_tc[size_t(I)] ? 4 * c_nkb[size_t(I)]
                                          : c_bitmap[size_t(I)] ? 8 * c_nsw[size_t(I)] : p.miss_cnt[size_t(r)]) +
                         p.pres_cnt[size_t(r)] + 8;
                    r++;
                }
                Tile t{};
                t.r0 = int32_t(s); t.r1 = int32_t(r); t.comm = I; t.wbeg = wbeg; t.wlen = wlen;
                t.sub0 = p.row_sub0[size_t(s)];
                if (c_tc[size_t(I)]) {
                    const int64_t nM = (r - s + TC_MBLOCK - 1) / TC_MBLOCK;
                    t.flags |= TILE_TC;
                    t.wbeg = c_kb0[size_t(I)] * TC_KBLOCK;
                    t.wlen = 0;
                    t.nsw = c_nkb[size_t(I)];
                    bm_words = (bm_words + TC_MBLOCK * 4 - 1) / (TC_MBLOCK * 4) * (TC_MBLOCK * 4);   // whole blocks
                    t.bm_off = bm_words;
                    bm_words += nM * int64_t(t.nsw) * TC_MBLOCK * 4;
                    p.tc_tiles++;
                    p.tc_rows += r - s;
                    p.tc_mask_bits += nM * TC_MBLOCK * int64_t(t.nsw) * TC_KBLOCK;
                } else if (p.valued) {
                    t.flags |= TILE_VALUED;
                } else {
                    if (c_inwin[size_t(I)]) t.flags |= TILE_MISS_IN_WINDOW;
                    if (!std::binary_search(p.dcol.begin() + p.dptr[I], p.dcol.begin() + p.dptr[I + 1], I))
                        t.flags |= TILE_PRES_CHECK;
                }
                if (c_bitmap[size_t(I)]) {
                    t.flags |= TILE_BITMAP;
                    t.nsw = c_nsw[size_t(I)];
                    t.bm_off = bm_words;
                    bm_words += (r - s) * int64_t(t.nsw) * 32;
                }
                for (int64_t q = s; q < r; q++) p.row_tile[size_t(q)] = int32_t(p.tiles.size());
                t.g0 = int32_t(p.groups.size());
                // groups over the tile's sub-rows [row_sub0[s], row_sub0[r])
                int64_t v = s, k = 0;             // current sub-row = (row v, piece k)
                while (v < r) {
                    Group G{};
                    G.off = goff;
                    G.sub0 = p.row_sub0[size_t(v)] + int32_t(k);
                    int64_t size = 0;
                    std::vector<std::pair<int64_t, int64_t>> members;
                    bool all_short = true;        // every member fits one int4 per lane
                    while (v < r) {
                        const int64_t si = sub_ints(v, k);
                        const bool short_ = si - 4 <= SHORT_SUB_INTS;
                        const int64_t cap = (all_short && short_ && in.entry_bytes == 8 && !p.valued)
                                                ? GROUP_MAX_SUB_SHORT : GROUP_MAX_SUB;
                        if (int64_t(members.size()) >= cap) break;
                        if (!members.empty() && size + si > in.slot_ints) break;
                        members.emplace_back(v, k);
                        all_short = all_short && short_;
                        size += si;
                        if (++k == p.row_sub0[size_t(v) + 1] - p.row_sub0[size_t(v)]) { k = 0; v++; }
                    }
                    G.nsub = int32_t(members.size());
                    G.len = int32_t(size);
                    int64_t pos = goff + 4 * G.nsub;
                    for (size_t m = 0; m < members.size(); m++) {            // [missing | present] per sub-row
                        int64_t mb, mn, pb, pn;
                        sub_parts(members[m].first, members[m].second, mb, mn, pb, pn);
                        const int64_t sg = G.sub0 + int64_t(m);
                        p.sub_hdr[size_t(sg)] = goff + 4 * int64_t(m);
                        sub_mpos[size_t(sg)] = pos;
                        pos += round_up4(mn);
                        sub_ppos[size_t(sg)] = pos;
                        pos += round_up4(pn);
                    }
                    goff += size;
                    p.groups.push_back(G);
                }
                t.g1 = int32_t(p.groups.size());
                p.tiles.push_back(t);
                tile_work.push_back(w);
            }
        }
        p.gstream.assign(size_t(std::max<int64_t>(goff, 4)), 0);
        p.bitmap.assign(size_t(std::max<int64_t>(bm_words, 4)), 0u);

        // ---- fill: mark dense-block neighbours in a bitmap, scan the dense
        // column ranges for zeros (skipping the row's own diagonal entry),
        // collect the sparse-block neighbours; then write the row's entries
        // into its sub-row segments with headers and padding.
        #pragma omp parallel
        {
            std::vector<uint64_t> bits(size_t((n + 63) / 64), 0);
            std::vector<int32_t> ms, pr;
            std::vector<int32_t> vmark(p.valued ? size_t(n) : size_t(0), 0);   // value of each neighbour
            std::vector<std::pair<int32_t, int32_t>> prv;
            #pragma omp for schedule(dynamic, 256)
            for (int64_t v = 0; v < n; v++) {
                int32_t I = p.node_comm[size_t(v)];
                int64_t o = p.perm[size_t(v)];
                ms.clear();
                pr.clear();
                if (p.valued) {
                    // dense blocks: every column whose value differs from the block's value,
                    // weight A - v; sparse blocks: the entries, weight A
                    prv.clear();
                    for (int64_t k = in.row_ptr[o]; k < in.row_ptr[o + 1]; k++) {
                        int32_t c = in.col[k];
                        if (c == o) continue;
                        int32_t w = p.inv_perm[size_t(c)];
                        if (dense_value(p, I, in.label[c])) vmark[size_t(w)] = in.val[k];
                        else prv.emplace_back(w, in.val[k]);
                    }
                    std::sort(prv.begin(), prv.end());
                    for (const auto& e : prv) pr.push_back(valued_pack(e.first, e.second));
                    for (int64_t k = p.dptr[I]; k < p.dptr[I + 1]; k++) {
                        const int32_t J = p.dcol[size_t(k)], bv = p.dval[size_t(k)];
                        for (int64_t w = p.comm_off[size_t(J)]; w < p.comm_off[size_t(J) + 1]; w++)
                            if (w != v && vmark[size_t(w)] != bv) ms.push_back(valued_pack(w, vmark[size_t(w)] - bv));
                    }
                    for (int64_t k = in.row_ptr[o]; k < in.row_ptr[o + 1]; k++)
                        if (in.col[k] != o) vmark[size_t(p.inv_perm[size_t(in.col[k])])] = 0;
                } else {
                for (int64_t k = in.row_ptr[o]; k < in.row_ptr[o + 1]; k++) {
                    int32_t c = in.col[k];
                    if (c == o) continue;
                    int32_t w = p.inv_perm[size_t(c)];
                    if (is_dense(p, I, in.label[c])) bits[size_t(w) >> 6] |= uint64_t(1) << (w & 63);
                    else pr.push_back(w);
                }
                std::sort(pr.begin(), pr.end());
                for (int64_t k = p.dptr[I]; k < p.dptr[I + 1]; k++) {
                    int32_t J = p.dcol[size_t(k)];
                    int64_t b = p.comm_off[size_t(J)], e = p.comm_off[size_t(J) + 1];
                    for (int64_t w = b; w < e;) {
                        int64_t word = w >> 6, lo = w & 63;
                        int64_t hi = std::min<int64_t>(64, lo + (e - w));
                        uint64_t zeros = ~bits[size_t(word)];
                        zeros >>= lo;
                        if (hi - lo < 64) zeros &= (uint64_t(1) << (hi - lo)) - 1;
                        while (zeros) {
                            int t = __builtin_ctzll(zeros);
                            int64_t col = w + t;
                            if (col != v) ms.push_back(int32_t(col));
                            zeros &= zeros - 1;
                        }
                        w += hi - lo;
                    }
                }
                for (int64_t k = in.row_ptr[o]; k < in.row_ptr[o + 1]; k++) {
                    int32_t c = in.col[k];
                    if (c == o) continue;
                    int32_t w = p.inv_perm[size_t(c)];
                    bits[size_t(w) >> 6] = 0;
                }
                }
                // tensor-core rows: the missing entries become mask bits
                if (c_tc[size_t(I)]) {
                    const Tile& T = p.tiles[size_t(p.row_tile[size_t(v)])];
                    const int64_t lr = v - T.r0, nM = (T.r1 - T.r0 + TC_MBLOCK - 1) / TC_MBLOCK;
                    const int64_t m = lr / TC_MBLOCK, rr = lr % TC_MBLOCK;
                    for (int32_t c : ms) {
                        const int64_t k = int64_t(c) - T.wbeg, kb = k / TC_KBLOCK, kc = k % TC_KBLOCK;
                        p.bitmap[size_t(T.bm_off + ((kb * nM + m) * TC_MBLOCK + rr) * 4 + (kc >> 5))] |=
                            uint32_t(1) << (kc & 31);
                    }
                    ms.clear();
                }
                // bitmap rows: the missing entries become bits over the window
                if (c_bitmap[size_t(I)]) {
                    const Tile& T = p.tiles[size_t(p.row_tile[size_t(v)])];
                    uint32_t* bm = p.bitmap.data() + T.bm_off + (v - T.r0) * int64_t(T.nsw) * 32;
                    for (int32_t c : ms) {
                        const int64_t k = int64_t(c) - T.wbeg;
                        bm[(k >> 10) * 32 + (k & 31)] |= uint32_t(1) << ((k >> 5) & 31);
                    }
                    ms.clear();
                }
                // sub-rows of row v
                const int32_t s0 = p.row_sub0[size_t(v)], s1 = p.row_sub0[size_t(v) + 1];
                for (int32_t sg = s0; sg < s1; sg++) {
                    int64_t mb, mn, pb, pn;
                    sub_parts(v, sg - s0, mb, mn, pb, pn);
                    int32_t* hdr = p.gstream.data() + p.sub_hdr[size_t(sg)];
                    int32_t* mdst = p.gstream.data() + sub_mpos[size_t(sg)];
                    int32_t* pdst = p.gstream.data() + sub_ppos[size_t(sg)];
                    if (p.valued) {
                        const int32_t pad = valued_pack(n, 0);
                        for (int64_t q = 0; q < mn; q++) mdst[q] = ms[size_t(mb + q)];
                        for (int64_t q = mn; q < round_up4(mn); q++) mdst[q] = pad;
                        for (int64_t q = 0; q < pn; q++) pdst[q] = pr[size_t(pb + q)];
                        for (int64_t q = pn; q < round_up4(pn); q++) pdst[q] = pad;
                    } else {
                        balance_banks(ms.data() + mb, mn, p.tiles[size_t(p.row_tile[size_t(v)])].wbeg,
                                      in.entry_bytes >= 16 ? 8 : 16, mdst);
                        for (int64_t q = mn; q < round_up4(mn); q++) mdst[q] = c_mpad[size_t(I)];
                        for (int64_t q = 0; q < pn; q++) pdst[q] = pr[size_t(pb + q)];
                        for (int64_t q = pn; q < round_up4(pn); q++) pdst[q] = int32_t(n);
                    }
                    hdr[1] = int32_t(mn);
                    hdr[3] = int32_t(pn);
                }
            }
        }
        // header offsets relative to the group start
        for (const Group& G : p.groups)
            for (int32_t m = 0; m < G.nsub; m++) {
                int32_t* hdr = p.gstream.data() + G.off + 4 * m;
                hdr[0] = int32_t(sub_mpos[size_t(G.sub0 + m)] - G.off);
                hdr[2] = int32_t(sub_ppos[size_t(G.sub0 + m)] - G.off);
            }
        // launch order: longest tiles first (CTAs start in index order, so the
        // last wave holds the shortest tiles); ties keep community order
        {
            std::vector<int32_t> order(p.tiles.size());
            for (size_t q = 0; q < order.size(); q++) order[q] = int32_t(q);
            std::stable_sort(order.begin(), order.end(),
                             [&](int32_t a, int32_t b) { return tile_work[size_t(a)] > tile_work[size_t(b)]; });
            std::vector<Tile> sorted(p.tiles.size());
            std::vector<int32_t> new_index(p.tiles.size());
            for (size_t q = 0; q < order.size(); q++) {
                sorted[q] = p.tiles[size_t(order[q])];
                new_index[size_t(order[q])] = int32_t(q);
            }
            p.tiles.swap(sorted);
            for (int64_t v = 0; v < n; v++) p.row_tile[size_t(v)] = new_index[size_t(p.row_tile[size_t(v)])];
        }
    } catch (const std::bad_alloc&) {
        err = "out of host memory while building the block plan";
        return 2;
    }
    return 0;
}

}  // namespace kura
