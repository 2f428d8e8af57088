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
        int64_t nonempty = 0, ndense = 0;
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
                    if (zero_frac < in.tau) { dense_of[size_t(I)].push_back(J); ndense++; }
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
        for (int32_t I = 0; I < nc; I++)
            std::copy(dense_of[size_t(I)].begin(), dense_of[size_t(I)].end(), p.dcol.begin() + p.dptr[I]);
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
                if (is_dense(p, I, in.label[c])) in_dense++; else np_++;
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

        // ---- tiles (rows of one community, bounded work and rows; staged
        // window = the community's own columns joined with its dense column
        // blocks when that span fits the cap, else the community's columns)
        // and row groups (consecutive rows of a tile whose packed stream fits
        // one slot of the row kernel; a row alone larger than a slot is an
        // oversized group read in place).
        auto row_ints = [&](int64_t v) {
            return 4 + round_up4(p.miss_cnt[size_t(v)]) + round_up4(p.pres_cnt[size_t(v)]);
        };
        int64_t total_work = 0;
        for (int64_t v = 0; v < n; v++) total_work += p.miss_cnt[size_t(v)] + p.pres_cnt[size_t(v)] + 8;
        const int64_t target = in.tile_work > 0 ? in.tile_work : std::max<int64_t>(2048, total_work / (152 * 12));
        std::vector<int64_t> row_pos(static_cast<size_t>(n));       // start of each row's missing segment in gstream
        p.row_group.resize(size_t(n));
        int64_t goff = 0;
        for (int32_t I = 0; I < nc; I++) {
            int64_t rb = p.comm_off[I], re = p.comm_off[I + 1];
            if (rb == re) continue;
            int64_t lo = rb, hi = re;
            for (int64_t k = p.dptr[I]; k < p.dptr[I + 1]; k++) {
                lo = std::min(lo, p.comm_off[size_t(p.dcol[size_t(k)])]);
                hi = std::max(hi, p.comm_off[size_t(p.dcol[size_t(k)]) + 1]);
            }
            if (hi - lo > in.window_cap) { lo = rb; hi = re; }
            int64_t wb = lo & ~int64_t(1), we = (hi + 1) & ~int64_t(1);
            int32_t wbeg = int32_t(wb), wlen = int32_t(we - wb);
            if (wlen > in.window_cap + 2) { wbeg = 0; wlen = 0; }
            p.max_wlen = std::max(p.max_wlen, wlen);
            int64_t r = rb;
            while (r < re) {
                int64_t w = 0, s = r;
                while (r < re && (r == s || (w < target && r - s < in.tile_max_rows))) {
                    w += p.miss_cnt[size_t(r)] + p.pres_cnt[size_t(r)] + 8;
                    r++;
                }
                Tile t{};
                t.r0 = int32_t(s); t.r1 = int32_t(r); t.comm = I; t.wbeg = wbeg; t.wlen = wlen;
                t.g0 = int32_t(p.groups.size());
                // groups of the tile rows [s, r)
                int64_t q = s;
                while (q < r) {
                    Group G{};
                    G.off = goff;
                    G.r0 = int32_t(q);
                    int64_t size = row_ints(q);
                    if (size > in.slot_ints) {
                        G.flags = GROUP_OVERSIZED;
                        q++;
                    } else {
                        q++;
                        while (q < r && size + row_ints(q) <= in.slot_ints) size += row_ints(q++);
                    }
                    G.r1 = int32_t(q);
                    G.len = int32_t(size);
                    // positions inside the group: headers, then missing, then present segments
                    int64_t mpos = goff + 4 * (G.r1 - G.r0);
                    for (int64_t v = G.r0; v < G.r1; v++) { row_pos[size_t(v)] = mpos; mpos += round_up4(p.miss_cnt[size_t(v)]); }
                    const int32_t gi = int32_t(p.groups.size());
                    for (int64_t v = G.r0; v < G.r1; v++) p.row_group[size_t(v)] = gi;
                    goff += size;
                    p.groups.push_back(G);
                }
                t.g1 = int32_t(p.groups.size());
                p.tiles.push_back(t);
            }
        }
        p.gstream.assign(size_t(std::max<int64_t>(goff, 4)), 0);
        // headers (offsets relative to the group start)
        #pragma omp parallel for schedule(dynamic, 64)
        for (int64_t gi = 0; gi < int64_t(p.groups.size()); gi++) {
            const Group& G = p.groups[size_t(gi)];
            int64_t mtot = 0;
            for (int64_t v = G.r0; v < G.r1; v++) mtot += round_up4(p.miss_cnt[size_t(v)]);
            int64_t ppos = row_pos[size_t(G.r0)] + mtot;
            for (int64_t v = G.r0; v < G.r1; v++) {
                int32_t* hdr = p.gstream.data() + G.off + 4 * (v - G.r0);
                hdr[0] = int32_t(row_pos[size_t(v)] - G.off);
                hdr[1] = p.miss_cnt[size_t(v)];
                hdr[2] = int32_t(ppos - G.off);
                hdr[3] = p.pres_cnt[size_t(v)];
                ppos += round_up4(p.pres_cnt[size_t(v)]);
            }
        }

        // ---- fill: mark dense-block neighbours in a bitmap, scan the dense
        // column ranges for zeros (skipping the row's own diagonal entry),
        // collect the sparse-block neighbours.
        #pragma omp parallel
        {
            std::vector<uint64_t> bits(size_t((n + 63) / 64), 0);
            #pragma omp for schedule(dynamic, 256)
            for (int64_t v = 0; v < n; v++) {
                int32_t I = p.node_comm[size_t(v)];
                int64_t o = p.perm[size_t(v)];
                const Group& G = p.groups[size_t(p.row_group[size_t(v)])];
                const int32_t* hdr = p.gstream.data() + G.off + 4 * (v - G.r0);
                int32_t* pr = p.gstream.data() + G.off + hdr[2];
                int64_t np_ = 0;
                for (int64_t k = in.row_ptr[o]; k < in.row_ptr[o + 1]; k++) {
                    int32_t c = in.col[k];
                    if (c == o) continue;
                    int32_t w = p.inv_perm[size_t(c)];
                    if (is_dense(p, I, in.label[c])) bits[size_t(w) >> 6] |= uint64_t(1) << (w & 63);
                    else pr[np_++] = w;
                }
                std::sort(pr, pr + np_);
                int32_t* ms = p.gstream.data() + G.off + hdr[0];
                int64_t nm = 0;
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
                            if (col != v) ms[nm++] = int32_t(col);
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
        }
    } catch (const std::bad_alloc&) {
        err = "out of host memory while building the block plan";
        return 2;
    }
    return 0;
}

}  // namespace kura
