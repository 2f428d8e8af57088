// Host-side block plan for the localised-order-parameter right-hand side
// (eq:KuramotoGraphApproach, Sec. 3 of arXiv 2102.07167).
//
// The plan permutes the nodes so that communities are contiguous (P A P^T,
// Sec. 3 "Community detection in graphs"), classifies every block (I, J) as
// dense or sparse by its zero fraction, and writes two correction streams per
// row: the missing entries of the row's dense blocks ("zeros", subtracted from
// the precomputed block sums) and the present entries of its sparse blocks
// (summed directly).  It also cuts the rows into tiles for the row kernel.
// Pure host code: no CUDA here, so the planner is testable without a GPU.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace kura {

struct Tile {              // 48 bytes, read by the row kernel
    int32_t r0, r1;        // rows [r0, r1) in permuted order, all in one community
    int32_t comm;          // community of the rows
    int32_t wbeg, wlen;    // staged table window [wbeg, wbeg + wlen) (wlen = 0: none)
    int32_t g0, g1;        // row groups [g0, g1) of the tile
    int32_t sub0;          // global index of the tile's first sub-row
    int64_t bm_off;        // TILE_BITMAP: first word of the tile's row bitmaps
    int32_t nsw;           // TILE_BITMAP: 1024-column super-words per row
    int32_t flags;
};
// The tile's missing entries are given as bitmaps over its window instead of
// index lists: per row nsw super-words of 32 words, bit j of word q of
// super-word w set iff window column w * 1024 + 32 j + q is a missing entry.
constexpr int32_t TILE_BITMAP = 1;
// every dense column of the tile lies in its window: missing entries are read
// from the window without a range check, and missing-segment padding is
// wbeg - 1, which the row kernel maps to a zero entry kept just before the
// staged window (other tiles pad with n and range-check every gather)
constexpr int32_t TILE_MISS_IN_WINDOW = 2;
// the diagonal block is sparse: present entries may lie in the window and are
// range-checked (otherwise they are gathered from the global table directly)
constexpr int32_t TILE_PRES_CHECK = 4;
constexpr int32_t BITMAP_MAX_SW = 5;
// Tensor-core tile: the missing entries of the tile's dense blocks form a 0/1
// mask over K-blocks of 128 permuted columns, [wbeg, wbeg + 128 nsw) with wbeg
// a multiple of 128 (wlen = 0: no staged window).  The row kernel multiplies
// the mask by the base-16 digits of the fixed-point (sin, cos) of those
// columns on the tensor cores.  Bits at bitmap[bm_off ...] in blocks of
// 128 rows x 128 columns, block (kb, m) at (kb * nM + m) * 512 words with
// nM = ceil((r1 - r0) / 128); row r of the block is 4 words, bit c & 31 of
// word c >> 5 for column wbeg + 128 kb + c, tile row 128 m + r.
constexpr int32_t TILE_TC = 8;
// Finite-valued adjacency (PlanInput::val): every listed entry is packed as
// column | (weight + 128) << 24, the weight being A_ml - v_IJ for the
// exceptions of a dense block of value v_IJ and A_ml for a sparse block's
// entries (padding: column n, weight 0); both parts are added with their
// weights.  No window shortcuts, no tensor cores, no bitmaps.
constexpr int32_t TILE_VALUED = 16;
constexpr int32_t VALUED_MAX = 127;             // values 1..127
constexpr int64_t VALUED_MAX_N = (int64_t(1) << 24) - 2;
inline int32_t valued_pack(int64_t col, int32_t w) { return int32_t(uint32_t(col) | (uint32_t(w + 128) << 24)); }
constexpr int32_t TC_KBLOCK = 128;      // columns per K-block
constexpr int32_t TC_MBLOCK = 128;      // rows per M-block (tensor-core tile height)

// Rows are cut into sub-rows of at most SUBROW_MAX entries (missing entries
// first, then present entries, in the row's order), so that one warp holds a
// whole sub-row's indices in registers (4 int4 per lane).
constexpr int32_t SUBROW_MAX = 508;

// A row group: consecutive sub-rows of one tile (at most GROUP_MAX_SUB of
// them) whose packed stream fits one shared-memory slot of the row kernel.
// Packed layout at gstream[off, off + len) (int32 units, 16-byte aligned):
//   nsub x int4 header {miss_rel, n_miss, pres_rel, n_pres} (offsets relative
//   to off), then per sub-row its missing entries followed directly by its
//   present entries (pres_rel = miss_rel + round_up4(n_miss)), each part
//   padded to a multiple of 4 with the index of a zero (sin, cos) entry:
//   n for present parts; for missing parts wbeg - 1 in TILE_MISS_IN_WINDOW
//   tiles, else n.
constexpr int32_t GROUP_MAX_SUB = 16;
// With 8-byte table entries (mixed precision), a group of short sub-rows (each
// at most SHORT_SUB_INTS stream ints: one int4 per lane) may hold up to
// GROUP_MAX_SUB_SHORT of them: then every consumer warp takes two (j and
// j + GROUP_MAX_SUB) and gathers both at once.
constexpr int32_t GROUP_MAX_SUB_SHORT = 32;
constexpr int32_t SHORT_SUB_INTS = 128;
struct Group {
    int64_t off;
    int32_t len;
    int32_t sub0;          // global index of the group's first sub-row
    int32_t nsub;
    int32_t pad;
};

struct PlanInput {
    int64_t n = 0;
    const int64_t* row_ptr = nullptr;   // [n+1]
    const int32_t* col = nullptr;       // [nnz], strictly increasing per row
    const int32_t* label = nullptr;     // [n] in [0, n_comm)
    int32_t n_comm = 0;
    double tau = 0.5;                   // dense iff zero fraction < tau
    int32_t window_cap = 4096;          // max staged window entries per tile
    int64_t tile_work = 0;              // target entries per tile (0: automatic)
    // SM count of the GPU the plan is for: the automatic tile work aims at
    // about 12 tiles per SM (the host-only plan builder assumes GB300's 152)
    int32_t n_sms = 152;
    int32_t tile_max_rows = 512;
    int32_t tile_max_sub = 768;         // sub-rows per tile (stash capacity of the row kernel)
    int32_t slot_ints = 4096;           // capacity of one row-group slot (int32 units)
    // bitmap encoding for a community's dense blocks when its zero fraction
    // there exceeds this (and the window holds every dense column); < 0: never
    double bitmap_zmin = -1.0;
    int32_t entry_bytes = 8;            // (sin, cos) table entry size of the row kernel: 8 or 16
    // values of the listed edges (1..VALUED_MAX, parallel to col); null: a 0/1 matrix
    const int32_t* val = nullptr;
    // tensor-core mask encoding of a community's dense blocks (TILE_TC):
    // 0 never, 1 when its mask bits take fewer bytes than its index lists,
    // 2 whenever the window holds every dense column
    int32_t tensor_cores = 1;
};

struct Plan {
    int64_t n = 0;
    int32_t n_comm = 0;
    double tau = 0.5;
    int64_t nnz_in = 0, self_loops = 0;
    std::vector<int32_t> perm;          // perm[new] = old (stable sort by label)
    std::vector<int32_t> inv_perm;      // inv_perm[old] = new
    std::vector<int64_t> comm_off;      // [n_comm+1] community boundaries (permuted order)
    std::vector<int32_t> node_comm;     // [n] community of each permuted node
    std::vector<int32_t> deg;           // [n] degree without self-loops (permuted order)
    std::vector<int64_t> dptr;          // [n_comm+1] dense column blocks of each row block
    std::vector<int32_t> dcol;
    std::vector<int32_t> dval;          // value of each dense block (1 for a 0/1 matrix)
    bool valued = false;                // finite-valued matrix (TILE_VALUED streams)
    int32_t max_weight = 1;             // largest |weight| of a listed entry or block value
    // per-row counts, sub-rows and the packed group stream (see Group)
    std::vector<int32_t> miss_cnt, pres_cnt;
    std::vector<int32_t> row_sub0;      // [n+1] global index of each row's first sub-row
    std::vector<int32_t> gstream;       // permuted global column indices + headers
    std::vector<Group> groups;
    std::vector<Tile> tiles;
    std::vector<int64_t> sub_hdr;       // [n_sub] position of each sub-row's header in gstream
    std::vector<int64_t> sub_mpos, sub_ppos;   // [n_sub] positions of its missing / present segments
    std::vector<uint32_t> bitmap;              // row bitmaps of TILE_BITMAP tiles, mask bits of TILE_TC tiles
    std::vector<int32_t> row_tile;             // [n] tile of each row
    int64_t bitmap_rows = 0;
    int64_t tc_tiles = 0, tc_rows = 0, tc_mask_bits = 0;   // tensor-core tiles, their rows and mask bits
    int32_t max_wlen = 0;
    // statistics
    int64_t dense_blocks = 0, sparse_blocks = 0, nonempty_blocks = 0;
    int64_t miss_total = 0, pres_total = 0;
    int64_t max_row_entries = 0;
};

// Validates the CSR and labels and builds the plan.  Returns 0, or 1 with a
// message for invalid input, 2 for allocation failure.
int build_plan(const PlanInput& in, Plan& out, std::string& err);

}  // namespace kura
