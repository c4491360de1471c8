// pr_internal.cuh -- device-side layout and helpers shared by the library's
// translation units (graph build, solver).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>

#include "../../include/pr.h"

namespace pr {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
pr_status fail(pr_status st, const std::string &msg);
pr_status cuda_fail(cudaError_t e, const char *what);

#define PR_CK(...)                                                      \
    do {                                                                \
        cudaError_t _e = (__VA_ARGS__);                                 \
        if (_e != cudaSuccess) return ::pr::cuda_fail(_e, #__VA_ARGS__); \
    } while (0)

#define PR_TRY(...)                                                     \
    do {                                                                \
        pr_status _s = (__VA_ARGS__);                                   \
        if (_s != PR_OK) return _s;                                     \
    } while (0)

// ---------------------------------------------------------------- memory
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, size_t bytes, cudaStream_t s);

// A device buffer owned by the library (allocator hook aware).
struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    pr_free_fn ffn = nullptr;  // allocator hook that made p (nullptr: cudaMalloc)
    void *fctx = nullptr;
    bool stream_ordered = false;  // made by alloc_async: freed with cudaFreeAsync on s
    pr_status alloc(size_t nbytes, cudaStream_t stream);
    // cudaMallocAsync on `stream` (from `pool` when given), never the allocator
    // hook: for the server's own thread, which must not call back into the host
    // program
    pr_status alloc_async(size_t nbytes, cudaStream_t stream, cudaMemPool_t pool = nullptr);
    void release();
    template <typename T> T *as() const { return static_cast<T *>(p); }
    void swap(Buf &o) noexcept {
        std::swap(p, o.p);
        std::swap(bytes, o.bytes);
        std::swap(s, o.s);
        std::swap(ffn, o.ffn);
        std::swap(fctx, o.fctx);
        std::swap(stream_ordered, o.stream_ordered);
    }
    ~Buf() { release(); }
    Buf() = default;
    Buf(const Buf &) = delete;
    Buf &operator=(const Buf &) = delete;
};

// ---------------------------------------------------------------- graph
// Vertex renumbering: internal ids are ordered by class and, inside a class,
// by total in-degree (descending):
//   [0, n_ref)      non-dangling with in-edges   ("referenced")
//   [n_ref, n_nd)   non-dangling without in-edges ("unreferenced", Sec. 2.1)
//   [n_nd, n)       dangling (deg = 0)
// Out-lists are sorted by target, so the targets < n_nd (non-dangling) form
// a prefix of length ndeg[i]: the IFP2 valid edges.  In-lists are split into
// two segments: sources < n_ref ("ref") and sources in [n_ref, n_nd)
// ("unref", which can only push while their residual is not yet spent).
struct DevGraph {
    int32_t n, n_nd, n_ref;
    int64_t m, m_ref, m_unref;
    const int32_t *out_off;   // [n+1]
    const int32_t *out_dst;   // [m]
    const int32_t *ndeg;      // [n_nd]
    const double *inv_deg64;  // [n_nd] 1/deg
    const float *inv_deg32;   // [n_nd]
    const float2 *inv_degdf;  // [n_nd] 1/deg as a double-float pair (hi, lo)
    const int32_t *inr_off;   // [n+1]
    const int32_t *inr_src;   // [m_ref]
    const int32_t *inu_off;   // [n+1]
    const int32_t *inu_src;   // [m_unref]
    const int32_t *perm;      // [n] internal -> caller id
    const int32_t *inv;       // [n] caller id -> internal
    const int32_t *gs_back;   // [n_nd] level-ordered graphs: valid out-edges into the row's own or a lower level
    const int32_t *tile_row;  // first row of every gather tile (short-row ranges), see Seg::t0
};

// Row ranges of a gather kernel, by work-group size.  Rows inside each
// class are sorted by in-degree, so each bin is a contiguous range.  A
// segment's rows are processed by groups of `lanes` threads (1..32, a power
// of two; 0 = the whole block per row).
struct Seg {
    int32_t lo, hi;   // rows [lo, hi)
    int32_t lanes;    // threads per row; 0 = one block per row; kTileLanes = gather tiles
    int32_t blk0;     // first block of this segment
    int32_t nblk;     // blocks assigned
    int32_t t0, nt;   // gather tiles: rows [tile_row[t0 + k], tile_row[t0 + k + 1]), k < nt
};
// Short rows (in-list length <= kTileDeg) can be gathered by tiles: a block
// loads the pending values of up to kTileE consecutive in-list entries at once
// (independent loads) into shared memory, then each thread sums its rows there.
// A tile is a run of whole rows: row j's units are its entries plus kTileW, and
// tile k holds the rows whose first unit lies in [k U, (k+1) U) for
// U = kTileE - kTileDeg - kTileW, so a tile has at most kTileE entries and
// kTileRows rows.
#ifndef PR_TILE_E
#define PR_TILE_E 1024
#endif
constexpr int kTileLanes = -1;
// Level-ordered rounds serve each row with more than kClusterRowMin in-list
// entries by a cluster of kLevelCluster blocks (lanes = kClusterLanes): one
// level launch is as long as its longest row, and one block takes a 100k-entry
// row through about 50 dependent load steps.
constexpr int kClusterLanes = -2;
constexpr int kLevelCluster = 8;
constexpr int kClusterRowMin = 16384;
// and rows above kLevelBlockRowMin entries get a whole block there, whatever
// the tuned block-row threshold (a warp takes a 16k-entry row through 64 steps)
constexpr int kLevelBlockRowMin = 4096;
#ifndef PR_LEVEL_ROUND_BLOCKS
#define PR_LEVEL_ROUND_BLOCKS 16384
#endif
constexpr int kLevelRoundBlocks = PR_LEVEL_ROUND_BLOCKS;  // lane-bin blocks of one level-ordered round, all launches
constexpr int kTileE = PR_TILE_E;
constexpr int kTileDeg = 64;
constexpr int kTileW = 2;
constexpr int kTileU = kTileE - kTileDeg - kTileW;
constexpr int kTileRows = kTileU / kTileW + 1;
constexpr int kMaxSeg = 128;   // levels x 7 bins + the unreferenced rows + 7 dangling bins
constexpr int kMaxLevels = 16;  // levels of level-ordered rounds
struct Plan {
    Seg seg[kMaxSeg];
    int32_t nseg;
    int32_t nblocks;
};

constexpr int kThreads = 256;       // block size of every row/vertex kernel
constexpr int kMaxBlocks = 32768;   // partial-sum slots of a reduction (>= any grid; one level-ordered round shares them)
constexpr int kWarpRowMin = 32;     // push bins: out-degree above which a vertex gets a warp
constexpr int kCtaRowMin = 4096;    // push bins: out-degree above which a vertex gets a CTA
// Pull bins (in-degree d): d > thr[0] block per row; thr[k] < d <= thr[k-1]
// gets 32 >> (k-1) lanes; d <= thr[5] one lane.
constexpr int kNumThr = 6;
constexpr int32_t kDefaultThr[kNumThr] = {4096, 64, 32, 16, 8, 4};

}  // namespace pr

// The opaque ABI handle.
struct pr_graph {
    uint64_t uid = 0;  // process-unique serial number (caches keyed by graph use it, not the address)
    // bumped whenever the pull plans change (set_bins): captured CUDA graphs and
    // tile tables hold plans by value and are rebuilt when it moves
    uint64_t plan_gen = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    pr::DevGraph G{};
    pr_graph_info info{};
    // storage
    pr::Buf out_off, out_dst, ndeg, inv_deg64, inv_deg32, inv_degdf, inr_off, inr_src, inu_off, inu_src,
        perm, inv;
    // pull bins: row boundaries of the in-degree sorted classes and the in-list
    // entries in front of each boundary (ref + unref segments)
    int32_t thr[pr::kNumThr] = {};
    // Bin ranges: the referenced class (one range, or one per level), then the
    // dangling class; each range sorted by in-degree, split at 6 bounds.
    // ranges[k] = {lo, hi}; bounds[6k..6k+5]; edges at lo, bounds, hi.
    int32_t nranges = 0;
    int32_t range_lo[pr::kMaxLevels + 1] = {}, range_hi[pr::kMaxLevels + 1] = {};
    int32_t bounds[(pr::kMaxLevels + 1) * pr::kNumThr] = {};
    long long range_edges[(pr::kMaxLevels + 1) * (pr::kNumThr + 2)] = {};
    int32_t block_budget = 0;
    // level-ordered rounds (pr_graph_opts.levels): the referenced class is cut
    // into `levels` contiguous row ranges [level_lo[l], level_lo[l+1])
    int32_t levels = 0;
    int32_t level_lo[pr::kMaxLevels + 1] = {};
    int32_t cl_hi[pr::kMaxLevels + 1] = {};  // per level: rows [level_lo, cl_hi) are served by block clusters
    int32_t lb_hi[pr::kMaxLevels + 1] = {};  // per level: rows above kLevelBlockRowMin entries end here
    pr::Buf gs_back;  // [n_nd] valid out-edges of a row into its own or a lower level
    pr::Plan plan_lvl[pr::kMaxLevels]{}, plan_unref{};
    double pull_ratio = 0.04;  // AUTO push/pull switch used when a solve passes 0
    int64_t scan_nd_ref = 0, scan_nd_unref = 0;  // in-list entries of the non-dangling rows, per segment
    pr::Plan plan_nd{}, plan_d{}, plan_all{};
    // the same rows with the short-row bins replaced by gather tiles (single
    // solves); the batch engine and the server cut plan_nd / plan_d
    pr::Plan plan_nd_t{}, plan_d_t{}, plan_all_t{};
    pr::Buf tile_row;                                        // tile starts of every range, then its end
    int32_t tile_t0[pr::kMaxLevels + 1] = {}, tile_nt[pr::kMaxLevels + 1] = {};  // per range (0 tiles: none)
    int32_t tile_lo[pr::kMaxLevels + 1] = {};                // first row of the range's tiled rows
    // solver workspace (lazily allocated, reused across solves)
    void *ws = nullptr;
};

namespace pr {
void build_plans(pr_graph *g);
// pull bins from in-degree thresholds (non-increasing) and a block budget;
// rebuilds every plan of g (on error g keeps its bins)
pr_status set_bins(pr_graph *g, const int32_t *thr, int32_t budget, cudaStream_t s);
void destroy_workspace(pr_graph *g);
}  // namespace pr
