// Memory layout shared by the host code and every kernel of libzmc,
// including the kernels compiled at run time for expression integrands
// (hence no CUDA runtime header here).  Not part of the public ABI.
#pragma once

#ifndef __CUDACC_RTC__
#include <stdint.h>
#endif
#include "../../include/zmc.h"

namespace zmc {

constexpr int kMaxParams = 2 * ZMC_MAX_DIM + 2;

// Integrand registry ids (the order is internal to the CUDA path).
enum Integrand : int32_t {
    kConstant = 0,
    kLinear = 1,
    kSinSum = 2,
    kGaussNorm = 3,
    kGenzOsc = 4,
    kGenzProdPeak = 5,
    kGenzGauss = 6,
    kGenzCorner = 7,
    kNumIntegrands = 8,
    kExpression = 100,
};

// Work units of the sampling kernel, and therefore the order in which each
// (cell, trial) sum is added up: a (cell, trial) tile is cut into `chunks`
// units of about equal numbers of point groups so that a level has at least
// target_units units when it can, but no unit has fewer than
// min_unit_groups groups ("samples per thread": a lane takes one group in
// 32 of its unit; a group is 4 points in FP64, 11 in the FP32 modes).  Lane tiles: a unit of 32 consecutive tiles, each lane one
// whole tile, in place of one tile per warp (which leaves lanes idle on small
// tiles and pays a per-tile set-up and FP64 warp reduction); taken for tiles
// of fewer than lane_tile_groups point groups always, and for tiles of fewer
// than lane_tile_max_groups groups when the level has at least
// lane_tile_min_tiles tiles, enough units of 32 to keep every warp busy.
// The registry kernels use lane tiles; expression kernels keep one tile per
// warp.  Everything is a function of the plan, the level's tile count and n,
// never of the GPU or the launch shape.  The field order is that of
// zmc_result::work_plan.
struct WorkPlan {
    int64_t target_units;
    int64_t min_unit_groups;
    int64_t lane_tile_groups;
    int64_t lane_tile_max_groups;
    int64_t lane_tile_min_tiles;
};
static_assert(sizeof(WorkPlan) == ZMC_PLAN_FIELDS * 8, "WorkPlan is the result's work_plan");

// Everything the kernels need to know about one integration, uploaded to
// device memory before each run.  Plain old data, host-computed.
struct Desc {
    int32_t d, k, T, depth;
    int32_t integrand, mode;
    int64_t n;                       // points per (cell, trial)
    int64_t K;                       // k^d children per split cell
    int64_t kpow[ZMC_MAX_DIM];       // k^i
    uint32_t key[2];                 // Philox key = (seed lo, seed hi)
    double m;                        // sigma multiplier
    int64_t max_cells, max_samples;  // refinement budget
    int64_t cap_cells;               // capacity of the per-level buffers
    double lo[ZMC_MAX_DIM];
    double width[ZMC_MAX_DEPTH + 1][ZMC_MAX_DIM];  // (hi - lo) / k^L
    double volume[ZMC_MAX_DEPTH + 1];              // prod_i width[L][i]
    // Per-dimension integrand parameters (pa, pb) and scalars (c[0..3]),
    // rearranged on the host from the user's parameter list.
    double pa[ZMC_MAX_DIM], pb[ZMC_MAX_DIM];
    double c[4];
    WorkPlan plan;                   // work decomposition of the sampling kernel
};

// Work decomposition of one level under the run's work plan: computed once,
// by the kernel that sets the level's cell count (level_plan below), and read
// by the sampling and statistics kernels.
struct UnitPlan {
    int64_t units, chunks, tiles;  // chunks: unit slots per tile (1 for lane tiles)
    uint32_t ngroups, tail;        // point groups per tile; real points of the last
    int32_t T, lane_tiles;         // trials; a unit is 32 tiles, one per lane
};

// Tree state of one run, written only by the kernels.  Index L = level.
struct State {
    int64_t cells[ZMC_MAX_DEPTH + 2];
    int64_t flagged[ZMC_MAX_DEPTH + 2];
    double mu[ZMC_MAX_DEPTH + 2];
    double sigma[ZMC_MAX_DEPTH + 2];
    double theta[ZMC_MAX_DEPTH + 2];
    double min_margin[ZMC_MAX_DEPTH + 2];
    int32_t refine[ZMC_MAX_DEPTH + 2];
    int64_t samples;
    int32_t status;      // ZMC_OK or a ZMC_ERR_* code
    int32_t levels_run;
    uint32_t ticket[4];  // last-block arrival counters (self-resetting)
    uint32_t check_site; // bounds-guarded build: first failing check (0: none)
    UnitPlan uplan[ZMC_MAX_DEPTH + 2];            // work decomposition per level
    unsigned long long queue[ZMC_MAX_DEPTH + 2];  // sampling units taken per level
};



// The default plan; target_units is also the most any plan may ask for (the
// partial-sum buffer is sized for it).
constexpr int64_t kTargetUnits = int64_t(1) << 18;
constexpr WorkPlan kDefaultPlan = {kTargetUnits, 1024, 64, 1024, int64_t(1) << 18};

// A point "group" of the mode's stream: four points from one Philox block
// per dimension (FP64: its 32-bit words) or eleven from a pair of blocks
// (FP32 modes: 23-bit fields, see zmc_device.cuh).
#ifdef __CUDACC__
__host__ __device__
#endif
inline int points_per_group(int mode) { return mode == ZMC_FP64 ? 4 : 11; }
#ifdef __CUDACC__
__host__ __device__
#endif
inline int blocks_per_group(int mode) { return mode == ZMC_FP64 ? 1 : 2; }

#ifdef __CUDACC__
__host__ __device__
#endif
inline int64_t groups_of(int64_t n, int mode) {
    const int G = points_per_group(mode);
    return (n + G - 1) / G;
}

// Capacities of a handle's per-level buffers, in elements: unit partial
// sums (a level of `tiles` tiles has at most tiles + target_units <=
// tiles + kTargetUnits units), cell statistics, and each parent list
// (flagged cells x d coordinates).
#ifdef __CUDACC__
__host__ __device__
#endif
inline int64_t cap_partial_sums(const Desc& D) { return D.cap_cells * D.T + kTargetUnits; }
#ifdef __CUDACC__
__host__ __device__
#endif
inline int64_t cap_parents(const Desc& D) { return (D.cap_cells / D.K + 1) * D.d; }

#ifdef __CUDACC__
__host__ __device__
#endif
inline int64_t unit_chunks(int64_t tiles, int64_t ngroups, const WorkPlan& w) {
    if (tiles <= 0) return 1;
    int64_t want = (w.target_units + tiles - 1) / tiles;
    int64_t most = ngroups / w.min_unit_groups;
    if (most < 1) most = 1;
    return want < most ? (want < 1 ? 1 : want) : most;
}

#ifdef __CUDACC__
__host__ __device__
#endif
inline bool lane_tiles(int64_t tiles, int64_t ngroups, const WorkPlan& w) {
    return ngroups < w.lane_tile_groups ||
           (ngroups < w.lane_tile_max_groups && tiles >= w.lane_tile_min_tiles);
}

// Work units of a level of `tiles` tiles of `ngroups` groups each.
#ifdef __CUDACC__
__host__ __device__
#endif
inline int64_t level_units(int64_t tiles, int64_t ngroups, bool allow_lane_tiles,
                           const WorkPlan& w) {
    if (allow_lane_tiles && lane_tiles(tiles, ngroups, w)) return (tiles + 31) / 32;
    return tiles * unit_chunks(tiles, ngroups, w);
}

// The work decomposition of a level of C cells.  Lane tiles write one slot
// per tile, so their chunk count is 1 whatever unit_chunks says; registry
// integrands may use lane tiles, expressions never do.
#ifdef __CUDACC__
__host__ __device__
#endif
inline UnitPlan level_plan(const Desc& D, int64_t C) {
    UnitPlan p;
    p.T = D.T;
    p.ngroups = (uint32_t)groups_of(D.n, D.mode);           // < 2^32: n * d < 2^34
    p.tail = (uint32_t)(D.n - (int64_t)points_per_group(D.mode) * (int64_t)(p.ngroups - 1));
    p.tiles = C * D.T;
    const bool allow = D.integrand != kExpression;
    p.lane_tiles = (allow && lane_tiles(p.tiles, p.ngroups, D.plan)) ? 1 : 0;
    p.chunks = p.lane_tiles ? 1 : unit_chunks(p.tiles, p.ngroups, D.plan);
    p.units = level_units(p.tiles, p.ngroups, allow, D.plan);
    return p;
}

}  // namespace zmc
