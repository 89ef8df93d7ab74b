// Kernel (a): the fused sample-generate / evaluate / reduce kernel.
//
// Work is cut into units by the descriptor's work plan.  Usually a unit is a
// contiguous range of the point groups of one (cell, trial) tile
// (unit_chunks() units per tile); for small tiles on large levels
// (lane_tiles()) a unit is 32 consecutive whole tiles, one per lane.  Every warp takes its first unit by its index and the rest
// from the level's atomic counter; the level's cell count is read from device
// memory, so the host never needs it.  Per unit of one tile:
//   1. lanes < d decode the cell's lattice coordinates from the slot index
//      (level 1: base-k digits; deeper: parent coordinates * k + child digit)
//      and fold the cell's geometry into the integrand's per-dimension
//      coefficients, in the warp's slice of shared memory;
//   2. every lane takes groups of G consecutive samples (G = 4 in FP64, 11 in
//      the FP32 modes); for each dimension one Philox4x32-10 block (FP64,
//      counter (g*d + i, t, q, L): four 32-bit words) or a pair of blocks
//      (FP32, counters 2(g*d + i) and 2(g*d + i) + 1: eleven 23-bit fields)
//      gives that dimension's coordinate for all G samples (Sec. 2.2: random
//      numbers are produced where they are used, nothing is stored);
//   3. f and f^2 are summed per lane, then across the warp with shuffles, and
//      lane 0 writes the unit's (S1, S2) to the partial-sum array.  The
//      statistics kernel adds a tile's units in a fixed order.
// A lane-tile unit does 1-3 per lane for its own tile and writes the tile's
// sums without a warp reduction (lane_tile_unit).
// No CTA-wide barrier is involved, and the summation order depends on n, d,
// the level's size and the work plan (WorkPlan, in the descriptor) only --
// not on the CTA size or grid chosen to run it.
//
// There is one kernel per dimension d in 1..16 and the dimension loop is
// unrolled, so the Philox chains of successive dimensions interleave.
// Registry integrands fold each coordinate into G independent accumulators
// as it is produced; expression integrands (compiled at run time, d fixed)
// keep the G points' coordinates in registers and evaluate the expression on
// each.
//
// MODE 0: FP64 throughout.  MODE 1: FP32 points and integrand, FP32 partial
// sums over 8 groups (88 points) flushed into FP64 per-lane sums, FP64 warp
// reduction.  MODE 2: FP32 points and integrand with TwoSum-compensated
// per-lane sums and a TwoSum warp reduction; the (sum, error) float pair is
// widened to FP64 only for the stored result.  The Gaussian integrands run
// in the log2 domain in MODE 1 and 2 (LogLaneSums).
#pragma once

#include "zmc_device.cuh"

namespace zmc {

constexpr int kEvalMaxThreads = 256;
constexpr int kEvalMaxWarps = kEvalMaxThreads / 32;
// CTAs of kEvalMaxThreads per SM the register allocation must allow: 3
// caps registers at 85 (80 used).  The FP32 kernels of the sine of a sum and
// of the oscillatory Genz family (a cosine of a linear sum) take 2 (up to 128
// registers, no spills, 16 warps per SM): measured 0.6-1.0% faster on the
// sine workloads and up to 1.7% on the oscillatory ones, while the
// corner-peak and Gaussian kernels lost 0.3-0.95% that way and keep 3.
// Expression kernels use the mode's value.
template <int MODE>
constexpr int eval_min_blocks() { return 3; }
template <int MODE, int FN>
constexpr int eval_min_blocks_fn() {
    return (MODE != ZMC_FP64 && (FN == kSinSum || FN == kGenzOsc)) ? 2 : eval_min_blocks<MODE>();
}
// The dimension loop of a point group (group_values) is unrolled 8-way,
// which covers d <= 8 completely; for d = 9..16 the FP32 modes unroll it
// completely, since the remainder iteration of an 8-way unroll cost 2-4%.
// FP64 keeps 8: its library exp and sin would spill under a full unroll.
constexpr int kFlushGroups = 8;   // groups per FP32 partial sum (MODE 1): 88 points

template <int MODE>
struct ModeTraits {
    using R = float;
    using R2 = float2;
};
template <>
struct ModeTraits<ZMC_FP64> {
    using R = double;
    using R2 = double2;
};

// Points per group of the mode's stream (4 or 11) and Philox blocks per
// group and dimension (1 or 2).
template <int MODE>
constexpr int kGroup = MODE == ZMC_FP64 ? 4 : 11;
template <int MODE>
constexpr int kBlocks = MODE == ZMC_FP64 ? 1 : 2;

// The G assembled 1.m values of one group and dimension: the four 32-bit
// words of block w (FP64 stream), or the eleven 23-bit fields of the pair
// (w, w2) (FP32 stream; w2 is unused in FP64).
template <int MODE>
__device__ __forceinline__ void block_points(uint4 w, uint4 w2,
                                             typename ModeTraits<MODE>::R (&v)[kGroup<MODE>]) {
    if constexpr (MODE == ZMC_FP64) {
        v[0] = one_plus_word_f64(w.x);
        v[1] = one_plus_word_f64(w.y);
        v[2] = one_plus_word_f64(w.z);
        v[3] = one_plus_word_f64(w.w);
    } else {
        fields_1m(w, v[0], v[1], v[2], v[3], v[4]);
        fields_1m(w2, v[5], v[6], v[7], v[8], v[9]);
        v[10] = cross_1m(w, w2);
    }
}

// Sum and sum of squares of a group's eleven FP32 values, as a balanced tree.
__device__ __forceinline__ void group_sums(const float (&f)[11], float& g1, float& g2) {
    g1 = (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7]))) +
         ((f[8] + f[9]) + f[10]);
    const float q0 = fmaf(f[0], f[0], f[1] * f[1]), q1 = fmaf(f[2], f[2], f[3] * f[3]);
    const float q2 = fmaf(f[4], f[4], f[5] * f[5]), q3 = fmaf(f[6], f[6], f[7] * f[7]);
    const float q4 = fmaf(f[8], f[8], f[9] * f[9]);
    g2 = ((q0 + q1) + (q2 + q3)) + fmaf(f[10], f[10], q4);
}

// Per-lane running sums of f and f^2 in the mode's arithmetic.  MODE 1 keeps
// its FP64 sums in the lane's shared-memory slot (touched once per 88
// points), so they hold no registers in the sampling loop.
template <int MODE>
struct LaneSums {
    float s1 = 0.f, e1 = 0.f, s2 = 0.f, e2 = 0.f;  // MODE 1 partials / MODE 2 (sum, err)
    double S1d = 0.0, S2d = 0.0;                   // MODE 0
    double2* slot;                                 // MODE 1

    __device__ __forceinline__ explicit LaneSums(double2* s, double = 1.0) : slot(s) {
        if constexpr (MODE == ZMC_FP32_FP64ACC) *slot = make_double2(0.0, 0.0);
    }

    // One group's values: four (FP64) or eleven (FP32) points.
    template <typename R>
    __device__ __forceinline__ void add(const R (&f)[kGroup<MODE>]) {
        if constexpr (MODE == ZMC_FP64) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                S1d += f[j];
                S2d = fma(f[j], f[j], S2d);
            }
        } else {
            float g1, g2;
            group_sums(f, g1, g2);
            if constexpr (MODE == ZMC_FP32_FP64ACC) {
                s1 += g1;
                s2 += g2;
            } else {
                float t, r;
                two_sum(s1, g1, t, r); s1 = t; e1 += r;
                two_sum(s2, g2, t, r); s2 = t; e2 += r;
            }
        }
    }

    // End of a chunk of kFlushGroups groups: MODE 1 moves its FP32 partials
    // into the FP64 sums.
    __device__ __forceinline__ void flush() {
        if constexpr (MODE == ZMC_FP32_FP64ACC) {
            double2 v = *slot;
            v.x += (double)s1;
            v.y += (double)s2;
            *slot = v;
            s1 = 0.f; s2 = 0.f;
        }
    }

    // Warp reduction; lane 0 writes the unit's (S1, S2).
    __device__ __forceinline__ void reduce_store(double2* out) {
        double a, b;
        if constexpr (MODE == ZMC_FP64) {
            a = warp_sum(S1d);
            b = warp_sum(S2d);
        } else if constexpr (MODE == ZMC_FP32_FP64ACC) {
            const double2 v = *slot;
            a = warp_sum(v.x);
            b = warp_sum(v.y);
        } else {
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const float os1 = __shfl_xor_sync(0xFFFFFFFFu, s1, o);
                const float oe1 = __shfl_xor_sync(0xFFFFFFFFu, e1, o);
                const float os2 = __shfl_xor_sync(0xFFFFFFFFu, s2, o);
                const float oe2 = __shfl_xor_sync(0xFFFFFFFFu, e2, o);
                float t, r;
                two_sum(s1, os1, t, r); s1 = t; e1 = e1 + oe1 + r;
                two_sum(s2, os2, t, r); s2 = t; e2 = e2 + oe2 + r;
            }
            a = (double)s1 + (double)e1;
            b = (double)s2 + (double)e2;
        }
        if ((threadIdx.x & 31) == 0) *out = make_double2(a, b);
    }

    // This lane's own sums (a tile run by one lane): no warp reduction.
    __device__ __forceinline__ void store_lane(double2* out) {
        if constexpr (MODE == ZMC_FP64) *out = make_double2(S1d, S2d);
        else if constexpr (MODE == ZMC_FP32_FP64ACC) *out = *slot;
        else *out = make_double2((double)s1 + (double)e1, (double)s2 + (double)e2);
    }
};

// FP32 modes for integrands of the form C * 2^t (the Gaussians): the group
// delivers t = log2(f / C) and the lane sums 2^(t - k) and 2^(2 (t - k)) in
// FP32, k an integer reference exponent that follows the largest t the lane
// has seen (a rebase scales the partial sums by an exact power of two).  The
// values keep FP32's relative precision whatever their magnitude, so a cell
// whose values all lie below FP32's range (1e-38) still has a spread, as in
// FP64.  MODE 1 moves its partials into absolute FP64 sums (ldexp by k, 2k)
// every kFlushGroups groups; MODE 2 keeps (sum, error) pairs per lane and
// brings the warp to its largest k before the compensated reduction.  C
// (FP64) multiplies the unit's sums at the end.
__device__ __forceinline__ float neg_inf() { return __int_as_float((int)0xff800000u); }

template <int MODE>
struct LogLaneSums {
    float k = neg_inf();                          // reference exponent (an integer)
    float s1 = 0.f, e1 = 0.f, s2 = 0.f, e2 = 0.f;
    double2* slot;                                // MODE 1
    double scale;                                 // C

    __device__ __forceinline__ LogLaneSums(double2* s, double c) : slot(s), scale(c) {
        if constexpr (MODE == ZMC_FP32_FP64ACC) *slot = make_double2(0.0, 0.0);
    }

    // Scale the partial sums from reference k to kn >= k: 2^(k - kn), exact
    // (or 0 once below FP32's normal range, where they no longer count).
    __device__ __forceinline__ void rebase(float kn) {
        const float d = k - kn;
        const float sc = d < -126.f ? 0.f : __int_as_float(((int)d + 127) << 23);
        const float sc2 = d < -63.f ? 0.f : sc * sc;
        s1 *= sc; e1 *= sc;
        s2 *= sc2; e2 *= sc2;
        k = kn;
    }

    __device__ __forceinline__ void add(const float (&t)[kGroup<MODE>]) {
        float tm = t[0];
#pragma unroll
        for (int j = 1; j < kGroup<MODE>; ++j) tm = fmaxf(tm, t[j]);
        if (tm > k) rebase(ceilf(tm));
        float f[kGroup<MODE>];
#pragma unroll
        for (int j = 0; j < kGroup<MODE>; ++j) f[j] = exp2f(t[j] - k);
        float g1, g2;
        group_sums(f, g1, g2);
        if constexpr (MODE == ZMC_FP32_FP64ACC) {
            s1 += g1;
            s2 += g2;
        } else {
            float a, r;
            two_sum(s1, g1, a, r); s1 = a; e1 += r;
            two_sum(s2, g2, a, r); s2 = a; e2 += r;
        }
    }

    // The exponent for ldexp: FP64 sums vanish below 2^-1074, so clamping k
    // at -4000 changes nothing and keeps the conversion to int in range.
    static __device__ __forceinline__ int exp_of(float k) { return (int)fmaxf(k, -4000.f); }

    __device__ __forceinline__ void flush() {
        if constexpr (MODE == ZMC_FP32_FP64ACC) {
            if (s1 != 0.f || s2 != 0.f) {
                const int ke = exp_of(k);
                double2 v = *slot;
                v.x += ldexp((double)s1, ke);
                v.y += ldexp((double)s2, 2 * ke);
                *slot = v;
            }
            s1 = 0.f; s2 = 0.f;
        }
    }

    __device__ __forceinline__ void reduce_store(double2* out) {
        double a, b;
        if constexpr (MODE == ZMC_FP32_FP64ACC) {
            const double2 v = *slot;
            a = warp_sum(v.x);
            b = warp_sum(v.y);
        } else {
            float km = k;
#pragma unroll
            for (int o = 16; o; o >>= 1) km = fmaxf(km, __shfl_xor_sync(0xFFFFFFFFu, km, o));
            if (km > k) rebase(km);
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const float os1 = __shfl_xor_sync(0xFFFFFFFFu, s1, o);
                const float oe1 = __shfl_xor_sync(0xFFFFFFFFu, e1, o);
                const float os2 = __shfl_xor_sync(0xFFFFFFFFu, s2, o);
                const float oe2 = __shfl_xor_sync(0xFFFFFFFFu, e2, o);
                float t, r;
                two_sum(s1, os1, t, r); s1 = t; e1 = e1 + oe1 + r;
                two_sum(s2, os2, t, r); s2 = t; e2 = e2 + oe2 + r;
            }
            const int ke = exp_of(km);
            a = (km == neg_inf()) ? 0.0 : ldexp((double)s1 + (double)e1, ke);
            b = (km == neg_inf()) ? 0.0 : ldexp((double)s2 + (double)e2, 2 * ke);
        }
        if ((threadIdx.x & 31) == 0) *out = make_double2(a * scale, b * (scale * scale));
    }

    __device__ __forceinline__ void store_lane(double2* out) {
        double a, b;
        if constexpr (MODE == ZMC_FP32_FP64ACC) {
            const double2 v = *slot;
            a = v.x;
            b = v.y;
        } else {
            const int ke = exp_of(k);
            a = (k == neg_inf()) ? 0.0 : ldexp((double)s1 + (double)e1, ke);
            b = (k == neg_inf()) ? 0.0 : ldexp((double)s2 + (double)e2, 2 * ke);
        }
        *out = make_double2(a * scale, b * (scale * scale));
    }
};

// The lane accumulator of integrand FN in mode MODE.
template <bool B, class T, class F> struct pick_type { using type = T; };
template <class T, class F> struct pick_type<false, T, F> { using type = F; };
template <int MODE, int FN>
constexpr bool log_domain() { return MODE != ZMC_FP64 && Fn<FN, float>::kLog2; }
template <int MODE, int FN>
using SumsFor = typename pick_type<log_domain<MODE, FN>(), LogLaneSums<MODE>, LaneSums<MODE>>::type;
template <int MODE, int FN>
__device__ __forceinline__ double value_scale(const Desc& D) {
    if constexpr (log_domain<MODE, FN>()) return Fn<FN, float>::value_scale(D);
    else return 1.0;
}

// Mask the points past n in the tile's last group (only it can be short):
// `tail` is the number of real points of that group, 1..G; they become
// `fill` (0, or -inf for a log2-domain group).
template <typename R, int G>
__device__ __forceinline__ void mask_tail(bool last, uint32_t tail, R (&f)[G], R fill = R(0)) {
    if (last) {
#pragma unroll
        for (int j = 1; j < G; ++j)
            if ((uint32_t)j >= tail) f[j] = fill;
    }
}

// Distribution of a level's units over the warps of the sampling kernel:
// a warp's first unit is its global warp index, every further one comes
// from the level's counter in the tree state (one atomic per unit of at
// least the plan's min_unit_groups point groups).  A unit's sums do not depend on which warp runs it, so the
// results are the same under any order; the queue keeps every warp busy up
// to the level's last unit, where a fixed stride leaves the warps that the
// schedulers favoured idle at the end.
struct UnitQueue {
    unsigned long long* head;
    int64_t nwarps;
    __device__ __forceinline__ UnitQueue(State* st, int level)
        : head(&st->queue[level]), nwarps((int64_t)gridDim.x * (blockDim.x >> 5)) {}
    __device__ __forceinline__ int64_t first() const {
        return (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    }
    __device__ __forceinline__ int64_t next() const {
        unsigned long long mine = 0ull;
        if ((threadIdx.x & 31) == 0) mine = atomicAdd(head, 1ull);
        return nwarps + (int64_t)__shfl_sync(0xFFFFFFFFu, mine, 0);
    }
};

// Unit u -> (slot q, trial t, group range [g0, g1)).
struct Unit {
    int64_t q;
    uint32_t t, g0, g1;
};

__device__ __forceinline__ Unit unit_of(const UnitPlan& p, int64_t u) {
    Unit r;
    const int64_t tile = u / p.chunks;
    const int64_t chunk = u - tile * p.chunks;
    r.q = tile / p.T;
    r.t = (uint32_t)(tile - r.q * p.T);
    r.g0 = (uint32_t)(chunk * p.ngroups / p.chunks);
    r.g1 = (uint32_t)((chunk + 1) * p.ngroups / p.chunks);
    return r;
}

// The cell's shift b_i = lo_i + c_i w_L - s w_L, where s turns the assembled
// 1.m value into the uniform (1 - 2^-33 in FP64, 1 - 2^-24 in FP32), so that
// the point is x_i = w_L * 1.m + b_i = lo_i + (c_i + u) w_L.
template <int MODE>
__device__ __forceinline__ double cell_shift(const Desc& D, int level, int64_t q, int i,
                                             const uint32_t* parents, double w, const State* st) {
    const double s = (MODE == ZMC_FP64) ? 1.0 - 0x1p-33 : 1.0 - 0x1p-24;
    const int64_t c = cell_coord(D, level, q, i, parents, st);
    return D.lo[i] + (double)c * w - s * w;
}

// Per-unit set-up of a registry integrand (lanes < d, then a warp barrier):
// each dimension's fold coefficients (alpha, beta) from the cell's width and
// shift (see Fn), and the fold's start value init + sum_i term_i (FP64,
// rounded once).
template <int MODE, int FN>
__device__ __forceinline__ typename ModeTraits<MODE>::R fold_setup(
    const Desc& D, int level, int64_t q, const uint32_t* parents,
    typename ModeTraits<MODE>::R2* w_coef, double* w_term, const State* st) {
    using R = typename ModeTraits<MODE>::R;
    using F = Fn<FN, R>;
    const int lane = threadIdx.x & 31;
    if (lane < D.d) {
        const double w = D.width[level][lane];
        const double b = cell_shift<MODE>(D, level, q, lane, parents, w, st);
        const Prep p = F::prep(w, b, D.pa[lane], D.pb[lane]);
        w_coef[lane].x = (R)p.alpha;
        w_coef[lane].y = (R)p.beta;
        w_term[lane] = p.term;
    }
    __syncwarp();
    double a0 = (double)F::init();
    for (int i = 0; i < D.d; ++i) a0 += w_term[i];
    return (R)a0;
}

// Where group_values finds dimension i's fold coefficients (alpha, beta):
// one pair per dimension for the whole warp (a unit of one tile), or the
// warp's alpha with this lane's own beta (lane tiles: beta carries the
// cell's position, alpha only the level's width).
template <typename R, typename R2>
struct WarpCoef {
    const R2* ab;
    __device__ __forceinline__ R2 operator()(int i) const { return ab[i]; }
};
template <typename R, typename R2>
struct LaneCoef {
    const R2* ab;     // [d], the warp's (alpha, unused)
    const R* beta;    // [d * 32], this lane's at beta[i * 32]
    __device__ __forceinline__ R2 operator()(int i) const {
        R2 r = ab[i];
        r.y = beta[i * 32];
        return r;
    }
};

// FP64 sine of a sum with one width in every dimension (a cube domain): the
// argument start + sum_i alpha (1 + w_i 2^-32) is (start + alpha d) +
// (alpha 2^-32) S with S = sum_i w_i, an exact 64-bit integer sum of the
// Philox words (< 2^36), so a point needs one FP64 add (S to double through
// its bits) and one FMA instead of d FMAs.  GB300 runs FP64 at two
// operations per SM per clock and the integer ALU is idle in this mode.
// `on` is decided per unit from the fold coefficients' bits.
struct EqFold {
    bool on;
    double al32, c0;
};
template <int MODE, int FN>
__device__ __forceinline__ EqFold eq_fold(const typename ModeTraits<MODE>::R2* ab, int nd,
                                          typename ModeTraits<MODE>::R start) {
    EqFold e{false, 0.0, 0.0};
    if constexpr (MODE == ZMC_FP64 && FN == kSinSum) {
        const long long a0 = __double_as_longlong(ab[0].x);
        bool same = true;
        for (int i = 1; i < nd; ++i) same = same && __double_as_longlong(ab[i].x) == a0;
        if (same) e = EqFold{true, ab[0].x * 0x1p-32, fma(ab[0].x, (double)nd, start)};
    }
    return e;
}

// The values of one point group (G points) of a registry integrand: the
// Philox block (FP64) or pair of blocks (FP32) of every dimension (round 1's
// product A * c0 given as P, the 64-bit product for the group's first block),
// each folded into the G running sums, then the finishing function.
template <int MODE, int FN, int DIM, class Coef>
__device__ __forceinline__ void group_values(
    const PhiloxKeys& keys, const StreamConst& sc, const Coef& coef,
    const typename ModeTraits<MODE>::R* s_pb,
    const typename ModeTraits<MODE>::R* s_c, typename ModeTraits<MODE>::R start, uint64_t P,
    int nd, typename ModeTraits<MODE>::R (&f)[kGroup<MODE>], const EqFold& eq = EqFold{}) {
    using R = typename ModeTraits<MODE>::R;
    using R2 = typename ModeTraits<MODE>::R2;
    using F = Fn<FN, R>;
    constexpr int G = kGroup<MODE>;
    if constexpr (MODE == ZMC_FP64 && FN == kSinSum) {
        if (eq.on) {
            unsigned long long S[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll 8
            for (int i = 0; i < nd; ++i) {
                const uint4 w = philox_from_product(keys, sc, (uint32_t)(P >> 32), (uint32_t)P);
                P += kPhiloxMulA;
                S[0] += w.x;
                S[1] += w.y;
                S[2] += w.z;
                S[3] += w.w;
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const double s = __longlong_as_double(0x4330000000000000LL | (long long)S[p]) -
                                 0x1p52;
                f[p] = F::finish(fma(eq.al32, s, eq.c0), s_c, nd);
            }
            return;
        }
    }
    R a[G];
#pragma unroll
    for (int p = 0; p < G; ++p) a[p] = start;
    auto dimension = [&](int i) {
        const uint4 w = philox_from_product(keys, sc, (uint32_t)(P >> 32), (uint32_t)P);
        P += kPhiloxMulA;
        uint4 w2 = w;
        if constexpr (MODE != ZMC_FP64) {
            w2 = philox_from_product(keys, sc, (uint32_t)(P >> 32), (uint32_t)P);
            P += kPhiloxMulA;
        }
        const R2 ab = coef(i);
        const R pb = s_pb[i];
        R v[G];
        block_points<MODE>(w, w2, v);
#pragma unroll
        for (int p = 0; p < G; ++p) a[p] = F::fold(a[p], v[p], ab.x, ab.y, pb);
    };
    if constexpr (MODE != ZMC_FP64 && DIM > 8) {
#pragma unroll
        for (int i = 0; i < DIM; ++i) dimension(i);
    } else {
#pragma unroll 8
        for (int i = 0; i < nd; ++i) dimension(i);
    }
    if constexpr (log_domain<MODE, FN>()) {
#pragma unroll
        for (int p = 0; p < G; ++p) f[p] = F::finish_log2(a[p], s_c);
    } else {
#pragma unroll
        for (int p = 0; p < G; ++p) f[p] = F::finish(a[p], s_c, nd);
    }
}

// The sample loop of one unit for a registry integrand, dimension DIM (a
// compile-time constant, or 0 to take the dimension from dim_rt).
// Round 1's product A * c0 is carried as a 64-bit running sum: c0 =
// B*(g*d + i) + b for the b-th of the B blocks of dimension i (B = 1 in FP64,
// 2 in FP32) grows by one per block and by 32*B*d per group of this lane.  Only the
// tile's last group can hold points past n; it is left out of the main loop
// and run, masked, by the one lane it falls to in the unit that holds it.
template <int MODE, int FN, int DIM>
__device__ __forceinline__ void sample_unit_fold(
    SumsFor<MODE, FN>& acc, const PhiloxKeys& keys, const StreamConst& sc,
    const typename ModeTraits<MODE>::R2* w_coef, const typename ModeTraits<MODE>::R* s_pb,
    const typename ModeTraits<MODE>::R* s_c, typename ModeTraits<MODE>::R start,
    uint32_t g0, uint32_t g1, uint32_t last_group, uint32_t tail, int dim_rt = 0) {
    using R = typename ModeTraits<MODE>::R;
    using R2 = typename ModeTraits<MODE>::R2;
    const int nd = DIM > 0 ? DIM : dim_rt;
    constexpr uint32_t B = kBlocks<MODE>;
    const uint64_t step = (uint64_t)kPhiloxMulA * (uint64_t)(32 * B * nd);
    uint32_t g = g0 + (threadIdx.x & 31);
    uint64_t Pg = (uint64_t)kPhiloxMulA * (uint64_t)(g * B * nd);
    constexpr int G = kGroup<MODE>;
    const EqFold eq = eq_fold<MODE, FN>(w_coef, nd, start);
    const uint32_t full_end = g1 <= last_group ? g1 : last_group;
    while (g < full_end) {
        for (int j = 0; j < kFlushGroups && g < full_end; ++j, g += 32, Pg += step) {
            R f[G];
            group_values<MODE, FN, DIM>(keys, sc, WarpCoef<R, R2>{w_coef}, s_pb, s_c, start, Pg,
                                        nd, f, eq);
            acc.add(f);
        }
        acc.flush();
    }
    if (g == last_group && g < g1) {
        R f[G];
        group_values<MODE, FN, DIM>(keys, sc, WarpCoef<R, R2>{w_coef}, s_pb, s_c, start, Pg, nd,
                                    f, eq);
        mask_tail(true, tail, f, log_domain<MODE, FN>() ? R(neg_inf()) : R(0));
        acc.add(f);
        acc.flush();
    }
}

// A unit of 32 small tiles, one per lane (plan.lane_tiles): each lane sets up
// its own cell (the same FP64 fold coefficients and start value as
// fold_setup), runs all of its tile's groups in order and writes the tile's
// sums itself -- no warp reduction.  The level's alpha per dimension goes to
// w_coef[i].x (equal for every lane, lanes < d write it), the lane's beta to
// lane_beta[i * 32 + lane].  Ends with the warp converged.
template <int MODE, int FN, int DIM>
__device__ __forceinline__ void lane_tile_unit(
    const Desc& D, int level, const UnitPlan& plan, int64_t u, const uint32_t* parents,
    const PhiloxKeys& keys, typename ModeTraits<MODE>::R2* w_coef,
    typename ModeTraits<MODE>::R* lane_beta,
    const typename ModeTraits<MODE>::R* s_pb, const typename ModeTraits<MODE>::R* s_c,
    double2* slot, double2* partial, const State* st) {
    using R = typename ModeTraits<MODE>::R;
    using R2 = typename ModeTraits<MODE>::R2;
    using F = Fn<FN, R>;
    constexpr int G = kGroup<MODE>;
    const int lane = threadIdx.x & 31;
    const int64_t tile = u * 32 + lane;
    const bool active = tile < plan.tiles;
    const int64_t q = active ? tile / plan.T : 0;
    const uint32_t t = active ? (uint32_t)(tile - q * plan.T) : 0u;
    double a0 = (double)F::init();
    for (int i = 0; i < DIM; ++i) {
        const double w = D.width[level][i];
        const double b = active ? cell_shift<MODE>(D, level, q, i, parents, w, st) : 0.0;
        const Prep p = F::prep(w, b, D.pa[i], D.pb[i]);
        if (lane == i) w_coef[i].x = (R)p.alpha;
        lane_beta[i * 32 + lane] = (R)p.beta;
        a0 += p.term;
    }
    __syncwarp();
    if (!active) return;
    const R start = (R)a0;
    const LaneCoef<R, R2> coef{w_coef, lane_beta + lane};
    const EqFold eq = eq_fold<MODE, FN>(w_coef, DIM, start);
    const StreamConst sc = stream_const(keys, t, (uint32_t)q, (uint32_t)level);
    SumsFor<MODE, FN> acc(slot, value_scale<MODE, FN>(D));
    const uint64_t step = (uint64_t)kPhiloxMulA * (uint64_t)(DIM * kBlocks<MODE>);
    const uint32_t last = plan.ngroups - 1;
    uint64_t Pg = 0;
    uint32_t g = 0;
    while (g < last) {
        for (int j = 0; j < kFlushGroups && g < last; ++j, ++g, Pg += step) {
            R f[G];
            group_values<MODE, FN, DIM>(keys, sc, coef, s_pb, s_c, start, Pg, DIM, f, eq);
            acc.add(f);
        }
        acc.flush();
    }
    R f[G];
    group_values<MODE, FN, DIM>(keys, sc, coef, s_pb, s_c, start, Pg, DIM, f, eq);
    mask_tail(true, plan.tail, f, log_domain<MODE, FN>() ? R(neg_inf()) : R(0));
    acc.add(f);
    acc.flush();
    if (in_bounds(st, tile, cap_partial_sums(D), kSiteLaneSum)) acc.store_lane(partial + tile);
}

// One kernel per dimension DIM: each holds only the sample loop its d needs.
template <int MODE, int FN, int DIM>
__global__ void __launch_bounds__(kEvalMaxThreads, eval_min_blocks_fn<MODE, FN>())
zmc_eval_reduce(const Desc* __restrict__ desc, State* st,
                const uint32_t* __restrict__ parents, double2* __restrict__ partial,
                int level, const PhiloxKeys keys) {
    using R = typename ModeTraits<MODE>::R;
    using R2 = typename ModeTraits<MODE>::R2;
    __shared__ R2 s_coef[kEvalMaxWarps][ZMC_MAX_DIM];
    __shared__ double s_term[kEvalMaxWarps][ZMC_MAX_DIM];
    __shared__ R s_pb[ZMC_MAX_DIM], s_c[4];
    __shared__ double2 s_acc[MODE == ZMC_FP32_FP64ACC ? kEvalMaxThreads : 1];
    __shared__ R s_lane_beta[kEvalMaxWarps][DIM * 32];

    const Desc& D = *desc;
    const int64_t C = st->cells[level];
    if (C <= 0) return;
    const int d = D.d;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid < d) s_pb[tid] = (R)D.pb[tid];
    if (tid < 4) s_c[tid] = (R)D.c[tid];
    __syncthreads();

    const UnitPlan plan = st->uplan[level];
    const UnitQueue queue(st, level);
    double2* slot = &s_acc[MODE == ZMC_FP32_FP64ACC ? tid : 0];
    for (int64_t u = queue.first(); u < plan.units; u = queue.next()) {
        if (plan.lane_tiles) {
            lane_tile_unit<MODE, FN, DIM>(D, level, plan, u, parents, keys, s_coef[warp],
                                          s_lane_beta[warp], s_pb, s_c, slot, partial, st);
            __syncwarp();
            continue;
        }
        const Unit un = unit_of(plan, u);
        const R start =
            fold_setup<MODE, FN>(D, level, un.q, parents, s_coef[warp], s_term[warp], st);
        const StreamConst sc = stream_const(keys, un.t, (uint32_t)un.q, (uint32_t)level);
        SumsFor<MODE, FN> acc(slot, value_scale<MODE, FN>(D));
        sample_unit_fold<MODE, FN, DIM>(acc, keys, sc, s_coef[warp], s_pb, s_c, start, un.g0,
                                        un.g1, plan.ngroups - 1, plan.tail);
        if (in_bounds(st, u, cap_partial_sums(D), kSiteUnitSum)) acc.reduce_store(partial + u);
        __syncwarp();   // the warp's coefficient slice is rewritten by the next unit
    }
}

// Body of the kernel for an expression integrand E with dimension DIM known
// at compile time: E::eval(x, p) reads x[0..DIM-1] and the parameters p[].
template <int MODE, int DIM, class E>
__device__ __forceinline__ void eval_expr_body(const Desc* __restrict__ desc,
                                               State* st,
                                               const uint32_t* __restrict__ parents,
                                               double2* __restrict__ partial, int level,
                                               const PhiloxKeys& keys) {
    using R = typename ModeTraits<MODE>::R;
    using R2 = typename ModeTraits<MODE>::R2;
    __shared__ R2 s_wb[kEvalMaxWarps][ZMC_MAX_DIM];
    __shared__ R s_p[2 * ZMC_MAX_DIM + 4];
    __shared__ double2 s_acc[MODE == ZMC_FP32_FP64ACC ? kEvalMaxThreads : 1];

    const Desc& D = *desc;
    const int64_t C = st->cells[level];
    if (C <= 0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < ZMC_MAX_DIM) {
        s_p[tid] = (R)D.pa[tid];
        s_p[ZMC_MAX_DIM + tid] = (R)D.pb[tid];
    }
    if (tid < 4) s_p[2 * ZMC_MAX_DIM + tid] = (R)D.c[tid];
    __syncthreads();

    const UnitPlan plan = st->uplan[level];
    const UnitQueue queue(st, level);
    double2* slot = &s_acc[MODE == ZMC_FP32_FP64ACC ? tid : 0];
    R2* wb = s_wb[warp];
    constexpr int G = kGroup<MODE>;
    for (int64_t u = queue.first(); u < plan.units; u = queue.next()) {
        const Unit un = unit_of(plan, u);
        if (lane < DIM) {
            const double w = D.width[level][lane];
            wb[lane].x = (R)w;
            wb[lane].y = (R)cell_shift<MODE>(D, level, un.q, lane, parents, w, st);
        }
        __syncwarp();
        const StreamConst sc = stream_const(keys, un.t, (uint32_t)un.q, (uint32_t)level);
        LaneSums<MODE> acc(slot);
        // the G points of group gg: coordinates from the blocks, then E.  An
        // FP32 group is evaluated in two halves (points 0..4 from each
        // dimension's first block, then 5..10 from its second block and the
        // pair's cross field), so only six points' coordinates are live.
        auto values = [&](uint32_t gg, R (&f)[G]) {
            if constexpr (MODE == ZMC_FP64) {
                R x[G][DIM];
                const uint32_t cbase = gg * DIM;
#pragma unroll
                for (int i = 0; i < DIM; ++i) {
                    const uint4 w = philox_stream(keys, sc, cbase + i);
                    const R2 c = wb[i];
                    R v[G];
                    block_points<MODE>(w, w, v);
#pragma unroll
                    for (int p = 0; p < G; ++p) x[p][i] = fma(v[p], c.x, c.y);
                }
#pragma unroll
                for (int p = 0; p < G; ++p) f[p] = E::eval(x[p], s_p);
            } else {
                R x[6][DIM];
                uint4 first[DIM];
                const uint32_t cbase = 2 * gg * DIM;
#pragma unroll
                for (int i = 0; i < DIM; ++i) {
                    first[i] = philox_stream(keys, sc, cbase + 2 * i);
                    const R2 c = wb[i];
                    R v[5];
                    fields_1m(first[i], v[0], v[1], v[2], v[3], v[4]);
#pragma unroll
                    for (int p = 0; p < 5; ++p) x[p][i] = fma(v[p], c.x, c.y);
                }
#pragma unroll
                for (int p = 0; p < 5; ++p) f[p] = E::eval(x[p], s_p);
#pragma unroll
                for (int i = 0; i < DIM; ++i) {
                    const uint4 w2 = philox_stream(keys, sc, cbase + 2 * i + 1);
                    const R2 c = wb[i];
                    R v[6];
                    fields_1m(w2, v[0], v[1], v[2], v[3], v[4]);
                    v[5] = cross_1m(first[i], w2);
#pragma unroll
                    for (int p = 0; p < 6; ++p) x[p][i] = fma(v[p], c.x, c.y);
                }
#pragma unroll
                for (int p = 0; p < 6; ++p) f[5 + p] = E::eval(x[p], s_p);
            }
        };
        // as in sample_unit_fold: the tile's last group, the only one that
        // can run past n, is left to the one lane it falls to
        const uint32_t last = plan.ngroups - 1;
        const uint32_t full_end = un.g1 <= last ? un.g1 : last;
        uint32_t g = un.g0 + lane;
        while (g < full_end) {
            for (int j = 0; j < kFlushGroups && g < full_end; ++j, g += 32) {
                R f[G];
                values(g, f);
                acc.add(f);
            }
            acc.flush();
        }
        if (g == last && g < un.g1) {
            R f[G];
            values(g, f);
            mask_tail(true, plan.tail, f);
            acc.add(f);
            acc.flush();
        }
        if (in_bounds(st, u, cap_partial_sums(D), kSiteUnitSum)) acc.reduce_store(partial + u);
        __syncwarp();
    }
}

#ifndef __CUDACC_RTC__
// One mode's registry instantiations, indexed by integrand id and dimension.
template <int MODE, int FN>
inline const void* eval_kernel_dim(int d) {
    switch (d) {
    case 1: return (const void*)zmc_eval_reduce<MODE, FN, 1>;
    case 2: return (const void*)zmc_eval_reduce<MODE, FN, 2>;
    case 3: return (const void*)zmc_eval_reduce<MODE, FN, 3>;
    case 4: return (const void*)zmc_eval_reduce<MODE, FN, 4>;
    case 5: return (const void*)zmc_eval_reduce<MODE, FN, 5>;
    case 6: return (const void*)zmc_eval_reduce<MODE, FN, 6>;
    case 7: return (const void*)zmc_eval_reduce<MODE, FN, 7>;
    case 8: return (const void*)zmc_eval_reduce<MODE, FN, 8>;
    case 9: return (const void*)zmc_eval_reduce<MODE, FN, 9>;
    case 10: return (const void*)zmc_eval_reduce<MODE, FN, 10>;
    case 11: return (const void*)zmc_eval_reduce<MODE, FN, 11>;
    case 12: return (const void*)zmc_eval_reduce<MODE, FN, 12>;
    case 13: return (const void*)zmc_eval_reduce<MODE, FN, 13>;
    case 14: return (const void*)zmc_eval_reduce<MODE, FN, 14>;
    case 15: return (const void*)zmc_eval_reduce<MODE, FN, 15>;
    case 16: return (const void*)zmc_eval_reduce<MODE, FN, 16>;
    default: return nullptr;
    }
}
// The registry kernels of one precision mode are compiled in four parts,
// translation units that the build generates (build.py): part p holds
// integrands 2p and 2p + 1 of the registry order, so the parts compile in
// parallel.  The bounds-guarded test build compiles sin_sum and genz_corner
// only.
template <int FN>
constexpr bool in_build() {
#ifdef ZMC_CHECKED
    return FN == kSinSum || FN == kGenzCorner;
#else
    return true;
#endif
}
template <int MODE, int PART>
inline const void* eval_kernel_pair(int fn, int d) {
    constexpr int F0 = 2 * PART, F1 = 2 * PART + 1;
    if constexpr (in_build<F0>()) {
        if (fn == F0) return eval_kernel_dim<MODE, F0>(d);
    }
    if constexpr (in_build<F1>()) {
        if (fn == F1) return eval_kernel_dim<MODE, F1>(d);
    }
    return nullptr;
}
#endif

}  // namespace zmc
