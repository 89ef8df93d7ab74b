// Batched sampling kernel (kernel (a) over many integrals).  One persistent
// kernel per group of a batch (same integrand, dimension in 1..8 or 9..16): its warps pop work
// units of the group's integrals from an atomic queue, find the unit's
// integral by binary search in the group's prefix sums and run the unit
// exactly as the single-integral kernel would (same unit decomposition, same
// sample loop compiled for the integral's dimension, same order of
// summation, partial sums written to the integral's own slots), so every
// integral's result equals its single-integral result bit for bit.
#pragma once

#include "eval_kernel.cuh"
#include "zmc_internal.h"

namespace zmc {

// CTAs per SM the batched kernel's register allocation must allow.  In the
// FP32 modes one fewer than the single kernel: an integral's Philox round
// keys are loaded into registers per unit (the single kernel takes them from
// the constant bank as kernel parameters).
// FP32 kernels keep 80 registers (3 CTAs per SM) except the oscillatory
// family's, which, like the single kernel's, runs faster at up to 128 (2 CTAs
// per SM: -1.2% time on the 512-integral batch's oscillatory group); the
// other families measured slower there (they spill more as the compiler
// unrolls further).
template <int MODE, int FN = -1>
constexpr int batch_min_blocks() {
    return MODE == ZMC_FP64 ? eval_min_blocks<MODE>() : (FN == kGenzOsc ? 2 : 3);
}
static_assert(kBatchThreads == kEvalMaxThreads, "shared slices are sized for kEvalMaxThreads");

template <int MODE, int FN, bool HI>
__global__ void __launch_bounds__(kBatchThreads, batch_min_blocks<MODE, FN>())
zmc_batch_eval(const BatchEval* __restrict__ items, int count, int level,
               const int64_t* __restrict__ offsets, unsigned long long* head) {
    using R = typename ModeTraits<MODE>::R;
    using R2 = typename ModeTraits<MODE>::R2;
    __shared__ R2 s_coef[kEvalMaxWarps][ZMC_MAX_DIM];
    __shared__ double s_term[kEvalMaxWarps][ZMC_MAX_DIM];
    __shared__ R s_pb[kEvalMaxWarps][ZMC_MAX_DIM];
    __shared__ R s_c[kEvalMaxWarps][4];
    __shared__ double2 s_acc[MODE == ZMC_FP32_FP64ACC ? kBatchThreads : 1];
    __shared__ R s_lane_beta[kEvalMaxWarps][(HI ? 16 : 8) * 32];   // lane tiles' betas

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t total = offsets[count];
    double2* slot = &s_acc[MODE == ZMC_FP32_FP64ACC ? tid : 0];
    R2* wc = s_coef[warp];
    double* wt = s_term[warp];
    R* wp = s_pb[warp];
    R* wcst = s_c[warp];
    for (;;) {
        unsigned long long mine = 0ull;
        if (lane == 0) mine = atomicAdd(head, 1ull);
        const int64_t u = (int64_t)__shfl_sync(0xFFFFFFFFu, mine, 0);
        if (u >= total) break;
        int lo = 0, hi = count;          // the integral i with offsets[i] <= u < offsets[i+1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (offsets[mid] <= u) lo = mid;
            else hi = mid;
        }
        const BatchEval& it = items[lo];
        const Desc& D = *it.desc;
        const UnitPlan plan = it.st->uplan[level];
        const int64_t local = u - offsets[lo];
        if (lane < D.d) wp[lane] = (R)D.pb[lane];
        if (lane < 4) wcst[lane] = (R)D.c[lane];
        const PhiloxKeys keys = it.keys;
        if (plan.lane_tiles) {
            __syncwarp();
#define ZMC_LANE_CASE(DD)                                                                     \
    case DD:                                                                                  \
        lane_tile_unit<MODE, FN, DD>(D, level, plan, local, it.parents[level & 1], keys, wc,  \
                                     s_lane_beta[warp], wp, wcst, slot, it.sums, it.st);      \
        break;
            if constexpr (HI) {
                switch (D.d) {
                    ZMC_LANE_CASE(9) ZMC_LANE_CASE(10) ZMC_LANE_CASE(11) ZMC_LANE_CASE(12)
                    ZMC_LANE_CASE(13) ZMC_LANE_CASE(14) ZMC_LANE_CASE(15) ZMC_LANE_CASE(16)
                    default: break;
                }
            } else {
                switch (D.d) {
                    ZMC_LANE_CASE(1) ZMC_LANE_CASE(2) ZMC_LANE_CASE(3) ZMC_LANE_CASE(4)
                    ZMC_LANE_CASE(5) ZMC_LANE_CASE(6) ZMC_LANE_CASE(7) ZMC_LANE_CASE(8)
                    default: break;
                }
            }
#undef ZMC_LANE_CASE
            __syncwarp();   // the warp's shared slices are rewritten by its next unit
            continue;
        }
        const Unit un = unit_of(plan, local);
        const R start = fold_setup<MODE, FN>(D, level, un.q, it.parents[level & 1], wc, wt, it.st);
        const StreamConst sc = stream_const(keys, un.t, (uint32_t)un.q, (uint32_t)level);
        SumsFor<MODE, FN> acc(slot, value_scale<MODE, FN>(D));
#define ZMC_BATCH_CASE(DD)                                                                    \
    case DD:                                                                                  \
        sample_unit_fold<MODE, FN, DD>(acc, keys, sc, wc, wp, wcst, start, un.g0, un.g1, \
                                             plan.ngroups - 1, plan.tail);                     \
        break;
        if constexpr (HI) {
            switch (D.d) {
                ZMC_BATCH_CASE(9) ZMC_BATCH_CASE(10) ZMC_BATCH_CASE(11) ZMC_BATCH_CASE(12)
                ZMC_BATCH_CASE(13) ZMC_BATCH_CASE(14) ZMC_BATCH_CASE(15) ZMC_BATCH_CASE(16)
                default: break;
            }
        } else {
            switch (D.d) {
                ZMC_BATCH_CASE(1) ZMC_BATCH_CASE(2) ZMC_BATCH_CASE(3) ZMC_BATCH_CASE(4)
                ZMC_BATCH_CASE(5) ZMC_BATCH_CASE(6) ZMC_BATCH_CASE(7) ZMC_BATCH_CASE(8)
                default: break;
            }
        }
#undef ZMC_BATCH_CASE
        if (in_bounds(it.st, local, cap_partial_sums(D), kSiteUnitSum))
            acc.reduce_store(it.sums + local);
        __syncwarp();   // the warp's shared slices are rewritten by its next unit
    }
}

// One mode's batched instantiations, compiled in the same four parts as the
// single-integral kernels (eval_kernel_pair): part p holds integrands 2p and
// 2p + 1, each as a kernel for d in 1..8 and one for d in 9..16.
template <int MODE, int FN>
inline const void* batch_kernel_dims(int d) {
    return d > 8 ? (const void*)zmc_batch_eval<MODE, FN, true>
                 : (const void*)zmc_batch_eval<MODE, FN, false>;
}
template <int MODE, int PART>
inline const void* batch_kernel_pair(int fn, int d) {
    constexpr int F0 = 2 * PART, F1 = 2 * PART + 1;
    if constexpr (in_build<F0>()) {
        if (fn == F0) return batch_kernel_dims<MODE, F0>(d);
    }
    if constexpr (in_build<F1>()) {
        if (fn == F1) return batch_kernel_dims<MODE, F1>(d);
    }
    return nullptr;
}

}  // namespace zmc
