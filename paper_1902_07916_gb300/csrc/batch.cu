// Batched integration: many independent integrals (uneven dimension, cell
// count and depth) advance one tree level at a time.  Per level:
//   1. zmc_batch_plan: each integral's number of sampling units at this level
//      (from its own tree state) and their exclusive prefix sum;
//   2. zmc_batch_eval: ONE persistent kernel over the units of all integrals.
//      Each warp pops the next unit from an atomic queue, finds its integral
//      by binary search in the prefix sums and runs it exactly as the
//      single-integral kernel would (same unit decomposition, same order of
//      summation, partial sums written to the integral's own slots), so every
//      integral's result equals its single-integral result bit for bit;
//   3. the selection kernels with one grid row (blockIdx.y) per integral.
// The host captures each level into a CUDA graph once and replays it.
#include "eval_kernel.cuh"
#include "zmc_internal.h"

namespace zmc {

// Batched-kernel register cap: per-integral Philox keys live in registers.
constexpr int kBatchMinBlocks = 3;

__global__ void zmc_batch_plan(const BatchEval* __restrict__ items, int count, int level,
                               int64_t* __restrict__ offsets, unsigned long long* head) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const Desc& D = *items[i].desc;
        const int64_t C = items[i].st->cells[level];
        int64_t units = 0;
        if (C > 0) {
            const int64_t tiles = C * D.T;
            units = tiles * unit_chunks(tiles, groups_of(D.n, D.mode));
        }
        offsets[i + 1] = units;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        offsets[0] = 0;
        for (int i = 0; i < count; ++i) offsets[i + 1] += offsets[i];
        *head = 0ull;
    }
}

template <int MODE, int FN, bool WIDE>
__device__ __forceinline__ void batch_unit(LaneSums<MODE>& acc, const Desc& D, int level,
                                           const Unit& un, const UnitPlan& plan,
                                           const uint32_t* parents, const PhiloxKeys& keys,
                                           typename ModeTraits<MODE>::R2* w_coef, double* w_term,
                                           const typename ModeTraits<MODE>::R* w_pb,
                                           const typename ModeTraits<MODE>::R* w_c) {
    const typename ModeTraits<MODE>::R start =
        fold_setup<MODE, FN>(D, level, un.q, parents, w_coef, w_term);
    const StreamConst sc = stream_const(keys, un.t, (uint32_t)un.q, (uint32_t)level);
    sample_unit_fold<MODE, FN, WIDE, 0>(acc, keys, sc, w_coef, w_pb, w_c, start, un.g0, un.g1,
                                        plan.ngroups - 1, plan.tail, D.d);
}

template <int MODE>
__global__ void __launch_bounds__(kEvalMaxThreads, kBatchMinBlocks)
zmc_batch_eval(const BatchEval* __restrict__ items, int count, int level,
               const int64_t* __restrict__ offsets, unsigned long long* head) {
    using R = typename ModeTraits<MODE>::R;
    using R2 = typename ModeTraits<MODE>::R2;
    __shared__ R2 s_coef[kEvalMaxWarps][ZMC_MAX_DIM];
    __shared__ double s_term[kEvalMaxWarps][ZMC_MAX_DIM];
    __shared__ R s_pb[kEvalMaxWarps][ZMC_MAX_DIM];
    __shared__ R s_c[kEvalMaxWarps][4];
    __shared__ double2 s_acc[MODE == ZMC_FP32_FP64ACC ? kEvalMaxThreads : 1];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t total = offsets[count];
    double2* slot = &s_acc[MODE == ZMC_FP32_FP64ACC ? tid : 0];
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
        const UnitPlan plan = unit_plan<MODE>(D, it.st->cells[level]);
        const int64_t local = u - offsets[lo];
        const Unit un = unit_of(plan, local);
        if (lane < D.d) s_pb[warp][lane] = (R)D.pb[lane];
        if (lane < 4) s_c[warp][lane] = (R)D.c[lane];
        const PhiloxKeys keys = it.keys;
        const uint32_t* parents = it.parents[level & 1];
        LaneSums<MODE> acc(slot);
        R2* wc = s_coef[warp];
        double* wt = s_term[warp];
        const R* wp = s_pb[warp];
        const R* wcst = s_c[warp];
        switch (it.fn) {
        case kConstant:
            batch_unit<MODE, kConstant, false>(acc, D, level, un, plan, parents, keys, wc, wt, wp, wcst);
            break;
        case kLinear:
            batch_unit<MODE, kLinear, false>(acc, D, level, un, plan, parents, keys, wc, wt, wp, wcst);
            break;
        case kSinSum:
            if (it.wide) batch_unit<MODE, kSinSum, true>(acc, D, level, un, plan, parents, keys, wc, wt, wp, wcst);
            else batch_unit<MODE, kSinSum, false>(acc, D, level, un, plan, parents, keys, wc, wt, wp, wcst);
            break;
        case kGaussNorm:
            batch_unit<MODE, kGaussNorm, false>(acc, D, level, un, plan, parents, keys, wc, wt, wp, wcst);
            break;
        case kGenzOsc:
            if (it.wide) batch_unit<MODE, kGenzOsc, true>(acc, D, level, un, plan, parents, keys, wc, wt, wp, wcst);
            else batch_unit<MODE, kGenzOsc, false>(acc, D, level, un, plan, parents, keys, wc, wt, wp, wcst);
            break;
        case kGenzProdPeak:
            batch_unit<MODE, kGenzProdPeak, false>(acc, D, level, un, plan, parents, keys, wc, wt, wp, wcst);
            break;
        case kGenzGauss:
            batch_unit<MODE, kGenzGauss, false>(acc, D, level, un, plan, parents, keys, wc, wt, wp, wcst);
            break;
        case kGenzCorner:
            batch_unit<MODE, kGenzCorner, false>(acc, D, level, un, plan, parents, keys, wc, wt, wp, wcst);
            break;
        default:
            break;
        }
        acc.reduce_store(it.sums + local);
        __syncwarp();   // the warp's shared slices are rewritten by its next unit
    }
}

const void* batch_eval_kernel(int mode) {
    switch (mode) {
    case ZMC_FP64: return (const void*)zmc_batch_eval<ZMC_FP64>;
    case ZMC_FP32_FP64ACC: return (const void*)zmc_batch_eval<ZMC_FP32_FP64ACC>;
    default: return (const void*)zmc_batch_eval<ZMC_FP32_KAHAN>;
    }
}

cudaError_t launch_batch_level(const BatchEval* items, int count, int level, int64_t* offsets,
                               unsigned long long* head, int mode, int grid, cudaStream_t s) {
    zmc_batch_plan<<<1, 256, 0, s>>>(items, count, level, offsets, head);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&items, (void*)&count, (void*)&level, (void*)&offsets, (void*)&head};
    return cudaLaunchKernel(batch_eval_kernel(mode), dim3(grid), dim3(kBatchThreads), args, 0, s);
}

}  // namespace zmc
