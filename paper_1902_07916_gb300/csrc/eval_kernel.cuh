// Kernel (a): the fused sample-generate / evaluate / reduce kernel.
//
// One CTA owns one (cell, trial) tile at a time and walks the level's tiles
// persistently (tile += gridDim.x); the number of cells of the level is read
// from device memory, so the host never needs it.  Per tile:
//   1. d threads decode the cell's lattice coordinates from the slot index
//      (level 1: base-k digits; deeper: parent coordinates * k + child digit)
//      into per-dimension (width, shift) pairs in shared memory;
//   2. every thread takes groups of four consecutive samples; for each
//      dimension one Philox4x32-10 block (counter (g*d + i, t, q, L)) gives
//      that dimension's coordinate for all four samples (Sec. 2.2: random
//      numbers are produced where they are used, nothing is stored);
//   3. the values f and f^2 are summed per thread, then across the warp with
//      shuffles and across warps through shared memory, and one thread writes
//      the tile's (S1, S2) as two doubles.
//
// The dimension loop is compiled for every d in 1..16 (a switch picks the
// copy once per tile) and unrolled by four, so up to four Philox chains of
// successive dimensions interleave with little loop control.  Registry
// integrands fold each coordinate into four independent accumulators as it
// is produced; expression integrands (compiled at run time) keep the four
// points' coordinates in registers and evaluate the expression on each.
//
// MODE 0: FP64 throughout.  MODE 1: FP32 points and integrand, FP32 partial
// sums over 16 groups (64 points) flushed into FP64 per-thread sums, FP64
// block reduction.  MODE 2: FP32 points and integrand with TwoSum-compensated
// per-thread sums and a TwoSum block reduction; the (sum, error) float pair
// is widened to FP64 only for the stored result.
#pragma once

#include "zmc_device.cuh"

namespace zmc {

constexpr int kEvalMaxThreads = 256;
// CTAs of kEvalMaxThreads per SM the register allocation must allow: caps
// registers at 42 (FP32 modes) and 85 (FP64, whose values take two).
template <int MODE>
constexpr int eval_min_blocks() { return MODE == ZMC_FP64 ? 3 : 5; }
// Philox chains of successive dimensions in flight per thread.
constexpr int kDimUnroll = 4;
constexpr int kFlushGroups = 16;  // groups per FP32 partial sum (MODE 1)

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

template <int MODE>
__device__ __forceinline__ typename ModeTraits<MODE>::R point(uint32_t w,
                                                            typename ModeTraits<MODE>::R2 wb) {
    if constexpr (MODE == ZMC_FP64) return fma(one_plus_word_f64(w), wb.x, wb.y);
    else return fmaf(one_plus_word_f32(w), wb.x, wb.y);
}

// Per-thread running sums of f and f^2 in the mode's arithmetic.  MODE 1
// keeps its FP64 sums in shared memory (one double2 per thread, touched once
// per 64 points) so they hold no registers in the sampling loop.
template <int MODE>
struct ThreadSums {
    double S1d = 0.0, S2d = 0.0;                   // MODE 0 (MODE 1: at the end only)
    float s1 = 0.f, e1 = 0.f, s2 = 0.f, e2 = 0.f;  // MODE 1 partials / MODE 2 (sum, err)
    double2* slot = nullptr;                       // MODE 1: this thread's FP64 sums

    __device__ __forceinline__ explicit ThreadSums(double2* s_acc) {
        if constexpr (MODE == ZMC_FP32_FP64ACC) {
            slot = s_acc + threadIdx.x;
            *slot = make_double2(0.0, 0.0);
        }
    }

    template <typename R>
    __device__ __forceinline__ void add4(R f0, R f1, R f2, R f3) {
        if constexpr (MODE == ZMC_FP64) {
            S1d += f0; S1d += f1; S1d += f2; S1d += f3;
            S2d = fma(f0, f0, S2d); S2d = fma(f1, f1, S2d);
            S2d = fma(f2, f2, S2d); S2d = fma(f3, f3, S2d);
        } else if constexpr (MODE == ZMC_FP32_FP64ACC) {
            s1 += (f0 + f1) + (f2 + f3);
            s2 += fmaf(f0, f0, f1 * f1) + fmaf(f2, f2, f3 * f3);
        } else {
            float t, r;
            two_sum(s1, (f0 + f1) + (f2 + f3), t, r); s1 = t; e1 += r;
            two_sum(s2, fmaf(f0, f0, f1 * f1) + fmaf(f2, f2, f3 * f3), t, r); s2 = t; e2 += r;
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

    // Block reduction; thread 0 writes the tile's (S1, S2) and flags a
    // non-finite result.  Ends with a barrier so shared memory can be reused.
    __device__ __forceinline__ void reduce_store(double2* sums, int64_t tile, State* st) {
        __shared__ double s_red[32][2];
        __shared__ float s_redf[32][4];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int nwarps = blockDim.x >> 5;
        double a = 0.0, b = 0.0;
        if constexpr (MODE != ZMC_FP32_KAHAN) {
            if constexpr (MODE == ZMC_FP32_FP64ACC) {
                const double2 v = *slot;
                S1d = v.x;
                S2d = v.y;
            }
            S1d = warp_sum(S1d);
            S2d = warp_sum(S2d);
            if (lane == 0) { s_red[warp][0] = S1d; s_red[warp][1] = S2d; }
            __syncthreads();
            if (warp == 0) {
                a = warp_sum(lane < nwarps ? s_red[lane][0] : 0.0);
                b = warp_sum(lane < nwarps ? s_red[lane][1] : 0.0);
            }
        } else {
            merge_pairs();
            if (lane == 0) {
                s_redf[warp][0] = s1; s_redf[warp][1] = e1;
                s_redf[warp][2] = s2; s_redf[warp][3] = e2;
            }
            __syncthreads();
            if (warp == 0) {
                s1 = lane < nwarps ? s_redf[lane][0] : 0.f;
                e1 = lane < nwarps ? s_redf[lane][1] : 0.f;
                s2 = lane < nwarps ? s_redf[lane][2] : 0.f;
                e2 = lane < nwarps ? s_redf[lane][3] : 0.f;
                merge_pairs();
                a = (double)s1 + (double)e1;
                b = (double)s2 + (double)e2;
            }
        }
        if (threadIdx.x == 0) {
            sums[tile] = make_double2(a, b);
            if (!(isfinite(a) && isfinite(b))) atomicMax(&st->status, ZMC_ERR_NONFINITE);
        }
        __syncthreads();
    }

    // Warp-wide TwoSum merge of the (sum, err) pairs: error terms are carried.
    __device__ __forceinline__ void merge_pairs() {
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
    }
};

// Per-tile set-up: the cell's per-dimension (width, shift) pairs.  The shift
// turns the assembled 1.m value into the uniform (1 - 2^-33 in FP64,
// 1 - 2^-24 in FP32), so that point = fma(1.m, w_L, shift) = lo + (c + u) w_L.
template <int MODE>
__device__ __forceinline__ void tile_setup(const Desc& D, int level, int64_t q,
                                           const uint32_t* parents,
                                           typename ModeTraits<MODE>::R2* s_wb) {
    using R = typename ModeTraits<MODE>::R;
    const double shift = (MODE == ZMC_FP64) ? 1.0 - 0x1p-33 : 1.0 - 0x1p-24;
    const int tid = threadIdx.x;
    if (tid < D.d) {
        const double w = D.width[level][tid];
        const int64_t c = cell_coord(D, level, q, tid, parents);
        s_wb[tid].x = (R)w;
        s_wb[tid].y = (R)(D.lo[tid] + (double)c * w - shift * w);
    }
    __syncthreads();
}

// Mask the points past n in the last group (only it can be short): `tail`
// is the number of real points of the last group, 1..4.
template <typename R>
__device__ __forceinline__ void mask_tail(bool last, uint32_t tail, R& f1, R& f2, R& f3) {
    if (last) {
        if (tail < 4) f3 = R(0);
        if (tail < 3) f2 = R(0);
        if (tail < 2) f1 = R(0);
    }
}

// The sample loop of one tile for a registry integrand, dimension DIM.
template <int MODE, int FN, bool WIDE, int DIM>
__device__ __forceinline__ void sample_tile_fold(
    ThreadSums<MODE>& acc, const PhiloxKeys& keys, const StreamConst& sc,
    const typename ModeTraits<MODE>::R2* s_wb, const typename ModeTraits<MODE>::R2* s_ab,
    const typename ModeTraits<MODE>::R* s_c, uint32_t ngroups, uint32_t tail) {
    using R = typename ModeTraits<MODE>::R;
    using R2 = typename ModeTraits<MODE>::R2;
    using F = Fn<FN, R>;
    uint32_t g = threadIdx.x;
    while (g < ngroups) {
        for (int j = 0; j < kFlushGroups && g < ngroups; ++j, g += blockDim.x) {
            R a0 = F::init(), a1 = F::init(), a2 = F::init(), a3 = F::init();
            const uint32_t cbase = g * DIM;
#pragma unroll kDimUnroll
            for (int i = 0; i < DIM; ++i) {
                const uint4 w = philox_stream(keys, sc, cbase + i);
                const R2 wb = s_wb[i];
                const R2 ab = s_ab[i];
                a0 = F::fold(a0, point<MODE>(w.x, wb), ab.x, ab.y);
                a1 = F::fold(a1, point<MODE>(w.y, wb), ab.x, ab.y);
                a2 = F::fold(a2, point<MODE>(w.z, wb), ab.x, ab.y);
                a3 = F::fold(a3, point<MODE>(w.w, wb), ab.x, ab.y);
            }
            R f0 = F::template finish<WIDE>(a0, s_c, DIM), f1 = F::template finish<WIDE>(a1, s_c, DIM);
            R f2 = F::template finish<WIDE>(a2, s_c, DIM), f3 = F::template finish<WIDE>(a3, s_c, DIM);
            mask_tail(g == ngroups - 1, tail, f1, f2, f3);
            acc.add4(f0, f1, f2, f3);
        }
        acc.flush();
    }
}

template <int MODE, int FN, bool WIDE>
__global__ void __launch_bounds__(kEvalMaxThreads, eval_min_blocks<MODE>())
zmc_eval_reduce(const Desc* __restrict__ desc, State* __restrict__ st,
                const uint32_t* __restrict__ parents, double2* __restrict__ sums,
                int level, const PhiloxKeys keys) {
    using R = typename ModeTraits<MODE>::R;
    using R2 = typename ModeTraits<MODE>::R2;
    __shared__ R2 s_wb[ZMC_MAX_DIM], s_ab[ZMC_MAX_DIM];
    __shared__ R s_c[4];
    __shared__ double2 s_acc[MODE == ZMC_FP32_FP64ACC ? kEvalMaxThreads : 1];

    const Desc& D = *desc;
    const int64_t C = st->cells[level];
    if (C <= 0) return;
    const int d = D.d, T = D.T;
    const int64_t n = D.n;
    const int64_t tiles = C * T;
    const uint32_t ngroups = (uint32_t)((n + 3) >> 2);        // < 2^32: n * d < 2^34
    const uint32_t tail = (uint32_t)(n - 4 * (int64_t)(ngroups - 1));
    const int tid = threadIdx.x;

    if (tid < d) {
        s_ab[tid].x = (R)D.pa[tid];
        s_ab[tid].y = (R)D.pb[tid];
    }
    if (tid < 4) s_c[tid] = (R)D.c[tid];

    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t q = tile / T;
        const uint32_t t = (uint32_t)(tile - q * T);
        tile_setup<MODE>(D, level, q, parents, s_wb);
        const StreamConst sc = stream_const(keys, t, (uint32_t)q, (uint32_t)level);
        ThreadSums<MODE> acc(s_acc);
#define ZMC_FOLD_CASE(DD)                                                              \
    case DD:                                                                           \
        sample_tile_fold<MODE, FN, WIDE, DD>(acc, keys, sc, s_wb, s_ab, s_c, ngroups, tail); \
        break;
        switch (d) {
            ZMC_FOLD_CASE(1) ZMC_FOLD_CASE(2) ZMC_FOLD_CASE(3) ZMC_FOLD_CASE(4)
            ZMC_FOLD_CASE(5) ZMC_FOLD_CASE(6) ZMC_FOLD_CASE(7) ZMC_FOLD_CASE(8)
            ZMC_FOLD_CASE(9) ZMC_FOLD_CASE(10) ZMC_FOLD_CASE(11) ZMC_FOLD_CASE(12)
            ZMC_FOLD_CASE(13) ZMC_FOLD_CASE(14) ZMC_FOLD_CASE(15) ZMC_FOLD_CASE(16)
            default: break;
        }
#undef ZMC_FOLD_CASE
        acc.reduce_store(sums, tile, st);
    }
}

// Body of the kernel for an expression integrand E with dimension DIM known
// at compile time: E::eval(x, p) reads x[0..DIM-1] and the parameters p[].
template <int MODE, int DIM, class E>
__device__ __forceinline__ void eval_expr_body(const Desc* __restrict__ desc, State* __restrict__ st,
                                               const uint32_t* __restrict__ parents,
                                               double2* __restrict__ sums, int level,
                                               const PhiloxKeys& keys) {
    using R = typename ModeTraits<MODE>::R;
    using R2 = typename ModeTraits<MODE>::R2;
    __shared__ R2 s_wb[ZMC_MAX_DIM];
    __shared__ R s_p[2 * ZMC_MAX_DIM + 4];
    __shared__ double2 s_acc[MODE == ZMC_FP32_FP64ACC ? kEvalMaxThreads : 1];

    const Desc& D = *desc;
    const int64_t C = st->cells[level];
    if (C <= 0) return;
    const int T = D.T;
    const int64_t n = D.n;
    const int64_t tiles = C * T;
    const uint32_t ngroups = (uint32_t)((n + 3) >> 2);
    const uint32_t tail = (uint32_t)(n - 4 * (int64_t)(ngroups - 1));
    const int tid = threadIdx.x;

    if (tid < ZMC_MAX_DIM) {
        s_p[tid] = (R)D.pa[tid];
        s_p[ZMC_MAX_DIM + tid] = (R)D.pb[tid];
    }
    if (tid < 4) s_p[2 * ZMC_MAX_DIM + tid] = (R)D.c[tid];

    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t q = tile / T;
        const uint32_t t = (uint32_t)(tile - q * T);
        tile_setup<MODE>(D, level, q, parents, s_wb);
        const StreamConst sc = stream_const(keys, t, (uint32_t)q, (uint32_t)level);
        ThreadSums<MODE> acc(s_acc);
        uint32_t g = tid;
        while (g < ngroups) {
            for (int j = 0; j < kFlushGroups && g < ngroups; ++j, g += blockDim.x) {
                R x0[DIM], x1[DIM], x2[DIM], x3[DIM];
                const uint32_t cbase = g * DIM;
#pragma unroll
                for (int i = 0; i < DIM; ++i) {
                    const uint4 w = philox_stream(keys, sc, cbase + i);
                    const R2 wb = s_wb[i];
                    x0[i] = point<MODE>(w.x, wb);
                    x1[i] = point<MODE>(w.y, wb);
                    x2[i] = point<MODE>(w.z, wb);
                    x3[i] = point<MODE>(w.w, wb);
                }
                R f0 = E::eval(x0, s_p), f1 = E::eval(x1, s_p);
                R f2 = E::eval(x2, s_p), f3 = E::eval(x3, s_p);
                mask_tail(g == ngroups - 1, tail, f1, f2, f3);
                acc.add4(f0, f1, f2, f3);
            }
            acc.flush();
        }
        acc.reduce_store(sums, tile, st);
    }
}

#ifndef __CUDACC_RTC__
// One mode's registry instantiations, indexed by integrand id.  `wide`
// selects the sine/cosine variants that accept any argument; the host
// chooses the bounded ones when it can prove |argument| <= kFastTrigLimit.
template <int MODE>
inline const void* eval_kernel_for(int fn, bool wide) {
    const bool w = wide && MODE != ZMC_FP64;
    switch (fn) {
    case kConstant: return (const void*)zmc_eval_reduce<MODE, kConstant, false>;
    case kLinear: return (const void*)zmc_eval_reduce<MODE, kLinear, false>;
    case kSinSum:
        return w ? (const void*)zmc_eval_reduce<MODE, kSinSum, true>
                 : (const void*)zmc_eval_reduce<MODE, kSinSum, false>;
    case kGaussNorm: return (const void*)zmc_eval_reduce<MODE, kGaussNorm, false>;
    case kGenzOsc:
        return w ? (const void*)zmc_eval_reduce<MODE, kGenzOsc, true>
                 : (const void*)zmc_eval_reduce<MODE, kGenzOsc, false>;
    case kGenzProdPeak: return (const void*)zmc_eval_reduce<MODE, kGenzProdPeak, false>;
    case kGenzGauss: return (const void*)zmc_eval_reduce<MODE, kGenzGauss, false>;
    case kGenzCorner: return (const void*)zmc_eval_reduce<MODE, kGenzCorner, false>;
    default: return nullptr;
    }
}
#endif

}  // namespace zmc
