// Kernel (a): the fused sample-generate / evaluate / reduce kernel.
//
// One CTA owns one (cell, trial) tile at a time and walks the level's tiles
// persistently (tile += gridDim.x); the number of cells of the level is read
// from device memory, so the host never needs it.  Per tile:
//   1. d threads decode the cell's lattice coordinates from the slot index
//      (level 1: base-k digits; deeper: parent coordinates * k + child digit)
//      into per-dimension shifts in shared memory;
//   2. every thread takes groups of four consecutive samples; for each
//      dimension one Philox4x32-10 block (counter (g*d + i, t, q, L)) gives
//      that dimension's coordinate for all four samples (Sec. 2.2: random
//      numbers are produced where they are used, nothing is stored);
//   3. the values f and f^2 are summed per thread, then across the warp with
//      shuffles and across warps through shared memory, and one thread writes
//      the tile's (S1, S2) as two doubles.
//
// Registry integrands fold each coordinate into four independent
// accumulators as it is produced.  Expression integrands (compiled at run
// time, dimension fixed at compile time) keep the four points' coordinates in
// registers and evaluate the expression on each.
//
// MODE 0: FP64 throughout.  MODE 1: FP32 points and integrand, FP32 partial
// sums over 16 groups (64 points) flushed into FP64 per-thread sums, FP64
// block reduction.  MODE 2: FP32 points and integrand with TwoSum-compensated
// per-thread sums and a TwoSum block reduction; the (sum, error) float pair
// is widened to FP64 only for the stored result.
#pragma once

#include "zmc_device.cuh"

namespace zmc {

constexpr int kEvalMaxThreads = 512;
constexpr int kFlushGroups = 16;  // MODE 1: FP32 partials cover 64 points

template <int MODE>
struct ModeTraits { using R = float; };
template <>
struct ModeTraits<ZMC_FP64> { using R = double; };

template <int MODE>
__device__ __forceinline__ typename ModeTraits<MODE>::R point(uint32_t w, typename ModeTraits<MODE>::R wid,
                                                            typename ModeTraits<MODE>::R base) {
    if constexpr (MODE == ZMC_FP64) return fma(one_plus_word_f64(w), wid, base);
    else return fmaf(one_plus_word_f32(w), wid, base);
}

// Per-thread running sums of f and f^2 in the mode's arithmetic.
template <int MODE>
struct ThreadSums {
    double S1d = 0.0, S2d = 0.0;               // MODE 0 and 1
    float s1 = 0.f, e1 = 0.f, s2 = 0.f, e2 = 0.f;  // MODE 1 partials / MODE 2 (sum, err)
    int pending = 0;

    template <typename R>
    __device__ __forceinline__ void add4(R f0, R f1, R f2, R f3) {
        if constexpr (MODE == ZMC_FP64) {
            S1d += f0; S1d += f1; S1d += f2; S1d += f3;
            S2d = fma(f0, f0, S2d); S2d = fma(f1, f1, S2d);
            S2d = fma(f2, f2, S2d); S2d = fma(f3, f3, S2d);
        } else if constexpr (MODE == ZMC_FP32_FP64ACC) {
            s1 += (f0 + f1) + (f2 + f3);
            s2 += fmaf(f0, f0, f1 * f1) + fmaf(f2, f2, f3 * f3);
            if (++pending == kFlushGroups) {
                S1d += (double)s1; S2d += (double)s2;
                s1 = 0.f; s2 = 0.f; pending = 0;
            }
        } else {
            float t, r;
            two_sum(s1, (f0 + f1) + (f2 + f3), t, r); s1 = t; e1 += r;
            two_sum(s2, fmaf(f0, f0, f1 * f1) + fmaf(f2, f2, f3 * f3), t, r); s2 = t; e2 += r;
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
            if constexpr (MODE == ZMC_FP32_FP64ACC) { S1d += (double)s1; S2d += (double)s2; }
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

// Shared per-tile set-up: the cell's per-dimension shifts.  `shift` turns
// the assembled 1.m value into the uniform (1 - 2^-33 in FP64, 1 - 2^-24 in
// FP32), so that point = fma(1.m, w_L, base) = lo + (c + u) w_L.
template <int MODE>
__device__ __forceinline__ void tile_setup(const Desc& D, int level, int64_t q,
                                           const uint32_t* parents,
                                           typename ModeTraits<MODE>::R* s_base) {
    using R = typename ModeTraits<MODE>::R;
    const double shift = (MODE == ZMC_FP64) ? 1.0 - 0x1p-33 : 1.0 - 0x1p-24;
    const int tid = threadIdx.x;
    if (tid < D.d) {
        const double w = D.width[level][tid];
        const int64_t c = cell_coord(D, level, q, tid, parents);
        s_base[tid] = (R)(D.lo[tid] + (double)c * w - shift * w);
    }
    __syncthreads();
}

template <int MODE, int FN>
__global__ void __launch_bounds__(kEvalMaxThreads)
zmc_eval_reduce(const Desc* __restrict__ desc, State* __restrict__ st,
                const uint32_t* __restrict__ parents, double2* __restrict__ sums,
                int level) {
    using R = typename ModeTraits<MODE>::R;
    using F = Fn<FN, R>;
    __shared__ R s_base[ZMC_MAX_DIM], s_wid[ZMC_MAX_DIM];
    __shared__ R s_pa[ZMC_MAX_DIM], s_pb[ZMC_MAX_DIM], s_c[4];

    const Desc& D = *desc;
    const int64_t C = st->cells[level];
    if (C <= 0) return;
    const int d = D.d, T = D.T;
    const int64_t n = D.n;
    const int64_t tiles = C * T;
    const int64_t ngroups = (n + 3) >> 2;
    const uint32_t k0 = D.key[0], k1 = D.key[1];
    const int tid = threadIdx.x;

    if (tid < d) {
        s_wid[tid] = (R)D.width[level][tid];
        s_pa[tid] = (R)D.pa[tid];
        s_pb[tid] = (R)D.pb[tid];
    }
    if (tid < 4) s_c[tid] = (R)D.c[tid];

    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t q = tile / T;
        const uint32_t t = (uint32_t)(tile - q * T);
        tile_setup<MODE>(D, level, q, parents, s_base);

        ThreadSums<MODE> acc;
        for (int64_t g = tid; g < ngroups; g += blockDim.x) {
            R a0 = F::init(), a1 = F::init(), a2 = F::init(), a3 = F::init();
            const uint32_t cbase = (uint32_t)(g * d);
            for (int i = 0; i < d; ++i) {
                const uint4 w = philox4x32_10(
                    make_uint4(cbase + i, t, (uint32_t)q, (uint32_t)level), k0, k1);
                const R wi = s_wid[i], bi = s_base[i], pa = s_pa[i], pb = s_pb[i];
                a0 = F::fold(a0, point<MODE>(w.x, wi, bi), pa, pb);
                a1 = F::fold(a1, point<MODE>(w.y, wi, bi), pa, pb);
                a2 = F::fold(a2, point<MODE>(w.z, wi, bi), pa, pb);
                a3 = F::fold(a3, point<MODE>(w.w, wi, bi), pa, pb);
            }
            R f0 = F::finish(a0, s_c, d), f1 = F::finish(a1, s_c, d);
            R f2 = F::finish(a2, s_c, d), f3 = F::finish(a3, s_c, d);
            const int64_t left = n - 4 * g;   // only the last group can be short
            if (left < 4) {
                f3 = R(0);
                if (left < 3) f2 = R(0);
                if (left < 2) f1 = R(0);
            }
            acc.add4(f0, f1, f2, f3);
        }
        acc.reduce_store(sums, tile, st);
    }
}

// Body of the kernel for an expression integrand E with dimension DIM known
// at compile time: E::eval(x, p) reads x[0..DIM-1] and the parameters p[].
template <int MODE, int DIM, class E>
__device__ __forceinline__ void eval_expr_body(const Desc* __restrict__ desc, State* __restrict__ st,
                                               const uint32_t* __restrict__ parents,
                                               double2* __restrict__ sums, int level) {
    using R = typename ModeTraits<MODE>::R;
    __shared__ R s_base[ZMC_MAX_DIM], s_wid[ZMC_MAX_DIM];
    __shared__ R s_p[2 * ZMC_MAX_DIM + 4];

    const Desc& D = *desc;
    const int64_t C = st->cells[level];
    if (C <= 0) return;
    const int T = D.T;
    const int64_t n = D.n;
    const int64_t tiles = C * T;
    const int64_t ngroups = (n + 3) >> 2;
    const uint32_t k0 = D.key[0], k1 = D.key[1];
    const int tid = threadIdx.x;

    if (tid < DIM) s_wid[tid] = (R)D.width[level][tid];
    if (tid < ZMC_MAX_DIM) {
        s_p[tid] = (R)D.pa[tid];
        s_p[ZMC_MAX_DIM + tid] = (R)D.pb[tid];
    }
    if (tid < 4) s_p[2 * ZMC_MAX_DIM + tid] = (R)D.c[tid];

    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t q = tile / T;
        const uint32_t t = (uint32_t)(tile - q * T);
        tile_setup<MODE>(D, level, q, parents, s_base);

        ThreadSums<MODE> acc;
        for (int64_t g = tid; g < ngroups; g += blockDim.x) {
            R x0[DIM], x1[DIM], x2[DIM], x3[DIM];
            const uint32_t cbase = (uint32_t)(g * DIM);
#pragma unroll
            for (int i = 0; i < DIM; ++i) {
                const uint4 w = philox4x32_10(
                    make_uint4(cbase + i, t, (uint32_t)q, (uint32_t)level), k0, k1);
                x0[i] = point<MODE>(w.x, s_wid[i], s_base[i]);
                x1[i] = point<MODE>(w.y, s_wid[i], s_base[i]);
                x2[i] = point<MODE>(w.z, s_wid[i], s_base[i]);
                x3[i] = point<MODE>(w.w, s_wid[i], s_base[i]);
            }
            R f0 = E::eval(x0, s_p), f1 = E::eval(x1, s_p);
            R f2 = E::eval(x2, s_p), f3 = E::eval(x3, s_p);
            const int64_t left = n - 4 * g;
            if (left < 4) {
                f3 = R(0);
                if (left < 3) f2 = R(0);
                if (left < 2) f1 = R(0);
            }
            acc.add4(f0, f1, f2, f3);
        }
        acc.reduce_store(sums, tile, st);
    }
}

#ifndef __CUDACC_RTC__
// Table of one mode's registry instantiations, indexed by integrand id.
template <int MODE>
inline const void* eval_kernel_for(int fn) {
    switch (fn) {
    case kConstant: return (const void*)zmc_eval_reduce<MODE, kConstant>;
    case kLinear: return (const void*)zmc_eval_reduce<MODE, kLinear>;
    case kSinSum: return (const void*)zmc_eval_reduce<MODE, kSinSum>;
    case kGaussNorm: return (const void*)zmc_eval_reduce<MODE, kGaussNorm>;
    case kGenzOsc: return (const void*)zmc_eval_reduce<MODE, kGenzOsc>;
    case kGenzProdPeak: return (const void*)zmc_eval_reduce<MODE, kGenzProdPeak>;
    case kGenzGauss: return (const void*)zmc_eval_reduce<MODE, kGenzGauss>;
    case kGenzCorner: return (const void*)zmc_eval_reduce<MODE, kGenzCorner>;
    default: return nullptr;
    }
}
#endif

}  // namespace zmc
