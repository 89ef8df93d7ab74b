// Device-side building blocks of the sampling kernel: the Philox4x32-10
// generator, the word -> uniform -> point maps, the registry integrands and
// the lattice decode of a work-list slot.  Written for sm_103a.
#pragma once

#include "zmc_layout.h"

namespace zmc {

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): each of the ten rounds
// multiplies counter words 0 and 2 by fixed odd constants (32x32 -> 64 bit),
// XORs the high halves with the other two words and the round key, and
// permutes; the two key words advance by Weyl increments between rounds.
constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeylA = 0x9E3779B9u;  // 2^32 * (golden ratio - 1)
constexpr uint32_t kPhiloxWeylB = 0xBB67AE85u;  // 2^32 * (sqrt(3) - 1)

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kPhiloxMulA, c.x);
        const uint32_t lo0 = kPhiloxMulA * c.x;
        const uint32_t hi1 = __umulhi(kPhiloxMulB, c.z);
        const uint32_t lo1 = kPhiloxMulB * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += kPhiloxWeylA;
        k1 += kPhiloxWeylB;
    }
    return c;
}

// ------------------------------------------------------ word -> point maps
// The stream of (level L, slot q, trial t): dimension i of samples 4g..4g+3
// is the block with counter (g*d + i, t, q, L), one lane per sample.
//
// FP64 reading: u = (w + 1/2) 2^-32.  The double 1 + w 2^-32 is assembled
// from the word's bits; x = lo + (c + u) w_L is then one FMA against the
// per-cell shift base = lo + c w_L - (1 - 2^-33) w_L.
__device__ __forceinline__ double one_plus_word_f64(uint32_t w) {
    return __hiloint2double(0x3FF00000 | (int)(w >> 12), (int)(w << 20));
}
// FP32 reading: u = (floor(w / 2^9) + 1/2) 2^-23, exact in binary32; the
// float 1 + floor(w/2^9) 2^-23 is assembled from the bits, and
// x = fma(1.m, w_L, base) with base = lo + c w_L - (1 - 2^-24) w_L.
__device__ __forceinline__ float one_plus_word_f32(uint32_t w) {
    return __uint_as_float(0x3F800000u | (w >> 9));
}

// ------------------------------------------------------------ integrands
// Every registry integrand is a fold over the dimensions followed by a
// finishing function: f(x) = finish(fold_i(acc, x_i, pa_i, pb_i)).  The
// per-dimension pair (pa_i, pb_i) and scalars c[0..3] are laid out on the
// host (api.cu) from the user's parameters.
template <int FN, typename R>
struct Fn;

template <typename R> struct Fn<kConstant, R> {      // c0
    static __device__ __forceinline__ R init() { return R(0); }
    static __device__ __forceinline__ R fold(R a, R, R, R) { return a; }
    static __device__ __forceinline__ R finish(R, const R* c, int) { return c[0]; }
};
template <typename R> struct Fn<kLinear, R> {        // c0 + sum pa_i x_i
    static __device__ __forceinline__ R init() { return R(0); }
    static __device__ __forceinline__ R fold(R a, R x, R pa, R) { return fma(pa, x, a); }
    static __device__ __forceinline__ R finish(R a, const R* c, int) { return c[0] + a; }
};
template <typename R> struct Fn<kSinSum, R> {        // sin(sum x_i), Eq. (1)
    static __device__ __forceinline__ R init() { return R(0); }
    static __device__ __forceinline__ R fold(R a, R x, R, R) { return a + x; }
    static __device__ __forceinline__ R finish(R a, const R*, int) { return sin(a); }
};
template <typename R> struct Fn<kGaussNorm, R> {     // c1 exp(c0 |x|^2), Eq. (2)
    static __device__ __forceinline__ R init() { return R(0); }
    static __device__ __forceinline__ R fold(R a, R x, R, R) { return fma(x, x, a); }
    static __device__ __forceinline__ R finish(R a, const R* c, int) { return c[1] * exp(c[0] * a); }
};
template <typename R> struct Fn<kGenzOsc, R> {       // cos(c0 + sum pa_i x_i)
    static __device__ __forceinline__ R init() { return R(0); }
    static __device__ __forceinline__ R fold(R a, R x, R pa, R) { return fma(pa, x, a); }
    static __device__ __forceinline__ R finish(R a, const R* c, int) { return cos(c[0] + a); }
};
template <typename R> struct Fn<kGenzProdPeak, R> {  // 1 / prod (pb_i + (x_i - pa_i)^2)
    static __device__ __forceinline__ R init() { return R(1); }
    static __device__ __forceinline__ R fold(R a, R x, R pa, R pb) {
        const R t = x - pa;
        return a * fma(t, t, pb);
    }
    static __device__ __forceinline__ R finish(R a, const R*, int) { return R(1) / a; }
};
template <typename R> struct Fn<kGenzGauss, R> {     // exp(-sum (pa_i (x_i - pb_i))^2)
    static __device__ __forceinline__ R init() { return R(0); }
    static __device__ __forceinline__ R fold(R a, R x, R pa, R pb) {
        const R t = pa * (x - pb);
        return fma(t, t, a);
    }
    static __device__ __forceinline__ R finish(R a, const R*, int) { return exp(-a); }
};
template <typename R> struct Fn<kGenzCorner, R> {    // (1 + sum pa_i x_i)^-(d+1)
    static __device__ __forceinline__ R init() { return R(1); }
    static __device__ __forceinline__ R fold(R a, R x, R pa, R) { return fma(pa, x, a); }
    static __device__ __forceinline__ R finish(R a, const R*, int d) {
        // r^(d+1) with r = 1/a, by binary powering
        R r = R(1) / a, p = R(1);
        for (int e = d + 1; e; e >>= 1) {
            if (e & 1) p *= r;
            r *= r;
        }
        return p;
    }
};

// ------------------------------------------------------- cell geometry
// Lattice coordinate (dimension i) of work-list slot q at `level`.  Level 1
// is the full row-major lattice (dimension 0 fastest); at deeper levels slot
// q is child (q mod K) of the (q div K)-th flagged cell of the previous
// level, whose coordinates are in `parents` (flagged * d, uint32).
__device__ __forceinline__ int64_t cell_coord(const Desc& D, int level, int64_t q,
                                              int i, const uint32_t* parents) {
    if (level == 1) return (q / D.kpow[i]) % D.k;
    const int64_t r = q / D.K;
    const int64_t digit = q - r * D.K;
    return (int64_t)D.k * parents[r * D.d + i] + (digit / D.kpow[i]) % D.k;
}

// ------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// Same for doubles.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

}  // namespace zmc
