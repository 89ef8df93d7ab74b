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

// Round keys of one seed: k0 + r * WeylA, k1 + r * WeylB for r = 0..9.
// Computed once on the host and passed by value, so the kernels read them
// as constant-bank operands of the XOR instructions.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

// Rounds 1 and 2 of every block of one (level L, slot q, trial t) stream
// have parts that depend on (t, q, L) only: with counter (c0, t, q, L),
// round 1 multiplies c0 and q, and round 2 multiplies round 1's first word,
// which does not involve c0.  Those products are taken once per stream.
struct StreamConst {
    uint32_t r1z;  // L ^ k1[0]:                  round 1, word 2 = hi(A c0) ^ r1z
    uint32_t r2x;  // lo(B q) ^ k0[1]:            round 2, word 0 = hi(B z1) ^ r2x
    uint32_t r2z;  // hi(A x1) ^ k1[1]:           round 2, word 2 = r2z ^ lo(A c0)
    uint32_t r2w;  // lo(A x1), x1 = hi(B q) ^ t ^ k0[0]: round 2, word 3
};

__device__ __forceinline__ StreamConst stream_const(const PhiloxKeys& K, uint32_t t,
                                                    uint32_t q, uint32_t L) {
    const uint32_t x1 = __umulhi(kPhiloxMulB, q) ^ t ^ K.k0[0];
    StreamConst s;
    s.r1z = L ^ K.k1[0];
    s.r2x = (kPhiloxMulB * q) ^ K.k0[1];
    s.r2z = __umulhi(kPhiloxMulA, x1) ^ K.k1[1];
    s.r2w = kPhiloxMulA * x1;
    return s;
}

// Philox4x32-10 of counter (c0, t, q, L) given the stream's constants and
// round 1's product A * c0 as (hi, lo).  The sampling kernel walks c0 in
// steps of one, so it carries that product as a 64-bit running sum instead
// of multiplying again.
__device__ __forceinline__ uint4 philox_from_product(const PhiloxKeys& K, const StreamConst& s,
                                                     uint32_t hi0, uint32_t lo0) {
    const uint32_t z1 = hi0 ^ s.r1z;                                          // round 1
    const uint32_t hi1 = __umulhi(kPhiloxMulB, z1), lo1 = kPhiloxMulB * z1;   // round 2
    uint4 c = make_uint4(hi1 ^ s.r2x, lo1, s.r2z ^ lo0, s.r2w);
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const uint32_t h0 = __umulhi(kPhiloxMulA, c.x), l0 = kPhiloxMulA * c.x;
        const uint32_t h1 = __umulhi(kPhiloxMulB, c.z), l1 = kPhiloxMulB * c.z;
        c = make_uint4(h1 ^ c.y ^ K.k0[r], l1, h0 ^ c.w ^ K.k1[r], l0);
    }
    return c;
}

// Philox4x32-10 of counter (c0, t, q, L) given the stream's constants.
__device__ __forceinline__ uint4 philox_stream(const PhiloxKeys& K, const StreamConst& s,
                                               uint32_t c0) {
    return philox_from_product(K, s, __umulhi(kPhiloxMulA, c0), kPhiloxMulA * c0);
}

// ------------------------------------------------------ word -> point maps
// The stream of (level L, slot q, trial t).  FP64 stream: dimension i of
// samples 4g .. 4g + 3 are the four 32-bit words of the block with counter
// (g*d + i, t, q, L).  FP32 stream: dimension i of samples 11g .. 11g + 10
// come from the PAIR of blocks with counters (2(g*d + i), t, q, L) and
// (2(g*d + i) + 1, t, q, L), each read as a 128-bit integer: samples 0..4 of
// the group take the first block's 23-bit fields (bits 23f .. 23f + 22),
// samples 5..9 the second block's, and sample 10 the 23-bit value made of the
// first block's bits 115..127 (low 13 bits) and the second block's bits
// 115..124 (high 10 bits) -- 253 of the pair's 256 bits, where five fields
// per block used 230.
//
// FP64 stream: u = (w + 1/2) 2^-32.  The double 1 + w 2^-32 is assembled
// from the word's bits, and the point lo + (c + u) w_L is formed from it as
// w_L * (1 + w 2^-32) + (lo + c w_L - (1 - 2^-33) w_L).
__device__ __forceinline__ double one_plus_word_f64(uint32_t w) {
    return __hiloint2double(0x3FF00000 | (int)(w >> 12), (int)(w << 20));
}
// FP32 stream: u = (field + 1/2) 2^-23, exact in binary32.  The float
// 1 + field 2^-23 is assembled from the bits, and the point is
// w_L * (1.m) + (lo + c w_L - (1 - 2^-24) w_L).
// One three-input LOP3, (field & 0x7FFFFF) | exponent, with the exponent
// held in a register: left to itself the compiler splits it into two
// instructions (one immediate operand per LOP3), and the integer ALU is one
// of the sampling kernel's two busiest pipes.
__device__ __forceinline__ float one_plus_field(uint32_t field23) {
    uint32_t r;
    asm("lop3.b32 %0, %1, 0x7FFFFF, %2, 0xEA;" : "=r"(r) : "r"(field23), "r"(0x3F800000u));
    return __uint_as_float(r);
}
// The five 23-bit fields of one block.
__device__ __forceinline__ void fields_1m(uint4 w, float& v0, float& v1, float& v2, float& v3,
                                          float& v4) {
    v0 = one_plus_field(w.x);                              // bits   0 ..  22
    v1 = one_plus_field(__funnelshift_r(w.x, w.y, 23));    // bits  23 ..  45
    v2 = one_plus_field(__funnelshift_r(w.y, w.z, 14));    // bits  46 ..  68
    v3 = one_plus_field(w.z >> 5);                         // bits  69 ..  91
    v4 = one_plus_field(__funnelshift_r(w.z, w.w, 28));    // bits  92 .. 114
}
// The pair's eleventh field: bits 115..127 of a (a.w >> 19) below bits
// 115..124 of b (b.w bits 19..28, moved to bits 13..22).
__device__ __forceinline__ float cross_1m(uint4 a, uint4 b) {
    const uint32_t f = (a.w >> 19) | ((b.w >> 6) & 0x7FE000u);
    return __uint_as_float(f | 0x3F800000u);
}

// ------------------------------------------------ elementary functions
// FP64 mode uses the CUDA math library.  FP32 mode carries the argument of
// sin/cos in turns (the per-cell fold coefficients are scaled by 1/(2 pi) in
// FP64): t - rint(t) is then an exact reduction for every float t, and the
// hardware sine/cosine takes the reduced turn times 2 pi, within [-pi, pi]
// (absolute error about 2^-21).  exp goes through the hardware 2^x.
constexpr float kTwoPi = 0x1.921fb6p+2f;         // 2 pi, to FP32
constexpr double kInvTwoPiD = 0.15915494309189535;  // 1 / (2 pi)
constexpr float kLog2E = 0x1.715476p+0f;         // log2(e), to FP32

__device__ __forceinline__ float zsin_turns(float t) { return __sinf((t - rintf(t)) * kTwoPi); }
__device__ __forceinline__ float zcos_turns(float t) { return __cosf((t - rintf(t)) * kTwoPi); }
__device__ __forceinline__ float zexp(float x) { return exp2f(x * kLog2E); }
__device__ __forceinline__ float zrcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double zexp(double x) { return exp(x); }
__device__ __forceinline__ double zrcp(double x) { return 1.0 / x; }

// ------------------------------------------------------------ integrands
// Every registry integrand is a fold over the dimensions followed by a
// finishing function.  The sampling kernel never forms the point itself: a
// coordinate is x_i = w_i v + b_i with v = 1.m in [1, 2) assembled from the
// Philox word, and each integrand folds the affine map into per-tile,
// per-dimension constants computed in FP64 by prep():
//   alpha_i, beta_i  -- the fold's coefficients of v,
//   term_i           -- summed into the fold's start value,
// so that fold(acc, v, alpha_i, beta_i, pb_i) costs one or two FMAs.  The
// parameters (pa_i, pb_i, c[0..3]) are laid out by the host from the user's
// list (api.cu).
template <int FN, typename R>
struct Fn;

struct Prep {
    double alpha, beta, term;
};

template <typename R> struct Fn<kConstant, R> {      // c0
    static constexpr bool kLog2 = false;
    static __device__ __forceinline__ Prep prep(double, double, double, double) { return {0, 0, 0}; }
    static __device__ __forceinline__ R init() { return R(0); }
    static __device__ __forceinline__ R fold(R a, R, R, R, R) { return a; }
    static __device__ __forceinline__ R finish(R, const R* c, int) { return c[0]; }
};
template <typename R> struct Fn<kLinear, R> {        // c0 + sum pa_i x_i
    static constexpr bool kLog2 = false;
    static __device__ __forceinline__ Prep prep(double w, double b, double pa, double) {
        return {pa * w, 0.0, pa * b};
    }
    static __device__ __forceinline__ R init() { return R(0); }
    static __device__ __forceinline__ R fold(R a, R v, R al, R, R) { return fma(al, v, a); }
    static __device__ __forceinline__ R finish(R a, const R* c, int) { return c[0] + a; }
};
template <typename R> struct Fn<kSinSum, R> {        // sin(sum x_i), Eq. (1)
    static constexpr bool kLog2 = false;
    static constexpr double kScale = sizeof(R) == 4 ? kInvTwoPiD : 1.0;  // FP32: turns
    static __device__ __forceinline__ Prep prep(double w, double b, double, double) {
        return {w * kScale, 0.0, b * kScale};
    }
    static __device__ __forceinline__ R init() { return R(0); }
    static __device__ __forceinline__ R fold(R a, R v, R al, R, R) { return fma(al, v, a); }
    static __device__ __forceinline__ R finish(R a, const R*, int) {
        if constexpr (sizeof(R) == 4) return zsin_turns(a);
        else return sin(a);
    }
};
template <typename R> struct Fn<kGaussNorm, R> {     // c1 exp(c0 |x|^2), Eq. (2)
    static constexpr bool kLog2 = true;
    static __device__ __forceinline__ Prep prep(double w, double b, double, double) {
        return {w, b, 0.0};
    }
    static __device__ __forceinline__ R init() { return R(0); }
    static __device__ __forceinline__ R fold(R a, R v, R al, R be, R) {
        const R x = fma(v, al, be);
        return fma(x, x, a);
    }
    static __device__ __forceinline__ R finish(R a, const R* c, int) { return c[1] * zexp(c[0] * a); }
    // FP32 modes: log2 of the value over c1 (c2 = c0 log2 e); c1 in FP64
    static __device__ __forceinline__ R finish_log2(R a, const R* c) { return c[2] * a; }
    static __device__ __forceinline__ double value_scale(const Desc& D) { return D.c[1]; }
};
template <typename R> struct Fn<kGenzOsc, R> {       // cos(c0 + sum pa_i x_i)
    static constexpr bool kLog2 = false;
    static constexpr double kScale = sizeof(R) == 4 ? kInvTwoPiD : 1.0;  // FP32: turns
    static __device__ __forceinline__ Prep prep(double w, double b, double pa, double) {
        return {pa * w * kScale, 0.0, pa * b * kScale};
    }
    static __device__ __forceinline__ R init() { return R(0); }
    static __device__ __forceinline__ R fold(R a, R v, R al, R, R) { return fma(al, v, a); }
    // c0 = 2 pi u1 in radians; c1 = u1, the same phase in turns
    static __device__ __forceinline__ R finish(R a, const R* c, int) {
        if constexpr (sizeof(R) == 4) return zcos_turns(c[1] + a);
        else return cos(c[0] + a);
    }
};
template <typename R> struct Fn<kGenzProdPeak, R> {  // 1 / prod (pb_i + (x_i - pa_i)^2)
    static constexpr bool kLog2 = false;
    static __device__ __forceinline__ Prep prep(double w, double b, double pa, double) {
        return {w, b - pa, 0.0};
    }
    static __device__ __forceinline__ R init() { return R(1); }
    static __device__ __forceinline__ R fold(R a, R v, R al, R be, R pb) {
        const R t = fma(v, al, be);
        return a * fma(t, t, pb);
    }
    static __device__ __forceinline__ R finish(R a, const R*, int) { return zrcp(a); }
};
template <typename R> struct Fn<kGenzGauss, R> {     // exp(-sum (pa_i (x_i - pb_i))^2)
    static constexpr bool kLog2 = true;
    static __device__ __forceinline__ Prep prep(double w, double b, double pa, double pb) {
        return {pa * w, pa * (b - pb), 0.0};
    }
    static __device__ __forceinline__ R init() { return R(0); }
    static __device__ __forceinline__ R fold(R a, R v, R al, R be, R) {
        const R t = fma(v, al, be);
        return fma(t, t, a);
    }
    static __device__ __forceinline__ R finish(R a, const R*, int) { return zexp(-a); }
    static __device__ __forceinline__ R finish_log2(R a, const R*) { return -kLog2E * a; }
    static __device__ __forceinline__ double value_scale(const Desc&) { return 1.0; }
};
template <typename R> struct Fn<kGenzCorner, R> {    // (1 + sum pa_i x_i)^-(d+1)
    static constexpr bool kLog2 = false;
    static __device__ __forceinline__ Prep prep(double w, double b, double pa, double) {
        return {pa * w, 0.0, pa * b};
    }
    static __device__ __forceinline__ R init() { return R(1); }
    static __device__ __forceinline__ R fold(R a, R v, R al, R, R) { return fma(al, v, a); }
    static __device__ __forceinline__ R finish(R a, const R*, int d) {
        // r^(d+1) with r = 1/a, by binary powering
        R r = zrcp(a), p = R(1);
        for (int e = d + 1; e; e >>= 1) {
            if (e & 1) p *= r;
            r *= r;
        }
        return p;
    }
};

// ------------------------------------------------- bounds-guarded build
// Compiled with ZMC_CHECKED (a test build of the library), every index into a
// partial-sum, cell-statistics or parent-list buffer is checked against the
// buffer's capacity before the access; a failed check records its site in
// the tree state (the first to fail wins), raises the run's status to
// ZMC_ERR_CHECK and skips the access, so a bad index shows up as a status
// instead of a fault.  In the normal build the checks compile away.
enum CheckSite : uint32_t {
    kSiteUnitSum = 1,      // sampling kernel: a unit's (S1, S2) slot
    kSiteLaneSum = 2,      // sampling kernel: a lane tile's slot
    kSiteParentRead = 3,   // a parent's coordinates (deeper levels)
    kSiteSumsRead = 4,     // statistics kernel: a cell's unit slots
    kSiteStatsWrite = 5,   // statistics kernel: a cell's (mean, spread)
    kSiteStatsRead = 6,    // flag and compaction kernels: a cell's statistics
    kSiteParentWrite = 7,  // compaction kernel: a flagged cell's coordinates
};

__device__ __forceinline__ bool in_bounds(const State* st, int64_t idx, int64_t cap,
                                          uint32_t site) {
#ifdef ZMC_CHECKED
    if (idx >= 0 && idx < cap) return true;
    State* w = const_cast<State*>(st);
    atomicCAS(&w->check_site, 0u, site);
    atomicMax(&w->status, ZMC_ERR_CHECK);
    return false;
#else
    (void)st; (void)idx; (void)cap; (void)site;
    return true;
#endif
}

// ------------------------------------------------------- cell geometry
// Lattice coordinate (dimension i) of work-list slot q at `level`.  Level 1
// is the full row-major lattice (dimension 0 fastest); at deeper levels slot
// q is child (q mod K) of the (q div K)-th flagged cell of the previous
// level, whose coordinates are in `parents` (flagged * d, uint32).  `st` is
// the run's tree state, used by the bounds-guarded build only.
__device__ __forceinline__ int64_t cell_coord(const Desc& D, int level, int64_t q,
                                              int i, const uint32_t* parents,
                                              const State* st) {
    if (level == 1) return (q / D.kpow[i]) % D.k;
    const int64_t r = q / D.K;
    const int64_t digit = q - r * D.K;
    if (!in_bounds(st, r * D.d + i, cap_parents(D), kSiteParentRead)) return 0;
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
