// Pipe-rate probe: the per-SM instruction throughputs that bound the
// sampling kernel, measured on the GPU the library runs on.  The sampling
// kernel is bound by integer work (Philox4x32-10: 32x32 -> 64-bit products
// and three-input XORs), for which no vendor peak is published; these
// kernels measure one instruction kind each, in independent chains, so that
// the roofline denominators are reproducible from this repository.
//
// Every kind runs kProbeChains independent chains per thread; one iteration
// is one step of every chain.  Thread 0 of each CTA records %clock64,
// %globaltimer and %smid around the loop (after a CTA barrier on both sides):
// the CTAs are not spread evenly over the SMs, so the rate per SM per clock
// is the work of the CTAs an SM ran over that SM's own cycle span (first
// start to last end on its %clock64), not the kernel's time at an assumed
// clock.
#include <stdint.h>

#include "zmc_internal.h"

namespace zmc {

namespace {

constexpr int kProbeChains = 8;

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A Philox4x32-10 block whose round products take their high half from
// mul.hi with an immediate multiplier and their low half from mul.lo with the
// multiplier held in a kernel parameter (mA, mB equal to the constants at run
// time), so the compiler cannot pair them into one 64-bit product.  Same
// words as philox_from_product.
__device__ __forceinline__ uint4 philox_split(const PhiloxKeys& K, const StreamConst& s,
                                              uint32_t hi0, uint32_t lo0, uint32_t mA,
                                              uint32_t mB) {
    const uint32_t z1 = hi0 ^ s.r1z;
    const uint32_t hi1 = __umulhi(kPhiloxMulB, z1), lo1 = mB * z1;
    uint4 c = make_uint4(hi1 ^ s.r2x, lo1, s.r2z ^ lo0, s.r2w);
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const uint32_t h0 = __umulhi(kPhiloxMulA, c.x), l0 = mA * c.x;
        const uint32_t h1 = __umulhi(kPhiloxMulB, c.z), l1 = mB * c.z;
        c = make_uint4(h1 ^ c.y ^ K.k0[r], l1, h0 ^ c.w ^ K.k1[r], l0);
    }
    return c;
}

template <int KIND>
__global__ void __launch_bounds__(256)
zmc_pipe_probe_kernel(int64_t iters, uint32_t seed, uint32_t mA, uint32_t mB,
                      const PhiloxKeys keys, uint32_t* __restrict__ sink,
                      long long* __restrict__ clocks) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    __syncthreads();
    long long c0 = 0, t0 = 0;
    if (threadIdx.x == 0) {
        t0 = global_ns();
        c0 = clock64();
    }
    uint32_t out = 0;
    if constexpr (KIND == ZMC_PROBE_IMAD_WIDE) {
        uint64_t acc[kProbeChains];
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) acc[j] = (uint64_t)(seed ^ (tid * 8 + j)) << 1;
        for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kProbeChains; ++j)
                asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc[j]) : "r"((uint32_t)acc[j]), "r"(mA));
        }
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) out ^= (uint32_t)acc[j] ^ (uint32_t)(acc[j] >> 32);
    } else if constexpr (KIND == ZMC_PROBE_IMAD || KIND == ZMC_PROBE_IMAD_HI ||
                         KIND == ZMC_PROBE_LOP3) {
        uint32_t x[kProbeChains];
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) x[j] = seed ^ (tid * 8 + j);
        for (int64_t i = 0; i < iters; ++i) {
            uint32_t nx[kProbeChains];
#pragma unroll
            for (int j = 0; j < kProbeChains; ++j) {
                const uint32_t y = x[(j + 1) % kProbeChains];
                if constexpr (KIND == ZMC_PROBE_IMAD)
                    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(nx[j]) : "r"(x[j]), "r"(mA), "r"(y));
                else if constexpr (KIND == ZMC_PROBE_IMAD_HI)
                    asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(nx[j]) : "r"(x[j]), "r"(mA), "r"(y));
                else
                    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(nx[j]) : "r"(x[j]), "r"(y), "r"(mB));
            }
#pragma unroll
            for (int j = 0; j < kProbeChains; ++j) x[j] = nx[j];
        }
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) out ^= x[j];
    } else if constexpr (KIND == ZMC_PROBE_HILO_PAIRED || KIND == ZMC_PROBE_HILO_SPLIT) {
        // both halves of one product, combined by a three-input XOR: the
        // shape of a Philox round's multiply
        uint32_t x[kProbeChains];
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) x[j] = seed ^ (tid * 8 + j);
        for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kProbeChains; ++j) {
                const uint32_t h = __umulhi(kPhiloxMulA, x[j]);
                const uint32_t l = (KIND == ZMC_PROBE_HILO_SPLIT ? mA : kPhiloxMulA) * x[j];
                x[j] = h ^ l ^ mB;
            }
        }
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) out ^= x[j];
    } else if constexpr (KIND == ZMC_PROBE_FFMA) {
        float f[kProbeChains];
        const float a = -0.5f + 1e-7f * (float)(seed & 7u);
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) f[j] = (float)(tid * 8 + j);
        for (int64_t i = 0; i < iters; ++i) {
            float nf[kProbeChains];
#pragma unroll
            for (int j = 0; j < kProbeChains; ++j) nf[j] = fmaf(f[j], a, f[(j + 1) % kProbeChains]);
#pragma unroll
            for (int j = 0; j < kProbeChains; ++j) f[j] = nf[j];
        }
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) out ^= __float_as_uint(f[j]);
    } else if constexpr (KIND == ZMC_PROBE_DFMA) {
        double f[kProbeChains];
        const double a = -0.5 + 1e-12 * (double)(seed & 7u);
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) f[j] = (double)(tid * 8 + j);
        for (int64_t i = 0; i < iters; ++i) {
            double nf[kProbeChains];
#pragma unroll
            for (int j = 0; j < kProbeChains; ++j) nf[j] = fma(f[j], a, f[(j + 1) % kProbeChains]);
#pragma unroll
            for (int j = 0; j < kProbeChains; ++j) f[j] = nf[j];
        }
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) out ^= (uint32_t)__double_as_longlong(f[j]);
    } else {
        // Philox4x32-10 blocks with consecutive counters of one stream, as
        // the sampling kernel forms them: round 1's product of the counter as
        // a 64-bit running sum, the stream-invariant products hoisted.
        const StreamConst sc = stream_const(keys, seed & 7u, tid, 1u);
        uint64_t P = (uint64_t)kPhiloxMulA * (uint64_t)(tid * kProbeChains);
        const uint64_t step = (uint64_t)kPhiloxMulA * (uint64_t)(gridDim.x * blockDim.x * kProbeChains);
        for (int64_t i = 0; i < iters; ++i) {
            uint64_t Q = P;
#pragma unroll
            for (int j = 0; j < kProbeChains; ++j) {
                const uint4 w = KIND == ZMC_PROBE_PHILOX_SPLIT
                                    ? philox_split(keys, sc, (uint32_t)(Q >> 32), (uint32_t)Q, mA, mB)
                                    : philox_from_product(keys, sc, (uint32_t)(Q >> 32), (uint32_t)Q);
                out ^= w.x ^ w.y ^ w.z ^ w.w;
                Q += kPhiloxMulA;
            }
            P += step;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long c1 = clock64(), t1 = global_ns();
        uint32_t sm;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
        long long* rec = clocks + 6 * blockIdx.x;
        rec[0] = c0;
        rec[1] = c1;
        rec[2] = t0;
        rec[3] = t1;
        rec[4] = (long long)sm;
        rec[5] = 0;
    }
    sink[tid] = out;
}

const void* probe_kernel(int kind) {
    switch (kind) {
    case ZMC_PROBE_IMAD_WIDE: return (const void*)zmc_pipe_probe_kernel<ZMC_PROBE_IMAD_WIDE>;
    case ZMC_PROBE_IMAD: return (const void*)zmc_pipe_probe_kernel<ZMC_PROBE_IMAD>;
    case ZMC_PROBE_IMAD_HI: return (const void*)zmc_pipe_probe_kernel<ZMC_PROBE_IMAD_HI>;
    case ZMC_PROBE_HILO_PAIRED: return (const void*)zmc_pipe_probe_kernel<ZMC_PROBE_HILO_PAIRED>;
    case ZMC_PROBE_HILO_SPLIT: return (const void*)zmc_pipe_probe_kernel<ZMC_PROBE_HILO_SPLIT>;
    case ZMC_PROBE_LOP3: return (const void*)zmc_pipe_probe_kernel<ZMC_PROBE_LOP3>;
    case ZMC_PROBE_FFMA: return (const void*)zmc_pipe_probe_kernel<ZMC_PROBE_FFMA>;
    case ZMC_PROBE_DFMA: return (const void*)zmc_pipe_probe_kernel<ZMC_PROBE_DFMA>;
    case ZMC_PROBE_PHILOX: return (const void*)zmc_pipe_probe_kernel<ZMC_PROBE_PHILOX>;
    case ZMC_PROBE_PHILOX_SPLIT: return (const void*)zmc_pipe_probe_kernel<ZMC_PROBE_PHILOX_SPLIT>;
    default: return nullptr;
    }
}

}  // namespace

cudaError_t launch_pipe_probe(int kind, int64_t iters, int blocks, int threads, uint32_t* sink,
                              long long* clocks, cudaStream_t s) {
    const void* k = probe_kernel(kind);
    const uint32_t seed = 0x2545F491u;
    uint32_t mA = kPhiloxMulA, mB = kPhiloxMulB;
    const PhiloxKeys keys = philox_keys(0x243F6A8885A308D3ull);
    void* args[] = {(void*)&iters, (void*)&seed, (void*)&mA, (void*)&mB, (void*)&keys,
                    (void*)&sink, (void*)&clocks};
    return cudaLaunchKernel(k, dim3(blocks), dim3(threads), args, 0, s);
}

bool pipe_probe_kind_valid(int kind) { return probe_kernel(kind) != nullptr; }

}  // namespace zmc
