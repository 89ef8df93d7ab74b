// Host-side declarations shared by the translation units of libzmc: the
// device buffers of a handle and the kernel launchers.  Not part of the
// public ABI (include/zmc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "zmc_layout.h"
#include "zmc_device.cuh"

namespace zmc {

// Device buffers of one handle.
struct Buffers {
    Desc* desc;
    State* state;
    double2* sums;        // [cap_cells * T]   (S1, S2) per (cell, trial)
    double2* cell_stats;  // [cap_cells]       (mean, spread)
    uint32_t* parents[2]; // [cap_parents * d] flagged cells, ping-pong
    double* part_stats;   // [kSelGrid * 3]    (count, mean, M2)
    int64_t* part_count;  // [kSelGrid]
    int64_t* part_offset; // [kSelGrid]
    double* part_margin;  // [kSelGrid]
    double* part_acc;     // [kPartAccDoubles] see below
    zmc_result* result;
};

// Selection kernels run on a fixed grid so that their reduction order, and
// hence every bit of the result, does not depend on the GPU's SM count.
// Levels of little work use fewer of the grid's CTAs (active_ctas).  256
// measured best overall: 608 (four CTAs on each of GB300's 152 SMs) saved
// 0.04 ms per 6-D sine step but cost 3 ms per 512-integral batch, whose
// 256 x 512 grid is mostly CTAs that exit at once.
constexpr int kSelGrid = 256;
constexpr int kSelThreads = 256;
// part_acc: the compaction CTAs' compensated (value, variance) partials of
// the level being compacted, kSelGrid x 4, then one slot of 4 per level
// (0 .. ZMC_MAX_DEPTH) written by the level's last CTA and read by the
// final reduction.
constexpr size_t kPartAccDoubles = 4 * ((size_t)kSelGrid + ZMC_MAX_DEPTH + 1);

// Launch shape of the sampling kernel.
struct EvalShape {
    int threads;   // per CTA, multiple of 32, <= 1024
    int grid;      // persistent CTAs
};

// Kernels (b): per-cell statistics + threshold, flag + count, compaction.
cudaError_t launch_init(const Buffers& b, int64_t level1_cells, cudaStream_t s);
cudaError_t launch_select(const Buffers& b, int level, const uint32_t* parents_prev,
                          uint32_t* parents_next, cudaStream_t s);
// Kernel (c): compensated final reduction into the result.
cudaError_t launch_final(const Buffers& b, cudaStream_t s);

// Round keys of a seed (host side).
PhiloxKeys philox_keys(uint64_t seed);

cudaError_t launch_uniforms(uint64_t seed, int level, uint32_t slot, uint32_t trial, int d,
                            int mode, int64_t first, int64_t count, double* out, cudaStream_t s);

// zmc_level_stats_noalloc (select.cu): returns ZMC_OK or an error code with
// the message in noalloc_last_error().
int level_stats_noalloc(const double* sums, int64_t cells, int trials, int64_t n, double volume,
                        double sigma_multiplier, double* cell_stats, double* level_stats,
                        cudaStream_t s);
const char* noalloc_last_error();

// CTA size of the batched sampling kernel.
constexpr int kBatchThreads = 256;

// What the batched sampling kernel needs of one integral.
struct BatchEval {
    const Desc* desc;
    const State* st;
    double2* sums;
    const uint32_t* parents[2];
    PhiloxKeys keys;
    int32_t fn;
};

// Sampling kernels (single-integral and batched) of precision mode MODE for
// registry integrands 2*PART and 2*PART + 1, by integrand id and dimension;
// nullptr for any other integrand.  Each (MODE, PART) is one translation unit
// generated by the build (eval_kernel_pair / batch_kernel_pair).
template <int MODE, int PART> const void* eval_kernel_part(int fn, int d);
template <int MODE, int PART> const void* batch_kernel_part(int fn, int d);
#define ZMC_DECLARE_KERNEL_PART(M, P)                                   \
    template <> const void* eval_kernel_part<M, P>(int fn, int d);      \
    template <> const void* batch_kernel_part<M, P>(int fn, int d);
#define ZMC_DECLARE_KERNEL_PARTS(M) \
    ZMC_DECLARE_KERNEL_PART(M, 0) ZMC_DECLARE_KERNEL_PART(M, 1) \
    ZMC_DECLARE_KERNEL_PART(M, 2) ZMC_DECLARE_KERNEL_PART(M, 3)
ZMC_DECLARE_KERNEL_PARTS(ZMC_FP64)
ZMC_DECLARE_KERNEL_PARTS(ZMC_FP32_FP64ACC)
ZMC_DECLARE_KERNEL_PARTS(ZMC_FP32_KAHAN)
#undef ZMC_DECLARE_KERNEL_PARTS
#undef ZMC_DECLARE_KERNEL_PART
constexpr int kKernelParts = 4;

// Batched form (batch.cu, select.cu): `items` / `level1_cells` / `out` are
// device arrays of `count` entries; row y of each selection grid works on
// integral y.
// Plan + sampling kernel of one group of `count` integrals (same integrand):
// `offsets` has count + 1 entries, `head` is the group's queue counter.
cudaError_t launch_batch_level(const BatchEval* items, int count, int level, int64_t* offsets,
                               unsigned long long* head, const void* kernel, int grid,
                               cudaStream_t s);
cudaError_t launch_init_batch(const Buffers* items, const int64_t* level1_cells, int count,
                              cudaStream_t s);
cudaError_t launch_select_batch(const Buffers* items, int count, int level, cudaStream_t s);
cudaError_t launch_final_batch(const Buffers* items, zmc_result* out, int count, cudaStream_t s);

cudaError_t launch_philox(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                          uint32_t c3, int64_t count, uint32_t* out,
                          cudaStream_t s);

// zmc_pipe_probe (probe.cu).
bool pipe_probe_kind_valid(int kind);
cudaError_t launch_pipe_probe(int kind, int64_t iters, int blocks, int threads, uint32_t* sink,
                              long long* clocks, cudaStream_t s);

}  // namespace zmc
