// FP32-evaluation / FP64-accumulation instantiations of the batched sampling kernel.
#include "batch_kernel.cuh"

namespace zmc {
const void* batch_kernel_fp32_fp64acc(int fn, int d) { return batch_kernel_for<ZMC_FP32_FP64ACC>(fn, d); }
}  // namespace zmc
