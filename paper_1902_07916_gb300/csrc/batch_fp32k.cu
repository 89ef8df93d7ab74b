// FP32-evaluation / FP32-Kahan-accumulation instantiations of the batched sampling kernel.
#include "batch_kernel.cuh"

namespace zmc {
const void* batch_kernel_fp32_kahan(int fn, int d) { return batch_kernel_for<ZMC_FP32_KAHAN>(fn, d); }
}  // namespace zmc
