// FP32-evaluation instantiations of the sampling kernel (kernel (a)):
// FP64 accumulation and FP32 Kahan accumulation.
#include "eval_kernel.cuh"

namespace zmc {
const void* eval_kernel_fp32_fp64acc(int fn) { return eval_kernel_for<ZMC_FP32_FP64ACC>(fn); }
const void* eval_kernel_fp32_kahan(int fn) { return eval_kernel_for<ZMC_FP32_KAHAN>(fn); }
}  // namespace zmc
