// FP32-evaluation / FP64-accumulation instantiations of the sampling kernel.
#include "eval_kernel.cuh"

namespace zmc {
const void* eval_kernel_fp32_fp64acc(int fn, int d) { return eval_kernel_for<ZMC_FP32_FP64ACC>(fn, d); }
}  // namespace zmc
