// FP32-evaluation / FP32-Kahan-accumulation instantiations of the sampling kernel.
#include "eval_kernel.cuh"

namespace zmc {
const void* eval_kernel_fp32_kahan(int fn, int d) { return eval_kernel_for<ZMC_FP32_KAHAN>(fn, d); }
}  // namespace zmc
