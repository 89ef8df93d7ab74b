// FP64 instantiations of the sampling kernel (kernel (a)).
#include "eval_kernel.cuh"

namespace zmc {
const void* eval_kernel_fp64(int fn, int d) { return eval_kernel_for<ZMC_FP64>(fn, d); }
}  // namespace zmc
