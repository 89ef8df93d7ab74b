// FP64 instantiations of the batched sampling kernel.
#include "batch_kernel.cuh"

namespace zmc {
const void* batch_kernel_fp64(int fn, int d) { return batch_kernel_for<ZMC_FP64>(fn, d); }
}  // namespace zmc
