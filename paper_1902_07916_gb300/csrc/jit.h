// Run-time compilation of expression integrands ("expr:<...>") with NVRTC.
// The generated kernel is kernel (a) of eval_kernel.cuh with the expression
// as its integrand and the dimension fixed at compile time.
#pragma once

#include <string>

namespace zmc {

struct JitKernel {
    const void* kernel;   // cudaKernel_t usable with cudaLaunchKernel
};

// Compile (or fetch from the process-wide cache) the sampling kernel for
// `expr` in dimension `dim` with `n_params` parameters and precision `mode`.
// Returns ZMC_OK or ZMC_ERR_COMPILE / ZMC_ERR_ARG / ZMC_ERR_CUDA with a
// message (the NVRTC log on a compile error) in *log.
int jit_compile(const char* expr, int dim, int n_params, int mode, JitKernel* out,
                std::string* log);
void jit_release(JitKernel* k);
// Compile `expr` for compute capability major.minor without a device (the
// cubin is dropped).  ZMC_OK or ZMC_ERR_ARG / ZMC_ERR_COMPILE with *log.
int jit_check(const char* expr, int dim, int mode, int major, int minor, std::string* log);

}  // namespace zmc
