// Batched integration: many independent integrals (uneven dimension, cell
// count and depth) advance one tree level at a time.  The integrals are
// grouped by integrand; per level and group:
//   1. zmc_batch_plan: each integral's number of sampling units at this level
//      (from its own tree state) and their exclusive prefix sum;
//   2. zmc_batch_eval (batch_kernel.cuh): one persistent kernel over the
//      units of the group's integrals, atomic queue;
// the groups run as parallel branches of the level's graph, then
//   3. the selection kernels with one grid row (blockIdx.y) per integral.
// The host captures each level into a CUDA graph once and replays it.
#include "eval_kernel.cuh"
#include "zmc_internal.h"

namespace zmc {

__global__ void zmc_batch_plan(const BatchEval* __restrict__ items, int count, int level,
                               int64_t* __restrict__ offsets, unsigned long long* head) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const State* st = items[i].st;
        offsets[i + 1] = st->cells[level] > 0 ? st->uplan[level].units : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        offsets[0] = 0;
        for (int i = 0; i < count; ++i) offsets[i + 1] += offsets[i];
        *head = 0ull;
    }
}

cudaError_t launch_batch_level(const BatchEval* items, int count, int level, int64_t* offsets,
                               unsigned long long* head, const void* kernel, int grid,
                               cudaStream_t s) {
    zmc_batch_plan<<<1, 256, 0, s>>>(items, count, level, offsets, head);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&items, (void*)&count, (void*)&level, (void*)&offsets, (void*)&head};
    return cudaLaunchKernel(kernel, dim3(grid), dim3(kBatchThreads), args, 0, s);
}

}  // namespace zmc
