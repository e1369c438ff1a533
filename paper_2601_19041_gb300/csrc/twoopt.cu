// 2-opt kernels (one warp per instance); the search itself is in twoopt.cuh.
#include "twoopt.cuh"

namespace hac {

__global__ void k_two_opt_nn(const DevInst *insts)
{
    const DevInst &I = insts[blockIdx.x];
    if (!I.local_search) return;
    warp_two_opt(I, I.nn_tour);
    const double L = warp_tour_length(I, I.nn_tour);
    if (threadIdx.x == 0) I.st->L_nn = L;
}

__global__ void k_two_opt_ib(const DevInst *insts)
{
    const DevInst &I = insts[blockIdx.x];
    if (!I.local_search || !I.st->active) return;
    warp_two_opt(I, I.ib_tour);
    const double L = warp_tour_length(I, I.ib_tour);
    if (threadIdx.x == 0) I.st->L_ib = L;
}

void launch_two_opt_nn(const DevInst *d_inst, int count, cudaStream_t s)
{
    k_two_opt_nn<<<count, 32, 0, s>>>(d_inst);
}

void launch_two_opt_ib(const DevInst *d_inst, int count, cudaStream_t s)
{
    k_two_opt_ib<<<count, 32, 0, s>>>(d_inst);
}

}  // namespace hac
