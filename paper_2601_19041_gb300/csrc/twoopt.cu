// Local-search kernels (one warp per tour, its arrays in shared memory when
// they fit): 2-opt (local_search 1 and 2; twoopt.cuh, or the directed 2-opt of
// threeopt.cuh for the ATSP) or 3-opt (3 and 4, threeopt.cuh).
#include "threeopt.cuh"

namespace hac {

// One block of LS_WARPS warps per instance: warp 0 runs the search, the other
// warps help with its long segment reversals and wide pre-tests (twoopt.cuh,
// 2-opt of symmetric instances) and are released when it ends.
constexpr int LS_WARPS = 8;   // at most LS_WARPS_MAX

__global__ void k_two_opt_nn(const DevInst *insts, unsigned smem_bytes)
{
    extern __shared__ __align__(16) unsigned char ls_sm[];
    __shared__ int coop[LS_COOP_WORDS];
    const DevInst &I = insts[blockIdx.x];
    if (!I.local_search) return;   // the same for the whole block
    const bool w0 = threadIdx.x < 32;
    LsMem M = ls_shared(I, I.nn_tour, ls_sm, smem_bytes, ls_global(I, I.nn_tour), w0);
    if (blockDim.x > 32) { M.coop = coop; M.coop_warps = (int)(blockDim.x >> 5); }
    if (!w0) { ls_coop_help(I, M); return; }
    if (I.local_search >= 3) warp_three_opt(I, I.nn_tour, M);
    else warp_two_opt_any(I, I.nn_tour, M);
    ls_coop_end(M);
    const double L = warp_tour_length(I, I.nn_tour);
    if (threadIdx.x == 0) I.st->L_nn = L;
}

__global__ void k_two_opt_ib(const DevInst *insts, unsigned smem_bytes)
{
    extern __shared__ __align__(16) unsigned char ls_sm[];
    __shared__ int coop[LS_COOP_WORDS];
    const DevInst &I = insts[blockIdx.x];
    if ((I.local_search != 1 && I.local_search != 3) || !I.st->active) return;   // the same for the whole block
    const bool w0 = threadIdx.x < 32;
    LsMem M = ls_shared(I, I.ib_tour, ls_sm, smem_bytes, ls_global(I, I.ib_tour), w0);
    if (blockDim.x > 32) { M.coop = coop; M.coop_warps = (int)(blockDim.x >> 5); }
    if (!w0) { ls_coop_help(I, M); return; }
    if (I.local_search == 3) warp_three_opt(I, I.ib_tour, M);
    else warp_two_opt_any(I, I.ib_tour, M);
    ls_coop_end(M);
    const double L = warp_tour_length(I, I.ib_tour);
    if (threadIdx.x == 0) I.st->L_ib = L;
}

// local_search = 2 or 4 (Algorithm 1's local search on every ant): ant blockIdx.x % max_m of instance
// blockIdx.x / max_m, right after construction; its length is recomputed
__global__ void k_two_opt_all(const DevInst *insts, int max_m, unsigned smem_bytes)
{
    extern __shared__ __align__(16) unsigned char ls_sm[];
    const DevInst &I = insts[blockIdx.x / max_m];
    const int a = blockIdx.x % max_m;
    if ((I.local_search != 2 && I.local_search != 4) || a >= I.m || I.st->t >= I.iters) return;
    int32_t *tour = I.tours + (size_t)a * I.n;
    const LsMem M = ls_shared(I, tour, ls_sm, smem_bytes, ls_ant(I, a));
    if (I.local_search == 4) warp_three_opt(I, tour, M);
    else warp_two_opt_any(I, tour, M);
    const double L = warp_tour_length(I, tour);
    if (threadIdx.x == 0) I.lens[a] = L;
}

// shared memory sized for the largest instance, capped (each instance then
// takes what fits, the rest stays in the workspace)
static size_t ls_launch_smem(int max_n)
{
    const size_t cap = 220 * 1024;
    if (ls_smem_full(max_n) <= cap) return ls_smem_full(max_n);
    return ls_smem_core(max_n) <= cap ? ls_smem_core(max_n) : 0;
}

template <typename Kern>
static void ls_launch(Kern kern, const DevInst *d_inst, int count, int max_n, cudaStream_t s)
{
    const size_t smem = ls_launch_smem(max_n);
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<count, 32 * LS_WARPS, smem, s>>>(d_inst, (unsigned)smem);
}

void launch_two_opt_all(const DevInst *d_inst, int count, int max_m, int max_n, cudaStream_t s)
{
    const size_t smem = ls_launch_smem(max_n);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_two_opt_all, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_two_opt_all<<<count * max_m, 32, smem, s>>>(d_inst, max_m, (unsigned)smem);
}

void launch_two_opt_nn(const DevInst *d_inst, int count, int max_n, cudaStream_t s)
{
    ls_launch(k_two_opt_nn, d_inst, count, max_n, s);
}

void launch_two_opt_ib(const DevInst *d_inst, int count, int max_n, cudaStream_t s)
{
    ls_launch(k_two_opt_ib, d_inst, count, max_n, s);
}

}  // namespace hac
