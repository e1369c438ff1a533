// Tour construction, Algorithm 2, one launch per iteration: every ant of every
// active instance builds one tour, reading candidate rows from global memory
// (128-bit loads of ids and choice values).  The per-ant work is build_tours
// in ant.cuh; this file maps warps to (instance, ants) through the warp table.
#include "ant_lane.cuh"
#include "ant_pair.cuh"

namespace hac {

template <int APW>
__global__ void __launch_bounds__(256, 1) k_construct(const DevInst *__restrict__ insts,
                                                   const int4 *__restrict__ warpmap, int nwarps,
                                                   int nwords_max)
{
    extern __shared__ unsigned int smem_vis[];
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    if (gw >= nwarps) return;                       // warp-uniform
    const int4 wm = warpmap[gw];
    const DevInst &I = insts[wm.x];
    const int t = I.st->t;
    if (t >= I.iters) return;                       // warp-uniform
    GlobalRows rows{reinterpret_cast<const int4 *>(I.cand), reinterpret_cast<const float4 *>(I.choice),
                    I.k_pad >> 2, I.n};
    build_tours<APW>(I, rows, GlobalList{I.fbl}, t, wm.y, I.m, smem_vis + (size_t)wib * APW * nwords_max,
                     nwords_max, reinterpret_cast<const float2 *>(I.xy));
}

// one ant per lane: warp w of the table builds ants a0..a0+31 of its instance
template <int NG>
__global__ void __launch_bounds__(256, 1) k_construct_lane(const DevInst *__restrict__ insts,
                                                        const int4 *__restrict__ warpmap, int nwarps,
                                                        int nwords_max)
{
    extern __shared__ unsigned int smem_vis[];
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    if (gw >= nwarps) return;
    const int4 wm = warpmap[gw];
    const DevInst &I = insts[wm.x];
    const int t = I.st->t;
    if (t >= I.iters) return;
    GlobalRows rows{reinterpret_cast<const int4 *>(I.cand), reinterpret_cast<const float4 *>(I.choice),
                    I.k_pad >> 2, I.n};
    build_tours_lane<NG>(I, rows, GlobalList{I.fbl}, t, wm.y, I.m, smem_vis + (size_t)wib * 32 * nwords_max,
                         reinterpret_cast<const float2 *>(I.xy));
}

// one ant per lane pair: warp w of the table builds ants a0..a0+15 of its instance
template <int NGL>
__global__ void __launch_bounds__(256, 1) k_construct_pair(const DevInst *__restrict__ insts,
                                                        const int4 *__restrict__ warpmap, int nwarps,
                                                        int nwords_max)
{
    extern __shared__ unsigned int smem_vis[];
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    if (gw >= nwarps) return;
    const int4 wm = warpmap[gw];
    const DevInst &I = insts[wm.x];
    const int t = I.st->t;
    if (t >= I.iters) return;
    GlobalRows rows{reinterpret_cast<const int4 *>(I.cand), reinterpret_cast<const float4 *>(I.choice),
                    I.k_pad >> 2, I.n};
    build_tours_pair<NGL>(I, rows, GlobalList{I.fbl}, t, wm.y, I.m, smem_vis + (size_t)wib * 16 * nwords_max,
                          nwords_max, reinterpret_cast<const float2 *>(I.xy));
}

// fallback distances, then every ant's length (one block per instance)
__global__ void k_lengths(const DevInst *insts)
{
    const DevInst &I = insts[blockIdx.x];
    if (I.st->t >= I.iters) return;
    fallback_distances(I, 0, I.m);
    ant_lengths(I, 0, I.m);
}

template <int APW>
static void launch_construct_apw(const DevInst *d_inst, const int4 *d_warpmap, int warpmap_len,
                                 int warps_per_block, int max_n, cudaStream_t s)
{
    int nwords = (max_n + 32) / 32;   // visited bits 0..n (n: padding id)
    size_t smem = (size_t)warps_per_block * APW * nwords * sizeof(unsigned);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_construct<APW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    int blocks = (warpmap_len + warps_per_block - 1) / warps_per_block;
    k_construct<APW><<<blocks, warps_per_block * 32, smem, s>>>(d_inst, d_warpmap, warpmap_len,
                                                                 nwords);
}

int launch_construct(const DevInst *d_inst, const int4 *d_warpmap, int warpmap_len, int apw,
                     int warps_per_block, int max_n, int max_kp, int count, cudaStream_t s)
{
    if (apw == 32) {
        const int nwords = (max_n + 32) / 32;
        const size_t smem = (size_t)warps_per_block * 32 * nwords * sizeof(unsigned);
        const int blocks = (warpmap_len + warps_per_block - 1) / warps_per_block;
        const int G = max_kp / 4;
        auto go = [&](auto kern) {
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kern<<<blocks, warps_per_block * 32, smem, s>>>(d_inst, d_warpmap, warpmap_len, nwords);
        };
        if (G <= 3) go(k_construct_lane<3>);
        else if (G <= 5) go(k_construct_lane<5>);
        else go(k_construct_lane<8>);
        k_lengths<<<count, 256, 0, s>>>(d_inst);
        return 2;
    }
    if (apw == 16) {
        const int nwords = (max_n + 32) / 32;
        const size_t smem = (size_t)warps_per_block * 16 * nwords * sizeof(unsigned);
        const int blocks = (warpmap_len + warps_per_block - 1) / warps_per_block;
        const int G = max_kp / 4;
        auto go = [&](auto kern) {
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kern<<<blocks, warps_per_block * 32, smem, s>>>(d_inst, d_warpmap, warpmap_len, nwords);
        };
        if (G <= 4) go(k_construct_pair<2>);
        else if (G <= 6) go(k_construct_pair<3>);
        else go(k_construct_pair<4>);
        k_lengths<<<count, 256, 0, s>>>(d_inst);
        return 2;
    }
    if (apw == 4) launch_construct_apw<4>(d_inst, d_warpmap, warpmap_len, warps_per_block, max_n, s);
    else if (apw == 2) launch_construct_apw<2>(d_inst, d_warpmap, warpmap_len, warps_per_block, max_n, s);
    else launch_construct_apw<1>(d_inst, d_warpmap, warpmap_len, warps_per_block, max_n, s);
    k_lengths<<<count, 256, 0, s>>>(d_inst);
    return 2;
}

}  // namespace hac
