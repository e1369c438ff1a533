// Persistent fused iteration kernel: one thread-block cluster per instance runs
// whole MMAS iterations (the search loop of Algorithm 1) without leaving the GPU.
//
// Per instance the candidate table C_i (uint16 ids, padding slots hold n) and
// choice_info (FP32)
// live in the shared memory of the cluster's C CTAs, interleaved by row (row
// i in CTA i mod C).  Every construction step reads its row from local shared
// memory or, through the cluster's distributed shared memory, from a
// neighbouring SM, instead of from L2.  The ants are split over the CTAs, each
// ant being a warp segment (ant.cuh).  Per iteration:
//   construct (all CTAs) -> cluster barrier ->
//   iteration best, optional 2-opt of T_ib, global best, bounds, succ/pred
//   (CTA 0) -> cluster barrier ->
//   bounded evaporation/deposit of every row, new choice_info written to
//   shared memory (each CTA its own rows) -> cluster barrier.
// Cluster barriers are hardware barriers (no spinning); all CTAs of a cluster
// run the same number of iterations.  The arithmetic is exactly that of the
// per-iteration kernels (ant.cuh, iter.cuh, twoopt.cuh).
#include <cooperative_groups.h>

#include "ant_lane.cuh"
#include "ant_pair.cuh"
#include "iter.cuh"
#include "threeopt.cuh"

namespace cg = cooperative_groups;

namespace hac {

struct FusedArgs {
    const DevInst *insts;
    const int32_t *order;     // cluster -> instance
    const int32_t *iters_of;  // cluster -> iterations to run (null: iters_request for all)
    int iters_request;
    int rows_cap;             // shared-memory rows per CTA (max over the group)
    int kp_cap;               // max k_pad of the group
    int stride;               // words per visited mask (max over the group)
    int warps;                // warps per CTA
    int apw;
    int xy_cap;               // nodes whose coordinates fit in shared memory (0: read from global)
    int list_rows;            // lookup-list rows per CTA in shared memory (0: lists from global)
};

__host__ __device__ inline size_t fused_table_bytes(int rows_cap, int kp_cap)
{
    size_t ch = (size_t)rows_cap * kp_cap * 4;
    size_t ix = ((size_t)rows_cap * kp_cap * 2 + 15) & ~(size_t)15;
    return ch + ix;
}

// APW ants per warp: 2 or 4 (warp segments, ant.cuh), 16 (one ant per lane
// pair, ant_pair.cuh, NG slot groups per lane) or 32 (one ant per lane,
// ant_lane.cuh, NG candidate groups).  Shared memory per CTA:
//   choice rows (FP32) | candidate ids (uint16) | visited masks |
//   coordinates (optional) | lookup lists (uint16, optional)
template <int APW, int NG, int CLOG>
__global__ void __launch_bounds__(512, 1) k_fused(FusedArgs A)
{
    // this CTA is resident: a launch that depends on this one programmatically
    // (the next layout group) may start once every CTA of this grid is
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    constexpr int C = 1 << CLOG;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int cid = blockIdx.x >> CLOG;
    const DevInst &I = A.insts[A.order[cid]];
    InstState *st = I.st;
    extern __shared__ __align__(16) unsigned char smem[];
    float *sch = reinterpret_cast<float *>(smem);
    uint16_t *sidx = reinterpret_cast<uint16_t *>(smem + (size_t)A.rows_cap * A.kp_cap * 4);
    unsigned *svis = reinterpret_cast<unsigned *>(smem + fused_table_bytes(A.rows_cap, A.kp_cap));
    float2 *sxy = reinterpret_cast<float2 *>(smem + fused_table_bytes(A.rows_cap, A.kp_cap) +
                                             (size_t)A.warps * APW * A.stride * 4);
    uint16_t *slist = reinterpret_cast<uint16_t *>(reinterpret_cast<unsigned char *>(sxy) + (size_t)A.xy_cap * 8);

    const int n = I.n, kp = I.k_pad, m = I.m;
    const int R = (n + C - 1) >> CLOG;   // local rows: i = rank + C*l
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;

    for (int e = threadIdx.x; e < R * kp; e += blockDim.x) {
        const int l = e / kp, c = e - l * kp;
        const int i = rank + (l << CLOG);
        if (i < n) {
            const int j = I.cand[(size_t)i * kp + c];
            sidx[e] = (uint16_t)(j < 0 ? n : j);   // padding: node n, whose visited bit is preset
            sch[e] = I.choice[(size_t)i * kp + c];
        } else {
            sidx[e] = (uint16_t)n;
            sch[e] = 0.0f;
        }
    }
    const bool xy_shared = I.kind == 0 && I.n <= A.xy_cap;
    if (xy_shared)
        for (int e = threadIdx.x; e < n; e += blockDim.x) sxy[e] = reinterpret_cast<const float2 *>(I.xy)[e];
    const float2 *xy_scan = xy_shared ? sxy : reinterpret_cast<const float2 *>(I.xy);
    const bool list_shared = I.fbl != nullptr && A.list_rows >= R;
    if (list_shared)
        for (int e = threadIdx.x; e < R * FBL; e += blockDim.x) {
            const int l = e / FBL, k = e - l * FBL;
            const int i = rank + (l << CLOG);
            const int v = i < n ? I.fbl[(size_t)i * FBL + k] : -1;
            slist[e] = v < 0 ? (uint16_t)0xffff : (uint16_t)v;
        }
    ClusterRows<CLOG> rows;
    rows.idx_base = (uint32_t)__cvta_generic_to_shared(sidx);
    rows.ch_base = (uint32_t)__cvta_generic_to_shared(sch);
    rows.kp = kp;
    const ClusterList<CLOG> clist{list_shared ? (uint32_t)__cvta_generic_to_shared(slist) : 0u};
    const GlobalList glist{I.fbl};
    const int t0 = st->t;
    cl.sync();

    const int t_end = min(I.iters, t0 + (A.iters_of ? A.iters_of[cid] : A.iters_request));
    const int apc = (m + C - 1) >> CLOG;   // ants per CTA
    const int a_lo = rank * apc, a_hi = min(m, a_lo + apc);
    const float omega = __double2float_rn(__dsub_rn(1.0, I.rho));
    unsigned *vis_w = svis + (size_t)wib * APW * A.stride;

    for (int t = t0; t < t_end; ++t) {
        const int a_first = a_lo + wib * APW;
        if (a_first < a_hi) {
            if constexpr (APW == 32) {
                if (list_shared) build_tours_lane<NG>(I, rows, clist, t, a_first, a_hi, vis_w, xy_scan);
                else build_tours_lane<NG>(I, rows, glist, t, a_first, a_hi, vis_w, xy_scan);
            } else if constexpr (APW == 16) {
                if (list_shared) build_tours_pair<NG>(I, rows, clist, t, a_first, a_hi, vis_w, A.stride, xy_scan);
                else build_tours_pair<NG>(I, rows, glist, t, a_first, a_hi, vis_w, A.stride, xy_scan);
            } else {
                if (list_shared)
                    build_tours<APW, ClusterRows<CLOG>, ClusterList<CLOG>, NG>(I, rows, clist, t, a_first, a_hi,
                                                                             vis_w, A.stride, xy_scan);
                else
                    build_tours<APW, ClusterRows<CLOG>, GlobalList, NG>(I, rows, glist, t, a_first, a_hi, vis_w,
                                                                      A.stride, xy_scan);
            }
        }
        __syncthreads();
        fallback_distances(I, a_lo, a_hi);     // this CTA's ants only: no cluster barrier needed
        if (I.local_search == 2 || I.local_search == 4) {   // Algorithm 1's local search on every ant
            for (int a = a_first; a < min(a_first + APW, a_hi); ++a) {   // each warp its own
                int32_t *tour = I.tours + (size_t)a * n;
                if (I.local_search == 4) warp_three_opt(I, tour, ls_ant(I, a));
                else warp_two_opt_any(I, tour, ls_ant(I, a));
                const double L = warp_tour_length(I, tour);
                if (lane == 0) I.lens[a] = L;
            }
            __syncthreads();
        } else {
            ant_lengths(I, a_lo, a_hi);
        }
        __threadfence();
        cl.sync();
        if (rank == 0) {
            block_iteration_best(I, st);
            if (I.local_search == 1 || I.local_search == 3) {
                if (wib == 0) {
                    if (I.local_search == 3) warp_three_opt(I, I.ib_tour, ls_global(I, I.ib_tour));
                    else warp_two_opt_any(I, I.ib_tour, ls_global(I, I.ib_tour));
                    const double L = warp_tour_length(I, I.ib_tour);
                    if (lane == 0) st->L_ib = L;
                }
                __syncthreads();
            }
            block_global_best(I, st);
            __threadfence();
        }
        cl.sync();
        const float delta = __double2float_rn(__ddiv_rn(1.0, st->L_dep));
        const float tmin = st->tau_min, tmax = st->tau_max;
        for (int e = threadIdx.x; e < R * kp; e += blockDim.x) {
            const int j = sidx[e];
            if (j >= n) continue;   // padding
            const int l = e / kp, c = e - l * kp;
            const int i = rank + (l << CLOG);
            sch[e] = update_slot(I, (size_t)i * kp + c, i, j, omega, delta, tmin, tmax);
        }
        if (I.schedule) {   // restart check over every CTA's rows, then the next u_gb
            __threadfence();
            cl.sync();
            if (schedule_check_due(I, st)) {
                unsigned long long cnt = 0;
                for (int l = threadIdx.x; l < R; l += blockDim.x) {
                    const int i = rank + (l << CLOG);
                    if (i < n) cnt += (unsigned long long)row_branching(I, i);
                }
                if (cnt) atomicAdd(&st->bf_count, cnt);
                __threadfence();
                cl.sync();
                if (schedule_restart(I, st->bf_count)) {
                    for (int e = threadIdx.x; e < R * kp; e += blockDim.x) {
                        if ((int)sidx[e] >= n) continue;
                        const int l = e / kp, c = e - l * kp;
                        const size_t s = (size_t)(rank + (l << CLOG)) * kp + c;
                        I.tau[s] = tmax;
                        sch[e] = choice_value(I, tmax, I.W[s]);
                    }
                    if (rank == 0 && threadIdx.x == 0) schedule_finish(I, st, true);
                } else if (rank == 0 && threadIdx.x == 0) {
                    schedule_finish(I, st, false);
                }
            } else if (rank == 0 && threadIdx.x == 0) {
                schedule_finish(I, st, false);
            }
            __threadfence();
        }
        cl.sync();
    }
    for (int e = threadIdx.x; e < R * kp; e += blockDim.x) {
        const int l = e / kp, c = e - l * kp;
        const int i = rank + (l << CLOG);
        if (i < n) I.choice[(size_t)i * kp + c] = sch[e];
    }
    cl.sync();
}

// ------------------------------------------------------------ host side

template <typename Kern>
static cudaError_t launch_cluster(Kern kern, int clog, const FusedArgs &A, int clusters, int warps,
                                  size_t smem, cudaStream_t s, bool after_resident)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters << clog), 1, 1);
    cfg.blockDim = dim3((unsigned)(warps * 32), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1 << clog;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    // after_resident: start as soon as every CTA of the previous launch on the
    // stream is resident (programmatic dependent launch), not when it ends
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = after_resident ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kern, A);
}

size_t fused_smem_bytes(int rows_cap, int kp_cap, int warps, int apw, int stride, int xy_cap,
                        int list_rows)
{
    return fused_table_bytes(rows_cap, kp_cap) + (size_t)warps * apw * stride * 4 + (size_t)xy_cap * 8 +
           (size_t)list_rows * FBL * 2;
}

cudaError_t launch_fused(const DevInst *d_inst, const int32_t *d_order, const int32_t *d_iters,
                         int clusters, int clog, int apw, int warps, int rows_cap, int kp_cap, int stride,
                         int xy_cap, int list_rows, int iters, cudaStream_t s, bool after_resident)
{
    FusedArgs A{d_inst, d_order, d_iters, iters, rows_cap, kp_cap, stride, warps, apw, xy_cap, list_rows};
    const size_t smem = fused_smem_bytes(rows_cap, kp_cap, warps, apw, stride, xy_cap, list_rows);
#define CLUSTER_SWITCH(APWV, NGV) \
    switch (clog) { \
    case 0: return launch_cluster(k_fused<APWV, NGV, 0>, 0, A, clusters, warps, smem, s, after_resident); \
    case 1: return launch_cluster(k_fused<APWV, NGV, 1>, 1, A, clusters, warps, smem, s, after_resident); \
    case 2: return launch_cluster(k_fused<APWV, NGV, 2>, 2, A, clusters, warps, smem, s, after_resident); \
    default: return launch_cluster(k_fused<APWV, NGV, 3>, 3, A, clusters, warps, smem, s, after_resident); }
    if (apw == 32) {
        const int G = kp_cap / 4;
        if (G <= 3) { CLUSTER_SWITCH(32, 3) }
        if (G <= 5) { CLUSTER_SWITCH(32, 5) }
        CLUSTER_SWITCH(32, 8)
    }
    if (apw == 16) {
        const int G = kp_cap / 4;   // slot groups; lane h of a pair holds groups 2j + h
        if (G <= 4) { CLUSTER_SWITCH(16, 2) }
        if (G <= 6) { CLUSTER_SWITCH(16, 3) }
        CLUSTER_SWITCH(16, 4)
    }
    // 2 or 4 ants per warp: the group totals are gathered (5 groups for k <= 20, else 8)
    if (apw == 2) {
        if (kp_cap <= 20) { CLUSTER_SWITCH(2, 5) }
        CLUSTER_SWITCH(2, 8)
    }
    if (kp_cap <= 20) { CLUSTER_SWITCH(4, 5) }
    CLUSTER_SWITCH(4, 8)
#undef CLUSTER_SWITCH
}

}  // namespace hac
