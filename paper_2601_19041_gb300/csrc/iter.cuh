// End-of-iteration steps (Algorithm 1 lines 12-19) as block-level device
// functions, shared by the per-iteration kernels and the fused cluster kernel:
//   iteration_best   T_ib = argmin over ants of L (ties to the lower ant), copied out
//   global_best      new global best -> T_gb, L_gb and bounds (eq. tau_init /
//                    tau_min_nols from L_gb); succ/pred of T+ = T_ib; trace; t+1
//   update_slot      tau <- min(tau_max, max(tau_min, fl32(tau*(1-rho))
//                    [+ fl32(1/L_ib) on T+ edges])) (eqs. pheromone_update,
//                    pheromone_delta) and choice = fl32(tau^alpha * W)
// A symmetric instance deposits on the slot of either orientation of a tour
// edge, an ATSP on i -> succ(i) only; deposits go to stored candidate slots.
#pragma once

#include "hac_internal.cuh"

namespace hac {

// all threads of the block; returns the iteration-best ant (same in all threads)
__device__ __forceinline__ int block_iteration_best(const DevInst &I, InstState *st)
{
    __shared__ double rl[32];
    __shared__ int ra[32];
    __shared__ int ib_s;
    double bl = __longlong_as_double(0x7ff0000000000000ll);
    int ba = 0x7fffffff;
    for (int a = threadIdx.x; a < I.m; a += blockDim.x) {
        const double L = I.lens[a];
        if (L < bl || (L == bl && a < ba)) { bl = L; ba = a; }
    }
    for (int o = 16; o; o >>= 1) {
        const double l2 = __shfl_xor_sync(0xffffffffu, bl, o);
        const int a2 = __shfl_xor_sync(0xffffffffu, ba, o);
        if (l2 < bl || (l2 == bl && a2 < ba)) { bl = l2; ba = a2; }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { rl[w] = bl; ra[w] = ba; }
    __syncthreads();
    if (w == 0) {
        bl = lane < nw ? rl[lane] : __longlong_as_double(0x7ff0000000000000ll);
        ba = lane < nw ? ra[lane] : 0x7fffffff;
        for (int o = 16; o; o >>= 1) {
            const double l2 = __shfl_xor_sync(0xffffffffu, bl, o);
            const int a2 = __shfl_xor_sync(0xffffffffu, ba, o);
            if (l2 < bl || (l2 == bl && a2 < ba)) { bl = l2; ba = a2; }
        }
        if (lane == 0) {
            if (ba >= I.m) ba = 0;   // only if every length were NaN; keeps the copy in range
            ib_s = ba;
            st->ib = ba;
            st->L_ib = bl;
            st->active = 1;
        }
    }
    __syncthreads();
    const int ib = ib_s;
    const int32_t *src = I.tours + (size_t)ib * I.tour_sa;
    for (int s = threadIdx.x; s < I.n; s += blockDim.x) I.ib_tour[s] = src[(size_t)s * I.tour_ss];
    __syncthreads();
    return ib;
}

__device__ __forceinline__ void bounds_from(const DevInst &I, InstState *st, double L)
{
    const double tmax = __ddiv_rn(1.0, __dmul_rn(I.rho, L));
    double tmin;
    if (I.local_search) tmin = __ddiv_rn(tmax, __dmul_rn(2.0, (double)I.n));
    else tmin = __ddiv_rn(__dmul_rn(tmax, __dsub_rn(1.0, st->p_x)),
                          __dmul_rn(__ddiv_rn((double)(I.k_eff - 1), 2.0), st->p_x));
    st->tau_max64 = tmax;
    st->tau_min64 = tmin;
    st->tau_max = __double2float_rn(tmax);
    st->tau_min = __double2float_rn(tmin);
}

// all threads of the block, after T_ib (and its 2-opt) is final
__device__ __forceinline__ void block_global_best(const DevInst &I, InstState *st)
{
    const double Lib = st->L_ib;
    const bool better = Lib < st->L_gb;
    const int n = I.n;
    __syncthreads();
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        const int u = I.ib_tour[s], v = I.ib_tour[s + 1 < n ? s + 1 : 0];
        I.succ[u] = v;
        I.pred[v] = u;
        if (better) I.gb_tour[s] = u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (better) {
            st->L_gb = Lib;
            bounds_from(I, st, Lib);
        }
        const int t = st->t;
        if (I.trace && t < I.iters) {
            I.trace[TRACE_W * t] = (double)st->ib;
            I.trace[TRACE_W * t + 1] = Lib;
            I.trace[TRACE_W * t + 2] = st->L_gb;
        }
        st->t = t + 1;
    }
    __syncthreads();
}

// fl32(tau^alpha * W).  For alpha = 1 the FP64 product of two floats is exact
// (48 significant bits), so rounding it once to FP32 equals the FP32 product.
__device__ __forceinline__ float choice_value(const DevInst &I, float tau, float W)
{
    if (I.alpha == 1.0) return __fmul_rn(tau, W);
    const double a = det_exp(__dmul_rn(I.alpha, det_ln((double)tau)));
    return __double2float_rn(__dmul_rn(a, (double)W));
}

// new tau of real slot s = (i, c) with candidate j; writes tau, returns choice
__device__ __forceinline__ float update_slot(const DevInst &I, size_t s, int i, int j, float omega,
                                             float delta, float tmin, float tmax)
{
    float x = __fmul_rn(I.tau[s], omega);
    if (I.succ[i] == j || (I.kind == 0 && I.pred[i] == j)) x = __fadd_rn(x, delta);
    const float y = x > tmin ? x : tmin;
    const float tau = y < tmax ? y : tmax;
    I.tau[s] = tau;
    return choice_value(I, tau, I.W[s]);
}

}  // namespace hac
