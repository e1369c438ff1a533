// End-of-iteration steps of Algorithm 1 as block-level device
// functions, shared by the per-iteration kernels and the fused cluster kernel:
//   iteration_best   T_ib = argmin over ants of L (ties to the lower ant), copied out
//   global_best      restart-best T_rb (schedule = 1), new global best -> T_gb,
//                    L_gb and bounds (eq. tau_init / tau_min_nols from L_gb);
//                    the elite T+ (T_ib, or T_rb every u_gb iterations) and
//                    its succ/pred; trace; t+1
//   update_slot      tau <- min(tau_max, max(tau_min, fl32(tau*(1-rho))
//                    [+ fl32(1/L(T+)) on T+ edges])) (eqs. pheromone_update,
//                    pheromone_delta) and choice = fl32(tau^alpha * W)
//   schedule end     (schedule = 1) every 100 iterations, when T_rb has not
//                    improved for more than 250 iterations, the branching
//                    factor; below 1 + 1e-5 a restart (tau <- tau_max, T_rb
//                    cleared, T_gb kept); then the next u_gb (Sec. III-B)
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
    const int t1 = st->t + 1;                                 // this iteration, counted from 1
    const bool rb_better = I.schedule && Lib < st->L_rb;
    const bool use_rb = I.schedule && t1 % st->u_gb == 0;
    __syncthreads();
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        const int u = I.ib_tour[s];
        if (better) I.gb_tour[s] = u;
        if (rb_better) I.rb_tour[s] = u;
    }
    __syncthreads();
    const int32_t *elite = use_rb ? I.rb_tour : I.ib_tour;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        const int u = elite[s], v = elite[s + 1 < n ? s + 1 : 0];
        I.succ[u] = v;
        I.pred[v] = u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (better) {
            st->L_gb = Lib;
            bounds_from(I, st, Lib);
        }
        if (rb_better) {
            st->L_rb = Lib;
            st->t_rbimp = t1;
        }
        st->L_dep = use_rb ? st->L_rb : Lib;
        st->bf_count = 0;
        const int t = t1 - 1;
        if (I.trace && t < I.iters) {
            I.trace[TRACE_W * t] = (double)st->ib;
            I.trace[TRACE_W * t + 1] = Lib;
            I.trace[TRACE_W * t + 2] = st->L_gb;
            I.trace[TRACE_W * t + 3] = st->L_rb;
            I.trace[TRACE_W * t + 4] = use_rb ? 1.0 : 0.0;
        }
        st->t = t1;
    }
    __syncthreads();
}

// u_gb from the iterations since the last restart (MMAS: 25, 5, 3, 2, 1)
__device__ __forceinline__ int ugb_of(int s)
{
    return s < 25 ? 25 : s < 75 ? 5 : s < 125 ? 3 : s < 250 ? 2 : 1;
}

// whether the iteration just finished (st->t) checks the branching factor
__device__ __forceinline__ bool schedule_check_due(const DevInst &I, const InstState *st)
{
    const int t1 = st->t;
    return I.schedule && t1 % 100 == 0 && t1 - st->t_rbimp > 250;
}

// branching count of row i: real slots with tau >= min + 0.05 (max - min), in FP64
__device__ __forceinline__ int row_branching(const DevInst &I, int i)
{
    const size_t r = (size_t)i * I.k_pad;
    double lo = __longlong_as_double(0x7ff0000000000000ll), hi = -lo;
    for (int c = 0; c < I.k_pad; ++c) {
        if (I.cand[r + c] < 0) continue;
        const double v = (double)I.tau[r + c];
        lo = v < lo ? v : lo;
        hi = v > hi ? v : hi;
    }
    const double cut = __dadd_rn(lo, __dmul_rn(0.05, __dsub_rn(hi, lo)));
    int cnt = 0;
    for (int c = 0; c < I.k_pad; ++c)
        if (I.cand[r + c] >= 0 && (double)I.tau[r + c] >= cut) ++cnt;
    return cnt;
}

// the branching factor from the summed counts is below lambda_bf = 1 + 1e-5
__device__ __forceinline__ bool schedule_restart(const DevInst &I, unsigned long long count)
{
    const double bf = __ddiv_rn((double)count, __dmul_rn((double)I.n, (double)I.degree_target));
    return bf < 1.0 + 1e-5;
}

// one thread: state after a restart (or none), then the next u_gb
__device__ __forceinline__ void schedule_finish(const DevInst &I, InstState *st, bool restart)
{
    const int t1 = st->t;
    if (restart) {
        st->L_rb = __longlong_as_double(0x7ff0000000000000ll);
        st->t_restart = t1;
        st->t_rbimp = t1;
        st->n_restarts += 1;
        if (I.trace && t1 - 1 < I.iters) {
            I.trace[TRACE_W * (t1 - 1) + 3] = st->L_rb;
            I.trace[TRACE_W * (t1 - 1) + 4] += 2.0;
        }
    }
    st->u_gb = ugb_of(t1 - st->t_restart);
}

// fl32(tau^alpha * W).  For alpha = 1 the FP64 product of two floats is exact
// (48 significant bits), so rounding it once to FP32 equals the FP32 product.
__device__ __forceinline__ float choice_value(const DevInst &I, float tau, float W)
{
    if (I.alpha == 1.0) return __fmul_rn(tau, W);
    const double a = det_exp(__dmul_rn(I.alpha, det_ln((double)tau)));
    return __double2float_rn(__dmul_rn(a, (double)W));
}

// one block per instance (per-iteration path): the end of the schedule
__device__ __forceinline__ void block_schedule_end(const DevInst &I, InstState *st)
{
    __shared__ unsigned long long cnt_s;
    __shared__ int restart_s;
    if (!I.schedule) return;
    const bool due = schedule_check_due(I, st);
    if (threadIdx.x == 0) { cnt_s = 0; restart_s = 0; }
    __syncthreads();
    if (due) {
        unsigned long long c = 0;
        for (int i = threadIdx.x; i < I.n; i += blockDim.x) c += (unsigned long long)row_branching(I, i);
        atomicAdd(&cnt_s, c);
        __syncthreads();
        if (threadIdx.x == 0) restart_s = schedule_restart(I, cnt_s) ? 1 : 0;
        __syncthreads();
        if (restart_s) {
            const float tmax = st->tau_max;
            for (size_t s = threadIdx.x; s < (size_t)I.n * I.k_pad; s += blockDim.x)
                if (I.cand[s] >= 0) {
                    I.tau[s] = tmax;
                    I.choice[s] = choice_value(I, tmax, I.W[s]);
                }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) schedule_finish(I, st, restart_s != 0);
    __syncthreads();
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
