// End of an iteration, Algorithm 1 lines 12-19:
//   k_select   iteration-best ant (ties to the lower ant), T_ib copied out
//   k_gb       new global best -> T_gb, L_gb and bounds recomputed (eq.
//              tau_init / tau_min_nols from L_gb); succ/pred of T+ = T_ib
//   k_update   every candidate slot: tau <- min(tau_max, max(tau_min,
//              fl32(tau*(1-rho)) [+ fl32(1/L_ib) on T+ edges])) (eqs.
//              pheromone_update, pheromone_delta), fused with the next
//              iteration's choice = fl32(tau^alpha * W) (eq. transition)
// A symmetric instance deposits on the slot of either orientation of a tour
// edge, an ATSP on i -> succ(i) only; deposits go to stored candidate slots.
#include "hac_internal.cuh"

namespace hac {

constexpr unsigned FULLU = 0xffffffffu;

__global__ void k_select(const DevInst *insts)
{
    const DevInst &I = insts[blockIdx.x];
    InstState *st = I.st;
    if (st->t >= I.iters) {
        if (threadIdx.x == 0) st->active = 0;
        return;
    }
    __shared__ double rl[32];
    __shared__ int ra[32];
    __shared__ int ib_s;
    double bl = __longlong_as_double(0x7ff0000000000000ll);
    int ba = 0x7fffffff;
    for (int a = threadIdx.x; a < I.m; a += blockDim.x) {
        double L = I.lens[a];
        if (L < bl || (L == bl && a < ba)) { bl = L; ba = a; }
    }
    for (int o = 16; o; o >>= 1) {
        double l2 = __shfl_xor_sync(FULLU, bl, o);
        int a2 = __shfl_xor_sync(FULLU, ba, o);
        if (l2 < bl || (l2 == bl && a2 < ba)) { bl = l2; ba = a2; }
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { rl[w] = bl; ra[w] = ba; }
    __syncthreads();
    if (w == 0) {
        bl = lane < nw ? rl[lane] : __longlong_as_double(0x7ff0000000000000ll);
        ba = lane < nw ? ra[lane] : 0x7fffffff;
        for (int o = 16; o; o >>= 1) {
            double l2 = __shfl_xor_sync(FULLU, bl, o);
            int a2 = __shfl_xor_sync(FULLU, ba, o);
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
    const int32_t *src = I.tours + (size_t)ib_s * I.n;
    for (int s = threadIdx.x; s < I.n; s += blockDim.x) I.ib_tour[s] = src[s];
}

__device__ __forceinline__ void bounds_from(const DevInst &I, InstState *st, double L)
{
    double tmax = __ddiv_rn(1.0, __dmul_rn(I.rho, L));
    double tmin;
    if (I.local_search) tmin = __ddiv_rn(tmax, __dmul_rn(2.0, (double)I.n));
    else tmin = __ddiv_rn(__dmul_rn(tmax, __dsub_rn(1.0, st->p_x)),
                          __dmul_rn(__ddiv_rn((double)(I.k_eff - 1), 2.0), st->p_x));
    st->tau_max64 = tmax; st->tau_min64 = tmin;
    st->tau_max = __double2float_rn(tmax);
    st->tau_min = __double2float_rn(tmin);
}

__global__ void k_gb(const DevInst *insts)
{
    const DevInst &I = insts[blockIdx.x];
    InstState *st = I.st;
    if (!st->active) return;
    const double Lib = st->L_ib;
    const bool better = Lib < st->L_gb;
    const int n = I.n;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        int u = I.ib_tour[s], v = I.ib_tour[s + 1 < n ? s + 1 : 0];
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
        int t = st->t;
        if (I.trace && t < I.iters) {
            I.trace[TRACE_W * t] = (double)st->ib;
            I.trace[TRACE_W * t + 1] = Lib;
            I.trace[TRACE_W * t + 2] = st->L_gb;
        }
        st->t = t + 1;
    }
}

__device__ __forceinline__ float choice_value(const DevInst &I, float tau, float W)
{
    double a = I.alpha == 1.0 ? (double)tau : det_exp(__dmul_rn(I.alpha, det_ln((double)tau)));
    return __double2float_rn(__dmul_rn(a, (double)W));
}

__global__ void k_update(const DevInst *insts, const int2 *slotmap)
{
    const int2 sm = slotmap[blockIdx.x];
    const DevInst &I = insts[sm.x];
    const InstState *st = I.st;
    if (!st->active) return;
    const size_t s = (size_t)sm.y + threadIdx.x;
    if (s >= (size_t)I.n * I.k_pad) return;
    const int j = I.cand[s];
    if (j < 0) return;
    const int i = (int)(s / I.k_pad);
    const float omega = __double2float_rn(__dsub_rn(1.0, I.rho));
    const float delta = __double2float_rn(__ddiv_rn(1.0, st->L_ib));
    float x = __fmul_rn(I.tau[s], omega);
    if (I.succ[i] == j || (I.kind == 0 && I.pred[i] == j)) x = __fadd_rn(x, delta);
    const float y = x > st->tau_min ? x : st->tau_min;
    const float tau = y < st->tau_max ? y : st->tau_max;
    I.tau[s] = tau;
    I.choice[s] = choice_value(I, tau, I.W[s]);
}

void launch_two_opt_ib(const DevInst *d_inst, int count, cudaStream_t s);

int launch_iteration_tail(const DevInst *d_inst, int count, const int2 *d_slotmap,
                          int slotmap_len, bool any_ls, cudaStream_t s)
{
    k_select<<<count, 256, 0, s>>>(d_inst);
    if (any_ls) launch_two_opt_ib(d_inst, count, s);
    k_gb<<<count, 256, 0, s>>>(d_inst);
    k_update<<<slotmap_len, 1024, 0, s>>>(d_inst, d_slotmap);
    return any_ls ? 4 : 3;
}

}  // namespace hac
