// End of an iteration as separate launches (the per-iteration path):
// k_select (iteration best), k_gb (global best, bounds, succ/pred) and
// k_update (bounded evaporation/deposit fused with the next choice_info).
// The arithmetic is in iter.cuh.
#include "iter.cuh"

namespace hac {

__global__ void k_select(const DevInst *insts)
{
    const DevInst &I = insts[blockIdx.x];
    InstState *st = I.st;
    if (st->t >= I.iters) {
        if (threadIdx.x == 0) st->active = 0;
        return;
    }
    block_iteration_best(I, st);
}

__global__ void k_gb(const DevInst *insts)
{
    const DevInst &I = insts[blockIdx.x];
    InstState *st = I.st;
    if (!st->active) return;
    block_global_best(I, st);
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
    const float omega = __double2float_rn(__dsub_rn(1.0, I.rho));
    const float delta = __double2float_rn(__ddiv_rn(1.0, st->L_dep));
    I.choice[s] = update_slot(I, s, (int)(s / I.k_pad), j, omega, delta, st->tau_min, st->tau_max);
}

// MMAS schedule end (restart check, next u_gb); one block per instance
__global__ void k_schedule(const DevInst *insts)
{
    const DevInst &I = insts[blockIdx.x];
    InstState *st = I.st;
    if (!st->active || !I.schedule) return;
    block_schedule_end(I, st);
}

void launch_two_opt_ib(const DevInst *d_inst, int count, int max_n, cudaStream_t s);
void launch_two_opt_all(const DevInst *d_inst, int count, int max_m, int max_n, cudaStream_t s);

int launch_iteration_tail(const DevInst *d_inst, int count, const int2 *d_slotmap,
                          int slotmap_len, bool any_ls, int max_n, int ls_all_m, cudaStream_t s)
{
    if (ls_all_m > 0) launch_two_opt_all(d_inst, count, ls_all_m, max_n, s);
    k_select<<<count, 256, 0, s>>>(d_inst);
    if (any_ls) launch_two_opt_ib(d_inst, count, max_n, s);
    k_gb<<<count, 256, 0, s>>>(d_inst);
    k_update<<<slotmap_len, 1024, 0, s>>>(d_inst, d_slotmap);
    k_schedule<<<count, 256, 0, s>>>(d_inst);
    return (any_ls ? 5 : 4) + (ls_all_m > 0 ? 1 : 0);
}

}  // namespace hac
