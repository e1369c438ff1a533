// First-improvement 2-opt with geometric neighbour lists and don't-look bits
// (Sec. III-D), one warp per instance, applied to T_NN once (Alg. 1 line 4)
// and to the iteration-best tour before it updates the pheromone.
//
// The search is sequential by definition; the warp parallelises inside it:
// the up-to-32 neighbour moves of a city are evaluated by one lane each and
// the first improving one in list order is taken by ballot + ffs; don't-look
// bits of 32 tour positions are tested per ballot; segment reversals swap
// element pairs across lanes.  Order of the search:
//   rounds start with all bits clear; a round repeats passes over the tour
//   positions until a pass makes no move; the search ends after a round whose
//   first pass made no move (a local optimum of the neighbour-list moves).
//   For city a, the successor direction is tried first, then the predecessor
//   direction; b runs over nbr(a) in (d, j) order while d(a, b) < d(a, dir a);
//   the first move with gain > 1e-10 is applied, the bits of a, dir a, b and
//   dir b are cleared and a is examined again; a city without a move gets its
//   bit set.  A move replacing (a, succ a), (b, succ b) by (a, b), (succ a,
//   succ b) reverses positions pos(succ a)..pos(b), or pos(succ b)..pos(a) when
//   the first range is longer than n/2; a predecessor move is the successor
//   move of (pred a, pred b).  A call stops after 64n + 1024 moves (a bound
//   that strictly decreasing tour lengths never reach in practice), so the
//   kernel always terminates.
#pragma once

#include "lengths.cuh"

namespace hac {

constexpr unsigned FULL2 = 0xffffffffu;

__device__ __forceinline__ int wrap_next(int p, int n) { return p + 1 < n ? p + 1 : 0; }
__device__ __forceinline__ int wrap_prev(int p, int n) { return p > 0 ? p - 1 : n - 1; }

// reverse so that (a, succ a), (b, succ b) become (a, b), (succ a, succ b)
__device__ __forceinline__ void apply_succ_move(int32_t *tour, int32_t *pos, int n, int a, int b)
{
    const int lane = threadIdx.x & 31;
    int i0 = wrap_next(pos[a], n);
    int len = pos[b] - i0;
    if (len < 0) len += n;
    len += 1;
    if (2 * len > n) {
        i0 = wrap_next(pos[b], n);
        len = pos[a] - i0;
        if (len < 0) len += n;
        len += 1;
    }
    __syncwarp();
    for (int x = lane; x < len / 2; x += 32) {
        int p = i0 + x;
        if (p >= n) p -= n;
        int q = i0 + len - 1 - x;
        if (q >= n) q -= n;
        int u = tour[p], v = tour[q];
        tour[p] = v;
        tour[q] = u;
        pos[v] = p;
        pos[u] = q;
    }
    __syncwarp();
}

static __device__ __noinline__ void warp_two_opt(const DevInst &I, int32_t *tour)
{
    const int lane = threadIdx.x & 31;
    const int n = I.n, K = I.ls_k;
    int32_t *pos = I.ls_pos;
    uint8_t *dlb = I.ls_dlb;
    for (int p = lane; p < n; p += 32) pos[tour[p]] = p;
    __syncwarp();
    const long long max_moves = 64LL * n + 1024;
    long long moves = 0;
    int round_moves;
    do {
        round_moves = 0;
        for (int p = lane; p < n; p += 32) dlb[p] = 0;
        __syncwarp();
        bool improved = true;
        while (improved && moves < max_moves) {
            improved = false;
            int p = 0;
            while (p < n && moves < max_moves) {
                const int pp = p + lane;
                const bool clear = pp < n && !dlb[tour[pp]];
                const unsigned cm = __ballot_sync(FULL2, clear);
                if (!cm) { p += 32; continue; }
                p += __ffs(cm) - 1;
                const int a = tour[p];
                for (;;) {
                    bool moved = false;
                    for (int dir = 0; dir < 2 && !moved; ++dir) {
                        const int pa = pos[a];
                        const int an = dir == 0 ? tour[wrap_next(pa, n)] : tour[wrap_prev(pa, n)];
                        const double da = dist64(I, a, an);
                        bool ok = false;
                        int b = 0, bn = 0;
                        if (lane < K) {
                            b = I.nbr[(size_t)a * K + lane];
                            const double g1 = __dsub_rn(da, I.nbrd[(size_t)a * K + lane]);
                            if (g1 > 0.0) {
                                const int pb = pos[b];
                                bn = dir == 0 ? tour[wrap_next(pb, n)] : tour[wrap_prev(pb, n)];
                                if (!(b == an || bn == a)) {
                                    const double gain =
                                        __dsub_rn(__dadd_rn(g1, dist64(I, b, bn)), dist64(I, an, bn));
                                    ok = gain > LS_GAIN;
                                }
                            }
                        }
                        const unsigned om = __ballot_sync(FULL2, ok);
                        if (om) {
                            const int src = __ffs(om) - 1;
                            b = __shfl_sync(FULL2, b, src);
                            bn = __shfl_sync(FULL2, bn, src);
                            if (dir == 0) apply_succ_move(tour, pos, n, a, b);
                            else apply_succ_move(tour, pos, n, an, bn);
                            if (lane == 0) { dlb[a] = 0; dlb[an] = 0; dlb[b] = 0; dlb[bn] = 0; }
                            __syncwarp();
                            moved = true;
                            improved = true;
                            ++round_moves;
                            ++moves;
                        }
                    }
                    if (!moved || moves >= max_moves) break;
                }
                if (lane == 0) dlb[a] = 1;
                __syncwarp();
                ++p;
            }
        }
    } while (round_moves > 0 && moves < max_moves);
}

}  // namespace hac
