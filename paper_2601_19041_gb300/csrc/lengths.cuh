// Tour lengths, eq. (tour_length), in FP64.
//
// Summation order (shared with the CPU oracle): edge e joins tour[e] and
// tour[e+1] (the closing edge is e = n-1); edge e is added to partial sum
// e mod 32 in increasing e, and the 32 partials are combined by the pairwise
// tree.  A warp keeps partial l in lane l (one FP64 add per edge, all lanes
// busy) and combines the partials with a butterfly of shuffles (by
// commutativity every lane ends with the same tree value).  FP64 adds have a
// long latency on GB300, so an ant's chain is n/32 + 5 adds long instead of n.
//
// Construction records the chosen slot of every step; the d of a candidate
// step is the slot's precomputed distance.  Nearest-unvisited steps are listed
// per ant and get their d from a full-width pass, together with the closing
// edge (stored at step index 0).
#pragma once

#include "hac_internal.cuh"

namespace hac {

constexpr uint8_t SLOT_FALLBACK = 0xff;   // slot record of a nearest-unvisited step

__device__ __forceinline__ size_t step_ix(const DevInst &I, int a, int s)
{
    return (size_t)a * I.tour_sa + (size_t)s * I.tour_ss;
}

// d of the listed nearest-unvisited steps and of the closing edge of ants
// [a_lo, a_hi) (at most 1024 ants): the CTA flattens all (ant, entry) pairs
// and every thread takes several, so many FP64 square roots are in flight.
// Call with all threads of the block.
__device__ __forceinline__ void fallback_distances(const DevInst &I, int a_lo, int a_hi)
{
    __shared__ int off[1025];
    const int n = I.n, na = a_hi > a_lo ? a_hi - a_lo : 0;   // a CTA may own no ant
    // exclusive prefix over (fallbacks + 1 closing edge) per ant
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int q = 0; q < na; ++q) { off[q] = acc; acc += I.fbcnt[a_lo + q] + 1; }
        off[na] = acc;
    }
    __syncthreads();
    const int total = off[na];
    for (int e0 = threadIdx.x; e0 < total; e0 += 4 * blockDim.x) {
        int from[4], to[4];
        size_t ix[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = e0 + k * blockDim.x;
            ix[k] = (size_t)-1;
            if (e >= total) continue;
            int lo = 0, hi = na - 1;           // ant of entry e: last q with off[q] <= e
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (off[mid] <= e) lo = mid; else hi = mid - 1;
            }
            const int a = a_lo + lo, kk = e - off[lo];
            if (kk < I.fbcnt[a]) {
                const int s = I.fbs[(size_t)a * n + kk];
                from[k] = I.tours[step_ix(I, a, s - 1)];
                to[k] = I.tours[step_ix(I, a, s)];
                ix[k] = step_ix(I, a, s);
            } else {                           // closing edge, stored at step 0
                from[k] = I.tours[step_ix(I, a, n - 1)];
                to[k] = I.tours[step_ix(I, a, 0)];
                ix[k] = step_ix(I, a, 0);
            }
        }
        double d[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) d[k] = ix[k] != (size_t)-1 ? dist64(I, from[k], to[k]) : 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) if (ix[k] != (size_t)-1) I.dstep[ix[k]] = d[k];
    }
    if (threadIdx.x == 0) atomicAdd(&I.st->n_fallback, (unsigned long long)(total - na));
    __syncthreads();
}

// lengths of NA ants at once (whole warp; results in every lane): the loops
// of the NA ants share one body, so their FP64 chains overlap
template <int NA>
__device__ __forceinline__ void warp_ant_lengths(const DevInst &I, const int (&ants)[NA], double (&out)[NA])
{
    const int lane = threadIdx.x & 31, n = I.n, kp = I.k_pad;
    const double *__restrict__ cdist = I.cdist;
    double P[NA];
#pragma unroll
    for (int h = 0; h < NA; ++h) P[h] = 0.0;
    constexpr int U = 4;   // edges per ant whose loads are in flight together
    int e = lane;
    for (; e + 32 * (U - 1) < n - 1; e += 32 * U) {
        int from[NA][U];
        uint8_t c[NA][U];
#pragma unroll
        for (int h = 0; h < NA; ++h)
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const int s = e + 32 * k + 1;             // the edge enters step s (< n)
                from[h][k] = I.tours[step_ix(I, ants[h], s - 1)];
                c[h][k] = I.slots[step_ix(I, ants[h], s)];
            }
        double d[NA][U];
#pragma unroll
        for (int h = 0; h < NA; ++h)
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const int s = e + 32 * k + 1;
                d[h][k] = c[h][k] != SLOT_FALLBACK ? cdist[(size_t)from[h][k] * kp + c[h][k]]
                                                   : I.dstep[step_ix(I, ants[h], s)];
            }
#pragma unroll
        for (int k = 0; k < U; ++k)
#pragma unroll
            for (int h = 0; h < NA; ++h) P[h] = __dadd_rn(P[h], d[h][k]);
    }
    for (; e < n; e += 32) {
#pragma unroll
        for (int h = 0; h < NA; ++h) {
            const int a = ants[h];
            double d;
            if (e == n - 1) {
                d = I.dstep[step_ix(I, a, 0)];            // closing edge
            } else {
                const uint8_t c = I.slots[step_ix(I, a, e + 1)];
                d = c != SLOT_FALLBACK ? cdist[(size_t)I.tours[step_ix(I, a, e)] * kp + c]
                                       : I.dstep[step_ix(I, a, e + 1)];
            }
            P[h] = __dadd_rn(P[h], d);
        }
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1)
#pragma unroll
        for (int h = 0; h < NA; ++h) P[h] = __dadd_rn(P[h], __shfl_xor_sync(0xffffffffu, P[h], o));
#pragma unroll
    for (int h = 0; h < NA; ++h) out[h] = P[h];
}

// lengths of ants [a_lo, a_hi): one warp per ant, two ants per warp at a time
__device__ __forceinline__ void ant_lengths(const DevInst &I, int a_lo, int a_hi)
{
    const int wib = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int a = a_lo + wib; a < a_hi; a += 2 * nw) {
        const int b = a + nw;
        if (b < a_hi) {
            const int ab[2] = {a, b};
            double L[2];
            warp_ant_lengths<2>(I, ab, L);
            if (lane == 0) { I.lens[a] = L[0]; I.lens[b] = L[1]; }
        } else {
            const int a1[1] = {a};
            double L[1];
            warp_ant_lengths<1>(I, a1, L);
            if (lane == 0) I.lens[a] = L[0];
        }
    }
}

// length of an explicit tour (T_NN, T_ib after 2-opt), whole warp, same order
__device__ __forceinline__ double warp_tour_length(const DevInst &I, const int32_t *tour)
{
    const int lane = threadIdx.x & 31, n = I.n;
    double P = 0.0;
    for (int e = lane; e < n; e += 32) P = __dadd_rn(P, dist64(I, tour[e], tour[e + 1 < n ? e + 1 : 0]));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) P = __dadd_rn(P, __shfl_xor_sync(0xffffffffu, P, o));
    return P;
}

}  // namespace hac
