// First-improvement 2-opt with geometric neighbour lists and don't-look bits
// (Sec. III-D), one warp per instance, applied to T_NN once (Algorithm 1's initialisation)
// and to the iteration-best tour before it updates the pheromone.
//
// Order of the search (it defines the result):
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
//
// Moves follow the FP64 gain (d_ij as in the length, gain = (d(a,dir a) -
// d(a,b)) + d(b,dir b) - d(dir a,dir b)), but most candidates are decided from
// FP32 copies: el[p] holds d(tour[p], tour[p+1]) in FP32 and nbrd32 the
// neighbour distances.  Each FP32 distance is within 4 units of 2^-24 (relative) of the
// FP64 one, so the FP32 estimate of the four-term gain is within about
// 8 * 2^-24 of the sum of the four magnitudes.  With tol = 4e-6 times that
// sum (plus 1e-18 for FP32 underflow), an estimate below 1e-10 - tol means the
// FP64 gain is certainly <= 1e-10, one above 1e-10 + tol that it is certainly
// above; only estimates in between are decided in FP64.  Likewise d(a, b) is
// compared with d(a, dir a) in FP32 with a relative margin of 4e-6 on either
// side.  The moves taken are therefore exactly those of the plain FP64 search;
// the FP32 edge lengths stored for the new edges are FP32 estimates too.
//
// Parallelism inside the sequential search: when more than LS_FEW of the
// next 32 tour positions hold cities whose bit is clear, a pass tests them at
// once with the FP32 test only, their candidate moves spread over the lanes;
// the cities before the first one that might move have no move and get their
// bit at once (as they would one by one, since examining a city without a move
// changes nothing else).  A city that might move, or the first clear one when
// few are clear, is examined by the whole warp, one neighbour per lane (FP32
// classes, then FP64 when the first candidate is undecided).  Segment
// reversals swap element pairs across lanes.
#pragma once

#include "lengths.cuh"

namespace hac {

constexpr unsigned FULL2 = 0xffffffffu;
constexpr float LS_G1_LO = 0.999996f;   // FP32 margin between d(a,b) and d(a,dir a): g1 <= 0 or > 0 for certain
constexpr int LS_FEW = 4;               // at most this many clear cities in 32 positions: one at a time

__device__ __forceinline__ int wrap_next(int p, int n) { return p + 1 < n ? p + 1 : 0; }
__device__ __forceinline__ int wrap_prev(int p, int n) { return p > 0 ? p - 1 : n - 1; }

// bring the cache lines of a global row of `bytes` bytes into L1 (no result)
__device__ __forceinline__ void ls_prefetch_row(const void *row, int bytes)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(row));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(static_cast<const char *>(row) + bytes - 1));
}

// the arrays of one search: shared memory (a kernel of its own) or the workspace
struct LsMem {
    int32_t *tour;      // the tour being improved
    int32_t *pos;       // pos[city]
    uint8_t *dlb;       // don't-look bit by city
    float *el;          // el[p] ~ d(tour[p], tour[p+1 mod n]), FP32
    const float2 *xy;   // coordinates
    int *coop = nullptr;   // shared command words of the helper warps (null: warp 0 alone)
    int coop_warps = 1;    // warps of the block (warp 0 searches, the others help)
};

// Helper warps.  The search is sequential and runs in warp 0; in a block of
// several warps the others wait at named barrier 1 and take their share of
// each long segment reversal (its element pairs are independent, so the
// result does not depend on who swaps which pair) and of each wide FP32
// pre-test of 32 positions (ls_first_may_move, more than 32 work items).
// Protocol: warp 0 writes a command to coop and every warp arrives at the
// barrier; then
//   1 (reverse i0 .. i0+len-1): every warp swaps its pairs, arrives again;
//   2 (pre-test of the staged cities): the block deals the items 32 * warps
//     at a time, each round ending at the barrier after the per-warp minima
//     are written; every thread reads the same minima, so all leave after
//     the same round (the first with a possible move);
//   3 (examine city a): warp 1 searches a's predecessor direction while
//     warp 0 searches the successor direction (both only read the tour),
//     writes what it found, and every warp arrives again; warp 0 takes the
//     successor move if there is one, else warp 1's (the order of the
//     sequential search);
//   0: the helpers return.
// Every path through the search ends with command 0.
constexpr int LS_COOP_LEN = 192;   // reversals of at least this many positions are shared
// coop words: [0] command (0 exit, 1 reverse, 2 pre-test, 3 examine), [1] i0,
// item count or city, [2] len; [3..8] warp 1's predecessor move (found, an, b,
// bn, d(a,b) and d(an,bn) as FP32 bits); from LS_ST the staged cities (al,
// an0, an1, c0, incl, da0, da1; 32 each); from LS_MIN the per-warp minima of
// two rounds (2 x 8)
constexpr int LS_ST = 10, LS_MIN = LS_ST + 7 * 32, LS_COOP_WORDS = LS_MIN + 16;
constexpr int LS_WARPS_MAX = 8;

__device__ __forceinline__ void ls_coop_bar(int warps)
{
    asm volatile("bar.sync 1, %0;" ::"r"(32 * warps) : "memory");
}

__device__ __forceinline__ float ls_d32(const float2 *xy, int u, int v)
{
    const float2 p = xy[u], q = xy[v];
    const float dx = __fsub_rn(q.x, p.x), dy = __fsub_rn(q.y, p.y);
    return __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
}

// the FP64 gain from FP32 estimates of its terms: 0 certainly <= LS_GAIN,
// 2 certainly above, 1 undecided
__device__ __forceinline__ int ls_gain_class(float da, float dab, float dbb, float dn)
{
    const float est = __fsub_rn(__fadd_rn(__fsub_rn(da, dab), dbb), dn);
    const float mag = __fadd_rn(__fadd_rn(da, dab), __fadd_rn(dbb, dn));
    const float tol = __fadd_rn(__fmul_rn(4e-6f, mag), 1e-18f);
    if (!(est > __fsub_rn((float)LS_GAIN, tol))) return 0;
    return est > __fadd_rn((float)LS_GAIN, tol) ? 2 : 1;
}

// false only if the FP64 gain is certainly <= LS_GAIN
__device__ __forceinline__ bool ls_may_improve(float da, float dab, float dbb, float dn)
{
    return ls_gain_class(da, dab, dbb, dn) != 0;
}

// the element swaps of reversing positions i0 .. i0+len-1 (mod n) that fall to
// thread `tid` of `nth`: tour/pos pairs and the inner edge lengths; the pairs
// of different t are disjoint, so each thread loads two pairs before it
// stores them
__device__ __forceinline__ void ls_reverse_part(const LsMem &M, int n, int i0, int len, int tid, int nth)
{
    const int h = len / 2;
    for (int t = tid; t < h; t += 2 * nth) {
        const bool two = t + nth < h;
        int p0 = i0 + t, q0 = i0 + len - 1 - t;
        int p1 = p0 + nth, q1 = q0 - nth;
        if (p0 >= n) p0 -= n;
        if (q0 >= n) q0 -= n;
        if (p1 >= n) p1 -= n;
        if (q1 >= n) q1 -= n;
        const int u0 = M.tour[p0], v0 = M.tour[q0];
        const int u1 = two ? M.tour[p1] : 0, v1 = two ? M.tour[q1] : 0;
        M.tour[p0] = v0;
        M.tour[q0] = u0;
        M.pos[v0] = p0;
        M.pos[u0] = q0;
        if (two) {
            M.tour[p1] = v1;
            M.tour[q1] = u1;
            M.pos[v1] = p1;
            M.pos[u1] = q1;
        }
    }
    const int he = (len - 1) / 2;
    for (int t = tid; t < he; t += 2 * nth) {
        const bool two = t + nth < he;
        int p0 = i0 + t, q0 = i0 + len - 2 - t;
        int p1 = p0 + nth, q1 = q0 - nth;
        if (p0 >= n) p0 -= n;
        if (q0 >= n) q0 -= n;
        if (p1 >= n) p1 -= n;
        if (q1 >= n) q1 -= n;
        const float u0 = M.el[p0], v0 = M.el[q0];
        const float u1 = two ? M.el[p1] : 0.0f, v1 = two ? M.el[q1] : 0.0f;
        M.el[p0] = v0;
        M.el[q0] = u0;
        if (two) {
            M.el[p1] = v1;
            M.el[q1] = u1;
        }
    }
}

// One pre-test work item: candidate move of city a in direction dir (0: succ,
// 1: pred) with its q-th neighbour; true unless the FP64 gain is certainly
// <= LS_GAIN.  an, da: the city's dir-neighbour and FP32 edge length.
__device__ __forceinline__ bool ls_item_may_improve(const DevInst &I, const LsMem &M, int n, int K, int a, int dir,
                                                   int q, int an, float da)
{
    const int b = I.nbr[(size_t)a * K + q];
    const float dab = I.nbrd32[(size_t)a * K + q];
    const int pb = M.pos[b];
    const int pe = dir == 0 ? pb : wrap_prev(pb, n);     // the edge (b, dir b)
    const int bn = M.tour[dir == 0 ? wrap_next(pb, n) : pe];
    return b != an && bn != a && ls_may_improve(da, dab, M.el[pe], ls_d32(M.xy, an, bn));
}

// The block's side of a shared pre-test (every thread of the block): items
// t = tid, tid + 32*warps, ... of the staged cities, in rounds; the first
// round with a possible move gives the answer (the smallest staged lane that
// owns one), as in the warp's own loop.  All threads return the same value.
__device__ __forceinline__ int ls_pretest_rounds(const DevInst &I, const LsMem &M, int n, int K, int total)
{
    const int *st = M.coop + LS_ST;
    const int *s_al = st, *s_an0 = st + 32, *s_an1 = st + 64, *s_c0 = st + 96, *s_incl = st + 128;
    const float *s_da0 = reinterpret_cast<const float *>(st + 160), *s_da1 = reinterpret_cast<const float *>(st + 192);
    int *mins = M.coop + LS_MIN;
    const int tid = (int)threadIdx.x, nth = 32 * M.coop_warps, w = tid >> 5;
    for (int base = 0, r = 0; base < total; base += nth, ++r) {
        const int t = base + tid;
        int c = 0;
        bool hit = false;
        if (t < total) {
#pragma unroll
            for (int s2 = 16; s2 >= 1; s2 >>= 1)
                if (s_incl[c + s2 - 1] <= t) c += s2;
            const int j = t - (c ? s_incl[c - 1] : 0);
            const int cc0 = s_c0[c];
            const int dir = j < cc0 ? 0 : 1;
            hit = ls_item_may_improve(I, M, n, K, s_al[c], dir, dir == 0 ? j : j - cc0,
                                      dir == 0 ? s_an0[c] : s_an1[c], dir == 0 ? s_da0[c] : s_da1[c]);
        }
        const unsigned wmin = __reduce_min_sync(FULL2, hit ? (unsigned)c : 32u);
        if ((tid & 31) == 0) mins[(r & 1) * 8 + w] = (int)wmin;
        ls_coop_bar(M.coop_warps);
        int first = 32;
        for (int q = 0; q < M.coop_warps; ++q) first = min(first, mins[(r & 1) * 8 + q]);
        if (first < 32) return first;
    }
    return 32;
}

__device__ __forceinline__ void ls_pred_search(const DevInst &I, const LsMem &M, int a);

// the helper warps' side of the protocol above (warps 1 .. coop_warps-1)
__device__ __forceinline__ void ls_coop_help(const DevInst &I, const LsMem &M)
{
    const int n = I.n, nth = 32 * M.coop_warps;
    for (;;) {
        ls_coop_bar(M.coop_warps);
        const int cmd = M.coop[0];
        if (cmd == 1) {
            ls_reverse_part(M, n, M.coop[1], M.coop[2], (int)threadIdx.x, nth);
            ls_coop_bar(M.coop_warps);
        } else if (cmd == 2) {
            ls_pretest_rounds(I, M, n, I.ls_k, M.coop[1]);
        } else if (cmd == 3) {
            if ((threadIdx.x >> 5) == 1) ls_pred_search(I, M, M.coop[1]);
            ls_coop_bar(M.coop_warps);
        } else {
            break;
        }
    }
}

// warp 0: releases the helper warps (the final arrival of the protocol)
__device__ __forceinline__ void ls_coop_end(const LsMem &M)
{
    if (!M.coop) return;
    if ((threadIdx.x & 31) == 0) M.coop[0] = 0;
    __syncwarp();
    ls_coop_bar(M.coop_warps);
}

// reverse so that (x, succ x), (y, succ y) become (x, y), (succ x, succ y);
// the inner edges of the reversed range swap, the two new edges get dxy, dss
__device__ __forceinline__ void apply_succ_move(const LsMem &M, int n, int x, int y, float dxy, float dss)
{
    const int lane = threadIdx.x & 31;
    int i0 = wrap_next(M.pos[x], n);
    int len = M.pos[y] - i0;
    if (len < 0) len += n;
    len += 1;
    if (2 * len > n) {
        i0 = wrap_next(M.pos[y], n);
        len = M.pos[x] - i0;
        if (len < 0) len += n;
        len += 1;
    }
    __syncwarp();
    if (M.coop && len >= LS_COOP_LEN) {
        if (lane == 0) { M.coop[0] = 1; M.coop[1] = i0; M.coop[2] = len; }
        __syncwarp();
        ls_coop_bar(M.coop_warps);
        ls_reverse_part(M, n, i0, len, lane, 32 * M.coop_warps);
        ls_coop_bar(M.coop_warps);
    } else {
        ls_reverse_part(M, n, i0, len, lane, 32);
    }
    __syncwarp();
    if (lane == 0) {
        M.el[wrap_prev(i0, n)] = dxy;
        int e = i0 + len - 1;
        if (e >= n) e -= n;
        M.el[e] = dss;
    }
    __syncwarp();
}

// FP32 pre-test of the clear cities of 32 consecutive positions (lane l holds
// the city al at position pp = p + l): the lane of the first city that might
// move, or 32.  A work item is one candidate move of one city: a direction and
// a neighbour b while d(a, b) is below d(a, dir a) (FP32, with the margin);
// the list ascends, so each direction's items are a prefix of the list.  The
// items of all cities are dealt to the lanes in position order, 32 at a time;
// after the first group with a possible move every earlier city has been
// tested in full, so the search stops there.
__device__ __forceinline__ int ls_first_may_move(const DevInst &I, const LsMem &M, int n, int K, bool clear, int al,
                                                 int pp)
{
    const int lane = threadIdx.x & 31;
    int an0 = 0, an1 = 0, c0 = 0, c1 = 0;
    float da0 = 0.0f, da1 = 0.0f;
    if (clear) {
        const int pv = wrap_prev(pp, n);
        an0 = M.tour[wrap_next(pp, n)];
        an1 = M.tour[pv];
        da0 = M.el[pp];
        da1 = M.el[pv];
        ls_prefetch_row(I.nbr + (size_t)al * K, K * 4);      // read by the work items below
        const float *nd = I.nbrd32 + (size_t)al * K;
        for (int k0 = 0; k0 < K; k0 += 4) {
            float lim[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                lim[q] = k0 + q < K ? __fmul_rn(nd[k0 + q], LS_G1_LO) : __int_as_float(0x7f800000);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                c0 += da0 > lim[q];
                c1 += da1 > lim[q];
            }
            if (!(da0 > lim[3] || da1 > lim[3])) break;
        }
    }
    const int cnt = c0 + c1;
    int incl = cnt;     // inclusive prefix sum of the item counts over the lanes
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const int v = __shfl_up_sync(FULL2, incl, s);
        if (lane >= s) incl += v;
    }
    const int excl = incl - cnt;
    const int total = __shfl_sync(FULL2, incl, 31);
    if (M.coop && total > 32) {    // more than one round: shared with the helper warps
        int *st = M.coop + LS_ST;
        st[lane] = al;
        st[32 + lane] = an0;
        st[64 + lane] = an1;
        st[96 + lane] = c0;
        st[128 + lane] = incl;
        st[160 + lane] = __float_as_int(da0);
        st[192 + lane] = __float_as_int(da1);
        if (lane == 0) { M.coop[0] = 2; M.coop[1] = total; }
        __syncwarp();
        ls_coop_bar(M.coop_warps);
        return ls_pretest_rounds(I, M, n, K, total);
    }
    for (int base = 0; base < total; base += 32) {
        const int t = base + lane;
        int c = 0;      // the lane whose city owns item t: the number of lanes with incl <= t
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1)
            if (__shfl_sync(FULL2, incl, c + s - 1) <= t) c += s;
        const int j = t - __shfl_sync(FULL2, excl, c);
        const int cc0 = __shfl_sync(FULL2, c0, c);
        const int a = __shfl_sync(FULL2, al, c);
        const int xan0 = __shfl_sync(FULL2, an0, c), xan1 = __shfl_sync(FULL2, an1, c);
        const float xda0 = __shfl_sync(FULL2, da0, c), xda1 = __shfl_sync(FULL2, da1, c);
        bool hit = false;
        if (t < total) {
            const int dir = j < cc0 ? 0 : 1;
            hit = ls_item_may_improve(I, M, n, K, a, dir, dir == 0 ? j : j - cc0, dir == 0 ? xan0 : xan1,
                                      dir == 0 ? xda0 : xda1);
        }
        const unsigned first = __reduce_min_sync(FULL2, hit ? (unsigned)c : 32u);
        if (first < 32u) return (int)first;
    }
    return 32;
}

// One direction of city a, one neighbour per lane: the first improving move
// in list order, decided in FP64.
__device__ __forceinline__ bool ls_find_move(const DevInst &I, const LsMem &M, int n, int K, int a, int dir,
                                             int nb, float nd32, double nd64, int &an, int &b, int &bn,
                                             float &dab, float &dn)
{
    const int lane = threadIdx.x & 31;
    const int pa = M.pos[a];
    an = dir == 0 ? M.tour[wrap_next(pa, n)] : M.tour[wrap_prev(pa, n)];
    const float da32 = M.el[dir == 0 ? pa : wrap_prev(pa, n)];
    bool cand = false, sure = false;
    int bb = 0, bbn = 0;
    float dnn = 0.0f;
    if (lane < K && da32 > __fmul_rn(nd32, LS_G1_LO)) {
        bb = nb;
        const int pb = M.pos[bb];
        bbn = dir == 0 ? M.tour[wrap_next(pb, n)] : M.tour[wrap_prev(pb, n)];
        if (!(bb == an || bbn == a)) {
            const float dbb = M.el[dir == 0 ? pb : wrap_prev(pb, n)];
            dnn = ls_d32(M.xy, an, bbn);
            const int g = ls_gain_class(da32, nd32, dbb, dnn);
            cand = g != 0;
            sure = g == 2 && __fmul_rn(da32, LS_G1_LO) > nd32;   // and d(a, b) < d(a, dir a) for certain
        }
    }
    const unsigned cm = __ballot_sync(FULL2, cand);
    if (!cm) return false;
    int src = __ffs(cm) - 1;
    if (!((__ballot_sync(FULL2, sure) >> src) & 1u)) {
        // the first candidate is undecided in FP32: decide all of them in FP64
        const double da = dist64(I, a, an);
        bool ok = false;
        if (cand) {
            const double g1 = __dsub_rn(da, nd64);
            if (g1 > 0.0) {
                const double gain = __dsub_rn(__dadd_rn(g1, dist64(I, bb, bbn)), dist64(I, an, bbn));
                ok = gain > LS_GAIN;
            }
        }
        const unsigned om = __ballot_sync(FULL2, ok);
        if (!om) return false;
        src = __ffs(om) - 1;
    }
    b = __shfl_sync(FULL2, bb, src);
    bn = __shfl_sync(FULL2, bbn, src);
    dab = __shfl_sync(FULL2, nd32, src);
    dn = __shfl_sync(FULL2, dnn, src);
    return true;
}

// Command 3, warp 1: the predecessor direction of city a, written to coop.
__device__ __forceinline__ void ls_pred_search(const DevInst &I, const LsMem &M, int a)
{
    const int lane = threadIdx.x & 31, K = I.ls_k;
    const int nb = lane < K ? I.nbr[(size_t)a * K + lane] : 0;
    const float nd32 = lane < K ? I.nbrd32[(size_t)a * K + lane] : 0.0f;
    const double nd64 = lane < K ? I.nbrd[(size_t)a * K + lane] : 0.0;
    int an = 0, b = 0, bn = 0;
    float dab = 0.0f, dn = 0.0f;
    const bool found = ls_find_move(I, M, I.n, K, a, 1, nb, nd32, nd64, an, b, bn, dab, dn);
    if (lane == 0) {
        M.coop[3] = found ? 1 : 0;
        M.coop[4] = an;
        M.coop[5] = b;
        M.coop[6] = bn;
        M.coop[7] = __float_as_int(dab);
        M.coop[8] = __float_as_int(dn);
    }
    __syncwarp();
}

// Improves `tour` (global memory) in place.  M holds the working arrays; when
// M.tour is not `tour`, the tour is copied in and back out.  The array
// pointers are copied into a local first: the search stores through generic
// pointers, and pointers read through a reference would be reloaded after
// every store.
static __device__ __noinline__ void warp_two_opt(const DevInst &I, int32_t *tour, const LsMem &Mref)
{
    const LsMem M = Mref;
    const int lane = threadIdx.x & 31;
    const int n = I.n, K = I.ls_k;
    if (M.tour != tour)
        for (int p = lane; p < n; p += 32) M.tour[p] = tour[p];
    __syncwarp();
    for (int p = lane; p < n; p += 32) M.pos[M.tour[p]] = p;
    for (int p = lane; p < n; p += 32) M.el[p] = ls_d32(M.xy, M.tour[p], M.tour[wrap_next(p, n)]);
    __syncwarp();
    const long long max_moves = 64LL * n + 1024;
    long long moves = 0;
    int round_moves;
    do {
        round_moves = 0;
        for (int p = lane; p < n; p += 32) M.dlb[p] = 0;
        __syncwarp();
        bool improved = true;
        while (improved && moves < max_moves) {
            improved = false;
            int p = 0;
            while (p < n && moves < max_moves) {
                const int pp = p + lane;
                const int al = pp < n ? M.tour[pp] : 0;
                const bool clear = pp < n && !M.dlb[al];
                const unsigned cm = __ballot_sync(FULL2, clear);
                if (!cm) { p += 32; continue; }
                if (__popc(cm) <= LS_FEW) {
                    p += __ffs(cm) - 1;     // few clear cities: the warp examines the first one
                } else {
                    // many: the next 32 positions at once, FP32 test only; the
                    // lists of the 32 positions after them are warmed for the next test
                    if (pp + 32 < n) {
                        const int ah = M.tour[pp + 32];
                        ls_prefetch_row(I.nbrd32 + (size_t)ah * K, K * 4);
                        ls_prefetch_row(I.nbr + (size_t)ah * K, K * 4);
                    }
                    const int f = ls_first_may_move(I, M, n, K, clear, al, pp);
                    if (clear && lane < f) M.dlb[al] = 1;   // examined, no move
                    __syncwarp();
                    if (f == 32) { p += 32; continue; }
                    p += f;
                }
                const int a = M.tour[p];
                const int nb = lane < K ? I.nbr[(size_t)a * K + lane] : 0;
                const float nd32 = lane < K ? I.nbrd32[(size_t)a * K + lane] : 0.0f;
                const double nd64 = lane < K ? I.nbrd[(size_t)a * K + lane] : 0.0;
                for (;;) {
                    bool moved = false;
                    int an = 0, b = 0, bn = 0, dir = -1;
                    float dab = 0.0f, dn = 0.0f;
                    if (M.coop) {   // both directions at once (command 3), successor first
                        if (lane == 0) { M.coop[0] = 3; M.coop[1] = a; }
                        __syncwarp();
                        ls_coop_bar(M.coop_warps);
                        const bool f0 = ls_find_move(I, M, n, K, a, 0, nb, nd32, nd64, an, b, bn, dab, dn);
                        ls_coop_bar(M.coop_warps);
                        if (f0) {
                            dir = 0;
                        } else if (M.coop[3]) {
                            dir = 1;
                            an = M.coop[4];
                            b = M.coop[5];
                            bn = M.coop[6];
                            dab = __int_as_float(M.coop[7]);
                            dn = __int_as_float(M.coop[8]);
                        }
                    } else {
                        for (int d = 0; d < 2 && dir < 0; ++d)
                            if (ls_find_move(I, M, n, K, a, d, nb, nd32, nd64, an, b, bn, dab, dn)) dir = d;
                    }
                    if (dir >= 0) {
                        if (dir == 0) apply_succ_move(M, n, a, b, dab, dn);
                        else apply_succ_move(M, n, an, bn, dn, dab);
                        if (lane == 0) { M.dlb[a] = 0; M.dlb[an] = 0; M.dlb[b] = 0; M.dlb[bn] = 0; }
                        __syncwarp();
                        moved = true;
                        improved = true;
                        ++round_moves;
                        ++moves;
                    }
                    if (!moved || moves >= max_moves) break;
                }
                if (lane == 0) M.dlb[a] = 1;
                __syncwarp();
                ++p;
            }
        }
    } while (round_moves > 0 && moves < max_moves);
    if (M.tour != tour)
        for (int p = lane; p < n; p += 32) tour[p] = M.tour[p];
    __syncwarp();
}

// the workspace arrays of an instance (no shared memory)
__device__ __forceinline__ LsMem ls_global(const DevInst &I, int32_t *tour)
{
    return LsMem{tour, I.ls_pos, I.ls_dlb, I.ls_el, reinterpret_cast<const float2 *>(I.xy)};
}

// the workspace arrays of ant a's own search (local_search = 2; ant-major tours)
__device__ __forceinline__ LsMem ls_ant(const DevInst &I, int a)
{
    const size_t o = (size_t)a * I.n;
    return LsMem{I.tours + o, I.lsa_pos + o, I.lsa_dlb + o, I.lsa_el + o, reinterpret_cast<const float2 *>(I.xy)};
}

// shared memory: tour, pos, el (4n bytes each), dlb (n bytes), then the
// coordinates at a 16-byte boundary when they fit as well
__host__ __device__ inline size_t ls_smem_core(int n) { return (size_t)n * 13; }
__host__ __device__ inline size_t ls_xy_offset(int n) { return ((size_t)n * 13 + 15) & ~(size_t)15; }
__host__ __device__ inline size_t ls_smem_full(int n) { return ls_xy_offset(n) + (size_t)n * 8; }

// arrays in `sm` (smem_bytes) where they fit, else `fallback`; one warp
// (copy = false: the same pointers without filling the coordinates, for the
// helper warps of a block)
__device__ __forceinline__ LsMem ls_shared(const DevInst &I, int32_t *tour, unsigned char *sm, size_t smem_bytes,
                                           const LsMem &fallback, bool copy = true)
{
    const int n = I.n;
    if (ls_smem_core(n) > smem_bytes) return fallback;
    LsMem M;
    M.tour = reinterpret_cast<int32_t *>(sm);
    M.pos = reinterpret_cast<int32_t *>(sm + (size_t)n * 4);
    M.el = reinterpret_cast<float *>(sm + (size_t)n * 8);
    M.dlb = sm + (size_t)n * 12;
    M.xy = reinterpret_cast<const float2 *>(I.xy);
    if (I.kind == 0 && ls_smem_full(n) <= smem_bytes) {
        float2 *sxy = reinterpret_cast<float2 *>(sm + ls_xy_offset(n));
        if (copy) {
            for (int p = threadIdx.x & 31; p < n; p += 32) sxy[p] = reinterpret_cast<const float2 *>(I.xy)[p];
            __syncwarp();
        }
        M.xy = sxy;
    }
    return M;
}

}  // namespace hac
