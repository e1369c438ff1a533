// First-improvement 3-opt with geometric neighbour lists and don't-look bits
// (Sec. III-D), one warp per tour.
//
// The search (its order defines the result):
//   cities are examined in tour-position order, skipping those whose bit is
//   set; passes repeat until one makes no move, and rounds (all bits cleared)
//   until a round whose first pass made no move; a call stops after 64n + 1024
//   moves.  For the examined city t2 = a and t1 = dir(a) (successor
//   direction, then predecessor direction), t3 runs over nbr(t2) while
//   g1 = d(t1,t2) - d(t2,t3) > 0, and t4 over dir(t3), then the other tour
//   neighbour of t3.  With t4 = dir(t3) the 2-opt closing (t4, t1) is tried
//   first, gain (g1 + d34) - d41.  Then t5 runs over nbr(t4) while
//   g2 = (g1 + d34) - d(t4,t5) > 0 (t5 = t3 skipped) and t6 over (succ t5,
//   pred t5) (t6 = t1 skipped), gain (g2 + d56) - d61.  Removed edges (t1,t2),
//   (t3,t4)[, (t5,t6)], added (t2,t3), (t4,t5)[, (t6,t1)] or (t4,t1).  The
//   first candidate in this order whose gain exceeds 1e-10 and whose
//   reconnection leaves a single cycle is applied; its cities' bits are
//   cleared and a is examined again; a city without a move gets its bit set.
//   Gains are FP64, each operation rounded once, in the order written.
//
// Parallelism: one t5 per lane (both t6 of it), the first lane with an
// admissible move wins; the g1 values of all t3 are computed at once, one
// per lane.
//
// Applying a move: the removed edges sit at tour positions e_0 < e_1 (< e_2)
// (edge e joins tour[e] and tour[e+1 mod n]); positions outside
// [e_0 + 1, e_last] keep their cities and the middle positions receive the
// middle segments in the order and orientation in which the new cycle
// visits them after leaving tour[e_0].  The warp writes the middle through
// a scratch array (the FP32 edge array of the 2-opt, unused here).
#pragma once

#include "twoopt.cuh"

namespace hac {

__device__ __forceinline__ double ls3_d64(const float2 *xy, int u, int v)
{
    const float2 a = xy[u], b = xy[v];
    const double dx = __dsub_rn((double)b.x, (double)a.x), dy = __dsub_rn((double)b.y, (double)a.y);
    return __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

// A planned exchange: r removed edges at sorted positions e[], the middle
// segments j = seg[q] (positions e[j]+1 .. e[j+1]) in visiting order, rev[q]
// set when segment seg[q] is walked backwards.
struct Xchg {
    int r;
    int e[3];
    int seg[2], rev[2];
};

// position of the tour edge joining cities u and v, or -1 if they are not adjacent
__device__ __forceinline__ int ls3_edge(const LsMem &M, int n, int u, int v)
{
    const int pu = M.pos[u], pv = M.pos[v];
    if (pv == (pu + 1 == n ? 0 : pu + 1)) return pu;
    if (pu == (pv + 1 == n ? 0 : pv + 1)) return pv;
    return -1;
}

// Checks that removing the r edges {c[2k], c[2k+1]} and adding the r edges
// {c[2k+1], c[(2k+2) mod 2r]} (that is (t2,t3), (t4,t5), (t6,t1) for
// c = t1..t6, or (t2,t3), (t4,t1) for r = 2) leaves one cycle; plans it.
template <int R>
__device__ __forceinline__ bool ls3_plan(const LsMem &M, int n, const int (&c)[2 * R], Xchg &X)
{
    int e[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        e[k] = ls3_edge(M, n, c[2 * k], c[2 * k + 1]);
        if (e[k] < 0) return false;
    }
    // rank of each removed edge by position
    int rk[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        int q = 0;
#pragma unroll
        for (int l = 0; l < R; ++l) {
            if (l != k && e[l] == e[k]) return false;
            q += e[l] < e[k];
        }
        rk[k] = q;
    }
    // endpoint slot of city c[i] on its removed edge k = i/2: 2*rank + 0 when it
    // is tour[e] (end of the part before the edge), + 1 when it is tour[e+1]
    int slot[2 * R];
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) {
        const int k = i >> 1;
        slot[i] = 2 * rk[k] + (M.tour[e[k]] == c[i] ? 0 : 1);
    }
    // added edge i joins slot[2i+1] and slot[(2i+2) mod 2R]
    int partner[2 * R];
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) partner[i] = -1;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int u = slot[2 * i + 1], v = slot[(2 * i + 2) % (2 * R)];
        if (u == v || partner[u] >= 0 || partner[v] >= 0) return false;
        partner[u] = v;
        partner[v] = u;
    }
    // walk from the end of the fixed part (slot 0) until its start (slot 2R-1);
    // middle segment j starts at slot 2j+1 and ends at slot 2j+2
    bool used[R - 1];
#pragma unroll
    for (int j = 0; j < R - 1; ++j) used[j] = false;
    int cur = 0, cnt = 0;
#pragma unroll
    for (int step = 0; step < R; ++step) {
        const int s = partner[cur];
        if (s == 2 * R - 1) break;
        if (s == 0) return false;
        const bool back = (s & 1) == 0;
        const int j = back ? (s >> 1) - 1 : (s - 1) >> 1;
        if (j < 0 || j >= R - 1 || used[j] || cnt >= R - 1) return false;
        used[j] = true;
        X.seg[cnt] = j;
        X.rev[cnt] = back ? 1 : 0;
        ++cnt;
        cur = back ? 2 * j + 1 : 2 * j + 2;
    }
    if (cnt != R - 1 || partner[cur] != 2 * R - 1) return false;
    X.r = R;
    // sorted positions
#pragma unroll
    for (int k = 0; k < R; ++k) X.e[rk[k]] = e[k];
    return true;
}

// rewrites the middle positions of the planned exchange (whole warp)
__device__ __forceinline__ void ls3_apply(const LsMem &M, const Xchg &X)
{
    const int lane = threadIdx.x & 31;
    int32_t *tmp = reinterpret_cast<int32_t *>(M.el);
    const int lo = X.e[0] + 1;
    const int a0 = X.e[X.seg[0]] + 1, b0 = X.e[X.seg[0] + 1];
    const int len0 = b0 - a0 + 1;
    int a1 = 0, b1 = -1;
    if (X.r == 3) { a1 = X.e[X.seg[1]] + 1; b1 = X.e[X.seg[1] + 1]; }
    const int total = len0 + (b1 - a1 + 1);
    __syncwarp();
    for (int w = lane; w < total; w += 32) {
        int src;
        if (w < len0) src = X.rev[0] ? b0 - w : a0 + w;
        else src = X.rev[1] ? b1 - (w - len0) : a1 + (w - len0);
        tmp[w] = M.tour[src];
    }
    __syncwarp();
    for (int w = lane; w < total; w += 32) {
        const int c = tmp[w];
        M.tour[lo + w] = c;
        M.pos[c] = lo + w;
    }
    __syncwarp();
}

__device__ __forceinline__ Xchg ls3_bcast(const Xchg &X, int src)
{
    Xchg Y;
    Y.r = __shfl_sync(FULL2, X.r, src);
#pragma unroll
    for (int k = 0; k < 3; ++k) Y.e[k] = __shfl_sync(FULL2, X.e[k], src);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        Y.seg[k] = __shfl_sync(FULL2, X.seg[k], src);
        Y.rev[k] = __shfl_sync(FULL2, X.rev[k], src);
    }
    return Y;
}

// One examination of city a: finds and applies the first admissible move;
// true if a move was made (its cities' bits cleared).
__device__ __forceinline__ bool ls3_examine(const DevInst &I, const LsMem &M, int n, int K, int a)
{
    const int lane = threadIdx.x & 31;
    const float2 *xy = M.xy;
    auto succ = [&](int c) { const int p = M.pos[c]; return M.tour[p + 1 == n ? 0 : p + 1]; };
    auto pred = [&](int c) { const int p = M.pos[c]; return M.tour[p == 0 ? n - 1 : p - 1]; };
    for (int dir = 0; dir < 2; ++dir) {
        const int t2 = a, t1 = dir == 0 ? succ(a) : pred(a);
        const double d12 = ls3_d64(xy, t1, t2);
        const int t3l = lane < K ? I.nbr[(size_t)a * K + lane] : 0;
        const double g1l = lane < K ? __dsub_rn(d12, I.nbrd[(size_t)a * K + lane]) : 0.0;
        const unsigned stop = __ballot_sync(FULL2, lane >= K || !(g1l > 0.0));
        const int Q = stop ? __ffs(stop) - 1 : 32;   // t3 candidates 0..Q-1
        for (int q = 0; q < Q; ++q) {
            const int t3 = __shfl_sync(FULL2, t3l, q);
            const double g1 = __shfl_sync(FULL2, g1l, q);
            for (int c4 = 0; c4 < 2; ++c4) {
                const int t4 = (c4 == 0) == (dir == 0) ? succ(t3) : pred(t3);
                if ((t3 == t1 && t4 == t2) || (t3 == t2 && t4 == t1)) continue;
                const double d34 = ls3_d64(xy, t3, t4);
                if (c4 == 0 && t4 != t1) {
                    const double gain = __dsub_rn(__dadd_rn(g1, d34), ls3_d64(xy, t4, t1));
                    if (gain > LS_GAIN) {
                        const int c[4] = {t1, t2, t3, t4};
                        Xchg X;
                        if (ls3_plan<2>(M, n, c, X)) {
                            ls3_apply(M, X);
                            if (lane == 0) { M.dlb[t1] = 0; M.dlb[t2] = 0; M.dlb[t3] = 0; M.dlb[t4] = 0; }
                            __syncwarp();
                            return true;
                        }
                    }
                }
                const double g1b = __dadd_rn(g1, d34);
                const int t5 = lane < K ? I.nbr[(size_t)t4 * K + lane] : 0;
                const double g2 = lane < K ? __dsub_rn(g1b, I.nbrd[(size_t)t4 * K + lane]) : 0.0;
                const unsigned stop5 = __ballot_sync(FULL2, lane >= K || !(g2 > 0.0));
                const int R5 = stop5 ? __ffs(stop5) - 1 : 32;
                int hit = -1;
                Xchg X;
                if (lane < R5 && t5 != t3) {
#pragma unroll
                    for (int c6 = 0; c6 < 2 && hit < 0; ++c6) {
                        const int t6 = c6 == 0 ? succ(t5) : pred(t5);
                        if (t6 == t1) continue;
                        const double gain = __dsub_rn(__dadd_rn(g2, ls3_d64(xy, t5, t6)), ls3_d64(xy, t6, t1));
                        if (!(gain > LS_GAIN)) continue;
                        const int c[6] = {t1, t2, t3, t4, t5, t6};
                        if (ls3_plan<3>(M, n, c, X)) hit = c6;
                    }
                }
                const unsigned hm = __ballot_sync(FULL2, hit >= 0);
                if (hm) {
                    const int src = __ffs(hm) - 1;
                    const Xchg Y = ls3_bcast(X, src);
                    const int w5 = __shfl_sync(FULL2, t5, src);
                    const int w6 = __shfl_sync(FULL2, hit == 0 ? succ(t5) : hit == 1 ? pred(t5) : 0, src);
                    ls3_apply(M, Y);
                    if (lane == 0) {
                        M.dlb[t1] = 0; M.dlb[t2] = 0; M.dlb[t3] = 0; M.dlb[t4] = 0; M.dlb[w5] = 0; M.dlb[w6] = 0;
                    }
                    __syncwarp();
                    return true;
                }
            }
        }
    }
    return false;
}

// ---------------------------------------------------------------------------
// Directed 2-opt for the ATSP (Sec. III-D; the reading of the Jonker-Volgenant
// based 2-opt): the move removes two arcs, adds two arcs and reverses the
// path between them, so its gain adds the path's forward arc sum F and
// subtracts its backward sum R.  Examined city a, successor side first:
//   a+ = succ(a), b over nbr(a) while g1 = c(a,a+) - c(a,b) > 0 (b = a+ or
//   succ(b) = a skipped): remove (a,a+), (b,b+), add (a,b), (a+,b+),
//   reverse a+ .. b, gain = (((g1 + c(b,b+)) - c(a+,b+)) + F) - R;
//   predecessor side: a- = pred(a), g1 = c(a-,a) - c(a,b) (b = a- or
//   pred(b) = a skipped): remove (a-,a), (b-,b), add (a-,b-), (a,b), reverse
//   a .. b-, gain = (((g1 + c(b-,b)) - c(a-,b-)) + F) - R.
// F and R are summed in the order of the tour length (arc k of the path into
// lane k mod 32, then the pairwise tree), the path always reversed in place.

__device__ __forceinline__ double ls_arc(const DevInst &I, int n, int u, int v)
{
    return (double)I.cost[(size_t)u * n + v];
}

// forward (backward = false) or backward arc sum of the path of len cities
// starting at position i0 (whole warp, every lane gets the result)
__device__ __forceinline__ double ls_path_cost(const DevInst &I, const LsMem &M, int n, int i0, int len, bool backward)
{
    const int lane = threadIdx.x & 31;
    double P = 0.0;
    for (int k = lane; k + 1 < len; k += 32) {
        int p0 = i0 + k, p1 = i0 + k + 1;
        if (p0 >= n) p0 -= n;
        if (p1 >= n) p1 -= n;
        const int u = M.tour[p0], v = M.tour[p1];
        P = __dadd_rn(P, backward ? ls_arc(I, n, v, u) : ls_arc(I, n, u, v));
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) P = __dadd_rn(P, __shfl_xor_sync(FULL2, P, o));
    return P;
}

// reverses positions i0 .. i0+len-1 (cyclic) in place (whole warp)
__device__ __forceinline__ void ls_reverse_path(const LsMem &M, int n, int i0, int len)
{
    const int lane = threadIdx.x & 31;
    __syncwarp();
    for (int t = lane; t < len / 2; t += 32) {
        int p = i0 + t, q = i0 + len - 1 - t;
        if (p >= n) p -= n;
        if (q >= n) q -= n;
        const int u = M.tour[p], v = M.tour[q];
        M.tour[p] = v;
        M.tour[q] = u;
        M.pos[v] = p;
        M.pos[u] = q;
    }
    __syncwarp();
}

__device__ __forceinline__ bool ls2d_examine(const DevInst &I, const LsMem &M, int n, int K, int a)
{
    const int lane = threadIdx.x & 31;
    for (int dir = 0; dir < 2; ++dir) {
        const int pa = M.pos[a];
        const int x = dir == 0 ? M.tour[pa + 1 == n ? 0 : pa + 1] : M.tour[pa == 0 ? n - 1 : pa - 1];
        const double cx = dir == 0 ? ls_arc(I, n, a, x) : ls_arc(I, n, x, a);
        const int bl = lane < K ? I.nbr[(size_t)a * K + lane] : 0;
        const double g1l = lane < K ? __dsub_rn(cx, I.nbrd[(size_t)a * K + lane]) : 0.0;
        const unsigned stop = __ballot_sync(FULL2, lane >= K || !(g1l > 0.0));
        const int Q = stop ? __ffs(stop) - 1 : 32;
        for (int q = 0; q < Q; ++q) {
            const int b = __shfl_sync(FULL2, bl, q);
            const double g1 = __shfl_sync(FULL2, g1l, q);
            const int pb = M.pos[b];
            const int y = dir == 0 ? M.tour[pb + 1 == n ? 0 : pb + 1] : M.tour[pb == 0 ? n - 1 : pb - 1];
            if (b == x || y == a) continue;
            const int i0 = dir == 0 ? M.pos[x] : pa;
            const int i1 = dir == 0 ? pb : M.pos[y];
            int len = i1 - i0;
            if (len < 0) len += n;
            len += 1;
            const double F = ls_path_cost(I, M, n, i0, len, false);
            const double R = ls_path_cost(I, M, n, i0, len, true);
            const double cby = dir == 0 ? ls_arc(I, n, b, y) : ls_arc(I, n, y, b);
            const double gain = __dsub_rn(__dadd_rn(__dsub_rn(__dadd_rn(g1, cby), ls_arc(I, n, x, y)), F), R);
            if (gain > LS_GAIN) {
                ls_reverse_path(M, n, i0, len);
                if (lane == 0) { M.dlb[a] = 0; M.dlb[x] = 0; M.dlb[b] = 0; M.dlb[y] = 0; }
                __syncwarp();
                return true;
            }
        }
    }
    return false;
}

// passes and rounds of the neighbour-list searches with don't-look bits
// (as the 2-opt): examine(a) finds and applies one move of city a
template <typename Examine>
__device__ __forceinline__ void ls_rounds(const LsMem &M, int n, Examine &&examine)
{
    const int lane = threadIdx.x & 31;
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
                const bool clear = pp < n && !M.dlb[M.tour[pp]];
                const unsigned cm = __ballot_sync(FULL2, clear);
                if (!cm) { p += 32; continue; }
                p += __ffs(cm) - 1;
                const int a = M.tour[p];
                for (;;) {
                    if (!examine(a)) break;
                    improved = true;
                    ++round_moves;
                    ++moves;
                    if (moves >= max_moves) break;
                }
                if (lane == 0) M.dlb[a] = 1;
                __syncwarp();
                ++p;
            }
        }
    } while (round_moves > 0 && moves < max_moves);
}

// Improves the ATSP `tour` (global memory) in place by the directed 2-opt.
static __device__ __noinline__ void warp_two_opt_directed(const DevInst &I, int32_t *tour, const LsMem &Mref)
{
    const LsMem M = Mref;   // a local copy: see warp_two_opt
    const int lane = threadIdx.x & 31;
    const int n = I.n, K = I.ls_k;
    if (M.tour != tour)
        for (int p = lane; p < n; p += 32) M.tour[p] = tour[p];
    __syncwarp();
    for (int p = lane; p < n; p += 32) M.pos[M.tour[p]] = p;
    __syncwarp();
    ls_rounds(M, n, [&](int a) { return ls2d_examine(I, M, n, K, a); });
    if (M.tour != tour)
        for (int p = lane; p < n; p += 32) tour[p] = M.tour[p];
    __syncwarp();
}

// the 2-opt of the instance's kind: symmetric (twoopt.cuh) or directed
static __device__ __forceinline__ void warp_two_opt_any(const DevInst &I, int32_t *tour, const LsMem &M)
{
    if (I.kind == 1) warp_two_opt_directed(I, tour, M);
    else warp_two_opt(I, tour, M);
}

// Improves `tour` (global memory) in place; M as for warp_two_opt (its el
// array serves as the scratch of the middle rewrite).
static __device__ __noinline__ void warp_three_opt(const DevInst &I, int32_t *tour, const LsMem &Mref)
{
    const LsMem M = Mref;   // a local copy: see warp_two_opt
    const int lane = threadIdx.x & 31;
    const int n = I.n, K = I.ls_k;
    if (M.tour != tour)
        for (int p = lane; p < n; p += 32) M.tour[p] = tour[p];
    __syncwarp();
    for (int p = lane; p < n; p += 32) M.pos[M.tour[p]] = p;
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
                const bool clear = pp < n && !M.dlb[M.tour[pp]];
                const unsigned cm = __ballot_sync(FULL2, clear);
                if (!cm) { p += 32; continue; }
                p += __ffs(cm) - 1;
                const int a = M.tour[p];
                for (;;) {
                    const bool moved = ls3_examine(I, M, n, K, a);
                    if (!moved) break;
                    improved = true;
                    ++round_moves;
                    ++moves;
                    if (moves >= max_moves) break;
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

}  // namespace hac
