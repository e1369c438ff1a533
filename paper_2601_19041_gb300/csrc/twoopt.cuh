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
};

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
    // the pairs (p, q) of different t are disjoint, so each lane loads two
    // pairs before it stores them
    const int h = len / 2;
    for (int t = lane; t < h; t += 64) {
        const bool two = t + 32 < h;
        int p0 = i0 + t, q0 = i0 + len - 1 - t;
        int p1 = p0 + 32, q1 = q0 - 32;
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
    for (int t = lane; t < he; t += 64) {
        const bool two = t + 32 < he;
        int p0 = i0 + t, q0 = i0 + len - 2 - t;
        int p1 = p0 + 32, q1 = q0 - 32;
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
            const int q = dir == 0 ? j : j - cc0;
            const int an = dir == 0 ? xan0 : xan1;
            const float da = dir == 0 ? xda0 : xda1;
            const int b = I.nbr[(size_t)a * K + q];
            const float dab = I.nbrd32[(size_t)a * K + q];
            const int pb = M.pos[b];
            const int pe = dir == 0 ? pb : wrap_prev(pb, n);     // the edge (b, dir b)
            const int bn = M.tour[dir == 0 ? wrap_next(pb, n) : pe];
            if (b != an && bn != a) hit = ls_may_improve(da, dab, M.el[pe], ls_d32(M.xy, an, bn));
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
                    for (int dir = 0; dir < 2 && !moved; ++dir) {
                        int an, b, bn;
                        float dab, dn;
                        if (ls_find_move(I, M, n, K, a, dir, nb, nd32, nd64, an, b, bn, dab, dn)) {
                            if (dir == 0) apply_succ_move(M, n, a, b, dab, dn);
                            else apply_succ_move(M, n, an, bn, dn, dab);
                            if (lane == 0) { M.dlb[a] = 0; M.dlb[an] = 0; M.dlb[b] = 0; M.dlb[bn] = 0; }
                            __syncwarp();
                            moved = true;
                            improved = true;
                            ++round_moves;
                            ++moves;
                        }
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
__device__ __forceinline__ LsMem ls_shared(const DevInst &I, int32_t *tour, unsigned char *sm, size_t smem_bytes,
                                           const LsMem &fallback)
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
        for (int p = threadIdx.x & 31; p < n; p += 32) sxy[p] = reinterpret_cast<const float2 *>(I.xy)[p];
        __syncwarp();
        M.xy = sxy;
    }
    return M;
}

}  // namespace hac
