// Uniform grid over the coordinates of a Euclidean instance, for the
// nearest-unvisited rule of Algorithm 2 (line 5) and reading 4: the unvisited
// node of smallest (FP32 squared distance, index).
//
// Built only for n >= GRID_MIN_N: on smaller instances a scan of the
// unvisited bits (a few words per lane) is cheaper than the ring search.
//
// The grid has G x G square cells of side cs over the bounding box (G is the
// smallest integer with 2 G^2 >= n, so about two nodes per cell); node i lies
// in cell (cx, cy) with cx = min(G-1, (int)fl32(fl32(x_i - x0) / cs)), the
// same arithmetic in the preparation and in the search.  The search examines
// the rings of cells around the current node's cell (ring r: the cells at
// Chebyshev distance r) and stops after ring r once some unvisited node is
// closer than any node outside the rings seen so far can be:
//   a node in a cell at Chebyshev distance >= r+1 lies at least (r - 0.01) cs
//   away along x or y (the computed cell of a node differs from its exact one
//   only within G * 2.4e-7 cell widths of a cell boundary, far below 0.01),
//   so its FP32 key is at least 0.9999 (r - 0.01)^2 cs^2.
// Within the rings examined the minimum is exact, so the node found is the
// one a scan over all unvisited nodes finds.
#pragma once

#include "hac_internal.cuh"

namespace hac {

// smallest G with 2 G^2 >= n
__host__ __device__ inline int grid_side(int n)
{
    int g = 1;
    while (2 * g * g < n) ++g;
    return g;
}

struct GridView {
    const int32_t *start;   // G*G + 1: nodes of cell c at node[start[c] .. start[c+1])
    const int32_t *node;
    int G;
    float x0, y0, cs;
    __device__ __forceinline__ int cell_of(float v, float v0) const
    {
        int c = (int)__fdiv_rn(__fsub_rn(v, v0), cs);
        return c < 0 ? 0 : c > G - 1 ? G - 1 : c;
    }
};

// ring r >= 1 has 8r cells: top row, bottom row, left and right columns
__device__ __forceinline__ void ring_cell(int r, int q, int &dx, int &dy)
{
    if (q < 2 * r + 1) { dx = q - r; dy = -r; return; }
    q -= 2 * r + 1;
    if (q < 2 * r + 1) { dx = q - r; dy = r; return; }
    q -= 2 * r + 1;
    if (q < 2 * r - 1) { dx = -r; dy = q - r + 1; return; }
    q -= 2 * r - 1;
    dx = r;
    dy = q - r + 1;
}

// Whole warp: the unvisited node nearest to `cur` by (FP32 key, index).
// Visited masks: `vis` word-major for one ant (stride 1), or the lane-minor
// layout of one ant per lane (word w of lane L at w*32 + L: stride 32, L).
// Every lane returns the node.  Kept out of line: it runs only after a
// lookup-list miss, and inlining it into the construction loop costs more
// than the call.
static __device__ __noinline__ int grid_nearest(const GridView &gv, const float2 *xy, int cur,
                                                const unsigned *vis, int stride, int L)
{
    auto visited = [&](int u) { return (vis[(u >> 5) * stride + L] >> (u & 31)) & 1u; };
    const int lane = threadIdx.x & 31;
    const float2 pc = xy[cur];
    const int G = gv.G;
    const int ccx = gv.cell_of(pc.x, gv.x0), ccy = gv.cell_of(pc.y, gv.y0);
    const int rmax = max(max(ccx, G - 1 - ccx), max(ccy, G - 1 - ccy));
    float bk = __int_as_float(0x7f800000);
    int bu = 0x7fffffff;
    for (int r = 0; r <= rmax; ++r) {
        const int cnt = r == 0 ? 1 : 8 * r;
        for (int q = lane; q < cnt; q += 32) {
            int dx = 0, dy = 0;
            if (r) ring_cell(r, q, dx, dy);
            const int cx = ccx + dx, cy = ccy + dy;
            if (cx < 0 || cy < 0 || cx >= G || cy >= G) continue;
            const int c = cy * G + cx;
            const int e = gv.start[c + 1];
            for (int p = gv.start[c]; p < e; ++p) {
                const int u = gv.node[p];
                if (visited(u)) continue;
                const float k = key32_xy(pc, xy[u]);
                if (key_less(k, u, bk, bu)) { bk = k; bu = u; }
            }
        }
        if (r >= 1) {
            const float lbd = __fmul_rn(__fsub_rn((float)r, 0.01f), gv.cs);
            const float lbk = __fmul_rn(__fmul_rn(lbd, lbd), 0.9999f);
            if (__any_sync(0xffffffffu, bk < lbk)) break;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float k2 = __shfl_xor_sync(0xffffffffu, bk, o);
        const int u2 = __shfl_xor_sync(0xffffffffu, bu, o);
        if (key_less(k2, u2, bk, bu)) { bk = k2; bu = u2; }
    }
    return bu;
}

}  // namespace hac
