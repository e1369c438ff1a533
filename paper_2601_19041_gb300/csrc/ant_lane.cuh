// One ant per lane (32 ants per warp): Algorithm 2 with the whole candidate
// row of the current node in the lane's registers.
//
// The arithmetic is exactly that of the warp-segment construction (ant.cuh):
// the k_pad slots form groups of 4 with sequential in-group partial sums, the
// 8 group totals are combined by the same inclusive Hillis-Steele pattern
// (offsets 1, 2, 4; zero totals beyond k_pad/4), slot prefixes are the
// exclusive group prefix plus the in-group sum, r = fl32(u * total), and the
// first live slot with r < prefix (or the last live slot) is chosen.  Only
// where the values live differs (one lane instead of 8 lanes and shuffles).
//
// Per-ant state in shared memory: the visited mask, stored word-major and
// lane-minor (word w of lane l at w*32 + l) so that every lookup of a warp is
// free of bank conflicts.  Tours and chosen slots are written step-major
// (step s of ant a at s*m + a): 32 ants of a warp store one coalesced line
// per step.  The tour length is not summed here: the chosen slot (or 0xff
// for a nearest-unvisited step) is recorded, fallback steps are queued, and
// lengths are summed afterwards, one ant per lane (full-width FP64).
//
// Nearest unvisited node: the whole warp serves the lanes that need it, one
// lane at a time (lookup list, then a scan of that lane's unvisited bits).
#pragma once

#include "ant.cuh"

namespace hac {


template <int NG, typename Rows, typename List>
__device__ __forceinline__ void build_tours_lane(const DevInst &I, const Rows &rows, const List &list,
                                                 int t, int a_first, int a_end, unsigned *vis_warp,
                                                 const float2 *xy_scan)
{
    const int lane = threadIdx.x & 31;
    const int a = a_first + lane;
    const bool real = a < a_end;
    const int n = I.n, kp = I.k_pad, G = kp >> 2, kind = I.kind, m = I.m;
    const uint64_t seed = I.seed;
    const float *__restrict__ cost = I.cost;
    const float2 *__restrict__ xy = xy_scan;
    const int nwords = (n + 31) >> 5;
    int32_t *__restrict__ tourT = I.tours;      // step-major: [s * m + a]
    uint8_t *__restrict__ slotT = I.slots;      // step-major
    int32_t *__restrict__ fbs = I.fbs + (size_t)(real ? a : 0) * n;
    int nfb = 0;

    for (int w = 0; w <= (n >> 5); ++w) vis_warp[w * 32 + lane] = 0u;   // bits 0..n
    vis_warp[(n >> 5) * 32 + lane] |= 1u << (n & 31);                   // padding node n: never live
    U4 rnd = draw_block(seed, (uint32_t)t, (uint32_t)(real ? a : 0), 0u);
    const int start = (int)__umulhi(rnd.x, (uint32_t)n);
    int cur = start;
    if (real) {
        vis_warp[(cur >> 5) * 32 + lane] |= 1u << (cur & 31);
        tourT[a] = cur;
    }

    for (int s = 1; s < n; ++s) {
        // ---- the row of cur, all k_pad slots in registers
        float w[4 * NG];
        int id[4 * NG];
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            int4 i4 = make_int4(n, n, n, n);
            float4 c4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (real && g < G) rows.load(cur, g, i4, c4);
            id[4 * g] = i4.x; id[4 * g + 1] = i4.y; id[4 * g + 2] = i4.z; id[4 * g + 3] = i4.w;
            w[4 * g] = c4.x; w[4 * g + 1] = c4.y; w[4 * g + 2] = c4.z; w[4 * g + 3] = c4.w;
        }
        unsigned lg[NG];
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            unsigned bits = 0u;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 4 * g + q;
                const int j = id[c];
                const bool u = !((vis_warp[(j >> 5) * 32 + lane] >> (j & 31)) & 1u);
                w[c] = u ? w[c] : 0.0f;
                bits |= (w[c] > 0.0f ? 1u : 0u) << q;
            }
            lg[g] = bits << (4 * g);
        }
        unsigned live = 0u;
#pragma unroll
        for (int g = 0; g < NG; ++g) live |= lg[g];
        // ---- prefix sums in the fixed order
        float p[4 * NG], T[8];
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            p[4 * g] = w[4 * g];
            p[4 * g + 1] = __fadd_rn(p[4 * g], w[4 * g + 1]);
            p[4 * g + 2] = __fadd_rn(p[4 * g + 1], w[4 * g + 2]);
            p[4 * g + 3] = __fadd_rn(p[4 * g + 2], w[4 * g + 3]);
            T[g] = p[4 * g + 3];
        }
#pragma unroll
        for (int g = NG; g < 8; ++g) T[g] = 0.0f;
        float I1[8], I2[8], I4[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) I1[g] = g >= 1 ? __fadd_rn(T[g], T[g - 1]) : T[g];
#pragma unroll
        for (int g = 0; g < 8; ++g) I2[g] = g >= 2 ? __fadd_rn(I1[g], I1[g - 2]) : I1[g];
#pragma unroll
        for (int g = 0; g < 8; ++g) I4[g] = g >= 4 ? __fadd_rn(I2[g], I2[g - 4]) : I2[g];
        const float total = I4[7];

        // ---- draw s: word s&3 of block s>>2
        if ((s & 3) == 0) rnd = draw_block(seed, (uint32_t)t, (uint32_t)(real ? a : 0), (uint32_t)(s >> 2));
        const float r = __fmul_rn(unif24(word_of(rnd, s & 3)), total);
        unsigned hg[NG];
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            unsigned bits = 0u;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 4 * g + q;
                const float S = g == 0 ? p[c] : __fadd_rn(I4[g - 1], p[c]);
                bits |= (r < S ? 1u : 0u) << q;
            }
            hg[g] = bits << (4 * g);
        }
        unsigned hit = 0u;
#pragma unroll
        for (int g = 0; g < NG; ++g) hit |= hg[g];
        hit &= live;
        const int cstar = hit ? __ffs(hit) - 1 : 31 - __clz(live | 1u);
        // id[cstar] without dynamic register indexing: an OR-tree of masked ids
        int pick[NG];
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const int b = 4 * g;
            pick[g] = (cstar == b ? id[b] : 0) | (cstar == b + 1 ? id[b + 1] : 0) |
                      (cstar == b + 2 ? id[b + 2] : 0) | (cstar == b + 3 ? id[b + 3] : 0);
        }
        int nxt = 0;
#pragma unroll
        for (int g = 0; g < NG; ++g) nxt |= pick[g];
        uint8_t slot = (uint8_t)cstar;

        // ---- nearest unvisited node for the lanes with no live candidate
        unsigned need = __ballot_sync(FULL_MASK, real && live == 0u);
        if (need) {
            __syncwarp();
            while (need) {
                const int L = __ffs(need) - 1;
                need &= need - 1u;
                const int scur = __shfl_sync(FULL_MASK, cur, L);
                int found = -1;
                if (list.present()) {
                    const int u = list.get(scur, lane);
                    const bool ok = u >= 0 && !((vis_warp[(u >> 5) * 32 + L] >> (u & 31)) & 1u);
                    const unsigned bm = __ballot_sync(FULL_MASK, ok);
                    if (bm) found = __shfl_sync(FULL_MASK, u, __ffs(bm) - 1);
                    if (found < 0 && I.fbl2)
                        found = lookup2(I.fbl2, scur, lane,
                                        [&](int u2) { return (vis_warp[(u2 >> 5) * 32 + L] >> (u2 & 31)) & 1u; });
                }
                if (found < 0) {
                    float bk = __int_as_float(0x7f800000);
                    int bu = 0x7fffffff;
                    const float2 pc = kind == 0 ? xy[scur] : make_float2(0.f, 0.f);
                    const float *crow = kind == 1 ? cost + (size_t)scur * n : nullptr;
                    for (int wd = lane; wd < nwords; wd += 32) {
                        unsigned um = ~vis_warp[wd * 32 + L];
                        if (wd == nwords - 1 && (n & 31)) um &= (1u << (n & 31)) - 1u;
                        while (um) {
                            int u4[4];
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                u4[k] = um ? (wd << 5) | (__ffs(um) - 1) : -1;
                                um &= um - 1u;
                            }
                            float k4[4];
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                k4[k] = u4[k] < 0 ? __int_as_float(0x7f800000)
                                      : kind == 0 ? key32_xy(pc, xy[u4[k]]) : crow[u4[k]];
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                if (u4[k] >= 0 && key_less(k4[k], u4[k], bk, bu)) { bk = k4[k]; bu = u4[k]; }
                        }
                    }
#pragma unroll
                    for (int o = 16; o; o >>= 1) {
                        const float k2 = __shfl_xor_sync(FULL_MASK, bk, o);
                        const int u2 = __shfl_xor_sync(FULL_MASK, bu, o);
                        if (key_less(k2, u2, bk, bu)) { bk = k2; bu = u2; }
                    }
                    found = bu;
                }
                if (lane == L) {
                    nxt = found;
                    slot = SLOT_FALLBACK;
                    fbs[nfb++] = s;
                }
            }
        }
        if ((unsigned)nxt >= (unsigned)n) nxt = 0;   // unreachable for finite keys; keeps indices in range
        if (real) {
            vis_warp[(nxt >> 5) * 32 + lane] |= 1u << (nxt & 31);
            tourT[(size_t)s * m + a] = nxt;
            slotT[(size_t)s * m + a] = slot;
        }
        cur = nxt;
    }
    if (real) I.fbcnt[a] = nfb;
}

}  // namespace hac
