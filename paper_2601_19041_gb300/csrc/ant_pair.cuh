// One ant per lane pair (16 ants per warp): Algorithm 2 with the candidate row
// of the current node split between the two lanes of a pair.
//
// Lane h (0 or 1) of a pair holds the slot groups g = 2j + h (j < NGL) of the
// row: 4 consecutive slots per group, one vector load of ids and one of
// choice values each.  The arithmetic is exactly that of the warp-segment
// construction (ant.cuh) and of the oracle:
//   - in-group partial sums, sequential over the group's 4 slots;
//   - the group totals are swapped between the two lanes (one shuffle per
//     group pair), so both lanes hold all of them, and the inclusive
//     Hillis-Steele scan with offsets 1, 2, 4 over the 8 group totals is
//     evaluated in registers (groups without slots hold +0, and adding +0 to
//     a non-negative float is exact, so those additions are skipped);
//   - slot prefix = exclusive group prefix + in-group partial sum,
//     r = fl32(u * total), the first live slot with r < prefix is chosen,
//     or the last live slot when rounding leaves none.
// Each lane finds the first qualifying slot among its own groups; one
// shuffle between the lanes gives the pair's first slot and its node.
//
// Compared with 8-lane segments this takes one shuffle round instead of four
// per step, and 16 instead of 4 ants share each warp instruction, so a warp
// spends about a quarter of the instructions per ant-step.
//
// The visited mask of pair p is stored word-major, pair-minor (word w at
// w*16 + p): the 16 pairs of a warp use disjoint banks.  Lane 0 of the pair
// sets the bits.  Nearest-unvisited steps (no live candidate) are served by
// the whole warp, one pair after the other, as in ant.cuh.  Tours are written
// ant-major, one entry per step, with the chosen slot (0xff for a
// nearest-unvisited step); lengths are summed afterwards (lengths.cuh).
#pragma once

#include "ant.cuh"

namespace hac {

template <int NGL, typename Rows, typename List>
__device__ __forceinline__ void build_tours_pair(const DevInst &I, const Rows &rows, const List &list, int t,
                                                 int a_first, int a_end, unsigned *vis_warp, int stride,
                                                 const float2 *xy_scan)
{
    constexpr int GT = 2 * NGL < 8 ? 2 * NGL : 8;   // groups that may hold slots
    const int lane = threadIdx.x & 31;
    const int h = lane & 1, p = lane >> 1, pbase = lane & ~1;
    const int a = a_first + p;
    const bool real = a < a_end;
    const int aa = real ? a : 0;
    const int n = I.n, kp = I.k_pad, G = kp >> 2, kind = I.kind;
    const uint64_t seed = I.seed;
    const float *__restrict__ cost = I.cost;
    const float2 *__restrict__ xy = xy_scan;
    const int nwords = (n + 31) >> 5;
    (void)stride;
    unsigned *vis = vis_warp + p;                  // word w of this pair's mask at vis[16 * w]

    for (int w = h; w <= (n >> 5); w += 2) vis[16 * w] = 0u;   // bits 0..n
    __syncwarp();

    // draw s is word (s & 3) of Philox block (s >> 2); lane h holds the block
    // of the current 8-step window whose index has parity h
    U4 rnd = draw_block(seed, (uint32_t)t, (uint32_t)aa, (uint32_t)h);
    const int start = (int)__umulhi(__shfl_sync(FULL_MASK, rnd.x, pbase), (uint32_t)n);
    if (h == 0) {
        vis[16 * (n >> 5)] |= 1u << (n & 31);        // padding node: never live
        if (real) vis[16 * (start >> 5)] |= 1u << (start & 31);
    }
    __syncwarp();
    int32_t *tour = I.tours + (size_t)aa * n;
    uint8_t *slots = I.slots + (size_t)aa * n;
    int32_t *fbs = I.fbs + (size_t)aa * n;
    if (real && h == 0) { tour[0] = start; slots[0] = SLOT_FALLBACK; }
    int nfb = 0;
    int cur = start;

    int4 idv[NGL];
    float4 chv[NGL];
#pragma unroll
    for (int j = 0; j < NGL; ++j) {
        idv[j] = make_int4(n, n, n, n);
        chv[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int g = 2 * j + h;
        if (real && g < G) rows.load(cur, g, idv[j], chv[j]);
    }

    for (int s = 1; s < n; ++s) {
        if ((s & 7) == 0) rnd = draw_block(seed, (uint32_t)t, (uint32_t)aa, (uint32_t)((s >> 2) + h));
        const uint32_t x = __shfl_sync(FULL_MASK, word_of(rnd, s & 3), pbase + ((s >> 2) & 1));

        // live weights and in-group partial sums of the own groups
        float pp[NGL][4];
        float T[8];
        unsigned live = 0u;   // bit 4j+q: own slot (j, q) live
#pragma unroll
        for (int j = 0; j < NGL; ++j) {
            const int idq[4] = {idv[j].x, idv[j].y, idv[j].z, idv[j].w};
            const float chq[4] = {chv[j].x, chv[j].y, chv[j].z, chv[j].w};
            float acc = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int id = idq[q];
                const unsigned word = vis[16 * (id >> 5)];
                const float w = (__funnelshift_r(word, 0u, (unsigned)id) & 1u) ? 0.0f : chq[q];
                live |= (w > 0.0f ? 1u : 0u) << (4 * j + q);
                acc = q == 0 ? w : __fadd_rn(acc, w);
                pp[j][q] = acc;
            }
        }
        // all group totals: own groups 2j+h, the partner's 2j+1-h
#pragma unroll
        for (int j = 0; j < NGL; ++j) {
            const float own = pp[j][3];
            const float oth = __shfl_xor_sync(FULL_MASK, own, 1);
            if (2 * j < 8) T[2 * j] = h ? oth : own;
            if (2 * j + 1 < 8) T[2 * j + 1] = h ? own : oth;
        }
#pragma unroll
        for (int g = 2 * NGL; g < 8; ++g) T[g] = 0.0f;
        GroupScan<GT> sc;
        sc.run(T);
        const float total = sc.C[7];
        const float r = __fmul_rn(unif24(x), total);

        // first own slot with r < prefix among live slots; scanning downwards
        // leaves the smallest one
        int fslot = 63, fnode = 0;
#pragma unroll
        for (int j = NGL - 1; j >= 0; --j) {
            const int g = 2 * j + h;
            // exclusive prefix of group g: C[g-1], +0 for g = 0
            float ex;
            if (j == 0) ex = h ? sc.C[0] : 0.0f;
            else ex = h ? sc.C[2 * j] : sc.C[2 * j - 1];
            const int idq[4] = {idv[j].x, idv[j].y, idv[j].z, idv[j].w};
#pragma unroll
            for (int q = 3; q >= 0; --q) {
                const float S = __fadd_rn(ex, pp[j][q]);
                if (((live >> (4 * j + q)) & 1u) && r < S) { fslot = 4 * g + q; fnode = idq[q]; }
            }
        }
        // the pair's choice: the smaller slot of the two lanes
        const int mine = (fnode << 8) | (live ? 64 : 0) | fslot;
        const int other = __shfl_xor_sync(FULL_MASK, mine, 1);
        const int best = ((other & 63) < fslot) ? other : mine;
        int nxt = best >> 8;
        unsigned slot = (unsigned)(best & 63);
        const bool plive = ((mine | other) & 64) != 0;
        // rare: live slots but no r < prefix (rounding) -> the last live slot
        const unsigned corner = __ballot_sync(FULL_MASK, real && plive && slot == 63u);
        if (corner) {
            int lslot = -1, lnode = 0;
#pragma unroll
            for (int j = 0; j < NGL; ++j) {
                const int g = 2 * j + h;
                const int idq[4] = {idv[j].x, idv[j].y, idv[j].z, idv[j].w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if ((live >> (4 * j + q)) & 1u) { lslot = 4 * g + q; lnode = idq[q]; }
            }
            const int lm = (lnode << 8) | (lslot + 1);
            const int lo = __shfl_xor_sync(FULL_MASK, lm, 1);
            const int lb = ((lo & 255) > (lm & 255)) ? lo : lm;
            if ((corner >> lane) & 1u) { nxt = lb >> 8; slot = (unsigned)((lb & 255) - 1); }
        }

        // ---- nearest unvisited node, one needing pair at a time, whole warp
        unsigned need = __ballot_sync(FULL_MASK, h == 0 && real && !plive);
        while (need) {
            const int sb = __ffs(need) - 1;          // lane 0 of the needing pair
            need &= need - 1u;
            const int scur = __shfl_sync(FULL_MASK, cur, sb);
            const unsigned *sv = vis_warp + (sb >> 1);
            int found = -1;
            if (list.present()) {
                const int u = list.get(scur, lane);
                const bool ok = u >= 0 && !((sv[16 * (u >> 5)] >> (u & 31)) & 1u);
                const unsigned bm = __ballot_sync(FULL_MASK, ok);
                if (bm) found = __shfl_sync(FULL_MASK, u, __ffs(bm) - 1);
                if (found < 0 && I.fbl2)
                    found = lookup2(I.fbl2, scur, lane, [&](int u2) { return (sv[16 * (u2 >> 5)] >> (u2 & 31)) & 1u; });
            }
            if (found < 0) {
                float bk = __int_as_float(0x7f800000);
                int bu = 0x7fffffff;
                const float2 pc = kind == 0 ? xy[scur] : make_float2(0.f, 0.f);
                const float *crow = kind == 1 ? cost + (size_t)scur * n : nullptr;
                for (int w = lane; w < nwords; w += 32) {
                    unsigned um = ~sv[16 * w];
                    if (w == nwords - 1 && (n & 31)) um &= (1u << (n & 31)) - 1u;
                    while (um) {
                        int u4[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            u4[k] = um ? (w << 5) | (__ffs(um) - 1) : -1;
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
            if (pbase == sb) {
                nxt = found;
                slot = SLOT_FALLBACK;
                if (h == 0) fbs[nfb++] = s;
            }
        }
        if ((unsigned)nxt >= (unsigned)n) nxt = 0;   // unreachable for finite keys; keeps indices in range

        // next row first, so its latency overlaps the bookkeeping below
        if (s + 1 < n) {
#pragma unroll
            for (int j = 0; j < NGL; ++j) {
                const int g = 2 * j + h;
                if (real && g < G) rows.load(nxt, g, idv[j], chv[j]);
            }
        }
        if (h == 0 && real) {
            vis[16 * (nxt >> 5)] |= 1u << (nxt & 31);
            tour[s] = nxt;
            slots[s] = (uint8_t)slot;
        }
        __syncwarp();
        cur = nxt;
    }
    if (h == 0 && real) I.fbcnt[a] = nfb;
}

}  // namespace hac
