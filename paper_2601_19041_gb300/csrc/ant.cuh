// One ant's tour (Algorithm 2), shared by the per-iteration kernel
// (candidate rows in global memory) and the fused cluster kernel (rows in
// shared / distributed shared memory).
//
// An ant is a segment of SEG = 32/APW lanes of a warp; all segments of a warp
// advance in lockstep (same step s).  Per step, lanes g < k_pad/4 of a segment
// hold candidate slots 4g..4g+3 (ids and choice values, one vector load each).
//
// Roulette (eq. transition): in-lane sequential partial sums, an inclusive
// Hillis-Steele shuffle scan over the 8 lane totals (offsets 1, 2, 4), slot
// prefix = exclusive lane prefix + in-lane partial sum; r = fl32(u * total)
// selects the first live slot with r < prefix (ballot + ffs), or the last
// live slot when rounding leaves none.
//
// Fallback (N_i empty): the nearest unvisited node by (FP32 key, index).  The
// whole warp serves the segments that need it, one after the other: first the
// node's 32-entry list of nearest nodes in key order (the first unvisited entry
// of that list is the exact answer when there is one), else a scan of the
// unvisited bits of the ant's mask.
#pragma once

#include "lengths.cuh"

namespace hac {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr int FBL = FBL1_LEN;   // fallback list length (nearest nodes in key order)

__device__ __forceinline__ uint32_t word_of(const U4 &v, int w)
{
    return w == 0 ? v.x : w == 1 ? v.y : w == 2 ? v.z : v.w;
}

__device__ __forceinline__ int int_of(const int4 &v, int w)
{
    return w == 0 ? v.x : w == 1 ? v.y : w == 2 ? v.z : v.w;
}

// Candidate rows hand out padding slots as node n: the construction presets
// bit n of every visited mask, so a padding slot is never live and no slot
// needs a validity test of its own.

// candidate rows in global memory (int32 ids, -1 on padding; FP32 choice)
struct GlobalRows {
    const int4 *cand4;
    const float4 *ch4;
    int G, n;
    __device__ __forceinline__ void load(int cur, int g, int4 &id, float4 &ch) const
    {
        id = __ldg(cand4 + (size_t)cur * G + g);
        ch = __ldg(ch4 + (size_t)cur * G + g);
        id.x = id.x < 0 ? n : id.x;
        id.y = id.y < 0 ? n : id.y;
        id.z = id.z < 0 ? n : id.z;
        id.w = id.w < 0 ? n : id.w;
    }
};

// shared-memory loads by 32-bit shared-window address; for C > 1 the address
// is first mapped to the owning CTA of the cluster (distributed shared memory)
__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ uint2 ld_dsmem_u2(uint32_t a)
{
    uint2 v;
    asm volatile("ld.shared::cluster.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ float4 ld_dsmem_f4(uint32_t a)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

__device__ __forceinline__ uint2 ld_smem_u2(uint32_t a)
{
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ float4 ld_smem_f4(uint32_t a)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

// candidate rows in the shared memory of the CTAs of a cluster, interleaved by
// row (row i lives in CTA i & (C-1) at local row i >> CLOG); uint16 ids with
// n for padding.  Same layout (and offsets) in every CTA.
template <int CLOG>
struct ClusterRows {
    uint32_t idx_base, ch_base;   // shared-window addresses in the calling CTA
    int kp;
    __device__ __forceinline__ void load(int cur, int g, int4 &id, float4 &chv) const
    {
        const uint32_t loc = (uint32_t)cur >> CLOG;
        const uint32_t off = loc * (uint32_t)kp + 4u * (uint32_t)g;
        uint32_t ia = idx_base + 2u * off, ca = ch_base + 4u * off;
        uint2 raw;
        if (CLOG == 0) {
            raw = ld_smem_u2(ia);
            chv = ld_smem_f4(ca);
        } else {
            const uint32_t owner = (uint32_t)cur & ((1u << CLOG) - 1u);
            raw = ld_dsmem_u2(map_to_rank(ia, owner));
            chv = ld_dsmem_f4(map_to_rank(ca, owner));
        }
        id.x = (int)(raw.x & 0xffffu);
        id.y = (int)(raw.x >> 16);
        id.z = (int)(raw.y & 0xffffu);
        id.w = (int)(raw.y >> 16);
    }
};

// nearest-unvisited lookup lists: global int32 (I.fbl) or the uint16 copy in
// the cluster's shared memory (same row interleaving as the candidate table)
struct GlobalList {
    const int32_t *fbl;
    __device__ __forceinline__ bool present() const { return fbl != nullptr; }
    __device__ __forceinline__ int get(int node, int k) const { return fbl[(size_t)node * FBL + k]; }
};

template <int CLOG>
struct ClusterList {
    uint32_t base;   // shared-window address of this CTA's list rows (0: no list)
    __device__ __forceinline__ bool present() const { return base != 0u; }
    __device__ __forceinline__ int get(int node, int k) const
    {
        const uint32_t loc = (uint32_t)node >> CLOG;
        uint32_t a = base + 2u * (loc * FBL + (uint32_t)k);
        unsigned short v;
        if (CLOG == 0) asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
        else {
            a = map_to_rank(a, (uint32_t)node & ((1u << CLOG) - 1u));
            asm volatile("ld.shared::cluster.u16 %0, [%1];" : "=h"(v) : "r"(a));
        }
        return v == 0xffff ? -1 : (int)v;
    }
};

// Second-level lookup (whole warp): the next FBL2_LEN nodes of `node`'s key
// order, 8 per lane in order (lane L holds ranks 32 + 8L .. 32 + 8L + 7).
// Returns the first one that `visited` reports unvisited, or -1 (then the
// nearest unvisited node lies further out and the scan finds it).
template <typename Visited>
__device__ __forceinline__ int lookup2(const uint16_t *fbl2, int node, int lane, Visited visited)
{
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(fbl2 + (size_t)node * FBL2_LEN) + lane);
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
    int first = -1;
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        const int u = (int)((w[k >> 1] >> (16 * (k & 1))) & 0xffffu);
        if (u != 0xffff && !visited(u)) first = u;
    }
    const unsigned bm = __ballot_sync(FULL_MASK, first >= 0);
    return bm ? __shfl_sync(FULL_MASK, first, __ffs(bm) - 1) : -1;
}

// Hillis-Steele inclusive scan (offsets 1, 2, 4) over 8 group totals, of
// which only the first GT can be non-zero; the exclusive prefix of group g is
// ex(g) = C[g-1] and the total is C[7].  Additions of a known +0 are skipped
// (exact for non-negative operands).
template <int GT>
struct GroupScan {
    float C[8];
    __device__ __forceinline__ void run(const float (&T)[8])
    {
        float A[8], B[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const bool zg = g >= GT, zp = g - 1 >= GT;   // T[g], T[g-1] known zero
            if (g == 0 || zp) A[g] = zg ? 0.0f : T[g];
            else A[g] = zg ? T[g - 1] : __fadd_rn(T[g], T[g - 1]);
        }
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const bool zg = g - 1 >= GT, zp = g - 3 >= GT;   // A[g], A[g-2] known zero
            if (g < 2 || zp) B[g] = A[g];
            else B[g] = zg ? A[g - 2] : __fadd_rn(A[g], A[g - 2]);
        }
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const bool zg = g - 3 >= GT, zp = g - 7 >= GT;   // B[g], B[g-4] known zero
            if (g < 4 || zp) C[g] = B[g];
            else C[g] = zg ? B[g - 4] : __fadd_rn(B[g], B[g - 4]);
        }
    }
};

// Builds the tours of the warp's APW ants (ants a = a_first + seg, real when
// a < a_end) in iteration t.  vis_warp: APW bitmasks of `stride` words.
// NGS > 0: every lane gathers the first NGS group totals of its segment (one
// shuffle each, all independent) and evaluates the Hillis-Steele scan in
// registers (GroupScan), instead of three dependent shuffle rounds; NGS must
// be at least k_pad/4 of every instance.  Same values either way.
// Tours (and the chosen slot of every step, 0xff for a nearest-unvisited
// step) are written ant-major; lengths are summed afterwards (lengths.cuh).
template <int APW, typename Rows, typename List, int NGS = 0>
__device__ __forceinline__ void build_tours(const DevInst &I, const Rows &rows, const List &list, int t,
                                            int a_first, int a_end, unsigned *vis_warp, int stride,
                                            const float2 *xy_scan)
{
    constexpr int SEG = 32 / APW;
    constexpr unsigned SEGMASK = SEG == 32 ? 0xffffffffu : ((1u << SEG) - 1u);
    const int lane = threadIdx.x & 31;
    const int seg = lane / SEG, sl = lane % SEG, segbase = seg * SEG;
    const int a = a_first + seg;
    const bool real = a < a_end;
    const int n = I.n, kp = I.k_pad, G = kp >> 2, kind = I.kind;
    const uint64_t seed = I.seed;
    const float *__restrict__ cost = I.cost;
    const float2 *__restrict__ xy = xy_scan;   // coordinates for the fallback scan
    const int nwords = (n + 31) >> 5;
    unsigned *vis = vis_warp + seg * stride;

    for (int w = sl; w <= (n >> 5); w += SEG) vis[w] = 0u;   // bits 0..n
    __syncwarp();

    uint32_t qbase = 0;
    U4 rnd = draw_block(seed, (uint32_t)t, (uint32_t)(real ? a : 0), (uint32_t)sl);
    const int start = (int)__umulhi(__shfl_sync(FULL_MASK, rnd.x, segbase), (uint32_t)n);
    if (sl == 0) {
        vis[n >> 5] |= 1u << (n & 31);                       // padding node: never live
        if (real) vis[start >> 5] |= 1u << (start & 31);
    }
    __syncwarp();
    int tb = sl == 0 ? start : 0;                  // step s of the tour / slot at lane s % SEG
    unsigned sb8 = 0xffu;
    int32_t *tour = I.tours + (size_t)(real ? a : 0) * n;
    uint8_t *slots = I.slots + (size_t)(real ? a : 0) * n;
    int32_t *fbs = I.fbs + (size_t)(real ? a : 0) * n;
    int nfb = 0;
    int cur = start;
    // the row of the current node is loaded at the end of the previous step
    int4 id = make_int4(n, n, n, n);
    float4 ch = make_float4(0.f, 0.f, 0.f, 0.f);
    if (real && sl < G) rows.load(cur, sl, id, ch);

    for (int s = 1; s < n; ++s) {
        // draw s first: independent of the row, its shuffle overlaps the checks
        const uint32_t q = (uint32_t)s >> 2;
        if (q >= qbase + SEG) {
            qbase += SEG;
            rnd = draw_block(seed, (uint32_t)t, (uint32_t)(real ? a : 0), qbase + sl);
        }
        const uint32_t x = __shfl_sync(FULL_MASK, word_of(rnd, s & 3), (int)(q - qbase), SEG);

        auto unv = [&](int j) { return !((vis[j >> 5] >> (j & 31)) & 1u); };
        const float w0 = unv(id.x) ? ch.x : 0.0f;
        const float w1 = unv(id.y) ? ch.y : 0.0f;
        const float w2 = unv(id.z) ? ch.z : 0.0f;
        const float w3 = unv(id.w) ? ch.w : 0.0f;
        const float p0 = w0, p1 = __fadd_rn(p0, w1), p2 = __fadd_rn(p1, w2), p3 = __fadd_rn(p2, w3);
        float ex, total;
        if constexpr (NGS > 0) {
            float T[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) T[g] = g < NGS ? __shfl_sync(FULL_MASK, p3, g, 8) : 0.0f;
            GroupScan<NGS> sc;
            sc.run(T);
            total = sc.C[7];
            const int gq = lane & 7;
            ex = 0.0f;   // exclusive prefix C[g-1]; +0 for the first group leaves p_c unchanged
#pragma unroll
            for (int g = 1; g < NGS; ++g) ex = gq == g ? sc.C[g - 1] : ex;
        } else {
            float inc = p3;
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const float v = __shfl_up_sync(FULL_MASK, inc, o, 8);
                if ((lane & 7) >= o) inc = __fadd_rn(inc, v);
            }
            // exclusive prefix; +0 for the first group leaves p_c unchanged (p_c >= 0)
            const float exu = __shfl_up_sync(FULL_MASK, inc, 1, 8);
            ex = (lane & 7) == 0 ? 0.0f : exu;
            total = __shfl_sync(FULL_MASK, inc, 7, SEG);
        }
        const float S0 = __fadd_rn(ex, p0);
        const float S1 = __fadd_rn(ex, p1);
        const float S2 = __fadd_rn(ex, p2);
        const float S3 = __fadd_rn(ex, p3);
        const float r = __fmul_rn(unif24(x), total);

        int hq = -1;
        if (w3 > 0.0f && r < S3) hq = 3;
        if (w2 > 0.0f && r < S2) hq = 2;
        if (w1 > 0.0f && r < S1) hq = 1;
        if (w0 > 0.0f && r < S0) hq = 0;
        // an idle segment (no ant) counts as decided
        const unsigned hit_all = __ballot_sync(FULL_MASK, hq >= 0 || (!real && sl == 0));
        const unsigned hit_bits = (hit_all >> segbase) & SEGMASK;
        // segments without a hit (no live slot, or the rounding corner case):
        // the top bit of every all-zero SEG-bit field (exact per field, no
        // carries between fields)
        unsigned nohit;
        if (SEG == 32) nohit = hit_all == 0u;
        else {
            constexpr unsigned LOW = SEG == 16 ? 0x7fff7fffu : SEG == 8 ? 0x7f7f7f7fu : 0u;
            nohit = ~(((hit_all & LOW) + LOW) | hit_all | LOW);
        }
        int src, myq;
        bool live = true;
        unsigned need = 0u;
        if (!nohit) {                                   // common case: one ballot
            src = __ffs(hit_bits) - 1;
            myq = hq < 0 ? 0 : hq;
        } else {
            const bool anyw = (w0 > 0.0f) | (w1 > 0.0f) | (w2 > 0.0f) | (w3 > 0.0f);
            const unsigned live_all = __ballot_sync(FULL_MASK, anyw);
            const unsigned live_bits = (live_all >> segbase) & SEGMASK;
            live = live_bits != 0u || !real;
            const int lastq = w3 > 0.0f ? 3 : w2 > 0.0f ? 2 : w1 > 0.0f ? 1 : 0;
            src = hit_bits ? __ffs(hit_bits) - 1 : 31 - __clz(live_bits | 1u);
            myq = hit_bits ? (hq < 0 ? 0 : hq) : lastq;
            need = __ballot_sync(FULL_MASK, sl == 0 && !live);
        }
        // chosen node and slot in one shuffle: (node << 2) | slot-in-lane
        const int packed = __shfl_sync(FULL_MASK, (int)(((unsigned)int_of(id, myq) << 2) | (unsigned)myq),
                                       src, SEG);
        int nxt = packed >> 2;
        unsigned slot = (unsigned)(src * 4 + (packed & 3));

        // ---- nearest unvisited node, one needing segment at a time, whole warp
        while (need) {
            const int sb = __ffs(need) - 1;
            need &= need - 1u;
            const int scur = __shfl_sync(FULL_MASK, cur, sb);
            const unsigned *sv = vis_warp + (sb / SEG) * stride;
            int found = -1;
            if (list.present()) {
                const int u = list.get(scur, lane);
                const bool ok = u >= 0 && !((sv[u >> 5] >> (u & 31)) & 1u);
                const unsigned bm = __ballot_sync(FULL_MASK, ok);
                if (bm) found = __shfl_sync(FULL_MASK, u, __ffs(bm) - 1);
                if (found < 0 && I.fbl2)
                    found = lookup2(I.fbl2, scur, lane, [&](int u2) { return (sv[u2 >> 5] >> (u2 & 31)) & 1u; });
            }
            if (found < 0) {
                float bk = __int_as_float(0x7f800000);
                int bu = 0x7fffffff;
                const float2 pc = kind == 0 ? xy[scur] : make_float2(0.f, 0.f);
                const float *crow = kind == 1 ? cost + (size_t)scur * n : nullptr;
                for (int w = lane; w < nwords; w += 32) {
                    unsigned um = ~sv[w];
                    if (w == nwords - 1 && (n & 31)) um &= (1u << (n & 31)) - 1u;
                    while (um) {   // four unvisited nodes per round: independent loads
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
            if (segbase == sb) {
                nxt = found;
                slot = SLOT_FALLBACK;
                if (sl == 0) fbs[nfb++] = s;
            }
        }
        if ((unsigned)nxt >= (unsigned)n) nxt = 0;   // unreachable for finite keys; keeps indices in range

        // next row first, so its latency overlaps the bookkeeping below
        if (real && sl < G && s + 1 < n) rows.load(nxt, sl, id, ch);
        if (sl == 0 && real) vis[nxt >> 5] |= 1u << (nxt & 31);
        __syncwarp();
        const int ts = s % SEG;
        if (sl == ts) { tb = nxt; sb8 = slot; }
        if (ts == SEG - 1 || s == n - 1) {
            if (real && sl <= ts) {
                tour[s - ts + sl] = tb;
                slots[s - ts + sl] = (uint8_t)sb8;
            }
        }
        cur = nxt;
    }
    if (sl == 0 && real) I.fbcnt[a] = nfb;
}

}  // namespace hac
