// Tour construction, Algorithm 2: every ant of every active instance builds
// one tour per iteration.
//
// Mapping.  An ant is a segment of SEG = 32/APW lanes of a warp (APW = 1, 2
// or 4 ants per warp).  The ant's visited set is a bitmask in shared memory.
// Per step, lanes g < k_pad/4 of the segment load slots 4g..4g+3 of row
// C_cur as one int4 (candidate ids) and one float4 (choice = tau^alpha * W),
// both 16-byte aligned 128-bit loads.
//
// Roulette (eq. transition, probability w_j / sum w over unvisited j in C_i):
// inside a lane the four partial sums are sequential, the 8 lane totals are
// combined by an inclusive Hillis-Steele warp-shuffle scan (offsets 1, 2, 4),
// and slot c's prefix is the exclusive lane prefix plus the in-lane partial
// sum.  r = fl32(u * total) picks the first live slot with r < prefix (ballot
// + ffs), or the last live slot if rounding leaves none.  u is the top 24
// bits of the Philox draw for (iteration, ant, step).  This fixed order is
// what makes tours reproducible bit for bit.
//
// Fallback (Alg. 2, N_i empty): the nearest unvisited node by the FP32 key
// (squared distance or cost), ties to the lower index; the segment scans the
// unvisited bits of the mask word by word and reduces (key, node) by shuffles.
//
// Length: FP64 sum in step order (the candidate edge's d_ij comes from the
// precomputed slot distance, a fallback edge's is computed), closing edge last.
#include "hac_internal.cuh"

namespace hac {

constexpr unsigned FULLW = 0xffffffffu;

__device__ __forceinline__ uint32_t pick_word(const U4 &v, int w)
{
    return w == 0 ? v.x : w == 1 ? v.y : w == 2 ? v.z : v.w;
}

__device__ __forceinline__ int pick_int(const int4 &v, int w)
{
    return w == 0 ? v.x : w == 1 ? v.y : w == 2 ? v.z : v.w;
}

template <int APW>
__global__ void __launch_bounds__(256) k_construct(const DevInst *__restrict__ insts,
                                                   const int4 *__restrict__ warpmap, int nwarps,
                                                   int nwords_max)
{
    constexpr int SEG = 32 / APW;
    constexpr unsigned SEGMASK = SEG == 32 ? 0xffffffffu : ((1u << SEG) - 1u);
    extern __shared__ unsigned int smem_vis[];

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    if (gw >= nwarps) return;                       // warp-uniform
    const int4 wm = warpmap[gw];
    const DevInst &I = insts[wm.x];
    InstState *st = I.st;
    const int t = st->t;
    if (t >= I.iters) return;                       // warp-uniform

    const int seg = lane / SEG, sl = lane % SEG;
    const int segbase = seg * SEG;
    const int a = wm.y + seg;
    const bool real = a < I.m;
    const int n = I.n, kp = I.k_pad, G = kp >> 2;
    const int nwords = (n + 31) >> 5;
    unsigned int *vis = smem_vis + (size_t)(wib * APW + seg) * nwords_max;
    const int4 *cand4 = reinterpret_cast<const int4 *>(I.cand);
    const float4 *ch4 = reinterpret_cast<const float4 *>(I.choice);
    const float2 *xy = reinterpret_cast<const float2 *>(I.xy);

    for (int w = sl; w < nwords; w += SEG) vis[w] = 0u;
    __syncwarp();

    // Philox cache: lane sl holds block (qbase + sl) = draws 4(qbase+sl) .. +3
    uint32_t qbase = 0;
    U4 rnd = draw_block(I.seed, (uint32_t)t, (uint32_t)a, (uint32_t)sl);

    const int start = (int)__umulhi(__shfl_sync(FULLW, rnd.x, segbase), (uint32_t)n);
    if (sl == 0 && real) vis[start >> 5] |= 1u << (start & 31);
    __syncwarp();
    int tb = sl == 0 ? start : 0;                   // tour write buffer (step s at lane s % SEG)
    int32_t *tour = I.tours + (size_t)(real ? a : 0) * n;
    double L = 0.0;
    unsigned nfb = 0;
    int cur = start;

    for (int s = 1; s < n; ++s) {
        // ---- candidate row of cur
        int4 id = make_int4(-1, -1, -1, -1);
        float4 ch = make_float4(0.f, 0.f, 0.f, 0.f);
        if (real && sl < G) {
            id = __ldg(cand4 + (size_t)cur * G + sl);
            ch = __ldg(ch4 + (size_t)cur * G + sl);
        }
        auto unv = [&](int j) { return j >= 0 && !((vis[j >> 5] >> (j & 31)) & 1u); };
        const float w0 = unv(id.x) ? ch.x : 0.0f;
        const float w1 = unv(id.y) ? ch.y : 0.0f;
        const float w2 = unv(id.z) ? ch.z : 0.0f;
        const float w3 = unv(id.w) ? ch.w : 0.0f;
        const float p0 = w0, p1 = __fadd_rn(p0, w1), p2 = __fadd_rn(p1, w2), p3 = __fadd_rn(p2, w3);
        float inc = p3;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            float v = __shfl_up_sync(FULLW, inc, o, 8);
            if ((lane & 7) >= o) inc = __fadd_rn(inc, v);
        }
        const float ex = __shfl_up_sync(FULLW, inc, 1, 8);
        const bool g0 = (lane & 7) == 0;
        const float S0 = g0 ? p0 : __fadd_rn(ex, p0);
        const float S1 = g0 ? p1 : __fadd_rn(ex, p1);
        const float S2 = g0 ? p2 : __fadd_rn(ex, p2);
        const float S3 = g0 ? p3 : __fadd_rn(ex, p3);
        const float total = __shfl_sync(FULLW, inc, 7, SEG);

        const bool anyw = (w0 > 0.0f) | (w1 > 0.0f) | (w2 > 0.0f) | (w3 > 0.0f);
        const unsigned live_bits = (__ballot_sync(FULLW, anyw) >> segbase) & SEGMASK;
        const bool live = live_bits != 0u || !real;

        // ---- draw s (uniform refill: all segments are at the same step)
        const uint32_t q = (uint32_t)s >> 2;
        if (q >= qbase + SEG) {
            qbase += SEG;
            rnd = draw_block(I.seed, (uint32_t)t, (uint32_t)a, qbase + sl);
        }
        const uint32_t x = __shfl_sync(FULLW, pick_word(rnd, s & 3), (int)(q - qbase), SEG);
        const float r = __fmul_rn(unif24(x), total);

        int hq = -1;
        if (w3 > 0.0f && r < S3) hq = 3;
        if (w2 > 0.0f && r < S2) hq = 2;
        if (w1 > 0.0f && r < S1) hq = 1;
        if (w0 > 0.0f && r < S0) hq = 0;
        const unsigned hit_bits = (__ballot_sync(FULLW, hq >= 0) >> segbase) & SEGMASK;
        int lastq = w3 > 0.0f ? 3 : w2 > 0.0f ? 2 : w1 > 0.0f ? 1 : 0;
        const int src = hit_bits ? __ffs(hit_bits) - 1 : 31 - __clz(live_bits | 1u);
        const int myq = hit_bits ? (hq < 0 ? 0 : hq) : lastq;
        const int nxt_r = __shfl_sync(FULLW, pick_int(id, myq), src, SEG);
        const int cq = __shfl_sync(FULLW, myq, src, SEG);
        int nxt = nxt_r;

        // ---- nearest unvisited node when no candidate is left
        const unsigned fb_bits = __ballot_sync(FULLW, !live);
        if (fb_bits) {
            float bk = __int_as_float(0x7f800000);
            int bu = 0x7fffffff;
            if (!live) {
                const float2 pc = I.kind == 0 ? xy[cur] : make_float2(0.f, 0.f);
                const float *crow = I.kind == 1 ? I.cost + (size_t)cur * n : nullptr;
                for (int w = sl; w < nwords; w += SEG) {
                    unsigned um = ~vis[w];
                    if (w == nwords - 1 && (n & 31)) um &= (1u << (n & 31)) - 1u;
                    while (um) {
                        const int b = __ffs(um) - 1;
                        um &= um - 1u;
                        const int u = (w << 5) | b;
                        const float kk = I.kind == 0 ? key32_xy(pc, xy[u]) : crow[u];
                        if (key_less(kk, u, bk, bu)) { bk = kk; bu = u; }
                    }
                }
            }
#pragma unroll
            for (int o = SEG / 2; o; o >>= 1) {
                const float k2 = __shfl_xor_sync(FULLW, bk, o, SEG);
                const int u2 = __shfl_xor_sync(FULLW, bu, o, SEG);
                if (key_less(k2, u2, bk, bu)) { bk = k2; bu = u2; }
            }
            if (!live) nxt = bu;
        }
        if ((unsigned)nxt >= (unsigned)n) nxt = 0;   // unreachable for finite keys; keeps indices in range

        // ---- length, visited set, tour
        if (sl == 0 && real) {
            double d;
            if (!live) { d = dist64(I, cur, nxt); ++nfb; }
            else d = I.cdist[(size_t)cur * kp + src * 4 + cq];
            L = __dadd_rn(L, d);
            vis[nxt >> 5] |= 1u << (nxt & 31);
        }
        __syncwarp();
        const int slot = s % SEG;
        if (sl == slot) tb = nxt;
        if (slot == SEG - 1 || s == n - 1) {
            if (real && sl <= slot) tour[s - slot + sl] = tb;
        }
        cur = nxt;
    }
    if (sl == 0 && real) {
        L = __dadd_rn(L, dist64(I, cur, start));
        I.lens[a] = L;
        if (nfb) atomicAdd(&st->n_fallback, (unsigned long long)nfb);
    }
}

template <int APW>
static void launch_construct_apw(const DevInst *d_inst, const int4 *d_warpmap, int warpmap_len,
                                 int warps_per_block, int max_n, cudaStream_t s)
{
    int nwords = (max_n + 31) / 32;
    size_t smem = (size_t)warps_per_block * APW * nwords * sizeof(unsigned);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_construct<APW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    int blocks = (warpmap_len + warps_per_block - 1) / warps_per_block;
    k_construct<APW><<<blocks, warps_per_block * 32, smem, s>>>(d_inst, d_warpmap, warpmap_len,
                                                                 nwords);
}

int launch_construct(const DevInst *d_inst, const int4 *d_warpmap, int warpmap_len, int apw,
                     int warps_per_block, int max_n, cudaStream_t s)
{
    if (apw == 4) launch_construct_apw<4>(d_inst, d_warpmap, warpmap_len, warps_per_block, max_n, s);
    else if (apw == 2) launch_construct_apw<2>(d_inst, d_warpmap, warpmap_len, warps_per_block, max_n, s);
    else launch_construct_apw<1>(d_inst, d_warpmap, warpmap_len, warps_per_block, max_n, s);
    return 1;
}

}  // namespace hac
