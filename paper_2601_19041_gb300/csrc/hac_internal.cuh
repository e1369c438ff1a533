// Internal declarations of the HeatACO CUDA library (sm_103a).
//
// Every floating-point operation whose result can change a tour is written
// with an explicit round-to-nearest intrinsic (__fadd_rn, __dmul_rn, ...),
// and the library is compiled with --fmad=false, so no multiply-add is ever
// contracted and each operation is one IEEE operation.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/heataco.h"

namespace hac {

constexpr int KMAX = HAC_KMAX;
constexpr int FBL1_LEN = 32;           // nearest-unvisited lookup list: the 32 first nodes in key order
constexpr int FBL2_LEN = 256;          // second-level nearest-unvisited list: key-order ranks 32..287
constexpr int FBL2_SORT = 512;         // its sort buffer (a power of two >= 32 + FBL2_LEN)
constexpr double DFLOOR = 1e-9;     // eta = 1/max(d, 1e-9): coincident points
constexpr double LS_GAIN = 1e-10;   // 2-opt moves need a gain above this
constexpr int TRACE_W = 5;          // trace entries per iteration: ib ant, L_ib, L_gb, L_rb, code

// Per-instance scalars that live on the device (read back through HAC_F_SCALARS).
struct InstState {
    double q90, Rhat, kappa, p_x, L_nn, tau_max64, tau_min64, L_gb, L_ib;
    float tau_max, tau_min;
    int32_t t;          // iterations done
    int32_t ib;         // iteration-best ant of the last iteration
    int32_t active;     // 1 while the current iteration runs for this instance
    int32_t n_lambda;
    unsigned long long n_fallback;
    int32_t fbl_unsafe; // 1: some choice value could reach 0, lookup lists keep the candidates
    // MMAS schedule (schedule = 1)
    double L_rb;        // restart-best length, +inf while cleared
    double L_dep;       // length of the tour T+ that deposits this iteration
    int32_t t_restart;  // iteration of the last restart (0: none)
    int32_t t_rbimp;    // iteration of the last restart-best improvement
    int32_t u_gb;       // T_rb deposits when the iteration is a multiple of this
    int32_t n_restarts;
    unsigned long long bf_count;   // branching-factor count of the current check
    unsigned long long n_edges;    // sum of |P_i|: heatmap entries above theta_h (Edges/n diagnostic)
};

// Device view of one instance: sizes, parameters and pointers into the workspace.
struct DevInst {
    int32_t n, kind, k, k_eff, k_pad, m, iters, ls_k;
    int32_t degree_target, local_search, baseline_scope, symmetrize, h_half, schedule, kappa_mode;
    uint64_t seed;
    double alpha, beta, rho, theta_h, eps, c_cap, q_level, p_best, logw_clip;
    // inputs
    const float *xy;          // n*2
    const float *cost;        // n*n
    const int32_t *rowptr;    // n+1
    const int32_t *col;       // nnz
    const void *val;          // nnz (f32 or f16)
    int32_t nnz;
    // transposed heatmap (symmetrize only): column i of H as a sorted row
    int32_t *trowptr, *tcol, *tfill;
    double *tval;
    // heatmap support sets P_i with their h values, row i at rowptr[i]+trowptr[i]
    int32_t *mem_j, *mem_cnt;
    double *mem_h;
    // preparation
    int32_t *cand;            // n*k_pad
    double *cdist, *conf, *evid, *logev;
    double *base;             // n
    float *W, *tau, *choice;  // n*k_pad
    int32_t *nbr;             // n*ls_k geometric 2-opt neighbour lists, ascending (d, j)
    double *nbrd;             // n*ls_k their d_ij
    float *nbrd32;            // n*ls_k fl32(d_ij) (2-opt FP32 pre-test)
    float *ls_el;             // n, 2-opt FP32 edge lengths by position (when not in shared memory)
    int32_t *lsa_pos;         // m*n, 2-opt of every ant (local_search = 2): positions of ant a at a*n
    float *lsa_el;            // m*n, its FP32 edge lengths
    uint8_t *lsa_dlb;         // m*n, its don't-look bits
    int32_t *ls_pos;          // n, 2-opt position index
    uint8_t *ls_dlb;          // n, don't-look bits
    int32_t *fbl;             // n*fbl_len (nearest-unvisited lookup list)
    int32_t fbl_len;
    uint16_t *fbl2;           // n*FBL2_LEN second-level list (the next nodes of the same order), or null
    // search state
    int32_t *nn_tour, *gb_tour, *ib_tour, *succ, *pred;   // n each
    int32_t *rb_tour;         // n, restart-best tour (schedule = 1)
    int32_t *tours;           // m*n: tour of ant a, step s at a*tour_sa + s*tour_ss
    int32_t tour_sa, tour_ss; // (n, 1) ant-major, or (1, m) step-major (one ant per lane)
    uint8_t *slots;           // m*n chosen slot per step (same layout as tours), 0xff: nearest-unvisited
    double *dstep;            // m*n d of the edge entering step s (same layout); s = 0: closing edge
    int32_t *fbs;             // m*n nearest-unvisited steps of ant a at a*n + k
    int32_t *fbcnt;           // m   their number in the current iteration
    double *lens;             // m
    double *trace;            // TRACE_W*iters
    InstState *st;
};

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// multiply-xor bijection with the Weyl key schedule.
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        U4 nx;
        nx.x = hi1 ^ c.y ^ k0;
        nx.y = lo1;
        nx.z = hi0 ^ c.w ^ k1;
        nx.w = lo0;
        c = nx;
    }
    return c;
}

// The 4 draws of block q of ant a in iteration t: draw s is word (s & 3) of
// block (s >> 2); counter (q, a, t, 0), key (lo32 seed, hi32 seed).
__device__ __forceinline__ U4 draw_block(uint64_t seed, uint32_t t, uint32_t a, uint32_t q)
{
    U4 c{q, a, t, 0u};
    return philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ float unif24(uint32_t x)
{
    return __fmul_rn((float)(x >> 8), 0x1p-24f);   // exact: 24-bit integer times 2^-24
}

// ------------------------------------------------------- exp / ln (FP64)
// Deterministic elementary functions from +,-,*,/ only.
//   exp: x = k ln2 + r with ln2 split into a 40-bit head and its remainder
//        (Cody-Waite), e^r by its Taylor series to r^13 in Horner form, then
//        multiplication by the exact power 2^k.
//   ln:  x = m 2^e with m in [sqrt(1/2), sqrt(2)]; ln m = 2 atanh(s) with
//        s = (m-1)/(m+1) summed as an odd series to s^23 in Horner form in s^2;
//        ln x = (e*ln2_lo + ln m) + e*ln2_hi.
namespace dm {
constexpr double LN2_HI = 0x1.62e42fefa2000p-1;
constexpr double LN2_LO = 0x1.9ef35793c7673p-41;
constexpr double INV_LN2 = 0x1.71547652b82fep+0;
constexpr double SQRT2 = 0x1.6a09e667f3bcdp+0;
}  // namespace dm

__device__ __forceinline__ double taylor_coef(int i)
{
    // 1/i! for i = 0..13, each the double nearest to the exact rational
    switch (i) {
    case 0: return 1.0;
    case 1: return 1.0;
    case 2: return 0.5;
    case 3: return 1.0 / 6.0;
    case 4: return 1.0 / 24.0;
    case 5: return 1.0 / 120.0;
    case 6: return 1.0 / 720.0;
    case 7: return 1.0 / 5040.0;
    case 8: return 1.0 / 40320.0;
    case 9: return 1.0 / 362880.0;
    case 10: return 1.0 / 3628800.0;
    case 11: return 1.0 / 39916800.0;
    case 12: return 1.0 / 479001600.0;
    default: return 1.0 / 6227020800.0;
    }
}

__device__ __forceinline__ double det_exp(double x)
{
    if (x != x) return x;
    if (x > 709.0) return __longlong_as_double(0x7ff0000000000000ll);
    if (x < -708.0) return 0.0;
    double kd = floor(__dadd_rn(__dmul_rn(x, dm::INV_LN2), 0.5));
    double r = __dsub_rn(__dsub_rn(x, __dmul_rn(kd, dm::LN2_HI)), __dmul_rn(kd, dm::LN2_LO));
    double p = taylor_coef(13);
#pragma unroll
    for (int i = 12; i >= 0; --i) p = __dadd_rn(__dmul_rn(p, r), taylor_coef(i));
    long long kb = (long long)((int)kd + 1023) << 52;
    return __dmul_rn(p, __longlong_as_double(kb));
}

__device__ __forceinline__ double det_ln(double x)
{
    if (!(x > 0.0)) return x == 0.0 ? __longlong_as_double(0xfff0000000000000ll)
                                    : __longlong_as_double(0x7ff8000000000000ll);
    long long bits = __double_as_longlong(x);
    int e = (int)((bits >> 52) & 0x7ff);
    if (e == 0x7ff) return x;
    if (e == 0) {
        bits = __double_as_longlong(__dmul_rn(x, 0x1p54));
        e = (int)((bits >> 52) & 0x7ff) - 54;
    }
    e -= 1023;
    double m = __longlong_as_double((bits & 0x000fffffffffffffll) | 0x3ff0000000000000ll);
    if (m > dm::SQRT2) { m = __dmul_rn(m, 0.5); e += 1; }
    double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    double z = __dmul_rn(s, s);
    double P = 1.0 / 23.0;
    P = __dadd_rn(__dmul_rn(P, z), 1.0 / 21.0);
    P = __dadd_rn(__dmul_rn(P, z), 1.0 / 19.0);
    P = __dadd_rn(__dmul_rn(P, z), 1.0 / 17.0);
    P = __dadd_rn(__dmul_rn(P, z), 1.0 / 15.0);
    P = __dadd_rn(__dmul_rn(P, z), 1.0 / 13.0);
    P = __dadd_rn(__dmul_rn(P, z), 1.0 / 11.0);
    P = __dadd_rn(__dmul_rn(P, z), 1.0 / 9.0);
    P = __dadd_rn(__dmul_rn(P, z), 1.0 / 7.0);
    P = __dadd_rn(__dmul_rn(P, z), 1.0 / 5.0);
    P = __dadd_rn(__dmul_rn(P, z), 1.0 / 3.0);
    double lnm = __dmul_rn(2.0, __dadd_rn(s, __dmul_rn(s, __dmul_rn(z, P))));
    double ed = (double)e;
    return __dadd_rn(__dadd_rn(__dmul_rn(ed, dm::LN2_LO), lnm), __dmul_rn(ed, dm::LN2_HI));
}

// ------------------------------------------------------------ distances
// d_ij in FP64 (Sec. II-A): Euclidean distance of the FP32 coordinates with
// every operation rounded once, or the FP32 cost widened.
__device__ __forceinline__ double dist64(const DevInst &I, int i, int j)
{
    if (I.kind == 1) return (double)I.cost[(size_t)i * I.n + j];
    float2 a = reinterpret_cast<const float2 *>(I.xy)[i];
    float2 b = reinterpret_cast<const float2 *>(I.xy)[j];
    double dx = __dsub_rn((double)b.x, (double)a.x);
    double dy = __dsub_rn((double)b.y, (double)a.y);
    return __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

// Nearest-unvisited key: FP32 squared distance or FP32 cost (ties: lower index).
__device__ __forceinline__ float key32_xy(float2 a, float2 b)
{
    float dx = __fsub_rn(b.x, a.x), dy = __fsub_rn(b.y, a.y);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

__device__ __forceinline__ bool key_less(float k1, int u1, float k2, int u2)
{
    return k1 < k2 || (k1 == k2 && u1 < u2);
}

// heatmap value (FP32 or binary16) widened to FP64 exactly
__device__ __forceinline__ double heat_val(const DevInst &I, int p)
{
    if (I.h_half) {
        unsigned short h = reinterpret_cast<const unsigned short *>(I.val)[p];
        return (double)__half2float(*reinterpret_cast<const __half *>(&h));
    }
    return (double)reinterpret_cast<const float *>(I.val)[p];
}

// ---------------------------------------------------------- host helpers
struct Launch {
    cudaStream_t s;
};

// kernels (defined in the .cu files), launched by the host orchestration
// Each launcher returns the number of kernels it launched.
int launch_prep(const DevInst *d_inst, const DevInst *h_inst, int count, const int2 *d_rowmap,
                int rowmap_len, const int2 *d_slotmap, int slotmap_len, int *d_err,
                cudaStream_t s);
int launch_construct(const DevInst *d_inst, const int4 *d_warpmap, int warpmap_len, int apw,
                     int warps_per_block, int max_n, int max_kp, int count, cudaStream_t s);
int launch_iteration_tail(const DevInst *d_inst, int count, const int2 *d_slotmap,
                          int slotmap_len, bool any_ls, int max_n, int ls_all_m, cudaStream_t s);
// fused cluster kernel (fused.cu): one cluster of 2^clog CTAs per instance;
// d_iters (parallel to d_order, may be null) gives each cluster its own
// iteration count instead of `iters`
size_t fused_smem_bytes(int rows_cap, int kp_cap, int warps, int apw, int stride, int xy_cap,
                        int list_rows);
cudaError_t launch_fused(const DevInst *d_inst, const int32_t *d_order, const int32_t *d_iters,
                         int clusters, int clog, int apw, int warps, int rows_cap, int kp_cap, int stride,
                         int xy_cap, int list_rows, int iters, cudaStream_t s, bool after_resident);
constexpr size_t FUSED_SMEM_LIMIT = 220 * 1024;   // dynamic shared memory per CTA we allow

}  // namespace hac
