// Preparation of every instance of a batch: the preparation and initialisation
// steps of Algorithm 1.
//
//   heatmap view    h = (H + H^T)/2 when symmetrised (Sec. II-B): column i of H
//                   is materialised as a sorted row (counting transpose)
//   candidates      C_i from P_i = {j : h_ij > theta_h} (eq. heatmap_support),
//                   k closest members, filled with the nearest non-members
//   evidence        c_ij, b_i, e_ij (eqs. confidence, background, evidence)
//   kappa           q90 of the positive log-margins (eq. q90) by radix
//                   selection, R = tau_max/tau_min (eq. tau_ratio), eq. kappa
//   weights         W = fl32(eta^beta * exp(min(kappa ln e, clip)))
//   T_NN, bounds    nearest-neighbour tour, eq. tau_init / tau_min_nols, tau <- tau_max
//
// Work decomposition: rows of all instances are spread over warps through a
// host-built (instance, first row) table; per-instance reductions run one
// block per instance.
#include <cuda_fp16.h>

#include "lengths.cuh"

namespace hac {

constexpr int ROW_WARPS = 8;           // warps (= rows) per block in row kernels
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ void set_err(int *err, int code) { atomicCAS(err, 0, code); }

// ------------------------------------------------------------ validation

// Device-side check of a heatmap given by device pointers (host inputs are
// checked on the host): ranges, strict ordering, no self loops, values in [0,1].
__global__ void k_validate(const DevInst *insts, const int2 *rowmap, int *err)
{
    int2 rm = rowmap[blockIdx.x];
    const DevInst &I = insts[rm.x];
    int i = rm.y + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (i >= I.n) return;
    int b = I.rowptr[i], e = I.rowptr[i + 1];
    if (lane == 0 && (b < 0 || e < b || e > I.nnz || (i == 0 && b != 0) || (i == I.n - 1 && e != I.nnz)))
        set_err(err, HAC_EINVAL);
    if (b < 0 || e < b || e > I.nnz) return;
    for (int p = b + lane; p < e; p += 32) {
        int j = I.col[p];
        if (j < 0 || j >= I.n || j == i) set_err(err, HAC_EINVAL);
        if (p > b && I.col[p - 1] >= j) set_err(err, HAC_EINVAL);
        double v = heat_val(I, p);
        if (!(v >= 0.0 && v <= 1.0)) set_err(err, HAC_EINVAL);
    }
    if (I.kind == 0 && lane == 0) {
        float2 a = reinterpret_cast<const float2 *>(I.xy)[i];
        if (!isfinite(a.x) || !isfinite(a.y)) set_err(err, HAC_EINVAL);
        // with local search the 2-opt pre-test needs finite FP32 squared differences
        if (I.local_search && !(fabsf(a.x) <= 1e18f && fabsf(a.y) <= 1e18f)) set_err(err, HAC_EINVAL);
    }
    if (I.kind == 1)
        for (int j = lane; j < I.n; j += 32)
            if (!isfinite(I.cost[(size_t)i * I.n + j])) set_err(err, HAC_EINVAL);
}

// ------------------------------------------------------------ transpose

__global__ void k_tcount(const DevInst *insts, const int2 *rowmap)
{
    int2 rm = rowmap[blockIdx.x];
    const DevInst &I = insts[rm.x];
    if (!I.symmetrize) return;
    int i = rm.y + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (i >= I.n) return;
    for (int p = I.rowptr[i] + lane; p < I.rowptr[i + 1]; p += 32)
        atomicAdd(&I.trowptr[I.col[p] + 1], 1);
}

// in-place inclusive scan of trowptr[1..n] (one block per instance)
__global__ void k_tscan(const DevInst *insts)
{
    const DevInst &I = insts[blockIdx.x];
    if (!I.symmetrize) return;
    __shared__ int carry;
    __shared__ int wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 1; base <= I.n; base += blockDim.x) {
        int idx = base + threadIdx.x;
        int v = idx <= I.n ? I.trowptr[idx] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(FULL, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) wsum[w] = v;
        __syncthreads();
        if (w == 0) {
            int s = lane < nw ? wsum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(FULL, s, o);
                if (lane >= o) s += u;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        int add = carry + (w ? wsum[w - 1] : 0);
        if (idx <= I.n) I.trowptr[idx] = v + add;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = v + add;
        __syncthreads();
    }
}

// scatter the entries (i, j, v) to column j; order within a column is fixed later
__global__ void k_tfill(const DevInst *insts, const int2 *rowmap)
{
    int2 rm = rowmap[blockIdx.x];
    const DevInst &I = insts[rm.x];
    if (!I.symmetrize) return;
    int i = rm.y + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (i >= I.n) return;
    for (int p = I.rowptr[i] + lane; p < I.rowptr[i + 1]; p += 32) {
        int j = I.col[p];
        int q = I.trowptr[j] + atomicAdd(&I.tfill[j], 1);
        I.tcol[q] = i;
        I.tval[q] = heat_val(I, p);
    }
}

// sort each transposed row by source index (indices within a column are
// distinct); rows of kNN heatmaps are short, so a warp odd-even sort suffices.
__global__ void k_tsort(const DevInst *insts, const int2 *rowmap)
{
    int2 rm = rowmap[blockIdx.x];
    const DevInst &I = insts[rm.x];
    if (!I.symmetrize) return;
    int j = rm.y + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (j >= I.n) return;
    int b = I.trowptr[j], e = I.trowptr[j + 1], len = e - b;
    // odd-even transposition sort, repeated until the row is ordered
    for (int pass = 0; pass < len; ++pass) {
        bool sorted = true;
        for (int p = b + lane; p + 1 < e; p += 32)
            if (I.tcol[p] > I.tcol[p + 1]) sorted = false;
        if (__all_sync(FULL, sorted)) break;
        // odd-even transposition step pair
        for (int ph = 0; ph < 2; ++ph) {
            for (int p = b + ph + 2 * lane; p + 1 < e; p += 64) {
                int c0 = I.tcol[p], c1 = I.tcol[p + 1];
                if (c0 > c1) {
                    double v0 = I.tval[p], v1 = I.tval[p + 1];
                    I.tcol[p] = c1; I.tcol[p + 1] = c0;
                    I.tval[p] = v1; I.tval[p + 1] = v0;
                }
            }
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------ heatmap rows

struct RowView {
    int a0, a1;   // H row i: [a0, a1)
    int b0, b1;   // H^T row i (symmetrised view only): [b0, b1)
};

__device__ __forceinline__ RowView row_view(const DevInst &I, int i)
{
    RowView r;
    r.a0 = I.rowptr[i]; r.a1 = I.rowptr[i + 1];
    if (I.symmetrize) { r.b0 = I.trowptr[i]; r.b1 = I.trowptr[i + 1]; }
    else { r.b0 = r.b1 = 0; }
    return r;
}

__device__ __forceinline__ int find_sorted(const int32_t *col, int lo, int hi, int j)
{
    hi -= 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int c = col[mid];
        if (c == j) return mid;
        if (c < j) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// Entry q of the union enumeration of row i: returns false for an entry of
// H^T row i whose index also appears in H row i (it was already produced).
__device__ __forceinline__ bool row_entry(const DevInst &I, const RowView &r, int q, int &j,
                                          double &h)
{
    int la = r.a1 - r.a0;
    if (q < la) {
        j = I.col[r.a0 + q];
        double a = heat_val(I, r.a0 + q);
        if (!I.symmetrize) { h = a; return true; }
        int p = find_sorted(I.tcol, r.b0, r.b1, j);
        double b = p >= 0 ? I.tval[p] : 0.0;
        h = __dmul_rn(__dadd_rn(a, b), 0.5);
        return true;
    }
    int p = r.b0 + (q - la);
    j = I.tcol[p];
    if (find_sorted(I.col, r.a0, r.a1, j) >= 0) return false;
    h = __dmul_rn(__dadd_rn(0.0, I.tval[p]), 0.5);
    return true;
}

// ------------------------------------------------------------ warp selections

__device__ __forceinline__ bool dj_less(double d1, int j1, double d2, int j2)
{
    return d1 < d2 || (d1 == d2 && j1 < j2);
}

__device__ __forceinline__ void warp_min_dj(double &d, int &j)
{
    for (int o = 16; o; o >>= 1) {
        double d2 = __shfl_xor_sync(FULL, d, o);
        int j2 = __shfl_xor_sync(FULL, j, o);
        if (dj_less(d2, j2, d, j)) { d = d2; j = j2; }
    }
}

__device__ __forceinline__ void warp_min_kj(float &k, int &j)
{
    for (int o = 16; o; o >>= 1) {
        float k2 = __shfl_xor_sync(FULL, k, o);
        int j2 = __shfl_xor_sync(FULL, j, o);
        if (key_less(k2, j2, k, j)) { k = k2; j = j2; }
    }
}

#define DINF __longlong_as_double(0x7ff0000000000000ll)

// K smallest (d_ij, j) over j != i with pred(j) true, ascending, into lanes
// 0..K-1 of (dout, jout).  Euclidean instances first bound the answer with the
// FP32 squared distance (relative error below 4e-7) and evaluate the FP64
// distance only for nodes within a 1e-5 relative margin of the K-th key, a set
// that provably contains the exact K smallest; each of those distances is
// computed once (up to CACHE per lane, recomputed beyond).  Cost instances
// order by the FP32 cost directly (its FP64 widening is exact and monotone).
constexpr int CACHE = 4;

template <typename Pred>
__device__ void warp_knn(const DevInst &I, int i, int K, Pred pred, double &dout, int &jout)
{
    int lane = threadIdx.x & 31;
    const float2 *xy = reinterpret_cast<const float2 *>(I.xy);
    float2 pi = I.kind == 0 ? xy[i] : make_float2(0.f, 0.f);
    auto key = [&](int u) -> float {
        return I.kind == 0 ? key32_xy(pi, xy[u]) : I.cost[(size_t)i * I.n + u];
    };
    // pass 1: K-th smallest (key, u)
    float pk = -1.0f;
    int pu = -1;
    for (int r = 0; r < K; ++r) {
        float bk = __int_as_float(0x7f800000);
        int bu = 0x7fffffff;
        for (int u = lane; u < I.n; u += 32) {
            if (u == i || !pred(u)) continue;
            float kk = key(u);
            if (key_less(pk, pu, kk, u) && key_less(kk, u, bk, bu)) { bk = kk; bu = u; }
        }
        warp_min_kj(bk, bu);
        if (I.kind == 1 && lane == r) { dout = (double)bk; jout = bu; }
        pk = bk; pu = bu;
    }
    if (I.kind == 1) return;
    float thr = __fadd_rn(__fmul_rn(pk, 1.00001f), 1e-30f);
    // pass 2: exact (d, j) order among the nodes inside the margin
    double cd[CACHE];
    int cu[CACHE];
    int nc = 0;
    bool ovf = false;
    for (int u = lane; u < I.n; u += 32) {
        if (u == i || !pred(u) || !(key(u) <= thr)) continue;
        if (nc < CACHE) {
#pragma unroll
            for (int c = 0; c < CACHE; ++c)
                if (c == nc) { cd[c] = dist64(I, i, u); cu[c] = u; }
            ++nc;
        } else {
            ovf = true;
        }
    }
    double pd = -1.0;
    int pj = -1;
    for (int r = 0; r < K; ++r) {
        double bd = DINF;
        int bj = 0x7fffffff;
#pragma unroll
        for (int c = 0; c < CACHE; ++c)
            if (c < nc && dj_less(pd, pj, cd[c], cu[c]) && dj_less(cd[c], cu[c], bd, bj)) {
                bd = cd[c]; bj = cu[c];
            }
        if (ovf) {
            int seen = 0;
            for (int u = lane; u < I.n; u += 32) {
                if (u == i || !pred(u) || !(key(u) <= thr)) continue;
                if (seen++ < CACHE) continue;
                double d = dist64(I, i, u);
                if (dj_less(pd, pj, d, u) && dj_less(d, u, bd, bj)) { bd = d; bj = u; }
            }
        }
        warp_min_dj(bd, bj);
        if (lane == r) { dout = bd; jout = bj; }
        pd = bd; pj = bj;
    }
}

// ------------------------------------------------------------ heatmap support sets

// P_i with its h values, compacted into the row's region of the member buffer
// (capacity |H row i| + |H^T row i|), in enumeration order.
__global__ void k_members(const DevInst *insts, const int2 *rowmap)
{
    int2 rm = rowmap[blockIdx.x];
    const DevInst &I = insts[rm.x];
    int i = rm.y + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (i >= I.n) return;
    RowView rv = row_view(I, i);
    int total = (rv.a1 - rv.a0) + (rv.b1 - rv.b0);
    int base = rv.a0 + rv.b0;
    int cnt = 0;
    for (int q0 = 0; q0 < total; q0 += 32) {
        int q = q0 + lane;
        int j = 0;
        double h = 0.0;
        bool mem = q < total && row_entry(I, rv, q, j, h) && h > I.theta_h;
        unsigned bal = __ballot_sync(FULL, mem);
        if (mem) {
            int p = base + cnt + __popc(bal & ((1u << lane) - 1u));
            I.mem_j[p] = j;
            I.mem_h[p] = h;
        }
        cnt += __popc(bal);
    }
    if (lane == 0) I.mem_cnt[i] = cnt;
}

// ------------------------------------------------------------ candidate lists

// C_i (Sec. III-A): the k_eff members of P_i closest to i, or all members plus
// the nearest non-members; stored in ascending (d_ij, j) order with c_ij
// (eq. confidence).  Members are ordered by their FP32 key first; the FP64
// distance is taken only inside the margin that contains the exact answer.
__global__ void k_candidates(const DevInst *insts, const int2 *rowmap)
{
    int2 rm = rowmap[blockIdx.x];
    const DevInst &I = insts[rm.x];
    int i = rm.y + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (i >= I.n) return;
    RowView rv = row_view(I, i);
    const int base = rv.a0 + rv.b0;
    const int cnt = I.mem_cnt[i];
    const int32_t *mj = I.mem_j + base;
    const double *mh = I.mem_h + base;
    const int K = I.k_eff;
    const int km = cnt < K ? cnt : K;
    const float2 *xy = reinterpret_cast<const float2 *>(I.xy);
    float2 pi = I.kind == 0 ? xy[i] : make_float2(0.f, 0.f);
    auto key = [&](int u) -> float {
        return I.kind == 0 ? key32_xy(pi, xy[u]) : I.cost[(size_t)i * I.n + u];
    };
    // threshold: every member when there are at most k of them, else a margin
    // above the k-th smallest (key, j) (exact for cost instances)
    float thr = __int_as_float(0x7f800000);
    if (cnt > K) {
        float pk = -1.0f;
        int pu = -1;
        for (int r = 0; r < K; ++r) {
            float bk = __int_as_float(0x7f800000);
            int bu = 0x7fffffff;
            for (int q = lane; q < cnt; q += 32) {
                int j = mj[q];
                float kk = key(j);
                if (key_less(pk, pu, kk, j) && key_less(kk, j, bk, bu)) { bk = kk; bu = j; }
            }
            warp_min_kj(bk, bu);
            pk = bk; pu = bu;
        }
        thr = I.kind == 0 ? __fadd_rn(__fmul_rn(pk, 1.00001f), 1e-30f) : pk;
    }
    // exact distances of the members inside the threshold, once each
    double cd[CACHE], ch[CACHE];
    int cj[CACHE];
    int nc = 0;
    bool ovf = false;
    for (int q = lane; q < cnt; q += 32) {
        int j = mj[q];
        if (!(key(j) <= thr)) continue;
        if (nc < CACHE) {
#pragma unroll
            for (int c = 0; c < CACHE; ++c)
                if (c == nc) { cd[c] = dist64(I, i, j); cj[c] = j; ch[c] = mh[q]; }
            ++nc;
        } else {
            ovf = true;
        }
    }
    double md = DINF, mhv = 0.0;
    int mjv = 0x7fffffff;
    double pd = -1.0;
    int pj = -1;
    for (int r = 0; r < km; ++r) {
        double bd = DINF, bh = 0.0;
        int bj = 0x7fffffff;
#pragma unroll
        for (int c = 0; c < CACHE; ++c)
            if (c < nc && dj_less(pd, pj, cd[c], cj[c]) && dj_less(cd[c], cj[c], bd, bj)) {
                bd = cd[c]; bj = cj[c]; bh = ch[c];
            }
        if (ovf) {
            int seen = 0;
            for (int q = lane; q < cnt; q += 32) {
                int j = mj[q];
                if (!(key(j) <= thr)) continue;
                if (seen++ < CACHE) continue;
                double d = dist64(I, i, j);
                if (dj_less(pd, pj, d, j) && dj_less(d, j, bd, bj)) { bd = d; bj = j; bh = mh[q]; }
            }
        }
        for (int o = 16; o; o >>= 1) {
            double d2 = __shfl_xor_sync(FULL, bd, o);
            int j2 = __shfl_xor_sync(FULL, bj, o);
            double h2 = __shfl_xor_sync(FULL, bh, o);
            if (dj_less(d2, j2, bd, bj)) { bd = d2; bj = j2; bh = h2; }
        }
        if (lane == r) { md = bd; mjv = bj; mhv = bh; }
        pd = bd; pj = bj;
    }
    // nearest non-members fill the remaining slots (lanes km..K-1)
    double fd = DINF;
    int fj = 0x7fffffff;
    if (km < K) {
        auto nonmember = [&](int u) {
            for (int q = 0; q < cnt; ++q) if (mj[q] == u) return false;
            return true;
        };
        double d0 = DINF;
        int j0 = 0x7fffffff;
        warp_knn(I, i, K - km, nonmember, d0, j0);
        int src = lane - km;
        double dsh = __shfl_sync(FULL, d0, src < 0 ? 0 : src);
        int jsh = __shfl_sync(FULL, j0, src < 0 ? 0 : src);
        if (lane >= km && lane < K) { fd = dsh; fj = jsh; }
    }
    // merge: lane c holds one entry; its slot is its rank in ascending (d, j)
    bool have = lane < K;
    double d = lane < km ? md : fd;
    int j = lane < km ? mjv : fj;
    double h = lane < km ? mhv : 0.0;
    int rank = 0;
    for (int l = 0; l < K; ++l) {
        double d2 = __shfl_sync(FULL, d, l);
        int j2 = __shfl_sync(FULL, j, l);
        if (have && dj_less(d2, j2, d, j)) ++rank;
    }
    size_t row = (size_t)i * I.k_pad;
    if (have) {
        I.cand[row + rank] = j;
        I.cdist[row + rank] = d;
        I.conf[row + rank] = h > I.theta_h ? h : 0.0;
    } else if (lane < I.k_pad) {
        I.cand[row + lane] = -1;
        I.cdist[row + lane] = 0.0;
        I.conf[row + lane] = 0.0;
    }
}

// ------------------------------------------------------------ evidence

__global__ void k_evidence(const DevInst *insts, const int2 *rowmap)
{
    int2 rm = rowmap[blockIdx.x];
    const DevInst &I = insts[rm.x];
    int i = rm.y + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (i >= I.n) return;
    size_t row = (size_t)i * I.k_pad;
    int ds = I.degree_target;
    double v = lane < I.k_eff ? I.conf[row + lane] : 0.0;
    double stat = 0.0;
    if (I.baseline_scope == 0) {
        // (d*+1)-th largest positive c over the candidate slots
        int rank = 0;
        for (int l = 0; l < 32; ++l) {
            double v2 = __shfl_sync(FULL, v, l);
            if (v2 > v || (v2 == v && l < lane)) ++rank;
        }
        unsigned hit = __ballot_sync(FULL, v > 0.0 && rank == ds);
        if (hit) stat = __shfl_sync(FULL, v, __ffs(hit) - 1);
    } else {
        // (d*+1)-th largest positive h over the whole heatmap row (P_i)
        RowView rv = row_view(I, i);
        const int cnt = I.mem_cnt[i];
        const double *mh = I.mem_h + rv.a0 + rv.b0;
        double ph = DINF;
        int pq = -1;
        bool found = true;
        for (int r = 0; r <= ds && found; ++r) {
            double bh = -1.0;
            int bq = 0x7fffffff;
            for (int q = lane; q < cnt; q += 32) {
                double h = mh[q];
                // next in (descending h, ascending position) order after (ph, pq)
                bool after = h < ph || (h == ph && q > pq);
                bool better = h > bh || (h == bh && q < bq);
                if (after && better) { bh = h; bq = q; }
            }
            for (int o = 16; o; o >>= 1) {
                double h2 = __shfl_xor_sync(FULL, bh, o);
                int q2 = __shfl_xor_sync(FULL, bq, o);
                if (h2 > bh || (h2 == bh && q2 < bq)) { bh = h2; bq = q2; }
            }
            if (bh < 0.0) found = false;
            else { ph = bh; pq = bq; }
        }
        stat = found ? ph : 0.0;
    }
    double b = stat > I.eps ? stat : I.eps;
    if (lane == 0) I.base[i] = b;
    if (lane < I.k_pad) {
        double e = 0.0, le = 0.0;
        if (lane < I.k_eff) {
            double cc = v > I.eps ? v : I.eps;
            double r = __ddiv_rn(cc, b);
            e = r > 1.0 ? r : 1.0;
            le = e > 1.0 ? det_ln(e) : 0.0;
        }
        I.evid[row + lane] = e;
        I.logev[row + lane] = le;
    }
}

// ------------------------------------------------------------ q90 and kappa

// rank-th smallest (0-based) of the positive entries of logev (bit patterns of
// positive doubles order like unsigned integers): 8 passes of 8-bit digits.
__device__ double block_select(const DevInst &I, size_t nslots, long long rank, int *hist)
{
    unsigned long long prefix = 0, pmask = 0;
    long long r = rank;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[t] = 0;
        __syncthreads();
        for (size_t s = threadIdx.x; s < nslots; s += blockDim.x) {
            double x = I.logev[s];
            if (!(x > 0.0)) continue;
            unsigned long long k = (unsigned long long)__double_as_longlong(x);
            if ((k & pmask) != prefix) continue;
            atomicAdd(&hist[(k >> shift) & 255], 1);
        }
        __syncthreads();
        __shared__ int digit;
        __shared__ long long before;
        if (threadIdx.x == 0) {
            long long acc = 0;
            int d = 0;
            for (; d < 256; ++d) {
                if (acc + hist[d] > r) break;
                acc += hist[d];
            }
            digit = d; before = acc;
        }
        __syncthreads();
        prefix |= (unsigned long long)digit << shift;
        pmask |= 255ull << shift;
        r -= before;
        __syncthreads();
    }
    return __longlong_as_double((long long)prefix);
}

__global__ void k_kappa(const DevInst *insts)
{
    const DevInst &I = insts[blockIdx.x];
    __shared__ int hist[256];
    __shared__ int wcount[32];
    size_t nslots = (size_t)I.n * I.k_pad;
    int c = 0;
    for (size_t s = threadIdx.x; s < nslots; s += blockDim.x) c += I.logev[s] > 0.0;
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if ((threadIdx.x & 31) == 0) wcount[threadIdx.x >> 5] = c;
    __syncthreads();
    long long N = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) N += wcount[w];
    __syncthreads();
    // Edges/n diagnostic (Sec. VI-A): sum of the support-set sizes |P_i|
    long long ne = 0;
    for (int i = threadIdx.x; i < I.n; i += blockDim.x) ne += I.mem_cnt[i];
    for (int o = 16; o; o >>= 1) ne += __shfl_xor_sync(FULL, ne, o);
    __shared__ long long wne[32];
    if ((threadIdx.x & 31) == 0) wne[threadIdx.x >> 5] = ne;
    __syncthreads();
    long long NE = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) NE += wne[w];
    double q = 0.0;
    if (N > 0) {
        double h = __dmul_rn((double)(N - 1), I.q_level);
        double lo = floor(h);
        long long l = (long long)lo;
        if (l >= N - 1) {
            q = block_select(I, nslots, N - 1, hist);
        } else {
            double x0 = block_select(I, nslots, l, hist);
            double x1 = block_select(I, nslots, l + 1, hist);
            q = __dadd_rn(x0, __dmul_rn(__dsub_rn(h, lo), __dsub_rn(x1, x0)));
        }
    }
    if (threadIdx.x == 0) {
        InstState *st = I.st;
        double px = det_exp(__ddiv_rn(det_ln(I.p_best), (double)I.n));
        double R;
        if (I.local_search) R = __dmul_rn(2.0, (double)I.n);
        else R = __ddiv_rn(__dmul_rn(__ddiv_rn((double)(I.k_eff - 1), 2.0), px), __dsub_rn(1.0, px));
        // eq. kappa; kappa_mode 1 and 2 are the ablation variants of Sec. V-D
        // (fixed kappa = 1; the cap factor c_cap dropped)
        double kap = 0.0;
        if (I.kappa_mode == 1) kap = 1.0;
        else if (q > 0.0 && R > 1.0)
            kap = __ddiv_rn(__dmul_rn(I.kappa_mode == 2 ? I.alpha : __dmul_rn(I.c_cap, I.alpha), det_ln(R)), q);
        st->q90 = q; st->Rhat = R; st->kappa = kap; st->p_x = px;
        st->n_lambda = (int)N;
        st->n_edges = (unsigned long long)NE;
    }
}

// ------------------------------------------------------------ weights

__global__ void k_weights(const DevInst *insts, const int2 *slotmap)
{
    int2 sm = slotmap[blockIdx.x];
    const DevInst &I = insts[sm.x];
    size_t s = (size_t)sm.y + threadIdx.x;
    size_t nslots = (size_t)I.n * I.k_pad;
    if (s >= nslots) return;
    int c = (int)(s % I.k_pad);
    if (c >= I.k_eff) { I.W[s] = 0.0f; return; }
    double d = I.cdist[s] > DFLOOR ? I.cdist[s] : DFLOOR;
    double eta = __ddiv_rn(1.0, d);
    double hb = I.beta == 2.0 ? __dmul_rn(eta, eta) : det_exp(__dmul_rn(I.beta, det_ln(eta)));
    double E = 1.0;
    double le = I.logev[s];
    if (le > 0.0) {
        double lw = __dmul_rn(I.st->kappa, le);
        E = det_exp(lw < I.logw_clip ? lw : I.logw_clip);
    }
    I.W[s] = __double2float_rn(__dmul_rn(hb, E));
}

// ------------------------------------------------------------ 2-opt neighbour lists

__global__ void k_nbr(const DevInst *insts, const int2 *rowmap)
{
    int2 rm = rowmap[blockIdx.x];
    const DevInst &I = insts[rm.x];
    if (!I.local_search) return;
    int a = rm.y + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (a >= I.n) return;
    double d = 0.0;
    int j = 0;
    warp_knn(I, a, I.ls_k, [](int) { return true; }, d, j);
    if (lane < I.ls_k) {
        I.nbr[(size_t)a * I.ls_k + lane] = j;
        I.nbrd[(size_t)a * I.ls_k + lane] = d;
        I.nbrd32[(size_t)a * I.ls_k + lane] = __double2float_rn(d);
    }
}

// ------------------------------------------------------------ nearest-unvisited lookup lists

// The fallback of Alg. 2 happens when no candidate of the current node has a
// positive weight.  When every candidate's choice value stays positive for
// the whole run (alpha = 1 and fl32(tau_min * W) > 0 at the smallest bound,
// which only grows), that means all candidates are visited, so the lookup
// list may skip them.
__global__ void k_fbl_check(const DevInst *insts, const int2 *slotmap)
{
    int2 sm = slotmap[blockIdx.x];
    const DevInst &I = insts[sm.x];
    if (!I.fbl) return;
    size_t s = (size_t)sm.y + threadIdx.x;
    if (s >= (size_t)I.n * I.k_pad) return;
    if (I.alpha != 1.0) { if (s == 0) I.st->fbl_unsafe = 1; return; }
    if (I.cand[s] >= 0 && !(__fmul_rn(I.st->tau_min, I.W[s]) > 0.0f)) I.st->fbl_unsafe = 1;
}

// For the fallback of Alg. 2 (instances without a second-level list, n >
// 65535): the 32 nodes u != i (not in C_i when that is safe, see
// k_fbl_check) with the smallest (FP32 key, u), ascending, -1 when fewer
// exist.  If one of them is unvisited at a fallback, the first unvisited
// one is the nearest unvisited node, exactly.
__global__ void k_fbl(const DevInst *insts, const int2 *rowmap, int words_per_warp)
{
    extern __shared__ unsigned int excl_mask[];
    int2 rm = rowmap[blockIdx.x];
    const DevInst &I = insts[rm.x];
    if (!I.fbl || I.fbl2) return;   // with a second-level list, k_fbl2 writes both
    const int i = rm.y + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (i >= I.n) return;
    unsigned *mask = excl_mask + (size_t)(threadIdx.x / 32) * words_per_warp;
    const int nw = (I.n + 31) >> 5;
    for (int w = lane; w < nw; w += 32) mask[w] = 0u;
    __syncwarp();
    const bool excl = I.st->fbl_unsafe == 0;
    if (excl && lane < I.k_pad) {
        const int j = I.cand[(size_t)i * I.k_pad + lane];
        if (j >= 0) atomicOr(&mask[j >> 5], 1u << (j & 31));
    }
    __syncwarp();
    const float2 *xy = reinterpret_cast<const float2 *>(I.xy);
    const float2 pi = I.kind == 0 ? xy[i] : make_float2(0.f, 0.f);
    const int avail = I.n - 1 - (excl ? I.k_eff : 0);
    const int K = avail < 32 ? avail : 32;
    float pk = -1.0f;
    int pu = -1, mine = -1;
    for (int r = 0; r < K; ++r) {
        float bk = __int_as_float(0x7f800000);
        int bu = 0x7fffffff;
        for (int u = lane; u < I.n; u += 32) {
            if (u == i || ((mask[u >> 5] >> (u & 31)) & 1u)) continue;
            const float kk = I.kind == 0 ? key32_xy(pi, xy[u]) : I.cost[(size_t)i * I.n + u];
            if (key_less(pk, pu, kk, u) && key_less(kk, u, bk, bu)) { bk = kk; bu = u; }
        }
        warp_min_kj(bk, bu);
        if (lane == r) mine = bu;
        pk = bk;
        pu = bu;
    }
    I.fbl[(size_t)i * 32 + lane] = lane < K ? mine : -1;
}

// Order-preserving bit pattern of a key: unsigned comparison of the patterns
// is the float comparison (-0 is taken as +0, as the float compare does).
__device__ __forceinline__ unsigned ord_key(float k)
{
    const unsigned b = __float_as_uint(__fadd_rn(k, 0.0f));
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Both lookup lists for the fallback of Alg. 2 (instances of n <= 65535):
// ranks 0..31 of the order of k_fbl (nodes u != i, not in C_i when that is
// safe, by (FP32 key, u)) into fbl, -1 past the last node, and ranks 32..287
// into the second-level list, 0xffff past the last node.  When the 32 nearest
// are all visited, the first unvisited node of the second list is the
// nearest unvisited node, exactly.
// One warp per row: the key of rank T = min(288, available) by an exact
// radix selection (four 8-bit digits of ord_key), the nodes below it plus
// the lowest-index nodes at it, then a bitonic sort of those (key, u) pairs.
// Shared memory per warp: sort buffer (FBL2_SORT x 8 B) | histogram (256) |
// exclusion mask (`words_per_warp`, even).
__global__ void k_fbl2(const DevInst *insts, const int2 *rowmap, int words_per_warp)
{
    extern __shared__ unsigned long long fbl2_smem[];
    const int2 rm = rowmap[blockIdx.x];
    const DevInst &I = insts[rm.x];
    if (!I.fbl2) return;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = rm.y + wib;
    if (i >= I.n) return;
    unsigned long long *buf = fbl2_smem + (size_t)wib * (FBL2_SORT + (256 + words_per_warp) / 2);
    unsigned *hist = reinterpret_cast<unsigned *>(buf + FBL2_SORT);
    unsigned *mask = hist + 256;
    const int n = I.n, nw = (n + 31) >> 5;
    for (int w = lane; w < nw; w += 32) mask[w] = 0u;
    __syncwarp();
    if (I.st->fbl_unsafe == 0 && lane < I.k_pad) {
        const int j = I.cand[(size_t)i * I.k_pad + lane];
        if (j >= 0) atomicOr(&mask[j >> 5], 1u << (j & 31));
    }
    if (lane == 0) atomicOr(&mask[i >> 5], 1u << (i & 31));
    __syncwarp();
    const float2 *xy = reinterpret_cast<const float2 *>(I.xy);
    const float2 pi = I.kind == 0 ? xy[i] : make_float2(0.f, 0.f);
    const float *crow = I.kind == 1 ? I.cost + (size_t)i * n : nullptr;
    auto okey = [&](int u) { return ord_key(I.kind == 0 ? key32_xy(pi, xy[u]) : crow[u]); };
    auto live = [&](int u) { return !((mask[u >> 5] >> (u & 31)) & 1u); };

    int avail = 0;
    for (int w = lane; w < nw; w += 32) {
        unsigned v = ~mask[w];
        if (w == nw - 1 && (n & 31)) v &= (1u << (n & 31)) - 1u;
        avail += __popc(v);
    }
    avail = __reduce_add_sync(FULL, avail);
    const int T = min(avail, FBL1_LEN + FBL2_LEN);
    uint16_t *out = I.fbl2 + (size_t)i * FBL2_LEN;
    int32_t *out1 = I.fbl + (size_t)i * FBL1_LEN;
    if (T == 0) {
        out1[lane] = -1;
        for (int r = lane; r < FBL2_LEN; r += 32) out[r] = (uint16_t)0xffff;
        return;
    }

    // radix selection of the key of rank T (1-based); `need` ends as the
    // number of nodes taken at that key
    unsigned prefix = 0u, pmask = 0u;
    int need = T;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = lane; b < 256; b += 32) hist[b] = 0u;
        __syncwarp();
        for (int u = lane; u < n; u += 32) {
            if (!live(u)) continue;
            const unsigned k = okey(u);
            if ((k & pmask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
        }
        __syncwarp();
        unsigned c[8], tot = 0u;
#pragma unroll
        for (int b = 0; b < 8; ++b) { c[b] = hist[8 * lane + b]; tot += c[b]; }
        unsigned inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += v;
        }
        const unsigned exc = inc - tot;
        const unsigned owner = __ballot_sync(FULL, exc < (unsigned)need && (unsigned)need <= inc);
        const int L = __ffs(owner) - 1;
        int d = 0;
        unsigned before = 0u;
        if (lane == L) {
            unsigned acc = exc;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                if (acc + c[b] >= (unsigned)need) { d = 8 * lane + b; before = acc; break; }
                acc += c[b];
            }
        }
        d = __shfl_sync(FULL, d, L);
        before = __shfl_sync(FULL, before, L);
        need -= (int)before;
        prefix |= (unsigned)d << shift;
        pmask |= 255u << shift;
        __syncwarp();
    }

    // the T smallest (key, u): every node below the selected key and the
    // `need` lowest-index nodes at it, compacted in index order
    int pos = 0, ties = 0;
    for (int base = 0; base < n; base += 32) {
        const int u = base + lane;
        unsigned k = 0xffffffffu;
        bool lt = false, eq = false;
        if (u < n && live(u)) { k = okey(u); lt = k < prefix; eq = k == prefix; }
        const unsigned below = (1u << lane) - 1u;
        const unsigned beq = __ballot_sync(FULL, eq);
        const bool take = lt || (eq && ties + __popc(beq & below) < need);
        const unsigned bt = __ballot_sync(FULL, take);
        if (take) buf[pos + __popc(bt & below)] = ((unsigned long long)k << 32) | (unsigned)u;
        pos += __popc(bt);
        ties += __popc(beq);
    }
    for (int r = pos + lane; r < FBL2_SORT; r += 32) buf[r] = ~0ull;
    __syncwarp();
    // bitonic sort, ascending (each element is in exactly one pair per stage)
    for (int k = 2; k <= FBL2_SORT; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int x = lane; x < FBL2_SORT; x += 32) {
                const int y = x ^ j;
                if (y > x) {
                    const unsigned long long a = buf[x], b = buf[y];
                    if ((a > b) == ((x & k) == 0)) { buf[x] = b; buf[y] = a; }
                }
            }
            __syncwarp();
        }
    out1[lane] = lane < T ? (int32_t)(buf[lane] & 0xffffffffu) : -1;
    for (int r = lane; r < FBL2_LEN; r += 32)
        out[r] = r + FBL1_LEN < T ? (uint16_t)(buf[r + FBL1_LEN] & 0xffffu) : (uint16_t)0xffff;
}

// ------------------------------------------------------------ T_NN

// Nearest-neighbour tour from node 0 (one block per instance): each step takes
// the unvisited node of smallest (FP32 key, index); then L_nn.
__global__ void k_nn_tour(const DevInst *insts)
{
    const DevInst &I = insts[blockIdx.x];
    extern __shared__ unsigned int vis[];
    __shared__ float rk[32];
    __shared__ int ru[32];
    __shared__ int cur_s;
    int n = I.n, nw = (n + 31) >> 5;
    for (int w = threadIdx.x; w < nw; w += blockDim.x) vis[w] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) { vis[0] = 1u; I.nn_tour[0] = 0; cur_s = 0; }
    __syncthreads();
    const float2 *xy = reinterpret_cast<const float2 *>(I.xy);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int cur = 0;
    for (int s = 1; s < n; ++s) {
        float2 pc = I.kind == 0 ? xy[cur] : make_float2(0.f, 0.f);
        float bk = __int_as_float(0x7f800000);
        int bu = 0x7fffffff;
        for (int u = threadIdx.x; u < n; u += blockDim.x) {
            if (vis[u >> 5] & (1u << (u & 31))) continue;
            float kk = I.kind == 0 ? key32_xy(pc, xy[u]) : I.cost[(size_t)cur * n + u];
            if (key_less(kk, u, bk, bu)) { bk = kk; bu = u; }
        }
        warp_min_kj(bk, bu);
        if (lane == 0) { rk[wid] = bk; ru[wid] = bu; }
        __syncthreads();
        if (wid == 0) {
            bk = lane < nwarps ? rk[lane] : __int_as_float(0x7f800000);
            bu = lane < nwarps ? ru[lane] : 0x7fffffff;
            warp_min_kj(bk, bu);
            if (lane == 0) {
                if ((unsigned)bu >= (unsigned)n) bu = 0;   // unreachable for finite keys
                vis[bu >> 5] |= 1u << (bu & 31);
                I.nn_tour[s] = bu;
                cur_s = bu;
            }
        }
        __syncthreads();
        cur = cur_s;
    }
    __syncthreads();
    if (wid == 0) {   // eq. (tour_length) in the blocked pairwise order
        const double Ln = warp_tour_length(I, I.nn_tour);
        if (lane == 0) I.st->L_nn = Ln;
    }
}

// ------------------------------------------------------------ bounds and tau

__device__ __forceinline__ void set_bounds(const DevInst &I, InstState *st, double L)
{
    double tmax = __ddiv_rn(1.0, __dmul_rn(I.rho, L));
    double tmin;
    if (I.local_search) tmin = __ddiv_rn(tmax, __dmul_rn(2.0, (double)I.n));
    else tmin = __ddiv_rn(__dmul_rn(tmax, __dsub_rn(1.0, st->p_x)),
                          __dmul_rn(__ddiv_rn((double)(I.k_eff - 1), 2.0), st->p_x));
    st->tau_max64 = tmax; st->tau_min64 = tmin;
    st->tau_max = __double2float_rn(tmax);
    st->tau_min = __double2float_rn(tmin);
}

// fl32(tau^alpha * W); for alpha = 1 the exact FP64 product rounded once is the FP32 product
__device__ __forceinline__ float choice_of(const DevInst &I, float tau, float W)
{
    if (I.alpha == 1.0) return __fmul_rn(tau, W);
    double a = det_exp(__dmul_rn(I.alpha, det_ln((double)tau)));
    return __double2float_rn(__dmul_rn(a, (double)W));
}

__global__ void k_init_bounds(const DevInst *insts)
{
    const DevInst &I = insts[blockIdx.x];
    InstState *st = I.st;
    if (threadIdx.x == 0) {
        set_bounds(I, st, st->L_nn);
        st->L_gb = st->L_nn;
        st->L_ib = 0.0;
        st->t = 0; st->ib = -1; st->active = 0; st->n_fallback = 0;
        st->L_rb = __longlong_as_double(0x7ff0000000000000ll);   // no restart-best yet
        st->L_dep = 0.0; st->t_restart = 0; st->t_rbimp = 0; st->u_gb = 25; st->n_restarts = 0;
        st->bf_count = 0;
    }
    for (int s = threadIdx.x; s < I.n; s += blockDim.x) I.gb_tour[s] = I.nn_tour[s];
}

__global__ void k_init_tau(const DevInst *insts, const int2 *slotmap)
{
    int2 sm = slotmap[blockIdx.x];
    const DevInst &I = insts[sm.x];
    size_t s = (size_t)sm.y + threadIdx.x;
    if (s >= (size_t)I.n * I.k_pad) return;
    bool real = I.cand[s] >= 0;
    float tau = real ? I.st->tau_max : 0.0f;
    I.tau[s] = tau;
    I.choice[s] = real ? choice_of(I, tau, I.W[s]) : 0.0f;
}

// defined in twoopt.cu
void launch_two_opt_nn(const DevInst *d_inst, int count, int max_n, cudaStream_t s);

int launch_prep(const DevInst *d_inst, const DevInst *h_inst, int count, const int2 *d_rowmap,
                int rowmap_len, const int2 *d_slotmap, int slotmap_len, int *d_err,
                cudaStream_t s)
{
    int threads = ROW_WARPS * 32;
    bool any_sym = false, any_ls = false;
    int max_n = 0;
    for (int b = 0; b < count; ++b) {
        any_sym |= h_inst[b].symmetrize != 0;
        any_ls |= h_inst[b].local_search != 0;
        max_n = h_inst[b].n > max_n ? h_inst[b].n : max_n;
    }
    int launched = 0;
    k_validate<<<rowmap_len, threads, 0, s>>>(d_inst, d_rowmap, d_err);
    ++launched;
    if (any_sym) {
        k_tcount<<<rowmap_len, threads, 0, s>>>(d_inst, d_rowmap);
        k_tscan<<<count, 1024, 0, s>>>(d_inst);
        k_tfill<<<rowmap_len, threads, 0, s>>>(d_inst, d_rowmap);
        k_tsort<<<rowmap_len, threads, 0, s>>>(d_inst, d_rowmap);
        launched += 4;
    }
    k_members<<<rowmap_len, threads, 0, s>>>(d_inst, d_rowmap);
    k_candidates<<<rowmap_len, threads, 0, s>>>(d_inst, d_rowmap);
    k_evidence<<<rowmap_len, threads, 0, s>>>(d_inst, d_rowmap);
    k_kappa<<<count, 1024, 0, s>>>(d_inst);
    k_weights<<<slotmap_len, 1024, 0, s>>>(d_inst, d_slotmap);
    launched += 5;
    if (any_ls) { k_nbr<<<rowmap_len, threads, 0, s>>>(d_inst, d_rowmap); ++launched; }
    size_t vis_bytes = (size_t)((max_n + 31) / 32) * 4;
    k_nn_tour<<<count, 1024, vis_bytes, s>>>(d_inst);
    if (any_ls) { launch_two_opt_nn(d_inst, count, max_n, s); ++launched; }
    k_init_bounds<<<count, 256, 0, s>>>(d_inst);
    k_fbl_check<<<slotmap_len, 1024, 0, s>>>(d_inst, d_slotmap);
    const int wpw = (max_n + 31) / 32;
    const size_t fbl_smem = (size_t)ROW_WARPS * wpw * sizeof(unsigned);
    if (fbl_smem > 48 * 1024)
        cudaFuncSetAttribute(k_fbl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fbl_smem);
    k_fbl<<<rowmap_len, threads, fbl_smem, s>>>(d_inst, d_rowmap, wpw);
    const int wpw2 = ((wpw < 2048 ? wpw : 2048) + 1) & ~1;   // lists of n <= 65535 only
    const size_t fbl2_smem = (size_t)ROW_WARPS * (FBL2_SORT * 8 + (256 + wpw2) * 4);
    if (fbl2_smem > 48 * 1024)
        cudaFuncSetAttribute(k_fbl2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fbl2_smem);
    k_fbl2<<<rowmap_len, threads, fbl2_smem, s>>>(d_inst, d_rowmap, wpw2);
    k_init_tau<<<slotmap_len, 1024, 0, s>>>(d_inst, d_slotmap);
    return launched + 6;
}

}  // namespace hac
