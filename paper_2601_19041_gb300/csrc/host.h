// Host-side helpers shared by the batch API (api.cu) and the server
// (serve.cu): input checks, the workspace layout of one instance, and the
// grouping of instances for the fused cluster kernel.
#pragma once

#include <algorithm>
#include <atomic>
#include <thread>
#include <cmath>
#include <cstring>
#include <vector>

#include "hac_internal.cuh"

namespace hac {
namespace host {

extern thread_local int g_last_cuda;

#define CK(x)                                              \
    do {                                                   \
        cudaError_t e_ = (x);                              \
        if (e_ != cudaSuccess) {                           \
            g_last_cuda = (int)e_;                         \
            return HAC_ECUDA;                              \
        }                                                  \
    } while (0)

constexpr int ROWS_PER_BLOCK = 8;      // matches the row kernels (8 warps, a row each)
constexpr int SLOTS_PER_BLOCK = 1024;  // matches the slot kernels
constexpr int GRAPH_CHUNK = 10;        // iterations per captured graph
constexpr int FBL_LEN = FBL1_LEN;      // nearest-unvisited lookup list

struct Arena {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        off = (off + 255) & ~(size_t)255;
        size_t o = off;
        off += bytes;
        return o;
    }
};

struct Sizes {
    int n, kind, kp, k_eff, m, iters, ls, ls_k, sym, half;
    long long nnz;
};

inline bool finite_f(float x) { return std::isfinite(x); }

inline int check_params(const hac_instance &in, const hac_params &p)
{
    if (in.n < 3 || in.n > HAC_NMAX) return HAC_EINVAL;
    if (in.kind != 0 && in.kind != 1) return HAC_EINVAL;
    if (in.kind == 0 && !in.coords) return HAC_EINVAL;
    if (in.kind == 1 && !in.cost) return HAC_EINVAL;
    if (!in.h_rowptr || (in.h_dtype != 0 && in.h_dtype != 1)) return HAC_EINVAL;
    if (p.k < 1 || p.k > HAC_KMAX || p.m < 1 || p.m > HAC_MMAX || p.iterations < 0) return HAC_EINVAL;
    if (!(p.rho > 0.0 && p.rho < 1.0) || p.degree_target < 1) return HAC_EINVAL;
    if (!(p.alpha > 0.0) || !(p.beta >= 0.0) || !(p.theta_h >= 0.0) || !(p.eps > 0.0)) return HAC_EINVAL;
    if (!(p.q_level >= 0.0 && p.q_level <= 1.0) || !(p.p_best > 0.0 && p.p_best < 1.0)) return HAC_EINVAL;
    if (!(p.c_cap >= 0.0) || !(p.logw_clip > 0.0)) return HAC_EINVAL;
    if (p.baseline_scope != 0 && p.baseline_scope != 1) return HAC_EINVAL;
    if (p.schedule != 0 && p.schedule != 1) return HAC_EINVAL;
    if (p.kappa_mode < 0 || p.kappa_mode > 2) return HAC_EINVAL;
    if (p.local_search < 0 || p.local_search > 4) return HAC_EINVAL;
    if (p.local_search) {
        if (in.kind != 0 && p.local_search >= 3) return HAC_EUNSUPPORTED;   // 3-opt: symmetric only
        if (p.ls_k < 1 || p.ls_k > 32 || p.ls_k > in.n - 1) return HAC_EINVAL;
    }
    if (in.symmetrize != 0 && in.symmetrize != 1) return HAC_EINVAL;
    return HAC_OK;
}

// |x|, |y| bound with local search: the 2-opt pre-test's FP32 squared
// differences stay finite (2e18^2 * 2 < FLT_MAX)
constexpr double LS_COORD_MAX = 1e18;

// full check of host-resident inputs (device inputs are checked by a kernel)
inline int check_host_data(const hac_instance &in, const hac_params &p)
{
    const int n = in.n;
    if (in.h_rowptr[0] != 0) return HAC_EINVAL;
    for (int i = 0; i < n; ++i) {
        int b = in.h_rowptr[i], e = in.h_rowptr[i + 1];
        if (e < b) return HAC_EINVAL;
        for (int q = b; q < e; ++q) {
            int j = in.h_col[q];
            if (j < 0 || j >= n || j == i) return HAC_EINVAL;
            if (q > b && in.h_col[q - 1] >= j) return HAC_EINVAL;
            double v;
            if (in.h_dtype == 1) {
                uint16_t hb = ((const uint16_t *)in.h_val)[q];
                int ex = (hb >> 10) & 31;
                if (ex == 31) return HAC_EINVAL;
                v = (hb >> 15) ? -1.0 : std::ldexp((double)(ex ? ((hb & 1023) | 1024) : (hb & 1023)),
                                                   ex ? ex - 25 : -24);
            } else {
                v = ((const float *)in.h_val)[q];
            }
            if (!(v >= 0.0 && v <= 1.0)) return HAC_EINVAL;
        }
    }
    if (in.kind == 0) {
        for (long long q = 0; q < 2LL * n; ++q) if (!finite_f(in.coords[q])) return HAC_EINVAL;
        if (p.local_search)
            for (long long q = 0; q < 2LL * n; ++q)
                if (!(std::fabs((double)in.coords[q]) <= LS_COORD_MAX)) return HAC_EINVAL;
    } else {
        for (long long q = 0; q < (long long)n * n; ++q) if (!finite_f(in.cost[q])) return HAC_EINVAL;
    }
    return HAC_OK;
}

// check_host_data of every instance of a batch: on up to 16 host threads
// when the batch holds more than a million heatmap entries and cost-matrix
// or coordinate values; the status of the first failing instance in batch
// order (the same as the serial loop)
inline int check_host_all(const hac_instance *ins, const hac_params *ps, int count)
{
    size_t work = 0;
    for (int b = 0; b < count; ++b)
        work += (size_t)ins[b].h_nnz + (ins[b].kind == 1 ? (size_t)ins[b].n * ins[b].n : 2 * (size_t)ins[b].n);
    const int hw = (int)std::thread::hardware_concurrency();
    const int nt = std::min(std::min(hw > 0 ? hw : 1, 16), count);
    std::vector<int> res(count, HAC_OK);
    std::atomic<int> next{0};
    auto worker = [&] {
        for (int b; (b = next.fetch_add(1)) < count;) res[b] = check_host_data(ins[b], ps[b]);
    };
    std::vector<std::thread> th;
    if (work > (1u << 20))
        try {
            for (int t = 1; t < nt; ++t) th.emplace_back(worker);
        } catch (...) {   // no threads available: the calling thread does the rest
        }
    worker();
    for (std::thread &x : th) x.join();
    for (int b = 0; b < count; ++b)
        if (res[b] != HAC_OK) return res[b];
    return HAC_OK;
}

inline int instance_sizes(const hac_instance &in, const hac_params &p, int on_dev, Sizes &z)
{
    int st = check_params(in, p);
    if (st) return st;
    z.n = in.n;
    z.kind = in.kind;
    z.kp = 4 * ((p.k + 3) / 4);
    z.k_eff = std::min(p.k, in.n - 1);
    z.m = p.m;
    z.iters = p.iterations;
    z.ls = p.local_search;
    z.ls_k = p.local_search ? p.ls_k : 0;
    z.sym = in.symmetrize;
    z.half = in.h_dtype;
    const long long last = in.h_nnz;
    if (last < 0 || last > (1LL << 31) - 1) return HAC_EINVAL;
    if (!on_dev && in.h_rowptr[in.n] != last) return HAC_EINVAL;
    if (last > 0 && (!in.h_col || !in.h_val)) return HAC_EINVAL;
    z.nnz = last;
    return HAC_OK;
}

// Replays the same sequence of slices for sizing and for binding pointers.
template <typename F>
void layout_instance(Arena &A, const Sizes &z, int on_dev, F &&put)
{
    const size_t n = z.n, S = n * z.kp, nnz = (size_t)z.nnz;
    const size_t cap = nnz + (z.sym ? nnz : 0);
    if (!on_dev) {
        if (z.kind == 0) put("xy", A.take(n * 8));
        else put("cost", A.take(n * n * 4));
        put("rowptr", A.take((n + 1) * 4));
        put("col", A.take(nnz * 4 + 4));
        put("val", A.take(nnz * (z.half ? 2 : 4) + 4));
    }
    if (z.sym) {
        put("tcol", A.take(nnz * 4 + 4));
        put("tval", A.take(nnz * 8 + 8));
    }
    put("mem_j", A.take(cap * 4 + 4));
    put("mem_h", A.take(cap * 8 + 8));
    put("mem_cnt", A.take(n * 4));
    put("cand", A.take(S * 4));
    put("cdist", A.take(S * 8));
    put("conf", A.take(S * 8));
    put("evid", A.take(S * 8));
    put("logev", A.take(S * 8));
    put("base", A.take(n * 8));
    put("W", A.take(S * 4));
    put("tau", A.take(S * 4));
    put("choice", A.take(S * 4));
    if (z.ls) {
        put("nbr", A.take(n * z.ls_k * 4));
        put("nbrd", A.take(n * z.ls_k * 8));
        put("nbrd32", A.take(n * z.ls_k * 4));
        put("ls_pos", A.take(n * 4));
        put("ls_el", A.take(n * 4));
        put("ls_dlb", A.take(n));
        if (z.ls == 2 || z.ls == 4) {   // every ant's local search: its own positions, scratch, bits
            put("lsa_pos", A.take((size_t)z.m * n * 4));
            put("lsa_el", A.take((size_t)z.m * n * 4));
            put("lsa_dlb", A.take((size_t)z.m * n));
        }
    }
    put("fbl", A.take(n * FBL_LEN * 4));
    put("fbl2", A.take(n * FBL2_LEN * 2));
    put("nn_tour", A.take(n * 4));
    put("gb_tour", A.take(n * 4));
    put("rb_tour", A.take(n * 4));
    put("ib_tour", A.take(n * 4));
    put("succ", A.take(n * 4));
    put("pred", A.take(n * 4));
    put("tours", A.take((size_t)z.m * n * 4));
    put("slots", A.take((size_t)z.m * n));
    put("dstep", A.take((size_t)z.m * n * 8));
    put("fbs", A.take((size_t)z.m * n * 4));
    put("fbcnt", A.take((size_t)z.m * 4));
    put("lens", A.take((size_t)z.m * 8));
    put("trace", A.take((size_t)TRACE_W * std::max(z.iters, 1) * 8));
}

// zero-initialised part: states, transpose counters, error word
template <typename F>
void layout_zero(Arena &A, const Sizes &z, F &&put)
{
    put("st", A.take(sizeof(InstState)));
    if (z.sym) {
        put("trowptr", A.take(((size_t)z.n + 1) * 4));
        put("tfill", A.take((size_t)z.n * 4));
    }
}

inline size_t map_sizes(const std::vector<Sizes> &zs, size_t &rows, size_t &slots, size_t &warps)
{
    rows = slots = warps = 0;
    for (const Sizes &z : zs) {
        rows += (z.n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK;
        slots += ((size_t)z.n * z.kp + SLOTS_PER_BLOCK - 1) / SLOTS_PER_BLOCK;
        warps += z.m;   // bound for one ant per warp
    }
    return rows;
}

struct Plan {
    std::vector<Sizes> zs;
    size_t zero_bytes = 0, total = 0;
};

inline int plan_batch(const hac_instance *ins, const hac_params *ps, int count, int on_dev, Plan &P)
{
    if (!ins || !ps || count < 1) return HAC_EINVAL;
    P.zs.resize(count);
    for (int b = 0; b < count; ++b) {
        int st = instance_sizes(ins[b], ps[b], on_dev, P.zs[b]);
        if (st) return st;
    }
    Arena A;
    A.take((size_t)count * sizeof(DevInst));
    size_t rows, slots, warps;
    map_sizes(P.zs, rows, slots, warps);
    A.take(rows * sizeof(int2));
    A.take(slots * sizeof(int2));
    A.take(slots * sizeof(int2));              // slot table relative to each part's first instance
    A.take(warps * sizeof(int4));
    A.take((size_t)count * sizeof(int32_t));   // fused-kernel cluster -> instance order
    size_t z0 = A.take(sizeof(int));       // error word starts the zero region
    for (const Sizes &z : P.zs) layout_zero(A, z, [](const char *, size_t) {});
    P.zero_bytes = A.off - z0;
    for (const Sizes &z : P.zs) layout_instance(A, z, on_dev, [](const char *, size_t) {});
    P.total = A.off + 256;
    return HAC_OK;
}


struct FusedGroup {
    int clog = 0, apw = 4, count = 0, order_off = 0;
    int rows_cap = 0, kp_cap = 0, stride = 0, warps = 0, xy_cap = 0, list_rows = 0;
};

// pointers of the zero-initialised part of one instance
inline void bind_zero(DevInst &D, const Sizes &z, Arena &A, char *B)
{
    layout_zero(A, z, [&](const char *name, size_t off) {
        if (!std::strcmp(name, "st")) D.st = (InstState *)(B + off);
        else if (!std::strcmp(name, "trowptr")) D.trowptr = (int32_t *)(B + off);
        else if (!std::strcmp(name, "tfill")) D.tfill = (int32_t *)(B + off);
    });
}

// sizes, parameters and workspace pointers of one instance
inline void bind_instance(DevInst &D, const hac_instance &in, const hac_params &p, const Sizes &z,
                          int inputs_on_device, const hac_exec &ex, Arena &A, char *B)
{
    D.n = z.n; D.kind = z.kind; D.k = p.k; D.k_eff = z.k_eff; D.k_pad = z.kp;
    D.m = p.m; D.iters = p.iterations; D.ls_k = z.ls_k;
    D.degree_target = p.degree_target; D.local_search = p.local_search;
    D.baseline_scope = p.baseline_scope; D.symmetrize = in.symmetrize; D.h_half = in.h_dtype;
    D.schedule = p.schedule;
    D.kappa_mode = p.kappa_mode;
    D.seed = p.seed;
    D.nnz = (int32_t)z.nnz;
    D.alpha = p.alpha; D.beta = p.beta; D.rho = p.rho; D.theta_h = p.theta_h; D.eps = p.eps;
    D.c_cap = p.c_cap; D.q_level = p.q_level; D.p_best = p.p_best; D.logw_clip = p.logw_clip;
    if (inputs_on_device) {
        D.xy = in.coords; D.cost = in.cost; D.rowptr = in.h_rowptr; D.col = in.h_col;
        D.val = in.h_val;
    }
    layout_instance(A, z, inputs_on_device, [&](const char *name, size_t off) {
        void *ptr = B + off;
#define SETP(f, T) if (!std::strcmp(name, #f)) D.f = (T)ptr;
        SETP(tcol, int32_t *) SETP(tval, double *) SETP(mem_j, int32_t *) SETP(mem_h, double *)
        SETP(mem_cnt, int32_t *) SETP(cand, int32_t *) SETP(cdist, double *) SETP(conf, double *)
        SETP(evid, double *) SETP(logev, double *) SETP(base, double *) SETP(W, float *)
        SETP(tau, float *) SETP(choice, float *) SETP(nbr, int32_t *) SETP(nbrd, double *)
        SETP(ls_pos, int32_t *) SETP(ls_dlb, uint8_t *) SETP(nn_tour, int32_t *)
        SETP(nbrd32, float *) SETP(ls_el, float *)
        SETP(lsa_pos, int32_t *) SETP(lsa_el, float *) SETP(lsa_dlb, uint8_t *)
        SETP(gb_tour, int32_t *) SETP(ib_tour, int32_t *) SETP(succ, int32_t *) SETP(rb_tour, int32_t *)
        SETP(pred, int32_t *) SETP(tours, int32_t *) SETP(lens, double *) SETP(trace, double *)
        SETP(fbl, int32_t *) SETP(fbl2, uint16_t *) SETP(slots, uint8_t *) SETP(dstep, double *) SETP(fbs, int32_t *)
        SETP(fbcnt, int32_t *)
#undef SETP
        if (!std::strcmp(name, "xy")) D.xy = (const float *)ptr;
        if (!std::strcmp(name, "cost")) D.cost = (const float *)ptr;
        if (!std::strcmp(name, "rowptr")) D.rowptr = (const int32_t *)ptr;
        if (!std::strcmp(name, "col")) D.col = (const int32_t *)ptr;
        if (!std::strcmp(name, "val")) D.val = ptr;
    });
    if (!ex.fallback_list) D.fbl = nullptr;
    if (!ex.fallback_list || z.n > 65535) D.fbl2 = nullptr;   // uint16 node ids
    if (ex.ants_per_warp == 32) { D.tour_sa = 1; D.tour_ss = p.m; }   // step-major tours
    else { D.tour_sa = z.n; D.tour_ss = 1; }
    D.fbl_len = ex.fallback_list;
}

// host -> device copies of one instance's inputs into its workspace slices
inline int upload_inputs(const DevInst &D, const hac_instance &in, const Sizes &z, cudaStream_t s)
{
    const size_t n = z.n, nnz = (size_t)z.nnz;
    if (z.kind == 0) CK(cudaMemcpyAsync((void *)D.xy, in.coords, n * 8, cudaMemcpyHostToDevice, s));
    else CK(cudaMemcpyAsync((void *)D.cost, in.cost, n * n * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync((void *)D.rowptr, in.h_rowptr, (n + 1) * 4, cudaMemcpyHostToDevice, s));
    if (nnz) {
        CK(cudaMemcpyAsync((void *)D.col, in.h_col, nnz * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync((void *)D.val, in.h_val, nnz * (z.half ? 2 : 4), cudaMemcpyHostToDevice, s));
    }
    return HAC_OK;
}

// Groups the given instances by layout: ants per warp and cluster size (the
// fewest CTAs whose shared memory holds the instance's share of the
// candidate table and visited masks, at least 2^clog_min), each group ordered
// by decreasing work.  apw = 0 chooses per instance ("mixed"): 4 ants per warp
// on one CTA where the instance fits one with its coordinates and lookup
// lists (many ants per SM), else 2 ants per warp on the smallest cluster that
// holds it (fewer ants per SM, a shorter step for the large instances that
// bound the batch).  `order` lists
// instance indices group after group.
inline int plan_groups(const std::vector<Sizes> &zs, const std::vector<int> &members, int apw,
                       int clog_min, int fallback_list, std::vector<FusedGroup> &groups,
                       std::vector<int32_t> &order)
{
    const int count = (int)members.size();
    std::vector<int> clog(count, -1), qapw(count, apw);
    auto fits = [&](int q, int cl, int a, int &rows, int &warps) {
        const Sizes &z = zs[members[q]];
        const int C = 1 << cl;
        rows = (z.n + C - 1) / C;
        const int apc = (z.m + C - 1) / C;
        warps = (apc + a - 1) / a;
        if (warps > 16) return false;   // k_fused is compiled for at most 512 threads
        return fused_smem_bytes(rows, z.kp, warps, a, (z.n + 32) / 32, 0, 0) <= FUSED_SMEM_LIMIT;
    };
    for (int q = 0; q < count; ++q) {
        if (zs[members[q]].n > 65534) return HAC_EUNSUPPORTED;
        int rows, warps;
        if (apw == 0) {
            // one CTA (one SM) whenever the table, the visited masks and the
            // coordinates of the fallback scan fit; the lookup lists then stay
            // in global memory unless the group's CTAs have room for them.
            // One SM per instance instead of a cluster of two frees SMs for
            // the rest of the batch, whose makespan is otherwise bound by the
            // SM time of the clusters rather than by its longest instance.
            const Sizes &z = zs[members[q]];
            if (clog_min == 0 && fits(q, 0, 4, rows, warps) &&
                fused_smem_bytes(rows, z.kp, warps, 4, (z.n + 32) / 32, z.n, 0) <= FUSED_SMEM_LIMIT) {
                clog[q] = 0;
                qapw[q] = 4;
                continue;
            }
            qapw[q] = 2;
        }
        for (int cl = clog_min; cl <= 3; ++cl)
            if (fits(q, cl, qapw[q], rows, warps)) { clog[q] = cl; break; }
        if (clog[q] < 0) return HAC_EUNSUPPORTED;
    }
    const int apws[4] = {2, 4, 16, 32};
    for (;;) {   // group caps may exceed the limit when members differ: move a group up
        groups.clear();
        bool again = false;
        for (int cl = 0; cl <= 3 && !again; ++cl)
            for (int ai = 0; ai < 4 && !again; ++ai) {
                const int a = apws[ai];
                FusedGroup G;
                G.clog = cl;
                G.apw = a;
                for (int q = 0; q < count; ++q) {
                    if (clog[q] != cl || qapw[q] != a) continue;
                    int rows, warps;
                    fits(q, cl, a, rows, warps);
                    const Sizes &z = zs[members[q]];
                    G.count++;
                    G.rows_cap = std::max(G.rows_cap, rows);
                    G.kp_cap = std::max(G.kp_cap, z.kp);
                    G.stride = std::max(G.stride, (z.n + 32) / 32);   // bits 0..n (n: padding)
                    G.warps = std::max(G.warps, warps);
                }
                if (!G.count) continue;
                const size_t base = fused_smem_bytes(G.rows_cap, G.kp_cap, G.warps, a, G.stride, 0, 0);
                if (base > FUSED_SMEM_LIMIT) {
                    if (cl == 3) return HAC_EUNSUPPORTED;
                    for (int q = 0; q < count; ++q) if (clog[q] == cl && qapw[q] == a) clog[q] = cl + 1;
                    again = true;
                    break;
                }
                // coordinates of the fallback scan in shared memory when they still fit
                int nmax = 0;
                for (int q = 0; q < count; ++q)
                    if (clog[q] == cl && qapw[q] == a) nmax = std::max(nmax, zs[members[q]].n);
                if (base + (size_t)nmax * 8 <= FUSED_SMEM_LIMIT) G.xy_cap = nmax;
                // and the lookup lists of this CTA's rows
                if (fallback_list &&
                    fused_smem_bytes(G.rows_cap, G.kp_cap, G.warps, a, G.stride, G.xy_cap, G.rows_cap) <=
                        FUSED_SMEM_LIMIT)
                    G.list_rows = G.rows_cap;
                groups.push_back(G);
            }
        if (!again) break;
    }
    // groups in order of their largest instance's work: the group launched
    // first gets SMs first, and the largest instances bound the batch
    auto work = [&](int i) { const Sizes &z = zs[i]; return (long long)z.m * z.n * z.iters; };
    std::vector<long long> gmax(groups.size(), 0);
    for (size_t g = 0; g < groups.size(); ++g)
        for (int q = 0; q < count; ++q)
            if (clog[q] == groups[g].clog && qapw[q] == groups[g].apw) gmax[g] = std::max(gmax[g], work(members[q]));
    std::vector<size_t> gi(groups.size());
    for (size_t g = 0; g < gi.size(); ++g) gi[g] = g;
    std::stable_sort(gi.begin(), gi.end(), [&](size_t x, size_t y) { return gmax[x] > gmax[y]; });
    std::vector<FusedGroup> sorted;
    for (size_t g : gi) sorted.push_back(groups[g]);
    groups.swap(sorted);
    order.clear();
    for (FusedGroup &G : groups) {
        G.order_off = (int)order.size();
        std::vector<int32_t> mem;
        for (int q = 0; q < count; ++q) if (clog[q] == G.clog && qapw[q] == G.apw) mem.push_back(members[q]);
        std::stable_sort(mem.begin(), mem.end(), [&](int x, int y) { return work(x) > work(y); });
        order.insert(order.end(), mem.begin(), mem.end());
    }
    return HAC_OK;
}

// Launches the groups on `s`: group 0 (the batch's longest instances) first,
// then each further group as a programmatic dependent of the one before it,
// so that it starts once every CTA of its predecessor is resident rather than
// when it ends.  Group 0's clusters thus take their SMs before any CTA of a
// later group can: when the groups' CTAs outnumber the SMs and the launches
// race (concurrent streams, or a graph's parallel branches), single CTAs may
// fragment the GPCs so that a 2-CTA cluster of a longest instance finds no
// free pair of SMs and waits for a small instance to end.  The later groups'
// surplus CTAs wait in the hardware queue for the SMs that free first.
// d_iters (parallel to d_order, may be null) holds per-instance iteration
// counts.
inline cudaError_t launch_groups(const DevInst *d_inst, const int32_t *d_order, const int32_t *d_iters,
                                 const std::vector<FusedGroup> &groups, int iters, cudaStream_t s)
{
    cudaError_t err = cudaSuccess;
    for (size_t g = 0; g < groups.size(); ++g) {
        const FusedGroup &G = groups[g];
        cudaError_t e = launch_fused(d_inst, d_order + G.order_off, d_iters ? d_iters + G.order_off : nullptr,
                                     G.count, G.clog, G.apw, G.warps,
                                     G.rows_cap, G.kp_cap, G.stride, G.xy_cap, G.list_rows, iters, s, g > 0);
        if (e != cudaSuccess && err == cudaSuccess) err = e;
    }
    return err;
}

}  // namespace host
}  // namespace hac
