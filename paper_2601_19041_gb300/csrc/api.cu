// Host orchestration behind the C ABI of heataco.h: workspace layout, input
// upload and validation, work tables, the iteration loop (optionally captured
// in a CUDA graph) and read-back.  No device memory is allocated here: every
// device array is a slice of the caller's workspace.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "hac_internal.cuh"

using namespace hac;

namespace {

thread_local int g_last_cuda = 0;

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
constexpr int FBL_LEN = 32;            // nearest-unvisited lookup list (ant.cuh FBL)

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

bool finite_f(float x) { return std::isfinite(x); }

int check_params(const hac_instance &in, const hac_params &p)
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
    if (p.local_search != 0 && p.local_search != 1) return HAC_EINVAL;
    if (p.local_search) {
        if (in.kind != 0) return HAC_EUNSUPPORTED;
        if (p.ls_k < 1 || p.ls_k > 32 || p.ls_k > in.n - 1) return HAC_EINVAL;
    }
    if (in.symmetrize != 0 && in.symmetrize != 1) return HAC_EINVAL;
    return HAC_OK;
}

// full check of host-resident inputs (device inputs are checked by a kernel)
int check_host_data(const hac_instance &in)
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
    } else {
        for (long long q = 0; q < (long long)n * n; ++q) if (!finite_f(in.cost[q])) return HAC_EINVAL;
    }
    return HAC_OK;
}

int instance_sizes(const hac_instance &in, const hac_params &p, int on_dev, Sizes &z)
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
        put("ls_pos", A.take(n * 4));
        put("ls_dlb", A.take(n));
    }
    put("fbl", A.take(n * FBL_LEN * 4));
    put("nn_tour", A.take(n * 4));
    put("gb_tour", A.take(n * 4));
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

size_t map_sizes(const std::vector<Sizes> &zs, size_t &rows, size_t &slots, size_t &warps)
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

int plan_batch(const hac_instance *ins, const hac_params *ps, int count, int on_dev, Plan &P)
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
    A.take(warps * sizeof(int4));
    A.take((size_t)count * sizeof(int32_t));   // fused-kernel cluster -> instance order
    size_t z0 = A.take(sizeof(int));       // error word starts the zero region
    for (const Sizes &z : P.zs) layout_zero(A, z, [](const char *, size_t) {});
    P.zero_bytes = A.off - z0;
    for (const Sizes &z : P.zs) layout_instance(A, z, on_dev, [](const char *, size_t) {});
    P.total = A.off + 256;
    return HAC_OK;
}

}  // namespace

struct FusedGroup {
    int clog = 0, count = 0, order_off = 0;
    int rows_cap = 0, kp_cap = 0, stride = 0, warps = 0, xy_cap = 0, list_rows = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

struct hac_batch {
    int count = 0;
    cudaStream_t stream = nullptr;
    hac_exec ex{};
    std::vector<Sizes> zs;
    std::vector<DevInst> hi;
    DevInst *d_inst = nullptr;
    int2 *d_rowmap = nullptr;
    int rowmap_len = 0;
    int2 *d_slotmap = nullptr;
    int slotmap_len = 0;
    int4 *d_warpmap = nullptr;
    int warpmap_len = 0;
    int32_t *d_order = nullptr;
    std::vector<FusedGroup> groups;   // non-empty when the fused kernel is used
    int *d_err = nullptr;
    int max_n = 0, max_kp = 0;
    bool any_ls = false;
    std::vector<int> t_host;
    cudaGraphExec_t gexec = nullptr;
    int graph_kernels = 0;          // kernels inside one graph replay
    long long launches = 0;         // kernels issued so far
    // profiling: event pairs per kernel group, folded into totals on read
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<int> ev_group;      // group of each recorded pair
    double group_ms[4] = {0, 0, 0, 0};
    long long group_launches[4] = {0, 0, 0, 0};
};

namespace {

// records an event pair around the kernels `body` launches (profile mode)
template <typename Body>
int timed(hac_batch *bt, int group, Body &&body)
{
    if (!bt->ex.profile) return body();
    while (bt->ev_pool.size() < bt->ev_used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return body();
        bt->ev_pool.push_back(e);
    }
    cudaEvent_t a = bt->ev_pool[bt->ev_used], b = bt->ev_pool[bt->ev_used + 1];
    cudaEventRecord(a, bt->stream);
    int k = body();
    cudaEventRecord(b, bt->stream);
    bt->ev_used += 2;
    bt->ev_group.push_back(group);
    bt->group_launches[group] += k;
    return k;
}

int fold_events(hac_batch *bt)
{
    if (!bt->ev_used) return HAC_OK;
    CK(cudaStreamSynchronize(bt->stream));
    for (size_t q = 0; q < bt->ev_group.size(); ++q) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, bt->ev_pool[2 * q], bt->ev_pool[2 * q + 1]));
        bt->group_ms[bt->ev_group[q]] += ms;
    }
    bt->ev_used = 0;
    bt->ev_group.clear();
    return HAC_OK;
}

}  // namespace

// Groups the instances by cluster size (the fewest CTAs whose shared memory
// holds the instance's share of the candidate table and visited masks, at
// least 2^cluster_log2), each group ordered by decreasing work.
static int plan_fused(hac_batch *bt, std::vector<int32_t> &order)
{
    const int apw = bt->ex.ants_per_warp == 2 ? 2 : bt->ex.ants_per_warp == 32 ? 32 : 4;
    if (apw != bt->ex.ants_per_warp) return HAC_EUNSUPPORTED;   // the fused kernel has no 1-ant-per-warp form
    const int count = bt->count;
    std::vector<int> clog(count, -1);
    auto fits = [&](int b, int cl, int &rows, int &warps) {
        const Sizes &z = bt->zs[b];
        const int C = 1 << cl;
        rows = (z.n + C - 1) / C;
        const int apc = (z.m + C - 1) / C;
        warps = (apc + apw - 1) / apw;
        if (warps > 16) return false;   // k_fused is compiled for at most 512 threads
        return fused_smem_bytes(rows, z.kp, warps, apw, (z.n + 31) / 32, 0, 0) <= FUSED_SMEM_LIMIT;
    };
    for (int b = 0; b < count; ++b) {
        if (bt->zs[b].n > 65534) return HAC_EUNSUPPORTED;
        int rows, warps;
        for (int cl = bt->ex.cluster_log2; cl <= 3; ++cl)
            if (fits(b, cl, rows, warps)) { clog[b] = cl; break; }
        if (clog[b] < 0) return HAC_EUNSUPPORTED;
    }
    for (;;) {   // group caps may exceed the limit when members differ: move a group up
        bt->groups.clear();
        bool again = false;
        for (int cl = 0; cl <= 3 && !again; ++cl) {
            FusedGroup G;
            G.clog = cl;
            for (int b = 0; b < count; ++b) {
                if (clog[b] != cl) continue;
                int rows, warps;
                fits(b, cl, rows, warps);
                G.count++;
                G.rows_cap = std::max(G.rows_cap, rows);
                G.kp_cap = std::max(G.kp_cap, bt->zs[b].kp);
                G.stride = std::max(G.stride, (bt->zs[b].n + 31) / 32);
                G.warps = std::max(G.warps, warps);
            }
            if (!G.count) continue;
            const size_t base = fused_smem_bytes(G.rows_cap, G.kp_cap, G.warps, apw, G.stride, 0, 0);
            if (base > FUSED_SMEM_LIMIT) {
                if (cl == 3) return HAC_EUNSUPPORTED;
                for (int b = 0; b < count; ++b) if (clog[b] == cl) clog[b] = cl + 1;
                again = true;
                break;
            }
            // coordinates of the fallback scan in shared memory when they still fit
            int nmax = 0;
            for (int b = 0; b < count; ++b) if (clog[b] == cl) nmax = std::max(nmax, bt->zs[b].n);
            if (base + (size_t)nmax * 8 <= FUSED_SMEM_LIMIT) G.xy_cap = nmax;
            // and the lookup lists of this CTA's rows (lane kernel only)
            if (bt->ex.fallback_list &&
                fused_smem_bytes(G.rows_cap, G.kp_cap, G.warps, apw, G.stride, G.xy_cap, G.rows_cap) <=
                    FUSED_SMEM_LIMIT)
                G.list_rows = G.rows_cap;
            bt->groups.push_back(G);
        }
        if (!again) break;
    }
    order.clear();
    for (FusedGroup &G : bt->groups) {
        G.order_off = (int)order.size();
        std::vector<int32_t> mem;
        for (int b = 0; b < count; ++b) if (clog[b] == G.clog) mem.push_back(b);
        std::stable_sort(mem.begin(), mem.end(), [&](int x, int y) {
            const Sizes &a = bt->zs[x], &c = bt->zs[y];
            return (long long)a.m * a.n * a.iters > (long long)c.m * c.n * c.iters;
        });
        order.insert(order.end(), mem.begin(), mem.end());
    }
    return HAC_OK;
}

extern "C" {

int hac_version(void) { return 1; }

int hac_last_cuda_error(void) { return g_last_cuda; }

const char *hac_strerror(int status)
{
    switch (status) {
    case HAC_OK: return "ok";
    case HAC_EINVAL: return "invalid argument or malformed instance";
    case HAC_ENOMEM: return "workspace too small or host allocation failed";
    case HAC_ECUDA: return "CUDA runtime error";
    case HAC_ETIMEOUT: return "device-side wait timed out";
    case HAC_EUNSUPPORTED: return "unsupported combination";
    case HAC_EBUSY: return "busy";
    default: return "unknown status";
    }
}

int hac_params_default(hac_params *p, int32_t kind)
{
    if (!p || (kind != 0 && kind != 1)) return HAC_EINVAL;
    std::memset(p, 0, sizeof *p);
    p->m = 32; p->k = 20; p->iterations = 5000;
    p->alpha = 1.0; p->beta = 2.0; p->rho = kind == 1 ? 0.2 : 0.8;
    p->theta_h = 1e-4; p->eps = 1e-9; p->c_cap = 0.5; p->q_level = 0.90;
    p->p_best = 0.05; p->logw_clip = 30.0;
    p->degree_target = kind == 1 ? 1 : 2;
    p->local_search = 0; p->baseline_scope = 0; p->ls_k = 20; p->seed = 0;
    return HAC_OK;
}

int hac_exec_default(hac_exec *e)
{
    if (!e) return HAC_EINVAL;
    e->ants_per_warp = 0;
    e->warps_per_block = 0;
    e->use_graph = 1;
    e->fused = 0;
    e->fallback_list = 0;
    e->profile = 0;
    e->cluster_log2 = 0;
    return HAC_OK;
}

int hac_batch_workspace_size(const hac_instance *ins, const hac_params *ps, int32_t count,
                             int32_t inputs_on_device, size_t *bytes)
{
    if (!bytes) return HAC_EINVAL;
    Plan P;
    int st = plan_batch(ins, ps, count, inputs_on_device, P);
    if (st) return st;
    *bytes = P.total;
    return HAC_OK;
}

int hac_batch_create(const hac_instance *ins, const hac_params *ps, int32_t count,
                     int32_t inputs_on_device, void *workspace, size_t ws_bytes,
                     const hac_exec *exec, void *stream, hac_batch **out)
{
    if (!out) return HAC_EINVAL;
    *out = nullptr;
    Plan P;
    int st = plan_batch(ins, ps, count, inputs_on_device, P);
    if (st) return st;
    if (!workspace || ws_bytes < P.total) return HAC_ENOMEM;
    if (!inputs_on_device)
        for (int b = 0; b < count; ++b)
            if ((st = check_host_data(ins[b]))) return st;
    hac_exec ex;
    hac_exec_default(&ex);
    if (exec) ex = *exec;
    if (ex.ants_per_warp == 0) ex.ants_per_warp = 4;
    if (ex.ants_per_warp != 1 && ex.ants_per_warp != 2 && ex.ants_per_warp != 4 && ex.ants_per_warp != 32)
        return HAC_EINVAL;
    if (ex.warps_per_block == 0) ex.warps_per_block = 4;
    if (ex.warps_per_block < 1 || ex.warps_per_block > 8) return HAC_EINVAL;
    if (ex.fallback_list != 0 && ex.fallback_list != FBL_LEN) return HAC_EINVAL;
    if (ex.cluster_log2 < 0 || ex.cluster_log2 > 3) return HAC_EINVAL;

    hac_batch *bt = new (std::nothrow) hac_batch;
    if (!bt) return HAC_ENOMEM;
    bt->count = count;
    bt->stream = (cudaStream_t)stream;
    bt->ex = ex;
    bt->zs = P.zs;
    bt->hi.resize(count);
    bt->t_host.assign(count, 0);
    cudaStream_t s = bt->stream;

    // align the base, then replay the plan with real addresses
    uintptr_t base = ((uintptr_t)workspace + 255) & ~(uintptr_t)255;
    char *B = (char *)base;
    Arena A;
    bt->d_inst = (DevInst *)(B + A.take((size_t)count * sizeof(DevInst)));
    size_t rows, slots, warps;
    map_sizes(P.zs, rows, slots, warps);
    bt->d_rowmap = (int2 *)(B + A.take(rows * sizeof(int2)));
    bt->d_slotmap = (int2 *)(B + A.take(slots * sizeof(int2)));
    bt->d_warpmap = (int4 *)(B + A.take(warps * sizeof(int4)));
    bt->d_order = (int32_t *)(B + A.take((size_t)count * sizeof(int32_t)));
    size_t z0 = A.take(sizeof(int));
    bt->d_err = (int *)(B + z0);
    for (int b = 0; b < count; ++b) {
        DevInst &D = bt->hi[b];
        std::memset(&D, 0, sizeof D);
        layout_zero(A, P.zs[b], [&](const char *name, size_t off) {
            if (!std::strcmp(name, "st")) D.st = (InstState *)(B + off);
            else if (!std::strcmp(name, "trowptr")) D.trowptr = (int32_t *)(B + off);
            else if (!std::strcmp(name, "tfill")) D.tfill = (int32_t *)(B + off);
        });
    }
    const size_t zero_end = A.off;
    CK(cudaMemsetAsync(B + z0, 0, zero_end - z0, s));

    for (int b = 0; b < count; ++b) {
        const hac_instance &in = ins[b];
        const hac_params &p = ps[b];
        const Sizes &z = P.zs[b];
        DevInst &D = bt->hi[b];
        D.n = z.n; D.kind = z.kind; D.k = p.k; D.k_eff = z.k_eff; D.k_pad = z.kp;
        D.m = p.m; D.iters = p.iterations; D.ls_k = z.ls_k;
        D.degree_target = p.degree_target; D.local_search = p.local_search;
        D.baseline_scope = p.baseline_scope; D.symmetrize = in.symmetrize; D.h_half = in.h_dtype;
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
            SETP(gb_tour, int32_t *) SETP(ib_tour, int32_t *) SETP(succ, int32_t *)
            SETP(pred, int32_t *) SETP(tours, int32_t *) SETP(lens, double *) SETP(trace, double *)
            SETP(fbl, int32_t *) SETP(slots, uint8_t *) SETP(dstep, double *) SETP(fbs, int32_t *)
            SETP(fbcnt, int32_t *)
#undef SETP
            if (!std::strcmp(name, "xy")) D.xy = (const float *)ptr;
            if (!std::strcmp(name, "cost")) D.cost = (const float *)ptr;
            if (!std::strcmp(name, "rowptr")) D.rowptr = (const int32_t *)ptr;
            if (!std::strcmp(name, "col")) D.col = (const int32_t *)ptr;
            if (!std::strcmp(name, "val")) D.val = ptr;
        });
        if (!ex.fallback_list) D.fbl = nullptr;
        if (ex.ants_per_warp == 32) { D.tour_sa = 1; D.tour_ss = p.m; }   // step-major tours
        else { D.tour_sa = z.n; D.tour_ss = 1; }
        D.fbl_len = ex.fallback_list;
        if (!inputs_on_device) {
            const size_t n = z.n, nnz = (size_t)z.nnz;
            if (z.kind == 0) CK(cudaMemcpyAsync((void *)D.xy, in.coords, n * 8, cudaMemcpyHostToDevice, s));
            else CK(cudaMemcpyAsync((void *)D.cost, in.cost, n * n * 4, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync((void *)D.rowptr, in.h_rowptr, (n + 1) * 4, cudaMemcpyHostToDevice, s));
            if (nnz) {
                CK(cudaMemcpyAsync((void *)D.col, in.h_col, nnz * 4, cudaMemcpyHostToDevice, s));
                CK(cudaMemcpyAsync((void *)D.val, in.h_val, nnz * (z.half ? 2 : 4),
                                   cudaMemcpyHostToDevice, s));
            }
        }
        bt->max_n = std::max(bt->max_n, z.n);
        bt->max_kp = std::max(bt->max_kp, z.kp);
        bt->any_ls |= z.ls != 0;
    }
    // work tables
    std::vector<int2> rowmap, slotmap;
    std::vector<int4> warpmap;
    const int apw = bt->ex.ants_per_warp;
    for (int b = 0; b < count; ++b) {
        const Sizes &z = P.zs[b];
        for (int r = 0; r < z.n; r += ROWS_PER_BLOCK) rowmap.push_back(make_int2(b, r));
        const size_t S = (size_t)z.n * z.kp;
        for (size_t q = 0; q < S; q += SLOTS_PER_BLOCK) slotmap.push_back(make_int2(b, (int)q));
        for (int a = 0; a < z.m; a += apw) warpmap.push_back(make_int4(b, a, 0, 0));
    }
    bt->rowmap_len = (int)rowmap.size();
    bt->slotmap_len = (int)slotmap.size();
    bt->warpmap_len = (int)warpmap.size();
    CK(cudaMemcpyAsync(bt->d_rowmap, rowmap.data(), rowmap.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(bt->d_slotmap, slotmap.data(), slotmap.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(bt->d_warpmap, warpmap.data(), warpmap.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(bt->d_inst, bt->hi.data(), (size_t)count * sizeof(DevInst), cudaMemcpyHostToDevice, s));
    if (bt->ex.fused) {
        std::vector<int32_t> order;
        if (plan_fused(bt, order) == HAC_OK) {
            CK(cudaMemcpyAsync(bt->d_order, order.data(), order.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, s));
            for (size_t g = 1; g < bt->groups.size(); ++g) {
                FusedGroup &G = bt->groups[g];
                CK(cudaStreamCreateWithFlags(&G.side, cudaStreamNonBlocking));
                CK(cudaEventCreateWithFlags(&G.fork, cudaEventDisableTiming));
                CK(cudaEventCreateWithFlags(&G.join, cudaEventDisableTiming));
            }
        } else {
            bt->ex.fused = 0;   // some instance does not fit the fused kernel: per-iteration path
            bt->groups.clear();
        }
    }

    bt->launches += timed(bt, 2, [&] {
        return launch_prep(bt->d_inst, bt->hi.data(), count, bt->d_rowmap, bt->rowmap_len,
                           bt->d_slotmap, bt->slotmap_len, bt->d_err, s);
    });
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        delete bt;
        return HAC_ECUDA;
    }
    *out = bt;
    return HAC_OK;
}

static int remaining(const hac_batch *bt)
{
    int rem = 0;
    for (int b = 0; b < bt->count; ++b) rem = std::max(rem, bt->zs[b].iters - bt->t_host[b]);
    return rem;
}

static int enqueue_iteration(hac_batch *bt)
{
    int k = timed(bt, 0, [&] {
        return launch_construct(bt->d_inst, bt->d_warpmap, bt->warpmap_len, bt->ex.ants_per_warp,
                                bt->ex.warps_per_block, bt->max_n, bt->max_kp, bt->count, bt->stream);
    });
    k += timed(bt, 1, [&] {
        return launch_iteration_tail(bt->d_inst, bt->count, bt->d_slotmap, bt->slotmap_len,
                                     bt->any_ls, bt->stream);
    });
    return k;
}

// the fused groups run concurrently: group 0 on the batch stream, the others on
// side streams forked from and joined back into it
static int enqueue_fused(hac_batch *bt, int iters)
{
    cudaError_t err = cudaSuccess;
    const int k = timed(bt, 3, [&] {
        cudaStream_t s = bt->stream;
        for (size_t g = 1; g < bt->groups.size(); ++g) {
            cudaEventRecord(bt->groups[g].fork, s);
            cudaStreamWaitEvent(bt->groups[g].side, bt->groups[g].fork, 0);
        }
        for (size_t g = 0; g < bt->groups.size(); ++g) {
            const FusedGroup &G = bt->groups[g];
            cudaError_t e = launch_fused(bt->d_inst, bt->d_order + G.order_off, G.count, G.clog,
                                         bt->ex.ants_per_warp, G.warps, G.rows_cap, G.kp_cap,
                                         G.stride, G.xy_cap, G.list_rows, iters, g ? G.side : s);
            if (e != cudaSuccess && err == cudaSuccess) err = e;
        }
        for (size_t g = 1; g < bt->groups.size(); ++g) {
            cudaEventRecord(bt->groups[g].join, bt->groups[g].side);
            cudaStreamWaitEvent(s, bt->groups[g].join, 0);
        }
        return (int)bt->groups.size();
    });
    if (err != cudaSuccess) { g_last_cuda = (int)err; return HAC_ECUDA; }
    bt->launches += k;
    return HAC_OK;
}

int hac_batch_iterate(hac_batch *bt, int32_t iters)
{
    if (!bt || iters < 0) return HAC_EINVAL;
    int todo = std::min(iters, remaining(bt));
    const int done = todo;
    cudaStream_t s = bt->stream;
    if (bt->ex.fused && !bt->groups.empty()) {
        if (todo > 0) {
            int st = enqueue_fused(bt, todo);
            if (st) return st;
        }
        CK(cudaGetLastError());
        for (int b = 0; b < bt->count; ++b) bt->t_host[b] = std::min(bt->zs[b].iters, bt->t_host[b] + done);
        return HAC_OK;
    }
    if (bt->ex.use_graph && !bt->ex.profile && s != nullptr && todo >= GRAPH_CHUNK) {
        if (!bt->gexec) {
            cudaGraph_t g;
            CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            bt->graph_kernels = 0;
            for (int q = 0; q < GRAPH_CHUNK; ++q) bt->graph_kernels += enqueue_iteration(bt);
            cudaError_t e1 = cudaGetLastError();
            cudaError_t e2 = cudaStreamEndCapture(s, &g);
            if (e1 != cudaSuccess) { g_last_cuda = (int)e1; return HAC_ECUDA; }
            CK(e2);
            cudaError_t e3 = cudaGraphInstantiate(&bt->gexec, g, 0);
            cudaGraphDestroy(g);
            CK(e3);
        }
        while (todo >= GRAPH_CHUNK) {
            CK(cudaGraphLaunch(bt->gexec, s));
            bt->launches += bt->graph_kernels;
            todo -= GRAPH_CHUNK;
        }
    }
    for (; todo > 0; --todo) bt->launches += enqueue_iteration(bt);
    CK(cudaGetLastError());
    for (int b = 0; b < bt->count; ++b) bt->t_host[b] = std::min(bt->zs[b].iters, bt->t_host[b] + done);
    return HAC_OK;
}

int hac_batch_run(hac_batch *bt)
{
    if (!bt) return HAC_EINVAL;
    return hac_batch_iterate(bt, remaining(bt));
}

int hac_batch_sync(hac_batch *bt)
{
    if (!bt) return HAC_EINVAL;
    CK(cudaStreamSynchronize(bt->stream));
    int err = 0;
    CK(cudaMemcpy(&err, bt->d_err, sizeof err, cudaMemcpyDeviceToHost));
    return err;
}

int hac_batch_read(hac_batch *bt, int32_t b, int32_t field, void *host_dst, size_t bytes)
{
    if (!bt || b < 0 || b >= bt->count || !host_dst) return HAC_EINVAL;
    int st = hac_batch_sync(bt);
    if (st) return st;
    const DevInst &D = bt->hi[b];
    const size_t n = D.n, S = n * D.k_pad, m = D.m;
    const void *src = nullptr;
    size_t sz = 0;
    switch (field) {
    case HAC_F_CAND: src = D.cand; sz = S * 4; break;
    case HAC_F_CDIST: src = D.cdist; sz = S * 8; break;
    case HAC_F_CONF: src = D.conf; sz = S * 8; break;
    case HAC_F_BASE: src = D.base; sz = n * 8; break;
    case HAC_F_EVID: src = D.evid; sz = S * 8; break;
    case HAC_F_W: src = D.W; sz = S * 4; break;
    case HAC_F_TAU: src = D.tau; sz = S * 4; break;
    case HAC_F_CHOICE: src = D.choice; sz = S * 4; break;
    case HAC_F_NN_TOUR: src = D.nn_tour; sz = n * 4; break;
    case HAC_F_GB_TOUR: src = D.gb_tour; sz = n * 4; break;
    case HAC_F_IB_TOUR: src = D.ib_tour; sz = n * 4; break;
    case HAC_F_TOURS:
        if (D.tour_ss != 1) {   // step-major on the device: transpose into ant-major
            if (bytes < m * n * 4) return HAC_EINVAL;
            std::vector<int32_t> tmp(m * n);
            CK(cudaMemcpy(tmp.data(), D.tours, m * n * 4, cudaMemcpyDeviceToHost));
            int32_t *o = (int32_t *)host_dst;
            for (size_t a = 0; a < m; ++a)
                for (size_t q = 0; q < n; ++q) o[a * n + q] = tmp[q * m + a];
            return HAC_OK;
        }
        src = D.tours; sz = m * n * 4; break;
    case HAC_F_LENS: src = D.lens; sz = m * 8; break;
    case HAC_F_NBR:
        if (!D.ls_k) return HAC_EINVAL;
        src = D.nbr; sz = n * D.ls_k * 4; break;
    case HAC_F_TRACE: src = D.trace; sz = (size_t)TRACE_W * std::max(D.iters, 1) * 8; break;
    case HAC_F_SCALARS: {
        if (bytes < 16 * sizeof(double)) return HAC_EINVAL;
        InstState S0;
        CK(cudaMemcpy(&S0, D.st, sizeof S0, cudaMemcpyDeviceToHost));
        double *o = (double *)host_dst;
        o[0] = S0.q90; o[1] = S0.Rhat; o[2] = S0.kappa; o[3] = S0.p_x; o[4] = S0.L_nn;
        o[5] = S0.tau_max64; o[6] = S0.tau_min64; o[7] = S0.tau_max; o[8] = S0.tau_min;
        o[9] = S0.L_gb; o[10] = S0.L_ib; o[11] = S0.n_lambda; o[12] = S0.t; o[13] = S0.ib;
        o[14] = (double)S0.n_fallback; o[15] = D.k_pad;
        return HAC_OK;
    }
    default: return HAC_EINVAL;
    }
    if (bytes < sz) return HAC_EINVAL;
    CK(cudaMemcpy(host_dst, src, sz, cudaMemcpyDeviceToHost));
    return HAC_OK;
}

int hac_batch_results(hac_batch *bt, int32_t *const *best_tours, double *best_lens)
{
    if (!bt) return HAC_EINVAL;
    std::vector<InstState> sts(bt->count);
    for (int b = 0; b < bt->count; ++b) {
        if (best_tours && best_tours[b])
            CK(cudaMemcpyAsync(best_tours[b], bt->hi[b].gb_tour, (size_t)bt->hi[b].n * 4,
                               cudaMemcpyDeviceToHost, bt->stream));
        if (best_lens)
            CK(cudaMemcpyAsync(&sts[b], bt->hi[b].st, sizeof(InstState), cudaMemcpyDeviceToHost,
                               bt->stream));
    }
    int st = hac_batch_sync(bt);
    if (st) return st;
    if (best_lens)
        for (int b = 0; b < bt->count; ++b) best_lens[b] = sts[b].L_gb;
    return HAC_OK;
}

int hac_batch_counters(hac_batch *bt, int64_t *ant_steps, int64_t *fallback_steps)
{
    if (!bt) return HAC_EINVAL;
    int64_t as = 0;
    for (int b = 0; b < bt->count; ++b)
        as += (int64_t)bt->zs[b].m * bt->zs[b].n * bt->t_host[b];
    if (ant_steps) *ant_steps = as;
    if (fallback_steps) {
        int st = hac_batch_sync(bt);
        if (st) return st;
        int64_t fb = 0;
        for (int b = 0; b < bt->count; ++b) {
            InstState S0;
            CK(cudaMemcpy(&S0, bt->hi[b].st, sizeof S0, cudaMemcpyDeviceToHost));
            fb += (int64_t)S0.n_fallback;
        }
        *fallback_steps = fb;
    }
    return HAC_OK;
}

int hac_batch_launches(hac_batch *bt, int64_t *launches)
{
    if (!bt || !launches) return HAC_EINVAL;
    *launches = bt->launches;
    return HAC_OK;
}

int hac_batch_kernel_time(hac_batch *bt, int32_t group, double *ms, int64_t *launches)
{
    if (!bt || group < 0 || group > 3) return HAC_EINVAL;
    if (!bt->ex.profile) return HAC_EINVAL;
    int st = fold_events(bt);
    if (st) return st;
    if (ms) *ms = bt->group_ms[group];
    if (launches) *launches = bt->group_launches[group];
    return HAC_OK;
}

int hac_batch_destroy(hac_batch *bt)
{
    if (!bt) return HAC_EINVAL;
    if (bt->gexec) cudaGraphExecDestroy(bt->gexec);
    for (cudaEvent_t e : bt->ev_pool) cudaEventDestroy(e);
    for (FusedGroup &G : bt->groups) {
        if (G.side) cudaStreamDestroy(G.side);
        if (G.fork) cudaEventDestroy(G.fork);
        if (G.join) cudaEventDestroy(G.join);
    }
    delete bt;
    return HAC_OK;
}

int hac_solve_batch(const hac_instance *ins, const hac_params *ps, int32_t count,
                    int32_t inputs_on_device, void *workspace, size_t ws_bytes,
                    const hac_exec *exec, int32_t *const *best_tours, double *best_lens,
                    int32_t *statuses, void *stream)
{
    hac_batch *bt = nullptr;
    int st = hac_batch_create(ins, ps, count, inputs_on_device, workspace, ws_bytes, exec, stream, &bt);
    if (!st) st = hac_batch_run(bt);
    if (!st) st = hac_batch_results(bt, best_tours, best_lens);
    if (bt) hac_batch_destroy(bt);
    if (statuses)
        for (int b = 0; b < count; ++b) statuses[b] = st;
    return st;
}

int hac_solve(const hac_instance *in, const hac_params *p, int32_t inputs_on_device,
              void *workspace, size_t ws_bytes, int32_t *best_tour, double *best_len, void *stream)
{
    int32_t *tours[1] = {best_tour};
    return hac_solve_batch(in, p, 1, inputs_on_device, workspace, ws_bytes, nullptr, tours,
                           best_len, nullptr, stream);
}

}  // extern "C"
