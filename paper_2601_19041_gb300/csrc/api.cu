// Host orchestration behind the C ABI of heataco.h: workspace layout, input
// upload and validation, work tables, the iteration loop (optionally captured
// in a CUDA graph) and read-back.  Every device array is a slice of the
// caller's workspace; only a one-shot call given no workspace takes one from
// the stream-ordered pool for its own duration.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "host.h"

using namespace hac;
using namespace hac::host;

namespace hac {
namespace host {
thread_local int g_last_cuda = 0;
}
}  // namespace hac

// a contiguous range of instances iterated on its own stream (per-step path)
struct BatchPart {
    int b0 = 0, count = 0;                 // instances b0 .. b0+count-1
    int warp_off = 0, warp_len = 0;        // slice of the warp table (instance index relative to b0)
    int slot_off = 0, slot_len = 0;        // slice of the relative slot table
    int max_n = 0, max_kp = 0, ls_all_m = 0;
    bool any_ls = false;
    cudaStream_t stream = nullptr;         // the batch's stream when there is one part
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_kernels = 0;
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
    int2 *d_slotmap_rel = nullptr;      // slot table with instance indices relative to the part
    std::vector<BatchPart> parts;
    int4 *d_warpmap = nullptr;
    int warpmap_len = 0;
    int32_t *d_order = nullptr;
    std::vector<FusedGroup> groups;   // non-empty when the fused kernel is used
    int *d_err = nullptr;
    int max_n = 0, max_kp = 0;
    bool any_ls = false;
    int ls_all_m = 0;               // largest m among the instances with local search on every ant
    std::vector<int> t_host;
    cudaGraphExec_t fexec = nullptr;   // fused groups (fork/join included) for fexec_iters iterations
    int fexec_iters = -1;
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

static int plan_fused(hac_batch *bt, std::vector<int32_t> &order)
{
    const int apw = bt->ex.ants_per_warp;   // 0: chosen per instance (plan_groups)
    if (apw != 0 && apw != 2 && apw != 4 && apw != 16 && apw != 32)
        return HAC_EUNSUPPORTED;            // the fused kernel has no 1-ant-per-warp form
    std::vector<int> members(bt->count);
    for (int b = 0; b < bt->count; ++b) members[b] = b;
    return plan_groups(bt->zs, members, apw, bt->ex.cluster_log2, bt->ex.fallback_list, bt->groups, order);
}

// Everything hac_batch_create does after allocating the handle; on failure
// the caller releases the handle (and the streams and events made so far).
static int batch_setup(hac_batch *bt, const hac_instance *ins, const hac_params *ps, int32_t count,
                       int32_t inputs_on_device, void *workspace, const hac_exec &ex, void *stream,
                       const Plan &P)
{
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
    bt->d_slotmap_rel = (int2 *)(B + A.take(slots * sizeof(int2)));
    bt->d_warpmap = (int4 *)(B + A.take(warps * sizeof(int4)));
    bt->d_order = (int32_t *)(B + A.take((size_t)count * sizeof(int32_t)));
    size_t z0 = A.take(sizeof(int));
    bt->d_err = (int *)(B + z0);
    for (int b = 0; b < count; ++b) {
        DevInst &D = bt->hi[b];
        std::memset(&D, 0, sizeof D);
        bind_zero(D, P.zs[b], A, B);
    }
    const size_t zero_end = A.off;
    CK(cudaMemsetAsync(B + z0, 0, zero_end - z0, s));

    for (int b = 0; b < count; ++b) {
        const hac_instance &in = ins[b];
        const hac_params &p = ps[b];
        const Sizes &z = P.zs[b];
        DevInst &D = bt->hi[b];
        bind_instance(D, in, p, z, inputs_on_device, ex, A, B);
        if (!inputs_on_device) {
            int st2 = upload_inputs(D, in, z, s);
            if (st2) return st2;
        }
        bt->max_n = std::max(bt->max_n, z.n);
        bt->max_kp = std::max(bt->max_kp, z.kp);
        bt->any_ls |= z.ls != 0;
        if (z.ls == 2 || z.ls == 4) bt->ls_all_m = std::max(bt->ls_all_m, z.m);
    }
    // parts of the per-step path: contiguous instance ranges of about equal work
    const int nparts = std::max(1, std::min(std::min((int)bt->ex.parts, 64), count));
    {
        long long total = 0;
        for (int b = 0; b < count; ++b) total += (long long)P.zs[b].m * P.zs[b].n * P.zs[b].iters;
        long long acc = 0;
        int b0 = 0;
        for (int b = 0; b < count; ++b) {
            acc += (long long)P.zs[b].m * P.zs[b].n * P.zs[b].iters;
            const int made = (int)bt->parts.size();
            const bool last = b == count - 1;
            const bool cut = made + 1 < nparts && acc * nparts >= total * (made + 1) && count - b - 1 >= nparts - made - 1;
            if (cut || last) {
                BatchPart pt;
                pt.b0 = b0;
                pt.count = b + 1 - b0;
                bt->parts.push_back(pt);
                b0 = b + 1;
            }
        }
    }
    // work tables (warp and relative slot tables part by part)
    std::vector<int2> rowmap, slotmap, slotrel;
    std::vector<int4> warpmap;
    const int apw = bt->ex.ants_per_warp ? bt->ex.ants_per_warp : 4;   // per-step path (also the fallback)
    for (BatchPart &pt : bt->parts) {
        pt.warp_off = (int)warpmap.size();
        pt.slot_off = (int)slotrel.size();
        for (int b = pt.b0; b < pt.b0 + pt.count; ++b) {
            const Sizes &z = P.zs[b];
            for (int r = 0; r < z.n; r += ROWS_PER_BLOCK) rowmap.push_back(make_int2(b, r));
            const size_t S = (size_t)z.n * z.kp;
            for (size_t q = 0; q < S; q += SLOTS_PER_BLOCK) {
                slotmap.push_back(make_int2(b, (int)q));
                slotrel.push_back(make_int2(b - pt.b0, (int)q));
            }
            for (int a = 0; a < z.m; a += apw) warpmap.push_back(make_int4(b - pt.b0, a, 0, 0));
            pt.max_n = std::max(pt.max_n, z.n);
            pt.max_kp = std::max(pt.max_kp, z.kp);
            pt.any_ls |= z.ls != 0;
            if (z.ls == 2 || z.ls == 4) pt.ls_all_m = std::max(pt.ls_all_m, z.m);
        }
        pt.warp_len = (int)warpmap.size() - pt.warp_off;
        pt.slot_len = (int)slotrel.size() - pt.slot_off;
        if (bt->parts.size() == 1) {
            pt.stream = s;
        } else {
            CK(cudaStreamCreateWithFlags(&pt.stream, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&pt.fork, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&pt.join, cudaEventDisableTiming));
        }
    }
    bt->rowmap_len = (int)rowmap.size();
    bt->slotmap_len = (int)slotmap.size();
    bt->warpmap_len = (int)warpmap.size();
    CK(cudaMemcpyAsync(bt->d_slotmap_rel, slotrel.data(), slotrel.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(bt->d_rowmap, rowmap.data(), rowmap.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(bt->d_slotmap, slotmap.data(), slotmap.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(bt->d_warpmap, warpmap.data(), warpmap.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(bt->d_inst, bt->hi.data(), (size_t)count * sizeof(DevInst), cudaMemcpyHostToDevice, s));
    if (bt->ex.fused) {
        std::vector<int32_t> order;
        if (plan_fused(bt, order) == HAC_OK) {
            CK(cudaMemcpyAsync(bt->d_order, order.data(), order.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, s));
        } else {
            bt->ex.fused = 0;   // some instance does not fit the fused kernel: per-iteration path
            if (bt->ex.ants_per_warp == 0) bt->ex.ants_per_warp = 4;
            bt->groups.clear();
        }
    }

    bt->launches += timed(bt, 2, [&] {
        return launch_prep(bt->d_inst, bt->hi.data(), count, bt->d_rowmap, bt->rowmap_len,
                           bt->d_slotmap, bt->slotmap_len, bt->d_err, s);
    });
    CK(cudaGetLastError());
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
    e->parts = 0;
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
    if (!inputs_on_device && (st = check_host_all(ins, ps, count))) return st;
    hac_exec ex;
    hac_exec_default(&ex);
    if (exec) ex = *exec;
    if (ex.ants_per_warp == 0 && !ex.fused) ex.ants_per_warp = 4;   // fused: 0 = per instance
    if (ex.ants_per_warp != 0 && ex.ants_per_warp != 1 && ex.ants_per_warp != 2 && ex.ants_per_warp != 4 && ex.ants_per_warp != 16 &&
        ex.ants_per_warp != 32)
        return HAC_EINVAL;
    if (ex.warps_per_block == 0) ex.warps_per_block = 4;
    if (ex.warps_per_block < 1 || ex.warps_per_block > 8) return HAC_EINVAL;
    if (ex.fallback_list != 0 && ex.fallback_list != FBL_LEN) return HAC_EINVAL;
    if (ex.cluster_log2 < 0 || ex.cluster_log2 > 3) return HAC_EINVAL;
    if (ex.parts < 0 || ex.parts > 64) return HAC_EINVAL;
    if (ex.ants_per_warp == 32)   // step-major tours: 2-opt on every ant needs them ant by ant
        for (int b = 0; b < count; ++b)
            if (ps[b].local_search == 2 || ps[b].local_search == 4) return HAC_EUNSUPPORTED;

    hac_batch *bt = new (std::nothrow) hac_batch;
    if (!bt) return HAC_ENOMEM;
    st = batch_setup(bt, ins, ps, count, inputs_on_device, workspace, ex, stream, P);
    if (st) {
        hac_batch_destroy(bt);
        return st;
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

static int enqueue_iteration(hac_batch *bt, const BatchPart &pt)
{
    const DevInst *d = bt->d_inst + pt.b0;
    if (bt->parts.size() > 1)   // several parts: no per-group timing (the fork/join region is timed)
        return launch_construct(d, bt->d_warpmap + pt.warp_off, pt.warp_len, bt->ex.ants_per_warp,
                                bt->ex.warps_per_block, pt.max_n, pt.max_kp, pt.count, pt.stream) +
               launch_iteration_tail(d, pt.count, bt->d_slotmap_rel + pt.slot_off, pt.slot_len, pt.any_ls,
                                     pt.max_n, pt.ls_all_m, pt.stream);
    int k = timed(bt, 0, [&] {
        return launch_construct(d, bt->d_warpmap + pt.warp_off, pt.warp_len, bt->ex.ants_per_warp,
                                bt->ex.warps_per_block, pt.max_n, pt.max_kp, pt.count, pt.stream);
    });
    k += timed(bt, 1, [&] {
        return launch_iteration_tail(d, pt.count, bt->d_slotmap_rel + pt.slot_off, pt.slot_len, pt.any_ls,
                                     pt.max_n, pt.ls_all_m, pt.stream);
    });
    return k;
}

// `todo` iterations of one part on its stream (CUDA graphs of GRAPH_CHUNK
// iterations when enabled)
static int iterate_part(hac_batch *bt, BatchPart &pt, int todo)
{
    cudaStream_t s = pt.stream;
    if (bt->ex.use_graph && !bt->ex.profile && s != nullptr && todo >= GRAPH_CHUNK) {
        if (!pt.gexec) {
            cudaGraph_t g;
            CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            pt.graph_kernels = 0;
            for (int q = 0; q < GRAPH_CHUNK; ++q) pt.graph_kernels += enqueue_iteration(bt, pt);
            cudaError_t e1 = cudaGetLastError();
            cudaError_t e2 = cudaStreamEndCapture(s, &g);
            if (e1 != cudaSuccess) { g_last_cuda = (int)e1; if (e2 == cudaSuccess) cudaGraphDestroy(g); return HAC_ECUDA; }
            CK(e2);
            cudaError_t e3 = cudaGraphInstantiate(&pt.gexec, g, 0);
            cudaGraphDestroy(g);
            CK(e3);
        }
        while (todo >= GRAPH_CHUNK) {
            CK(cudaGraphLaunch(pt.gexec, s));
            bt->launches += pt.graph_kernels;
            todo -= GRAPH_CHUNK;
        }
    }
    for (; todo > 0; --todo) bt->launches += enqueue_iteration(bt, pt);
    CK(cudaGetLastError());
    return HAC_OK;
}

// the fused groups' launches (launch_groups); with CUDA graphs on, they are
// captured once per iteration count and replayed
static int enqueue_fused(hac_batch *bt, int iters)
{
    if (bt->ex.use_graph && !bt->ex.profile && bt->stream != nullptr) {
        if (!bt->fexec || bt->fexec_iters != iters) {
            if (bt->fexec) { cudaGraphExecDestroy(bt->fexec); bt->fexec = nullptr; }
            cudaGraph_t g;
            CK(cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e1 = launch_groups(bt->d_inst, bt->d_order, nullptr, bt->groups,
                                           iters, bt->stream);
            cudaError_t e2 = cudaStreamEndCapture(bt->stream, &g);
            if (e1 != cudaSuccess) { g_last_cuda = (int)e1; if (e2 == cudaSuccess) cudaGraphDestroy(g); return HAC_ECUDA; }
            CK(e2);
            cudaError_t e3 = cudaGraphInstantiate(&bt->fexec, g, 0);
            cudaGraphDestroy(g);
            CK(e3);
            bt->fexec_iters = iters;
        }
        CK(cudaGraphLaunch(bt->fexec, bt->stream));
        bt->launches += (long long)bt->groups.size();
        return HAC_OK;
    }
    cudaError_t err = cudaSuccess;
    const int k = timed(bt, 3, [&] {
        err = launch_groups(bt->d_inst, bt->d_order, nullptr, bt->groups, iters, bt->stream);
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
    if (todo > 0) {
        if (bt->parts.size() == 1) {
            int st = iterate_part(bt, bt->parts[0], todo);
            if (st) return st;
        } else {
            // the parts run on their own streams, forked from and joined into the batch's
            int st = HAC_OK;
            timed(bt, 0, [&] {
                for (BatchPart &pt : bt->parts) {
                    cudaEventRecord(pt.fork, s);
                    cudaStreamWaitEvent(pt.stream, pt.fork, 0);
                }
                // chunk by chunk, round robin over the parts, so that no part's
                // launches fill the launch queue before the next part's start
                for (int left = todo; left > 0 && !st;) {
                    const int chunk = std::min(left, GRAPH_CHUNK);
                    for (BatchPart &pt : bt->parts)
                        if (!st) st = iterate_part(bt, pt, chunk);
                    left -= chunk;
                }
                for (BatchPart &pt : bt->parts) {
                    cudaEventRecord(pt.join, pt.stream);
                    cudaStreamWaitEvent(s, pt.join, 0);
                }
                return 0;
            });
            if (st) return st;
        }
    }
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
    case HAC_F_FBL:
        if (!D.fbl) return HAC_EINVAL;
        src = D.fbl; sz = n * FBL_LEN * 4; break;
    case HAC_F_FBL2:
        if (!D.fbl2) return HAC_EINVAL;
        src = D.fbl2; sz = n * FBL2_LEN * 2; break;
    case HAC_F_SCALARS: {
        if (bytes < 21 * sizeof(double)) return HAC_EINVAL;
        InstState S0;
        CK(cudaMemcpy(&S0, D.st, sizeof S0, cudaMemcpyDeviceToHost));
        double *o = (double *)host_dst;
        o[0] = S0.q90; o[1] = S0.Rhat; o[2] = S0.kappa; o[3] = S0.p_x; o[4] = S0.L_nn;
        o[5] = S0.tau_max64; o[6] = S0.tau_min64; o[7] = S0.tau_max; o[8] = S0.tau_min;
        o[9] = S0.L_gb; o[10] = S0.L_ib; o[11] = S0.n_lambda; o[12] = S0.t; o[13] = S0.ib;
        o[14] = (double)S0.n_fallback; o[15] = D.k_pad;
        o[16] = S0.L_rb; o[17] = S0.n_restarts; o[18] = S0.t_restart; o[19] = S0.u_gb;
        o[20] = (double)S0.n_edges / (2.0 * (double)D.n);
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
    if (bt->fexec) cudaGraphExecDestroy(bt->fexec);
    for (BatchPart &pt : bt->parts) {
        if (pt.gexec) cudaGraphExecDestroy(pt.gexec);
        if (pt.fork) cudaEventDestroy(pt.fork);
        if (pt.join) cudaEventDestroy(pt.join);
        if (pt.stream && pt.stream != bt->stream) cudaStreamDestroy(pt.stream);
    }
    for (cudaEvent_t e : bt->ev_pool) cudaEventDestroy(e);
    delete bt;
    return HAC_OK;
}

int hac_solve_batch(const hac_instance *ins, const hac_params *ps, int32_t count,
                    int32_t inputs_on_device, void *workspace, size_t ws_bytes,
                    const hac_exec *exec, int32_t *const *best_tours, double *best_lens,
                    int32_t *statuses, hac_stats *stats, void *stream)
{
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    void *own = nullptr;   // stream-ordered workspace of a call given none
    int st = HAC_OK;
    if (!workspace) {
        st = hac_batch_workspace_size(ins, ps, count, inputs_on_device, &ws_bytes);
        if (!st) {
            cudaError_t e = cudaMallocAsync(&own, ws_bytes, s);
            if (e != cudaSuccess) {
                g_last_cuda = (int)e;
                cudaGetLastError();
                st = HAC_ENOMEM;
                own = nullptr;
            }
            workspace = own;
        }
    }
    hac_batch *bt = nullptr;
    if (!st) st = hac_batch_create(ins, ps, count, inputs_on_device, workspace, ws_bytes, exec, stream, &bt);
    if (!st) st = hac_batch_run(bt);
    if (!st) st = hac_batch_results(bt, best_tours, best_lens);
    if (!st && stats) {
        for (int b = 0; b < count; ++b) {
            InstState S0;
            cudaError_t e = cudaMemcpy(&S0, bt->hi[b].st, sizeof S0, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) { g_last_cuda = (int)e; st = HAC_ECUDA; break; }
            const Sizes &z = bt->zs[b];
            hac_stats &o = stats[b];
            o.iterations = S0.t;
            o.restarts = S0.n_restarts;
            o.ant_steps = (int64_t)z.m * z.n * S0.t;
            o.fallback_steps = (int64_t)S0.n_fallback;
            o.kappa = S0.kappa;
            o.edges_per_n = (double)S0.n_edges / (2.0 * (double)z.n);
            o.L_nn = S0.L_nn;
        }
    }
    if (bt) hac_batch_destroy(bt);
    if (own) {
        cudaError_t e = cudaFreeAsync(own, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess && !st) { g_last_cuda = (int)e; st = HAC_ECUDA; }
    }
    if (!st && stats) {
        const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int b = 0; b < count; ++b) stats[b].seconds = sec;
    }
    if (statuses)
        for (int b = 0; b < count; ++b) statuses[b] = st;
    return st;
}

int hac_batch_autotune(const hac_instance *ins, const hac_params *ps, int32_t count,
                       int32_t inputs_on_device, void *workspace, size_t ws_bytes, int32_t trial_iters,
                       void *stream, hac_exec *best, double *ms_per_iter)
{
    if (!best || trial_iters < 1) return HAC_EINVAL;
    Plan P;
    int st = plan_batch(ins, ps, count, inputs_on_device, P);
    if (st) return st;
    if (!workspace || ws_bytes < P.total) return HAC_ENOMEM;
    // candidates: every execution layout (none changes a result)
    std::vector<hac_exec> cands;
    for (int apw : {0, 16, 4, 2, 32})
        for (int clog = 0; clog <= 2; ++clog)
            for (int fbl : {FBL_LEN, 0}) {
                hac_exec e;
                hac_exec_default(&e);
                e.fused = 1; e.ants_per_warp = apw; e.cluster_log2 = clog; e.fallback_list = fbl;
                cands.push_back(e);
            }
    for (int apw : {16, 4, 2, 1})
        for (int wpb : {4, 8})
            for (int parts : {1, 4}) {
                if (parts > count) continue;
                hac_exec e;
                hac_exec_default(&e);
                e.fused = 0; e.ants_per_warp = apw; e.warps_per_block = wpb; e.fallback_list = FBL_LEN;
                e.parts = parts;
                cands.push_back(e);
            }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t ev[2];
    CK(cudaEventCreate(&ev[0]));
    if (cudaEventCreate(&ev[1]) != cudaSuccess) { cudaEventDestroy(ev[0]); return HAC_ECUDA; }
    double best_ms = -1.0;
    int rc = HAC_OK;
    for (const hac_exec &c : cands) {
        hac_exec e = c;
        e.use_graph = 0;
        hac_batch *bt = nullptr;
        st = hac_batch_create(ins, ps, count, inputs_on_device, workspace, ws_bytes, &e, stream, &bt);
        if (st == HAC_EUNSUPPORTED) continue;
        if (st) { rc = st; break; }
        if (e.fused && !bt->ex.fused) {   // does not fit the cluster kernel: same as a per-step candidate
            hac_batch_destroy(bt);
            continue;
        }
        float ms = 0.f;
        st = hac_batch_iterate(bt, 1);
        if (!st && cudaEventRecord(ev[0], s) != cudaSuccess) st = HAC_ECUDA;
        if (!st) st = hac_batch_iterate(bt, trial_iters);
        if (!st && cudaEventRecord(ev[1], s) != cudaSuccess) st = HAC_ECUDA;
        if (!st) st = hac_batch_sync(bt);
        if (!st && cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) st = HAC_ECUDA;
        hac_batch_destroy(bt);
        if (st) { rc = st; break; }
        if (best_ms < 0.0 || ms < best_ms) {
            best_ms = ms;
            *best = c;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc) return rc;
    if (best_ms < 0.0) return HAC_EUNSUPPORTED;
    best->use_graph = 1;
    if (ms_per_iter) *ms_per_iter = best_ms / trial_iters;
    return HAC_OK;
}

int hac_solve(const hac_instance *in, const hac_params *p, int32_t inputs_on_device,
              void *workspace, size_t ws_bytes, int32_t *best_tour, double *best_len,
              hac_stats *stats, void *stream)
{
    int32_t *tours[1] = {best_tour};
    return hac_solve_batch(in, p, 1, inputs_on_device, workspace, ws_bytes, nullptr, tours,
                           best_len, nullptr, stats, stream);
}

}  // extern "C"
