// Continuous-batching decode server behind the hac_server_* entry points of
// heataco.h.
//
// A server owns a caller-provided device workspace: a header (one DevInst per
// slot, the cluster -> slot order of the fused kernel, an error word) and a
// heap from which every admitted request takes one region holding its whole
// decoder state (inputs, candidate tables, pheromone, tours, T_gb, bounds).
// The state stays resident from admission until the result is collected.
//
//   submit: checks the request, finds a free slot and a heap region (first
//           fit; HAC_EBUSY when either is missing, so admission follows free
//           memory), stages the inputs in a pinned upload ring, copies them
//           and runs the preparation kernels (candidate lists, evidence,
//           kappa, W, T_NN, bounds, tau_0) on one of PREP_STREAMS side
//           streams, so that preparations overlap each other and the running
//           iterations, and submit returns without waiting for the device.
//   tick:   admits the requests whose preparation has finished, then runs
//           the tick's MMAS iterations of every admitted request.  Requests
//           below step_min_n nodes run in one launch of the persistent
//           cluster kernel per cluster size (the batch API's fused path);
//           larger ones, whose candidate tables would pin several SMs for a
//           few ants, run the per-step kernels (rows read through L2, many
//           instances per SM) on a stream of their own, concurrently.  Each
//           instance continues from its own iteration counter, so requests
//           at different points of their search share a launch.  Requests
//           that reach their iteration count get their T_gb and L_gb copied
//           to pinned host staging.
//   poll:   returns a finished request's result and frees its slot and region.
//
// Per request the arithmetic is exactly that of hac_solve (the random numbers
// depend on the instance's seed, iteration, ant and step only), so a request
// decodes to the same tour alone and in any mix.
#include <algorithm>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include "host.h"

using namespace hac;
using namespace hac::host;

namespace {

enum ReqState { R_FREE = 0, R_PREP, R_RUN, R_RETIRE };

constexpr int PREP_STREAMS = 4;
constexpr size_t RING_BYTES = (size_t)64 << 20;   // pinned upload ring

struct RingEntry {
    size_t off, bytes;
    cudaEvent_t ev;                 // the copies out of this entry are done
};

struct Slot {
    int state = R_FREE;
    uint64_t ticket = 0;
    size_t off = 0, bytes = 0;      // heap region (offset from the heap base)
    Sizes z{};
    int route = 0;                  // 0: cluster kernel, 1: per-step kernels
    int t = 0;                      // iterations enqueued so far
    cudaEvent_t ready = nullptr;    // preparation done (prep stream)
    cudaEvent_t done = nullptr;     // result staged (main stream)
    int32_t *h_tour = nullptr;      // pinned staging: T_gb
    InstState *h_st = nullptr;      // pinned staging: final state (L_gb)
};

struct Block {
    size_t off, bytes;
};

// request region: zero part, instance layout, row and slot work tables
struct Region {
    size_t zero_end = 0, rowmap = 0, slotmap = 0, total = 0;
    int rows = 0, slots = 0;
};

Region region_of(const Sizes &z)
{
    Region R;
    Arena A;
    layout_zero(A, z, [](const char *, size_t) {});
    R.zero_end = A.off;
    layout_instance(A, z, 0, [](const char *, size_t) {});
    R.rows = (z.n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK;
    R.slots = (int)(((size_t)z.n * z.kp + SLOTS_PER_BLOCK - 1) / SLOTS_PER_BLOCK);
    R.rowmap = A.take((size_t)R.rows * sizeof(int2));
    R.slotmap = A.take((size_t)R.slots * sizeof(int2));
    R.total = (A.off + 255) & ~(size_t)255;
    return R;
}

}  // namespace

struct hac_server {
    hac_server_cfg cfg{};
    hac_exec ex{};
    cudaStream_t stream = nullptr;
    cudaStream_t prep[PREP_STREAMS] = {};
    int next_prep = 0;
    char *ring = nullptr;           // pinned, RING_BYTES
    size_t ring_head = 0;
    std::deque<RingEntry> ring_q;   // live entries, oldest first
    std::vector<cudaEvent_t> ring_ev;   // idle events
    DevInst *d_inst = nullptr;
    int32_t *d_order[2] = {nullptr, nullptr};   // alternating per tick
    int32_t *d_iters[2] = {nullptr, nullptr};   // iterations of each cluster this tick
    int *d_err = nullptr;
    char *heap = nullptr;
    size_t heap_bytes = 0;
    std::vector<Block> free_list;   // sorted by offset, coalesced
    std::vector<Slot> slots;
    std::vector<DevInst> hi;        // host copy of each slot's DevInst
    std::vector<Sizes> zs;          // per slot (valid while occupied)
    char *pinned = nullptr;
    int32_t *h_order[2] = {nullptr, nullptr};   // pinned sources of d_order, then d_iters
    uint64_t next_ticket = 1;
    cudaEvent_t tick_ev[2] = {nullptr, nullptr};
    // per-step route: stream, fork/join, per-tick compact instance and work tables
    cudaStream_t sstream = nullptr;
    cudaEvent_t sfork = nullptr, sjoin = nullptr;
    hac_exec sex{};
    size_t swarp_cap = 0, sslot_cap = 0;
    DevInst *d_sinst[2] = {nullptr, nullptr}, *h_sinst[2] = {nullptr, nullptr};
    int4 *d_swarp[2] = {nullptr, nullptr}, *h_swarp[2] = {nullptr, nullptr};
    int2 *d_sslot[2] = {nullptr, nullptr}, *h_sslot[2] = {nullptr, nullptr};
    bool tick_rec[2] = {false, false};
    long long ticks = 0;
    long long launches = 0;
};

namespace {

bool heap_alloc(hac_server *sv, size_t bytes, size_t &off)
{
    for (size_t q = 0; q < sv->free_list.size(); ++q) {
        Block &b = sv->free_list[q];
        if (b.bytes < bytes) continue;
        off = b.off;
        b.off += bytes;
        b.bytes -= bytes;
        if (!b.bytes) sv->free_list.erase(sv->free_list.begin() + q);
        return true;
    }
    return false;
}

void heap_free(hac_server *sv, size_t off, size_t bytes)
{
    auto &L = sv->free_list;
    size_t q = 0;
    while (q < L.size() && L[q].off < off) ++q;
    L.insert(L.begin() + q, Block{off, bytes});
    if (q + 1 < L.size() && L[q].off + L[q].bytes == L[q + 1].off) {
        L[q].bytes += L[q + 1].bytes;
        L.erase(L.begin() + q + 1);
    }
    if (q > 0 && L[q - 1].off + L[q - 1].bytes == L[q].off) {
        L[q - 1].bytes += L[q].bytes;
        L.erase(L.begin() + q);
    }
}

size_t free_total(const hac_server *sv)
{
    size_t f = 0;
    for (const Block &b : sv->free_list) f += b.bytes;
    return f;
}

// whether the fused kernel takes this request on its own
int fits_fused(const hac_server *sv, const Sizes &z)
{
    std::vector<Sizes> one{z};
    std::vector<int> mem{0};
    std::vector<FusedGroup> g;
    std::vector<int32_t> o;
    return plan_groups(one, mem, sv->ex.ants_per_warp, sv->ex.cluster_log2, sv->ex.fallback_list, g, o);
}

// per-tick tables of the per-step route: warp and slot work items
void step_caps(const hac_server_cfg &c, int apw, size_t &warps, size_t &slots)
{
    warps = slots = 0;
    if (c.step_min_n <= 0) return;
    warps = (size_t)c.max_slots * ((HAC_MMAX + apw - 1) / apw);
    slots = (size_t)c.max_slots * (((size_t)c.max_n * HAC_KMAX + SLOTS_PER_BLOCK - 1) / SLOTS_PER_BLOCK);
}

size_t header_bytes(const hac_server_cfg &c, int step_apw)
{
    Arena A;
    A.take((size_t)c.max_slots * sizeof(DevInst));
    for (int q = 0; q < 4; ++q) A.take((size_t)c.max_slots * sizeof(int32_t));
    A.take(sizeof(int));
    size_t w, s;
    step_caps(c, step_apw, w, s);
    if (c.step_min_n > 0)
        for (int q = 0; q < 2; ++q) {
            A.take((size_t)c.max_slots * sizeof(DevInst));
            A.take(w * sizeof(int4));
            A.take(s * sizeof(int2));
        }
    return (A.off + 255) & ~(size_t)255;
}

// iterations one request runs in a tick
int tick_iters(const hac_server *sv, const Slot &S)
{
    int it = sv->cfg.iters_per_tick;
    if (sv->cfg.steps_per_tick > 0) it = std::max(1, std::min(it, sv->cfg.steps_per_tick / S.z.n));
    return std::min(it, S.z.iters - S.t);
}

int enqueue_groups(hac_server *sv, std::vector<FusedGroup> &groups, const int32_t *d_order,
                   const int32_t *d_iters)
{
    cudaError_t e = launch_groups(sv->d_inst, d_order, d_iters, groups, 0, sv->stream);
    if (e != cudaSuccess) { g_last_cuda = (int)e; return HAC_ECUDA; }
    sv->launches += (long long)groups.size();
    return HAC_OK;
}

// Reserves `bytes` of the upload ring (bytes <= RING_BYTES), waiting for the
// oldest entries' copies when it is full.  Entries are taken in ring order.
int ring_take(hac_server *sv, size_t bytes, size_t &off)
{
    auto overlaps = [&](size_t pos) {
        for (const RingEntry &r : sv->ring_q)
            if (pos < r.off + r.bytes && r.off < pos + bytes) return true;
        return false;
    };
    for (;;) {
        if (sv->ring_q.empty()) sv->ring_head = 0;
        const size_t pos = sv->ring_head + bytes <= RING_BYTES ? sv->ring_head : 0;
        if (!overlaps(pos)) {
            off = pos;
            sv->ring_head = pos + bytes;
            return HAC_OK;
        }
        RingEntry r = sv->ring_q.front();
        CK(cudaEventSynchronize(r.ev));
        sv->ring_q.pop_front();
        sv->ring_ev.push_back(r.ev);
    }
}

// Host -> device copies of one request (inputs, work tables, DevInst) through
// the pinned ring on stream ps; falls back to plain copies from the caller's
// memory when the request is larger than the ring.
struct Upload {
    const void *src;
    void *dst;
    size_t bytes;
};

int upload_staged(hac_server *sv, const std::vector<Upload> &ups, cudaStream_t ps)
{
    size_t total = 0;
    for (const Upload &u : ups) total += (u.bytes + 15) & ~(size_t)15;
    if (total > RING_BYTES) {
        for (const Upload &u : ups)
            if (u.bytes) CK(cudaMemcpyAsync(u.dst, u.src, u.bytes, cudaMemcpyHostToDevice, ps));
        return HAC_OK;
    }
    // retire finished entries first, then reserve
    while (!sv->ring_q.empty() && cudaEventQuery(sv->ring_q.front().ev) == cudaSuccess) {
        sv->ring_ev.push_back(sv->ring_q.front().ev);
        sv->ring_q.pop_front();
    }
    size_t off;
    int st = ring_take(sv, total, off);
    if (st) return st;
    cudaEvent_t ev;
    if (!sv->ring_ev.empty()) { ev = sv->ring_ev.back(); sv->ring_ev.pop_back(); }
    else CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    size_t o = off;
    for (const Upload &u : ups) {
        if (u.bytes) {
            std::memcpy(sv->ring + o, u.src, u.bytes);
            CK(cudaMemcpyAsync(u.dst, sv->ring + o, u.bytes, cudaMemcpyHostToDevice, ps));
        }
        o += (u.bytes + 15) & ~(size_t)15;
    }
    CK(cudaEventRecord(ev, ps));
    sv->ring_q.push_back(RingEntry{off, total, ev});
    return HAC_OK;
}

// The per-step route of one tick: a compact DevInst array of the members (its
// entries point into the members' resident regions), their warp and slot work
// tables, and min over members of the tick's iteration budget, each iteration
// one construction launch and one iteration tail, on the route's own stream.
int enqueue_step_route(hac_server *sv, const std::vector<int> &mem, int par)
{
    const int apw = sv->sex.ants_per_warp;
    DevInst *hI = sv->h_sinst[par];
    int4 *hw = sv->h_swarp[par];
    int2 *hs = sv->h_sslot[par];
    size_t nw = 0, ns = 0;
    int it = sv->cfg.iters_per_tick, max_n = 0, max_kp = 0;
    bool any_ls = false;
    int ls_all_m = 0;
    for (size_t b = 0; b < mem.size(); ++b) {
        const Slot &S = sv->slots[mem[b]];
        hI[b] = sv->hi[mem[b]];
        for (int a = 0; a < S.z.m; a += apw) hw[nw++] = make_int4((int)b, a, 0, 0);
        const size_t SS = (size_t)S.z.n * S.z.kp;
        for (size_t q = 0; q < SS; q += SLOTS_PER_BLOCK) hs[ns++] = make_int2((int)b, (int)q);
        it = std::min(it, tick_iters(sv, S));
        max_n = std::max(max_n, S.z.n);
        max_kp = std::max(max_kp, S.z.kp);
        any_ls |= S.z.ls != 0;
        if (S.z.ls == 2 || S.z.ls == 4) ls_all_m = std::max(ls_all_m, S.z.m);
    }
    const int count = (int)mem.size();
    cudaStream_t ss = sv->sstream;
    CK(cudaEventRecord(sv->sfork, sv->stream));
    CK(cudaStreamWaitEvent(ss, sv->sfork, 0));
    CK(cudaMemcpyAsync(sv->d_sinst[par], hI, count * sizeof(DevInst), cudaMemcpyHostToDevice, ss));
    CK(cudaMemcpyAsync(sv->d_swarp[par], hw, nw * sizeof(int4), cudaMemcpyHostToDevice, ss));
    CK(cudaMemcpyAsync(sv->d_sslot[par], hs, ns * sizeof(int2), cudaMemcpyHostToDevice, ss));
    for (int q = 0; q < it; ++q) {
        sv->launches += launch_construct(sv->d_sinst[par], sv->d_swarp[par], (int)nw, apw,
                                         sv->sex.warps_per_block, max_n, max_kp, count, ss);
        sv->launches += launch_iteration_tail(sv->d_sinst[par], count, sv->d_sslot[par], (int)ns, any_ls, max_n,
                                              ls_all_m, ss);
    }
    CK(cudaGetLastError());
    for (int q : mem) sv->slots[q].t += it;
    return HAC_OK;
}

}  // namespace

extern "C" {

int hac_server_request_bytes(const hac_instance *in, const hac_params *p, size_t *bytes)
{
    if (!in || !p || !bytes) return HAC_EINVAL;
    Sizes z;
    int st = instance_sizes(*in, *p, 0, z);
    if (st) return st;
    *bytes = region_of(z).total;
    return HAC_OK;
}

int hac_server_create(const hac_server_cfg *cfg, void *workspace, size_t ws_bytes, void *stream,
                      hac_server **out)
{
    if (!out || !cfg) return HAC_EINVAL;
    *out = nullptr;
    const hac_server_cfg c = *cfg;
    if (c.max_slots < 1 || c.max_slots > 4096 || c.iters_per_tick < 1 || c.max_n < 3 || c.max_n > 65534 ||
        c.steps_per_tick < 0 || c.step_min_n < 0)
        return HAC_EINVAL;
    const int s_apw = c.step_ants_per_warp ? c.step_ants_per_warp : 1;
    const int s_wpb = c.step_warps_per_block ? c.step_warps_per_block : 8;
    if ((s_apw != 1 && s_apw != 2 && s_apw != 4 && s_apw != 16) || s_wpb < 1 || s_wpb > 8) return HAC_EINVAL;
    hac_exec ex = c.exec;
    if (ex.ants_per_warp == 0) ex.ants_per_warp = 4;
    if (ex.ants_per_warp != 2 && ex.ants_per_warp != 4 && ex.ants_per_warp != 16 && ex.ants_per_warp != 32)
        return HAC_EINVAL;
    if (ex.fallback_list != 0 && ex.fallback_list != FBL_LEN) return HAC_EINVAL;
    if (ex.cluster_log2 < 0 || ex.cluster_log2 > 3) return HAC_EINVAL;
    ex.fused = 1;
    ex.profile = 0;
    const size_t hdr = header_bytes(c, s_apw);
    if (!workspace || ws_bytes < hdr + 256 + 4096) return HAC_ENOMEM;

    hac_server *sv = new (std::nothrow) hac_server;
    if (!sv) return HAC_ENOMEM;
    sv->cfg = c;
    sv->ex = ex;
    sv->stream = (cudaStream_t)stream;
    char *B = (char *)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    Arena A;
    sv->d_inst = (DevInst *)(B + A.take((size_t)c.max_slots * sizeof(DevInst)));
    sv->d_order[0] = (int32_t *)(B + A.take((size_t)c.max_slots * sizeof(int32_t)));
    sv->d_order[1] = (int32_t *)(B + A.take((size_t)c.max_slots * sizeof(int32_t)));
    sv->d_iters[0] = (int32_t *)(B + A.take((size_t)c.max_slots * sizeof(int32_t)));
    sv->d_iters[1] = (int32_t *)(B + A.take((size_t)c.max_slots * sizeof(int32_t)));
    sv->d_err = (int *)(B + A.take(sizeof(int)));
    sv->sex = ex;
    sv->sex.fused = 0;
    sv->sex.ants_per_warp = s_apw;
    sv->sex.warps_per_block = s_wpb;
    step_caps(c, s_apw, sv->swarp_cap, sv->sslot_cap);
    if (c.step_min_n > 0)
        for (int q = 0; q < 2; ++q) {
            sv->d_sinst[q] = (DevInst *)(B + A.take((size_t)c.max_slots * sizeof(DevInst)));
            sv->d_swarp[q] = (int4 *)(B + A.take(sv->swarp_cap * sizeof(int4)));
            sv->d_sslot[q] = (int2 *)(B + A.take(sv->sslot_cap * sizeof(int2)));
        }
    sv->heap = B + hdr;
    sv->heap_bytes = ((uintptr_t)workspace + ws_bytes - (uintptr_t)sv->heap) & ~(size_t)255;
    sv->free_list.push_back(Block{0, sv->heap_bytes});
    sv->slots.resize(c.max_slots);
    sv->hi.resize(c.max_slots);
    sv->zs.resize(c.max_slots);

    auto fail = [&](cudaError_t e) {
        g_last_cuda = (int)e;
        hac_server_destroy(sv);
        return HAC_ECUDA;
    };
    cudaError_t e;
    const size_t stage = ((size_t)c.max_n * 4 + sizeof(InstState) + 255) & ~(size_t)255;
    const size_t ord = ((size_t)c.max_slots * 8 + 255) & ~(size_t)255;
    if ((e = cudaHostAlloc((void **)&sv->pinned, stage * c.max_slots + 2 * ord, cudaHostAllocDefault)) !=
        cudaSuccess)
        return fail(e);
    sv->h_order[0] = (int32_t *)(sv->pinned + stage * c.max_slots);
    sv->h_order[1] = (int32_t *)(sv->pinned + stage * c.max_slots + ord);
    if (c.step_min_n > 0) {
        const size_t per = (size_t)c.max_slots * sizeof(DevInst) + sv->swarp_cap * sizeof(int4) +
                           sv->sslot_cap * sizeof(int2);
        char *hp = nullptr;
        if ((e = cudaHostAlloc((void **)&hp, 2 * per, cudaHostAllocDefault)) != cudaSuccess) return fail(e);
        for (int q = 0; q < 2; ++q) {   // the block is released through h_sinst[0]
            char *b = hp + q * per;
            sv->h_sinst[q] = (DevInst *)b;
            sv->h_swarp[q] = (int4 *)(b + (size_t)c.max_slots * sizeof(DevInst));
            sv->h_sslot[q] = (int2 *)(b + (size_t)c.max_slots * sizeof(DevInst) + sv->swarp_cap * sizeof(int4));
        }
        if ((e = cudaStreamCreateWithFlags(&sv->sstream, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
        if ((e = cudaEventCreateWithFlags(&sv->sfork, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
        if ((e = cudaEventCreateWithFlags(&sv->sjoin, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
    }
    for (int q = 0; q < c.max_slots; ++q) {
        Slot &S = sv->slots[q];
        S.h_tour = (int32_t *)(sv->pinned + stage * q);
        S.h_st = (InstState *)(sv->pinned + stage * q + (size_t)c.max_n * 4);
        if ((e = cudaEventCreateWithFlags(&S.ready, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
        if ((e = cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
    }
    for (int g = 0; g < PREP_STREAMS; ++g)
        if ((e = cudaStreamCreateWithFlags(&sv->prep[g], cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    if ((e = cudaHostAlloc((void **)&sv->ring, RING_BYTES, cudaHostAllocDefault)) != cudaSuccess) return fail(e);
    for (int g = 0; g < 2; ++g)
        if ((e = cudaEventCreateWithFlags(&sv->tick_ev[g], cudaEventDisableTiming)) != cudaSuccess) return fail(e);
    // the preparation kernels are the ones that report into the error word
    if ((e = cudaMemsetAsync(sv->d_err, 0, sizeof(int), sv->prep[0])) != cudaSuccess) return fail(e);
    if ((e = cudaStreamSynchronize(sv->prep[0])) != cudaSuccess) return fail(e);
    *out = sv;
    return HAC_OK;
}

int hac_server_submit(hac_server *sv, const hac_instance *in, const hac_params *p, uint64_t *ticket)
{
    if (!sv || !in || !p || !ticket) return HAC_EINVAL;
    Sizes z;
    int st = instance_sizes(*in, *p, 0, z);
    if (st) return st;
    if (z.n > sv->cfg.max_n) return HAC_EINVAL;
    if ((st = check_host_data(*in, *p))) return st;
    const int route = sv->cfg.step_min_n > 0 && z.n >= sv->cfg.step_min_n ? 1 : 0;
    if (!route && (st = fits_fused(sv, z))) return st;
    if (!route && sv->ex.ants_per_warp == 32 && (z.ls == 2 || z.ls == 4)) return HAC_EUNSUPPORTED;   // step-major tours
    int q = 0;
    while (q < sv->cfg.max_slots && sv->slots[q].state != R_FREE) ++q;
    if (q == sv->cfg.max_slots) return HAC_EBUSY;
    const Region R = region_of(z);
    size_t off;
    if (!heap_alloc(sv, R.total, off)) return HAC_EBUSY;

    Slot &S = sv->slots[q];
    char *B = sv->heap + off;
    DevInst &D = sv->hi[q];
    std::memset(&D, 0, sizeof D);
    Arena A;
    bind_zero(D, z, A, B);
    bind_instance(D, *in, *p, z, 0, route ? sv->sex : sv->ex, A, B);
    std::vector<int2> rowmap(R.rows), slotmap(R.slots);
    for (int r = 0; r < R.rows; ++r) rowmap[r] = make_int2(0, r * ROWS_PER_BLOCK);
    for (int r = 0; r < R.slots; ++r) slotmap[r] = make_int2(0, r * SLOTS_PER_BLOCK);
    int2 *d_rowmap = (int2 *)(B + R.rowmap), *d_slotmap = (int2 *)(B + R.slotmap);
    cudaStream_t ps = sv->prep[sv->next_prep];
    auto undo = [&](int code) {
        heap_free(sv, off, R.total);
        return code;
    };
    if (cudaMemsetAsync(B, 0, R.zero_end, ps) != cudaSuccess) return undo(HAC_ECUDA);
    std::vector<Upload> ups;
    const size_t n = z.n, nnz = (size_t)z.nnz;
    if (z.kind == 0) ups.push_back(Upload{in->coords, (void *)D.xy, n * 8});
    else ups.push_back(Upload{in->cost, (void *)D.cost, n * n * 4});
    ups.push_back(Upload{in->h_rowptr, (void *)D.rowptr, (n + 1) * 4});
    if (nnz) {
        ups.push_back(Upload{in->h_col, (void *)D.col, nnz * 4});
        ups.push_back(Upload{in->h_val, (void *)D.val, nnz * (z.half ? 2 : 4)});
    }
    ups.push_back(Upload{rowmap.data(), d_rowmap, rowmap.size() * sizeof(int2)});
    ups.push_back(Upload{slotmap.data(), d_slotmap, slotmap.size() * sizeof(int2)});
    ups.push_back(Upload{&D, sv->d_inst + q, sizeof(DevInst)});
    if ((st = upload_staged(sv, ups, ps))) return undo(st);
    sv->next_prep = (sv->next_prep + 1) % PREP_STREAMS;
    sv->launches += launch_prep(sv->d_inst + q, &D, 1, d_rowmap, R.rows, d_slotmap, R.slots, sv->d_err, ps);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(S.ready, ps);
    if (e != cudaSuccess) { g_last_cuda = (int)e; return undo(HAC_ECUDA); }
    S.state = R_PREP;
    S.ticket = sv->next_ticket++;
    S.off = off;
    S.bytes = R.total;
    S.z = z;
    S.route = route;
    S.t = 0;
    sv->zs[q] = z;
    *ticket = S.ticket;
    return HAC_OK;
}

int hac_server_tick(hac_server *sv)
{
    if (!sv) return HAC_EINVAL;
    // at most two ticks in flight: wait for the one before the previous (which
    // also frees that tick's pinned order buffer)
    const int par = (int)(sv->ticks & 1);
    if (sv->tick_rec[par]) CK(cudaEventSynchronize(sv->tick_ev[par]));
    std::vector<int> members, smembers;
    for (int q = 0; q < sv->cfg.max_slots; ++q) {
        Slot &S = sv->slots[q];
        if (S.state == R_PREP) {
            cudaError_t e = cudaEventQuery(S.ready);
            if (e == cudaErrorNotReady) continue;
            CK(e);
            CK(cudaStreamWaitEvent(sv->stream, S.ready, 0));
            S.state = R_RUN;
        }
        if (S.state == R_RUN && S.t < S.z.iters) (S.route ? smembers : members).push_back(q);
    }
    if (!smembers.empty()) {
        int st = enqueue_step_route(sv, smembers, par);
        if (st) return st;
    }
    if (!members.empty()) {
        std::vector<FusedGroup> groups;
        std::vector<int32_t> order;
        int32_t *d_order = sv->d_order[par], *d_iters = sv->d_iters[par];
        int32_t *h_ord = sv->h_order[par], *h_it = sv->h_order[par] + sv->cfg.max_slots;
        const size_t cnt = members.size();
        const bool together = plan_groups(sv->zs, members, sv->ex.ants_per_warp, sv->ex.cluster_log2,
                                          sv->ex.fallback_list, groups, order) == HAC_OK;
        if (together) std::copy(order.begin(), order.end(), h_ord);
        else std::copy(members.begin(), members.end(), h_ord);
        for (size_t r = 0; r < cnt; ++r) h_it[r] = tick_iters(sv, sv->slots[h_ord[r]]);
        CK(cudaMemcpyAsync(d_order, h_ord, cnt * sizeof(int32_t), cudaMemcpyHostToDevice, sv->stream));
        CK(cudaMemcpyAsync(d_iters, h_it, cnt * sizeof(int32_t), cudaMemcpyHostToDevice, sv->stream));
        if (together) {
            int st = enqueue_groups(sv, groups, d_order, d_iters);
            if (st) return st;
        } else {
            // the members' shared-memory caps do not fit together: one launch each
            for (size_t r = 0; r < cnt; ++r) {
                std::vector<int> one{h_ord[r]};
                int st = plan_groups(sv->zs, one, sv->ex.ants_per_warp, sv->ex.cluster_log2,
                                     sv->ex.fallback_list, groups, order);
                if (st) return st;
                if ((st = enqueue_groups(sv, groups, d_order + r, d_iters + r))) return st;
            }
        }
        for (size_t r = 0; r < cnt; ++r) sv->slots[h_ord[r]].t += h_it[r];
    }
    if (!smembers.empty()) {
        CK(cudaEventRecord(sv->sjoin, sv->sstream));
        CK(cudaStreamWaitEvent(sv->stream, sv->sjoin, 0));
    }
    // stage the results of the requests that have reached their iteration count
    for (int q = 0; q < sv->cfg.max_slots; ++q) {
        Slot &S = sv->slots[q];
        if (S.state != R_RUN || S.t < S.z.iters) continue;
        const DevInst &D = sv->hi[q];
        CK(cudaMemcpyAsync(S.h_tour, D.gb_tour, (size_t)S.z.n * 4, cudaMemcpyDeviceToHost, sv->stream));
        CK(cudaMemcpyAsync(S.h_st, D.st, sizeof(InstState), cudaMemcpyDeviceToHost, sv->stream));
        CK(cudaEventRecord(S.done, sv->stream));
        S.state = R_RETIRE;
    }
    CK(cudaEventRecord(sv->tick_ev[par], sv->stream));
    sv->tick_rec[par] = true;
    sv->ticks++;
    CK(cudaGetLastError());
    return HAC_OK;
}

int hac_server_poll(hac_server *sv, uint64_t ticket, int32_t *tour, double *len)
{
    if (!sv || !ticket) return HAC_EINVAL;
    for (int q = 0; q < sv->cfg.max_slots; ++q) {
        Slot &S = sv->slots[q];
        if (S.state == R_FREE || S.ticket != ticket) continue;
        if (S.state != R_RETIRE) return HAC_EBUSY;
        cudaError_t e = cudaEventQuery(S.done);
        if (e == cudaErrorNotReady) return HAC_EBUSY;
        CK(e);
        if (tour) std::memcpy(tour, S.h_tour, (size_t)S.z.n * 4);
        if (len) *len = S.h_st->L_gb;
        heap_free(sv, S.off, S.bytes);
        S.state = R_FREE;
        S.ticket = 0;
        return HAC_OK;
    }
    return HAC_EINVAL;
}

int hac_server_stats(hac_server *sv, int32_t *resident, int32_t *finished, size_t *free_bytes,
                     int32_t *device_error)
{
    if (!sv) return HAC_EINVAL;
    int res = 0, fin = 0;
    for (const Slot &S : sv->slots) {
        if (S.state == R_FREE) continue;
        ++res;
        if (S.state == R_RETIRE && cudaEventQuery(S.done) == cudaSuccess) ++fin;
    }
    if (resident) *resident = res;
    if (finished) *finished = fin;
    if (free_bytes) *free_bytes = free_total(sv);
    if (device_error) {
        for (int g = 0; g < PREP_STREAMS; ++g) CK(cudaStreamSynchronize(sv->prep[g]));
        CK(cudaStreamSynchronize(sv->stream));
        int err = 0;
        CK(cudaMemcpy(&err, sv->d_err, sizeof err, cudaMemcpyDeviceToHost));
        *device_error = err;
    }
    return HAC_OK;
}

int hac_server_launches(hac_server *sv, int64_t *launches)
{
    if (!sv || !launches) return HAC_EINVAL;
    *launches = sv->launches;
    return HAC_OK;
}

int hac_server_destroy(hac_server *sv)
{
    if (!sv) return HAC_EINVAL;
    for (int g = 0; g < PREP_STREAMS; ++g) if (sv->prep[g]) cudaStreamSynchronize(sv->prep[g]);
    cudaStreamSynchronize(sv->stream);
    for (Slot &S : sv->slots) {
        if (S.ready) cudaEventDestroy(S.ready);
        if (S.done) cudaEventDestroy(S.done);
    }
    for (int g = 0; g < 2; ++g) if (sv->tick_ev[g]) cudaEventDestroy(sv->tick_ev[g]);
    if (sv->sstream) { cudaStreamSynchronize(sv->sstream); cudaStreamDestroy(sv->sstream); }
    if (sv->sfork) cudaEventDestroy(sv->sfork);
    if (sv->sjoin) cudaEventDestroy(sv->sjoin);
    if (sv->h_sinst[0]) cudaFreeHost(sv->h_sinst[0]);
    for (int g = 0; g < PREP_STREAMS; ++g) if (sv->prep[g]) cudaStreamDestroy(sv->prep[g]);
    for (const RingEntry &r : sv->ring_q) cudaEventDestroy(r.ev);
    for (cudaEvent_t ev : sv->ring_ev) cudaEventDestroy(ev);
    if (sv->ring) cudaFreeHost(sv->ring);
    if (sv->pinned) cudaFreeHost(sv->pinned);
    delete sv;
    return HAC_OK;
}

}  // extern "C"
