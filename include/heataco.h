/*
 * heataco.h -- C ABI of the GB300 (sm_103a) HeatACO decoder.
 *
 * HeatACO (arXiv 2601.19041) decodes a fixed edge-confidence heatmap H into a
 * TSP / ATSP tour with a Max-Min Ant System whose construction weight is
 * tau^alpha * eta^beta * e^kappa (Sec. III-A, eq. transition).  The decoding
 * problem it solves is g(H, D) -> tour (Sec. II-B): distances (coordinates or
 * a cost matrix) and a sparse heatmap in, a feasible tour and its length out,
 * following Algorithm 1 (the MMAS loop) and Algorithm 2 (one ant's tour).
 *
 * Conventions used by every entry point:
 *   - All functions return an int status: HAC_OK (0) or a negative HAC_E* code.
 *     No function aborts, throws or exits; hac_strerror() names a code.
 *   - The caller passes a device workspace of at least the size reported by
 *     the matching *_workspace_size call (any allocator: cudaMalloc, a
 *     PyTorch tensor, a pool).  The workspace must stay valid, and must not be
 *     used by anyone else, until the handle that was created on it is
 *     destroyed.  The only device allocation the library ever makes is the
 *     one-shot calls' (hac_solve, hac_solve_batch) when they are given a NULL
 *     workspace: then they take one from the stream-ordered pool
 *     (cudaMallocAsync on `stream`) and return it before they return.  The
 *     library keeps host memory for its handles only.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All
 *     device work of a handle is issued on the stream given at its creation.
 *   - Input pointers are host pointers unless `inputs_on_device` is 1, in which
 *     case they are device pointers that must stay valid and unchanged until
 *     the handle is destroyed.  Outputs are caller-owned host buffers.
 *   - Tours are permutations of 0..n-1 in visiting order, in the orientation
 *     and rotation the search produced them.  Lengths are FP64 (eq. tour_length).
 *   - Results are a deterministic function of the inputs and parameters: the
 *     random numbers come from a counter-based Philox4x32-10 keyed by the
 *     instance's seed and (iteration, ant, step), so an instance decodes to the
 *     same tour alone, in any batch and in any serving mix.
 */
#ifndef HEATACO_H
#define HEATACO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum hac_status {
    HAC_OK = 0,
    HAC_EINVAL = -1,        /* invalid argument or malformed instance */
    HAC_ENOMEM = -2,        /* workspace too small, or host allocation failed */
    HAC_ECUDA = -3,         /* a CUDA runtime call failed (see hac_last_cuda_error) */
    HAC_ETIMEOUT = -4,      /* a bounded device-side wait gave up */
    HAC_EUNSUPPORTED = -5,  /* combination not supported (e.g. 3-opt on an ATSP) */
    HAC_EBUSY = -6          /* serving: request not finished yet / no slot free */
};

#define HAC_KMAX 32         /* candidate-list size limit (one 8-lane warp segment) */
#define HAC_NMAX (1 << 20)  /* node-count limit of one instance */
#define HAC_MMAX 1024       /* ants per instance */

/* One decode problem (Sec. II-A, II-B).
 *   kind 0: symmetric Euclidean; d_ij = sqrt((x_j-x_i)^2 + (y_j-y_i)^2) in FP64
 *           of the FP32 coordinates `coords` (n*2, x0 y0 x1 y1 ...).
 *   kind 1: explicit costs `cost` (n*n FP32 row-major, c_ij = cost[i*n+j]);
 *           directed (ATSP): the pheromone deposit is one-directional.
 * The heatmap H (eq. heatmap_def) is CSR: h_rowptr (n+1 int32, h_rowptr[0]=0,
 * h_rowptr[n]=h_nnz), h_col (h_nnz int32, strictly increasing within a row, no
 * i==j), h_val (h_nnz values in [0,1], FP32 when h_dtype==0, IEEE binary16
 * when h_dtype==1).  h_nnz is passed explicitly so that sizing never has to
 * read device memory; a mismatch with h_rowptr[n] is HAC_EINVAL.
 * symmetrize=1 makes the decoder use (H + H^T)/2 (Sec. II-B). */
typedef struct {
    int32_t n;
    int32_t kind;
    const float *coords;
    const float *cost;
    const int32_t *h_rowptr;
    const int32_t *h_col;
    const void *h_val;
    int64_t h_nnz;
    int32_t h_dtype;
    int32_t symmetrize;
} hac_instance;

/* Decoder parameters (Sec. IV-D).  hac_params_default() fills the paper's
 * values: m=32, k=20, I=5000, alpha=1, beta=2, rho=0.8 (0.2 for kind 1),
 * theta_h=1e-4, eps=1e-9, c_cap=0.5, q_level=0.90, p_best=0.05, d*=2 (1 for
 * kind 1), no local search, baseline over C_i, ls_k=20.
 *   logw_clip       cap of the log-weight kappa*ln(e) (end of Sec. III-C; the
 *                   paper says "a large constant"; default 30).
 *   local_search    0 none; 1 first-improvement 2-opt with geometric
 *                   neighbour lists and don't-look bits (Sec. III-D) on the
 *                   iteration-best tour and on T_NN; 2 the same 2-opt on
 *                   every ant's tour right after its construction (the
 *                   local search of Algorithm 1) and on T_NN; 3 and 4 the
 *                   same with first-improvement 3-opt (sequential exchanges
 *                   of up to three edges, neighbour lists, don't-look bits)
 *                   instead of 2-opt; tau_min = tau_max/(2n) for all.
 *                   With kind 1 (ATSP), modes 1 and 2 run the directed 2-opt
 *                   (the 2-opt move that reverses a path, its gain counting
 *                   the path's backward minus forward arc costs; the paper's
 *                   Jonker-Volgenant based 2-opt) and modes 3 and 4 are
 *                   HAC_EUNSUPPORTED.  With kind 0 local search needs
 *                   |x|, |y| <= 1e18.
 *                   Modes 2 and 4 are not available with 32 ants per warp
 *                   (HAC_EUNSUPPORTED).
 *   baseline_scope  0: order statistic b_i over the candidates C_i; 1: over all
 *                   heatmap entries of row i (eq. background defines c on C_i
 *                   but speaks of "row i"; both readings are offered).
 *   schedule        0 (default): T+ = the iteration-best tour every iteration;
 *                   1: the MMAS machinery of Sec. III-B and Algorithm 1 --
 *                   restart-best tour T_rb, elite T+ = T_rb every u_gb
 *                   iterations (u_gb = 25, 5, 3, 2, 1 after 0, 25, 75, 125,
 *                   250 iterations since the last restart), and every 100
 *                   iterations a restart (tau <- tau_max, T_rb cleared, T_gb
 *                   kept) when T_rb has not improved for more than 250
 *                   iterations and the branching factor (band 0.05, per node,
 *                   divided by d*) is below 1 + 1e-5.
 *   kappa_mode      scale of the evidence factor: 0 (default) eq. kappa,
 *                   kappa = c_cap*alpha*ln(R)/q90; the two ablation variants
 *                   of Sec. V-D: 1 "fixed kappa = 1"; 2 "no cap", the cap
 *                   factor c_cap dropped from eq. kappa (alpha*ln(R)/q90).
 *   seed            key of the instance's Philox stream. */
typedef struct {
    int32_t m, k, iterations;
    double alpha, beta, rho;
    double theta_h, eps, c_cap, q_level, p_best, logw_clip;
    int32_t degree_target;
    int32_t local_search;
    int32_t baseline_scope;
    int32_t ls_k;
    int32_t schedule;
    int32_t kappa_mode;
    uint64_t seed;
} hac_params;

/* Execution options of a batch (none of them changes any result). */
typedef struct {
    int32_t ants_per_warp;    /* 1, 2 or 4 ants share one warp (8-lane segments), 16 (one ant per
                                 lane pair) or 32 (one ant per lane); 0 = auto (fused: per
                                 instance, 4 on one CTA when its table, visited masks and
                                 coordinates fit in one SM's shared memory, else 2 on a cluster) */
    int32_t warps_per_block;  /* construction block size in warps; 0 = auto */
    int32_t use_graph;        /* 1: capture the iteration loop (per-step kernels: 10 iterations
                                 per graph; fused: the group launches) in a CUDA
                                 graph, replayed; needs a non-NULL stream */
    int32_t fused;            /* 1: persistent fused construct+update kernel; 0: per-step launches */
    int32_t fallback_list;    /* 32: look up the 32 nearest nodes (key order) before scanning; 0: scan only */
    int32_t profile;          /* 1: bracket every kernel group with CUDA events (no graphs) */
    int32_t cluster_log2;     /* fused kernel: at least 2^cluster_log2 CTAs per instance (0 = fewest that fit) */
    int32_t parts;            /* per-step kernels: the instances are split into this many contiguous
                                 parts of about equal work, each iterated on a stream of its own, so
                                 one part's local search overlaps another part's construction
                                 (0 or 1: one part on the batch's stream; at most 64) */
} hac_exec;

int hac_params_default(hac_params *p, int32_t kind);
int hac_exec_default(hac_exec *e);
const char *hac_strerror(int status);
/* The last CUDA error seen by the calling thread (cudaError_t as int, 0 if none). */
int hac_last_cuda_error(void);
int hac_version(void);

/* ------------------------------------------------------------------ batches
 * A batch is `count` independent instances decoded together on one GPU: each
 * instance has its own parameters (m, k, iterations, seed, ...), pheromone and
 * best-tour state, all resident in the workspace.  The preparation steps of
 * Algorithm 1 (candidate lists of Sec. III-A, evidence and kappa of Sec. III-C,
 * T_NN and the bounds of eq. tau_init / tau_min_nols) run in hac_batch_create;
 * its search loop (construction by Algorithm 2, iteration best, global best
 * with recomputed bounds, bounded evaporation/deposit of eq. pheromone_update)
 * runs in hac_batch_iterate. */
typedef struct hac_batch hac_batch;

/* Bytes of device workspace needed by hac_batch_create for these instances.
 * Host-only; validates sizes and parameters (not the heatmap contents). */
int hac_batch_workspace_size(const hac_instance *ins, const hac_params *ps, int32_t count,
                             int32_t inputs_on_device, size_t *bytes);

/* Creates the handle, copies the inputs into the workspace (host->device
 * copies when inputs_on_device==0), validates the heatmap on the device and
 * enqueues the preparation.  Asynchronous on `stream`; errors found by the
 * device validation are reported by the next synchronising call.
 * exec may be NULL (defaults).  On failure *out is NULL. */
int hac_batch_create(const hac_instance *ins, const hac_params *ps, int32_t count,
                     int32_t inputs_on_device, void *workspace, size_t ws_bytes,
                     const hac_exec *exec, void *stream, hac_batch **out);

/* Enqueues `iters` more iterations of every instance that has not reached its
 * own iteration budget (instances stop at their budget).  Asynchronous. */
int hac_batch_iterate(hac_batch *bt, int32_t iters);

/* Enqueues all remaining iterations.  Asynchronous. */
int hac_batch_run(hac_batch *bt);

/* Synchronises the stream and reports the first device-side error (bad
 * heatmap, timeout) as a status. */
int hac_batch_sync(hac_batch *bt);

/* Fields readable with hac_batch_read (sizes in elements):
 *   CAND   int32  n*k_pad   candidate list C_i, -1 on padding, ascending (d, j)
 *   CDIST  f64    n*k_pad   d_ij of each candidate slot
 *   CONF   f64    n*k_pad   thresholded confidence c_ij (eq. confidence)
 *   BASE   f64    n         degree baseline b_i (eq. background)
 *   EVID   f64    n*k_pad   evidence factor e_ij (eq. evidence)
 *   W      f32    n*k_pad   static weight fl32(eta^beta * e^kappa)
 *   TAU    f32    n*k_pad   pheromone
 *   CHOICE f32    n*k_pad   fl32(tau^alpha * W), the numerator of eq. transition
 *   NN_TOUR int32 n         T_NN
 *   GB_TOUR int32 n         T_gb
 *   IB_TOUR int32 n         last iteration-best tour (after local search)
 *   TOURS  int32  m*n       the m tours of the last iteration
 *   LENS   f64    m         their lengths
 *   SCALARS f64   21        q90, Rhat, kappa, p_x, L_nn, tau_max64, tau_min64,
 *                           tau_max, tau_min, L_gb, L_ib, n_lambda, t, ib_ant,
 *                           n_fallback, k_pad, L_rb, n_restarts, t_restart, u_gb,
 *                           edges_per_n (|{(i,j): h_ij > theta_h}| / (2n), the
 *                           candidate density diagnostic Edges/n of Sec. VI-A)
 *   NBR    int32  n*ls_k    geometric 2-opt neighbour lists
 *   TRACE  f64    5*I       per iteration: ib ant, L_ib, L_gb, L_rb (+inf when
 *                           cleared), code (1: T_rb deposited, 2: restart)
 *   FBL    int32  n*32      nearest-unvisited lookup list of node i: the nodes
 *                           u != i (not in C_i when every candidate's choice
 *                           value stays positive) by (FP32 key, u), -1 past
 *                           the end; HAC_EINVAL when the exec has no lists
 *   FBL2   uint16 n*256     the next 256 nodes of the same order (ranks
 *                           32..287), 0xffff past the end; HAC_EINVAL when
 *                           absent (no lists, or n > 65535)
 * The call synchronises the stream. */
enum hac_field {
    HAC_F_CAND = 1, HAC_F_CDIST, HAC_F_CONF, HAC_F_BASE, HAC_F_EVID, HAC_F_W, HAC_F_TAU,
    HAC_F_CHOICE, HAC_F_NN_TOUR, HAC_F_GB_TOUR, HAC_F_IB_TOUR, HAC_F_TOURS, HAC_F_LENS,
    HAC_F_SCALARS, HAC_F_NBR, HAC_F_TRACE, HAC_F_FBL, HAC_F_FBL2
};
int hac_batch_read(hac_batch *bt, int32_t b, int32_t field, void *host_dst, size_t bytes);

/* Copies every instance's best tour T_gb (best_tours[b]: n_b int32) and length
 * L_gb (best_lens[b]) to host buffers; synchronises.  Either array may be NULL. */
int hac_batch_results(hac_batch *bt, int32_t *const *best_tours, double *best_lens);

/* Total ant-steps (sum of m*n*iterations done) and fallback steps so far. */
int hac_batch_counters(hac_batch *bt, int64_t *ant_steps, int64_t *fallback_steps);

/* Kernel launches this handle has issued (graph replays count the kernels
 * they contain).  Host-side count; does not synchronise. */
int hac_batch_launches(hac_batch *bt, int64_t *launches);

/* With exec->profile==1: device time (ms, CUDA events on the handle's stream)
 * and launch count of one kernel group since creation:
 *   0 construction (Algorithm 2), 1 iteration tail (iteration best, 2-opt,
 *   global best, pheromone update), 2 preparation, 3 fused iterations
 *   (construction and tail in the persistent cluster kernel).  Synchronises. */
int hac_batch_kernel_time(hac_batch *bt, int32_t group, double *ms, int64_t *launches);

/* Autotuner: decodes the batch's first trial_iters + 1 iterations once per
 * candidate execution layout and returns in *best the layout whose last
 * trial_iters iterations took the least device time (CUDA events on
 * `stream`), with use_graph = 1, and that time per iteration in *ms_per_iter
 * (may be NULL).  Candidates: the fused cluster kernel with 2, 4, 16 or 32
 * ants per warp, smallest cluster 1, 2 or 4 CTAs, with and without the
 * 32-entry nearest-unvisited lookup list; the per-step kernels with 1, 2, 4
 * or 16 ants per warp and 4 or 8 warps per block.  No layout changes a result, so the choice
 * is a matter of speed only; the method's parameters (m, k, ...) are never
 * changed.  Uses `workspace` (hac_batch_workspace_size bytes) for each trial
 * in turn; synchronises `stream`.  Candidates an instance does not support
 * are skipped. */
int hac_batch_autotune(const hac_instance *ins, const hac_params *ps, int32_t count,
                       int32_t inputs_on_device, void *workspace, size_t ws_bytes, int32_t trial_iters,
                       void *stream, hac_exec *best, double *ms_per_iter);

/* Releases the host handle; the workspace can be reused afterwards.  Does not
 * synchronise: the caller must not reuse the workspace before the stream has
 * drained. */
int hac_batch_destroy(hac_batch *bt);

/* ------------------------------------------------------------------ one-shot
 * Decode one instance / a batch end to end: the decoding problem g(H, D) ->
 * tour of Sec. II-B, by Algorithm 1 (REQUIRE: the distances D, the heatmap H
 * and the parameters m, I, k, alpha, beta, rho, c_cap of hac_params; ENSURE:
 * the global-best tour T_gb), each instance run for its own p.iterations.
 * Create, run, results and destroy in one call; synchronises `stream`.
 *
 *   workspace, ws_bytes  device memory of at least hac_batch_workspace_size
 *                   bytes, or NULL: the call then allocates that much from the
 *                   stream-ordered pool (cudaMallocAsync on `stream`) and
 *                   frees it before it returns (HAC_ENOMEM if the pool cannot
 *                   supply it).  With a NULL workspace nothing is required of
 *                   the caller but host buffers, so a plain C program can
 *                   decode host inputs (inputs_on_device = 0) in one call.
 *   best_tour(s)    caller-owned host buffers of n (n_b) int32: T_gb
 *   best_len(s)     L_gb (eq. tour_length), FP64
 *   statuses        count entries, may be NULL: the call's status per instance
 *   stats           1 (count) entries, may be NULL: per-instance counters
 *                   (hac_stats), filled on success
 *   exec            execution layout (hac_solve_batch; NULL = defaults)
 */
typedef struct {
    int32_t iterations;      /* MMAS iterations run (the instance's p.iterations) */
    int32_t restarts;        /* pheromone restarts (schedule = 1) */
    int64_t ant_steps;       /* sum over the iterations of m * n construction steps */
    int64_t fallback_steps;  /* steps that took the nearest-unvisited rule (Alg. 2) */
    double kappa;            /* the evidence scale used (eq. kappa or its kappa_mode variant) */
    double edges_per_n;      /* candidate density |{h_ij > theta_h}| / (2n) (Sec. VI-A) */
    double L_nn;             /* length of the initial tour T_NN (Alg. 1) */
    double seconds;          /* wall time of the whole call (the same for every instance) */
} hac_stats;

int hac_solve(const hac_instance *in, const hac_params *p, int32_t inputs_on_device,
              void *workspace, size_t ws_bytes, int32_t *best_tour, double *best_len,
              hac_stats *stats, void *stream);
int hac_solve_batch(const hac_instance *ins, const hac_params *ps, int32_t count,
                    int32_t inputs_on_device, void *workspace, size_t ws_bytes,
                    const hac_exec *exec, int32_t *const *best_tours, double *best_lens,
                    int32_t *statuses, hac_stats *stats, void *stream);

/* ------------------------------------------------------------------ serving
 * Continuous batching of decode requests (the paper has no serving layer;
 * this is how the decoder of Algorithm 1 is offered to a request stream).
 * A server owns one caller-provided device workspace; each admitted request
 * takes a region of it (hac_server_request_bytes) that holds its whole state,
 * pheromone and T_gb included, from admission until its result is polled.
 * Requests that arrive while others run are admitted whenever a slot and a
 * region are free, and all admitted requests advance together, each from its
 * own iteration, in the persistent cluster kernel (hac_exec.fused).  A request
 * returns the same tour and length as hac_solve on the same instance and
 * parameters, alone or in any mix.  Inputs are host pointers; the server
 * copies them (into its pinned upload ring, or for a request larger than the
 * ring straight to the device) during hac_server_submit, so the caller may
 * reuse them at once.
 * A server is not thread-safe: call it from one host thread at a time.
 *
 *   max_slots       requests resident at once (1..4096)
 *   iters_per_tick  MMAS iterations a tick runs for every running request
 *   max_n           largest n accepted (3..65534); sizes the pinned staging
 *   steps_per_tick  0, or a per-tick budget of construction steps per ant: a
 *                   request of n nodes then runs max(1, min(iters_per_tick,
 *                   steps_per_tick / n)) iterations a tick, so that small and
 *                   large requests take about the same time per tick
 *   step_min_n      0, or the n from which requests run on the per-step
 *                   kernels (rows through L2, ants of many instances on each
 *                   SM) instead of the cluster kernel (candidate table in
 *                   the shared memory of 2^c SMs, which leaves few ants per
 *                   SM for large n); those requests all run the smallest
 *                   budget among them each tick
 *   step_ants_per_warp, step_warps_per_block
 *                   layout of that route (0 -> 1 and 8; 1, 2, 4 or 16 and 1..8)
 *   exec            ants_per_warp (0 -> 4; 2, 4, 16 or 32), cluster_log2 (the
 *                   smallest cluster size, log2), fallback_list (0 or 32);
 *                   fused is implied, the other fields are ignored */
typedef struct {
    int32_t max_slots;
    int32_t iters_per_tick;
    int32_t max_n;
    int32_t steps_per_tick;
    int32_t step_min_n;
    int32_t step_ants_per_warp;
    int32_t step_warps_per_block;
    hac_exec exec;
} hac_server_cfg;

typedef struct hac_server hac_server;

/* Device bytes one request takes from a server's workspace. */
int hac_server_request_bytes(const hac_instance *in, const hac_params *p, size_t *bytes);

/* Creates a server on `workspace` (device memory, ws_bytes; header of about
 * max_slots * 1 KB, the rest is the request heap) and `stream`.  Allocates
 * pinned host staging of about max_slots * (4 * max_n + 512) bytes (and,
 * with step_min_n > 0, per-tick work tables of about max_slots * (16 KB +
 * max_n / 4) bytes, twice, on both sides), one side stream for the per-step
 * route, four preparation streams and a pinned upload ring of 64 MB.
 * HAC_ENOMEM if the workspace cannot hold the header and a minimal heap. */
int hac_server_create(const hac_server_cfg *cfg, void *workspace, size_t ws_bytes, void *stream,
                      hac_server **out);

/* Admits a request: checks it (as hac_batch_create does for host inputs),
 * takes a free slot and the first heap region that fits, uploads the inputs
 * and enqueues the preparation (Sec. III-A: candidate lists, evidence, kappa,
 * W; T_NN and the bounds) on the next preparation stream.  Does not wait for
 * the device unless the upload ring is full.  Returns a ticket > 0.
 * HAC_EBUSY when no slot or no region is free (retry after polling finished
 * requests); HAC_EINVAL for n > max_n or a malformed request;
 * HAC_EUNSUPPORTED when a request routed to the cluster kernel does not fit
 * it. */
int hac_server_submit(hac_server *sv, const hac_instance *in, const hac_params *p, uint64_t *ticket);

/* Runs the tick's iterations of every running request (requests
 * whose preparation has finished join here) and stages the results of the
 * requests that reach their iteration count.  Asynchronous; keeps at most two
 * ticks in flight (waits for the tick before the previous one). */
int hac_server_tick(hac_server *sv);

/* Result of a request: T_gb (n int32, may be NULL) and L_gb (may be NULL).
 * HAC_EBUSY while the request is still preparing, running or staging;
 * HAC_EINVAL for an unknown ticket.  On HAC_OK the slot and region are freed
 * and the ticket is no longer valid.  Does not block. */
int hac_server_poll(hac_server *sv, uint64_t ticket, int32_t *tour, double *len);

/* Requests resident (admitted, not yet polled), finished requests waiting to
 * be polled, and free heap bytes.  With device_error non-NULL the call also
 * synchronises and reports the first device-side error of the preparation
 * kernels (0 if none).  Any pointer may be NULL. */
int hac_server_stats(hac_server *sv, int32_t *resident, int32_t *finished, size_t *free_bytes,
                     int32_t *device_error);

/* Kernel launches issued so far (preparation and cluster kernels). */
int hac_server_launches(hac_server *sv, int64_t *launches);

/* Synchronises the server's streams and releases its host resources; the
 * workspace may be reused afterwards.  Unpolled results are dropped. */
int hac_server_destroy(hac_server *sv);

/* ------------------------------------------------------------------ no allocation
 * Decode one instance without any device allocation, for callers that cannot
 * call cudaMalloc: a host application whose allocator or memory budget owns
 * the free device memory, or a serving loop where an allocation could
 * synchronise the device or fail under memory pressure.  (The paper has no
 * counterpart; this is a property of the library, not of the method.)
 *
 * Same result as hac_solve on the same arguments.  The scratch is a fixed
 * array of HAC_NOALLOC_MAX_BYTES compiled into the library: every GPU that
 * loads the library holds it until the process exits.  An instance whose
 * workspace (hac_batch_workspace_size) exceeds it is rejected with
 * HAC_ENOMEM and nothing runs.  The call allocates no device memory (it uses
 * no CUDA graph and no events); it uses a little host heap for its transient
 * handle.  Inputs follow inputs_on_device as in hac_solve; best_tour (n
 * int32) and best_len are host buffers.  The call synchronises `stream`.
 *
 * The first call on a device looks up the array's device address (with that
 * device current), so make that first call before any stream capture.  All
 * calls on a device share the one array and it keeps the previous call's
 * contents; each call clears what must start at zero.  Calls that overlap on
 * the GPU (other host threads, other streams) race on the array: serialise
 * them. */
#define HAC_NOALLOC_MAX_BYTES (16u << 20)
int hac_solve_noalloc(const hac_instance *in, const hac_params *p, int32_t inputs_on_device,
                      int32_t *best_tour, double *best_len, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HEATACO_H */
