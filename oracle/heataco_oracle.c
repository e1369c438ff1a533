/*
 * HeatACO oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential CPU restatement of the heatmap-guided Max-Min Ant
 * System of arXiv 2601.19041 (Sec. III, Algorithm 1 and Algorithm 2).  Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it; the library never does.  It shares no code with the CUDA path.
 *
 * Every floating-point step below is written as a sequence of single IEEE
 * operations (build with -ffp-contract=off, no fast-math), so the result is a
 * fixed function of the inputs.  Where the paper leaves an arithmetic or
 * ordering detail open, the reading used here is stated at the point of use.
 *
 * Pins (what this file is checked against, tests/test_oracle_*.py):
 *   Philox4x32-10      published known-answer vectors (Salmon et al., SC'11)
 *   orc_exp / orc_ln   libm and mpmath to within 2 ulp
 *   candidate lists    k-nearest-neighbour lists (empty / full heatmap)
 *   evidence, kappa    hand-worked rows; kappa*q90 = c_cap*alpha*ln(R) (Sec. III-C)
 *   q90                numpy's linear (type 7) quantile
 *   roulette           chi-square against w/sum(w); brute force on tiny vectors
 *   decode             brute-force optima (n <= 9), closed-form optima (circle,
 *                      grid) under a heatmap concentrated on the optimal tour
 *   2-opt              no improving neighbour-list move remains; never lengthens
 *   MMAS schedule      u_gb tightens from 25 to 1 (Sec. III-B); branching factor
 *                      on pheromone matrices of known form (all equal: k_eff/d*;
 *                      converged: 1); restarts only at checks, T_gb kept
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ types */

typedef struct {
    int32_t n;
    int32_t kind;            /* 0: Euclidean from coords, 1: explicit cost c_ij */
    const float *coords;     /* n*2 */
    const float *cost;       /* n*n row-major */
    const int32_t *rowptr;   /* n+1 */
    const int32_t *col;      /* nnz, strictly increasing within a row */
    const void *val;         /* nnz values, float32 or IEEE binary16 */
    int32_t val_is_half;
    int32_t symmetrize;      /* 1: h = (H + H^T)/2 (Sec. II-B) */
} orc_instance;

typedef struct {
    int32_t m, k, iterations;
    double alpha, beta, rho;
    double theta_h, eps, c_cap, q_level, p_best, logw_clip;
    int32_t degree_target;   /* d* of Sec. III-C: 2 symmetric, 1 ATSP */
    int32_t local_search;    /* 0 none; 2-opt: 1 on the iteration-best tour, 2 on every ant's tour;
                                3-opt: 3 on the iteration-best tour, 4 on every ant's tour */
    int32_t baseline_scope;  /* 0 order statistic over C_i, 1 over the whole heatmap row */
    int32_t ls_k;            /* geometric neighbour-list size of the 2-opt */
    int32_t schedule;        /* 0: T+ = T_ib always; 1: MMAS u_gb schedule and restarts */
    int32_t kappa_mode;      /* 0: eq. (kappa); 1: fixed kappa = 1; 2: eq. (kappa) without c_cap */
    uint64_t seed;
} orc_params;

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2 };

#define ORC_KMAX 32
#define ORC_DFLOOR 1e-9      /* eta = 1/max(d, 1e-9): guard for coincident points */
#define ORC_LS_GAIN 1e-10    /* a 2-opt move is taken when its gain exceeds this */

/* --------------------------------------------------- Philox4x32-10 (SC'11) */

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof c);
}

/* Draw s of ant a in iteration t (all 0-based): word (s mod 4) of the Philox
 * block with counter (floor(s/4), a, t, 0) under key (lo32(seed), hi32(seed)).
 * The paper only says each ant has its own generator (Sec. IV-D). */
uint32_t orc_draw(uint64_t seed, uint32_t t, uint32_t a, uint32_t s)
{
    uint32_t ctr[4] = {s >> 2, a, t, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[s & 3u];
}

/* u in [0,1): the top 24 bits of a draw scaled by 2^-24 (exact in float). */
static float unif24(uint32_t x) { return (float)(x >> 8) * 0x1p-24f; }

/* ----------------------------------------------- deterministic exp and ln */
/* Own FP64 routines from +,-,*,/ only, so that the CUDA path can reproduce
 * them bit for bit.  exp: Cody-Waite reduction x = k ln2 + r (two-part ln2)
 * and the Taylor series of e^r to degree 13 in Horner form, then the exact
 * scaling by 2^k.  ln: x = m 2^e with m in [sqrt(1/2), sqrt(2)], then
 * ln m = 2 atanh(s), s = (m-1)/(m+1), by its odd series to s^23. */

static const double LN2_HI = 0x1.62e42fefa2000p-1;   /* ln 2 to 40 bits */
static const double LN2_LO = 0x1.9ef35793c7673p-41;  /* ln 2 - LN2_HI   */
static const double INV_LN2 = 0x1.71547652b82fep+0;
static const double SQRT2 = 0x1.6a09e667f3bcdp+0;

static const double INV_FACT[14] = {   /* 1/i!, i = 0..13, rounded to double */
    1.0, 1.0, 0x1.0000000000000p-1, 0x1.5555555555555p-3, 0x1.5555555555555p-5,
    0x1.1111111111111p-7, 0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13,
    0x1.a01a01a01a01ap-16, 0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22,
    0x1.ae64567f544e4p-26, 0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};

static const double INV_ODD[12] = {    /* 1/(2j+1), j = 0..11 */
    1.0, 0x1.5555555555555p-2, 0x1.999999999999ap-3, 0x1.2492492492492p-3,
    0x1.c71c71c71c71cp-4, 0x1.745d1745d1746p-4, 0x1.3b13b13b13b14p-4,
    0x1.1111111111111p-4, 0x1.e1e1e1e1e1e1ep-5, 0x1.af286bca1af28p-5,
    0x1.8618618618618p-5, 0x1.642c8590b2164p-5};

static double pow2i(int k)   /* 2^k for -1022 <= k <= 1023, exact */
{
    uint64_t bits = (uint64_t)(k + 1023) << 52;
    double r;
    memcpy(&r, &bits, sizeof r);
    return r;
}

double orc_exp(double x)
{
    if (x != x) return x;
    if (x > 709.0) return INFINITY;
    if (x < -708.0) return 0.0;
    double kd = floor(x * INV_LN2 + 0.5);
    double r = (x - kd * LN2_HI) - kd * LN2_LO;
    double p = INV_FACT[13];
    for (int i = 12; i >= 0; --i) p = p * r + INV_FACT[i];
    return p * pow2i((int)kd);
}

double orc_ln(double x)
{
    if (!(x > 0.0)) return x == 0.0 ? -INFINITY : NAN;
    if (isinf(x)) return x;
    uint64_t bits;
    memcpy(&bits, &x, sizeof bits);
    int e = (int)((bits >> 52) & 0x7ff);
    if (e == 0) {                      /* subnormal: rescale by 2^54 first */
        double y = x * 0x1p54;
        memcpy(&bits, &y, sizeof bits);
        e = (int)((bits >> 52) & 0x7ff) - 54;
    }
    e -= 1023;
    uint64_t mb = (bits & 0x000fffffffffffffull) | 0x3ff0000000000000ull;
    double m;
    memcpy(&m, &mb, sizeof m);         /* m in [1, 2) */
    if (m > SQRT2) { m = m * 0.5; e += 1; }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double P = INV_ODD[11];
    for (int j = 10; j >= 1; --j) P = P * z + INV_ODD[j];
    double lnm = 2.0 * (s + s * (z * P));
    double ed = (double)e;
    return (ed * LN2_LO + lnm) + ed * LN2_HI;
}

/* --------------------------------------------------------- instance access */

static double half_bits_to_double(uint16_t h)
{
    int sgn = (h >> 15) & 1, ex = (h >> 10) & 0x1f, man = h & 0x3ff;
    double v;
    if (ex == 0) v = ldexp((double)man, -24);
    else if (ex == 31) v = man ? NAN : INFINITY;
    else v = ldexp((double)(man | 0x400), ex - 25);
    return sgn ? -v : v;
}

static double raw_val(const orc_instance *in, int64_t p)
{
    if (in->val_is_half) return half_bits_to_double(((const uint16_t *)in->val)[p]);
    return (double)((const float *)in->val)[p];
}

/* H_ij from the CSR rows (zero when absent). */
static double raw_heat(const orc_instance *in, int i, int j)
{
    int lo = in->rowptr[i], hi = in->rowptr[i + 1] - 1;
    while (lo <= hi) {
        int mid = lo + (hi - lo) / 2;
        int c = in->col[mid];
        if (c == j) return raw_val(in, mid);
        if (c < j) lo = mid + 1; else hi = mid - 1;
    }
    return 0.0;
}

/* h_ij as consumed by the decoder (Sec. II-B): (H_ij + H_ji)/2 when symmetrised. */
double orc_heat(const orc_instance *in, int i, int j)
{
    double a = raw_heat(in, i, j);
    if (!in->symmetrize) return a;
    return (a + raw_heat(in, j, i)) * 0.5;
}

/* d_ij (Sec. II-A): FP64 Euclidean distance of the FP32 coordinates, or c_ij. */
double orc_dist(const orc_instance *in, int i, int j)
{
    if (in->kind == 1) return (double)in->cost[(int64_t)i * in->n + j];
    double dx = (double)in->coords[2 * j] - (double)in->coords[2 * i];
    double dy = (double)in->coords[2 * j + 1] - (double)in->coords[2 * i + 1];
    return sqrt(dx * dx + dy * dy);
}

/* Key of the "nearest unvisited node" rule (Alg. 2) and of the NN tour: the
 * FP32 squared distance (monotone in d up to FP32 rounding) or the FP32 cost;
 * ties go to the smaller node index. */
float orc_key(const orc_instance *in, int i, int j)
{
    if (in->kind == 1) return in->cost[(int64_t)i * in->n + j];
    float dx = in->coords[2 * j] - in->coords[2 * i];
    float dy = in->coords[2 * j + 1] - in->coords[2 * i + 1];
    return dx * dx + dy * dy;
}

/* ------------------------------------------------------------------ sorting */

typedef struct { double d; int32_t j; } dj_pair;

static int cmp_dj(const void *a, const void *b)
{
    const dj_pair *x = a, *y = b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return (x->j > y->j) - (x->j < y->j);
}

static int cmp_desc(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) - (x > y);
}

static int cmp_asc(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------- state */

typedef struct {
    orc_instance in;
    orc_params p;
    int n, k_eff, k_pad;
    /* preparation (Algorithm 1) */
    int32_t *cand;      /* n*k_pad, -1 on pad slots, ascending (d, j) */
    double *cdist;      /* n*k_pad, d_ij of each slot */
    double *conf;       /* n*k_pad, thresholded confidence c_ij, eq. (confidence) */
    double *base;       /* n, degree baseline b_i, eq. (background) */
    double *evid;       /* n*k_pad, e_ij, eq. (evidence) */
    double *logev;      /* n*k_pad, ln e_ij (0 where e_ij = 1) */
    float *W;           /* n*k_pad, fl32(eta^beta * e^kappa) */
    int64_t n_lambda;
    int64_t n_edges;    /* |E_theta(h)| = sum_i |P_i|, directed entries above theta_h (Sec. VI-A) */
    double q90, Rhat, kappa, p_x;
    int32_t *nbr;       /* n*ls_k geometric lists for 2-opt */
    int ls_k;
    /* initialisation */
    int32_t *nn_tour;
    double L_nn;
    double tau_max64, tau_min64;
    float tau_max, tau_min;
    float *tau, *choice;
    int32_t *gb_tour;
    double L_gb;
    /* search */
    int32_t t;          /* iterations done */
    int32_t *tours;     /* m*n, last iteration */
    double *lens;       /* m */
    int32_t *ib_tour;   /* n, last iteration-best (after local search) */
    double L_ib;
    /* MMAS schedule (schedule = 1) */
    int32_t *rb_tour;   /* restart-best tour */
    double L_rb;        /* +inf while cleared */
    int32_t t_restart;  /* iteration of the last restart (0: none) */
    int32_t t_rbimp;    /* iteration of the last restart-best improvement */
    int32_t u_gb;       /* period of the T_rb deposit for the next iteration */
    int32_t n_restarts;
    int32_t cap;        /* trace capacity */
    int32_t *tr_ib;     /* per iteration: iteration-best ant */
    double *tr_Lib, *tr_Lgb, *tr_Lrb;
    int32_t *tr_code;   /* per iteration: 1 = T_rb deposited, 2 = restart (or both) */
    int64_t n_fallback; /* construction steps that took the nearest-unvisited rule */
    uint8_t *visited;
} orc_state;

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

/* ---------------------------------------------- candidate lists (Sec. III-A) */

static void build_candidates(orc_state *S)
{
    const orc_instance *in = &S->in;
    int n = S->n, k = S->k_eff, kp = S->k_pad;
    dj_pair *mem = xcalloc((size_t)n, sizeof *mem);
    dj_pair *non = xcalloc((size_t)n, sizeof *non);
    for (int i = 0; i < n; ++i) {
        int nm = 0, nn = 0;
        for (int j = 0; j < n; ++j) {                 /* P_i = {j != i : h_ij > theta_h} */
            if (j == i) continue;
            dj_pair q = {orc_dist(in, i, j), j};
            if (orc_heat(in, i, j) > S->p.theta_h) mem[nm++] = q; else non[nn++] = q;
        }
        S->n_edges += nm;
        qsort(mem, (size_t)nm, sizeof *mem, cmp_dj);
        dj_pair list[ORC_KMAX];
        int c = 0;
        for (; c < k && c < nm; ++c) list[c] = mem[c];   /* |P_i| > k: k closest members */
        if (c < k) {                                     /* |P_i| < k: nearest non-members */
            qsort(non, (size_t)nn, sizeof *non, cmp_dj);
            for (int q = 0; c < k; ++q) list[c++] = non[q];
        }
        /* Reading: the slot order of C_i (which the roulette sums follow) is
         * ascending (d_ij, j); the paper does not fix an order. */
        qsort(list, (size_t)k, sizeof *list, cmp_dj);
        for (c = 0; c < kp; ++c) {
            int64_t s = (int64_t)i * kp + c;
            if (c < k) {
                int j = list[c].j;
                double h = orc_heat(in, i, j);
                S->cand[s] = j;
                S->cdist[s] = list[c].d;
                S->conf[s] = h > S->p.theta_h ? h : 0.0;    /* eq. (confidence) */
            } else {
                S->cand[s] = -1; S->cdist[s] = 0.0; S->conf[s] = 0.0;
            }
        }
    }
    free(mem); free(non);
}

/* ------------------------------------------- evidence and kappa (Sec. III-C) */

/* Type-7 (linear interpolation) sample quantile of an ascending array. */
double orc_quantile7(const double *x, int64_t N, double q)
{
    if (N <= 0) return 0.0;
    double h = (double)(N - 1) * q;
    double lo = floor(h);
    int64_t l = (int64_t)lo;
    if (l >= N - 1) return x[N - 1];
    return x[l] + (h - lo) * (x[l + 1] - x[l]);
}

/* p_x = p_best^(1/n) and the dynamic range R = tau_max/tau_min of eq. (tau_init)
 * or eq. (tau_min_nols).  R does not involve L_nn, which is why kappa can be
 * set before the nearest-neighbour tour exists, as Algorithm 1 orders them.
 * Reading: the "k" of eq. (tau_min_nols) is the candidate-list size in use,
 * min(k, n-1). */
static void dynamic_range(orc_state *S)
{
    S->p_x = orc_exp(orc_ln(S->p.p_best) / (double)S->n);
    if (S->p.local_search) S->Rhat = 2.0 * (double)S->n;
    else S->Rhat = (((double)(S->k_eff - 1) / 2.0) * S->p_x) / (1.0 - S->p_x);
}

static void build_evidence(orc_state *S)
{
    const orc_instance *in = &S->in;
    int n = S->n, k = S->k_eff, kp = S->k_pad, ds = S->p.degree_target;
    double *pos = xcalloc((size_t)(n > kp ? n : kp), sizeof *pos);
    double *lam = xcalloc((size_t)n * kp, sizeof *lam);
    int64_t N = 0;
    for (int i = 0; i < n; ++i) {
        int np = 0;
        if (S->p.baseline_scope == 0) {           /* positive c_ij over j in C_i */
            for (int c = 0; c < k; ++c)
                if (S->conf[(int64_t)i * kp + c] > 0.0) pos[np++] = S->conf[(int64_t)i * kp + c];
        } else {                                  /* positive h_ij over the whole row */
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                double h = orc_heat(in, i, j);
                if (h > S->p.theta_h) pos[np++] = h;
            }
        }
        qsort(pos, (size_t)np, sizeof *pos, cmp_desc);
        double stat = np > ds ? pos[ds] : 0.0;    /* c_i^(d*+1); missing -> 0 */
        double b = stat > S->p.eps ? stat : S->p.eps;   /* eq. (background) */
        S->base[i] = b;
        for (int c = 0; c < kp; ++c) {
            int64_t s = (int64_t)i * kp + c;
            if (c >= k) { S->evid[s] = 0.0; S->logev[s] = 0.0; continue; }
            double cc = S->conf[s] > S->p.eps ? S->conf[s] : S->p.eps;
            double r = cc / b;
            double e = r > 1.0 ? r : 1.0;          /* eq. (evidence) */
            S->evid[s] = e;
            S->logev[s] = e > 1.0 ? orc_ln(e) : 0.0;
            if (e > 1.0) lam[N++] = S->logev[s];
        }
    }
    qsort(lam, (size_t)N, sizeof *lam, cmp_asc);
    S->n_lambda = N;
    S->q90 = orc_quantile7(lam, N, S->p.q_level);   /* eq. (q90) */
    dynamic_range(S);                                /* eq. (tau_ratio) */
    /* eq. (kappa), and the two ablation variants of Sec. V-D: "fixed kappa = 1"
     * drops the instance-level scale altogether; "no cap" keeps the scale by
     * q90 and the pheromone range but drops the cap factor c_cap (reading:
     * the paper prints no formula for this variant). */
    if (S->p.kappa_mode == 1)
        S->kappa = 1.0;
    else if (S->q90 > 0.0 && S->Rhat > 1.0)
        S->kappa = ((S->p.kappa_mode == 2 ? S->p.alpha : S->p.c_cap * S->p.alpha) * orc_ln(S->Rhat)) / S->q90;
    else
        S->kappa = 0.0;
    free(pos); free(lam);
}

/* Static weight eta^beta * e^kappa folded in preparation (end of Sec. III-C),
 * with the log-weight kappa*ln(e) clipped at logw_clip. */
static void build_weights(orc_state *S)
{
    int n = S->n, k = S->k_eff, kp = S->k_pad;
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < kp; ++c) {
            int64_t s = (int64_t)i * kp + c;
            if (c >= k) { S->W[s] = 0.0f; continue; }
            double d = S->cdist[s] > ORC_DFLOOR ? S->cdist[s] : ORC_DFLOOR;
            double eta = 1.0 / d;
            double hb = S->p.beta == 2.0 ? eta * eta : orc_exp(S->p.beta * orc_ln(eta));
            double E = 1.0;
            if (S->logev[s] > 0.0) {
                double lw = S->kappa * S->logev[s];
                E = orc_exp(lw < S->p.logw_clip ? lw : S->p.logw_clip);
            }
            S->W[s] = (float)(hb * E);
        }
}

/* --------------------------------------------------------- 2-opt (Sec. III-D) */

static void build_nbr(orc_state *S)
{
    int n = S->n, K = S->ls_k;
    dj_pair *all = xcalloc((size_t)n, sizeof *all);
    for (int a = 0; a < n; ++a) {
        int c = 0;
        for (int j = 0; j < n; ++j) if (j != a) { all[c].d = orc_dist(&S->in, a, j); all[c].j = j; ++c; }
        qsort(all, (size_t)c, sizeof *all, cmp_dj);
        for (int q = 0; q < K; ++q) S->nbr[(int64_t)a * K + q] = all[q].j;
    }
    free(all);
}

/* Reverse the cyclic position range [i, i+len-1] of the tour in place. */
static void reverse_cyclic(int32_t *tour, int32_t *pos, int n, int i, int len)
{
    for (int x = 0; x < len / 2; ++x) {
        int p = (i + x) % n, q = (i + len - 1 - x) % n;
        int32_t u = tour[p], v = tour[q];
        tour[p] = v; tour[q] = u;
        pos[v] = p; pos[u] = q;
    }
}

/* Replace edges (a, succ a) and (b, succ b) by (a, b) and (succ a, succ b):
 * reverse positions pos(succ a)..pos(b), or the complementary range
 * pos(succ b)..pos(a) when that one is shorter (strictly more than half). */
static void apply_2opt_succ(int32_t *tour, int32_t *pos, int n, int a, int b)
{
    int i = (pos[a] + 1) % n, j = pos[b];
    int len = (j - i + n) % n + 1;
    if (2 * len > n) {
        int i2 = (pos[b] + 1) % n, j2 = pos[a];
        int len2 = (j2 - i2 + n) % n + 1;
        reverse_cyclic(tour, pos, n, i2, len2);
    } else {
        reverse_cyclic(tour, pos, n, i, len);
    }
}

/* First-improvement 2-opt over geometric neighbour lists with don't-look bits.
 * Reading of "first-improvement 2-opt with don't-look bits" (Sec. III-D):
 * full passes over the tour positions are repeated until a pass makes no move;
 * a city whose bit is set is skipped; for city a the moves are tried for the
 * successor direction and then the predecessor direction, each over nbr(a) in
 * list order, stopping a direction at the first b with d(a,b) >= d(a, dir a);
 * the first move with gain > 1e-10 is applied, the bits of its four end points
 * are cleared and a is examined again; a city with no move gets its bit set.
 * A reversal flips succ/pred inside the reversed range, which can open moves
 * at cities whose bits are set, so the passes run in rounds that start with
 * all bits clear; the search ends after a round whose first pass (over every
 * city) makes no move, i.e. at a local optimum of the neighbour-list moves.
 * A call stops after 64n + 1024 moves, a guard that strictly decreasing tour
 * lengths never reach in practice. */
int orc_two_opt(const orc_instance *in, const int32_t *nbr, int K, int32_t *tour)
{
    int n = in->n;
    int32_t *pos = xcalloc((size_t)n, sizeof *pos);
    uint8_t *dlb = xcalloc((size_t)n, 1);
    if (!pos || !dlb) { free(pos); free(dlb); return ORC_ENOMEM; }
    for (int p = 0; p < n; ++p) pos[tour[p]] = p;
    int moves = 0, round_moves;
    const long long max_moves = 64LL * n + 1024;
    do {
      round_moves = 0;
      memset(dlb, 0, (size_t)n);
      int improved = 1;
      while (improved && moves < max_moves) {
        improved = 0;
        for (int p = 0; p < n && moves < max_moves; ++p) {
            int a = tour[p];
            if (dlb[a]) continue;
            int moved;
            do {
                moved = 0;
                for (int dir = 0; dir < 2 && !moved; ++dir) {
                    int an = dir == 0 ? tour[(pos[a] + 1) % n] : tour[(pos[a] + n - 1) % n];
                    double da = orc_dist(in, a, an);
                    for (int q = 0; q < K; ++q) {
                        int b = nbr[(int64_t)a * K + q];
                        double g1 = da - orc_dist(in, a, b);
                        if (g1 <= 0.0) break;
                        int bn = dir == 0 ? tour[(pos[b] + 1) % n] : tour[(pos[b] + n - 1) % n];
                        if (b == an || bn == a) continue;
                        double gain = (g1 + orc_dist(in, b, bn)) - orc_dist(in, an, bn);
                        if (gain > ORC_LS_GAIN) {
                            if (dir == 0) apply_2opt_succ(tour, pos, n, a, b);
                            else apply_2opt_succ(tour, pos, n, an, bn);   /* (pred a, pred b) */
                            dlb[a] = dlb[an] = dlb[b] = dlb[bn] = 0;
                            moved = 1; improved = 1; ++moves; ++round_moves;
                            break;
                        }
                    }
                }
            } while (moved && moves < max_moves);
            dlb[a] = 1;
        }
      }
    } while (round_moves > 0 && moves < max_moves);
    free(pos); free(dlb);
    return moves;
}

/* ----------------------------------------- directed 2-opt for the ATSP (Sec. III-D)
 *
 * Reading (the paper names a directed 2-opt based on the Jonker-Volgenant
 * reduction): in the 2n-node symmetric graph of that reduction every city is
 * a pair (in-copy, out-copy) joined by a fixed edge, and an ATSP tour is a
 * symmetric tour that alternates the copies.  The 2-opt move that reverses
 * a run of whole pairs keeps every fixed edge and turns the arcs of the run
 * around; in the directed tour it removes two arcs, adds two arcs and
 * reverses the path between them, whose cost changes from its forward sum F
 * to its backward sum R.  The search is that of the 2-opt above with arc
 * costs: for the examined city a,
 *   successor side: a+ = succ(a), b over nbr(a) (smallest c(a, b)) while
 *     g1 = c(a, a+) - c(a, b) > 0 (b = a+ or succ(b) = a skipped); remove
 *     (a, a+), (b, b+), add (a, b), (a+, b+), reverse the path a+ .. b;
 *     gain = (((g1 + c(b, b+)) - c(a+, b+)) + F) - R;
 *   predecessor side: a- = pred(a), b over nbr(a) while g1 = c(a-, a) -
 *     c(a, b) > 0 (b = a- or pred(b) = a skipped); remove (a-, a), (b-, b),
 *     add (a-, b-), (a, b), reverse the path a .. b-;
 *     gain = (((g1 + c(b-, b)) - c(a-, b-)) + F) - R.
 * F and R sum the path's arcs in the order of the tour length (arc k of the
 * path into partial k mod 32, then the pairwise tree).  The path is always
 * reversed in place (its complement would reverse the tour's direction). */

static double path_cost(const orc_instance *in, const int32_t *tour, int n, int i, int len, int backward)
{
    double P[32];
    for (int q = 0; q < 32; ++q) P[q] = 0.0;
    for (int k = 0; k + 1 < len; ++k) {
        int u = tour[(i + k) % n], v = tour[(i + k + 1) % n];
        P[k % 32] = P[k % 32] + (backward ? orc_dist(in, v, u) : orc_dist(in, u, v));
    }
    for (int w = 1; w < 32; w *= 2)
        for (int q = 0; q < 32; q += 2 * w) P[q] = P[q] + P[q + w];
    return P[0];
}

int orc_two_opt_directed(const orc_instance *in, const int32_t *nbr, int K, int32_t *tour)
{
    int n = in->n;
    int32_t *pos = xcalloc((size_t)n, sizeof *pos);
    uint8_t *dlb = xcalloc((size_t)n, 1);
    if (!pos || !dlb) { free(pos); free(dlb); return ORC_ENOMEM; }
    for (int p = 0; p < n; ++p) pos[tour[p]] = p;
    int moves = 0, round_moves;
    const long long max_moves = 64LL * n + 1024;
    do {
      round_moves = 0;
      memset(dlb, 0, (size_t)n);
      int improved = 1;
      while (improved && moves < max_moves) {
        improved = 0;
        for (int p = 0; p < n && moves < max_moves; ++p) {
            int a = tour[p];
            if (dlb[a]) continue;
            int moved;
            do {
                moved = 0;
                for (int dir = 0; dir < 2 && !moved; ++dir) {
                    int x = dir == 0 ? tour[(pos[a] + 1) % n] : tour[(pos[a] + n - 1) % n];   /* a+ or a- */
                    double cx = dir == 0 ? orc_dist(in, a, x) : orc_dist(in, x, a);
                    for (int q = 0; q < K; ++q) {
                        int b = nbr[(int64_t)a * K + q];
                        double g1 = cx - orc_dist(in, a, b);
                        if (g1 <= 0.0) break;
                        int y = dir == 0 ? tour[(pos[b] + 1) % n] : tour[(pos[b] + n - 1) % n];  /* b+ or b- */
                        if (b == x || y == a) continue;
                        int i0 = dir == 0 ? pos[x] : pos[a];          /* path start */
                        int i1 = dir == 0 ? pos[b] : pos[y];          /* path end */
                        int len = (i1 - i0 + n) % n + 1;
                        double F = path_cost(in, tour, n, i0, len, 0);
                        double R = path_cost(in, tour, n, i0, len, 1);
                        double gain = dir == 0
                            ? (((g1 + orc_dist(in, b, y)) - orc_dist(in, x, y)) + F) - R
                            : (((g1 + orc_dist(in, y, b)) - orc_dist(in, x, y)) + F) - R;
                        if (gain > ORC_LS_GAIN) {
                            reverse_cyclic(tour, pos, n, i0, len);
                            dlb[a] = dlb[x] = dlb[b] = dlb[y] = 0;
                            moved = 1; improved = 1; ++moves; ++round_moves;
                            break;
                        }
                    }
                }
            } while (moved && moves < max_moves);
            dlb[a] = 1;
        }
      }
    } while (round_moves > 0 && moves < max_moves);
    free(pos); free(dlb);
    return moves;
}

/* ------------------------------------------------------------ 3-opt (Sec. III-D)
 *
 * First-improvement 3-opt restricted to the geometric neighbour lists, with
 * don't-look bits.  Reading (the paper names the operator only): a move is a
 * sequential exchange in the notation of Lin and Kernighan.  For the examined
 * city t2 = a and t1 = dir(a) (successor direction first), t3 runs over
 * nbr(t2) while g1 = d(t1,t2) - d(t2,t3) > 0; for t4 = dir(t3) (then the
 * other tour neighbour of t3): closing with (t4, t1) is the 2-opt move of the
 * 2-opt above; otherwise t5 runs over nbr(t4) while g2 = g1 + d(t3,t4) -
 * d(t4,t5) > 0 and t6 over (succ t5, pred t5).  Removed edges (t1,t2),
 * (t3,t4), (t5,t6), added (t2,t3), (t4,t5), (t6,t1); a candidate counts when
 * the result is one Hamiltonian cycle and its gain exceeds 1e-10.  Gains are
 * FP64 in the order written: (g1 + d34) - d41 and ((g1 + d34) - d45 + d56)
 * - d61.  The first such candidate in this order is applied; the bits of its
 * cities are cleared and a is examined again; a city without a move gets its
 * bit set.  Passes and rounds are those of the 2-opt above.
 *
 * Applying a move: the removed edges sit at tour positions e (edge between
 * tour[e] and tour[e+1 mod n]); positions outside [e_min + 1, e_max] keep
 * their cities, and the middle range is rewritten with the middle segments
 * in the order and orientation the new cycle visits them when it leaves
 * tour[e_min] (so the array changes only between the first and last removed
 * edge). */

typedef struct {
    int r;          /* removed edges (2 or 3) */
    int e[3];       /* their positions */
    int seg[2];     /* middle segments in visiting order (index into the sorted edges) */
    int rev[2];     /* 1: that segment is walked backwards */
} orc_xchg;

static int edge_pos(const int32_t *pos, int n, int u, int v)
{
    if (pos[v] == (pos[u] + 1) % n) return pos[u];
    if (pos[u] == (pos[v] + 1) % n) return pos[v];
    return -1;
}

/* The removed edges ed[k] (as city pairs) and the added edges given as pairs
 * of (edge k, city); fills X when the exchange leaves one cycle. */
static int orc_reconnect(const int32_t *tour, const int32_t *pos, int n, int r, const int (*ed)[2],
                         const int (*add)[4], orc_xchg *X)
{
    int e[3], ord[3];
    for (int k = 0; k < r; ++k) {
        e[k] = edge_pos(pos, n, ed[k][0], ed[k][1]);
        if (e[k] < 0) return 0;
        ord[k] = k;
    }
    for (int a = 0; a < r; ++a)
        for (int b = a + 1; b < r; ++b) if (e[a] == e[b]) return 0;
    for (int a = 0; a < r; ++a)              /* sort by position */
        for (int b = a + 1; b < r; ++b)
            if (e[ord[b]] < e[ord[a]]) { int t = ord[a]; ord[a] = ord[b]; ord[b] = t; }
    int rank[3];
    for (int j = 0; j < r; ++j) rank[ord[j]] = j;
    /* slot of a city on removed edge k: 2*j + side, j = position rank, side 0
     * for tour[e] (end of the segment before the edge), 1 for tour[e+1] */
    int partner[6];
    for (int q = 0; q < 6; ++q) partner[q] = -1;
    for (int a = 0; a < r; ++a) {
        int sl[2];
        for (int h = 0; h < 2; ++h) {
            int k = add[a][2 * h], c = add[a][2 * h + 1];
            int ek = e[k];
            int side;
            if (tour[ek] == c) side = 0;
            else if (tour[(ek + 1) % n] == c) side = 1;
            else return 0;
            sl[h] = 2 * rank[k] + side;
        }
        if (partner[sl[0]] >= 0 || partner[sl[1]] >= 0 || sl[0] == sl[1]) return 0;
        partner[sl[0]] = sl[1];
        partner[sl[1]] = sl[0];
    }
    /* middle segment j (0 <= j < r-1) runs from slot 2j+1 (head) to slot
     * 2(j+1) (tail); the fixed part ends at slot 0 and starts at slot 2r-1 */
    int used[2] = {0, 0}, cnt = 0, cur = 0;
    for (;;) {
        int s = partner[cur];
        if (s == 2 * r - 1) break;
        if (s == 0) return 0;
        int j, back;
        if (s % 2 == 1) { j = (s - 1) / 2; back = 0; } else { j = s / 2 - 1; back = 1; }
        if (j < 0 || j >= r - 1 || used[j] || cnt >= r - 1) return 0;
        used[j] = 1;
        X->seg[cnt] = j; X->rev[cnt] = back; ++cnt;
        cur = back ? 2 * j + 1 : 2 * (j + 1);
    }
    if (cnt != r - 1) return 0;
    X->r = r;
    for (int j = 0; j < r; ++j) X->e[j] = e[ord[j]];
    return 1;
}

static void orc_apply_xchg(int32_t *tour, int32_t *pos, int n, const orc_xchg *X, int32_t *tmp)
{
    int lo = X->e[0] + 1, w = 0;
    for (int q = 0; q < X->r - 1; ++q) {
        int j = X->seg[q];
        int a = X->e[j] + 1, b = X->e[j + 1];      /* segment positions a..b */
        if (!X->rev[q]) for (int p = a; p <= b; ++p) tmp[w++] = tour[p];
        else for (int p = b; p >= a; --p) tmp[w++] = tour[p];
    }
    for (int q = 0; q < w; ++q) { tour[lo + q] = tmp[q]; pos[tmp[q]] = lo + q; }
}

int orc_three_opt(const orc_instance *in, const int32_t *nbr, int K, int32_t *tour)
{
    int n = in->n;
    int32_t *pos = xcalloc((size_t)n, sizeof *pos);
    int32_t *tmp = xcalloc((size_t)n, sizeof *tmp);
    uint8_t *dlb = xcalloc((size_t)n, 1);
    if (!pos || !dlb || !tmp) { free(pos); free(dlb); free(tmp); return ORC_ENOMEM; }
    for (int p = 0; p < n; ++p) pos[tour[p]] = p;
#define SUCC(c) tour[(pos[c] + 1) % n]
#define PRED(c) tour[(pos[c] + n - 1) % n]
    int moves = 0, round_moves;
    const long long max_moves = 64LL * n + 1024;
    do {
      round_moves = 0;
      memset(dlb, 0, (size_t)n);
      int improved = 1;
      while (improved && moves < max_moves) {
        improved = 0;
        for (int p = 0; p < n && moves < max_moves; ++p) {
            int a = tour[p];
            if (dlb[a]) continue;
            int moved;
            do {
                moved = 0;
                for (int dir = 0; dir < 2 && !moved; ++dir) {
                    int t2 = a, t1 = dir == 0 ? SUCC(a) : PRED(a);
                    double d12 = orc_dist(in, t1, t2);
                    for (int q = 0; q < K && !moved; ++q) {
                        int t3 = nbr[(int64_t)a * K + q];
                        double g1 = d12 - orc_dist(in, t2, t3);
                        if (g1 <= 0.0) break;
                        for (int c4 = 0; c4 < 2 && !moved; ++c4) {
                            int t4 = (c4 == 0) == (dir == 0) ? SUCC(t3) : PRED(t3);
                            if ((t3 == t1 && t4 == t2) || (t3 == t2 && t4 == t1)) continue;
                            double d34 = orc_dist(in, t3, t4);
                            orc_xchg X;
                            if (c4 == 0 && t4 != t1) {
                                double gain = (g1 + d34) - orc_dist(in, t4, t1);
                                int ed[2][2] = {{t1, t2}, {t3, t4}};
                                int add[2][4] = {{0, t2, 1, t3}, {1, t4, 0, t1}};
                                if (gain > ORC_LS_GAIN && orc_reconnect(tour, pos, n, 2, ed, add, &X)) {
                                    orc_apply_xchg(tour, pos, n, &X, tmp);
                                    dlb[t1] = dlb[t2] = dlb[t3] = dlb[t4] = 0;
                                    moved = 1;
                                    break;
                                }
                            }
                            double g1b = g1 + d34;
                            for (int r = 0; r < K && !moved; ++r) {
                                int t5 = nbr[(int64_t)t4 * K + r];
                                double g2 = g1b - orc_dist(in, t4, t5);
                                if (g2 <= 0.0) break;
                                if (t5 == t3) continue;
                                for (int c6 = 0; c6 < 2; ++c6) {
                                    int t6 = c6 == 0 ? SUCC(t5) : PRED(t5);
                                    if (t6 == t1) continue;
                                    double gain = (g2 + orc_dist(in, t5, t6)) - orc_dist(in, t6, t1);
                                    if (!(gain > ORC_LS_GAIN)) continue;
                                    int ed[3][2] = {{t1, t2}, {t3, t4}, {t5, t6}};
                                    int add[3][4] = {{0, t2, 1, t3}, {1, t4, 2, t5}, {2, t6, 0, t1}};
                                    if (!orc_reconnect(tour, pos, n, 3, ed, add, &X)) continue;
                                    orc_apply_xchg(tour, pos, n, &X, tmp);
                                    dlb[t1] = dlb[t2] = dlb[t3] = dlb[t4] = dlb[t5] = dlb[t6] = 0;
                                    moved = 1;
                                    break;
                                }
                            }
                        }
                    }
                }
                if (moved) { improved = 1; ++moves; ++round_moves; }
            } while (moved && moves < max_moves);
            dlb[a] = 1;
        }
      }
    } while (round_moves > 0 && moves < max_moves);
#undef SUCC
#undef PRED
    free(pos); free(dlb); free(tmp);
    return moves;
}

/* ------------------------------------------------------------ tour length */

/* Eq. (tour_length) in FP64.  Reading: the paper fixes no summation order.
 * Edge e joins tour[e] and tour[e+1] (the closing edge is e = n-1).  Edge e
 * goes to partial sum P[e mod 32]; each partial adds its edges in increasing
 * e, starting from 0; the 32 partials are then combined by the pairwise tree
 * (adjacent pairs, then pairs of pair sums, five levels). */
double orc_tour_length(const orc_instance *in, const int32_t *tour)
{
    int n = in->n;
    double P[32];
    for (int q = 0; q < 32; ++q) P[q] = 0.0;
    for (int e = 0; e < n; ++e) P[e % 32] = P[e % 32] + orc_dist(in, tour[e], tour[(e + 1) % n]);
    for (int w = 1; w < 32; w *= 2)
        for (int q = 0; q < 32; q += 2 * w) P[q] = P[q] + P[q + w];
    return P[0];
}

/* ---------------------------------------------- nearest-neighbour tour T_NN */

static int nearest_unvisited(const orc_instance *in, const uint8_t *vis, int i)
{
    int best = -1;
    float bk = 0.0f;
    for (int u = 0; u < in->n; ++u) {
        if (vis[u]) continue;
        float kk = orc_key(in, i, u);
        if (best < 0 || kk < bk) { best = u; bk = kk; }
    }
    return best;
}

/* 2-opt of the instance's kind: symmetric, or directed for the ATSP. */
static void orc_local_2opt(orc_state *S, int32_t *tour)
{
    if (S->in.kind == 1) orc_two_opt_directed(&S->in, S->nbr, S->ls_k, tour);
    else orc_two_opt(&S->in, S->nbr, S->ls_k, tour);
}

/* Reading: T_NN starts at node 0 (Algorithm 1 does not say where). */
static void nn_tour(orc_state *S)
{
    int n = S->n;
    memset(S->visited, 0, (size_t)n);
    S->nn_tour[0] = 0;
    S->visited[0] = 1;
    for (int s = 1; s < n; ++s) {
        int j = nearest_unvisited(&S->in, S->visited, S->nn_tour[s - 1]);
        S->nn_tour[s] = j;
        S->visited[j] = 1;
    }
    if (S->p.local_search == 1 || S->p.local_search == 2) orc_local_2opt(S, S->nn_tour);
    if (S->p.local_search >= 3) orc_three_opt(&S->in, S->nbr, S->ls_k, S->nn_tour);
    S->L_nn = orc_tour_length(&S->in, S->nn_tour);
}

/* --------------------------------------- pheromone bounds (eqs. tau_init ...) */

static void set_bounds(orc_state *S, double L)
{
    S->tau_max64 = 1.0 / (S->p.rho * L);
    if (S->p.local_search)
        S->tau_min64 = S->tau_max64 / (2.0 * (double)S->n);
    else
        S->tau_min64 = (S->tau_max64 * (1.0 - S->p_x)) / (((double)(S->k_eff - 1) / 2.0) * S->p_x);
    S->tau_max = (float)S->tau_max64;
    S->tau_min = (float)S->tau_min64;
}

/* choice = fl32(tau^alpha * W), the numerator of eq. (transition). */
static float choice_of(const orc_state *S, float tau, float W)
{
    double a = S->p.alpha == 1.0 ? (double)tau : orc_exp(S->p.alpha * orc_ln((double)tau));
    return (float)(a * (double)W);
}

/* ------------------------------------------------------- roulette (Alg. 2) */

/* Sampling j with probability w_j / sum_l w_l (Alg. 2), with one fixed
 * evaluation order.  Slots are taken in 8 groups of 4; inside a group the
 * partial sums are sequential, the 8 group totals are combined by an
 * inclusive Hillis-Steele scan with offsets 1, 2, 4, and the prefix of slot c
 * is the exclusive group prefix plus the in-group partial sum.  The draw
 * r = fl32(u * total) selects the first live slot with r < prefix; if rounding
 * leaves none, the last live slot. */
int orc_roulette(const float *w, int k_pad, float u)
{
    float p[8][4], I[8], S[ORC_KMAX];
    for (int g = 0; g < 8; ++g) {
        float acc = 0.0f;
        for (int q = 0; q < 4; ++q) {
            int c = 4 * g + q;
            float wc = c < k_pad ? w[c] : 0.0f;
            acc = q == 0 ? wc : acc + wc;
            p[g][q] = acc;
        }
        I[g] = p[g][3];
    }
    for (int o = 1; o < 8; o *= 2) {
        float nx[8];
        for (int g = 0; g < 8; ++g) nx[g] = g >= o ? I[g] + I[g - o] : I[g];
        memcpy(I, nx, sizeof I);
    }
    for (int c = 0; c < k_pad; ++c) {
        int g = c / 4, q = c % 4;
        S[c] = g == 0 ? p[0][q] : I[g - 1] + p[g][q];
    }
    float r = u * I[7];
    int last = -1;
    for (int c = 0; c < k_pad; ++c) {
        if (!(w[c] > 0.0f)) continue;
        if (r < S[c]) return c;
        last = c;
    }
    return last;
}

/* ---------------------------------------------- one ant's tour (Alg. 2) */

static void construct(orc_state *S, int a, int32_t *T, double *Lout)
{
    const orc_instance *in = &S->in;
    int n = S->n, kp = S->k_pad;
    uint32_t t = (uint32_t)S->t;
    memset(S->visited, 0, (size_t)n);
    uint32_t x0 = orc_draw(S->p.seed, t, (uint32_t)a, 0);
    int start = (int)(((uint64_t)x0 * (uint64_t)n) >> 32);   /* random start node */
    T[0] = start;
    S->visited[start] = 1;
    float w[ORC_KMAX];
    for (int s = 1; s < n; ++s) {
        int i = T[s - 1];
        int any = 0;
        for (int c = 0; c < kp; ++c) {                   /* N_i = C_i minus visited */
            int32_t j = S->cand[(int64_t)i * kp + c];
            w[c] = (j >= 0 && !S->visited[j]) ? S->choice[(int64_t)i * kp + c] : 0.0f;
            if (w[c] > 0.0f) any = 1;
        }
        int j;
        if (any) {
            float u = unif24(orc_draw(S->p.seed, t, (uint32_t)a, (uint32_t)s));
            int c = orc_roulette(w, kp, u);
            j = S->cand[(int64_t)i * kp + c];
        } else {                                         /* nearest unvisited node */
            j = nearest_unvisited(in, S->visited, i);
            S->n_fallback++;
        }
        T[s] = j;
        S->visited[j] = 1;
    }
    *Lout = orc_tour_length(in, T);
}

/* --------------------------------------------- MMAS schedule (Alg. 1, III-B)
 *
 * What Sec. III-B and Sec. IV-D fix: which tour deposits alternates between
 * T_ib and the restart-best T_rb, T_rb taking a growing share (its period
 * u_gb shrinks from 25 to 1); a stagnation check runs every 100 iterations
 * and, if T_rb is more than 250 iterations old and the branching factor
 * (band 0.05) is under 1 + 1e-5, resets every trail to tau_max and forgets
 * T_rb while T_gb survives.  The steps of
 * u_gb and the branching-factor normalisation are not printed in the paper;
 * the ones used here are the MMAS ones (Stuetzle and Hoos, 2000): u_gb = 25,
 * 5, 3, 2, 1 for s < 25, 75, 125, 250 and beyond, s = iterations since the
 * last restart (or the start), and the mean per-node count of candidate
 * slots with tau >= min_i + xi_bf (max_i - min_i), divided by d*.
 */

int orc_ugb(int32_t s)
{
    if (s < 25) return 25;
    if (s < 75) return 5;
    if (s < 125) return 3;
    if (s < 250) return 2;
    return 1;
}

double orc_branching(const float *tau, const int32_t *cand, int n, int kp, int dstar)
{
    int64_t count = 0;
    for (int i = 0; i < n; ++i) {
        double lo = INFINITY, hi = -INFINITY;
        for (int c = 0; c < kp; ++c) {
            int64_t s = (int64_t)i * kp + c;
            if (cand[s] < 0) continue;
            double v = (double)tau[s];
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        double cut = lo + 0.05 * (hi - lo);
        for (int c = 0; c < kp; ++c) {
            int64_t s = (int64_t)i * kp + c;
            if (cand[s] >= 0 && (double)tau[s] >= cut) ++count;
        }
    }
    return (double)count / ((double)n * (double)dstar);
}

/* ------------------------------------------------- one iteration (Alg. 1) */

static void iterate_once(orc_state *S)
{
    int n = S->n, m = S->p.m, kp = S->k_pad;
    for (int a = 0; a < m; ++a) construct(S, a, S->tours + (int64_t)a * n, &S->lens[a]);
    if (S->p.local_search == 2 || S->p.local_search == 4)   /* Algorithm 1: local search on every ant */
        for (int a = 0; a < m; ++a) {
            if (S->p.local_search == 2) orc_local_2opt(S, S->tours + (int64_t)a * n);
            else orc_three_opt(&S->in, S->nbr, S->ls_k, S->tours + (int64_t)a * n);
            S->lens[a] = orc_tour_length(&S->in, S->tours + (int64_t)a * n);
        }
    int ib = 0;                                          /* iteration best, ties -> lowest ant */
    for (int a = 1; a < m; ++a) if (S->lens[a] < S->lens[ib]) ib = a;
    memcpy(S->ib_tour, S->tours + (int64_t)ib * n, (size_t)n * sizeof(int32_t));
    S->L_ib = S->lens[ib];
    if (S->p.local_search == 1 || S->p.local_search == 3) {   /* local search on T_ib before it is used */
        if (S->p.local_search == 1) orc_local_2opt(S, S->ib_tour);
        else orc_three_opt(&S->in, S->nbr, S->ls_k, S->ib_tour);
        S->L_ib = orc_tour_length(&S->in, S->ib_tour);
    }
    const int32_t t1 = S->t + 1;                         /* this iteration, counted from 1 */
    int use_rb = 0, code = 0;
    if (S->p.schedule) {                                 /* restart-best, then the elite choice */
        if (S->L_ib < S->L_rb) {
            memcpy(S->rb_tour, S->ib_tour, (size_t)n * sizeof(int32_t));
            S->L_rb = S->L_ib;
            S->t_rbimp = t1;
        }
        use_rb = t1 % S->u_gb == 0;
        code = use_rb;
    }
    if (S->L_ib < S->L_gb) {                             /* new global best: recompute bounds */
        memcpy(S->gb_tour, S->ib_tour, (size_t)n * sizeof(int32_t));
        S->L_gb = S->L_ib;
        set_bounds(S, S->L_gb);
    }
    /* Evaporate and deposit on T+ (T_ib, or T_rb by the schedule), eqs.
     * (pheromone_update)/(pheromone_delta), on the stored candidate edges only.
     * A symmetric instance deposits on the slot of either orientation of a
     * tour edge; an ATSP only on i -> succ(i). */
    const int32_t *elite = use_rb ? S->rb_tour : S->ib_tour;
    const double L_elite = use_rb ? S->L_rb : S->L_ib;
    int32_t *succ = xcalloc((size_t)n, sizeof *succ), *pred = xcalloc((size_t)n, sizeof *pred);
    for (int s = 0; s < n; ++s) {
        int u = elite[s], v = elite[(s + 1) % n];
        succ[u] = v; pred[v] = u;
    }
    float omega = (float)(1.0 - S->p.rho);
    float delta = (float)(1.0 / L_elite);
    int sym = S->in.kind == 0;
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < kp; ++c) {
            int64_t s = (int64_t)i * kp + c;
            int32_t j = S->cand[s];
            if (j < 0) continue;
            float x = S->tau[s] * omega;
            if (succ[i] == j || (sym && pred[i] == j)) x = x + delta;
            float y = x > S->tau_min ? x : S->tau_min;
            S->tau[s] = y < S->tau_max ? y : S->tau_max;
            S->choice[s] = choice_of(S, S->tau[s], S->W[s]);
        }
    free(succ); free(pred);
    if (S->p.schedule) {                                 /* restart check, then the next u_gb */
        if (t1 % 100 == 0 && t1 - S->t_rbimp > 250 &&
            orc_branching(S->tau, S->cand, n, kp, S->p.degree_target) < 1.0 + 1e-5) {
            for (int64_t s = 0; s < (int64_t)n * kp; ++s)
                if (S->cand[s] >= 0) {
                    S->tau[s] = S->tau_max;
                    S->choice[s] = choice_of(S, S->tau[s], S->W[s]);
                }
            S->L_rb = INFINITY;
            S->t_restart = t1;
            S->t_rbimp = t1;
            S->n_restarts++;
            code |= 2;
        }
        S->u_gb = orc_ugb(t1 - S->t_restart);
    }
    if (S->t < S->cap) {
        S->tr_ib[S->t] = ib; S->tr_Lib[S->t] = S->L_ib; S->tr_Lgb[S->t] = S->L_gb;
        S->tr_Lrb[S->t] = S->L_rb; S->tr_code[S->t] = code;
    }
    S->t++;
}

/* ------------------------------------------------------------- public API */

static int check_inputs(const orc_instance *in, const orc_params *p)
{
    if (!in || !p || in->n < 3) return ORC_EINVAL;
    if (p->k < 1 || p->k > ORC_KMAX || p->m < 1 || p->iterations < 0) return ORC_EINVAL;
    if (in->kind == 0 && !in->coords) return ORC_EINVAL;
    if (in->kind == 1 && !in->cost) return ORC_EINVAL;
    if (in->kind != 0 && in->kind != 1) return ORC_EINVAL;
    if (!in->rowptr || in->rowptr[0] != 0) return ORC_EINVAL;
    for (int i = 0; i < in->n; ++i) {
        if (in->rowptr[i + 1] < in->rowptr[i]) return ORC_EINVAL;
        for (int q = in->rowptr[i]; q < in->rowptr[i + 1]; ++q) {
            if (in->col[q] < 0 || in->col[q] >= in->n || in->col[q] == i) return ORC_EINVAL;
            if (q > in->rowptr[i] && in->col[q] <= in->col[q - 1]) return ORC_EINVAL;
            double v = raw_val(in, q);
            if (!(v >= 0.0 && v <= 1.0)) return ORC_EINVAL;
        }
    }
    if (p->rho <= 0.0 || p->rho >= 1.0 || p->degree_target < 1) return ORC_EINVAL;
    if (p->schedule != 0 && p->schedule != 1) return ORC_EINVAL;
    if (p->kappa_mode < 0 || p->kappa_mode > 2) return ORC_EINVAL;
    if (p->local_search < 0 || p->local_search > 4) return ORC_EINVAL;
    if (p->local_search && (p->ls_k < 1 || p->ls_k > in->n - 1)) return ORC_EINVAL;
    if (p->local_search >= 3 && in->kind != 0) return ORC_EINVAL;   /* 3-opt: symmetric only */
    /* the 2-opt's FP32 pre-test needs finite squared coordinate differences:
     * |x|, |y| <= 1e18 with local search (the CUDA path checks the same) */
    if (p->local_search && in->kind == 0)
        for (int64_t q = 0; q < 2 * (int64_t)in->n; ++q)
            if (!(fabs((double)in->coords[q]) <= 1e18)) return ORC_EINVAL;
    return ORC_OK;
}

void orc_destroy(void *h)
{
    orc_state *S = h;
    if (!S) return;
    free(S->cand); free(S->cdist); free(S->conf); free(S->base); free(S->evid);
    free(S->logev); free(S->W); free(S->nbr); free(S->nn_tour); free(S->tau);
    free(S->choice); free(S->gb_tour); free(S->tours); free(S->lens); free(S->ib_tour);
    free(S->tr_ib); free(S->tr_Lib); free(S->tr_Lgb); free(S->visited);
    free(S->rb_tour); free(S->tr_Lrb); free(S->tr_code);
    free(S);
}

/* Preparation and initialisation of Algorithm 1. */
void *orc_create(const orc_instance *in, const orc_params *p, int32_t *status)
{
    int st = check_inputs(in, p);
    if (status) *status = st;
    if (st) return NULL;
    orc_state *S = xcalloc(1, sizeof *S);
    if (!S) { if (status) *status = ORC_ENOMEM; return NULL; }
    S->in = *in; S->p = *p;
    S->n = in->n;
    S->k_eff = p->k < in->n - 1 ? p->k : in->n - 1;
    S->k_pad = 4 * ((p->k + 3) / 4);
    S->ls_k = p->local_search ? p->ls_k : 0;
    size_t n = (size_t)S->n, slots = n * (size_t)S->k_pad, m = (size_t)p->m;
    S->cand = xcalloc(slots, sizeof *S->cand); S->cdist = xcalloc(slots, sizeof *S->cdist);
    S->conf = xcalloc(slots, sizeof *S->conf); S->base = xcalloc(n, sizeof *S->base);
    S->evid = xcalloc(slots, sizeof *S->evid); S->logev = xcalloc(slots, sizeof *S->logev);
    S->W = xcalloc(slots, sizeof *S->W); S->nbr = xcalloc(n * (size_t)(S->ls_k ? S->ls_k : 1), sizeof *S->nbr);
    S->nn_tour = xcalloc(n, sizeof *S->nn_tour); S->tau = xcalloc(slots, sizeof *S->tau);
    S->choice = xcalloc(slots, sizeof *S->choice); S->gb_tour = xcalloc(n, sizeof *S->gb_tour);
    S->tours = xcalloc(m * n, sizeof *S->tours); S->lens = xcalloc(m, sizeof *S->lens);
    S->ib_tour = xcalloc(n, sizeof *S->ib_tour); S->visited = xcalloc(n, 1);
    S->cap = p->iterations > 0 ? p->iterations : 1;
    S->tr_ib = xcalloc((size_t)S->cap, sizeof *S->tr_ib);
    S->tr_Lib = xcalloc((size_t)S->cap, sizeof *S->tr_Lib);
    S->tr_Lgb = xcalloc((size_t)S->cap, sizeof *S->tr_Lgb);
    S->tr_Lrb = xcalloc((size_t)S->cap, sizeof *S->tr_Lrb);
    S->tr_code = xcalloc((size_t)S->cap, sizeof *S->tr_code);
    S->rb_tour = xcalloc(n, sizeof *S->rb_tour);
    if (!S->cand || !S->cdist || !S->conf || !S->base || !S->evid || !S->logev || !S->W ||
        !S->nbr || !S->nn_tour || !S->tau || !S->choice || !S->gb_tour || !S->tours ||
        !S->lens || !S->ib_tour || !S->visited || !S->tr_ib || !S->tr_Lib || !S->tr_Lgb ||
        !S->tr_Lrb || !S->tr_code || !S->rb_tour) {
        orc_destroy(S);
        if (status) *status = ORC_ENOMEM;
        return NULL;
    }
    build_candidates(S);                  /* candidate lists */
    build_evidence(S);                    /* e_ij, q90, kappa */
    build_weights(S);
    if (S->ls_k) build_nbr(S);
    nn_tour(S);                           /* T_NN */
    set_bounds(S, S->L_nn);               /* bounds from L_nn */
    for (size_t s = 0; s < slots; ++s) {
        int real = S->cand[s] >= 0;
        S->tau[s] = real ? S->tau_max : 0.0f;
        S->choice[s] = real ? choice_of(S, S->tau[s], S->W[s]) : 0.0f;
    }
    memcpy(S->gb_tour, S->nn_tour, n * sizeof(int32_t));   /* T_gb = T_NN */
    S->L_gb = S->L_nn;
    S->L_rb = INFINITY;                   /* restart-best: none yet */
    S->u_gb = 25;
    return S;
}

/* The search loop of Algorithm 1 for `iters` more iterations. */
int orc_iterate(void *h, int32_t iters)
{
    orc_state *S = h;
    if (!S || iters < 0) return ORC_EINVAL;
    for (int32_t q = 0; q < iters; ++q) iterate_once(S);
    return ORC_OK;
}

/* Copy-out of the state, by field code (see oracle.py). */
enum {
    ORC_F_CAND = 1, ORC_F_CDIST, ORC_F_CONF, ORC_F_BASE, ORC_F_EVID, ORC_F_LOGEV, ORC_F_W,
    ORC_F_TAU, ORC_F_CHOICE, ORC_F_NN_TOUR, ORC_F_GB_TOUR, ORC_F_TOURS, ORC_F_LENS,
    ORC_F_IB_TOUR, ORC_F_TRACE_IB, ORC_F_TRACE_LIB, ORC_F_TRACE_LGB, ORC_F_NBR,
    ORC_F_SCALARS, ORC_F_INTS, ORC_F_RB_TOUR, ORC_F_TRACE_LRB, ORC_F_TRACE_CODE
};

int orc_get(void *h, int32_t field, void *dst, int64_t bytes)
{
    orc_state *S = h;
    if (!S || !dst) return ORC_EINVAL;
    size_t n = (size_t)S->n, slots = n * (size_t)S->k_pad, m = (size_t)S->p.m;
    const void *src = NULL;
    size_t sz = 0;
    double scal[14];
    int64_t ints[10];
    switch (field) {
    case ORC_F_CAND: src = S->cand; sz = slots * 4; break;
    case ORC_F_CDIST: src = S->cdist; sz = slots * 8; break;
    case ORC_F_CONF: src = S->conf; sz = slots * 8; break;
    case ORC_F_BASE: src = S->base; sz = n * 8; break;
    case ORC_F_EVID: src = S->evid; sz = slots * 8; break;
    case ORC_F_LOGEV: src = S->logev; sz = slots * 8; break;
    case ORC_F_W: src = S->W; sz = slots * 4; break;
    case ORC_F_TAU: src = S->tau; sz = slots * 4; break;
    case ORC_F_CHOICE: src = S->choice; sz = slots * 4; break;
    case ORC_F_NN_TOUR: src = S->nn_tour; sz = n * 4; break;
    case ORC_F_GB_TOUR: src = S->gb_tour; sz = n * 4; break;
    case ORC_F_TOURS: src = S->tours; sz = m * n * 4; break;
    case ORC_F_LENS: src = S->lens; sz = m * 8; break;
    case ORC_F_IB_TOUR: src = S->ib_tour; sz = n * 4; break;
    case ORC_F_TRACE_IB: src = S->tr_ib; sz = (size_t)S->cap * 4; break;
    case ORC_F_TRACE_LIB: src = S->tr_Lib; sz = (size_t)S->cap * 8; break;
    case ORC_F_TRACE_LGB: src = S->tr_Lgb; sz = (size_t)S->cap * 8; break;
    case ORC_F_NBR: src = S->nbr; sz = n * (size_t)(S->ls_k ? S->ls_k : 1) * 4; break;
    case ORC_F_RB_TOUR: src = S->rb_tour; sz = n * 4; break;
    case ORC_F_TRACE_LRB: src = S->tr_Lrb; sz = (size_t)S->cap * 8; break;
    case ORC_F_TRACE_CODE: src = S->tr_code; sz = (size_t)S->cap * 4; break;
    case ORC_F_SCALARS:
        scal[0] = S->q90; scal[1] = S->Rhat; scal[2] = S->kappa; scal[3] = S->p_x;
        scal[4] = S->L_nn; scal[5] = S->tau_max64; scal[6] = S->tau_min64;
        scal[7] = (double)S->tau_max; scal[8] = (double)S->tau_min; scal[9] = S->L_gb;
        scal[10] = S->L_ib; scal[11] = (double)S->n_lambda; scal[12] = S->L_rb;
        scal[13] = (double)S->n_edges / (2.0 * (double)S->n);   /* Edges/n, Sec. VI-A */
        src = scal; sz = sizeof scal; break;
    case ORC_F_INTS:
        ints[0] = S->n; ints[1] = S->k_eff; ints[2] = S->k_pad; ints[3] = S->t;
        ints[4] = S->n_fallback; ints[5] = S->ls_k; ints[6] = S->n_restarts; ints[7] = S->t_restart;
        ints[8] = S->t_rbimp; ints[9] = S->u_gb;
        src = ints; sz = sizeof ints; break;
    default: return ORC_EINVAL;
    }
    if ((size_t)bytes < sz) return ORC_EINVAL;
    memcpy(dst, src, sz);
    return (int)sz;
}
