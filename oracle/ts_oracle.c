/*
 * CPU oracle of the differentiable agent-based traffic simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the benchmark's CPU
 * baseline may load this library.  It shares no code with the CUDA path.
 *
 * Plain, slow, obviously-correct restatement of the method, step by step in the
 * paper's order: one simulator step phi = g o f (Results, "Differentiable
 * agent-based traffic simulation"), f = the per-link car-following model of SI-A
 * (Eq. 1 and the equations after Eq. first_term, Alg. S1), g = the node model of
 * SI-B (link choice, merge choice, differentiable vehicle transfer Eq. transfer,
 * Alg. S2), counting of SI-D, and the reverse-mode derivative of the
 * straight-through / trajectory-grafting surrogate (SI-B, SI-C).
 *
 * Built twice from this one source:
 *   ORACLE_FP32 undefined : all floating point in double (the reference)
 *   ORACLE_FP32 defined   : positions, utilities and Gumbel keys in float, so
 *                           that every decision (arrival, vacancy, argmax) is
 *                           taken in the kernel's precision; the Gumbel
 *                           transform uses or_log32 below.
 *
 * Readings of the paper that this file takes (each is listed in the design notes):
 *  - headways follow the text of SI-A (differences of the *sorted* positions);
 *  - utility is beta/c (text of SI-B) plus a linear feature term;
 *  - arrival means x >= L - eps_arr (Alg. S2), vacancy X_min > 1/kappa dn (strict);
 *  - outflow credit (int fixed point, 2^-16 veh) limits link exits;
 *  - vehicles wait in per-origin FIFO queues (virtual inflow links of length 0);
 *  - a candidate whose link ends in its destination zone leaves to a sink;
 *  - U-turns are excluded from the choice set unless they are the only way out;
 *  - forward choice = argmax(V + g) (exact Gumbel-max draw, temperature-free);
 *  - merge noise is keyed by (vehicle, step) (one target per vehicle per step);
 *  - max(l)^T in the merge mask is a constant mask (no gradient);
 *  - min/max ties of the car-following update are resolved by a dead-band tag.
 *
 * What pins it (tests that run without a GPU, against facts fixed outside this
 * file): Philox known-answer vectors; or_log32 within 2 ulp of a double log;
 * Gumbel moments and distribution; lone-vehicle link times and the Newell
 * capacity of a saturated entry; outflow-credit limits, conservation, FIFO and
 * the other invariants of the node model; softmax turn frequencies; exact
 * enumeration of a small fork and merge; closed-form bin speeds; the relaxed
 * weights tending to the forward's one-hot as the temperature falls; the
 * closed-form gradient and the descent outcome of the trajectory-grafting toy
 * (SI-C); a dense N x L formulation of Alg. S1/S2 differentiated by autograd;
 * finite differences of the frozen surrogate.
 *
 * Parity unpinned by the paper: the demand gradient (the paper does not
 * differentiate demand; here a straight-through demand weight), the 16-feature
 * utility of the calibration parameterisation, and the link speeds and travel
 * times of the counting step, whose definitions are readings.  Their code is
 * pinned by finite differences and closed forms; their definitions are not.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <stdio.h>

#ifdef ORACLE_FP32
typedef float real;
#else
typedef double real;
#endif

#define FX_ONE 65536LL

/* ------------------------------------------------------------------------- */
/* Scenario description (mirrored by a ctypes Structure in oracle/oracle.py)   */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t V, L, F, Z, N, n_od;
    const int32_t *tail, *head;
    const float *length, *u, *kappa, *alpha, *beta, *cost;
    const int32_t *q_fx;
    const float *phi, *psi, *w;
    const int32_t *node_zone;
    const float *dest_feat;
    const int32_t *origin, *dest_zone, *dep_step, *od;
    const float *od_lambda;
    float dt, dn, tau, M, eps_arr, eps_tag, alpha_origin;
    uint64_t seed;
    uint32_t scenario_id;
    int32_t obs_every;
} or_scenario;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy */
/* as 1, 2, 3", SC'11): 10 rounds of the Philox S-box with multipliers          */
/* 0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 / 0xBB67AE85.     */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Natural logarithm in float, written from the textbook method: split x = 2^e m
 * with m in (sqrt(1/2), sqrt(2)], log m = 2 atanh(r), r = (m-1)/(m+1), atanh by
 * its Taylor series through r^11, and e*ln2 added in two parts (Cody & Waite,
 * "Software Manual for the Elementary Functions", 1980).  Valid for positive
 * normal x.  Used only by the float build so that Gumbel keys are reproducible. */
float or_log32(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    int e = (int)((b >> 23) & 0xffu) - 127;
    uint32_t mb = (b & 0x7fffffu) | 0x3f800000u;
    float m;
    memcpy(&m, &mb, 4);
    if (m > 0x1.6a09e6p+0f) { m = m * 0.5f; e += 1; }
    float f = m - 1.0f;
    float d = m + 1.0f;
    float r = f / d;
    float r2 = r * r;
    float p = 0x1.745d18p-4f;              /* 1/11 */
    p = 0x1.c71c72p-4f + r2 * p;           /* 1/9  */
    p = 0x1.24924ap-3f + r2 * p;           /* 1/7  */
    p = 0x1.99999ap-3f + r2 * p;           /* 1/5  */
    p = 0x1.555556p-2f + r2 * p;           /* 1/3  */
    float q = r2 * p;
    float lm = 2.0f * (r + r * q);
    float fe = (float)e;
    float hi = fe * 0x1.62ep-1f;           /* ln2 high part, 12 significant bits */
    float lo = fe * 0x1.0bfbe8p-15f;       /* ln2 - high part */
    return hi + (lm + lo);
}

static real rlog(real x)
{
#ifdef ORACLE_FP32
    return or_log32(x);
#else
    return log(x);
#endif
}

/* uniform in (0,1) from one 32-bit word: ((w >> 9) + 1/2) 2^-23, exact in float */
static real uniform_from_word(uint32_t w)
{
    real a = (real)(w >> 9);
    a = a + (real)0.5;
    return a * (real)(1.0 / 8388608.0);
}

/* Gumbel(0,1) sample keyed by (vehicle, step, stream, slot) */
static real gumbel(uint64_t seed, uint32_t scen, int32_t vid, int32_t t, int stream, int slot)
{
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) ^ scen };
    uint32_t ctr[4] = { (uint32_t)vid, (uint32_t)t, (uint32_t)stream, (uint32_t)(slot >> 2) };
    uint32_t o[4];
    or_philox4x32_10(ctr, key, o);
    real uu = uniform_from_word(o[slot & 3]);
    real a = rlog(uu);
    a = -a;
    real b = rlog(a);
    return -b;
}

double or_gumbel(uint64_t seed, uint32_t scen, int32_t vid, int32_t t, int stream, int slot)
{
    return (double)gumbel(seed, scen, vid, t, stream, slot);
}

/* ------------------------------------------------------------------------- */
/* Simulator state                                                            */
/* ------------------------------------------------------------------------- */
enum { TAG_FREE = 0, TAG_CONG = 1, TAG_STOP = 2 };
enum { TGT_NONE = -1, TGT_SINK = -2, TGT_BLOCKED = -3 };
#define VEH_WAITING (-1)
#define VEH_ARRIVED (-2)

typedef struct {     /* one candidate of one step (history for the backward) */
    int32_t vid, src_link, src_node;   /* src_link >= 0 for link leaders, else -1 */
    int32_t target, slot, valid, won;
    real x;                            /* post-f position (0 for origin queues) */
} or_cand;

typedef struct {     /* per-step record kept when history is on */
    int32_t *vlink;          /* [N] link at the start of the step (S_t) */
    real *xpre, *xpost;      /* [N] positions before / after f */
    int8_t *tag;             /* [N] car-following branch tag */
    int32_t *fifo_ptr;       /* [V] */
    or_cand *cand;
    int32_t n_cand;
} or_hist;

typedef struct {
    or_scenario sc;
    /* copies of inputs */
    int32_t *tail, *head, *node_zone, *origin, *dest_zone, *dep_step, *od, *q_fx;
    float *length, *u, *kappa, *alpha, *beta, *cost, *phi, *psi, *w, *dest_feat, *od_lambda;
    /* derived */
    real *len, *s, *udt, *Uu, *Gg, *alpha_r, *half_len, *dtag;
    int64_t *cap_fx;
    int64_t dn_fx;
    int32_t *lo_ptr, *lo_idx;       /* choice set after each link (U-turns filtered) */
    int32_t *no_ptr, *no_idx;       /* out-links of each node */
    int32_t *fifo_beg, *fifo_end, *fifo_list, *fifo_ptr;
    /* vehicle state */
    int32_t *vlink, *ventry;
    real *vx;
    int64_t *vseq;
    /* link state */
    int64_t *credit, *exits;
    /* observation accumulators (distance summed in double in both builds) */
    double *acc_dx;
    int64_t *acc_n, *tt_sum, *tt_cnt, *C_prev;
    int32_t t, T, n_bins;
    int32_t *out_counts;      /* [n_bins][L] */
    double *out_speed, *out_tt;
    int64_t *n_wait, *n_on, *n_arr;     /* [T+1] */
    int64_t cnt_wait, cnt_on, cnt_arr;
    /* last step records */
    int32_t *rec_link_cand, *rec_link_target, *rec_node_cand, *rec_node_target, *rec_link_in;
    double *rec_link_margin, *rec_node_margin, *rec_merge_margin;
    double *rec_arr_margin, *rec_vac_margin;
    /* history (for the backward) */
    int keep_hist;
    or_hist *hist;
    int32_t *route_len, *route_cap;
    int32_t **route_t, **route_m;
    /* scratch */
    int32_t *mem_cnt, *mem_ptr, *mem_list;
    real *xnew;
    int8_t *tagbuf;
    char err[256];
    int failed;
} or_sim;

static void *xcalloc(size_t n, size_t sz) { void *p = calloc(n ? n : 1, sz ? sz : 1); return p; }

#define COPY(dst, src, n, T) do { (dst) = (T *)xcalloc((n), sizeof(T)); memcpy((dst), (src), (size_t)(n) * sizeof(T)); } while (0)

static void fail(or_sim *o, const char *msg, int a, int b)
{
    if (!o->failed) snprintf(o->err, sizeof o->err, "%s (%d, %d)", msg, a, b);
    o->failed = 1;
}

const char *or_error(or_sim *o) { return o->failed ? o->err : ""; }

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

static const or_sim *g_sort_ctx;
static int cmp_fifo(const void *a, const void *b)
{
    int i = *(const int *)a, j = *(const int *)b;
    int di = g_sort_ctx->dep_step[i], dj = g_sort_ctx->dep_step[j];
    if (di != dj) return (di > dj) - (di < dj);
    return (i > j) - (i < j);
}

/* argsort(-x~) of SI-A: positions descending; equal positions by earlier entry */
static int cmp_pos_desc(const void *a, const void *b)
{
    int i = *(const int *)a, j = *(const int *)b;
    real xi = g_sort_ctx->vx[i], xj = g_sort_ctx->vx[j];
    if (xi != xj) return xi > xj ? -1 : 1;
    int64_t si = g_sort_ctx->vseq[i], sj = g_sort_ctx->vseq[j];
    return (si > sj) - (si < sj);
}

or_sim *or_create(const or_scenario *sc, int keep_hist)
{
    or_sim *o = (or_sim *)xcalloc(1, sizeof(or_sim));
    o->sc = *sc;
    int V = sc->V, L = sc->L, F = sc->F, Z = sc->Z, N = sc->N;
    COPY(o->tail, sc->tail, L, int32_t);
    COPY(o->head, sc->head, L, int32_t);
    COPY(o->node_zone, sc->node_zone, V, int32_t);
    COPY(o->origin, sc->origin, N, int32_t);
    COPY(o->dest_zone, sc->dest_zone, N, int32_t);
    COPY(o->dep_step, sc->dep_step, N, int32_t);
    COPY(o->od, sc->od, N, int32_t);
    COPY(o->q_fx, sc->q_fx, L, int32_t);
    COPY(o->length, sc->length, L, float);
    COPY(o->u, sc->u, L, float);
    COPY(o->kappa, sc->kappa, L, float);
    COPY(o->alpha, sc->alpha, L, float);
    COPY(o->beta, sc->beta, L, float);
    COPY(o->cost, sc->cost, L, float);
    COPY(o->phi, sc->phi, (size_t)L * F, float);
    COPY(o->psi, sc->psi, (size_t)L * F, float);
    COPY(o->w, sc->w, F, float);
    COPY(o->dest_feat, sc->dest_feat, (size_t)Z * V, float);
    COPY(o->od_lambda, sc->od_lambda, sc->n_od, float);
    o->sc.tail = o->tail; o->sc.head = o->head;
    o->keep_hist = keep_hist;

    /* out-links of each node, in increasing link id */
    o->no_ptr = (int32_t *)xcalloc(V + 1, sizeof(int32_t));
    o->no_idx = (int32_t *)xcalloc(L, sizeof(int32_t));
    for (int j = 0; j < L; ++j) o->no_ptr[o->tail[j] + 1]++;
    for (int n = 0; n < V; ++n) o->no_ptr[n + 1] += o->no_ptr[n];
    {
        int32_t *fill = (int32_t *)xcalloc(V, sizeof(int32_t));
        for (int j = 0; j < L; ++j) { int n = o->tail[j]; o->no_idx[o->no_ptr[n] + fill[n]++] = j; }
        free(fill);
    }
    /* choice set after link l: out-links of head(l) minus those returning to tail(l),
     * unless nothing else leaves that node */
    o->lo_ptr = (int32_t *)xcalloc(L + 1, sizeof(int32_t));
    int total = 0;
    for (int l = 0; l < L; ++l) {
        int n = o->head[l], c = 0, any = 0;
        for (int k = o->no_ptr[n]; k < o->no_ptr[n + 1]; ++k) { any++; if (o->head[o->no_idx[k]] != o->tail[l]) c++; }
        total += c ? c : any;
    }
    o->lo_idx = (int32_t *)xcalloc(total, sizeof(int32_t));
    total = 0;
    for (int l = 0; l < L; ++l) {
        int n = o->head[l], c = 0;
        o->lo_ptr[l] = total;
        for (int k = o->no_ptr[n]; k < o->no_ptr[n + 1]; ++k) if (o->head[o->no_idx[k]] != o->tail[l]) c++;
        for (int k = o->no_ptr[n]; k < o->no_ptr[n + 1]; ++k) {
            int m = o->no_idx[k];
            if (!c || o->head[m] != o->tail[l]) o->lo_idx[total++] = m;
        }
    }
    o->lo_ptr[L] = total;

    /* origin FIFOs: vehicles of each origin sorted by (departure step, id) */
    o->fifo_beg = (int32_t *)xcalloc(V + 1, sizeof(int32_t));
    o->fifo_end = (int32_t *)xcalloc(V, sizeof(int32_t));
    o->fifo_ptr = (int32_t *)xcalloc(V, sizeof(int32_t));
    o->fifo_list = (int32_t *)xcalloc(N, sizeof(int32_t));
    for (int i = 0; i < N; ++i) o->fifo_beg[o->origin[i] + 1]++;
    for (int n = 0; n < V; ++n) o->fifo_beg[n + 1] += o->fifo_beg[n];
    {
        int32_t *fill = (int32_t *)xcalloc(V, sizeof(int32_t));
        for (int i = 0; i < N; ++i) { int n = o->origin[i]; o->fifo_list[o->fifo_beg[n] + fill[n]++] = i; }
        free(fill);
    }
    g_sort_ctx = o;
    for (int n = 0; n < V; ++n) {
        o->fifo_end[n] = o->fifo_beg[n + 1];
        qsort(o->fifo_list + o->fifo_beg[n], (size_t)(o->fifo_end[n] - o->fifo_beg[n]), sizeof(int32_t), cmp_fifo);
    }

    /* derived per-link quantities, computed in the working precision */
    o->len = (real *)xcalloc(L, sizeof(real));
    o->s = (real *)xcalloc(L, sizeof(real));
    o->udt = (real *)xcalloc(L, sizeof(real));
    o->Uu = (real *)xcalloc(L, sizeof(real));
    o->Gg = (real *)xcalloc(L, sizeof(real));
    o->alpha_r = (real *)xcalloc(L, sizeof(real));
    o->half_len = (real *)xcalloc(L, sizeof(real));
    o->dtag = (real *)xcalloc(L, sizeof(real));
    o->cap_fx = (int64_t *)xcalloc(L, sizeof(int64_t));
    o->dn_fx = (int64_t)llrint((double)sc->dn * (double)FX_ONE);
    for (int j = 0; j < L; ++j) {
        real dn = (real)sc->dn, dt = (real)sc->dt;
        o->len[j] = (real)o->length[j];
        o->s[j] = dn / (real)o->kappa[j];                  /* jam spacing 1/kappa dn */
        o->udt[j] = (real)o->u[j] * dt;                    /* free-flow displacement */
        o->alpha_r[j] = (real)o->alpha[j];
        o->half_len[j] = o->len[j] * (real)0.5;            /* counter at the midpoint */
        o->dtag[j] = (real)sc->eps_tag * ((real)1 + o->len[j]);
        /* link utility: beta / c plus the static feature terms */
        real a = (real)o->beta[j] / (real)o->cost[j];
        real g = 0;
        for (int f = 0; f < F; ++f) {
            real wf = (real)o->w[f];
            a = a + wf * (real)o->phi[(size_t)j * F + f];
            g = g + wf * (real)o->psi[(size_t)j * F + f];
        }
        o->Uu[j] = a;
        o->Gg[j] = g;
        int64_t q = o->q_fx[j];
        o->cap_fx[j] = q > o->dn_fx ? q : o->dn_fx;
    }

    o->vlink = (int32_t *)xcalloc(N, sizeof(int32_t));
    o->ventry = (int32_t *)xcalloc(N, sizeof(int32_t));
    o->vx = (real *)xcalloc(N, sizeof(real));
    o->vseq = (int64_t *)xcalloc(N, sizeof(int64_t));
    o->credit = (int64_t *)xcalloc(L, sizeof(int64_t));
    o->exits = (int64_t *)xcalloc(L, sizeof(int64_t));
    o->acc_dx = (double *)xcalloc(L, sizeof(double));
    o->acc_n = (int64_t *)xcalloc(L, sizeof(int64_t));
    o->tt_sum = (int64_t *)xcalloc(L, sizeof(int64_t));
    o->tt_cnt = (int64_t *)xcalloc(L, sizeof(int64_t));
    o->C_prev = (int64_t *)xcalloc(L, sizeof(int64_t));
    o->rec_link_cand = (int32_t *)xcalloc(L, sizeof(int32_t));
    o->rec_link_target = (int32_t *)xcalloc(L, sizeof(int32_t));
    o->rec_node_cand = (int32_t *)xcalloc(V, sizeof(int32_t));
    o->rec_node_target = (int32_t *)xcalloc(V, sizeof(int32_t));
    o->rec_link_in = (int32_t *)xcalloc(L, sizeof(int32_t));
    o->rec_link_margin = (double *)xcalloc(L, sizeof(double));
    o->rec_node_margin = (double *)xcalloc(V, sizeof(double));
    o->rec_merge_margin = (double *)xcalloc(L, sizeof(double));
    o->rec_arr_margin = (double *)xcalloc(L, sizeof(double));
    o->rec_vac_margin = (double *)xcalloc(L, sizeof(double));
    o->mem_cnt = (int32_t *)xcalloc(L + 1, sizeof(int32_t));
    o->mem_ptr = (int32_t *)xcalloc(L + 1, sizeof(int32_t));
    o->mem_list = (int32_t *)xcalloc(N, sizeof(int32_t));
    o->xnew = (real *)xcalloc(N, sizeof(real));
    o->tagbuf = (int8_t *)xcalloc(N, sizeof(int8_t));
    o->route_len = (int32_t *)xcalloc(N, sizeof(int32_t));
    o->route_cap = (int32_t *)xcalloc(N, sizeof(int32_t));
    o->route_t = (int32_t **)xcalloc(N, sizeof(int32_t *));
    o->route_m = (int32_t **)xcalloc(N, sizeof(int32_t *));
    return o;
}

static void free_hist(or_sim *o)
{
    if (!o->hist) return;
    for (int t = 0; t < o->T; ++t) {
        or_hist *h = &o->hist[t];
        free(h->vlink); free(h->xpre); free(h->xpost); free(h->tag); free(h->fifo_ptr); free(h->cand);
    }
    free(o->hist);
    o->hist = NULL;
}

/* Reset to t = 0 with horizon T: every vehicle waits, every link is empty and
 * holds a full outflow credit. */
int or_reset(or_sim *o, int32_t T)
{
    const or_scenario *sc = &o->sc;
    int V = sc->V, L = sc->L, N = sc->N;
    free_hist(o);
    o->failed = 0;
    o->t = 0;
    o->T = T;
    o->n_bins = (T + sc->obs_every - 1) / sc->obs_every;
    for (int i = 0; i < N; ++i) { o->vlink[i] = VEH_WAITING; o->vx[i] = 0; o->vseq[i] = 0; o->ventry[i] = 0; o->route_len[i] = 0; }
    for (int n = 0; n < V; ++n) o->fifo_ptr[n] = o->fifo_beg[n];
    for (int j = 0; j < L; ++j) {
        o->credit[j] = o->cap_fx[j]; o->exits[j] = 0; o->acc_dx[j] = 0; o->acc_n[j] = 0;
        o->tt_sum[j] = 0; o->tt_cnt[j] = 0; o->C_prev[j] = 0;
    }
    free(o->out_counts); free(o->out_speed); free(o->out_tt);
    free(o->n_wait); free(o->n_on); free(o->n_arr);
    o->out_counts = (int32_t *)xcalloc((size_t)o->n_bins * L, sizeof(int32_t));
    o->out_speed = (double *)xcalloc((size_t)o->n_bins * L, sizeof(double));
    o->out_tt = (double *)xcalloc((size_t)o->n_bins * L, sizeof(double));
    o->n_wait = (int64_t *)xcalloc(T + 1, sizeof(int64_t));
    o->n_on = (int64_t *)xcalloc(T + 1, sizeof(int64_t));
    o->n_arr = (int64_t *)xcalloc(T + 1, sizeof(int64_t));
    o->cnt_wait = N; o->cnt_on = 0; o->cnt_arr = 0;
    o->n_wait[0] = N;
    if (o->keep_hist) o->hist = (or_hist *)xcalloc(T, sizeof(or_hist));
    return 0;
}

static void route_push(or_sim *o, int i, int t, int m)
{
    if (o->route_len[i] == o->route_cap[i]) {
        int nc = o->route_cap[i] ? 2 * o->route_cap[i] : 8;
        o->route_t[i] = (int32_t *)realloc(o->route_t[i], (size_t)nc * sizeof(int32_t));
        o->route_m[i] = (int32_t *)realloc(o->route_m[i], (size_t)nc * sizeof(int32_t));
        o->route_cap[i] = nc;
    }
    o->route_t[i][o->route_len[i]] = t;
    o->route_m[i][o->route_len[i]] = m;
    o->route_len[i]++;
}

/* members of every link, each list sorted by argsort(-x~) (SI-A) */
static void build_members(or_sim *o)
{
    int L = o->sc.L, N = o->sc.N;
    memset(o->mem_cnt, 0, (size_t)(L + 1) * sizeof(int32_t));
    for (int i = 0; i < N; ++i) if (o->vlink[i] >= 0) o->mem_cnt[o->vlink[i] + 1]++;
    o->mem_ptr[0] = 0;
    for (int j = 0; j < L; ++j) o->mem_ptr[j + 1] = o->mem_ptr[j] + o->mem_cnt[j + 1];
    memset(o->mem_cnt, 0, (size_t)(L + 1) * sizeof(int32_t));
    for (int i = 0; i < N; ++i) {
        int j = o->vlink[i];
        if (j >= 0) o->mem_list[o->mem_ptr[j] + o->mem_cnt[j]++] = i;
    }
    g_sort_ctx = o;
    for (int j = 0; j < L; ++j)
        qsort(o->mem_list + o->mem_ptr[j], (size_t)(o->mem_ptr[j + 1] - o->mem_ptr[j]), sizeof(int32_t), cmp_pos_desc);
}

static real rmin(real a, real b) { return a < b ? a : b; }
static real rmax(real a, real b) { return a > b ? a : b; }

/* utility of turning into link m for a vehicle bound for zone z */
static real utility(const or_sim *o, int m, int z)
{
    real df = (real)o->dest_feat[(size_t)z * o->sc.V + o->head[m]];
    real gd = o->Gg[m] * df;
    return o->Uu[m] + gd;
}

/* One time step phi = g o f.  Returns 0, or -1 on an internal inconsistency. */
int or_step(or_sim *o)
{
    const or_scenario *sc = &o->sc;
    int V = sc->V, L = sc->L, N = sc->N;
    int t = o->t;
    if (o->failed) return -1;
    if (t >= o->T) { fail(o, "step beyond horizon", t, o->T); return -1; }
    const real M = (real)sc->M;
    or_hist *H = o->keep_hist ? &o->hist[t] : NULL;

    build_members(o);
    if (H) {
        H->vlink = (int32_t *)xcalloc(N, sizeof(int32_t));
        H->xpre = (real *)xcalloc(N, sizeof(real));
        H->xpost = (real *)xcalloc(N, sizeof(real));
        H->tag = (int8_t *)xcalloc(N, sizeof(int8_t));
        H->fifo_ptr = (int32_t *)xcalloc(V, sizeof(int32_t));
        memcpy(H->vlink, o->vlink, (size_t)N * sizeof(int32_t));
        memcpy(H->xpre, o->vx, (size_t)N * sizeof(real));
        memcpy(H->fifo_ptr, o->fifo_ptr, (size_t)V * sizeof(int32_t));
    }

    /* ---------------- f: car-following on every link (SI-A) ---------------- */
    for (int j = 0; j < L; ++j) {
        int b = o->mem_ptr[j], e = o->mem_ptr[j + 1];
        for (int k = b; k < e; ++k) {
            int i = o->mem_list[k];
            real x = o->vx[i];
            real h = (k == b) ? M : o->vx[o->mem_list[k - 1]] - x;   /* headway h_i */
            real d = h - o->s[j];
            real dx_cong = rmax(d, (real)0);                         /* max(h - dn/kappa, 0) */
            real dx = rmin(o->udt[j], dx_cong);                      /* min(dx_free, dx_cong) */
            real xp = x + dx;                                        /* x' */
            real xn = rmin(xp, o->len[j]);                           /* min(x', x_limit) */
            o->xnew[i] = xn;
            int8_t tag;
            if (d <= o->dtag[j]) tag = TAG_STOP;
            else if (d >= o->udt[j] - o->dtag[j]) tag = TAG_FREE;
            else tag = TAG_CONG;
            o->tagbuf[i] = tag;
            o->acc_dx[j] += (double)(xn - x);
            o->acc_n[j] += 1;
        }
    }
    for (int j = 0; j < L; ++j)
        for (int k = o->mem_ptr[j]; k < o->mem_ptr[j + 1]; ++k) {
            int i = o->mem_list[k];
            o->vx[i] = o->xnew[i];
        }
    if (H) {
        memcpy(H->xpost, o->vx, (size_t)N * sizeof(real));
        memcpy(H->tag, o->tagbuf, (size_t)N * sizeof(int8_t));
    }

    /* ---------------- g: node model (SI-B) ---------------- */
    /* outflow credit */
    for (int j = 0; j < L; ++j) {
        int64_t c = o->credit[j] + o->q_fx[j];
        o->credit[j] = c < o->cap_fx[j] ? c : o->cap_fx[j];
    }
    /* vacancy: rearmost position X_min > 1/kappa dn, or an empty link */
    char *vacant = (char *)xcalloc(L, 1);
    for (int j = 0; j < L; ++j) {
        int b = o->mem_ptr[j], e = o->mem_ptr[j + 1];
        o->rec_vac_margin[j] = INFINITY;
        o->rec_arr_margin[j] = INFINITY;
        if (b == e) { vacant[j] = 1; continue; }
        real xm = o->vx[o->mem_list[b]];
        for (int k = b; k < e; ++k) xm = rmin(xm, o->vx[o->mem_list[k]]);
        vacant[j] = xm > o->s[j];
        /* distances of the two position comparisons of this step from their
         * thresholds (near-tie flags): rearmost vehicle vs the jam spacing, leader
         * vs the arrival line */
        o->rec_vac_margin[j] = (double)xm - (double)o->s[j];
        o->rec_arr_margin[j] = (double)o->vx[o->mem_list[b]] - ((double)o->len[j] - (double)sc->eps_arr);
    }
    /* candidates: arrived leaders with credit, and the heads of origin queues */
    int max_c = L + V;
    or_cand *cand = (or_cand *)xcalloc(max_c, sizeof(or_cand));
    int nc = 0;
    for (int j = 0; j < L; ++j) { o->rec_link_cand[j] = -1; o->rec_link_target[j] = TGT_NONE; o->rec_link_in[j] = -1; o->rec_link_margin[j] = INFINITY; o->rec_merge_margin[j] = INFINITY; }
    for (int n = 0; n < V; ++n) { o->rec_node_cand[n] = -1; o->rec_node_target[n] = TGT_NONE; o->rec_node_margin[n] = INFINITY; }
    for (int j = 0; j < L; ++j) {
        int b = o->mem_ptr[j], e = o->mem_ptr[j + 1];
        int arrived = -1, n_arr = 0;
        for (int k = b; k < e; ++k) {
            int i = o->mem_list[k];
            if (o->vx[i] >= o->len[j] - (real)sc->eps_arr) { if (arrived < 0) arrived = i; n_arr++; }
        }
        if (n_arr > 1) { fail(o, "several vehicles arrived on one link", j, n_arr); free(vacant); free(cand); return -1; }
        if (arrived < 0 || o->credit[j] < o->dn_fx) continue;
        or_cand *c = &cand[nc++];
        c->vid = arrived; c->src_link = j; c->src_node = o->head[j]; c->x = o->vx[arrived];
        c->target = TGT_NONE; c->slot = -1; c->valid = 0; c->won = 0;
    }
    for (int n = 0; n < V; ++n) {
        int p = o->fifo_ptr[n];
        if (p >= o->fifo_end[n]) continue;
        int i = o->fifo_list[p];
        if (o->dep_step[i] > t) continue;
        or_cand *c = &cand[nc++];
        c->vid = i; c->src_link = -1; c->src_node = n; c->x = 0;
        c->target = TGT_NONE; c->slot = -1; c->valid = 0; c->won = 0;
    }
    /* link choice: argmax over the choice set of V + g (Eqs. softmax, gumbel,
     * straightthrough: the one-hot of the Gumbel-softmax sample) */
    for (int ci = 0; ci < nc; ++ci) {
        or_cand *c = &cand[ci];
        int i = c->vid, z = o->dest_zone[i];
        int node = c->src_node;
        if (o->node_zone[node] == z) { c->target = TGT_SINK; continue; }
        const int32_t *set; int deg;
        if (c->src_link >= 0) { set = o->lo_idx + o->lo_ptr[c->src_link]; deg = o->lo_ptr[c->src_link + 1] - o->lo_ptr[c->src_link]; }
        else { set = o->no_idx + o->no_ptr[node]; deg = o->no_ptr[node + 1] - o->no_ptr[node]; }
        int best = -1; real bk = 0, second = -INFINITY;
        for (int k = 0; k < deg; ++k) {
            real key = utility(o, set[k], z) + gumbel(sc->seed, sc->scenario_id, i, t, 0, k);
            if (best < 0 || key > bk) { if (best >= 0) second = bk; best = k; bk = key; }
            else if (key > second) second = key;
        }
        c->slot = best;
        c->target = set[best];
        c->valid = vacant[c->target];
        if (c->src_link >= 0) o->rec_link_margin[c->src_link] = (double)(bk - second);
        else o->rec_node_margin[node] = (double)(bk - second);
    }
    /* merge: per target link, argmax over its valid candidates of alpha_src + g'
     * (ties to the lowest vehicle id) */
    int32_t *winner = (int32_t *)xcalloc(L, sizeof(int32_t));
    real *wkey = (real *)xcalloc(L, sizeof(real));
    real *wsecond = (real *)xcalloc(L, sizeof(real));
    for (int j = 0; j < L; ++j) { winner[j] = -1; wsecond[j] = -INFINITY; }
    for (int ci = 0; ci < nc; ++ci) {
        or_cand *c = &cand[ci];
        if (c->target < 0 || !c->valid) continue;
        real a = c->src_link >= 0 ? o->alpha_r[c->src_link] : (real)sc->alpha_origin;
        real key = a + gumbel(sc->seed, sc->scenario_id, c->vid, t, 1, 0);
        int m = c->target;
        int w = winner[m];
        if (w < 0) { winner[m] = ci; wkey[m] = key; }
        else if (key > wkey[m] || (key == wkey[m] && c->vid < cand[w].vid)) {
            wsecond[m] = wkey[m]; winner[m] = ci; wkey[m] = key;
        } else if (key > wsecond[m]) wsecond[m] = key;
    }
    for (int ci = 0; ci < nc; ++ci) {
        or_cand *c = &cand[ci];
        if (c->src_link >= 0) { o->rec_link_cand[c->src_link] = c->vid; o->rec_link_target[c->src_link] = (c->target >= 0 && !c->valid) ? TGT_BLOCKED : c->target; }
        else { o->rec_node_cand[c->src_node] = c->vid; o->rec_node_target[c->src_node] = (c->target >= 0 && !c->valid) ? TGT_BLOCKED : c->target; }
    }
    /* apply all transfers simultaneously (Eq. transfer) */
    for (int m = 0; m < L; ++m) {
        if (winner[m] < 0) continue;
        cand[winner[m]].won = 1;
        o->rec_merge_margin[m] = (double)(wkey[m] - wsecond[m]);
    }
    for (int ci = 0; ci < nc; ++ci) {
        or_cand *c = &cand[ci];
        int leaves = c->target == TGT_SINK || c->won;
        if (!leaves) continue;
        int i = c->vid;
        if (c->src_link >= 0) {
            int j = c->src_link;
            o->credit[j] -= o->dn_fx;
            o->exits[j] += 1;
            o->tt_sum[j] += (int64_t)(t + 1 - o->ventry[i]);
            o->tt_cnt[j] += 1;
        } else {
            o->fifo_ptr[c->src_node]++;
            o->cnt_wait--;
            o->cnt_on++;
        }
        if (c->target == TGT_SINK) {
            o->vlink[i] = VEH_ARRIVED; o->vx[i] = 0;
            o->cnt_on--; o->cnt_arr++;
        } else {
            int m = c->target;
            o->vlink[i] = m; o->vx[i] = 0; o->vseq[i] = t + 1; o->ventry[i] = t + 1;
            o->rec_link_in[m] = i;
            route_push(o, i, t, m);
        }
    }
    if (H) { H->cand = cand; H->n_cand = nc; } else free(cand);
    free(winner); free(wkey); free(wsecond); free(vacant);

    /* ---------------- counters and observation (SI-D) ---------------- */
    o->t = t + 1;
    o->n_wait[t + 1] = o->cnt_wait; o->n_on[t + 1] = o->cnt_on; o->n_arr[t + 1] = o->cnt_arr;
    if ((t + 1) % sc->obs_every == 0 || t + 1 == o->T) {
        int bin = t / sc->obs_every;
        build_members(o);
        for (int j = 0; j < L; ++j) {
            int64_t past = 0;
            for (int k = o->mem_ptr[j]; k < o->mem_ptr[j + 1]; ++k)
                if (o->vx[o->mem_list[k]] >= o->half_len[j]) past++;
            int64_t C = o->exits[j] + past;
            o->out_counts[(size_t)bin * L + j] = (int32_t)(C - o->C_prev[j]);
            o->C_prev[j] = C;
            o->out_speed[(size_t)bin * L + j] = o->acc_n[j] ? o->acc_dx[j] / ((double)o->acc_n[j] * (double)sc->dt) : 0.0;
            o->out_tt[(size_t)bin * L + j] = o->tt_cnt[j] ? (double)o->tt_sum[j] * (double)sc->dt / (double)o->tt_cnt[j] : 0.0;
            o->acc_dx[j] = 0; o->acc_n[j] = 0; o->tt_sum[j] = 0; o->tt_cnt[j] = 0;
        }
    }
    return 0;
}

int or_run(or_sim *o, int32_t n_steps)
{
    for (int k = 0; k < n_steps; ++k) if (or_step(o)) return -1;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Accessors                                                                  */
/* ------------------------------------------------------------------------- */
int32_t or_time(const or_sim *o) { return o->t; }
int32_t or_n_bins(const or_sim *o) { return o->n_bins; }

void or_outputs(const or_sim *o, int32_t *counts, double *speed, double *tt,
                int64_t *n_wait, int64_t *n_on, int64_t *n_arr)
{
    size_t nb = (size_t)o->n_bins * o->sc.L;
    if (counts) memcpy(counts, o->out_counts, nb * sizeof(int32_t));
    if (speed) memcpy(speed, o->out_speed, nb * sizeof(double));
    if (tt) memcpy(tt, o->out_tt, nb * sizeof(double));
    if (n_wait) memcpy(n_wait, o->n_wait, (size_t)(o->T + 1) * sizeof(int64_t));
    if (n_on) memcpy(n_on, o->n_on, (size_t)(o->T + 1) * sizeof(int64_t));
    if (n_arr) memcpy(n_arr, o->n_arr, (size_t)(o->T + 1) * sizeof(int64_t));
}

/* State in the exchange layout: per vehicle link (-1 waiting, -2 arrived),
 * position, rank in its link queue (0 = leader) and entry step; per link credit
 * and cumulative exits; per node the origin-queue pointer as an offset. */
void or_export_state(or_sim *o, int32_t *veh_link, double *veh_pos, int32_t *veh_rank,
                     int32_t *veh_entry, int64_t *link_credit, int64_t *link_exits,
                     int32_t *fifo_off)
{
    int N = o->sc.N, L = o->sc.L, V = o->sc.V;
    build_members(o);
    for (int i = 0; i < N; ++i) {
        if (veh_link) veh_link[i] = o->vlink[i];
        if (veh_pos) veh_pos[i] = (double)o->vx[i];
        if (veh_rank) veh_rank[i] = -1;
        if (veh_entry) veh_entry[i] = o->ventry[i];
    }
    if (veh_rank)
        for (int j = 0; j < L; ++j)
            for (int k = o->mem_ptr[j]; k < o->mem_ptr[j + 1]; ++k) veh_rank[o->mem_list[k]] = k - o->mem_ptr[j];
    for (int j = 0; j < L; ++j) {
        if (link_credit) link_credit[j] = o->credit[j];
        if (link_exits) link_exits[j] = o->exits[j];
    }
    if (fifo_off) for (int n = 0; n < V; ++n) fifo_off[n] = o->fifo_ptr[n] - o->fifo_beg[n];
}

/* Decisions of the last step: candidate vehicle and target per link and per
 * origin node (-1 none, -2 sink, -3 blocked by vacancy), the vehicle that
 * entered each link, and the top-2 key gaps used to flag near-ties. */
void or_records(const or_sim *o, int32_t *link_cand, int32_t *link_target, int32_t *node_cand,
                int32_t *node_target, int32_t *link_in, double *link_margin,
                double *node_margin, double *merge_margin)
{
    int L = o->sc.L, V = o->sc.V;
    if (link_cand) memcpy(link_cand, o->rec_link_cand, (size_t)L * sizeof(int32_t));
    if (link_target) memcpy(link_target, o->rec_link_target, (size_t)L * sizeof(int32_t));
    if (node_cand) memcpy(node_cand, o->rec_node_cand, (size_t)V * sizeof(int32_t));
    if (node_target) memcpy(node_target, o->rec_node_target, (size_t)V * sizeof(int32_t));
    if (link_in) memcpy(link_in, o->rec_link_in, (size_t)L * sizeof(int32_t));
    if (link_margin) memcpy(link_margin, o->rec_link_margin, (size_t)L * sizeof(double));
    if (node_margin) memcpy(node_margin, o->rec_node_margin, (size_t)V * sizeof(double));
    if (merge_margin) memcpy(merge_margin, o->rec_merge_margin, (size_t)L * sizeof(double));
}

/* Position margins of the last step, for flagging near-ties of the two position
 * comparisons of the node model: arr_margin[j] = x_lead - (L_j - eps_arr) of
 * link j's leader after f (Alg. S2 arrival test), vac_margin[j] = x_min - 1/kappa
 * dn of its rearmost vehicle after f (vacancy test); INFINITY for empty links. */
void or_position_margins(const or_sim *o, double *arr_margin, double *vac_margin)
{
    int L = o->sc.L;
    if (arr_margin) memcpy(arr_margin, o->rec_arr_margin, (size_t)L * sizeof(double));
    if (vac_margin) memcpy(vac_margin, o->rec_vac_margin, (size_t)L * sizeof(double));
}

/* Replace the state by a given one at step t of the current horizon (the layout
 * of or_export_state; positions are rounded to the working precision), so that
 * a lockstep comparison can continue from another simulator's state.  The
 * observation bin containing t restarts at t: its counts, speeds and travel
 * times cover [t, bin end).  Forward-only runs (no history).  Returns 0 or -1
 * (state inconsistent: a field out of range, ranks that are not the order of
 * the positions, waiting vehicles that do not match the origin queues). */
int or_import_state(or_sim *o, int32_t t, const int32_t *veh_link, const double *veh_pos,
                    const int32_t *veh_rank, const int32_t *veh_entry, const int64_t *link_credit,
                    const int64_t *link_exits, const int32_t *fifo_off)
{
    const int N = o->sc.N, L = o->sc.L, V = o->sc.V;
    if (o->keep_hist) { fail(o, "state import is for runs without history", t, 0); return -1; }
    if (t < 0 || t > o->T) { fail(o, "import step outside the horizon", t, o->T); return -1; }
    int64_t queued = 0;
    for (int n = 0; n < V; ++n) {
        int len = o->fifo_end[n] - o->fifo_beg[n];
        if (fifo_off[n] < 0 || fifo_off[n] > len) { fail(o, "origin queue offset out of range", n, fifo_off[n]); return -1; }
        o->fifo_ptr[n] = o->fifo_beg[n] + fifo_off[n];
        queued += len - fifo_off[n];
    }
    o->cnt_wait = o->cnt_on = o->cnt_arr = 0;
    for (int i = 0; i < N; ++i) {
        int j = veh_link[i];
        if (j < VEH_ARRIVED || j >= L) { fail(o, "vehicle link out of range", i, j); return -1; }
        o->vlink[i] = j;
        if (j == VEH_WAITING) { o->cnt_wait++; o->vx[i] = 0; continue; }
        if (j == VEH_ARRIVED) { o->cnt_arr++; o->vx[i] = 0; continue; }
        if (!(veh_pos[i] >= 0.0 && veh_pos[i] <= (double)o->length[j])) { fail(o, "position outside its link", i, j); return -1; }
        o->cnt_on++;
        o->vx[i] = (real)veh_pos[i];
        o->ventry[i] = veh_entry[i];
        o->vseq[i] = veh_entry[i];
    }
    if (queued != o->cnt_wait) { fail(o, "waiting vehicles do not match the origin queues", (int)queued, (int)o->cnt_wait); return -1; }
    for (int n = 0; n < V; ++n)
        for (int p = o->fifo_ptr[n]; p < o->fifo_end[n]; ++p)
            if (o->vlink[o->fifo_list[p]] != VEH_WAITING) { fail(o, "queued vehicle not waiting", n, o->fifo_list[p]); return -1; }
    build_members(o);
    for (int j = 0; j < L; ++j) {
        int64_t past = 0;
        for (int k = o->mem_ptr[j]; k < o->mem_ptr[j + 1]; ++k) {
            int i = o->mem_list[k];
            if (veh_rank[i] != k - o->mem_ptr[j]) { fail(o, "ranks are not the order of the positions", i, j); return -1; }
            if (o->vx[i] >= o->half_len[j]) past++;
        }
        o->credit[j] = link_credit[j];
        o->exits[j] = link_exits[j];
        o->C_prev[j] = link_exits[j] + past;
        o->acc_dx[j] = 0; o->acc_n[j] = 0; o->tt_sum[j] = 0; o->tt_cnt[j] = 0;
    }
    o->t = t;
    o->n_wait[t] = o->cnt_wait; o->n_on[t] = o->cnt_on; o->n_arr[t] = o->cnt_arr;
    o->failed = 0;
    return 0;
}

/* Route log of one vehicle: steps and links of its entries, in order. */
int32_t or_route(const or_sim *o, int32_t i, int32_t *steps, int32_t *links, int32_t cap)
{
    int n = o->route_len[i];
    for (int k = 0; k < n && k < cap; ++k) { if (steps) steps[k] = o->route_t[i][k]; if (links) links[k] = o->route_m[i][k]; }
    return n;
}

void or_destroy(or_sim *o)
{
    if (!o) return;
    free_hist(o);
    free(o->tail); free(o->head); free(o->node_zone); free(o->origin); free(o->dest_zone);
    free(o->dep_step); free(o->od); free(o->q_fx); free(o->length); free(o->u); free(o->kappa);
    free(o->alpha); free(o->beta); free(o->cost); free(o->phi); free(o->psi); free(o->w);
    free(o->dest_feat); free(o->od_lambda);
    free(o->len); free(o->s); free(o->udt); free(o->Uu); free(o->Gg); free(o->alpha_r);
    free(o->half_len); free(o->dtag); free(o->cap_fx);
    free(o->lo_ptr); free(o->lo_idx); free(o->no_ptr); free(o->no_idx);
    free(o->fifo_beg); free(o->fifo_end); free(o->fifo_list); free(o->fifo_ptr);
    free(o->vlink); free(o->ventry); free(o->vx); free(o->vseq); free(o->credit); free(o->exits);
    free(o->acc_dx); free(o->acc_n); free(o->tt_sum); free(o->tt_cnt); free(o->C_prev);
    free(o->out_counts); free(o->out_speed); free(o->out_tt); free(o->n_wait); free(o->n_on); free(o->n_arr);
    free(o->rec_link_cand); free(o->rec_link_target); free(o->rec_node_cand); free(o->rec_node_target);
    free(o->rec_link_in); free(o->rec_link_margin); free(o->rec_node_margin); free(o->rec_merge_margin);
    free(o->rec_arr_margin); free(o->rec_vac_margin);
    free(o->mem_cnt); free(o->mem_ptr); free(o->mem_list); free(o->xnew); free(o->tagbuf);
    for (int i = 0; i < o->sc.N; ++i) { free(o->route_t[i]); free(o->route_m[i]); }
    free(o->route_len); free(o->route_cap); free(o->route_t); free(o->route_m);
    free(o);
}

/* ------------------------------------------------------------------------- */
/* Reverse mode of the straight-through / trajectory-grafting surrogate       */
/* ------------------------------------------------------------------------- */
/*
 * Every discrete decision of the recorded rollout is frozen (argmaxes, masks,
 * comparisons, car-following branch tags) and every stop_gradient(v) is the
 * recorded value; the result is the derivative jax.grad takes of the dense
 * formulation (SI-A Alg. S1, SI-B Alg. S2) with the readings in the file header.
 * The dense state X[i, j] (agent i on link j, -M elsewhere) is represented by
 *   xbar[i]     the adjoint of agent i's valid entry (its current link, or its
 *               origin queue = a virtual inflow link of length 0), and
 *   eadj[i][r]  the adjoint of X[i, m_r] right after agent i's r-th entry: by
 *               the identity of an invalid slot through time, the adjoint of
 *               the slot (i, m) at any earlier time since i last left m is the
 *               adjoint right after i's next entry into m (0 if it never enters).
 * Reverse step t, from the state after the step back to its start:
 *   (1) observation at t+1 (SI-D): dC_j/dx_i = s sigma (1 - sigma), s = 5/L_j;
 *       demand weights 1 + (lambda - sg lambda)/lambda give dC/dlambda;
 *   (2) node model (SI-B): for the valid candidates of each target m,
 *       abar_i = M (Ebar_i(m) - Xbar_i(l_i)) - x_i Xbar_i(l_i)   (Eq. transfer),
 *       merge softmax pi' over (alpha_src + g')/tau -> alpha, lbar;
 *       link-choice softmax pi over (V + g)/tau -> U_m = beta/c + w.phi, G_m = w.psi;
 *       the winner's old entry receives its new entry's adjoint (grafting);
 *   (3) car-following (SI-A) by tag: free x' = x + u dt, cong x' = x_lead - s,
 *       stop x' = x; the TG clip passes the adjoint unchanged.
 */
static double sigmoid_d(double z) { return 1.0 / (1.0 + exp(-z)); }

/* adjoint right after vehicle i's first entry into link m at a step > t
 * (entries are in step order); 0 if it never enters m again */
static double next_entry_adj(const or_sim *o, double **eadj, int i, int m, int t)
{
    for (int r = 0; r < o->route_len[i]; ++r)
        if (o->route_t[i][r] > t && o->route_m[i][r] == m) return eadj[i][r];
    return 0.0;
}

/* Relaxed link-choice weights of candidate c at step t: pi = softmax((V + g)/tau)
 * over its choice set (SI-B Eqs. softmax and gumbel), the weights whose
 * straight-through one-hot the forward takes (Eq. straigththrough).  Writes deg
 * weights to pk and the choice set to *set_out; returns deg. */
static int choice_weights(const or_sim *o, const or_cand *c, int t, double tau, double *pk,
                          const int32_t **set_out)
{
    const or_scenario *sc = &o->sc;
    const int i = c->vid, z = o->dest_zone[i];
    const int32_t *set; int deg;
    if (c->src_link >= 0) { set = o->lo_idx + o->lo_ptr[c->src_link]; deg = o->lo_ptr[c->src_link + 1] - o->lo_ptr[c->src_link]; }
    else { set = o->no_idx + o->no_ptr[c->src_node]; deg = o->no_ptr[c->src_node + 1] - o->no_ptr[c->src_node]; }
    double pmax = -INFINITY, ps = 0.0;
    for (int q = 0; q < deg; ++q) {
        pk[q] = ((double)utility(o, set[q], z) + (double)gumbel(sc->seed, sc->scenario_id, i, t, 0, q)) / tau;
        if (pk[q] > pmax) pmax = pk[q];
    }
    for (int q = 0; q < deg; ++q) { pk[q] = exp(pk[q] - pmax); ps += pk[q]; }
    for (int q = 0; q < deg; ++q) pk[q] /= ps;
    if (set_out) *set_out = set;
    return deg;
}

/* Relaxed merge weights of a target link at step t: pi' = softmax((alpha_src +
 * g')/tau) over its valid candidates (SI-B "Merge choice"), given as the nm
 * candidate indices idx (in candidate order).  Writes the weights to w. */
static void merge_weights(const or_sim *o, const or_cand *cand, const int *idx, int nm, int t, double tau,
                          double *w)
{
    const or_scenario *sc = &o->sc;
    double kmax = -INFINITY, zs = 0.0;
    for (int k = 0; k < nm; ++k) {
        const or_cand *c = &cand[idx[k]];
        const double al = c->src_link >= 0 ? (double)o->alpha[c->src_link] : (double)sc->alpha_origin;
        w[k] = (al + (double)gumbel(sc->seed, sc->scenario_id, c->vid, t, 1, 0)) / tau;
        if (w[k] > kmax) kmax = w[k];
    }
    for (int k = 0; k < nm; ++k) { w[k] = exp(w[k] - kmax); zs += w[k]; }
    for (int k = 0; k < nm; ++k) w[k] /= zs;
}

/* Valid candidates of every target link, in candidate order: those of link m
 * are idx[ptr[m] .. ptr[m + 1]).  ptr has L + 1 entries, idx nc. */
static void merge_lists(const or_sim *o, const or_cand *cand, int nc, int *ptr, int *idx)
{
    const int L = o->sc.L;
    memset(ptr, 0, (size_t)(L + 1) * sizeof(int));
    for (int ci = 0; ci < nc; ++ci)
        if (cand[ci].target >= 0 && cand[ci].valid) ptr[cand[ci].target + 1]++;
    for (int m = 0; m < L; ++m) ptr[m + 1] += ptr[m];
    int *fill = (int *)xcalloc(L, sizeof(int));
    for (int ci = 0; ci < nc; ++ci)
        if (cand[ci].target >= 0 && cand[ci].valid) { int m = cand[ci].target; idx[ptr[m] + fill[m]++] = ci; }
    free(fill);
}

/* The relaxed weights of a recorded rollout (history needed) at temperature tau,
 * exported to pin them: the link-choice weights of the candidate at source link
 * src_link (or origin node src_node when src_link < 0) at step t, with the
 * forward's chosen slot in *slot; returns the choice-set size, 0 when that
 * source had no choosing candidate at t, -1 without history. */
int32_t or_choice_weights(const or_sim *o, int32_t t, int32_t src_link, int32_t src_node, double tau,
                          double *pi, int32_t *slot)
{
    if (!o->keep_hist || !o->hist || t < 0 || t >= o->t) return -1;
    const or_hist *H = &o->hist[t];
    for (int ci = 0; ci < H->n_cand; ++ci) {
        const or_cand *c = &H->cand[ci];
        if (src_link >= 0 ? c->src_link != src_link : (c->src_link >= 0 || c->src_node != src_node)) continue;
        if (c->slot < 0) return 0;                           /* left to the sink: no choice */
        if (slot) *slot = c->slot;
        return choice_weights(o, c, t, tau, pi, NULL);
    }
    return 0;
}

/* The merge weights of target link m at step t at temperature tau, with each
 * candidate's vehicle id and whether it won; returns their number (0 without
 * valid candidates, -1 without history).  vid / won need room for L + V. */
int32_t or_merge_weights(const or_sim *o, int32_t t, int32_t m, double tau, double *w, int32_t *vid,
                         int32_t *won)
{
    if (!o->keep_hist || !o->hist || t < 0 || t >= o->t) return -1;
    const or_hist *H = &o->hist[t];
    int *ptr = (int *)xcalloc(o->sc.L + 1, sizeof(int));
    int *idx = (int *)xcalloc(H->n_cand, sizeof(int));
    merge_lists(o, H->cand, H->n_cand, ptr, idx);
    const int nm = ptr[m + 1] - ptr[m];
    merge_weights(o, H->cand, idx + ptr[m], nm, t, tau, w);
    for (int k = 0; k < nm; ++k) { vid[k] = H->cand[idx[ptr[m] + k]].vid; won[k] = H->cand[idx[ptr[m] + k]].won; }
    free(ptr); free(idx);
    return nm;
}

int or_backward(or_sim *o, const double *ybar, const double *xbarT, int no_tg,
                double *d_u, double *d_kappa, double *d_alpha, double *d_alpha_origin,
                double *d_beta, double *d_cost, double *d_w, double *d_lambda)
{
    const or_scenario *sc = &o->sc;
    const int N = sc->N, L = sc->L, V = sc->V, F = sc->F, T = o->T;
    if (!o->keep_hist || !o->hist || o->t != T) { fail(o, "backward needs a full recorded rollout", o->t, T); return -1; }
    const double M = (double)sc->M, tau = (double)sc->tau, dt = (double)sc->dt;
    const int nb = o->n_bins;
    double *xbar = (double *)xcalloc(N, sizeof(double));
    double **eadj = (double **)xcalloc(N, sizeof(double *));
    for (int i = 0; i < N; ++i) eadj[i] = (double *)xcalloc(o->route_len[i] ? o->route_len[i] : 1, sizeof(double));
    double *gu = (double *)xcalloc(L, sizeof(double)), *gs = (double *)xcalloc(L, sizeof(double));
    double *ga = (double *)xcalloc(L, sizeof(double)), *gU = (double *)xcalloc(L, sizeof(double));
    double *gG = (double *)xcalloc(L, sizeof(double)), *glam = (double *)xcalloc(sc->n_od ? sc->n_od : 1, sizeof(double));
    double gao = 0.0;
    /* adjoint of C_j at the end of each bin: Cbar[b][j] = ybar[b][j] - ybar[b+1][j] */
    double *Cbar = (double *)xcalloc((size_t)nb * L, sizeof(double));
    for (int b = 0; b < nb; ++b)
        for (int j = 0; j < L; ++j)
            Cbar[(size_t)b * L + j] = ybar[(size_t)b * L + j] - (b + 1 < nb ? ybar[(size_t)(b + 1) * L + j] : 0.0);
    /* exits at step t count in every C_j(t_b) with t_b >= t + 1: suffix of Cbar */
    double *Csuf = (double *)xcalloc((size_t)(nb + 1) * L, sizeof(double));
    for (int b = nb - 1; b >= 0; --b)
        for (int j = 0; j < L; ++j) Csuf[(size_t)b * L + j] = Csuf[(size_t)(b + 1) * L + j] + Cbar[(size_t)b * L + j];
    if (xbarT)
        for (int i = 0; i < N; ++i) if (o->vlink[i] >= 0) xbar[i] = xbarT[i];
    int *order = (int *)xcalloc(N, sizeof(int));
    int *cnt = (int *)xcalloc(L + 1, sizeof(int));
    double *xn = (double *)xcalloc(N, sizeof(double));

    for (int t = T - 1; t >= 0; --t) {
        or_hist *H = &o->hist[t];
        const int32_t *vl1 = (t + 1 < T) ? o->hist[t + 1].vlink : o->vlink;
        const real *x1 = (t + 1 < T) ? o->hist[t + 1].xpre : o->vx;
        /* (1) observation at time t + 1 */
        if ((t + 1) % sc->obs_every == 0 || t + 1 == T) {
            const int b = t / sc->obs_every;
            for (int i = 0; i < N; ++i) {
                const int j = vl1[i];
                if (j < 0) continue;
                const double cb = Cbar[(size_t)b * L + j];
                const double len = (double)o->length[j], s5 = 5.0 / len;
                const double x = (double)x1[i];
                const double sg = sigmoid_d(s5 * (x - 0.5 * len));
                xbar[i] += cb * s5 * sg * (1.0 - sg);
                if (x >= (double)o->half_len[j]) glam[o->od[i]] += cb / (double)o->od_lambda[o->od[i]];
            }
        }
        /* (2) node model of step t */
        or_cand *cand = H->cand;
        const int nc = H->n_cand;
        /* entries of step t: record the adjoint right after the entry */
        for (int ci = 0; ci < nc; ++ci) {
            or_cand *c = &cand[ci];
            if (!c->won) continue;
            const int i = c->vid;
            for (int r = 0; r < o->route_len[i]; ++r)
                if (o->route_t[i][r] == t) { eadj[i][r] = xbar[i]; break; }
        }
        /* exits of step t (transfers and sinks): demand weight of the exit count */
        for (int ci = 0; ci < nc; ++ci) {
            or_cand *c = &cand[ci];
            if (c->src_link < 0 || !(c->won || c->target == TGT_SINK)) continue;
            const int b0 = t / sc->obs_every;      /* bins whose end is >= t + 1 */
            glam[o->od[c->vid]] += Csuf[(size_t)b0 * L + c->src_link] / (double)o->od_lambda[o->od[c->vid]];
        }
        double *wm = (double *)xcalloc(nc ? nc : 1, sizeof(double));
        double *abar = (double *)xcalloc(nc ? nc : 1, sizeof(double));
        int *mptr = (int *)xcalloc(L + 1, sizeof(int));
        int *midx = (int *)xcalloc(nc ? nc : 1, sizeof(int));
        merge_lists(o, cand, nc, mptr, midx);
        int maxdeg = 1;
        for (int n = 0; n < V; ++n) if (o->no_ptr[n + 1] - o->no_ptr[n] > maxdeg) maxdeg = o->no_ptr[n + 1] - o->no_ptr[n];
        double *pk = (double *)xcalloc(maxdeg, sizeof(double));
        for (int m = 0; m < L; ++m) {
            /* merge softmax over the valid candidates of target m */
            const int nm = mptr[m + 1] - mptr[m];
            if (nm == 0) continue;
            const int *idx = midx + mptr[m];
            merge_weights(o, cand, idx, nm, t, tau, wm);
            double S = 0.0;
            for (int k = 0; k < nm; ++k) {
                or_cand *c = &cand[idx[k]];
                const int i = c->vid;
                double Enew, Xold;
                if (c->won) {
                    int rw = -1;
                    for (int r = 0; r < o->route_len[i]; ++r) if (o->route_t[i][r] == t) { rw = r; break; }
                    Enew = xbar[i];
                    Xold = 0.0;
                    if (c->src_link >= 0)
                        for (int r = rw + 1; r < o->route_len[i]; ++r)
                            if (o->route_m[i][r] == c->src_link) { Xold = eadj[i][r]; break; }
                } else {
                    Enew = next_entry_adj(o, eadj, i, m, t);
                    Xold = xbar[i];
                }
                abar[k] = M * (Enew - Xold) - (double)c->x * Xold;
                S += wm[k] * abar[k];
            }
            for (int k = 0; k < nm; ++k) {
                or_cand *c = &cand[idx[k]];
                const double vbar = wm[k] * (abar[k] - S) / tau;          /* adjoint of V'_i = p_i */
                const double al = c->src_link >= 0 ? (double)o->alpha[c->src_link] : (double)sc->alpha_origin;
                if (c->src_link >= 0) ga[c->src_link] += vbar; else gao += vbar;
                const double lbar = al * vbar;                            /* adjoint of l_i at m */
                /* link choice of this candidate: pi = softmax((V + g)/tau) over its choice set */
                const int z = o->dest_zone[c->vid];
                const int32_t *set;
                const int deg = choice_weights(o, c, t, tau, pk, &set);
                for (int q = 0; q < deg; ++q) {
                    const double Vbar = pk[q] * ((q == c->slot ? 1.0 : 0.0) - pk[c->slot]) * lbar / tau;
                    const int mq = set[q];
                    gU[mq] += Vbar;
                    gG[mq] += Vbar * (double)o->dest_feat[(size_t)z * V + o->head[mq]];
                }
            }
        }
        free(wm); free(abar); free(mptr); free(midx); free(pk);
        /* grafting: a winner's old entry gets its new entry's adjoint (xbar[i]
         * carries over unchanged); without TG the old entry gets nothing */
        if (no_tg)
            for (int ci = 0; ci < nc; ++ci) if (cand[ci].won) xbar[cand[ci].vid] = 0.0;
        /* (3) car-following of step t, per link in the order of argsort(-x) */
        memset(cnt, 0, (size_t)(L + 1) * sizeof(int));
        for (int i = 0; i < N; ++i) if (H->vlink[i] >= 0) cnt[H->vlink[i] + 1]++;
        for (int j = 0; j < L; ++j) cnt[j + 1] += cnt[j];
        {
            int *fill = (int *)xcalloc(L, sizeof(int));
            for (int i = 0; i < N; ++i) {
                const int j = H->vlink[i];
                if (j >= 0) order[cnt[j] + fill[j]++] = i;
            }
            free(fill);
        }
        for (int j = 0; j < L; ++j) {
            const int b = cnt[j], e = cnt[j + 1];
            /* sort this link's vehicles by time-t position, descending */
            for (int a = b + 1; a < e; ++a) {
                int v = order[a], q = a - 1;
                while (q >= b && (H->xpre[order[q]] < H->xpre[v])) { order[q + 1] = order[q]; --q; }
                order[q + 1] = v;
            }
            for (int q = b; q < e; ++q) {
                const int i = order[q];
                double g = xbar[i];
                if (no_tg) {
                    const real xa = (q == b) ? (real)sc->M : H->xpre[order[q - 1]] - H->xpre[i];
                    const real dd = xa - o->s[j];
                    const real dx = rmin(o->udt[j], rmax(dd, (real)0));
                    if (H->xpre[i] + dx > o->len[j]) g = 0.0;         /* clipped: constant L */
                }
                xn[i] = g;
            }
            for (int q = b; q < e; ++q) {
                const int i = order[q];
                const int tag = H->tag[i];
                double pre = (tag == TAG_CONG) ? 0.0 : xn[i];
                if (q + 1 < e && H->tag[order[q + 1]] == TAG_CONG) pre += xn[order[q + 1]];
                if (tag == TAG_FREE) gu[j] += dt * xn[i];
                if (tag == TAG_CONG) gs[j] -= xn[i];
                xbar[i] = pre;
            }
        }
    }
    for (int j = 0; j < L; ++j) {
        const double kap = (double)o->kappa[j], c = (double)o->cost[j], be = (double)o->beta[j];
        if (d_u) d_u[j] = gu[j];
        if (d_kappa) d_kappa[j] = gs[j] * (-(double)sc->dn / (kap * kap));
        if (d_alpha) d_alpha[j] = ga[j];
        if (d_beta) d_beta[j] = gU[j] / c;
        if (d_cost) d_cost[j] = -gU[j] * be / (c * c);
    }
    if (d_alpha_origin) *d_alpha_origin = gao;
    if (d_w)
        for (int f = 0; f < F; ++f) {
            double s = 0.0;
            for (int j = 0; j < L; ++j)
                s += gU[j] * (double)o->phi[(size_t)j * F + f] + gG[j] * (double)o->psi[(size_t)j * F + f];
            d_w[f] = s;
        }
    if (d_lambda) for (int k = 0; k < sc->n_od; ++k) d_lambda[k] = glam[k];
    for (int i = 0; i < N; ++i) free(eadj[i]);
    free(eadj); free(xbar); free(gu); free(gs); free(ga); free(gU); free(gG); free(glam);
    free(Cbar); free(Csuf); free(order); free(cnt); free(xn);
    return 0;
}

/* positions of the current state per vehicle (0 off-network) */
void or_positions(const or_sim *o, double *x)
{
    for (int i = 0; i < o->sc.N; ++i) x[i] = o->vlink[i] >= 0 ? (double)o->vx[i] : 0.0;
}
