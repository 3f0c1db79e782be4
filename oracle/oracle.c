/*
 * oracle.c -- plain, single-threaded CPU simulator of the DPSNN-STDP
 * per-millisecond step (Paolucci et al., arXiv 1310.8478).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, the smoke check in
 * __graft_entry__ and the cpu_baseline / reference leg of bench.py may load
 * this library.  It shares no code, header, table or constant generator with
 * the CUDA path; the two are written independently from the paper and meet
 * only in the test harness.
 *
 * What it computes (section references are to the paper):
 *   - network construction, Sec. 2 "Projection of synapses with individual
 *     delay" and "Bidimensional arrays of neural columns": every neuron owns
 *     M forward synapses (delay D, weight W, target K); inhibitory neurons
 *     project only to excitatory neurons of their own column with the minimum
 *     delay; excitatory neurons project to their own column and to the 1st,
 *     2nd and 3rd rings of neighbouring columns on a toroidal grid, with
 *     delays uniform in 1..20 ms.  Draws come from a counter-based generator
 *     keyed by global ids, so the network does not depend on how it is laid
 *     out (Sec. 2 "Distributed generation of reproducible connections").
 *   - the simulation loop, Sec. 2 "Mixed time-driven and event driven
 *     simulation", steps 2.1-2.7, taken in the order
 *       S1 deliver spikes due now (2.3-2.5) + long-term depression (2.6),
 *       S2 thalamic drive + neuron update (2.7),
 *       S3 spike list / rastergram / queueing of the new spikes (2.2),
 *       S4 long-term potentiation for the neurons that just fired (2.1),
 *       S5 every period: long-term plasticity (w += bias + sd, sd *= decay),
 *     i.e. the paper's cycle rotated so that a spike carries the index of the
 *     step whose integration produced it.
 *   - the Izhikevich neuron, Sec. 2 "Spiking neuron model" (the equation
 *     block there), read as dv/dt = 0.04 v^2 + 5 v + 140 - u + I and
 *     du/dt = a (b v - u) (the printed "a(bv - c)" has no resting state near
 *     -70 mV, which the paper's Sec. 2 observables paragraph reports), with
 *     v integrated in two 0.5 ms Euler substeps (Sec. 3, time step paragraph)
 *     and u in one 1 ms step; spike when v >= 30 mV, then v = c, u += d.
 *   - the STDP pair rule, Sec. 2 "Synaptic update" equation:
 *     t = t_post - t_pre - d; t >= 0 potentiates by A+ exp(-t/tau+),
 *     t < 0 depresses by A- exp(t/tau-).  Nearest-neighbour pairing: a
 *     spike arriving at step ta pairs with the target's latest spike at or
 *     before ta-1 (depression); a target spike at step tp pairs with the
 *     source's latest spike whose arrival ta = t_pre + d is <= tp
 *     (potentiation).  Plasticity changes the derivative sd of excitatory
 *     synapses only.
 *
 * Arithmetic: weights, currents and derivatives are int32 fixed point with
 * 16 fractional bits (Q16, 1 mV = 65536).  STDP amounts are the closed form
 * rounded to Q16 with llround, evaluated in double for every event.  The
 * neuron update is IEEE fp32, one rounding per written operation; this file
 * must be compiled with -ffp-contract=off so no multiply-add is fused.
 *
 * Mechanism (deliberately different from the GPU path): every neuron keeps
 * the full vector of its spike times; a spike is expanded at emission into
 * its M synapse ids, which are queued in the bucket of their arrival step;
 * LTP searches the source's spike-time vector directly.  A second, brute
 * force delivery mode scans every synapse every step instead of queueing.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <stdio.h>

#include "oracle.h"

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11).  Each of the ten rounds multiplies words 0 and */
/* 2 by the two Philox constants, keeps the low halves as new words 1 and 3 */
/* and xors the high halves with the other two words and the round key; the */
/* key is bumped by the two Weyl constants between rounds.                  */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod_a = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
        uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
        uint32_t n0 = hi_b ^ x1 ^ k0;
        uint32_t n1 = lo_b;
        uint32_t n2 = hi_a ^ x3 ^ k1;
        uint32_t n3 = lo_a;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uniform integer in [0, n): the high word of r * n */
static uint32_t scale_draw(uint32_t r, uint32_t n)
{
    return (uint32_t)(((uint64_t)r * (uint64_t)n) >> 32);
}

static void draw(const orc_config *c, uint32_t a, uint32_t b, uint32_t domain,
                 uint32_t sub, uint32_t out[4])
{
    uint32_t ctr[4] = {a, b, domain, sub};
    uint32_t key[2] = {(uint32_t)(c->seed & 0xffffffffu), (uint32_t)(c->seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* STDP amounts in Q16: the pair rule of Sec. 2 ("Synaptic update") at an   */
/* integer lag k >= 0, rounded to nearest (halves away from zero).          */
/* ------------------------------------------------------------------------ */
int32_t orc_stdp_q16(double amplitude_mv, double tau_ms, int32_t lag_ms)
{
    double value = amplitude_mv * exp(-(double)lag_ms / tau_ms) * 65536.0;
    return (int32_t)llround(value);
}

/* ------------------------------------------------------------------------ */
/* Izhikevich neuron, one 1 ms step (see header comment for the reading).   */
/* ------------------------------------------------------------------------ */
static void neuron_kind(int excitatory, float *a, float *b, float *c, float *d)
{
    /* Sec. 2: RS a=0.02 b=0.2 c=-65 d=8; FS a=0.1 b=0.2 c=-65 d=2 */
    if (excitatory) { *a = 0.02f; *b = 0.2f; *c = -65.0f; *d = 8.0f; }
    else            { *a = 0.1f;  *b = 0.2f; *c = -65.0f; *d = 2.0f; }
}

int orc_neuron_step_f32(float *v, float *u, int32_t current_q16, int excitatory)
{
    float a, b, c, d;
    neuron_kind(excitatory, &a, &b, &c, &d);
    float cur = (float)current_q16 * 0x1p-16f;
    float vv = *v, uu = *u, x;
    for (int half = 0; half < 2; ++half) {      /* two 0.5 ms substeps of v */
        x = 0.04f * vv;
        x = x + 5.0f;
        x = x * vv;
        x = x + 140.0f;
        x = x - uu;
        x = x + cur;
        x = 0.5f * x;
        vv = vv + x;
    }
    x = b * vv;                                  /* one 1 ms step of u */
    x = x - uu;
    x = a * x;
    uu = uu + x;
    int fired = 0;
    if (vv >= 30.0f) { fired = 1; vv = c; uu = uu + d; }
    *v = vv; *u = uu;
    return fired;
}

int orc_neuron_step_f64(double *v, double *u, int32_t current_q16, int excitatory)
{
    /* the same scheme and operation order in double, decimal parameters */
    double a = excitatory ? 0.02 : 0.1, b = 0.2, c = -65.0, d = excitatory ? 8.0 : 2.0;
    double cur = (double)current_q16 / 65536.0;
    double vv = *v, uu = *u;
    for (int half = 0; half < 2; ++half)
        vv = vv + 0.5 * ((0.04 * vv + 5.0) * vv + 140.0 - uu + cur);
    uu = uu + a * (b * vv - uu);
    int fired = 0;
    if (vv >= 30.0) { fired = 1; vv = c; uu = uu + d; }
    *v = vv; *u = uu;
    return fired;
}

/* ------------------------------------------------------------------------ */
/* Long-term plasticity: w += bias + sd (clamped to [0, wmax]) and          */
/* sd *= decay, in Q16 with int64 intermediates; the product is rounded to  */
/* nearest with halves going up: floor((sd * decay + 2^15) / 2^16).         */
/* ------------------------------------------------------------------------ */
static int64_t floor_div_65536(int64_t x)
{
    int64_t q = x / 65536;
    if ((x % 65536) != 0 && x < 0) q -= 1;
    return q;
}

void orc_deriv_q16(int32_t *w, int32_t *sd, int32_t bias_q16, int32_t decay_q16, int32_t wmax_q16)
{
    int64_t nw = (int64_t)*w + (int64_t)bias_q16 + (int64_t)*sd;
    if (nw < 0) nw = 0;
    if (nw > wmax_q16) nw = wmax_q16;
    int64_t ns = floor_div_65536((int64_t)*sd * (int64_t)decay_q16 + 32768);
    *w = (int32_t)nw;
    *sd = (int32_t)ns;
}

/* ------------------------------------------------------------------------ */
/* growable arrays                                                          */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t *v; int64_t n, cap; } vec64;
typedef struct { int32_t *v; int64_t n, cap; } vec32;

static int vec64_push(vec64 *a, int64_t x)
{
    if (a->n == a->cap) {
        int64_t nc = a->cap ? 2 * a->cap : 64;
        int64_t *nv = (int64_t *)realloc(a->v, (size_t)nc * sizeof(int64_t));
        if (!nv) return -1;
        a->v = nv; a->cap = nc;
    }
    a->v[a->n++] = x;
    return 0;
}

static int vec32_push(vec32 *a, int32_t x)
{
    if (a->n == a->cap) {
        int64_t nc = a->cap ? 2 * a->cap : 16;
        int32_t *nv = (int32_t *)realloc(a->v, (size_t)nc * sizeof(int32_t));
        if (!nv) return -1;
        a->v = nv; a->cap = nc;
    }
    a->v[a->n++] = x;
    return 0;
}

#define QUEUE_SLOTS 64   /* > any delay; arrival buckets indexed by step mod 64 */

struct orc_sim {
    orc_config cfg;
    uint32_t n_neurons;
    int64_t n_syn;
    /* forward synapses in canonical (source, ordinal) order */
    int64_t *row_off;         /* n_neurons + 1 */
    uint32_t *src;            /* source neuron of every synapse */
    int32_t *tgt;
    uint8_t *dly;
    int32_t *w;
    int32_t *sd;
    /* incoming excitatory synapses of every neuron (synapse ids, ascending) */
    int64_t *in_off;          /* n_neurons + 1 */
    int64_t *in_syn;
    /* neuron state */
    float *v, *u;
    double *vd, *ud;
    int32_t *cur;
    vec32 *spikes;            /* all spike times of every neuron, ascending */
    /* queued arrivals, bucket = arrival step mod QUEUE_SLOTS */
    vec64 queue[QUEUE_SLOTS];
    /* external stimulus events, sorted by step */
    orc_stim *stim;
    int64_t n_stim, stim_pos;
    /* rastergram */
    vec32 raster_t, raster_gid;
    /* counters */
    int64_t n_spikes, e_all, e_exc, l_exc;
    int32_t t;
    char err[256];
};

static int is_exc(const orc_sim *s, uint32_t gid)
{
    return (gid % s->cfg.neurons_per_col) < s->cfg.exc_per_col;
}

/* ------------------------------------------------------------------------ */
/* one generated synapse: source gid, ordinal j  ->  (target gid, delay)    */
/* ------------------------------------------------------------------------ */
static const int ring_dx[3][4] = {{1, -1, 0, 0}, {1, -1, 1, -1}, {2, -2, 0, 0}};
static const int ring_dy[3][4] = {{0, 0, 1, -1}, {1, 1, -1, -1}, {0, 0, 2, -2}};

static int wrap(int x, int n)
{
    int r = x % n;
    return r < 0 ? r + n : r;
}

void orc_generate_synapse(const orc_config *c, uint32_t src, uint32_t j,
                          uint32_t *target_out, uint32_t *delay_out)
{
    uint32_t npc = c->neurons_per_col, ne = c->exc_per_col, m = c->fanout;
    uint32_t col = src / npc, local = src % npc;
    uint32_t r[4];
    draw(c, src, j, 0u, 0u, r);
    if (local >= ne) {
        /* inhibitory: an excitatory neuron of its own column, minimum delay */
        *target_out = col * npc + scale_draw(r[0], ne);
        *delay_out = 1;
        return;
    }
    *delay_out = 1 + scale_draw(r[1], c->max_delay_ms);
    /* ring of the ordinal: cumulative percentages of M, floored */
    uint32_t acc = 0, ring = 3, start = 0, prev_end = 0;
    for (uint32_t k = 0; k < 4; ++k) {
        acc += c->pct_ring[k];
        uint32_t end = (uint32_t)(((uint64_t)m * acc) / 100u);
        if (j < end) { ring = k; start = prev_end; break; }
        prev_end = end;
    }
    int cx = (int)(col % c->grid_x), cy = (int)(col / c->grid_x);
    int tx = cx, ty = cy;
    if (ring > 0) {
        uint32_t member = (j - start) % 4u;
        tx = wrap(cx + ring_dx[ring - 1][member], (int)c->grid_x);
        ty = wrap(cy + ring_dy[ring - 1][member], (int)c->grid_y);
    }
    uint32_t tcol = (uint32_t)ty * c->grid_x + (uint32_t)tx;
    uint32_t tl;
    if (tcol == col) {
        tl = scale_draw(r[0], npc - 1);       /* any neuron but itself */
        if (tl >= local) tl += 1;
    } else {
        tl = scale_draw(r[0], npc);
    }
    *target_out = tcol * npc + tl;
}

uint32_t orc_thalamic_target(const orc_config *c, int32_t t, uint32_t col, uint32_t k)
{
    uint32_t r[4];
    draw(c, (uint32_t)t, col, 1u, k, r);
    return col * c->neurons_per_col + scale_draw(r[0], c->neurons_per_col);
}

/* ------------------------------------------------------------------------ */
/* construction                                                             */
/* ------------------------------------------------------------------------ */
static int check_config(const orc_config *c, char *err)
{
    if (c->grid_x == 0 || c->grid_y == 0) { strcpy(err, "empty grid"); return -1; }
    if (c->neurons_per_col < 2 || c->exc_per_col == 0 || c->exc_per_col > c->neurons_per_col) {
        strcpy(err, "bad column size"); return -1;
    }
    if (c->max_delay_ms == 0 || c->max_delay_ms >= QUEUE_SLOTS - 1) { strcpy(err, "bad max delay"); return -1; }
    if (c->pct_ring[0] + c->pct_ring[1] + c->pct_ring[2] + c->pct_ring[3] != 100) {
        strcpy(err, "ring percentages must sum to 100"); return -1;
    }
    if ((uint64_t)c->grid_x * c->grid_y * c->neurons_per_col > 0x7fffffffu) {
        strcpy(err, "too many neurons"); return -1;
    }
    return 0;
}

static orc_sim *alloc_sim(const orc_config *c, int64_t n_syn)
{
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->cfg = *c;
    s->n_neurons = c->grid_x * c->grid_y * c->neurons_per_col;
    s->n_syn = n_syn;
    uint32_t n = s->n_neurons;
    s->row_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    s->src = (uint32_t *)malloc((size_t)(n_syn ? n_syn : 1) * sizeof(uint32_t));
    s->tgt = (int32_t *)malloc((size_t)(n_syn ? n_syn : 1) * sizeof(int32_t));
    s->dly = (uint8_t *)malloc((size_t)(n_syn ? n_syn : 1));
    s->w = (int32_t *)malloc((size_t)(n_syn ? n_syn : 1) * sizeof(int32_t));
    s->sd = (int32_t *)calloc((size_t)(n_syn ? n_syn : 1), sizeof(int32_t));
    s->v = (float *)malloc((size_t)n * sizeof(float));
    s->u = (float *)malloc((size_t)n * sizeof(float));
    s->vd = (double *)malloc((size_t)n * sizeof(double));
    s->ud = (double *)malloc((size_t)n * sizeof(double));
    s->cur = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    s->spikes = (vec32 *)calloc((size_t)n, sizeof(vec32));
    s->in_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!s->row_off || !s->src || !s->tgt || !s->dly || !s->w || !s->sd || !s->v || !s->u ||
        !s->vd || !s->ud || !s->cur || !s->spikes || !s->in_off) {
        orc_free(s);
        return NULL;
    }
    return s;
}

/* initial state (not given by the paper): v = -65 mV, u = b v */
static void init_neurons(orc_sim *s)
{
    for (uint32_t i = 0; i < s->n_neurons; ++i) {
        float a, b, c, d;
        neuron_kind(is_exc(s, i), &a, &b, &c, &d);
        s->v[i] = -65.0f;
        s->u[i] = b * s->v[i];
        s->vd[i] = -65.0;
        s->ud[i] = 0.2 * -65.0;
    }
}

/* incoming excitatory synapses of every target, in ascending synapse id */
static int build_incoming(orc_sim *s)
{
    uint32_t n = s->n_neurons;
    int64_t *count = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    if (!count) return -1;
    for (uint32_t p = 0; p < n; ++p) {
        if (!is_exc(s, p)) continue;
        for (int64_t k = s->row_off[p]; k < s->row_off[p + 1]; ++k) count[s->tgt[k]]++;
    }
    s->in_off[0] = 0;
    for (uint32_t i = 0; i < n; ++i) s->in_off[i + 1] = s->in_off[i] + count[i];
    s->in_syn = (int64_t *)malloc((size_t)(s->in_off[n] ? s->in_off[n] : 1) * sizeof(int64_t));
    if (!s->in_syn) { free(count); return -1; }
    for (uint32_t i = 0; i < n; ++i) count[i] = s->in_off[i];
    for (uint32_t p = 0; p < n; ++p) {
        if (!is_exc(s, p)) continue;
        for (int64_t k = s->row_off[p]; k < s->row_off[p + 1]; ++k) s->in_syn[count[s->tgt[k]]++] = k;
    }
    free(count);
    return 0;
}

orc_sim *orc_create(const orc_config *c, char *err, size_t err_cap)
{
    char msg[256] = {0};
    if (check_config(c, msg) != 0) {
        if (err && err_cap) snprintf(err, err_cap, "%s", msg);
        return NULL;
    }
    uint64_t n = (uint64_t)c->grid_x * c->grid_y * c->neurons_per_col;
    orc_sim *s = alloc_sim(c, (int64_t)(n * c->fanout));
    if (!s) {
        if (err && err_cap) snprintf(err, err_cap, "out of host memory");
        return NULL;
    }
    for (uint32_t p = 0; p < s->n_neurons; ++p) {
        int64_t base = (int64_t)p * c->fanout;
        s->row_off[p] = base;
        int exc = is_exc(s, p);
        for (uint32_t j = 0; j < c->fanout; ++j) {
            uint32_t tg, dl;
            orc_generate_synapse(c, p, j, &tg, &dl);
            s->src[base + j] = p;
            s->tgt[base + j] = (int32_t)tg;
            s->dly[base + j] = (uint8_t)dl;
            s->w[base + j] = exc ? c->w_exc0_q16 : c->w_inh0_q16;
        }
    }
    s->row_off[s->n_neurons] = s->n_syn;
    if (build_incoming(s) != 0) {
        orc_free(s);
        if (err && err_cap) snprintf(err, err_cap, "out of host memory");
        return NULL;
    }
    init_neurons(s);
    return s;
}

orc_sim *orc_create_explicit(const orc_config *c, const int64_t *row_off, const int32_t *tgt,
                             const uint8_t *delay, const int32_t *w, char *err, size_t err_cap)
{
    char msg[256] = {0};
    if (check_config(c, msg) != 0) {
        if (err && err_cap) snprintf(err, err_cap, "%s", msg);
        return NULL;
    }
    uint32_t n = c->grid_x * c->grid_y * c->neurons_per_col;
    int64_t n_syn = row_off[n];
    for (uint32_t p = 0; p < n; ++p) {
        if (row_off[p + 1] < row_off[p]) {
            if (err && err_cap) snprintf(err, err_cap, "row offsets must not decrease");
            return NULL;
        }
    }
    for (int64_t k = 0; k < n_syn; ++k) {
        if (tgt[k] < 0 || (uint32_t)tgt[k] >= n || delay[k] < 1 || delay[k] > c->max_delay_ms) {
            if (err && err_cap) snprintf(err, err_cap, "synapse %lld out of range", (long long)k);
            return NULL;
        }
    }
    orc_sim *s = alloc_sim(c, n_syn);
    if (!s) {
        if (err && err_cap) snprintf(err, err_cap, "out of host memory");
        return NULL;
    }
    memcpy(s->row_off, row_off, ((size_t)n + 1) * sizeof(int64_t));
    if (n_syn) {
        memcpy(s->tgt, tgt, (size_t)n_syn * sizeof(int32_t));
        memcpy(s->dly, delay, (size_t)n_syn);
        memcpy(s->w, w, (size_t)n_syn * sizeof(int32_t));
    }
    for (uint32_t p = 0; p < n; ++p)
        for (int64_t k = row_off[p]; k < row_off[p + 1]; ++k) s->src[k] = p;
    if (build_incoming(s) != 0) {
        orc_free(s);
        if (err && err_cap) snprintf(err, err_cap, "out of host memory");
        return NULL;
    }
    init_neurons(s);
    return s;
}

void orc_free(orc_sim *s)
{
    if (!s) return;
    free(s->row_off); free(s->src); free(s->tgt); free(s->dly); free(s->w); free(s->sd);
    free(s->in_off); free(s->in_syn);
    free(s->v); free(s->u); free(s->vd); free(s->ud); free(s->cur);
    if (s->spikes) {
        for (uint32_t i = 0; i < s->n_neurons; ++i) free(s->spikes[i].v);
        free(s->spikes);
    }
    for (int q = 0; q < QUEUE_SLOTS; ++q) free(s->queue[q].v);
    free(s->stim);
    free(s->raster_t.v); free(s->raster_gid.v);
    free(s);
}

int orc_set_stimulus(orc_sim *s, const orc_stim *ev, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        if (ev[i].gid < 0 || (uint32_t)ev[i].gid >= s->n_neurons) return -1;
        if (i > 0 && ev[i].t < ev[i - 1].t) return -1;
    }
    free(s->stim);
    s->stim = NULL;
    s->n_stim = 0;
    s->stim_pos = 0;
    if (n > 0) {
        s->stim = (orc_stim *)malloc((size_t)n * sizeof(orc_stim));
        if (!s->stim) return -1;
        memcpy(s->stim, ev, (size_t)n * sizeof(orc_stim));
        s->n_stim = n;
    }
    while (s->stim_pos < s->n_stim && s->stim[s->stim_pos].t < s->t) s->stim_pos++;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* spike-time queries on the per-neuron vectors                             */
/* ------------------------------------------------------------------------ */
/* latest spike of neuron i at or before step `limit`; returns 0 if none */
static int latest_spike_at_or_before(const orc_sim *s, uint32_t i, int32_t limit, int32_t *when)
{
    const vec32 *a = &s->spikes[i];
    for (int64_t k = a->n - 1; k >= 0; --k) {
        if (a->v[k] <= limit) { *when = a->v[k]; return 1; }
    }
    return 0;
}

static int spiked_at(const orc_sim *s, uint32_t i, int32_t when)
{
    const vec32 *a = &s->spikes[i];
    for (int64_t k = a->n - 1; k >= 0; --k) {
        if (a->v[k] == when) return 1;
        if (a->v[k] < when) return 0;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* the step                                                                 */
/* ------------------------------------------------------------------------ */
static void deliver_one(orc_sim *s, int64_t syn, uint32_t pre, int32_t t)
{
    const orc_config *c = &s->cfg;
    int32_t post = s->tgt[syn];
    s->cur[post] += s->w[syn];                       /* Sec. 2 step 2.5 */
    s->e_all++;
    if (is_exc(s, pre)) {
        s->e_exc++;
        if (!(c->flags & ORC_STDP_OFF)) {            /* step 2.6: depression */
            int32_t tl;
            if (latest_spike_at_or_before(s, (uint32_t)post, t - 1, &tl))
                s->sd[syn] -= orc_stdp_q16(c->a_minus_mv, c->tau_minus_ms, t - tl);
        }
    }
}

static uint32_t source_of(const orc_sim *s, int64_t syn)
{
    return s->src[syn];
}

int orc_step(orc_sim *s)
{
    const orc_config *c = &s->cfg;
    const int32_t t = s->t;
    const uint32_t n = s->n_neurons;
    const uint32_t npc = c->neurons_per_col;
    const uint32_t ncol = c->grid_x * c->grid_y;

    /* S1: spikes due now (Sec. 2 steps 2.3-2.6) */
    if (!(c->flags & ORC_DELIVERY_OFF)) {
        if (c->flags & ORC_BRUTE_DELIVERY) {
            /* every synapse, every step: does its source fire at t - delay? */
            for (uint32_t p = 0; p < n; ++p)
                for (int64_t k = s->row_off[p]; k < s->row_off[p + 1]; ++k)
                    if (t - (int32_t)s->dly[k] >= 0 && spiked_at(s, p, t - (int32_t)s->dly[k]))
                        deliver_one(s, k, p, t);
        } else {
            vec64 *q = &s->queue[t % QUEUE_SLOTS];
            for (int64_t i = 0; i < q->n; ++i) {
                int64_t syn = q->v[i];
                deliver_one(s, syn, source_of(s, syn), t);
            }
            q->n = 0;
        }
    }

    /* S2: thalamic drive, one random neuron per column per event (Sec. 2,
       reproducible generation; Table 2 note on the thalamic model) */
    for (uint32_t col = 0; col < ncol; ++col)
        for (uint32_t k = 0; k < c->thal_per_col_per_ms; ++k)
            s->cur[orc_thalamic_target(c, t, col, k)] += c->thal_amp_q16;
    while (s->stim_pos < s->n_stim && s->stim[s->stim_pos].t == t) {
        s->cur[s->stim[s->stim_pos].gid] += s->stim[s->stim_pos].q16;
        s->stim_pos++;
    }

    /* S2: neuron update (step 2.7); S3: spike list and raster (step 2.2) */
    int64_t first_new = s->raster_gid.n;
    for (uint32_t i = 0; i < n; ++i) {
        int fired;
        int exc = (i % npc) < c->exc_per_col;
        if (c->flags & ORC_FP64) fired = orc_neuron_step_f64(&s->vd[i], &s->ud[i], s->cur[i], exc);
        else fired = orc_neuron_step_f32(&s->v[i], &s->u[i], s->cur[i], exc);
        s->cur[i] = 0;
        if (fired) {
            if (vec32_push(&s->spikes[i], t) || vec32_push(&s->raster_t, t) ||
                vec32_push(&s->raster_gid, (int32_t)i)) {
                snprintf(s->err, sizeof s->err, "out of host memory");
                return -1;
            }
            s->n_spikes++;
        }
    }
    /* queue the new spikes' synapses at their arrival steps */
    if (!(c->flags & ORC_DELIVERY_OFF) && !(c->flags & ORC_BRUTE_DELIVERY)) {
        for (int64_t r = first_new; r < s->raster_gid.n; ++r) {
            uint32_t p = (uint32_t)s->raster_gid.v[r];
            for (int64_t k = s->row_off[p]; k < s->row_off[p + 1]; ++k) {
                if (vec64_push(&s->queue[(t + s->dly[k]) % QUEUE_SLOTS], k)) {
                    snprintf(s->err, sizeof s->err, "out of host memory");
                    return -1;
                }
            }
        }
    }

    /* S4: potentiation of the incoming excitatory synapses of every neuron
       that fired now (step 2.1), paired with the source's latest arrival */
    for (int64_t r = first_new; r < s->raster_gid.n; ++r) {
        uint32_t post = (uint32_t)s->raster_gid.v[r];
        s->l_exc += s->in_off[post + 1] - s->in_off[post];
        if (c->flags & ORC_STDP_OFF) continue;
        for (int64_t k = s->in_off[post]; k < s->in_off[post + 1]; ++k) {
            int64_t syn = s->in_syn[k];
            uint32_t pre = source_of(s, syn);
            int32_t d = (int32_t)s->dly[syn];
            int32_t tp;
            if (latest_spike_at_or_before(s, pre, t - d, &tp))
                s->sd[syn] += orc_stdp_q16(c->a_plus_mv, c->tau_plus_ms, t - tp - d);
        }
    }

    /* S5: long-term plasticity at the end of every period (Table 2 row) */
    if (c->deriv_period_ms > 0 && ((uint32_t)t + 1) % c->deriv_period_ms == 0) {
        for (uint32_t p = 0; p < n; ++p) {
            if (!is_exc(s, p)) continue;
            for (int64_t k = s->row_off[p]; k < s->row_off[p + 1]; ++k)
                orc_deriv_q16(&s->w[k], &s->sd[k], c->deriv_bias_q16, c->deriv_decay_q16, c->wmax_q16);
        }
    }
    s->t = t + 1;
    return 0;
}

int orc_run(orc_sim *s, int32_t n_ms)
{
    for (int32_t i = 0; i < n_ms; ++i)
        if (orc_step(s) != 0) return -1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* read-back                                                                */
/* ------------------------------------------------------------------------ */
uint32_t orc_n_neurons(const orc_sim *s) { return s->n_neurons; }
int64_t orc_n_synapses(const orc_sim *s) { return s->n_syn; }
int32_t orc_time(const orc_sim *s) { return s->t; }
int64_t orc_raster_size(const orc_sim *s) { return s->raster_gid.n; }
const char *orc_error(const orc_sim *s) { return s->err; }

void orc_read_raster(const orc_sim *s, int32_t *t_out, int32_t *gid_out)
{
    memcpy(t_out, s->raster_t.v, (size_t)s->raster_t.n * sizeof(int32_t));
    memcpy(gid_out, s->raster_gid.v, (size_t)s->raster_gid.n * sizeof(int32_t));
}

void orc_read_synapses(const orc_sim *s, int32_t *tgt, uint8_t *delay, int32_t *w, int32_t *sd)
{
    size_t n = (size_t)s->n_syn;
    if (tgt) memcpy(tgt, s->tgt, n * sizeof(int32_t));
    if (delay) memcpy(delay, s->dly, n);
    if (w) memcpy(w, s->w, n * sizeof(int32_t));
    if (sd) memcpy(sd, s->sd, n * sizeof(int32_t));
}

void orc_read_row_offsets(const orc_sim *s, int64_t *row_off)
{
    memcpy(row_off, s->row_off, ((size_t)s->n_neurons + 1) * sizeof(int64_t));
}

void orc_read_neurons(const orc_sim *s, float *v, float *u, double *vd, double *ud)
{
    size_t n = s->n_neurons;
    if (v) memcpy(v, s->v, n * sizeof(float));
    if (u) memcpy(u, s->u, n * sizeof(float));
    if (vd) memcpy(vd, s->vd, n * sizeof(double));
    if (ud) memcpy(ud, s->ud, n * sizeof(double));
}

void orc_read_counters(const orc_sim *s, int64_t out[4])
{
    out[0] = s->n_spikes;
    out[1] = s->e_all;
    out[2] = s->e_exc;
    out[3] = s->l_exc;
}
