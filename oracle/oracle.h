/*
 * oracle.h -- interface of the plain CPU simulator in oracle.c.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE: see oracle.c.  This header is
 * private to oracle/ and is not the product's C ABI.
 */
#ifndef DPSNN_ORACLE_H
#define DPSNN_ORACLE_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ORC_STDP_OFF = 1,        /* no depression, no potentiation */
    ORC_DELIVERY_OFF = 2,    /* spikes are not delivered */
    ORC_FP64 = 4,            /* neuron state in double */
    ORC_BRUTE_DELIVERY = 8   /* scan every synapse every step instead of queueing */
};

typedef struct {
    uint32_t grid_x, grid_y;            /* columns on a torus */
    uint32_t neurons_per_col, exc_per_col;
    uint32_t fanout;                    /* M forward synapses per neuron */
    uint32_t pct_ring[4];               /* own column, 1st, 2nd, 3rd ring (percent of M) */
    uint32_t max_delay_ms;              /* excitatory delays 1..max; inhibitory 1 */
    int32_t w_exc0_q16, w_inh0_q16, wmax_q16;
    double a_plus_mv, a_minus_mv;       /* STDP amplitudes (A-: magnitude removed) */
    double tau_plus_ms, tau_minus_ms;
    uint32_t deriv_period_ms;           /* long-term plasticity period (0 = never) */
    int32_t deriv_bias_q16, deriv_decay_q16;
    uint32_t thal_per_col_per_ms;
    int32_t thal_amp_q16;
    uint64_t seed;
    uint32_t flags;
} orc_config;

typedef struct { int32_t t; int32_t gid; int32_t q16; } orc_stim;

typedef struct orc_sim orc_sim;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int32_t orc_stdp_q16(double amplitude_mv, double tau_ms, int32_t lag_ms);
int orc_neuron_step_f32(float *v, float *u, int32_t current_q16, int excitatory);
int orc_neuron_step_f64(double *v, double *u, int32_t current_q16, int excitatory);
void orc_deriv_q16(int32_t *w, int32_t *sd, int32_t bias_q16, int32_t decay_q16, int32_t wmax_q16);
void orc_generate_synapse(const orc_config *c, uint32_t src, uint32_t j,
                          uint32_t *target_out, uint32_t *delay_out);
uint32_t orc_thalamic_target(const orc_config *c, int32_t t, uint32_t col, uint32_t k);

orc_sim *orc_create(const orc_config *c, char *err, size_t err_cap);
orc_sim *orc_create_explicit(const orc_config *c, const int64_t *row_off, const int32_t *tgt,
                             const uint8_t *delay, const int32_t *w, char *err, size_t err_cap);
void orc_free(orc_sim *s);
int orc_set_stimulus(orc_sim *s, const orc_stim *ev, int64_t n);
int orc_step(orc_sim *s);
int orc_run(orc_sim *s, int32_t n_ms);

uint32_t orc_n_neurons(const orc_sim *s);
int64_t orc_n_synapses(const orc_sim *s);
int32_t orc_time(const orc_sim *s);
int64_t orc_raster_size(const orc_sim *s);
const char *orc_error(const orc_sim *s);
void orc_read_raster(const orc_sim *s, int32_t *t_out, int32_t *gid_out);
void orc_read_synapses(const orc_sim *s, int32_t *tgt, uint8_t *delay, int32_t *w, int32_t *sd);
void orc_read_row_offsets(const orc_sim *s, int64_t *row_off);
void orc_read_neurons(const orc_sim *s, float *v, float *u, double *vd, double *ud);
void orc_read_counters(const orc_sim *s, int64_t out[4]);

#ifdef __cplusplus
}
#endif
#endif
