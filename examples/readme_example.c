/*
 * readme_example.c -- the smallest use of the C ABI (include/snn.h): one
 * column of 1000 RS + 250 FS neurons with 100 synapses each, one simulated
 * second, then the event counters and the first spike of the raster.
 * Build: gcc -std=c11 -I include examples/readme_example.c \
 *            paper_1310_8478_gb300/_build/libsnn.so
 */
#include <stdio.h>
#include <stdlib.h>
#include "snn.h"

int main(void)
{
    /* one column of 1000 RS + 250 FS neurons, 100 synapses each */
    snn_config c = {0};
    c.grid_x = 1; c.grid_y = 1;
    c.neurons_per_col = 1250; c.exc_per_col = 1000;
    c.fanout = 100;
    c.pct_ring[0] = 100;
    c.max_delay_ms = 20;
    c.w_exc0_q16 = 6 * 65536; c.w_inh0_q16 = -5 * 65536; c.wmax_q16 = 10 * 65536;
    c.a_plus_mv = 0.1; c.a_minus_mv = 0.12; c.tau_plus_ms = 20.0; c.tau_minus_ms = 20.0;
    c.deriv_period_ms = 1000; c.deriv_bias_q16 = 655; c.deriv_decay_q16 = 58982;
    c.thal_per_col_per_ms = 1; c.thal_amp_q16 = 20 * 65536;
    c.seed = 1;
    c.raster_capacity = 1 << 20;

    snn_net *net = NULL;
    int rc = snn_build_network(&c, NULL, 0, &net);
    if (rc != SNN_OK) { fprintf(stderr, "%s: %s\n", snn_strerror(rc), snn_last_error()); return 1; }
    rc = snn_run(net, 1000);                       /* one simulated second */
    snn_counters k;
    if (rc == SNN_OK) rc = snn_read_counters(net, &k);
    size_t n = 0;
    snn_spike *spikes = malloc(sizeof(snn_spike) << 20);
    if (rc == SNN_OK) rc = snn_read_raster(net, 0, 1000, spikes, 1 << 20, &n);
    if (rc == SNN_OK)
        printf("%lld spikes, %lld synaptic events, first spike: neuron %d at %d ms\n",
               (long long)k.spikes, (long long)k.e_all, n ? spikes[0].gid : -1, n ? spikes[0].t_ms : -1);
    else
        fprintf(stderr, "%s: %s\n", snn_strerror(rc), snn_last_error());
    free(spikes);
    snn_free(net);
    return rc == SNN_OK ? 0 : 1;
}
