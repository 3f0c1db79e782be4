/*
 * snn.h -- C ABI of the GB300 engine for the DPSNN-STDP per-millisecond step
 * (Paolucci et al., "Distributed simulation of polychronous and plastic
 * spiking neural networks", arXiv 1310.8478).
 *
 * One step of simulated time (1 ms) runs, on the device, the paper's cycle
 * (Sec. 2 "Mixed time-driven and event driven simulation", steps 2.1-2.7) in
 * the order
 *   S1 delivery of the axonal spikes due now through the delay-bucketed
 *      synapse lists, current injection and long-term depression (2.3-2.6);
 *   S2 thalamic drive and Izhikevich update of every neuron (2.7);
 *   S3 compaction of the neurons that fired into the axonal-delay ring and
 *      the rastergram (2.2);
 *   S4 long-term potentiation of the incoming synapses of every neuron that
 *      fired (2.1);
 *   S5 at the end of every plasticity period, the long-term update
 *      w += bias + sd (clamped to [0, wmax]), sd *= decay (Table 2,
 *      "long term synaptic plasticity").
 *
 * Conventions for every call:
 *   - Pointers named host_* or documented as host memory are ordinary host
 *     buffers owned by the caller; the library never keeps them.
 *   - The library owns the snn_net handle and all device memory behind it
 *     (allocated with cudaMalloc on the current device, or through the
 *     allocator installed by snn_set_allocator).
 *   - Return value: SNN_OK (0) or a negative SNN_E* code; snn_strerror gives a
 *     message.  A failed call leaves the handle usable unless it returned
 *     SNN_ECUDA.
 *   - Fixed point: weights, currents and synaptic derivatives are int32 with
 *     16 fractional bits ("Q16"; 1 mV = 65536).
 *   - Neuron ids: gid = column * neurons_per_col + local, column = y * grid_x
 *     + x; local ids below exc_per_col are excitatory (RS), the rest
 *     inhibitory (FS) (Sec. 2 "Spiking neuron model").
 */
#ifndef SNN_H
#define SNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SNN_OK 0
#define SNN_EINVAL (-1)     /* bad argument or configuration */
#define SNN_ENOMEM (-2)     /* device budget exceeded or allocation failed */
#define SNN_ECUDA (-3)      /* CUDA runtime error; the handle must be freed */
#define SNN_EOVERFLOW (-4)  /* the int32 Q16 current bound cannot be guaranteed */
#define SNN_ETIMEOUT (-5)   /* a bounded device-side wait gave up */
#define SNN_ETRUNC (-6)     /* output buffer too small; *n_out holds the size needed */
#define SNN_ESTATE (-7)     /* the call does not fit the handle's state */
#define SNN_EBOUNDS (-8)    /* checked build (-DSNN_CHECKED): a kernel met an index out of
                               range, skipped the access and set the device error word */

/* cfg.flags */
#define SNN_STDP_OFF 1u      /* no depression / potentiation (sd stays 0) */
#define SNN_DELIVERY_OFF 2u  /* spikes are not delivered (neurons see drive only) */
#define SNN_FP64 4u          /* physics check: v and u in double precision (same scheme and
                                operation order; slower neuron update, 8 more bytes per neuron) */

/*
 * Network and model configuration (plain old data).
 * Topology: Sec. 2 "Bidimensional arrays of neural columns" (toroidal grid of
 * columns; excitatory neurons project to their own column and to the 1st, 2nd
 * and 3rd rings of neighbours, inhibitory neurons only to excitatory neurons
 * of their own column) and "Projection of synapses with individual delay"
 * (M forward synapses per neuron; excitatory delays uniform in
 * 1..max_delay_ms, inhibitory delays 1 ms).  STDP: Sec. 2 "Synaptic update"
 * equation, A+/A- in mV, tau in ms.
 */
typedef struct {
    uint32_t grid_x, grid_y;             /* columns on the torus */
    uint32_t neurons_per_col;            /* >= 2 */
    uint32_t exc_per_col;                /* 1..neurons_per_col */
    uint32_t fanout;                     /* M synapses per neuron, 1..65535 */
    uint32_t pct_ring[4];                /* % of M: own column, ring 1, 2, 3; sum 100 */
    uint32_t max_delay_ms;               /* 1..31 */
    int32_t w_exc0_q16, w_inh0_q16;      /* initial weights */
    int32_t wmax_q16;                    /* excitatory weights are clamped to [0, wmax] */
    double a_plus_mv, a_minus_mv;        /* A+ (added) and A- (subtracted), both >= 0 */
    double tau_plus_ms, tau_minus_ms;
    uint32_t deriv_period_ms;            /* long-term update period; 0 = never */
    int32_t deriv_bias_q16;              /* added to w at each update */
    int32_t deriv_decay_q16;             /* sd = (sd * decay + 2^15) >> 16 */
    uint32_t thal_per_col_per_ms;        /* thalamic events per column per ms (times the
                                            columns: at most 2^31 - 1) */
    int32_t thal_amp_q16;                /* current of one thalamic event */
    uint64_t seed;                       /* key of the Philox4x32-10 draws */
    uint32_t flags;                      /* SNN_STDP_OFF | SNN_DELIVERY_OFF | SNN_FP64 */
    uint32_t reserved;                   /* must be 0 */
    uint64_t raster_capacity;            /* spikes kept on the device; 0 = no raster */
} snn_config;

typedef struct { int32_t t_ms; int32_t gid; } snn_spike;

/* External current event: adds q16 to neuron gid's input at step t. */
typedef struct { int32_t t; int32_t gid; int32_t q16; } snn_stimulus;

typedef struct {
    int64_t t;               /* steps simulated so far */
    int64_t spikes;          /* all spikes emitted */
    int64_t e_all;           /* synaptic events delivered (spike x synapse) */
    int64_t e_exc;           /* of which on excitatory (plastic) synapses */
    int64_t l_exc;           /* potentiation visits: sum over spikes of excitatory in-degree */
    int64_t raster_kept;     /* spikes stored in the device raster */
    int64_t raster_dropped;  /* spikes not stored because the raster was full */
    int32_t error;           /* device error word (0 = none) */
    int32_t reserved;
} snn_counters;

/*
 * Launch shape of the step kernels.  Any shape gives bit-identical results
 * (integer accumulation; the spike lists' order does not matter).
 * Zero fields keep the current value.
 */
typedef struct {
    uint32_t deliver_block;          /* threads per block of the event-driven delivery (multiple of 32;
                                        the column-ordered delivery gives one column to each block
                                        and takes at most 256 threads) */
    uint32_t deliver_blocks_per_sm;  /* resident blocks per SM of the event-driven delivery (at most) */
    uint32_t neuron_block;           /* threads per block of the neuron update */
    uint32_t ltp_block;              /* threads per block of the event-driven potentiation */
    uint32_t ltp_blocks_per_sm;
    uint32_t deriv_block;
    uint32_t graph_steps;            /* steps per captured CUDA graph; even; 1 = no graphs */
    uint32_t dense_block;            /* threads per block of the dense synapse pass (32..1024) */
    uint32_t dense_rows;             /* source rows per block of the dense pass */
    uint32_t dense_permille;         /* a step takes the dense pass when at least this many
                                        neurons per 1000 fired in the step before (default 250,
                                        the measured crossover); 1001 = never */
    uint32_t staged_permille;        /* a step without the dense pass delivers column by column
                                        through shared memory when its expected events (spikes of
                                        the last max_delay steps x fan-out / max_delay, plus
                                        inhibitory spikes of the step before x fan-out) reach this
                                        many per 1000 neurons; 0xffffffff = never (the default:
                                        the column-ordered delivery, which stages the source
                                        column's own neurons, is faster on the measured nets) */
    uint32_t ring_permille;          /* nets with compact targets: a step without the dense pass
                                        whose expected events stay below this many per 1000
                                        neurons delivers from the ring's spike lists instead of
                                        walking every column (default: never, i.e. 0, which a
                                        shape cannot set again since 0 means "unchanged": 1 is
                                        practically never; 0xffffffff = every such step).  Off by
                                        default: slower than the column walk on the measured nets */
} snn_launch;

/* Per-kernel device time collected while profiling is on (CUDA events), and
   the work the dense synapse pass did (always counted). */
typedef struct {
    int64_t launches[5];             /* deliver, neuron, ltp, deriv, dense */
    double ms[5];
    int64_t dense_steps;             /* steps that took the dense pass */
    int64_t dense_deriv_steps;       /* of which closed a plasticity period */
    int64_t dense_events;            /* synaptic events delivered by the dense pass */
    int64_t dense_exc_events;
    int64_t dense_ltp_visits;        /* potentiation visits done by the dense pass */
    int64_t kernels;                 /* kernels launched by the profiled steps, every kind (a
                                        kind above may group two: k_fold + k_deriv, the
                                        column-ordered + column-staged deliveries) */
} snn_profile;

typedef struct snn_net snn_net;

/*
 * snn_build_network -- construct the network of cfg on the current device
 * (Sec. 2 "Initial construction" and "Distributed generation of reproducible
 * connections"): for every source gid and ordinal j, Philox4x32-10 with key
 * (seed low, seed high) and counter (gid, j, 0, 0) draws the target neuron and
 * the delay, so the network does not depend on the device layout.  Builds the
 * delay-bucketed forward lists, the reverse (incoming excitatory) index and
 * the initial state (v = -65 mV, u = 0.2 v).
 *   cuda_stream: cudaStream_t the engine works on (NULL: a private stream).
 *     The net also owns a side stream: in a step that closes no period the
 *     potentiation owed by the last step runs there beside the delivery,
 *     forked from and joined back into cuda_stream within the step.
 *   hbm_budget_bytes: upper bound of device memory the net may use (0: no bound).
 *   out: receives the handle.
 * Errors: SNN_EINVAL (bad cfg), SNN_ENOMEM (footprint above the budget or
 * allocation failure), SNN_EOVERFLOW (in-degree * wmax + drive may exceed
 * int32), SNN_ECUDA.
 */
int snn_build_network(const snn_config *cfg, void *cuda_stream, size_t hbm_budget_bytes,
                      snn_net **out);

/*
 * snn_build_network_explicit -- same, from explicit host synapse lists in
 * canonical order (Sec. 2 "Projection of synapses": each source i owns
 * synapses (D, W, K)): source p owns host_tgt/host_delay/host_w[row_off[p]
 * .. row_off[p+1]), N = grid_x * grid_y * neurons_per_col.  cfg.fanout,
 * pct_ring and seed are ignored for the topology (seed still keys the
 * thalamic drive).  Rows may be empty; a row holds at most 65535 synapses.
 */
int snn_build_network_explicit(const snn_config *cfg, const int64_t *host_row_off,
                               const int32_t *host_tgt, const uint8_t *host_delay,
                               const int32_t *host_w, void *cuda_stream,
                               size_t hbm_budget_bytes, snn_net **out);

/*
 * snn_set_stimulus -- external current events (host array, any order; n may
 * be 0 to clear), applied in S2 of their step before the neuron update.  The
 * thalamic drive of Sec. 2 / Table 2 ("thalamic input") is separate and
 * always on unless thal_per_col_per_ms = 0.  Events before the current step
 * are ignored.  SNN_EINVAL if a gid is out of range.  The events are staged
 * in library-owned pinned memory and copied on the net's stream: the call
 * may return before the copy ends, and the caller's array is free at once.
 */
int snn_set_stimulus(snn_net *net, const snn_stimulus *host_events, size_t n);

/*
 * snn_set_thalamic -- on = 0: the net stops drawing its own thalamic events
 * (the caller then supplies the drive, e.g. snn_thalamic_events through
 * snn_run_host); on = 1: back to cfg.thal_per_col_per_ms events per column.
 */
int snn_set_thalamic(snn_net *net, int on);

/*
 * snn_set_tile -- make the net one tile of a torus partitioned by columns,
 * as the paper's processes own sets of columns (Sec. 2 "Delivery of spiking
 * messages": a process integrates its own neurons and receives, every step,
 * the spikes of the other processes' neurons that reach its synapses).  From
 * the first step on the net integrates only the neurons of columns
 * [first_col, first_col + n_cols), delivers spikes only to them (from every
 * source whose synapses reach them, wherever it sits), potentiates only their
 * incoming synapses, and counts only those events and their spikes; so each
 * synapse is served by the tile that owns its target.  The spikes of the other
 * columns' neurons must be supplied after every step with snn_inject_spikes.
 * The tile keeps the whole torus's state arrays (one GPU holds every tile
 * here); only ownership is partitioned.  Tiles take the column-ordered
 * delivery in every step (the dense pass and the staged delivery are off).
 * first_col = 0, n_cols = all columns makes the net whole again.
 * Errors: SNN_EINVAL (range outside the torus), SNN_ESTATE (the net has
 * stepped already, or is not a generated net with compact targets).
 */
int snn_set_tile(snn_net *net, uint32_t first_col, uint32_t n_cols);

/*
 * snn_inject_spikes -- the spikes of the step just completed (t = steps
 * simulated - 1) of neurons the tile does not own (host array of n gids, any
 * order, each at most once), as received from their owners: they join the
 * step's spike lists after the tile's own, and the neurons' spike history and
 * last spike, so that delivery and potentiation treat them as the tile's own.
 * Returns after the device has taken them.  Errors: SNN_EINVAL (a gid out of
 * range, owned by the tile, or repeated), SNN_ESTATE (not a tile, no step
 * run yet).
 */
int snn_inject_spikes(snn_net *net, const int32_t *host_gids, uint32_t n);

/* snn_set_launch / snn_get_launch -- launch shape (see snn_launch). */
int snn_set_launch(snn_net *net, const snn_launch *launch);
int snn_get_launch(const snn_net *net, snn_launch *launch);

/*
 * snn_step -- advance one millisecond (S1..S5 above).  Enqueued on the net's
 * stream; returns after the step has completed and the device error word has
 * been checked.
 */
int snn_step(snn_net *net);

/*
 * snn_run -- advance n_ms steps (CUDA-graph replays of graph_steps steps where
 * the alignment allows and no step of the chunk closes a plasticity period,
 * single steps otherwise); returns after completion and the error-word check.
 */
int snn_run(snn_net *net, uint32_t n_ms);

/*
 * snn_run_host -- the end-to-end call for a caller that lives in host memory:
 * copies host_stimulus (n_stim events, may be NULL) to the device as the
 * external stimulus of the coming steps, advances n_ms steps and, if
 * host_spikes is not NULL, copies the spikes of those steps, sorted by
 * (t, gid), into host_spikes (capacity cap) and resets the device raster.
 * *n_out = spikes emitted in the window.  SNN_ETRUNC if cap is too small (the
 * simulation still advanced) or the device raster overflowed.  Without
 * host_spikes the call synchronises with the stream once: the counters are
 * copied out before and after the steps into pinned memory on the stream.
 */
int snn_run_host(snn_net *net, uint32_t n_ms, const snn_stimulus *host_stimulus, size_t n_stim,
                 snn_spike *host_spikes, size_t cap, size_t *n_out);

/*
 * snn_read_raster -- rastergram (Sec. 2 "Production of observables") of steps
 * [t0, t1): host_buf receives (t, gid) sorted by t then gid; cap entries at
 * most; *n_out = entries in the window.  SNN_ETRUNC if cap < *n_out or part
 * of the window was dropped because the device raster was full.
 */
int snn_read_raster(snn_net *net, int32_t t0, int32_t t1, snn_spike *host_buf, size_t cap,
                    size_t *n_out);

/* snn_raster_reset -- forget the stored raster (frees room for later steps). */
int snn_raster_reset(snn_net *net);

/*
 * snn_read_synapses -- synapses of sources [first, first + count) in canonical
 * (source, ordinal) order; any host pointer may be NULL.  *n_out = synapses in
 * the range; SNN_ETRUNC if cap is smaller.  Inhibitory synapses keep their
 * weight and sd = 0.
 */
int snn_read_synapses(snn_net *net, uint32_t first, uint32_t count, int32_t *host_tgt,
                      uint8_t *host_delay, int32_t *host_w, int32_t *host_sd, size_t cap,
                      size_t *n_out);

/*
 * snn_read_synapses_noalloc -- snn_read_synapses without any device
 * allocation.  The paper has no counterpart; it serves callers that cannot
 * allocate device memory once networks are running: a serving loop that has
 * committed its whole HBM budget to resident networks, code that must not
 * pay the device-wide synchronization of cudaMalloc / cudaFree while other
 * networks' steps are in flight on other streams, or hosts whose device
 * memory belongs to a framework allocator they cannot reach from here.
 * The device staging is a fixed array compiled into the library
 * (SNN_NOALLOC_MAX_SYNAPSES synapses, about 13 MiB).  It becomes resident on
 * a device when the first net is built there (the build looks up the array's
 * device address with that device current, which loads the library's module)
 * and stays until the process exits; it is not counted in hbm_budget_bytes.
 * Every build looks the address up again, so a device reset between nets
 * leaves no stale address; a net that outlives a reset of its device is
 * invalid anyway.  This call itself does no lookup, so it may come after a
 * stream capture has started on another stream.  A range with more synapses
 * is rejected with SNN_EINVAL; split it.  Every call shares the array: calls
 * that overlap on the GPU (different threads, different nets on the same
 * device) race, so serialize them.  Arguments, results and errors otherwise
 * as snn_read_synapses.
 */
#define SNN_NOALLOC_MAX_SYNAPSES (1u << 20)
int snn_read_synapses_noalloc(snn_net *net, uint32_t first, uint32_t count, int32_t *host_tgt,
                              uint8_t *host_delay, int32_t *host_w, int32_t *host_sd, size_t cap,
                              size_t *n_out);

/* snn_read_weights -- w and sd of every synapse, canonical order (cap >= synapses). */
int snn_read_weights(snn_net *net, int32_t *host_w, int32_t *host_sd, size_t cap, size_t *n_out);

/* snn_read_neurons -- v and u of neurons [first, first + count) (host, may be NULL). */
int snn_read_neurons(snn_net *net, uint32_t first, uint32_t count, float *host_v, float *host_u);

/* snn_read_neurons_f64 -- v and u in double (exact for SNN_FP64 nets, widened otherwise). */
int snn_read_neurons_f64(snn_net *net, uint32_t first, uint32_t count, double *host_v, double *host_u);

/*
 * snn_set_probe -- membrane traces of chosen neurons (Sec. 2 "Production of
 * observables", which offers optional recording of v and the other state
 * variables of selected neurons; Fig. 2-3): from the next
 * step on, v and u of host_gids[0..n) after every step's update are kept on
 * the device for up to max_steps steps.  n = 0 switches the probe off.
 * SNN_EINVAL for a gid out of range.
 */
int snn_set_probe(snn_net *net, const int32_t *host_gids, uint32_t n, uint32_t max_steps);

/* snn_read_probe -- the traces recorded so far, [step][neuron] order, as
   float (host buffers of cap values each, either may be NULL);
   *steps = steps recorded. */
int snn_read_probe(snn_net *net, float *host_v, float *host_u, size_t cap, uint32_t *steps);

/* snn_read_counters -- event counters and the device error word. */
int snn_read_counters(snn_net *net, snn_counters *out);

/* snn_net_info -- neurons, synapses, device bytes held. */
int snn_net_info(const snn_net *net, uint32_t *n_neurons, int64_t *n_synapses,
                 size_t *device_bytes);

/* snn_set_profile -- 1: time every kernel with CUDA events (no graphs; the
 * kernels of a step run one after another on the net's stream); 0: off. */
int snn_set_profile(snn_net *net, int on);
int snn_read_profile(snn_net *net, snn_profile *out);

/*
 * snn_save_state / snn_load_state -- checkpoint of the dynamic state (t,
 * neurons, spike history, ring, weights, derivatives, counters, raster step
 * offsets) into / from a host buffer.  Call with host_buf NULL to get the
 * size in *n.  Loading needs a net built from the same configuration;
 * SNN_EINVAL (net untouched) for a checkpoint of another configuration or
 * one that changes an inhibitory weight of a generated net (those synapses
 * are not plastic).
 */
int snn_save_state(snn_net *net, void *host_buf, size_t cap, size_t *n);
int snn_load_state(snn_net *net, const void *host_buf, size_t n);

/*
 * snn_autotune -- pick the fastest launch shape for this net: every candidate
 * shape (rows per dense block, resident blocks of the event-driven kernels,
 * neuron block, steps per graph) runs probe_ms steps from a reset, timed with
 * CUDA events; the best is kept and the net is left reset at t = 0.  Results
 * never depend on the shape.  Generated nets only (SNN_ESTATE otherwise).
 * *best (may be NULL) receives the chosen shape.
 */
int snn_autotune(snn_net *net, uint32_t probe_ms, snn_launch *best);

/*
 * Batches: many independent networks on one GPU (the paper's networks of
 * different sizes and fan-outs, Table 3, run side by side).  A batch advances
 * every net it holds with one CUDA-graph launch per chunk of graph_steps
 * steps; inside the chunk every step is one launch per kind of step kernel
 * for all nets together (each block works for one net, on that net's own
 * step, counters and cursors; nets get blocks in proportion to their
 * synapses), so small, launch-bound nets share the GPU with large ones
 * instead of queueing one after another.  Steps that do not fill a chunk run
 * each net's own launches on parallel streams.  Each net
 * keeps its own state and step count (nets may stand at different steps and
 * have different periods), bit-identical to running it alone.  The batch
 * owns no net: free the batch before its nets.  All nets must be on the
 * current device and have profiling off.  A change to any net (stimulus,
 * launch shape, raster reset) makes the batch capture its graph again.
 *   graph_steps: steps per captured chunk (even; 0 = 10).
 * Errors: SNN_EINVAL (empty list, a net twice), SNN_ESTATE (profiling),
 * SNN_ECUDA.
 */
typedef struct snn_batch snn_batch;
int snn_batch_create(snn_net *const *nets, uint32_t n_nets, uint32_t graph_steps, snn_batch **out);

/* snn_batch_run -- advance every net of the batch n_ms steps; returns after
   completion and each net's error-word check. */
int snn_batch_run(snn_batch *batch, uint32_t n_ms);

/* snn_batch_free -- release the batch (not its nets; NULL is allowed). */
void snn_batch_free(snn_batch *batch);

/*
 * snn_batch_set_launch / snn_batch_get_launch -- launch shape of the batch's
 * kernels (deliver_block: threads per column of the column-ordered
 * delivery; deliver_blocks_per_sm, ltp_blocks_per_sm: resident blocks per SM
 * of the event-driven kernels, shared out among the nets in proportion to
 * their synapses; ltp_block, neuron_block, deriv_block, dense_block;
 * graph_steps: steps per captured chunk, even, >= 2).  Zero fields keep the
 * current value; the other fields and the nets' own shapes are not used.
 * Results never depend on the shape.  Errors: SNN_EINVAL.
 */
int snn_batch_set_launch(snn_batch *batch, const snn_launch *launch);
int snn_batch_get_launch(const snn_batch *batch, snn_launch *launch);

/*
 * snn_batch_autotune -- the batch's own autotuner: every candidate shape
 * (threads per column of the column-ordered delivery 128 / 256,
 * resident blocks per SM 4 / 8, steps per chunk 10 / 50) advances every net
 * probe_ms steps from a reset, timed with CUDA events on the batch's stream;
 * the fastest shape is kept and every net is left reset at t = 0.  Generated
 * nets only (SNN_ESTATE otherwise).  *best (may be NULL) receives the shape.
 */
int snn_batch_autotune(snn_batch *batch, uint32_t probe_ms, snn_launch *best);

/*
 * snn_reset -- return a generated net to its initial state (t = 0, initial
 * weights, sd = 0, v = -65 mV, u = 0.2 v, empty ring and raster, counters 0)
 * without rebuilding it; external stimulus is cleared.  SNN_ESTATE for nets
 * built from explicit lists (their initial weights are not kept).
 */
int snn_reset(snn_net *net);

/*
 * snn_thalamic_events -- the thalamic drive of cfg for steps [t0, t0 + n_ms)
 * as host events (Sec. 2 "Distributed generation of reproducible ... external
 * 'thalamic' stimulus": per column and step, thal_per_col_per_ms events, the
 * k-th on neuron floor(r0 * neurons_per_col / 2^32) of Philox4x32-10 with key
 * (seed low, seed high) and counter (t, column, 1, k)), sorted by step.
 * A net built with thal_per_col_per_ms = 0 that receives these events through
 * snn_set_stimulus / snn_run_host evolves bit-identically to one that draws
 * them itself.  Host-only computation; needs no GPU.  *n_out = number of
 * events; SNN_ETRUNC if cap is smaller (host_events may then be NULL).
 */
int snn_thalamic_events(const snn_config *cfg, int32_t t0, uint32_t n_ms, snn_stimulus *host_events,
                        size_t cap, size_t *n_out);

/*
 * snn_microbench_atomics -- measurement only: the rates (10^9 operations per
 * second) of the memory operations the event-driven delivery and
 * potentiation are built from, at the access patterns they use (Sec. 2
 * steps 2.4-2.6: every synaptic event adds its weight into the target's Q16
 * input and reads the target's last spike; Table 2 rows "axonal spikes ->
 * synaptic spikes" and "currents + LTD").  On an int32 array of array_bytes
 * (the size of a net's input array), ops_per_thread operations per thread of
 * one resident wave, each timed once after a warm-up with CUDA events on
 * cuda_stream (NULL: the legacy default stream):
 *   red_global_random   red.global.add.s32 at uniformly random words
 *   red_global_window   the same inside one 1250-word window per warp (one
 *                       column's inputs), the window moving every 64 ops
 *   red_global_coalesced 32 consecutive words per warp instruction
 *   ld_global_random    4-byte loads at uniformly random words (L2 gathers)
 *   atom_shared_window  shared-memory atomicAdd at random words of 1250
 * Allocates array_bytes of device memory with cudaMalloc for the call.
 * Errors: SNN_EINVAL (array below 10 000 bytes or above 16 GiB, no ops),
 * SNN_ENOMEM, SNN_ECUDA.
 */
typedef struct {
    double red_global_random_gops;
    double red_global_window_gops;
    double red_global_coalesced_gops;
    double ld_global_random_gops;
    double atom_shared_window_gops;
    double array_bytes;
    double threads;
} snn_atomic_rates;
int snn_microbench_atomics(size_t array_bytes, uint32_t ops_per_thread, void *cuda_stream,
                           snn_atomic_rates *out);

/* snn_free -- release the handle and its device memory (NULL is allowed). */
void snn_free(snn_net *net);

/* snn_strerror -- static message of an SNN_E* code. */
const char *snn_strerror(int code);

/* snn_last_error -- message of the last failure in this thread (never NULL). */
const char *snn_last_error(void);

/*
 * snn_set_allocator -- route device allocations of nets built afterwards
 * through alloc(bytes, stream, ctx) / release(ptr, ctx) (e.g. a framework's
 * caching allocator).  NULL restores cudaMalloc / cudaFree.  Blocks must be
 * 256-byte aligned (the kernels use 16-byte vector accesses and bulk L2
 * prefetches); a misaligned block is released and the build fails with
 * SNN_ENOMEM.
 */
void snn_set_allocator(void *(*alloc)(size_t bytes, void *stream, void *ctx),
                       void (*release)(void *ptr, void *ctx), void *ctx);

#ifdef __cplusplus
}
#endif
#endif
