// snn_internal.cuh -- device-side data layout and helpers of the GB300 engine
// for the DPSNN-STDP step (arXiv 1310.8478).  Private to csrc/.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "snn.h"

namespace snn {

constexpr int kLut = 256;            // STDP amounts for lags 0..255 (the rest are 0)
constexpr int kDoffStride = 32;      // uint16 delay offsets per source row: [0..D], D <= 31
constexpr int32_t kNever = -(1 << 30);  // "no spike yet" time stamp
constexpr int kNeuronsPerThread = 8; // S2/S3: neurons handled by one thread
constexpr int kKinds = 5;            // profiled kernel kinds: deliver, neuron, ltp, deriv, dense
constexpr int kSlots = 13;           // own column + 3 rings of 4 neighbour columns
constexpr int kSlotStride = 16;      // entries per column in the neighbour table
constexpr int32_t kNoPending = -(1 << 30);  // ltp_pending value when no LTP is owed
constexpr uint32_t kMaxCompactNpc = 4096;    // compact targets slot * npc + local stay below 2^16
constexpr uint32_t kMinCompactNpc = 2;       // the slot reciprocal ceil(2^32 / npc) fits 32 bits
constexpr uint32_t kDenseMaxNpc = 2800;      // staged columns must fit in shared memory
static_assert(kSlots * kMaxCompactNpc <= 65536, "compact targets must fit 16 bits");
constexpr int kUnroll = 4;                   // event-driven walks: synapses per lane in flight

// Device counters and per-step bookkeeping (one struct, device memory).
struct DevCounters {
    unsigned long long spikes, e_all, e_exc, l_exc;
    unsigned long long raster_total, raster_dropped;
    int error;
    int raster_first_drop_t;
    int step_cnt[2][4];              // [t & 1][exc, inh, all, -]: spikes of step t so far
    int t_slot[2];                   // t_slot[t & 1] = t while step t runs
    int ltp_pending;                 // step whose LTP (and long-term update) is still owed
    unsigned done_blocks;            // blocks of k_neuron finished (last block closes the step)
    unsigned long long dense_e_all, dense_e_exc, dense_l_exc;  // work done by the dense pass
    unsigned long long dense_steps, dense_deriv_steps;
    unsigned long long l_exc_mark;   // l_exc when the last step closed
    unsigned long long l_exc_last;   // excitatory in-degree of the neurons that fired in the last step
    unsigned dense_cursor;           // work units of the dense pass handed out in this step
    unsigned staged_cursor;          // columns of the column-staged delivery handed out in this step
    unsigned fold_cursor;            // chunks of reverse entries handed out by the current fold
    int sd_rev_dirty;                // the event-driven potentiation wrote sd_rev since the last fold
    unsigned fold_done;              // blocks of the current fold finished (the last one clears the flag)
};

// Everything a step kernel needs, passed by value.
struct DevNet {
    uint32_t N, npc, ne, C, D;       // neurons, per column, excitatory per column, columns, max delay
    uint32_t D_inh;                  // largest delay of an inhibitory synapse (1 for generated nets)
    int staged_ok;                   // the column-staged delivery may run (compact targets, staging fits)
    int ordered_ok;                  // the column-ordered delivery replaces the ring-order one (compact targets)
    unsigned long long staged_min_events;   // it runs when a step's expected events reach this
    unsigned long long ring_max_events;     // compact nets: a step whose expected events stay below this
                                            // delivers from the ring's spike lists (0: never)
    int32_t w_inh;                   // generated nets: the weight of every inhibitory synapse (not
                                     //                 plastic); the dense pass reads no inhibitory w
    uint32_t uniform_m;              // > 0: row p starts at p * uniform_m (generated nets; the
                                     //       row stride, a multiple of 8 for compact targets)
    uint32_t canon_m;                // generated nets: synapses per row (the fan-out M)
    int64_t S;                       // stored synapse slots (rows padded to the stride)
    const int64_t *row_off;          // [N + 1] first synapse of every source row
    const uint16_t *doff;            // [N][kDoffStride]: synapses of delay <= d, d = 0..D
    int32_t *tgt;                    // [S] target gid (explicit nets / big columns), or NULL
    uint16_t *tgt16;                 // [S] compact target: slot * npc + local id, or NULL
    uint32_t npc_recip;              // ceil(2^32 / npc): slot = umulhi(v, npc_recip) for v < 2^16
    const int32_t *nbr;              // [C][kSlotStride] global column of every slot
    int32_t *w, *sd;                 // [S] weight, STDP derivative; rows sorted by delay
    const int64_t *rin_off;          // [N + 1] reverse index (incoming excitatory synapses)
    const uint64_t *rin;             // source | ordinal-in-row << 32 | delay << 48, or NULL
    const uint32_t *rin32;           // nets with compact targets and rows of at most 2048 slots:
                                     // 4-byte entries (rin32_entry), or NULL
    int32_t *sd_rev;                 // [n_rin] LTP of the event-driven pass, accumulated in
                                     //         reverse-index order (contiguous per target);
                                     //         folded into sd before every long-term update
                                     //         and every read
    int64_t n_rin;
    float *v, *u;                    // [N] membrane potential, recovery variable
    double *vd, *ud;                 // [N] the same in double (SNN_FP64 nets), else NULL
    const int32_t *probe_gid;        // [probe_n] neurons whose v, u are traced
    float *probe_v, *probe_u;        // [probe_cap][probe_n]
    uint32_t probe_n, probe_cap;
    int32_t probe_t0;                // step stored in row 0
    int32_t *I;                      // [N] Q16 input accumulated during S1/S2
    uint2 *hl;                       // [N] x: bit k = fired at step t - k; y: latest spike
                                     //     older than that 32-step window (one 8-byte word,
                                     //     so the LTP gather is a single access)
    int32_t *last_spike;             // [N] latest spike
    int32_t *ring_ids;               // [D][N] spike ids of step s in slot s % D: exc from the
                                     //         front, inh from the back
    int32_t *ring_cnt;               // [D][2] exc / inh counts of every slot
    int32_t *raster_gid;             // [raster_cap]
    int64_t *raster_step_off;        // [steps + 1] raster index of the first spike of a step
    uint64_t raster_cap;
    int32_t raster_t0;               // step whose spikes sit at raster index 0
    const int32_t *lut_p, *lut_m;    // [kLut] LTP / LTD amounts in Q16
    const int32_t *stim_gid, *stim_q16;  // external events sorted by step
    const int64_t *stim_off;         // [stim_t1 - stim_t0 + 1]
    int32_t stim_t0, stim_t1;
    DevCounters *ctr;
    uint32_t thal_per_col;
    int32_t thal_amp;
    uint32_t seed_lo, seed_hi;
    uint32_t flags;
    int32_t deriv_bias, deriv_decay, wmax;
    uint32_t deriv_period;
    uint32_t dense_min_spikes;       // spikes of step t-1 from which step t takes the dense pass
    uint32_t dense_rows;             // source rows per block of the dense pass
    // a tile of a torus partitioned by columns (Sec. 2 "Delivery of spiking
    // messages"): the net integrates and delivers to the neurons of columns
    // [own_c0, own_c1) only; the spikes of the other columns arrive from their
    // owners (snn_inject_spikes).  A whole net owns every column (tile = 0).
    uint32_t own_c0, own_c1;
    int tile;
};

__device__ __forceinline__ bool owned_column(const DevNet &n, uint32_t col)
{
    return col >= n.own_c0 && col < n.own_c1;
}

// The blocks among which one net's share of a launch is split: the whole
// grid of a single-net launch, or the net's range of blocks in a launch that
// steps every net of a batch.  Kernels index their work by (bid, nblk)
// instead of (blockIdx.x, gridDim.x).
struct Part {
    uint32_t bid, nblk;
};

__device__ __forceinline__ Part whole_grid() { return Part{blockIdx.x, gridDim.x}; }
__device__ __forceinline__ uint32_t part_tid(const Part &g) { return g.bid * blockDim.x + threadIdx.x; }
__device__ __forceinline__ uint32_t part_threads(const Part &g) { return g.nblk * blockDim.x; }

// One launch of a kind of step kernel for every net of a batch: block b
// works for net net_of[b] as block b - first[net] of count[net] (a net's
// blocks are contiguous); the net's step t has parity (parity[net] + k) & 1,
// k being the step's index in the captured chunk of steps.
struct BatchLaunch {
    const DevNet *nets;              // [n_nets]
    const uint32_t *first;           // [n_nets] first block of every net
    const uint32_t *count;           // [n_nets] blocks of every net
    const uint32_t *net_of;          // [grid] net of every block
    const uint8_t *parity;           // [n_nets] parity of every net's step at the chunk's start
    uint32_t k;                      // step of the chunk
};

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon et al., SC'11): ten rounds,
// each a pair of 32x32->64 multiplies of words 0 and 2 by the Philox
// multipliers, a word permutation, and xors with the round key; the key
// advances by the golden-ratio and sqrt(3)-1 Weyl increments every round.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
#else
        const uint32_t hi0 = (uint32_t)(((uint64_t)0xD2511F53u * c.x) >> 32);
        const uint32_t hi1 = (uint32_t)(((uint64_t)0xCD9E8D57u * c.z) >> 32);
#endif
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// uniform integer in [0, n) from a 32-bit draw: high word of r * n
__host__ __device__ __forceinline__ uint32_t draw_below(uint32_t r, uint32_t n)
{
#ifdef __CUDA_ARCH__
    return __umulhi(r, n);
#else
    return (uint32_t)(((uint64_t)r * n) >> 32);
#endif
}

// Network-generation parameters (Sec. 2, "Projection of synapses with
// individual delay" and "Bidimensional arrays of neural columns").
struct GenParams {
    uint32_t npc, ne, m, D, gx, gy;
    uint32_t m_store;                // row stride (>= m; the tail of a row is padding)
    uint32_t ring_end[4];            // ordinals of ring k are [ring_end[k-1], ring_end[k])
    uint32_t seed_lo, seed_hi;
    int32_t w_exc0, w_inh0;
};

// slot (0: own column, 1 + 4 (ring - 1) + member) -> column offset on the torus:
// ring 1 members (+1,0) (-1,0) (0,+1) (0,-1); ring 2 (+1,+1) (-1,+1) (+1,-1)
// (-1,-1); ring 3 (+2,0) (-2,0) (0,+2) (0,-2)
__host__ __device__ __forceinline__ void slot_offset(uint32_t slot, int &dx, int &dy)
{
    if (slot == 0) { dx = dy = 0; return; }
    const uint32_t ring = 1 + (slot - 1) / 4, member = (slot - 1) & 3u;
    if (ring == 2) {
        dx = (member & 1u) ? -1 : 1;
        dy = (member & 2u) ? -1 : 1;
    } else {
        const int s = (ring == 1) ? 1 : 2;
        const int sign = (member & 1u) ? -s : s;
        dx = (member < 2u) ? sign : 0;
        dy = (member < 2u) ? 0 : sign;
    }
}

__host__ __device__ __forceinline__ uint32_t slot_column(uint32_t col, uint32_t slot, uint32_t gx, uint32_t gy)
{
    int dx, dy;
    slot_offset(slot, dx, dy);
    int tx = ((int)(col % gx) + dx) % (int)gx;
    if (tx < 0) tx += (int)gx;
    int ty = ((int)(col / gx) + dy) % (int)gy;
    if (ty < 0) ty += (int)gy;
    return (uint32_t)ty * gx + (uint32_t)tx;
}

// Target, delay and slot of ordinal j of source src.  Inhibitory sources: an
// excitatory neuron of the own column, 1 ms.  Excitatory sources: delay
// uniform in 1..D; ordinals are split into the own column and the three rings
// of neighbours by the cumulative percentages; inside a ring the ordinal picks
// the ring's four columns in turn; the target neuron is uniform in the
// column, excluding the source itself.
__host__ __device__ __forceinline__ void gen_synapse(const GenParams &g, uint32_t src, uint32_t j,
                                                     uint32_t &target, uint32_t &delay, uint32_t &slot)
{
    const uint4 r = philox10(make_uint4(src, j, 0u, 0u), g.seed_lo, g.seed_hi);
    const uint32_t col = src / g.npc;
    const uint32_t local = src - col * g.npc;
    slot = 0;
    if (local >= g.ne) {
        target = col * g.npc + draw_below(r.x, g.ne);
        delay = 1;
        return;
    }
    delay = 1 + draw_below(r.y, g.D);
    uint32_t tcol = col;
    if (j >= g.ring_end[0]) {
        const uint32_t ring = (j < g.ring_end[1]) ? 1u : (j < g.ring_end[2]) ? 2u : 3u;
        slot = 1u + 4u * (ring - 1u) + ((j - g.ring_end[ring - 1]) & 3u);
        tcol = slot_column(col, slot, g.gx, g.gy);
    }
    uint32_t tl;
    if (tcol == col) {
        tl = draw_below(r.x, g.npc - 1);
        tl += (tl >= local) ? 1u : 0u;
    } else {
        tl = draw_below(r.x, g.npc);
    }
    target = tcol * g.npc + tl;
}

// the slot of the opposite column offset: the column of slot s seen from
// the target's side (ring 1 and 3 members come in +/- pairs, ring 2 members
// pair with their diagonal opposite)
__host__ __device__ __forceinline__ uint32_t inverse_slot(uint32_t slot)
{
    if (slot == 0) return 0;
    const uint32_t ring = (slot - 1) / 4, member = (slot - 1) & 3u;
    return 1 + 4 * ring + (ring == 1 ? 3u - member : member ^ 1u);
}

// 4-byte reverse entry: bits 0..15 the source as inverse_slot * npc + local
// id (the same packing as the compact forward targets, relative to the
// target's column), bits 16..20 the delay, bits 21..31 the synapse's position
// in the stored source row
constexpr uint32_t kRin32MaxRow = 2048;
__host__ __device__ __forceinline__ uint32_t rin32_entry(uint32_t inv_slot, uint32_t npc, uint32_t local, uint32_t d,
                                                         uint32_t pos)
{
    return (inv_slot * npc + local) | (d << 16) | (pos << 21);
}

// target gid of synapse k whose source lives in column src_col
__device__ __forceinline__ uint32_t target_gid(const DevNet &n, uint32_t src_col, int64_t k)
{
    if (n.tgt16) {
        const uint32_t v = n.tgt16[k];
        const uint32_t slot = __umulhi(v, n.npc_recip);
        return (uint32_t)n.nbr[src_col * kSlotStride + slot] * n.npc + (v - slot * n.npc);
    }
    return (uint32_t)n.tgt[k];
}

// the step takes the dense pass when enough neurons fired in the previous step
__device__ __forceinline__ bool dense_selected(const DevNet &n, int t)
{
    if (!n.tgt16 || n.npc > kDenseMaxNpc || t < 1) return false;
    const int slot = (t - 1) % (int)n.D;
    return (uint32_t)(n.ring_cnt[2 * slot] + n.ring_cnt[2 * slot + 1]) >= n.dense_min_spikes;
}

// Checked builds (-DSNN_CHECKED) verify every computed index before use: a
// bad one sets the device error word to SNN_EBOUNDS (first error kept) and the
// caller skips the access.  Other builds compile the checks out.
#ifdef SNN_CHECKED
__device__ __forceinline__ bool out_of_range(const DevNet &n, bool ok)
{
    if (!ok) atomicCAS(&n.ctr->error, 0, SNN_EBOUNDS);
    return !ok;
}
#else
__device__ __forceinline__ bool out_of_range(const DevNet &, bool)
{
    return false;
}
#endif

// a step's expected events: excitatory spikes of t - d reach bucket d (about
// M / D synapses), inhibitory spikes of t - 1 their whole row (generated
// nets: inhibitory delay 1)
__device__ __forceinline__ unsigned long long expected_events(const DevNet &n, int t)
{
    if (t < 1) return 0;
    unsigned long long exc = 0;
    for (int d = 1; d <= (int)n.D && d <= t; ++d) exc += (unsigned)n.ring_cnt[2 * ((t - d) % (int)n.D)];
    const unsigned long long inh = (unsigned)n.ring_cnt[2 * ((t - 1) % (int)n.D) + 1];
    return exc * n.canon_m / n.D + inh * n.canon_m;
}

// a step without the dense pass delivers column by column through shared
// memory when its expected events reach staged_min_events
__device__ __forceinline__ bool staged_selected(const DevNet &n, int t)
{
    if (!n.staged_ok || t < 1 || dense_selected(n, t)) return false;
    return expected_events(n, t) >= n.staged_min_events;
}

// compact nets deliver a step with few expected events from the ring's
// spike lists (a few rounds of latency, no scan of every row's history)
__device__ __forceinline__ bool light_selected(const DevNet &n, int t)
{
    return n.ordered_ok && !n.tile && n.ring_max_events && !dense_selected(n, t) && !staged_selected(n, t) &&
           expected_events(n, t) < n.ring_max_events;
}

// compact nets deliver the remaining event-driven steps column by column
__device__ __forceinline__ bool ordered_selected(const DevNet &n, int t)
{
    return n.ordered_ok && !dense_selected(n, t) && !staged_selected(n, t) && !light_selected(n, t);
}

// the ring-order delivery: nets without compact targets, and light steps
__device__ __forceinline__ bool ring_selected(const DevNet &n, int t)
{
    if (dense_selected(n, t) || staged_selected(n, t)) return false;
    return !n.ordered_ok || light_selected(n, t);
}

__device__ __forceinline__ int64_t row_base(const DevNet &n, uint32_t p)
{
    return n.uniform_m ? (int64_t)p * n.uniform_m : n.row_off[p];
}

// synapses of row p, and the canonical (unpadded) index of its first synapse
__device__ __forceinline__ int64_t row_len(const DevNet &n, uint32_t p)
{
    return n.uniform_m ? (int64_t)n.canon_m : n.row_off[p + 1] - n.row_off[p];
}

__device__ __forceinline__ int64_t canon_base(const DevNet &n, uint32_t p)
{
    return n.uniform_m ? (int64_t)p * n.canon_m : n.row_off[p];
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---- kernel entry points (defined in snn_build.cu / snn_step.cu) ----------
// ---------------------------------------------------------------------------
// device helpers shared by the step kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ void red_add(int32_t *p, int32_t v)
{
    asm volatile("red.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ T block_sum(T x)
{
    __shared__ T s_part[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_part[warp] = x;
    __syncthreads();
    T r = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += s_part[i];
    __syncthreads();
    return r;   // valid in thread 0
}

__device__ __forceinline__ int32_t deriv_w(const DevNet &n, int32_t w, int32_t s)
{
    long long nw = (long long)w + n.deriv_bias + s;
    nw = nw < 0 ? 0 : (nw > n.wmax ? n.wmax : nw);
    return (int32_t)nw;
}

__device__ __forceinline__ int32_t deriv_sd(const DevNet &n, int32_t s)
{
    return (int32_t)(((long long)s * n.deriv_decay + 32768) >> 16);
}

// Bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a
// multiple of 16); nothing waits on it.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The 16-byte-aligned part of [p, p + bytes) into L2 (never past either end).
__device__ __forceinline__ void prefetch_inside(const void *p, size_t bytes)
{
    const uintptr_t a = ((uintptr_t)p + 15u) & ~(uintptr_t)15u, b = ((uintptr_t)p + bytes) & ~(uintptr_t)15u;
    if (b > a) prefetch_l2(reinterpret_cast<const void *>(a), (uint32_t)(b - a));
}

// thalamic drive (thal_per_col events per column, Philox keyed by (t, col))
// and the external events of step t, by the threads of a whole grid
__device__ __forceinline__ void drive(const DevNet &n, int t, uint32_t gtid, uint32_t gthreads)
{
    const uint32_t n_thal = n.C * n.thal_per_col;
    for (uint32_t e = gtid; e < n_thal; e += gthreads) {
        const uint32_t col = e / n.thal_per_col, k = e - col * n.thal_per_col;
        const uint4 r = philox10(make_uint4((uint32_t)t, col, 1u, k), n.seed_lo, n.seed_hi);
        red_add(&n.I[col * n.npc + draw_below(r.x, n.npc)], n.thal_amp);
    }
    if (t >= n.stim_t0 && t < n.stim_t1) {
        const int64_t lo = n.stim_off[t - n.stim_t0], hi = n.stim_off[t - n.stim_t0 + 1];
        for (int64_t e = lo + gtid; e < hi; e += gthreads) red_add(&n.I[n.stim_gid[e]], n.stim_q16[e]);
    }
}

__global__ void k_gen_rows(GenParams g, uint32_t n_rows, uint16_t *doff, int32_t *tgt, uint16_t *tgt16,
                           int32_t *w, int32_t *sd);
__global__ void k_count_indeg(DevNet n, int32_t *indeg_exc, int32_t *indeg_inh);
__global__ void k_scan_sums(const int32_t *in, uint32_t n, long long *block_sums);
__global__ void k_scan_carry(long long *block_sums, uint32_t n_blocks);
__global__ void k_scan_write(const int32_t *in, uint32_t n, const long long *block_sums, int64_t *out);
__global__ void k_fill_reverse(DevNet n, int32_t *cursor, uint64_t *rin, uint32_t *rin32);
__global__ void k_max2(const int32_t *a, const int32_t *b, uint32_t n, int32_t *out2);
__global__ void k_init_state(DevNet n);
__global__ void k_reset_weights(DevNet n, int32_t w_exc0, int32_t w_inh0);
__global__ void k_read_rows(DevNet n, GenParams g, const uint8_t *canon_delay, uint32_t first,
                            uint32_t count, int64_t out_base, int32_t *o_tgt, uint8_t *o_delay,
                            int32_t *o_w, int32_t *o_sd);

__global__ void k_deliver(DevNet n, const int *t_now);
__global__ void k_dense(DevNet n, const int *t_now);
__global__ void k_deliver_cols(DevNet n, const int *t_now);
__global__ void k_deliver_ordered(DevNet n, const int *t_now);
__global__ void k_neuron_f32(DevNet n, const int *t_now, int *t_next);
__global__ void k_neuron_f64(DevNet n, const int *t_now, int *t_next);
__global__ void k_probe(DevNet n, const int *t_now);
__global__ void k_ltp(DevNet n, const int *t_now, int force);
__global__ void k_deriv(DevNet n, const int *t_now, int force);
__global__ void k_fold(DevNet n, const int *t_now, int force);
__global__ void k_inject(DevNet n, int t, const int32_t *gid, uint32_t count);

// the same kernels for every net of a batch in one launch (BatchLaunch)
__global__ void k_deliver_b(BatchLaunch b);
__global__ void k_dense_b(BatchLaunch b);
__global__ void k_deliver_cols_b(BatchLaunch b);
__global__ void k_deliver_ordered_b(BatchLaunch b);
__global__ void k_neuron_f32_b(BatchLaunch b);
__global__ void k_neuron_f64_b(BatchLaunch b);
__global__ void k_probe_b(BatchLaunch b);
__global__ void k_ltp_b(BatchLaunch b);
__global__ void k_deriv_b(BatchLaunch b);
__global__ void k_fold_b(BatchLaunch b);

// net, part and step slots of a block of a batched launch
struct BatchBlock {
    uint32_t net;
    Part part;
    const int *t_now;
    int *t_next;
};

__device__ __forceinline__ BatchBlock batch_block(const BatchLaunch &b)
{
    BatchBlock x;
    x.net = b.net_of[blockIdx.x];
    x.part = Part{blockIdx.x - b.first[x.net], b.count[x.net]};
    const int par = (int)((b.parity[x.net] + b.k) & 1u);
    x.t_now = &b.nets[x.net].ctr->t_slot[par];
    x.t_next = &b.nets[x.net].ctr->t_slot[par ^ 1];
    return x;
}

size_t dense_smem_bytes(uint32_t npc, uint32_t block);
size_t staged_smem_bytes(uint32_t npc, uint32_t block);
size_t ordered_smem_bytes(uint32_t npc, uint32_t block);
constexpr uint32_t kStagedBlock = 512;      // threads per block of the column-staged delivery
// the column-ordered delivery is compiled for five resident blocks of at most
// this many threads per SM (47 registers; the measured optimum): a launch
// shape asking for more threads per block is clamped to it
constexpr uint32_t kOrderedMaxBlock = 256;
__host__ __device__ __forceinline__ uint32_t ordered_block(uint32_t deliver_block)
{
    return deliver_block < kOrderedMaxBlock ? deliver_block : kOrderedMaxBlock;
}

}  // namespace snn
