// snn_dense.cu -- the dense synapse pass of the DPSNN-STDP step on GB300.
//
// In steps where a large part of the network fired, the first bracket of the
// step, [S4(t-1) S5(t-1) S1(t)] (paper Sec. 2, cycle steps 2.1 and 2.3-2.6,
// Table 2 "long term synaptic plasticity"), is done by one pass that streams
// every source row once: per synapse LTP(t-1) -> long-term update at a period
// end -> delivery + LTD(t), in the same per-synapse order as the event-driven
// kernels of snn_step.cu, so both give bit-identical results.
#include "snn_internal.cuh"

namespace snn {

// ---------------------------------------------------------------------------
size_t dense_smem_bytes(uint32_t npc, uint32_t block)
{
    const size_t warps = block / 32;
    return 2 * kLut * 4                       // LTP / LTD tables
           + (size_t)kSlots * npc * 4         // staged input
           + warps * 32 * 4 * 2               // per-warp bucket offsets, LTP amounts
           + (((size_t)kSlots * npc * 2 + 15) & ~size_t(15));  // packed target words
}

// Packed per-target word of the dense pass, one per staged neuron: bit 15 set
// when the neuron fired in the previous step (its incoming synapses owe LTP),
// bits 0..14 the depression an arrival now applies (LTD table at the lag since
// its last spike; 0 without STDP).  The host enables the dense pass only when
// every LTD amount fits 15 bits.
constexpr uint32_t kFiredLast = 0x8000u;
constexpr uint32_t kDepMask = 0x7fffu;

// One row of the dense pass: the lane takes 8 consecutive synapses per pass,
// with one 16-byte target load and two 16-byte weight and derivative loads.
// A chunk of 8 lies in one or two delay buckets almost always (buckets hold
// M / D synapses); the deliver flags (bit d of fbits: the source fired at
// t - d) and LTP amounts of its positions come from bit masks, and only a
// chunk spread over three or more buckets walks them position by position.
// kDeriv: the step closes a plasticity period (the long-term update runs
// between LTP and delivery) -- excitatory rows only.
constexpr int kPrefetchAhead = 1;   // segments of 256 synapses between a warp's loads and its prefetches

// The 256 synapses from position k (a multiple of 8) into L2: targets, and
// weights and derivatives when asked.
__device__ __forceinline__ void prefetch_segment(const DevNet &n, int64_t k, bool w, bool sd)
{
    if (k >= n.S) return;
    const uint32_t cnt = (uint32_t)min((int64_t)256, n.S - k);
    prefetch_l2(n.tgt16 + k, cnt * 2u);
    if (w) prefetch_l2(n.w + k, cnt * 4u);
    if (sd) prefetch_l2(n.sd + k, cnt * 4u);
}

template <bool kExc, bool kDeriv>
__device__ __forceinline__ void dense_row_walk(const DevNet &n, int64_t base, int m, int D, float scale, uint32_t fbits,
                                               bool stdp, bool ltp_on, const int32_t *w_off, const int32_t *w_amt,
                                               int32_t *s_in, const uint16_t *s_x, int lane, int64_t next_base,
                                               bool next_exc)
{
    const uint4 *rt4 = reinterpret_cast<const uint4 *>(n.tgt16 + base);
    int4 *rw4 = reinterpret_cast<int4 *>(n.w + base);
    int4 *rs4 = reinterpret_cast<int4 *>(n.sd + base);
    // what the row needs at all: its chunks' loads go out before the bucket
    // search so that the search runs under their latency
    const bool row_w = kDeriv || fbits != 0;
    const bool row_sd = kExc && (kDeriv || ltp_on || (stdp && fbits != 0));
    const uint32_t staged = kSlots * n.npc;
    for (int c = lane; c * 8 < m; c += 32) {
        const int k0 = c * 8;
        // the warp's next 256-synapse segment (in this row or at the
        // start of its next row) goes to L2 while this chunk is processed: a
        // pipeline that costs no registers
        if (lane == 0) {
            const int ka = k0 + kPrefetchAhead * 256, mr = (m + 255) & ~255;
            if (ka < m) prefetch_segment(n, base + ka, row_w, row_sd);
            else if (next_base >= 0) prefetch_segment(n, next_base + (ka - mr), true, next_exc);
        }
        if (out_of_range(n, base + k0 + 8 <= n.S)) continue;
        const uint4 tv = rt4[c];
        int4 wa = make_int4(0, 0, 0, 0), wb = wa, sa = wa, sb = wa;
        if (row_w) {
            wa = rw4[2 * c];
            wb = rw4[2 * c + 1];
        }
        if (row_sd) {
            sa = rs4[2 * c];
            sb = rs4[2 * c + 1];
        }
        // bucket of k0 (first d with end > k0): delays are near uniform along
        // a row, so the interpolated guess is right or one off almost always
        int lo = min(D, 1 + (int)((float)k0 * scale));
        while (w_off[lo] <= k0) ++lo;         // bucket D ends at m > k0
        while (w_off[lo - 1] > k0) --lo;      // w_off[0] = 0 <= k0
        const int nv = min(8, m - k0);        // valid positions (the row's last chunk is short)
        const int e0 = w_off[lo];
        const int n0 = min(e0 - k0, nv);      // positions in bucket lo
        uint32_t fmask = ((fbits >> lo) & 1u) ? (1u << n0) - 1u : 0u;
        const int32_t a0 = kExc ? w_amt[lo] : 0;
        int32_t a1 = 0;
        int n1 = n0;                          // positions before n1 are in bucket lo or lo + 1
        if (n0 < nv && w_off[lo + 1] >= k0 + nv) {   // lo < D here: bucket D ends at m
            n1 = nv;
            fmask |= ((fbits >> (lo + 1)) & 1u) ? ((1u << nv) - 1u) & ~((1u << n0) - 1u) : 0u;
            if (kExc) a1 = w_amt[lo + 1];
        }
        int32_t am[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) am[u] = (u < n0) ? a0 : ((u < nv) ? a1 : 0);
        if (n1 < nv) {
            // three or more buckets (or an empty one) inside the chunk
            int d = lo, nb = e0;
            fmask = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + u;
                if (u < nv) {
                    while (k >= nb) nb = w_off[++d];
                    fmask |= ((fbits >> d) & 1u) << u;
                    am[u] = kExc ? w_amt[d] : 0;
                }
            }
        }
        const uint32_t tw[4] = {tv.x, tv.y, tv.z, tv.w};
        int32_t wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
        if (!kExc) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t v = (u & 1) ? (tw[u >> 1] >> 16) : (tw[u >> 1] & 0xffffu);
                if (out_of_range(n, v < staged)) continue;
                if ((fmask >> u) & 1u) atomicAdd(&s_in[v], wv[u]);
            }
            continue;
        }
        int32_t sv[8] = {sa.x, sa.y, sa.z, sa.w, sb.x, sb.y, sb.z, sb.w};
        bool sd_dirty = kDeriv;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const bool f = (fmask >> u) & 1u;
            const uint32_t v = (u & 1) ? (tw[u >> 1] >> 16) : (tw[u >> 1] & 0xffffu);
            if (out_of_range(n, v < staged)) continue;
            const uint32_t x = s_x[v];
            int32_t sdv = sv[u];
            if ((x & kFiredLast) && am[u]) {
                sdv += am[u];
                sd_dirty = true;
            }
            if (kDeriv && u < nv) {
                wv[u] = deriv_w(n, wv[u], sdv);
                sdv = deriv_sd(n, sdv);
            }
            if (f) {
                atomicAdd(&s_in[v], wv[u]);
                const int32_t dep = (int32_t)(x & kDepMask);
                sdv -= dep;
                sd_dirty |= dep != 0;
            }
            sv[u] = sdv;
        }
        if (sd_dirty) {
            rs4[2 * c] = make_int4(sv[0], sv[1], sv[2], sv[3]);
            rs4[2 * c + 1] = make_int4(sv[4], sv[5], sv[6], sv[7]);
        }
        if (kDeriv) {
            rw4[2 * c] = make_int4(wv[0], wv[1], wv[2], wv[3]);
            rw4[2 * c + 1] = make_int4(wv[4], wv[5], wv[6], wv[7]);
        }
    }
}

__device__ __forceinline__ void dense_body(const DevNet &n, const int *t_now, const Part &g)
{
    extern __shared__ int4 smem_i4[];
    const int t = *t_now;
    if (!dense_selected(n, t)) return;
    const uint32_t npc = n.npc;
    const uint32_t nwarps = blockDim.x >> 5;
    int32_t *s_lutp = reinterpret_cast<int32_t *>(smem_i4);
    int32_t *s_lutm = s_lutp + kLut;
    int32_t *s_in = s_lutm + kLut;                              // [kSlots * npc]
    int32_t *s_off = s_in + kSlots * npc;                       // [nwarps][32] bucket end offsets
    int32_t *s_amt = s_off + nwarps * 32;                       // [nwarps][32] LTP amount
    uint16_t *s_x = reinterpret_cast<uint16_t *>(s_amt + nwarps * 32);   // [kSlots * npc] packed words
    __shared__ uint32_t s_col[kSlots];

    const bool stdp = !(n.flags & SNN_STDP_OFF);
    const bool deliver_on = !(n.flags & SNN_DELIVERY_OFF);
    const bool owed = n.ctr->ltp_pending == t - 1;
    const bool ltp_on = owed && stdp;
    const bool deriv_on = owed && n.deriv_period && (t % (int)n.deriv_period) == 0;
    const uint32_t chunks = (npc + n.dense_rows - 1) / n.dense_rows;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kLut; i += blockDim.x) {
        s_lutp[i] = n.lut_p[i];
        s_lutm[i] = n.lut_m[i];
    }
    drive(n, t, part_tid(g), part_threads(g));
    int32_t *w_off = s_off + warp * 32;
    int32_t *w_amt = s_amt + warp * 32;
    const int D = (int)n.D;
    const uint32_t dmask = (2u << D) - 2u;            // buckets 1..D
    unsigned long long ev_all = 0, ev_exc = 0;
    // the grid is at most one wave of resident blocks; a block takes work
    // units (a column and a chunk of its rows) from a step-wide cursor
    __shared__ uint32_t s_unit;
    for (uint32_t unit = g.bid; unit < n.C * chunks;) {
        const uint32_t col = unit / chunks;
        const uint32_t r0 = (unit - col * chunks) * n.dense_rows;
        const uint32_t r1 = min(npc, r0 + n.dense_rows);
        if (threadIdx.x < kSlots) s_col[threadIdx.x] = (uint32_t)n.nbr[col * kSlotStride + threadIdx.x];
        // every warp's first row starts streaming into L2 while the block stages
        if (lane == 0 && r0 + warp < r1) {
            const int64_t b = row_base(n, col * npc + r0 + warp);
            for (int sgm = 0; sgm < kPrefetchAhead; ++sgm)
                prefetch_segment(n, b + sgm * 256, true, r0 + warp < n.ne);
        }
        __syncthreads();
        for (int sl = 0; sl < kSlots; ++sl) {
            const int32_t *ls = n.last_spike + (size_t)s_col[sl] * npc;
            uint16_t *x_row = s_x + sl * npc;
            int32_t *in_row = s_in + sl * npc;
            for (uint32_t loc = threadIdx.x; loc < npc; loc += blockDim.x) {
                const int lag = min(t - ls[loc], 255);
                x_row[loc] = (uint16_t)((lag == 1 ? kFiredLast : 0u) | (stdp ? (uint32_t)s_lutm[lag] : 0u));
                in_row[loc] = 0;
            }
        }
        __syncthreads();
        // row metadata goes out one row ahead: the spike-history word and, in lane
        // d <= D, the end of delay bucket d
        uint2 hv_next = make_uint2(0u, 0u);
        int off_next = 0;
        if (r0 + warp < r1) {
            const uint32_t p = col * npc + r0 + warp;
            hv_next = n.hl[p];
            off_next = (lane <= D) ? (int)n.doff[(size_t)p * kDoffStride + lane] : 0;
        }
        for (uint32_t r = r0 + warp; r < r1; r += nwarps) {
            const uint32_t p = col * npc + r;
            const bool exc = r < n.ne;
            const uint2 hv = hv_next;
            const int hi = off_next;
            if (r + nwarps < r1) {
                hv_next = n.hl[p + nwarps];
                off_next = (lane <= D) ? (int)n.doff[(size_t)(p + nwarps) * kDoffStride + lane] : 0;
            }
            const uint32_t h = hv.x;                      // bit k: fired at t - 1 - k
            const uint32_t fbits = deliver_on ? (h << 1) & dmask : 0u;
            const int lo = __shfl_up_sync(0xffffffffu, hi, 1);
            const int m = __shfl_sync(0xffffffffu, hi, D);
            // lane d (1..D) prepares bucket d
            int len = 0;
            int32_t amt = 0;
            if (lane == 0) w_off[0] = 0;
            if (lane >= 1 && lane <= D) {
                len = hi - lo;
                w_off[lane] = hi;
                if (exc && ltp_on && len) {
                    const uint32_t recent = h & (0xffffffffu << lane);
                    const int lag = recent ? (__ffs(recent) - 1 - lane) : (t - 1 - (int)hv.y - lane);
                    amt = lag < kLut ? s_lutp[lag] : 0;
                }
                w_amt[lane] = amt;
            }
            const int delivered = ((fbits >> lane) & 1u) ? len : 0;
            const bool busy = fbits != 0 || __any_sync(0xffffffffu, amt != 0) || (exc && deriv_on);
            const int dl = __reduce_add_sync(0xffffffffu, delivered);
            if (lane == 0) {
                ev_all += (unsigned long long)dl;
                if (exc) ev_exc += (unsigned long long)dl;
            }
            __syncwarp();
            if (!exc && n.D_inh == 1) {
                // inhibitory row of a generated net: one bucket (delay 1), one
                // weight, nothing plastic
                if (fbits & 2u) {
                    const int64_t base = row_base(n, p);
                    const uint4 *rt4 = reinterpret_cast<const uint4 *>(n.tgt16 + base);
                    const int64_t nbase = r + nwarps < r1 ? row_base(n, p + nwarps) : -1;
                    for (int c = lane; c * 8 < m; c += 32) {
                        if (lane == 0) {        // next segment of targets, as in the row walk
                            const int ka = c * 8 + 256, mr = (m + 255) & ~255;
                            if (ka < m) prefetch_segment(n, base + ka, false, false);
                            else if (nbase >= 0) prefetch_segment(n, nbase + (ka - mr), false, false);
                        }
                        if (out_of_range(n, base + c * 8 + 8 <= n.S)) continue;
                        const uint4 tv = rt4[c];
                        const int nv = min(8, m - c * 8);
                        const uint32_t tw[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const uint32_t v = (u & 1) ? (tw[u >> 1] >> 16) : (tw[u >> 1] & 0xffffu);
                            if (u < nv && !out_of_range(n, v < kSlots * npc)) atomicAdd(&s_in[v], n.w_inh);
                        }
                    }
                }
            } else if (busy) {
                const float scale = (float)D / (float)m;
                const int64_t base = row_base(n, p);     // a multiple of 8: rows are padded
                const int64_t nbase = r + nwarps < r1 ? row_base(n, p + nwarps) : -1;
                const bool nexc = r + nwarps < n.ne;
                if (!exc)
                    dense_row_walk<false, false>(n, base, m, D, scale, fbits, stdp, ltp_on, w_off, w_amt, s_in, s_x,
                                                 lane, nbase, nexc);
                else if (deriv_on)
                    dense_row_walk<true, true>(n, base, m, D, scale, fbits, stdp, ltp_on, w_off, w_amt, s_in, s_x,
                                               lane, nbase, nexc);
                else
                    dense_row_walk<true, false>(n, base, m, D, scale, fbits, stdp, ltp_on, w_off, w_amt, s_in, s_x,
                                                lane, nbase, nexc);
            }
            __syncwarp();
        }
        __syncthreads();
        for (int sl = 0; sl < kSlots; ++sl) {
            int32_t *dst = n.I + (size_t)s_col[sl] * npc;
            const int32_t *in_row = s_in + sl * npc;
            for (uint32_t loc = threadIdx.x; loc < npc; loc += blockDim.x) {
                const int32_t v = in_row[loc];
                if (v) red_add(&dst[loc], v);
            }
        }
        if (threadIdx.x == 0) s_unit = g.nblk + atomicAdd(&n.ctr->dense_cursor, 1u);
        __syncthreads();
        unit = s_unit;
    }
    if (lane != 0) ev_all = ev_exc = 0;
    const unsigned long long ba = block_sum(ev_all);
    const unsigned long long be = block_sum(ev_exc);
    if (threadIdx.x == 0) {
        if (ba) {
            atomicAdd(&n.ctr->e_all, ba);
            atomicAdd(&n.ctr->e_exc, be);
            atomicAdd(&n.ctr->dense_e_all, ba);
            atomicAdd(&n.ctr->dense_e_exc, be);
        }
        if (g.bid == 0) {
            // potentiation visits: every incoming excitatory synapse of the
            // neurons that fired at t - 1 (counted when those spikes closed)
            if (ltp_on) n.ctr->dense_l_exc += n.ctr->l_exc_last;
            n.ctr->dense_steps += 1;
            if (deriv_on) n.ctr->dense_deriv_steps += 1;
        }
    }
}

__global__ void __launch_bounds__(1024) k_dense(DevNet n, const int *t_now) { dense_body(n, t_now, whole_grid()); }

__global__ void __launch_bounds__(1024) k_dense_b(BatchLaunch b)
{
    const BatchBlock x = batch_block(b);
    const DevNet n = b.nets[x.net];
    dense_body(n, x.t_now, x.part);
}

}  // namespace snn
