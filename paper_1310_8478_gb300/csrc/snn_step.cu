// snn_step.cu -- the per-millisecond step of the DPSNN-STDP engine on GB300.
//
// Paper, Sec. 2 "Mixed time-driven and event driven simulation": synapses are
// event driven, neurons time driven.  The cycle 2.1-2.7 is taken as
//   S1 delivery of the spikes due at t + LTD       (2.3-2.6)
//   S2 thalamic drive + Izhikevich update          (2.7)
//   S3 spike compaction into the ring and raster   (2.2)
//   S4 LTP of the incoming synapses of the spikers (2.1)
//   S5 long-term update at the end of each period
// The device runs step t as
//   [S4(t-1) S5(t-1) S1(t)] then [S2(t) S3(t)]
// i.e. the potentiation owed by the previous step travels with this step's
// delivery, so that one pass over the synapses can do both.  Two
// interchangeable implementations of the first bracket exist:
//   sparse (event driven): k_ltp (reverse index of the spikers of t-1; the
//       amounts accumulate in sd_rev, laid out like the reverse index so the
//       updates of one target are contiguous), k_fold (sd += sd_rev before a
//       long-term update), k_deriv, and one of three deliveries of the
//       flagged delay buckets: k_deliver_ordered (compact nets, sources
//       column by column, global reductions), k_deliver_cols (compact nets,
//       many events: column by column through shared memory), k_deliver
//       (other nets, (spike, delay) items of the ring lists);
//   dense (snn_dense.cu): k_dense streams every source row once, in
//       per-synapse order LTP(t-1) -> long-term update -> delivery + LTD(t),
//       with the target columns' input and post-spike state staged in shared
//       memory.
// The choice is taken on the device from the ring counts (the spikes of step
// t-1 for the dense pass, the expected events of step t for the staged
// delivery; every kernel of the step reads the same counts); all give
// bit-identical results because all synaptic arithmetic is int32 and the
// per-synapse order of the updates is the same.  An LTP still owed when a run ends is applied
// by the host-side flush (k_ltp + k_deriv with force = 1) before any read.
#include <type_traits>

#include "snn_internal.cuh"

namespace snn {

// ---------------------------------------------------------------------------
// sparse S1: work items are (spike, delay) pairs -- every excitatory spike of
// step t - d for d = 1..D and every inhibitory spike of step t - d for
// d = 1..D_inh (generated nets: inhibitory synapses all have delay 1).  Lanes
// add the weight into the target's Q16 input with a fire-and-forget L2
// reduction and, on plastic synapses, subtract the LTD amount at lag
// t - last_spike[target].
// ---------------------------------------------------------------------------
__device__ __forceinline__ void deliver_ring(const DevNet &n, const int *t_now, const Part &g)
{
    __shared__ int32_t s_lut[kLut];
    __shared__ int s_start[2 * 32 + 1];
    __shared__ const int32_t *s_list[2 * 32];
    __shared__ int64_t s_tile_lo[32 * 32];       // per warp: first synapse of each of its 32 items
    __shared__ int s_tile_start[32 * 33];        // per warp: prefix of the items' lengths
    __shared__ uint32_t s_tile_info[32 * 32];    // per warp: kind and source column of each item
    const int t = *t_now;
    if (!ring_selected(n, t)) return;
    const bool stdp = !(n.flags & SNN_STDP_OFF);
    const int nl = (int)(n.D + n.D_inh);
    for (int i = threadIdx.x; i < kLut; i += blockDim.x) s_lut[i] = n.lut_m[i];
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int l = 0; l < nl; ++l) {
            const bool inh = l >= (int)n.D;
            const int d = inh ? l - (int)n.D + 1 : l + 1;
            int cnt = 0;
            const int32_t *list = nullptr;
            if (!(n.flags & SNN_DELIVERY_OFF) && t - d >= 0) {
                const int slot = (t - d) % (int)n.D;
                cnt = n.ring_cnt[2 * slot + (inh ? 1 : 0)];
                list = n.ring_ids + (size_t)slot * n.N;
            }
            s_start[l] = acc;
            s_list[l] = list;
            acc += cnt;
        }
        s_start[nl] = acc;
    }
    __syncthreads();
    const uint32_t gtid = part_tid(g);
    const uint32_t gthreads = part_threads(g);
    drive(n, t, gtid, gthreads);

    const int total = s_start[nl];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t warps = gthreads >> 5;
    unsigned long long ev_all = 0, ev_exc = 0;
    // A warp takes 32 items at a time (one per lane), prefix-sums their bucket
    // lengths and walks the concatenated synapses with all 32 lanes, so short
    // buckets do not leave lanes idle.
    int64_t *w_lo = s_tile_lo + warp * 32;
    int *w_start = s_tile_start + warp * 33;
    uint32_t *w_info = s_tile_info + warp * 32;
    for (uint32_t tile = (gtid >> 5) * 32; tile < (uint32_t)total; tile += warps * 32) {
        const uint32_t item = tile + lane;
        int len = 0;
        int64_t lo = 0;
        uint32_t info = 0;                       // bit 0: excitatory; bits 1..: source column
        if (item < (uint32_t)total) {
            int l = 0;
            while (s_start[l + 1] <= (int)item) ++l;
            const int idx = (int)item - s_start[l];
            const bool inh = l >= (int)n.D;
            const int d = inh ? l - (int)n.D + 1 : l + 1;
            const uint32_t p = (uint32_t)(inh ? s_list[l][n.N - 1 - idx] : s_list[l][idx]);
            if (!out_of_range(n, p < n.N)) {
                const uint16_t *off = n.doff + (size_t)p * kDoffStride;
                lo = row_base(n, p) + off[d - 1];
                len = (int)off[d] - (int)off[d - 1];
                info = (inh ? 0u : 1u) | ((p / n.npc) << 1);
            }
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int tile_len = __shfl_sync(0xffffffffu, incl, 31);
        const int exc_len = __reduce_add_sync(0xffffffffu, (info & 1u) ? len : 0);
        w_lo[lane] = lo;
        w_start[lane] = incl - len;
        w_info[lane] = info;
        if (lane == 0) {
            w_start[32] = tile_len;
            ev_all += (unsigned long long)tile_len;
            ev_exc += (unsigned long long)exc_len;
        }
        __syncwarp();
        // kUnroll synapses per lane in flight: weights, derivatives and
        // targets first, then the target-side gathers, then the updates
        int j = 0;
        for (int e0 = lane; e0 < tile_len; e0 += 32 * kUnroll) {
            int64_t k[kUnroll];
            uint32_t inf[kUnroll], tg[kUnroll];
            int32_t wk[kUnroll], ls[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int e = e0 + 32 * u;
                k[u] = -1;
                if (e < tile_len) {
                    while (w_start[j + 1] <= e) ++j;
                    k[u] = w_lo[j] + (e - w_start[j]);
                    if (out_of_range(n, k[u] < n.S)) {
                        k[u] = -1;
                        continue;
                    }
                    inf[u] = w_info[j];
                    wk[u] = n.w[k[u]];
                    tg[u] = target_gid(n, inf[u] >> 1, k[u]);
                    if (out_of_range(n, tg[u] < n.N)) k[u] = -1;
                }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                if (k[u] < 0) continue;
                red_add(&n.I[tg[u]], wk[u]);
                ls[u] = ((inf[u] & 1u) && stdp) ? n.last_spike[tg[u]] : 0;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                if (k[u] < 0 || !((inf[u] & 1u) && stdp)) continue;
                const int lag = t - ls[u];                     // >= 1
                if (lag < kLut) {
                    const int32_t a = s_lut[lag];
                    if (a) red_add(&n.sd[k[u]], -a);
                }
            }
        }
        __syncwarp();
    }
    if (lane != 0) ev_all = ev_exc = 0;
    const unsigned long long ba = block_sum(ev_all);
    const unsigned long long be = block_sum(ev_exc);
    if (threadIdx.x == 0 && ba) {
        atomicAdd(&n.ctr->e_all, ba);
        atomicAdd(&n.ctr->e_exc, be);
    }
}

// ---------------------------------------------------------------------------
// sparse S1, column by column (generated nets with compact targets).  A
// persistent grid takes source columns from a step-wide cursor, so the
// columns in flight form a narrow band of the torus and so do the targets
// they reach.  Per column, every thread first issues its share of the loads
// of the column's spike-history words and its neurons' last spikes (one
// round of latency for the whole column).  Then the warps take 32-row groups
// from a block cursor, the inhibitory groups first (an inhibitory spike
// delivers its whole row at delay 1, an excitatory one a single delay
// bucket: longest work first, so the warps finish the column together); a
// warp turns every delay bucket d whose source fired at t - d into an item
// and walks the 8-synapse chunks of 32 items with all lanes, one 16-byte
// load of 8 targets (and of 4 weights / derivatives twice) per chunk.
//   kStage (steps with many events): the input accumulators and LTD amounts
//   of the 13 columns the block's synapses reach are staged in shared memory,
//   so an event costs a shared atomic and a shared load; the input is flushed
//   with one coalesced reduction per touched neuron.
//   otherwise: only the source column's own neurons are staged (the targets
//   of every inhibitory synapse and of the local share of the excitatory
//   ones); an event on another column is an L2 reduction into the target's
//   input and a gather of its last spike, both on the band of columns in
//   flight, which stays in L2.
// ---------------------------------------------------------------------------
constexpr int kItemCap = 96;                // per warp: pending (row, bucket) items
// per warp: first chunk, chunk-count prefix, first / end synapse, kind of each
// item, pending items
constexpr int kTileWords = 32 + 33 + 32 + 32 + 32 + kItemCap;

size_t staged_smem_bytes(uint32_t npc, uint32_t block)
{
    return (size_t)kLut * 4 + (size_t)kSlots * npc * 4 + (size_t)npc * 4 + (size_t)(block / 32) * kTileWords * 4 +
           (((size_t)kSlots * npc * 2 + 15) & ~size_t(15));
}

size_t ordered_smem_bytes(uint32_t npc, uint32_t block)
{
    return (size_t)kLut * 4 + (size_t)npc * 16 + (size_t)(block / 32) * kTileWords * 4;
}

// s_amt: kStage -> uint16 LTD amounts of the 13 staged columns;
//        otherwise int32 LTD amounts of the source column's own neurons.
// s_hist: the history words (bit k: fired at t - k) of the column's rows.
template <bool kStage>
__device__ __forceinline__ void deliver_cols(const DevNet &n, int t, int32_t *s_lut, int32_t *s_in, int32_t *s_tile,
                                             void *s_amt, uint32_t *s_hist, const Part &g, uint32_t *s_inh = nullptr)
{
    __shared__ uint32_t s_col[kSlots];
    __shared__ uint32_t s_unit[2];             // the next column, claimed while this one is walked
    __shared__ uint32_t s_grp;                 // row groups of the current column handed out
    __shared__ uint32_t s_ninh;                // inhibitory rows of the column that fired at t - 1
    uint16_t *s_x = reinterpret_cast<uint16_t *>(s_amt);
    int32_t *s_ltd = reinterpret_cast<int32_t *>(s_amt);
    const uint32_t npc = n.npc;
    const uint32_t ngroups = (npc + 31) / 32;
    const bool stdp = !(n.flags & SNN_STDP_OFF);
    const bool deliver_on = !(n.flags & SNN_DELIVERY_OFF);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kLut; i += blockDim.x) s_lut[i] = n.lut_m[i];
    drive(n, t, part_tid(g), part_threads(g));
    __syncthreads();                  // the table is read by every thread's column setup below
    const int D = (int)n.D;
    const uint32_t dmask_e = (2u << D) - 2u, dmask_i = (2u << n.D_inh) - 2u;
    int32_t *w_c0 = s_tile + warp * kTileWords;                // [32] first chunk (column-relative)
    int32_t *w_start = w_c0 + 32;                              // [33] prefix of the chunk counts
    int32_t *w_a = w_start + 33;                               // [32] first synapse (column-relative)
    int32_t *w_b = w_a + 32;                                   // [32] end synapse
    int32_t *w_exc = w_b + 32;                                 // [32] 1: excitatory row
    uint32_t *w_items = reinterpret_cast<uint32_t *>(w_exc + 32);   // [kItemCap] pending items
    unsigned long long ev_all = 0, ev_exc = 0;
    uint32_t par = 0;
    for (uint32_t col = g.bid; col < n.C; par ^= 1u) {
        if (threadIdx.x < kSlots) s_col[threadIdx.x] = (uint32_t)n.nbr[col * kSlotStride + threadIdx.x];
        if (threadIdx.x == 0) {
            s_grp = 0;
            s_ninh = 0;
            s_unit[par] = g.nblk + atomicAdd(&n.ctr->staged_cursor, 1u);
        }
        if (kStage) __syncthreads();
        // one round of loads for the whole column: history words, and the
        // staged neurons' last spikes turned into LTD amounts at lag
        // t - last_spike >= 1 (saturated at the table end, whose entry is 0)
        if (!kStage) {
            constexpr int kSetup = 8;                  // rows per thread in flight
            const int32_t *ls = n.last_spike + (size_t)col * npc;
            const uint2 *hl = n.hl + (size_t)col * npc;
            for (uint32_t base = threadIdx.x; base < npc; base += kSetup * blockDim.x) {
                uint32_t hv[kSetup];
                int32_t lv[kSetup];
#pragma unroll
                for (int q = 0; q < kSetup; ++q) {
                    const uint32_t loc = base + q * blockDim.x;
                    hv[q] = 0;
                    lv[q] = kNever;
                    if (loc < npc) {
                        if (deliver_on) hv[q] = hl[loc].x;
                        lv[q] = ls[loc];
                    }
                }
#pragma unroll
                for (int q = 0; q < kSetup; ++q) {
                    const uint32_t loc = base + q * blockDim.x;
                    if (loc < npc) {
                        s_hist[loc] = hv[q];
                        s_ltd[loc] = stdp ? s_lut[min(t - lv[q], kLut - 1)] : 0;
                        s_in[loc] = 0;
                    }
                }
            }
        } else {
            for (uint32_t loc = threadIdx.x; loc < npc; loc += blockDim.x)
                s_hist[loc] = deliver_on ? n.hl[col * npc + loc].x : 0u;
            // at most 15 bits per amount: the host checks the table
            for (int sl = 0; sl < kSlots; ++sl) {
                const int32_t *ls = n.last_spike + (size_t)s_col[sl] * npc;
                uint16_t *x_row = s_x + sl * npc;
                int32_t *in_row = s_in + sl * npc;
                for (uint32_t loc = threadIdx.x; loc < npc; loc += blockDim.x) {
                    x_row[loc] = stdp ? (uint16_t)s_lut[min(t - ls[loc], kLut - 1)] : (uint16_t)0;
                    in_row[loc] = 0;
                }
            }
        }
        __syncthreads();
        const int64_t cbase = (int64_t)col * npc * n.uniform_m;   // first synapse of the column (8-aligned)
        const uint4 *t4 = reinterpret_cast<const uint4 *>(n.tgt16 + cbase);
        const int4 *w4 = reinterpret_cast<const int4 *>(n.w + cbase);
        const int64_t col_syn = (int64_t)npc * n.uniform_m;       // synapse slots of the column
        // one tile: lane i takes item (row r, bucket d) when valid, the warp
        // prefix-sums the items' chunk counts and walks the concatenated
        // chunks with all lanes
        auto tile = [&](uint32_t r, int d, bool valid) {
            int a = 0, b = 0, exc = 0, c0 = 0, nch = 0;
            if (valid) {
                const uint16_t *off = n.doff + (size_t)(col * npc + r) * kDoffStride;
                a = (int)(r * n.uniform_m) + off[d - 1];
                b = (int)(r * n.uniform_m) + off[d];
                exc = r < n.ne ? 1 : 0;
                c0 = a >> 3;
                nch = b > a ? ((b - 1) >> 3) - c0 + 1 : 0;
            }
            int incl = nch;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            const int len_all = __reduce_add_sync(0xffffffffu, b - a);
            const int len_exc = __reduce_add_sync(0xffffffffu, exc ? b - a : 0);
            w_c0[lane] = c0;
            w_start[lane] = incl - nch;
            w_a[lane] = a;
            w_b[lane] = b;
            w_exc[lane] = exc;
            if (lane == 0) {
                w_start[32] = total;
                if (!n.tile) {                 // a tile counts the events on its own columns below
                    ev_all += (unsigned long long)len_all;
                    ev_exc += (unsigned long long)len_exc;
                }
            }
            __syncwarp();
            int j = 0;
            for (int e = lane; e < total; e += 32) {
                while (w_start[j + 1] <= e) ++j;
                const int c = w_c0[j] + (e - w_start[j]);
                const int k0 = 8 * c;                               // column-relative first synapse
                const int ia = w_a[j], ib = w_b[j];
                const bool ex = w_exc[j] != 0;
                if (out_of_range(n, k0 >= 0 && k0 + 8 <= col_syn && cbase + k0 + 8 <= n.S)) continue;
                // positions of the chunk inside the item's bucket
                const uint32_t lo_u = (uint32_t)max(ia - k0, 0), hi_u = (uint32_t)min(ib - k0, 8);
                const uint32_t mask = ((1u << hi_u) - 1u) & ~((1u << lo_u) - 1u);
                const uint4 tv = t4[c];
                int4 wa = make_int4(n.w_inh, n.w_inh, n.w_inh, n.w_inh), wb = wa;
                if (ex) {
                    wa = w4[2 * c];
                    wb = w4[2 * c + 1];
                }
                const uint32_t tw[4] = {tv.x, tv.y, tv.z, tv.w};
                const int32_t wk[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
                int tile_ev = 0;                                    // tiles: events on own columns
                int32_t am[8];                                      // LTD amount, or (remote) last spike
                uint32_t remote = 0;                                // bit u: target on another column
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    am[u] = 0;
                    if (!((mask >> u) & 1u)) continue;
                    const uint32_t v = (tw[u >> 1] >> (16 * (u & 1))) & 0xffffu;
                    if (out_of_range(n, v < kSlots * npc)) continue;
                    if (kStage) {
                        atomicAdd(&s_in[v], wk[u]);
                        am[u] = (ex && stdp) ? (int32_t)s_x[v] : 0;
                    } else {
                        const uint32_t slot = __umulhi(v, n.npc_recip);
                        const uint32_t loc = v - slot * npc;
                        if (n.tile && !owned_column(n, s_col[slot])) continue;   // another tile's target
                        if (n.tile) ++tile_ev;
                        if (slot == 0) {
                            atomicAdd(&s_in[loc], wk[u]);
                            am[u] = (ex && stdp) ? s_ltd[loc] : 0;
                        } else {
                            const uint32_t gid = s_col[slot] * npc + loc;        // target gid
                            red_add(&n.I[gid], wk[u]);
                            if (ex && stdp) {
                                am[u] = n.last_spike[gid];
                                remote |= 1u << u;
                            }
                        }
                    }
                }
                if (n.tile) {
                    ev_all += (unsigned long long)tile_ev;
                    if (ex) ev_exc += (unsigned long long)tile_ev;
                }
                if (ex && stdp) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (!((mask >> u) & 1u)) continue;
                        int32_t x = am[u];
                        if ((remote >> u) & 1u) {
                            const int lag = t - x;                            // >= 1
                            x = lag < kLut ? s_lut[lag] : 0;
                        }
                        if (x) red_add(&n.sd[cbase + k0 + u], -x);     // no load: most amounts are 0
                    }
                }
            }
            __syncwarp();
        };
        // Without 13-column staging, the inhibitory rows that fired at t - 1
        // are walked by the whole block first: such a row delivers all of its
        // synapses at delay 1, with one weight, to excitatory neurons of its
        // own column (generated nets), so the block lists them and spreads
        // the concatenated rows' chunks over all threads -- an even share
        // whatever the rows' distribution over the groups.
        if (!kStage) {
            const bool mine = deliver_on && (!n.tile || owned_column(n, col));
            if (mine)
                for (uint32_t r = n.ne + threadIdx.x; r < npc; r += blockDim.x)
                    if (s_hist[r] & 1u) s_inh[atomicAdd(&s_ninh, 1u)] = r;
            __syncthreads();
            const uint32_t ninh = s_ninh;
            const uint32_t m = n.canon_m, cpr = (m + 7u) / 8u;
            for (uint32_t c = threadIdx.x; c < ninh * cpr; c += blockDim.x) {
                const uint32_t it = c / cpr, ci = c - it * cpr;
                const int64_t k0 = (int64_t)s_inh[it] * n.uniform_m + 8 * ci;   // column-relative
                if (out_of_range(n, k0 + 8 <= col_syn && cbase + k0 + 8 <= n.S)) continue;
                const uint4 tv = t4[k0 >> 3];
                const uint32_t nv = min(8u, m - 8u * ci);
                const uint32_t tw[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const uint32_t v = (tw[u >> 1] >> (16 * (u & 1))) & 0xffffu;
                    if ((uint32_t)u < nv && !out_of_range(n, v < npc)) atomicAdd(&s_in[v], n.w_inh);
                }
            }
            if (threadIdx.x == 0) ev_all += (unsigned long long)ninh * m;
        }
        // Items (row << 5 | bucket) collect in the warp's buffer across row
        // groups and are walked 32 at a time, so that a tile is full even when
        // few rows of a group fired; a group with too many items for the
        // buffer is walked directly, one flagged bucket per lane and pass.
        // (Without staging the inhibitory rows are done above: the groups
        // cover the excitatory rows only.)
        const uint32_t ngroups_w = kStage ? ngroups : (n.ne + 31u) / 32u;
        int cnt = 0;                                   // items in the buffer
        bool groups_left = true;                       // warp-uniform
        uint32_t fb = 0, r = 0;                        // a group walked directly: its remaining flags
        for (;;) {
            uint32_t tr = 0;
            int td = 0;
            bool tv = false;
            if (__any_sync(0xffffffffu, fb != 0)) {
                // direct walk: every lane takes the lowest flagged bucket of its row
                td = fb ? __ffs(fb) - 1 : 0;
                fb &= fb - 1u;
                tr = r;
                tv = td != 0;
            } else if (cnt >= 32 || (cnt > 0 && !groups_left)) {
                const int take = min(cnt, 32);
                cnt -= take;
                const uint32_t it = lane < take ? w_items[cnt + lane] : 0u;
                tr = it >> 5;
                td = (int)(it & 31u);
                tv = lane < take;
            } else if (groups_left) {
                uint32_t grp = 0;
                if (lane == 0) grp = atomicAdd(&s_grp, 1u);
                grp = __shfl_sync(0xffffffffu, grp, 0);
                if (grp >= ngroups_w) {
                    groups_left = false;
                    continue;
                }
                r = (ngroups_w - 1u - grp) * 32u + lane;   // the last groups (inhibitory rows) first
                uint32_t f = 0;                        // bit d: the row's source fired at t - d
                if (r < npc && (kStage || r < n.ne)) f = (s_hist[r] << 1) & (r < n.ne ? dmask_e : dmask_i);
                const int mine = __popc(f);
                int incl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                // a group of inhibitory rows is walked at once: each of its
                // items is a whole row, long enough to fill a tile, and
                // walking them first is what the longest-first order is for
                const bool inh_group = (r - lane) >= n.ne;
                if (!inh_group && cnt + total <= kItemCap) {
                    int pos = cnt + incl - mine;
                    while (f) {
                        w_items[pos++] = (r << 5) | (uint32_t)(__ffs(f) - 1);
                        f &= f - 1u;
                    }
                    cnt += total;
                    __syncwarp();
                } else {
                    fb = f;                            // walk this group directly, one flagged bucket per lane and pass
                }
                continue;
            } else {
                break;
            }
            tile(tr, td, tv);
        }
        __syncthreads();
        if (kStage) {
            for (int sl = 0; sl < kSlots; ++sl) {
                int32_t *dst = n.I + (size_t)s_col[sl] * npc;
                const int32_t *in_row = s_in + sl * npc;
                for (uint32_t loc = threadIdx.x; loc < npc; loc += blockDim.x) {
                    const int32_t x = in_row[loc];
                    if (x) red_add(&dst[loc], x);
                }
            }
        } else {
            int32_t *dst = n.I + (size_t)col * npc;
            for (uint32_t loc = threadIdx.x; loc < npc; loc += blockDim.x) {
                const int32_t x = s_in[loc];
                if (x) red_add(&dst[loc], x);
            }
        }
        __syncthreads();
        col = s_unit[par];
    }
    if (lane != 0 && !n.tile) ev_all = ev_exc = 0;
    const unsigned long long ba = block_sum(ev_all);
    const unsigned long long be = block_sum(ev_exc);
    if (threadIdx.x == 0 && ba) {
        atomicAdd(&n.ctr->e_all, ba);
        atomicAdd(&n.ctr->e_exc, be);
    }
}

__device__ __forceinline__ void deliver_staged(const DevNet &n, const int *t_now, const Part &g)
{
    extern __shared__ int4 smem_i4[];
    const int t = *t_now;
    if (!staged_selected(n, t)) return;
    const uint32_t npc = n.npc, nwarps = blockDim.x >> 5;
    int32_t *s_lut = reinterpret_cast<int32_t *>(smem_i4);
    int32_t *s_in = s_lut + kLut;                                        // [kSlots * npc]
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(s_in + kSlots * npc);   // [npc]
    int32_t *s_tile = reinterpret_cast<int32_t *>(s_hist + npc);         // [nwarps][kTileWords]
    uint16_t *s_x = reinterpret_cast<uint16_t *>(s_tile + nwarps * kTileWords);   // [kSlots * npc]
    deliver_cols<true>(n, t, s_lut, s_in, s_tile, s_x, s_hist, g);
}

__device__ __forceinline__ void deliver_ordered(const DevNet &n, const int *t_now, const Part &g)
{
    extern __shared__ int4 smem_i4[];
    const int t = *t_now;
    if (!ordered_selected(n, t)) return;
    const uint32_t npc = n.npc;
    int32_t *s_lut = reinterpret_cast<int32_t *>(smem_i4);
    int32_t *s_in = s_lut + kLut;                                        // [npc]
    int32_t *s_ltd = s_in + npc;                                         // [npc]
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(s_ltd + npc);        // [npc]
    uint32_t *s_inh = s_hist + npc;                                      // [npc]
    int32_t *s_tile = reinterpret_cast<int32_t *>(s_inh + npc);          // [nwarps][kTileWords]
    deliver_cols<false>(n, t, s_lut, s_in, s_tile, s_ltd, s_hist, g, s_inh);
}

// One target's reverse entries [lo, hi), walked by a warp, kUnroll entries
// per lane and pass: the entries, then the sources' history words, then a
// reduction of every non-zero amount into the entry's accumulator (no load:
// an entry whose source did not fire inside the window costs its 4 or 8
// bytes and nothing else).  The entries of the next pass are loaded before
// the current pass's histories are gathered, so that the two loads'
// latencies overlap.  Returns whether the lane added into an accumulator.
template <bool kCompact>
__device__ __forceinline__ bool ltp_walk(const DevNet &n, int64_t lo, int64_t hi, int lane, const int32_t *nb,
                                         const int32_t *s_lut, int tp)
{
    using Raw = typename std::conditional<kCompact, uint32_t, uint64_t>::type;
    constexpr Raw kNone = ~(Raw)0;                // no entry (never a valid one: the delay is below 32)
    auto load = [&](int64_t e) -> Raw {
        if (e >= hi || out_of_range(n, e < n.n_rin)) return kNone;
        if constexpr (kCompact) return n.rin32[e];
        else return n.rin[e];
    };
    bool wrote = false;
    Raw next[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) next[u] = load(lo + lane + 32 * u);
    for (int64_t e0 = lo + lane; e0 < hi; e0 += 32 * kUnroll) {
        Raw r[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            r[u] = next[u];
            next[u] = load(e0 + 32 * (kUnroll + u));
        }
        uint2 h[kUnroll];
        uint32_t dl[kUnroll];
        bool ok[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            ok[u] = r[u] != kNone;
            if (!ok[u]) continue;
            uint32_t src;
            if constexpr (kCompact) {
                const uint32_t v = r[u] & 0xffffu;
                const uint32_t sl = __umulhi(v, n.npc_recip);
                src = (uint32_t)nb[sl] * n.npc + (v - sl * n.npc);
                dl[u] = (r[u] >> 16) & 31u;
            } else {
                src = (uint32_t)r[u];
                dl[u] = (uint32_t)(r[u] >> 48);
            }
            if (out_of_range(n, src < n.N)) {
                ok[u] = false;
                continue;
            }
            h[u] = n.hl[src];
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (!ok[u]) continue;
            const uint32_t d = dl[u];
            const uint32_t recent = h[u].x & (0xffffffffu << d);
            const int lag = recent ? (__ffs(recent) - 1 - (int)d) : (tp - (int)h[u].y - (int)d);
            if (lag < kLut) {
                const int32_t a = s_lut[lag];
                if (a) {
                    red_add(&n.sd_rev[e0 + 32 * u], a);   // coalesced: the target's entries are contiguous
                    wrote = true;
                }
            }
        }
    }
    return wrote;
}

// ---------------------------------------------------------------------------
// sparse S4 for step t - 1: warp per neuron that fired at t - 1; lanes walk
// its incoming excitatory synapses.  The nearest arrival with t_pre + d <=
// t - 1 is the lowest set bit k >= d of the source's 32-step history (lag
// k - d), else its latest older spike last_old (lag t - 1 - last_old - d).
// Reverse entries are 4 bytes on nets with compact targets (the source as
// slot * npc + local id relative to the target's column, the delay and the
// source row position; see rin32_entry) and 8 bytes otherwise.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ltp_body(const DevNet &n, const int *t_now, int force, const Part &g)
{
    __shared__ int32_t s_lut[kLut];
    __shared__ int32_t s_nb[32][kSlotStride];        // per warp: the neighbour columns of its target
    const int t = *t_now;
    const int tp = t - 1;
    if (n.ctr->ltp_pending != tp || (n.flags & SNN_STDP_OFF)) return;
    if (!force && dense_selected(n, t)) return;
    const int slot = tp % (int)n.D;
    const int ce = n.ring_cnt[2 * slot], ci = n.ring_cnt[2 * slot + 1];
    const int total = ce + ci;
    // a block whose first warp has no spiker leaves at once (steps with few
    // spikes use a small part of the grid)
    if ((int64_t)((g.bid * blockDim.x) >> 5) >= (int64_t)total) return;
    for (int i = threadIdx.x; i < kLut; i += blockDim.x) s_lut[i] = n.lut_p[i];
    __syncthreads();
    const int32_t *ring = n.ring_ids + (size_t)slot * n.N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t warps = part_threads(g) >> 5;
    const bool compact = n.rin32 != nullptr;
    int32_t *nb = s_nb[warp];
    bool wrote = false;                           // this thread added into sd_rev
    auto spiker = [&](uint32_t item) -> int32_t {
        return (int)item < ce ? ring[item] : ring[n.N - 1 - ((int)item - ce)];
    };
    // the reverse-entry ranges of the warp's next two spikers are known one
    // item ahead, and the next one's entries go to L2 while this one is walked
    // (compact entries: lanes 0..15 hold the neighbour columns of those
    // spikers' columns, loaded as far ahead)
    const uint32_t first = part_tid(g) >> 5;
    int64_t lo1 = 0, hi1 = 0, lo2 = 0, hi2 = 0;
    int32_t nb1 = 0, nb2 = 0;
    auto neighbours = [&](int32_t p) -> int32_t {
        return (compact && lane < kSlotStride) ? n.nbr[((uint32_t)p / n.npc) * kSlotStride + lane] : 0;
    };
    if (first < (uint32_t)total) {
        const int32_t p = spiker(first);
        lo1 = n.rin_off[p];
        hi1 = n.rin_off[p + 1];
        nb1 = neighbours(p);
    }
    if (first + warps < (uint32_t)total) {
        const int32_t p = spiker(first + warps);
        lo2 = n.rin_off[p];
        hi2 = n.rin_off[p + 1];
        nb2 = neighbours(p);
    }
    for (uint32_t item = first; item < (uint32_t)total; item += warps) {
        int64_t lo = lo1, hi = hi1;
        if (n.tile && !owned_column(n, (uint32_t)spiker(item) / n.npc)) hi = lo;   // another tile's synapses
        if (compact) {
            if (lane < kSlotStride) nb[lane] = nb1;
            __syncwarp();
        }
        lo1 = lo2;
        hi1 = hi2;
        nb1 = nb2;
        if (lane == 0 && hi1 > lo1) {
            if (compact) prefetch_inside(n.rin32 + lo1, (size_t)(hi1 - lo1) * 4);
            else prefetch_inside(n.rin + lo1, (size_t)(hi1 - lo1) * 8);
        }
        if (item + 2 * warps < (uint32_t)total) {
            const int32_t p = spiker(item + 2 * warps);
            lo2 = n.rin_off[p];
            hi2 = n.rin_off[p + 1];
            nb2 = neighbours(p);
        }
        if (compact) wrote |= ltp_walk<true>(n, lo, hi, lane, nb, s_lut, tp);
        else wrote |= ltp_walk<false>(n, lo, hi, lane, nb, s_lut, tp);
        __syncwarp();
    }
    if (__any_sync(0xffffffffu, wrote) && lane == 0) n.ctr->sd_rev_dirty = 1;
}

// ---------------------------------------------------------------------------
// fold the event-driven LTP accumulated in reverse order into the forward
// derivatives (each forward excitatory synapse has exactly one reverse entry)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fold_body(const DevNet &n, const int *t_now, int force, const Part &g)
{
    if (!force) {
        const int t = *t_now;        // only before a long-term update (t closes a period)
        if (!n.deriv_period || t <= 0 || (t % (int)n.deriv_period) != 0) return;
    }
    // Chunks of kFoldTargets consecutive targets are handed out in order, so
    // the targets in flight form a narrow band of the torus and so do the
    // source rows their synapses scatter into: the scatter stays in L2.  A
    // warp takes one target at a time, four entries per lane in flight.
    // nothing to fold when no potentiation was accumulated since the last
    // fold (every block sees the same flag: it is cleared only after all of
    // them have finished)
    if (!*(volatile int *)&n.ctr->sd_rev_dirty) return;
    __shared__ uint32_t s_chunk;
    __shared__ int32_t s_nb[32][kSlotStride];
    constexpr uint32_t kFoldTargets = 64;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool compact = n.rin32 != nullptr;
    int32_t *nb = s_nb[warp];
    for (uint32_t c0 = g.bid * kFoldTargets; c0 < n.N;) {
        const uint32_t c1 = min(c0 + kFoldTargets, n.N);
        for (uint32_t p = c0 + warp; p < c1; p += nw) {
            const int64_t lo = n.rin_off[p], hi = n.rin_off[p + 1];
            if (compact) {
                if (lane < kSlotStride) nb[lane] = n.nbr[(p / n.npc) * kSlotStride + lane];
                __syncwarp();
            }
            for (int64_t e0 = lo + lane; e0 < hi; e0 += 32 * 4) {
                int32_t v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t e = e0 + 32 * u;
                    v[u] = (e < hi && !out_of_range(n, e < n.n_rin)) ? n.sd_rev[e] : 0;
                }
                int64_t fwd[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (!v[u]) continue;
                    uint32_t src, pos;
                    if (compact) {
                        const uint32_t r = n.rin32[e0 + 32 * u];
                        const uint32_t x = r & 0xffffu;
                        const uint32_t sl = __umulhi(x, n.npc_recip);
                        src = (uint32_t)nb[sl] * n.npc + (x - sl * n.npc);
                        pos = r >> 21;
                    } else {
                        const uint64_t r = n.rin[e0 + 32 * u];
                        src = (uint32_t)r;
                        pos = (uint32_t)(r >> 32) & 0xffffu;
                    }
                    fwd[u] = row_base(n, src) + pos;
                    if (out_of_range(n, src < n.N && fwd[u] < n.S)) v[u] = 0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (!v[u]) continue;
                    red_add(&n.sd[fwd[u]], v[u]);
                    n.sd_rev[e0 + 32 * u] = 0;
                }
            }
            __syncwarp();
        }
        __syncthreads();
        if (threadIdx.x == 0) s_chunk = (g.nblk + atomicAdd(&n.ctr->fold_cursor, 1u)) * kFoldTargets;
        __syncthreads();
        c0 = s_chunk;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&n.ctr->fold_done, 1u) == g.nblk - 1) {
            n.ctr->sd_rev_dirty = 0;
            n.ctr->fold_done = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// sparse S5 closing step t - 1 (when t is a multiple of the period): warp per
// excitatory row (grid-stride, so a step that closes no period costs one tiny
// launch): w = clamp(w + bias + sd, 0, wmax), sd = (sd*decay + 2^15) >> 16.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void deriv_body(const DevNet &n, const int *t_now, int force, const Part &g)
{
    const int t = *t_now;
    if (!n.deriv_period || t <= 0 || (t % (int)n.deriv_period) != 0) return;
    if (n.ctr->ltp_pending != t - 1) return;
    if (!force && dense_selected(n, t)) return;
    const int lane = threadIdx.x & 31;
    const uint32_t rows = n.C * n.ne;
    const uint32_t warps = part_threads(g) >> 5;
    for (uint32_t r = part_tid(g) >> 5; r < rows; r += warps) {
        const uint32_t p = (r / n.ne) * n.npc + (r % n.ne);
        const int64_t lo = row_base(n, p), hi = lo + row_len(n, p);
        for (int64_t k = lo + lane; k < hi; k += 32) {
            const int32_t s = n.sd[k];
            n.w[k] = deriv_w(n, n.w[k], s);
            n.sd[k] = deriv_sd(n, s);
        }
    }
}

// ---------------------------------------------------------------------------
// S2 + S3: Izhikevich update (paper Sec. 2 "Spiking neuron model"; v in two
// 0.5 ms Euler substeps, u in one 1 ms step, Sec. 3) of kNeuronsPerThread
// neurons per thread, one block-wide compaction of the neurons that fired
// into ring slot t % D (exc ids from the front, inh ids from the back) and
// into the raster.  The last block to finish closes the step: ring counts,
// counters, raster step offset, LTP owed for step t, next time stamp.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool izhikevich_step(float &v, float &u, int32_t iq, bool exc)
{
    const float a = exc ? 0.02f : 0.1f;
    const float b = 0.2f;
    const float c = -65.0f;
    const float d = exc ? 8.0f : 2.0f;
    const float cur = __fmul_rn(__int2float_rn(iq), 0x1p-16f);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float x = __fmul_rn(0.04f, v);
        x = __fadd_rn(x, 5.0f);
        x = __fmul_rn(x, v);
        x = __fadd_rn(x, 140.0f);
        x = __fsub_rn(x, u);
        x = __fadd_rn(x, cur);
        x = __fmul_rn(0.5f, x);
        v = __fadd_rn(v, x);
    }
    float y = __fmul_rn(b, v);
    y = __fsub_rn(y, u);
    y = __fmul_rn(a, y);
    u = __fadd_rn(u, y);
    if (v >= 30.0f) {
        v = c;
        u = __fadd_rn(u, d);
        return true;
    }
    return false;
}

// the same scheme in double (SNN_FP64): identical operation order, decimal
// parameters
__device__ __forceinline__ bool izhikevich_step(double &v, double &u, int32_t iq, bool exc)
{
    const double a = exc ? 0.02 : 0.1;
    const double b = 0.2;
    const double c = -65.0;
    const double d = exc ? 8.0 : 2.0;
    const double cur = __dmul_rn(__int2double_rn(iq), 0x1p-16);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        double x = __dmul_rn(0.04, v);
        x = __dadd_rn(x, 5.0);
        x = __dmul_rn(x, v);
        x = __dadd_rn(x, 140.0);
        x = __dsub_rn(x, u);
        x = __dadd_rn(x, cur);
        x = __dmul_rn(0.5, x);
        v = __dadd_rn(v, x);
    }
    double y = __dmul_rn(b, v);
    y = __dsub_rn(y, u);
    y = __dmul_rn(a, y);
    u = __dadd_rn(u, y);
    if (v >= 30.0) {
        v = c;
        u = __dadd_rn(u, d);
        return true;
    }
    return false;
}

template <typename F> __device__ __forceinline__ F *state_v(const DevNet &n);
template <> __device__ __forceinline__ float *state_v<float>(const DevNet &n) { return n.v; }
template <> __device__ __forceinline__ double *state_v<double>(const DevNet &n) { return n.vd; }
template <typename F> __device__ __forceinline__ F *state_u(const DevNet &n);
template <> __device__ __forceinline__ float *state_u<float>(const DevNet &n) { return n.u; }
template <> __device__ __forceinline__ double *state_u<double>(const DevNet &n) { return n.ud; }

template <typename F>
__device__ __forceinline__ void neuron_body(const DevNet &n, const int *t_now, int *t_next, const Part &g)
{
    F *const sv = state_v<F>(n);
    F *const su = state_u<F>(n);
    const int t = *t_now;
    const int par = t & 1;
    const uint32_t tile = blockDim.x * kNeuronsPerThread;
    const uint32_t first = g.bid * tile;
    uint32_t fe = 0, fi = 0;          // bit it: neuron first + it * blockDim + tid fired
    unsigned long long indeg = 0;     // excitatory in-degree of the neurons that fired
    // all loads of the thread's neurons first, then the updates and stores
    int32_t iq[kNeuronsPerThread];
    F vv[kNeuronsPerThread], uu[kNeuronsPerThread];
    uint2 hh[kNeuronsPerThread];
#pragma unroll
    for (int it = 0; it < kNeuronsPerThread; ++it) {
        const uint32_t i = first + it * blockDim.x + threadIdx.x;
        if (i < n.N) {
            iq[it] = n.I[i];
            vv[it] = sv[i];
            uu[it] = su[i];
            hh[it] = n.hl[i];
        }
    }
#pragma unroll
    for (int it = 0; it < kNeuronsPerThread; ++it) {
        const uint32_t i = first + it * blockDim.x + threadIdx.x;
        if (i >= n.N) break;
        const bool exc = (i % n.npc) < n.ne;
        F v = vv[it], u = uu[it];
        // a tile leaves the neurons of other columns to their owners (their
        // spikes of this step are injected afterwards)
        const bool mine = !n.tile || owned_column(n, i / n.npc);
        const bool fired = mine && izhikevich_step(v, u, iq[it], exc);
        n.I[i] = 0;
        if (mine) {
            sv[i] = v;
            su[i] = u;
        }
        uint2 h = hh[it];
        if (h.x & 0x80000000u) h.y = (uint32_t)(t - 32);
        h.x = (h.x << 1) | (fired ? 1u : 0u);
        n.hl[i] = h;
        if (fired) {
            n.last_spike[i] = t;
            if (exc) fe |= 1u << it; else fi |= 1u << it;
        }
    }
#pragma unroll
    for (int it = 0; it < kNeuronsPerThread; ++it) {
        if (!(((fe | fi) >> it) & 1u)) continue;
        const uint32_t i = first + it * blockDim.x + threadIdx.x;
        indeg += (unsigned long long)(n.rin_off[i + 1] - n.rin_off[i]);
    }
    // block-wide exclusive prefix of the per-thread counts (exc, inh)
    __shared__ int s_w[2][32];
    __shared__ int s_base[3];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ce = __popc(fe), ci = __popc(fi);
    int ie = ce, ii = ci;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ye = __shfl_up_sync(0xffffffffu, ie, o);
        const int yi = __shfl_up_sync(0xffffffffu, ii, o);
        if (lane >= o) { ie += ye; ii += yi; }
    }
    if (lane == 31) { s_w[0][warp] = ie; s_w[1][warp] = ii; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int se = 0, si = 0;
        for (int k = 0; k < nw; ++k) {
            const int a = s_w[0][k], b = s_w[1][k];
            s_w[0][k] = se; s_w[1][k] = si;
            se += a; si += b;
        }
        s_base[0] = se ? atomicAdd(&n.ctr->step_cnt[par][0], se) : 0;
        s_base[1] = si ? atomicAdd(&n.ctr->step_cnt[par][1], si) : 0;
        s_base[2] = (se + si) ? atomicAdd(&n.ctr->step_cnt[par][2], se + si) : 0;
    }
    __syncthreads();
    if (fe | fi) {
        int pe = s_base[0] + s_w[0][warp] + ie - ce;
        int pi = s_base[1] + s_w[1][warp] + ii - ci;
        int32_t *ring = n.ring_ids + (size_t)(t % (int)n.D) * n.N;
        const unsigned long long rbase = n.ctr->raster_total;
        int pr = s_base[2] + (s_w[0][warp] + ie - ce) + (s_w[1][warp] + ii - ci);
#pragma unroll
        for (int it = 0; it < kNeuronsPerThread; ++it) {
            const uint32_t i = first + it * blockDim.x + threadIdx.x;
            const bool e = (fe >> it) & 1u, q = (fi >> it) & 1u;
            if (!(e || q)) continue;
            const int pos = e ? pe++ : (int)n.N - 1 - (pi++);
            if (!out_of_range(n, pos >= 0 && pos < (int)n.N)) ring[pos] = (int32_t)i;
            const unsigned long long r = rbase + (unsigned long long)(pr++);
            if (r < n.raster_cap) n.raster_gid[r] = (int32_t)i;
        }
    }
    const unsigned long long bdeg = block_sum(indeg);
    if (threadIdx.x == 0) {
        if (bdeg) atomicAdd(&n.ctr->l_exc, bdeg);
        __threadfence();
        s_last = atomicAdd(&n.ctr->done_blocks, 1u) == g.nblk - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    // last block: every other block's counts and writes are complete
    __threadfence();
    DevCounters *c = n.ctr;
    volatile int *sc = c->step_cnt[par];
    const int te = sc[0], ti = sc[1];
    const int total = te + ti;
    const int slot = t % (int)n.D;
    n.ring_cnt[2 * slot] = te;
    n.ring_cnt[2 * slot + 1] = ti;
    c->spikes += (unsigned long long)total;
    const unsigned long long rt = c->raster_total;
    const unsigned long long room = (n.raster_cap > rt) ? n.raster_cap - rt : 0ull;
    const unsigned long long kept = (unsigned long long)total < room ? (unsigned long long)total : room;
    if (kept < (unsigned long long)total) {
        if (c->raster_dropped == 0) c->raster_first_drop_t = t;
        c->raster_dropped += (unsigned long long)total - kept;
    }
    c->raster_total = rt + kept;
    if (n.raster_step_off) n.raster_step_off[t + 1 - n.raster_t0] = (int64_t)(rt + kept);
    c->step_cnt[par ^ 1][0] = 0;
    c->step_cnt[par ^ 1][1] = 0;
    c->step_cnt[par ^ 1][2] = 0;
    c->l_exc_last = c->l_exc - c->l_exc_mark;
    c->l_exc_mark = c->l_exc;
    c->dense_cursor = 0;
    c->staged_cursor = 0;
    c->fold_cursor = 0;
    c->ltp_pending = t;
    c->done_blocks = 0;
    *t_next = t + 1;
}

}  // namespace snn

namespace snn {

// membrane traces: v and u of the probed neurons after the update of step t
__device__ __forceinline__ void probe_body(const DevNet &n, const int *t_now, const Part &g)
{
    const uint32_t k = part_tid(g);
    if (k >= n.probe_n) return;
    const int row = *t_now - n.probe_t0;
    if (row < 0 || (uint32_t)row >= n.probe_cap) return;
    const int32_t gid = n.probe_gid[k];
    const size_t o = (size_t)row * n.probe_n + k;
    n.probe_v[o] = n.vd ? (float)n.vd[gid] : n.v[gid];
    n.probe_u[o] = n.ud ? (float)n.ud[gid] : n.u[gid];
}


// ---------------------------------------------------------------------------
// kernels: one net over the whole grid, or every net of a batch in one
// launch (each block works for the net its BatchLaunch table names, on that
// net's own step, counters and cursors)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_deliver(DevNet n, const int *t_now) { deliver_ring(n, t_now, whole_grid()); }

__global__ void __launch_bounds__(kStagedBlock) k_deliver_cols(DevNet n, const int *t_now)
{
    deliver_staged(n, t_now, whole_grid());
}

__global__ void __launch_bounds__(kOrderedMaxBlock, 5) k_deliver_ordered(DevNet n, const int *t_now)
{
    deliver_ordered(n, t_now, whole_grid());
}

__global__ void __launch_bounds__(1024) k_ltp(DevNet n, const int *t_now, int force)
{
    ltp_body(n, t_now, force, whole_grid());
}

__global__ void __launch_bounds__(1024) k_fold(DevNet n, const int *t_now, int force)
{
    fold_body(n, t_now, force, whole_grid());
}

__global__ void __launch_bounds__(1024) k_deriv(DevNet n, const int *t_now, int force)
{
    deriv_body(n, t_now, force, whole_grid());
}

__global__ void __launch_bounds__(1024) k_neuron_f32(DevNet n, const int *t_now, int *t_next)
{
    neuron_body<float>(n, t_now, t_next, whole_grid());
}

__global__ void __launch_bounds__(1024) k_neuron_f64(DevNet n, const int *t_now, int *t_next)
{
    neuron_body<double>(n, t_now, t_next, whole_grid());
}

__global__ void k_probe(DevNet n, const int *t_now) { probe_body(n, t_now, whole_grid()); }

__global__ void __launch_bounds__(1024) k_deliver_b(BatchLaunch b)
{
    const BatchBlock x = batch_block(b);
    const DevNet n = b.nets[x.net];
    deliver_ring(n, x.t_now, x.part);
}

__global__ void __launch_bounds__(kStagedBlock) k_deliver_cols_b(BatchLaunch b)
{
    const BatchBlock x = batch_block(b);
    const DevNet n = b.nets[x.net];
    deliver_staged(n, x.t_now, x.part);
}

__global__ void __launch_bounds__(kOrderedMaxBlock, 5) k_deliver_ordered_b(BatchLaunch b)
{
    const BatchBlock x = batch_block(b);
    const DevNet n = b.nets[x.net];
    deliver_ordered(n, x.t_now, x.part);
}

__global__ void __launch_bounds__(1024) k_ltp_b(BatchLaunch b)
{
    const BatchBlock x = batch_block(b);
    const DevNet n = b.nets[x.net];
    ltp_body(n, x.t_now, 0, x.part);
}

__global__ void __launch_bounds__(1024) k_fold_b(BatchLaunch b)
{
    const BatchBlock x = batch_block(b);
    const DevNet n = b.nets[x.net];
    fold_body(n, x.t_now, 0, x.part);
}

__global__ void __launch_bounds__(1024) k_deriv_b(BatchLaunch b)
{
    const BatchBlock x = batch_block(b);
    const DevNet n = b.nets[x.net];
    deriv_body(n, x.t_now, 0, x.part);
}

__global__ void __launch_bounds__(1024) k_neuron_f32_b(BatchLaunch b)
{
    const BatchBlock x = batch_block(b);
    const DevNet n = b.nets[x.net];
    neuron_body<float>(n, x.t_now, x.t_next, x.part);
}

__global__ void __launch_bounds__(1024) k_neuron_f64_b(BatchLaunch b)
{
    const BatchBlock x = batch_block(b);
    const DevNet n = b.nets[x.net];
    neuron_body<double>(n, x.t_now, x.t_next, x.part);
}

__global__ void k_probe_b(BatchLaunch b)
{
    const BatchBlock x = batch_block(b);
    const DevNet n = b.nets[x.net];
    probe_body(n, x.t_now, x.part);
}

// ---------------------------------------------------------------------------
// a tile receives the spikes of step t of neurons it does not own (their
// owners' compaction, Sec. 2 "Delivery of spiking messages"): each joins
// ring slot t % D after the tile's own spikes of its kind, and its history
// and last spike record it, so that delivery and potentiation see it as if
// the neuron were the tile's own.  One thread per received spike; positions
// come from the counts and a prefix within the launch (one block).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_inject(DevNet n, int t, const int32_t *gid, uint32_t count)
{
    __shared__ int s_base[2];
    __shared__ uint32_t s_cnt[2];
    const int slot = t % (int)n.D;
    if (threadIdx.x == 0) {
        s_base[0] = n.ring_cnt[2 * slot];
        s_base[1] = n.ring_cnt[2 * slot + 1];
        s_cnt[0] = s_cnt[1] = 0;
    }
    __syncthreads();
    int32_t *ring = n.ring_ids + (size_t)slot * n.N;
    for (uint32_t k0 = 0; k0 < count; k0 += blockDim.x) {
        const uint32_t k = k0 + threadIdx.x;
        if (k < count) {
            const uint32_t g = (uint32_t)gid[k];
            if (!out_of_range(n, g < n.N)) {
                const bool exc = (g % n.npc) < n.ne;
                const uint32_t pos = atomicAdd(&s_cnt[exc ? 0 : 1], 1u);
                const int at = exc ? s_base[0] + (int)pos : (int)n.N - 1 - (s_base[1] + (int)pos);
                if (!out_of_range(n, at >= 0 && at < (int)n.N)) ring[at] = (int32_t)g;
                n.hl[g].x |= 1u;                 // bit 0: fired at t (the step's update has run)
                n.last_spike[g] = t;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        n.ring_cnt[2 * slot] = s_base[0] + (int)s_cnt[0];
        n.ring_cnt[2 * slot + 1] = s_base[1] + (int)s_cnt[1];
    }
}

}  // namespace snn
