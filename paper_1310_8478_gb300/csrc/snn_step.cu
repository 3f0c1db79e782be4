// snn_step.cu -- the per-millisecond step of the DPSNN-STDP engine on GB300.
//
// Paper, Sec. 2 "Mixed time-driven and event driven simulation": synapses are
// event driven (only synapses of neurons that fired are touched), neurons are
// time driven (every neuron is updated every step).  One step t runs
//   k_deliver  S1: spikes emitted at t - d reach their delay-d synapses
//              (steps 2.3-2.5), depression of excitatory synapses against the
//              target's latest spike (2.6); thalamic and external drive.
//   k_neuron   S2: Izhikevich update of every neuron (2.7); S3: the neurons
//              that fired are compacted into the delay ring and the raster.
//   k_ltp      S4: potentiation of the incoming excitatory synapses of every
//              neuron that fired at t (2.1), through the reverse index.
//   k_deriv    S5: every deriv_period steps, w += bias + sd, sd *= decay.
// All synaptic arithmetic is int32 Q16, so the order of the atomic additions
// does not change any result; the neuron update is IEEE fp32 with one
// rounding per operation (explicit _rn intrinsics, no contraction).
#include "snn_internal.cuh"

namespace snn {

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

// ---------------------------------------------------------------------------
// S1: delivery + LTD.  Work items are (spike, delay) pairs: every excitatory
// spike of step t - d for d = 1..D and every inhibitory spike of step t - 1
// (inhibitory synapses all have delay 1).  One warp walks an item's
// delay-bucketed segment with coalesced loads; lanes add the weight into the
// target's Q16 input with a fire-and-forget L2 reduction and, for plastic
// synapses, subtract the LTD amount at lag t - last_spike[target].
// ---------------------------------------------------------------------------
__global__ void k_deliver(DevNet n, const int *t_now)
{
    __shared__ int32_t s_lut[kLut];
    __shared__ int s_start[34];       // item prefix over the lists: 0..D-1 exc(d = 1..D), D inh(d = 1)
    __shared__ const int32_t *s_list[33];
    __shared__ int s_inh[33];
    const int t = *t_now;
    const bool stdp = !(n.flags & SNN_STDP_OFF);
    for (int i = threadIdx.x; i < kLut; i += blockDim.x) s_lut[i] = n.lut_m[i];
    if (threadIdx.x == 0) {
        int acc = 0;
        const int nl = (int)n.D + 1;
        for (int l = 0; l < nl; ++l) {
            const int d = (l < (int)n.D) ? l + 1 : 1;
            const bool inh = (l == (int)n.D);
            int cnt = 0;
            const int32_t *list = nullptr;
            if (!(n.flags & SNN_DELIVERY_OFF) && t - d >= 0) {
                const int slot = (t - d) % (int)n.D;
                cnt = n.ring_cnt[2 * slot + (inh ? 1 : 0)];
                list = n.ring_ids + (size_t)slot * n.N;
            }
            s_start[l] = acc;
            s_list[l] = list;
            s_inh[l] = inh;
            acc += cnt;
        }
        s_start[nl] = acc;
    }
    __syncthreads();

    // thalamic drive: thal_per_col events per column (Philox keyed by (t, col))
    // and the external events of step t
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t gthreads = gridDim.x * blockDim.x;
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

    const int nl = (int)n.D + 1;
    const int total = s_start[nl];
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gthreads >> 5;
    unsigned long long ev_all = 0, ev_exc = 0;
    for (uint32_t item = gtid >> 5; item < (uint32_t)total; item += warps) {
        int l = 0;
        while (s_start[l + 1] <= (int)item) ++l;
        const int idx = (int)item - s_start[l];
        const bool inh = s_inh[l];
        const int d = inh ? 1 : l + 1;
        const uint32_t p = (uint32_t)(inh ? s_list[l][n.N - 1 - idx] : s_list[l][idx]);
        const uint16_t *off = n.doff + (size_t)p * kDoffStride;
        const int64_t base = row_base(n, p);
        const int64_t lo = base + off[d - 1], hi = base + off[d];
        ev_all += (unsigned long long)(hi - lo);
        if (!inh) ev_exc += (unsigned long long)(hi - lo);
        if (!inh && stdp) {
            for (int64_t k = lo + lane; k < hi; k += 32) {
                const int32_t tg = n.tgt[k];
                red_add(&n.I[tg], n.w[k]);
                const int lag = t - n.last_spike[tg];          // >= 1
                if (lag < kLut) {
                    const int32_t a = s_lut[lag];
                    if (a) n.sd[k] -= a;
                }
            }
        } else {
            for (int64_t k = lo + lane; k < hi; k += 32) red_add(&n.I[n.tgt[k]], n.w[k]);
        }
    }
    // lane 0 of each warp counted the items; sum over the block
    if (lane != 0) ev_all = ev_exc = 0;
    const unsigned long long ba = block_sum(ev_all);
    const unsigned long long be = block_sum(ev_exc);
    if (threadIdx.x == 0 && ba) {
        atomicAdd(&n.ctr->e_all, ba);
        atomicAdd(&n.ctr->e_exc, be);
    }
}

// ---------------------------------------------------------------------------
// S2 + S3: Izhikevich update (paper Sec. 2 "Spiking neuron model"; v in two
// 0.5 ms Euler substeps, u in one 1 ms step, Sec. 3) of kNeuronsPerThread
// neurons per thread, then one block-wide compaction of the neurons that
// fired into ring slot t % D (exc ids from the front, inh ids from the back)
// and into the raster.
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

__global__ void k_neuron(DevNet n, const int *t_now)
{
    const int t = *t_now;
    const int par = t & 1;
    const uint32_t tile = blockDim.x * kNeuronsPerThread;
    const uint32_t first = blockIdx.x * tile;
    uint32_t fe = 0, fi = 0;          // bit it: neuron first + it * blockDim + tid fired
#pragma unroll
    for (int it = 0; it < kNeuronsPerThread; ++it) {
        const uint32_t i = first + it * blockDim.x + threadIdx.x;
        if (i >= n.N) break;
        const bool exc = (i % n.npc) < n.ne;
        const int32_t iq = n.I[i];
        n.I[i] = 0;
        float v = n.v[i], u = n.u[i];
        const bool fired = izhikevich_step(v, u, iq, exc);
        n.v[i] = v;
        n.u[i] = u;
        uint32_t h = n.hist[i];
        if (h & 0x80000000u) n.last_old[i] = t - 32;
        h = (h << 1) | (fired ? 1u : 0u);
        n.hist[i] = h;
        if (fired) {
            n.last_spike[i] = t;
            if (exc) fe |= 1u << it; else fi |= 1u << it;
        }
    }
    // block-wide exclusive prefix of the per-thread counts (exc, inh)
    __shared__ int s_w[2][32];
    __shared__ int s_base[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int ce = __popc(fe), ci = __popc(fi);
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
    if (!(fe | fi)) return;
    int pe = s_base[0] + s_w[0][warp] + ie - ce;
    int pi = s_base[1] + s_w[1][warp] + ii - ci;
    // raster index: spikes kept so far + this block's place among this step's
    // spikes (exc of the block first, then inh)
    const int blk_e = s_w[0][nw - 1] + 0;  // not used when nw == 1 (see below)
    (void)blk_e;
    int32_t *ring = n.ring_ids + (size_t)(t % (int)n.D) * n.N;
    const unsigned long long rbase = n.ctr->raster_total;
    int pr = s_base[2] + (s_w[0][warp] + ie - ce) + (s_w[1][warp] + ii - ci);
#pragma unroll
    for (int it = 0; it < kNeuronsPerThread; ++it) {
        const uint32_t i = first + it * blockDim.x + threadIdx.x;
        const bool e = (fe >> it) & 1u, q = (fi >> it) & 1u;
        if (!(e || q)) continue;
        if (e) ring[pe++] = (int32_t)i;
        else ring[n.N - 1 - (pi++)] = (int32_t)i;
        const unsigned long long r = rbase + (unsigned long long)(pr++);
        if (r < n.raster_cap) n.raster_gid[r] = (int32_t)i;
    }
}

// ---------------------------------------------------------------------------
// S4: LTP.  Warp per neuron that fired at t; lanes walk its incoming
// excitatory synapses.  The nearest arrival of the source with
// t_pre + d <= t is the lowest set bit k >= d of the source's 32-step history
// (lag k - d), else its latest older spike last_old (lag t - last_old - d).
// Block 0 also closes the step: ring counts of slot t % D, counters, raster
// step offset, the next step's time stamp.
// ---------------------------------------------------------------------------
__global__ void k_ltp(DevNet n, const int *t_now, int *t_next)
{
    __shared__ int32_t s_lut[kLut];
    const int t = *t_now;
    const int par = t & 1;
    const bool stdp = !(n.flags & SNN_STDP_OFF);
    for (int i = threadIdx.x; i < kLut; i += blockDim.x) s_lut[i] = n.lut_p[i];
    __syncthreads();
    const int ce = n.ctr->step_cnt[par][0], ci = n.ctr->step_cnt[par][1];
    const int total = ce + ci;
    const int32_t *ring = n.ring_ids + (size_t)(t % (int)n.D) * n.N;
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long visits = 0;
    for (uint32_t item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < (uint32_t)total;
         item += warps) {
        const int32_t post = (int)item < ce ? ring[item] : ring[n.N - 1 - ((int)item - ce)];
        const int64_t lo = n.rin_off[post], hi = n.rin_off[post + 1];
        visits += (unsigned long long)(hi - lo);
        if (!stdp) continue;
        for (int64_t e = lo + lane; e < hi; e += 32) {
            const uint64_t r = n.rin[e];
            const uint32_t pre = (uint32_t)r;
            const uint32_t ord = (uint32_t)(r >> 32) & 0xffffu;
            const uint32_t d = (uint32_t)(r >> 48);
            const uint32_t recent = n.hist[pre] & (0xffffffffu << d);
            const int lag = recent ? (__ffs(recent) - 1 - (int)d) : (t - n.last_old[pre] - (int)d);
            if (lag < kLut) {
                const int32_t a = s_lut[lag];
                if (a) n.sd[row_base(n, pre) + ord] += a;
            }
        }
    }
    if (lane != 0) visits = 0;
    const unsigned long long bv = block_sum(visits);
    if (threadIdx.x == 0 && bv) atomicAdd(&n.ctr->l_exc, bv);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        DevCounters *c = n.ctr;
        const int slot = t % (int)n.D;
        n.ring_cnt[2 * slot] = ce;
        n.ring_cnt[2 * slot + 1] = ci;
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
        *t_next = t + 1;
    }
}

// ---------------------------------------------------------------------------
// S5: long-term plasticity over the excitatory rows of column blockIdx.y
// (rows c*npc .. c*npc+ne-1 are contiguous): w = clamp(w + bias + sd, 0,
// wmax), sd = (sd * decay + 2^15) >> 16, int64 intermediates.
// ---------------------------------------------------------------------------
__global__ void k_deriv(DevNet n, uint32_t chunk)
{
    (void)chunk;
    const uint32_t col = blockIdx.y;
    const int64_t lo = row_base(n, col * n.npc);
    const int64_t hi = n.uniform_m ? (int64_t)(col * n.npc + n.ne) * n.uniform_m
                                   : n.row_off[col * n.npc + n.ne];
    for (int64_t k = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < hi;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = n.sd[k];
        long long nw = (long long)n.w[k] + n.deriv_bias + s;
        nw = nw < 0 ? 0 : (nw > n.wmax ? n.wmax : nw);
        n.w[k] = (int32_t)nw;
        n.sd[k] = (int32_t)(((long long)s * n.deriv_decay + 32768) >> 16);
    }
}

}  // namespace snn
