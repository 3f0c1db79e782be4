// snn_build.cu -- device-side network construction for the DPSNN-STDP engine.
//
// Sec. 2 of the paper ("Initial construction of the connectivity
// infrastructure", "Distributed generation of reproducible connections"):
// each neuron's forward synapses are generated from global ids only, kept
// in one bucket per axonal delay value, and every target learns its
// incoming synapses.  On one GPU the MPI handshake becomes a device-side
// in-degree count, a prefix sum and a scatter into the reverse index.
#include "snn_internal.cuh"

namespace snn {

// ---------------------------------------------------------------------------
// One warp per source row: draw the row's (target, delay) pairs, count them
// per delay, write the delay offsets, then place every synapse at
// row_base + offset(delay) + rank, stable in the ordinal j.
// ---------------------------------------------------------------------------
__global__ void k_gen_rows(GenParams g, uint32_t n_rows, uint16_t *doff, int32_t *tgt, uint16_t *tgt16,
                           int32_t *w, int32_t *sd)
{
    constexpr int kWarps = 8;        // launched with 256 threads
    __shared__ int s_cnt[kWarps][32];
    __shared__ int s_cur[kWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    for (uint32_t p = blockIdx.x * kWarps + warp; p < n_rows; p += gridDim.x * kWarps) {
        const int64_t base = (int64_t)p * g.m_store;
        const bool exc = (p % g.npc) < g.ne;
        for (uint32_t j = g.m + lane; j < g.m_store; j += 32) {   // padding tail
            if (tgt16) tgt16[base + j] = 0;
            else tgt[base + j] = 0;
            w[base + j] = 0;
            sd[base + j] = 0;
        }
        s_cnt[warp][lane] = 0;
        __syncwarp();
        for (uint32_t j = lane; j < g.m; j += 32) {
            uint32_t t, d, sl;
            gen_synapse(g, p, j, t, d, sl);
            atomicAdd(&s_cnt[warp][d], 1);
        }
        __syncwarp();
        // inclusive prefix over delays: doff[d] = synapses of delay <= d
        int c = s_cnt[warp][lane];
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if ((uint32_t)lane <= g.D) doff[(size_t)p * kDoffStride + lane] = (uint16_t)incl;
        s_cur[warp][lane] = incl - c;
        __syncwarp();
        for (uint32_t j0 = 0; j0 < g.m; j0 += 32) {
            const uint32_t j = j0 + lane;
            const bool active = j < g.m;
            uint32_t t = 0, d = 0, sl = 0;
            if (active) gen_synapse(g, p, j, t, d, sl);
            const unsigned peers = __match_any_sync(0xffffffffu, d);   // d = 0: inactive lanes
            const int rank = __popc(peers & lt);
            const int start = s_cur[warp][d];
            __syncwarp();
            if (active && rank == __popc(peers) - 1) s_cur[warp][d] = start + __popc(peers);
            if (active) {
                const int64_t pos = base + start + rank;
                if (tgt16) tgt16[pos] = (uint16_t)(sl * g.npc + t % g.npc);
                else tgt[pos] = (int32_t)t;
                w[pos] = exc ? g.w_exc0 : g.w_inh0;
                sd[pos] = 0;
            }
            __syncwarp();
        }
    }
}

// Warp per source row: count incoming synapses per target, split by the
// source's kind (excitatory synapses are the plastic ones).
__global__ void k_count_indeg(DevNet n, int32_t *indeg_exc, int32_t *indeg_inh)
{
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n.N; p += warps) {
        const bool exc = (p % n.npc) < n.ne;
        int32_t *deg = exc ? indeg_exc : indeg_inh;
        const uint32_t col = p / n.npc;
        const int64_t lo = row_base(n, p), hi = lo + row_len(n, p);
        for (int64_t k = lo + lane; k < hi; k += 32) atomicAdd(&deg[target_gid(n, col, k)], 1);
    }
}

// ---------------------------------------------------------------------------
// exclusive prefix sum int32[n] -> int64[n + 1] in three launches
// (1024 inputs per block of 256 threads)
// ---------------------------------------------------------------------------
constexpr int kScanBlock = 256, kScanItems = 4, kScanChunk = kScanBlock * kScanItems;

__device__ __forceinline__ long long block_exclusive_scan(long long x, long long *total)
{
    __shared__ long long s_warp[kScanBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        long long s = (lane < kScanBlock / 32) ? s_warp[lane] : 0;
        long long si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        if (lane < kScanBlock / 32) s_warp[lane] = si - s;
        if (lane == kScanBlock / 32 - 1) *total = si;
    }
    __syncthreads();
    const long long r = s_warp[warp] + incl - x;
    __syncthreads();
    return r;
}

__global__ void k_scan_sums(const int32_t *in, uint32_t n, long long *block_sums)
{
    const uint64_t base = (uint64_t)blockIdx.x * kScanChunk;
    long long s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t k = base + (uint64_t)i * kScanBlock + threadIdx.x;
        if (k < n) s += in[k];
    }
    __shared__ long long s_tot;
    (void)block_exclusive_scan(s, &s_tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = s_tot;
}

// single block: block_sums[i] <- sum of block_sums[0..i) ; block_sums[n] <- total
__global__ void k_scan_carry(long long *block_sums, uint32_t n_blocks)
{
    __shared__ long long s_tot;
    long long carry = 0;
    for (uint32_t b0 = 0; b0 < n_blocks; b0 += kScanBlock) {
        const uint32_t k = b0 + threadIdx.x;
        const long long x = (k < n_blocks) ? block_sums[k] : 0;
        const long long e = block_exclusive_scan(x, &s_tot);
        if (k < n_blocks) block_sums[k] = carry + e;
        carry += s_tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) block_sums[n_blocks] = carry;
}

__global__ void k_scan_write(const int32_t *in, uint32_t n, const long long *block_sums, int64_t *out)
{
    const uint64_t base = (uint64_t)blockIdx.x * kScanChunk + (uint64_t)threadIdx.x * kScanItems;
    long long v[kScanItems];
    long long s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t k = base + i;
        v[i] = (k < n) ? in[k] : 0;
        s += v[i];
    }
    __shared__ long long s_tot;
    long long e = block_exclusive_scan(s, &s_tot) + block_sums[blockIdx.x];
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t k = base + i;
        if (k < n) out[k] = e;
        e += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = block_sums[gridDim.x];
}

// Warp per excitatory source row: append every synapse to its target's
// incoming list (order inside a list is irrelevant: LTP only adds integers),
// as a 4-byte entry (rin32) or an 8-byte one (rin).
__global__ void k_fill_reverse(DevNet n, int32_t *cursor, uint64_t *rin, uint32_t *rin32)
{
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n.N; p += warps) {
        if ((p % n.npc) >= n.ne) continue;
        const int64_t base = n.row_off[p];
        const uint32_t col = p / n.npc;
        const uint16_t *off = n.doff + (size_t)p * kDoffStride;
        for (uint32_t d = 1; d <= n.D; ++d) {
            const uint32_t lo = off[d - 1], hi = off[d];
            for (uint32_t k = lo + lane; k < hi; k += 32) {
                const uint32_t t = target_gid(n, col, base + k);
                const int slot = atomicAdd(&cursor[t], 1);
                if (rin32) {
                    const uint32_t sl = __umulhi((uint32_t)n.tgt16[base + k], n.npc_recip);
                    rin32[n.rin_off[t] + slot] = rin32_entry(inverse_slot(sl), n.npc, p % n.npc, d, k);
                } else {
                    rin[n.rin_off[t] + slot] = (uint64_t)p | ((uint64_t)k << 32) | ((uint64_t)d << 48);
                }
            }
        }
    }
}

__global__ void k_max2(const int32_t *a, const int32_t *b, uint32_t n, int32_t *out2)
{
    int ma = 0, mb = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        ma = max(ma, a[i]);
        mb = max(mb, b[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ma = max(ma, __shfl_xor_sync(0xffffffffu, ma, o));
        mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out2[0], ma);
        atomicMax(&out2[1], mb);
    }
}

// initial weights of a generated net (by source kind) and zero derivatives
__global__ void k_reset_weights(DevNet n, int32_t w_exc0, int32_t w_inh0)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n.S; k += stride) {
        const uint32_t p = (uint32_t)(k / n.uniform_m);
        n.w[k] = ((p % n.npc) < n.ne) ? w_exc0 : w_inh0;
        n.sd[k] = 0;
    }
}

// initial state: v = -65 mV, u = b v (b = 0.2 for both kinds), no history
__global__ void k_init_state(DevNet n)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n.N; i += gridDim.x * blockDim.x) {
        const float v0 = -65.0f;
        n.v[i] = v0;
        n.u[i] = __fmul_rn(0.2f, v0);
        if (n.vd) {
            n.vd[i] = -65.0;
            n.ud[i] = __dmul_rn(0.2, -65.0);
        }
        n.I[i] = 0;
        n.hl[i] = make_uint2(0u, (uint32_t)kNever);
        n.last_spike[i] = kNever;
    }
}

// Canonical-order read-back: thread per source row recovers the ordinal of
// every stored synapse from the canonical delays (regenerated, or kept for
// explicit nets) and the stable delay order.
__global__ void k_read_rows(DevNet n, GenParams g, const uint8_t *canon_delay, uint32_t first,
                            uint32_t count, int64_t out_base, int32_t *o_tgt, uint8_t *o_delay,
                            int32_t *o_w, int32_t *o_sd)
{
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < count; r += gridDim.x * blockDim.x) {
        const uint32_t p = first + r;
        const int64_t lo = row_base(n, p), len = row_len(n, p), cb = canon_base(n, p);
        const uint16_t *off = n.doff + (size_t)p * kDoffStride;
        uint16_t used[kDoffStride];
        for (int d = 0; d < kDoffStride; ++d) used[d] = 0;
        for (int64_t j = 0; j < len; ++j) {
            uint32_t d;
            if (canon_delay) {
                d = canon_delay[cb + j];
            } else {
                uint32_t t, sl;
                gen_synapse(g, p, (uint32_t)j, t, d, sl);
            }
            const int64_t pos = lo + off[d - 1] + used[d];
            used[d]++;
            const int64_t o = cb - out_base + j;
            if (o_tgt) o_tgt[o] = (int32_t)target_gid(n, p / n.npc, pos);
            if (o_delay) o_delay[o] = (uint8_t)d;
            if (o_w) o_w[o] = n.w[pos];
            if (o_sd) o_sd[o] = n.sd[pos];
        }
    }
}

}  // namespace snn
