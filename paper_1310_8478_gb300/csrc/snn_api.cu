// snn_api.cu -- host engine and C ABI of the GB300 DPSNN-STDP step (include/snn.h).
//
// Owns the device layout of one network, the construction sequence (device
// generation, in-degree count, prefix sum, reverse-index scatter), the step
// sequence (eager launches or CUDA-graph replays of graph_steps steps), the
// readers and the checkpoint format.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "snn_internal.cuh"

using namespace snn;

namespace {

thread_local std::string g_last_error = "";

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

void *(*g_alloc)(size_t, void *, void *) = nullptr;
void (*g_release)(void *, void *) = nullptr;
void *g_alloc_ctx = nullptr;

#define SNN_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            set_error("%s failed: %s", #call, cudaGetErrorString(e_));                   \
            return SNN_ECUDA;                                                            \
        }                                                                                \
    } while (0)

#define SNN_TRY(expr)                                                                    \
    do {                                                                                 \
        int r_ = (expr);                                                                 \
        if (r_ != SNN_OK) return r_;                                                     \
    } while (0)

constexpr uint32_t kStateMagic = 0x534e4e31u;  // "SNN1"

// Device staging of snn_read_synapses_noalloc: target, weight and sd words,
// then the delay bytes, for SNN_NOALLOC_MAX_SYNAPSES synapses.  Host code
// must not use this name as an address: it looks the address up per device.
constexpr size_t kNoAllocWords = (size_t)SNN_NOALLOC_MAX_SYNAPSES * 3 + SNN_NOALLOC_MAX_SYNAPSES / 4;
static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
int32_t *g_noalloc_ptr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mutex;

// device address of the staging array on the current device, looked up
// again at every net's set-up (so that the module holding the array is
// loaded before the net's budget is spent, and a device reset between nets
// leaves no stale address) and kept per device
int noalloc_lookup(int device, int32_t **out)
{
    if (device < 0 || device >= kMaxDevices) { set_error("device ordinal too large"); return SNN_EINVAL; }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaGetSymbolAddress of the staging array failed: %s", cudaGetErrorString(e));
        return SNN_ECUDA;
    }
    g_noalloc_ptr[device] = (int32_t *)ptr;
    *out = (int32_t *)ptr;
    return SNN_OK;
}

__global__ void k_fill_row_off(int64_t *row_off, uint32_t n, uint32_t m)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
        row_off[i] = (int64_t)i * m;
}

}  // namespace

struct WeightRange {
    int32_t exc_min, exc_max, inh_min, inh_max;   // initial weights by source kind
};

struct snn_net {
    snn_config cfg{};
    WeightRange wrange{};
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // the potentiation owed by the last step runs on a side stream beside
    // the delivery of the next one (they touch disjoint data), forked from
    // and joined back into `stream` in every step that closes no period
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool explicit_net = false;
    GenParams gen{};
    DevNet dn{};
    uint32_t N = 0;
    int64_t S = 0;                  // synapses
    int64_t S_store = 0;            // stored slots (generated rows padded to the stride)
    int64_t n_rin = 0;
    size_t budget = 0;
    size_t bytes_held = 0;
    struct Block { void *p; size_t bytes; };
    std::vector<Block> blocks;
    void *(*alloc)(size_t, void *, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;
    // device arrays (also reachable through dn)
    int64_t *row_off = nullptr;
    uint16_t *doff = nullptr;
    int32_t *tgt = nullptr, *w = nullptr, *sd = nullptr;
    uint8_t *canon_delay = nullptr;
    int64_t *rin_off = nullptr;
    uint64_t *rin = nullptr;
    uint32_t *rin32 = nullptr;
    DevCounters *ctr = nullptr;
    int32_t *lut = nullptr;
    int64_t raster_steps_cap = 0;   // entries of dn.raster_step_off
    uint16_t *tgt16 = nullptr;
    int32_t *nbr = nullptr;
    bool ltp_owed = false;          // the last step's LTP has not been applied yet
    int32_t *noalloc_base = nullptr; // device address of the no-allocation staging array
    int32_t *inject_buf = nullptr;  // tiles: device copy of the spikes received for a step
    bool dense_ok = false;          // the dense pass can run on this net
    int dense_grid = 0;             // blocks of the dense pass (at most one wave of resident blocks)
    int staged_grid = 0;            // blocks of the column-staged delivery (likewise)
    int ordered_grid = 0;           // blocks of the column-ordered delivery (likewise)
    uint64_t version = 0;           // bumped whenever captured launches go stale
    // stimulus
    size_t stim_cap = 0;
    int64_t stim_off_cap = 0;
    // pinned host memory: the counters read after a run ([1]) and before one
    // ([0]), and the staging of a stimulus upload
    DevCounters *host_ctr = nullptr;
    char *stim_stage = nullptr;
    size_t stim_stage_cap = 0;
    // host state
    int32_t t = 0;
    snn_launch launch{};
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    uint32_t graph_len = 0;
    bool graphs_dirty = true;
    bool profile = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_kind;
    size_t ev_used = 0;
    double prof_ms[kKinds] = {0};
    int64_t prof_n[kKinds] = {0};
    int64_t prof_kernels = 0;       // kernels launched by the profiled steps
};

// kinds of step kernel a batch launches once per step for all of its nets
enum BatchKind { kBLtp, kBFold, kBDeriv, kBOrdered, kBRing, kBStaged, kBDense, kBNeuron32, kBNeuron64, kBProbe,
                 kBKinds };

struct snn_batch {
    std::vector<snn_net *> nets;
    cudaStream_t main = nullptr;
    std::vector<cudaStream_t> branch;    // single eager steps: one stream per net
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    uint32_t L = 0;
    cudaGraphExec_t graph = nullptr;
    std::vector<uint64_t> versions;      // the nets' versions when the graph was captured
    std::vector<int> parity;             // the nets' step parity when the graph was captured
    snn_launch launch{};                 // block sizes and resident blocks of the batched kernels
    int sm_count = 0;
    int device = 0;
    // device tables of the batched launches (DevNet copies, parities, and per
    // kind the first block of every net and the net of every block)
    void *tables = nullptr;
    size_t tables_bytes = 0;
    struct Kind {
        BatchLaunch bl{};
        uint32_t grid = 0, block = 0;
        size_t smem = 0;
    } kind[kBKinds];
};

namespace {

int dalloc(snn_net *net, size_t bytes, void **out)
{
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    if (net->budget && net->bytes_held + bytes > net->budget) {
        set_error("device budget exceeded: %zu + %zu > %zu bytes", net->bytes_held, bytes, net->budget);
        return SNN_ENOMEM;
    }
    void *p = nullptr;
    if (net->alloc) {
        p = net->alloc(bytes, (void *)net->stream, net->alloc_ctx);
        if (!p) {
            set_error("allocator hook failed for %zu bytes", bytes);
            return SNN_ENOMEM;
        }
        if ((uintptr_t)p & 255u) {
            if (net->release) net->release(p, net->alloc_ctx);
            set_error("allocator hook returned a block that is not 256-byte aligned");
            return SNN_ENOMEM;
        }
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
            return SNN_ENOMEM;
        }
    }
    net->blocks.push_back({p, bytes});
    net->bytes_held += bytes;
    *out = p;
    return SNN_OK;
}

void dfree(snn_net *net, void *p)
{
    if (!p) return;
    for (size_t i = 0; i < net->blocks.size(); ++i) {
        if (net->blocks[i].p == p) {
            if (net->release) net->release(p, net->alloc_ctx);
            else cudaFree(p);
            net->bytes_held -= net->blocks[i].bytes;
            net->blocks.erase(net->blocks.begin() + (long)i);
            return;
        }
    }
}

template <typename T>
int dalloc_t(snn_net *net, size_t count, T **out)
{
    void *p = nullptr;
    int r = dalloc(net, count * sizeof(T), &p);
    *out = (T *)p;
    return r;
}

// every change of what the kernels see (DevNet, launch shape) goes through
// here: captured graphs of the net, and of batches holding it, are stale
void drop_graphs(snn_net *net)
{
    for (int i = 0; i < 2; ++i) {
        if (net->graph[i]) cudaGraphExecDestroy(net->graph[i]);
        net->graph[i] = nullptr;
    }
    net->graphs_dirty = true;
    net->version++;
}

int check_config(const snn_config *c)
{
    if (!c) { set_error("cfg is NULL"); return SNN_EINVAL; }
    if (c->grid_x == 0 || c->grid_y == 0) { set_error("grid must be at least 1x1"); return SNN_EINVAL; }
    if (c->neurons_per_col < 2 || c->exc_per_col == 0 || c->exc_per_col > c->neurons_per_col) {
        set_error("need neurons_per_col >= 2 and 1 <= exc_per_col <= neurons_per_col");
        return SNN_EINVAL;
    }
    const uint64_t n = (uint64_t)c->grid_x * c->grid_y * c->neurons_per_col;
    if (n > 0x7fffffffull) { set_error("too many neurons (%llu)", (unsigned long long)n); return SNN_EINVAL; }
    if ((uint64_t)c->grid_x * c->grid_y > 65535u) { set_error("at most 65535 columns"); return SNN_EINVAL; }
    if (c->fanout == 0 || c->fanout > 65535u) { set_error("fanout must be 1..65535"); return SNN_EINVAL; }
    if (c->pct_ring[0] + c->pct_ring[1] + c->pct_ring[2] + c->pct_ring[3] != 100) {
        set_error("pct_ring must sum to 100");
        return SNN_EINVAL;
    }
    if (c->max_delay_ms < 1 || c->max_delay_ms > 31) { set_error("max_delay_ms must be 1..31"); return SNN_EINVAL; }
    if (c->wmax_q16 < 0) { set_error("wmax must be >= 0"); return SNN_EINVAL; }
    if (!(c->a_plus_mv >= 0) || !(c->a_minus_mv >= 0) || !(c->tau_plus_ms > 0) || !(c->tau_minus_ms > 0)) {
        set_error("STDP amplitudes must be >= 0 and time constants > 0");
        return SNN_EINVAL;
    }
    if (c->reserved != 0) { set_error("reserved field must be 0"); return SNN_EINVAL; }
    if (c->flags & ~(SNN_STDP_OFF | SNN_DELIVERY_OFF | SNN_FP64)) { set_error("unknown flags"); return SNN_EINVAL; }
    if (c->deriv_period_ms > 0x3fffffffu) { set_error("deriv_period_ms too large"); return SNN_EINVAL; }
    // the drive enumerates the events of a step with 32-bit indices
    if ((uint64_t)c->grid_x * c->grid_y * c->thal_per_col_per_ms > 0x7fffffffull) {
        set_error("more than 2^31 - 1 thalamic events per ms");
        return SNN_EINVAL;
    }
    return SNN_OK;
}

// STDP amounts of the pair rule (Sec. 2 "Synaptic update" equation), rounded
// to Q16; the table must cover every non-zero amount.
int build_luts(const snn_config *c, std::vector<int32_t> &lut)
{
    lut.assign(2 * kLut, 0);
    const double amp[2] = {c->a_plus_mv, c->a_minus_mv};
    const double tau[2] = {c->tau_plus_ms, c->tau_minus_ms};
    for (int s = 0; s < 2; ++s) {
        for (int k = 0; k < kLut; ++k) {
            const double x = amp[s] * std::exp(-(double)k / tau[s]) * 65536.0;
            const long long q = std::llround(x);
            if (k == kLut - 1) {
                // lags of 255 and more all read the last entry: it must be 0
                if (q != 0) {
                    set_error("STDP window longer than %d ms (amount at lag %d is %lld)", kLut - 1, k, q);
                    return SNN_EINVAL;
                }
            } else {
                if (q > 0x3fffffff) { set_error("STDP amplitude too large"); return SNN_EINVAL; }
                lut[s * kLut + k] = (int32_t)q;
            }
        }
    }
    return SNN_OK;
}

int grid_for(const snn_net *net, uint32_t per_sm)
{
    return std::max(1, net->sm_count) * (int)std::max(1u, per_sm);
}

// grid of a grid-stride kernel over `units` work units, `per_block` units per
// block at most once, capped at blocks_per_sm resident waves
int sized_grid(const snn_net *net, uint32_t blocks_per_sm, int64_t units, int64_t per_block)
{
    const int64_t want = (units + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)grid_for(net, blocks_per_sm)));
}

// whether the reverse index takes 4-byte entries: compact targets and rows of
// at most kRin32MaxRow stored slots
bool rin32_ok(const snn_config *c, bool explicit_net)
{
    const uint32_t m_store = (c->fanout + 7u) & ~7u;
    return !explicit_net && c->neurons_per_col >= kMinCompactNpc && c->neurons_per_col <= kMaxCompactNpc &&
           m_store <= kRin32MaxRow;
}

bool rin32_ok(const snn_net *net)
{
    return net->tgt16 != nullptr && net->dn.uniform_m != 0 && net->dn.uniform_m <= kRin32MaxRow &&
           rin32_ok(&net->cfg, net->explicit_net);
}

// footprint of everything but the raster (bytes)
size_t footprint(const snn_config *c, uint32_t N, int64_t S, int64_t n_rin, bool explicit_net)
{
    const size_t D = c->max_delay_ms;
    size_t b = 0;
    b += (size_t)S * ((!explicit_net && c->neurons_per_col >= kMinCompactNpc && c->neurons_per_col <= kMaxCompactNpc)
                          ? 10 : 12);  // tgt, w, sd
    b += (size_t)c->grid_x * c->grid_y * kSlotStride * 4;                                  // neighbour table
    b += (size_t)N * kDoffStride * 2;             // delay offsets
    b += ((size_t)N + 1) * 8 * 2;                 // row_off, rin_off
    b += (size_t)n_rin * (rin32_ok(c, explicit_net) ? 8 : 12);   // reverse index + its LTP accumulator
    b += (size_t)N * 24;                          // v u I (hist, last_old) last_spike
    if (c->flags & SNN_FP64) b += (size_t)N * 16; // v u in double
    b += D * N * 4 + D * 8;                       // ring
    b += (size_t)N * 12 + ((size_t)N / 1024 + 2) * 8;  // build scratch
    if (explicit_net) b += (size_t)S;             // canonical delays
    b += 64 * 1024;
    return b;
}

uint32_t dense_threshold(uint32_t n_neurons, uint32_t permille)
{
    if (permille > 1000) return 0xffffffffu;
    const uint64_t v = ((uint64_t)n_neurons * permille + 999) / 1000;
    return (uint32_t)std::max<uint64_t>(1, v);
}

int alloc_common(snn_net *net)
{
    const uint32_t N = net->N;
    const uint32_t D = net->cfg.max_delay_ms;
    DevNet &dn = net->dn;
    const bool compact = !net->explicit_net && net->cfg.neurons_per_col >= kMinCompactNpc &&
                         net->cfg.neurons_per_col <= kMaxCompactNpc;
    if (compact) SNN_TRY(dalloc_t(net, (size_t)net->S_store, &net->tgt16));
    else SNN_TRY(dalloc_t(net, (size_t)net->S_store, &net->tgt));
    const uint32_t C = net->cfg.grid_x * net->cfg.grid_y;
    SNN_TRY(dalloc_t(net, (size_t)C * kSlotStride, &net->nbr));
    {
        std::vector<int32_t> nb((size_t)C * kSlotStride);
        for (uint32_t c = 0; c < C; ++c)
            for (uint32_t sl = 0; sl < (uint32_t)kSlotStride; ++sl)
                nb[(size_t)c * kSlotStride + sl] =
                    (int32_t)(sl < (uint32_t)kSlots ? slot_column(c, sl, net->cfg.grid_x, net->cfg.grid_y) : c);
        SNN_CUDA(cudaMemcpy(net->nbr, nb.data(), nb.size() * 4, cudaMemcpyHostToDevice));
    }
    SNN_TRY(dalloc_t(net, (size_t)net->S_store, &net->w));
    SNN_TRY(dalloc_t(net, (size_t)net->S_store, &net->sd));
    SNN_TRY(dalloc_t(net, (size_t)N * kDoffStride, &net->doff));
    SNN_TRY(dalloc_t(net, (size_t)N + 1, &net->row_off));
    SNN_TRY(dalloc_t(net, (size_t)N + 1, &net->rin_off));
    SNN_TRY(dalloc_t(net, (size_t)N, &dn.v));
    SNN_TRY(dalloc_t(net, (size_t)N, &dn.u));
    if (net->cfg.flags & SNN_FP64) {
        SNN_TRY(dalloc_t(net, (size_t)N, &dn.vd));
        SNN_TRY(dalloc_t(net, (size_t)N, &dn.ud));
    }
    SNN_TRY(dalloc_t(net, (size_t)N, &dn.I));
    SNN_TRY(dalloc_t(net, (size_t)N, &dn.hl));
    SNN_TRY(dalloc_t(net, (size_t)N, &dn.last_spike));
    SNN_TRY(dalloc_t(net, (size_t)D * N, &dn.ring_ids));
    SNN_TRY(dalloc_t(net, (size_t)2 * D, &dn.ring_cnt));
    SNN_TRY(dalloc_t(net, 1, &net->ctr));
    SNN_TRY(dalloc_t(net, (size_t)2 * kLut, &net->lut));
    if (net->cfg.raster_capacity) {
        SNN_TRY(dalloc_t(net, (size_t)net->cfg.raster_capacity, &dn.raster_gid));
        net->raster_steps_cap = 1 << 14;
        SNN_TRY(dalloc_t(net, (size_t)net->raster_steps_cap, &dn.raster_step_off));
    }
    dn.N = N;
    dn.npc = net->cfg.neurons_per_col;
    dn.ne = net->cfg.exc_per_col;
    dn.C = net->cfg.grid_x * net->cfg.grid_y;
    dn.D = D;
    dn.D_inh = 1;
    dn.S = net->S_store;
    dn.row_off = net->row_off;
    dn.doff = net->doff;
    dn.tgt = net->tgt;
    dn.tgt16 = net->tgt16;
    dn.npc_recip = net->cfg.neurons_per_col >= kMinCompactNpc
                       ? (uint32_t)(((1ull << 32) + net->cfg.neurons_per_col - 1) / net->cfg.neurons_per_col)
                       : 0u;
    dn.nbr = net->nbr;
    dn.w = net->w;
    dn.sd = net->sd;
    dn.rin_off = net->rin_off;
    dn.raster_cap = net->cfg.raster_capacity;
    dn.raster_t0 = 0;
    dn.lut_p = net->lut;
    dn.lut_m = net->lut + kLut;
    dn.stim_t0 = dn.stim_t1 = 0;
    dn.ctr = net->ctr;
    dn.thal_per_col = net->cfg.thal_per_col_per_ms;
    dn.thal_amp = net->cfg.thal_amp_q16;
    dn.seed_lo = (uint32_t)(net->cfg.seed & 0xffffffffu);
    dn.seed_hi = (uint32_t)(net->cfg.seed >> 32);
    dn.flags = net->cfg.flags;
    dn.deriv_period = net->cfg.deriv_period_ms;
    dn.dense_rows = net->launch.dense_rows ? net->launch.dense_rows : 64;
    dn.own_c0 = 0;
    dn.own_c1 = dn.C;
    dn.tile = 0;
    dn.dense_min_spikes = dense_threshold(net->N, net->launch.dense_permille);
    dn.deriv_bias = net->cfg.deriv_bias_q16;
    dn.deriv_decay = net->cfg.deriv_decay_q16;
    dn.wmax = net->cfg.wmax_q16;
    return SNN_OK;
}

// whether the dense pass and the column-staged delivery can run with the
// current launch shape (compact targets, shared memory)
int setup_dense(snn_net *net)
{
    net->dense_ok = false;
    net->dn.staged_ok = 0;
    net->dn.staged_min_events = ~0ull;
    net->dn.ordered_ok = 0;
    net->dn.ring_max_events = 0;
    if (!net->tgt16) return SNN_OK;
    {
        // the column-ordered delivery: deliver_block threads per column, at
        // most deliver_blocks_per_sm resident blocks per SM (one wave)
        int per_sm = 0;
        const uint32_t ob = ordered_block(net->launch.deliver_block);
        const size_t obytes = ordered_smem_bytes(net->cfg.neurons_per_col, ob);
        SNN_CUDA(cudaFuncSetAttribute(k_deliver_ordered, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)obytes));
        SNN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deliver_ordered, (int)ob, obytes));
        per_sm = std::min<int>(per_sm, (int)std::max(1u, net->launch.deliver_blocks_per_sm));
        if (per_sm >= 1) {
            net->dn.ordered_ok = 1;
            net->ordered_grid = (int)std::min<int64_t>(net->dn.C, (int64_t)per_sm * net->sm_count);
            const uint32_t pm = net->launch.ring_permille;
            net->dn.ring_max_events = pm == 0xffffffffu ? ~0ull : (unsigned long long)net->N * pm / 1000ull;
        }
    }
    // a tile takes the column-ordered delivery in every step (it alone
    // delivers to the tile's own columns only)
    if (net->cfg.neurons_per_col > kDenseMaxNpc || net->dn.tile) return SNN_OK;
    // both stage each depression amount in 15 bits
    std::vector<int32_t> lut;
    if (build_luts(&net->cfg, lut) != SNN_OK) return SNN_OK;
    for (int k = 0; k < kLut; ++k)
        if (lut[kLut + k] < 0 || lut[kLut + k] > 0x7fff) return SNN_OK;
    int optin = 0;
    SNN_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, net->device));
    const size_t sbytes = staged_smem_bytes(net->cfg.neurons_per_col, kStagedBlock);
    if (sbytes + 1024 <= (size_t)optin) {
        SNN_CUDA(cudaFuncSetAttribute(k_deliver_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sbytes));
        int per_sm = 0;
        SNN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deliver_cols, (int)kStagedBlock, sbytes));
        if (per_sm >= 1 && net->launch.staged_permille != 0xffffffffu) {
            net->dn.staged_ok = 1;
            net->staged_grid = (int)std::min<int64_t>(net->dn.C, (int64_t)per_sm * net->sm_count);
            const uint32_t pm = net->launch.staged_permille;
            net->dn.staged_min_events = pm == 0xffffffffu ? ~0ull : (unsigned long long)net->N * pm / 1000ull;
        }
    }
    const size_t bytes = dense_smem_bytes(net->cfg.neurons_per_col, net->launch.dense_block);
    if (bytes + 1024 > (size_t)optin) return SNN_OK;
    SNN_CUDA(cudaFuncSetAttribute(k_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    int per_sm = 0;
    SNN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense, (int)net->launch.dense_block, bytes));
    if (per_sm < 1) return SNN_OK;
    // rows per block: the launch's value, or (0) enough blocks for about 8
    // waves of resident blocks, with at least 64 rows to pay for the staging
    uint32_t rows = net->launch.dense_rows;
    if (rows == 0) {
        const uint32_t npc = net->cfg.neurons_per_col, C = net->dn.C;
        const uint64_t want = 8ull * per_sm * net->sm_count;
        uint32_t chunks = (uint32_t)std::max<uint64_t>(1, (want + C - 1) / C);
        chunks = std::min(chunks, std::max(1u, npc / 64));
        rows = (npc + chunks - 1) / chunks;
    }
    net->dn.dense_rows = rows;
    const int64_t units = (int64_t)net->dn.C * ((net->cfg.neurons_per_col + rows - 1) / rows);
    net->dense_grid = (int)std::min<int64_t>(units, (int64_t)per_sm * net->sm_count);
    net->dense_ok = true;
    return SNN_OK;
}

// in-degrees -> overflow check -> reverse index -> LUTs -> initial state
int finish_build(snn_net *net)
{
    const uint32_t N = net->N;
    cudaStream_t s = net->stream;
    DevNet &dn = net->dn;
    int32_t *indeg_exc = nullptr, *indeg_inh = nullptr, *cursor = nullptr, *mx = nullptr;
    long long *sums = nullptr;
    const uint32_t scan_blocks = (N + 1023) / 1024;
    SNN_TRY(dalloc_t(net, (size_t)N, &indeg_exc));
    SNN_TRY(dalloc_t(net, (size_t)N, &indeg_inh));
    SNN_TRY(dalloc_t(net, (size_t)N, &cursor));
    SNN_TRY(dalloc_t(net, 2, &mx));
    SNN_TRY(dalloc_t(net, (size_t)scan_blocks + 1, &sums));
    SNN_CUDA(cudaMemsetAsync(indeg_exc, 0, (size_t)N * 4, s));
    SNN_CUDA(cudaMemsetAsync(indeg_inh, 0, (size_t)N * 4, s));
    SNN_CUDA(cudaMemsetAsync(cursor, 0, (size_t)N * 4, s));
    SNN_CUDA(cudaMemsetAsync(mx, 0, 8, s));
    const int g = grid_for(net, 8);
    k_count_indeg<<<g, 256, 0, s>>>(dn, indeg_exc, indeg_inh);
    k_max2<<<g, 256, 0, s>>>(indeg_exc, indeg_inh, N, mx);
    int32_t hmx[2] = {0, 0};
    SNN_CUDA(cudaMemcpyAsync(hmx, mx, 8, cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    // Q16 current bound: every synapse of the busiest target at its extreme
    // weight plus all the thalamic drive of its column must stay in int32
    // (excitatory weights move inside [0, max(wmax, initial)], inhibitory
    // weights never change).
    {
        const snn_config &c = net->cfg;
        const WeightRange &r = net->wrange;
        const long long thal = (long long)c.thal_per_col_per_ms * c.thal_amp_q16;
        const long long pos = (long long)hmx[0] * std::max<long long>(c.wmax_q16, r.exc_max) +
                              (long long)hmx[1] * std::max<long long>(0, r.inh_max) + std::max(0ll, thal);
        const long long neg = (long long)hmx[0] * std::max<long long>(0, -(long long)r.exc_min) +
                              (long long)hmx[1] * std::max<long long>(0, -(long long)r.inh_min) +
                              std::max(0ll, -thal);
        if (pos > 0x7fffffffll || neg > 0x80000000ll) {
            set_error("int32 Q16 current bound violated (max exc in-degree %d, inh in-degree %d)", hmx[0], hmx[1]);
            return SNN_EOVERFLOW;
        }
    }
    k_scan_sums<<<scan_blocks, 256, 0, s>>>(indeg_exc, N, sums);
    k_scan_carry<<<1, 256, 0, s>>>(sums, scan_blocks);
    k_scan_write<<<scan_blocks, 256, 0, s>>>(indeg_exc, N, sums, net->rin_off);
    int64_t n_rin = 0;
    SNN_CUDA(cudaMemcpyAsync(&n_rin, net->rin_off + N, 8, cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    net->n_rin = n_rin;
    // 4-byte entries where the source fits the compact packing and the row
    // position 11 bits, else 8-byte entries
    if (rin32_ok(net)) {
        SNN_TRY(dalloc_t(net, (size_t)std::max<int64_t>(n_rin, 1), &net->rin32));
    } else {
        SNN_TRY(dalloc_t(net, (size_t)std::max<int64_t>(n_rin, 1), &net->rin));
    }
    dn.rin = net->rin;
    dn.rin32 = net->rin32;
    SNN_TRY(dalloc_t(net, (size_t)std::max<int64_t>(n_rin, 1), &dn.sd_rev));
    SNN_CUDA(cudaMemsetAsync(dn.sd_rev, 0, (size_t)std::max<int64_t>(n_rin, 1) * 4, s));
    dn.n_rin = n_rin;
    k_fill_reverse<<<g, 256, 0, s>>>(dn, cursor, net->rin, net->rin32);
    SNN_CUDA(cudaGetLastError());
    SNN_CUDA(cudaStreamSynchronize(s));
    dfree(net, indeg_exc);
    dfree(net, indeg_inh);
    dfree(net, cursor);
    dfree(net, mx);
    dfree(net, sums);

    std::vector<int32_t> lut;
    SNN_TRY(build_luts(&net->cfg, lut));
    SNN_CUDA(cudaMemcpyAsync(net->lut, lut.data(), lut.size() * 4, cudaMemcpyHostToDevice, s));
    k_init_state<<<g, 256, 0, s>>>(dn);
    DevCounters hc{};
    hc.raster_first_drop_t = 0x7fffffff;
    hc.ltp_pending = kNoPending;
    hc.t_slot[0] = 0;
    hc.t_slot[1] = 0;
    SNN_CUDA(cudaMemcpyAsync(net->ctr, &hc, sizeof hc, cudaMemcpyHostToDevice, s));
    SNN_CUDA(cudaMemsetAsync(dn.ring_cnt, 0, (size_t)2 * net->cfg.max_delay_ms * 4, s));
    if (dn.raster_step_off) SNN_CUDA(cudaMemsetAsync(dn.raster_step_off, 0, 8, s));
    SNN_CUDA(cudaGetLastError());
    SNN_CUDA(cudaStreamSynchronize(s));
    SNN_TRY(setup_dense(net));
    if (!net->dense_ok) net->dn.dense_min_spikes = 0xffffffffu;
    return SNN_OK;
}

int start_net(const snn_config *cfg, void *cuda_stream, size_t budget, snn_net **out, snn_net **made)
{
    SNN_TRY(check_config(cfg));
    if (!out) { set_error("out is NULL"); return SNN_EINVAL; }
    snn_net *net = new snn_net();
    *made = net;
    net->cfg = *cfg;
    net->budget = budget;
    net->alloc = g_alloc;
    net->release = g_release;
    net->alloc_ctx = g_alloc_ctx;
    net->N = cfg->grid_x * cfg->grid_y * cfg->neurons_per_col;
    net->launch.deliver_block = 256;
    net->launch.deliver_blocks_per_sm = 8;
    net->launch.neuron_block = 256;
    net->launch.ltp_block = 256;
    net->launch.ltp_blocks_per_sm = 8;
    net->launch.deriv_block = 256;
    net->launch.graph_steps = 50;
    net->launch.dense_block = 512;
    net->launch.dense_rows = 0;
    net->launch.dense_permille = 250;
    // the 13-column staging no longer pays against the column-ordered
    // delivery, which stages the source column's own neurons (measured on the
    // 64x64 M = 1125 onset and the 128x128 paper geometry): off by default
    // (no launch); a launch shape can still ask for it
    net->launch.staged_permille = 0xffffffffu;
    // the ring-list delivery for steps with few events is off by default:
    // on the 64x64 onset it took 0.64 ms at 1-2 M events (its global
    // reductions into the source's own column contend) against 0.07 ms for
    // the column walk
    net->launch.ring_permille = 0;
    (void)cuda_stream;
    return SNN_OK;
}

// device, SM count and stream (after every host-side check has passed)
int cuda_init(snn_net *net, void *cuda_stream)
{
    SNN_CUDA(cudaGetDevice(&net->device));
    SNN_CUDA(cudaDeviceGetAttribute(&net->sm_count, cudaDevAttrMultiProcessorCount, net->device));
    SNN_TRY(noalloc_lookup(net->device, &net->noalloc_base));
    if (cuda_stream) {
        net->stream = (cudaStream_t)cuda_stream;
    } else {
        SNN_CUDA(cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking));
        net->own_stream = true;
    }
    SNN_CUDA(cudaHostAlloc(&net->host_ctr, 2 * sizeof(DevCounters), cudaHostAllocDefault));
    SNN_CUDA(cudaStreamCreateWithFlags(&net->side, cudaStreamNonBlocking));
    SNN_CUDA(cudaEventCreateWithFlags(&net->ev_fork, cudaEventDisableTiming));
    SNN_CUDA(cudaEventCreateWithFlags(&net->ev_join, cudaEventDisableTiming));
    return SNN_OK;
}

int ensure_raster_steps(snn_net *net, int64_t needed)
{
    if (!net->dn.raster_step_off || needed <= net->raster_steps_cap) return SNN_OK;
    int64_t cap = net->raster_steps_cap;
    while (cap < needed) cap *= 2;
    int64_t *p = nullptr;
    SNN_TRY(dalloc_t(net, (size_t)cap, &p));
    SNN_CUDA(cudaMemcpyAsync(p, net->dn.raster_step_off, (size_t)net->raster_steps_cap * 8,
                             cudaMemcpyDeviceToDevice, net->stream));
    SNN_CUDA(cudaStreamSynchronize(net->stream));
    dfree(net, net->dn.raster_step_off);
    net->dn.raster_step_off = p;
    net->raster_steps_cap = cap;
    drop_graphs(net);
    return SNN_OK;
}

cudaEvent_t next_event(snn_net *net, int kind)
{
    if (net->ev_used == net->ev_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        net->ev_pool.push_back(e);
        net->ev_kind.push_back(0);
    }
    net->ev_kind[net->ev_used] = kind;
    return net->ev_pool[net->ev_used++];
}


// the LTP (and long-term update) owed by step t - 1, applied before any read
void launch_flush(snn_net *net)
{
    const DevNet &dn = net->dn;
    cudaStream_t s = net->stream;
    const int32_t t = net->t;
    const int *t_now = &net->ctr->t_slot[t & 1];
    k_ltp<<<grid_for(net, net->launch.ltp_blocks_per_sm), net->launch.ltp_block, 0, s>>>(dn, t_now, 1);
    k_fold<<<sized_grid(net, 8, net->n_rin, 4096), 256, 0, s>>>(dn, t_now, 1);
    cudaMemsetAsync(&net->ctr->fold_cursor, 0, sizeof(unsigned), s);      // no step closes after this fold
    const uint32_t P = net->cfg.deriv_period_ms;
    if (P && t > 0 && (uint32_t)t % P == 0)
        k_deriv<<<sized_grid(net, 8, (int64_t)dn.C * dn.ne, net->launch.deriv_block / 32), net->launch.deriv_block, 0,
                  s>>>(dn, t_now, 1);
    const int32_t none = kNoPending;
    cudaMemcpyAsync(&net->ctr->ltp_pending, &none, sizeof none, cudaMemcpyHostToDevice, s);
}

// exact_t: t is the step itself (an eager launch), not only its parity (a
// launch captured into a graph that serves many chunks of steps; the host
// captures and replays graphs only over chunks in which no step closes a
// period).  A step that closes a period runs its kernels one after another:
// potentiation, the long-term update (which reads the folded potentiation
// and changes the weights the delivery reads), delivery.  Any other step runs
// the potentiation owed by step t - 1 on the side stream beside the delivery
// of step t: one reads the histories and reverse index and accumulates into
// sd_rev, the other reads the weights and accumulates into I and sd.  While
// profiling, every step runs its kernels one after another, so that each
// kernel's CUDA-event time is its own.
void launch_step(snn_net *net, int32_t t, cudaStream_t s, bool exact_t)
{
    const DevNet &dn = net->dn;
    const int *t_now = &net->ctr->t_slot[t & 1];
    int *t_next = &net->ctr->t_slot[(t & 1) ^ 1];
    const snn_launch &L = net->launch;
    const bool prof = net->profile;
    const uint32_t P = net->cfg.deriv_period_ms;
    const bool closes = exact_t && P && t > 0 && (uint32_t)t % P == 0;
    const bool fork = !closes && !prof;
    cudaStream_t sl = fork ? net->side : s;        // the potentiation's stream
    auto mark = [&](int kind, cudaStream_t on) {
        if (prof) cudaEventRecord(next_event(net, kind), on);
    };
    // [S4(t-1) S5(t-1) S1(t)]: event-driven kernels and the dense pass; the
    // device picks one of the two (the other returns at once)
    if (fork) {
        cudaEventRecord(net->ev_fork, s);
        cudaStreamWaitEvent(sl, net->ev_fork, 0);
    }
    mark(2, sl);
    // sparse grids follow the net's size (a warp per spiker / per 32 buckets)
    const int g_ltp = sized_grid(net, L.ltp_blocks_per_sm, net->N, L.ltp_block / 32);
    const int g_del = sized_grid(net, L.deliver_blocks_per_sm, (int64_t)net->N * dn.D / 4, L.deliver_block);
    int launched = 0;
    k_ltp<<<g_ltp, L.ltp_block, 0, sl>>>(dn, t_now, 0);
    ++launched;
    mark(2, sl);
    if (fork) cudaEventRecord(net->ev_join, sl);
    // long-term update when t closes a period: the event-driven LTP is
    // folded into sd first, both passes read sd afterwards
    if (closes) {
        mark(3, s);
        k_fold<<<sized_grid(net, 8, net->n_rin, 4096), 256, 0, s>>>(dn, t_now, 0);
        k_deriv<<<sized_grid(net, 8, (int64_t)dn.C * dn.ne, L.deriv_block / 32), L.deriv_block, 0, s>>>(dn, t_now, 0);
        launched += 2;
        mark(3, s);
    }
    mark(0, s);
    if (dn.ordered_ok) {
        k_deliver_ordered<<<net->ordered_grid, ordered_block(L.deliver_block),
                            ordered_smem_bytes(dn.npc, ordered_block(L.deliver_block)), s>>>(dn, t_now);
        ++launched;
    }
    if (!dn.ordered_ok || dn.ring_max_events) {
        k_deliver<<<g_del, L.deliver_block, 0, s>>>(dn, t_now);
        ++launched;
    }
    if (dn.staged_ok) {
        k_deliver_cols<<<net->staged_grid, kStagedBlock, staged_smem_bytes(dn.npc, kStagedBlock), s>>>(dn, t_now);
        ++launched;
    }
    mark(0, s);
    if (net->dense_ok) {
        mark(4, s);
        k_dense<<<net->dense_grid, L.dense_block, dense_smem_bytes(dn.npc, L.dense_block), s>>>(dn, t_now);
        ++launched;
        mark(4, s);
    }
    if (fork) cudaStreamWaitEvent(s, net->ev_join, 0);
    // [S2(t) S3(t)]
    const int nb_neuron = (int)((net->N + L.neuron_block * kNeuronsPerThread - 1) /
                                (L.neuron_block * kNeuronsPerThread));
    mark(1, s);
    if (dn.vd) k_neuron_f64<<<nb_neuron, L.neuron_block, 0, s>>>(dn, t_now, t_next);
    else k_neuron_f32<<<nb_neuron, L.neuron_block, 0, s>>>(dn, t_now, t_next);
    ++launched;
    if (dn.probe_n) {
        k_probe<<<(dn.probe_n + 255) / 256, 256, 0, s>>>(dn, t_now);
        ++launched;
    }
    mark(1, s);
    if (prof) net->prof_kernels += launched;
}

uint32_t effective_graph_len(const snn_net *net)
{
    const uint32_t L = net->launch.graph_steps;
    if (net->profile || L < 2) return 0;
    return L & ~1u;
}

// one chunk of L steps starting at an even step (only the parity of t is
// baked into the launches; everything else is read on the device)
int build_graph(snn_net *net, uint32_t L)
{
    cudaGraph_t g = nullptr;
    SNN_CUDA(cudaStreamBeginCapture(net->stream, cudaStreamCaptureModeThreadLocal));
    for (uint32_t k = 0; k < L; ++k) launch_step(net, (int32_t)k, net->stream, false);
    cudaError_t e = cudaStreamEndCapture(net->stream, &g);
    if (e != cudaSuccess) {
        set_error("graph capture failed: %s", cudaGetErrorString(e));
        return SNN_ECUDA;
    }
    e = cudaGraphInstantiate(&net->graph[0], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        net->graph[0] = nullptr;
        set_error("graph instantiate failed: %s", cudaGetErrorString(e));
        return SNN_ECUDA;
    }
    return SNN_OK;
}

int read_counters_raw(snn_net *net, DevCounters *hc)
{
    SNN_CUDA(cudaMemcpyAsync(hc, net->ctr, sizeof *hc, cudaMemcpyDeviceToHost, net->stream));
    SNN_CUDA(cudaStreamSynchronize(net->stream));
    return SNN_OK;
}

// end of a run: the counters are copied out behind the steps and read after
// the one synchronisation (the device error word decides the return code)
int finish_run(snn_net *net)
{
    SNN_CUDA(cudaMemcpyAsync(&net->host_ctr[1], net->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, net->stream));
    SNN_CUDA(cudaStreamSynchronize(net->stream));
    SNN_CUDA(cudaGetLastError());
    if (net->profile && net->ev_used) {
        for (size_t i = 0; i + 1 < net->ev_used; i += 2) {
            float ms = 0.f;
            SNN_CUDA(cudaEventElapsedTime(&ms, net->ev_pool[i], net->ev_pool[i + 1]));
            net->prof_ms[net->ev_kind[i]] += ms;
            net->prof_n[net->ev_kind[i]] += 1;
        }
        net->ev_used = 0;
    }
    const DevCounters &hc = net->host_ctr[1];
    if (hc.error) {
        set_error("device error word %d", hc.error);
        return (hc.error == SNN_ETIMEOUT || hc.error == SNN_EBOUNDS) ? hc.error : SNN_ECUDA;
    }
    return SNN_OK;
}

// count_before: also copy the counters out ahead of the steps (host_ctr[0]),
// without a synchronisation of its own
int run_steps(snn_net *net, uint32_t n_ms, bool count_before = false)
{
    if ((int64_t)net->t + n_ms > 0x7fff0000ll) { set_error("time limit reached"); return SNN_ESTATE; }
    SNN_TRY(ensure_raster_steps(net, (int64_t)net->t + n_ms + 2 - net->dn.raster_t0));
    if (count_before)
        SNN_CUDA(cudaMemcpyAsync(&net->host_ctr[0], net->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                                 net->stream));
    const uint32_t L = effective_graph_len(net);
    if (L != net->graph_len) {
        drop_graphs(net);
        net->graph_len = L;
    }
    uint32_t left = n_ms;
    const uint32_t P = net->cfg.deriv_period_ms;
    while (left > 0) {
        const int32_t t = net->t;
        // the first step from t on that closes a period (t' > 0, t' % P == 0)
        const int64_t closing = P ? std::max<int64_t>((int64_t)P, ((int64_t)t + P - 1) / P * P) : INT64_MAX;
        if (L >= 2 && (t & 1) == 0 && left >= L && closing >= (int64_t)t + L) {
            if (net->graphs_dirty) {
                for (int i = 0; i < 2; ++i)
                    if (net->graph[i]) { cudaGraphExecDestroy(net->graph[i]); net->graph[i] = nullptr; }
                net->graphs_dirty = false;
            }
            if (!net->graph[0]) SNN_TRY(build_graph(net, L));
            SNN_CUDA(cudaGraphLaunch(net->graph[0], net->stream));
            net->t += (int32_t)L;
            left -= L;
            net->ltp_owed = true;
        } else {
            launch_step(net, t, net->stream, true);
            SNN_CUDA(cudaGetLastError());
            net->t += 1;
            left -= 1;
            net->ltp_owed = true;
        }
    }
    return finish_run(net);
}

// canonical (unpadded, source-major) index of the first synapse of row p
int canon_offset(snn_net *net, uint32_t p, int64_t *out)
{
    if (net->dn.uniform_m) {
        *out = (int64_t)p * net->dn.canon_m;
        return SNN_OK;
    }
    SNN_CUDA(cudaMemcpyAsync(out, net->row_off + p, 8, cudaMemcpyDeviceToHost, net->stream));
    SNN_CUDA(cudaStreamSynchronize(net->stream));
    return SNN_OK;
}

// apply the LTP / long-term update owed by the last step (before reads)
int flush_owed(snn_net *net)
{
    if (!net->ltp_owed) return SNN_OK;
    launch_flush(net);
    SNN_CUDA(cudaGetLastError());
    SNN_CUDA(cudaStreamSynchronize(net->stream));
    net->ltp_owed = false;
    return SNN_OK;
}

int set_stimulus_impl(snn_net *net, const snn_stimulus *ev, size_t n)
{
    DevNet &dn = net->dn;
    if (n == 0) {
        dn.stim_t0 = dn.stim_t1 = 0;
        drop_graphs(net);
        return SNN_OK;
    }
    if (!ev) { set_error("events is NULL"); return SNN_EINVAL; }
    std::vector<snn_stimulus> e;
    e.reserve(n);
    for (size_t i = 0; i < n; ++i) {
        if (ev[i].gid < 0 || (uint32_t)ev[i].gid >= net->N) {
            set_error("stimulus %zu: gid %d out of range", i, ev[i].gid);
            return SNN_EINVAL;
        }
        if (ev[i].t >= net->t) e.push_back(ev[i]);
    }
    if (e.empty()) {
        dn.stim_t0 = dn.stim_t1 = 0;
        drop_graphs(net);
        return SNN_OK;
    }
    auto by_t = [](const snn_stimulus &a, const snn_stimulus &b) { return a.t < b.t; };
    if (!std::is_sorted(e.begin(), e.end(), by_t)) std::stable_sort(e.begin(), e.end(), by_t);
    const int32_t t0 = e.front().t, t1 = e.back().t + 1;
    // staged in pinned host memory (the copies below run behind the caller;
    // the stream is idle here, every run ends with a synchronisation, so the
    // staging of an earlier upload is free)
    const size_t n_off = (size_t)(t1 - t0) + 1;
    const size_t stage = e.size() * 8 + n_off * 8;
    SNN_CUDA(cudaStreamSynchronize(net->stream));
    if (stage > net->stim_stage_cap) {
        if (net->stim_stage) cudaFreeHost(net->stim_stage);
        net->stim_stage = nullptr;
        net->stim_stage_cap = 0;
        SNN_CUDA(cudaHostAlloc(&net->stim_stage, stage, cudaHostAllocDefault));
        net->stim_stage_cap = stage;
    }
    int64_t *off = reinterpret_cast<int64_t *>(net->stim_stage);
    int32_t *gid = reinterpret_cast<int32_t *>(off + n_off);
    int32_t *q = gid + e.size();
    std::fill(off, off + n_off, 0);
    for (size_t i = 0; i < e.size(); ++i) {
        gid[i] = e[i].gid;
        q[i] = e[i].q16;
        off[(size_t)(e[i].t - t0) + 1]++;
    }
    for (size_t k = 1; k < n_off; ++k) off[k] += off[k - 1];
    if (e.size() > net->stim_cap) {
        dfree(net, (void *)dn.stim_gid);
        dfree(net, (void *)dn.stim_q16);
        dn.stim_gid = dn.stim_q16 = nullptr;
        int32_t *a = nullptr, *b = nullptr;
        SNN_TRY(dalloc_t(net, e.size(), &a));
        SNN_TRY(dalloc_t(net, e.size(), &b));
        dn.stim_gid = a;
        dn.stim_q16 = b;
        net->stim_cap = e.size();
    }
    if ((int64_t)n_off > net->stim_off_cap) {
        dfree(net, (void *)dn.stim_off);
        dn.stim_off = nullptr;
        int64_t *o = nullptr;
        SNN_TRY(dalloc_t(net, n_off, &o));
        dn.stim_off = o;
        net->stim_off_cap = (int64_t)n_off;
    }
    SNN_CUDA(cudaMemcpyAsync((void *)dn.stim_gid, gid, e.size() * 4, cudaMemcpyHostToDevice, net->stream));
    SNN_CUDA(cudaMemcpyAsync((void *)dn.stim_q16, q, e.size() * 4, cudaMemcpyHostToDevice, net->stream));
    SNN_CUDA(cudaMemcpyAsync((void *)dn.stim_off, off, n_off * 8, cudaMemcpyHostToDevice, net->stream));
    dn.stim_t0 = t0;
    dn.stim_t1 = t1;
    drop_graphs(net);
    return SNN_OK;
}

int raster_window(snn_net *net, int32_t t0, int32_t t1, std::vector<snn_spike> &out, bool &truncated)
{
    out.clear();
    truncated = false;
    DevNet &dn = net->dn;
    if (!dn.raster_gid) { set_error("the net keeps no raster (raster_capacity = 0)"); return SNN_ESTATE; }
    const int32_t lo = std::max(t0, dn.raster_t0), hi = std::min(t1, net->t);
    if (t0 < dn.raster_t0) truncated = true;
    if (hi <= lo) return SNN_OK;
    std::vector<int64_t> off((size_t)(hi - lo) + 1);
    SNN_CUDA(cudaMemcpyAsync(off.data(), dn.raster_step_off + (lo - dn.raster_t0), off.size() * 8,
                             cudaMemcpyDeviceToHost, net->stream));
    SNN_CUDA(cudaStreamSynchronize(net->stream));
    const int64_t a = off.front(), b = off.back();
    std::vector<int32_t> gid((size_t)(b - a));
    if (b > a) {
        SNN_CUDA(cudaMemcpyAsync(gid.data(), dn.raster_gid + a, (size_t)(b - a) * 4, cudaMemcpyDeviceToHost,
                                 net->stream));
        SNN_CUDA(cudaStreamSynchronize(net->stream));
    }
    out.resize(gid.size());
    for (int32_t t = lo; t < hi; ++t) {
        const int64_t s0 = off[(size_t)(t - lo)] - a, s1 = off[(size_t)(t - lo) + 1] - a;
        std::sort(gid.begin() + s0, gid.begin() + s1);
        for (int64_t k = s0; k < s1; ++k) out[(size_t)k] = snn_spike{t, gid[(size_t)k]};
    }
    DevCounters hc{};
    SNN_TRY(read_counters_raw(net, &hc));
    if (hc.raster_dropped && hi > hc.raster_first_drop_t) truncated = true;
    return SNN_OK;
}

int raster_reset_impl(snn_net *net)
{
    DevNet &dn = net->dn;
    if (!dn.raster_gid) return SNN_OK;
    DevCounters hc{};
    SNN_TRY(read_counters_raw(net, &hc));
    hc.raster_total = 0;
    hc.raster_dropped = 0;
    hc.raster_first_drop_t = 0x7fffffff;
    SNN_CUDA(cudaMemcpyAsync(net->ctr, &hc, sizeof hc, cudaMemcpyHostToDevice, net->stream));
    SNN_CUDA(cudaMemsetAsync(dn.raster_step_off, 0, 8, net->stream));
    SNN_CUDA(cudaStreamSynchronize(net->stream));
    dn.raster_t0 = net->t;
    drop_graphs(net);
    return SNN_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *snn_strerror(int code)
{
    switch (code) {
    case SNN_OK: return "ok";
    case SNN_EINVAL: return "invalid argument or configuration";
    case SNN_ENOMEM: return "device memory budget exceeded or allocation failed";
    case SNN_ECUDA: return "CUDA error";
    case SNN_EOVERFLOW: return "Q16 current bound cannot be guaranteed";
    case SNN_ETIMEOUT: return "bounded device wait gave up";
    case SNN_EBOUNDS: return "a kernel met an index out of range (checked build)";
    case SNN_ETRUNC: return "output truncated";
    case SNN_ESTATE: return "call does not fit the state of the handle";
    default: return "unknown error";
    }
}

const char *snn_last_error(void) { return g_last_error.c_str(); }

void snn_set_allocator(void *(*alloc)(size_t, void *, void *), void (*release)(void *, void *), void *ctx)
{
    g_alloc = alloc;
    g_release = release;
    g_alloc_ctx = ctx;
}

void snn_free(snn_net *net)
{
    if (!net) return;
    if (net->stream) cudaStreamSynchronize(net->stream);
    drop_graphs(net);
    for (cudaEvent_t e : net->ev_pool) cudaEventDestroy(e);
    while (!net->blocks.empty()) dfree(net, net->blocks.back().p);
    if (net->host_ctr) cudaFreeHost(net->host_ctr);
    if (net->ev_fork) cudaEventDestroy(net->ev_fork);
    if (net->ev_join) cudaEventDestroy(net->ev_join);
    if (net->side) cudaStreamDestroy(net->side);
    if (net->stim_stage) cudaFreeHost(net->stim_stage);
    if (net->own_stream && net->stream) cudaStreamDestroy(net->stream);
    delete net;
}

int snn_build_network(const snn_config *cfg, void *cuda_stream, size_t hbm_budget_bytes, snn_net **out)
{
    snn_net *net = nullptr;
    int r = start_net(cfg, cuda_stream, hbm_budget_bytes, out, &net);
    auto fail = [&](int code) { snn_free(net); if (out) *out = nullptr; return code; };
    if (r != SNN_OK) return fail(r);
    const snn_config &c = net->cfg;
    net->S = (int64_t)net->N * c.fanout;
    const bool compact = c.neurons_per_col >= kMinCompactNpc && c.neurons_per_col <= kMaxCompactNpc;
    const uint32_t m_store = compact ? ((c.fanout + 7u) & ~7u) : c.fanout;
    net->S_store = (int64_t)net->N * m_store;
    const int64_t n_rin_est = (int64_t)c.grid_x * c.grid_y * c.exc_per_col * c.fanout;
    const size_t need = footprint(&c, net->N, net->S_store, n_rin_est, false) + (size_t)c.raster_capacity * 4 + (1 << 17);
    if (hbm_budget_bytes && need > hbm_budget_bytes) {
        set_error("network needs about %zu bytes, budget is %zu", need, hbm_budget_bytes);
        return fail(SNN_ENOMEM);
    }
    if ((r = cuda_init(net, cuda_stream)) != SNN_OK) return fail(r);
    if ((r = alloc_common(net)) != SNN_OK) return fail(r);
    net->dn.uniform_m = m_store;
    net->dn.w_inh = c.w_inh0_q16;
    net->dn.canon_m = c.fanout;
    net->wrange = WeightRange{c.w_exc0_q16, c.w_exc0_q16, c.w_inh0_q16, c.w_inh0_q16};
    GenParams &g = net->gen;
    g.npc = c.neurons_per_col;
    g.ne = c.exc_per_col;
    g.m = c.fanout;
    g.m_store = m_store;
    g.D = c.max_delay_ms;
    g.gx = c.grid_x;
    g.gy = c.grid_y;
    uint32_t acc = 0;
    for (int k = 0; k < 4; ++k) {
        acc += c.pct_ring[k];
        g.ring_end[k] = (uint32_t)(((uint64_t)c.fanout * acc) / 100u);
    }
    g.seed_lo = net->dn.seed_lo;
    g.seed_hi = net->dn.seed_hi;
    g.w_exc0 = c.w_exc0_q16;
    g.w_inh0 = c.w_inh0_q16;
    const int gr = grid_for(net, 16);
    k_fill_row_off<<<gr, 256, 0, net->stream>>>(net->row_off, net->N, m_store);
    k_gen_rows<<<gr, 256, 0, net->stream>>>(g, net->N, net->doff, net->tgt, net->tgt16, net->w, net->sd);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(net->stream) != cudaSuccess) {
        set_error("network generation failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(SNN_ECUDA);
    }
    if ((r = finish_build(net)) != SNN_OK) return fail(r);
    *out = net;
    return SNN_OK;
}

int snn_build_network_explicit(const snn_config *cfg, const int64_t *host_row_off, const int32_t *host_tgt,
                               const uint8_t *host_delay, const int32_t *host_w, void *cuda_stream,
                               size_t hbm_budget_bytes, snn_net **out)
{
    snn_net *net = nullptr;
    int r = start_net(cfg, cuda_stream, hbm_budget_bytes, out, &net);
    auto fail = [&](int code) { snn_free(net); if (out) *out = nullptr; return code; };
    if (r != SNN_OK) return fail(r);
    if (!host_row_off) { set_error("row offsets are NULL"); return fail(SNN_EINVAL); }
    const uint32_t N = net->N;
    const uint32_t D = net->cfg.max_delay_ms;
    if (host_row_off[0] != 0) { set_error("row_off[0] must be 0"); return fail(SNN_EINVAL); }
    for (uint32_t p = 0; p < N; ++p) {
        const int64_t len = host_row_off[p + 1] - host_row_off[p];
        if (len < 0 || len > 65535) { set_error("row %u has %lld synapses (0..65535)", p, (long long)len); return fail(SNN_EINVAL); }
    }
    const int64_t S = host_row_off[N];
    if (S > 0 && (!host_tgt || !host_delay || !host_w)) { set_error("synapse arrays are NULL"); return fail(SNN_EINVAL); }
    for (int64_t k = 0; k < S; ++k) {
        if (host_tgt[k] < 0 || (uint32_t)host_tgt[k] >= N || host_delay[k] < 1 || host_delay[k] > D) {
            set_error("synapse %lld: target or delay out of range", (long long)k);
            return fail(SNN_EINVAL);
        }
    }
    net->explicit_net = true;
    net->S = S;
    net->S_store = S;
    int64_t n_exc = 0;
    net->wrange = WeightRange{0, 0, 0, 0};
    for (uint32_t p = 0; p < N; ++p) {
        const bool exc = (p % net->cfg.neurons_per_col) < net->cfg.exc_per_col;
        if (exc) n_exc += host_row_off[p + 1] - host_row_off[p];
        for (int64_t k = host_row_off[p]; k < host_row_off[p + 1]; ++k) {
            WeightRange &r = net->wrange;
            if (exc) { r.exc_min = std::min(r.exc_min, host_w[k]); r.exc_max = std::max(r.exc_max, host_w[k]); }
            else { r.inh_min = std::min(r.inh_min, host_w[k]); r.inh_max = std::max(r.inh_max, host_w[k]); }
        }
    }
    const size_t need = footprint(&net->cfg, N, S, n_exc, true) + (size_t)net->cfg.raster_capacity * 4 + (1 << 17);
    if (hbm_budget_bytes && need > hbm_budget_bytes) {
        set_error("network needs about %zu bytes, budget is %zu", need, hbm_budget_bytes);
        return fail(SNN_ENOMEM);
    }
    if ((r = cuda_init(net, cuda_stream)) != SNN_OK) return fail(r);
    if ((r = alloc_common(net)) != SNN_OK) return fail(r);
    if ((r = dalloc_t(net, (size_t)std::max<int64_t>(S, 1), &net->canon_delay)) != SNN_OK) return fail(r);
    net->dn.uniform_m = 0;
    net->dn.D_inh = 1;
    for (uint32_t p = 0; p < N; ++p)
        if ((p % net->cfg.neurons_per_col) >= net->cfg.exc_per_col)
            for (int64_t k = host_row_off[p]; k < host_row_off[p + 1]; ++k)
                net->dn.D_inh = std::max<uint32_t>(net->dn.D_inh, host_delay[k]);
    // stable counting sort of every row by delay
    std::vector<int32_t> tg((size_t)S), ww((size_t)S);
    std::vector<uint16_t> doff((size_t)N * kDoffStride, 0);
    for (uint32_t p = 0; p < N; ++p) {
        const int64_t lo = host_row_off[p], hi = host_row_off[p + 1];
        uint32_t cnt[kDoffStride] = {0};
        for (int64_t k = lo; k < hi; ++k) cnt[host_delay[k]]++;
        uint16_t *o = &doff[(size_t)p * kDoffStride];
        uint32_t accd = 0;
        uint32_t start[kDoffStride] = {0};
        for (uint32_t d = 0; d <= D; ++d) {
            start[d] = accd;
            accd += cnt[d];
            o[d] = (uint16_t)accd;
        }
        for (int64_t k = lo; k < hi; ++k) {
            const int64_t pos = lo + start[host_delay[k]]++;
            tg[(size_t)pos] = host_tgt[k];
            ww[(size_t)pos] = host_w[k];
        }
    }
    cudaStream_t s = net->stream;
    if (cudaMemcpyAsync(net->row_off, host_row_off, ((size_t)N + 1) * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(net->doff, doff.data(), doff.size() * 2, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        (S > 0 && (cudaMemcpyAsync(net->tgt, tg.data(), (size_t)S * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                   cudaMemcpyAsync(net->w, ww.data(), (size_t)S * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                   cudaMemsetAsync(net->sd, 0, (size_t)S * 4, s) != cudaSuccess ||
                   cudaMemcpyAsync(net->canon_delay, host_delay, (size_t)S, cudaMemcpyHostToDevice, s) != cudaSuccess)) ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(SNN_ECUDA);
    }
    if ((r = finish_build(net)) != SNN_OK) return fail(r);
    *out = net;
    return SNN_OK;
}

int snn_set_stimulus(snn_net *net, const snn_stimulus *host_events, size_t n)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    return set_stimulus_impl(net, host_events, n);
}

int snn_set_tile(snn_net *net, uint32_t first_col, uint32_t n_cols)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    const uint32_t C = net->dn.C;
    if (n_cols == 0 || first_col >= C || n_cols > C - first_col) { set_error("column range outside the torus"); return SNN_EINVAL; }
    if (net->t != 0) { set_error("a net becomes a tile before its first step"); return SNN_ESTATE; }
    if (!net->tgt16 || !net->dn.ordered_ok) {
        set_error("tiles need a generated net with compact targets");
        return SNN_ESTATE;
    }
    const bool whole = first_col == 0 && n_cols == C;
    if (!whole && !net->inject_buf) SNN_TRY(dalloc_t(net, (size_t)net->N, &net->inject_buf));
    net->dn.own_c0 = first_col;
    net->dn.own_c1 = first_col + n_cols;
    net->dn.tile = whole ? 0 : 1;
    net->dn.dense_min_spikes = dense_threshold(net->N, net->launch.dense_permille);
    SNN_TRY(setup_dense(net));
    if (!net->dense_ok) net->dn.dense_min_spikes = 0xffffffffu;
    drop_graphs(net);
    return SNN_OK;
}

int snn_inject_spikes(snn_net *net, const int32_t *host_gids, uint32_t n)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    if (!net->dn.tile) { set_error("spikes are injected into tiles only"); return SNN_ESTATE; }
    if (net->t < 1) { set_error("no step has run yet"); return SNN_ESTATE; }
    if (n == 0) return SNN_OK;
    if (!host_gids) { set_error("host_gids is NULL"); return SNN_EINVAL; }
    const uint32_t npc = net->dn.npc;
    std::vector<uint8_t> seen;
    for (uint32_t k = 0; k < n; ++k) {
        const int32_t g = host_gids[k];
        if (g < 0 || (uint32_t)g >= net->N) { set_error("gid %d out of range", g); return SNN_EINVAL; }
        const uint32_t col = (uint32_t)g / npc;
        if (col >= net->dn.own_c0 && col < net->dn.own_c1) {
            set_error("gid %d belongs to the tile itself", g);
            return SNN_EINVAL;
        }
    }
    if (n > net->N) { set_error("more spikes than neurons"); return SNN_EINVAL; }
    seen.assign(net->N, 0);
    for (uint32_t k = 0; k < n; ++k) {
        if (seen[(uint32_t)host_gids[k]]) { set_error("gid %d appears twice", host_gids[k]); return SNN_EINVAL; }
        seen[(uint32_t)host_gids[k]] = 1;
    }
    SNN_CUDA(cudaMemcpyAsync(net->inject_buf, host_gids, (size_t)n * 4, cudaMemcpyHostToDevice, net->stream));
    k_inject<<<1, 1024, 0, net->stream>>>(net->dn, net->t - 1, net->inject_buf, n);
    SNN_CUDA(cudaGetLastError());
    SNN_CUDA(cudaStreamSynchronize(net->stream));
    return SNN_OK;
}

int snn_set_thalamic(snn_net *net, int on)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    net->dn.thal_per_col = on ? net->cfg.thal_per_col_per_ms : 0u;
    drop_graphs(net);
    return SNN_OK;
}

int snn_set_launch(snn_net *net, const snn_launch *launch)
{
    if (!net || !launch) { set_error("NULL argument"); return SNN_EINVAL; }
    snn_launch L = net->launch;
    auto pick = [](uint32_t v, uint32_t cur) { return v ? v : cur; };
    L.deliver_block = pick(launch->deliver_block, L.deliver_block);
    L.deliver_blocks_per_sm = pick(launch->deliver_blocks_per_sm, L.deliver_blocks_per_sm);
    L.neuron_block = pick(launch->neuron_block, L.neuron_block);
    L.ltp_block = pick(launch->ltp_block, L.ltp_block);
    L.ltp_blocks_per_sm = pick(launch->ltp_blocks_per_sm, L.ltp_blocks_per_sm);
    L.deriv_block = pick(launch->deriv_block, L.deriv_block);
    L.graph_steps = pick(launch->graph_steps, L.graph_steps);
    L.dense_block = pick(launch->dense_block, L.dense_block);
    L.dense_rows = pick(launch->dense_rows, L.dense_rows);
    L.dense_permille = pick(launch->dense_permille, L.dense_permille);
    L.staged_permille = pick(launch->staged_permille, L.staged_permille);
    L.ring_permille = pick(launch->ring_permille, L.ring_permille);
    for (uint32_t b : {L.deliver_block, L.neuron_block, L.ltp_block, L.deriv_block}) {
        if (b < 32 || b > 1024 || b % 32) { set_error("block sizes must be multiples of 32 in 32..1024"); return SNN_EINVAL; }
    }
    if (L.dense_block < 32 || L.dense_block > 1024 || L.dense_block % 32) {
        set_error("dense_block must be a multiple of 32 in 32..1024");
        return SNN_EINVAL;
    }
    if (L.deliver_blocks_per_sm > 64 || L.ltp_blocks_per_sm > 64) { set_error("blocks per SM must be <= 64"); return SNN_EINVAL; }
    net->launch = L;
    net->dn.dense_min_spikes = dense_threshold(net->N, L.dense_permille);
    SNN_TRY(setup_dense(net));
    if (!net->dense_ok) net->dn.dense_min_spikes = 0xffffffffu;
    drop_graphs(net);
    return SNN_OK;
}

int snn_get_launch(const snn_net *net, snn_launch *launch)
{
    if (!net || !launch) { set_error("NULL argument"); return SNN_EINVAL; }
    *launch = net->launch;
    return SNN_OK;
}

int snn_step(snn_net *net)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    return run_steps(net, 1);
}

int snn_run(snn_net *net, uint32_t n_ms)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    if (n_ms == 0) return SNN_OK;
    return run_steps(net, n_ms);
}

int snn_run_host(snn_net *net, uint32_t n_ms, const snn_stimulus *host_stimulus, size_t n_stim,
                 snn_spike *host_spikes, size_t cap, size_t *n_out)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    const int32_t t0 = net->t;
    SNN_TRY(set_stimulus_impl(net, host_stimulus, host_stimulus ? n_stim : 0));
    if (!host_spikes) {
        // one synchronisation: the counters before and after the steps are
        // copied out on the stream around them
        SNN_TRY(run_steps(net, n_ms, true));
        if (n_out) *n_out = (size_t)(net->host_ctr[1].spikes - net->host_ctr[0].spikes);
        return SNN_OK;
    }
    if (!net->dn.raster_gid) { set_error("snn_run_host needs raster_capacity > 0"); return SNN_ESTATE; }
    if (net->dn.raster_t0 != t0) SNN_TRY(raster_reset_impl(net));
    SNN_TRY(run_steps(net, n_ms));
    std::vector<snn_spike> out;
    bool trunc = false;
    SNN_TRY(raster_window(net, t0, t0 + (int32_t)n_ms, out, trunc));
    if (n_out) *n_out = out.size();
    const size_t k = std::min(cap, out.size());
    if (k && host_spikes) std::memcpy(host_spikes, out.data(), k * sizeof(snn_spike));
    SNN_TRY(raster_reset_impl(net));
    if (trunc || out.size() > cap) { set_error("raster window truncated"); return SNN_ETRUNC; }
    return SNN_OK;
}

void snn_batch_free(snn_batch *b)
{
    if (!b) return;
    if (b->main) cudaStreamSynchronize(b->main);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->tables) cudaFree(b->tables);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaStream_t st : b->branch) cudaStreamDestroy(st);
    if (b->main) cudaStreamDestroy(b->main);
    delete b;
}

int snn_batch_create(snn_net *const *nets, uint32_t n_nets, uint32_t graph_steps, snn_batch **out)
{
    if (!out) { set_error("out is NULL"); return SNN_EINVAL; }
    *out = nullptr;
    if (!nets || n_nets == 0) { set_error("a batch needs at least one net"); return SNN_EINVAL; }
    int dev = 0;
    SNN_CUDA(cudaGetDevice(&dev));
    for (uint32_t i = 0; i < n_nets; ++i) {
        if (!nets[i]) { set_error("net %u is NULL", i); return SNN_EINVAL; }
        if (nets[i]->device != dev) { set_error("net %u lives on another device", i); return SNN_EINVAL; }
        if (nets[i]->profile) { set_error("net %u is profiling", i); return SNN_ESTATE; }
        for (uint32_t j = 0; j < i; ++j)
            if (nets[j] == nets[i]) { set_error("net %u appears twice", i); return SNN_EINVAL; }
    }
    snn_batch *b = new snn_batch();
    auto fail = [&](int code) { snn_batch_free(b); return code; };
    b->nets.assign(nets, nets + n_nets);
    b->L = (graph_steps ? graph_steps : 10) & ~1u;
    b->device = dev;
    b->launch = nets[0]->launch;
    b->launch.graph_steps = b->L;
    if (cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_error("cudaDeviceGetAttribute failed");
        return fail(SNN_ECUDA);
    }
    if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        set_error("stream / event creation failed");
        return fail(SNN_ECUDA);
    }
    b->branch.resize(n_nets, nullptr);
    b->join.resize(n_nets, nullptr);
    for (uint32_t i = 0; i < n_nets; ++i) {
        if (cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess) {
            set_error("stream / event creation failed");
            return fail(SNN_ECUDA);
        }
    }
    *out = b;
    return SNN_OK;
}

namespace {

// the next `count` steps of every net (from its own t), each net on its own
// branch stream, joined back into the batch's main stream (single eager
// steps that do not fill a captured chunk)
void batch_enqueue(snn_batch *b, uint32_t count, bool exact_t)
{
    cudaEventRecord(b->fork, b->main);
    for (size_t i = 0; i < b->nets.size(); ++i) {
        snn_net *n = b->nets[i];
        cudaStreamWaitEvent(b->branch[i], b->fork, 0);
        for (uint32_t k = 0; k < count; ++k) launch_step(n, n->t + (int32_t)k, b->branch[i], exact_t);
        cudaEventRecord(b->join[i], b->branch[i]);
        cudaStreamWaitEvent(b->main, b->join[i], 0);
    }
}

// blocks of every net in one batched launch of a kind: as many as the net
// would use alone (one resident wave, at most `cap`), so that whichever nets
// have work in a step (the device decides per net and step) can fill the
// GPU; the blocks of a net with nothing to do return at once.  Nets the
// kind does not apply to get none (weight 0).
void share_blocks(const std::vector<double> &weight, const std::vector<uint64_t> &cap, uint64_t wave,
                  std::vector<uint32_t> &cnt)
{
    cnt.assign(weight.size(), 0);
    for (size_t i = 0; i < weight.size(); ++i) {
        if (weight[i] <= 0) continue;
        const uint64_t c = std::max<uint64_t>(1, std::min<uint64_t>(wave, std::max<uint64_t>(1, cap[i])));
        cnt[i] = (uint32_t)std::min<uint64_t>(c, 1u << 20);
    }
}

// resident blocks per SM of a batched kernel (at least 1), capped at `cap`
int batch_occupancy(const void *kernel, uint32_t block, size_t smem, uint32_t cap)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, (int)block, smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    return std::max(1, std::min<int>(per_sm, (int)std::max(1u, cap)));
}

// the launch tables of every kind for the nets as they are now (DevNet
// copies, parities), uploaded to the batch's device buffer
int batch_tables(snn_batch *b)
{
    const size_t nn = b->nets.size();
    const snn_launch &L = b->launch;
    const uint64_t sms = (uint64_t)std::max(1, b->sm_count);
    std::vector<uint32_t> cnt[kBKinds];
    for (int k = 0; k < kBKinds; ++k) b->kind[k] = snn_batch::Kind{};
    std::vector<double> w(nn);
    std::vector<uint64_t> cap(nn);
    auto work = [&](size_t i) { return (double)b->nets[i]->N * (double)std::max<int64_t>(1, b->nets[i]->S / std::max<uint32_t>(1, b->nets[i]->N)); };
    int optin = 0;
    SNN_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
    // potentiation: warp per spiker
    for (size_t i = 0; i < nn; ++i) {
        const snn_net *n = b->nets[i];
        w[i] = (n->cfg.flags & SNN_STDP_OFF) ? 0.0 : work(i);
        cap[i] = (n->N + L.ltp_block / 32 - 1) / (L.ltp_block / 32);
    }
    b->kind[kBLtp].block = L.ltp_block;
    share_blocks(w, cap, sms * batch_occupancy((const void *)k_ltp_b, L.ltp_block, 0, L.ltp_blocks_per_sm), cnt[kBLtp]);
    // fold and long-term update (return at once off period ends)
    for (size_t i = 0; i < nn; ++i) {
        const snn_net *n = b->nets[i];
        w[i] = n->cfg.deriv_period_ms ? (double)std::max<int64_t>(1, n->n_rin) : 0.0;
        cap[i] = (n->N + 63) / 64;
    }
    b->kind[kBFold].block = 256;
    share_blocks(w, cap, sms * 8, cnt[kBFold]);
    for (size_t i = 0; i < nn; ++i) {
        const snn_net *n = b->nets[i];
        w[i] = n->cfg.deriv_period_ms ? work(i) : 0.0;
        cap[i] = ((uint64_t)n->dn.C * n->dn.ne + L.deriv_block / 32 - 1) / (L.deriv_block / 32);
    }
    b->kind[kBDeriv].block = L.deriv_block;
    share_blocks(w, cap, sms * 8, cnt[kBDeriv]);
    // deliveries: column-ordered (compact nets), ring order (the others),
    // column-staged (nets where it may run)
    size_t smem_o = 0, smem_s = 0, smem_d = 0;
    for (size_t i = 0; i < nn; ++i) {
        const snn_net *n = b->nets[i];
        w[i] = n->dn.ordered_ok ? work(i) : 0.0;
        cap[i] = n->dn.C;
        if (n->dn.ordered_ok) smem_o = std::max(smem_o, ordered_smem_bytes(n->dn.npc, ordered_block(L.deliver_block)));
    }
    b->kind[kBOrdered].block = ordered_block(L.deliver_block);
    b->kind[kBOrdered].smem = smem_o;
    if (smem_o) {
        if (smem_o + 1024 > (size_t)optin) { set_error("batch: ordered delivery needs too much shared memory"); return SNN_EINVAL; }
        SNN_CUDA(cudaFuncSetAttribute(k_deliver_ordered_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_o));
    }
    share_blocks(w, cap, sms * batch_occupancy((const void *)k_deliver_ordered_b, ordered_block(L.deliver_block), smem_o,
                                               L.deliver_blocks_per_sm), cnt[kBOrdered]);
    for (size_t i = 0; i < nn; ++i) {
        const snn_net *n = b->nets[i];
        w[i] = (!n->dn.ordered_ok || n->dn.ring_max_events) ? work(i) : 0.0;
        cap[i] = ((uint64_t)n->N * n->dn.D / 4 + L.deliver_block - 1) / L.deliver_block;
    }
    b->kind[kBRing].block = L.deliver_block;
    share_blocks(w, cap, sms * batch_occupancy((const void *)k_deliver_b, L.deliver_block, 0, L.deliver_blocks_per_sm),
                 cnt[kBRing]);
    for (size_t i = 0; i < nn; ++i) {
        const snn_net *n = b->nets[i];
        w[i] = n->dn.staged_ok ? work(i) : 0.0;
        cap[i] = n->dn.C;
        if (n->dn.staged_ok) smem_s = std::max(smem_s, staged_smem_bytes(n->dn.npc, kStagedBlock));
    }
    b->kind[kBStaged].block = kStagedBlock;
    b->kind[kBStaged].smem = smem_s;
    if (smem_s) {
        if (smem_s + 1024 > (size_t)optin) { set_error("batch: staged delivery needs too much shared memory"); return SNN_EINVAL; }
        SNN_CUDA(cudaFuncSetAttribute(k_deliver_cols_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_s));
    }
    share_blocks(w, cap, sms * batch_occupancy((const void *)k_deliver_cols_b, kStagedBlock, smem_s, 64), cnt[kBStaged]);
    // dense pass (nets where it may run), work units of dense_rows rows
    for (size_t i = 0; i < nn; ++i) {
        const snn_net *n = b->nets[i];
        w[i] = n->dense_ok ? (double)n->S : 0.0;
        cap[i] = (uint64_t)n->dn.C * ((n->dn.npc + n->dn.dense_rows - 1) / std::max(1u, n->dn.dense_rows));
        if (n->dense_ok) smem_d = std::max(smem_d, dense_smem_bytes(n->dn.npc, L.dense_block));
    }
    b->kind[kBDense].block = L.dense_block;
    b->kind[kBDense].smem = smem_d;
    if (smem_d) {
        if (smem_d + 1024 > (size_t)optin) { set_error("batch: dense pass needs too much shared memory"); return SNN_EINVAL; }
        SNN_CUDA(cudaFuncSetAttribute(k_dense_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_d));
    }
    share_blocks(w, cap, sms * batch_occupancy((const void *)k_dense_b, L.dense_block, smem_d, 64), cnt[kBDense]);
    // neuron update and probes: exact block counts
    for (int k : {kBNeuron32, kBNeuron64, kBProbe}) cnt[k].assign(nn, 0);
    for (size_t i = 0; i < nn; ++i) {
        const snn_net *n = b->nets[i];
        const uint32_t nb = (n->N + L.neuron_block * kNeuronsPerThread - 1) / (L.neuron_block * kNeuronsPerThread);
        cnt[n->dn.vd ? kBNeuron64 : kBNeuron32][i] = nb;
        cnt[kBProbe][i] = (n->dn.probe_n + 255) / 256;
    }
    b->kind[kBNeuron32].block = b->kind[kBNeuron64].block = L.neuron_block;
    b->kind[kBProbe].block = 256;
    // one device buffer: DevNet[nn], parity[nn], then per kind first[nn],
    // count[nn] and net_of[grid]
    size_t bytes = ((nn * sizeof(DevNet) + nn + 255) & ~size_t(255));
    size_t off_kind[kBKinds];
    for (int k = 0; k < kBKinds; ++k) {
        uint64_t grid = 0;
        for (uint32_t c : cnt[k]) grid += c;
        if (grid > 0x7fffffffull) { set_error("batch: too many blocks"); return SNN_EINVAL; }
        b->kind[k].grid = (uint32_t)grid;
        off_kind[k] = bytes;
        bytes += ((2 * nn + grid) * 4 + 255) & ~size_t(255);
    }
    std::vector<uint8_t> host(bytes, 0);
    DevNet *hn = reinterpret_cast<DevNet *>(host.data());
    uint8_t *hp = host.data() + nn * sizeof(DevNet);
    for (size_t i = 0; i < nn; ++i) {
        hn[i] = b->nets[i]->dn;
        hp[i] = (uint8_t)(b->nets[i]->t & 1);
    }
    // every net's blocks are contiguous; nets with the most synapses come
    // first, so that the longest work starts first
    std::vector<size_t> order(nn);
    for (size_t i = 0; i < nn; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return work(x) > work(y); });
    for (int k = 0; k < kBKinds; ++k) {
        uint32_t *first = reinterpret_cast<uint32_t *>(host.data() + off_kind[k]);
        uint32_t *count = first + nn;
        uint32_t *net_of = count + nn;
        uint32_t acc = 0;
        for (size_t i : order) {
            first[i] = acc;
            count[i] = cnt[k][i];
            for (uint32_t c = 0; c < cnt[k][i]; ++c) net_of[acc + c] = (uint32_t)i;
            acc += cnt[k][i];
        }
    }
    if (bytes > b->tables_bytes) {
        if (b->tables) cudaFree(b->tables);
        b->tables = nullptr;
        b->tables_bytes = 0;
        cudaError_t e = cudaMalloc(&b->tables, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("batch tables: cudaMalloc(%zu) failed", bytes);
            return SNN_ENOMEM;
        }
        b->tables_bytes = bytes;
    }
    SNN_CUDA(cudaMemcpyAsync(b->tables, host.data(), bytes, cudaMemcpyHostToDevice, b->main));
    SNN_CUDA(cudaStreamSynchronize(b->main));
    uint8_t *base = reinterpret_cast<uint8_t *>(b->tables);
    for (int k = 0; k < kBKinds; ++k) {
        BatchLaunch &bl = b->kind[k].bl;
        bl.nets = reinterpret_cast<const DevNet *>(base);
        bl.parity = base + nn * sizeof(DevNet);
        bl.first = reinterpret_cast<const uint32_t *>(base + off_kind[k]);
        bl.count = bl.first + nn;
        bl.net_of = bl.count + nn;
        bl.k = 0;
    }
    return SNN_OK;
}

// one step (index k of the chunk) of every net: each kind of kernel once
void batch_launch_step(snn_batch *b, uint32_t k)
{
    cudaStream_t s = b->main;
    auto go = [&](int kind, auto kernel) {
        const snn_batch::Kind &x = b->kind[kind];
        if (!x.grid) return;
        BatchLaunch bl = x.bl;
        bl.k = k;
        kernel<<<x.grid, x.block, x.smem, s>>>(bl);
    };
    // [S4(t-1) S5(t-1) S1(t)] then [S2(t) S3(t)], as launch_step
    go(kBLtp, k_ltp_b);
    go(kBFold, k_fold_b);
    go(kBDeriv, k_deriv_b);
    go(kBOrdered, k_deliver_ordered_b);
    go(kBRing, k_deliver_b);
    go(kBStaged, k_deliver_cols_b);
    go(kBDense, k_dense_b);
    go(kBNeuron32, k_neuron_f32_b);
    go(kBNeuron64, k_neuron_f64_b);
    go(kBProbe, k_probe_b);
}

// a chunk of L steps of every net as one graph: per step one launch per kind
// of kernel for the whole batch
int batch_capture(snn_batch *b)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    SNN_TRY(batch_tables(b));
    cudaGraph_t g = nullptr;
    SNN_CUDA(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal));
    for (uint32_t k = 0; k < b->L; ++k) batch_launch_step(b, k);
    cudaError_t e = cudaStreamEndCapture(b->main, &g);
    if (e != cudaSuccess) { set_error("batch capture failed: %s", cudaGetErrorString(e)); return SNN_ECUDA; }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        set_error("batch graph instantiate failed: %s", cudaGetErrorString(e));
        return SNN_ECUDA;
    }
    b->versions.clear();
    b->parity.clear();
    for (snn_net *n : b->nets) {
        b->versions.push_back(n->version);
        b->parity.push_back(n->t & 1);
    }
    return SNN_OK;
}

}  // namespace

int snn_batch_run(snn_batch *b, uint32_t n_ms)
{
    if (!b) { set_error("batch is NULL"); return SNN_EINVAL; }
    if (n_ms == 0) return SNN_OK;
    for (snn_net *n : b->nets) {
        if (n->profile) { set_error("a net of the batch is profiling"); return SNN_ESTATE; }
        if ((int64_t)n->t + n_ms > 0x7fff0000ll) { set_error("time limit reached"); return SNN_ESTATE; }
        SNN_TRY(ensure_raster_steps(n, (int64_t)n->t + n_ms + 2 - n->dn.raster_t0));
        SNN_CUDA(cudaStreamSynchronize(n->stream));
    }
    const uint32_t L = b->L;
    uint32_t left = n_ms;
    while (left > 0) {
        if (L >= 2 && left >= L) {
            // the graph holds each net's launches for its step parity at capture
            bool stale = !b->graph;
            for (size_t i = 0; !stale && i < b->nets.size(); ++i)
                stale = b->versions[i] != b->nets[i]->version || b->parity[i] != (b->nets[i]->t & 1);
            if (stale) SNN_TRY(batch_capture(b));
            SNN_CUDA(cudaGraphLaunch(b->graph, b->main));
            for (snn_net *n : b->nets) n->t += (int32_t)L;
            left -= L;
        } else {
            batch_enqueue(b, 1, true);
            SNN_CUDA(cudaGetLastError());
            for (snn_net *n : b->nets) n->t += 1;
            left -= 1;
        }
    }
    SNN_CUDA(cudaStreamSynchronize(b->main));
    SNN_CUDA(cudaGetLastError());
    int rc = SNN_OK;
    for (snn_net *n : b->nets) {
        n->ltp_owed = true;
        DevCounters hc{};
        SNN_TRY(read_counters_raw(n, &hc));
        if (hc.error && rc == SNN_OK) {
            set_error("device error word %d", hc.error);
            rc = (hc.error == SNN_ETIMEOUT || hc.error == SNN_EBOUNDS) ? hc.error : SNN_ECUDA;
        }
    }
    return rc;
}

int snn_batch_set_launch(snn_batch *b, const snn_launch *launch)
{
    if (!b || !launch) { set_error("NULL argument"); return SNN_EINVAL; }
    snn_launch L = b->launch;
    auto pick = [](uint32_t v, uint32_t cur) { return v ? v : cur; };
    L.deliver_block = pick(launch->deliver_block, L.deliver_block);
    L.deliver_blocks_per_sm = pick(launch->deliver_blocks_per_sm, L.deliver_blocks_per_sm);
    L.neuron_block = pick(launch->neuron_block, L.neuron_block);
    L.ltp_block = pick(launch->ltp_block, L.ltp_block);
    L.ltp_blocks_per_sm = pick(launch->ltp_blocks_per_sm, L.ltp_blocks_per_sm);
    L.deriv_block = pick(launch->deriv_block, L.deriv_block);
    L.dense_block = pick(launch->dense_block, L.dense_block);
    L.graph_steps = pick(launch->graph_steps, L.graph_steps);
    for (uint32_t x : {L.deliver_block, L.neuron_block, L.ltp_block, L.deriv_block, L.dense_block}) {
        if (x < 32 || x > 1024 || x % 32) { set_error("block sizes must be multiples of 32 in 32..1024"); return SNN_EINVAL; }
    }
    if (L.deliver_blocks_per_sm > 64 || L.ltp_blocks_per_sm > 64) { set_error("blocks per SM must be <= 64"); return SNN_EINVAL; }
    if (L.graph_steps < 2) { set_error("a batch needs graph_steps >= 2"); return SNN_EINVAL; }
    b->launch = L;
    b->L = L.graph_steps & ~1u;
    b->launch.graph_steps = b->L;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return SNN_OK;
}

int snn_batch_get_launch(const snn_batch *b, snn_launch *launch)
{
    if (!b || !launch) { set_error("NULL argument"); return SNN_EINVAL; }
    *launch = b->launch;
    return SNN_OK;
}

int snn_batch_autotune(snn_batch *b, uint32_t probe_ms, snn_launch *best)
{
    if (!b) { set_error("batch is NULL"); return SNN_EINVAL; }
    for (snn_net *n : b->nets)
        if (n->explicit_net) { set_error("autotuning restarts the nets: generated nets only"); return SNN_ESTATE; }
    if (probe_ms == 0) probe_ms = 50;
    const snn_launch base = b->launch;
    std::vector<snn_launch> cand;
    for (uint32_t db : {128u, 256u})
        for (uint32_t bps : {4u, 8u})
            for (uint32_t gs : {10u, 50u}) {
                snn_launch c = base;
                c.deliver_block = db;
                c.deliver_blocks_per_sm = bps;
                c.ltp_blocks_per_sm = bps;
                c.graph_steps = gs;
                cand.push_back(c);
            }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SNN_CUDA(cudaEventCreate(&e0));
    SNN_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    size_t best_i = 0;
    int rc = SNN_OK;
    for (size_t i = 0; i < cand.size() && rc == SNN_OK; ++i) {
        if ((rc = snn_batch_set_launch(b, &cand[i])) != SNN_OK) break;
        for (snn_net *n : b->nets)
            if ((rc = snn_reset(n)) != SNN_OK) break;
        if (rc != SNN_OK) break;
        cudaEventRecord(e0, b->main);
        if ((rc = snn_batch_run(b, probe_ms)) != SNN_OK) break;
        cudaEventRecord(e1, b->main);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best_i = i; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SNN_OK) return rc;
    SNN_TRY(snn_batch_set_launch(b, &cand[best_i]));
    for (snn_net *n : b->nets) SNN_TRY(snn_reset(n));
    if (best) *best = b->launch;
    return SNN_OK;
}

int snn_autotune(snn_net *net, uint32_t probe_ms, snn_launch *best)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    if (net->explicit_net) { set_error("autotuning restarts the net: generated nets only"); return SNN_ESTATE; }
    if (probe_ms == 0) probe_ms = 50;
    const snn_launch base = net->launch;
    std::vector<snn_launch> cand;
    const uint32_t rows_opts[] = {0, 64, 256};
    const uint32_t bps_opts[] = {4, 8};
    const uint32_t nb_opts[] = {128, 256};
    const uint32_t gs_opts[] = {10, 50};
    for (uint32_t rows : rows_opts)
        for (uint32_t bps : bps_opts)
            for (uint32_t nb : nb_opts)
                for (uint32_t gs : gs_opts) {
                    snn_launch c = base;
                    c.dense_rows = rows;
                    c.deliver_blocks_per_sm = bps;
                    c.ltp_blocks_per_sm = bps;
                    c.neuron_block = nb;
                    c.graph_steps = gs;
                    cand.push_back(c);
                }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SNN_CUDA(cudaEventCreate(&e0));
    SNN_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    size_t best_i = 0;
    int rc = SNN_OK;
    for (size_t i = 0; i < cand.size() && rc == SNN_OK; ++i) {
        net->launch = cand[i];
        net->dn.dense_min_spikes = dense_threshold(net->N, cand[i].dense_permille);
        if ((rc = setup_dense(net)) != SNN_OK) break;
        if (!net->dense_ok) net->dn.dense_min_spikes = 0xffffffffu;
        drop_graphs(net);
        if ((rc = snn_reset(net)) != SNN_OK) break;
        cudaEventRecord(e0, net->stream);
        if ((rc = run_steps(net, probe_ms)) != SNN_OK) break;
        cudaEventRecord(e1, net->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best_i = i; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SNN_OK) return rc;
    net->launch = cand[best_i];
    net->dn.dense_min_spikes = dense_threshold(net->N, net->launch.dense_permille);
    SNN_TRY(setup_dense(net));
    if (!net->dense_ok) net->dn.dense_min_spikes = 0xffffffffu;
    drop_graphs(net);
    SNN_TRY(snn_reset(net));
    if (best) *best = net->launch;
    return SNN_OK;
}

int snn_reset(snn_net *net)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    if (net->explicit_net) { set_error("explicit nets keep no copy of their initial weights"); return SNN_ESTATE; }
    cudaStream_t s = net->stream;
    const int g = grid_for(net, 8);
    k_reset_weights<<<g, 256, 0, s>>>(net->dn, net->gen.w_exc0, net->gen.w_inh0);
    SNN_CUDA(cudaMemsetAsync(net->dn.sd_rev, 0, (size_t)std::max<int64_t>(net->n_rin, 1) * 4, s));
    k_init_state<<<g, 256, 0, s>>>(net->dn);
    DevCounters hc{};
    hc.raster_first_drop_t = 0x7fffffff;
    hc.ltp_pending = kNoPending;
    SNN_CUDA(cudaMemcpyAsync(net->ctr, &hc, sizeof hc, cudaMemcpyHostToDevice, s));
    SNN_CUDA(cudaMemsetAsync(net->dn.ring_cnt, 0, (size_t)2 * net->cfg.max_delay_ms * 4, s));
    if (net->dn.raster_step_off) SNN_CUDA(cudaMemsetAsync(net->dn.raster_step_off, 0, 8, s));
    SNN_CUDA(cudaGetLastError());
    SNN_CUDA(cudaStreamSynchronize(s));
    net->t = 0;
    net->ltp_owed = false;
    net->dn.raster_t0 = 0;
    net->dn.stim_t0 = net->dn.stim_t1 = 0;
    drop_graphs(net);
    return SNN_OK;
}

int snn_thalamic_events(const snn_config *cfg, int32_t t0, uint32_t n_ms, snn_stimulus *host_events, size_t cap,
                        size_t *n_out)
{
    SNN_TRY(check_config(cfg));
    if (t0 < 0) { set_error("t0 must be >= 0"); return SNN_EINVAL; }
    const uint32_t C = cfg->grid_x * cfg->grid_y, K = cfg->thal_per_col_per_ms, npc = cfg->neurons_per_col;
    const size_t total = (size_t)n_ms * C * K;
    if (n_out) *n_out = total;
    if (total > cap || (!host_events && total)) { set_error("need %zu events", total); return SNN_ETRUNC; }
    const uint32_t k0 = (uint32_t)(cfg->seed & 0xffffffffu), k1 = (uint32_t)(cfg->seed >> 32);
    size_t i = 0;
    for (uint32_t s = 0; s < n_ms; ++s) {
        const uint32_t t = (uint32_t)t0 + s;
        for (uint32_t col = 0; col < C; ++col)
            for (uint32_t k = 0; k < K; ++k) {
                const uint4 r = philox10(make_uint4(t, col, 1u, k), k0, k1);
                host_events[i++] = snn_stimulus{(int32_t)t, (int32_t)(col * npc + draw_below(r.x, npc)),
                                                cfg->thal_amp_q16};
            }
    }
    return SNN_OK;
}

int snn_read_raster(snn_net *net, int32_t t0, int32_t t1, snn_spike *host_buf, size_t cap, size_t *n_out)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    std::vector<snn_spike> out;
    bool trunc = false;
    SNN_TRY(raster_window(net, t0, t1, out, trunc));
    if (n_out) *n_out = out.size();
    const size_t k = std::min(cap, out.size());
    if (k && host_buf) std::memcpy(host_buf, out.data(), k * sizeof(snn_spike));
    if (trunc || out.size() > cap) { set_error("raster window truncated"); return SNN_ETRUNC; }
    return SNN_OK;
}

int snn_raster_reset(snn_net *net)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    return raster_reset_impl(net);
}

int snn_read_synapses(snn_net *net, uint32_t first, uint32_t count, int32_t *host_tgt, uint8_t *host_delay,
                      int32_t *host_w, int32_t *host_sd, size_t cap, size_t *n_out)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    if ((uint64_t)first + count > net->N) { set_error("row range out of bounds"); return SNN_EINVAL; }
    SNN_TRY(flush_owed(net));
    int64_t ro[2];
    SNN_TRY(canon_offset(net, first, &ro[0]));
    SNN_TRY(canon_offset(net, first + count, &ro[1]));
    const int64_t total = ro[1] - ro[0];
    if (n_out) *n_out = (size_t)total;
    if ((size_t)total > cap) { set_error("need %lld entries", (long long)total); return SNN_ETRUNC; }
    if (total == 0) return SNN_OK;
    // chunks of rows of at most ~64 M synapses through device scratch
    const int64_t chunk_syn = 64ll << 20;
    uint32_t r0 = first;
    while (r0 < first + count) {
        // find r1 with row_off[r1] - row_off[r0] <= chunk_syn (rows hold <= 65535)
        uint32_t r1 = std::min<uint32_t>(first + count, r0 + (uint32_t)std::max<int64_t>(1, chunk_syn / 65536));
        int64_t a = 0, b = 0;
        SNN_TRY(canon_offset(net, r0, &a));
        SNN_TRY(canon_offset(net, r1, &b));
        const int64_t n = b - a;
        if (n > 0) {
            int32_t *dt = nullptr, *dw = nullptr, *ds = nullptr;
            uint8_t *dd = nullptr;
            if (host_tgt) SNN_TRY(dalloc_t(net, (size_t)n, &dt));
            if (host_delay) SNN_TRY(dalloc_t(net, (size_t)n, &dd));
            if (host_w) SNN_TRY(dalloc_t(net, (size_t)n, &dw));
            if (host_sd) SNN_TRY(dalloc_t(net, (size_t)n, &ds));
            k_read_rows<<<grid_for(net, 8), 128, 0, net->stream>>>(net->dn, net->gen, net->canon_delay, r0, r1 - r0,
                                                                   a, dt, dd, dw, ds);
            SNN_CUDA(cudaGetLastError());
            const size_t o = (size_t)(a - ro[0]);
            if (dt) SNN_CUDA(cudaMemcpyAsync(host_tgt + o, dt, (size_t)n * 4, cudaMemcpyDeviceToHost, net->stream));
            if (dd) SNN_CUDA(cudaMemcpyAsync(host_delay + o, dd, (size_t)n, cudaMemcpyDeviceToHost, net->stream));
            if (dw) SNN_CUDA(cudaMemcpyAsync(host_w + o, dw, (size_t)n * 4, cudaMemcpyDeviceToHost, net->stream));
            if (ds) SNN_CUDA(cudaMemcpyAsync(host_sd + o, ds, (size_t)n * 4, cudaMemcpyDeviceToHost, net->stream));
            SNN_CUDA(cudaStreamSynchronize(net->stream));
            dfree(net, dt);
            dfree(net, dd);
            dfree(net, dw);
            dfree(net, ds);
        }
        r0 = r1;
    }
    return SNN_OK;
}

int snn_read_synapses_noalloc(snn_net *net, uint32_t first, uint32_t count, int32_t *host_tgt, uint8_t *host_delay,
                              int32_t *host_w, int32_t *host_sd, size_t cap, size_t *n_out)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    if ((uint64_t)first + count > net->N) { set_error("row range out of bounds"); return SNN_EINVAL; }
    int64_t a = 0, b = 0;
    SNN_TRY(canon_offset(net, first, &a));
    SNN_TRY(canon_offset(net, first + count, &b));
    const int64_t total = b - a;
    if (n_out) *n_out = (size_t)total;
    if ((size_t)total > cap) { set_error("need %lld entries", (long long)total); return SNN_ETRUNC; }
    if (total > (int64_t)SNN_NOALLOC_MAX_SYNAPSES) {
        set_error("range holds %lld synapses, more than the %u the no-allocation read can stage; split it",
                  (long long)total, (unsigned)SNN_NOALLOC_MAX_SYNAPSES);
        return SNN_EINVAL;
    }
    if (total == 0) return SNN_OK;
    // device address of the staging array, looked up when the net was set
    // up on its device (with that device current)
    int32_t *base = net->noalloc_base;
    if (!base) { set_error("no staging address for this net's device"); return SNN_ECUDA; }
    SNN_TRY(flush_owed(net));
    const size_t M = SNN_NOALLOC_MAX_SYNAPSES;
    int32_t *dt = host_tgt ? base : nullptr;
    int32_t *dw = host_w ? base + M : nullptr;
    int32_t *ds = host_sd ? base + 2 * M : nullptr;
    uint8_t *dd = host_delay ? reinterpret_cast<uint8_t *>(base + 3 * M) : nullptr;
    // every staged entry of the range is written by the kernel: nothing to clear
    k_read_rows<<<grid_for(net, 8), 128, 0, net->stream>>>(net->dn, net->gen, net->canon_delay, first, count, a,
                                                           dt, dd, dw, ds);
    SNN_CUDA(cudaGetLastError());
    if (dt) SNN_CUDA(cudaMemcpyAsync(host_tgt, dt, (size_t)total * 4, cudaMemcpyDeviceToHost, net->stream));
    if (dd) SNN_CUDA(cudaMemcpyAsync(host_delay, dd, (size_t)total, cudaMemcpyDeviceToHost, net->stream));
    if (dw) SNN_CUDA(cudaMemcpyAsync(host_w, dw, (size_t)total * 4, cudaMemcpyDeviceToHost, net->stream));
    if (ds) SNN_CUDA(cudaMemcpyAsync(host_sd, ds, (size_t)total * 4, cudaMemcpyDeviceToHost, net->stream));
    SNN_CUDA(cudaStreamSynchronize(net->stream));
    return SNN_OK;
}

int snn_read_weights(snn_net *net, int32_t *host_w, int32_t *host_sd, size_t cap, size_t *n_out)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    return snn_read_synapses(net, 0, net->N, nullptr, nullptr, host_w, host_sd, cap, n_out);
}

int snn_read_neurons(snn_net *net, uint32_t first, uint32_t count, float *host_v, float *host_u)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    if ((uint64_t)first + count > net->N) { set_error("neuron range out of bounds"); return SNN_EINVAL; }
    if (net->dn.vd) {
        std::vector<double> tmp((size_t)count);
        const double *src[2] = {net->dn.vd + first, net->dn.ud + first};
        float *dst[2] = {host_v, host_u};
        for (int k = 0; k < 2; ++k) {
            if (!dst[k]) continue;
            SNN_CUDA(cudaMemcpyAsync(tmp.data(), src[k], (size_t)count * 8, cudaMemcpyDeviceToHost, net->stream));
            SNN_CUDA(cudaStreamSynchronize(net->stream));
            for (uint32_t i = 0; i < count; ++i) dst[k][i] = (float)tmp[i];
        }
        return SNN_OK;
    }
    if (host_v) SNN_CUDA(cudaMemcpyAsync(host_v, net->dn.v + first, (size_t)count * 4, cudaMemcpyDeviceToHost, net->stream));
    if (host_u) SNN_CUDA(cudaMemcpyAsync(host_u, net->dn.u + first, (size_t)count * 4, cudaMemcpyDeviceToHost, net->stream));
    SNN_CUDA(cudaStreamSynchronize(net->stream));
    return SNN_OK;
}

int snn_read_neurons_f64(snn_net *net, uint32_t first, uint32_t count, double *host_v, double *host_u)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    if ((uint64_t)first + count > net->N) { set_error("neuron range out of bounds"); return SNN_EINVAL; }
    if (net->dn.vd) {
        if (host_v) SNN_CUDA(cudaMemcpyAsync(host_v, net->dn.vd + first, (size_t)count * 8, cudaMemcpyDeviceToHost, net->stream));
        if (host_u) SNN_CUDA(cudaMemcpyAsync(host_u, net->dn.ud + first, (size_t)count * 8, cudaMemcpyDeviceToHost, net->stream));
        SNN_CUDA(cudaStreamSynchronize(net->stream));
        return SNN_OK;
    }
    std::vector<float> tmp((size_t)count);
    const float *src[2] = {net->dn.v + first, net->dn.u + first};
    double *dst[2] = {host_v, host_u};
    for (int k = 0; k < 2; ++k) {
        if (!dst[k]) continue;
        SNN_CUDA(cudaMemcpyAsync(tmp.data(), src[k], (size_t)count * 4, cudaMemcpyDeviceToHost, net->stream));
        SNN_CUDA(cudaStreamSynchronize(net->stream));
        for (uint32_t i = 0; i < count; ++i) dst[k][i] = tmp[i];
    }
    return SNN_OK;
}

int snn_set_probe(snn_net *net, const int32_t *host_gids, uint32_t n, uint32_t max_steps)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    DevNet &dn = net->dn;
    dfree(net, (void *)dn.probe_gid);
    dfree(net, dn.probe_v);
    dfree(net, dn.probe_u);
    dn.probe_gid = nullptr;
    dn.probe_v = dn.probe_u = nullptr;
    dn.probe_n = dn.probe_cap = 0;
    drop_graphs(net);
    if (n == 0 || max_steps == 0) return SNN_OK;
    if (!host_gids) { set_error("gids are NULL"); return SNN_EINVAL; }
    for (uint32_t k = 0; k < n; ++k)
        if (host_gids[k] < 0 || (uint32_t)host_gids[k] >= net->N) { set_error("probe gid %d out of range", host_gids[k]); return SNN_EINVAL; }
    int32_t *g = nullptr;
    float *pv = nullptr, *pu = nullptr;
    SNN_TRY(dalloc_t(net, n, &g));
    SNN_TRY(dalloc_t(net, (size_t)n * max_steps, &pv));
    SNN_TRY(dalloc_t(net, (size_t)n * max_steps, &pu));
    SNN_CUDA(cudaMemcpyAsync(g, host_gids, (size_t)n * 4, cudaMemcpyHostToDevice, net->stream));
    SNN_CUDA(cudaStreamSynchronize(net->stream));
    dn.probe_gid = g;
    dn.probe_v = pv;
    dn.probe_u = pu;
    dn.probe_n = n;
    dn.probe_cap = max_steps;
    dn.probe_t0 = net->t;
    return SNN_OK;
}

int snn_read_probe(snn_net *net, float *host_v, float *host_u, size_t cap, uint32_t *steps)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    const DevNet &dn = net->dn;
    const uint32_t rec = dn.probe_n ? (uint32_t)std::min<int64_t>(dn.probe_cap, std::max(0, net->t - dn.probe_t0)) : 0;
    if (steps) *steps = rec;
    const size_t need = (size_t)rec * dn.probe_n;
    if (need > cap && (host_v || host_u)) { set_error("need %zu values", need); return SNN_ETRUNC; }
    if (need == 0) return SNN_OK;
    if (host_v) SNN_CUDA(cudaMemcpyAsync(host_v, dn.probe_v, need * 4, cudaMemcpyDeviceToHost, net->stream));
    if (host_u) SNN_CUDA(cudaMemcpyAsync(host_u, dn.probe_u, need * 4, cudaMemcpyDeviceToHost, net->stream));
    SNN_CUDA(cudaStreamSynchronize(net->stream));
    return SNN_OK;
}

int snn_read_counters(snn_net *net, snn_counters *out)
{
    if (!net || !out) { set_error("NULL argument"); return SNN_EINVAL; }
    DevCounters hc{};
    SNN_TRY(read_counters_raw(net, &hc));
    out->t = net->t;
    out->spikes = (int64_t)hc.spikes;
    out->e_all = (int64_t)hc.e_all;
    out->e_exc = (int64_t)hc.e_exc;
    out->l_exc = (int64_t)hc.l_exc;
    out->raster_kept = (int64_t)hc.raster_total;
    out->raster_dropped = (int64_t)hc.raster_dropped;
    out->error = hc.error;
    out->reserved = 0;
    return SNN_OK;
}

int snn_net_info(const snn_net *net, uint32_t *n_neurons, int64_t *n_synapses, size_t *device_bytes)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    if (n_neurons) *n_neurons = net->N;
    if (n_synapses) *n_synapses = net->S;
    if (device_bytes) *device_bytes = net->bytes_held;
    return SNN_OK;
}

int snn_set_profile(snn_net *net, int on)
{
    if (!net) { set_error("net is NULL"); return SNN_EINVAL; }
    net->profile = on != 0;
    for (int k = 0; k < kKinds; ++k) { net->prof_ms[k] = 0; net->prof_n[k] = 0; }
    net->prof_kernels = 0;
    net->ev_used = 0;
    return SNN_OK;
}

int snn_read_profile(snn_net *net, snn_profile *out)
{
    if (!net || !out) { set_error("NULL argument"); return SNN_EINVAL; }
    for (int k = 0; k < kKinds; ++k) {
        out->launches[k] = net->prof_n[k];
        out->ms[k] = net->prof_ms[k];
    }
    out->kernels = net->prof_kernels;
    DevCounters hc{};
    SNN_TRY(read_counters_raw(net, &hc));
    out->dense_steps = (int64_t)hc.dense_steps;
    out->dense_deriv_steps = (int64_t)hc.dense_deriv_steps;
    out->dense_events = (int64_t)hc.dense_e_all;
    out->dense_exc_events = (int64_t)hc.dense_e_exc;
    out->dense_ltp_visits = (int64_t)hc.dense_l_exc;
    return SNN_OK;
}

// checkpoint layout: header, then the arrays in the order listed below
struct StateHeader {
    uint32_t magic, version;
    uint32_t N, D;
    int64_t S;
    int32_t t, raster_t0;
    snn_config cfg;
};

int snn_save_state(snn_net *net, void *host_buf, size_t cap, size_t *n)
{
    if (!net || !n) { set_error("NULL argument"); return SNN_EINVAL; }
    const size_t N = net->N, D = net->cfg.max_delay_ms, S = (size_t)net->S_store;
    const size_t fsz = net->dn.vd ? 8 : 4;      // v and u in double for SNN_FP64 nets
    const size_t need = sizeof(StateHeader) + N * (16 + 2 * fsz) + D * N * 4 + D * 8 + S * 8 + sizeof(DevCounters);
    *n = need;
    if (!host_buf) return SNN_OK;
    SNN_TRY(flush_owed(net));
    if (cap < need) { set_error("checkpoint needs %zu bytes", need); return SNN_ETRUNC; }
    char *p = (char *)host_buf;
    StateHeader h{};
    h.magic = kStateMagic;
    h.version = 1;
    h.N = net->N;
    h.D = (uint32_t)D;
    h.S = net->S;
    h.t = net->t;
    h.raster_t0 = net->t;
    h.cfg = net->cfg;
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    cudaStream_t s = net->stream;
    const DevNet &dn = net->dn;
    const void *sv = dn.vd ? (const void *)dn.vd : (const void *)dn.v;
    const void *su = dn.ud ? (const void *)dn.ud : (const void *)dn.u;
    const void *src[] = {sv, su, dn.I, dn.hl, dn.last_spike, dn.ring_ids, dn.ring_cnt, net->w, net->sd, net->ctr};
    const size_t len[] = {N * fsz, N * fsz, N * 4, N * 8, N * 4, D * N * 4, D * 8, S * 4, S * 4, sizeof(DevCounters)};
    for (int k = 0; k < 10; ++k) {
        if (len[k]) SNN_CUDA(cudaMemcpyAsync(p, src[k], len[k], cudaMemcpyDeviceToHost, s));
        p += len[k];
    }
    SNN_CUDA(cudaStreamSynchronize(s));
    return SNN_OK;
}

int snn_load_state(snn_net *net, const void *host_buf, size_t n)
{
    if (!net || !host_buf) { set_error("NULL argument"); return SNN_EINVAL; }
    const size_t N = net->N, D = net->cfg.max_delay_ms, S = (size_t)net->S_store;
    const size_t fsz = net->dn.vd ? 8 : 4;
    const size_t need = sizeof(StateHeader) + N * (16 + 2 * fsz) + D * N * 4 + D * 8 + S * 8 + sizeof(DevCounters);
    if (n < need) { set_error("checkpoint is %zu bytes, need %zu", n, need); return SNN_EINVAL; }
    StateHeader h{};
    std::memcpy(&h, host_buf, sizeof h);
    if (h.magic != kStateMagic || h.version != 1 || h.N != net->N || h.D != D || h.S != net->S ||
        std::memcmp(&h.cfg, &net->cfg, sizeof(snn_config)) != 0) {
        set_error("checkpoint does not belong to a net of this configuration");
        return SNN_EINVAL;
    }
    const char *p = (const char *)host_buf + sizeof h;
    if (!net->explicit_net) {
        // inhibitory synapses are not plastic: a checkpoint of this net keeps
        // their weight, and the dense pass relies on it
        const char *wb = p + N * (16 + 2 * fsz) + D * N * 4 + D * 8;
        const size_t stride = net->dn.uniform_m, m = net->dn.canon_m, npc = net->cfg.neurons_per_col;
        for (size_t q = 0; q < N; ++q) {
            if (q % npc < net->cfg.exc_per_col) continue;
            for (size_t j = 0; j < m; ++j) {
                int32_t w;
                std::memcpy(&w, wb + (q * stride + j) * 4, 4);
                if (w != net->dn.w_inh) {
                    set_error("checkpoint changes the weight of inhibitory synapse %zu of neuron %zu, "
                              "which is not plastic", j, q);
                    return SNN_EINVAL;
                }
            }
        }
    }
    cudaStream_t s = net->stream;
    DevNet &dn = net->dn;
    void *sv = dn.vd ? (void *)dn.vd : (void *)dn.v;
    void *su = dn.ud ? (void *)dn.ud : (void *)dn.u;
    void *dst[] = {sv, su, dn.I, dn.hl, dn.last_spike, dn.ring_ids, dn.ring_cnt, net->w, net->sd, net->ctr};
    const size_t len[] = {N * fsz, N * fsz, N * 4, N * 8, N * 4, D * N * 4, D * 8, S * 4, S * 4, sizeof(DevCounters)};
    for (int k = 0; k < 10; ++k) {
        if (len[k]) SNN_CUDA(cudaMemcpyAsync(dst[k], p, len[k], cudaMemcpyHostToDevice, s));
        p += len[k];
    }
    SNN_CUDA(cudaStreamSynchronize(s));
    SNN_CUDA(cudaMemsetAsync(dn.sd_rev, 0, (size_t)std::max<int64_t>(net->n_rin, 1) * 4, s));
    net->t = h.t;
    net->ltp_owed = false;
    // the raster restarts at the checkpoint's step
    DevCounters hc{};
    std::memcpy(&hc, (const char *)host_buf + need - sizeof(DevCounters), sizeof hc);
    hc.raster_total = 0;
    hc.raster_dropped = 0;
    hc.raster_first_drop_t = 0x7fffffff;
    hc.t_slot[h.t & 1] = h.t;
    hc.ltp_pending = kNoPending;
    hc.done_blocks = 0;
    hc.dense_cursor = 0;
    hc.staged_cursor = 0;
    hc.fold_cursor = 0;
    SNN_CUDA(cudaMemcpyAsync(net->ctr, &hc, sizeof hc, cudaMemcpyHostToDevice, s));
    if (dn.raster_step_off) SNN_CUDA(cudaMemsetAsync(dn.raster_step_off, 0, 8, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    dn.raster_t0 = h.t;
    drop_graphs(net);
    return SNN_OK;
}

}  // extern "C"
