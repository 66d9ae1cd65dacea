// C ABI of the GS-NFS GB300 codec: context and scratch arena, stream-ordered
// orchestration of the encode / decode kernels, and the bitstream container
// (header of Algorithm 1 plus this codec's own section layout).
//
// Container (little endian, every section 8-aligned):
//   header 96 B: u32 magic "GSN1", u32 version 1, u32 header_bytes, u32 J,
//     u32 C, u32 G, u64 N_v, f64 lo[3], f64 ext, f64 tau,
//     u64 occupancy_section_bytes, u64 attribute_section_bytes, u32 flags,
//     u32 reserved; then u32 level_size[J+1], u8 group[C], pad to 8,
//     f64 step[G].
//   occupancy section: u64 n_occ, u32 mode, u32 aux; mode 0 raw bytes,
//     mode 2 one constant byte (aux), mode 1 rANS: aux = chunks, u32 chunk
//     symbols, u32 0, u16 freq[256], u32 chunk_bytes[], pad 8, chunks
//     (32 u32 states + u16 words, padded to 4); rANS only when smaller.
//   attribute section (C > 0 and N_v > 0): u32 B, u32 nb, u32
//     block_words[nb*C] (block-major: b*C + c), payload words, pad 8.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gsnfs.h"
#include "kernels.cuh"
#include "status.cuh"

using namespace gsnfs;

// ---------------------------------------------------- launches / profiling
namespace {
std::atomic<uint64_t> g_launches{0};
struct Profiler {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> pool;
    struct Rec {
        int id;
        cudaEvent_t a, b;
    };
    std::vector<Rec> open[kStCount];
    std::vector<Rec> done;
    double ms[kStCount] = {};
    uint64_t cnt[kStCount] = {};
    cudaEvent_t get()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};
Profiler g_prof;
const char *kStageNames[kStCount] = {"voxelize", "sort", "dedup", "occupancy", "rans", "raht_prelude", "raht_forward",
                                     "raht_forward_pass0", "rlgr_encode", "container", "reconstruction",
                                     "occupancy_decode", "octree_decode", "rlgr_decode", "raht_inverse",
                                     "raht_inverse_pass0"};
}  // namespace

// While a call is being captured into a CUDA graph, its launches are counted
// into the graph (and added to the total at every replay), and its stage
// events become event-record nodes of the graph (events of their own, read
// after every replay while profiling is on).
thread_local uint64_t *t_capture_launches = nullptr;
thread_local std::vector<Profiler::Rec> *t_capture_stages = nullptr;
thread_local std::vector<Profiler::Rec> t_capture_open;

namespace gsnfs {
void count_launch()
{
    if (t_capture_launches)
        ++*t_capture_launches;
    else
        g_launches.fetch_add(1, std::memory_order_relaxed);
}
void stage_begin(cudaStream_t s, int id)
{
    if (t_capture_stages) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) == cudaSuccess && cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) == cudaSuccess)
            t_capture_open.push_back({id, e, nullptr});
        else if (e)
            cudaEventDestroy(e);
        return;
    }
    if (!g_prof.on || t_capture_launches) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    cudaEvent_t e = g_prof.get();
    cudaEventRecord(e, s);
    g_prof.open[id].push_back({id, e, nullptr});
}
void stage_end(cudaStream_t s, int id)
{
    if (t_capture_stages) {
        for (size_t k = t_capture_open.size(); k-- > 0;) {
            if (t_capture_open[k].id != id) continue;
            Profiler::Rec r = t_capture_open[k];
            t_capture_open.erase(t_capture_open.begin() + (long)k);
            if (cudaEventCreate(&r.b) == cudaSuccess &&
                cudaEventRecordWithFlags(r.b, s, cudaEventRecordExternal) == cudaSuccess) {
                t_capture_stages->push_back(r);
            } else {
                cudaEventDestroy(r.a);
                if (r.b) cudaEventDestroy(r.b);
            }
            break;
        }
        return;
    }
    if (!g_prof.on || t_capture_launches) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (g_prof.open[id].empty()) return;
    auto r = g_prof.open[id].back();
    g_prof.open[id].pop_back();
    r.b = g_prof.get();
    cudaEventRecord(r.b, s);
    g_prof.done.push_back(r);
}
}  // namespace gsnfs

// One captured encode: the request's shape and buffers (key) and the
// instantiated graph that replays its device work.
struct GraphEntry {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches = 0;  // kernels in the graph
    uint64_t last_use = 0;
    std::vector<Profiler::Rec> stages;  // stage events recorded by the graph (owned)
};

void destroy_graph(GraphEntry &g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    for (auto &r : g.stages) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g.stages.clear();
}

// After a replay has completed: its stage times, while profiling is on.
void add_graph_stage_times(const std::vector<Profiler::Rec> &stages)
{
    if (!g_prof.on) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (const auto &r : stages) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            g_prof.ms[r.id] += t;
            g_prof.cnt[r.id] += 1;
        }
    }
}

struct gsnfs_ctx {
    int device = 0;
    int num_sms = 0;
    void *arena = nullptr;
    size_t arena_cap = 0;
    unsigned char *pinned = nullptr;
    size_t pinned_cap = 0;
    DevState *st = nullptr;
    // launch-shape tunables (gsnfs_tune_set); 0 = built-in default
    uint32_t tune[4] = {0, 0, 0, 0};
    // level-of-detail scratch (full-depth attributes, node index), grown on demand
    void *lod = nullptr;
    size_t lod_cap = 0;
    // splat-rasteriser scratch: per-Gaussian arrays and the per-tile key lists, grown on demand
    void *rnd = nullptr, *rkeys = nullptr;
    size_t rnd_cap = 0, rkeys_cap = 0;
    cudaEvent_t ev_join = nullptr;  // stream_wait
    // high-priority side stream: the longer branch of a batched call, so that CTAs of the shorter branch
    // (on the caller's stream) take the SMs that branch leaves idle instead of delaying it
    cudaStream_t aux_hi = nullptr;
    cudaEvent_t ev_fork_hi = nullptr, ev_join_hi = nullptr;
    // CUDA graphs of the encoder (off by default)
    bool graphs = false;
    cudaStream_t gstream = nullptr;  // capture / replay stream, joined to the caller's by events
    cudaEvent_t gev_in = nullptr, gev_out = nullptr;
    std::vector<GraphEntry> gcache;
    uint64_t gtick = 0, ghits = 0, gcaptures = 0, gfailures = 0;
    // pinned staging of the asynchronous decoder: a ring of slots, each free once its event has completed
    unsigned char *aring[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t aring_cap[4] = {0, 0, 0, 0};
    cudaEvent_t aring_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    uint32_t aring_next = 0;
};

struct gsnfs_raht_plan {
    gsnfs_ctx *ctx = nullptr;
    void *mem = nullptr;
    RahtPlanDev dev{};
    float *pool = nullptr;
    float *qparams = nullptr;  // inv_step[C], step[C]
    double *pool64 = nullptr;  // survivor rows of the FP64 transforms (allocated on first use)
    double *qparams64 = nullptr;
    uint64_t surv_rows = 0;
    DevState *st = nullptr;
    uint64_t nv = 0;
    uint32_t C = 0, J = 0;
};

namespace {

const uint32_t kMagic = 0x314E5347u;
thread_local char g_last_error[256];

#define CK(x)                                                                          \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            snprintf(g_last_error, sizeof(g_last_error), "%s: %s", #x, cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? GSNFS_ERR_OOM : GSNFS_ERR_CUDA;   \
        }                                                                              \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d)
    {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard()
    {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Sub-allocator over one buffer: the first pass (base == nullptr) measures.
struct Carve {
    unsigned char *base;
    size_t off = 0;
    explicit Carve(void *b) : base((unsigned char *)b) {}
    template <typename T>
    T *take(uint64_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += (size_t)count * sizeof(T) + 16;
        return p;
    }
};

// Captured graphs hold arena and staging addresses: drop them when either moves.
void drop_graphs(gsnfs_ctx *ctx)
{
    for (auto &g : ctx->gcache) destroy_graph(g);
    ctx->gcache.clear();
}

gsnfs_status grow_arena(gsnfs_ctx *ctx, size_t need, cudaStream_t s)
{
    if (need <= ctx->arena_cap) return GSNFS_OK;
    CK(cudaStreamSynchronize(s));
    if (ctx->gstream) CK(cudaStreamSynchronize(ctx->gstream));
    drop_graphs(ctx);
    if (ctx->arena) CK(cudaFree(ctx->arena));
    ctx->arena = nullptr;
    ctx->arena_cap = 0;
    size_t cap = need + need / 8 + (64 << 20);
    CK(cudaMalloc(&ctx->arena, cap));
    ctx->arena_cap = cap;
    return GSNFS_OK;
}

gsnfs_status grow_pinned(gsnfs_ctx *ctx, size_t need)
{
    if (need <= ctx->pinned_cap) return GSNFS_OK;
    if (ctx->gstream) CK(cudaStreamSynchronize(ctx->gstream));
    drop_graphs(ctx);
    if (ctx->pinned) CK(cudaFreeHost(ctx->pinned));
    ctx->pinned = nullptr;
    size_t cap = need + (1 << 16);
    CK(cudaMallocHost((void **)&ctx->pinned, cap));
    ctx->pinned_cap = cap;
    return GSNFS_OK;
}

// Independent branches of one call: the work enqueued on the context's
// high-priority stream between fork_hi_begin and fork_hi_end starts after
// everything already on s, and s continues only after it (events also order
// captured graph nodes).  The block scheduler starts pending CTAs of a
// higher-priority stream first, so the longer branch goes there.
gsnfs_status fork_hi_begin(gsnfs_ctx *ctx, cudaStream_t s, cudaStream_t *hi)
{
    if (!ctx->aux_hi) {
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CK(cudaStreamCreateWithPriority(&ctx->aux_hi, cudaStreamNonBlocking, greatest));
        CK(cudaEventCreateWithFlags(&ctx->ev_fork_hi, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_join_hi, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(ctx->ev_fork_hi, s));
    CK(cudaStreamWaitEvent(ctx->aux_hi, ctx->ev_fork_hi, 0));
    *hi = ctx->aux_hi;
    return GSNFS_OK;
}

gsnfs_status fork_hi_end(gsnfs_ctx *ctx, cudaStream_t s)
{
    CK(cudaEventRecord(ctx->ev_join_hi, ctx->aux_hi));
    CK(cudaStreamWaitEvent(s, ctx->ev_join_hi, 0));
    return GSNFS_OK;
}

// Work on `waiter` enqueued from now on runs after everything enqueued on `from` so far.
gsnfs_status stream_wait(gsnfs_ctx *ctx, cudaStream_t waiter, cudaStream_t from)
{
    if (!ctx->ev_join) CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    CK(cudaEventRecord(ctx->ev_join, from));
    CK(cudaStreamWaitEvent(waiter, ctx->ev_join, 0));
    return GSNFS_OK;
}

// Small transfers between the pinned staging buffer and the device (a call's
// parameters and results) run as a kernel over the staging buffer's unified
// address instead of on the copy engines, so they never queue behind a
// caller's bulk copies in flight on other streams.
__global__ void stage_copy_kernel(unsigned char *dst, const unsigned char *src, uint64_t n)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    if ((((uintptr_t)dst | (uintptr_t)src | n) & 3) == 0) {
        uint32_t *d = reinterpret_cast<uint32_t *>(dst);
        const uint32_t *q = reinterpret_cast<const uint32_t *>(src);
        for (uint64_t i = t; i < n / 4; i += nt) d[i] = q[i];
    } else {
        for (uint64_t i = t; i < n; i += nt) dst[i] = src[i];
    }
}

cudaError_t stage_copy(void *dst, const void *src, size_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint64_t words = (n + 3) / 4;
    const uint32_t blocks = (uint32_t)std::min<uint64_t>((words + 255) / 256, 128);
    stage_copy_kernel<<<blocks, 256, 0, s>>>(static_cast<unsigned char *>(dst), static_cast<const unsigned char *>(src),
                                             n);
    count_launch();
    return cudaGetLastError();
}

__host__ __device__ inline uint64_t pad8(uint64_t x) { return (x + 7) & ~7ull; }

// the KLT matrices of the colour mode follow the steps: three f32 15 x 15 (Sec. 4)
__host__ __device__ inline uint64_t klt_bytes_padded() { return pad8(4ull * (uint64_t)kKltFloats); }
__host__ __device__ inline uint64_t header_bytes(uint32_t J, uint32_t C, uint32_t G, uint32_t color)
{
    return pad8(96 + 4ull * (J + 1) + C) + 8ull * G + (color ? klt_bytes_padded() : 0);
}

uint64_t occ_bound(uint64_t n, uint32_t J)
{
    uint64_t t = 0, p = 1;
    for (uint32_t d = 0; d < J; ++d) {
        t += std::min<uint64_t>(p, n);
        if (p < (1ull << 60)) p *= 8;
    }
    return t;
}

bool pow2(uint32_t x) { return x && !(x & (x - 1)); }

gsnfs_status check_quant(const gsnfs_quant *q)
{
    if (!q) return GSNFS_ERR_INVALID_ARG;
    if (q->num_channels > (uint32_t)kMaxC) return GSNFS_ERR_INVALID_ARG;
    if (q->rans_chunk < 32 || q->rans_chunk > (1u << 20) || (q->rans_chunk % 32)) return GSNFS_ERR_INVALID_ARG;
    if (q->num_channels == 0) return GSNFS_OK;
    if (q->num_groups < 1 || q->num_groups > 255 || !q->channel_group || !q->steps) return GSNFS_ERR_INVALID_ARG;
    if (!pow2(q->rlgr_block) || q->rlgr_block < 32 || q->rlgr_block > 65536) return GSNFS_ERR_INVALID_ARG;
    if (!(q->tau > 0.0 && q->tau <= 0.5)) return GSNFS_ERR_INVALID_ARG;
    if (q->color > 1 || (q->color && q->num_channels != 56)) return GSNFS_ERR_INVALID_ARG;
    for (uint32_t c = 0; c < q->num_channels; ++c)
        if (q->channel_group[c] >= q->num_groups) return GSNFS_ERR_INVALID_ARG;
    for (uint32_t g = 0; g < q->num_groups; ++g)
        if (!(q->steps[g] > 0.0) || !std::isfinite(q->steps[g])) return GSNFS_ERR_INVALID_ARG;
    return GSNFS_OK;
}

// ------------------------------------------------------ container kernels ---
struct StreamInfo {
    uint64_t off, hb, occ, attr;
};

// Header records of every stream, for a decoder that is given them instead of
// reading them back (GSNFS_HEADER_RECORD_BYTES each): the stream's header
// tables at 0, the first 24 bytes of its occupancy section at 4096 and the
// first 8 of its attribute section at 4160.  One CTA per stream.
// A record assembled in shared memory goes to the (pinned host) destination in
// 16-byte stores: byte stores to host memory would each cross the link alone.
static_assert(GSNFS_HEADER_RECORD_BYTES % 16 == 0, "records are copied in 16-byte words");
__device__ __forceinline__ void copy_record_out(uint8_t *r, const uint8_t *sr)
{
    uint4 *d = reinterpret_cast<uint4 *>(r);  // records start 16-byte aligned (4,224 = 264 x 16)
    const uint4 *q = reinterpret_cast<const uint4 *>(sr);
    for (uint32_t k = threadIdx.x; k < GSNFS_HEADER_RECORD_BYTES / 16; k += blockDim.x) d[k] = q[k];
}

__global__ void header_records_kernel(const uint8_t *out, const StreamInfo *si, uint32_t n, uint8_t *rec)
{
    const uint32_t i = blockIdx.x;
    if (i >= n) return;
    const StreamInfo x = si[i];
    uint8_t *r = rec + (uint64_t)i * GSNFS_HEADER_RECORD_BYTES;
    const uint8_t *b = out + x.off;
    const uint32_t hb = x.hb < 4096 ? (uint32_t)x.hb : 4096u;
    __shared__ __align__(16) uint8_t sr[GSNFS_HEADER_RECORD_BYTES];
    for (uint32_t k = threadIdx.x; k < GSNFS_HEADER_RECORD_BYTES; k += blockDim.x) {  // every byte: zeros elsewhere
        uint8_t v = 0;
        if (k < hb)
            v = b[k];
        else if (k >= 4096 && k < 4096 + 24 && k - 4096 < x.occ + x.attr)
            v = b[x.hb + (k - 4096)];
        else if (k >= 4160 && k < 4168 && x.attr >= 8)
            v = b[x.hb + x.occ + (k - 4160)];
        sr[k] = v;
    }
    __syncthreads();
    copy_record_out(r, sr);
}

// The same records read out of the streams themselves (a decoder not given
// them): frame f0 + i of a launch is CTA i, its stream at in + off[i] of
// off[i + 1] - off[i] bytes; record at rec + (f0 + i) * stride.  The section
// sizes come from the stream's fixed header; nothing outside the stream is
// read (a stream too short for its header gives a record the host rejects).
constexpr uint32_t kRecFrames = 64;
struct RecLaunch {
    const uint8_t *in;
    uint8_t *rec;
    uint64_t stride;
    uint32_t f0;
    uint64_t off[kRecFrames + 1];
};

__device__ __forceinline__ uint64_t rd_le(const uint8_t *p, int n)
{
    uint64_t v = 0;
    for (int k = n - 1; k >= 0; --k) v = (v << 8) | p[k];
    return v;
}

__global__ void stream_records_kernel(RecLaunch a)
{
    const uint32_t i = blockIdx.x;
    const uint64_t o = a.off[i], bytes = a.off[i + 1] - o;
    const uint8_t *b = a.in + o;
    uint8_t *r = a.rec + (uint64_t)(a.f0 + i) * a.stride;
    uint64_t hb = 0, occ = 0, attr = 0;
    if (bytes >= 96) {
        hb = rd_le(b + 8, 4);
        occ = rd_le(b + 72, 8);
        attr = rd_le(b + 80, 8);
    }
    const uint64_t nh = bytes < 96 ? bytes : (hb < 96 ? 96 : (hb > 4096 ? 4096 : hb));
    const bool heads = bytes >= 96 && hb <= 4096 && hb < bytes;
    __shared__ __align__(16) uint8_t sr[GSNFS_HEADER_RECORD_BYTES];
    for (uint32_t k = threadIdx.x; k < GSNFS_HEADER_RECORD_BYTES; k += blockDim.x) {  // every byte: zeros elsewhere
        uint8_t v = 0;
        if (k < nh && k < bytes)
            v = b[k];
        else if (heads && k >= 4096 && k < 4096 + 24 && hb + (k - 4096) < bytes)
            v = b[hb + (k - 4096)];
        else if (heads && k >= 4160 && k < 4168 && attr >= 8 && occ < bytes && hb + occ + (k - 4160) < bytes)
            v = b[hb + occ + (k - 4160)];
        sr[k] = v;
    }
    __syncthreads();
    copy_record_out(r, sr);
}

struct HdrParams {
    uint32_t F, R, C, G, B, chunk, color;
    double tau;
    uint64_t capacity;
};

__device__ __forceinline__ void wr32(uint8_t *p, uint32_t v)
{
    for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
__device__ __forceinline__ void wr64(uint8_t *p, uint64_t v)
{
    for (int i = 0; i < 8; ++i) p[i] = (uint8_t)(v >> (8 * i));
}

__global__ void sizes_kernel(HdrParams hp, const uint32_t *J, const uint32_t *vstart, const uint64_t *sec_bytes,
                             const uint64_t *blk_off, const uint64_t *block_off, StreamInfo *si, DevState *st)
{
    if (threadIdx.x != 0) return;
    uint64_t run = 0;
    for (uint32_t f = 0; f < hp.F; ++f) {
        const uint64_t nv = vstart[f + 1] - vstart[f];
        const uint64_t nb = (nv + hp.B - 1) / hp.B;
        for (uint32_t r = 0; r < hp.R; ++r) {
            StreamInfo x;
            x.hb = header_bytes(J[f], hp.C, hp.C ? hp.G : 0, hp.color);
            x.occ = sec_bytes[f];
            x.attr = 0;
            if (hp.C && nv) {
                const uint64_t b0 = blk_off[f] + (uint64_t)r * hp.C * nb;
                const uint64_t words = block_off[b0 + hp.C * nb] - block_off[b0];
                x.attr = pad8(8 + 4 * hp.C * nb + 4 * words);
            }
            x.off = run;
            run += x.hb + x.occ + x.attr;
            si[f * hp.R + r] = x;
        }
    }
    si[hp.F * hp.R].off = run;
    st->total_bytes = run;
    if (run > hp.capacity) set_error(&st->err, kErrCapacity);
}

__global__ void header_kernel(HdrParams hp, const uint32_t *J, const uint32_t *vstart, const FrameGrid *grid,
                              const uint32_t *lsz, const uint8_t *groups, const double *steps_rg,
                              const float *klt, const StreamInfo *si, const DevState *st, uint8_t *out)
{
    if (st->total_bytes > hp.capacity) return;
    const uint32_t s = blockIdx.x, f = s / hp.R, r = s % hp.R;
    const StreamInfo x = si[s];
    uint8_t *h = out + x.off;
    const uint32_t Jf = J[f];
    const uint32_t G = hp.C ? hp.G : 0;
    for (uint32_t i = threadIdx.x; i < x.hb; i += blockDim.x) h[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        wr32(h + 0, kMagic);
        wr32(h + 4, 1);
        wr32(h + 8, (uint32_t)x.hb);
        wr32(h + 12, Jf);
        wr32(h + 16, hp.C);
        wr32(h + 20, G);
        wr64(h + 24, vstart[f + 1] - vstart[f]);
        const FrameGrid g = grid[f];
        for (int a = 0; a < 3; ++a) wr64(h + 32 + 8 * a, (uint64_t)__double_as_longlong(g.lo[a]));
        wr64(h + 56, (uint64_t)__double_as_longlong(g.ext));
        wr64(h + 64, (uint64_t)__double_as_longlong(hp.tau));
        wr64(h + 72, x.occ);
        wr64(h + 80, x.attr);
        wr32(h + 88, hp.color);  // flags bit 0: colour decorrelation
    }
    for (uint32_t d = threadIdx.x; d <= Jf; d += blockDim.x) wr32(h + 96 + 4 * d, lsz[f * 22 + d]);
    for (uint32_t c = threadIdx.x; c < hp.C; c += blockDim.x) h[96 + 4 * (Jf + 1) + c] = groups[c];
    const uint64_t so = pad8(96 + 4ull * (Jf + 1) + hp.C);
    for (uint32_t g = threadIdx.x; g < G; g += blockDim.x)
        wr64(h + so + 8 * g, (uint64_t)__double_as_longlong(steps_rg[r * G + g]));
    if (hp.color)
        for (uint32_t i = threadIdx.x; i < (uint32_t)kKltFloats; i += blockDim.x)
            wr32(h + so + 8 * G + 4 * i, __float_as_uint(klt[(uint64_t)f * kKltFloats + i]));
}

struct OccCopyArgs {
    const uint8_t *occ;
    const uint64_t *occ_off;
    const uint32_t *mode;
    const uint64_t *chunk_off;
    const uint16_t *freq;
    const uint32_t *chunk_words, *chunk_top, *chunk_pos;
    const uint8_t *slots;
    uint64_t slot_bytes;
};

__global__ void occ_copy_kernel(HdrParams hp, OccCopyArgs a, const StreamInfo *si, const DevState *st, uint8_t *out)
{
    if (st->total_bytes > hp.capacity) return;
    const uint32_t s = blockIdx.y, f = s / hp.R;
    const StreamInfo x = si[s];
    uint8_t *sec = out + x.off + x.hb;
    const uint64_t n = a.occ_off[f + 1] - a.occ_off[f];
    const uint32_t mode = a.mode[f];
    const uint8_t *src = a.occ + a.occ_off[f];
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    if (tid == 0) {
        wr64(sec, n);
        wr32(sec + 8, mode);
    }
    if (mode == 2) {
        if (tid == 0) wr32(sec + 12, n ? src[0] : 0u);
        return;
    }
    if (mode == 0) {
        if (tid == 0) wr32(sec + 12, 0);
        for (uint64_t i = tid; i < x.occ - 16; i += nt) sec[16 + i] = (i < n) ? src[i] : (uint8_t)0;
        return;
    }
    const uint64_t c0 = a.chunk_off[f], nch = a.chunk_off[f + 1] - c0;
    const uint64_t table = pad8(16 + 8 + 512 + 4 * nch);
    if (tid == 0) {
        wr32(sec + 12, (uint32_t)nch);
        wr32(sec + 16, hp.chunk);
        wr32(sec + 20, 0);
    }
    for (uint64_t i = tid; i < 256; i += nt) {
        uint16_t v = a.freq[f * 256 + i];
        sec[24 + 2 * i] = (uint8_t)v;
        sec[24 + 2 * i + 1] = (uint8_t)(v >> 8);
    }
    for (uint64_t c = tid; c < nch; c += nt) {
        uint32_t b = (uint32_t)((128 + 2 * (uint64_t)a.chunk_words[c0 + c] + 3) & ~3ull);
        wr32(sec + 24 + 512 + 4 * c, b);
    }
    for (uint64_t i = 24 + 512 + 4 * nch + tid; i < table; i += nt) sec[i] = 0;
    // chunks: one block-stride loop over chunks, threads over bytes
    for (uint64_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const uint64_t gc = c0 + c;
        const uint8_t *slot = a.slots + gc * a.slot_bytes;
        const uint32_t w = a.chunk_words[gc], top = a.chunk_top[gc];
        uint8_t *dst = sec + a.chunk_pos[gc];
        // states: 32 words; renormalisation words: 16-bit units (slot and
        // destination are both 2-aligned there); then zero padding to 4 bytes
        const uint32_t *s32 = reinterpret_cast<const uint32_t *>(slot);
        uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
        for (uint32_t i = threadIdx.x; i < 32; i += blockDim.x) d32[i] = s32[i];
        const uint16_t *s16 = reinterpret_cast<const uint16_t *>(slot + 128 + 2 * (uint64_t)top);
        uint16_t *d16 = reinterpret_cast<uint16_t *>(dst + 128);
#pragma unroll 4
        for (uint32_t i = threadIdx.x; i < w; i += blockDim.x) d16[i] = s16[i];
        if (threadIdx.x == 0 && (w & 1)) d16[w] = 0;
    }
    if (tid == 0) {  // tail padding of the section
        uint64_t end = nch ? (a.chunk_pos[c0 + nch - 1] + ((128 + 2 * (uint64_t)a.chunk_words[c0 + nch - 1] + 3) & ~3ull)) : table;
        for (uint64_t i = end; i < x.occ; ++i) sec[i] = 0;
    }
}

struct AttrCopyArgs {
    const uint32_t *vstart;
    const uint64_t *blk_off;
    const uint64_t *block_off;  // scanned word offsets of all blocks
    const uint32_t *block_words;
    const uint32_t *slots;
    uint32_t slot_words;
};

__global__ void attr_copy_kernel(HdrParams hp, AttrCopyArgs a, const StreamInfo *si, const DevState *st, uint8_t *out)
{
    if (st->total_bytes > hp.capacity) return;
    const uint32_t s = blockIdx.y, f = s / hp.R, r = s % hp.R;
    const StreamInfo x = si[s];
    if (x.attr == 0) return;
    const uint64_t nv = a.vstart[f + 1] - a.vstart[f];
    const uint32_t nb = (uint32_t)((nv + hp.B - 1) / hp.B);
    const uint64_t nblk = (uint64_t)hp.C * nb;
    const uint64_t b0 = a.blk_off[f] + (uint64_t)r * nblk;
    uint32_t *sec = reinterpret_cast<uint32_t *>(out + x.off + x.hb + x.occ);
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    if (tid == 0) {
        sec[0] = hp.B;
        sec[1] = nb;
    }
    for (uint64_t k = tid; k < nblk; k += nt) sec[2 + k] = a.block_words[b0 + k];
    uint32_t *pay = sec + 2 + nblk;
    const uint64_t base = a.block_off[b0];
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t wid = tid >> 5, nwarps = nt >> 5;
    // a warp takes 32 consecutive block streams: their sizes and offsets in one
    // load, then four streams at a time, the first 96 words of all four loaded
    // before any is stored (a stream is ~75 words at the headline's rates)
    constexpr uint32_t kGroup = 4, kPerLane = 3;
    for (uint64_t k0 = wid * 32; k0 < nblk; k0 += nwarps * 32) {
        const uint64_t k = k0 + lane;
        uint32_t wl = 0;
        uint64_t ol = 0;
        if (k < nblk) {
            wl = a.block_words[b0 + k];
            ol = a.block_off[b0 + k] - base;
        }
        const uint32_t cnt = (nblk - k0) < 32 ? (uint32_t)(nblk - k0) : 32u;
        for (uint32_t j0 = 0; j0 < cnt; j0 += kGroup) {
            uint32_t w[kGroup], v[kGroup][kPerLane];
            uint64_t o[kGroup];
#pragma unroll
            for (uint32_t q = 0; q < kGroup; ++q) {
                const uint32_t j = j0 + q < cnt ? j0 + q : 0u;
                w[q] = __shfl_sync(0xFFFFFFFFu, wl, j);
                o[q] = __shfl_sync(0xFFFFFFFFu, ol, j);
                if (j0 + q >= cnt) w[q] = 0;
                const uint32_t *__restrict__ src = a.slots + (b0 + k0 + j0 + q) * a.slot_words;
#pragma unroll
                for (uint32_t u = 0; u < kPerLane; ++u) {
                    const uint32_t i = lane + 32 * u;
                    v[q][u] = i < w[q] ? __ldg(src + i) : 0u;
                }
            }
#pragma unroll
            for (uint32_t q = 0; q < kGroup; ++q) {
                uint32_t *__restrict__ dst = pay + o[q];
#pragma unroll
                for (uint32_t u = 0; u < kPerLane; ++u) {
                    const uint32_t i = lane + 32 * u;
                    if (i < w[q]) dst[i] = v[q][u];
                }
                // the rest of a longer stream
                const uint32_t *__restrict__ src = a.slots + (b0 + k0 + j0 + q) * a.slot_words;
                for (uint32_t i = 32 * kPerLane + lane; i < w[q]; i += 32) dst[i] = __ldg(src + i);
            }
        }
    }
    const uint64_t used = 8 + 4 * nblk + 4 * (a.block_off[b0 + nblk] - base);
    if (tid == 0 && used < x.attr) wr32(reinterpret_cast<uint8_t *>(sec) + used, 0);
}

// ------------------------------------------------------------- encoder ---
struct EncodeReq {
    uint32_t F = 1;
    const float *const *pos = nullptr;
    const float *const *attr = nullptr;
    const uint64_t *n = nullptr;
    const uint32_t *J = nullptr;
    uint32_t R = 1;
    const double *rung_scale = nullptr;
    const gsnfs_quant *q = nullptr;
    uint8_t *out = nullptr;
    uint64_t capacity = 0;
    float *recon_pos = nullptr;
    float *recon_attr = nullptr;
    double *dist = nullptr;  // host, F x R x C: squared quantisation error sums (or null)
    uint8_t *headers = nullptr;  // host, F x R records of GSNFS_HEADER_RECORD_BYTES (or null)
    // results
    uint64_t total_bytes = 0;
    uint64_t nv = 0;
    std::vector<uint64_t> offsets;
};

struct EncLayout {
    FrameGrid *grid;
    uint32_t *Jd, *vstart, *lsz, *hoff, *mode, *dpart, *opart, *seg, *row0, *vals, *vals_alt, *hist, *chunk_words,
        *chunk_top, *chunk_pos, *cum, *slots, *block_words, *overflow;
    const float **posp, **attrp;
    uint64_t *poff, *keys, *keys_alt, *codes, *occ_off, *chunk_off, *sec_bytes, *job_off, *blk_off, *block_off,
        *spart, *cta_lo;
    uint32_t *cta_seg;  // segmented sort of several frames: per-CTA element ranges and segment bounds
    uint16_t *freq;
    uint8_t *gap, *occ, *chunk_slots, *groups;
    float *inv_step, *step, *Y, *pool, *center, *klt;
    double *steps_rg, *dc, *sq_err, *kltpart;
    StreamInfo *si;
    RahtPlanDev plan;
    uint64_t occ_cap, max_chunks, jobs_bound, blocks_bound;
    uint32_t slot_words;
};

void carve_plan(Carve &cv, RahtPlanDev &p, uint64_t nv_cap, uint32_t T, const uint32_t *tune)
{
    if (tune && tune[GSNFS_TUNE_RAHT_TILE]) T = tune[GSNFS_TUNE_RAHT_TILE];
    p.xgrid_mult = tune ? tune[GSNFS_TUNE_RAHT_GRID] : 0u;
    p.pgrid_mult = tune ? tune[GSNFS_TUNE_PRELUDE_GRID] : 0u;
    p.xpipe_off = tune ? tune[GSNFS_TUNE_RAHT_PIPE] : 0u;
    uint64_t elems, tiles, surv;
    raht_plan_sizes(nv_cap, T, &elems, &tiles, &surv);
    p.T = T;
    p.cap_elems = (uint32_t)elems;
    p.cap_tiles = (uint32_t)tiles;
    p.cap_surv = (uint32_t)surv;
    p.pos = cv.take<uint32_t>(elems);
    p.endseq = cv.take<uint32_t>(elems);
    p.send = cv.take<uint32_t>(elems);
    p.gapseq = cv.take<uint8_t>(elems);
    p.dest = cv.take<uint32_t>(elems);
    p.tile_nbf = cv.take<uint32_t>(tiles);
    p.tile_nr = cv.take<uint32_t>(tiles);
    p.round_end = cv.take<uint16_t>(tiles * 64);
    p.bf_idx = cv.take<uint32_t>(tiles * T);
    p.bf_ab = cv.take<float2>(tiles * T);
    p.bf_w = nullptr;
    p.tile_carry = cv.take<uint32_t>(tiles);
    p.carry_list = cv.take<uint16_t>(tiles * kRahtCarrySlots);
    p.passes = cv.take<RahtPass>(kRahtMaxPasses + 1);
    p.npasses = cv.take<uint32_t>(1);
    p.pos0 = nullptr;
    p.end0 = nullptr;
    p.pipe_ctr = cv.take<uint32_t>(2);
}

size_t carve_encode(Carve &cv, EncLayout &L, const EncodeReq &rq, int num_sms, bool worst_slots,
                    const uint32_t *tune)
{
    const uint32_t F = rq.F, R = rq.R, C = rq.q->num_channels;
    uint64_t N = 0, occ_cap = 0, max_chunks = 0, jobs = 0;
    for (uint32_t f = 0; f < F; ++f) {
        N += rq.n[f];
        uint64_t ob = occ_bound(rq.n[f], rq.J[f]);
        occ_cap += ob;
        max_chunks += (ob + rq.q->rans_chunk - 1) / rq.q->rans_chunk;
        jobs += (rq.n[f] + rq.q->rlgr_block - 1) / rq.q->rlgr_block;  // row blocks (all rungs in one CTA)
    }
    L.occ_cap = (occ_cap + 64) & ~(uint64_t)63;
    L.max_chunks = max_chunks;
    L.jobs_bound = C ? jobs : 0;
    L.blocks_bound = L.jobs_bound * C * R;
    L.slot_words = rlgr_slot_words(rq.q->rlgr_block, worst_slots);
    L.grid = cv.take<FrameGrid>(F);
    L.Jd = cv.take<uint32_t>(F);
    L.posp = (const float **)cv.take<const float *>(F);
    L.attrp = (const float **)cv.take<const float *>(F);
    L.poff = cv.take<uint64_t>(F + 1);
    L.inv_step = cv.take<float>((uint64_t)R * C + 1);
    L.step = cv.take<float>((uint64_t)R * C + 1);
    L.steps_rg = cv.take<double>((uint64_t)R * 256);
    L.center = cv.take<float>((uint64_t)F * (C ? C : 1));
    L.dc = cv.take<double>((uint64_t)F * (C ? C : 1));
    L.sq_err = cv.take<double>((uint64_t)F * R * (C ? C : 1));
    L.klt = cv.take<float>((rq.q->color ? (uint64_t)F : 1) * kKltFloats);
    L.kltpart = cv.take<double>(rq.q->color ? color_klt_partial_words(F) : 1);
    L.groups = cv.take<uint8_t>(256);
    L.vstart = cv.take<uint32_t>(F + 1);
    L.lsz = cv.take<uint32_t>((uint64_t)F * 22);
    L.hoff = cv.take<uint32_t>((uint64_t)F * 22);
    L.occ_off = cv.take<uint64_t>(F + 1);
    L.chunk_off = cv.take<uint64_t>(F + 1);
    L.freq = cv.take<uint16_t>((uint64_t)F * 256);
    L.cum = cv.take<uint32_t>((uint64_t)F * 256);
    L.mode = cv.take<uint32_t>(F);
    L.sec_bytes = cv.take<uint64_t>(F);
    L.job_off = cv.take<uint64_t>(F + 1);
    L.blk_off = cv.take<uint64_t>(F + 1);
    L.si = cv.take<StreamInfo>((uint64_t)F * R + 1);
    L.overflow = cv.take<uint32_t>(4);
    L.keys = cv.take<uint64_t>(N + 1);
    L.keys_alt = cv.take<uint64_t>(N + 1);
    L.vals = cv.take<uint32_t>(N + 1);
    L.vals_alt = cv.take<uint32_t>(N + 1);
    L.hist = cv.take<uint32_t>(radix_sort_hist_words(N, num_sms, F));
    L.cta_lo = cv.take<uint64_t>(radix_sort_max_ctas(N, num_sms) + F + 1);
    L.cta_seg = cv.take<uint32_t>(2 * (radix_sort_max_ctas(N, num_sms) + F));
    L.codes = cv.take<uint64_t>(N + 1);
    L.seg = cv.take<uint32_t>(N + 2);
    L.row0 = cv.take<uint32_t>(N + 1);
    L.gap = cv.take<uint8_t>(N + 2);
    L.dpart = cv.take<uint32_t>(dedup_partial_words(N, num_sms) + 1);
    L.occ = cv.take<uint8_t>(L.occ_cap);
    L.opart = cv.take<uint32_t>(occupancy_partial_words(F, num_sms));
    L.chunk_slots = cv.take<uint8_t>(max_chunks * rans_chunk_slot_bytes(rq.q->rans_chunk) + 16);
    L.chunk_words = cv.take<uint32_t>(max_chunks + 1);
    L.chunk_top = cv.take<uint32_t>(max_chunks + 1);
    L.chunk_pos = cv.take<uint32_t>(max_chunks + 1);
    if (C) {
        uint32_t tune_c[4] = {tune ? tune[0] : 0u, tune ? tune[1] : 0u, tune ? tune[2] : 0u, tune ? tune[3] : 0u};
        if (rq.q->color) tune_c[GSNFS_TUNE_RAHT_TILE] = 0;  // colour transforms need whole rows in a tile
        carve_plan(cv, L.plan, N, raht_tile_size(C), tune_c);
        uint64_t elems, tiles, surv;
        raht_plan_sizes(N, L.plan.T, &elems, &tiles, &surv);
        L.pool = cv.take<float>(surv * C);
        L.Y = cv.take<float>(N * C + 4);
        L.slots = cv.take<uint32_t>(L.blocks_bound * L.slot_words + 4);
        L.block_words = cv.take<uint32_t>(L.blocks_bound + 1);
        L.block_off = cv.take<uint64_t>(L.blocks_bound + 2);
        L.spart = cv.take<uint64_t>(scan_partial_words(L.blocks_bound, num_sms) + 1);
    } else {
        L.plan = RahtPlanDev{};
        L.pool = L.Y = nullptr;
        L.slots = L.block_words = nullptr;
        L.block_off = nullptr;
        L.spart = cv.take<uint64_t>(4);
    }
    return cv.off;
}

constexpr size_t kGraphCacheSize = 64;

// Replays the graph captured for `key`, capturing it first on a miss.  The
// graph runs on the context's own stream, ordered after the caller's stream
// by one event and joined back by another.  A capture that fails runs the
// work eagerly instead (counted in gfailures).
template <typename Enqueue>
gsnfs_status run_graphed(gsnfs_ctx *ctx, cudaStream_t s, std::vector<uint64_t> key, Enqueue &enqueue,
                         std::vector<Profiler::Rec> *stages_out)
{
    if (!ctx->gstream) {
        CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ctx->gev_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->gev_out, cudaEventDisableTiming));
    }
    GraphEntry *hit = nullptr;
    for (auto &g : ctx->gcache)
        if (g.key == key) hit = &g;
    if (!hit) {
        uint64_t launches = 0;
        std::vector<Profiler::Rec> stages;
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal));
        t_capture_launches = &launches;
        t_capture_stages = &stages;
        t_capture_open.clear();
        gsnfs_status st = enqueue(ctx->gstream);
        t_capture_launches = nullptr;
        t_capture_stages = nullptr;
        for (auto &r : t_capture_open) cudaEventDestroy(r.a);  // a stage left open: not timed
        t_capture_open.clear();
        cudaError_t e = cudaStreamEndCapture(ctx->gstream, &graph);
        cudaGraphExec_t exec = nullptr;
        if (st == GSNFS_OK && e == cudaSuccess && graph)
            e = cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
        if (graph) cudaGraphDestroy(graph);
        if (st != GSNFS_OK || e != cudaSuccess || !exec) {
            for (auto &r : stages) {
                cudaEventDestroy(r.a);
                cudaEventDestroy(r.b);
            }
            cudaGetLastError();
            ++ctx->gfailures;
            return enqueue(s);
        }
        if (ctx->gcache.size() >= kGraphCacheSize) {
            auto lru = std::min_element(ctx->gcache.begin(), ctx->gcache.end(),
                                        [](const GraphEntry &a, const GraphEntry &b) { return a.last_use < b.last_use; });
            destroy_graph(*lru);
            ctx->gcache.erase(lru);
        }
        ctx->gcache.push_back(GraphEntry{std::move(key), exec, launches, 0, std::move(stages)});
        hit = &ctx->gcache.back();
        ++ctx->gcaptures;
    } else {
        ++ctx->ghits;
    }
    hit->last_use = ++ctx->gtick;
    CK(cudaEventRecord(ctx->gev_in, s));
    CK(cudaStreamWaitEvent(ctx->gstream, ctx->gev_in, 0));
    CK(cudaGraphLaunch(hit->exec, ctx->gstream));
    CK(cudaEventRecord(ctx->gev_out, ctx->gstream));
    CK(cudaStreamWaitEvent(s, ctx->gev_out, 0));
    g_launches.fetch_add(hit->launches, std::memory_order_relaxed);
    if (stages_out) *stages_out = hit->stages;
    return GSNFS_OK;
}

gsnfs_status encode_impl(gsnfs_ctx *ctx, cudaStream_t s, EncodeReq &rq, bool worst_slots)
{
    const uint32_t F = rq.F, R = rq.R;
    const gsnfs_quant *q = rq.q;
    const uint32_t C = q->num_channels, G = C ? q->num_groups : 0;
    uint64_t N = 0, nmax = 0;
    uint32_t Jmax = 0;
    for (uint32_t f = 0; f < F; ++f) {
        N += rq.n[f];
        nmax = std::max(nmax, rq.n[f]);
        Jmax = std::max(Jmax, rq.J[f]);
    }
    if (N >= 0x7FFFFFF0ull) return GSNFS_ERR_UNSUPPORTED;
    const uint32_t frame_shift = (F == 1) ? 64u : 3u * Jmax;
    uint32_t fbits = 0;
    while ((1u << fbits) < F) ++fbits;
    const uint32_t nbits = (F == 1) ? 3u * rq.J[0] : frame_shift + fbits;
    if (nbits > 64) return GSNFS_ERR_UNSUPPORTED;

    EncLayout L;
    Carve measure(nullptr);
    size_t need = carve_encode(measure, L, rq, ctx->num_sms, worst_slots, ctx->tune);
    gsnfs_status st = grow_arena(ctx, need, s);
    if (st) return st;
    Carve cv(ctx->arena);
    carve_encode(cv, L, rq, ctx->num_sms, worst_slots, ctx->tune);

    // ---- host parameters -> pinned staging -> one copy
    std::vector<unsigned char> hbuf;
    size_t o_pos = 0, o_attr, o_poff, o_J, o_inv, o_step, o_srg, o_grp, o_end;
    o_attr = o_pos + 8 * F;
    o_poff = o_attr + 8 * F;
    o_J = o_poff + 8 * (F + 1);
    o_inv = o_J + 4 * F;
    o_step = o_inv + 4 * (size_t)R * C;
    o_srg = (o_step + 4 * (size_t)R * C + 7) & ~(size_t)7;
    o_grp = o_srg + 8 * (size_t)R * 256;
    // several frames: each frame's keys are sorted on their own (its Morton bits only; no frame pass)
    const uint64_t max_ctas = radix_sort_max_ctas(N, ctx->num_sms) + F;
    const size_t o_ctalo = (o_grp + 256 + 7) & ~(size_t)7;
    const size_t o_ctaseg = o_ctalo + 8 * (max_ctas + 1);
    o_end = o_ctaseg + 8 * max_ctas;
    const size_t o_dist = ((o_end + 63) & ~(size_t)63) + 64;
    const size_t dist_bytes = rq.dist ? 8 * (size_t)F * R * C : 0;
    st = grow_pinned(ctx, o_dist + dist_bytes + 64);
    if (st) return st;
    CK(cudaStreamSynchronize(s));  // previous call's staging copies are done
    unsigned char *hp = ctx->pinned;
    uint64_t acc = 0;
    for (uint32_t f = 0; f < F; ++f) {
        ((const float **)(hp + o_pos))[f] = rq.pos[f];
        ((const float **)(hp + o_attr))[f] = rq.attr ? rq.attr[f] : nullptr;
        ((uint64_t *)(hp + o_poff))[f] = acc;
        acc += rq.n[f];
        ((uint32_t *)(hp + o_J))[f] = rq.J[f];
    }
    ((uint64_t *)(hp + o_poff))[F] = acc;
    const uint32_t sort_ctas = F > 1 ? radix_sort_segment_table((const uint64_t *)(hp + o_poff), F, ctx->num_sms,
                                                                (uint64_t *)(hp + o_ctalo), (uint32_t *)(hp + o_ctaseg))
                                     : 0u;
    for (uint32_t r = 0; r < R; ++r) {
        const double sc = rq.rung_scale ? rq.rung_scale[r] : 1.0;
        for (uint32_t c = 0; c < C; ++c) {
            const double stp = q->steps[q->channel_group[c]] * sc;
            ((float *)(hp + o_inv))[r * C + c] = (float)(1.0 / stp);
            ((float *)(hp + o_step))[r * C + c] = (float)stp;
        }
        for (uint32_t g = 0; g < G; ++g) ((double *)(hp + o_srg))[r * G + g] = q->steps[g] * sc;
    }
    for (uint32_t c = 0; c < C; ++c) hp[o_grp + c] = q->channel_group[c];
    uint64_t *res = (uint64_t *)(hp + ((o_end + 63) & ~(size_t)63));
    // ---- device work: stream-ordered and sized from host values only, so it
    // can be captured once per request shape and replayed as a CUDA graph
    auto enqueue = [&](cudaStream_t s) -> gsnfs_status {
        CK(stage_copy((void *)L.posp, hp + o_pos, 8 * F, s));
        CK(stage_copy((void *)L.attrp, hp + o_attr, 8 * F, s));
        CK(stage_copy(L.poff, hp + o_poff, 8 * (F + 1), s));
        CK(stage_copy(L.Jd, hp + o_J, 4 * F, s));
        if (C) {
            CK(stage_copy(L.inv_step, hp + o_inv, 4 * (size_t)R * C, s));
            CK(stage_copy(L.step, hp + o_step, 4 * (size_t)R * C, s));
            CK(stage_copy(L.steps_rg, hp + o_srg, 8 * (size_t)R * G, s));
            CK(stage_copy(L.groups, hp + o_grp, C, s));
        }
        if (sort_ctas) {
            CK(stage_copy(L.cta_lo, hp + o_ctalo, 8 * ((size_t)sort_ctas + 1), s));
            CK(stage_copy(L.cta_seg, hp + o_ctaseg, 8 * (size_t)sort_ctas, s));
        }
        CK(dev_memset(L.overflow, 0, 16, s));

        DevState *dst = ctx->st;
        const int sms = ctx->num_sms;
        FrameSet fs;
        fs.F = F;
        fs.frame_shift = frame_shift;
        fs.pos = L.posp;
        fs.attr = L.attrp;
        fs.poff = L.poff;
        fs.J = L.Jd;
        fs.grid = L.grid;

        // a1: voxelise + Morton
        stage_begin(s, kStVoxelize);
        launch_voxelize(fs, dst, N, nmax, L.keys, L.vals, sms, s);
        stage_end(s, kStVoxelize);
        // a2: radix sort
        stage_begin(s, kStSort);
        // one frame: its Morton bits; several: each frame on its own (the frame bits need no pass)
        bool alt = sort_ctas ? radix_sort_segments(L.keys, L.vals, L.keys_alt, L.vals_alt, L.hist, N, frame_shift,
                                                   sort_ctas, L.cta_lo, L.cta_seg, sms, s)
                             : radix_sort(L.keys, L.vals, L.keys_alt, L.vals_alt, L.hist, N, nbits, sms, s);
        stage_end(s, kStSort);
        const uint64_t *skeys = alt ? L.keys_alt : L.keys;
        const uint32_t *svals = alt ? L.vals_alt : L.vals;
        // a3: dedup
        stage_begin(s, kStDedup);
        launch_dedup(skeys, N, frame_shift, F, L.codes, L.seg, L.gap, L.vstart, L.dpart, dst, sms, s,
                     C ? svals : nullptr, L.row0);
        stage_end(s, kStDedup);
        // a4 + a5 (geometry) run on s beside a6-a9 (attributes, the longer branch) on the high-priority stream
        cudaStream_t sa = s;
        if (C) {
            const gsnfs_status fst = fork_hi_begin(ctx, s, &sa);
            if (fst) return fst;
        }
        // a4: octree occupancy
        OccupancyOut oo{L.occ, L.occ_cap, L.lsz, L.occ_off, L.hoff, L.opart};
        stage_begin(s, kStOccupancy);
        launch_occupancy(L.codes, L.gap, L.vstart, L.Jd, F, frame_shift, oo, dst, sms, s);
        stage_end(s, kStOccupancy);
        // a5: occupancy rANS
        RansFrames rf{F, L.occ, L.occ_off, q->rans_chunk, L.chunk_off, L.freq, L.cum, L.mode, L.chunk_words,
                      L.chunk_top, L.chunk_pos, L.chunk_slots, L.sec_bytes};
        stage_begin(s, kStRans);
        launch_rans_encode(rf, dst, L.max_chunks, sms, s);
        stage_end(s, kStRans);
        HdrParams hpar{F, R, C, G, C ? q->rlgr_block : 1u, q->rans_chunk, C ? q->color : 0u, q->tau, rq.capacity};
        if (C) {
            // a6: RAHT prelude; a7: forward transform with the cluster average fused into the first pass
            stage_begin(sa, kStPrelude);
            launch_raht_prelude(L.plan, L.gap, dst, nullptr, sms, sa);
            stage_end(sa, kStPrelude);
            launch_frame_centres(L.attrp, L.poff, F, C, L.center, sa);
            if (q->color) launch_color_klt(L.attrp, L.poff, F, L.klt, L.center, L.kltpart, sa);
            RahtIO io{};
            io.C = C;
            io.seg = L.seg;
            io.vals = svals;
            io.row0 = L.row0;
            io.codes = L.codes;
            io.attr = L.attrp;
            io.center = L.center;
            io.klt = q->color ? L.klt : nullptr;
            io.frame_shift = frame_shift;
            io.Y = L.Y;
            io.pool = L.pool;
            stage_begin(sa, kStRahtFwd);
            launch_raht_forward(L.plan, io, N, sms, sa);
            stage_end(sa, kStRahtFwd);
            launch_frame_dc(L.Y, L.vstart, F, C, L.center, L.steps_rg, L.groups, G, q->tau, L.dc, sa);
            // a8 + a9: quantise + block RLGR for every rung
            launch_rlgr_offsets(L.vstart, F, q->rlgr_block, R, C, L.job_off, L.blk_off, sa);
            RlgrJob j{};
            j.C = C;
            j.B = q->rlgr_block;
            j.R = R;
            j.Y = L.Y;
            j.vstart = L.vstart;
            j.F = F;
            j.inv_step = L.inv_step;
            j.tau = (float)q->tau;
            j.slots = L.slots;
            j.block_words = L.block_words;
            j.blk_off = L.blk_off;
            j.slot_words = L.slot_words;
            j.overflow = L.overflow;
            j.dc = L.dc;
            if (rq.dist) {
                CK(dev_memset(L.sq_err, 0, 8 * (size_t)F * R * C, sa));
                j.sq_err = L.sq_err;
                j.step = L.step;
            }
            j.steps_rg = L.steps_rg;
            j.groups = L.groups;
            j.G = G;
            j.tau64 = q->tau;
            stage_begin(sa, kStRlgrEnc);
            launch_rlgr_encode(j, L.job_off, L.jobs_bound, sa);
            stage_end(sa, kStRlgrEnc);
            launch_scan_u32_to_u64(L.block_words, L.blocks_bound, L.block_off, L.spart, sms, sa);
        }
        if (C) {
            const gsnfs_status fst = fork_hi_end(ctx, s);
            if (fst) return fst;
        }
        // a10: container
        stage_begin(s, kStContainer);
        sizes_kernel<<<1, 32, 0, s>>>(hpar, L.Jd, L.vstart, L.sec_bytes, L.blk_off, L.block_off, L.si, dst);
        count_launch();
        header_kernel<<<F * R, 128, 0, s>>>(hpar, L.Jd, L.vstart, L.grid, L.lsz, L.groups, L.steps_rg, L.klt, L.si, dst,
                                            rq.out);
        count_launch();
        OccCopyArgs oa{L.occ, L.occ_off, L.mode, L.chunk_off, L.freq, L.chunk_words, L.chunk_top, L.chunk_pos,
                       L.chunk_slots, rans_chunk_slot_bytes(q->rans_chunk)};
        occ_copy_kernel<<<dim3(std::max<uint32_t>(1, (uint32_t)sms * 4 / (F * R)), F * R), 256, 0, s>>>(hpar, oa, L.si,
                                                                                                      dst, rq.out);
        count_launch();
        if (C) {
            AttrCopyArgs aa{L.vstart, L.blk_off, L.block_off, L.block_words, L.slots, L.slot_words};
            attr_copy_kernel<<<dim3(std::max<uint32_t>(1, (uint32_t)sms * 8 / (F * R)), F * R), 256, 0, s>>>(
                hpar, aa, L.si, dst, rq.out);
            count_launch();
        }
        stage_end(s, kStContainer);
        // a13: optional reconstruction (first frame, first rung)
        stage_begin(s, kStRecon);
        if (F == 1 && rq.recon_pos) launch_voxel_centres_batch(L.codes, dst, N, frame_shift, L.Jd, L.grid, rq.recon_pos, s);
        if (F == 1 && C && rq.recon_attr) {
            RahtIO io{};
            io.C = C;
            io.Y = L.Y;
            io.out = rq.recon_attr;
            io.pool = L.pool;
            io.inv_step = L.inv_step;
            io.step = L.step;
            io.tau = (float)q->tau;
            io.frame_shift = frame_shift;
            if (q->color) {
                io.klt = L.klt;
                io.vstart = L.vstart;
                io.F = F;
                io.yuv_inv = yuv_inverse();
            }
            launch_raht_inverse(L.plan, io, N, sms, s);
        }
        stage_end(s, kStRecon);
        CK(cudaGetLastError());
        // results
        CK(stage_copy(res, &dst->err, 8, s));
        CK(stage_copy(res + 1, &dst->nv_total, 16, s));
        CK(stage_copy(res + 3, L.overflow, 4, s));
        if (dist_bytes) CK(stage_copy(hp + o_dist, L.sq_err, dist_bytes, s));
        return GSNFS_OK;
    };
    std::vector<Profiler::Rec> gstages;  // the replayed graph's stage events
    if (ctx->graphs) {
        std::vector<uint64_t> key = {F, R, C, G, C ? q->rlgr_block : 0u, q->rans_chunk, 0, rq.capacity,
                                     (uint64_t)(uintptr_t)rq.out, (uint64_t)(uintptr_t)rq.recon_pos,
                                     (uint64_t)(uintptr_t)rq.recon_attr, worst_slots ? 1u : 0u,
                                     (uint64_t)(uintptr_t)ctx->arena, ctx->arena_cap,
                                     (uint64_t)(uintptr_t)ctx->pinned, rq.attr ? 1u : 0u, rq.dist ? 1u : 0u,
                                     C ? q->color : 0u};
        memcpy(&key[6], &q->tau, 8);
        for (uint32_t f = 0; f < F; ++f) {
            key.push_back(rq.n[f]);
            key.push_back(rq.J[f]);
        }
        st = run_graphed(ctx, s, std::move(key), enqueue, &gstages);
    } else {
        st = enqueue(s);
    }
    if (st) return st;
    CK(cudaStreamSynchronize(s));
    add_graph_stage_times(gstages);
    const uint32_t derr = (uint32_t)(res[0] & 0xFFFFFFFFu);
    rq.nv = res[1];
    rq.total_bytes = res[2];
    const uint32_t ovf = (uint32_t)(res[3] & 0xFFFFFFFFu);
    if (ovf && !worst_slots) return encode_impl(ctx, s, rq, true);
    if (dist_bytes) memcpy(rq.dist, hp + o_dist, dist_bytes);
    if (derr == kErrCapacity) return GSNFS_ERR_CAPACITY;
    if (derr) return map_dev_error(derr);
    if (!rq.offsets.empty()) {
        std::vector<StreamInfo> si((size_t)F * R + 1);
        CK(cudaMemcpy(si.data(), L.si, sizeof(StreamInfo) * si.size(), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < si.size(); ++i) rq.offsets[i] = si[i].off;
    }
    if (rq.headers) {  // header records through the pinned staging buffer (the stream is idle here)
        const size_t nrec = (size_t)F * R, bytes = nrec * GSNFS_HEADER_RECORD_BYTES;
        st = grow_pinned(ctx, bytes);
        if (st) return st;
        header_records_kernel<<<(uint32_t)nrec, 256, 0, s>>>(rq.out, L.si, (uint32_t)nrec, ctx->pinned);
        count_launch();
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s));
        memcpy(rq.headers, ctx->pinned, bytes);
    }
    return GSNFS_OK;
}

// ------------------------------------------------------------- decoder ---
struct ParsedHeader {
    uint32_t J, C, G, hb;
    uint64_t nv, occ_bytes, attr_bytes, n_occ;
    double lo[3], ext, tau;
    uint32_t lsz[22];
    uint8_t groups[256];
    double steps[256];
    uint32_t occ_mode, occ_aux, chunk;
    uint32_t B, nb;
    uint32_t color;    // header flags bit 0
    uint64_t klt_off;  // byte offset of the KLT matrices in the stream (colour mode)
};

uint32_t rd32(const uint8_t *p) { uint32_t v; memcpy(&v, p, 4); return v; }
uint64_t rd64(const uint8_t *p) { uint64_t v; memcpy(&v, p, 8); return v; }
double rdf64(const uint8_t *p) { double v; memcpy(&v, p, 8); return v; }

gsnfs_status parse_fixed(const uint8_t *h, uint64_t bytes, ParsedHeader &P)
{
    if (bytes < 96 || rd32(h) != kMagic || rd32(h + 4) != 1) return GSNFS_ERR_CORRUPT;
    P.hb = rd32(h + 8);
    P.J = rd32(h + 12);
    P.C = rd32(h + 16);
    P.G = rd32(h + 20);
    P.nv = rd64(h + 24);
    for (int a = 0; a < 3; ++a) P.lo[a] = rdf64(h + 32 + 8 * a);
    P.ext = rdf64(h + 56);
    P.tau = rdf64(h + 64);
    P.occ_bytes = rd64(h + 72);
    P.attr_bytes = rd64(h + 80);
    const uint32_t flags = rd32(h + 88);
    P.color = flags & 1u;
    if (flags & ~1u) return GSNFS_ERR_CORRUPT;
    if (P.J < 1 || P.J > (uint32_t)kMaxJ || P.C > (uint32_t)kMaxC || P.G > 255) return GSNFS_ERR_CORRUPT;
    if (P.C > 0 && P.G == 0) return GSNFS_ERR_CORRUPT;
    if (P.color && P.C != 56) return GSNFS_ERR_CORRUPT;
    if (P.hb != header_bytes(P.J, P.C, P.C ? P.G : 0, P.color)) return GSNFS_ERR_CORRUPT;
    P.klt_off = pad8(96 + 4ull * (P.J + 1) + P.C) + 8ull * P.G;
    if (P.occ_bytes < 16 || P.occ_bytes > bytes || P.attr_bytes > bytes ||
        (uint64_t)P.hb + P.occ_bytes + P.attr_bytes > bytes)
        return GSNFS_ERR_CORRUPT;
    if (!(P.ext > 0.0) || !std::isfinite(P.ext)) return GSNFS_ERR_CORRUPT;
    if (P.nv >= 0x7FFFFFF0ull) return GSNFS_ERR_UNSUPPORTED;
    return GSNFS_OK;
}

gsnfs_status parse_tables(const uint8_t *h, ParsedHeader &P)
{
    P.n_occ = 0;
    for (uint32_t d = 0; d <= P.J; ++d) {
        P.lsz[d] = rd32(h + 96 + 4 * d);
        if (d < P.J) P.n_occ += P.lsz[d];
    }
    if (P.lsz[P.J] != P.nv) return GSNFS_ERR_CORRUPT;
    if (P.nv == 0) {
        for (uint32_t d = 0; d <= P.J; ++d)
            if (P.lsz[d]) return GSNFS_ERR_CORRUPT;
    } else {
        if (P.lsz[0] != 1) return GSNFS_ERR_CORRUPT;
        for (uint32_t d = 0; d < P.J; ++d)
            if (P.lsz[d + 1] < P.lsz[d] || (uint64_t)P.lsz[d + 1] > 8ull * P.lsz[d]) return GSNFS_ERR_CORRUPT;
    }
    for (uint32_t c = 0; c < P.C; ++c) {
        P.groups[c] = h[96 + 4 * (P.J + 1) + c];
        if (P.groups[c] >= P.G) return GSNFS_ERR_CORRUPT;
    }
    const uint64_t so = pad8(96 + 4ull * (P.J + 1) + P.C);
    for (uint32_t g = 0; g < (P.C ? P.G : 0); ++g) {
        P.steps[g] = rdf64(h + so + 8 * g);
        if (!(P.steps[g] > 0.0) || !std::isfinite(P.steps[g])) return GSNFS_ERR_CORRUPT;
    }
    return GSNFS_OK;
}

gsnfs_status parse_sections(const uint8_t *occ_hdr, const uint8_t *attr_hdr, ParsedHeader &P)
{
    if (rd64(occ_hdr) != P.n_occ) return GSNFS_ERR_CORRUPT;
    P.occ_mode = rd32(occ_hdr + 8);
    P.occ_aux = rd32(occ_hdr + 12);
    P.chunk = rd32(occ_hdr + 16);
    if (P.occ_mode == 0) {
        if (16 + P.n_occ > P.occ_bytes) return GSNFS_ERR_CORRUPT;
    } else if (P.occ_mode == 2) {
        if (P.occ_aux > 255) return GSNFS_ERR_CORRUPT;
    } else if (P.occ_mode == 1) {
        if (P.chunk < 32 || P.chunk % 32 || P.chunk > (1u << 20)) return GSNFS_ERR_CORRUPT;
        if ((uint64_t)P.occ_aux != (P.n_occ + P.chunk - 1) / P.chunk) return GSNFS_ERR_CORRUPT;
        if (pad8(16 + 8 + 512 + 4ull * P.occ_aux) > P.occ_bytes) return GSNFS_ERR_CORRUPT;
    } else {
        return GSNFS_ERR_CORRUPT;
    }
    P.B = 1;
    P.nb = 0;
    if (P.C > 0 && P.nv > 0) {
        if (P.attr_bytes < 8) return GSNFS_ERR_CORRUPT;
        P.B = rd32(attr_hdr);
        P.nb = rd32(attr_hdr + 4);
        if (!pow2(P.B) || P.B < 32 || P.B > 65536) return GSNFS_ERR_CORRUPT;
        if ((uint64_t)P.nb != (P.nv + P.B - 1) / P.B) return GSNFS_ERR_CORRUPT;
        if (8 + 4ull * P.C * P.nb > P.attr_bytes) return GSNFS_ERR_CORRUPT;
    } else if (P.attr_bytes != 0) {
        return GSNFS_ERR_CORRUPT;
    }
    return GSNFS_OK;
}

gsnfs_status read_headers(gsnfs_ctx *ctx, cudaStream_t s, const uint8_t *d_in, uint64_t bytes, ParsedHeader &P)
{
    gsnfs_status st = grow_pinned(ctx, 8192);
    if (st) return st;
    CK(cudaStreamSynchronize(s));
    uint8_t *hp = ctx->pinned;
    if (bytes < 96) return GSNFS_ERR_CORRUPT;
    CK(stage_copy(hp, d_in, 96, s));
    CK(cudaStreamSynchronize(s));
    st = parse_fixed(hp, bytes, P);
    if (st) return st;
    CK(stage_copy(hp, d_in, P.hb, s));
    CK(stage_copy(hp + 4096, d_in + P.hb, 24, s));
    if (P.attr_bytes >= 8) CK(stage_copy(hp + 4096 + 64, d_in + P.hb + P.occ_bytes, 8, s));
    CK(cudaStreamSynchronize(s));
    st = parse_tables(hp, P);
    if (st) return st;
    return parse_sections(hp + 4096, hp + 4096 + 64, P);
}

struct DecLayout {
    uint32_t *tabs;
    uint8_t *occ, *gap;
    uint64_t *nodes, *codes, *nvdev, *block_off, *spart;
    uint32_t *pref, *ppart;
    float *Y, *pool, *step, *ctab, *klt;
    uint32_t *vst;
    FrameGrid *grid;
    RahtPlanDev plan;
};

size_t carve_decode(Carve &cv, DecLayout &L, const ParsedHeader &P, int num_sms, const uint32_t *tune)
{
    L.grid = cv.take<FrameGrid>(1);
    L.tabs = cv.take<uint32_t>(rans_table_words());
    L.nvdev = cv.take<uint64_t>(1);
    L.step = cv.take<float>(P.C + 1);
    L.occ = cv.take<uint8_t>(P.n_occ + 8);
    L.pref = cv.take<uint32_t>(P.n_occ + 2);
    L.ppart = cv.take<uint32_t>(2 * (uint64_t)num_sms + 8);
    uint64_t nodes = 0;
    for (uint32_t d = 0; d < P.J; ++d) nodes += P.lsz[d];
    L.nodes = cv.take<uint64_t>(nodes + 1);
    L.codes = cv.take<uint64_t>(P.nv + 1);
    L.gap = cv.take<uint8_t>(P.nv + 2);
    L.ctab = cv.take<float>(((1ull << P.J) <= P.nv) ? (3ull << P.J) : 1);
    L.klt = cv.take<float>(kKltFloats);
    L.vst = cv.take<uint32_t>(2);
    if (P.C && P.nv) {
        uint32_t tune_c[4] = {tune ? tune[0] : 0u, tune ? tune[1] : 0u, tune ? tune[2] : 0u, tune ? tune[3] : 0u};
        if (P.color) tune_c[GSNFS_TUNE_RAHT_TILE] = 0;  // colour transforms need whole rows in a tile
        carve_plan(cv, L.plan, P.nv, raht_tile_size(P.C), tune_c);
        uint64_t elems, tiles, surv;
        raht_plan_sizes(P.nv, L.plan.T, &elems, &tiles, &surv);
        L.pool = cv.take<float>(surv * P.C);
        L.Y = cv.take<float>(P.nv * P.C + 4);
        L.block_off = cv.take<uint64_t>((uint64_t)P.C * P.nb + 2);
        L.spart = cv.take<uint64_t>(scan_partial_words((uint64_t)P.C * P.nb, num_sms) + 1);
    }
    return cv.off;
}

// Level-of-detail request of decode_impl: node centres and means at octree depth `depth` < J.
struct LodReq {
    uint32_t depth;
    float *pos, *attr;     // caller's outputs (either may be null)
    uint64_t capacity;     // rows of both
    uint64_t *out_nodes;
};

gsnfs_status lod_from_voxels(gsnfs_ctx *ctx, cudaStream_t s, cudaStream_t cs, const ParsedHeader &P, DecLayout &L,
                             bool attrs,
                             const LodReq &lod);

gsnfs_status decode_impl(gsnfs_ctx *ctx, cudaStream_t s, const uint8_t *d_in, uint64_t bytes, float *d_pos,
                         float *d_attr, uint64_t capacity_nv, uint64_t *out_nv, const uint64_t **codes_out = nullptr,
                         const LodReq *lod = nullptr)
{
    ParsedHeader P{};
    gsnfs_status st = read_headers(ctx, s, d_in, bytes, P);
    if (st) return st;
    if (out_nv) *out_nv = P.nv;
    if (P.nv > capacity_nv) return GSNFS_ERR_CAPACITY;
    if (P.nv == 0) return GSNFS_OK;
    DecLayout L;
    Carve m(nullptr);
    size_t need = carve_decode(m, L, P, ctx->num_sms, ctx->tune);
    st = grow_arena(ctx, need, s);
    if (st) return st;
    Carve cv(ctx->arena);
    carve_decode(cv, L, P, ctx->num_sms, ctx->tune);
    if (codes_out) *codes_out = L.codes;
    DevState *dst = ctx->st;
    // host-computed grid and steps
    unsigned char *hp = ctx->pinned;
    FrameGrid g;
    for (int a = 0; a < 3; ++a) g.lo[a] = P.lo[a];
    g.ext = P.ext;
    g.scale = std::ldexp(1.0, (int)P.J) / P.ext;
    g.cell = P.ext / std::ldexp(1.0, (int)P.J);
    memcpy(hp, &g, sizeof(g));
    memcpy(hp + 128, &P.nv, 8);
    const uint32_t vst_h[2] = {0u, (uint32_t)P.nv};
    memcpy(hp + 192, vst_h, 8);
    for (uint32_t c = 0; c < P.C; ++c) ((float *)(hp + 256))[c] = (float)P.steps[P.groups[c]];
    CK(stage_copy(L.grid, hp, sizeof(g), s));
    CK(stage_copy(L.nvdev, hp + 128, 8, s));
    CK(stage_copy(L.vst, hp + 192, 8, s));
    if (P.color) CK(stage_copy(L.klt, d_in + P.klt_off, 4 * kKltFloats, s));
    if (P.C) CK(stage_copy(L.step, hp + 256, 4 * P.C, s));
    CK(dev_memset(dst, 0, 8, s));
    const int sms = ctx->num_sms;
    // a12's RLGR decode needs only the block tables: it runs on s beside a11 and the schedule (the longer
    // branch), which run on the context's high-priority stream sg and take the RLGR branch's results last
    const bool attrs = P.C && d_attr;
    cudaStream_t sg = s;
    if (attrs) {
        st = fork_hi_begin(ctx, s, &sg);
        if (st) return st;
        const uint8_t *as = d_in + P.hb + P.occ_bytes;
        const uint32_t *bw = reinterpret_cast<const uint32_t *>(as + 8);
        const uint64_t nblk = (uint64_t)P.C * P.nb;
        const uint32_t *payload = bw + nblk;
        const uint64_t payload_words = (P.attr_bytes - 8 - 4 * nblk) / 4;
        launch_scan_u32_to_u64(bw, nblk, L.block_off, L.spart, sms, s);
        stage_begin(s, kStRlgrDec);
        launch_rlgr_decode(payload, payload_words, bw, L.block_off, P.nv, P.C, P.B, L.step, L.Y, dst, s);
        stage_end(s, kStRlgrDec);
    }
    // a11: occupancy bytes
    const uint8_t *sec = d_in + P.hb;
    const uint8_t *occ = L.occ;
    stage_begin(sg, kStOccDecode);
    if (P.occ_mode == 0)
        occ = sec + 16;
    else if (P.occ_mode == 2)
        launch_fill(L.occ, P.n_occ, (uint8_t)P.occ_aux, sg);
    else
        launch_rans_decode(sec, P.occ_bytes, P.n_occ, P.occ_aux, P.chunk, L.occ, L.tabs, dst, sms, sg);
    stage_end(sg, kStOccDecode);
    stage_begin(sg, kStOctreeDecode);
    launch_octree_decode(occ, P.n_occ, P.J, P.lsz, L.nodes, L.pref, L.ppart, L.codes, dst, sms, sg);
    if (d_pos) launch_voxel_centres(L.codes, P.nv, P.J, L.grid, d_pos, sg, L.ctab);
    stage_end(sg, kStOctreeDecode);
    if (lod) return lod_from_voxels(ctx, sg, s, P, L, attrs, *lod);
    // a12: schedule, then (after the RLGR branch) the inverse RAHT
    if (attrs) {
        stage_begin(sg, kStPrelude);
        launch_gap_levels(L.codes, P.nv, L.gap, sg);
        launch_raht_prelude(L.plan, L.gap, dst, L.nvdev, sms, sg);
        stage_end(sg, kStPrelude);
        st = stream_wait(ctx, sg, s);  // the coefficients
        if (st) return st;
        RahtIO io{};
        io.C = P.C;
        io.Y = L.Y;
        io.out = d_attr;
        io.pool = L.pool;
        io.frame_shift = 64;
        if (P.color) {
            io.klt = L.klt;
            io.vstart = L.vst;
            io.F = 1;
            io.yuv_inv = yuv_inverse();
        }
        stage_begin(sg, kStRahtInv);
        launch_raht_inverse(L.plan, io, P.nv, sms, sg);
        stage_end(sg, kStRahtInv);
        st = fork_hi_end(ctx, s);  // the caller's stream sees all of it
        if (st) return st;
    }
    CK(cudaGetLastError());
    uint32_t *res = (uint32_t *)(hp + 1024);
    CK(stage_copy(res, &dst->err, 4, s));
    CK(cudaStreamSynchronize(s));
    return map_dev_error(res[0]);
}

// Level of detail from a decoded voxel set (geometry decoded on s, the
// context's high-priority stream when attrs; the dequantised coefficients Y
// being decoded on the caller's stream cs): the nodes of depth lod.depth are runs of voxels sharing
// code >> 3(J - depth).  Each node becomes one element of a coarser RAHT
// sequence (its voxel run, the gap before its first voxel): its weight is its
// voxel count and its coefficients sit at its first voxel's row of Y, the
// rows that hold the high passes of the butterflies above the depth (Eq. 1,
// Algorithm 6).  The inverse over that sequence stops at the nodes, so the
// butterflies inside nodes are never applied; a node's result is its
// low-pass coefficient, and its mean attribute is that divided by sqrt(w).
gsnfs_status lod_from_voxels(gsnfs_ctx *ctx, cudaStream_t s, cudaStream_t cs, const ParsedHeader &P, DecLayout &L,
                             bool attrs,
                             const LodReq &lod)
{
    const int sms = ctx->num_sms;
    const uint64_t nv = P.nv;
    const uint32_t C = attrs && lod.attr ? P.C : 0;
    DevState *dst = ctx->st;
    uint32_t *flags = nullptr, *pos0 = nullptr, *end0 = nullptr;
    uint64_t *offs = nullptr, *starts = nullptr, *part = nullptr;
    uint8_t *gap0 = nullptr;
    auto carve = [&](Carve &cv) {
        flags = cv.take<uint32_t>(nv + 1);
        offs = cv.take<uint64_t>(nv + 2);
        starts = cv.take<uint64_t>(nv + 2);
        part = cv.take<uint64_t>(scan_partial_words(nv, sms) + 1);
        pos0 = cv.take<uint32_t>(nv + 1);
        end0 = cv.take<uint32_t>(nv + 1);
        gap0 = cv.take<uint8_t>(nv + 2);
        return cv.off;
    };
    Carve m(nullptr);
    const size_t need = carve(m);
    gsnfs_status res = GSNFS_OK;
    if (need > ctx->lod_cap) {
        if (ctx->lod) cudaFree(ctx->lod);
        ctx->lod = nullptr;
        ctx->lod_cap = 0;
        if (cudaMalloc(&ctx->lod, need) != cudaSuccess) {
            ctx->lod = nullptr;
            res = GSNFS_ERR_OOM;
        } else {
            ctx->lod_cap = need;
        }
    }
    // node count: known on the device only; with room for every voxel the outputs need no check before the
    // kernels, so the count is read back at the end (else once here, before anything is written)
    uint64_t nn = nv;
    const bool room = lod.capacity >= nv;
    uint64_t *hn = reinterpret_cast<uint64_t *>(ctx->pinned + 2048);
    const uint32_t sh = 3 * (P.J - lod.depth);
    if (!res) {
        Carve cv(ctx->lod);
        carve(cv);
        launch_lod_index(L.codes, nv, sh, flags, offs, part, starts, sms, s);
        if (!room) {
            if (stage_copy(hn, offs + nv, 8, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
                res = GSNFS_ERR_CUDA;
            else
                nn = *hn;
            *lod.out_nodes = nn;
            if (!res && nn > lod.capacity) res = GSNFS_ERR_CAPACITY;
        }
        if (!res && C) {
            launch_gap_levels(L.codes, nv, L.gap, s);
            launch_lod_sequence(starts, offs + nv, nv, nn, L.gap, pos0, end0, gap0, sms, s);
            L.plan.pos0 = pos0;
            L.plan.end0 = end0;
            stage_begin(s, kStPrelude);
            launch_raht_prelude(L.plan, gap0, dst, offs + nv, sms, s);
            stage_end(s, kStPrelude);
        }
    }
    if (attrs) {  // join the coefficient branch (on cs) before anything returns
        const gsnfs_status fst = stream_wait(ctx, s, cs);
        if (fst) return fst;
    }
    if (res) {
        cudaStreamSynchronize(s);
        return res;
    }
    if (C) {
        RahtIO io{};
        io.C = C;
        io.Y = L.Y;
        io.out = lod.attr;  // node rows, divided by sqrt(voxel count) as they are stored: the means
        io.lod_mean = 1;
        io.pool = L.pool;
        io.frame_shift = 64;
        if (P.color) {
            io.klt = L.klt;
            io.vstart = L.vst;
            io.F = 1;
            io.yuv_inv = yuv_inverse();
        }
        stage_begin(s, kStRahtInv);
        launch_raht_inverse(L.plan, io, nn, sms, s);
        stage_end(s, kStRahtInv);
    }
    LodGrid g;
    for (int a = 0; a < 3; ++a) g.lo[a] = P.lo[a];
    g.cell = P.ext / std::ldexp(1.0, (int)lod.depth);
    launch_lod_centres(L.codes, starts, offs + nv, nn, sh, lod.depth, g, lod.pos, sms, s);
    CK(cudaGetLastError());
    if (attrs) {  // the caller's stream sees all of it
        const gsnfs_status fst = fork_hi_end(ctx, cs);
        if (fst) return fst;
    }
    uint32_t *hres = reinterpret_cast<uint32_t *>(ctx->pinned + 1024);
    CK(stage_copy(hres, &dst->err, 4, cs));
    if (room) CK(stage_copy(hn, offs + nv, 8, cs));
    CK(cudaStreamSynchronize(cs));
    if (room) *lod.out_nodes = *hn;
    return map_dev_error(hres[0]);
}

// ------------------------------------------------------- batched decoder ---
// All frames of a batch are decoded by one sequence of launches: the header
// records are given (asynchronous decode) or read out of the streams by one
// kernel and one host wait for the whole batch, then every stage runs over all
// frames at once (frame tables on the device).
gsnfs_status decode_batch_impl(gsnfs_ctx *ctx, cudaStream_t s, uint32_t F, const uint8_t *d_in, const uint64_t *offs,
                               float *d_pos, float *d_attr, uint64_t capacity_rows, uint64_t *rows_out,
                               const uint8_t *h_headers = nullptr, uint32_t *status = nullptr)
{
    std::vector<ParsedHeader> P(F);
    gsnfs_status st = GSNFS_OK;
    const size_t stage_need = (size_t)F * 8192 + 65536;
    uint8_t *hp = nullptr;
    int ring = -1;
    if (status) {  // asynchronous: staging slot of its own, reused only once its last use has completed
        ring = (int)(ctx->aring_next++ & 3u);
        if (!ctx->aring_ev[ring]) {
            CK(cudaEventCreateWithFlags(&ctx->aring_ev[ring], cudaEventDisableTiming));
        } else {
            CK(cudaEventSynchronize(ctx->aring_ev[ring]));
        }
        if (ctx->aring_cap[ring] < stage_need) {
            if (ctx->aring[ring]) CK(cudaFreeHost(ctx->aring[ring]));
            ctx->aring[ring] = nullptr;
            ctx->aring_cap[ring] = 0;
            CK(cudaMallocHost((void **)&ctx->aring[ring], stage_need));
            ctx->aring_cap[ring] = stage_need;
        }
        hp = ctx->aring[ring];
    } else {
        st = grow_pinned(ctx, stage_need);
        if (st) return st;
        CK(cudaStreamSynchronize(s));
        hp = ctx->pinned;
    }
    // header record of frame f: given by the caller, or read back into the staging buffer
    auto rec = [&](uint32_t f) -> const uint8_t * {
        return h_headers ? h_headers + (size_t)f * GSNFS_HEADER_RECORD_BYTES : hp + (size_t)f * 8192;
    };
    if (!h_headers) {  // every frame's record read out of its stream by one launch per 64 frames, one wait
        for (uint32_t f = 0; f < F; ++f)
            if (offs[f + 1] - offs[f] < 96) return GSNFS_ERR_CORRUPT;
        for (uint32_t f0 = 0; f0 < F; f0 += kRecFrames) {
            RecLaunch a;
            a.in = d_in;
            a.rec = hp;
            a.stride = 8192;
            a.f0 = f0;
            const uint32_t n = std::min<uint32_t>(kRecFrames, F - f0);
            for (uint32_t i = 0; i <= n; ++i) a.off[i] = offs[f0 + i];
            stream_records_kernel<<<n, 256, 0, s>>>(a);
            count_launch();
        }
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s));
    }
    for (uint32_t f = 0; f < F; ++f) {
        if (offs[f + 1] - offs[f] < 96) return GSNFS_ERR_CORRUPT;
        st = parse_fixed(rec(f), offs[f + 1] - offs[f], P[f]);
        if (st) return st;
        if (P[f].hb > 4096) return GSNFS_ERR_CORRUPT;
    }
    uint32_t C = 0, Jmax = 0;
    uint64_t N = 0, n_occ = 0, nodes = 0, nblk = 0, jobs = 0, max_occ = 0;
    uint32_t max_nch = 0, chunk_max = 0;
    uint64_t n_chunks = 0;
    bool any_rans = false;
    for (uint32_t f = 0; f < F; ++f) {
        const uint8_t *h = rec(f);
        st = parse_tables(h, P[f]);
        if (st) return st;
        st = parse_sections(h + 4096, h + 4096 + 64, P[f]);
        if (st) return st;
        if (f == 0) C = P[f].C;
        if (P[f].C != C) return GSNFS_ERR_UNSUPPORTED;  // one attribute layout per batch
        Jmax = std::max(Jmax, P[f].J);
        N += P[f].nv;
        n_occ += P[f].n_occ;
        max_occ = std::max(max_occ, P[f].n_occ);
        for (uint32_t d = 0; d < P[f].J; ++d) nodes += P[f].lsz[d];
        if (C && P[f].nv) {
            nblk += (uint64_t)P[f].nb * C;
            jobs += P[f].nb;
        }
        if (P[f].occ_mode == 1) {
            any_rans = true;
            max_nch = std::max(max_nch, P[f].occ_aux);
            n_chunks += P[f].occ_aux;
            chunk_max = std::max(chunk_max, P[f].chunk);
        }
    }
    rows_out[0] = 0;
    for (uint32_t f = 0; f < F; ++f) rows_out[f + 1] = rows_out[f] + P[f].nv;
    if (N > capacity_rows) return GSNFS_ERR_CAPACITY;
    if (N >= 0x7FFFFFF0ull) return GSNFS_ERR_UNSUPPORTED;
    if (N == 0) return GSNFS_OK;

    // ---- layout
    struct L_ {
        DecFrame *fr;
        uint32_t *vstart, *bw_all, *tabs, *tsum, *tile_pref;
        uint64_t *lvl_pref, *job_off, *blk_pref, *boff_all, *spart, *tbase, *tpart, *nodes, *nvdev;
        float *steps, *Y, *pool;
        uint8_t *occ, *gap;
        float *ctab, *klt;
        uint32_t *fcolor;
        uint64_t *cstart;  // byte offset of every rANS chunk inside its frame's occupancy section
        RahtPlanDev plan;
    } L;
    bool any_color = false;
    for (uint32_t f = 0; f < F; ++f) any_color |= P[f].color != 0;
    // voxel-centre tables for frames with 2^J <= N_v (see launch_batch_centre_tables)
    uint64_t ctab_total = 0;
    for (uint32_t f = 0; f < F; ++f)
        if (d_pos && P[f].nv && (1ull << P[f].J) <= P[f].nv) ctab_total += 3ull << P[f].J;
    auto carve = [&](Carve &cv) {
        L.fr = cv.take<DecFrame>(F);
        L.vstart = cv.take<uint32_t>(F + 1);
        L.lvl_pref = cv.take<uint64_t>((uint64_t)(Jmax + 1) * (F + 1));
        L.job_off = cv.take<uint64_t>(F + 1);
        L.blk_pref = cv.take<uint64_t>(F + 1);
        L.nvdev = cv.take<uint64_t>(1);
        L.steps = cv.take<float>((uint64_t)F * C + 1);
        L.tabs = cv.take<uint32_t>(any_rans ? (uint64_t)F * rans_table_words() : 1);
        L.cstart = cv.take<uint64_t>(n_chunks + 1);
        L.occ = cv.take<uint8_t>(n_occ + 8);
        L.tsum = cv.take<uint32_t>(occ_tiles(n_occ) + 1);
        L.tbase = cv.take<uint64_t>(occ_tiles(n_occ) + 2);
        L.tpart = cv.take<uint64_t>(scan_partial_words(occ_tiles(n_occ), ctx->num_sms) + 1);
        L.tile_pref = cv.take<uint32_t>((uint64_t)Jmax * (F + 1) + 1);
        L.nodes = cv.take<uint64_t>(nodes + 1);
        L.gap = cv.take<uint8_t>(N + 2);
        L.ctab = cv.take<float>(ctab_total + 1);
        L.klt = cv.take<float>((any_color ? (uint64_t)F : 1) * kKltFloats);
        L.fcolor = cv.take<uint32_t>(F + 1);
        if (C) {
            uint32_t tune_c[4] = {ctx->tune[0], ctx->tune[1], ctx->tune[2], ctx->tune[3]};
            if (any_color) tune_c[GSNFS_TUNE_RAHT_TILE] = 0;  // colour transforms need whole rows in a tile
            carve_plan(cv, L.plan, N, raht_tile_size(C), tune_c);
            uint64_t elems, tiles, surv;
            raht_plan_sizes(N, L.plan.T, &elems, &tiles, &surv);
            L.pool = cv.take<float>(surv * C);
            L.Y = cv.take<float>(N * C + 4);
            L.bw_all = cv.take<uint32_t>(nblk + 1);
            L.boff_all = cv.take<uint64_t>(nblk + 2);
            L.spart = cv.take<uint64_t>(scan_partial_words(nblk, ctx->num_sms) + 1);
        }
        return cv.off;
    };
    Carve m(nullptr);
    st = grow_arena(ctx, carve(m), s);
    if (st) return st;
    Carve cv(ctx->arena);
    carve(cv);

    // ---- frame tables, packed into pinned memory after the headers
    unsigned char *tp = hp + (size_t)F * 8192;
    size_t o_fr = 0, o_vs = o_fr + sizeof(DecFrame) * F, o_lp = (o_vs + 4 * (F + 1) + 7) & ~(size_t)7;
    size_t o_jo = o_lp + 8 * (size_t)(Jmax + 1) * (F + 1), o_bp = o_jo + 8 * (F + 1), o_nv = o_bp + 8 * (F + 1);
    size_t o_st = o_nv + 8, o_fc = o_st + 4 * (size_t)F * C, o_tp = o_fc + 4 * (size_t)(F + 1);
    size_t o_end = o_tp + 4 * ((size_t)Jmax * (F + 1) + 1);
    const size_t need = (size_t)F * 8192 + o_end + 128;  // and the status word after the tables
    if (status ? ctx->aring_cap[ring] < need : ctx->pinned_cap < need) {
        // the headers are parsed by now: the staging buffer holds nothing still needed
        if (status) {  // the slot's last use has completed (its event was waited on above)
            CK(cudaFreeHost(ctx->aring[ring]));
            ctx->aring[ring] = nullptr;
            ctx->aring_cap[ring] = 0;
            CK(cudaMallocHost((void **)&ctx->aring[ring], need));
            ctx->aring_cap[ring] = need;
            hp = ctx->aring[ring];
        } else {
            st = grow_pinned(ctx, need);
            if (st) return st;
            hp = ctx->pinned;
        }
        tp = hp + (size_t)F * 8192;
    }
    DecFrame *hf = reinterpret_cast<DecFrame *>(tp + o_fr);
    uint32_t *hvs = reinterpret_cast<uint32_t *>(tp + o_vs);
    uint64_t *hlp = reinterpret_cast<uint64_t *>(tp + o_lp);
    uint64_t *hjo = reinterpret_cast<uint64_t *>(tp + o_jo);
    uint64_t *hbp = reinterpret_cast<uint64_t *>(tp + o_bp);
    float *hst = reinterpret_cast<float *>(tp + o_st);
    uint32_t *hfc = reinterpret_cast<uint32_t *>(tp + o_fc);
    uint32_t *htp = reinterpret_cast<uint32_t *>(tp + o_tp);
    uint64_t vs = 0, oo = 0, no = 0, bo = 0, jo = 0, co = 0, pb = 0, cho = 0;
    for (uint32_t f = 0; f < F; ++f) {
        const ParsedHeader &H = P[f];
        DecFrame d{};
        d.ctab_off = ~0ull;
        if (d_pos && H.nv && (1ull << H.J) <= H.nv) {
            d.ctab_off = co;
            co += 3ull << H.J;
        }
        const uint8_t *base = d_in + offs[f];
        d.occ_sec = base + H.hb;
        d.occ_bytes = H.occ_bytes;
        const uint8_t *as = base + H.hb + H.occ_bytes;
        d.bw = reinterpret_cast<const uint32_t *>(as + 8);
        d.payload = d.bw + (uint64_t)H.nb * C;
        d.payload_words = (C && H.nv) ? (H.attr_bytes - 8 - 4ull * C * H.nb) / 4 : 0;
        d.occ_off = oo;
        d.n_occ = H.n_occ;
        d.chunk_off = cho;
        if (H.occ_mode == 1) cho += H.occ_aux;
        d.blk_off = bo;
        d.vstart = (uint32_t)vs;
        d.nv = (uint32_t)H.nv;
        d.J = H.J;
        d.mode = H.occ_mode;
        d.aux = H.occ_aux;
        d.chunk = H.chunk;
        d.B = H.B;
        d.nb = H.nb;
        for (int a = 0; a < 3; ++a) d.grid.lo[a] = H.lo[a];
        d.grid.ext = H.ext;
        d.grid.scale = std::ldexp(1.0, (int)H.J) / H.ext;
        d.grid.cell = H.ext / std::ldexp(1.0, (int)H.J);
        uint64_t b2 = 0;
        for (uint32_t lv = 0; lv <= H.J; ++lv) {
            d.lsz[lv] = H.lsz[lv];
            d.boff[lv] = b2;
            if (lv < H.J) {
                d.noff[lv] = no;
                d.pbase[lv] = pb;  // the bytes of a level hold as many set bits as the next level has nodes
                no += H.lsz[lv];
                b2 += H.lsz[lv];
                pb += H.lsz[lv + 1];
            }
        }
        hf[f] = d;
        hvs[f] = (uint32_t)vs;
        hjo[f] = jo;
        hbp[f] = bo;
        for (uint32_t c = 0; c < C; ++c) hst[(uint64_t)f * C + c] = (float)H.steps[H.groups[c]];
        hfc[f] = H.color;
        vs += H.nv;
        oo += H.n_occ;
        if (C && H.nv) {
            bo += (uint64_t)H.nb * C;
            jo += H.nb;
        }
    }
    hvs[F] = (uint32_t)vs;
    hjo[F] = jo;
    hbp[F] = bo;
    for (uint32_t lv = 0; lv <= Jmax; ++lv) {
        uint64_t run = 0;
        for (uint32_t f = 0; f < F; ++f) {
            hlp[(uint64_t)lv * (F + 1) + f] = run;
            if (lv < P[f].J) run += P[f].lsz[lv];
        }
        hlp[(uint64_t)lv * (F + 1) + F] = run;
    }
    std::vector<uint32_t> level_tiles(Jmax);  // CTAs of each level launch
    for (uint32_t lv = 0; lv < Jmax; ++lv) {
        uint32_t run = 0;
        for (uint32_t f = 0; f < F; ++f) {
            htp[(uint64_t)lv * (F + 1) + f] = run;
            if (lv < P[f].J && P[f].lsz[lv]) {
                const uint64_t a0 = hf[f].occ_off + hf[f].boff[lv];
                run += (uint32_t)(occ_tile_first(a0 + P[f].lsz[lv] - 1) - occ_tile_first(a0) + 1);
            }
        }
        htp[(uint64_t)lv * (F + 1) + F] = run;
        level_tiles[lv] = run;
    }
    memcpy(tp + o_nv, &N, 8);
    CK(stage_copy(L.fr, tp + o_fr, sizeof(DecFrame) * F, s));
    CK(stage_copy(L.vstart, tp + o_vs, 4 * (F + 1), s));
    CK(stage_copy(L.lvl_pref, tp + o_lp, 8 * (size_t)(Jmax + 1) * (F + 1), s));
    CK(stage_copy(L.job_off, tp + o_jo, 8 * (F + 1), s));
    CK(stage_copy(L.blk_pref, tp + o_bp, 8 * (F + 1), s));
    CK(stage_copy(L.nvdev, tp + o_nv, 8, s));
    if (Jmax) CK(stage_copy(L.tile_pref, tp + o_tp, 4 * (size_t)Jmax * (F + 1), s));
    if (C) CK(stage_copy(L.steps, tp + o_st, 4 * (size_t)F * C, s));
    if (any_color) {
        CK(stage_copy(L.fcolor, tp + o_fc, 4 * (size_t)F, s));
        for (uint32_t f = 0; f < F; ++f)
            if (P[f].color)
                CK(stage_copy(L.klt + (uint64_t)f * kKltFloats, d_in + offs[f] + P[f].klt_off, 4 * kKltFloats, s));
    }
    DevState *dst = ctx->st;
    CK(dev_memset(dst, 0, 8, s));
    const int sms = ctx->num_sms;

    // a12's RLGR decode needs only the streams' block tables: it runs on s beside a11 and the prelude (the
    // longer branch), which run on the context's high-priority stream
    const bool attrs = C && d_attr;
    cudaStream_t sg = s;
    if (attrs) {
        st = fork_hi_begin(ctx, s, &sg);
        if (st) return st;
        stage_begin(s, kStRlgrDec);
        launch_batch_block_tables(L.fr, F, L.blk_pref, nblk, L.bw_all, sms, s);
        launch_scan_u32_to_u64(L.bw_all, nblk, L.boff_all, L.spart, sms, s);
        launch_rlgr_decode_batch(L.fr, F, L.job_off, jobs, L.bw_all, L.boff_all, L.steps, C, L.Y, dst, s);
        stage_end(s, kStRlgrDec);
    }
    // a11: occupancy bytes of every frame, octree levels, voxel centres
    stage_begin(sg, kStOccDecode);
    launch_batch_occ_bytes(L.fr, F, L.occ, max_occ, sms, sg);
    if (any_rans) launch_batch_rans_decode(L.fr, F, max_nch, chunk_max, L.occ, L.tabs, L.cstart, dst, sg);
    stage_end(sg, kStOccDecode);
    stage_begin(sg, kStOctreeDecode);
    if (ctab_total) launch_batch_centre_tables(L.fr, F, Jmax, L.ctab, sms, sg);
    launch_occ_tile_bases(L.occ, n_occ, L.tsum, L.tbase, L.tpart, sms, sg);
    launch_batch_roots(L.fr, F, L.nodes, L.gap, N, sg);
    for (uint32_t lv = 0; lv < Jmax; ++lv)
        launch_batch_level(L.fr, F, lv, L.tile_pref + (uint64_t)lv * (F + 1), level_tiles[lv], L.occ, n_occ,
                           L.tbase, L.nodes, L.ctab, d_pos, L.gap, dst, sg);
    stage_end(sg, kStOctreeDecode);
    // a12: RAHT schedule, then (after the RLGR branch) the inverse RAHT
    if (attrs) {
        stage_begin(sg, kStPrelude);
        launch_raht_prelude(L.plan, L.gap, dst, L.nvdev, sms, sg);
        stage_end(sg, kStPrelude);
        st = fork_hi_end(ctx, s);
        if (st) return st;
        RahtIO io{};
        io.C = C;
        io.Y = L.Y;
        io.out = d_attr;
        io.pool = L.pool;
        io.frame_shift = 64;
        if (any_color) {
            io.klt = L.klt;
            io.frame_color = L.fcolor;
            io.vstart = L.vstart;
            io.F = F;
            io.yuv_inv = yuv_inverse();
        }
        stage_begin(s, kStRahtInv);
        launch_raht_inverse(L.plan, io, N, sms, s);
        stage_end(s, kStRahtInv);
    }
    CK(cudaGetLastError());
    if (status) {  // the device's status word goes to the caller's word; the staging slot is busy until here
        CK(stage_copy(status, &dst->err, 4, s));
        CK(cudaEventRecord(ctx->aring_ev[ring], s));
        return GSNFS_OK;
    }
    uint32_t *res = reinterpret_cast<uint32_t *>(tp + ((o_end + 63) & ~(size_t)63));
    CK(stage_copy(res, &dst->err, 4, s));
    CK(cudaStreamSynchronize(s));
    return map_dev_error(res[0]);
}

}  // namespace

// ======================================================================
extern "C" {

const char *gsnfs_status_string(gsnfs_status s)
{
    switch (s) {
    case GSNFS_OK: return "ok";
    case GSNFS_ERR_INVALID_ARG: return "invalid argument";
    case GSNFS_ERR_CAPACITY: return "output capacity too small";
    case GSNFS_ERR_CORRUPT: return "corrupt bitstream";
    case GSNFS_ERR_CUDA: return g_last_error[0] ? g_last_error : "CUDA error";
    case GSNFS_ERR_TIMEOUT: return "bounded device wait expired";
    case GSNFS_ERR_OOM: return "device allocation failed";
    case GSNFS_ERR_UNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

gsnfs_status gsnfs_create(gsnfs_ctx **out, int cuda_device)
{
    if (!out) return GSNFS_ERR_INVALID_ARG;
    *out = nullptr;
    DeviceGuard dg(cuda_device);
    int n = 0;
    CK(cudaGetDeviceCount(&n));
    if (cuda_device < 0 || cuda_device >= n) return GSNFS_ERR_INVALID_ARG;
    gsnfs_ctx *c = new (std::nothrow) gsnfs_ctx();
    if (!c) return GSNFS_ERR_OOM;
    c->device = cuda_device;
    cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, cuda_device);
    if (e == cudaSuccess) e = cudaMalloc(&c->st, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMemset(c->st, 0, sizeof(DevState));
    if (e != cudaSuccess) {
        snprintf(g_last_error, sizeof(g_last_error), "gsnfs_create: %s", cudaGetErrorString(e));
        if (c->st) cudaFree(c->st);
        delete c;
        return GSNFS_ERR_CUDA;
    }
    *out = c;
    return GSNFS_OK;
}

void gsnfs_destroy(gsnfs_ctx *ctx)
{
    if (!ctx) return;
    DeviceGuard dg(ctx->device);
    cudaDeviceSynchronize();
    drop_graphs(ctx);
    if (ctx->lod) cudaFree(ctx->lod);
    if (ctx->rnd) cudaFree(ctx->rnd);
    if (ctx->rkeys) cudaFree(ctx->rkeys);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->aux_hi) cudaStreamDestroy(ctx->aux_hi);
    if (ctx->ev_fork_hi) cudaEventDestroy(ctx->ev_fork_hi);
    if (ctx->ev_join_hi) cudaEventDestroy(ctx->ev_join_hi);
    if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
    if (ctx->gev_in) cudaEventDestroy(ctx->gev_in);
    if (ctx->gev_out) cudaEventDestroy(ctx->gev_out);
    if (ctx->arena) cudaFree(ctx->arena);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    for (int k = 0; k < 4; ++k) {
        if (ctx->aring[k]) cudaFreeHost(ctx->aring[k]);
        if (ctx->aring_ev[k]) cudaEventDestroy(ctx->aring_ev[k]);
    }
    if (ctx->st) cudaFree(ctx->st);
    delete ctx;
}

gsnfs_status gsnfs_set_graphs(gsnfs_ctx *ctx, int enable)
{
    if (!ctx) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    if (!enable && ctx->gstream) {
        CK(cudaStreamSynchronize(ctx->gstream));
        drop_graphs(ctx);
    }
    ctx->graphs = enable != 0;
    return GSNFS_OK;
}

gsnfs_status gsnfs_tune_set(gsnfs_ctx *ctx, int which, uint32_t value)
{
    if (!ctx || which < 0 || which > GSNFS_TUNE_RAHT_PIPE) return GSNFS_ERR_INVALID_ARG;
    if (which == GSNFS_TUNE_RAHT_PIPE && value > 2) return GSNFS_ERR_INVALID_ARG;
    if (which == GSNFS_TUNE_RAHT_TILE && value && (!pow2(value) || value < 256 || value > 4096))
        return GSNFS_ERR_INVALID_ARG;
    if (which != GSNFS_TUNE_RAHT_TILE && value > 32) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    if (ctx->tune[which] != value && ctx->gstream) {  // captured graphs hold the old launch shapes
        CK(cudaStreamSynchronize(ctx->gstream));
        drop_graphs(ctx);
    }
    ctx->tune[which] = value;
    return GSNFS_OK;
}

gsnfs_status gsnfs_tune_get(gsnfs_ctx *ctx, int which, uint32_t *value)
{
    if (!ctx || !value || which < 0 || which > GSNFS_TUNE_RAHT_PIPE) return GSNFS_ERR_INVALID_ARG;
    *value = ctx->tune[which];
    return GSNFS_OK;
}

gsnfs_status gsnfs_graph_stats(gsnfs_ctx *ctx, uint64_t *out /* 4: replays, captures, failures, cached */)
{
    if (!ctx || !out) return GSNFS_ERR_INVALID_ARG;
    out[0] = ctx->ghits;
    out[1] = ctx->gcaptures;
    out[2] = ctx->gfailures;
    out[3] = ctx->gcache.size();
    return GSNFS_OK;
}

gsnfs_status gsnfs_max_bitstream_bytes(uint64_t n, uint32_t J, const gsnfs_quant *q, uint64_t *out)
{
    if (!out || J < 1 || J > (uint32_t)kMaxJ) return GSNFS_ERR_INVALID_ARG;
    gsnfs_status st = check_quant(q);
    if (st) return st;
    const uint32_t C = q->num_channels;
    uint64_t b = header_bytes(J, C, C ? q->num_groups : 0, C ? q->color : 0u);
    b += 16 + pad8(occ_bound(n, J));
    if (C) {
        uint64_t nb = (n + q->rlgr_block - 1) / q->rlgr_block;
        b += 8 + 4ull * C * nb + 4ull * C * nb * rlgr_slot_words(q->rlgr_block, true) + 8;
    }
    *out = b;
    return GSNFS_OK;
}

gsnfs_status gsnfs_reserve(gsnfs_ctx *ctx, uint64_t n, uint32_t C, uint32_t J, const gsnfs_quant *q)
{
    if (!ctx || !q || J < 1 || J > (uint32_t)kMaxJ) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    EncodeReq rq;
    gsnfs_quant qq = *q;
    qq.num_channels = C;
    rq.q = &qq;
    rq.n = &n;
    rq.J = &J;
    EncLayout L;
    Carve m(nullptr);
    size_t need = carve_encode(m, L, rq, ctx->num_sms, false, ctx->tune);
    return grow_arena(ctx, need, 0);
}

gsnfs_status gsnfs_encode_frame(gsnfs_ctx *ctx, void *stream, const float *d_pos, const float *d_attr, uint64_t n,
                                uint32_t J, const gsnfs_quant *q, uint8_t *d_bitstream, uint64_t capacity,
                                uint64_t *out_bytes, float *d_recon_pos, float *d_recon_attr, uint64_t *out_nv)
{
    if (!ctx || J < 1 || J > (uint32_t)kMaxJ || !d_bitstream) return GSNFS_ERR_INVALID_ARG;
    gsnfs_status st = check_quant(q);
    if (st) return st;
    if (n > 0 && !d_pos) return GSNFS_ERR_INVALID_ARG;
    if (n > 0 && q->num_channels > 0 && !d_attr) return GSNFS_ERR_INVALID_ARG;
    if ((uintptr_t)d_bitstream % 8 || (uintptr_t)d_attr % 16) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    EncodeReq rq;
    rq.F = 1;
    const float *pp[1] = {d_pos};
    const float *ap[1] = {d_attr};
    rq.pos = pp;
    rq.attr = ap;
    rq.n = &n;
    rq.J = &J;
    rq.q = q;
    rq.out = d_bitstream;
    rq.capacity = capacity;
    rq.recon_pos = d_recon_pos;
    rq.recon_attr = d_recon_attr;
    st = encode_impl(ctx, (cudaStream_t)stream, rq, false);
    if (out_bytes) *out_bytes = rq.total_bytes;
    if (out_nv) *out_nv = rq.nv;
    return st;
}

static gsnfs_status encode_batch_impl(gsnfs_ctx *ctx, void *stream, uint32_t frames, const float *const *h_pos,
                                      const float *const *h_attr, const uint64_t *h_n, const uint32_t *h_J,
                                      uint32_t rungs, const double *h_rung_scale, const gsnfs_quant *q,
                                      uint8_t *d_out, uint64_t capacity, uint64_t *h_offsets, double *h_sq_err,
                                      uint8_t *h_headers = nullptr)
{
    if (!ctx || frames < 1 || frames > (uint32_t)kMaxFrames || rungs < 1 || rungs > (uint32_t)kMaxRungs || !h_pos ||
        !h_n || !h_J || !d_out || !h_offsets)
        return GSNFS_ERR_INVALID_ARG;
    gsnfs_status st = check_quant(q);
    if (st) return st;
    if ((uint64_t)rungs * q->num_channels > 1024) return GSNFS_ERR_UNSUPPORTED;  // rungs x channels threads per block
    for (uint32_t f = 0; f < frames; ++f) {
        if (h_J[f] < 1 || h_J[f] > 19) return GSNFS_ERR_INVALID_ARG;
        if (h_n[f] > 0 && !h_pos[f]) return GSNFS_ERR_INVALID_ARG;
        if (q->num_channels && h_n[f] > 0 && (!h_attr || !h_attr[f] || (uintptr_t)h_attr[f] % 16))
            return GSNFS_ERR_INVALID_ARG;
    }
    if (h_rung_scale)
        for (uint32_t r = 0; r < rungs; ++r)
            if (!(h_rung_scale[r] > 0.0)) return GSNFS_ERR_INVALID_ARG;
    if ((uintptr_t)d_out % 8) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    EncodeReq rq;
    rq.F = frames;
    rq.pos = h_pos;
    rq.attr = h_attr;
    rq.n = h_n;
    rq.J = h_J;
    rq.R = rungs;
    rq.rung_scale = h_rung_scale;
    rq.q = q;
    rq.out = d_out;
    rq.capacity = capacity;
    rq.offsets.assign((size_t)frames * rungs + 1, 0);
    rq.dist = q->num_channels ? h_sq_err : nullptr;
    rq.headers = h_headers;
    st = encode_impl(ctx, (cudaStream_t)stream, rq, false);
    if (st == GSNFS_OK)
        for (size_t i = 0; i < rq.offsets.size(); ++i) h_offsets[i] = rq.offsets[i];
    else if (st == GSNFS_ERR_CAPACITY)
        h_offsets[(size_t)frames * rungs] = rq.total_bytes;
    return st;
}

gsnfs_status gsnfs_encode_batch(gsnfs_ctx *ctx, void *stream, uint32_t frames, const float *const *h_pos,
                                const float *const *h_attr, const uint64_t *h_n, const uint32_t *h_J, uint32_t rungs,
                                const double *h_rung_scale, const gsnfs_quant *q, uint8_t *d_out, uint64_t capacity,
                                uint64_t *h_offsets)
{
    return encode_batch_impl(ctx, stream, frames, h_pos, h_attr, h_n, h_J, rungs, h_rung_scale, q, d_out, capacity,
                             h_offsets, nullptr);
}

gsnfs_status gsnfs_encode_batch_headers(gsnfs_ctx *ctx, void *stream, uint32_t frames, const float *const *h_pos,
                                        const float *const *h_attr, const uint64_t *h_n, const uint32_t *h_J,
                                        uint32_t rungs, const double *h_rung_scale, const gsnfs_quant *q,
                                        uint8_t *d_out, uint64_t capacity, uint64_t *h_offsets, uint8_t *h_headers)
{
    if (!h_headers) return GSNFS_ERR_INVALID_ARG;
    return encode_batch_impl(ctx, stream, frames, h_pos, h_attr, h_n, h_J, rungs, h_rung_scale, q, d_out, capacity,
                             h_offsets, nullptr, h_headers);
}

gsnfs_status gsnfs_encode_batch_rd(gsnfs_ctx *ctx, void *stream, uint32_t frames, const float *const *h_pos,
                                   const float *const *h_attr, const uint64_t *h_n, const uint32_t *h_J,
                                   uint32_t rungs, const double *h_rung_scale, const gsnfs_quant *q, uint8_t *d_out,
                                   uint64_t capacity, uint64_t *h_offsets, double *h_sq_err)
{
    if (!h_sq_err) return GSNFS_ERR_INVALID_ARG;
    return encode_batch_impl(ctx, stream, frames, h_pos, h_attr, h_n, h_J, rungs, h_rung_scale, q, d_out, capacity,
                             h_offsets, h_sq_err);
}

gsnfs_status gsnfs_peek_frame(const uint8_t *header, uint64_t bytes, uint64_t *out_nv, uint32_t *out_C,
                              uint32_t *out_J)
{
    if (!header) return GSNFS_ERR_INVALID_ARG;
    if (bytes < 96) return GSNFS_ERR_CORRUPT;
    // device memory: its first 96 bytes are copied to the host; host, pinned and managed memory are read in place
    // (a pointer the runtime does not know, or no device at all, counts as host memory)
    cudaPointerAttributes pa{};
    const cudaError_t pe = cudaPointerGetAttributes(&pa, header);
    if (pe != cudaSuccess) (void)cudaGetLastError();  // clear only the error this query set
    const bool on_device = pe == cudaSuccess && pa.type == cudaMemoryTypeDevice;
    uint8_t copy[96];
    const uint8_t *h_header = header;
    if (on_device) {
        if (cudaMemcpy(copy, header, sizeof copy, cudaMemcpyDeviceToHost) != cudaSuccess) {
            (void)cudaGetLastError();
            return GSNFS_ERR_CUDA;
        }
        h_header = copy;
    }
    ParsedHeader P{};
    if (rd32(h_header) != kMagic || rd32(h_header + 4) != 1) return GSNFS_ERR_CORRUPT;
    P.J = rd32(h_header + 12);
    P.C = rd32(h_header + 16);
    P.nv = rd64(h_header + 24);
    if (P.J < 1 || P.J > (uint32_t)kMaxJ) return GSNFS_ERR_CORRUPT;
    if (out_nv) *out_nv = P.nv;
    if (out_C) *out_C = P.C;
    if (out_J) *out_J = P.J;
    return GSNFS_OK;
}

gsnfs_status gsnfs_decode_frame(gsnfs_ctx *ctx, void *stream, const uint8_t *d_bitstream, uint64_t bytes, float *d_pos,
                                float *d_attr, uint64_t capacity_nv, uint64_t *out_nv)
{
    if (!ctx || !d_bitstream) return GSNFS_ERR_INVALID_ARG;
    if ((uintptr_t)d_bitstream % 8 || (uintptr_t)d_attr % 16) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    return decode_impl(ctx, (cudaStream_t)stream, d_bitstream, bytes, d_pos, d_attr, capacity_nv, out_nv);
}

gsnfs_status gsnfs_decode_frame_lod(gsnfs_ctx *ctx, void *stream, const uint8_t *d_bitstream, uint64_t bytes,
                                    uint32_t depth, float *d_pos, float *d_attr, uint64_t capacity_nodes,
                                    uint64_t *out_nodes)
{
    if (!ctx || !d_bitstream || !out_nodes) return GSNFS_ERR_INVALID_ARG;
    if ((uintptr_t)d_bitstream % 8 || (uintptr_t)d_attr % 4 || (uintptr_t)d_pos % 4) return GSNFS_ERR_INVALID_ARG;
    if (bytes < 96) return GSNFS_ERR_CORRUPT;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t h[96];
    CK(cudaMemcpyAsync(h, d_bitstream, 96, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    uint64_t nv = 0;
    uint32_t C = 0, J = 0;
    gsnfs_status st = gsnfs_peek_frame(h, 96, &nv, &C, &J);
    if (st) return st;
    if (depth > J) return GSNFS_ERR_INVALID_ARG;
    *out_nodes = 0;
    if (nv == 0) return GSNFS_OK;
    if (depth == J) {  // the nodes are the voxels: the plain decode
        uint64_t n = 0;
        st = decode_impl(ctx, s, d_bitstream, bytes, d_pos, d_attr, capacity_nodes, &n);
        *out_nodes = n;
        return st;
    }
    LodReq r{depth, d_pos, d_attr, capacity_nodes, out_nodes};
    uint64_t n = 0;
    return decode_impl(ctx, s, d_bitstream, bytes, nullptr, d_attr, ~0ull, &n, nullptr, &r);
}

gsnfs_status gsnfs_decode_batch_async(gsnfs_ctx *ctx, void *stream, uint32_t frames, const uint8_t *d_in,
                                      const uint64_t *h_in_offsets, const uint8_t *h_headers, float *d_pos,
                                      float *d_attr, uint64_t capacity_rows, uint64_t *h_out_rows, uint32_t *status)
{
    if (!ctx || !d_in || !h_in_offsets || !h_out_rows || !status || frames == 0 || frames > (uint32_t)kMaxFrames)
        return GSNFS_ERR_INVALID_ARG;
    for (uint32_t f = 0; f < frames; ++f)
        if (h_in_offsets[f + 1] < h_in_offsets[f] || (h_in_offsets[f] % 8)) return GSNFS_ERR_INVALID_ARG;
    if ((uintptr_t)d_in % 8 || (uintptr_t)d_attr % 16 || (uintptr_t)status % 4) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    return decode_batch_impl(ctx, (cudaStream_t)stream, frames, d_in, h_in_offsets, d_pos, d_attr, capacity_rows,
                             h_out_rows, h_headers, status);
}

gsnfs_status gsnfs_decode_batch(gsnfs_ctx *ctx, void *stream, uint32_t frames, const uint8_t *d_in,
                                const uint64_t *h_in_offsets, float *d_pos, float *d_attr, uint64_t capacity_rows,
                                uint64_t *h_out_rows)
{
    if (!ctx || !d_in || !h_in_offsets || !h_out_rows || frames == 0 || frames > (uint32_t)kMaxFrames)
        return GSNFS_ERR_INVALID_ARG;
    for (uint32_t f = 0; f < frames; ++f)
        if (h_in_offsets[f + 1] < h_in_offsets[f] || (h_in_offsets[f] % 8)) return GSNFS_ERR_INVALID_ARG;
    if ((uintptr_t)d_in % 8 || (uintptr_t)d_attr % 16) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    return decode_batch_impl(ctx, (cudaStream_t)stream, frames, d_in, h_in_offsets, d_pos, d_attr, capacity_rows,
                             h_out_rows);
}

}  // extern "C"

// ====================================================== stage entry points
namespace {

__global__ void stage_si_kernel(const uint64_t *sec_bytes, StreamInfo *si, DevState *st)
{
    StreamInfo x{0, 0, sec_bytes[0], 0};
    si[0] = x;
    si[1].off = sec_bytes[0];
    st->total_bytes = sec_bytes[0];
}

struct GeoLayout {
    FrameGrid *grid;
    uint32_t *Jd, *vstart, *vals, *vals_alt, *hist, *seg, *dpart, *lsz, *hoff, *opart;
    const float **posp;
    uint64_t *poff, *keys, *keys_alt, *codes, *occ_off;
    uint8_t *gap, *occ;
};

size_t carve_geo(Carve &cv, GeoLayout &L, uint64_t n, uint64_t occ_cap, int sms)
{
    L.grid = cv.take<FrameGrid>(1);
    L.Jd = cv.take<uint32_t>(1);
    L.posp = (const float **)cv.take<const float *>(1);
    L.poff = cv.take<uint64_t>(2);
    L.vstart = cv.take<uint32_t>(2);
    L.keys = cv.take<uint64_t>(n + 1);
    L.keys_alt = cv.take<uint64_t>(n + 1);
    L.vals = cv.take<uint32_t>(n + 1);
    L.vals_alt = cv.take<uint32_t>(n + 1);
    L.hist = cv.take<uint32_t>(radix_sort_hist_words(n, sms));
    L.codes = cv.take<uint64_t>(n + 1);
    L.seg = cv.take<uint32_t>(n + 2);
    L.gap = cv.take<uint8_t>(n + 2);
    L.dpart = cv.take<uint32_t>(dedup_partial_words(n, sms) + 1);
    L.lsz = cv.take<uint32_t>(22);
    L.hoff = cv.take<uint32_t>(22);
    L.occ_off = cv.take<uint64_t>(2);
    L.opart = cv.take<uint32_t>(occupancy_partial_words(1, sms));
    L.occ = cv.take<uint8_t>(occ_cap + 64);
    return cv.off;
}

}  // namespace

extern "C" {

gsnfs_status gsnfs_voxelize(gsnfs_ctx *ctx, void *stream, const float *d_pos, uint64_t n, uint32_t J,
                            uint64_t *d_codes, double *h_grid, uint64_t *out_nv)
{
    if (!ctx || J < 1 || J > (uint32_t)kMaxJ || (n && (!d_pos || !d_codes))) return GSNFS_ERR_INVALID_ARG;
    if (n >= 0x7FFFFFF0ull) return GSNFS_ERR_UNSUPPORTED;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    GeoLayout L;
    Carve m(nullptr);
    gsnfs_status st = grow_arena(ctx, carve_geo(m, L, n, 0, ctx->num_sms), s);
    if (st) return st;
    Carve cv(ctx->arena);
    carve_geo(cv, L, n, 0, ctx->num_sms);
    st = grow_pinned(ctx, 4096);
    if (st) return st;
    CK(cudaStreamSynchronize(s));
    unsigned char *hp = ctx->pinned;
    ((const float **)hp)[0] = d_pos;
    ((uint64_t *)(hp + 64))[0] = 0;
    ((uint64_t *)(hp + 64))[1] = n;
    ((uint32_t *)(hp + 128))[0] = J;
    CK(cudaMemcpyAsync((void *)L.posp, hp, 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(L.poff, hp + 64, 16, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(L.Jd, hp + 128, 4, cudaMemcpyHostToDevice, s));
    FrameSet fs{1, 64, L.posp, nullptr, L.poff, L.Jd, L.grid};
    launch_voxelize(fs, ctx->st, n, n, L.keys, L.vals, ctx->num_sms, s);
    bool alt = radix_sort(L.keys, L.vals, L.keys_alt, L.vals_alt, L.hist, n, 3 * J, ctx->num_sms, s);
    launch_dedup(alt ? L.keys_alt : L.keys, n, 64, 1, L.codes, L.seg, L.gap, L.vstart, L.dpart, ctx->st,
                 ctx->num_sms, s);
    if (n) CK(cudaMemcpyAsync(d_codes, L.codes, 8 * n, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(hp + 256, L.grid, sizeof(FrameGrid), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hp + 512, &ctx->st->nv_total, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    FrameGrid g;
    memcpy(&g, hp + 256, sizeof(g));
    if (h_grid) {
        for (int a = 0; a < 3; ++a) h_grid[a] = g.lo[a];
        h_grid[3] = g.ext;
    }
    if (out_nv) memcpy(out_nv, hp + 512, 8);
    return GSNFS_OK;
}

gsnfs_status gsnfs_octree_encode(gsnfs_ctx *ctx, void *stream, const uint64_t *d_codes, uint64_t nv, uint32_t J,
                                 uint8_t *d_occ, uint64_t occ_capacity, uint32_t *h_level_sizes,
                                 uint64_t *out_occ_bytes)
{
    if (!ctx || J < 1 || J > (uint32_t)kMaxJ || (nv && !d_codes) || !h_level_sizes) return GSNFS_ERR_INVALID_ARG;
    if (nv >= 0x7FFFFFF0ull) return GSNFS_ERR_UNSUPPORTED;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t ob = occ_bound(nv, J);
    GeoLayout L;
    Carve m(nullptr);
    gsnfs_status st = grow_arena(ctx, carve_geo(m, L, nv, ob, ctx->num_sms), s);
    if (st) return st;
    Carve cv(ctx->arena);
    carve_geo(cv, L, nv, ob, ctx->num_sms);
    st = grow_pinned(ctx, 4096);
    if (st) return st;
    CK(cudaStreamSynchronize(s));
    unsigned char *hp = ctx->pinned;
    ((uint32_t *)hp)[0] = 0;
    ((uint32_t *)hp)[1] = (uint32_t)nv;
    ((uint32_t *)hp)[2] = J;
    CK(cudaMemcpyAsync(L.vstart, hp, 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(L.Jd, hp + 8, 4, cudaMemcpyHostToDevice, s));
    CK(dev_memset(ctx->st, 0, 8, s));
    if (nv) CK(cudaMemcpyAsync(L.codes, d_codes, 8 * nv, cudaMemcpyDeviceToDevice, s));
    launch_gap_levels(L.codes, nv, L.gap, s);
    OccupancyOut oo{L.occ, (ob + 64) & ~(uint64_t)63, L.lsz, L.occ_off, L.hoff, L.opart};
    launch_occupancy(L.codes, L.gap, L.vstart, L.Jd, 1, 64, oo, ctx->st, ctx->num_sms, s);
    CK(cudaMemcpyAsync(hp + 256, L.lsz, 4 * 22, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hp + 512, L.occ_off, 16, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hp + 640, ctx->st, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    if (((uint32_t *)(hp + 640))[0]) return map_dev_error(((uint32_t *)(hp + 640))[0]);
    const uint64_t nb = ((uint64_t *)(hp + 512))[1];
    for (uint32_t d = 0; d <= J; ++d) h_level_sizes[d] = ((uint32_t *)(hp + 256))[d];
    if (out_occ_bytes) *out_occ_bytes = nb;
    if (nb > occ_capacity) return GSNFS_ERR_CAPACITY;
    if (nb) CK(cudaMemcpyAsync(d_occ, L.occ, nb, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return GSNFS_OK;
}

gsnfs_status gsnfs_octree_decode(gsnfs_ctx *ctx, void *stream, const uint8_t *d_occ, uint64_t occ_bytes, uint32_t J,
                                 const uint32_t *h_level_sizes, uint64_t *d_codes)
{
    if (!ctx || J < 1 || J > (uint32_t)kMaxJ || !h_level_sizes) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    ParsedHeader P{};
    P.J = J;
    P.nv = h_level_sizes[J];
    P.n_occ = 0;
    for (uint32_t d = 0; d <= J; ++d) {
        P.lsz[d] = h_level_sizes[d];
        if (d < J) P.n_occ += P.lsz[d];
    }
    if (P.n_occ != occ_bytes) return GSNFS_ERR_CORRUPT;
    if (P.nv == 0) return P.n_occ == 0 ? GSNFS_OK : GSNFS_ERR_CORRUPT;
    if (P.lsz[0] != 1) return GSNFS_ERR_CORRUPT;
    for (uint32_t d = 0; d < J; ++d)
        if (P.lsz[d + 1] < P.lsz[d] || (uint64_t)P.lsz[d + 1] > 8ull * P.lsz[d]) return GSNFS_ERR_CORRUPT;
    if (!d_occ || !d_codes) return GSNFS_ERR_INVALID_ARG;
    P.C = 0;
    P.nb = 0;
    DecLayout L;
    Carve m(nullptr);
    gsnfs_status st = grow_arena(ctx, carve_decode(m, L, P, ctx->num_sms, ctx->tune), s);
    if (st) return st;
    Carve cv(ctx->arena);
    carve_decode(cv, L, P, ctx->num_sms, ctx->tune);
    st = grow_pinned(ctx, 4096);
    if (st) return st;
    CK(dev_memset(ctx->st, 0, 8, s));
    launch_octree_decode(d_occ, P.n_occ, J, P.lsz, L.nodes, L.pref, L.ppart, d_codes, ctx->st, ctx->num_sms, s);
    CK(cudaMemcpyAsync(ctx->pinned, ctx->st, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    return map_dev_error(((uint32_t *)ctx->pinned)[0]);
}

gsnfs_status gsnfs_occupancy_section_encode(gsnfs_ctx *ctx, void *stream, const uint8_t *d_in, uint64_t n,
                                            uint32_t rans_chunk, uint8_t *d_out, uint64_t capacity,
                                            uint64_t *out_bytes)
{
    if (!ctx || (n && !d_in) || !d_out || rans_chunk < 32 || rans_chunk % 32 || rans_chunk > (1u << 20))
        return GSNFS_ERR_INVALID_ARG;
    if ((uintptr_t)d_out % 8) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t nch = (n + rans_chunk - 1) / rans_chunk;
    auto carve = [&](Carve &cv, uint64_t **occ_off, uint64_t **chunk_off, uint16_t **freq, uint32_t **cum,
                     uint32_t **mode, uint32_t **cw, uint32_t **ct, uint32_t **cp, uint8_t **slots, uint64_t **sec,
                     StreamInfo **si) {
        *occ_off = cv.take<uint64_t>(2);
        *chunk_off = cv.take<uint64_t>(2);
        *freq = cv.take<uint16_t>(256);
        *cum = cv.take<uint32_t>(256);
        *mode = cv.take<uint32_t>(1);
        *cw = cv.take<uint32_t>(nch + 1);
        *ct = cv.take<uint32_t>(nch + 1);
        *cp = cv.take<uint32_t>(nch + 1);
        *slots = cv.take<uint8_t>(nch * rans_chunk_slot_bytes(rans_chunk) + 16);
        *sec = cv.take<uint64_t>(1);
        *si = cv.take<StreamInfo>(2);
        return cv.off;
    };
    uint64_t *occ_off, *chunk_off, *sec;
    uint16_t *freq;
    uint32_t *cum, *mode, *cw, *ct, *cp;
    uint8_t *slots;
    StreamInfo *si;
    Carve m(nullptr);
    gsnfs_status st = grow_arena(ctx, carve(m, &occ_off, &chunk_off, &freq, &cum, &mode, &cw, &ct, &cp, &slots, &sec, &si), s);
    if (st) return st;
    Carve cv(ctx->arena);
    carve(cv, &occ_off, &chunk_off, &freq, &cum, &mode, &cw, &ct, &cp, &slots, &sec, &si);
    st = grow_pinned(ctx, 4096);
    if (st) return st;
    CK(cudaStreamSynchronize(s));
    uint64_t *hp = (uint64_t *)ctx->pinned;
    hp[0] = 0;
    hp[1] = n;
    CK(cudaMemcpyAsync(occ_off, hp, 16, cudaMemcpyHostToDevice, s));
    CK(dev_memset(ctx->st, 0, 8, s));
    RansFrames rf{1, d_in, occ_off, rans_chunk, chunk_off, freq, cum, mode, cw, ct, cp, slots, sec};
    launch_rans_encode(rf, ctx->st, nch, ctx->num_sms, s);
    stage_si_kernel<<<1, 1, 0, s>>>(sec, si, ctx->st);
    count_launch();
    HdrParams hpar{1, 1, 0, 0, 1, rans_chunk, 0u, 0.5, capacity};
    OccCopyArgs oa{d_in, occ_off, mode, chunk_off, freq, cw, ct, cp, slots, rans_chunk_slot_bytes(rans_chunk)};
    occ_copy_kernel<<<dim3(ctx->num_sms, 1), 256, 0, s>>>(hpar, oa, si, ctx->st, d_out);
    count_launch();
    CK(cudaMemcpyAsync(hp + 8, sec, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    if (out_bytes) *out_bytes = hp[8];
    return hp[8] > capacity ? GSNFS_ERR_CAPACITY : GSNFS_OK;
}

gsnfs_status gsnfs_occupancy_section_decode(gsnfs_ctx *ctx, void *stream, const uint8_t *d_sec, uint64_t sec_bytes,
                                            uint8_t *d_out, uint64_t n)
{
    if (!ctx || !d_sec || (n && !d_out) || sec_bytes < 16) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    gsnfs_status st = grow_pinned(ctx, 4096);
    if (st) return st;
    CK(cudaStreamSynchronize(s));
    uint8_t *hp = ctx->pinned;
    CK(cudaMemcpyAsync(hp, d_sec, sec_bytes < 24 ? 16 : 24, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ParsedHeader P{};
    P.n_occ = n;
    P.occ_bytes = sec_bytes;
    P.C = 0;
    P.nv = 0;
    st = parse_sections(hp, nullptr, P);
    if (st) return st;
    CK(dev_memset(ctx->st, 0, 8, s));
    if (P.occ_mode == 0) {
        if (n) CK(cudaMemcpyAsync(d_out, d_sec + 16, n, cudaMemcpyDeviceToDevice, s));
    } else if (P.occ_mode == 2) {
        launch_fill(d_out, n, (uint8_t)P.occ_aux, s);
    } else {
        Carve m(nullptr);
        m.take<uint32_t>(rans_table_words());
        st = grow_arena(ctx, m.off, s);
        if (st) return st;
        Carve cv(ctx->arena);
        uint32_t *tabs = cv.take<uint32_t>(rans_table_words());
        launch_rans_decode(d_sec, sec_bytes, n, P.occ_aux, P.chunk, d_out, tabs, ctx->st, ctx->num_sms, s);
    }
    CK(cudaMemcpyAsync(hp + 64, ctx->st, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    return map_dev_error(((uint32_t *)(hp + 64))[0]);
}

gsnfs_status gsnfs_raht_plan_create(gsnfs_ctx *ctx, void *stream, const uint64_t *d_codes, uint64_t nv, uint32_t J,
                                    uint32_t C, gsnfs_raht_plan **out)
{
    if (!ctx || !out || J < 1 || J > (uint32_t)kMaxJ || C < 1 || C > (uint32_t)kMaxC || (nv && !d_codes))
        return GSNFS_ERR_INVALID_ARG;
    if (nv >= 0x7FFFFFF0ull) return GSNFS_ERR_UNSUPPORTED;
    *out = nullptr;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    gsnfs_raht_plan *pl = new (std::nothrow) gsnfs_raht_plan();
    if (!pl) return GSNFS_ERR_OOM;
    pl->ctx = ctx;
    pl->nv = nv;
    pl->C = C;
    pl->J = J;
    uint8_t *gap = nullptr;
    uint64_t *nvd = nullptr;
    auto carve = [&](Carve &cv) {
        carve_plan(cv, pl->dev, nv, raht_tile_size(C), ctx->tune);
        uint64_t elems, tiles, surv;
        raht_plan_sizes(nv, pl->dev.T, &elems, &tiles, &surv);
        pl->dev.bf_w = cv.take<uint2>(tiles * pl->dev.T);
        pl->surv_rows = surv;
        pl->pool = cv.take<float>(surv * C);
        pl->qparams = cv.take<float>(2 * (uint64_t)C);
        pl->st = cv.take<DevState>(1);
        gap = cv.take<uint8_t>(nv + 2);
        nvd = cv.take<uint64_t>(1);
        return cv.off;
    };
    Carve m(nullptr);
    size_t need = carve(m);
    cudaError_t e = cudaMalloc(&pl->mem, need);
    if (e != cudaSuccess) {
        delete pl;
        return GSNFS_ERR_OOM;
    }
    Carve cv(pl->mem);
    carve(cv);
    CK(dev_memset(pl->st, 0, sizeof(DevState), s));
    CK(cudaMemcpyAsync(nvd, &pl->nv, 8, cudaMemcpyHostToDevice, s));
    if (nv) launch_gap_levels(d_codes, nv, gap, s);
    launch_raht_prelude(pl->dev, gap, pl->st, nvd, ctx->num_sms, s);
    CK(cudaStreamSynchronize(s));
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(g_last_error, sizeof(g_last_error), "raht plan: %s", cudaGetErrorString(e));
        cudaFree(pl->mem);
        delete pl;
        return GSNFS_ERR_CUDA;
    }
    *out = pl;
    return GSNFS_OK;
}

void gsnfs_raht_plan_destroy(gsnfs_raht_plan *plan)
{
    if (!plan) return;
    DeviceGuard dg(plan->ctx->device);
    cudaDeviceSynchronize();
    cudaFree(plan->mem);
    if (plan->pool64) cudaFree(plan->pool64);
    delete plan;
}

gsnfs_status gsnfs_raht_forward(gsnfs_raht_plan *plan, void *stream, const float *d_in, float *d_out)
{
    if (!plan || (plan->nv && (!d_in || !d_out))) return GSNFS_ERR_INVALID_ARG;
    if ((uintptr_t)d_in % 16 || (uintptr_t)d_out % 16) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(plan->ctx->device);
    if (plan->nv == 0) return GSNFS_OK;
    RahtIO io{};
    io.C = plan->C;
    io.in = d_in;
    io.Y = d_out;
    io.pool = plan->pool;
    io.frame_shift = 64;
    launch_raht_forward(plan->dev, io, plan->nv, plan->ctx->num_sms, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return GSNFS_OK;
}

gsnfs_status gsnfs_raht_inverse(gsnfs_raht_plan *plan, void *stream, const float *d_in, float *d_out,
                                const gsnfs_quant *q)
{
    if (!plan || (plan->nv && (!d_in || !d_out))) return GSNFS_ERR_INVALID_ARG;
    if ((uintptr_t)d_in % 16 || (uintptr_t)d_out % 16) return GSNFS_ERR_INVALID_ARG;
    if (q) {
        gsnfs_status st = check_quant(q);
        if (st) return st;
        if (q->num_channels != plan->C) return GSNFS_ERR_INVALID_ARG;
    }
    DeviceGuard dg(plan->ctx->device);
    if (plan->nv == 0) return GSNFS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    RahtIO io{};
    io.C = plan->C;
    io.Y = const_cast<float *>(d_in);
    io.out = d_out;
    io.pool = plan->pool;
    io.frame_shift = 64;
    if (q) {
        std::vector<float> h(2 * plan->C);
        for (uint32_t c = 0; c < plan->C; ++c) {
            const double stp = q->steps[q->channel_group[c]];
            h[c] = (float)(1.0 / stp);
            h[plan->C + c] = (float)stp;
        }
        CK(cudaMemcpyAsync(plan->qparams, h.data(), 8 * plan->C, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        io.inv_step = plan->qparams;
        io.step = plan->qparams + plan->C;
        io.tau = (float)q->tau;
    }
    launch_raht_inverse(plan->dev, io, plan->nv, plan->ctx->num_sms, s);
    CK(cudaGetLastError());
    return GSNFS_OK;
}

namespace {

// survivor pool and step tables of the FP64 transforms, allocated on first use
gsnfs_status plan_f64_buffers(gsnfs_raht_plan *plan)
{
    if (plan->pool64) return GSNFS_OK;
    void *m = nullptr;
    const size_t bytes = (plan->surv_rows * plan->C + 2 * (uint64_t)plan->C) * sizeof(double);
    if (cudaMalloc(&m, bytes) != cudaSuccess) {
        cudaGetLastError();
        return GSNFS_ERR_OOM;
    }
    plan->pool64 = (double *)m;
    plan->qparams64 = plan->pool64 + plan->surv_rows * plan->C;
    return GSNFS_OK;
}

}  // namespace

gsnfs_status gsnfs_raht_forward_f64(gsnfs_raht_plan *plan, void *stream, const double *d_in, double *d_out)
{
    if (!plan || (plan->nv && (!d_in || !d_out))) return GSNFS_ERR_INVALID_ARG;
    if ((uintptr_t)d_in % 16 || (uintptr_t)d_out % 16) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(plan->ctx->device);
    if (plan->nv == 0) return GSNFS_OK;
    gsnfs_status st = plan_f64_buffers(plan);
    if (st) return st;
    RahtIOT<double> io{};
    io.C = plan->C;
    io.in = d_in;
    io.Y = d_out;
    io.pool = plan->pool64;
    io.frame_shift = 64;
    launch_raht_forward(plan->dev, io, plan->nv, plan->ctx->num_sms, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return GSNFS_OK;
}

gsnfs_status gsnfs_raht_inverse_f64(gsnfs_raht_plan *plan, void *stream, const double *d_in, double *d_out,
                                    const gsnfs_quant *q)
{
    if (!plan || (plan->nv && (!d_in || !d_out))) return GSNFS_ERR_INVALID_ARG;
    if ((uintptr_t)d_in % 16 || (uintptr_t)d_out % 16) return GSNFS_ERR_INVALID_ARG;
    if (q) {
        gsnfs_status st = check_quant(q);
        if (st) return st;
        if (q->num_channels != plan->C) return GSNFS_ERR_INVALID_ARG;
    }
    DeviceGuard dg(plan->ctx->device);
    if (plan->nv == 0) return GSNFS_OK;
    gsnfs_status st = plan_f64_buffers(plan);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    RahtIOT<double> io{};
    io.C = plan->C;
    io.Y = const_cast<double *>(d_in);
    io.out = d_out;
    io.pool = plan->pool64;
    io.frame_shift = 64;
    if (q) {
        std::vector<double> h(2 * plan->C);
        for (uint32_t c = 0; c < plan->C; ++c) {
            const double stp = q->steps[q->channel_group[c]];
            h[c] = 1.0 / stp;
            h[plan->C + c] = stp;
        }
        CK(cudaMemcpyAsync(plan->qparams64, h.data(), 16 * plan->C, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        io.inv_step = plan->qparams64;
        io.step = plan->qparams64 + plan->C;
        io.tau = q->tau;
    }
    launch_raht_inverse(plan->dev, io, plan->nv, plan->ctx->num_sms, s);
    CK(cudaGetLastError());
    return GSNFS_OK;
}

uint32_t gsnfs_rlgr_slot_words(uint32_t B) { return rlgr_slot_words(B, true); }

gsnfs_status gsnfs_rlgr_encode_indices(gsnfs_ctx *ctx, void *stream, const int32_t *d_q, uint64_t nv, uint32_t C,
                                       uint32_t B, uint32_t *d_slots, uint32_t *d_block_words)
{
    if (!ctx || !pow2(B) || B < 32 || B > 65536 || C < 1 || C > (uint32_t)kMaxC) return GSNFS_ERR_INVALID_ARG;
    if (nv && (!d_q || !d_slots || !d_block_words)) return GSNFS_ERR_INVALID_ARG;
    if (nv >= 0x7FFFFFF0ull) return GSNFS_ERR_UNSUPPORTED;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    gsnfs_status st = grow_pinned(ctx, 4096);
    if (st) return st;
    Carve m(nullptr);
    m.take<uint32_t>(4);
    m.take<uint64_t>(4);
    m.take<uint64_t>(4);
    m.take<uint32_t>(4);
    st = grow_arena(ctx, m.off, s);
    if (st) return st;
    Carve cv(ctx->arena);
    uint32_t *vstart = cv.take<uint32_t>(4);
    uint64_t *job_off = cv.take<uint64_t>(4);
    uint64_t *blk_off = cv.take<uint64_t>(4);
    uint32_t *ovf = cv.take<uint32_t>(4);
    CK(cudaStreamSynchronize(s));
    uint32_t *hp = (uint32_t *)ctx->pinned;
    hp[0] = 0;
    hp[1] = (uint32_t)nv;
    CK(cudaMemcpyAsync(vstart, hp, 8, cudaMemcpyHostToDevice, s));
    CK(dev_memset(ovf, 0, 16, s));
    launch_rlgr_offsets(vstart, 1, B, 1, C, job_off, blk_off, s);
    launch_rlgr_encode_indices(d_q, vstart, C, B, d_slots, rlgr_slot_words(B, true), d_block_words, job_off, blk_off,
                               (nv + B - 1) / B, ovf, s);
    CK(cudaGetLastError());
    return GSNFS_OK;
}

gsnfs_status gsnfs_rlgr_decode_indices(gsnfs_ctx *ctx, void *stream, const uint32_t *d_slots,
                                       const uint32_t *d_block_words, uint64_t nv, uint32_t C, uint32_t B,
                                       int32_t *d_q)
{
    if (!ctx || !pow2(B) || B < 32 || B > 65536 || C < 1 || C > (uint32_t)kMaxC) return GSNFS_ERR_INVALID_ARG;
    if (nv && (!d_q || !d_slots || !d_block_words)) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    gsnfs_status st = grow_pinned(ctx, 4096);
    if (st) return st;
    CK(dev_memset(ctx->st, 0, 8, s));
    const uint32_t sw = rlgr_slot_words(B, true);
    const uint64_t nb = (nv + B - 1) / B;
    launch_rlgr_decode_indices(d_slots, (uint64_t)C * nb * sw, d_block_words, sw, nv, C, B, d_q, ctx->st, s);
    CK(cudaMemcpyAsync(ctx->pinned, ctx->st, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    return map_dev_error(((uint32_t *)ctx->pinned)[0]);
}

}  // extern "C"

extern "C" {

uint64_t gsnfs_launch_count(void) { return g_launches.load(); }

gsnfs_status gsnfs_profile_enable(int enable)
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.on = enable != 0;
    return GSNFS_OK;
}

int gsnfs_profile_stage_names(const char **names, int cap)
{
    for (int i = 0; i < cap && i < kStCount; ++i) names[i] = kStageNames[i];
    return kStCount;
}

gsnfs_status gsnfs_profile_read(double *ms, uint64_t *count, int cap)
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (auto &r : g_prof.done) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess) return GSNFS_ERR_CUDA;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            g_prof.ms[r.id] += t;
            g_prof.cnt[r.id] += 1;
        }
        g_prof.pool.push_back(r.a);
        g_prof.pool.push_back(r.b);
    }
    g_prof.done.clear();
    for (int i = 0; i < cap && i < kStCount; ++i) {
        if (ms) ms[i] = g_prof.ms[i];
        if (count) count[i] = g_prof.cnt[i];
        g_prof.ms[i] = 0;
        g_prof.cnt[i] = 0;
    }
    return GSNFS_OK;
}

}  // extern "C"

namespace {
// grows a context-owned scratch buffer to at least `need` bytes (contents not kept)
gsnfs_status grow(void **buf, size_t *cap, size_t need)
{
    if (need <= *cap) return GSNFS_OK;
    if (*buf) CK(cudaFree(*buf));
    *buf = nullptr;
    *cap = 0;
    CK(cudaMalloc(buf, need));
    *cap = need;
    return GSNFS_OK;
}
}  // namespace

gsnfs_status gsnfs_render(gsnfs_ctx *ctx, void *stream, const float *d_pos, const float *d_attr, uint64_t n,
                          const gsnfs_camera *cam, float *d_image)
{
    if (!ctx || !cam || !d_image || (n && (!d_pos || !d_attr))) return GSNFS_ERR_INVALID_ARG;
    if ((uintptr_t)d_pos % 4 || (uintptr_t)d_attr % 4 || (uintptr_t)d_image % 4) return GSNFS_ERR_INVALID_ARG;
    if (cam->width == 0 || cam->height == 0 || cam->width > 16384 || cam->height > 16384) return GSNFS_ERR_INVALID_ARG;
    if (!(cam->znear > 0.0) || n >= (1ull << 32)) return GSNFS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = ctx->num_sms;
    RenderCam rc;
    const double *V = cam->view;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) rc.R[3 * r + c] = V[4 * r + c];
        rc.t[r] = V[4 * r + 3];
    }
    for (int c = 0; c < 3; ++c)  // camera centre -R^T t
        rc.campos[c] = -(V[c] * V[3] + V[4 + c] * V[7] + V[8 + c] * V[11]);
    rc.fx = cam->fx;
    rc.fy = cam->fy;
    rc.cx = cam->cx;
    rc.cy = cam->cy;
    rc.znear = cam->znear;
    rc.W = (int)cam->width;
    rc.H = (int)cam->height;
    rc.TX = (rc.W + 15) / 16;
    rc.TY = (rc.H + 15) / 16;
    for (int c = 0; c < 3; ++c) rc.bg[c] = (float)cam->background[c];
    const uint64_t tiles = (uint64_t)rc.TX * rc.TY;
    const uint64_t m = n ? n : 1;
    auto carve1 = [&](Carve &cv, void **sp, float **depth, int4 **rect, uint32_t **count, uint64_t **offs,
                      uint64_t **part, uint2 **ranges) {
        *sp = cv.take<unsigned char>(m * render_splat_bytes());
        *depth = cv.take<float>(m);
        *rect = cv.take<int4>(m);
        *count = cv.take<uint32_t>(m);
        *offs = cv.take<uint64_t>(m + 2);
        *part = cv.take<uint64_t>(scan_partial_words(m, sms) + 1);
        *ranges = cv.take<uint2>(tiles);
        return cv.off;
    };
    void *sp;
    float *depth;
    int4 *rect;
    uint32_t *count;
    uint64_t *offs, *part;
    uint2 *ranges;
    Carve m1(nullptr);
    gsnfs_status st = grow(&ctx->rnd, &ctx->rnd_cap, carve1(m1, &sp, &depth, &rect, &count, &offs, &part, &ranges));
    if (st) return st;
    Carve c1(ctx->rnd);
    carve1(c1, &sp, &depth, &rect, &count, &offs, &part, &ranges);
    uint64_t total = 0;
    if (n) {
        launch_render_prepare(d_pos, d_attr, n, rc, sp, depth, rect, count, offs, part, sms, s);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&total, offs + n, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (total >= (1ull << 32)) return GSNFS_ERR_CAPACITY;
    }
    const uint64_t mt = total ? total : 1;
    auto carve2 = [&](Carve &cv, uint64_t **k, uint32_t **v, uint64_t **ka, uint32_t **va, uint32_t **hist) {
        *k = cv.take<uint64_t>(mt);
        *ka = cv.take<uint64_t>(mt);
        *v = cv.take<uint32_t>(mt);
        *va = cv.take<uint32_t>(mt);
        *hist = cv.take<uint32_t>(radix_sort_hist_words(mt, sms));
        return cv.off;
    };
    uint64_t *keys, *keys_alt;
    uint32_t *vals, *vals_alt, *hist;
    Carve m2(nullptr);
    st = grow(&ctx->rkeys, &ctx->rkeys_cap, carve2(m2, &keys, &vals, &keys_alt, &vals_alt, &hist));
    if (st) return st;
    Carve c2(ctx->rkeys);
    carve2(c2, &keys, &vals, &keys_alt, &vals_alt, &hist);
    launch_render_tiles(n, rect, depth, count, offs, total, rc, sp, keys, vals, keys_alt, vals_alt, hist, ranges,
                        d_image, sms, s);
    CK(cudaGetLastError());
    return GSNFS_OK;
}
