// LSD radix sort of (64-bit Morton key, 32-bit point index) pairs
// (Algorithm 1: "RadixSort" of the Morton codes).  Only the 3J significant
// key bits are sorted, 8 bits per pass; the frames of a batch, which arrive
// grouped, are sorted as separate segments so that their id bits need no pass.
//
// Each pass is reduce-then-scan: every CTA owns one contiguous chunk of the
// array, counts its digits (upsweep), one CTA scans the digit-major count
// matrix, and every CTA re-reads its chunk tile by tile, ranks keys stably
// with warp match/popc, stages the tile digit-sorted in shared memory and
// writes it out in runs (downsweep).  No CTA waits on another CTA.
#include "kernels.cuh"

namespace gsnfs {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kKeysPerThread = 8;
constexpr int kTile = kThreads * kKeysPerThread;  // 2048
constexpr int kRadix = 256;
constexpr int kCtasPerSm = 4;  // downsweep CTAs resident per SM (registers capped to fit)

struct SortGeom {
    uint32_t P;       // CTAs
    uint64_t chunk;   // elements per CTA
};

SortGeom sort_geom(uint64_t n, int num_sms)
{
    SortGeom g;
    uint64_t tiles = (n + kTile - 1) / kTile;
    uint64_t pmax = (uint64_t)num_sms * kCtasPerSm;
    g.P = (uint32_t)(tiles < 1 ? 1 : (tiles < pmax ? tiles : pmax));
    g.chunk = (n + g.P - 1) / g.P;
    return g;
}

// CTA p sorts elements [b, e): p * chunk onwards, or cta_lo[p] .. cta_lo[p + 1]
// when the array is cut into independently sorted segments
__device__ __forceinline__ void cta_range(const uint64_t *cta_lo, uint64_t chunk, uint64_t n, uint64_t &b,
                                          uint64_t &e)
{
    if (cta_lo) {
        b = cta_lo[blockIdx.x];
        e = cta_lo[blockIdx.x + 1];
    } else {
        b = (uint64_t)blockIdx.x * chunk;
        e = b + chunk;
        if (e > n) e = n;
    }
}

__global__ void __launch_bounds__(kThreads) upsweep_kernel(const uint64_t *__restrict__ keys, uint64_t n,
                                                           uint32_t shift, uint64_t chunk, uint32_t *hist,
                                                           const uint64_t *__restrict__ cta_lo)
{
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    uint64_t b, e;
    cta_range(cta_lo, chunk, n, b, e);
    for (uint64_t i = b + threadIdx.x; i < e; i += kThreads) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
    __syncthreads();
    hist[(uint64_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// hist is digit-major [256][P]: warp d scans row d in place (exclusive) and
// stores the digit total at hist[256 * P + d]
__global__ void __launch_bounds__(256) scan_cols_kernel(uint32_t *hist, uint32_t P)
{
    const uint32_t d = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    uint32_t *row = hist + (uint64_t)d * P;
    uint32_t run = 0;
    for (uint32_t b = 0; b < P; b += 32) {
        const uint32_t c = b + lane;
        const uint32_t v = (c < P) ? row[c] : 0u;
        const uint32_t inc = warp_inclusive_sum(v);
        if (c < P) row[c] = run + inc - v;
        run += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
    if (lane == 0) hist[(uint64_t)kRadix * P + d] = run;
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm) downsweep_kernel(const uint64_t *__restrict__ keys,
                                                             const uint32_t *__restrict__ vals, uint64_t n,
                                                             uint32_t shift, uint64_t chunk,
                                                             const uint32_t *__restrict__ hist,
                                                             uint64_t *__restrict__ keys_out,
                                                             uint32_t *__restrict__ vals_out,
                                                             const uint64_t *__restrict__ cta_lo,
                                                             const uint32_t *__restrict__ cta_seg)
{
    __shared__ uint32_t s_base[kRadix];
    __shared__ uint32_t s_wcnt[kWarps][kRadix];
    __shared__ uint32_t s_toff[kRadix];
    __shared__ uint64_t s_keys[kTile];
    __shared__ uint32_t s_vals[kTile];
    __shared__ uint32_t s_scan[33];

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t P = gridDim.x;
    if (!cta_seg) {  // digit d starts after all smaller digits, then after the same digit of earlier CTAs
        uint32_t tot;
        const uint32_t doff = block_exclusive_sum<uint32_t>(hist[(uint64_t)kRadix * P + tid], s_scan, &tot);
        s_base[tid] = doff + hist[(uint64_t)tid * P + blockIdx.x];
    } else {  // the same within this CTA's segment (CTAs p0 .. p1 - 1), which starts at element cta_lo[p0]
        const uint32_t p0 = cta_seg[2 * blockIdx.x], p1 = cta_seg[2 * blockIdx.x + 1];
        const uint32_t c0 = hist[(uint64_t)tid * P + p0];
        const uint32_t c1 = p1 < P ? hist[(uint64_t)tid * P + p1] : hist[(uint64_t)kRadix * P + tid];
        uint32_t tot;
        const uint32_t doff = block_exclusive_sum<uint32_t>(c1 - c0, s_scan, &tot);
        s_base[tid] = (uint32_t)cta_lo[p0] + doff + (hist[(uint64_t)tid * P + blockIdx.x] - c0);
    }
    uint64_t cb, ce;
    cta_range(cta_lo, chunk, n, cb, ce);
    const uint32_t ltmask = lanemask_lt();
    // Five barriers per tile.  Thread t owns digit t's column of the warp counters and digit t's output base:
    // it zeroes the column once the tile's ranks are placed (the write-out does not read the counters) and
    // advances the base after the write-out, so neither needs a barrier or a pass of its own.
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) s_wcnt[ww][tid] = 0;
    __syncthreads();
    for (uint64_t t0 = cb; t0 < ce; t0 += kTile) {
        uint64_t k[kKeysPerThread];
        uint32_t v[kKeysPerThread], rk[kKeysPerThread];
        uint32_t dg[kKeysPerThread];
#pragma unroll
        for (int r = 0; r < kKeysPerThread; ++r) {
            uint64_t p = t0 + (uint64_t)w * (32 * kKeysPerThread) + (uint64_t)r * 32 + lane;
            bool ok = p < ce;
            k[r] = ok ? keys[p] : 0ull;
            v[r] = ok ? vals[p] : 0u;
            uint32_t d = ok ? (uint32_t)((k[r] >> shift) & 0xFF) : (kRadix + lane);
            dg[r] = d;
            uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
            uint32_t before = __popc(peers & ltmask);
            uint32_t base = ok ? s_wcnt[w][d] : 0u;
            rk[r] = base + before;
            __syncwarp();
            if (ok && before == 0) s_wcnt[w][d] = base + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive prefix over warps, then the tile's exclusive prefix over digits
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            uint32_t c = s_wcnt[ww][tid];
            s_wcnt[ww][tid] = run;
            run += c;
        }
        const uint32_t inc = warp_inclusive_sum(run);
        if (lane == 31) s_scan[w] = inc;
        __syncthreads();
        uint32_t woff = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) woff += ww < w ? s_scan[ww] : 0u;
        s_toff[tid] = woff + inc - run;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kKeysPerThread; ++r) {
            if (dg[r] < kRadix) {
                uint32_t slot = s_toff[dg[r]] + s_wcnt[w][dg[r]] + rk[r];
                s_keys[slot] = k[r];
                s_vals[slot] = v[r];
            }
        }
        __syncthreads();
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) s_wcnt[ww][tid] = 0;
        uint32_t cnt = (uint32_t)((ce - t0) < (uint64_t)kTile ? (ce - t0) : (uint64_t)kTile);
        for (uint32_t slot = tid; slot < cnt; slot += kThreads) {
            uint64_t key = s_keys[slot];
            uint32_t d = (uint32_t)((key >> shift) & 0xFF);
            uint64_t op = (uint64_t)s_base[d] + (slot - s_toff[d]);
            keys_out[op] = key;
            vals_out[op] = s_vals[slot];
        }
        __syncthreads();
        s_base[tid] += run;  // read again only after the next tile's barriers
    }
}

}  // namespace

uint64_t radix_sort_hist_words(uint64_t n, int num_sms, uint32_t segments)
{
    return (uint64_t)kRadix * (sort_geom(n, num_sms).P + segments) + kRadix;
}

uint64_t radix_sort_max_ctas(uint64_t n, int num_sms) { return sort_geom(n, num_sms).P; }

uint32_t radix_sort_segment_table(const uint64_t *seg_lo, uint32_t segments, int num_sms, uint64_t *cta_lo,
                                  uint32_t *cta_seg)
{
    const uint64_t n = seg_lo[segments];
    const SortGeom g = sort_geom(n, num_sms);
    uint32_t P = 0;
    for (uint32_t f = 0; f < segments; ++f) {
        const uint64_t b = seg_lo[f], e = seg_lo[f + 1];
        const uint32_t p0 = P;
        for (uint64_t x = b; x < e; x += g.chunk) cta_lo[P++] = x;
        for (uint32_t p = p0; p < P; ++p) cta_seg[2 * p] = p0;
        for (uint32_t p = p0; p < P; ++p) cta_seg[2 * p + 1] = P;
    }
    cta_lo[P] = n;
    return P;
}

static bool sort_passes(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint32_t *hist,
                        uint64_t n, uint32_t nbits, uint32_t P, uint64_t chunk, const uint64_t *cta_lo,
                        const uint32_t *cta_seg, cudaStream_t s)
{
    uint64_t *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    bool flipped = false;
    for (uint32_t shift = 0; shift < nbits; shift += 8) {
        upsweep_kernel<<<P, kThreads, 0, s>>>(ki, n, shift, chunk, hist, cta_lo);
        count_launch();
        scan_cols_kernel<<<kRadix / 8, 256, 0, s>>>(hist, P);
        count_launch();
        downsweep_kernel<<<P, kThreads, 0, s>>>(ki, vi, n, shift, chunk, hist, ko, vo, cta_lo, cta_seg);
        count_launch();
        uint64_t *tk = ki;
        ki = ko;
        ko = tk;
        uint32_t *tv = vi;
        vi = vo;
        vo = tv;
        flipped = !flipped;
    }
    return flipped;
}

bool radix_sort(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint32_t *hist,
                uint64_t n, uint32_t nbits, int num_sms, cudaStream_t s)
{
    if (n <= 1 || nbits == 0) return false;
    const SortGeom g = sort_geom(n, num_sms);
    return sort_passes(keys, vals, keys_alt, vals_alt, hist, n, nbits, g.P, g.chunk, nullptr, nullptr, s);
}

bool radix_sort_segments(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint32_t *hist,
                         uint64_t n, uint32_t nbits, uint32_t ctas, const uint64_t *cta_lo, const uint32_t *cta_seg,
                         int num_sms, cudaStream_t s)
{
    if (n <= 1 || nbits == 0 || ctas == 0) return false;
    return sort_passes(keys, vals, keys_alt, vals_alt, hist, n, nbits, ctas, sort_geom(n, num_sms).chunk, cta_lo,
                       cta_seg, s);
}

}  // namespace gsnfs
