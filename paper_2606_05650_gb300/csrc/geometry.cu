// Geometry: cluster identification (Sec. 2.2 "Voxelization"), octree
// occupancy bytes (Sec. 2.2 "Octree construction" / "Bitstream generation",
// Algorithm 1) and octree decoding (Sec. 2.3, Algorithms 2-3).
//
// Occupancy without per-level passes.  For ascending distinct codes m_v the
// "gap level" g_v = msb(m_{v-1} xor m_v) + 1 is the binary level where v and
// v-1 first share an ancestor (g = kInfLevel at a frame start).  Voxel v
// starts a new octree node at height h (depth J-h) iff g_v > 3h, i.e. for
// h <= s_v = floor((g_v - 1) / 3).  So the level lists L_d of Algorithm 1 are
// the prefix counts of (s_v >= h), and the occupancy byte of a node is the OR
// of (1 << child digit) over its children, which every child contributes to
// its parent's byte.  One pass over L_J yields every level: counts per height
// (upsweep), per-frame scans, then ranks by warp ballots and warp-aggregated
// atomic ORs into the zeroed byte stream (downsweep).  The byte order is the
// breadth-first order of Algorithm 1 (depth 0 first, nodes in Morton order).
#include "kernels.cuh"

namespace gsnfs {

namespace {

constexpr int kThreads = 256;
constexpr int kH = 22;  // heights 0..21

struct Range {
    uint64_t b, e;
};

__device__ __forceinline__ Range cta_range(uint64_t vs, uint64_t ve, uint32_t x, uint32_t X)
{
    uint64_t len = (ve - vs + X - 1) / X;
    Range r;
    r.b = vs + (uint64_t)x * len;
    r.e = r.b + len;
    if (r.b > ve) r.b = ve;
    if (r.e > ve) r.e = ve;
    return r;
}

// ---------------------------------------------------------------- dedup ---
__global__ void __launch_bounds__(kThreads) dedup_up_kernel(const uint64_t *__restrict__ keys, uint64_t n,
                                                            uint64_t chunk, uint32_t *partials)
{
    uint64_t b = (uint64_t)blockIdx.x * chunk, e = b + chunk;
    if (e > n) e = n;
    uint32_t c = 0;
    for (uint64_t i = b + threadIdx.x; i < e; i += kThreads) c += (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
    __shared__ uint32_t sh[33];
    uint32_t tot;
    block_exclusive_sum<uint32_t>(c, sh, &tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kThreads) dedup_down_kernel(const uint64_t *__restrict__ keys, uint64_t n,
                                                              uint64_t chunk, const uint32_t *partials,
                                                              uint32_t frame_shift, uint64_t *codes,
                                                              uint32_t *seg, uint8_t *gap, uint32_t *vstart,
                                                              const uint32_t *__restrict__ vals, uint32_t *row0)
{
    __shared__ uint32_t sh[33];
    uint64_t b = (uint64_t)blockIdx.x * chunk, e = b + chunk;
    if (e > n) e = n;
    uint32_t run = partials[blockIdx.x];
    for (uint64_t t0 = b; t0 < e; t0 += kThreads) {
        uint64_t i = t0 + threadIdx.x;
        bool ok = i < e;
        uint64_t k = ok ? keys[i] : 0ull;
        uint64_t kp = (ok && i > 0) ? keys[i - 1] : 0ull;
        bool head = ok && (i == 0 || k != kp);
        uint32_t tot;
        uint32_t pre = block_exclusive_sum<uint32_t>(head ? 1u : 0u, sh, &tot);
        uint32_t v = run + pre;
        if (head) {
            codes[v] = k;
            seg[v] = (uint32_t)i;
            uint32_t g = (i == 0) ? kInfLevel : gap_level(kp, k, frame_shift);
            gap[v] = (uint8_t)g;
            if (g == kInfLevel) vstart[frame_shift < 64 ? (uint32_t)(k >> frame_shift) : 0u] = v;
            if (row0) row0[v] = vals[i] | ((i + 1 < n && keys[i + 1] == k) ? kCarry : 0u);
        }
        if (ok && i == n - 1) {
            seg[v + (head ? 1u : 0u)] = (uint32_t)n;
            gap[v + (head ? 1u : 0u)] = (uint8_t)kInfLevel;
        }
        run += tot;
    }
}

__global__ void dedup_fix_kernel(const uint32_t *partials, uint32_t P, uint32_t *vstart, uint32_t F,
                                 DevState *st)
{
    // partials were scanned in place; the total is the last prefix plus the last count
    uint32_t nv = partials[P];
    vstart[F] = nv;
    for (int f = (int)F - 1; f >= 0; --f)
        if (vstart[f] == 0xFFFFFFFFu) vstart[f] = vstart[f + 1];
    st->nv_total = nv;
}

// exclusive scan of P words with the total appended at [P] (one CTA)
__global__ void __launch_bounds__(1024) scan_total_kernel(uint32_t *a, uint32_t m)
{
    __shared__ uint32_t sh[33];
    uint32_t per = (m + 1023) / 1024;
    uint32_t b = per * threadIdx.x, e = b + per;
    if (e > m) e = m;
    if (b > m) b = m;
    uint32_t s = 0;
    for (uint32_t i = b; i < e; ++i) s += a[i];
    uint32_t tot;
    uint32_t run = block_exclusive_sum<uint32_t>(s, sh, &tot);
    for (uint32_t i = b; i < e; ++i) {
        uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
    if (threadIdx.x == 0) a[m] = tot;
}

// ------------------------------------------------------------ occupancy ---
__device__ __forceinline__ int height_of(uint8_t g, uint32_t J)
{
    return (g >= kInfLevel) ? (int)J : ((int)g - 1) / 3;
}

__global__ void __launch_bounds__(kThreads) occ_up_kernel(const uint8_t *__restrict__ gap,
                                                          const uint32_t *__restrict__ vstart,
                                                          const uint32_t *__restrict__ Jarr, uint32_t *partials)
{
    const uint32_t f = blockIdx.y, x = blockIdx.x, X = gridDim.x;
    const uint32_t J = Jarr[f];
    __shared__ uint32_t cnt[kH];
    if (threadIdx.x < kH) cnt[threadIdx.x] = 0;
    __syncthreads();
    Range r = cta_range(vstart[f], vstart[f + 1], x, X);
    for (uint64_t v = r.b + threadIdx.x; v < r.e; v += kThreads) {
        int s = height_of(gap[v], J);
        for (int h = 1; h <= s; ++h) atomicAdd(&cnt[h], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kH) partials[((uint64_t)f * kH + threadIdx.x) * X + x] = cnt[threadIdx.x];
}

// one CTA of 32 x kH threads per frame: warp h scans the CTA counts of height h
// (exclusive, in place), then level sizes and byte offsets of the frame
__global__ void __launch_bounds__(32 * kH) occ_scan_kernel(uint32_t *partials, uint32_t X,
                                                           const uint32_t *__restrict__ vstart,
                                                           const uint32_t *__restrict__ Jarr, uint32_t *lsz,
                                                           uint32_t *hoff, uint64_t *nocc)
{
    __shared__ uint32_t tot[kH];
    const uint32_t f = blockIdx.x, lane = threadIdx.x & 31, h = threadIdx.x >> 5;
    uint32_t *row = partials + ((uint64_t)f * kH + h) * X;
    uint32_t run = 0;
    for (uint32_t b = 0; b < X; b += 32) {
        const uint32_t x = b + lane;
        const uint32_t v = (x < X) ? row[x] : 0u;
        const uint32_t inc = warp_inclusive_sum(v);
        if (x < X) row[x] = run + inc - v;
        run += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
    if (lane == 0) tot[h] = run;
    __syncthreads();
    if (h == 0) {
        const uint32_t J = Jarr[f];
        // bytes of height h come after all heights above it (depth 0 first)
        const uint32_t sz = (lane >= 1 && lane <= J && lane < kH) ? tot[lane] : 0u;
        uint32_t above = 0;
        for (int h2 = 31; h2 >= 1; --h2) {
            const uint32_t t = __shfl_sync(0xFFFFFFFFu, sz, h2);
            if (h2 > (int)lane) above += t;
        }
        const uint32_t all = __reduce_add_sync(0xFFFFFFFFu, sz);
        if (lane < kH) hoff[f * kH + lane] = above;
        if (lane <= J && lane < kH) lsz[f * kH + (J - lane)] = (lane == 0) ? (vstart[f + 1] - vstart[f]) : tot[lane];
        if (lane == 0) nocc[f] = all;
    }
}

__global__ void occ_offsets_kernel(const uint64_t *nocc, uint32_t F, uint64_t *occ_off)
{
    if (threadIdx.x) return;
    uint64_t run = 0;
    for (uint32_t f = 0; f < F; ++f) {
        occ_off[f] = run;
        run += nocc[f];
    }
    occ_off[F] = run;
}

__global__ void zero_words_kernel(uint32_t *p, const uint64_t *nbytes_at, uint64_t cap_words)
{
    uint64_t nw = (*nbytes_at + 3) / 4;
    if (nw > cap_words) nw = cap_words;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = 0u;
}

// Occupancy bytes of one tile of kThreads voxels, all heights at once.  Voxel v
// starts a node at heights 1..s_v and is a child start at heights 1..s_v + 1;
// its node at height h is the last node start at or before it, whose byte
// index is the count of node starts up to v (per-height counts carried from
// earlier tiles and CTAs).  Child bits are OR-ed into the tile's bytes in
// shared memory (byte j of height h = the tile's j-th node start there; byte
// 0 = the node a previous tile started), then every nonzero word goes out
// with one atomic OR (the buffer is zeroed first; a word on the edge of a
// tile's range is shared with its neighbours).
constexpr int kOccWords = kThreads / 4 + 2;  // per height: bytes 0 .. kThreads, word-aligned either way

__global__ void __launch_bounds__(kThreads) occ_down_kernel(const uint64_t *__restrict__ codes,
                                                            const uint8_t *__restrict__ gap,
                                                            const uint32_t *__restrict__ vstart,
                                                            const uint32_t *__restrict__ Jarr,
                                                            const uint32_t *__restrict__ partials,
                                                            const uint32_t *__restrict__ hoff,
                                                            const uint64_t *__restrict__ occ_off,
                                                            uint32_t *occ_words, uint64_t occ_capacity,
                                                            DevState *st)
{
    const uint32_t f = blockIdx.y, x = blockIdx.x, X = gridDim.x;
    const uint32_t J = Jarr[f];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    __shared__ uint32_t s_run[kH], s_hoff[kH], s_tot[kH];
    __shared__ uint32_t s_w[kThreads / 32][kH];
    __shared__ uint32_t s_byte[kH][kOccWords];
    __shared__ int s_hm;
    if (tid < kH) {
        s_run[tid] = partials[((uint64_t)f * kH + tid) * X + x];
        s_hoff[tid] = hoff[f * kH + tid];
    }
    const uint64_t base = occ_off[f];
    const uint32_t lemask = lanemask_lt() | (1u << lane);
    const uint64_t cap_words = occ_capacity >> 2;
    Range r = cta_range(vstart[f], vstart[f + 1], x, X);
    for (uint64_t t0 = r.b; t0 < r.e; t0 += kThreads) {
        if (tid == 0) s_hm = 0;
        __syncthreads();
        const uint64_t v = t0 + tid;
        const bool ok = v < r.e;
        const int s = ok ? height_of(gap[v], J) : -1;
        const uint64_t m = ok ? codes[v] : 0ull;
        const int cm = ok ? ((s + 1) < (int)J ? (s + 1) : (int)J) : 0;
        // this warp's own highest height: above it the warp holds no node start and no child
        const int hw = (int)__reduce_max_sync(0xFFFFFFFFu, (uint32_t)cm);
        if (lane == 0) atomicMax(&s_hm, hw);
        __syncthreads();
        const int hm = s_hm;
        for (int i = tid; i < hm * kOccWords; i += kThreads) (&s_byte[1][0])[i] = 0u;
        for (int h = 1; h <= hm; ++h) {
            const uint32_t b = (h <= hw) ? __ballot_sync(0xFFFFFFFFu, s >= h) : 0u;
            if (lane == 0) s_w[w][h] = __popc(b);
        }
        __syncthreads();
        if (tid >= 1 && tid <= hm) {  // per height: exclusive prefix over warps, tile total
            uint32_t run = 0;
            for (int ww = 0; ww < kThreads / 32; ++ww) {
                const uint32_t c = s_w[ww][tid];
                s_w[ww][tid] = run;
                run += c;
            }
            s_tot[tid] = run;
        }
        __syncthreads();
        for (int h = 1; h <= hw; ++h) {
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, s >= h);
            if (h <= cm) {
                // byte index in the tile: node starts at height h up to and including this voxel
                const uint32_t j = s_w[w][h] + __popc(b & lemask);
                const uint32_t bit = (uint32_t)(m >> (3 * (h - 1))) & 7u;
                atomicOr(&s_byte[h][j >> 2], 1u << (bit + 8u * (j & 3u)));
            }
        }
        __syncthreads();
        // out: global word W = (g0 >> 2) + k of height h (g0 = the global byte of tile byte 0, one before
        // the tile's first node start there) holds tile bytes 4k - r .. 4k - r + 3, r = g0 mod 4
        for (int i = tid; i < hm * kOccWords; i += kThreads) {
            const int h = 1 + i / kOccWords, k = i - (h - 1) * kOccWords;
            const int64_t g0 = (int64_t)(base + s_hoff[h] + s_run[h]) - 1;
            const uint32_t r = (uint32_t)(g0 & 3);
            if (k > (int)((s_tot[h] + r) >> 2)) continue;
            const uint32_t lo = k >= 1 ? s_byte[h][k - 1] : 0u, hi = k < kOccWords - 1 ? s_byte[h][k] : 0u;
            const uint32_t val = __funnelshift_rc(lo, hi, 8u * (4u - r));
            if (val) {
                const int64_t W = (g0 >> 2) + k;  // arithmetic shift: floor
                if (W >= 0 && (uint64_t)W < cap_words)
                    atomicOr(occ_words + W, val);
                else
                    set_error(&st->err, kErrCapacity);
            }
        }
        __syncthreads();
        if (tid >= 1 && tid <= hm) s_run[tid] += s_tot[tid];
        __syncthreads();
    }
}

// ------------------------------------------------------- octree decode ---
// Exclusive prefix of the popcounts of the occupancy bytes (children before
// each node, Algorithm 3): CTA chunks of whole 16-byte groups, each thread
// handling 16 consecutive bytes per step (one vector load when aligned).
constexpr uint32_t kPopcVec = 16;

__device__ __forceinline__ void load16(const uint8_t *p, uint64_t i, uint64_t e, bool vec, uint32_t w[4])
{
    if (vec && i + kPopcVec <= e) {
        const uint4 v = *reinterpret_cast<const uint4 *>(p + i);
        w[0] = v.x;
        w[1] = v.y;
        w[2] = v.z;
        w[3] = v.w;
        return;
    }
    for (int k = 0; k < 4; ++k) {
        uint32_t x = 0;
        for (int b = 0; b < 4; ++b) {
            const uint64_t j = i + 4 * k + b;
            if (j < e) x |= (uint32_t)p[j] << (8 * b);
        }
        w[k] = x;
    }
}

__global__ void __launch_bounds__(kThreads) popc_up_kernel(const uint8_t *__restrict__ occ, uint64_t n,
                                                           uint64_t chunk, uint32_t *partials)
{
    uint64_t b = (uint64_t)blockIdx.x * chunk, e = b + chunk;
    if (e > n) e = n;
    const bool vec = ((uintptr_t)occ & 15) == 0;
    uint32_t c = 0;
    for (uint64_t i = b + (uint64_t)threadIdx.x * kPopcVec; i < e; i += (uint64_t)kThreads * kPopcVec) {
        uint32_t w[4];
        load16(occ, i, e, vec, w);
        c += __popc(w[0]) + __popc(w[1]) + __popc(w[2]) + __popc(w[3]);
    }
    __shared__ uint32_t sh[33];
    uint32_t tot;
    block_exclusive_sum<uint32_t>(c, sh, &tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kThreads) popc_down_kernel(const uint8_t *__restrict__ occ, uint64_t n,
                                                             uint64_t chunk, const uint32_t *partials,
                                                             uint32_t *pref)
{
    __shared__ uint32_t sh[33];
    uint64_t b = (uint64_t)blockIdx.x * chunk, e = b + chunk;
    if (e > n) e = n;
    const bool vec = ((uintptr_t)occ & 15) == 0 && ((uintptr_t)pref & 15) == 0;
    uint32_t run = partials[blockIdx.x];
    for (uint64_t t0 = b; t0 < e; t0 += (uint64_t)kThreads * kPopcVec) {
        const uint64_t i = t0 + (uint64_t)threadIdx.x * kPopcVec;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (i < e) load16(occ, i, e, vec, w);
        uint32_t pc[16];
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            pc[k] = c;
            c += __popc((w[k >> 2] >> (8 * (k & 3))) & 0xFFu);
        }
        uint32_t tot;
        const uint32_t pre = run + block_exclusive_sum<uint32_t>(c, sh, &tot);
        if (vec && i + kPopcVec <= e) {
            uint4 *o = reinterpret_cast<uint4 *>(pref + i);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                o[q] = make_uint4(pre + pc[4 * q], pre + pc[4 * q + 1], pre + pc[4 * q + 2], pre + pc[4 * q + 3]);
        } else {
            for (int k = 0; k < 16; ++k)
                if (i + k < e) pref[i + k] = pre + pc[k];
        }
        run += tot;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) pref[n] = partials[gridDim.x];
}

__global__ void root_kernel(uint64_t *nodes) { nodes[0] = 0ull; }

// one level of Algorithm 3: node p of L_d writes (code << 3) + i for each set bit i
__global__ void __launch_bounds__(kThreads) expand_kernel(const uint64_t *__restrict__ Ld, uint32_t Md,
                                                          const uint8_t *__restrict__ occ, uint64_t boff,
                                                          const uint32_t *__restrict__ pref, uint64_t *Ld1,
                                                          uint32_t Md1, DevState *st)
{
    const uint32_t base = pref[boff];
    if (blockIdx.x == 0 && threadIdx.x == 0 && pref[boff + Md] - base != Md1) set_error(&st->err, kErrCorrupt);
    for (uint32_t p = blockIdx.x * kThreads + threadIdx.x; p < Md; p += gridDim.x * kThreads) {
        uint32_t byte = occ[boff + p];
        if (byte == 0) {
            set_error(&st->err, kErrCorrupt);
            continue;
        }
        uint64_t c = Ld[p] << 3;
        uint32_t w = pref[boff + p] - base;
        for (uint32_t bits = byte; bits; bits &= bits - 1u) {  // set bits in increasing order
            if (w < Md1) Ld1[w] = c + (uint32_t)(__ffs(bits) - 1);
            ++w;
        }
    }
}

// Algorithm 3 for the small top levels d < d_end in one CTA (levels are
// separated by block barriers), saving one launch per level.
struct LevelTable {
    uint32_t M[kH];      // level sizes
    uint64_t noff[kH];   // node offset of each level in the node array
    uint64_t boff[kH];   // byte offset of each level in the occupancy stream
};

__global__ void __launch_bounds__(1024) expand_top_kernel(LevelTable lt, uint32_t d_end, uint64_t *nodes,
                                                          const uint8_t *__restrict__ occ,
                                                          const uint32_t *__restrict__ pref, DevState *st)
{
    for (uint32_t d = 0; d < d_end; ++d) {
        const uint32_t Md = lt.M[d], Md1 = lt.M[d + 1];
        const uint64_t boff = lt.boff[d];
        const uint64_t *Ld = nodes + lt.noff[d];
        uint64_t *Ld1 = nodes + lt.noff[d + 1];
        const uint32_t base = pref[boff];
        if (threadIdx.x == 0 && pref[boff + Md] - base != Md1) set_error(&st->err, kErrCorrupt);
        for (uint32_t p = threadIdx.x; p < Md; p += blockDim.x) {
            const uint32_t byte = occ[boff + p];
            if (byte == 0) {
                set_error(&st->err, kErrCorrupt);
                continue;
            }
            const uint64_t c = Ld[p] << 3;
            uint32_t w = pref[boff + p] - base;
            for (uint32_t bits = byte; bits; bits &= bits - 1u) {  // set bits in increasing order
                if (w < Md1) Ld1[w] = c + (uint32_t)(__ffs(bits) - 1);
                ++w;
            }
        }
        __threadfence_block();
        __syncthreads();
    }
}

__global__ void gap_kernel(const uint64_t *__restrict__ codes, uint64_t nv, uint8_t *gap)
{
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= nv; v += (uint64_t)gridDim.x * blockDim.x)
        gap[v] = (v == 0 || v == nv) ? (uint8_t)kInfLevel : (uint8_t)gap_level(codes[v - 1], codes[v], 64);
}

__device__ __forceinline__ uint32_t compact3(uint64_t m)
{
    m &= 0x1249249249249249ull;
    m = (m | (m >> 2)) & 0x10C30C30C30C30C3ull;
    m = (m | (m >> 4)) & 0x100F00F00F00F00Full;
    m = (m | (m >> 8)) & 0x001F0000FF0000FFull;
    m = (m | (m >> 16)) & 0x001F00000000FFFFull;
    m = (m | (m >> 32)) & 0x00000000001FFFFFull;
    return (uint32_t)m;
}

__device__ __forceinline__ void centre(uint64_t m, const FrameGrid &g, float *out)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double vv = (double)compact3(m >> a);
        double off = __dmul_rn(__dadd_rn(vv, 0.5), g.cell);
        out[a] = (float)__dadd_rn(g.lo[a], off);
    }
}

__global__ void centres_kernel(const uint64_t *__restrict__ codes, uint64_t nv, const FrameGrid *grid, float *pos)
{
    const FrameGrid g = *grid;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (uint64_t)gridDim.x * blockDim.x)
        centre(codes[v], g, pos + 3 * v);
}

// per-axis centre table of one frame: entry a * 2^J + v = (float)(lo_a + (v + 0.5) cell)
__global__ void centre_table_kernel(const FrameGrid *grid, uint32_t J, float *ctab)
{
    const FrameGrid g = *grid;
    const uint64_t side = 1ull << J;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * side;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = (uint32_t)(e >> J);
        const double off = __dmul_rn(__dadd_rn((double)(e & (side - 1)), 0.5), g.cell);
        ctab[e] = (float)__dadd_rn(g.lo[a], off);
    }
}

__global__ void centres_table_kernel(const uint64_t *__restrict__ codes, uint64_t nv, uint32_t J,
                                     const float *__restrict__ ctab, float *pos)
{
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t m = codes[v];
#pragma unroll
        for (int a = 0; a < 3; ++a) pos[3 * v + a] = ctab[((uint64_t)a << J) + (uint32_t)compact3(m >> a)];
    }
}

__global__ void centres_batch_kernel(const uint64_t *__restrict__ codes, const DevState *st, uint32_t frame_shift,
                                     const FrameGrid *grid, float *pos)
{
    const uint64_t nv = st->nv_total;
    const uint64_t mask = (frame_shift < 64) ? ((1ull << frame_shift) - 1) : ~0ull;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = codes[v];
        uint32_t f = (frame_shift < 64) ? (uint32_t)(k >> frame_shift) : 0u;
        centre(k & mask, grid[f], pos + 3 * v);
    }
}

uint32_t grid_for(uint64_t n, int num_sms)
{
    uint64_t b = (n + kThreads - 1) / kThreads;
    uint64_t cap = (uint64_t)num_sms * 8;
    if (b < 1) b = 1;
    return (uint32_t)(b < cap ? b : cap);
}

struct Chunks {
    uint32_t P;
    uint64_t chunk;
};

Chunks chunks_for(uint64_t n, int num_sms, uint32_t per_sm = 2)
{
    Chunks c;
    uint64_t t = (n + 1023) / 1024;
    uint64_t pmax = (uint64_t)num_sms * per_sm;
    c.P = (uint32_t)(t < 1 ? 1 : (t < pmax ? t : pmax));
    c.chunk = (n + c.P - 1) / c.P;
    if (c.chunk == 0) c.chunk = 1;
    return c;
}

// CTA chunks of whole 16-byte groups (so vector loads stay aligned), at most 2 per SM
Chunks popc_chunks(uint64_t n, int num_sms)
{
    Chunks c = chunks_for(n, num_sms);
    c.chunk = (c.chunk + kPopcVec - 1) / kPopcVec * kPopcVec;
    c.P = (uint32_t)((n + c.chunk - 1) / c.chunk);
    if (c.P == 0) c.P = 1;
    return c;
}

uint32_t occ_x(uint32_t F, int num_sms)
{
    uint32_t X = (uint32_t)(num_sms * 8) / F;
    return X < 16 ? 16 : X;
}

}  // namespace

// dedup: up to 8 CTAs of 256 threads per SM (each CTA scans its chunk in steps of 256 keys, so the SM needs many
// of them in flight to hide the key loads)
constexpr uint32_t kDedupPerSm = 8;
uint64_t dedup_partial_words(uint64_t n, int num_sms) { return chunks_for(n, num_sms, kDedupPerSm).P + 1; }

void launch_dedup(const uint64_t *keys, uint64_t n, uint32_t frame_shift, uint32_t F, uint64_t *codes,
                  uint32_t *seg, uint8_t *gap, uint32_t *vstart, uint32_t *partials, DevState *st, int num_sms,
                  cudaStream_t s, const uint32_t *vals, uint32_t *row0)
{
    if (!vals) row0 = nullptr;
    dev_memset(vstart, 0xFF, sizeof(uint32_t) * (F + 1), s);
    Chunks c = chunks_for(n, num_sms, kDedupPerSm);
    if (n == 0) {
        dev_memset(partials, 0, sizeof(uint32_t) * (c.P + 1), s);
        dev_memset(seg, 0, sizeof(uint32_t), s);
        dev_memset(gap, (int)kInfLevel, 1, s);
    } else {
        dedup_up_kernel<<<c.P, kThreads, 0, s>>>(keys, n, c.chunk, partials);
        count_launch();
        scan_total_kernel<<<1, 1024, 0, s>>>(partials, c.P);
        count_launch();
        dedup_down_kernel<<<c.P, kThreads, 0, s>>>(keys, n, c.chunk, partials, frame_shift, codes, seg, gap,
                                                   vstart, vals, row0);
        count_launch();
    }
    dedup_fix_kernel<<<1, 1, 0, s>>>(partials, c.P, vstart, F, st);
    count_launch();
}

uint64_t occupancy_partial_words(uint32_t F, int num_sms) { return (uint64_t)F * occ_x(F, num_sms) * kH + 2 * kMaxFrames + 8; }

void launch_occupancy(const uint64_t *codes, const uint8_t *gap, const uint32_t *vstart, const uint32_t *J,
                      uint32_t F, uint32_t frame_shift, const OccupancyOut &o, DevState *st, int num_sms,
                      cudaStream_t s)
{
    (void)frame_shift;
    uint32_t X = occ_x(F, num_sms);
    dim3 grid(X, F);
    occ_up_kernel<<<grid, kThreads, 0, s>>>(gap, vstart, J, o.partials);
    count_launch();
    uint64_t *nocc = reinterpret_cast<uint64_t *>(o.partials + (uint64_t)F * X * kH + ((F * X * kH) & 1u));
    occ_scan_kernel<<<F, 32 * kH, 0, s>>>(o.partials, X, vstart, J, o.level_sizes, o.hoff, nocc);
    count_launch();
    occ_offsets_kernel<<<1, 32, 0, s>>>(nocc, F, o.occ_off);
    count_launch();
    zero_words_kernel<<<num_sms * 2, 256, 0, s>>>((uint32_t *)o.occ, o.occ_off + F, o.occ_capacity / 4);
    count_launch();
    occ_down_kernel<<<grid, kThreads, 0, s>>>(codes, gap, vstart, J, o.partials, o.hoff, o.occ_off,
                                              (uint32_t *)o.occ, o.occ_capacity, st);
    count_launch();
}

uint64_t octree_decode_node_words(const uint32_t *h_level_sizes, uint32_t J)
{
    uint64_t t = 0;
    for (uint32_t d = 0; d < J; ++d) t += h_level_sizes[d];
    return t;
}

void launch_octree_decode(const uint8_t *occ, uint64_t n_occ, uint32_t J, const uint32_t *h_level_sizes,
                          uint64_t *nodes, uint32_t *pref, uint32_t *partials, uint64_t *leaves,
                          DevState *st, int num_sms, cudaStream_t s)
{
    if (h_level_sizes[0] == 0) return;
    Chunks c = popc_chunks(n_occ, num_sms);
    popc_up_kernel<<<c.P, kThreads, 0, s>>>(occ, n_occ, c.chunk, partials);
    count_launch();
    scan_total_kernel<<<1, 1024, 0, s>>>(partials, c.P);
    count_launch();
    popc_down_kernel<<<c.P, kThreads, 0, s>>>(occ, n_occ, c.chunk, partials, pref);
    count_launch();
    root_kernel<<<1, 1, 0, s>>>(nodes);
    count_launch();
    // levels whose children fit one CTA comfortably are expanded together
    LevelTable lt{};
    uint64_t noff = 0, boff = 0;
    for (uint32_t d = 0; d <= J; ++d) {
        lt.M[d] = h_level_sizes[d];
        lt.noff[d] = noff;
        lt.boff[d] = boff;
        noff += h_level_sizes[d];
        boff += h_level_sizes[d];
    }
    uint32_t d_end = 0;
    while (d_end + 1 < J && h_level_sizes[d_end + 1] <= 8192) ++d_end;
    if (d_end) {
        expand_top_kernel<<<1, 1024, 0, s>>>(lt, d_end, nodes, occ, pref, st);
        count_launch();
    }
    for (uint32_t d = d_end; d < J; ++d) {
        const uint32_t Md = h_level_sizes[d], Md1 = h_level_sizes[d + 1];
        uint64_t *Ld = nodes + lt.noff[d];
        uint64_t *Ld1 = (d + 1 == J) ? leaves : nodes + lt.noff[d + 1];
        expand_kernel<<<grid_for(Md, num_sms), kThreads, 0, s>>>(Ld, Md, occ, lt.boff[d], pref, Ld1, Md1, st);
        count_launch();
    }
}

void launch_gap_levels(const uint64_t *codes, uint64_t nv, uint8_t *gap, cudaStream_t s)
{
    gap_kernel<<<grid_for(nv + 1, 152), kThreads, 0, s>>>(codes, nv, gap);
    count_launch();
}

void launch_voxel_centres(const uint64_t *codes, uint64_t nv, uint32_t J, const FrameGrid *grid, float *pos,
                          cudaStream_t s, float *ctab)
{
    if (nv == 0) return;
    if (ctab && (1ull << J) <= nv) {
        centre_table_kernel<<<grid_for(3ull << J, 152), kThreads, 0, s>>>(grid, J, ctab);
        count_launch();
        centres_table_kernel<<<grid_for(nv, 152), kThreads, 0, s>>>(codes, nv, J, ctab, pos);
    } else {
        centres_kernel<<<grid_for(nv, 152), kThreads, 0, s>>>(codes, nv, grid, pos);
    }
    count_launch();
}

void launch_voxel_centres_batch(const uint64_t *codes, const DevState *st, uint64_t nv_bound,
                                uint32_t frame_shift, const uint32_t *J, const FrameGrid *grid, float *pos,
                                cudaStream_t s)
{
    (void)J;
    if (nv_bound == 0) return;
    centres_batch_kernel<<<grid_for(nv_bound, 152), kThreads, 0, s>>>(codes, st, frame_shift, grid, pos);
    count_launch();
}

}  // namespace gsnfs
