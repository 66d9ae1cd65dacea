// Batch-wide decoding steps: many frames (streams) decoded by one sequence
// of launches (Sec. 2.3 / Algorithms 2-3 for geometry, Sec. 3.4 and the
// inverse of Algorithm 6 for attributes, applied to every frame at once).
// Frames are described by a device table (DecFrame); every kernel finds the
// frame of its work item with a binary search over per-frame prefix sums.
#include "kernels.cuh"
#include "rans_dec.cuh"

namespace gsnfs {

namespace {

constexpr uint32_t kProbBits = 15;
constexpr uint32_t kM = 1u << kProbBits;

template <typename T>
__device__ __forceinline__ uint32_t find_frame(const T *pref, uint32_t F, uint64_t x)
{
    uint32_t lo = 0, hi = F;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((uint64_t)pref[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// raw and constant occupancy sections: bytes straight into the batch buffer
__global__ void occ_bytes_kernel(const DecFrame *fr, uint8_t *occ_all)
{
    const DecFrame &d = fr[blockIdx.y];
    if (d.mode == 1) return;
    uint8_t *dst = occ_all + d.occ_off;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d.n_occ; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = (d.mode == 2) ? (uint8_t)d.aux : d.occ_sec[16 + i];
}

// per frame: slot -> symbol table and freq << 16 | cum, then a corruption flag; and the byte offset of
// every chunk inside the section (a scan of the chunk size table)
__global__ void __launch_bounds__(1024) tables_kernel(const DecFrame *fr, uint32_t *tabs, uint64_t tab_words,
                                                      uint64_t *cstart, DevState *st)
{
    const DecFrame &d = fr[blockIdx.x];
    if (d.mode != 1) return;
    uint32_t *tab = tabs + (uint64_t)blockIdx.x * tab_words;
    __shared__ uint32_t s_cm[256];
    __shared__ uint32_t s_fc[256];
    const uint8_t *ftab = d.occ_sec + 24;
    if (threadIdx.x < 32) {
        uint32_t run = 0;
        for (int b = 0; b < 256; b += 32) {
            const int s2 = b + threadIdx.x;
            const uint32_t v = (uint32_t)(ftab[2 * s2] | (ftab[2 * s2 + 1] << 8));
            const uint32_t inc = warp_inclusive_sum(v);
            s_cm[s2] = run + inc - v;
            s_fc[s2] = (v << 16) | ((run + inc - v) & 0xFFFFu);
            run += __shfl_sync(0xFFFFFFFFu, inc, 31);
        }
        if (threadIdx.x == 0) {
            tab[kM / 4 + 256] = (run != kM);
            if (run != kM) set_error(&st->err, kErrCorrupt);
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < 256; t += blockDim.x) tab[kM / 4 + t] = s_fc[t];
    uint8_t *slot2sym = reinterpret_cast<uint8_t *>(tab);
    for (uint32_t t = threadIdx.x; t < kM; t += blockDim.x) {
        uint32_t lo = 0, hi = 256;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_cm[mid] <= t) lo = mid; else hi = mid;
        }
        slot2sym[t] = (uint8_t)lo;
    }
    // chunk offsets: after the section header, the frequency table and the size table (8-byte aligned)
    __shared__ uint64_t sh64[33];
    const uint32_t nch = d.aux;
    const uint8_t *ctab = d.occ_sec + 24 + 512;
    uint64_t run = (16 + 8 + 512 + 4 * (uint64_t)nch + 7) & ~7ull;
    for (uint32_t b = 0; b < nch; b += blockDim.x) {
        const uint32_t c = b + threadIdx.x;
        uint64_t sz = 0;
        if (c < nch) {
            const uint8_t *q = ctab + 4 * (uint64_t)c;
            sz = (uint32_t)q[0] | ((uint32_t)q[1] << 8) | ((uint32_t)q[2] << 16) | ((uint32_t)q[3] << 24);
        }
        uint64_t tot;
        const uint64_t ex = block_exclusive_sum<uint64_t>(sz, sh64, &tot);
        if (c < nch) cstart[d.chunk_off + c] = run + ex;
        run += tot;
    }
}

// grid (chunk groups, frames): warp per chunk of frame blockIdx.y, the chunk read in place (its words are
// consumed in order, so they come from L1 after the first lane of a sector asks), the tables in shared memory
constexpr uint32_t kRansWarps = 8;

__global__ void __launch_bounds__(32 * kRansWarps) rans_batch_kernel(const DecFrame *fr, const uint32_t *tabs,
                                                                     uint64_t tab_words, const uint64_t *cstart,
                                                                     uint8_t *occ_all, DevState *st)
{
    using namespace ransdec;
    extern __shared__ __align__(16) unsigned char dsm[];
    const DecFrame &d = fr[blockIdx.y];
    if (d.mode != 1) return;
    const uint32_t *tab = tabs + (uint64_t)blockIdx.y * tab_words;
    if (tab[kTabWords] != 0) return;
    const uint32_t nch = d.aux, chunk = d.chunk;
    const uint32_t lane = threadIdx.x & 31, wl = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (blockIdx.x * nwarps >= nch) return;  // no chunk of this frame for this CTA
    load_tables(reinterpret_cast<uint32_t *>(dsm), tab);
    __syncthreads();
    const uint8_t *slot2sym = dsm;
    const uint32_t *fc = reinterpret_cast<const uint32_t *>(dsm + kM);
    const uint8_t *ctab = d.occ_sec + 24 + 512;
    uint8_t *out = occ_all + d.occ_off;
    for (uint32_t c = blockIdx.x * nwarps + wl; c < nch; c += gridDim.x * nwarps) {
        const uint64_t start = cstart[d.chunk_off + c];
        const uint8_t *cp = ctab + 4 * c;
        const uint32_t cbytes = (uint32_t)cp[0] | ((uint32_t)cp[1] << 8) | ((uint32_t)cp[2] << 16) | ((uint32_t)cp[3] << 24);
        if (cbytes < 128 || (cbytes & 3) || cbytes > 128 + 2 * chunk + 2 || start + cbytes > d.occ_bytes) {
            if (lane == 0) set_error(&st->err, kErrCorrupt);
            continue;
        }
        const uint64_t s0 = (uint64_t)c * chunk;
        const uint32_t len = (uint32_t)((d.n_occ - s0) < chunk ? (d.n_occ - s0) : chunk);
        if (decode_chunk(slot2sym, fc, d.occ_sec + start, (cbytes - 128) / 2, len, out + s0, lane) && lane == 0)
            set_error(&st->err, kErrCorrupt);
    }
}

__device__ __forceinline__ uint32_t compact3b(uint64_t m)
{
    m &= 0x1249249249249249ull;
    m = (m | (m >> 2)) & 0x10C30C30C30C30C3ull;
    m = (m | (m >> 4)) & 0x100F00F00F00F00Full;
    m = (m | (m >> 8)) & 0x001F0000FF0000FFull;
    m = (m | (m >> 16)) & 0x001F00000000FFFFull;
    m = (m | (m >> 32)) & 0x00000000001FFFFFull;
    return (uint32_t)m;
}

__global__ void roots_kernel(const DecFrame *fr, uint32_t F, uint64_t *nodes, uint8_t *gap, uint64_t nv_total)
{
    const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f == 0) gap[nv_total] = (uint8_t)kInfLevel;  // sentinel after the last voxel
    if (f >= F || fr[f].nv == 0) return;
    nodes[fr[f].noff[0]] = 0ull;  // implicit root code of Algorithm 2
}

// ---- octree levels (Algorithm 3) by tiles of the batch occupancy buffer ----
// P(x) = number of set bits in the batch occupancy bytes before byte x.  Node w
// of level d of frame f (byte x = occ_off + boff[d] + w) has its children at
// indices P(x) - P(a0) .. of level d + 1, a0 the level's first byte.  P(a0) is
// known on the host (a level's popcounts add up to the next level's size);
// P at every kOccTile-byte boundary comes from a scan of tile popcounts, and
// a tile's CTA finds P(x) for its bytes with one block scan.  One launch per
// level covers every frame: its CTAs are the tiles that hold bytes of that
// level (a tile on a level boundary is visited by both levels' launches).
// At a frame's last level the leaf codes are not stored: the CTA writes the
// voxel centres (Sec. 2.1) and the gap levels of consecutive voxels instead.
constexpr uint32_t kOccTile = 1024;  // bytes per tile

__device__ __forceinline__ uint32_t word_at(const uint8_t *occ, uint64_t n, uint64_t x)  // bytes >= n read 0
{
    if (x >= n) return 0u;
    uint32_t v = *reinterpret_cast<const uint32_t *>(occ + x);  // x % 4 == 0; the buffer has 8 bytes of slack
    if (x + 4 > n) v &= (1u << (8u * (uint32_t)(n - x))) - 1u;
    return v;
}

__global__ void __launch_bounds__(256) occ_tile_popc_kernel(const uint8_t *__restrict__ occ, uint64_t n,
                                                            uint64_t ntiles, uint32_t *tsum)
{
    const uint32_t lane = threadIdx.x & 31;
    for (uint64_t t = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntiles;
         t += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
        uint32_t c = 0;
#pragma unroll
        for (uint32_t k = 0; k < kOccTile / 128; ++k) c += __popc(word_at(occ, n, t * kOccTile + 4ull * (lane + 32 * k)));
        c = __reduce_add_sync(0xFFFFFFFFu, c);
        if (lane == 0) tsum[t] = c;
    }
}

__device__ __forceinline__ void leaf_out(const DecFrame &d, const float *__restrict__ ctab, uint32_t v, uint64_t m,
                                         float *pos)
{
    if (d.ctab_off != ~0ull) {
        const float *t = ctab + d.ctab_off;
        float c[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) c[a] = __ldg(t + ((uint64_t)a << d.J) + compact3b(m >> a));
#pragma unroll
        for (int a = 0; a < 3; ++a) pos[3ull * v + a] = c[a];
    } else {
        const FrameGrid g = d.grid;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double off = __dmul_rn(__dadd_rn((double)compact3b(m >> a), 0.5), g.cell);
            pos[3ull * v + a] = (float)__dadd_rn(g.lo[a], off);
        }
    }
}

struct LevelArgs {
    const DecFrame *fr;
    uint32_t F, d;
    const uint32_t *tile_pref;  // F + 1: first CTA of each frame at this level
    const uint8_t *occ;
    uint64_t n_occ;
    const uint64_t *tbase;      // P at each tile's first byte
    uint64_t *nodes;
    const float *ctab;
    float *pos;                 // or null: no centres
    uint8_t *gap;
    DevState *st;
};

// A CTA of kLevelThreads threads takes one tile.  Its bytes are loaded 8 per
// thread and their set bits scanned; the per-byte prefixes go to shared
// memory, and the nodes are then taken strided (node j of the tile by thread
// j mod kLevelThreads), so that code loads and child stores of consecutive
// threads are consecutive.  Internal level: children codes go straight to
// the next level.  Leaf level: the children's codes are staged in shared
// memory at their rank among the tile's set bits, then one child per thread
// gets its gap level (from the staged code before it) and its centre, with
// coalesced stores (a tile with more set bits than the stage holds writes its
// voxels directly).
constexpr uint32_t kLevelThreads = kOccTile / 8;
constexpr uint32_t kLeafStage = 2048;

__device__ __forceinline__ uint64_t word8_at(const uint8_t *occ, uint64_t n, uint64_t x)  // bytes >= n read 0
{
    if (x >= n) return 0ull;
    uint64_t v = *reinterpret_cast<const uint64_t *>(occ + x);  // x % 8 == 0; the buffer has 8 bytes of slack
    if (x + 8 > n) v &= (1ull << (8u * (uint32_t)(n - x))) - 1ull;
    return v;
}

// the last child's code of node w (byte b) of a level, shifted to the next level
__device__ __forceinline__ uint64_t last_child(uint64_t code, uint32_t b)
{
    return (code << 3) + (b ? 31u - (uint32_t)__clz(b) : 0u);
}

__global__ void __launch_bounds__(kLevelThreads) expand_level_kernel(LevelArgs a)
{
    __shared__ uint64_t sh[33];
    __shared__ uint64_t s_leaf[kLeafStage];
    __shared__ uint16_t s_pref[kOccTile];
    __shared__ uint8_t s_occ[kOccTile];
    __shared__ uint32_t s_lo, s_hi;
    __shared__ uint64_t s_prev;
    __shared__ int s_first;  // the tile holds the level's first node (its first voxel starts a frame)
    const uint32_t g = blockIdx.x, t = threadIdx.x;
    const uint32_t f = find_frame(a.tile_pref, a.F, g);
    const DecFrame &fd = a.fr[f];
    const uint32_t d = a.d;
    const uint64_t a0 = fd.occ_off + fd.boff[d], a1 = a0 + fd.lsz[d];
    const uint64_t tile = a0 / kOccTile + (g - a.tile_pref[f]);
    const uint64_t tx = tile * kOccTile;
    const bool leaf = d + 1 == fd.J;
    const uint64_t *src = a.nodes + fd.noff[d];
    const uint64_t wv = word8_at(a.occ, a.n_occ, tx + 8ull * t);
    // the codes of this thread's nodes (tile bytes t, t + 128, ...) are loaded before the scan
    uint64_t code[8];
#pragma unroll
    for (uint32_t k = 0; k < 8; ++k) {
        const uint64_t x = tx + k * kLevelThreads + t;
        code[k] = (x >= a0 && x < a1) ? src[x - a0] : 0ull;
    }
    const uint64_t xs = tx > a0 ? tx : a0;  // the tile's first byte of this level
    if (t == 0) {
        s_first = xs == a0;
        s_prev = (leaf && xs > a0 && xs < a1) ? last_child(src[xs - 1 - a0], a.occ[xs - 1]) : 0ull;
    }
    const uint64_t tb = a.tbase[tile];
    uint64_t tot;
    uint32_t lp = (uint32_t)block_exclusive_sum<uint64_t>((uint64_t)__popcll(wv), sh, &tot);
#pragma unroll
    for (uint32_t k = 0; k < 8; ++k) {  // per byte: set bits of the tile before it
        const uint32_t b = (uint32_t)(wv >> (8u * k)) & 0xFFu;
        s_pref[8 * t + k] = (uint16_t)lp;
        s_occ[8 * t + k] = (uint8_t)b;
        lp += __popc(b);
    }
    const uint64_t base = fd.pbase[d];
    const uint32_t M1 = fd.lsz[d + 1];
    const bool stage = leaf && tot <= kLeafStage;
    if (t == 0) {  // the staged range: the tile's bytes of this level
        s_lo = 0;
        s_hi = (uint32_t)tot;
    }
    __syncthreads();
    bool bad = false;
#pragma unroll
    for (uint32_t k = 0; k < 8; ++k) {
        const uint32_t j = k * kLevelThreads + t;
        const uint64_t x = tx + j;
        if (x < a0 || x >= a1) continue;
        const uint32_t byte = s_occ[j];
        const uint32_t pj = s_pref[j];
        if (x == a0) s_lo = pj;
        if (x + 1 == a1) {
            if (tb + pj + __popc(byte) - base != M1) bad = true;  // the level's popcounts add up to the next level
            s_hi = pj + __popc(byte);
        }
        const uint64_t cw = tb + pj - base;
        if (byte == 0 || cw + (uint64_t)__popc(byte) > M1) {
            bad = true;
            continue;
        }
        const uint64_t c = code[k] << 3;
        if (!leaf) {
            uint64_t *dst = a.nodes + fd.noff[d + 1] + cw;
            for (uint32_t bits = byte; bits; bits &= bits - 1u) *dst++ = c + (uint32_t)(__ffs(bits) - 1);
        } else if (stage) {
            uint32_t sl = pj;
            for (uint32_t bits = byte; bits; bits &= bits - 1u) s_leaf[sl++] = c + (uint32_t)(__ffs(bits) - 1);
        } else {  // unstaged voxels: the one before comes from node x - 1
            uint32_t v = fd.vstart + (uint32_t)cw;
            bool have_prev = x > a0;
            uint64_t prev = have_prev ? last_child(src[x - 1 - a0], x > tx ? s_occ[j - 1] : a.occ[x - 1]) : 0ull;
            for (uint32_t bits = byte; bits; bits &= bits - 1u) {
                const uint64_t m = c + (uint32_t)(__ffs(bits) - 1);
                a.gap[v] = have_prev ? (uint8_t)gap_level(prev, m, 64) : (uint8_t)kInfLevel;
                if (a.pos) leaf_out(fd, a.ctab, v, m, a.pos);
                prev = m;
                have_prev = true;
                ++v;
            }
        }
    }
    if (bad) set_error(&a.st->err, kErrCorrupt);
    if (stage) {
        __syncthreads();
        const uint32_t lo = s_lo, hi = s_hi;
        const uint64_t vb = (uint64_t)fd.vstart + tb - base;  // voxel row of staged slot i: vb + i
        for (uint32_t i = lo + t; i < hi; i += kLevelThreads) {
            const uint64_t m = s_leaf[i];
            const uint32_t v = (uint32_t)(vb + i);
            a.gap[v] = (i > lo) ? (uint8_t)gap_level(s_leaf[i - 1], m, 64)
                                : (s_first ? (uint8_t)kInfLevel : (uint8_t)gap_level(s_prev, m, 64));
            if (a.pos) leaf_out(fd, a.ctab, v, m, a.pos);
        }
    }
}

// voxel-centre tables (Sec. 2.1), grid (x, frames): the centre table of frame blockIdx.y, entry a * 2^J + v =
// (float)(lo_a + (v + 0.5) * cell), the same FP64 expression as per voxel
__global__ void centre_tables_kernel(const DecFrame *fr, float *ctab)
{
    const DecFrame &d = fr[blockIdx.y];
    if (d.ctab_off == ~0ull) return;
    const uint64_t side = 1ull << d.J;
    float *t = ctab + d.ctab_off;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * side;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = (uint32_t)(e >> d.J);
        const uint64_t v = e & (side - 1);
        const double off = __dmul_rn(__dadd_rn((double)v, 0.5), d.grid.cell);
        t[e] = (float)__dadd_rn(d.grid.lo[a], off);
    }
}

__global__ void block_tables_kernel(const DecFrame *fr, uint32_t F, const uint64_t *blk_pref, uint64_t nblk,
                                    uint32_t *bw_all)
{
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nblk; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t f = find_frame(blk_pref, F, k);
        bw_all[k] = fr[f].bw[k - blk_pref[f]];
    }
}

uint32_t grid_for(uint64_t n, int num_sms)
{
    uint64_t b = (n + 255) / 256;
    const uint64_t cap = (uint64_t)num_sms * 8;
    if (b < 1) b = 1;
    return (uint32_t)(b < cap ? b : cap);
}

}  // namespace

void launch_batch_occ_bytes(const DecFrame *fr, uint32_t F, uint8_t *occ_all, uint64_t max_occ, int num_sms,
                            cudaStream_t s)
{
    if (max_occ == 0) return;
    uint32_t X = grid_for(max_occ, num_sms) / F + 1;
    occ_bytes_kernel<<<dim3(X, F), 256, 0, s>>>(fr, occ_all);
    count_launch();
}

void launch_batch_rans_decode(const DecFrame *fr, uint32_t F, uint32_t max_chunks_per_frame, uint32_t chunk_max,
                              uint8_t *occ_all, uint32_t *tabs, uint64_t *cstart, DevState *st, cudaStream_t s)
{
    (void)chunk_max;
    if (max_chunks_per_frame == 0) return;
    const uint64_t tab_words = kM / 4 + 256 + 4;
    tables_kernel<<<F, 1024, 0, s>>>(fr, tabs, tab_words, cstart, st);
    count_launch();
    const size_t smem = (size_t)ransdec::kTabWords * 4;
    cudaFuncSetAttribute(rans_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const uint32_t X = (max_chunks_per_frame + kRansWarps - 1) / kRansWarps;
    rans_batch_kernel<<<dim3(X, F), 32 * kRansWarps, smem, s>>>(fr, tabs, tab_words, cstart, occ_all, st);
    count_launch();
}

void launch_batch_roots(const DecFrame *fr, uint32_t F, uint64_t *nodes, uint8_t *gap, uint64_t nv_total,
                        cudaStream_t s)
{
    roots_kernel<<<(F + 63) / 64, 64, 0, s>>>(fr, F, nodes, gap, nv_total);
    count_launch();
}

uint64_t occ_tiles(uint64_t n_occ) { return (n_occ + kOccTile - 1) / kOccTile; }

void launch_occ_tile_bases(const uint8_t *occ, uint64_t n_occ, uint32_t *tsum, uint64_t *tbase, uint64_t *partials,
                           int num_sms, cudaStream_t s)
{
    const uint64_t nt = occ_tiles(n_occ);
    if (nt) {
        const uint64_t want = (nt + 7) / 8, cap = (uint64_t)num_sms * 8;
        occ_tile_popc_kernel<<<(uint32_t)(want < cap ? want : cap), 256, 0, s>>>(occ, n_occ, nt, tsum);
        count_launch();
    }
    launch_scan_u32_to_u64(tsum, nt, tbase, partials, num_sms, s);
}

void launch_batch_level(const DecFrame *fr, uint32_t F, uint32_t d, const uint32_t *tile_pref, uint32_t tiles,
                        const uint8_t *occ, uint64_t n_occ, const uint64_t *tbase, uint64_t *nodes, const float *ctab,
                        float *pos, uint8_t *gap, DevState *st, cudaStream_t s)
{
    if (tiles == 0) return;
    LevelArgs a{fr, F, d, tile_pref, occ, n_occ, tbase, nodes, ctab, pos, gap, st};
    expand_level_kernel<<<tiles, kLevelThreads, 0, s>>>(a);
    count_launch();
}

uint64_t occ_tile_first(uint64_t byte) { return byte / kOccTile; }

void launch_batch_centre_tables(const DecFrame *fr, uint32_t F, uint32_t Jmax, float *ctab, int num_sms,
                                cudaStream_t s)
{
    if (F == 0) return;
    uint32_t X = grid_for(3ull << Jmax, num_sms) / F + 1;
    centre_tables_kernel<<<dim3(X, F), 256, 0, s>>>(fr, ctab);
    count_launch();
}

void launch_batch_block_tables(const DecFrame *fr, uint32_t F, const uint64_t *blk_pref, uint64_t nblk,
                               uint32_t *bw_all, int num_sms, cudaStream_t s)
{
    if (nblk == 0) return;
    block_tables_kernel<<<grid_for(nblk, num_sms), 256, 0, s>>>(fr, F, blk_pref, nblk, bw_all);
    count_launch();
}

}  // namespace gsnfs
