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

// per frame: slot -> symbol table and freq << 16 | cum, then a corruption flag
__global__ void __launch_bounds__(1024) tables_kernel(const DecFrame *fr, uint32_t *tabs, uint64_t tab_words,
                                                      DevState *st)
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
}

// grid (chunk groups, frames): warp per chunk of frame blockIdx.y
__global__ void __launch_bounds__(32 * ransdec::kMaxWarps) rans_batch_kernel(const DecFrame *fr, const uint32_t *tabs,
                                                                             uint64_t tab_words, uint32_t chunk_max,
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
    const bool staged = chunk_max <= 32768;
    uint32_t *cbuf = reinterpret_cast<uint32_t *>(dsm + kTabWords * 4 + (size_t)wl * stage_bytes(chunk_max));
    const uint8_t *ctab = d.occ_sec + 24 + 512;
    const uint64_t table = (16 + 8 + 512 + 4 * (uint64_t)nch + 7) & ~7ull;
    uint8_t *out = occ_all + d.occ_off;
    for (uint32_t c = blockIdx.x * nwarps + wl; c < nch; c += gridDim.x * nwarps) {
        const uint64_t start = table + chunk_offset(ctab, c, lane);
        const uint8_t *cp = ctab + 4 * c;
        const uint32_t cbytes = (uint32_t)cp[0] | ((uint32_t)cp[1] << 8) | ((uint32_t)cp[2] << 16) | ((uint32_t)cp[3] << 24);
        if (cbytes < 128 || (cbytes & 3) || cbytes > 128 + 2 * chunk + 2 || start + cbytes > d.occ_bytes) {
            if (lane == 0) set_error(&st->err, kErrCorrupt);
            continue;
        }
        const uint8_t *src = d.occ_sec + start;
        if (staged) {
            stage_chunk(cbuf, reinterpret_cast<const uint32_t *>(src), cbytes / 4, lane);
            src = reinterpret_cast<const uint8_t *>(cbuf);
        }
        const uint64_t s0 = (uint64_t)c * chunk;
        const uint32_t len = (uint32_t)((d.n_occ - s0) < chunk ? (d.n_occ - s0) : chunk);
        if (decode_chunk(slot2sym, fc, src, (cbytes - 128) / 2, len, out + s0, lane) && lane == 0)
            set_error(&st->err, kErrCorrupt);
    }
}

__global__ void roots_kernel(const DecFrame *fr, uint32_t F, uint64_t *nodes, uint64_t *codes)
{
    const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F || fr[f].nv == 0) return;
    nodes[fr[f].noff[0]] = 0ull;  // implicit root code of Algorithm 2
    (void)codes;
}

// Levels d .. d + K (K <= 2) of Algorithm 3 for every frame with J > d in one
// launch: a thread takes one node of level d and walks its descendants depth
// first down to level min(d + K, J) (children in increasing bit order, so
// every level's nodes are visited in their breadth-first order), writing only
// that last level; the level in between is never stored.  K = 2 only where
// the second level holds at most 4 nodes per node of the first (chosen on the
// host): longer walks were measured slower (a thread's chain of dependent
// loads and the divergence of uneven subtrees outweigh the saved traffic).
// A thread's nodes mostly stay in one frame, so the frame's tables are looked
// up once per change.
constexpr int kExpandMaxLevels = 2;

struct ExpandFrame {
    const uint64_t *src;                    // level d codes
    uint64_t *dst;                          // last level's codes
    uint64_t bo[kExpandMaxLevels];          // byte offset of level d + k in the batch occupancy buffer
    uint32_t base[kExpandMaxLevels];        // popcount prefix at the start of level d + k
    uint32_t M[kExpandMaxLevels + 1];       // node count of level d + k
    int levels;                             // levels walked: min(K, J - d)
};

template <int k>
__device__ __forceinline__ void expand_walk(const ExpandFrame &x, const uint8_t *__restrict__ occ,
                                            const uint32_t *__restrict__ pref, uint64_t code, uint32_t w,
                                            DevState *st)
{
    // node w of level d + k, with its code
    if (k == x.levels) {
        x.dst[w] = code;
        return;
    }
    if constexpr (k < kExpandMaxLevels) {
        const uint32_t byte = occ[x.bo[k] + w];
        if (byte == 0) {
            set_error(&st->err, kErrCorrupt);
            return;
        }
        const uint64_t c = code << 3;
        uint32_t cw = pref[x.bo[k] + w] - x.base[k];
        for (uint32_t bits = byte; bits; bits &= bits - 1u) {  // set bits in increasing order
            if (cw < x.M[k + 1]) expand_walk<k + 1>(x, occ, pref, c + (uint32_t)(__ffs(bits) - 1), cw, st);
            else set_error(&st->err, kErrCorrupt);
            ++cw;
        }
    }
}

__global__ void __launch_bounds__(256) expand_batch_kernel(const DecFrame *fr, uint32_t F, uint32_t d, uint32_t K,
                                                           const uint64_t *lvl_pref, uint64_t count,
                                                           const uint8_t *__restrict__ occ_all,
                                                           const uint32_t *__restrict__ pref, uint64_t *nodes,
                                                           uint64_t *codes, DevState *st)
{
    uint64_t fbeg = 1, fend = 0;  // node range of the cached frame (empty at first)
    ExpandFrame x;
    for (uint64_t gp = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; gp < count;
         gp += (uint64_t)gridDim.x * blockDim.x) {
        if (gp < fbeg || gp >= fend) {
            const uint32_t f = find_frame(lvl_pref, F, gp);
            const DecFrame &fd = fr[f];
            fbeg = lvl_pref[f];
            fend = lvl_pref[f + 1];
            x.levels = (int)min(K, fd.J - d);
            x.src = nodes + fd.noff[d];
            x.dst = (d + (uint32_t)x.levels == fd.J) ? codes + fd.vstart : nodes + fd.noff[d + x.levels];
            x.M[0] = fd.lsz[d];
#pragma unroll
            for (int k = 0; k < kExpandMaxLevels; ++k) {
                if (k < x.levels) {
                    x.bo[k] = fd.occ_off + fd.boff[d + k];
                    x.base[k] = pref[x.bo[k]];
                    x.M[k + 1] = fd.lsz[d + k + 1];
                    // the popcounts of level d + k add up to the size of level d + k + 1
                    if (gp == fbeg && pref[x.bo[k] + x.M[k]] - x.base[k] != x.M[k + 1])
                        set_error(&st->err, kErrCorrupt);
                }
            }
        }
        const uint32_t p = (uint32_t)(gp - fbeg);
        expand_walk<0>(x, occ_all, pref, x.src[p], p, st);
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

// voxel centres (Sec. 2.1) and gap levels of every frame's voxels
// grid (x, frames): the centre table of frame blockIdx.y, entry a * 2^J + v =
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

__global__ void centres_gaps_kernel(const DecFrame *fr, uint32_t F, const uint32_t *vstart, uint64_t nv_total,
                                    const uint64_t *__restrict__ codes, const float *__restrict__ ctab, float *pos,
                                    uint8_t *gap)
{
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= nv_total;
         v += (uint64_t)gridDim.x * blockDim.x) {
        if (v == nv_total) {
            gap[v] = (uint8_t)kInfLevel;
            continue;
        }
        const uint32_t f = find_frame(vstart, F, v);
        const uint64_t m = codes[v];
        gap[v] = (v == vstart[f]) ? (uint8_t)kInfLevel : (uint8_t)gap_level(codes[v - 1], m, 64);
        if (pos) {
            const DecFrame &d = fr[f];
            if (d.ctab_off != ~0ull) {
                const float *t = ctab + d.ctab_off;
#pragma unroll
                for (int a = 0; a < 3; ++a) pos[3 * v + a] = t[((uint64_t)a << d.J) + compact3b(m >> a)];
            } else {
                const FrameGrid g = d.grid;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const double off = __dmul_rn(__dadd_rn((double)compact3b(m >> a), 0.5), g.cell);
                    pos[3 * v + a] = (float)__dadd_rn(g.lo[a], off);
                }
            }
        }
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
                              uint8_t *occ_all, uint32_t *tabs, DevState *st, cudaStream_t s)
{
    if (max_chunks_per_frame == 0) return;
    const uint64_t tab_words = kM / 4 + 256 + 4;
    tables_kernel<<<F, 1024, 0, s>>>(fr, tabs, tab_words, st);
    count_launch();
    const bool staged = chunk_max <= 32768;
    const uint32_t warps = staged ? ransdec::warps_per_cta(chunk_max) : ransdec::kMaxWarps;
    const size_t smem = staged ? ransdec::smem_bytes(chunk_max, warps) : (size_t)ransdec::kTabWords * 4;
    cudaFuncSetAttribute(rans_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const uint32_t X = (max_chunks_per_frame + warps - 1) / warps;
    rans_batch_kernel<<<dim3(X, F), 32 * warps, smem, s>>>(fr, tabs, tab_words, chunk_max, occ_all, st);
    count_launch();
}

void launch_batch_roots(const DecFrame *fr, uint32_t F, uint64_t *nodes, uint64_t *codes, cudaStream_t s)
{
    roots_kernel<<<(F + 63) / 64, 64, 0, s>>>(fr, F, nodes, codes);
    count_launch();
}

void launch_batch_expand(const DecFrame *fr, uint32_t F, uint32_t d, uint32_t K, const uint64_t *lvl_pref,
                         uint64_t count,
                         const uint8_t *occ_all, const uint32_t *pref, uint64_t *nodes, uint64_t *codes,
                         DevState *st, int num_sms, cudaStream_t s)
{
    if (count == 0) return;
    expand_batch_kernel<<<grid_for(count, num_sms), 256, 0, s>>>(fr, F, d, K, lvl_pref, count, occ_all, pref, nodes,
                                                                 codes, st);
    count_launch();
}

void launch_batch_centre_tables(const DecFrame *fr, uint32_t F, uint32_t Jmax, float *ctab, int num_sms,
                                cudaStream_t s)
{
    if (F == 0) return;
    uint32_t X = grid_for(3ull << Jmax, num_sms) / F + 1;
    centre_tables_kernel<<<dim3(X, F), 256, 0, s>>>(fr, ctab);
    count_launch();
}

void launch_batch_centres_gaps(const DecFrame *fr, uint32_t F, const uint32_t *vstart, uint64_t nv_total,
                               const uint64_t *codes, const float *ctab, float *pos, uint8_t *gap, int num_sms,
                               cudaStream_t s)
{
    centres_gaps_kernel<<<grid_for(nv_total + 1, num_sms), 256, 0, s>>>(fr, F, vstart, nv_total, codes, ctab, pos,
                                                                         gap);
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

namespace gsnfs {
uint32_t batch_expand_max_levels() { return (uint32_t)kExpandMaxLevels; }
}  // namespace gsnfs
