// Occupancy entropy stage (Sec. 2.2 last paragraph: the occupancy bytes are
// entropy coded with ANS; the paper uses a closed library, this codec its
// own static order-0 rANS after Duda 2013 with 32 interleaved states after
// Giesen 2014, so that one warp codes one chunk with one state per lane).
//
// Model: M = 2^15; f_s = floor(cnt_s * M / n), at least 1 for a present
// symbol; the most frequent symbol (lowest value on ties) absorbs M - sum f.
// 32-bit states, L = 2^16, 16-bit renormalisation words.  Symbol j of a
// chunk is coded by state j mod 32.  The encoder walks the chunk's groups of
// 32 symbols from last to first (lanes 31..0 within a group) pushing words on
// a stack; the decoder walks forward and pops them in lane order.
#include "kernels.cuh"
#include "rans_dec.cuh"

namespace gsnfs {

namespace {

constexpr uint32_t kProbBits = 15;
constexpr uint32_t kM = 1u << kProbBits;
constexpr uint32_t kL = 1u << 16;

// Byte histogram of each frame's occupancy bytes: 16 bytes per load (the
// bytes of a 16-byte word are counted from registers, so every thread keeps
// several loads in flight), counted into per-warp sub-histograms in shared
// memory (fewer lanes contend for a bin), added up per CTA.
__global__ void __launch_bounds__(256) hist_kernel(const uint8_t *__restrict__ occ, const uint64_t *occ_off,
                                                   DevState *st)
{
    __shared__ uint32_t h[8][256];
    const uint32_t f = blockIdx.y, t = threadIdx.x, wid = t >> 5;
    for (uint32_t k = t; k < 8 * 256; k += 256) (&h[0][0])[k] = 0;
    __syncthreads();
    const uint64_t b = occ_off[f], n = occ_off[f + 1] - b;
    const uint8_t *base = occ + b;
    const uint64_t head = n < ((16 - ((uintptr_t)base & 15)) & 15) ? n : ((16 - ((uintptr_t)base & 15)) & 15);
    const uint64_t n16 = (n - head) >> 4;
    const uint4 *v = reinterpret_cast<const uint4 *>(base + head);
    const uint64_t gt = (uint64_t)blockIdx.x * 256 + t, gs = (uint64_t)gridDim.x * 256;
    uint32_t *hw = h[wid];
    for (uint64_t i = gt; i < n16; i += 4 * gs) {
        uint4 x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = (i + u * gs < n16) ? __ldg(v + i + u * gs) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (i + u * gs >= n16) break;
            const uint32_t w[4] = {x[u].x, x[u].y, x[u].z, x[u].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                atomicAdd(&hw[w[e] & 255u], 1u);
                atomicAdd(&hw[(w[e] >> 8) & 255u], 1u);
                atomicAdd(&hw[(w[e] >> 16) & 255u], 1u);
                atomicAdd(&hw[w[e] >> 24], 1u);
            }
        }
    }
    // the bytes before the first 16-byte boundary and after the last one
    const uint64_t tail0 = head + (n16 << 4);
    if (gt < head) atomicAdd(&hw[base[gt]], 1u);
    if (gt < n - tail0) atomicAdd(&hw[base[tail0 + gt]], 1u);
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) c += h[w][t];
    if (c) atomicAdd(&st->hist[f][t], c);
}

// one CTA (256 threads) per frame: frequencies, cumulative table, mode
__global__ void __launch_bounds__(256) norm_kernel(const uint64_t *occ_off, DevState *st, uint16_t *freq,
                                                   uint32_t *cum, uint32_t *mode)
{
    const uint32_t f = blockIdx.x, s = threadIdx.x;
    const uint64_t n = occ_off[f + 1] - occ_off[f];
    const uint32_t cnt = st->hist[f][s];
    __shared__ uint32_t sh[33];
    __shared__ unsigned long long best;
    __shared__ uint32_t distinct;
    if (s == 0) {
        best = 0;
        distinct = 0;
    }
    __syncthreads();
    uint32_t fs = 0;
    if (cnt) {
        fs = (uint32_t)(((uint64_t)cnt * kM) / n);
        if (fs == 0) fs = 1;
        atomicAdd(&distinct, 1u);
        atomicMax(&best, ((unsigned long long)cnt << 8) | (255u - s));
    }
    uint32_t tot;
    block_exclusive_sum<uint32_t>(fs, sh, &tot);
    const uint32_t bs = 255u - (uint32_t)(best & 255u);
    if (cnt && s == bs) fs += kM - tot;
    uint32_t t2;
    uint32_t c = block_exclusive_sum<uint32_t>(fs, sh, &t2);
    freq[f * 256 + s] = (uint16_t)fs;
    cum[f * 256 + s] = c;
    if (s == 0) mode[f] = (n == 0) ? 0u : (distinct == 1 ? 2u : 1u);
}

__global__ void chunk_offsets_kernel(const uint64_t *occ_off, const uint32_t *mode, uint32_t F, uint32_t chunk,
                                     uint64_t *chunk_off)
{
    if (threadIdx.x) return;
    uint64_t run = 0;
    for (uint32_t f = 0; f < F; ++f) {
        chunk_off[f] = run;
        uint64_t n = occ_off[f + 1] - occ_off[f];
        if (mode[f] == 1) run += (n + chunk - 1) / chunk;
    }
    chunk_off[F] = run;
}

__device__ __forceinline__ uint32_t frame_of(const uint64_t *off, uint32_t F, uint64_t x)
{
    uint32_t lo = 0, hi = F;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// warp per chunk; slot layout: u32 state[32] at 0, u16 word stack [128, 128 + 2*chunk).
// Grid (x, frames): the CTAs of frame blockIdx.y share its coding tables in
// shared memory (reciprocals computed once per CTA); each warp stages its
// chunk's symbols in shared memory, 4,096 at a time.
constexpr int kEncWarps = 4;
constexpr uint32_t kStageSyms = 4096;  // symbols staged per pass

__global__ void __launch_bounds__(32 * kEncWarps) encode_kernel(const uint8_t *__restrict__ occ, const uint64_t *occ_off,
                                                               const uint64_t *chunk_off, uint32_t F, uint32_t chunk,
                                                               const uint16_t *freq, const uint32_t *cum, uint8_t *slots,
                                                               uint64_t slot_bytes, uint32_t *chunk_words,
                                                               uint32_t *chunk_top)
{
    __shared__ __align__(16) uint8_t s_sym[kEncWarps][kStageSyms];
    __shared__ uint32_t s_fc[256];   // freq << 16 | cum (cum < 2^15)
    __shared__ uint32_t s_rcp[256];  // ceil(2^32 / freq) for freq >= 2 (0 for freq < 2)
    const uint32_t lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const uint32_t f = blockIdx.y;
    (void)F;
    const uint64_t c0 = chunk_off[f], nch = chunk_off[f + 1] - c0;
    if ((uint64_t)blockIdx.x * kEncWarps >= nch) return;  // no chunk of this frame for this CTA
    for (uint32_t k = threadIdx.x; k < 256; k += blockDim.x) {
        const uint32_t fk = freq[f * 256 + k];
        s_fc[k] = (fk << 16) | cum[f * 256 + k];
        s_rcp[k] = fk >= 2 ? (uint32_t)((0x100000000ull + fk - 1) / fk) : 0u;
    }
    __syncthreads();
    const uint64_t n = occ_off[f + 1] - occ_off[f];
    for (uint64_t c = (uint64_t)blockIdx.x * kEncWarps + wl; c < nch; c += (uint64_t)gridDim.x * kEncWarps) {
        const uint64_t gc = c0 + c;
        const uint8_t *sym = occ + occ_off[f] + c * chunk;
        const uint32_t len = (uint32_t)((n - c * chunk) < chunk ? (n - c * chunk) : chunk);
        uint8_t *slot = slots + gc * slot_bytes;
        uint16_t *stack = reinterpret_cast<uint16_t *>(slot + 128);
        uint32_t top = chunk;
        uint32_t x = kL;
        const uint32_t G = (len + 31) / 32;
        // stage windows of symbols from the end of the chunk backwards
        int g = (int)G - 1;
        while (g >= 0) {
            const uint32_t win_lo_g = (uint32_t)g + 1 > kStageSyms / 32 ? (uint32_t)g + 1 - kStageSyms / 32 : 0u;
            const uint32_t b0 = win_lo_g * 32, b1 = ((uint32_t)g + 1) * 32 < len ? ((uint32_t)g + 1) * 32 : len;
            __syncwarp();
            {  // symbols [b0, b1): 16-byte loads over the aligned middle, bytes at the two ends
                const uintptr_t a0 = (uintptr_t)(sym + b0), a1 = (uintptr_t)(sym + b1);
                const uint32_t head = (uint32_t)((((a0 + 15) & ~(uintptr_t)15) - a0) < (a1 - a0)
                                                     ? ((a0 + 15) & ~(uintptr_t)15) - a0 : a1 - a0);
                const uint32_t nvec = (uint32_t)((b1 - b0 - head) >> 4);
                const uint4 *v = reinterpret_cast<const uint4 *>(sym + b0 + head);
                uint8_t *dst = &s_sym[wl][0];
                for (uint32_t k = lane; k < nvec; k += 32) {
                    const uint4 w = __ldg(v + k);
                    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst + head + 16 * k);  // byte-addressed smem
                    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (((head + 16 * k) & 3) == 0) {
                            d32[e] = ws[e];
                        } else {
#pragma unroll
                            for (int bb = 0; bb < 4; ++bb) dst[head + 16 * k + 4 * e + bb] = (uint8_t)(ws[e] >> (8 * bb));
                        }
                    }
                }
                if (lane < head) dst[lane] = sym[b0 + lane];
                const uint32_t t0 = head + 16 * nvec;
                if (lane < (b1 - b0) - t0) dst[t0 + lane] = sym[b0 + t0 + lane];
            }
            __syncwarp();
            for (; g >= (int)win_lo_g; --g) {
                const uint32_t j = (uint32_t)g * 32 + lane;
                const bool valid = j < len;
                const uint32_t sy = valid ? s_sym[wl][j - b0] : 0u;
                const uint32_t fc = s_fc[sy], rcp = s_rcp[sy];
                const uint32_t fs = fc >> 16, cs = fc & 0xFFFFu;
                const bool need = valid && ((uint64_t)x >= ((uint64_t)fs << 17));
                const uint32_t m = __ballot_sync(0xFFFFFFFFu, need);
                if (need) {
                    const uint32_t above = __popc(m >> lane) - 1u;  // emitting lanes above this one
                    stack[top - 1 - above] = (uint16_t)(x & 0xFFFFu);
                    x >>= 16;
                }
                top -= __popc(m);
                if (valid) {
                    // x / fs and x % fs: the estimate floor(x * ceil(2^32/fs) / 2^32) is the
                    // quotient or one more (the error term x / 2^32 is below 1)
                    uint32_t qt = fs >= 2 ? __umulhi(x, rcp) : x;
                    int32_t rm = (int32_t)(x - qt * fs);
                    if (rm < 0) {
                        --qt;
                        rm += (int32_t)fs;
                    }
                    x = (qt << kProbBits) + (uint32_t)rm + cs;
                }
            }
        }
        reinterpret_cast<uint32_t *>(slot)[lane] = x;
        if (lane == 0) {
            chunk_words[gc] = chunk - top;
            chunk_top[gc] = top;
        }
        __syncwarp();
    }
}

// per frame (one warp each): chunk positions by a warp scan of the chunk
// sizes, the occupancy section size and the final mode (rANS only when
// smaller than raw)
__global__ void __launch_bounds__(256) section_size_kernel(const uint64_t *occ_off, const uint64_t *chunk_off,
                                                           uint32_t F, const uint32_t *chunk_words,
                                                           uint32_t *chunk_pos, uint32_t *mode, uint64_t *sec_bytes)
{
    const uint32_t f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint32_t lane = threadIdx.x & 31;
    if (f >= F) return;
    const uint64_t n = occ_off[f + 1] - occ_off[f];
    const uint64_t raw = 16 + ((n + 7) & ~7ull);
    const uint32_t md = mode[f];
    if (md == 2) {
        if (lane == 0) sec_bytes[f] = 16;
        return;
    }
    if (md == 1) {
        const uint64_t c0 = chunk_off[f], nch = chunk_off[f + 1] - c0;
        uint64_t t = (16 + 8 + 512 + 4 * nch + 7) & ~7ull;
        for (uint64_t base = 0; base < nch; base += 32) {
            const uint64_t c = base + lane;
            const uint32_t sz = c < nch ? (uint32_t)((128 + 2 * (uint64_t)chunk_words[c0 + c] + 3) & ~3ull) : 0u;
            const uint32_t inc = warp_inclusive_sum(sz);
            if (c < nch) chunk_pos[c0 + c] = (uint32_t)(t + inc - sz);
            t += __shfl_sync(0xFFFFFFFFu, inc, 31);
        }
        t = (t + 7) & ~7ull;
        if (t < raw) {
            if (lane == 0) sec_bytes[f] = t;
            return;
        }
        __syncwarp();
        if (lane == 0) mode[f] = 0;
    }
    if (lane == 0) sec_bytes[f] = raw;
}

// ---- decoder: warp per chunk of one frame; the chunk (states and words) is
// copied to shared memory with coalesced loads, then decoded from there.

// slot -> symbol table (kM bytes) and freq << 16 | cum (256 words) of one
// section, followed by a corruption flag; one CTA of 1024 threads
__global__ void __launch_bounds__(1024) table_kernel(const uint8_t *__restrict__ sec, uint32_t *tabs, DevState *st)
{
    __shared__ uint32_t s_cm[256];
    __shared__ uint32_t s_fc[256];
    uint8_t *slot2sym = reinterpret_cast<uint8_t *>(tabs);
    const uint8_t *ftab = sec + 24;
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
            tabs[kM / 4 + 256] = (run != kM);
            if (run != kM) set_error(&st->err, kErrCorrupt);
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < 256; t += blockDim.x) tabs[kM / 4 + t] = s_fc[t];
    for (uint32_t t = threadIdx.x; t < kM; t += blockDim.x) {  // symbol of each slot: last s with cum[s] <= t
        uint32_t lo = 0, hi = 256;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_cm[mid] <= t) lo = mid; else hi = mid;
        }
        slot2sym[t] = (uint8_t)lo;
    }
}

// One frame's chunks, a warp per chunk read in place (its words are consumed
// in order, so they come from L1).  Each CTA first turns the chunk size table
// into chunk offsets in shared memory (one block scan per 1,024 chunks) when
// they fit (kSmemChunks), else each warp sums the sizes before its chunk.
constexpr uint32_t kSmemChunks = 4096;

__global__ void __launch_bounds__(32 * ransdec::kMaxWarps) decode_kernel(const uint8_t *__restrict__ sec,
                                                                         uint64_t sec_bytes, uint64_t n, uint32_t nch,
                                                                         uint32_t chunk, uint8_t *out, DevState *st,
                                                                         const uint32_t *tabs)
{
    using namespace ransdec;
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ uint32_t sh[33];
    // decoding tables built once by table_kernel: copy them in
    if (tabs[kTabWords] != 0) return;  // frequencies did not sum to M (reported by table_kernel)
    load_tables(reinterpret_cast<uint32_t *>(dsm), tabs);
    const uint8_t *ctab = sec + 24 + 512;
    const uint64_t table = (16 + 8 + 512 + 4 * (uint64_t)nch + 7) & ~7ull;
    const bool local = nch <= kSmemChunks && sec_bytes < (1ull << 32);
    uint32_t *s_start = reinterpret_cast<uint32_t *>(dsm + kTabWords * 4);
    if (local) {
        uint32_t run = (uint32_t)table;
        for (uint32_t b = 0; b < nch; b += blockDim.x) {
            const uint32_t c = b + threadIdx.x;
            uint32_t sz = 0;
            if (c < nch) {
                const uint8_t *q = ctab + 4 * c;
                sz = (uint32_t)q[0] | ((uint32_t)q[1] << 8) | ((uint32_t)q[2] << 16) | ((uint32_t)q[3] << 24);
            }
            uint32_t tot;
            const uint32_t ex = block_exclusive_sum<uint32_t>(sz, sh, &tot);
            if (c < nch) s_start[c] = run + ex;  // wraps only for sizes that fail the bounds check below
            run += tot;
        }
    }
    __syncthreads();
    const uint8_t *slot2sym = dsm;
    const uint32_t *fc = reinterpret_cast<const uint32_t *>(dsm + kM);
    const uint32_t lane = threadIdx.x & 31, wl = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (uint32_t c = blockIdx.x * nwarps + wl; c < nch; c += gridDim.x * nwarps) {
        const uint64_t start = local ? s_start[c] : table + chunk_offset(ctab, c, lane);
        const uint8_t *cp = ctab + 4 * c;
        const uint32_t cbytes = (uint32_t)cp[0] | ((uint32_t)cp[1] << 8) | ((uint32_t)cp[2] << 16) | ((uint32_t)cp[3] << 24);
        if (cbytes < 128 || (cbytes & 3) || cbytes > 128 + 2 * chunk + 2 || start + cbytes > sec_bytes) {
            if (lane == 0) set_error(&st->err, kErrCorrupt);
            continue;
        }
        const uint64_t s0 = (uint64_t)c * chunk;
        const uint32_t len = (uint32_t)((n - s0) < chunk ? (n - s0) : chunk);
        if (decode_chunk(slot2sym, fc, sec + start, (cbytes - 128) / 2, len, out + s0, lane) && lane == 0)
            set_error(&st->err, kErrCorrupt);
    }
}

__global__ void fill_kernel(uint8_t *out, uint64_t n, uint8_t v)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = v;
}

}  // namespace

uint64_t rans_chunk_slot_bytes(uint32_t chunk) { return 128 + 2 * (uint64_t)chunk + 16; }

void launch_rans_encode(const RansFrames &r, DevState *st, uint64_t max_chunks, int num_sms, cudaStream_t s)
{
    dev_memset(&st->hist[0][0], 0, sizeof(uint32_t) * 256 * r.F, s);
    dim3 g(num_sms, r.F);
    if (r.F > 8) g.x = (num_sms * 8 + r.F - 1) / r.F;
    hist_kernel<<<g, 256, 0, s>>>(r.occ, r.occ_off, st);
    count_launch();
    norm_kernel<<<r.F, 256, 0, s>>>(r.occ_off, st, r.freq, r.cum, r.mode);
    count_launch();
    chunk_offsets_kernel<<<1, 32, 0, s>>>(r.occ_off, r.mode, r.F, r.chunk, r.chunk_off);
    count_launch();
    if (max_chunks) {
        // per frame: enough CTAs to fill the GPU when every frame has chunks, at most one chunk per warp
        uint64_t per = ((uint64_t)num_sms * 8 + r.F - 1) / r.F;
        const uint64_t need = (max_chunks + kEncWarps - 1) / kEncWarps;
        if (per > need) per = need;
        if (per < 1) per = 1;
        encode_kernel<<<dim3((uint32_t)per, r.F), 32 * kEncWarps, 0, s>>>(r.occ, r.occ_off, r.chunk_off, r.F, r.chunk, r.freq, r.cum,
                                                        r.chunk_slots, rans_chunk_slot_bytes(r.chunk), r.chunk_words,
                                                        r.chunk_top);
        count_launch();
    }
    section_size_kernel<<<(r.F + 7) / 8, 256, 0, s>>>(r.occ_off, r.chunk_off, r.F, r.chunk_words, r.chunk_pos,
                                                      r.mode, r.sec_bytes);
    count_launch();
}

uint64_t rans_table_words() { return kM / 4 + 256 + 4; }

void launch_rans_decode(const uint8_t *sec, uint64_t sec_bytes, uint64_t n, uint32_t nch, uint32_t chunk,
                        uint8_t *out, uint32_t *tabs, DevState *st, int num_sms, cudaStream_t s)
{
    if (nch == 0) return;
    table_kernel<<<1, 1024, 0, s>>>(sec, tabs, st);
    count_launch();
    const uint32_t warps = ransdec::kMaxWarps;
    uint32_t blocks = (nch + warps - 1) / warps;
    if (blocks > (uint32_t)num_sms * 4) blocks = (uint32_t)num_sms * 4;
    const size_t smem = (size_t)ransdec::kTabWords * 4 + 4 * (size_t)kSmemChunks;
    cudaFuncSetAttribute(decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    decode_kernel<<<blocks, 32 * warps, smem, s>>>(sec, sec_bytes, n, nch, chunk, out, st, tabs);
    count_launch();
}

void launch_fill(uint8_t *out, uint64_t n, uint8_t v, cudaStream_t s)
{
    if (n) {
        fill_kernel<<<64, 256, 0, s>>>(out, n, v);
        count_launch();
    }
}

}  // namespace gsnfs
