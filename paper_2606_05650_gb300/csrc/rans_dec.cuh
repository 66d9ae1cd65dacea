// Decoding side of the occupancy rANS (Sec. 2.3 entropy stage; format of the
// occupancy section: 32 interleaved 32-bit states per chunk, L = 2^16,
// 16-bit renormalisation words, M = 2^15), shared by the one-frame and the
// batched decoders.  One warp decodes one chunk: lane j owns state j and
// symbols j, j + 32, ...; the words each step needs are handed out in lane
// order by a ballot.
#pragma once
#include "common.cuh"

namespace gsnfs {
namespace ransdec {

constexpr uint32_t kProbBits = 15;
constexpr uint32_t kM = 1u << kProbBits;
constexpr uint32_t kL = 1u << 16;
constexpr uint32_t kTabWords = kM / 4 + 256;  // slot -> symbol bytes, then freq << 16 | cum per symbol
constexpr uint32_t kMaxWarps = 8;

// whole CTA: copies the decoding tables (16-byte aligned, kTabWords words) into shared memory
__device__ __forceinline__ void load_tables(uint32_t *dst, const uint32_t *tab)
{
    const uint4 *s = reinterpret_cast<const uint4 *>(tab);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    for (uint32_t k = threadIdx.x; k < kTabWords / 4; k += blockDim.x) d[k] = s[k];
}

// one warp: decodes len symbols of a chunk (states then W words at src) to out;
// returns true if the chunk asked for more words than it holds
__device__ __forceinline__ bool decode_chunk(const uint8_t *slot2sym, const uint32_t *fc, const uint8_t *src,
                                             uint32_t W, uint32_t len, uint8_t *out, uint32_t lane)
{
    const uint16_t *words = reinterpret_cast<const uint16_t *>(src + 128);
    uint32_t x = reinterpret_cast<const uint32_t *>(src)[lane];
    const uint32_t ltm = lanemask_lt();
    uint32_t wp = 0;
    bool bad = false;
    for (uint32_t g = 0; g * 32 < len; ++g) {
        const uint32_t j = g * 32 + lane;
        bool need = false;
        if (j < len) {
            const uint32_t slot = x & (kM - 1);
            const uint32_t sy = slot2sym[slot];
            const uint32_t f = fc[sy];
            out[j] = (uint8_t)sy;
            x = (f >> 16) * (x >> kProbBits) + slot - (f & 0xFFFFu);
            need = x < kL;
        }
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, need);
        if (need) {
            const uint32_t k = wp + __popc(m & ltm);
            if (k < W) x = (x << 16) | words[k];
            else bad = true;
        }
        wp += __popc(m);
    }
    return __any_sync(0xFFFFFFFFu, bad);
}

// one warp: byte offset of chunk c inside the chunk area (sum of the sizes before it)
__device__ __forceinline__ uint64_t chunk_offset(const uint8_t *ctab, uint32_t c, uint32_t lane)
{
    uint64_t off = 0;
    for (uint32_t k = lane; k < c; k += 32) {
        const uint8_t *p = ctab + 4 * k;
        off += (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
    }
    for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xFFFFFFFFu, off, o);
    return off;
}

}  // namespace ransdec
}  // namespace gsnfs
