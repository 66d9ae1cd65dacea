// Quantisation and block RLGR entropy coding of RAHT coefficients
// (Sec. 3.4 "Quantization and Entropy Coding"; App. H, Table A.5).
//
// Each attribute channel is cut into blocks of B consecutive coefficients
// (Morton / in-place order of the transform output) and every block is one
// independent adaptive run-length Golomb-Rice stream coded by one thread
// (the paper's block parallelisation).  Threads of a CTA are the channels of
// one block of rows, so the row-major coefficient matrix is read row by row
// with coalesced loads; the quantiser (dead-zone / uniform, per group step)
// is applied on the fly.  RLGR constants (Malvar 2006 reading):
//   u = zigzag(q); k = K >> 4, kR = KR >> 4; K = 0, KR = 32 at block start.
//   k == 0: GR(u, kR); u == 0 -> K += 3 (cap 240), else K -= 3 (floor 0).
//   k >  0: a full run of 2^k zeros -> bit 0, K += 4; r < 2^k zeros then
//           u != 0 -> bit 1, r in k bits, GR(u - 1, kR), K -= 6; a run cut
//           by the block end -> bit 0 (the decoder clamps).
//   GR(v, k): p = v >> k; p < 24 -> p ones, a zero, the k low bits of v;
//            else 24 ones, 6-bit length n of v, the n bits of v.
//            p == 0 -> KR -= 2 (floor 0); p > 1 -> KR += p + 1 (cap 384).
//   Bits are packed least-significant first into 32-bit words; a block ends
//   on a word boundary.  At most 78 bits per coefficient.
#include "kernels.cuh"

namespace gsnfs {

namespace {

constexpr int kUnaryEsc = 24;

// Bits are appended LSB first to a 32-bit word (cur, nacc bits used); a value
// that straddles the word boundary leaves its upper part in the next word via
// one funnel shift.  Words beyond `cap` are counted but not stored.
struct BitWriter {
    uint32_t cur;
    uint32_t nacc;
    uint32_t nw;
    uint32_t *out;
    uint32_t cap;
    __device__ __forceinline__ void emit(uint32_t w)
    {
        if (nw < cap) out[nw] = w;
        ++nw;
    }
    __device__ __forceinline__ void put(uint32_t v, uint32_t n)  // n <= 32, v < 2^n
    {
        const uint32_t spill = __funnelshift_l(v, 0u, nacc);  // bits of v above the word, if any
        cur |= v << nacc;  // nacc < 32
        nacc += n;
        if (nacc >= 32u) {
            emit(cur);
            cur = spill;
            nacc -= 32u;
        }
    }
    __device__ __forceinline__ void flush()
    {
        if (nacc) {
            emit(cur);
            cur = 0;
            nacc = 0;
        }
    }
};

__device__ __forceinline__ uint32_t zz(int32_t q)
{
    return q >= 0 ? ((uint32_t)q << 1) : ((((uint32_t)(-(q + 1))) << 1) | 1u);
}

__device__ __forceinline__ int32_t unzz(uint32_t u)
{
    return (u & 1u) ? -(int32_t)(u >> 1) - 1 : (int32_t)(u >> 1);
}

__device__ __forceinline__ void adapt_kr(uint32_t p, int &KR)
{
    // p = 0: KR - 2, p = 1: unchanged, p > 1: KR + p + 1; within [0, 384]
    const int d = p >= 2u ? (int)(p > 384u ? 384u : p) + 1 : (p == 1u ? 0 : -2);
    KR = min(max(KR + d, 0), 384);
}

__device__ __forceinline__ void gr_put(BitWriter &bw, uint32_t v, uint32_t k, int &KR)
{
    const uint32_t p = v >> k;
    if (__builtin_expect(p + 1u + k <= 32u && p < (uint32_t)kUnaryEsc, 1)) {  // common case: one write
        // p ones, a zero, then the k low bits of v, least significant first:
        // ((2 low + 1) << p) - 1, where low = v mod 2^k (k <= 24)
        const uint32_t low = v & ((1u << k) - 1u);
        bw.put((((low << 1) | 1u) << p) - 1u, p + 1u + k);
    } else if (p < (uint32_t)kUnaryEsc) {
        bw.put((1u << p) - 1u, p + 1u);
        bw.put(v & ((1u << k) - 1u), k);
    } else {
        const uint32_t n = 32u - (uint32_t)__clz(v);
        bw.put((1u << kUnaryEsc) - 1u, kUnaryEsc);
        bw.put(n, 6);
        bw.put(v, n);
    }
    adapt_kr(p, KR);
}

// Streaming RLGR coder state of one block.
struct Rlgr {
    int K, KR;
    uint32_t z;  // pending zeros of an open run
    __device__ __forceinline__ void init()
    {
        K = 0;
        KR = 32;
        z = 0;
    }
    __device__ __forceinline__ void code(BitWriter &bw, uint32_t u)
    {
        const uint32_t k = (uint32_t)K >> 4;
        if (__builtin_expect(k == 0, 1)) {  // Golomb-Rice mode
            gr_put(bw, u, (uint32_t)KR >> 4, KR);
            K = u == 0 ? K + 3 : (K >= 3 ? K - 3 : 0);  // Golomb-Rice mode runs while K < 16: no cap at 240
        } else if (u == 0) {
            if (++z == (1u << k)) {
                bw.put(0, 1);
                K += 4;
                if (K > 240) K = 240;
                z = 0;
            }
        } else {
            bw.put(1u | (z << 1), 1u + k);  // bit 1, then the run length in k bits (z < 2^k, k <= 15)
            gr_put(bw, u - 1u, (uint32_t)KR >> 4, KR);
            K = K >= 6 ? K - 6 : 0;
            z = 0;
        }
    }
    __device__ __forceinline__ void finish(BitWriter &bw)
    {
        if (z) bw.put(0, 1);
        bw.flush();
    }
};

// ---- encoder: one CTA per rb row blocks; thread = (row block, rung, channel) --
// Each thread reads its channel's coefficients straight from global memory
// (lanes of a warp are consecutive channels of a row, so a warp's load is one
// contiguous run of the row) with the next kPrefetch rows in flight in
// registers while the current ones are coded; threads never wait for each
// other after the CTA's one barrier.  Threads of the other rungs of a row
// read the same words (served by L1).
struct EncJobs {
    RlgrJob j;
    const uint64_t *job_off;  // F + 1: first job (row block) of each frame
};

constexpr uint32_t kPrefetch = 4;

// Row blocks per CTA: enough that rb * W (W = rungs x channels threads per
// row block) fills whole warps (rb = 32 / gcd(W, 32)), at most 512 threads.
__host__ __device__ inline uint32_t row_blocks_per_cta(uint32_t W)
{
    uint32_t g = 32;
    while (W % g) g >>= 1;
    uint32_t rb = 32 / g;
    if (rb * W > 512) rb = W >= 512 ? 1 : 512 / W;
    return rb;
}

struct EncBlock {  // one row block of a CTA
    uint64_t gbase;  // first coefficient (row-major) of the block
    uint32_t f, b, nb, len;
};

template <bool FROM_INT, bool DIST>
__global__ void __launch_bounds__(512) rlgr_encode_kernel(EncJobs E, const int32_t *qin, uint32_t rb)
{
    __shared__ EncBlock blk_info[32];
    const RlgrJob &j = E.j;
    const uint32_t C = j.C, W = j.R * C;
    const uint64_t njobs = E.job_off[j.F];
    const uint32_t t = threadIdx.x;
    if (t < rb) {  // describe the CTA's row blocks
        EncBlock e{0, 0, 0, 0, 0};
        const uint64_t job = (uint64_t)blockIdx.x * rb + t;
        if (job < njobs) {
            uint32_t lo = 0, hi = j.F;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (E.job_off[mid] <= job) lo = mid; else hi = mid;
            }
            const uint32_t vs = j.vstart[lo], nv = j.vstart[lo + 1] - vs;
            e.f = lo;
            e.b = (uint32_t)(job - E.job_off[lo]);
            e.nb = (nv + j.B - 1) / j.B;
            const uint32_t row0 = e.b * j.B;
            e.len = (nv - row0) < j.B ? (nv - row0) : j.B;
            e.gbase = ((uint64_t)vs + row0) * C;
        }
        blk_info[t] = e;
    }
    __syncthreads();
    const uint32_t jl = t / W;
    if (jl >= rb) return;
    const EncBlock me = blk_info[jl];
    if (me.len == 0) return;
    const uint32_t w = t - jl * W;
    const uint32_t r = w / C, c = w - r * C;
    const uint64_t blk = j.blk_off[me.f] + ((uint64_t)r * me.nb + me.b) * C + c;
    BitWriter bw{0u, 0u, 0u, j.slots + blk * j.slot_words, j.slot_words};
    Rlgr st;
    st.init();
    const float inv = FROM_INT ? 0.f : j.inv_step[r * C + c];
    const float stp = DIST ? j.step[r * C + c] : 0.f;
    float sq = 0.f;
    double dc_err = 0.0;
    const uint32_t *src = FROM_INT ? reinterpret_cast<const uint32_t *>(qin) : reinterpret_cast<const uint32_t *>(j.Y);
    const uint32_t *col = src + me.gbase + c;  // row i of this channel at col[i * C]
    const uint32_t len = me.len;
    uint32_t i = 0;
    if (!FROM_INT && j.dc && me.b == 0) {  // the frame's DC: quantised from its FP64 value
        const double y = j.dc[(uint64_t)me.f * C + c], st64 = j.steps_rg[r * j.G + j.groups[c]];
        const int32_t q = quantize_f64(y, st64, j.tau64);
        st.code(bw, zz(q));
        if (DIST) {
            const double e = __dsub_rn(y, __dmul_rn((double)q, st64));
            dc_err = __dmul_rn(e, e);
        }
        i = 1;
    }
    auto code_one = [&](uint32_t x) {
        if (DIST) {  // squared error of the dequantised coefficient (Parseval: of the attributes)
            const float y = __uint_as_float(x);
            const int32_t q = quantize_f32(y, inv, j.tau);
            const float e = __fsub_rn(y, __fmul_rn((float)q, stp));
            sq = __fadd_rn(sq, __fmul_rn(e, e));
            st.code(bw, zz(q));
        } else {
            st.code(bw, FROM_INT ? zz((int32_t)x) : quantize_zz_f32(__uint_as_float(x), inv, j.tau));
        }
    };
    uint32_t cur[kPrefetch];
#pragma unroll
    for (uint32_t d = 0; d < kPrefetch; ++d) cur[d] = (i + d < len) ? __ldg(col + (uint64_t)(i + d) * C) : 0u;
    for (; i + kPrefetch <= len; i += kPrefetch) {
        uint32_t nx[kPrefetch];
        const uint32_t *q = col + (uint64_t)(i + kPrefetch) * C;
#pragma unroll
        for (uint32_t d = 0; d < kPrefetch; ++d) nx[d] = (i + kPrefetch + d < len) ? __ldg(q + d * C) : 0u;
#pragma unroll
        for (uint32_t d = 0; d < kPrefetch; ++d) code_one(cur[d]);
#pragma unroll
        for (uint32_t d = 0; d < kPrefetch; ++d) cur[d] = nx[d];
    }
#pragma unroll
    for (uint32_t d = 0; d < kPrefetch; ++d)
        if (i + d < len) code_one(cur[d]);
    st.finish(bw);
    j.block_words[blk] = bw.nw;
    if (bw.nw > j.slot_words) atomicExch(j.overflow, 1u);
    if (DIST) atomicAdd(j.sq_err + ((uint64_t)me.f * j.R + r) * C + c, __dadd_rn((double)sq, dc_err));
}

// ---- decoder ------------------------------------------------------------------
// Bits are looked at through a 32-bit window over two consecutive words
// (cur, nxt) at bit offset pos: one funnel shift per look and one word load
// every 32 bits consumed.  Words past the end of a stream read as zero, so a
// malformed stream cannot make the reader leave it; whether the stream was
// overrun is checked once, after its last coefficient, from the bits consumed.
struct WinReader {
    const uint32_t *w;
    uint32_t nw, cur, nxt, pos, idx;
    __device__ __forceinline__ void init(const uint32_t *p, uint32_t n)
    {
        w = p;
        nw = n;
        cur = n > 0 ? p[0] : 0u;
        nxt = n > 1 ? p[1] : 0u;
        pos = 0;
        idx = 2;
    }
    __device__ __forceinline__ uint32_t peek() const { return __funnelshift_r(cur, nxt, pos); }
    __device__ __forceinline__ void skip(uint32_t n)  // n <= 32
    {
        pos += n;
        if (pos >= 32u) {
            pos -= 32u;
            cur = nxt;
            nxt = idx < nw ? w[idx] : 0u;
            ++idx;
        }
    }
    __device__ __forceinline__ bool overrun() const
    {
        return (uint64_t)(idx - 2u) * 32u + pos > (uint64_t)nw * 32u;
    }
};


// Rare path of gr_read: the remainder crosses the window, or the escape code.
__device__ __forceinline__ uint32_t gr_read_slow(WinReader &r, uint32_t k, uint32_t p, bool &bad)
{
    if (p < (uint32_t)kUnaryEsc) {
        r.skip(p + 1u);
        const uint32_t v = (p << k) | (r.peek() & ((1u << k) - 1u));
        r.skip(k);
        return v;
    }
    r.skip(kUnaryEsc);  // 24 ones, a 6-bit length n, n bits of value
    const uint32_t n = r.peek() & 63u;
    r.skip(6);
    if (n > 32u) {
        bad = true;
        return 0;
    }
    const uint32_t y = r.peek();
    const uint32_t v = n == 32u ? y : (y & ((1u << n) - 1u));
    r.skip(n);
    return v;
}

// Golomb-Rice value with parameter k (<= 24): p ones and a zero, then k low
// bits; p >= 24 is the escape (24 ones, a 6-bit length n, n bits of value).
__device__ __forceinline__ uint32_t gr_read(WinReader &r, uint32_t k, int &KR, bool &bad)
{
    const uint32_t x = r.peek();
    uint32_t p = (uint32_t)__ffs(~x) - 1u;  // leading ones (all ones: wraps to >= 32)
    const uint32_t n = p + 1u + k;
    uint32_t v;
    if (__builtin_expect(p < (uint32_t)kUnaryEsc && n <= 32u, 1)) {  // prefix and remainder inside the window
        v = (p << k) | ((x >> (p + 1u)) & ((1u << k) - 1u));
        r.skip(n);
    } else {
        v = gr_read_slow(r, k, p, bad);
        p = v >> k;
    }
    adapt_kr(p, KR);
    return v;
}

// Decodes one block stream (len coefficients of one channel) to out[i * C],
// i < len: dequantised (times sc) or as indices.  Runs are kept as pending
// zeros (and the nonzero that ends a partial run as a pending value), so a
// lane writes one or two rows per iteration: a lane that ends an iteration in
// Golomb-Rice mode decodes a second symbol in the same iteration (fewer loop
// and mode tests per symbol).
template <bool TO_INT>
__device__ __forceinline__ void decode_stream(const uint32_t *wp, uint32_t nw, uint32_t len, uint32_t C, float sc,
                                              float *yout, int32_t *qout, DevState *st)
{
    WinReader r;
    r.init(wp, nw);
    int K = 0, KR = 32;
    uint32_t zeros = 0;
    bool has_pending = false, bad = false;
    int32_t pending = 0;
    for (uint32_t i = 0; i < len; ++i) {
        int32_t q = 0;
        const uint32_t k = (uint32_t)K >> 4;
        if (__builtin_expect(!(zeros | (uint32_t)has_pending | k), 1)) {  // the common case: Golomb-Rice mode
            const uint32_t u = gr_read(r, (uint32_t)KR >> 4, KR, bad);
            q = unzz(u);
            K = u == 0 ? K + 3 : (K >= 3 ? K - 3 : 0);  // Golomb-Rice mode runs while K < 16: no cap at 240
        } else if (zeros) {
            --zeros;
        } else if (has_pending) {
            q = pending;
            has_pending = false;
        } else {
            const uint32_t x = r.peek();
            if (!(x & 1u)) {  // a full run of 2^k zeros (clamped at the block end)
                r.skip(1);
                const uint32_t run = 1u << k;
                zeros = (run < len - i ? run : len - i) - 1;
                K += 4;
                if (K > 240) K = 240;
            } else {  // r < 2^k zeros, then a nonzero
                const uint32_t rr = (x >> 1) & ((1u << k) - 1u);
                r.skip(1u + k);
                const uint32_t v = gr_read(r, (uint32_t)KR >> 4, KR, bad);
                if (rr >= len - i || v == 0xFFFFFFFFu) bad = true;
                K = K >= 6 ? K - 6 : 0;
                if (rr == 0) {
                    q = unzz(v + 1u);
                } else {
                    zeros = rr - 1;
                    pending = unzz(v + 1u);
                    has_pending = true;
                }
            }
        }
        if (TO_INT) {
            *qout = q;
            qout += C;
        } else {
            *yout = __fmul_rn((float)q, sc);
            yout += C;
        }
        if (i + 1 < len && !(zeros | (uint32_t)has_pending | ((uint32_t)K >> 4))) {  // a second GR-mode symbol
            const uint32_t u = gr_read(r, (uint32_t)KR >> 4, KR, bad);
            const int32_t q2 = unzz(u);
            K = u == 0 ? K + 3 : (K >= 3 ? K - 3 : 0);
            ++i;
            if (TO_INT) {
                *qout = q2;
                qout += C;
            } else {
                *yout = __fmul_rn((float)q2, sc);
                yout += C;
            }
        }
    }
    if (bad || r.overrun()) set_error(&st->err, kErrCorrupt);
}

// One frame: thread (local row block jl, channel c) of CTA x decodes block
// b = x * rb + jl of channel c.  Streams at block_off[b*C+c] (words) when
// block_off is given, else at (b*C+c) * stride.
template <bool TO_INT>
__global__ void __launch_bounds__(512, 4) rlgr_decode_kernel(const uint32_t *payload, uint64_t payload_words,
                                                          const uint32_t *block_words, const uint64_t *block_off,
                                                          uint32_t stride, uint32_t nv, uint32_t C, uint32_t B,
                                                          uint32_t rb, const float *step, float *Y, int32_t *qout,
                                                          DevState *st)
{
    const uint32_t jl = threadIdx.x / C;
    if (jl >= rb) return;
    const uint32_t c = threadIdx.x - jl * C;
    const uint64_t b = (uint64_t)blockIdx.x * rb + jl;
    const uint64_t row0 = b * B;
    if (row0 >= nv) return;
    const uint32_t len = (nv - row0) < B ? (uint32_t)(nv - row0) : B;
    const uint64_t blk = b * C + c;
    const uint64_t off = block_off ? block_off[blk] : blk * stride;
    uint32_t nw = block_words[blk];
    if (off + nw > payload_words) {
        set_error(&st->err, kErrCorrupt);
        nw = 0;
    }
    decode_stream<TO_INT>(payload + off, nw, len, C, TO_INT ? 0.f : step[c], TO_INT ? nullptr : Y + row0 * C + c,
                          TO_INT ? qout + row0 * C + c : nullptr, st);
}

// All frames of a batch: row blocks numbered across frames (job_off), rb per CTA.
__global__ void __launch_bounds__(512, 4) rlgr_decode_batch_kernel(const DecFrame *fr, uint32_t F,
                                                                const uint64_t *job_off, const uint32_t *bw_all,
                                                                const uint64_t *boff_all, const float *steps_all,
                                                                uint32_t C, uint32_t rb, float *Y, DevState *st)
{
    const uint32_t jl = threadIdx.x / C;
    if (jl >= rb) return;
    const uint32_t c = threadIdx.x - jl * C;
    const uint64_t job = (uint64_t)blockIdx.x * rb + jl;
    if (job >= job_off[F]) return;
    uint32_t lo = 0, hi = F;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (job_off[mid] <= job) lo = mid; else hi = mid;
    }
    const DecFrame &d = fr[lo];
    const uint32_t b = (uint32_t)(job - job_off[lo]);
    const uint32_t row0 = b * d.B;
    const uint32_t len = (d.nv - row0) < d.B ? (d.nv - row0) : d.B;
    const uint64_t base = boff_all[d.blk_off];
    const uint64_t blk = d.blk_off + (uint64_t)b * C + c;
    const uint64_t off = boff_all[blk] - base;
    uint32_t nw = bw_all[blk];
    if (off + nw > d.payload_words) {
        set_error(&st->err, kErrCorrupt);
        nw = 0;
    }
    decode_stream<false>(d.payload + off, nw, len, C, steps_all[(uint64_t)lo * C + c],
                         Y + ((uint64_t)d.vstart + row0) * C + c, nullptr, st);
}

__global__ void job_offsets_kernel(const uint32_t *vstart, uint32_t F, uint32_t B, uint32_t R, uint32_t C,
                                   uint64_t *job_off, uint64_t *blk_off)
{
    if (threadIdx.x != 0) return;
    uint64_t jo = 0, bo = 0;
    for (uint32_t f = 0; f < F; ++f) {
        job_off[f] = jo;
        blk_off[f] = bo;
        uint64_t nb = ((uint64_t)(vstart[f + 1] - vstart[f]) + B - 1) / B;
        jo += nb;
        bo += nb * R * C;
    }
    job_off[F] = jo;
    blk_off[F] = bo;
}

}  // namespace

// A slot holds 16 bits per coefficient on average (ample for quantised
// attribute coefficients); the worst case is 78 bits per coefficient.
uint32_t rlgr_slot_words(uint32_t B, bool worst_case)
{
    return worst_case ? (uint32_t)(((uint64_t)78 * B + 31) / 32 + 2) : (uint32_t)(B / 2 + 4);
}

void launch_rlgr_offsets(const uint32_t *vstart, uint32_t F, uint32_t B, uint32_t R, uint32_t C, uint64_t *job_off,
                         uint64_t *blk_off, cudaStream_t s)
{
    job_offsets_kernel<<<1, 32, 0, s>>>(vstart, F, B, R, C, job_off, blk_off);
    count_launch();
}

void launch_rlgr_encode(const RlgrJob &j, const uint64_t *job_off, uint64_t jobs_bound, cudaStream_t s)
{
    if (jobs_bound == 0 || j.C == 0) return;
    EncJobs E{j, job_off};
    const uint32_t rb = row_blocks_per_cta(j.R * j.C);
    const uint32_t threads = (rb * j.R * j.C + 31) / 32 * 32;
    if (j.sq_err)
        rlgr_encode_kernel<false, true><<<(uint32_t)((jobs_bound + rb - 1) / rb), threads, 0, s>>>(E, nullptr, rb);
    else
        rlgr_encode_kernel<false, false><<<(uint32_t)((jobs_bound + rb - 1) / rb), threads, 0, s>>>(E, nullptr, rb);
    count_launch();
}

void launch_rlgr_encode_indices(const int32_t *q, const uint32_t *vstart, uint32_t C, uint32_t B, uint32_t *slots,
                                uint32_t slot_words, uint32_t *bw, const uint64_t *job_off, const uint64_t *blk_off,
                                uint64_t jobs_bound, uint32_t *overflow, cudaStream_t s)
{
    if (jobs_bound == 0 || C == 0) return;
    RlgrJob j{};
    j.C = C;
    j.B = B;
    j.R = 1;
    j.vstart = vstart;
    j.F = 1;
    j.slots = slots;
    j.block_words = bw;
    j.blk_off = blk_off;
    j.slot_words = slot_words;
    j.overflow = overflow;
    EncJobs E{j, job_off};
    const uint32_t rb = row_blocks_per_cta(C);
    const uint32_t threads = (rb * C + 31) / 32 * 32;
    rlgr_encode_kernel<true, false><<<(uint32_t)((jobs_bound + rb - 1) / rb), threads, 0, s>>>(E, q, rb);
    count_launch();
}

void launch_rlgr_decode(const uint32_t *payload, uint64_t payload_words, const uint32_t *block_words,
                        const uint64_t *block_off, uint64_t nv, uint32_t C, uint32_t B, const float *step, float *Y,
                        DevState *st, cudaStream_t s)
{
    if (nv == 0 || C == 0) return;
    const uint64_t nb = (nv + B - 1) / B;
    const uint32_t rb = row_blocks_per_cta(C);
    // Streams are read in place: staging them in shared memory would cap the
    // number of resident threads, and this sequential decoder needs them all.
    rlgr_decode_kernel<false><<<(uint32_t)((nb + rb - 1) / rb), rb * C, 0, s>>>(
        payload, payload_words, block_words, block_off, 0u, (uint32_t)nv, C, B, rb, step, Y, nullptr, st);
    count_launch();
}

void launch_rlgr_decode_batch(const DecFrame *fr, uint32_t F, const uint64_t *job_off, uint64_t jobs_bound,
                              const uint32_t *bw_all, const uint64_t *boff_all, const float *steps_all, uint32_t C,
                              float *Y, DevState *st, cudaStream_t s)
{
    if (jobs_bound == 0 || C == 0) return;
    const uint32_t rb = row_blocks_per_cta(C);
    rlgr_decode_batch_kernel<<<(uint32_t)((jobs_bound + rb - 1) / rb), rb * C, 0, s>>>(
        fr, F, job_off, bw_all, boff_all, steps_all, C, rb, Y, st);
    count_launch();
}

void launch_rlgr_decode_indices(const uint32_t *words, uint64_t total_words, const uint32_t *bw, uint32_t stride,
                                uint64_t nv, uint32_t C, uint32_t B, int32_t *q, DevState *st, cudaStream_t s)
{
    if (nv == 0 || C == 0) return;
    const uint64_t nb = (nv + B - 1) / B;
    const uint32_t rb = row_blocks_per_cta(C);
    rlgr_decode_kernel<true><<<(uint32_t)((nb + rb - 1) / rb), rb * C, 0, s>>>(
        words, total_words, bw, nullptr, stride, (uint32_t)nv, C, B, rb, nullptr, nullptr, q, st);
    count_launch();
}

}  // namespace gsnfs
