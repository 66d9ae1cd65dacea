// RAHT prelude and transform (Sec. 3.1 Eq. 1, Sec. 3.2-3.3, App. D,
// Algorithms 4-6).
//
// Schedule from gap levels.  For ascending distinct codes, gap i (between
// voxels i-1 and i) has level g_i = msb(m_{i-1} xor m_i) + 1: the binary
// level at which the two voxels' branches merge.  Every gap is exactly one
// butterfly of Algorithm 6: its high pass lands at i1 = i, its low pass at
// i0 = the nearest gap to the left with a larger level (the start of the
// merged node), and the weights are run lengths w0 = i - i0, w1 = e - i with
// e the nearest larger gap to the right.  This is the level list of
// Algorithm 4 without materialising I_l / F_l for all 3J levels.
//
// Tiles instead of one launch per level.  The voxel sequence is cut into
// tiles of T elements.  A gap whose enclosing node lies inside its tile is
// processed in shared memory (all its descendants are in the tile too); the
// tile's maximal subtrees ("survivors") carry their low-pass rows to the
// next pass, which runs the same tile procedure on the survivor sequence
// (gap levels between survivors are the original gaps at their starts,
// weights are differences of original positions).  Passes shrink the
// sequence by a factor of ~T/(survivors per tile); the first three passes
// run grid-wide, the remainder inside one CTA.  A survivor bounded by frame
// boundaries on both sides is a frame's DC and is written in place.
// In-tile butterflies are ordered by level, so each level is one round
// between barriers.  The inverse runs the passes top-down with the rounds
// reversed and the transposed rotation.
#include <type_traits>

#include "kernels.cuh"

namespace gsnfs {

namespace {

constexpr int kThreads = 256;   // prelude kernels
constexpr int kXThreads = 512;  // transform kernels: 16 warps per tile, 3 tiles per SM
constexpr int kRounds = 64;  // gap levels of in-tile butterflies are below kRounds (a 64-bit level mask)
constexpr uint32_t kSmemRowBytes = 56 * 1024;

// ------------------------------------------------------------- prelude ---
struct PreludeArgs {
    RahtPlanDev p;
    const uint8_t *gap0;  // gap levels of pass 0 (voxel sequence)
    const DevState *st;
};

__device__ __forceinline__ uint32_t seq_pos(const RahtPlanDev &p, const RahtPass &ps, int q, uint64_t j)
{
    return q == 0 ? (p.pos0 ? p.pos0[j] : (uint32_t)j) : p.pos[ps.seq_off + j];
}

__device__ __forceinline__ uint8_t seq_gap(const PreludeArgs &a, const RahtPass &ps, int q, uint64_t j)
{
    return q == 0 ? a.gap0[j] : a.p.gapseq[ps.seq_off + j];
}

// one past the last voxel covered by element j (its subtree is contiguous)
__device__ __forceinline__ uint32_t seq_end(const RahtPlanDev &p, const RahtPass &ps, int q, uint64_t j)
{
    return q == 0 ? (p.end0 ? p.end0[j] : (uint32_t)(j + 1)) : p.endseq[ps.seq_off + j];
}

constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

template <int TMAX>
struct PreludeSmem {
    static constexpr int kWords = (TMAX + 1 + 31) / 32;  // bit words covering positions 0..T
    static constexpr int kLog = ilog2(TMAX) + 1;          // range-maximum levels 0 .. log2(TMAX)
    uint8_t g[TMAX + 1];
    uint8_t mx[kLog][TMAX + 1];  // mx[k][x] = max g[x .. x + 2^k) (k >= 1; level 0 is g)
    uint8_t inl[TMAX];        // gap i is processed inside the tile
    uint32_t p[TMAX + 1];
    uint32_t e[TMAX];
    uint16_t prv[TMAX];
    uint16_t nxt[TMAX];
    uint32_t surv[kWords];    // survivors (start a maximal in-tile subtree)
    uint32_t carry[kWords];   // survivors carried to the next pass
    uint32_t cpre[kWords];    // exclusive prefix of carry popcounts
    uint32_t lvl_cnt[kRounds + 1];
    uint32_t lvl_off[kRounds + 1];
    uint32_t scan[33];
};

// lowest set bit of mask at a position in (i, lim], or -1
__device__ __forceinline__ int next_set(const uint32_t *mask, uint32_t i, uint32_t lim)
{
    const uint32_t j = i + 1;
    int w = (int)(j >> 5);
    const int wl = (int)(lim >> 5);
    uint32_t b = mask[w] & (~0u << (j & 31));
    while (!b) {
        if (++w > wl) return -1;
        b = mask[w];
    }
    const int r = w * 32 + __ffs(b) - 1;
    return r <= (int)lim ? r : -1;
}

// The threads that build one tile's schedule: a whole CTA (barriers between
// phases) or, for tiles of at most 256 elements, one warp (each warp of a CTA
// its own tile and its own shared-memory slice, so no phase waits on the
// CTA's other warps).
struct CtaGroup {
    uint32_t rank, wid;
    static constexpr uint32_t size = kThreads, nwarps = kThreads / 32;
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct WarpGroup {
    uint32_t rank, wid;  // wid = 0
    static constexpr uint32_t size = 32, nwarps = 1;
    __device__ __forceinline__ void sync() const { __syncwarp(); }
};

// Builds the schedule of tile t of pass q (one thread group).
template <int TMAX, class Grp>
__device__ void prelude_tile(const PreludeArgs &a, PreludeSmem<TMAX> &S, int q, const RahtPass &ps, uint32_t t,
                             const Grp &G)
{
    const RahtPlanDev &p = a.p;
    const uint32_t T = p.T;
    const uint64_t j0 = (uint64_t)t * T;
    const uint32_t m = (uint32_t)((ps.n - j0) < T ? (ps.n - j0) : T);
    const uint32_t tid = G.rank, lane = threadIdx.x & 31, wid = G.wid;
    const uint32_t W = (m + 1 + 31) / 32;  // words covering positions 0..m
    for (uint32_t i = tid; i <= m; i += Grp::size) {
        S.g[i] = seq_gap(a, ps, q, j0 + i);
        S.p[i] = seq_pos(p, ps, q, j0 + i);
        if (i < m) S.e[i] = seq_end(p, ps, q, j0 + i);
    }
    for (int i = (int)tid; i <= kRounds; i += Grp::size) S.lvl_cnt[i] = 0;
    G.sync();
    // range maxima of the gap levels over power-of-two windows
    constexpr int K = PreludeSmem<TMAX>::kLog;
    for (int k = 1; k < K; ++k) {
        const uint32_t half = 1u << (k - 1), span = 1u << k;
        const uint8_t *src = (k == 1) ? S.g : S.mx[k - 1];
        for (uint32_t x = tid; x + span <= m + 1; x += Grp::size) {
            const uint8_t u = src[x], v = src[x + half];
            S.mx[k][x] = u > v ? u : v;
        }
        G.sync();
    }
    // nearest larger gap on each side (the tile's boundary gaps g[0], g[m]
    // count), by binary lifting over the range maxima
    for (uint32_t i = tid; i < m; i += Grp::size) {
        uint8_t f = 0;
        if (i > 0) {
            const uint32_t gi = S.g[i];  // < kInfLevel whenever a larger gap exists
            if (gi < (uint32_t)kRounds) {
                uint32_t lp = i;  // [lp, i) holds no larger gap
                for (int k = K - 1; k >= 0; --k) {
                    const uint32_t st = 1u << k;
                    if (lp >= st && (k ? S.mx[k][lp - st] : S.g[lp - st]) <= gi) lp -= st;
                }
                uint32_t rp = i + 1;  // (i, rp) holds no larger gap
                for (int k = K - 1; k >= 0; --k) {
                    const uint32_t st = 1u << k;
                    if (rp + st <= m + 1 && (k ? S.mx[k][rp] : S.g[rp]) <= gi) rp += st;
                }
                if (lp > 0 && rp <= m) {
                    f = 1;
                    S.prv[i] = (uint16_t)(lp - 1);
                    S.nxt[i] = (uint16_t)rp;
                    atomicAdd(&S.lvl_cnt[gi], 1u);
                }
            }
        }
        S.inl[i] = f;
    }
    G.sync();
    // survivor mask; level offsets of the butterflies (one warp)
    for (uint32_t w = wid; w < W; w += Grp::nwarps) {
        const uint32_t i = w * 32 + lane;
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, i < m && !S.inl[i]);
        if (lane == 0) S.surv[w] = b;
    }
    if (wid == 0) {
        uint32_t run = 0;
        for (int base = 0; base <= kRounds; base += 32) {
            const int l = base + lane;
            const uint32_t c = (l <= kRounds) ? S.lvl_cnt[l] : 0u;
            const uint32_t inc = warp_inclusive_sum(c);
            if (l <= kRounds) S.lvl_off[l] = run + inc - c;
            run += __shfl_sync(0xFFFFFFFFu, inc, 31);
        }
    }
    G.sync();
    // Rounds as early as possible (the range-maximum table is dead now and holds the scratch): a
    // butterfly's round is one more than the later of its two children's, so the butterflies are walked
    // level by level (children before parents) keeping, per node start, the round that completed it.
    // Butterflies of one level touch disjoint nodes; the arithmetic of each is unchanged, so the
    // coefficients do not depend on the order.
    static_assert((PreludeSmem<TMAX>::kLog - 1) * (TMAX + 1) >= 4 * TMAX + 1, "round scratch exceeds the table");
    uint16_t *ord = reinterpret_cast<uint16_t *>(&S.mx[1][0]);   // butterflies in level order (mx[0] is unused;
                                                                 // mx[1] starts at an even offset)
    uint8_t *dep = reinterpret_cast<uint8_t *>(ord + TMAX);       // round of the butterfly at element i
    uint8_t *dnode = dep + TMAX;                                 // round that completed the node starting at x
    for (int l = (int)tid; l <= kRounds; l += Grp::size) S.lvl_cnt[l] = 0;  // fill counters
    for (uint32_t x = tid; x <= m; x += Grp::size) dnode[x] = 0;
    G.sync();
    for (uint32_t i = tid; i < m; i += Grp::size)
        if (S.inl[i]) ord[S.lvl_off[S.g[i]] + atomicAdd(&S.lvl_cnt[S.g[i]], 1u)] = (uint16_t)i;
    G.sync();
    // the nonempty levels (butterflies have levels below kRounds = 64), lowest first
    uint64_t levels = (uint64_t)__ballot_sync(0xFFFFFFFFu, S.lvl_cnt[lane] != 0) |
                      ((uint64_t)__ballot_sync(0xFFFFFFFFu, S.lvl_cnt[lane + 32] != 0) << 32);
    for (; levels; levels &= levels - 1) {
        const int l = __ffsll((long long)levels) - 1;
        const uint32_t cnt = S.lvl_cnt[l];
        const uint32_t off = S.lvl_off[l];
        for (uint32_t k = tid; k < cnt; k += Grp::size) {
            const uint32_t i = ord[off + k], lft = S.prv[i];
            const uint32_t d = 1u + (dnode[lft] > dnode[i] ? dnode[lft] : dnode[i]);
            dep[i] = (uint8_t)d;
            dnode[lft] = (uint8_t)d;
        }
        G.sync();
    }
    for (int l = (int)tid; l <= kRounds; l += Grp::size) S.lvl_cnt[l] = 0;  // butterflies per round
    G.sync();
    for (uint32_t i = tid; i < m; i += Grp::size)
        if (S.inl[i]) atomicAdd(&S.lvl_cnt[dep[i]], 1u);
    G.sync();
    if (wid == 0) {  // round offsets and ends (rounds 1 .. nr are all nonempty)
        uint32_t run = 0, nr = 0;
        uint16_t *re = p.round_end + (uint64_t)(ps.tile_off + t) * kRounds;
        for (int base = 1; base <= kRounds; base += 32) {
            const int l = base + lane;
            const uint32_t c = (l <= kRounds) ? S.lvl_cnt[l] : 0u;
            const uint32_t inc = warp_inclusive_sum(c);
            if (l <= kRounds) S.lvl_off[l] = run + inc - c;
            if (c) re[l - 1] = (uint16_t)(run + inc);
            nr += __popc(__ballot_sync(0xFFFFFFFFu, c != 0));
            run += __shfl_sync(0xFFFFFFFFu, inc, 31);
        }
        if (lane == 0) {
            p.tile_nbf[ps.tile_off + t] = run;
            p.tile_nr[ps.tile_off + t] = nr;
        }
    }
    G.sync();
    for (int l = (int)tid; l <= kRounds; l += Grp::size) S.lvl_cnt[l] = 0;  // reused as fill counters
    G.sync();
    // butterflies, destinations, frame roots; carried survivors marked in S.inl (2)
    const uint64_t sbase = (uint64_t)(ps.tile_off + t) * T;
    for (uint32_t i = tid; i < m; i += Grp::size) {
        if (S.inl[i]) {
            // children cover elements [l, i) and [i, r); neither range crosses a frame
            // boundary, so their voxels are contiguous.  The right end is taken from
            // the last element's own end: a frame finished in an earlier pass may have
            // been dropped between this frame and the element at r.
            const uint32_t l = S.prv[i], r = S.nxt[i];
            const uint32_t w0 = S.p[i] - S.p[l], w1 = S.e[r - 1] - S.p[i];
            const float fw0 = (float)w0, fw1 = (float)w1, fs = (float)(w0 + w1);
            const float ca = __fsqrt_rn(__fdiv_rn(fw0, fs)), cb = __fsqrt_rn(__fdiv_rn(fw1, fs));
            const uint32_t slot = S.lvl_off[dep[i]] + atomicAdd(&S.lvl_cnt[dep[i]], 1u);
            p.bf_idx[sbase + slot] = l | (i << 16);
            p.bf_ab[sbase + slot] = make_float2(ca, cb);
            if (p.bf_w) p.bf_w[sbase + slot] = make_uint2(w0, w1);
            p.dest[ps.seq_off + j0 + i] = S.p[i];
        } else {
            // survivor: a frame root (final) iff both bounding gaps are frame boundaries
            int r = next_set(S.surv, i, m - 1);
            if (r < 0) r = (int)m;
            if (S.g[i] >= kInfLevel && S.g[r] >= kInfLevel) {
                p.dest[ps.seq_off + j0 + i] = S.p[i];
            } else {
                S.inl[i] = 2;
                p.send[ps.seq_off + j0 + i] = S.e[r - 1];  // the survivor's subtree ends with element r-1
            }
        }
    }
    G.sync();
    // local carried ranks: popcounts of the carried mask
    for (uint32_t w = wid; w < W; w += Grp::nwarps) {
        const uint32_t i = w * 32 + lane;
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, i < m && S.inl[i] == 2);
        if (lane == 0) S.carry[w] = b;
    }
    G.sync();
    if (wid == 0) {
        uint32_t run = 0;
        for (uint32_t base = 0; base < W; base += 32) {
            const uint32_t w = base + lane;
            const uint32_t c = (w < W) ? __popc(S.carry[w]) : 0u;
            const uint32_t inc = warp_inclusive_sum(c);
            if (w < W) S.cpre[w] = run + inc - c;
            run += __shfl_sync(0xFFFFFFFFu, inc, 31);
        }
        if (lane == 0) p.tile_carry[ps.tile_off + t] = run;
    }
    G.sync();
    for (uint32_t i = tid; i < m; i += Grp::size)
        if (S.inl[i] == 2) {
            const uint32_t w = i >> 5;
            const uint32_t rank = S.cpre[w] + __popc(S.carry[w] & ((1u << (i & 31)) - 1u));
            p.dest[ps.seq_off + j0 + i] = kCarry | rank;
            if (rank < kRahtCarrySlots) p.carry_list[(uint64_t)(ps.tile_off + t) * kRahtCarrySlots + rank] = (uint16_t)i;
        }
    G.sync();
}

__global__ void __launch_bounds__(kThreads) prelude_init_kernel(RahtPlanDev p, const DevState *st,
                                                                 const uint64_t *nv_override)
{
    if (threadIdx.x == 0) {
        uint32_t n = (uint32_t)(nv_override ? *nv_override : st->nv_total);
        RahtPass ps = {};
        ps.n = n;
        ps.ntiles = (n + p.T - 1) / p.T;
        p.passes[0] = ps;
        for (int q = 1; q <= kRahtMaxPasses; ++q) p.passes[q] = RahtPass{};
        *p.npasses = n ? 1u : 0u;
        p.pipe_ctr[0] = 0;
        p.pipe_ctr[1] = 0;
    }
}

// tiles of at most 256 elements: one warp per tile; larger tiles: one CTA per tile
template <int TMAX>
constexpr bool kWarpTiles = TMAX <= 256;

template <int TMAX>
constexpr size_t prelude_smem_bytes()
{
    return (kWarpTiles<TMAX> ? (size_t)(kThreads / 32) : (size_t)1) * sizeof(PreludeSmem<TMAX>);
}

template <int TMAX>
__global__ void __launch_bounds__(kThreads) prelude_tiles_kernel(PreludeArgs a, int q)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RahtPass ps = a.p.passes[q];
    if constexpr (kWarpTiles<TMAX>) {
        const uint32_t wid = threadIdx.x >> 5;
        PreludeSmem<TMAX> &S = reinterpret_cast<PreludeSmem<TMAX> *>(smem_raw)[wid];
        const WarpGroup G{threadIdx.x & 31u, 0u};
        const uint32_t nw = gridDim.x * (kThreads / 32);
        for (uint32_t t = blockIdx.x * (kThreads / 32) + wid; t < ps.ntiles; t += nw) prelude_tile(a, S, q, ps, t, G);
    } else {
        PreludeSmem<TMAX> &S = *reinterpret_cast<PreludeSmem<TMAX> *>(smem_raw);
        const CtaGroup G{threadIdx.x, threadIdx.x >> 5};
        for (uint32_t t = blockIdx.x; t < ps.ntiles; t += gridDim.x) prelude_tile(a, S, q, ps, t, G);
    }
}

// one CTA: exclusive scan of carried counts over the pass's tiles, next pass
__device__ void prelude_scan_body(const RahtPlanDev &p, int q, uint32_t *sh)
{
    const RahtPass ps = p.passes[q];
    // each thread sums a contiguous run of tiles (all its loads in flight together), one block scan of the
    // run totals, then each thread writes its run's prefixes
    const uint32_t per = (ps.ntiles + blockDim.x - 1) / blockDim.x;
    const uint32_t b = threadIdx.x * per < ps.ntiles ? threadIdx.x * per : ps.ntiles;
    const uint32_t e = b + per < ps.ntiles ? b + per : ps.ntiles;
    uint32_t *tc = p.tile_carry + ps.tile_off;
    uint32_t sum = 0;
    for (uint32_t t = b; t < e; ++t) sum += tc[t];
    uint32_t run;
    uint32_t pre = block_exclusive_sum<uint32_t>(sum, sh, &run);
    for (uint32_t t = b; t < e; ++t) {
        const uint32_t c = tc[t];
        tc[t] = pre;
        pre += c;
    }
    if (threadIdx.x == 0) {
        RahtPass nx = {};
        if (q + 1 < kRahtMaxPasses) {
            nx.n = run;
            nx.ntiles = (run + p.T - 1) / p.T;
            nx.seq_off = ps.seq_off + ps.n + 1;
            nx.tile_off = ps.tile_off + ps.ntiles;
            nx.surv_off = (q == 0) ? 0u : ps.surv_off + ps.n;
            p.passes[q + 1] = nx;
            if (run) *p.npasses = (uint32_t)(q + 2);
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024) prelude_scan_kernel(RahtPlanDev p, int q)
{
    __shared__ uint32_t sh[33];
    if (p.passes[q].n == 0) return;
    prelude_scan_body(p, q, sh);
}

// carried elements: global index, next sequence arrays, sentinel.  A warp
// per tile walks the tile's list of carried survivors (their global index is
// the tile's scanned base plus their rank), so elements that are not carried
// are never read.
__device__ void prelude_compact_body(const PreludeArgs &a, int q, uint32_t warp0, uint32_t nwarps)
{
    const RahtPlanDev &p = a.p;
    const RahtPass ps = p.passes[q];
    const RahtPass nx = p.passes[q + 1];
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t t = warp0; t < ps.ntiles; t += nwarps) {
        const uint32_t b0 = p.tile_carry[ps.tile_off + t];
        const uint32_t b1 = t + 1 < ps.ntiles ? p.tile_carry[ps.tile_off + t + 1] : nx.n;
        for (uint32_t r = lane; r < b1 - b0 && r < kRahtCarrySlots; r += 32) {
            const uint32_t i = p.carry_list[(uint64_t)(ps.tile_off + t) * kRahtCarrySlots + r];
            const uint64_t j = (uint64_t)t * p.T + i;
            const uint32_t gi = b0 + r;
            p.dest[ps.seq_off + j] = kCarry | gi;
            p.pos[nx.seq_off + gi] = seq_pos(p, ps, q, j);
            p.gapseq[nx.seq_off + gi] = seq_gap(a, ps, q, j);
            p.endseq[nx.seq_off + gi] = p.send[ps.seq_off + j];
        }
    }
    if (warp0 == 0 && lane == 0 && nx.n) {
        p.pos[nx.seq_off + nx.n] = seq_pos(p, ps, q, ps.n);
        p.gapseq[nx.seq_off + nx.n] = (uint8_t)kInfLevel;
    }
}

__global__ void __launch_bounds__(kThreads) prelude_compact_kernel(PreludeArgs a, int q)
{
    if (a.p.passes[q].n == 0 || q + 1 >= kRahtMaxPasses) return;
    prelude_compact_body(a, q, blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5), gridDim.x * (kThreads / 32));
}

// remaining passes inside one CTA
template <int TMAX>
__global__ void __launch_bounds__(kThreads) prelude_finish_kernel(PreludeArgs a, int q0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PreludeSmem<TMAX> *S = reinterpret_cast<PreludeSmem<TMAX> *>(smem_raw);
    for (int q = q0; q + 1 < kRahtMaxPasses; ++q) {
        const RahtPass ps = a.p.passes[q];
        if (ps.n == 0) break;
        if constexpr (kWarpTiles<TMAX>) {
            const uint32_t wid = threadIdx.x >> 5;
            const WarpGroup G{threadIdx.x & 31u, 0u};
            for (uint32_t t = wid; t < ps.ntiles; t += kThreads / 32) prelude_tile(a, S[wid], q, ps, t, G);
        } else {
            const CtaGroup G{threadIdx.x, threadIdx.x >> 5};
            for (uint32_t t = 0; t < ps.ntiles; ++t) prelude_tile(a, S[0], q, ps, t, G);
        }
        __syncthreads();
        prelude_scan_body(a.p, q, S[0].scan);
        __syncthreads();
        prelude_compact_body(a, q, threadIdx.x >> 5, kThreads / 32);
        __syncthreads();
    }
}

// ----------------------------------------------------------- transform ---
struct TileSched {
    uint32_t nbf, nr;
    uint16_t re[kRounds];
};

template <typename S, int VEC>
struct Vec;
template <>
struct Vec<float, 1> {
    typedef float T;
    __device__ static T ld(const float *p) { return *p; }
    __device__ static void st(float *p, T v) { *p = v; }
};
template <>
struct Vec<float, 4> {
    typedef float4 T;
    __device__ static T ld(const float *p) { return *reinterpret_cast<const float4 *>(p); }
    __device__ static void st(float *p, T v) { *reinterpret_cast<float4 *>(p) = v; }
};
template <>
struct Vec<double, 1> {
    typedef double T;
    __device__ static T ld(const double *p) { return *p; }
    __device__ static void st(double *p, T v) { *p = v; }
};
template <>
struct Vec<double, 2> {
    typedef double2 T;
    __device__ static T ld(const double *p) { return *reinterpret_cast<const double2 *>(p); }
    __device__ static void st(double *p, T v) { *reinterpret_cast<double2 *>(p) = v; }
};

__device__ __forceinline__ float add_rn(float x, float y) { return __fadd_rn(x, y); }
__device__ __forceinline__ double add_rn(double x, double y) { return __dadd_rn(x, y); }
__device__ __forceinline__ float div_rn(float x, float y) { return __fdiv_rn(x, y); }
__device__ __forceinline__ double div_rn(double x, double y) { return __ddiv_rn(x, y); }

// asynchronous global -> shared copy of N bytes (4, 8 or 16; both addresses N-aligned)
template <int N>
__device__ __forceinline__ void cp_async_vec(void *smem, const void *gmem)
{
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    if (N == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
    else if (N == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Eq. (1): forward (a*y0 + b*y1, a*y1 - b*y0); inverse (transposed) (a*y0 - b*y1, b*y0 + a*y1).
// FP32: one rounded product, then a fused multiply-add (every kernel uses this
// same sequence, so all FP32 paths agree bit for bit).  FP64: each product and
// sum rounds once (no contraction).
template <bool INV>
__device__ __forceinline__ void rot(float a, float b, float &y0, float &y1)
{
    const float u = y0, v = y1;
    if (!INV) {
        y0 = __fmaf_rn(a, u, __fmul_rn(b, v));
        y1 = __fmaf_rn(a, v, -__fmul_rn(b, u));
    } else {
        y0 = __fmaf_rn(a, u, -__fmul_rn(b, v));
        y1 = __fmaf_rn(b, u, __fmul_rn(a, v));
    }
}

template <bool INV>
__device__ __forceinline__ void rot(double a, double b, double &y0, double &y1)
{
    const double u = y0, v = y1;
    if (!INV) {
        y0 = __dadd_rn(__dmul_rn(a, u), __dmul_rn(b, v));
        y1 = __dsub_rn(__dmul_rn(a, v), __dmul_rn(b, u));
    } else {
        y0 = __dsub_rn(__dmul_rn(a, u), __dmul_rn(b, v));
        y1 = __dadd_rn(__dmul_rn(b, u), __dmul_rn(a, v));
    }
}

template <bool INV>
__device__ __forceinline__ void rot(float a, float b, float4 &y0, float4 &y1)
{
    rot<INV>(a, b, y0.x, y1.x);
    rot<INV>(a, b, y0.y, y1.y);
    rot<INV>(a, b, y0.z, y1.z);
    rot<INV>(a, b, y0.w, y1.w);
}

template <bool INV>
__device__ __forceinline__ void rot(double a, double b, double2 &y0, double2 &y1)
{
    rot<INV>(a, b, y0.x, y1.x);
    rot<INV>(a, b, y0.y, y1.y);
}

__device__ __forceinline__ float qdq(float y, float inv, float step, float tau)
{
    return __fmul_rn((float)quantize_f32(y, inv, tau), step);
}

// the same quantiser evaluated in FP64 (index bounded by 2^30 like the FP32 one)
__device__ __forceinline__ double qdq(double y, double inv, double step, double tau)
{
    double t = floor(__dadd_rn(__dmul_rn(fabs(y), inv), tau));
    t = fmin(t, 1073741824.0);
    return __dmul_rn(y < 0.0 ? -t : t, step);
}

__device__ __forceinline__ uint32_t frame_of_voxel(const uint32_t *vstart, uint32_t F, uint64_t j)
{
    uint32_t lo = 0, hi = F;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((uint64_t)vstart[mid] <= j) lo = mid; else hi = mid;
    }
    return lo;
}

template <typename S>
struct XformArgs {
    RahtPlanDev p;
    RahtIOT<S> io;
    uint32_t Cg;  // channels per group held in shared memory
};

// Shared-memory carve of the transform kernels (T = tile size).
template <typename S>
struct XformSmem {
    uint32_t *s_idx;   // T: butterfly i0 | i1 << 16
    S *s_ab;           // 2T: butterfly coefficients (a, b)
    uint32_t *s_src;   // T + 1: gather segment starts (forward pass 0) or row sources (inverse)
    uint32_t *s_dst;   // T: row destinations (forward)
    uint32_t *s_vals;  // 2T: point indices of the tile's gather
    uint8_t *s_frame;  // T: frame of each voxel (batched gather)
    S *rows;           // T x Cg
    float *klt_s;      // 3 x 15 x 15: the colour KLT of the tile's first frame
};

template <typename S>
__host__ __device__ inline size_t xform_meta_bytes(uint32_t T)
{
    return 2 * sizeof(S) * T + 4 * T + 4 * (T + 1) + 4 * T + 8 * T + T + 64;
}

template <typename S>
__device__ inline XformSmem<S> carve_xform(unsigned char *raw, uint32_t T, uint32_t Cg)
{
    XformSmem<S> X;
    X.s_ab = reinterpret_cast<S *>(raw);
    X.s_idx = reinterpret_cast<uint32_t *>(raw + 2 * sizeof(S) * T);
    X.s_src = X.s_idx + T;
    X.s_dst = X.s_src + T + 1;
    X.s_vals = X.s_dst + T;
    X.s_frame = reinterpret_cast<uint8_t *>(X.s_vals + 2 * T);
    X.rows = reinterpret_cast<S *>(raw + ((xform_meta_bytes<S>(T) + 15) & ~(size_t)15));
    X.klt_s = reinterpret_cast<float *>(raw + ((xform_meta_bytes<S>(T) + 15) & ~(size_t)15) +
                                        sizeof(S) * (size_t)T * Cg);
    return X;
}

// level of detail: element j of the coarse first pass is a node of w voxels; its low pass over sqrt(w) is
// the mean of its voxels (the same expression as a per-node division after the transform)
template <typename S>
__device__ __forceinline__ S lod_divisor(const RahtPlanDev &p, uint64_t j)
{
    return (S)__fsqrt_rn((float)(p.end0[j] - p.pos0[j]));
}

// butterfly k of a tile: FP32 coefficients come from the plan; FP64 ones are
// computed here from the integer weights, a = sqrt(w0/(w0+w1)), b = sqrt(w1/(w0+w1))
__device__ __forceinline__ void load_coeffs(const RahtPlanDev &p, uint64_t at, float *ab)
{
    const float2 c = p.bf_ab[at];
    ab[0] = c.x;
    ab[1] = c.y;
}

__device__ __forceinline__ void load_coeffs(const RahtPlanDev &p, uint64_t at, double *ab)
{
    const uint2 w = p.bf_w[at];
    const double s = (double)w.x + (double)w.y;
    ab[0] = __dsqrt_rn(__ddiv_rn((double)w.x, s));
    ab[1] = __dsqrt_rn(__ddiv_rn((double)w.y, s));
}

// Processes tile t of pass q for channel group [c0, c0 + Cg).
template <typename S, bool INV, int VEC, bool GATHER, bool QDQ>
__device__ void xform_tile(const XformArgs<S> &A, const XformSmem<S> &X, TileSched &sch, int q, const RahtPass &ps,
                           const RahtPass &nx, uint32_t t)
{
    typedef typename Vec<S, VEC>::T V;
    const RahtPlanDev &p = A.p;
    const RahtIOT<S> &io = A.io;
    const uint32_t T = p.T, C = io.C;
    const uint64_t j0 = (uint64_t)t * T;
    const uint32_t m = (uint32_t)((ps.n - j0) < T ? (ps.n - j0) : T);
    const int tid = threadIdx.x;
    const uint32_t tile = ps.tile_off + t;
    const bool gather = GATHER && q == 0;
    // ---- schedule and per-row metadata, coalesced into shared memory
    if (tid == 0) {
        sch.nbf = p.tile_nbf[tile];
        sch.nr = p.tile_nr[tile];
    }
    for (uint32_t i = tid; i < m; i += kXThreads) {
        const uint32_t d = p.dest[ps.seq_off + j0 + i];
        if (INV) X.s_src[i] = d; else X.s_dst[i] = d;
        if (gather) {
            X.s_src[i] = io.seg[j0 + i];
            if (io.frame_shift < 64) X.s_frame[i] = (uint8_t)(io.codes[j0 + i] >> io.frame_shift);
        }
    }
    if (gather && tid == 0) X.s_src[m] = io.seg[j0 + m];
    __syncthreads();
    // colour mode: the KLT of the tile's first frame, staged for the per-row transforms
    uint32_t kfr = 0xFFFFFFFFu;
    if constexpr (std::is_same<S, float>::value) {
        if (io.klt && ((!INV && gather) || (INV && q == 0))) {
            kfr = INV ? frame_of_voxel(io.vstart, io.F, j0) : (io.frame_shift < 64 ? X.s_frame[0] : 0u);
            for (uint32_t k = tid; k < (uint32_t)kKltFloats; k += kXThreads)
                X.klt_s[k] = io.klt[(uint64_t)kfr * kKltFloats + k];
        }
    }
    for (uint32_t r = tid; r < sch.nr; r += kXThreads) sch.re[r] = p.round_end[(uint64_t)tile * kRounds + r];
    for (uint32_t k = tid; k < sch.nbf; k += kXThreads) {
        X.s_idx[k] = p.bf_idx[(uint64_t)tile * T + k];
        load_coeffs(p, (uint64_t)tile * T + k, X.s_ab + 2 * k);
    }
    uint32_t g0 = 0;
    bool staged = false;
    if (gather) {
        g0 = X.s_src[0];
        const uint32_t gcount = X.s_src[m] - g0;
        staged = gcount <= 2 * T;
        if (staged)
            for (uint32_t k = tid; k < gcount; k += kXThreads) X.s_vals[k] = io.vals[g0 + k];
        __syncthreads();
    }
    for (uint32_t c0 = 0; c0 < C; c0 += A.Cg) {
        const uint32_t Cg = (C - c0) < A.Cg ? (C - c0) : A.Cg;
        const uint32_t L = Cg / VEC;           // vector lanes per row
        const uint32_t slots = kXThreads / L;   // rows processed per sweep
        const uint32_t slot = tid / L, lane = tid - slot * L;
        const uint32_t c = c0 + lane * VEC;
        const bool act = slot < slots;
        // ---- load rows: every element of the tile is copied by an asynchronous
        // copy (no registers held, all of them in flight at once); the thread
        // that copied an element then finishes it in place: the average of a
        // voxel holding several points (forward gather) or the quantise ->
        // dequantise of a coefficient (inverse with QDQ)
        if (act) {
            for (uint32_t i = slot; i < m; i += slots) {
                const uint64_t j = j0 + i;
                const S *src;
                if (!INV) {
                    if (gather) {
                        const uint32_t s0 = X.s_src[i];
                        const uint32_t row = staged ? X.s_vals[s0 - g0] : io.vals[s0];
                        src = io.attr[io.frame_shift < 64 ? X.s_frame[i] : 0] + (uint64_t)row * C + c;
                    } else if (q == 0) {
                        src = io.in + j * C + c;
                    } else {
                        src = io.pool + ((uint64_t)ps.surv_off + j) * C + c;
                    }
                } else {
                    const uint32_t d = X.s_src[i];
                    src = (d & kCarry) ? io.pool + ((uint64_t)nx.surv_off + (d & ~kCarry)) * C + c
                                       : io.Y + (uint64_t)d * C + c;
                }
                cp_async_vec<sizeof(V)>(X.rows + (uint64_t)i * Cg + lane * VEC, src);
            }
        }
        cp_async_commit_wait_all();
        if (act && ((GATHER && gather) || QDQ)) {
            for (uint32_t i = slot; i < m; i += slots) {
                S *pr = X.rows + (uint64_t)i * Cg + lane * VEC;
                if (!INV) {
                    const uint32_t s0 = X.s_src[i], s1 = X.s_src[i + 1];
                    const uint32_t fr = io.frame_shift < 64 ? X.s_frame[i] : 0u;
                    bool ctr_any = io.center != nullptr;
                    if constexpr (std::is_same<S, float>::value) ctr_any = ctr_any && !io.klt;
                    if (s1 - s0 > 1 || ctr_any) {
                        V acc = Vec<S, VEC>::ld(pr);
                        S *pa = reinterpret_cast<S *>(&acc);
                        if (s1 - s0 > 1) {  // voxels holding several points: average in input order
                            const S *base = io.attr[fr];
                            for (uint32_t g = s0 + 1; g < s1; ++g) {
                                const uint32_t row = staged ? X.s_vals[g - g0] : io.vals[g];
                                V xv = Vec<S, VEC>::ld(base + (uint64_t)row * C + c);
                                const S *px = reinterpret_cast<const S *>(&xv);
#pragma unroll
                                for (int e = 0; e < VEC; ++e) pa[e] = add_rn(pa[e], px[e]);
                            }
                            const S cnt = (S)(s1 - s0);
#pragma unroll
                            for (int e = 0; e < VEC; ++e) pa[e] = div_rn(pa[e], cnt);
                        }
                        if (ctr_any) {  // centred rows keep the low-pass sums small (FP32 accuracy)
                            const S *ctr = io.center + (uint64_t)fr * C + c;
#pragma unroll
                            for (int e = 0; e < VEC; ++e) pa[e] = add_rn(pa[e], -ctr[e]);
                        }
                        Vec<S, VEC>::st(pr, acc);
                    }
                } else if (QDQ && !(X.s_src[i] & kCarry)) {
                    V v = Vec<S, VEC>::ld(pr);
                    S *pv = reinterpret_cast<S *>(&v);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) pv[e] = qdq(pv[e], io.inv_step[c + e], io.step[c + e], io.tau);
                    Vec<S, VEC>::st(pr, v);
                }
            }
        }
        if constexpr (std::is_same<S, float>::value) {
            if (!INV && gather && io.klt) {  // colour decorrelation of whole rows (Cg == C), then centring
                __syncthreads();
                for (uint32_t e = tid; e < m * 16; e += kXThreads)  // YUV per (row, SH function)
                    color_yuv_task(X.rows + (uint64_t)(e >> 4) * Cg, (int)(e & 15), kYuvFwd);
                __syncthreads();
                for (uint32_t e = tid; e < m * 3; e += kXThreads) {  // KLT per (row, YUV channel)
                    const uint32_t i = e / 3, ch = e - 3 * i;
                    const uint32_t fr = io.frame_shift < 64 ? X.s_frame[i] : 0u;
                    const float *K = (fr == kfr ? X.klt_s : io.klt + (uint64_t)fr * kKltFloats) + ch * kKltN * kKltN;
                    color_klt_task<false>(X.rows + (uint64_t)i * Cg, (int)ch, K);
                }
                if (io.center) {
                    __syncthreads();
                    for (uint32_t e = tid; e < m * C; e += kXThreads) {
                        const uint32_t i = e / C, cc = e - i * C;
                        const uint32_t fr = io.frame_shift < 64 ? X.s_frame[i] : 0u;
                        X.rows[(uint64_t)i * Cg + cc] = __fadd_rn(X.rows[(uint64_t)i * Cg + cc],
                                                                  -io.center[(uint64_t)fr * C + cc]);
                    }
                }
            }
        }
        __syncthreads();
        // ---- rounds
        for (uint32_t rr = 0; rr < sch.nr; ++rr) {
            const uint32_t r = INV ? (sch.nr - 1 - rr) : rr;
            const uint32_t kb = r ? sch.re[r - 1] : 0u, ke = sch.re[r];
            if (act) {
                for (uint32_t k = kb + slot; k < ke; k += slots) {
                    const uint32_t ix = X.s_idx[k];
                    const S a = X.s_ab[2 * k], b = X.s_ab[2 * k + 1];
                    S *r0 = X.rows + (uint64_t)(ix & 0xFFFFu) * Cg + lane * VEC;
                    S *r1 = X.rows + (uint64_t)(ix >> 16) * Cg + lane * VEC;
                    V y0 = Vec<S, VEC>::ld(r0), y1 = Vec<S, VEC>::ld(r1);
                    rot<INV>(a, b, y0, y1);
                    Vec<S, VEC>::st(r0, y0);
                    Vec<S, VEC>::st(r1, y1);
                }
            }
            __syncthreads();
        }
        if constexpr (std::is_same<S, float>::value) {
            if (INV && q == 0 && io.klt) {  // undo the colour decorrelation of whole rows (Cg == C)
                for (uint32_t e = tid; e < m * 3; e += kXThreads) {  // KLT^T per (row, YUV channel)
                    const uint32_t i = e / 3, ch = e - 3 * i;
                    const uint32_t fr = frame_of_voxel(io.vstart, io.F, j0 + i);
                    if (io.frame_color && !io.frame_color[fr]) continue;
                    const float *K = (fr == kfr ? X.klt_s : io.klt + (uint64_t)fr * kKltFloats) + ch * kKltN * kKltN;
                    color_klt_task<true>(X.rows + (uint64_t)i * Cg, (int)ch, K);
                }
                __syncthreads();
                for (uint32_t e = tid; e < m * 16; e += kXThreads) {  // inverse YUV per (row, SH function)
                    const uint32_t i = e >> 4;
                    const uint32_t fr = io.F > 1 ? frame_of_voxel(io.vstart, io.F, j0 + i) : 0u;
                    if (io.frame_color && !io.frame_color[fr]) continue;
                    color_yuv_task(X.rows + (uint64_t)i * Cg, (int)(e & 15), io.yuv_inv.m);
                }
                __syncthreads();
            }
        }
        // ---- store rows
        if (act) {
            for (uint32_t i = slot; i < m; i += slots) {
                const uint64_t j = j0 + i;
                V v = Vec<S, VEC>::ld(X.rows + (uint64_t)i * Cg + lane * VEC);
                if (!INV) {
                    const uint32_t d = X.s_dst[i];
                    if (d & kCarry)
                        Vec<S, VEC>::st(io.pool + ((uint64_t)nx.surv_off + (d & ~kCarry)) * C + c, v);
                    else
                        Vec<S, VEC>::st(io.Y + (uint64_t)d * C + c, v);
                } else {
                    if (q == 0 && io.lod_mean) {
                        S *pv = reinterpret_cast<S *>(&v);
                        const S dv = lod_divisor<S>(p, j);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) pv[e] = div_rn(pv[e], dv);
                    }
                    if (q == 0)
                        Vec<S, VEC>::st(io.out + j * C + c, v);
                    else
                        Vec<S, VEC>::st(io.pool + ((uint64_t)ps.surv_off + j) * C + c, v);
                }
            }
        }
        __syncthreads();
    }
}

template <typename S, bool INV, int VEC, bool GATHER, bool QDQ>
__global__ void __launch_bounds__(kXThreads, 3) xform_pass_kernel(XformArgs<S> A, int q)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ TileSched sch;
    const XformSmem<S> X = carve_xform<S>(smem_raw, A.p.T, A.Cg);
    const RahtPass ps = A.p.passes[q];
    const RahtPass nx = A.p.passes[q + 1];
    for (uint32_t t = blockIdx.x; t < ps.ntiles; t += gridDim.x)
        xform_tile<S, INV, VEC, GATHER, QDQ>(A, X, sch, q, ps, nx, t);
}

// passes q0 .. npasses-1 in one CTA (forward: ascending; inverse: descending)
template <typename S, bool INV, int VEC, bool QDQ>
__global__ void __launch_bounds__(kXThreads, 3) xform_finish_kernel(XformArgs<S> A, int q0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ TileSched sch;
    const XformSmem<S> X = carve_xform<S>(smem_raw, A.p.T, A.Cg);
    const int np = (int)*A.p.npasses;
    for (int k = 0; k < np - q0; ++k) {
        const int q = INV ? (np - 1 - k) : (q0 + k);
        const RahtPass ps = A.p.passes[q];
        const RahtPass nx = A.p.passes[q + 1];
        for (uint32_t t = 0; t < ps.ntiles; ++t)
            xform_tile<S, INV, VEC, false, QDQ>(A, X, sch, q, ps, nx, t);
        __threadfence_block();
        __syncthreads();
    }
}

// ---- software-pipelined first pass (FP32, whole rows in shared memory) -----
// A CTA walks its tiles (blockIdx.x + k * gridDim.x) with NR row buffers and
// NR + 1 metadata buffers, loads issued as cp.async groups ahead of use:
//   NR = 1 (three CTAs per SM): the metadata of tile k + 1 lands while tile k
//          is transformed; tile k + 1's rows are issued once tile k is stored;
//   NR = 3 (one CTA per SM): the rows of tiles k + 1 and k + 2 and the
//          metadata of tile k + 3 are in flight while tile k is transformed.
// Per tile the arithmetic is that of xform_tile, in the same order, so the
// results are bit-identical.

struct PipeStage {
    uint64_t *codes;  // T: voxel codes (frame id), forward gather of several frames
    float2 *ab;       // T: butterfly coefficients
    uint32_t *io;     // T: row destination (forward) or source (inverse)
    uint32_t *row0;   // T: input row of the voxel's first point | kCarry (forward gather)
    uint32_t *idx;    // T: butterfly i0 | i1 << 16
    uint16_t *re;     // kRounds: end of each round
    uint32_t *cnt;    // 2: butterflies, rounds
};

__host__ __device__ inline size_t pipe_meta_bytes(uint32_t T) { return ((size_t)28 * T + 2 * kRounds + 16 + 15) & ~(size_t)15; }

// Row stride in shared memory (floats): rows are packed.
__host__ __device__ inline uint32_t pipe_stride(uint32_t C) { return C; }

__host__ __device__ inline size_t pipe_smem(uint32_t NR, uint32_t T, uint32_t C, bool color)
{
    return NR * (size_t)T * pipe_stride(C) * 4 + (NR + 1) * pipe_meta_bytes(T) +
           (color ? 4 * (size_t)kKltFloats + 16 : 0);
}

__device__ __forceinline__ PipeStage pipe_stage(unsigned char *base, uint32_t T)
{
    PipeStage s;
    s.codes = reinterpret_cast<uint64_t *>(base);
    s.ab = reinterpret_cast<float2 *>(base + 8 * (size_t)T);
    s.io = reinterpret_cast<uint32_t *>(base + 16 * (size_t)T);
    s.row0 = s.io + T;
    s.idx = s.row0 + T;
    s.re = reinterpret_cast<uint16_t *>(base + 28 * (size_t)T);
    s.cnt = reinterpret_cast<uint32_t *>(base + 28 * (size_t)T + 2 * kRounds);
    return s;
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ float4 lds4(uint32_t a)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a)
                 : "memory");
    return v;
}
__device__ __forceinline__ void sts4(uint32_t a, float4 v)
{
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}
__device__ __forceinline__ void cp_async16_s(uint32_t sa, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint32_t pipe_rows(const RahtPass &ps, uint32_t T, uint32_t t)
{
    const uint64_t j0 = (uint64_t)t * T;
    return (uint32_t)((ps.n - j0) < T ? (ps.n - j0) : T);
}

template <bool GATHER>
__device__ void pipe_issue_meta(const XformArgs<float> &A, const RahtPass &ps, uint32_t t, const PipeStage &M)
{
    const RahtPlanDev &p = A.p;
    const RahtIO &io = A.io;
    const uint32_t T = p.T, m = pipe_rows(ps, T, t), tile = ps.tile_off + t;
    const uint64_t j0 = (uint64_t)t * T;
    for (uint32_t i = threadIdx.x; i < m; i += kXThreads) {
        cp_async_vec<4>(M.io + i, p.dest + ps.seq_off + j0 + i);
        if (GATHER) {
            cp_async_vec<4>(M.row0 + i, io.row0 + j0 + i);
            if (io.frame_shift < 64) cp_async_vec<8>(M.codes + i, io.codes + j0 + i);
        }
    }
    // whole per-tile schedule arrays (T butterflies, kRounds round ends): the
    // count is not known yet, the entries past it are never read
    for (uint32_t k = threadIdx.x; k < T; k += kXThreads) {
        cp_async_vec<4>(M.idx + k, p.bf_idx + (uint64_t)tile * T + k);
        cp_async_vec<8>(M.ab + k, p.bf_ab + (uint64_t)tile * T + k);
    }
    if (threadIdx.x < 2 * kRounds / 16)
        cp_async_vec<16>(reinterpret_cast<unsigned char *>(M.re) + 16 * threadIdx.x,
                         reinterpret_cast<const unsigned char *>(p.round_end + (uint64_t)tile * kRounds) +
                             16 * threadIdx.x);
    if (threadIdx.x == 0) {
        cp_async_vec<4>(M.cnt, p.tile_nbf + tile);
        cp_async_vec<4>(M.cnt + 1, p.tile_nr + tile);
    }
}

__device__ __forceinline__ uint32_t pipe_frame(const RahtIO &io, const PipeStage &M, uint32_t i)
{
    return io.frame_shift < 64 ? (uint32_t)(uint8_t)(M.codes[i] >> io.frame_shift) : 0u;
}

template <bool INV, bool GATHER>
__device__ void pipe_issue_rows(const XformArgs<float> &A, const RahtPass &ps, const RahtPass &nx, uint32_t t,
                                const PipeStage &M, float *R)
{
    const RahtIO &io = A.io;
    const uint32_t T = A.p.T, C = io.C, m = pipe_rows(ps, T, t);
    const uint64_t j0 = (uint64_t)t * T;
    const uint32_t L = C / 4, slots = kXThreads / L, slot = threadIdx.x / L, lane = threadIdx.x - slot * L;
    const uint32_t c = lane * 4;
    if (slot >= slots) return;
    const uint32_t rs = pipe_stride(C) * 4;  // row stride in bytes
    uint32_t sa = smem_addr(R) + slot * rs + c * 4;
    const float *base = nullptr;
    uint32_t bfr = 0xFFFFFFFFu;
    for (uint32_t i = slot; i < m; i += slots, sa += slots * rs) {
        const float *src;
        if (!INV) {
            if (GATHER) {
                const uint32_t fr = pipe_frame(io, M, i);
                if (fr != bfr) {
                    base = io.attr[fr] + c;
                    bfr = fr;
                }
                src = base + (size_t)(M.row0[i] & ~kCarry) * C;
            } else {
                src = io.in + (j0 + i) * C + c;
            }
        } else {
            const uint32_t d = M.io[i];
            src = (d & kCarry) ? io.pool + ((uint64_t)nx.surv_off + (d & ~kCarry)) * C + c : io.Y + (uint64_t)d * C + c;
        }
        cp_async16_s(sa, src);
    }
}

// Threads map to (row slot, 4-channel column): 14 consecutive threads cover a
// 56-channel row, so every butterfly reads and writes whole rows contiguously.
template <bool INV, bool GATHER, bool QDQ>
__device__ void pipe_compute(const XformArgs<float> &A, const RahtPass &ps, const RahtPass &nx, uint32_t t,
                             const PipeStage &M, float *R, float *klt_s, uint32_t &klt_fr)
{
    typedef Vec<float, 4> V4;
    const RahtIO &io = A.io;
    const uint32_t T = A.p.T, C = io.C, CP = pipe_stride(C), m = pipe_rows(ps, T, t);
    const uint64_t j0 = (uint64_t)t * T;
    const int tid = threadIdx.x;
    const uint32_t L = C / 4, slots = kXThreads / L, slot = tid / L, lane = tid - slot * L;
    const uint32_t c = lane * 4;
    const bool act = slot < slots;
    const uint32_t rs = CP * 4, sR = smem_addr(R), sbase = sR + c * 4;  // byte addresses in shared memory
    const bool col_fwd = !INV && GATHER && io.klt, col_inv = INV && io.klt;
    // colour mode: the KLT of the tile's first frame, staged once per change of frame
    uint32_t kfr = 0xFFFFFFFFu;
    if (col_fwd || col_inv) {
        kfr = col_fwd ? pipe_frame(io, M, 0) : frame_of_voxel(io.vstart, io.F, j0);
        if (kfr != klt_fr) {
            __syncthreads();  // the previous tile's readers of klt_s are done
            for (uint32_t k = tid; k < (uint32_t)kKltFloats; k += kXThreads)
                klt_s[k] = io.klt[(uint64_t)kfr * kKltFloats + k];
            klt_fr = kfr;
            __syncthreads();
        }
    }
    // finishing in place: cluster average and centring (forward), quantise -> dequantise (inverse)
    if (act && !INV && GATHER) {
        const bool ctr_any = io.center != nullptr && !io.klt;
        uint32_t cfr = 0xFFFFFFFFu;
        float4 ctr = make_float4(0.f, 0.f, 0.f, 0.f);
        for (uint32_t i = slot; i < m; i += slots) {
            const bool multi = (M.row0[i] & kCarry) != 0;
            if (!multi && !ctr_any) continue;
            const uint32_t fr = pipe_frame(io, M, i);
            const uint32_t pr = sbase + i * rs;
            float4 acc = lds4(pr);
            float *pa = reinterpret_cast<float *>(&acc);
            if (multi) {  // voxels holding several points: average in input order
                const uint32_t s0 = io.seg[j0 + i], s1 = io.seg[j0 + i + 1];
                const float *base = io.attr[fr];
                for (uint32_t g = s0 + 1; g < s1; ++g) {
                    const float4 xv = V4::ld(base + (uint64_t)io.vals[g] * C + c);
                    const float *px = reinterpret_cast<const float *>(&xv);
#pragma unroll
                    for (int e = 0; e < 4; ++e) pa[e] = add_rn(pa[e], px[e]);
                }
                const float cnt = (float)(s1 - s0);
#pragma unroll
                for (int e = 0; e < 4; ++e) pa[e] = div_rn(pa[e], cnt);
            }
            if (ctr_any) {  // centred rows keep the low-pass sums small (FP32 accuracy)
                if (fr != cfr) {
                    ctr = V4::ld(io.center + (uint64_t)fr * C + c);
                    cfr = fr;
                }
                const float *pc = reinterpret_cast<const float *>(&ctr);
#pragma unroll
                for (int e = 0; e < 4; ++e) pa[e] = add_rn(pa[e], -pc[e]);
            }
            sts4(pr, acc);
        }
    } else if (act && INV && QDQ) {
        const float4 inv = V4::ld(io.inv_step + c), stp = V4::ld(io.step + c);
        const float *pi = reinterpret_cast<const float *>(&inv), *pt = reinterpret_cast<const float *>(&stp);
        for (uint32_t i = slot; i < m; i += slots) {
            if (M.io[i] & kCarry) continue;
            const uint32_t pr = sbase + i * rs;
            float4 v = lds4(pr);
            float *pv = reinterpret_cast<float *>(&v);
#pragma unroll
            for (int e = 0; e < 4; ++e) pv[e] = qdq(pv[e], pi[e], pt[e], io.tau);
            sts4(pr, v);
        }
    }
    if (col_fwd) {  // colour decorrelation of whole rows, then centring
        __syncthreads();
        for (uint32_t e = tid; e < m * 16; e += kXThreads)
            color_yuv_task(R + (uint64_t)(e >> 4) * CP, (int)(e & 15), kYuvFwd);
        __syncthreads();
        for (uint32_t e = tid; e < m * 3; e += kXThreads) {
            const uint32_t i = e / 3, ch = e - 3 * i;
            const uint32_t fr = pipe_frame(io, M, i);
            const float *K = (fr == kfr ? klt_s : io.klt + (uint64_t)fr * kKltFloats) + ch * kKltN * kKltN;
            color_klt_task<false>(R + (uint64_t)i * CP, (int)ch, K);
        }
        if (io.center) {
            __syncthreads();
            for (uint32_t e = tid; e < m * C; e += kXThreads) {
                const uint32_t i = e / C, cc = e - i * C;
                const uint32_t fr = pipe_frame(io, M, i);
                R[(uint64_t)i * CP + cc] = __fadd_rn(R[(uint64_t)i * CP + cc], -io.center[(uint64_t)fr * C + cc]);
            }
        }
    }
    __syncthreads();
    // rounds
    const uint32_t nr = M.cnt[1];
    for (uint32_t rr = 0; rr < nr; ++rr) {
        const uint32_t r = INV ? (nr - 1 - rr) : rr;
        const uint32_t kb = r ? M.re[r - 1] : 0u, ke = M.re[r];
        if (act) {
            for (uint32_t k = kb + slot; k < ke; k += slots) {
                const uint32_t ix = M.idx[k];
                const float2 ab = M.ab[k];
                const uint32_t r0 = sbase + (ix & 0xFFFFu) * rs, r1 = sbase + (ix >> 16) * rs;
                float4 y0 = lds4(r0), y1 = lds4(r1);
                rot<INV>(ab.x, ab.y, y0, y1);
                sts4(r0, y0);
                sts4(r1, y1);
            }
        }
        __syncthreads();
    }
    if (col_inv) {  // undo the colour decorrelation of whole rows
        for (uint32_t e = tid; e < m * 3; e += kXThreads) {
            const uint32_t i = e / 3, ch = e - 3 * i;
            const uint32_t fr = frame_of_voxel(io.vstart, io.F, j0 + i);
            if (io.frame_color && !io.frame_color[fr]) continue;
            const float *K = (fr == kfr ? klt_s : io.klt + (uint64_t)fr * kKltFloats) + ch * kKltN * kKltN;
            color_klt_task<true>(R + (uint64_t)i * CP, (int)ch, K);
        }
        __syncthreads();
        for (uint32_t e = tid; e < m * 16; e += kXThreads) {
            const uint32_t i = e >> 4;
            const uint32_t fr = io.F > 1 ? frame_of_voxel(io.vstart, io.F, j0 + i) : 0u;
            if (io.frame_color && !io.frame_color[fr]) continue;
            color_yuv_task(R + (uint64_t)i * CP, (int)(e & 15), io.yuv_inv.m);
        }
        __syncthreads();
    }
    // store rows (the buffer is refilled only after a later barrier)
    if (act) {
        for (uint32_t i = slot; i < m; i += slots) {
            const float4 v = lds4(sbase + i * rs);
            if (!INV) {
                const uint32_t d = M.io[i];
                if (d & kCarry)
                    V4::st(io.pool + ((uint64_t)nx.surv_off + (d & ~kCarry)) * C + c, v);
                else
                    V4::st(io.Y + (uint64_t)d * C + c, v);
            } else if (io.lod_mean) {
                const float dv = lod_divisor<float>(A.p, j0 + i);
                V4::st(io.out + (j0 + i) * C + c, make_float4(__fdiv_rn(v.x, dv), __fdiv_rn(v.y, dv),
                                                              __fdiv_rn(v.z, dv), __fdiv_rn(v.w, dv)));
            } else {
                V4::st(io.out + (j0 + i) * C + c, v);
            }
        }
    }
}

template <int NR, bool INV, bool GATHER, bool QDQ>
__global__ void __launch_bounds__(kXThreads, NR == 1 ? 3 : 1) xform_pipe_kernel(XformArgs<float> A)
{
    constexpr uint32_t NM = NR + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RahtPass ps = A.p.passes[0];
    const RahtPass nx = A.p.passes[1];
    const uint32_t T = A.p.T, C = A.io.C;
    const size_t rowb = (size_t)T * pipe_stride(C) * 4, metab = pipe_meta_bytes(T);
    float *klt_s = reinterpret_cast<float *>(smem_raw + NR * rowb + NM * metab);
    const uint32_t G = gridDim.x, b = blockIdx.x, nt = ps.ntiles;
    const uint32_t cnt = b < nt ? (nt - 1 - b) / G + 1 : 0u;  // tiles of this CTA
    auto rows = [&](uint32_t k) { return reinterpret_cast<float *>(smem_raw + (size_t)(k % NR) * rowb); };
    auto meta = [&](uint32_t k) { return pipe_stage(smem_raw + NR * rowb + (size_t)(k % NM) * metab, T); };
    uint32_t klt_fr = 0xFFFFFFFFu;
    if constexpr (NR == 1) {
        // Tiles are claimed from a global counter as the CTA goes (the next but one while the current one is
        // transformed), so a CTA that starts late or runs slow (its SM shared with other work) takes fewer
        // tiles; the claims ascend, so a claim past the last tile ends the CTA's loop.
        __shared__ uint32_t s_claim[4];
        if (threadIdx.x == 0) {
            s_claim[0] = atomicAdd(A.p.pipe_ctr, 1u);
            s_claim[1] = atomicAdd(A.p.pipe_ctr, 1u);
        }
        __syncthreads();
        if (s_claim[0] < nt) pipe_issue_meta<GATHER>(A, ps, s_claim[0], meta(0));
        if (s_claim[1] < nt) pipe_issue_meta<GATHER>(A, ps, s_claim[1], meta(1));
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        if (s_claim[0] < nt) pipe_issue_rows<INV, GATHER>(A, ps, nx, s_claim[0], meta(0), rows(0));
        cp_async_commit();
        for (uint32_t k = 0;; ++k) {
            const uint32_t tk = s_claim[k & 3];
            if (tk >= nt) break;
            // complete: rows of tile k, metadata of tile k + 1.  Without colour transforms no barrier is needed
            // here: a thread first touches only the row chunks it copied itself (same thread-to-chunk mapping
            // for the copy and the finishing step, complete for it after its own wait), tile k's metadata became
            // visible at the previous tile's first barrier, and the barrier before the rounds orders the rest.
            cp_async_wait<0>();
            if (A.io.klt) __syncthreads();  // the colour steps read other threads' rows
            pipe_compute<INV, GATHER, QDQ>(A, ps, nx, tk, meta(k), rows(k), klt_s, klt_fr);
            if (threadIdx.x == 0) s_claim[(k + 2) & 3] = atomicAdd(A.p.pipe_ctr, 1u);
            __syncthreads();  // the row buffer and tile k's metadata are free; the new claim is visible
            const uint32_t t1 = s_claim[(k + 1) & 3], t2 = s_claim[(k + 2) & 3];
            if (t2 < nt) pipe_issue_meta<GATHER>(A, ps, t2, meta(k + 2));
            if (t1 < nt) pipe_issue_rows<INV, GATHER>(A, ps, nx, t1, meta(k + 1), rows(k + 1));
            cp_async_commit();
        }
        cp_async_wait<0>();
        if (threadIdx.x == 0) {  // the last CTA to finish leaves the counters at zero for the next launch
            __threadfence();
            if (atomicAdd(A.p.pipe_ctr + 1, 1u) == gridDim.x - 1) {
                A.p.pipe_ctr[0] = 0;
                A.p.pipe_ctr[1] = 0;
                __threadfence();
            }
        }
        return;
    }
    // prologue: metadata of tiles 0 .. NR - 1, then the rows of tiles 0 .. NR - 2
    constexpr uint32_t kMeta0 = NR == 1 ? 2u : NR, kRows0 = NR == 1 ? 1u : NR - 1;
    for (uint32_t k = 0; k < kMeta0 && k < cnt; ++k) pipe_issue_meta<GATHER>(A, ps, b + k * G, meta(k));
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    for (uint32_t k = 0; k < kRows0; ++k) {
        if (k < cnt) pipe_issue_rows<INV, GATHER>(A, ps, nx, b + k * G, meta(k), rows(k));
        cp_async_commit();
    }
    for (uint32_t k = 0; k < cnt; ++k) {
        if constexpr (NR == 1) {
            break;  // tiles are claimed dynamically below
        } else {
            // complete: rows of tile k, metadata of tile k + NR - 1 (only the rows of k + NR - 2 may still fly)
            cp_async_wait<1>();
            __syncthreads();
            if (k + NR < cnt) pipe_issue_meta<GATHER>(A, ps, b + (k + NR) * G, meta(k + NR));
            cp_async_commit();
            if (k + NR - 1 < cnt)
                pipe_issue_rows<INV, GATHER>(A, ps, nx, b + (k + NR - 1) * G, meta(k + NR - 1), rows(k + NR - 1));
            cp_async_commit();
            pipe_compute<INV, GATHER, QDQ>(A, ps, nx, b + k * G, meta(k), rows(k), klt_s, klt_fr);
        }
    }
    cp_async_wait<0>();
}

int max_optin_smem()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// The pipelined first pass applies to FP32 transforms with 4-float vectors and
// whole rows per tile whose buffers fit one CTA's shared memory.  Returns NR, or
// 0 for the plain passes.
template <typename S, int VEC>
int pipe_depth(const XformArgs<S> &A, size_t *smem)
{
    if (!std::is_same<S, float>::value || VEC != 4 || A.p.xpipe_off == 1) return 0;
    if (A.Cg != A.io.C || A.io.C % 4 || A.io.C / 4 > (uint32_t)kXThreads) return 0;
    const int nr = A.p.xpipe_off == 2 ? 3 : 1;
    *smem = pipe_smem(nr, A.p.T, A.io.C, A.io.klt != nullptr);
    return *smem <= (size_t)max_optin_smem() ? nr : 0;
}

template <int NR, bool INV, bool GATHER, bool QDQ>
void launch_pipe(const XformArgs<float> &A, uint64_t nv_bound, size_t smem, int num_sms, cudaStream_t s)
{
    auto k = xform_pipe_kernel<NR, INV, GATHER, QDQ>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;  // resident CTAs per SM with this shared memory (one wave)
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kXThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const uint64_t tiles = (nv_bound + A.p.T - 1) / A.p.T;
    const uint64_t cap = (uint64_t)num_sms * (uint64_t)per_sm;
    const uint32_t grid = (uint32_t)(tiles < 1 ? 1 : (tiles < cap ? tiles : cap));
    k<<<grid, kXThreads, smem, s>>>(A);
    count_launch();
}

template <bool INV, bool GATHER, bool QDQ>
void launch_pipe_nr(int nr, const XformArgs<float> &A, uint64_t nv_bound, size_t smem, int num_sms, cudaStream_t s)
{
    if (nr == 3)
        launch_pipe<3, INV, GATHER, QDQ>(A, nv_bound, smem, num_sms, s);
    else
        launch_pipe<1, INV, GATHER, QDQ>(A, nv_bound, smem, num_sms, s);
}

uint32_t channel_group(uint32_t C, uint32_t T, uint32_t elem)
{
    uint32_t cg = kSmemRowBytes / (elem * T);
    if (cg >= C) return C;
    if (C % 4 == 0) cg &= ~3u;
    return cg < 1 ? 1 : cg;
}

template <typename S>
size_t xform_smem(uint32_t T, uint32_t Cg, bool color)
{
    return ((xform_meta_bytes<S>(T) + 15) & ~(size_t)15) + sizeof(S) * T * Cg +
           (color ? 4 * (size_t)kKltFloats + 16 : 0);
}

template <typename S, bool INV, int VEC, bool GATHER, bool QDQ>
void launch_pass(const XformArgs<S> &A, int q, uint32_t grid, size_t smem, cudaStream_t s)
{
    auto k = xform_pass_kernel<S, INV, VEC, GATHER, QDQ>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<grid, kXThreads, smem, s>>>(A, q);
    count_launch();
}

template <typename S, bool INV, int VEC, bool QDQ>
void launch_finish(const XformArgs<S> &A, int q0, size_t smem, cudaStream_t s)
{
    auto k = xform_finish_kernel<S, INV, VEC, QDQ>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<1, kXThreads, smem, s>>>(A, q0);
    count_launch();
}

template <typename S, int VEC>
void forward_all(const XformArgs<S> &A, uint64_t nv_bound, int num_sms, cudaStream_t s)
{
    const uint32_t T = A.p.T;
    const size_t smem = xform_smem<S>(T, A.Cg, A.io.klt != nullptr);
    uint64_t tiles = (nv_bound + T - 1) / T;
    const uint64_t gcap = (uint64_t)num_sms * (A.p.xgrid_mult ? A.p.xgrid_mult : 4u);
    uint32_t grid0 = (uint32_t)(tiles < 1 ? 1 : (tiles < gcap ? tiles : gcap));
    for (int q = 0; q < kRahtMultiPasses; ++q) {
        uint32_t g = q == 0 ? grid0 : (grid0 < (uint32_t)num_sms ? grid0 : (uint32_t)num_sms);
        if (q == 0) stage_begin(s, kStRahtFwd0);
        size_t psm = 0;
        if constexpr (std::is_same<S, float>::value) {
            const int nr = q == 0 && (!A.io.seg || A.io.row0) ? pipe_depth<S, VEC>(A, &psm) : 0;
            if (nr) {
                if (A.io.seg)
                    launch_pipe_nr<false, true, false>(nr, A, nv_bound, psm, num_sms, s);
                else
                    launch_pipe_nr<false, false, false>(nr, A, nv_bound, psm, num_sms, s);
                stage_end(s, kStRahtFwd0);
                continue;
            }
        }
        if (q == 0 && A.io.seg)
            launch_pass<S, false, VEC, true, false>(A, q, g, smem, s);
        else
            launch_pass<S, false, VEC, false, false>(A, q, g, smem, s);
        if (q == 0) stage_end(s, kStRahtFwd0);
    }
    launch_finish<S, false, VEC, false>(A, kRahtMultiPasses, smem, s);
}

template <typename S, int VEC>
void inverse_all(const XformArgs<S> &A, uint64_t nv_bound, int num_sms, cudaStream_t s)
{
    const uint32_t T = A.p.T;
    const size_t smem = xform_smem<S>(T, A.Cg, A.io.klt != nullptr);
    uint64_t tiles = (nv_bound + T - 1) / T;
    const uint64_t gcap = (uint64_t)num_sms * (A.p.xgrid_mult ? A.p.xgrid_mult : 4u);
    uint32_t grid0 = (uint32_t)(tiles < 1 ? 1 : (tiles < gcap ? tiles : gcap));
    const bool qd = A.io.inv_step != nullptr;
    if (qd)
        launch_finish<S, true, VEC, true>(A, kRahtMultiPasses, smem, s);
    else
        launch_finish<S, true, VEC, false>(A, kRahtMultiPasses, smem, s);
    for (int q = kRahtMultiPasses - 1; q >= 0; --q) {
        uint32_t g = q == 0 ? grid0 : (grid0 < (uint32_t)num_sms ? grid0 : (uint32_t)num_sms);
        if (q == 0) stage_begin(s, kStRahtInv0);
        size_t psm = 0;
        if constexpr (std::is_same<S, float>::value) {
            const int nr = q == 0 ? pipe_depth<S, VEC>(A, &psm) : 0;
            if (nr) {
                if (qd)
                    launch_pipe_nr<true, false, true>(nr, A, nv_bound, psm, num_sms, s);
                else
                    launch_pipe_nr<true, false, false>(nr, A, nv_bound, psm, num_sms, s);
                stage_end(s, kStRahtInv0);
                continue;
            }
        }
        if (qd)
            launch_pass<S, true, VEC, false, true>(A, q, g, smem, s);
        else
            launch_pass<S, true, VEC, false, false>(A, q, g, smem, s);
        if (q == 0) stage_end(s, kStRahtInv0);
    }
}

}  // namespace

uint32_t raht_tile_size(uint32_t C)
{
    if (C == 0) return 4096;
    uint32_t t = kSmemRowBytes / (4u * C);
    uint32_t T = 256;
    while (T * 2 <= t && T < 4096) T *= 2;
    return T;
}

void raht_plan_sizes(uint64_t nv_cap, uint32_t T, uint64_t *elems, uint64_t *tiles, uint64_t *surv_rows)
{
    // a full tile keeps at most 2*63+1 < T/2 survivors, so every pass at least
    // halves the sequence up to one partial tile (<= 127 extra per pass)
    *elems = 2 * nv_cap + 130 * (kRahtMaxPasses + 1);
    *tiles = 2 * ((nv_cap + T - 1) / T) + 2 * (kRahtMaxPasses + 1);
    *surv_rows = nv_cap + 128 * (kRahtMaxPasses + 1);
}

template <int TMAX>
void prelude_launches(const PreludeArgs &a, const RahtPlanDev &p, const DevState *st, const uint64_t *nv_dev,
                      int num_sms, cudaStream_t s)
{
    const size_t smem = prelude_smem_bytes<TMAX>();
    cudaFuncSetAttribute(prelude_tiles_kernel<TMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(prelude_finish_kernel<TMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prelude_init_kernel<<<1, 32, 0, s>>>(p, st, nv_dev);
    count_launch();
    uint32_t grid = (uint32_t)num_sms * (p.pgrid_mult ? p.pgrid_mult : 8u);
    for (int q = 0; q < kRahtMultiPasses; ++q) {
        prelude_tiles_kernel<TMAX><<<grid, kThreads, smem, s>>>(a, q);
        count_launch();
        prelude_scan_kernel<<<1, 1024, 0, s>>>(p, q);
        count_launch();
        prelude_compact_kernel<<<grid, kThreads, 0, s>>>(a, q);
        count_launch();
    }
    prelude_finish_kernel<TMAX><<<1, kThreads, smem, s>>>(a, kRahtMultiPasses);
    count_launch();
}

void launch_raht_prelude(const RahtPlanDev &p, const uint8_t *gap, const DevState *st, const uint64_t *nv_dev,
                         int num_sms, cudaStream_t s)
{
    PreludeArgs a;
    a.p = p;
    a.gap0 = gap;
    a.st = st;
    if (p.T <= 256)
        prelude_launches<256>(a, p, st, nv_dev, num_sms, s);
    else if (p.T <= 1024)
        prelude_launches<1024>(a, p, st, nv_dev, num_sms, s);
    else
        prelude_launches<4096>(a, p, st, nv_dev, num_sms, s);
}

template <typename S>
void launch_raht_forward(const RahtPlanDev &p, const RahtIOT<S> &io, uint64_t nv_bound, int num_sms, cudaStream_t s)
{
    if (io.C == 0) return;
    XformArgs<S> A;
    A.p = p;
    A.io = io;
    A.Cg = channel_group(io.C, p.T, sizeof(S));
    constexpr int kV = 16 / sizeof(S);  // 16-byte vectors: 4 floats or 2 doubles
    if (A.Cg % kV == 0 && io.C % kV == 0)
        forward_all<S, kV>(A, nv_bound, num_sms, s);
    else
        forward_all<S, 1>(A, nv_bound, num_sms, s);
}

template <typename S>
void launch_raht_inverse(const RahtPlanDev &p, const RahtIOT<S> &io, uint64_t nv_bound, int num_sms, cudaStream_t s)
{
    if (io.C == 0) return;
    XformArgs<S> A;
    A.p = p;
    A.io = io;
    A.Cg = channel_group(io.C, p.T, sizeof(S));
    constexpr int kV = 16 / sizeof(S);
    if (A.Cg % kV == 0 && io.C % kV == 0)
        inverse_all<S, kV>(A, nv_bound, num_sms, s);
    else
        inverse_all<S, 1>(A, nv_bound, num_sms, s);
}

template void launch_raht_forward<float>(const RahtPlanDev &, const RahtIOT<float> &, uint64_t, int, cudaStream_t);
template void launch_raht_forward<double>(const RahtPlanDev &, const RahtIOT<double> &, uint64_t, int, cudaStream_t);
template void launch_raht_inverse<float>(const RahtPlanDev &, const RahtIOT<float> &, uint64_t, int, cudaStream_t);
template void launch_raht_inverse<double>(const RahtPlanDev &, const RahtIOT<double> &, uint64_t, int, cudaStream_t);

// ---- centring of the forward transform ---------------------------------------
// RAHT is linear with T 1 = sqrt(N_v) e_DC (a constant has no high pass), so
// T (A - c 1) = T A - c sqrt(N_v) e_DC for any c: centring changes only the DC
// and, in FP32, keeps the low-pass sums near the data's spread instead of its
// mean (the high-pass coefficients of large nodes are differences of such sums).
namespace {

constexpr uint32_t kCentreRows = 1024;

__global__ void __launch_bounds__(256) frame_centres_kernel(const float *const *attr, const uint64_t *poff,
                                                            uint32_t C, float *center)
{
    __shared__ float part[256];
    const uint32_t f = blockIdx.x;
    const uint32_t lanes = blockDim.x / C;  // row phases
    const uint32_t t = threadIdx.x, j = t / C, c = t - j * C;
    const uint64_t n = poff[f + 1] - poff[f];
    const uint32_t m = (uint32_t)(n < kCentreRows ? n : kCentreRows);
    const float *a = attr[f];
    float sum = 0.f;
    if (j < lanes) {  // rows j, j + lanes, ... added in that order; 16 loads in flight at a time
        constexpr uint32_t kAhead = 16;
        uint32_t r = j;
        for (; r + (kAhead - 1) * lanes < m; r += kAhead * lanes) {
            float x[kAhead];
#pragma unroll
            for (uint32_t u = 0; u < kAhead; ++u) x[u] = __ldg(a + (uint64_t)(r + u * lanes) * C + c);
#pragma unroll
            for (uint32_t u = 0; u < kAhead; ++u) sum = __fadd_rn(sum, x[u]);
        }
        for (; r < m; r += lanes) sum = __fadd_rn(sum, a[(uint64_t)r * C + c]);
    }
    if (j < lanes) part[t] = sum;
    __syncthreads();
    if (j == 0) {
        float tot = 0.f;
        for (uint32_t q = 0; q < lanes; ++q) tot = __fadd_rn(tot, part[q * C + c]);
        center[(uint64_t)f * C + c] = m ? __fdiv_rn(tot, (float)m) : 0.f;
    }
}

__global__ void frame_dc_kernel(float *Y, const uint32_t *vstart, uint32_t C, const float *center,
                                const double *steps_rg, const uint8_t *groups, uint32_t G, double tau, double *dc)
{
    const uint32_t f = blockIdx.x;
    const uint32_t v0 = vstart[f], nv = vstart[f + 1] - v0;
    for (uint32_t c = threadIdx.x; c < C; c += blockDim.x) {
        if (nv == 0) {
            dc[(uint64_t)f * C + c] = 0.0;
            continue;
        }
        float *y = Y + (uint64_t)v0 * C + c;
        const double d = __dadd_rn((double)*y, __dmul_rn(__dsqrt_rn((double)nv), (double)center[(uint64_t)f * C + c]));
        dc[(uint64_t)f * C + c] = d;
        const double st0 = steps_rg[groups[c]];  // rung 0
        *y = (float)__dmul_rn((double)quantize_f64(d, st0, tau), st0);
    }
}

}  // namespace

void launch_frame_centres(const float *const *attr, const uint64_t *poff, uint32_t F, uint32_t C, float *center,
                          cudaStream_t s)
{
    if (F == 0 || C == 0) return;
    uint32_t lanes = 256 / C;
    if (lanes < 1) lanes = 1;
    frame_centres_kernel<<<F, lanes * C, 0, s>>>(attr, poff, C, center);
    count_launch();
}

void launch_frame_dc(float *Y, const uint32_t *vstart, uint32_t F, uint32_t C, const float *center,
                     const double *steps_rg, const uint8_t *groups, uint32_t G, double tau, double *dc, cudaStream_t s)
{
    if (F == 0 || C == 0) return;
    frame_dc_kernel<<<F, 64, 0, s>>>(Y, vstart, C, center, steps_rg, groups, G, tau, dc);
    count_launch();
}

}  // namespace gsnfs
