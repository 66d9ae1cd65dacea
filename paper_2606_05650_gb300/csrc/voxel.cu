// Voxelisation and Morton coding (Sec. 2.1 "Voxelization", Sec. 2.2 "Morton
// Codes" and "Voxelization"; Algorithm 1 step 1).
//
// Grid contract (the paper fixes no arithmetic): per frame the bounding box
// lo/hi of the float32 positions, one cube of side ext = max_a(hi_a - lo_a)
// (1 when 0), scale = 2^J / ext by one IEEE FP64 division, and per point
//   v_a = min(2^J - 1, floor(((double)p_a - lo_a) * scale))
// with each operation a separately rounded FP64 op (no FMA), so the voxel
// set is bit-identical to a CPU evaluation of the same contract.
#include "kernels.cuh"

namespace gsnfs {

namespace {

constexpr int kThreads = 256;

__global__ void init_bbox_kernel(DevState *st, uint32_t F)
{
    int t = threadIdx.x;
    if (t == 0) {
        st->err = 0;
        st->err_info = 0;
        st->nv_total = 0;
        st->total_bytes = 0;
    }
    for (int i = t; i < (int)F * 3; i += blockDim.x) {
        (&st->bbox_min[0][0])[i] = 0xFFFFFFFFu;
        (&st->bbox_max[0][0])[i] = 0u;
    }
}

// grid (X, F): block (x, f) reduces a strided share of frame f's points
__global__ void __launch_bounds__(kThreads) bbox_kernel(FrameSet fs, DevState *st)
{
    const uint32_t f = blockIdx.y;
    const float *pos = fs.pos[f];
    const uint64_t n = fs.poff[f + 1] - fs.poff[f];
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (uint64_t)gridDim.x * kThreads) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float p = __ldg(pos + 3 * i + a);
            mn[a] = fminf(mn[a], p);
            mx[a] = fmaxf(mx[a], p);
        }
    }
    __shared__ float smn[3][kThreads / 32], smx[3][kThreads / 32];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xFFFFFFFFu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xFFFFFFFFu, mx[a], o));
        }
        if ((threadIdx.x & 31) == 0) {
            smn[a][threadIdx.x >> 5] = mn[a];
            smx[a][threadIdx.x >> 5] = mx[a];
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        int a = threadIdx.x;
        float m0 = INFINITY, m1 = -INFINITY;
        for (int w = 0; w < kThreads / 32; ++w) {
            m0 = fminf(m0, smn[a][w]);
            m1 = fmaxf(m1, smx[a][w]);
        }
        if (m0 <= m1) {
            atomicMin(&st->bbox_min[f][a], float_to_ordered(m0));
            atomicMax(&st->bbox_max[f][a], float_to_ordered(m1));
        }
    }
}

__global__ void grid_kernel(FrameSet fs, DevState *st)
{
    uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= fs.F) return;
    FrameGrid g;
    const uint64_t n = fs.poff[f + 1] - fs.poff[f];
    const double cells = (double)(1ull << fs.J[f]);
    if (n == 0) {
        g.lo[0] = g.lo[1] = g.lo[2] = 0.0;
        g.ext = 1.0;
    } else {
        double e = 0.0;
        for (int a = 0; a < 3; ++a) {
            double lo = (double)ordered_to_float(st->bbox_min[f][a]);
            double hi = (double)ordered_to_float(st->bbox_max[f][a]);
            g.lo[a] = lo;
            double d = __dsub_rn(hi, lo);
            if (d > e) e = d;
        }
        g.ext = (e > 0.0) ? e : 1.0;
    }
    g.scale = __ddiv_rn(cells, g.ext);
    g.cell = __ddiv_rn(g.ext, cells);
    fs.grid[f] = g;
}

// spreads the low 21 bits of v so that bit b moves to bit 3b
__device__ __forceinline__ uint64_t spread3(uint64_t v)
{
    v &= 0x1FFFFFull;
    v = (v | (v << 32)) & 0x001F00000000FFFFull;
    v = (v | (v << 16)) & 0x001F0000FF0000FFull;
    v = (v | (v << 8)) & 0x100F00F00F00F00Full;
    v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// Voxel index of one coordinate: floor(RN64(RN64(p - lo) * scale)) clamped to
// [0, vmax], exactly as the FP64 definition gives it, mostly without FP64
// arithmetic (GB300's FP64 rate is a small fraction of its FP32 rate).  The
// product is first evaluated in double-float arithmetic (Knuth's TwoSum for
// p - lo, Dekker's exact product via a fused multiply-add) with lo and scale
// split into two floats each: for x = (p - lo) * scale < 2^23 its value x~ is
// within 2^-21 + 4 |lo| scale 2^-48 of x (the second term from the split of
// lo), and the FP64 result within 2^-28 of x, so when x~ lies farther than
// that margin from every integer both have the same floor.  Otherwise (a
// coordinate on or next to a voxel face) the FP64 definition decides.
struct AxisGrid {
    float lo_hi, lo_lo, sc_hi, sc_lo, margin;
    double lo, scale;
};

__device__ __forceinline__ AxisGrid axis_grid(double lo, double scale)
{
    AxisGrid a;
    a.lo = lo;
    a.scale = scale;
    a.lo_hi = (float)lo;
    a.lo_lo = (float)__dsub_rn(lo, (double)a.lo_hi);
    a.sc_hi = (float)scale;
    a.sc_lo = (float)__dsub_rn(scale, (double)a.sc_hi);
    // 2^-20 + 8 |lo| scale 2^-48 (twice the bound above), rounded up
    const double m = 9.5367431640625e-07 + 8.0 * fabs(lo) * scale * 3.552713678800501e-15;
    a.margin = m < 0.25 ? (float)(m * 1.0000002) : 2.0f;  // 2: always the FP64 definition
    return a;
}

__device__ __forceinline__ uint64_t voxel_index(float p, const AxisGrid &g, uint64_t vmax)
{
    // t = p - lo as s + t_lo (TwoSum of p and -lo_hi, then the low part of lo)
    const float s = __fsub_rn(p, g.lo_hi);
    const float bv = __fsub_rn(s, p);
    const float e1 = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bv)), __fsub_rn(-g.lo_hi, bv));
    const float t_lo = __fsub_rn(e1, g.lo_lo);
    // x = t * scale as hi + lo (exact product of s and sc_hi, plus the small cross terms)
    const float hi = __fmul_rn(s, g.sc_hi);
    const float perr = __fmaf_rn(s, g.sc_hi, -hi);
    const float lo = __fadd_rn(perr, __fadd_rn(__fmul_rn(s, g.sc_lo), __fmul_rn(t_lo, g.sc_hi)));
    if (hi >= 1.0f && hi < 8388608.0f) {  // 1 <= x~ < 2^23: fractional part resolvable in FP32
        const float fh = floorf(hi);
        const float f = __fadd_rn(__fsub_rn(hi, fh), lo);
        if (f >= g.margin && f <= 1.0f - g.margin) {  // the same floor as the FP64 definition
            const uint64_t q = (uint64_t)fh;
            return q > vmax ? vmax : q;
        }
    } else if (hi >= 8388608.0f && (double)hi > (double)vmax + 2.0) {
        return vmax;  // far beyond the last voxel either way
    }
    const double u = floor(__dmul_rn(__dsub_rn((double)p, g.lo), g.scale));
    const uint64_t q = (u <= 0.0) ? 0ull : (uint64_t)u;
    return q > vmax ? vmax : q;
}

__global__ void __launch_bounds__(kThreads) morton_kernel(FrameSet fs, uint64_t *keys, uint32_t *vals)
{
    const uint32_t f = blockIdx.y;
    const float *pos = fs.pos[f];
    const uint64_t base = fs.poff[f];
    const uint64_t n = fs.poff[f + 1] - base;
    const uint32_t J = fs.J[f];
    const FrameGrid g = fs.grid[f];
    const uint64_t vmax = (1ull << J) - 1;
    const uint64_t fbits = (fs.frame_shift < 64) ? ((uint64_t)f << fs.frame_shift) : 0ull;
    const AxisGrid ax[3] = {axis_grid(g.lo[0], g.scale), axis_grid(g.lo[1], g.scale), axis_grid(g.lo[2], g.scale)};
    for (uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (uint64_t)gridDim.x * kThreads) {
        uint64_t v[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = voxel_index(__ldg(pos + 3 * i + a), ax[a], vmax);
        keys[base + i] = fbits | spread3(v[0]) | (spread3(v[1]) << 1) | (spread3(v[2]) << 2);
        vals[base + i] = (uint32_t)i;
    }
}

}  // namespace

void launch_voxelize(const FrameSet &fs, DevState *st, uint64_t n_total, uint64_t n_max, uint64_t *keys,
                     uint32_t *vals, int num_sms, cudaStream_t s)
{
    init_bbox_kernel<<<1, 256, 0, s>>>(st, fs.F);
    count_launch();
    // X blocks per frame: enough for the largest frame, ~4 CTAs per SM overall
    uint64_t want = (n_max + kThreads - 1) / kThreads;
    uint64_t cap = (uint64_t)num_sms * 4 / fs.F;
    if (cap < 16) cap = 16;
    uint32_t X = (uint32_t)(want < 1 ? 1 : (want > cap ? cap : want));
    dim3 grid(X, fs.F);
    if (n_total > 0) {
        bbox_kernel<<<grid, kThreads, 0, s>>>(fs, st);
        count_launch();
    }
    grid_kernel<<<1, 64, 0, s>>>(fs, st);
    count_launch();
    if (n_total > 0) {
        morton_kernel<<<grid, kThreads, 0, s>>>(fs, keys, vals);
        count_launch();
    }
}

}  // namespace gsnfs
