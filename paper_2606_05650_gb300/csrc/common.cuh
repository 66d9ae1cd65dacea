// Shared device helpers and internal data structures of the GS-NFS GB300 codec.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gsnfs {

// Gap level given to a frame boundary (any value above 3*21 = 63 works).
constexpr uint32_t kInfLevel = 64;
// Bit 31 of a destination index marks "carried to the next RAHT pass".
constexpr uint32_t kCarry = 0x80000000u;
// Device error codes (first error wins).
constexpr uint32_t kErrCorrupt = 1;
constexpr uint32_t kErrCapacity = 2;
constexpr uint32_t kErrInternal = 3;
constexpr uint32_t kErrTimeout = 4;

constexpr int kMaxFrames = 64;
constexpr int kMaxRungs = 8;
constexpr int kMaxJ = 21;
constexpr int kMaxC = 256;

// Per-frame grid parameters (Sec. 2.1 voxelisation contract).
struct FrameGrid {
    double lo[3];
    double ext;
    double scale;  // 2^J / ext
    double cell;   // ext / 2^J
};

// Small device-resident counters and results of one encode / decode.
struct DevState {
    uint32_t err;
    uint32_t err_info;
    uint32_t bbox_min[kMaxFrames][3];  // order-preserving float encodings
    uint32_t bbox_max[kMaxFrames][3];
    uint64_t nv_total;
    uint64_t total_bytes;  // container size (plain path)
    uint32_t hist[kMaxFrames][256];  // occupancy byte histograms
};

__device__ __forceinline__ void set_error(uint32_t *err, uint32_t code)
{
    atomicCAS(err, 0u, code);
}

__device__ __forceinline__ uint32_t float_to_ordered(float f)
{
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float ordered_to_float(uint32_t o)
{
    uint32_t b = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
    return __uint_as_float(b);
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_sum(T v)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if ((int)lane_id() >= o) v += t;
    }
    return v;
}

// Block-wide exclusive sum for blockDim.x a multiple of 32 (<= 1024).
// `sh` must hold 33 elements.  Returns the exclusive prefix; *total gets
// the block total.  Contains __syncthreads.
template <typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T *sh, T *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_inclusive_sum(v);
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T w = (lane < nw) ? sh[lane] : T(0);
        T wi = warp_inclusive_sum(w);
        if (lane < nw) sh[lane] = wi - w;
        if (lane == nw - 1) sh[32] = wi;
    }
    __syncthreads();
    T res = inc - v + sh[wid];
    *total = sh[32];
    __syncthreads();
    return res;
}

__device__ __forceinline__ uint32_t msb64(uint64_t x) { return 63u - (uint32_t)__clzll((long long)x); }

// Gap level between two consecutive distinct codes of the same frame: the
// binary RAHT level at which they first share an ancestor (1..3J), or
// kInfLevel when they belong to different frames (bits >= frame_shift).
__device__ __forceinline__ uint32_t gap_level(uint64_t a, uint64_t b, uint32_t frame_shift)
{
    uint64_t x = a ^ b;
    if (frame_shift < 64 && (x >> frame_shift) != 0) return kInfLevel;
    return msb64(x) + 1u;
}

// Uniform / dead-zone quantiser of Sec. 3.4 evaluated in FP32:
// q = sign(y) floor(|y| * (1/step) + tau), |q| <= 2^30.
__device__ __forceinline__ int32_t quantize_f32(float y, float inv_step, float tau)
{
    int32_t m = __float2int_rd(__fadd_rn(__fmul_rn(fabsf(y), inv_step), tau));  // floor, saturating
    m = min(m, 1073741824);
    return (y < 0.0f) ? -m : m;
}

// zigzag index of the FP32 quantiser in one step: t = floor(|y| inv + tau)
// (capped at 2^30), u = 2t for q = t >= 0 and 2t - 1 for q = -t < 0
__device__ __forceinline__ uint32_t quantize_zz_f32(float y, float inv_step, float tau)
{
    int32_t t = __float2int_rd(__fadd_rn(__fmul_rn(fabsf(y), inv_step), tau));
    t = min(t, 1073741824);
    return ((uint32_t)t << 1) - (uint32_t)(y < 0.0f && t > 0);
}

// the quantiser of Sec. 3.4 in FP64: sign(y) floor(|y| / step + tau)
__device__ __forceinline__ int32_t quantize_f64(double y, double step, double tau)
{
    double t = floor(__dadd_rn(__ddiv_rn(fabs(y), step), tau));
    t = fmin(t, 1073741824.0);
    const int32_t m = (int32_t)t;
    return (y < 0.0) ? -m : m;
}

}  // namespace gsnfs
