// SH colour decorrelation (Sec. 4) applied to one 56-channel row held in
// shared memory: BT.601 YUV on every SH function (DC at channels 8-10, AC
// function k at 11+k, 26+k, 41+k), then a' = K_ch a for each YUV channel's 15
// AC values (K: three row-major 15 x 15, rows = eigenvectors).  The inverse
// applies K^T, then the inverse YUV matrix (passed in, computed from the
// forward one in FP64 on the host).
#pragma once

namespace gsnfs {

constexpr int kKltN = 15;
constexpr int kKltFloats = 3 * kKltN * kKltN;

struct YuvInv {
    float m[9];
};

__device__ __forceinline__ int sh_chan(int k, int col) { return k == 0 ? 8 + col : 11 + kKltN * col + (k - 1); }

__device__ __forceinline__ void yuv3(const float *m, float &a, float &b, float &c)
{
    const float x = a, y = b, z = c;
    a = __fadd_rn(__fadd_rn(__fmul_rn(m[0], x), __fmul_rn(m[1], y)), __fmul_rn(m[2], z));
    b = __fadd_rn(__fadd_rn(__fmul_rn(m[3], x), __fmul_rn(m[4], y)), __fmul_rn(m[5], z));
    c = __fadd_rn(__fadd_rn(__fmul_rn(m[6], x), __fmul_rn(m[7], y)), __fmul_rn(m[8], z));
}

__device__ __forceinline__ void color_forward_row(float *row, const float *K)
{
    const float M[9] = {0.299f, 0.587f, 0.114f, -0.14713f, -0.28886f, 0.436f, 0.615f, -0.51499f, -0.10001f};
    for (int k = 0; k <= kKltN; ++k)
        yuv3(M, row[sh_chan(k, 0)], row[sh_chan(k, 1)], row[sh_chan(k, 2)]);
    for (int ch = 0; ch < 3; ++ch) {
        float a[kKltN];
        float *p = row + 11 + kKltN * ch;
#pragma unroll
        for (int k = 0; k < kKltN; ++k) a[k] = p[k];
        const float *Kc = K + ch * kKltN * kKltN;
        for (int r = 0; r < kKltN; ++r) {
            float t = 0.f;
#pragma unroll
            for (int k = 0; k < kKltN; ++k) t = __fadd_rn(t, __fmul_rn(Kc[r * kKltN + k], a[k]));
            p[r] = t;
        }
    }
}

__device__ __forceinline__ void color_inverse_row(float *row, const float *K, const YuvInv &inv)
{
    for (int ch = 0; ch < 3; ++ch) {
        float a[kKltN];
        float *p = row + 11 + kKltN * ch;
#pragma unroll
        for (int r = 0; r < kKltN; ++r) a[r] = p[r];
        const float *Kc = K + ch * kKltN * kKltN;
        for (int k = 0; k < kKltN; ++k) {
            float t = 0.f;
#pragma unroll
            for (int r = 0; r < kKltN; ++r) t = __fadd_rn(t, __fmul_rn(Kc[r * kKltN + k], a[r]));
            p[k] = t;
        }
    }
    for (int k = 0; k <= kKltN; ++k)
        yuv3(inv.m, row[sh_chan(k, 0)], row[sh_chan(k, 1)], row[sh_chan(k, 2)]);
}

// one SH function of a row: RGB -> YUV (forward) or back (inverse matrix)
__device__ __forceinline__ void color_yuv_task(float *row, int k, const float *m)
{
    yuv3(m, row[sh_chan(k, 0)], row[sh_chan(k, 1)], row[sh_chan(k, 2)]);
}

// one YUV channel's AC vector of a row: a' = K_ch a (forward) or a = K_ch^T a'
template <bool INV>
__device__ __forceinline__ void color_klt_task(float *row, int ch, const float *Kc)
{
    float a[kKltN];
    float *p = row + 11 + kKltN * ch;
#pragma unroll
    for (int k = 0; k < kKltN; ++k) a[k] = p[k];
#pragma unroll
    for (int r = 0; r < kKltN; ++r) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kKltN; ++k)
            t = __fadd_rn(t, __fmul_rn(INV ? Kc[k * kKltN + r] : Kc[r * kKltN + k], a[k]));
        p[r] = t;
    }
}

__device__ __constant__ const float kYuvFwd[9] = {0.299f, 0.587f, 0.114f, -0.14713f, -0.28886f, 0.436f,
                                                   0.615f, -0.51499f, -0.10001f};

YuvInv yuv_inverse();

}  // namespace gsnfs
