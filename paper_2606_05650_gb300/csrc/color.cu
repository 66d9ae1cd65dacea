// KLT of the SH colour decorrelation (Sec. 4): per frame, the covariance of
// each YUV channel's 15 AC values over the frame's first (up to 4096) input
// points (FP32 sums over 16 slices of 256 rows, added in FP64 in a fixed
// order); its eigenvectors by cyclic Jacobi rotations in FP32 (one warp per
// channel, lanes over the matrix columns); rows of K = eigenvectors by
// decreasing eigenvalue, the largest component of each made positive.  The
// frame's centring constants are then carried into the same domain.
#include "color.cuh"
#include "kernels.cuh"

namespace gsnfs {

namespace {

constexpr int kSample = 4096;
constexpr int kSlices = 16;                   // CTAs per frame for the sample sums
constexpr int kSliceRows = kSample / kSlices;  // 256
constexpr int kRowsPerChunk = 32;
constexpr int kPairs = kKltN * (kKltN + 1) / 2;  // 120
constexpr int kPartWords = 3 * (kPairs + kKltN);  // per slice: pair sums, then sums, per channel

__device__ __forceinline__ void pair_of(int p, int &x, int &y)
{
    x = 0;
    while (x < kKltN && p >= kKltN - x) {
        p -= kKltN - x;
        ++x;
    }
    y = x + p;
}

// grid (slices, frames), 3 warps (YUV channels): FP32 sums of the AC products
// and values over one slice of the frame's first 4096 input rows
__global__ void __launch_bounds__(96) klt_partials_kernel(const float *const *attr, const uint64_t *poff,
                                                          double *part)
{
    __shared__ float rows[kRowsPerChunk][48];  // YUV of the 16 SH functions of a chunk of rows
    const uint32_t f = blockIdx.y, sl = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, ch = t >> 5;
    const uint64_t n = poff[f + 1] - poff[f];
    const int m = (int)(n < (uint64_t)kSample ? n : (uint64_t)kSample);
    const int rb = sl * kSliceRows, re = (rb + kSliceRows) < m ? (rb + kSliceRows) : m;
    const float *a = attr[f];
    const float M[9] = {0.299f, 0.587f, 0.114f, -0.14713f, -0.28886f, 0.436f, 0.615f, -0.51499f, -0.10001f};
    float acc[4] = {0.f, 0.f, 0.f, 0.f}, sum = 0.f;
    int px[4], py[4];
    for (int j = 0; j < 4; ++j) pair_of(lane + 32 * j, px[j], py[j]);
    for (int r0 = rb; r0 < re; r0 += kRowsPerChunk) {
        const int cnt = (re - r0) < kRowsPerChunk ? (re - r0) : kRowsPerChunk;
        for (int e = t; e < cnt * 16; e += blockDim.x) {
            const int r = e >> 4, k = e & 15;
            const float *row = a + (uint64_t)(r0 + r) * 56;
            float y0 = row[sh_chan(k, 0)], y1 = row[sh_chan(k, 1)], y2 = row[sh_chan(k, 2)];
            yuv3(M, y0, y1, y2);
            rows[r][k * 3 + 0] = y0;
            rows[r][k * 3 + 1] = y1;
            rows[r][k * 3 + 2] = y2;
        }
        __syncthreads();
        for (int r = 0; r < cnt; ++r) {
            const float *rr = rows[r];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (lane + 32 * j < kPairs)
                    acc[j] = __fadd_rn(acc[j], __fmul_rn(rr[(px[j] + 1) * 3 + ch], rr[(py[j] + 1) * 3 + ch]));
            if (lane < kKltN) sum = __fadd_rn(sum, rr[(lane + 1) * 3 + ch]);
        }
        __syncthreads();
    }
    double *o = part + ((uint64_t)f * kSlices + sl) * kPartWords + ch * (kPairs + kKltN);
    for (int j = 0; j < 4; ++j)
        if (lane + 32 * j < kPairs) o[lane + 32 * j] = (double)acc[j];
    if (lane < kKltN) o[kPairs + lane] = (double)sum;
}

// one CTA (3 warps) per frame: covariance from the slices (fixed order, FP64),
// eigenvectors by cyclic Jacobi (FP32, lanes over columns), ordering and signs
__global__ void __launch_bounds__(96) klt_solve_kernel(const uint64_t *poff, const double *part, float *klt,
                                                       float *center)
{
    __shared__ float S[3][kKltN * kKltN];
    __shared__ float V[3][kKltN * kKltN];
    __shared__ double mu[3][kKltN];
    __shared__ float cs[3][2];
    __shared__ int order[3][kKltN];
    const uint32_t f = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, ch = t >> 5;
    const uint64_t n = poff[f + 1] - poff[f];
    const int m = (int)(n < (uint64_t)kSample ? n : (uint64_t)kSample);
    const double inv_m = m ? 1.0 / (double)m : 0.0;
    const double *pf = part + (uint64_t)f * kSlices * kPartWords + ch * (kPairs + kKltN);
    if (lane < kKltN) {
        double s = 0.0;
        for (int sl = 0; sl < kSlices; ++sl) s += pf[(uint64_t)sl * kPartWords + kPairs + lane];
        mu[ch][lane] = s * inv_m;
    }
    __syncwarp();
    for (int j = 0; j < 4; ++j) {
        const int p = lane + 32 * j;
        if (p < kPairs) {
            double s = 0.0;
            for (int sl = 0; sl < kSlices; ++sl) s += pf[(uint64_t)sl * kPartWords + p];
            int x, y;
            pair_of(p, x, y);
            const float c = (float)(s * inv_m - mu[ch][x] * mu[ch][y]);
            S[ch][x * kKltN + y] = c;
            S[ch][y * kKltN + x] = c;
        }
    }
    if (lane < kKltN)
        for (int k = 0; k < kKltN; ++k) V[ch][lane * kKltN + k] = (lane == k) ? 1.f : 0.f;
    __syncwarp();
    float *Sc = S[ch], *Vc = V[ch];
    float tr2 = 0.f;
    for (int k = 0; k < kKltN; ++k) tr2 += Sc[k * kKltN + k] * Sc[k * kKltN + k];
    for (int sweep = 0; sweep < 30; ++sweep) {
        float off = 0.f;
        for (int p = 0; p < kKltN; ++p)
            for (int q = p + 1; q < kKltN; ++q) off += Sc[p * kKltN + q] * Sc[p * kKltN + q];
        if (!(off > 1e-14f * tr2)) break;
        for (int p = 0; p < kKltN; ++p)
            for (int q = p + 1; q < kKltN; ++q) {
                if (lane == 0) {
                    const float apq = Sc[p * kKltN + q];
                    float c = 1.f, s = 0.f;
                    if (fabsf(apq) > 1e-30f) {
                        const float theta = (Sc[q * kKltN + q] - Sc[p * kKltN + p]) / (2.f * apq);
                        const float tt = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
                        c = 1.f / sqrtf(tt * tt + 1.f);
                        s = tt * c;
                    }
                    cs[ch][0] = c;
                    cs[ch][1] = s;
                }
                __syncwarp();
                const float c = cs[ch][0], s = cs[ch][1];
                if (s != 0.f) {
                    if (lane < kKltN) {  // columns p, q
                        const float skp = Sc[lane * kKltN + p], skq = Sc[lane * kKltN + q];
                        Sc[lane * kKltN + p] = c * skp - s * skq;
                        Sc[lane * kKltN + q] = s * skp + c * skq;
                    }
                    __syncwarp();
                    if (lane < kKltN) {  // rows p, q; eigenvector columns
                        const float spk = Sc[p * kKltN + lane], sqk = Sc[q * kKltN + lane];
                        Sc[p * kKltN + lane] = c * spk - s * sqk;
                        Sc[q * kKltN + lane] = s * spk + c * sqk;
                        const float vkp = Vc[lane * kKltN + p], vkq = Vc[lane * kKltN + q];
                        Vc[lane * kKltN + p] = c * vkp - s * vkq;
                        Vc[lane * kKltN + q] = s * vkp + c * vkq;
                    }
                }
                __syncwarp();
            }
    }
    if (lane == 0) {  // decreasing eigenvalue, stable
        for (int k = 0; k < kKltN; ++k) order[ch][k] = k;
        for (int x = 0; x < kKltN; ++x)
            for (int y = x + 1; y < kKltN; ++y)
                if (Sc[order[ch][y] * kKltN + order[ch][y]] > Sc[order[ch][x] * kKltN + order[ch][x]]) {
                    const int tmp = order[ch][x];
                    order[ch][x] = order[ch][y];
                    order[ch][y] = tmp;
                }
    }
    __syncwarp();
    float *Kf = klt + (uint64_t)f * kKltFloats + ch * kKltN * kKltN;
    if (lane < kKltN) {
        const int e = order[ch][lane];
        int big = 0;
        for (int k = 1; k < kKltN; ++k)
            if (fabsf(Vc[k * kKltN + e]) > fabsf(Vc[big * kKltN + e])) big = k;
        const float sg = Vc[big * kKltN + e] < 0.f ? -1.f : 1.f;
        for (int k = 0; k < kKltN; ++k) Kf[lane * kKltN + k] = sg * Vc[k * kKltN + e];
    }
    __syncthreads();
    if (t == 0 && center) color_forward_row(center + (uint64_t)f * 56, klt + (uint64_t)f * kKltFloats);
}

}  // namespace

YuvInv yuv_inverse()
{
    const double m[3][3] = {{0.299, 0.587, 0.114}, {-0.14713, -0.28886, 0.436}, {0.615, -0.51499, -0.10001}};
    const double det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
                       m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                       m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    const double inv[9] = {(m[1][1] * m[2][2] - m[1][2] * m[2][1]) / det, (m[0][2] * m[2][1] - m[0][1] * m[2][2]) / det,
                           (m[0][1] * m[1][2] - m[0][2] * m[1][1]) / det, (m[1][2] * m[2][0] - m[1][0] * m[2][2]) / det,
                           (m[0][0] * m[2][2] - m[0][2] * m[2][0]) / det, (m[0][2] * m[1][0] - m[0][0] * m[1][2]) / det,
                           (m[1][0] * m[2][1] - m[1][1] * m[2][0]) / det, (m[0][1] * m[2][0] - m[0][0] * m[2][1]) / det,
                           (m[0][0] * m[1][1] - m[0][1] * m[1][0]) / det};
    YuvInv r;
    for (int i = 0; i < 9; ++i) r.m[i] = (float)inv[i];
    return r;
}

uint64_t color_klt_partial_words(uint32_t F) { return (uint64_t)F * kSlices * kPartWords; }

void launch_color_klt(const float *const *attr, const uint64_t *poff, uint32_t F, float *klt, float *center,
                      double *partials, cudaStream_t s)
{
    if (F == 0) return;
    klt_partials_kernel<<<dim3(kSlices, F), 96, 0, s>>>(attr, poff, partials);
    count_launch();
    klt_solve_kernel<<<F, 96, 0, s>>>(poff, partials, klt, center);
    count_launch();
}

}  // namespace gsnfs
