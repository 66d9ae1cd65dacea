// KLT of the SH colour decorrelation (Sec. 4): per frame, the covariance of
// each YUV channel's 15 AC values over the frame's first (up to 4096) input
// points, in FP64; its eigenvectors by cyclic Jacobi rotations (one warp per
// channel, lanes over the matrix columns); rows of K = eigenvectors by
// decreasing eigenvalue, the largest component of each made positive.  The
// frame's centring constants are then carried into the same domain.
#include "color.cuh"
#include "kernels.cuh"

namespace gsnfs {

namespace {

constexpr int kSample = 4096;
constexpr int kRowsPerChunk = 32;

__device__ __forceinline__ void yuv3d(double &a, double &b, double &c)
{
    const double x = a, y = b, z = c;
    a = 0.299 * x + 0.587 * y + 0.114 * z;
    b = -0.14713 * x - 0.28886 * y + 0.436 * z;
    c = 0.615 * x - 0.51499 * y - 0.10001 * z;
}

// one CTA (3 warps) per frame
__global__ void __launch_bounds__(96) klt_kernel(const float *const *attr, const uint64_t *poff, float *klt,
                                                 float *center)
{
    __shared__ double rows[kRowsPerChunk][48];  // SH values of a chunk of rows, YUV per function
    __shared__ double S[3][kKltN * kKltN];
    __shared__ double V[3][kKltN * kKltN];
    __shared__ double mu[3][kKltN];
    __shared__ double cs[3][2];
    __shared__ int order[3][kKltN];
    const uint32_t f = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, ch = t >> 5;
    const uint64_t n = poff[f + 1] - poff[f];
    const int m = (int)(n < (uint64_t)kSample ? n : (uint64_t)kSample);
    const float *a = attr[f];
    // covariance accumulators: lane owns pairs (x, y) = p, p + 32, ... of the 120 with x <= y, and mean lane
    double acc[4] = {0, 0, 0, 0}, sum = 0.0;
    int px[4], py[4];
    for (int j = 0; j < 4; ++j) {
        int p = lane + 32 * j, x = 0;
        while (p >= kKltN - x && x < kKltN) {
            p -= kKltN - x;
            ++x;
        }
        px[j] = x;
        py[j] = x + p;
    }
    for (int r0 = 0; r0 < m; r0 += kRowsPerChunk) {
        const int cnt = (m - r0) < kRowsPerChunk ? (m - r0) : kRowsPerChunk;
        for (int e = t; e < cnt * 16; e += blockDim.x) {  // (row, SH function): load RGB, store YUV
            const int r = e >> 4, k = e & 15;
            const float *row = a + (uint64_t)(r0 + r) * 56;
            double y0 = row[sh_chan(k, 0)], y1 = row[sh_chan(k, 1)], y2 = row[sh_chan(k, 2)];
            yuv3d(y0, y1, y2);
            rows[r][k * 3 + 0] = y0;
            rows[r][k * 3 + 1] = y1;
            rows[r][k * 3 + 2] = y2;
        }
        __syncthreads();
        for (int r = 0; r < cnt; ++r) {
            const double *rr = rows[r];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (lane + 32 * j < 120) acc[j] += rr[(px[j] + 1) * 3 + ch] * rr[(py[j] + 1) * 3 + ch];
            if (lane < kKltN) sum += rr[(lane + 1) * 3 + ch];
        }
        __syncthreads();
    }
    const double inv_m = m ? 1.0 / (double)m : 0.0;
    if (lane < kKltN) mu[ch][lane] = sum * inv_m;
    __syncwarp();
    for (int j = 0; j < 4; ++j)
        if (lane + 32 * j < 120) {
            const double c = acc[j] * inv_m - mu[ch][px[j]] * mu[ch][py[j]];
            S[ch][px[j] * kKltN + py[j]] = c;
            S[ch][py[j] * kKltN + px[j]] = c;
        }
    if (lane < kKltN)
        for (int k = 0; k < kKltN; ++k) V[ch][lane * kKltN + k] = (lane == k) ? 1.0 : 0.0;
    __syncwarp();
    // cyclic Jacobi: rotation (p, q) zeroes S[p][q]; lanes update column / row k
    double *Sc = S[ch], *Vc = V[ch];
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < kKltN; ++p)
            for (int q = p + 1; q < kKltN; ++q) off += Sc[p * kKltN + q] * Sc[p * kKltN + q];
        if (off < 1e-30) break;
        for (int p = 0; p < kKltN; ++p)
            for (int q = p + 1; q < kKltN; ++q) {
                if (lane == 0) {
                    const double apq = Sc[p * kKltN + q];
                    double c = 1.0, s = 0.0;
                    if (fabs(apq) >= 1e-300) {
                        const double theta = (Sc[q * kKltN + q] - Sc[p * kKltN + p]) / (2.0 * apq);
                        const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(tt * tt + 1.0);
                        s = tt * c;
                    }
                    cs[ch][0] = c;
                    cs[ch][1] = s;
                }
                __syncwarp();
                const double c = cs[ch][0], s = cs[ch][1];
                if (s != 0.0) {
                    if (lane < kKltN) {  // columns p, q
                        const double skp = Sc[lane * kKltN + p], skq = Sc[lane * kKltN + q];
                        Sc[lane * kKltN + p] = c * skp - s * skq;
                        Sc[lane * kKltN + q] = s * skp + c * skq;
                    }
                    __syncwarp();
                    if (lane < kKltN) {  // rows p, q
                        const double spk = Sc[p * kKltN + lane], sqk = Sc[q * kKltN + lane];
                        Sc[p * kKltN + lane] = c * spk - s * sqk;
                        Sc[q * kKltN + lane] = s * spk + c * sqk;
                        const double vkp = Vc[lane * kKltN + p], vkq = Vc[lane * kKltN + q];
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
            if (fabs(Vc[k * kKltN + e]) > fabs(Vc[big * kKltN + e])) big = k;
        const double sg = Vc[big * kKltN + e] < 0 ? -1.0 : 1.0;
        for (int k = 0; k < kKltN; ++k) Kf[lane * kKltN + k] = (float)(sg * Vc[k * kKltN + e]);
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

void launch_color_klt(const float *const *attr, const uint64_t *poff, uint32_t F, float *klt, float *center,
                      cudaStream_t s)
{
    if (F == 0) return;
    klt_kernel<<<F, 96, 0, s>>>(attr, poff, klt, center);
    count_launch();
}

}  // namespace gsnfs
