// KLT of the SH colour decorrelation (Sec. 4): per frame, the covariance of
// each YUV channel's 15 AC values over the frame's first (up to 4096) input
// points, and its eigenvectors; rows of K = eigenvectors by decreasing
// eigenvalue, the largest component of each made positive.  Everything here
// is FP64 (the sample is 4096 rows, so this costs next to nothing): the YUV
// values of the sample, per-slice means and centred co-moments (64 slices of
// 64 rows, one CTA each), the slices combined in a fixed order by the
// pairwise update of Chan, Golub and LeVeque, and cyclic Jacobi rotations
// (one warp per channel, seven disjoint rotations at a time).  K is rounded to
// FP32 once, for the header and the per-row transforms.  The frame's
// centring constants are then carried into the same domain.
#include "color.cuh"
#include "kernels.cuh"

namespace gsnfs {

namespace {

constexpr int kSample = 4096;
constexpr int kSlices = 64;                   // CTAs per frame for the sample sums
constexpr int kSliceRows = kSample / kSlices;  // 64
constexpr int kRowsPerChunk = 32;
constexpr int kPairs = kKltN * (kKltN + 1) / 2;  // 120
constexpr int kPartWords = 3 * (kPairs + kKltN) + 1;  // per slice: co-moments, then means, per channel; row count

__device__ __forceinline__ void pair_of(int p, int &x, int &y)
{
    x = 0;
    while (x < kKltN && p >= kKltN - x) {
        p -= kKltN - x;
        ++x;
    }
    y = x + p;
}

// BT.601 analogue YUV of one SH function's RGB in FP64, each product and sum
// rounded separately (the order of the definition: m0 x + m1 y + m2 z)
__device__ __forceinline__ void yuv3_f64(const float *row, int k, double out[3])
{
    const double M[9] = {0.299, 0.587, 0.114, -0.14713, -0.28886, 0.436, 0.615, -0.51499, -0.10001};
    const double x = row[sh_chan(k, 0)], y = row[sh_chan(k, 1)], z = row[sh_chan(k, 2)];
    for (int r = 0; r < 3; ++r)
        out[r] = __dadd_rn(__dadd_rn(__dmul_rn(M[3 * r], x), __dmul_rn(M[3 * r + 1], y)), __dmul_rn(M[3 * r + 2], z));
}

// grid (slices, frames), 3 warps (YUV channels): the mean and the centred
// co-moments (sums of products of deviations) of one slice of the frame's
// first 4096 input rows, in two passes over the slice
__global__ void __launch_bounds__(96) klt_partials_kernel(const float *const *attr, const uint64_t *poff,
                                                          double *part)
{
    __shared__ double rows[kRowsPerChunk][48];  // YUV of the 16 SH functions of a chunk of rows
    __shared__ double mean[3][kKltN];
    const uint32_t f = blockIdx.y, sl = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, ch = t >> 5;
    const uint64_t n = poff[f + 1] - poff[f];
    const int m = (int)(n < (uint64_t)kSample ? n : (uint64_t)kSample);
    const int rb = sl * kSliceRows, re = (rb + kSliceRows) < m ? (rb + kSliceRows) : m;
    const int cnt_rows = re > rb ? re - rb : 0;
    const float *a = attr[f];
    int px[4], py[4];
    for (int j = 0; j < 4; ++j) pair_of(lane + 32 * j, px[j], py[j]);
    double acc[4] = {0.0, 0.0, 0.0, 0.0}, sum = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int r0 = rb; r0 < re; r0 += kRowsPerChunk) {
            const int cnt = (re - r0) < kRowsPerChunk ? (re - r0) : kRowsPerChunk;
            for (int e = t; e < cnt * 16; e += blockDim.x) {
                const int r = e >> 4, k = e & 15;
                double y[3];
                yuv3_f64(a + (uint64_t)(r0 + r) * 56, k, y);
                rows[r][k * 3 + 0] = y[0];
                rows[r][k * 3 + 1] = y[1];
                rows[r][k * 3 + 2] = y[2];
            }
            __syncthreads();
            for (int r = 0; r < cnt; ++r) {
                const double *rr = rows[r];
                if (pass == 0) {
                    if (lane < kKltN) sum = __dadd_rn(sum, rr[(lane + 1) * 3 + ch]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (lane + 32 * j < kPairs) {
                            const double dx = __dsub_rn(rr[(px[j] + 1) * 3 + ch], mean[ch][px[j]]);
                            const double dy = __dsub_rn(rr[(py[j] + 1) * 3 + ch], mean[ch][py[j]]);
                            acc[j] = __dadd_rn(acc[j], __dmul_rn(dx, dy));
                        }
                }
            }
            __syncthreads();
        }
        if (pass == 0) {
            if (lane < kKltN) mean[ch][lane] = cnt_rows ? __ddiv_rn(sum, (double)cnt_rows) : 0.0;
            __syncthreads();
        }
    }
    double *ps = part + ((uint64_t)f * kSlices + sl) * kPartWords;
    double *o = ps + ch * (kPairs + kKltN);
    for (int j = 0; j < 4; ++j)
        if (lane + 32 * j < kPairs) o[lane + 32 * j] = acc[j];
    if (lane < kKltN) o[kPairs + lane] = mean[ch][lane];
    if (t == 0) ps[kPartWords - 1] = (double)cnt_rows;
}

// one CTA (3 warps) per frame: covariance from the slices (pairwise update,
// fixed order, FP64), eigenvectors by cyclic Jacobi (FP64, lanes over
// columns), ordering and signs; K rounded to FP32
__global__ void __launch_bounds__(96) klt_solve_kernel(const uint64_t *poff, const double *part, float *klt,
                                                       float *center)
{
    __shared__ double S[3][kKltN * kKltN];
    __shared__ double V[3][kKltN * kKltN];
    __shared__ double mu[3][kKltN];
    __shared__ double cs[3][7][2];
    __shared__ int pq[3][7][2];
    __shared__ int order[3][kKltN];
    const uint32_t f = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, ch = t >> 5;
    const uint64_t n = poff[f + 1] - poff[f];
    const int m = (int)(n < (uint64_t)kSample ? n : (uint64_t)kSample);
    const double *pf = part + (uint64_t)f * kSlices * kPartWords;
    // running combination over slices: count nA, mean muA (lane < 15), co-moments CA (4 pairs per lane)
    double nA = 0.0, muA = 0.0, CA[4] = {0.0, 0.0, 0.0, 0.0};
    int px[4], py[4];
    for (int j = 0; j < 4; ++j) pair_of(lane + 32 * j, px[j], py[j]);
    for (int sl = 0; sl < kSlices; ++sl) {
        const double *ps = pf + (uint64_t)sl * kPartWords;
        const double nB = ps[kPartWords - 1];
        if (nB == 0.0) continue;
        const double *o = ps + ch * (kPairs + kKltN);
        const double nAB = __dadd_rn(nA, nB);
        const double w = __ddiv_rn(__dmul_rn(nA, nB), nAB);
        // delta of the means for both coordinates of each pair (read from this slice's and the running means)
        if (lane < kKltN) mu[ch][lane] = __dsub_rn(o[kPairs + lane], muA);  // delta_k = muB_k - muA_k
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (lane + 32 * j < kPairs)
                CA[j] = __dadd_rn(__dadd_rn(CA[j], o[lane + 32 * j]),
                                  __dmul_rn(w, __dmul_rn(mu[ch][px[j]], mu[ch][py[j]])));
        if (lane < kKltN) muA = __dadd_rn(muA, __dmul_rn(mu[ch][lane], __ddiv_rn(nB, nAB)));
        nA = nAB;
        __syncwarp();
    }
    const double inv_m = m ? 1.0 / (double)m : 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (lane + 32 * j < kPairs) {
            const double c = __dmul_rn(CA[j], inv_m);
            S[ch][px[j] * kKltN + py[j]] = c;
            S[ch][py[j] * kKltN + px[j]] = c;
        }
    if (lane < kKltN)
        for (int k = 0; k < kKltN; ++k) V[ch][lane * kKltN + k] = (lane == k) ? 1.0 : 0.0;
    __syncwarp();
    double *Sc = S[ch], *Vc = V[ch];
    double tr2 = 0.0;
    for (int k = 0; k < kKltN; ++k) tr2 += Sc[k * kKltN + k] * Sc[k * kKltN + k];
    // Jacobi sweeps in parallel order: 15 rounds of 7 disjoint (p, q) pairs (a
    // round-robin over the 15 indices and one idle slot), the 7 rotations of a
    // round computed from the same S and applied together (they act on
    // disjoint rows and columns); every pair is met once per sweep.  Stop when
    // the off-diagonal mass is down to FP64 rounding of the diagonal.
    for (int sweep = 0; sweep < 20; ++sweep) {
        double off = 0.0;
        if (lane < kKltN)
            for (int q = lane + 1; q < kKltN; ++q) off += Sc[lane * kKltN + q] * Sc[lane * kKltN + q];
        for (int o = 16; o; o >>= 1) off += __shfl_xor_sync(0xFFFFFFFFu, off, o);
        if (!(off > 1e-28 * tr2)) break;
        for (int rd = 0; rd < kKltN; ++rd) {
            if (lane < 7) {
                const int a = (rd + lane + 1) % kKltN, b = (rd - lane - 1 + kKltN) % kKltN;
                const int p = a < b ? a : b, q = a < b ? b : a;
                const double apq = Sc[p * kKltN + q];
                double c = 1.0, sn = 0.0;
                if (fabs(apq) > 1e-300) {
                    const double theta = (Sc[q * kKltN + q] - Sc[p * kKltN + p]) / (2.0 * apq);
                    const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                    c = 1.0 / sqrt(tt * tt + 1.0);
                    sn = tt * c;
                }
                cs[ch][lane][0] = c;
                cs[ch][lane][1] = sn;
                pq[ch][lane][0] = p;
                pq[ch][lane][1] = q;
            }
            __syncwarp();
            if (lane < kKltN) {  // columns p, q of S and of V (lane = row)
                for (int i = 0; i < 7; ++i) {
                    const int p = pq[ch][i][0], q = pq[ch][i][1];
                    const double c = cs[ch][i][0], sn = cs[ch][i][1];
                    const double skp = Sc[lane * kKltN + p], skq = Sc[lane * kKltN + q];
                    Sc[lane * kKltN + p] = c * skp - sn * skq;
                    Sc[lane * kKltN + q] = sn * skp + c * skq;
                    const double vkp = Vc[lane * kKltN + p], vkq = Vc[lane * kKltN + q];
                    Vc[lane * kKltN + p] = c * vkp - sn * vkq;
                    Vc[lane * kKltN + q] = sn * vkp + c * vkq;
                }
            }
            __syncwarp();
            if (lane < kKltN) {  // rows p, q of S (lane = column)
                for (int i = 0; i < 7; ++i) {
                    const int p = pq[ch][i][0], q = pq[ch][i][1];
                    const double c = cs[ch][i][0], sn = cs[ch][i][1];
                    const double spk = Sc[p * kKltN + lane], sqk = Sc[q * kKltN + lane];
                    Sc[p * kKltN + lane] = c * spk - sn * sqk;
                    Sc[q * kKltN + lane] = sn * spk + c * sqk;
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
        const double sg = Vc[big * kKltN + e] < 0.0 ? -1.0 : 1.0;
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
