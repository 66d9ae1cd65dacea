// Splat rasteriser for rendered-view quality of decoded frames (the standard
// 3DGS forward pass, from its definition): per Gaussian, the projected mean,
// the EWA 2-D covariance J R S S^T R^T J^T + 0.3 I and its inverse (conic),
// a footprint square of radius ceil(3 sqrt(largest eigenvalue)), opacity
// sigmoid(logit) and a degree-3 real-SH colour at the viewing direction; one
// key per overlapped 16 x 16 tile, (tile << 32 | depth bits), sorted stably
// (so a tile's list is by depth, then input index); one CTA per tile
// composites its list front to back for its 256 pixels.  Attributes are the
// 56-channel 3DGS rows: log-scale 0-2, rotation (w, x, y, z) 3-6, opacity
// logit 7, SH DC RGB 8-10, SH AC 11-55 as R[15] G[15] B[15].
//
// Precision: everything per Gaussian (projection, covariance, conic, tile
// rectangle, opacity, colour) is evaluated in FP64 and rounded once to FP32
// for the per-pixel loop, which runs in FP32.  The projected centre is kept
// as an unevaluated sum of two floats, so a pixel's offset from it is exact
// to FP32 rounding of the offset itself (a single float would carry an
// absolute error of its ulp at hundreds of pixels).  The conic enters the
// loop through its Cholesky factor, conic = L^T L with
// L = [[l1, l2], [0, l3]]: the exponent is -(|L d|^2) / 2, a sum of two
// squares, which FP32 evaluates without cancellation even for elongated
// footprints.
#include "kernels.cuh"

namespace gsnfs {

namespace {

constexpr int kTile = 16;

struct Splat {
    float u, ulo, v, vlo;  // projected centre as hi + lo
    float l1, l2, l3;      // Cholesky factor of the conic
    float opacity, r, g, b;
    float pad;
};

__device__ __forceinline__ void sh_basis_d(double x, double y, double z, double Y[16])
{
    const double pi = 3.14159265358979323846;
    const double c0 = 0.5 / sqrt(pi), c1 = sqrt(3.0 / (4.0 * pi));
    const double c2a = 0.5 * sqrt(15.0 / pi), c2b = 0.25 * sqrt(5.0 / pi), c2c = 0.25 * sqrt(15.0 / pi);
    const double c3a = 0.25 * sqrt(35.0 / (2.0 * pi)), c3b = 0.5 * sqrt(105.0 / pi);
    const double c3c = 0.25 * sqrt(21.0 / (2.0 * pi)), c3d = 0.25 * sqrt(7.0 / pi), c3e = 0.25 * sqrt(105.0 / pi);
    Y[0] = c0;
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    Y[4] = c2a * x * y;
    Y[5] = -c2a * y * z;
    Y[6] = c2b * (2.0 * z * z - x * x - y * y);
    Y[7] = -c2a * x * z;
    Y[8] = c2c * (x * x - y * y);
    Y[9] = -c3a * y * (3.0 * x * x - y * y);
    Y[10] = c3b * x * y * z;
    Y[11] = -c3c * y * (4.0 * z * z - x * x - y * y);
    Y[12] = c3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    Y[13] = -c3c * x * (4.0 * z * z - x * x - y * y);
    Y[14] = c3e * z * (x * x - y * y);
    Y[15] = -c3a * x * (x * x - 3.0 * y * y);
}

__global__ void __launch_bounds__(256) preprocess_kernel(const float *__restrict__ pos,
                                                         const float *__restrict__ attr, uint64_t n, RenderCam cam,
                                                         Splat *sp, float *depth, int4 *rect, uint32_t *count)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        count[i] = 0;
        const float *p = pos + 3 * i, *a = attr + 56 * i;
        double pc[3];
        for (int r = 0; r < 3; ++r)
            pc[r] = cam.R[3 * r] * (double)p[0] + cam.R[3 * r + 1] * (double)p[1] + cam.R[3 * r + 2] * (double)p[2] +
                    cam.t[r];
        const double z = pc[2];
        if (!(z > cam.znear)) continue;
        double qw = a[3], qx = a[4], qy = a[5], qz = a[6];
        double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
        if (!(qn > 0.0)) {
            qw = 1.0;
            qx = qy = qz = 0.0;
            qn = 1.0;
        }
        const double w = qw / qn, x = qx / qn, y = qy / qn, zq = qz / qn;
        const double Rq[9] = {1 - 2 * (y * y + zq * zq), 2 * (x * y - w * zq), 2 * (x * zq + w * y),
                              2 * (x * y + w * zq), 1 - 2 * (x * x + zq * zq), 2 * (y * zq - w * x),
                              2 * (x * zq - w * y), 2 * (y * zq + w * x), 1 - 2 * (x * x + y * y)};
        const double sc[3] = {exp((double)a[0]), exp((double)a[1]), exp((double)a[2])};
        double M[9], S[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * sc[c];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) S[3 * r + c] = M[3 * r] * M[3 * c] + M[3 * r + 1] * M[3 * c + 1] + M[3 * r + 2] * M[3 * c + 2];
        const double J[6] = {cam.fx / z, 0.0, -cam.fx * pc[0] / (z * z), 0.0, cam.fy / z, -cam.fy * pc[1] / (z * z)};
        double T[6], TS[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c)
                T[3 * r + c] = J[3 * r] * cam.R[c] + J[3 * r + 1] * cam.R[3 + c] + J[3 * r + 2] * cam.R[6 + c];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) TS[3 * r + c] = T[3 * r] * S[c] + T[3 * r + 1] * S[3 + c] + T[3 * r + 2] * S[6 + c];
        const double ca = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + 0.3;
        const double cb = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
        const double cc = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + 0.3;
        const double det = ca * cc - cb * cb;
        if (!(det > 0.0)) continue;
        // conic Q = [[cc, -cb], [-cb, ca]] / det; Q = L^T L with L = [[l1, l2], [0, l3]]
        const double q00 = cc / det, q01 = -cb / det;
        const double l1 = sqrt(q00), l2 = q01 / l1, l3 = sqrt(1.0 / (det * q00));  // det(Q) = 1 / det
        const double mid = 0.5 * (ca + cc);
        const double disc = mid * mid - det;
        const double lmax = mid + sqrt(disc > 0.1 ? disc : 0.1);
        const double rad = ceil(3.0 * sqrt(lmax));
        const double u = cam.fx * pc[0] / z + cam.cx, v = cam.fy * pc[1] / z + cam.cy;
        int tx0 = (int)floor((u - rad) / kTile), tx1 = (int)floor((u + rad) / kTile);
        int ty0 = (int)floor((v - rad) / kTile), ty1 = (int)floor((v + rad) / kTile);
        tx0 = max(tx0, 0);
        ty0 = max(ty0, 0);
        tx1 = min(tx1, cam.TX - 1);
        ty1 = min(ty1, cam.TY - 1);
        if (tx0 > tx1 || ty0 > ty1) continue;
        Splat s;
        s.u = (float)u;
        s.ulo = (float)(u - (double)s.u);
        s.v = (float)v;
        s.vlo = (float)(v - (double)s.v);
        s.l1 = (float)l1;
        s.l2 = (float)l2;
        s.l3 = (float)l3;
        s.opacity = (float)(1.0 / (1.0 + exp(-(double)a[7])));
        double d[3] = {(double)p[0] - cam.campos[0], (double)p[1] - cam.campos[1], (double)p[2] - cam.campos[2]};
        const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const double id = dn > 0.0 ? 1.0 / dn : 1.0;
        double Y[16];
        sh_basis_d(d[0] * id, d[1] * id, d[2] * id, Y);
        float col[3];
        for (int c = 0; c < 3; ++c) {
            double val = Y[0] * (double)a[8 + c];
            for (int k = 1; k < 16; ++k) val += Y[k] * (double)a[11 + 15 * c + (k - 1)];
            val += 0.5;
            col[c] = val > 0.0 ? (float)val : 0.f;
        }
        s.r = col[0];
        s.g = col[1];
        s.b = col[2];
        s.pad = 0.f;
        sp[i] = s;
        depth[i] = (float)z;
        rect[i] = make_int4(tx0, tx1, ty0, ty1);
        count[i] = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
    }
}

__global__ void emit_kernel(uint64_t n, const int4 *rect, const float *depth, const uint32_t *count,
                            const uint64_t *offs, int TX, uint64_t *keys, uint32_t *vals)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (!count[i]) continue;
        const int4 r = rect[i];
        const uint32_t db = __float_as_uint(depth[i]);  // positive: integer order = float order
        uint64_t o = offs[i];
        for (int ty = r.z; ty <= r.w; ++ty)
            for (int tx = r.x; tx <= r.y; ++tx) {
                keys[o] = ((uint64_t)(uint32_t)(ty * TX + tx) << 32) | db;
                vals[o] = (uint32_t)i;
                ++o;
            }
    }
}

__global__ void ranges_kernel(const uint64_t *keys, uint64_t total, uint2 *ranges)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t tile = (uint32_t)(keys[i] >> 32);
        if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != tile) ranges[tile].x = (uint32_t)i;
        if (i + 1 == total || (uint32_t)(keys[i + 1] >> 32) != tile) ranges[tile].y = (uint32_t)(i + 1);
    }
}

// one CTA per tile, thread per pixel; the tile's splats in batches of 256 through shared memory
__global__ void __launch_bounds__(256) render_kernel(const uint2 *ranges, const uint32_t *vals, const Splat *sp,
                                                     RenderCam cam, float *image)
{
    __shared__ Splat batch[256];
    const int tx = blockIdx.x, ty = blockIdx.y;
    const int lx = threadIdx.x & 15, ly = threadIdx.x >> 4;
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool inside = px < cam.W && py < cam.H;
    const uint2 rg = ranges[ty * cam.TX + tx];
    const float fxp = px + 0.5f, fyp = py + 0.5f;
    float T = 1.f, col[3] = {0.f, 0.f, 0.f};
    bool done = !inside;
    for (uint32_t b0 = rg.x; b0 < rg.y; b0 += 256) {
        if (__syncthreads_count(done ? 0 : 1) == 0) break;  // every pixel of the tile has finished
        const uint32_t k = b0 + threadIdx.x;
        if (k < rg.y) batch[threadIdx.x] = sp[vals[k]];
        __syncthreads();
        const uint32_t cnt = (rg.y - b0) < 256u ? (rg.y - b0) : 256u;
        for (uint32_t j = 0; j < cnt && !done; ++j) {
            const Splat s = batch[j];
            const float dx = (s.u - fxp) + s.ulo, dy = (s.v - fyp) + s.vlo;
            const float e0 = fmaf(s.l1, dx, s.l2 * dy), e1 = s.l3 * dy;
            const float power = -0.5f * fmaf(e0, e0, e1 * e1);
            const float alpha = fminf(0.99f, s.opacity * expf(power));
            if (alpha < 1.f / 255.f) continue;
            const float tn = T * (1.f - alpha);
            if (tn < 1e-4f) {
                done = true;
                break;
            }
            col[0] += s.r * alpha * T;
            col[1] += s.g * alpha * T;
            col[2] += s.b * alpha * T;
            T = tn;
        }
    }
    if (inside)
        for (int c = 0; c < 3; ++c) image[((uint64_t)py * cam.W + px) * 3 + c] = col[c] + T * cam.bg[c];
}

uint32_t rgrid(uint64_t n, int num_sms)
{
    uint64_t b = (n + 255) / 256;
    const uint64_t cap = (uint64_t)num_sms * 8;
    return (uint32_t)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

size_t render_splat_bytes() { return sizeof(Splat); }

void launch_render_prepare(const float *pos, const float *attr, uint64_t n, const RenderCam &cam, void *splats,
                           float *depth, int4 *rect, uint32_t *count, uint64_t *offs, uint64_t *partials,
                           int num_sms, cudaStream_t s)
{
    preprocess_kernel<<<rgrid(n, num_sms), 256, 0, s>>>(pos, attr, n, cam, (Splat *)splats, depth, rect, count);
    count_launch();
    launch_scan_u32_to_u64(count, n, offs, partials, num_sms, s);
}

void launch_render_tiles(uint64_t n, const int4 *rect, const float *depth, const uint32_t *count,
                         const uint64_t *offs, uint64_t total, const RenderCam &cam, const void *splats,
                         uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint32_t *hist,
                         uint2 *ranges, float *image, int num_sms, cudaStream_t s)
{
    const uint32_t tiles = (uint32_t)(cam.TX * cam.TY);
    dev_memset(ranges, 0, sizeof(uint2) * tiles, s);
    if (total) {
        emit_kernel<<<rgrid(n, num_sms), 256, 0, s>>>(n, rect, depth, count, offs, cam.TX, keys, vals);
        count_launch();
        uint32_t tb = 0;
        while ((1u << tb) < tiles) ++tb;
        const bool alt = radix_sort(keys, vals, keys_alt, vals_alt, hist, total, 32 + tb, num_sms, s);
        const uint64_t *sk = alt ? keys_alt : keys;
        const uint32_t *sv = alt ? vals_alt : vals;
        ranges_kernel<<<rgrid(total, num_sms), 256, 0, s>>>(sk, total, ranges);
        count_launch();
        render_kernel<<<dim3(cam.TX, cam.TY), 256, 0, s>>>(ranges, sv, (const Splat *)splats, cam, image);
    } else {
        render_kernel<<<dim3(cam.TX, cam.TY), 256, 0, s>>>(ranges, vals, (const Splat *)splats, cam, image);
    }
    count_launch();
}

}  // namespace gsnfs
