// Exclusive prefix sums used to lay out variable-length outputs (block word
// offsets of the RLGR payload).  Reduce-then-scan: no CTA waits on another.
#include <algorithm>

#include "kernels.cuh"

namespace gsnfs {

namespace {

constexpr int kThreads = 256;

struct Geom {
    uint32_t P;
    uint64_t chunk;
};

Geom geom(uint64_t n, int num_sms)
{
    Geom g;
    uint64_t t = (n + 2047) / 2048;
    uint64_t pmax = (uint64_t)num_sms * 2;
    g.P = (uint32_t)(t < 1 ? 1 : (t < pmax ? t : pmax));
    g.chunk = (n + g.P - 1) / g.P;
    if (g.chunk == 0) g.chunk = 1;
    return g;
}

__global__ void __launch_bounds__(kThreads) up_kernel(const uint32_t *in, uint64_t n, uint64_t chunk, uint64_t *part)
{
    uint64_t b = (uint64_t)blockIdx.x * chunk, e = b + chunk;
    if (e > n) e = n;
    uint64_t s = 0;
    for (uint64_t i = b + threadIdx.x; i < e; i += kThreads) s += in[i];
    __shared__ uint64_t sh[33];
    uint64_t tot;
    block_exclusive_sum<uint64_t>(s, sh, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) mid_kernel(uint64_t *part, uint32_t P)
{
    __shared__ uint64_t sh[33];
    uint64_t v = (threadIdx.x < P) ? part[threadIdx.x] : 0ull;
    uint64_t tot;
    uint64_t pre = block_exclusive_sum<uint64_t>(v, sh, &tot);
    if (threadIdx.x < P) part[threadIdx.x] = pre;
    if (threadIdx.x == 0) part[P] = tot;
}

__global__ void __launch_bounds__(kThreads) down_kernel(const uint32_t *in, uint64_t n, uint64_t chunk,
                                                        const uint64_t *part, uint64_t *out)
{
    __shared__ uint64_t sh[33];
    uint64_t b = (uint64_t)blockIdx.x * chunk, e = b + chunk;
    if (e > n) e = n;
    uint64_t run = part[blockIdx.x];
    for (uint64_t t0 = b; t0 < e; t0 += kThreads) {
        uint64_t i = t0 + threadIdx.x;
        uint64_t v = (i < e) ? in[i] : 0ull;
        uint64_t tot;
        uint64_t pre = block_exclusive_sum<uint64_t>(v, sh, &tot);
        if (i < e) out[i] = run + pre;
        run += tot;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = part[gridDim.x];
}

}  // namespace

uint64_t scan_partial_words(uint64_t n, int num_sms) { return geom(n, num_sms).P + 1; }

void launch_scan_u32_to_u64(const uint32_t *in, uint64_t n, uint64_t *out, uint64_t *partials, int num_sms,
                            cudaStream_t s)
{
    Geom g = geom(n, num_sms);
    if (n == 0) {
        dev_memset(out, 0, sizeof(uint64_t), s);
        return;
    }
    up_kernel<<<g.P, kThreads, 0, s>>>(in, n, g.chunk, partials);
    count_launch();
    mid_kernel<<<1, 1024, 0, s>>>(partials, g.P);
    count_launch();
    down_kernel<<<g.P, kThreads, 0, s>>>(in, n, g.chunk, partials, out);
    count_launch();
}


// Device memset as a kernel (stream-ordered like cudaMemsetAsync, but never
// queued on a copy engine behind a caller's bulk copies in flight).
namespace {
__global__ void memset_kernel(unsigned char *p, uint32_t v4, unsigned char v, uint64_t n)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t head = (16 - ((uintptr_t)p & 15)) & 15;
    const uint64_t h = head < n ? head : n;
    for (uint64_t i = t; i < h; i += nt) p[i] = v;
    const uint64_t nvec = (n - h) / 16;
    uint4 *q = reinterpret_cast<uint4 *>(p + h);
    for (uint64_t i = t; i < nvec; i += nt) q[i] = make_uint4(v4, v4, v4, v4);
    for (uint64_t i = h + 16 * nvec + t; i < n; i += nt) p[i] = v;
}
}  // namespace

cudaError_t dev_memset(void *p, int value, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) return cudaSuccess;
    const unsigned char v = (unsigned char)value;
    const uint32_t v4 = 0x01010101u * v;
    const uint64_t units = (bytes + 15) / 16;
    const uint32_t blocks = (uint32_t)std::min<uint64_t>((units + 255) / 256, 1024);
    memset_kernel<<<blocks, 256, 0, s>>>(static_cast<unsigned char *>(p), v4, v, bytes);
    count_launch();
    return cudaGetLastError();
}

}  // namespace gsnfs
