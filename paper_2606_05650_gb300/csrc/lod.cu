// Level of detail: a decoded frame reduced to the nodes of octree depth Jp
// (Algorithm 2's shift read as J - Jp).  A node is the run of voxels sharing
// code >> 3(J - Jp); it is placed at the centre of its cell at depth Jp and
// carries the mean of its voxels' decoded attributes, which by Eq. (1) is
// its RAHT low-pass coefficient divided by sqrt(voxel count).
#include "kernels.cuh"

namespace gsnfs {

namespace {

__global__ void lod_flags_kernel(const uint64_t *__restrict__ codes, uint64_t nv, uint32_t sh, uint32_t *flags)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (uint64_t)gridDim.x * blockDim.x)
        flags[i] = (i == 0 || (codes[i] >> sh) != (codes[i - 1] >> sh)) ? 1u : 0u;
}

__global__ void lod_starts_kernel(const uint32_t *__restrict__ flags, const uint64_t *__restrict__ offs, uint64_t nv,
                                  uint64_t *starts)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (uint64_t)gridDim.x * blockDim.x)
        if (flags[i]) starts[offs[i]] = i;
    if (blockIdx.x == 0 && threadIdx.x == 0) starts[offs[nv]] = nv;
}

// thread per (node, channel): FP64 mean over the node's voxels in voxel order;
// channel 0's thread also writes the node centre
__global__ void lod_nodes_kernel(const uint64_t *__restrict__ codes, const uint64_t *__restrict__ starts,
                                 const uint64_t *__restrict__ offs, uint64_t nv, uint32_t sh, uint32_t Jp,
                                 uint32_t C, const float *__restrict__ attr, LodGrid g, float *pos, float *out)
{
    const uint64_t nn = offs[nv];
    const uint32_t Cw = C ? C : 1;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn * Cw;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = t / Cw;
        const uint32_t c = (uint32_t)(t - k * Cw);
        const uint64_t b = starts[k], e = starts[k + 1];
        if (C && out) {
            double sum = 0.0;
            for (uint64_t i = b; i < e; ++i) sum = __dadd_rn(sum, (double)attr[i * C + c]);
            out[k * C + c] = (float)__ddiv_rn(sum, (double)(e - b));
        }
        if (c == 0 && pos) {
            const uint64_t m = codes[b] >> sh;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                uint32_t v = 0;
                for (uint32_t bit = 0; bit < Jp; ++bit) v |= (uint32_t)((m >> (3 * bit + a)) & 1u) << bit;
                const double off = __dmul_rn(__dadd_rn((double)v, 0.5), g.cell);
                pos[3 * k + a] = (float)__dadd_rn(g.lo[a], off);
            }
        }
    }
}

uint32_t lod_grid(uint64_t n, int num_sms)
{
    uint64_t b = (n + 255) / 256;
    const uint64_t cap = (uint64_t)num_sms * 8;
    return (uint32_t)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

void launch_lod_index(const uint64_t *codes, uint64_t nv, uint32_t sh, uint32_t *flags, uint64_t *offs,
                      uint64_t *partials, uint64_t *starts, int num_sms, cudaStream_t s)
{
    lod_flags_kernel<<<lod_grid(nv, num_sms), 256, 0, s>>>(codes, nv, sh, flags);
    count_launch();
    launch_scan_u32_to_u64(flags, nv, offs, partials, num_sms, s);
    lod_starts_kernel<<<lod_grid(nv, num_sms), 256, 0, s>>>(flags, offs, nv, starts);
    count_launch();
}

void launch_lod_nodes(const uint64_t *codes, const uint64_t *starts, const uint64_t *offs, uint64_t nv,
                      uint64_t n_nodes, uint32_t sh, uint32_t Jp, uint32_t C, const float *attr, const LodGrid &g,
                      float *pos, float *out, int num_sms, cudaStream_t s)
{
    lod_nodes_kernel<<<lod_grid(n_nodes * (C ? C : 1), num_sms), 256, 0, s>>>(codes, starts, offs, nv, sh, Jp, C,
                                                                               attr, g, pos, out);
    count_launch();
}

}  // namespace gsnfs
