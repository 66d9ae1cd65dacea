// Level of detail: a frame decoded to the nodes of octree depth Jp
// (Algorithm 2's shift read as J - Jp).  A node is the run of voxels sharing
// code >> 3(J - Jp); it is placed at the centre of its cell at depth Jp and
// carries the mean of its voxels' decoded attributes, which by Eq. (1) is
// its RAHT low-pass coefficient divided by sqrt(voxel count).  The low-pass
// coefficients come from an inverse RAHT over the node sequence (the
// butterflies inside nodes are never applied), which divides them as it
// stores them; this file builds the node sequence and the node centres.
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

// The nodes as the first pass of a coarser RAHT sequence: element k covers
// voxels [starts[k], starts[k + 1]) and follows a gap of the voxel sequence
// (the gap before its first voxel, above the depth's level, or a frame edge);
// sentinels after the last node.
__global__ void lod_sequence_kernel(const uint64_t *__restrict__ starts, const uint64_t *__restrict__ n_nodes_dev,
                                    uint64_t nv, const uint8_t *__restrict__ gap, uint32_t *pos0, uint32_t *end0,
                                    uint8_t *gap0)
{
    const uint64_t nn = *n_nodes_dev;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= nn; k += (uint64_t)gridDim.x * blockDim.x) {
        if (k < nn) {
            const uint64_t b = starts[k];
            pos0[k] = (uint32_t)b;
            end0[k] = (uint32_t)starts[k + 1];
            gap0[k] = k == 0 ? (uint8_t)kInfLevel : gap[b];
        } else {
            pos0[k] = (uint32_t)nv;
            gap0[k] = (uint8_t)kInfLevel;
        }
    }
}

// thread per node: its cell centre at depth Jp (the same FP64 expression as a voxel centre at that depth)
__global__ void lod_centres_kernel(const uint64_t *__restrict__ codes, const uint64_t *__restrict__ starts,
                                   const uint64_t *__restrict__ n_nodes_dev, uint32_t sh, uint32_t Jp, LodGrid g,
                                   float *pos)
{
    const uint64_t nn = *n_nodes_dev;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t m = codes[starts[k]] >> sh;
#pragma unroll
        for (uint32_t a = 0; a < 3; ++a) {
            uint32_t v = 0;
            for (uint32_t bit = 0; bit < Jp; ++bit) v |= (uint32_t)((m >> (3 * bit + a)) & 1u) << bit;
            const double off = __dmul_rn(__dadd_rn((double)v, 0.5), g.cell);
            pos[3 * k + a] = (float)__dadd_rn(g.lo[a], off);
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

void launch_lod_sequence(const uint64_t *starts, const uint64_t *n_nodes_dev, uint64_t nv, uint64_t n_nodes,
                         const uint8_t *gap, uint32_t *pos0, uint32_t *end0, uint8_t *gap0, int num_sms,
                         cudaStream_t s)
{
    lod_sequence_kernel<<<lod_grid(n_nodes + 1, num_sms), 256, 0, s>>>(starts, n_nodes_dev, nv, gap, pos0, end0, gap0);
    count_launch();
}

void launch_lod_centres(const uint64_t *codes, const uint64_t *starts, const uint64_t *n_nodes_dev, uint64_t n_nodes,
                        uint32_t sh, uint32_t Jp, const LodGrid &g, float *pos, int num_sms, cudaStream_t s)
{
    if (!pos) return;
    lod_centres_kernel<<<lod_grid(n_nodes, num_sms), 256, 0, s>>>(codes, starts, n_nodes_dev, sh, Jp, g, pos);
    count_launch();
}

}  // namespace gsnfs
