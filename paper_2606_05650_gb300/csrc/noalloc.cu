// Allocation-free variant of the octree occupancy encoder (gsnfs_octree_encode).
//
// Some callers cannot let a library allocate device memory once they are
// running: hosts that hand all device memory to their own pool at start-up
// and forbid cudaMalloc afterwards, and real-time loops that cannot afford the
// device-wide synchronisation and driver locks that cudaMalloc / cudaFree may
// take.  For them this file keeps the scratch that the occupancy kernels need
// in one fixed file-scope device array, reserved when the library is loaded,
// so the call below allocates nothing.  The caller still provides the input
// codes and the output byte buffer.
//
// The array is shared by every call on a device and keeps whatever the last
// call left in it; each call re-initialises the parts that must start at zero
// before its kernels run.  Calls that overlap on the GPU (on different
// streams, or from different host threads) use the same array and race:
// serialise them.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/gsnfs.h"
#include "kernels.cuh"
#include "status.cuh"

using namespace gsnfs;

namespace {

constexpr uint64_t kMaxVoxels = GSNFS_STATIC_MAX_VOXELS;
constexpr int kMaxSms = 256;  // bound on SMs used to size the per-CTA partial counts
constexpr size_t kStatePart = (sizeof(DevState) + 255) & ~(size_t)255;
constexpr size_t kSmallPart = 1024;                        // vstart, J, level sizes, height offsets, byte offsets
constexpr size_t kPartials = (size_t)occupancy_partial_words_one_frame(kMaxSms) * 4 + 256;  // per-CTA height counts
constexpr size_t kScratchBytes = kStatePart + kSmallPart + kPartials + ((kMaxVoxels + 2 + 255) & ~(uint64_t)255);

// Every GPU that loads the library holds this array (about 1.3 MB) until exit.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

struct DeviceScratch {
    bool ready = false;
    unsigned char *base = nullptr;  // device address of g_static_scratch on this device
    int sms = 0;
};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
DeviceScratch g_dev[kMaxDevices];

// Once per device, with that device current: the device address of the
// array (in host code its name is only a host-side stand-in).
gsnfs_status scratch_for_current_device(DeviceScratch **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GSNFS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceScratch &d = g_dev[dev];
    if (!d.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return GSNFS_ERR_CUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GSNFS_ERR_CUDA;
        if (sms > kMaxSms) sms = kMaxSms;
        d.base = (unsigned char *)p;
        d.sms = sms;
        d.ready = true;
    }
    *out = &d;
    return GSNFS_OK;
}

// Resets the words that must start at zero and stores the frame description.
__global__ void static_init_kernel(DevState *st, uint32_t *vstart, uint32_t *Jd, uint32_t nv, uint32_t J)
{
    if (threadIdx.x == 0) {
        st->err = 0;
        st->err_info = 0;
        vstart[0] = 0;
        vstart[1] = nv;
        Jd[0] = J;
    }
}

}  // namespace

extern "C" gsnfs_status gsnfs_octree_encode_static(void *stream, const uint64_t *d_codes, uint64_t nv, uint32_t J,
                                                   uint8_t *d_occ, uint64_t occ_capacity,
                                                   uint32_t *h_level_sizes, uint64_t *out_occ_bytes)
{
    if (J < 1 || J > (uint32_t)kMaxJ || !h_level_sizes || (nv && !d_codes) || (occ_capacity && !d_occ))
        return GSNFS_ERR_INVALID_ARG;
    if ((uintptr_t)d_occ % 4) return GSNFS_ERR_INVALID_ARG;
    if (nv > kMaxVoxels) return GSNFS_ERR_UNSUPPORTED;  // beyond the fixed scratch: use gsnfs_octree_encode
    DeviceScratch *ds = nullptr;
    gsnfs_status st = scratch_for_current_device(&ds);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // A launch error left pending by the caller's earlier work would otherwise
    // be read below as this call's own; clear it before launching.
    (void)cudaGetLastError();
    unsigned char *b = ds->base;
    DevState *dst = (DevState *)b;
    unsigned char *small = b + kStatePart;
    uint32_t *vstart = (uint32_t *)(small + 0);
    uint32_t *Jd = (uint32_t *)(small + 16);
    uint32_t *lsz = (uint32_t *)(small + 64);
    uint32_t *hoff = (uint32_t *)(small + 64 + 22 * 4);
    uint64_t *occ_off = (uint64_t *)(small + 256);
    uint32_t *partials = (uint32_t *)(b + kStatePart + kSmallPart);
    uint8_t *gap = b + kStatePart + kSmallPart + kPartials;

    static_init_kernel<<<1, 32, 0, s>>>(dst, vstart, Jd, (uint32_t)nv, J);
    launch_gap_levels(d_codes, nv, gap, s);
    OccupancyOut oo{d_occ, occ_capacity & ~(uint64_t)3, lsz, occ_off, hoff, partials};
    launch_occupancy(d_codes, gap, vstart, Jd, 1, 64, oo, dst, ds->sms, s);
    if (cudaGetLastError() != cudaSuccess) return GSNFS_ERR_CUDA;

    uint32_t h_lsz[22];
    uint64_t h_off[2];
    uint32_t h_err = 0;
    if (cudaMemcpyAsync(h_lsz, lsz, sizeof(h_lsz), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(h_off, occ_off, sizeof(h_off), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&h_err, &dst->err, sizeof(h_err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GSNFS_ERR_CUDA;
    for (uint32_t d = 0; d <= J; ++d) h_level_sizes[d] = h_lsz[d];
    if (out_occ_bytes) *out_occ_bytes = h_off[1];
    if (h_off[1] > occ_capacity) return GSNFS_ERR_CAPACITY;
    return map_dev_error(h_err);
}
