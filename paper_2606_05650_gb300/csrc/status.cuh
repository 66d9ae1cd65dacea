// Mapping of the device-side error word (first error wins) to the C ABI's
// status codes, shared by every entry point that reads it back.
#pragma once

#include "../../include/gsnfs.h"
#include "common.cuh"

namespace gsnfs {

inline gsnfs_status map_dev_error(uint32_t e)
{
    switch (e) {
    case 0: return GSNFS_OK;
    case kErrCorrupt: return GSNFS_ERR_CORRUPT;
    case kErrCapacity: return GSNFS_ERR_CAPACITY;
    case kErrTimeout: return GSNFS_ERR_TIMEOUT;
    default: return GSNFS_ERR_CUDA;
    }
}

}  // namespace gsnfs
