// status.cuh -- the library status of a failed CUDA runtime call (host).
#pragma once
#include <cuda_runtime.h>

#include "ifa.h"

namespace ifa {

// A refused allocation is not sticky, but the runtime keeps it as the
// thread's last error, where the next launch check (cudaGetLastError)
// would report it again: clear it here.
inline ifa_status cuda_status(cudaError_t e) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? IFA_ERR_OOM : IFA_ERR_CUDA;
}

}  // namespace ifa
