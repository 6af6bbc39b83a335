// Bounds checks of the indices the kernels read from device data (topics in z
// and in the per-word tables).  A build with -DPULDA_CHECKED replaces such an
// index outside [0, n) by 0, so the access stays in bounds, and sets
// ERR_BOUNDS in the chain's error word, which pulda_sync reports; without it
// the index is used as it is (host validation keeps the inputs in range and
// the kernels write only topics below K).  compute-sanitizer is not
// available here, so the checked build plus the oracle lockstep tests stand in
// for it.
#pragma once
#include <cstdint>

#include "pulda_internal.h"

namespace pulda {

__device__ __forceinline__ int guard_index(int i, int n, unsigned long long *stats) {
#ifdef PULDA_CHECKED
    if (static_cast<unsigned>(i) >= static_cast<unsigned>(n)) {
        atomicOr(&stats[ST_ERROR], ERR_BOUNDS);
        return 0;
    }
#else
    (void)n;
    (void)stats;
#endif
    return i;
}

}  // namespace pulda
