// Access to a domain's internals for the library's other translation units
// (the fault-path check in lbm_debug.cu); defined in lbm_api.cu.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "lbm.h"

namespace lbmgpu {

int* domain_error_flag(lbm_domain* d);          // device word of the domain's error bits
cudaStream_t domain_stream(lbm_domain* d);
bool domain_poisoned(const lbm_domain* d);
int32_t* domain_ghost_corners(lbm_domain* d);    // device [GK][n_ghosts] corner node indices
int64_t domain_ghosts(const lbm_domain* d);
int64_t domain_plane(const lbm_domain* d);      // entries of each device field
lbm_status domain_fail(lbm_domain* d, lbm_status s, const char* msg);   // records msg for lbm_last_error

}  // namespace lbmgpu
