// Fault-path checks (declared in lbm.h): lbm_debug_expire_halo_wait for the
// step kernel's bounded halo-copy wait, and lbm_debug_bounds_checked /
// lbm_debug_plant_bad_index for the bounds-checked library.
//
// The step kernel copies a tile's color/velocity halo with tiled TMA loads
// that complete on a shared-memory mbarrier, and waits for that barrier with
// mbar_wait, bounded by a time limit and a poll count.  When the wait gives
// up, the block sets the domain's timeout bit and the host reports
// LBM_ERR_TIMEOUT at the next synchronising call.  A copy that never lands
// cannot be produced on purpose without faulting the GPU, so this entry point
// reaches the same state safely: one block arms an mbarrier for bytes that no
// copy will deliver (mbarrier.arrive.expect_tx, and no TMA or bulk copy is
// ever issued), waits on it with the same mbar_wait and a short limit, sets
// the same bit and returns.  Nothing is in flight when the wait ends.
#include <cstdint>

#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_domain_access.h"
#include "lbm_kernels.cuh"

namespace {

using namespace lbmgpu;

constexpr unsigned kUndeliveredBytes = 4096;      // below the mbarrier's transaction-count limit

__global__ void __launch_bounds__(32) k_expire_halo_wait(int* err, uint64_t timeout_ns,
                                                         unsigned long long* waited_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    // the one expected arrival, plus a transaction count that no copy will pay off
    if (threadIdx.x == 0) mbar_expect_tx(&bar, kUndeliveredBytes);
    const uint64_t t0 = globaltimer_ns();
    const bool done = mbar_wait(&bar, 0, timeout_ns);
    const uint64_t t1 = globaltimer_ns();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!done) atomicOr(err, kErrCopyTimeout);
        if (waited_ns) *waited_ns = (unsigned long long)(t1 - t0);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_addr(&bar)) : "memory");
    }
}

}  // namespace

extern "C" lbm_status lbm_debug_expire_halo_wait(lbm_domain* dom, int64_t timeout_ns, int64_t* waited_ns) {
    if (!dom) return LBM_ERR_ARG;
    if (timeout_ns < 1000 || timeout_ns > 1000000000)
        return domain_fail(dom, LBM_ERR_ARG, "timeout_ns must lie in [1e3, 1e9]");
    if (domain_poisoned(dom))
        return domain_fail(dom, LBM_ERR_TIMEOUT, "the domain already saw a halo-copy timeout");
    const cudaStream_t s = domain_stream(dom);
    unsigned long long* d_waited = nullptr;
    if (waited_ns) {
        // the measured wait comes back through a small device buffer (a debug path, not a step)
        if (cudaMallocAsync((void**)&d_waited, sizeof(unsigned long long), s) != cudaSuccess) {
            cudaGetLastError();
            return domain_fail(dom, LBM_ERR_OOM, "cudaMallocAsync of 8 bytes failed");
        }
    }
    k_expire_halo_wait<<<1, 32, 0, s>>>(domain_error_flag(dom), (uint64_t)timeout_ns, d_waited);
    cudaError_t e = cudaGetLastError();
    if (waited_ns && e == cudaSuccess) {
        unsigned long long h = 0;
        e = cudaMemcpyAsync(&h, d_waited, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        *waited_ns = (int64_t)h;
    }
    if (d_waited) cudaFreeAsync(d_waited, s);
    if (e != cudaSuccess) return domain_fail(dom, LBM_ERR_CUDA, cudaGetErrorString(e));
    return LBM_OK;
}

// 1 in the library built with LBM_DEBUG_BOUNDS (liblbm_debug.so), else 0.
extern "C" int32_t lbm_debug_bounds_checked(void) { return kDebugBounds ? 1 : 0; }

extern "C" lbm_status lbm_debug_plant_bad_index(lbm_domain* dom, int32_t which) {
    if (!dom) return LBM_ERR_ARG;
    // Only the bounds-checked kernels test this index before using it; the
    // production kernels would read outside the color array, so there the
    // call refuses and writes nothing.
    if (!kDebugBounds)
        return domain_fail(dom, LBM_ERR_UNSUPPORTED, "only the bounds-checked library (liblbm_debug.so) takes this");
    if (which != 0) return domain_fail(dom, LBM_ERR_ARG, "which must be 0 (a ghost corner index)");
    if (domain_ghosts(dom) < 1) return domain_fail(dom, LBM_ERR_ARG, "the domain has no ghost nodes");
    // the first corner of ghost 0, pointed a few entries past the end of the color array
    const int32_t bad = (int32_t)(domain_plane(dom) + 7);
    const cudaError_t e = cudaMemcpyAsync(domain_ghost_corners(dom), &bad, sizeof(bad), cudaMemcpyHostToDevice,
                                          domain_stream(dom));
    if (e == cudaSuccess) {
        const cudaError_t e2 = cudaStreamSynchronize(domain_stream(dom));
        if (e2 != cudaSuccess) return domain_fail(dom, LBM_ERR_CUDA, cudaGetErrorString(e2));
        return LBM_OK;
    }
    return domain_fail(dom, LBM_ERR_CUDA, cudaGetErrorString(e));
}
