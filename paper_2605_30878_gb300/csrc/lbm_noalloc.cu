// Allocation-free per-phase sums: lbm_phase_sums_noalloc (declared in lbm.h).
//
// Some callers cannot allocate device memory at the moment they need these
// sums: a host program whose device memory is entirely owned by its own pool
// allocator, a real-time loop that forbids allocation after start-up, or a
// plugin whose host application reserves every allocation for itself.  This
// entry point therefore takes the caller's device buffers for its inputs and
// output and keeps its only scratch -- one FP64 partial record per thread
// block -- in the file-scope array g_noalloc_scratch below, which every GPU
// that loads the library holds (64 KiB) until the process exits.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "lbm.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int64_t NA_NODES_PER_BLOCK = 16384;           // 64 nodes per thread
constexpr int NA_MAX_BLOCKS = 1024;
constexpr int NA_REC = 8;                                // fields of one partial record
constexpr int64_t NA_MAX_NODES = NA_NODES_PER_BLOCK * NA_MAX_BLOCKS;   // 16,777,216 = 256^3
constexpr int NA_MAX_DEVICES = 64;

// The scratch: one record per block, written in full by every call (nothing in
// it needs clearing) and shared by all calls on the same GPU.
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_BLOCKS * NA_REC];

std::mutex g_setup_mutex;
double* g_scratch_addr[NA_MAX_DEVICES] = {};

// record: 0 fluid nodes, 1 sum phi, 2 sum (1 - phi), 3 max |u|^2, 4 non-finite count
template <typename T>
__global__ void __launch_bounds__(NA_THREADS) k_noalloc_partial(const uint8_t* __restrict__ cls,
                                                                const T* __restrict__ phi, const T* __restrict__ u,
                                                                int ncomp, int64_t n, int64_t plane,
                                                                double* __restrict__ scratch) {
    double acc[NA_REC] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t begin = blockIdx.x * NA_NODES_PER_BLOCK;
    const int64_t end = begin + NA_NODES_PER_BLOCK < n ? begin + NA_NODES_PER_BLOCK : n;
    for (int64_t node = begin + threadIdx.x; node < end; node += NA_THREADS) {
        if (cls[node] != 0) continue;
        const double ph = (double)phi[node];
        double u2 = 0.0;
        for (int a = 0; a < ncomp; ++a) {
            const double ua = (double)u[a * plane + node];
            u2 += ua * ua;
        }
        acc[0] += 1.0;
        acc[1] += ph;
        acc[2] += 1.0 - ph;
        if (isfinite(u2) && u2 > acc[3]) acc[3] = u2;
        if (!isfinite(u2) || !isfinite(ph)) acc[4] += 1.0;      // NaN or +-Inf in phi or u
    }
    __shared__ double s_w[NA_THREADS / 32][NA_REC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NA_REC; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, v, o);
            v = (k == 3) ? fmax(v, w) : v + w;
        }
        if (lane == 0) s_w[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NA_REC) {
        const int k = threadIdx.x;
        double v = s_w[0][k];
        for (int w = 1; w < NA_THREADS / 32; ++w) v = (k == 3) ? fmax(v, s_w[w][k]) : v + s_w[w][k];
        scratch[blockIdx.x * NA_REC + k] = v;
    }
}

__global__ void k_noalloc_final(int nblocks, const double* __restrict__ scratch, double rho_l, double rho_g,
                                double* __restrict__ out) {
    if (threadIdx.x != 0) return;
    double r[NA_REC] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
        for (int k = 0; k < NA_REC; ++k)
            r[k] = (k == 3) ? fmax(r[k], scratch[b * NA_REC + k]) : r[k] + scratch[b * NA_REC + k];
    out[0] = r[0];
    out[1] = r[1];
    out[2] = rho_l * r[1];
    out[3] = rho_g * r[2];
    out[4] = sqrt(r[3]);
    out[5] = r[4];
}

lbm_status report(char* err, size_t err_len, lbm_status st, const char* msg) {
    if (err && err_len > 0) std::snprintf(err, err_len, "%s", msg);
    return st;
}

}  // namespace

extern "C" lbm_status lbm_phase_sums_noalloc(const uint8_t* dev_class, const void* dev_phi, const void* dev_u,
                                             int32_t precision, int32_t n_components, int64_t n_nodes,
                                             int64_t plane, double rho_l, double rho_g, double* dev_out,
                                             void* cuda_stream, char* err, size_t err_len) {
    if (err && err_len > 0) err[0] = '\0';
    if (!dev_class || !dev_phi || !dev_out || (n_components > 0 && !dev_u))
        return report(err, err_len, LBM_ERR_ARG, "a device pointer is NULL");
    if (precision != LBM_FP32 && precision != LBM_FP64)
        return report(err, err_len, LBM_ERR_ARG, "precision must be LBM_FP32 or LBM_FP64");
    if (n_components < 0 || n_components > 3)
        return report(err, err_len, LBM_ERR_ARG, "n_components must be 0..3");
    if (n_nodes < 1) return report(err, err_len, LBM_ERR_ARG, "n_nodes must be >= 1");
    if (n_nodes > NA_MAX_NODES)
        return report(err, err_len, LBM_ERR_ARG,
                      "n_nodes exceeds 16777216, the capacity of the static scratch (1024 blocks x 16384 nodes)");
    if (plane < n_nodes) return report(err, err_len, LBM_ERR_ARG, "plane must be >= n_nodes");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
        return report(err, err_len, LBM_ERR_CUDA, "no current CUDA device");
    double* scratch = nullptr;
    {
        // one-time set-up per device, with that device current
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return report(err, err_len, LBM_ERR_CUDA, cudaGetErrorString(e));
            g_scratch_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int nblocks = (int)((n_nodes + NA_NODES_PER_BLOCK - 1) / NA_NODES_PER_BLOCK);
    if (precision == LBM_FP32)
        k_noalloc_partial<float><<<nblocks, NA_THREADS, 0, s>>>(dev_class, static_cast<const float*>(dev_phi),
                                                               static_cast<const float*>(dev_u), n_components,
                                                               n_nodes, plane, scratch);
    else
        k_noalloc_partial<double><<<nblocks, NA_THREADS, 0, s>>>(dev_class, static_cast<const double*>(dev_phi),
                                                                static_cast<const double*>(dev_u), n_components,
                                                                n_nodes, plane, scratch);
    k_noalloc_final<<<1, 32, 0, s>>>(nblocks, scratch, rho_l, rho_g, dev_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report(err, err_len, LBM_ERR_CUDA, cudaGetErrorString(e));
    return LBM_OK;
}
