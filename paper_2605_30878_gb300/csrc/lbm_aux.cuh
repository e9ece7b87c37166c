// Initialisation, state transfer and diagnostics kernels (not on the per-step path).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lbm_kernels.cuh"

namespace lbmgpu {

// Grid extents, the row pitch px >= nx of every device field (node = x + px *
// (y + ny * z); columns nx..px-1 are solid padding) and the plane stride.
struct Dims {
    int nx, ny, nz, px;
    int64_t plane;
    uint32_t periodic;
};

__device__ __forceinline__ int64_t padded_nodes(const Dims& d) { return (int64_t)d.px * d.ny * d.nz; }

__device__ __forceinline__ void node_xyz(int64_t node, const Dims& d, int& x, int& y, int& z) {
    x = (int)(node % d.px);
    y = (int)((node / d.px) % d.ny);
    z = (int)(node / ((int64_t)d.px * d.ny));
}

__device__ __forceinline__ int64_t shifted(const Dims& d, int x, int y, int z, int dx, int dy, int dz) {
    const int xx = wrap_any(x + dx, d.nx), yy = wrap_any(y + dy, d.ny), zz = wrap_any(z + dz, d.nz);
    return xx + (int64_t)d.px * (yy + (int64_t)d.ny * zz);
}

// Node classes of the padded grid from the host's row bit masks: rows r =
// y + ny z of W 64-bit words, bit x of F[r W + x / 64] set for a fluid node,
// of G for a ghost (a solid node with a fluid stencil neighbour); columns
// x >= nx are padding, solid.
static __global__ void k_expand_classes(Dims d, int W, const uint64_t* __restrict__ F, const uint64_t* __restrict__ G,
                                 uint8_t* __restrict__ cls) {
    const int nn = (int)padded_nodes(d);
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < nn; node += gridDim.x * blockDim.x) {
        const int x = node % d.px, r = node / d.px;
        uint8_t c = CLS_SOLID;
        if (x < d.nx) {
            const int w = r * W + (x >> 6), b = x & 63;
            if ((F[w] >> b) & 1u) c = CLS_FLUID;
            else if ((G[w] >> b) & 1u) c = CLS_GHOST;
        }
        cls[node] = c;
    }
}

// Per-node bounce-back mask from the node classes: bit i (1 <= i < Q) set when
// x - c_i (periodic wrap) is not a fluid node, MASK_NOT_FLUID for non-fluid x.
template <int Q>
__global__ void k_build_mask(Dims d, const uint8_t* __restrict__ cls, uint32_t* __restrict__ mask) {
    using L = Lattice<Q>;
    const int64_t nn = padded_nodes(d);
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < nn;
         node += (int64_t)gridDim.x * blockDim.x) {
        if (cls[node] != CLS_FLUID) {
            mask[node] = MASK_NOT_FLUID;
            continue;
        }
        int x, y, z;
        node_xyz(node, d, x, y, z);
        uint32_t m = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            int xx = x - L::cx(i), yy = y - L::cy(i), zz = z - L::cz(i);
            xx += xx < 0 ? d.nx : (xx >= d.nx ? -d.nx : 0);
            yy += yy < 0 ? d.ny : (yy >= d.ny ? -d.ny : 0);
            zz += zz < 0 ? d.nz : (zz >= d.nz ? -d.nz : 0);
            if (cls[xx + (int64_t)d.px * (yy + (int64_t)d.ny * zz)] != CLS_FLUID) m |= 1u << i;
        }
        mask[node] = m;
    }
}

// Color at t = 0 (Eq. equilibriumPhaseField and the ghost value of Sec. III).
// mode 0: drop of radius R0 at centre; mode 1: keep the fluid values already in phi.
template <int D, typename T>
__global__ void k_init_phi(Dims d, const uint8_t* __restrict__ cls, T* __restrict__ phi, int mode, double cx,
                           double cy, double cz, double R0, double W, double ghost_value) {
    // more than 10 W from the interface, |2 (R0 - r) / W| >= 20 and
    // 1 - |tanh| < 1e-17: the profile is 0 or 1 to double precision there, so
    // tanh (slow on this GPU's few FP64 units) runs only inside that band
    const double far = 10.0 * W, out2 = (R0 + far) * (R0 + far), in2 = R0 > far ? (R0 - far) * (R0 - far) : -1.0;
    // the same two tests first in FP32, with a margin far above FP32's error
    // in the squared distance (relative 1e-6): only nodes near the band's
    // edges or inside it take the FP64 path, whose answer they do not change
    const float out2f = (float)(out2 * (1.0 + 1e-4) + 1.0);
    const float in2f = in2 > 0.0 ? (float)(in2 * (1.0 - 1e-4) - 1.0) : -1.0f;
    const float fc[3] = {(float)cx, (float)cy, (float)cz};
    const int nn = (int)padded_nodes(d);                    // node indices are below 2^31
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < nn; node += gridDim.x * blockDim.x) {
        const uint8_t c = cls[node];
        if (c == CLS_FLUID) {
            if (mode == 0) {
                const int x = node % d.px, t = node / d.px, y = t % d.ny, z = t / d.ny;
                const double ctr[3] = {cx, cy, cz};
                const int n[3] = {d.nx, d.ny, d.nz};
                const int r[3] = {x, y, z};
                float d2f = 0.0f;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    float v = (float)r[a] - fc[a];
                    if (d.periodic & (1u << a)) {
                        const float h = 0.5f * (float)n[a];
                        while (v > h) v -= (float)n[a];
                        while (v < -h) v += (float)n[a];
                    }
                    d2f = fmaf(v, v, d2f);
                }
                if (d2f > out2f || d2f < in2f) {
                    phi[node] = d2f > out2f ? T(0) : T(1);
                    continue;
                }
                double d2 = 0.0;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    double v = r[a] - ctr[a];
                    // nearest periodic image, by whole periods (exact): no FP64
                    // divide, which this GPU's few FP64 units make the kernel's
                    // largest cost (the floor form differs only at an exact
                    // tie, where both images are as near)
                    if (d.periodic & (1u << a)) {
                        const double h = 0.5 * n[a];
                        while (v > h) v -= n[a];
                        while (v < -h) v += n[a];
                    }
                    d2 += v * v;
                }
                phi[node] = d2 >= out2 ? T(0)
                          : d2 <= in2  ? T(1)
                                       : (T)(0.5 * (1.0 + tanh(2.0 * (R0 - sqrt(d2)) / W)));
            }
        } else {
            phi[node] = (c == CLS_GHOST) ? (T)ghost_value : T(0);
        }
    }
}

// Populations at t = 0: post-streaming N_i = chi_i, B_i = phi chi_i, written in
// the pull layout (the value a later pull at x + c_i reads sits at x) and in
// the storage form of S (full values, or deviations N - chi_i, B - chi_i/2).
template <int Q, typename T, typename S>
__global__ void k_init_pops(Dims d, StepParams<T> P, const uint8_t* __restrict__ cls, const T* __restrict__ phi,
                            S* __restrict__ Nst, S* __restrict__ Bst) {
    using L = Lattice<Q>;
    constexpr bool kShift = PopStore<S>::kShift;
    const int nn = (int)padded_nodes(d);                    // node indices are below 2^31
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < nn; node += gridDim.x * blockDim.x) {
        if (cls[node] != CLS_FLUID) continue;
        const int x = node % d.px, t = node / d.px, y = t % d.ny, z = t / d.ny;
        const Wrap W(x, y, z, d.nx, d.ny, d.nz, d.px);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int dn = node + W.off(L::cx(i), L::cy(i), L::cz(i));
            const T ph = (cls[dn] == CLS_FLUID) ? phi[dn] : phi[node];
            const int pl = (int)d.plane, nd = node;
            // deviation storage: N_i - chi_i(stored) = the exact chi_i minus the
            // stored one; B_i - chi_i(stored)/2 = phi (that) + (phi - 1/2) chi_i(stored)
            const T e = P.chi_err[i == 0 ? 0 : (L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i) == 1
                                                    ? 1 : 2)];
            pop_store<S, T>(Nst, i, pl, nd, kShift ? e : P.chi[i], kScaleN);
            pop_store<S, T>(Bst, i, pl, nd, kShift ? (ph - T(0.5)) * P.chi[i] + ph * e : ph * P.chi[i], kScaleB);
        }
    }
}

// One direction i of post-streaming values -> pull layout: st_i[y] = post_i[y + c_i]
// if y + c_i is fluid, else post_opp[y]; stored as value - base (base = 0, chi_i or chi_i/2).
template <int Q, typename T, typename S>
__global__ void k_scatter_dir(Dims d, const uint8_t* __restrict__ cls, int i, const T* __restrict__ post_i,
                              const T* __restrict__ post_opp, T base, float scale, S* __restrict__ st) {
    using L = Lattice<Q>;
    const int64_t nn = padded_nodes(d);
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < nn;
         node += (int64_t)gridDim.x * blockDim.x) {
        if (cls[node] != CLS_FLUID) continue;
        int x, y, z;
        node_xyz(node, d, x, y, z);
        const int64_t dn = shifted(d, x, y, z, L::cx(i), L::cy(i), L::cz(i));
        const T v = (cls[dn] == CLS_FLUID) ? post_i[dn] : post_opp[node];
        pop_store<S, T>(st, i, (int)d.plane, (int)node, v - base, scale);
    }
}

// One direction i of the pull layout -> post-streaming values (0 at solid nodes).
template <int Q, typename T, typename S>
__global__ void k_gather_dir(Dims d, const uint8_t* __restrict__ cls, int i, const S* __restrict__ st, T base,
                             float scale, T* __restrict__ post) {
    using L = Lattice<Q>;
    const int64_t nn = padded_nodes(d);
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < nn;
         node += (int64_t)gridDim.x * blockDim.x) {
        T v = T(0);
        if (cls[node] == CLS_FLUID) {
            int x, y, z;
            node_xyz(node, d, x, y, z);
            const int64_t sn = shifted(d, x, y, z, -L::cx(i), -L::cy(i), -L::cz(i));
            const bool from_fluid = cls[sn] == CLS_FLUID;
            v = base + pop_load<S, T>(st, from_fluid ? i : L::opp(i), (int)d.plane, (int)(from_fluid ? sn : node),
                                      scale);
        }
        post[node] = v;
    }
}

// ---------------------------------------------------------------------------
// diagnostics: per-block FP64 partial records, then one fixed-order final sum
// ---------------------------------------------------------------------------
enum {
    DG_PHI = 0, DG_POP, DG_NFLUID, DG_PIN, DG_NIN, DG_POUT, DG_NOUT, DG_NIFACE, DG_NFIT,
    DG_A = 9,      // 16 entries: normal matrix of the circle/sphere fit
    DG_B = 25,     // 4 entries
    DG_NAN = 29,
    DG_MAXU2 = 30, // max entries
    DG_APEX = 31,
    DG_REC = 32
};
constexpr int DIAG_THREADS = 256;
constexpr int DIAG_MAX_BLOCKS = 1024;

struct ProbeDev {
    int kind;
    double center[3], radius, normal[3], exclude;
};

// The direction index of the lattice vector (dx, dy, dz).
template <int Q>
__host__ __device__ constexpr int dir_index(int dx, int dy, int dz) {
    for (int i = 0; i < Q; ++i)
        if (Lattice<Q>::cx(i) == dx && Lattice<Q>::cy(i) == dy && Lattice<Q>::cz(i) == dz) return i;
    return -1;
}

// Per-node values are computed in the domain's arithmetic type T (the values
// as stored, summed over the Q pulled populations), the per-thread sums in
// FP64 and the counts in integers, so a float domain costs a few FP64 adds
// per node.  Neighbours come from the bounce-back mask and 32-bit periodic
// offsets (node indices are below 2^31).
template <int Q, typename T, typename S>
__global__ void __launch_bounds__(DIAG_THREADS) k_diag_partial(Dims d, double rho_l, double rho_g,
                                                               const uint32_t* __restrict__ mask, StepParams<T> P,
                                                               const S* __restrict__ Nst, const T* __restrict__ phi,
                                                               const T* __restrict__ u, const T* __restrict__ p,
                                                               ProbeDev pr, double* __restrict__ partial) {
    using L = Lattice<Q>;
    constexpr int D = L::D;
    double acc[DG_REC];
#pragma unroll
    for (int k = 0; k < DG_REC; ++k) acc[k] = 0.0;
    acc[DG_APEX] = -INFINITY;
    int n_fluid = 0, n_in = 0, n_out = 0, n_nan = 0, n_iface = 0, n_fit = 0;
    T max_u2 = T(0);
    const int nn = (int)padded_nodes(d), pl = (int)d.plane;
    const int n[3] = {d.nx, d.ny, d.nz};
    const T rl = T(rho_l), rg = T(rho_g);
    // deviation storage: the per-node sum runs over the stored deviations (small
    // values, little rounding) and the references sum_i chi_i join in FP64
    double chi_total = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) chi_total += (double)P.chi[i];
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < nn; node += gridDim.x * blockDim.x) {
        const uint32_t m = mask[node];
        if (m & MASK_NOT_FLUID) continue;
        const int x = node % d.px, t = node / d.px, y = t % d.ny, z = t / d.ny;
        const Wrap W(x, y, z, d.nx, d.ny, d.nz, d.px);
        const T ph = phi[node];
        ++n_fluid;
        acc[DG_PHI] += (double)ph;
        // the populations after streaming: pulled from x - c_i, or bounced back
        T ps = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool from_fluid = i == 0 || !((m >> i) & 1u);
            const int src = from_fluid ? node + W.off(-L::cx(i), -L::cy(i), -L::cz(i)) : node;
            ps += pop_load<S, T>(Nst, from_fluid ? i : L::opp(i), pl, src, kScaleN);
        }
        acc[DG_POP] += PopStore<S>::kShift ? (double)ps + chi_total : (double)ps;
        T u2 = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const T ua = u[a * pl + node];
            u2 += ua * ua;
        }
        if (u2 > max_u2) max_u2 = u2;
        if (!isfinite(u2) || !isfinite(ph)) ++n_nan;                  // NaN or +-Inf in phi or u
        const T phh = (rl * ph + rg * (T(1) - ph)) * p[node];
        if (ph > T(1.0 - 1e-3)) { acc[DG_PIN] += (double)phh; ++n_in; }
        if (ph < T(1e-3)) { acc[DG_POUT] += (double)phh; ++n_out; }
        if (pr.kind == 0) continue;
        const int r[3] = {x, y, z};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            // the +e_a neighbour is x - c_k for c_k = -e_a
            constexpr int kBack[3] = {dir_index<Q>(-1, 0, 0), dir_index<Q>(0, -1, 0), dir_index<Q>(0, 0, -1)};
            if ((m >> kBack[a]) & 1u) continue;
            const int yn = node + W.off(a == 0, a == 1, a == 2);
            const double phd = (double)ph, p1 = (double)phi[yn];
            if ((phd >= 0.5) == (p1 >= 0.5)) continue;
            const double tt = (0.5 - phd) / (p1 - phd);
            double q[3] = {0.0, 0.0, 0.0};
            double q2 = 0.0, h = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                double v = r[k] + (k == a ? tt : 0.0) - pr.center[k];
                v -= n[k] * floor(v / n[k] + 0.5);
                q[k] = v;
                q2 += v * v;
                h += v * pr.normal[k];
            }
            ++n_iface;
            if (h > acc[DG_APEX]) acc[DG_APEX] = h;
            const double dist = (pr.kind == 1) ? sqrt(q2) - pr.radius : h;
            if (dist < pr.exclude) continue;
            double row[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int k = 0; k < D; ++k) row[k] = q[k];
            row[D] = 1.0;
#pragma unroll
            for (int i = 0; i <= D; ++i) {
#pragma unroll
                for (int j = 0; j <= D; ++j) acc[DG_A + 4 * i + j] += row[i] * row[j];
                acc[DG_B + i] += -q2 * row[i];
            }
            ++n_fit;
        }
    }
    acc[DG_NFLUID] = n_fluid;
    acc[DG_NIN] = n_in;
    acc[DG_NOUT] = n_out;
    acc[DG_NAN] = n_nan;
    acc[DG_NIFACE] = n_iface;
    acc[DG_NFIT] = n_fit;
    acc[DG_MAXU2] = (double)max_u2;
    // block reduction in a fixed order: warp shuffles, then warps in index order
    __shared__ double s_w[DIAG_THREADS / 32][DG_REC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < DG_REC; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, v, o);
            v = (k >= DG_MAXU2) ? fmax(v, w) : v + w;
        }
        if (lane == 0) s_w[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < DG_REC) {
        const int k = threadIdx.x;
        double v = s_w[0][k];
        for (int w = 1; w < DIAG_THREADS / 32; ++w) v = (k >= DG_MAXU2) ? fmax(v, s_w[w][k]) : v + s_w[w][k];
        partial[blockIdx.x * DG_REC + k] = v;
    }
}

// The per-block records summed in a fixed order: thread (j, k) of the
// 32 x 32 block sums entry k of blocks j, j + 32, j + 64, ..., then entry k's
// 32 partial sums are added in j order (32 loads in flight per entry instead
// of one after the other).
static __global__ void __launch_bounds__(1024) k_diag_final(int nblocks, const double* __restrict__ partial,
                                                            double* __restrict__ out) {
    __shared__ double s[32][DG_REC];
    const int k = threadIdx.x, j = threadIdx.y;
    const bool is_max = k >= DG_MAXU2;
    double v = is_max ? -INFINITY : 0.0;
    for (int b = j; b < nblocks; b += 32) {
        const double w = partial[b * DG_REC + k];
        v = is_max ? fmax(v, w) : v + w;
    }
    s[j][k] = v;
    __syncthreads();
    if (j == 0) {
        double r = s[0][k];
        for (int jj = 1; jj < 32; ++jj) r = is_max ? fmax(r, s[jj][k]) : r + s[jj][k];
        out[k] = r;
    }
}

}  // namespace lbmgpu
