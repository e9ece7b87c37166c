// CUDA kernels of the color-gradient lattice Boltzmann wetting step (sm_103a).
//
// Storage ("pull" layout): after a step the population arrays hold the
// post-collision values N*_i(x), B*_i(x) at the node x where they were
// computed.  Streaming happens when the next kernel reads them: the
// post-streaming population at fluid node x is
//     N_i(x) = N*_i(x - c_i)        if x - c_i is fluid,
//     N_i(x) = N*_opp(i)(x)         otherwise (halfway bounce-back, walls at rest),
// which is Eqs. (propTotal)/(propBlue) with bounce-back on the staircase solid.
//
// One time step is three launches on one stream:
//   k_ghost  Eq. (ghost-nodePrescription) at every ghost node, from the color
//            of the fluid corners of x_F (weights precomputed on the host)
//   k_step   at every fluid node: pull N, B; isotropic stencils of phi (and of
//            the previous velocity) from a shared-memory halo tile; forces of
//            Eqs. (surfaceTensionForce), (pressCorrection), (viscCorrection),
//            (totalForce); u, p of Eqs. (velUpdate), (pressureUpdate);
//            collision of Eq. (MRTCOLL) in closed form; segregation of Eq.
//            (segragationStepBlue); write N*, B*, u, p at the node
//   k_phi    Eq. (phiUpdate): pull B* and sum it at every fluid node
//
// Arrays are structure-of-arrays with a plane stride `plane` (a multiple of
// 64 elements): field[i * plane + node].  Node classes: 0 fluid, 1 ghost
// (solid boundary node), 2 bulk solid.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lbm_lattice.cuh"

namespace lbmgpu {

enum : uint8_t { CLS_FLUID = 0, CLS_GHOST = 1, CLS_SOLID = 2 };

template <typename T>
struct StepParams {
    int nx, ny, nz;
    int64_t plane;           // elements between consecutive planes of a field
    T rho_l, rho_g, drho;    // drho = rho_l - rho_g
    T inv_nu_l, inv_nu_g;    // 1/nu_l, 1/nu_g
    T sigma;
    T k48W, k3W2, two_over_W;   // 48/W, 3W/2, 2/W
    T g[3];
    T chi[19];
    T c2chi;                 // sum_i chi_i c_ix^2 = (1-alpha) c_s^2/(1-w_0)
    T exp_eps;               // exp(eps), eps = -(4/W) cos(theta)
};

template <typename T>
struct StepBuffers {
    const T* Nin;
    const T* Bin;
    T* Nout;
    T* Bout;
    T* phi;
    const T* u_in;           // velocity of the previous step (F_visc stencil)
    T* u_out;
    T* p;
    const uint8_t* cls;
    int* err;                // bit 0: non-finite value seen
};

template <int Q>
struct Tile {
    static constexpr int D = Lattice<Q>::D;
    static constexpr int TX = 32;
    static constexpr int TY = (D == 2) ? 8 : 4;
    static constexpr int TZ = (D == 2) ? 1 : 2;
    static constexpr int HX = TX + 2;
    static constexpr int HY = TY + 2;
    static constexpr int HZ = (D == 2) ? 1 : TZ + 2;
    static constexpr int HN = HX * HY * HZ;
    static constexpr int THREADS = TX * TY * TZ;
    // offset of the halo slot of x + c in a halo tile
    __host__ __device__ static constexpr int off(int cx, int cy, int cz) { return cx + HX * (cy + HY * cz); }
};

__device__ __forceinline__ int wrap_any(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// Load the node classes (and optionally color / velocity) of a block's tile
// with a one-node halo, periodic wrap on every axis.
template <int Q, typename T, bool LOAD_PHI, bool LOAD_U>
__device__ __forceinline__ void load_halo(const StepParams<T>& P, const uint8_t* __restrict__ cls,
                                          const T* __restrict__ phi, const T* __restrict__ u,
                                          uint8_t* s_cls, T* s_phi, T* s_u, int x0, int y0, int z0) {
    using Tl = Tile<Q>;
    constexpr int D = Tl::D;
    const int tid = threadIdx.x + Tl::TX * (threadIdx.y + Tl::TY * threadIdx.z);
    for (int k = tid; k < Tl::HN; k += Tl::THREADS) {
        const int hx = k % Tl::HX;
        const int hy = (k / Tl::HX) % Tl::HY;
        const int hz = k / (Tl::HX * Tl::HY);
        const int gx = wrap_any(x0 + hx - 1, P.nx);
        const int gy = wrap_any(y0 + hy - 1, P.ny);
        const int gz = (D == 2) ? 0 : wrap_any(z0 + hz - 1, P.nz);
        const int64_t node = gx + (int64_t)P.nx * (gy + (int64_t)P.ny * gz);
        const uint8_t c = cls[node];
        s_cls[k] = c;
        if (LOAD_PHI) s_phi[k] = (c != CLS_SOLID) ? phi[node] : T(0);
        if (LOAD_U) {
#pragma unroll
            for (int d = 0; d < D; ++d) s_u[d * Tl::HN + k] = (c == CLS_FLUID) ? u[d * P.plane + node] : T(0);
        }
    }
}

// Global node index of x + (dx, dy, dz), each |d| <= 1, periodic.
struct Nbr {
    int xs[3], ys[3], zs[3];
    int nx, ny;
    __device__ __forceinline__ Nbr(int x, int y, int z, int nx_, int ny_, int nz_) : nx(nx_), ny(ny_) {
        xs[0] = x == 0 ? nx_ - 1 : x - 1; xs[1] = x; xs[2] = x == nx_ - 1 ? 0 : x + 1;
        ys[0] = y == 0 ? ny_ - 1 : y - 1; ys[1] = y; ys[2] = y == ny_ - 1 ? 0 : y + 1;
        zs[0] = z == 0 ? nz_ - 1 : z - 1; zs[1] = z; zs[2] = z == nz_ - 1 ? 0 : z + 1;
    }
    __device__ __forceinline__ int64_t at(int dx, int dy, int dz) const {
        return xs[dx + 1] + (int64_t)nx * (ys[dy + 1] + (int64_t)ny * zs[dz + 1]);
    }
};

// ---------------------------------------------------------------------------
// k_phi: Eq. (phiUpdate) on pulled B*
// ---------------------------------------------------------------------------
template <int Q, typename T>
__global__ void __launch_bounds__(Tile<Q>::THREADS) k_phi(StepParams<T> P, const T* __restrict__ Bst,
                                                          const uint8_t* __restrict__ cls, T* __restrict__ phi) {
    using L = Lattice<Q>;
    using Tl = Tile<Q>;
    __shared__ uint8_t s_cls[Tl::HN];
    const int x0 = blockIdx.x * Tl::TX, y0 = blockIdx.y * Tl::TY, z0 = blockIdx.z * Tl::TZ;
    load_halo<Q, T, false, false>(P, cls, nullptr, nullptr, s_cls, nullptr, nullptr, x0, y0, z0);
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    if (x >= P.nx || y >= P.ny || z >= P.nz) return;
    const int hc = (threadIdx.x + 1) + Tl::HX * ((threadIdx.y + 1) + Tl::HY * (L::D == 2 ? 0 : threadIdx.z + 1));
    if (s_cls[hc] != CLS_FLUID) return;
    const Nbr nb(x, y, z, P.nx, P.ny, P.nz);
    const int64_t node = nb.at(0, 0, 0);
    T s = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const bool from_fluid = s_cls[hc - Tl::off(L::cx(i), L::cy(i), L::cz(i))] == CLS_FLUID;
        const T b = from_fluid ? __ldg(Bst + i * P.plane + nb.at(-L::cx(i), -L::cy(i), -L::cz(i)))
                               : __ldg(Bst + L::opp(i) * P.plane + node);
        s += b;
    }
    phi[node] = s;
}

// ---------------------------------------------------------------------------
// k_ghost: Eq. (ghost-nodePrescription)
// ---------------------------------------------------------------------------
template <int GK, typename T>
__global__ void __launch_bounds__(256) k_ghost(int64_t n_ghosts, const int32_t* __restrict__ g_node,
                                               const int32_t* __restrict__ g_corner, const T* __restrict__ g_wt,
                                               T exp_eps, T* __restrict__ phi) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n_ghosts) return;
    T phiF = T(0);
#pragma unroll
    for (int k = 0; k < GK; ++k) phiF += g_wt[k * n_ghosts + g] * phi[g_corner[k * n_ghosts + g]];
    phi[g_node[g]] = phiF / (phiF + (T(1) - phiF) * exp_eps);
}

// ---------------------------------------------------------------------------
// k_step: stencils, forces, macroscopic fields, collision, segregation
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T rcp(T v) { return T(1) / v; }

template <int Q, typename T, bool CONTRAST>
__global__ void __launch_bounds__(Tile<Q>::THREADS) k_step(StepParams<T> P, StepBuffers<T> b) {
    using L = Lattice<Q>;
    using Tl = Tile<Q>;
    constexpr int D = L::D;
    __shared__ uint8_t s_cls[Tl::HN];
    __shared__ T s_phi[Tl::HN];
    __shared__ T s_u[CONTRAST ? D * Tl::HN : 1];
    const int x0 = blockIdx.x * Tl::TX, y0 = blockIdx.y * Tl::TY, z0 = blockIdx.z * Tl::TZ;
    load_halo<Q, T, true, CONTRAST>(P, b.cls, b.phi, b.u_in, s_cls, s_phi, s_u, x0, y0, z0);
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    if (x >= P.nx || y >= P.ny || z >= P.nz) return;
    const int hc = (threadIdx.x + 1) + Tl::HX * ((threadIdx.y + 1) + Tl::HY * (D == 2 ? 0 : threadIdx.z + 1));
    if (s_cls[hc] != CLS_FLUID) return;
    const Nbr nb(x, y, z, P.nx, P.ny, P.nz);
    const int64_t node = nb.at(0, 0, 0);
    const int64_t pl = P.plane;

    // pull the post-streaming populations (bounce-back where x - c_i is solid)
    T N[Q], B[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const bool from_fluid = s_cls[hc - Tl::off(L::cx(i), L::cy(i), L::cz(i))] == CLS_FLUID;
        const int64_t src = from_fluid ? i * pl + nb.at(-L::cx(i), -L::cy(i), -L::cz(i)) : L::opp(i) * pl + node;
        N[i] = __ldg(b.Nin + src);
        B[i] = __ldg(b.Bin + src);
    }

    // isotropic stencils: grad f = 3 sum w c f(x+c), lap f = 6 sum w (f(x+c) - f(x))
    const T phi = s_phi[hc];
    T gp[3] = {T(0), T(0), T(0)};
    T lap = T(0);
    T du[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};   // du[a][b] = d_a u_b
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int h = hc + Tl::off(L::cx(i), L::cy(i), L::cz(i));
        const T wi = T(L::w(i));
        const T ph = s_phi[h];
        gp[0] += wi * T(L::cx(i)) * ph;
        gp[1] += wi * T(L::cy(i)) * ph;
        if (D == 3) gp[2] += wi * T(L::cz(i)) * ph;
        lap += wi * (ph - phi);
        if (CONTRAST) {
#pragma unroll
            for (int bb = 0; bb < D; ++bb) {
                const T ub = s_u[bb * Tl::HN + h];
                du[0][bb] += wi * T(L::cx(i)) * ub;
                du[1][bb] += wi * T(L::cy(i)) * ub;
                if (D == 3) du[2][bb] += wi * T(L::cz(i)) * ub;
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        gp[a] *= T(3);
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) du[a][bb] *= T(3);
    }
    lap *= T(6);

    // mixture density and viscosity (Sec. II), relaxation time (Appendix A)
    const T rho = P.rho_g + P.drho * phi;
    const T inv_rho = rcp(rho);
    const T nu = rcp(phi * P.inv_nu_l + (T(1) - phi) * P.inv_nu_g);
    const T tau = T(0.5) + T(3) * nu;

    // force-free velocity and the pressure of this step (Eq. pressureUpdate)
    constexpr double w0 = L::w(0);
    T u0[3] = {T(0), T(0), T(0)};
    T sum_moving = T(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        sum_moving += N[i];
        u0[0] += T(L::cx(i)) * N[i];
        u0[1] += T(L::cy(i)) * N[i];
        if (D == 3) u0[2] += T(L::cz(i)) * N[i];
    }
    const T pres_base = (sum_moving - (T(1) - P.chi[0])) * T(1.0 / 3.0);
    const T inv_1mw0 = T(1.0 / (1.0 - w0));
    const T uu0 = u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2];
    const T p0 = (pres_base - T(0.5 * w0) * uu0) * inv_1mw0;

    // forces
    const T muc = P.k48W * phi * (T(1) - phi) * (phi - T(0.5)) + P.k3W2 * lap;   // chemical potential / sigma
    T F[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) F[a] = (-P.sigma * muc) * gp[a] + rho * P.g[a];
    if (D == 2) F[2] = T(0);
    if (CONTRAST) {
        T gr[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) gr[a] = P.drho * gp[a];
        const T kv = (tau - T(0.5)) * T(1.0 / 3.0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            T sv = T(0);
#pragma unroll
            for (int bb = 0; bb < D; ++bb) sv += (du[a][bb] + du[bb][a]) * gr[bb];
            F[a] += kv * sv - p0 * gr[a];
        }
    }

    // Eq. (velUpdate), Eq. (pressureUpdate)
    T u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = u0[a] + T(0.5) * F[a] * inv_rho;
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const T p = (pres_base - T(0.5 * w0) * uu) * inv_1mw0;

    // non-equilibrium traceless second moments: Pi(N) - [(c2chi + p) I + u u]
    T Pxx = T(0), Pyy = T(0), Pzz = T(0), Pxy = T(0), Pxz = T(0), Pyz = T(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        if (cx) Pxx += N[i];
        if (cy) Pyy += N[i];
        if (cz) Pzz += N[i];
        if (cx * cy) Pxy += T(cx * cy) * N[i];
        if (cx * cz) Pxz += T(cx * cz) * N[i];
        if (cy * cz) Pyz += T(cy * cz) * N[i];
    }
    const T omega1 = T(1) - rcp(tau);        // 1 - s_nu
    T A0, A1, Axy, Axz, Ayz;
    if (D == 2) {
        A0 = omega1 * ((Pxx - Pyy) - (u[0] * u[0] - u[1] * u[1])) * T(0.25);     // m7 . f / |m7|^2
        A1 = T(0);
        Axy = omega1 * (Pxy - u[0] * u[1]) * T(0.25);                             // m8 . f / |m8|^2
        Axz = Ayz = T(0);
    } else {
        A0 = omega1 * ((T(2) * Pxx - Pyy - Pzz) - (T(2) * u[0] * u[0] - u[1] * u[1] - u[2] * u[2])) * T(1.0 / 36.0);
        A1 = omega1 * ((Pyy - Pzz) - (u[1] * u[1] - u[2] * u[2])) * T(1.0 / 12.0);
        Axy = omega1 * (Pxy - u[0] * u[1]) * T(0.25);
        Axz = omega1 * (Pxz - u[0] * u[2]) * T(0.25);
        Ayz = omega1 * (Pyz - u[1] * u[2]) * T(0.25);
    }

    // segregation: n_phi = grad phi / max(|grad phi|, 1e-6)
    const T gn = sqrt(gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2]);
    const T inv_gn = rcp(gn > T(1e-6) ? gn : T(1e-6));
    const T kseg = P.two_over_W * phi * (T(1) - phi) * inv_gn;
    const T three_p = T(3) * p;
    const T Fs = T(3) * inv_rho;   // F_i = 3 w_i (c_i . F)/rho

    T* __restrict__ Nout = b.Nout;
    T* __restrict__ Bout = b.Bout;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const T wi = T(L::w(i));
        const T cu = T(cx) * u[0] + T(cy) * u[1] + T(cz) * u[2];
        T neq;
        if (i == 0) neq = P.chi[0] - T(1.0 - w0) * three_p - T(1.5 * w0) * uu;
        else neq = P.chi[i] + wi * (three_p + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
        const T cF = T(cx) * F[0] + T(cy) * F[1] + T(cz) * F[2];
        T proj;
        if (D == 2) {
            proj = T(cx * cx - cy * cy) * A0 + T(cx * cy) * Axy;
        } else {
            const int c2 = cx * cx + cy * cy + cz * cz;
            proj = T(3 * cx * cx - c2) * A0 + T(cy * cy - cz * cz) * A1 + T(cx * cy) * Axy + T(cx * cz) * Axz +
                   T(cy * cz) * Ayz;
        }
        const T nst = neq + T(0.5) * wi * Fs * cF + proj;
        T bst = phi * nst;
        if (i != 0) {
            const T cg = T(cx) * gp[0] + T(cy) * gp[1] + T(cz) * gp[2];
            bst += kseg * cg * (P.chi[i] + wi * three_p);
        }
        Nout[i * pl + node] = nst;
        Bout[i * pl + node] = bst;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) b.u_out[a * pl + node] = u[a];
    b.p[node] = p;
    if (!(uu < T(1e30))) atomicOr(b.err, 1);   // also catches NaN
}

}  // namespace lbmgpu
