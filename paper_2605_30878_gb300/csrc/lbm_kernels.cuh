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
//   k_step   at every fluid node: pull N; isotropic stencils of phi (and of
//            the previous velocity) from a shared-memory halo tile; forces of
//            Eqs. (surfaceTensionForce), (pressCorrection), (viscCorrection),
//            (totalForce); u, p of Eqs. (velUpdate), (pressureUpdate);
//            collision of Eq. (MRTCOLL) in closed form; segregation of Eq.
//            (segragationStepBlue); write N*, B*, u, p at the node
//   k_phi    Eq. (phiUpdate): pull B* and sum it at every fluid node
//
// Arrays are structure-of-arrays with a plane stride `plane` (a multiple of
// 64 elements): field[i * plane + node], indexed in 32 bits (Q * plane < 2^31).
// Node classes: 0 fluid, 1 ghost (solid boundary node), 2 bulk solid; the step
// kernels read a per-node 32-bit bounce-back mask derived from them instead.
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
    const uint32_t* mask;    // per-node bounce-back mask, see MASK_NOT_FLUID
    int* err;                // bit 0: non-finite value seen
};

// Per-node mask: bit i (1 <= i < Q) is set when x - c_i is not a fluid node,
// so the pull in direction i bounces back; MASK_NOT_FLUID marks non-fluid x.
constexpr uint32_t MASK_NOT_FLUID = 0x80000000u;

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

// v in [-1, n + TX]: periodic image for v in [-1, n]; positions further out
// belong to threads outside the grid and are clamped to 0.
__device__ __forceinline__ int wrap_halo(int v, int n) {
    if (v < 0) return v + n;
    if (v >= n) v -= n;
    return v < n ? v : 0;
}

// Linear offsets (32-bit) from node (x, y, z) to its periodic lattice neighbours.
struct Wrap {
    int xm, xp, ym, yp, zm, zp;
    __device__ __forceinline__ Wrap(int x, int y, int z, int nx, int ny, int nz) {
        xm = (x == 0) ? nx - 1 : -1;
        xp = (x == nx - 1) ? 1 - nx : 1;
        ym = (y == 0) ? (ny - 1) * nx : -nx;
        yp = (y == ny - 1) ? (1 - ny) * nx : nx;
        const int sz = nx * ny;
        zm = (z == 0) ? (nz - 1) * sz : -sz;
        zp = (z == nz - 1) ? (1 - nz) * sz : sz;
    }
    __device__ __forceinline__ int off(int dx, int dy, int dz) const {
        return (dx < 0 ? xm : (dx > 0 ? xp : 0)) + (dy < 0 ? ym : (dy > 0 ? yp : 0)) +
               (dz < 0 ? zm : (dz > 0 ? zp : 0));
    }
};

// Load a block's color (and optionally velocity) tile with a one-node halo.
// Ghost nodes hold their fresh ghost color; the velocity at solid nodes is 0
// in memory (never written), so no node class is needed here.
template <int Q, typename T, bool LOAD_U>
__device__ __forceinline__ void load_halo(const StepParams<T>& P, const T* __restrict__ phi,
                                          const T* __restrict__ u, T* s_phi, T* s_u, int x0, int y0, int z0) {
    using Tl = Tile<Q>;
    constexpr int D = Tl::D;
    const int tid = threadIdx.x + Tl::TX * (threadIdx.y + Tl::TY * threadIdx.z);
    for (int k = tid; k < Tl::HN; k += Tl::THREADS) {
        const int hx = k % Tl::HX;
        const int hy = (k / Tl::HX) % Tl::HY;
        const int hz = k / (Tl::HX * Tl::HY);
        const int gx = wrap_halo(x0 + hx - 1, P.nx);
        const int gy = wrap_halo(y0 + hy - 1, P.ny);
        const int gz = (D == 2) ? 0 : wrap_halo(z0 + hz - 1, P.nz);
        const int node = gx + P.nx * (gy + P.ny * gz);
        s_phi[k] = phi[node];
        if (LOAD_U) {
#pragma unroll
            for (int d = 0; d < D; ++d) s_u[d * Tl::HN + k] = u[d * (int)P.plane + node];
        }
    }
}

// ---------------------------------------------------------------------------
// k_phi: Eq. (phiUpdate) on pulled B*
// ---------------------------------------------------------------------------
template <int Q, typename T>
__global__ void __launch_bounds__(Tile<Q>::THREADS) k_phi(StepParams<T> P, const T* __restrict__ Bst,
                                                          const uint32_t* __restrict__ mask, T* __restrict__ phi) {
    using L = Lattice<Q>;
    using Tl = Tile<Q>;
    const int x = blockIdx.x * Tl::TX + threadIdx.x;
    const int y = blockIdx.y * Tl::TY + threadIdx.y;
    const int z = blockIdx.z * Tl::TZ + threadIdx.z;
    if (x >= P.nx || y >= P.ny || z >= P.nz) return;
    const int node = x + P.nx * (y + P.ny * z);
    const uint32_t m = __ldg(mask + node);
    if (m & MASK_NOT_FLUID) return;
    const Wrap W(x, y, z, P.nx, P.ny, P.nz);
    const int pl = (int)P.plane;
    T s = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int src = ((m >> i) & 1u) ? L::opp(i) * pl + node
                                        : i * pl + node + W.off(-L::cx(i), -L::cy(i), -L::cz(i));
        s += __ldg(Bst + src);
    }
    phi[node] = s;
}

// ---------------------------------------------------------------------------
// k_ghost: Eq. (ghost-nodePrescription)
// ---------------------------------------------------------------------------
// RULE 0: the paper's rule; RULE 1: Eq. (ghostNodeFakhari) multiplied through by
// the conjugate, 4 phi_F / (a + sqrt(a^2 - 2 eps phi_F)) - phi_F, a = 1 + eps/2,
// which stays accurate as eps -> 0 (theta -> 90 deg) where the printed form cancels.
template <int GK, typename T, int RULE>
__global__ void __launch_bounds__(256) k_ghost(int64_t n_ghosts, const int32_t* __restrict__ g_node,
                                               const int32_t* __restrict__ g_corner, const T* __restrict__ g_wt,
                                               T exp_eps, T eps, T* __restrict__ phi) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n_ghosts) return;
    T phiF = T(0);
#pragma unroll
    for (int k = 0; k < GK; ++k) phiF += g_wt[k * n_ghosts + g] * phi[g_corner[k * n_ghosts + g]];
    T phiG;
    if (RULE == 0) {
        phiG = phiF / (phiF + (T(1) - phiF) * exp_eps);
    } else {
        const T a = T(1) + T(0.5) * eps;
        phiG = T(4) * phiF / (a + sqrt(a * a - T(2) * eps * phiF)) - phiF;
    }
    phi[g_node[g]] = phiG;
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
    __shared__ T s_phi[Tl::HN];
    __shared__ T s_u[CONTRAST ? D * Tl::HN : 1];
    const int x0 = blockIdx.x * Tl::TX, y0 = blockIdx.y * Tl::TY, z0 = blockIdx.z * Tl::TZ;
    load_halo<Q, T, CONTRAST>(P, b.phi, b.u_in, s_phi, s_u, x0, y0, z0);
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    if (x >= P.nx || y >= P.ny || z >= P.nz) return;
    const int node = x + P.nx * (y + P.ny * z);
    const uint32_t m = __ldg(b.mask + node);
    if (m & MASK_NOT_FLUID) return;
    const int hc = (threadIdx.x + 1) + Tl::HX * ((threadIdx.y + 1) + Tl::HY * (D == 2 ? 0 : threadIdx.z + 1));
    const Wrap Wr(x, y, z, P.nx, P.ny, P.nz);
    const int pl = (int)P.plane;

    // pull the post-streaming populations N (bounce-back where x - c_i is solid);
    // B enters the collision only through phi = sum B, which k_phi computed
    T N[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int src = ((m >> i) & 1u) ? L::opp(i) * pl + node
                                        : i * pl + node + Wr.off(-L::cx(i), -L::cy(i), -L::cz(i));
        N[i] = __ldg(b.Nin + src);
    }

    // isotropic stencils: grad f = 3 sum_i w_i c_i f(x+c_i), lap f = 6 sum_i w_i (f(x+c_i) - f(x)).
    // FP32 sums over +/- pairs (half the multiply-adds); FP64, the mode checked
    // against the FP64 oracle to 1e-12 over thousands of steps, sums in lattice
    // order as the definition is written.
    constexpr bool kPairs = sizeof(T) == 4;
    const T phi = s_phi[hc];
    T gp[3] = {T(0), T(0), T(0)};
    T lsum = T(0);
    T du[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};   // du[a][b] = d_a u_b
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const T wi = T(L::w(i));
        if (kPairs) {
            if (L::opp(i) < i) continue;
            const int hp = hc + Tl::off(cx, cy, cz), hm = hc - Tl::off(cx, cy, cz);
            const T pp = s_phi[hp], pm = s_phi[hm];
            const T dphi = wi * (pp - pm);
            if (cx) gp[0] += T(cx) * dphi;
            if (cy) gp[1] += T(cy) * dphi;
            if (cz) gp[2] += T(cz) * dphi;
            lsum += wi * ((pp - phi) + (pm - phi));
            if (CONTRAST) {
#pragma unroll
                for (int bb = 0; bb < D; ++bb) {
                    const T dub = wi * (s_u[bb * Tl::HN + hp] - s_u[bb * Tl::HN + hm]);
                    if (cx) du[0][bb] += T(cx) * dub;
                    if (cy) du[1][bb] += T(cy) * dub;
                    if (cz) du[2][bb] += T(cz) * dub;
                }
            }
        } else {
            const int h = hc + Tl::off(cx, cy, cz);
            const T ph = s_phi[h];
            gp[0] += wi * T(cx) * ph;
            gp[1] += wi * T(cy) * ph;
            if (D == 3) gp[2] += wi * T(cz) * ph;
            lsum += wi * (ph - phi);
            if (CONTRAST) {
#pragma unroll
                for (int bb = 0; bb < D; ++bb) {
                    const T ub = s_u[bb * Tl::HN + h];
                    du[0][bb] += wi * T(cx) * ub;
                    du[1][bb] += wi * T(cy) * ub;
                    if (D == 3) du[2][bb] += wi * T(cz) * ub;
                }
            }
        }
    }
    constexpr double w0 = L::w(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        gp[a] *= T(3);
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) du[a][bb] *= T(3);
    }
    const T lap = T(6) * lsum;

    // mixture density and viscosity (Sec. II), relaxation time (Appendix A)
    const T rho = P.rho_g + P.drho * phi;
    const T inv_rho = rcp(rho);
    const T nu = rcp(phi * P.inv_nu_l + (T(1) - phi) * P.inv_nu_g);
    const T tau = T(0.5) + T(3) * nu;

    // force-free velocity, moments and the pressure of this step (Eq. pressureUpdate)
    T u0[3] = {T(0), T(0), T(0)};
    T sum_moving = T(0);
    T Pxx = T(0), Pyy = T(0), Pzz = T(0), Pxy = T(0), Pxz = T(0), Pyz = T(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        sum_moving += N[i];
        if (cx > 0) { u0[0] += N[i]; Pxx += N[i]; }
        if (cx < 0) { u0[0] -= N[i]; Pxx += N[i]; }
        if (cy > 0) { u0[1] += N[i]; Pyy += N[i]; }
        if (cy < 0) { u0[1] -= N[i]; Pyy += N[i]; }
        if (cz > 0) { u0[2] += N[i]; Pzz += N[i]; }
        if (cz < 0) { u0[2] -= N[i]; Pzz += N[i]; }
        if (cx * cy > 0) Pxy += N[i];
        if (cx * cy < 0) Pxy -= N[i];
        if (cx * cz > 0) Pxz += N[i];
        if (cx * cz < 0) Pxz -= N[i];
        if (cy * cz > 0) Pyz += N[i];
        if (cy * cz < 0) Pyz -= N[i];
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

    // collision: traceless second moments of N - Neq, with sum Neq c c = (c2chi + p) I + u u
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
    const T halfF = T(1.5) * inv_rho;   // (1/2) F_i = (3/2) w_i (c_i . F)/rho
    const T base0 = T(3) * u[0], base1 = T(3) * u[1], base2 = T(3) * u[2];
    const T common = three_p - T(1.5) * uu;

    T* __restrict__ Nout = b.Nout;
    T* __restrict__ Bout = b.Bout;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const T wi = T(L::w(i));
        T neq, nst;
        if (i == 0) {
            neq = P.chi[0] - T(1.0 - w0) * three_p - T(1.5 * w0) * uu;
            nst = neq;
        } else {
            T cu3 = T(0), cF = T(0);   // 3 c.u and c.F
            if (cx) { cu3 += T(cx) * base0; cF += T(cx) * F[0]; }
            if (cy) { cu3 += T(cy) * base1; cF += T(cy) * F[1]; }
            if (cz) { cu3 += T(cz) * base2; cF += T(cz) * F[2]; }
            neq = P.chi[i] + wi * (common + cu3 + T(0.5) * cu3 * cu3);
            nst = neq + wi * halfF * cF;
        }
        T proj;
        if (D == 2) {
            proj = T(cx * cx - cy * cy) * A0 + T(cx * cy) * Axy;
        } else {
            const int c2 = cx * cx + cy * cy + cz * cz;
            proj = T(3 * cx * cx - c2) * A0 + T(cy * cy - cz * cz) * A1 + T(cx * cy) * Axy + T(cx * cz) * Axz +
                   T(cy * cz) * Ayz;
        }
        nst += proj;
        T bst = phi * nst;
        if (i != 0) {
            T cg = T(0);
            if (cx) cg += T(cx) * gp[0];
            if (cy) cg += T(cy) * gp[1];
            if (cz) cg += T(cz) * gp[2];
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
