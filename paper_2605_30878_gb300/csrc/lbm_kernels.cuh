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
// 64 elements): field[i * plane + node], indexed in 32 bits (Q * plane < 2^31),
// node = x + px * (y + ny * z) with the row pitch px = nx rounded up to 4 (the
// padding columns are solid), so rows are 16-byte multiples for TMA copies.
// Node classes: 0 fluid, 1 ghost (solid boundary node), 2 bulk solid; the step
// kernels read a per-node 32-bit bounce-back mask derived from them instead.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm_lattice.cuh"

namespace lbmgpu {

enum : uint8_t { CLS_FLUID = 0, CLS_GHOST = 1, CLS_SOLID = 2 };

template <typename T>
struct StepParams {
    int nx, ny, nz;
    int px;                  // row pitch: node = x + px * (y + ny * z), px = nx rounded up to 4
    int64_t plane;           // elements between consecutive planes of a field
    T rho_l, rho_g, drho;    // drho = rho_l - rho_g
    T inv_nu_l, inv_nu_g;    // 1/nu_l, 1/nu_g
    T sigma, W;
    T nu_l, nu_g;            // kinematic viscosities
    T k48W, k3W2, two_over_W;   // 48/W, 3W/2, 2/W
    T g[3];
    T chi[19];               // float arithmetic: the storage reference, on a 2^-24 grid, summing to exactly 1
    // chi_i - (the chi[i] above) by direction class (0 rest, 1 axis, 2
    // diagonal/edge): zero in FP64; in float arithmetic the equilibrium and the
    // pressure's zero are taken at the exact chi through these corrections
    T chi_err[3];
    T c2chi;                 // sum_i chi_i c_ix^2 = (1-alpha) c_s^2/(1-w_0)
    T exp_eps;               // exp(eps), eps = -(4/W) cos(theta)
};

// Population storage.  S = double: full values (FP64 mode, rounding as the
// oracle).  S = float: deviations from the rest state, N_i - chi_i and
// B_i - chi_i/2 (FP32 mode); the step computes directly in these deviations,
// an exact rewrite because sum chi = 1, sum c chi = 0 and chi is isotropic, and
// it keeps the small pressure of a dense liquid (p = p_h/rho ~ 1e-8 at density
// ratio 1000) representable.  S = __half: the same deviations, the rest
// populations (i = 0, whose B deviation reaches chi_0/2 ~ 0.46) as float in the
// first plane, the moving ones times 2^16 (N) and 2^7 (B) as FP16 in the
// following Q-1 planes.
constexpr float kScaleN = 65536.0f;
constexpr float kScaleB = 128.0f;

// float(h) + c, rounded to nearest: one mixed-precision add (sm_100 and
// later) instead of a conversion and an add; every FP16 value is exact in
// float, so the result is the same.
__device__ __forceinline__ float add_f16_f32(__half h, float c) {
    float r;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(r) : "h"(__half_as_ushort(h)), "f"(c));
    return r;
}

// Each array holds the rest plane (direction 0) followed by the Q-1 moving
// planes; rest(p) and moving(p, plane) return typed pointers to the two parts,
// moving direction d >= 1 lives at moving + (d - 1) * plane.
template <typename S> struct PopStore;
template <typename V> struct PlainStore {
    static constexpr int kRestBytes = sizeof(V), kMovingBytes = sizeof(V);
    using Rest = V;
    using Moving = V;
    __device__ static const V* rest(const V* p) { return p; }
    __device__ static V* rest(V* p) { return p; }
    __device__ static const V* moving(const V* p, int plane) { return p + plane; }
    __device__ static V* moving(V* p, int plane) { return p + plane; }
    __device__ static V load_rest(const V* r, int idx) { return __ldg(r + idx); }
    __device__ static V load_moving(const V* m, int idx, float) { return __ldg(m + idx); }
    __device__ static void store_rest(V* r, int idx, V v) { r[idx] = v; }
    __device__ static void store_moving(V* m, int idx, V v, float) { m[idx] = v; }
    // in storage units: the value itself
    __device__ static V load_units(const V* m, int idx) { return __ldg(m + idx); }
    __device__ static void accumulate(const V* m, int idx, V& acc) { acc += __ldg(m + idx); }
    // stores v; exact storage leaves nothing to account for, acc is untouched
    __device__ static void store_units(V* m, int idx, V v, V&) { m[idx] = v; }
};
template <> struct PopStore<double> : PlainStore<double> {
    static constexpr bool kShift = false, kExact = true;
};
template <> struct PopStore<float> : PlainStore<float> {
    static constexpr bool kShift = true, kExact = true;
    // two adjacent nodes (idx even, so 8-byte aligned): values in storage units
    __device__ static float2 load_units2(const float* m, int idx) {
        return __ldg(reinterpret_cast<const float2*>(m + idx));
    }
    __device__ static void store_units2(float* m, int idx, float va, float vb, float&, float&) {
        *reinterpret_cast<float2*>(m + idx) = make_float2(va, vb);
    }
    __device__ static void store_zero2(float* m) { *reinterpret_cast<float2*>(m) = make_float2(0.f, 0.f); }
};
template <> struct PopStore<__half> {
    static constexpr bool kShift = true, kExact = false;     // moving populations are rounded on store
    static constexpr int kRestBytes = 4, kMovingBytes = 2;
    __device__ static const float* rest(const __half* p) { return reinterpret_cast<const float*>(p); }
    __device__ static float* rest(__half* p) { return reinterpret_cast<float*>(p); }
    __device__ static const __half* moving(const __half* p, int plane) { return p + 2 * plane; }
    __device__ static __half* moving(__half* p, int plane) { return p + 2 * plane; }
    __device__ static float load_rest(const float* r, int idx) { return __ldg(r + idx); }
    __device__ static float load_moving(const __half* m, int idx, float scale) {
        return __half2float(__ldg(m + idx)) * (1.0f / scale);
    }
    __device__ static void store_rest(float* r, int idx, float v) { r[idx] = v; }
    __device__ static void store_moving(__half* m, int idx, float v, float scale) {
        m[idx] = __float2half_rn(v * scale);
    }
    // in storage units (value x scale): the step kernels fold the power-of-two
    // scales into their arithmetic instead of scaling every population
    __device__ static float load_units(const __half* m, int idx) { return __half2float(__ldg(m + idx)); }
    __device__ static void accumulate(const __half* m, int idx, float& acc) { acc = add_f16_f32(__ldg(m + idx), acc); }
    // stores v (already scaled) and adds the value stored to acc
    __device__ static void store_units(__half* m, int idx, float v, float& acc) {
        const __half h = __float2half_rn(v);
        m[idx] = h;
        acc = add_f16_f32(h, acc);
    }
    // two adjacent nodes (idx even, so 4-byte aligned): one 32-bit load or
    // store for both, each value rounded as store_units rounds it
    __device__ static float2 load_units2(const __half* m, int idx) {
        return __half22float2(__ldg(reinterpret_cast<const __half2*>(m + idx)));
    }
    __device__ static void store_units2(__half* m, int idx, float va, float vb, float& accA, float& accB) {
        const __half2 h = __floats2half2_rn(va, vb);
        *reinterpret_cast<__half2*>(m + idx) = h;
        accA = add_f16_f32(__low2half(h), accA);
        accB = add_f16_f32(__high2half(h), accB);
    }
};

// Runtime-direction access, for the initialisation and state-transfer kernels.
template <typename S, typename V>
__device__ __forceinline__ V pop_load(const S* p, int d, int plane, int node, float scale) {
    using PS = PopStore<S>;
    if (d == 0) return (V)PS::load_rest(PS::rest(p), node);
    return (V)PS::load_moving(PS::moving(p, plane), (d - 1) * plane + node, scale);
}
template <typename S, typename V>
__device__ __forceinline__ void pop_store(S* p, int d, int plane, int node, V v, float scale) {
    using PS = PopStore<S>;
    if (d == 0) PS::store_rest(PS::rest(p), node, v);
    else PS::store_moving(PS::moving(p, plane), (d - 1) * plane + node, v, scale);
}

template <typename T, typename S>
struct StepBuffers {
    const S* Nin;
    const S* Bin;
    S* Nout;
    S* Bout;
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

// Block tiles of the step kernels in the shapes the batch autotuner chooses
// between (V = 0 is the one-node single-domain kernel's tile), in nodes:
//   V                 0        1        2        3        4        5
//   D3Q19           32x4x2   32x2x4   32x8x1   32x2x2   32x4x4   64x2x2
//   D2Q9            32x8     64x4     128x2    32x4     32x16    64x4
//   threads (float)  128      256      256      64       512      128
//   threads (FP64)   256      256      256      128      512      256
// Float arithmetic runs shapes 0, 3 and 5 with the two-node kernel
// (k_step_pair_batched, PairTile: two x-adjacent nodes per thread); shape 5 is
// also the tile of the single-domain two-node kernel (k_step_pair).
constexpr int kTileVariants = 6;
constexpr int kPhiRows = kTileVariants;     // the batch color kernel on row chunks (k_phi_rows_batched)
constexpr int kPhiChunk = 128;              // nodes per block of the color kernels over row chunks
__host__ __device__ constexpr int tile_extent(int Q, int V, int axis) {
    return V == 5 ? (axis == 0 ? 64 : axis == 1 ? (Q == 9 ? 4 : 2) : (Q == 9 ? 1 : 2))
         : Q == 9 ? (axis == 0 ? (V == 1 ? 64 : (V == 2 ? 128 : 32))
                               : axis == 1 ? (V == 0 ? 8 : (V == 1 ? 4 : (V == 2 ? 2 : (V == 3 ? 4 : 16)))) : 1)
                  : (axis == 0 ? 32
                               : axis == 1 ? (V == 0 ? 4 : (V == 1 ? 2 : (V == 2 ? 8 : (V == 3 ? 2 : 4))))
                                           : (V == 0 ? 2 : (V == 1 ? 4 : (V == 2 ? 1 : (V == 3 ? 2 : 4)))));
}
template <int Q, int V = 0>
struct Tile {
    static constexpr int D = Lattice<Q>::D;
    static constexpr int TX = tile_extent(Q, V, 0);
    static constexpr int TY = tile_extent(Q, V, 1);
    static constexpr int TZ = tile_extent(Q, V, 2);
    // halo tile: x from x0 - XO (a multiple of 4 for tiled TMA copies) to
    // x0 + TX + XO - 1, y and z one node beyond the tile on each side
    static constexpr int XO = 4;
    static constexpr int HX = TX + 2 * XO;
    static constexpr int HY = TY + 2;
    static constexpr int HZ = (D == 2) ? 1 : TZ + 2;
    static constexpr int HN = HX * HY * HZ;
    static constexpr int BX = TX;              // threads along x: one node each
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

// Linear offsets (32-bit) from node (x, y, z) to its periodic lattice
// neighbours, rows px apart.
struct Wrap {
    int xm, xp, ym, yp, zm, zp;
    __device__ __forceinline__ Wrap(int x, int y, int z, int nx, int ny, int nz, int px) {
        xm = (x == 0) ? nx - 1 : -1;
        xp = (x == nx - 1) ? 1 - nx : 1;
        ym = (y == 0) ? (ny - 1) * px : -px;
        yp = (y == ny - 1) ? (1 - ny) * px : px;
        const int sz = px * ny;
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
// One 4- or 8-byte value global -> shared without a register round trip
// (cp.async); it lands at the next cp_async_wait_all.
template <typename T>
__device__ __forceinline__ void cp_async_value(T* dst_shared, const T* src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async copies 4, 8 or 16 bytes");
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_shared);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"((int)sizeof(T)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---- tiled TMA copies of the halo tile (cp.async.bulk.tensor), completed on
// a shared-memory mbarrier.  A tile uses them only when its whole halo lies
// inside the grid (no periodic image needed) and the grid's rows are a
// multiple of 16 bytes; the copy origin x0 - 4 is then a multiple of 4 floats.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_addr(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(smem_addr(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}
// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for phase `parity` of the barrier; false once timeout_ns have passed
// since the first unsuccessful poll, or after kMbarSpins polls, whichever
// comes first (the caller then flags an error instead of waiting on).  A
// copy that has landed is seen at the first poll, without reading the timer.
constexpr int kMbarSpins = 1 << 22;
constexpr uint64_t kMbarTimeoutNs = 1000000000ull;     // 1 s: a halo copy takes microseconds
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, uint64_t timeout_ns = kMbarTimeoutNs) {
    uint64_t t0 = 0;
    for (int k = 0; k < kMbarSpins; ++k) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if ((k & 15) == 0) {
            const uint64_t t = globaltimer_ns();
            if (k == 0) t0 = t;
            else if (t - t0 >= timeout_ns) return false;
        }
    }
    return false;
}
// error flag bits: 1 = non-finite value, 2 = a halo copy did not complete,
// 4 = an index out of range (debug bounds-check builds only)
constexpr int kErrNonFinite = 1, kErrCopyTimeout = 2, kErrBounds = 4;

// ---- debug bounds checks.  Built with LBM_DEBUG_BOUNDS, every index the step
// kernels compute for a device access is tested against its array first: a
// bad index sets kErrBounds in the domain's error word (the host reports
// LBM_ERR_BOUNDS) and the access is skipped -- a load reads element 0
// instead, a store is dropped.  Nothing traps.  Without the flag the tests
// are constant true and compile away.
#ifdef LBM_DEBUG_BOUNDS
constexpr bool kDebugBounds = true;
#else
constexpr bool kDebugBounds = false;
#endif
__device__ __forceinline__ bool idx_ok(long long idx, long long n, int* err) {
    if (kDebugBounds && (idx < 0 || idx >= n)) {
        if (err) atomicOr(err, kErrBounds);
        return false;
    }
    return true;
}
template <typename I>
__device__ __forceinline__ I idx_checked(I idx, long long n, int* err) {
    return idx_ok((long long)idx, n, err) ? idx : I(0);
}

// Issues the copies of the halo tile; the caller waits (cp_async_wait_all,
// then a barrier) before reading it.
template <class Tl, typename T, bool LOAD_U>
__device__ __forceinline__ void load_halo(const StepParams<T>& P, const T* __restrict__ phi,
                                          const T* __restrict__ u, T* s_phi, T* s_u, int x0, int y0, int z0,
                                          int* err) {
    // one warp per halo row (fixed hy, hz): the row's periodic y/z image is
    // computed once, lanes walk the row's HX consecutive x positions
    constexpr int D = Tl::D;
    constexpr int ROWS = Tl::HY * Tl::HZ;
    constexpr int WARPS = Tl::THREADS / 32;
    const int tid = threadIdx.x + Tl::BX * (threadIdx.y + Tl::TY * threadIdx.z);
    const int warp = tid >> 5, lane = tid & 31;
    const int uplane = (int)P.plane;
    for (int r = warp; r < ROWS; r += WARPS) {
        const int hy = r % Tl::HY, hz = r / Tl::HY;
        const int gy = wrap_halo(y0 + hy - 1, P.ny);
        const int gz = (D == 2) ? 0 : wrap_halo(z0 + hz - 1, P.nz);
        const int rowbase = P.px * (gy + P.ny * gz);
        const int sbase = Tl::HX * r + Tl::XO - 1;                 // slot of x0 - 1
        for (int e = lane; e < Tl::TX + 2; e += 32) {
            const int node = idx_checked(rowbase + wrap_halo(x0 + e - 1, P.nx), P.plane, err);
            const int slot = idx_checked(sbase + e, Tl::HN, err);
            cp_async_value(s_phi + slot, phi + node);
            if (LOAD_U) {
#pragma unroll
                for (int d = 0; d < D; ++d) cp_async_value(s_u + d * Tl::HN + slot, u + d * uplane + node);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// k_phi: Eq. (phiUpdate) on pulled B*
// ---------------------------------------------------------------------------
template <int Q, typename T, typename S>
__device__ __forceinline__ void phi_node(const StepParams<T>& P, const S* __restrict__ Bst,
                                         const uint32_t* __restrict__ mask, T* __restrict__ phi, int x, int y, int z,
                                         int* err) {
    using L = Lattice<Q>;
    if (x >= P.nx || y >= P.ny || z >= P.nz) return;
    const int node = idx_checked(x + P.px * (y + P.ny * z), P.plane, err);
    const uint32_t m = __ldg(mask + node);
    if (m & MASK_NOT_FLUID) return;
    const Wrap W(x, y, z, P.nx, P.ny, P.nz, P.px);
    const int pl = (int)P.plane;
    using PS = PopStore<S>;
    const auto* mv = PS::moving(Bst, pl);
    // FP64 sums in lattice order, as Eq. (phiUpdate) is written.  The
    // deviation forms sum the moving populations first, in storage units, and
    // add the rest population last: with FP16 storage the moving values lie on
    // a grid coarse enough for their float sum to be exact, so the node's color
    // comes back as k_step wrote it.
    const T rest = (T)PS::load_rest(PS::rest(Bst), node);
    T s = PS::kShift ? T(0) : rest;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int idx = ((m >> i) & 1u) ? (L::opp(i) - 1) * pl + node
                                        : (i - 1) * pl + node + W.off(-L::cx(i), -L::cy(i), -L::cz(i));
        PS::accumulate(mv, idx_checked(idx, (long long)(Q - 1) * pl, err), s);
    }
    if (PS::kShift) s = rest + (PS::kExact ? s : s * T(1.0 / kScaleB));
    // stored deviations B_i - chi_i/2 sum to phi - 1/2
    phi[node] = PS::kShift ? T(0.5) + s : s;
}

template <int Q, typename T, typename S>
__global__ void __launch_bounds__(Tile<Q>::THREADS) k_phi(StepParams<T> P, const S* __restrict__ Bst,
                                                          const uint32_t* __restrict__ mask, T* __restrict__ phi,
                                                          int* err) {
    using Tl = Tile<Q>;
    // tiles in the reverse of k_step's order: the B* that k_step wrote last is
    // still in L2 when this kernel starts
    const int bx = gridDim.x - 1 - blockIdx.x, by = gridDim.y - 1 - blockIdx.y, bz = gridDim.z - 1 - blockIdx.z;
    phi_node<Q, T, S>(P, Bst, mask, phi, bx * Tl::TX + threadIdx.x, by * Tl::TY + threadIdx.y, bz * Tl::TZ + threadIdx.z,
                      err);
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
                                               T exp_eps, T eps, T* __restrict__ phi, int64_t plane, int* err) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n_ghosts) return;
    T phiF = T(0);
#pragma unroll
    for (int k = 0; k < GK; ++k) phiF += g_wt[k * n_ghosts + g] * phi[idx_checked(g_corner[k * n_ghosts + g], plane, err)];
    T phiG;
    if (RULE == 0) {
        phiG = phiF / (phiF + (T(1) - phiF) * exp_eps);
    } else {
        const T a = T(1) + T(0.5) * eps;
        phiG = T(4) * phiF / (a + sqrt(a * a - T(2) * eps * phiF)) - phiF;
    }
    const int32_t gn = g_node[g];
    if (idx_ok(gn, plane, err)) phi[gn] = phiG;
}

// ---------------------------------------------------------------------------
// k_step: stencils, forces, macroscopic fields, collision, segregation
// ---------------------------------------------------------------------------
// Reciprocals: FP64 divides exactly, as the oracle.  FP32 takes the hardware
// approximation (PTX rcp.approx, within 1 ulp): its operands here (the mixture
// density, the mixture inverse viscosity, tau) are positive normal floats, so
// the correctly rounded form's special-case handling buys nothing but
// instructions, and 1 ulp of these factors is far below the float step's
// other rounding.
__device__ __forceinline__ double rcp(double v) { return 1.0 / v; }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float rcp(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ double inv_norm_floor(double g2, double floor) {
    const double gn = sqrt(g2);
    return 1.0 / (gn > floor ? gn : floor);
}
__device__ __forceinline__ float inv_norm_floor(float g2, float floor) {
    return rsqrtf(g2 > floor * floor ? g2 : floor * floor);
}

// FP64 node update written in the order the model is stated (Sec. II and
// Appendix A), as the FP64 oracle evaluates it, so that FP64 results follow the
// oracle to rounding; only the collision uses its closed form.  Inputs are the
// lattice-order sums gs[a] = sum w c_a phi, ls = sum w (phi_i - phi),
// us[a][b] = sum w c_a u_b.
template <int Q, bool CONTRAST>
__device__ __forceinline__ void node_update_literal(const StepParams<double>& P, const double* N, double phi,
                                                    const double* gs, double ls, const double (*us)[3], double* Nst,
                                                    double* Bst, double* u, double& p) {
    using L = Lattice<Q>;
    constexpr int D = L::D;
    const double cs2 = 1.0 / 3.0;
    const double w0 = L::w(0);
    double gphi[3], gu[3][3];
    for (int a = 0; a < 3; ++a) {
        gphi[a] = gs[a] / cs2;
        for (int c = 0; c < 3; ++c) gu[a][c] = us[a][c] / cs2;
    }
    const double lap = ls * (2.0 / cs2);
    const double rho = P.rho_l * phi + P.rho_g * (1.0 - phi);
    double grho[3];
    for (int a = 0; a < 3; ++a) grho[a] = (P.rho_l - P.rho_g) * gphi[a];
    const double nu = 1.0 / (phi / P.nu_l + (1.0 - phi) / P.nu_g);
    const double tau = 0.5 + nu / cs2;
    // force-free velocity and its pressure (Eq. pressureUpdate) for F_p
    double u0[3] = {0.0, 0.0, 0.0};
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (L::cx(i)) u0[0] += N[i] * L::cx(i);
        if (L::cy(i)) u0[1] += N[i] * L::cy(i);
        if (L::cz(i)) u0[2] += N[i] * L::cz(i);
        if (i > 0) s += N[i];
    }
    const double uu0 = u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2];
    const double p0 = (-(w0 / 2.0) * uu0 - (1.0 - P.chi[0]) * cs2 + s * cs2) / (1.0 - w0);
    // Eqs. (surfaceTensionForce), body force, (pressCorrection), (viscCorrection), (totalForce)
    const double mu = (48.0 / P.W) * phi * (1.0 - phi) * (phi - 0.5) + (3.0 * P.W / 2.0) * lap;
    double F[3];
    for (int a = 0; a < 3; ++a) {
        const double Fs = -P.sigma * mu * gphi[a];
        const double Fb = rho * P.g[a];
        double Fp = 0.0, Fv = 0.0;
        if (CONTRAST) {
            Fp = -p0 * grho[a];
            for (int c = 0; c < 3; ++c) Fv += (gu[a][c] + gu[c][a]) * grho[c];
            Fv *= cs2 * (tau - 0.5);
        }
        F[a] = Fv + Fp + Fs + Fb;
    }
    if (D == 2) F[2] = 0.0;
    // Eqs. (velUpdate), (pressureUpdate)
    for (int a = 0; a < 3; ++a) u[a] = u0[a] + F[a] / (2.0 * rho);
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    p = (-(w0 / 2.0) * uu - (1.0 - P.chi[0]) * cs2 + s * cs2) / (1.0 - w0);
    // Eq. (equilibriumDistribution), Eq. (forceGuo)
    double neq[Q], Fi[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double cu = L::cx(i) * u[0] + L::cy(i) * u[1] + L::cz(i) * u[2];
        if (i == 0) neq[i] = P.chi[0] - (1.0 - w0) * p / cs2 - w0 * uu / (2.0 * cs2);
        else neq[i] = P.chi[i] + L::w(i) * (p / cs2 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
        const double cF = L::cx(i) * F[0] + L::cy(i) * F[1] + L::cz(i) * F[2];
        Fi[i] = (L::w(i) / cs2) * cF / rho;
    }
    // Eq. (MRTCOLL) in closed form: N* = Neq + F_i/2 + (1 - 1/tau) sum_k m_k (m_k . (N - Neq)) / |m_k|^2
    // over the traceless second-order rows m_k
    double mf[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const double f = N[i] - neq[i];
        if (D == 2) {
            mf[0] += (cx * cx - cy * cy) * f;
            mf[1] += (cx * cy) * f;
        } else {
            const int c2 = cx * cx + cy * cy + cz * cz;
            mf[0] += (3 * cx * cx - c2) * f;
            mf[1] += (cy * cy - cz * cz) * f;
            mf[2] += (cx * cy) * f;
            mf[3] += (cy * cz) * f;
            mf[4] += (cx * cz) * f;
        }
    }
    const double om = 1.0 - 1.0 / tau;
    // segregation, Eq. (segragationStepBlue), n_phi = grad phi / max(|grad phi|, 1e-6)
    const double gn = sqrt(gphi[0] * gphi[0] + gphi[1] * gphi[1] + gphi[2] * gphi[2]);
    double n[3];
    for (int a = 0; a < 3; ++a) n[a] = gphi[a] / (gn > 1e-6 ? gn : 1e-6);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        double proj;
        if (D == 2) {
            proj = (cx * cx - cy * cy) * mf[0] / 4.0 + (cx * cy) * mf[1] / 4.0;
        } else {
            const int c2 = cx * cx + cy * cy + cz * cz;
            proj = (3 * cx * cx - c2) * mf[0] / 36.0 + (cy * cy - cz * cz) * mf[1] / 12.0 + (cx * cy) * mf[2] / 4.0 +
                   (cy * cz) * mf[3] / 4.0 + (cx * cz) * mf[4] / 4.0;
        }
        Nst[i] = neq[i] + 0.5 * Fi[i] + om * proj;
        const double cn = cx * n[0] + cy * n[1] + cz * n[2];
        const double neq0 = P.chi[i] + L::w(i) * (p / cs2);
        Bst[i] = phi * Nst[i] + 2.0 * (cn / P.W) * phi * (1.0 - phi) * neq0;
    }
}

// The pull of the post-streaming populations N of node (x, y, z), issued
// before the node's mask is known: every direction by streaming (x - c_i
// always lies in the grid), then the directions whose neighbour is not fluid
// are read again from the node's own opposite slot.  B enters the collision
// only through phi = sum B, which k_phi computed.  Values come in storage
// units (times kScaleN with FP16 storage).  Only the literal FP64 update reads
// the rest population: in the deviation form the pressure and every moment
// come from the moving populations (Eq. pressureUpdate), so N[0] is not read.
template <int Q, typename T, typename S>
__device__ __forceinline__ void pull_streaming(const StepParams<T>& P, const S* __restrict__ Nin, int node, int x,
                                               int y, int z, T (&N)[Q], int* err) {
    using L = Lattice<Q>;
    using PS = PopStore<S>;
    const Wrap Wr(x, y, z, P.nx, P.ny, P.nz, P.px);
    const int pl = (int)P.plane;
    N[0] = PS::kShift ? T(0) : (T)PS::load_rest(PS::rest(Nin), idx_checked(node, P.plane, err));
    const auto* mv = PS::moving(Nin, pl);
#pragma unroll
    for (int i = 1; i < Q; ++i)
        N[i] = (T)PS::load_units(mv, idx_checked((i - 1) * pl + node + Wr.off(-L::cx(i), -L::cy(i), -L::cz(i)),
                                                 (long long)(Q - 1) * pl, err));
}
template <int Q, typename T, typename S>
__device__ __forceinline__ void pull_bounce_back(const StepParams<T>& P, const S* __restrict__ Nin, uint32_t m,
                                                 int node, T (&N)[Q], int* err) {
    using L = Lattice<Q>;
    using PS = PopStore<S>;
    const int pl = (int)P.plane;
    const auto* mv = PS::moving(Nin, pl);
#pragma unroll
    for (int i = 1; i < Q; ++i)
        if ((m >> i) & 1u) N[i] = (T)PS::load_units(mv, idx_checked((L::opp(i) - 1) * pl + node,
                                                                    (long long)(Q - 1) * pl, err));
}

// Value types of the float node update.  SF is a float whose every
// operation is rounded on its own (round to nearest, never fused unless
// written as fma): the one-node kernels' type.  F2 holds the same value for
// two nodes in one 64-bit register pair and operates on both lanes with one
// packed instruction (PTX add/sub/mul/fma .rn .f32x2, sm_100 and later):
// the two-node kernel's type.  Each packed lane rounds exactly as the SF
// operation does, so one source of the update gives both kernels the same
// results to the bit, and the two-node kernel issues one float instruction
// where the one-node kernel issues two.
struct SF {
    float v;
    __device__ __forceinline__ SF() {}
    __device__ __forceinline__ SF(float x) : v(x) {}
};
__device__ __forceinline__ SF operator+(SF a, SF b) { return SF(__fadd_rn(a.v, b.v)); }
__device__ __forceinline__ SF operator-(SF a, SF b) { return SF(__fsub_rn(a.v, b.v)); }
__device__ __forceinline__ SF operator*(SF a, SF b) { return SF(__fmul_rn(a.v, b.v)); }
__device__ __forceinline__ SF operator-(SF a) { return SF(-a.v); }
__device__ __forceinline__ SF fma(SF a, SF b, SF c) { return SF(fmaf(a.v, b.v, c.v)); }
__device__ __forceinline__ SF rcp(SF a) { return SF(rcp(a.v)); }
__device__ __forceinline__ SF inv_norm_floor(SF g2, float floor) { return SF(inv_norm_floor(g2.v, floor)); }

struct F2 {
    unsigned long long v;                       // lane 0 (node A) low, lane 1 (node B) high
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(float a) { asm("mov.b64 %0, {%1, %1};" : "=l"(v) : "f"(a)); }
    __device__ __forceinline__ F2(float a, float b) { asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(a), "f"(b)); }
    __device__ __forceinline__ float lo() const {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
        return a;
    }
    __device__ __forceinline__ float hi() const {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
        return b;
    }
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) {
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
// -x exactly (sign flip, zeros included), as the scalar negation
__device__ __forceinline__ F2 operator-(F2 a) { return a * F2(-1.0f); }
__device__ __forceinline__ F2 rcp(F2 a) { return F2(rcp(a.lo()), rcp(a.hi())); }
__device__ __forceinline__ F2 inv_norm_floor(F2 g2, float floor) {
    return F2(inv_norm_floor(g2.lo(), floor), inv_norm_floor(g2.hi(), floor));
}

// a + k t for an integer coefficient k that is a constant once the direction
// loops are unrolled: k = 0 emits nothing, k = +/-1 no multiply, and the first
// term is taken as it is rather than added to a zero (IEEE addition of +0 is
// not the identity for -0, so the compiler keeps such adds).  The value is the
// sum the same terms give in the same order, started from zero.
template <typename V>
struct Acc {
    V v = V(0.f);
    bool set = false;
    __device__ __forceinline__ void add(int k, V t) {
        if (k == 0) return;
        if (!set) {
            v = k == 1 ? t : (k == -1 ? -t : V(float(k)) * t);
        } else {
            v = k == 1 ? v + t : (k == -1 ? v - t : fma(V(float(k)), t, v));
        }
        set = true;
    }
    __device__ __forceinline__ V get() const { return set ? v : V(0.f); }
};

// ---------------------------------------------------------------------------
// Float arithmetic of one fluid node (V = SF), or of the two nodes of a pair
// (V = F2, one packed lane each), written once so that the one-node and the
// two-node kernels round alike.  Inputs: the pulled populations N
// (deviations, in storage units with FP16 storage), the color phi at the node
// and its isotropic stencils gp = grad phi, lap = lap phi and gu[a][b] = d_a u_b
// (the stencil weights carry the 3 and the 6).
//
// Every operation of V rounds on its own and fuses only where written as fma,
// so the compiler has no choice of what to fuse: every kernel that inlines
// this code computes the same values.
// ---------------------------------------------------------------------------
template <int Q, bool UNITS, bool CONTRAST, typename V>
struct FloatNode {
    using L = Lattice<Q>;
    static constexpr int D = L::D;
    static constexpr double w0 = L::w(0);
    // storage units: times sN (N) and sB (B), 2^16 and 2^7 with FP16 storage,
    // else 1.  Being powers of two, the scales fold into the per-node factors
    // (the stress projections, the weights, phi, kseg) and the scaled values
    // round exactly as the unscaled ones would.
    static constexpr float sN = UNITS ? kScaleN : 1.0f, sB = UNITS ? kScaleB : 1.0f;
    V phi, u[3], uu, p;
    V F[3], gp[3];
    V A0, A1, Axy, Axz, Ayz;                   // stress projections of N - Neq, times (1 - 1/tau)
    V base0, base1, base2, three_p, halfF;
    V common1, common2, krc1, krc2;            // per direction class (1 axis, 2 diagonal/edge)
    V shb1, shb2;                              // (phi - 1/2) chi_i per class, in B's units
    V phiB;

    // raw moments of the pulled N (storage units): sum, first and second moments
    V m_sum, m_u0[3], m_xx, m_yy, m_zz, m_xy, m_xz, m_yz;

    // The moments need only the pulled populations, not the halo: the two-node
    // kernel takes them before its barrier, so that the pulled values are not
    // held across the stencils.
    __device__ __forceinline__ void moments(const V (&N)[Q]) {
        // force-free velocity and the moments of Eq. (pressureUpdate) and the collision
        Acc<V> u0s[3], sm, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
            // odd moments from N_i - N_opp, even ones from N_i + N_opp
            if (L::opp(i) < i) continue;
            const V sp = N[i] + N[L::opp(i)], dp = N[i] - N[L::opp(i)];
            sm.add(1, sp);
            u0s[0].add(cx, dp);
            u0s[1].add(cy, dp);
            u0s[2].add(cz, dp);
            Pxx.add(cx * cx, sp);
            Pyy.add(cy * cy, sp);
            Pzz.add(cz * cz, sp);
            Pxy.add(cx * cy, sp);
            Pxz.add(cx * cz, sp);
            Pyz.add(cy * cz, sp);
        }
        m_sum = sm.get();
#pragma unroll
        for (int a = 0; a < 3; ++a) m_u0[a] = u0s[a].get();
        m_xx = Pxx.get(); m_yy = Pyy.get(); m_zz = Pzz.get();
        m_xy = Pxy.get(); m_xz = Pxz.get(); m_yz = Pyz.get();
    }

    __device__ __forceinline__ void compute(const StepParams<float>& P, const V (&N)[Q], V phi_, const V (&gp_)[3],
                                            V lap, const V (&gu)[3][3]) {
        moments(N);
        compute(P, phi_, gp_, lap, gu);
    }

    // the rest of the node update, after moments()
    __device__ __forceinline__ void compute(const StepParams<float>& P, V phi_, const V (&gp_)[3], V lap,
                                            const V (&gu)[3][3]) {
        phi = phi_;
#pragma unroll
        for (int a = 0; a < 3; ++a) gp[a] = gp_[a];

        // mixture density and viscosity (Sec. II), relaxation time (Appendix A)
        const V rho = fma(V(P.drho), phi, V(P.rho_g));
        const V inv_rho = rcp(rho);
        const V nu = rcp(fma(phi, V(P.inv_nu_l - P.inv_nu_g), V(P.inv_nu_g)));   // 1 / (phi/nu_l + (1-phi)/nu_g)
        const V tau = fma(V(3.0f), nu, V(0.5f));

        // FP16 storage: N came in storage units (times sN = 2^16); the moments are
        // linear in N, so the scale is taken out where each is used (exactly, a
        // power of two): here for u0 and the pressure, in the stress projections
        // below for the second moments
        constexpr float r = 1.0f / sN;
        V u0[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) u0[a] = (a < D) ? (UNITS ? m_u0[a] * V(r) : m_u0[a]) : V(0.f);
        // Eq. (pressureUpdate) takes sum_{i>0} N_i - (1 - chi_0) with the exact
        // chi; the deviations are stored from the rounded chi of the storage, whose
        // moving values sum to 1 - chi[0], so the difference of the two is
        // chi_0 - chi[0], the rest class's correction (without it the float
        // pressure would sit a constant ~4e-8 off, which F_p = -p grad(rho)
        // turns into a velocity error at a density contrast)
        const V pres_base = (UNITS ? fma(m_sum, V(r), V(P.chi_err[0])) : m_sum + V(P.chi_err[0])) *
                            V(float(1.0 / 3.0));
        const V inv_1mw0 = V(float(1.0 / (1.0 - w0)));

        // forces: surface tension and body force, then (density contrast) the
        // pressure and viscous corrections
        const V muc = fma(V(P.k3W2), lap, V(P.k48W) * phi * (V(1.0f) - phi) * (phi - V(0.5f)));   // chemical potential / sigma
        const V smu = V(-P.sigma) * muc;
#pragma unroll
        for (int a = 0; a < D; ++a) F[a] = fma(smu, gp[a], rho * V(P.g[a]));
        if (D == 2) F[2] = V(0.f);
        if (CONTRAST) {
            // F_p = -p0 grad(rho), F_v = nu (grad u + grad u^T) . grad(rho), grad(rho) = drho grad(phi)
            const V uu0 = D == 2 ? fma(u0[0], u0[0], u0[1] * u0[1])
                                 : fma(u0[0], u0[0], fma(u0[1], u0[1], u0[2] * u0[2]));
            const V p0 = fma(V(-float(0.5 * w0)), uu0, pres_base) * inv_1mw0;
            const V kd = (tau - V(0.5f)) * V(float(1.0 / 3.0)) * V(P.drho), pd = -p0 * V(P.drho);
            V sv[3];
            if (D == 2) {
                const V t01 = gu[0][1] + gu[1][0];
                sv[0] = fma(t01, gp[1], (gu[0][0] + gu[0][0]) * gp[0]);
                sv[1] = fma(t01, gp[0], (gu[1][1] + gu[1][1]) * gp[1]);
            } else {
                const V t01 = gu[0][1] + gu[1][0], t02 = gu[0][2] + gu[2][0], t12 = gu[1][2] + gu[2][1];
                sv[0] = fma(t02, gp[2], fma(t01, gp[1], (gu[0][0] + gu[0][0]) * gp[0]));
                sv[1] = fma(t12, gp[2], fma(t01, gp[0], (gu[1][1] + gu[1][1]) * gp[1]));
                sv[2] = fma(t12, gp[1], fma(t02, gp[0], (gu[2][2] + gu[2][2]) * gp[2]));
            }
#pragma unroll
            for (int a = 0; a < D; ++a) F[a] = fma(kd, sv[a], fma(pd, gp[a], F[a]));
        }

        // Eq. (velUpdate), Eq. (pressureUpdate)
        const V hr = V(0.5f) * inv_rho;
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = (a < D) ? fma(F[a], hr, u0[a]) : V(0.f);
        uu = D == 2 ? fma(u[0], u[0], u[1] * u[1]) : fma(u[0], u[0], fma(u[1], u[1], u[2] * u[2]));
        p = fma(V(-float(0.5 * w0)), uu, pres_base) * inv_1mw0;

        // collision: traceless second moments of N - Neq, with sum Neq c c = (c2chi + p) I + u u,
        // in N's storage units (the moments are raw, the u u terms take the scale)
        const V omega1 = V(1.0f) - rcp(tau);                                        // 1 - s_nu
        const V o4 = omega1 * V(0.25f);
        base0 = V(3.0f) * u[0];
        base1 = V(3.0f) * u[1];
        base2 = V(3.0f) * u[2];
        if (D == 2) {
            A0 = o4 * fma(V(-sN), fma(u[0], u[0], -(u[1] * u[1])), m_xx - m_yy);   // m7 . f / |m7|^2
            A1 = V(0.f);
            Axy = o4 * fma(V(-sN) * u[0], u[1], m_xy);                              // m8 . f / |m8|^2
            Axz = Ayz = V(0.f);
        } else {
            // 2 ux^2 - uy^2 - uz^2 = 3 ux^2 - u.u
            A0 = (omega1 * V(float(1.0 / 36.0))) * fma(V(-sN), fma(base0, u[0], -uu), fma(V(2.0f), m_xx, -m_yy) - m_zz);
            A1 = (omega1 * V(float(1.0 / 12.0))) * fma(V(-sN), fma(u[1], u[1], -(u[2] * u[2])), m_yy - m_zz);
            const V su0 = V(-sN) * u[0];
            Axy = o4 * fma(su0, u[1], m_xy);
            Axz = o4 * fma(su0, u[2], m_xz);
            Ayz = o4 * fma(V(-sN) * u[1], u[2], m_yz);
        }

        // segregation: n_phi = grad phi / max(|grad phi|, 1e-6)
        const V g2 = D == 2 ? fma(gp[0], gp[0], gp[1] * gp[1]) : fma(gp[0], gp[0], fma(gp[1], gp[1], gp[2] * gp[2]));
        const V inv_gn = inv_norm_floor(g2, 1e-6f);
        const V kseg = V(P.two_over_W) * phi * (V(1.0f) - phi) * inv_gn;
        const V ksegB = UNITS ? kseg * V(sB) : kseg;                        // recoloring in B's units
        phiB = UNITS ? phi * V(sB / sN) : phi;                              // phi N*, from N's units to B's
        const V phmB = UNITS ? (phi - V(0.5f)) * V(sB) : phi - V(0.5f);
        shb1 = phmB * V(P.chi[1]);
        shb2 = phmB * V(P.chi[D == 2 ? 5 : 7]);
        three_p = V(3.0f) * p;
        halfF = V(1.5f) * inv_rho;   // (1/2) F_i = (3/2) w_i (c_i . F)/rho
        const V common = fma(V(-1.5f), uu, three_p);
        // per direction class (1 axis, 2 diagonal/edge): the equilibrium's constant
        // part w_i (3p - 3u^2/2) + (chi_i - stored chi_i), divided by w_i, and the
        // recolouring weight ksegB (chi_i + w_i 3p) with the exact chi_i
        constexpr double kW1 = L::w(1), kW2 = L::w(D == 2 ? 5 : 7);
        common1 = fma(V(P.chi_err[1]), V(float(1.0 / kW1)), common);
        common2 = fma(V(P.chi_err[2]), V(float(1.0 / kW2)), common);
        krc1 = ksegB * fma(V(float(kW1)), three_p, V(P.chi[1] + P.chi_err[1]));
        krc2 = ksegB * fma(V(float(kW2)), three_p, V(P.chi[D == 2 ? 5 : 7] + P.chi_err[2]));
    }

    // Direction i (opp(i) > i) and its opposite o, in storage units: the
    // post-collision N*_i - chi_i, N*_o - chi_o (they share the even part and
    // flip the odd part) and B*_i - chi_i/2, B*_o - chi_o/2 with
    // B* = phi N* + recolor, i.e. phi dN* + (phi - 1/2) chi_i + recolor.
    __device__ __forceinline__ void dir(int i, V& ni, V& no, V& bi, V& bo) const {
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const float wiN = float(L::w(i)) * sN;
        // the stress projection, 3 c.u, c.F and c.grad phi, each without the terms
        // whose lattice coefficient is zero
        Acc<V> proj, cu3, cF, cg;
        if (D == 2) {
            proj.add(cx * cx - cy * cy, A0);
            proj.add(cx * cy, Axy);
        } else {
            const int c2 = cx * cx + cy * cy + cz * cz;
            proj.add(3 * cx * cx - c2, A0);
            proj.add(cy * cy - cz * cz, A1);
            proj.add(cx * cy, Axy);
            proj.add(cx * cz, Axz);
            proj.add(cy * cz, Ayz);
        }
        cu3.add(cx, base0); cF.add(cx, F[0]); cg.add(cx, gp[0]);
        cu3.add(cy, base1); cF.add(cy, F[1]); cg.add(cy, gp[1]);
        cu3.add(cz, base2); cF.add(cz, F[2]); cg.add(cz, gp[2]);
        const bool axis = cx * cx + cy * cy + cz * cz == 1;
        const V krc = axis ? krc1 : krc2, g = cg.get();                // recoloring krc (c . grad phi), odd in c
        const V c3 = cu3.get();
        const V even = fma(V(wiN), fma(V(0.5f) * c3, c3, axis ? common1 : common2), proj.get());
        const V odd = fma(halfF, cF.get(), c3);                        // the odd part over wiN
        ni = fma(V(wiN), odd, even);
        no = fma(V(-wiN), odd, even);
        const V shift_b = axis ? shb1 : shb2;                          // (phi - 1/2) chi_i
        bi = fma(krc, g, fma(phiB, ni, shift_b));
        bo = fma(-krc, g, fma(phiB, no, shift_b));
    }

    // Rest direction (no forcing, no stress projection, no recoloring, c_0 = 0),
    // stored exactly (FP32): N*_0 - chi_0 and B*_0 - chi_0/2.
    __device__ __forceinline__ V rest_N(const StepParams<float>& P) const {
        return fma(V(-float(1.5 * w0)), uu, fma(V(-float(1.0 - w0)), three_p, V(P.chi_err[0])));
    }
    __device__ __forceinline__ V rest_B(const StepParams<float>& P, V nst0) const {
        return fma(phi, nst0, (phi - V(0.5f)) * V(P.chi[0]));
    }
    // With FP16 storage the float rest populations take the node totals the
    // collision fixes less the moving populations as stored (sumN, sumB in
    // storage units, one node each): sum_i (N*_i - chi_i) = 0 for any N, u, p
    // and F (the equilibrium sums to sum chi = 1; the stress projection and the
    // forcing have no zeroth moment) and sum_i (B*_i - chi_i/2) = phi - 1/2 (the
    // recoloring is odd in c), so FP16 rounding moves no mass between the
    // phases or out of the domain.
    __device__ __forceinline__ static float rest_N_from_sum(float sumN) { return -sumN * (1.0f / kScaleN); }
    __device__ __forceinline__ static float rest_B_from_sum(float sumB, float phi_node) {
        return fmaf(-sumB, 1.0f / kScaleB, phi_node - 0.5f);
    }
};

// One fluid node of the step: pulled populations N, the block's halo tile.
template <int Q, int V, typename T, typename S, bool CONTRAST>
__device__ __forceinline__ void step_node(const StepParams<T>& P, const StepBuffers<T, S>& b,
                                          const T* __restrict__ s_phi, const T* __restrict__ s_u, const T (&N)[Q],
                                          int node) {
    using L = Lattice<Q>;
    using Tl = Tile<Q, V>;
    constexpr int D = L::D;
    const int hc = (threadIdx.x + Tl::XO) + Tl::HX * ((threadIdx.y + 1) + Tl::HY * (D == 2 ? 0 : threadIdx.z + 1));
    const int pl = (int)P.plane;
    int* const err = b.err;
    // every store index below is a direction's plane offset plus this node
    if (!idx_ok(node, P.plane, err)) return;
    using PS = PopStore<S>;
    constexpr bool kShift = PS::kShift;

    // isotropic stencils: grad f = 3 sum_i w_i c_i f(x+c_i), lap f = 6 sum_i w_i (f(x+c_i) - f(x)).
    // FP32 sums over +/- pairs (half the multiply-adds); FP64, the mode checked
    // against the FP64 oracle to 1e-12 over thousands of steps, sums in lattice
    // order as the definition is written.
    constexpr bool kPairs = sizeof(T) == 4;
    const T phi = s_phi[idx_checked(hc, Tl::HN, err)];
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
            // each difference enters every component it feeds with one
            // multiply-add by the constant c_ia w_i
            const T pp = s_phi[idx_checked(hp, Tl::HN, err)], pm = s_phi[idx_checked(hm, Tl::HN, err)];
            const T dphi = pp - pm;
            // the weights carry the 3 of the gradient and the 6 of the laplacian
            const T g3 = T(3.0 * L::w(i)), l6 = T(6.0 * L::w(i));
            if (cx) gp[0] = fmadd(T(cx) * g3, dphi, gp[0]);
            if (cy) gp[1] = fmadd(T(cy) * g3, dphi, gp[1]);
            if (cz) gp[2] = fmadd(T(cz) * g3, dphi, gp[2]);
            lsum = fmadd(l6, (pp - phi) + (pm - phi), lsum);
            if (CONTRAST) {
#pragma unroll
                for (int bb = 0; bb < D; ++bb) {
                    const T dub = s_u[idx_checked(bb * Tl::HN + hp, D * Tl::HN, err)] -
                                  s_u[idx_checked(bb * Tl::HN + hm, D * Tl::HN, err)];
                    if (cx) du[0][bb] = fmadd(T(cx) * g3, dub, du[0][bb]);
                    if (cy) du[1][bb] = fmadd(T(cy) * g3, dub, du[1][bb]);
                    if (cz) du[2][bb] = fmadd(T(cz) * g3, dub, du[2][bb]);
                }
            }
        } else {
            const int h = hc + Tl::off(cx, cy, cz);
            const T ph = s_phi[idx_checked(h, Tl::HN, err)];
            gp[0] += wi * T(cx) * ph;
            gp[1] += wi * T(cy) * ph;
            if (D == 3) gp[2] += wi * T(cz) * ph;
            lsum += wi * (ph - phi);
            if (CONTRAST) {
#pragma unroll
                for (int bb = 0; bb < D; ++bb) {
                    const T ub = s_u[idx_checked(bb * Tl::HN + h, D * Tl::HN, err)];
                    du[0][bb] += wi * T(cx) * ub;
                    du[1][bb] += wi * T(cy) * ub;
                    if (D == 3) du[2][bb] += wi * T(cz) * ub;
                }
            }
        }
    }
    constexpr double w0 = L::w(0);
    if constexpr (sizeof(T) == 8) {
        double Ns[Q], Bs[Q], u[3], p;
        node_update_literal<Q, CONTRAST>(P, N, phi, gp, lsum, du, Ns, Bs, u, p);
        PS::store_rest(PS::rest(b.Nout), node, Ns[0]);
        PS::store_rest(PS::rest(b.Bout), node, Bs[0]);
        auto* Nmv = PS::moving(b.Nout, pl);
        auto* Bmv = PS::moving(b.Bout, pl);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            PS::store_moving(Nmv, (i - 1) * pl + node, Ns[i], kScaleN);
            PS::store_moving(Bmv, (i - 1) * pl + node, Bs[i], kScaleB);
        }
#pragma unroll
        for (int a = 0; a < D; ++a) b.u_out[a * pl + node] = u[a];
        b.p[node] = p;
        if (!(u[0] * u[0] + u[1] * u[1] + u[2] * u[2] < 1e30)) atomicOr(b.err, kErrNonFinite);
        return;
    } else {
    static_assert(kPairs && kShift, "float arithmetic runs on deviations, summed over +/- pairs");
    constexpr bool kUnits = !PS::kExact;
    using FN = FloatNode<Q, kUnits, CONTRAST, SF>;
    FN nd;
    {
        SF Ns[Q], gps[3], gus[3][3];
#pragma unroll
        for (int i = 0; i < Q; ++i) Ns[i] = SF(N[i]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gps[a] = SF(gp[a]);
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) gus[a][bb] = SF(du[a][bb]);
        }
        nd.compute(P, Ns, SF(phi), gps, SF(lsum), gus);
    }

    // u and p: FP16 storage writes them before the populations, which frees
    // their registers for the stored sums (no spills in the batched kernels);
    // FP32 writes them last, measured 0.7% faster
    auto store_u_p = [&]() {
#pragma unroll
        for (int a = 0; a < D; ++a) b.u_out[a * pl + node] = nd.u[a].v;
        b.p[node] = nd.p.v;
        if (!(nd.uu.v < T(1e30))) atomicOr(b.err, kErrNonFinite);   // also catches NaN
    };
    if constexpr (!PS::kExact) store_u_p();

    auto* __restrict__ Nmov = PS::moving(b.Nout, pl);
    auto* __restrict__ Bmov = PS::moving(b.Bout, pl);
    if constexpr (PS::kExact) {
        const SF nst0 = nd.rest_N(P);
        PS::store_rest(PS::rest(b.Nout), node, nst0.v);
        PS::store_rest(PS::rest(b.Bout), node, nd.rest_B(P, nst0).v);
    }
    // sums of the moving populations as stored (FP16 storage)
    T sumN = T(0), sumB = T(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (L::opp(i) < i) continue;
        const int o = L::opp(i);
        SF ni, no, bi, bo;
        nd.dir(i, ni, no, bi, bo);
        PS::store_units(Nmov, (i - 1) * pl + node, ni.v, sumN);
        PS::store_units(Nmov, (o - 1) * pl + node, no.v, sumN);
        PS::store_units(Bmov, (i - 1) * pl + node, bi.v, sumB);
        PS::store_units(Bmov, (o - 1) * pl + node, bo.v, sumB);
    }
    if constexpr (!PS::kExact) {
        PS::store_rest(PS::rest(b.Nout), node, FN::rest_N_from_sum(sumN));
        PS::store_rest(PS::rest(b.Bout), node, FN::rest_B_from_sum(sumB, nd.phi.v));
    }
    if constexpr (PS::kExact) store_u_p();
    }
}

// The periodic images of x = -1 and x = nx that a block at an x end of the
// grid patches into its halo after a tiled copy: one per halo row and field
// at each end, K per thread (1 unless the block has fewer threads than both
// ends' images).
template <class Tl, typename T, bool CONTRAST>
struct HaloFix {
    static constexpr int kFields = CONTRAST ? 1 + Tl::D : 1;
    static constexpr int kRows = Tl::HY * Tl::HZ;
    static constexpr int kPerCol = kRows * kFields;
    static constexpr int K = (2 * kPerCol + Tl::THREADS - 1) / Tl::THREADS;
    T v[K];
    int at[K];                                 // halo slot (phi, then the u fields), or -1
};

// A block's halo tile (color, and the previous velocity with a density
// contrast) with a one-node ring: issued by halo_issue, waited for by
// halo_complete, shared by the step kernels of every tile shape.  With maps
// (tiles whose halo needs no periodic image in y and z) two tiled TMA copies
// fill it, completed on the mbarrier `bar`; at the x ends of the grid the box
// reads zeros where x < 0 or x >= nx, and the stencil needs the periodic
// images of x = -1 and x = nx there: the threads load those values now (fx)
// and write them once the copy has landed.  Without maps the halo is copied
// element by element with cp.async.  halo_issue returns false when the debug
// bounds checks reject the tile's box.
template <class Tl, typename T, typename S, bool CONTRAST>
__device__ __forceinline__ bool halo_issue(const StepParams<T>& P, const StepBuffers<T, S>& b, T* s_phi, T* s_u,
                                           int x0, int y0, int z0, const CUtensorMap* tm_phi,
                                           const CUtensorMap* tm_u, uint64_t* bar, HaloFix<Tl, T, CONTRAST>& fx) {
    using Fx = HaloFix<Tl, T, CONTRAST>;
    const bool tma = tm_phi != nullptr;
#pragma unroll
    for (int j = 0; j < Fx::K; ++j) {
        fx.v[j] = T(0);
        fx.at[j] = -1;
    }
    constexpr int kHaloFields = Fx::kFields;
    if (tma && kDebugBounds) {
        // the box of a tiled copy: x origin on a 16-byte boundary, the whole
        // halo inside the grid in y and z (no periodic image needed there)
        const bool box_ok = ((x0 - Tl::XO) & 3) == 0 && y0 >= 1 && y0 + Tl::TY + 1 <= P.ny &&
                            (Tl::D == 2 || (z0 >= 1 && z0 + Tl::TZ + 1 <= P.nz));
        if (!box_ok) {
            if (threadIdx.x + threadIdx.y + threadIdx.z == 0) atomicOr(b.err, kErrBounds);
            return false;                                  // the whole block takes this branch
        }
    }
    if (tma) {
        const int tid = threadIdx.x + Tl::BX * (threadIdx.y + Tl::TY * threadIdx.z);
        if (tid == 0) {
            constexpr unsigned kBytes = (CONTRAST ? 1 + Tl::D : 1) * Tl::HN * sizeof(T);
            mbar_expect_tx(bar, kBytes);
            const int zc = Tl::D == 2 ? 0 : z0 - 1;
            tma_load_3d(s_phi, tm_phi, x0 - Tl::XO, y0 - 1, zc, bar);
            if (CONTRAST) tma_load_4d(s_u, tm_u, x0 - Tl::XO, y0 - 1, zc, 0, bar);
        }
        const bool lo = x0 == 0, hi = x0 + Tl::TX >= P.nx;
        constexpr int kRows = Fx::kRows, kPerCol = Fx::kPerCol;
        // image t of both x ends of a one-tile-wide grid at once: thread tid
        // takes t = tid, tid + THREADS, ...
        const int count = (int(lo) + int(hi)) * kPerCol;
#pragma unroll
        for (int j = 0; j < Fx::K; ++j) {
            const int t = tid + j * Tl::THREADS;
            if (t >= count) continue;
            const bool left = lo && t < kPerCol;                // x = -1, else x = nx
            const int k = t % kPerCol, field = k / kRows, r = k % kRows;
            const int hy = r % Tl::HY, hz = r / Tl::HY;
            const int gz = Tl::D == 2 ? 0 : z0 - 1 + hz;
            const int node = (left ? P.nx - 1 : 0) + P.px * (y0 - 1 + hy + P.ny * gz);
            const int fn = idx_checked(node, P.plane, b.err);
            fx.v[j] = field == 0 ? b.phi[fn] : b.u_in[(field - 1) * (int)P.plane + fn];
            fx.at[j] = (field == 0 ? 0 : Tl::HN * field) + (left ? Tl::XO - 1 : P.nx - x0 + Tl::XO) + Tl::HX * r;
            if (!idx_ok(fx.at[j], kHaloFields * Tl::HN, b.err)) fx.at[j] = -1;
        }
    } else {
        load_halo<Tl, T, CONTRAST>(P, b.phi, b.u_in, s_phi, s_u, x0, y0, z0, b.err);
    }
    return true;
}

// Waits for the halo issued by halo_issue and patches the x-end images;
// false if a tiled copy did not complete within the bounded wait.  The
// caller's barrier follows.
template <class Tl, typename T, typename S, class Fx>
__device__ __forceinline__ bool halo_complete(const StepBuffers<T, S>& b, bool tma, uint64_t* bar, T* s_phi,
                                              T* s_u, const Fx& fx) {
    if (!tma) {
        cp_async_wait_all();
        return true;
    }
    const bool halo_ok = mbar_wait(bar, 0);
    if (!halo_ok) {
        // the tile is skipped and the host is told (LBM_ERR_TIMEOUT; the domain
        // is refused further steps).  The copy may still be in flight into
        // this block's shared memory: wait for it once more, again bounded,
        // before the block exits, so that it does not land in a later block.
        if (threadIdx.x + threadIdx.y + threadIdx.z == 0) atomicOr(b.err, kErrCopyTimeout);
        mbar_wait(bar, 0);
    }
#pragma unroll
    for (int j = 0; j < Fx::K; ++j)
        if (halo_ok && fx.at[j] >= 0) (fx.at[j] < Tl::HN ? s_phi : s_u - Tl::HN)[fx.at[j]] = fx.v[j];
    return halo_ok;
}

// The tile at (x0, y0, z0): the halo copies are issued first, then every
// thread pulls its node's populations while they are in flight; after the
// barrier each fluid node is updated.
template <int Q, int V, typename T, typename S, bool CONTRAST>
__device__ __forceinline__ void step_tile(const StepParams<T>& P, const StepBuffers<T, S>& b, T* s_phi, T* s_u,
                                          int x0, int y0, int z0, const CUtensorMap* tm_phi = nullptr,
                                          const CUtensorMap* tm_u = nullptr, uint64_t* bar = nullptr) {
    using Tl = Tile<Q, V>;
    const bool tma = tm_phi != nullptr;
    HaloFix<Tl, T, CONTRAST> fx;
    if (!halo_issue<Tl, T, S, CONTRAST>(P, b, s_phi, s_u, x0, y0, z0, tm_phi, tm_u, bar, fx)) return;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    const bool in_grid = x < P.nx && y < P.ny && z < P.nz;
    const int node = in_grid ? idx_checked(x + P.px * (y + P.ny * z), P.plane, b.err) : 0;
    const uint32_t m = in_grid ? __ldg(b.mask + node) : MASK_NOT_FLUID;
    T N[Q];
    if (in_grid) pull_streaming<Q, T, S>(P, b.Nin, node, x, y, z, N, b.err);      // in flight with the mask load
    const bool fluid = !(m & MASK_NOT_FLUID);
    if (fluid && (m & ~MASK_NOT_FLUID)) pull_bounce_back<Q, T, S>(P, b.Nin, m, node, N, b.err);
    const bool halo_ok = halo_complete<Tl, T, S>(b, tma, bar, s_phi, s_u, fx);
    __syncthreads();
    if (fluid && halo_ok) step_node<Q, V, T, S, CONTRAST>(P, b, s_phi, s_u, N, node);
}

// Resident blocks per SM the step kernels are compiled for (registers per
// thread <= 65536 / (256 * blocks)): measured on the 192^3 bench case, FP32
// and FP16 storage run best at 5 (48 registers, no spills; FP16 storage at 6
// blocks spills at 40 registers and runs 1.5% slower, at 4 it is 4% slower);
// FP64 keeps the compiler's choice.
template <typename T, typename S> struct StepOccupancy { static constexpr int kBlocks = 1; };
template <> struct StepOccupancy<float, float> { static constexpr int kBlocks = 5; };
template <> struct StepOccupancy<float, __half> { static constexpr int kBlocks = 5; };
// the same register budget for other block sizes
template <typename T, typename S, int THREADS>
constexpr int step_min_blocks() {
    return StepOccupancy<T, S>::kBlocks * 256 / THREADS > 0 ? StepOccupancy<T, S>::kBlocks * 256 / THREADS : 1;
}

// tma != 0: the host made tensor maps of phi (nx, ny, nz) and of the previous
// velocity (nx, ny, nz, D) with box (HX, HY, HZ[, D]); tiles whose halo lies
// inside the grid copy it with them.
template <int Q, typename T, typename S, bool CONTRAST, int V = 0>
__global__ void __launch_bounds__(Tile<Q, V>::THREADS, (step_min_blocks<T, S, Tile<Q, V>::THREADS>()))
    k_step(StepParams<T> P, StepBuffers<T, S> b, const __grid_constant__ CUtensorMap tm_phi,
           const __grid_constant__ CUtensorMap tm_u, int tma) {
    using Tl = Tile<Q, V>;
    __shared__ __align__(128) T s_phi[Tl::HN];
    __shared__ __align__(128) T s_u[CONTRAST ? Tl::D * Tl::HN : 1];
    __shared__ __align__(8) uint64_t s_bar;
    const int x0 = blockIdx.x * Tl::TX, y0 = blockIdx.y * Tl::TY, z0 = blockIdx.z * Tl::TZ;
    // tiles whose halo needs no periodic image in y and z (x images are patched in step_tile)
    const bool interior = tma && y0 >= 1 && y0 + Tl::TY + 1 <= P.ny &&
                          (Tl::D == 2 || (z0 >= 1 && z0 + Tl::TZ + 1 <= P.nz));
    if (interior) {
        if (threadIdx.x + threadIdx.y + threadIdx.z == 0) mbar_init(&s_bar, 1);
        __syncthreads();                                      // the barrier exists before anyone waits on it
        step_tile<Q, V, T, S, CONTRAST>(P, b, s_phi, s_u, x0, y0, z0, &tm_phi, &tm_u, &s_bar);
    } else {
        step_tile<Q, V, T, S, CONTRAST>(P, b, s_phi, s_u, x0, y0, z0);
    }
}

// ---------------------------------------------------------------------------
// Batched launches: every domain of a batch in one launch per phase (two for
// the step kernel: domains with and without density contrast), one block per
// tile.  Tiles of all domains form one flat list of {slot, x0, y0, z0}.  Each
// domain's parameters and buffers sit in one slot of a constant-memory table;
// b[k] are the buffers for the k-th step parity of the launch.  A block reads
// its slot at a block-uniform index, so the parameters are constant-cache
// operands as kernel parameters are in the single-domain kernels.  Every tile
// is computed by the same step_tile as in the single-domain kernels, so
// results are bitwise identical.
// ---------------------------------------------------------------------------
constexpr int kBatchSlots = 96;        // domains of all live batches of one precision on one GPU

template <typename T, typename S>
struct BatchEntry {
    StepParams<T> P;
    StepBuffers<T, S> b[2];
    int tma;                           // the batch's map table holds this slot's halo maps
};

template <typename T, typename S>
__constant__ BatchEntry<T, S> c_batch[kBatchSlots];

// maps: tiled TMA maps of the halo fields for this tile shape, three per slot
// (phi, then u_in for step parity 0 and 1, with the box of Tile<Q, V>'s halo),
// in global memory; used on tiles needing no periodic image in y, z.
template <int Q, typename T, typename S, int V, bool CONTRAST>
__global__ void __launch_bounds__(Tile<Q, V>::THREADS, (step_min_blocks<T, S, Tile<Q, V>::THREADS>()))
    k_step_batched(const int4* __restrict__ tiles, const CUtensorMap* __restrict__ maps, int parity) {
    using Tl = Tile<Q, V>;
    __shared__ __align__(128) T s_phi[Tl::HN];
    __shared__ __align__(128) T s_u[CONTRAST ? Tl::D * Tl::HN : 1];
    __shared__ __align__(8) uint64_t s_bar;
    const int4 t = __ldg(tiles + blockIdx.x);          // {slot, x0, y0, z0}
    const BatchEntry<T, S>& e = c_batch<T, S>[idx_checked(t.x, kBatchSlots, c_batch<T, S>[0].b[0].err)];
    const int y0 = t.z, z0 = t.w;
    if (kDebugBounds && !(idx_ok(t.y, e.P.nx, e.b[0].err) && idx_ok(y0, e.P.ny, e.b[0].err) &&
                          idx_ok(z0, e.P.nz, e.b[0].err)))
        return;                                         // a tile outside its domain
    const bool tma = maps != nullptr && e.tma && y0 >= 1 && y0 + Tl::TY + 1 <= e.P.ny &&
                     (Tl::D == 2 || (z0 >= 1 && z0 + Tl::TZ + 1 <= e.P.nz));
    if (tma) {
        if (threadIdx.x + threadIdx.y + threadIdx.z == 0) mbar_init(&s_bar, 1);
        __syncthreads();                                      // the barrier exists before anyone waits on it
        step_tile<Q, V, T, S, CONTRAST>(e.P, e.b[parity], s_phi, s_u, t.y, y0, z0, maps + 3 * t.x,
                                        maps + 3 * t.x + 1 + parity, &s_bar);
    } else {
        step_tile<Q, V, T, S, CONTRAST>(e.P, e.b[parity], s_phi, s_u, t.y, y0, z0);
    }
}

template <int Q, typename T, typename S, int V>
__global__ void __launch_bounds__(Tile<Q, V>::THREADS) k_phi_batched(const int4* __restrict__ tiles, int parity) {
    const int4 t = __ldg(tiles + (gridDim.x - 1 - blockIdx.x));     // reverse order, as k_phi
    const BatchEntry<T, S>& e = c_batch<T, S>[idx_checked(t.x, kBatchSlots, c_batch<T, S>[0].b[0].err)];
    // this step's output B* is the buffer the step kernel wrote
    phi_node<Q, T, S>(e.P, e.b[parity].Bout, e.b[parity].mask, e.b[parity].phi, t.y + threadIdx.x, t.z + threadIdx.y,
                      t.w + threadIdx.z, e.b[parity].err);
}

// Color kernel of a batch over row chunks: a block takes kPhiChunk
// consecutive nodes of one z plane of one domain in the padded row order
// (tile {slot, x0, y0, z}: the chunk starts at (x0, y0)), crossing rows where
// a row ends, so that only the padding columns and a plane's last chunk leave
// threads idle (box tiles idle at the ragged x end of every row of a small
// domain), and every pull of the block reads one contiguous run per direction.
template <int Q, typename T, typename S>
__global__ void __launch_bounds__(kPhiChunk) k_phi_rows_batched(const int4* __restrict__ tiles, int parity) {
    const int4 t = __ldg(tiles + (gridDim.x - 1 - blockIdx.x));     // reverse order, as k_phi
    const BatchEntry<T, S>& e = c_batch<T, S>[idx_checked(t.x, kBatchSlots, c_batch<T, S>[0].b[0].err)];
    int x = t.y + (int)threadIdx.x, y = t.z;
    while (x >= e.P.px) {                         // at most kPhiChunk / px + 1 rows on
        x -= e.P.px;
        ++y;
    }
    if (x >= e.P.nx || y >= e.P.ny) return;       // padding column, or past the plane's end
    phi_node<Q, T, S>(e.P, e.b[parity].Bout, e.b[parity].mask, e.b[parity].phi, x, y, t.w, e.b[parity].err);
}

// Ghost tables of all domains: ghost g of the batch belongs to the domain d with
// ghost_begin[d] <= g < ghost_begin[d + 1].
template <typename T>
struct GhostTable {
    int64_t n;
    const int32_t* node;
    const int32_t* corner;
    const T* wt;
    T exp_eps, eps;
    T* phi;
    int rule;
    int64_t plane;                 // entries of phi (bounds of node and corner indices)
    int* err;                      // the domain's error word
};

template <int GK, typename T>
__global__ void __launch_bounds__(256) k_ghost_batched(const GhostTable<T>* __restrict__ tabs,
                                                       const int64_t* __restrict__ ghost_begin, int ndom,
                                                       int64_t total) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    int lo = 0, hi = ndom - 1;                     // last d with ghost_begin[d] <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ghost_begin[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const GhostTable<T>& t = tabs[lo];
    const int64_t k = g - ghost_begin[lo];
    const int64_t n = t.n;
    if (!idx_ok(k, n, t.err)) return;
    T phiF = T(0);
#pragma unroll
    for (int c = 0; c < GK; ++c) phiF += t.wt[c * n + k] * t.phi[idx_checked(t.corner[c * n + k], t.plane, t.err)];
    T phiG;
    if (t.rule == 0) {
        phiG = phiF / (phiF + (T(1) - phiF) * t.exp_eps);
    } else {
        const T a = T(1) + T(0.5) * t.eps;
        phiG = T(4) * phiF / (a + sqrt(a * a - T(2) * t.eps * phiF)) - phiF;
    }
    const int32_t gn = t.node[k];
    if (idx_ok(gn, t.plane, t.err)) t.phi[gn] = phiG;
}

}  // namespace lbmgpu
