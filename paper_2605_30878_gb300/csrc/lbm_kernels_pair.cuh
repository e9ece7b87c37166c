// Two-node step kernel (float arithmetic, FP32 or FP16 population storage).
//
// Every thread updates the two x-adjacent nodes A = (x0 + 2t, y, z) and
// B = (x0 + 2t + 1, y, z) of its row, with the arithmetic of k_step: the same
// stencil sums in the same order and FloatNode's per-node update, so the two
// kernels round alike.  Since A's index is even, the pair shares
//   - its mask (one 8-byte load),
//   - its streaming pulls along y and z (one two-wide load per direction with
//     c_x = 0; directions with c_x != 0 pull from odd offsets, two loads),
//   - its shared-memory stencil values (two-wide loads; the rows a +/- x
//     direction needs come from three aligned two-wide loads, shared by the
//     directions of that row),
//   - its stores of N*, B*, u and p (one two-wide store each),
// which halves the load/store and address instructions per node of the
// one-node kernel.  The float arithmetic of the two nodes runs on packed
// pairs (FloatNode<..., F2>: one add/mul/fma.f32x2 for both nodes, each lane
// rounded as the one-node kernel's scalar operation), which halves the float
// instructions too.  Blocks are TX/2 x TY x TZ threads covering TX x TY x TZ
// nodes; the halo tile is copied by the same halo_issue/halo_complete as
// k_step's (TMA boxes (TX + 8) x (TY + 2) x (TZ + 2) on interior tiles).  A node of
// the pair that is not fluid gets zero velocity and pressure; its population
// slots receive values that nothing reads (every pull of a fluid node reads
// fluid sources or its own slots, as the diagnostics and state transfer do).
#pragma once

#include "lbm_kernels.cuh"

namespace lbmgpu {

// TXn nodes along x (64: the single-domain kernel and batch shape 5; 32:
// batch shapes 0 and 3, narrower tiles for small domains' ragged x ends) and
// TYn along y (0: 4 in 2D, 2 in 3D; batch shape 0 takes 8 and 4)
template <int Q, int TXn = 64, int TYn = 0>
struct PairTile {
    static constexpr int D = Lattice<Q>::D;
    static constexpr int BX = TXn / 2;             // threads along x
    static constexpr int TX = TXn;                 // nodes along x
    static constexpr int TY = TYn ? TYn : (D == 2 ? 4 : 2);
    static constexpr int TZ = D == 2 ? 1 : 2;
    static constexpr int XO = 4;                   // halo origin x0 - 4: 16-byte aligned for tiled copies
    static constexpr int HX = TX + 2 * XO;
    static constexpr int HY = TY + 2;
    static constexpr int HZ = D == 2 ? 1 : TZ + 2;
    static constexpr int HN = HX * HY * HZ;
    static constexpr int THREADS = BX * TY * TZ;
    __host__ __device__ static constexpr int off(int cx, int cy, int cz) { return cx + HX * (cy + HY * cz); }
};

// Resident blocks per SM the pair kernel is compiled for (registers per
// thread <= 65536 / (THREADS * blocks)), measured at 192^3 with the packed
// node update: 6 (80 registers, no spills) for FP32 and FP16 storage; 7 (72
// registers) spills 50 bytes with FP16 storage and runs 9% slower; 4 is 20%
// slower; 8 spills 76 bytes or more.
template <typename S, int THREADS = 128> struct PairBlocks { static constexpr int value = 6 * 128 / THREADS; };

// The values at halo slots hc + o and hc + o + 1 (hc even): one aligned
// two-wide load for even o, else the odd half of the pair below and the even
// half of the pair above (loads of the same address are shared by the compiler
// across directions).
template <int HN>
__device__ __forceinline__ float2 halo_pair(const float* s, int hc, int o, int* err) {
    if ((o & 1) == 0) return *reinterpret_cast<const float2*>(s + idx_checked(hc + o, HN - 1, err));
    const float2 lo = *reinterpret_cast<const float2*>(s + idx_checked(hc + o - 1, HN - 1, err));
    const float2 hi = *reinterpret_cast<const float2*>(s + idx_checked(hc + o + 1, HN - 1, err));
    return make_float2(lo.y, hi.x);
}

// The pair tile at (x0, y0, z0); maps != nullptr: tiled halo copies (the
// caller checked the tile needs no periodic image in y and z and initialised
// the barrier).
template <int Q, typename S, bool CONTRAST, int TXn = 64, int TYn = 0>
__device__ __forceinline__ void step_pair_tile(const StepParams<float>& P, const StepBuffers<float, S>& b,
                                               float* s_phi, float* s_u, int x0, int y0, int z0,
                                               const CUtensorMap* tm_phi, const CUtensorMap* tm_u,
                                               uint64_t* bar) {
    using Tl = PairTile<Q, TXn, TYn>;
    using L = Lattice<Q>;
    using PS = PopStore<S>;
    constexpr int D = L::D;
    constexpr bool kUnits = !PS::kExact;
    int* const err = b.err;
    const bool interior = tm_phi != nullptr;
    HaloFix<Tl, float, CONTRAST> fx;
    if (!halo_issue<Tl, float, S, CONTRAST>(P, b, s_phi, s_u, x0, y0, z0, tm_phi, tm_u, bar, fx)) return;

    // the pair's populations, pulled while the halo is in flight
    const int xa = x0 + 2 * threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    const bool in_grid = xa < P.nx && y < P.ny && z < P.nz;      // A; B may be a padding column
    const bool b_in = in_grid && xa + 1 < P.nx;
    const int nodeA = in_grid ? idx_checked(xa + P.px * (y + P.ny * z), P.plane - 1, err) : 0;
    uint2 m = make_uint2(MASK_NOT_FLUID, MASK_NOT_FLUID);
    if (in_grid) m = __ldg(reinterpret_cast<const uint2*>(b.mask + nodeA));
    const bool fluidA = !(m.x & MASK_NOT_FLUID), fluidB = !(m.y & MASK_NOT_FLUID);
    const int pl = (int)P.plane;
    const long long nmv = (long long)(Q - 1) * pl;
    const auto* mv = PS::moving(b.Nin, pl);
    float NA[Q], NB[Q];
    NA[0] = NB[0] = 0.f;                          // the deviation form never reads the rest population
    if (in_grid) {
        const Wrap W(xa, y, z, P.nx, P.ny, P.nz, P.px);
        const int xpB = (xa + 1 == P.nx - 1) ? 1 - P.nx : 1;    // B (x >= 1) never wraps to the left
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
            const int row = (i - 1) * pl + nodeA + W.off(0, -cy, -cz);
            if (cx == 0) {
                const float2 v = PS::load_units2(mv, idx_checked(row, nmv - 1, err));
                NA[i] = v.x;
                NB[i] = v.y;
            } else if (cx > 0) {                  // from x - 1: A's may wrap, B's is A's own column
                NA[i] = (float)PS::load_units(mv, idx_checked(row + W.xm, nmv, err));
                NB[i] = (float)PS::load_units(mv, idx_checked(b_in ? row : row + W.xm, nmv, err));
            } else {                              // from x + 1
                NA[i] = (float)PS::load_units(mv, idx_checked(row + W.xp, nmv, err));
                NB[i] = (float)PS::load_units(mv, idx_checked(b_in ? row + 1 + xpB : row + W.xp, nmv, err));
            }
        }
        // halfway bounce-back: directions whose neighbour is not fluid read the node's own opposite slot
        if (fluidA && (m.x & ~MASK_NOT_FLUID)) {
#pragma unroll
            for (int i = 1; i < Q; ++i)
                if ((m.x >> i) & 1u)
                    NA[i] = (float)PS::load_units(mv, idx_checked((L::opp(i) - 1) * pl + nodeA, nmv, err));
        }
        if (fluidB && (m.y & ~MASK_NOT_FLUID)) {
#pragma unroll
            for (int i = 1; i < Q; ++i)
                if ((m.y >> i) & 1u)
                    NB[i] = (float)PS::load_units(mv, idx_checked((L::opp(i) - 1) * pl + nodeA + 1, nmv, err));
        }
    }
    // the moments of both nodes (one packed lane each) while the halo copy
    // completes; the pulled values are then dead, which keeps them out of the
    // registers the stencils need
    FloatNode<Q, kUnits, CONTRAST, F2> n2;
    {
        F2 N2[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) N2[i] = F2(NA[i], NB[i]);
        n2.moments(N2);
    }
    const bool halo_ok = halo_complete<Tl, float, S>(b, interior, bar, s_phi, s_u, fx);
    __syncthreads();
    // Whole sectors (FP32 storage): a pair without a fluid node writes zeros
    // to its slots when another pair of its group of 8 nodes (32 bytes, one
    // sector of every plane, since planes start at multiples of 64 nodes)
    // stores its update.  The L2 then writes back whole sectors, where a
    // partly written one would first be read from DRAM (a batch of 64 domains
    // of 48^3 to 128^3: 10% less DRAM read per step kernel launch, 6%
    // faster).  Nothing reads these slots: a fluid node pulls from fluid
    // nodes or its own slots, and u, p stay 0 at nodes that are not fluid.  With FP16 storage the extra
    // instructions cost more than the traffic saved (its k_step is
    // issue-bound: 0.77 of its roofline with the fill, 0.80 without).
    if constexpr (sizeof(S) == 4) {
        constexpr int kGroupShift = 3;
        const bool in_pitch = xa < P.px && y < P.ny && z < P.nz;     // A, B in the padded rows
        const int nodeP = in_pitch ? idx_checked(xa + P.px * (y + P.ny * z), P.plane - 1, err) : 0;
        unsigned lane;
        asm("mov.u32 %0, %%laneid;" : "=r"(lane));
        const int group = in_pitch ? (nodeP >> kGroupShift) : -1 - (int)lane;
        const unsigned same = __match_any_sync(0xffffffffu, group);
        const unsigned writers = __ballot_sync(0xffffffffu, fluidA || fluidB);
        if (!(fluidA || fluidB) && in_pitch && halo_ok && (same & writers)) {
            auto* __restrict__ Nm = PS::moving(b.Nout, pl) + nodeP;
            auto* __restrict__ Bm = PS::moving(b.Bout, pl) + nodeP;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                PS::store_zero2(Nm + (i - 1) * pl);
                PS::store_zero2(Bm + (i - 1) * pl);
            }
            const float2 zero = make_float2(0.f, 0.f);
            *reinterpret_cast<float2*>(PS::rest(b.Nout) + nodeP) = zero;
            *reinterpret_cast<float2*>(PS::rest(b.Bout) + nodeP) = zero;
#pragma unroll
            for (int a = 0; a < D; ++a) *reinterpret_cast<float2*>(b.u_out + a * pl + nodeP) = zero;
            *reinterpret_cast<float2*>(b.p + nodeP) = zero;
        }
    }
    if (!(fluidA || fluidB) || !halo_ok) return;

    // isotropic stencils of both nodes, over +/- pairs in the order of k_step
    const int hcA = (2 * threadIdx.x + Tl::XO) + Tl::HX * ((threadIdx.y + 1) + Tl::HY * (D == 2 ? 0 : threadIdx.z + 1));
    const float2 phv = halo_pair<Tl::HN>(s_phi, hcA, 0, err);
    const F2 ph(phv.x, phv.y);
    F2 g[3] = {F2(0.f), F2(0.f), F2(0.f)}, lap(0.f);
    F2 du[3][3] = {{F2(0.f), F2(0.f), F2(0.f)}, {F2(0.f), F2(0.f), F2(0.f)}, {F2(0.f), F2(0.f), F2(0.f)}};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (L::opp(i) < i) continue;
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const float wi = float(3.0 * L::w(i)), wl = float(6.0 * L::w(i));   // grad: 3 w_i, lap: 6 w_i
        const int o = Tl::off(cx, cy, cz);
        const float2 ppv = halo_pair<Tl::HN>(s_phi, hcA, o, err), pmv = halo_pair<Tl::HN>(s_phi, hcA, -o, err);
        const F2 pp(ppv.x, ppv.y), pm(pmv.x, pmv.y);
        const F2 dphi = pp - pm;
        if (cx) g[0] = fma(F2(float(cx) * wi), dphi, g[0]);
        if (cy) g[1] = fma(F2(float(cy) * wi), dphi, g[1]);
        if (cz) g[2] = fma(F2(float(cz) * wi), dphi, g[2]);
        lap = fma(F2(wl), (pp - ph) + (pm - ph), lap);
        if (CONTRAST) {
#pragma unroll
            for (int bb = 0; bb < D; ++bb) {
                const float2 upv = halo_pair<D * Tl::HN>(s_u, hcA + bb * Tl::HN, o, err);
                const float2 umv = halo_pair<D * Tl::HN>(s_u, hcA + bb * Tl::HN, -o, err);
                const F2 dub = F2(upv.x, upv.y) - F2(umv.x, umv.y);
                if (cx) du[0][bb] = fma(F2(float(cx) * wi), dub, du[0][bb]);
                if (cy) du[1][bb] = fma(F2(float(cy) * wi), dub, du[1][bb]);
                if (cz) du[2][bb] = fma(F2(float(cz) * wi), dub, du[2][bb]);
            }
        }
    }
    n2.compute(P, ph, g, lap, du);

    // u and p of the pair in one store per field; 0 at a node that is not fluid
    // (the velocity halo reads 0 at solid nodes)
#pragma unroll
    for (int a = 0; a < D; ++a)
        *reinterpret_cast<float2*>(b.u_out + a * pl + nodeA) =
            make_float2(fluidA ? n2.u[a].lo() : 0.f, fluidB ? n2.u[a].hi() : 0.f);
    *reinterpret_cast<float2*>(b.p + nodeA) = make_float2(fluidA ? n2.p.lo() : 0.f, fluidB ? n2.p.hi() : 0.f);
    if ((fluidA && !(n2.uu.lo() < 1e30f)) || (fluidB && !(n2.uu.hi() < 1e30f))) atomicOr(err, kErrNonFinite);

    auto* __restrict__ Nmov = PS::moving(b.Nout, pl);
    auto* __restrict__ Bmov = PS::moving(b.Bout, pl);
    float sNA = 0.f, sNB = 0.f, sBA = 0.f, sBB = 0.f;       // moving populations as stored (FP16 storage)
    // per-thread bases: each store's address is then the base plus a plane
    // offset that is the same for the whole grid (measured 3% faster with FP16
    // storage than indexing every store from the array start)
    auto* __restrict__ NmA = Nmov + nodeA;
    auto* __restrict__ BmA = Bmov + nodeA;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (L::opp(i) < i) continue;
        const int o = L::opp(i);
        F2 ni, no, bi, bo;
        n2.dir(i, ni, no, bi, bo);
        PS::store_units2(NmA, (i - 1) * pl, ni.lo(), ni.hi(), sNA, sNB);
        PS::store_units2(NmA, (o - 1) * pl, no.lo(), no.hi(), sNA, sNB);
        PS::store_units2(BmA, (i - 1) * pl, bi.lo(), bi.hi(), sBA, sBB);
        PS::store_units2(BmA, (o - 1) * pl, bo.lo(), bo.hi(), sBA, sBB);
    }
    float2 rn, rb;
    if constexpr (PS::kExact) {
        const F2 n0 = n2.rest_N(P), b0 = n2.rest_B(P, n0);
        rn = make_float2(n0.lo(), n0.hi());
        rb = make_float2(b0.lo(), b0.hi());
    } else {
        using FN = FloatNode<Q, kUnits, CONTRAST, F2>;
        rn = make_float2(FN::rest_N_from_sum(sNA), FN::rest_N_from_sum(sNB));
        rb = make_float2(FN::rest_B_from_sum(sBA, n2.phi.lo()), FN::rest_B_from_sum(sBB, n2.phi.hi()));
    }
    *reinterpret_cast<float2*>(PS::rest(b.Nout) + nodeA) = rn;
    *reinterpret_cast<float2*>(PS::rest(b.Bout) + nodeA) = rb;
}

template <int Q, typename S, bool CONTRAST>
__global__ void __launch_bounds__(PairTile<Q>::THREADS, PairBlocks<S>::value)
    k_step_pair(StepParams<float> P, StepBuffers<float, S> b, const __grid_constant__ CUtensorMap tm_phi,
                const __grid_constant__ CUtensorMap tm_u, int tma) {
    using Tl = PairTile<Q>;
    constexpr int D = Tl::D;
    __shared__ __align__(128) float s_phi[Tl::HN];
    __shared__ __align__(128) float s_u[CONTRAST ? D * Tl::HN : 2];
    __shared__ __align__(8) uint64_t s_bar;
    const int x0 = blockIdx.x * Tl::TX, y0 = blockIdx.y * Tl::TY, z0 = blockIdx.z * Tl::TZ;
    // tiles whose halo needs no periodic image in y and z (x images are patched)
    const bool interior = tma && y0 >= 1 && y0 + Tl::TY + 1 <= P.ny &&
                          (D == 2 || (z0 >= 1 && z0 + Tl::TZ + 1 <= P.nz));
    if (interior) {
        if (threadIdx.x + threadIdx.y + threadIdx.z == 0) mbar_init(&s_bar, 1);
        __syncthreads();                                      // the barrier exists before anyone waits on it
    }
    step_pair_tile<Q, S, CONTRAST>(P, b, s_phi, s_u, x0, y0, z0, interior ? &tm_phi : nullptr, &tm_u, &s_bar);
}

// Batched form: one pair tile of one domain per block, the domain's
// parameters in its constant-memory slot (as k_step_batched): 64 nodes wide
// for tile shape 5, 32 for tile shapes 0 and 3.
template <int Q, typename S, bool CONTRAST, int TXn = 64, int TYn = 0>
__global__ void __launch_bounds__(PairTile<Q, TXn, TYn>::THREADS,
                                  (PairBlocks<S, PairTile<Q, TXn, TYn>::THREADS>::value))
    k_step_pair_batched(const int4* __restrict__ tiles, const CUtensorMap* __restrict__ maps, int parity) {
    using Tl = PairTile<Q, TXn, TYn>;
    constexpr int D = Tl::D;
    __shared__ __align__(128) float s_phi[Tl::HN];
    __shared__ __align__(128) float s_u[CONTRAST ? D * Tl::HN : 2];
    __shared__ __align__(8) uint64_t s_bar;
    const int4 t = __ldg(tiles + blockIdx.x);          // {slot, x0, y0, z0}
    const BatchEntry<float, S>& e = c_batch<float, S>[idx_checked(t.x, kBatchSlots, c_batch<float, S>[0].b[0].err)];
    const int y0 = t.z, z0 = t.w;
    if (kDebugBounds && !(idx_ok(t.y, e.P.nx, e.b[0].err) && idx_ok(y0, e.P.ny, e.b[0].err) &&
                          idx_ok(z0, e.P.nz, e.b[0].err)))
        return;                                         // a tile outside its domain
    const bool tma = maps != nullptr && e.tma && y0 >= 1 && y0 + Tl::TY + 1 <= e.P.ny &&
                     (D == 2 || (z0 >= 1 && z0 + Tl::TZ + 1 <= e.P.nz));
    if (tma) {
        if (threadIdx.x + threadIdx.y + threadIdx.z == 0) mbar_init(&s_bar, 1);
        __syncthreads();                                      // the barrier exists before anyone waits on it
    }
    step_pair_tile<Q, S, CONTRAST, TXn, TYn>(e.P, e.b[parity], s_phi, s_u, t.y, y0, z0, tma ? maps + 3 * t.x : nullptr,
                                        maps + 3 * t.x + 1 + parity, &s_bar);
}

}  // namespace lbmgpu
