// Definitions of the typed kernel launchers declared in lbm_launch.cuh.
// Included only by the per-precision translation units, which instantiate
// Launch<T, S> (and so every kernel) once each.
#pragma once

#include <type_traits>

#include <cmath>

#include "lbm_launch.cuh"

namespace lbmgpu {

// chi for float arithmetic: the moving values on a grid of 2^-24 and chi_0 =
// 1 minus their sum, a multiple of 2^-24 below 1 and so exact in float, so the
// float values sum to exactly 1.  sum chi = 1 is what makes the collision keep
// each node's color (sum_i B*_i = phi sum_i chi_i); values rounded one by one
// sum to 1 + delta (delta ~ 3e-8 from chi_0 alone) and move (phi - 1/2) delta
// of color per node and step, a drift of 1e-4 of a drop's color in 300 steps.
inline void chi_for_float(const double* chi, double* out) {
    double rest = 1.0;
    for (int i = 1; i < 19; ++i) {
        out[i] = std::ldexp(std::nearbyint(std::ldexp(chi[i], 24)), -24);
        rest -= out[i];
    }
    out[0] = rest;
}

template <typename T, typename S>
StepParams<T> Launch<T, S>::params(const StepConfig& c) {
    StepParams<T> P;
    P.nx = c.d.nx; P.ny = c.d.ny; P.nz = c.d.nz;
    P.px = c.d.px;
    P.plane = c.d.plane;
    P.rho_l = (T)c.rho_l; P.rho_g = (T)c.rho_g; P.drho = (T)(c.rho_l - c.rho_g);
    P.inv_nu_l = (T)(1.0 / c.nu_l); P.inv_nu_g = (T)(1.0 / c.nu_g);
    P.sigma = (T)c.sigma;
    P.W = (T)c.W;
    P.nu_l = (T)c.nu_l; P.nu_g = (T)c.nu_g;
    P.k48W = (T)(48.0 / c.W); P.k3W2 = (T)(1.5 * c.W); P.two_over_W = (T)(2.0 / c.W);
    for (int a = 0; a < 3; ++a) P.g[a] = (T)c.g[a];
    double chi[19];
    if (sizeof(T) == 4) chi_for_float(c.chi, chi);
    else std::memcpy(chi, c.chi, sizeof(chi));
    for (int i = 0; i < 19; ++i) P.chi[i] = (T)chi[i];
    // exact chi minus the stored reference, by class: rest, axis (direction 1),
    // diagonal/edge (direction 5 of D2Q9, 7 of D3Q19); zero in FP64
    const int diag = c.Q == 9 ? 5 : 7;
    P.chi_err[0] = (T)(c.chi[0] - chi[0]);
    P.chi_err[1] = (T)(c.chi[1] - chi[1]);
    P.chi_err[2] = (T)(c.chi[diag] - chi[diag]);
    P.c2chi = (T)c.c2chi;
    P.exp_eps = (T)c.exp_eps;
    return P;
}

template <typename T, typename S>
template <int Q>
dim3 Launch<T, S>::step_grid(const Dims& d) {
    using Tl = Tile<Q>;
    return dim3((d.nx + Tl::TX - 1) / Tl::TX, (d.ny + Tl::TY - 1) / Tl::TY, (d.nz + Tl::TZ - 1) / Tl::TZ);
}

template <typename T, typename S>
template <int Q>
dim3 Launch<T, S>::step_block() {
    using Tl = Tile<Q>;
    return dim3(Tl::TX, Tl::TY, Tl::TZ);
}

template <typename T, typename S>
template <int Q>
dim3 Launch<T, S>::pair_grid(const Dims& d) {
    using Tl = PairTile<Q>;
    return dim3((d.nx + Tl::TX - 1) / Tl::TX, (d.ny + Tl::TY - 1) / Tl::TY, (d.nz + Tl::TZ - 1) / Tl::TZ);
}

template <typename T, typename S>
template <int Q>
void Launch<T, S>::step_q(const StepConfig& c, const StepPtrs& p, cudaStream_t s) {
    const StepParams<T> P = params(c);
    StepBuffers<T, S> b;
    b.Nin = (const S*)p.Nin; b.Bin = (const S*)p.Bin; b.Nout = (S*)p.Nout; b.Bout = (S*)p.Bout;
    b.phi = (T*)p.phi; b.u_in = (const T*)p.u_in; b.u_out = (T*)p.u_out; b.p = (T*)p.p;
    b.mask = p.mask; b.err = p.err;
    CUtensorMap tm_phi{}, tm_u{};
    int tma = 0;
    if constexpr (sizeof(T) == 4) {
        if (c.pair) {
            using Tl = PairTile<Q>;
            if (p.tm2_phi && p.tm2_u) {
                tm_phi = *p.tm2_phi;
                tm_u = *p.tm2_u;
                tma = 1;
            }
            const dim3 block(Tl::BX, Tl::TY, Tl::TZ);
            if (c.contrast)
                k_step_pair<Q, S, true><<<pair_grid<Q>(c.d), block, 0, s>>>(P, b, tm_phi, tm_u, tma);
            else
                k_step_pair<Q, S, false><<<pair_grid<Q>(c.d), block, 0, s>>>(P, b, tm_phi, tm_u, tma);
            return;
        }
    }
    if (sizeof(T) == 4 && p.tm_phi && p.tm_u) {
        tm_phi = *p.tm_phi;
        tm_u = *p.tm_u;
        tma = 1;
    }
    if (c.contrast)
        k_step<Q, T, S, true><<<step_grid<Q>(c.d), step_block<Q>(), 0, s>>>(P, b, tm_phi, tm_u, tma);
    else
        k_step<Q, T, S, false><<<step_grid<Q>(c.d), step_block<Q>(), 0, s>>>(P, b, tm_phi, tm_u, tma);
}

template <typename T, typename S>
void Launch<T, S>::step(const StepConfig& c, const StepPtrs& p, cudaStream_t s) {
    if (c.Q == 9) step_q<9>(c, p, s); else step_q<19>(c, p, s);
}

template <typename T, typename S>
void Launch<T, S>::phi(const StepConfig& c, const void* Bst, const uint32_t* mask, void* phi, int* err,
                       cudaStream_t s) {
    const StepParams<T> P = params(c);
    if (c.Q == 9)
        k_phi<9, T, S><<<step_grid<9>(c.d), step_block<9>(), 0, s>>>(P, (const S*)Bst, mask, (T*)phi, err);
    else
        k_phi<19, T, S><<<step_grid<19>(c.d), step_block<19>(), 0, s>>>(P, (const S*)Bst, mask, (T*)phi, err);
}

template <typename T, typename S>
void Launch<T, S>::ghost(int GK, int rule, int64_t ng, const int32_t* node, const int32_t* corner, const void* wt,
                  double exp_eps, double eps, void* phi, int64_t plane, int* err, cudaStream_t s) {
    if (ng == 0) return;
    const unsigned blocks = (unsigned)((ng + 255) / 256);
    const T* w = (const T*)wt;
    T* f = (T*)phi;
    if (GK == 4 && rule == 0) k_ghost<4, T, 0><<<blocks, 256, 0, s>>>(ng, node, corner, w, (T)exp_eps, (T)eps, f, plane, err);
    if (GK == 4 && rule == 1) k_ghost<4, T, 1><<<blocks, 256, 0, s>>>(ng, node, corner, w, (T)exp_eps, (T)eps, f, plane, err);
    if (GK == 8 && rule == 0) k_ghost<8, T, 0><<<blocks, 256, 0, s>>>(ng, node, corner, w, (T)exp_eps, (T)eps, f, plane, err);
    if (GK == 8 && rule == 1) k_ghost<8, T, 1><<<blocks, 256, 0, s>>>(ng, node, corner, w, (T)exp_eps, (T)eps, f, plane, err);
}

template <typename T, typename S>
unsigned Launch<T, S>::flat_blocks(const Dims& d) {
    const int64_t nn = (int64_t)d.px * d.ny * d.nz;
    int64_t b = (nn + 255) / 256;
    return (unsigned)(b > 8192 ? 8192 : (b < 1 ? 1 : b));
}

template <typename T, typename S>
void Launch<T, S>::init_phi(const StepConfig& c, const uint8_t* cls, void* phi, int mode, const double ctr[3], double R0,
                     double ghost_value, cudaStream_t s) {
    if (c.Q == 9)
        k_init_phi<2, T><<<flat_blocks(c.d), 256, 0, s>>>(c.d, cls, (T*)phi, mode, ctr[0], ctr[1], ctr[2], R0, c.W,
                                                          ghost_value);
    else
        k_init_phi<3, T><<<flat_blocks(c.d), 256, 0, s>>>(c.d, cls, (T*)phi, mode, ctr[0], ctr[1], ctr[2], R0, c.W,
                                                          ghost_value);
}

template <typename T, typename S>
void Launch<T, S>::init_pops(const StepConfig& c, const uint8_t* cls, const void* phi, void* N, void* B, cudaStream_t s) {
    const StepParams<T> P = params(c);
    if (c.Q == 9)
        k_init_pops<9, T, S><<<flat_blocks(c.d), 256, 0, s>>>(c.d, P, cls, (const T*)phi, (S*)N, (S*)B);
    else
        k_init_pops<19, T, S><<<flat_blocks(c.d), 256, 0, s>>>(c.d, P, cls, (const T*)phi, (S*)N, (S*)B);
}

template <typename T, typename S>
void Launch<T, S>::expand_classes(const StepConfig& c, int W, const uint64_t* F, const uint64_t* G, uint8_t* cls,
                                  cudaStream_t s) {
    k_expand_classes<<<flat_blocks(c.d), 256, 0, s>>>(c.d, W, F, G, cls);
}

template <typename T, typename S>
void Launch<T, S>::build_mask(const StepConfig& c, const uint8_t* cls, uint32_t* mask, cudaStream_t s) {
    if (c.Q == 9)
        k_build_mask<9><<<flat_blocks(c.d), 256, 0, s>>>(c.d, cls, mask);
    else
        k_build_mask<19><<<flat_blocks(c.d), 256, 0, s>>>(c.d, cls, mask);
}

// base subtracted from direction i of N (is_b = false) or B (true) in storage
template <typename T, typename S>
double Launch<T, S>::storage_base(const StepConfig& c, int i, bool is_b) {
    if (!PopStore<S>::kShift) return 0.0;
    double chi[19];                     // the deviations are taken from the chi the kernels use
    if (sizeof(T) == 4) chi_for_float(c.chi, chi);
    else std::memcpy(chi, c.chi, sizeof(chi));
    return is_b ? 0.5 * chi[i] : chi[i];
}

template <typename T, typename S>
void Launch<T, S>::scatter_dir(const StepConfig& c, const uint8_t* cls, int i, bool is_b, const void* post_i,
                        const void* post_opp, void* st, cudaStream_t s) {
    // the host subtracted storage_base in double: the values arrive as what is stored
    const T base = T(0);
    const float scale = is_b ? kScaleB : kScaleN;
    if (c.Q == 9)
        k_scatter_dir<9, T, S><<<flat_blocks(c.d), 256, 0, s>>>(c.d, cls, i, (const T*)post_i,
                                                               (const T*)post_opp, base, scale, (S*)st);
    else
        k_scatter_dir<19, T, S><<<flat_blocks(c.d), 256, 0, s>>>(c.d, cls, i, (const T*)post_i,
                                                                (const T*)post_opp, base, scale, (S*)st);
}

template <typename T, typename S>
void Launch<T, S>::gather_dir(const StepConfig& c, const uint8_t* cls, int i, bool is_b, const void* st, void* post,
                       cudaStream_t s) {
    // the stored values as they are; the host adds storage_base in double
    const T base = T(0);
    const float scale = is_b ? kScaleB : kScaleN;
    if (c.Q == 9)
        k_gather_dir<9, T, S><<<flat_blocks(c.d), 256, 0, s>>>(c.d, cls, i, (const S*)st, base, scale, (T*)post);
    else
        k_gather_dir<19, T, S><<<flat_blocks(c.d), 256, 0, s>>>(c.d, cls, i, (const S*)st, base, scale, (T*)post);
}

// ---- batched launches (one block per tile of a flat tile list)
template <typename T, typename S>
template <int Qc, int V>
void Launch<T, S>::step_batched_v(const int4* tiles, const CUtensorMap* maps, int ntiles, int ncontrast, int parity,
                                  cudaStream_t s) {
    using Tl = Tile<Qc, V>;
    const dim3 block(Tl::TX, Tl::TY, Tl::TZ);     // the tile shape, as in the single-domain kernels
    if constexpr ((V == 5 || V == 3 || V == 0) && sizeof(T) == 4) {
        // float arithmetic: the two-node kernel over the same tiles, two nodes
        // per thread (64 nodes wide for shape 5, 32 for shapes 0 and 3)
        constexpr int TXn = Tl::TX, TYn = Tl::TY;
        using Pt = PairTile<Qc, TXn, TYn>;
        static_assert(Pt::TX == Tl::TX && Pt::TY == Tl::TY && Pt::TZ == Tl::TZ, "the pair tile covers the shape's tile");
        const dim3 pblock(Pt::BX, Pt::TY, Pt::TZ);
        if (ncontrast > 0)
            k_step_pair_batched<Qc, S, true, TXn, TYn><<<ncontrast, pblock, 0, s>>>(tiles, maps, parity);
        if (ntiles > ncontrast)
            k_step_pair_batched<Qc, S, false, TXn, TYn><<<ntiles - ncontrast, pblock, 0, s>>>(tiles + ncontrast,
                                                                                             maps, parity);
    } else {
        if (ncontrast > 0)
            k_step_batched<Qc, T, S, V, true><<<ncontrast, block, 0, s>>>(tiles, maps, parity);
        if (ntiles > ncontrast)
            k_step_batched<Qc, T, S, V, false><<<ntiles - ncontrast, block, 0, s>>>(tiles + ncontrast, maps,
                                                                                    parity);
    }
}

// step kernels then color kernel of every domain (the ghost update precedes them);
// tiles[0, ncontrast) belong to domains with density contrast
template <typename T, typename S>
void Launch<T, S>::step_phi_batched(int Q, int V, const int4* tiles, const CUtensorMap* maps, int ntiles, int ncontrast,
                                    int Vphi, const int4* phi_tiles, int phi_ntiles, int parity, cudaStream_t s) {
    if (ntiles == 0) return;
    auto steps = [&](auto q) {
        constexpr int Qc = decltype(q)::value;
        if (V == 0) step_batched_v<Qc, 0>(tiles, maps, ntiles, ncontrast, parity, s);
        if (V == 1) step_batched_v<Qc, 1>(tiles, maps, ntiles, ncontrast, parity, s);
        if (V == 2) step_batched_v<Qc, 2>(tiles, maps, ntiles, ncontrast, parity, s);
        if (V == 3) step_batched_v<Qc, 3>(tiles, maps, ntiles, ncontrast, parity, s);
        if (V == 4) step_batched_v<Qc, 4>(tiles, maps, ntiles, ncontrast, parity, s);
        if (V == 5) step_batched_v<Qc, 5>(tiles, maps, ntiles, ncontrast, parity, s);
        // the color kernel on its own tile list (it needs no halo, so its shape
        // need not be the step's)
        auto phi = [&](auto v) {
            constexpr int Vc = decltype(v)::value;
            using Tl = Tile<Qc, Vc>;
            k_phi_batched<Qc, T, S, Vc><<<phi_ntiles, dim3(Tl::TX, Tl::TY, Tl::TZ), 0, s>>>(phi_tiles, parity);
        };
        if (Vphi == 0) phi(std::integral_constant<int, 0>{});
        if (Vphi == 1) phi(std::integral_constant<int, 1>{});
        if (Vphi == 2) phi(std::integral_constant<int, 2>{});
        if (Vphi == 3) phi(std::integral_constant<int, 3>{});
        if (Vphi == 4) phi(std::integral_constant<int, 4>{});
        if (Vphi == 5) phi(std::integral_constant<int, 5>{});
        if (Vphi == kPhiRows)
            k_phi_rows_batched<Qc, T, S><<<phi_ntiles, kPhiChunk, 0, s>>>(phi_tiles, parity);
    };
    if (Q == 9) steps(std::integral_constant<int, 9>{});
    else steps(std::integral_constant<int, 19>{});
}

template <typename T, typename S>
void Launch<T, S>::fill_entry(void* out, const StepConfig& c, const StepPtrs p[2], bool tma) {
    BatchEntry<T, S> e;
    e.P = params(c);
    for (int k = 0; k < 2; ++k) {
        StepBuffers<T, S>& b = e.b[k];
        b.Nin = (const S*)p[k].Nin; b.Bin = (const S*)p[k].Bin; b.Nout = (S*)p[k].Nout; b.Bout = (S*)p[k].Bout;
        b.phi = (T*)p[k].phi; b.u_in = (const T*)p[k].u_in; b.u_out = (T*)p[k].u_out; b.p = (T*)p[k].p;
        b.mask = p[k].mask; b.err = p[k].err;
    }
    e.tma = (sizeof(T) == 4 && tma) ? 1 : 0;
    std::memcpy(out, &e, sizeof(e));
}

template <typename T, typename S>
cudaError_t Launch<T, S>::upload_entries(int slot0, const void* entries, int n) {
    return cudaMemcpyToSymbol(c_batch<T, S>, entries, n * sizeof(BatchEntry<T, S>),
                              slot0 * sizeof(BatchEntry<T, S>), cudaMemcpyHostToDevice);
}

template <typename T, typename S>
void Launch<T, S>::ghost_batched(int GK, const void* tabs, const int64_t* begin, int ndom, int64_t total, cudaStream_t s) {
    if (total == 0) return;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (GK == 4) k_ghost_batched<4, T><<<blocks, 256, 0, s>>>((const GhostTable<T>*)tabs, begin, ndom, total);
    else k_ghost_batched<8, T><<<blocks, 256, 0, s>>>((const GhostTable<T>*)tabs, begin, ndom, total);
}

template <typename T, typename S>
void Launch<T, S>::fill_ghost_table(void* out, int64_t n, const int32_t* node, const int32_t* corner, const void* wt,
                             double exp_eps, double eps, void* phi, int rule, int64_t plane, int* err) {
    GhostTable<T> g;
    g.n = n; g.node = node; g.corner = corner; g.wt = (const T*)wt; g.exp_eps = (T)exp_eps; g.eps = (T)eps;
    g.phi = (T*)phi; g.rule = rule; g.plane = plane; g.err = err;
    std::memcpy(out, &g, sizeof(g));
}

template <typename T, typename S>
int Launch<T, S>::diag_blocks(const Dims& d) {
    const int64_t nn = (int64_t)d.px * d.ny * d.nz;
    int64_t b = (nn + DIAG_THREADS - 1) / DIAG_THREADS;
    return (int)(b > DIAG_MAX_BLOCKS ? DIAG_MAX_BLOCKS : (b < 1 ? 1 : b));
}

template <typename T, typename S>
void Launch<T, S>::diag(const StepConfig& c, const uint32_t* mask, const void* Nst, const void* phi, const void* u,
                 const void* p, const ProbeDev& pr, double* partial, double* out, cudaStream_t s) {
    const int nb = diag_blocks(c.d);
    const StepParams<T> P = params(c);
    if (c.Q == 9)
        k_diag_partial<9, T, S><<<nb, DIAG_THREADS, 0, s>>>(c.d, c.rho_l, c.rho_g, mask, P, (const S*)Nst,
                                                            (const T*)phi, (const T*)u, (const T*)p, pr, partial);
    else
        k_diag_partial<19, T, S><<<nb, DIAG_THREADS, 0, s>>>(c.d, c.rho_l, c.rho_g, mask, P, (const S*)Nst,
                                                             (const T*)phi, (const T*)u, (const T*)p, pr, partial);
    k_diag_final<<<1, dim3(DG_REC, 32), 0, s>>>(nb, partial, out);
}

}  // namespace lbmgpu
