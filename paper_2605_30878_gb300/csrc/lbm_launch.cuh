// Typed kernel launchers: T is the arithmetic type, S the population storage
// type.  lbm_kern_f64.cu, lbm_kern_f32.cu and lbm_kern_f16.cu instantiate
// Launch<double, double>, Launch<float, float> and Launch<float, __half>; the
// host API only sees these functions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lbm_aux.cuh"
#include "lbm_kernels.cuh"

namespace lbmgpu {

// Everything a step launch needs, in double precision (converted per type).
struct StepConfig {
    int Q;
    bool contrast;                 // rho_l != rho_g: F_p and F_visc are active
    Dims d;
    double rho_l, rho_g, nu_l, nu_g, sigma, W;
    double g[3];
    double chi[19];
    double c2chi;
    double exp_eps;
    double eps;                    // -(4/W) cos(theta)
    int ghost_rule;                // lbm_ghost_rule
};

struct StepPtrs {
    const void* Nin;
    const void* Bin;
    void* Nout;
    void* Bout;
    void* phi;
    const void* u_in;
    void* u_out;
    void* p;
    const uint32_t* mask;
    int* err;
};

template <typename T, typename S>
struct Launch {
    static StepParams<T> params(const StepConfig& c) {
        StepParams<T> P;
        P.nx = c.d.nx; P.ny = c.d.ny; P.nz = c.d.nz;
        P.plane = c.d.plane;
        P.rho_l = (T)c.rho_l; P.rho_g = (T)c.rho_g; P.drho = (T)(c.rho_l - c.rho_g);
        P.inv_nu_l = (T)(1.0 / c.nu_l); P.inv_nu_g = (T)(1.0 / c.nu_g);
        P.sigma = (T)c.sigma;
        P.W = (T)c.W;
        P.nu_l = (T)c.nu_l; P.nu_g = (T)c.nu_g;
        P.k48W = (T)(48.0 / c.W); P.k3W2 = (T)(1.5 * c.W); P.two_over_W = (T)(2.0 / c.W);
        for (int a = 0; a < 3; ++a) P.g[a] = (T)c.g[a];
        for (int i = 0; i < 19; ++i) P.chi[i] = (T)c.chi[i];
        P.c2chi = (T)c.c2chi;
        P.exp_eps = (T)c.exp_eps;
        return P;
    }

    template <int Q>
    static dim3 step_grid(const Dims& d) {
        using Tl = Tile<Q>;
        return dim3((d.nx + Tl::TX - 1) / Tl::TX, (d.ny + Tl::TY - 1) / Tl::TY, (d.nz + Tl::TZ - 1) / Tl::TZ);
    }
    template <int Q>
    static dim3 step_block() {
        using Tl = Tile<Q>;
        return dim3(Tl::TX, Tl::TY, Tl::TZ);
    }

    template <int Q>
    static void step_q(const StepConfig& c, const StepPtrs& p, cudaStream_t s) {
        const StepParams<T> P = params(c);
        StepBuffers<T, S> b;
        b.Nin = (const S*)p.Nin; b.Bin = (const S*)p.Bin; b.Nout = (S*)p.Nout; b.Bout = (S*)p.Bout;
        b.phi = (T*)p.phi; b.u_in = (const T*)p.u_in; b.u_out = (T*)p.u_out; b.p = (T*)p.p;
        b.mask = p.mask; b.err = p.err;
        if (c.contrast)
            k_step<Q, T, S, true><<<step_grid<Q>(c.d), step_block<Q>(), 0, s>>>(P, b);
        else
            k_step<Q, T, S, false><<<step_grid<Q>(c.d), step_block<Q>(), 0, s>>>(P, b);
    }
    static void step(const StepConfig& c, const StepPtrs& p, cudaStream_t s) {
        if (c.Q == 9) step_q<9>(c, p, s); else step_q<19>(c, p, s);
    }

    static void phi(const StepConfig& c, const void* Bst, const uint32_t* mask, void* phi, cudaStream_t s) {
        const StepParams<T> P = params(c);
        if (c.Q == 9)
            k_phi<9, T, S><<<step_grid<9>(c.d), step_block<9>(), 0, s>>>(P, (const S*)Bst, mask, (T*)phi);
        else
            k_phi<19, T, S><<<step_grid<19>(c.d), step_block<19>(), 0, s>>>(P, (const S*)Bst, mask, (T*)phi);
    }

    static void ghost(int GK, int rule, int64_t ng, const int32_t* node, const int32_t* corner, const void* wt,
                      double exp_eps, double eps, void* phi, cudaStream_t s) {
        if (ng == 0) return;
        const unsigned blocks = (unsigned)((ng + 255) / 256);
        const T* w = (const T*)wt;
        if (GK == 4 && rule == 0) k_ghost<4, T, 0><<<blocks, 256, 0, s>>>(ng, node, corner, w, (T)exp_eps, (T)eps, (T*)phi);
        if (GK == 4 && rule == 1) k_ghost<4, T, 1><<<blocks, 256, 0, s>>>(ng, node, corner, w, (T)exp_eps, (T)eps, (T*)phi);
        if (GK == 8 && rule == 0) k_ghost<8, T, 0><<<blocks, 256, 0, s>>>(ng, node, corner, w, (T)exp_eps, (T)eps, (T*)phi);
        if (GK == 8 && rule == 1) k_ghost<8, T, 1><<<blocks, 256, 0, s>>>(ng, node, corner, w, (T)exp_eps, (T)eps, (T*)phi);
    }

    static unsigned flat_blocks(const Dims& d) {
        const int64_t nn = (int64_t)d.nx * d.ny * d.nz;
        int64_t b = (nn + 255) / 256;
        return (unsigned)(b > 8192 ? 8192 : (b < 1 ? 1 : b));
    }

    static void init_phi(const StepConfig& c, const uint8_t* cls, void* phi, int mode, const double ctr[3], double R0,
                         double ghost_value, cudaStream_t s) {
        if (c.Q == 9)
            k_init_phi<2, T><<<flat_blocks(c.d), 256, 0, s>>>(c.d, cls, (T*)phi, mode, ctr[0], ctr[1], ctr[2], R0, c.W,
                                                              ghost_value);
        else
            k_init_phi<3, T><<<flat_blocks(c.d), 256, 0, s>>>(c.d, cls, (T*)phi, mode, ctr[0], ctr[1], ctr[2], R0, c.W,
                                                              ghost_value);
    }

    static void init_pops(const StepConfig& c, const uint8_t* cls, const void* phi, void* N, void* B, cudaStream_t s) {
        const StepParams<T> P = params(c);
        if (c.Q == 9)
            k_init_pops<9, T, S><<<flat_blocks(c.d), 256, 0, s>>>(c.d, P, cls, (const T*)phi, (S*)N, (S*)B);
        else
            k_init_pops<19, T, S><<<flat_blocks(c.d), 256, 0, s>>>(c.d, P, cls, (const T*)phi, (S*)N, (S*)B);
    }

    // base subtracted from direction i of N (is_b = false) or B (true) in storage
    static double storage_base(const StepConfig& c, int i, bool is_b) {
        if (!PopStore<S>::kShift) return 0.0;
        return is_b ? 0.5 * c.chi[i] : c.chi[i];
    }

    static void scatter_dir(const StepConfig& c, const uint8_t* cls, int i, bool is_b, const void* post_i,
                            const void* post_opp, void* st, cudaStream_t s) {
        const T base = (T)storage_base(c, i, is_b);
        const float scale = is_b ? kScaleB : kScaleN;
        if (c.Q == 9)
            k_scatter_dir<9, T, S><<<flat_blocks(c.d), 256, 0, s>>>(c.d, cls, i, (const T*)post_i,
                                                                   (const T*)post_opp, base, scale, (S*)st);
        else
            k_scatter_dir<19, T, S><<<flat_blocks(c.d), 256, 0, s>>>(c.d, cls, i, (const T*)post_i,
                                                                    (const T*)post_opp, base, scale, (S*)st);
    }

    static void gather_dir(const StepConfig& c, const uint8_t* cls, int i, bool is_b, const void* st, void* post,
                           cudaStream_t s) {
        const T base = (T)storage_base(c, i, is_b);
        const float scale = is_b ? kScaleB : kScaleN;
        if (c.Q == 9)
            k_gather_dir<9, T, S><<<flat_blocks(c.d), 256, 0, s>>>(c.d, cls, i, (const S*)st, base, scale, (T*)post);
        else
            k_gather_dir<19, T, S><<<flat_blocks(c.d), 256, 0, s>>>(c.d, cls, i, (const S*)st, base, scale, (T*)post);
    }

    static int diag_blocks(const Dims& d) {
        const int64_t nn = (int64_t)d.nx * d.ny * d.nz;
        int64_t b = (nn + DIAG_THREADS - 1) / DIAG_THREADS;
        return (int)(b > DIAG_MAX_BLOCKS ? DIAG_MAX_BLOCKS : (b < 1 ? 1 : b));
    }

    static void diag(const StepConfig& c, const uint8_t* cls, const void* Nst, const void* phi, const void* u,
                     const void* p, const ProbeDev& pr, double* partial, double* out, cudaStream_t s) {
        const int nb = diag_blocks(c.d);
        const StepParams<T> P = params(c);
        if (c.Q == 9)
            k_diag_partial<9, T, S><<<nb, DIAG_THREADS, 0, s>>>(c.d, c.rho_l, c.rho_g, cls, P, (const S*)Nst,
                                                                (const T*)phi, (const T*)u, (const T*)p, pr, partial);
        else
            k_diag_partial<19, T, S><<<nb, DIAG_THREADS, 0, s>>>(c.d, c.rho_l, c.rho_g, cls, P, (const S*)Nst,
                                                                 (const T*)phi, (const T*)u, (const T*)p, pr, partial);
        k_diag_final<<<1, 32, 0, s>>>(nb, partial, out);
    }
};

extern template struct Launch<double, double>;
extern template struct Launch<float, float>;
extern template struct Launch<float, __half>;

}  // namespace lbmgpu
