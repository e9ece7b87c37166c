// Typed kernel launchers: T is the arithmetic type, S the population storage
// type.  This header declares them; lbm_launch_impl.cuh defines them, and only
// lbm_kern_f64.cu, lbm_kern_f32.cu and lbm_kern_f16.cu include it, to
// instantiate Launch<double, double>, Launch<float, float> and
// Launch<float, __half> (with their kernels) once each.  The host API sees
// declarations only, so no kernel is compiled twice.
#pragma once

#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "lbm_aux.cuh"
#include "lbm_kernels.cuh"
#include "lbm_kernels_pair.cuh"

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
    bool pair = false;             // float arithmetic: the two-node step kernel (k_step_pair)
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
    const CUtensorMap* tm_phi = nullptr;   // tiled maps of phi and of u_in for the halo copies, or none
    const CUtensorMap* tm_u = nullptr;
    const CUtensorMap* tm2_phi = nullptr;  // the same with the two-node kernel's box
    const CUtensorMap* tm2_u = nullptr;
};

template <typename T, typename S>
struct Launch {
    static StepParams<T> params(const StepConfig& c);
    template <int Q>
    static dim3 step_grid(const Dims& d);
    template <int Q>
    static dim3 step_block();
    template <int Q>
    static dim3 pair_grid(const Dims& d);
    template <int Q>
    static void step_q(const StepConfig& c, const StepPtrs& p, cudaStream_t s);
    static void step(const StepConfig& c, const StepPtrs& p, cudaStream_t s);
    static void phi(const StepConfig& c, const void* Bst, const uint32_t* mask, void* phi, int* err, cudaStream_t s);
    static void ghost(int GK, int rule, int64_t ng, const int32_t* node, const int32_t* corner, const void* wt,
                      double exp_eps, double eps, void* phi, int64_t plane, int* err, cudaStream_t s);
    static unsigned flat_blocks(const Dims& d);
    static void init_phi(const StepConfig& c, const uint8_t* cls, void* phi, int mode, const double ctr[3], double R0,
                         double ghost_value, cudaStream_t s);
    static void init_pops(const StepConfig& c, const uint8_t* cls, const void* phi, void* N, void* B, cudaStream_t s);
    static void build_mask(const StepConfig& c, const uint8_t* cls, uint32_t* mask, cudaStream_t s);
    static void expand_classes(const StepConfig& c, int W, const uint64_t* F, const uint64_t* G, uint8_t* cls,
                               cudaStream_t s);
    // base subtracted from direction i of N (is_b = false) or B (true) in
    // storage; scatter_dir takes and gather_dir returns the values less this
    // base (the host adds and subtracts it in double, so a float domain's
    // state crosses the ABI with the precision of its stored deviations)
    static double storage_base(const StepConfig& c, int i, bool is_b);
    static void scatter_dir(const StepConfig& c, const uint8_t* cls, int i, bool is_b, const void* post_i,
                            const void* post_opp, void* st, cudaStream_t s);
    static void gather_dir(const StepConfig& c, const uint8_t* cls, int i, bool is_b, const void* st, void* post,
                           cudaStream_t s);
    // ---- batched launches (one block per tile of a flat tile list)
    template <int Qc, int V>
    static void step_batched_v(const int4* tiles, const CUtensorMap* maps, int ntiles, int ncontrast, int parity,
                               cudaStream_t s);
    // step kernels then color kernel of every domain (the ghost update precedes them);
    // tiles[0, ncontrast) belong to domains with density contrast; the color
    // kernel runs on phi_tiles of shape Vphi, or of row chunks (Vphi == kPhiRows)
    static void step_phi_batched(int Q, int V, const int4* tiles, const CUtensorMap* maps, int ntiles, int ncontrast,
                                 int Vphi, const int4* phi_tiles, int phi_ntiles, int parity, cudaStream_t s);
    // Slot tables: entry_size() bytes per domain, filled by fill_entry, copied
    // to slots [slot0, slot0 + n) of the constant table by upload_entries.
    static size_t entry_size() { return sizeof(BatchEntry<T, S>); }
    static void fill_entry(void* out, const StepConfig& c, const StepPtrs p[2], bool tma);
    static cudaError_t upload_entries(int slot0, const void* entries, int n);
    static void ghost_batched(int GK, const void* tabs, const int64_t* begin, int ndom, int64_t total, cudaStream_t s);
    static size_t ghost_table_size() { return sizeof(GhostTable<T>); }
    static void fill_ghost_table(void* out, int64_t n, const int32_t* node, const int32_t* corner, const void* wt,
                                 double exp_eps, double eps, void* phi, int rule, int64_t plane, int* err);
    static int diag_blocks(const Dims& d);
    static void diag(const StepConfig& c, const uint32_t* mask, const void* Nst, const void* phi, const void* u,
                     const void* p, const ProbeDev& pr, double* partial, double* out, cudaStream_t s);
};

extern template struct Launch<double, double>;
extern template struct Launch<float, float>;
extern template struct Launch<float, __half>;

}  // namespace lbmgpu
