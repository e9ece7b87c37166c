/*
 * oracle.h -- plain FP64 CPU oracle of the color-gradient lattice Boltzmann
 * step with the ghost-node wetting rule (Bhattacharya et al., "Color-gradient
 * lattice Boltzmann modeling of wetting boundary condition on curved solid
 * boundaries", arXiv 2605.30878).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this code: only tests/, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py use it, to check and to time against the CUDA library.
 * It shares no code, header, table or helper with that library.
 *
 * Every array is node-major inside a field: a node index is
 *     node = x + nx*(y + ny*z)
 * populations are stored as [q][node].  Solid nodes carry no populations
 * (their slots stay 0).  All floating point is double precision.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t lattice;      /* 9 (D2Q9, Appendix A) or 19 (D3Q19, 3D extension) */
    int32_t nx, ny, nz;   /* nz = 1 for D2Q9 */
    uint32_t periodic;    /* bit0 x, bit1 y, bit2 z; a non-periodic axis needs solid end layers */
    int32_t ghost_rule;   /* 0: Eq. (ghost-nodePrescription); 1: Eq. (ghostNodeFakhari) */
    double rho_l, rho_g;  /* liquid (phi=1) and gas (phi=0) densities, Sec. II */
    double mu_l, mu_g;    /* dynamic viscosities */
    double sigma;         /* surface tension, Eq. (surfaceTensionForce) */
    double W;             /* interface width, W >= 4 (Eq. ghost-nodePrescription) */
    double M_phi;         /* interface mobility, sets alpha (Appendix A) */
    double theta;         /* contact angle in radians, measured through the liquid */
    double g[3];          /* body acceleration, F_b = rho g */
} orc_params;

typedef struct { int64_t node; double n[3]; } orc_ghost;   /* unit normal out of the solid */

typedef struct {
    int32_t kind;          /* 0 none, 1 circle/sphere, 2 plane */
    int32_t reserved;
    double center[3];      /* circle/sphere centre; any point on the plane */
    double radius;         /* circle/sphere radius */
    double normal[3];      /* plane normal out of the solid; apex axis for kind 1 */
    double exclude;        /* drop interface points closer than this to the surface */
} orc_probe;

typedef struct {
    double phi_sum, mass_liquid, mass_gas, pop_sum, max_u;
    double p_in, p_out;
    double fit_center[3], fit_radius, contact_angle, apex;
    int64_t n_in, n_out, n_iface, n_fit, n_fluid, step;
    int32_t nan_flag, reserved;
} orc_diag;

enum { ORC_N = 0, ORC_B = 1, ORC_PHI = 2, ORC_U = 3, ORC_P = 4 };

typedef struct orc_sim orc_sim;

/* status: 0 ok, -1 bad argument (message in err) */
int  orc_create(const orc_params* prm, const uint8_t* solid, const orc_ghost* ghosts,
                int64_t n_ghosts, orc_sim** out, char* err, int errlen);
void orc_destroy(orc_sim* s);
void orc_init_phi(orc_sim* s, const double* phi);
void orc_init_droplet(orc_sim* s, const double centre[3], double R0);
void orc_step(orc_sim* s, int64_t n);
void orc_get(const orc_sim* s, int field, double* out);
void orc_set(orc_sim* s, int field, const double* in);
void orc_diagnostics(const orc_sim* s, const orc_probe* probe, orc_diag* out);
void orc_step_sample(const orc_sim* s, const int64_t* nodes, int64_t n,
                     double* N_out, double* B_out, double* u_out, double* p_out, double* phi_out);
int64_t orc_ghost_fallbacks(const orc_sim* s);
void orc_update_ghosts(orc_sim* s);
void orc_ghost_table(const orc_sim* s, int64_t* corner, double* weight, int32_t* ncorner);
int  orc_node_class(const orc_sim* s, int64_t node);

/* single-node pieces, exposed for the pins in tests/ */
int    orc_lattice_tables(int lattice, double M_phi, int gram_schmidt, int32_t* c, double* w,
                          double* chi, int32_t* opp, double* M, double* Minv, int32_t* is_stress);
void   orc_equilibrium(int lattice, double M_phi, const double u[3], double p, double* neq);
void   orc_macro(int lattice, double M_phi, const double* N, const double F[3], double rho,
                 double u[3], double* p);
void   orc_collide(int lattice, double M_phi, const double* N, const double u[3], double p,
                   const double F[3], double rho, double tau, double* Nst);
/* Eq. (segragationStepBlue) at one node: B* from N*, phi, grad phi and p (W the interface width) */
void   orc_segregate(int lattice, double M_phi, double W, double phi, const double gphi[3], double p,
                     const double* Nst, double* Bst);
double orc_ghost_rule(double phiF, double eps);
double orc_ghost_rule_fakhari(double phiF, double eps);

#ifdef __cplusplus
}
#endif
#endif
