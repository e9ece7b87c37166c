/*
 * oracle.c -- plain, slow, literal FP64 reference of one time step of the
 * color-gradient lattice Boltzmann model with the ghost-node wetting rule of
 * Bhattacharya et al. (arXiv 2605.30878).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may call it.  It shares no code with the CUDA
 * library and never reads anything the CUDA library produced except state
 * that a test hands it explicitly.
 *
 * The step follows the paper's equations in the paper's order:
 *   stencils and forces  Eqs. (surfaceTensionForce), (totalForce),
 *                        (pressCorrection), (viscCorrection), (forceGuo)
 *   macroscopic fields   Eqs. (velUpdate), (pressureUpdate)
 *   equilibrium          Eq. (equilibriumDistribution)
 *   collision            Eq. (MRTCOLL), literally: moments by the matrix M,
 *                        relaxation by S, back by the inverse of M
 *   segregation          Eq. (segragationStepBlue)
 *   propagation          Eqs. (propTotal), (propBlue) with halfway
 *                        bounce-back on the staircase solid (Sec. II)
 *   color                Eq. (phiUpdate)
 *   ghost nodes          Eq. (ghost-nodePrescription) with x_F = x_G + n_s
 *                        and bilinear (trilinear in 3D) interpolation (Fig. 2)
 *
 * Readings where the paper is silent (each one is also used by the CUDA
 * library, which implements it independently):
 *   gradient and Laplacian: isotropic lattice stencils
 *       grad f = (1/cs2) sum_i w_i c_i f(x+c_i),
 *       lap f  = (2/cs2) sum_i w_i (f(x+c_i) - f(x));
 *   F_p uses the pressure of the current step from Eq. (pressureUpdate)
 *   with the force-free velocity sum_i N_i c_i (a one-step lag of p in F_p
 *   diverges at density ratio 1000); F_visc uses a stencil of the velocity
 *   of the previous step (zero at solid nodes, zero before the first step);
 *   alpha is set from M_phi at reference pressure p = 0;
 *   bilinear corners of x_F that are solid are dropped and the remaining
 *   weights renormalised; with no fluid corner the ghost takes the color of
 *   its fluid lattice neighbour most aligned with n_s;
 *   D3Q19 (not in the paper): same equations with the D3Q19 velocities and
 *   weights, chi_i = (1-alpha) w_i/(1-w_0), and an orthogonal M from
 *   Gram-Schmidt over monomials whose five traceless second-order rows relax
 *   at 1/tau and all others at 1;
 *   time step order: update the ghosts from the current fluid color, collide
 *   (stencils read fluid and fresh ghost values), stream, recompute the
 *   color.  The initial ghost value (1+cos theta)/2 of Sec. III is the stored
 *   ghost color at t = 0 and is replaced before any stencil reads it.
 *   n_phi = grad phi / max(|grad phi|, 1e-6): the unit normal wherever
 *   |grad phi| >= 1e-6, shrinking linearly to 0 below.  At a critical point of
 *   phi (a drop centre) rounding noise in grad phi would otherwise give n_phi
 *   a random unit direction times phi(1-phi).
 */
#include "oracle.h"
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define QMAX 19
#define GMAX 8             /* corners per ghost: 4 (bilinear) or 8 (trilinear) */
#define NPHI_FLOOR 1e-6    /* |grad phi| below which n_phi shrinks linearly to 0 */

typedef struct {
    int Q, D;
    int c[QMAX][3];
    double w[QMAX];
    double chi[QMAX];
    int opp[QMAX];
    double M[QMAX][QMAX];
    double Minv[QMAX][QMAX];
    int is_stress[QMAX];
    double alpha, cs2;
} lattice_t;

struct orc_sim {
    orc_params prm;
    lattice_t L;
    int64_t nn;
    uint8_t* cls;          /* 0 fluid, 1 ghost (solid boundary node), 2 bulk solid */
    double *N, *B;         /* [Q][nn] post-streaming populations */
    double* phi;           /* [nn] color (fluid and ghost nodes) */
    double* u;             /* [3][nn] velocity from the last step (0 at solids) */
    double* p;             /* [nn] auxiliary pressure from the last step */
    double *Nst, *Bst, *u_new, *p_new;   /* step scratch, allocated on first step */
    int64_t ng;
    int64_t* g_node;
    double* g_n;           /* [ng][3] */
    int32_t* g_nc;         /* corners used */
    int64_t* g_corner;     /* [ng][GMAX] */
    double* g_wt;          /* [ng][GMAX] */
    int64_t n_fallback;
    double nu_l, nu_g, eps, exp_eps;
    int64_t step;
};

/* ------------------------------------------------------------------ */
/* lattice constants                                                    */
/* ------------------------------------------------------------------ */

/* Gauss-Jordan inverse with partial pivoting, n x n, row-major QMAX stride. */
static int invert(int n, double A[QMAX][QMAX], double Ainv[QMAX][QMAX]) {
    double a[QMAX][2 * QMAX];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j)
            a[i][j] = (j < n) ? A[i][j] : (j - n == i ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (fabs(a[piv][col]) < 1e-300) return -1;
        if (piv != col)
            for (int j = 0; j < 2 * n; ++j) { double t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t; }
        double d = a[col][col];
        for (int j = 0; j < 2 * n; ++j) a[col][j] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double f = a[r][col];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * n; ++j) a[r][j] -= f * a[col][j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ainv[i][j] = a[i][j + n];
    return 0;
}

/* Monomial rows for the Gram-Schmidt construction of M.  The traceless
 * second-order rows come right after the conserved and energy rows, so the
 * stress subspace is exactly their span. */
static double monomial(int D, int k, const int* c) {
    double x = c[0], y = c[1], z = c[2];
    double c2 = x * x + y * y + z * z;
    if (D == 2) {
        switch (k) {
        case 0: return 1;
        case 1: return c2;
        case 2: return x;
        case 3: return y;
        case 4: return x * x - y * y;
        case 5: return x * y;
        case 6: return c2 * c2;
        case 7: return c2 * x;
        case 8: return c2 * y;
        }
    } else {
        switch (k) {
        case 0: return 1;
        case 1: return c2;
        case 2: return x;
        case 3: return y;
        case 4: return z;
        case 5: return 3 * x * x - c2;
        case 6: return y * y - z * z;
        case 7: return x * y;
        case 8: return y * z;
        case 9: return x * z;
        case 10: return c2 * c2;
        case 11: return c2 * x;
        case 12: return c2 * y;
        case 13: return c2 * z;
        case 14: return c2 * (3 * x * x - c2);
        case 15: return c2 * (y * y - z * z);
        case 16: return x * (y * y - z * z);
        case 17: return y * (z * z - x * x);
        case 18: return z * (x * x - y * y);
        }
    }
    return 0;
}

static int gram_schmidt(lattice_t* L) {
    int Q = L->Q;
    for (int k = 0; k < Q; ++k) {
        double v[QMAX];
        for (int i = 0; i < Q; ++i) v[i] = monomial(L->D, k, L->c[i]);
        for (int j = 0; j < k; ++j) {
            double num = 0, den = 0;
            for (int i = 0; i < Q; ++i) { num += v[i] * L->M[j][i]; den += L->M[j][i] * L->M[j][i]; }
            for (int i = 0; i < Q; ++i) v[i] -= (num / den) * L->M[j][i];
        }
        double nrm = 0;
        for (int i = 0; i < Q; ++i) nrm += v[i] * v[i];
        if (nrm < 1e-9) return -1;
        for (int i = 0; i < Q; ++i) L->M[k][i] = v[i];
        L->is_stress[k] = (L->D == 2) ? (k == 4 || k == 5) : (k >= 5 && k <= 9);
    }
    return 0;
}

/* lattice: 9 or 19.  gram_schmidt != 0 builds M for D2Q9 by the same
 * procedure as for D3Q19 (used only by a test); otherwise D2Q9 takes the
 * matrix printed in Appendix A. */
static int build_lattice(lattice_t* L, int lattice, double M_phi, int gs) {
    memset(L, 0, sizeof(*L));
    L->cs2 = 1.0 / 3.0;                     /* c_s = 1/sqrt(3), Appendix A */
    if (lattice == 9) {
        /* lattice velocities and weights, Appendix A */
        static const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        static const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
        L->Q = 9; L->D = 2;
        for (int i = 0; i < 9; ++i) {
            L->c[i][0] = cx[i]; L->c[i][1] = cy[i]; L->c[i][2] = 0;
            L->w[i] = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        }
        if (!gs) {
            /* transformation matrix M, Appendix A */
            static const double Mp[9][9] = {
                { 1,  1,  1,  1,  1, 1,  1,  1,  1},
                {-4, -1, -1, -1, -1, 2,  2,  2,  2},
                { 4, -2, -2, -2, -2, 1,  1,  1,  1},
                { 0,  1,  0, -1,  0, 1, -1, -1,  1},
                { 0, -2,  0,  2,  0, 1, -1, -1,  1},
                { 0,  0,  1,  0, -1, 1,  1, -1, -1},
                { 0,  0, -2,  0,  2, 1,  1, -1, -1},
                { 0,  1, -1,  1, -1, 0,  0,  0,  0},
                { 0,  0,  0,  0,  0, 1, -1,  1, -1}};
            for (int i = 0; i < 9; ++i)
                for (int j = 0; j < 9; ++j) L->M[i][j] = Mp[i][j];
            /* S = diag(1,1,1,1,1,1,1,s7,s8), s7 = s8 = 1/tau */
            L->is_stress[7] = L->is_stress[8] = 1;
        } else if (gram_schmidt(L)) return -1;
    } else if (lattice == 19) {
        static const int c3[19][3] = {
            {0, 0, 0},
            {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
            {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
            {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
            {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        L->Q = 19; L->D = 3;
        for (int i = 0; i < 19; ++i) {
            for (int a = 0; a < 3; ++a) L->c[i][a] = c3[i][a];
            L->w[i] = (i == 0) ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
        }
        if (gram_schmidt(L)) return -1;
    } else {
        return -1;
    }
    for (int i = 0; i < L->Q; ++i) {
        L->opp[i] = -1;
        for (int j = 0; j < L->Q; ++j)
            if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2])
                L->opp[i] = j;
    }
    /* alpha from M_phi = (cs2/2) [ sum_i chi_i c_ix^2 / cs2 + p/cs2 ] at p = 0;
     * for D2Q9 sum_i chi_i c_ix^2 / cs2 = 9(1-alpha)/5 as in Appendix A. */
    double w0 = L->w[0];
    L->alpha = 1.0 - 2.0 * M_phi * (1.0 - w0) / L->cs2;
    if (lattice == 9) {
        /* color weights chi, Eq. (ChiTerm) */
        for (int i = 0; i < 9; ++i)
            L->chi[i] = (i == 0) ? L->alpha : (i <= 4 ? (1.0 - L->alpha) / 5.0 : (1.0 - L->alpha) / 20.0);
    } else {
        for (int i = 0; i < L->Q; ++i)
            L->chi[i] = (i == 0) ? L->alpha : (1.0 - L->alpha) * L->w[i] / (1.0 - w0);
    }
    return invert(L->Q, L->M, L->Minv);
}

/* ------------------------------------------------------------------ */
/* single-node pieces                                                   */
/* ------------------------------------------------------------------ */

/* Eq. (equilibriumDistribution) */
static void equilibrium(const lattice_t* L, const double u[3], double p, double* neq) {
    double cs2 = L->cs2, uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < L->Q; ++i) {
        if (i == 0) {
            neq[0] = L->chi[0] - (1.0 - L->w[0]) * p / cs2 - L->w[0] * uu / (2.0 * cs2);
        } else {
            double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
            neq[i] = L->chi[i] + L->w[i] * (p / cs2 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
        }
    }
}

/* Eqs. (velUpdate) and (pressureUpdate) */
static void macro(const lattice_t* L, const double* N, const double F[3], double rho, double u[3], double* p) {
    for (int a = 0; a < 3; ++a) {
        double j = 0;
        for (int i = 0; i < L->Q; ++i) j += N[i] * L->c[i][a];
        u[a] = j + F[a] / (2.0 * rho);
    }
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double s = 0;
    for (int i = 1; i < L->Q; ++i) s += N[i];
    double w0 = L->w[0];
    *p = (-(w0 / 2.0) * uu - (1.0 - L->chi[0]) * L->cs2 + s * L->cs2) / (1.0 - w0);
}

/* Eq. (MRTCOLL) taken literally: N* = N - M^-1 S M (N - Neq) + M^-1 (I - S/2) M F,
 * with the forcing populations of Eq. (forceGuo). */
static void collide(const lattice_t* L, const double* N, const double u[3], double p,
                    const double F[3], double rho, double tau, double* Nst) {
    int Q = L->Q;
    double neq[QMAX], Fi[QMAX], m[QMAX], meq[QMAX], mF[QMAX], ms[QMAX];
    equilibrium(L, u, p, neq);
    for (int i = 0; i < Q; ++i) {
        double cF = L->c[i][0] * F[0] + L->c[i][1] * F[1] + L->c[i][2] * F[2];
        Fi[i] = (L->w[i] / L->cs2) * cF / rho;
    }
    for (int k = 0; k < Q; ++k) {
        m[k] = meq[k] = mF[k] = 0;
        for (int i = 0; i < Q; ++i) {
            m[k] += L->M[k][i] * N[i];
            meq[k] += L->M[k][i] * neq[i];
            mF[k] += L->M[k][i] * Fi[i];
        }
    }
    for (int k = 0; k < Q; ++k) {
        double s = L->is_stress[k] ? 1.0 / tau : 1.0;
        ms[k] = m[k] - s * (m[k] - meq[k]) + (1.0 - s / 2.0) * mF[k];
    }
    for (int i = 0; i < Q; ++i) {
        double v = 0;
        for (int k = 0; k < Q; ++k) v += L->Minv[i][k] * ms[k];
        Nst[i] = v;
    }
}

/* Eq. (ghost-nodePrescription) */
double orc_ghost_rule(double phiF, double eps) {
    return phiF / (phiF + (1.0 - phiF) * exp(eps));
}

/* Eq. (ghostNodeFakhari), the comparison scheme.  As printed it divides a
 * difference that vanishes with eps by eps (theta = 90 deg needs care,
 * Sec. II); multiplying by the conjugate gives the same expression without
 * that cancellation:  (2/eps)(a - sqrt(a^2 - 2 eps phi_F)) = 4 phi_F / (a + sqrt(...)),
 * a = 1 + eps/2, which is phi_G = phi_F at eps = 0. */
double orc_ghost_rule_fakhari(double phiF, double eps) {
    double a = 1.0 + eps / 2.0;
    return 4.0 * phiF / (a + sqrt(a * a - 2.0 * eps * phiF)) - phiF;
}

/* ------------------------------------------------------------------ */
/* grid helpers                                                         */
/* ------------------------------------------------------------------ */

static int64_t neighbour(const orc_sim* s, int64_t node, int i, int sign) {
    int nx = s->prm.nx, ny = s->prm.ny, nz = s->prm.nz;
    int64_t x = node % nx, y = (node / nx) % ny, z = node / ((int64_t)nx * ny);
    x = ((x + sign * s->L.c[i][0]) % nx + nx) % nx;
    y = ((y + sign * s->L.c[i][1]) % ny + ny) % ny;
    z = ((z + sign * s->L.c[i][2]) % nz + nz) % nz;
    return x + (int64_t)nx * (y + (int64_t)ny * z);
}

static void coords(const orc_sim* s, int64_t node, double r[3]) {
    int nx = s->prm.nx, ny = s->prm.ny;
    r[0] = (double)(node % nx);
    r[1] = (double)((node / nx) % ny);
    r[2] = (double)(node / ((int64_t)nx * ny));
}

/* ------------------------------------------------------------------ */
/* Eq. (segragationStepBlue) with N^{eq,u=0}: B*_i = phi N*_i + (2/W)(c_i . n_phi)
 * phi (1 - phi) N^{eq,u=0}_i, n_phi = grad phi / max(|grad phi|, 1e-6) */
static void segregate(const lattice_t* L, double W, double phi, const double gphi[3], double p,
                      const double* Nst, double* Bst) {
    int Q = L->Q;
    double gn = sqrt(gphi[0] * gphi[0] + gphi[1] * gphi[1] + gphi[2] * gphi[2]);
    double n[3];
    for (int a = 0; a < 3; ++a) n[a] = gphi[a] / (gn > NPHI_FLOOR ? gn : NPHI_FLOOR);
    double neq0[QMAX], zero[3] = {0, 0, 0};
    equilibrium(L, zero, p, neq0);
    for (int i = 0; i < Q; ++i) {
        double cn = L->c[i][0] * n[0] + L->c[i][1] * n[1] + L->c[i][2] * n[2];
        Bst[i] = phi * Nst[i] + 2.0 * (cn / W) * phi * (1.0 - phi) * neq0[i];
    }
}

/* one node: stencils, forces, macroscopic fields, collision, segregation */
/* ------------------------------------------------------------------ */

static void collide_node(const orc_sim* s, const double* phif, int64_t x, double* Nst, double* Bst, double u[3], double* p_out) {
    const lattice_t* L = &s->L;
    const orc_params* P = &s->prm;
    int Q = L->Q;
    int64_t nn = s->nn;
    double N[QMAX];
    for (int i = 0; i < Q; ++i) N[i] = s->N[i * nn + x];
    double phi = phif[x];

    /* isotropic stencils over the lattice neighbours (fluid or ghost) */
    double gphi[3] = {0, 0, 0}, lap = 0, gu[3][3] = {{0}};   /* gu[a][b] = d_a u_b */
    for (int i = 0; i < Q; ++i) {
        int64_t y = neighbour(s, x, i, +1);
        double phin = phif[y];
        double un[3] = {0, 0, 0};
        if (s->cls[y] == 0)
            for (int b = 0; b < 3; ++b) un[b] = s->u[b * nn + y];
        for (int a = 0; a < 3; ++a) gphi[a] += L->w[i] * L->c[i][a] * phin;
        lap += L->w[i] * (phin - phi);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) gu[a][b] += L->w[i] * L->c[i][a] * un[b];
    }
    for (int a = 0; a < 3; ++a) {
        gphi[a] /= L->cs2;
        for (int b = 0; b < 3; ++b) gu[a][b] /= L->cs2;
    }
    lap *= 2.0 / L->cs2;

    /* mixture rules, Sec. II; tau from Appendix A */
    double rho = P->rho_l * phi + P->rho_g * (1.0 - phi);
    double grho[3];
    for (int a = 0; a < 3; ++a) grho[a] = (P->rho_l - P->rho_g) * gphi[a];
    double nu = 1.0 / (phi / s->nu_l + (1.0 - phi) / s->nu_g);
    double tau = 0.5 + nu / L->cs2;

    /* pressure of this step for F_p: Eq. (pressureUpdate) with the force-free
     * velocity sum_i N_i c_i (p depends on the force only through u^2) */
    double u0[3], p0, zeroF[3] = {0, 0, 0};
    macro(L, N, zeroF, rho, u0, &p0);

    /* Eq. (surfaceTensionForce), body force, Eqs. (pressCorrection), (viscCorrection), (totalForce) */
    double mu = (48.0 / P->W) * phi * (1.0 - phi) * (phi - 0.5) + (3.0 * P->W / 2.0) * lap;
    double F[3];
    for (int a = 0; a < 3; ++a) {
        double Fs = -P->sigma * mu * gphi[a];
        double Fb = rho * P->g[a];
        double Fp = -p0 * grho[a];
        double Fv = 0;
        for (int b = 0; b < 3; ++b) Fv += (gu[a][b] + gu[b][a]) * grho[b];
        Fv *= L->cs2 * (tau - 0.5);
        F[a] = Fv + Fp + Fs + Fb;
    }
    if (L->D == 2) F[2] = 0;

    double p;
    macro(L, N, F, rho, u, &p);
    collide(L, N, u, p, F, rho, tau, Nst);

    segregate(L, P->W, phi, gphi, p, Nst, Bst);
    *p_out = p;
}

/* ------------------------------------------------------------------ */
/* ghost table: x_F = x_G + n_s, bilinear/trilinear over fluid corners    */
/* ------------------------------------------------------------------ */

static void build_ghost_entry(orc_sim* s, int64_t g) {
    int D = s->L.D;
    int nxs[3] = {s->prm.nx, s->prm.ny, s->prm.nz};
    double xg[3];
    coords(s, s->g_node[g], xg);
    double base[3] = {0, 0, 0}, f[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
        double xf = xg[a] + s->g_n[3 * g + a];
        base[a] = floor(xf);
        f[a] = xf - base[a];
    }
    int nc = 0;
    double wsum = 0;
    int64_t* cor = s->g_corner + g * GMAX;
    double* wt = s->g_wt + g * GMAX;
    for (int k = 0; k < (1 << D); ++k) {
        int64_t idx[3] = {0, 0, 0};
        double wk = 1.0;
        for (int a = 0; a < D; ++a) {
            int bit = (k >> a) & 1;
            int64_t v = (int64_t)base[a] + bit;
            idx[a] = ((v % nxs[a]) + nxs[a]) % nxs[a];
            wk *= bit ? f[a] : (1.0 - f[a]);
        }
        int64_t node = idx[0] + (int64_t)nxs[0] * (idx[1] + (int64_t)nxs[1] * idx[2]);
        if (s->cls[node] == 0) {
            cor[nc] = node;
            wt[nc] = wk;
            wsum += wk;
            ++nc;
        }
    }
    if (nc > 0 && wsum > 0) {
        for (int k = 0; k < nc; ++k) wt[k] /= wsum;
    } else {
        /* no fluid corner: the fluid lattice neighbour most aligned with n_s
         * (largest c_i . n_s; a tie goes to the smaller node index) */
        int64_t best = -1;
        double best_dot = -INFINITY;
        for (int i = 1; i < s->L.Q; ++i) {
            int64_t y = neighbour(s, s->g_node[g], i, +1);
            if (s->cls[y] != 0) continue;
            double dot = 0;
            for (int a = 0; a < 3; ++a) dot += s->L.c[i][a] * s->g_n[3 * g + a];
            if (dot > best_dot || (dot == best_dot && y < best)) { best_dot = dot; best = y; }
        }
        nc = 1;
        cor[0] = best;
        wt[0] = 1.0;
        s->n_fallback++;
    }
    s->g_nc[g] = nc;
}

/* phi_out[ghost] = rule(interpolated phi_in); phi_out may alias phi_in since
 * corners are fluid nodes and only ghost entries are written. */
static void update_ghosts(const orc_sim* s, const double* phi_in, double* phi_out) {
    for (int64_t g = 0; g < s->ng; ++g) {
        double phiF = 0;
        for (int k = 0; k < s->g_nc[g]; ++k) phiF += s->g_wt[g * GMAX + k] * phi_in[s->g_corner[g * GMAX + k]];
        phi_out[s->g_node[g]] = (s->prm.ghost_rule == 1) ? orc_ghost_rule_fakhari(phiF, s->eps)
                                                         : phiF / (phiF + (1.0 - phiF) * s->exp_eps);
    }
}

/* ------------------------------------------------------------------ */
/* creation and validation                                               */
/* ------------------------------------------------------------------ */

#define FAIL(...) do { if (err) snprintf(err, errlen, __VA_ARGS__); orc_destroy(s); return -1; } while (0)

int orc_create(const orc_params* prm, const uint8_t* solid, const orc_ghost* ghosts,
               int64_t n_ghosts, orc_sim** out, char* err, int errlen) {
    *out = NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    if (!s) { if (err) snprintf(err, errlen, "out of memory"); return -1; }
    s->prm = *prm;
    if (prm->lattice != 9 && prm->lattice != 19) FAIL("lattice must be 9 or 19");
    if (prm->nx < 1 || prm->ny < 1 || prm->nz < 1) FAIL("grid sizes must be positive");
    if (prm->lattice == 9 && prm->nz != 1) FAIL("D2Q9 needs nz == 1");
    if (!(prm->W >= 4.0)) FAIL("W must be >= 4 lattice units");
    if (prm->ghost_rule != 0 && prm->ghost_rule != 1) FAIL("ghost_rule must be 0 or 1");
    if (!(prm->rho_l > 0 && prm->rho_g > 0 && prm->mu_l > 0 && prm->mu_g > 0)) FAIL("densities and viscosities must be positive");
    if (build_lattice(&s->L, prm->lattice, prm->M_phi, 0)) FAIL("lattice construction failed");
    if (!(s->L.alpha > 0 && s->L.alpha < 1)) FAIL("M_phi gives alpha outside (0,1)");
    s->nu_l = prm->mu_l / prm->rho_l;
    s->nu_g = prm->mu_g / prm->rho_g;
    s->eps = -(4.0 / prm->W) * cos(prm->theta);
    s->exp_eps = exp(s->eps);
    int64_t nn = (int64_t)prm->nx * prm->ny * prm->nz;
    s->nn = nn;
    int Q = s->L.Q;
    s->cls = (uint8_t*)calloc(nn, 1);
    s->N = (double*)calloc((size_t)Q * nn, sizeof(double));
    s->B = (double*)calloc((size_t)Q * nn, sizeof(double));
    s->phi = (double*)calloc(nn, sizeof(double));
    s->u = (double*)calloc(3 * (size_t)nn, sizeof(double));
    s->p = (double*)calloc(nn, sizeof(double));
    if (!s->cls || !s->N || !s->B || !s->phi || !s->u || !s->p) FAIL("out of memory");

    /* node classes: a solid node with a fluid lattice neighbour is a ghost (Sec. I) */
    for (int64_t x = 0; x < nn; ++x) s->cls[x] = solid[x] ? 2 : 0;
    for (int64_t x = 0; x < nn; ++x) {
        if (!solid[x]) continue;
        for (int i = 1; i < Q; ++i)
            if (!solid[neighbour(s, x, i, +1)]) { s->cls[x] = 1; break; }
    }
    /* non-periodic axes need solid end layers */
    int nxs[3] = {prm->nx, prm->ny, prm->nz};
    for (int a = 0; a < s->L.D; ++a) {
        if (prm->periodic & (1u << a)) continue;
        for (int64_t x = 0; x < nn; ++x) {
            double r[3];
            coords(s, x, r);
            if ((r[a] == 0 || r[a] == nxs[a] - 1) && !solid[x]) FAIL("axis %d is not periodic but has fluid on an end layer", a);
        }
    }
    /* the ghost list must name every ghost exactly once, with unit normals */
    int64_t n_cls_ghost = 0;
    for (int64_t x = 0; x < nn; ++x) n_cls_ghost += (s->cls[x] == 1);
    if (n_ghosts != n_cls_ghost) FAIL("ghost list has %lld entries, mask has %lld ghost nodes", (long long)n_ghosts, (long long)n_cls_ghost);
    uint8_t* seen = (uint8_t*)calloc(nn, 1);
    if (!seen) FAIL("out of memory");
    s->ng = n_ghosts;
    s->g_node = (int64_t*)calloc(n_ghosts + 1, sizeof(int64_t));
    s->g_n = (double*)calloc(3 * (n_ghosts + 1), sizeof(double));
    s->g_nc = (int32_t*)calloc(n_ghosts + 1, sizeof(int32_t));
    s->g_corner = (int64_t*)calloc(GMAX * (n_ghosts + 1), sizeof(int64_t));
    s->g_wt = (double*)calloc(GMAX * (n_ghosts + 1), sizeof(double));
    if (!s->g_node || !s->g_n || !s->g_nc || !s->g_corner || !s->g_wt) { free(seen); FAIL("out of memory"); }
    for (int64_t g = 0; g < n_ghosts; ++g) {
        int64_t node = ghosts[g].node;
        if (node < 0 || node >= nn || s->cls[node] != 1) { free(seen); FAIL("ghost %lld (node %lld) is not a solid node with a fluid neighbour", (long long)g, (long long)node); }
        if (seen[node]) { free(seen); FAIL("node %lld listed twice", (long long)node); }
        seen[node] = 1;
        double nrm = 0;
        for (int a = 0; a < 3; ++a) nrm += ghosts[g].n[a] * ghosts[g].n[a];
        if (fabs(sqrt(nrm) - 1.0) > 1e-6) { free(seen); FAIL("ghost %lld normal is not a unit vector", (long long)g); }
        if (s->L.D == 2 && ghosts[g].n[2] != 0.0) { free(seen); FAIL("ghost %lld has a z normal on a 2D lattice", (long long)g); }
        s->g_node[g] = node;
        for (int a = 0; a < 3; ++a) s->g_n[3 * g + a] = ghosts[g].n[a];
    }
    free(seen);
    for (int64_t g = 0; g < n_ghosts; ++g) build_ghost_entry(s, g);
    *out = s;
    return 0;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    free(s->cls); free(s->N); free(s->B); free(s->phi); free(s->u); free(s->p);
    free(s->Nst); free(s->Bst); free(s->u_new); free(s->p_new);
    free(s->g_node); free(s->g_n); free(s->g_nc); free(s->g_corner); free(s->g_wt);
    free(s);
}

/* ------------------------------------------------------------------ */
/* initial state                                                         */
/* ------------------------------------------------------------------ */

/* phi given at fluid nodes; ghosts take (1+cos theta)/2 (Sec. III);
 * N = Neq(u=0, p=0) = chi, B = phi N; u = 0, p = 0. */
void orc_init_phi(orc_sim* s, const double* phi) {
    int Q = s->L.Q;
    int64_t nn = s->nn;
    for (int64_t x = 0; x < nn; ++x) {
        s->p[x] = 0;
        for (int a = 0; a < 3; ++a) s->u[a * nn + x] = 0;
        if (s->cls[x] == 0) {
            s->phi[x] = phi[x];
            for (int i = 0; i < Q; ++i) {
                s->N[i * nn + x] = s->L.chi[i];
                s->B[i * nn + x] = phi[x] * s->L.chi[i];
            }
        } else {
            s->phi[x] = (s->cls[x] == 1) ? 0.5 * (1.0 + cos(s->prm.theta)) : 0.0;
            for (int i = 0; i < Q; ++i) s->N[i * nn + x] = s->B[i * nn + x] = 0;
        }
    }
    s->step = 0;
}

/* Eq. (equilibriumPhaseField): phi = (1 + tanh(2 (R0 - |x - c|) / W)) / 2, liquid inside;
 * on periodic axes |x - c| is the distance to the nearest periodic image of c. */
void orc_init_droplet(orc_sim* s, const double centre[3], double R0) {
    double* phi = (double*)malloc(sizeof(double) * s->nn);
    int nxs[3] = {s->prm.nx, s->prm.ny, s->prm.nz};
    for (int64_t x = 0; x < s->nn; ++x) {
        double r[3], d2 = 0;
        coords(s, x, r);
        for (int a = 0; a < s->L.D; ++a) {
            double d = r[a] - centre[a];
            if (s->prm.periodic & (1u << a)) d -= nxs[a] * floor(d / nxs[a] + 0.5);
            d2 += d * d;
        }
        phi[x] = 0.5 * (1.0 + tanh(2.0 * (R0 - sqrt(d2)) / s->prm.W));
    }
    orc_init_phi(s, phi);
    free(phi);
}

/* ------------------------------------------------------------------ */
/* the time step                                                         */
/* ------------------------------------------------------------------ */

void orc_step(orc_sim* s, int64_t nsteps) {
    int Q = s->L.Q;
    int64_t nn = s->nn;
    if (!s->Nst) {
        s->Nst = (double*)calloc((size_t)Q * nn, sizeof(double));
        s->Bst = (double*)calloc((size_t)Q * nn, sizeof(double));
        s->u_new = (double*)calloc(3 * (size_t)nn, sizeof(double));
        s->p_new = (double*)calloc(nn, sizeof(double));
    }
    for (int64_t t = 0; t < nsteps; ++t) {
        /* Eq. (ghost-nodePrescription) at every ghost node */
        update_ghosts(s, s->phi, s->phi);
        /* collision and segregation at every fluid node */
#pragma omp parallel for schedule(static)
        for (int64_t x = 0; x < nn; ++x) {
            if (s->cls[x] != 0) continue;
            double Nst[QMAX], Bst[QMAX], u[3], p;
            collide_node(s, s->phi, x, Nst, Bst, u, &p);
            for (int i = 0; i < Q; ++i) { s->Nst[i * nn + x] = Nst[i]; s->Bst[i * nn + x] = Bst[i]; }
            for (int a = 0; a < 3; ++a) s->u_new[a * nn + x] = u[a];
            s->p_new[x] = p;
        }
        /* propagation with halfway bounce-back, then the color, Eq. (phiUpdate) */
#pragma omp parallel for schedule(static)
        for (int64_t x = 0; x < nn; ++x) {
            if (s->cls[x] != 0) continue;
            double phi = 0;
            for (int i = 0; i < Q; ++i) {
                int64_t src = neighbour(s, x, i, -1);
                int64_t from = (s->cls[src] == 0) ? src : x;
                int iq = (s->cls[src] == 0) ? i : s->L.opp[i];
                s->N[i * nn + x] = s->Nst[iq * nn + from];
                s->B[i * nn + x] = s->Bst[iq * nn + from];
                phi += s->B[i * nn + x];
            }
            s->phi[x] = phi;
            for (int a = 0; a < 3; ++a) s->u[a * nn + x] = s->u_new[a * nn + x];
            s->p[x] = s->p_new[x];
        }
        s->step++;
    }
}

/* ------------------------------------------------------------------ */
/* state access                                                          */
/* ------------------------------------------------------------------ */

static double* field_ptr(const orc_sim* s, int field, int64_t* count) {
    int64_t nn = s->nn;
    switch (field) {
    case ORC_N: *count = s->L.Q * nn; return s->N;
    case ORC_B: *count = s->L.Q * nn; return s->B;
    case ORC_PHI: *count = nn; return s->phi;
    case ORC_U: *count = 3 * nn; return s->u;
    case ORC_P: *count = nn; return s->p;
    }
    *count = 0;
    return NULL;
}

void orc_get(const orc_sim* s, int field, double* out) {
    int64_t cnt;
    double* f = field_ptr(s, field, &cnt);
    if (f) memcpy(out, f, sizeof(double) * cnt);
}

void orc_set(orc_sim* s, int field, const double* in) {
    int64_t cnt;
    double* f = field_ptr(s, field, &cnt);
    if (f) memcpy(f, in, sizeof(double) * cnt);
}

int64_t orc_ghost_fallbacks(const orc_sim* s) { return s->n_fallback; }

/* Eq. (ghost-nodePrescription) applied once to the current color field. */
void orc_update_ghosts(orc_sim* s) { update_ghosts(s, s->phi, s->phi); }

int orc_node_class(const orc_sim* s, int64_t node) { return s->cls[node]; }

void orc_ghost_table(const orc_sim* s, int64_t* corner, double* weight, int32_t* ncorner) {
    for (int64_t g = 0; g < s->ng; ++g) {
        ncorner[g] = s->g_nc[g];
        for (int k = 0; k < GMAX; ++k) {
            corner[g * GMAX + k] = k < s->g_nc[g] ? s->g_corner[g * GMAX + k] : -1;
            weight[g * GMAX + k] = k < s->g_nc[g] ? s->g_wt[g * GMAX + k] : 0.0;
        }
    }
}

/* ------------------------------------------------------------------ */
/* one step evaluated only at sampled nodes (state left untouched)        */
/* ------------------------------------------------------------------ */

static void streamed_at(const orc_sim* s, const double* phif, int64_t x, double* N, double* B) {
    int Q = s->L.Q;
    double Nst[QMAX], Bst[QMAX], u[3], p;
    for (int i = 0; i < Q; ++i) {
        int64_t src = neighbour(s, x, i, -1);
        if (s->cls[src] == 0) {
            collide_node(s, phif, src, Nst, Bst, u, &p);
            N[i] = Nst[i]; B[i] = Bst[i];
        } else {
            collide_node(s, phif, x, Nst, Bst, u, &p);
            N[i] = Nst[s->L.opp[i]]; B[i] = Bst[s->L.opp[i]];
        }
    }
}

/* State after one step at the listed nodes: streamed N and B, u, p and phi at
 * fluid nodes; the ghost color the step's opening ghost update writes at ghost
 * nodes.  The simulation itself is left untouched. */
void orc_step_sample(const orc_sim* s, const int64_t* nodes, int64_t n,
                     double* N_out, double* B_out, double* u_out, double* p_out, double* phi_out) {
    int Q = s->L.Q;
    double* phif = (double*)malloc(sizeof(double) * s->nn);
    memcpy(phif, s->phi, sizeof(double) * s->nn);
    update_ghosts(s, s->phi, phif);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < n; ++k) {
        int64_t x = nodes[k];
        double N[QMAX], B[QMAX];
        for (int i = 0; i < Q; ++i) { N[i] = B[i] = 0; }
        double u[3] = {0, 0, 0}, p = 0, phi = 0;
        if (s->cls[x] == 0) {
            double Nst[QMAX], Bst[QMAX];
            collide_node(s, phif, x, Nst, Bst, u, &p);
            streamed_at(s, phif, x, N, B);
            for (int i = 0; i < Q; ++i) phi += B[i];
        } else if (s->cls[x] == 1) {
            phi = phif[x];
        }
        for (int i = 0; i < Q; ++i) { N_out[k * Q + i] = N[i]; B_out[k * Q + i] = B[i]; }
        for (int a = 0; a < 3; ++a) u_out[3 * k + a] = u[a];
        p_out[k] = p;
        phi_out[k] = phi;
    }
    free(phif);
}

/* ------------------------------------------------------------------ */
/* diagnostics: masses, velocity, pressure jump, interface fit           */
/* ------------------------------------------------------------------ */

/* Solve the small symmetric system A z = b by Gauss-Jordan (n <= 4). */
static int solve_small(int n, double A[4][4], double b[4], double z[4]) {
    double Ab[QMAX][QMAX], Ai[QMAX][QMAX];
    memset(Ab, 0, sizeof(Ab));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ab[i][j] = A[i][j];
    if (invert(n, Ab, Ai)) return -1;
    for (int i = 0; i < n; ++i) {
        z[i] = 0;
        for (int j = 0; j < n; ++j) z[i] += Ai[i][j] * b[j];
    }
    return 0;
}

void orc_diagnostics(const orc_sim* s, const orc_probe* probe, orc_diag* out) {
    const orc_params* P = &s->prm;
    int D = s->L.D;
    int64_t nn = s->nn;
    int nxs[3] = {P->nx, P->ny, P->nz};
    memset(out, 0, sizeof(*out));
    const double delta = 1e-3;
    double sum_in = 0, sum_out = 0, maxu2 = 0;
    for (int64_t x = 0; x < nn; ++x) {
        if (s->cls[x] != 0) continue;
        double phi = s->phi[x];
        out->n_fluid++;
        out->phi_sum += phi;
        out->mass_liquid += P->rho_l * phi;
        out->mass_gas += P->rho_g * (1.0 - phi);
        for (int i = 0; i < s->L.Q; ++i) out->pop_sum += s->N[i * nn + x];
        double u2 = 0;
        for (int a = 0; a < 3; ++a) u2 += s->u[a * nn + x] * s->u[a * nn + x];
        if (u2 > maxu2) maxu2 = u2;
        if (!(u2 == u2) || !(phi == phi)) out->nan_flag = 1;
        double ph = (P->rho_l * phi + P->rho_g * (1.0 - phi)) * s->p[x];   /* p_h = rho p */
        if (phi > 1.0 - delta) { sum_in += ph; out->n_in++; }
        if (phi < delta) { sum_out += ph; out->n_out++; }
    }
    out->max_u = sqrt(maxu2);
    out->p_in = out->n_in ? sum_in / out->n_in : 0;
    out->p_out = out->n_out ? sum_out / out->n_out : 0;
    out->step = s->step;
    out->contact_angle = NAN;
    out->apex = NAN;
    if (!probe || probe->kind == 0) return;

    /* interface points: phi = 1/2 crossings on lattice edges between fluid nodes */
    double A[4][4] = {{0}}, b[4] = {0};
    double apex = -INFINITY;
    for (int64_t x = 0; x < nn; ++x) {
        if (s->cls[x] != 0) continue;
        double r[3];
        coords(s, x, r);
        for (int a = 0; a < D; ++a) {
            double rn[3] = {r[0], r[1], r[2]};
            rn[a] = fmod(rn[a] + 1.0, nxs[a]);
            int64_t y = (int64_t)rn[0] + (int64_t)nxs[0] * ((int64_t)rn[1] + (int64_t)nxs[1] * (int64_t)rn[2]);
            if (s->cls[y] != 0) continue;
            double p0 = s->phi[x], p1 = s->phi[y];
            if ((p0 >= 0.5) == (p1 >= 0.5)) continue;
            double t = (0.5 - p0) / (p1 - p0);
            double q[3] = {0, 0, 0};
            for (int k = 0; k < D; ++k) {
                double v = r[k] + (k == a ? t : 0.0) - probe->center[k];
                v -= nxs[k] * floor(v / nxs[k] + 0.5);        /* nearest periodic image */
                q[k] = v;
            }
            out->n_iface++;
            double h = 0;
            for (int k = 0; k < D; ++k) h += q[k] * probe->normal[k];
            if (h > apex) apex = h;
            double dist;
            if (probe->kind == 1) {
                double d2 = 0;
                for (int k = 0; k < D; ++k) d2 += q[k] * q[k];
                dist = sqrt(d2) - probe->radius;
            } else {
                dist = h;
            }
            if (dist < probe->exclude) continue;
            /* Kasa circle/sphere fit: |q|^2 + sum_k a_k q_k + b0 = 0 */
            double row[4] = {0, 0, 0, 1};
            double q2 = 0;
            for (int k = 0; k < D; ++k) { row[k] = q[k]; q2 += q[k] * q[k]; }
            row[D] = 1.0;
            for (int i = 0; i <= D; ++i) {
                for (int j = 0; j <= D; ++j) A[i][j] += row[i] * row[j];
                b[i] += -q2 * row[i];
            }
            out->n_fit++;
        }
    }
    out->apex = apex;
    double z[4];
    if (out->n_fit < D + 2 || solve_small(D + 1, A, b, z)) return;
    double c2 = 0;
    for (int k = 0; k < D; ++k) {
        double ck = -z[k] / 2.0;
        out->fit_center[k] = ck + probe->center[k];
        c2 += ck * ck;
    }
    out->fit_radius = sqrt(c2 - z[D]);
    double r = out->fit_radius;
    if (probe->kind == 1) {
        double R = probe->radius, d = sqrt(c2);
        out->contact_angle = acos((R * R + r * r - d * d) / (2.0 * R * r));
    } else {
        double h = 0;
        for (int k = 0; k < D; ++k) h += (-z[k] / 2.0) * probe->normal[k];
        out->contact_angle = acos(-h / r);
    }
}

/* ------------------------------------------------------------------ */
/* single-node entry points for the pins                                 */
/* ------------------------------------------------------------------ */

int orc_lattice_tables(int lattice, double M_phi, int gram_schmidt, int32_t* c, double* w,
                       double* chi, int32_t* opp, double* M, double* Minv, int32_t* is_stress) {
    lattice_t L;
    if (build_lattice(&L, lattice, M_phi, gram_schmidt)) return -1;
    int Q = L.Q;
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
        w[i] = L.w[i];
        chi[i] = L.chi[i];
        opp[i] = L.opp[i];
        is_stress[i] = L.is_stress[i];
        for (int j = 0; j < Q; ++j) { M[i * Q + j] = L.M[i][j]; Minv[i * Q + j] = L.Minv[i][j]; }
    }
    return Q;
}

void orc_equilibrium(int lattice, double M_phi, const double u[3], double p, double* neq) {
    lattice_t L;
    build_lattice(&L, lattice, M_phi, 0);
    equilibrium(&L, u, p, neq);
}

void orc_macro(int lattice, double M_phi, const double* N, const double F[3], double rho, double u[3], double* p) {
    lattice_t L;
    build_lattice(&L, lattice, M_phi, 0);
    macro(&L, N, F, rho, u, p);
}

void orc_collide(int lattice, double M_phi, const double* N, const double u[3], double p,
                 const double F[3], double rho, double tau, double* Nst) {
    lattice_t L;
    build_lattice(&L, lattice, M_phi, 0);
    collide(&L, N, u, p, F, rho, tau, Nst);
}

void orc_segregate(int lattice, double M_phi, double W, double phi, const double gphi[3], double p,
                   const double* Nst, double* Bst) {
    lattice_t L;
    build_lattice(&L, lattice, M_phi, 0);
    segregate(&L, W, phi, gphi, p, Nst, Bst);
}
