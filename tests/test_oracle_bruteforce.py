"""Brute force on tiny grids (D2Q9 8x8, D3Q19 5x4x4): one time step written as
dense NumPy operators -- shift matrices for the stencils, the paper's M and S
of Appendix A for a literal M^-1 [...] M collision, and a (Q*n) x (Q*n)
streaming matrix with halfway bounce-back -- against the oracle's loop-based
step on the same state.

The formulation follows Appendix A of the paper (Eqs. MRTCOLL,
equilibriumDistribution, forceGuo, totalForce, pressCorrection,
viscCorrection, segragationStepBlue, phiUpdate, velUpdate, pressureUpdate,
propTotal, propBlue), Eq. (surfaceTensionForce), the ghost rule of Eq.
(ghost-nodePrescription) and the readings taken where the paper is
silent: isotropic lattice stencils, halfway bounce-back, the force-free
pressure in F_p and the previous step's velocity in F_visc, the ghost update
at the start of the step, n_phi = grad phi / max(|grad phi|, 1e-6).  The
ghost interpolation table (corners and weights of x_F) is geometry: it is
taken from the oracle as an input here and pinned on its own in
test_oracle_ghost.py.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_30878_gb300 import workloads as wl

# Appendix A, D2Q9: velocities, weights, the transformation matrix M
C = np.array([[0, 1, 0, -1, 0, 1, -1, -1, 1],
              [0, 0, 1, 0, -1, 1, 1, -1, -1]])
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
M = np.array([[1, 1, 1, 1, 1, 1, 1, 1, 1],
              [-4, -1, -1, -1, -1, 2, 2, 2, 2],
              [4, -2, -2, -2, -2, 1, 1, 1, 1],
              [0, 1, 0, -1, 0, 1, -1, -1, 1],
              [0, -2, 0, 2, 0, 1, -1, -1, 1],
              [0, 0, 1, 0, -1, 1, 1, -1, -1],
              [0, 0, -2, 0, 2, 1, 1, -1, -1],
              [0, 1, -1, 1, -1, 0, 0, 0, 0],
              [0, 0, 0, 0, 0, 1, -1, 1, -1]], dtype=float)
CS2 = 1.0 / 3.0
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]

# D3Q19 (the model's 3D extension; not in the paper): rest, +-x, +-y, +-z,
# then the twelve edges in +- pairs; w = 1/3, 1/18, 1/36
C19 = np.array([[0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
                [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1],
                [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]])
W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
OPP19 = [0] + [i + 1 if i % 2 else i - 1 for i in range(1, 19)]


def d3q19_moment_basis():
    """An orthogonal moment basis whose rows 4..8 span the five traceless
    second-order moments (relaxed at 1/tau); every other row relaxes at 1, so
    the collision does not depend on which such basis is taken."""
    cx, cy, cz = C19
    c2 = cx * cx + cy * cy + cz * cz
    rows = [np.ones(19), cx, cy, cz, 3 * cx * cx - c2, cy * cy - cz * cz, cx * cy, cy * cz, cx * cz]
    A = np.array(rows, dtype=float).T                         # 19 x 9, columns mutually orthogonal
    rest = np.linalg.qr(np.hstack([A, np.eye(19)]))[0][:, 9:19]   # orthonormal complement
    rest -= A @ np.linalg.lstsq(A, rest, rcond=None)[0]
    return np.vstack([A.T, rest.T]), [4, 5, 6, 7, 8]


def shift_matrix(nx, ny, cx, cy):
    """(S f)[x] = f[x + c] on the periodic nx x ny grid, node = x + nx*y."""
    n = nx * ny
    S = np.zeros((n, n))
    for y in range(ny):
        for x in range(nx):
            S[x + nx * y, (x + cx) % nx + nx * ((y + cy) % ny)] = 1.0
    return S


def shift_matrix3(nx, ny, nz, c):
    """(S f)[x] = f[x + c] on the periodic grid, node = x + nx*(y + ny*z)."""
    n = nx * ny * nz
    S = np.zeros((n, n))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                S[x + nx * (y + ny * z), (x + c[0]) % nx + nx * ((y + c[1]) % ny + ny * ((z + c[2]) % nz))] = 1.0
    return S


def brute_force_step(state, P, solid, corners, weights, nx, ny, nz=1):
    Q = P["lattice"]
    D = 2 if Q == 9 else 3
    n = nx * ny * nz
    fluid = solid.reshape(-1) == 0
    if Q == 9:
        Cq, Wq, opp, Mq, stress = C, W9, OPP, M, [7, 8]
        alpha = 1.0 - 10.0 * P["M_phi"] / 3.0
        chi = np.array([alpha] + [(1 - alpha) / 5] * 4 + [(1 - alpha) / 20] * 4)
    else:
        Cq, Wq, opp = C19, W19, OPP19
        Mq, stress = d3q19_moment_basis()
        alpha = 1.0 - 2.0 * P["M_phi"] * (1 - Wq[0]) / CS2
        chi = np.concatenate([[alpha], (1 - alpha) * Wq[1:] / (1 - Wq[0])])
    C_, W_ = Cq, Wq
    N, B = state["N"].copy(), state["B"].copy()              # (Q, n)
    phi, u_prev = state["phi"].copy(), state["u"][:D].copy()
    shifts = [shift_matrix3(nx, ny, nz, C_[:, i]) if D == 3 else shift_matrix(nx, ny, C_[0, i], C_[1, i])
              for i in range(Q)]
    # ghost rule at every ghost node from the current fluid color (Jacobi)
    eps = -(4.0 / P["W"]) * math.cos(P["theta"])
    ghosts = state["ghost_nodes"]
    phiF = np.sum(weights * phi[corners], axis=1)
    phi[ghosts] = phiF / (phiF + (1 - phiF) * math.exp(eps))
    # stencils as operators: grad f = (1/cs2) sum w_i c_i S_i f, lap f = (2/cs2) sum w_i (S_i f - f)
    G = [sum(W_[i] * C_[a, i] * shifts[i] for i in range(Q)) / CS2 for a in range(D)]
    Lap = sum(W_[i] * (shifts[i] - np.eye(n)) for i in range(Q)) * (2.0 / CS2)
    gphi = np.stack([G[a] @ phi for a in range(D)])           # (D, n)
    lap = Lap @ phi
    du = np.array([[G[a] @ u_prev[b] for b in range(D)] for a in range(D)])   # du[a, b] = d_a u_b
    rho = P["rho_l"] * phi + P["rho_g"] * (1 - phi)
    nu = 1.0 / (phi / (P["mu_l"] / P["rho_l"]) + (1 - phi) / (P["mu_g"] / P["rho_g"]))
    tau = 0.5 + nu / CS2
    grho = (P["rho_l"] - P["rho_g"]) * gphi
    # force-free velocity and the pressure it gives (Eq. pressureUpdate)
    u0 = C_ @ N
    press = lambda uu: (-W_[0] / 2 * (uu ** 2).sum(0) - (1 - chi[0]) * CS2 + CS2 * N[1:].sum(0)) / (1 - W_[0])  # noqa: E731
    p0 = press(u0)
    Fs = -P["sigma"] * (48 / P["W"] * phi * (1 - phi) * (phi - 0.5) + 1.5 * P["W"] * lap) * gphi
    Fb = rho * np.array(P["g"][:D])[:, None]
    Fp = -p0 * grho
    sym = du + du.transpose(1, 0, 2)
    Fv = CS2 * (tau - 0.5) * np.einsum("abn,bn->an", sym, grho)
    F = Fv + Fp + Fs + Fb
    u = u0 + F / (2 * rho)
    p = press(u)
    # equilibrium, forcing, literal MRT collision per node
    cu = C_.T @ u                                              # (Q, n)
    uu = (u ** 2).sum(0)
    Neq = chi[:, None] + W_[:, None] * (p / CS2 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - uu / (2 * CS2))
    Neq[0] = chi[0] - (1 - W_[0]) * p / CS2 - W_[0] * uu / (2 * CS2)
    Fi = W_[:, None] / CS2 * (C_.T @ F) / rho
    Minv = np.linalg.inv(Mq)
    Nst = np.zeros_like(N)
    for x in np.flatnonzero(fluid):
        sdiag = np.ones(Q)
        sdiag[stress] = 1 / tau[x]
        S = np.diag(sdiag)
        Nst[:, x] = (N[:, x] - Minv @ S @ Mq @ (N[:, x] - Neq[:, x])
                     + Minv @ (np.eye(Q) - S / 2) @ Mq @ Fi[:, x])
    # segregation (Eq. segragationStepBlue) with N^{eq, u=0}
    gn = np.sqrt((gphi ** 2).sum(0))
    nhat = gphi / np.maximum(gn, 1e-6)
    Neq0 = chi[:, None] + W_[:, None] * p / CS2
    Neq0[0] = chi[0] - (1 - W_[0]) * p / CS2
    Bst = phi * Nst + 2 * (C_.T @ nhat) / P["W"] * phi * (1 - phi) * Neq0
    # streaming with halfway bounce-back as one (Qn x Qn) matrix on the fluid nodes
    T = np.zeros((Q * n, Q * n))
    for i in range(Q):
        back = shifts[opp[i]]                                 # (S_opp f)[x] = f[x - c_i]
        for x in np.flatnonzero(fluid):
            src = int(np.argmax(back[x]))
            if fluid[src]:
                T[i * n + x, i * n + src] = 1.0
            else:
                T[i * n + x, opp[i] * n + x] = 1.0
    Nn = (T @ Nst.reshape(-1)).reshape(Q, n)
    Bn = (T @ Bst.reshape(-1)).reshape(Q, n)
    phin = phi.copy()
    phin[fluid] = Bn[:, fluid].sum(0)
    return dict(N=Nn, B=Bn, phi=phin, u=u, p=p)


@pytest.mark.parametrize("rho_ratio,theta_deg", [(1.0, 60.0), (10.0, 120.0)])
def test_one_step_equals_the_dense_operator_formulation(rho_ratio, theta_deg):
    nx = ny = 8
    solid = np.zeros((1, ny, nx), np.uint8)
    solid[0, 3:6, 2:5] = 1                                    # 3x3 block: 8 ghosts around a bulk solid node
    ghosts = wl.ghost_list(solid, 9, wl._radial_normals((3.0, 4.0, 0.0), 2))
    P = dict(lattice=9, nx=nx, ny=ny, nz=1, periodic=7, rho_l=rho_ratio, rho_g=1.0, mu_l=0.2, mu_g=0.1,
             sigma=0.01, W=4.0, M_phi=0.02, theta=math.radians(theta_deg), g=(1e-6, -2e-6, 0))
    o = oracle.Oracle(P, solid, ghosts)
    n = nx * ny
    fl = solid.reshape(-1) == 0
    rng = np.random.default_rng(7)
    xs, ys = np.meshgrid(np.arange(nx), np.arange(ny))
    phi = (0.5 + 0.45 * np.sin(2 * np.pi * xs / nx + 0.3) * np.cos(2 * np.pi * ys / ny)).reshape(-1)
    phi[~fl] = 0.0
    alpha = 1.0 - 10.0 * 0.02 / 3.0
    chi = np.array([alpha] + [(1 - alpha) / 5] * 4 + [(1 - alpha) / 20] * 4)
    N = chi[:, None] * (1 + 0.02 * rng.standard_normal((9, n)))
    N[:, ~fl] = 0.0
    B = N * phi[None, :] * (1 + 0.01 * rng.standard_normal((9, n)))
    phi[fl] = B[:, fl].sum(0)
    u = np.zeros((3, n))
    u[:2, fl] = 1e-3 * rng.standard_normal((2, fl.sum()))
    p = np.zeros(n)
    p[fl] = 1e-4 * rng.standard_normal(fl.sum())
    for f, v in (("N", N), ("B", B), ("phi", phi), ("u", u), ("p", p)):
        o.set(f, v)
    cor, wt, _ = o.ghost_table()
    state = dict(N=N, B=B, phi=phi, u=u, ghost_nodes=ghosts[0])
    want = brute_force_step(state, P, solid, cor[:, :4], wt[:, :4], nx, ny)
    o.step(1)
    for f in ("N", "B"):
        a, b = o.get(f)[:, fl], want[f][:, fl]
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max(), f
    assert np.abs(o.get("u")[:2, fl] - want["u"][:, fl]).max() <= 1e-15
    assert np.abs(o.get("p")[fl] - want["p"][fl]).max() <= 1e-15
    ph, pw = o.get("phi"), want["phi"]
    assert np.abs(ph[fl] - pw[fl]).max() <= 1e-13
    assert np.abs(ph[ghosts[0]] - pw[ghosts[0]]).max() <= 1e-14


@pytest.mark.parametrize("rho_ratio,theta_deg", [(1.0, 45.0), (10.0, 135.0)])
def test_one_step_d3q19_equals_the_dense_operator_formulation(rho_ratio, theta_deg):
    nx, ny, nz = 5, 4, 4
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[1:3, 1:3, 1:3] = 1                                  # 2x2x2 block, every node a ghost
    ghosts = wl.ghost_list(solid, 19, wl._radial_normals((1.5, 1.5, 1.5), 3))
    P = dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=7, rho_l=rho_ratio, rho_g=1.0, mu_l=0.2, mu_g=0.1,
             sigma=0.01, W=4.0, M_phi=0.02, theta=math.radians(theta_deg), g=(1e-6, -2e-6, 3e-6))
    o = oracle.Oracle(P, solid, ghosts)
    n = nx * ny * nz
    fl = solid.reshape(-1) == 0
    rng = np.random.default_rng(9)
    zs, ys, xs = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = (0.5 + 0.4 * np.sin(2 * np.pi * xs / nx + 0.3) * np.cos(2 * np.pi * (ys / ny + zs / nz))).reshape(-1)
    phi[~fl] = 0.0
    alpha = 1.0 - 2.0 * 0.02 * (2.0 / 3.0) * 3.0
    chi = np.concatenate([[alpha], (1 - alpha) * W19[1:] / (1 - W19[0])])
    N = chi[:, None] * (1 + 0.02 * rng.standard_normal((19, n)))
    N[:, ~fl] = 0.0
    B = N * phi[None, :] * (1 + 0.01 * rng.standard_normal((19, n)))
    phi[fl] = B[:, fl].sum(0)
    u = np.zeros((3, n))
    u[:, fl] = 1e-3 * rng.standard_normal((3, fl.sum()))
    p = np.zeros(n)
    p[fl] = 1e-4 * rng.standard_normal(fl.sum())
    for f, v in (("N", N), ("B", B), ("phi", phi), ("u", u), ("p", p)):
        o.set(f, v)
    cor, wt, _ = o.ghost_table()
    state = dict(N=N, B=B, phi=phi, u=u, ghost_nodes=ghosts[0])
    want = brute_force_step(state, P, solid, cor[:, :8], wt[:, :8], nx, ny, nz)
    o.step(1)
    for f in ("N", "B"):
        a, b = o.get(f)[:, fl], want[f][:, fl]
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max(), f
    assert np.abs(o.get("u")[:, fl] - want["u"][:, fl]).max() <= 1e-15
    assert np.abs(o.get("p")[fl] - want["p"][fl]).max() <= 1e-15
    ph, pw = o.get("phi"), want["phi"]
    assert np.abs(ph[fl] - pw[fl]).max() <= 1e-13
    assert np.abs(ph[ghosts[0]] - pw[ghosts[0]]).max() <= 1e-14
