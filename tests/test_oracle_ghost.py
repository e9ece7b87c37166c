"""Pins for the ghost-node wetting rule, Eq. (ghost-nodePrescription), and the
oracle's ghost table (x_F = x_G + n_s with bilinear/trilinear weights, Fig. 2)."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle
from paper_2605_30878_gb300 import workloads as wl


def fakhari(phiF, eps):
    """Eq. (ghostNodeFakhari)."""
    a = 1 + eps / 2
    return (2 / eps) * (a - math.sqrt(a * a - 2 * eps * phiF)) - phiF


def test_fixed_points_and_range():
    for eps in np.linspace(-1, 1, 21):
        assert oracle.ghost_rule(0.0, eps) == 0.0
        assert oracle.ghost_rule(1.0, eps) == 1.0
        for phiF in np.linspace(0.01, 0.99, 25):
            g = oracle.ghost_rule(phiF, eps)
            assert 0.0 < g < 1.0
    for phiF in np.linspace(0, 1, 11):                      # theta = 90 deg -> eps = 0
        assert abs(oracle.ghost_rule(phiF, 0.0) - phiF) < 1e-16


def test_logistic_shift_identity():
    """With phi_F = 1/(1+exp(-s)) the rule gives 1/(1+exp(-(s - eps))): the
    equilibrium tanh profile continued by one lattice spacing."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        s, eps = rng.uniform(-8, 8), rng.uniform(-1, 1)
        phiF = 1 / (1 + math.exp(-s))
        assert abs(oracle.ghost_rule(phiF, eps) - 1 / (1 + math.exp(-(s - eps)))) < 1e-15


@pytest.mark.parametrize("theta_deg", [30, 60, 120, 150])
def test_rule_integrates_the_normal_ode(theta_deg):
    """Eq. (odePhiNs), d phi/d eta_s = -(4/W) phi (1-phi) cos(theta), integrated from
    x_G (phi_G) over one lattice spacing, reaches phi_F."""
    W = 4.0
    eps = -(4.0 / W) * math.cos(math.radians(theta_deg))
    for phiF in (0.05, 0.3, 0.5, 0.8, 0.97):
        phiG = oracle.ghost_rule(phiF, eps)
        sol = solve_ivp(lambda t, y: -(4 / W) * y * (1 - y) * math.cos(math.radians(theta_deg)),
                        (0, 1), [phiG], rtol=1e-12, atol=1e-14)
        assert abs(sol.y[0, -1] - phiF) < 1e-9


def test_difference_from_fakhari_is_the_cubic_series():
    """Eq. (differenceSeriesPrescription): the two rules differ by
    (eps^3/12)[1 - 3(1-phi_F)phi_F] phi_F (1-phi_F) + O(eps^4)."""
    for phiF in (0.1, 0.3, 0.5, 0.7):
        res = []
        for eps in (0.04, 0.02, 0.01):
            series = eps ** 3 / 12 * (1 - 3 * (1 - phiF) * phiF) * phiF * (1 - phiF)
            diff = oracle.ghost_rule(phiF, eps) - fakhari(phiF, eps)
            res.append(abs(diff - series))
            assert abs(diff - series) < 0.05 * eps ** 3
        # the remainder shrinks at least like eps^4 (ratio 16 per halving, allow 12)
        assert res[0] / max(res[1], 1e-300) > 12 or res[0] < 1e-15


def _planar_profile(x, y, theta, W, x0, y0):
    """Equilibrium tanh interface meeting the wall y = const (normal +y) at theta:
    n_phi = (sin theta, -cos theta) so that n_s . n_phi = -cos theta (Eq. sharpWettingCondition)."""
    eta = math.sin(theta) * (x - x0) - math.cos(theta) * (y - y0)
    return wl.tanh_field(eta, W)


@pytest.mark.parametrize("theta_deg", [30, 60, 90, 135])
def test_grid_aligned_wall_extends_the_profile_exactly(theta_deg):
    nx, ny, W = 40, 16, 4.0
    solid, ghosts = wl.wall_domain(9, (1, ny, nx), bottom=1, top=1)
    prm = dict(lattice=9, nx=nx, ny=ny, nz=1, periodic=1, rho_l=1, rho_g=1, mu_l=1 / 6, mu_g=1 / 6,
               sigma=0.01, W=W, M_phi=0.02, theta=math.radians(theta_deg))
    o = oracle.Oracle(prm, solid, ghosts)
    assert o.ghost_fallbacks() == 0
    _, y, x = wl.node_coords((1, ny, nx))
    exact = _planar_profile(x, y, math.radians(theta_deg), W, nx / 2, 3.0).reshape(-1)
    phi = np.where(solid.reshape(-1) == 0, exact, 0.0)
    o.set("phi", phi)
    o.update_ghosts()
    got = o.get("phi")
    bottom = (y.reshape(-1) == 0)
    assert np.abs(got[bottom] - exact[bottom]).max() < 1e-14


def test_grid_aligned_wall_3d():
    n, W, theta = 12, 4.0, math.radians(50)
    solid, ghosts = wl.wall_domain(19, (n, n, n), bottom=1, top=1)
    prm = dict(lattice=19, nx=n, ny=n, nz=n, periodic=3, rho_l=1, rho_g=1, mu_l=1 / 6, mu_g=1 / 6,
               sigma=0.01, W=W, M_phi=0.02, theta=theta)
    o = oracle.Oracle(prm, solid, ghosts)
    z, y, x = wl.node_coords((n, n, n))
    # interface normal with -cos(theta) along the wall normal (+z) and the rest in the x-y plane
    nphi = np.array([math.sin(theta) * 0.6, math.sin(theta) * 0.8, -math.cos(theta)])
    eta = nphi[0] * (x - 6) + nphi[1] * (y - 6) + nphi[2] * (z - 3)
    exact = wl.tanh_field(eta, W).reshape(-1)
    o.set("phi", np.where(solid.reshape(-1) == 0, exact, 0.0))
    o.update_ghosts()
    bottom = z.reshape(-1) == 0
    assert np.abs(o.get("phi")[bottom] - exact[bottom]).max() < 1e-14


def _check_weights(o, nodes, normals, shape, D):
    cor, wt, nc = o.ghost_table()
    nz, ny, nx = shape
    dims = np.array([nx, ny, nz])
    full = 0
    for g in range(len(nodes)):
        k = nc[g]
        assert k >= 1
        assert abs(wt[g, :k].sum() - 1) < 1e-14 and (wt[g, :k] >= 0).all()
        for c in cor[g, :k]:
            assert o.node_class(c) == 0                        # corners are fluid nodes
        xg = np.array([nodes[g] % nx, (nodes[g] // nx) % ny, nodes[g] // (nx * ny)], float)
        xf = xg + normals[g]
        if k == 2 ** D:
            full += 1
            pts = np.stack([cor[g, :k] % nx, (cor[g, :k] // nx) % ny, cor[g, :k] // (nx * ny)], 1).astype(float)
            # minimal image of each corner relative to x_F
            d = pts - xf[None, :]
            d -= dims[None, :] * np.round(d / dims[None, :])
            assert np.abs(wt[g, :k] @ d[:, :D]).max() < 1e-12   # bilinear weights reproduce x_F
            assert np.abs(d[:, :D]).max() < 1.0 + 1e-12
    return full


def test_curved_ghost_table_2d():
    cfg = wl.cylinder_config()
    o = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])
    full = _check_weights(o, cfg["ghosts"][0], cfg["ghosts"][1], (1, 64, 64), 2)
    assert full > 0


def test_curved_ghost_table_3d():
    cfg = wl.sphere_config(n=32, R=8, R0=6)
    o = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])
    full = _check_weights(o, cfg["ghosts"][0], cfg["ghosts"][1], (32, 32, 32), 3)
    assert full > 0


def test_ghost_list_validation():
    cfg = wl.cylinder_config()
    nodes, normals = cfg["ghosts"]
    with pytest.raises(ValueError):
        oracle.Oracle(cfg["params"], cfg["solid"], (nodes[:-1], normals[:-1]))      # one missing
    bad = normals.copy()
    bad[0] *= 1.1
    with pytest.raises(ValueError):
        oracle.Oracle(cfg["params"], cfg["solid"], (nodes, bad))                    # not unit
    prm = dict(cfg["params"], W=3.0)
    with pytest.raises(ValueError):
        oracle.Oracle(prm, cfg["solid"], cfg["ghosts"])                             # W < 4


def test_fakhari_rule_solves_its_midpoint_relation():
    """Eq. (ghostNodeFakhari) is the root of the wetting ODE discretised at the
    midpoint s = (phi_G + phi_F)/2: phi_F - phi_G = eps s (1 - s)."""
    rng = np.random.default_rng(12)
    for _ in range(200):
        phiF, eps = rng.uniform(0, 1), rng.uniform(-1, 1)
        g = oracle.ghost_rule_fakhari(phiF, eps)
        s = 0.5 * (g + phiF)
        assert abs((phiF - g) - eps * s * (1 - s)) < 1e-15
    for eps in (-1.0, -0.3, 0.4, 1.0):
        assert abs(oracle.ghost_rule_fakhari(0.0, eps)) < 1e-15
        assert abs(oracle.ghost_rule_fakhari(1.0, eps) - 1.0) < 1e-14
    for phiF in np.linspace(0, 1, 11):
        assert oracle.ghost_rule_fakhari(phiF, 0.0) == phiF            # theta = 90 deg
        # eps computed from theta = pi/2 is -6e-17, not 0: the rule must still return phi_F
        eps90 = -(4.0 / 4.0) * math.cos(math.pi / 2)
        assert abs(oracle.ghost_rule_fakhari(phiF, eps90) - phiF) < 1e-15
    for eps in (1e-3, 1e-8, -1e-12):                                   # well conditioned near 0
        phiF = 0.37
        g = oracle.ghost_rule_fakhari(phiF, eps)
        s = 0.5 * (g + phiF)
        assert abs((phiF - g) - eps * s * (1 - s)) < 4e-16          # a few ulps of phi


def test_oracle_rules_differ_by_the_papers_series():
    """Eq. (differenceSeriesPrescription) between the oracle's two rules."""
    for phiF in (0.2, 0.5, 0.8):
        for eps in (0.02, -0.02, 0.01):
            series = eps ** 3 / 12 * (1 - 3 * (1 - phiF) * phiF) * phiF * (1 - phiF)
            diff = oracle.ghost_rule(phiF, eps) - oracle.ghost_rule_fakhari(phiF, eps)
            assert abs(diff - series) < 0.05 * abs(eps) ** 3


def test_grid_ghost_update_uses_the_selected_rule():
    nx, ny, W, theta = 40, 16, 4.0, math.radians(40)
    solid, ghosts = wl.wall_domain(9, (1, ny, nx), bottom=1, top=1)
    prm = dict(lattice=9, nx=nx, ny=ny, nz=1, periodic=1, rho_l=1, rho_g=1, mu_l=1 / 6, mu_g=1 / 6,
               sigma=0.01, W=W, M_phi=0.02, theta=theta, ghost_rule=1)
    o = oracle.Oracle(prm, solid, ghosts)
    _, y, x = wl.node_coords((1, ny, nx))
    exact = _planar_profile(x, y, theta, W, nx / 2, 3.0).reshape(-1)
    o.set("phi", np.where(solid.reshape(-1) == 0, exact, 0.0))
    o.update_ghosts()
    got = o.get("phi")
    eps = -(4.0 / W) * math.cos(theta)
    for xx in range(nx):
        g, f = xx, xx + nx                      # ghost (x, 0) and its fluid point (x, 1)
        assert abs(got[g] - oracle.ghost_rule_fakhari(exact[f], eps)) < 1e-15
