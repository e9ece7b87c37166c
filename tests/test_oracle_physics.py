"""Whole-model pins for the oracle: results the mathematics or the paper fixes
(shear-wave viscosity, exact Poiseuille flow with halfway bounce-back,
stationary planar interface, two-layer channel flow, Laplace law, exact mass
conservation, mirror symmetry, equilibrium drop shapes and contact angles)."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_bvp
from scipy.optimize import brentq

import oracle
from paper_2605_30878_gb300 import workloads as wl

EMPTY = (np.zeros(0, np.int64), np.zeros((0, 3)))


def _base(Q, shape, **kw):
    nz, ny, nx = shape
    p = dict(lattice=Q, nx=nx, ny=ny, nz=nz, periodic=7, rho_l=1.0, rho_g=1.0, mu_l=1 / 6, mu_g=1 / 6,
             sigma=0.01, W=4.0, M_phi=0.02, theta=math.pi / 2, g=(0, 0, 0))
    p.update(kw)
    return p


def _single_phase(o, Q, u_field, solid):
    """phi = 1 everywhere (one phase), N = Neq(u, p=0), B = N."""
    nn = solid.size
    fluid = solid.reshape(-1) == 0
    N = np.zeros((Q, nn))
    for x in np.nonzero(fluid)[0]:
        N[:, x] = oracle.equilibrium(Q, u_field[:, x], 0.0)
    o.set("N", N)
    o.set("B", N)
    o.set("phi", fluid.astype(float))
    o.set("u", u_field * fluid[None, :])
    o.set("p", np.zeros(nn))


@pytest.mark.parametrize("Q", [9, 19])
@pytest.mark.parametrize("tau", [0.6, 1.3])
def test_shear_wave_decays_at_the_lattice_viscosity(Q, tau):
    """A shear wave u_x = U sin(k y) decays as exp(-nu k^2 t), nu = cs2 (tau - 1/2)."""
    shape = (1, 32, 2) if Q == 9 else (2, 32, 2)
    nu = (tau - 0.5) / 3
    solid = np.zeros(shape, np.uint8)
    o = oracle.Oracle(_base(Q, shape, mu_l=nu, mu_g=nu, sigma=0.0), solid, EMPTY)
    _, y, _ = wl.node_coords(shape)
    y = y.reshape(-1).astype(float)
    k = 2 * math.pi / shape[1]
    u = np.zeros((3, y.size))
    u[0] = 1e-4 * np.sin(k * y)
    _single_phase(o, Q, u, solid)
    ts, amps = [], []
    for t in range(0, 301, 10):
        if t:
            o.step(10)
        if t >= 30:
            ts.append(t)
            amps.append(2.0 / y.size * np.sum(o.get("u")[0] * np.sin(k * y)))
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    assert abs(rate / (nu * k * k) - 1) < 3e-3


@pytest.mark.parametrize("Q", [9, 19])
def test_poiseuille_is_exact_at_the_magic_tau(Q):
    """Body-force channel flow between halfway bounce-back walls at y = 1/2 and
    H + 1/2.  With every non-stress rate 1 and tau = 7/8, (tau-1/2)(1-1/2) = 3/16 and
    the parabola is reproduced to rounding; at tau = 1 the wall slip stays small."""
    H, g = 16, 1e-6
    shape = (1, H + 2, 2) if Q == 9 else (H + 2, 2, 2)
    for tau, tol in ((7 / 8, 1e-9), (1.0, 2e-3)):
        nu = (tau - 0.5) / 3
        solid, ghosts = wl.wall_domain(Q, shape, 1, 1)
        prm = _base(Q, shape, periodic=5 if Q == 9 else 3, mu_l=nu, mu_g=nu, sigma=0.0, g=(g, 0, 0))
        o = oracle.Oracle(prm, solid, ghosts)
        _single_phase(o, Q, np.zeros((3, solid.size)), solid)
        o.step(int(8 * H * H / nu))
        u = o.get("u")[0].reshape(shape)
        prof = u[0, :, 0] if Q == 9 else u[:, 0, 0]
        yy = np.arange(H + 2.0)
        exact = g / (2 * nu) * (yy - 0.5) * (H + 0.5 - yy)
        assert np.abs(prof[1:H + 1] - exact[1:H + 1]).max() / exact.max() < tol


@pytest.mark.parametrize("Q", [9, 19])
def test_planar_interface_is_a_steady_state(Q):
    """The tanh profile of width W, Eq. (equilibriumPhaseField), solves Eq.
    (phaseFieldEvolution) at rest: a periodic liquid slab keeps its position and width."""
    shape = (1, 64, 2) if Q == 9 else (64, 2, 2)
    o = oracle.Oracle(_base(Q, shape), np.zeros(shape, np.uint8), EMPTY)
    z, y, _ = wl.node_coords(shape)
    c = (y if Q == 9 else z).reshape(-1).astype(float)
    o.init_phi(0.5 * (np.tanh(2 * (c - 16) / 4) - np.tanh(2 * (c - 48) / 4)))
    o.step(3000)
    prof = o.get("phi").reshape(shape)
    prof = prof[0, :, 0] if Q == 9 else prof[:, 0, 0]
    from scipy.optimize import curve_fit
    cc = np.arange(64.0)
    f = lambda c, a, b, Wf: 0.5 * (np.tanh(2 * (c - a) / Wf) - np.tanh(2 * (c - b) / Wf))
    (a, b, Wf), _ = curve_fit(f, cc, prof, p0=(16, 48, 4))
    assert abs(a - 16) < 1e-3 and abs(b - 48) < 1e-3
    assert abs(Wf / 4.0 - 1) < 0.03
    assert np.abs(o.get("u")).max() < 1e-6


def _two_layer(rho_ratio, W, H):
    """Liquid slab between gas layers in a body-force channel, equal kinematic
    viscosity.  Returns (LBM profile, continuum profile of (mu u')' = -rho g with
    the LBM's own color profile, parabola of (nu u')' = -g)."""
    nu, g = 0.1, 1e-6
    shape = (1, H + 2, 2)
    solid, ghosts = wl.wall_domain(9, shape, 1, 1)
    prm = _base(9, shape, periodic=1, rho_l=rho_ratio, mu_l=rho_ratio * nu, mu_g=nu, W=W, g=(g, 0, 0))
    o = oracle.Oracle(prm, solid, ghosts)
    _, y, _ = wl.node_coords(shape)
    yy = y.reshape(-1).astype(float)
    phi0 = 0.5 * (np.tanh(2 * (yy - 0.3 * H) / W) - np.tanh(2 * (yy - 0.75 * H) / W))
    o.init_phi(np.where(solid.reshape(-1) == 0, phi0, 0.0))
    o.step(int(3 * H * H / nu))
    u = o.get("u")[0].reshape(shape)[0, :, 0][1:H + 1]
    phi = o.get("phi").reshape(shape)[0, :, 0][1:H + 1]
    ys = np.arange(1, H + 1.0)

    def rhs(yq, Y):
        ph = np.interp(yq, ys, phi)
        rho = rho_ratio * ph + (1 - ph)
        return np.vstack([Y[1] / (rho * nu), -rho * g])
    yq = np.linspace(0.5, H + 0.5, 2001)
    sol = solve_bvp(rhs, lambda a, b: np.array([a[0], b[0]]), yq, np.zeros((2, yq.size)),
                    tol=1e-10, max_nodes=100000)
    ref = sol.sol(ys)[0]
    par = g / (2 * nu) * (ys - 0.5) * (H + 0.5 - ys)
    return u, ref, par


def test_two_layer_channel_needs_and_gets_the_viscous_correction():
    """Eq. (viscCorrection) turns the lattice's kinematic viscous term into
    (1/rho) div(rho nu (grad u + grad u^T)): the steady profile solves (mu u')' = -rho g,
    not (nu u')' = -g, and the diffuse-interface error falls as W grows."""
    errs = []
    for W, H in ((4.0, 40), (8.0, 80)):
        u, ref, par = _two_layer(10.0, W, H)
        errs.append(np.abs(u - ref).max() / ref.max())
        assert np.abs(u - par).max() / ref.max() > 0.5        # far from the uncorrected parabola
    assert errs[0] < 0.15 and errs[1] < 0.035 and errs[0] / errs[1] > 3.5
    u, ref, _ = _two_layer(2.0, 4.0, 40)
    assert np.abs(u - ref).max() / ref.max() < 0.005


def _free_drop(Q, n, R, steps, **kw):
    shape = (1, n, n) if Q == 9 else (n, n, n)
    o = oracle.Oracle(_base(Q, shape, **kw), np.zeros(shape, np.uint8), EMPTY)
    o.init_droplet((n / 2, n / 2, n / 2 if Q == 19 else 0), R)
    o.step(steps)
    return o.diagnostics()


def test_laplace_law_2d():
    """Delta p_h = sigma / R for a 2D drop at rest (density ratio 1)."""
    d = _free_drop(9, 64, 16, 3000)
    Req = math.sqrt(d["phi_sum"] / math.pi)
    assert abs((d["p_in"] - d["p_out"]) / (0.01 / Req) - 1) < 0.07
    assert d["max_u"] < 5e-5


def test_laplace_law_2d_density_ratio_1000():
    """Same at rho_l/rho_g = 1000, mu_l/mu_g = 100 (rho_g = 1, mu_g = 0.1), where the
    pressure correction of Eq. (pressCorrection) carries the jump; spurious currents
    stay O(1e-7), the paper's order of magnitude."""
    d = _free_drop(9, 64, 16, 9000, rho_l=1000.0, mu_l=10.0, mu_g=0.1)
    Req = math.sqrt(d["phi_sum"] / math.pi)
    assert abs((d["p_in"] - d["p_out"]) / (0.01 / Req) - 1) < 0.04
    assert d["max_u"] < 1e-6


def test_laplace_law_3d():
    """Delta p_h = 2 sigma / R for a sphere (D3Q19 extension)."""
    d = _free_drop(19, 32, 10, 900)
    Req = (3 * d["phi_sum"] / (4 * math.pi)) ** (1 / 3)
    assert abs((d["p_in"] - d["p_out"]) / (0.02 / Req) - 1) < 0.06


@pytest.mark.parametrize("Q", [9, 19])
def test_mass_is_conserved_exactly(Q):
    """Collision and segregation keep each node's sums (sum N* = 1, sum B* = phi);
    halfway bounce-back and streaming permute populations; ghosts are not fluid."""
    if Q == 9:
        cfg = wl.cylinder_config()
        cfg["params"].update(rho_l=1000.0, mu_l=10.0, mu_g=0.1)
        steps = 300
    else:
        cfg = wl.sphere_config(n=24, R=6, R0=5, theta_deg=60)
        steps = 40
    o = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])
    o.init_droplet(cfg["drop_center"], cfg["R0"])
    d0 = o.diagnostics()
    o.step(steps)
    d1 = o.diagnostics()
    assert abs(d1["phi_sum"] - d0["phi_sum"]) < 1e-13 * d0["phi_sum"] * steps
    assert abs(d1["pop_sum"] - d1["n_fluid"]) < 1e-13 * d1["n_fluid"]
    N = o.get("N")
    fluid = cfg["solid"].reshape(-1) == 0
    assert np.isfinite(N).all() and np.abs(N[:, ~fluid]).max() == 0


def test_mirror_symmetry_is_preserved():
    """A drop on a cylinder, symmetric about x = 32, stays symmetric: phi(x) = phi(64 - x),
    u_x antisymmetric, u_y symmetric."""
    cfg = wl.cylinder_config()
    o = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])
    o.init_droplet(cfg["drop_center"], cfg["R0"])
    o.step(200)
    phi = o.get("phi").reshape(64, 64)
    u = o.get("u").reshape(3, 64, 64)
    mirror = (-np.arange(64)) % 64
    assert np.abs(phi - phi[:, mirror]).max() < 1e-11
    assert np.abs(u[0] + u[0][:, mirror]).max() < 1e-13
    assert np.abs(u[1] - u[1][:, mirror]).max() < 1e-13


def _drop_on_circle_apex(A, R, theta):
    """Circular-arc drop of area A on a circle of radius R at contact angle theta:
    d^2 = R^2 + r^2 - 2 R r cos(theta); A = pi r^2 - lens(R, r, d); apex = d + r."""
    def area(r):
        d = math.sqrt(R * R + r * r - 2 * R * r * math.cos(theta))
        lens = (r * r * math.acos((d * d + r * r - R * R) / (2 * d * r))
                + R * R * math.acos((d * d + R * R - r * r) / (2 * d * R))
                - 0.5 * math.sqrt((-d + r + R) * (d + r - R) * (d - r + R) * (d + r + R)))
        return math.pi * r * r - lens - A
    r = brentq(area, 1e-3 * R, 100 * R)
    return math.sqrt(R * R + r * r - 2 * R * r * math.cos(theta)) + r, r


def test_drop_on_cylinder_reaches_the_circular_arc_equilibrium():
    """64x64 box, cylinder R = 12, drop R0 = 10 tangent on top, theta = 60 deg:
    the steady drop is the circular arc of the same area meeting the cylinder at
    theta (Sec. III B).  The staircase cylinder is taken at the radius of its
    solid area, sqrt(N_solid / pi)."""
    cfg = wl.cylinder_config()
    o = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])
    o.init_droplet(cfg["drop_center"], cfg["R0"])
    o.step(16000)
    probe = oracle.make_probe(1, cfg["solid_center"], cfg["R"], (0, 1, 0), 6.0)
    d = o.diagnostics(probe)
    R_eff = math.sqrt(cfg["solid"].sum() / math.pi)
    apex, r = _drop_on_circle_apex(d["phi_sum"], R_eff, math.radians(60))
    assert abs(d["apex"] / apex - 1) < 0.005
    # the phi = 1/2 circle sits inside the equal-area circle by O(W^2 / r)
    assert abs(d["fit_radius"] / r - 1) < 0.03
    assert abs(math.degrees(d["contact_angle"]) - 60) < 3.0
    assert d["max_u"] < 1e-4


@pytest.mark.parametrize("theta_deg,Rc", [(60, 40), (120, 30)])
def test_flat_plate_contact_angle_within_the_papers_bound(theta_deg, Rc):
    """Drop on a flat plate at W = 6: the measured angle, by the circle fit and by
    Eq. (measuredContactAnglePlate) with S the half base width and H the height,
    is within 2 deg of the set angle (Sec. III A reports < 2 deg for W >= 6)."""
    th, W = math.radians(theta_deg), 6.0
    nx = int(2.6 * Rc * max(math.sin(th), 0.6)) + 40
    ny = int(Rc * (1 - math.cos(th))) + 30
    shape = (1, ny, nx)
    solid, ghosts = wl.wall_domain(9, shape, 1, 1)
    o = oracle.Oracle(_base(9, shape, periodic=1, W=W, theta=th), solid, ghosts)
    _, y, x = wl.node_coords(shape)
    yw = 0.5                                   # halfway bounce-back wall
    xc, yc = nx / 2, yw - Rc * math.cos(th)
    phi = wl.tanh_field(Rc - np.sqrt((x - xc) ** 2 + (y - yc) ** 2), W).reshape(-1)
    o.init_phi(phi * (solid.reshape(-1) == 0))
    o.step(3000)
    d = o.diagnostics(oracle.make_probe(2, (xc, yw, 0), 0.0, (0, 1, 0), 1.5 * W))
    assert abs(math.degrees(d["contact_angle"]) - theta_deg) < 2.0
    ph = o.get("phi").reshape(ny, nx)
    col = ph[:, int(round(xc))]
    j = np.nonzero(col[1:] < 0.5)[0][0] + 1
    Hh = (j - 1) + (col[j - 1] - 0.5) / (col[j - 1] - col[j]) - yw
    row = ph[1]
    inside = np.nonzero(row >= 0.5)[0]
    lo, hi = inside[0], inside[-1]
    S = ((hi + (row[hi] - 0.5) / (row[hi] - row[hi + 1])) - (lo - (row[lo] - 0.5) / (row[lo] - row[lo - 1]))) / 2
    theta_m = math.degrees(math.acos((S * S - Hh * Hh) / (S * S + Hh * Hh)))
    assert abs(theta_m - theta_deg) < 2.0
