"""Physics of the GPU path on the paper's own benchmarks, at the paper's sizes
(too long for the oracle; the oracle pins the same physics at small sizes in
test_oracle_physics.py), and the error of each storage precision against the
FP64 oracle."""
import math
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2605_30878_gb300 import lbm
from paper_2605_30878_gb300 import workloads as wl

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import analytic  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_30878_gb300 import build
    build.build()
    lbm.load()


def _cylinder_run(theta_deg, rule, steps=80000, precision=lbm.FP32):
    """Drop on a cylinder, Sec. III B: box 5R x 5R with R = 40, cylinder at
    (Lx/2, Ly/4), drop of area A = 3000 started at its equilibrium shape, all
    periodic, rho_l/rho_g = 1000, mu_l/mu_g = 100 (rho_g = 1, mu_g = 0.1),
    sigma = 0.01, W = 4, M_phi = 0.02."""
    R, L = 40.0, 200
    th = math.radians(theta_deg)
    center = (L / 2, L / 4, 0)
    solid, ghosts = wl.sphere_domain(9, (1, L, L), center, R)
    P = dict(lattice=9, nx=L, ny=L, nz=1, periodic=7, precision=precision, ghost_rule=rule, rho_l=1000.0,
             rho_g=1.0, mu_l=10.0, mu_g=0.1, sigma=0.01, W=4.0, M_phi=0.02, theta=th)
    r, d = analytic.drop_on_circle(3000.0, R, th)
    _, y, x = wl.node_coords((1, L, L))
    phi = wl.tanh_field(r - np.sqrt((x - center[0]) ** 2 + (y - center[1] - d) ** 2), 4.0).reshape(-1)
    dom = lbm.Domain(P, solid, ghosts)
    dom.init_phi(phi)
    dom.step(steps)
    dg = dom.diagnostics(lbm.make_probe(1, center, R, (0, 1, 0), 6.0))
    r1, d1 = analytic.drop_on_circle(dg["phi_sum"], R, th)
    return (dg["apex"] - (d1 + r1)) / R, dg


def test_drop_on_cylinder_apex_height():
    """h_max/R against the circular-arc solution for theta = 30..150 deg: the
    paper reports errors of -0.35% (30 deg) and +0.26% (150 deg) for its scheme and
    -0.76% / +0.70% for Fakhari et al.'s; both rules coincide at 90 deg."""
    errs = {}
    for theta in (30, 60, 90, 120, 150):
        for rule in (lbm.GHOST_PRESENT, lbm.GHOST_FAKHARI):
            errs[(theta, rule)], dg = _cylinder_run(theta, rule)
            assert dg["nan_flag"] == 0 and dg["max_u"] < 1e-4
    print("h_max/R error:", {k: round(100 * v, 3) for k, v in errs.items()})
    for theta in (30, 60, 90, 120, 150):
        assert abs(errs[(theta, lbm.GHOST_PRESENT)]) < 0.005
    assert errs[(90, lbm.GHOST_PRESENT)] == errs[(90, lbm.GHOST_FAKHARI)]
    assert abs(errs[(150, lbm.GHOST_PRESENT)]) < abs(errs[(150, lbm.GHOST_FAKHARI)])


def _plate_run(theta_deg, precision, steps):
    """Drop on a flat plate, Sec. III A: 500 x 300, periodic in x, walls in y,
    drop area A = 1e4 started as the circular cap, density ratio 1000."""
    nx, ny = 500, 300
    th = math.radians(theta_deg)
    shape = (1, ny, nx)
    solid, ghosts = wl.wall_domain(9, shape, 1, 1)
    P = dict(lattice=9, nx=nx, ny=ny, nz=1, periodic=1, precision=precision, rho_l=1000.0, rho_g=1.0,
             mu_l=10.0, mu_g=0.1, sigma=0.01, W=4.0, M_phi=0.02, theta=th)
    Rc, yc = analytic.cap_on_plane(1e4, th)
    _, y, x = wl.node_coords(shape)
    phi = wl.tanh_field(Rc - np.sqrt((x - nx / 2) ** 2 + (y - 0.5 - yc) ** 2), 4.0).reshape(-1)
    dom = lbm.Domain(P, solid, ghosts)
    dom.init_phi(phi)
    dom.step(steps)
    return dom.diagnostics(lbm.make_probe(2, (nx / 2, 0.5, 0), 0.0, (0, 1, 0), 6.0))


@pytest.mark.parametrize("theta_deg,bound", [(30, 1.5e-6), (150, 5e-6)])
def test_drop_on_plate_spurious_currents(theta_deg, bound):
    """The paper reports max |u| = 5.74e-7 (30 deg) and 7e-7 (150 deg) at rest and
    O(1e-6) as typical (Sec. IV).  Here (FP32 and FP64 agree): 6.7e-7 at 30 deg;
    2.2-2.9e-6 at 150 deg, in the gas next to the contact line.  The measured angle
    stays at the set angle on a flat wall."""
    dg = _plate_run(theta_deg, lbm.FP32, 60000)
    print("plate", theta_deg, "max|u| %.3e" % dg["max_u"], "theta %.4f" % math.degrees(dg["contact_angle"]))
    assert dg["max_u"] < bound
    assert abs(math.degrees(dg["contact_angle"]) - theta_deg) < 0.5


# ---------------------------------------------------------------- precision vs FP64 oracle

@pytest.fixture(scope="module")
def cylinder_oracle():
    """The FP64 oracle on the 64x64 drop-on-cylinder case, 16000 steps."""
    cfg = wl.cylinder_config()
    o = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])
    o.init_droplet(cfg["drop_center"], cfg["R0"])
    o.step(16000)
    return cfg, o.diagnostics(oracle.make_probe(1, cfg["solid_center"], cfg["R"], (0, 1, 0), 6.0))


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32, lbm.FP16])
def test_contact_angle_per_storage_precision(cylinder_oracle, precision):
    """Contact angle of the equilibrated drop on the cylinder against the FP64
    oracle after 16000 steps of spreading, measured: FP64 1.2e-12 deg, FP32
    0.020 deg, FP16 storage 3.0e-3 deg (FP16 keeps 11 significant bits of the
    stored deviations; the float rest populations take the node totals less
    the rounded moving ones).  Bound: 0.5 deg."""
    cfg, do = cylinder_oracle
    g = lbm.Domain(dict(cfg["params"], precision=precision), cfg["solid"], cfg["ghosts"])
    g.init_droplet(cfg["drop_center"], cfg["R0"])
    g.step(16000)
    dg = g.diagnostics(lbm.make_probe(1, cfg["solid_center"], cfg["R"], (0, 1, 0), 6.0))
    err = abs(math.degrees(dg["contact_angle"] - do["contact_angle"]))
    print("precision", precision, "contact angle error vs FP64 oracle: %.3e deg" % err,
          "apex %.6f vs %.6f" % (dg["apex"], do["apex"]))
    assert err < 0.5


@pytest.fixture(scope="module")
def laplace_oracle():
    """The FP64 oracle on a free 2D drop (64^2, R = 16) at density ratio 1000, 9000 steps."""
    n = 64
    params = dict(lattice=9, nx=n, ny=n, nz=1, periodic=7, rho_l=1000.0, rho_g=1.0, mu_l=10.0, mu_g=0.1,
                  sigma=0.01, W=4.0, M_phi=0.02, theta=math.pi / 2)
    solid = np.zeros((1, n, n), np.uint8)
    empty = (np.zeros(0, np.int64), np.zeros((0, 3)))
    o = oracle.Oracle(params, solid, empty)
    o.init_droplet((n / 2, n / 2, 0), 16.0)
    o.step(9000)
    return params, solid, empty, o.diagnostics()


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32, lbm.FP16])
def test_laplace_pressure_and_spurious_current_per_storage_precision(laplace_oracle, precision):
    """Laplace pressure jump and spurious current of a free drop at density ratio
    1000 against the FP64 oracle (same discretisation, same steps)."""
    params, solid, empty, do = laplace_oracle
    g = lbm.Domain(dict(params, precision=precision), solid, empty)
    g.init_droplet((32, 32, 0), 16.0)
    g.step(9000)
    dg = g.diagnostics()
    dp_o, dp_g = do["p_in"] - do["p_out"], dg["p_in"] - dg["p_out"]
    print("precision", precision, "Laplace dP %.6e vs oracle %.6e (rel %.2e)" % (dp_g, dp_o, abs(dp_g / dp_o - 1)),
          "max|u| %.3e vs %.3e" % (dg["max_u"], do["max_u"]))
    # measured: FP64 2.5e-10, FP32 1.0e-3, FP16 storage 5.0e-4 relative
    bound = {lbm.FP64: 1e-9, lbm.FP32: 5e-3, lbm.FP16: 5e-3}[precision]
    assert abs(dp_g / dp_o - 1) < bound
    # The spurious current against the oracle's (1.83e-7): FP64 to 1e-6
    # relative (the same discretisation, settled to equilibrium); FP32 within 10% (measured 5%: float rounding of the color,
    # amplified by the Laplacian in the surface tension, perturbs the force at
    # the interface each step); FP16 storage within 10% plus its noise floor.
    # That floor: each stored moving B value rounds by up to 2^-12 of
    # max|B - chi/2| = chi_1/2 (at phi = 0 or 1), so the color a node gathers
    # from its Q - 1 moving neighbours carries up to (Q - 1) 2^-12 chi_1/2;
    # the Laplacian gains it 12 (1 - w_0), the surface tension carries it as
    # sigma 3W/2 |grad phi| (|grad phi| <= 1/W) into the force, and u takes
    # F / (2 rho_g): 6.5e-7 here.
    tab = oracle.lattice_tables(9, params["M_phi"])
    w0, chi1 = tab["w"][0], tab["chi"][1]
    floor16 = (params["sigma"] * 1.5 * params["W"] * 12 * (1 - w0) * 8 * 2.0 ** -12 * chi1 / 2
               * (1 / params["W"]) / (2 * params["rho_g"]))
    rel_u, floor_u = {lbm.FP64: (1e-6, 0.0), lbm.FP32: (0.1, 0.0), lbm.FP16: (0.1, floor16)}[precision]
    assert abs(dg["max_u"] - do["max_u"]) <= rel_u * do["max_u"] + floor_u, (dg["max_u"], do["max_u"], floor_u)
    assert dg["max_u"] < 1e-6
