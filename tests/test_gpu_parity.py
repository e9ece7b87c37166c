"""GPU path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Populations N, B and phi: relative L-infinity error over fluid nodes,
max|gpu - oracle| / max|oracle|, at most 1e-12 (FP64), 1e-4 (FP32) or 2e-3
(FP16 population storage).  u and p on their own scale: at most that bound
times max|oracle| plus the rounding budget of the sums that produce them
(tests/parity_util.py states and derives it)."""
import math
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2605_30878_gb300 import lbm
from paper_2605_30878_gb300 import workloads as wl

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import parity_util as pu  # noqa: E402

pytestmark = pytest.mark.gpu

# FP16 storage keeps 11 significant bits of the stored deviations; a B
# deviation reaches chi_0/2 ~ 0.46, so one stored value carries up to 2.2e-4 of
# rounding (2.4e-4 relative to max B) and phi sums 19 of them: 2e-3 leaves room
# for a few steps of accumulation.
TOL = pu.TOL
rel = pu.rel


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_30878_gb300 import build
    build.build()
    lbm.load()


def pair(cfg, precision):
    P = dict(cfg["params"], precision=precision)
    g = lbm.Domain(P, cfg["solid"], cfg["ghosts"])
    o = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])
    return g, o


def compare(g, o, cfg, precision, steps, label=""):
    """Every field of the GPU state against the oracle's (see parity_util)."""
    fluid = cfg["solid"].reshape(-1) == 0
    return pu.check(pu.read_gpu(g), pu.read_oracle(o), cfg["params"], precision, fluid, steps, label)


def small_3d(theta=60.0, rho_ratio=1000.0, shape=(28, 36, 40), R=7.0, R0=6.0):
    nz, ny, nx = shape
    center = (nx / 2.0 - 0.3, ny / 2.0 + 0.2, nz / 2.0 - 0.1)
    solid, ghosts = wl.sphere_domain(19, shape, center, R)
    params = dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=7, rho_l=rho_ratio, rho_g=1.0,
                  mu_l=0.1 * (100.0 if rho_ratio > 1 else 1.0), mu_g=0.1, sigma=0.005, W=4.0, M_phi=0.02,
                  theta=math.radians(theta), g=(0, 0, 0))
    drop = wl.droplet_on_sphere_center(center, R, R0, math.radians(theta))
    return dict(params=params, solid=solid, ghosts=ghosts, drop_center=tuple(drop), R0=R0)


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32, lbm.FP16])
def test_state_roundtrip(precision):
    cfg = small_3d()
    g = lbm.Domain(dict(cfg["params"], precision=precision), cfg["solid"], cfg["ghosts"])
    fluid = cfg["solid"].reshape(-1) == 0
    o = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])
    o.init_droplet(cfg["drop_center"], cfg["R0"])
    chi = o.get("N")[:, np.nonzero(fluid)[0][0]]
    N, B, u, p = wl.random_state(19, fluid.size, fluid, seed=1, base=chi)     # near the rest state
    phi = np.where(fluid, np.random.default_rng(2).uniform(0, 1, fluid.size), 0.0)
    for f, v in (("N", N), ("B", B), ("u", u), ("p", p), ("phi", phi)):
        g.write(f, v)
        r = g.read(f)
        tol = {lbm.FP64: 0.0, lbm.FP32: 1e-7, lbm.FP16: 5e-4}[precision]
        if precision == lbm.FP16 and f in ("u", "p", "phi"):
            tol = 1e-7                      # fields stay FP32 in this mode
        assert rel(r, v, fluid) <= tol, f


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32, lbm.FP16])
def test_initial_state_matches(precision):
    cfg = wl.cylinder_config()
    g, o = pair(cfg, precision)
    g.init_droplet(cfg["drop_center"], cfg["R0"])
    o.init_droplet(cfg["drop_center"], cfg["R0"])
    compare(g, o, cfg, precision, 0, "initial state")
    # the ghost table is the same reading of Fig. 2 on both sides
    gc, gw, gn = g.ghost_table()
    oc, ow, on = o.ghost_table()
    assert np.array_equal(gn, on)
    for k in range(len(gn)):
        m = gn[k]
        assert np.array_equal(gc[k, :m], oc[k, :m])
        assert np.abs(gw[k, :m] - ow[k, :m]).max() < 1e-15
    assert g.ghost_fallbacks() == o.ghost_fallbacks()


@pytest.mark.parametrize("Q", [9, 19])
@pytest.mark.parametrize("rho_ratio", [1.0, 1000.0])
@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32, lbm.FP16])
def test_one_step_from_a_random_state(Q, rho_ratio, precision):
    """One step from identical seeded non-equilibrium states (every term active)."""
    if Q == 9:
        cfg = wl.cylinder_config(nx=48, ny=40, R=9.0, R0=7.0)
        cfg["params"].update(rho_l=rho_ratio, mu_l=0.1 * (100 if rho_ratio > 1 else 1), mu_g=0.1,
                             g=(1e-6, -2e-6, 0))
    else:
        cfg = small_3d(rho_ratio=rho_ratio)
        cfg["params"]["g"] = (1e-6, 0, -2e-6)
    g, o = pair(cfg, precision)
    fluid = cfg["solid"].reshape(-1) == 0
    o.init_droplet(cfg["drop_center"], cfg["R0"])
    chi = o.get("N")[:, np.nonzero(fluid)[0][0]]
    N, B, u, p = wl.random_state(Q, fluid.size, fluid, seed=7, base=chi)
    phi0 = o.get("phi")
    B = N * np.where(fluid, phi0, 0.0)[None, :] + 1e-4 * (B - N * 0.5)
    phi = np.where(fluid, B.sum(0), phi0)
    for obj in (g, o):
        setter = obj.write if obj is g else obj.set
        setter("N", N); setter("B", B); setter("u", u); setter("p", p); setter("phi", phi)
    g.step(1)
    o.step(1)
    compare(g, o, cfg, precision, 1, "random state, Q=%d ratio=%g" % (Q, rho_ratio))


def _resync_one_step(g, cfg, precision):
    """Give the oracle the GPU's current state, advance both one step, compare:
    the step map itself, from identical inputs, at the full tolerance."""
    o = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])
    for f in ("N", "B", "phi", "u", "p"):
        o.set(f, g.read(f))
    g.step(1)
    o.step(1)
    compare(g, o, cfg, precision, 1, "resync at step %d" % g.diagnostics()["step"])


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32])
def test_cylinder_64_parity_over_2000_steps(precision):
    """D2Q9 64x64, cylinder R = 12, drop R0 = 10 tangent on top, theta = 60 deg,
    density ratio 1, tau = 1, GPU vs oracle over 2000 steps.

    The spreading of the tangent drop amplifies rounding: on the oracle alone a
    2e-16 perturbation of the initial populations grows ~500x by step 100.  So at
    each checkpoint (1, 10, 100, 2000 steps) (a) the trajectories may differ by no
    more than 1e-12 or 100x the growth of such a 1-ulp perturbation on the oracle
    itself, and (b) the step map, restarted from the GPU's state on both sides,
    agrees to the full tolerance."""
    cfg = wl.cylinder_config()
    g, o = pair(cfg, precision)
    g.init_droplet(cfg["drop_center"], cfg["R0"])
    o.init_droplet(cfg["drop_center"], cfg["R0"])
    ref = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])       # 1-ulp perturbed oracle
    ref.init_droplet(cfg["drop_center"], cfg["R0"])
    rng = np.random.default_rng(21)
    for f in ("N", "B"):
        v = ref.get(f)
        ref.set(f, v * (1.0 + 2e-16 * rng.uniform(-1, 1, v.shape)))
    fluid = cfg["solid"].reshape(-1) == 0
    tol = TOL[precision]
    done = 0
    for target in (1, 10, 100, 2000):
        g.step(target - done)
        o.step(target - done)
        ref.step(target - done)
        done = target
        for f in ("N", "B", "phi"):
            sens = rel(ref.get(f), o.get(f), fluid)
            gap = rel(g.read(f), o.get(f), fluid)
            assert gap <= max(tol, 100.0 * sens), (target, f, gap, sens)
        if target == 2000:
            probe_o = oracle.make_probe(1, cfg["solid_center"], cfg["R"], (0, 1, 0), 6.0)
            probe_g = lbm.make_probe(1, cfg["solid_center"], cfg["R"], (0, 1, 0), 6.0)
            dg, do = g.diagnostics(probe_g), o.diagnostics(probe_o)
            dtol = 1e-10 if precision == lbm.FP64 else 1e-4
            for k in ("phi_sum", "pop_sum", "mass_liquid", "mass_gas", "fit_radius", "apex", "p_in", "p_out"):
                assert abs(dg[k] - do[k]) <= dtol * max(1.0, abs(do[k])), k
            assert abs(dg["max_u"] - do["max_u"]) <= dtol * 10 * do["max_u"] + 1e-15
            assert dg["n_fluid"] == do["n_fluid"] and dg["n_iface"] == do["n_iface"]
            assert abs(math.degrees(dg["contact_angle"] - do["contact_angle"])) < (1e-6 if precision == lbm.FP64
                                                                                      else 0.5)
        _resync_one_step(g, cfg, precision)
        o.step(1)
        ref.step(1)
        done += 1


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32, lbm.FP16])
def test_sphere_3d_parity_ragged_tiles(precision):
    """D3Q19 40x36x28 (ragged against the 32x4x2 tiles), sphere R = 7, drop on its
    pole at theta = 60 deg, density ratio 1000, viscosity ratio 100."""
    cfg = small_3d()
    g, o = pair(cfg, precision)
    g.init_droplet(cfg["drop_center"], cfg["R0"])
    o.init_droplet(cfg["drop_center"], cfg["R0"])
    done = 0
    for target in (1, 10, 40):
        g.step(target - done)
        o.step(target - done)
        done = target
        compare(g, o, cfg, precision, target, "sphere 40x36x28 step %d" % target)
    _resync_one_step(g, cfg, precision)                # the step map from the evolved state


@pytest.mark.parametrize("shape,Q", [((1, 3, 5), 9), ((3, 2, 5), 19), ((1, 1, 1), 9), ((2, 2, 2), 19)])
def test_tiny_and_solid_free_domains(shape, Q):
    nz, ny, nx = shape
    solid = np.zeros(shape, np.uint8)
    params = dict(lattice=Q, nx=nx, ny=ny, nz=nz, periodic=7, rho_l=10.0, rho_g=1.0, mu_l=1.0, mu_g=0.1,
                  sigma=0.01, W=4.0, M_phi=0.02, theta=math.radians(45), g=(1e-5, 0, 0))
    empty = (np.zeros(0, np.int64), np.zeros((0, 3)))
    cfg = dict(params=params, solid=solid, ghosts=empty)
    g, o = pair(cfg, lbm.FP64)
    rng = np.random.default_rng(5)
    phi = rng.uniform(0, 1, nx * ny * nz)
    g.init_phi(phi)
    o.init_phi(phi)
    g.step(3)
    o.step(3)
    compare(g, o, cfg, lbm.FP64, 3, "tiny %s" % (shape,))
    assert g.launches_per_step() == 2


@pytest.mark.parametrize("precision,want", [(lbm.FP32, 344.0), (lbm.FP16, 200.0), (lbm.FP64, 688.0)])
def test_algorithmic_bytes_per_fluid_node(precision, want):
    """Whole-step bytes per fluid node, D3Q19 with a density contrast.  Float
    arithmetic: k_step pulls the 18 moving N (the rest population enters no
    moment of the deviation form), N* and B* are written and B* pulled by k_phi
    (3 x 19 values, the rest plane float), phi written and read, u read and
    written, p written, the mask read twice.  FP32: 72 + 228 + 8 + 24 + 4 + 8.
    FP16 storage: 36 + 3 x 40 + 8 + 24 + 4 + 8.  FP64 reads the rest
    population too: 152 + 456 + 16 + 48 + 8 + 8."""
    cfg = small_3d()
    g = lbm.Domain(dict(cfg["params"], precision=precision), cfg["solid"], cfg["ghosts"])
    assert g.bytes_per_fluid_node() == want


def test_neutral_angle_and_flat_wall_fp64():
    """theta = 90 deg (eps = 0, phi_G = phi_F) on flat walls in a non-periodic channel."""
    shape = (1, 24, 40)
    solid, ghosts = wl.wall_domain(9, shape, 1, 1)
    params = dict(lattice=9, nx=40, ny=24, nz=1, periodic=1, rho_l=1.0, rho_g=1.0, mu_l=1 / 6, mu_g=1 / 6,
                  sigma=0.01, W=4.0, M_phi=0.02, theta=math.pi / 2, g=(0, 0, 0))
    cfg = dict(params=params, solid=solid, ghosts=ghosts)
    g, o = pair(cfg, lbm.FP64)
    g.init_droplet((20, 1, 0), 9)
    o.init_droplet((20, 1, 0), 9)
    g.step(50)
    o.step(50)
    compare(g, o, cfg, lbm.FP64, 50, "flat walls, 90 deg")


def test_mass_conservation_and_determinism_fp64():
    cfg = small_3d(rho_ratio=10.0)
    P = dict(cfg["params"], precision=lbm.FP64)
    runs = []
    for _ in range(2):
        g = lbm.Domain(P, cfg["solid"], cfg["ghosts"])
        g.init_droplet(cfg["drop_center"], cfg["R0"])
        d0 = g.diagnostics()
        g.step(300)
        d1 = g.diagnostics()
        assert abs(d1["phi_sum"] - d0["phi_sum"]) < 1e-12 * d0["phi_sum"] * 10
        assert abs(d1["pop_sum"] - d1["n_fluid"]) < 1e-12 * d1["n_fluid"]
        runs.append((g.read("N"), g.read("B")))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16])
def test_mass_conservation_float_storage(precision):
    """Color (sum phi) and population (sum N = fluid nodes) totals over 300
    steps.  Streaming permutes stored values and the collision fixes each
    node's totals (sum_i B*_i = phi sum chi, sum_i N*_i = sum chi, the float
    chi summing to exactly 1).  FP16 storage writes the float rest populations
    as those totals less the rounded moving populations; the moving values lie
    on a coarse grid, their float sums are exact, and the color comes back to
    ~5e-9.  FP32 writes all 19 values from their formulas: each node's total
    carries ~2e-9 of float rounding per step that does not average out, 3e-5
    to 4e-5 of the color here (1.1e-4 with chi rounded one by one).  A wrong
    node total would move O(1e-2) or more per step."""
    cfg = small_3d(rho_ratio=10.0)
    g = lbm.Domain(dict(cfg["params"], precision=precision), cfg["solid"], cfg["ghosts"])
    g.init_droplet(cfg["drop_center"], cfg["R0"])
    g.step(1)
    d0 = g.diagnostics()
    g.step(300)
    d1 = g.diagnostics()
    dphi = abs(d1["phi_sum"] / d0["phi_sum"] - 1)
    dpop = abs(d1["pop_sum"] / d1["n_fluid"] - 1)
    print("precision", precision, "phi_sum drift %.2e, pop_sum - fluid %.2e" % (dphi, dpop))
    assert dphi < {lbm.FP32: 1e-4, lbm.FP16: 1e-6}[precision] and dpop < 1e-6


def test_instability_is_reported_not_faulted():
    """A blow-up (sigma far beyond stability) surfaces as LBM_ERR_UNSTABLE at the
    next synchronising call; the context stays usable."""
    cfg = wl.cylinder_config()
    P = dict(cfg["params"], precision=lbm.FP32, sigma=50.0)
    g = lbm.Domain(P, cfg["solid"], cfg["ghosts"])
    g.init_droplet(cfg["drop_center"], cfg["R0"])
    g.step(400)
    with pytest.raises(lbm.LbmError) as e:
        g.sync()
    assert e.value.status == lbm.LBM_ERR_UNSTABLE
    g.init_droplet(cfg["drop_center"], cfg["R0"])     # re-initialising clears the flag
    g.sync()


def test_step_arguments():
    cfg = wl.cylinder_config()
    g = lbm.Domain(dict(cfg["params"], precision=lbm.FP32), cfg["solid"], cfg["ghosts"])
    g.init_droplet(cfg["drop_center"], cfg["R0"])
    g.step(0)
    with pytest.raises(lbm.LbmError) as e:
        g.step(-1)
    assert e.value.status == lbm.LBM_ERR_ARG
    a = lbm.Domain(dict(cfg["params"], precision=lbm.FP64), cfg["solid"], cfg["ghosts"], workspace="library")
    b = lbm.Domain(dict(cfg["params"], precision=lbm.FP64), cfg["solid"], cfg["ghosts"], workspace="torch")
    for d in (a, b):
        d.init_droplet(cfg["drop_center"], cfg["R0"])
        d.step(13)       # odd count: exercises both single-step graphs and the 8-step graph
    assert np.array_equal(a.read("B"), b.read("B"))


@pytest.mark.parametrize("theta_deg", [30.0, 90.0])
def test_fakhari_rule_parity_fp64(theta_deg):
    """The comparison scheme, Eq. (ghostNodeFakhari), selected by ghost_rule = 1
    (theta = 90 deg exercises eps ~ -6e-17, where it must reduce to phi_G = phi_F)."""
    cfg = wl.cylinder_config(theta_deg=theta_deg)
    cfg["params"].update(ghost_rule=1, rho_l=10.0, mu_l=1.0, mu_g=0.1)
    g, o = pair(cfg, lbm.FP64)
    g.init_droplet(cfg["drop_center"], cfg["R0"])
    o.init_droplet(cfg["drop_center"], cfg["R0"])
    g.step(300)
    o.step(300)
    compare(g, o, cfg, lbm.FP64, 300, "Fakhari rule %g deg" % theta_deg)
    if theta_deg == 90.0:
        cor, wt, nc = o.ghost_table()
        phi = g.read("phi")
        g.step(1)                        # the step opens with the ghost update
        ghost_nodes = cfg["ghosts"][0]
        phiF = np.array([np.dot(wt[k, :nc[k]], phi[cor[k, :nc[k]]]) for k in range(len(ghost_nodes))])
        assert np.abs(g.read("phi")[ghost_nodes] - phiF).max() < 1e-14


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16])
@pytest.mark.parametrize("Q", [9, 19])
def test_two_node_kernel_equals_one_node_kernel(precision, Q, monkeypatch):
    """The two-node step kernel (each thread updates x-adjacent nodes, two-wide
    loads and stores) and the one-node kernel round alike: the same state to
    the bit after 11 steps, on grids whose odd x extent leaves the last pair
    half outside the grid, with tiled and element-copied halos."""
    if Q == 19:
        cfg = wl.sphere_config(n=70, R=14.0, R0=10.0, theta_deg=50.0, rho_ratio=1000.0, precision=precision)
        shape = (67, 70, 69)                       # nz, ny, nx: odd nx
        center = (34.3, 35.2, 33.6)
        solid, ghosts = wl.sphere_domain(19, shape, center, 14.0)
        cfg.update(solid=solid, ghosts=ghosts, drop_center=tuple(wl.droplet_on_sphere_center(
            center, 14.0, 10.0, math.radians(50.0))))
        cfg["params"].update(nx=69, ny=70, nz=67)
    else:
        cfg = wl.cylinder_config(nx=161, ny=130, R=20.0, R0=16.0, theta_deg=110.0)
        cfg["params"].update(precision=precision, rho_l=1000.0, rho_g=1.0, mu_l=10.0, mu_g=0.1)
    states = {}
    for kernel in ("single", "pair"):
        for halo in ("tma", "elements"):
            monkeypatch.setenv("LBM_STEP_KERNEL", kernel)
            if halo == "elements":
                monkeypatch.setenv("LBM_HALO_COPY", "elements")
            else:
                monkeypatch.delenv("LBM_HALO_COPY", raising=False)
            d = lbm.Domain(dict(cfg["params"], precision=precision), cfg["solid"], cfg["ghosts"])
            monkeypatch.delenv("LBM_STEP_KERNEL")
            monkeypatch.delenv("LBM_HALO_COPY", raising=False)
            d.init_droplet(cfg["drop_center"], cfg["R0"])
            d.step(11)
            d.sync()
            states[(kernel, halo)] = {f: d.read(f) for f in ("N", "B", "phi", "u", "p")}
    ref = states[("single", "tma")]
    for key, st in states.items():
        for f in ref:
            assert np.array_equal(st[f], ref[f]), (key, f)
