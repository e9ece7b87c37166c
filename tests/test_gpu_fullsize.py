"""Parity at the bench's full sizes: the D3Q19 192^3 drop on a sphere (density
ratio 1000), the 256^3 sphere packing (density ratio 1, 2.3M ghost nodes)
and two of the paper's Table I grids in D2Q9 (drop on a 1000 x 600 plate and
on a cylinder in 601 x 601, density ratio 1000) and six of the bench's 64
batched cases stepped by the batch, with the same CUDA graphs the bench
times, against the FP64 oracle on sampled nodes.  The oracle takes the GPU's state after a few steps
and computes one step at the sampled nodes only (orc_step_sample); the GPU
advances the same step; the two must agree within the precision's tolerance.
Samples: random fluid nodes, fluid nodes next to the sphere (bounce-back),
interface nodes (0.05 < phi < 0.95) and ghost nodes (their updated color)."""
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

TOL = pu.TOL


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_30878_gb300 import build
    build.build()
    lbm.load()


def _samples(cfg, phi, rng):
    """Random fluid nodes, fluid nodes next to a solid, interface nodes, ghosts."""
    solid = cfg["solid"].reshape(-1)
    fluid = np.flatnonzero(solid == 0)
    # fluid nodes with a solid stencil neighbour: the fluid side of the wall
    wall = wl.ghost_mask((cfg["solid"] == 0).astype(np.uint8), cfg["params"]["lattice"]).reshape(-1) & (solid == 0)
    inter = np.flatnonzero((solid == 0) & (phi > 0.05) & (phi < 0.95))
    pick = lambda a, k: rng.choice(a, min(k, len(a)), replace=False) if len(a) else a  # noqa: E731
    return np.unique(np.concatenate([pick(fluid, 1500), pick(np.flatnonzero(wall), 300), pick(inter, 300),
                                     pick(cfg["ghosts"][0], 200)]))


def _oracle_one_step(cfg, g):
    """The FP64 oracle takes g's state and steps the sampled nodes once:
    (nodes, the oracle's values there, the u and p rounding budgets)."""
    precision = cfg["params"]["precision"]
    state = {f: g.read(f) for f in ("N", "B", "phi", "u", "p")}
    rng = np.random.default_rng(11)
    nodes = _samples(cfg, state["phi"], rng)
    o = oracle.Oracle(dict(cfg["params"], precision=0), cfg["solid"], cfg["ghosts"])
    for f, v in state.items():
        o.set(f, v)
    want = o.step_sample(nodes)
    # rounding budgets of u and p for one step from this state (parity_util)
    E = dict(zip(("u", "p"), pu.budget(cfg["params"], precision, state, cfg["solid"].reshape(-1) == 0, 1)))
    return nodes, want, E


def _compare(cfg, g, nodes, want, E, label, min_ghosts=50):
    """g, stepped once more, against the oracle's step at the sampled nodes."""
    precision = cfg["params"]["precision"]
    solid = cfg["solid"].reshape(-1)[nodes]
    fl = solid == 0
    ghost = np.isin(nodes, cfg["ghosts"][0])
    got = {"N": g.read("N")[:, nodes].T, "B": g.read("B")[:, nodes].T, "u": g.read("u")[:, nodes].T,
           "p": g.read("p")[nodes], "phi": g.read("phi")[nodes]}
    err = {}
    for f in ("N", "B"):
        a, b = got[f][fl], want[f][fl]
        err[f] = np.abs(a - b).max() / np.abs(b).max()
    # u and p on their own scale: max|diff| <= tol max|oracle| + E, reported as
    # the ratio to that bound times tol so that every entry compares with tol
    for f in ("u", "p"):
        a, b = got[f][fl], want[f][fl]
        bound = TOL[precision] * np.abs(b).max() + E[f]
        err[f] = np.abs(a - b).max() / bound * TOL[precision]
        err[f + "/own scale"] = np.abs(a - b).max() / np.abs(b).max()
    # phi after the step at fluid nodes, and the ghost color of the step's opening ghost update
    # (the GPU's phi array holds the ghost values of the step just taken)
    a, b = got["phi"][fl], want["phi"][fl]
    err["phi"] = np.abs(a - b).max() / np.abs(b).max()
    err["phi_ghost"] = np.abs(got["phi"][ghost] - want["phi"][ghost]).max()
    print(label, precision, len(nodes), {k: "%.2e" % v for k, v in err.items()})
    assert all(v <= TOL[precision] for k, v in err.items() if "own" not in k), err
    assert ghost.sum() > min_ghosts and fl.sum() > 1500


def _check_one_step(cfg, precision, g, label, min_ghosts=50):
    """The oracle takes g's state, steps the sampled nodes once; g steps once."""
    nodes, want, E = _oracle_one_step(cfg, g)
    g.step(1)
    _compare(cfg, g, nodes, want, E, label, min_ghosts)


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP64, lbm.FP16])
def test_bench_case_step_on_sampled_nodes(precision):
    cfg = wl.sphere_config(n=192, R=32.0, R0=24.0, theta_deg=60.0, rho_ratio=1000.0, mu_ratio=100.0,
                           precision=precision)
    g = lbm.Domain(cfg["params"], cfg["solid"], cfg["ghosts"])
    g.init_droplet(cfg["drop_center"], cfg["R0"])
    g.step(16)                                   # the 8-step graph, as the bench runs it
    _check_one_step(cfg, precision, g, "192^3 sampled parity")
    g.close()


@pytest.fixture(scope="module")
def packing():
    """The bench's 256^3 packing: spheres of radius U(8, 16), porosity 0.45 in
    x >= 24, seed 1; liquid slab 0 <= x < 16 in the reservoir; theta = 45 deg,
    density and viscosity ratio 1 (the step kernel without density contrast)."""
    n = 256
    c, rad = wl.sphere_packing(n=n)
    solid, ghosts = wl.packing_domain(c, rad, n=n)
    x = np.tile(np.arange(n), n * n)
    d_slab = np.minimum(np.abs(x - 7.5), n - np.abs(x - 7.5))
    phi0 = wl.tanh_field(8.0 - d_slab, 4.0)
    P = dict(lattice=19, nx=n, ny=n, nz=n, periodic=7, rho_l=1.0, rho_g=1.0, mu_l=0.1, mu_g=0.1, sigma=0.01,
             W=4.0, M_phi=0.02, theta=np.radians(45.0))
    return {"params": P, "solid": solid, "ghosts": ghosts, "phi0": phi0}


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16])
def test_packing_step_on_sampled_nodes(packing, precision):
    cfg = dict(packing, params=dict(packing["params"], precision=precision))
    g = lbm.Domain(cfg["params"], cfg["solid"], cfg["ghosts"])
    g.init_phi(cfg["phi0"])
    g.step(16)
    _check_one_step(cfg, precision, g, "256^3 packing sampled parity", min_ghosts=100)
    g.close()


def _table1_case(name):
    """The bench's Table I grids: drop on a plate (walls at y = 0 and ny - 1,
    periodic x, drop area 1e4 at 500 x 300 scaled with the grid) and on a
    cylinder (R = 0.2 L at the centre, all periodic); density ratio 1000,
    viscosity ratio 100, theta = 60 deg."""
    if name == "plate":
        nx, ny = 1000, 600
        solid, ghosts = wl.wall_domain(9, (1, ny, nx), 1, 1)
        r = np.sqrt(1e4 / np.pi) * nx / 500.0
        center, periodic = (nx / 2.0, 1.0 + 0.6 * r, 0.0), 1
    else:
        nx = ny = 601
        R = 0.2 * nx
        solid, ghosts = wl.sphere_domain(9, (1, ny, nx), (nx / 2.0, ny / 2.0, 0.0), R)
        r = 0.5 * R
        center, periodic = (nx / 2.0, ny / 2.0 + R + 0.5 * r, 0.0), 7
    P = dict(lattice=9, nx=nx, ny=ny, nz=1, periodic=periodic, rho_l=1000.0, rho_g=1.0, mu_l=10.0, mu_g=0.1,
             sigma=0.01, W=4.0, M_phi=0.02, theta=np.radians(60.0))
    return {"params": P, "solid": solid, "ghosts": ghosts, "drop_center": center, "R0": r}


@pytest.mark.parametrize("name", ["plate", "cylinder"])
@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP64, lbm.FP16])
def test_table1_grid_step_on_sampled_nodes(name, precision):
    base = _table1_case(name)
    cfg = dict(base, params=dict(base["params"], precision=precision))
    g = lbm.Domain(cfg["params"], cfg["solid"], cfg["ghosts"])
    g.init_droplet(cfg["drop_center"], cfg["R0"])
    g.step(16)
    _check_one_step(cfg, precision, g, "Table I %s sampled parity" % name)
    g.close()


def test_batched_cases_step_on_sampled_nodes():
    """Six of the bench's 64 batched cases (D3Q19 drop on a sphere, n = 64 to
    128, density ratios 1 and 10, ragged rows) advanced together by the batch
    with the 64-wide two-node tiles the tuner picks there, against the FP64
    oracle on sampled nodes of every domain."""
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    cfgs = bench.batch_cases()[:6]
    doms = []
    for c in cfgs:
        d = lbm.Domain(c["params"], c["solid"], c["ghosts"])
        d.init_droplet(c["drop_center"], c["R0"])
        doms.append(d)
    b = lbm.Batch(doms)
    b.set_variant(5)
    b.step(16)
    b.sync()
    ref = [_oracle_one_step(c, d) for c, d in zip(cfgs, doms)]
    b.step(1)
    b.sync()
    for k, (c, d, (nodes, want, E)) in enumerate(zip(cfgs, doms, ref)):
        _compare(c, d, nodes, want, E, "batched case %d (n = %d, ratio %g)" %
                 (k, c["params"]["nx"], c["params"]["rho_l"] / c["params"]["rho_g"]))
    b.close()
