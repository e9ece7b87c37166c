"""The seeded input generators.  They hold none of the method's arithmetic, but
the parity and physics tests and the bench take their geometry from them, so
the properties their docstrings state are checked here: the sphere packing of
the porous-imbibition workload is seeded, its spheres do not overlap beyond
the stated tolerance, stay out of the inlet reservoir and fill the requested
solid fraction; the ghost lists it and the other domains produce satisfy the
contract the oracle and the C ABI validate (every solid node with a fluid
neighbour listed once, unit normals)."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_30878_gb300 import workloads as wl

N, RES = 64, 10
ARGS = dict(n=N, r_min=4.0, r_max=7.0, porosity=0.45, reservoir=RES, seed=4)


@pytest.fixture(scope="module")
def packing():
    return wl.sphere_packing(**ARGS)


def test_sphere_packing_is_seeded(packing):
    c, r = packing
    c2, r2 = wl.sphere_packing(**ARGS)
    assert np.array_equal(c, c2) and np.array_equal(r, r2)
    c3, _ = wl.sphere_packing(**dict(ARGS, seed=5))
    assert not np.array_equal(c, c3)


def test_sphere_packing_does_not_overlap_and_keeps_the_reservoir_free(packing):
    c, r = packing
    assert r.min() >= 4.0 and r.max() <= 7.0
    d = c[:, None, :] - c[None, :, :]
    d[..., 1:] -= N * np.round(d[..., 1:] / N)            # periodic in y and z, not in x
    dist = np.linalg.norm(d, axis=2)
    overlap = r[:, None] + r[None, :] - dist
    np.fill_diagonal(overlap, -np.inf)
    assert overlap.max() <= 0.02 + 1e-9
    assert (c[:, 0] - r >= RES - 1e-9).all() and (c[:, 0] + r <= N + 1e-9).all()


def test_packing_domain_fills_the_solid_fraction(packing):
    """The sphere count is the target solid fraction of the region over the
    mean sphere volume of U(r_min, r_max); the staircase mask holds the drawn
    spheres' volume (lattice points inside a sphere average its volume); the
    region's fraction then differs from the target only by the draw of the
    radii (+6.8% of sphere volume for this seed, a 2-sigma draw of 162)."""
    c, r = packing
    lo, hi = ARGS["r_min"], ARGS["r_max"]
    span = N - RES
    mean_vol = 4.0 / 3.0 * math.pi * (hi ** 4 - lo ** 4) / (4.0 * (hi - lo))
    assert len(r) == round(span * N * N * (1 - ARGS["porosity"]) / mean_vol)
    solid, (nodes, normals) = wl.packing_domain(c, r, n=N)
    assert solid[:, :, :RES].sum() == 0                   # (z, y, x): the reservoir columns are free
    assert abs(solid.sum() / (4.0 / 3.0 * math.pi * (r ** 3).sum()) - 1) < 0.01
    frac = solid[:, :, RES:].mean()
    print("solid fraction of the packing region %.3f (target %.2f)" % (frac, 1 - ARGS["porosity"]))
    assert abs(frac - (1 - ARGS["porosity"])) < 0.05


def test_packing_ghost_list_meets_the_contract(packing):
    c, r = packing
    solid, ghosts = wl.packing_domain(c, r, n=N)
    nodes, normals = ghosts
    g = wl.ghost_mask(solid, 19).reshape(-1)
    assert np.array_equal(nodes, np.flatnonzero(g))       # every boundary solid node, once, in order
    assert np.allclose(np.linalg.norm(normals, axis=1), 1.0, atol=1e-12)
    # the oracle validates the same contract as lbm_create_domain and refuses a bad list
    params = dict(lattice=19, nx=N, ny=N, nz=N, periodic=7, rho_l=1.0, rho_g=1.0, mu_l=0.1, mu_g=0.1,
                  sigma=0.01, W=4.0, M_phi=0.02, theta=math.radians(60.0), g=(0, 0, 0))
    o = oracle.Oracle(params, solid, ghosts)
    assert o.ghost_fallbacks() >= 0


@pytest.mark.parametrize("lattice,shape", [(9, (1, 48, 64)), (19, (32, 32, 40))])
def test_multi_sphere_normals_are_radial_from_the_nearest_surface(lattice, shape):
    """Each ghost's normal is the outward radial direction of the sphere whose
    surface is nearest; for ghosts touching only one sphere that is the
    direction from its centre."""
    nz, ny, nx = shape
    if lattice == 9:
        centers, radii = [(16.0, 24.0, 0.0), (46.0, 20.0, 0.0)], [9.0, 7.0]
    else:
        centers, radii = [(12.0, 16.0, 16.0), (30.0, 15.0, 14.0)], [7.0, 6.0]
    solid, (nodes, normals) = wl.multi_sphere_domain(lattice, shape, centers, radii)
    x = nodes % nx
    y = (nodes // nx) % ny
    z = nodes // (nx * ny)
    pts = np.stack([x, y, z], axis=1).astype(float)
    for c, R in zip(centers, radii):
        d = pts - np.asarray(c)
        if lattice == 9:
            d[:, 2] = 0.0
        near = np.abs(np.linalg.norm(d, axis=1) - R) < 2.0
        assert near.any()
        radial = d[near] / np.linalg.norm(d[near], axis=1)[:, None]
        assert np.allclose(normals[near], radial, atol=1e-12)
