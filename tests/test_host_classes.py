"""Host-side node classification of lbm_create_domain (no GPU needed).

The library classifies nodes with row bit masks: 64 nodes per word, the
stencil as shifted and ORed neighbour rows.  A ghost is a solid node with a
fluid node among its Q - 1 lattice neighbours (periodic wrap on every axis).
Here that classification is pinned to a brute-force NumPy one on random
masks, at row widths that are and are not multiples of 64 (ragged last
words), with grids one node thick along an axis.  The library accepts a
ghost list only if it is exactly the mask's set of ghost nodes: its messages
tell us how many ghosts it found, and that every listed node is a ghost.
Creation stops before any device call because the last normal is made
invalid, so the check needs no GPU."""
import numpy as np
import pytest

from paper_2605_30878_gb300 import build as lbm_build
from paper_2605_30878_gb300 import lbm


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbm_build.build()
    lbm.load()


def stencil(q):
    if q == 9:
        return [(dx, dy, 0) for dx in (-1, 0, 1) for dy in (-1, 0, 1) if (dx, dy) != (0, 0)]
    out = []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                n = abs(dx) + abs(dy) + abs(dz)
                if n in (1, 2):
                    out.append((dx, dy, dz))
    assert len(out) == 18
    return out


def brute_ghosts(solid, q):
    """solid: (nz, ny, nx) bool.  Ghost = solid and some neighbour fluid."""
    fluid = ~solid
    near = np.zeros_like(solid)
    for dx, dy, dz in stencil(q):
        # neighbour at x + c: roll by -c brings it to x
        near |= np.roll(fluid, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
    return solid & near


def params(q, nx, ny, nz):
    return dict(lattice=q, nx=nx, ny=ny, nz=nz, periodic=7 if q == 19 else 3, precision=lbm.FP32,
                rho_l=1.0, rho_g=1.0, mu_l=0.1, mu_g=0.1, sigma=0.01, W=4.0, M_phi=0.02, theta=1.0)


CASES = [
    (9, 63, 17, 1), (9, 64, 9, 1), (9, 65, 5, 1), (9, 130, 3, 1), (9, 7, 1, 1),
    (19, 63, 5, 4), (19, 64, 3, 3), (19, 65, 4, 2), (19, 129, 2, 1), (19, 8, 1, 5), (19, 1, 6, 6),
]


@pytest.mark.parametrize("q,nx,ny,nz", CASES)
def test_ghost_classes_match_brute_force(q, nx, ny, nz):
    rng = np.random.default_rng(nx * 1000 + ny * 10 + nz)
    for frac in (0.3, 0.7):
        solid = rng.random((nz, ny, nx)) < frac
        ghosts = brute_ghosts(solid, q)
        nodes = np.flatnonzero(ghosts.reshape(-1))
        if len(nodes) < 2:
            continue
        normals = np.zeros((len(nodes), 3))
        normals[:, 0] = 1.0
        P = params(q, nx, ny, nz)
        s8 = solid.astype(np.uint8)
        # the full list, last normal invalid: every listed node was accepted as a
        # ghost and the counts agreed, so the error is the normal's
        bad = normals.copy()
        bad[-1] = (2.0, 0.0, 0.0)
        with pytest.raises(lbm.LbmError) as e:
            lbm.Domain(P, s8, (nodes, bad), workspace="library", stream=0)
        assert "ghost %d normal is not a unit vector" % (len(nodes) - 1) in str(e.value), str(e.value)
        # one ghost left out: the library reports the mask's own count
        with pytest.raises(lbm.LbmError) as e:
            lbm.Domain(P, s8, (nodes[1:], normals[1:]), workspace="library", stream=0)
        assert "mask has %d ghost nodes" % len(nodes) in str(e.value), str(e.value)
        # a solid node without a fluid neighbour, or a fluid node, is refused
        others = np.flatnonzero((~ghosts).reshape(-1))
        if len(others):
            wrong = nodes.copy()
            wrong[0] = others[0]
            with pytest.raises(lbm.LbmError) as e:
                lbm.Domain(P, s8, (wrong, normals), workspace="library", stream=0)
            assert "is not a solid node with a fluid neighbour" in str(e.value), str(e.value)
        # a node listed twice
        dup = nodes.copy()
        dup[1] = dup[0]
        with pytest.raises(lbm.LbmError) as e:
            lbm.Domain(P, s8, (dup, normals), workspace="library", stream=0)
        assert "listed twice" in str(e.value), str(e.value)
