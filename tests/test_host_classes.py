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
    (19, 130, 130, 130), (9, 2000, 1500, 1),      # large enough to be split over the host thread pool
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


def _validation_error(q=19, nx=130, ny=130, nz=130, seed=0):
    rng = np.random.default_rng(seed)
    solid = rng.random((nz, ny, nx)) < 0.5
    nodes = np.flatnonzero(brute_ghosts(solid, q).reshape(-1))
    normals = np.zeros((len(nodes), 3))
    normals[:, 0] = 1.0
    normals[-1] = (2.0, 0.0, 0.0)
    try:
        lbm.Domain(params(q, nx, ny, nz), solid.astype(np.uint8), (nodes, normals), workspace="library", stream=0)
    except lbm.LbmError as e:
        return str(e), len(nodes)
    return "no error", len(nodes)


def test_concurrent_creations_share_the_host_pool():
    """Creation's host work runs on a shared thread pool (these 2.2M-node
    grids are split over it); calls from several host threads at once are
    serialised on it and each gets its own answer."""
    import threading
    out = {}

    def worker(k):
        out[k] = [_validation_error(seed=k)[0] for _ in range(10)]

    th = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=60)
    assert len(out) == 4
    for k in range(4):
        msg, n = _validation_error(seed=k)
        assert all(m == msg for m in out[k]) and ("ghost %d normal" % (n - 1)) in msg


def _child(q):
    q.put(_validation_error()[0])


@pytest.mark.filterwarnings("ignore::DeprecationWarning")
def test_forked_child_gets_its_own_pool():
    """A child forked after the pool started has none of its threads; its
    creation calls still finish (on a pool of its own)."""
    import multiprocessing as mp
    _validation_error()                        # the parent's pool exists
    ctx = mp.get_context("fork")
    q = ctx.Queue()
    p = ctx.Process(target=_child, args=(q,))
    p.start()
    p.join(timeout=60)
    assert p.exitcode == 0
    assert "normal is not a unit vector" in q.get(timeout=5)
