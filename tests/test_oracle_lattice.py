"""Pins for the oracle's lattice constants, equilibrium, macroscopic fields
and collision (Appendix A of the paper), checked against the tables the paper
prints and against identities the mathematics fixes -- never against the
oracle itself."""
import itertools

import numpy as np
import pytest

import oracle
from conftest import read_golden

MPHI = 0.02


def _floats(rows):
    return np.array([[float(v) for v in r] for r in rows])


def test_d2q9_tables_match_appendix_a():
    g = read_golden("d2q9_appendix_a.txt")
    t = oracle.lattice_tables(9, MPHI)
    assert np.array_equal(t["c"][:, :2].T, _floats(g["c"]).astype(int))
    assert np.allclose(t["w"], _floats(g["w"])[0], rtol=0, atol=1e-16)
    alpha = 1.0 - 10.0 * MPHI / 3.0          # M_phi = (cs2/2)*9(1-alpha)/5 at p = 0
    chi = _floats(g["chi_alpha"])[0] * alpha + _floats(g["chi_one_minus_alpha"])[0] * (1 - alpha)
    assert np.allclose(t["chi"], chi, rtol=0, atol=1e-16)
    assert np.array_equal(t["M"], _floats(g["M"]))
    rows = [int(v) for v in g["S_one_over_tau_rows"][0]]
    assert list(np.nonzero(t["is_stress"])[0]) == rows


@pytest.mark.parametrize("Q", [9, 19])
def test_lattice_isotropy(Q):
    t = oracle.lattice_tables(Q, MPHI)
    c, w = t["c"].astype(float), t["w"]
    D = 2 if Q == 9 else 3
    cs2 = 1.0 / 3.0
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c)[:D, :D], cs2 * np.eye(D), atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-16)
    d = np.eye(D)
    iso4 = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                       + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)[:D, :D, :D, :D], iso4, atol=1e-15)
    # opposite directions
    assert np.array_equal(c[t["opp"]], -c)
    # velocity set: rest + nearest + (2D: diagonals | 3D: edge diagonals), each once
    norms = sorted((c ** 2).sum(1).astype(int).tolist())
    assert norms == ([0] + [1] * 4 + [2] * 4 if Q == 9 else [0] + [1] * 6 + [2] * 12)
    assert len({tuple(v) for v in t["c"]}) == Q


@pytest.mark.parametrize("Q", [9, 19])
def test_color_weights_and_mobility(Q):
    """sum chi = 1, chi isotropic; its second moment reproduces M_phi = (cs2/2)[...]
    of Appendix A at p = 0 (for D3Q19 via chi_i = (1-alpha) w_i/(1-w_0))."""
    t = oracle.lattice_tables(Q, MPHI)
    c, chi, w = t["c"].astype(float), t["chi"], t["w"]
    D = 2 if Q == 9 else 3
    assert abs(chi.sum() - 1) < 1e-15
    m2 = np.einsum("i,ia,ib->ab", chi, c, c)[:D, :D]
    assert np.allclose(m2, m2[0, 0] * np.eye(D), atol=1e-16)
    assert abs(0.5 * m2[0, 0] - MPHI) < 1e-15          # M_phi = (1/2) sum chi c_x^2 at p = 0
    assert np.allclose(chi[1:], (1 - chi[0]) * w[1:] / (1 - w[0]), atol=1e-16)


@pytest.mark.parametrize("Q", [9, 19])
def test_transform_matrix_orthogonal_and_invertible(Q):
    t = oracle.lattice_tables(Q, MPHI)
    M, Minv = t["M"], t["Minv"]
    G = M @ M.T
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-12
    assert np.abs(M @ Minv - np.eye(Q)).max() < 1e-13
    assert np.allclose(M[0], 1)                          # density row


def test_d3q19_stress_rows_span_traceless_second_moments():
    t = oracle.lattice_tables(19, MPHI)
    c = t["c"].astype(float)
    x, y, z = c.T
    c2 = x * x + y * y + z * z
    target = np.stack([3 * x * x - c2, y * y - z * z, x * y, y * z, x * z])
    S = t["M"][t["is_stress"]]
    P = S.T @ np.linalg.solve(S @ S.T, S)               # projector on the stress rows
    assert np.abs(P @ target.T - target.T).max() < 1e-12
    assert np.linalg.matrix_rank(S) == 5
    # the remaining rows are orthogonal to the stress subspace
    others = t["M"][~t["is_stress"]]
    assert np.abs(others @ target.T).max() < 1e-12


def test_gram_schmidt_in_2d_gives_the_papers_projector():
    tp = oracle.lattice_tables(9, MPHI)
    tg = oracle.lattice_tables(9, MPHI, gram_schmidt=True)

    def proj(t):
        S = t["M"][t["is_stress"]]
        return S.T @ np.linalg.solve(S @ S.T, S)
    assert np.abs(proj(tp) - proj(tg)).max() < 1e-14


@pytest.mark.parametrize("Q", [9, 19])
def test_equilibrium_moments(Q):
    t = oracle.lattice_tables(Q, MPHI)
    c = t["c"].astype(float)
    D = 2 if Q == 9 else 3
    rng = np.random.default_rng(5)
    m2chi = np.einsum("i,i->", t["chi"], c[:, 0] ** 2)
    for _ in range(20):
        u = np.zeros(3)
        u[:D] = rng.uniform(-0.1, 0.1, D)
        p = rng.uniform(-0.05, 0.05)
        neq = oracle.equilibrium(Q, u, p, MPHI)
        assert abs(neq.sum() - 1) < 1e-14
        assert np.allclose(neq @ c, u, atol=1e-15)
        # momentum flux: (sum chi c_x^2 + p) I + u u
        Pi = np.einsum("i,ia,ib->ab", neq, c, c)[:D, :D]
        assert np.allclose(Pi, (m2chi + p) * np.eye(D) + np.outer(u[:D], u[:D]), atol=1e-15)


@pytest.mark.parametrize("Q", [9, 19])
def test_pressure_update_inverts_equilibrium(Q):
    """Eq. (pressureUpdate) applied to Eq. (equilibriumDistribution) returns p,
    and Eq. (velUpdate) returns u + F/(2 rho)."""
    rng = np.random.default_rng(6)
    D = 2 if Q == 9 else 3
    for _ in range(20):
        u = np.zeros(3)
        u[:D] = rng.uniform(-0.1, 0.1, D)
        p = rng.uniform(-0.05, 0.05)
        neq = oracle.equilibrium(Q, u, p, MPHI)
        F = np.zeros(3)
        rho = rng.uniform(1, 1000)
        u2, p2 = oracle.macro(Q, neq, F, rho, MPHI)
        assert np.allclose(u2, u, atol=1e-15) and abs(p2 - p) < 1e-14
        F[:D] = rng.uniform(-1e-2, 1e-2, D)
        uF, _ = oracle.macro(Q, neq, F, rho, MPHI)
        assert np.allclose(uF, u + F / (2 * rho), atol=1e-15)


def _random_pops(Q, rng):
    t = oracle.lattice_tables(Q, MPHI)
    return t, t["chi"] + 1e-3 * rng.uniform(-1, 1, Q)


@pytest.mark.parametrize("Q", [9, 19])
def test_collision_conserves_and_forces(Q):
    """Rows with s = 1 send the density to sum Neq = 1 and the momentum to
    u + F/(2 rho) (Eq. MRTCOLL with Eq. forceGuo)."""
    rng = np.random.default_rng(7)
    D = 2 if Q == 9 else 3
    for _ in range(20):
        t, N = _random_pops(Q, rng)
        c = t["c"].astype(float)
        F = np.zeros(3)
        F[:D] = rng.uniform(-1e-3, 1e-3, D)
        rho = rng.uniform(1, 10)
        u, p = oracle.macro(Q, N, F, rho, MPHI)
        tau = rng.uniform(0.51, 2.0)
        Ns = oracle.collide(Q, N, u, p, F, rho, tau, MPHI)
        assert abs(Ns.sum() - 1) < 1e-14
        assert np.allclose(Ns @ c, u + F / (2 * rho), atol=1e-15)


@pytest.mark.parametrize("Q", [9, 19])
def test_post_collision_total_is_fixed(Q):
    """sum_i N*_i = sum chi = 1 for any N, u, p and F, not only the u and p of
    N: the equilibrium's zeroth moment is sum chi (its p and u^2 terms in the
    moving directions cancel against the rest population's), the stress
    projection is traceless and the forcing has no zeroth moment.  The
    recoloring term of Eq. (segragationStepBlue) is odd in c_i, chi and w are
    even, so sum_i B*_i = phi sum_i N*_i as well.  FP16 population storage
    writes each node's float rest populations from these two totals."""
    rng = np.random.default_rng(17)
    D = 2 if Q == 9 else 3
    t = oracle.lattice_tables(Q, MPHI)
    c, w, chi, opp = t["c"], t["w"], t["chi"], np.asarray(t["opp"])
    assert abs(chi.sum() - 1) < 1e-15
    assert np.array_equal(chi[opp], chi) and np.array_equal(w[opp], w) and np.array_equal(c[opp], -c)
    for _ in range(50):
        N = chi + rng.normal(0, 0.05, Q)
        u = np.zeros(3)
        u[:D] = rng.normal(0, 0.05, D)
        F = np.zeros(3)
        F[:D] = rng.normal(0, 1e-3, D)
        Ns = oracle.collide(Q, N, u, rng.normal(0, 0.01), F, rng.uniform(0.5, 1000), rng.uniform(0.51, 2), MPHI)
        assert abs(Ns.sum() - 1) < 1e-14


@pytest.mark.parametrize("Q", [9, 19])
def test_segregation_moves_color_up_its_gradient_and_conserves_it(Q):
    """Eq. (segragationStepBlue) writes B*_i = phi N*_i plus a recoloring
    term.  The term carries no color: sum_i B*_i = phi sum_i N*_i, the fact FP16
    storage writes its rest populations from.  Inside the interface it sends
    color along grad phi: B*_i - phi N*_i has the sign of c_i . grad phi.  It
    vanishes in the pure phases (phi = 0, 1) and where grad phi = 0."""
    rng = np.random.default_rng(19)
    D = 2 if Q == 9 else 3
    t = oracle.lattice_tables(Q, MPHI)
    c = t["c"].astype(float)
    for _ in range(50):
        Nst = t["chi"] + rng.normal(0, 0.02, Q)
        phi = rng.uniform(0.05, 0.95)
        g = np.zeros(3)
        g[:D] = rng.normal(0, 0.1, D)
        p = rng.uniform(-5e-3, 5e-3)
        B = oracle.segregate(Q, Nst, phi, g, p)
        assert abs(B.sum() - phi * Nst.sum()) < 1e-14
        rec, cg = B - phi * Nst, c @ g
        assert rec[0] == 0.0
        assert np.array_equal(np.sign(rec[1:]), np.sign(cg[1:]))
    Nst = t["chi"] + rng.normal(0, 0.02, Q)
    g = np.array([0.1, -0.05, 0.02 if D == 3 else 0.0])
    for phi in (0.0, 1.0):
        assert np.array_equal(oracle.segregate(Q, Nst, phi, g, 1e-3), phi * Nst)
    assert np.array_equal(oracle.segregate(Q, Nst, 0.3, np.zeros(3), 1e-3), 0.3 * Nst)


@pytest.mark.parametrize("Q", [9, 19])
def test_collision_at_tau_one_is_bgk(Q):
    """At tau = 1 every rate is 1 and Eq. (MRTCOLL) reduces to N* = Neq + F_i / 2."""
    rng = np.random.default_rng(8)
    D = 2 if Q == 9 else 3
    for _ in range(10):
        t, N = _random_pops(Q, rng)
        c, w = t["c"].astype(float), t["w"]
        F = np.zeros(3)
        F[:D] = rng.uniform(-1e-3, 1e-3, D)
        rho = rng.uniform(1, 10)
        u, p = oracle.macro(Q, N, F, rho, MPHI)
        Ns = oracle.collide(Q, N, u, p, F, rho, 1.0, MPHI)
        Fi = 3.0 * w * (c @ F) / rho
        assert np.allclose(Ns, oracle.equilibrium(Q, u, p, MPHI) + 0.5 * Fi, atol=1e-15)


@pytest.mark.parametrize("Q", [9, 19])
def test_collision_relaxes_only_the_traceless_stress(Q):
    """Off tau = 1, N* - (Neq + F/2) is (1 - 1/tau) times the non-equilibrium part
    projected (orthogonally) onto the traceless second moments; nothing else survives."""
    rng = np.random.default_rng(9)
    D = 2 if Q == 9 else 3
    for _ in range(10):
        t, N = _random_pops(Q, rng)
        c, w = t["c"].astype(float), t["w"]
        x, y, z = c.T
        c2 = x * x + y * y + z * z
        basis = np.stack([x * x - y * y, x * y]) if Q == 9 else \
            np.stack([3 * x * x - c2, y * y - z * z, x * y, y * z, x * z])
        P = basis.T @ np.linalg.solve(basis @ basis.T, basis)
        F = np.zeros(3)
        F[:D] = rng.uniform(-1e-3, 1e-3, D)
        rho, tau = rng.uniform(1, 10), rng.uniform(0.51, 2.0)
        u, p = oracle.macro(Q, N, F, rho, MPHI)
        neq = oracle.equilibrium(Q, u, p, MPHI)
        Fi = 3.0 * w * (c @ F) / rho
        Ns = oracle.collide(Q, N, u, p, F, rho, tau, MPHI)
        assert np.allclose(Ns, neq + 0.5 * Fi + (1 - 1 / tau) * P @ (N - neq), atol=1e-15)
