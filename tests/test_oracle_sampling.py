"""The oracle's one-step-at-sampled-nodes entry (used for parity at sizes the
full oracle cannot step) agrees with its full step."""
import numpy as np
import pytest

import oracle
from paper_2605_30878_gb300 import workloads as wl


@pytest.mark.parametrize("Q", [9, 19])
def test_sampled_step_equals_full_step(Q):
    if Q == 9:
        cfg = wl.cylinder_config()
        cfg["params"].update(rho_l=1000.0, mu_l=10.0, mu_g=0.1)
    else:
        cfg = wl.sphere_config(n=20, R=5, R0=4, theta_deg=120)
    o = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])
    o.init_droplet(cfg["drop_center"], cfg["R0"])
    o.step(3)
    nn = cfg["solid"].size
    rng = np.random.default_rng(3)
    nodes = np.concatenate([rng.choice(nn, 60, replace=False), cfg["ghosts"][0][:10]])
    s = o.step_sample(nodes)
    o.step(1)
    N, B, u, p, phi = o.get("N"), o.get("B"), o.get("u"), o.get("p"), o.get("phi")
    fluid = cfg["solid"].reshape(-1)[nodes] == 0
    assert np.array_equal(s["N"][fluid], N[:, nodes[fluid]].T)
    assert np.array_equal(s["B"][fluid], B[:, nodes[fluid]].T)
    assert np.array_equal(s["u"][fluid], u[:, nodes[fluid]].T)
    assert np.array_equal(s["p"][fluid], p[nodes[fluid]])
    ghost = np.isin(nodes, cfg["ghosts"][0])
    assert np.array_equal(s["phi"][fluid | ghost], phi[nodes[fluid | ghost]])


def test_droplet_init_uses_the_nearest_periodic_image():
    cfg = wl.cylinder_config()
    o = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])
    o.init_droplet((32.0, 62.0, 0.0), 6.0)
    phi = o.get("phi").reshape(64, 64)
    # the drop centred at y = 62 continues across y = 63 -> 0
    assert abs(phi[0, 32] - phi[60, 32]) < 1e-15 and abs(phi[1, 32] - phi[59, 32]) < 1e-15
    assert phi[0, 32] > 0.98
