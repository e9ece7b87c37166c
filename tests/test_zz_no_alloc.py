"""lbm_phase_sums_noalloc against NumPy sums of the same arrays.

The allocation-free entry point exists for callers that cannot allocate
device memory at the moment they want the per-phase sums -- for example a
program whose device memory is all handed to its own pool allocator, or a
real-time loop that may not allocate after start-up.  Such a caller passes its
own device buffers in and out, and the library uses only a static scratch
array.  The expected values here are plain NumPy reductions of the host
arrays that are copied to the device, so the check does not lean on any other
part of the library.  This file sorts last so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh
process.
"""
import numpy as np
import pytest

from paper_2605_30878_gb300 import lbm
from paper_2605_30878_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_30878_gb300 import build
    build.build()
    lbm.load()


def _node_classes(solid, lattice):
    cls = np.where(solid.reshape(-1) != 0, 2, 0).astype(np.uint8)
    cls[wl.ghost_mask(solid, lattice).reshape(-1)] = 1
    return cls


def _numpy_sums(cls, phi, u, rho_l, rho_g):
    """The six outputs, from their definitions, over the fluid nodes (class 0)."""
    f = cls == 0
    ph = phi[f]
    u2 = (u[:, f] ** 2).sum(0)
    finite_u2 = u2[np.isfinite(u2)]
    return np.array([f.sum(), ph.sum(), rho_l * ph.sum(), rho_g * (1.0 - ph).sum(),
                     np.sqrt(finite_u2.max()) if finite_u2.size else 0.0,
                     np.count_nonzero(~np.isfinite(ph) | ~np.isfinite(u2))])


def _call(cls_d, phi, u, precision, rho_l, rho_g, out):
    import torch
    dtype = torch.float32 if precision == lbm.FP32 else torch.float64
    phi_d = torch.tensor(phi, dtype=dtype, device="cuda")
    u_d = torch.tensor(u, dtype=dtype, device="cuda")
    n = phi.size
    out.fill_(float("nan"))
    lbm.phase_sums_noalloc(cls_d.data_ptr(), phi_d.data_ptr(), u_d.data_ptr(), precision, 3, n, n, rho_l, rho_g,
                           out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP64])
def test_noalloc_sums_match_numpy_on_two_calls_in_a_row(precision):
    import torch
    cfg = wl.sphere_config(n=40, R=8.0, R0=7.0, theta_deg=60.0, rho_ratio=1000.0)
    P = dict(cfg["params"], precision=precision)
    dom = lbm.Domain(P, cfg["solid"], cfg["ghosts"])
    dom.init_droplet(cfg["drop_center"], cfg["R0"])
    cls = _node_classes(cfg["solid"], 19)
    cls_d = torch.from_numpy(cls).cuda()
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    as_stored = np.float32 if precision == lbm.FP32 else np.float64
    for call in range(2):
        dom.step(17)                                       # a different state for each call
        phi = dom.read("phi").astype(as_stored).astype(np.float64)
        u = dom.read("u").astype(as_stored).astype(np.float64)
        got = _call(cls_d, phi, u, precision, P["rho_l"], P["rho_g"], out)
        want = _numpy_sums(cls, phi, u, P["rho_l"], P["rho_g"])
        assert got[0] == want[0] and got[5] == want[5] == 0, call
        assert want[4] > 0, call                           # the drop moves: a real max to find
        for k in range(1, 5):
            assert abs(got[k] - want[k]) <= 1e-12 * abs(want[k]), (call, k, got[k], want[k])


def test_noalloc_counts_nan_and_inf():
    """One NaN in phi and one Inf in a velocity component, on fluid nodes, are
    both counted; the maximum skips the infinite speed."""
    import torch
    cfg = wl.sphere_config(n=24, R=5.0, R0=4.0, theta_deg=60.0, rho_ratio=1.0)
    cls = _node_classes(cfg["solid"], 19)
    rng = np.random.default_rng(3)
    n = cls.size
    phi = rng.uniform(0.0, 1.0, n)
    u = rng.normal(0.0, 1e-3, (3, n))
    fluid = np.flatnonzero(cls == 0)
    phi[fluid[5]] = np.nan
    u[1, fluid[9]] = np.inf
    cls_d = torch.from_numpy(cls).cuda()
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    for precision in (lbm.FP64, lbm.FP32):
        got = _call(cls_d, phi, u, precision, 2.0, 1.0, out)
        as_stored = np.float32 if precision == lbm.FP32 else np.float64
        want = _numpy_sums(cls, phi, u.astype(as_stored).astype(np.float64), 2.0, 1.0)
        assert got[5] == want[5] == 2, precision
        assert got[0] == want[0]
        assert abs(got[4] - want[4]) <= 1e-12 * want[4], precision


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.phase_sums_noalloc(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), lbm.FP64, 1, 16777217, 16777217,
                               1.0, 1.0, buf.data_ptr())
    assert e.value.status == lbm.LBM_ERR_ARG and "16777216" in str(e.value)
