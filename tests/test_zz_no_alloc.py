"""lbm_phase_sums_noalloc against lbm_diagnostics.

The allocation-free entry point exists for callers that cannot allocate
device memory at the moment they want the per-phase sums -- for example a
program whose device memory is all handed to its own pool allocator, or a
real-time loop that may not allocate after start-up.  Such a caller passes its
own device buffers in and out, and the library uses only a static scratch
array.  This file sorts last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
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


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP64])
def test_noalloc_sums_match_diagnostics_on_two_calls_in_a_row(precision):
    import torch
    cfg = wl.sphere_config(n=40, R=8.0, R0=7.0, theta_deg=60.0, rho_ratio=1000.0)
    P = dict(cfg["params"], precision=precision)
    dom = lbm.Domain(P, cfg["solid"], cfg["ghosts"])
    dom.init_droplet(cfg["drop_center"], cfg["R0"])
    n = cfg["solid"].size
    dtype = torch.float32 if precision == lbm.FP32 else torch.float64
    cls = torch.from_numpy(_node_classes(cfg["solid"], 19)).cuda()
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        dom.step(17)                       # a different state for each call
        want = dom.diagnostics()
        phi = torch.tensor(dom.read("phi"), dtype=dtype, device="cuda")
        u = torch.tensor(dom.read("u"), dtype=dtype, device="cuda")
        out.fill_(float("nan"))
        lbm.phase_sums_noalloc(cls.data_ptr(), phi.data_ptr(), u.data_ptr(), precision, 3, n, n,
                               P["rho_l"], P["rho_g"], out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[0] == want["n_fluid"], call
        for k, name in ((1, "phi_sum"), (2, "mass_liquid"), (3, "mass_gas"), (4, "max_u")):
            assert abs(got[k] - want[name]) <= 1e-12 * abs(want[name]), (call, name)
        assert got[5] == 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.phase_sums_noalloc(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), lbm.FP64, 1, 16777217, 16777217,
                               1.0, 1.0, buf.data_ptr())
    assert e.value.status == lbm.LBM_ERR_ARG and "16777216" in str(e.value)
