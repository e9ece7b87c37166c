"""Workspaces the library allocates come from a memory pool per device that
keeps a destroyed domain's workspace for the next domain; lbm_release_cached_memory
gives it back to the device."""
import numpy as np
import pytest

from paper_2605_30878_gb300 import lbm
from paper_2605_30878_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SLACK = 64 << 20          # bytes: pool granularity and other allocations of the process


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_30878_gb300 import build
    build.build()
    lbm.load()


def _run(cfg, steps=5):
    d = lbm.Domain(cfg["params"], cfg["solid"], cfg["ghosts"], workspace="library")
    d.init_droplet(cfg["drop_center"], cfg["R0"])
    d.step(steps)
    state = {f: d.read(f) for f in ("N", "B", "phi", "u", "p")}
    d.close()
    return state


def test_pooled_workspace_is_kept_reused_and_released():
    import torch
    cfg = wl.sphere_config(n=96, R=20.0, R0=14.0, theta_deg=70.0, rho_ratio=1000.0, precision=lbm.FP32)
    need = lbm.domain_bytes(cfg["params"], len(cfg["ghosts"][0]))
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    lbm.release_cached_memory()
    free0 = torch.cuda.mem_get_info()[0]
    first = _run(cfg)
    torch.cuda.empty_cache()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 >= need - SLACK                 # the workspace stayed in the pool
    # the next domain takes the cached workspace, stale contents and all, and
    # steps to the same state
    second = _run(cfg)
    torch.cuda.empty_cache()
    free2 = torch.cuda.mem_get_info()[0]
    assert abs(free2 - free1) <= SLACK
    for f in first:
        assert np.array_equal(first[f], second[f]), f
    lbm.release_cached_memory()
    free3 = torch.cuda.mem_get_info()[0]
    assert free3 >= free0 - SLACK
