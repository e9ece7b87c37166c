"""The bounds-checked build of the library (liblbm_debug.so: the same sources
compiled with LBM_DEBUG_BOUNDS).  Its kernels test every index they compute
against the array it addresses before the access; a bad index sets an error
bit (reported as LBM_ERR_BOUNDS) and the access is skipped, so nothing traps.

The parity suite runs against it in a child process (LBM_LIBRARY=debug); any
bit set would fail those tests at their next synchronising call.  A planted
ghost-corner index past the end of the color array shows that the checks are
live: the debug build reports it, the production build refuses to plant it."""
import os
import subprocess
import sys

import pytest

from paper_2605_30878_gb300 import lbm
from paper_2605_30878_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_30878_gb300 import build
    build.build()
    lbm.load()


def _child(args, timeout):
    env = dict(os.environ, LBM_LIBRARY="debug")
    return subprocess.run(args, env=env, cwd=ROOT, capture_output=True, text=True, timeout=timeout)


def test_parity_suite_passes_with_every_index_checked():
    r = _child([sys.executable, "-m", "pytest", "tests/test_gpu_parity.py", "tests/test_gpu_batch.py",
                "tests/test_gpu_failure.py", "-m", "gpu", "-q", "-x", "-p", "no:cacheprovider"], 1800)
    tail = r.stdout[-4000:] + r.stderr[-2000:]
    print(tail[-600:])
    assert r.returncode == 0 and " passed" in r.stdout, tail


PLANT = """
import sys
sys.path.insert(0, ".")
from paper_2605_30878_gb300 import lbm, workloads as wl
assert lbm.LIB_PATH.endswith("liblbm_debug.so") and lbm.bounds_checked()
cfg = wl.cylinder_config()
d = lbm.Domain(dict(cfg["params"], precision=lbm.FP32), cfg["solid"], cfg["ghosts"])
d.init_droplet(cfg["drop_center"], cfg["R0"])
d.step(20)
d.sync()
print("clean")
d.debug_plant_bad_index(0)
d.step(1)
try:
    d.sync()
    print("not caught")
except lbm.LbmError as e:
    print("caught", e.status)
"""


def test_checked_build_catches_a_planted_index():
    r = _child([sys.executable, "-c", PLANT], 600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "clean" in r.stdout and ("caught %d" % lbm.LBM_ERR_BOUNDS) in r.stdout, r.stdout + r.stderr


def test_production_build_refuses_to_plant():
    assert not lbm.bounds_checked()
    cfg = wl.cylinder_config()
    d = lbm.Domain(dict(cfg["params"], precision=lbm.FP32), cfg["solid"], cfg["ghosts"])
    d.init_droplet(cfg["drop_center"], cfg["R0"])
    with pytest.raises(lbm.LbmError) as e:
        d.debug_plant_bad_index(0)
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
    d.step(5)
    d.sync()
