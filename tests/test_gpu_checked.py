"""The bounds-checked build (every population, density, geometry, staging
and shared-ring index tested before use; see lbm_fault_word in
include/lbm.h) runs a spread of workloads -- ragged and degenerate shapes,
three storages, reservoirs and velocity cells, per-component n_s, the
single-pass step, several launch shapes, batched steps and a CUDA graph --
without recording a single out-of-range access, and gives the default
build's results to float32 rounding.  The checked library runs in a child process, since
one process loads one library."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2206_11524_gb300 import build, lbm

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    lbm.load()


def test_checked_build_records_no_fault_and_matches(tmp_path):
    sys.path.insert(0, HERE)
    import _checked_scenarios
    ref = _checked_scenarios.run()
    assert int(ref["checked"]) == 0 and not ref["faults"].any()
    lib = build.build(checked=True)
    out = tmp_path / "checked.npz"
    env = dict(os.environ, HMCSC_LBM_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "_checked_scenarios.py"), str(out)],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    got = np.load(out)
    assert int(got["checked"]) == 1
    assert not got["faults"].any(), got["faults"]
    # the checked code may contract multiply-adds differently, so results
    # agree to float32 rounding rather than bit for bit
    for key in ref:
        if key in ("faults", "checked"):
            continue
        a, b = np.asarray(got[key], np.float64), np.asarray(ref[key], np.float64)
        scale = max(np.abs(b).max(), 1e-30)
        assert np.abs(a - b).max() <= 1e-5 * scale, key
