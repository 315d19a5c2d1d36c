"""The library's host-side checks of caller arrays (n_s in [0, 1], finite
adhesion, finite positive densities; csrc/lbm_validate.h) agree with the
same conditions written plainly, on special values (signed zeros, NaN,
infinities, denormals, the largest floats) and on long arrays with bad
values planted; built with g++ the way the library builds its host code
(-O3, no contraction) and once without optimisation."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2206_11524_gb300", "csrc")


@pytest.mark.parametrize("opt", [["-O3", "-ffp-contract=off"], ["-O0"]])
def test_validation_helpers(tmp_path, opt):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "validate_harness")
    subprocess.run([gxx, "-std=c++17", *opt, "-I", CSRC,
                    os.path.join(ROOT, "tests", "validate_harness.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "ok"
