"""GPU test of lbm_reduce_fields_noalloc, the entry point for callers that
cannot allocate device memory where they need the observables (a host
framework that lends out only its own buffers, a real-time loop where an
allocation would stall the device).  It must give what lbm_reduce gives for
the same state, call after call, while allocating nothing itself.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2206_11524_gb300 import build, lbm, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    lbm.load()


def _close(a, b):
    """Same tolerance as the workspace reduction's own tests: the two
    reductions sum the same float64 terms in a different grouping."""
    assert np.allclose(a["mass"], b["mass"], rtol=1e-12, atol=0)
    assert abs(a["sat1"] - b["sat1"]) <= 1e-12
    for k in range(6):
        if np.isnan(b["p_face"][k]):
            assert np.isnan(a["p_face"][k])
        else:
            assert abs(a["p_face"][k] / b["p_face"][k] - 1) <= 1e-12
    assert a["nonfinite"] == b["nonfinite"]


def _as_dict(o):
    return {"mass": np.array(o.mass[:]), "sat1": o.sat1,
            "p_face": np.array(o.p_face[:]), "nonfinite": o.nonfinite}


def test_noalloc_observables_match_workspace_reduction_twice():
    shape = (12, 20, 24)
    nz, ny, nx = shape
    ns, gads = synth.random_geometry(shape, 81)
    layers = [4, 3, 0, 2, 0, 0]
    lat = lbm.Lattice(nx, ny, nz, tau=(1.0, 0.9), G=1.75, F_ext=(1e-5, 0, 0))
    lat.set_geometry(ns, gads)
    lat.set_bc(0, 4, 1.04, 0.01)
    lat.set_bc(1, 3, 0.01, 0.99)
    lat.set_bc(3, 2, 0.5, 0.5)
    ra = np.where(np.arange(nx) < nx // 2, 0.99, 0.01) * np.ones(shape)
    lat.init_equilibrium(ra, 1.0 - ra)
    stream = lat.stream

    results = []
    for _ in range(2):
        lat.step(7)
        want = lat.observables()                       # lbm_reduce
        f = lat.fields()
        d_ra = torch.from_numpy(f["rho_a"]).cuda()
        d_rb = torch.from_numpy(f["rho_b"]).cuda()
        d_ns = torch.from_numpy(ns.astype(np.float32)).cuda()
        torch.cuda.synchronize()
        st, out = lbm.lbm_reduce_fields_noalloc(
            d_ra.data_ptr(), d_rb.data_ptr(), d_ns.data_ptr(), nx, ny, nz,
            layers, 1.75, stream.cuda_stream)
        assert st == lbm.LBM_OK
        got = _as_dict(out)
        _close(got, want)
        results.append(got)
    # the two calls saw different states (7 more steps in between)
    assert not np.array_equal(results[0]["mass"], results[1]["mass"]) or \
        results[0]["sat1"] != results[1]["sat1"]
    lat.close()


def test_noalloc_rejects_lattices_beyond_its_scratch():
    d = torch.zeros(8, device="cuda")
    p = d.data_ptr()
    st, _ = lbm.lbm_reduce_fields_noalloc(p, p, p, 512, 256, 129, None, 1.75, 0)
    assert st == lbm.LBM_ETOOLARGE
    st, _ = lbm.lbm_reduce_fields_noalloc(p, p, p, 0, 1, 1, None, 1.75, 0)
    assert st == lbm.LBM_EINVAL
    st, _ = lbm.lbm_reduce_fields_noalloc(p, p, p, 2, 2, 2, [3, 0, 0, 0, 0, 0],
                                          1.75, 0)
    assert st == lbm.LBM_EINVAL
