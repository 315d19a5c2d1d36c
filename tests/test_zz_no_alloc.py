"""GPU test of lbm_reduce_fields_noalloc, the entry point for callers that
cannot allocate device memory where they need the observables (a host
framework that lends out only its own buffers, a real-time loop where an
allocation would stall the device).  It must give the observables of the
density fields it is handed -- the FP64 oracle's, and lbm_reduce's for the
same state -- call after call, from the smallest lattice to the largest it
accepts, while allocating nothing itself.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2206_11524_gb300 import build, lbm, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    lbm.load()
    oracle.build()


def _as_dict(o):
    return {"mass": np.array(o.mass[:]), "sat1": o.sat1,
            "p_face": np.array(o.p_face[:]), "nonfinite": o.nonfinite}


def _close(a, b, rtol=1e-12):
    """The reductions sum the same float64 terms in different groupings."""
    assert np.allclose(a["mass"], b["mass"], rtol=rtol, atol=0)
    assert abs(a["sat1"] - b["sat1"]) <= rtol
    for k in range(6):
        if np.isnan(b["p_face"][k]):
            assert np.isnan(a["p_face"][k])
        else:
            assert abs(a["p_face"][k] / b["p_face"][k] - 1) <= rtol


def _call(ra, rb, ns, shape, layers, G, stream=0):
    nz, ny, nx = shape
    d = [torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda() for v in (ra, rb, ns)]
    torch.cuda.synchronize()
    st, out = lbm.lbm_reduce_fields_noalloc(d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(),
                                            nx, ny, nz, layers, G, stream)
    del d
    return st, _as_dict(out)


def _oracle(ra, rb, ns, shape, layers, G):
    """The oracle's observables of the same float32 fields (widened)."""
    nz, ny, nx = shape
    res = {k: (L, 1.0, 1.0) for k, L in enumerate(layers or [0] * 6) if L}
    p = oracle.Params(nx, ny, nz, G=float(np.float32(G)), reservoirs=res)
    w = lambda a: np.asarray(a, np.float32).astype(np.float64)
    return oracle.observables_of_densities(p, w(ns), w(ra), w(rb))


def _fields(shape, seed):
    rng = np.random.default_rng(seed)
    ra = rng.uniform(0.0, 1.0, shape).astype(np.float32)
    rb = (1.02 - ra).astype(np.float32)
    ns = np.where(rng.random(shape) < 0.3, 1.0,
                  np.where(rng.random(shape) < 0.5, 0.0, rng.random(shape))).astype(np.float32)
    return ra, rb, ns


def test_noalloc_observables_match_oracle_and_workspace_reduction_twice():
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
    results = []
    for _ in range(2):
        lat.step(7)
        want = lat.observables()                       # lbm_reduce
        f = lat.fields()
        st, got = _call(f["rho_a"], f["rho_b"], ns, shape, layers, 1.75,
                        lat.stream.cuda_stream)
        assert st == lbm.LBM_OK
        _close(got, want)
        _close(got, _oracle(f["rho_a"], f["rho_b"], ns, shape, layers, 1.75))
        assert got["nonfinite"] == want["nonfinite"] == 0
        results.append(got)
    # the two calls saw different states (7 more steps in between)
    assert not np.array_equal(results[0]["mass"], results[1]["mass"]) or \
        results[0]["sat1"] != results[1]["sat1"]
    lat.close()


@pytest.mark.parametrize("shape", [(1, 1, 12289),      # 3 * 4096 + 1 nodes
                                   (256, 256, 256)])   # the largest accepted
def test_noalloc_many_blocks_match_oracle(shape):
    """Lattices of several thousand-node blocks: one node past a multiple of
    the per-block count, and exactly LBM_NOALLOC_MAX_NODES (every block slot
    and the totals slot of the scratch in use), against the oracle."""
    assert shape[0] * shape[1] * shape[2] <= lbm.LBM_NOALLOC_MAX_NODES
    ra, rb, ns = _fields(shape, sum(shape))
    layers = [0, 0, 0, 0, 2, 3] if shape[0] > 4 else [5, 7, 0, 0, 0, 0]
    st, got = _call(ra, rb, ns, shape, layers, 1.6)
    assert st == lbm.LBM_OK
    _close(got, _oracle(ra, rb, ns, shape, layers, 1.6), rtol=1e-11)


def test_noalloc_uses_the_contexts_float_G():
    """A G that float32 cannot hold (1.7): the pressure is the one lbm_reduce
    gives, which uses the context's float G."""
    shape = (6, 8, 16)
    nz, ny, nx = shape
    ns, gads = synth.random_geometry(shape, 3)
    lat = lbm.Lattice(nx, ny, nz, G=1.7)
    lat.set_geometry(ns, gads)
    lat.set_bc(0, 2, 1.0, 0.05)
    lat.set_bc(1, 2, 0.05, 1.0)
    ra = np.where(np.arange(nx) < nx // 2, 0.98, 0.03) * np.ones(shape)
    lat.init_equilibrium(ra, 1.0 - ra)
    lat.step(3)
    want = lat.observables()
    f = lat.fields()
    st, got = _call(f["rho_a"], f["rho_b"], ns, shape, [2, 2, 0, 0, 0, 0], 1.7,
                    lat.stream.cuda_stream)
    assert st == lbm.LBM_OK
    _close(got, want)
    lat.close()


def test_noalloc_allocates_nothing():
    """Across calls (after a first one, which may load the library's device
    code), neither PyTorch's allocator nor the device's free memory moves."""
    shape = (64, 64, 64)
    ra, rb, ns = _fields(shape, 5)
    d = [torch.from_numpy(v).cuda() for v in (ra, rb, ns)]
    torch.cuda.synchronize()
    args = (d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), 64, 64, 64, None, 1.75, 0)
    assert lbm.lbm_reduce_fields_noalloc(*args)[0] == lbm.LBM_OK
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
    outs = [lbm.lbm_reduce_fields_noalloc(*args) for _ in range(3)]
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
    assert before == after
    assert all(st == lbm.LBM_OK for st, _ in outs)
    assert len({tuple(o.mass[:]) for _, o in outs}) == 1


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
