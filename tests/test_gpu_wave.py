"""The wavefront step (lbm_set_wavefront): every population after several
steps of both AA parities is bit-identical to the two-pass step, for every
tile shape and several
lags, ragged and degenerate shapes, reservoirs and velocity cells, every
population storage and per-component n_s; no wait runs out; repeated
launches (the ticket and epoch carried from launch to launch) and graph
replays stay identical; at the 256^3 electrode in the bench's launch
configuration it matches the two-pass step bit for bit.  (The oracle
comparison of the wavefront step itself is in test_gpu_parity.py.)"""
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


def _pair(shape, storage="f32", wave=(1, 0), res=True, per_component=False, seed=0,
          stream=None):
    nz, ny, nx = shape
    ns, gads = synth.random_geometry(shape, seed)
    ns2, _ = synth.random_geometry(shape, seed + 7)
    f0 = synth.random_state(shape, seed + 1).astype(np.float32)
    lats = []
    for use_wave in (False, True):
        g = lbm.Lattice(nx, ny, nz, tau=(0.9, 1.2), G=1.6, F_ext=(1e-5, -2e-5, 0),
                        storage=storage, rho0=(0.5, 0.5), ns_per_component=per_component,
                        stream=stream)
        g.set_geometry(ns, gads, ns2=ns2 if per_component else None)
        if res:
            g.set_bc(0, min(2, nx), 1.0, 0.03)
            g.set_bc(3, 1, 0.2, 0.7, u=(0.01, 0.0, -0.005))
            g.set_bc(5, 1, 0.6, 0.1)
        g.set_populations(f0)
        if use_wave:
            g.set_wavefront(*wave)
        lats.append(g)
    return lats


def _fault(g):
    return lbm.lbm_fault_word(g.ctx)


SHAPES = [(5, 4, 7), (3, 9, 33), (17, 20, 64), (2, 1, 40), (1, 12, 256), (9, 8, 32),
          (6, 17, 100), (4, 3, 1)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("wave", [(1, 0), (2, 3), (3, 7), (2, 5)])
def test_wave_equals_two_pass_f32(shape, wave):
    a, b = _pair(shape, wave=wave, seed=sum(shape))
    for n in (1, 1, 3):
        a.step(n)
        b.step(n)
        assert np.array_equal(a.populations(), b.populations()), (shape, wave, a.t)
    assert _fault(b) == 0
    fa, fb = a.fields(), b.fields()
    for key in ("rho_a", "rho_b", "u", "p"):
        assert np.array_equal(fa[key], fb[key]), key
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["f16", "bf16", "f16l", "bf16l"])
@pytest.mark.parametrize("wave", [(1, 0), (2, 0), (3, 5)])
def test_wave_equals_two_pass_16bit(storage, wave):
    a, b = _pair((6, 17, 100), storage=storage, wave=wave, seed=3)
    for n in (1, 2, 3):
        a.step(n)
        b.step(n)
        assert np.array_equal(a.populations(), b.populations()), (storage, a.t)
    assert _fault(b) == 0
    a.close()
    b.close()


@pytest.mark.parametrize("wave", [(1, 0), (2, 0)])
def test_wave_per_component(wave):
    a, b = _pair((7, 12, 48), wave=wave, per_component=True, seed=11)
    a.step(4)
    b.step(4)
    assert np.array_equal(a.populations(), b.populations())
    assert _fault(b) == 0
    a.close()
    b.close()


def test_wave_many_launches_and_switching():
    """Thirty launches of a lattice with many items per SM (tickets and
    epochs carried over), then back to two passes and on again."""
    a, b = _pair((40, 96, 128), wave=(1, 0), seed=5)
    a.step(30)
    b.step(30)
    assert np.array_equal(a.populations(), b.populations())
    b.set_wavefront(0)
    a.step(3)
    b.step(3)
    b.set_wavefront(2, 6)
    a.step(5)
    b.step(5)
    assert np.array_equal(a.populations(), b.populations())
    assert _fault(b) == 0
    a.close()
    b.close()


@pytest.mark.parametrize("wave", [(1, 0), (2, 0)])
def test_wave_graph_replay(wave):
    """Two wavefront steps captured in a CUDA graph and replayed three times
    equal six two-pass steps."""
    s = torch.cuda.Stream()
    a, b = _pair((12, 40, 96), wave=wave, seed=9, stream=s)
    b.step(1)          # warm-up outside the capture (attributes, occupancy)
    a.step(1)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        b.step(2)
    for _ in range(3):
        graph.replay()
    a.step(6)
    torch.cuda.synchronize()
    assert np.array_equal(a.populations(), b.populations())
    assert _fault(b) == 0
    a.close()
    b.close()


def test_wave_rejects_bad_arguments():
    g = lbm.Lattice(8, 4, 4)
    for shape, lag in ((4, 0), (-1, 0), (1, 2), (1, -3), (1, 2**31 - 1)):
        with pytest.raises(lbm.LbmError):
            g.set_wavefront(shape, lag)
    g.set_wavefront(0)
    g.close()


def test_wave_full_size_electrode_matches_two_pass():
    """The 256^3 electrode of the benchmark: the wavefront step (shapes 1
    and 2) at the default lag against the two-pass step with the bench's
    default shapes: two steps (both parities), every population bit for
    bit."""
    shape = (256, 256, 256)
    case = synth.electrode(shape)
    lats = []
    for use_wave in (0, 1, 2):
        g = lbm.Lattice(256, 256, 256, tau=case.tau, G=case.G, F_ext=case.F_ext,
                        rho0=(0.5, 0.5))
        g.set_geometry(case.ns, case.gads2)
        for face, (L, r1, r2) in case.reservoirs.items():
            g.set_bc(face, L, r1, r2)
        g.init_equilibrium(case.rho_a, case.rho_b)
        if use_wave:
            g.set_wavefront(use_wave)
        lats.append(g)
    for g in lats:
        g.step(2)
    pa = lats[0].populations()
    for g in lats[1:]:
        assert np.array_equal(pa, g.populations())
        assert _fault(g) == 0
    for g in lats:
        g.close()
