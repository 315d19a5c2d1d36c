"""The single-pass step (lbm_set_single_pass): every population after
several steps of both AA parities is bit-identical to the two-pass step,
for ragged and degenerate shapes, reservoirs and velocity cells, every
population storage and per-component n_s."""
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


def _pair(shape, storage="f32", planes=4, res=True, per_component=False, seed=0):
    nz, ny, nx = shape
    ns, gads = synth.random_geometry(shape, seed)
    ns2, _ = synth.random_geometry(shape, seed + 7)
    f0 = synth.random_state(shape, seed + 1).astype(np.float32)
    lats = []
    for single in (False, True):
        g = lbm.Lattice(nx, ny, nz, tau=(0.9, 1.2), G=1.6, F_ext=(1e-5, -2e-5, 0),
                        storage=storage, rho0=(0.5, 0.5), ns_per_component=per_component)
        g.set_geometry(ns, gads, ns2=ns2 if per_component else None)
        if res:
            g.set_bc(0, min(2, nx), 1.0, 0.03)
            g.set_bc(3, 1, 0.2, 0.7, u=(0.01, 0.0, -0.005))
        g.set_populations(f0)
        if single:
            g.set_single_pass(planes)
        lats.append(g)
    return lats


SHAPES = [(5, 4, 7), (3, 9, 33), (17, 20, 64), (2, 1, 40), (1, 12, 256), (9, 8, 32),
          (6, 17, 100)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("planes", [1, 3, 8])
def test_single_pass_equals_two_pass_f32(shape, planes):
    a, b = _pair(shape, planes=planes, seed=sum(shape))
    for n in (1, 1, 3):
        a.step(n)
        b.step(n)
        assert np.array_equal(a.populations(), b.populations()), (shape, planes, a.t)
    fa, fb = a.fields(), b.fields()
    for key in ("rho_a", "rho_b", "u", "p"):
        assert np.array_equal(fa[key], fb[key]), key
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["f16", "bf16", "f16l", "bf16l"])
def test_single_pass_equals_two_pass_16bit(storage):
    a, b = _pair((6, 17, 100), storage=storage, planes=5, seed=3)
    for n in (1, 2, 3):
        a.step(n)
        b.step(n)
        assert np.array_equal(a.populations(), b.populations()), (storage, a.t)
    a.close()
    b.close()


def test_single_pass_per_component():
    a, b = _pair((7, 12, 48), planes=4, per_component=True, seed=11)
    a.step(4)
    b.step(4)
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()


def test_single_pass_mixed_with_halves():
    """Single-pass steps, two-pass halves and observables interleave."""
    a, b = _pair((4, 10, 40), planes=3, seed=5)
    a.step(3)
    b.step(1)
    lbm.lbm_density(b.ctx)
    lbm.lbm_collide_stream(b.ctx)
    b.step(1)
    assert np.array_equal(a.populations(), b.populations())
    assert a.observables()["mass"].tolist() == b.observables()["mass"].tolist()
    a.close()
    b.close()


def test_single_pass_rejects_wide_lattices():
    g = lbm.Lattice(300, 2, 2)
    with pytest.raises(lbm.LbmError):
        g.set_single_pass(4)
    with pytest.raises(lbm.LbmError):
        g.set_single_pass(-1)
    g.close()
