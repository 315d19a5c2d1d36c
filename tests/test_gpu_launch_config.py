"""Launch shapes change speed, never results; the autotuner picks one and
keeps it in its table."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2206_11524_gb300 import autotune, build, lbm, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    lbm.load()


def _run(storage, cfg, shape=(9, 13, 70), steps=5):
    nz, ny, nx = shape
    ns, gads = synth.random_geometry(shape, 55)
    g = lbm.Lattice(nx, ny, nz, tau=(0.9, 1.2), G=1.75, F_ext=(1e-5, 2e-5, 0),
                    storage=storage, rho0=(0.5, 0.5))
    g.set_geometry(ns, gads)
    g.set_bc(0, 3, 1.04, 0.01)
    g.set_bc(5, 2, 0.01, 0.99)
    ra = np.where(np.arange(nx) < nx // 2, 0.99, 0.03) * np.ones(shape)
    g.init_equilibrium(ra, 1.02 - ra)
    g.set_launch_config(*cfg)
    g.step(steps)
    f = g.populations()
    g.close()
    return f


@pytest.mark.parametrize("storage", ["f32", "f16l"])
def test_every_launch_shape_gives_identical_results(storage):
    ref = _run(storage, (0, 0, 0))
    cfgs = [(d, 0, 0) for d in range(1, lbm.LBM_DENSITY_CONFIGS)]
    cfgs += [(0, e, 0) for e in range(1, lbm.LBM_COLLIDE_CONFIGS)]
    cfgs += [(0, 0, o) for o in range(1, lbm.LBM_COLLIDE_CONFIGS)]
    for cfg in cfgs:
        assert np.array_equal(_run(storage, cfg), ref), cfg


def test_autotune_records_and_applies(tmp_path):
    table = autotune.TuneTable(str(tmp_path / "t.json"))
    g = lbm.Lattice(64, 48, 40)
    g.set_geometry(np.zeros((40, 48, 64)))
    g.init_equilibrium(np.ones((40, 48, 64)), np.ones((40, 48, 64)))
    cfg = g.autotune(table)
    assert len(cfg) == 6 and cfg[3] == 0          # no single-pass unless asked
    assert g.wavefront()[0] == cfg[4]
    assert cfg[4] == 0 or (cfg[4], cfg[5]) in autotune.WAVE_CANDIDATES
    again = autotune.TuneTable(str(tmp_path / "t.json"))
    assert again.get(64, 48, 40, "f32") == tuple(cfg)
    with pytest.raises(lbm.LbmError):
        g.set_launch_config(0, lbm.LBM_COLLIDE_CONFIGS, 0)
    g.step(2)
    g.close()


def test_autotune_weighs_the_single_pass(tmp_path):
    """With single_pass the table entry's fourth value is a box depth or 0
    (the fifth and sixth the wavefront shape and lag), and applying it gives
    the same populations as the defaults."""
    table = autotune.TuneTable(str(tmp_path / "t.json"))
    shape = (40, 48, 64)
    ns, gads = synth.random_geometry(shape, 3)
    f0 = synth.random_state(shape, 4)
    out = []
    for tuned in (False, True):
        g = lbm.Lattice(64, 48, 40, tau=(0.9, 1.1), G=1.5)
        g.set_geometry(ns, gads)
        g.set_populations(f0)
        if tuned:
            cfg = g.autotune(table, single_pass=True)
            assert len(cfg) == 6 and cfg[3] >= 0
            assert not (cfg[3] > 0 and cfg[4] > 0)   # one step kind at most
        g.step(3)
        out.append(g.populations())
        g.close()
    assert np.array_equal(out[0], out[1])
