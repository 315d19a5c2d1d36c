"""Failure detection on the GPU, without faulting it.

  - A wavefront wait that runs out: the wavefront launch is told to leave
    one density flag unpublished (a flag that nothing sets) and to give up a
    wait after a few thousand polls.  The launch ends, the fault word holds
    LBM_FAULT_WAIT, the synchronising calls and lbm_step return EINTERNAL,
    and after the state is reloaded from a checkpoint the run continues
    exactly like an undisturbed one.
  - Non-finite densities (LBM_ENAN): an inlet reservoir set to an absurd
    density drives a small lattice to overflow within a few steps (the
    oracle shows the same in FP64); lbm_reduce reports it, and loading the
    checkpoint taken before the change and restoring the reservoir gives a
    clean continuation, bit for bit the same as a run that never saw it.
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


def _lattice(shape, seed, wave=0):
    nz, ny, nx = shape
    ns, gads = synth.random_geometry(shape, seed)
    g = lbm.Lattice(nx, ny, nz, tau=(1.0, 0.9), G=1.75, F_ext=(1e-5, 0, 0))
    g.set_geometry(ns, gads)
    g.set_bc(0, 2, 1.02, 0.02)
    ra = np.where(np.arange(nx) < nx // 2, 0.98, 0.02) * np.ones(shape)
    g.init_equilibrium(ra, 1.0 - ra)
    if wave:
        g.set_wavefront(wave)
    return g


@pytest.mark.parametrize("wave", [2, 1])
def test_wavefront_wait_that_runs_out_is_reported(wave):
    shape = (8, 12, 64)
    nz, ny, nx = shape
    g = _lattice(shape, 3, wave)
    ref = _lattice(shape, 3)                 # two passes, never disturbed
    g.step(3)
    ref.step(3)
    ck = g.save()
    by = {1: 4, 2: 2}[wave]
    ntx, nty = (nx + 31) // 32, (ny + by - 1) // by
    held = 2 * nty * ntx + 2 * ntx + 1        # a tile flag of a middle plane
    lbm.lbm_set_wavefront_limits(g.ctx, 2000, held)
    g.step(1)                                 # enqueued; the launch ends by itself
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_sync(g.ctx, 60.0)
    assert e.value.status == lbm.LBM_EINTERNAL
    with pytest.raises(lbm.LbmError) as e:
        g.step(1)                             # refuses to advance an undefined state
    assert e.value.status == lbm.LBM_EINTERNAL
    with pytest.raises(lbm.LbmError) as e:
        g.observables()
    assert e.value.status == lbm.LBM_EINTERNAL
    assert lbm.lbm_fault_word(g.ctx, clear=False) & lbm.LBM_FAULT_WAIT
    # back to normal limits, reload, and the run goes on as if undisturbed
    lbm.lbm_set_wavefront_limits(g.ctx, 0, -1)
    g.load(ck)
    assert lbm.lbm_fault_word(g.ctx, clear=False) == 0
    g.step(5)
    ref.step(5)
    assert np.array_equal(g.populations(), ref.populations())
    lbm.lbm_sync(g.ctx, 60.0)
    g.close()
    ref.close()


def test_fault_word_clear_lets_stepping_resume():
    """Clearing the fault word (lbm_fault_word with clear) is the other way
    out; the launch after it waits normally again."""
    shape = (4, 6, 40)
    nz, ny, nx = shape
    g = _lattice(shape, 7, 2)
    lbm.lbm_set_wavefront_limits(g.ctx, 500, 2 * ((ny + 1) // 2) + 1)  # plane 1
    g.step(1)
    word = lbm.lbm_fault_word(g.ctx, clear=True)
    assert word & lbm.LBM_FAULT_WAIT
    lbm.lbm_set_wavefront_limits(g.ctx, 0, -1)
    g.step(2)
    lbm.lbm_sync(g.ctx, 60.0)
    assert lbm.lbm_fault_word(g.ctx, clear=False) == 0
    g.close()


@pytest.mark.parametrize("wave", [0, 2])
def test_nonfinite_densities_detected_and_rolled_back(wave):
    shape = (6, 8, 16)
    g = _lattice(shape, 5, wave)
    ref = _lattice(shape, 5, wave)
    g.step(4)
    ref.step(4)
    ck = g.save()
    g.set_bc(0, 2, 1e6, 0.01)                 # host-chosen unstable inlet
    hit = None
    for k in range(1, 41):
        g.step(1)
        o = g.observables(allow_nan=True)
        if o["nonfinite"] > 0:
            hit = k
            break
    assert hit is not None and hit <= 20, hit
    with pytest.raises(lbm.LbmError) as e:
        g.observables()
    assert e.value.status == lbm.LBM_ENAN
    # roll back: the checkpoint restores the state and the reservoirs in
    # force; the inlet goes back to its value
    g.load(ck)
    g.set_bc(0, 2, 1.02, 0.02)
    g.step(6)
    ref.step(6)
    assert g.observables()["nonfinite"] == 0
    assert np.array_equal(g.populations(), ref.populations())
    g.close()
    ref.close()
