"""Batched stepping, CUDA graphs and the continuous-batching server: every
simulation's result matches the FP64 oracle and is the same alone and in the
mix (bit for bit: the batched kernels run the same per-node arithmetic), for
both batched forms: the two batched passes, and the persistent wavefront
launch over all lattices (contexts on the wavefront step)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2206_11524_gb300 import build, lbm, serve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    lbm.load()


def _w64(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("wave", [0, 2])
def test_batch_matches_oracle(wave):
    """A mixed batch -- three lattice sizes (ragged x-tiles), reservoirs on
    two of them, unequal tau, a body force, random states and geometry --
    against the oracle: every population after each batched call, also once
    the lattices' AA parities differ."""
    shapes = ((5, 9, 40), (8, 6, 33), (3, 12, 64))
    res_of = ({0: (2, 1.04, 0.02)}, {}, {1: (3, 0.02, 0.99), 2: (1, 0.5, 0.4)})
    tau, G, F = (0.9, 1.2), 1.6, (1e-5, -2e-5, 3e-5)
    gpu, ref = [], []
    for k, shape in enumerate(shapes):
        nz, ny, nx = shape
        ns, gads = synth.random_geometry(shape, 40 + k)
        f0 = synth.random_state(shape, 50 + k).astype(np.float32)
        g = lbm.Lattice(nx, ny, nz, tau=tau, G=G, F_ext=F)
        g.set_geometry(ns, gads)
        for face, (L, a, b) in res_of[k].items():
            g.set_bc(face, L, a, b)
        g.set_populations(f0)
        g.set_wavefront(wave)
        p = oracle.Params(nx, ny, nz, tau=tuple(float(np.float32(t)) for t in tau),
                          G=float(np.float32(G)), Fext=tuple(float(np.float32(v)) for v in F),
                          reservoirs={f: (L, float(np.float32(a)), float(np.float32(b)))
                                      for f, (L, a, b) in res_of[k].items()})
        r = oracle.Sim(p, _w64(ns), _w64(gads))
        r.set_populations(f0.astype(np.float64))
        gpu.append(g)
        ref.append(r)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()

    def check(tag):
        for g, r in zip(gpu, ref):
            assert g.t == r.t
            assert np.abs(g.populations() - r.f).max() <= 2e-6 * np.abs(r.f).max(), (tag, g.t)

    lbm.lbm_batch_step([g.ctx for g in gpu], 1, stream.cuda_stream)
    stream.synchronize()
    for r in ref:
        r.step(1)
    check("all")
    gpu[1].step(1)                      # lattice 1 alone: parities differ now
    ref[1].step(1)
    torch.cuda.synchronize()
    lbm.lbm_batch_step([g.ctx for g in gpu], 2, stream.cuda_stream)
    stream.synchronize()
    for r in ref:
        r.step(2)
    check("mixed parities")
    for g in gpu:
        assert lbm.lbm_fault_word(g.ctx) == 0
        g.close()


def _lattices(storage, shapes=((20, 12, 40), (8, 30, 64), (17, 9, 33)), wave=0):
    lats = []
    for k, shape in enumerate(shapes):
        ns, gads = synth.random_geometry(shape, 100 + k)
        nz, ny, nx = shape
        g = lbm.Lattice(nx, ny, nz, tau=(0.9, 1.1), G=1.75, F_ext=(1e-5, 0, 2e-5),
                        storage=storage, rho0=(0.5, 0.5))
        g.set_geometry(ns, gads)
        g.set_bc(0, 3, 1.04, 0.01)
        ra = np.where(np.arange(nx) < nx // 2, 0.99, 0.02) * np.ones(shape)
        g.init_equilibrium(ra, 1.01 - ra)
        g.set_wavefront(wave)
        lats.append(g)
    return lats


@pytest.mark.parametrize("wave", [0, 2])
@pytest.mark.parametrize("storage", ["f32", "f16", "f16l", "bf16", "bf16l"])
def test_batch_step_equals_single_steps(storage, wave):
    """Batched steps equal single steps bit for bit, also while the
    lattices of one batched call are at different AA parities (one launch
    per parity present)."""
    alone = _lattices(storage)
    mixed = _lattices(storage, wave=wave)
    for g in alone:
        g.step(7)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    lbm.lbm_batch_step([g.ctx for g in mixed], 3, stream.cuda_stream)
    lbm.lbm_batch_step([g.ctx for g in mixed[1:]], 1, stream.cuda_stream)
    # parities differ now: lattice 0 at t = 3, the others at t = 4
    lbm.lbm_batch_step([g.ctx for g in mixed], 3, stream.cuda_stream)
    lbm.lbm_batch_step([mixed[0].ctx], 1, stream.cuda_stream)
    stream.synchronize()
    for a, b in zip(alone, mixed):
        assert a.t == b.t == 7
        assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("wave", [0, 2])
def test_graph_replay_equals_steps_and_guards_state(wave):
    alone = _lattices("f32")
    mixed = _lattices("f32", wave=wave)
    stream = torch.cuda.Stream()
    lbm.lbm_batch_step([g.ctx for g in mixed], 1, stream.cuda_stream)  # reservoirs in force
    stream.synchronize()
    graph = lbm.lbm_batch_graph_create([g.ctx for g in mixed], 4, stream.cuda_stream)
    for _ in range(3):
        lbm.lbm_batch_graph_launch(graph, stream.cuda_stream)
    stream.synchronize()
    for a in alone:
        a.step(13)
    for a, b in zip(alone, mixed):
        assert b.t == 13
        assert np.array_equal(a.populations(), b.populations())
    # a lattice stepped outside the graph breaks its parity: refused
    mixed[1].step(1)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_graph_launch(graph, stream.cuda_stream)
    assert e.value.status == lbm.LBM_ESTATE
    lbm.lbm_batch_graph_destroy(graph)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_batch_step([mixed[0].ctx, mixed[0].ctx], 1, stream.cuda_stream)


def _alone_state(req, storage):
    lat = serve._lattice_for(req, storage, torch.cuda.current_stream())
    lat.step(req.steps)
    f = lat.populations()
    lat.close()
    return f


@pytest.mark.parametrize("wave", [0, 2])
@pytest.mark.parametrize("storage", ["f32", "f16l"])
def test_server_results_equal_alone_results(storage, wave):
    reqs = serve.make_requests(n_req=5, seed=7, L_min=20, L_max=52, steps_min=20,
                               steps_max=60, base_n=64)
    for k, r in enumerate(reqs):        # staggered arrivals: the mix changes
        r.arrival = 0.05 * k
    srv = serve.Server(storage=storage, tick_steps=8, keep_state=True, wave=wave)
    results = {r.rid: r for r in srv.run(reqs)}
    assert srv.graph_launches > 0
    for req in reqs:
        got = results[req.rid].observables["populations"]
        assert np.array_equal(got, _alone_state(req, storage)), req.rid
    summary = serve.summarize(list(results.values()))
    assert summary["requests"] == 5 and summary["p99_s"] >= summary["p50_s"] > 0


def test_sequential_baseline_runs():
    reqs = serve.make_requests(n_req=2, seed=3, L_min=16, L_max=24, steps_min=10,
                               steps_max=20, base_n=32)
    res = serve.run_sequential(reqs)
    assert len(res) == 2 and all(r.observables["nonfinite"] == 0 for r in res)


def test_compare_reports_capacity_and_arrival_arms():
    """The serving comparison on a tiny trace: the capacity run with a
    second batched storage and the arrival run, every request answered in
    every arm, and each batched result set beside its float32 one (the
    local-offset storage stays close on so few steps)."""
    out = serve.compare(n_req=6, L_min=16, L_max=28, steps_min=8, steps_max=24,
                        storage="f16l", load=0.9, seed=5, tick_steps=8,
                        overload_storages=("f16",))
    ov = out["overload"]
    for arm in ("sequential", "batched", "batched_f16"):
        assert ov[arm]["requests"] == 6 and ov[arm]["mlups"] > 0
    assert ov["batched"]["storage"] == "f16l" and ov["batched_f16"]["storage"] == "f16"
    for arm in ("batched", "sequential"):
        assert out[arm]["requests"] == 6
        assert out[arm]["p99_s"] >= out[arm]["p50_s"] > 0
    d = out["batched_vs_sequential_f32"]
    assert d["sat1_abs_max"] < 1e-2 and d["mass_rel_max"] < 1e-2
    assert ov["batched"]["vs_sequential_f32"]["mass_rel_max"] < 1e-2
    assert serve.compare(n_req=2, L_min=16, L_max=16, steps_min=4, steps_max=4,
                         load=0, seed=6, tick_steps=4).keys() == {"overload"}


def test_wave_batch_split_into_sets_equals_single_steps():
    """Lattices whose planes in flight do not fit half of L2 together (two
    256 x 260 / 256 x 272 planes need ~60 MB each at lag 4) go to separate
    sets of the batched wavefront launch; with a small lattice beside them
    and AA parities that differ, every population equals the lattices
    stepped alone with two passes."""
    shapes = ((5, 9, 40), (4, 260, 256), (3, 272, 256))
    alone = _lattices("f32", shapes=shapes)
    mixed = _lattices("f32", shapes=shapes, wave=2)
    for g in alone:
        g.step(5)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    lbm.lbm_batch_step([g.ctx for g in mixed], 2, stream.cuda_stream)
    lbm.lbm_batch_step([mixed[1].ctx], 1, stream.cuda_stream)
    lbm.lbm_batch_step([g.ctx for g in mixed], 2, stream.cuda_stream)
    lbm.lbm_batch_step([g.ctx for k, g in enumerate(mixed) if k != 1], 1, stream.cuda_stream)
    stream.synchronize()
    for a, b in zip(alone, mixed):
        assert a.t == b.t == 5
        assert np.array_equal(a.populations(), b.populations())
        assert lbm.lbm_fault_word(b.ctx) == 0
