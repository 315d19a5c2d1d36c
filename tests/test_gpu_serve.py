"""Batched stepping, CUDA graphs and the continuous-batching server: every
simulation's result is the same alone and in the mix (bit for bit: the
batched kernels run the same per-node arithmetic)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2206_11524_gb300 import build, lbm, serve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    lbm.load()


def _lattices(storage, shapes=((20, 12, 40), (8, 30, 64), (17, 9, 33))):
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
        lats.append(g)
    return lats


@pytest.mark.parametrize("storage", ["f32", "f16l"])
def test_batch_step_equals_single_steps(storage):
    alone = _lattices(storage)
    mixed = _lattices(storage)
    for g in alone:
        g.step(7)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    lbm.lbm_batch_step([g.ctx for g in mixed], 3, stream.cuda_stream)
    lbm.lbm_batch_step([g.ctx for g in mixed[1:]], 1, stream.cuda_stream)  # parities differ now
    lbm.lbm_batch_step([mixed[0].ctx], 1, stream.cuda_stream)
    lbm.lbm_batch_step([g.ctx for g in mixed], 3, stream.cuda_stream)
    stream.synchronize()
    for a, b in zip(alone, mixed):
        assert a.t == b.t == 7
        assert np.array_equal(a.populations(), b.populations())


def test_graph_replay_equals_steps_and_guards_state():
    alone = _lattices("f32")
    mixed = _lattices("f32")
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


@pytest.mark.parametrize("storage", ["f32", "f16l"])
def test_server_results_equal_alone_results(storage):
    reqs = serve.make_requests(n_req=5, seed=7, L_min=20, L_max=52, steps_min=20,
                               steps_max=60, base_n=64)
    for k, r in enumerate(reqs):        # staggered arrivals: the mix changes
        r.arrival = 0.05 * k
    srv = serve.Server(storage=storage, tick_steps=8, keep_state=True)
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
