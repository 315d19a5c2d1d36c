"""Workloads run twice by test_gpu_checked.py: once with the default library
in the test process and once, in a child process, with the bounds-checked
library (HMCSC_LBM_LIBRARY).  Run as a script it writes every result and the
fault word of every lattice to the .npz file named on the command line."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2206_11524_gb300 import lbm, synth  # noqa: E402


def _lattice(shape, storage="f32", per_component=False, seed=0, bcs=True):
    nz, ny, nx = shape
    g = lbm.Lattice(nx, ny, nz, tau=(0.9, 1.2), G=1.6, F_ext=(1e-5, -2e-5, 0),
                    storage=storage, rho0=(0.5, 0.5), ns_per_component=per_component)
    ns, gads = synth.random_geometry(shape, seed)
    ns2, _ = synth.random_geometry(shape, seed + 7)
    g.set_geometry(ns, gads, ns2=ns2 if per_component else None)
    if bcs:
        g.set_bc(0, min(2, nx), 1.0, 0.03)
        g.set_bc(3, 1, 0.2, 0.7, u=(0.01, 0.0, -0.005))
    g.set_populations(synth.random_state(shape, seed + 1))
    return g


def run():
    out, faults = {}, []

    def keep(name, g):
        out[name + "_f"] = g.populations()
        fl = g.fields()
        for k, v in fl.items():
            out[f"{name}_{k}"] = v
        out[name + "_mass"] = g.observables(allow_nan=True)["mass"]
        faults.append(lbm.lbm_fault_word(g.ctx))
        g.close()

    for k, shape in enumerate([(5, 4, 7), (3, 9, 33), (1, 1, 1), (2, 5, 64), (4, 1, 1)]):
        for st in ("f32", "f16l", "bf16"):
            g = _lattice(shape, st, seed=k)
            g.step(3)
            keep(f"s{k}_{st}", g)
    g = _lattice((4, 6, 40), per_component=True, seed=11)
    g.step(3)
    keep("pc", g)
    for cfg in ((0, 8, 9), (0, 6, 7)):   # prefetching shapes, per component
        g = _lattice((5, 9, 37), "f32", per_component=True, seed=14)
        g.set_launch_config(*cfg)
        g.step(4)
        keep("pc_cfg" + "".join(map(str, cfg)), g)
    g = _lattice((6, 17, 100), seed=12)
    g.set_single_pass(3)
    g.step(4)
    keep("single", g)
    for k, (shape, st, wave) in enumerate([((6, 17, 100), "f32", (2, 0)),
                                           ((5, 9, 37), "f16l", (1, 3)),
                                           ((3, 4, 7), "bf16", (3, 6))]):
        g = _lattice(shape, st, seed=30 + k)
        g.set_wavefront(*wave)
        g.step(3)
        keep(f"wave{k}", g)
    for cfg in ((2, 3, 3), (1, 1, 1), (0, 2, 2), (0, 6, 7), (0, 8, 9), (0, 5, 5), (0, 4, 4)):
        g = _lattice((5, 9, 40), "f16l", seed=13)
        g.set_launch_config(*cfg)
        g.step(2)
        keep("cfg" + "".join(map(str, cfg)), g)
    import torch
    lats = [_lattice((4, 6, 40), seed=20), _lattice((3, 5, 33), seed=21)]
    torch.cuda.synchronize()
    stream = torch.cuda.Stream().cuda_stream   # graph capture needs a stream of its own
    lbm.lbm_batch_step([g.ctx for g in lats], 2, stream)
    graph = lbm.lbm_batch_graph_create([g.ctx for g in lats], 2, stream)
    lbm.lbm_batch_graph_launch(graph, stream)
    torch.cuda.synchronize()
    lbm.lbm_batch_graph_destroy(graph)
    for k, g in enumerate(lats):
        keep(f"batch{k}", g)
    g = lbm.Lattice(20, 6, 3)
    g.set_geometry(np.full((3, 6, 20), 0.3))
    g.init_equilibrium(np.full((3, 6, 20), 0.7), np.full((3, 6, 20), 0.3))
    g.step(2)
    keep("init", g)
    out["faults"] = np.array(faults, dtype=np.uint32)
    out["checked"] = np.array(lbm.lbm_build_checked())
    return out


if __name__ == "__main__":
    lbm.load()
    np.savez(sys.argv[1], **run())
