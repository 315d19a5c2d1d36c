"""Autotuner of the launch shapes (thread-block shape and register budget) of
the density pass and of the fused pass on even and odd steps, of the choice
between the two-pass step and the wavefront step (one persistent launch),
and optionally of the single-pass step.

`tune(nx, ny, nz, storage)` times every shape on a scratch lattice of that
size and storage (a synthetic gray medium with two-phase densities; the
kernels' cost does not depend on the values) and returns the fastest.
`TuneTable` keeps the winners in a JSON file keyed by GPU name, lattice size
and storage, so a lattice of a known size is configured without timing
(`apply(lattice)`).  The table lives at $HMCSC_TUNE_TABLE, else
~/.cache/hmcsc/launch_table.json.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import lbm


def _default_path() -> str:
    return os.environ.get("HMCSC_TUNE_TABLE") or os.path.join(
        os.path.expanduser("~"), ".cache", "hmcsc", "launch_table.json")


def _key(nx, ny, nz, storage) -> str:
    import torch
    name = torch.cuda.get_device_name(torch.cuda.current_device())
    return f"{name}|{nx}x{ny}x{nz}|{storage}"


class TuneTable:
    def __init__(self, path: str | None = None):
        self.path = path or _default_path()
        self.entries = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as fh:
                    self.entries = json.load(fh)
            except (OSError, ValueError):
                self.entries = {}

    def get(self, nx, ny, nz, storage):
        e = self.entries.get(_key(nx, ny, nz, storage))
        return tuple(e["config"]) if e else None

    def put(self, nx, ny, nz, storage, config, timings):
        self.entries[_key(nx, ny, nz, storage)] = {"config": list(config),
                                                   "timings_ms": timings}
        os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
        tmp = self.path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(self.entries, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def _scratch(nx, ny, nz, storage):
    """A lattice shaped like an imbibition run: solid, open and gray nodes
    mixed, adhesion in the gray ones, density reservoirs on both x faces
    (the reservoir checks are part of what the shapes pay for)."""
    shape = (nz, ny, nx)
    rng = np.random.default_rng(0)
    lat = lbm.Lattice(nx, ny, nz, tau=(1.0, 1.0), G=1.75, storage=storage,
                      rho0=(0.5, 0.5))
    u = rng.random(shape)
    ns = np.where(u < 0.5, 1.0, np.where(u < 0.8, 0.0, 0.2 + 0.7 * rng.random(shape)))
    lat.set_geometry(ns, np.where((ns > 0) & (ns < 1), 0.2, 0.0))
    layers = min(4, nx // 2)
    if layers > 0:
        lat.set_bc(0, layers, 1.04, 0.01)
        lat.set_bc(1, layers, 0.01, 0.99)
    ra = np.where(rng.random(shape) < 0.5, 0.99, 0.03)
    lat.init_equilibrium(ra, 1.02 - ra)
    return lat


def _time(lat, fn, reps):
    import torch
    st = lat.stream
    fn()  # warm-up (and the first launch of this shape)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        fn()
    b.record(st)
    b.synchronize()
    return a.elapsed_time(b) / reps


def _step_ms(lat, steps=10):
    import torch
    st = lat.stream
    lat.step(2)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    lat.step(steps)
    b.record(st)
    b.synchronize()
    return a.elapsed_time(b) / steps


def _single_pass_candidates(ny, nz, sms):
    """Box depths whose boxes fill one or two waves of two boxes per SM."""
    nyb = (ny + 7) // 8
    out = []
    for waves in (1, 2):
        nzc = max(1, min(nz, (waves * 2 * sms) // nyb))
        planes = max(1, round(nz / nzc))
        if planes not in out:
            out.append(planes)
    return out


# Wavefront (shape, lag) pairs the tuner weighs against the two-pass step.
WAVE_CANDIDATES = ((2, 4), (1, 4), (2, 5), (3, 4))


def tune(nx, ny, nz, storage="f32", reps=10, single_pass=False, margin=0.03,
         wavefront=True):
    """Fastest (density, even, odd) launch shapes and all timings (ms),
    extended to (density, even, odd, single-pass depth, wavefront shape,
    wavefront lag).  Whole steps of the best two-pass shapes are timed
    against the wavefront step at WAVE_CANDIDATES (with `wavefront`) and, with
    single_pass, against the single-pass step at box depths that fit the SM
    count; another step than the two-pass one is kept only if it is faster by
    more than `margin` (single-pass depth 0 and wavefront shape 0 otherwise)."""
    lat = _scratch(nx, ny, nz, storage)
    ctx = lat.ctx
    timings = {"density": [], "even": [], "odd": []}
    for d in range(lbm.LBM_DENSITY_CONFIGS):
        lbm.lbm_set_launch_config(ctx, d, 0, 0)
        timings["density"].append(_time(lat, lambda: lbm.lbm_density(ctx), reps))
    best_d = int(np.argmin(timings["density"]))

    def fused_only(parity):
        # one full step to reach the wanted parity, then time the fused pass
        # of that parity: density + fused of the other parity are untimed
        import torch
        ev = []
        st = lat.stream
        for _ in range(reps + 1):
            if lbm.lbm_time(ctx) % 2 != parity:
                lbm.lbm_step(ctx, 1)
            lbm.lbm_density(ctx)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            lbm.lbm_collide_stream(ctx)
            b.record(st)
            ev.append((a, b))
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev[1:]]))

    for e in range(lbm.LBM_COLLIDE_CONFIGS):
        lbm.lbm_set_launch_config(ctx, best_d, e, 0)
        timings["even"].append(fused_only(0))
    best_e = int(np.argmin(timings["even"]))
    for o in range(lbm.LBM_COLLIDE_CONFIGS):
        lbm.lbm_set_launch_config(ctx, best_d, best_e, o)
        timings["odd"].append(fused_only(1))
    best_o = int(np.argmin(timings["odd"]))
    cfg = (best_d, best_e, best_o)
    best_sp, best_wave = 0, (0, 0)
    if single_pass or wavefront:
        lbm.lbm_set_launch_config(ctx, *cfg)
        two = _step_ms(lat)
        timings["two_pass_step"] = two
        best_ms = two * (1.0 - margin)
        if wavefront:
            for shape, lag in WAVE_CANDIDATES:
                lat.set_wavefront(shape, lag)
                ms = _step_ms(lat)
                timings[f"wavefront_{shape}_{lag}"] = ms
                if ms < best_ms:
                    best_wave, best_ms = (shape, lag), ms
            lat.set_wavefront(0)
        if single_pass and nx <= lbm.SINGLE_PASS_MAX_NX:
            import torch
            sms = torch.cuda.get_device_properties(
                torch.cuda.current_device()).multi_processor_count
            for planes in _single_pass_candidates(ny, nz, sms):
                lat.set_single_pass(planes)
                ms = _step_ms(lat)
                timings[f"single_pass_{planes}"] = ms
                if ms < best_ms:
                    best_sp, best_wave, best_ms = planes, (0, 0), ms
            lat.set_single_pass(0)
    lat.close()
    return cfg + (best_sp,) + best_wave, timings


def apply(lattice, table: TuneTable | None = None, tune_if_missing=True,
          single_pass=False, wavefront=True):
    """Configure `lattice` from the table, tuning (and recording) its size
    and storage first when the table has no entry.  An entry's optional
    fourth value is the single-pass box depth (0: two passes), its optional
    fifth and sixth the wavefront shape (0: off) and lag."""
    table = table or TuneTable()
    nz, ny, nx = lattice.shape
    storage = lattice.storage_name
    cfg = table.get(nx, ny, nz, storage)
    if cfg is None and tune_if_missing:
        cfg, timings = tune(nx, ny, nz, storage, single_pass=single_pass,
                            wavefront=wavefront)
        table.put(nx, ny, nz, storage, cfg, timings)
    if cfg is not None:
        lbm.lbm_set_launch_config(lattice.ctx, *cfg[:3])
        lattice.set_single_pass(cfg[3] if len(cfg) > 3 else 0)
        lattice.set_wavefront(*(cfg[4:6] if len(cfg) > 5 else (0, 0)))
    return cfg
