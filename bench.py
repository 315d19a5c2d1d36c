"""Throughput benchmark of the HMCSC D3Q19 step on GB300.

Workload: the synthetic 256^3 electrode-imbibition problem (Boolean model of
solid spheres, gray binder blobs with per-blob n_s, reservoirs at x = 0 and
x = 255, Table 1 parameters), float32 populations.  A benchmark step is one
lattice time step over the whole domain in the form the autotuner picks:
the wavefront launch (density sums and the fused force/collide/bounce-back/
stream work in one persistent launch) or the density pass followed by the
fused pass (``--no-wavefront`` keeps the two passes).

Prints one JSON line:
  value    aggregate MLUPS (lattice node updates per second / 1e6, both
           components) over all ranks, device-timed with CUDA events;
  e2e      the same metric through the C ABI with host buffers: geometry and
           density upload, the steps, and the field read-back inside the
           timed region;
  roofline the dominant launch's algorithmic bytes over its average
           duration (the wavefront launch, or the fused pass of the two-pass
           step), against the measured HBM copy bandwidth;
  cpu_baseline  the FP64 oracle on the host cores on a bounded sample.

``--impl reference`` times the FP64 CPU oracle instead (rank 0 only).
Multi-GPU (torchrun): every rank advances its own replica of the domain; no
data crosses ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "2-comp D3Q19 MLUPS"
UNIT = "MLUPS"
# Algorithmic bytes per node and step (float32 storage):
#   density pass: read 2 x 19 x 4, write 2 x 4              = 160
#   fused pass:   read 2 x 19 x 4 + rho 8 + n_s 4 + a 4,
#                 write 2 x 19 x 4                          = 320
#   wavefront launch (whole step): read 2 x 19 x 4 + n_s 4 + a 4,
#                 write 2 x 19 x 4 + rho 8                  = 320
BYTES_DENSITY = 160
BYTES_COLLIDE = 320
# 16-bit storages (2 B per population): offset kinds 84 / 168; local kinds
# also read the node's own previous density (8 B) in both passes.
STORAGE_BYTES = {"f32": (160, 320), "f16": (84, 168), "bf16": (84, 168),
                 "f16l": (92, 176), "bf16l": (92, 176)}
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 8000.0   # GB300 HBM3e nominal, for context only
PIPE_FIRST = 5             # first fused-pass launch shape of k_collide_pipe


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _seam_nodes(nx, ny, nz, planes, box_rows=8):
    """Nodes of the single-pass seams: the last row of every box of
    box_rows rows and the last plane of every run of about `planes` planes."""
    nzc = max(1, min(nz, (nz + planes // 2) // planes))
    seam_rows = (ny + box_rows - 1) // box_rows
    return nx * (seam_rows * nz + (ny - seam_rows) * nzc)


def _kernel_sha():
    """Hash of the device code (comments and blank lines removed, so that an
    edit of comments alone keeps a capture valid)."""
    import re
    h = hashlib.sha256()
    for f in ("lbm_device.cuh", "lbm_internal.cuh", "lbm_storage_impl.cuh"):
        with open(os.path.join(ROOT, "paper_2206_11524_gb300", "csrc", f)) as fh:
            code = re.sub(r"//[^\n]*", "", fh.read())
        h.update("\n".join(l.rstrip() for l in code.splitlines() if l.strip()).encode())
    return h.hexdigest()[:16]


def _profiled_traffic(kernel):
    """DRAM bytes per node of `kernel` from the committed ncu summary, if the
    summary was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_electrode256.md")
    if not os.path.exists(path):
        return None
    sha = bpn = None
    for line in open(path):
        if line.startswith("kernel_source_sha256_16:"):
            sha = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_node:"):
            bpn = float(line.split(":", 1)[1].strip())
    if sha != _kernel_sha() or bpn is None:
        return None
    return bpn


_UNIT_SCALE = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "tbyte": 1e12,
               "nsecond": 1e-9, "usecond": 1e-6, "msecond": 1e-3, "second": 1.0,
               "ns": 1e-9, "us": 1e-6, "ms": 1e-3, "s": 1.0}


def record_traffic(csv_path, kernel, nodes):
    """Per-launch DRAM bytes of `kernel` from an ncu --csv log of
    dram__bytes_read.sum, dram__bytes_write.sum and gpu__time_duration.sum;
    writes the machine-readable lines (source hash, bytes per node) of
    profiles/<kernel>_electrode256.md and returns the per-launch rows."""
    import csv
    import re
    rows = {}
    with open(csv_path, newline="") as fh:
        lines = [l for l in fh if l.startswith('"')]
    for r in csv.DictReader(lines):
        name = r.get("Kernel Name", "")
        if name != kernel and not re.search(r"(^|[^A-Za-z0-9_])" + kernel + r"[<(]", name):
            continue
        key = r["ID"]
        val = float(r["Metric Value"].replace(",", ""))
        val *= _UNIT_SCALE.get(r["Metric Unit"].strip().lower(), 1.0)
        rows.setdefault(key, {"kernel": name})[r["Metric Name"]] = val
    out = []
    for key in sorted(rows, key=int):
        m = rows[key]
        rd, wr = m["dram__bytes_read.sum"], m["dram__bytes_write.sum"]
        out.append({"id": int(key), "kernel": m["kernel"],
                    "us": m.get("gpu__time_duration.sum", float("nan")) * 1e6,
                    "read_per_node": rd / nodes, "write_per_node": wr / nodes,
                    "total_per_node": (rd + wr) / nodes})
    if not out:
        raise SystemExit(f"no launches of {kernel} in {csv_path}")
    bpn = sum(r["total_per_node"] for r in out) / len(out)
    short = kernel[2:] if kernel.startswith("k_") else kernel
    path = os.path.join(ROOT, "profiles", f"{short}_electrode256.md")
    text = open(path).read() if os.path.exists(path) else ""
    keep = [l for l in text.splitlines()
            if not l.startswith(("kernel_source_sha256_16:", "dram_bytes_per_node:"))]
    while keep and not keep[-1].strip():
        keep.pop()
    keep += ["", f"kernel_source_sha256_16: {_kernel_sha()}",
             f"dram_bytes_per_node: {bpn:.2f}"]
    with open(path, "w") as fh:
        fh.write("\n".join(keep) + "\n")
    return out, bpn


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate_max(value: float, world: int) -> float:
    """Max of a float over ranks (identity when world == 1)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_oracle_mlups(case_small, budget_s: float, max_steps: int | None = None):
    """Time the FP64 oracle on a bounded sample; returns (MLUPS, steps, s)."""
    import oracle
    oracle.build()
    nz, ny, nx = case_small.shape
    p = oracle.Params(nx, ny, nz, tau=case_small.tau, G=case_small.G,
                      Fext=case_small.F_ext, reservoirs=case_small.reservoirs)
    s = oracle.Sim(p, case_small.ns, case_small.gads2)
    s.init_equilibrium(case_small.rho_a, case_small.rho_b)
    s.step(1)                      # warm-up (page-in, thread start)
    steps = 0
    t0 = time.perf_counter()
    while True:
        s.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_steps and steps >= max_steps):
            break
    return case_small.n_nodes * steps / el / 1e6, steps, el


def _single_core_oracle(seconds):
    """The same oracle sample on one host core (a child process started with
    OMP_NUM_THREADS=1, since the thread count is fixed when the library
    loads)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, os.path.abspath(__file__),
                              "--cpu-probe", str(seconds)], env=env,
                             capture_output=True, text=True, timeout=300)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # the single-core figure is context only
        return {"unavailable": str(e)[:200]}


def _cpu_probe(seconds):
    from paper_2206_11524_gb300 import synth
    small = synth.electrode((64, 64, 64))
    mlups, st, el = cpu_oracle_mlups(small, seconds)
    print(json.dumps({"value": mlups, "unit": UNIT, "cores": 1,
                      "sample": f"64^3 synthetic electrode, {st} FP64 time "
                                f"steps in {el:.1f} s"}), flush=True)
    return 0


def _cores():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


def run_reference(args, world, rank):
    """The FP64 oracle on the host cores, on the same workload's generator at
    64^3 (a bounded sample): W untimed time steps, then K timed ones."""
    if rank != 0:
        return 0
    import oracle
    from paper_2206_11524_gb300 import synth
    oracle.build()
    small = synth.electrode((64, 64, 64))
    nz, ny, nx = small.shape
    p = oracle.Params(nx, ny, nz, tau=small.tau, G=small.G, Fext=small.F_ext,
                      reservoirs=small.reservoirs)
    sim = oracle.Sim(p, small.ns, small.gads2)
    sim.init_equilibrium(small.rho_a, small.rho_b)
    sim.step(args.warmup)
    t0 = time.perf_counter()
    sim.step(args.steps)
    el = time.perf_counter() - t0
    v = small.n_nodes * args.steps / el / 1e6
    sample = (f"synthetic electrode generator at 64^3 ({small.n_nodes} nodes), "
              f"one FP64 time step per benchmark step")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"electrode imbibition {args.size}^3 "
                                   "(sampled at 64^3 on the host cores)",
                       "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": _cores(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def serving_leg(args):
    """Continuous batching (local half-offset storage, the two batched passes
    per step over the batch, CUDA graphs) against one-at-a-time float32 runs
    (two passes each) on the same seeded trace of heterogeneous requests:
    the trace of the serving workload (256 requests, cubic L log-uniform in
    [32, 192]) with the step budgets scaled down, offered at 0.9
    of the sequential capacity and with every request arriving at once; the
    capacity run also serves the faster half offsets from a constant (f16)."""
    from paper_2206_11524_gb300 import serve
    out = serve.compare(n_req=args.serve_requests, L_min=32, L_max=args.serve_lmax,
                        steps_min=args.serve_steps_min, steps_max=args.serve_steps_max,
                        storage=args.serve_storage, load=0.9, seed=2206, overload=True,
                        overload_storages=("f16",))
    out["config"] = (f"{args.serve_requests} requests, L in [32, {args.serve_lmax}], steps "
                     f"U{{{args.serve_steps_min}..{args.serve_steps_max}}} (the 5,000-40,000 "
                     f"of the full trace scaled by {args.serve_steps_max / 40000:.3g})")
    return out


def _lattice_for(case, storage, stream):
    from paper_2206_11524_gb300 import lbm
    nz, ny, nx = case.shape
    lat = lbm.Lattice(nx, ny, nz, tau=case.tau, G=case.G, F_ext=case.F_ext,
                      stream=stream, storage=storage, rho0=(0.5, 0.5))
    lat.set_geometry(case.ns, case.gads2)
    for face, (L, r1, r2) in case.reservoirs.items():
        lat.set_bc(face, L, r1, r2)
    lat.init_equilibrium(case.rho_a, case.rho_b)
    return lat


# Two-pass launch shapes (density, even, odd) measured fastest per storage
# on the benchmark lattice (the 16-bit storages keep the two-pass step:
# their wavefront step is slower)
DEFAULT_LAUNCH = {"f32": (1, 6, 7), "f16": (0, 6, 8), "bf16": (0, 6, 8),
                  "f16l": (0, 9, 9), "bf16l": (0, 9, 9)}


def _time_two_pass(lat, steps, stream):
    """Mean ms per step and of the fused pass (CUDA events on the stream)."""
    import torch
    from paper_2206_11524_gb300 import lbm
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for e0, e1, e2 in ev:
        e0.record(stream)
        lbm.lbm_density(lat.ctx)
        e1.record(stream)
        lbm.lbm_collide_stream(lat.ctx)
        e2.record(stream)
    torch.cuda.synchronize()
    step = sum(a.elapsed_time(c) for a, _, c in ev) / steps
    fused = sum(b.elapsed_time(c) for _, b, c in ev) / steps
    return step, fused


def storage_record(case, storage, steps, warmup, peak):
    """Two-pass step of one population storage on the benchmark lattice
    (float32 included: its fused pass is the fused step of the method, timed
    apart from the wavefront launch the headline uses): MLUPS and the fused
    pass's roofline on its own algorithmic bytes."""
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        lat = _lattice_for(case, storage, stream)
    lat.set_launch_config(*DEFAULT_LAUNCH[storage])
    lat.step(warmup)
    step_ms, fused_ms = _time_two_pass(lat, steps, stream)
    N = case.n_nodes
    bd, bc = STORAGE_BYTES[storage]
    obs = lat.observables()
    lat.close()
    achieved = bc * N / (fused_ms / 1e3) / 1e9
    return {"storage": storage, "step": "two passes (density pass, fused pass)",
            "launch_config": list(DEFAULT_LAUNCH[storage]),
            "mlups": N / (step_ms / 1e3) / 1e6, "ms_per_step": step_ms,
            "roofline": {"bound": "hbm", "kernel": "fused pass (k_collide_pipe)",
                         "algorithmic_bytes_per_node": bc, "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak},
            "step_bytes_per_node": bd + bc,
            "step_frac": (bd + bc) * N / (step_ms / 1e3) / 1e9 / peak,
            "nonfinite": int(obs["nonfinite"])}


def large_domain_record(args, peak):
    """Config 4: the 512 x 512 x 384 synthetic electrode (~100M nodes) in
    half-precision offset storage: MLUPS, the fused pass's roofline, the end
    to end rate through the C ABI with host buffers, and the L-infinity
    error of the saturation curve S_1(t) against a float32 run."""
    import numpy as np
    import torch
    from paper_2206_11524_gb300 import lbm, synth
    nx, ny, nz = (int(v) for v in args.large_shape.split(","))
    t0 = time.perf_counter()
    case = synth.electrode((nz, ny, nx))
    gen_s = time.perf_counter() - t0
    N = case.n_nodes
    stream = torch.cuda.Stream()
    curves = {}
    rec = {"shape": [nx, ny, nz], "nodes": N, "storage": args.large_storage,
           "generation_s": gen_s}
    for storage in (args.large_storage, "f32"):
        with torch.cuda.stream(stream):
            lat = _lattice_for(case, storage, stream)
        lat.set_launch_config(*DEFAULT_LAUNCH[storage])
        curve = []
        for _ in range(args.large_s1_steps // args.large_s1_every):
            lat.step(args.large_s1_every)
            curve.append(lat.observables()["sat1"])
        curves[storage] = np.array(curve)
        if storage == args.large_storage:
            lat.step(args.warmup)
            step_ms, fused_ms = _time_two_pass(lat, args.large_steps, stream)
            bd, bc = STORAGE_BYTES[storage]
            achieved = bc * N / (fused_ms / 1e3) / 1e9
            rec.update({"mlups": N / (step_ms / 1e3) / 1e6, "ms_per_step": step_ms,
                        "workspace_gb": lat.workspace.numel() / 1e9,
                        "roofline": {"bound": "hbm", "kernel": "fused pass (k_collide_pipe)",
                                     "algorithmic_bytes_per_node": bc,
                                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                                     "frac": achieved / peak}})
            # end to end through the C ABI: host geometry and densities in,
            # the steps, every field back
            def pinned(shape):
                return torch.empty(shape, dtype=torch.float32, pin_memory=True).numpy()
            h = [pinned(case.shape) for _ in range(4)]
            for a, v in zip(h, (case.ns, case.gads2, case.rho_a, case.rho_b)):
                a[...] = v
            out = [pinned(case.shape) for _ in range(3)] + [pinned((3,) + case.shape)]
            K = args.large_steps
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            lbm.lbm_set_geometry(lat.ctx, h[0], h[1], N)
            lbm.lbm_init_equilibrium(lat.ctx, h[2], h[3], N)
            lbm.lbm_step(lat.ctx, K)
            lbm.lbm_read_fields(lat.ctx, out[0], out[1], out[3], out[2])
            e2e_s = time.perf_counter() - t1
            rec["e2e"] = {"value": N * K / e2e_s / 1e6, "unit": UNIT,
                          "h2d_bytes_per_step": 4 * 4 * N / K,
                          "d2h_bytes_per_step": 6 * 4 * N / K}
        lat.close()
        del lat
        torch.cuda.empty_cache()
    err = float(np.abs(curves[args.large_storage] - curves["f32"]).max())
    rec["sat1_vs_f32"] = {"linf": err, "steps": args.large_s1_steps,
                          "every": args.large_s1_every,
                          "sat1_final_f32": float(curves["f32"][-1])}
    return rec


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch
    from paper_2206_11524_gb300 import build as lib_build
    from paper_2206_11524_gb300 import lbm, synth

    lib_build.build()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    if args.shape:
        nx, ny, nz = (int(v) for v in args.shape.split(","))
    else:
        nx = ny = nz = args.size
    case = synth.electrode((nz, ny, nx))
    N = case.n_nodes
    storage = args.storage
    bytes_density, bytes_collide = STORAGE_BYTES[storage]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        lat = lbm.Lattice(nx, ny, nz, tau=case.tau, G=case.G, F_ext=case.F_ext,
                          stream=stream, storage=storage, rho0=(0.5, 0.5))
    ctx = lat.ctx
    lat.set_geometry(case.ns, case.gads2)
    for face, (L, r1, r2) in case.reservoirs.items():
        lat.set_bc(face, L, r1, r2)
    lat.init_equilibrium(case.rho_a, case.rho_b)
    launch = None
    if args.launch_config:
        launch = [int(v) for v in args.launch_config.split(",")]
        lat.set_launch_config(*launch)
    elif not args.no_autotune:
        import tempfile
        from paper_2206_11524_gb300 import autotune
        table = autotune.TuneTable(os.path.join(tempfile.mkdtemp(), "launch_table.json"))
        launch = list(lat.autotune(table))
    launch = list(lat.launch_config())   # the shapes actually in use

    single = args.single_pass > 0
    if single:
        lat.set_single_pass(args.single_pass)
    if args.wavefront:
        lat.set_wavefront(*([int(v) for v in args.wavefront.split(",")] + [0])[:2])
    elif args.no_wavefront:
        lat.set_wavefront(0)
    wave = list(lat.wavefront())          # the step in use (tuned or asked for)
    if wave[0] == 0 or single:
        wave = None
    one_launch = single or wave is not None
    for _ in range(args.warmup):
        if one_launch:
            lbm.lbm_step(ctx, 1)
        else:
            lbm.lbm_density(ctx)
            lbm.lbm_collide_stream(ctx)
    torch.cuda.synchronize()

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    start.record(stream)
    for k in range(K):
        e0, e1, e2 = ev[k]
        e0.record(stream)
        if one_launch:
            lbm.lbm_step(ctx, 1)   # wavefront launch, or bulk sweep + seam launches
        else:
            lbm.lbm_density(ctx)
        e1.record(stream)
        if not one_launch:
            lbm.lbm_collide_stream(ctx)
        e2.record(stream)
    stop.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = start.elapsed_time(stop)
    ms_density = sum(a.elapsed_time(b) for a, b, _ in ev) / K
    ms_collide = sum(b.elapsed_time(c) for _, b, c in ev) / K
    ms_max = aggregate_max(ms, world)
    value = world * N * K / (ms_max / 1e3) / 1e6
    obs = lat.observables()
    assert obs["nonfinite"] == 0, "non-finite densities in the benchmark run"

    # End to end through the C ABI with host buffers (pinned).
    def pinned(shape):
        return torch.empty(shape, dtype=torch.float32, pin_memory=True).numpy()
    h_ns, h_g = pinned(case.shape), pinned(case.shape)
    h_ra, h_rb = pinned(case.shape), pinned(case.shape)
    h_ns[...] = case.ns
    h_g[...] = case.gads2
    h_ra[...] = case.rho_a
    h_rb[...] = case.rho_b
    o_ra, o_rb, o_p = pinned(case.shape), pinned(case.shape), pinned(case.shape)
    o_u = pinned((3,) + case.shape)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm.lbm_set_geometry(ctx, h_ns, h_g, N)
    lbm.lbm_init_equilibrium(ctx, h_ra, h_rb, N)
    lbm.lbm_step(ctx, K)
    lbm.lbm_read_fields(ctx, o_ra, o_rb, o_u, o_p)
    e2e_s = aggregate_max(time.perf_counter() - t0, world)
    e2e_value = world * N * K / e2e_s / 1e6
    h2d = 4 * 4 * N
    d2h = 6 * 4 * N

    peak, peak_kind = _peaks()
    dims = f"{nx}^3" if nx == ny == nz else f"{nx}x{ny}x{nz}"
    if wave is not None:
        # whole step in one launch: the fused pass's bytes (the populations
        # through DRAM once; the densities written instead of read)
        kernel_name = "k_wave"
        bytes_launch = bytes_collide * N
        achieved = bytes_launch / (ms_density / 1e3) / 1e9
        traffic_bpn = _profiled_traffic("wave") if storage == "f32" else None
        step_gbs = bytes_launch / (ms_max / K / 1e3) / 1e9
    elif single:
        # whole single-pass step: every node 320 B as in the fused pass, and
        # the density pass's 160 B again only for the seam nodes
        n_seam = _seam_nodes(nx, ny, nz, args.single_pass)
        kernel_name = "single-pass step (k_sp_bulk + k_sp_seams)"
        bytes_launch = bytes_collide * N + bytes_density * n_seam
        achieved = bytes_launch / (ms_density / 1e3) / 1e9
        traffic_bpn = None
        step_gbs = bytes_launch / (ms_max / K / 1e3) / 1e9
    else:
        step_gbs = (bytes_density + bytes_collide) * N / (ms_max / K / 1e3) / 1e9
        # fused-pass shapes from PIPE_FIRST on run the prefetching kernel
        names = sorted({"k_collide_pipe" if c >= PIPE_FIRST else "k_collide_stream"
                        for c in launch[1:3]})
        kernel_name = " / ".join(names)
        bytes_launch = bytes_collide * N
        achieved = bytes_collide * N / (ms_collide / 1e3) / 1e9
        traffic_bpn = _profiled_traffic("collide_stream") if storage == "f32" else None
    ws_gb = lat.workspace.numel() / 1e9
    if rank != 0:
        return 0
    lat.close()
    del lat
    torch.cuda.empty_cache()
    storages = {}
    if world == 1 and args.storages:
        for st in args.storages.split(","):
            storages[f"storage_{st}"] = storage_record(case, st, args.storage_steps,
                                                       args.warmup, peak)
    large = None
    if world == 1 and args.large_shape:
        large = large_domain_record(args, peak)
    serving = None
    if world == 1 and args.serve_requests > 0:
        serving = serving_leg(args)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        small = synth.electrode((64, 64, 64))
        mlups, st, el = cpu_oracle_mlups(small, args.cpu_seconds)
        cpu = {"value": mlups, "unit": UNIT, "cores": _cores(), "kind": "oracle",
               "sample": f"64^3 crop-size synthetic electrode, {st} FP64 "
                         f"time steps in {el:.1f} s",
               "single_core": _single_core_oracle(args.cpu_seconds / 3)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": ms_max / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"electrode imbibition {dims}: synthetic "
                               "overlapping-sphere solid (n_s=1) + gray binder "
                               "blobs (n_s~U[0.2,0.9]), reservoirs at x=0 and "
                               f"x={nx - 1}, tau=1, G=1.75, {storage} storage",
                   "storage": storage,
                   "nodes": N, "global_nodes": N * world,
                   "l2": "inputs larger than L2 (working set "
                         f"{ws_gb:.2f} GB)",
                   "parallelism": f"replicas x{world}",
                   "launch_config": launch,
                   "wavefront": ({"shape": wave[0], "lag": wave[1]}
                                 if wave is not None else None)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": f"{peak_kind} hbm_gbs",
                     "kernel": kernel_name,
                     "algorithmic_bytes_per_node": bytes_launch / N,
                     "traffic": (traffic_bpn * N if traffic_bpn else None)},
        "kernels_ms": ({"wavefront_step": ms_density} if wave is not None else
                       {"single_pass_step": ms_density} if single else
                       {"density": ms_density, "collide_stream": ms_collide}),
        "step_hbm_gbs": step_gbs,
        "step_frac": step_gbs / peak,
        "frac_of_nominal_8tbs": {"fused_pass": achieved / NOMINAL_HBM_GBS,
                                 "step": step_gbs / NOMINAL_HBM_GBS},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / K,
                "d2h_bytes_per_step": d2h / K},
        # density pass + fused pass per step, bulk sweep + 2 seam launches,
        # or one wavefront launch
        "gpu_launches": (1 if wave is not None else 3 if single else 2) * K,
        "clocks": clk,
        "cpu_baseline": cpu,
        "large_domain": large,
        "serving": serving,
    }
    line.update(storages)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--shape", default="", help="nx,ny,nz (overrides --size)")
    ap.add_argument("--storage", default="f32", choices=sorted(STORAGE_BYTES))
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--wavefront", default="",
                    help="time the wavefront step: SHAPE[,LAG] (see lbm_set_wavefront)")
    ap.add_argument("--no-wavefront", action="store_true",
                    help="time the two-pass step even where the tuner picks the wavefront")
    ap.add_argument("--single-pass", type=int, default=0,
                    help="time the single-pass step with boxes of about this many planes")
    ap.add_argument("--launch-config", default="",
                    help="density,even,odd launch shapes (skips the autotuner)")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--serve-lmax", type=int, default=192)
    ap.add_argument("--serve-steps-min", type=int, default=156)
    ap.add_argument("--serve-steps-max", type=int, default=1250)
    ap.add_argument("--serve-storage", default="f16l")
    ap.add_argument("--storages", default="f32,f16,f16l",
                    help="storages whose two-pass step is timed on the same lattice "
                         "(comma list; '' skips)")
    ap.add_argument("--storage-steps", type=int, default=40)
    ap.add_argument("--large-shape", default="512,512,384",
                    help="nx,ny,nz of the large single-domain record ('' skips)")
    ap.add_argument("--large-storage", default="f16")
    ap.add_argument("--large-steps", type=int, default=20)
    ap.add_argument("--large-s1-steps", type=int, default=400)
    ap.add_argument("--large-s1-every", type=int, default=50)
    ap.add_argument("--cpu-probe", type=float, default=0.0, help=argparse.SUPPRESS)
    ap.add_argument("--record-traffic", default="",
                    help="ncu --csv log of the DRAM-byte metrics: write the traffic lines "
                         "of the kernel's profile summary (no GPU needed)")
    ap.add_argument("--record-kernel", default="k_wave")
    args = ap.parse_args(argv)
    if args.cpu_probe > 0:
        return _cpu_probe(args.cpu_probe)
    if args.record_traffic:
        if args.shape:
            nx, ny, nz = (int(v) for v in args.shape.split(","))
        else:
            nx = ny = nz = args.size
        rows, bpn = record_traffic(args.record_traffic, args.record_kernel, nx * ny * nz)
        for r in rows:
            print(json.dumps(r))
        print(json.dumps({"dram_bytes_per_node": bpn, "kernel_source_sha256_16": _kernel_sha()}))
        return 0
    world, rank, local = _dist()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_gpu(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
