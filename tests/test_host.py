"""CPU tests of the host side: the C library builds, loads and exports every
entry point of include/lbm.h; argument validation that runs before any CUDA
call; the paper's parameter conversions."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2206_11524_gb300 import build, lbm, params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lbm.load()


def _header_symbols():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    return sorted(set(re.findall(r"^LBM_API\s+[\w\s\*]+?\b(lbm_\w+)\s*\(", src, re.M)))


def test_header_declares_the_binding_symbols():
    assert _header_symbols() == sorted(lbm.ABI_SYMBOLS)


def test_header_constants_match_the_binding():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    defs = dict(re.findall(r"^#define\s+(LBM_\w+)\s+(\d+)u?\b", src, re.M))
    for name in ("LBM_DENSITY_CONFIGS", "LBM_COLLIDE_CONFIGS", "LBM_BATCH_MAX",
                 "LBM_WAVE_SHAPES", "LBM_FAULT_WAIT"):
        assert int(defs[name]) == getattr(lbm, name), name


def test_library_exports_every_declared_symbol(lib):
    for name in _header_symbols():
        assert hasattr(lib, name), name
    # nothing else of the library's internals leaks as a C symbol
    out = os.popen(f"nm -D --defined-only {build.LIB}").read()
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(_header_symbols()) <= exported
    assert not [s for s in exported if "hmcsc" in s]


def _params(nx=8, ny=4, nz=2, tau=(1.0, 1.0)):
    p = lbm.lbm_params()
    p.nx, p.ny, p.nz, p.storage = nx, ny, nz, lbm.LBM_STORAGE_F32
    p.tau[0], p.tau[1] = tau
    p.G = 1.75
    return p


def test_workspace_bytes_and_validation(lib):
    n = lbm.lbm_workspace_bytes(_params())
    assert n >= 2 * 19 * 64 * 4 and n % 256 == 0
    big = lbm.lbm_workspace_bytes(_params(256, 256, 256))
    assert big >= 16777216 * (2 * 19 * 4 + 8 + 8)
    assert lbm.lbm_workspace_bytes(_params(0, 4, 4)) == 0
    assert lbm.lbm_workspace_bytes(_params(tau=(0.5, 1.0))) == 0
    assert lbm.lbm_workspace_bytes(_params(70000, 70000, 1)) == 0  # > 2^31 nodes


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    p = _params()
    ctx = ctypes.c_void_p()
    st = lib.lbm_create(ctypes.byref(p), None, 1 << 20, None, ctypes.byref(ctx))
    assert st == lbm.LBM_EINVAL
    st = lib.lbm_create(ctypes.byref(p), ctypes.c_void_p(256), 16, None,
                        ctypes.byref(ctx))
    assert st == lbm.LBM_ENOMEM
    st = lib.lbm_create(ctypes.byref(p), ctypes.c_void_p(257), 1 << 30, None,
                        ctypes.byref(ctx))
    assert st == lbm.LBM_EINVAL          # workspace not 256-byte aligned
    assert lib.lbm_time(None) == -1
    assert lib.lbm_last_error(None) == b"context is NULL"


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            rows.append([float(v) for v in line.split()])
    return np.array(rows)


def test_contact_angle_conversion_matches_table3():
    """Eq. 15 with Table 1's parameters reproduces the theta_H column of
    Table 3 to its printed precision."""
    for gads, theta in _golden("washburn_contact_angle_table3.txt"):
        assert abs(params.contact_angle_from_gads(gads) - theta) < 0.051
        back = params.gads_from_contact_angle(params.contact_angle_from_gads(gads))
        assert abs(back - gads) < 1e-12


def test_binder_wettability_and_viscosity():
    # theta = 60 deg binder (Sec. 4): G_ads,2 = 1.75 * 0.98 / 8
    assert abs(params.gads_from_contact_angle(60.0) - 0.214375) < 1e-12
    assert abs(params.viscosity(1.0) - 1 / 6) < 1e-15       # Table 1: 1.667e-1
    assert abs(params.permeability(0.5) - 1 / 12) < 1e-15   # Eq. 2


def test_tune_table_persists(tmp_path, monkeypatch):
    from paper_2206_11524_gb300 import autotune
    monkeypatch.setattr(autotune, "_key", lambda nx, ny, nz, st: f"GPU|{nx}x{ny}x{nz}|{st}")
    t = autotune.TuneTable(str(tmp_path / "tab.json"))
    assert t.get(8, 8, 8, "f32") is None
    t.put(8, 8, 8, "f32", (1, 2, 3), {"density": [0.1]})
    assert autotune.TuneTable(str(tmp_path / "tab.json")).get(8, 8, 8, "f32") == (1, 2, 3)


def test_droplet_measurement_helpers():
    """Equivalent radius and pressure jump of the Laplace study on a
    synthetic sharp sphere with a known inside / outside pressure."""
    from paper_2206_11524_gb300 import studies, synth
    n, R0 = 64, 12.0
    case = synth.droplet(n=n, radius=R0, hi=0.98, lo=0.04)
    R = studies.droplet_radius(case.rho_a)
    assert abs(R - R0) < 0.02 * R0
    p = np.where(case.rho_a > 0.5, 0.31, 0.30)
    assert abs(studies.pressure_jump(p, R) - 0.01) < 1e-12


def test_serving_result_differences():
    """The batched-versus-float32 comparison matches requests by id and
    reports the largest and median S_1 and relative mass differences."""
    from paper_2206_11524_gb300 import serve

    def res(rid, sat1, mass):
        return serve.Result(rid, 0.0, 0.0, 1.0, 8, 2, {"sat1": sat1, "mass": mass})
    ref = [res(0, 0.5, (10.0, 2.0)), res(1, 0.25, (4.0, 4.0)), res(2, 0.0, (1.0, 1.0))]
    got = [res(2, 0.001, (1.0, 1.0)), res(0, 0.5, (10.0, 2.01)), res(1, 0.2, (4.4, 4.0))]
    d = serve.result_differences(got, ref)
    assert abs(d["sat1_abs_max"] - 0.05) < 1e-12
    assert abs(d["sat1_abs_median"] - 0.001) < 1e-12
    assert abs(d["mass_rel_max"] - 0.1) < 1e-12
    assert abs(d["mass_rel_median"] - 0.005) < 1e-12


def test_traffic_recorder_reads_ncu_csv(tmp_path, monkeypatch):
    """bench.py --record-traffic: per-launch DRAM bytes of the named kernel
    only (not k_wave_batch), units scaled, the mean per node written with the
    hash of the device code into the profile's machine-readable lines."""
    import bench
    hdr = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
           '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
           '"Metric Value"\n')

    def row(i, name, metric, unit, value):
        return (f'"{i}","1","python","h","{name}","1","7","(32, 2, 1)","(1216, 1, 1)","0",'
                f'"10.3","Command line profiler metrics","{metric}","{unit}","{value}"\n')
    kw = "void unnamed>::k_wave<1, 0, 0, 2>(StepParams, Workspace, unnamed>::WaveArgs)"
    kb = "void unnamed>::k_wave_batch<1, 0, 0, 2>(unnamed>::WaveBatch)"
    csv = tmp_path / "t.csv"
    csv.write_text("==PROF== Connected\n" + hdr +
                   row(0, kw, "dram__bytes_read.sum", "Gbyte", "3.0") +
                   row(0, kw, "dram__bytes_write.sum", "byte", "1,000,000,000") +
                   row(0, kw, "gpu__time_duration.sum", "ns", "1,200,000") +
                   row(1, kb, "dram__bytes_read.sum", "byte", "99") +
                   row(1, kb, "dram__bytes_write.sum", "byte", "99") +
                   row(2, kw, "dram__bytes_read.sum", "Mbyte", "1000") +
                   row(2, kw, "dram__bytes_write.sum", "Kbyte", "1000000") +
                   row(2, kw, "gpu__time_duration.sum", "us", "1100"))
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "wave_electrode256.md").write_text("# summary\n\nkernel_source_sha256_16: old\n"
                                               "dram_bytes_per_node: 1.0\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_kernel_sha", lambda: "abc")
    rows, bpn = bench.record_traffic(str(csv), "k_wave", 1000)
    assert [r["id"] for r in rows] == [0, 2]
    assert abs(rows[0]["total_per_node"] - 4.0e6) < 1e-6
    assert abs(rows[1]["total_per_node"] - 2.0e6) < 1e-6
    assert abs(rows[0]["us"] - 1200.0) < 1e-9 and abs(rows[1]["us"] - 1100.0) < 1e-9
    assert bpn == 3.0e6
    text = (prof / "wave_electrode256.md").read_text()
    assert "kernel_source_sha256_16: abc" in text and "dram_bytes_per_node: 3000000.00" in text
    assert text.count("kernel_source_sha256_16") == 1 and text.startswith("# summary")
