"""16-bit population storage (an offset f_i - w_i rho_ref kept as half or
bfloat16, float32 arithmetic): codec exactness, one-step parity with the
oracle, and the error of the paper's observables against the FP64 oracle.
Storages: "f16"/"bf16" offset from a constant rho0 per component; "f16l"/
"bf16l" offset from the density of the node that wrote the population.  The
measured errors are written to $HMCSC_PRECISION_OUT (JSON) when that
variable is set.

Tolerances follow from the storage precision: a stored offset d carries an
absolute rounding error of at most 2^-11 |d| (half) or 2^-8 |d| (bfloat16).
The observables' tolerances are about three times the errors measured on a
GB300 (MEASURED below; the runs are deterministic), so a regression of the
storage error by a factor of three or more fails.
"""
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2206_11524_gb300 import build, lbm, params, synth

pytestmark = pytest.mark.gpu

EPS = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8, "f16l": 2.0 ** -11,
       "bf16l": 2.0 ** -8}
CX = np.array([0, -1, 0, 0, -1, -1, -1, -1, 0, 0, 1, 0, 0, 1, 1, 1, 1, 0, 0])
CY = np.array([0, 0, -1, 0, -1, 1, 0, 0, -1, -1, 0, 1, 0, 1, -1, 0, 0, 1, 1])
CZ = np.array([0, 0, 0, -1, 0, 0, -1, 1, -1, 1, 0, 0, 1, 0, 0, 1, -1, 1, -1])
W = np.array([1 / 3] + [1 / 18] * 3 + [1 / 36] * 6 + [1 / 18] * 3 + [1 / 36] * 6,
             dtype=np.float32)
RESULTS = {}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    lbm.load()
    oracle.build()
    yield
    out = os.environ.get("HMCSC_PRECISION_OUT")
    if out and RESULTS:
        with open(out, "w") as fh:
            json.dump(RESULTS, fh, indent=1, sort_keys=True)


def w64(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _bf16_round(x32):
    """float32 -> bfloat16 (round to nearest even) -> float32, bit exact."""
    b = np.asarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32)


def _codec(storage, f, rho0):
    f = f.astype(np.float32)
    if storage.endswith("l"):
        # reference of population i of x: w_i times x's own density, the
        # state's densities summed in direction order
        rho = np.zeros((2,) + f.shape[2:], dtype=np.float32)
        for i in range(19):
            rho = (rho + f[:, i]).astype(np.float32)
        ref = (W[None, :, None, None, None] * rho[:, None]).astype(np.float32)
    else:
        ref = (W[None, :, None, None, None] *
               np.array(rho0, dtype=np.float32)[:, None, None, None, None]).astype(np.float32)
    d = (f - ref).astype(np.float32)
    if storage.startswith("f16"):
        # half offsets are kept scaled by 2^14 (exact power of two)
        q = (d * np.float32(16384.0)).astype(np.float16).astype(np.float32) \
            * np.float32(1.0 / 16384.0)
    else:
        q = _bf16_round(d)
    return (ref + q).astype(np.float32)


@pytest.mark.parametrize("storage", ["f16", "bf16", "f16l", "bf16l"])
def test_codec_is_offset_then_round_to_nearest(storage):
    shape = (3, 4, 37)
    rho0 = (0.7, 0.25)
    f = synth.random_state(shape, 5).astype(np.float32)
    g = lbm.Lattice(37, 4, 3, storage=storage, rho0=rho0)
    g.set_geometry(np.zeros(shape))
    g.set_populations(f)
    assert np.array_equal(g.populations(), _codec(storage, f, rho0))
    g.close()


@pytest.mark.parametrize("storage", ["f16", "bf16", "f16l", "bf16l"])
def test_one_step_parity_on_the_stored_state(storage):
    """From the same (decoded) state, one and two steps agree with the
    oracle up to the rounding of the stored offsets of the result."""
    shape = (4, 6, 40)
    ns, gads = synth.random_geometry(shape, 7)
    rho0 = (0.8, 0.2)
    rho_a = np.full(shape, 0.8) + 0.1 * np.random.default_rng(1).standard_normal(shape) ** 2
    rho_b = np.full(shape, 0.2)
    g = lbm.Lattice(40, 6, 4, tau=(0.9, 1.2), G=1.75, F_ext=(1e-5, 0, 0),
                    storage=storage, rho0=rho0)
    g.set_geometry(ns, gads)
    g.init_equilibrium(rho_a, rho_b)
    f0 = g.populations().astype(np.float64)
    p = oracle.Params(40, 6, 4, tau=(float(np.float32(0.9)), float(np.float32(1.2))),
                      G=1.75, Fext=(float(np.float32(1e-5)), 0, 0))
    r = oracle.Sim(p, w64(ns), w64(gads))
    r.set_populations(f0)
    for k in (1, 2):
        prev_rho = r.f.sum(axis=1)
        g.step(1)
        r.step(1)
        if storage.endswith("l"):
            # offsets from the owner's previous rest equilibrium: bounded by
            # the deviation of each population from w_i rho(t - 1)
            ref = W[None, :, None, None, None] * prev_rho[:, None]
        else:
            ref = W[None, :, None, None, None] * np.array(rho0)[:, None, None, None, None]
        bound = 4 * EPS[storage] * np.abs(r.f - ref).max() + 2e-6 * np.abs(r.f).max()
        assert np.abs(g.populations() - r.f).max() <= bound, k
    g.close()


# Errors against the FP64 oracle measured on a GB300 (every launch form
# gives the same bits): relative error of the Eq. 2 permeability, relative
# error of the droplet's Laplace pressure jump, L-infinity error of the
# S_1(t) curve of the 48^3 electrode.
MEASURED = {
    "permeability": {"f32": 1.67e-3, "f16": 1.67e-3, "bf16": 1.68e-3, "f16l": 1.67e-3,
                     "bf16l": 8.35e-4},
    "laplace": {"f32": 4.52e-6, "f16": 0.121, "bf16": 0.603, "f16l": 6.41e-5,
                "bf16l": 2.16e-3},
    "sat1": {"f32": 0.0, "f16": 1.13e-3, "bf16": 6.52e-3, "f16l": 4.83e-5, "bf16l": 2.11e-4},
}


def _tol(study, storage, floor=0.0):
    """Three times the measured error (at least `floor`)."""
    return max(3.0 * MEASURED[study][storage], floor)


def _permeability(storage, ns=0.3, n=16, steps=400):
    F = 1e-5
    shape = (n, n, n)
    g = lbm.Lattice(n, n, n, tau=(1.0, 1.0), G=0.0, F_ext=(F, 0, 0),
                    storage=storage, rho0=(0.99, 0.01))
    g.set_geometry(np.full(shape, ns))
    g.init_equilibrium(np.full(shape, 0.99), np.full(shape, 0.01))
    g.step(steps)
    fl = g.fields()
    rho_u = float((fl["u"][0].astype(np.float64)
                   * (fl["rho_a"] + fl["rho_b"])).mean())
    g.close()
    return params.viscosity(1.0) * rho_u / F


def test_permeability_error_by_storage():
    """Eq. 8 on a uniform gray medium (n_s = 0.3, F = 1e-5 as in Sec. 3.1)
    against Eq. 2, exact for the scheme.  The Darcy velocity is 1.2e-5, so
    float32 itself carries ~2e-3 (the momentum of populations ~0.05 is
    resolved to ~1e-8 per node)."""
    exact = params.permeability(0.3)
    for st in ("f32", "f16", "bf16", "f16l", "bf16l"):
        k = _permeability(st)
        err = abs(k / exact - 1)
        RESULTS[f"permeability_rel_err_{st}"] = err
        assert err < _tol("permeability", st), (st, k, exact)


def _droplet_dp(fields, n, R):
    c = n / 2 - 0.5
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    p = fields["p"]
    return float(p[r < R / 2].mean() - p[r > R + 8].mean())


def test_laplace_pressure_jump_by_storage():
    """A 3D droplet (48^3, R = 10, G = 1.75, n_s = 0.3) after 1500 steps: the
    pressure jump of each storage against the FP64 oracle."""
    n, R, steps = 48, 10.0, 1500
    case = synth.droplet(n=n, radius=R, ns=0.3, hi=0.98739, lo=0.03548)
    p = oracle.Params(n, n, n, tau=(1.0, 1.0), G=1.75)
    r = oracle.Sim(p, w64(case.ns), w64(case.gads2))
    r.init_equilibrium(w64(case.rho_a), w64(case.rho_b))
    r.step(steps)
    dp_ref = _droplet_dp(r.fields(), n, R)
    for st in ("f32", "f16", "bf16", "f16l", "bf16l"):
        g = lbm.Lattice(n, n, n, tau=(1.0, 1.0), G=1.75, storage=st, rho0=(0.5, 0.5))
        g.set_geometry(case.ns, case.gads2)
        g.init_equilibrium(case.rho_a, case.rho_b)
        g.step(steps)
        dp = _droplet_dp(g.fields(), n, R)
        g.close()
        err = abs(dp / dp_ref - 1)
        RESULTS[f"laplace_dp_rel_err_{st}"] = err
        assert err < _tol("laplace", st), (st, dp, dp_ref)
    RESULTS["laplace_dp_oracle"] = dp_ref


def test_saturation_curve_by_storage():
    """Imbibition into a 48^3 synthetic electrode: S_1(t) every 100 steps for
    1500 steps; float32 against the oracle, 16-bit storages against the
    oracle as well (L-infinity over the curve)."""
    n, steps, every = 48, 1500, 100
    case = synth.electrode((n, n, n), seed=11)
    p = oracle.Params(n, n, n, tau=case.tau, G=case.G, reservoirs=case.reservoirs)
    r = oracle.Sim(p, w64(case.ns), w64(case.gads2))
    r.init_equilibrium(w64(case.rho_a), w64(case.rho_b))
    ref = []
    for _ in range(steps // every):
        r.step(every)
        ref.append(r.observables()["sat1"])
    ref = np.array(ref)
    # float32 (measured: no difference) may put a couple of nodes within
    # float32 rounding of rho_1 = 0.5 on the other side: two nodes' weight
    inner = np.zeros(case.shape, bool)
    inner[..., 4:n - 4] = True
    two_nodes = 2.0 / float((1.0 - w64(case.ns))[inner].sum())
    for st in ("f32", "f16", "bf16", "f16l", "bf16l"):
        tol = _tol("sat1", st, floor=two_nodes)
        g = lbm.Lattice(n, n, n, tau=case.tau, G=case.G, storage=st, rho0=(0.5, 0.5))
        g.set_geometry(case.ns, case.gads2)
        for face, (L, a, b) in case.reservoirs.items():
            g.set_bc(face, L, a, b)
        g.init_equilibrium(case.rho_a, case.rho_b)
        cur = []
        for _ in range(steps // every):
            g.step(every)
            cur.append(g.observables()["sat1"])
        g.close()
        err = float(np.abs(np.array(cur) - ref).max())
        RESULTS[f"sat1_linf_err_{st}"] = err
        assert err < tol, (st, err)
    RESULTS["sat1_final_oracle"] = float(ref[-1])
