"""Validation studies on the GPU path at the paper's workload sizes.

`laplace`     static droplets in homogeneous gray media (Sec. 3.3): the
              pressure jump of Eq. A.6 against 1/R for several radii and
              solid fractions; the slope of the fit is 2 gamma (3D Laplace
              law), and gamma should not depend on n_s.
`saturation`  imbibition into the synthetic electrode (Sec. 4): the
              saturation curve S_1(t) of Eq. 19 for several population
              storages, each against the float32 run of the same case.
`relperm`     relative permeabilities of two immiscible fluids in a
              homogeneous gray medium (Sec. 3.1, Eqs. 9-10): stratified
              layers of fluid 1 and fluid 2 along the body force.
`washburn`    capillary imbibition into a homogeneous gray medium (Sec. 3.4,
              Eq. 16, Table 3): the front position against time for the
              paper's G_ads and n_s series, fitted as x = A sqrt(B t).
`buckley_leverett`  waterflooding of a homogeneous gray medium (SI,
              Buckley-Leverett experiment): saturation profiles and front
              displacement against the Buckley-Leverett solution with
              k_r = S^a and (1 - S)^a for the paper's bounds a = 1.01, 1.3.
`serving`     a stream of independent imbibition requests of different
              sizes, microstructures and wettabilities: continuous batching
              in 16-bit storage against one-at-a-time float32 runs (p50 / p99
              time to result, aggregate MLUPS).

Run as ``python -m paper_2206_11524_gb300.studies <study> [options]``; the
result is printed and written as JSON to ``--out``.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import lbm, synth

# Flat-interface coexistence densities at G = 1.75 (both tau = 1), used as
# the droplet's inner / outer densities so it starts near equilibrium.
COEXIST_175 = (0.98739, 0.03548)


def droplet_radius(rho_a):
    """Equivalent radius of the fluid-1 droplet: its volume is the sum of the
    fluid-1 density normalised between the extreme values, R = (3V/4pi)^1/3."""
    lo, hi = float(rho_a.min()), float(rho_a.max())
    vol = float(((rho_a.astype(np.float64) - lo) / (hi - lo)).sum())
    return (3.0 * vol / (4.0 * math.pi)) ** (1.0 / 3.0)


def pressure_jump(p, R, margin=10.0):
    """Mean pressure inside r < R/2 minus the mean over the nodes farther than
    R + margin from the centre of the (centred) droplet."""
    n = p.shape[0]
    c = n / 2 - 0.5
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij", sparse=True)
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    inner = r < R / 2
    outer = r > R + margin
    return float(p[inner].mean() - p[outer].mean())


def laplace(n=128, radii=(10, 15, 20, 25, 30), ns_values=(0.0, 0.3, 0.6),
            steps=20000, G=1.75, storage="f32"):
    rows = []
    for ns in ns_values:
        for R0 in radii:
            case = synth.droplet(n=n, radius=float(R0), ns=ns, G=G,
                                 hi=COEXIST_175[0], lo=COEXIST_175[1])
            lat = lbm.Lattice(n, n, n, tau=(1.0, 1.0), G=G, storage=storage,
                              rho0=(0.5, 0.5))
            lat.set_geometry(case.ns)
            lat.init_equilibrium(case.rho_a, case.rho_b)
            lat.step(steps)
            fl = lat.fields()
            obs = lat.observables()
            lat.close()
            R = droplet_radius(fl["rho_a"])
            dp = pressure_jump(fl["p"], R)
            rows.append({"ns": ns, "R0": R0, "R": R, "dp": dp,
                         "gamma_R": dp * R / 2.0,
                         "max_u": float(np.abs(fl["u"]).max()),
                         "mass": list(map(float, obs["mass"]))})
    fits = {}
    for ns in ns_values:
        sel = [r for r in rows if r["ns"] == ns]
        inv = np.array([1.0 / r["R"] for r in sel])
        dp = np.array([r["dp"] for r in sel])
        A = np.stack([inv, np.ones_like(inv)], axis=1)
        (slope, icpt), *_ = np.linalg.lstsq(A, dp, rcond=None)
        pred = A @ np.array([slope, icpt])
        ss_res = float(((dp - pred) ** 2).sum())
        ss_tot = float(((dp - dp.mean()) ** 2).sum())
        fits[str(ns)] = {"gamma": slope / 2.0, "intercept": float(icpt),
                         "r2": 1.0 - ss_res / ss_tot if ss_tot > 0 else 1.0,
                         "gamma_largest_R": max(sel, key=lambda r: r["R"])["gamma_R"]}
    g = [f["gamma"] for f in fits.values()]
    return {"study": "laplace", "n": n, "steps": steps, "G": G, "storage": storage,
            "rows": rows, "fits": fits,
            "gamma_spread_rel": (max(g) - min(g)) / float(np.mean(g))}


def _s1_curve(case, storage, steps, every):
    import torch
    nz, ny, nx = case.shape
    lat = lbm.Lattice(nx, ny, nz, tau=case.tau, G=case.G, storage=storage,
                      rho0=(0.5, 0.5))
    lat.set_geometry(case.ns, case.gads2)
    for face, (L, a, b) in case.reservoirs.items():
        lat.set_bc(face, L, a, b)
    lat.init_equilibrium(case.rho_a, case.rho_b)
    curve, t_step = [], 0.0
    for _ in range(steps // every):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.step(every)
        torch.cuda.synchronize()
        t_step += time.perf_counter() - t0
        curve.append(lat.observables()["sat1"])
    lat.close()
    return np.array(curve), case.n_nodes * steps / t_step / 1e6


def saturation(shape=(256, 256, 256), storages=("f32", "f16", "bf16", "f16l", "bf16l"),
               steps=50000, every=1000, seed=2206):
    nx, ny, nz = shape
    case = synth.electrode((nz, ny, nx), seed=seed)
    out = {"study": "saturation", "shape": [nx, ny, nz], "steps": steps,
           "every": every, "curves": {}, "linf_vs_f32": {}, "mlups": {}}
    ref = None
    for st in ("f32",) + tuple(s for s in storages if s != "f32"):
        curve, mlups = _s1_curve(case, st, steps, every)
        out["curves"][st] = curve.tolist()
        out["mlups"][st] = mlups
        if ref is None:
            ref = curve
        else:
            out["linf_vs_f32"][st] = float(np.abs(curve - ref).max())
    return out


# D3Q19 x-components in the order of Eq. A.8 (for the momentum of the
# read-back populations).
_CX = np.array([0, -1, 0, 0, -1, -1, -1, -1, 0, 0, 1, 0, 0, 1, 1, 1, 1, 0, 0],
               dtype=np.float64)


def component_flux(lat, ns, F):
    """Mean x-momentum of each component with Eq. 7's weighting,
    (1 - n_s)(j_sigma + F_sigma / 2), where F_sigma = rho_sigma / rho F_ext
    along x (the fluid-fluid forces of a flat interface along the flow and
    the adhesion of a uniform medium have no mean x-component)."""
    f = lat.populations().astype(np.float64)
    rho = f.sum(axis=1)                                  # [2, nz, ny, nx]
    jx = np.tensordot(_CX, f, axes=([0], [1]))           # [2, nz, ny, nx]
    share = rho / rho.sum(axis=0)
    return [(1.0 - ns) * float((jx[k] + 0.5 * share[k] * F).mean()) for k in range(2)]


def relperm(n=50, ns_values=(0.1, 0.5, 0.9), saturations=(0.0, 0.2, 0.4, 0.6, 0.8, 1.0),
            steps=3000, F=1e-5, G=1.75):
    """k_r,sigma(S_1) = k(S_sigma) / k(S_sigma = 1), k = nu <rho_sigma u_sigma>
    / F_ext (Eqs. 9-10), for stratified layers (fluid 1 in the first S_1 n
    rows) driven along x, n x n x 1 lattice, tau = 1, G_ads = 0."""
    nu = 1.0 / 6.0
    hi, lo = COEXIST_175
    out = {"study": "relperm", "n": n, "steps": steps, "rows": []}
    for ns in ns_values:
        flux = {}
        for S in saturations:
            shape = (1, n, n)
            rows1 = int(round(S * n))
            y = np.arange(n)[None, :, None] * np.ones(shape)
            ra = np.where(y < rows1, hi, lo)
            lat = lbm.Lattice(n, n, 1, tau=(1.0, 1.0), G=G, F_ext=(F, 0.0, 0.0))
            lat.set_geometry(np.full(shape, ns))
            lat.init_equilibrium(ra, hi + lo - ra)
            lat.step(steps)
            flux[S] = component_flux(lat, ns, F)
            lat.close()
        k1_full, k2_full = nu * flux[1.0][0] / F, nu * flux[0.0][1] / F
        for S in saturations:
            out["rows"].append({"ns": ns, "S1": S,
                                "kr1": nu * flux[S][0] / F / k1_full,
                                "kr2": nu * flux[S][1] / F / k2_full,
                                "k_single": k1_full})
    return out


def washburn_setup(gads, ns, H=500, storage="f32"):
    """Imbibition along x through H lu: an inlet reservoir of fluid 1
    (x = 0..3), uniform gray medium (n_s, G_ads) in between, an outlet
    reservoir of fluid 2 (x = H-4..H-1), the reservoir layers free of
    medium; uniform across y, so one row (periodic) suffices.  This reads the
    paper's set-up (Sec. 3.4), whose axes are garbled in the text."""
    x = np.arange(H)
    medium = (x >= 4) & (x < H - 4)
    lat = lbm.Lattice(H, 1, 1, tau=(1.0, 1.0), G=1.75, storage=storage,
                      rho0=(0.5, 0.5))
    lat.set_geometry(np.where(medium, ns, 0.0)[None, None],
                     np.where(medium, gads, 0.0)[None, None])
    lat.set_bc(0, 4, 0.99, 0.01)
    lat.set_bc(1, 4, 0.01, 0.99)
    ra = np.where(x < 4, 0.99, 0.01)[None, None] * 1.0
    lat.init_equilibrium(ra, 1.0 - ra)
    return lat


def front_position(rho1, x0=4):
    """Where rho_1 falls through 0.5 behind the inlet (linear interpolation),
    measured from the medium's face at x0; 0 before the front enters."""
    for k in range(x0, len(rho1) - 1):
        if rho1[k] >= 0.5 > rho1[k + 1]:
            return k - x0 + 0.5 + (rho1[k] - 0.5) / (rho1[k] - rho1[k + 1])
    return 0.0


def washburn_front(gads, ns, H=500, steps=50000, samples=20):
    lat = washburn_setup(gads, ns, H)
    ts, xs = [], []
    for _ in range(samples):
        lat.step(steps // samples)
        ts.append(lat.t)
        xs.append(front_position(lat.fields()["rho_a"][0, 0]))
    lat.close()
    return np.array(ts, float), np.array(xs)


def washburn(gads_values=(0.05, 0.10, 0.15, 0.20, 0.25, 0.30, 0.35, 0.40),
             ns_values=(0.1, 0.5, 0.9), H=500, steps=50000):
    """Table 3's two series: n_s = 0.5 with G_ads varied, and G_ads = 0.2
    with n_s varied.  Eq. 16 squared, x^2 = A^2 B t, is fitted through the
    origin (a = A^2 B); the paper holds B in the first series and A in the
    second, so both a and R^2 (of x against sqrt(a t)) are reported."""
    out = {"study": "washburn", "H": H, "steps": steps, "gads_series": [],
           "ns_series": []}

    def fit(ts, xs):
        a = float((xs ** 2) @ ts / (ts @ ts))
        r2 = 1 - float(((xs - np.sqrt(a * ts)) ** 2).sum() / ((xs - xs.mean()) ** 2).sum())
        return a, r2

    for g in gads_values:
        ts, xs = washburn_front(g, 0.5, H, steps)
        a, r2 = fit(ts, xs)
        out["gads_series"].append({"gads": g, "ns": 0.5, "a": a, "r2": r2,
                                   "x_final": float(xs[-1])})
    for n in ns_values:
        ts, xs = washburn_front(0.2, n, H, steps)
        a, r2 = fit(ts, xs)
        out["ns_series"].append({"gads": 0.2, "ns": n, "a": a, "r2": r2,
                                 "x_final": float(xs[-1])})
    return out


# ---- Buckley-Leverett waterflooding (SI) ----
#
# Set-up as read from the text (whose axes are garbled: it drives the flow
# with a body force along the periodic axis while the inlet and outlet sit
# at the ends of the other): displacement along x through H lu, the body
# force 1e-4 along x, fluid 1 held at the inlet layers x = 0..3 and fluid 2
# at the outlet layers, every cell (reservoir layers included) with the same
# n_s and G_ads = 0, the domain W lu wide and periodic across y.  The
# reservoirs hold the flat-interface coexistence densities at G = 1.75, so
# the fluids enter as the bulk phases they are in the medium.  Saturation of
# fluid 1 is rho_1 normalised between those densities; with both fluids
# carried in full by every homogenized cell the porosity of the mass balance
# is 1, and the flux q of the Buckley-Leverett equation is the mean x
# velocity of Eq. 7 over the medium.


def bl_fractional_flow(S, a):
    """f(S) = (1 + k_r2 / k_r1)^-1 with k_r1 = S^a, k_r2 = (1 - S)^a."""
    S = np.asarray(S, dtype=np.float64)
    return S ** a / (S ** a + (1.0 - S) ** a)


def bl_dfds(S, a):
    """df/dS of bl_fractional_flow."""
    S = np.asarray(S, dtype=np.float64)
    d = S ** a + (1.0 - S) ** a
    return a * S ** (a - 1) * (1.0 - S) ** (a - 1) / d ** 2


def bl_welge(a):
    """Shock saturation S_f and shock speed factor f(S_f)/S_f of Welge's
    tangent from the initial state S = 0: the S where f(S)/S = f'(S)
    (bisection; S f' - f is positive near 0 and -1 at S = 1 for a > 1)."""
    lo, hi = 1e-9, 1.0 - 1e-12
    g = lambda S: float(S * bl_dfds(S, a) - bl_fractional_flow(S, a))
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0:
            lo = mid
        else:
            hi = mid
    Sf = 0.5 * (lo + hi)
    return Sf, float(bl_fractional_flow(Sf, a)) / Sf


def bl_profile(x, Q, a, phi=1.0):
    """Buckley-Leverett saturation at distance x from the inlet after an
    injected volume Q per unit area: S travels at (Q / phi) f'(S) for S in
    [S_f, 1] (f' falls monotonically there), S = 0 ahead of the shock at
    (Q / phi) f(S_f) / S_f."""
    Sf, speed = bl_welge(a)
    S = np.linspace(Sf, 1.0, 20001)
    xs = (Q / phi) * bl_dfds(S, a)          # decreasing in S
    x = np.asarray(x, dtype=np.float64)
    out = np.interp(x, xs[::-1], S[::-1])   # 1 behind the slowest, S_f at the shock
    return np.where(x >= (Q / phi) * speed, 0.0, out)


def bl_setup(ns, H=100, W=5, F=1e-4, storage="f32"):
    hi, lo = COEXIST_175
    x = np.arange(H)
    lat = lbm.Lattice(H, W, 1, tau=(1.0, 1.0), G=1.75, F_ext=(F, 0, 0), storage=storage,
                      rho0=(0.5, 0.5))
    lat.set_geometry(np.full((1, W, H), ns))
    lat.set_bc(0, 4, hi, lo)
    lat.set_bc(1, 4, lo, hi)
    ra = np.broadcast_to(np.where(x < 4, hi, lo), (1, W, H)).astype(np.float64)
    lat.init_equilibrium(ra, hi + lo - ra)
    return lat


def bl_saturation(rho1):
    hi, lo = COEXIST_175
    return (np.asarray(rho1, dtype=np.float64) - lo) / (hi - lo)


def bl_front(S, x0=4):
    """Where S falls through 0.5 behind the inlet (linear interpolation),
    as an x coordinate; x0 before the front enters."""
    for k in range(x0, len(S) - 1):
        if S[k] >= 0.5 > S[k + 1]:
            return k + (S[k] - 0.5) / (S[k] - S[k + 1])
    return float(x0)


def bl_run(ns, H=100, W=5, steps=200000, samples=40, storage="f32"):
    """Sample times, front positions, injected volume Q(t) (trapezoid over
    the samples of the mean velocity of the medium) and the last profile
    S(x) (mean over y)."""
    lat = bl_setup(ns, H, W, storage=storage)
    ts, fronts, Q = [0], [4.0], [0.0]
    q_prev = 0.0
    for _ in range(samples):
        lat.step(steps // samples)
        fl = lat.fields()
        S = bl_saturation(fl["rho_a"][0].mean(axis=0))
        q = float(fl["u"][0][0][:, 4:H - 4].astype(np.float64).mean())
        Q.append(Q[-1] + 0.5 * (q + q_prev) * (lat.t - ts[-1]))
        q_prev = q
        ts.append(lat.t)
        fronts.append(bl_front(S))
    lat.close()
    return np.array(ts, float), np.array(fronts), np.array(Q), S


def buckley_leverett(ns_values=(0.1, 0.5, 0.9), H=100, W=5, steps=200000, samples=40,
                     bounds=(1.01, 1.3)):
    """Per n_s: the front displacement over the last four fifths of the run,
    the injected volume in that time and their ratio (the shock speed factor
    f(S_f)/S_f of the Buckley-Leverett solution, to be compared with the
    bounds'), and the final profile against the two bounds' profiles at the
    measured injected volume (the inlet face at x = 4)."""
    out = {"study": "buckley_leverett", "H": H, "W": W, "steps": steps,
           "bounds": {str(a): dict(zip(("S_f", "speed"), bl_welge(a))) for a in bounds},
           "runs": []}
    for ns in ns_values:
        ts, fr, Q, S = bl_run(ns, H, W, steps, samples)
        k0 = samples // 5
        dQ = float(Q[-1] - Q[k0])
        ratio = float((fr[-1] - fr[k0]) / dQ) if dQ > 0 else float("nan")
        x = np.arange(H) - 4.0
        prof = {str(a): bl_profile(x, float(Q[-1]), a).tolist() for a in bounds}
        out["runs"].append({"ns": ns, "front": float(fr[-1]), "Q": float(Q[-1]),
                            "shift": float(fr[-1] - fr[k0]), "dQ": dQ,
                            "speed_ratio": ratio, "profile": S.tolist(),
                            "bound_profiles": prof})
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="study", required=True)
    a = sub.add_parser("laplace")
    a.add_argument("--n", type=int, default=128)
    a.add_argument("--steps", type=int, default=20000)
    a.add_argument("--radii", default="10,15,20,25,30")
    a.add_argument("--ns", default="0,0.3,0.6")
    a.add_argument("--out", default="")
    b = sub.add_parser("saturation")
    b.add_argument("--shape", default="256,256,256")
    b.add_argument("--steps", type=int, default=50000)
    b.add_argument("--every", type=int, default=1000)
    b.add_argument("--storages", default="f32,f16,bf16,f16l,bf16l")
    b.add_argument("--out", default="")
    e = sub.add_parser("washburn")
    e.add_argument("--steps", type=int, default=50000)
    e.add_argument("--out", default="")
    d = sub.add_parser("relperm")
    d.add_argument("--n", type=int, default=50)
    d.add_argument("--steps", type=int, default=3000)
    d.add_argument("--out", default="")
    f = sub.add_parser("buckley_leverett")
    f.add_argument("--steps", type=int, default=200000)
    f.add_argument("--out", default="")
    c = sub.add_parser("serving")
    c.add_argument("--requests", type=int, default=256)
    c.add_argument("--lmin", type=int, default=32)
    c.add_argument("--lmax", type=int, default=192)
    c.add_argument("--steps-min", type=int, default=5000)
    c.add_argument("--steps-max", type=int, default=40000)
    c.add_argument("--storage", default="f16l")
    c.add_argument("--load", type=float, default=0.9)
    c.add_argument("--out", default="")
    args = ap.parse_args(argv)
    from . import build
    build.build()
    lbm.load()
    if args.study == "laplace":
        res = laplace(n=args.n, steps=args.steps,
                      radii=tuple(int(v) for v in args.radii.split(",")),
                      ns_values=tuple(float(v) for v in args.ns.split(",")))
    elif args.study == "washburn":
        res = washburn(steps=args.steps)
    elif args.study == "relperm":
        res = relperm(n=args.n, steps=args.steps)
    elif args.study == "buckley_leverett":
        res = buckley_leverett(steps=args.steps)
    elif args.study == "saturation":
        res = saturation(shape=tuple(int(v) for v in args.shape.split(",")),
                         storages=tuple(args.storages.split(",")),
                         steps=args.steps, every=args.every)
    else:
        from . import serve
        res = serve.compare(n_req=args.requests, L_min=args.lmin, L_max=args.lmax,
                            steps_min=args.steps_min, steps_max=args.steps_max,
                            storage=args.storage, load=args.load)
        res["study"] = "serving"
    text = json.dumps(res, indent=1)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(text)
    summary = {k: v for k, v in res.items() if k not in ("rows", "curves", "runs")}
    print(json.dumps(summary))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
