"""FP64 CPU oracle of the HMCSC D3Q19 step (arXiv 2206.11524).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It is
the plain, slow statement of the method (``hmcsc_oracle.c``, compiled with gcc
``-O2 -ffp-contract=off``) against which the CUDA library is checked; it shares
no code with that library and the library never falls back to it.

Every array here is float64 numpy in the layout of the paper's lattice:
populations ``f[sigma, i, z, y, x]`` (sigma = fluid 1 / fluid 2, i in the
D3Q19 order of Eq. A.8), scalar fields ``[z, y, x]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hmcsc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

Q = 19
FACES = ("-x", "+x", "-y", "+y", "-z", "+z")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction, so FP64 rounding is the
    plain IEEE rounding of each written operation)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("tau", ctypes.c_double * 2),
        ("G", ctypes.c_double),
        ("Fext", ctypes.c_double * 3),
        ("res_layers", ctypes.c_int * 6),
        ("res_rho", (ctypes.c_double * 2) * 6),
        ("res_u", (ctypes.c_double * 3) * 6),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        lib.orc_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), dp,
                                    ctypes.POINTER(ctypes.c_int)]
        lib.orc_feq.argtypes = [ctypes.c_double, dp, dp]
        lib.orc_init_equilibrium.argtypes = [pp, dp, dp, dp]
        lib.orc_step.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        lib.orc_run.argtypes = [pp, dp, dp, dp, dp, dp, dp, ctypes.c_int]
        lib.orc_fields.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_observables.argtypes = [pp, dp, dp, dp, dp]
        lib.orc_observables_rho.argtypes = [pp, dp, dp, dp]
        for name in ("orc_lattice", "orc_feq", "orc_init_equilibrium",
                     "orc_step", "orc_run", "orc_fields", "orc_observables",
                     "orc_observables_rho"):
            getattr(lib, name).restype = None
        _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def observables_of_densities(params: Params, ns, rho_a, rho_b):
    """The observables of Sec. 4 (masses, S_1 of Eq. 19, reservoir mean
    pressures of Eq. A.6) of given density fields [nz, ny, nx], with n_s,1 =
    ns weighting S_1: the second half of Sim.observables, for densities
    that do not come from an oracle state."""
    shape = (params.nz, params.ny, params.nx)
    rho = np.ascontiguousarray(np.stack([np.asarray(rho_a, np.float64).reshape(shape),
                                         np.asarray(rho_b, np.float64).reshape(shape)]))
    ns_c = np.ascontiguousarray(np.asarray(ns, np.float64).reshape(shape))
    out = np.zeros(9)
    cp = params.c_struct()
    _load().orc_observables_rho(ctypes.byref(cp), _ptr(ns_c), _ptr(rho), _ptr(out))
    return {"mass": out[0:2].copy(), "sat1": float(out[2]), "p_face": out[3:9].copy()}


def lattice():
    """(c[19,3] int, w[19] float64, opp[19] int) as the oracle holds them."""
    lib = _load()
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    lib.orc_lattice(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(w),
                    opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return c, w, opp


def feq(rho: float, u) -> np.ndarray:
    """Maxwell-Boltzmann equilibrium f^eq_i(rho, u), Eq. A.3."""
    out = np.zeros(Q)
    uu = np.ascontiguousarray(u, dtype=np.float64)
    _load().orc_feq(float(rho), _ptr(uu), _ptr(out))
    return out


@dataclass
class Params:
    """Model parameters (Table 1 names).  ``reservoirs`` maps a face index
    (0..5 = -x,+x,-y,+y,-z,+z) to (layers, rho_1, rho_2) -- a density
    reservoir at rest -- or (layers, rho_1, rho_2, (ux, uy, uz)) -- boundary
    cells held at that velocity."""
    nx: int
    ny: int
    nz: int
    tau: tuple = (1.0, 1.0)
    G: float = 1.75
    Fext: tuple = (0.0, 0.0, 0.0)
    reservoirs: dict = field(default_factory=dict)

    def c_struct(self) -> _Params:
        p = _Params()
        p.nx, p.ny, p.nz = self.nx, self.ny, self.nz
        p.tau[0], p.tau[1] = self.tau
        p.G = self.G
        for d in range(3):
            p.Fext[d] = self.Fext[d]
        for k in range(6):
            entry = self.reservoirs.get(k, (0, 0.0, 0.0))
            layers, r1, r2 = entry[:3]
            u = entry[3] if len(entry) > 3 else (0.0, 0.0, 0.0)
            p.res_layers[k] = layers
            p.res_rho[k][0] = r1
            p.res_rho[k][1] = r2
            for d in range(3):
                p.res_u[k][d] = u[d]
        return p


class Sim:
    """Oracle simulation state.  Inputs are float64 arrays [nz, ny, nx].

    ``ns`` is the bounce-back fraction of Eq. 1: one field [nz, ny, nx] for
    both components, or one per component [2, nz, ny, nx] (n_s,sigma)."""

    def __init__(self, params: Params, ns, gads2=None):
        self.p = params
        self._cp = params.c_struct()
        shape = (params.nz, params.ny, params.nx)
        ns = np.asarray(ns, dtype=np.float64)
        if ns.ndim == 4:
            self.ns_c = np.ascontiguousarray(ns.reshape((2,) + shape))
        else:
            one = ns.reshape(shape)
            self.ns_c = np.ascontiguousarray(np.stack([one, one]))
        self.ns = self.ns_c[0]
        if gads2 is None:
            gads2 = np.zeros(shape)
        self.gads2 = np.ascontiguousarray(gads2, dtype=np.float64).reshape(shape)
        self.N = params.nx * params.ny * params.nz
        self.f = np.zeros((2, Q) + shape)
        self._tmp = np.zeros_like(self.f)
        self._post = np.zeros_like(self.f)
        self._rho = np.zeros((2,) + shape)
        self.t = 0

    def init_equilibrium(self, rho_a, rho_b):
        shape = self.ns.shape
        ra = np.ascontiguousarray(rho_a, dtype=np.float64).reshape(shape)
        rb = np.ascontiguousarray(rho_b, dtype=np.float64).reshape(shape)
        _load().orc_init_equilibrium(ctypes.byref(self._cp), _ptr(ra), _ptr(rb),
                                     _ptr(self.f))
        self.t = 0

    def set_reservoirs(self, reservoirs: dict):
        """Change the reservoir faces; the new values reset the layers at the
        end of the next step (an inlet density ramp, Sec. 4)."""
        self.p.reservoirs = dict(reservoirs)
        self._cp = self.p.c_struct()

    def set_populations(self, f):
        self.f[...] = np.asarray(f, dtype=np.float64).reshape(self.f.shape)

    def step(self, n: int = 1):
        if n > 0:
            _load().orc_run(ctypes.byref(self._cp), _ptr(self.ns_c),
                            _ptr(self.gads2), _ptr(self.f), _ptr(self._tmp),
                            _ptr(self._rho), _ptr(self._post), int(n))
        self.t += n

    def fields(self):
        """dict with rho_a, rho_b [nz,ny,nx], u [3,nz,ny,nx] (Eq. 7),
        p (Eq. A.6) and ftot [2,3,nz,ny,nx] (Eqs. 3-5)."""
        shape = self.ns.shape
        out = {"rho_a": np.zeros(shape), "rho_b": np.zeros(shape),
               "u": np.zeros((3,) + shape), "p": np.zeros(shape),
               "ftot": np.zeros((2, 3) + shape)}
        _load().orc_fields(ctypes.byref(self._cp), _ptr(self.ns_c),
                           _ptr(self.gads2), _ptr(self.f), _ptr(self._rho),
                           _ptr(out["rho_a"]), _ptr(out["rho_b"]),
                           _ptr(out["u"]), _ptr(out["p"]), _ptr(out["ftot"]))
        return out

    def observables(self):
        """dict: mass (2,), sat1, p_face (6,) -- Sec. 4, Eqs. 18-19."""
        out = np.zeros(9)
        _load().orc_observables(ctypes.byref(self._cp), _ptr(self.ns_c),
                                _ptr(self.f), _ptr(self._rho), _ptr(out))
        return {"mass": out[0:2].copy(), "sat1": float(out[2]),
                "p_face": out[3:9].copy()}
