"""ctypes binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

The functions here carry the C names (``lbm_create``, ``lbm_step`` ...) and
take the same arguments; every step of the computation runs in the CUDA
library.  ``Lattice`` is a thin convenience wrapper that allocates the device
workspace as a PyTorch tensor and passes PyTorch's current stream.

If the compiled library is missing the import fails loudly: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENAN, LBM_ETIMEOUT, \
    LBM_ESTATE, LBM_EINTERNAL, LBM_ETOOLARGE = range(9)
LBM_NOALLOC_MAX_NODES = 16777216
LBM_STORAGE_F32, LBM_STORAGE_F16_OFFSET, LBM_STORAGE_BF16_OFFSET, \
    LBM_STORAGE_F16_LOCAL, LBM_STORAGE_BF16_LOCAL = range(5)
STORAGES = {"f32": LBM_STORAGE_F32, "f16": LBM_STORAGE_F16_OFFSET,
            "bf16": LBM_STORAGE_BF16_OFFSET, "f16l": LBM_STORAGE_F16_LOCAL,
            "bf16l": LBM_STORAGE_BF16_LOCAL}
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENAN",
                5: "ETIMEOUT", 6: "ESTATE", 7: "EINTERNAL", 8: "ETOOLARGE"}

#: every entry point declared in include/lbm.h
ABI_SYMBOLS = (
    "lbm_workspace_bytes", "lbm_create", "lbm_destroy", "lbm_set_geometry",
    "lbm_init_equilibrium", "lbm_set_populations", "lbm_get_populations",
    "lbm_set_bc", "lbm_step", "lbm_density", "lbm_collide_stream", "lbm_time",
    "lbm_read_fields", "lbm_reduce", "lbm_sync", "lbm_checkpoint_bytes",
    "lbm_save", "lbm_load", "lbm_last_error", "lbm_reduce_fields_noalloc",
    "lbm_batch_step", "lbm_batch_graph_create", "lbm_batch_graph_launch",
    "lbm_batch_graph_destroy", "lbm_set_launch_config",
    "lbm_set_geometry_per_component", "lbm_set_bc_velocity", "lbm_set_single_pass",
    "lbm_build_checked", "lbm_fault_word", "lbm_get_launch_config",
    "lbm_set_wavefront", "lbm_get_wavefront", "lbm_set_wavefront_limits",
)
LBM_DENSITY_CONFIGS, LBM_COLLIDE_CONFIGS = 3, 10
SINGLE_PASS_MAX_NX = 256
LBM_WAVE_SHAPES = 4
LBM_FAULT_WAIT = 128
LBM_BATCH_MAX = 64


class lbm_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("tau", ctypes.c_double * 2), ("G", ctypes.c_double),
                ("F_ext", ctypes.c_double * 3), ("rho0", ctypes.c_double * 2),
                ("ns_per_component", ctypes.c_int32)]


class lbm_observables(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double * 2), ("sat1", ctypes.c_double),
                ("p_face", ctypes.c_double * 6), ("nonfinite", ctypes.c_int64)]


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_LIBPATH = _build.LIB


def library_path() -> str:
    return _LIBPATH


def load(path: str | None = None):
    """Load the shared library (build it first with ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("HMCSC_LBM_LIBRARY") or _LIBPATH
    if not os.path.exists(path):
        raise ImportError(
            f"CUDA library not built: {path} is missing "
            "(run __graft_entry__.build() or python -m paper_2206_11524_gb300.build)")
    lib = ctypes.CDLL(path)
    vp, fp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)
    P = ctypes.POINTER(lbm_params)
    sig = {
        "lbm_workspace_bytes": (ctypes.c_size_t, [P]),
        "lbm_create": (ctypes.c_int, [P, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]),
        "lbm_destroy": (None, [vp]),
        "lbm_set_geometry": (ctypes.c_int, [vp, fp, fp]),
        "lbm_set_geometry_per_component": (ctypes.c_int, [vp, fp, fp, fp]),
        "lbm_init_equilibrium": (ctypes.c_int, [vp, fp, fp]),
        "lbm_set_populations": (ctypes.c_int, [vp, fp]),
        "lbm_get_populations": (ctypes.c_int, [vp, fp]),
        "lbm_set_bc": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
        "lbm_set_bc_velocity": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 5),
        "lbm_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_set_single_pass": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_set_wavefront": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
        "lbm_get_wavefront": (ctypes.c_int, [vp] + [ctypes.POINTER(ctypes.c_int)] * 2),
        "lbm_set_wavefront_limits": (ctypes.c_int, [vp, ctypes.c_uint32, ctypes.c_int64]),
        "lbm_build_checked": (ctypes.c_int, []),
        "lbm_get_launch_config": (ctypes.c_int, [vp] + [ctypes.POINTER(ctypes.c_int)] * 3),
        "lbm_fault_word": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]),
        "lbm_density": (ctypes.c_int, [vp]),
        "lbm_collide_stream": (ctypes.c_int, [vp]),
        "lbm_time": (ctypes.c_int64, [vp]),
        "lbm_read_fields": (ctypes.c_int, [vp, fp, fp, fp, fp]),
        "lbm_reduce": (ctypes.c_int, [vp, ctypes.POINTER(lbm_observables)]),
        "lbm_sync": (ctypes.c_int, [vp, ctypes.c_double]),
        "lbm_checkpoint_bytes": (ctypes.c_size_t, [vp]),
        "lbm_save": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
        "lbm_load": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
        "lbm_last_error": (ctypes.c_char_p, [vp]),
        "lbm_batch_step": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, vp]),
        "lbm_batch_graph_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int,
                                                  vp, ctypes.POINTER(vp)]),
        "lbm_batch_graph_launch": (ctypes.c_int, [vp, vp]),
        "lbm_batch_graph_destroy": (None, [vp]),
        "lbm_set_launch_config": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "lbm_reduce_fields_noalloc": (ctypes.c_int, [vp, vp, vp, ctypes.c_int32,
                                                     ctypes.c_int32, ctypes.c_int32,
                                                     ctypes.POINTER(ctypes.c_int32),
                                                     ctypes.c_double, vp,
                                                     ctypes.POINTER(lbm_observables)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _f32(a, n=None):
    """Contiguous float32 host array and its pointer (or NULL)."""
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float32)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


# ---- thin wrappers with the C names ---------------------------------------

def lbm_workspace_bytes(params: lbm_params) -> int:
    return load().lbm_workspace_bytes(ctypes.byref(params))


def lbm_create(params: lbm_params, d_workspace: int, workspace_bytes: int,
               cuda_stream: int) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    st = load().lbm_create(ctypes.byref(params), ctypes.c_void_p(d_workspace),
                           workspace_bytes, ctypes.c_void_p(cuda_stream),
                           ctypes.byref(ctx))
    if st != LBM_OK:
        raise LbmError(st, "lbm_create failed")
    return ctx


def _check(ctx, st):
    if st != LBM_OK:
        msg = load().lbm_last_error(ctx)
        raise LbmError(st, msg.decode() if msg else "")
    return st


def lbm_destroy(ctx):
    load().lbm_destroy(ctx)


def lbm_set_geometry(ctx, ns, gads2=None, n=None):
    a, pa = _f32(ns, n)
    b, pb = _f32(gads2, n)
    return _check(ctx, load().lbm_set_geometry(ctx, pa, pb))


def lbm_set_geometry_per_component(ctx, ns1, ns2, gads2=None, n=None):
    a, pa = _f32(ns1, n)
    b, pb = _f32(ns2, n)
    c, pc = _f32(gads2, n)
    return _check(ctx, load().lbm_set_geometry_per_component(ctx, pa, pb, pc))


def lbm_init_equilibrium(ctx, rho_a, rho_b, n=None):
    a, pa = _f32(rho_a, n)
    b, pb = _f32(rho_b, n)
    return _check(ctx, load().lbm_init_equilibrium(ctx, pa, pb))


def lbm_set_populations(ctx, f):
    a, pa = _f32(f)
    return _check(ctx, load().lbm_set_populations(ctx, pa))


def lbm_get_populations(ctx, out: np.ndarray):
    assert out.dtype == np.float32 and out.flags["C_CONTIGUOUS"]
    return _check(ctx, load().lbm_get_populations(
        ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))


def lbm_set_bc(ctx, face, layers, rho_a, rho_b):
    return _check(ctx, load().lbm_set_bc(ctx, face, layers, rho_a, rho_b))


def lbm_set_bc_velocity(ctx, face, layers, rho_a, rho_b, ux, uy, uz):
    return _check(ctx, load().lbm_set_bc_velocity(ctx, face, layers, rho_a, rho_b,
                                                  ux, uy, uz))


def lbm_step(ctx, n_steps):
    return _check(ctx, load().lbm_step(ctx, int(n_steps)))


def lbm_get_launch_config(ctx):
    v = [ctypes.c_int(0) for _ in range(3)]
    _check(ctx, load().lbm_get_launch_config(ctx, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def lbm_build_checked():
    return int(load().lbm_build_checked())


def lbm_fault_word(ctx, clear=True):
    v = ctypes.c_uint32(0)
    _check(ctx, load().lbm_fault_word(ctx, ctypes.byref(v), 1 if clear else 0))
    return int(v.value)


def lbm_set_single_pass(ctx, planes):
    return _check(ctx, load().lbm_set_single_pass(ctx, int(planes)))


def lbm_set_wavefront(ctx, shape, lag=0):
    return _check(ctx, load().lbm_set_wavefront(ctx, int(shape), int(lag)))


def lbm_set_wavefront_limits(ctx, spin_limit=0, withhold_flag=-1):
    return _check(ctx, load().lbm_set_wavefront_limits(ctx, int(spin_limit),
                                                        int(withhold_flag)))


def lbm_get_wavefront(ctx):
    shape, lag = ctypes.c_int(0), ctypes.c_int(0)
    _check(ctx, load().lbm_get_wavefront(ctx, ctypes.byref(shape), ctypes.byref(lag)))
    return shape.value, lag.value


def lbm_density(ctx):
    return _check(ctx, load().lbm_density(ctx))


def lbm_collide_stream(ctx):
    return _check(ctx, load().lbm_collide_stream(ctx))


def lbm_time(ctx) -> int:
    return load().lbm_time(ctx)


def lbm_read_fields(ctx, rho_a=None, rho_b=None, u=None, p=None):
    def ptr(a):
        if a is None:
            return None
        assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    return _check(ctx, load().lbm_read_fields(ctx, ptr(rho_a), ptr(rho_b),
                                              ptr(u), ptr(p)))


def lbm_reduce(ctx, allow_nan: bool = False) -> lbm_observables:
    out = lbm_observables()
    st = load().lbm_reduce(ctx, ctypes.byref(out))
    if st == LBM_ENAN and allow_nan:
        return out
    _check(ctx, st)
    return out


def lbm_sync(ctx, timeout_s: float):
    return _check(ctx, load().lbm_sync(ctx, float(timeout_s)))


def lbm_checkpoint_bytes(ctx) -> int:
    return load().lbm_checkpoint_bytes(ctx)


def lbm_save(ctx, buf: bytearray):
    cbuf = (ctypes.c_char * len(buf)).from_buffer(buf)
    return _check(ctx, load().lbm_save(ctx, ctypes.addressof(cbuf), len(buf)))


def lbm_load(ctx, buf: bytes):
    cbuf = ctypes.create_string_buffer(bytes(buf), len(buf))
    return _check(ctx, load().lbm_load(ctx, ctypes.addressof(cbuf), len(buf)))


def lbm_set_launch_config(ctx, density_cfg, even_cfg, odd_cfg):
    return _check(ctx, load().lbm_set_launch_config(ctx, int(density_cfg), int(even_cfg),
                                                    int(odd_cfg)))


def lbm_last_error(ctx) -> str:
    msg = load().lbm_last_error(ctx)
    return msg.decode() if msg else ""


def lbm_reduce_fields_noalloc(d_rho_a: int, d_rho_b: int, d_ns: int, nx: int,
                              ny: int, nz: int, layers, G: float,
                              cuda_stream: int):
    """Allocation-free observables from device density fields (pointers as
    ints).  Returns (status, lbm_observables); the caller checks the status
    because there is no context to carry a message."""
    out = lbm_observables()
    lay = (ctypes.c_int32 * 6)(*(layers if layers is not None else [0] * 6))
    st = load().lbm_reduce_fields_noalloc(
        ctypes.c_void_p(d_rho_a), ctypes.c_void_p(d_rho_b), ctypes.c_void_p(d_ns),
        nx, ny, nz, lay, float(G), ctypes.c_void_p(cuda_stream),
        ctypes.byref(out))
    return st, out


def _ctx_array(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    return arr


def lbm_batch_step(ctxs, n_steps, cuda_stream):
    """Advance the contexts together (one launch per pass for all)."""
    arr = _ctx_array(ctxs)
    st = load().lbm_batch_step(arr, len(ctxs), int(n_steps), ctypes.c_void_p(cuda_stream))
    if st != LBM_OK:
        raise LbmError(st, load().lbm_last_error(ctxs[0]).decode() if ctxs else "")
    return st


def lbm_batch_graph_create(ctxs, n_steps, cuda_stream):
    arr = _ctx_array(ctxs)
    g = ctypes.c_void_p()
    st = load().lbm_batch_graph_create(arr, len(ctxs), int(n_steps),
                                       ctypes.c_void_p(cuda_stream), ctypes.byref(g))
    if st != LBM_OK:
        raise LbmError(st, load().lbm_last_error(ctxs[0]).decode() if ctxs else "")
    return g


def lbm_batch_graph_launch(graph, cuda_stream):
    st = load().lbm_batch_graph_launch(graph, ctypes.c_void_p(cuda_stream))
    if st != LBM_OK:
        raise LbmError(st, "graph launch refused")
    return st


def lbm_batch_graph_destroy(graph):
    load().lbm_batch_graph_destroy(graph)


# ---- convenience wrapper ------------------------------------------------

class Lattice:
    """One HMCSC lattice on the current CUDA device.

    Allocates the device workspace with PyTorch (``torch.empty`` uint8) and
    runs on PyTorch's current stream (or ``stream``).  Arrays in and out are
    numpy, shaped ``[nz, ny, nx]`` (populations ``[2, 19, nz, ny, nx]``).
    """

    def __init__(self, nx, ny, nz, tau=(1.0, 1.0), G=1.75, F_ext=(0, 0, 0),
                 stream=None, device=None, storage="f32", rho0=(0.0, 0.0),
                 ns_per_component=False):
        import torch
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        p = lbm_params()
        p.nx, p.ny, p.nz = nx, ny, nz
        p.storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
        self.storage_name = {v: k for k, v in STORAGES.items()}[p.storage]
        p.rho0[0], p.rho0[1] = rho0
        p.tau[0], p.tau[1] = tau
        p.G = G
        for d in range(3):
            p.F_ext[d] = F_ext[d]
        p.ns_per_component = 1 if ns_per_component else 0
        self.params = p
        nbytes = lbm_workspace_bytes(p)
        if nbytes == 0:
            raise LbmError(LBM_EINVAL, "invalid lattice parameters")
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.ctx = lbm_create(p, self.workspace.data_ptr(), nbytes,
                              self.stream.cuda_stream)

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, ns, gads2=None, ns2=None):
        """n_s (both components, or fluid 1 when ns2 is given), G_ads,2 and
        optionally n_s,2 (needs ns_per_component=True)."""
        if ns2 is None:
            lbm_set_geometry(self.ctx, ns, gads2, self.N)
        else:
            lbm_set_geometry_per_component(self.ctx, ns, ns2, gads2, self.N)

    def init_equilibrium(self, rho_a, rho_b):
        lbm_init_equilibrium(self.ctx, rho_a, rho_b, self.N)

    def set_populations(self, f):
        lbm_set_populations(self.ctx, np.asarray(f).reshape(2, 19, self.N))

    def populations(self):
        out = np.empty((2, 19) + self.shape, dtype=np.float32)
        lbm_get_populations(self.ctx, out)
        return out

    def set_bc(self, face, layers, rho_a=1.0, rho_b=1.0, u=None):
        """Density reservoir on `face` (u None), or velocity boundary cells
        held at f^eq(rho, u)."""
        if u is None:
            lbm_set_bc(self.ctx, face, layers, rho_a, rho_b)
        else:
            lbm_set_bc_velocity(self.ctx, face, layers, rho_a, rho_b, *u)

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def launch_config(self):
        """(density, even, odd) launch shapes in use."""
        return lbm_get_launch_config(self.ctx)

    def set_single_pass(self, planes):
        """Single-pass lbm_step with boxes of `planes` planes (0: two passes)."""
        lbm_set_single_pass(self.ctx, planes)

    def set_wavefront(self, shape, lag=0):
        """Wavefront lbm_step of tile shape `shape` (1: 32 x 4, 2: 32 x 2,
        3: 32 x 8 nodes; 0: off) with densities `lag` planes ahead (0:
        default); lbm_batch_step then also steps such lattices together in
        one wavefront launch."""
        lbm_set_wavefront(self.ctx, shape, lag)

    def wavefront(self):
        """(shape, lag) of the wavefront step in use (shape 0: off)."""
        return lbm_get_wavefront(self.ctx)

    def set_launch_config(self, density_cfg=0, even_cfg=0, odd_cfg=0):
        lbm_set_launch_config(self.ctx, density_cfg, even_cfg, odd_cfg)

    def autotune(self, table=None, single_pass=False):
        """Launch shapes for this size and storage from the tuning table
        (timed on a scratch lattice first if the table has none); with
        single_pass the tuner also weighs the single-pass step."""
        from . import autotune
        return autotune.apply(self, table, single_pass=single_pass)

    @property
    def t(self):
        return lbm_time(self.ctx)

    def fields(self):
        out = {"rho_a": np.empty(self.shape, np.float32),
               "rho_b": np.empty(self.shape, np.float32),
               "u": np.empty((3,) + self.shape, np.float32),
               "p": np.empty(self.shape, np.float32)}
        lbm_read_fields(self.ctx, out["rho_a"], out["rho_b"], out["u"], out["p"])
        return out

    def observables(self, allow_nan=False):
        o = lbm_reduce(self.ctx, allow_nan)
        return {"mass": np.array(o.mass[:]), "sat1": o.sat1,
                "p_face": np.array(o.p_face[:]), "nonfinite": o.nonfinite}

    def save(self) -> bytearray:
        buf = bytearray(lbm_checkpoint_bytes(self.ctx))
        lbm_save(self.ctx, buf)
        return buf

    def load(self, buf):
        lbm_load(self.ctx, buf)
