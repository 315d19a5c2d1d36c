"""Bounce-back fraction per component, n_s,sigma (Eq. 1; the adhesion
indicator s = n_s,sigma of Eq. 4; Eq. 7 weights each component by
1 - n_s,sigma): the CUDA path against the FP64 oracle, the membrane property
of Sec. 4 on the GPU, and batched == alone for such lattices.

Tolerances as in test_gpu_parity.py (float32 against float64).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2206_11524_gb300 import build, lbm, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    lbm.load()
    oracle.build()


def w64(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _pc_pair(shape, ns1, ns2, gads, tau=(0.8, 1.3), G=1.75, F=(2e-5, -1e-5, 3e-5),
             storage="f32"):
    nz, ny, nx = shape
    g = lbm.Lattice(nx, ny, nz, tau=tau, G=G, F_ext=F, ns_per_component=True,
                    storage=storage, rho0=(0.5, 0.5))
    g.set_geometry(ns1, gads, ns2=ns2)
    p = oracle.Params(nx, ny, nz, tau=tuple(float(np.float32(t)) for t in tau),
                      G=float(np.float32(G)),
                      Fext=tuple(float(np.float32(v)) for v in F))
    r = oracle.Sim(p, np.stack([w64(ns1), w64(ns2)]), w64(gads))
    return g, r


@pytest.mark.parametrize("shape", [(5, 4, 7), (3, 9, 33), (2, 5, 64)])
def test_per_component_populations_and_fields(shape):
    """Random state, independent random n_s,1 and n_s,2 (0 and 1 included),
    random G_ads: every population after 1-3 steps and the fields."""
    seed = 7 * sum(shape)
    ns1, gads = synth.random_geometry(shape, seed)
    ns2, _ = synth.random_geometry(shape, seed + 3)
    g, r = _pc_pair(shape, ns1, ns2, gads)
    f0 = synth.random_state(shape, seed + 1).astype(np.float32)
    g.set_populations(f0)
    r.set_populations(f0.astype(np.float64))
    for k in range(1, 4):
        g.step(1)
        r.step(1)
        assert np.abs(g.populations() - r.f).max() <= 2e-6 * np.abs(r.f).max(), k
    fg, fr = g.fields(), r.fields()
    for key in ("rho_a", "rho_b", "p"):
        assert np.abs(fg[key] - fr[key]).max() <= 1e-5 * np.abs(fr[key]).max(), key
    assert np.abs(fg["u"] - fr["u"]).max() <= 1e-5 * np.abs(fr["u"]).max()
    g.close()


def test_one_fraction_equals_the_common_path():
    """A per-component workspace given n_s,1 = n_s,2 steps bit-identically to
    a lattice with one fraction; u_macro of Eq. 7 is summed per component
    there, so it agrees to float32 rounding."""
    shape = (4, 6, 40)
    ns, gads = synth.random_geometry(shape, 5)
    f0 = synth.random_state(shape, 6).astype(np.float32)
    a = lbm.Lattice(40, 6, 4, tau=(0.9, 1.1), G=1.5, F_ext=(1e-5, 0, 0))
    b = lbm.Lattice(40, 6, 4, tau=(0.9, 1.1), G=1.5, F_ext=(1e-5, 0, 0),
                    ns_per_component=True)
    a.set_geometry(ns, gads)
    b.set_geometry(ns, gads, ns2=ns)
    for lat in (a, b):
        lat.set_populations(f0)
        lat.step(5)
    assert np.array_equal(a.populations(), b.populations())
    fa, fb = a.fields(), b.fields()
    for key in ("rho_a", "rho_b", "p"):
        assert np.array_equal(fa[key], fb[key]), key
    assert np.abs(fa["u"] - fb["u"]).max() <= 1e-6 * np.abs(fa["u"]).max()
    a.close()
    b.close()


def test_membrane_keeps_fluid_2_on_its_side():
    """Membranes n_s,2 = 1, n_s,1 = 0 at x = 0 and x = 8 of a periodic box
    (Sec. 4): fluid 2's content of B (x = 9..15, plus the populations at the
    membranes that arrived from B) is conserved to float32 rounding over
    300 steps while fluid 1 flows between the sides."""
    nx, shape = 16, (3, 4, 16)
    x = np.arange(nx)
    memb = (x == 0) | (x == 8)
    B = x >= 9
    ns1 = np.zeros(shape)
    ns2 = np.where(memb, 1.0, 0.0) * np.ones(shape)
    ra = np.where(B, 0.8, 0.5) * np.ones(shape)
    rb = np.where(B, 0.1, 0.4) * np.ones(shape)
    g = lbm.Lattice(nx, 4, 3, tau=(1.0, 0.9), G=0.4, ns_per_component=True)
    g.set_geometry(ns1, None, ns2=ns2)
    g.init_equilibrium(ra, rb)
    c, _, _ = oracle.lattice()

    def content_B(f, sg):
        f = f.astype(np.float64)
        into8 = [i for i in range(19) if c[i, 0] == -1]
        into0 = [i for i in range(19) if c[i, 0] == 1]
        return (f[sg][..., B].sum() + f[sg][into8][..., 8].sum()
                + f[sg][into0][..., 0].sum())

    f0 = g.populations()
    m2, m1 = content_B(f0, 1), content_B(f0, 0)
    g.step(300)
    f = g.populations()
    assert abs(content_B(f, 1) - m2) <= 1e-5 * m2
    assert content_B(f, 0) < 0.98 * m1
    g.close()


def test_batched_per_component_equals_alone():
    """Two per-component lattices of different sizes stepped together by the
    batched kernels match each stepped alone, bit for bit."""
    out = []
    for batched in (False, True):
        lats = []
        for k, shape in enumerate([(4, 6, 40), (3, 5, 33)]):
            nz, ny, nx = shape
            ns1, gads = synth.random_geometry(shape, 20 + k)
            ns2, _ = synth.random_geometry(shape, 30 + k)
            lat = lbm.Lattice(nx, ny, nz, tau=(1.0, 0.8), G=1.6,
                              ns_per_component=True)
            lat.set_geometry(ns1, gads, ns2=ns2)
            lat.set_populations(synth.random_state(shape, 40 + k))
            lats.append(lat)
        if batched:
            lbm.lbm_batch_step([l.ctx for l in lats], 4,
                               torch.cuda.current_stream().cuda_stream)
        else:
            for l in lats:
                l.step(4)
        out.append([l.populations() for l in lats])
        for l in lats:
            l.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_one_fraction_context_rejects_two():
    g = lbm.Lattice(8, 2, 2)
    ns = np.zeros((2, 2, 8))
    with pytest.raises(lbm.LbmError):
        g.set_geometry(ns, None, ns2=ns)
    g.close()
