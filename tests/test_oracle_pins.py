"""Pins of the FP64 oracle to facts fixed by the paper and by the mathematics.

Each test ties one part of the oracle to something other than the oracle
itself: a table or value the paper prints (``tests/golden/``), a closed form
the paper states or that follows exactly from Eq. 1, an exact invariant, or a
symmetry of the lattice.  They are chosen so that a plausible slip (a dropped
(1 - n_s) factor, a wrong bounce-back index, a sign in a force, a swapped
weight, a wrong relaxation time) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CS2 = 1.0 / 3.0


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


def _momentum(f):
    """Total momentum density sum_sigma sum_i f c_i at every node -> [3,...]."""
    c, _, _ = oracle.lattice()
    return np.einsum("sizyx,id->dzyx", f, c.astype(np.float64))


# --------------------------------------------------------------------------
# Lattice (Eq. A.8) and equilibrium (Eq. A.3)
# --------------------------------------------------------------------------

def test_velocity_set_is_the_printed_eq_A8():
    table = _golden("d3q19_velocity_set_eqA8.txt").astype(int)
    c, w, opp = oracle.lattice()
    assert np.array_equal(table[:, 0], np.arange(19))
    assert np.array_equal(table[:, 1:], c)
    n2 = (c * c).sum(1)
    expect_w = np.where(n2 == 0, 1 / 3, np.where(n2 == 1, 1 / 18, 1 / 36))
    assert np.allclose(w, expect_w, rtol=0, atol=1e-17)
    for i in range(19):
        assert np.array_equal(c[opp[i]], -c[i])


def test_lattice_isotropy_moments():
    """sum w = 1, sum w c = 0, sum w c c = cs2 I, fourth moment isotropic:
    the properties that make Eq. A.3 recover Navier-Stokes (Appendix A)."""
    c, w, _ = oracle.lattice()
    c = c.astype(np.float64)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(np.einsum("i,id->d", w, c)).max() < 1e-16
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), CS2 * np.eye(3),
                       atol=1e-16)
    d = np.eye(3)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d)
                      + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    assert np.allclose(m4, iso, atol=1e-16)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibrium_moments(seed):
    """Eq. A.3 has density rho, momentum rho u and second moment
    rho (cs2 I + u u) exactly (a dropped or mis-scaled term breaks one)."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.01, 2.0)
    u = rng.uniform(-0.1, 0.1, 3)
    c, _, _ = oracle.lattice()
    c = c.astype(np.float64)
    fe = oracle.feq(rho, u)
    assert abs(fe.sum() - rho) < 1e-14
    assert np.allclose(fe @ c, rho * u, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib->ab", fe, c, c),
                       rho * (CS2 * np.eye(3) + np.outer(u, u)), atol=1e-15)


# --------------------------------------------------------------------------
# Exact consequences of Eq. 1 on uniform states
# --------------------------------------------------------------------------

def _uniform_sim(shape, ns, tau, G, F, rho=(0.7, 0.3), u=((0, 0, 0), (0, 0, 0)),
                 gads=0.0):
    nz, ny, nx = shape
    p = oracle.Params(nx, ny, nz, tau=tau, G=G, Fext=F)
    s = oracle.Sim(p, np.full(shape, ns), np.full(shape, gads))
    f = np.zeros((2, 19) + shape)
    for sg in range(2):
        f[sg] = oracle.feq(rho[sg], np.array(u[sg], float))[:, None, None, None]
    s.set_populations(f)
    return s


@pytest.mark.parametrize("ns,tau", [(0.05, (0.8, 1.3)), (0.3, (1.0, 1.0)),
                                    (0.5, (0.6, 1.7)), (0.77, (1.2, 0.9)),
                                    (0.999, (1.0, 2.0))])
def test_exact_darcy_recurrence(ns, tau):
    """Uniform medium, uniform densities: F_inter = F_ads = 0 and summing
    Eq. 1 over sigma and i gives J' = (1 - 2 n_s) J + (1 - n_s) F exactly for
    the mixture momentum J (the u' of Eq. 6 cancels), so
    J_n = J* + (1 - 2 n_s)^n (J_0 - J*),  J* = (1 - n_s) F / (2 n_s), and
    rho u_macro = (1 - n_s)(J + F/2) (Eq. 7), whose limit is the Darcy
    permeability of Eq. 2: k = nu (1 - n_s) / (2 n_s)."""
    F = np.array([1e-5, -2e-5, 3e-6])
    u0 = ((0.01, -0.02, 0.005), (-0.03, 0.01, 0.0))
    s = _uniform_sim((3, 2, 4), ns, tau, 1.75, tuple(F), u=u0, gads=0.2)
    J0 = _momentum(s.f)[:, 0, 0, 0]
    Jstar = (1 - ns) * F / (2 * ns)
    for n in (1, 2, 7, 40):
        s.step(n - (s.t if s.t else 0))
        J = _momentum(s.f)[:, 0, 0, 0]
        expect = Jstar + (1 - 2 * ns) ** n * (J0 - Jstar)
        assert np.allclose(J, expect, rtol=1e-11, atol=1e-17), (n, J, expect)
        fl = s.fields()
        rho_u = fl["u"][:, 0, 0, 0] * (fl["rho_a"][0, 0, 0] + fl["rho_b"][0, 0, 0])
        assert np.allclose(rho_u, (1 - ns) * (expect + F / 2), rtol=1e-11,
                           atol=1e-17)


@pytest.mark.parametrize("ns", [0.1, 0.5, 0.9])
def test_permeability_eq2(ns):
    """Eq. 8 applied to the converged uniform run equals Eq. 2 (Sec. 3.1)."""
    F = 1e-5
    tau = 1.0
    nu = CS2 * (tau - 0.5)
    s = _uniform_sim((2, 2, 2), ns, (tau, tau), 0.0, (F, 0.0, 0.0),
                     rho=(0.99, 0.01))
    s.step(300)
    fl = s.fields()
    rho_u = (fl["u"][0] * (fl["rho_a"] + fl["rho_b"])).mean()
    k = nu * rho_u / F
    assert abs(k - (1 - ns) / (2 * ns) * nu) < 1e-10 * k


def test_rest_state_is_fixed_point():
    """No force and no flow: Eq. 1 maps f^eq(rho, 0) to itself."""
    s = _uniform_sim((3, 3, 3), 0.4, (0.9, 1.1), 1.75, (0, 0, 0), gads=0.3)
    f0 = s.f.copy()
    s.step(5)
    assert np.abs(s.f - f0).max() < 1e-15


# --------------------------------------------------------------------------
# Invariants of Eq. 1 on random states
# --------------------------------------------------------------------------

def _random_sim(seed, shape=(5, 4, 7), G=1.75, F=(2e-5, -1e-5, 3e-5),
                tau=(0.8, 1.3), ns_choice=None):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    ns = rng.uniform(0, 1, shape)
    ns.flat[::5] = 0.0
    ns.flat[::7] = 1.0
    if ns_choice is not None:
        ns = np.full(shape, ns_choice)
    gads = rng.uniform(-0.3, 0.3, shape)
    p = oracle.Params(nx, ny, nz, tau=tau, G=G, Fext=F)
    s = oracle.Sim(p, ns, gads)
    _, w, _ = oracle.lattice()
    base = np.array([0.8, 0.2])[:, None, None, None, None] * \
        w[None, :, None, None, None]
    f = base * rng.uniform(0.7, 1.3, (2, 19) + shape)
    s.set_populations(f)
    return s


@pytest.mark.parametrize("seed", [3, 4])
def test_component_mass_conserved(seed):
    """Sum_i of the right-hand side of Eq. 1 is rho_sigma at every node and
    streaming permutes populations, so each component's mass is invariant in
    a closed periodic lattice."""
    s = _random_sim(seed)
    m0 = s.observables()["mass"]
    s.step(60)
    m1 = s.observables()["mass"]
    assert np.allclose(m1, m0, rtol=1e-13, atol=0)


def test_full_bounce_back_has_period_two():
    """n_s = 1 everywhere is pure bounce-back (Appendix A): f(t+2) = f(t)
    bit for bit, f(t+1) != f(t)."""
    s = _random_sim(5, ns_choice=1.0)
    f0 = s.f.copy()
    s.step(1)
    assert np.abs(s.f - f0).max() > 1e-3
    s.step(1)
    assert np.array_equal(s.f, f0)


def test_uniform_medium_adhesion_vanishes():
    """With uniform n_s and uniform G_ads the stencil of Eq. 4 sums to zero,
    so the result does not depend on G_ads (the mechanism behind the paper's
    finding that gamma is independent of G_ads, Sec. 3.3)."""
    out = []
    for g in (0.0, 0.25):
        s = _random_sim(6, ns_choice=0.3)
        s.gads2[...] = g
        s.step(15)
        out.append(s.f.copy())
    assert np.abs(out[0] - out[1]).max() < 1e-15


def test_rotation_and_mirror_symmetry():
    """A quarter turn about z and the mirror x -> -x map the lattice onto
    itself; the densities of the transformed run are the transformed
    densities (pins the velocity table, the stencil signs and the
    bounce-back index together)."""
    rng = np.random.default_rng(7)
    shape = (4, 6, 6)
    ns = rng.uniform(0, 1, shape)
    gads = rng.uniform(-0.3, 0.3, shape)
    ra = rng.uniform(0.05, 1.0, shape)
    rb = rng.uniform(0.05, 1.0, shape)

    def run(ns, gads, ra, rb):
        p = oracle.Params(shape[2], shape[1], shape[0], tau=(0.9, 1.2), G=1.5)
        s = oracle.Sim(p, ns, gads)
        s.init_equilibrium(ra, rb)
        s.step(12)
        fl = s.fields()
        return fl["rho_a"], fl["rho_b"]

    base = run(ns, gads, ra, rb)
    rot = lambda a: np.ascontiguousarray(np.rot90(a, 1, axes=(1, 2)))
    mir = lambda a: np.ascontiguousarray(a[:, :, ::-1])
    for T in (rot, mir):
        got = run(T(ns), T(gads), T(ra), T(rb))
        for g, b in zip(got, base):
            assert np.abs(g - T(b)).max() < 1e-13


def test_component_swap_symmetry():
    """Relabelling fluid 1 <-> fluid 2 together with G_ads,2 -> -G_ads,2 and
    tau_1 <-> tau_2 swaps the two density fields (Eqs. 3-6 are symmetric in
    sigma once G_ads,1 = -G_ads,2, Table 1)."""
    rng = np.random.default_rng(8)
    shape = (3, 5, 6)
    ns = rng.uniform(0, 1, shape)
    gads = rng.uniform(-0.3, 0.3, shape)
    ra = rng.uniform(0.05, 1.0, shape)
    rb = rng.uniform(0.05, 1.0, shape)

    def run(gads, ra, rb, tau):
        p = oracle.Params(shape[2], shape[1], shape[0], tau=tau, G=1.75,
                          Fext=(1e-4, 0, -2e-4))
        s = oracle.Sim(p, ns, gads)
        s.init_equilibrium(ra, rb)
        s.step(10)
        fl = s.fields()
        return fl["rho_a"], fl["rho_b"]

    a1, b1 = run(gads, ra, rb, (0.8, 1.4))
    a2, b2 = run(-gads, rb, ra, (1.4, 0.8))
    assert np.abs(a1 - b2).max() < 1e-13
    assert np.abs(b1 - a2).max() < 1e-13


# --------------------------------------------------------------------------
# Textbook special case: LBGK shear wave (Appendix A, Eq. A.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("tau", [0.8, 1.4])
def test_shear_wave_viscosity(tau):
    """n_s = 0, G = 0: Eq. 1 is LBGK (Eq. A.1) with nu = cs2 (tau - 1/2); a
    shear wave u_y = U sin(2 pi x / L) decays as exp(-nu k^2 t)."""
    L = 64
    U = 1e-4
    nu = CS2 * (tau - 0.5)
    p = oracle.Params(L, 1, 1, tau=(tau, tau), G=0.0)
    s = oracle.Sim(p, np.zeros((1, 1, L)))
    f = np.zeros((2, 19, 1, 1, L))
    for x in range(L):
        u = np.array([0.0, U * math.sin(2 * math.pi * x / L), 0.0])
        f[0, :, 0, 0, x] = oracle.feq(0.6, u)
        f[1, :, 0, 0, x] = oracle.feq(0.4, u)
    s.set_populations(f)
    k = 2 * math.pi / L
    T = int(round(math.log(2) / (nu * k * k)))   # one half-life
    s.step(T)
    uy = s.fields()["u"][1, 0, 0]
    amp = 2 / L * (uy * np.sin(k * np.arange(L))).sum()
    # O(k^2) lattice correction to the continuum rate: 0.3 % at k = 2 pi / 64
    assert abs(amp / (U * math.exp(-nu * k * k * T)) - 1) < 1e-2


# --------------------------------------------------------------------------
# Darcy-Brinkman benchmarks of Sec. 3.2 and Table C.1
# --------------------------------------------------------------------------

def _open_boundary_umax(ns_right, steps):
    H = 100
    F = 1e-6
    ns = np.zeros((1, 1, H))
    ns[..., : H // 2 + 1] = 0.9          # x in [0, H/2]
    ns[..., H // 2 + 1:] = ns_right      # x in ]H/2, H]
    p = oracle.Params(H, 1, 1, tau=(1.0, 1.0), G=0.0, Fext=(0.0, F, 0.0))
    s = oracle.Sim(p, ns)
    s.init_equilibrium(np.full(ns.shape, 0.99), np.full(ns.shape, 0.01))
    s.step(steps)
    return s.fields()["u"][1, 0, 0].max()


def _eq13_right_centre(ns_l, ns_r, H=100, F=1e-6, nu=1 / 6):
    """Eq. 13b with Table 2's parameters, at the centre x = 3H/4."""
    kl = (1 - ns_l) / (2 * ns_l) * nu
    kr = (1 - ns_r) / (2 * ns_r) * nu
    U0r = kr * F / nu
    pr = kl / kr
    qr = math.sqrt(ns_r / ns_l)
    rl = math.sqrt(2 * ns_l / nu)
    rr = math.sqrt(2 * ns_r / nu)
    coth = lambda v: math.cosh(v) / math.sinh(v)
    return U0r * (1 + (pr - 1) / (math.sinh(rr * H / 4)
                                  * (qr * coth(rl * H / 4) + coth(rr * H / 4))))


@pytest.mark.parametrize("row", [1, 2, 3, 4])
def test_open_boundary_umax_table(row):
    """Table C.1: u_max of the two-layer open-boundary flow (Sec. 3.2)."""
    ns_r, umax = _golden("open_boundary_umax_tableC1.txt")[row]
    got = _open_boundary_umax(ns_r, 3000)
    assert abs(got / umax - 1) < 1e-3


def test_open_boundary_brinkman_row_follows_eq13():
    """Row n_s,right = 0.001 of Table C.1 prints 4.732e-4, but Eq. 13b with
    Table 2's parameters gives 4.372e-4 at the layer centre; the oracle is
    held to Eq. 13b (2 %), the closed form the paper says the runs match."""
    got = _open_boundary_umax(0.001, 20000)
    assert abs(got / _eq13_right_centre(0.9, 0.001) - 1) < 0.02


@pytest.mark.parametrize("ns", [0.001, 0.01, 0.1, 0.5, 0.9])
def test_poiseuille_with_bounce_back_walls(ns):
    """Sec. 3.2 paragraph 1: walls are n_s = 1 cells (x = 0 and x = H+1),
    fluid cells 1..H sit at x_a = i - 1/2 from the wall; the profile is
    Eq. 11.  The centre value matches to 1e-6 where the centre is Darcy-like
    (n_s >= 0.1) and to 1e-3 otherwise; the whole
    profile to 1 % of u_max in the Brinkman regime (n_s <= 0.1), where the
    paper reports excellent agreement."""
    H, F, nu = 50, 1e-5, 1 / 6
    steps = {0.001: 30000, 0.01: 8000}.get(ns, 2500)
    nsf = np.full((1, 1, H + 2), ns)
    nsf[..., 0] = nsf[..., -1] = 1.0
    p = oracle.Params(H + 2, 1, 1, tau=(1.0, 1.0), G=0.0, Fext=(0.0, F, 0.0))
    s = oracle.Sim(p, nsf)
    s.init_equilibrium(np.full(nsf.shape, 0.99), np.full(nsf.shape, 0.01))
    s.step(steps)
    u = s.fields()["u"][1, 0, 0, 1:-1]
    k = (1 - ns) / (2 * ns) * nu
    r = math.sqrt(2 * ns / nu)
    xa = np.arange(1, H + 1) - 0.5
    ua = F * k / nu * (1 - np.cosh(r * (xa - H / 2)) / np.cosh(r * H / 2))
    assert abs(u[H // 2] / ua[H // 2] - 1) < (1e-6 if ns >= 0.1 else 1e-3)
    if ns <= 0.1:
        assert np.abs(u - ua).max() < 0.01 * ua.max()


# --------------------------------------------------------------------------
# Bubble test (Sec. 3.3): Laplace law, gamma(G), independence of n_s
# --------------------------------------------------------------------------

def _coexistence(G):
    """Bulk densities of a flat interface at rest (1D run of the oracle)."""
    H = 48
    x = np.arange(H)
    inside = (x >= H // 4) & (x < 3 * H // 4)
    p = oracle.Params(H, 1, 1, tau=(1.0, 1.0), G=G)
    s = oracle.Sim(p, np.zeros((1, 1, H)))
    s.init_equilibrium(np.where(inside, 0.99, 0.01)[None, None],
                       np.where(inside, 0.01, 0.99)[None, None])
    s.step(6000)
    fl = s.fields()
    return fl["rho_a"][0, 0, H // 2], fl["rho_b"][0, 0, H // 2]


def _bubble_gamma(G, ns, steps, H=64, R=14):
    hi, lo = _coexistence(G)
    yy, xx = np.meshgrid(np.arange(H), np.arange(H), indexing="ij")
    r = np.hypot(xx - H / 2 + 0.5, yy - H / 2 + 0.5)
    inside = r < R
    p = oracle.Params(H, H, 1, tau=(1.0, 1.0), G=G)
    s = oracle.Sim(p, np.full((1, H, H), ns))
    s.init_equilibrium(np.where(inside, hi, lo)[None],
                       np.where(inside, lo, hi)[None])
    s.step(steps)
    fl = s.fields()
    a, pr = fl["rho_a"][0], fl["p"][0]
    area = ((a - a.min()) / (a.max() - a.min())).sum()
    Req = math.sqrt(area / math.pi)
    dp = pr[r < Req / 2].mean() - pr[r > Req + 8].mean()
    return dp * Req          # 2D Laplace law: gamma = dp R (Sec. 3.3)


@pytest.mark.slow
def test_laplace_gamma_vs_G_and_ns():
    """gamma = dp R (Sec. 3.3) on a 64 x 64 bubble of radius 14.  The paper
    notes that gamma measured in small domains comes out high and converges
    to 0.077 only for H >= 100; at H = 64 this measurement reads 7-13 % high,
    so the printed gamma(G) is held to 15 %, the printed ratio
    gamma(2.0)/gamma(1.5) = 2.04 to 8 %, and gamma at n_s = 0.5 must equal
    gamma at n_s = 0 within 1 % (the paper's central claim for the model).
    A force of the wrong sign dissolves the bubble, a factor-2 slip in G moves
    gamma far outside these bands."""
    table = _golden("interfacial_tension_sec33.txt")
    got = {G: _bubble_gamma(G, 0.0, 3000) for G in table[:, 0]}
    for G, gam in table:
        assert abs(got[G] / gam - 1) < 0.15, (G, got[G], gam)
    ratio = got[2.0] / got[1.5]
    assert abs(ratio / (0.104 / 0.051) - 1) < 0.08, ratio
    g_half = _bubble_gamma(1.75, 0.5, 6000)
    assert abs(g_half / got[1.75] - 1) < 0.01


# --------------------------------------------------------------------------
# Reservoirs and observables (Sec. 4, Eqs. 18-19, Eq. A.6)
# --------------------------------------------------------------------------

def test_reservoir_layers_and_observables():
    """After a step the reservoir layers hold f^eq(rho_res, 0) exactly; the
    mean pressure over a reservoir is Eq. A.6 at the prescribed densities;
    S_1 (Eq. 19) weights each non-reservoir cell by 1 - n_s and counts it
    when rho_1 >= 0.5."""
    nx, ny, nz = 12, 3, 2
    G = 1.75
    res = {0: (4, 1.04, 0.01), 1: (4, 0.01, 0.99)}
    p = oracle.Params(nx, ny, nz, tau=(1.0, 1.0), G=G, reservoirs=res)
    rng = np.random.default_rng(9)
    ns = rng.uniform(0, 1, (nz, ny, nx))
    s = oracle.Sim(p, ns, rng.uniform(-0.2, 0.2, (nz, ny, nx)))
    ra = np.where(np.arange(nx) < 6, 0.99, 0.01)[None, None].repeat(ny, 1).repeat(nz, 0)
    s.init_equilibrium(ra, 1.0 - ra)
    s.step(3)
    for face, (L, r1, r2) in res.items():
        xs = range(L) if face == 0 else range(nx - L, nx)
        for x in xs:
            assert np.array_equal(s.f[0, :, :, :, x],
                                  np.broadcast_to(oracle.feq(r1, np.zeros(3))[:, None, None],
                                                  (19, nz, ny)))
            assert np.array_equal(s.f[1, :, :, :, x],
                                  np.broadcast_to(oracle.feq(r2, np.zeros(3))[:, None, None],
                                                  (19, nz, ny)))
    obs = s.observables()
    for face, (L, r1, r2) in res.items():
        assert abs(obs["p_face"][face] - CS2 * (r1 + r2 + G * r1 * r2)) < 1e-15
    assert all(math.isnan(v) for v in obs["p_face"][2:])
    fl = s.fields()
    inner = np.zeros((nz, ny, nx), bool)
    inner[..., 4:nx - 4] = True
    wgt = (1 - ns)[inner]
    filled = (fl["rho_a"] >= 0.5)[inner]
    assert abs(obs["sat1"] - wgt[filled].sum() / wgt.sum()) < 1e-14
    assert np.allclose(obs["mass"], [fl["rho_a"].sum(), fl["rho_b"].sum()],
                       rtol=1e-15)


def _saturation_state(nx=10, ny=2, nz=2):
    """A state whose S_1 (Eq. 19) is known by construction.  Reservoir layers
    of 2 cells at x = 0, 1 (fluid 1) and x = 8, 9 (fluid 2); the six columns
    between them carry (rho_1, n_s):
        x = 2: (1.0,    0.0)   filled, weight 1
        x = 3: (0.5,    0.25)  exactly at the threshold: filled, weight 0.75
        x = 4: (0.7,    1.0)   filled but solid: weight 0
        x = 5: (0.4999, 0.5)   not filled, weight 0.5
        x = 6: (0.9,    0.9)   filled, weight 0.1
        x = 7: (0.1,    0.0)   not filled, weight 1
    so S_1 = (1 + 0.75 + 0.1) / (1 + 0.75 + 0 + 0.5 + 0.1 + 1) = 37 / 67.
    Each density sits in the rest population alone, so sum_i f_i is exactly
    the value above."""
    cols = {0: (1.0, 0.0), 1: (1.0, 0.0), 2: (1.0, 0.0), 3: (0.5, 0.25), 4: (0.7, 1.0),
            5: (0.4999, 0.5), 6: (0.9, 0.9), 7: (0.1, 0.0), 8: (0.2, 0.3), 9: (0.2, 0.3)}
    shape = (nz, ny, nx)
    ns = np.zeros(shape)
    f = np.zeros((2, 19) + shape)
    for x, (r1, s_) in cols.items():
        ns[..., x] = s_
        f[0, 0, ..., x] = r1
        f[1, 0, ..., x] = 0.3
    res = {0: (2, 1.0, 0.01), 1: (2, 0.01, 1.0)}
    return shape, ns, f, res


def test_saturation_of_a_constructed_state():
    """S_1 of Eq. 19 on a state built to a known value (see
    _saturation_state): the tie rho_1 = 0.5 counts as filled, each cell is
    weighted by its fluid fraction 1 - n_s, solid cells and the reservoir
    layers do not count.  Counting rho_1 > 0.5, weighting by n_s, counting
    all nodes or the reservoirs all give other values."""
    shape, ns, f, res = _saturation_state()
    nz, ny, nx = shape
    s = oracle.Sim(oracle.Params(nx, ny, nz, reservoirs=res), ns)
    s.set_populations(f)
    obs = s.observables()
    assert abs(obs["sat1"] - 37.0 / 67.0) < 1e-14, obs["sat1"]
    # the same observables computed from the density fields alone
    dens = oracle.observables_of_densities(oracle.Params(nx, ny, nz, reservoirs=res), ns,
                                           f[0].sum(axis=0), f[1].sum(axis=0))
    assert dens["sat1"] == obs["sat1"] and np.array_equal(dens["mass"], obs["mass"])
    assert abs(obs["mass"][0] - 4 * (3 * 1.0 + 0.5 + 0.7 + 0.4999 + 0.9 + 0.1 + 0.4)) < 1e-13
    # Eq. 19 with a fraction per component weights by fluid 1's own: a
    # different n_s,2 changes nothing
    ns2 = np.where(ns > 0.5, 0.0, 1.0)
    s2 = oracle.Sim(oracle.Params(nx, ny, nz, reservoirs=res), np.stack([ns, ns2]))
    s2.set_populations(f)
    assert s2.observables()["sat1"] == obs["sat1"]
    # the same state with every column of fluid 1 below the threshold
    f_empty = f.copy()
    f_empty[0, 0] = 0.25
    s.set_populations(f_empty)
    assert s.observables()["sat1"] == 0.0
    # and with the fluid fraction summing to zero (all solid between the
    # reservoirs) S_1 is undefined
    s3 = oracle.Sim(oracle.Params(nx, ny, nz, reservoirs=res), np.ones(shape))
    s3.set_populations(f)
    assert math.isnan(s3.observables()["sat1"])


# --------------------------------------------------------------------------
# Bounce-back fraction per component, n_s,sigma (Eq. 1, Eq. 4 with
# s = n_s,sigma, Eq. 7; membranes of Sec. 4, porous obstacles of Sec. 3.5)
# --------------------------------------------------------------------------

def _per_component_sim(shape, ns_pair, tau, G, F, rho, u, gads=0.0):
    nz, ny, nx = shape
    p = oracle.Params(nx, ny, nz, tau=tau, G=G, Fext=F)
    ns = np.stack([np.full(shape, ns_pair[0]), np.full(shape, ns_pair[1])])
    s = oracle.Sim(p, ns, np.full(shape, gads))
    f = np.zeros((2, 19) + shape)
    for sg in range(2):
        f[sg] = oracle.feq(rho[sg], np.array(u[sg], float))[:, None, None, None]
    s.set_populations(f)
    return s


def _component_momentum(f):
    c, _, _ = oracle.lattice()
    return np.einsum("sizyx,id->sdzyx", f, c.astype(np.float64))


@pytest.mark.parametrize("ns_pair,tau", [((0.2, 0.05), (1.0, 0.8)),
                                         ((0.0, 0.6), (0.7, 1.4)),
                                         ((0.9, 0.3), (1.3, 1.0))])
def test_per_component_darcy_recurrence(ns_pair, tau):
    """Uniform medium, uniform densities, n_s,1 != n_s,2.  Eq. 1 summed over
    i with first-moment weights gives, per component (omega = 1/tau, bounce-
    back reverses momentum, Eqs. 5-6 with F_inter = F_ads = 0):
      j_s' = [(1 - n_s)(1 - omega_s) - n_s] j_s
             + (1 - n_s) omega_s rho_s u' + (1 - n_s) rho_s F / rho,
      u'   = (sum_s omega_s j_s) / (sum_s omega_s rho_s),
    a 2 x 2 linear recurrence iterated here in plain float64; Eq. 7 then gives
    rho u_macro = sum_s (1 - n_s)(j_s + rho_s F / (2 rho))."""
    rho = (0.7, 0.3)
    F = np.array([1e-5, -2e-5, 3e-6])
    u0 = ((0.01, -0.02, 0.005), (-0.03, 0.01, 0.0))
    s = _per_component_sim((3, 2, 4), ns_pair, tau, 0.5, tuple(F), rho, u0, gads=0.15)
    om = [1.0 / t for t in tau]
    rt = rho[0] + rho[1]
    j = [rho[k] * np.array(u0[k]) for k in range(2)]
    for n in range(1, 41):
        up = (om[0] * j[0] + om[1] * j[1]) / (om[0] * rho[0] + om[1] * rho[1])
        j = [((1 - ns_pair[k]) * (1 - om[k]) - ns_pair[k]) * j[k]
             + (1 - ns_pair[k]) * om[k] * rho[k] * up
             + (1 - ns_pair[k]) * rho[k] * F / rt for k in range(2)]
        s.step(1)
        if n in (1, 2, 7, 40):
            got = _component_momentum(s.f)[:, :, 0, 0, 0]
            for k in range(2):
                assert np.allclose(got[k], j[k], rtol=1e-11, atol=1e-17), (n, k)
            fl = s.fields()
            rho_u = fl["u"][:, 0, 0, 0] * rt
            expect = sum((1 - ns_pair[k]) * (j[k] + rho[k] * F / (2 * rt))
                         for k in range(2))
            assert np.allclose(rho_u, expect, rtol=1e-11, atol=1e-17)


def test_membrane_blocks_only_its_component():
    """Two membrane planes (x = 0 and x = 8: n_s,2 = 1, n_s,1 = 0) split a
    periodic box into A (x = 1..7) and B (x = 9..15).  A full bounce-back
    node returns every population of fluid 2 to the side it came from, so
    fluid 2's content of B -- its densities in B plus the populations at the
    membranes that arrived from B -- never changes, whatever G does; fluid 1
    crosses freely and equalises between the sides (Sec. 4 membranes)."""
    nx, shape = 16, (3, 4, 16)
    c, _, _ = oracle.lattice()
    x = np.arange(nx)
    memb = (x == 0) | (x == 8)
    B = (x >= 9)
    ns = np.zeros((2,) + shape)
    ns[1][..., memb] = 1.0
    ra = np.where(B, 0.8, 0.5) * np.ones(shape)
    rb = np.where(B, 0.1, 0.4) * np.ones(shape)
    p = oracle.Params(nx, 4, 3, tau=(1.0, 0.9), G=0.4)
    s = oracle.Sim(p, ns, np.zeros(shape))
    s.init_equilibrium(ra, rb)

    def content_B(f, sg):
        tot = f[sg][..., B].sum()
        into8 = [i for i in range(19) if c[i, 0] == -1]   # arrived at x=8 from x=9
        into0 = [i for i in range(19) if c[i, 0] == 1]    # arrived at x=0 from x=15
        return tot + f[sg][into8][..., 8].sum() + f[sg][into0][..., 0].sum()

    m2 = content_B(s.f, 1)
    m1 = content_B(s.f, 0)
    s.step(300)
    assert abs(content_B(s.f, 1) - m2) <= 1e-12 * m2
    rho1 = s.f[0].sum(axis=0)
    # fluid 1 has flowed from B (0.8) into A (0.5)
    assert content_B(s.f, 0) < m1 - 0.05 * (m1 - 0.5 / 0.8 * m1)
    assert rho1[..., 1:8].mean() > 0.52


def test_adhesion_indicator_is_the_components_own_fraction():
    """Eq. 4 with s = n_s,sigma: when n_s,2 is uniform its adhesion sum
    vanishes, so F_tot,2 does not depend on G_ads while F_tot,1 (varying
    n_s,1) does."""
    shape = (4, 5, 6)
    rng = np.random.default_rng(3)
    ns = np.stack([rng.uniform(0, 0.8, shape), np.full(shape, 0.3)])
    ra = rng.uniform(0.2, 0.8, shape)
    rb = 1.0 - ra
    out = []
    for gads in (0.0, 0.12):
        p = oracle.Params(6, 5, 4, tau=(1.0, 1.0), G=1.0)
        s = oracle.Sim(p, ns, np.full(shape, gads))
        s.init_equilibrium(ra, rb)
        out.append(s.fields()["ftot"])
    # the uniform sum vanishes up to FP64 rounding of the unpaired terms
    assert np.abs(out[0][1] - out[1][1]).max() < 1e-15
    assert np.abs(out[0][0] - out[1][0]).max() > 1e-3


# --------------------------------------------------------------------------
# Velocity boundary cells: Couette flow in a homogeneous gray medium
# (Sec. 3.1, Eq. 14)
# --------------------------------------------------------------------------

def _couette_profile(ns, steps, H=50, U0=0.01):
    """Channel of H + 1 node layers along x: boundary cells x = 0 (u = 0)
    and x = H (u = U0 along y) held at equilibrium at that velocity, the
    medium n_s in between, periodic along y; G = 0, fluid 2 dissolved only.
    Returns u_y(x) (Eq. 7)."""
    nx = H + 1
    res = {0: (1, 1.0, 0.01, (0.0, 0.0, 0.0)), 1: (1, 1.0, 0.01, (0.0, U0, 0.0))}
    p = oracle.Params(nx, 4, 1, tau=(1.0, 1.0), G=0.0, reservoirs=res)
    ns_f = np.full((1, 4, nx), ns)
    ns_f[..., 0] = ns_f[..., H] = 0.0
    s = oracle.Sim(p, ns_f)
    s.init_equilibrium(np.full((1, 4, nx), 1.0), np.full((1, 4, nx), 0.01))
    s.step(steps)
    return s.fields()["u"][1, 0, 0, :]


def test_couette_without_medium_is_linear():
    """n_s = 0: the steady Couette profile between the velocity cells is the
    straight line U0 x / H (to the decay of the slowest transient mode,
    exp(-nu (pi/H)^2 t) ~ 2e-6 after 20000 steps)."""
    H, U0 = 50, 0.01
    u = _couette_profile(0.0, 20000)
    x = np.arange(H + 1)
    assert np.abs(u - U0 * x / H).max() <= 1e-5 * U0
    assert abs(u[0]) <= 1e-15 and abs(u[H] - U0) <= 1e-15


@pytest.mark.parametrize("ns", [0.001, 0.01, 0.1, 0.5, 0.9])
def test_couette_brinkman_profile_eq14(ns):
    """Eq. 14: u = U0 sinh(r x) / sinh(r H), r = sqrt(2 n_s / nu).  The paper
    reports agreement in the Brinkman regime and deviations next to the
    moving boundary for larger n_s; held here to 3 % of U0 everywhere and
    0.5 % of U0 for x <= 0.9 H."""
    H, U0, nu = 50, 0.01, 1.0 / 6.0
    u = _couette_profile(ns, 20000 if ns < 0.005 else 6000)
    x = np.arange(H + 1)
    r = math.sqrt(2 * ns / nu)
    ua = U0 * np.sinh(r * x) / math.sinh(r * H)
    err = np.abs(u - ua)
    assert err.max() <= 0.03 * U0, err.max() / U0
    assert err[x <= 0.9 * H].max() <= 0.005 * U0


# --------------------------------------------------------------------------
# Washburn imbibition (Sec. 3.4, Eq. 16, Table 3)
# --------------------------------------------------------------------------

def _washburn_front(gads, ns, H=500, steps=50000, samples=20):
    """Imbibition along x into a homogeneous gray medium (n_s, G_ads uniform)
    between an inlet reservoir of fluid 1 (x = 0..3) and an outlet reservoir
    of fluid 2 (x = H-4..H-1), the reservoir layers free of medium; the
    domain is uniform across y (periodic), so one row suffices.  Returns
    sample times and the interface position (rho_1 = 0.5, interpolated)
    measured from the medium's face."""
    res = {0: (4, 0.99, 0.01), 1: (4, 0.01, 0.99)}
    p = oracle.Params(H, 1, 1, tau=(1.0, 1.0), G=1.75, reservoirs=res)
    x = np.arange(H)
    medium = (x >= 4) & (x < H - 4)
    s = oracle.Sim(p, np.where(medium, ns, 0.0)[None, None],
                   np.where(medium, gads, 0.0)[None, None])
    ra = np.where(x < 4, 0.99, 0.01)[None, None] * 1.0
    rb = np.where(x < 4, 0.01, 0.99)[None, None] * 1.0
    s.init_equilibrium(ra, rb)
    ts, xs = [], []
    for _ in range(samples):
        s.step(steps // samples)
        r1 = s.f[0].sum(axis=0)[0, 0]
        pos = 0.0
        for k in range(4, H - 5):
            if r1[k] >= 0.5 > r1[k + 1]:
                pos = k - 4 + 0.5 + (r1[k] - 0.5) / (r1[k] - r1[k + 1])
                break
        ts.append(s.t)
        xs.append(pos)
    return np.array(ts, float), np.array(xs)


def _washburn_fit(ts, xs):
    """x^2 = a t through the origin (Eq. 16 squared: a = A^2 B) and the R^2
    of x against its fit."""
    a = float((xs ** 2) @ ts / (ts @ ts))
    fit = np.sqrt(a * ts)
    r2 = 1 - ((xs - fit) ** 2).sum() / ((xs - xs.mean()) ** 2).sum()
    return a, r2


@pytest.mark.slow
def test_washburn_fronts_follow_table3():
    """Reading of the garbled set-up (H = 500 lu of medium with reservoirs at
    both ends, imbibition along x, uniform n_s and G_ads): the front follows
    x ~ sqrt(t) (R^2 > 0.97, the paper's criterion), and Eq. 16 fitted the
    paper's way reproduces Table 3 -- A (with B held at the table's
    R_eff(0.5)) within 10 % for G_ads = 0.05, 0.2, 0.4 at n_s = 0.5, and B
    (with A held at the table's A(0.2)) within 10 % for n_s = 0.1 and 20 %
    for n_s = 0.9, the fit the paper rates lowest (R_B^2 = 0.972).  An
    adhesion force of the wrong sign or taken at the wrong node stops or
    reverses the front; a slip in Eq. 2's permeability moves B."""
    t3 = _golden("washburn_fits_table3.txt")
    A_tab = {round(g, 2): v for k, g, v in t3 if k == 0}
    B_tab = {round(n, 2): v for k, n, v in t3 if k == 1}
    A_prev = 0.0
    for gads in (0.05, 0.2, 0.4):
        a, r2 = _washburn_fit(*_washburn_front(gads, 0.5))
        A = math.sqrt(a / B_tab[0.5])
        assert r2 > 0.97, (gads, r2)
        assert abs(A / A_tab[gads] - 1) < 0.10, (gads, A, A_tab[gads])
        assert A > A_prev
        A_prev = A
    for ns, tol in ((0.1, 0.10), (0.9, 0.20)):
        a, r2 = _washburn_fit(*_washburn_front(0.2, ns))
        B = a / A_tab[0.2] ** 2
        assert r2 > 0.97, (ns, r2)
        assert abs(B / B_tab[ns] - 1) < tol, (ns, B, B_tab[ns])


# --------------------------------------------------------------------------
# Buckley-Leverett waterflooding (SI: Buckley-Leverett experiment)
# --------------------------------------------------------------------------

def test_buckley_leverett_solution_closed_forms():
    """The analytic side the oracle is held to: Welge's tangent from S = 0
    for k_r = S^2, (1 - S)^2 touches f at S_f = 1/sqrt(2) with speed factor
    (1 + sqrt(2))/2 (f(S)/S = f'(S) solved by hand); the solution conserves
    the injected volume (integral of S over x equals Q at porosity 1, the
    Welge balance); and the paper's bounds a = 1.01 and 1.3 give shocks of
    speed factor just above 1 and about 1.08, a=1.01 the faster-filling."""
    from paper_2206_11524_gb300 import studies
    Sf, sp = studies.bl_welge(2.0)
    assert abs(Sf - 1 / math.sqrt(2)) < 1e-12
    assert abs(sp - (1 + math.sqrt(2)) / 2) < 1e-12
    for a in (1.01, 1.3, 2.0):
        Sf, sp = studies.bl_welge(a)
        assert abs(studies.bl_dfds(Sf, a) - sp) < 1e-9        # tangent
        x = np.linspace(0, 60, 600001)
        S = studies.bl_profile(x, 40.0, a)
        vol = float(np.sum(0.5 * (S[1:] + S[:-1])) * (x[1] - x[0]))
        assert abs(vol / 40.0 - 1) < 2e-3, (a, vol)
        assert S[0] == 1.0 and S[-1] == 0.0
    assert 1.0 < studies.bl_welge(1.01)[1] < 1.01
    assert 1.07 < studies.bl_welge(1.3)[1] < 1.08


def _bl_oracle(ns, H=100, steps=100000, samples=20):
    """The waterflooding set-up (displacement along x, F = 1e-4 along x,
    coexistence densities held at both ends, uniform n_s, G_ads = 0; one
    row, the y extent being periodic and the state uniform in y) on the
    oracle.  Returns fronts (S = 0.5, as x), injected volume Q (trapezoid of
    the medium's mean Eq. 7 velocity) and the last saturation profile."""
    hi, lo = 0.98739, 0.03548
    res = {0: (4, hi, lo), 1: (4, lo, hi)}
    s = oracle.Sim(oracle.Params(H, 1, 1, tau=(1.0, 1.0), G=1.75, Fext=(1e-4, 0, 0),
                                 reservoirs=res), np.full((1, 1, H), ns))
    x = np.arange(H)
    ra = np.where(x < 4, hi, lo)[None, None] * 1.0
    s.init_equilibrium(ra, hi + lo - ra)
    fronts, Q, q_prev = [4.0], [0.0], 0.0
    for _ in range(samples):
        s.step(steps // samples)
        fl = s.fields()
        S = (fl["rho_a"][0, 0] - lo) / (hi - lo)
        q = float(fl["u"][0, 0, 0][4:H - 4].mean())
        Q.append(Q[-1] + 0.5 * (q + q_prev) * (steps // samples))
        q_prev = q
        front = 4.0
        for k in range(4, H - 1):
            if S[k] >= 0.5 > S[k + 1]:
                front = k + (S[k] - 0.5) / (S[k] - S[k + 1])
                break
        fronts.append(front)
    return np.array(fronts), np.array(Q), S


@pytest.mark.slow
@pytest.mark.parametrize("ns, min_dQ", [(0.1, 20.0), (0.5, 2.5)])
def test_buckley_leverett_front_between_the_papers_bounds(ns, min_dQ):
    """The oracle's waterflooding over 100,000 steps: fluid 1 advances with
    the Darcy flux (the injected volume grows by more than min_dQ lu), the
    front's displacement over the last four fifths of the run lies between
    the injected volume times the shock speed factors of the paper's bounds
    a = 1.01 and 1.3, give or take 0.5 lu (the diffuse interface, ~3 lu
    wide, settles by a fraction of a node), and behind the front the
    saturation lies between the a = 1.3 profile and the (piston-like)
    a = 1.01 one, ahead of it fluid 2 remains.  A dropped force term stops
    the front; a wrong half-force term in Eq. 7 shifts q by ~12 % (more at
    n_s = 0.5), which moves the band by more than 0.5 lu."""
    from paper_2206_11524_gb300 import studies
    fr, Q, S = _bl_oracle(ns)
    k0 = 4
    dQ = Q[-1] - Q[k0]
    assert dQ > min_dQ, dQ
    shift = fr[-1] - fr[k0]
    lo_b, hi_b = studies.bl_welge(1.01)[1], studies.bl_welge(1.3)[1]
    assert lo_b * dQ - 0.5 < shift < hi_b * dQ + 0.5, (shift, dQ)
    x = np.arange(len(S))
    behind = (x >= 4) & (x < fr[-1] - 3)
    ahead = (x > fr[-1] + 3) & (x < len(S) - 4)
    low = studies.bl_profile(x - 4.0, Q[-1], 1.3)
    assert behind.sum() >= 2 and ahead.sum() >= 10
    assert np.all(S[behind] >= low[behind] - 0.02), (S[behind], low[behind])
    assert np.all(S[behind] <= 1.005)
    assert np.all(np.abs(S[ahead]) <= 0.02)


# --------------------------------------------------------------------------
# Sessile droplet contact angle against Eq. 15 (Sec. 3.4, Table 3's theta_H)
# --------------------------------------------------------------------------

def _sessile_theta(gads, nx=80, ny=48, R=14, steps=12000, wall=3):
    """A 2D droplet of fluid 1 (coexistence densities at G = 1.75) started
    as a half disc on a wall of `wall` rows with n_s = 1 and adhesion
    G_ads,2 = gads (a second, neutral wall closes the top; x periodic); the
    wall cells start nearly empty (1e-6 of each fluid: solid nodes without
    fluid, as in the multicomponent Shan-Chen droplets Eq. 15 was derived
    from; an empty cell has no velocity, Eq. 6).  The angle of the circular
    cap from its height h on the centre column and the half-width a of its
    base on the first fluid row: theta = 2 atan(h / a)."""
    hi, lo = 0.98739, 0.03548
    ns = np.zeros((1, ny, nx))
    ga = np.zeros((1, ny, nx))
    ns[0, :wall] = 1.0
    ga[0, :wall] = gads
    ns[0, ny - wall:] = 1.0
    y, x = np.mgrid[0:ny, 0:nx]
    r = np.hypot(x - (nx / 2 - 0.5), y - (wall - 0.5))
    ra = np.where((r < R) & (y >= wall), hi, lo)[None] * 1.0
    rb = hi + lo - ra
    ra[ns > 0.5] = 1e-6
    rb[ns > 0.5] = 1e-6
    s = oracle.Sim(oracle.Params(nx, ny, 1, tau=(1.0, 1.0), G=1.75), ns, ga)
    s.init_equilibrium(ra, rb)
    s.step(steps)
    r1 = s.fields()["rho_a"][0]
    mid = 0.5 * (hi + lo)
    col = 0.5 * (r1[:, nx // 2 - 1] + r1[:, nx // 2])
    h = next(k + (col[k] - mid) / (col[k] - col[k + 1]) for k in range(wall, ny - 1)
             if col[k] >= mid > col[k + 1]) - (wall - 0.5)
    row = r1[wall]
    xs = [k + (row[k] - mid) / (row[k] - row[k + 1]) for k in range(nx - 1)
          if (row[k] - mid) * (row[k + 1] - mid) < 0]
    a = (max(xs) - min(xs)) / 2
    return math.degrees(2 * math.atan2(h, a))


@pytest.mark.slow
def test_sessile_droplet_contact_angle_follows_eq15():
    """The oracle's sessile droplets against Eq. 15, cos theta_H = 4 G_ads,2
    / (G (rho_1 - rho_dis,2)): a neutral wall gives 90 deg (within 3), and
    G_ads,2 = +-0.2 give angles within 10 deg of theta_H = 61.3 / 118.7 deg
    (the paper calls the correlation approximate and sees deviations of
    this size, Table 3), on the right side of 90.  A sign error in the
    adhesion force swaps the two; a dropped adhesion term leaves all at
    90; adhesion half as strong gives 72.8 deg at G_ads,2 = 0.2 (11.5 off),
    twice as strong spreads the droplet into a film."""
    hi, lo, G = 0.98739, 0.03548, 1.75
    th0 = _sessile_theta(0.0)
    assert abs(th0 - 90.0) < 3.0, th0
    for gads in (0.2, -0.2):
        th = _sessile_theta(gads)
        th_h = math.degrees(math.acos(4 * gads / (G * (hi - lo))))
        assert abs(th - th_h) < 10.0, (gads, th, th_h)
        assert (th < th0) == (gads > 0), (gads, th, th0)
