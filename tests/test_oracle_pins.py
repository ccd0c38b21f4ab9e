"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms (the paper's two-particle oscillator, Eq. 6), finite differences of the
potential (Eq. 1 vs Eq. 2), Newton's third law, energy conservation of
velocity Verlet (Section 2.2), an independent linear static solve, the
paper's spring table (Section 3.1), and brute-force enumeration of the
lattice. A plausible slip in the oracle (a dropped term, a wrong sign, a
wrong index or factor) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from gen.images import inclusion_image, one_phase_materials, two_phase_materials

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_kv(name):
    out = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split()
            out[key] = float(val)
    return out


def _read_table(name):
    rows = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows[parts[0]] = tuple(float(p) for p in parts[1:])
    return rows


# ------------------------------------------------------------ lattice build

def _brute_springs(phase, k_tab, e_tab, k2_ratio, a):
    """Every pair of occupied sites at squared lattice distance 1 or 2,
    enumerated over all pairs (not via forward offsets)."""
    if phase.ndim == 2:
        phase = phase[None]
    nz, ny, nx = phase.shape
    sites = [(ix, iy, iz) for iz in range(nz) for iy in range(ny) for ix in range(nx)
             if phase[iz, iy, ix]]
    index = {s: t for t, s in enumerate(sites)}
    springs = {}
    for (i, si) in enumerate(sites):
        for (j, sj) in enumerate(sites):
            if j <= i:
                continue
            d2 = sum((u - w) ** 2 for u, w in zip(si, sj))
            if d2 not in (1, 2):
                continue
            pi = phase[si[2], si[1], si[0]]
            pj = phase[sj[2], sj[1], sj[0]]
            k = k_tab[pi - 1, pj - 1] * (k2_ratio if d2 == 2 else 1.0)
            r0 = a * math.sqrt(d2)
            rc = r0 * (1.0 + e_tab[pi - 1, pj - 1])
            springs[(i, j)] = (k, r0, rc * rc)
    assert len(index) == len(sites)
    return sites, springs


@pytest.mark.parametrize("shape,seed", [((7, 6), 0), ((4, 3, 5), 1)])
def test_build_matches_brute_force(oracle_mod, shape, seed):
    rng = np.random.default_rng(seed)
    phase = rng.integers(0, 3, size=shape).astype(np.uint8)  # voids included
    k_tab = np.array([[1.0, 0.3], [0.3, 0.1]])
    e_tab = np.array([[0.05, 0.2], [0.2, 0.3]])
    o = oracle_mod.Oracle.from_image(phase, k_tab, e_tab, k2_ratio=0.5, a=1.5)
    sites, springs = _brute_springs(phase, k_tab, e_tab, 0.5, 1.5)
    t = o.topology()
    assert o.n == len(sites)
    assert o.m == len(springs)
    keys = sorted(springs)
    assert list(zip(t["si"].tolist(), t["sj"].tolist())) == keys  # canonical order
    for s, key in enumerate(keys):
        k, r0, rc2 = springs[key]
        assert t["k"][s] == k
        assert t["r0"][s] == pytest.approx(r0, rel=1e-15)
        assert t["rc2"][s] == pytest.approx(rc2, rel=1e-14)
    # reference positions of the raster-order particles
    for p, (ix, iy, iz) in enumerate(sites):
        assert t["X"][0, p] == ix * 1.5 and t["X"][1, p] == iy * 1.5


def test_spring_count_closed_form(oracle_mod):
    # full nx x ny image: (nx-1)ny + nx(ny-1) first + 2(nx-1)(ny-1) second neighbours
    for nx, ny in [(64, 64), (5, 9)]:
        o = oracle_mod.Oracle.from_image(np.ones((ny, nx), np.uint8), [[1.0]], [[0.1]])
        assert o.m == (nx - 1) * ny + nx * (ny - 1) + 2 * (nx - 1) * (ny - 1)
    # full cube: 3 face families + 6 edge-diagonal families
    n = 5
    o = oracle_mod.Oracle.from_image(np.ones((n, n, n), np.uint8), [[1.0]], [[0.1]])
    assert o.m == 3 * (n - 1) * n * n + 6 * (n - 1) * (n - 1) * n
    assert o.n == n ** 3


def test_reference_config_sizes(oracle_mod):
    img = inclusion_image(64, 64, 3.0, 8.0, 0.30, 0)
    k, e, m = two_phase_materials()
    o = oracle_mod.Oracle.from_image(img, k, e, m)
    assert o.n == 4096 and o.m == 16002
    assert 0.30 <= (img == 2).mean() < 0.40


# ---------------------------------------------------------- force / energy

def _perturbed_lattice(oracle_mod, shape, seed, amp=0.05):
    rng = np.random.default_rng(seed)
    phase = rng.integers(1, 3, size=shape).astype(np.uint8)
    k_tab = np.array([[1.0, 0.4], [0.4, 0.1]])
    e_tab = np.full((2, 2), 10.0)  # nothing breaks
    o = oracle_mod.Oracle.from_image(phase, k_tab, e_tab, k2_ratio=0.7)
    x, _, _ = o.state()
    x = x + amp * rng.standard_normal(x.shape)
    return o, x


@pytest.mark.parametrize("shape,seed", [((5, 5), 3), ((3, 3, 3), 4)])
def test_force_is_minus_energy_gradient(oracle_mod, shape, seed):
    """Eq. 2 is the negative gradient of Eq. 1 (central differences)."""
    o, x = _perturbed_lattice(oracle_mod, shape, seed)
    F, U, _ = o.forces(x)
    h = 1e-6
    fd = np.zeros_like(x)
    for c in range(x.shape[0]):
        for p in range(x.shape[1]):
            xp = x.copy(); xp[c, p] += h
            xm = x.copy(); xm[c, p] -= h
            fd[c, p] = -(o.forces(xp)[1] - o.forces(xm)[1]) / (2 * h)
    scale = np.abs(F).max()
    assert scale > 1e-3
    assert np.abs(F - fd).max() <= 1e-7 * scale


@pytest.mark.parametrize("shape,seed", [((6, 7), 5), ((3, 4, 3), 6)])
def test_newton_third_law(oracle_mod, shape, seed):
    o, x = _perturbed_lattice(oracle_mod, shape, seed)
    F, _, _ = o.forces(x)
    total = F.sum(axis=1)
    assert np.abs(total).max() <= 1e-14 * np.abs(F).sum()


def test_single_spring_direction_and_tension_sign(oracle_mod):
    # one stretched spring along a random direction: the force on the lower
    # particle points to the other one (tension), magnitude is linear in stretch
    X = np.array([[0.0, 1.0], [0.0, 0.0]])
    o = oracle_mod.Oracle.from_network(X, [0], [1], [2.0], [1.0], [np.inf])
    th = 0.3
    for r in (1.1, 1.2):
        x = np.array([[0.0, r * math.cos(th)], [0.0, r * math.sin(th)]])
        F, U, _ = o.forces(x)
        f0 = F[:, 0]
        assert f0 @ np.array([math.cos(th), math.sin(th)]) > 0
        assert np.hypot(*f0) == pytest.approx(2.0 * (r - 1.0), rel=1e-13)
        assert U == pytest.approx(0.5 * 2.0 * (r - 1.0) ** 2, rel=1e-13)
        assert np.allclose(F[:, 1], -f0, rtol=0, atol=0)


# -------------------------------------------------------------- integrator

def test_paper_oscillator_closed_form(oracle_mod):
    """The paper's two-particle oscillator (Eq. 6): velocity Verlet on a
    linear spring gives y_n = y_0 cos(n theta) exactly, cos theta = 1 - (w dt)^2/2,
    and stays within O((w dt)^2) of the continuous cosine over the run."""
    g = _read_kv("paper_oscillator.txt")
    X = np.array([[0.0, g["x_start"]], [0.0, 0.0]])
    fix = np.array([[1, 0], [1, 0]], np.uint8)
    o = oracle_mod.Oracle.from_network(X, [0], [1], [g["k"]], [g["r0"]], [np.inf],
                                       mass=[g["m"], g["m"]], fix=fix, dt=g["dt"], damping=0.0)
    w = math.sqrt(g["k"] / g["m"])
    theta = math.acos(1.0 - 0.5 * (w * g["dt"]) ** 2)
    y0 = g["x_start"] - g["r0"]
    n_out = int(round(g["t_out"] / g["dt"]))
    n_end = int(round(g["t_end"] / g["dt"]))
    worst_exact, worst_cont = 0.0, 0.0
    for n in range(n_out, n_end + 1, n_out):
        o.step(n_out)
        x, v, _ = o.state()
        y = x[0, 1] - g["r0"]
        worst_exact = max(worst_exact, abs(y - y0 * math.cos(n * theta)))
        worst_cont = max(worst_cont, abs(y - y0 * math.cos(w * n * g["dt"])))
        assert x[1, 1] == 0.0 and x[0, 0] == 0.0
    assert worst_exact <= 1e-12 * y0
    assert worst_cont <= 1e-3 * y0 and worst_cont > 1e-9 * y0


def _damped_error(oracle_mod, dt, t_end=60.0, k=1.0, gamma=0.3):
    X = np.array([[0.0, 2.0], [0.0, 0.0]])
    fix = np.array([[1, 0], [1, 1]], np.uint8)
    o = oracle_mod.Oracle.from_network(X, [0], [1], [k], [1.0], [np.inf], fix=fix, dt=dt,
                                       damping=gamma)
    nsteps = int(round(t_end / dt))
    o.step(nsteps)
    y = o.state()[0][0, 1] - 1.0
    # m y'' + gamma y' + k y = 0, y(0)=1, y'(0)=0 (underdamped, m = 1)
    wd = math.sqrt(k - 0.25 * gamma * gamma)
    t = nsteps * dt
    exact = math.exp(-0.5 * gamma * t) * (math.cos(wd * t) + 0.5 * gamma / wd * math.sin(wd * t))
    return abs(y - exact), abs(exact)


def test_viscous_damping_converges_to_damped_oscillator(oracle_mod):
    """Damping -gamma*vh: the discrete solution tends to the continuous damped
    oscillator as dt -> 0 (first order, since the drag uses the half-step
    velocity). A wrong sign or factor on gamma gives an O(1) error instead."""
    e1, scale = _damped_error(oracle_mod, 0.02)
    e2, _ = _damped_error(oracle_mod, 0.01)
    assert e1 < 5e-3 * max(scale, 1e-6) + 1e-5
    assert 1.6 < e1 / e2 < 2.4


def _energy_drift(oracle_mod, dt, t_end=40.0):
    rng = np.random.default_rng(7)
    phase = rng.integers(1, 3, size=(6, 6)).astype(np.uint8)
    k_tab = np.array([[1.0, 0.4], [0.4, 0.2]])
    o = oracle_mod.Oracle.from_image(phase, k_tab, np.full((2, 2), 10.0), grip_mode=1,
                                     dt=dt, damping=0.0)
    x, v, a = o.state()
    _, _, _ = o.forces(x)
    t = o.topology()
    v = 0.05 * rng.standard_normal(v.shape) * (1 - t["fix"])
    x = x + 0.02 * rng.standard_normal(x.shape) * (1 - t["fix"])
    F, _, _ = o.forces(x)
    o.set_state(x=x, v=v, a=F / t["mass"][None, :] * (1 - t["fix"]))
    ob = o.observe()
    e0 = ob["pe"] + ob["ke"]
    worst = 0.0
    n = int(round(t_end / dt))
    for _ in range(20):
        o.step(n // 20)
        ob = o.observe()
        worst = max(worst, abs(ob["pe"] + ob["ke"] - e0))
    return worst / e0


def test_energy_conserved_without_damping(oracle_mod):
    """Velocity Verlet is symplectic: no secular drift and an O(dt^2) energy error."""
    d1 = _energy_drift(oracle_mod, 0.1)
    d2 = _energy_drift(oracle_mod, 0.05)
    assert d1 < 5e-3
    assert 3.0 < d1 / d2 < 5.0


# --------------------------------------------------- statics and the modulus

def _stiffness(t, x):
    """Linear stiffness matrix of the intact network about positions x
    (independent of the oracle's force routine)."""
    dim, n = x.shape
    K = np.zeros((dim * n, dim * n))
    for s in range(t["si"].size):
        i, j = int(t["si"][s]), int(t["sj"][s])
        d = x[:, j] - x[:, i]
        e = d / np.linalg.norm(d)
        kk = t["k"][s] * np.outer(e, e)
        ii = [c * n + i for c in range(dim)]
        jj = [c * n + j for c in range(dim)]
        K[np.ix_(ii, ii)] += kk
        K[np.ix_(jj, jj)] += kk
        K[np.ix_(ii, jj)] -= kk
        K[np.ix_(jj, ii)] -= kk
    return K


@pytest.mark.parametrize("shape", [(8, 8), (4, 4, 4)])
def test_relaxed_state_matches_linear_static_solve(oracle_mod, shape):
    """At small strain the relaxed oracle state equals the solution of
    K u = 0 with prescribed grip displacements, up to O(eps) geometric terms.
    Also: the virial stress equals the grip traction at equilibrium."""
    k_tab, e_tab, mass = one_phase_materials(1.0, 0.5)
    o = oracle_mod.Oracle.from_image(np.ones(shape, np.uint8), k_tab, e_tab, mass,
                                     dt=0.2, damping=0.35)
    eps = 1e-6
    o.apply_strain(eps)
    st, taken = o.relax(tol=1e-13, max_steps=200000, check_every=50)
    assert st == 0, taken
    t = o.topology()
    X = t["X"]
    x, _, _ = o.state()
    u = (x - X).reshape(-1)
    K = _stiffness(t, X)
    fixed = t["fix"].reshape(-1).astype(bool)
    u_fix = np.zeros_like(u)
    xc = 0.5 * (shape[-1] - 1)
    u_fix[: X.shape[1]] = eps * (X[0] - xc)
    u_fix[~fixed] = 0.0
    free = ~fixed
    rhs = -K[np.ix_(free, fixed)] @ u_fix[fixed]
    u_free = np.linalg.lstsq(K[np.ix_(free, free)], rhs, rcond=None)[0]
    u_lin = u_fix.copy()
    u_lin[free] = u_free
    # remove the zero-stiffness rigid translations the min-norm solve fixes
    # differently (none are excited: the start is at rest and symmetric)
    err = np.abs(u - u_lin).max() / np.abs(u_lin).max()
    assert err < 1e-5
    ob = o.observe()
    R = -(K @ u_lin)  # reaction on the right grip, x components
    right = (t["grip"] == 2)
    area = np.prod(shape[:-1])
    sig_lin = -(K @ u_lin)[: X.shape[1]][right].sum() * -1.0 / area
    assert ob["sigma_grip"] == pytest.approx(sig_lin, rel=1e-5)
    # static equilibrium: the internal virial equals the grip reaction times the
    # current grip separation, so sigma_vir = sigma_grip (1 + eps) exactly
    assert ob["sigma_vir"] == pytest.approx(ob["sigma_grip"] * (1 + eps), rel=1e-8)
    assert R.shape == u.shape


def test_square_lattice_modulus_tends_to_three_halves_k(oracle_mod):
    """Uniform square lattice, equal first/second-neighbour k, roller grips:
    the effective Young's modulus of the affine continuum limit is 1.5 k
    (C11 = 2k, C12 = C66 = k, plane problem). A 32x32 specimen is within 1%."""
    n = 32
    k_tab, e_tab, mass = one_phase_materials(1.0, 0.5)
    o = oracle_mod.Oracle.from_image(np.ones((n, n), np.uint8), k_tab, e_tab, mass,
                                     dt=0.3, damping=0.15)
    eps = 1e-6
    o.apply_strain(eps)
    st, taken = o.relax(tol=1e-13, max_steps=400000, check_every=100)
    assert st == 0
    ob = o.observe()
    # sigma over the reference box is R / (ny a); R / (eps ny) -> E as n grows,
    # with the grips' own stiffness contributing O(1/n)
    modulus = ob["sigma_grip"] / eps
    assert modulus == pytest.approx(1.5, rel=0.012)
    assert ob["sigma_vir"] == pytest.approx(ob["sigma_grip"] * (1 + eps), rel=1e-8)


def test_cubic_lattice_modulus_tends_to_five_halves_k(oracle_mod):
    """Uniform cubic lattice with its 3 face and 6 edge-diagonal springs per
    particle, equal k: the affine continuum limit has C11 = 3k, C12 = C44 = k
    (per bond, k r0^2 n_i n_j n_k n_l over the cell volume), so uniaxial stress
    gives E = (C11 - C12)(C11 + 2 C12) / (C11 + C12) = 2.5 k. The free lateral
    surfaces soften finite cubes by O(1/n); a fit E(n) = E + c1/n + c2/n^2
    over n = 16, 24, 32 recovers the limit."""
    k_tab, e_tab, mass = one_phase_materials(1.0, 0.5)
    ns, es = [16, 24, 32], []
    eps = 1e-6
    for n in ns:
        o = oracle_mod.Oracle.from_image(np.ones((n, n, n), np.uint8), k_tab, e_tab, mass, dt=0.3, damping=0.15)
        o.apply_strain(eps)
        st, _ = o.relax(tol=1e-13, max_steps=20000, check_every=100)  # converges in ~800
        assert st == 0
        ob = o.observe()
        assert ob["sigma_vir"] == pytest.approx(ob["sigma_grip"] * (1 + eps), rel=1e-8)
        es.append(ob["sigma_grip"] / eps)
    assert es[0] < es[1] < es[2] < 2.5  # softer surfaces, less so as n grows
    A = np.array([[1.0, 1.0 / n, 1.0 / n ** 2] for n in ns])
    e_inf = np.linalg.solve(A, np.array(es))[0]
    assert e_inf == pytest.approx(2.5, rel=2e-3)


def test_cubic_lattice_poisson_ratio_is_one_quarter(oracle_mod):
    """The same cube under uniaxial stress along x contracts laterally with
    nu = C12 / (C11 + C12) = 1/4, equally in y and z (cubic symmetry): an
    affine fit of the displacement over the central 6 x 6 x 6 particles of a
    24^3 specimen, away from the free surfaces."""
    n = 24
    k_tab, e_tab, mass = one_phase_materials(1.0, 0.5)
    o = oracle_mod.Oracle.from_image(np.ones((n, n, n), np.uint8), k_tab, e_tab, mass, dt=0.3, damping=0.15)
    eps = 1e-6
    o.apply_strain(eps)
    st, _ = o.relax(tol=1e-13, max_steps=20000, check_every=100)  # converges in ~800
    assert st == 0
    x, _, _ = o.state()
    X = o.topology()["X"]
    c = (n - 1) / 2.0
    mid = np.all(np.abs(X - c) <= 2.5, axis=0)
    A = np.vstack([X[0, mid], X[1, mid], X[2, mid], np.ones(mid.sum())]).T
    grad = np.linalg.lstsq(A, (x - X)[:, mid].T, rcond=None)[0]
    nu_y, nu_z = -grad[1, 1] / grad[0, 0], -grad[2, 2] / grad[0, 0]
    assert nu_y == pytest.approx(0.25, rel=1e-2)
    assert nu_z == pytest.approx(nu_y, rel=1e-6)


def test_relaxed_energy_not_above_affine_energy(oracle_mod):
    """Minimum potential energy: with the grips fixed, the relaxed two-phase
    state stores no more energy than the affine field at the same strain."""
    img = inclusion_image(16, 16, 2.0, 4.0, 0.3, 11)
    k, e, m = two_phase_materials()
    o = oracle_mod.Oracle.from_image(img, k, e, m, dt=0.2, damping=0.3)
    o.apply_strain(0.01)
    pe_aff = o.observe()["pe"]
    st, _ = o.relax(tol=1e-12, max_steps=200000, check_every=50)
    assert st == 0
    ob = o.observe()
    assert ob["n_broken"] == 0
    assert ob["pe"] < pe_aff
    assert ob["sigma_vir"] == pytest.approx(ob["sigma_grip"] * 1.01, rel=1e-8)


# ---------------------------------------------------------------- breaking

def test_break_is_strict_and_same_step(oracle_mod):
    """A spring at exactly rc stays intact (strict '>' switch); just beyond it
    breaks in the next step and gives zero force in that step."""
    img = np.ones((1, 2), np.uint8)
    o = oracle_mod.Oracle.from_image(img, [[1.0]], [[0.5]])  # rc = 1.5
    o.step(3)
    o.apply_strain(0.5)  # grips at -0.25 and 1.25: r = 1.5 exactly
    o.step(1)
    mask, bs, fb = o.broken()
    assert mask[0] == 0 and fb == -1
    o.apply_strain(0.5 + 2.0 ** -20)
    o.step(1)
    mask, bs, fb = o.broken()
    assert mask[0] == 1 and bs[0] == 4 and fb == 4
    F, U, _ = o.forces(o.state()[0])
    assert np.all(F == 0.0) and U == 0.0


def test_paper_spring_table_break_order_and_strains(oracle_mod):
    """The paper's three fracture springs, stretched together: stiff-stiff
    breaks first (rc = 10.1), then stiff-soft (10.4), then soft-soft (11.0)."""
    tab = _read_table("paper_spring_table.txt")
    names = ["stiff-stiff", "stiff-soft", "soft-soft"]
    X = np.array([[0.0, 10.0, 0.0, 10.0, 0.0, 10.0], [0.0, 0.0, 20.0, 20.0, 40.0, 40.0]])
    k = [tab[q][0] for q in names]
    r0 = [tab[q][1] for q in names]
    rc2 = [tab[q][2] ** 2 for q in names]
    fix = np.zeros((2, 6), np.uint8)
    fix[:, :] = 1
    grip = np.array([1, 2, 1, 2, 1, 2], np.uint8)
    o = oracle_mod.Oracle.from_network(X, [0, 2, 4], [1, 3, 5], k, r0, rc2, fix=fix, grip=grip,
                                       xc=5.0, omega=10.0 * 40.0, grip_area=60.0, dt=0.1)
    order = []
    eps_at = {}
    for i in range(1, 121):
        eps = (i - 0.5) * 1e-3  # half-way between the critical strains' grid
        o.apply_strain(eps)
        o.step(1)
        mask, _, _ = o.broken()
        for s in range(3):
            if mask[s] and names[s] not in order:
                order.append(names[s])
                eps_at[names[s]] = eps
    assert order == names
    for q in names:
        crit = tab[q][2] / tab[q][1] - 1.0
        assert crit < eps_at[q] <= crit + 1e-3 + 1e-12


def test_break_is_irreversible(oracle_mod):
    img = np.ones((1, 2), np.uint8)
    o = oracle_mod.Oracle.from_image(img, [[1.0]], [[0.05]])
    o.apply_strain(0.06)
    o.step(1)
    assert o.broken()[0][0] == 1
    o.apply_strain(-0.02)  # compress the broken spring
    o.step(5)
    assert o.broken()[0][0] == 1
    F, U, _ = o.forces(o.state()[0])
    assert np.all(F == 0.0)


def test_image_rc_from_paper_constants(oracle_mod):
    """rc^2 = (r0 (1 + eps_c))^2 with r0 = a: the paper's springs (r0 = 10)
    reproduce its printed rc values."""
    tab = _read_table("paper_spring_table.txt")
    k_tab = np.array([[tab["stiff-stiff"][0], tab["stiff-soft"][0]],
                      [tab["stiff-soft"][0], tab["soft-soft"][0]]])
    e_tab = np.array([[tab["stiff-stiff"][2] / 10 - 1, tab["stiff-soft"][2] / 10 - 1],
                      [tab["stiff-soft"][2] / 10 - 1, tab["soft-soft"][2] / 10 - 1]])
    img = np.array([[1, 1, 2, 2]], np.uint8)
    o = oracle_mod.Oracle.from_image(img, k_tab, e_tab, a=10.0)
    t = o.topology()
    assert np.sqrt(t["rc2"]).tolist() == pytest.approx([10.1, 10.4, 11.0], rel=1e-14)
    assert t["k"].tolist() == [2e-3, 1.25e-4, 2e-5]


def test_virial_kinetic_term_sign(oracle_mod):
    """Eq. 7: a moving, force-free particle lowers sigma_xx by m v_x^2 / Omega."""
    X = np.array([[0.0, 1.0], [0.0, 0.0]])
    o = oracle_mod.Oracle.from_network(X, [0], [1], [1.0], [1.0], [np.inf], omega=4.0,
                                       mass=[2.0, 3.0])
    o.set_state(v=np.array([[0.5, 0.0], [0.7, 0.0]]))
    ob = o.observe()
    assert ob["sigma_vir"] == pytest.approx(-(2.0 * 0.25) / 4.0, rel=1e-15)
    assert ob["ke"] == pytest.approx(0.5 * 2.0 * (0.25 + 0.49), rel=1e-15)


def test_threaded_spring_pass_is_bit_identical(oracle_mod):
    """The threaded spring pass (per-spring forces, then each particle's
    springs in ascending order) gives the sequential scatter's bits, through
    breaks, in 2D and 3D."""
    from gen.images import foam_volume, one_phase_materials
    cases = [(inclusion_image(24, 20, 2.0, 4.0, 0.3, 3), two_phase_materials(), 1.2e-2),
             (foam_volume(10, 1.5, 0.5, seed=4), one_phase_materials(1.0, 0.02), 6e-3)]
    for img, mats, inc in cases:
        k, e, m = mats
        a = oracle_mod.Oracle.from_image(img, k, e, m)
        b = oracle_mod.Oracle.from_image(img, k, e, m)
        nt = b.set_threads(4)
        assert nt >= 1
        for i in range(1, 9):
            a.apply_strain(i * inc)
            b.apply_strain(i * inc)
            a.step(15)
            b.step(15)
        xa, va, aa = a.state()
        xb, vb, ab = b.state()
        assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(aa, ab)
        ma, sa, fa = a.broken()
        mb, sb, fb = b.broken()
        assert np.array_equal(ma, mb) and np.array_equal(sa, sb) and fa == fb
        assert ma.sum() > 0  # the run crossed breaks


# ----------------------------------------------------- fields (Eqs. 7-8)

def _interior(o, shape):
    """Indices of particles two or more sites away from every image edge
    (full images: particle index = raster index)."""
    idx = np.arange(o.n).reshape(shape)
    sl = tuple(slice(2, s - 2) for s in shape)
    return idx[sl].ravel()


def test_fields_closed_form_uniaxial_stretch(oracle_mod):
    """Uniform square lattice (k = 1, a = 1) stretched affinely by eps along x,
    at rest: an interior particle's virial stress is
      xx = k eps (1 + eps) + 2 (1 + eps)^2 k (r - sqrt 2) / r,
      yy = 2 k (r - sqrt 2) / r,  xy = 0,   r = sqrt((1 + eps)^2 + 1)
    (two axial springs and four diagonals, half of each per endpoint) and its
    Lagrangian strain is ((1 + eps)^2 - 1) / 2, 0, 0."""
    img = np.ones((10, 12), np.uint8)
    k, e, m = two_phase_materials()
    o = oracle_mod.Oracle.from_image(img, k, e, m)
    X = o.topology()["X"]
    for eps in (0.01, -0.02, 0.05):
        x = X.copy()
        x[0] *= 1.0 + eps
        o.set_state(x, np.zeros_like(x))
        st, sn = o.fields()
        r = math.sqrt((1 + eps) ** 2 + 1)
        g = (r - math.sqrt(2.0)) / r
        want_s = [eps * (1 + eps) + 2 * (1 + eps) ** 2 * g, 2 * g, 0.0]
        want_e = [((1 + eps) ** 2 - 1) / 2, 0.0, 0.0]
        for p in _interior(o, img.shape):
            assert np.allclose(st[:, p], want_s, rtol=1e-12, atol=1e-15)
            assert np.allclose(sn[:, p], want_e, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_fields_strain_of_rotated_stretch(oracle_mod, dim):
    """x = R U X (stretch U, then rotation R): every particle whose first
    shell spans the space has Lagrangian strain (U^2 - I) / 2 exactly,
    unaffected by R (a J J^T or transposed fit would see the rotation)."""
    rng = np.random.default_rng(11)
    shape = (6, 7) if dim == 2 else (4, 5, 6)
    img = np.ones(shape, np.uint8)
    from gen.images import one_phase_materials
    k, e, m = one_phase_materials(1.0, 0.5)
    o = oracle_mod.Oracle.from_image(img, k, e, m)
    X = o.topology()["X"]
    Msym = rng.standard_normal((dim, dim)) * 0.05
    U = np.eye(dim) + 0.5 * (Msym + Msym.T)
    Q, _ = np.linalg.qr(rng.standard_normal((dim, dim)))
    x = Q @ U @ X + rng.standard_normal((dim, 1))
    o.set_state(x, np.zeros_like(x))
    _, sn = o.fields()
    E = 0.5 * (U.T @ U - np.eye(dim))
    pairs = [(0, 0), (1, 1), (0, 1)] if dim == 2 else [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    want = np.array([E[a, b] for a, b in pairs])
    assert np.all(np.isfinite(sn))  # full lattice: every first shell spans
    assert np.allclose(sn, want[:, None], rtol=0, atol=1e-12)


def test_fields_sum_to_the_global_virial(oracle_mod):
    """Sum over particles of cell x stress_xx equals the numerator of the
    global virial stress (Eq. 7 over the whole body), taken from the
    independent observable code, through dynamics and breaks, in 2D and 3D."""
    from gen.images import foam_volume, one_phase_materials
    cases = [(inclusion_image(20, 16, 2.0, 4.0, 0.3, 5), two_phase_materials(), 1.5e-2, 1.0),
             (foam_volume(8, 1.5, 0.55, seed=6), one_phase_materials(1.0, 0.03), 8e-3, 2.0)]
    for img, mats, inc, a in cases:
        k, e, m = mats
        o = oracle_mod.Oracle.from_image(img, k, e, m, a=a)
        for i in range(1, 6):
            o.apply_strain(i * inc)
            o.step(10)
        cell = a ** o.dim
        st, _ = o.fields(cell)
        obs = o.observe()
        omega = (img.shape[-1] - 1) * a * np.prod([s * a for s in img.shape[:-1]])
        assert st[0].sum() * cell / omega == pytest.approx(obs["sigma_vir"], rel=1e-11, abs=1e-14)
        assert o.broken()[0].sum() > 0 or o.dim == 3


def test_fields_degenerate_shell_is_nan(oracle_mod):
    """A one-pixel-high strip: the first shell of each particle lies on a line,
    so the affine fit is undefined (NaN); the stress stays finite."""
    img = np.ones((1, 9), np.uint8)
    k, e, m = two_phase_materials()
    o = oracle_mod.Oracle.from_image(img, k, e, m)
    o.apply_strain(0.01)
    st, sn = o.fields()
    assert np.all(np.isnan(sn)) and np.all(np.isfinite(st))


# --------------------------------------------- triangular packing (lattice 1)

def _tri_sites(img):
    """Sites of the triangular packing of an image, straight from the rule
    (rows at y = iy sqrt(3)/2 pixels up to ny - 1; odd rows shifted by half a
    pixel and one site shorter; each site takes its nearest pixel), with
    floating-point geometry in place of the build's integer arithmetic."""
    ny, nx = img.shape
    out = []
    iy = 0
    while iy * math.sqrt(3) / 2 <= ny - 1 + 1e-12:
        y = iy * math.sqrt(3) / 2
        for ix in range(nx - (iy & 1)):
            x = ix + 0.5 * (iy & 1)
            ph = img[int(math.floor(y + 0.5)), int(math.floor(x + 0.5))]
            if ph:
                out.append((x, y, ph))
        iy += 1
    return out, iy


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_triangular_build_matches_brute_force(oracle_mod, seed):
    """Triangular packing: particles where the rule puts them, in raster
    order, and springs = every pair of particles at distance a (all-pairs
    search), in canonical order, with k and rc from the endpoint phases."""
    rng = np.random.default_rng(40 + seed)
    img = rng.integers(0, 3, size=(9, 11)).astype(np.uint8)
    k, e, m = two_phase_materials()
    a = 1.7
    o = oracle_mod.Oracle.from_image(img, k, e, m, a=a, lattice=1)
    sites, _ = _tri_sites(img)
    t = o.topology()
    assert o.n == len(sites)
    want_X = np.array([[x * a for x, _, _ in sites], [y * a for _, y, _ in sites]])
    assert np.allclose(t["X"], want_X, rtol=0, atol=1e-12)
    ph = np.array([p for _, _, p in sites])
    pairs = []
    for i in range(o.n):
        for j in range(i + 1, o.n):
            if abs(np.sum((want_X[:, j] - want_X[:, i]) ** 2) - a * a) < 1e-9:
                pairs.append((i, j))
    assert list(zip(t["si"].tolist(), t["sj"].tolist())) == pairs
    for s, (i, j) in enumerate(pairs):
        assert t["k"][s] == k[ph[i] - 1, ph[j] - 1]
        assert t["r0"][s] == a
        assert t["rc2"][s] == pytest.approx((a * (1 + e[ph[i] - 1, ph[j] - 1])) ** 2, rel=1e-15)


def test_triangular_counts_closed_form(oracle_mod):
    """Full image: R rows alternate nx and nx - 1 sites; springs are
    (sites - R) within rows plus 2 (nx - 1) between each pair of rows."""
    k, e, m = two_phase_materials()
    for nx, ny in [(6, 5), (13, 30), (40, 2)]:
        o = oracle_mod.Oracle.from_image(np.ones((ny, nx), np.uint8), k, e, m, lattice=1)
        R = 1 + max(r for r in range(ny * 2) if 3 * r * r <= 4 * (ny - 1) ** 2)
        sites = R * nx - R // 2
        assert o.n == sites
        assert o.m == (sites - R) + (R - 1) * 2 * (nx - 1)


def test_triangular_lattice_modulus_and_poisson_ratio(oracle_mod):
    """Uniform triangular lattice of central springs (first neighbours, k):
    the plane continuum has lambda = mu = sqrt(3) k / 4, so E = 2 k / sqrt 3
    and nu = 1/3. Under roller grips with free edges the homogeneous
    uniaxial-stress field meets every boundary condition to first order (the
    inclined springs are unstretched when nu = 1/3), so the relaxed specimen
    shows E and nu up to O(eps)."""
    from gen.images import one_phase_materials
    k_tab, e_tab, mass = one_phase_materials(1.0, 0.5)
    img = np.ones((14, 16), np.uint8)
    o = oracle_mod.Oracle.from_image(img, k_tab, e_tab, mass, dt=0.3, damping=0.2, lattice=1)
    eps = 1e-5
    o.apply_strain(eps)
    st, _ = o.relax(tol=1e-13, max_steps=400000, check_every=100)
    assert st == 0
    ob = o.observe()
    assert ob["sigma_grip"] / eps == pytest.approx(2.0 / math.sqrt(3.0), rel=1e-3)
    x, _, _ = o.state()
    X = o.topology()["X"]
    lat = (x[1].max() - x[1].min()) / (X[1].max() - X[1].min()) - 1.0
    assert -lat / eps == pytest.approx(1.0 / 3.0, rel=1e-3)
    # per-particle stress of an interior particle (cell a h) equals E eps
    st_f, _ = o.fields(math.sqrt(3.0) / 2)
    mid = np.argmin((X[0] - X[0].mean()) ** 2 + (X[1] - X[1].mean()) ** 2)
    assert st_f[0, mid] / eps == pytest.approx(2.0 / math.sqrt(3.0), rel=1e-3)
    assert abs(st_f[1, mid]) < 1e-3 * eps


# --------------------------------------------------- constant strain rate

def test_strain_rate_equals_per_step_grip_increments(oracle_mod):
    """Constant strain-rate loading (grips moved every step) is the same
    trajectory, bit for bit, as one grips-only load increment of rate dt per
    step; the applied strain after s steps is eps0 + s rate dt exactly; an
    increment in between restarts the ramp from the new strain."""
    img = inclusion_image(20, 14, 2.0, 4.0, 0.3, 9)
    k, e, m = two_phase_materials()
    a = oracle_mod.Oracle.from_image(img, k, e, m, load_mode=1)
    b = oracle_mod.Oracle.from_image(img, k, e, m, load_mode=1)
    rate, dt = 2e-2, 0.01
    a.set_strain_rate(rate)
    eps_b = 0.0
    for s in range(1, 151):
        b.apply_strain(0.0 + float(s) * (rate * dt))
        b.step(1)
        if s % 50 == 0:
            a.step(50)
            assert a.observe()["eps"] == b.observe()["eps"] == float(s) * (rate * dt)
    xa, va, _ = a.state()
    xb, vb, _ = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    X = a.topology()["X"]
    grips = a.topology()["grip"] > 0
    eps = 150 * (rate * dt)
    xc = 0.5 * (img.shape[1] - 1)
    assert np.array_equal(xa[0, grips], X[0, grips] + eps * (X[0, grips] - xc))
    # an explicit increment restarts the ramp
    a.apply_strain(0.05)
    a.step(10)
    assert a.observe()["eps"] == 0.05 + 10.0 * (rate * dt)
