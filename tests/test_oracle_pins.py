"""Pins of the FP64 oracle to facts outside itself (closed forms, invariants, independent
libraries, brute force).  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from inputs import generate as gen

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def liquid(ncell=5, seed=1, T=1.0, rho=1.2, shake=0.05):
    """Small disordered mixture: FCC lattice with a seeded random displacement."""
    n = 4 * ncell ** 3
    L = gen.box_for(n, rho)
    pos = gen.fcc_lattice(ncell, L)
    rng = np.random.default_rng(seed)
    pos = (pos + rng.uniform(-shake, shake, pos.shape)) % L
    sp = gen.assign_species(n, n // 5, seed)
    vel = gen.maxwell_boltzmann(n, T, seed, np.ones(n))
    return pos, vel, sp, L


# ------------------------------------------------------------------ pair potential ----

def test_params_match_paper():
    g = _gold("mixture_params.json")
    p = oracle.ka_params()
    for a in range(2):
        assert p.mass[a] == g["mass"][a]
        for b in range(2):
            assert p.sigma[a][b] == g["sigma"][a][b]
            assert p.eps[a][b] == g["eps"][a][b]


@pytest.mark.parametrize("ab", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_dimer_minimum(ab):
    """Eq. lj0: minimum -eps_ab at r = 2^(1/6) sigma_ab with zero force."""
    a, b = ab
    p = oracle.ka_params(shift=oracle.SHIFT_NONE)
    eps, sig = p.eps[a][b], p.sigma[a][b]
    rmin = 2.0 ** (1.0 / 6.0) * sig
    hit, V, f = oracle.pair(p, a, b, rmin * rmin)
    assert hit
    assert V == pytest.approx(-eps, rel=1e-14)
    assert abs(f) < 1e-12
    # energy shift lowers the well by V(rc) (rc = 2.5 sigma): V(rc) = 4eps(2.5^-12 - 2.5^-6)
    pe = oracle.ka_params(shift=oracle.SHIFT_ENERGY)
    _, Ve, fe = oracle.pair(pe, a, b, rmin * rmin)
    vrc = 4 * eps * (2.5 ** -12 - 2.5 ** -6)
    assert Ve == pytest.approx(-eps - vrc, rel=1e-13)
    assert fe == pytest.approx(f, abs=1e-12)


@pytest.mark.parametrize("shift", [0, 1, 2])
@pytest.mark.parametrize("pot", [0, 1])
def test_force_is_minus_energy_gradient(shift, pot):
    """f = -(dV*/dr)/r checked against a Richardson-extrapolated central difference."""
    p = oracle.ka_params(potential=pot, shift=shift)
    for a, b in [(0, 0), (0, 1), (1, 1)]:
        sig = p.sigma[a][b]
        for r in np.linspace(0.85 * sig, 2.45 * sig, 17):
            def V(x):
                return oracle.pair(p, a, b, x * x)[1]
            h = 1e-4 * sig
            d1 = (V(r + h) - V(r - h)) / (2 * h)
            d2 = (V(r + 2 * h) - V(r - 2 * h)) / (4 * h)
            dV = (4 * d1 - d2) / 3
            f = oracle.pair(p, a, b, r * r)[2]
            assert f * r == pytest.approx(-dV, rel=1e-7, abs=1e-9)


def test_truncation_forms():
    """Eq. mod0 (shifted force): V*(rc) = 0 and F*(rc) = 0; energy shift: V*(rc) = 0;
    everything vanishes at and beyond rc (strict cutoff r^2 < rc^2)."""
    for a, b in [(0, 0), (0, 1), (1, 1)]:
        rc = 2.5 * oracle.ka_params().sigma[a][b]
        below = (rc * (1 - 1e-9)) ** 2
        pf = oracle.ka_params(shift=oracle.SHIFT_FORCE)
        hit, V, f = oracle.pair(pf, a, b, below)
        assert hit and abs(V) < 1e-9 and abs(f) < 1e-8
        pe = oracle.ka_params(shift=oracle.SHIFT_ENERGY)
        hit, V, f = oracle.pair(pe, a, b, below)
        assert hit and abs(V) < 1e-9 and abs(f) > 1e-3  # force jumps at rc
        for pp in (pf, pe, oracle.ka_params(shift=0)):
            assert oracle.pair(pp, a, b, rc * rc) == (False, 0.0, 0.0)


def test_soft_sphere_value():
    """Eq. sc0: V(sigma) = 4 eps (no shift)."""
    p = oracle.ka_params(potential=oracle.POT_SOFT, shift=0)
    for a, b in [(0, 0), (0, 1), (1, 1)]:
        s = p.sigma[a][b]
        assert oracle.pair(p, a, b, s * s)[1] == pytest.approx(4 * p.eps[a][b], rel=1e-14)


# ------------------------------------------------------------------- lattice sums ----

def test_fcc_shell_table_by_enumeration():
    """The golden FCC shell table equals a direct count of D3 lattice vectors."""
    g = _gold("fcc_shells.json")
    r = np.arange(-4, 5)
    X, Y, Z = np.meshgrid(r, r, r, indexing="ij")
    even = (X + Y + Z) % 2 == 0
    norm = (X * X + Y * Y + Z * Z)[even]
    for m, c in zip(g["shell_r2_over_nn2"], g["coordination"]):
        assert int((norm == 2 * m).sum()) == c


@pytest.mark.parametrize("method", ["brute", "cells", "cells_full"])
@pytest.mark.parametrize("shift", [0, 1, 2])
def test_fcc_lattice_energy_and_zero_forces(method, shift):
    """Perfect all-A FCC crystal at rho=1.2: per-particle energy equals half the shell sum
    over the FCC coordination shells inside rc, and every force vanishes by symmetry."""
    g = _gold("fcc_shells.json")
    ncell = 7
    n = 4 * ncell ** 3
    L = gen.box_for(n, 1.2)
    pos = gen.fcc_lattice(ncell, L)
    sp = np.zeros(n, dtype=np.uint8)
    p = oracle.ka_params(shift=shift)
    F, u, W, PE = oracle.forces(pos, sp, L, p, method=method)
    a = L / ncell
    nn2 = a * a / 2.0
    expect = 0.0
    for m, c in zip(g["shell_r2_over_nn2"], g["coordination"]):
        r2 = m * nn2
        expect += 0.5 * c * oracle.pair(p, 0, 0, r2)[1]
    assert np.allclose(u, expect, rtol=1e-12, atol=1e-12)
    assert PE == pytest.approx(n * expect, rel=1e-12)
    assert np.abs(F).max() < 1e-10


# --------------------------------------------------------------- many-body forces ----

@pytest.mark.parametrize("shift", [1, 2])
def test_newton3_and_gradient(shift):
    pos, _, sp, L = liquid(ncell=4, seed=3)
    p = oracle.ka_params(shift=shift)
    F, u, W, PE = oracle.forces(pos, sp, L, p)
    assert np.abs(F.sum(axis=0)).max() < 1e-12 * np.abs(F).sum()
    assert u.sum() == pytest.approx(PE, rel=1e-12)
    # -dPE/dx_i by central differences for a few particles and axes
    rng = np.random.default_rng(0)
    for i in rng.choice(len(pos), 6, replace=False):
        for d in range(3):
            h = 1e-6
            pp = pos.copy()
            pp[i, d] += h
            Ep = oracle.forces(pp, sp, L, p)[3]
            pp[i, d] -= 2 * h
            Em = oracle.forces(pp, sp, L, p)[3]
            assert F[i, d] == pytest.approx(-(Ep - Em) / (2 * h), rel=2e-6, abs=2e-5)


def test_virial_by_uniform_scaling():
    """W = sum r.F equals -dPE/d(ln s) under a uniform scaling x -> s x (no cutoff
    crossings for the shifted-force form, which is continuous)."""
    pos, _, sp, L = liquid(ncell=4, seed=4)
    p = oracle.ka_params(shift=2)
    _, _, W, PE = oracle.forces(pos, sp, L, p)
    h = 1e-6
    Ep = oracle.forces(pos * (1 + h), sp, L * (1 + h), p)[3]
    Em = oracle.forces(pos * (1 - h), sp, L * (1 - h), p)[3]
    assert W == pytest.approx(-(Ep - Em) / (2 * h), rel=1e-6)


def test_translation_invariance_and_cells_equal_brute():
    pos, _, sp, L = liquid(ncell=6, seed=5)
    p = oracle.ka_params()
    F, u, W, PE = oracle.forces(pos, sp, L, p, "brute")
    Fc, uc, Wc, PEc = oracle.forces(pos, sp, L, p, "cells")
    assert np.allclose(Fc, F, rtol=1e-12, atol=1e-11)
    assert np.allclose(uc, u, rtol=1e-12, atol=1e-12)
    assert Wc == pytest.approx(W, rel=1e-12)
    shifted = (pos + np.array([0.37, -1.21, 2.9])) % L
    Fs = oracle.forces(shifted, sp, L, p)[0]
    assert np.allclose(Fs, F, rtol=1e-9, atol=1e-9)


def test_all_core_form_equals_brute_and_steps_like_cells():
    """The all-core full-stencil form (the CPU baseline's second mode) gives the O(N^2)
    definition's forces, energies and PE; a short Nose-Hoover run with it follows the
    linked-cell run to rounding."""
    pos, vel, sp, L = liquid(ncell=6, seed=7, shake=0.15)
    p = oracle.ka_params()
    F, u, W, PE = oracle.forces(pos, sp, L, p, "brute")
    Ff, uf, Wf, PEf = oracle.forces(pos, sp, L, p, "cells_full")
    assert np.allclose(Ff, F, rtol=1e-12, atol=1e-11)
    assert np.allclose(uf, u, rtol=1e-12, atol=1e-12)
    assert PEf == pytest.approx(PE, rel=1e-12)
    assert oracle.threads() >= 1
    a = oracle.MDState(pos, vel, sp, L, p)
    b = oracle.MDState(pos, vel, sp, L, p)
    oracle.md_run(a, 10, 0.005, thermo=(1.0, 1.0, 0.5), use_cells=True)
    oracle.md_run(b, 10, 0.005, thermo=(1.0, 1.0, 0.5), use_cells="all_cores")
    assert np.abs(a.pos - b.pos).max() < 1e-10 and np.abs(a.vel - b.vel).max() < 1e-9


# ---------------------------------------------------------- cells and neighbour sets ----

def test_quantize_and_cell_containment():
    pos, _, sp, L = liquid(ncell=6, seed=6)
    xfix, k = oracle.quantize(pos, L)
    assert k == 61 - int(math.floor(math.log2(L)))
    Lfix = int(np.ldexp(L, k))
    assert np.all(xfix >= 0) and np.all(xfix < Lfix)
    # quantization error below half a unit
    assert np.abs(oracle.dequantize(xfix, k) - pos).max() <= 2.0 ** (-k)
    nc, D = oracle.cell_grid(L, k, 2.8)
    for d in range(3):
        side = np.ldexp(float(D[d]), -k)
        assert side >= 2.8 and nc[d] == int(L // 2.8) or side >= 2.8
        assert int(D[d]).bit_length() - (int(D[d]) & -int(D[d])).bit_length() + 1 <= 24
        assert np.float32(side) == side  # the cell side is exact in FP32
    cell = oracle.bin_cells(xfix, nc, D)
    ax = cell % nc[0]
    ay = (cell // nc[0]) % nc[1]
    az = cell // (nc[0] * nc[1])
    for d, a in enumerate((ax, ay, az)):
        lo = a * D[d]
        hi = np.where(a == nc[d] - 1, Lfix, (a + 1) * D[d])
        assert np.all(xfix[:, d] >= lo) and np.all(xfix[:, d] < hi)


def test_neighbor_sets_brute_cells_and_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    pos, _, sp, L = liquid(ncell=6, seed=7, shake=0.2)
    xfix, k = oracle.quantize(pos, L)
    p = oracle.ka_params()
    R2 = oracle.list_R2(p, 0.3)
    off, nbr = oracle.neighbors(xfix, sp, L, k, R2, "brute")
    offc, nbrc = oracle.neighbors(xfix, sp, L, k, R2, "cells", rcell=2.8)
    assert np.array_equal(off, offc) and np.array_equal(nbr, nbrc)
    n = len(pos)
    sets = [set(nbr[off[i]:off[i + 1]].tolist()) for i in range(n)]
    # symmetric rule -> symmetric sets
    for i in range(n):
        for j in sets[i]:
            assert i in sets[j]
    # independent library: periodic KD-tree pairs within the largest radius, then the
    # per-species radius; pairs within 1e-9 of a radius are not decided here
    xq = oracle.dequantize(xfix, k)
    tree = spatial.cKDTree(xq, boxsize=L)
    pairs = tree.query_pairs(math.sqrt(R2.max()) + 1e-6, output_type="ndarray")
    d = xq[pairs[:, 1]] - xq[pairs[:, 0]]
    d -= L * np.round(d / L)
    r2 = (d * d).sum(1)
    lim = R2[sp[pairs[:, 0]], sp[pairs[:, 1]]]
    sure = np.abs(r2 - lim) > 1e-9
    inside = r2 < lim
    for (i, j), s, ins in zip(pairs, sure, inside):
        if s:
            assert (j in sets[i]) == bool(ins)
    expect_total = 2 * int((inside & sure).sum())
    got_total = sum(len(s) for s in sets)
    assert abs(got_total - expect_total) <= 2 * int((~sure).sum())


# ------------------------------------------------------------------ integration ----

def test_time_reversibility():
    pos, vel, sp, L = liquid(ncell=4, seed=8, T=1.0)
    p = oracle.ka_params()
    st = oracle.MDState(pos, vel, sp, L, p)
    oracle.md_run(st, 200, 0.005)
    st.vel *= -1.0
    oracle.md_run(st, 200, 0.005)
    d = st.pos - pos
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-9
    assert np.allclose(-st.vel, vel, atol=1e-9)


def test_nve_energy_error_scales_as_dt2():
    """Velocity Verlet is second order: the total-energy fluctuation over a fixed time
    drops about 4x when dt is halved."""
    pos, vel, sp, L = liquid(ncell=4, seed=9, T=1.0)
    p = oracle.ka_params(shift=2)  # continuous force: clean dt^2 behaviour

    def fluct(dt, nsteps):
        st = oracle.MDState(pos, vel, sp, L, p)
        lg = oracle.md_run(st, nsteps, dt, log=True)
        E = lg[:, 0] + lg[:, 1]
        return E.max() - E.min()

    a = fluct(0.004, 250)
    b = fluct(0.002, 500)
    assert 3.0 < a / b < 5.0


def test_nve_drift_and_momentum():
    pos, vel, sp, L = liquid(ncell=6, seed=10, T=2.0)
    p = oracle.ka_params()
    st = oracle.MDState(pos, vel, sp, L, p)
    lg = oracle.md_run(st, 600, 0.005, use_cells=True, log=True)
    E = (lg[:, 0] + lg[:, 1]) / st.n
    # velocity Verlet fluctuates (std ~4e-4 here) but does not drift: window means agree
    assert abs(E[500:].mean() - E[100:200].mean()) < 1e-4
    _, P = oracle.kinetic(st.vel, sp, p)
    assert np.abs(P).max() < 1e-11


def test_nose_hoover_free_gas_matches_ode():
    """With no interactions the Nose-Hoover equations reduce to dK/dt = -2 xi K,
    dxi/dt = (2K - gT)/Q; integrate them independently with scipy and compare."""
    integ = pytest.importorskip("scipy.integrate")
    n = 500
    L = gen.box_for(n, 0.01)
    rng = np.random.default_rng(11)
    pos = rng.uniform(0, L, (n, 3))
    sp = np.zeros(n, dtype=np.uint8)
    vel = gen.maxwell_boltzmann(n, 2.0, 11, np.ones(n))
    p = oracle.ka_params()
    for a in range(2):
        for b in range(2):
            p.eps[a][b] = 0.0  # non-interacting
    T, tau, dt, nsteps = 0.5, 0.5, 0.005, 800
    st = oracle.MDState(pos, vel, sp, L, p)
    lg = oracle.md_run(st, nsteps, dt, thermo=(T, T, tau), log=True)
    g = 3 * n - 3
    Q = g * T * tau * tau
    K0 = oracle.kinetic(vel, sp, p)[0]

    def rhs(t, y):
        K, xi = y
        return [-2 * xi * K, (2 * K - g * T) / Q]

    t_end = nsteps * dt
    sol = integ.solve_ivp(rhs, (0, t_end), [K0, 0.0], rtol=1e-11, atol=1e-11,
                          t_eval=[t_end])
    assert lg[-1, 0] == pytest.approx(sol.y[0, -1], rel=2e-4)
    assert st.nh.xi == pytest.approx(sol.y[1, -1], rel=2e-3, abs=2e-4)


def test_nose_hoover_ramp_follows_the_ode_with_stepwise_targets():
    """Linear cooling (Sec. 4): step k of a call of nsteps steps thermostats to
    T_k = T_start + (T_end - T_start) k / nsteps, constant within the step, with Q = g T_k
    tau^2.  On a free gas the Nose-Hoover equations reduce to dK/dt = -2 xi K and
    dxi/dt = (2K - g T_k) / (g T_k tau^2); scipy integrates them step interval by step
    interval and the oracle must land on the same K and xi.  A target taken one step late
    or early (k + 1, or nsteps - 1 in the ratio) moves K by about 1e-2 here, against an
    integrator error near 1e-5."""
    integ = pytest.importorskip("scipy.integrate")
    n = 400
    L = gen.box_for(n, 0.01)
    rng = np.random.default_rng(21)
    pos = rng.uniform(0, L, (n, 3))
    sp = np.zeros(n, dtype=np.uint8)
    vel = gen.maxwell_boltzmann(n, 2.0, 21, np.ones(n))
    p = oracle.ka_params()
    for a in range(2):
        for b in range(2):
            p.eps[a][b] = 0.0  # non-interacting
    T0, T1, tau, dt, nsteps = 2.0, 0.3, 0.2, 0.002, 100
    st = oracle.MDState(pos, vel, sp, L, p)
    lg = oracle.md_run(st, nsteps, dt, thermo=(T0, T1, tau), log=True)
    g = 3 * n - 3
    # the recorded target of the first and of the last step of the call
    assert lg[0, 4] == T0
    assert lg[-1, 4] == pytest.approx(T0 + (T1 - T0) * (nsteps - 1) / nsteps, rel=1e-15)
    y = [oracle.kinetic(vel, sp, p)[0], 0.0]
    Ks = []
    for k in range(nsteps):
        Tk = T0 + (T1 - T0) * k / nsteps
        Q = g * Tk * tau * tau

        def rhs(t, yy, Tk=Tk, Q=Q):
            return [-2.0 * yy[1] * yy[0], (2.0 * yy[0] - g * Tk) / Q]

        sol = integ.solve_ivp(rhs, (0.0, dt), y, rtol=1e-12, atol=1e-12, method="DOP853")
        y = [sol.y[0, -1], sol.y[1, -1]]
        Ks.append(y[0])
    assert np.allclose(lg[:, 0], Ks, rtol=1e-4)
    assert st.nh.xi == pytest.approx(y[1], rel=1e-4, abs=1e-5)
    # and the thermostat followed the ramp down: K well below its start
    assert lg[-1, 0] < 0.7 * lg[0, 0]


def test_wrap_image_counters_of_free_particles():
    """Free particles at constant velocity cross the periodic box several times in both
    directions: the stored position plus L times the image counter is the straight line
    x0 + v t, and the counter is floor((x0 + v t) / L) (the number of boxes crossed)."""
    n = 24
    L = 9.0
    rng = np.random.default_rng(31)
    x0 = rng.uniform(0, L, (n, 3))
    v = rng.uniform(-12.0, 12.0, (n, 3))
    v[0] = [11.5, -11.5, 0.0]
    sp = np.zeros(n, dtype=np.uint8)
    p = oracle.ka_params()
    for a in range(2):
        for b in range(2):
            p.eps[a][b] = 0.0  # no forces: straight lines
    dt, nsteps = 0.01, 500
    st = oracle.MDState(x0, v, sp, L, p)
    oracle.md_run(st, nsteps, dt)
    line = x0 + v * (nsteps * dt)
    assert np.abs(st.pos + L * st.image - line).max() < 1e-10
    expect = np.floor(line / L)
    clear = np.abs(line / L - np.round(line / L)) > 1e-9  # not on a box face
    assert np.array_equal(st.image[clear], expect[clear].astype(np.int32))
    assert st.image.min() <= -5 and st.image.max() >= 5  # several boxes, both directions
    assert np.all((st.pos >= 0.0) & (st.pos < L))


def test_nose_hoover_extended_energy_conserved():
    """H = K + U + Q xi^2/2 + g T eta is conserved up to the integrator's O(dt^2) error:
    halving dt cuts its spread about 4x, and the spread matches the NVE energy spread."""
    pos, vel, sp, L = liquid(ncell=4, seed=12, T=1.0)
    p = oracle.ka_params(shift=2)
    T, tau = 0.8, 0.5

    def spreads(dt, nsteps):
        st = oracle.MDState(pos, vel, sp, L, p)
        lg = oracle.md_run(st, nsteps, dt, thermo=(T, T, tau), log=True)
        g = 3 * st.n - 3
        Q = g * T * tau * tau
        H = lg[:, 0] + lg[:, 1] + 0.5 * Q * lg[:, 2] ** 2 + g * T * lg[:, 3]
        st2 = oracle.MDState(pos, vel, sp, L, p)
        lg2 = oracle.md_run(st2, nsteps, dt, log=True)
        E = lg2[:, 0] + lg2[:, 1]
        return (H.max() - H.min()) / st.n, (E.max() - E.min()) / st.n, lg, g

    h1, e1, lg, g = spreads(0.003, 600)
    h2, e2, _, _ = spreads(0.0015, 1200)
    assert 3.0 < h1 / h2 < 5.0
    assert h1 < 2.0 * e1
    # the thermostat does act: xi moves and K heads toward g T / 2
    assert np.abs(lg[:, 2]).max() > 0.1
    assert abs(lg[-1, 0] - 0.5 * g * T) < abs(lg[0, 0] - 0.5 * g * T)


def test_steepest_descent_lowers_energy():
    n = 400
    L = gen.box_for(n, 1.2)
    pos = gen.rsa_positions(n, L, 0.7, 13)
    sp = gen.assign_species(n, n // 5, 13)
    p = oracle.ka_params()
    E0 = oracle.forces(pos, sp, L, p)[3]
    relaxed = oracle.sd_run(pos, sp, L, p, 100)
    E1 = oracle.forces(relaxed, sp, L, p)[3]
    assert E1 < E0


def test_steepest_descent_step_rule():
    """One step moves every particle by h F_i with h = min(hmax, dmax / max_i |F_i|): the
    displacement is parallel to the force, and the largest one is dmax when the force cap
    binds, hmax max|F| when it does not."""
    n = 400
    L = gen.box_for(n, 1.2)
    pos = gen.rsa_positions(n, L, 0.7, 17)
    sp = gen.assign_species(n, n // 5, 17)
    p = oracle.ka_params()
    F = oracle.forces(pos, sp, L, p)[0]
    fmax = np.linalg.norm(F, axis=1).max()
    # displacements stay below L/2 so that the minimum image recovers them
    for hmax, dmax in ((1e-3, 0.05), (0.2 / fmax, 1.0)):
        moved = oracle.sd_run(pos, sp, L, p, 1, hmax=hmax, dmax=dmax)
        d = moved - pos
        d -= L * np.round(d / L)
        h = min(hmax, dmax / fmax)
        assert np.allclose(d, h * F, rtol=1e-9, atol=1e-12)
        assert np.linalg.norm(d, axis=1).max() == pytest.approx(min(dmax, hmax * fmax), rel=1e-9)


def test_kinetic_energy_and_kick_use_each_species_mass():
    """Species masses 1 and 3: K = sum m v^2 / 2 and P = sum m v by species, and one NVE
    step of a resting pair of unlike particles changes each velocity by F dt / m (to
    first order), so the heavier one moves a third as fast."""
    p = oracle.ka_params(mass=(1.0, 3.0))
    rng = np.random.default_rng(4)
    vel = rng.normal(size=(10, 3))
    sp = np.array([0, 1] * 5, dtype=np.uint8)
    K, P = oracle.kinetic(vel, sp, p)
    m = np.where(sp == 1, 3.0, 1.0)
    assert K == pytest.approx(0.5 * (m[:, None] * vel ** 2).sum(), rel=1e-14)
    assert np.allclose(P, (m[:, None] * vel).sum(0), rtol=1e-14, atol=1e-14)
    L, r0, dt = 9.0, 1.0, 1e-4
    pos = np.array([[2.0, 3.0, 4.0], [2.0 + r0, 3.0, 4.0]])
    st = oracle.MDState(pos, np.zeros((2, 3)), np.array([0, 1], dtype=np.uint8), L, p)
    oracle.md_run(st, 1, dt)
    f = oracle.forces(pos, np.array([0, 1], dtype=np.uint8), L, p)[0]
    assert np.allclose(st.vel[0], f[0] * dt / 1.0, rtol=1e-3)
    assert np.allclose(st.vel[1], f[1] * dt / 3.0, rtol=1e-3)
    assert st.vel[1, 0] == pytest.approx(-st.vel[0, 0] / 3.0, rel=1e-3)


# ------------------------------------------------------------------- observables ----

def test_gr_counts_against_pdist():
    spatial = pytest.importorskip("scipy.spatial")
    n = 600
    L = 12.0
    rng = np.random.default_rng(14)
    pos = rng.uniform(0, L, (n, 3))
    sp = gen.assign_species(n, n // 5, 14)
    xfix, k = oracle.quantize(pos, L)
    nb, rmax = 100, 5.0
    cnt = oracle.gr_counts(xfix, sp, L, k, nb, rmax)
    xq = oracle.dequantize(xfix, k)
    d = xq[:, None, :] - xq[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(-1))
    dr = rmax / nb
    frac = r / dr - np.floor(r / dr)
    assert (np.minimum(frac, 1 - frac)[~np.eye(n, dtype=bool)] > 1e-9).all()
    for a in range(2):
        for b in range(2):
            m = (sp[:, None] == a) & (sp[None, :] == b) & ~np.eye(n, dtype=bool)
            h, _ = np.histogram(r[m], bins=nb, range=(0, rmax))
            assert np.array_equal(cnt[a, b].astype(np.int64), h)
    # ideal gas: g ~ 1 beyond the first few bins
    g = oracle.gr_normalize(cnt, sp, L, rmax)
    assert abs(g[0, 0, 50:].mean() - 1.0) < 0.05
    _ = spatial


def test_gr_normalisation_of_single_pairs():
    """A lone pair at a known distance: its bin holds the two ordered pairs, and g there
    is the box volume over the shell volume times the species counts of the definition
    (N_a N_b for a != b, N_a (N_a - 1) for a = b).  Swapping N_b - 1 for N_b, or the shell
    volume for a slab, changes the value by a factor."""
    L, rmax, nb = 20.0, 5.0, 50
    dr = rmax / nb
    r0 = 2.345
    q = int(r0 / dr)
    shell = 4.0 * math.pi / 3.0 * ((q + 1) ** 3 - q ** 3) * dr ** 3
    V = L ** 3
    far = [15.0, 15.0, 15.0]  # farther than rmax from the pair (minimum image)
    # two B particles and one distant A: N_B = 2, N_B' = 1
    pos = np.array([[2.0, 2.0, 2.0], [2.0 + r0, 2.0, 2.0], far])
    sp = np.array([1, 1, 0], dtype=np.uint8)
    xfix, k = oracle.quantize(pos, L)
    cnt = oracle.gr_counts(xfix, sp, L, k, nb, rmax)
    assert cnt[1, 1, q] == 2 and cnt.sum() == 2
    g = oracle.gr_normalize(cnt, sp, L, rmax)
    assert g[1, 1, q] == pytest.approx(V * 2 / (2 * 1 * shell), rel=1e-12)
    # one A and one B at r0, one distant B: N_A = 1, N_B = 2
    sp = np.array([0, 1, 1], dtype=np.uint8)
    cnt = oracle.gr_counts(xfix, sp, L, k, nb, rmax)
    assert cnt[0, 1, q] == 1 and cnt[1, 0, q] == 1 and cnt.sum() == 2
    g = oracle.gr_normalize(cnt, sp, L, rmax)
    assert g[0, 1, q] == pytest.approx(V * 1 / (1 * 2 * shell), rel=1e-12)
    assert g[1, 0, q] == pytest.approx(V * 1 / (2 * 1 * shell), rel=1e-12)


def test_msd_fs_closed_forms():
    pos, _, sp, L = liquid(ncell=3, seed=15)
    im = np.zeros(pos.shape, dtype=np.int32)
    msd, fs = oracle.msd_fs(pos, im, pos, im, sp, L)
    assert np.allclose(msd, 0.0) and np.allclose(fs, 1.0)
    dvec = np.array([0.3, -0.7, 1.9])
    moved = pos + dvec
    im2 = np.floor(moved / L).astype(np.int32)
    moved = moved - L * im2
    msd, fs = oracle.msd_fs(moved, im2, pos, im, sp, L, kvec=7.25)
    assert np.allclose(msd, (dvec ** 2).sum(), rtol=1e-12)
    assert np.allclose(fs, np.cos(7.25 * dvec).mean(), rtol=1e-10)


def test_msd_fs_per_species_and_through_many_boxes():
    """Species A and B moved by different vectors, B by more than a box length: each
    species' MSD and F_s is its own vector's closed form, so a species mix-up, a dropped
    image counter or a wrong average fails here."""
    pos, _, sp, L = liquid(ncell=3, seed=21)
    im = np.zeros(pos.shape, dtype=np.int32)
    d = {0: np.array([0.25, 0.5, -0.125]), 1: np.array([-1.5 * L, 0.75, 2.25 * L])}
    moved = pos + np.where((sp == 1)[:, None], d[1], d[0])
    im2 = np.floor(moved / L).astype(np.int32)
    moved = moved - L * im2
    k = 7.25
    msd, fs = oracle.msd_fs(moved, im2, pos, im, sp, L, kvec=k)
    for a in (0, 1):
        assert msd[a] == pytest.approx((d[a] ** 2).sum(), rel=1e-12)
        assert fs[a] == pytest.approx(np.cos(k * d[a]).mean(), rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("method", ["brute", "cells", "cells_full"])
def test_two_body_systems_each_species_pair(method):
    """Many-body loop picks the right species pair: an isolated A-A, A-B or B-B dimer at
    r = 2^(1/6) sigma_ab has PE = -eps_ab - V_ab(rc) and zero force (energy shift)."""
    p = oracle.ka_params(shift=oracle.SHIFT_ENERGY)
    L = 9.0
    for a, b in [(0, 0), (0, 1), (1, 0), (1, 1)]:
        eps, sig = p.eps[a][b], p.sigma[a][b]
        r = 2.0 ** (1.0 / 6.0) * sig
        pos = np.array([[1.0, 2.0, 3.0], [1.0 + r, 2.0, 3.0]])
        sp = np.array([a, b], dtype=np.uint8)
        F, u, W, PE = oracle.forces(pos, sp, L, p, method)
        assert PE == pytest.approx(-eps - 4 * eps * (2.5 ** -12 - 2.5 ** -6), rel=1e-13)
        assert np.abs(F).max() < 1e-11
        assert np.allclose(u, PE / 2)


def test_subset_functions_equal_full():
    pos, _, sp, L = liquid(ncell=6, seed=16, shake=0.2)
    p = oracle.ka_params()
    F, u, _, _ = oracle.forces(pos, sp, L, p)
    idx = np.array([0, 5, 77, 400, 863])
    Fs, us = oracle.forces_subset(pos, sp, L, p, idx)
    assert np.allclose(Fs, F[idx], rtol=1e-12, atol=1e-12)
    assert np.allclose(us, u[idx], rtol=1e-12, atol=1e-12)
    xfix, k = oracle.quantize(pos, L)
    R2 = oracle.list_R2(p, 0.3)
    off, nbr = oracle.neighbors(xfix, sp, L, k, R2)
    offs, nbrs = oracle.neighbors_subset(xfix, sp, L, k, R2, idx, 2.8)
    for s, i in enumerate(idx):
        assert np.array_equal(nbrs[offs[s]:offs[s + 1]], nbr[off[i]:off[i + 1]])
