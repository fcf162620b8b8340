"""GPU-vs-oracle parity through the C ABI (libbbmd.so), on seeded generator inputs.

Bars: cells and Verlet neighbour sets bit-exact; mixed-precision forces e_i <= 1e-5
(median) and <= 1e-4 (max); potential energy of every particle within 1e-6 absolute (the
energy pass evaluates pair energies in FP64 from the exact integer positions, so the
tests hold 1e-9); 100-step position RMS <= 1e-4; the FP64 form within 1e-10 relative per
force."""
import numpy as np
import pytest

import oracle
from inputs import generate as gen
from tests.helpers import force_errors, min_image_rms, mixture, oracle_params, quantized

pytestmark = pytest.mark.gpu

bbmd = pytest.importorskip("paper_1105_5613_gb300.bbmd")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_5613_gb300 import build as b

    b.build()
    bbmd.load()


def make(ncell=10, seed=0, T=2.0, shake=0.1, rc_all=None, **kw):
    """rc_all: one cutoff for every species pair (the glass study of Sec. 4 uses 1.2)."""
    n, L, pos, vel, sp = mixture(ncell, seed=seed, T=T, shake=shake)
    p = bbmd.ka_params(**kw)
    if rc_all is not None:
        for a in range(2):
            for b in range(2):
                p.rcut[a][b] = rc_all
    sim = bbmd.Sim(p, n, L, sp, pos, vel)
    return sim, n, L, pos, vel, sp, p


# (potential, truncation, one cutoff for every pair or None for 2.5 sigma_ab): the
# benchmark mixture, and the soft-sphere shifted-force model of Sec. 2.1 at 2.5 sigma_ab
# and at the glass run's r_c = 1.2 (Sec. 4)
MODELS = [(0, 1, None), (1, 2, None), (1, 2, 1.2)]


# ------------------------------------------------------------------- binning / lists ----

@pytest.mark.parametrize("shake", [0.0, 0.12])
def test_cells_bit_exact(shake):
    sim, n, L, pos, vel, sp, p = make(ncell=10, shake=shake)
    info = sim.info()
    xq, xfix, k = quantized(pos, L)
    assert info["fix_exponent"] == k
    nc, D = oracle.cell_grid(L, k, 2.5 + 0.3)
    assert list(nc) == info["nc"] and list(D) == info["cell_side_fix"]
    assert np.array_equal(sim.get_cells(), oracle.bin_cells(xfix, nc, D))
    sim.close()


@pytest.mark.parametrize("ncell,shake", [(10, 0.0), (10, 0.15), (7, 0.2)])
def test_neighbor_sets_bit_exact(ncell, shake):
    sim, n, L, pos, vel, sp, p = make(ncell=ncell, shake=shake)
    xq, xfix, k = quantized(pos, L)
    R2 = oracle.list_R2(oracle_params(p), 0.3)
    off, nbr = sim.get_neighbors()
    offo, nbro = oracle.neighbors(xfix, sp, L, k, R2, "cells", rcell=2.8)
    assert np.array_equal(off, offo)
    assert np.array_equal(nbr, nbro)
    sim.close()


# ---------------------------------------------------------------------------- forces ----

@pytest.mark.parametrize("pot,shift,rc_all", [(0, 1, None), (0, 0, None), (0, 2, None),
                                             (1, 1, None), (1, 2, None), (1, 2, 1.2)])
@pytest.mark.parametrize("mode", [0, 1])
def test_forces_mixed(pot, shift, rc_all, mode):
    sim, n, L, pos, vel, sp, p = make(ncell=10, shake=0.12, potential=pot, shift=shift,
                                      nbr_mode=mode, rc_all=rc_all)
    xq, _, _ = quantized(pos, L)
    po = oracle_params(p)
    Fo, uo, Wo, PEo = oracle.forces(xq, sp, L, po)
    F, u = sim.get_forces(energies=True)
    e = force_errors(F, Fo)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4, (np.median(e), e.max())
    obs = sim.observe(bbmd.OBS_ENERGY | bbmd.OBS_VIRIAL)
    assert abs(obs["pe"] - PEo) / n <= 1e-6
    assert abs(obs["virial"] - Wo) <= 1e-6 * abs(Wo)
    # per-particle energies: the bar is 1e-6 absolute; the FP64 energy pass reaches
    # rounding level
    assert np.abs(u - uo).max() <= 1e-9, np.abs(u - uo).max()
    sim.close()


@pytest.mark.parametrize("bz", [0, 4, 8])
def test_forces_liquid_37k_every_particle(bz):
    # every particle of a 37 044-particle liquid (melted for 40 steps from a shaken
    # lattice) against the oracle: in the shape the autotuner picks (0), and in the two
    # shapes of largest extent (2 x 2 x 4 and 4 x 4 x 2: FP32 coordinates up to 3 cells
    # from their frame)
    sim, n, L, pos, vel, sp, p = make(ncell=21, shake=0.12, block_z=bz)
    sim.step(40, 0.005)
    gp, _, _ = sim.get_state()
    xq, _, _ = quantized(gp, L)
    Fo = oracle.forces(xq, sp, L, oracle_params(p))[0]
    e = force_errors(sim.get_forces(), Fo)
    assert sim.observe(0)["n_rebuilds"] > 1
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4, (np.median(e), e.max())
    sim.close()


@pytest.mark.parametrize("ncell", [8, 10])
@pytest.mark.parametrize("pot,shift,rc_all", [(0, 1, None), (0, 2, None), (1, 2, None),
                                             (1, 2, 1.2)])
@pytest.mark.parametrize("mode", [0, 1])
def test_forces_fp64_form(pot, shift, rc_all, mode, ncell):
    # ncell 10: L * 2^k close to 2^62 and an odd number of cells per axis
    sim, n, L, pos, vel, sp, p = make(ncell=ncell, shake=0.12, precision=bbmd.PREC_FP64,
                                      potential=pot, shift=shift, nbr_mode=mode,
                                      rc_all=rc_all)
    xq, _, _ = quantized(pos, L)
    po = oracle_params(p)
    Fo, uo, Wo, PEo = oracle.forces(xq, sp, L, po)
    F, u = sim.get_forces(energies=True)
    rel = np.linalg.norm(F - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), 1e-3)
    assert rel.max() <= 1e-10, rel.max()
    obs = sim.observe(bbmd.OBS_ENERGY | bbmd.OBS_VIRIAL)
    assert abs(obs["pe"] - PEo) <= 1e-10 * abs(PEo)
    assert np.allclose(u, uo, rtol=1e-10, atol=1e-12)
    sim.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_forces_near_the_seam(prec):
    """Lattice shifted so that many particles sit next to the periodic boundary (odd cell
    count, L * 2^k close to 2^62)."""
    n, L, pos, vel, sp = mixture(10, T=2.0, shake=0.0)
    shifted = (pos + 0.5 * L / 10 * np.array([0.9, 0.3, 0.7]) + 0.13) % L
    rng = np.random.default_rng(3)
    shifted = (shifted + rng.uniform(-0.1, 0.1, shifted.shape)) % L
    p = bbmd.ka_params(precision=prec)
    sim = bbmd.Sim(p, n, L, sp, shifted, vel)
    xq, _, _ = quantized(shifted, L)
    Fo = oracle.forces(xq, sp, L, oracle_params(p))[0]
    F = sim.get_forces()
    if prec == 1:
        rel = np.linalg.norm(F - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), 1e-3)
        assert rel.max() <= 1e-10
    else:
        e = force_errors(F, Fo)
        assert np.median(e) <= 1e-5 and e.max() <= 1e-4
    sim.close()


def test_zero_net_force_and_lattice():
    # perfect lattice, all A: every force vanishes (FP32 path: small residual)
    ncell = 8
    n = 4 * ncell ** 3
    L = gen.box_for(n, 1.2)
    pos = gen.fcc_lattice(ncell, L)
    sp = np.zeros(n, dtype=np.uint8)
    sim = bbmd.Sim(bbmd.ka_params(), n, L, sp, pos, np.zeros((n, 3)))
    F = sim.get_forces()
    assert np.abs(F).max() < 1e-3
    sim.close()
    sim, n, L, pos, vel, sp, p = make(ncell=10, shake=0.12)
    F = sim.get_forces()
    assert np.abs(F.sum(0)).max() <= 1e-6 * np.abs(F).sum()
    sim.close()


# ------------------------------------------------------------------- trajectories ----

@pytest.mark.parametrize("prec,tol", [(0, 1e-4), (1, 1e-9)])
def test_trajectory_nve_100_steps(prec, tol):
    sim, n, L, pos, vel, sp, p = make(ncell=10, shake=0.0, T=2.0, precision=prec)
    xq, _, _ = quantized(pos, L)
    st = oracle.MDState(xq, vel, sp, L, oracle_params(p))
    oracle.md_run(st, 100, 0.005, use_cells=True)
    sim.step(100, 0.005)
    gp, gv, gi = sim.get_state()
    assert min_image_rms(gp, st.pos, L) <= tol
    assert np.sqrt(((gv - st.vel) ** 2).sum(1).mean()) <= 50 * tol
    sim.close()


def test_trajectory_split_calls_equal_one_call():
    a, n, L, pos, vel, sp, p = make(ncell=8, shake=0.05)
    p.block_z = a.info()["block_z"]  # same block shape: same summation order
    b = bbmd.Sim(p, n, L, sp, pos, vel)
    a.step(60, 0.005)
    for _ in range(6):
        b.step(10, 0.005)
    pa, va, _ = a.get_state()
    pb, vb, _ = b.get_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    a.close()
    b.close()


def test_nose_hoover_split_calls_equal_one_call():
    # the closing half kick and thermostat scale of a call are carried into the next
    # call's first update (same dt), exactly as between two steps of one call; an observe
    # between the calls leaves the state alone
    a, n, L, pos, vel, sp, p = make(ncell=8, shake=0.05)
    p.block_z = a.info()["block_z"]
    b = bbmd.Sim(p, n, L, sp, pos, vel)
    th = (bbmd.THERMO_NH, 0.9, 0.9, 0.5)
    a.step(60, 0.005, th)
    for _ in range(6):
        b.step(10, 0.005, th)
        b.observe(bbmd.OBS_ENERGY)
    pa, va, _ = a.get_state()
    pb, vb, _ = b.get_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    assert a.observe(bbmd.OBS_ENERGY)["xi"] == b.observe(bbmd.OBS_ENERGY)["xi"]
    a.close()
    b.close()


def test_dt_change_between_calls_finishes_the_last_step():
    # a new dt applies the pending closing kick first: the same state as reading the
    # velocities out between the calls
    a, n, L, pos, vel, sp, p = make(ncell=8, shake=0.05)
    p.block_z = a.info()["block_z"]
    b = bbmd.Sim(p, n, L, sp, pos, vel)
    th = (bbmd.THERMO_NH, 0.9, 0.9, 0.5)
    a.step(10, 0.005, th)
    a.step(10, 0.004, th)
    b.step(10, 0.005, th)
    b.get_state()
    b.step(10, 0.004, th)
    pa, va, _ = a.get_state()
    pb, vb, _ = b.get_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    a.close()
    b.close()


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("prec,tol", [(0, 1e-4), (1, 1e-9)])
def test_trajectory_nose_hoover_100_steps(prec, tol, model):
    pot, shift, rc_all = model
    sim, n, L, pos, vel, sp, p = make(ncell=10, shake=0.0, T=2.0, precision=prec,
                                      potential=pot, shift=shift, rc_all=rc_all)
    xq, _, _ = quantized(pos, L)
    st = oracle.MDState(xq, vel, sp, L, oracle_params(p))
    th = (0.5, 0.5, 0.5)
    oracle.md_run(st, 100, 0.005, thermo=th, use_cells=True)
    sim.step(100, 0.005, (bbmd.THERMO_NH, *th))
    gp, gv, _ = sim.get_state()
    obs = sim.observe(bbmd.OBS_ENERGY)
    assert min_image_rms(gp, st.pos, L) <= tol
    assert obs["xi"] == pytest.approx(st.nh.xi, rel=50 * tol, abs=50 * tol)
    sim.close()


def test_nose_hoover_ramp_matches_oracle():
    sim, n, L, pos, vel, sp, p = make(ncell=8, shake=0.0, T=2.0)
    xq, _, _ = quantized(pos, L)
    st = oracle.MDState(xq, vel, sp, L, oracle_params(p))
    th = (2.0, 0.4, 0.5)
    oracle.md_run(st, 80, 0.005, thermo=th, use_cells=True)
    sim.step(80, 0.005, (bbmd.THERMO_NH, *th))
    gp, gv, _ = sim.get_state()
    assert min_image_rms(gp, st.pos, L) <= 1e-4
    K, _ = oracle.kinetic(st.vel, sp, oracle_params(p))
    assert sim.observe(0)["ke"] == pytest.approx(K, rel=1e-4)
    sim.close()


def test_nve_energy_conservation():
    """Same criterion as the oracle's own pin: velocity Verlet fluctuates but does not drift
    (means of 100-step windows agree within 1e-4 per particle)."""
    sim, n, L, pos, vel, sp, p = make(ncell=10, shake=0.05, T=2.0)
    E = []
    for _ in range(600):
        sim.step(1, 0.005)
        o = sim.observe(bbmd.OBS_ENERGY | bbmd.OBS_MOMENTUM)
        E.append((o["ke"] + o["pe"]) / n)
    E = np.array(E)
    assert abs(E[500:].mean() - E[100:200].mean()) < 1e-4, (E[500:].mean(), E[100:200].mean())
    assert np.abs(o["momentum"]).max() < 1e-3
    assert o["n_rebuilds"] > 20
    sim.close()


# ------------------------------------------------------------------- observables ----

@pytest.mark.parametrize("ncell", [10, 11])
def test_gr_counts_bit_exact(ncell):
    sim, n, L, pos, vel, sp, p = make(ncell=ncell, shake=0.15)
    xq, xfix, k = quantized(pos, L)
    o = sim.observe(bbmd.OBS_GR, nbins=500, rmax=5.0)
    ref = oracle.gr_counts(xfix, sp, L, k, 500, 5.0)
    assert np.array_equal(o["gr_counts"], ref)
    g = oracle.gr_normalize(ref, sp, L, 5.0)
    assert np.allclose(o["gr"], g, rtol=1e-12, atol=1e-12)
    sim.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_msd_fs_per_particle_displacements(prec):
    """Every particle moved by its own seeded displacement, B particles by larger ones and
    some particles by more than a box length (image counters through several boxes):
    per-species MSD and F_s(k, t) equal the oracle's on the same positions and counters."""
    sim, n, L, pos, vel, sp, p = make(ncell=8, shake=0.1, precision=prec)
    xq0, _, _ = quantized(pos, L)
    sim.observe(bbmd.OBS_SET_REF)
    rng = np.random.default_rng(41)
    disp = rng.normal(0.0, 0.4, (n, 3))
    disp[sp == 1] *= 3.0
    far = rng.choice(n, 60, replace=False)
    disp[far] += rng.choice([-1.0, 1.0], (60, 3)) * rng.uniform(1.0, 3.5, (60, 3)) * L
    moved = xq0 + disp
    img = np.floor(moved / L).astype(np.int32)
    wrapped = moved - L * img
    sim.set_state(wrapped, vel, img)
    gp, _, gi = sim.get_state()
    assert np.array_equal(gi, img)
    xq1, _, _ = quantized(wrapped, L)
    assert np.array_equal(gp, xq1)
    for kv in (7.25, 3.1):
        o = sim.observe(bbmd.OBS_MSD | bbmd.OBS_FS, k=kv)
        msd, fs = oracle.msd_fs(xq1, img, xq0, np.zeros_like(img), sp, L, kv)
        assert np.allclose(o["msd"], msd, rtol=1e-12, atol=0), (o["msd"], msd)
        assert np.allclose(o["fs"], fs, rtol=1e-12, atol=1e-13), (o["fs"], fs)
    assert abs(msd[1] - msd[0]) > 0.1 * msd[0]  # the species averages are told apart
    sim.close()


@pytest.mark.parametrize("prec,tol", [(0, 2e-3), (1, 1e-7)])
def test_msd_fs_after_200_steps(prec, tol):
    """200 Nose-Hoover steps from the same start through the library and the oracle:
    per-species MSD and F_s(k = 7.25, t) agree to the trajectory's own precision."""
    sim, n, L, pos, vel, sp, p = make(ncell=8, shake=0.05, T=2.0, precision=prec)
    xq, _, _ = quantized(pos, L)
    st = oracle.MDState(xq, vel, sp, L, oracle_params(p))
    sim.observe(bbmd.OBS_SET_REF)
    th = (1.5, 1.5, 0.5)
    sim.step(200, 0.005, (bbmd.THERMO_NH, *th))
    oracle.md_run(st, 200, 0.005, thermo=th, use_cells=True)
    o = sim.observe(bbmd.OBS_MSD | bbmd.OBS_FS)
    msd, fs = oracle.msd_fs(st.pos, st.image, xq, np.zeros((n, 3), np.int32), sp, L, 7.25)
    assert np.allclose(o["msd"], msd, rtol=tol), (o["msd"], msd)
    assert np.allclose(o["fs"], fs, rtol=0, atol=tol), (o["fs"], fs)
    assert msd.min() > 0.05  # the particles did move
    sim.close()


def test_msd_fs_several_time_origins():
    """Three time origins set 40 steps apart, each measured at the end against the oracle's
    positions and image counters at that origin (FP64 form: the trajectories agree to
    1e-9); an origin never set is refused."""
    sim, n, L, pos, vel, sp, p = make(ncell=8, shake=0.05, T=2.0, precision=bbmd.PREC_FP64)
    xq, _, _ = quantized(pos, L)
    st = oracle.MDState(xq, vel, sp, L, oracle_params(p))
    th = (1.5, 1.5, 0.5)
    refs = []
    for o in range(3):
        sim.observe(bbmd.OBS_SET_REF, origin=o)
        refs.append((st.pos.copy(), st.image.copy()))
        sim.step(40, 0.005, (bbmd.THERMO_NH, *th))
        oracle.md_run(st, 40, 0.005, thermo=th, use_cells=True)
    got = [sim.observe(bbmd.OBS_MSD | bbmd.OBS_FS, origin=o) for o in range(3)]
    for o in range(3):
        msd, fs = oracle.msd_fs(st.pos, st.image, refs[o][0], refs[o][1], sp, L, 7.25)
        assert np.allclose(got[o]["msd"], msd, rtol=1e-7), (o, got[o]["msd"], msd)
        assert np.allclose(got[o]["fs"], fs, rtol=0, atol=1e-7), (o, got[o]["fs"], fs)
    assert got[0]["msd"][0] > got[1]["msd"][0] > got[2]["msd"][0] > 0  # longer lag, farther
    with pytest.raises(bbmd.BBMDError) as e:
        sim.observe(bbmd.OBS_MSD, origin=5)
    assert e.value.code == 8  # BBMD_ERR_STATE
    with pytest.raises(bbmd.BBMDError) as e:
        sim.observe(bbmd.OBS_MSD, origin=bbmd.MAX_ORIGINS)
    assert e.value.code == 1
    sim.close()


def test_msd_fs_rigid_translation():
    sim, n, L, pos, vel, sp, p = make(ncell=8, shake=0.1)
    sim.observe(bbmd.OBS_SET_REF)
    o = sim.observe(bbmd.OBS_MSD | bbmd.OBS_FS)
    assert np.allclose(o["msd"], 0.0) and np.allclose(o["fs"], 1.0)
    dvec = np.array([0.3, -0.7, 1.9])
    moved = pos + dvec
    img = np.floor(moved / L).astype(np.int32)
    sim.set_state(moved - L * img, vel, img)
    o = sim.observe(bbmd.OBS_MSD | bbmd.OBS_FS, k=7.25)
    assert np.allclose(o["msd"], (dvec ** 2).sum(), rtol=1e-9)
    assert np.allclose(o["fs"], np.cos(7.25 * dvec).mean(), rtol=1e-9, atol=1e-12)
    sim.close()


# ------------------------------------------------------------------ edge cases ----

def test_edge_minimal_box_and_ragged_n():
    # N = 864 (L = 8.96): three cells per axis, the smallest legal grid
    sim, n, L, pos, vel, sp, p = make(ncell=6, shake=0.1)
    assert sim.info()["nc"] == [3, 3, 3]
    xq, xfix, k = quantized(pos, L)
    Fo = oracle.forces(xq, sp, L, oracle_params(p))[0]
    e = force_errors(sim.get_forces(), Fo)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4
    sim.close()
    # ragged N (not a lattice size), non-cubic box, random non-overlapping positions
    n = 1237
    box = np.array([9.5, 11.0, 10.3])
    rng = np.random.default_rng(5)
    pos = gen.rsa_positions(n, 9.5, 0.75, 21) * (box / 9.5)
    sp = (rng.uniform(size=n) < 0.3).astype(np.uint8)
    p = bbmd.ka_params()
    sim = bbmd.Sim(p, n, box, sp, pos, np.zeros((n, 3)))
    xfix, k = oracle.quantize(pos, box)
    xq = oracle.dequantize(xfix, k)
    Fo = oracle.forces(xq, sp, box, oracle_params(p))[0]
    e = force_errors(sim.get_forces(), Fo)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4
    R2 = oracle.list_R2(oracle_params(p), 0.3)
    off, nbr = sim.get_neighbors()
    offo, nbro = oracle.neighbors(xfix, sp, box, k, R2, "brute")
    assert np.array_equal(off, offo) and np.array_equal(nbr, nbro)
    sim.close()


def test_edge_crowded_cells_and_single_species():
    # a dense slab puts more than 32 particles into some cells (chunked tiles)
    n = 2000
    L = 11.5
    rng = np.random.default_rng(9)
    pos = gen.rsa_positions(n, L, 0.62, 33)
    pos[:, 2] = pos[:, 2] * 0.6
    sp = np.ones(n, dtype=np.uint8)
    p = bbmd.ka_params(stencil_capacity=2000, list_capacity=256)
    sim = bbmd.Sim(p, n, L, sp, pos, np.zeros((n, 3)))
    xq, xfix, k = quantized(pos, L)
    cells = sim.get_cells()
    assert np.bincount(cells).max() > 32
    Fo = oracle.forces(xq, sp, L, oracle_params(p))[0]
    e = force_errors(sim.get_forces(), Fo)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4
    off, nbr = sim.get_neighbors()
    offo, nbro = oracle.neighbors(xfix, sp, L, k, oracle.list_R2(oracle_params(p), 0.3))
    assert np.array_equal(off, offo) and np.array_equal(nbr, nbro)
    sim.close()
    _ = rng


def test_errors_are_reported():
    n, L, pos, vel, sp = mixture(5)
    with pytest.raises(bbmd.BBMDError) as ei:  # 500 particles: fewer than 3 cells per axis
        bbmd.Sim(bbmd.ka_params(), n, L, sp, pos, vel)
    assert ei.value.code == 2
    n, L, pos, vel, sp = mixture(8)
    bad = bbmd.ka_params()
    bad.mass[1] = 0.0
    with pytest.raises(bbmd.BBMDError) as ei:
        bbmd.Sim(bad, n, L, sp, pos, vel)
    assert ei.value.code == 1
    p2 = pos.copy()
    p2[3, 1] = np.nan
    with pytest.raises(bbmd.BBMDError) as ei:
        bbmd.Sim(bbmd.ka_params(), n, L, sp, p2, vel)
    assert ei.value.code == 1
    # staged capacity far below one block region, in every shape, precision and mode: the
    # kernels take only the staged particles and the overflow is reported
    for prec in (bbmd.PREC_MIXED, bbmd.PREC_FP64):
        for mode in (bbmd.NBR_VERLET, bbmd.NBR_CELL):
            with pytest.raises(bbmd.BBMDError) as ei:
                bbmd.Sim(bbmd.ka_params(precision=prec, nbr_mode=mode, stencil_capacity=64),
                         n, L, sp, pos, vel)
            assert ei.value.code == 5
    sim = bbmd.Sim(bbmd.ka_params(), n, L, sp, pos, vel)
    with pytest.raises(bbmd.BBMDError):
        sim.step(10, -1.0)
    with pytest.raises(bbmd.BBMDError):
        sim.observe(bbmd.OBS_MSD)  # no reference yet
    sim.step(5, 0.005)
    sim.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_lists_grow_beyond_the_capacity(prec):
    """A list capacity far below the lists: creation grows it to the longest list and the
    lists and forces are those of the oracle."""
    sim, n, L, pos, vel, sp, p = make(ncell=8, shake=0.12, list_capacity=16, precision=prec)
    assert sim.info()["list_capacity"] >= 100
    xq, xfix, k = quantized(pos, L)
    off, nbr = sim.get_neighbors()
    offo, nbro = oracle.neighbors(xfix, sp, L, k, oracle.list_R2(oracle_params(p), 0.3),
                                  "cells", rcell=2.8)
    assert np.array_equal(off, offo) and np.array_equal(nbr, nbro)
    Fo = oracle.forces(xq, sp, L, oracle_params(p))[0]
    F = sim.get_forces()
    if prec == 1:
        rel = np.linalg.norm(F - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), 1e-3)
        assert rel.max() <= 1e-10
    else:
        e = force_errors(F, Fo)
        assert np.median(e) <= 1e-5 and e.max() <= 1e-4
    sim.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-4), (1, 1e-9)])
def test_cut_lists_fall_back_to_the_stencil(prec, tol):
    """At rho = 1.19 the lattice's seventh shell lies just beyond rc + skin, so its lists
    hold 86 entries at most, against up to about 115 in the liquid it melts into.  With a
    capacity of 88 the rebuilds of the run cut lists, and the steps take their forces
    from the cell stencil instead.  The trajectory still follows the oracle, and the next
    synchronising call grows the lists."""
    n = 4 * 10 ** 3
    L = gen.box_for(n, 1.19)
    pos = gen.fcc_lattice(10, L)
    sp = gen.assign_species(n, n // 5, 0)
    vel = gen.maxwell_boltzmann(n, 2.0, 0, np.ones(n))
    p = bbmd.ka_params(precision=prec, list_capacity=88)
    sim = bbmd.Sim(p, n, L, sp, pos, vel)
    assert sim.info()["list_capacity"] == 88
    xq, _, _ = quantized(pos, L)
    st = oracle.MDState(xq, vel, sp, L, oracle_params(p))
    oracle.md_run(st, 100, 0.005, use_cells=True)
    sim.step(100, 0.005)
    gp, gv, _ = sim.get_state()
    assert min_image_rms(gp, st.pos, L) <= tol
    assert np.sqrt(((gv - st.vel) ** 2).sum(1).mean()) <= 50 * tol
    assert sim.info()["list_capacity"] > 88
    oracle.md_run(st, 20, 0.005, use_cells=True)
    sim.step(20, 0.005)
    gp, _, _ = sim.get_state()
    assert min_image_rms(gp, st.pos, L) <= tol
    sim.close()


def test_deterministic_repeat():
    a, n, L, pos, vel, sp, p = make(ncell=8, shake=0.1)
    p.block_z = a.info()["block_z"]  # bitwise repeatable for a given block shape
    b = bbmd.Sim(p, n, L, sp, pos, vel)
    a.step(40, 0.005, (bbmd.THERMO_NH, 1.0, 1.0, 0.5))
    b.step(40, 0.005, (bbmd.THERMO_NH, 1.0, 1.0, 0.5))
    pa, va, ia = a.get_state()
    pb, vb, ib = b.get_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb) and np.array_equal(ia, ib)
    a.close()
    b.close()


def test_state_round_trip_and_resume():
    sim, n, L, pos, vel, sp, p = make(ncell=8, shake=0.1)
    sim.step(30, 0.005)
    gp, gv, gi = sim.get_state()
    twin = bbmd.Sim(p, n, L, sp, gp, gv)
    twin.set_state(gp, gv, gi)
    tp, tv, ti = twin.get_state()
    assert np.array_equal(tp, gp) and np.array_equal(tv, gv) and np.array_equal(ti, gi)
    # a non-finite upload is refused (checked on the device) and leaves the state as it was
    bad_p, bad_v = gp.copy(), gv.copy()
    bad_p[n // 2, 1] = np.inf
    bad_v[n // 3, 2] = np.nan
    for up_p, up_v in ((bad_p, gv), (gp, bad_v)):
        with pytest.raises(bbmd.BBMDError) as ei:
            twin.set_state(up_p, up_v, gi)
        assert ei.value.code == 1
        tp, tv, ti = twin.get_state()
        assert np.array_equal(tp, gp) and np.array_equal(tv, gv) and np.array_equal(ti, gi)
    sim.step(30, 0.005)
    twin.step(30, 0.005)
    ap, _, _ = sim.get_state()
    bp, _, _ = twin.get_state()
    assert min_image_rms(ap, bp, L) <= 1e-5
    sim.close()
    twin.close()


def test_minimize_matches_oracle():
    """Steepest descent from random sequential addition: the trajectory follows the oracle
    while the step is force-limited; with h = 1e-3 the iteration is unstable along the
    stiffest pair directions (h > 2 / largest curvature), which amplifies rounding
    differences, so later steps are compared by the energy they reach."""
    n = 1500
    L = gen.box_for(n, 1.2)
    pos = gen.rsa_positions(n, L, 0.7, 3)
    sp = gen.assign_species(n, 300, 3)
    p = bbmd.ka_params()
    xq, _, _ = quantized(pos, L)
    sim = bbmd.Sim(p, n, L, sp, pos, np.zeros((n, 3)))
    e0 = sim.observe(bbmd.OBS_ENERGY)["pe"]
    sim.minimize(15)
    gp, _, _ = sim.get_state()
    relaxed = oracle.sd_run(xq, sp, L, oracle_params(p), 15, use_cells=True)
    assert min_image_rms(gp, relaxed, L) <= 1e-5
    sim.minimize(35)
    e1 = sim.observe(bbmd.OBS_ENERGY)["pe"]
    relaxed = oracle.sd_run(relaxed, sp, L, oracle_params(p), 35, use_cells=True)
    eo = oracle.forces(relaxed, sp, L, oracle_params(p))[3]
    assert e1 < e0 and eo < e0
    assert abs(e1 - eo) <= 1e-3 * abs(e0 - eo)
    sim.close()


@pytest.mark.parametrize("jitter", [0.0, 0.07])
def test_device_generated_initial_state_matches_generator(jitter):
    ncell = 9
    n = 4 * ncell ** 3
    L = gen.box_for(n, 1.2)
    sp = gen.assign_species(n, n // 5, 4)
    sim = bbmd.Sim(bbmd.ka_params(init_jitter=jitter), n, L, sp, None, None, T0=1.5, seed=4)
    gp, gv, _ = sim.get_state()
    xq, _, _ = quantized(gen.fcc_sites(ncell, L, np.arange(n), jitter=jitter, seed=4), L)
    assert np.array_equal(gp, xq)
    if jitter == 0.0:
        assert np.array_equal(xq, quantized(gen.fcc_lattice(ncell, L), L)[0])
    ref = gen.maxwell_boltzmann(n, 1.5, 4, np.ones(n))
    assert np.abs(gv - ref).max() < 1e-12
    sim.close()


def test_torch_allocator_and_stream():
    torch = pytest.importorskip("torch")
    n, L, pos, vel, sp = mixture(8, shake=0.1)
    s = torch.cuda.Stream()
    sim = bbmd.Sim(bbmd.ka_params(), n, L, sp, pos, vel, stream=s.cuda_stream,
                   use_torch_allocator=True)
    assert sim.info()["device_bytes"] > 0
    sim.step(20, 0.005)
    o = sim.observe(bbmd.OBS_ENERGY)
    assert np.isfinite(o["pe"])
    sim.close()


# -------------------------------------------------------------- full-size samples ----

@pytest.mark.parametrize("ncell", [40, 160])
def test_full_size_sampled(ncell):
    """The benchmark configurations (256 000 and 16 384 000 particles), in the launch
    configuration the benchmark uses: bins checked for every particle, neighbour sets
    and forces for a seeded sample computed one by one by the oracle."""
    n = 4 * ncell ** 3
    L = gen.box_for(n, 1.2)
    sp = gen.assign_species(n, n // 5, 0)
    sim = bbmd.Sim(bbmd.ka_params(), n, L, sp, None, None, T0=2.0, seed=0)
    sim.step(20, 0.005, (bbmd.THERMO_NH, 2.0, 2.0, 0.5))
    pos = gen.fcc_lattice(ncell, L)
    # restart from generator positions with a seeded shake so no oracle input comes
    # from the device trajectory
    rng = np.random.default_rng(77)
    pos = (pos + rng.uniform(-0.12, 0.12, pos.shape)) % L
    vel = gen.maxwell_boltzmann(n, 2.0, 0, np.ones(n))
    sim.set_state(pos, vel)
    xq, xfix, k = quantized(pos, L)
    nc, D = oracle.cell_grid(L, k, 2.8)
    assert np.array_equal(sim.get_cells(), oracle.bin_cells(xfix, nc, D))
    idx = np.sort(np.random.default_rng(1).choice(n, 400, replace=False))
    F = sim.get_forces()
    Fo, _ = oracle.forces_subset(xq, sp, L, oracle.ka_params(), idx)
    e = force_errors(F[idx], Fo)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4, (np.median(e), e.max())
    off, nbr = sim.get_neighbors(idx)
    R2 = oracle.list_R2(oracle.ka_params(), 0.3)
    offo, nbro = oracle.neighbors_subset(xfix, sp, L, k, R2, idx, 2.8)
    assert np.array_equal(off, offo) and np.array_equal(nbr, nbro)
    sim.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_lists_stay_valid_until_the_rebuild_trigger(mode):
    """The rebuild trigger (two neighbouring cells' largest displacements summing beyond the
    skin) keeps every interacting pair in the aged lists / cell stencils: at many points of
    a hot NVE run the forces from the aged structures equal those of a fresh handle built at
    the same positions (only the FP32 summation order differs)."""
    sim, n, L, pos, vel, sp, p = make(ncell=10, shake=0.05, T=3.0, nbr_mode=mode)
    p.block_z = sim.info()["block_z"]
    worst = 0.0
    for k in range(40):
        sim.step(3, 0.005)
        gp, gv, _ = sim.get_state()
        twin = bbmd.Sim(p, n, L, sp, gp, gv)
        e = force_errors(sim.get_forces(), twin.get_forces())
        twin.close()
        worst = max(worst, float(e.max()))
    rebuilds = sim.observe(0)["n_rebuilds"]
    sim.close()
    assert worst <= 1e-4, worst
    assert rebuilds >= 5  # the run did cross several rebuilds
