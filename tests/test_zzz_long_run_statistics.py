"""Long runs compared with the oracle by statistics: a 2048-particle mixture melted at
T = 2.0, cooled to T = 1.0 and run for 2000 Nose-Hoover steps, once through the library
(mixed precision) and once through the oracle, from the same seeded state.  The
trajectories part ways within a few hundred steps (chaos), so the comparison is of
block averages, each within four combined standard errors: the first peaks of g_AA(r),
g_AB(r) and g_BB(r); the per-species MSD over each block; and the energies per particle
sampled through each block -- potential U/N, total E/N = (K + U)/N, and the drift of the
conserved Nose-Hoover energy (E plus the thermostat's Q xi^2/2 + g T eta) since the
start of the first block, dH/N, whose block means would walk away from the oracle's if
the library's integration drifted.  Two oracle runs
with different seeds pass the same comparison (CPU check in this file)."""
import numpy as np
import pytest

import oracle
from inputs import generate as gen

bbmd = pytest.importorskip("paper_1105_5613_gb300.bbmd")

NCELL, RHO, T_HOT, T, DT, TAU = 8, 1.2, 2.0, 1.0, 0.005, 0.5
COOL, HOLD, NBLOCK, BLOCK, SAMPLE = 600, 200, 5, 400, 50
RMAX, NB = 3.0, 150
Z_MAX = 4.0


def initial_state(seed):
    n = 4 * NCELL ** 3
    L = gen.box_for(n, RHO)
    sp = gen.assign_species(n, n // 5, 0)
    pos = gen.fcc_lattice(NCELL, L)
    vel = gen.maxwell_boltzmann(n, T_HOT, seed, np.ones(n))
    return n, L, sp, pos, vel


class OracleRun:
    """The oracle behind the calls the test makes of a library handle."""

    def __init__(self, n, L, sp, pos, vel):
        self.n, self.L, self.sp = n, L, sp
        self.st = oracle.MDState(pos, vel, sp, L, oracle.ka_params())
        self.ref = None

    def step(self, nsteps, dt, thermo):
        _, t0, t1, tau = thermo
        lg = oracle.md_run(self.st, nsteps, dt, thermo=(t0, t1, tau), use_cells="all_cores",
                           log=True)
        g = 3 * self.n - 3
        K, U, xi, eta, Tk = lg[-1]
        self.last = (U, K + U, K + U + 0.5 * g * Tk * tau * tau * xi * xi + g * Tk * eta)

    def energies(self):
        """(potential, total, conserved Nose-Hoover) energy after the last step."""
        return self.last

    def set_ref(self):
        self.ref = (self.st.pos.copy(), self.st.image.copy())

    def gr(self):
        xfix, k = oracle.quantize(self.st.pos, self.L)
        return oracle.gr_normalize(oracle.gr_counts(xfix, self.sp, self.L, k, NB, RMAX),
                                   self.sp, self.L, RMAX)

    def msd(self):
        return oracle.msd_fs(self.st.pos, self.st.image, self.ref[0], self.ref[1], self.sp,
                             self.L)[0]


class LibraryRun:
    def __init__(self, n, L, sp, pos, vel):
        self.sim = bbmd.Sim(bbmd.ka_params(), n, L, sp, pos, vel)

    def step(self, nsteps, dt, thermo):
        self.sim.step(nsteps, dt, thermo)

    def set_ref(self):
        self.sim.observe(bbmd.OBS_SET_REF)

    def gr(self):
        return self.sim.observe(bbmd.OBS_GR, nbins=NB, rmax=RMAX)["gr"]

    def msd(self):
        return self.sim.observe(bbmd.OBS_MSD)["msd"]

    def energies(self):
        o = self.sim.observe(bbmd.OBS_ENERGY)
        return o["pe"], o["ke"] + o["pe"], o["conserved"]


def block_statistics(run, n):
    """Per block: the first-peak heights of the block-averaged partial g(r), the MSD of
    each species over the block, and the means of U/N, E/N and H/N sampled through the
    block.  Returned as (mean over blocks, standard error) per quantity."""
    run.step(COOL, DT, (1, T_HOT, T, TAU))
    run.step(HOLD, DT, (1, T, T, TAU))
    peaks, msd, en = [], [], []
    H0 = run.energies()[2]
    for _ in range(NBLOCK):
        run.set_ref()
        g, e = [], []
        for _ in range(BLOCK // SAMPLE):
            run.step(SAMPLE, DT, (1, T, T, TAU))
            g.append(np.array(run.gr()))
            U, E, H = run.energies()
            e.append(np.array([U, E, H - H0]) / n)
        gm = np.mean(g, axis=0)
        peaks.append([gm[0, 0].max(), gm[0, 1].max(), gm[1, 1].max()])
        msd.append(np.array(run.msd()))
        en.append(np.mean(e, axis=0))
    peaks, msd, en = np.array(peaks), np.array(msd), np.array(en)
    se = lambda a: a.std(ddof=1) / np.sqrt(len(a))  # noqa: E731
    cols = {"g_AA peak": peaks[:, 0], "g_AB peak": peaks[:, 1], "g_BB peak": peaks[:, 2],
            "MSD A": msd[:, 0], "MSD B": msd[:, 1], "U/N": en[:, 0], "E/N": en[:, 1],
            "dH/N": en[:, 2]}
    return {k: (v.mean(), se(v)) for k, v in cols.items()}


def z_scores(a, b):
    return {k: abs(a[k][0] - b[k][0]) / np.sqrt(a[k][1] ** 2 + b[k][1] ** 2) for k in a}


@pytest.mark.slow
def test_two_oracle_runs_pass_the_comparison():
    """The procedure itself, on two statistically equivalent runs (different velocity
    seeds), both through the oracle."""
    s1, s2 = initial_state(1), initial_state(2)
    a = block_statistics(OracleRun(*s1), s1[0])
    b = block_statistics(OracleRun(*s2), s2[0])
    z = z_scores(a, b)
    assert max(z.values()) < Z_MAX, (a, b, z)


@pytest.mark.gpu
@pytest.mark.slow
def test_long_run_statistics_match_the_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_5613_gb300 import build as b

    b.build()
    bbmd.load()
    state = initial_state(1)
    lib_stats = block_statistics(LibraryRun(*state), state[0])
    ora_stats = block_statistics(OracleRun(*state), state[0])
    z = z_scores(lib_stats, ora_stats)
    assert max(z.values()) < Z_MAX, (lib_stats, ora_stats, z)
