"""Long runs compared with the oracle by statistics: a 2048-particle mixture melted at
T = 2.0, cooled to T = 1.0 and run for 2000 Nose-Hoover steps, once through the library
(mixed precision) and once through the oracle, from the same seeded state.  The
trajectories part ways within a few hundred steps (chaos), so the comparison is of
block averages: the first peak of g_AA(r) and the per-species MSD over each block, each
within four combined standard errors.  Two oracle runs with different seeds pass the
same comparison with |z| < 1.5 (CPU check in this file)."""
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
        oracle.md_run(self.st, nsteps, dt, thermo=(t0, t1, tau), use_cells="all_cores")

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


def block_statistics(run):
    """Per block: the first-peak height of the block-averaged g_AA(r) and the MSD of
    each species over the block; returned as (mean, standard error) per quantity."""
    run.step(COOL, DT, (1, T_HOT, T, TAU))
    run.step(HOLD, DT, (1, T, T, TAU))
    peaks, msd = [], []
    for _ in range(NBLOCK):
        run.set_ref()
        g = []
        for _ in range(BLOCK // SAMPLE):
            run.step(SAMPLE, DT, (1, T, T, TAU))
            g.append(np.array(run.gr())[0, 0])
        peaks.append(np.mean(g, axis=0).max())
        msd.append(np.array(run.msd()))
    peaks, msd = np.array(peaks), np.array(msd)
    se = lambda a: a.std(ddof=1) / np.sqrt(len(a))  # noqa: E731
    return {"g_AA peak": (peaks.mean(), se(peaks)),
            "MSD A": (msd[:, 0].mean(), se(msd[:, 0])),
            "MSD B": (msd[:, 1].mean(), se(msd[:, 1]))}


def z_scores(a, b):
    return {k: abs(a[k][0] - b[k][0]) / np.sqrt(a[k][1] ** 2 + b[k][1] ** 2) for k in a}


@pytest.mark.slow
def test_two_oracle_runs_pass_the_comparison():
    """The procedure itself, on two statistically equivalent runs (different velocity
    seeds), both through the oracle."""
    a = block_statistics(OracleRun(*initial_state(1)))
    b = block_statistics(OracleRun(*initial_state(2)))
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
    lib_stats = block_statistics(LibraryRun(*state))
    ora_stats = block_statistics(OracleRun(*state))
    z = z_scores(lib_stats, ora_stats)
    assert max(z.values()) < Z_MAX, (lib_stats, ora_stats, z)
