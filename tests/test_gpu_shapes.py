"""Every block shape of the force and list kernels (codes 1, 2, 4: 2 x 2 x Z cells per CTA;
8: 4 x 4 x 2 cells) against the oracle, and the creation-time autotuner that picks one.

nc = 8 cells per axis (ncell 16); nc = 9 (ncell 18): the last block along z is ragged for
Z = 2 and 4, and along x and y for the 4 x 4 x 2 block."""
import numpy as np
import pytest

import oracle
from tests.helpers import force_errors, min_image_rms, mixture, oracle_params, quantized

pytestmark = pytest.mark.gpu

bbmd = pytest.importorskip("paper_1105_5613_gb300.bbmd")

SHAPES = [1, 2, 4, 8]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_5613_gb300 import build as b

    b.build()
    bbmd.load()


def make(ncell, bz, shake=0.12, **kw):
    n, L, pos, vel, sp = mixture(ncell, shake=shake)
    p = bbmd.ka_params(block_z=bz, **kw)
    sim = bbmd.Sim(p, n, L, sp, pos, vel)
    assert sim.info()["block_z"] == bz
    return sim, n, L, pos, vel, sp, p


@pytest.mark.parametrize("ncell", [16, 18])
@pytest.mark.parametrize("bz", SHAPES)
def test_shape_neighbor_sets_and_forces(bz, ncell):
    sim, n, L, pos, vel, sp, p = make(ncell, bz)
    xq, xfix, k = quantized(pos, L)
    po = oracle_params(p)
    off, nbr = sim.get_neighbors()
    offo, nbro = oracle.neighbors(xfix, sp, L, k, oracle.list_R2(po, 0.3), "cells", rcell=2.8)
    assert np.array_equal(off, offo) and np.array_equal(nbr, nbro)
    Fo, uo, Wo, PEo = oracle.forces(xq, sp, L, po, "cells")
    F = sim.get_forces()
    e = force_errors(F, Fo)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4, (np.median(e), e.max())
    obs = sim.observe(bbmd.OBS_ENERGY | bbmd.OBS_VIRIAL)
    assert abs(obs["pe"] - PEo) / n <= 1e-6
    sim.close()


@pytest.mark.parametrize("bz", SHAPES)
def test_shape_cell_mode_and_fp64(bz):
    sim, n, L, pos, vel, sp, p = make(16, bz, nbr_mode=bbmd.NBR_CELL)
    xq, _, _ = quantized(pos, L)
    Fo = oracle.forces(xq, sp, L, oracle_params(p), "cells")[0]
    e = force_errors(sim.get_forces(), Fo)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4, (np.median(e), e.max())
    sim.close()
    sim, n, L, pos, vel, sp, p = make(16, bz, precision=bbmd.PREC_FP64)
    F = sim.get_forces()
    rel = np.linalg.norm(F - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), 1e-3)
    assert rel.max() <= 1e-10, rel.max()
    sim.close()


@pytest.mark.parametrize("bz", SHAPES)
def test_shape_trajectory_nose_hoover(bz):
    sim, n, L, pos, vel, sp, p = make(16, bz, shake=0.0)
    xq, _, _ = quantized(pos, L)
    st = oracle.MDState(xq, vel, sp, L, oracle_params(p))
    th = (1.0, 1.0, 0.5)
    oracle.md_run(st, 100, 0.005, thermo=th, use_cells=True)
    sim.step(100, 0.005, (bbmd.THERMO_NH, *th))
    gp, _, _ = sim.get_state()
    assert min_image_rms(gp, st.pos, L) <= 1e-4
    sim.close()


def test_autotuner_picks_a_timed_shape():
    n, L, pos, vel, sp = mixture(16, shake=0.12)
    p = bbmd.ka_params()
    sim = bbmd.Sim(p, n, L, sp, pos, vel)
    info = sim.info()
    assert info["block_z"] in SHAPES
    k = SHAPES.index(info["block_z"])
    assert all(t > 0 for t in info["shape_force_ms"])
    assert all(t > 0 for t in info["shape_list_ms"])
    cost = [f + 0.25 * l for f, l in zip(info["shape_force_ms"], info["shape_list_ms"])]
    assert cost[k] <= min(cost) * (1 + 1e-6)
    xq, xfix, kx = quantized(pos, L)
    Fo = oracle.forces(xq, sp, L, oracle_params(p), "cells")[0]
    e = force_errors(sim.get_forces(), Fo)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4
    sim.close()


def test_shapes_that_do_not_fit_are_skipped():
    # nc = 3 along each axis: 2 x 2 x 4 and 4 x 4 x 2 do not fit (a block's cells must be
    # distinct cells of the box), the autotuner times 1 and 2 only
    n, L, pos, vel, sp = mixture(7, shake=0.12)
    sim = bbmd.Sim(bbmd.ka_params(), n, L, sp, pos, vel)
    info = sim.info()
    assert info["nc"] == [3, 3, 3]
    assert info["block_z"] in (1, 2)
    assert info["shape_force_ms"][2] == 0.0 and info["shape_force_ms"][3] == 0.0
    sim.close()
    for bz in (4, 8):
        with pytest.raises(bbmd.BBMDError):
            bbmd.Sim(bbmd.ka_params(block_z=bz), n, L, sp, pos, vel)


def test_tune_on_the_current_state():
    n, L, pos, vel, sp = mixture(16, shake=0.12)
    sim = bbmd.Sim(bbmd.ka_params(), n, L, sp, pos, vel)
    sim.step(50, 0.005, (bbmd.THERMO_NH, 2.0, 2.0, 0.5))
    F0 = sim.get_forces()
    sim.tune()
    info = sim.info()
    assert info["block_z"] in SHAPES
    e = force_errors(sim.get_forces(), F0)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4
    sim.step(20, 0.005, (bbmd.THERMO_NH, 2.0, 2.0, 0.5))
    assert np.isfinite(sim.observe(bbmd.OBS_ENERGY)["pe"])
    sim.close()
    fixed = bbmd.Sim(bbmd.ka_params(block_z=4), n, L, sp, pos, vel)
    fixed.tune()
    assert fixed.info()["block_z"] == 4
    fixed.close()
