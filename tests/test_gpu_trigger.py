"""The rebuild trigger on a constructed worst case (Sec. 2.2: a pair interacts only inside
r_c, and the cell side bounds the stencil).

Box of side 4 x 2.81, so the cell grid has 4 cells of side D = 2.81 per axis, just above
r_c + skin = 2.8.  Two particles sit in cells two apart along x, 2.82 apart: outside each
other's Verlet list and outside each other's 27-cell stencil.  They fly toward each other
at equal speed while 8 more particles rest far from everything.  They interact once they
have closed 0.32, i.e. after moving 0.16 each: less than the skin for either alone, and
their build cells are not neighbours.  Every step, the forces of the aged lists (or
stencils) must equal the oracle's at the same positions, and a rebuild must have run
before the pair came inside r_c."""
import numpy as np
import pytest

import oracle
from tests.helpers import force_errors, oracle_params

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


L = 4 * 2.81


def closing_pair_state(speed):
    # the pair on the line y = z = 1, cells 0 and 2 along x (cells start at 0, 2.81, 5.62);
    # the speed is chosen so that no step ends with the pair at r_c to rounding
    pair = np.array([[2.805, 1.0, 1.0], [5.625, 1.0, 1.0]])
    # resting particles at least 2.8 from each other, from the pair's line and its images
    rest = np.array([[x, y, z] for x in (1.4, 7.0) for y in (4.0, 8.0) for z in (4.0, 8.0)])
    pos = np.vstack([pair, rest])
    vel = np.zeros_like(pos)
    vel[0, 0], vel[1, 0] = speed, -speed
    return pos, vel


@pytest.mark.parametrize("prec", [bbmd.PREC_MIXED, bbmd.PREC_FP64])
@pytest.mark.parametrize("mode", [bbmd.NBR_VERLET, bbmd.NBR_CELL])
def test_pair_from_cells_two_apart_is_never_missed(mode, prec):
    pos, vel = closing_pair_state(0.77)
    n = len(pos)
    sp = np.zeros(n, dtype=np.uint8)
    p = bbmd.ka_params(nbr_mode=mode, precision=prec)
    sim = bbmd.Sim(p, n, L, sp, pos, vel)
    info = sim.info()
    assert info["nc"] == [4, 4, 4]
    D = info["cell_side_fix"][0] * 2.0 ** -info["fix_exponent"]
    assert 0.0 < D - 2.5 - 0.3 < 0.02  # the cells barely hold r_c + skin
    po = oracle_params(p)
    reb0 = sim.observe(0)["n_rebuilds"]
    inside_at = None
    for step in range(1, 61):
        sim.step(1, 0.005)
        gp, _, _ = sim.get_state()
        F = sim.get_forces()
        Fo = oracle.forces(gp, sp, L, po, "brute")[0]
        d = gp[1] - gp[0]
        d -= L * np.round(d / L)
        r = float(np.linalg.norm(d))
        if np.abs(Fo).max() == 0.0:
            assert np.abs(F).max() == 0.0, (step, r)
        else:
            e = force_errors(F, Fo)
            assert e.max() <= (1e-10 if prec == bbmd.PREC_FP64 else 1e-4), (step, r, e.max())
        if r < 2.5 and inside_at is None:
            inside_at = step
            assert sim.observe(0)["n_rebuilds"] > reb0, "no rebuild before the pair interacted"
    assert inside_at is not None and inside_at > 30  # the pair did close in during the run
    sim.close()
