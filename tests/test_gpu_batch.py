"""Replica batches (bbmd_create_batch / bbmd_step_batch): every replica of a batch against
the oracle on its own generated inputs, at its own temperature; the persistent step (one
cooperative launch per step) and the batch graph both equal, bit for bit, to stepping
each replica handle on its own; argument errors; a persistent-step wait that runs out
(BBMD_ERR_TIMEOUT on every replica, the device usable after)."""
import numpy as np
import pytest

import oracle
from inputs import generate as gen
from tests.helpers import min_image_rms, oracle_params, quantized

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


def lattice_replicas(ms, temps, shake=0.05, rho=1.2):
    ns, boxes, pos, vel, sp = [], [], [], [], []
    for r, (m, T) in enumerate(zip(ms, temps)):
        n = 4 * m ** 3
        L = gen.box_for(n, rho)
        rng = np.random.default_rng(100 + r)
        pos.append((gen.fcc_lattice(m, L) + rng.uniform(-shake, shake, (n, 3))) % L)
        vel.append(gen.maxwell_boltzmann(n, T, r, np.ones(n)))
        sp.append(gen.assign_species(n, n // 5, r))
        ns.append(n)
        boxes.append(L)
    return ns, boxes, pos, vel, sp


@pytest.mark.parametrize("prec,mode,tol,lcap", [(0, 0, 1e-4, 0), (1, 0, 1e-9, 0), (0, 1, 1e-4, 0),
                                                (0, 0, 1e-4, 88), (1, 0, 1e-9, 88)])
def test_batch_replicas_match_oracle(prec, mode, tol, lcap):
    # lcap 88 holds the lists of the lattice at rho = 1.19 (86 at most: its seventh shell
    # lies just beyond rc + skin) but not those of the liquid: the replicas' lists are cut
    # during the run and their forces come from the cell stencil
    ms, temps = [8, 9, 10, 11], [0.5, 1.0, 1.5, 2.0]
    if lcap:
        ns, boxes, pos, vel, sp = lattice_replicas(ms, temps, shake=0.0, rho=1.19)
    else:
        ns, boxes, pos, vel, sp = lattice_replicas(ms, temps)
    p = bbmd.ka_params(precision=prec, nbr_mode=mode, list_capacity=lcap)
    b = bbmd.Batch(p, ns, boxes, sp, pos, vel)
    # mixed precision takes the persistent step by default; the FP64 form the graph
    assert b.uses_persistent() == (prec == 0)
    th = [(bbmd.THERMO_NH, T, T, 0.5) for T in temps]
    b.step(100, 0.005, th)
    for r in range(len(ns)):
        xq, _, _ = quantized(pos[r], boxes[r])
        st = oracle.MDState(xq, vel[r], sp[r], boxes[r], oracle_params(p))
        oracle.md_run(st, 100, 0.005, thermo=th[r][1:], use_cells=True)
        gp, _, _ = b.replica(r).get_state()
        assert min_image_rms(gp, st.pos, boxes[r]) <= tol, r
        obs = b.replica(r).observe(bbmd.OBS_ENERGY)
        assert obs["step"] == 100
        assert obs["xi"] == pytest.approx(st.nh.xi, rel=1e-3, abs=1e-3)
    b.close()


@pytest.mark.parametrize("path,branches,nbr", [("graph", 1, 0), ("graph", 2, 0), ("graph", 5, 0),
                                              ("persistent", 0, 0), ("persistent", 0, 1)])
def test_batch_step_equals_replica_steps(path, branches, nbr):
    """RSA replicas of uneven size relaxed by steepest descent, then stepped by the batch
    (the persistent step, or the graph with replicas grouped into `branches` branches, one
    launch per phase and group) in one batch and replica by replica in a twin batch:
    identical states."""
    ns, boxes, pos, sp = gen.replica_batch(5, 2048, 6000, 7)
    temps = list(np.linspace(0.4, 2.0, 5))
    p = bbmd.ka_params(nbr_mode=nbr)  # the batch default shape: the persistent kernel's
    twins = [bbmd.Batch(p, ns, boxes, sp, pos, None, T0=temps, seed=11) for _ in range(2)]
    for b in twins:
        for r in range(len(ns)):
            b.replica(r).minimize(50)
    th = [(bbmd.THERMO_NH, T, T, 0.5) for T in temps]
    if path == "graph":
        twins[0].set_mode(bbmd.BATCH_GRAPH)
        twins[0].set_branches(branches)
        assert not twins[0].uses_persistent()
    else:
        twins[0].set_mode(bbmd.BATCH_PERSISTENT)
        assert twins[0].uses_persistent()
    twins[0].step(60, 0.005, th)
    for r in range(len(ns)):
        twins[1].replica(r).step(60, 0.005, th[r])
    for r in range(len(ns)):
        pa, va, ia = twins[0].replica(r).get_state()
        pb, vb, ib = twins[1].replica(r).get_state()
        assert np.array_equal(pa, pb) and np.array_equal(va, vb) and np.array_equal(ia, ib), r
        assert np.isfinite(twins[0].replica(r).observe(bbmd.OBS_ENERGY)["pe"])
    for b in twins:
        b.close()


def test_batch_argument_errors():
    ms, temps = [8, 9], [1.0, 1.5]
    ns, boxes, pos, vel, sp = lattice_replicas(ms, temps)
    b = bbmd.Batch(bbmd.ka_params(), ns, boxes, sp, pos, vel)
    with pytest.raises(bbmd.BBMDError):  # mixed thermostat kinds
        b.step(5, 0.005, [(bbmd.THERMO_NH, 1.0, 1.0, 0.5), (bbmd.THERMO_NVE, 0, 0, 0)])
    with pytest.raises(ValueError):  # one thermostat per replica
        b.step(5, 0.005, [(bbmd.THERMO_NH, 1.0, 1.0, 0.5)])
    b.step(5, 0.005)  # NVE for all
    assert b.replica(1).observe(0)["step"] == 5
    with pytest.raises(bbmd.BBMDError):
        b.set_branches(0)
    with pytest.raises(bbmd.BBMDError):
        b.set_mode(7)
    b.close()
    # the persistent step needs mixed precision: asked for with the FP64 form, it is refused
    b = bbmd.Batch(bbmd.ka_params(precision=bbmd.PREC_FP64), ns, boxes, sp, pos, vel)
    b.set_mode(bbmd.BATCH_PERSISTENT)
    assert not b.uses_persistent()
    with pytest.raises(bbmd.BBMDError) as e:
        b.step(2, 0.005)
    assert e.value.code == 8  # BBMD_ERR_STATE
    b.set_mode(bbmd.BATCH_AUTO)
    b.step(2, 0.005)
    b.close()
    with pytest.raises(bbmd.BBMDError):  # a replica whose box holds fewer than 3 cells
        bbmd.Batch(bbmd.ka_params(), [4000, 500], [gen.box_for(4000, 1.2), gen.box_for(500, 1.2)],
                   [np.zeros(4000, np.uint8), np.zeros(500, np.uint8)])


def test_persistent_wait_that_runs_out_reports_timeout():
    """Failure detection without a GPU fault.  With a dependency-wait limit of 1 ns, the
    first wait of the persistent step that is not met at once gives up: the launch aborts,
    every replica reports BBMD_ERR_TIMEOUT at its next synchronising call, and the device
    stays usable (a new batch then steps like the oracle)."""
    ms, temps = [8, 9, 10, 11], [0.5, 1.0, 1.5, 2.0]
    ns, boxes, pos, vel, sp = lattice_replicas(ms, temps)
    p = bbmd.ka_params()
    th = [(bbmd.THERMO_NH, T, T, 0.5) for T in temps]
    b = bbmd.Batch(p, ns, boxes, sp, pos, vel)
    assert b.uses_persistent()
    with pytest.raises(bbmd.BBMDError) as e:
        b.set_wait_limit(0)
    assert e.value.code == 1  # BBMD_ERR_ARG
    b.set_wait_limit(1)
    b.step(20, 0.005, th)  # asynchronous: the status is read by the next synchronising call
    for r in range(len(ns)):
        with pytest.raises(bbmd.BBMDError) as e:
            b.replica(r).observe(0)
        assert e.value.code == 7, r  # BBMD_ERR_TIMEOUT
    b.close()
    b = bbmd.Batch(p, ns, boxes, sp, pos, vel)
    assert b.uses_persistent()
    b.step(20, 0.005, th)
    for r in range(len(ns)):
        xq, _, _ = quantized(pos[r], boxes[r])
        st = oracle.MDState(xq, vel[r], sp[r], boxes[r], oracle_params(p))
        oracle.md_run(st, 20, 0.005, thermo=th[r][1:], use_cells=True)
        gp, _, _ = b.replica(r).get_state()
        assert min_image_rms(gp, st.pos, boxes[r]) <= 1e-4, r
        assert b.replica(r).observe(0)["step"] == 20
    b.close()
