"""bbmd_gr_counts_noalloc (the g(r) pair counts without device allocation) against
bbmd_observe(BBMD_OBS_GR): identical integer counts on two calls in a row, on both search
paths; no device memory taken by the call; oversize systems rejected with a message.

Kept in a file of its own, collected after the other GPU tests, so that it is exercised both
in a fresh process and after everything else has run in the same process."""
import numpy as np
import pytest

from helpers import mixture
from paper_1105_5613_gb300 import bbmd

pytestmark = pytest.mark.gpu


def _sim(ncell, shake, steps=20, torch_alloc=False):
    n, L, pos, vel, sp = mixture(ncell, shake=shake)
    sim = bbmd.Sim(bbmd.ka_params(), n, L, sp, pos, vel, use_torch_allocator=torch_alloc)
    if steps:
        sim.step(steps, 0.005)
    return sim


# ncell 12, rmax 5: coarse-grid path (3 cells per axis); ncell 10: all-pairs path (2 cells);
# ncell 16, rmax 4, 300 bins: coarse grid with other bin settings
@pytest.mark.parametrize("ncell,nbins,rmax", [(12, 500, 5.0), (10, 500, 5.0), (16, 300, 4.0)])
def test_noalloc_counts_equal_observe(ncell, nbins, rmax):
    sim = _sim(ncell, 0.05)
    first = sim.gr_counts_noalloc(nbins, rmax)
    second = sim.gr_counts_noalloc(nbins, rmax)
    ref = sim.observe(bbmd.OBS_GR, nbins=nbins, rmax=rmax)["gr_counts"]
    sim.close()
    assert ref.sum() > 0
    assert np.array_equal(first, ref)
    assert np.array_equal(second, ref)


def test_noalloc_after_observe_and_steps():
    sim = _sim(12, 0.05)
    ref0 = sim.observe(bbmd.OBS_GR)["gr_counts"]
    assert np.array_equal(sim.gr_counts_noalloc(), ref0)
    sim.step(30, 0.005)
    ref1 = sim.observe(bbmd.OBS_GR)["gr_counts"]
    got = sim.gr_counts_noalloc()
    sim.close()
    assert not np.array_equal(ref0, ref1)
    assert np.array_equal(got, ref1)


def test_noalloc_takes_no_device_memory():
    torch = pytest.importorskip("torch")
    sim = _sim(12, 0.05, torch_alloc=True)
    sim.gr_counts_noalloc()  # first call on the device: address look-up, kernels loaded
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    torch0 = torch.cuda.memory_allocated()
    held0 = sim.info()["device_bytes"]
    counts = sim.gr_counts_noalloc()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    torch1 = torch.cuda.memory_allocated()
    held1 = sim.info()["device_bytes"]
    sim.close()
    assert counts.sum() > 0
    assert (free1, torch1, held1) == (free0, torch0, held0)


def test_noalloc_rejects_oversize():
    # n = 4 * 82^3: 2n alone exceeds the 2^22 fixed scratch entries
    sim = _sim(82, 0.0, steps=0)
    with pytest.raises(bbmd.BBMDError) as e:
        sim.gr_counts_noalloc()
    assert e.value.code == 1  # BBMD_ERR_ARG
    assert "scratch" in str(e.value)
    # the handle stays usable
    sim.step(2, 0.005)
    assert np.isfinite(sim.observe(bbmd.OBS_ENERGY)["pe"])
    sim.close()


def test_calls_use_the_handles_device():
    """A handle works on the device it was created on, whatever device the caller has
    current, and the caller's device is current again after the call.  Needs two GPUs."""
    torch = pytest.importorskip("torch")
    if torch.cuda.device_count() < 2:
        pytest.skip("a single device: nothing to switch to")
    with torch.cuda.device(0):
        sim = _sim(12, 0.05)
        ref = sim.observe(bbmd.OBS_GR)["gr_counts"]
    with torch.cuda.device(1):
        got = sim.gr_counts_noalloc()
        again = sim.observe(bbmd.OBS_GR)["gr_counts"]
        assert torch.cuda.current_device() == 1
    sim.close()
    assert np.array_equal(got, ref) and np.array_equal(again, ref)
