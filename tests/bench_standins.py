"""bench.py run end to end on the CPU with stand-ins for the CUDA pieces of torch (events,
streams, pinned memory) and for the library handle: no kernel runs, so the numbers are
meaningless, but every leg of the bench goes through its host code and the JSON line is
printed.  Run as a script by tests/test_bench_host.py (it patches torch in-process)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_1105_5613_gb300 import bbmd, build  # noqa: E402


class StandinEvent:
    """CUDA event: every record advances a clock by 1 ms."""

    clock = 0.0

    def __init__(self, enable_timing=True):
        self.t = 0.0

    def record(self, stream=None):
        StandinEvent.clock += 1.0
        self.t = StandinEvent.clock

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return other.t - self.t


class StandinStream:
    cuda_stream = 0

    def synchronize(self):
        pass


class StandinSim:
    """The calls bench.py makes of a library handle, with their argument checks."""

    def __init__(self, p, n, L, sp, pos, vel, T0=1.0, seed=0, stream=None,
                 use_torch_allocator=False):
        assert isinstance(p, bbmd.bbmd_params)
        self.n = n
        self.steps = 0
        self.pos = np.zeros((n, 3))
        self.vel = np.zeros((n, 3))
        self.img = np.zeros((n, 3), np.int32)

    def step(self, nsteps, dt, thermostat=None):
        assert thermostat is None or (len(thermostat) == 4 and thermostat[0] in (0, 1))
        self.steps += nsteps

    def tune(self):
        pass

    def rebuild(self):
        pass

    def minimize(self, nsteps, hmax=1e-3, dmax=0.05):
        pass

    def step_profiled(self, nsteps, dt, thermostat=None):
        return {q: 0.1 * nsteps for q in bbmd.PHASES}, 1

    def info(self):
        return {"block_z": 4, "device_bytes": 123 * self.n, "shape_force_ms": [0.4, 0.3, 0.2, 0.0],
                "shape_list_ms": [1.0, 0.9, 0.8, 0.0]}

    def observe(self, mask, nbins=500, rmax=5.0, k=7.25):
        return {"temperature": 1.0, "pe": -5.0 * self.n, "ke": 1.5 * self.n, "xi": 0.0,
                "step": self.steps, "n_rebuilds": self.steps // 5}

    def get_state(self, out=None):
        if out is None:
            return self.pos.copy(), self.vel.copy(), self.img.copy()
        for o, a in zip(out, (self.pos, self.vel, self.img)):
            o[...] = a
        return out

    def set_state(self, pos, vel, image=None):
        assert pos.shape == (self.n, 3) and vel.shape == (self.n, 3)

    def close(self):
        pass


class StandinBatch:
    def __init__(self, p, ns, boxes, sp, pos, vel, T0=None, seed=0, stream=None):
        self.rep = [StandinSim(p, n, L, s, q, None) for n, L, s, q in zip(ns, boxes, sp, pos)]

    def replica(self, r):
        return self.rep[r]

    def step(self, nsteps, dt, thermostats):
        assert len(thermostats) == len(self.rep)

    def set_branches(self, branches):
        pass

    def uses_persistent(self):
        return True

    def close(self):
        pass


def main():
    build.build = lambda *a, **k: None
    bbmd.load = lambda *a, **k: None
    bbmd.Sim = StandinSim
    bbmd.Batch = StandinBatch
    bbmd.fma_peak = lambda precision=0: (80.0 if precision == 0 else 1.2, 152)
    bbmd.smem_scatter_rate = lambda kind: 1e12
    torch.cuda.Event = StandinEvent
    torch.cuda.Stream = StandinStream
    torch.cuda.synchronize = lambda *a, **k: None
    torch.cuda.current_device = lambda: 0
    torch.cuda.get_device_properties = lambda dev: type("Props", (), {"multi_processor_count": 152})
    torch.cuda.empty_cache = lambda: None
    empty = torch.empty
    torch.empty = lambda *a, **k: empty(*a, **{key: v for key, v in k.items()
                                               if key != "pin_memory"})
    import bench

    sys.argv = ["bench.py", "--ncell", "4", "--equil", "2", "--steps", "3", "--warmup", "3",
                "--e2e-steps", "2", "--replicas", "3", "--replica-steps", "2",
                "--large-steps", "1", "--large-fp64-steps", "1", "--large-ncell", "4",
                "--soft-steps", "2", "--cpu-seconds", "1"]
    bench.main()


if __name__ == "__main__":
    main()
